// The persistent level-blocked kernel k_mpk instantiated for block shape 2 (kShapes[2]).
#include "mpk_kernel_dev.cuh"

namespace mpk {
void *select_mpk_shape2(int mode, int m, bool trace, int vtype, bool a32) {
    return select_mpk_shape<2>(mode, m, trace, vtype, a32);
}
}  // namespace mpk
