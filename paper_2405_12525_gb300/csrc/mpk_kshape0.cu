// The persistent level-blocked kernel k_mpk instantiated for block shape 0 (kShapes[0]).
#include "mpk_kernel_dev.cuh"

namespace mpk {
void *select_mpk_shape0(int mode, int m, bool trace, int vtype, bool a32) {
    return select_mpk_shape<0>(mode, m, trace, vtype, a32);
}
}  // namespace mpk
