// The persistent level-blocked kernel k_mpk instantiated for block shape 1 (kShapes[1]).
#include "mpk_kernel_dev.cuh"

namespace mpk {
void *select_mpk_shape1(int mode, int m, bool trace, int vtype, bool a32) {
    return select_mpk_shape<1>(mode, m, trace, vtype, a32);
}
}  // namespace mpk
