// The persistent level-blocked kernel k_mpk instantiated for block shape 4 (kShapes[4]: two
// 32-row slices a compute warp per unit).
#include "mpk_kernel_dev.cuh"

namespace mpk {
void *select_mpk_shape4(int mode, int m, bool trace, int vtype, bool a32) {
    return select_mpk_shape<4>(mode, m, trace, vtype, a32);
}
}  // namespace mpk
