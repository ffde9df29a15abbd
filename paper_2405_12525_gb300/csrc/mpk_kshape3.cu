// The persistent level-blocked kernel k_mpk instantiated for block shape 3 (kShapes[3], input rows staged).
#include "mpk_kernel_dev.cuh"

namespace mpk {
void *select_mpk_shape3(int mode, int m, bool trace, int vtype, bool a32) {
    return select_mpk_shape<3>(mode, m, trace, vtype, a32);
}
}  // namespace mpk
