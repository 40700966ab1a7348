// Stream-collide kernel instances for D3Q27 with F16 storage.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_INSTANCE(Fclb, __half, d3q27_f16)
}  // namespace lbm
