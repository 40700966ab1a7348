// Stream-collide kernel instances for D3Q19 with F16 storage.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_INSTANCE(MrtLes, __half, d3q19_f16)
}  // namespace lbm
