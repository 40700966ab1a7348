// Stream-collide kernel instances for D3Q19 with F32 storage.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_INSTANCE(MrtLes, float, d3q19_f32)
}  // namespace lbm
