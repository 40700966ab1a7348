// Stream-collide kernel instances for D3Q19 with F32 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(MrtLes, float, d3q19_f32)
}  // namespace lbm
