// Stream-collide kernel instances for D3Q19 with F16 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(MrtLes, __half, d3q19_f16)
}  // namespace lbm
