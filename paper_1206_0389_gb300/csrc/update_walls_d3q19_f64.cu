// Stream-collide kernel instances for D3Q19 with F64 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(MrtLes, double, d3q19_f64)
}  // namespace lbm
