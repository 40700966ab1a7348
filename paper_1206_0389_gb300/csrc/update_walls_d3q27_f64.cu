// Stream-collide kernel instances for D3Q27 with F64 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(Fclb, double, d3q27_f64)
}  // namespace lbm
