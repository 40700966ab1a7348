// Stream-collide kernel instances for D3Q27 with F32 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(Fclb, float, d3q27_f32)
}  // namespace lbm
