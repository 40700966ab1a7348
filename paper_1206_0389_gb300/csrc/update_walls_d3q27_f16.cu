// Stream-collide kernel instances for D3Q27 with F16 storage and y/z walls.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_WALL_INSTANCE(Fclb, __half, d3q27_f16)
}  // namespace lbm
