// Stream-collide kernel instances for D3Q27 with F64 storage.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_INSTANCE(Fclb, double, d3q27_f64)
}  // namespace lbm
