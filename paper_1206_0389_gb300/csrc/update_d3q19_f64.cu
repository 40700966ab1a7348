// Stream-collide kernel instances for D3Q19 with F64 storage.
#include "update.cuh"

namespace lbm {
LBM_UPDATE_INSTANCE(MrtLes, double, d3q19_f64)
}  // namespace lbm
