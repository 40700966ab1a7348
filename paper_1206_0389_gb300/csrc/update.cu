// Dispatch of the fused stream-collide kernel (update.cuh) over model and
// storage and walls; each (model, storage) pair is compiled in its own
// translation units (update_<model>_<storage>.cu, update_walls_<model>_<storage>.cu)
// so the build runs in parallel.
#include "update.cuh"

namespace lbm {

cudaError_t launch_update(int model, int storage, const UpdateArgs& a, int threads, int minb, int ctas,
                          cudaStream_t st) {
  const bool w = a.walls != 0;
  if (model == LBM_D3Q19_MRT_LES) {
    if (storage == LBM_F64)
      return w ? launch_update_walls_d3q19_f64(a, threads, minb, ctas, st) : launch_update_d3q19_f64(a, threads, minb, ctas, st);
    if (storage == LBM_F32)
      return w ? launch_update_walls_d3q19_f32(a, threads, minb, ctas, st) : launch_update_d3q19_f32(a, threads, minb, ctas, st);
    return w ? launch_update_walls_d3q19_f16(a, threads, minb, ctas, st) : launch_update_d3q19_f16(a, threads, minb, ctas, st);
  }
  if (storage == LBM_F64)
    return w ? launch_update_walls_d3q27_f64(a, threads, minb, ctas, st) : launch_update_d3q27_f64(a, threads, minb, ctas, st);
  if (storage == LBM_F32)
    return w ? launch_update_walls_d3q27_f32(a, threads, minb, ctas, st) : launch_update_d3q27_f32(a, threads, minb, ctas, st);
  return w ? launch_update_walls_d3q27_f16(a, threads, minb, ctas, st) : launch_update_d3q27_f16(a, threads, minb, ctas, st);
}

cudaError_t update_occupancy(int model, int storage, bool walls, int threads, int minb, int* n) {
  if (model == LBM_D3Q19_MRT_LES) {
    if (storage == LBM_F64)
      return walls ? occupancy_update_walls_d3q19_f64(threads, minb, n) : occupancy_update_d3q19_f64(threads, minb, n);
    if (storage == LBM_F32)
      return walls ? occupancy_update_walls_d3q19_f32(threads, minb, n) : occupancy_update_d3q19_f32(threads, minb, n);
    return walls ? occupancy_update_walls_d3q19_f16(threads, minb, n) : occupancy_update_d3q19_f16(threads, minb, n);
  }
  if (storage == LBM_F64)
    return walls ? occupancy_update_walls_d3q27_f64(threads, minb, n) : occupancy_update_d3q27_f64(threads, minb, n);
  if (storage == LBM_F32)
    return walls ? occupancy_update_walls_d3q27_f32(threads, minb, n) : occupancy_update_d3q27_f32(threads, minb, n);
  return walls ? occupancy_update_walls_d3q27_f16(threads, minb, n) : occupancy_update_d3q27_f16(threads, minb, n);
}

}  // namespace lbm
