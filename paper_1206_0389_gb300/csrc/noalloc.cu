// Mass/momentum audit that allocates nothing (lbm_mass_momentum_noalloc).
//
// Some callers cannot let a library call cudaMalloc: code that runs while a
// CUDA graph is being captured (allocation is not capturable), frameworks
// that own all device memory through their own caching pool (a raw
// cudaMalloc bypasses the pool and may synchronise the device), and
// time-critical loops that must not stall on an allocation.  This entry
// point serves them: the caller passes the distributions and the 4-double
// result buffer, both in device memory it already owns, and the partial sums
// live in a file-scope device array of fixed size instead of allocated
// scratch.
//
// The array is LBM_NOALLOC_MAX_BLOCKS * 4 doubles (2 MiB); every GPU that
// loads this library holds it until the process exits.  Every call shares
// it and it keeps the previous call's contents; each call overwrites the
// slots it reads, so nothing needs clearing, but two calls that overlap on
// the same GPU (different streams or threads) race on it.  A call looks up
// the array's device address on the current device (cudaGetSymbolAddress)
// whenever its stream is not capturing, and remembers it per device; a call
// made while its stream is being captured uses the remembered address, so
// the first call on a device must come before any stream capture (and, after
// a cudaDeviceReset, the first call again).
#include <mutex>

#include "collide.cuh"
#include "kernels.cuh"

namespace lbm {

static __device__ __align__(256) double g_noalloc_partials[LBM_NOALLOC_MAX_BLOCKS * 4];

namespace {

constexpr int kMaxDevices = 64;
double* g_scratch[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// device address of the static array on the current device: looked up
// again on every call outside stream capture (so a device reset, which
// moves the array, is picked up), the remembered one under capture
cudaError_t scratch_on_current_device(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cs);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    double* p = nullptr;
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partials);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = p;
  } else if (g_scratch[dev] == nullptr) {
    return cudaErrorStreamCaptureUnsupported;
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

// One CTA per 8^3 block: float64 sums (delta rho, j_x, j_y, j_z) of its 512
// cells into the block's slot of the static array.
template <class M, class S>
__global__ void __launch_bounds__(256) k_block_sums(const S* __restrict__ f, double* __restrict__ part) {
  constexpr int Q = M::Q;
  double s[4] = {0, 0, 0, 0};
  const S* fb = f + int64_t(blockIdx.x) * Q * kCells;
  for (int c = threadIdx.x; c < kCells; c += blockDim.x) {
    static_for<Q>([&](auto i) {
      const double g = double(Store<S>::template get<Q, i>(fb + int(i) * kCells + c));
      // zero velocity components are skipped at compile time (IEEE rules
      // keep 0.0 * g as a float64 operation otherwise)
      s[0] += g;
      if constexpr (Lattice<Q>::ex(i) != 0) s[1] += Lattice<Q>::ex(i) > 0 ? g : -g;
      if constexpr (Lattice<Q>::ey(i) != 0) s[2] += Lattice<Q>::ey(i) > 0 ? g : -g;
      if constexpr (Lattice<Q>::ez(i) != 0) s[3] += Lattice<Q>::ez(i) > 0 ? g : -g;
    });
  }
  __shared__ double sh[4][8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
    part[int64_t(blockIdx.x) * 4 + threadIdx.x] = v;
  }
}

// Fixed-order sum of the n block slots into out[4].
__global__ void __launch_bounds__(256) k_sum_slots(const double* __restrict__ part, int n, double* out) {
  __shared__ double sh[4][256];
  double s[4] = {0, 0, 0, 0};
  for (int b = threadIdx.x; b < n; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += part[int64_t(b) * 4 + k];
#pragma unroll
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = s[k];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sh[threadIdx.x][0];
}

template <class M, class S>
cudaError_t sums_ms(const void* f, int nblocks, double* part, double* out, cudaStream_t st) {
  k_block_sums<M, S><<<nblocks, 256, 0, st>>>(reinterpret_cast<const S*>(f), part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum_slots<<<1, 256, 0, st>>>(part, nblocks, out);
  return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_mass_momentum_noalloc(int model, int storage, const void* f, int64_t nblocks,
                                         double* out, void* cuda_stream) {
  using namespace lbm;
  if (model != LBM_D3Q19_MRT_LES && model != LBM_D3Q27_FCLB) return LBM_ERR_ARG;
  if (storage != LBM_F64 && storage != LBM_F32 && storage != LBM_F16) return LBM_ERR_ARG;
  if (f == nullptr || out == nullptr || nblocks < 1) return LBM_ERR_ARG;
  if (nblocks > LBM_NOALLOC_MAX_BLOCKS) return LBM_ERR_ARG;  // beyond the static scratch
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  double* part = nullptr;
  if (scratch_on_current_device(st, &part) != cudaSuccess) return LBM_ERR_CUDA;
  const int nb = int(nblocks);
  cudaError_t e;
  if (model == LBM_D3Q19_MRT_LES) {
    e = storage == LBM_F64   ? sums_ms<MrtLes, double>(f, nb, part, out, st)
        : storage == LBM_F32 ? sums_ms<MrtLes, float>(f, nb, part, out, st)
                             : sums_ms<MrtLes, __half>(f, nb, part, out, st);
  } else {
    e = storage == LBM_F64   ? sums_ms<Fclb, double>(f, nb, part, out, st)
        : storage == LBM_F32 ? sums_ms<Fclb, float>(f, nb, part, out, st)
                             : sums_ms<Fclb, __half>(f, nb, part, out, st);
  }
  return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}
