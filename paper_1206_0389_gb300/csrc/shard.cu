// Block sharding of the grid (lbm_shard_*): the level-0 block columns along
// x are cut into parts of balanced work, each part an ordinary context over
// its slab with one halo block column beyond each cut; before every coarse
// step each cut exchanges, in both directions, the populations of the
// boundary cell layer that cross it.  The paper partitions its blocks over
// MPI processes with a halo exchange of the populations leaving each
// partition (Sections 1 and 3.2); here the parts live on one device and the
// exchange is pack -> device-to-device copy -> unpack, the sequence a
// multi-GPU build would run with peer copies into the receiving GPU's own
// memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "lattice.cuh"
#include "plan.h"

int create_context(lbm_ctx** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
                   double cs, void* cuda_stream, const lbm::PlanOptions& opt);

namespace lbm {
void set_create_error(const std::string& m);  // the message lbm_create_error() returns
const GridPlan& ctx_plan(const lbm_ctx* c);
void* ctx_level0_buffer(lbm_ctx* c);
cudaStream_t ctx_stream(const lbm_ctx* c);

namespace {

// populations crossing a cut: e_x = dir (at most 9)
struct Pops {
  int n;
  int i[9];
};
Pops crossing(int Q, int dir) {
  Pops p{};
  for (int i = 0; i < Q; ++i)
    if (ex27(i) == dir) p.i[p.n++] = i;
  return p;
}

// One value per thread: t = ((k * BZ + bz) * BY + by) * 64 + cy + 8 cz, k the
// index into the crossing populations; the box column bx, cell layer x = lx.
template <class E>
__global__ void k_halo_pack(const E* __restrict__ box, int Q, int BX, int BY, int BZ, int bx, int lx, Pops p,
                            E* __restrict__ buf) {
  const int64_t n = int64_t(p.n) * BY * BZ * 64;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = int(t & 63);
  const int64_t r = t >> 6;
  const int by = int(r % BY), bz = int((r / BY) % BZ), k = int(r / (int64_t(BY) * BZ));
  int q = p.i[0];
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (j == k) q = p.i[j];
  const int64_t b = bx + int64_t(BX) * (by + int64_t(BY) * bz);
  buf[t] = box[(b * Q + q) * kCells + lx + 8 * (c & 7) + 64 * (c >> 3)];
}
template <class E>
__global__ void k_halo_unpack(E* __restrict__ box, int Q, int BX, int BY, int BZ, int bx, int lx, Pops p,
                              const E* __restrict__ buf) {
  const int64_t n = int64_t(p.n) * BY * BZ * 64;
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int c = int(t & 63);
  const int64_t r = t >> 6;
  const int by = int(r % BY), bz = int((r / BY) % BZ), k = int(r / (int64_t(BY) * BZ));
  int q = p.i[0];
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (j == k) q = p.i[j];
  const int64_t b = bx + int64_t(BX) * (by + int64_t(BY) * bz);
  box[(b * Q + q) * kCells + lx + 8 * (c & 7) + 64 * (c >> 3)] = buf[t];
}

template <class E>
cudaError_t halo_move(bool pack, void* box, int Q, int BX, int BY, int BZ, int bx, int lx, const Pops& p, void* buf,
                      cudaStream_t st) {
  const int64_t n = int64_t(p.n) * BY * BZ * 64;
  const unsigned grid = unsigned((n + 255) / 256);
  if (pack)
    k_halo_pack<E><<<grid, 256, 0, st>>>(static_cast<const E*>(box), Q, BX, BY, BZ, bx, lx, p, static_cast<E*>(buf));
  else
    k_halo_unpack<E><<<grid, 256, 0, st>>>(static_cast<E*>(box), Q, BX, BY, BZ, bx, lx, p, static_cast<const E*>(buf));
  return cudaGetLastError();
}

cudaError_t halo_launch(bool pack, int storage, void* box, int Q, int BX, int BY, int BZ, int bx, int lx,
                        const Pops& p, void* buf, cudaStream_t st) {
  if (storage == LBM_F64) return halo_move<double>(pack, box, Q, BX, BY, BZ, bx, lx, p, buf, st);
  if (storage == LBM_F32) return halo_move<float>(pack, box, Q, BX, BY, BZ, bx, lx, p, buf, st);
  return halo_move<unsigned short>(pack, box, Q, BX, BY, BZ, bx, lx, p, buf, st);
}

// work of every level-0 block column: cells times substeps of all levels
// above it (level-l blocks under the column, 2^l substeps, 512 cells each)
std::vector<double> column_work(const lbm_grid& g) {
  std::vector<double> w(g.nbx, 0.0);
  std::vector<uint8_t> region(size_t(g.nbx) * g.nby * g.nbz, 1);
  int64_t off = 0;
  for (int l = 0; l < g.levels; ++l) {
    const int nx = g.nbx << l, ny = g.nby << l, nz = g.nbz << l;
    for (int bz = 0; bz < nz; ++bz)
      for (int by = 0; by < ny; ++by)
        for (int bx = 0; bx < nx; ++bx)
          if (region[bx + size_t(nx) * (by + size_t(ny) * bz)]) w[bx >> l] += std::ldexp(1.0, l);
    if (l + 1 == g.levels) break;
    std::vector<uint8_t> next(size_t(2 * nx) * 2 * ny * 2 * nz, 0);
    for (int bz = 0; bz < nz; ++bz)
      for (int by = 0; by < ny; ++by)
        for (int bx = 0; bx < nx; ++bx)
          if (g.refine[off + bx + int64_t(nx) * (by + int64_t(ny) * bz)])
            for (int k = 0; k < 8; ++k)
              next[(2 * bx + (k & 1)) + size_t(2 * nx) * ((2 * by + ((k >> 1) & 1)) + size_t(2 * ny) * (2 * bz + (k >> 2)))] = 1;
    off += int64_t(nx) * ny * nz;
    region.swap(next);
  }
  return w;
}

// level-0 columns no cut may come near: those holding a refined block, and
// those under the nozzle with a margin of 16 coarse cells
std::vector<uint8_t> refined_columns(const lbm_grid& g) {
  std::vector<uint8_t> r(g.nbx, 0);
  if (g.levels >= 2)
    for (int bz = 0; bz < g.nbz; ++bz)
      for (int by = 0; by < g.nby; ++by)
        for (int bx = 0; bx < g.nbx; ++bx)
          if (g.refine[bx + int64_t(g.nbx) * (by + int64_t(g.nby) * bz)]) r[bx] = 1;
  if (g.nozzle_r > 0) {
    const int a = std::max(0, int(std::floor((g.nozzle_x0 - 16.0) / 8.0)));
    const int b = std::min(g.nbx - 1, int(std::floor((g.nozzle_x1 + 16.0) / 8.0)));
    for (int bx = a; bx <= b; ++bx) r[bx] = 1;
  }
  return r;
}

// cuts[0] = 0 < cuts[1] < ... < cuts[P] = nbx: part p owns columns
// [cuts[p], cuts[p+1]).  A cut c (between columns c-1 and c) is allowed when
// columns c-2 .. c+1 hold no refined block and lie clear of the nozzle
// (wrapping for a periodic x; the
// periodic wrap itself is a cut between column nbx-1 and 0).  Greedy: each
// cut at the allowed position whose work prefix is nearest an even split of
// the work left to the remaining parts (a refined region that cannot be cut
// stays whole in one part, and the rest is shared evenly).
std::string choose_cuts(const lbm_grid& g, int P, std::vector<int>& cuts) {
  const int n = g.nbx;
  if (P < 1) return "nparts must be >= 1";
  if (P > n) return "more parts than level-0 block columns";
  const std::vector<uint8_t> rc = refined_columns(g);
  auto col = [&](int c) { return g.periodic_x ? ((c % n) + n) % n : c; };
  auto refined_near = [&](int c) {
    for (int k = c - 2; k <= c + 1; ++k) {
      const int j = col(k);
      if (j >= 0 && j < n && rc[j]) return true;
    }
    return false;
  };
  if (P > 1 && g.periodic_x && refined_near(0)) return "refinement within a block of the periodic x wrap";
  const std::vector<double> w = column_work(g);
  std::vector<double> pre(n + 1, 0.0);
  for (int c = 0; c < n; ++c) pre[c + 1] = pre[c] + w[c];
  cuts.assign(1, 0);
  for (int k = 1; k < P; ++k) {
    const int last = cuts.back();
    const double target = pre[last] + (pre[n] - pre[last]) / double(P - k + 1);
    int best = -1;
    for (int c = cuts.back() + 1; c <= n - (P - k); ++c) {
      if (refined_near(c)) continue;
      if (best < 0 || std::fabs(pre[c] - target) < std::fabs(pre[best] - target)) best = c;
    }
    if (best < 0) return "no cut between parts keeps clear of the refined blocks";
    cuts.push_back(best);
  }
  cuts.push_back(n);
  return "";
}

}  // namespace
}  // namespace lbm

using namespace lbm;

struct lbm_shard {
  int P = 0, model = 0, storage = 0, Q = 19, levels = 1;
  lbm_grid g{};
  std::vector<uint8_t> refine;
  std::vector<int> cuts;
  std::vector<lbm_ctx*> parts;
  std::vector<std::vector<uint8_t>> part_refine;
  std::vector<int> part_levels;  // levels of each part (finer levels only where its slab refines)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // each part steps on a stream of its own (the stand-in for a GPU of its
  // own), joined to `stream` around the halo exchange by events
  std::vector<cudaStream_t> pstream;
  std::vector<cudaEvent_t> pevent;
  cudaEvent_t exchanged = nullptr;
  // one stream per cut and direction: the exchanges of different cuts and
  // directions touch different layers and run side by side
  std::vector<cudaStream_t> xstream;
  std::vector<cudaEvent_t> xevent;
  Pops plus{}, minus{};
  // one cut: left part L, right part R (R = 0 for the periodic wrap); buffers
  // for L -> R (e_x = +1 values of L's last layer) and R -> L (e_x = -1 of
  // R's first layer), a send buffer on the sender and a receive buffer on
  // the receiver
  struct Cut {
    int L, R;
    void *send_lr = nullptr, *recv_lr = nullptr, *send_rl = nullptr, *recv_rl = nullptr;
  };
  std::vector<Cut> cut;
  size_t face_bytes_plus = 0, face_bytes_minus = 0;
  std::string err;
};

namespace {

int sfail(lbm_shard* s, int code, const std::string& m) {
  if (s) s->err = m;
  return code;
}

void shard_free(lbm_shard* s) {
  for (auto& c : s->cut) {
    cudaFree(c.send_lr);
    cudaFree(c.recv_lr);
    cudaFree(c.send_rl);
    cudaFree(c.recv_rl);
  }
  for (lbm_ctx* p : s->parts) lbm_destroy(p);
  for (cudaEvent_t e : s->pevent) cudaEventDestroy(e);
  for (cudaStream_t t : s->pstream) cudaStreamDestroy(t);
  for (cudaEvent_t e : s->xevent) cudaEventDestroy(e);
  for (cudaStream_t t : s->xstream) cudaStreamDestroy(t);
  if (s->exchanged) cudaEventDestroy(s->exchanged);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

// the refine flags of columns [c0, c1) of every level
std::vector<uint8_t> slice_refine(const lbm_grid& g, int c0, int c1) {
  std::vector<uint8_t> out;
  int64_t off = 0;
  for (int l = 0; l + 1 < g.levels; ++l) {
    const int nx = g.nbx << l, ny = g.nby << l, nz = g.nbz << l;
    const int x0 = c0 << l, x1 = c1 << l;
    for (int bz = 0; bz < nz; ++bz)
      for (int by = 0; by < ny; ++by)
        for (int bx = x0; bx < x1; ++bx) out.push_back(g.refine[off + bx + int64_t(nx) * (by + int64_t(ny) * bz)]);
    off += int64_t(nx) * ny * nz;
  }
  return out;
}

// level-0 box column of the part's level-0 column c (c = -1: low halo,
// c = nbx: high halo)
int box_col(const lbm_ctx* part, int c) { return c - ctx_plan(part).lv[0].ox; }

// The halo exchange of every cut, both directions, after all work queued on
// `stream`: each direction (pack on the sender, device-to-device copy,
// unpack into the receiver's halo) on a stream of its own; `exchanged` is
// recorded on `stream` once all of them are done.
int exchange(lbm_shard* s) {
  cudaError_t e = cudaEventRecord(s->exchanged, s->stream);
  for (size_t k = 0; k < s->cut.size() && e == cudaSuccess; ++k) {
    const auto& c = s->cut[k];
    lbm_ctx *L = s->parts[c.L], *R = s->parts[c.R];
    const LevelPlan &pl = ctx_plan(L).lv[0], &pr = ctx_plan(R).lv[0];
    const int nl = pl.nbx;
    cudaStream_t lr = s->xstream[2 * k], rl = s->xstream[2 * k + 1];
    if ((e = cudaStreamWaitEvent(lr, s->exchanged, 0)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(rl, s->exchanged, 0)) != cudaSuccess)
      break;
    // L's last layer x = 7 of column nl - 1, e_x = +1 -> R's low halo (column -1, layer 7)
    if ((e = halo_launch(true, s->storage, ctx_level0_buffer(L), s->Q, pl.BX, pl.BY, pl.BZ, box_col(L, nl - 1), 7,
                         s->plus, c.send_lr, lr)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c.recv_lr, c.send_lr, s->face_bytes_plus, cudaMemcpyDeviceToDevice, lr)) != cudaSuccess ||
        (e = halo_launch(false, s->storage, ctx_level0_buffer(R), s->Q, pr.BX, pr.BY, pr.BZ, box_col(R, -1), 7,
                         s->plus, c.recv_lr, lr)) != cudaSuccess)
      break;
    // R's first layer x = 0 of column 0, e_x = -1 -> L's high halo (column nl, layer 0)
    if ((e = halo_launch(true, s->storage, ctx_level0_buffer(R), s->Q, pr.BX, pr.BY, pr.BZ, box_col(R, 0), 0,
                         s->minus, c.send_rl, rl)) != cudaSuccess ||
        (e = cudaMemcpyAsync(c.recv_rl, c.send_rl, s->face_bytes_minus, cudaMemcpyDeviceToDevice, rl)) != cudaSuccess ||
        (e = halo_launch(false, s->storage, ctx_level0_buffer(L), s->Q, pl.BX, pl.BY, pl.BZ, box_col(L, nl), 0,
                         s->minus, c.recv_rl, rl)) != cudaSuccess)
      break;
  }
  for (size_t j = 0; j < s->xstream.size() && e == cudaSuccess; ++j)
    if ((e = cudaEventRecord(s->xevent[j], s->xstream[j])) == cudaSuccess)
      e = cudaStreamWaitEvent(s->stream, s->xevent[j], 0);
  if (e == cudaSuccess) e = cudaEventRecord(s->exchanged, s->stream);
  if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("halo exchange: ") + cudaGetErrorString(e));
  return LBM_OK;
}

// dense per-level arrays: part p's x range [x0, x0 + nxp) of the global one
void slab_copy(bool to_part, double* part, double* global, int comps, int64_t NX, int64_t NY, int64_t NZ,
               int64_t x0, int64_t nxp) {
  for (int c = 0; c < comps; ++c)
    for (int64_t z = 0; z < NZ; ++z)
      for (int64_t y = 0; y < NY; ++y) {
        double* gp = global + ((c * NZ + z) * NY + y) * NX + x0;
        double* pp = part + ((c * NZ + z) * NY + y) * nxp;
        if (to_part) std::memcpy(pp, gp, nxp * sizeof(double));
        else std::memcpy(gp, pp, nxp * sizeof(double));
      }
}

}  // namespace

extern "C" {

int lbm_shard_plan(const lbm_grid* g, int nparts, int* cuts) {
  if (!g || !cuts) return LBM_ERR_ARG;
  GridPlan P;
  if (!build_plan(*g, LBM_D3Q19_MRT_LES, LBM_F32, 1.0, P).empty()) return LBM_ERR_ARG;
  std::vector<int> c;
  if (!choose_cuts(*g, nparts, c).empty()) return LBM_ERR_ARG;
  for (int k = 0; k <= nparts; ++k) cuts[k] = c[k];
  return LBM_OK;
}

int lbm_shard_create(lbm_shard** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
                     double cs, int nparts, void* cuda_stream) {
  if (!out) return LBM_ERR_ARG;
  *out = nullptr;
  if (!g) return LBM_ERR_ARG;
  lbm_shard* s = new (std::nothrow) lbm_shard();
  if (!s) return LBM_ERR_OOM;
  auto bail = [&](int code) {
    shard_free(s);
    delete s;
    return code;
  };
  set_create_error("");
  GridPlan whole;
  std::string e = build_plan(*g, int(model), int(storage), omega, whole);
  if (e.empty()) e = choose_cuts(*g, nparts, s->cuts);
  if (e.empty() && g->nozzle_r > 0 && nparts > 1 && !(g->nozzle_x1 + 16.0 < 8.0 * s->cuts[1]))
    e = "the nozzle (with a margin of 16 coarse cells) must lie in part 0";
  if (!e.empty()) {
    set_create_error(e);
    return bail(LBM_ERR_ARG);
  }
  s->P = nparts;
  s->model = int(model);
  s->storage = int(storage);
  s->Q = whole.Q;
  s->levels = g->levels;
  s->g = *g;
  const int64_t nref = [&] {
    int64_t n = 0;
    for (int l = 0; l + 1 < g->levels; ++l) n += (int64_t(g->nbx) * g->nby * g->nbz) << (3 * l);
    return n;
  }();
  s->refine.assign(g->refine, g->refine + nref);
  s->g.refine = s->refine.data();
  if (cuda_stream) {
    s->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(LBM_ERR_CUDA);
    s->own_stream = true;
  }
  const bool px = g->periodic_x != 0;
  if (nparts > 1) {
    s->pstream.assign(nparts, nullptr);
    s->pevent.assign(nparts, nullptr);
    for (int p = 0; p < nparts; ++p)
      if (cudaStreamCreateWithFlags(&s->pstream[p], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s->pevent[p], cudaEventDisableTiming) != cudaSuccess)
        return bail(LBM_ERR_CUDA);
    if (cudaEventCreateWithFlags(&s->exchanged, cudaEventDisableTiming) != cudaSuccess) return bail(LBM_ERR_CUDA);
  }
  s->part_refine.resize(nparts);
  for (int p = 0; p < nparts; ++p) {
    const int c0 = s->cuts[p], c1 = s->cuts[p + 1];
    lbm_grid gp = *g;
    PlanOptions opt;
    if (nparts > 1) {
      gp.nbx = c1 - c0;
      gp.periodic_x = 0;
      opt.halo_lo = px || p > 0;
      opt.halo_hi = px || p < nparts - 1;
      if (opt.halo_lo) gp.walls &= ~16;
      if (opt.halo_hi) {
        gp.walls &= ~32;
        gp.outlet = 0;
      }
      s->part_refine[p] = slice_refine(*g, c0, c1);
      gp.refine = s->part_refine[p].data();
      // a part keeps the levels its own slab refines into (the flags of a
      // level come after those of the coarser levels, so a trailing run of
      // levels without flags is dropped)
      int levels = 1;
      size_t off = 0;
      for (int l = 0; l + 1 < g->levels; ++l) {
        const size_t n = size_t(c1 - c0) * g->nby * g->nbz << (3 * l);
        bool any = false;
        for (size_t k = 0; k < n && !any; ++k) any = s->part_refine[p][off + k] != 0;
        if (!any) break;
        levels = l + 2;
        off += n;
      }
      gp.levels = levels;
      if (p > 0) gp.nozzle_r = 0;
      gp.nozzle_x0 -= 8.0 * c0;
      gp.nozzle_x1 -= 8.0 * c0;
    }
    lbm_ctx* ctx = nullptr;
    const int rc = create_context(&ctx, model, storage, &gp, omega, cs, nparts > 1 ? s->pstream[p] : s->stream, opt);
    if (rc != LBM_OK) {
      set_create_error("part " + std::to_string(p) + ": " + std::string(lbm_create_error()));
      return bail(rc);
    }
    s->parts.push_back(ctx);
    s->part_levels.push_back(gp.levels);
  }
  if (nparts > 1) {
    s->plus = crossing(s->Q, +1);
    s->minus = crossing(s->Q, -1);
    const size_t sb = storage_bytes(s->storage);
    const size_t layer = size_t(g->nby) * g->nbz * 64;
    s->face_bytes_plus = size_t(s->plus.n) * layer * sb;
    s->face_bytes_minus = size_t(s->minus.n) * layer * sb;
    for (int p = 0; p + 1 < nparts; ++p) s->cut.push_back(lbm_shard::Cut{p, p + 1});
    if (px) s->cut.push_back(lbm_shard::Cut{nparts - 1, 0});
    s->xstream.assign(2 * s->cut.size(), nullptr);
    s->xevent.assign(2 * s->cut.size(), nullptr);
    for (size_t j = 0; j < s->xstream.size(); ++j)
      if (cudaStreamCreateWithFlags(&s->xstream[j], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&s->xevent[j], cudaEventDisableTiming) != cudaSuccess)
        return bail(LBM_ERR_CUDA);
    for (auto& c : s->cut)
      if (cudaMalloc(&c.send_lr, s->face_bytes_plus) != cudaSuccess ||
          cudaMalloc(&c.recv_lr, s->face_bytes_plus) != cudaSuccess ||
          cudaMalloc(&c.send_rl, s->face_bytes_minus) != cudaSuccess ||
          cudaMalloc(&c.recv_rl, s->face_bytes_minus) != cudaSuccess)
        return bail(LBM_ERR_OOM);
  }
  *out = s;
  return LBM_OK;
}

void lbm_shard_destroy(lbm_shard* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (cudaStream_t t : s->pstream) cudaStreamSynchronize(t);
  for (cudaStream_t t : s->xstream) cudaStreamSynchronize(t);
  shard_free(s);
  delete s;
}

const char* lbm_shard_last_error(const lbm_shard* s) { return s ? s->err.c_str() : "NULL shard"; }

int lbm_shard_part(lbm_shard* s, int part, lbm_ctx** ctx, int* col0, int* col1) {
  if (!s || part < 0 || part >= s->P) return LBM_ERR_ARG;
  if (ctx) *ctx = s->parts[part];
  if (col0) *col0 = s->cuts[part];
  if (col1) *col1 = s->cuts[part + 1];
  return LBM_OK;
}

int lbm_shard_halo_bytes(const lbm_shard* s, int64_t* bytes_per_coarse_step) {
  if (!s || !bytes_per_coarse_step) return LBM_ERR_ARG;
  *bytes_per_coarse_step = int64_t(s->cut.size()) * int64_t(s->face_bytes_plus + s->face_bytes_minus);
  return LBM_OK;
}

int lbm_shard_set_inflow(lbm_shard* s, double y0, double z0, double diameter, double u_in, double perturb,
                         uint64_t seed) {
  if (!s) return LBM_ERR_ARG;
  for (lbm_ctx* p : s->parts) {
    const int rc = lbm_set_inflow(p, y0, z0, diameter, u_in, perturb, seed);
    if (rc) return sfail(s, rc, lbm_last_error(p));
  }
  return LBM_OK;
}

int lbm_shard_init_equilibrium(lbm_shard* s, int level, const double* rho, const double* u) {
  if (!s) return LBM_ERR_ARG;
  if (level < 0 || level >= s->levels) return sfail(s, LBM_ERR_ARG, "level out of range");
  const int64_t NX = int64_t(8) * s->g.nbx << level, NY = int64_t(8) * s->g.nby << level,
                NZ = int64_t(8) * s->g.nbz << level;
  for (int p = 0; p < s->P; ++p) {
    const int64_t x0 = int64_t(8) * s->cuts[p] << level, nxp = int64_t(8) * (s->cuts[p + 1] - s->cuts[p]) << level;
    std::vector<double> r, v;
    if (rho) {
      r.resize(size_t(nxp * NY * NZ));
      slab_copy(true, r.data(), const_cast<double*>(rho), 1, NX, NY, NZ, x0, nxp);
    }
    if (u) {
      v.resize(size_t(3 * nxp * NY * NZ));
      slab_copy(true, v.data(), const_cast<double*>(u), 3, NX, NY, NZ, x0, nxp);
    }
    if (level >= s->part_levels[p]) continue;  // the part's slab has no cells of this level
    const int rc = lbm_init_equilibrium(s->parts[p], level, rho ? r.data() : nullptr, u ? v.data() : nullptr);
    if (rc) return sfail(s, rc, lbm_last_error(s->parts[p]));
  }
  return LBM_OK;
}

int lbm_shard_step(lbm_shard* s, int coarse_steps) {
  if (!s) return LBM_ERR_ARG;
  if (coarse_steps < 0) return sfail(s, LBM_ERR_ARG, "coarse_steps must be >= 0");
  if (s->P == 1) {
    const int rc = lbm_step(s->parts[0], coarse_steps);
    return rc ? sfail(s, rc, lbm_last_error(s->parts[0])) : LBM_OK;
  }
  // the exchange on `stream` after everything queued on the part streams
  // (it reads each part's boundary layer of the current state), then every
  // part's coarse step on its own stream after the exchange; at the end
  // `stream` waits for all parts again
  auto join_parts = [&]() -> int {
    for (int p = 0; p < s->P; ++p) {
      cudaError_t e = cudaEventRecord(s->pevent[p], s->pstream[p]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s->stream, s->pevent[p], 0);
      if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("join: ") + cudaGetErrorString(e));
    }
    return LBM_OK;
  };
  for (int n = 0; n < coarse_steps; ++n) {
    if (int rc = join_parts()) return rc;
    if (int rc = exchange(s)) return rc;
    cudaError_t e = cudaSuccess;
    for (int p = 0; p < s->P && e == cudaSuccess; ++p) e = cudaStreamWaitEvent(s->pstream[p], s->exchanged, 0);
    if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, std::string("fork: ") + cudaGetErrorString(e));
    for (lbm_ctx* p : s->parts) {
      const int rc = lbm_step(p, 1);
      if (rc) return sfail(s, rc, lbm_last_error(p));
    }
  }
  return join_parts();
}

int lbm_shard_get_state(lbm_shard* s, int level, double* f, size_t count) {
  if (!s || !f) return LBM_ERR_ARG;
  if (level < 0 || level >= s->levels) return sfail(s, LBM_ERR_ARG, "level out of range");
  const int64_t NX = int64_t(8) * s->g.nbx << level, NY = int64_t(8) * s->g.nby << level,
                NZ = int64_t(8) * s->g.nbz << level;
  if (count != size_t(s->Q) * NX * NY * NZ) return sfail(s, LBM_ERR_ARG, "count mismatch");
  for (int p = 0; p < s->P; ++p) {
    const int64_t x0 = int64_t(8) * s->cuts[p] << level, nxp = int64_t(8) * (s->cuts[p + 1] - s->cuts[p]) << level;
    std::vector<double> part(size_t(s->Q * nxp * NY * NZ), std::numeric_limits<double>::quiet_NaN());
    if (level < s->part_levels[p]) {
      const int rc = lbm_get_state(s->parts[p], level, part.data(), part.size());
      if (rc) return sfail(s, rc, lbm_last_error(s->parts[p]));
    }
    slab_copy(false, part.data(), f, s->Q, NX, NY, NZ, x0, nxp);
  }
  return LBM_OK;
}

int lbm_shard_macroscopic(lbm_shard* s, int level, double* rho, double* u) {
  if (!s || !rho || !u) return LBM_ERR_ARG;
  if (level < 0 || level >= s->levels) return sfail(s, LBM_ERR_ARG, "level out of range");
  const int64_t NX = int64_t(8) * s->g.nbx << level, NY = int64_t(8) * s->g.nby << level,
                NZ = int64_t(8) * s->g.nbz << level;
  for (int p = 0; p < s->P; ++p) {
    const int64_t x0 = int64_t(8) * s->cuts[p] << level, nxp = int64_t(8) * (s->cuts[p + 1] - s->cuts[p]) << level;
    const double nan = std::numeric_limits<double>::quiet_NaN();
    std::vector<double> r(size_t(nxp * NY * NZ), nan), v(size_t(3 * nxp * NY * NZ), nan);
    if (level < s->part_levels[p]) {
      const int rc = lbm_macroscopic(s->parts[p], level, r.data(), v.data());
      if (rc) return sfail(s, rc, lbm_last_error(s->parts[p]));
    }
    slab_copy(false, r.data(), rho, 1, NX, NY, NZ, x0, nxp);
    slab_copy(false, v.data(), u, 3, NX, NY, NZ, x0, nxp);
  }
  return LBM_OK;
}

int lbm_shard_mass_momentum(lbm_shard* s, double out[4]) {
  if (!s || !out) return LBM_ERR_ARG;
  double acc[4] = {0, 0, 0, 0};
  for (lbm_ctx* p : s->parts) {
    double m[4];
    const int rc = lbm_mass_momentum(p, m);
    if (rc) return sfail(s, rc, lbm_last_error(p));
    for (int k = 0; k < 4; ++k) acc[k] += m[k];  // the float64 sum over parts (an allreduce)
  }
  for (int k = 0; k < 4; ++k) out[k] = acc[k];
  return LBM_OK;
}

int lbm_shard_sync(lbm_shard* s) {
  if (!s) return LBM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(s->stream);
  for (size_t p = 0; p < s->pstream.size() && e == cudaSuccess; ++p) e = cudaStreamSynchronize(s->pstream[p]);
  if (e != cudaSuccess) return sfail(s, LBM_ERR_CUDA, cudaGetErrorString(e));
  return LBM_OK;
}

}  // extern "C"
