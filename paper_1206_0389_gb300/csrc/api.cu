// C ABI of liblbm.so: context, schedule of the time-nested substeps, CUDA
// graphs, autotuner and host <-> device staging.
//
// One coarse step of an L-level grid is 2^(L-1) finest substeps k.  At k the
// levels l with k % 2^(L-1-l) == 0 take a step (level l takes 2^l per coarse
// step, Sections 1 and 3.2); all of them run in ONE stream-collide launch,
// preceded by the coarse-to-fine transfers into their ghost cells and their
// boundary ghosts, and followed by the fine-to-coarse transfer of every level
// that has just finished its second substep.  This is the same sequence of
// values as the recursive schedule (level l, then its two fine substeps, then
// the restriction), regrouped so independent levels share a launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "plan.h"

using namespace lbm;

namespace {

thread_local std::string g_create_error;

struct Op {
  enum Kind { UPDATE, C2F, F2C, BC, LINK, INC } kind;
  int k = 0;            // finest-level substep of the coarse step the op belongs to
  bool level0 = false;  // an update of level-0 blocks alone (first substep of a nested grid)
  UpdateArgs ua{};
  C2FArgs ca{};
  F2CArgs fa{};
  BCArgs ba{};
  LinkArgs la{};
};

struct DevLevel {
  void* f[2] = {nullptr, nullptr};
  void* aux[2] = {nullptr, nullptr};
  uint8_t* kind = nullptr;
  C2FItem* c2f = nullptr;
  C2FChunk* c2f_chunks = nullptr;
  C2FCell* c2f_cells = nullptr;
  BCItem* c2f_bc = nullptr;
  F2CItem* f2c = nullptr;
  BCItem* bc = nullptr;
  LinkItem* links = nullptr;
  double* force = nullptr;
  float* force_f = nullptr;  // float copy for FP32/FP16 storage (compute type)
  double* stats = nullptr;   // time statistics sums [7][nblocks*512]
};

}  // namespace

struct lbm_ctx {
  GridPlan plan;
  int model = 0, storage = 0, Q = 19, L = 1;
  double omega = 1.0, cs = 0.0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // streams and events of the coarse-step graph's branches: the inflow
  // launch beside the coarse-to-fine launch (side), and the fine-level chain
  // (fine, high priority) beside the level-0 update (the capturing stream)
  cudaStream_t side = nullptr, fine = nullptr;
  std::vector<cudaEvent_t> fork_join;
  int device = 0, sms = 1;
  std::vector<DevLevel> dl;
  WorkItem* items = nullptr;          // merged lists for each lowest level
  std::vector<int64_t> list_off, list_len;
  uint32_t* masks = nullptr;
  long long* d_step = nullptr;
  double* partial = nullptr;          // reduction scratch [L][4*sms][4]
  double* d_out = nullptr;            // 4 doubles
  int* d_flag = nullptr;
  double* stage = nullptr;            // staging buffer for dense transfers
  size_t stage_bytes = 0;
  int parity0 = 0;                    // buffer of level 0 holding the current state
  int64_t step = 0;
  bool need_restrict = false;
  bool has_force = false;
  long long stats_n = 0;  // samples in the statistics sums
  // inflow
  double y0 = 0, z0 = 0, diameter = 0, u_in = 0, perturb = 0;
  double rho_out = 1.0;  // pressure outlet density
  uint64_t seed = 0;
  // launch configuration
  int threads = 256, minb = 1, ctas = 0;
  // graphs, one per level-0 parity
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool graphs_valid = false;
  bool profiling = false;
  // adjoint: checkpoints every `every` steps, segment buffers, lambda, dL/dF
  int adj_T = 0, adj_every = 0;
  bool adj_ready = false;
  uint64_t adj_gen = 0;  // completed lbm_adjoint_forward calls
  long long step_dev = 0;  // host source of a device step-counter update
  std::vector<void*> adj_ck, adj_seg;
  void* adj_lam[2] = {nullptr, nullptr};
  void* adj_gF = nullptr;
  size_t adj_state_bytes = 0;
  double prof_ms[5] = {0, 0, 0, 0, 0};
  int64_t prof_n[5] = {0, 0, 0, 0, 0};
  std::string err;
};

namespace {

int fail(lbm_ctx* c, int code, const std::string& m) {
  if (c) c->err = m;
  return code;
}
int cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define CK(call)                                               \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
  } while (0)

size_t real_bytes(int storage) { return storage == LBM_F64 ? 8 : 4; }

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc(dst, v.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// frees the adjoint buffers and forgets the recorded forward
void release_adjoint(lbm_ctx* c) {
  for (void* p : c->adj_ck) cudaFree(p);
  for (void* p : c->adj_seg) cudaFree(p);
  cudaFree(c->adj_lam[0]);
  cudaFree(c->adj_lam[1]);
  cudaFree(c->adj_gF);
  c->adj_ck.clear();
  c->adj_seg.clear();
  c->adj_lam[0] = c->adj_lam[1] = c->adj_gF = nullptr;
  c->adj_state_bytes = 0;
  c->adj_ready = false;
}

void free_all(lbm_ctx* c) {
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
  for (DevLevel& d : c->dl) {
    cudaFree(d.f[0]);
    cudaFree(d.f[1]);
    cudaFree(d.aux[0]);
    cudaFree(d.aux[1]);
    cudaFree(d.kind);
    cudaFree(d.c2f);
    cudaFree(d.c2f_chunks);
    cudaFree(d.c2f_cells);
    cudaFree(d.c2f_bc);
    cudaFree(d.f2c);
    cudaFree(d.bc);
    cudaFree(d.links);
    cudaFree(d.force);
    cudaFree(d.force_f);
    cudaFree(d.stats);
  }
  cudaFree(c->items);
  cudaFree(c->masks);
  cudaFree(c->d_step);
  cudaFree(c->partial);
  cudaFree(c->d_out);
  cudaFree(c->d_flag);
  cudaFree(c->stage);
  release_adjoint(c);
  for (cudaEvent_t e : c->fork_join) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->fine) cudaStreamDestroy(c->fine);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

// --------------------------------------------------------------- schedule
// Whether the coarse-step graph runs level 0's work beside the fine levels'
// chain (nested grids with FP16 storage).  Measured on the paper-scale
// 3-level jet: FP16 1.454 -> 1.427 ms per coarse step (its half-scale copy
// 0.303 -> 0.280); FP32 2.100 -> 2.204 ms and the 2-level FP32 jets 1-2 %
// slower, where the level-0 update is bandwidth-bound on its own and the
// two branches only compete for DRAM and L2.
bool split_level0(const lbm_ctx* c) { return c->L > 1 && c->storage == LBM_F16; }

std::vector<Op> build_schedule(lbm_ctx* c, int p0) {
  std::vector<Op> ops;
  const int L = c->L;
  int par[kMaxL] = {0, 0, 0, 0};
  par[0] = p0;
  const double cs2_3 = 3.0 * c->cs * c->cs;
  const bool les = c->model == LBM_D3Q19_MRT_LES;
  const int K = 1 << (L - 1);
  for (int k = 0; k < K; ++k) {
    int lmin = L - 1;
    for (int l = 0; l < L; ++l)
      if (k % (1 << (L - 1 - l)) == 0) {
        lmin = l;
        break;
      }
    auto sub = [&](int l) { return k / (1 << (L - 1 - l)); };
    // coarse-to-fine for every level starting a substep: one launch (level
    // l writes its ghost cells and reads active / hidden-1 cells of l-1)
    if (std::max(lmin, 1) < L) {
      Op op;
      op.kind = Op::C2F;
      C2FArgs& a = op.ca;
      a.cs2_3 = cs2_3;
      a.step = c->d_step;
      a.y0 = c->y0;
      a.z0 = c->z0;
      a.r2 = (0.5 * c->diameter) * (0.5 * c->diameter);
      a.u_in = c->u_in;
      a.perturb = c->perturb;
      a.seed = c->seed;
      a.closed = c->plan.nozzle_level >= 0;
      for (int l = std::max(lmin, 1); l < L; ++l) {
        const int s = sub(l) % 2;
        const LevelPlan& fp = c->plan.lv[l];
        const LevelPlan& cp = c->plan.lv[l - 1];
        if (fp.c2f_chunks.empty()) continue;
        C2FLevel& v = a.lv[a.nlv++];
        v.chunks = c->dl[l].c2f_chunks;
        v.items = c->dl[l].c2f;
        v.cells = c->dl[l].c2f_cells;
        v.bc = c->dl[l].c2f_bc;
        v.level = l;
        v.substep = sub(l);
        v.NY = fp.NY;
        v.inv_scale = std::ldexp(1.0, -l);
        v.n = int(fp.c2f_chunks.size());
        const int pc = par[l - 1];
        v.c_old = c->dl[l - 1].f[s == 0 ? pc : 1 - pc];
        v.c_new = c->dl[l - 1].f[pc];
        v.a_old = les ? c->dl[l - 1].aux[s == 0 ? pc : 1 - pc] : nullptr;
        v.a_new = les ? c->dl[l - 1].aux[pc] : nullptr;
        v.f_dst = c->dl[l].f[par[l]];
        v.fa_dst = les ? c->dl[l].aux[par[l]] : nullptr;
        v.s = s;
        v.tau0_c = cp.tau0;
        v.tau0_f = fp.tau0;
        a.n += v.n;
      }
      if (a.n > 0) {
        op.k = k;
        ops.push_back(op);
      }
    }
    // inflow / outflow ghosts of the same levels (after the interface: an
    // inflow ghost may take its density from a coarse-to-fine ghost cell)
    if (!c->plan.periodic_x) {
      Op op;
      op.kind = Op::BC;
      BCArgs& b = op.ba;
      b.step = c->d_step;
      b.y0 = c->y0;
      b.z0 = c->z0;
      b.r2 = (0.5 * c->diameter) * (0.5 * c->diameter);
      b.u_in = c->u_in;
      b.perturb = c->perturb;
      b.seed = c->seed;
      b.rl_out = c->rho_out - 1.0;
      b.closed = c->plan.nozzle_level >= 0;
      for (int l = lmin; l < L; ++l) {
        const LevelPlan& lp = c->plan.lv[l];
        if (lp.bc.empty()) continue;
        BCLevel& v = b.lv[b.nlv++];
        v.items = c->dl[l].bc;
        v.n = int(lp.bc.size());
        v.f = c->dl[l].f[par[l]];
        v.level = l;
        v.substep = sub(l);
        v.NY = lp.NY;
        v.inv_scale = std::ldexp(1.0, -l);
        b.n += v.n;
      }
      op.k = k;
      if (b.n > 0) ops.push_back(op);
    }
    // nozzle links of its level (after the level's previous update, before
    // this one; they touch only cells near the body)
    const int ln = c->plan.nozzle_level;
    if (ln >= lmin && !c->plan.lv[ln].links.empty()) {
      Op op;
      op.kind = Op::LINK;
      LinkArgs& a = op.la;
      a.items = c->dl[ln].links;
      a.n = int(c->plan.lv[ln].links.size());
      a.f = c->dl[ln].f[par[ln]];
      a.level = ln;
      a.substep = sub(ln);
      a.NY = c->plan.lv[ln].NY;
      a.inv_scale = std::ldexp(1.0, -ln);
      a.step = c->d_step;
      a.y0 = c->y0;
      a.z0 = c->z0;
      a.r2 = (0.5 * c->diameter) * (0.5 * c->diameter);
      a.u_in = c->u_in;
      a.perturb = c->perturb;
      a.seed = c->seed;
      op.k = k;
      ops.push_back(op);
    }
    Op up;
    up.kind = Op::UPDATE;
    UpdateArgs& u = up.ua;
    for (int l = 0; l < L; ++l) {
      const LevelPlan& lp = c->plan.lv[l];
      u.lv[l].src = c->dl[l].f[par[l]];
      u.lv[l].dst = c->dl[l].f[1 - par[l]];
      u.lv[l].aux_dst = les && L > 1 ? c->dl[l].aux[1 - par[l]] : nullptr;
      u.lv[l].BX = lp.BX;
      u.lv[l].BY = lp.BY;
      u.lv[l].BZ = lp.BZ;
      u.lv[l].tau0 = lp.tau0;
    }
    u.items = c->items + c->list_off[lmin];
    u.nitems = int(c->list_len[lmin]);
    u.masks = c->masks;
    u.cs2_18 = 18.0 * c->cs * c->cs;
    u.force = !c->has_force ? nullptr
              : c->storage == LBM_F64 ? static_cast<const void*>(c->dl[0].force)
                                       : static_cast<const void*>(c->dl[0].force_f);
    u.walls = c->plan.walls;
    u.slip = c->plan.slip;
    up.k = k;
    if (lmin == 0 && split_level0(c)) {
      // the first substep updates level 0 in a launch of its own: nothing
      // reads its result before the midpoint of the coarse step, so the
      // graph runs it beside the fine levels' first half
      Op u0 = up;
      u0.level0 = true;
      u0.ua.nitems = int(c->list_len[0] - c->list_len[1]);
      up.ua.items = c->items + c->list_off[1];
      up.ua.nitems = int(c->list_len[1]);
      ops.push_back(u0);
    }
    ops.push_back(up);
    for (int l = lmin; l < L; ++l) par[l] ^= 1;
    // fine-to-coarse after the second substep of each fine level: one launch
    // (level l-1's hidden cells take level l's active cells, which no other
    // level of the launch writes)
    {
      Op op;
      op.kind = Op::F2C;
      F2CArgs& a = op.fa;
      a.cs2_3 = cs2_3;
      for (int l = L - 1; l >= std::max(lmin, 1); --l) {
        if (sub(l) % 2 != 1) continue;
        const LevelPlan& fp = c->plan.lv[l];
        const LevelPlan& cp = c->plan.lv[l - 1];
        if (cp.f2c.empty()) continue;
        F2CLevel& v = a.lv[a.nlv++];
        v.items = c->dl[l - 1].f2c;
        v.n = int(cp.f2c.size());
        v.f_src = c->dl[l].f[par[l]];
        v.fa_src = les ? c->dl[l].aux[par[l]] : nullptr;
        v.c_dst = c->dl[l - 1].f[par[l - 1]];
        v.ca_dst = les ? c->dl[l - 1].aux[par[l - 1]] : nullptr;
        v.tau0_c = cp.tau0;
        v.tau0_f = fp.tau0;
        a.n += v.n;
        op.level0 = l == 1;
      }
      op.k = k;
      // a restriction into level 0 alone: nothing later in the coarse step
      // touches level 0, so the graph runs it beside the rest
      op.level0 = op.level0 && a.nlv == 1 && split_level0(c);
      if (a.n > 0) ops.push_back(op);
    }
  }
  Op inc;
  inc.k = K - 1;
  inc.kind = Op::INC;
  ops.push_back(inc);
  return ops;
}

cudaError_t run_op(lbm_ctx* c, const Op& op, cudaStream_t st) {
  switch (op.kind) {
    case Op::UPDATE: return launch_update(c->model, c->storage, op.ua, c->threads, c->minb, c->ctas, st);
    case Op::C2F: return launch_c2f(c->model, c->storage, op.ca, st);
    case Op::F2C: return launch_f2c(c->model, c->storage, op.fa, st);
    case Op::BC: return launch_bc(c->model, c->storage, op.ba, st);
    case Op::LINK: return launch_links(c->model, c->storage, op.la, st);
    case Op::INC: return launch_step_inc(c->d_step, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t run_op(lbm_ctx* c, const Op& op) { return run_op(c, op, c->stream); }

int op_kind_index(const Op& op) {
  switch (op.kind) {
    case Op::UPDATE: return 0;
    case Op::C2F: return 1;
    case Op::F2C: return 2;
    case Op::BC:
    case Op::LINK: return 3;
    default: return 4;
  }
}

// restriction of every hidden layer from the current fine state (after an
// equilibrium initialisation), finest level first
int restrict_all(lbm_ctx* ctx) {
  const bool les = ctx->model == LBM_D3Q19_MRT_LES;
  for (int l = ctx->L - 1; l >= 1; --l) {
    F2CArgs a{};
    F2CLevel& v = a.lv[0];
    a.nlv = 1;
    v.items = ctx->dl[l - 1].f2c;
    v.n = a.n = int(ctx->plan.lv[l - 1].f2c.size());
    v.f_src = ctx->dl[l].f[0];
    v.fa_src = les ? ctx->dl[l].aux[0] : nullptr;
    const int pc = l - 1 == 0 ? ctx->parity0 : 0;
    v.c_dst = ctx->dl[l - 1].f[pc];
    v.ca_dst = les ? ctx->dl[l - 1].aux[pc] : nullptr;
    v.tau0_c = ctx->plan.lv[l - 1].tau0;
    v.tau0_f = ctx->plan.lv[l].tau0;
    a.cs2_3 = 3.0 * ctx->cs * ctx->cs;
    CK(launch_f2c(ctx->model, ctx->storage, a, ctx->stream));
  }
  ctx->need_restrict = false;
  return LBM_OK;
}

int build_graphs(lbm_ctx* ctx) {
  const int K = 1 << (ctx->L - 1);
  for (int p = 0; p < 2; ++p) {
    if (ctx->graph[p]) {
      cudaGraphExecDestroy(ctx->graph[p]);
      ctx->graph[p] = nullptr;
    }
    std::vector<Op> ops = build_schedule(ctx, p);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    size_t ev = 0;
    auto next_event = [&](cudaEvent_t* out) {
      if (ev >= ctx->fork_join.size()) return cudaErrorInvalidValue;
      *out = ctx->fork_join[ev++];
      return cudaSuccess;
    };
    // Nested FP16 grids: the chain of ops runs on the high-priority stream `fine`;
    // the level-0 update of the first substep runs on the capturing stream
    // beside it, after the level-0 inflow (and nozzle links) it reads, and
    // joins the chain before the first op of the second half of the coarse
    // step (the coarse-to-fine launch that reads level 0's new state, the
    // restriction into level 0); that restriction in turn runs beside the
    // rest of the chain (nothing after it touches level 0).  The level-0
    // blocks fill the SMs the short interface launches leave idle.
    const bool split = split_level0(ctx);
    cudaStream_t st = ctx->stream;
    cudaEvent_t u0_after = nullptr, u0_done = nullptr, r0_done = nullptr, evt = nullptr;
    if (split) {
      if ((e = next_event(&evt)) == cudaSuccess && (e = cudaEventRecord(evt, ctx->stream)) == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->fine, evt, 0);
      st = ctx->fine;
    }
    for (size_t k = 0; k < ops.size() && e == cudaSuccess; ++k) {
      const Op& op = ops[k];
      if (u0_done && op.k >= K / 2) {
        if ((e = cudaStreamWaitEvent(st, u0_done, 0)) != cudaSuccess) break;
        u0_done = nullptr;
      }
      // the inflow launch after a coarse-to-fine launch touches other cells
      // (inflow ghosts fed by ghost cells are written by the latter), so the
      // graph runs the two side by side
      if (op.kind == Op::C2F && k + 1 < ops.size() && ops[k + 1].kind == Op::BC) {
        cudaEvent_t fork = nullptr, join = nullptr;
        if ((e = next_event(&fork)) != cudaSuccess || (e = next_event(&join)) != cudaSuccess ||
            (e = cudaEventRecord(fork, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->side, fork, 0)) != cudaSuccess ||
            (e = run_op(ctx, ops[k + 1], ctx->side)) != cudaSuccess ||
            (e = run_op(ctx, op, st)) != cudaSuccess ||
            (e = cudaEventRecord(join, ctx->side)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess)
          break;
        if (ops[k + 1].k == 0) u0_after = join;  // the inflow is done
        ++k;
        continue;
      }
      if (split && op.level0 && op.kind == Op::UPDATE) {
        if (u0_after && (e = cudaStreamWaitEvent(ctx->stream, u0_after, 0)) != cudaSuccess) break;
        if ((e = run_op(ctx, op, ctx->stream)) != cudaSuccess || (e = next_event(&u0_done)) != cudaSuccess ||
            (e = cudaEventRecord(u0_done, ctx->stream)) != cudaSuccess)
          break;
        continue;
      }
      if (split && op.level0 && op.kind == Op::F2C && !u0_done && !r0_done) {
        // after the chain so far; joined at the end of the coarse step
        cudaEvent_t here = nullptr;
        if ((e = next_event(&here)) != cudaSuccess || (e = cudaEventRecord(here, st)) != cudaSuccess ||
            (e = cudaStreamWaitEvent(ctx->stream, here, 0)) != cudaSuccess ||
            (e = run_op(ctx, op, ctx->stream)) != cudaSuccess || (e = next_event(&r0_done)) != cudaSuccess ||
            (e = cudaEventRecord(r0_done, ctx->stream)) != cudaSuccess)
          break;
        continue;
      }
      if ((e = run_op(ctx, op, st)) != cudaSuccess) break;
      if (split && op.k == 0 && (op.kind == Op::BC || (op.kind == Op::LINK && op.la.level == 0))) {
        // the level-0 update waits for the chain up to here
        if ((e = next_event(&u0_after)) != cudaSuccess || (e = cudaEventRecord(u0_after, st)) != cudaSuccess) break;
      }
    }
    if (split && e == cudaSuccess) {
      if (u0_done) e = cudaStreamWaitEvent(st, u0_done, 0);
      if (r0_done && e == cudaSuccess) e = cudaStreamWaitEvent(st, r0_done, 0);
      if (e == cudaSuccess && (e = next_event(&evt)) == cudaSuccess && (e = cudaEventRecord(evt, st)) == cudaSuccess)
        e = cudaStreamWaitEvent(ctx->stream, evt, 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(ctx, e, "capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    // kernel nodes carry the priority of the stream they were captured from
    e = cudaGraphInstantiateWithFlags(&ctx->graph[p], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiateWithFlags");
  }
  ctx->graphs_valid = true;
  return LBM_OK;
}

// Pick the stream-collide launch shape by timing the largest update launch of
// the schedule: threads per CTA in {128, 256} with register caps, one CTA per block or a
// persistent grid of (CTAs per SM x SMs).  Writes only the other buffer.
int autotune(lbm_ctx* ctx) {
  const char* env = std::getenv("LBM_AUTOTUNE");
  if (env && std::strcmp(env, "0") == 0) return LBM_OK;
  std::vector<Op> ops = build_schedule(ctx, ctx->parity0);
  const Op* big = nullptr;
  for (const Op& op : ops)
    if (op.kind == Op::UPDATE && (!big || op.ua.nitems > big->ua.nitems)) big = &op;
  if (!big || big->ua.nitems == 0) return LBM_OK;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int bt = 256, bm = 1, bc = 0;
  // (no 512-thread shape: with one pass over the 512 cells of a block its
  // kernel is optimised into differently rounded arithmetic)
  const int shapes[5][2] = {{128, 1}, {256, 1}, {128, 8}, {256, 4}, {128, 7}};
  // LBM_LAUNCH_SHAPE="threads,min_ctas_per_sm,persistent" fixes one of the
  // shapes below without timing (profilers distort the timings).
  if (const char* fixed = std::getenv("LBM_LAUNCH_SHAPE")) {
    int t = 0, mb = 0, pers = -1;
    bool ok = std::sscanf(fixed, "%d,%d,%d", &t, &mb, &pers) == 3 && (pers == 0 || pers == 1);
    bool listed = false;
    for (const auto& sh : shapes) listed |= sh[0] == t && sh[1] == mb;
    int occ = 0;
    ok = ok && listed && update_occupancy(ctx->model, ctx->storage, ctx->plan.walls != 0, t, mb, &occ) == cudaSuccess && occ >= 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) return fail(ctx, LBM_ERR_ARG, std::string("LBM_LAUNCH_SHAPE not a listed shape: ") + fixed);
    ctx->threads = t;
    ctx->minb = mb;
    ctx->ctas = pers ? occ * ctx->sms : 0;
    return LBM_OK;
  }
  for (const auto& sh : shapes) {
    const int t = sh[0], mb = sh[1];
    int occ = 0;
    if (update_occupancy(ctx->model, ctx->storage, ctx->plan.walls != 0, t, mb, &occ) != cudaSuccess || occ < 1) continue;
    const int clist[2] = {0, occ * ctx->sms};
    for (int cc : clist) {
      if (launch_update(ctx->model, ctx->storage, big->ua, t, mb, cc, ctx->stream) != cudaSuccess) continue;
      CK(launch_update(ctx->model, ctx->storage, big->ua, t, mb, cc, ctx->stream));
      // best of three groups of four launches
      float ms = 1e30f;
      for (int grp = 0; grp < 3; ++grp) {
        CK(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 4; ++r) CK(launch_update(ctx->model, ctx->storage, big->ua, t, mb, cc, ctx->stream));
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float g = 0;
        CK(cudaEventElapsedTime(&g, e0, e1));
        ms = std::min(ms, g);
      }
      if (ms < best) {
        best = ms;
        bt = t;
        bm = mb;
        bc = cc;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->threads = bt;
  ctx->minb = bm;
  ctx->ctas = bc;
  return LBM_OK;
}

int ensure_stage(lbm_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return LBM_OK;
  if (ctx->stage) cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  cudaError_t e = cudaMalloc(&ctx->stage, bytes);
  if (e != cudaSuccess) return fail(ctx, LBM_ERR_OOM, std::string("staging buffer: ") + cudaGetErrorString(e));
  ctx->stage_bytes = bytes;
  return LBM_OK;
}

int cur_parity(const lbm_ctx* ctx, int level) { return level == 0 ? ctx->parity0 : 0; }

// Move a dense per-level array through the device slab by slab.  hin[c] /
// hout[c] are the host arrays of the comps components ([NZ][NY][NX] each);
// a NULL input component is filled with fill[c] on the device.
int slab_transfer(lbm_ctx* ctx, int level, int mode, const double* const* hin, double* const* hout,
                  int comps, const double* fill = nullptr, void* raw = nullptr, double scale = 1.0) {
  const LevelPlan& lp = ctx->plan.lv[level];
  const int64_t plane = int64_t(lp.NX) * lp.NY;
  int nz = 8;
  while (nz < lp.NZ && int64_t(2 * nz) * plane * comps * 8 <= (int64_t(256) << 20)) nz *= 2;
  nz = std::min(nz, lp.NZ);
  int rc = ensure_stage(ctx, size_t(nz) * plane * comps * sizeof(double));
  if (rc) return rc;
  for (int z0 = 0; z0 < lp.NZ; z0 += nz) {
    const int n = std::min(nz, lp.NZ - z0);
    const int64_t cnt = int64_t(n) * plane;
    if (hin)
      for (int c = 0; c < comps; ++c) {
        if (hin[c])
          CK(cudaMemcpyAsync(ctx->stage + c * cnt, hin[c] + z0 * plane, cnt * sizeof(double),
                             cudaMemcpyHostToDevice, ctx->stream));
        else
          CK(launch_fill(ctx->stage + c * cnt, cnt, fill ? fill[c] : 0.0, ctx->stream));
      }
    SlabArgs a{};
    a.f = ctx->dl[level].f[cur_parity(ctx, level)];
    a.kind = ctx->dl[level].kind;
    a.force = ctx->dl[level].force;
    if (mode == SLAB_MACRO && !(ctx->has_force && level == 0)) a.force = nullptr;
    a.ox = lp.ox;
    a.oy = lp.oy;
    a.oz = lp.oz;
    a.BX = lp.BX;
    a.BY = lp.BY;
    a.BZ = lp.BZ;
    a.NX = lp.NX;
    a.NY = lp.NY;
    a.z0 = z0;
    a.nz = n;
    a.in = ctx->stage;
    a.out = ctx->stage;
    a.mode = mode;
    a.raw = raw;
    a.scale = scale;
    CK(launch_slab(ctx->model, ctx->storage, a, ctx->stream));
    if (hout)
      for (int c = 0; c < comps; ++c)
        CK(cudaMemcpyAsync(hout[c] + z0 * plane, ctx->stage + c * cnt, cnt * sizeof(double),
                           cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

bool all_finite(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

}  // namespace

int create_context(lbm_ctx** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
                   double cs, void* cuda_stream, const PlanOptions& opt);

// ======================================================================= C ABI
extern "C" {

int lbm_plan(const lbm_grid* g, int model, int storage, lbm_plan_info* out) {
  if (!g || !out) return LBM_ERR_ARG;
  GridPlan P;
  std::string e = build_plan(*g, model, storage, 1.0, P);
  if (!e.empty()) return LBM_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->levels = P.levels;
  for (int l = 0; l < P.levels; ++l) {
    const LevelPlan& lp = P.lv[l];
    out->blocks[l] = lp.nblocks();
    out->level_blocks[l] = lp.level_blocks;
    out->active_cells[l] = lp.active_cells;
    out->updated_cells[l] = lp.updated_cells;
    out->hidden_cells[l] = lp.hidden_cells;
    out->ghost_cells[l] = lp.ghost_cells;
    out->bc_cells[l] = lp.bc_cells;
    out->updates_per_coarse_step += lp.updated_cells << l;
    out->active_updates_per_coarse_step += lp.active_cells << l;
  }
  out->device_bytes = P.device_bytes;
  out->nozzle_level = P.nozzle_level;
  out->solid_cells = P.nozzle_level >= 0 ? P.lv[P.nozzle_level].solid_cells : 0;
  out->nozzle_links = P.nozzle_level >= 0 ? int64_t(P.lv[P.nozzle_level].links.size()) : 0;
  return LBM_OK;
}

const char* lbm_create_error(void) { return g_create_error.c_str(); }

int lbm_create(lbm_ctx** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
               double cs, void* cuda_stream) {
  return create_context(out, model, storage, g, omega, cs, cuda_stream, PlanOptions());
}

}  // extern "C"

// lbm_create with plan options (the parts of a sharded grid)
int create_context(lbm_ctx** out, lbm_model model, lbm_storage storage, const lbm_grid* g, double omega,
                   double cs, void* cuda_stream, const PlanOptions& opt) {
  g_create_error.clear();
  if (!out) {
    g_create_error = "out is NULL";
    return LBM_ERR_ARG;
  }
  *out = nullptr;
  if (!g) {
    g_create_error = "grid is NULL";
    return LBM_ERR_ARG;
  }
  if (!(cs >= 0.0 && cs < 1.0)) {
    g_create_error = "cs must be in [0, 1)";
    return LBM_ERR_ARG;
  }
  lbm_ctx* ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) {
    g_create_error = "host allocation failed";
    return LBM_ERR_OOM;
  }
  std::string e = build_plan(*g, int(model), int(storage), omega, ctx->plan, opt);
  if (!e.empty()) {
    g_create_error = e;
    delete ctx;
    return LBM_ERR_ARG;
  }
  ctx->model = int(model);
  ctx->storage = int(storage);
  ctx->Q = ctx->plan.Q;
  ctx->L = ctx->plan.levels;
  ctx->omega = omega;
  ctx->cs = model == LBM_D3Q19_MRT_LES ? cs : 0.0;
  auto bail = [&](int code, const std::string& m) {
    g_create_error = m;
    free_all(ctx);
    delete ctx;
    return code;
  };
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0)
    return bail(LBM_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(ce));
  cudaGetDevice(&ctx->device);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (cuda_stream) {
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    ce = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(ce));
    ctx->own_stream = true;
  }
  {
    // the fine-level chain of the coarse-step graph runs at the highest
    // stream priority, the level-0 update beside it at the caller's
    int least = 0, greatest = 0;
    ce = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, greatest);
    if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&ctx->fine, cudaStreamNonBlocking, greatest);
    if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(ce));
  }
  // events of one coarse-step capture: a fork and a join per coarse-to-fine
  // launch, and at most six for the level-0 branches
  ctx->fork_join.assign(2 * (1 << (ctx->L - 1)) + 8, nullptr);
  for (cudaEvent_t& e : ctx->fork_join) {
    ce = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, std::string("event: ") + cudaGetErrorString(ce));
  }
  const size_t sb = storage_bytes(ctx->storage), rb = real_bytes(ctx->storage);
  const bool aux = ctx->model == LBM_D3Q19_MRT_LES && ctx->L > 1;
  ctx->dl.resize(ctx->L);
  std::vector<WorkItem> all;
  std::vector<uint32_t> masks;
  std::vector<std::vector<WorkItem>> per(ctx->L);
  for (int l = 0; l < ctx->L; ++l) {
    const LevelPlan& lp = ctx->plan.lv[l];
    DevLevel& d = ctx->dl[l];
    const size_t fb = size_t(lp.nblocks()) * 512 * ctx->Q * sb;
    for (int p = 0; p < 2; ++p) {
      ce = cudaMalloc(&d.f[p], fb);
      if (ce != cudaSuccess) return bail(LBM_ERR_OOM, "distribution buffers: " + std::string(cudaGetErrorString(ce)));
      ce = cudaMemsetAsync(d.f[p], 0, fb, ctx->stream);
      if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, cudaGetErrorString(ce));
      if (aux) {
        ce = cudaMalloc(&d.aux[p], size_t(lp.nblocks()) * 512 * rb);
        if (ce != cudaSuccess) return bail(LBM_ERR_OOM, "strain buffers: " + std::string(cudaGetErrorString(ce)));
        ce = cudaMemsetAsync(d.aux[p], 0, size_t(lp.nblocks()) * 512 * rb, ctx->stream);
        if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, cudaGetErrorString(ce));
      }
    }
    if ((ce = upload(&d.kind, lp.kind)) != cudaSuccess || (ce = upload(&d.c2f, lp.c2f)) != cudaSuccess ||
        (ce = upload(&d.c2f_chunks, lp.c2f_chunks)) != cudaSuccess ||
        (ce = upload(&d.c2f_cells, lp.c2f_cells)) != cudaSuccess ||
        (ce = upload(&d.c2f_bc, lp.c2f_bc)) != cudaSuccess ||
        (ce = upload(&d.f2c, lp.f2c)) != cudaSuccess || (ce = upload(&d.bc, lp.bc)) != cudaSuccess ||
        (ce = upload(&d.links, lp.links)) != cudaSuccess)
      return bail(LBM_ERR_OOM, std::string("plan tables: ") + cudaGetErrorString(ce));
    const int16_t moff = int16_t(masks.size() / 16);
    masks.insert(masks.end(), lp.masks.begin(), lp.masks.end());
    for (WorkItem w : lp.items) {
      if (w.mask >= 0) w.mask = int16_t(w.mask + moff);
      per[l].push_back(w);
    }
  }
  if (masks.size() / 16 > 32767) return bail(LBM_ERR_ARG, "too many masked blocks");
  ctx->list_off.assign(ctx->L, 0);
  ctx->list_len.assign(ctx->L, 0);
  for (int lmin = 0; lmin < ctx->L; ++lmin) {
    ctx->list_off[lmin] = int64_t(all.size());
    for (int l = lmin; l < ctx->L; ++l) all.insert(all.end(), per[l].begin(), per[l].end());
    ctx->list_len[lmin] = int64_t(all.size()) - ctx->list_off[lmin];
  }
  if (all.size() > size_t(1) << 31) return bail(LBM_ERR_ARG, "too many blocks");
  if ((ce = upload(&ctx->items, all)) != cudaSuccess || (ce = upload(&ctx->masks, masks)) != cudaSuccess)
    return bail(LBM_ERR_OOM, std::string("work lists: ") + cudaGetErrorString(ce));
  if ((ce = cudaMalloc(&ctx->d_step, sizeof(long long))) != cudaSuccess ||
      (ce = cudaMemsetAsync(ctx->d_step, 0, sizeof(long long), ctx->stream)) != cudaSuccess ||
      (ce = cudaMalloc(&ctx->partial, size_t(ctx->L) * 4 * ctx->sms * 4 * sizeof(double))) != cudaSuccess ||
      (ce = cudaMalloc(&ctx->d_out, 4 * sizeof(double))) != cudaSuccess ||
      (ce = cudaMalloc(&ctx->d_flag, sizeof(int))) != cudaSuccess)
    return bail(LBM_ERR_OOM, std::string("scratch: ") + cudaGetErrorString(ce));
  ctx->need_restrict = ctx->L > 1;
  ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, std::string("init: ") + cudaGetErrorString(ce));
  if (int rc = autotune(ctx); rc != LBM_OK) return bail(rc, "autotune: " + ctx->err);
  // the tuning runs wrote the second buffers; clear them again
  for (int l = 0; l < ctx->L; ++l) {
    const size_t fb = size_t(ctx->plan.lv[l].nblocks()) * 512 * ctx->Q * sb;
    cudaMemsetAsync(ctx->dl[l].f[1], 0, fb, ctx->stream);
    if (aux) cudaMemsetAsync(ctx->dl[l].aux[1], 0, size_t(ctx->plan.lv[l].nblocks()) * 512 * rb, ctx->stream);
  }
  ce = cudaStreamSynchronize(ctx->stream);
  if (ce != cudaSuccess) return bail(LBM_ERR_CUDA, std::string("init: ") + cudaGetErrorString(ce));
  *out = ctx;
  return LBM_OK;
}

extern "C" {

void lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  delete ctx;
}

const char* lbm_last_error(const lbm_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

int lbm_set_inflow(lbm_ctx* ctx, double y0, double z0, double diameter, double u_in, double perturb,
                   uint64_t seed) {
  if (!ctx) return LBM_ERR_ARG;
  if (ctx->plan.periodic_x) return fail(ctx, LBM_ERR_STATE, "inflow needs a non-periodic x axis");
  if (!std::isfinite(y0) || !std::isfinite(z0) || !std::isfinite(diameter) || !std::isfinite(u_in) ||
      !std::isfinite(perturb))
    return fail(ctx, LBM_ERR_NONFINITE, "non-finite inflow parameter");
  if (diameter < 0 || std::fabs(u_in) >= 0.5 || perturb < 0 || perturb > 1)
    return fail(ctx, LBM_ERR_ARG, "inflow parameters out of range");
  ctx->y0 = y0;
  ctx->z0 = z0;
  ctx->diameter = diameter;
  ctx->u_in = u_in;
  ctx->perturb = perturb;
  ctx->seed = seed;
  ctx->graphs_valid = false;
  return LBM_OK;
}

int lbm_set_outlet(lbm_ctx* ctx, double rho_out) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->plan.outlet) return fail(ctx, LBM_ERR_STATE, "the grid has no pressure outlet");
  if (!std::isfinite(rho_out)) return fail(ctx, LBM_ERR_NONFINITE, "non-finite outlet density");
  if (!(rho_out > 0.5 && rho_out < 2.0)) return fail(ctx, LBM_ERR_ARG, "outlet density out of range");
  ctx->rho_out = rho_out;
  ctx->graphs_valid = false;
  return LBM_OK;
}

int lbm_init_equilibrium(lbm_ctx* ctx, int level, const double* rho, const double* u) {
  if (!ctx) return LBM_ERR_ARG;
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  if ((rho && !all_finite(rho, n)) || (u && !all_finite(u, 3 * n)))
    return fail(ctx, LBM_ERR_NONFINITE, "non-finite rho or u");
  if (rho)
    for (size_t i = 0; i < n; ++i)
      if (!(rho[i] > 0)) return fail(ctx, LBM_ERR_ARG, "rho must be positive");
  const double* hin[4] = {rho, u, u ? u + n : nullptr, u ? u + 2 * n : nullptr};
  const double fill[4] = {1.0, 0.0, 0.0, 0.0};
  int rc = slab_transfer(ctx, level, SLAB_INIT_EQ, hin, nullptr, 4, fill);
  if (rc) return rc;
  const bool aux = ctx->model == LBM_D3Q19_MRT_LES && ctx->L > 1;
  if (aux)
    for (int p = 0; p < 2; ++p)
      CK(cudaMemsetAsync(ctx->dl[level].aux[p], 0, size_t(lp.nblocks()) * 512 * real_bytes(ctx->storage),
                         ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->need_restrict = ctx->L > 1;
  return LBM_OK;
}

int lbm_set_force(lbm_ctx* ctx, const double* F) {
  if (!ctx) return LBM_ERR_ARG;
  // the backward sweep reads the force: a recorded forward no longer matches
  ctx->adj_ready = false;
  if (F == nullptr) {
    ctx->has_force = false;
    ctx->graphs_valid = false;
    return LBM_OK;
  }
  if (ctx->model != LBM_D3Q27_FCLB || ctx->L != 1)
    return fail(ctx, LBM_ERR_STATE, "body force is defined for single-level D3Q27 grids");
  const LevelPlan& lp = ctx->plan.lv[0];
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  if (!all_finite(F, 3 * n)) return fail(ctx, LBM_ERR_NONFINITE, "non-finite force");
  if (!ctx->dl[0].force) {
    CK(cudaMalloc(&ctx->dl[0].force, size_t(lp.nblocks()) * 512 * 3 * sizeof(double)));
    CK(cudaMemsetAsync(ctx->dl[0].force, 0, size_t(lp.nblocks()) * 512 * 3 * sizeof(double), ctx->stream));
  }
  const double* hin[3] = {F, F + n, F + 2 * n};
  int rc = slab_transfer(ctx, 0, SLAB_SET_FORCE, hin, nullptr, 3);
  if (rc) return rc;
  if (ctx->storage != LBM_F64) {
    const long long nf = (long long)lp.nblocks() * 512 * 3;
    if (!ctx->dl[0].force_f) CK(cudaMalloc(&ctx->dl[0].force_f, size_t(nf) * sizeof(float)));
    CK(launch_to_float(ctx->dl[0].force, ctx->dl[0].force_f, nf, ctx->stream));
  }
  ctx->has_force = true;
  ctx->graphs_valid = false;
  return LBM_OK;
}

int lbm_step(lbm_ctx* ctx, int coarse_steps) {
  if (!ctx) return LBM_ERR_ARG;
  if (coarse_steps < 0) return fail(ctx, LBM_ERR_ARG, "coarse_steps must be >= 0");
  if (coarse_steps == 0) return LBM_OK;
  if (ctx->need_restrict) {
    int rc = restrict_all(ctx);
    if (rc) return rc;
  }
  if (ctx->profiling) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int n = 0; n < coarse_steps; ++n) {
      std::vector<Op> ops = build_schedule(ctx, ctx->parity0);
      for (const Op& op : ops) {
        CK(cudaEventRecord(e0, ctx->stream));
        CK(run_op(ctx, op));
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const int k = op_kind_index(op);
        ctx->prof_ms[k] += ms;
        ctx->prof_n[k] += 1;
      }
      ctx->parity0 ^= 1;
      ctx->step++;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return LBM_OK;
  }
  if (!ctx->graphs_valid) {
    int rc = build_graphs(ctx);
    if (rc) return rc;
  }
  for (int n = 0; n < coarse_steps; ++n) {
    CK(cudaGraphLaunch(ctx->graph[ctx->parity0], ctx->stream));
    ctx->parity0 ^= 1;
    ctx->step++;
  }
  return LBM_OK;
}

int lbm_sync(lbm_ctx* ctx) {
  if (!ctx) return LBM_ERR_ARG;
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  return LBM_OK;
}

int lbm_macroscopic(lbm_ctx* ctx, int level, double* rho, double* u) {
  if (!ctx || !rho || !u) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  double* hout[4] = {rho, u, u + n, u + 2 * n};
  return slab_transfer(ctx, level, SLAB_MACRO, nullptr, hout, 4);
}

int lbm_stats_reset(lbm_ctx* ctx) {
  if (!ctx) return LBM_ERR_ARG;
  for (int l = 0; l < ctx->L; ++l) {
    const size_t bytes = size_t(ctx->plan.lv[l].nblocks()) * 512 * 7 * sizeof(double);
    if (!ctx->dl[l].stats) {
      cudaError_t e = cudaMalloc(&ctx->dl[l].stats, bytes);
      if (e != cudaSuccess) return fail(ctx, LBM_ERR_OOM, std::string("statistics: ") + cudaGetErrorString(e));
    }
    CK(cudaMemsetAsync(ctx->dl[l].stats, 0, bytes, ctx->stream));
  }
  ctx->stats_n = 0;
  return LBM_OK;
}

int lbm_stats_accumulate(lbm_ctx* ctx) {
  if (!ctx) return LBM_ERR_ARG;
  if (!ctx->dl[0].stats) return fail(ctx, LBM_ERR_STATE, "call lbm_stats_reset first");
  for (int l = 0; l < ctx->L; ++l) {
    StatsArgs a{};
    a.f = ctx->dl[l].f[cur_parity(ctx, l)];
    a.kind = ctx->dl[l].kind;
    a.ncells = ctx->plan.lv[l].nblocks() * 512;
    a.sums = ctx->dl[l].stats;
    CK(launch_stats(ctx->model, ctx->storage, a, ctx->stream));
  }
  ctx->stats_n++;
  return LBM_OK;
}

int lbm_stats_get(lbm_ctx* ctx, int level, double* mean, double* var, int64_t* nsamples) {
  if (!ctx || !mean || !var) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  if (!ctx->dl[0].stats || ctx->stats_n == 0) return fail(ctx, LBM_ERR_STATE, "no samples accumulated");
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  double* hout[7] = {mean, mean + n, mean + 2 * n, mean + 3 * n, var, var + n, var + 2 * n};
  if (nsamples) *nsamples = ctx->stats_n;
  return slab_transfer(ctx, level, SLAB_GET_STATS, nullptr, hout, 7, nullptr, ctx->dl[level].stats,
                       1.0 / double(ctx->stats_n));
}

int lbm_stats_radial(lbm_ctx* ctx, int level, double y0, double z0, double dr, int nbins, int nstations,
                     const double* x, double* mean_ux, double* var_ux, int64_t* counts) {
  if (!ctx || !x || !mean_ux || !var_ux || !counts) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < -1 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  if (!std::isfinite(y0) || !std::isfinite(z0) || !std::isfinite(dr))
    return fail(ctx, LBM_ERR_NONFINITE, "non-finite profile parameter");
  if (!(dr > 0) || nbins < 1 || nstations < 1 || int64_t(nbins) * nstations > (int64_t(1) << 24))
    return fail(ctx, LBM_ERR_ARG, "need dr > 0, nbins >= 1, nstations >= 1");
  if (!ctx->dl[0].stats || ctx->stats_n == 0) return fail(ctx, LBM_ERR_STATE, "no samples accumulated");
  // one level, or every level's unrefined cells weighted by their area
  const int l0 = level < 0 ? 0 : level, l1 = level < 0 ? ctx->L - 1 : level;
  std::vector<int> xs(static_cast<size_t>(nstations) * (l1 - l0 + 1));
  for (int l = l0; l <= l1; ++l)
    for (int s = 0; s < nstations; ++s) {
      if (!std::isfinite(x[s])) return fail(ctx, LBM_ERR_NONFINITE, "non-finite station");
      const double X = std::floor(std::ldexp(x[s], l));
      if (X < 0 || X >= ctx->plan.lv[l].NX) return fail(ctx, LBM_ERR_ARG, "station outside the level");
      xs[size_t(l - l0) * nstations + s] = int(X);
    }
  const size_t nb = size_t(nbins) * nstations;
  double* acc = nullptr;
  unsigned long long* cnt = nullptr;
  int* dxs = nullptr;
  cudaError_t e = cudaMalloc(&acc, nb * 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, nb * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&dxs, xs.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, nb * 3 * sizeof(double), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, nb * sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dxs, xs.data(), xs.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->stream);
  for (int l = l0; l <= l1 && e == cudaSuccess; ++l) {
    const LevelPlan& lp = ctx->plan.lv[l];
    RadialArgs a{};
    a.sums = ctx->dl[l].stats;
    a.kind = ctx->dl[l].kind;
    a.ox = lp.ox;
    a.oy = lp.oy;
    a.oz = lp.oz;
    a.BX = lp.BX;
    a.BY = lp.BY;
    a.BZ = lp.BZ;
    a.NY = lp.NY;
    a.NZ = lp.NZ;
    a.xs = dxs + size_t(l - l0) * nstations;
    a.nst = nstations;
    a.nbins = nbins;
    a.y0 = y0;
    a.z0 = z0;
    a.dr = dr;
    a.inv_scale = std::ldexp(1.0, -l);
    a.scale = 1.0 / double(ctx->stats_n);
    a.weight = level < 0 ? std::ldexp(1.0, -2 * l) : 1.0;
    a.active_only = level < 0 ? 1 : 0;
    a.acc = acc;
    a.cnt = cnt;
    e = launch_radial(a, ctx->stream);
  }
  std::vector<double> hacc(nb * 3);
  std::vector<unsigned long long> hcnt(nb);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hacc.data(), acc, nb * 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hcnt.data(), cnt, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(acc);
  cudaFree(cnt);
  cudaFree(dxs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "radial profile");
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (size_t o = 0; o < nb; ++o) {
    counts[o] = int64_t(hcnt[o]);
    mean_ux[o] = hcnt[o] ? hacc[3 * o] / hacc[3 * o + 2] : nan;
    var_ux[o] = hcnt[o] ? hacc[3 * o + 1] / hacc[3 * o + 2] : nan;
  }
  return LBM_OK;
}

int lbm_jet_fit(int nbins, double dr, const double* mean_ux, const double* var_ux, const int64_t* counts,
                double out[5]) {
  if (!mean_ux || !var_ux || !counts || !out || nbins < 1 || !(dr > 0)) return LBM_ERR_ARG;
  const double nan = std::numeric_limits<double>::quiet_NaN();
  for (int k = 0; k < 5; ++k) out[k] = nan;
  if (counts[0] == 0 || !(mean_ux[0] > 0)) return LBM_OK;
  const double um = mean_ux[0];
  out[0] = um;
  out[2] = std::sqrt(std::max(var_ux[0], 0.0)) / um;
  // half width: first ring at or below u_m / e, linear between ring centres
  const double lev = um / std::exp(1.0);
  double be = nan;
  for (int b = 1; b < nbins; ++b) {
    if (counts[b] == 0 || counts[b - 1] == 0) continue;
    if (mean_ux[b] <= lev) {
      be = (b - 0.5) * dr + (mean_ux[b - 1] - lev) / (mean_ux[b - 1] - mean_ux[b]) * dr;
      break;
    }
  }
  if (!std::isfinite(be)) return LBM_OK;
  out[1] = be;
  // least squares of ln(u / u_m) against (r / b_e)^2
  double n = 0, sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (int b = 0; b < nbins; ++b) {
    const double r = (b + 0.5) * dr;
    if (counts[b] > 0 && mean_ux[b] >= 0.05 * um && r <= 2.0 * be) {
      const double X = (r / be) * (r / be), Y = std::log(mean_ux[b] / um);
      n += 1;
      sx += X;
      sy += Y;
      sxx += X * X;
      sxy += X * Y;
    }
  }
  const double den = n * sxx - sx * sx;
  if (n < 2 || den == 0) return LBM_OK;
  const double slope = (n * sxy - sx * sy) / den;
  out[3] = std::exp((sy - slope * sx) / n);
  out[4] = -slope;
  return LBM_OK;
}

int lbm_mass_momentum(lbm_ctx* ctx, double out[4]) {
  if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  const int ctas = reduce_ctas_per_sm(ctx->storage) * ctx->sms;  // one wave of the audit kernel
  for (int l = 0; l < ctx->L; ++l) {
    ReduceArgs a{};
    a.f = ctx->dl[l].f[cur_parity(ctx, l)];
    a.kind = ctx->dl[l].kind;
    a.ncells = ctx->plan.lv[l].nblocks() * 512;
    a.vol = std::ldexp(1.0, -3 * l);
    a.partial = ctx->partial + size_t(l) * ctas * 4;
    CK(launch_reduce(ctx->model, ctx->storage, a, ctas, ctx->stream));
  }
  CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->stream));
  CK(launch_reduce_final(ctx->partial, ctas * ctx->L, ctx->d_out, ctx->d_flag, ctx->stream));
  int flag = 0;
  CK(cudaMemcpyAsync(out, ctx->d_out, 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (flag) return fail(ctx, LBM_ERR_NONFINITE, "NaN or Inf in the distributions");
  return LBM_OK;
}

int lbm_get_state(lbm_ctx* ctx, int level, double* f, size_t count) {
  if (!ctx || !f) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  if (count != size_t(ctx->Q) * lp.NX * lp.NY * lp.NZ) return fail(ctx, LBM_ERR_ARG, "count mismatch");
  std::vector<double*> hout(ctx->Q);
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  for (int i = 0; i < ctx->Q; ++i) hout[i] = f + i * n;
  return slab_transfer(ctx, level, SLAB_GET_STATE, nullptr, hout.data(), ctx->Q);
}

int lbm_set_state(lbm_ctx* ctx, int level, const double* f, size_t count) {
  if (!ctx || !f) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  if (count != size_t(ctx->Q) * lp.NX * lp.NY * lp.NZ) return fail(ctx, LBM_ERR_ARG, "count mismatch");
  for (size_t i = 0; i < count; ++i)
    if (std::isinf(f[i])) return fail(ctx, LBM_ERR_NONFINITE, "infinite value in state");
  std::vector<const double*> hin(ctx->Q);
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  for (int i = 0; i < ctx->Q; ++i) hin[i] = f + i * n;
  int rc = slab_transfer(ctx, level, SLAB_SET_STATE, hin.data(), nullptr, ctx->Q);
  if (rc) return rc;
  ctx->need_restrict = false;
  return LBM_OK;
}

int lbm_raw_state_bytes(const lbm_ctx* ctx, int level, size_t* bytes) {
  if (!ctx || !bytes || level < 0 || level >= ctx->L) return LBM_ERR_ARG;
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t fb = size_t(lp.nblocks()) * 512 * ctx->Q * storage_bytes(ctx->storage);
  const size_t ab = ctx->dl[level].aux[0] ? size_t(lp.nblocks()) * 512 * real_bytes(ctx->storage) : 0;
  *bytes = fb + ab;
  return LBM_OK;
}

int lbm_get_raw_state(lbm_ctx* ctx, int level, void* buf, size_t bytes) {
  size_t need = 0;
  if (lbm_raw_state_bytes(ctx, level, &need) != LBM_OK || !buf) return fail(ctx, LBM_ERR_ARG, "bad argument");
  if (bytes != need) return fail(ctx, LBM_ERR_ARG, "bytes must equal lbm_raw_state_bytes");
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t fb = size_t(lp.nblocks()) * 512 * ctx->Q * storage_bytes(ctx->storage);
  const int p = cur_parity(ctx, level);
  CK(cudaMemcpyAsync(buf, ctx->dl[level].f[p], fb, cudaMemcpyDeviceToHost, ctx->stream));
  if (need > fb)
    CK(cudaMemcpyAsync(static_cast<char*>(buf) + fb, ctx->dl[level].aux[p], need - fb, cudaMemcpyDeviceToHost,
                       ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

int lbm_set_raw_state(lbm_ctx* ctx, int level, const void* buf, size_t bytes) {
  size_t need = 0;
  if (lbm_raw_state_bytes(ctx, level, &need) != LBM_OK || !buf) return fail(ctx, LBM_ERR_ARG, "bad argument");
  if (bytes != need) return fail(ctx, LBM_ERR_ARG, "bytes must equal lbm_raw_state_bytes");
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t fb = size_t(lp.nblocks()) * 512 * ctx->Q * storage_bytes(ctx->storage);
  const int p = cur_parity(ctx, level);
  CK(cudaMemcpyAsync(ctx->dl[level].f[p], buf, fb, cudaMemcpyHostToDevice, ctx->stream));
  if (need > fb)
    CK(cudaMemcpyAsync(ctx->dl[level].aux[p], static_cast<const char*>(buf) + fb, need - fb,
                       cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->need_restrict = false;
  return LBM_OK;
}

int lbm_get_strain(lbm_ctx* ctx, int level, double* S, size_t count) {
  if (!ctx || !S) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  if (count != size_t(lp.NX) * lp.NY * lp.NZ) return fail(ctx, LBM_ERR_ARG, "count mismatch");
  void* aux = ctx->dl[level].aux[cur_parity(ctx, level)];
  if (!aux) {
    for (size_t i = 0; i < count; ++i) S[i] = 0.0;
    return LBM_OK;
  }
  double* hout[1] = {S};
  return slab_transfer(ctx, level, SLAB_GET_AUX, nullptr, hout, 1, nullptr, aux);
}

int lbm_set_strain(lbm_ctx* ctx, int level, const double* S, size_t count) {
  if (!ctx || !S) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  const LevelPlan& lp = ctx->plan.lv[level];
  if (count != size_t(lp.NX) * lp.NY * lp.NZ) return fail(ctx, LBM_ERR_ARG, "count mismatch");
  void* aux = ctx->dl[level].aux[cur_parity(ctx, level)];
  if (!aux) return LBM_OK;
  for (size_t i = 0; i < count; ++i)
    if (std::isinf(S[i])) return fail(ctx, LBM_ERR_NONFINITE, "infinite strain value");
  const double* hin[1] = {S};
  return slab_transfer(ctx, level, SLAB_SET_AUX, hin, nullptr, 1, nullptr, aux);
}

int lbm_get_cells(lbm_ctx* ctx, int level, size_t n, const int64_t* cells, double* f) {
  if (!ctx || (n && (!cells || !f))) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (level < 0 || level >= ctx->L) return fail(ctx, LBM_ERR_ARG, "level out of range");
  if (n == 0) return LBM_OK;
  const LevelPlan& lp = ctx->plan.lv[level];
  const size_t bytes = n * sizeof(long long) + n * ctx->Q * sizeof(double);
  int rc = ensure_stage(ctx, bytes + 16);
  if (rc) return rc;
  long long* dc = reinterpret_cast<long long*>(ctx->stage);
  double* dout = ctx->stage + n;
  CK(cudaMemcpyAsync(dc, cells, n * sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
  GatherArgs a{};
  a.f = ctx->dl[level].f[cur_parity(ctx, level)];
  a.ox = lp.ox;
  a.oy = lp.oy;
  a.oz = lp.oz;
  a.BX = lp.BX;
  a.BY = lp.BY;
  a.BZ = lp.BZ;
  a.NX = lp.NX;
  a.NY = lp.NY;
  a.NZ = lp.NZ;
  a.cells = dc;
  a.n = (long long)n;
  a.out = dout;
  CK(launch_gather(ctx->model, ctx->storage, a, ctx->stream));
  CK(cudaMemcpyAsync(f, dout, n * ctx->Q * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

int lbm_get_step(const lbm_ctx* ctx, int64_t* step) {
  if (!ctx || !step) return LBM_ERR_ARG;
  *step = ctx->step;
  return LBM_OK;
}

int lbm_set_step(lbm_ctx* ctx, int64_t step) {
  if (!ctx) return LBM_ERR_ARG;
  if (step < 0) return fail(ctx, LBM_ERR_ARG, "step must be >= 0");
  long long s = step;
  CK(cudaMemcpyAsync(ctx->d_step, &s, sizeof(s), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->step = step;
  return LBM_OK;
}

int lbm_set_profiling(lbm_ctx* ctx, int enable) {
  if (!ctx) return LBM_ERR_ARG;
  ctx->profiling = enable != 0;
  for (int k = 0; k < 5; ++k) {
    ctx->prof_ms[k] = 0;
    ctx->prof_n[k] = 0;
  }
  return LBM_OK;
}

int lbm_get_profile(lbm_ctx* ctx, double ms[5], int64_t launches[5]) {
  if (!ctx || !ms || !launches) return LBM_ERR_ARG;
  for (int k = 0; k < 5; ++k) {
    ms[k] = ctx->prof_ms[k];
    launches[k] = ctx->prof_n[k];
  }
  return LBM_OK;
}

int lbm_adjoint_forward(lbm_ctx* ctx, int T, int checkpoint_every) {
  if (!ctx) return LBM_ERR_ARG;
  if (ctx->model != LBM_D3Q27_FCLB || ctx->L != 1 || !ctx->plan.periodic_x)
    return fail(ctx, LBM_ERR_STATE, "the adjoint is defined for single-level periodic D3Q27 grids");
  if (ctx->plan.walls || ctx->plan.nozzle_level >= 0)
    return fail(ctx, LBM_ERR_STATE, "the adjoint is defined without walls or a nozzle");
  if (ctx->storage == LBM_F16) return fail(ctx, LBM_ERR_STATE, "the adjoint needs F32 or F64 storage");
  if (T < 1 || checkpoint_every < 0 || checkpoint_every > T)
    return fail(ctx, LBM_ERR_ARG, "need T >= 1 and 0 <= checkpoint_every <= T");
  const LevelPlan& lp = ctx->plan.lv[0];
  const size_t sb = size_t(lp.nblocks()) * 512 * 27 * storage_bytes(ctx->storage);
  const size_t gb = size_t(lp.nblocks()) * 512 * 3 * real_bytes(ctx->storage);
  int every = checkpoint_every;
  if (every == 0) {
    // keep every state when T of them (plus the two adjoint buffers) fit in
    // half of the free device memory, counting what the adjoint already holds
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    size_t held = ctx->adj_gF ? gb : 0;
    for (void* p : ctx->adj_ck) held += p ? ctx->adj_state_bytes : 0;
    for (void* p : ctx->adj_seg) held += p ? ctx->adj_state_bytes : 0;
    for (void* p : ctx->adj_lam) held += p ? ctx->adj_state_bytes : 0;
    every = (double(T) + 2.0) * double(sb) + double(gb) <= 0.5 * double(fr + held)
                ? 1
                : std::max(1, int(std::ceil(std::sqrt(double(T)))));
  }
  const int nck = (T + every - 1) / every;
  if (ctx->adj_state_bytes != sb || int(ctx->adj_ck.size()) < nck || int(ctx->adj_seg.size()) < every) {
    CK(cudaStreamSynchronize(ctx->stream));
    release_adjoint(ctx);
    // LBM_INJECT_ADJOINT_OOM=k makes the k-th buffer allocation below fail on
    // the host, as cudaMalloc would when the device is full (tests of the
    // failure path; no device fault is involved)
    int inject = 0;
    if (const char* e = std::getenv("LBM_INJECT_ADJOINT_OOM")) inject = std::atoi(e);
    int grabs = 0;
    auto grab = [&](void** p, size_t n) -> int {
      cudaError_t e = (inject > 0 && ++grabs == inject) ? cudaErrorMemoryAllocation : cudaMalloc(p, n);
      if (e != cudaSuccess) {
        // nothing half-allocated stays behind: the next call starts afresh
        release_adjoint(ctx);
        return fail(ctx, LBM_ERR_OOM, std::string("adjoint buffers: ") + cudaGetErrorString(e));
      }
      return LBM_OK;
    };
    ctx->adj_ck.assign(nck, nullptr);
    ctx->adj_seg.assign(every, nullptr);
    for (size_t k = 0; k < ctx->adj_ck.size(); ++k)
      if (int rc = grab(&ctx->adj_ck[k], sb)) return rc;
    for (size_t k = 1; k < ctx->adj_seg.size(); ++k)
      if (int rc = grab(&ctx->adj_seg[k], sb)) return rc;
    for (int k = 0; k < 2; ++k)
      if (int rc = grab(&ctx->adj_lam[k], sb)) return rc;
    if (int rc = grab(&ctx->adj_gF, gb)) return rc;
    ctx->adj_state_bytes = sb;
  }
  if (ctx->need_restrict) {
    int rc = restrict_all(ctx);
    if (rc) return rc;
  }
  ctx->adj_ready = false;
  if (every == 1) {
    // every state kept: the update writes step t's input straight into its
    // slot (no copies); the last step writes the context's other buffer
    std::vector<Op> ops = build_schedule(ctx, ctx->parity0);
    UpdateArgs ua{};
    for (const Op& op : ops)
      if (op.kind == Op::UPDATE) ua = op.ua;
    CK(cudaMemcpyAsync(ctx->adj_ck[0], ctx->dl[0].f[ctx->parity0], sb, cudaMemcpyDeviceToDevice, ctx->stream));
    for (int t = 0; t < T; ++t) {
      ua.lv[0].src = ctx->adj_ck[t];
      ua.lv[0].dst = t + 1 < T ? ctx->adj_ck[t + 1] : ctx->dl[0].f[1 - ctx->parity0];
      CK(launch_update(ctx->model, ctx->storage, ua, ctx->threads, ctx->minb, ctx->ctas, ctx->stream));
    }
    ctx->parity0 ^= 1;
    ctx->step += T;
    ctx->step_dev = ctx->step;
    CK(cudaMemcpyAsync(ctx->d_step, &ctx->step_dev, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
  } else {
    if (!ctx->graphs_valid) {
      int rc = build_graphs(ctx);
      if (rc) return rc;
    }
    for (int t = 0; t < T; ++t) {
      if (t % every == 0)
        CK(cudaMemcpyAsync(ctx->adj_ck[t / every], ctx->dl[0].f[ctx->parity0], sb, cudaMemcpyDeviceToDevice,
                           ctx->stream));
      CK(cudaGraphLaunch(ctx->graph[ctx->parity0], ctx->stream));
      ctx->parity0 ^= 1;
      ctx->step++;
    }
  }
  ctx->adj_T = T;
  ctx->adj_every = every;
  ctx->adj_ready = true;
  ctx->adj_gen++;
  return LBM_OK;
}

int lbm_adjoint_generation(const lbm_ctx* ctx, uint64_t* generation, int* checkpoint_every) {
  if (!ctx || !generation) return LBM_ERR_ARG;
  *generation = ctx->adj_ready ? ctx->adj_gen : 0;
  if (checkpoint_every) *checkpoint_every = ctx->adj_ready ? ctx->adj_every : 0;
  return LBM_OK;
}

int lbm_adjoint_backward(lbm_ctx* ctx, const double* dLdf_T, double* dLdF) {
  if (!ctx || !dLdf_T || !dLdF) return fail(ctx, LBM_ERR_ARG, "NULL argument");
  if (!ctx->adj_ready) return fail(ctx, LBM_ERR_STATE, "call lbm_adjoint_forward first");
  const LevelPlan& lp = ctx->plan.lv[0];
  const size_t n = size_t(lp.NX) * lp.NY * lp.NZ;
  if (!all_finite(dLdf_T, 27 * n)) return fail(ctx, LBM_ERR_NONFINITE, "non-finite dL/df_T");
  const size_t rb = real_bytes(ctx->storage);
  // lambda_T into the block layout
  CK(cudaMemsetAsync(ctx->adj_lam[0], 0, ctx->adj_state_bytes, ctx->stream));
  std::vector<const double*> hin(27);
  for (int i = 0; i < 27; ++i) hin[i] = dLdf_T + i * n;
  int rc = slab_transfer(ctx, 0, SLAB_SET_LAMBDA, hin.data(), nullptr, 27, nullptr, ctx->adj_lam[0]);
  if (rc) return rc;
  CK(cudaMemsetAsync(ctx->adj_gF, 0, size_t(lp.nblocks()) * 512 * 3 * rb, ctx->stream));
  // the update launch of the single level, retargeted to segment buffers
  std::vector<Op> ops = build_schedule(ctx, 0);
  UpdateArgs ua{};
  for (const Op& op : ops)
    if (op.kind == Op::UPDATE) ua = op.ua;
  AdjointArgs aa{};
  aa.dLdF = ctx->adj_gF;
  aa.force = !ctx->has_force ? nullptr
             : ctx->storage == LBM_F64 ? static_cast<const void*>(ctx->dl[0].force)
                                        : static_cast<const void*>(ctx->dl[0].force_f);
  aa.BX = lp.BX;
  aa.BY = lp.BY;
  aa.BZ = lp.BZ;
  aa.nblocks = int(lp.nblocks());
  aa.omega = 1.0 / lp.tau0;
  const int T = ctx->adj_T, every = ctx->adj_every;
  const int nck = (T + every - 1) / every;
  int cur = 0;
  cudaEvent_t pe0 = nullptr, pe1 = nullptr;
  if (ctx->profiling) {
    CK(cudaEventCreate(&pe0));
    CK(cudaEventCreate(&pe1));
    CK(cudaEventRecord(pe0, ctx->stream));
  }
  for (int s = nck - 1; s >= 0; --s) {
    const int t0 = s * every, t1 = std::min(T, t0 + every), m = t1 - t0;
    // segment slot 0 is the checkpoint itself; slots 1.. hold the recomputed states
    auto seg = [&](int k) { return k == 0 ? ctx->adj_ck[s] : ctx->adj_seg[k]; };
    for (int k = 0; k + 1 < m; ++k) {
      ua.lv[0].src = seg(k);
      ua.lv[0].dst = seg(k + 1);
      CK(launch_update(ctx->model, ctx->storage, ua, ctx->threads, ctx->minb, ctx->ctas, ctx->stream));
    }
    for (int k = m - 1; k >= 0; --k) {
      aa.f_t = seg(k);
      aa.lam_in = ctx->adj_lam[cur];
      aa.lam_out = ctx->adj_lam[1 - cur];
      CK(launch_adjoint(ctx->storage, aa, ctx->stream));
      cur ^= 1;
    }
  }
  if (ctx->profiling) {
    CK(cudaEventRecord(pe1, ctx->stream));
    CK(cudaEventSynchronize(pe1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, pe0, pe1));
    ctx->prof_ms[4] += ms;
    ctx->prof_n[4] += 1;
    cudaEventDestroy(pe0);
    cudaEventDestroy(pe1);
  }
  double* hout[3] = {dLdF, dLdF + n, dLdF + 2 * n};
  return slab_transfer(ctx, 0, SLAB_GET_FIELD3, nullptr, hout, 3, nullptr, ctx->adj_gF);
}

int lbm_get_tuning(const lbm_ctx* ctx, int* threads, int* min_ctas_per_sm, int* ctas) {
  if (!ctx || !threads || !min_ctas_per_sm || !ctas) return LBM_ERR_ARG;
  *threads = ctx->threads;
  *min_ctas_per_sm = ctx->minb;
  *ctas = ctx->ctas;
  return LBM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ access for the sharded grid (shard.cu)
namespace lbm {
void set_create_error(const std::string& m) { g_create_error = m; }
const GridPlan& ctx_plan(const lbm_ctx* c) { return c->plan; }
void* ctx_level0_buffer(lbm_ctx* c) { return c->dl[0].f[c->parity0]; }
cudaStream_t ctx_stream(const lbm_ctx* c) { return c->stream; }
}  // namespace lbm
