// Launch-parameter structures shared by the host side and the kernels, and
// the host-callable launchers (implemented in the .cu files).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lbm.h"

namespace lbm {

constexpr int kCells = 512;  // cells per 8^3 block, index x + 8 y + 64 z
constexpr int kMaxL = LBM_MAX_LEVELS;

// one unit of stream-collide work: a block of one level, optionally masked.
// edges: bit 2a (2a+1) set when the block sits on the low (high) face of a
// level box that wraps periodically along axis a (x, y, z); bit 6 set when
// its +x face is the zero-gradient outflow x = NX (the populations entering
// through it are pulled from the cell x = NX - 1 itself); bit 7 set for a
// level-0 block whose -x face is the domain face x = 0 when that face is a
// wall.
struct WorkItem {
  int32_t block;
  uint8_t level;
  uint8_t edges;
  int16_t mask;  // -1: all 512 cells; else index into the mask table
};

// cell kinds kept per level on the device (for outputs and audits)
enum CellKind : uint8_t {
  K_NONE = 0,     // allocated but holds no value of the level
  K_ACTIVE = 1,   // unrefined cell of the level
  K_HIDDEN1 = 2,  // refined, Chebyshev distance 1 from an active cell
  K_HIDDEN2 = 3,  // refined, distance 2
  K_REFINED = 4,  // refined, deeper inside
  K_GHOST = 5,    // coarse-to-fine ghost cell
  K_BC = 6,       // inflow/outflow ghost cell
  K_SOLID = 7,    // inside the nozzle (not updated; its link populations are set)
  K_HALO = 8      // halo column of a sharded part: a copy of the neighbouring part
};

struct LevelPtrs {
  const void* src;    // storage [nblocks][Q][512], nblocks = BX*BY*BZ
  void* dst;
  void* aux_dst;      // |S| per cell [nblocks][512] (real) or nullptr
  int BX, BY, BZ;     // level box in blocks
  double tau0;
};

struct UpdateArgs {
  LevelPtrs lv[kMaxL];
  const WorkItem* items;
  int nitems;
  const uint32_t* masks;  // 16 words per mask
  double cs2_18;          // 18 Cs^2
  const void* force;      // level 0 body force [3][nblocks*512] (block order) in the
                          // compute type (double for F64 storage, else float) or nullptr
  int walls, slip;        // level-0 wall faces (bit 0/1 low/high y, 2/3 low/high z, 4/5
                          // the faces x = 0 / x = NX, no-slip) and the free-slip ones
                          // among the y/z walls; read by the W = true kernels
  int pf_ahead;           // FP16 kernels: a CTA asks L2 for the block of work item
                          // it + pf_ahead (about half a wave ahead); 0 = off (set by
                          // the launcher)
};

// coarse-to-fine work comes in chunks of consecutive ghost cells (sorted by
// their coarse stencil); a chunk lists its distinct coarse stencil cells once
// (sorted by address), one CTA stages their values in shared memory, and the
// items index that list
struct C2FChunk {
  int32_t first_item;
  int32_t first_cell;
  int16_t nitems;
  int16_t ncells;
};
struct C2FCell {
  int32_t cblock;
  int16_t ccell;
  int16_t pad;
};
struct C2FItem {
  int32_t fblock;
  int16_t fcell;
  uint8_t tbits;      // bit a: weight of the upper coarse index along axis a is 3/4 (else 1/4)
  uint8_t pad;
  uint32_t need;      // bit i: population i is pulled by an updated cell of the level
  uint16_t slot[8];   // stencil cells (dz, dy, dx order, dx fastest; 0 = lower,
                      // 1 = upper index) as indices into the chunk's cell list
  int32_t bc;         // the inflow ghost that takes its density from this ghost
                      // cell (index into the level's c2f_bc list), or -1
};
// chunk limits (distinct cells x Q values of the compute type stay at 27 KB
// of shared memory)
__host__ __device__ constexpr int c2f_max_cells(int storage) { return storage == LBM_F64 ? 128 : 256; }
constexpr int kC2FMaxItems = 128;  // = threads per CTA
// resident 256-thread CTAs per SM of the float64 audit (one wave): three for
// FP16 storage (0.373 -> 0.351 ms per 256^3 D3Q27 call), two otherwise
// (three cost FP32 8 %)
__host__ __device__ constexpr int reduce_ctas_per_sm(int storage) { return storage == LBM_F16 ? 3 : 2; }

// fine-to-coarse: one hidden coarse cell and its 8 children as 4 x-pairs
// (pair p = dy + 2 dz): the children (2X, ...) at fcell[p] and (2X+1, ...) at
// fcell[p] + 1 of block fblock[p]; fcell[p] is even, so a pair is one aligned
// two-element load
struct F2CItem {
  int32_t cblock;
  int16_t ccell;
  int16_t pad;
  int32_t fblock[4];
  int16_t fcell[4];
};

// boundary ghost cell
struct BCItem {
  int32_t gblock;
  int16_t gcell;
  int8_t type;  // 0 inflow (x = -1): the populations with e_x = +1 are
                // written; 1 pressure outlet (x = NX): those with e_x = -1
  int8_t pad;
  int32_t sblock;
  int16_t scell;
  int16_t pad2;
  int32_t y, z;  // level-local cell coordinates of the face cell
};

// The interface and boundary launches each cover every level that needs the
// transfer at that point of the schedule (they touch disjoint cells); level
// j of a launch owns items [sum_{k<j} n_k, sum_{k<=j} n_k).
struct C2FLevel {
  const C2FChunk* chunks;
  const C2FItem* items;
  const C2FCell* cells;
  const BCItem* bc;   // inflow ghosts whose source is a ghost cell of this level
  int n;              // chunks
  int s;              // fine substep 0 or 1
  int level, substep, NY;  // for those inflow ghosts (substep = index within the coarse step)
  double inv_scale;        // 2^-level
  const void* c_old;  // coarse storage at t
  const void* c_new;  // coarse storage at t+1 (used when s == 1)
  const void* a_old;  // coarse |S| at t (LES) or nullptr
  const void* a_new;
  void* f_dst;        // fine storage receiving the ghost values
  void* fa_dst;       // fine |S| (LES) or nullptr
  double tau0_c, tau0_f;
};
struct C2FArgs {
  C2FLevel lv[kMaxL];
  int nlv;
  int n;           // chunks of all levels
  double cs2_3;    // 3 Cs^2
  const long long* step;  // inflow (see BCArgs)
  double y0, z0, r2, u_in, perturb;
  unsigned long long seed;
  int closed;             // the face inflow holds u = 0 (the inflow sits on the nozzle's cap)
};

struct F2CLevel {
  const F2CItem* items;
  int n;
  const void* f_src;  // fine storage at t+1
  const void* fa_src;
  void* c_dst;        // coarse storage at t+1
  void* ca_dst;
  double tau0_c, tau0_f;
};
struct F2CArgs {
  F2CLevel lv[kMaxL];
  int nlv;
  int n;
  double cs2_3;
};

struct BCLevel {
  const BCItem* items;
  int n;
  void* f;  // level storage at the current time (ghosts written in place)
  int level, substep, NY;
  double inv_scale;  // 2^-level
};
struct BCArgs {
  BCLevel lv[kMaxL];
  int nlv;
  int n;
  const long long* step;  // device coarse-step counter
  double y0, z0, r2, u_in, perturb;
  unsigned long long seed;
  double rl_out;  // pressure outlet: rho_out - 1 (the density-like value of the storage)
  int closed;     // the face inflow holds u = 0 (the inflow sits on the nozzle's cap)
};

// a link of the nozzle's surface: fluid cell f, direction i towards the solid
// cell b = f + e_i, ib the opposite direction.  type 0 (no-slip, Bouzidi
// linear interpolation at fraction q): population ib of b is set from
// f~_i(f), f~_i(s) with s = f - e_i (sblock < 0: s is solid, half-way
// bounce-back) and f~_ib(f).  type 1 (on the downstream cap): population ib
// of b is f_eq(rho(s), u_bc) with s = b + x^ and u_bc the inflow disc
// velocity at the level-local (y, z) of b.
struct LinkItem {
  double q;
  int32_t fblock, bblock, sblock;
  int16_t fcell, bcell, scell;
  uint8_t i, ib;
  uint8_t type, pad;
  int16_t pad2;
  int32_t y, z;
};
struct LinkArgs {
  const LinkItem* items;
  int n;
  void* f;  // storage of the nozzle's level at the current time
  int level, substep, NY;
  double inv_scale;
  const long long* step;
  double y0, z0, r2, u_in, perturb;
  unsigned long long seed;
};

// ------------------------------------------------------------------ launchers
// model: 0 D3Q19 MRT-LES, 1 D3Q27 FCLB; storage: lbm_storage.
cudaError_t launch_update(int model, int storage, const UpdateArgs& a, int threads, int minb, int ctas,
                          cudaStream_t st);
cudaError_t update_occupancy(int model, int storage, bool walls, int threads, int minb, int* ctas_per_sm);
cudaError_t launch_c2f(int model, int storage, const C2FArgs& a, cudaStream_t st);
cudaError_t launch_f2c(int model, int storage, const F2CArgs& a, cudaStream_t st);
cudaError_t launch_bc(int model, int storage, const BCArgs& a, cudaStream_t st);
cudaError_t launch_links(int model, int storage, const LinkArgs& a, cudaStream_t st);
cudaError_t launch_step_inc(long long* step, cudaStream_t st);

// dense <-> block staging for one slab of cell layers [z0, z0 + nz) of a level
enum SlabMode { SLAB_SET_STATE = 0, SLAB_GET_STATE = 1, SLAB_INIT_EQ = 2, SLAB_MACRO = 3,
                SLAB_SET_FORCE = 4, SLAB_SET_LAMBDA = 5, SLAB_GET_FIELD3 = 6, SLAB_GET_AUX = 7,
                SLAB_SET_AUX = 8, SLAB_GET_STATS = 9 };
struct SlabArgs {
  void* f;                // level storage (current buffer)
  const uint8_t* kind;    // [nblocks][512] cell kinds
  double* force;          // level body force [3][nblocks*512] or nullptr
  int ox, oy, oz, BX, BY, BZ;  // level box
  int NX, NY, z0, nz;
  const double* in;       // SET_STATE: f [Q][n]; INIT_EQ: rho [n], u [3][n]; SET_FORCE: F [3][n]
  double* out;            // GET_STATE: f [Q][n]; MACRO: rho [n], u [3][n]
  int mode;
  void* raw;              // SET_LAMBDA: [block][Q][512] (compute type); GET_FIELD3: [3][nblocks*512];
                          // GET_STATS: the statistics sums [7][nblocks*512] (double)
  double scale;           // GET_STATS: 1 / number of samples
};

// time statistics of a level: sums over samples of rho, u_x, u_y, u_z,
// u_x^2, u_y^2, u_z^2 per cell ([7][nblocks*512], block order, float64)
struct StatsArgs {
  const void* f;
  const uint8_t* kind;
  long long ncells;  // nblocks * 512
  double* sums;
};
cudaError_t launch_stats(int model, int storage, const StatsArgs& a, cudaStream_t st);

// ring sums of the time mean and variance of u_x on cross-sections x = const
// of one level: thread per (station, y, z) cell; float64 atomics of the
// weighted mean, weighted variance and weight into acc[station][ring][3] and
// the cell count into cnt[station][ring]
struct RadialArgs {
  const double* sums;     // statistics sums [7][nblocks*512]
  const uint8_t* kind;
  int ox, oy, oz, BX, BY, BZ;
  int NY, NZ;
  const int* xs;          // level cell x of each station
  int nst, nbins;
  double y0, z0, dr, inv_scale, scale;  // scale = 1 / samples
  double weight;          // per cell (the cross-section area 4^-level over all levels, else 1)
  int active_only;        // 1: unrefined cells only (all levels), 0: every cell holding a value
  double* acc;
  unsigned long long* cnt;
};
cudaError_t launch_radial(const RadialArgs& a, cudaStream_t st);
cudaError_t launch_slab(int model, int storage, const SlabArgs& a, cudaStream_t st);
cudaError_t launch_fill(double* p, long long n, double v, cudaStream_t st);
// float copy of a float64 array (the compute-type body force of FP32/FP16 storage)
cudaError_t launch_to_float(const double* in, float* out, long long n, cudaStream_t st);

struct GatherArgs {
  const void* f;
  int ox, oy, oz, BX, BY, BZ;
  int NX, NY, NZ;
  const long long* cells;
  long long n;
  double* out;  // [n][Q]
};
cudaError_t launch_gather(int model, int storage, const GatherArgs& a, cudaStream_t st);

// one adjoint step of a periodic single-level D3Q27 grid (adjoint.cu)
struct AdjointArgs {
  const void* f_t;      // post-collision state at t, [nblocks][27][512] (compute type)
  const void* lam_in;   // lambda_{t+1}, same layout
  void* lam_out;        // lambda_t
  void* dLdF;           // [3][nblocks*512] accumulator (compute type)
  const void* force;    // [3][nblocks*512] in the compute type, or nullptr
  int BX, BY, BZ, nblocks;
  double omega;
};
cudaError_t launch_adjoint(int storage, const AdjointArgs& a, cudaStream_t st);

struct ReduceArgs {
  const void* f;
  const uint8_t* kind;
  long long ncells;  // nblocks * 512
  double vol;
  double* partial;   // [gridDim][4]
};
cudaError_t launch_reduce(int model, int storage, const ReduceArgs& a, int ctas, cudaStream_t st);
cudaError_t launch_reduce_final(const double* partial, int n, double* out, int* nonfinite,
                                cudaStream_t st);

}  // namespace lbm
