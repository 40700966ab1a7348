// Fused pull-stream + collide kernel (one launch covers the work of every
// level that takes a substep at that time).
//
// f(x, t+1) = f~(x - e_i, t) (the streaming on the left of Eqs. lbgk / MRT),
// then the local collision of Section 2, then f~(x, t+1) is stored.
// Storage per level: a dense box of 8^3 blocks, [block][i][512 cells], cell
// index x + 8 y + 64 z.  A warp covers four x-rows of one block, so loads of
// one population are 128-byte (F32) contiguous runs, shifted by one cell for
// populations with e_x != 0.
//
// Neighbour blocks are found arithmetically in the level box: per thread the
// extra element offset for leaving the block along -x is Xm (non-zero only
// for cells with x == 0), along +x Xp (x == 7), likewise Ym/Yp/Zm/Zp, so the
// source of population i is own_block + i*512 + cell - (e_x + 8 e_y + 64 e_z)
// + X(e_x) + Y(e_y) + Z(e_z) with X(+1) = Xm, X(-1) = Xp, X(0) = 0.  On the
// zero-gradient outflow face (Xp = -1 for x == 7) the ghost copy of cell
// (NX - 1, y', z') is read from that cell directly.
//
// Walls (instances with W = true): a pull of a level-0 cell that would cross
// a wall face of the domain (y, z, or the no-slip x faces) is replaced after
// the periodic pull, for the cells next to a wall only.  No-slip (half-way
// bounce-back): f_i(x) = f~_opp(i)(x), the opposite population of the cell
// itself.  Free-slip (specular reflection): the population with the
// wall-normal components flipped, pulled along the axes not crossed only,
// f_i(x) = f~_m(i)(x - e_i + (e_i . n) n).  A no-slip crossing wins over a
// free-slip one; two free-slip crossings flip both components.  Opposite and
// mirrored populations have the same weight, so the storage decode of i
// applies to them unchanged.
#pragma once
#include <algorithm>
#include <type_traits>

#include "collide.cuh"
#include "kernels.cuh"
#include "pair.cuh"

namespace lbm {

// read-only half load that asks L2 to fetch the surrounding 256 bytes
__device__ __forceinline__ __half ldg_half_l2(const __half* p) {
  unsigned short v;
  asm("ld.global.nc.L2::256B.b16 %0, [%1];" : "=h"(v) : "l"(p));
  return __ushort_as_half(v);
}
// the same for float storage (the pulls of a warp's next rows then find
// their sectors in L2: 0.5225 -> 0.5203 ms per 256^3 D3Q27 FP32 step)
__device__ __forceinline__ float ldg_f32_l2(const float* p) {
  float v;
  asm("ld.global.nc.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

template <class M, class S, int TPB, int MINB, bool W>
__global__ void __launch_bounds__(TPB, MINB) k_update(const UpdateArgs a) {
  using St = Store<S>;
  using T = typename St::T;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  // FP16 storage holds (f_i - w_i) / w_i: the collision takes and returns
  // that form directly (the weights fold into its constants)
  constexpr bool kScaled = std::is_same<S, __half>::value;
  // FP16 D3Q19 prefetches the next cell (fits in 64 registers; measured
  // 0.79 -> 0.81 of the copy peak); the D3Q27 collision has no registers to
  // spare for it (the prefetch spills and runs 25 % slower)
  constexpr bool kPipeline = kScaled && Q == 19;
  // FP16 D3Q27 instead prefetches the next cells into L2 (0.78 -> 0.80 of
  // the copy peak; on the FP32 kernels, already HBM-bound, it gained nothing)
  constexpr bool kPrefetch = kScaled && !kPipeline;
  const int pf_lane = threadIdx.x & 31;  // the population this lane prefetches
  int pf_shift = 0;                      // its in-block pull shift e_x + 8 e_y + 64 e_z
  static_for<Q>([&](auto i) {
    if (pf_lane == int(i)) pf_shift = Lattice<Q>::ex(i) + 8 * Lattice<Q>::ey(i) + 64 * Lattice<Q>::ez(i);
  });
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const WorkItem w = a.items[it];
    const LevelPtrs& L = a.lv[w.level];
    const int BX = L.BX, BXY = L.BX * L.BY;
    // block deltas towards -x, +x, -y, +y (periodic wrap on box faces); the
    // planner keeps BX * BY * Q * 512 below 2^31, so x and y offsets fit an
    // int.  A wrap across z moves by up to nblocks * Q * 512 elements, past
    // the int range on large boxes: the blocks below and above are reached
    // through 64-bit base pointers instead (the source bases of e_z = +1 pulls
    // of the cells z == 0 and of e_z = -1 pulls of the cells z == 7).
    const int dxm = (w.edges & 1) ? (L.BX - 1) : -1;
    const int dxp = (w.edges & 2) ? -(L.BX - 1) : 1;
    const int dym = (w.edges & 4) ? BX * (L.BY - 1) : -BX;
    const int dyp = (w.edges & 8) ? -BX * (L.BY - 1) : BX;
    // (z block deltas in blocks fit an int: the box holds fewer than 2^31
    // blocks; the element offset is widened per cell)
    const int dzm = (w.edges & 16) ? BXY * (L.BZ - 1) : -BXY;
    const int dzp = (w.edges & 32) ? -BXY * (L.BZ - 1) : BXY;
    // wall faces this block touches (bit 0/1 low/high y, 2/3 low/high z):
    // the level-0 box spans the domain in y and z, so its wrapping faces
    // are the walls; the x faces come from edges bits 7 (x = 0) and 6 (the
    // face x = NX, whose fused outflow read the fix-up then replaces)
    const int wf = (W && w.level == 0)
                       ? (a.walls & (((w.edges >> 2) & 15) | ((w.edges & 128) ? 16 : 0) | ((w.edges & 64) ? 32 : 0)))
                       : 0;
    const T tau0 = T(L.tau0);
    const S* __restrict__ src = reinterpret_cast<const S*>(L.src) + int64_t(w.block) * QS;
    S* __restrict__ dst = reinterpret_cast<S*>(L.dst) + int64_t(w.block) * QS;
    // source of population i for cell c: base(e_z) + c + i*512 - (e_x + 8 e_y
    // + 64 e_z) + the x / y block offsets of the faces the pull crosses, with
    // base(0) = src, base(+1) = the block below for z == 0 (else src),
    // base(-1) = the block above for z == 7 (else src)
    auto offsets = [&](int c, int& Xm, int& Xp, int& Ym, int& Yp) {
      const int x = c & 7, y = (c >> 3) & 7;
      Xm = (x == 0) ? dxm * QS + 8 : 0;
      Xp = (x == 7) ? ((w.edges & 64) ? -1 : dxp * QS - 8) : 0;
      Ym = (y == 0) ? dym * QS + 64 : 0;
      Yp = (y == 7) ? dyp * QS - 64 : 0;
    };
    auto zbase = [&](int c, const S*& b1, const S*& bm) {
      const int z = c >> 6;
      b1 = src + c + (z == 0 ? int64_t(dzm) * QS + 512 : int64_t(0));
      bm = src + c + (z == 7 ? int64_t(dzp) * QS - 512 : int64_t(0));
    };
    auto pull = [&](int c, auto&& load) {
      int Xm, Xp, Ym, Yp;
      offsets(c, Xm, Xp, Ym, Yp);
      const S *b1, *bm;
      zbase(c, b1, bm);
      const S* p = src + c;
      static_for<Q>([&](auto i) {
        constexpr int ex = Lattice<Q>::ex(i), ey = Lattice<Q>::ey(i), ez = Lattice<Q>::ez(i);
        constexpr int k = int(i) * kCells - (ex + 8 * ey + 64 * ez);
        int o = 0;
        if constexpr (ex == 1) o += Xm;
        if constexpr (ex == -1) o += Xp;
        if constexpr (ey == 1) o += Ym;
        if constexpr (ey == -1) o += Yp;
        if constexpr (ez == 1) load(i, b1 + o + k);
        else if constexpr (ez == -1) load(i, bm + o + k);
        else load(i, p + o + k);
      });
    };
    auto active = [&](int c) {
      if (w.mask < 0) return true;
      const uint32_t m = __ldg(a.masks + w.mask * 16 + (c >> 5));
      return bool((m >> (c & 31)) & 1u);
    };
    // replaces, for a cell next to a wall face, the populations whose pull
    // crossed it (the periodic pull above read a valid but unused value)
    auto wall_fix = [&](int c, T (&g)[Q]) {
      const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
      const bool yl = (wf & 1) && y == 0, yh = (wf & 2) && y == 7;
      const bool zl = (wf & 4) && z == 0, zh = (wf & 8) && z == 7;
      const bool xl = (wf & 16) && x == 0, xh = (wf & 32) && x == 7;
      if (!(yl || yh || zl || zh || xl || xh)) return;
      int Xm, Xp, Ym, Yp;
      offsets(c, Xm, Xp, Ym, Yp);
      const S *b1, *bm;
      zbase(c, b1, bm);
      const S* p = src + c;
      static_for<Q>([&](auto i) {
        constexpr int ex = Lattice<Q>::ex(i), ey = Lattice<Q>::ey(i), ez = Lattice<Q>::ez(i);
        if constexpr (ex != 0 || ey != 0 || ez != 0) {
          const bool cy = ey == 1 ? yl : ey == -1 ? yh : false;
          const bool cz = ez == 1 ? zl : ez == -1 ? zh : false;
          const bool cx = ex == 1 ? xl : ex == -1 ? xh : false;  // x walls are no-slip
          if (cy || cz || cx) {
            const bool sy = a.slip & (ey == 1 ? 1 : 2), sz = a.slip & (ez == 1 ? 4 : 8);
            const int X = ex == 1 ? Xm : ex == -1 ? Xp : 0;
            const int Y = ey == 1 ? Ym : ey == -1 ? Yp : 0;
            constexpr int ib = Lattice<Q>::index(-ex, -ey, -ez);
            constexpr int iy = Lattice<Q>::index(ex, -ey, ez);
            constexpr int iz = Lattice<Q>::index(ex, ey, -ez);
            constexpr int iyz = Lattice<Q>::index(ex, -ey, -ez);
            // the reflected source: the cell itself (bounce-back), or the
            // pull along the axes not crossed (z pulls from the z base)
            const S* q;
            if (cx || (cy && !sy) || (cz && !sz)) q = p + ib * kCells;
            else if (cy && cz) q = p + (iyz * kCells - ex + X);
            else if (cy) q = (ez == 1 ? b1 : ez == -1 ? bm : p) + (iy * kCells - (ex + 64 * ez) + X);
            else q = p + (iz * kCells - (ex + 8 * ey) + X + Y);
            if constexpr (kScaled) g[i] = __half2float(__ldg(q));
            else g[i] = St::template get<Q, i>(q);
          }
        }
      });
    };
    auto collide_store = [&](int c, T (&g)[Q]) {
      if constexpr (Q == 19) {
        const T S_ = collide19<T, kScaled>(g, tau0, T(a.cs2_18));
        if (L.aux_dst) reinterpret_cast<T*>(L.aux_dst)[int64_t(w.block) * kCells + c] = S_;
      } else {
        if (a.force != nullptr && w.level == 0) {
          const int64_t n = int64_t(L.BX) * L.BY * L.BZ * kCells;
          const int64_t j = int64_t(w.block) * kCells + c;
          const T* F = reinterpret_cast<const T*>(a.force);
          collide27_closed<T, true, kScaled>(g, T(1) / tau0, F[j], F[n + j], F[2 * n + j]);
        } else {
          collide27_closed<T, false, kScaled>(g, T(1) / tau0, T(0), T(0), T(0));
        }
      }
      S* q = dst + c;
      static_for<Q>([&](auto i) {
        if constexpr (kScaled) q[int(i) * kCells] = __float2half_rn(g[i]);
        else St::template put<Q, i>(q + int(i) * kCells, g[i]);
      });
    };
    if constexpr (kPipeline) {
      // half-size loads keep half the bytes in flight, so the raw values of
      // the thread's next cell are loaded while this one collides
      __half cur[Q], nxt[Q];
      pull(threadIdx.x, [&](auto i, const S* p) { cur[i] = __ldg(p); });
#pragma unroll 1
      for (int c = threadIdx.x; c < kCells; c += TPB) {
        if (c + TPB < kCells) pull(c + TPB, [&](auto i, const S* p) { nxt[i] = __ldg(p); });
        if (active(c)) {
          T g[Q];
          static_for<Q>([&](auto i) { g[i] = __half2float(cur[i]); });
          if constexpr (W) if (wf) wall_fix(c, g);
          collide_store(c, g);
        }
        static_for<Q>([&](auto i) { cur[i] = nxt[i]; });
      }
    } else {
#pragma unroll 1
      for (int c = threadIdx.x; c < kCells; c += TPB) {
        if constexpr (kPrefetch) {
          // the warp's next cells in this block: lane q asks L2 for the run
          // of population q they pull (one instruction per warp, no
          // registers held), so the next loads wait on L2, not DRAM
          const int cn = (c & ~31) + TPB;
          if (pf_lane < Q && cn < kCells) {
            int sc = cn - pf_shift;
            sc = sc < 0 ? 0 : sc > kCells - 1 ? kCells - 1 : sc;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(src + pf_lane * kCells + sc));
          }
        }
        if (!active(c)) continue;
        T g[Q];
        pull(c, [&](auto i, const S* p) {
          if constexpr (kScaled) g[i] = __half2float(ldg_half_l2(p));
          else if constexpr (std::is_same<S, float>::value) g[i] = ldg_f32_l2(p);
          else g[i] = St::template get<Q, i>(p);
        });
        if constexpr (W) if (wf) wall_fix(c, g);
        collide_store(c, g);
      }
    }
  }
}

// FP16 storage: each thread updates an x-adjacent pair of cells (c, c + 1),
// c even, through the two-cell arithmetic of pair.cuh.  Packed FP32x2
// instructions run the two collisions for about the instruction count of
// one (the single-cell FP16 kernel was close to issue-bound), populations
// with e_x = 0 come in as one aligned half2 load for both cells, and every
// population leaves as one half2 store.  Pulls with e_x != 0 are two scalar
// loads (their sources straddle the pair alignment).  Mixed pairs (one cell
// masked out) store only the active cell.
template <class M, int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_update_pair(const UpdateArgs a) {
  using S = __half;
  constexpr int Q = M::Q;
  constexpr int QS = Q * kCells;
  constexpr int NP = kCells / 2;  // pairs per block
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const WorkItem w = a.items[it];
    const LevelPtrs& L = a.lv[w.level];
    const int BX = L.BX, BXY = L.BX * L.BY;
    if (threadIdx.x == 0 && a.pf_ahead > 0 && it + a.pf_ahead < a.nitems) {
      // the block a CTA about half a wave later takes: its whole [Q][512] run
      // (contiguous, 16-byte aligned) into L2 by one bulk prefetch of the
      // TMA unit, so that CTA's loads find L2 instead of DRAM
      const WorkItem wn = a.items[it + a.pf_ahead];
      const char* pb = reinterpret_cast<const char*>(a.lv[wn.level].src) + int64_t(wn.block) * QS * int64_t(sizeof(S));
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pb), "r"(int(QS * sizeof(S))) : "memory");
    }
    // block deltas as in k_update (x / y offsets 32-bit, z widened per pair)
    const int dxm = (w.edges & 1) ? (L.BX - 1) : -1;
    const int dxp = (w.edges & 2) ? -(L.BX - 1) : 1;
    const int dym = (w.edges & 4) ? BX * (L.BY - 1) : -BX;
    const int dyp = (w.edges & 8) ? -BX * (L.BY - 1) : BX;
    const int dzm = (w.edges & 16) ? BXY * (L.BZ - 1) : -BXY;
    const int dzp = (w.edges & 32) ? -BXY * (L.BZ - 1) : BXY;
    const V2 tau0 = V2(float(L.tau0), float(L.tau0));
    const S* __restrict__ src = reinterpret_cast<const S*>(L.src) + int64_t(w.block) * QS;
    S* __restrict__ dst = reinterpret_cast<S*>(L.dst) + int64_t(w.block) * QS;
    auto active = [&](int c) {
      if (w.mask < 0) return true;
      const uint32_t m = __ldg(a.masks + w.mask * 16 + (c >> 5));
      return bool((m >> (c & 31)) & 1u);
    };
#pragma unroll 1
    for (int p = threadIdx.x; p < NP; p += TPB) {
      const int c0 = 2 * p;
      const bool a0 = active(c0), a1 = active(c0 + 1);
      if (!a0 && !a1) continue;
      const int x0 = c0 & 7, y = (c0 >> 3) & 7, z = c0 >> 6;
      // cell c0 pulls e_x = +1 across the -x face when x0 == 0; cell c0 + 1
      // pulls e_x = -1 across the +x face when x0 == 6 (from that cell itself
      // on the zero-gradient outflow face)
      const int Xm0 = (x0 == 0) ? dxm * QS + 8 : 0;
      const int Xp1 = (x0 == 6) ? ((w.edges & 64) ? -1 : dxp * QS - 8) : 0;
      const int Ym = (y == 0) ? dym * QS + 64 : 0;
      const int Yp = (y == 7) ? dyp * QS - 64 : 0;
      const S* p0 = src + c0;
      const S* b1 = p0 + (z == 0 ? int64_t(dzm) * QS + 512 : int64_t(0));
      const S* bm = p0 + (z == 7 ? int64_t(dzp) * QS - 512 : int64_t(0));
      V2 g[Q];
      static_for<Q>([&](auto i) {
        constexpr int ex = Lattice<Q>::ex(i), ey = Lattice<Q>::ey(i), ez = Lattice<Q>::ez(i);
        constexpr int k = int(i) * kCells - (ex + 8 * ey + 64 * ez);
        int o = 0;
        if constexpr (ey == 1) o += Ym;
        if constexpr (ey == -1) o += Yp;
        const S* b = ez == 1 ? b1 : ez == -1 ? bm : p0;
        if constexpr (ex == 0) {
          // both sources adjacent at an even element offset: one half2 load
          const __half2 h = __ldg(reinterpret_cast<const __half2*>(b + o + k));
          g[i] = V2(__low2float(h), __high2float(h));
        } else if constexpr (ex == 1) {
          g[i] = V2(__half2float(ldg_half_l2(b + o + k + Xm0)), __half2float(ldg_half_l2(b + o + k + 1)));
        } else {
          g[i] = V2(__half2float(ldg_half_l2(b + o + k)), __half2float(ldg_half_l2(b + o + k + 1 + Xp1)));
        }
      });
      if constexpr (Q == 19) {
        const V2 S_ = collide19<V2, true>(g, tau0, V2(float(a.cs2_18), float(a.cs2_18)));
        if (L.aux_dst) {
          float* ad = reinterpret_cast<float*>(L.aux_dst) + int64_t(w.block) * kCells + c0;
          if (a0) ad[0] = S_.x;
          if (a1) ad[1] = S_.y;
        }
      } else {
        if (a.force != nullptr && w.level == 0) {
          const int64_t n = int64_t(L.BX) * L.BY * L.BZ * kCells;
          const int64_t j = int64_t(w.block) * kCells + c0;
          const float* F = reinterpret_cast<const float*>(a.force);
          collide27_closed<V2, true, true>(g, V2(1.0) / tau0, V2(F[j], F[j + 1]), V2(F[n + j], F[n + j + 1]),
                                           V2(F[2 * n + j], F[2 * n + j + 1]));
        } else {
          collide27_closed<V2, false, true>(g, V2(1.0) / tau0, V2(0.0), V2(0.0), V2(0.0));
        }
      }
      S* q = dst + c0;
      if (a0 && a1) {
        // streaming stores: the new state is not read again before the next
        // step, so its lines go first when L2 needs room for prefetched blocks
        static_for<Q>([&](auto i) {
          __stcs(reinterpret_cast<__half2*>(q + int(i) * kCells), __floats2half2_rn(g[i].x, g[i].y));
        });
      } else if (a0) {
        static_for<Q>([&](auto i) { q[int(i) * kCells] = __float2half_rn(g[i].x); });
      } else {
        static_for<Q>([&](auto i) { q[int(i) * kCells + 1] = __float2half_rn(g[i].y); });
      }
    }
  }
}

// Launch shapes the autotuner chooses from: threads per CTA, and a minimum
// number of resident CTAs per SM that caps the registers (higher occupancy
// for the FP16 variants, whose half-size loads keep fewer bytes in flight).
// FP16 storage without walls runs the cell-pair kernel; a listed shape maps
// onto it with half the minimum CTAs per SM (two cells per thread hold about
// twice the registers): (128,1) (256,1) (128,4) (256,2) (128,5).
template <class M, int TPB, int MINB>
cudaError_t launch_pair_shape(UpdateArgs a, int grid, bool persistent, cudaStream_t st) {
  // prefetch distance: half the CTAs resident at once (one CTA per block:
  // measured better than one or two full waves, whose prefetched blocks
  // wait longer in L2) or the grid (persistent CTAs take items grid apart)
  static int occ = 0;  // CTAs per SM of this instance (a property of the kernel)
  if (occ == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_update_pair<M, TPB, MINB>, TPB, 0);
    if (e != cudaSuccess) return e;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  a.pf_ahead = persistent ? grid : occ * sms / 2;
  k_update_pair<M, TPB, MINB><<<grid, TPB, 0, st>>>(a);
  return cudaGetLastError();
}
template <class M>
cudaError_t launch_pair(const UpdateArgs& a, int threads, int minb, int grid, bool persistent, cudaStream_t st) {
  if (threads == 128 && minb == 7) return launch_pair_shape<M, 128, 5>(a, grid, persistent, st);
  if (threads == 128 && minb == 1) return launch_pair_shape<M, 128, 1>(a, grid, persistent, st);
  if (threads == 256 && minb == 1) return launch_pair_shape<M, 256, 1>(a, grid, persistent, st);
  if (threads == 128 && minb == 8) return launch_pair_shape<M, 128, 4>(a, grid, persistent, st);
  if (threads == 256 && minb == 4) return launch_pair_shape<M, 256, 2>(a, grid, persistent, st);
  return cudaErrorInvalidValue;
}
template <class M>
cudaError_t occ_pair(int threads, int minb, int* n) {
  if (threads == 128 && minb == 7) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update_pair<M, 128, 5>, 128, 0);
  if (threads == 128 && minb == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update_pair<M, 128, 1>, 128, 0);
  if (threads == 256 && minb == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update_pair<M, 256, 1>, 256, 0);
  if (threads == 128 && minb == 8) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update_pair<M, 128, 4>, 128, 0);
  if (threads == 256 && minb == 4) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update_pair<M, 256, 2>, 256, 0);
  return cudaErrorInvalidValue;
}

template <class M, class S, bool W>
cudaError_t launch_ms(const UpdateArgs& a, int threads, int minb, int ctas, cudaStream_t st) {
  if (a.nitems == 0) return cudaSuccess;
  const int grid = ctas > 0 ? std::min(ctas, a.nitems) : a.nitems;
  if constexpr (std::is_same<S, __half>::value && !W) {
    return launch_pair<M>(a, threads, minb, grid, ctas > 0, st);
  } else {
    if (threads == 128 && minb == 7) k_update<M, S, 128, 7, W><<<grid, 128, 0, st>>>(a);
    else if (threads == 128 && minb == 1) k_update<M, S, 128, 1, W><<<grid, 128, 0, st>>>(a);
    else if (threads == 256 && minb == 1) k_update<M, S, 256, 1, W><<<grid, 256, 0, st>>>(a);
    else if (threads == 128 && minb == 8) k_update<M, S, 128, 8, W><<<grid, 128, 0, st>>>(a);
    else if (threads == 256 && minb == 4) k_update<M, S, 256, 4, W><<<grid, 256, 0, st>>>(a);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
  }
}

template <class M, class S, bool W>
cudaError_t occ_ms(int threads, int minb, int* n) {
  if constexpr (std::is_same<S, __half>::value && !W) {
    return occ_pair<M>(threads, minb, n);
  } else {
    if (threads == 128 && minb == 7) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update<M, S, 128, 7, W>, 128, 0);
    if (threads == 128 && minb == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update<M, S, 128, 1, W>, 128, 0);
    if (threads == 256 && minb == 1) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update<M, S, 256, 1, W>, 256, 0);
    if (threads == 128 && minb == 8) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update<M, S, 128, 8, W>, 128, 0);
    if (threads == 256 && minb == 4) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, k_update<M, S, 256, 4, W>, 256, 0);
    return cudaErrorInvalidValue;
  }
}

// one translation unit per (model, storage) instantiates the periodic
// kernels, another the wall kernels (update_walls_<model>_<storage>.cu)
#define LBM_UPDATE_INSTANCE(M, S, NAME)                                                               \
  cudaError_t launch_update_##NAME(const UpdateArgs& a, int threads, int minb, int ctas, cudaStream_t st) { \
    return launch_ms<M, S, false>(a, threads, minb, ctas, st);                                       \
  }                                                                                                  \
  cudaError_t occupancy_update_##NAME(int threads, int minb, int* n) { return occ_ms<M, S, false>(threads, minb, n); }

#define LBM_UPDATE_WALL_INSTANCE(M, S, NAME)                                                          \
  cudaError_t launch_update_walls_##NAME(const UpdateArgs& a, int threads, int minb, int ctas,        \
                                         cudaStream_t st) {                                          \
    return launch_ms<M, S, true>(a, threads, minb, ctas, st);                                        \
  }                                                                                                  \
  cudaError_t occupancy_update_walls_##NAME(int threads, int minb, int* n) {                         \
    return occ_ms<M, S, true>(threads, minb, n);                                                     \
  }

#define LBM_UPDATE_DECL(NAME)                                                                          \
  cudaError_t launch_update_##NAME(const UpdateArgs& a, int threads, int minb, int ctas, cudaStream_t st); \
  cudaError_t occupancy_update_##NAME(int threads, int minb, int* n);                                   \
  cudaError_t launch_update_walls_##NAME(const UpdateArgs& a, int threads, int minb, int ctas,          \
                                         cudaStream_t st);                                             \
  cudaError_t occupancy_update_walls_##NAME(int threads, int minb, int* n);

LBM_UPDATE_DECL(d3q19_f64)
LBM_UPDATE_DECL(d3q19_f32)
LBM_UPDATE_DECL(d3q19_f16)
LBM_UPDATE_DECL(d3q27_f64)
LBM_UPDATE_DECL(d3q27_f32)
LBM_UPDATE_DECL(d3q27_f16)

}  // namespace lbm
