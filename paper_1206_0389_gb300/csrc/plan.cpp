// Host-side grid planner: levels, dense level boxes, cell kinds and the work
// lists of the stream-collide, interface and boundary kernels.  Pure C++.
//
// Reading of the interface scheme of Yu et al. (cited in Sections 1 and 3.2
// of the paper, which do not write it out), cell-centred 2:1:
//   active   cells of unrefined blocks of the level;
//   hidden 1 / hidden 2: refined cells at Chebyshev distance 1 / 2 from an
//            active cell; they receive the fine-to-coarse transfer, and
//            hidden 1 is also streamed and collided on the coarse level so the
//            coarse-to-fine temporal interpolation has a value at t+1;
//   ghost    cells outside the level's blocks at distance 1 from them; they
//            receive the coarse-to-fine transfer before every substep.
#include "plan.h"

#include "lattice.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace lbm {

size_t storage_bytes(int st) { return st == LBM_F64 ? 8 : st == LBM_F32 ? 4 : 2; }

int32_t LevelPlan::box_id(int bx, int by, int bz) const {
  const int X = bx - ox, Y = by - oy, Z = bz - oz;
  if (X < 0 || X >= BX || Y < 0 || Y >= BY || Z < 0 || Z >= BZ) return -1;
  return X + BX * (Y + BY * Z);
}

namespace {

inline int wrapi(int v, int n) { return ((v % n) + n) % n; }

// Chebyshev distance from local cell c of a block to the nearest cell of the
// neighbouring block in direction (dx, dy, dz)
inline int cheb(int c, int dx, int dy, int dz) {
  const int x = c & 7, y = (c >> 3) & 7, z = c >> 6;
  auto ax = [](int p, int d) { return d == 0 ? 0 : d < 0 ? p + 1 : 8 - p; };
  return std::max(ax(x, dx), std::max(ax(y, dy), ax(z, dz)));
}

struct DomainLevel {
  int nbx, nby, nbz;
  bool px;
  std::vector<uint8_t> region, refined;  // [nbz][nby][nbx]
  // flat index of block (bx, by, bz) after periodic wrap, -1 outside x range
  int64_t at(int bx, int by, int bz) const {
    if (px) bx = wrapi(bx, nbx);
    else if (bx < 0 || bx >= nbx) return -1;
    by = wrapi(by, nby);
    bz = wrapi(bz, nbz);
    return bx + int64_t(nbx) * (by + int64_t(nby) * bz);
  }
  bool reg(int bx, int by, int bz) const {
    const int64_t i = at(bx, by, bz);
    return i >= 0 && region[i];
  }
  bool act(int bx, int by, int bz) const {
    const int64_t i = at(bx, by, bz);
    return i >= 0 && region[i] && !refined[i];
  }
};

}  // namespace

std::string build_plan(const lbm_grid& g, int model, int storage, double omega, GridPlan& P,
                       const PlanOptions& opt) {
  char msg[256];
  if (model != LBM_D3Q19_MRT_LES && model != LBM_D3Q27_FCLB) return "model must be 0 (D3Q19 MRT-LES) or 1 (D3Q27 FCLB)";
  if (storage != LBM_F64 && storage != LBM_F32 && storage != LBM_F16) return "storage must be 0 (F64), 1 (F32) or 2 (F16)";
  if (g.nbx < 1 || g.nby < 1 || g.nbz < 1) return "block counts must be >= 1";
  if (g.levels < 1 || g.levels > kMaxL) return "levels must be in 1..4";
  if (g.levels > 1 && g.refine == nullptr) return "refine flags required when levels > 1";
  if (!(omega > 0.0 && omega < 2.0)) return "omega must be in (0, 2)";
  if ((g.walls & 3) % 3 != 0 || (g.walls & 12) % 12 != 0 || (g.walls & ~63) || (g.slip & ~(g.walls & 15)))
    return "y/z walls come in pairs per axis (bits 0|1 for y, 2|3 for z); slip must be a subset of them";
  if ((g.walls & 48) && g.periodic_x) return "x walls (bits 4, 5) need a non-periodic x axis";
  if ((g.walls & 32) && g.outlet) return "the face x = NX is either a wall or the pressure outlet";
  if (g.outlet != 0 && g.outlet != 1) return "outlet must be 0 (zero-gradient) or 1 (fixed pressure)";
  if (g.outlet && g.periodic_x) return "a pressure outlet needs a non-periodic x axis";
  const bool nozzle = g.nozzle_r > 0;
  // (the bound keeps every level's cell coordinates of the nozzle in the int range)
  auto modest = [](double v) { return std::isfinite(v) && std::fabs(v) < 1e6; };
  if (nozzle && !(modest(g.nozzle_y0) && modest(g.nozzle_z0) && modest(g.nozzle_r) && modest(g.nozzle_x0) &&
                  modest(g.nozzle_x1) && g.nozzle_x0 < g.nozzle_x1))
    return "nozzle: finite values below 1e6 in magnitude with x0 < x1 required";
  const int L = g.levels;
  const int64_t top = int64_t(g.nbx) * g.nby * g.nbz << (3 * (L - 1));
  if (int64_t(g.nbx) << (L - 1) > (1 << 20) || int64_t(g.nby) << (L - 1) > (1 << 20) ||
      int64_t(g.nbz) << (L - 1) > (1 << 20) || top > (int64_t(1) << 40))
    return "grid too large";

  P = GridPlan();
  P.model = model;
  P.storage = storage;
  P.Q = model == LBM_D3Q19_MRT_LES ? 19 : 27;
  P.levels = L;
  P.periodic_x = g.periodic_x != 0;
  P.walls = g.walls;
  P.slip = g.slip;
  P.outlet = g.outlet;
  const bool px = P.periodic_x;
  if ((opt.halo_lo || opt.halo_hi) && px) return "internal: a sharded part has a non-periodic x axis";
  if (opt.halo_lo && (g.walls & 16)) return "internal: a cut face cannot be the x = 0 wall";
  if (opt.halo_hi && ((g.walls & 32) || g.outlet)) return "internal: a cut face cannot be the x = NX wall or outlet";

  // ---------------------------------------------------------------- levels
  std::vector<DomainLevel> D(L);
  int64_t off = 0;
  for (int l = 0; l < L; ++l) {
    DomainLevel& d = D[l];
    d.nbx = g.nbx << l;
    d.nby = g.nby << l;
    d.nbz = g.nbz << l;
    d.px = px;
    const int64_t n = int64_t(d.nbx) * d.nby * d.nbz;
    if (l == 0) d.region.assign(n, 1);
    d.refined.assign(n, 0);
    if (l < L - 1) {
      int64_t cnt = 0;
      for (int64_t i = 0; i < n; ++i) {
        const uint8_t v = g.refine[off + i];
        if (v > 1) return "refine flags must be 0 or 1";
        if (v && !d.region[i]) {
          snprintf(msg, sizeof msg, "refine flag on a block outside level %d", l);
          return msg;
        }
        d.refined[i] = v;
        cnt += v;
      }
      off += n;
      if (l == 0 && g.walls) {  // refined blocks keep one block away from the walls
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by)
            for (int bx = 0; bx < d.nbx; ++bx)
              if (d.refined[d.at(bx, by, bz)] && (((g.walls & 3) && (by == 0 || by == d.nby - 1)) ||
                                                  ((g.walls & 12) && (bz == 0 || bz == d.nbz - 1)) ||
                                                  ((g.walls & 16) && bx == 0) ||
                                                  ((g.walls & 32) && bx == d.nbx - 1))) {
                snprintf(msg, sizeof msg, "refined block (%d,%d,%d) touches a wall face", bx, by, bz);
                return msg;
              }
      }
      if (l == 0 && (opt.halo_lo || opt.halo_hi)) {  // and away from the cuts of a sharded part
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by)
            for (int bx = 0; bx < d.nbx; ++bx)
              if (d.refined[d.at(bx, by, bz)] && ((opt.halo_lo && bx <= 1) || (opt.halo_hi && bx >= d.nbx - 2))) {
                snprintf(msg, sizeof msg, "refined block (%d,%d,%d) within a block of a cut between parts", bx, by,
                         bz);
                return msg;
              }
      }
      if (l == 0 && g.outlet) {  // and away from the pressure outlet
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by)
            if (d.refined[d.at(d.nbx - 1, by, bz)]) {
              snprintf(msg, sizeof msg, "refined block (%d,%d,%d) touches the pressure outlet", d.nbx - 1, by, bz);
              return msg;
            }
      }
      if (cnt == 0) {
        snprintf(msg, sizeof msg, "level %d refines no block", l);
        return msg;
      }
      if (l >= 1) {  // nesting rule
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by)
            for (int bx = 0; bx < d.nbx; ++bx) {
              if (!d.refined[d.at(bx, by, bz)]) continue;
              for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                  for (int dx = -1; dx <= 1; ++dx) {
                    const int64_t j = d.at(bx + dx, by + dy, bz + dz);
                    if (j >= 0 && !d.region[j]) {
                      snprintf(msg, sizeof msg,
                               "refined block (%d,%d,%d) of level %d touches the level boundary", bx,
                               by, bz, l);
                      return msg;
                    }
                  }
            }
      }
      // children form the next level
      DomainLevel& c = D[l + 1];
      c.nbx = 2 * d.nbx;
      c.nby = 2 * d.nby;
      c.nbz = 2 * d.nbz;
      c.region.assign(int64_t(c.nbx) * c.nby * c.nbz, 0);
      for (int bz = 0; bz < d.nbz; ++bz)
        for (int by = 0; by < d.nby; ++by)
          for (int bx = 0; bx < d.nbx; ++bx)
            if (d.refined[bx + int64_t(d.nbx) * (by + int64_t(d.nby) * bz)])
              for (int k = 0; k < 8; ++k)
                c.region[(2 * bx + (k & 1)) + int64_t(c.nbx) * ((2 * by + ((k >> 1) & 1)) +
                                                               int64_t(c.nby) * (2 * bz + (k >> 2)))] = 1;
    }
  }

  // ---------------------------------------------------------------- boxes and kinds
  P.lv.resize(L);
  const double tau00 = 1.0 / omega;
  for (int l = 0; l < L; ++l) {
    DomainLevel& d = D[l];
    LevelPlan& lp = P.lv[l];
    lp.l = l;
    lp.nbx = d.nbx;
    lp.nby = d.nby;
    lp.nbz = d.nbz;
    lp.NX = 8 * d.nbx;
    lp.NY = 8 * d.nby;
    lp.NZ = 8 * d.nbz;
    lp.tau0 = 0.5 + std::ldexp(tau00 - 0.5, l);
    const int64_t n = int64_t(d.nbx) * d.nby * d.nbz;
    // used blocks: region, ghost (l >= 1, in domain, next to region), bc columns
    std::vector<uint8_t> ghost(n, 0);
    std::vector<uint8_t> usedx(d.nbx + 2, 0), usedy(d.nby, 0), usedz(d.nbz, 0);
    std::vector<uint8_t> bcl(int64_t(d.nby) * d.nbz, 0), bch(int64_t(d.nby) * d.nbz, 0);
    for (int bz = 0; bz < d.nbz; ++bz)
      for (int by = 0; by < d.nby; ++by)
        for (int bx = 0; bx < d.nbx; ++bx) {
          const int64_t i = d.at(bx, by, bz);
          if (d.region[i]) {
            lp.level_blocks++;
            usedx[bx + 1] = usedy[by] = usedz[bz] = 1;
            if (!px) {
              for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy) {
                  const int64_t f = wrapi(by + dy, d.nby) + int64_t(d.nby) * wrapi(bz + dz, d.nbz);
                  if (bx == 0) bcl[f] = 1;
                  if (bx == d.nbx - 1) bch[f] = 1;
                }
            }
            continue;
          }
          if (l == 0) continue;
          bool adj = false;
          for (int dz = -1; dz <= 1 && !adj; ++dz)
            for (int dy = -1; dy <= 1 && !adj; ++dy)
              for (int dx = -1; dx <= 1 && !adj; ++dx) adj = d.reg(bx + dx, by + dy, bz + dz);
          if (adj) {
            ghost[i] = 1;
            usedx[bx + 1] = usedy[by] = usedz[bz] = 1;
          }
        }
    for (int64_t f = 0; f < int64_t(d.nby) * d.nbz; ++f) {
      if (bcl[f]) usedx[0] = usedy[f % d.nby] = usedz[f / d.nby] = 1;
      if (bch[f]) usedx[d.nbx + 1] = usedy[f % d.nby] = usedz[f / d.nby] = 1;
    }
    auto range = [](const std::vector<uint8_t>& u, int shift, int& o, int& B) {
      int lo = -1, hi = -1;
      for (int i = 0; i < int(u.size()); ++i)
        if (u[i]) {
          if (lo < 0) lo = i;
          hi = i;
        }
      o = lo - shift;
      B = hi - lo + 1;
    };
    if (px) {
      lp.ox = 0;
      lp.BX = d.nbx;
      lp.wrap[0] = true;
      std::vector<uint8_t> ux(usedx.begin() + 1, usedx.end() - 1);
      range(ux, 0, lp.ox, lp.BX);
      lp.wrap[0] = lp.BX == d.nbx;
    } else {
      range(usedx, 1, lp.ox, lp.BX);
      lp.wrap[0] = false;
    }
    range(usedy, 0, lp.oy, lp.BY);
    range(usedz, 0, lp.oz, lp.BZ);
    lp.wrap[1] = lp.BY == d.nby;
    lp.wrap[2] = lp.BZ == d.nbz;
    const int64_t nb = lp.nblocks();
    if (nb * 512 * P.Q >= (int64_t(1) << 46) || nb >= (int64_t(1) << 31)) return "level box too large";
    // the streaming kernels form x / y neighbour offsets in 32 bits (z
    // neighbours go through 64-bit bases): one z layer of blocks must stay
    // below 2^31 stored values
    if (int64_t(lp.BX) * lp.BY * 512 * P.Q >= (int64_t(1) << 31))
      return "level box cross-section too large: BX * BY * Q * 512 must be below 2^31";
    lp.kind.assign(nb * 512, K_NONE);

    auto box_of = [&](int bx, int by, int bz) -> int32_t {  // domain coords (wrapped)
      if (px) bx = wrapi(bx, d.nbx);
      by = wrapi(by, d.nby);
      bz = wrapi(bz, d.nbz);
      return lp.box_id(bx, by, bz);
    };

    // region blocks: active / hidden / refined cells; work items
    for (int bz = 0; bz < d.nbz; ++bz)
      for (int by = 0; by < d.nby; ++by)
        for (int bx = 0; bx < d.nbx; ++bx) {
          const int64_t i = d.at(bx, by, bz);
          if (!d.region[i]) continue;
          const int32_t b = lp.box_id(bx, by, bz);
          if (b < 0) return "internal: region block outside its box";
          // region blocks must not sit on a non-wrapping box face
          const int X = bx - lp.ox, Y = by - lp.oy, Z = bz - lp.oz;
          if ((!lp.wrap[0] && (X == 0 || X == lp.BX - 1)) || (!lp.wrap[1] && (Y == 0 || Y == lp.BY - 1)) ||
              (!lp.wrap[2] && (Z == 0 || Z == lp.BZ - 1)))
            return "internal: level block on the face of a non-periodic box";
          uint8_t* k = &lp.kind[int64_t(b) * 512];
          WorkItem w;
          w.block = b;
          w.level = uint8_t(l);
          w.edges = uint8_t((lp.wrap[0] && X == 0 ? 1 : 0) | (lp.wrap[0] && X == lp.BX - 1 ? 2 : 0) |
                            (lp.wrap[1] && Y == 0 ? 4 : 0) | (lp.wrap[1] && Y == lp.BY - 1 ? 8 : 0) |
                            (lp.wrap[2] && Z == 0 ? 16 : 0) | (lp.wrap[2] && Z == lp.BZ - 1 ? 32 : 0) |
                            (!px && !P.outlet && !(l == 0 && opt.halo_hi) && bx == d.nbx - 1 ? 64 : 0) |
                            (l == 0 && (P.walls & 16) && bx == 0 ? 128 : 0));
          if (!d.refined[i]) {
            std::fill(k, k + 512, uint8_t(K_ACTIVE));
            lp.active_cells += 512;
            lp.updated_cells += 512;
            w.mask = -1;
            lp.items.push_back(w);
            continue;
          }
          uint32_t m[16] = {0};
          bool any = false;
          for (int c = 0; c < 512; ++c) {
            int dist = 99;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                  if ((dx | dy | dz) && d.act(bx + dx, by + dy, bz + dz))
                    dist = std::min(dist, cheb(c, dx, dy, dz));
            k[c] = dist == 1 ? K_HIDDEN1 : dist == 2 ? K_HIDDEN2 : K_REFINED;
            if (dist == 1) {
              m[c >> 5] |= 1u << (c & 31);
              any = true;
              lp.updated_cells++;
            }
            if (dist <= 2) lp.hidden_cells++;
          }
          if (any) {
            w.mask = int16_t(lp.masks.size() / 16);
            if (lp.masks.size() / 16 >= 32767) return "too many masked blocks";
            lp.masks.insert(lp.masks.end(), m, m + 16);
            lp.items.push_back(w);
          }
        }
    // ghost blocks (l >= 1)
    for (int bz = 0; bz < d.nbz; ++bz)
      for (int by = 0; by < d.nby; ++by)
        for (int bx = 0; bx < d.nbx; ++bx) {
          const int64_t i = d.at(bx, by, bz);
          if (!ghost[i]) continue;
          const int32_t b = lp.box_id(bx, by, bz);
          uint8_t* k = &lp.kind[int64_t(b) * 512];
          for (int c = 0; c < 512; ++c) {
            int dist = 99;
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                  if ((dx | dy | dz) && d.reg(bx + dx, by + dy, bz + dz))
                    dist = std::min(dist, cheb(c, dx, dy, dz));
            if (dist == 1) {
              k[c] = K_GHOST;
              lp.ghost_cells++;
            }
          }
        }
    // inflow ghost column x = -1 (the outflow needs none: the stream-collide
    // kernel reads its zero-gradient ghosts from x = NX - 1, edges bit 6)
    // halo columns of a sharded part's cuts (level 0): copies of the
    // neighbouring part's boundary layer, never updated
    if (l == 0)
      for (int side = 0; side < 2; ++side) {
        if (!(side == 0 ? opt.halo_lo : opt.halo_hi)) continue;
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by) {
            const int32_t hb = lp.box_id(side == 0 ? -1 : d.nbx, by, bz);
            if (hb < 0) return "internal: halo block outside its box";
            std::fill(&lp.kind[int64_t(hb) * 512], &lp.kind[int64_t(hb) * 512] + 512, uint8_t(K_HALO));
          }
      }
    if (!px) {
      // (a cut face of a sharded part has no inflow: its halo is filled by
      // the exchange)
      if (!(l == 0 && opt.halo_lo))
      for (int bz = 0; bz < d.nbz; ++bz)
        for (int by = 0; by < d.nby; ++by) {
          if (!bcl[by + int64_t(d.nby) * bz]) continue;
          const int32_t gb = lp.box_id(-1, by, bz);
          const int32_t sb = lp.box_id(0, by, bz);
          if (gb < 0) return "internal: boundary block outside its box";
          if (sb < 0) continue;
          for (int cz = 0; cz < 8; ++cz)
            for (int cy = 0; cy < 8; ++cy) {
              const int sc = 8 * cy + 64 * cz;
              if (lp.kind[int64_t(sb) * 512 + sc] == K_NONE) continue;
              const int gc = 7 + 8 * cy + 64 * cz;
              lp.kind[int64_t(gb) * 512 + gc] = K_BC;
              lp.bc_cells++;
              BCItem it{};
              it.gblock = gb;
              it.gcell = int16_t(gc);
              it.type = 0;
              it.sblock = sb;
              it.scell = int16_t(sc);
              it.y = 8 * by + cy;
              it.z = 8 * bz + cz;
              // a coarse-to-fine ghost source only gets its value in the
              // same substep: that kernel writes this inflow ghost too
              if (lp.kind[int64_t(sb) * 512 + sc] == K_GHOST) lp.c2f_bc.push_back(it);
              else lp.bc.push_back(it);
            }
        }
      // pressure-outlet ghost column x = NX (refined blocks keep away from
      // it, so its sources are active cells)
      if (P.outlet)
        for (int bz = 0; bz < d.nbz; ++bz)
          for (int by = 0; by < d.nby; ++by) {
            if (!bch[by + int64_t(d.nby) * bz]) continue;
            const int32_t gb = lp.box_id(d.nbx, by, bz);
            const int32_t sb = lp.box_id(d.nbx - 1, by, bz);
            if (gb < 0) return "internal: boundary block outside its box";
            if (sb < 0) continue;
            for (int cz = 0; cz < 8; ++cz)
              for (int cy = 0; cy < 8; ++cy) {
                const int sc = 7 + 8 * cy + 64 * cz;
                if (lp.kind[int64_t(sb) * 512 + sc] == K_NONE) continue;
                if (lp.kind[int64_t(sb) * 512 + sc] == K_GHOST) return "internal: outlet source is a ghost cell";
                const int gc = 8 * cy + 64 * cz;
                lp.kind[int64_t(gb) * 512 + gc] = K_BC;
                lp.bc_cells++;
                BCItem it{};
                it.gblock = gb;
                it.gcell = int16_t(gc);
                it.type = 1;
                it.sblock = sb;
                it.scell = int16_t(sc);
                it.y = 8 * by + cy;
                it.z = 8 * bz + cz;
                lp.bc.push_back(it);
              }
          }
    }
    (void)box_of;
  }

  // ---------------------------------------------------------------- interface lists
  // a ghost cell with its full stencil, before chunking
  struct Ghost {
    C2FItem it;
    int32_t cblock[8];
    int16_t ccell[8];
  };
  const int max_cells = c2f_max_cells(storage);
  for (int l = 1; l < L; ++l) {
    LevelPlan& f = P.lv[l];
    const LevelPlan& c = P.lv[l - 1];
    const DomainLevel& dc = D[l - 1];
    std::vector<Ghost> ghosts;
    for (int bz = f.oz; bz < f.oz + f.BZ; ++bz)
      for (int by = f.oy; by < f.oy + f.BY; ++by)
        for (int bx = f.ox; bx < f.ox + f.BX; ++bx) {
          const int32_t b = f.box_id(bx, by, bz);
          for (int cc = 0; cc < 512; ++cc) {
            if (f.kind[int64_t(b) * 512 + cc] != K_GHOST) continue;
            const int X = 8 * bx + (cc & 7), Y = 8 * by + ((cc >> 3) & 7), Z = 8 * bz + (cc >> 6);
            int lo[3], hi[3];
            uint8_t tb = 0;
            const int XYZ[3] = {X, Y, Z};
            const int NC[3] = {c.NX, c.NY, c.NZ};
            for (int a = 0; a < 3; ++a) {
              const int v = XYZ[a];
              int i0 = (v - 1) >= 0 ? (v - 1) / 2 : -1;  // floor((v-1)/2) for v >= 0
              int i1 = i0 + 1;
              if (v % 2 == 0) tb |= uint8_t(1u << a);
              if (a == 0 && !px) {
                i0 = std::min(std::max(i0, 0), NC[a] - 1);
                i1 = std::min(std::max(i1, 0), NC[a] - 1);
              } else {
                i0 = wrapi(i0, NC[a]);
                i1 = wrapi(i1, NC[a]);
              }
              lo[a] = i0;
              hi[a] = i1;
            }
            Ghost gh{};
            C2FItem& it = gh.it;
            it.bc = -1;
            it.fblock = b;
            it.fcell = int16_t(cc);
            it.tbits = tb;
            // populations some updated fine cell pulls from this ghost cell;
            // all of them where an inflow/outflow ghost is taken from it
            if (!px && (X == 0 || X == f.NX - 1)) it.need = (1u << P.Q) - 1u;
            for (int i = 0; i < P.Q; ++i) {
              int nx = X + ex27(i), ny = wrapi(Y + ey27(i), f.NY), nz = wrapi(Z + ez27(i), f.NZ);
              if (px) nx = wrapi(nx, f.NX);
              if (nx < 0 || nx >= f.NX) continue;
              const int32_t nbk = f.box_id(nx >> 3, ny >> 3, nz >> 3);
              if (nbk < 0) continue;
              const uint8_t nk = f.kind[int64_t(nbk) * 512 + (nx & 7) + 8 * (ny & 7) + 64 * (nz & 7)];
              if (nk == K_ACTIVE || nk == K_HIDDEN1) it.need |= 1u << i;
            }
            for (int k = 0; k < 8; ++k) {
              const int ix = (k & 1) ? hi[0] : lo[0];
              const int iy = (k & 2) ? hi[1] : lo[1];
              const int iz = (k & 4) ? hi[2] : lo[2];
              const int32_t cb = c.box_id(ix >> 3, iy >> 3, iz >> 3);
              const int ccell = (ix & 7) + 8 * (iy & 7) + 64 * (iz & 7);
              if (cb < 0) return "internal: interpolation stencil outside the coarse box";
              const uint8_t ck = c.kind[int64_t(cb) * 512 + ccell];
              if (ck != K_ACTIVE && ck != K_HIDDEN1)
                return "interpolation stencil leaves the updated coarse cells (grid too tight)";
              gh.cblock[k] = cb;
              gh.ccell[k] = int16_t(ccell);
            }
            ghosts.push_back(gh);
          }
        }
    (void)dc;
    // fine ghost cells that share coarse stencils become neighbours, then
    // consecutive ghosts form chunks of at most kC2FMaxItems items and
    // max_cells distinct stencil cells
    std::stable_sort(ghosts.begin(), ghosts.end(), [](const Ghost& a, const Ghost& b) {
      if (a.cblock[0] != b.cblock[0]) return a.cblock[0] < b.cblock[0];
      return a.ccell[0] < b.ccell[0];
    });
    auto key = [](int32_t cb, int16_t cc) { return int64_t(cb) * 512 + cc; };
    size_t g0 = 0;
    while (g0 < ghosts.size()) {
      std::vector<int64_t> cells;
      size_t g1 = g0;
      while (g1 < ghosts.size() && g1 - g0 < size_t(kC2FMaxItems)) {
        int64_t add[8];
        int na = 0;
        for (int k = 0; k < 8; ++k) {
          const int64_t kk = key(ghosts[g1].cblock[k], ghosts[g1].ccell[k]);
          if (!std::binary_search(cells.begin(), cells.end(), kk) && std::find(add, add + na, kk) == add + na)
            add[na++] = kk;
        }
        if (int(cells.size()) + na > max_cells) break;
        for (int k = 0; k < na; ++k) cells.insert(std::upper_bound(cells.begin(), cells.end(), add[k]), add[k]);
        ++g1;
      }
      C2FChunk ch{};
      ch.first_item = int32_t(f.c2f.size());
      ch.first_cell = int32_t(f.c2f_cells.size());
      ch.nitems = int16_t(g1 - g0);
      ch.ncells = int16_t(cells.size());
      for (int64_t k : cells) f.c2f_cells.push_back(C2FCell{int32_t(k / 512), int16_t(k % 512), 0});
      for (size_t g = g0; g < g1; ++g) {
        C2FItem it = ghosts[g].it;
        for (int k = 0; k < 8; ++k) {
          const int64_t kk = key(ghosts[g].cblock[k], ghosts[g].ccell[k]);
          it.slot[k] = uint16_t(std::lower_bound(cells.begin(), cells.end(), kk) - cells.begin());
        }
        f.c2f.push_back(it);
      }
      f.c2f_chunks.push_back(ch);
      g0 = g1;
    }
    if (f.c2f_cells.size() >= (size_t(1) << 31)) return "too many coarse-to-fine cells";
    if (!f.c2f_bc.empty()) {
      std::vector<int32_t> at(size_t(f.nblocks()) * 512, -1);
      for (size_t k = 0; k < f.c2f.size(); ++k) at[int64_t(f.c2f[k].fblock) * 512 + f.c2f[k].fcell] = int32_t(k);
      for (size_t j = 0; j < f.c2f_bc.size(); ++j) {
        const int32_t k = at[int64_t(f.c2f_bc[j].sblock) * 512 + f.c2f_bc[j].scell];
        if (k < 0) return "internal: inflow ghost source is not a coarse-to-fine ghost";
        f.c2f[k].bc = int32_t(j);
      }
    }
  }
  for (int l = 0; l + 1 < L; ++l) {
    LevelPlan& c = P.lv[l];
    const LevelPlan& f = P.lv[l + 1];
    for (int bz = c.oz; bz < c.oz + c.BZ; ++bz)
      for (int by = c.oy; by < c.oy + c.BY; ++by)
        for (int bx = c.ox; bx < c.ox + c.BX; ++bx) {
          const int32_t b = c.box_id(bx, by, bz);
          for (int cc = 0; cc < 512; ++cc) {
            const uint8_t k = c.kind[int64_t(b) * 512 + cc];
            if (k != K_HIDDEN1 && k != K_HIDDEN2) continue;
            const int X = 8 * bx + (cc & 7), Y = 8 * by + ((cc >> 3) & 7), Z = 8 * bz + (cc >> 6);
            F2CItem it{};
            it.cblock = b;
            it.ccell = int16_t(cc);
            for (int ch = 0; ch < 8; ++ch) {
              const int x = 2 * X + (ch & 1), y = 2 * Y + ((ch >> 1) & 1), z = 2 * Z + (ch >> 2);
              const int32_t fb = f.box_id(x >> 3, y >> 3, z >> 3);
              const int fc = (x & 7) + 8 * (y & 7) + 64 * (z & 7);
              if (fb < 0 || f.kind[int64_t(fb) * 512 + fc] != K_ACTIVE)
                return "internal: restriction child is not an active fine cell";
              if (ch & 1) continue;  // the odd child is fcell + 1 of the same block (x = 2X is even)
              it.fblock[ch >> 1] = fb;
              it.fcell[ch >> 1] = int16_t(fc);
            }
            c.f2c.push_back(it);
          }
        }
  }

  // ---------------------------------------------------------------- nozzle
  if (nozzle) {
    const double y0 = g.nozzle_y0, z0 = g.nozzle_z0, R = g.nozzle_r, x0 = g.nozzle_x0, x1 = g.nozzle_x1;
    // the finest level whose blocks cover the cylinder grown by two of its
    // cells, all of them and their 26 neighbours non-refined blocks of the
    // level (no interface stencil reaches the body)
    int ln = -1;
    double box[3][2];
    for (int l = L - 1; l >= 0 && ln < 0; --l) {
      const double sc = std::ldexp(1.0, l);
      const double b[3][2] = {{x0 * sc - 2, x1 * sc + 2}, {(y0 - R) * sc - 2, (y0 + R) * sc + 2},
                              {(z0 - R) * sc - 2, (z0 + R) * sc + 2}};
      const DomainLevel& d = D[l];
      const int nbs[3] = {d.nbx, d.nby, d.nbz};
      int lo[3], hi[3];
      bool ok = true;
      for (int a = 0; a < 3; ++a) {
        lo[a] = int(std::floor(b[a][0] / 8));
        hi[a] = int(std::floor(b[a][1] / 8));
        ok = ok && lo[a] - 1 >= 0 && hi[a] + 1 <= nbs[a] - 1;
      }
      for (int bz = lo[2]; ok && bz <= hi[2]; ++bz)
        for (int by = lo[1]; ok && by <= hi[1]; ++by)
          for (int bx = lo[0]; ok && bx <= hi[0]; ++bx) {
            for (int dz = -1; dz <= 1; ++dz)
              for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx)
                  if (!d.reg(bx + dx, by + dy, bz + dz) || d.refined[d.at(bx + dx, by + dy, bz + dz)]) ok = false;
          }
      if (ok) {
        ln = l;
        for (int a = 0; a < 3; ++a) box[a][0] = b[a][0], box[a][1] = b[a][1];
      }
    }
    if (ln < 0)
      return "the nozzle must lie inside non-refined blocks of one level, one block away from its "
             "interfaces and the domain faces";
    P.nozzle_level = ln;
    LevelPlan& lp = P.lv[ln];
    const double s = std::ldexp(1.0, -ln);
    // cell-centre test of the closed cylinder (coarse units)
    auto solid = [&](int X, int Y, int Z) {
      const double xc = (X + 0.5) * s, yc = (Y + 0.5) * s, zc = (Z + 0.5) * s;
      const double dy = yc - y0, dz = zc - z0;
      return xc >= x0 && xc <= x1 && dy * dy + dz * dz <= R * R;
    };
    int clo[3], chi[3];
    for (int a = 0; a < 3; ++a) {
      clo[a] = int(std::floor(box[a][0]));
      chi[a] = int(std::ceil(box[a][1]));
    }
    auto loc = [&](int X, int Y, int Z, int32_t& b, int16_t& c) {
      b = lp.box_id(X >> 3, Y >> 3, Z >> 3);
      c = int16_t((X & 7) + 8 * (Y & 7) + 64 * (Z & 7));
      return b >= 0;
    };
    // solid cells leave the stream-collide work (masked items)
    std::vector<int32_t> item_of(size_t(lp.nblocks()), -1);
    for (size_t k = 0; k < lp.items.size(); ++k) item_of[lp.items[k].block] = int32_t(k);
    std::vector<char> drop(lp.items.size(), 0);
    for (int Z = clo[2]; Z <= chi[2]; ++Z)
      for (int Y = clo[1]; Y <= chi[1]; ++Y)
        for (int X = clo[0]; X <= chi[0]; ++X) {
          if (!solid(X, Y, Z)) continue;
          int32_t b;
          int16_t c;
          if (!loc(X, Y, Z, b, c) || lp.kind[int64_t(b) * 512 + c] != K_ACTIVE || item_of[b] < 0)
            return "internal: nozzle cell outside the active cells of its level";
          lp.kind[int64_t(b) * 512 + c] = K_SOLID;
          lp.solid_cells++;
          lp.active_cells--;
          lp.updated_cells--;
          WorkItem& w = lp.items[item_of[b]];
          if (w.mask < 0) {
            if (lp.masks.size() / 16 >= 32767) return "too many masked blocks";
            w.mask = int16_t(lp.masks.size() / 16);
            lp.masks.insert(lp.masks.end(), 16, 0xffffffffu);
          }
          uint32_t* m = &lp.masks[size_t(w.mask) * 16];
          m[c >> 5] &= ~(1u << (c & 31));
        }
    for (size_t k = 0; k < lp.items.size(); ++k) {
      const WorkItem& w = lp.items[k];
      if (w.mask < 0) continue;
      bool any = false;
      for (int j = 0; j < 16; ++j) any = any || lp.masks[size_t(w.mask) * 16 + j] != 0;
      drop[k] = !any;
    }
    {
      std::vector<WorkItem> keep;
      for (size_t k = 0; k < lp.items.size(); ++k)
        if (!drop[k]) keep.push_back(lp.items[k]);
      lp.items.swap(keep);
    }
    // links: fluid cells whose neighbour along e_i is solid; the segment
    // between the cell centres enters the cylinder at the later of its
    // entries into the slab x0 <= x <= x1 and the infinite cylinder r <= R
    const int Q = P.Q;
    for (int Z = clo[2]; Z <= chi[2]; ++Z)
      for (int Y = clo[1]; Y <= chi[1]; ++Y)
        for (int X = clo[0]; X <= chi[0]; ++X) {
          if (solid(X, Y, Z)) continue;
          for (int i = 1; i < Q; ++i) {
            const int ex = Q == 19 ? Lattice<19>::ex(i) : Lattice<27>::ex(i);
            const int ey = Q == 19 ? Lattice<19>::ey(i) : Lattice<27>::ey(i);
            const int ez = Q == 19 ? Lattice<19>::ez(i) : Lattice<27>::ez(i);
            if (!solid(X + ex, Y + ey, Z + ez)) continue;
            LinkItem it{};
            if (!loc(X, Y, Z, it.fblock, it.fcell) || lp.kind[int64_t(it.fblock) * 512 + it.fcell] != K_ACTIVE ||
                !loc(X + ex, Y + ey, Z + ez, it.bblock, it.bcell))
              return "internal: nozzle link outside the active cells of its level";
            it.i = uint8_t(i);
            it.ib = uint8_t(Q == 19 ? Lattice<19>::index(-ex, -ey, -ez) : Lattice<27>::index(-ex, -ey, -ez));
            const double px = (X + 0.5) * s, py = (Y + 0.5) * s - y0, pz = (Z + 0.5) * s - z0;
            const double dx = ex * s, dy = ey * s, dz = ez * s;
            double ts;
            bool cap1 = false;
            if (px >= x0 && px <= x1) {
              ts = 0.0;
            } else if (px > x1) {
              ts = (x1 - px) / dx;
              cap1 = true;
            } else {
              ts = (x0 - px) / dx;
            }
            const double cc = py * py + pz * pz - R * R;
            double tc = 0.0;
            if (cc > 0) {
              const double aa = dy * dy + dz * dz;
              const double bb = 2.0 * (py * dy + pz * dz);
              tc = (-bb - std::sqrt(bb * bb - 4.0 * aa * cc)) / (2.0 * aa);
            }
            if (ts >= tc) {
              it.q = ts;
            } else {
              it.q = tc;
              cap1 = false;
            }
            it.type = cap1 ? 1 : 0;
            it.y = Y + ey;
            it.z = Z + ez;
            if (cap1) {
              // the fluid cell straight downstream of the solid cell
              if (!loc(X + ex + 1, Y + ey, Z + ez, it.sblock, it.scell) ||
                  lp.kind[int64_t(it.sblock) * 512 + it.scell] != K_ACTIVE)
                return "internal: cap link without a fluid cell downstream";
            } else if (solid(X - ex, Y - ey, Z - ez)) {
              it.sblock = -1;
            } else if (!loc(X - ex, Y - ey, Z - ez, it.sblock, it.scell) ||
                       lp.kind[int64_t(it.sblock) * 512 + it.scell] != K_ACTIVE) {
              return "internal: nozzle link's second cell is not active";
            }
            lp.links.push_back(it);
          }
        }
  }

  // ---------------------------------------------------------------- memory estimate
  const size_t sb = storage_bytes(storage);
  const bool aux = model == LBM_D3Q19_MRT_LES && L > 1;
  const size_t rb = storage == LBM_F64 ? 8 : 4;
  int64_t bytes = 0;
  for (const LevelPlan& lp : P.lv) {
    bytes += 2 * lp.nblocks() * 512 * P.Q * int64_t(sb);
    if (aux) bytes += 2 * lp.nblocks() * 512 * int64_t(rb);
    bytes += lp.nblocks() * 512;  // kinds
    bytes += int64_t(lp.items.size() * sizeof(WorkItem) + lp.masks.size() * 4 +
                     lp.c2f.size() * sizeof(C2FItem) + lp.c2f_chunks.size() * sizeof(C2FChunk) +
                     lp.c2f_cells.size() * sizeof(C2FCell) + lp.f2c.size() * sizeof(F2CItem) +
                     (lp.bc.size() + lp.c2f_bc.size()) * sizeof(BCItem) + lp.links.size() * sizeof(LinkItem));
  }
  P.device_bytes = bytes;
  return "";
}

}  // namespace lbm
