// Host-side plan of the block-structured, time-nested grid (no CUDA calls).
//
// Each level is stored as a dense box of 8^3-cell blocks that covers the
// level's own blocks, its coarse-to-fine ghost blocks and (x not periodic) the
// inflow/outflow ghost columns.  Block id = bx + BX (by + BY bz) in box
// coordinates.  Blocks of the box that belong to none of those sets are
// allocated but never touched.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "kernels.cuh"

namespace lbm {

struct LevelPlan {
  int l = 0;
  int nbx = 0, nby = 0, nbz = 0;  // level block grid of the whole domain
  int NX = 0, NY = 0, NZ = 0;     // level cells of the whole domain
  int ox = 0, oy = 0, oz = 0;     // box origin in level block coordinates
  int BX = 0, BY = 0, BZ = 0;     // box size in blocks
  bool wrap[3] = {false, false, false};  // box spans a periodic axis
  double tau0 = 0.5;
  int64_t nblocks() const { return int64_t(BX) * BY * BZ; }

  std::vector<uint8_t> kind;        // [nblocks][512] CellKind
  std::vector<WorkItem> items;      // stream-collide work of this level
  std::vector<uint32_t> masks;      // 16 words per masked item
  std::vector<C2FItem> c2f;         // ghost cells of this level (l >= 1), in chunks
  std::vector<C2FChunk> c2f_chunks;
  std::vector<C2FCell> c2f_cells;   // distinct coarse stencil cells per chunk
  std::vector<F2CItem> f2c;         // hidden cells of this level (l < L-1)
  std::vector<BCItem> bc;           // inflow ghost cells
  std::vector<BCItem> c2f_bc;       // inflow ghosts whose source is a c2f ghost cell
                                    // (written by the coarse-to-fine kernel)
  std::vector<LinkItem> links;      // nozzle surface links (the nozzle's level only)
  std::vector<int32_t> block_of;    // [nbz][nby][nbx] in-domain block -> box id or -1

  int64_t level_blocks = 0, active_cells = 0, updated_cells = 0, hidden_cells = 0;
  int64_t ghost_cells = 0, bc_cells = 0, solid_cells = 0;

  // box id of level block (bx, by, bz) given in level coordinates, -1 if
  // outside the box
  int32_t box_id(int bx, int by, int bz) const;
};

struct GridPlan {
  int model = 0, storage = 0, Q = 19;
  int levels = 1;
  bool periodic_x = true;
  int walls = 0, slip = 0;  // level-0 wall faces (bit 0/1 low/high y, 2/3 low/high z), free-slip subset
  int outlet = 0;           // 1: pressure outlet on x = NX (level 0)
  int nozzle_level = -1;    // level holding the nozzle, -1 if none
  std::vector<LevelPlan> lv;
  int64_t device_bytes = 0;
};

// A part of a block-sharded grid (lbm_shard_*): its x faces marked here are
// cuts between parts instead of domain faces.  The level-0 box then keeps one
// halo block column beyond such a face, filled with the neighbouring part's
// boundary layer before each coarse step; the face gets no inflow, outflow
// or outlet, and no refined block may come within one block of it (finer
// levels stay inside one part).
struct PlanOptions {
  bool halo_lo = false;  // the face x = 0 is a cut
  bool halo_hi = false;  // the face x = NX is a cut
};

// Builds the plan; returns an empty string on success, else the reason.
std::string build_plan(const lbm_grid& g, int model, int storage, double omega, GridPlan& out,
                       const PlanOptions& opt = PlanOptions());

size_t storage_bytes(int storage);

}  // namespace lbm
