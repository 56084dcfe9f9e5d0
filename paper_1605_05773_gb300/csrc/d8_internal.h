// d8_internal.h -- types shared by the libd8 host code and kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "d8.h"

namespace d8 {

constexpr int NT = 256;                 // threads per tile block
constexpr uint32_t ROOT = 0xFFFFFFFFu;  // "no parent" in the combine
constexpr int MAX_ROUNDS = 40;          // pointer-jumping rounds (>= log2 of any slot count)

// One DEM of a call (a single call has one; a batch has many).
struct DemDesc {
  const float* z;
  int64_t ldz;
  uint8_t* dir;
  int64_t lddir;
  void* A;  // uint32 counts or fp32 areas / gradients
  int64_t ldA;
  const float* w;  // weights (weighted) or dL/dA (backward)
  int64_t ldw;
  int64_t H, W;
  int64_t ntx, nty;
  int64_t tile_base;  // global index of this DEM's first tile
  int halo;           // direction stencil: bit 0 the row above row 0 is readable (z - ldz) and row 0
                      // is not a grid edge; bit 1 the same for the row below row H-1 (a strip of a
                      // taller grid)
};

// The DEMs of a launch: either one descriptor passed by value, or a device
// table plus a per-tile DEM index.
struct DemTable {
  DemDesc one;
  const DemDesc* table;    // device, ndem entries (ndem > 1)
  const int32_t* tile_dem; // device, ntiles entries (ndem > 1)
  int ndem;
};

// First-pass modes: unit counts from a direction field; unit counts with the
// directions computed first from z (the direction kernel, then the same tile
// pass); weighted (float) areas from a direction field.
enum UpMode { UP_UNIT_DIR = 0, UP_UNIT_Z = 1, UP_WEIGHTED = 2 };

// Device workspace of one pipeline run (all arrays indexed by global slot id
// = tile * 4T + slot unless noted).
// In-tile frontier strategies of the unit-count tile pass (the weighted pass
// always uses the ring): how a lane whose walk stopped finds its next source.
// Strategy 2 keeps the ring walks in the tiles and replaces the combine's
// top-level queue walk by pointer jumping, for DEMs whose exit forest holds
// very long chains (a channel that crosses tile borders many times).
enum Strategy { STRAT_RING = 0, STRAT_LANE_MASK = 1, STRAT_JUMP = 2, STRAT_COUNT = 3 };

struct Pipe {
  int T;
  int strat;  // Strategy of the unit-count tile pass
  int64_t ntiles, nslots;
  int rounds;
  uint16_t* pex;     // per slot: exit code of the in-tile path
  void* pval;        // per slot: in-tile area at exits (fwd) / path sum (bwd)
  uint32_t* P[2];    // flat combines (adjoint, allocation-free entry): pointer-jumping parents
  void* S;           // per slot: final value at exits, read by the finalising pass
  void* S2;          // flat combines: second value buffer (adjoint) / delta buffer (counts)
  uint32_t* flags;   // combine: per-round "still active" flags, MAX_ROUNDS+2
  uint32_t* status;  // device status word (OR of 1 << d8_status)
  uint32_t* queue;   // tile work-queue counters (one per stage)
  uint16_t* xid;     // adjoint only: per cell (row-major, W per row) the slot of its tile exit, or NO_EXIT
  uint32_t* list[2]; // adjoint only: the exits still open in the combine's rounds (even / odd)
  const uint32_t* top_in;  // unit counts: inflow entering row 0 from above, per column (or null)
  const uint32_t* bot_in;  // unit counts: inflow entering row H-1 from below, per column (or null)
};
constexpr uint16_t NO_EXIT = 0xFFFFu;

// ---- launchers (d8_flowdir.cu / d8_fwd.cu / d8_bwd.cu) ---------------------
// Each enqueues its kernels on `s` and adds the number of kernel launches it
// made to *nlaunch.
cudaError_t launch_flowdir(const DemTable& dt, int64_t ntiles, int T, int rule, uint32_t* status, cudaStream_t s,
                           int* nlaunch);
cudaError_t launch_up(const DemTable& dt, const Pipe& p, int mode, int rule, cudaStream_t s, int* nlaunch);
// flat pointer-jumping combine of unit counts (the allocation-free entry point)
cudaError_t launch_combine_flat(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_down(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s, int* nlaunch);
// unit counts, one DEM: the inflow entering across its top and bottom rows
// (p.top_in, p.bot_in) added to the tile summaries' exit values before the
// combine
cudaError_t launch_inject_inflow(const DemDesc& d, const Pipe& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_bwd_up(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_combine_bwd(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch);
cudaError_t launch_bwd_down(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch);

// ---- layered combine (d8_combine.cu) --------------------------------------
// Level 0 units are the tiles; a level-l unit is a G x G block of level-(l-1)
// units.  Every level has per-unit perimeter summaries of the same format:
// per perimeter slot the exit code (pex), the in-unit value at exits (pval)
// and, after the down sweep, the final value at exits (fin).  Values are
// uint32 counts (unit weights) or float-float areas (weighted).
constexpr int HMAX = 8;
struct HLevel {
  int S;            // unit side in cells
  int64_t nunits;   // units over all DEMs
  DemTable dt;      // per-DEM unit grid (ntx, nty, tile_base) at this level
  uint16_t* pex;
  void* pval;       // uint32 / ff
  void* fin;        // uint32 / ff
};
struct HTop {  // the top level's solve in global memory (queue method or pointer jumping)
  bool jump;      // pointer jumping instead of the queue walk
  uint32_t* par;
  uint32_t* par2;  // pointer jumping: the second parent buffer
  uint32_t* flags; // pointer jumping: per-round "still active" flags (MAX_ROUNDS + 2)
  uint32_t* deg;  // 8 bytes per slot: unit counts pack children left (high) and value (low);
                  // pointer jumping: this round's additions (value type)
  uint32_t* list;
  uint32_t* counters;  // [0] sources, [1] exits, [2] finished
  uint32_t* status;
};
struct HPlan {
  bool weighted;  // float-float values instead of uint32 counts
  int nlev;  // group levels 1..nlev above the tiles
  HLevel lev[HMAX];
  bool need_top;
  HTop top;
  uint32_t* queue;  // 32 work-queue counters
  uint32_t* status;
};
// group sides of the levels above tiles of side T, for grids up to max_side
int hier_levels(int T, int64_t max_side, int* S, int* G, int max_levels);
cudaError_t launch_combine_hier(const HPlan& hp, cudaStream_t s, int* nlaunch);

// tile passes, unit counts or weighted (d8_unit.cu)
cudaError_t launch_up_unit(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s);
cudaError_t launch_down_unit(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s);

// ---- pit and flat removal (d8_fill.cu)
size_t fill_ws_bytes(int64_t H, int64_t W);
cudaError_t run_fill(const float* z, int64_t H, int64_t W, int64_t ldz, float eps, float* F, int64_t ldF, void* ws,
                     uint32_t* status, cudaStream_t s, int64_t max_rounds, int64_t* rounds_out, bool* timed_out,
                     int* nlaunch);

// shared-memory bytes of the per-tile kernels (0 = configuration unsupported)
size_t up_smem_bytes(int T, int mode);
size_t down_smem_bytes(int T, bool weighted);

}  // namespace d8
