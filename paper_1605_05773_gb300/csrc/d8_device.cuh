// d8_device.cuh -- device helpers shared by the libd8 kernels.
//
// Tile model (the paper's "slave partition", section "The Algorithm"): a DEM of
// H x W cells is cut into T x T tiles (ragged at the right and bottom).  A tile
// is held by one thread block in shared memory, cell (i, j) of the tile at
// local index i*T + j.  The cells on a tile's border are its perimeter; each
// perimeter cell has a fixed "slot" in a 4T-entry per-tile table:
//   top row    (i == 0)          : slot j
//   bottom row (i == th-1 > 0)   : slot T + j
//   left col   (j == 0, 0<i<th-1): slot 2T + i
//   right col  (j == tw-1 > 0, 0<i<th-1): slot 3T + i
// so a tile's perimeter summary is a fixed-stride array and the global slot id
// of a perimeter cell is tile * 4T + slot.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "d8_internal.h"

namespace d8 {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---- direction codes ----------------------------------------------------
// 0..7 = N, NE, E, SE, S, SW, W, NW (row index grows to the south)
__device__ __forceinline__ int code_di(int k) { return (int)((0x01222100u >> (4 * k)) & 0xFu) - 1; }
__device__ __forceinline__ int code_dj(int k) { return (int)((0x00012221u >> (4 * k)) & 0xFu) - 1; }
__device__ __forceinline__ int opposite(int k) { return (k + 4) & 7; }

// fp32 nearest 1/sqrt(2): the diagonal distance factor of the steepest rule
__device__ __forceinline__ float inv_sqrt2_f32() { return __uint_as_float(0x3F3504F3u); }


// ---- compensated fp32 ("float-float") ------------------------------------
struct ff {
  float hi, lo;
};

// Knuth TwoSum of the high parts, error terms folded in, renormalised with
// Fast2Sum.  Explicit _rn intrinsics keep the compiler from contracting or
// reassociating anything.
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bv = __fsub_rn(s, a.hi);
  const float av = __fsub_rn(s, bv);
  float e = __fadd_rn(__fsub_rn(a.hi, av), __fsub_rn(b.hi, bv));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float hi = __fadd_rn(s, e);
  const float lo = __fsub_rn(e, __fsub_rn(hi, s));
  return ff{hi, lo};
}

template <class V>
struct VOps;

template <>
struct VOps<uint32_t> {
  static __device__ __forceinline__ uint32_t zero() { return 0u; }
  static __device__ __forceinline__ uint32_t add(uint32_t a, uint32_t b) { return a + b; }
  static __device__ __forceinline__ void atomic_add(uint32_t* p, uint32_t v) { atomicAdd(p, v); }
  static __device__ __forceinline__ bool nonzero(uint32_t v) { return v != 0u; }
};


// ---- asynchronous global -> shared copies (bytes in flight cost no registers)
// nbytes < copy size zero-fills the rest; a 16-byte copy needs both addresses
// 16-byte aligned, a 4-byte copy 4-byte aligned
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int nbytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(nbytes)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int nbytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(nbytes)
               : "memory");
}
// Shared-memory atomic add with acquire-release semantics at CTA scope: the
// writes this thread made before it are visible to any thread whose later
// acquire atomic on the same word reads its result (or a later one), and the
// reads this thread makes after it see what those earlier releasers wrote.
__device__ __forceinline__ uint32_t atomic_add_acq_rel_cta(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;\n"
               : "=r"(old)
               : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(v)
               : "memory");
  return old;
}

// The same in global memory at GPU scope.
__device__ __forceinline__ uint32_t atomic_add_acq_rel_gpu(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;\n" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// DEM of a tile, by value so its fields can live in registers
__device__ __forceinline__ DemDesc dem_of(const DemTable& t, int64_t tile) {
  if (t.ndem == 1) return t.one;
  return t.table[t.tile_dem[tile]];
}

__device__ __forceinline__ uint32_t* pick(uint32_t* a, uint32_t* b, int second) { return second ? b : a; }

// ---- tile geometry --------------------------------------------------------
struct TileGeo {
  int64_t i0, j0;  // global origin
  int th, tw;      // extent (ragged at the right/bottom)
};

__device__ __forceinline__ TileGeo tile_geo(const DemDesc& d, int64_t local_tile, int T) {
  TileGeo g;
  const int64_t ty = local_tile / d.ntx, tx = local_tile % d.ntx;
  g.i0 = ty * T;
  g.j0 = tx * T;
  g.th = (int)min64(T, d.H - g.i0);
  g.tw = (int)min64(T, d.W - g.j0);
  return g;
}

// slot of perimeter cell (i, j) of a th x tw tile, or -1 for an inner cell
__device__ __forceinline__ int slot_of(int i, int j, int th, int tw, int T) {
  if (i == 0) return j;
  if (i == th - 1) return T + j;
  if (j == 0) return 2 * T + i;
  if (j == tw - 1) return 3 * T + i;
  return -1;
}

// cell of slot s, or false if the slot is unused for this tile extent
__device__ __forceinline__ bool slot_cell(int s, int th, int tw, int T, int& i, int& j) {
  if (s < T) {
    i = 0;
    j = s;
    return j < tw;
  }
  if (s < 2 * T) {
    i = th - 1;
    j = s - T;
    return th > 1 && j < tw;
  }
  if (s < 3 * T) {
    i = s - 2 * T;
    j = 0;
    return i >= 1 && i <= th - 2;
  }
  i = s - 3 * T;
  j = tw - 1;
  return tw > 1 && i >= 1 && i <= th - 2;
}

// Global slot id of the cell (gi, gj) of DEM d (the cell must lie on the
// perimeter of its tile).
__device__ __forceinline__ int64_t global_slot(const DemDesc& d, int64_t gi, int64_t gj, int T) {
  const int64_t ty = gi / T, tx = gj / T;
  const int i = (int)(gi - ty * T), j = (int)(gj - tx * T);
  const int th = (int)min64(T, d.H - ty * T), tw = (int)min64(T, d.W - tx * T);
  return (d.tile_base + ty * d.ntx + tx) * (int64_t)(4 * T) + slot_of(i, j, th, tw, T);
}

// ---- perimeter exit codes (per slot, uint16) ------------------------------
// PEX_EXIT | k : the cell itself leaves the tile, towards direction k
// PEX_TERM     : the cell's in-tile path ends inside the tile (outlet, sink,
//                off-grid target)
// otherwise    : slot of the perimeter cell where the in-tile path leaves
constexpr uint16_t PEX_EXIT = 0x8000u;
constexpr uint16_t PEX_TERM = 0x7FFFu;

// ---- per-cell class flags in shared memory ---------------------------------
constexpr uint8_t CL_IN = 0x08;      // target inside the tile; bits 0..2 = code
constexpr uint8_t CL_EXIT = 0x10;    // target in another tile; bits 0..2 = code
constexpr uint8_t CL_TERM = 0x20;    // path ends here
constexpr uint8_t CL_ABSENT = 0x40;  // outside a ragged tile

// Classify a code of cell (i, j) of a tile: in-tile target, exit, or end.
__device__ __forceinline__ uint8_t classify(int code, int i, int j, const TileGeo& g, const DemDesc& d,
                                            uint32_t* status) {
  if (code > 9) {
    atomicOr(status, 1u << D8_ERR_ARG);
    return CL_TERM;
  }
  if (code >= 8) return CL_TERM;
  const int di = code_di(code), dj = code_dj(code);
  const int64_t gi = g.i0 + i + di, gj = g.j0 + j + dj;
  if (gi < 0 || gj < 0 || gi >= d.H || gj >= d.W) return CL_TERM;
  const int li = i + di, lj = j + dj;
  if (li >= 0 && lj >= 0 && li < g.th && lj < g.tw) return (uint8_t)(CL_IN | code);
  return (uint8_t)(CL_EXIT | code);
}

__device__ __forceinline__ void set_status(uint32_t* status, int code) { atomicOr(status, 1u << code); }

// Tile work queue: persistent blocks take tile indices until the n tiles run
// out.  Block b starts with tile b; later indices come from a device counter
// (zeroed before the launch) offset by the grid size.  With plenty of tiles
// per block (more than 4), thread 0 fetches one index ahead: the atomic for
// the next tile is issued when the current one is handed out and consumed at
// the next call, so its round trip to L2 overlaps the current tile's work.
// With few tiles per block a fetched-ahead index would sit reserved behind a
// busy block, so then each index is fetched when it is needed.
struct TileQueue {
  uint32_t* q;
  bool look;
  uint32_t ahead = 0;  // thread 0: the index fetched for the next call
  __device__ TileQueue(uint32_t* queue, int64_t n) : q(queue), look(n > 4 * (int64_t)gridDim.x) {}
  __device__ __forceinline__ int64_t first() {
    __syncthreads();
    if (look && threadIdx.x == 0) ahead = gridDim.x + atomicAdd(q, 1u);
    return blockIdx.x;
  }
  __device__ __forceinline__ int64_t next() {
    __shared__ int64_t sh_tile;
    __syncthreads();
    if (threadIdx.x == 0) {
      const uint32_t now = look ? ahead : gridDim.x + atomicAdd(q, 1u);
      if (look) ahead = gridDim.x + atomicAdd(q, 1u);
      sh_tile = (int64_t)now;
    }
    __syncthreads();
    return sh_tile;
  }
};

}  // namespace d8
