// d8_unit.cu -- the unit-count tile passes (the headline path).
//
//  k_up_unit    per tile: codes from the direction field, the in-tile
//               dependency count (Algorithm 1), the in-tile up-slope counts
//               with inflow from other tiles unknown = 0 (Algorithms 2-4),
//               written to A, and the perimeter summary.
//  k_fin_unit   per tile finalise (Algorithms 7-8): A already holds the
//               in-tile counts; the resolved inflow from neighbouring tiles
//               is pushed down the in-tile paths it reaches and added there.
//
// Layout choices for GB300:
//  * one packed 32-bit word per cell in shared memory holds the cell's
//    in-tile count, its number of unfinished in-tile inputs, its D8 code and
//    class bits.  One shared atomicAdd both delivers a finished cell's count
//    to its down-slope cell and tells the sender whether it was the last
//    input; only then does the sender continue (Algorithm 2's tail
//    recursion).  The in-tile count of a 128 x 128 tile fits in 16 bits;
//  * the walks are latency-bound, so shared memory per tile is kept small
//    (the word array, a uint16 segment record per cell and a 64-entry ring
//    of pending sources per warp: 24.6 KB for 64 x 64) to fit eight tiles per
//    SM, and the launch bounds hold registers to the same eight;
//  * each warp feeds idle lanes from its ring with ballots (no shared
//    atomics), refilling the ring by scanning its own cells as it goes;
//  * every walk records its segment (the cells it finished) and where the
//    segment ended (at a tile exit or path end, or at the junction where
//    another walk took over), so the exit of any perimeter cell's in-tile
//    path is a short chase over segment records instead of a walk over cells;
//  * the first pass writes the in-tile counts to A, so the finalising pass
//    only walks the paths down-slope of the perimeter cells that receive
//    inflow from other tiles, adding that inflow along them, instead of
//    re-running the whole tile.
#include <type_traits>

#include "d8_device.cuh"

namespace d8 {
namespace unit {

constexpr int NTU = 128;  // threads per tile block (4 warps)
constexpr int NTW = 256;  // threads per weighted tile block of side 64 and up (8 warps)
// Threads per tile of the first pass: a weighted 64 x 64 tile needs 49 KB of
// shared memory (4 per SM), so weighted tiles of 64 and up get 8 warps each
// to keep enough warps resident; 32 x 32 tiles have too few cells for that.
template <int T, bool WT>
struct UpThreads {
  static constexpr int N = (WT && T >= 64) ? NTW : NTU;
};
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int RING = 64;  // pending sources per warp (a power of two > 63)
constexpr int UNIT_STEPS = 3;  // walk steps per loop iteration (unit counts)
constexpr int NTF = 256;  // threads per finalising block (its walks are few; the loads want warps)

// In-tile offset of direction k (N, NE, E, SE, S, SW, W, NW) for row stride T.
// For T <= 64 the eight offsets fit in signed bytes of one 64-bit constant
// held in registers (a __constant__ table indexed by each lane's own code
// would be serialised across the distinct addresses of a warp).
template <int T>
__device__ __forceinline__ int toff_tab(int k) {
  if (T == 64) return (int)(signed char)(0xBFFF3F404101C1C0ull >> (8 * k));
  if (T == 32) return (int)(signed char)(0xDFFF1F202101E1E0ull >> (8 * k));
  const int di = (int)((0x01222100u >> (4 * k)) & 0xFu) - 1;
  const int dj = (int)((0x00012221u >> (4 * k)) & 0xFu) - 1;
  return di * T + dj;
}

// The packed per-cell word.  Inputs still to arrive sit in bits 28..31, so
// one unsigned compare of the value an atomic returns tells the last arriver
// (left was 1 iff old < 2 << 28); IN (target inside the tile) is bit 25,
// EXIT (target in another tile) bit 26; the count starts at bit 0.  For
// T <= 64 the count takes 13 bits and bits 13..24 hold the in-tile index of
// the down-slope cell (IN cells) or the code (others), so a walk step reads
// its next cell with one shift and mask.  A 128 x 128 tile needs 15 count
// bits and an index of 14, so there bits 15..18 hold the code instead and the
// next cell is computed from it.
constexpr uint32_t W_IN = 1u << 25, W_EXIT = 1u << 26, W_LEFT1 = 1u << 28;
// Weighted tiles keep no count in the word: bits 0..7 hold which neighbours
// are in-tile inputs (bit k: the input lies in direction k) and bit 27 marks a
// cell present in the tile.  A source has no input and nothing left.
constexpr uint32_t W_PRES = 1u << 27, W_SRC_W = 0xF0000000u | W_PRES | 0xFFu;
// Unit words use bit 27 to mark a cell whose inputs were all delivered by the
// source sweep (the cell then starts a walk).
constexpr uint32_t W_READY = 1u << 27;
template <int T>
struct WL {
  static constexpr bool IDX = T <= 64;
  static constexpr int CB = IDX ? 13 : 15;  // count bits; the next field starts here
  static constexpr uint32_t CNT = (1u << CB) - 1;
  static constexpr uint32_t SRC_MASK = 0xF0000000u | CNT;  // a source: count 1, nothing left
  __device__ static __forceinline__ uint32_t cnt(uint32_t w) { return w & CNT; }
  __device__ static __forceinline__ bool last(uint32_t old) { return old < 2 * W_LEFT1; }
  __device__ static __forceinline__ int code(uint32_t w) { return (int)((w >> CB) & 0xFu); }  // non-IN cells
  __device__ static __forceinline__ int next(uint32_t w, int c) {
    if (IDX) return (int)((w >> CB) & (uint32_t)(T * T - 1));
    return c + toff_tab<T>(code(w) & 7);  // (only used for IN cells, codes 0..7)
  }
};

// Segment records (one uint16 per cell).  A finished non-source cell holds
// the source cell whose walk finished it.  A source cell holds its walk's end
// record: SEG_REC | SEG_END | cell (the walk ended at that cell: a tile exit
// or a path end, told apart by the cell's class bits) or SEG_REC | cell (the
// walk stopped before that junction cell, which another walk finished).
constexpr uint16_t SEG_REC = 0x8000u, SEG_END = 0x4000u;


// Bits of the neighbours of tile cell (i, j) that lie outside a th x tw tile.
__device__ __forceinline__ uint32_t row_off_mask(int i, int th) {
  return (i == 0 ? 0x83u : 0u) | (i == th - 1 ? 0x38u : 0u);  // N, NE, NW / SE, S, SW
}
__device__ __forceinline__ uint32_t col_off_mask(int j, int tw) {
  return (j == 0 ? 0xE0u : 0u) | (j == tw - 1 ? 0x0Eu : 0u);  // SW, W, NW / NE, E, SE
}

// Per-cell bookkeeping once its code is known: the cell's own word (count 1,
// or the present bit for weighted tiles; next field; class bits) and, when its
// target is inside the tile, one more input for the target (and, weighted,
// the direction it arrives from).  A code 0..7 whose target is outside the tile is an
// exit when the target cell (gi, gj) + offset is on the grid, otherwise the
// path ends there; that test runs only for those perimeter cells.
template <int T, bool WT>
__device__ __forceinline__ void add_cell(uint32_t* word, int c, int code, uint32_t off_mask, int64_t gi, int64_t gj,
                                         const DemDesc& d, uint32_t* status) {
  using W = WL<T>;
  uint32_t own = WT ? W_PRES : 1u;
  if (code < 8) {
    if (!((off_mask >> code) & 1u)) {
      const int t = c + toff_tab<T>(code);
      atomicAdd(&word[t], W_LEFT1 | (WT ? 1u << opposite(code) : 0u));
      own |= W_IN | ((uint32_t)(W::IDX ? t : code) << W::CB);
    } else {
      const int64_t ti = gi + code_di(code), tj = gj + code_dj(code);
      if (ti >= 0 && tj >= 0 && ti < d.H && tj < d.W) own |= W_EXIT;
      own |= (uint32_t)code << W::CB;
    }
  } else {
    if (code > 9) {
      set_status(status, D8_ERR_ARG);
      code = 10;
    }
    own |= (uint32_t)code << W::CB;
  }
  atomicAdd(&word[c], own);
}

template <int T, bool WT>
struct UpLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_word = 0;
  static constexpr size_t off_seg = TT * 4;             // unit counts only (weighted tiles chase next pointers)
  static constexpr size_t off_ring = off_seg + (WT ? 0 : TT * 2);  // one ring of RING entries per warp
  static constexpr size_t off_misc = off_ring + (size_t)(UpThreads<T, WT>::N / 32) * RING * 2;
  static constexpr size_t off_val = off_misc + 64;  // weighted: float-float value per cell
  static constexpr size_t bytes = off_val + (WT ? TT * sizeof(ff) : 0);
};

// finalising pass, unit counts: F is the inflow routed through each cell
template <int T>
struct FinLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_f = 0;                     // uint32 per cell: A + inflow
  static constexpr size_t off_code = TT * 4;             // uint8 code per cell
  static constexpr size_t off_rcell = off_code + TT;     // uint16 per perimeter slot
  static constexpr size_t off_rin = off_rcell + (size_t)4 * T * 2;  // uint32 per slot
  static constexpr size_t off_ring = off_rin + (size_t)4 * T * 4;   // uint8 codes around the tile
  static constexpr size_t off_misc = (off_ring + 2 * (T + 2) + 2 * T + 15) / 16 * 16;
  static constexpr size_t bytes = off_misc + 64;
};

// finalising pass, weighted: the inflow routed through each cell as a
// fixed-point number in three 32-bit words (FxLimbs; word 0 of every cell,
// then word 1, then word 2)
template <int T>
struct FinWLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_w = 0;                     // uint32 [3][TT]
  static constexpr size_t off_code = TT * 12;            // uint8 code per cell
  static constexpr size_t off_rcell = off_code + TT;     // uint16 per perimeter slot
  static constexpr size_t off_rin = off_rcell + (size_t)4 * T * 2;  // ff per slot
  static constexpr size_t off_ring = off_rin + (size_t)4 * T * sizeof(ff);  // uint8 codes around the tile
  static constexpr size_t off_misc = (off_ring + 2 * (T + 2) + 2 * T + 15) / 16 * 16;
  static constexpr size_t bytes = off_misc + 64;
};

// Codes of tile g from a given direction field into word[], four consecutive
// cells per thread per step (one 32-bit load when the layout allows); for a
// weighted tile also the weights into val[].
template <int T, bool WT>
__device__ __forceinline__ void tile_codes_from_dir(const DemDesc& d, const TileGeo& g, uint32_t* word, ff* val,
                                                    uint32_t* status) {
  constexpr int NT = UpThreads<T, WT>::N;
  constexpr int NQ = T * T / 4 / NT;  // four-cell groups per thread
  const bool vec = (g.tw == T) && ((reinterpret_cast<uintptr_t>(d.dir) & 3u) == 0) && (d.lddir % 4 == 0);
  // issue every load of this thread before using any (hides the memory latency)
  uint32_t fours[NQ];
#pragma unroll
  for (int r = 0; r < NQ; r++) {
    const int c = (threadIdx.x + r * NT) * 4, i = c / T, j = c - i * T;
    fours[r] = 0;
    if (i < g.th) {
      const uint8_t* src = d.dir + (g.i0 + i) * d.lddir + (g.j0 + j);
      if (vec) {
        fours[r] = __ldg(reinterpret_cast<const unsigned int*>(src));
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (j + k < g.tw) fours[r] |= (uint32_t)src[k] << (8 * k);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < NQ; r++) {
    const int q = threadIdx.x + r * NT;
    const int c = q * 4, i = c / T, j = c - i * T;
    if (i >= g.th) continue;
    const uint32_t four = fours[r];
    const uint32_t rm = row_off_mask(i, g.th);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (j + k >= g.tw) break;
      const int code = (four >> (8 * k)) & 0xFF;
      add_cell<T, WT>(word, c + k, code, rm | col_off_mask(j + k, g.tw), g.i0 + i, g.j0 + j + k, d, status);
    }
    if (WT) {  // each cell's own weight starts its value
      const float* wr = d.w + (g.i0 + i) * d.ldw + (g.j0 + j);
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (j + k < g.tw) val[c + k] = ff{__ldg(wr + k), 0.0f};
    }
  }
}

// A[tile] = the in-tile counts held in word[], four consecutive cells per
// thread per step (one 16-byte store when the layout allows).
template <int T>
__device__ __forceinline__ void store_counts(const DemDesc& d, const TileGeo& g, const uint32_t* word) {
  for (int q = threadIdx.x; q < T * T / 4; q += NTU) {
    const int c = q * 4, i = c / T, j = c - i * T;
    if (i >= g.th) continue;
    uint32_t* dst = static_cast<uint32_t*>(d.A) + (g.i0 + i) * d.ldA + (g.j0 + j);
    const uint4 wq = reinterpret_cast<const uint4*>(word)[q];
    using W = WL<T>;
    const uint4 o = make_uint4(W::cnt(wq.x), W::cnt(wq.y), W::cnt(wq.z), W::cnt(wq.w));
    if (g.tw == T && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
      *reinterpret_cast<uint4*>(dst) = o;
    } else {
      const uint32_t ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (j + k < g.tw) dst[k] = ov[k];
    }
  }
}

// Weighted: A[tile] = the in-tile areas held in val[], rounded to fp32.
template <int T>
__device__ __forceinline__ void store_areas(const DemDesc& d, const TileGeo& g, const ff* val) {
  for (int q = threadIdx.x; q < T * T / 4; q += UpThreads<T, true>::N) {
    const int c = q * 4, i = c / T, j = c - i * T;
    if (i >= g.th) continue;
    float* dst = static_cast<float*>(d.A) + (g.i0 + i) * d.ldA + (g.j0 + j);
    float o[4];
#pragma unroll
    for (int k = 0; k < 4; k++) o[k] = __fadd_rn(val[c + k].hi, val[c + k].lo);
    if (g.tw == T && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
      *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (j + k < g.tw) dst[k] = o[k];
    }
  }
}

// Weighted value of a cell whose inputs have all arrived: its weight plus its
// inputs' values, pulled in N..NW order with compensated adds (deterministic).
template <int T>
__device__ __forceinline__ ff pull_value(const ff* val, int c, uint32_t w) {
  ff v = val[c];
  for (uint32_t m = w & 0xFFu; m; m &= m - 1) v = ff_add(v, val[c + toff_tab<T>(__ffs(m) - 1)]);
  return v;
}

// Perimeter summary of a finished tile: for each perimeter slot, the exit of
// the cell's in-tile path (Algorithms 3-4 seen from the exit side) found by a
// chase over the walks' segment records (resolved records are written back),
// and the in-tile count / area at the slot.
template <int T, bool WT>
__device__ __forceinline__ void perimeter_summary(const TileGeo& g, int64_t t, const uint32_t* word, uint16_t* seg,
                                                  const ff* val, bool cyc, const Pipe& p) {
  using W = WL<T>;
  constexpr int TT = T * T;
  constexpr int NT = UpThreads<T, WT>::N;
  for (int s = threadIdx.x; s < 4 * T; s += NT) {
    int i, j;
    uint16_t pe = PEX_TERM;
    uint32_t pv = 0;
    ff pvw{0.0f, 0.0f};
    if (slot_cell(s, g.th, g.tw, T, i, j)) {
      const int c = i * T + j;
      const uint32_t w = word[c];
      if (WT)
        pvw = val[c];
      else
        pv = W::cnt(w);
      if (w & W_EXIT) {
        pe = (uint16_t)(PEX_EXIT | W::code(w));
      } else if (WT && (w & W_IN) && !cyc) {
        // weighted tiles keep no segment records: follow the next pointers
        int e = c;
        uint32_t we = w;
        for (int guard = 0; (we & W_IN) && guard < TT; guard++) {
          e = W::next(we, e);
          we = word[e];
        }
        if (we & W_EXIT) pe = (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T);
      } else if ((w & W_IN) && !cyc) {
        volatile uint16_t* vs = seg;
        const uint16_t v = vs[c];
        const int hh = (v & SEG_REC) ? c : (int)(v & (TT - 1));
        uint16_t r = (v & SEG_REC) ? v : vs[hh];
        for (int guard = 0; !(r & SEG_END) && guard < TT; guard++) {
          const int jn = r & (TT - 1);  // junction: continue with the walk that finished it
          const uint16_t vj = vs[jn];
          r = (vj & SEG_REC) ? vj : vs[vj & (TT - 1)];
        }
        if (r & SEG_END) {
          vs[hh] = r;  // path compression
          const int e = r & (TT - 1);
          if (word[e] & W_EXIT) pe = (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T);
        } else {
          set_status(p.status, D8_ERR_CYCLE);
        }
      }
    }
    p.pex[t * (4 * T) + s] = pe;
    if (WT)
      static_cast<ff*>(p.pval)[t * (4 * T) + s] = pvw;
    else
      static_cast<uint32_t*>(p.pval)[t * (4 * T) + s] = pv;
  }
}

template <int T, bool WT>
__global__ void __launch_bounds__(UpThreads<T, WT>::N, WT ? 4 : 8) k_up_unit(DemTable dt, Pipe p) {
  constexpr int NT = UpThreads<T, WT>::N;
  using L = UpLayout<T, WT>;
  using W = WL<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* word = reinterpret_cast<uint32_t*>(sm + L::off_word);
  uint16_t* seg = reinterpret_cast<uint16_t*>(sm + L::off_seg);
  uint16_t* ring = reinterpret_cast<uint16_t*>(sm + L::off_ring) + (threadIdx.x >> 5) * RING;
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  ff* val = reinterpret_cast<ff*>(sm + L::off_val);  // weighted only
  constexpr int TT = T * T;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;

  TileQueue tq(p.queue + 0, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    uint4* w4 = reinterpret_cast<uint4*>(word);
    for (int c = threadIdx.x; c < TT / 4; c += NT) w4[c] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) misc[0] = 0;
    __syncthreads();
    tile_codes_from_dir<T, WT>(d, g, word, val, p.status);  // Algorithm 1
    __syncthreads();
    int done = 0;
    if (!WT) {
      // Source sweep (unit counts).  A source (count 1, no input) would start
      // a walk whose first step delivers its 1 to its target; on terrain two
      // cells in five are sources and most such walks end after that step.
      // So every source delivers in one data-parallel pass instead, and the
      // source that delivers a target's last input marks the target READY:
      // walks start only at READY cells (one cell in seven), carrying their
      // count.  A swept source's segment record says its one-step walk stopped
      // before its target (or ended at the source itself).
#pragma unroll 4
      for (int r = 0; r < TT / NT; r++) {
        const int c = threadIdx.x + r * NT;
        const uint32_t w = word[c];
        if ((w & W::SRC_MASK) != 1u) continue;
        done++;
        if (w & W_IN) {
          const int s = W::next(w, c);
          const uint32_t old = atomicAdd(&word[s], 1u - W_LEFT1);
          seg[c] = (uint16_t)(SEG_REC | s);
          if (W::last(old)) atomicOr(&word[s], W_READY);
        } else {
          seg[c] = (uint16_t)(SEG_REC | SEG_END | c);
        }
      }
      __syncthreads();
    }
    // Algorithm 2.  Every lane walks down-slope from a start cell while it is
    // the last input to arrive at the next cell; a lane whose walk stopped
    // takes the warp's next pending start.  Pending starts sit in a per-warp
    // ring, refilled by scanning the warp's own cells (c = lane + 32 w + NT r)
    // a row at a time with a ballot.  Unit counts start at READY cells (a
    // cell reached by a walk's last arrival never carries the mark, so a scan
    // running behind the walks never takes it).  Weighted tiles start at
    // sources (no input left, present) and carry values instead of counts: a
    // finished cell stores its value before the atomic that publishes its
    // arrival (block fence between), and the last arriver pulls its inputs'
    // values after it (fence again).
    {
      int r = 0, head = 0, tail = 0, cur = -1, h = 0;
      uint32_t acc = 0, wv = 0;
      ff v{0.0f, 0.0f};
      for (;;) {
        while (tail - head < 32 && r < TT / NT) {  // at most RING - 1 pending
          const int c = threadIdx.x + r * NT;
          const bool src = WT ? (word[c] & W_SRC_W) == W_PRES : (word[c] & W_READY) != 0u;
          const unsigned m = __ballot_sync(FULL, src);
          if (src) ring[(tail + __popc(m & lt)) & (RING - 1)] = (uint16_t)c;
          tail += __popc(m);
          r++;
        }
        __syncwarp();
        const unsigned need = __ballot_sync(FULL, cur < 0);
        if (head < tail) {
          const int idx = head + __popc(need & lt);
          if (cur < 0 && idx < tail) {
            cur = ring[idx & (RING - 1)];
            h = cur;
            wv = word[cur];
            acc = WT ? 1u : W::cnt(wv);  // a READY cell's count (unit) / a source
            if (WT) v = val[cur];  // its weight
            done++;
          }
          head = min(head + __popc(need), tail);
        } else if (need == FULL) {
          break;
        }
        // unit counts: a lane whose walk continues takes a second step in the
        // same iteration, so the refill and hand-out above are paid once per
        // two steps of the long walks
#pragma unroll
        for (int k = 0; k < (WT ? 2 : UNIT_STEPS); k++) {
          if (cur < 0) break;
          if (WT) val[cur] = v;
          if (wv & W_IN) {
            const int s = W::next(wv, cur);
            // weighted: the value store above is released by the atomic, and
            // the last arriver's pull below is ordered after it (acquire)
            const uint32_t old = WT ? atomic_add_acq_rel_cta(&word[s], 0u - W_LEFT1) : atomicAdd(&word[s], acc - W_LEFT1);
            if (W::last(old)) {  // last input to arrive: continue there
              if (!WT) seg[s] = (uint16_t)h;
              if (WT) {
                v = pull_value<T>(val, s, old);
              } else {
                acc += W::cnt(old);
              }
              wv = old;
              cur = s;
              done++;
            } else {
              if (!WT) seg[h] = (uint16_t)(SEG_REC | s);
              cur = -1;
            }
          } else {
            if (!WT) seg[h] = (uint16_t)(SEG_REC | SEG_END | cur);
            cur = -1;
          }
        }
      }
    }
    // a cell never finished lies on or below a cycle of the direction field
    atomicAdd(&misc[0], done);
    __syncthreads();
    const bool cyc = misc[0] != g.th * g.tw;
    if (threadIdx.x == 0 && cyc) set_status(p.status, D8_ERR_CYCLE);
    // in-tile counts / areas (inflow from other tiles = 0) go to A now; the
    // finalising pass adds the inflow only where some reaches
    if (WT)
      store_areas<T>(d, g, val);
    else
      store_counts<T>(d, g, word);
    perimeter_summary<T, WT>(g, t, word, seg, val, cyc, p);
  }
}

// The unit-count tile pass with the lane-mask walk (frontier strategy 1).
// Same codes phase, walks, segment records and perimeter summary as
// k_up_unit; only the way idle lanes find sources differs.  Thread t owns
// the cells t + NTU * r (r = 0 .. T*T/NTU - 1) and, once the in-tile input
// counts are complete, holds which of them are sources as a bit mask in
// registers.  A lane whose walk stopped takes its own next source (find-first-
// set, no warp vote); only when a lane has none left does the warp pair its
// idle lanes with lanes that still have spare sources, each donor handing over
// its last one through a 32-entry per-warp mailbox in shared memory.  The loop
// body is a handful of instructions when no lane is out of work, against a
// ballot-driven ring refill on every step in k_up_unit.
template <int T>
struct LaneMask {
  static constexpr int CPT = T * T / NTU;     // cells per thread
  static constexpr int NM = (CPT + 31) / 32;  // 32-bit mask words per thread
};

template <int T>
__global__ void __launch_bounds__(NTU, 8) k_up_lm(DemTable dt, Pipe p) {
  using L = UpLayout<T, false>;
  using W = WL<T>;
  constexpr int TT = T * T;
  constexpr int CPT = LaneMask<T>::CPT, NM = LaneMask<T>::NM;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* word = reinterpret_cast<uint32_t*>(sm + L::off_word);
  uint16_t* seg = reinterpret_cast<uint16_t*>(sm + L::off_seg);
  uint16_t* offer = reinterpret_cast<uint16_t*>(sm + L::off_ring) + (threadIdx.x >> 5) * 32;
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;

  TileQueue tq(p.queue + 0, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    uint4* w4 = reinterpret_cast<uint4*>(word);
    for (int c = threadIdx.x; c < TT / 4; c += NTU) w4[c] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) misc[0] = 0;
    __syncthreads();
    tile_codes_from_dir<T, false>(d, g, word, nullptr, p.status);  // Algorithm 1
    __syncthreads();
    // this thread's sources: count 1 and no input left (absent cells of a
    // ragged tile have count 0)
    uint32_t m[NM];
#pragma unroll
    for (int k = 0; k < NM; k++) m[k] = 0u;
#pragma unroll
    for (int r = 0; r < CPT; r++)
      m[r / 32] |= (uint32_t)((word[threadIdx.x + NTU * r] & W::SRC_MASK) == 1u) << (r % 32);
    // Algorithm 2: walk down-slope while last to arrive
    int done = 0;
    {
      int cur = -1, h = 0;
      uint32_t acc = 0, wv = 0;
      for (;;) {
        if (cur < 0) {
#pragma unroll
          for (int k = 0; k < NM; k++) {
            if (m[k]) {
              const int r = __ffs(m[k]) - 1;
              m[k] &= m[k] - 1u;
              cur = threadIdx.x + NTU * (32 * k + r);
              break;
            }
          }
          if (cur >= 0) {
            h = cur;
            wv = word[cur];
            acc = 1;
            done++;
          }
        }
        const unsigned idle = __ballot_sync(FULL, cur < 0);
        if (idle) {
          bool spare = false;
#pragma unroll
          for (int k = 0; k < NM; k++) spare |= (m[k] != 0u);
          const unsigned donors = __ballot_sync(FULL, spare);
          if (!donors) {
            if (idle == FULL) break;
          } else {
            const int ni = __popc(idle), nd = __popc(donors);
            if (spare && __popc(donors & lt) < ni) {  // hand over the last own source
#pragma unroll
              for (int k = NM - 1; k >= 0; k--) {
                if (m[k]) {
                  const int r = 31 - __clz(m[k]);
                  m[k] &= ~(1u << r);
                  offer[__popc(donors & lt)] = (uint16_t)(threadIdx.x + NTU * (32 * k + r));
                  break;
                }
              }
            }
            __syncwarp();
            if (cur < 0 && __popc(idle & lt) < nd) {
              cur = offer[__popc(idle & lt)];
              h = cur;
              wv = word[cur];
              acc = 1;
              done++;
            }
            __syncwarp();  // the mailbox is read before it is written again
          }
        }
        if (cur >= 0) {
          if (wv & W_IN) {
            const int s = W::next(wv, cur);
            const uint32_t old = atomicAdd(&word[s], acc - W_LEFT1);
            if (W::last(old)) {  // last input to arrive: continue there
              seg[s] = (uint16_t)h;
              acc += W::cnt(old);
              wv = old;
              cur = s;
              done++;
            } else {
              seg[h] = (uint16_t)(SEG_REC | s);
              cur = -1;
            }
          } else {
            seg[h] = (uint16_t)(SEG_REC | SEG_END | cur);
            cur = -1;
          }
        }
      }
    }
    atomicAdd(&misc[0], done);
    __syncthreads();
    const bool cyc = misc[0] != g.th * g.tw;
    if (threadIdx.x == 0 && cyc) set_status(p.status, D8_ERR_CYCLE);
    store_counts<T>(d, g, word);
    perimeter_summary<T, false>(g, t, word, seg, nullptr, cyc, p);
  }
}

// The codes of tile g copied straight into code[] (16 at a time, by
// asynchronous copies when the rows allow) and the codes of the one-cell ring
// around it into ring[] (top T+2, bottom T+2, left T, right T; 0xFF off the
// grid), all requested before any is waited for.  Returns once this thread's
// copies have landed; the caller's barrier makes them visible to the block.
template <int T>
__device__ __forceinline__ void fin_codes(const DemDesc& d, const TileGeo& g, uint8_t* code, uint8_t* ring) {
  constexpr int TT = T * T;
  const bool vecD = g.tw == T && ((reinterpret_cast<uintptr_t>(d.dir) & 15u) == 0) && (d.lddir % 16 == 0);
  for (int q = threadIdx.x; q < TT / 16; q += NTF) {  // 16 codes at a time
    const int c = q * 16, i = c / T, j = c - i * T;
    uint8_t* dst = code + c;
    if (i >= g.th) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(0x08080808u, 0x08080808u, 0x08080808u, 0x08080808u);
      continue;
    }
    const uint8_t* src = d.dir + (g.i0 + i) * d.lddir + (g.j0 + j);
    if (vecD) {
      cp_async16(dst, src, 16);
    } else {
#pragma unroll 4
      for (int k = 0; k < 16; k++) dst[k] = j + k < g.tw ? src[k] : (uint8_t)8;
    }
  }
  cp_async_commit();
  for (int q = threadIdx.x; q < 2 * (T + 2) + 2 * T; q += NTF) {
    int li, lj;
    if (q < T + 2) {
      li = -1;
      lj = q - 1;
    } else if (q < 2 * (T + 2)) {
      li = g.th;
      lj = q - (T + 2) - 1;
    } else if (q < 2 * (T + 2) + T) {
      li = q - 2 * (T + 2);
      lj = -1;
    } else {
      li = q - 2 * (T + 2) - T;
      lj = g.tw;
    }
    const int64_t gi = g.i0 + li, gj = g.j0 + lj;
    uint8_t v = 0xFF;
    if (gi >= 0 && gj >= 0 && gi < d.H && gj < d.W && li <= g.th && lj <= g.tw && (q < 2 * (T + 2) || li < g.th))
      v = d.dir[gi * d.lddir + gj];
    ring[q] = v;
  }
  cp_async_wait<0>();
}

// code of the cell (li, lj) just outside tile g, from the ring
template <int T>
__device__ __forceinline__ uint32_t fin_ring_code(const uint8_t* ring, const TileGeo& g, int li, int lj) {
  if (li < 0) return ring[lj + 1];
  if (li >= g.th) return ring[(T + 2) + lj + 1];
  if (lj < 0) return ring[2 * (T + 2) + li];
  return ring[2 * (T + 2) + T + li];
}

// Algorithms 7-8 restricted to where they change anything.  The final count
// is A(c) + F(c), where A holds the in-tile counts and F(c) is the inflow
// from other tiles routed through c.  Inflow enters a tile only at its
// receivers (perimeter cells with an up-slope neighbour in another tile) and
// follows the unique down-slope path from there, so F(c) is the sum of the
// receivers' inflows over the receivers whose in-tile path passes through c.
// Each receiver therefore walks its path once adding its inflow to every cell
// on it: additions commute, so the walks need no ordering between them and
// no reply from the shared atomics, and only the cells down-slope of a
// receiver (about a sixth of a 64 x 64 tile on fractal terrain) are touched.
// The work is the summed length of the receivers' in-tile paths (at most
// 4T * T^2 for adversarial fields, about the sub-forest size on terrain).
//
// Memory: the tile's codes and the codes of the one-cell ring around it are
// requested together (asynchronous copies into shared memory), so a tile
// costs one round trip for them, one for the receivers' resolved inflows and
// a read-modify-write of the 16-byte quads of A where the inflow is non-zero.  (Reading
// the tile's whole A up front instead, into the array the walks add to, was
// slower: the sparse read-modify-write moves fewer bytes.)
template <int T>
__global__ void __launch_bounds__(NTF, 8) k_fin_unit(DemTable dt, Pipe p) {
  using L = FinLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* F = reinterpret_cast<uint32_t*>(sm + L::off_f);  // inflow through each cell
  uint8_t* code = sm + L::off_code;
  uint16_t* rcell = reinterpret_cast<uint16_t*>(sm + L::off_rcell);
  uint32_t* rin = reinterpret_cast<uint32_t*>(sm + L::off_rin);
  uint8_t* ring = sm + L::off_ring;        // codes around the tile: top T+2, bottom T+2, left T, right T
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  const uint32_t* xval = static_cast<const uint32_t*>(p.S);
  constexpr int TT = T * T;
  constexpr int NQ = TT / 4 / NTF > 0 ? TT / 4 / NTF : 1;  // quads per thread in the write-back

  // F starts at zero; every tile leaves the words it touched at zero again
  for (int q = threadIdx.x; q < TT / 4; q += NTF) reinterpret_cast<uint4*>(F)[q] = make_uint4(0, 0, 0, 0);
  TileQueue tq(p.queue + 1, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    if (threadIdx.x == 0) misc[0] = 0;
    fin_codes<T>(d, g, code, ring);
    __syncthreads();
    // Algorithm 7: the receivers and their resolved inflow, listed
    for (int s = threadIdx.x; s < 4 * T; s += NTF) {
      int i, j;
      if (!slot_cell(s, g.th, g.tw, T, i, j)) continue;
      uint32_t in = 0;
      bool any = false;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int li = i + code_di(k), lj = j + code_dj(k);
        if (li >= 0 && lj >= 0 && li < g.th && lj < g.tw) continue;
        if (fin_ring_code<T>(ring, g, li, lj) != (uint32_t)opposite(k)) continue;  // also rejects cells off the grid
        in += xval[global_slot(d, g.i0 + li, g.j0 + lj, T)];
        any = true;
      }
      // flow entering across the grid's first or last row (a strip)
      if (p.top_in && g.i0 + i == 0 && p.top_in[g.j0 + j]) {
        in += p.top_in[g.j0 + j];
        any = true;
      }
      if (p.bot_in && g.i0 + i == d.H - 1 && p.bot_in[g.j0 + j]) {
        in += p.bot_in[g.j0 + j];
        any = true;
      }
      if (any) {
        const int r = atomicAdd(&misc[0], 1);
        rcell[r] = (uint16_t)(i * T + j);
        rin[r] = in;
      }
    }
    __syncthreads();
    const int nrec = misc[0];
    // Algorithm 8 on the receivers' paths (a path inside one tile has at most
    // T^2 cells; the bound only matters for a field with a cycle, which the
    // first pass reports)
    for (int r = threadIdx.x; r < nrec; r += NTF) {
      const uint32_t in = rin[r];
      int c = rcell[r], i = c / T, j = c & (T - 1);
      atomicAdd(&F[c], in);
      for (int step = 0; step < TT; step++) {
        const int k = code[c];
        if (k >= 8) break;
        i += code_di(k);
        j += code_dj(k);
        if ((unsigned)i >= (unsigned)g.th || (unsigned)j >= (unsigned)g.tw) break;
        c = i * T + j;
        atomicAdd(&F[c], in);
      }
    }
    __syncthreads();
    // A += F where F is non-zero; those F words go back to zero
#pragma unroll
    for (int r = 0; r < NQ; r++) {
      const int q = threadIdx.x + r * NTF;
      const uint4 f = reinterpret_cast<const uint4*>(F)[q];
      if (!(f.x | f.y | f.z | f.w)) continue;
      reinterpret_cast<uint4*>(F)[q] = make_uint4(0, 0, 0, 0);
      const int c = q * 4, i = c / T, j = c - i * T;
      if (i >= g.th) continue;
      uint32_t* dst = static_cast<uint32_t*>(d.A) + (g.i0 + i) * d.ldA + (g.j0 + j);
      if (g.tw == T && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
        uint4 a = *reinterpret_cast<uint4*>(dst);
        a.x += f.x;
        a.y += f.y;
        a.z += f.z;
        a.w += f.w;
        *reinterpret_cast<uint4*>(dst) = a;
      } else {
        const uint32_t fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (j + k < g.tw && fv[k]) dst[k] += fv[k];
      }
    }
  }
}

// 96-bit two's-complement fixed point, three 32-bit words (w0 lowest).
struct fx96 {
  uint32_t w0, w1, w2;
};

// round(f * 2^q) (ties away from zero) for a finite f with |f| 2^q < 2^94
__device__ __forceinline__ fx96 fx96_of(float f, int q) {
  const uint32_t bits = __float_as_uint(f);
  const int E = (int)((bits >> 23) & 0xFFu);
  const uint32_t mant = (bits & 0x7FFFFFu) | (E ? 0x800000u : 0u);
  const int s = (E ? E : 1) - 150 + q;  // f * 2^q = mant * 2^s
  uint64_t lo = 0;
  uint32_t hi = 0;
  if (mant != 0u) {
    if (s >= 64) {
      hi = mant << (s - 64);
    } else if (s >= 0) {
      lo = (uint64_t)mant << s;
      hi = s > 40 ? (uint32_t)(mant >> (64 - s)) : 0u;
    } else if (s > -26) {
      lo = ((uint64_t)mant + (1ull << (-s - 1))) >> (-s);
    }
  }
  if (bits >> 31) {  // negate the 96-bit value
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1u : 0u);
  }
  return fx96{(uint32_t)lo, (uint32_t)(lo >> 32), hi};
}

__device__ __forceinline__ fx96 fx96_add(fx96 a, fx96 b) {
  const uint64_t al = a.w0 | ((uint64_t)a.w1 << 32), bl = b.w0 | ((uint64_t)b.w1 << 32);
  const uint64_t l = al + bl;
  return fx96{(uint32_t)l, (uint32_t)(l >> 32), a.w2 + b.w2 + (l < al ? 1u : 0u)};
}

// The finalise's per-cell fixed-point accumulator: word 0 is the low 32 bits,
// summed modulo 2^32 with the carry of each addition taken from the atomic's
// reply; words 1 and 2 are limbs of LB bits (unsigned, then signed) summed
// without carries, their spare bits absorbing up to 4T additions (one per
// receiver).  A value x with |x| < 2^(32 + 2 LB) enters as x0 = x mod 2^32,
// x1 = (x >> 32) mod 2^LB, x2 = x >> (32 + LB); the three words then hold the
// exact sum as w0 + w1 2^32 + w2 2^(32 + LB), whatever the order.
template <int T>
struct FxLimbs {
  static constexpr int LB = T >= 128 ? 22 : (T >= 64 ? 23 : 24);  // 4T (LB-bit limb + carry) sums < 2^31
  static constexpr int VB = 32 + 2 * LB;                          // value bits, sign included
};

template <int T>
__device__ __forceinline__ void fx_split(fx96 v, uint32_t& x0, uint32_t& x1, uint32_t& x2) {
  constexpr int LB = FxLimbs<T>::LB;
  const long long rest = (long long)(v.w1 | ((unsigned long long)v.w2 << 32));  // v >> 32, |rest| < 2^(2 LB)
  x0 = v.w0;
  x1 = (uint32_t)rest & ((1u << LB) - 1u);
  x2 = (uint32_t)(int)(rest >> LB);
}

// the three words of a cell back to a 96-bit two's-complement value
template <int T>
__device__ __forceinline__ fx96 fx_join(uint32_t w0, uint32_t w1, uint32_t w2) {
  constexpr int LB = FxLimbs<T>::LB;
  const uint64_t lo = (uint64_t)w0 + ((uint64_t)w1 << 32);  // w1 < 2^31
  const long long t = (long long)(int)w2;                  // signed sum of the top limbs
  const uint64_t tl = (uint64_t)t << (32 + LB);
  const fx96 a{(uint32_t)lo, (uint32_t)(lo >> 32), 0u};
  const fx96 b{(uint32_t)tl, (uint32_t)(tl >> 32), (uint32_t)(t >> (32 - LB))};
  return fx96_add(a, b);
}

// 2^k as fp32 for -126 <= k <= 127 (built from its exponent field: exact)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }

// The fixed-point value (w0, w1, w2) * 2^-q as float-float: the top 62 bits
// of the magnitude rounded to fp32, plus their exact remainder rounded to
// fp32 (a relative error of at most 2^-48 from the remainder's rounding and
// 2^-61 from the bits below the top 62).  2^-q is passed as two powers of two
// p1 * p2 of the normal range; each product below is exact until the last,
// which rounds once.
__device__ __forceinline__ ff fx96_to_ff(uint32_t w0, uint32_t w1, uint32_t w2, float p1, float p2) {
  uint64_t lo = w0 | ((uint64_t)w1 << 32);
  uint32_t hi = w2;
  const bool neg = (hi >> 31) != 0u;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1u : 0u);
  }
  const int p = hi ? 95 - __clz(hi) : (lo ? 63 - __clzll(lo) : 0);  // leading bit
  int sh = 0;
  uint64_t U = lo;
  if (p > 61) {
    sh = p - 61;
    U = (lo >> sh) | (hi ? ((uint64_t)hi << (64 - sh)) : 0ull);
  }
  const float fh = __ull2float_rn(U);  // U < 2^62 rounded to 24 bits: an integer
  const float fl = __ll2float_rn((long long)(U - __float2ull_rn(fh)));
  const float sc = pow2f(sh);  // sh <= 34
  const ff r{__fmul_rn(__fmul_rn(__fmul_rn(fh, sc), p1), p2), __fmul_rn(__fmul_rn(__fmul_rn(fl, sc), p1), p2)};
  return neg ? ff{-r.hi, -r.lo} : r;
}

// Algorithms 7-8 for weighted areas, on the same sub-forest and with the same
// walks as the unit finalise.  The inflow is added in fixed point so that the
// additions stay exact and commute: F(c) is an integer in units of 2^-q held
// in three 32-bit words (FxLimbs: VB = 78 value bits for 64 x 64 tiles).  The
// scale is set per tile from the receivers' inflows: with |in_r| < 2^e_r,
// S = sum over receivers of 2^e_r (an exact integer sum of powers of two, so
// the same in every run) bounds the sum of their magnitudes, and q makes
// S * 2^q <= 2^(VB - 2), so that no partial sum reaches 2^(VB - 1) in
// magnitude.  Each receiver's float-float inflow is rounded once to a
// multiple of 2^-q, an error below 2^-q <= 2^-(VB - 4) * sum |in_r| (2^-74
// for 64 x 64 tiles), far below fp32 resolution even when the tile's inflows
// span twenty orders of magnitude; after that the sums are exact, so the
// result does not depend on the schedule.  Finally A = fp32(A +
// F), F converted to float-float.  A non-finite inflow (non-finite weights)
// cannot be scaled: the tile keeps its in-tile areas and D8_ERR_NONFINITE is
// raised.
template <int T>
__global__ void __launch_bounds__(NTF, T >= 64 ? 4 : 8) k_fin_w(DemTable dt, Pipe p) {
  using L = FinWLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* F0 = reinterpret_cast<uint32_t*>(sm + L::off_w);  // words 0, 1, 2 at F0, F0 + TT, F0 + 2 TT
  uint8_t* code = sm + L::off_code;
  uint16_t* rcell = reinterpret_cast<uint16_t*>(sm + L::off_rcell);
  ff* rin = reinterpret_cast<ff*>(sm + L::off_rin);
  uint8_t* ring = sm + L::off_ring;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + L::off_misc);
  const ff* xval = static_cast<const ff*>(p.S);
  constexpr int TT = T * T;
  constexpr int NQ = TT / 4 / NTF > 0 ? TT / 4 / NTF : 1;  // quads per thread in the write-back

  // F starts at zero; every tile leaves the words it touched at zero again
  for (int q = threadIdx.x; q < 3 * TT / 4; q += NTF) reinterpret_cast<uint4*>(F0)[q] = make_uint4(0, 0, 0, 0);
  TileQueue tq(p.queue + 1, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    unsigned long long* S = reinterpret_cast<unsigned long long*>(misc + 2);
    if (threadIdx.x == 0) {
      misc[0] = 0;  // receivers
      misc[1] = 0;  // largest exponent bound, + 1024
      misc[4] = 0;  // a non-finite inflow seen
      *S = 0ull;
    }
    fin_codes<T>(d, g, code, ring);
    __syncthreads();
    // |x| < 2^ebound(x) for finite x (subnormals and zero: 2^-126)
    auto ebound = [](float x) -> int {
      const int eb = (int)((__float_as_uint(x) >> 23) & 0xFFu);
      return eb == 0 ? -126 : eb - 126;
    };
    // Algorithm 7: the receivers and their resolved inflow, listed
    for (int s = threadIdx.x; s < 4 * T; s += NTF) {
      int i, j;
      if (!slot_cell(s, g.th, g.tw, T, i, j)) continue;
      ff in{0.0f, 0.0f};
      bool any = false;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int li = i + code_di(k), lj = j + code_dj(k);
        if (li >= 0 && lj >= 0 && li < g.th && lj < g.tw) continue;
        if (fin_ring_code<T>(ring, g, li, lj) != (uint32_t)opposite(k)) continue;  // also rejects cells off the grid
        in = ff_add(in, xval[global_slot(d, g.i0 + li, g.j0 + lj, T)]);
        any = true;
      }
      if (any) {
        const int r = (int)atomicAdd(&misc[0], 1u);
        rcell[r] = (uint16_t)(i * T + j);
        rin[r] = in;
        if (isfinite(in.hi))
          atomicMax(&misc[1], (uint32_t)(ebound(in.hi) + 1024));
        else
          misc[4] = 1u;
      }
    }
    __syncthreads();
    const int nrec = (int)misc[0];
    if (misc[4]) {  // an infinite or NaN inflow
      if (threadIdx.x == 0) set_status(p.status, D8_ERR_NONFINITE);
      __syncthreads();  // misc is reset by the next tile
      continue;
    }
    if (nrec == 0) {  // no inflow: A is final
      __syncthreads();
      continue;
    }
    // S = sum of 2^(e_r - emax + 40), each term rounded up to at least 1
    const int emax = (int)misc[1] - 1024;
    for (int r = threadIdx.x; r < nrec; r += NTF) {
      const int sh = ebound(rin[r].hi) - emax + 40;
      atomicAdd(S, sh <= 0 ? 1ull : 1ull << sh);
    }
    __syncthreads();
    // sum |in_r| < S * 2^(emax - 40) <= 2^(ceil(log2 S) + emax - 40)
    const int q = FxLimbs<T>::VB - 2 - (64 - __clzll(*S - 1ull)) - (emax - 40);
    // 2^-q as two powers of two of the normal range (|q| <= 250: -126 <= emax <= 128)
    const float p1 = pow2f(-q / 2), p2 = pow2f(-q - (-q / 2));
    // Algorithm 8 on the receivers' paths, in fixed point
    for (int r = threadIdx.x; r < nrec; r += NTF) {
      const ff in = rin[r];
      uint32_t x0, x1, x2;
      fx_split<T>(fx96_add(fx96_of(in.hi, q), fx96_of(in.lo, q)), x0, x1, x2);
      int c = rcell[r], i = c / T, j = c & (T - 1);
      for (int step = 0; step <= TT; step++) {
        const uint32_t o0 = atomicAdd(F0 + c, x0);
        const int k = code[c];  // the walk goes on while the reply is in flight
        const uint32_t up = x1 + ((o0 + x0 < o0) ? 1u : 0u);
        if (up) atomicAdd(F0 + TT + c, up);
        if (x2) atomicAdd(F0 + 2 * TT + c, x2);
        if (k >= 8) break;
        i += code_di(k);
        j += code_dj(k);
        if ((unsigned)i >= (unsigned)g.th || (unsigned)j >= (unsigned)g.tw) break;
        c = i * T + j;
      }
    }
    __syncthreads();
    // A = fp32(A + F) where F is non-zero; those words go back to zero
#pragma unroll
    for (int rr = 0; rr < NQ; rr++) {
      const int qd = threadIdx.x + rr * NTF;
      const uint4 a4 = reinterpret_cast<const uint4*>(F0)[qd];
      const uint4 b4 = reinterpret_cast<const uint4*>(F0 + TT)[qd];
      const uint4 c4 = reinterpret_cast<const uint4*>(F0 + 2 * TT)[qd];
      if (!(a4.x | a4.y | a4.z | a4.w | b4.x | b4.y | b4.z | b4.w | c4.x | c4.y | c4.z | c4.w)) continue;
      reinterpret_cast<uint4*>(F0)[qd] = make_uint4(0, 0, 0, 0);
      reinterpret_cast<uint4*>(F0 + TT)[qd] = make_uint4(0, 0, 0, 0);
      reinterpret_cast<uint4*>(F0 + 2 * TT)[qd] = make_uint4(0, 0, 0, 0);
      const int c = qd * 4, i = c / T, j = c - i * T;
      if (i >= g.th) continue;
      const uint32_t w0[4] = {a4.x, a4.y, a4.z, a4.w}, w1[4] = {b4.x, b4.y, b4.z, b4.w},
                     w2[4] = {c4.x, c4.y, c4.z, c4.w};
      ff f[4];
      bool on[4];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const fx96 v = fx_join<T>(w0[k], w1[k], w2[k]);
        on[k] = (v.w0 | v.w1 | v.w2) != 0u;
        f[k] = on[k] ? fx96_to_ff(v.w0, v.w1, v.w2, p1, p2) : ff{0.0f, 0.0f};
      }
      float* dst = static_cast<float*>(d.A) + (g.i0 + i) * d.ldA + (g.j0 + j);
      if (g.tw == T && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
        float4 a = *reinterpret_cast<float4*>(dst);
        float* av = reinterpret_cast<float*>(&a);
#pragma unroll
        for (int k = 0; k < 4; k++) {
          const ff r = ff_add(ff{av[k], 0.0f}, f[k]);
          if (on[k]) av[k] = __fadd_rn(r.hi, r.lo);
        }
        *reinterpret_cast<float4*>(dst) = a;
      } else {
#pragma unroll
        for (int k = 0; k < 4; k++) {
          if (j + k >= g.tw || !on[k]) continue;
          const ff r = ff_add(ff{dst[k], 0.0f}, f[k]);
          dst[k] = __fadd_rn(r.hi, r.lo);
        }
      }
    }
  }
}

template <class K>
static unsigned persistent_grid_u(K kernel, int threads, size_t smem, int64_t ntiles) {
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * sms;
  if (g > ntiles) g = ntiles;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int T, bool WT>
static cudaError_t launch_up_unit_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = UpLayout<T, WT>::bytes;
  auto k = (!WT && p.strat == STRAT_LANE_MASK) ? k_up_lm<T> : k_up_unit<T, WT>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<persistent_grid_u(k, UpThreads<T, WT>::N, bytes, p.ntiles), UpThreads<T, WT>::N, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

template <int T, bool WT>
static cudaError_t launch_down_unit_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = WT ? FinWLayout<T>::bytes : FinLayout<T>::bytes;
  auto k = WT ? k_fin_w<T> : k_fin_unit<T>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k<<<persistent_grid_u(k, NTF, bytes, p.ntiles), NTF, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

}  // namespace unit

cudaError_t launch_up_unit(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s) {
  switch (p.T) {
    case 32: return weighted ? unit::launch_up_unit_t<32, true>(dt, p, s) : unit::launch_up_unit_t<32, false>(dt, p, s);
    case 64: return weighted ? unit::launch_up_unit_t<64, true>(dt, p, s) : unit::launch_up_unit_t<64, false>(dt, p, s);
    case 128:
      return weighted ? unit::launch_up_unit_t<128, true>(dt, p, s) : unit::launch_up_unit_t<128, false>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_down_unit(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s) {
  switch (p.T) {
    case 32:
      return weighted ? unit::launch_down_unit_t<32, true>(dt, p, s) : unit::launch_down_unit_t<32, false>(dt, p, s);
    case 64:
      return weighted ? unit::launch_down_unit_t<64, true>(dt, p, s) : unit::launch_down_unit_t<64, false>(dt, p, s);
    case 128:
      return weighted ? unit::launch_down_unit_t<128, true>(dt, p, s) : unit::launch_down_unit_t<128, false>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace d8
