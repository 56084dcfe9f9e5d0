// d8_unit.cu -- the unit-count tile passes (the headline path).
//
//  k_up_unit    per tile: D8 directions (fused, from z) or codes (from dir),
//               the in-tile dependency count (Algorithm 1), the in-tile
//               up-slope counts with inflow from other tiles unknown = 0
//               (Algorithms 2-4) and the perimeter summary.
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
//  * the first pass writes the in-tile counts to A, so the finalising pass
//    only walks the paths down-slope of the perimeter cells that receive
//    inflow from other tiles, adding that inflow along them, instead of
//    re-running the whole tile;
//  * one warp spans the tile width, each lane owning T/32 adjacent columns:
//    it slides a 3-row register window down its columns with vector loads of
//    z straight from global memory (coalesced), left/right neighbours come
//    from warp shuffles, and the eight slopes are formed with packed fp32x2
//    arithmetic (each cardinal neighbour paired with a diagonal);
//  * each warp draws the starting cells of its walks (sources: no in-tile
//    input) from its own pool with ballots, without shared atomics;
//  * every walk records its segment (the cells it finished) and where the
//    segment ended (at a tile exit or path end, or at the junction where
//    another walk took over), so the exit of any perimeter cell's in-tile
//    path is a short chase over segment records instead of a walk over cells.
#include "d8_device.cuh"

namespace d8 {
namespace unit {

constexpr int NTU = 128;  // threads per tile block (4 warps)
constexpr int NWU = NTU / 32;
#ifndef D8_WALK_WARPS
#define D8_WALK_WARPS 4
#endif
// Warps that walk (Algorithm 2).  A walk phase lasts at least as many steps as
// the longest in-tile flow path (about 1.3 T) whatever the number of walkers;
// measured on GB300 (64 x 64 tiles) all four warps walking is fastest.
constexpr int NWALK = D8_WALK_WARPS;
constexpr unsigned FULL = 0xFFFFFFFFu;

// word: count 0..15 | inputs left 16..19 | code 20..23 | IN 24 | EXIT 25 |
// PRESENT 26
constexpr uint32_t W_IN = 1u << 24, W_EXIT = 1u << 25, W_PRES = 1u << 26;
__device__ __forceinline__ uint32_t w_cnt(uint32_t w) { return w & 0xFFFFu; }
__device__ __forceinline__ uint32_t w_left(uint32_t w) { return (w >> 16) & 0xFu; }
__device__ __forceinline__ int w_code(uint32_t w) { return (int)((w >> 20) & 0xFu); }

// Segment records (one uint16 per cell).  A finished non-source cell holds
// the source cell whose walk finished it.  A source cell holds its walk's end
// record: SEG_REC | SEG_END | cell (the walk ended at that cell: a tile exit
// or a path end, told apart by the cell's class bits) or SEG_REC | cell (the
// walk stopped before that junction cell, which another walk finished).
constexpr uint16_t SEG_REC = 0x8000u, SEG_END = 0x4000u;

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

// D8 code of an interior cell from its 3x3 window (a = row above, b = own
// row, c = row below; 0 = left, 1 = centre, 2 = right).
// Steepest: the slope towards neighbour n is (z - zn) for a cardinal and
// (z - zn) * R for a diagonal, R = fp32(1/sqrt 2).  Formed here as the exact
// negations (zn - z) and (zn - z) * R with packed fp32x2 adds/multiplies
// (cardinal and diagonal of each pair share an instruction; x * 1.0 is
// exact), and the most negative one wins -- strict comparisons in N..NW
// order, so ties keep the earlier direction and only a strictly positive
// drop counts.  Lowest: the smallest neighbour below z, same tie rule.
__device__ __forceinline__ int d8_window_code(float a0, float a1, float a2, float b0, float b1, float b2, float c0,
                                              float c1, float c2, int rule) {
  int code = 9;
  if (rule == 0) {
    const float2 nz = make_float2(-b1, -b1);
    const float2 sc = make_float2(1.0f, inv_sqrt2_f32());
    const float2 p0 = __fmul2_rn(__fadd2_rn(make_float2(a1, a2), nz), sc);  // N, NE
    const float2 p1 = __fmul2_rn(__fadd2_rn(make_float2(b2, c2), nz), sc);  // E, SE
    const float2 p2 = __fmul2_rn(__fadd2_rn(make_float2(c1, c0), nz), sc);  // S, SW
    const float2 p3 = __fmul2_rn(__fadd2_rn(make_float2(b0, a0), nz), sc);  // W, NW
    float best = 0.0f;
    if (p0.x < best) { best = p0.x; code = 0; }
    if (p0.y < best) { best = p0.y; code = 1; }
    if (p1.x < best) { best = p1.x; code = 2; }
    if (p1.y < best) { best = p1.y; code = 3; }
    if (p2.x < best) { best = p2.x; code = 4; }
    if (p2.y < best) { best = p2.y; code = 5; }
    if (p3.x < best) { best = p3.x; code = 6; }
    if (p3.y < best) { best = p3.y; code = 7; }
  } else {
    float best = b1;
    if (a1 < best) { best = a1; code = 0; }
    if (a2 < best) { best = a2; code = 1; }
    if (b2 < best) { best = b2; code = 2; }
    if (c2 < best) { best = c2; code = 3; }
    if (c1 < best) { best = c1; code = 4; }
    if (c0 < best) { best = c0; code = 5; }
    if (b0 < best) { best = b0; code = 6; }
    if (a0 < best) { best = a0; code = 7; }
  }
  return code;
}

// Bits of the neighbours of tile cell (i, j) that lie outside a th x tw tile.
__device__ __forceinline__ uint32_t row_off_mask(int i, int th) {
  return (i == 0 ? 0x83u : 0u) | (i == th - 1 ? 0x38u : 0u);  // N, NE, NW / SE, S, SW
}
__device__ __forceinline__ uint32_t col_off_mask(int j, int tw) {
  return (j == 0 ? 0xE0u : 0u) | (j == tw - 1 ? 0x0Eu : 0u);  // SW, W, NW / NE, E, SE
}

// Per-cell bookkeeping once its code is known: the cell's own word (count 1,
// code, class bits) and, when its target is inside the tile, one more input
// for the target.  A code 0..7 whose target is outside the tile is an exit
// when the target is on the grid (`grid_target_ok`), otherwise the path ends.
template <int T>
__device__ __forceinline__ void add_cell(uint32_t* word, int c, int code, uint32_t off_mask, bool grid_target_ok,
                                         uint32_t* status) {
  uint32_t cls = 0;
  if (code < 8) {
    if (!((off_mask >> code) & 1u)) {
      cls = W_IN;
      atomicAdd(&word[c + toff_tab<T>(code)], 1u << 16);
    } else if (grid_target_ok) {
      cls = W_EXIT;
    }
  } else if (code > 9) {
    set_status(status, D8_ERR_ARG);
    code = 10;
  }
  atomicAdd(&word[c], 1u | ((uint32_t)code << 20) | cls | W_PRES);
}

template <int T>
struct UpLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_word = 0;
  static constexpr size_t off_seg = TT * 4;
  static constexpr size_t off_src = off_seg + TT * 2;
  static constexpr size_t off_misc = off_src + TT * 2;
  static constexpr size_t bytes = off_misc + 64;
};

template <int T>
struct FinLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_f = 0;                     // uint32 F per cell
  static constexpr size_t off_code = TT * 4;             // uint8 code per cell
  static constexpr size_t off_rcell = off_code + TT;     // uint16 per perimeter slot
  static constexpr size_t off_rin = off_rcell + (size_t)4 * T * 2;  // uint32 per slot
  static constexpr size_t off_misc = off_rin + (size_t)4 * T * 4;
  static constexpr size_t bytes = off_misc + 64;
};

// Directions of tile g from z into word[] and the dir grid.  One warp spans
// the tile width; each lane owns CPL = T/32 adjacent columns and walks down
// ROWS = T/4 rows with a register window of three rows.
template <int T>
__device__ __forceinline__ void tile_dirs_from_z(const DemDesc& d, const TileGeo& g, int rule, uint32_t* word,
                                                 uint32_t* status) {
  constexpr int CPL = T / 32;
  constexpr int ROWS = T / NWU;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r0 = warp * ROWS;
  const int jb = lane * CPL;                      // first own column
  const int ncols = max(0, min(CPL, g.tw - jb));  // own columns present
  const int64_t gjb = g.j0 + jb;
  const bool has_l = gjb >= 1;
  const bool right_here = ncols > 0 && (jb + CPL >= g.tw);  // owns the tile's last column
  const bool has_r = g.j0 + g.tw < d.W;
  const bool vec_ok = (ncols == CPL) && ((reinterpret_cast<uintptr_t>(d.z) & 15u) == 0) && (d.ldz % 4 == 0);
  const int64_t rows_left = d.H - g.i0;
  const int i_last = (int)min64(rows_left, (int64_t)T + 1);
  const int i_first = g.i0 > 0 ? -1 : 0;
  const int i_top_edge = (g.i0 == 0) ? 0 : -10;
  const int i_bot_edge = (rows_left <= T) ? (int)rows_left - 1 : -10;
  uint32_t colm[CPL];
  bool coledge[CPL];
#pragma unroll
  for (int k = 0; k < CPL; k++) {
    colm[k] = col_off_mask(jb + k, g.tw);
    const int64_t gj = gjb + k;
    coledge[k] = (gj == 0) || (gj == d.W - 1);
  }
  const float* p0 = d.z + (g.i0 + r0 - 1) * d.ldz + gjb;
  uint8_t* dp = d.dir + (g.i0 + r0) * d.lddir + gjb;

  // Raw values of one z row for this lane: own columns, plus the column to
  // the left (lane 0) or right (lane holding the tile's last column).
  struct Raw {
    float v[CPL];
    float l, r;
  };
  constexpr int NR = ROWS + 2;  // rows r0-1 .. r0+ROWS
  constexpr int PD = 4;         // rows loaded ahead of use
  auto issue = [&](Raw& R, int q) {
    const int li = r0 - 1 + q;
    const bool rv = (li >= i_first) && (li < i_last) && ncols > 0;
    const float* p = p0 + (int64_t)q * d.ldz;
    if (vec_ok) {
      if (CPL == 4) {
        const float4 t = rv ? __ldg(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
        R.v[0] = t.x;
        R.v[CPL > 1 ? 1 : 0] = t.y;
        R.v[CPL > 2 ? 2 : 0] = t.z;
        R.v[CPL > 3 ? 3 : 0] = t.w;
      } else if (CPL == 2) {
        const float2 t = rv ? __ldg(reinterpret_cast<const float2*>(p)) : make_float2(0.f, 0.f);
        R.v[0] = t.x;
        R.v[CPL > 1 ? 1 : 0] = t.y;
      } else {
        R.v[0] = rv ? __ldg(p) : 0.0f;
      }
    } else {
#pragma unroll
      for (int k = 0; k < CPL; k++) R.v[k] = (rv && k < ncols) ? __ldg(p + k) : 0.0f;
    }
    R.l = (lane == 0 && rv && has_l) ? __ldg(p - 1) : 0.0f;
    R.r = (right_here && rv && has_r) ? __ldg(p + ncols) : 0.0f;
  };
  // window row from raw values: neighbours across lanes by shuffles
  auto finish = [&](float(&Wr)[CPL + 2], const Raw& R) {
#pragma unroll
    for (int k = 0; k < CPL; k++) Wr[1 + k] = R.v[k];
    const float ls = __shfl_up_sync(FULL, R.v[CPL - 1], 1);
    const float rs = __shfl_down_sync(FULL, R.v[0], 1);
    Wr[0] = (lane == 0) ? R.l : ls;
    Wr[CPL + 1] = rs;
    if (right_here) {
#pragma unroll
      for (int k = 0; k <= CPL; k++)
        if (k == ncols) Wr[k + 1] = R.r;
    }
  };
  auto emit_row = [&](const float(&U)[CPL + 2], const float(&M)[CPL + 2], const float(&D)[CPL + 2], int i) {
    if (i >= g.th || ncols == 0) return;
    const uint32_t rm = row_off_mask(i, g.th);
    const bool redge = (i == i_top_edge) || (i == i_bot_edge);
    uint8_t* rowp = dp + (int64_t)(i - r0) * d.lddir;
#pragma unroll
    for (int k = 0; k < CPL; k++) {
      if (k < ncols) {
        const float zc = M[1 + k];
        const bool fin = isfinite(zc);
        int code;
        if (redge || coledge[k]) {
          code = 8;
        } else if (!fin) {
          code = 9;
        } else {
          code = d8_window_code(U[k], U[k + 1], U[k + 2], M[k], M[k + 1], M[k + 2], D[k], D[k + 1], D[k + 2], rule);
        }
        if (!fin) set_status(status, D8_ERR_NONFINITE);
        rowp[k] = (uint8_t)code;
        add_cell<T>(word, i * T + jb + k, code, rm | colm[k], true, status);
      }
    }
  };

  // software pipeline, fully unrolled: rows are loaded PD steps before use and
  // the three window rows rotate by register renaming
  Raw raw[NR];
  float win[3][CPL + 2];
#pragma unroll
  for (int q = 0; q < PD && q < NR; q++) issue(raw[q], q);
#pragma unroll
  for (int q = 0; q < NR; q++) {
    if (q + PD < NR) issue(raw[q + PD], q + PD);
    finish(win[q % 3], raw[q]);
    if (q >= 2) emit_row(win[(q + 1) % 3], win[(q + 2) % 3], win[q % 3], r0 + q - 2);
  }
}

// Codes of tile g from a given direction field into word[], four consecutive
// cells per thread per step (one 32-bit load when the layout allows).
template <int T>
__device__ __forceinline__ void tile_codes_from_dir(const DemDesc& d, const TileGeo& g, uint32_t* word,
                                                    uint32_t* status) {
  constexpr int NQ = T * T / 4 / NTU;  // four-cell groups per thread
  const bool vec = (g.tw == T) && ((reinterpret_cast<uintptr_t>(d.dir) & 3u) == 0) && (d.lddir % 4 == 0);
  // issue every load of this thread before using any (hides the memory latency)
  uint32_t fours[NQ];
#pragma unroll
  for (int r = 0; r < NQ; r++) {
    const int c = (threadIdx.x + r * NTU) * 4, i = c / T, j = c - i * T;
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
    const int q = threadIdx.x + r * NTU;
    const int c = q * 4, i = c / T, j = c - i * T;
    if (i >= g.th) continue;
    const uint32_t four = fours[r];
    const uint32_t rm = row_off_mask(i, g.th);
#pragma unroll
    for (int k = 0; k < 4; k++) {
      if (j + k >= g.tw) break;
      const int code = (four >> (8 * k)) & 0xFF;
      bool ok = true;
      if (code < 8) {
        const int64_t gi = g.i0 + i + code_di(code), gj = g.j0 + j + k + code_dj(code);
        ok = gi >= 0 && gj >= 0 && gi < d.H && gj < d.W;
      }
      add_cell<T>(word, c + k, code, rm | col_off_mask(j + k, g.tw), ok, status);
    }
  }
}

// Build this warp's pool: the cells it owns (c = lane + 32*warp + NTU*r) with
// no in-tile input.  Returns the pool size (warp-uniform).
template <int T>
__device__ __forceinline__ int warp_sources(const uint32_t* word, uint16_t* srcl) {
  const int lane = threadIdx.x & 31;
  int n = 0;
#pragma unroll 4
  for (int r = 0; r < T * T / NTU; r++) {
    const int c = threadIdx.x + r * NTU;
    const uint32_t w = word[c];
    const bool s = (w & W_PRES) && w_left(w) == 0u;
    const unsigned m = __ballot_sync(FULL, s);
    if (s) srcl[n + __popc(m & ((1u << lane) - 1u))] = (uint16_t)c;
    n += __popc(m);
  }
  return n;
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
    const uint4 o = make_uint4(w_cnt(wq.x), w_cnt(wq.y), w_cnt(wq.z), w_cnt(wq.w));
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

template <int T, bool FROM_Z>
__global__ void __launch_bounds__(NTU, 7) k_up_unit(DemTable dt, Pipe p, int rule) {
  using L = UpLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* word = reinterpret_cast<uint32_t*>(sm + L::off_word);
  uint16_t* seg = reinterpret_cast<uint16_t*>(sm + L::off_seg);
  uint16_t* srcl = reinterpret_cast<uint16_t*>(sm + L::off_src) + (threadIdx.x >> 5) * (T * T / NWU);
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  uint32_t* pval = static_cast<uint32_t*>(p.pval);
  constexpr int TT = T * T;
  const int lane = threadIdx.x & 31;

  for (int64_t t = next_tile(p.queue + 0); t < p.ntiles; t = next_tile(p.queue + 0)) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    uint4* w4 = reinterpret_cast<uint4*>(word);
    for (int c = threadIdx.x; c < TT / 4; c += NTU) w4[c] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) misc[0] = 0;
    __syncthreads();
    if (FROM_Z)
      tile_dirs_from_z<T>(d, g, rule, word, p.status);
    else
      tile_codes_from_dir<T>(d, g, word, p.status);
    __syncthreads();
    // Algorithm 2: every warp lists the sources among its cells; once all lists
    // are built the walking warps draw from them
    {
      const int n = warp_sources<T>(word, srcl);
      if (lane == 0) misc[4 + (threadIdx.x >> 5)] = n;
    }
    __syncthreads();
    int done = 0;
    if ((threadIdx.x >> 5) < NWALK) {
      // One iteration = one step for every lane with a cell in hand, written
      // as straight-line predicated code so the warp never splits.
      int li = threadIdx.x >> 5, head = 0, cur = -1, h = 0;
      const uint16_t* pool = reinterpret_cast<uint16_t*>(sm + L::off_src) + li * (TT / NWU);
      int nsrc = misc[4 + li];
      uint32_t acc = 0, wv = 0;
      const unsigned lt = (1u << lane) - 1u;
      for (;;) {
        if (NWALK < NWU) {
          while (head >= nsrc && li + NWALK < NWU) {  // next list of this walker
            li += NWALK;
            pool = reinterpret_cast<uint16_t*>(sm + L::off_src) + li * (TT / NWU);
            nsrc = misc[4 + li];
            head = 0;
          }
        }
        const unsigned need = __ballot_sync(FULL, cur < 0);
        if (head < nsrc) {
          const int idx = head + __popc(need & lt);
          if (cur < 0 && idx < nsrc) {
            cur = pool[idx];
            h = cur;
            wv = word[cur];
            acc = w_cnt(wv);
            if (!FROM_Z) done++;
          }
          head += __popc(need);
        } else if (need == FULL) {
          break;
        }
        if (cur >= 0) {
          if (wv & W_IN) {
            const int s = cur + toff_tab<T>(w_code(wv));
            const uint32_t old = atomicAdd(&word[s], acc + 0xFFFF0000u);
            if (w_left(old) == 1u) {  // last input to arrive: continue there
              seg[s] = (uint16_t)h;
              acc += w_cnt(old);
              wv = old;
              cur = s;
              if (!FROM_Z) done++;
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
    // directions derived from elevations descend strictly, so only a given
    // direction field can hold a cycle (cells never finished)
    if (!FROM_Z) atomicAdd(&misc[0], done);
    __syncthreads();
    const bool cyc = !FROM_Z && misc[0] != g.th * g.tw;
    if (threadIdx.x == 0 && cyc) set_status(p.status, D8_ERR_CYCLE);
    // in-tile counts (inflow from other tiles = 0) go to A now; the finalising
    // pass adds the inflow only where some reaches
    store_counts<T>(d, g, word);
    // perimeter summary: the exit of each perimeter cell's in-tile path, by a
    // chase over segment records (resolved records are written back)
    for (int s = threadIdx.x; s < 4 * T; s += NTU) {
      int i, j;
      uint16_t pe = PEX_TERM;
      uint32_t pv = 0;
      if (slot_cell(s, g.th, g.tw, T, i, j)) {
        const int c = i * T + j;
        const uint32_t w = word[c];
        pv = w_cnt(w);
        if (w & W_EXIT) {
          pe = (uint16_t)(PEX_EXIT | w_code(w));
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
      pval[t * (4 * T) + s] = pv;
    }
  }
}

// Algorithms 7-8 restricted to where they change anything.  A already holds
// the in-tile counts; the final count is A(c) + F(c), where F(c) is the
// inflow from other tiles routed through c.  Inflow enters a tile only at its
// receivers (perimeter cells with an up-slope neighbour in another tile) and
// follows the unique down-slope path from there, so F(c) is the sum of the
// receivers' inflows over the receivers whose in-tile path passes through c.
// Each receiver therefore walks its path once adding its inflow to every cell
// on it: additions commute, so the walks need no ordering between them and
// no reply from the shared atomics, and only the cells down-slope of a
// receiver (about a sixth of a 64 x 64 tile on fractal terrain) are touched.
// The work is the summed length of the receivers' in-tile paths (at most
// 4T * T^2 for adversarial fields, about the sub-forest size on terrain).
template <int T>
__global__ void __launch_bounds__(NTU) k_fin_unit(DemTable dt, Pipe p) {
  using L = FinLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* F = reinterpret_cast<uint32_t*>(sm + L::off_f);
  uint8_t* code = sm + L::off_code;
  uint16_t* rcell = reinterpret_cast<uint16_t*>(sm + L::off_rcell);
  uint32_t* rin = reinterpret_cast<uint32_t*>(sm + L::off_rin);
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  const uint32_t* xval = static_cast<const uint32_t*>(p.S);
  constexpr int TT = T * T;

  // F[] starts at zero; every tile leaves it at zero again (the output pass
  // clears the words the walks touched)
  for (int c = threadIdx.x; c < TT / 4; c += NTU) reinterpret_cast<uint4*>(F)[c] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) misc[0] = 0;

  for (int64_t t = next_tile(p.queue + 1); t < p.ntiles; t = next_tile(p.queue + 1)) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    // the tile's codes (cells outside a ragged tile are never reached)
    {
      const bool vec = (g.tw == T) && ((reinterpret_cast<uintptr_t>(d.dir) & 3u) == 0) && (d.lddir % 4 == 0);
      for (int q = threadIdx.x; q < TT / 4; q += NTU) {
        const int c = q * 4, i = c / T, j = c - i * T;
        if (i >= g.th) continue;
        const uint8_t* src = d.dir + (g.i0 + i) * d.lddir + (g.j0 + j);
        uint32_t four = 0x08080808u;
        if (vec) {
          four = __ldg(reinterpret_cast<const unsigned int*>(src));
        } else {
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (j + k < g.tw) four = (four & ~(0xFFu << (8 * k))) | ((uint32_t)src[k] << (8 * k));
        }
        reinterpret_cast<uint32_t*>(code)[q] = four;
      }
    }
    // Algorithm 7: the receivers and their resolved inflow, listed
    for (int s = threadIdx.x; s < 4 * T; s += NTU) {
      int i, j;
      if (!slot_cell(s, g.th, g.tw, T, i, j)) continue;
      uint32_t in = 0;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int li = i + code_di(k), lj = j + code_dj(k);
        if (li >= 0 && lj >= 0 && li < g.th && lj < g.tw) continue;
        const int64_t gi = g.i0 + li, gj = g.j0 + lj;
        if (gi < 0 || gj < 0 || gi >= d.H || gj >= d.W) continue;
        if (d.dir[gi * d.lddir + gj] != opposite(k)) continue;
        in += xval[global_slot(d, gi, gj, T)];
      }
      if (in) {
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
    for (int r = threadIdx.x; r < nrec; r += NTU) {
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
    if (threadIdx.x == 0) misc[0] = 0;
    // A += F where F is nonzero; touched words go back to zero
    for (int q = threadIdx.x; q < TT / 4; q += NTU) {
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

template <class K>
static unsigned persistent_grid_u(K kernel, size_t smem, int64_t ntiles) {
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NTU, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * sms;
  if (g > ntiles) g = ntiles;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int T, bool FROM_Z>
static cudaError_t launch_up_unit_t(const DemTable& dt, const Pipe& p, int rule, cudaStream_t s) {
  const size_t bytes = UpLayout<T>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_up_unit<T, FROM_Z>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_up_unit<T, FROM_Z><<<persistent_grid_u(k_up_unit<T, FROM_Z>, bytes, p.ntiles), NTU, bytes, s>>>(dt, p, rule);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_down_unit_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = FinLayout<T>::bytes;
  cudaError_t e = cudaFuncSetAttribute(k_fin_unit<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_fin_unit<T><<<persistent_grid_u(k_fin_unit<T>, bytes, p.ntiles), NTU, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

}  // namespace unit

cudaError_t launch_up_unit(const DemTable& dt, const Pipe& p, bool from_z, int rule, cudaStream_t s) {
  switch (p.T) {
    case 32: return from_z ? unit::launch_up_unit_t<32, true>(dt, p, rule, s) : unit::launch_up_unit_t<32, false>(dt, p, rule, s);
    case 64: return from_z ? unit::launch_up_unit_t<64, true>(dt, p, rule, s) : unit::launch_up_unit_t<64, false>(dt, p, rule, s);
    case 128: return from_z ? unit::launch_up_unit_t<128, true>(dt, p, rule, s) : unit::launch_up_unit_t<128, false>(dt, p, rule, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_down_unit(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  switch (p.T) {
    case 32: return unit::launch_down_unit_t<32>(dt, p, s);
    case 64: return unit::launch_down_unit_t<64>(dt, p, s);
    case 128: return unit::launch_down_unit_t<128>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace d8
