// d8_flowdir.cu -- the D8 direction stencil ("The Algorithm": steepest slope
// over the eight neighbours, slope = drop / distance between cell centres;
// "Introduction": lowest neighbour) as a streaming kernel.
//
// Reads 4 bytes of z and writes 1 byte of code per cell, so it is bound by
// HBM bandwidth, which needs tens of KB in flight per SM.  GB300 layout:
//  * one warp per T x T tile of the pipeline's tiling (so a batch of DEMs
//    maps onto warps through the same tile table); the warp streams down the
//    tile's rows, each row buffered in shared memory with the columns
//    j0 - 4 .. j0 + T + 3 around it (the halo columns, widened to 16-byte
//    boundaries);
//  * rows are fetched PD = 6 rows ahead with cp.async into a per-warp ring,
//    so the bytes in flight cost no registers: 16-byte zero-filling copies
//    when the rows of z are 16-byte aligned, 4-byte copies otherwise;
//  * each lane owns T/32 adjacent columns; it takes them from the ring with
//    one vector load per row, the neighbouring columns with warp shuffles,
//    and keeps a three-row window in registers;
//  * codes leave as one packed store per lane per row.
#include "d8_device.cuh"

namespace d8 {
namespace fdir {

constexpr int NTF = 128;  // threads per block: four warps, four tiles
constexpr int WPB = NTF / 32;
constexpr int PD = 6;  // rows in flight per warp
constexpr unsigned FULL = 0xFFFFFFFFu;

// D8 code of an interior cell from its 3x3 window (a = row above, b = own
// row, c = row below; 0 = left, 1 = centre, 2 = right).  Steepest: the slope
// towards neighbour n is (z - zn) for a cardinal and (z - zn) * R for a
// diagonal with R = fp32(1/sqrt 2), one rounded multiply; it is formed here as
// the exact negation (zn - z) [* R] with packed fp32x2 arithmetic (cardinals
// paired with cardinals, diagonals with diagonals for the multiply) and the
// most negative one wins.  Comparisons are strict and in N, NE, E, SE, S, SW,
// W, NW order, so the first of equal slopes wins and only a strictly positive
// drop counts.  Lowest: the smallest neighbour below z, same tie rule.
__device__ __forceinline__ int window_code(float a0, float a1, float a2, float b0, float b1, float b2, float c0,
                                           float c1, float c2, int rule) {
  int code = 9;
  if (rule == 0) {
    const float2 nz = make_float2(-b1, -b1);
    const float2 rr = make_float2(inv_sqrt2_f32(), inv_sqrt2_f32());
    const float2 ne = __fadd2_rn(make_float2(a1, b2), nz);                        // N, E
    const float2 sw = __fadd2_rn(make_float2(c1, b0), nz);                        // S, W
    const float2 d0 = __fmul2_rn(__fadd2_rn(make_float2(a2, c2), nz), rr);        // NE, SE
    const float2 d1 = __fmul2_rn(__fadd2_rn(make_float2(c0, a0), nz), rr);        // SW, NW
    float best = 0.0f;
    if (ne.x < best) { best = ne.x; code = 0; }
    if (d0.x < best) { best = d0.x; code = 1; }
    if (ne.y < best) { best = ne.y; code = 2; }
    if (d0.y < best) { best = d0.y; code = 3; }
    if (sw.x < best) { best = sw.x; code = 4; }
    if (d1.x < best) { best = d1.x; code = 5; }
    if (sw.y < best) { best = sw.y; code = 6; }
    if (d1.y < best) { best = d1.y; code = 7; }
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


// NODATA masks (the rule's NODATA bit): a cell with a non-finite elevation is
// outside the study area and gets OUTLET, and so does every cell next to one
// (the area's edge drains off it, as the grid's edge does); nothing is
// reported as an error.
template <int T, bool NODATA>
__global__ void __launch_bounds__(NTF) k_flowdir_rows(DemTable dt, int64_t ntiles, int rule, uint32_t* status) {
  constexpr int CPL = T / 32;  // columns per lane
  constexpr int RW = T + 8;    // floats per buffered row: columns j0 - 4 .. j0 + T + 3
  static_assert(PD % 3 == 0, "the window index must be static in the unrolled loop");
  __shared__ __align__(16) float ring_all[WPB * PD * RW];
  float* ring = ring_all + (threadIdx.x >> 5) * (PD * RW);
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * WPB;
  for (int64_t t = (int64_t)blockIdx.x * WPB + (threadIdx.x >> 5); t < ntiles; t += nwarps) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    const bool vec = ((reinterpret_cast<uintptr_t>(d.z) & 15u) == 0) && ((d.ldz & 3) == 0);
    const int jb = lane * CPL;  // first own column
    const int nq = g.th + 2;    // rows q = 0 .. th + 1 are tile-local rows -1 .. th
    // this lane's part of a buffered row: 16-byte chunks ch0 (and ch0 + 32
    // when T = 128) or 4-byte elements lane, lane + 32, ...; the number of
    // bytes of each that lie on the grid is the same for every row
    constexpr int NCH = RW / 4;
    const int64_t col0 = g.j0 - 4 + (vec ? 4 * lane : lane);
    auto valid_bytes = [&](int64_t col) -> int {
      if (vec) return col < 0 ? 0 : 4 * (int)min64(4, d.W - col < 0 ? 0 : d.W - col);
      return (col >= 0 && col < d.W) ? 4 : 0;
    };
    const int nb0 = valid_bytes(col0);
    const int nb1 = valid_bytes(col0 + (vec ? 128 : 32));
    // rows q in [qlo, qhi) lie on the grid (the others only neighbour edge
    // cells, whose code is OUTLET, and are never fetched); row q + PD is
    // fetched while row q is used, from a pointer advanced by ldz per row
    // (a strip of a taller grid also reads the row above its first row or
    // below its last, d.halo, whose cells are then not grid edges)
    const int qlo = (g.i0 == 0 && !(d.halo & 1)) ? 1 : 0;
    const int qhi = (int)min64((int64_t)nq, d.H - g.i0 + ((d.halo & 2) ? 2 : 1));
    // fetch() is called for q = 0, 1, 2, ... in order: a running row pointer
    const float* fsrc = d.z + (g.i0 - 1) * d.ldz + col0;  // row q = 0; only formed, not read, when i0 == 0
    int fq = 0;
    auto fetch = [&](int slot) {
      if (fq >= qlo && fq < qhi) {
        float* dst = ring + slot * RW;
        if (vec) {
          if (lane < NCH) cp_async16(dst + 4 * lane, nb0 ? fsrc : d.z, nb0);
          if (NCH > 32 && lane + 32 < NCH) cp_async16(dst + 4 * lane + 128, nb1 ? fsrc + 128 : d.z, nb1);
        } else {
          for (int c = lane, k = 0; c < RW; c += 32, k++) {
            const int nb = k == 0 ? nb0 : (k == 1 ? nb1 : valid_bytes(col0 + 32 * k));
            cp_async4(dst + c, nb ? fsrc + 32 * k : d.z, nb);
          }
        }
      }
      fsrc += d.ldz;
      fq++;
    };
    // window row from ring slot `slot`: own columns, neighbours by shuffles
    auto take = [&](float(&Wr)[CPL + 2], int slot) {
      const float* row = ring + slot * RW + 4 + jb;
      if (CPL == 4) {
        const float4 v = *reinterpret_cast<const float4*>(row);
        Wr[1] = v.x;
        Wr[CPL > 1 ? 2 : 1] = v.y;
        Wr[CPL > 2 ? 3 : 1] = v.z;
        Wr[CPL > 3 ? 4 : 1] = v.w;
      } else if (CPL == 2) {
        const float2 v = *reinterpret_cast<const float2*>(row);
        Wr[1] = v.x;
        Wr[CPL > 1 ? 2 : 1] = v.y;
      } else {
        Wr[1] = row[0];
      }
      const float ls = __shfl_up_sync(FULL, Wr[CPL], 1);
      const float rs = __shfl_down_sync(FULL, Wr[1], 1);
      Wr[0] = lane == 0 ? row[-1] : ls;
      Wr[CPL + 1] = lane == 31 ? row[CPL] : rs;
    };
    const int i_top_edge = (g.i0 == 0 && !(d.halo & 1)) ? 0 : -10;
    const int i_bot_edge = (g.i0 + g.th == d.H && !(d.halo & 2)) ? g.th - 1 : -10;
    const int ncols = max(0, min(CPL, g.tw - jb));  // own columns present
    uint8_t* drow = d.dir + g.i0 * d.lddir + g.j0 + jb;  // emit() is called for rows 0, 1, 2, ... in order
    const bool st_vec = (ncols == CPL) && ((reinterpret_cast<uintptr_t>(drow) & (CPL - 1)) == 0) &&
                        (d.lddir % CPL == 0);
    bool coledge[CPL];
#pragma unroll
    for (int k = 0; k < CPL; k++) {
      const int64_t gj = g.j0 + jb + k;
      coledge[k] = (gj == 0) || (gj == d.W - 1);
    }
    auto emit = [&](const float(&U)[CPL + 2], const float(&M)[CPL + 2], const float(&D)[CPL + 2], int i) {
      uint8_t* rowp = drow;
      drow += d.lddir;
      if (ncols == 0) return;
      const bool redge = (i == i_top_edge) || (i == i_bot_edge);
      uint32_t packed = 0;
      bool bad = false;
#pragma unroll
      for (int k = 0; k < CPL; k++) {
        const float zc = M[1 + k];
        const bool fin = isfinite(zc);
        int code;
        if (redge || coledge[k]) {
          code = 8;
        } else if (!fin) {
          code = NODATA ? 8 : 9;
        } else if (NODATA && !(isfinite(U[k]) && isfinite(U[k + 1]) && isfinite(U[k + 2]) && isfinite(M[k]) &&
                               isfinite(M[k + 2]) && isfinite(D[k]) && isfinite(D[k + 1]) && isfinite(D[k + 2]))) {
          code = 8;
        } else {
          code = window_code(U[k], U[k + 1], U[k + 2], M[k], M[k + 1], M[k + 2], D[k], D[k + 1], D[k + 2], rule);
        }
        if (!NODATA) bad |= (k < ncols) && !fin;
        packed |= (uint32_t)code << (8 * k);
      }
      if (bad) set_status(status, D8_ERR_NONFINITE);
      if (st_vec) {
        if (CPL == 4)
          *reinterpret_cast<uint32_t*>(rowp) = packed;
        else if (CPL == 2)
          *reinterpret_cast<uint16_t*>(rowp) = (uint16_t)packed;
        else
          *rowp = (uint8_t)packed;
      } else {
#pragma unroll
        for (int k = 0; k < CPL; k++)
          if (k < ncols) rowp[k] = (uint8_t)(packed >> (8 * k));
      }
    };

    // row q sits in slot q % PD; one cp.async group per row, so waiting until
    // at most PD - 1 groups are pending means row q has landed
#pragma unroll
    for (int u = 0; u < PD; u++) {
      fetch(u);
      cp_async_commit();
    }
    float win[3][CPL + 2];
    for (int qb = 0; qb < nq; qb += PD) {
#pragma unroll
      for (int u = 0; u < PD; u++) {
        const int q = qb + u;
        if (q < nq) {
          cp_async_wait<PD - 1>();
          __syncwarp();
          take(win[u % 3], u);
          __syncwarp();  // every lane has read the slot before it is refilled
          fetch(u);  // row q + PD
          cp_async_commit();
          if (q >= 2) emit(win[(u + 1) % 3], win[(u + 2) % 3], win[u % 3], q - 2);
        }
      }
    }
    cp_async_wait<0>();  // nothing may land in the ring after the tile is done
    __syncwarp();
  }
}

template <int T>
static cudaError_t launch_t(const DemTable& dt, int64_t ntiles, int rule, uint32_t* status, cudaStream_t s) {
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto k = (rule & 2) ? k_flowdir_rows<T, true> : k_flowdir_rows<T, false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTF, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t grid = (ntiles + WPB - 1) / WPB;
  const int64_t cap = (int64_t)sms * per_sm;
  if (grid > cap) grid = cap;
  k<<<(unsigned)(grid < 1 ? 1 : grid), NTF, 0, s>>>(dt, ntiles, rule & 1, status);
  return cudaGetLastError();
}

}  // namespace fdir

cudaError_t launch_flowdir(const DemTable& dt, int64_t ntiles, int T, int rule, uint32_t* status, cudaStream_t s,
                           int* nlaunch) {
  ++*nlaunch;
  switch (T) {
    case 32: return fdir::launch_t<32>(dt, ntiles, rule, status, s);
    case 64: return fdir::launch_t<64>(dt, ntiles, rule, status, s);
    case 128: return fdir::launch_t<128>(dt, ntiles, rule, status, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace d8
