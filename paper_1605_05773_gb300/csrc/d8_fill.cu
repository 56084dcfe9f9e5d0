// d8_fill.cu -- pit and flat removal by epsilon filling on the GPU (the
// method's precondition, "The Algorithm", first paragraph: pits raised and
// flats resolved so that every interior cell drains).
//
// The filled surface F is the unique array with F = z on the grid's edge and,
// for every interior cell c with m = the lowest of its 8 neighbouring F,
//     F(c) = z(c) if z(c) > m,   else   F(c) = up(m) = max(fl32(m + eps), next fp32 above m).
// The update G(F)(c) = (z(c) > m ? z(c) : up(m)) is monotone in F and every
// fixed point is the same array, so iterating it from any start above F
// converges to F exactly, whatever the order in which cells are updated:
// starting from +inf inside, every value only ever decreases, and reading a
// neighbour's older (higher) value can only delay, never spoil, the result.
//
// GPU layout: 64 x 64 tiles.  A round visits the tiles marked active: a
// thread block loads the tile's z and the current F of the tile and its
// one-cell halo into shared memory and relaxes the tile to a local fixed
// point, first in waves (a wave updates the cells marked dirty; a cell whose
// value drops marks its neighbours dirty for the next wave), then, if a few
// waves do not settle it, in directional sweeps along rows and columns; then
// it writes the tile back.  A tile whose border values dropped marks its eight neighbouring
// tiles active for the next round.  A round in which no tile marks any
// other ends the fill: every tile is then at a fixed point of its final halo,
// so F is the global fixed point.
#include <cmath>
#include <cstdio>

#include "d8_device.cuh"

namespace d8 {
namespace fill {

constexpr int T = 64;
constexpr int NTF = 256;
constexpr int HW = T + 2;               // halo row width
constexpr int SWEEP_AFTER = 2;          // waves before the tile switches to directional sweeps
constexpr int MAX_SWEEPS = 4 * T;       // sweep passes (four directions each) before giving up

struct Layout {
  static constexpr size_t off_f = 0;                                   // float (T+2)^2: F with halo
  static constexpr size_t off_z = (size_t)HW * HW * 4;                 // float T^2
  static constexpr size_t off_m0 = off_z + (size_t)T * T * 4;          // dirty masks, 2 x T^2 bits
  static constexpr size_t off_m1 = off_m0 + (size_t)T * T / 8;
  static constexpr size_t off_misc = off_m1 + (size_t)T * T / 8;
  static constexpr size_t bytes = off_misc + 64;
};

__device__ __forceinline__ float up(float m, float eps) { return fmaxf(__fadd_rn(m, eps), nextafterf(m, INFINITY)); }

// F = z on the grid's edge, +inf inside; non-finite z reported
__global__ void k_fill_init(const float* z, int64_t H, int64_t W, int64_t ldz, float* F, int64_t ldF,
                            uint32_t* status) {
  const int64_t n = H * W, stride = (int64_t)gridDim.x * blockDim.x;
  bool bad = false;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
    const int64_t i = c / W, j = c - i * W;
    const float zc = z[i * ldz + j];
    bad |= !isfinite(zc);
    const bool edge = i == 0 || j == 0 || i == H - 1 || j == W - 1;
    F[i * ldF + j] = edge ? zc : INFINITY;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) set_status(status, D8_ERR_NONFINITE);
}

// Relax tile cell (i, j) once: F(c) = z(c) if z(c) > m else up(m), m the lowest
// of its eight neighbours' current values; returns whether F(c) dropped.
__device__ __forceinline__ bool relax_cell(float* Fh, const float* zt, int i, int j, float eps) {
  float* fc = &Fh[(i + 1) * HW + (j + 1)];
  const float m = fminf(fminf(fminf(fc[-HW - 1], fc[-HW]), fminf(fc[-HW + 1], fc[-1])),
                        fminf(fminf(fc[1], fc[HW - 1]), fminf(fc[HW], fc[HW + 1])));
  const float zc = zt[i * T + j];
  const float v = zc > m ? zc : up(m, eps);
  if (v < *fc) {
    *fc = v;
    return true;
  }
  return false;
}

// One round over the active tiles.  act_cur / act_next: one byte per tile;
// count: tiles marked for the next round by this round.
__global__ void __launch_bounds__(NTF) k_fill_round(const float* z, int64_t H, int64_t W, int64_t ldz, float* F,
                                                    int64_t ldF, float eps, int64_t ntx, int64_t nty,
                                                    uint8_t* act_cur, uint8_t* act_next, uint8_t* settled,
                                                    uint32_t* count) {
  extern __shared__ __align__(16) unsigned char sm[];
  float* Fh = reinterpret_cast<float*>(sm + Layout::off_f);
  float* zt = reinterpret_cast<float*>(sm + Layout::off_z);
  uint32_t* mk0 = reinterpret_cast<uint32_t*>(sm + Layout::off_m0);  // the two masks, back to back
  constexpr int MW = T * T / 32;                                       // words per mask
  const int64_t ntiles = ntx * nty;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    if (act_cur[t] == 0) continue;  // uniform across the block
    __syncthreads();                // the previous tile's readers are done with shared memory
    if (threadIdx.x == 0) act_cur[t] = 0;
    const int64_t ty = t / ntx, tx = t - ty * ntx, i0 = ty * T, j0 = tx * T;
    const int th = (int)min64(T, H - i0), tw = (int)min64(T, W - j0);
    // F with halo (+inf off the grid; L2 reads: other blocks write F this round)
    for (int q = threadIdx.x; q < HW * HW; q += NTF) {
      const int hi = q / HW - 1, hj = q % HW - 1;
      const int64_t gi = i0 + hi, gj = j0 + hj;
      float v = INFINITY;
      if (gi >= 0 && gj >= 0 && gi < H && gj < W && hi <= th && hj <= tw) v = __ldcg(&F[gi * ldF + gj]);
      Fh[q] = v;
    }
    // z, and the first wave: every interior grid cell of the tile on its
    // first visit; on later visits, when the tile was left at a fixed point
    // of its halo and only the halo can have changed since, the cells next
    // to the halo (the tile's border ring)
    const bool ring_only = settled[t] != 0;
    for (int q = threadIdx.x; q < T * T; q += NTF) {
      const int i = q / T, j = q % T;
      zt[q] = (i < th && j < tw) ? z[(i0 + i) * ldz + (j0 + j)] : 0.0f;
    }
    for (int q = threadIdx.x; q < T * T / 32; q += NTF) {
      const int i = (q * 32) / T, jb = (q * 32) % T;  // 32 cells of one row
      const int64_t gi = i0 + i;
      uint32_t bits = 0u;
      if (i < th && gi > 0 && gi < H - 1) {
        const bool row_ring = i == 0 || i == th - 1;
        for (int b = 0; b < 32; b++) {
          const int64_t gj = j0 + jb + b;
          const bool ring = row_ring || jb + b == 0 || jb + b == tw - 1;
          if (jb + b < tw && gj > 0 && gj < W - 1 && (ring || !ring_only)) bits |= 1u << b;
        }
      }
      mk0[q] = bits;
      mk0[MW + q] = 0u;
    }
    __syncthreads();
    bool tile_changed = false, border_changed = false, settled_now = false;
    int wave = 0;
    for (; wave < SWEEP_AFTER; wave++) {
      uint32_t* cur = mk0 + (wave & 1) * MW;
      uint32_t* nxt = mk0 + ((wave + 1) & 1) * MW;
      bool changed = false;
      // 16 cells per thread per wave: half of one 32-bit mask word
      for (int q = threadIdx.x; q < T * T / 16; q += NTF) {
        uint32_t bits = (cur[q >> 1] >> (16 * (q & 1))) & 0xFFFFu;
        while (bits) {
          const int b = __ffs(bits) - 1;
          bits &= bits - 1;
          const int c = q * 16 + b, i = c / T, j = c % T;
          if (relax_cell(Fh, zt, i, j, eps)) {
            changed = true;
            if (i == 0 || j == 0 || i == th - 1 || j == tw - 1) border_changed = true;
#pragma unroll
            for (int k = 0; k < 8; k++) {
              const int ni = i + code_di(k), nj = j + code_dj(k);
              if (ni < 0 || nj < 0 || ni >= th || nj >= tw) continue;
              const int64_t gi = i0 + ni, gj = j0 + nj;
              if (gi <= 0 || gj <= 0 || gi >= H - 1 || gj >= W - 1) continue;  // edge cells stay at z
              const int n = ni * T + nj;
              atomicOr(&nxt[n >> 5], 1u << (n & 31));
            }
          }
        }
      }
      tile_changed |= changed;
      const bool any = __syncthreads_or(changed);
      for (int q = threadIdx.x; q < MW; q += NTF) cur[q] = 0u;
      __syncthreads();
      if (!any) {
        settled_now = true;
        break;
      }
    }
    if (!settled_now) {
      // Still changing after SWEEP_AFTER waves: a wave moves a change one cell
      // per pass, so values that must cross the tile (a depression filling
      // from its pour point) switch to directional sweeps, each carrying a
      // change along a whole row or column in one pass: thread r walks row r
      // left to right, then right to left, then thread r walks column r down
      // and up.  Any order of updates reaches the same fixed point (the
      // update is monotone and its fixed point unique), so the result does
      // not depend on the mix of waves and sweeps.
      const int r = threadIdx.x;
      const bool rin = r < th && i0 + r > 0 && i0 + r < H - 1;  // row r holds interior cells
      const bool cin = r < tw && j0 + r > 0 && j0 + r < W - 1;  // column r holds interior cells
      const int jlo = j0 == 0 ? 1 : 0, jhi = (int)min64(tw, W - 1 - j0);  // interior columns [jlo, jhi)
      const int ilo = i0 == 0 ? 1 : 0, ihi = (int)min64(th, H - 1 - i0);  // interior rows [ilo, ihi)
      // a row pass changes a border cell at its first or last column, or on
      // the tile's first or last row; a column pass likewise
      const bool redge = r == 0 || r == th - 1, cedge = r == 0 || r == tw - 1;
      for (int sw = 0; sw < MAX_SWEEPS; sw++) {
        bool changed = false;
        if (rin)
          for (int j = jlo; j < jhi; j++)
            if (relax_cell(Fh, zt, r, j, eps)) {
              changed = true;
              border_changed |= redge || j == 0 || j == tw - 1;
            }
        __syncthreads();
        if (rin)
          for (int j = jhi - 1; j >= jlo; j--)
            if (relax_cell(Fh, zt, r, j, eps)) {
              changed = true;
              border_changed |= redge || j == 0 || j == tw - 1;
            }
        __syncthreads();
        if (cin)
          for (int i = ilo; i < ihi; i++)
            if (relax_cell(Fh, zt, i, r, eps)) {
              changed = true;
              border_changed |= cedge || i == 0 || i == th - 1;
            }
        __syncthreads();
        if (cin)
          for (int i = ihi - 1; i >= ilo; i--)
            if (relax_cell(Fh, zt, i, r, eps)) {
              changed = true;
              border_changed |= cedge || i == 0 || i == th - 1;
            }
        tile_changed |= changed;
        if (!__syncthreads_or(changed)) {
          settled_now = true;
          break;
        }
      }
    }
    const bool tile_any = __syncthreads_or(tile_changed);
    const bool border_any = __syncthreads_or(border_changed);
    if (tile_any) {
      for (int q = threadIdx.x; q < T * T; q += NTF) {
        const int i = q / T, j = q % T;
        if (i < th && j < tw) F[(i0 + i) * ldF + (j0 + j)] = Fh[(i + 1) * HW + (j + 1)];
      }
    }
    if (threadIdx.x == 0) {
      uint32_t marked = 0;
      if (border_any) {
        for (int k = 0; k < 8; k++) {
          const int64_t a = ty + code_di(k), b = tx + code_dj(k);
          if (a < 0 || b < 0 || a >= nty || b >= ntx) continue;
          act_next[a * ntx + b] = 1;
          marked++;
        }
      }
      if (!settled_now) {  // not settled within the caps: visit it again, every cell
        act_next[t] = 1;
        settled[t] = 0;
        marked++;
      } else {
        settled[t] = 1;
      }
      if (marked) atomicAdd(count, marked);
    }
  }
}

}  // namespace fill

size_t fill_ws_bytes(int64_t H, int64_t W) {
  const int64_t ntiles = ((H + fill::T - 1) / fill::T) * ((W + fill::T - 1) / fill::T);
  return (size_t)3 * ntiles + 256 + sizeof(uint32_t) * 64;
}

// The fill: init, then rounds until one marks nothing.  The host reads the
// round's mark count every CHUNK rounds (synchronising the stream) and stops
// after max_rounds with D8_ERR_TIMEOUT.
cudaError_t run_fill(const float* z, int64_t H, int64_t W, int64_t ldz, float eps, float* F, int64_t ldF, void* ws,
                     uint32_t* status, cudaStream_t s, int64_t max_rounds, int64_t* rounds_out, bool* timed_out,
                     int* nlaunch) {
  using namespace fill;
  const int64_t ntx = (W + T - 1) / T, nty = (H + T - 1) / T, ntiles = ntx * nty;
  uint8_t* act[2] = {static_cast<uint8_t*>(ws), static_cast<uint8_t*>(ws) + ntiles};
  uint8_t* settled = static_cast<uint8_t*>(ws) + 2 * ntiles;
  uint32_t* counts = reinterpret_cast<uint32_t*>(static_cast<char*>(ws) + ((3 * ntiles + 255) / 256) * 256);
  constexpr int CHUNK = 16;  // rounds between host checks; counts[r % CHUNK]
  *timed_out = false;
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaFuncSetAttribute(k_fill_round, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Layout::bytes);
  if (e != cudaSuccess) return e;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fill_round, NTF, Layout::bytes) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > ntiles) grid = ntiles;
  e = cudaMemsetAsync(act[0], 1, (size_t)ntiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(act[1], 0, (size_t)ntiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(settled, 0, (size_t)ntiles, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * CHUNK, s);
  if (e != cudaSuccess) return e;
  int64_t nb = (H * W + 255) / 256;
  if (nb > (int64_t)sms * 16) nb = (int64_t)sms * 16;
  k_fill_init<<<(unsigned)(nb < 1 ? 1 : nb), 256, 0, s>>>(z, H, W, ldz, F, ldF, status);
  ++*nlaunch;
  int64_t r = 0;
  for (;;) {
    for (int k = 0; k < CHUNK; k++, r++) {
      k_fill_round<<<(unsigned)grid, NTF, Layout::bytes, s>>>(z, H, W, ldz, F, ldF, eps, ntx, nty, act[r & 1],
                                                              act[(r + 1) & 1], settled, counts + (r % CHUNK));
      ++*nlaunch;
    }
    uint32_t h[CHUNK];
    e = cudaMemcpyAsync(h, counts, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * CHUNK, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    int64_t last = -1;  // the first round of the chunk that marked nothing
    for (int k = 0; k < CHUNK; k++)
      if (h[k] == 0) {
        last = r - CHUNK + k;
        break;
      }
    if (last >= 0) {
      *rounds_out = last + 1;
      return cudaGetLastError();
    }
    if (r >= max_rounds) {
      *rounds_out = r;
      *timed_out = true;
      return cudaGetLastError();
    }
  }
}

}  // namespace d8
