// d8_fwd.cu -- the weighted forward pipeline and the flat combine of libd8.
//
//  k_up       per tile ("slave partition"), weighted: the in-tile dependency
//             count (Algorithm 1), the in-tile up-slope area with inflow from
//             other tiles treated as unknown = 0 (Algorithms 2-4), and the
//             perimeter summary: for every perimeter cell the perimeter cell
//             where its in-tile path leaves the tile (the exit-side view of
//             Cell_V / Origin) and the in-tile area.
//  k_pj_*     the flat combine (Algorithms 5-6): the exits of all tiles form
//             a forest (an exit's parent is the exit its path reaches next);
//             its subtree sums are found by pointer jumping with scatter-adds,
//             ceil(log2(depth)) rounds.  Used by the weighted pipeline and,
//             with uint32 values, by the allocation-free entry point.
//  k_down     per tile finalise, weighted (Algorithms 7-8): every perimeter
//             cell gets the resolved inflow from the exits of neighbouring
//             tiles that drain into it, then the in-tile accumulation is
//             re-run with those seeds and the final areas are written.
//
// The unit-count tile passes live in d8_unit.cu, the direction stencil in
// d8_flowdir.cu; launch_up and launch_down route the unit modes there.
//
// The in-tile accumulation is the paper's queue method in shared memory: each
// cell counts its in-tile inputs (and remembers which neighbours they are),
// the cells with none are the sources, and a thread walking down-slope from a
// source keeps going while it is the last input to arrive at the next cell
// (Algorithm 2's tail recursion).  Values are pulled from the inputs in fixed
// neighbour order, so results are deterministic.
#include <cstdio>

#include "d8_device.cuh"

namespace d8 {

// ---------------------------------------------------------------------------
// shared-memory layouts

template <int T, class V>
struct UpLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_dm = (TT * 2 + 15) / 16 * 16;  // after jp (uint16 per cell)
  static constexpr size_t off_val = off_dm + TT * 4;
  static constexpr size_t off_cl = off_val + TT * sizeof(V);
  static constexpr size_t off_misc = off_cl + (TT + 15) / 16 * 16;
  static constexpr size_t bytes = off_misc + 16;
};

template <int T, class V>
struct DownLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_dm = 0;
  static constexpr size_t off_val = TT * 4;
  static constexpr size_t off_cl = off_val + TT * sizeof(V);
  static constexpr size_t off_misc = off_cl + (TT + 15) / 16 * 16;
  static constexpr size_t bytes = off_misc + 16;
};

template <class V>
__device__ __forceinline__ V seed_of(const DemDesc& d, int64_t gi, int64_t gj);
template <>
__device__ __forceinline__ uint32_t seed_of<uint32_t>(const DemDesc&, int64_t, int64_t) {
  return 1u;
}
template <>
__device__ __forceinline__ ff seed_of<ff>(const DemDesc& d, int64_t gi, int64_t gj) {
  return ff{d.w[gi * d.ldw + gj], 0.0f};
}

__device__ __forceinline__ void store_out(const DemDesc& d, int64_t gi, int64_t gj, uint32_t v) {
  static_cast<uint32_t*>(d.A)[gi * d.ldA + gj] = v;
}
__device__ __forceinline__ void store_out(const DemDesc& d, int64_t gi, int64_t gj, ff v) {
  static_cast<float*>(d.A)[gi * d.ldA + gj] = __fadd_rn(v.hi, v.lo);
}

// ---------------------------------------------------------------------------
// in-tile building blocks

// In-tile dependency counts (Algorithm 1): dm[c] bits 0..7 = number of
// in-tile inputs, bits 8..15 = which neighbours (by direction from c) they are.
template <int T, bool WITH_JP>
__device__ __forceinline__ void count_inputs(uint32_t* dm, const uint8_t* cl, uint16_t* jp) {
  for (int c = threadIdx.x; c < T * T; c += NT) {
    const uint8_t f = cl[c];
    uint16_t jv = JP_TERM;
    if (f & CL_IN) {
      const int k = f & 7;
      const int s = c + code_di(k) * T + code_dj(k);
      atomicAdd(&dm[s], 1u | (1u << (8 + opposite(k))));
      jv = (uint16_t)s;
    } else if (f & CL_EXIT) {
      jv = (uint16_t)c;
    }
    if (WITH_JP) jp[c] = jv;
  }
}

// Bit r set for each of this thread's cells (tid + r*NT) that has no in-tile input.
template <int T>
__device__ __forceinline__ uint64_t find_sources(const uint32_t* dm, const uint8_t* cl) {
  constexpr int CPT = T * T / NT;
  uint64_t src = 0;
#pragma unroll
  for (int r = 0; r < CPT; r++) {
    const int c = threadIdx.x + r * NT;
    if (!(cl[c] & CL_ABSENT) && (dm[c] & 0xFFu) == 0u) src |= 1ull << r;
  }
  return src;
}

// Algorithm 2 in shared memory.  From each source, walk down-slope: finish the
// cell (its seed plus its inputs' values, pulled in N..NW order), then
// decrement the next cell's count; continue there only if this was its last
// input.  The fences order a cell's value store before the decrement that
// publishes it, and the last arriver's loads after its decrement.
// Returns the number of cells this thread finished.
template <int T, class V>
__device__ __forceinline__ int walk_tile(uint64_t src, uint32_t* dm, V* val, const uint8_t* cl) {
  int done = 0;
  while (src) {
    const int r = __ffsll((long long)src) - 1;
    src &= src - 1;
    int cur = threadIdx.x + r * NT;
    uint32_t mask = 0;
    for (;;) {
      V v = val[cur];
      for (uint32_t m = mask; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        v = VOps<V>::add(v, val[cur + code_di(k) * T + code_dj(k)]);
      }
      val[cur] = v;
      done++;
      const uint8_t f = cl[cur];
      if (!(f & CL_IN)) break;
      const int k = f & 7;
      const int s = cur + code_di(k) * T + code_dj(k);
      __threadfence_block();
      const uint32_t old = atomicSub(&dm[s], 1u);
      if ((old & 0xFFu) != 1u) break;
      __threadfence_block();
      cur = s;
      mask = (old >> 8) & 0xFFu;
    }
  }
  return done;
}

// Exit of cell c's in-tile path by pointer halving on jp (jp[x] = next cell,
// x itself at an exit, JP_TERM where the path ends in the tile).  Concurrent
// halving by other threads only ever moves a pointer further down the same
// path, so races are benign.  Returns the exit cell or -1 (path ends inside).
template <int T>
__device__ __forceinline__ int find_exit(volatile uint16_t* jp, int c, uint32_t* status) {
  int x = c;
  for (int it = 0; it < T * T + 4; it++) {
    const int y = jp[x];
    if (y == JP_TERM) return -1;
    if (y == x) return x;
    const int z = jp[y];
    if (z == JP_TERM) return -1;
    if (z == y) return y;
    jp[x] = (uint16_t)z;
    x = z;
  }
  set_status(status, D8_ERR_CYCLE);
  return -1;
}

// ---------------------------------------------------------------------------
// kernels

template <int T, class V>
__global__ void __launch_bounds__(NT) k_up(DemTable dt, Pipe p) {
  using L = UpLayout<T, V>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint16_t* jp = reinterpret_cast<uint16_t*>(sm);
  uint32_t* dm = reinterpret_cast<uint32_t*>(sm + L::off_dm);
  V* val = reinterpret_cast<V*>(sm + L::off_val);
  uint8_t* cl = sm + L::off_cl;
  uint32_t* misc = reinterpret_cast<uint32_t*>(sm + L::off_misc);
  V* pval = static_cast<V*>(p.pval);

  TileQueue tq(p.queue + 0, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    if (threadIdx.x == 0) misc[0] = 0;
    // codes, classes and seeds
    for (int c = threadIdx.x; c < T * T; c += NT) {
      const int i = c / T, j = c - i * T;
      dm[c] = 0;
      if (i >= g.th || j >= g.tw) {
        cl[c] = CL_ABSENT;
        continue;
      }
      const int64_t gi = g.i0 + i, gj = g.j0 + j;
      cl[c] = classify(d.dir[gi * d.lddir + gj], i, j, g, d, p.status);
      val[c] = seed_of<V>(d, gi, gj);
    }
    __syncthreads();
    count_inputs<T, true>(dm, cl, jp);
    __syncthreads();
    const uint64_t src = find_sources<T>(dm, cl);
    __syncthreads();
    const int done = walk_tile<T, V>(src, dm, val, cl);
    atomicAdd(&misc[0], (uint32_t)done);
    __syncthreads();
    if (threadIdx.x == 0 && misc[0] != (uint32_t)(g.th * g.tw)) set_status(p.status, D8_ERR_CYCLE);
    // perimeter summary
    for (int s = threadIdx.x; s < 4 * T; s += NT) {
      int i, j;
      uint16_t pe = PEX_TERM;
      V pv = VOps<V>::zero();
      if (slot_cell(s, g.th, g.tw, T, i, j)) {
        const int c = i * T + j;
        const int r = find_exit<T>(jp, c, p.status);
        if (r < 0)
          pe = PEX_TERM;
        else if (r == c)
          pe = (uint16_t)(PEX_EXIT | (cl[c] & 7));
        else
          pe = (uint16_t)slot_of(r / T, r % T, g.th, g.tw, T);
        pv = val[c];
      }
      p.pex[t * (4 * T) + s] = pe;
      pval[t * (4 * T) + s] = pv;
    }
    __syncthreads();
  }
}

// combine: initial parents and values of the exit forest
template <int T, class V>
__global__ void k_pj_init(DemTable dt, Pipe p) {
  V* S = static_cast<V*>(p.S);
  const V* pval = static_cast<const V*>(p.pval);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += stride) {
    const uint16_t pe = p.pex[g];
    uint32_t par = ROOT;
    V v = VOps<V>::zero();
    if (pe & PEX_EXIT) {
      const int64_t t = g / (4 * T);
      const int s = (int)(g - t * (4 * T));
      const DemDesc d = dem_of(dt, t);
      const TileGeo geo = tile_geo(d, t - d.tile_base, T);
      int i, j;
      slot_cell(s, geo.th, geo.tw, T, i, j);
      const int k = pe & 7;
      const int64_t y = global_slot(d, geo.i0 + i + code_di(k), geo.j0 + j + code_dj(k), T);
      const uint16_t pey = p.pex[y];
      if (pey & PEX_EXIT)
        par = (uint32_t)y;
      else if (pey != PEX_TERM)
        par = (uint32_t)((y / (4 * T)) * (4 * T) + pey);
      v = pval[g];
      if (par != ROOT) p.flags[0] = 1u;
    }
    p.P[0][g] = par;
    S[g] = v;
  }
}

// one round: every node adds its partial sum to its 2^r-th ancestor, then jumps
template <class V>
__global__ void k_pj_scatter(Pipe p, int r) {
  if (*(volatile uint32_t*)&p.flags[r] == 0u) return;
  const V* S = static_cast<const V*>(p.S);
  V* Dl = static_cast<V*>(p.S2);
  const uint32_t* Pc = pick(p.P[0], p.P[1], r & 1);
  uint32_t* Pn = pick(p.P[0], p.P[1], (r + 1) & 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool active = false;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += stride) {
    const uint32_t par = Pc[g];
    if (par == ROOT) {
      Pn[g] = ROOT;
      continue;
    }
    VOps<V>::atomic_add(&Dl[par], S[g]);
    const uint32_t pp = Pc[par];
    Pn[g] = pp;
    active |= (pp != ROOT);
  }
  if (__syncthreads_or(active) && threadIdx.x == 0) p.flags[r + 1] = 1u;
}

template <class V>
__global__ void k_pj_apply(Pipe p, int r) {
  if (*(volatile uint32_t*)&p.flags[r] == 0u) return;
  V* S = static_cast<V*>(p.S);
  V* Dl = static_cast<V*>(p.S2);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += stride) {
    const V dv = Dl[g];
    if (VOps<V>::nonzero(dv)) {
      S[g] = VOps<V>::add(S[g], dv);
      Dl[g] = VOps<V>::zero();
    }
  }
}

// nodes still active after the last round: the exit graph has a cycle
__global__ void k_pj_check(Pipe p, int R) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && p.flags[R] != 0u) set_status(p.status, D8_ERR_CYCLE);
}

template <int T, class V>
__global__ void __launch_bounds__(NT) k_down(DemTable dt, Pipe p) {
  using L = DownLayout<T, V>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t* dm = reinterpret_cast<uint32_t*>(sm + L::off_dm);
  V* val = reinterpret_cast<V*>(sm + L::off_val);
  uint8_t* cl = sm + L::off_cl;
  const V* xval = static_cast<const V*>(p.S);

  TileQueue tq(p.queue + 1, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    for (int c = threadIdx.x; c < T * T; c += NT) {
      const int i = c / T, j = c - i * T;
      dm[c] = 0;
      if (i >= g.th || j >= g.tw) {
        cl[c] = CL_ABSENT;
        continue;
      }
      const int64_t gi = g.i0 + i, gj = g.j0 + j;
      cl[c] = classify(d.dir[gi * d.lddir + gj], i, j, g, d, p.status);
      val[c] = seed_of<V>(d, gi, gj);
    }
    __syncthreads();
    count_inputs<T, false>(dm, cl, nullptr);
    // Algorithm 7: seed each perimeter cell with the resolved inflow from the
    // exits of neighbouring tiles that drain into it
    for (int s = threadIdx.x; s < 4 * T; s += NT) {
      int i, j;
      if (!slot_cell(s, g.th, g.tw, T, i, j)) continue;
      V in = VOps<V>::zero();
      bool any = false;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int li = i + code_di(k), lj = j + code_dj(k);
        if (li >= 0 && lj >= 0 && li < g.th && lj < g.tw) continue;
        const int64_t gi = g.i0 + li, gj = g.j0 + lj;
        if (gi < 0 || gj < 0 || gi >= d.H || gj >= d.W) continue;
        if (d.dir[gi * d.lddir + gj] != opposite(k)) continue;
        in = VOps<V>::add(in, xval[global_slot(d, gi, gj, T)]);
        any = true;
      }
      if (any) val[i * T + j] = VOps<V>::add(val[i * T + j], in);
    }
    __syncthreads();
    const uint64_t src = find_sources<T>(dm, cl);
    __syncthreads();
    walk_tile<T, V>(src, dm, val, cl);  // Algorithm 8
    __syncthreads();
    for (int c = threadIdx.x; c < T * T; c += NT) {
      const int i = c / T, j = c - i * T;
      if (i >= g.th || j >= g.tw) continue;
      store_out(d, g.i0 + i, g.j0 + j, val[c]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host launchers

static int g_num_sms = 0;
static int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 1;
  }
  return g_num_sms;
}

static unsigned grid_for(int64_t n, int per_thread_block = 256) {
  int64_t b = (n + per_thread_block - 1) / per_thread_block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Persistent grid: as many blocks as can be resident at once (never more
// than there are tiles); they drain the tile work queue.
template <class K>
static unsigned persistent_grid(K kernel, size_t smem, int64_t ntiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * num_sms();
  if (g > ntiles) g = ntiles;
  return (unsigned)(g < 1 ? 1 : g);
}

template <class K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// shared memory of the weighted tile kernels (the unit-count kernels always fit)
size_t up_smem_bytes(int T, int mode) {
  if (mode != UP_WEIGHTED) return (T == 32 || T == 64 || T == 128) ? 1 : 0;
  size_t b = 0;
  switch (T) {
    case 32: b = UpLayout<32, ff>::bytes; break;
    case 64: b = UpLayout<64, ff>::bytes; break;
    case 128: b = UpLayout<128, ff>::bytes; break;
    default: return 0;
  }
  return b <= 227 * 1024 ? b : 0;
}

size_t down_smem_bytes(int T, bool weighted) {
  if (!weighted) return (T == 32 || T == 64 || T == 128) ? 1 : 0;
  size_t b = 0;
  switch (T) {
    case 32: b = DownLayout<32, ff>::bytes; break;
    case 64: b = DownLayout<64, ff>::bytes; break;
    case 128: b = DownLayout<128, ff>::bytes; break;
    default: return 0;
  }
  return b <= 227 * 1024 ? b : 0;
}

template <int T>
static cudaError_t launch_up_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = UpLayout<T, ff>::bytes;
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = set_smem(k_up<T, ff>, bytes);
  if (e != cudaSuccess) return e;
  k_up<T, ff><<<persistent_grid(k_up<T, ff>, bytes, p.ntiles), NT, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

// UP_UNIT_Z: directions first (d8_flowdir.cu), then the unit tile pass on them
cudaError_t launch_up(const DemTable& dt, const Pipe& p, int mode, int rule, cudaStream_t s, int* nlaunch) {
  if (mode == UP_UNIT_Z) {
    const cudaError_t e = launch_flowdir(dt, p.ntiles, p.T, rule, p.status, s, nlaunch);
    if (e != cudaSuccess) return e;
  }
  ++*nlaunch;
  if (mode == UP_UNIT_Z || mode == UP_UNIT_DIR) return launch_up_unit(dt, p, s);
  if (mode != UP_WEIGHTED) return cudaErrorInvalidValue;
  switch (p.T) {
    case 32: return launch_up_t<32>(dt, p, s);
    case 64: return launch_up_t<64>(dt, p, s);
    case 128: return launch_up_t<128>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

template <int T, class V>
static cudaError_t launch_combine_fwd_t(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  cudaError_t e = cudaMemsetAsync(p.flags, 0, sizeof(uint32_t) * (MAX_ROUNDS + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.S2, 0, sizeof(V) * (size_t)p.nslots, s);
  if (e != cudaSuccess) return e;
  const unsigned gb = grid_for(p.nslots);
  k_pj_init<T, V><<<gb, 256, 0, s>>>(dt, p);
  ++*nlaunch;
  for (int r = 0; r < p.rounds; r++) {
    k_pj_scatter<V><<<gb, 256, 0, s>>>(p, r);
    k_pj_apply<V><<<gb, 256, 0, s>>>(p, r);
    *nlaunch += 2;
  }
  k_pj_check<<<1, 32, 0, s>>>(p, p.rounds);
  ++*nlaunch;
  return cudaGetLastError();
}

cudaError_t launch_combine_fwd(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s, int* nlaunch) {
  switch (p.T) {
    case 32: return weighted ? launch_combine_fwd_t<32, ff>(dt, p, s, nlaunch) : launch_combine_fwd_t<32, uint32_t>(dt, p, s, nlaunch);
    case 64: return weighted ? launch_combine_fwd_t<64, ff>(dt, p, s, nlaunch) : launch_combine_fwd_t<64, uint32_t>(dt, p, s, nlaunch);
    case 128: return weighted ? launch_combine_fwd_t<128, ff>(dt, p, s, nlaunch) : launch_combine_fwd_t<128, uint32_t>(dt, p, s, nlaunch);
  }
  return cudaErrorInvalidValue;
}

template <int T, class V>
static cudaError_t launch_down_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = DownLayout<T, V>::bytes;
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = set_smem(k_down<T, V>, bytes);
  if (e != cudaSuccess) return e;
  k_down<T, V><<<persistent_grid(k_down<T, V>, bytes, p.ntiles), NT, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

cudaError_t launch_down(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s, int* nlaunch) {
  ++*nlaunch;
  if (!weighted) return launch_down_unit(dt, p, s);
  switch (p.T) {
    case 32: return launch_down_t<32, ff>(dt, p, s);
    case 64: return launch_down_t<64, ff>(dt, p, s);
    case 128: return launch_down_t<128, ff>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace d8
