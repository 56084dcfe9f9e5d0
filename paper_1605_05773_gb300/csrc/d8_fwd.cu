// d8_fwd.cu -- pipeline routing and the flat combine of libd8.
//
//  launch_up / launch_down   route each pipeline mode to its kernels: the
//             direction stencil (d8_flowdir.cu) and the tile passes
//             (d8_unit.cu; unit counts or weighted areas).
//  k_pj_*     the flat combine (Algorithms 5-6) used by the allocation-free
//             entry point, whose scratch is one fixed array: the exits of all
//             tiles form a forest (an exit's parent is the exit its path
//             reaches next) and its subtree sums are found by pointer jumping
//             with scatter-adds, ceil(log2(depth)) rounds.  The context entry
//             points use the layered combine (d8_combine.cu).
#include <atomic>
#include <cstdio>

#include "d8_device.cuh"

namespace d8 {

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

// Inflow entering the grid across its first and last rows (a strip of a
// taller grid receiving from its neighbours): the flow entering cell (0, j)
// or (H-1, j) follows that cell's in-tile path, so it is added to the value of
// the tile exit the path reaches (Algorithm 7's receivers, seen from the
// combine), or to nothing when the path ends in the tile.  The finalising pass
// then adds it along the path itself.
template <int T>
__global__ void k_inject_inflow(DemDesc d, Pipe p) {
  uint32_t* pval = static_cast<uint32_t*>(p.pval);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 2 * d.W; q += stride) {
    const bool bottom = q >= d.W;
    const int64_t j = bottom ? q - d.W : q, gi = bottom ? d.H - 1 : 0;
    const uint32_t* in = bottom ? p.bot_in : p.top_in;
    if (!in) continue;
    const uint32_t v = in[j];
    if (!v) continue;
    const int64_t ty = gi / T, tx = j / T, t = ty * d.ntx + tx;
    const int th = (int)min64(T, d.H - ty * T), tw = (int)min64(T, d.W - tx * T);
    const int s = slot_of((int)(gi - ty * T), (int)(j - tx * T), th, tw, T);
    const uint16_t pe = p.pex[t * (4 * T) + s];
    const int e = (pe & PEX_EXIT) ? s : (pe == PEX_TERM ? -1 : (int)pe);
    if (e >= 0) atomicAdd(&pval[t * (4 * T) + e], v);
  }
}

// ---------------------------------------------------------------------------
// host launchers

// SM count of the current device, cached per device index (the calls may
// come from several host threads and several devices)
static std::atomic<int> g_num_sms[64];
static int num_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int n = g_num_sms[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 1;
    }
    g_num_sms[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

static unsigned grid_for(int64_t n, int per_thread_block = 256) {
  int64_t b = (n + per_thread_block - 1) / per_thread_block;
  const int64_t cap = (int64_t)num_sms() * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// every tile side the tile passes support fits in shared memory
size_t up_smem_bytes(int T, int) { return (T == 32 || T == 64 || T == 128) ? 1 : 0; }
size_t down_smem_bytes(int T, bool) { return (T == 32 || T == 64 || T == 128) ? 1 : 0; }

// UP_UNIT_Z: directions first (d8_flowdir.cu), then the unit tile pass on them
cudaError_t launch_up(const DemTable& dt, const Pipe& p, int mode, int rule, cudaStream_t s, int* nlaunch) {
  if (mode == UP_UNIT_Z) {
    const cudaError_t e = launch_flowdir(dt, p.ntiles, p.T, rule, p.status, s, nlaunch);
    if (e != cudaSuccess) return e;
  }
  ++*nlaunch;
  if (mode != UP_UNIT_Z && mode != UP_UNIT_DIR && mode != UP_WEIGHTED) return cudaErrorInvalidValue;
  return launch_up_unit(dt, p, mode == UP_WEIGHTED, s);
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

cudaError_t launch_combine_flat(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  switch (p.T) {
    case 32: return launch_combine_fwd_t<32, uint32_t>(dt, p, s, nlaunch);
    case 64: return launch_combine_fwd_t<64, uint32_t>(dt, p, s, nlaunch);
    case 128: return launch_combine_fwd_t<128, uint32_t>(dt, p, s, nlaunch);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_inject_inflow(const DemDesc& d, const Pipe& p, cudaStream_t s, int* nlaunch) {
  const unsigned g = grid_for(2 * d.W);
  ++*nlaunch;
  switch (p.T) {
    case 32: k_inject_inflow<32><<<g, 256, 0, s>>>(d, p); break;
    case 64: k_inject_inflow<64><<<g, 256, 0, s>>>(d, p); break;
    case 128: k_inject_inflow<128><<<g, 256, 0, s>>>(d, p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_down(const DemTable& dt, const Pipe& p, bool weighted, cudaStream_t s, int* nlaunch) {
  ++*nlaunch;
  return launch_down_unit(dt, p, weighted, s);
}

}  // namespace d8
