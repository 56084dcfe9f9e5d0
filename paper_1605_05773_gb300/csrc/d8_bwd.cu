// d8_bwd.cu -- adjoint of the weighted up-slope area.
//
// With L a loss of A and dA = dL/dA, Eq. 1 transposed gives
//   dw(q) = dL/dw(q) = dA(q) + dw(down-slope neighbour of q)   (0 past a path end),
// i.e. the sum of dA along q's flow path.  Same partition scheme as forward:
//  k_bwd_up    per tile: path sums to the tile exit for every cell by pointer
//              jumping in shared memory; the perimeter summary records, per
//              perimeter cell, its exit slot and its in-tile path sum.
//  k_bpj_*     combine: for each exit x with successor y in the next tile,
//              H(x) = (path sum of y inside its tile) + H(exit of y); a path
//              sum over the exit forest, found by pointer jumping (gathers
//              only, so deterministic).
//              It also writes every cell's in-tile path sum to dw and the
//              slot of its tile exit to a per-cell array.
//  k_bwd_fix   streaming: dw(q) += H(exit of q) for the cells whose path
//              leaves their tile (float-float add of the rounded path sum).
#include "d8_device.cuh"

namespace d8 {

constexpr uint16_t NX_END = 0xFFFFu;

template <int T>
struct BwdLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_gs = 0;                          // ff [2][TT]
  static constexpr size_t off_nx = off_gs + 2 * TT * sizeof(ff);  // u16 [2][TT]
  static constexpr size_t off_en = off_nx + 2 * TT * 2;         // u16 [2][TT]
  static constexpr size_t off_cl = off_en + 2 * TT * 2;         // u8 [TT]
  static constexpr size_t off_misc = off_cl + (TT + 15) / 16 * 16;
  static constexpr size_t bytes = off_misc + 16;
};

size_t bwd_smem_bytes(int T) {
  size_t b = 0;
  switch (T) {
    case 32: b = BwdLayout<32>::bytes; break;
    case 64: b = BwdLayout<64>::bytes; break;
    case 128: b = BwdLayout<128>::bytes; break;
    default: return 0;
  }
  return b <= 227 * 1024 ? b : 0;
}

// In-tile path sums by synchronous pointer jumping: after round r, gs[c] is the
// sum of dA over the first 2^r cells of c's in-tile path, nx[c] the next cell
// not yet included (or NX_END) and en[c] the last cell included.  Converges in
// ceil(log2(longest in-tile path)) rounds.  Returns the buffer holding the result.
template <int T>
__device__ int tile_path_sums(const DemDesc& d, const TileGeo& g, unsigned char* sm, uint32_t* status) {
  using L = BwdLayout<T>;
  ff* gs = reinterpret_cast<ff*>(sm + L::off_gs);
  uint16_t* nx = reinterpret_cast<uint16_t*>(sm + L::off_nx);
  uint16_t* en = reinterpret_cast<uint16_t*>(sm + L::off_en);
  uint8_t* cl = sm + L::off_cl;
  constexpr int TT = T * T;
  for (int c = threadIdx.x; c < TT; c += NT) {
    const int i = c / T, j = c - i * T;
    uint16_t n = NX_END;
    ff v{0.0f, 0.0f};
    if (i >= g.th || j >= g.tw) {
      cl[c] = CL_ABSENT;
    } else {
      const int64_t gi = g.i0 + i, gj = g.j0 + j;
      const uint8_t f = classify(d.dir[gi * d.lddir + gj], i, j, g, d, status);
      cl[c] = f;
      if (f & CL_IN) {
        const int k = f & 7;
        n = (uint16_t)(c + code_di(k) * T + code_dj(k));
      }
      v.hi = d.w[gi * d.ldw + gj];
    }
    gs[c] = v;
    nx[c] = n;
    en[c] = (uint16_t)c;
  }
  __syncthreads();
  int b = 0;
  bool any = true;
  for (int round = 0; round < 2 * 14 + 2 && any; round++) {
    bool act = false;
    const ff* gsb = gs + b * TT;
    const uint16_t* nxb = nx + b * TT;
    const uint16_t* enb = en + b * TT;
    ff* gso = gs + (b ^ 1) * TT;
    uint16_t* nxo = nx + (b ^ 1) * TT;
    uint16_t* eno = en + (b ^ 1) * TT;
    for (int c = threadIdx.x; c < TT; c += NT) {
      const uint16_t a = nxb[c];
      if (a == NX_END) {
        gso[c] = gsb[c];
        nxo[c] = NX_END;
        eno[c] = enb[c];
      } else {
        gso[c] = ff_add(gsb[c], gsb[a]);
        const uint16_t na = nxb[a];
        nxo[c] = na;
        eno[c] = enb[a];
        act |= (na != NX_END);
      }
    }
    b ^= 1;
    any = __syncthreads_or(act);
  }
  if (any && threadIdx.x == 0) set_status(status, D8_ERR_CYCLE);
  return b;
}

template <int T>
__global__ void __launch_bounds__(NT) k_bwd_up(DemTable dt, Pipe p) {
  using L = BwdLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  ff* gs = reinterpret_cast<ff*>(sm + L::off_gs);
  uint16_t* en = reinterpret_cast<uint16_t*>(sm + L::off_en);
  const uint8_t* cl = sm + L::off_cl;
  ff* pval = static_cast<ff*>(p.pval);
  constexpr int TT = T * T;
  TileQueue tq(p.queue + 2, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    const int b = tile_path_sums<T>(d, g, sm, p.status);
    for (int s = threadIdx.x; s < 4 * T; s += NT) {
      int i, j;
      uint16_t pe = PEX_TERM;
      ff v{0.0f, 0.0f};
      if (slot_cell(s, g.th, g.tw, T, i, j)) {
        const int c = i * T + j;
        const int e = en[b * TT + c];
        if (cl[e] & CL_EXIT) pe = (e == c) ? (uint16_t)(PEX_EXIT | (cl[c] & 7)) : (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T);
        v = gs[b * TT + c];
      }
      p.pex[t * (4 * T) + s] = pe;
      pval[t * (4 * T) + s] = v;
    }
    // every cell: its in-tile path sum (to dw) and its exit's slot
    for (int c = threadIdx.x; c < TT; c += NT) {
      const int i = c / T, j = c - i * T;
      if (i >= g.th || j >= g.tw) continue;
      const ff v = gs[b * TT + c];
      const int e = en[b * TT + c];
      const int64_t gi = g.i0 + i, gj = g.j0 + j;
      static_cast<float*>(d.A)[gi * d.ldA + gj] = __fadd_rn(v.hi, v.lo);
      p.xid[gi * d.W + gj] = (cl[e] & CL_EXIT) ? (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T) : NO_EXIT;
    }
    __syncthreads();
  }
}

// combine init: H0(x) = path sum of x's successor inside its tile, parent =
// the exit that successor's path reaches
template <int T>
__global__ void k_bpj_init(DemTable dt, Pipe p) {
  ff* H = static_cast<ff*>(p.S);
  const ff* pval = static_cast<const ff*>(p.pval);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += stride) {
    const uint16_t pe = p.pex[g];
    uint32_t par = ROOT;
    ff v{0.0f, 0.0f};
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
      v = pval[y];
      if (par != ROOT) p.flags[0] = 1u;
    }
    p.P[0][g] = par;
    H[g] = v;
  }
}

// one round of path doubling: H <- H + H(parent), parent <- parent(parent)
__global__ void k_bpj_round(Pipe p, int r) {
  if (*(volatile uint32_t*)&p.flags[r] == 0u) return;
  const ff* Hc = static_cast<const ff*>((r & 1) ? p.S2 : p.S);
  ff* Hn = static_cast<ff*>((r & 1) ? p.S : p.S2);
  const uint32_t* Pc = pick(p.P[0], p.P[1], r & 1);
  uint32_t* Pn = pick(p.P[0], p.P[1], (r + 1) & 1);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool active = false;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < p.nslots; g += stride) {
    const uint32_t par = Pc[g];
    ff h = Hc[g];
    uint32_t pp = ROOT;
    if (par != ROOT) {
      h = ff_add(h, Hc[par]);
      pp = Pc[par];
    }
    Hn[g] = h;
    Pn[g] = pp;
    active |= (pp != ROOT);
  }
  if (__syncthreads_or(active) && threadIdx.x == 0) p.flags[r + 1] = 1u;
  if (blockIdx.x == 0 && threadIdx.x == 0) p.flags[MAX_ROUNDS + 1] = (uint32_t)(r + 1);
}

__global__ void k_bpj_check(Pipe p, int R) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && p.flags[R] != 0u) set_status(p.status, D8_ERR_CYCLE);
}

// dw(q) = (in-tile path sum of q, already in dw) + H(exit of q); four
// consecutive cells of a row per thread (8-byte exit-slot loads, 16-byte dw
// accesses) when the row layout allows, else one cell per thread
template <int T, bool VEC>
__global__ void k_bwd_fix(DemTable dt, Pipe p) {
  const DemDesc d = dt.one;
  const uint32_t last = *(volatile uint32_t*)&p.flags[MAX_ROUNDS + 1];
  const ff* H = static_cast<const ff*>((last & 1) ? p.S2 : p.S);
  constexpr int V = VEC ? 4 : 1;
  const int64_t wq = d.W / V;  // groups per row
  const int64_t n = d.H * wq;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int64_t gi = k / wq, gj = (k - gi * wq) * V;
    uint16_t e[V];
    if (VEC) {
      const uint2 e4 = *reinterpret_cast<const uint2*>(p.xid + gi * d.W + gj);
      e[0] = (uint16_t)e4.x;
      e[V > 1 ? 1 : 0] = (uint16_t)(e4.x >> 16);
      e[V > 2 ? 2 : 0] = (uint16_t)e4.y;
      e[V > 3 ? 3 : 0] = (uint16_t)(e4.y >> 16);
    } else {
      e[0] = p.xid[gi * d.W + gj];
    }
    bool any = false;
#pragma unroll
    for (int u = 0; u < V; u++) any |= e[u] != NO_EXIT;
    if (!any) continue;
    float* dst = static_cast<float*>(d.A) + gi * d.ldA + gj;
    const int64_t trow = (gi / T) * d.ntx;
    if (VEC) {
      float4 a = *reinterpret_cast<float4*>(dst);
      float* av = reinterpret_cast<float*>(&a);
#pragma unroll
      for (int u = 0; u < V; u++) {
        if (e[u] == NO_EXIT) continue;
        const ff v = ff_add(ff{av[u], 0.0f}, H[(trow + (gj + u) / T) * (4 * T) + e[u]]);
        av[u] = __fadd_rn(v.hi, v.lo);
      }
      *reinterpret_cast<float4*>(dst) = a;
    } else {
      const ff v = ff_add(ff{*dst, 0.0f}, H[(trow + gj / T) * (4 * T) + e[0]]);
      *dst = __fadd_rn(v.hi, v.lo);
    }
  }
}

// ---------------------------------------------------------------------------

template <class K>
static unsigned persistent_grid_b(K kernel, size_t smem, int64_t ntiles) {
  int dev = 0, sms = 1, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, NT, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  int64_t g = (int64_t)per_sm * sms;
  if (g > ntiles) g = ntiles;
  return (unsigned)(g < 1 ? 1 : g);
}

static unsigned grid_for_b(int64_t n) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

template <int T>
static cudaError_t launch_bwd_up_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = BwdLayout<T>::bytes;
  if (bytes > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_bwd_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_bwd_up<T><<<persistent_grid_b(k_bwd_up<T>, bytes, p.ntiles), NT, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_bwd_fix_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const DemDesc& d = dt.one;
  const bool vec = d.W % 4 == 0 && d.ldA % 4 == 0 && (reinterpret_cast<uintptr_t>(d.A) & 15u) == 0;
  const int64_t n = d.H * (vec ? d.W / 4 : d.W);
  int64_t b = (n + 255) / 256;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (b > (int64_t)sms * 32) b = (int64_t)sms * 32;
  if (b < 1) b = 1;
  if (vec)
    k_bwd_fix<T, true><<<(unsigned)b, 256, 0, s>>>(dt, p);
  else
    k_bwd_fix<T, false><<<(unsigned)b, 256, 0, s>>>(dt, p);
  return cudaGetLastError();
}

cudaError_t launch_bwd_up(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  ++*nlaunch;
  switch (p.T) {
    case 32: return launch_bwd_up_t<32>(dt, p, s);
    case 64: return launch_bwd_up_t<64>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

template <int T>
static cudaError_t launch_combine_bwd_t(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  cudaError_t e = cudaMemsetAsync(p.flags, 0, sizeof(uint32_t) * (MAX_ROUNDS + 2), s);
  if (e != cudaSuccess) return e;
  const unsigned gb = grid_for_b(p.nslots);
  k_bpj_init<T><<<gb, 256, 0, s>>>(dt, p);
  ++*nlaunch;
  for (int r = 0; r < p.rounds; r++) {
    k_bpj_round<<<gb, 256, 0, s>>>(p, r);
    ++*nlaunch;
  }
  k_bpj_check<<<1, 32, 0, s>>>(p, p.rounds);
  ++*nlaunch;
  return cudaGetLastError();
}

cudaError_t launch_combine_bwd(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  switch (p.T) {
    case 32: return launch_combine_bwd_t<32>(dt, p, s, nlaunch);
    case 64: return launch_combine_bwd_t<64>(dt, p, s, nlaunch);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_bwd_down(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  ++*nlaunch;
  switch (p.T) {
    case 32: return launch_bwd_fix_t<32>(dt, p, s);
    case 64: return launch_bwd_fix_t<64>(dt, p, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace d8
