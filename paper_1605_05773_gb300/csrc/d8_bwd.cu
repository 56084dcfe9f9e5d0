// d8_bwd.cu -- adjoint of the weighted up-slope area.
//
// With L a loss of A and dA = dL/dA, Eq. 1 transposed gives
//   dw(q) = dL/dw(q) = dA(q) + dw(down-slope neighbour of q)   (0 past a path end),
// i.e. the sum of dA along q's flow path.  Same partition scheme as forward:
//  k_bwd_up    per tile: path sums to the tile exit for every cell by pointer
//              jumping; the perimeter summary records, per perimeter cell,
//              its exit slot and its in-tile path sum.  It also writes every
//              cell's in-tile path sum to dw and the slot of its tile exit to
//              a per-cell array.
//  k_bpj_*     combine: for each exit x with successor y in the next tile,
//              H(x) = (path sum of y inside its tile) + H(exit of y); a path
//              sum over the exit forest, found by pointer jumping (gathers
//              only, so deterministic) over a list of the exits whose sums
//              are still open.
//  k_bwd_fix   streaming: dw(q) += H(exit of q) for the cells whose path
//              leaves their tile (float-float add of the rounded path sum).
//
// Both pointer-jumping stages are synchronous (Jacobi) rounds, so every sum is
// formed in the same order whatever the schedule: the result does not depend
// on the launch configuration.  Work per round is proportional to the cells
// or exits whose sums are still open, not to the tile or slot count.
#include "d8_device.cuh"

namespace d8 {

// nx entry of a cell whose in-tile path sum is complete; the low bits hold the
// last cell of its in-tile path (a tile exit or a path end)
constexpr uint16_t NX_DONE = 0x8000u;

// 64 x 64 tiles take 512 threads (8 cells each), 32 x 32 tiles 256 (4 each)
template <int T>
struct BwdCfg {
  static constexpr int NTB = T >= 64 ? 512 : 256;
  static constexpr int CPT = T * T / NTB;
  static constexpr int MAXR = T >= 64 ? 13 : 11;  // > log2 of the longest in-tile path (T*T cells)
};

template <int T>
struct BwdLayout {
  static constexpr size_t TT = (size_t)T * T;
  static constexpr size_t off_gs = 0;                      // ff [2][TT]: path sum over the cells included so far
  static constexpr size_t off_nx = 2 * TT * sizeof(ff);    // u16 [2][TT]: next cell not yet included, or NX_DONE | last
  static constexpr size_t off_cl = off_nx + 2 * TT * 2;    // u8 [TT]: class of the cell
  static constexpr size_t bytes = off_cl + TT;
};

// In-tile path sums by synchronous pointer jumping.  Thread t owns the cells
// t + NTB k and keeps their state (sum so far, next cell) in registers; two
// shared buffers hold everyone's state for the gathers.  Round r reads buffer
// r & 1 and, for each owned cell c still open, sets sum(c) += sum(a),
// next(c) = next(a) with a = next(c), written to the other buffer; after
// round r an open cell's sum covers the first 2^(r+1) cells of its path.  A
// cell is closed once next(c) carries NX_DONE (its sum then reaches its tile
// exit or path end); it copies its final state into the other buffer once,
// in the round after it closed, and is never touched again, so a round costs
// only the cells still open.  Cells that start closed are written to both
// buffers, so after the last round the buffer written last is final
// everywhere.
template <int T>
__global__ void __launch_bounds__(BwdCfg<T>::NTB, T >= 64 ? 2 : 4) k_bwd_up(DemTable dt, Pipe p) {
  constexpr int NTB = BwdCfg<T>::NTB, CPT = BwdCfg<T>::CPT, TT = T * T;
  using L = BwdLayout<T>;
  extern __shared__ __align__(16) unsigned char sm[];
  ff* gs = reinterpret_cast<ff*>(sm + L::off_gs);
  uint16_t* nx = reinterpret_cast<uint16_t*>(sm + L::off_nx);
  uint8_t* cl = sm + L::off_cl;
  ff* pval = static_cast<ff*>(p.pval);
  TileQueue tq(p.queue + 2, p.ntiles);
  for (int64_t t = tq.first(); t < p.ntiles; t = tq.next()) {
    const DemDesc d = dem_of(dt, t);
    const TileGeo g = tile_geo(d, t - d.tile_base, T);
    // this thread's cells are (i0 + k * NTB / T, j) for k = 0 .. CPT-1: row
    // pointers step by NTB / T rows; all loads issued before any is used
    const int i0 = threadIdx.x / T, j = threadIdx.x % T;
    constexpr int RS = NTB / T;  // rows between a thread's cells
    const bool colin = j < g.tw;
    const uint8_t* dp = d.dir + (g.i0 + i0) * d.lddir + (g.j0 + j);
    const float* wp = d.w + (g.i0 + i0) * d.ldw + (g.j0 + j);
    uint8_t code[CPT];
    float w[CPT];
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      code[k] = 0;
      w[k] = 0.0f;
      if (colin && i0 + k * RS < g.th) {
        code[k] = dp[(int64_t)k * RS * d.lddir];
        w[k] = wp[(int64_t)k * RS * d.ldw];
      }
    }
    ff v[CPT];
    uint32_t n[CPT];
    uint32_t open = 0;
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      const int c = threadIdx.x + k * NTB, i = i0 + k * RS;
      uint8_t f = CL_ABSENT;
      n[k] = NX_DONE | (uint32_t)c;
      if (colin && i < g.th) {
        // class of the code: in-tile target (local test), else exit or path
        // end (grid test, perimeter cells only)
        const int kk = code[k];
        if (kk >= 8) {
          f = CL_TERM;
          if (kk > 9) set_status(p.status, D8_ERR_ARG);
        } else {
          const int li = i + code_di(kk), lj = j + code_dj(kk);
          if ((unsigned)li < (unsigned)g.th && (unsigned)lj < (unsigned)g.tw) {
            f = (uint8_t)(CL_IN | kk);
            n[k] = (uint32_t)(li * T + lj);
            open |= 1u << k;
          } else {
            const int64_t gi = g.i0 + li, gj = g.j0 + lj;
            f = (gi < 0 || gj < 0 || gi >= d.H || gj >= d.W) ? CL_TERM : (uint8_t)(CL_EXIT | kk);
          }
        }
      }
      v[k] = ff{w[k], 0.0f};
      cl[c] = f;
      gs[c] = v[k];
      nx[c] = (uint16_t)n[k];
      if (!((open >> k) & 1u)) {
        gs[TT + c] = v[k];
        nx[TT + c] = (uint16_t)n[k];
      }
    }
    bool any = __syncthreads_or(open != 0);
    int b = 0;
    uint32_t closed = 0;  // cells that closed in the previous round
    for (int round = 0; any && round < BwdCfg<T>::MAXR; round++) {
      const ff* gsb = gs + b * TT;
      const uint16_t* nxb = nx + b * TT;
      ff* gso = gs + (b ^ 1) * TT;
      uint16_t* nxo = nx + (b ^ 1) * TT;
      uint32_t now = 0;
#pragma unroll
      for (int k = 0; k < CPT; k++) {
        const int c = threadIdx.x + k * NTB;
        if ((open >> k) & 1u) {
          const uint32_t na = nxb[n[k]];
          v[k] = ff_add(v[k], gsb[n[k]]);
          n[k] = na;
          gso[c] = v[k];
          nxo[c] = (uint16_t)na;
          if (na & NX_DONE) now |= 1u << k;
        } else if ((closed >> k) & 1u) {
          gso[c] = v[k];
          nxo[c] = (uint16_t)n[k];
        }
      }
      open &= ~now;
      closed = now;
      b ^= 1;
      any = __syncthreads_or(open != 0);
    }
    const ff* gsf = gs + b * TT;  // final everywhere
    const uint16_t* nxf = nx + b * TT;
    if (any && threadIdx.x == 0) set_status(p.status, D8_ERR_CYCLE);
    // perimeter summary from the final shared state
    for (int s = threadIdx.x; s < 4 * T; s += NTB) {
      int i, j;
      uint16_t pe = PEX_TERM;
      ff pv{0.0f, 0.0f};
      if (slot_cell(s, g.th, g.tw, T, i, j)) {
        const int c = i * T + j;
        const int e = nxf[c] & (TT - 1);
        if (cl[e] & CL_EXIT) pe = (e == c) ? (uint16_t)(PEX_EXIT | (cl[c] & 7)) : (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T);
        pv = gsf[c];
      }
      p.pex[t * (4 * T) + s] = pe;
      pval[t * (4 * T) + s] = pv;
    }
    // every owned cell: its in-tile path sum (to dw) and its exit's slot
    float* ap = static_cast<float*>(d.A) + (g.i0 + i0) * d.ldA + (g.j0 + j);
    uint16_t* xp = p.xid + (g.i0 + i0) * d.W + (g.j0 + j);
#pragma unroll
    for (int k = 0; k < CPT; k++) {
      if (!colin || i0 + k * RS >= g.th) continue;
      const int e = n[k] & (TT - 1);
      ap[(int64_t)k * RS * d.ldA] = __fadd_rn(v[k].hi, v[k].lo);
      xp[(int64_t)k * RS * d.W] = (cl[e] & CL_EXIT) ? (uint16_t)slot_of(e / T, e % T, g.th, g.tw, T) : NO_EXIT;
    }
    __syncthreads();
  }
}

// Append the lanes whose `take` is set to list[] at the position counter
// *cnt hands out (one atomic per warp); every lane of the warp calls this.
__device__ __forceinline__ void warp_append(bool take, uint32_t item, uint32_t* list, uint32_t* cnt) {
  const unsigned m = __ballot_sync(0xFFFFFFFFu, take);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
  uint32_t pos = 0;
  if (lane == leader) pos = atomicAdd(cnt, (uint32_t)__popc(m));
  pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
  if (take) list[pos + __popc(m & ((1u << lane) - 1u))] = item;
}

// combine init: H0(x) = path sum of x's successor inside its tile, parent =
// the exit that successor's path reaches.  Slots without a parent are final
// now and go to both value buffers; the others are listed for round 0
// (flags[r] counts the list of round r).
template <int T>
__global__ void k_bpj_init(DemTable dt, Pipe p) {
  ff* H = static_cast<ff*>(p.S);
  ff* H2 = static_cast<ff*>(p.S2);
  const ff* pval = static_cast<const ff*>(p.pval);
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < p.nslots; base += stride) {
    const int64_t g = base + lane;
    uint32_t par = ROOT;
    if (g < p.nslots) {
      const uint16_t pe = p.pex[g];
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
      }
      p.P[0][g] = par;
      H[g] = v;
      if (par == ROOT) {
        p.P[1][g] = ROOT;
        H2[g] = v;
      }
    }
    warp_append(par != ROOT, (uint32_t)g, p.list[0], &p.flags[0]);
  }
}

// One round of path doubling over the listed exits: H <- H + H(parent),
// parent <- parent(parent), written to the other buffers.  An exit whose
// parent became ROOT is listed once more, for a round that only copies its
// final H into the other buffer, so that both buffers end up final for every
// slot (a later round may gather it from either).  Each thread takes BPJ_U
// list items per pass and issues all their loads before using any (the
// gathers are dependent pairs of random loads).  The pass loop runs the same
// number of times in every lane of a warp (the stride is a multiple of 32),
// as warp_append requires.
constexpr int BPJ_U = 4;
__global__ void __launch_bounds__(256) k_bpj_round(Pipe p, int r) {
  const uint32_t n = *(volatile uint32_t*)&p.flags[r];
  if (n == 0u) return;
  const ff* Hc = static_cast<const ff*>((r & 1) ? p.S2 : p.S);
  ff* Hn = static_cast<ff*>((r & 1) ? p.S : p.S2);
  const uint32_t* Pc = pick(p.P[0], p.P[1], r & 1);
  uint32_t* Pn = pick(p.P[0], p.P[1], (r + 1) & 1);
  const uint32_t* lc = p.list[r & 1];
  uint32_t* ln = p.list[(r + 1) & 1];
  const int lane = threadIdx.x & 31;
  const int64_t nt = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; base < (int64_t)n; base += BPJ_U * nt) {
    uint32_t g[BPJ_U], par[BPJ_U], pp[BPJ_U];
    ff h[BPJ_U], hp[BPJ_U];
    bool ok[BPJ_U];
#pragma unroll
    for (int u = 0; u < BPJ_U; u++) {
      const int64_t i = base + lane + u * nt;
      ok[u] = i < (int64_t)n;
      g[u] = ok[u] ? lc[i] : 0u;
    }
#pragma unroll
    for (int u = 0; u < BPJ_U; u++) {
      par[u] = ROOT;
      if (ok[u]) {
        par[u] = Pc[g[u]];
        h[u] = Hc[g[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < BPJ_U; u++) {
      pp[u] = ROOT;
      if (ok[u] && par[u] != ROOT) {
        hp[u] = Hc[par[u]];
        pp[u] = Pc[par[u]];
      }
    }
#pragma unroll
    for (int u = 0; u < BPJ_U; u++) {
      bool keep = false;
      if (ok[u]) {
        if (par[u] != ROOT) {
          h[u] = ff_add(h[u], hp[u]);
          keep = true;
        }
        Hn[g[u]] = h[u];
        Pn[g[u]] = pp[u];
      }
      warp_append(keep, g[u], ln, &p.flags[r + 1]);
    }
  }
}

// after R rounds the list must be empty; an exit still open lies on a cycle
__global__ void k_bpj_check(Pipe p, int R) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && p.flags[R] != 0u) set_status(p.status, D8_ERR_CYCLE);
}

// dw(q) = (in-tile path sum of q, already in dw) + H(exit of q); four
// consecutive cells of a row per thread (8-byte exit-slot loads, 16-byte dw
// accesses) when the row layout allows, else one cell per thread
template <int T, int V>
__global__ void k_bwd_fix(DemTable dt, Pipe p) {
  const DemDesc d = dt.one;
  const ff* H = static_cast<const ff*>(p.S);  // final in both buffers
  const int64_t wq = d.W / V;  // groups per row
  const int64_t n = d.H * wq;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) {
    const int64_t gi = k / wq, gj = (k - gi * wq) * V;
    uint16_t e[V];
    const uint16_t* xp = p.xid + gi * d.W + gj;
    if constexpr (V == 8) {
      const uint4 x = *reinterpret_cast<const uint4*>(xp);
      const uint32_t xw[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int u = 0; u < V; u++) e[u] = (uint16_t)(xw[(u / 2) & 3] >> (16 * (u & 1)));
    } else if constexpr (V == 4) {
      const uint2 x = *reinterpret_cast<const uint2*>(xp);
      const uint32_t xw[2] = {x.x, x.y};
#pragma unroll
      for (int u = 0; u < V; u++) e[u] = (uint16_t)(xw[(u / 2) & 1] >> (16 * (u & 1)));
    } else {
      e[0] = xp[0];
    }
    bool any = false;
#pragma unroll
    for (int u = 0; u < V; u++) any |= e[u] != NO_EXIT;
    if (!any) continue;
    float* dst = static_cast<float*>(d.A) + gi * d.ldA + gj;
    const int64_t trow = (gi / T) * d.ntx;
    if constexpr (V >= 4) {
      float4 a[V / 4];
#pragma unroll
      for (int h = 0; h < V / 4; h++) a[h] = reinterpret_cast<const float4*>(dst)[h];
      float* av = reinterpret_cast<float*>(a);
#pragma unroll
      for (int u = 0; u < V; u++) {
        if (e[u] == NO_EXIT) continue;
        const ff v = ff_add(ff{av[u], 0.0f}, H[(trow + (gj + u) / T) * (4 * T) + e[u]]);
        av[u] = __fadd_rn(v.hi, v.lo);
      }
#pragma unroll
      for (int h = 0; h < V / 4; h++) reinterpret_cast<float4*>(dst)[h] = a[h];
    } else {
      const ff v = ff_add(ff{*dst, 0.0f}, H[(trow + gj / T) * (4 * T) + e[0]]);
      *dst = __fadd_rn(v.hi, v.lo);
    }
  }
}

// ---------------------------------------------------------------------------

template <class K>
static unsigned persistent_grid_b(K kernel, int threads, size_t smem, int64_t ntiles) {
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

static unsigned grid_for_b(int64_t n, int per_sm) {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (n + 255) / 256;
  if (b > (int64_t)sms * per_sm) b = (int64_t)sms * per_sm;
  return (unsigned)(b < 1 ? 1 : b);
}

template <int T>
static cudaError_t launch_bwd_up_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  const size_t bytes = BwdLayout<T>::bytes;
  constexpr int NTB = BwdCfg<T>::NTB;
  cudaError_t e = cudaFuncSetAttribute(k_bwd_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_bwd_up<T><<<persistent_grid_b(k_bwd_up<T>, NTB, bytes, p.ntiles), NTB, bytes, s>>>(dt, p);
  return cudaGetLastError();
}

template <int T>
static cudaError_t launch_bwd_fix_t(const DemTable& dt, const Pipe& p, cudaStream_t s) {
  // eight or four cells per thread (16- or 8-byte exit-slot loads, 16-byte
  // dw accesses) when every row start stays aligned, else one
  const DemDesc& d = dt.one;
  const bool a16 = (reinterpret_cast<uintptr_t>(d.A) & 15u) == 0;
  const int v = (a16 && d.W % 8 == 0 && d.ldA % 8 == 0) ? 8 : (a16 && d.W % 4 == 0 && d.ldA % 4 == 0) ? 4 : 1;
  const unsigned b = grid_for_b(d.H * (d.W / v), 32);
  if (v == 8)
    k_bwd_fix<T, 8><<<b, 256, 0, s>>>(dt, p);
  else if (v == 4)
    k_bwd_fix<T, 4><<<b, 256, 0, s>>>(dt, p);
  else
    k_bwd_fix<T, 1><<<b, 256, 0, s>>>(dt, p);
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

// Rounds R = rounds + 2: any chain of the exit forest closes within `rounds`
// (2^rounds > slot count), and the copy round of the last exits to close
// comes one round later, so the list of round R is empty unless a cycle holds
// exits open.  Rounds after the list empties return at once.
template <int T>
static cudaError_t launch_combine_bwd_t(const DemTable& dt, const Pipe& p, cudaStream_t s, int* nlaunch) {
  const int R = p.rounds + 2;
  if (R > MAX_ROUNDS + 1) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(p.flags, 0, sizeof(uint32_t) * (MAX_ROUNDS + 2), s);
  if (e != cudaSuccess) return e;
  k_bpj_init<T><<<grid_for_b(p.nslots, 16), 256, 0, s>>>(dt, p);
  ++*nlaunch;
  const unsigned gr = grid_for_b((p.nslots + BPJ_U - 1) / BPJ_U, 4);
  for (int r = 0; r < R; r++) {
    k_bpj_round<<<gr, 256, 0, s>>>(p, r);
    ++*nlaunch;
  }
  k_bpj_check<<<1, 32, 0, s>>>(p, R);
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
