// d8_combine.cu -- the combine of the unit-count pipeline (Algorithms 5-6),
// layered as the paper's conclusion suggests.
//
// Level 0 units are the tiles; each has a perimeter summary (per perimeter
// slot: the exit of the slot's in-tile path, and the in-tile count at exits).
// A level-l unit ("group") is a G x G block of level-(l-1) units.  The exits
// of the children form a forest inside the group: a child exit's parent is
// the child exit that its successor's path reaches next.  k_group_up solves
// that forest in shared memory with the same last-arriver walks as the tiles
// (Algorithm 2 on the exit forest) and writes the group's own perimeter
// summary in the same format -- so the next level runs the same kernel.
// Above the last shared-memory level, k_top_* solve the remaining exit forest
// in global memory: the master's queue method (Algorithms 5-6) with global
// atomics, a short walk because few units remain.  k_group_down then runs
// each level back down: the resolved inflow across a group's border seeds
// its child exits and the same walks give every child exit its final area;
// at level 0 that is the final area of every tile exit, which the tiles'
// finalising pass reads.
//
// Unit counts travel as uint32, weighted areas as float-float values (fp32
// arithmetic throughout, with compensated atomic adds).
#include <cstring>

#include "d8_device.cuh"

namespace d8 {

namespace cmb {

constexpr int NTG = 256;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr uint16_t N_ROOT = 0xFFFFu;  // path ends inside the group
constexpr uint16_t N_OUT = 0xFFFEu;   // parent lies outside the group (a group exit)
constexpr uint16_t N_NONE = 0xFFFDu;  // not an exit slot

template <int S, int G, class V>
struct GroupLayout {
  static constexpr int NS = G * G * 4 * S;  // child slots of a group
  static constexpr size_t off_spx = 0;                                       // u16 child exit codes
  static constexpr size_t off_val = ((size_t)NS * 2 + 15) / 16 * 16;         // value
  static constexpr size_t off_pd = off_val + (size_t)NS * sizeof(V);         // u32 parent << 16 | children left
  static constexpr size_t off_src = off_pd + (size_t)NS * 4;                 // u16 source lists
  static constexpr size_t off_misc = off_src + (size_t)NS * 2;
  static constexpr size_t bytes = off_misc + 64;
};

__device__ __forceinline__ DemDesc dem_by_index(const DemTable& t, int k) { return t.ndem == 1 ? t.one : t.table[k]; }

// Value arithmetic: uint32 counts, or float-float areas.  A float-float
// atomic add (fp32 atomics exist in shared and global memory; fp64 arithmetic
// is slow on this GPU) adds the high part with an atomic that returns the old
// value, takes that add's exact rounding error by TwoSum and adds it with the
// low part into the low word: only the rounding of the low word's own sums is
// lost.  The parts are not renormalised between adds, which float-float
// addition tolerates.
__device__ __forceinline__ uint32_t vadd(uint32_t a, uint32_t b) { return a + b; }
__device__ __forceinline__ ff vadd(ff a, ff b) { return ff_add(a, b); }
__device__ __forceinline__ void vatomic_add(uint32_t* p, uint32_t x) { atomicAdd(p, x); }
__device__ __forceinline__ void vatomic_add(ff* p, ff x) {
  const float old = atomicAdd(&p->hi, x.hi);
  const float s = __fadd_rn(old, x.hi);
  const float bv = __fsub_rn(s, old);
  const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(s, bv)), __fsub_rn(x.hi, bv));
  atomicAdd(&p->lo, __fadd_rn(err, x.lo));
}
__device__ __forceinline__ uint32_t vload_volatile(const uint32_t* p) { return *(volatile const uint32_t*)p; }
__device__ __forceinline__ ff vload_volatile(const ff* p) {
  return ff{*(volatile const float*)&p->hi, *(volatile const float*)&p->lo};
}

struct UnitGeo {
  int64_t i0, j0;
  int h, w;
};

__device__ __forceinline__ UnitGeo unit_geo(const DemDesc& d, int64_t uy, int64_t ux, int S) {
  UnitGeo u;
  u.i0 = uy * S;
  u.j0 = ux * S;
  u.h = (int)min64(S, d.H - u.i0);
  u.w = (int)min64(S, d.W - u.j0);
  return u;
}

// Load the children of group (gy, gx) and compute every child exit's parent
// inside the group and the children count of every node.
// Returns the number of child exits this thread loaded.
// pd[n]: node n's parent (bits 16..31, or N_ROOT / N_OUT / N_NONE) and its
// number of unfinished children (bits 0..15; a group has fewer than 2^16
// nodes), one 32-bit word so that both live in native 32-bit atomics.
__device__ __forceinline__ uint32_t pd_par(uint32_t w) { return w >> 16; }
__device__ __forceinline__ uint32_t pd_deg(uint32_t w) { return w & 0xFFFFu; }

template <int S, int G, class V, class CV>
__device__ int group_load(const DemDesc& cd, int64_t gy, int64_t gx, const uint16_t* cpex, const CV* cpval,
                          uint16_t* spx, V* val, uint32_t* pd) {
  constexpr int NS = G * G * 4 * S;
  constexpr int SPT = 4 * S;  // slots per child, a multiple of 8
  constexpr int NQ = NS / 8 / NTG > 0 ? NS / 8 / NTG : 1;
  static_assert(SPT % 8 == 0 && NS % (8 * NTG) == 0, "eight slots per load, whole rounds per thread");
  int exits = 0;
  // eight consecutive slots of one child per 16-byte load of codes, with
  // their values loaded unconditionally beside them: every load of this
  // thread is issued before any is used (one round trip to memory)
  uint4 pe8[NQ];
  CV v8[NQ][8];
#pragma unroll
  for (int r = 0; r < NQ; r++) {
    const int n = (threadIdx.x + r * NTG) * 8;
    const int lt = n / SPT, s = n - lt * SPT;
    const int64_t cy = gy * G + lt / G, cx = gx * G + lt % G;
    pe8[r] = make_uint4(PEX_TERM | (PEX_TERM << 16), PEX_TERM | (PEX_TERM << 16), PEX_TERM | (PEX_TERM << 16),
                        PEX_TERM | (PEX_TERM << 16));
    if (cy < cd.nty && cx < cd.ntx) {
      const int64_t g0 = (cd.tile_base + cy * cd.ntx + cx) * SPT + s;
      pe8[r] = *reinterpret_cast<const uint4*>(cpex + g0);
      const uint4* vp = reinterpret_cast<const uint4*>(cpval + g0);
      uint4 raw[8 * sizeof(CV) / 16];
#pragma unroll
      for (int k = 0; k < (int)(8 * sizeof(CV) / 16); k++) raw[k] = vp[k];
      memcpy(v8[r], raw, sizeof(raw));
    }
  }
#pragma unroll
  for (int r = 0; r < NQ; r++) {
    const int n = (threadIdx.x + r * NTG) * 8;
    const uint16_t* pe = reinterpret_cast<const uint16_t*>(&pe8[r]);
    V vo[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      const bool ex = (pe[k] & PEX_EXIT) != 0;
      exits += ex;
      vo[k] = ex ? V(v8[r][k]) : V{};
    }
    *reinterpret_cast<uint4*>(spx + n) = pe8[r];
#pragma unroll
    for (int k = 0; k < 8; k++) val[n + k] = vo[k];
    *reinterpret_cast<uint4*>(pd + n) = make_uint4(0, 0, 0, 0);
    *reinterpret_cast<uint4*>(pd + n + 4) = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  for (int n = threadIdx.x; n < NS; n += NTG) {
    const uint16_t pe = spx[n];
    uint16_t pr = N_NONE;
    if (pe & PEX_EXIT) {
      const int lt = n / (4 * S), s = n - lt * (4 * S);
      const int64_t cy = gy * G + lt / G, cx = gx * G + lt % G;
      const UnitGeo u = unit_geo(cd, cy, cx, S);
      int i, j;
      slot_cell(s, u.h, u.w, S, i, j);
      const int k = pe & 7;
      const int64_t ti = u.i0 + i + code_di(k), tj = u.j0 + j + code_dj(k);
      const int64_t ty = ti / S, tx = tj / S;
      const int64_t a = ty - gy * G, b = tx - gx * G;
      if (a >= 0 && b >= 0 && a < G && b < G) {
        const UnitGeo tu = unit_geo(cd, ty, tx, S);
        const int lt2 = (int)(a * G + b);
        const int n2 = lt2 * (4 * S) + slot_of((int)(ti - tu.i0), (int)(tj - tu.j0), tu.h, tu.w, S);
        const uint16_t pe2 = spx[n2];
        if (pe2 & PEX_EXIT)
          pr = (uint16_t)n2;
        else if (pe2 == PEX_TERM)
          pr = N_ROOT;
        else
          pr = (uint16_t)(lt2 * (4 * S) + pe2);
        if (pr < N_NONE) atomicAdd(&pd[pr], 1u);
      } else {
        pr = N_OUT;
      }
    }
    if (pr != 0) atomicAdd(&pd[n], (uint32_t)pr << 16);
  }
  __syncthreads();
  return exits;
}

// Algorithm 2 on the exit forest of a group: last-arriver walks from the
// nodes without unfinished children.  A finished node adds its value to its
// parent, then (after a block fence) decrements the parent's children count;
// the last child continues at the parent (its acquire-release count atomic
// orders it after every child's addition).  Returns the number of nodes this thread finished.
template <int S, int G, class V>
__device__ int group_walk(uint16_t* spx, V* val, uint32_t* pd, uint16_t* srcl) {
  constexpr int NS = G * G * 4 * S;
  constexpr int NW = NTG / 32;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint16_t* my = srcl + warp * (NS / NW);
  int n = 0;
  for (int r = 0; r < NS / NTG; r++) {
    const int c = threadIdx.x + r * NTG;
    const bool s = (spx[c] & PEX_EXIT) && pd_deg(pd[c]) == 0u;
    const unsigned m = __ballot_sync(FULL, s);
    if (s) my[n + __popc(m & ((1u << lane) - 1u))] = (uint16_t)c;
    n += __popc(m);
  }
  __syncthreads();
  int done = 0, head = 0, cur = -1;
  V v{};
  const unsigned lt = (1u << lane) - 1u;
  for (;;) {
    if (head < n) {
      const unsigned need = __ballot_sync(FULL, cur < 0);
      const int idx = head + __popc(need & lt);
      if (cur < 0 && idx < n) {
        cur = my[idx];
        v = val[cur];
        done++;
      }
      head += __popc(need);
    } else if (!__any_sync(FULL, cur >= 0)) {
      break;
    }
    if (cur >= 0) {
      const uint32_t p = pd_par(pd[cur]);
      if (p >= N_NONE) {
        cur = -1;
        continue;
      }
      vatomic_add(&val[p], v);
      // the addition above is released by the count's atomic; the last child
      // reads the parent's value after it (acquire)
      const uint32_t old = atomic_add_acq_rel_cta(&pd[p], 0u - 1u);
      if (pd_deg(old) == 1u) {
        cur = p;
        v = vload_volatile(&val[p]);
        done++;
      } else {
        cur = -1;
      }
    }
  }
  return done;
}

template <int S, int G, class V, class CV>
__global__ void __launch_bounds__(NTG) k_group_up(DemTable cdt, DemTable gdt, const uint16_t* cpex, const CV* cpval,
                                                    uint16_t* gpex, V* gpval, int64_t ngroups, uint32_t* queue,
                                                    uint32_t* status) {
  using L = GroupLayout<S, G, V>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint16_t* spx = reinterpret_cast<uint16_t*>(sm + L::off_spx);
  V* val = reinterpret_cast<V*>(sm + L::off_val);
  uint32_t* pd = reinterpret_cast<uint32_t*>(sm + L::off_pd);
  uint16_t* srcl = reinterpret_cast<uint16_t*>(sm + L::off_src);
  int* misc = reinterpret_cast<int*>(sm + L::off_misc);
  constexpr int NS = L::NS;
  constexpr int GS = G * S;
  TileQueue tq(queue, ngroups);
  for (int64_t gu = tq.first(); gu < ngroups; gu = tq.next()) {
    const DemDesc gd = dem_of(gdt, gu);
    const int dem = gdt.ndem == 1 ? 0 : gdt.tile_dem[gu];
    const DemDesc cd = dem_by_index(cdt, dem);
    const int64_t lg = gu - gd.tile_base;
    const int64_t gy = lg / gd.ntx, gx = lg % gd.ntx;
    if (threadIdx.x == 0) {
      misc[0] = 0;
      misc[1] = 0;
    }
    const int exits = group_load<S, G, V, CV>(cd, gy, gx, cpex, cpval, spx, val, pd);
    const int done = group_walk<S, G, V>(spx, val, pd, srcl);
    atomicAdd(&misc[0], done);
    atomicAdd(&misc[1], exits);
    __syncthreads();
    // every exit node must have been finished, else the exit graph has a cycle
    if (threadIdx.x == 0 && misc[0] != misc[1]) set_status(status, D8_ERR_CYCLE);
    // the group's own perimeter summary
    const UnitGeo gg = unit_geo(gd, gy, gx, GS);
    for (int gs = threadIdx.x; gs < 4 * GS; gs += NTG) {
      int ci, cj;
      uint16_t gpe = PEX_TERM;
      V gv{};
      if (slot_cell(gs, gg.h, gg.w, GS, ci, cj)) {
        const int a = ci / S, b = cj / S;
        const UnitGeo cu = unit_geo(cd, gy * G + a, gx * G + b, S);
        const int lt = a * G + b;
        const int n0 = lt * (4 * S) + slot_of(ci - a * S, cj - b * S, cu.h, cu.w, S);
        const uint16_t pe = spx[n0];
        int x = -1;
        if (pe & PEX_EXIT) {
          if (pd_par(pd[n0]) == N_OUT) {
            gpe = (uint16_t)(PEX_EXIT | (pe & 7));
            gv = val[n0];
          } else {
            x = n0;
          }
        } else if (pe != PEX_TERM) {
          x = lt * (4 * S) + pe;
        }
        if (x >= 0) {
          for (int it = 0; it < NS && pd_par(pd[x]) < N_NONE; it++) x = (int)pd_par(pd[x]);
          if (pd_par(pd[x]) == N_OUT) {
            const int xlt = x / (4 * S), xs = x - xlt * (4 * S);
            const UnitGeo xu = unit_geo(cd, gy * G + xlt / G, gx * G + xlt % G, S);
            int xi, xj;
            slot_cell(xs, xu.h, xu.w, S, xi, xj);
            gpe = (uint16_t)slot_of((xlt / G) * S + xi, (xlt % G) * S + xj, gg.h, gg.w, GS);
          }
        }
      }
      gpex[gu * (4 * GS) + gs] = gpe;
      gpval[gu * (4 * GS) + gs] = gv;
    }
    // (the queue's barrier protects shared memory before the next group)
  }
}

template <int S, int G, class V, class CV>
__global__ void __launch_bounds__(NTG) k_group_down(DemTable cdt, DemTable gdt, const uint16_t* cpex, const CV* cpval,
                                                      V* cfin, const V* gfin, int64_t ngroups, uint32_t* queue) {
  using L = GroupLayout<S, G, V>;
  extern __shared__ __align__(16) unsigned char sm[];
  uint16_t* spx = reinterpret_cast<uint16_t*>(sm + L::off_spx);
  V* val = reinterpret_cast<V*>(sm + L::off_val);
  uint32_t* pd = reinterpret_cast<uint32_t*>(sm + L::off_pd);
  uint16_t* srcl = reinterpret_cast<uint16_t*>(sm + L::off_src);
  constexpr int NS = L::NS;
  constexpr int GS = G * S;
  TileQueue tq(queue, ngroups);
  for (int64_t gu = tq.first(); gu < ngroups; gu = tq.next()) {
    const DemDesc gd = dem_of(gdt, gu);
    const int dem = gdt.ndem == 1 ? 0 : gdt.tile_dem[gu];
    const DemDesc cd = dem_by_index(cdt, dem);
    const int64_t lg = gu - gd.tile_base;
    const int64_t gy = lg / gd.ntx, gx = lg % gd.ntx;
    group_load<S, G, V, CV>(cd, gy, gx, cpex, cpval, spx, val, pd);
    // inflow across the group border: each border cell r receives the final
    // areas of the outside cells draining into it; the inflow then follows
    // r's path inside its child unit to that child's exit
    const UnitGeo gg = unit_geo(gd, gy, gx, GS);
    for (int gs = threadIdx.x; gs < 4 * GS; gs += NTG) {
      int ci, cj;
      if (!slot_cell(gs, gg.h, gg.w, GS, ci, cj)) continue;
      const int64_t gi = gg.i0 + ci, gj = gg.j0 + cj;
      V in{};
      bool any = false;
#pragma unroll
      for (int k = 0; k < 8; k++) {
        const int li = ci + code_di(k), lj = cj + code_dj(k);
        if (li >= 0 && lj >= 0 && li < gg.h && lj < gg.w) continue;
        const int64_t ni = gi + code_di(k), nj = gj + code_dj(k);
        if (ni < 0 || nj < 0 || ni >= gd.H || nj >= gd.W) continue;
        if (gd.dir[ni * gd.lddir + nj] != opposite(k)) continue;
        in = vadd(in, gfin[global_slot(gd, ni, nj, GS)]);
        any = true;
      }
      if (!any) continue;
      const int a = ci / S, b = cj / S;
      const UnitGeo cu = unit_geo(cd, gy * G + a, gx * G + b, S);
      const int lt = a * G + b;
      const int n0 = lt * (4 * S) + slot_of(ci - a * S, cj - b * S, cu.h, cu.w, S);
      const uint16_t pe = spx[n0];
      if (pe & PEX_EXIT)
        vatomic_add(&val[n0], in);
      else if (pe != PEX_TERM)
        vatomic_add(&val[lt * (4 * S) + pe], in);
    }
    __syncthreads();
    group_walk<S, G, V>(spx, val, pd, srcl);
    __syncthreads();
    for (int n = threadIdx.x; n < NS; n += NTG) {
      if (!(spx[n] & PEX_EXIT)) continue;
      const int lt = n / (4 * S), s = n - lt * (4 * S);
      const int64_t cy = gy * G + lt / G, cx = gx * G + lt % G;
      cfin[(cd.tile_base + cy * cd.ntx + cx) * (4 * S) + s] = val[n];
    }
  }
}

// ---- top level: Algorithms 5-6 over the remaining units, in global memory

template <int S, class V, class CV>
__global__ void k_top_init(DemTable dt, const uint16_t* pex, const CV* pval, V* fin, uint32_t* par, uint32_t* deg,
                           int64_t nslots) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nslots; g += stride) {
    const uint16_t pe = pex[g];
    uint32_t pr = ROOT;
    if (pe & PEX_EXIT) {
      const int64_t t = g / (4 * S);
      const int s = (int)(g - t * (4 * S));
      const DemDesc d = dem_of(dt, t);
      const int64_t lt = t - d.tile_base;
      const UnitGeo u = unit_geo(d, lt / d.ntx, lt % d.ntx, S);
      int i, j;
      slot_cell(s, u.h, u.w, S, i, j);
      const int k = pe & 7;
      const int64_t y = global_slot(d, u.i0 + i + code_di(k), u.j0 + j + code_dj(k), S);
      const uint16_t pey = pex[y];
      if (pey & PEX_EXIT)
        pr = (uint32_t)y;
      else if (pey != PEX_TERM)
        pr = (uint32_t)((y / (4 * S)) * (4 * S) + pey);
      if constexpr (std::is_same<V, uint32_t>::value) {
        // unit counts: children left (high half) and value (low half) in one
        // 64-bit word per node (zeroed before the launch)
        unsigned long long* fd = reinterpret_cast<unsigned long long*>(deg);
        if (pr != ROOT) atomicAdd(&fd[pr], 1ull << 32);
        atomicAdd(&fd[g], (unsigned long long)pval[g]);
      } else {
        if (pr != ROOT) atomicAdd(&deg[pr], 1u);
        fin[g] = pval[g];
      }
    }
    par[g] = pr;
  }
}

// The sources (exits without children) listed, and the exits counted, with
// one atomic per block on each grid-wide counter: a first pass counts this
// thread's sources, a block scan gives each thread its offset inside the
// block's range, and a second pass writes them (same slots, same order).
// (PK: children counts packed in the high half of 64-bit node words)
template <bool PK>
__global__ void __launch_bounds__(256) k_top_sources(const uint16_t* pex, const uint32_t* deg, uint32_t* list,
                                                     uint32_t* counters, int64_t nslots) {
  auto childless = [&](int64_t g) {
    return PK ? (reinterpret_cast<const unsigned long long*>(deg)[g] >> 32) == 0ull : deg[g] == 0u;
  };
  __shared__ uint32_t sh[256];
  __shared__ uint32_t sh_base;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t nsrc = 0, nex = 0;
  for (int64_t g = g0; g < nslots; g += stride) {
    const bool ex = (pex[g] & PEX_EXIT) != 0;
    nex += ex;
    nsrc += ex && childless(g);
  }
  // block-wide inclusive scan of the source counts (Hillis-Steele)
  sh[threadIdx.x] = nsrc;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const uint32_t add = threadIdx.x >= off ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += add;
    __syncthreads();
  }
  const uint32_t block_src = sh[255];
  uint32_t excl = sh[threadIdx.x] - nsrc;
  __syncthreads();
  // exits: reduce into sh[0] with a second scan-free pass
  sh[threadIdx.x] = nex;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    sh_base = block_src ? atomicAdd(&counters[0], block_src) : 0u;
    if (sh[0]) atomicAdd(&counters[1], sh[0]);
  }
  __syncthreads();
  uint32_t pos = sh_base + excl;
  if (nsrc)
    for (int64_t g = g0; g < nslots; g += stride)
      if ((pex[g] & PEX_EXIT) && childless(g)) list[pos++] = (uint32_t)g;
}

// Algorithm 6 with global atomics: last-arriver walks up the exit forest.
// Unit counts: one packed 64-bit atomic per step delivers the value and tells
// the last child (no fences); each finished node stores its value for the
// down sweep.  Float-float: value add, fence, children count, fence.
template <class V>
__global__ void k_top_walk(const uint32_t* par, V* fin, uint32_t* deg, const uint32_t* list, uint32_t* counters) {
  const uint32_t n = *(volatile const uint32_t*)&counters[0];
  uint32_t done = 0;
  if constexpr (std::is_same<V, uint32_t>::value) {
    unsigned long long* fd = reinterpret_cast<unsigned long long*>(deg);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      uint32_t x = list[i];
      uint32_t v = (uint32_t)fd[x];  // a source: its own value
      for (;;) {
        fin[x] = v;
        done++;
        const uint32_t p = par[x];
        if (p == ROOT) break;
        const unsigned long long old = atomicAdd(&fd[p], (unsigned long long)v - (1ull << 32));
        if ((old >> 32) != 1ull) break;
        v += (uint32_t)old;
        x = p;
      }
    }
  } else {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      uint32_t x = list[i];
      V v = fin[x];
      done++;
      for (;;) {
        const uint32_t p = par[x];
        if (p == ROOT) break;
        vatomic_add(&fin[p], v);
        if (atomic_add_acq_rel_gpu(&deg[p], 0u - 1u) != 1u) break;  // releases the addition; acquires the others'
        x = p;
        v = vload_volatile(&fin[p]);
        done++;
      }
    }
  }
  if (done) atomicAdd(&counters[2], done);
}

__global__ void k_top_check(const uint32_t* counters, uint32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && counters[1] != counters[2]) set_status(status, D8_ERR_CYCLE);
}

// ---- top level by pointer jumping (strategy 2).  The queue walk above costs
// one dependent global atomic per node of the longest chain, which a channel
// crossing the top-level units 10^5 times makes tens of milliseconds.  Here
// every exit y keeps P(y) = its 2^r-th ancestor (ROOT past the root); a round
// adds each exit's partial sum to P(y) and jumps (P(y) = P(P(y))), the sums
// are applied, and after ceil(log2(depth)) rounds every exit holds its
// subtree sum (Algorithm 6's result) in fin.  Rounds after the last active
// one return at once (a per-round flag).

// parents, values (fin = pval at exits), additions zeroed, first round flag
template <int S, class V, class CV>
__global__ void k_topj_init(DemTable dt, const uint16_t* pex, const CV* pval, V* fin, uint32_t* par, V* add,
                            uint32_t* flags, int64_t nslots) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  bool any = false;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nslots; g += stride) {
    const uint16_t pe = pex[g];
    uint32_t pr = ROOT;
    if (pe & PEX_EXIT) {
      const int64_t t = g / (4 * S);
      const int s = (int)(g - t * (4 * S));
      const DemDesc d = dem_of(dt, t);
      const int64_t lt = t - d.tile_base;
      const UnitGeo u = unit_geo(d, lt / d.ntx, lt % d.ntx, S);
      int i, j;
      slot_cell(s, u.h, u.w, S, i, j);
      const int k = pe & 7;
      const int64_t y = global_slot(d, u.i0 + i + code_di(k), u.j0 + j + code_dj(k), S);
      const uint16_t pey = pex[y];
      if (pey & PEX_EXIT)
        pr = (uint32_t)y;
      else if (pey != PEX_TERM)
        pr = (uint32_t)((y / (4 * S)) * (4 * S) + pey);
      fin[g] = V(pval[g]);
      add[g] = V{};
      any |= pr != ROOT;
    }
    par[g] = pr;
  }
  if (__syncthreads_or(any) && threadIdx.x == 0) flags[0] = 1u;
}

// one round over the listed exits: scatter to the 2^r-th ancestor, then jump
template <class V>
__global__ void k_topj_round(const uint32_t* list, const uint32_t* counters, const uint32_t* pc, uint32_t* pn,
                             const V* fin, V* add, uint32_t* flags, int r) {
  if (*(volatile const uint32_t*)&flags[r] == 0u) return;
  const uint32_t n = counters[0];
  bool active = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t y = list[i];
    const uint32_t a = pc[y];
    if (a == ROOT) {
      pn[y] = ROOT;
      continue;
    }
    vatomic_add(&add[a], fin[y]);
    const uint32_t aa = pc[a];
    pn[y] = aa;
    active |= aa != ROOT;
  }
  if (__syncthreads_or(active) && threadIdx.x == 0) flags[r + 1] = 1u;
}

template <class V>
__global__ void k_topj_apply(const uint32_t* list, const uint32_t* counters, V* fin, V* add, const uint32_t* flags,
                             int r) {
  if (*(volatile const uint32_t*)&flags[r] == 0u) return;
  const uint32_t n = counters[0];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t y = list[i];
    const V dv = add[y];
    fin[y] = vadd(fin[y], dv);
    add[y] = V{};
  }
}

// exits still jumping after the last round: the exit forest has a cycle
__global__ void k_topj_check(const uint32_t* flags, int R, uint32_t* status) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && flags[R] != 0u) set_status(status, D8_ERR_CYCLE);
}

// every exit listed (same scheme as k_top_sources: one atomic per block)
__global__ void __launch_bounds__(256) k_topj_list(const uint16_t* pex, uint32_t* list, uint32_t* counters,
                                                   int64_t nslots) {
  __shared__ uint32_t sh[256];
  __shared__ uint32_t sh_base;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t nex = 0;
  for (int64_t g = g0; g < nslots; g += stride) nex += (pex[g] & PEX_EXIT) != 0;
  sh[threadIdx.x] = nex;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const uint32_t a = threadIdx.x >= off ? sh[threadIdx.x - off] : 0u;
    __syncthreads();
    sh[threadIdx.x] += a;
    __syncthreads();
  }
  if (threadIdx.x == 255) sh_base = sh[255] ? atomicAdd(&counters[0], sh[255]) : 0u;
  __syncthreads();
  uint32_t pos = sh_base + sh[threadIdx.x] - nex;
  if (nex)
    for (int64_t g = g0; g < nslots; g += stride)
      if (pex[g] & PEX_EXIT) list[pos++] = (uint32_t)g;
}

template <int S, int G, class V, class CV>
static cudaError_t launch_level_up(const DemTable& cdt, const DemTable& gdt, const uint16_t* cpex, const void* cpval,
                                   uint16_t* gpex, void* gpval, int64_t ngroups, uint32_t* queue, uint32_t* status,
                                   cudaStream_t s) {
  using L = GroupLayout<S, G, V>;
  auto k = k_group_up<S, G, V, CV>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 1, dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTG, L::bytes);
  int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  if (grid > ngroups) grid = ngroups;
  e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, NTG, L::bytes, s>>>(cdt, gdt, cpex, static_cast<const CV*>(cpval), gpex, static_cast<V*>(gpval),
                                          ngroups, queue, status);
  return cudaGetLastError();
}

template <int S, int G, class V, class CV>
static cudaError_t launch_level_down(const DemTable& cdt, const DemTable& gdt, const uint16_t* cpex, const void* cpval,
                                     void* cfin, const void* gfin, int64_t ngroups, uint32_t* queue, cudaStream_t s) {
  using L = GroupLayout<S, G, V>;
  auto k = k_group_down<S, G, V, CV>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes);
  if (e != cudaSuccess) return e;
  int per_sm = 1, dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTG, L::bytes);
  int64_t grid = (int64_t)(per_sm < 1 ? 1 : per_sm) * sms;
  if (grid > ngroups) grid = ngroups;
  e = cudaMemsetAsync(queue, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)grid, NTG, L::bytes, s>>>(cdt, gdt, cpex, static_cast<const CV*>(cpval), static_cast<V*>(cfin),
                                          static_cast<const V*>(gfin), ngroups, queue);
  return cudaGetLastError();
}

template <int S, class V, class CV>
static cudaError_t launch_top_jump(const DemTable& dt, const HLevel& lv, const HTop& top, cudaStream_t s, int* nl) {
  const int64_t ns = lv.nunits * 4 * S;
  cudaError_t e = cudaMemsetAsync(top.flags, 0, sizeof(uint32_t) * (MAX_ROUNDS + 2), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(top.counters, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (ns + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  if (b < 1) b = 1;
  V* fin = static_cast<V*>(lv.fin);
  V* add = reinterpret_cast<V*>(top.deg);
  k_topj_init<S, V, CV><<<(unsigned)b, 256, 0, s>>>(dt, lv.pex, static_cast<const CV*>(lv.pval), fin, top.par, add,
                                                    top.flags, ns);
  k_topj_list<<<(unsigned)b, 256, 0, s>>>(lv.pex, top.list, top.counters, ns);
  // rounds: enough for a chain through every slot
  int R = 1;
  while (R < MAX_ROUNDS && ((int64_t)1 << R) < ns) R++;
  for (int r = 0; r < R; r++) {
    uint32_t* pc = (r & 1) ? top.par2 : top.par;
    uint32_t* pn = (r & 1) ? top.par : top.par2;
    k_topj_round<V><<<(unsigned)b, 256, 0, s>>>(top.list, top.counters, pc, pn, fin, add, top.flags, r);
    k_topj_apply<V><<<(unsigned)b, 256, 0, s>>>(top.list, top.counters, fin, add, top.flags, r);
  }
  k_topj_check<<<1, 32, 0, s>>>(top.flags, R, top.status);
  *nl += 3 + 2 * R;
  return cudaGetLastError();
}

template <int S, class V, class CV>
static cudaError_t launch_top(const DemTable& dt, const HLevel& lv, const HTop& top, cudaStream_t s, int* nl) {
  if (top.jump) return launch_top_jump<S, V, CV>(dt, lv, top, s, nl);
  const int64_t ns = lv.nunits * 4 * S;
  cudaError_t e = cudaMemsetAsync(top.deg, 0, sizeof(unsigned long long) * (size_t)ns, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(top.counters, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t b = (ns + 255) / 256;
  if (b > (int64_t)sms * 16) b = (int64_t)sms * 16;
  if (b < 1) b = 1;
  k_top_init<S, V, CV><<<(unsigned)b, 256, 0, s>>>(dt, lv.pex, static_cast<const CV*>(lv.pval),
                                                   static_cast<V*>(lv.fin), top.par, top.deg, ns);
  k_top_sources<std::is_same<V, uint32_t>::value><<<(unsigned)b, 256, 0, s>>>(lv.pex, top.deg, top.list,
                                                                             top.counters, ns);
  k_top_walk<V><<<(unsigned)(sms * 8), 256, 0, s>>>(top.par, static_cast<V*>(lv.fin), top.deg, top.list,
                                                    top.counters);
  k_top_check<<<1, 32, 0, s>>>(top.counters, top.status);
  *nl += 4;
  return cudaGetLastError();
}

}  // namespace cmb

// Level schedule: tiles of side T, then groups of G = 4 (from 32 or 64) or
// G = 2 children, up to a group side of 512 cells; the global queue solve
// takes the rest.  (A 1024-cell level cost more than the longer top-level
// chains it saves: measured at 8192^2 and 32768^2.)
int hier_levels(int T, int64_t max_side, int* S, int* G, int max_levels) {
  int n = 0;
  int s = T;
  while (n < max_levels && s < max_side && s < 512) {
    const int g = (s <= 64) ? 4 : 2;
    S[n] = s;
    G[n] = g;
    s *= g;
    n++;
  }
  return n;
}

namespace cmb {

// V: accumulation type above the tiles; CV0: the tiles' stored pval type
template <class V, class CV0>
static cudaError_t combine_hier_t(const HPlan& hp, cudaStream_t s, int* nlaunch) {
  cudaError_t e = cudaSuccess;
  // up: level l-1 -> l
  for (int l = 1; l <= hp.nlev && e == cudaSuccess; l++) {
    const HLevel& c = hp.lev[l - 1];
    const HLevel& g = hp.lev[l];
    const int S = c.S, G = g.S / c.S;
#define D8_UP(SS, GG)                                                                                             \
  if (S == SS && G == GG) {                                                                                      \
    e = l == 1 ? launch_level_up<SS, GG, V, CV0>(c.dt, g.dt, c.pex, c.pval, g.pex, g.pval, g.nunits, hp.queue + l,  \
                                                 hp.status, s)                                                   \
               : launch_level_up<SS, GG, V, V>(c.dt, g.dt, c.pex, c.pval, g.pex, g.pval, g.nunits, hp.queue + l,    \
                                               hp.status, s);                                                    \
    ++*nlaunch;                                                                                                  \
    continue;                                                                                                    \
  }
    D8_UP(32, 4) D8_UP(64, 4) D8_UP(128, 2) D8_UP(256, 2) D8_UP(512, 2)
#undef D8_UP
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  // top
  const HLevel& t = hp.lev[hp.nlev];
  if (hp.need_top) {
    const bool l0 = hp.nlev == 0;
#define D8_TOP(SS)                                                                                 \
  case SS:                                                                                         \
    e = l0 ? launch_top<SS, V, CV0>(t.dt, t, hp.top, s, nlaunch) : launch_top<SS, V, V>(t.dt, t, hp.top, s, nlaunch); \
    break;
    switch (t.S) {
      D8_TOP(32) D8_TOP(64) D8_TOP(128) D8_TOP(256) D8_TOP(512) D8_TOP(1024)
      default: return cudaErrorInvalidValue;
    }
#undef D8_TOP
    if (e != cudaSuccess) return e;
  }
  // down: level l -> l-1
  for (int l = hp.nlev; l >= 1 && e == cudaSuccess; l--) {
    const HLevel& c = hp.lev[l - 1];
    const HLevel& g = hp.lev[l];
    const int S = c.S, G = g.S / c.S;
#define D8_DN(SS, GG)                                                                                               \
  if (S == SS && G == GG) {                                                                                        \
    e = l == 1 ? launch_level_down<SS, GG, V, CV0>(c.dt, g.dt, c.pex, c.pval, c.fin, g.fin, g.nunits,               \
                                                   hp.queue + 16 + l, s)                                           \
               : launch_level_down<SS, GG, V, V>(c.dt, g.dt, c.pex, c.pval, c.fin, g.fin, g.nunits, hp.queue + 16 + l, \
                                                 s);                                                               \
    ++*nlaunch;                                                                                                    \
    continue;                                                                                                      \
  }
    D8_DN(32, 4) D8_DN(64, 4) D8_DN(128, 2) D8_DN(256, 2) D8_DN(512, 2)
#undef D8_DN
    return cudaErrorInvalidValue;
  }
  return e;
}

}  // namespace cmb

cudaError_t launch_combine_hier(const HPlan& hp, cudaStream_t s, int* nlaunch) {
  if (!hp.weighted) return cmb::combine_hier_t<uint32_t, uint32_t>(hp, s, nlaunch);
  return cmb::combine_hier_t<ff, ff>(hp, s, nlaunch);
}

}  // namespace d8
