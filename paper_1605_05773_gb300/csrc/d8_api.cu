// d8_api.cu -- the C ABI of libd8 (declared in include/d8.h): contexts,
// workspace, argument checks, stage timing, the forward / weighted / backward
// pipelines and the batch plan with CUDA-graph replay.
#include <nvtx3/nvToolsExt.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "d8.h"
#include "d8_internal.h"

using namespace d8;

namespace {

enum Stage { ST_FLOWDIR = 0, ST_UP, ST_COMBINE, ST_DOWN, ST_BWD_UP, ST_BWD_COMBINE, ST_BWD_DOWN, ST_FILL, ST_COUNT };
const char* const kStageNames[ST_COUNT] = {"flowdir", "tile_up", "combine", "tile_down",
                                           "bwd_tile_up", "bwd_combine", "bwd_tile_down", "fill"};

struct Timing {
  int stage;
  cudaEvent_t a, b;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int bit_width(uint64_t x) {
  int r = 0;
  while (x) {
    r++;
    x >>= 1;
  }
  return r;
}

}  // namespace

struct d8_ctx {
  int device = 0;
  int T = 64;
  int strat = d8::STRAT_RING;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint32_t* status = nullptr;
  int profiling = 0;
  std::vector<cudaEvent_t> free_events;
  std::vector<Timing> pending;
  double ms[ST_COUNT] = {};
  int64_t launches[ST_COUNT] = {};
  // the last forward call's combine, for d8_combine_stats
  int last_levels = 0;
  int64_t last_top_units = 0;
  bool last_jump = false;
  uint32_t* last_counters = nullptr;
  uint32_t* last_flags = nullptr;
};

struct d8_batch {
  d8_ctx* ctx = nullptr;
  int n = 0;
  int T = 64;
  int strat = d8::STRAT_RING;
  std::vector<DemDesc> host_desc;
  DemDesc* dev_desc = nullptr;
  int32_t* dev_tile_dem = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int64_t ntiles = 0;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  int graph_rule = -1;
  cudaStream_t graph_stream = nullptr;
  int launches_per_run = 0;
  // layered combine: per level l >= 1, a table of per-DEM unit grids and a
  // unit -> DEM map (level 0 uses the tile table above)
  int nlev = 0;
  bool need_top = false;
  int lev_S[HMAX + 1] = {};
  int64_t lev_units[HMAX + 1] = {};
  std::vector<DemDesc> lev_host[HMAX + 1];
  DemDesc* lev_desc[HMAX + 1] = {};
  int32_t* lev_map[HMAX + 1] = {};
  size_t pipe_part = 0;
};

namespace {

d8_status cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return D8_ERR_NOMEM;
  return e == cudaSuccess ? D8_OK : D8_ERR_CUDA;
}

cudaEvent_t get_event(d8_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// RAII bracket of one stage: an NVTX range named after the stage (host
// side, around the stage's launches), launch counting, and CUDA events when
// profiling is on
struct StageScope {
  d8_ctx* c;
  int st;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  int n = 0;
  StageScope(d8_ctx* c_, int st_, cudaStream_t s_) : c(c_), st(st_), s(s_) {
    nvtxRangePushA(kStageNames[st]);
    if (c->profiling) {
      a = get_event(c);
      cudaEventRecord(a, s);
    }
  }
  ~StageScope() {
    nvtxRangePop();
    c->launches[st] += n;
    if (c->profiling && a) {
      cudaEvent_t b = get_event(c);
      cudaEventRecord(b, s);
      c->pending.push_back(Timing{st, a, b});
    }
  }
};

bool bad_grid(const void* p, int64_t H, int64_t W, int64_t ld) { return !p || H < 1 || W < 1 || ld < W; }

// Workspace for a pipeline over `ntiles` tiles of side T with value size vbytes.
size_t pipe_bytes(int64_t ntiles, int T, size_t vbytes) {
  const size_t ns = (size_t)ntiles * 4 * T;
  return align256(ns * 2) + align256(ns * vbytes) + 2 * align256(ns * 4) + 2 * align256(ns * vbytes) +
         align256(sizeof(uint32_t) * (MAX_ROUNDS + 2)) + align256(sizeof(uint32_t) * 16);
}

Pipe carve_pipe(void* base, int64_t ntiles, int T, size_t vbytes, uint32_t* status) {
  Pipe p{};
  p.T = T;
  p.ntiles = ntiles;
  p.nslots = ntiles * 4 * T;
  p.rounds = bit_width((uint64_t)p.nslots);
  if (p.rounds > MAX_ROUNDS) p.rounds = MAX_ROUNDS;
  const size_t ns = (size_t)p.nslots;
  char* q = static_cast<char*>(base);
  p.pex = reinterpret_cast<uint16_t*>(q);
  q += align256(ns * 2);
  p.pval = q;
  q += align256(ns * vbytes);
  p.P[0] = reinterpret_cast<uint32_t*>(q);
  q += align256(ns * 4);
  p.P[1] = reinterpret_cast<uint32_t*>(q);
  q += align256(ns * 4);
  p.S = q;
  q += align256(ns * vbytes);
  p.S2 = q;
  q += align256(ns * vbytes);
  p.flags = reinterpret_cast<uint32_t*>(q);
  q += align256(sizeof(uint32_t) * (MAX_ROUNDS + 2));
  p.queue = reinterpret_cast<uint32_t*>(q);
  p.status = status;
  return p;
}

// ---- layered combine plan (single DEM or batch) ---------------------------
struct HShape {
  int nlev = 0;
  int S[HMAX + 1] = {};
  int64_t nunits[HMAX + 1] = {};
  bool need_top = false;
};

// Levels above tiles of side T for the given DEM shapes.
HShape hier_shape(int T, int n, const int64_t* H, const int64_t* W) {
  HShape hs;
  int64_t mx = 1;
  for (int k = 0; k < n; k++) mx = H[k] > mx ? H[k] : (W[k] > mx ? W[k] : mx);
  for (int k = 0; k < n; k++) mx = W[k] > mx ? W[k] : mx;
  int S[HMAX], G[HMAX];
  hs.nlev = hier_levels(T, mx, S, G, HMAX - 1);
  hs.S[0] = T;
  for (int l = 1; l <= hs.nlev; l++) hs.S[l] = S[l - 1] * G[l - 1];
  for (int l = 0; l <= hs.nlev; l++) {
    int64_t u = 0;
    for (int k = 0; k < n; k++) {
      const int64_t nu = ((H[k] + hs.S[l] - 1) / hs.S[l]) * ((W[k] + hs.S[l] - 1) / hs.S[l]);
      u += nu;
      if (l == hs.nlev && nu > 1) hs.need_top = true;
    }
    hs.nunits[l] = u;
  }
  return hs;
}

// vb: bytes per level value (4 for unit counts, 8 for weighted float-float)
size_t hier_bytes(const HShape& hs, size_t vb) {
  size_t b = 0;
  for (int l = 1; l <= hs.nlev; l++) {
    const size_t ns = (size_t)hs.nunits[l] * 4 * hs.S[l];
    b += align256(ns * 2) + 2 * align256(ns * vb);
  }
  const size_t nt = (size_t)hs.nunits[hs.nlev] * 4 * hs.S[hs.nlev];
  // par, par2, list; children counts or additions (8 B); round flags
  if (hs.need_top) b += 3 * align256(nt * 4) + align256(nt * 8) + align256(sizeof(uint32_t) * (MAX_ROUNDS + 2));
  b += align256(sizeof(uint32_t) * 64);
  return b;
}

// Carve the level arrays; level 0 takes the tile pipeline's arrays.  `dts`
// holds each level's DEM table (filled by the caller).
HPlan carve_hier(void* base, const HShape& hs, const Pipe& p, const DemTable* dts, bool weighted) {
  HPlan hp{};
  hp.weighted = weighted;
  hp.top.jump = p.strat == STRAT_JUMP;
  hp.nlev = hs.nlev;
  hp.need_top = hs.need_top;
  hp.status = p.status;
  hp.lev[0].S = hs.S[0];
  hp.lev[0].nunits = hs.nunits[0];
  hp.lev[0].dt = dts[0];
  hp.lev[0].pex = p.pex;
  hp.lev[0].pval = p.pval;
  hp.lev[0].fin = p.S;
  const size_t vb = weighted ? 8 : 4;
  char* q = static_cast<char*>(base);
  for (int l = 1; l <= hs.nlev; l++) {
    const size_t ns = (size_t)hs.nunits[l] * 4 * hs.S[l];
    HLevel& L = hp.lev[l];
    L.S = hs.S[l];
    L.nunits = hs.nunits[l];
    L.dt = dts[l];
    L.pex = reinterpret_cast<uint16_t*>(q);
    q += align256(ns * 2);
    L.pval = q;
    q += align256(ns * vb);
    L.fin = q;
    q += align256(ns * vb);
  }
  const size_t nt = (size_t)hs.nunits[hs.nlev] * 4 * hs.S[hs.nlev];
  if (hs.need_top) {
    hp.top.par = reinterpret_cast<uint32_t*>(q);
    q += align256(nt * 4);
    hp.top.par2 = reinterpret_cast<uint32_t*>(q);
    q += align256(nt * 4);
    hp.top.deg = reinterpret_cast<uint32_t*>(q);  // 8 bytes per slot (unit counts pack value and count)
    q += align256(nt * 8);
    hp.top.list = reinterpret_cast<uint32_t*>(q);
    q += align256(nt * 4);
    hp.top.flags = reinterpret_cast<uint32_t*>(q);
    q += align256(sizeof(uint32_t) * (MAX_ROUNDS + 2));
  }
  hp.queue = reinterpret_cast<uint32_t*>(q);
  hp.top.counters = hp.queue + 48;
  hp.top.status = p.status;
  return hp;
}

d8_status ensure_ws(d8_ctx* c, size_t bytes) {
  if (c->ws_bytes >= bytes) return D8_OK;
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&c->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c->ws = nullptr;
    return D8_ERR_NOMEM;
  }
  c->ws_bytes = bytes;
  return D8_OK;
}

DemDesc make_desc(int64_t H, int64_t W, int T) {
  DemDesc d{};
  d.H = H;
  d.W = W;
  d.ntx = (W + T - 1) / T;
  d.nty = (H + T - 1) / T;
  d.tile_base = 0;
  return d;
}

DemTable single(const DemDesc& d) {
  DemTable t{};
  t.one = d;
  t.ndem = 1;
  return t;
}

bool slots_fit(int64_t ntiles, int T) { return (uint64_t)ntiles * 4 * (uint64_t)T < 0xFFFFFFF0ull; }

// forward pipeline on one DEM: directions (when z is given), tile pass,
// combine, finalise
d8_status run_forward(d8_ctx* c, const DemDesc& d0, int mode, int rule, cudaStream_t s,
                      const uint32_t* top_in = nullptr, const uint32_t* bot_in = nullptr) {
  const int T = c->T;
  DemDesc d = d0;
  const int64_t ntiles = d.ntx * d.nty;
  if (!slots_fit(ntiles, T)) return D8_ERR_SHAPE;
  const bool weighted = (mode == UP_WEIGHTED);
  const size_t vb = weighted ? 8 : 4;
  if (up_smem_bytes(T, mode) == 0 || down_smem_bytes(T, weighted) == 0) return D8_ERR_ARG;
  const HShape hs = hier_shape(T, 1, &d.H, &d.W);
  const size_t hb = hier_bytes(hs, vb);
  const size_t pb = align256(pipe_bytes(ntiles, T, vb));
  d8_status st = ensure_ws(c, pb + hb);
  if (st != D8_OK) return st;
  Pipe p = carve_pipe(c->ws, ntiles, T, vb, c->status);
  p.strat = c->strat;
  p.top_in = top_in;
  p.bot_in = bot_in;
  DemTable dt = single(d);
  cudaError_t e = cudaMemsetAsync(p.queue, 0, sizeof(uint32_t) * 16, s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (mode == UP_UNIT_Z) {
    StageScope sc(c, ST_FLOWDIR, s);
    e = launch_flowdir(dt, ntiles, T, rule, c->status, s, &sc.n);
    mode = UP_UNIT_DIR;
  }
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_UP, s);
    e = launch_up(dt, p, mode, rule, s, &sc.n);
    if (e == cudaSuccess && (top_in || bot_in)) e = launch_inject_inflow(d, p, s, &sc.n);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_COMBINE, s);
    DemTable dts[HMAX + 1];
    for (int l = 0; l <= hs.nlev; l++) {
      DemDesc dl = d;
      dl.ntx = (d.W + hs.S[l] - 1) / hs.S[l];
      dl.nty = (d.H + hs.S[l] - 1) / hs.S[l];
      dl.tile_base = 0;
      dts[l] = single(dl);
    }
    const HPlan hp = carve_hier(static_cast<char*>(c->ws) + pb, hs, p, dts, weighted);
    c->last_levels = hs.nlev;
    c->last_top_units = hs.need_top ? hs.nunits[hs.nlev] : 0;
    c->last_jump = hp.top.jump;
    c->last_counters = hs.need_top ? hp.top.counters : nullptr;
    c->last_flags = hs.need_top ? hp.top.flags : nullptr;
    e = launch_combine_hier(hp, s, &sc.n);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_DOWN, s);
    e = launch_down(dt, p, weighted, s, &sc.n);
  }
  return cuda_fail(e);
}

}  // namespace

extern "C" {

const char* d8_version(void) { return "libd8 0.1 (sm_103a)"; }

const char* d8_status_string(d8_status s) {
  switch (s) {
    case D8_OK: return "ok";
    case D8_ERR_ARG: return "invalid argument or direction code";
    case D8_ERR_SHAPE: return "grid too large for the output type";
    case D8_ERR_NONFINITE: return "non-finite elevation";
    case D8_ERR_CYCLE: return "direction field contains a cycle";
    case D8_ERR_NOMEM: return "out of device memory";
    case D8_ERR_CUDA: return "CUDA runtime error";
    case D8_ERR_TIMEOUT: return "bounded device wait timed out";
    case D8_ERR_CAPACITY: return "grid exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

const char* d8_stage_name(int stage) { return (stage >= 0 && stage < ST_COUNT) ? kStageNames[stage] : nullptr; }

d8_status d8_create(d8_ctx** out, int device) {
  if (!out) return D8_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
    cudaGetLastError();
    return D8_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return D8_ERR_CUDA;
  d8_ctx* c = new (std::nothrow) d8_ctx();
  if (!c) return D8_ERR_NOMEM;
  c->device = device;
  if (cudaMalloc(&c->status, 256) != cudaSuccess || cudaMemset(c->status, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return D8_ERR_NOMEM;
  }
  *out = c;
  return D8_OK;
}

d8_status d8_destroy(d8_ctx* c) {
  if (!c) return D8_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  if (c->ws) cudaFree(c->ws);
  if (c->status) cudaFree(c->status);
  for (auto& t : c->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : c->free_events) cudaEventDestroy(e);
  delete c;
  return D8_OK;
}

d8_status d8_set_tile(d8_ctx* c, int tile) {
  if (!c || (tile != 32 && tile != 64 && tile != 128)) return D8_ERR_ARG;
  c->T = tile;
  return D8_OK;
}

d8_status d8_set_strategy(d8_ctx* c, int strategy) {
  if (!c || strategy < 0 || strategy >= STRAT_COUNT) return D8_ERR_ARG;
  c->strat = strategy;
  return D8_OK;
}

d8_status d8_set_profiling(d8_ctx* c, int on) {
  if (!c) return D8_ERR_ARG;
  c->profiling = on ? 1 : 0;
  return D8_OK;
}

d8_status d8_stage_times(d8_ctx* c, float* ms, int64_t* launches, int max, int* n) {
  if (!c) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  for (auto& t : c->pending) {
    if (cudaEventSynchronize(t.b) != cudaSuccess) return D8_ERR_CUDA;
    float x = 0.0f;
    cudaEventElapsedTime(&x, t.a, t.b);
    c->ms[t.stage] += x;
    c->free_events.push_back(t.a);
    c->free_events.push_back(t.b);
  }
  c->pending.clear();
  for (int s = 0; s < ST_COUNT && s < max; s++) {
    if (ms) ms[s] = (float)c->ms[s];
    if (launches) launches[s] = c->launches[s];
  }
  for (int s = 0; s < ST_COUNT; s++) {
    c->ms[s] = 0.0;
    c->launches[s] = 0;
  }
  if (n) *n = ST_COUNT;
  return D8_OK;
}

d8_status d8_combine_stats(d8_ctx* c, d8_stream stream, int64_t* out, int n) {
  if (!c || !out || n < 4) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  out[0] = c->last_levels;
  out[1] = c->last_top_units;
  out[2] = 0;
  out[3] = -1;
  if (!c->last_counters) return D8_OK;
  uint32_t cnt[4] = {}, fl[MAX_ROUNDS + 2] = {};
  cudaError_t e = cudaMemcpyAsync(cnt, c->last_counters, sizeof(cnt), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && c->last_jump) e = cudaMemcpyAsync(fl, c->last_flags, sizeof(fl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return D8_ERR_CUDA;
  if (c->last_jump) {
    out[2] = cnt[0];  // every exit listed
    int r = 0;
    while (r < MAX_ROUNDS + 1 && fl[r]) r++;
    out[3] = r;
  } else {
    out[2] = cnt[1];  // exits counted by the source listing
  }
  return D8_OK;
}

d8_status d8_get_status(d8_ctx* c, d8_stream stream) {
  if (!c) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, c->status, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return D8_ERR_CUDA;
  const d8_status order[] = {D8_ERR_NONFINITE, D8_ERR_ARG, D8_ERR_CYCLE, D8_ERR_TIMEOUT};
  for (d8_status o : order)
    if (h & (1u << o)) return o;
  return D8_OK;
}

d8_status d8_flowdir(d8_ctx* c, const float* z, int64_t H, int64_t W, int64_t ldz, uint8_t* dir, int64_t lddir,
                     d8_rule rule, d8_stream stream) {
  if (!c || bad_grid(z, H, W, ldz) || bad_grid(dir, H, W, lddir) || (rule < 0 || rule > 3)) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.z = z;
  d.ldz = ldz;
  d.dir = dir;
  d.lddir = lddir;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StageScope sc(c, ST_FLOWDIR, s);
  return cuda_fail(launch_flowdir(single(d), d.ntx * d.nty, c->T, (int)rule, c->status, s, &sc.n));
}

d8_status d8_accumulate(d8_ctx* c, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir, uint32_t* A,
                        int64_t ldA, d8_stream stream) {
  if (!c || bad_grid(dir, H, W, lddir) || bad_grid(A, H, W, ldA)) return D8_ERR_ARG;
  if ((uint64_t)H * (uint64_t)W > 0xFFFFFFFFull) return D8_ERR_SHAPE;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.dir = const_cast<uint8_t*>(dir);
  d.lddir = lddir;
  d.A = A;
  d.ldA = ldA;
  return run_forward(c, d, UP_UNIT_DIR, 0, static_cast<cudaStream_t>(stream));
}

d8_status d8_flowdir_strip(d8_ctx* c, const float* z, int64_t H, int64_t W, int64_t ldz, int halo, d8_rule rule,
                           uint8_t* dir, int64_t lddir, d8_stream stream) {
  if (!c || bad_grid(z, H, W, ldz) || bad_grid(dir, H, W, lddir) || (rule < 0 || rule > 3) || halo < 0 || halo > 3)
    return D8_ERR_ARG;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.z = z;
  d.ldz = ldz;
  d.dir = dir;
  d.lddir = lddir;
  d.halo = halo;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  StageScope sc(c, ST_FLOWDIR, s);
  return cuda_fail(launch_flowdir(single(d), d.ntx * d.nty, c->T, (int)rule, c->status, s, &sc.n));
}

d8_status d8_accumulate_inflow(d8_ctx* c, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                               const uint32_t* top_in, const uint32_t* bottom_in, uint32_t* A, int64_t ldA,
                               d8_stream stream) {
  if (!c || bad_grid(dir, H, W, lddir) || bad_grid(A, H, W, ldA)) return D8_ERR_ARG;
  if ((uint64_t)H * (uint64_t)W > 0xFFFFFFFFull) return D8_ERR_SHAPE;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.dir = const_cast<uint8_t*>(dir);
  d.lddir = lddir;
  d.A = A;
  d.ldA = ldA;
  return run_forward(c, d, UP_UNIT_DIR, 0, static_cast<cudaStream_t>(stream), top_in, bottom_in);
}

d8_status d8_flowdir_accumulate(d8_ctx* c, const float* z, int64_t H, int64_t W, int64_t ldz, d8_rule rule,
                                uint8_t* dir, int64_t lddir, uint32_t* A, int64_t ldA, d8_stream stream) {
  if (!c || bad_grid(z, H, W, ldz) || bad_grid(dir, H, W, lddir) || bad_grid(A, H, W, ldA) ||
      (rule < 0 || rule > 3))
    return D8_ERR_ARG;
  if ((uint64_t)H * (uint64_t)W > 0xFFFFFFFFull) return D8_ERR_SHAPE;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.z = z;
  d.ldz = ldz;
  d.dir = dir;
  d.lddir = lddir;
  d.A = A;
  d.ldA = ldA;
  return run_forward(c, d, UP_UNIT_Z, (int)rule, static_cast<cudaStream_t>(stream));
}

d8_status d8_accumulate_weighted(d8_ctx* c, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                                 const float* w, int64_t ldw, float* A, int64_t ldA, d8_stream stream) {
  if (!c || bad_grid(dir, H, W, lddir) || bad_grid(w, H, W, ldw) || bad_grid(A, H, W, ldA)) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  DemDesc d = make_desc(H, W, c->T);
  d.dir = const_cast<uint8_t*>(dir);
  d.lddir = lddir;
  d.w = w;
  d.ldw = ldw;
  d.A = A;
  d.ldA = ldA;
  return run_forward(c, d, UP_WEIGHTED, 0, static_cast<cudaStream_t>(stream));
}

d8_status d8_accumulate_backward(d8_ctx* c, const uint8_t* dir, int64_t H, int64_t W, int64_t lddir,
                                 const float* dA, int64_t lddA, float* dw, int64_t lddw, d8_stream stream) {
  if (!c || bad_grid(dir, H, W, lddir) || bad_grid(dA, H, W, lddA) || bad_grid(dw, H, W, lddw)) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  // The adjoint's tile pass keeps 21 bytes of shared memory per cell, so 64 x 64
  // tiles fit two per SM; a context set to 32 x 32 tiles uses those (128 x 128
  // would not fit).
  const int T = c->T == 32 ? 32 : 64;
  DemDesc d = make_desc(H, W, T);
  d.dir = const_cast<uint8_t*>(dir);
  d.lddir = lddir;
  d.w = dA;
  d.ldw = lddA;
  d.A = dw;
  d.ldA = lddw;
  const int64_t ntiles = d.ntx * d.nty;
  if (!slots_fit(ntiles, T)) return D8_ERR_SHAPE;
  // the pipe, one uint16 per cell (the slot of the cell's tile exit) and two
  // lists of slots for the combine's rounds
  const size_t pb = align256(pipe_bytes(ntiles, T, 8));
  const size_t xb = align256((size_t)H * (size_t)W * 2);
  const size_t lb = align256((size_t)ntiles * 4 * T * 4);
  d8_status st = ensure_ws(c, pb + xb + 2 * lb);
  if (st != D8_OK) return st;
  Pipe p = carve_pipe(c->ws, ntiles, T, 8, c->status);
  p.xid = reinterpret_cast<uint16_t*>(static_cast<char*>(c->ws) + pb);
  p.list[0] = reinterpret_cast<uint32_t*>(static_cast<char*>(c->ws) + pb + xb);
  p.list[1] = reinterpret_cast<uint32_t*>(static_cast<char*>(c->ws) + pb + xb + lb);
  DemTable dt = single(d);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(p.queue, 0, sizeof(uint32_t) * 16, s);
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_BWD_UP, s);
    e = launch_bwd_up(dt, p, s, &sc.n);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_BWD_COMBINE, s);
    e = launch_combine_bwd(dt, p, s, &sc.n);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  {
    StageScope sc(c, ST_BWD_DOWN, s);
    e = launch_bwd_down(dt, p, s, &sc.n);
  }
  return cuda_fail(e);
}

d8_status d8_fill(d8_ctx* c, const float* z, int64_t H, int64_t W, int64_t ldz, float eps, float* F, int64_t ldF,
                  int64_t* rounds, d8_stream stream) {
  if (!c || bad_grid(z, H, W, ldz) || bad_grid(F, H, W, ldF) || !(eps >= 0.0f) || !(eps < INFINITY))
    return D8_ERR_ARG;
  // the output must not overlap the input (the fill reads z throughout)
  const char *zb = reinterpret_cast<const char*>(z), *ze = zb + ((H - 1) * ldz + W) * sizeof(float);
  const char *fb = reinterpret_cast<const char*>(F), *fe = fb + ((H - 1) * ldF + W) * sizeof(float);
  if (zb < fe && fb < ze) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  d8_status st = ensure_ws(c, fill_ws_bytes(H, W));
  if (st != D8_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t r = 0;
  bool timed_out = false;
  cudaError_t e;
  {
    StageScope sc(c, ST_FILL, s);
    e = run_fill(z, H, W, ldz, eps, F, ldF, c->ws, c->status, s, (int64_t)1 << 20, &r, &timed_out, &sc.n);
  }
  if (rounds) *rounds = r;
  if (e != cudaSuccess) return cuda_fail(e);
  return timed_out ? D8_ERR_TIMEOUT : D8_OK;
}

// ---------------------------------------------------------------------------
// batch

d8_status d8_batch_plan(d8_ctx* c, int n, const int64_t* H, const int64_t* W, d8_batch** out) {
  if (!c || !out || n < 1 || !H || !W) return D8_ERR_ARG;
  *out = nullptr;
  cudaSetDevice(c->device);
  d8_batch* b = new (std::nothrow) d8_batch();
  if (!b) return D8_ERR_NOMEM;
  b->ctx = c;
  b->n = n;
  b->T = c->T;
  b->strat = c->strat;
  b->host_desc.resize(n);
  int64_t base = 0;
  for (int k = 0; k < n; k++) {
    if (H[k] < 1 || W[k] < 1) {
      delete b;
      return D8_ERR_ARG;
    }
    if ((uint64_t)H[k] * (uint64_t)W[k] > 0xFFFFFFFFull) {
      delete b;
      return D8_ERR_SHAPE;
    }
    DemDesc d = make_desc(H[k], W[k], b->T);
    d.ldz = d.lddir = d.ldA = W[k];
    d.tile_base = base;
    base += d.ntx * d.nty;
    b->host_desc[k] = d;
  }
  b->ntiles = base;
  if (!slots_fit(base, b->T)) {
    delete b;
    return D8_ERR_SHAPE;
  }
  std::vector<int32_t> tile_dem((size_t)base);
  for (int k = 0; k < n; k++) {
    const DemDesc& d = b->host_desc[k];
    for (int64_t t = 0; t < d.ntx * d.nty; t++) tile_dem[(size_t)(d.tile_base + t)] = k;
  }
  std::vector<int64_t> Hv(H, H + n), Wv(W, W + n);
  const HShape hs = hier_shape(b->T, n, Hv.data(), Wv.data());
  b->nlev = hs.nlev;
  b->need_top = hs.need_top;
  for (int l = 0; l <= hs.nlev; l++) {
    b->lev_S[l] = hs.S[l];
    b->lev_units[l] = hs.nunits[l];
  }
  b->pipe_part = align256(pipe_bytes(base, b->T, 4));
  b->ws_bytes = b->pipe_part + hier_bytes(hs, 4);
  for (int l = 1; l <= hs.nlev; l++) {
    std::vector<int32_t> map((size_t)hs.nunits[l]);
    b->lev_host[l].resize(n);
    int64_t ub = 0;
    for (int k = 0; k < n; k++) {
      DemDesc d = make_desc(H[k], W[k], hs.S[l]);
      d.ldz = d.lddir = d.ldA = W[k];
      d.tile_base = ub;
      for (int64_t u = 0; u < d.ntx * d.nty; u++) map[(size_t)(ub + u)] = k;
      ub += d.ntx * d.nty;
      b->lev_host[l][k] = d;
    }
    if (cudaMalloc(&b->lev_desc[l], sizeof(DemDesc) * n) != cudaSuccess ||
        cudaMalloc(&b->lev_map[l], sizeof(int32_t) * map.size()) != cudaSuccess ||
        cudaMemcpy(b->lev_map[l], map.data(), sizeof(int32_t) * map.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      d8_batch_destroy(b);
      return D8_ERR_NOMEM;
    }
  }
  if (cudaMalloc(&b->dev_desc, sizeof(DemDesc) * n) != cudaSuccess ||
      cudaMalloc(&b->dev_tile_dem, sizeof(int32_t) * (size_t)base) != cudaSuccess ||
      cudaMalloc(&b->ws, b->ws_bytes) != cudaSuccess) {
    cudaGetLastError();
    d8_batch_destroy(b);
    return D8_ERR_NOMEM;
  }
  if (cudaMemcpy(b->dev_tile_dem, tile_dem.data(), sizeof(int32_t) * (size_t)base, cudaMemcpyHostToDevice) !=
      cudaSuccess) {
    d8_batch_destroy(b);
    return D8_ERR_CUDA;
  }
  *out = b;
  return D8_OK;
}

static cudaError_t batch_enqueue(d8_batch* b, int rule, cudaStream_t s, int* n_up, int* n_comb, int* n_down) {
  DemTable dt{};
  dt.table = b->dev_desc;
  dt.tile_dem = b->dev_tile_dem;
  dt.ndem = b->n;
  dt.one = b->host_desc[0];
  if (b->n == 1) dt.ndem = 1;
  Pipe p = carve_pipe(b->ws, b->ntiles, b->T, 4, b->ctx->status);
  p.strat = b->strat;
  HShape hs;
  hs.nlev = b->nlev;
  hs.need_top = b->need_top;
  DemTable dts[HMAX + 1];
  dts[0] = dt;
  for (int l = 0; l <= b->nlev; l++) {
    hs.S[l] = b->lev_S[l];
    hs.nunits[l] = b->lev_units[l];
    if (l == 0) continue;
    DemTable t{};
    t.ndem = b->n;
    t.one = b->lev_host[l][0];
    t.table = b->lev_desc[l];
    t.tile_dem = b->lev_map[l];
    if (b->n == 1) t.ndem = 1;
    dts[l] = t;
  }
  const HPlan hp = carve_hier(static_cast<char*>(b->ws) + b->pipe_part, hs, p, dts, false);
  cudaError_t e = cudaMemsetAsync(p.queue, 0, sizeof(uint32_t) * 16, s);
  if (e == cudaSuccess) e = launch_up(dt, p, UP_UNIT_Z, rule, s, n_up);
  if (e == cudaSuccess) e = launch_combine_hier(hp, s, n_comb);
  if (e == cudaSuccess) e = launch_down(dt, p, false, s, n_down);
  return e;
}

d8_status d8_batch_flowdir_accumulate(d8_batch* b, const float* const* z, uint8_t* const* dir, uint32_t* const* A,
                                      d8_rule rule, d8_stream stream) {
  if (!b || !z || !dir || !A || (rule < 0 || rule > 3)) return D8_ERR_ARG;
  d8_ctx* c = b->ctx;
  cudaSetDevice(c->device);
  for (int k = 0; k < b->n; k++) {
    if (!z[k] || !dir[k] || !A[k]) return D8_ERR_ARG;
    b->host_desc[k].z = z[k];
    b->host_desc[k].dir = dir[k];
    b->host_desc[k].A = A[k];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the descriptor table is read by the kernels at run time, so new buffer
  // pointers need no re-capture: upload it ahead of the graph on the stream
  cudaError_t e = cudaMemcpyAsync(b->dev_desc, b->host_desc.data(), sizeof(DemDesc) * b->n, cudaMemcpyHostToDevice, s);
  for (int l = 1; l <= b->nlev && e == cudaSuccess; l++) {
    for (int k = 0; k < b->n; k++) {
      b->lev_host[l][k].z = z[k];
      b->lev_host[l][k].dir = dir[k];
      b->lev_host[l][k].A = A[k];
    }
    e = cudaMemcpyAsync(b->lev_desc[l], b->lev_host[l].data(), sizeof(DemDesc) * b->n, cudaMemcpyHostToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  if (b->n == 1 || !b->exec || b->graph_rule != (int)rule) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (b->graph) {
      cudaGraphDestroy(b->graph);
      b->graph = nullptr;
    }
    if (b->n == 1) {
      // a single DEM passes its descriptor by value: run it directly
      int nu = 0, nc = 0, nd = 0;
      StageScope su(c, ST_UP, s);
      e = batch_enqueue(b, (int)rule, s, &nu, &nc, &nd);
      su.n = nu + nc + nd;
      return cuda_fail(e);
    }
    cudaStream_t cap = s;
    bool own = false;
    if (cap == nullptr || cap == cudaStreamLegacy || cap == cudaStreamPerThread) {
      if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return D8_ERR_CUDA;
      own = true;
    }
    int nu = 0, nc = 0, nd = 0;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t e2 = batch_enqueue(b, (int)rule, cap, &nu, &nc, &nd);
      e = cudaStreamEndCapture(cap, &b->graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (own) cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return D8_ERR_CUDA;
    }
    b->graph_rule = (int)rule;
    b->launches_per_run = nu + nc + nd;
  }
  StageScope sc(c, ST_UP, s);
  sc.n = b->launches_per_run;
  return cuda_fail(cudaGraphLaunch(b->exec, s));
}

d8_status d8_batch_destroy(d8_batch* b) {
  if (!b) return D8_OK;
  cudaSetDevice(b->ctx->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->dev_desc) cudaFree(b->dev_desc);
  if (b->dev_tile_dem) cudaFree(b->dev_tile_dem);
  if (b->ws) cudaFree(b->ws);
  for (int l = 0; l <= HMAX; l++) {
    if (b->lev_desc[l]) cudaFree(b->lev_desc[l]);
    if (b->lev_map[l]) cudaFree(b->lev_map[l]);
  }
  delete b;
  return D8_OK;
}

// Autotuner for batches: the tile side sets how the paper's partitions map
// onto the GPU (shared memory per tile, tiles per SM, perimeter share, combine
// depth) and the frontier strategy how the chains of the flow forest are
// traversed; the best pair depends on the mix of DEM sizes and on how far
// their channels wind across tiles, so it is measured.  Each point: one run
// that captures the graph and warms the caches, then AT_REPS replays timed one
// by one; the point's time is their median.
d8_status d8_batch_autotune(d8_ctx* c, int n, const int64_t* H, const int64_t* W, const float* const* z,
                            uint8_t* const* dir, uint32_t* const* A, d8_rule rule, d8_stream stream, int* best_tile,
                            int* best_strategy, float* ms) {
  if (!c || !best_tile || n < 1 || !H || !W || !z || !dir || !A || (rule < 0 || rule > 3)) return D8_ERR_ARG;
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  static const int kTiles[3] = {32, 64, 128};
  constexpr int AT_REPS = 5;
  const int old_T = c->T, old_S = c->strat;
  int best = -1, best_st = 0;
  float best_ms = 0.0f;
  d8_status first_err = D8_OK;
  cudaEvent_t ev[AT_REPS + 1] = {};
  for (auto& e : ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      for (auto& f : ev)
        if (f) cudaEventDestroy(f);
      cudaGetLastError();
      return D8_ERR_CUDA;
    }
  }
  for (int k = 0; k < 3; k++) {
    for (int st = 0; st < STRAT_COUNT; st++) {
      const int pt = k * STRAT_COUNT + st;
      if (ms) ms[pt] = -1.0f;
      c->T = kTiles[k];
      c->strat = st;
      d8_batch* b = nullptr;
      d8_status r = d8_batch_plan(c, n, H, W, &b);
      if (r == D8_OK) r = d8_batch_flowdir_accumulate(b, z, dir, A, rule, stream);
      if (r == D8_OK && cudaEventRecord(ev[0], s) != cudaSuccess) r = D8_ERR_CUDA;
      for (int q = 0; q < AT_REPS && r == D8_OK; q++) {
        r = d8_batch_flowdir_accumulate(b, z, dir, A, rule, stream);
        if (r == D8_OK && cudaEventRecord(ev[q + 1], s) != cudaSuccess) r = D8_ERR_CUDA;
      }
      if (r == D8_OK && cudaEventSynchronize(ev[AT_REPS]) != cudaSuccess) r = D8_ERR_CUDA;
      float t[AT_REPS] = {};
      for (int q = 0; q < AT_REPS && r == D8_OK; q++)
        if (cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]) != cudaSuccess) r = D8_ERR_CUDA;
      if (b) d8_batch_destroy(b);
      if (r != D8_OK) {
        if (first_err == D8_OK) first_err = r;
        cudaGetLastError();
        continue;
      }
      for (int i = 1; i < AT_REPS; i++)  // median of the replays
        for (int j = i; j > 0 && t[j] < t[j - 1]; j--) {
          const float x = t[j];
          t[j] = t[j - 1];
          t[j - 1] = x;
        }
      const float med = t[AT_REPS / 2];
      if (ms) ms[pt] = med;
      if (best < 0 || med < best_ms) {
        best = kTiles[k];
        best_st = st;
        best_ms = med;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (best < 0) {
    c->T = old_T;
    c->strat = old_S;
    return first_err == D8_OK ? D8_ERR_CUDA : first_err;
  }
  c->T = best;
  c->strat = best_st;
  *best_tile = best;
  if (best_strategy) *best_strategy = best_st;
  return D8_OK;
}

}  // extern "C"
