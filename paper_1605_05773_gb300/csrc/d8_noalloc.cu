// d8_noalloc.cu -- directions + unit up-slope counts without any allocation.
//
// Some callers cannot allocate device memory at the time they need the
// result: code running inside a fixed memory budget (an embedded or real-time
// process that reserved all its memory up front), callers holding a pool or
// arena allocator that owns every byte of the device, and callers that cannot
// create a library context because d8_create itself allocates.  For them,
// d8_flowdir_accumulate_noalloc runs the same pipeline as
// d8_flowdir_accumulate (same kernels, same results) but takes its scratch --
// the per-tile perimeter summaries, the combine's arrays and counters -- from
// the fixed array below, which is part of the library image and is placed on
// a device when the library's code is loaded there.  It never calls
// cudaMalloc, cudaFree or any allocating routine.
//
// The paper has no counterpart: this is an interface for callers, not a step
// of the method.
#include <mutex>

#include "d8.h"
#include "d8_internal.h"

namespace {

constexpr int NA_TILE = 64;
constexpr size_t NA_SCRATCH_BYTES = (size_t)64 << 20;  // 64 MiB per device
constexpr int NA_MAX_DEVICES = 64;

// The scratch.  Every device that loads the library holds these 64 MiB until
// the process exits.  All calls share it: it keeps whatever the last call
// left there, and calls whose GPU work overlaps in time (different streams,
// different host threads, no ordering between them) race on it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_SCRATCH_BYTES];

void* g_dev_ptr[NA_MAX_DEVICES] = {};
std::mutex g_mu;

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int bits(uint64_t x) {
  int r = 0;
  while (x) {
    r++;
    x >>= 1;
  }
  return r;
}

// Scratch layout: [status word, 256 B] [pipeline arrays for ntiles tiles]
size_t needed_bytes(int64_t ntiles) {
  const size_t ns = (size_t)ntiles * 4 * NA_TILE;
  return 256 + a256(ns * 2) + a256(ns * 4) + 2 * a256(ns * 4) + 2 * a256(ns * 4) +
         a256(sizeof(uint32_t) * (d8::MAX_ROUNDS + 2)) + a256(sizeof(uint32_t) * 16);
}

// Device address of the scratch for the current device.  The host-side name
// of a __device__ array is only a stand-in for it, so the address must come
// from cudaGetSymbolAddress, once per device with that device current.
d8_status scratch_ptr(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    cudaGetLastError();
    return D8_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return D8_ERR_CUDA;
    }
    g_dev_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_dev_ptr[dev]);
  return D8_OK;
}

d8_status cuda_rc(cudaError_t e) { return e == cudaSuccess ? D8_OK : D8_ERR_CUDA; }

}  // namespace

extern "C" d8_status d8_flowdir_accumulate_noalloc(const float* z, int64_t H, int64_t W, int64_t ldz, d8_rule rule,
                                                   uint8_t* dir, int64_t lddir, uint32_t* A, int64_t ldA,
                                                   uint32_t* status, d8_stream stream) {
  if (!z || !dir || !A || H < 1 || W < 1 || ldz < W || lddir < W || ldA < W || (rule < 0 || rule > 3))
    return D8_ERR_ARG;
  if ((uint64_t)H * (uint64_t)W > 0xFFFFFFFFull) return D8_ERR_SHAPE;
  d8::DemDesc d{};
  d.z = z;
  d.ldz = ldz;
  d.dir = dir;
  d.lddir = lddir;
  d.A = A;
  d.ldA = ldA;
  d.H = H;
  d.W = W;
  d.ntx = (W + NA_TILE - 1) / NA_TILE;
  d.nty = (H + NA_TILE - 1) / NA_TILE;
  d.tile_base = 0;
  const int64_t ntiles = d.ntx * d.nty;
  if (needed_bytes(ntiles) > NA_SCRATCH_BYTES) return D8_ERR_CAPACITY;
  unsigned char* base = nullptr;
  d8_status st = scratch_ptr(&base);
  if (st != D8_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // carve the pipeline arrays out of the scratch
  d8::Pipe p{};
  p.T = NA_TILE;
  p.strat = d8::STRAT_RING;
  p.ntiles = ntiles;
  p.nslots = ntiles * 4 * NA_TILE;
  p.rounds = bits((uint64_t)p.nslots);
  if (p.rounds > d8::MAX_ROUNDS) p.rounds = d8::MAX_ROUNDS;
  const size_t ns = (size_t)p.nslots;
  unsigned char* q = base + 256;
  p.pex = reinterpret_cast<uint16_t*>(q);
  q += a256(ns * 2);
  p.pval = q;
  q += a256(ns * 4);
  p.P[0] = reinterpret_cast<uint32_t*>(q);
  q += a256(ns * 4);
  p.P[1] = reinterpret_cast<uint32_t*>(q);
  q += a256(ns * 4);
  p.S = q;
  q += a256(ns * 4);
  p.S2 = q;
  q += a256(ns * 4);
  p.flags = reinterpret_cast<uint32_t*>(q);
  q += a256(sizeof(uint32_t) * (d8::MAX_ROUNDS + 2));
  p.queue = reinterpret_cast<uint32_t*>(q);
  p.status = status ? status : reinterpret_cast<uint32_t*>(base);

  // what must start at zero: the status word, the tile work-queue counters
  // (the combine clears its own round flags and delta array)
  cudaError_t e = cudaMemsetAsync(p.status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p.queue, 0, sizeof(uint32_t) * 16, s);
  if (e != cudaSuccess) return cuda_rc(e);
  d8::DemTable dt{};
  dt.one = d;
  dt.ndem = 1;
  int n = 0;
  e = d8::launch_up(dt, p, d8::UP_UNIT_Z, (int)rule, s, &n);
  if (e == cudaSuccess) e = d8::launch_combine_flat(dt, p, s, &n);
  if (e == cudaSuccess) e = d8::launch_down(dt, p, false, s, &n);
  return cuda_rc(e);
}
