/*
 * d8_cpuref.c -- MULTI-CORE CPU REFERENCE for D8 flow directions and
 * up-slope counts: the CPU baseline the benchmark reports beside the GPU.
 *
 * MEASUREMENT INFRASTRUCTURE ONLY.  The benchmark's CPU-baseline leg and the
 * tests (which check it against the oracle) are its only callers; the CUDA
 * library never calls it and shares no code with it.
 *
 * Method (Barnes, Lehman, Mulla, PDPTA 2011):
 *   - directions: the rule of "The Algorithm" (steepest slope, slope = drop /
 *     distance between cell centres; the diagonal distance factor is the fp32
 *     value nearest 1/sqrt(2), one rounded multiply, no contraction) or of
 *     the "Introduction" (lowest neighbour); ties to the first of N, NE, E,
 *     SE, S, SW, W, NW; edge cells OUTLET (8), no strictly lower neighbour
 *     SINK (9).  Rows are split over the OpenMP threads.
 *   - counts: Algorithm 1 (FindDependencies) and Algorithm 2
 *     (InternalUpslope) in the shared-memory form the paper describes, with
 *     one queue per thread so that the threads do not contend for a queue:
 *     the input counts are made with atomic increments, each thread queues
 *     the cells without inputs in its share of the rows, and a thread that
 *     pops a cell adds the cell's count into its down-slope cell (atomic),
 *     then decrements that cell's input count; the thread that brings it to
 *     zero queues it on its own queue.  The release/acquire pair on the count
 *     makes every addition visible to that thread.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CR_OK = 0, CR_ERR_ARG = 1, CR_ERR_NONFINITE = 3, CR_ERR_CYCLE = 4, CR_ERR_NOMEM = 5 };

static const int CDI[8] = {-1, -1, 0, 1, 1, 1, 0, -1};
static const int CDJ[8] = {0, 1, 1, 1, 0, -1, -1, -1};

static float inv_sqrt2_f32(void) {
  uint32_t b = 0x3F3504F3u;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

static int finite_f32(float x) { return x - x == 0.0f; }

int cpuref_flowdir(const float* z, int64_t H, int64_t W, int rule, int nthreads, uint8_t* dir) {
  if (!z || !dir || H < 1 || W < 1 || (rule != 0 && rule != 1)) return CR_ERR_ARG;
  const float R = inv_sqrt2_f32();
  int nonfinite = 0;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : nonfinite)
  for (int64_t i = 0; i < H; i++) {
    for (int64_t j = 0; j < W; j++) {
      const float zc = z[i * W + j];
      if (!finite_f32(zc)) nonfinite = 1;
      if (i == 0 || j == 0 || i == H - 1 || j == W - 1) {
        dir[i * W + j] = 8;
        continue;
      }
      if (!finite_f32(zc)) {
        dir[i * W + j] = 9;
        continue;
      }
      int best_k = 9;
      float best = rule == 0 ? 0.0f : zc;
      for (int k = 0; k < 8; k++) {
        const float zn = z[(i + CDI[k]) * W + (j + CDJ[k])];
        if (rule == 0) {
          float s = zc - zn;
          if (k & 1) s = s * R;
          if (s > best) {
            best = s;
            best_k = k;
          }
        } else if (zn < best) {
          best = zn;
          best_k = k;
        }
      }
      dir[i * W + j] = (uint8_t)best_k;
    }
  }
  return nonfinite ? CR_ERR_NONFINITE : CR_OK;
}

/* down-slope cell of c, or -1 (OUTLET, SINK, a target off the grid); *bad
 * set for codes above 9 */
static int64_t target(const uint8_t* dir, int64_t H, int64_t W, int64_t c, int* bad) {
  const int k = dir[c];
  if (k > 9) {
    *bad = 1;
    return -1;
  }
  if (k >= 8) return -1;
  const int64_t i = c / W + CDI[k], j = c % W + CDJ[k];
  if (i < 0 || j < 0 || i >= H || j >= W) return -1;
  return i * W + j;
}

int cpuref_accumulate(const uint8_t* dir, int64_t H, int64_t W, int nthreads, uint32_t* A) {
  if (!dir || !A || H < 1 || W < 1 || nthreads < 1) return CR_ERR_ARG;
  const int64_t n = H * W;
  uint8_t* D = (uint8_t*)calloc((size_t)n, 1);
  if (!D) return CR_ERR_NOMEM;
  int bad = 0;
  int64_t done = 0;
  int nomem = 0;
  /* Algorithm 1: input counts */
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : bad)
  for (int64_t c = 0; c < n; c++) {
    A[c] = 1u;
    const int64_t t = target(dir, H, W, c, &bad);
    if (t >= 0) __atomic_fetch_add(&D[t], (uint8_t)1, __ATOMIC_RELAXED);
  }
  /* Algorithm 2: per-thread queues */
#pragma omp parallel num_threads(nthreads) reduction(+ : done) reduction(| : nomem)
  {
    const int nt = omp_get_num_threads(), me = omp_get_thread_num();
    const int64_t r0 = H * me / nt, r1 = H * (me + 1) / nt;
    int64_t cap = 1024, head = 0, tail = 0;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
    if (!q) nomem = 1;
    int dummy = 0;
    for (int64_t c = r0 * W; q && c < r1 * W; c++) {
      if (__atomic_load_n(&D[c], __ATOMIC_RELAXED) != 0) continue;
      if (tail == cap) {
        int64_t* q2 = (int64_t*)realloc(q, sizeof(int64_t) * (size_t)(cap * 2));
        if (!q2) {
          nomem = 1;
          break;
        }
        q = q2;
        cap *= 2;
      }
      q[tail++] = c;
    }
    /* every thread's sources are listed before any count changes */
#pragma omp barrier
    while (q && !nomem && head < tail) {
      int64_t c = q[head++];
      /* the cell's own chain continues on this thread while it brings the
         next cell's input count to zero (Algorithm 2's tail recursion) */
      for (;;) {
        done++;
        const int64_t t = target(dir, H, W, c, &dummy);
        if (t < 0) break;
        const uint32_t a = __atomic_load_n(&A[c], __ATOMIC_RELAXED);
        __atomic_fetch_add(&A[t], a, __ATOMIC_RELAXED);
        if (__atomic_sub_fetch(&D[t], (uint8_t)1, __ATOMIC_ACQ_REL) != 0) break;
        c = t;
      }
    }
    free(q);
  }
  free(D);
  if (nomem) return CR_ERR_NOMEM;
  if (bad) return CR_ERR_ARG;
  return done == n ? CR_OK : CR_ERR_CYCLE;
}
