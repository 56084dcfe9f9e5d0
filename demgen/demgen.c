/*
 * demgen.c -- seeded synthetic digital elevation models (DEMs) and direction
 * fields used as INPUTS by the tests, the benchmark and the CPU oracle.
 *
 * This module holds none of the D8 up-slope-area arithmetic: it never picks a
 * flow direction from elevations and never accumulates area.  It only makes
 * elevations (diamond-square fractal, tilted plane, serpentine channel) and
 * removes pits and flats with an epsilon priority-flood, which is the
 * preprocessing the method assumes has already happened ("The Algorithm",
 * first paragraph: pits and flats are removed before flow directions are
 * taken).  The one direction field it writes (the serpentine) is a fixed
 * geometric pattern, not derived from elevations.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood 2014) used as a
 * counter-based generator: the n-th value for seed s is mix(s + (n+1)*gamma),
 * which is exactly the n-th output of a SplitMix64 stream started at s.  Every
 * lattice point draws from its own counter, so the loops may run in parallel
 * and the output does not depend on the thread count.
 *
 * Pit filling: Priority-Flood+epsilon (Barnes, Lehman, Mulla 2014,
 * "Priority-flood: an optimal depression-filling and watershed-labeling
 * algorithm", Algorithm 3) with a monotone radix heap as the priority queue
 * and a FIFO for raised cells; a raised cell becomes max(parent + eps,
 * nextafterf(parent)) in fp32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define SM_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* n-th output of a SplitMix64 stream seeded with `seed`, as a double in [0,1). */
static inline double sm_uniform(uint64_t seed, uint64_t n) {
  return (double)(sm_mix(seed + (n + 1) * SM_GAMMA) >> 11) * 0x1.0p-53;
}

/* Uniform in [-1, 1). */
static inline double sm_sym(uint64_t seed, uint64_t n) { return 2.0 * sm_uniform(seed, n) - 1.0; }

/* Exposed for the Python side's test of the generator itself. */
uint64_t demgen_splitmix64_at(uint64_t seed, uint64_t n) { return sm_mix(seed + (n + 1) * SM_GAMMA); }

/* ------------------------------------------------------------------------ */
/* Diamond-square on a lattice of (by x bx) squares of side s = 2^k, cropped. */

int demgen_fractal(float* z, int64_t H, int64_t W, uint64_t seed, double rough, double relief) {
  if (H < 1 || W < 1 || !z) return 1;
  int64_t mn = H < W ? H : W;
  int64_t s = 1;
  while (2 * s <= mn - 1) s *= 2;           /* largest power of two <= min(H,W)-1 */
  int64_t bx = (W - 1 + s - 1) / s, by = (H - 1 + s - 1) / s;
  if (bx < 1) bx = 1;
  if (by < 1) by = 1;
  int64_t LH = by * s + 1, LW = bx * s + 1;
  double* L = (double*)malloc(sizeof(double) * (size_t)(LH * LW));
  if (!L) return 2;
  /* coarse corners */
  double amp = 1.0;
  for (int64_t i = 0; i < LH; i += s)
    for (int64_t j = 0; j < LW; j += s) L[i * LW + j] = amp * sm_sym(seed, (uint64_t)(i * LW + j));
  const double decay = pow(2.0, -rough);
  for (int64_t step = s; step > 1; step /= 2) {
    int64_t half = step / 2;
    amp *= decay;
    /* square step: centre of each square from its four corners */
#pragma omp parallel for schedule(static)
    for (int64_t i = half; i < LH; i += step)
      for (int64_t j = half; j < LW; j += step) {
        double a = L[(i - half) * LW + (j - half)] + L[(i - half) * LW + (j + half)] +
                   L[(i + half) * LW + (j - half)] + L[(i + half) * LW + (j + half)];
        L[i * LW + j] = 0.25 * a + amp * sm_sym(seed, (uint64_t)(i * LW + j));
      }
    /* diamond step: edge midpoints from the (up to four) points at distance half */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < LH; i += half) {
      int64_t j0 = ((i / half) % 2 == 0) ? half : 0;
      for (int64_t j = j0; j < LW; j += step) {
        double a = 0.0;
        int cnt = 0;
        if (i - half >= 0) { a += L[(i - half) * LW + j]; cnt++; }
        if (i + half < LH) { a += L[(i + half) * LW + j]; cnt++; }
        if (j - half >= 0) { a += L[i * LW + (j - half)]; cnt++; }
        if (j + half < LW) { a += L[i * LW + (j + half)]; cnt++; }
        L[i * LW + j] = a / cnt + amp * sm_sym(seed, (uint64_t)(i * LW + j));
      }
    }
  }
  /* crop to H x W and rescale linearly to [0, relief] in double, then store fp32 */
  double lo = INFINITY, hi = -INFINITY;
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) {
      double v = L[i * LW + j];
      if (v < lo) lo = v;
      if (v > hi) hi = v;
    }
  double scale = (hi > lo) ? relief / (hi - lo) : 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) z[i * W + j] = (float)((L[i * LW + j] - lo) * scale);
  free(L);
  return 0;
}

/* Tilted plane z = sy*(H-1-i) + sx*(W-1-j) + noise + U(-noise, noise) (the
 * offset keeps every elevation >= 0, as the fill requires). */
int demgen_plane(float* z, int64_t H, int64_t W, uint64_t seed, double sy, double sx, double noise) {
  if (H < 1 || W < 1 || !z) return 1;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++)
      z[i * W + j] = (float)(sy * (double)(H - 1 - i) + sx * (double)(W - 1 - j) + noise +
                             noise * sm_sym(seed, (uint64_t)(i * W + j)));
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Monotone radix heap over (uint32 key, uint32 index), keys = fp32 bit patterns
 * of non-negative floats (monotone in the float order). */

typedef struct {
  uint64_t* a;
  size_t n, cap;
} vec64;

static int vpush(vec64* v, uint64_t x) {
  if (v->n == v->cap) {
    size_t nc = v->cap ? v->cap * 2 : 1024;
    uint64_t* na = (uint64_t*)realloc(v->a, nc * sizeof(uint64_t));
    if (!na) return 1;
    v->a = na;
    v->cap = nc;
  }
  v->a[v->n++] = x;
  return 0;
}

typedef struct {
  vec64 b[33];
  uint32_t last;
  size_t size;
} radix_heap;

static inline int rh_bucket(uint32_t key, uint32_t last) {
  uint32_t x = key ^ last;
  return x == 0 ? 0 : 32 - __builtin_clz(x);
}

static int rh_push(radix_heap* h, uint32_t key, uint32_t idx) {
  h->size++;
  return vpush(&h->b[rh_bucket(key, h->last)], ((uint64_t)key << 32) | idx);
}

static uint64_t rh_pop(radix_heap* h) {
  if (h->b[0].n == 0) {
    int i = 1;
    while (h->b[i].n == 0) i++;
    uint32_t mn = 0xFFFFFFFFu;
    for (size_t k = 0; k < h->b[i].n; k++) {
      uint32_t key = (uint32_t)(h->b[i].a[k] >> 32);
      if (key < mn) mn = key;
    }
    h->last = mn;
    for (size_t k = 0; k < h->b[i].n; k++) {
      uint64_t e = h->b[i].a[k];
      vpush(&h->b[rh_bucket((uint32_t)(e >> 32), mn)], e);
    }
    h->b[i].n = 0;
  }
  h->size--;
  return h->b[0].a[--h->b[0].n];
}

static inline uint32_t fkey(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

static inline float raise_above(float parent, float eps) {
  float r = parent + eps;
  float nx = nextafterf(parent, INFINITY);
  return r > nx ? r : nx;
}

/* Priority-Flood+epsilon.  Border cells seed the flood; every interior cell
 * that is not strictly above the cell it is reached from is raised above it.
 * Afterwards every interior cell has a strictly lower 8-neighbour (the cell it
 * was reached from).  Elevations must be finite and >= 0.  Works on a copy
 * padded with a one-cell frame; a cell is "closed" once its sign bit is set
 * (all elevations are >= 0), so one array serves as both elevation and
 * closed flag and the neighbour loop needs no bounds checks. */
int demgen_eps_fill(float* z, int64_t H, int64_t W, float eps) {
  if (H < 1 || W < 1 || !z) return 1;
  int64_t N = H * W;
  int64_t PW = W + 2, PH = H + 2, PN = PH * PW;
  if (PN > 0xFFFFFFFFLL) return 1;
  for (int64_t c = 0; c < N; c++)
    if (!(z[c] >= 0.0f) || isinf(z[c])) return 3;
  float* pz = (float*)malloc(sizeof(float) * (size_t)PN);
  uint32_t* pit = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)N);
  if (!pz || !pit) {
    free(pz);
    free(pit);
    return 2;
  }
  for (int64_t j = 0; j < PW; j++) {
    pz[j] = -1.0f;
    pz[(PH - 1) * PW + j] = -1.0f;
  }
  for (int64_t i = 0; i < PH; i++) {
    pz[i * PW] = -1.0f;
    pz[i * PW + PW - 1] = -1.0f;
  }
  for (int64_t i = 0; i < H; i++) memcpy(pz + (i + 1) * PW + 1, z + i * W, sizeof(float) * (size_t)W);
  radix_heap h;
  memset(&h, 0, sizeof(h));
  for (int b = 0; b < 33; b++) {
    h.b[b].cap = 1 << 16;
    h.b[b].a = (uint64_t*)malloc(sizeof(uint64_t) * h.b[b].cap);
  }
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++)
      if (i == 0 || j == 0 || i == H - 1 || j == W - 1) {
        int64_t c = (i + 1) * PW + (j + 1);
        rh_push(&h, fkey(pz[c]), (uint32_t)c);
        pz[c] = -pz[c];
      }
  const int64_t off[8] = {-PW, -PW + 1, 1, PW + 1, PW, PW - 1, -1, -PW - 1};
  size_t ph = 0, pt = 0; /* FIFO of raised cells */
  while (ph < pt || h.size > 0) {
    int64_t c;
    float zc;
    if (ph < pt) {
      c = pit[ph++];
      zc = -pz[c];
    } else {
      uint64_t e = rh_pop(&h);
      c = (int64_t)(uint32_t)e;
      uint32_t kb = (uint32_t)(e >> 32);
      memcpy(&zc, &kb, 4);
    }
    for (int k = 0; k < 8; k++) {
      int64_t n = c + off[k];
      float zn = pz[n];
      if (signbit(zn)) continue;
      if (zn <= zc) {
        pz[n] = -raise_above(zc, eps);
        pit[pt++] = (uint32_t)n;
      } else {
        pz[n] = -zn;
        rh_push(&h, fkey(zn), (uint32_t)n);
      }
    }
  }
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) z[i * W + j] = -pz[(i + 1) * PW + 1 + j];
  for (int b = 0; b < 33; b++) free(h.b[b].a);
  free(pz);
  free(pit);
  return 0;
}

/* Number of interior cells with no strictly lower 8-neighbour (0 means every
 * interior cell can drain; used as the generator's post-condition). */
int64_t demgen_count_undrained(const float* z, int64_t H, int64_t W) {
  int64_t bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(static)
  for (int64_t i = 1; i < H - 1; i++)
    for (int64_t j = 1; j < W - 1; j++) {
      float zc = z[i * W + j];
      int ok = 0;
      for (int a = -1; a <= 1 && !ok; a++)
        for (int b = -1; b <= 1; b++)
          if ((a || b) && z[(i + a) * W + (j + b)] < zc) {
            ok = 1;
            break;
          }
      bad += !ok;
    }
  return bad;
}

/* ------------------------------------------------------------------------ */
/* Serpentine direction field: boustrophedon over the whole grid.  Codes use the
 * library's numbering 0..7 = N,NE,E,SE,S,SW,W,NW.  Even rows run east, odd rows
 * west, the row end steps south, and the last cell points south off the grid,
 * so every cell lies on one path of length H*W. */
int demgen_serpentine_dirs(uint8_t* dir, int64_t H, int64_t W) {
  if (H < 1 || W < 1 || !dir) return 1;
  const uint8_t E = 2, S = 4, Wd = 6;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) {
      uint8_t d;
      if (i % 2 == 0)
        d = (j == W - 1) ? S : E;
      else
        d = (j == 0) ? S : Wd;
      dir[i * W + j] = d;
    }
  return 0;
}

/* Serpentine DEM: one-cell-wide channels on odd rows separated by one-cell-wide
 * ridges on even rows, joined by a gap in the ridge at alternate ends; the grid
 * border sits above every interior cell except one low outlet at the end of
 * the last channel.  Channel elevations strictly decrease along the channel
 * (consecutive fp32 bit patterns), so a steepest or lowest D8 rule follows the
 * channel.  Needs H >= 5 and W >= 4. */
int demgen_serpentine_dem(float* z, int64_t H, int64_t W) {
  if (H < 5 || W < 4 || !z) return 1;
  const float top = 3.0e6f;   /* channels start just below this */
  const float ridge = 4.0e6f; /* above every channel cell */
  const float border = 5.0e6f;
  for (int64_t c = 0; c < H * W; c++) z[c] = ridge;
  for (int64_t i = 0; i < H; i++) {
    z[i * W + 0] = border;
    z[i * W + W - 1] = border;
  }
  for (int64_t j = 0; j < W; j++) {
    z[0 * W + j] = border;
    z[(H - 1) * W + j] = border;
  }
  uint32_t bits;
  memcpy(&bits, &top, 4);
  int64_t last_row = -1, last_col = -1;
  int east = 1;
  for (int64_t r = 1; r <= H - 2; r += 2) {
    if (r > 1) {
      /* gap cell in the ridge row above this channel, at the column where the
         previous channel ended */
      int64_t gc = east ? 1 : W - 2;
      float v;
      memcpy(&v, &bits, 4);
      z[(r - 1) * W + gc] = v;
      bits--;
    }
    for (int64_t k = 0; k < W - 2; k++) {
      int64_t j = east ? 1 + k : W - 2 - k;
      float v;
      memcpy(&v, &bits, 4);
      z[r * W + j] = v;
      bits--;
      last_row = r;
      last_col = j;
    }
    east = !east;
  }
  /* the outlet: a border cell next to the end of the last channel */
  if (last_row == H - 2)
    z[(H - 1) * W + last_col] = 0.0f;
  else
    z[last_row * W + (last_col == 1 ? 0 : W - 1)] = 0.0f;
  return 0;
}
