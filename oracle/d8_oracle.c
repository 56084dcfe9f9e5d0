/*
 * d8_oracle.c -- CPU ORACLE for D8 flow directions and up-slope area.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference leg may load or run this code.  The
 * product (the CUDA library and its Python binding) never calls it, includes
 * it or shares any code, header or table with it.
 *
 * Plain, sequential, obviously-correct code.  Sources (Barnes, Lehman, Mulla,
 * "Distributed Parallel D8 Up-Slope Area Calculation in Digital Elevation
 * Models", PDPTA 2011):
 *   - Eq. 1 (section "Up-Slope Area"): A(p) = 1 + sum of A(i) over the cells i
 *     whose flow enters p; cells may carry a weight other than one, giving
 *     A(p) = w(p) + sum A(i).
 *   - D8 flow direction ("Introduction" and "The Algorithm"): all of a cell's
 *     flow goes to ONE neighbour, the lowest neighbour (Introduction) or the
 *     neighbour of steepest slope, slope = drop / Euclidean distance between
 *     cell centres ("The Algorithm").  Both rules are provided.
 *   - Algorithm 1 (FindDependencies) and Algorithm 2 (InternalUpslope): count
 *     each cell's inputs, queue the cells with none, then pop a cell, set its
 *     area to its weight plus its inputs' areas, decrement its down-slope
 *     neighbour's count and continue down-slope while that count reaches zero.
 *     Run here with ONE worker, so the queue is a plain FIFO.
 *
 * Readings of points the paper leaves open (stated once here, used below):
 *   - direction codes 0..7 = N, NE, E, SE, S, SW, W, NW (row index grows to
 *     the south), 8 = OUTLET (grid edge cell), 9 = SINK (no strictly lower
 *     neighbour);
 *   - every cell in the first/last row or column is an OUTLET: it receives
 *     flow but passes none on (the DEM edge drains off-grid);
 *   - ties: the first direction in N, NE, E, SE, S, SW, W, NW order wins
 *     (strict comparison while scanning in that order);
 *   - only a strictly positive drop counts; none gives SINK;
 *   - steepest slope: cardinal slope = drop, diagonal slope = drop * R with R
 *     the fp32 value nearest 1/sqrt(2), one rounded fp32 multiply, no fused
 *     multiply-add (build with -ffp-contract=off);
 *   - for accumulation over an arbitrary direction field, a code 0..7 whose
 *     target lies off the grid ends the path, 8 and 9 end the path, any
 *     other code is an error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NONFINITE = 3, OR_ERR_CYCLE = 4, OR_ERR_NOMEM = 5, OR_ERR_OVERFLOW = 8 };

/* Neighbour k = 0..7: N, NE, E, SE, S, SW, W, NW. */
static const int ODI[8] = {-1, -1, 0, 1, 1, 1, 0, -1};
static const int ODJ[8] = {0, 1, 1, 1, 0, -1, -1, -1};

/* fp32 nearest to 1/sqrt(2): 0x3F3504F3 = 0.707106769... */
static float oracle_inv_sqrt2(void) {
  uint32_t b = 0x3F3504F3u;
  float f;
  memcpy(&f, &b, 4);
  return f;
}

/* D8 flow direction of every cell ("The Algorithm": steepest slope with the
 * Euclidean distance between centres; "Introduction": lowest neighbour).
 * rule bit 0: 0 = steepest, 1 = lowest.  rule bit 1 (NODATA masks): a cell
 * with a non-finite elevation lies outside the study area and gets OUTLET,
 * and so does every cell next to one (the area's edge drains off it, as the
 * grid's edge does).  Returns OR_OK, or (without the NODATA bit)
 * OR_ERR_NONFINITE if any elevation is NaN or infinite (a non-finite cell
 * itself gets SINK). */
int oracle_flowdir(const float* z, int64_t H, int64_t W, int rule, uint8_t* dir) {
  if (!z || !dir || H < 1 || W < 1 || rule < 0 || rule > 3) return OR_ERR_ARG;
  const int nodata = rule & 2;
  rule &= 1;
  const float R = oracle_inv_sqrt2();
  int nonfinite = 0;
  for (int64_t i = 0; i < H; i++) {
    for (int64_t j = 0; j < W; j++) {
      float zc = z[i * W + j];
      if (!isfinite(zc)) nonfinite = 1;
      if (i == 0 || j == 0 || i == H - 1 || j == W - 1) {
        dir[i * W + j] = 8; /* OUTLET */
        continue;
      }
      if (nodata) {
        int hole = !isfinite(zc);
        for (int k = 0; k < 8; k++) hole |= !isfinite(z[(i + ODI[k]) * W + (j + ODJ[k])]);
        if (hole) {
          dir[i * W + j] = 8; /* outside the study area, or on its edge */
          continue;
        }
      }
      if (!isfinite(zc)) {
        dir[i * W + j] = 9;
        continue;
      }
      int best_k = 9; /* SINK unless a strictly lower neighbour exists */
      if (rule == 0) {
        float best = 0.0f;
        for (int k = 0; k < 8; k++) {
          float zn = z[(i + ODI[k]) * W + (j + ODJ[k])];
          float drop = zc - zn;
          float slope = (k & 1) ? drop * R : drop;
          if (slope > best) {
            best = slope;
            best_k = k;
          }
        }
      } else {
        float best = zc;
        for (int k = 0; k < 8; k++) {
          float zn = z[(i + ODI[k]) * W + (j + ODJ[k])];
          if (zn < best) {
            best = zn;
            best_k = k;
          }
        }
      }
      dir[i * W + j] = (uint8_t)best_k;
    }
  }
  return (nonfinite && !nodata) ? OR_ERR_NONFINITE : OR_OK;
}

/* Down-slope neighbour of cell c, or -1 if its path ends at c; -2 for an
 * invalid code. */
static int64_t succ_of(const uint8_t* dir, int64_t H, int64_t W, int64_t c) {
  int code = dir[c];
  if (code > 9) return -2;
  if (code >= 8) return -1;
  int64_t i = c / W + ODI[code], j = c % W + ODJ[code];
  if (i < 0 || j < 0 || i >= H || j >= W) return -1;
  return i * W + j;
}

/* Algorithm 1 (FindDependencies) + Algorithm 2 (InternalUpslope) with one
 * worker.  Computes A(p) = w(p) + sum over inputs of A (Eq. 1) in fp64 (w ==
 * NULL means unit weights) and, if order != NULL, the order in which cells
 * were finished.  Returns OR_ERR_CYCLE if some cells are never finished
 * (their directions form a cycle), OR_ERR_ARG for an invalid code. */
int oracle_accumulate_f64(const uint8_t* dir, int64_t H, int64_t W, const double* w, double* A, int64_t* order) {
  if (!dir || !A || H < 1 || W < 1) return OR_ERR_ARG;
  int64_t N = H * W;
  for (int64_t c = 0; c < N; c++)
    if (dir[c] > 9) return OR_ERR_ARG;
  uint8_t* D = (uint8_t*)calloc((size_t)N, 1);
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  if (!D || !Q) {
    free(D);
    free(Q);
    return OR_ERR_NOMEM;
  }
  /* Algorithm 1: D(c) = number of neighbours whose flow is directed into c;
     cells with none go on the back of Q. */
  int64_t qt = 0;
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) {
      int64_t c = i * W + j;
      for (int k = 0; k < 8; k++) {
        int64_t ni = i + ODI[k], nj = j + ODJ[k];
        if (ni < 0 || nj < 0 || ni >= H || nj >= W) continue;
        if (succ_of(dir, H, W, ni * W + nj) == c) D[c]++;
      }
      if (D[c] == 0) Q[qt++] = c;
    }
  /* Algorithm 2, one worker: pop the front of Q, then follow the flow path
     while the next cell's dependencies are all satisfied. */
  int64_t qh = 0, done = 0;
  while (qh < qt) {
    int64_t c = Q[qh++];
    for (;;) {
      int64_t ci = c / W, cj = c % W;
      double a = w ? w[c] : 1.0;
      for (int k = 0; k < 8; k++) {
        int64_t ni = ci + ODI[k], nj = cj + ODJ[k];
        if (ni < 0 || nj < 0 || ni >= H || nj >= W) continue;
        int64_t n = ni * W + nj;
        if (succ_of(dir, H, W, n) == c) a += A[n];
      }
      A[c] = a;
      if (order) order[done] = c;
      done++;
      int64_t s = succ_of(dir, H, W, c);
      if (s < 0) break;
      D[s]--;
      if (D[s] != 0) break;
      c = s;
    }
  }
  free(D);
  free(Q);
  return done == N ? OR_OK : OR_ERR_CYCLE;
}

/* Unit-weight counts (Eq. 1 with w = 1) as exact 64-bit integers; the same
 * queue method as above.  Returns OR_ERR_OVERFLOW if a count exceeds
 * 2^32 - 1 (the width of the library's output). */
int oracle_accumulate_u64(const uint8_t* dir, int64_t H, int64_t W, uint64_t* A) {
  if (!dir || !A || H < 1 || W < 1) return OR_ERR_ARG;
  int64_t N = H * W;
  for (int64_t c = 0; c < N; c++)
    if (dir[c] > 9) return OR_ERR_ARG;
  uint8_t* D = (uint8_t*)calloc((size_t)N, 1);
  int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  if (!D || !Q) {
    free(D);
    free(Q);
    return OR_ERR_NOMEM;
  }
  int64_t qt = 0;
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++) {
      int64_t c = i * W + j;
      for (int k = 0; k < 8; k++) {
        int64_t ni = i + ODI[k], nj = j + ODJ[k];
        if (ni < 0 || nj < 0 || ni >= H || nj >= W) continue;
        if (succ_of(dir, H, W, ni * W + nj) == c) D[c]++;
      }
      if (D[c] == 0) Q[qt++] = c;
    }
  int64_t qh = 0, done = 0;
  int overflow = 0;
  while (qh < qt) {
    int64_t c = Q[qh++];
    for (;;) {
      int64_t ci = c / W, cj = c % W;
      uint64_t a = 1;
      for (int k = 0; k < 8; k++) {
        int64_t ni = ci + ODI[k], nj = cj + ODJ[k];
        if (ni < 0 || nj < 0 || ni >= H || nj >= W) continue;
        int64_t n = ni * W + nj;
        if (succ_of(dir, H, W, n) == c) a += A[n];
      }
      A[c] = a;
      if (a > 0xFFFFFFFFull) overflow = 1;
      done++;
      int64_t s = succ_of(dir, H, W, c);
      if (s < 0) break;
      D[s]--;
      if (D[s] != 0) break;
      c = s;
    }
  }
  free(D);
  free(Q);
  if (done != N) return OR_ERR_CYCLE;
  return overflow ? OR_ERR_OVERFLOW : OR_OK;
}

/* Transposed solve (the adjoint of Eq. 1): with L = sum_p c(p) A(p),
 * dL/dw(q) = G(q) = c(q) + G(down-slope neighbour of q), G = 0 past the end
 * of a path.  Evaluated in fp64 by walking the forward finishing order
 * backwards, so every cell's down-slope neighbour is done first. */
int oracle_transposed_f64(const uint8_t* dir, int64_t H, int64_t W, const double* cvec, double* G) {
  if (!dir || !cvec || !G || H < 1 || W < 1) return OR_ERR_ARG;
  int64_t N = H * W;
  double* A = (double*)malloc(sizeof(double) * (size_t)N);
  int64_t* order = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
  if (!A || !order) {
    free(A);
    free(order);
    return OR_ERR_NOMEM;
  }
  int rc = oracle_accumulate_f64(dir, H, W, NULL, A, order);
  if (rc == OR_OK) {
    for (int64_t t = N - 1; t >= 0; t--) {
      int64_t q = order[t];
      int64_t s = succ_of(dir, H, W, q);
      G[q] = cvec[q] + (s >= 0 ? G[s] : 0.0);
    }
  }
  free(A);
  free(order);
  return rc;
}

/* ---- Pit and flat removal (the method's precondition, "The Algorithm",
 * first paragraph: the DEM has had its pits raised or drilled and its flats
 * resolved, so that every interior cell drains).
 *
 * Reading taken: epsilon filling.  The filled surface F is the unique array
 * with F = z on the grid's edge cells and, for every interior cell c, with
 * m = the smallest F among its eight neighbours,
 *     F(c) = z(c)      if z(c) > m,
 *     F(c) = up(m)     otherwise,     up(x) = max(fl32(x + eps), next fp32 above x).
 * Every interior cell of F has a strictly lower neighbour.  The map is
 * monotone and raises strictly, so the array is unique; a priority flood
 * from the edge (cells leave a min-heap in order of F, and a cell first
 * reached from a cell p gets z if z is above F(p), else up(F(p))) meets every
 * cell first from its lowest neighbour and so produces exactly that array.
 * That priority flood is what this function runs: a binary heap ordered by
 * (F, cell index), one worker, fp32 arithmetic, no contraction. */
typedef struct {
  float f;
  int64_t c;
} fill_item;

static int fill_less(fill_item a, fill_item b) { return a.f < b.f || (a.f == b.f && a.c < b.c); }

static void heap_push(fill_item* h, int64_t* n, fill_item x) {
  int64_t i = (*n)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!fill_less(x, h[p])) break;
    h[i] = h[p];
    i = p;
  }
  h[i] = x;
}

static fill_item heap_pop(fill_item* h, int64_t* n) {
  fill_item top = h[0], x = h[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    fill_item best = x;
    if (l < *n && fill_less(h[l], best)) {
      m = l;
      best = h[l];
    }
    if (r < *n && fill_less(h[r], best)) m = r;
    if (m == i) break;
    h[i] = h[m];
    i = m;
  }
  if (*n > 0) h[i] = x;
  return top;
}

static float fill_up(float x, float eps) {
  float a = x + eps;
  float b = nextafterf(x, INFINITY);
  return a > b ? a : b;
}

/* F from z (both H x W, row-major).  Returns OR_OK, OR_ERR_NONFINITE (F is
 * then unspecified), OR_ERR_NOMEM or OR_ERR_ARG. */
int oracle_fill_eps(const float* z, int64_t H, int64_t W, float eps, float* F) {
  if (!z || !F || H < 1 || W < 1 || !(eps >= 0.0f)) return OR_ERR_ARG;
  int64_t N = H * W;
  for (int64_t c = 0; c < N; c++)
    if (!isfinite(z[c])) return OR_ERR_NONFINITE;
  uint8_t* closed = (uint8_t*)calloc((size_t)N, 1);
  fill_item* h = (fill_item*)malloc(sizeof(fill_item) * (size_t)N);
  if (!closed || !h) {
    free(closed);
    free(h);
    return OR_ERR_NOMEM;
  }
  int64_t n = 0;
  for (int64_t i = 0; i < H; i++)
    for (int64_t j = 0; j < W; j++)
      if (i == 0 || j == 0 || i == H - 1 || j == W - 1) {
        int64_t c = i * W + j;
        F[c] = z[c];
        closed[c] = 1;
        fill_item it = {F[c], c};
        heap_push(h, &n, it);
      }
  while (n > 0) {
    fill_item p = heap_pop(h, &n);
    int64_t pi = p.c / W, pj = p.c % W;
    for (int k = 0; k < 8; k++) {
      int64_t i = pi + ODI[k], j = pj + ODJ[k];
      if (i < 0 || j < 0 || i >= H || j >= W) continue;
      int64_t c = i * W + j;
      if (closed[c]) continue;
      closed[c] = 1;
      F[c] = z[c] > p.f ? z[c] : fill_up(p.f, eps);
      fill_item it = {F[c], c};
      heap_push(h, &n, it);
    }
  }
  free(closed);
  free(h);
  return OR_OK;
}
