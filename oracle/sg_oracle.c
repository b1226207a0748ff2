/*
 * sg_oracle.c -- plain, slow, obviously-correct CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py, never by the library.  It shares
 * no code with the CUDA path.  Build with -ffp-contract=off so that a*b+c is
 * never silently fused (fmaf is used only where the program says FMA).
 *
 * Paper: Kolesnichenko, Poskitt, Nanz, Meyer, "Contract-Based General-Purpose
 * GPU Programming" (SafeGPU).  Each function cites the passage it follows.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_*.py against
 * closed forms, brute force on <= 8 elements, exact rational arithmetic or
 * finite differences; none is "parity unpinned".
 */
#include "sg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Expression evaluation.  Sec. 3.2: agents (functions / predicates) applied
 * to every element; Sec. 5 / Fig. 3: the fused form a*X[i]+Y[i] is just a
 * longer expression over the same element index.  Evaluated in binary32
 * with round-to-nearest-even, one operation at a time, in program order.    */

#define OR_STACK 64

static int is_true(float v) { return v != 0.0f; }

static float fmin_nan(float a, float b) {
  if (isnan(a) || isnan(b)) return NAN;
  return (a < b) ? a : b;
}
static float fmax_nan(float a, float b) {
  if (isnan(a) || isnan(b)) return NAN;
  return (a > b) ? a : b;
}

/* Returns 0 and the top of the stack in *res, or OR_ERR_EXPR. */
static int eval_at(int nops, const int* op, const int* arg, const float* cst,
                   int nin, const float* const* in, int64_t i, float* res) {
  float s[OR_STACK];
  int sp = 0; /* number of values on the stack */
  for (int p = 0; p < nops; ++p) {
    float a, b, c;
    switch (op[p]) {
      case ORX_LOAD:
        if (arg[p] < 0 || arg[p] >= nin || sp >= OR_STACK) return OR_ERR_EXPR;
        s[sp++] = in[arg[p]][i];
        break;
      case ORX_CONST:
        if (sp >= OR_STACK) return OR_ERR_EXPR;
        s[sp++] = cst[p];
        break;
      case ORX_INDEX:
        if (sp >= OR_STACK) return OR_ERR_EXPR;
        s[sp++] = (float)i;
        break;
      case ORX_ADD: case ORX_SUB: case ORX_MUL: case ORX_DIV:
      case ORX_MIN: case ORX_MAX:
      case ORX_LT: case ORX_LE: case ORX_GT: case ORX_GE: case ORX_EQ: case ORX_NE:
      case ORX_AND: case ORX_OR:
        if (sp < 2) return OR_ERR_EXPR;
        b = s[--sp];
        a = s[--sp];
        switch (op[p]) {
          case ORX_ADD: c = a + b; break;
          case ORX_SUB: c = a - b; break;
          case ORX_MUL: c = a * b; break;
          case ORX_DIV: c = a / b; break;
          case ORX_MIN: c = fmin_nan(a, b); break;
          case ORX_MAX: c = fmax_nan(a, b); break;
          case ORX_LT: c = (a < b) ? 1.0f : 0.0f; break;
          case ORX_LE: c = (a <= b) ? 1.0f : 0.0f; break;
          case ORX_GT: c = (a > b) ? 1.0f : 0.0f; break;
          case ORX_GE: c = (a >= b) ? 1.0f : 0.0f; break;
          case ORX_EQ: c = (a == b) ? 1.0f : 0.0f; break;
          case ORX_NE: c = (a != b) ? 1.0f : 0.0f; break;
          case ORX_AND: c = (is_true(a) && is_true(b)) ? 1.0f : 0.0f; break;
          default:      c = (is_true(a) || is_true(b)) ? 1.0f : 0.0f; break;
        }
        s[sp++] = c;
        break;
      case ORX_FMA:
        if (sp < 3) return OR_ERR_EXPR;
        c = s[--sp];
        b = s[--sp];
        a = s[--sp];
        s[sp++] = fmaf(a, b, c);
        break;
      case ORX_NEG: case ORX_ABS: case ORX_SQRT: case ORX_NOT:
        if (sp < 1) return OR_ERR_EXPR;
        a = s[sp - 1];
        if (op[p] == ORX_NEG) a = -a;
        else if (op[p] == ORX_ABS) a = fabsf(a);
        else if (op[p] == ORX_SQRT) a = sqrtf(a);
        else a = is_true(a) ? 0.0f : 1.0f;
        s[sp - 1] = a;
        break;
      case ORX_SELECT:
        if (sp < 3) return OR_ERR_EXPR;
        b = s[--sp]; /* f */
        a = s[--sp]; /* t */
        c = s[--sp]; /* cond */
        s[sp++] = is_true(c) ? a : b;
        break;
      case ORX_DUP:
        if (sp < 1 || sp >= OR_STACK) return OR_ERR_EXPR;
        s[sp] = s[sp - 1];
        ++sp;
        break;
      case ORX_SWAP:
        if (sp < 2) return OR_ERR_EXPR;
        a = s[sp - 1];
        s[sp - 1] = s[sp - 2];
        s[sp - 2] = a;
        break;
      default:
        return OR_ERR_EXPR;
    }
  }
  if (sp != 1) return OR_ERR_EXPR;
  *res = s[0];
  return 0;
}

/* `project` / `for_each` (Table 2; Sec. 3.2): out[i] = f(inputs at i). */
int or_map(int nops, const int* op, const int* arg, const float* cst,
           int nin, const float* const* in, int64_t n, float* out) {
  for (int64_t i = 0; i < n; ++i) {
    float r;
    int e = eval_at(nops, op, arg, cst, nin, in, i, &r);
    if (e) return e;
    out[i] = r;
  }
  return 0;
}

/* `for_all` (Table 2): the smallest index where the predicate is false, or -1
 * when it holds everywhere (so for_all on an empty collection holds). */
int64_t or_first_false(int nops, const int* op, const int* arg, const float* cst,
                       int nin, const float* const* in, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    float r;
    if (eval_at(nops, op, arg, cst, nin, in, i, &r)) return OR_ERR_EXPR;
    if (!is_true(r)) return i;
  }
  return -1;
}

/* `exists` (Table 2): the smallest index where the predicate holds, or -1
 * (so exists on an empty collection is false). */
int64_t or_first_true(int nops, const int* op, const int* arg, const float* cst,
                      int nin, const float* const* in, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    float r;
    if (eval_at(nops, op, arg, cst, nin, in, i, &r)) return OR_ERR_EXPR;
    if (is_true(r)) return i;
  }
  return -1;
}

/* `filter` (Table 2; Sec. 3.2 example a < 5): the items of in[0] for which
 * the predicate holds, kept in index order.  Returns their count. */
int64_t or_filter(int nops, const int* op, const int* arg, const float* cst,
                  int nin, const float* const* in, int64_t n, float* out) {
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i) {
    float r;
    if (eval_at(nops, op, arg, cst, nin, in, i, &r)) return OR_ERR_EXPR;
    if (is_true(r)) out[m++] = in[0][i];
  }
  return m;
}

/* Vector `sum` (Sec. 3.3): exact products are not involved; the terms are
 * added in index order in binary64.  An empty sum is 0. */
double or_sum_f32(const float* x, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += (double)x[i];
  return s;
}

/* Vector `min` / `max` (Sec. 3.3).  NaN anywhere gives NaN.  n must be > 0. */
float or_min_f32(const float* x, int64_t n) {
  float m = x[0];
  for (int64_t i = 1; i < n; ++i) m = fmin_nan(m, x[i]);
  return m;
}
float or_max_f32(const float* x, int64_t n) {
  float m = x[0];
  for (int64_t i = 1; i < n; ++i) m = fmax_nan(m, x[i]);
  return m;
}

/* ------------------------------------------------------------------------ */
/* Sorting (Listing 4: left (<) ++ mid (=) ++ right (>), i.e. ascending).
 * The C library's qsort is the sorting primitive; keys are signed int32.     */

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

void or_sort_i32(const int32_t* x, int64_t n, int32_t* out) {
  if (n <= 0) return;
  memcpy(out, x, (size_t)n * sizeof(int32_t));
  qsort(out, (size_t)n, sizeof(int32_t), cmp_i32);
}

/* `is_sorted` (Sec. 3.3; Listing 4 postcondition): the smallest i with
 * x[i] > x[i+1], or -1. */
/* IEEE 754 totalOrder written out by classes: negative NaNs (larger payload
 * first), negative numbers and -inf, -0, +0, positive numbers and +inf,
 * positive NaNs (smaller payload first).                                    */
static int f32_class(float v, uint32_t bits) {
  const int neg = (int)(bits >> 31);
  if (v != v) return neg ? 0 : 5;
  if (v == 0.0f) return neg ? 2 : 3;
  return neg ? 1 : 4;
}

static int cmp_f32_total(const void* a, const void* b) {
  float x, y;
  uint32_t bx, by;
  memcpy(&x, a, 4);
  memcpy(&y, b, 4);
  memcpy(&bx, a, 4);
  memcpy(&by, b, 4);
  const int cx = f32_class(x, bx), cy = f32_class(y, by);
  if (cx != cy) return (cx > cy) - (cx < cy);
  if (cx == 1 || cx == 4) return (x > y) - (x < y);
  const uint32_t px = bx & 0x7fffffffu, py = by & 0x7fffffffu;
  if (cx == 0) return (px < py) - (px > py);   /* negative NaNs: larger payload first */
  return (px > py) - (px < py);                /* positive NaNs (and the zeros) */
}

void or_sort_f32(const float* x, int64_t n, float* out) {
  if (n <= 0) return;
  memcpy(out, x, (size_t)n * sizeof(float));
  qsort(out, (size_t)n, sizeof(float), cmp_f32_total);
}

int64_t or_first_unsorted_f32(const float* x, int64_t n) {
  for (int64_t i = 0; i + 1 < n; ++i)
    if (x[i] > x[i + 1]) return i;
  return -1;
}

int64_t or_first_unsorted_i32(const int32_t* x, int64_t n) {
  for (int64_t i = 0; i + 1 < n; ++i)
    if (x[i] > x[i + 1]) return i;
  return -1;
}

/* Listing 4's `Result.count = a.count`, strengthened to multiset equality:
 * both sorted copies are equal element by element. */
int or_same_multiset_i32(const int32_t* a, const int32_t* b, int64_t n) {
  if (n <= 0) return 1;
  int32_t* sa = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  int32_t* sb = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!sa || !sb) { free(sa); free(sb); return OR_ERR_ARG; }
  or_sort_i32(a, n, sa);
  or_sort_i32(b, n, sb);
  int eq = memcmp(sa, sb, (size_t)n * sizeof(int32_t)) == 0;
  free(sa);
  free(sb);
  return eq;
}

/* ------------------------------------------------------------------------ */
/* Matrix `transpose` (Sec. 3.4; Listing 1): At[j][i] = A[i][j], row-major,
 * rows x cols in, cols x rows out.                                          */

void or_transpose_f32(const float* A, int64_t rows, int64_t cols, float* At) {
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t j = 0; j < cols; ++j) At[j * rows + i] = A[i * cols + j];
}

/* `right_multiply` (Sec. 3.4; Listing 1): y = A x, y[i] = sum_j A[i][j] x[j];
 * `left_multiply`: y = x^T A, y[j] = sum_i x[i] A[i][j].  Binary32 inputs
 * widened exactly, products and sums in binary64, index ascending.          */

void or_matvec_f64(const float* A, int64_t rows, int64_t cols, const float* x, double* y) {
  for (int64_t i = 0; i < rows; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < cols; ++j) s += (double)A[i * cols + j] * (double)x[j];
    y[i] = s;
  }
}

void or_vecmat_f64(const float* x, const float* A, int64_t rows, int64_t cols, double* y) {
  for (int64_t j = 0; j < cols; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < rows; ++i) s += (double)x[i] * (double)A[i * cols + j];
    y[j] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Matrix `multiply` (Sec. 3.4): C = A B, row-major, binary32 inputs widened
 * exactly to binary64, products and sums in binary64, k ascending.          */

void or_matmul_f64(const float* A, const float* B, int64_t M, int64_t K,
                   int64_t N, double* C) {
  for (int64_t i = 0; i < M; ++i) {
    double* c = C + i * N;
    for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double a = (double)A[i * K + k];
      const float* b = B + k * N;
      for (int64_t j = 0; j < N; ++j) c[j] += a * (double)b[j];
    }
  }
}

/* The same definition for a chosen subset of rows of C. */
void or_matmul_rows_f64(const float* A, const float* B, int64_t M, int64_t K,
                        int64_t N, const int64_t* rows, int64_t nrows,
                        double* C) {
  (void)M;
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    double* c = C + r * N;
    for (int64_t j = 0; j < N; ++j) c[j] = 0.0;
    for (int64_t k = 0; k < K; ++k) {
      double a = (double)A[i * K + k];
      const float* b = B + k * N;
      for (int64_t j = 0; j < N; ++j) c[j] += a * (double)b[j];
    }
  }
}

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): the state
 * after t increments is seed + t * 0x9E3779B97F4A7C15; the output mixes it. */
uint64_t or_splitmix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Listing 3's postcondition Current = old Current (Sec. 4): the collection
 * after the routine equals, unit for unit (bit patterns, so a NaN equals
 * itself and -0 differs from +0), the collection when the routine was
 * entered.  The plain definition: the first index of a unit (16- or 32-bit)
 * whose bits differ, or -1.                                                 */
int64_t or_first_changed(const void* before, const void* after, int64_t units,
                         int unit_bytes) {
  const unsigned char* a = (const unsigned char*)before;
  const unsigned char* b = (const unsigned char*)after;
  for (int64_t i = 0; i < units; ++i)
    if (memcmp(a + i * unit_bytes, b + i * unit_bytes, (size_t)unit_bytes) != 0) return i;
  return -1;
}

/* The library keeps `old` as a fingerprint instead of a copy.  Its
 * definition, written out: unit i (its bits w, zero-extended) contributes
 * h_i = SplitMix64's output function applied to i * 2^32 + w; f[0] = sum h_i
 * and f[1] = sum (h_i >> 32) * (h_i mod 2^32), both mod 2^64, i ascending. */
void or_fingerprint_old(const void* x, int64_t units, int unit_bytes, uint64_t* f) {
  const unsigned char* p = (const unsigned char*)x;
  uint64_t f1 = 0, f2 = 0;
  for (int64_t i = 0; i < units; ++i) {
    uint64_t w = 0;
    if (unit_bytes == 2) {
      uint16_t u;
      memcpy(&u, p + 2 * i, 2);
      w = u;
    } else {
      uint32_t u;
      memcpy(&u, p + 4 * i, 4);
      w = u;
    }
    const uint64_t h = or_splitmix64(((uint64_t)i << 32) | w);
    f1 += h;
    f2 += (h >> 32) * (h & 0xFFFFFFFFull);
  }
  f[0] = f1;
  f[1] = f2;
}

/* Rademacher entry j of check vector v (0-based) for an n-vector: the t-th
 * SplitMix64 draw of the stream `seed`, t = v*n + j + 1; its top bit picks
 * the sign (1 -> -1.0, 0 -> +1.0). */
double or_rademacher(uint64_t seed, int64_t v, int64_t n, int64_t j) {
  uint64_t t = (uint64_t)(v * n + j + 1);
  uint64_t z = or_splitmix64(seed + t * 0x9E3779B97F4A7C15ull);
  return (z >> 63) ? -1.0 : 1.0;
}

/* Freivalds' check of C = A B (square N x N), `nvec` Rademacher vectors r:
 *   z = A (B r), w = C r (binary64), row i is violated when |z_i - w_i| > tau_i,
 *   tau_i = c * u_eff * sqrt( sum_k a_ik^2 * ((B r)_k^2 + s_k) ),
 *   s_k = sum_j b_kj^2.
 * tau is a c-sigma bound of the rounding noise of a product whose operands and
 * accumulation have unit roundoff u_eff (the paper states no tolerance).
 * Returns the smallest violated row (over all vectors) or -1; gap[i], tau[i]
 * (optional) receive, per row, the largest |z_i - w_i| / tau_i pair seen.   */
int64_t or_freivalds(const float* A, const float* B, const float* C, int64_t N,
                     uint64_t seed, int nvec, double c, double u_eff,
                     double* gap, double* tau) {
  double* r = (double*)malloc((size_t)N * sizeof(double));
  double* br = (double*)malloc((size_t)N * sizeof(double));
  double* s = (double*)malloc((size_t)N * sizeof(double));
  if (!r || !br || !s) { free(r); free(br); free(s); return OR_ERR_ARG; }
  for (int64_t k = 0; k < N; ++k) {
    double acc = 0.0;
    for (int64_t j = 0; j < N; ++j) acc += (double)B[k * N + j] * (double)B[k * N + j];
    s[k] = acc;
  }
  if (gap) for (int64_t i = 0; i < N; ++i) gap[i] = 0.0;
  if (tau) for (int64_t i = 0; i < N; ++i) tau[i] = 0.0;
  int64_t first = -1;
  for (int v = 0; v < nvec; ++v) {
    for (int64_t j = 0; j < N; ++j) r[j] = or_rademacher(seed, v, N, j);
    for (int64_t k = 0; k < N; ++k) {
      double acc = 0.0;
      for (int64_t j = 0; j < N; ++j) acc += (double)B[k * N + j] * r[j];
      br[k] = acc;
    }
    for (int64_t i = 0; i < N; ++i) {
      double z = 0.0, w = 0.0, q = 0.0;
      for (int64_t k = 0; k < N; ++k) {
        double a = (double)A[i * N + k];
        z += a * br[k];
        q += a * a * (br[k] * br[k] + s[k]);
      }
      for (int64_t j = 0; j < N; ++j) w += (double)C[i * N + j] * r[j];
      double t = c * u_eff * sqrt(q);
      double g = fabs(z - w);
      if (gap && (tau[i] == 0.0 || g / t > gap[i] / tau[i])) { gap[i] = g; tau[i] = t; }
      if (g > t && (first < 0 || i < first)) first = i;
    }
  }
  free(r);
  free(br);
  free(s);
  return first;
}

/* ------------------------------------------------------------------------ */
/* Gaussian elimination (Sec. 5, Listing 6).  The listing eliminates without
 * pivoting; it is read here as the textbook right-looking elimination with
 * partial pivoting: at step k the pivot row is the lowest index i >= k with
 * the largest |a_ik| (compared in binary64), rows k and piv[k] are swapped,
 * the multipliers l_ik = a_ik / a_kk are stored below the diagonal and the
 * trailing block is updated a_ij -= l_ik a_kj.  A is n x n row-major, in
 * place.  Returns 0, or k+1 when the pivot of step k is exactly zero.      */
int or_gepp_f64(double* A, int64_t n, int32_t* piv) {
  int info = 0;
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = k;
    double best = fabs(A[k * n + k]);
    for (int64_t i = k + 1; i < n; ++i) {
      double m = fabs(A[i * n + k]);
      if (m > best) { best = m; p = i; }
    }
    piv[k] = (int32_t)p;
    if (p != k)
      for (int64_t j = 0; j < n; ++j) {
        double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
    double d = A[k * n + k];
    if (d == 0.0) {
      if (!info) info = (int)(k + 1);
      continue;
    }
    for (int64_t i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / d;
      A[i * n + k] = l;
      for (int64_t j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return info;
}

/* Solve A x = b from P A = L U: apply the row swaps to b, then forward
 * substitution with the unit lower L and back substitution with U. */
void or_lu_solve_f64(const double* LU, const int32_t* piv, int64_t n,
                     double* b) {
  for (int64_t k = 0; k < n; ++k) {
    int64_t p = piv[k];
    if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
  }
  for (int64_t i = 0; i < n; ++i) {
    double s = b[i];
    for (int64_t j = 0; j < i; ++j) s -= LU[i * n + j] * b[j];
    b[i] = s;
  }
  for (int64_t i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int64_t j = i + 1; j < n; ++j) s -= LU[i * n + j] * b[j];
    b[i] = s / LU[i * n + i];
  }
}

/* x = A^{-1} b for a binary32 matrix (widened exactly) and binary64 b. */
int or_solve_f32a(const float* A, const double* b, int64_t n, double* x) {
  double* LU = (double*)malloc((size_t)(n * n) * sizeof(double));
  int32_t* piv = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!LU || !piv) { free(LU); free(piv); return OR_ERR_ARG; }
  for (int64_t i = 0; i < n * n; ++i) LU[i] = (double)A[i];
  int info = or_gepp_f64(LU, n, piv);
  if (!info) {
    memcpy(x, b, (size_t)n * sizeof(double));
    or_lu_solve_f64(LU, piv, n, x);
  }
  free(LU);
  free(piv);
  return info;
}

/* The determinant that Listing 6 aims at: det A = (-1)^(#swaps) prod u_kk. */
double or_det_f64(const double* LU, const int32_t* piv, int64_t n) {
  double d = 1.0;
  for (int64_t k = 0; k < n; ++k) {
    d *= LU[k * n + k];
    if (piv[k] != k) d = -d;
  }
  return d;
}

/* ------------------------------------------------------------------------ */
/* Batched chain over ragged segments: for each segment s (elements
 * off[s] .. off[s+1]-1 of x), in index order:
 *   y = map(x)                     (the map program, input 0 = x)
 *   require for_all(pre(y))        (first violating index within the segment,
 *                                   or -1)
 *   kept = filter(y, filt)         (count of kept elements)
 *   sums = sum(kept) in binary64   (the filter output is only summed).
 * Sec. 3.2 (project, filter, for_all) and Sec. 3.3 (sum) applied per
 * collection.  A segment whose precondition fails still reports its sum. */
int or_batch_chain(int nm, const int* mop, const int* marg, const float* mcst,
                   int np, const int* pop, const int* parg, const float* pcst,
                   int nf, const int* fop, const int* farg, const float* fcst,
                   const float* x, const int64_t* off, int64_t nseg,
                   double* sums, int64_t* first_viol, int64_t* kept) {
  for (int64_t s = 0; s < nseg; ++s) {
    const int64_t b = off[s], L = off[s + 1] - off[s];
    double acc = 0.0;
    int64_t cnt = 0, fv = -1;
    float* y = (float*)malloc((size_t)(L > 0 ? L : 1) * sizeof(float));
    if (!y) return OR_ERR_ARG;
    /* each agent sees the collection's own elements and index k = 0..L-1 */
    const float* xin[1] = {x + b};
    const float* yin[1] = {y};
    for (int64_t k = 0; k < L; ++k)
      if (eval_at(nm, mop, marg, mcst, 1, xin, k, &y[k])) { free(y); return OR_ERR_EXPR; }
    for (int64_t k = 0; k < L; ++k) {
      float pr, fr;
      if (eval_at(np, pop, parg, pcst, 1, yin, k, &pr) ||
          eval_at(nf, fop, farg, fcst, 1, yin, k, &fr)) { free(y); return OR_ERR_EXPR; }
      if (!is_true(pr) && fv < 0) fv = k;
      if (is_true(fr)) { acc += (double)y[k]; ++cnt; }
    }
    free(y);
    sums[s] = acc;
    first_viol[s] = fv;
    kept[s] = cnt;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 2x64 MLP cost model: yhat = W3 relu(W2 relu(W1 x + b1) + b2) + b3.
 * Parameter vector P = [W1 (H x d_in, row-major), b1 (H), W2 (H x H), b2 (H),
 * W3 (H), b3 (1)].  Loss = mean over the batch of (yhat - y)^2.  ReLU'(0) = 0.
 * Adam as in Kingma & Ba (ICLR 2015), bias-corrected.                       */

int64_t or_mlp_nparams(int d_in, int H) {
  return (int64_t)H * d_in + H + (int64_t)H * H + H + H + 1;
}

static void mlp_rows(const double* P, int d_in, int H, const double* x,
                     double* z1, double* h1, double* z2, double* h2,
                     double* yhat) {
  const double* W1 = P;
  const double* b1 = W1 + (int64_t)H * d_in;
  const double* W2 = b1 + H;
  const double* b2 = W2 + (int64_t)H * H;
  const double* W3 = b2 + H;
  const double* b3 = W3 + H;
  for (int j = 0; j < H; ++j) {
    double a = b1[j];
    for (int k = 0; k < d_in; ++k) a += W1[(int64_t)j * d_in + k] * x[k];
    z1[j] = a;
    h1[j] = a > 0.0 ? a : 0.0;
  }
  for (int j = 0; j < H; ++j) {
    double a = b2[j];
    for (int k = 0; k < H; ++k) a += W2[(int64_t)j * H + k] * h1[k];
    z2[j] = a;
    h2[j] = a > 0.0 ? a : 0.0;
  }
  double o = b3[0];
  for (int k = 0; k < H; ++k) o += W3[k] * h2[k];
  *yhat = o;
}

void or_mlp_forward(const double* P, int d_in, int H, const double* X,
                    int64_t B, double* yhat) {
  double* buf = (double*)malloc((size_t)4 * H * sizeof(double));
  if (!buf) return;
  for (int64_t b = 0; b < B; ++b)
    mlp_rows(P, d_in, H, X + b * d_in, buf, buf + H, buf + 2 * H, buf + 3 * H,
             &yhat[b]);
  free(buf);
}

/* Loss and its gradient G (same layout as P) by backpropagation. */
double or_mlp_loss_grad(const double* P, int d_in, int H, const double* X,
                        const double* y, int64_t B, double* G) {
  int64_t np = or_mlp_nparams(d_in, H);
  for (int64_t i = 0; i < np; ++i) G[i] = 0.0;
  const double* W2 = P + (int64_t)H * d_in + H;
  const double* W3 = W2 + (int64_t)H * H + H;
  double* gW1 = G;
  double* gb1 = gW1 + (int64_t)H * d_in;
  double* gW2 = gb1 + H;
  double* gb2 = gW2 + (int64_t)H * H;
  double* gW3 = gb2 + H;
  double* gb3 = gW3 + H;
  double* buf = (double*)malloc((size_t)6 * H * sizeof(double));
  if (!buf) return NAN;
  double *z1 = buf, *h1 = buf + H, *z2 = buf + 2 * H, *h2 = buf + 3 * H;
  double *d2 = buf + 4 * H, *d1 = buf + 5 * H;
  double loss = 0.0;
  for (int64_t b = 0; b < B; ++b) {
    const double* x = X + b * d_in;
    double yh;
    mlp_rows(P, d_in, H, x, z1, h1, z2, h2, &yh);
    double e = yh - y[b];
    loss += e * e;
    double dy = 2.0 * e / (double)B;
    gb3[0] += dy;
    for (int k = 0; k < H; ++k) {
      gW3[k] += dy * h2[k];
      d2[k] = z2[k] > 0.0 ? dy * W3[k] : 0.0;
    }
    for (int j = 0; j < H; ++j) {
      gb2[j] += d2[j];
      for (int k = 0; k < H; ++k) gW2[(int64_t)j * H + k] += d2[j] * h1[k];
    }
    for (int k = 0; k < H; ++k) {
      double a = 0.0;
      for (int j = 0; j < H; ++j) a += W2[(int64_t)j * H + k] * d2[j];
      d1[k] = z1[k] > 0.0 ? a : 0.0;
    }
    for (int j = 0; j < H; ++j) {
      gb1[j] += d1[j];
      for (int k = 0; k < d_in; ++k) gW1[(int64_t)j * d_in + k] += d1[j] * x[k];
    }
  }
  free(buf);
  return loss / (double)B;
}

void or_adam_step(double* P, const double* G, double* m, double* v,
                  int64_t np, int64_t t, double lr, double b1, double b2,
                  double eps) {
  double c1 = 1.0 - pow(b1, (double)t);
  double c2 = 1.0 - pow(b2, (double)t);
  for (int64_t i = 0; i < np; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * G[i];
    v[i] = b2 * v[i] + (1.0 - b2) * G[i] * G[i];
    double mh = m[i] / c1;
    double vh = v[i] / c2;
    P[i] -= lr * mh / (sqrt(vh) + eps);
  }
}
