/*
 * sg_oracle.h -- declarations of the plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * header, helper, table or constant with the CUDA library: its expression
 * op numbering below is its own.
 *
 * Everything here is the slow, obviously-correct definition of an operation
 * of "Contract-Based General-Purpose GPU Programming" (Kolesnichenko, Poskitt,
 * Nanz, Meyer; SafeGPU):  collection operations of Table 2 and Sec. 3.2-3.4,
 * contracts of Sec. 4, the Gaussian elimination of Sec. 5 (Listing 6, read as
 * textbook elimination with partial pivoting), plus the matrix-product check
 * (Freivalds), the iterative-refinement solve, the batched chain and the
 * 2x64 MLP cost model that the GPU library adds on top of the paper.
 */
#ifndef SG_ORACLE_H
#define SG_ORACLE_H
#include <stdint.h>

/* Expression op codes (oracle numbering).  Postfix program over a stack of
 * IEEE binary32 values; booleans are 1.0f / 0.0f; a value is "true" when it
 * compares unequal to 0.0f (so NaN is true). */
enum {
  ORX_LOAD = 1,  /* arg = input index k: push in[k][i]              */
  ORX_CONST,     /* cst: push the binary32 constant                 */
  ORX_ADD, ORX_SUB, ORX_MUL, ORX_DIV, /* pop b, pop a, push a op b     */
  ORX_FMA,       /* pop c, b, a: push fmaf(a, b, c) (one rounding)   */
  ORX_MIN, ORX_MAX, /* NaN if either is NaN, else (a<b?a:b) / (a>b?a:b) */
  ORX_NEG, ORX_ABS, ORX_SQRT,
  ORX_LT, ORX_LE, ORX_GT, ORX_GE, ORX_EQ, ORX_NE,
  ORX_AND, ORX_OR, ORX_NOT,
  ORX_SELECT,    /* pop f, t, c: push (c true) ? t : f               */
  ORX_DUP, ORX_SWAP,
  ORX_INDEX      /* push (float)i (element index, rounded to binary32) */
};

#define OR_ERR_EXPR   (-2)  /* malformed program (stack under/overflow, bad op) */
#define OR_ERR_ARG    (-3)

/* ---- collection operations (Table 2; Sec. 3.2-3.3) ---- */
int     or_map(int nops, const int* op, const int* arg, const float* cst,
               int nin, const float* const* in, int64_t n, float* out);
int64_t or_first_false(int nops, const int* op, const int* arg, const float* cst,
                       int nin, const float* const* in, int64_t n);
int64_t or_first_true(int nops, const int* op, const int* arg, const float* cst,
                      int nin, const float* const* in, int64_t n);
int64_t or_filter(int nops, const int* op, const int* arg, const float* cst,
                  int nin, const float* const* in, int64_t n, float* out);
double  or_sum_f32(const float* x, int64_t n);
float   or_min_f32(const float* x, int64_t n);
float   or_max_f32(const float* x, int64_t n);

/* ---- sort and its contracts (Listing 4 postconditions; is_sorted) ---- */
void    or_sort_i32(const int32_t* x, int64_t n, int32_t* out);
int64_t or_first_unsorted_i32(const int32_t* x, int64_t n);
int     or_same_multiset_i32(const int32_t* a, const int32_t* b, int64_t n);
/* binary32 keys (Listing 4 sorts REAL_32): ascending in IEEE 754 totalOrder
 * (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN); is_sorted in the
 * IEEE comparison: first i with x[i] > x[i+1] (NaN compares false)        */
void    or_sort_f32(const float* x, int64_t n, float* out);
int64_t or_first_unsorted_f32(const float* x, int64_t n);

/* ---- matrix product and its check (Sec. 3.4 `multiply`) ---- */
void    or_matmul_f64(const float* A, const float* B, int64_t M, int64_t K,
                      int64_t N, double* C);
void    or_matmul_rows_f64(const float* A, const float* B, int64_t M, int64_t K,
                           int64_t N, const int64_t* rows, int64_t nrows,
                           double* C);
/* ---- transpose and matrix-vector products (Sec. 3.4 `transpose`,
 *      `right_multiply`, `left_multiply`; Listing 1) ---- */
void    or_transpose_f32(const float* A, int64_t rows, int64_t cols, float* At);
void    or_matvec_f64(const float* A, int64_t rows, int64_t cols, const float* x,
                      double* y);
void    or_vecmat_f64(const float* x, const float* A, int64_t rows, int64_t cols,
                      double* y);
uint64_t or_splitmix64(uint64_t state_after_increment);
/* ---- `old` (Sec. 4, Listing 3: Current = old Current) ---- */
int64_t or_first_changed(const void* before, const void* after, int64_t units, int unit_bytes);
void    or_fingerprint_old(const void* x, int64_t units, int unit_bytes, uint64_t* f);
double  or_rademacher(uint64_t seed, int64_t v, int64_t n, int64_t j);
int64_t or_freivalds(const float* A, const float* B, const float* C, int64_t N,
                     uint64_t seed, int nvec, double c, double u_eff,
                     double* gap, double* tau);

/* ---- Gaussian elimination (Sec. 5, Listing 6 read as GEPP) ---- */
int     or_gepp_f64(double* A, int64_t n, int32_t* piv);
void    or_lu_solve_f64(const double* LU, const int32_t* piv, int64_t n,
                        double* b);
int     or_solve_f32a(const float* A, const double* b, int64_t n, double* x);
double  or_det_f64(const double* LU, const int32_t* piv, int64_t n);

/* ---- batched chain: map -> require for_all -> filter -> sum ---- */
int     or_batch_chain(int nm, const int* mop, const int* marg, const float* mcst,
                       int np, const int* pop, const int* parg, const float* pcst,
                       int nf, const int* fop, const int* farg, const float* fcst,
                       const float* x, const int64_t* off, int64_t nseg,
                       double* sums, int64_t* first_viol, int64_t* kept);

/* ---- 2x64 MLP cost model (FP64) ---- */
void    or_mlp_forward(const double* P, int d_in, int H, const double* X,
                       int64_t B, double* yhat);
double  or_mlp_loss_grad(const double* P, int d_in, int H, const double* X,
                         const double* y, int64_t B, double* G);
void    or_adam_step(double* P, const double* G, double* m, double* v,
                     int64_t np, int64_t t, double lr, double b1, double b2,
                     double eps);
int64_t or_mlp_nparams(int d_in, int H);

#endif
