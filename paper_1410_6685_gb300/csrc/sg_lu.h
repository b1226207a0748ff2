// sg_lu.h -- elimination and solve kernels (k_lu.cu).  Internal.
#pragma once
#include "sg_internal.h"

namespace sgk {

constexpr int kLuPanel = 32;      // panel width of the blocked factorisation
constexpr int kLuOuter = 128;     // outer block: one tensor-core update per 128 columns
constexpr int kLuMaxN = 9216;     // the panel must fit the cluster's shared memory

size_t lu_panel_max_smem(int n);
// moves: the panel's slot of kLuMoveInts ints, zero before the call; the
// kernel lists there the rows its interchanges moved (count, sources,
// destinations) for launch_lu_laswp.
constexpr int kLuMoveInts = 1 + 4 * kLuPanel;
cudaError_t launch_lu_panel(float* LU, int n, int k, int jb, int* piv, int* info, int* moves,
                            cudaStream_t s, Prof* prof);
// the panel's interchanges on every column outside the panel
cudaError_t launch_lu_laswp(float* LU, int n, int k, int jb, const int* moves, cudaStream_t s,
                            Prof* prof);
// rows k..k+jb of columns [c0, c1) := L11^-1 (them), L11 = unit lower at (k, k)
cudaError_t launch_lu_trsm(float* LU, int n, int k, int jb, int c0, int c1, cudaStream_t s,
                           Prof* prof);
// perm[i] = the row of A that the interchanges piv[0..n) moved to row i
// (dynamic shared memory of n ints: n <= kLuMaxN)
cudaError_t launch_lu_perm(const int* piv, int n, int* perm, cudaStream_t s);
// y = U^-1 L^-1 P rhs in binary32 (P rhs gathered through perm).
// flags: 2*ceil(n/32) words that never hold `epoch` before the call.
cudaError_t launch_lu_solve(const float* LU, int n, const int* perm, const double* rhs,
                            bool rhs_is_residual, float* y, unsigned* flags, unsigned epoch,
                            unsigned* tickets, int* err, cudaStream_t s, Prof* prof);
// r = b - A x in binary64; norms[0] = max|r|; rows with |r_i| > thresh
// (or NaN) raise ~i into *viol (when viol is not null).
cudaError_t launch_residual(const float* A, int n, const double* b, const double* x, double* r,
                            double* norms, double thresh, unsigned long long* viol,
                            cudaStream_t s, Prof* prof);
cudaError_t launch_anorm(const float* A, int n, double* norms, cudaStream_t s);   // norms[3]
// out[0] = sign of det A (0 if singular), out[1] = log |det A|, from the factors
cudaError_t launch_lu_det(const float* LU, int n, const int* piv, double* out, cudaStream_t s,
                          Prof* prof);
// x = d (init) or x += d; norms[1] = max|d|, norms[2] = max|x|, norms[4] = max|b|
cudaError_t launch_update(double* x, const float* d, const double* b, int n, bool init,
                          double* norms, cudaStream_t s);

}  // namespace sgk
