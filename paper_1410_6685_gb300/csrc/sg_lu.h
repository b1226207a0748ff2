// sg_lu.h -- elimination and solve kernels (k_lu.cu).  Internal.
#pragma once
#include "sg_internal.h"

namespace sgk {

constexpr int kLuPanel = 32;      // panel width of the blocked factorisation
constexpr int kLuOuter = 128;     // outer block: one tensor-core update per 128 columns
constexpr int kLuMaxN = 9216;     // the panel must fit the cluster's shared memory

size_t lu_panel_max_smem(int n);
// kernel attributes (shared-memory sizes, the panel's cluster size) for
// factorisations up to n; called before a factorisation is captured
cudaError_t lu_prepare(int n);
// moves: the panel's slot of kLuMoveInts ints, zero before the call; the
// kernel lists there the rows its interchanges moved (count, sources,
// destinations) and applies them itself to the columns [c_lo, c_hi) of its
// outer block outside the panel.
constexpr int kLuMoveInts = 1 + 4 * kLuPanel;
cudaError_t launch_lu_panel(float* LU, int n, int k, int jb, int* piv, int* info, int* moves,
                            int c_lo, int c_hi, cudaStream_t s, Prof* prof);
// the interchanges of the nlists panels of the outer block [K, K + KB) (their
// moves slots, consecutive) on every column outside it and on perm
cudaError_t launch_lu_laswp_outer(float* LU, int n, const int* moves, int nlists, int K, int KB,
                                  int* perm, cudaStream_t s, Prof* prof);
// after the panel at j (32 columns) inside an outer block: rows j..j+32 of
// columns [c0, c1) := L11^-1 (them), then rows j+32..n of those columns -=
// L21 U12.  counter: one zero word per call.
cudaError_t launch_lu_inner(float* LU, int n, int j, int c0, int c1, unsigned* counter,
                            cudaStream_t s, Prof* prof);
// rows K..K+KB of columns [c0, c1) := L11^-1 (them), L11 = the unit lower
// triangle at (K, K); KB a multiple of 32, at most kLuOuter
cudaError_t launch_lu_trsm_outer(float* LU, int n, int K, int KB, int c0, int c1, cudaStream_t s,
                                 Prof* prof);
// perm[i] = i; the outer blocks' interchange launches then turn it into
// perm[i] = the row of A that elimination moved to row i
cudaError_t launch_lu_iota(int* perm, int n, cudaStream_t s);
// y = U^-1 L^-1 P rhs in binary32 (P rhs gathered through perm).
// flags: 2*ceil(n/64) words (or more) that never hold `epoch` before the call.
cudaError_t launch_lu_solve(const float* LU, const float* inv, int n, const int* perm,
                            const double* rhs, bool rhs_is_residual, float* y, unsigned* flags,
                            unsigned epoch, unsigned* tickets, int* err, cudaStream_t s,
                            Prof* prof);
// inv: lu_diag_inv_bytes(n): 2 * ceil(n/64) blocks of 64x64 floats, the
// inverses of the diagonal blocks of L (unit lower) then of U, row-major,
// for launch_lu_solve
size_t lu_diag_inv_bytes(int n);
cudaError_t launch_lu_diag_inv(const float* LU, int n, float* inv, cudaStream_t s);
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
