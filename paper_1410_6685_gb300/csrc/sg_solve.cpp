// sg_solve.cpp -- Gaussian elimination with partial pivoting and the solve
// with iterative refinement (Sec. 5, Listing 6; the mixed-precision form
// and the residual postcondition are the library's).
//
//   1. P A = L U in binary32 storage: panels of 32 columns factored by a
//      thread-block cluster, trailing updates A22 -= L21 U12 on the tensor
//      cores (bf16 / fp16 operands, binary32 accumulation) or in binary32 on
//      the CUDA cores.
//   2. x0 = U^-1 L^-1 P b (binary32 substitution of b rounded to binary32).
//   3. repeat: r = b - A x in binary64 (A widened exactly), d = LU \ r in
//      binary32, x += d in binary64, until max|d| <= refine_tol max|x|, or
//      the correction stops shrinking (max|d| > max|d_prev| / 2: the
//      binary64 residual limits what refinement can reach), or max_iter
//      steps (SG_ERR_NOT_CONVERGED).
//   4. postcondition (mode >= PRE_POST): max|b - A x| <= residual_tol
//      (|A|_inf max|x| + max|b|), evaluated in binary64; the first row over
//      the bound is reported.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_linalg_kernels.h"
#include "sg_lu.h"
#include "sg_runtime.h"

struct sg_matrix : public sg_vector {};

namespace {

sg_status err(sg_ctx* c, sg_status s, const char* m) {
  if (c) c->err = m;
  return s;
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

struct SolveWork {
  float* lu;
  int* piv;
  float* y;
  double* r;
  unsigned* flags;
  unsigned* tickets;
  int* dev_err;
  int* info;
  double* norms;          // [0] max|r| [1] max|d| [2] max|x| [3] |A|_inf [4] max|b|
  unsigned long long* viol;
};

// Blocked elimination with partial pivoting of the n x n binary32 matrix in
// `lu` (row-major), in place: L (unit lower) and U overwrite it, piv[k] is
// the row interchanged with row k at step k, *info = k+1 at an exactly zero
// pivot.  moves: ceil(n / kLuPanel) * kLuMoveInts ints, zero on entry.
// gemm: tensor-core scratch (gemm_tc_scratch_bytes(n, n, kLuOuter)),
// unused for binary32 updates.
cudaError_t factor_in_place(sg_ctx* c, float* lu, int n, int* piv, int* perm, int* info,
                            int* moves, unsigned* counters, void* gemm, sg_precision prec,
                            cudaStream_t s, sgk::Prof* prof) {
  cudaError_t e = cudaSuccess;
  // two levels: 32-column panels inside 128-column outer blocks.  Inside an
  // outer block each panel applies its interchanges to the block's other
  // columns and one fused kernel updates the block's columns to its right;
  // per outer block one launch applies its interchanges everywhere else, one
  // solves U12 for its 128 rows, and the trailing matrix is updated with
  // K = 128 (tensor cores, or binary32 SIMT)
  const bool tc = prec != SG_PREC_F32_SIMT;
  auto at = [&](int r, int col) { return lu + (size_t)r * n + col; };
  for (int K = 0; K < n && e == cudaSuccess; K += sgk::kLuOuter) {
    const int KB = std::min(sgk::kLuOuter, n - K);
    int* mv0 = moves + (size_t)(K / sgk::kLuPanel) * sgk::kLuMoveInts;
    int np = 0;
    for (int j = K; j < K + KB && e == cudaSuccess; j += sgk::kLuPanel, ++np) {
      const int jb = std::min(sgk::kLuPanel, K + KB - j);
      int* mv = moves + (size_t)(j / sgk::kLuPanel) * sgk::kLuMoveInts;
      e = sgk::launch_lu_panel(lu, n, j, jb, piv, info, mv, K, K + KB, s, prof);
      c->kernels += 1;
      if (e == cudaSuccess && j + jb < K + KB) {
        e = sgk::launch_lu_inner(lu, n, j, j + jb, K + KB, counters + j / sgk::kLuPanel, s, prof);
        c->kernels += 1;
      }
    }
    if (e == cudaSuccess) {
      e = sgk::launch_lu_laswp_outer(lu, n, mv0, np, K, KB, perm, s, prof);
      c->kernels += 1;
    }
    const int rest = n - K - KB;
    if (rest > 0 && e == cudaSuccess) {
      e = sgk::launch_lu_trsm_outer(lu, n, K, KB, K + KB, n, s, prof);
      c->kernels += 1;
      if (e == cudaSuccess && tc) {
        e = sgk::launch_gemm_tc(at(K + KB, K), n, at(K, K + KB), n, at(K + KB, K + KB), n, rest,
                                rest, KB, prec == SG_PREC_F16_TC, true, gemm, s, prof,
                                &c->kernels);
      } else if (e == cudaSuccess) {
        e = sgk::launch_gemm_f32(at(K + KB, K), n, at(K, K + KB), n, at(K + KB, K + KB), n, rest,
                                 rest, KB, true, s, prof);
        c->kernels += 1;
      }
    }
  }
  return e;
}

// Factors A (n x n binary32) into the context's cached workspace: the first
// call for a size and precision allocates it and captures the blocked
// elimination (memsets and about 7 n / 32 kernels) as a CUDA graph on a
// private stream; every call copies A in and replays the graph on the
// context's stream.  Afterwards c->lu.lu holds L\U, c->lu.piv the
// interchanges and c->lu.info the zero-pivot report.
sg_status lu_factor(sg_ctx* c, const float* A, int n, sg_precision prec) {
  LuCache& L = c->lu;
  if (L.n != n || L.prec != (int)prec || !L.exec) {
    L.clear();
    const int np = (n + sgk::kLuPanel - 1) / sgk::kLuPanel;
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t o2 = off;
      off = al(off + bytes);
      return o2;
    };
    const size_t o_lu = take((size_t)n * n * 4);
    const size_t o_piv = take((size_t)n * 4);
    const size_t o_perm = take((size_t)n * 4);
    const size_t o_inv = take(sgk::lu_diag_inv_bytes(n));
    const size_t o_info = take(64);
    const size_t o_moves = take((size_t)np * sgk::kLuMoveInts * 4 + (size_t)np * 4);
    const size_t o_gemm =
        take((prec == SG_PREC_F32_SIMT ? 0 : sgk::gemm_tc_scratch_bytes(n, n, sgk::kLuOuter)) + 256);
    if (cudaMalloc(&L.base, off) != cudaSuccess ||
        cudaStreamCreateWithFlags(&L.cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      L.clear();
      return err(c, SG_ERR_OOM, "factorisation workspace allocation failed");
    }
    char* base = static_cast<char*>(L.base);
    L.lu = reinterpret_cast<float*>(base + o_lu);
    L.piv = reinterpret_cast<int*>(base + o_piv);
    L.perm = reinterpret_cast<int*>(base + o_perm);
    L.inv = reinterpret_cast<float*>(base + o_inv);
    L.info = reinterpret_cast<int*>(base + o_info);
    int* moves = reinterpret_cast<int*>(base + o_moves);
    const int64_t k0 = c->kernels;
    cudaGraph_t g = nullptr;
    cudaError_t e = sgk::lu_prepare(n);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(L.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaMemsetAsync(L.info, 0, 64, L.cap);
      if (le == cudaSuccess)
        le = cudaMemsetAsync(moves, 0, (size_t)np * sgk::kLuMoveInts * 4 + (size_t)np * 4, L.cap);
      if (le == cudaSuccess) le = sgk::launch_lu_iota(L.perm, n, L.cap);
      if (le == cudaSuccess)
        le = factor_in_place(c, L.lu, n, L.piv, L.perm, L.info, moves,
                             reinterpret_cast<unsigned*>(moves + (size_t)np * sgk::kLuMoveInts),
                             base + o_gemm, prec, L.cap, nullptr);
      if (le == cudaSuccess) le = sgk::launch_lu_diag_inv(L.lu, n, L.inv, L.cap);
      if (le == cudaSuccess) c->kernels += 2;
      e = cudaStreamEndCapture(L.cap, &g);
      if (e == cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&L.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    L.kernels = c->kernels - k0;
    c->kernels = k0;
    if (e != cudaSuccess) {
      cudaGetLastError();
      L.clear();
      return err(c, SG_ERR_CUDA, "factorisation graph capture failed");
    }
    L.n = n;
    L.prec = (int)prec;
  }
  cudaError_t e = cudaMemcpyAsync(L.lu, A, (size_t)n * n * 4, cudaMemcpyDeviceToDevice, c->stream);
  sgk::prof_begin(&c->prof, "lu_factor_graph", c->stream);
  if (e == cudaSuccess) e = cudaGraphLaunch(L.exec, c->stream);
  sgk::prof_end(&c->prof, c->stream);
  c->kernels += L.kernels;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(c, SG_ERR_CUDA, cudaGetErrorString(e));
  }
  return SG_OK;
}

}  // namespace

extern "C" sg_status sg_solve(sg_ctx* c, sg_matrix* A, sg_vector* b, const sg_solve_opts* opts,
                              sg_vector** xout, sg_solve_info* info) {
  if (!c || !A || !b || !xout || !A->v || !b->v) return err(c, SG_ERR_INVALID_ARG, "bad solve arguments");
  if (c->planning_only) return err(c, SG_ERR_UNSUPPORTED, "planning-only context");
  const int64_t n64 = A->v->rows;
  if (A->v->cols != n64 || b->v->n != n64)
    return err(c, SG_ERR_SHAPE, "solve needs a square matrix and a right-hand side of its size");
  if (A->v->dt != SG_F32 || b->v->dt != SG_F64)
    return err(c, SG_ERR_DTYPE, "solve needs SG_F32 A and SG_F64 b");
  if (n64 > sgk::kLuMaxN) return err(c, SG_ERR_SHAPE, "solve supports n <= 9216");
  sg_solve_opts o{SG_PREC_BF16_TC, 30, 1e-14, 1e-12, 0};
  if (opts) {
    o = *opts;
    if (o.max_iter <= 0) o.max_iter = 30;
    if (o.refine_tol <= 0) o.refine_tol = 1e-14;
    if (o.residual_tol <= 0) o.residual_tol = 1e-12;
  }
  if (o.precision < SG_PREC_F32_SIMT || o.precision > SG_PREC_F16_TC)
    return err(c, SG_ERR_INVALID_ARG, "bad precision");
  // queued work that produces A or b runs first
  sg_status st = sg_flush(c);
  if (st && st != SG_ERR_PRECONDITION && st != SG_ERR_POSTCONDITION) return st;
  if (A->v->poisoned || b->v->poisoned) return err(c, SG_ERR_POISONED, "input depends on a failed contract");
  const int n = (int)n64;
  if (n == 0) {
    auto v = std::make_shared<Value>();
    v->dt = SG_F64;
    v->n = 0;
    v->rows = 0;
    v->st = std::make_shared<Storage>();
    auto* h = new sg_vector;
    h->ctx = c;
    h->v = v;
    v->handles = 1;
    *xout = h;
    if (info) *info = sg_solve_info{0, 0, 0.0, 0.0};
    return SG_OK;
  }
  const int nb = (n + 31) / 32;

  // workspace (one allocation, freed at the end of the call)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o2 = off;
    off = al(off + bytes);
    return o2;
  };
  const size_t o_y = take((size_t)n * 4);
  const size_t o_r = take((size_t)n * 8);
  const size_t o_flags = take((size_t)2 * nb * 4);
  const size_t o_tk = take(64);
  const size_t o_err = take(64);
  const size_t o_norms = take(8 * 8);
  const size_t o_viol = take(8);
  char* base = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&base, off, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(c, SG_ERR_OOM, "solve workspace allocation failed");
  }
  SolveWork w;
  w.y = reinterpret_cast<float*>(base + o_y);
  w.r = reinterpret_cast<double*>(base + o_r);
  w.flags = reinterpret_cast<unsigned*>(base + o_flags);
  w.tickets = reinterpret_cast<unsigned*>(base + o_tk);
  w.dev_err = reinterpret_cast<int*>(base + o_err);
  w.norms = reinterpret_cast<double*>(base + o_norms);
  w.viol = reinterpret_cast<unsigned long long*>(base + o_viol);

  // the solution vector (owned by the returned handle)
  auto xv = std::make_shared<Value>();
  xv->dt = SG_F64;
  xv->n = n;
  xv->rows = n;
  xv->st = std::make_shared<Storage>();
  xv->st->bytes = (size_t)n * 8;
  xv->st->stream = c->stream;
  e = cudaMallocAsync(&xv->st->ptr, xv->st->bytes, c->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFreeAsync(base, c->stream);
    return err(c, SG_ERR_OOM, "solution allocation failed");
  }
  xv->st->owned = true;
  double* x = static_cast<double*>(xv->st->ptr);
  join_transfers(c, A->v->st.get());
  join_transfers(c, b->v->st.get());
  const float* a = static_cast<const float*>(A->v->st->ptr);
  const double* bb = static_cast<const double*>(b->v->st->ptr);
  sgk::Prof* prof = &c->prof;
  cudaStream_t s = c->stream;

  sg_solve_info inf{0, 0, 0.0, 0.0};
  sg_status status = SG_OK;
  double hn[8];
  unsigned long long hviol = 0;
  int hinfo = 0, herr = 0;
  unsigned epoch = 0;
  auto sync_read = [&]() -> bool {
    e = cudaMemcpyAsync(hn, w.norms, sizeof hn, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w.dev_err, sizeof herr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hviol, w.viol, sizeof hviol, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess;
  };

  // 1. factorisation of a copy of A (the context's cached graph)
  e = cudaMemsetAsync(base + o_flags, 0, o_norms + 64 - o_flags, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(w.viol, 0, 8, s);
  if (e == cudaSuccess) e = sgk::launch_anorm(a, n, w.norms, s);
  if (e == cudaSuccess) {
    status = lu_factor(c, a, n, o.precision);
    if (status) {
      cudaFreeAsync(base, s);
      return status;
    }
  }
  w.lu = c->lu.lu;
  w.piv = c->lu.piv;
  w.info = c->lu.info;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hinfo, w.info, sizeof hinfo, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    status = err(c, SG_ERR_CUDA, cudaGetErrorString(e));
    cudaGetLastError();
  } else if (hinfo < 0) {
    status = err(c, SG_ERR_TIMEOUT, "panel exchange wait gave up");
  } else if (hinfo) {
    inf.info = hinfo;
    status = err(c, SG_ERR_SINGULAR, "exactly zero pivot");
  }

  // 2. initial solve, 3. refinement
  bool converged = false;
  if (!status) {
    e = sgk::launch_lu_solve(w.lu, c->lu.inv, n, c->lu.perm, bb, false, w.y, w.flags, ++epoch, w.tickets,
                             w.dev_err, s, prof);
    if (e == cudaSuccess) e = sgk::launch_update(x, w.y, bb, n, true, w.norms, s);
    c->kernels += 4;
    double prev = -1.0;
    for (int it = 0; it < o.max_iter && e == cudaSuccess; ++it) {
      e = cudaMemsetAsync(w.norms, 0, 3 * 8, s);
      if (e == cudaSuccess) e = sgk::launch_residual(a, n, bb, x, w.r, w.norms, 0.0, nullptr, s, prof);
      if (e == cudaSuccess)
        e = sgk::launch_lu_solve(w.lu, c->lu.inv, n, c->lu.perm, w.r, true, w.y, w.flags, ++epoch, w.tickets,
                                 w.dev_err, s, prof);
      if (e == cudaSuccess) e = sgk::launch_update(x, w.y, bb, n, false, w.norms, s);
      c->kernels += 5;
      if (e != cudaSuccess || !sync_read()) break;
      inf.iterations = it + 1;
      inf.last_correction = hn[2] > 0 ? hn[1] / hn[2] : hn[1];
      if (herr) break;
      if (inf.last_correction <= o.refine_tol) {
        converged = true;
        break;
      }
      if (prev >= 0.0 && inf.last_correction > 0.5 * prev) {
        converged = true;   // stagnated: no further accuracy to gain
        break;
      }
      prev = inf.last_correction;
    }
    if (e != cudaSuccess) {
      status = err(c, SG_ERR_CUDA, cudaGetErrorString(e));
      cudaGetLastError();
    } else if (herr) {
      status = err(c, SG_ERR_TIMEOUT, "triangular solve wait gave up");
    }
  }

  // 4. final residual and the postcondition
  if (!status) {
    // the bound needs |A|_inf (norms[3]), max|x| (norms[2]) and max|b| (norms[4])
    e = cudaMemsetAsync(w.norms, 0, 8, s);
    if (e == cudaSuccess && sync_read()) {
      const double denom = hn[3] * hn[2] + hn[4];
      const bool check = c->mode >= SG_CONTRACTS_PRE_POST;
      e = cudaMemsetAsync(w.viol, 0, 8, s);
      if (e == cudaSuccess)
        e = sgk::launch_residual(a, n, bb, x, w.r, w.norms, o.residual_tol * denom,
                                 check ? w.viol : nullptr, s, prof);
      c->kernels += 1;
      if (e == cudaSuccess && sync_read()) {
        inf.residual = denom > 0 ? hn[0] / denom : hn[0];
        if (!converged) {
          status = err(c, SG_ERR_NOT_CONVERGED, "refinement did not converge");
        } else if (check && hviol) {
          c->has_violation = true;
          c->last_violation.contract_id = -1;
          c->last_violation.role = SG_POST;
          c->last_violation.kind = SG_C_RESIDUAL;
          c->last_violation.op_id = -1;
          c->last_violation.first_index = (int64_t)~hviol;
          c->last_violation.observed = inf.residual;
          xv->poisoned = true;
          status = err(c, SG_ERR_POSTCONDITION, "residual postcondition failed");
        }
      }
    }
    if (e != cudaSuccess && !status) {
      status = err(c, SG_ERR_CUDA, cudaGetErrorString(e));
      cudaGetLastError();
    }
  }
  if (c->prof.on) c->prof.collect();
  cudaFreeAsync(base, s);
  if (info) *info = inf;
  if (status == SG_OK || status == SG_ERR_NOT_CONVERGED || status == SG_ERR_POSTCONDITION) {
    auto* h = new sg_vector;
    h->ctx = c;
    h->v = xv;
    xv->handles = 1;
    *xout = h;
  }
  return status;
}

extern "C" sg_status sg_det(sg_ctx* c, sg_matrix* A, sg_precision prec, sg_det_result* out) {
  if (!c || !A || !A->v || !out) return err(c, SG_ERR_INVALID_ARG, "bad det arguments");
  if (c->planning_only) return err(c, SG_ERR_UNSUPPORTED, "planning-only context");
  if (prec < SG_PREC_F32_SIMT || prec > SG_PREC_F16_TC)
    return err(c, SG_ERR_INVALID_ARG, "bad precision");
  const int64_t n64 = A->v->rows;
  if (A->v->cols != n64) return err(c, SG_ERR_SHAPE, "det needs a square matrix");
  if (A->v->dt != SG_F32) return err(c, SG_ERR_DTYPE, "det needs SG_F32");
  if (n64 > sgk::kLuMaxN) return err(c, SG_ERR_SHAPE, "det supports n <= 9216");
  sg_status st = sg_flush(c);
  if (st && st != SG_ERR_PRECONDITION && st != SG_ERR_POSTCONDITION) return st;
  if (A->v->poisoned) return err(c, SG_ERR_POISONED, "input depends on a failed contract");
  const int n = (int)n64;
  if (n == 0) {   // the empty product
    *out = sg_det_result{1, 0, 0.0, 1.0};
    return SG_OK;
  }
  cudaStream_t s = c->stream;
  double* dout = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&dout, 64, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(c, SG_ERR_OOM, "det workspace allocation failed");
  }
  join_transfers(c, A->v->st.get());
  sg_status st2 = lu_factor(c, static_cast<const float*>(A->v->st->ptr), n, prec);
  if (st2) {
    cudaFreeAsync(dout, s);
    return st2;
  }
  e = sgk::launch_lu_det(c->lu.lu, n, c->lu.piv, dout, s, &c->prof);
  c->kernels += 1;
  int* info = c->lu.info;
  double h[2] = {0.0, 0.0};
  int hinfo = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dout, sizeof h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hinfo, info, sizeof hinfo, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (c->prof.on) c->prof.collect();
  cudaFreeAsync(dout, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return err(c, SG_ERR_CUDA, cudaGetErrorString(e));
  }
  if (hinfo < 0) return err(c, SG_ERR_TIMEOUT, "panel exchange wait gave up");
  sg_det_result r;
  r.info = hinfo;
  if (hinfo) {   // the elimination stopped at an exactly zero pivot
    r.sign = 0;
    r.log_abs = -INFINITY;
    r.det = 0.0;
  } else {
    r.sign = (int32_t)h[0];
    r.log_abs = h[1];
    r.det = r.sign == 0 ? 0.0 : (double)r.sign * std::exp(h[1]);
  }
  *out = r;
  return SG_OK;
}

void LuCache::clear() {
  if (exec) cudaGraphExecDestroy(exec);
  if (base) cudaFree(base);
  if (cap) cudaStreamDestroy(cap);
  exec = nullptr;
  base = nullptr;
  cap = nullptr;
  lu = nullptr;
  piv = nullptr;
  perm = nullptr;
  inv = nullptr;
  info = nullptr;
  n = 0;
  prec = -1;
  kernels = 0;
}
