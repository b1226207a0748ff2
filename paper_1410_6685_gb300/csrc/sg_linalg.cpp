// sg_linalg.cpp -- matrix product (Sec. 3.4 `multiply`) and its Freivalds
// postcondition, dispatched from the executor.
#include <cmath>
#include <cstring>

#include "sg_linalg_kernels.h"
#include "sg_plan.h"
#include "sg_runtime.h"

namespace {

// effective unit roundoff of a product: operand rounding (two operands) plus
// binary32 accumulation over n terms
float u_eff_for(int prec, long long n) {
  const double acc = std::ldexp(1.0, -24) * std::sqrt((double)n);
  switch (prec) {
    case SG_PREC_BF16_TC: return (float)(std::ldexp(1.0, -8) + acc);
    case SG_PREC_F16_TC: return (float)(std::ldexp(1.0, -10) + acc);
    default: return (float)acc;
  }
}

}  // namespace

bool sg_linalg_can_fuse(const Node* mm, const Node* chk) {
  return mm->kind == NK::MATMUL && chk->kind == NK::CHECK && chk->ckind == SG_C_FREIVALDS &&
         mm->prec != SG_PREC_F32_SIMT && chk->nvec >= 1 && chk->nvec <= 4 &&
         mm->out.get() == chk->in[0].get() && mm->in[0].get() == chk->in[1].get() &&
         mm->in[1].get() == chk->in[2].get() && mm->in[0]->rows == mm->in[0]->cols &&
         mm->in[1]->rows == mm->in[1]->cols && mm->in[0]->rows == mm->in[1]->rows &&
         mm->in[0]->rows > 0;
}

size_t sg_linalg_scratch(sg_ctx*, Node* n, Node* fused) {
  if (n->kind == NK::MATMUL) {
    if (n->prec == SG_PREC_F32_SIMT) return 0;
    const size_t g = sgk::gemm_tc_scratch_bytes((int)n->in[0]->rows, (int)n->in[1]->cols,
                                                (int)n->in[0]->cols);
    return fused ? g + sgk::frv_fused_scratch_bytes((int)n->in[0]->rows) : g;
  }
  return sgk::freivalds_scratch_bytes((int)n->in[0]->rows, n->nvec);
}

sg_status sg_exec_linalg(sg_ctx* c, Node* n, Node* fused, void* rec, void* work, cudaError_t* e) {
  if (n->kind == NK::MATMUL) {
    Value* A = n->in[0].get();
    Value* B = n->in[1].get();
    Value* Cv = n->out.get();
    if (!Cv->st) {
      auto st = std::make_shared<Storage>();
      st->bytes = (size_t)Cv->n * 4;
      st->stream = c->stream;
      if (st->bytes) {
        cudaError_t ae = cudaMallocAsync(&st->ptr, st->bytes, c->stream);
        if (ae != cudaSuccess) {
          cudaGetLastError();
          c->err = "matrix allocation failed";
          return SG_ERR_OOM;
        }
        st->owned = true;
      }
      Cv->st = std::move(st);
    }
    const int M = (int)A->rows, K = (int)A->cols, N = (int)B->cols;
    const float* a = static_cast<const float*>(A->st->ptr);
    const float* b = static_cast<const float*>(B->st->ptr);
    float* cc = static_cast<float*>(Cv->st->ptr);
    // a planted element error (contract testing) goes to the next tc product
    const int ir = (int)c->mm_inject.row, ic = (int)c->mm_inject.col;
    const float id = c->mm_inject.delta;
    if (n->prec != SG_PREC_F32_SIMT) c->mm_inject.row = c->mm_inject.col = -1;
    if (fused) {
      *e = sgk::launch_gemm_tc_checked(a, b, cc, N, n->prec == SG_PREC_F16_TC, fused->seed,
                                       fused->nvec, (float)fused->tol, u_eff_for(n->prec, N),
                                       work, static_cast<sgk::FreivaldsResult*>(rec), c->stream,
                                       &c->prof, &c->kernels, ir, ic, id);
      return SG_OK;
    }
    if (n->prec == SG_PREC_F32_SIMT) {
      *e = sgk::launch_gemm_f32(a, K, b, N, cc, N, M, N, K, false, c->stream, &c->prof);
      c->kernels += 1;
    } else {
      *e = sgk::launch_gemm_tc(a, K, b, N, cc, N, M, N, K, n->prec == SG_PREC_F16_TC, false,
                               work, c->stream, &c->prof, &c->kernels, ir, ic, id);
    }
    return SG_OK;
  }
  // Freivalds: in[0] = C (target), in[1] = A, in[2] = B
  const int N = (int)n->in[0]->rows;
  // the precision of the product that produced C, when the check is built in
  const int prec = n->in[0]->producer && n->in[0]->producer->kind == NK::MATMUL
                       ? n->in[0]->producer->prec
                       : n->prec;
  *e = sgk::launch_freivalds(static_cast<const float*>(n->in[1]->st->ptr),
                             static_cast<const float*>(n->in[2]->st->ptr),
                             static_cast<const float*>(n->in[0]->st->ptr), N, n->seed, n->nvec,
                             (float)n->tol, u_eff_for(prec, N), work,
                             static_cast<sgk::FreivaldsResult*>(rec), c->stream, &c->prof,
                             &c->kernels);
  return SG_OK;
}

bool sg_linalg_result(sg_ctx*, Node* n, Node* fused, const void* rec, long long* row,
                      double* observed) {
  if (n->kind != NK::CHECK && !fused) return false;
  sgk::FreivaldsResult r;
  memcpy(&r, rec, sizeof r);
  *observed = r.max_ratio;
  if (!r.viol_enc) return false;
  *row = (long long)~r.viol_enc;
  return true;
}

