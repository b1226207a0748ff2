// sg_linalg.cpp -- matrix product (Sec. 3.4 `multiply`) and its Freivalds
// postcondition, dispatched from the executor.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sg_linalg_kernels.h"
#include "sg_plan.h"
#include "sg_runtime.h"
#include "sg_sched.h"

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

// The product's tile form (SG_SCHED_PRODUCT): 1 one CTA per 128 x 256
// tile, 2 a CTA pair per 256 x 256 tile.  Learned or autotuned; a sweep
// times both forms' products the first time (M, N, K, precision) is seen,
// unless the stream is being captured.
int product_form(sg_ctx* c, int M, int N, int K, bool fp16, const float* a, const float* b,
                 float* cc, void* work, cudaError_t* e) {
  const std::vector<sg_sched_choice> cand = sg_product_candidates(sgk::gemm_pair_available());
  if (cand.size() < 2 || M <= 0 || N <= 0 || K <= 0) return 0;
  const ProductWork w{M, N, K, fp16};
  std::vector<float> X(cand.size() * kSchedFeatures);
  const sg_sched_choice d = sg_product_default(true);
  int def = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    sg_product_features(w, cand[i], c->num_sms, &X[i * kSchedFeatures]);
    if (cand[i].chunk == d.chunk) def = (int)i;
  }
  const uint64_t key = sg_sched_key(SG_SCHED_PRODUCT, {(uint64_t)M, (uint64_t)N, (uint64_t)K,
                                                       (uint64_t)fp16});
  int learned = -1;
  std::vector<float> pred;
  std::vector<double> us;
  int idx = sg_sched_lookup(c, SG_SCHED_PRODUCT, key, X, def, &learned, &pred, &us);
  if (idx < 0) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      idx = def;
    } else {
      std::vector<int> forms;
      for (auto& ch : cand) forms.push_back(ch.blocks_per_sm == 2 ? 2 : 1);
      us.assign(cand.size(), 0.0);
      *e = sgk::time_gemm_forms(a, K, b, N, cc, N, M, N, K, fp16, work, c->stream, forms.data(),
                                (int)forms.size(), us.data(), &c->kernels);
      if (*e != cudaSuccess) return 0;
      idx = (int)(std::min_element(us.begin(), us.end()) - us.begin());
      sg_sched_log_sweep(c, SG_SCHED_PRODUCT, X, us, def);
      learned = sg_sched_learned_index(c, SG_SCHED_PRODUCT, X, def, &pred);
      sg_sched_set_tuned(c, SG_SCHED_PRODUCT, key, idx, us, learned);
    }
  }
  sg_sched_note(c, SG_SCHED_PRODUCT, cand, us, def, learned, idx, pred);
  return cand[idx].blocks_per_sm == 2 ? 2 : 1;
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
    const bool fp16 = n->prec == SG_PREC_F16_TC;
    const int form =
        n->prec == SG_PREC_F32_SIMT ? 0 : product_form(c, M, N, K, fp16, a, b, cc, work, e);
    if (*e != cudaSuccess) return SG_OK;
    if (fused) {
      *e = sgk::launch_gemm_tc_checked(a, b, cc, N, fp16, fused->seed, fused->nvec,
                                       (float)fused->tol, u_eff_for(n->prec, N), work,
                                       static_cast<sgk::FreivaldsResult*>(rec), c->stream,
                                       &c->prof, &c->kernels, ir, ic, id, form);
      return SG_OK;
    }
    if (n->prec == SG_PREC_F32_SIMT) {
      *e = sgk::launch_gemm_f32(a, K, b, N, cc, N, M, N, K, false, c->stream, &c->prof);
      c->kernels += 1;
    } else {
      *e = sgk::launch_gemm_tc(a, K, b, N, cc, N, M, N, K, fp16, false, work, c->stream,
                               &c->prof, &c->kernels, ir, ic, id, form);
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

