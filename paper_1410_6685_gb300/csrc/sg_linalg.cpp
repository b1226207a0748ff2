// sg_linalg.cpp -- matrix product and its Freivalds postcondition (Sec. 3.4
// `multiply`), dispatched from the executor.
#include "sg_plan.h"

size_t sg_linalg_scratch(sg_ctx*, Node*) { return 0; }

sg_status sg_exec_linalg(sg_ctx* c, Node*, void*, void*, cudaError_t*) {
  c->err = "matrix product not built yet";
  return SG_ERR_UNSUPPORTED;
}

bool sg_linalg_result(sg_ctx*, Node*, const void*, long long*, double*) { return false; }

extern "C" sg_status sg_solve(sg_ctx* c, sg_matrix*, sg_vector*, const sg_solve_opts*,
                              sg_vector**, sg_solve_info*) {
  if (c) c->err = "solve not built yet";
  return SG_ERR_UNSUPPORTED;
}

extern "C" sg_status sg_batch_run(sg_ctx* c, const sg_chain*, const float*, const int64_t*,
                                  int64_t, double*, int64_t*, int64_t*) {
  if (c) c->err = "batch not built yet";
  return SG_ERR_UNSUPPORTED;
}
