// sg_plan.h -- the optimizer (Sec. 5) and executor of the deferred queue.
#pragma once
#include <string>

#include "sg_runtime.h"

// Plans, launches and post-processes every queued node of the context, then
// clears the queue.  Returns the first failure (a CUDA error, a timeout, or
// the role of the first violated contract).
sg_status sg_execute_pending(sg_ctx* c);

// One line per kernel (group) that sg_execute_pending would launch now.
sg_status sg_describe_pending(sg_ctx* c, std::string* out);

// Matrix product and Freivalds check kernels (sg_linalg.cpp).
// fused: a built-in Freivalds check folded into the product `n` (or nullptr)
size_t sg_linalg_scratch(sg_ctx* c, Node* n, Node* fused);
sg_status sg_exec_linalg(sg_ctx* c, Node* n, Node* fused, void* rec, void* work, cudaError_t* e);
// a product whose Freivalds check can be folded into it
bool sg_linalg_can_fuse(const Node* mm, const Node* chk);
// True when the node's check failed; fills the violating row and the
// observed |z_i - w_i| / tau_i.
bool sg_linalg_result(sg_ctx* c, Node* n, Node* fused, const void* rec, long long* row,
                      double* observed);
