// sg_plan.cpp -- the optimizer and executor of the deferred queue (Sec. 5).
//
// The queue of one context is a DAG of data nodes (values) and kernel nodes
// (the queued calls), in a valid topological order.  The optimizer walks it
// in order and merges element-wise calls over collections of one count into
// passes of the fused streaming kernel:
//   * map chains become one expression (Fig. 3: X[i]+Y[i] -> a*X[i]+Y[i]):
//     a value produced earlier in the pass is substituted into its consumer;
//   * a map and the reduction that consumes it share the pass (Fig. 2);
//   * for_all / exists queries and range contracts on values of the pass are
//     evaluated in the same pass (Sec. 4, range contracts on the device);
//   * a filter whose result is only summed becomes a masked reduction, so
//     the filtered collection is never built;
//   * an intermediate is written to memory only if a handle still refers to
//     it or a later pass needs it ("collapsing intermediate dependencies").
// Sort, filter, matrix product and their contracts become their own kernel
// groups; the sort's built-in postconditions ride in its last pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <string>

#include "sg_internal.h"
#include "sg_jit.h"
#include "sg_linalg_kernels.h"
#include "sg_plan.h"
#include "sg_sched.h"

namespace {

using sgk::Prog;

struct Op {
  uint8_t op;
  int8_t arg;
  float cst;
};

enum class PK { STREAM, FILTER, SORT, CHECK_SORTED, CHECK_PERM, MATMUL, FREIVALDS, TRANSPOSE, MATVEC,
                CONCAT, FPRINT, CHECK_SAME };

// bytes of a value, and the unit its fingerprint reads (2 for bf16 / fp16)
size_t value_bytes(const Value* v) {
  const size_t es = (v->dt == SG_F64 || v->dt == SG_I64) ? 8
                    : (v->dt == SG_BF16 || v->dt == SG_F16) ? 2 : 4;
  return (size_t)v->n * es;
}
int fprint_unit(const Value* v) { return (v->dt == SG_BF16 || v->dt == SG_F16) ? 2 : 4; }

struct Pass {
  PK kind = PK::STREAM;
  int64_t n = 0;
  std::vector<Node*> nodes;
  // STREAM
  std::vector<Value*> inputs;                  // loaded values, slot = index
  std::map<Value*, std::vector<Op>> inl;       // values produced in the pass
  std::map<Value*, std::vector<Op>> mask;      // masked (filtered) values
  std::map<Value*, Value*> mask_base;          // masked value -> filtered input
  std::vector<Value*> stores;                  // materialised outputs
  std::vector<Op> prog;
  std::vector<Node*> preds;                    // slot = index
  Value* reduce_of = nullptr;
  std::vector<Node*> reduces;
  int est_ops = 0;
  int depth = 0;
  // SORT (+ its fused checks), FILTER, CHECK_*, MATMUL, FREIVALDS
  Node* main = nullptr;
  Node* chk_sorted = nullptr;
  Node* chk_perm = nullptr;
  Node* chk_frv = nullptr;    // MATMUL: built-in Freivalds check folded in
  Node* chk_post = nullptr;   // FILTER: a for_all postcondition on its result folded in
  Node* vtrans = nullptr;     // MATVEC y = A x with A the pending transpose of vtrans->in[0]
  // STREAM over a compacted filter's result of the same flush: that filter,
  // whose count (on the device) bounds the pass
  Node* count_src = nullptr;
};

bool is_f32_stream_node(const Node* n) {
  switch (n->kind) {
    case NK::MAP:
    case NK::REDUCE:
    case NK::QUANT:
      return true;
    case NK::CHECK:
      return n->ckind == SG_C_FOR_ALL || n->ckind == SG_C_EXISTS;
    default:
      return false;
  }
}

int64_t node_len(const Node* n) { return n->in[0] ? n->in[0]->n : 0; }

// Depth bookkeeping of a finished program: depth before each op, max depth.
bool program_depths(const std::vector<Op>& ops, std::vector<uint8_t>* before, int* maxd) {
  int d = 0, mx = 0;
  if (before) before->clear();
  for (const Op& o : ops) {
    if (before) before->push_back((uint8_t)d);
    int need = 0, delta = 0;
    switch (o.op) {
      case SG_OP_LOAD: case SG_OP_CONST: case SG_OP_INDEX: delta = 1; break;
      case SG_OP_FMA: case SG_OP_SELECT: need = 3; delta = -2; break;
      case SG_OP_NEG: case SG_OP_ABS: case SG_OP_SQRT: case SG_OP_NOT: need = 1; break;
      case SG_OP_DUP: need = 1; delta = 1; break;
      case SG_OP_SWAP: need = 2; break;
      case sgk::K_STORE: need = 1; break;
      case sgk::K_PRED: case sgk::K_MASK: case sgk::K_REDUCE: case sgk::K_POP:
        need = 1; delta = -1; break;
      default: need = 2; delta = -1; break;   // binary arithmetic / comparison
    }
    if (d < need) return false;
    d += delta;
    mx = std::max(mx, d);
  }
  if (d != 0) return false;
  *maxd = mx;
  return mx <= sgk::kMaxDepth;
}

// The program of an element-wise expression whose value is read off the
// stack (a filter predicate, a contract): depths are computed with a trailing
// pop that is not part of the program.
sgk::Prog value_prog(const sg_expr& ex, int* max_depth = nullptr) {
  sgk::Prog pr{};
  std::vector<Op> ops;
  for (int p = 0; p < ex.nops; ++p) ops.push_back(Op{(uint8_t)ex.ops[p].op, 0, ex.ops[p].value});
  ops.push_back(Op{sgk::K_POP, 0, 0.0f});
  std::vector<uint8_t> before;
  int md = 0;
  program_depths(ops, &before, &md);
  ops.pop_back();
  pr.nops = (int)ops.size();
  for (size_t p = 0; p < ops.size(); ++p) {
    pr.op[p] = ops[p].op;
    pr.arg[p] = ops[p].arg;
    pr.cst[p] = ops[p].cst;
    pr.depth[p] = before[p];
  }
  if (max_depth) *max_depth = md;
  return pr;
}

struct Planner {
  sg_ctx* c;
  bool fuse;                    // merge passes (Sec. 5), else one pass per call
  std::vector<Node*> nodes;
  std::set<Node*> unmaskable;   // filters that must be compacted
  std::vector<Pass> passes;
  std::map<Value*, std::vector<Node*>> consumers;

  explicit Planner(sg_ctx* ctx) : Planner(ctx, ctx->fusion == SG_FUSE_ON) {}
  Planner(sg_ctx* ctx, bool f) : c(ctx), fuse(f) {
    for (auto& n : c->pending) nodes.push_back(n.get());
    for (Node* n : nodes)
      for (int k = 0; k < n->nin; ++k)
        if (n->in[k]) consumers[n->in[k].get()].push_back(n);
  }

  // A filter can become a mask when only reductions consume its result and
  // no handle refers to it.
  bool maskable(Node* f) {
    if (!fuse || unmaskable.count(f)) return false;
    Value* y = f->out.get();
    if (y->handles > 0) return false;
    auto it = consumers.find(y);
    if (it == consumers.end()) return true;
    for (Node* u : it->second)
      if (u->kind != NK::REDUCE) return false;
    return true;
  }

  // A for_all postcondition whose only operand is the compacted result of a
  // filter of this plan is checked by the specialised filter on each kept
  // item as it is written (no pass over the result): the filter's pass.
  int post_fold_target(Node* n) {
    if (!fuse || c->codegen != SG_CODEGEN_SPECIALIZE || !sgk::jit_available()) return -1;
    if (n->kind != NK::CHECK || n->ckind != SG_C_FOR_ALL || n->nin != 1 || !n->in[0]) return -1;
    Node* f = n->in[0]->producer;
    if (!f || f->kind != NK::FILTER || n->in[0]->dt != SG_F32) return -1;
    for (int p = 0; p < n->expr.nops; ++p)
      if (n->expr.ops[p].op == SG_OP_LOAD && n->expr.ops[p].arg != 0) return -1;
    if (f->expr.nops + 1 + n->expr.nops + 1 > sgk::kMaxProg) return -1;
    for (size_t i = passes.size(); i-- > 0;) {
      const Pass& P = passes[i];
      if (P.kind == PK::FILTER && P.main == f) return P.chk_post ? -1 : (int)i;
    }
    return -1;
  }

  bool dead(Node* n) {
    // a map / transpose / product whose result nobody will ever see is not computed
    const bool pure = (n->kind == NK::MAP && !n->inplace) || n->kind == NK::TRANSPOSE ||
                      n->kind == NK::MATVEC || n->kind == NK::CONCAT;
    if (!pure) return false;
    Value* v = n->out.get();
    return v->handles == 0 && consumers.find(v) == consumers.end();
  }

  // A transpose that only right-multiplies vectors (and has no handle) is
  // never materialised: y = A^T x is computed as x^T A on the source.
  std::set<Node*> virtual_t;
  bool virtual_transpose(Node* n) {
    if (!fuse || n->kind != NK::TRANSPOSE) return false;
    Value* v = n->out.get();
    if (v->handles > 0) return false;
    auto it = consumers.find(v);
    if (it == consumers.end()) return false;
    for (Node* u : it->second)
      if (u->kind != NK::MATVEC || u->left || u->in[0].get() != v || u->in[1].get() == v)
        return false;
    return true;
  }

  // the filter whose compacted result (count not yet known) node n reads,
  // when that filter runs as its own pass earlier in this plan
  Node* counted_source(const Node* n) const {
    for (int k = 0; k < n->nin; ++k) {
      const Value* v = n->in[k].get();
      if (!v || v->count_known || !v->producer || v->producer->kind != NK::FILTER) continue;
      for (const Pass& Q : passes)
        if (Q.kind == PK::FILTER && Q.main == v->producer) return v->producer;
    }
    return nullptr;
  }

  int slot_of(Pass& P, Value* v, bool add) {
    for (size_t i = 0; i < P.inputs.size(); ++i)
      if (P.inputs[i] == v) return (int)i;
    if (!add || P.inputs.size() >= (size_t)sgk::kMaxIn) return -1;
    P.inputs.push_back(v);
    return (int)P.inputs.size() - 1;
  }

  // Ops computing value v inside pass P (a load, or the substituted
  // expression of a value produced earlier in P).
  bool value_ops(Pass& P, Value* v, std::vector<Op>* out) {
    if (P.mask.count(v)) return false;   // a masked value is only reducible
    auto it = P.inl.find(v);
    if (it != P.inl.end()) {
      out->insert(out->end(), it->second.begin(), it->second.end());
      return true;
    }
    int s = slot_of(P, v, true);
    if (s < 0) return false;
    out->push_back(Op{SG_OP_LOAD, (int8_t)s, 0.0f});
    return true;
  }

  bool expand(Pass& P, const sg_expr& e, Node* n, std::vector<Op>* out) {
    for (int p = 0; p < e.nops; ++p) {
      const sg_expr_op& o = e.ops[p];
      if (o.op == SG_OP_LOAD) {
        if (!value_ops(P, n->in[o.arg].get(), out)) return false;
      } else {
        out->push_back(Op{(uint8_t)o.op, 0, o.value});
      }
    }
    return true;
  }

  // Try to add node n to the open stream pass; all-or-nothing.
  bool try_add(Pass& P, Node* n) {
    // memory written in place earlier in this pass is only read through the
    // written value itself (a subset view of it starts a new pass)
    for (Node* m : P.nodes) {
      if (!m->inplace) continue;
      for (int k = 0; k < n->nin; ++k) {
        Value* v = n->in[k].get();
        if (v && v != m->out.get() && v != m->in[0].get() &&
            storage_related(v->st.get(), m->out->st.get()))
          return false;
      }
    }
    Pass T = P;   // tentative copy (small)
    std::vector<Op> ops;
    int extra = 0;
    switch (n->kind) {
      case NK::MAP: {
        if (!expand(T, n->expr, n, &ops)) return false;
        extra = 2;   // a possible STORE + POP
        T.inl[n->out.get()] = ops;
        break;
      }
      case NK::FILTER: {
        // masked value: y = x where pred(x)
        std::vector<Op> xo, mo;
        Value* x = n->in[0].get();
        if (!value_ops(T, x, &xo)) return false;
        for (int p = 0; p < n->expr.nops; ++p) {
          const sg_expr_op& o = n->expr.ops[p];
          if (o.op == SG_OP_LOAD) mo.insert(mo.end(), xo.begin(), xo.end());
          else mo.push_back(Op{(uint8_t)o.op, 0, o.value});
        }
        T.mask[n->out.get()] = mo;
        T.inl[n->out.get()] = xo;
        ops = {};
        break;
      }
      case NK::REDUCE: {
        Value* v = n->in[0].get();
        if (T.reduce_of && T.reduce_of != v) return false;
        if (!T.reduce_of) {
          std::vector<Op> r;
          auto mk = T.mask.find(v);
          if (mk != T.mask.end()) {
            r = mk->second;
            r.push_back(Op{sgk::K_MASK, 0, 0.0f});
            auto vi = T.inl.find(v);
            r.insert(r.end(), vi->second.begin(), vi->second.end());
          } else if (!value_ops(T, v, &r)) {
            return false;
          }
          r.push_back(Op{sgk::K_REDUCE, 0, 0.0f});
          ops = r;
          T.reduce_of = v;
        }
        T.reduces.push_back(n);
        break;
      }
      case NK::QUANT:
      case NK::CHECK: {
        if ((int)T.preds.size() >= sgk::kMaxPred) return false;
        if (!expand(T, n->expr, n, &ops)) return false;
        ops.push_back(Op{sgk::K_PRED, (int8_t)T.preds.size(), 0.0f});
        T.preds.push_back(n);
        break;
      }
      default:
        return false;
    }
    if (T.est_ops + (int)ops.size() + extra > sgk::kMaxProg) return false;
    if (n->kind != NK::MAP && n->kind != NK::FILTER) {
      int d = 0;
      std::vector<Op> chk = ops;
      if (!program_depths(chk, nullptr, &d)) return false;
    } else if (n->kind == NK::MAP) {
      std::vector<Op> chk = T.inl[n->out.get()];
      chk.push_back(Op{sgk::K_POP, 0, 0.0f});
      int d = 0;
      if (!program_depths(chk, nullptr, &d)) return false;
    }
    T.est_ops += (int)ops.size() + extra;
    T.nodes.push_back(n);
    P = std::move(T);
    return true;
  }

  void group() {
    passes.clear();
    virtual_t.clear();
    bool open = false;
    for (Node* n : nodes) {
      if (dead(n)) continue;
      const int pf = post_fold_target(n);
      if (pf >= 0) {
        passes[pf].chk_post = n;
        passes[pf].nodes.push_back(n);
        continue;
      }
      const bool streamable = is_f32_stream_node(n) || (n->kind == NK::FILTER && maskable(n));
      if (streamable) {
        const int64_t len = node_len(n);
        // a reduction over a compacted filter's result of this flush covers
        // the filter's count, known only on the device: a pass of its own
        Node* csrc = counted_source(n);
        if (!csrc && open && fuse && passes.back().n == len && !passes.back().count_src &&
            try_add(passes.back(), n))
          continue;
        Pass P;
        P.kind = PK::STREAM;
        P.n = len;
        P.count_src = csrc;
        if (!try_add(P, n)) {
          // cannot fail for a lone node with loaded inputs unless the node
          // consumes a masked value produced in a closed pass
          if (n->kind == NK::REDUCE) unmaskable.insert(n->in[0]->producer);
          P = Pass{};
          P.kind = PK::STREAM;
          P.n = len;
          try_add(P, n);
        }
        passes.push_back(std::move(P));
        open = csrc == nullptr;
        continue;
      }
      open = false;
      Pass P;
      P.n = node_len(n);
      P.main = n;
      P.nodes.push_back(n);
      switch (n->kind) {
        case NK::FILTER: P.kind = PK::FILTER; break;
        case NK::SORT: P.kind = PK::SORT; break;
        case NK::MATMUL: P.kind = PK::MATMUL; break;
        case NK::TRANSPOSE:
          if (virtual_transpose(n)) {
            virtual_t.insert(n);
            continue;
          }
          P.kind = PK::TRANSPOSE;
          break;
        case NK::CONCAT: P.kind = PK::CONCAT; break;
        case NK::SNAPSHOT: P.kind = PK::FPRINT; break;
        case NK::MATVEC:
          P.kind = PK::MATVEC;
          if (!n->left && n->in[0]->producer && virtual_t.count(n->in[0]->producer))
            P.vtrans = n->in[0]->producer;
          break;
        case NK::CHECK:
          if (n->ckind == SG_C_SORTED) {
            // fuse into the sort that produced the checked value
            if (fuse && !passes.empty() && passes.back().kind == PK::SORT &&
                passes.back().main->out.get() == n->in[0].get() && !passes.back().chk_sorted) {
              passes.back().chk_sorted = n;
              passes.back().nodes.push_back(n);
              continue;
            }
            P.kind = PK::CHECK_SORTED;
          } else if (n->ckind == SG_C_PERMUTATION) {
            if (fuse && !passes.empty() && passes.back().kind == PK::SORT &&
                passes.back().main->out.get() == n->in[0].get() &&
                passes.back().main->in[0].get() == n->in[1].get() && !passes.back().chk_perm) {
              passes.back().chk_perm = n;
              passes.back().nodes.push_back(n);
              continue;
            }
            P.kind = PK::CHECK_PERM;
          } else if (n->ckind == SG_C_UNCHANGED) {
            P.kind = PK::CHECK_SAME;
          } else {
            // fold into the tensor-core product that produced the checked value
            if (fuse && !passes.empty() && passes.back().kind == PK::MATMUL &&
                !passes.back().chk_frv && sg_linalg_can_fuse(passes.back().main, n)) {
              passes.back().chk_frv = n;
              passes.back().nodes.push_back(n);
              continue;
            }
            P.kind = PK::FREIVALDS;
          }
          break;
        default:
          break;
      }
      passes.push_back(std::move(P));
    }
  }

  // Masked filters whose reductions ended up in another pass are compacted.
  bool validate() {
    bool ok = true;
    for (Pass& P : passes) {
      if (P.kind != PK::STREAM) continue;
      for (auto& kv : P.mask) {
        Value* y = kv.first;
        for (Node* u : consumers[y]) {
          if (std::find(P.nodes.begin(), P.nodes.end(), u) == P.nodes.end()) {
            unmaskable.insert(y->producer);
            ok = false;
          }
        }
      }
    }
    return ok;
  }

  int pass_of_node(Node* n) {
    for (size_t i = 0; i < passes.size(); ++i)
      if (std::find(passes[i].nodes.begin(), passes[i].nodes.end(), n) != passes[i].nodes.end())
        return (int)i;
    return -1;
  }

  bool must_store(const Pass& P, Node* n) {
    Value* v = n->out.get();
    if (n->inplace || v->handles > 0) return true;
    for (Node* u : consumers[v])
      if (std::find(P.nodes.begin(), P.nodes.end(), u) == P.nodes.end()) return true;
    return false;
  }

  // Emit the program of every stream pass (after grouping is final).
  void emit() {
    for (Pass& P : passes) {
      if (P.kind != PK::STREAM) continue;
      // rebuild inline expressions in node order and emit ops
      Pass E;
      E.kind = PK::STREAM;
      E.n = P.n;
      E.count_src = P.count_src;
      E.nodes = P.nodes;
      for (Node* n : P.nodes) {
        switch (n->kind) {
          case NK::MAP: {
            std::vector<Op> ops;
            expand(E, n->expr, n, &ops);
            E.inl[n->out.get()] = ops;
            if (must_store(P, n)) {
              int slot = (int)E.stores.size();
              E.stores.push_back(n->out.get());
              E.prog.insert(E.prog.end(), ops.begin(), ops.end());
              E.prog.push_back(Op{sgk::K_STORE, (int8_t)slot, 0.0f});
              E.prog.push_back(Op{sgk::K_POP, 0, 0.0f});
            }
            break;
          }
          case NK::FILTER: {
            std::vector<Op> xo, mo;
            value_ops(E, n->in[0].get(), &xo);
            for (int p = 0; p < n->expr.nops; ++p) {
              const sg_expr_op& o = n->expr.ops[p];
              if (o.op == SG_OP_LOAD) mo.insert(mo.end(), xo.begin(), xo.end());
              else mo.push_back(Op{(uint8_t)o.op, 0, o.value});
            }
            E.mask[n->out.get()] = mo;
            E.inl[n->out.get()] = xo;
            break;
          }
          case NK::REDUCE: {
            Value* v = n->in[0].get();
            E.reduces.push_back(n);
            if (E.reduce_of) break;
            E.reduce_of = v;
            auto mk = E.mask.find(v);
            if (mk != E.mask.end()) {
              E.prog.insert(E.prog.end(), mk->second.begin(), mk->second.end());
              E.prog.push_back(Op{sgk::K_MASK, 0, 0.0f});
              auto& vi = E.inl[v];
              E.prog.insert(E.prog.end(), vi.begin(), vi.end());
            } else {
              value_ops(E, v, &E.prog);
            }
            E.prog.push_back(Op{sgk::K_REDUCE, 0, 0.0f});
            break;
          }
          default: {  // QUANT / CHECK
            std::vector<Op> ops;
            expand(E, n->expr, n, &ops);
            E.prog.insert(E.prog.end(), ops.begin(), ops.end());
            E.prog.push_back(Op{sgk::K_PRED, (int8_t)E.preds.size(), 0.0f});
            E.preds.push_back(n);
            break;
          }
        }
      }
      program_depths(E.prog, nullptr, &E.depth);
      P = std::move(E);
    }
  }

  void plan() {
    for (int it = 0; it < 8; ++it) {
      group();
      if (validate()) break;
    }
    emit();
  }
};


// ---------------------------------------------------------------------------
// execution

constexpr int kStreamBlock = 256;
constexpr long long kNone = 0x7fffffffffffffffLL;

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

sg_status cuda_fail(sg_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  c->err = buf;
  return SG_ERR_CUDA;
}

sg_status ensure_storage(sg_ctx* c, Value* v) {
  if (v->st) return SG_OK;
  size_t es = (v->dt == SG_F64 || v->dt == SG_I64) ? 8 : (v->dt == SG_BF16 || v->dt == SG_F16) ? 2 : 4;
  auto st = std::make_shared<Storage>();
  st->bytes = (size_t)v->n * es;
  st->stream = c->stream;
  if (st->bytes) {
    cudaError_t e = cudaMallocAsync(&st->ptr, st->bytes, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "output allocation");
    st->owned = true;
  }
  v->st = std::move(st);
  return SG_OK;
}

sg_status ensure_scratch(sg_ctx* c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return SG_OK;
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream sync");
  if (c->scratch) cudaFree(c->scratch);
  c->scratch = nullptr;
  c->scratch_bytes = 0;
  size_t nb = round_up(std::max(bytes, (size_t)1 << 20), (size_t)1 << 20);
  e = cudaMalloc(&c->scratch, nb);
  if (e != cudaSuccess) return cuda_fail(c, e, "scratch allocation");
  c->scratch_bytes = nb;
  return SG_OK;
}

sg_status ensure_host_res(sg_ctx* c, size_t bytes) {
  if (c->host_res_bytes >= bytes) return SG_OK;
  if (c->host_res) cudaFreeHost(c->host_res);
  c->host_res = nullptr;
  size_t nb = round_up(std::max(bytes, (size_t)4096), 4096);
  cudaError_t e = cudaMallocHost(&c->host_res, nb);
  if (e != cudaSuccess) return cuda_fail(c, e, "pinned result buffer");
  c->host_res_bytes = nb;
  // with unified addressing the pinned buffer has the same address on the
  // device, so a kernel can store the results into it: the flush does so
  // while a large asynchronous read of another value is on the copy engine
  // (a copy would queue behind it)
  cudaPointerAttributes a{};
  c->host_res_mapped = cudaPointerGetAttributes(&a, c->host_res) == cudaSuccess &&
                       a.devicePointer == c->host_res;
  cudaGetLastError();
  return SG_OK;
}

int stream_grid(sg_ctx* c, const Pass& P) {
  const long long units = std::max<long long>(1, (P.n + 3) / 4);
  const long long want = (units + kStreamBlock - 1) / kStreamBlock;
  const int occ = sgk::stream_max_blocks_per_sm((int)P.inputs.size(), P.depth, kStreamBlock);
  const long long cap = (long long)c->num_sms * occ;
  return (int)std::max<long long>(1, std::min(want, cap));
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

void record_violation(sg_ctx* c, Node* n, int64_t first, double observed, bool* have,
                      sg_status* status) {
  n->failed = true;
  n->first = first;
  n->observed = observed;
  if (*have) return;
  *have = true;
  c->has_violation = true;
  c->last_violation.contract_id = n->builtin ? -1 : n->cid;
  c->last_violation.role = n->role;
  c->last_violation.kind = n->ckind;
  c->last_violation.op_id = n->in[0] && n->in[0]->producer ? n->in[0]->producer->id : -1;
  c->last_violation.first_index = first;
  c->last_violation.observed = observed;
  *status = n->role == SG_PRE ? SG_ERR_PRECONDITION : SG_ERR_POSTCONDITION;
}

// One launch's time: a warm-up, then the better of two runs (CUDA events on
// the context's stream; waits for it).  A launch shorter than 16 us is
// repeated within each timed run (up to 64 times) and the run divided: the
// events resolve about half a microsecond, too coarse for one short launch.
template <class F>
cudaError_t time_launch(sg_ctx* c, F&& launch, double* us) {
  cudaEvent_t ev[2] = {nullptr, nullptr};
  cudaError_t e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  double best = 1e300;
  int reps = 1;
  for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
    e = cudaEventRecord(ev[0], c->stream);
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    const double t = 1000.0 * ms / reps;
    if (r == 0)
      reps = t >= 16.0 ? 1 : (int)std::min(64.0, std::ceil(16.0 / std::max(t, 0.25)));
    else
      best = std::min(best, t);
  }
  for (cudaEvent_t v : ev)
    if (v) cudaEventDestroy(v);
  *us = best;
  return e;
}

// a sweep would wait for the stream: not while it is being captured
bool stream_capturing(sg_ctx* c) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + bytes && y < x + bytes;
}

// the structure of a program (operators, operand slots, depths), not its
// constants
uint64_t prog_shape(const sgk::Prog& pr) {
  uint64_t h = 1469598103934665603ull;
  for (int p = 0; p < pr.nops; ++p) {
    h = (h ^ pr.op[p]) * 1099511628211ull;
    h = (h ^ pr.arg[p]) * 1099511628211ull;
    h = (h ^ pr.depth[p]) * 1099511628211ull;
  }
  return h;
}

// The launch shape of a specialised stream pass (SG_SCHED_STREAM): learned,
// autotuned (a sweep the first time the workload is seen, unless the pass
// writes over one of its inputs or the stream is being captured), else the
// plain table's.
cudaError_t launch_stream_scheduled(sg_ctx* c, cudaKernel_t jk, const sgk::StreamArgs& a,
                                    int nout, bool minmax) {
  StreamWork w;
  w.n = a.n;
  w.nin = a.nin;
  w.nout = nout;
  w.ops = a.prog.nops;
  w.depth = a.depth;
  w.npred = a.npred;
  w.reduce = a.has_reduce != 0;
  w.minmax = minmax;
  w.vec4 = a.vec4 != 0;
  const std::vector<sg_sched_choice> cand = sg_stream_candidates(w.n, c->num_sms);
  const sg_sched_choice d = sg_stream_default();
  const int gd = sg_stream_grid(w.n, d, c->num_sms);
  std::vector<float> X(cand.size() * kSchedFeatures);
  int def = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    sg_stream_features(w, cand[i], c->num_sms, &X[i * kSchedFeatures]);
    if (def < 0 && cand[i].chunk == d.chunk && sg_stream_grid(w.n, cand[i], c->num_sms) == gd)
      def = (int)i;
  }
  if (def < 0) def = 0;
  const uint64_t key =
      sg_sched_key(SG_SCHED_STREAM, {(uint64_t)w.n, prog_shape(a.prog), (uint64_t)w.nin,
                                     (uint64_t)w.nout, (uint64_t)w.npred, a.pred_exists,
                                     (uint64_t)(w.reduce + 2 * w.minmax + 4 * w.vec4)});
  int learned = -1;
  std::vector<float> pred;
  std::vector<double> us;
  int idx = sg_sched_lookup(c, SG_SCHED_STREAM, key, X, def, &learned, &pred, &us);
  cudaError_t e = cudaSuccess;
  if (idx < 0) {
    bool in_place = false;
    for (int k = 0; k < a.nin; ++k)
      for (int o = 0; o < nout; ++o)
        in_place |= ranges_overlap(a.in[k], a.out[o], (size_t)w.n * 4);
    if (in_place || cand.size() < 2 || stream_capturing(c)) {
      idx = def;
    } else {
      us.assign(cand.size(), 0.0);
      for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
        const int g = sg_stream_grid(w.n, cand[i], c->num_sms), b = (int)cand[i].chunk;
        e = time_launch(c,
                        [&]() {
                          c->kernels += 1;
                          return sgk::launch_jit_stream(jk, a, g, b, c->stream, nullptr);
                        },
                        &us[i]);
      }
      if (e != cudaSuccess) return e;
      idx = (int)(std::min_element(us.begin(), us.end()) - us.begin());
      sg_sched_log_sweep(c, SG_SCHED_STREAM, X, us, def);
      learned = sg_sched_learned_index(c, SG_SCHED_STREAM, X, def, &pred);
      sg_sched_set_tuned(c, SG_SCHED_STREAM, key, idx, us, learned);
    }
  }
  sg_sched_note(c, SG_SCHED_STREAM, cand, us, def, learned, idx, pred);
  return sgk::launch_jit_stream(jk, a, sg_stream_grid(w.n, cand[idx], c->num_sms),
                                (int)cand[idx].chunk, c->stream, &c->prof);
}

// The tile of the specialised filter (SG_SCHED_FILTER): learned, autotuned
// (a sweep the first time the length and predicate shape are seen, unless
// the look-back testing controls are set or the stream is being captured),
// else the plain table's 8192 items.  *ran is false when no specialised
// kernel could be built (the caller interprets).
cudaError_t launch_filter_scheduled(sg_ctx* c, const sgk::Prog& pr, const float* x, float* out,
                                    long long n, void* dwork, sgk::FilterResult* rec, bool* ran,
                                    const sgk::Prog* post) {
  *ran = false;
  const std::vector<sg_sched_choice> cand = sg_filter_candidates();
  const sg_sched_choice d = sg_filter_default();
  FilterWork w;
  w.n = n;
  w.ops = pr.nops;
  std::vector<float> X(cand.size() * kSchedFeatures);
  int def = 0;
  for (size_t i = 0; i < cand.size(); ++i) {
    sg_filter_features(w, cand[i], sgk::filter_tile_occupancy((int)cand[i].chunk), c->num_sms,
                       &X[i * kSchedFeatures]);
    if (cand[i].chunk == d.chunk) def = (int)i;
  }
  const uint64_t key = sg_sched_key(SG_SCHED_FILTER, {(uint64_t)n, prog_shape(pr),
                                                      post ? prog_shape(*post) + 1 : 0});
  int learned = -1;
  std::vector<float> pred;
  std::vector<double> us;
  int idx = sg_sched_lookup(c, SG_SCHED_FILTER, key, X, def, &learned, &pred, &us);
  cudaError_t e = cudaSuccess;
  auto kernel = [&](int i) {
    return sgk::jit_filter_kernel(pr, nullptr, (int)cand[i].chunk, post);
  };
  auto launch = [&](cudaKernel_t k, int i, sgk::Prof* prof) {
    return sgk::launch_filter_specialised(k, x, out, n, pr, dwork, rec, c->stream, c->num_sms,
                                          &c->kernels, prof, c->lookback, (int)cand[i].chunk,
                                          post);
  };
  if (idx < 0) {
    const bool debug = c->lookback.spin_limit != 0 || c->lookback.skip_tile >= 0;
    bool all = true;
    for (size_t i = 0; i < cand.size() && !debug; ++i) all &= kernel((int)i) != nullptr;
    if (debug || !all || n <= 0 || stream_capturing(c)) {
      idx = def;
    } else {
      us.assign(cand.size(), 0.0);
      for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
        cudaKernel_t k = kernel((int)i);
        e = time_launch(c, [&]() { return launch(k, (int)i, nullptr); }, &us[i]);
      }
      if (e != cudaSuccess) return e;
      idx = (int)(std::min_element(us.begin(), us.end()) - us.begin());
      sg_sched_log_sweep(c, SG_SCHED_FILTER, X, us, def);
      learned = sg_sched_learned_index(c, SG_SCHED_FILTER, X, def, &pred);
      sg_sched_set_tuned(c, SG_SCHED_FILTER, key, idx, us, learned);
    }
  }
  cudaKernel_t k = kernel(idx);
  if (!k && idx != def) {
    idx = def;
    k = kernel(idx);
  }
  if (!k) return cudaSuccess;
  sg_sched_note(c, SG_SCHED_FILTER, cand, us, def, learned, idx, pred);
  *ran = true;
  return launch(k, idx, &c->prof);
}

}  // namespace

namespace {

// One execution of the queued work under the fused (Sec. 5) or the unfused
// plan.  commit: the results go to the handles and the queue is emptied (the
// flush itself); otherwise (a measurement of the fusion boundaries) only the
// kernels run, and *us receives their device time (CUDA events on the
// context's stream).
sg_status run_flush(sg_ctx* c, bool fuse, bool commit, double* us) {
  // is an asynchronous read still on the copy engine?  (asked before this
  // flush launches anything; "not ready" is not an error of this flush)
  bool dl_busy = false;
  if (c->host_res_mapped && c->last_download) {
    const cudaError_t q = cudaEventQuery(c->last_download);
    if (q == cudaErrorNotReady) {
      dl_busy = true;
      cudaGetLastError();
    }
  }
  Planner pl(c, fuse);
  pl.plan();
  std::vector<Pass>& passes = pl.passes;
  c->has_violation = false;

  // scratch: result records, then the largest per-pass work area
  const size_t res_bytes = round_up(std::max<size_t>(1, passes.size()) * sgk::kResultBytes, 256);
  size_t work = 0;
  for (Pass& P : passes) {
    switch (P.kind) {
      case PK::STREAM:
        work = std::max(work, (size_t)std::max(stream_grid(c, P), c->num_sms * 8) *
                                  sizeof(sgk::PassResult));
        break;
      case PK::SORT: work = std::max(work, sgk::sort_scratch_bytes(P.n)); break;
      case PK::FILTER: work = std::max(work, sgk::filter_jit_scratch_bytes(P.n)); break;
      case PK::CHECK_SORTED:
      case PK::CHECK_PERM: work = std::max(work, sgk::check_scratch_bytes()); break;
      case PK::MATMUL:
      case PK::FREIVALDS: work = std::max(work, sg_linalg_scratch(c, P.main, P.chk_frv)); break;
      case PK::TRANSPOSE:
      case PK::CONCAT:
      case PK::FPRINT:
      case PK::CHECK_SAME: break;
      case PK::MATVEC: {
        const Node* n = P.main;
        const Value* A = P.vtrans ? P.vtrans->in[0].get() : n->left ? n->in[1].get() : nullptr;
        if (A) work = std::max(work, sgk::vecmat_scratch_bytes((int)A->rows, (int)A->cols));
        break;
      }
    }
  }
  sg_status st = ensure_scratch(c, res_bytes + work);
  if (!st) st = ensure_host_res(c, res_bytes);
  if (st) {
    if (commit) c->pending.clear();
    return st;
  }
  char* dres = static_cast<char*>(c->scratch);
  void* dwork = dres + res_bytes;
  // Passes that leave nothing for the host (pure maps, transposes, products,
  // concatenations) need no result records: then the flush neither clears
  // nor reads them back and does not wait for the device -- stream order
  // keeps every later use correct, and reads synchronise.
  bool need_records = false;
  for (Pass& P : passes) {
    switch (P.kind) {
      case PK::STREAM:
        need_records |= !P.prog.empty() && (P.reduce_of != nullptr || !P.preds.empty());
        break;
      case PK::MATMUL: need_records |= P.chk_frv != nullptr; break;
      case PK::TRANSPOSE:
      case PK::MATVEC:
      case PK::CONCAT: break;
      default: need_records = true; break;
    }
  }
  cudaError_t e = need_records ? cudaMemsetAsync(dres, 0, res_bytes, c->stream) : cudaSuccess;
  sg_status status = SG_OK;
  cudaEvent_t tev[2] = {nullptr, nullptr};
  if (us && e == cudaSuccess) {
    e = cudaEventCreate(&tev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&tev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(tev[0], c->stream);
  }

  for (size_t i = 0; i < passes.size() && e == cudaSuccess && !status; ++i) {
    Pass& P = passes[i];
    void* rec = dres + i * sgk::kResultBytes;
    switch (P.kind) {
      case PK::STREAM: {
        if (P.prog.empty()) break;
        sgk::StreamArgs a{};
        bool vec = true;
        for (size_t k = 0; k < P.inputs.size(); ++k) {
          Value* v = P.inputs[k];
          if (!v->st) { status = SG_ERR_INVALID_ARG; c->err = "internal: unmaterialised input"; break; }
          a.in[k] = static_cast<const float*>(v->st->ptr);
          vec &= aligned16(a.in[k]);
        }
        for (size_t k = 0; k < P.stores.size() && !status; ++k) {
          status = ensure_storage(c, P.stores[k]);
          if (!status) {
            a.out[k] = static_cast<float*>(P.stores[k]->st->ptr);
            vec &= aligned16(a.out[k]);
          }
        }
        if (status) break;
        a.n = P.n;
        if (P.count_src)
          for (size_t q = 0; q < i; ++q)
            if (passes[q].kind == PK::FILTER && passes[q].main == P.count_src)
              a.count = reinterpret_cast<const long long*>(dres + q * sgk::kResultBytes);
        a.prog.nops = (int)P.prog.size();
        std::vector<uint8_t> before;
        int md = 0;
        program_depths(P.prog, &before, &md);
        for (size_t p = 0; p < P.prog.size(); ++p) {
          a.prog.op[p] = P.prog[p].op;
          a.prog.arg[p] = P.prog[p].arg;
          a.prog.cst[p] = P.prog[p].cst;
          a.prog.depth[p] = before[p];
        }
        a.nin = (int)P.inputs.size();
        a.depth = md;
        a.has_reduce = P.reduce_of != nullptr;
        a.npred = (int)P.preds.size();
        a.pred_exists = 0;
        for (size_t p = 0; p < P.preds.size(); ++p) {
          Node* q = P.preds[p];
          const bool ex = q->kind == NK::QUANT ? q->exists : q->ckind == SG_C_EXISTS;
          if (ex) a.pred_exists |= 1u << p;
        }
        a.partials = static_cast<sgk::PassResult*>(dwork);
        a.counter = c->counter;
        a.result = static_cast<sgk::PassResult*>(rec);
        a.vec4 = vec ? 1 : 0;
        cudaKernel_t jk = nullptr;
        bool minmax = false;
        for (Node* q : P.reduces) minmax |= q->rop == SG_REDUCE_MIN || q->rop == SG_REDUCE_MAX;
        if (c->codegen == SG_CODEGEN_SPECIALIZE)
          jk = sgk::jit_stream_kernel(a.prog, a.nin, (int)P.stores.size(), a.npred,
                                      a.has_reduce != 0, minmax, a.pred_exists, nullptr);
        if (jk) {
          e = launch_stream_scheduled(c, jk, a, (int)P.stores.size(), minmax);
        } else {
          e = sgk::launch_stream(a, stream_grid(c, P), kStreamBlock, c->stream, &c->prof);
        }
        c->kernels++;
        break;
      }
      case PK::FILTER: {
        Node* n = P.main;
        Value* x = n->in[0].get();
        status = ensure_storage(c, n->out.get());
        if (status) break;
        int md = 0;
        const sgk::Prog pr = value_prog(n->expr, &md);
        sgk::Prog post{};
        if (P.chk_post) post = value_prog(P.chk_post->expr);
        bool ran = false;
        if (c->codegen == SG_CODEGEN_SPECIALIZE)
          e = launch_filter_scheduled(c, pr, static_cast<const float*>(x->st->ptr),
                                      static_cast<float*>(n->out->st->ptr), P.n, dwork,
                                      static_cast<sgk::FilterResult*>(rec), &ran,
                                      P.chk_post ? &post : nullptr);
        if (!ran && P.chk_post && e == cudaSuccess) {
          // the folded postcondition exists only in the specialised kernel
          status = SG_ERR_UNSUPPORTED;
          c->err = "the specialised filter with its folded postcondition could not be built";
          break;
        }
        if (!ran && e == cudaSuccess)
          e = sgk::launch_filter(static_cast<const float*>(x->st->ptr),
                                 static_cast<float*>(n->out->st->ptr), P.n, pr, md, dwork,
                                 static_cast<sgk::FilterResult*>(rec), c->stream, c->num_sms,
                                 &c->kernels, &c->prof, c->lookback);
        break;
      }
      case PK::SORT: {
        Node* n = P.main;
        status = ensure_storage(c, n->out.get());
        if (status) break;
        e = sgk::launch_sort(static_cast<const int32_t*>(n->in[0]->st->ptr),
                             static_cast<int32_t*>(n->out->st->ptr), P.n,
                             P.chk_sorted || P.chk_perm, dwork,
                             static_cast<sgk::SortResult*>(rec), c->stream, c->num_sms,
                             &c->kernels, &c->inject, &c->prof, n->in[0]->dt == SG_F32,
                             c->lookback);
        c->inject = sgk::SortInject{};
        break;
      }
      case PK::CHECK_SORTED: {
        Node* n = P.main;
        e = sgk::launch_check_sorted(static_cast<const int32_t*>(n->in[0]->st->ptr), P.n,
                                     static_cast<sgk::SortResult*>(rec), dwork, c->stream,
                                     c->num_sms, &c->kernels, &c->prof,
                                     n->in[0]->dt == SG_F32);
        break;
      }
      case PK::CHECK_PERM: {
        Node* n = P.main;
        e = sgk::launch_check_perm(static_cast<const int32_t*>(n->in[0]->st->ptr),
                                   static_cast<const int32_t*>(n->in[1]->st->ptr), P.n,
                                   static_cast<sgk::SortResult*>(rec), dwork, c->stream,
                                   c->num_sms, &c->kernels, &c->prof);
        break;
      }
      case PK::MATMUL:
      case PK::FREIVALDS:
        status = sg_exec_linalg(c, P.main, P.chk_frv, rec, dwork, &e);
        break;
      case PK::FPRINT: {
        Node* n = P.main;
        status = ensure_storage(c, n->out.get());
        if (status) break;
        const Value* x = n->in[0].get();
        e = sgk::launch_fprint(x->st ? x->st->ptr : nullptr, value_bytes(x), fprint_unit(x),
                               static_cast<unsigned long long*>(n->out->st->ptr), c->stream,
                               c->num_sms, &c->kernels, &c->prof);
        break;
      }
      case PK::CHECK_SAME: {
        // the fingerprint now, beside the one sg_old took, in the record
        Node* n = P.main;
        const Value* x = n->in[0].get();
        auto* r = static_cast<sgk::SortResult*>(rec);
        e = sgk::launch_fprint(x->st ? x->st->ptr : nullptr, value_bytes(x), fprint_unit(x),
                               r->fp_out, c->stream, c->num_sms, &c->kernels, &c->prof);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(r->fp_in, n->in[1]->st->ptr, sizeof r->fp_in,
                              cudaMemcpyDeviceToDevice, c->stream);
        break;
      }
      case PK::CONCAT: {
        Node* n = P.main;
        status = ensure_storage(c, n->out.get());
        if (status) break;
        const Value* a = n->in[0].get();
        const Value* b = n->in[1].get();
        const size_t es = (a->dt == SG_F64 || a->dt == SG_I64) ? 8
                          : (a->dt == SG_BF16 || a->dt == SG_F16) ? 2 : 4;
        char* dst = static_cast<char*>(n->out->st->ptr);
        if (a->n) e = sgk::launch_copy(dst, a->st->ptr, (size_t)a->n * es, c->num_sms, c->stream);
        if (e == cudaSuccess && b->n)
          e = sgk::launch_copy(dst + (size_t)a->n * es, b->st->ptr, (size_t)b->n * es, c->num_sms,
                               c->stream);
        c->kernels += 2;
        break;
      }
      case PK::TRANSPOSE: {
        Node* n = P.main;
        status = ensure_storage(c, n->out.get());
        if (status) break;
        const Value* A = n->in[0].get();
        e = sgk::launch_transpose(static_cast<const float*>(A->st->ptr), (int)A->rows,
                                  (int)A->cols, static_cast<float*>(n->out->st->ptr), c->stream,
                                  &c->prof);
        c->kernels += 1;
        break;
      }
      case PK::MATVEC: {
        Node* n = P.main;
        status = ensure_storage(c, n->out.get());
        if (status) break;
        float* y = static_cast<float*>(n->out->st->ptr);
        if (n->left || P.vtrans) {
          // y = x^T A; for a folded transpose, A is the transpose's source
          const Value* x = n->left ? n->in[0].get() : n->in[1].get();
          const Value* A = n->left ? n->in[1].get() : P.vtrans->in[0].get();
          e = sgk::launch_vecmat(static_cast<const float*>(x->st->ptr),
                                 static_cast<const float*>(A->st->ptr), (int)A->rows,
                                 (int)A->cols, y, dwork, c->stream, &c->prof);
          c->kernels += 2;
        } else {
          const Value* A = n->in[0].get();
          e = sgk::launch_matvec(static_cast<const float*>(A->st->ptr), (int)A->rows,
                                 (int)A->cols, static_cast<const float*>(n->in[1]->st->ptr), y,
                                 c->stream, &c->prof);
          c->kernels += 1;
        }
        break;
      }
    }
  }
  if (us && e == cudaSuccess && !status) e = cudaEventRecord(tev[1], c->stream);
  // while an asynchronous read is still on the copy engine, the records are
  // stored by a kernel instead of queueing a copy behind it
  if (e == cudaSuccess && !status && need_records) {
    if (dl_busy) {
      e = sgk::launch_copy(c->host_res, dres, passes.size() * sgk::kResultBytes, c->num_sms,
                           c->stream);
      c->kernels += 1;
    } else {
      e = cudaMemcpyAsync(c->host_res, dres, passes.size() * sgk::kResultBytes,
                          cudaMemcpyDeviceToHost, c->stream);
    }
  }
  if (e == cudaSuccess && !status && need_records) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess && !status && !need_records) e = cudaGetLastError();
  if (us) {
    float ms = 0.0f;
    if (e == cudaSuccess && !status) e = cudaEventSynchronize(tev[1]);
    if (e == cudaSuccess && !status) e = cudaEventElapsedTime(&ms, tev[0], tev[1]);
    *us = 1000.0 * ms;
    for (cudaEvent_t v : tev)
      if (v) cudaEventDestroy(v);
  }
  if (e != cudaSuccess && !status) status = cuda_fail(c, e, "kernel execution");
  if (e == cudaSuccess) c->prof.collect();
  if (!commit) return status;

  bool have = false;
  sg_status cstatus = SG_OK;
  if (!status) {
    const char* hres = static_cast<const char*>(c->host_res);
    for (size_t i = 0; i < passes.size(); ++i) {
      Pass& P = passes[i];
      const char* rec = hres + i * sgk::kResultBytes;
      switch (P.kind) {
        case PK::STREAM: {
          if (P.prog.empty()) break;
          sgk::PassResult r;
          memcpy(&r, rec, sizeof r);
          for (Node* n : P.reduces) {
            const bool empty = r.count == 0;
            double v = 0.0;
            switch (n->rop) {
              case SG_REDUCE_SUM: v = r.sum; break;
              case SG_REDUCE_COUNT: v = (double)r.count; break;
              case SG_REDUCE_MIN: v = (r.nan_seen || empty) ? NAN : (double)r.mn; break;
              case SG_REDUCE_MAX: v = (r.nan_seen || empty) ? NAN : (double)r.mx; break;
              case SG_REDUCE_AVG: v = empty ? NAN : r.sum / (double)r.count; break;
            }
            n->sout->value = v;
            n->sout->index = -1;
          }
          for (size_t p = 0; p < P.preds.size(); ++p) {
            Node* q = P.preds[p];
            const long long f = r.first[p];
            const bool hit = f != kNone;
            if (q->kind == NK::QUANT) {
              q->sout->value = q->exists ? (hit ? 1.0 : 0.0) : (hit ? 0.0 : 1.0);
              q->sout->index = hit ? f : -1;
            } else if (q->ckind == SG_C_FOR_ALL ? hit : !hit) {
              record_violation(c, q, q->ckind == SG_C_FOR_ALL ? f : -1, 0.0, &have, &cstatus);
            }
          }
          break;
        }
        case PK::FILTER: {
          sgk::FilterResult r;
          memcpy(&r, rec, sizeof r);
          if (r.timeout) {
            status = SG_ERR_TIMEOUT;
            c->err = "filter look-back wait gave up";
            r.count = 0;   // the kept items of a timed-out compaction are no result
          }
          P.main->out->n = r.count;
          P.main->out->rows = r.count;
          P.main->out->count_known = true;
          if (P.chk_post && !r.timeout && r.post_enc != 0)
            record_violation(c, P.chk_post, (int64_t)~r.post_enc, 0.0, &have, &cstatus);
          break;
        }
        case PK::SORT:
        case PK::CHECK_SORTED:
        case PK::CHECK_PERM: {
          sgk::SortResult r;
          memcpy(&r, rec, sizeof r);
          if (r.timeout) {
            status = SG_ERR_TIMEOUT;
            c->err = "sort look-back wait gave up";
          }
          Node* ks = P.kind == PK::SORT ? P.chk_sorted : P.kind == PK::CHECK_SORTED ? P.main : nullptr;
          Node* kp = P.kind == PK::SORT ? P.chk_perm : P.kind == PK::CHECK_PERM ? P.main : nullptr;
          if (ks && r.unsorted_enc != 0)
            record_violation(c, ks, (int64_t)~r.unsorted_enc, 0.0, &have, &cstatus);
          if (kp && (r.fp_in[0] != r.fp_out[0] || r.fp_in[1] != r.fp_out[1] ||
                     r.cnt_in != r.cnt_out))
            record_violation(c, kp, -1, 0.0, &have, &cstatus);
          break;
        }
        case PK::CHECK_SAME: {
          sgk::SortResult r;
          memcpy(&r, rec, sizeof r);
          if (r.fp_in[0] != r.fp_out[0] || r.fp_in[1] != r.fp_out[1])
            record_violation(c, P.main, -1, 0.0, &have, &cstatus);
          break;
        }
        case PK::TRANSPOSE:
        case PK::MATVEC:
        case PK::CONCAT:
        case PK::FPRINT:
          break;
        case PK::MATMUL:
        case PK::FREIVALDS: {
          double observed = 0.0;
          long long row = -1;
          if (sg_linalg_result(c, P.main, P.chk_frv, rec, &row, &observed))
            record_violation(c, P.chk_frv ? P.chk_frv : P.main, row, observed, &have, &cstatus);
          break;
        }
      }
    }
  }

  // poison: a failed contract poisons its target and everything computed
  // from it (queue order is a topological order)
  for (Node* n : pl.nodes)
    if (n->failed && n->in[0]) n->in[0]->poisoned = true;
  for (Node* n : pl.nodes) {
    bool p = false;
    for (int k = 0; k < n->nin; ++k) p |= n->in[k] && n->in[k]->poisoned;
    if (n->kind == NK::CHECK) continue;
    if (p && n->out) n->out->poisoned = true;
    if (p && n->sout) n->sout->poisoned = true;
  }
  for (Node* n : pl.nodes) {
    if (n->out) {
      n->out->producer = nullptr;
      if (!n->out->count_known && status) n->out->count_known = true, n->out->n = 0;
    }
    if (n->sout) {
      n->sout->producer = nullptr;
      n->sout->done = true;
      if (status) n->sout->poisoned = true;
    }
  }
  c->pending.clear();
  if (status) return status;
  return cstatus;
}

// The fusion boundaries (SG_SCHED_FUSION) of a flush whose work is only
// element-wise passes: true for the fused plan.  The fused plan unless a
// forced choice, the learned model or the autotuner's measurement of both
// plans over the whole flush (a warm-up, then the better of two runs, each
// plan's kernels timed by CUDA events) prefers one kernel per queued call.
bool choose_fusion(sg_ctx* c) {
  // the shape of the queued calls: kinds, programs (not their constants),
  // which call feeds which, lengths, and which results a handle keeps
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
  std::map<const Value*, int> ext;
  std::map<const Value*, int> made;
  int idx_node = 0;
  for (auto& np : c->pending) {
    const Node* nd = np.get();
    const bool elementwise = (nd->kind == NK::MAP && !nd->inplace) || nd->kind == NK::REDUCE ||
                             nd->kind == NK::QUANT || nd->kind == NK::CHECK;
    if (!elementwise) return true;
    mix((uint64_t)nd->kind);
    mix((uint64_t)nd->nin);
    mix((uint64_t)nd->rop);
    mix((uint64_t)nd->ckind * 2 + (nd->exists ? 1 : 0));
    for (int p = 0; p < nd->expr.nops; ++p) {
      mix((uint64_t)nd->expr.ops[p].op);
      mix((uint64_t)(uint32_t)nd->expr.ops[p].arg);
    }
    for (int k = 0; k < nd->nin; ++k) {
      const Value* v = nd->in[k].get();
      if (!v) continue;
      mix((uint64_t)v->n);
      auto m = made.find(v);
      if (m != made.end()) {
        mix(0x100000000ull + (uint64_t)m->second);
      } else {
        auto e = ext.find(v);
        const int id = e == ext.end() ? (int)ext.size() : e->second;
        if (e == ext.end()) ext[v] = id;
        mix(0x200000000ull + (uint64_t)id);
      }
    }
    if (nd->out) {
      made[nd->out.get()] = idx_node;
      mix(nd->out->handles > 0 ? 1 : 2);
    }
    ++idx_node;
  }
  const uint64_t key = sg_sched_key(SG_SCHED_FUSION, {h});
  const int forced = c->schedst.forced[SG_SCHED_FUSION];
  SchedState& ss = c->schedst;
  if (forced < 0 || forced > 1) {
    if (c->sched == SG_SCHED_LEARNED && ss.model[SG_SCHED_FUSION].trained)
      for (auto& t : ss.learned_memo)
        if (t.first == key) return t.second == 0;
    const int tuned = sg_sched_tuned(c, key);
    if (tuned >= 0 && !(c->sched == SG_SCHED_LEARNED && ss.model[SG_SCHED_FUSION].trained))
      return tuned == 0;
  }
  // first sight: both plans, which must be element-wise passes alone and differ
  Planner pf(c, true), pu(c, false);
  pf.plan();
  pu.plan();
  FusionWork w;
  w.nodes = (int)c->pending.size();
  bool ok = true;
  Planner* pls[2] = {&pf, &pu};
  for (int k = 0; k < 2; ++k)
    for (const Pass& P : pls[k]->passes) {
      if (P.kind != PK::STREAM) {
        ok = false;
        continue;
      }
      if (P.prog.empty()) continue;
      w.passes[k] += 1;
      w.bytes[k] += 4.0 * (double)P.n * (double)(P.inputs.size() + P.stores.size());
      w.n = std::max<long long>(w.n, P.n);
    }
  for (auto& np : c->pending) {
    const Node* nd = np.get();
    w.reduces += nd->kind == NK::REDUCE;
    w.preds += nd->kind == NK::QUANT || nd->kind == NK::CHECK;
    w.ops += nd->expr.nops;
  }
  if (!ok || w.passes[0] == w.passes[1]) {
    if (forced < 0) sg_sched_set_tuned(c, SG_SCHED_FUSION, key, 0);
    return true;
  }
  const std::vector<sg_sched_choice> cand = sg_fusion_candidates(w);
  std::vector<float> X(2 * kSchedFeatures);
  for (int k = 0; k < 2; ++k) sg_fusion_features(w, k, &X[(size_t)k * kSchedFeatures]);
  std::vector<float> pred;
  std::vector<double> us;
  int learned = -1, idx = 0;
  if (forced == 0 || forced == 1) {
    idx = forced;
  } else if (c->sched == SG_SCHED_LEARNED && ss.model[SG_SCHED_FUSION].trained) {
    learned = sg_sched_learned_index(c, SG_SCHED_FUSION, X, 0, &pred);
    idx = learned >= 0 ? learned : 0;
    ss.learned_memo.push_back({key, idx});
  } else if (!stream_capturing(c)) {
    us.assign(2, 0.0);
    for (int k = 0; k < 2; ++k) {
      double best = 1e300;
      for (int r = 0; r < 3; ++r) {
        double t = 0.0;
        if (run_flush(c, k == 0, false, &t) != SG_OK) return true;
        if (r > 0) best = std::min(best, t);
      }
      us[k] = best;
    }
    idx = us[1] < kFusionMargin * us[0] ? 1 : 0;
    sg_sched_log_sweep(c, SG_SCHED_FUSION, X, us, 0);
    learned = sg_sched_learned_index(c, SG_SCHED_FUSION, X, 0, &pred);
    sg_sched_set_tuned(c, SG_SCHED_FUSION, key, idx, us, learned);
  }
  sg_sched_note(c, SG_SCHED_FUSION, cand, us, 0, learned, idx, pred);
  return idx == 0;
}

}  // namespace

sg_status sg_execute_pending(sg_ctx* c) {
  bool fuse = c->fusion == SG_FUSE_ON;
  if (fuse && !c->pending.empty()) fuse = choose_fusion(c);
  return run_flush(c, fuse, true, nullptr);
}

sg_status sg_describe_pending(sg_ctx* c, std::string* out) {
  Planner pl(c);
  pl.plan();
  std::string s;
  char buf[256];
  for (Pass& P : pl.passes) {
    switch (P.kind) {
      case PK::STREAM:
        if (P.prog.empty()) continue;
        snprintf(buf, sizeof buf, "stream n=%lld%s in=%zu store=%zu pred=%zu reduce=%d ops=%zu\n",
                 (long long)P.n, P.count_src ? " (the filter's count)" : "", P.inputs.size(),
                 P.stores.size(), P.preds.size(), P.reduce_of ? 1 : 0, P.prog.size());
        break;
      case PK::FILTER:
        snprintf(buf, sizeof buf, "filter n=%lld%s\n", (long long)P.n,
                 P.chk_post ? " for_all=1" : "");
        break;
      case PK::SORT:
        snprintf(buf, sizeof buf, "sort n=%lld sorted=%d perm=%d\n", (long long)P.n,
                 P.chk_sorted ? 1 : 0, P.chk_perm ? 1 : 0);
        break;
      case PK::CHECK_SORTED: snprintf(buf, sizeof buf, "check_sorted n=%lld\n", (long long)P.n); break;
      case PK::CHECK_PERM: snprintf(buf, sizeof buf, "check_perm n=%lld\n", (long long)P.n); break;
      case PK::MATMUL:
        snprintf(buf, sizeof buf, "matmul %lldx%lldx%lld prec=%d%s\n",
                 (long long)P.main->in[0]->rows, (long long)P.main->in[0]->cols,
                 (long long)P.main->in[1]->cols, P.main->prec,
                 P.chk_frv ? " +freivalds(fused)" : "");
        break;
      case PK::FREIVALDS:
        snprintf(buf, sizeof buf, "freivalds n=%lld nvec=%d\n", (long long)P.main->in[0]->rows,
                 P.main->nvec);
        break;
      case PK::TRANSPOSE:
        snprintf(buf, sizeof buf, "transpose %lldx%lld\n", (long long)P.main->in[0]->rows,
                 (long long)P.main->in[0]->cols);
        break;
      case PK::CONCAT:
        snprintf(buf, sizeof buf, "concat %lld+%lld\n", (long long)P.main->in[0]->n,
                 (long long)P.main->in[1]->n);
        break;
      case PK::FPRINT:
        snprintf(buf, sizeof buf, "fingerprint(old) n=%lld\n", (long long)P.main->in[0]->n);
        break;
      case PK::CHECK_SAME:
        snprintf(buf, sizeof buf, "check_unchanged n=%lld\n", (long long)P.main->in[0]->n);
        break;
      case PK::MATVEC: {
        const Node* n = P.main;
        const Value* A = P.vtrans ? P.vtrans->in[0].get() : n->left ? n->in[1].get() : n->in[0].get();
        snprintf(buf, sizeof buf, "%s %lldx%lld%s\n", (n->left || P.vtrans) ? "vecmat" : "matvec",
                 (long long)A->rows, (long long)A->cols, P.vtrans ? " (transpose folded)" : "");
        break;
      }
    }
    s += buf;
  }
  *out = std::move(s);
  return SG_OK;
}
