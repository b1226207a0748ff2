// sg_eval.cuh -- device-side evaluation of the fused element-wise programs
// (postfix ops with per-op stack depths, see sg_internal.h), shared by the
// streaming, filter and batched kernels.
#pragma once
#include <math_constants.h>

#include "sg_internal.h"

namespace sgk {
namespace ev {

constexpr long long kNoIndex = 0x7fffffffffffffffLL;

struct Acc {
  double sum;
  float hi, lo;   // per-thread double-float partial sum (folded into sum)
  long long cnt;
  float mn, mx;
  int nan_seen;
  long long first[kMaxPred];
};

__device__ __forceinline__ bool truthy(float v) { return v != 0.0f; }
__device__ __forceinline__ float b2f(bool b) { return b ? 1.0f : 0.0f; }

__device__ __forceinline__ float min_nan(float a, float b) {
  return (isnan(a) || isnan(b)) ? CUDART_NAN_F : (a < b ? a : b);
}
__device__ __forceinline__ float max_nan(float a, float b) {
  return (isnan(a) || isnan(b)) ? CUDART_NAN_F : (a > b ? a : b);
}

template <int L>
__device__ __forceinline__ void acc_reduce(Acc& acc, const float (&v)[L],
                                           const float (&mask)[L]) {
  float t[L];
  int c = 0;
  bool any_inf = false;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const bool m = mask[l] != 0.0f;
    t[l] = m ? v[l] : 0.0f;
    c += m ? 1 : 0;
    any_inf |= isinf(t[l]);
    if (m) {
      if (isnan(v[l])) {
        acc.nan_seen = 1;
      } else {
        acc.mn = v[l] < acc.mn ? v[l] : acc.mn;
        acc.mx = v[l] > acc.mx ? v[l] : acc.mx;
      }
    }
  }
  acc.cnt += c;
  // Knuth's TwoSum per element into a binary32 double-float accumulator
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const float s = __fadd_rn(acc.hi, t[l]);
    const float bp = __fsub_rn(s, acc.hi);
    const float e = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bp)), __fsub_rn(t[l], bp));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, e);
  }
  (void)any_inf;
}

// Execute op `op` with the stack holding D values before it.
template <int D, int L, int NX, int DEPTH>
__device__ __forceinline__ void exec_at(int op, int arg, float cst,
                                        const StreamArgs& a,
                                        float (&s)[DEPTH][L],
                                        const float (&x)[NX][L],
                                        float (&mask)[L], const bool (&vm)[L],
                                        long long i0, Acc& acc) {
  if constexpr (D > DEPTH) {
    return;
  } else {
  switch (op) {
    case SG_OP_LOAD:
      if constexpr (D < DEPTH) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
          float v = x[0][l];
#pragma unroll
          for (int k = 1; k < NX; ++k)
            if (arg == k) v = x[k][l];
          s[D][l] = v;
        }
      }
      break;
    case SG_OP_CONST:
      if constexpr (D < DEPTH) {
#pragma unroll
        for (int l = 0; l < L; ++l) s[D][l] = cst;
      }
      break;
    case SG_OP_INDEX:
      if constexpr (D < DEPTH) {
#pragma unroll
        for (int l = 0; l < L; ++l) s[D][l] = __ll2float_rn(i0 + l);
      }
      break;
    case SG_OP_DUP:
      if constexpr (D >= 1 && D < DEPTH) {
#pragma unroll
        for (int l = 0; l < L; ++l) s[D][l] = s[D - 1][l];
      }
      break;
#define SG_BIN(OPC, EXPR)                                          \
  case OPC:                                                        \
    if constexpr (D >= 2) {                                        \
      _Pragma("unroll") for (int l = 0; l < L; ++l) {              \
        const float A = s[D - 2][l], B = s[D - 1][l];              \
        s[D - 2][l] = (EXPR);                                      \
      }                                                            \
    }                                                              \
    break;
      SG_BIN(SG_OP_ADD, __fadd_rn(A, B))
      SG_BIN(SG_OP_SUB, __fsub_rn(A, B))
      SG_BIN(SG_OP_MUL, __fmul_rn(A, B))
      SG_BIN(SG_OP_DIV, __fdiv_rn(A, B))
      SG_BIN(SG_OP_MIN, min_nan(A, B))
      SG_BIN(SG_OP_MAX, max_nan(A, B))
      SG_BIN(SG_OP_LT, b2f(A < B))
      SG_BIN(SG_OP_LE, b2f(A <= B))
      SG_BIN(SG_OP_GT, b2f(A > B))
      SG_BIN(SG_OP_GE, b2f(A >= B))
      SG_BIN(SG_OP_EQ, b2f(A == B))
      SG_BIN(SG_OP_NE, b2f(A != B))
      SG_BIN(SG_OP_AND, b2f(truthy(A) && truthy(B)))
      SG_BIN(SG_OP_OR, b2f(truthy(A) || truthy(B)))
#undef SG_BIN
    case SG_OP_SWAP:
      if constexpr (D >= 2) {
#pragma unroll
        for (int l = 0; l < L; ++l) {
          const float t = s[D - 1][l];
          s[D - 1][l] = s[D - 2][l];
          s[D - 2][l] = t;
        }
      }
      break;
#define SG_UN(OPC, EXPR)                                           \
  case OPC:                                                        \
    if constexpr (D >= 1) {                                        \
      _Pragma("unroll") for (int l = 0; l < L; ++l) {              \
        const float A = s[D - 1][l];                               \
        s[D - 1][l] = (EXPR);                                      \
      }                                                            \
    }                                                              \
    break;
      SG_UN(SG_OP_NEG, -A)
      SG_UN(SG_OP_ABS, fabsf(A))
      SG_UN(SG_OP_SQRT, __fsqrt_rn(A))
      SG_UN(SG_OP_NOT, b2f(!truthy(A)))
#undef SG_UN
    case SG_OP_FMA:
      if constexpr (D >= 3) {
#pragma unroll
        for (int l = 0; l < L; ++l)
          s[D - 3][l] = __fmaf_rn(s[D - 3][l], s[D - 2][l], s[D - 1][l]);
      }
      break;
    case SG_OP_SELECT:
      if constexpr (D >= 3) {
#pragma unroll
        for (int l = 0; l < L; ++l)
          s[D - 3][l] = truthy(s[D - 3][l]) ? s[D - 2][l] : s[D - 1][l];
      }
      break;
    case K_STORE:
      if constexpr (D >= 1) {
        float* o = a.out[0];
#pragma unroll
        for (int k = 1; k < kMaxOut; ++k)
          if (arg == k) o = a.out[k];
        if constexpr (L == 4) {
          *reinterpret_cast<float4*>(o + i0) =
              make_float4(s[D - 1][0], s[D - 1][1 % L], s[D - 1][2 % L],
                          s[D - 1][3 % L]);
        } else {
#pragma unroll
          for (int l = 0; l < L; ++l) o[i0 + l] = s[D - 1][l];
        }
      }
      break;
    case K_PRED:
      if constexpr (D >= 1) {
        const bool ex = (a.pred_exists >> arg) & 1u;
        long long hit = kNoIndex;
#pragma unroll
        for (int l = L - 1; l >= 0; --l) {
          const bool t = truthy(s[D - 1][l]);
          if (vm[l] && (ex ? t : !t)) hit = i0 + l;
        }
#pragma unroll
        for (int p = 0; p < kMaxPred; ++p)
          if (p == arg && hit < acc.first[p]) acc.first[p] = hit;
      }
      break;
    case K_MASK:
      if constexpr (D >= 1) {
#pragma unroll
        for (int l = 0; l < L; ++l) mask[l] = b2f(vm[l] && truthy(s[D - 1][l]));
      }
      break;
    case K_REDUCE:
      if constexpr (D >= 1) {
        float v[L];
#pragma unroll
        for (int l = 0; l < L; ++l) v[l] = s[D - 1][l];
        acc_reduce<L>(acc, v, mask);
#pragma unroll
        for (int l = 0; l < L; ++l) mask[l] = b2f(vm[l]);
      }
      break;
    default:  // K_POP: the host's depth bookkeeping already dropped the value
      break;
  }
  }
}

// vm: lanes that hold a real element (sinks ignore the others)
template <int L, int NX, int DEPTH>
__device__ __forceinline__ void run_prog(const StreamArgs& a,
                                         const float (&x)[NX][L], long long i0,
                                         const bool (&vm)[L], Acc& acc) {
  float s[DEPTH][L];
  float mask[L];
#pragma unroll
  for (int l = 0; l < L; ++l) mask[l] = b2f(vm[l]);
  const int nops = a.prog.nops;
  for (int pc = 0; pc < nops; ++pc) {
    const int op = a.prog.op[pc];
    const int arg = a.prog.arg[pc];
    const float c = a.prog.cst[pc];
    switch (a.prog.depth[pc]) {
      case 0: exec_at<0, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 1: exec_at<1, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 2: exec_at<2, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 3: exec_at<3, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 4: exec_at<4, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 5: exec_at<5, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 6: exec_at<6, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 7: exec_at<7, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      default: exec_at<8, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
    }
  }
}

__device__ __forceinline__ void acc_fold(Acc& a) {
  a.sum += (double)a.hi + (double)a.lo;
  a.hi = 0.0f;
  a.lo = 0.0f;
}

__device__ __forceinline__ void acc_merge(Acc& a, const Acc& b) {
  a.sum += b.sum + ((double)b.hi + (double)b.lo);
  a.cnt += b.cnt;
  a.mn = b.mn < a.mn ? b.mn : a.mn;
  a.mx = b.mx > a.mx ? b.mx : a.mx;
  a.nan_seen |= b.nan_seen;
#pragma unroll
  for (int p = 0; p < kMaxPred; ++p)
    a.first[p] = b.first[p] < a.first[p] ? b.first[p] : a.first[p];
}

__device__ __forceinline__ void warp_reduce(Acc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Acc b;
    b.hi = 0.0f;
    b.lo = 0.0f;
    b.sum = __shfl_xor_sync(0xffffffffu, a.sum, o);
    b.cnt = __shfl_xor_sync(0xffffffffu, a.cnt, o);
    b.mn = __shfl_xor_sync(0xffffffffu, a.mn, o);
    b.mx = __shfl_xor_sync(0xffffffffu, a.mx, o);
    b.nan_seen = __shfl_xor_sync(0xffffffffu, a.nan_seen, o);
#pragma unroll
    for (int p = 0; p < kMaxPred; ++p)
      b.first[p] = __shfl_xor_sync(0xffffffffu, a.first[p], o);
    acc_merge(a, b);
  }
}

__device__ __forceinline__ void to_rec(const Acc& a, PassResult& r) {
  r.sum = a.sum;
  r.count = a.cnt;
  r.mn = a.mn;
  r.mx = a.mx;
  r.nan_seen = a.nan_seen;
  r.pad = 0;
#pragma unroll
  for (int p = 0; p < kMaxPred; ++p) r.first[p] = a.first[p];
}

__device__ __forceinline__ void from_rec(const PassResult* r, Acc& a) {
  a.sum = __ldcg(&r->sum);
  a.hi = 0.0f;
  a.lo = 0.0f;
  a.cnt = __ldcg(&r->count);
  a.mn = __ldcg(&r->mn);
  a.mx = __ldcg(&r->mx);
  a.nan_seen = __ldcg(&r->nan_seen);
#pragma unroll
  for (int p = 0; p < kMaxPred; ++p) a.first[p] = __ldcg(&r->first[p]);
}

__device__ __forceinline__ void acc_init(Acc& a) {
  a.sum = 0.0;
  a.hi = 0.0f;
  a.lo = 0.0f;
  a.cnt = 0;
  a.mn = CUDART_INF_F;
  a.mx = -CUDART_INF_F;
  a.nan_seen = 0;
#pragma unroll
  for (int p = 0; p < kMaxPred; ++p) a.first[p] = kNoIndex;
}

// Block-wide reduction of `a` into thread 0 (fixed order).
__device__ __forceinline__ void block_reduce(Acc& a) {
  __shared__ Acc sh[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  warp_reduce(a);
  if (lane == 0) sh[w] = a;
  __syncthreads();
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    if (lane < nw) a = sh[lane]; else acc_init(a);
    warp_reduce(a);
  }
  __syncthreads();
}


// Evaluates a program that leaves exactly one value (no sinks) and returns
// it per lane.
template <int L, int NX, int DEPTH>
__device__ __forceinline__ void eval_value(const StreamArgs& a, const float (&x)[NX][L],
                                           long long i0, float (&v)[L]) {
  float s[DEPTH][L];
  float mask[L];
  bool vm[L];
  Acc acc;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    mask[l] = 1.0f;
    vm[l] = true;
  }
  const int nops = a.prog.nops;
  for (int pc = 0; pc < nops; ++pc) {
    const int op = a.prog.op[pc];
    const int arg = a.prog.arg[pc];
    const float c = a.prog.cst[pc];
    switch (a.prog.depth[pc]) {
      case 0: exec_at<0, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 1: exec_at<1, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 2: exec_at<2, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 3: exec_at<3, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 4: exec_at<4, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 5: exec_at<5, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 6: exec_at<6, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      case 7: exec_at<7, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
      default: exec_at<8, L, NX, DEPTH>(op, arg, c, a, s, x, mask, vm, i0, acc); break;
    }
  }
#pragma unroll
  for (int l = 0; l < L; ++l) v[l] = s[0][l];
}

}  // namespace ev
}  // namespace sgk
