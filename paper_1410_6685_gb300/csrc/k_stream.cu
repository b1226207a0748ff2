// k_stream.cu -- the fused streaming pass (sm_103a).
//
// One grid-stride pass over n elements that evaluates the optimizer's fused
// program (Sec. 5: map chains rewritten into one expression, Fig. 3; a map
// merged with its reduction, Fig. 2; range contracts for_all / exists of
// Sec. 4 folded into the same pass).  Per element it may store up to four
// outputs, check up to four predicates (recording the smallest index where a
// for_all fails or an exists holds) and feed one masked reduction
// (sum / count / min / max).
//
// Memory: inputs are read once with 128-bit loads (4 elements per thread per
// step), outputs written once with 128-bit stores; the rest is registers.
// The per-block partial records and the last-block-done combine make the
// result deterministic (fixed combine order for a fixed grid).
#include "sg_eval.cuh"

namespace sgk {
namespace {

using namespace ev;

template <int NIN, int DEPTH>
__global__ void __launch_bounds__(256) k_stream(const StreamArgs a) {
  constexpr int NX = NIN > 0 ? NIN : 1;
  Acc acc;
  acc_init(acc);
  long long n = a.n;
  if (a.count) {
    const long long c = *a.count;
    n = c < 0 ? 0 : c < n ? c : n;
  }
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long tail_start = 0;
  if (a.vec4) {
    const long long nv = n >> 2;
    tail_start = nv << 2;
    for (long long v = tid; v < nv; v += stride) {
      float x[NX][4];
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        if (k < NIN) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(a.in[k]) + v);
          x[k][0] = t.x; x[k][1] = t.y; x[k][2] = t.z; x[k][3] = t.w;
        } else {
          x[k][0] = x[k][1] = x[k][2] = x[k][3] = 0.0f;
        }
      }
      const bool vm[4] = {true, true, true, true};
      run_prog<4, NX, DEPTH>(a, x, v << 2, vm, acc);
    }
  }
  for (long long i = tail_start + tid; i < n; i += stride) {
    float x[NX][1];
#pragma unroll
    for (int k = 0; k < NX; ++k) x[k][0] = (k < NIN) ? a.in[k][i] : 0.0f;
    const bool vm[1] = {true};
    run_prog<1, NX, DEPTH>(a, x, i, vm, acc);
  }

  if (!a.has_reduce && a.npred == 0) return;

  acc_fold(acc);
  block_reduce(acc);
  __shared__ bool am_last;
  if (threadIdx.x == 0) {
    PassResult r;
    to_rec(acc, r);
    a.partials[blockIdx.x] = r;
    __threadfence();
    const unsigned t = atomicAdd(a.counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  Acc tot;
  acc_init(tot);
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    Acc p;
    from_rec(&a.partials[b], p);
    acc_merge(tot, p);
  }
  block_reduce(tot);
  if (threadIdx.x == 0) {
    PassResult r;
    to_rec(tot, r);
    *a.result = r;
    *a.counter = 0u;
  }
}

}  // namespace

template <int NIN, int DEPTH>
static int occ(int block) {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, k_stream<NIN, DEPTH>, block, 0);
  return e == cudaSuccess && nb > 0 ? nb : 1;
}

int stream_max_blocks_per_sm(int nin, int depth, int block) {
  const bool deep = depth > 4;
  switch (nin) {
    case 0: return deep ? occ<0, 8>(block) : occ<0, 4>(block);
    case 1: return deep ? occ<1, 8>(block) : occ<1, 4>(block);
    case 2: return deep ? occ<2, 8>(block) : occ<2, 4>(block);
    case 3: return deep ? occ<3, 8>(block) : occ<3, 4>(block);
    default: return deep ? occ<4, 8>(block) : occ<4, 4>(block);
  }
}

template <int NIN>
static void launch_nin(const StreamArgs& a, bool deep, int grid, int block,
                       cudaStream_t s) {
  if (deep)
    k_stream<NIN, 8><<<grid, block, 0, s>>>(a);
  else
    k_stream<NIN, 4><<<grid, block, 0, s>>>(a);
}

cudaError_t launch_stream(const StreamArgs& a, int grid, int block,
                          cudaStream_t s, Prof* prof) {
  const bool deep = a.depth > 4;
  prof_begin(prof, "stream", s);
  switch (a.nin) {
    case 0: launch_nin<0>(a, deep, grid, block, s); break;
    case 1: launch_nin<1>(a, deep, grid, block, s); break;
    case 2: launch_nin<2>(a, deep, grid, block, s); break;
    case 3: launch_nin<3>(a, deep, grid, block, s); break;
    case 4: launch_nin<4>(a, deep, grid, block, s); break;
    default: return cudaErrorInvalidValue;
  }
  prof_end(prof, s);
  return cudaGetLastError();
}

}  // namespace sgk
