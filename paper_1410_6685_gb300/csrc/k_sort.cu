// k_sort.cu -- ascending sort of signed int32 keys (sm_103a) with the
// postconditions of Listing 4 (`Result.is_sorted`, and `Result.count =
// a.count` strengthened to "Result is a permutation of a") fused into the
// last pass.
//
// Method: least-significant-digit radix sort with 8-bit digits.
//   1. k_radix_hist: one read of the input builds the four 256-bin digit
//      histograms and the input's multiset fingerprint; its last block turns
//      the histograms into per-digit global start offsets.
//   2. k_onesweep x4: each CTA takes the next tile (a global atomic ticket,
//      so tiles start in order; 6144 keys, 24 per thread), prefetches the
//      tile one resident wave ahead into L2 (cp.async.bulk.prefetch), ranks its keys
//      stably inside the tile (warp-private counters; the lanes sharing a
//      digit are found by match_any or by ballots), publishes its per-digit tile
//      counts, finds the exclusive prefix of each digit over the preceding
//      tiles by a decoupled look-back (bounded waits; the words of several
//      preceding tiles per memory round trip), sorts the tile in
//      shared memory by digit and writes it out in digit runs.
//   The last pass flips the sign bit (signed order) and, when the contracts
//   are on, (a) checks every adjacent pair inside each tile-local digit run,
//   (b) carries the last key of every digit run through the look-back words
//   so each run's first key is compared with its predecessor in the output,
//   and (c) accumulates the output's multiset fingerprint (sum of mix(k),
//   sum of mix(k)^2 mod 2^64, count; mix(k) = rot16(k * c1) * c2 with odd
//   c1, c2, a bijection of 32-bit words) for comparison with the input's.  No
//   extra pass over the keys is needed.
#include <stdint.h>

#include <climits>

#include "sg_internal.h"

namespace sgk {
namespace {

constexpr int kSortBlock = 256;
constexpr int kSortMinBlocks = 4;   // resident CTAs per SM the registers are sized for
constexpr int kKpt = 24;
constexpr int kTile = kSortBlock * kKpt;   // 6144 keys
constexpr int kMatchEvery = 8;
constexpr int kRadix = 256;
constexpr int kWarps = kSortBlock / 32;
constexpr int kWarpKeys = 32 * kKpt;
constexpr unsigned kSpinLimit = 1u << 22;
// look-back window: the words of this many preceding tiles are loaded
// together and then taken in order, so one memory round trip covers several
// steps of the walk (4 for the 32-bit words, 2 for the 64-bit words of the
// checked last pass: the fastest of 1, 2, 4 and 8 for each, 15% and 8% faster
// passes than one word at a time)
constexpr int kLook = 4;
constexpr int kLookWide = 2;

constexpr unsigned kCntMask = (1u << 30) - 1;
constexpr unsigned kAgg = 1u;
constexpr unsigned kPre = 2u;

static_assert(kSortBlock % kRadix == 0, "threads 0..255 own one digit each");

struct SortHdr {
  unsigned hist[4][kRadix];
  unsigned offs[4][kRadix];
  unsigned tile_ctr[4];
  unsigned done_ctr;
  unsigned pad[27];
  // a look-back wait gave up (also recorded in the result record); on a line
  // of its own, away from the tickets and the result record's atomics, since
  // every CTA of a later pass reads it when it starts
  int failed;
  unsigned pad2[31];
};
static_assert(sizeof(SortHdr) % 128 == 0, "header lines");

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Order-preserving unsigned image of a key: signed int32 order (flip the
// sign bit), or for binary32 bit patterns the IEEE totalOrder (negative
// patterns: flip every bit; positive: flip the sign bit).
template <bool FLT>
__device__ __forceinline__ unsigned okey(int k) {
  const unsigned u = (unsigned)k;
  return FLT ? (u ^ ((unsigned)(k >> 31) | 0x80000000u)) : (u ^ 0x80000000u);
}

// digit of a key in a pass: byte `pass` of okey.  sel = 0x4440 | pass: one
// byte permute moves that byte to the low byte and zeroes the rest.  For
// int32 keys only the last pass's byte differs from the raw key's.
template <bool LAST, bool FLT>
__device__ __forceinline__ unsigned digit_of(int k, unsigned sel) {
  if (FLT) return __byte_perm(okey<true>(k), 0u, sel);
  const unsigned u = (unsigned)k;
  return LAST ? ((u >> 24) ^ 0x80u) : __byte_perm(u, 0u, sel);
}

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Exclusive scan of one value per thread over the 256-thread block.
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* s_warp) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned t = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < kWarps) s_warp[lane] = t - s_warp[lane];   // exclusive warp offsets
  }
  __syncthreads();
  return x - v + s_warp[w];
}

// The key mix of the multiset fingerprint: multiply by an odd constant,
// rotate by 16, multiply by another odd constant.  Each step is a bijection
// of 32-bit words, so replacing one key by another always changes the sums
// below; the rotation makes the map non-linear in the key.  Two multiplies
// and one byte permute: cheap enough for a pass bound by instruction issue.
__device__ __forceinline__ unsigned key_mix(unsigned k) {
  return __byte_perm(k * 0x9E3779B1u, 0u, 0x1032) * 0x85EBCA77u;
}

// f1 += m, f2 += m * m as 64-bit sums, both as multiply-adds (the FMA pipe,
// which the ranking leaves idle)
__device__ __forceinline__ void fp_add(unsigned long long& f1, unsigned long long& f2, int k) {
  const unsigned m = key_mix((unsigned)k);
  asm("mad.wide.u32 %0, %1, 1, %0;" : "+l"(f1) : "r"(m));
  asm("mad.wide.u32 %0, %1, %1, %0;" : "+l"(f2) : "r"(m));
}

// 64-bit look-back word of the checked last pass: flag (2 bits) | count (30)
// | the last key before the end of this tile's run of the digit (32)
__device__ __forceinline__ unsigned long long lb_word(unsigned flag, unsigned c, int k) {
  return ((unsigned long long)((flag << 30) | c) << 32) | (unsigned)k;
}

// The lanes holding the same 8-bit digit: one ballot per digit bit; a lane
// keeps the ballot where its own bit is set and its complement where it is
// clear.  Written as PTX so that each bit costs a predicate, a vote, a
// predicated complement and an AND (the compiler's code for the same C was
// measured 9% slower per pass).
__device__ __forceinline__ unsigned digit_peers(unsigned d) {
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    asm("{\n\t.reg .pred p;\n\t.reg .b32 m, t;\n\t"
        "and.b32 t, %1, %2;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "vote.sync.ballot.b32 m, p, 0xffffffff;\n\t"
        "@!p not.b32 m, m;\n\t"
        "and.b32 %0, %0, m;\n\t}"
        : "+r"(peers)
        : "r"(d), "r"(1u << b));
  }
  return peers;
}

// The block's fingerprint sums into dst with one pair of atomics per CTA
// (one pair per warp put some 10^5 same-address atomics on one L2 line per
// pass).  s_fp: 2 x (blockDim.x / 32) words of shared memory.  Contains
// __syncthreads: every thread of the block calls it.
__device__ __forceinline__ void fp_flush(unsigned long long f1, unsigned long long f2,
                                         unsigned long long* dst, unsigned long long* s_fp) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    f1 += __shfl_xor_sync(0xffffffffu, f1, o);
    f2 += __shfl_xor_sync(0xffffffffu, f2, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_fp[w] = f1;
    s_fp[nw + w] = f2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0, b = 0;
    for (int i = 0; i < nw; ++i) {
      a += s_fp[i];
      b += s_fp[nw + i];
    }
    atomicAdd(dst, a);
    atomicAdd(dst + 1, b);
  }
}

// ---------------------------------------------------------------------------
// FP: also the input's multiset fingerprint (only the permutation check
// needs it)
template <bool FLT, bool FP>
__global__ void __launch_bounds__(256) k_radix_hist(const int* __restrict__ in, long long n,
                                                    SortHdr* h, SortResult* res) {
  __shared__ unsigned sh[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  unsigned long long f1 = 0, f2 = 0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long start = 0;
  auto count = [&](int k) {
    const unsigned u = okey<FLT>(k);
    atomicAdd(&sh[0][u & 0xFFu], 1u);
    atomicAdd(&sh[1][(u >> 8) & 0xFFu], 1u);
    atomicAdd(&sh[2][(u >> 16) & 0xFFu], 1u);
    atomicAdd(&sh[3][u >> 24], 1u);
    if (FP) fp_add(f1, f2, k);
  };
  if (((uintptr_t)in & 15) == 0) {
    const long long nv = n >> 2;
    start = nv << 2;
    const int4* in4 = reinterpret_cast<const int4*>(in);
    long long v = tid;
    // two 16-byte loads in flight per thread before their keys are counted
    for (; v + stride < nv; v += 2 * stride) {
      const int4 q0 = __ldcs(in4 + v), q1 = __ldcs(in4 + v + stride);
      count(q0.x); count(q0.y); count(q0.z); count(q0.w);
      count(q1.x); count(q1.y); count(q1.z); count(q1.w);
    }
    for (; v < nv; v += stride) {
      const int4 q = __ldcs(in4 + v);
      count(q.x); count(q.y); count(q.z); count(q.w);
    }
  }
  for (long long i = start + tid; i < n; i += stride) count(in[i]);
  __shared__ unsigned long long s_fp[2 * 8];
  if (FP) fp_flush(f1, f2, res->fp_in, s_fp);
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) {
    const unsigned c = (&sh[0][0])[i];
    if (c) atomicAdd(&(&h->hist[0][0])[i], c);
  }
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(&h->done_ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // per-digit start offsets: one exclusive scan over the block per histogram
  // (thread d owns digit d)
  __shared__ unsigned s_warp[kWarps];
  unsigned c[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) c[p] = __ldcg(&h->hist[p][threadIdx.x]);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    h->offs[p][threadIdx.x] = block_excl_scan(c[p], s_warp);
    __syncthreads();
  }
  if (threadIdx.x == 0) res->cnt_in = n;
}

// ---------------------------------------------------------------------------
template <bool CK>
struct SortSmem {
  int keys[kTile + 1];   // + a sentinel after the tile's keys (checked pass)
  unsigned whist[kWarps][kRadix];
  // checked pass: the last key of each warp's keys of each digit, so that a
  // tile's digit runs know their last keys before the tile is sorted in
  // shared memory
  int lastk[CK ? kWarps : 1][kRadix];
  int gbase[kRadix];
  unsigned warp[kWarps];
  unsigned tile;
  int timeout;
  unsigned long long fp[2 * kWarps];
  unsigned short rank[kTile];
};

// One tile of one pass.  FULL: the tile holds kTile keys (every tile but the
// last), so no index is checked against n.
template <bool LAST, bool CHECK, bool FULL, bool FLT>
__device__ __forceinline__ void onesweep_tile(SortSmem<LAST && CHECK>& sm, const int* __restrict__ in,
                                              int* __restrict__ out, long long n, int pass,
                                              SortHdr* h, unsigned* st32,
                                              unsigned long long* st64, SortResult* res,
                                              unsigned tile, const LookbackCtl lb) {
  int* const s_keys = sm.keys;
  unsigned (*const s_whist)[kRadix] = sm.whist;
  int* const s_gbase = sm.gbase;
  unsigned short* const s_rank = sm.rank;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long base = (long long)tile * kTile;
  const unsigned dsel = 0x4440u | (unsigned)pass;   // digit selector of this pass
  const int valid_cnt = FULL ? kTile : (int)(n - base < kTile ? n - base : kTile);
  // the look-back testing switch: a tile that publishes nothing, a short wait
  const bool publish = (int)tile != lb.skip_tile;
  const unsigned spin_limit = lb.spin_limit ? lb.spin_limit : kSpinLimit;

  // load: warp w owns keys [w*kWarpKeys, (w+1)*kWarpKeys) of the tile, 32
  // consecutive per round
  int key[kKpt];
  const long long wbase = base + (long long)w * kWarpKeys + lane;
  constexpr bool full = FULL;
  const int lbase = w * kWarpKeys + lane;   // this thread's keys: s_keys[lbase + 32 r]
#pragma unroll
  for (int r = 0; r < kKpt; ++r) {
    const long long idx = wbase + r * 32;
    key[r] = (full || idx < n) ? __ldcs(in + idx) : 0;
  }

  // stable rank of each key among the warp's keys of the same digit; the
  // lanes holding the same digit are found with match_any, or with eight
  // ballots (one per digit bit) and a ninth that separates the padding lanes
  // of a partial tile.  match_any costs grow with the number of distinct
  // digits among the lanes (uniform keys: about 28 of 32), so it takes one
  // round in kMatchEvery, where it overlaps the ballots of the others
  const unsigned lt = lanemask_lt();
#pragma unroll
  for (int r = 0; r < kKpt; ++r) {
    const bool ok = full || (wbase + r * 32) < n;
    const unsigned d = digit_of<LAST, FLT>(key[r], dsel);
    unsigned peers;
    if (r % kMatchEvery == kMatchEvery - 1) {
      peers = __match_any_sync(0xffffffffu, ok ? d : 0x1000u);
    } else {
      peers = digit_peers(d);
      if (!full) {
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        peers &= ok ? bal : ~bal;
      }
    }
    const unsigned before = __popc(peers & lt);
    const unsigned prev = ok ? s_whist[w][d] : 0u;
    __syncwarp();
    if (ok && before == 0) s_whist[w][d] = prev + __popc(peers);
    // checked pass: the highest lane of the group holds the warp's latest
    // key of this digit (rounds are in key order)
    if (LAST && CHECK && ok && (peers >> lane) == 1u) sm.lastk[w][d] = key[r];
    __syncwarp();
    s_rank[lbase + r * 32] = (unsigned short)(prev + before);
  }
  __syncthreads();

  // per digit (threads 0..255): tile count and exclusive offsets of the warps
  const bool dig = kSortBlock == kRadix || tid < kRadix;
  unsigned cnt = 0;
  int last_key = 0;   // checked pass: last key of this tile's run of digit tid
  if (dig) {
    const int d = tid;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const unsigned t = s_whist[ww][d];
      s_whist[ww][d] = cnt;
      cnt += t;
      if (LAST && CHECK && t) last_key = sm.lastk[ww][d];
    }
    // publish the tile aggregate as early as possible
    if (publish) {
      if (!(LAST && CHECK))
        st_relaxed(&st32[(size_t)tile * kRadix + tid], ((tile == 0 ? kPre : kAgg) << 30) | cnt);
      else
        st_relaxed64(&st64[(size_t)tile * kRadix + tid], lb_word(tile == 0 ? kPre : kAgg, cnt, last_key));
    }
  }
  const unsigned start = block_excl_scan(cnt, sm.warp);
  if (dig) {
    // from here s_whist[w][d] is where warp w's keys of digit d start in the tile
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s_whist[ww][tid] += start;
  }
  __syncthreads();

  // sort the tile in shared memory by digit (stable)
#pragma unroll
  for (int r = 0; r < kKpt; ++r) {
    if (full || (wbase + r * 32) < n) {
      const unsigned d = digit_of<LAST, FLT>(key[r], dsel);
      s_keys[s_whist[w][d] + s_rank[lbase + r * 32]] = key[r];
    }
  }
  // checked pass: a sentinel above every key (okey 0xFFFFFFFF) after the
  // last one, so that every key has a successor to be compared with
  if (LAST && CHECK && tid == 0) s_keys[valid_cnt] = FLT ? 0x7FFFFFFF : INT_MAX;
  __syncthreads();

  // decoupled look-back: exclusive prefix of digit `tid` over earlier tiles
  const int d = tid;
  unsigned long long excl = 0;
  bool timeout = false;
  if (!dig) {
    // no digit of this thread
  } else if (!(LAST && CHECK)) {
    if (tile > 0) {
      // walk back from tile - 1 to the nearest inclusive prefix; a word not
      // yet published stops the walk there and is polled again.  Every word
      // is written once as an aggregate and once as an inclusive prefix (tile
      // 0 only as the prefix), so any published value read is a valid step.
      // Below tile 0 stands an empty inclusive prefix (never reached: tile
      // 0's word is one).
      long long j = (long long)tile - 1;
      unsigned spins = 0;
      bool done = false;
      while (!done) {
        unsigned v[kLook];
#pragma unroll
        for (int u = 0; u < kLook; ++u)
          v[u] = j - u >= 0 ? ld_relaxed(&st32[(size_t)(j - u) * kRadix + d]) : (kPre << 30);
        int u = 0;
#pragma unroll
        for (; u < kLook; ++u) {
          const unsigned flag = v[u] >> 30;
          if (flag == 0) break;
          excl += v[u] & kCntMask;
          if (flag == kPre) {
            done = true;
            break;
          }
        }
        if (done) break;
        if (u < kLook) {
          j -= u;
          if (++spins > spin_limit) { timeout = true; break; }
          if (spins > 32) __nanosleep(64);
        } else {
          j -= kLook;
        }
      }
      if (publish) st_relaxed(&st32[(size_t)tile * kRadix + d], (kPre << 30) | (unsigned)(excl + cnt));
    }
  } else {
    // 64-bit words: flag(2) | count(30) | last key of the digit run (32),
    // the aggregate published above with the run's last key
    const int first_key = cnt ? s_keys[start] : 0;
    auto word = lb_word;
    bool found = false;
    int pred_last = 0;
    if (tile > 0) {
      // the same windowed walk as above; the first run met with keys
      // gives the last key before this tile's run
      long long j = (long long)tile - 1;
      unsigned spins = 0;
      bool done = false;
      while (!done) {
        unsigned long long v[kLookWide];
#pragma unroll
        for (int u = 0; u < kLookWide; ++u)
          v[u] = j - u >= 0 ? ld_relaxed64(&st64[(size_t)(j - u) * kRadix + d])
                            : word(kPre, 0u, 0);
        int u = 0;
#pragma unroll
        for (; u < kLookWide; ++u) {
          const unsigned hi = (unsigned)(v[u] >> 32);
          const unsigned flag = hi >> 30;
          if (flag == 0) break;
          const unsigned c = hi & kCntMask;
          if (!found && c > 0) {
            found = true;
            pred_last = (int)(unsigned)v[u];
          }
          excl += c;
          if (flag == kPre) {
            done = true;
            break;
          }
        }
        if (done) break;
        if (u < kLookWide) {
          j -= u;
          if (++spins > spin_limit) { timeout = true; break; }
          if (spins > 32) __nanosleep(64);
        } else {
          j -= kLookWide;
        }
      }
      const int carry = cnt ? last_key : pred_last;
      if (publish) st_relaxed64(&st64[(size_t)tile * kRadix + d], word(kPre, (unsigned)(excl + cnt), carry));
    }
    // the first key of this run must not be below the last key before it
    if (cnt && found && okey<FLT>(first_key) < okey<FLT>(pred_last)) {
      const long long pos = (long long)h->offs[pass][d] + (long long)excl - 1;
      atomicMax(&res->unsorted_enc, ~(unsigned long long)pos);
    }
  }
  if (timeout) {
    atomicExch(&res->timeout, 1);
    atomicExch(&h->failed, 1);
    sm.timeout = 1;
  }
  if (dig) s_gbase[d] = (int)h->offs[pass][d] + (int)excl - (int)start;
  __syncthreads();
  // a look-back that gave up leaves this tile's offsets unknown: write nothing
  const bool write = sm.timeout == 0;

  // write the tile out in digit runs
  unsigned long long f1 = 0, f2 = 0;
  int bad = INT_MAX;
#pragma unroll 4
  for (int i = tid; i < valid_cnt; i += kSortBlock) {
    const int k = s_keys[i];
    const unsigned dk = digit_of<LAST, FLT>(k, dsel);
    const int pos = s_gbase[dk] + i;
    // the last pass runs after the host's contract-test fault planting (a key
    // changed between passes can carry a digit run past the histogram's
    // offsets): there, never write outside the output.  Earlier passes read
    // what the previous pass wrote, whose digit counts are the histogram's.
    if (write && (!LAST || (unsigned)pos < (unsigned)n)) __stcs(out + pos, k);
    if (LAST && CHECK) {
      fp_add(f1, f2, k);
      // the tile is sorted by the most significant digit and each digit
      // run by the lower ones: every adjacent pair of the tile is in order
      // (runs of different digits trivially), and pairs inside a run are
      // adjacent in the output too
      const int k2 = s_keys[i + 1];
      const bool desc = FLT ? okey<true>(k) > okey<true>(k2) : k > k2;
      if (desc) bad = min(bad, pos);
    }
  }
  if (LAST && CHECK) {
    fp_flush(f1, f2, res->fp_out, sm.fp);
    unsigned long long enc = bad != INT_MAX ? ~(unsigned long long)(long long)bad : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long e2 = __shfl_xor_sync(0xffffffffu, enc, o);
      enc = e2 > enc ? e2 : enc;
    }
    if (lane == 0 && enc) atomicMax(&res->unsorted_enc, enc);
    if (tid == 0) {
      atomicAdd((unsigned long long*)&res->cnt_out, (unsigned long long)valid_cnt);
      if (tile == 0) res->checked = 1;
    }
  }
}

template <bool LAST, bool CHECK, bool FLT>
__global__ void __launch_bounds__(kSortBlock, kSortMinBlocks) k_onesweep(
    const int* __restrict__ in, int* __restrict__ out, long long n, int pass, SortHdr* h,
    unsigned* st32, unsigned long long* st64, SortResult* res, unsigned ahead,
    const LookbackCtl lb) {
  __shared__ SortSmem<LAST && CHECK> sm;
  const int tid = threadIdx.x;
  if (tid == 0) {
    // an earlier pass whose look-back gave up left its output incomplete:
    // this pass does nothing
    sm.timeout = pass > 0 ? *reinterpret_cast<volatile int*>(&h->failed) : 0;
    if (!sm.timeout) sm.tile = atomicAdd(&h->tile_ctr[pass], 1u);
  }
  for (int i = tid; i < kWarps * kRadix; i += kSortBlock) (&sm.whist[0][0])[i] = 0;
  __syncthreads();
  if (sm.timeout) return;
  const unsigned tile = sm.tile;
  // tiles are taken in ticket order: the tile one resident wave ahead is
  // fetched into L2 now, so that its CTA's key loads hit L2
  if (tid == 0 && ((uintptr_t)in & 15) == 0) {
    const long long t2 = (long long)tile + ahead;
    if ((t2 + 1) * kTile <= n)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(in + t2 * kTile),
                   "r"((unsigned)(kTile * sizeof(int)))
                   : "memory");
  }
  if ((long long)(tile + 1) * kTile <= n)
    onesweep_tile<LAST, CHECK, true, FLT>(sm, in, out, n, pass, h, st32, st64, res, tile, lb);
  else
    onesweep_tile<LAST, CHECK, false, FLT>(sm, in, out, n, pass, h, st32, st64, res, tile, lb);
}

// ---------------------------------------------------------------------------
// Stand-alone checks (re-read the vector).

// is_sorted: first i with x[i] > x[i+1]; signed int32, or the IEEE
// comparison of binary32 values (NaN compares false)
template <bool FLT>
__device__ __forceinline__ bool gt_key(int a, int b) {
  return FLT ? (__int_as_float(a) > __int_as_float(b)) : (a > b);
}

template <bool FLT>
__global__ void __launch_bounds__(256) k_check_sorted(const int* __restrict__ x, long long n,
                                                      SortResult* res) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long bad = -1;
  for (long long i = tid; i + 1 < n && bad < 0; i += stride)
    if (gt_key<FLT>(__ldg(x + i), __ldg(x + i + 1))) bad = i;
  unsigned long long enc = bad >= 0 ? ~(unsigned long long)bad : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long e2 = __shfl_xor_sync(0xffffffffu, enc, o);
    enc = e2 > enc ? e2 : enc;
  }
  if ((threadIdx.x & 31) == 0 && enc) atomicMax(&res->unsorted_enc, enc);
}

__global__ void __launch_bounds__(256) k_fingerprint(const int* __restrict__ x, long long n,
                                                     unsigned long long* fp, long long* cnt) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long f1 = 0, f2 = 0;
  for (long long i = tid; i < n; i += stride) fp_add(f1, f2, __ldg(x + i));
  __shared__ unsigned long long s_fp[2 * 8];
  fp_flush(f1, f2, fp, s_fp);
  if (tid == 0) *cnt = n;
}

struct Layout {
  size_t st32[3];
  size_t st64;
  size_t zero_bytes;
  size_t tmp;
  size_t total;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(long long n) {
  Layout L;
  const size_t ntiles = (size_t)((n + kTile - 1) / kTile);
  size_t off = align256(sizeof(SortHdr));
  for (int p = 0; p < 3; ++p) {
    L.st32[p] = off;
    off = align256(off + ntiles * kRadix * sizeof(unsigned));
  }
  L.st64 = off;
  off = align256(off + ntiles * kRadix * sizeof(unsigned long long));
  L.zero_bytes = off;
  L.tmp = off;
  off = align256(off + (size_t)n * sizeof(int));
  L.total = off;
  return L;
}

int grid_for(long long units, int num_sms, int per_sm) {
  long long g = (units + 255) / 256;
  long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t sort_scratch_bytes(long long n) { return layout(n).total; }

namespace {

template <bool FLT>
cudaError_t sort_impl(const int32_t* in, int32_t* out, long long n, bool contracts,
                        void* scratch, SortResult* res, cudaStream_t s, int num_sms,
                        int64_t* kernels, const SortInject* inject, Prof* prof,
                        const LookbackCtl lb) {
  if (n <= 0) return cudaSuccess;
  const Layout L = layout(n);
  char* base = static_cast<char*>(scratch);
  SortHdr* h = reinterpret_cast<SortHdr*>(base);
  unsigned* st32[3];
  for (int p = 0; p < 3; ++p) st32[p] = reinterpret_cast<unsigned*>(base + L.st32[p]);
  unsigned long long* st64 = reinterpret_cast<unsigned long long*>(base + L.st64);
  int* tmp = reinterpret_cast<int*>(base + L.tmp);
  cudaError_t e = cudaMemsetAsync(base, 0, L.zero_bytes, s);
  if (e != cudaSuccess) return e;
  prof_begin(prof, "radix_hist", s);
  if (contracts)
    k_radix_hist<FLT, true><<<grid_for((n + 3) / 4 / 8, num_sms, 8), 256, 0, s>>>(in, n, h, res);
  else
    k_radix_hist<FLT, false><<<grid_for((n + 3) / 4 / 8, num_sms, 8), 256, 0, s>>>(in, n, h, res);
  prof_end(prof, s);
  const unsigned ntiles = (unsigned)((n + kTile - 1) / kTile);
  const unsigned ahead = (unsigned)num_sms * kSortMinBlocks;
  prof_begin(prof, "onesweep", s);
  k_onesweep<false, false, FLT><<<ntiles, kSortBlock, 0, s>>>(in, tmp, n, 0, h, st32[0], st64, res, ahead, lb);
  prof_end(prof, s);
  prof_begin(prof, "onesweep", s);
  k_onesweep<false, false, FLT><<<ntiles, kSortBlock, 0, s>>>(tmp, out, n, 1, h, st32[1], st64, res, ahead, lb);
  prof_end(prof, s);
  prof_begin(prof, "onesweep", s);
  k_onesweep<false, false, FLT><<<ntiles, kSortBlock, 0, s>>>(out, tmp, n, 2, h, st32[2], st64, res, ahead, lb);
  prof_end(prof, s);
  if (inject && inject->mode == 1 && inject->i < n && inject->j < n) {
    // swap through the (now free) output buffer: stream-ordered host copies
    e = cudaMemcpyAsync(out, tmp + inject->i, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp + inject->i, tmp + inject->j, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tmp + inject->j, out, sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  } else if (inject && inject->mode == 2 && inject->i < n) {
    static int value;   // pageable source: the copy is staged before it returns
    value = (int)inject->j;
    e = cudaMemcpyAsync(tmp + inject->i, &value, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
  }
  // the last pass uses the (zeroed) 64-bit area; without contracts only its
  // first half, as 32-bit words
  unsigned* st_last = reinterpret_cast<unsigned*>(st64);
  prof_begin(prof, contracts ? "onesweep_last_checked" : "onesweep", s);
  if (contracts)
    k_onesweep<true, true, FLT><<<ntiles, kSortBlock, 0, s>>>(tmp, out, n, 3, h, st_last, st64, res, ahead, lb);
  else
    k_onesweep<true, false, FLT><<<ntiles, kSortBlock, 0, s>>>(tmp, out, n, 3, h, st_last, st64, res, ahead, lb);
  prof_end(prof, s);
  *kernels += 5;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sort(const int32_t* in, int32_t* out, long long n, bool contracts,
                        void* scratch, SortResult* res, cudaStream_t s, int num_sms,
                        int64_t* kernels, const SortInject* inject, Prof* prof, bool flt,
                        const LookbackCtl& lb) {
  return flt ? sort_impl<true>(in, out, n, contracts, scratch, res, s, num_sms, kernels, inject,
                               prof, lb)
             : sort_impl<false>(in, out, n, contracts, scratch, res, s, num_sms, kernels, inject,
                                prof, lb);
}

size_t check_scratch_bytes() { return 0; }

cudaError_t launch_check_sorted(const int32_t* x, long long n, SortResult* res, void*,
                                cudaStream_t s, int num_sms, int64_t* kernels, Prof* prof,
                                bool flt) {
  if (n <= 1) return cudaSuccess;
  prof_begin(prof, "check_sorted", s);
  if (flt) k_check_sorted<true><<<grid_for(n, num_sms, 8), 256, 0, s>>>(x, n, res);
  else k_check_sorted<false><<<grid_for(n, num_sms, 8), 256, 0, s>>>(x, n, res);
  prof_end(prof, s);
  *kernels += 1;
  return cudaGetLastError();
}

cudaError_t launch_check_perm(const int32_t* x, const int32_t* ref, long long n,
                              SortResult* res, void*, cudaStream_t s, int num_sms,
                              int64_t* kernels, Prof* prof) {
  if (n <= 0) return cudaSuccess;
  prof_begin(prof, "fingerprint", s);
  k_fingerprint<<<grid_for(n, num_sms, 8), 256, 0, s>>>(x, n, res->fp_out, &res->cnt_out);
  k_fingerprint<<<grid_for(n, num_sms, 8), 256, 0, s>>>(ref, n, res->fp_in, &res->cnt_in);
  prof_end(prof, s);
  *kernels += 2;
  return cudaGetLastError();
}

}  // namespace sgk
