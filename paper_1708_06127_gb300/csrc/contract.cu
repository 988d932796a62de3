// Cluster contraction (Sec. 4.1, "contract it"; contraction semantics, Sec. 3):
// every block of a labelling becomes one vertex, intra-block edges vanish and
// parallel edges between two blocks merge with summed weight.  Block ids are the
// ranks of the label values.  Steps: relabel (flag + scan), the optional correcting
// step, pre-merge per fine vertex (lp.cu), then either
//   * the cluster merge: a counting sort of the pre-merged pairs by source cluster,
//     then a warp per cluster of at most kMergeMax pairs (registers, or a bitonic sort
//     in shared memory), a block per cluster of at most kMergeBlockMax, and one radix
//     sort for all larger ("giant") clusters together; each writes its distinct
//     targets in ascending order at the front of its segment, or
//   * pair build, LSD radix sort on (cid v, cid u) and a run reduction (when the giant
//     clusters hold more than half of the pairs).
#include <limits.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "kernels.cuh"
#include "prims.cuh"
#include "regvisit.cuh"

namespace vc {

__global__ void mark_labels_k(const int32_t* __restrict__ lab, int64_t n, int32_t* __restrict__ flags) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (lab[v] >= 0) flags[lab[v]] = 1;  // label -1: the vertex is dropped (batches)
}

__global__ void apply_rank_k(const int32_t* __restrict__ lab, int64_t n, const int32_t* __restrict__ rank,
                             int32_t* __restrict__ cid) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    cid[v] = lab[v] >= 0 ? rank[lab[v]] : -1;
}

void relabel(const int32_t* lab, int64_t n, int32_t* cid, ContractScratch& cs, int* c_dev, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(cs.flags, 0, sizeof(int32_t) * n, s));
  int grid = grid_for(n, 256, kSMs * 8);
  mark_labels_k<<<grid, 256, 0, s>>>(lab, n, cs.flags);
  count_launch();
  VC_CHECK_LAUNCH();
  exclusive_scan<int, int>(cs.flags, cs.rank, n, c_dev, cs.scan_scr32, s);
  apply_rank_k<<<grid, 256, 0, s>>>(lab, n, cs.rank, cid);
  count_launch();
  VC_CHECK_LAUNCH();
}

// W lanes per fine vertex copy its pre-merged list into the contiguous pair arrays: a
// thread per vertex where lists are short (two entries on average on clustered graphs),
// wider groups where they run up to the degree (unclustered graphs).
template <int W>
__global__ void build_pairs_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cid,
                              const int32_t* __restrict__ cnt, const long long* __restrict__ pos, PairOut in,
                              int bits, unsigned long long* __restrict__ keys, long long* __restrict__ vals) {
  const int lane = threadIdx.x & (W - 1);
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / W);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / W; v < n; v += groups) {
    const int k = cnt[v];
    if (k == 0) continue;
    const int64_t src = off[v];
    const long long dst = pos[v];
    const unsigned long long hi = (unsigned long long)cid[v] << bits;
    for (int j = lane; j < k; j += W) {
      int32_t kk;
      long long x;
      in.get(v, src, j, &kk, &x);
      keys[dst + j] = hi | (unsigned long long)(uint32_t)kk;
      vals[dst + j] = x;
    }
  }
}

void build_pairs(const GraphView& g, const int32_t* cid, const ContractScratch& cs, int bits, int64_t pairs,
                 unsigned long long* keys, long long* vals, cudaStream_t s) {
  const PairOut in{cs.tmp_key, cs.tmp_val, cs.cmp_key, cs.cmp_val};
  if (pairs <= 2 * g.n)
    build_pairs_k<1><<<grid_for(g.n, 256, kSMs * 8), 256, 0, s>>>(g.n, g.off, cid, cs.cnt, cs.pos, in, bits, keys, vals);
  else if (pairs <= 16 * g.n)
    build_pairs_k<8><<<grid_for(g.n, 32, kSMs * 16), 256, 0, s>>>(g.n, g.off, cid, cs.cnt, cs.pos, in, bits, keys, vals);
  else
    build_pairs_k<32><<<grid_for(g.n, 8, kSMs * 16), 256, 0, s>>>(g.n, g.off, cid, cs.cnt, cs.pos, in, bits, keys, vals);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void run_heads_k(const unsigned long long* __restrict__ keys, int64_t m, int32_t* __restrict__ heads) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Every element adds its value to its run's output: run index = (heads up to and
// including it) - 1 = hpos[i] + heads[i] - 1.  The lanes of a warp in one run add their
// sum once (runs can be long: a giant cluster's pairs to one target); cw must be zero.
// The run's head writes the target and source ids.
__global__ void run_reduce_k(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
                             int64_t m, int bits, const int32_t* __restrict__ heads,
                             const long long* __restrict__ hpos, int32_t* __restrict__ cadj,
                             long long* __restrict__ cw, int32_t* __restrict__ cv) {
  const unsigned long long mask = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1ULL);
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; b < m;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = b + lane;
    const bool ok = i < m;
    const long long r = ok ? hpos[i] + heads[i] - 1 : -1 - lane;
    const long long x = ok ? vals[i] : 0;
    // runs are consecutive lanes: a segmented inclusive sum, added by each run's last lane
    long long sum = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, sum, o);
      const long long ry = __shfl_up_sync(0xffffffffu, r, o);
      if (lane >= o && ry == r) sum += y;
    }
    const long long rn = __shfl_down_sync(0xffffffffu, r, 1);
    if (ok && (lane == 31 || rn != r)) atomicAdd((unsigned long long*)(cw + r), (unsigned long long)sum);
    if (ok && heads[i]) {
      const unsigned long long k = keys[i];
      cadj[r] = (int32_t)(k & mask);
      cv[r] = (int32_t)(k >> bits);
    }
  }
}

// offsets from the source-vertex column of the (sorted) unique entries
__global__ void build_offsets_k(const int32_t* __restrict__ cv, const long long* __restrict__ nnz_dev,
                                int64_t c, int64_t* __restrict__ coff) {
  const long long m = *nnz_dev;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m == 0) {
    for (int64_t x = t0; x <= c; x += T) coff[x] = 0;
    return;
  }
  for (int64_t j = t0; j <= m; j += T) {
    // entry j starts the lists of every vertex in (cv[j-1], cv[j]]
    int64_t lo = (j == 0) ? -1 : cv[j - 1];
    int64_t hi = (j == m) ? c : cv[j];
    for (int64_t x = lo + 1; x <= hi; ++x) coff[x] = j;
  }
}

void reduce_pairs(const unsigned long long* keys, const long long* vals, int64_t pairs, int bits,
                  int64_t c, int32_t* heads, long long* hpos, long long* scan_scr, int64_t* coff,
                  int32_t* cadj, long long* cw, int32_t* cv_tmp, long long* nnz_dev, cudaStream_t s) {
  int grid = grid_for(pairs, 256, kSMs * 8);
  if (pairs > 0) {
    run_heads_k<<<grid, 256, 0, s>>>(keys, pairs, heads);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  exclusive_scan<int, long long>(heads, hpos, pairs, nnz_dev, scan_scr, s);
  if (pairs > 0) {
    VC_CUDA(cudaMemsetAsync(cw, 0, sizeof(long long) * pairs, s));
    run_reduce_k<<<grid, 256, 0, s>>>(keys, vals, pairs, bits, heads, hpos, cadj, cw, cv_tmp);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  build_offsets_k<<<grid_for(pairs + c + 1, 256, kSMs * 8), 256, 0, s>>>(cv_tmp, nnz_dev, c, (int64_t*)coff);
  count_launch();
  VC_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- cluster merge
// Warp-level grouping of the lanes whose vertices share a cluster (consecutive
// vertices often do), so that one atomic per group and warp moves its counter.
// Returns the sum of k over the lane's group and the sum over the group's lower
// lanes; sk is the warp's 32-entry scratch.
__device__ __forceinline__ void group_sums(int32_t c, int k, int lane, int* sk, unsigned* peers_out, int* total,
                                           int* below) {
  const unsigned peers = __match_any_sync(0xffffffffu, c);
  sk[lane] = k;
  __syncwarp();
  int t = 0, b = 0;
  for (unsigned m = peers; m; m &= m - 1) {
    const int j = __ffs(m) - 1;
    t += sk[j];
    if (j < lane) b += sk[j];
  }
  __syncwarp();
  *peers_out = peers;
  *total = t;
  *below = b;
}

// The largest pairs-per-cluster count and the total, over ccount[0, n).
__global__ void __launch_bounds__(256) cluster_stats_k(int64_t n, const int32_t* __restrict__ ccount, int* maxt,
                                                       long long* pairs, int* ngiant, long long* gpairs) {
  __shared__ int s_max;
  __shared__ unsigned long long s_sum;
  if (threadIdx.x == 0) { s_max = 0; s_sum = 0; }
  __syncthreads();
  int top = 0;
  long long sum = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = ccount[i];
    top = max(top, x);
    sum += x;
    if (x > kMergeBlockMax) {  // rare
      atomicAdd(ngiant, 1);
      atomicAdd((unsigned long long*)gpairs, (unsigned long long)x);
    }
  }
  const unsigned wtop = __reduce_max_sync(0xffffffffu, (unsigned)top);
  const long long w = warp_sum(sum);
  if ((threadIdx.x & 31) == 0) {
    if (wtop) atomicMax(&s_max, (int)wtop);
    if (w) atomicAdd(&s_sum, (unsigned long long)w);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_max) atomicMax(maxt, s_max);
    if (s_sum) atomicAdd((unsigned long long*)pairs, s_sum);
  }
}

// The pieces of a warp copied with the lanes on consecutive entries: lane j brings a
// piece of len entries (0: none) read from src + i and written to dst + i (i < len);
// load(s) reads the entry at source index s and put(d, j, value) writes it at
// destination index d (j: the piece's lane).  kPieceUnroll entries per lane at a time,
// all loads before the stores, so that they are in flight together.  Long lists of a
// few lanes and short lists of many lanes keep every lane busy alike.
constexpr int kPieceUnroll = 4;
template <typename T, typename LOAD, typename PUT>
__device__ __forceinline__ void warp_pieces(int64_t len, int64_t src, int64_t dst, LOAD load, PUT put) {
  const int lane = threadIdx.x & 31;
  int64_t incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
  const int64_t excl = incl - len;  // where lane j's piece starts among the laid-out pieces
  for (int64_t p0 = 0; p0 < total; p0 += 32 * kPieceUnroll) {
    int jj[kPieceUnroll];
    int64_t sp[kPieceUnroll], dp[kPieceUnroll];
    T val[kPieceUnroll];
#pragma unroll
    for (int u = 0; u < kPieceUnroll; ++u) {
      const int64_t p = p0 + lane + 32 * u;
      // the piece holding place p: the last lane whose piece starts at or before p
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int t = j + step;
        const int64_t ex = __shfl_sync(0xffffffffu, excl, t & 31);
        if (t < 32 && ex <= p) j = t;
      }
      const int64_t i = p - __shfl_sync(0xffffffffu, excl, j);
      sp[u] = __shfl_sync(0xffffffffu, src, j) + i;
      dp[u] = __shfl_sync(0xffffffffu, dst, j) + i;
      jj[u] = p < total ? j : -1;
    }
#pragma unroll
    for (int u = 0; u < kPieceUnroll; ++u)
      if (jj[u] >= 0) val[u] = load(sp[u]);
#pragma unroll
    for (int u = 0; u < kPieceUnroll; ++u)
      if (jj[u] >= 0) put(dp[u], jj[u], val[u]);
  }
}

struct KeyVal {
  int32_t k;
  long long v;
};

// Counting-sort scatter: the pre-merged pairs of fine vertex v move, in one piece,
// into their cluster's segment (cursor = the segments' running write positions).
// Lists of more than kScatterWarpMin pairs are copied by the whole warp.
constexpr int kScatterWarpMin = 16;
__global__ void __launch_bounds__(256) cluster_scatter_k(int64_t n, const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ cid,
                                                         const int32_t* __restrict__ cnt, PairOut in,
                                                         long long* __restrict__ cursor, int32_t* __restrict__ seg_key,
                                                         long long* __restrict__ seg_val) {
  __shared__ int s_k[8][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t v = base + lane;
    const int k = v < n ? cnt[v] : 0;
    const int32_t c = k > 0 ? cid[v] : -1;
    unsigned peers;
    int t, b;
    group_sums(c, k, lane, s_k[wid], &peers, &t, &b);
    const int leader = __ffs(peers) - 1;
    long long at = 0;
    if (c >= 0 && lane == leader) at = atomicAdd((unsigned long long*)&cursor[c], (unsigned long long)t);
    at = __shfl_sync(0xffffffffu, at, leader);
    const long long dst = at + b;
    if (c >= 0) {
      // the first kPairSlots pairs from the dense strip, all in flight at once
      int32_t kk[kPairSlots];
      long long vv[kPairSlots];
#pragma unroll
      for (int j = 0; j < kPairSlots; ++j)
        if (j < k) { kk[j] = in.ckey[v * kPairSlots + j]; vv[j] = in.cval[v * kPairSlots + j]; }
#pragma unroll
      for (int j = 0; j < kPairSlots; ++j)
        if (j < k) { seg_key[dst + j] = kk[j]; seg_val[dst + j] = vv[j]; }
      if (k > kPairSlots && k <= kScatterWarpMin) {  // short rest: this thread
        const int64_t src = off[v];
        for (int j = kPairSlots; j < k; ++j) {
          seg_key[dst + j] = in.tkey[src + j];
          seg_val[dst + j] = in.tval[src + j];
        }
      }
    }
    // the rest of the long lists, laid end to end over the lanes (coalesced)
    const bool longl = c >= 0 && k > kScatterWarpMin;
    if (__any_sync(0xffffffffu, longl)) {
      warp_pieces<KeyVal>(
          longl ? (int64_t)(k - kPairSlots) : 0, longl ? off[v] + kPairSlots : 0, dst + kPairSlots,
          [&](int64_t at) { return KeyVal{in.tkey[at], in.tval[at]}; },
          [&](int64_t at, int, const KeyVal& kv) {
            seg_key[at] = kv.k;
            seg_val[at] = kv.v;
          });
    }
  }
}

// A warp per cluster of at most kMergeMax pairs, the distinct targets written back in
// ascending order at the front of the segment; dcount[c] = their number.  The pairs go
// into registers and the warp takes one step per distinct target (summing its
// weights) while targets are few; a cluster reaching kMergeWarpKeys targets is sorted
// instead, in the warp's shared-memory buffer (bitonic network), and every run head
// sums its run (a step per target costs slots x compares, which only pays while
// targets are few).  With sort_first (a contraction whose clusters are mostly one or
// two vertices: nearly every pair its own target) a cluster of at least kMergeSortMin
// pairs is sorted without walking first.
constexpr int kMergeWarpKeys = 32;
constexpr int kMergeSortMin = 12;

__global__ void __launch_bounds__(256) cluster_merge_k(int64_t c, const long long* __restrict__ cbase,
                                                       int32_t* __restrict__ seg_key, long long* __restrict__ seg_val,
                                                       int32_t* __restrict__ dcount, bool sort_first) {
  constexpr int S = kMergeMax / 32;
  __shared__ int32_t sk_all[8][kMergeMax];
  __shared__ long long sv_all[8][kMergeMax];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* sk = sk_all[wid];
  long long* sv = sv_all[wid];
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < c; x += warps) {
    const long long b = cbase[x];
    const int T = (int)(cbase[x + 1] - b);
    if (T > kMergeMax) continue;  // the block kernel takes it
    RegList<S> L;
    L.slots = (T + 31) >> 5;
    L.todo = 0;
#pragma unroll
    for (int r = 0; r < S; ++r) {
      const int i = lane + 32 * r;
      L.k[r] = -1;
      L.wt[r] = 0;
      if (32 * r < T && i < T) {  // 32 r < T is the same in every lane
        L.k[r] = seg_key[b + i];
        L.wt[r] = seg_val[b + i];
        L.todo |= 1u << r;
      }
    }
    bool walk = !sort_first || T < kMergeSortMin;
    if (walk && T >= kMergeSortMin) {
      // probe: the distinct targets among the first row's pairs (one match); a row more
      // than half distinct (a cluster of one or two vertices of a weakly clustered
      // graph, or a long run of an exact-step round) is sorted without walking first
      const bool use = lane < T;
      const unsigned long long tag =
          use ? (unsigned long long)(uint32_t)L.k[0] : (0xffffffff00000000ull | (unsigned long long)lane);
      const unsigned peers = __match_any_sync(0xffffffffu, tag);
      const int nd = __popc(__ballot_sync(0xffffffffu, use && (__ffs(peers) - 1) == lane));
      if (2 * nd > (T < 32 ? T : 32)) walk = false;
    }
    if (walk) {
      int made = 0;  // warp-uniform
      int32_t ok = INT_MAX;
      long long ov = 0;
      reg_visit<long long, long long, 32, S>(L, 0xffffffffu, [&](int32_t key, long long total) {
        if (lane == made) { ok = key; ov = total; }
        return ++made >= kMergeWarpKeys;
      });
      if (made < kMergeWarpKeys) {
        // lane i holds target i: its rank among the made targets places it
        int rank = 0;
        for (int j = 0; j < made; ++j) rank += __shfl_sync(0xffffffffu, ok, j) < ok;
        if (lane < made) {
          seg_key[b + rank] = ok;
          seg_val[b + rank] = ov;
        }
        if (lane == 0) dcount[x] = made;
        continue;
      }
    }
    if (sort_first) {
      // pairs already strictly ascending (one vertex's list over near-monotone ids)
      // stay where they are
      bool asc = true;
#pragma unroll
      for (int r = 0; r < S; ++r) {
        if (32 * r < T) {
          const int32_t up = __shfl_up_sync(0xffffffffu, L.k[r], 1);
          const int32_t wrap = r > 0 ? __shfl_sync(0xffffffffu, L.k[r > 0 ? r - 1 : 0], 31) : INT_MIN;
          const int i = lane + 32 * r;
          if (i < T && i > 0 && (lane ? up : wrap) >= L.k[r]) asc = false;
        }
      }
      if (__all_sync(0xffffffffu, asc)) {
        if (lane == 0) dcount[x] = T;
        continue;
      }
    }
    // many targets: sort the pairs (from registers) in shared memory; each stage of the
    // bitonic network compares N / 2 pairs (i, i + j), i with bit j clear
    int N = 32;
    while (N < T) N <<= 1;
#pragma unroll
    for (int r = 0; r < S; ++r) {
      const int i = lane + 32 * r;
      if (i < N) {
        sk[i] = i < T ? L.k[r] : INT_MAX;
        sv[i] = i < T ? L.wt[r] : 0;
      }
    }
    __syncwarp();
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int p = lane; p < (N >> 1); p += 32) {
          const int i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
          const int l = i | j;
          const bool up = (i & k) == 0;
          const int32_t a = sk[i], q = sk[l];
          if (up ? a > q : a < q) {
            sk[i] = q;
            sk[l] = a;
            const long long t = sv[i];
            sv[i] = sv[l];
            sv[l] = t;
          }
        }
        __syncwarp();
      }
    }
    int out = 0;
    for (int c0 = 0; c0 < T; c0 += 32) {
      const int i = c0 + lane;
      const bool head = i < T && (i == 0 || sk[i - 1] != sk[i]);
      long long sum = 0;
      if (head) {
        sum = sv[i];
        for (int j = i + 1; j < T && sk[j] == sk[i]; ++j) sum += sv[j];
      }
      const unsigned bal = __ballot_sync(0xffffffffu, head);
      if (head) {
        const int at = out + __popc(bal & ((1u << lane) - 1u));
        seg_key[b + at] = sk[i];
        seg_val[b + at] = sum;
      }
      out += __popc(bal);
    }
    if (lane == 0) dcount[x] = out;
    __syncwarp();
  }
}

// Clusters of kMergeMax < T <= kMergeBlockMax pairs: a block per cluster sorts the
// pairs by target in shared memory (bitonic network over the next power of two,
// padding keys INT_MAX), then every run head sums its run; the distinct targets are
// written back in ascending order at the front of the segment.
// With a list (list_count not null) only the listed clusters are visited.
__global__ void __launch_bounds__(256) cluster_merge_block_k(int64_t c, const long long* __restrict__ cbase,
                                                             int32_t* __restrict__ seg_key,
                                                             long long* __restrict__ seg_val,
                                                             int32_t* __restrict__ dcount,
                                                             const int32_t* __restrict__ list = nullptr,
                                                             const int* __restrict__ list_count = nullptr) {
  extern __shared__ __align__(16) unsigned char mb_dyn[];
  long long* sv = (long long*)mb_dyn;
  int32_t* sk = (int32_t*)(sv + kMergeBlockMax);
  __shared__ int s_warp[8];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t total = list_count ? (int64_t)*list_count : c;
  for (int64_t xi = blockIdx.x; xi < total; xi += gridDim.x) {
    const int64_t x = list_count ? (int64_t)list[xi] : xi;
    const long long b = cbase[x];
    const int T = (int)(cbase[x + 1] - b);
    if (T <= kMergeMax || T > kMergeBlockMax) continue;  // the same in every thread of the block
    int N = 1;
    while (N < T) N <<= 1;
    for (int i = tid; i < N; i += 256) {
      sk[i] = i < T ? seg_key[b + i] : INT_MAX;
      sv[i] = i < T ? seg_val[b + i] : 0;
    }
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int p = tid; p < (N >> 1); p += 256) {  // pair (i, i + j), i with bit j clear
          const int i = ((p & ~(j - 1)) << 1) | (p & (j - 1));
          const int l = i | j;
          const bool up = (i & k) == 0;
          const int32_t a = sk[i], bb = sk[l];
          if (up ? a > bb : a < bb) {
            sk[i] = bb;
            sk[l] = a;
            const long long t = sv[i];
            sv[i] = sv[l];
            sv[l] = t;
          }
        }
        __syncthreads();
      }
    }
    // run heads, numbered by a block scan; each head sums its run
    constexpr int kPer = kMergeBlockMax / 256;
    int cnt = 0;
    for (int q = 0; q < kPer; ++q) {
      const int i = tid * kPer + q;
      if (i < N && sk[i] != INT_MAX && (i == 0 || sk[i] != sk[i - 1])) ++cnt;
    }
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[wid] = inc;
    __syncthreads();
    int before = 0, total = 0;
    for (int w2 = 0; w2 < 8; ++w2) {
      if (w2 < wid) before += s_warp[w2];
      total += s_warp[w2];
    }
    int at = before + inc - cnt;
    // the sorted copy is in shared memory, so the segment can be overwritten
    for (int q = 0; q < kPer; ++q) {
      const int i = tid * kPer + q;
      if (i < N && sk[i] != INT_MAX && (i == 0 || sk[i] != sk[i - 1])) {
        long long sum = sv[i];
        for (int j = i + 1; j < N && sk[j] == sk[i]; ++j) sum += sv[j];
        seg_key[b + at] = sk[i];
        seg_val[b + at] = sum;
        ++at;
      }
    }
    if (tid == 0) dcount[x] = total;
    __syncthreads();
  }
}

// The sorted distinct targets of every cluster, copied from the front of its segment
// to coff[c].
// Clusters with skip[x] != 0 (skip may be null) are left out (their lists are written
// by the sparse contraction's copy).
__global__ void __launch_bounds__(256) cluster_place_k(int64_t c, const long long* __restrict__ cbase,
                                                       const int64_t* __restrict__ coff,
                                                       const int32_t* __restrict__ seg_key,
                                                       const long long* __restrict__ seg_val,
                                                       int32_t* __restrict__ cadj, long long* __restrict__ cw,
                                                       int32_t* __restrict__ csrc,
                                                       const unsigned char* __restrict__ skip) {
  // 32 clusters per warp step, their lists laid end to end over the lanes
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); x0 < c; x0 += stride) {
    const int64_t x = x0 + lane;
    const bool take = x < c && !(skip && skip[x]);
    const long long b = take ? cbase[x] : 0;
    const int64_t o = take ? coff[x] : 0;
    const int64_t D = take ? coff[x + 1] - o : 0;
    warp_pieces<KeyVal>(
        D, b, o, [&](int64_t at) { return KeyVal{seg_key[at], seg_val[at]}; },
        [&](int64_t at, int j, const KeyVal& kv) {
          cadj[at] = kv.k;
          cw[at] = kv.v;
          csrc[at] = (int32_t)(x0 + j);
        });
  }
}


// ---------------------------------------------------------------- sparse contraction
// Contractions in which most vertices keep their own id as label, alone in their cluster
// (Padberg-Rinaldi passes and exact-step rounds by union-find roots, label-propagation
// levels that merge few vertices), on a graph with strictly increasing lists.  The
// cluster id of such a "lone" vertex is the rank of its own id among the labels, so lone
// neighbours keep their order and stay distinct under the renumbering.  The coarse list of
// a lone vertex is its fine list renumbered, except for the few entries that point into
// the other ("merged") clusters: those may repeat a target and sit out of order.
// A warp per lone vertex sums them per target in shared memory and merges the distinct
// ones into the renumbered list by rank -- one pass to count the coarse degree, one to
// write.  Only the members of merged groups (and lone vertices with more than
// kScMaxM such entries) go through the pre-merge and the cluster merge.
constexpr int kScMaxM = 32;  // entries into merged groups per lone vertex

// mflag[cid[v]] = 1 for every v not labelled by its own id (its cluster has another
// member, or its label is another vertex's id); a plain store of 1 from any number of
// threads.
__global__ void sc_merged_k(int64_t n, const int32_t* __restrict__ lab, const int32_t* __restrict__ cid,
                            unsigned char* __restrict__ mflag) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (lab[v] != (int32_t)v) mflag[cid[v]] = 1;
}

// cidm[u] = cid[u], with the sign bit set when u's group is merged: one gather per entry
// gives both.
__global__ void sc_pack_k(int64_t n, const int32_t* __restrict__ cid, const unsigned char* __restrict__ mflag,
                          int32_t* __restrict__ cidm) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = cid[v];
    cidm[v] = mflag[x] ? (int32_t)((uint32_t)x | 0x80000000u) : x;
  }
}

constexpr int kScUnroll = 2;  // rows of 32 entries in flight per warp

// The entries of lone vertex v's list that point into merged groups, collected row by
// row in the warp's shared arrays mk / mw (at most kScMaxM kept; the return value counts
// them all).
template <typename WT>
__device__ __forceinline__ int sc_collect(int64_t beg, int64_t end, int lane, const int32_t* __restrict__ adj,
                                          const WT* __restrict__ w, const int32_t* __restrict__ cidm, bool with_w,
                                          int32_t* mk, long long* mw) {
  int nm = 0;
  for (int64_t b = beg; b < end; b += 32 * kScUnroll) {
    int32_t u[kScUnroll], k[kScUnroll];
#pragma unroll
    for (int q = 0; q < kScUnroll; ++q) {
      const int64_t e = b + 32 * q + lane;
      u[q] = e < end ? __ldg(adj + e) : -1;
    }
#pragma unroll
    for (int q = 0; q < kScUnroll; ++q) k[q] = u[q] >= 0 ? __ldg(cidm + u[q]) : 0;
#pragma unroll
    for (int q = 0; q < kScUnroll; ++q) {
      const bool m = u[q] >= 0 && k[q] < 0;
      const unsigned bal = __ballot_sync(0xffffffffu, m);
      if (m) {
        const int at = nm + __popc(bal & ((1u << lane) - 1u));
        if (at < kScMaxM) {
          mk[at] = k[q] & 0x7fffffff;
          mw[at] = with_w ? ldw(w, b + 32 * q + lane) : 0;
        }
      }
      nm += __popc(bal);
    }
  }
  __syncwarp();
  return nm;
}

// Pass 1: the coarse degree of every lone vertex handled here (sdeg[v], else -1), and the
// vertices left to the pre-merge flagged in dirty.
template <typename WT>
__global__ void __launch_bounds__(256) sc_count_k(int64_t n, const int32_t* __restrict__ cidm,
                                                  const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                  const WT* __restrict__ w, int32_t* __restrict__ sdeg,
                                                  unsigned char* __restrict__ dirty) {
  __shared__ int32_t s_mk[8][kScMaxM];
  __shared__ long long s_mw[8][kScMaxM];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    const int64_t beg = off[v], end = off[v + 1];
    if (cidm[v] < 0) {  // a member of a merged group
      if (lane == 0) { sdeg[v] = -1; dirty[v] = 1; }
      continue;
    }
    const int nm = sc_collect<WT>(beg, end, lane, adj, w, cidm, false, s_mk[wid], s_mw[wid]);
    if (nm > kScMaxM) {
      if (lane == 0) { sdeg[v] = -1; dirty[v] = 1; }
      continue;
    }
    const bool have = lane < nm;
    const int32_t key = have ? s_mk[wid][lane] : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int nd = __popc(__ballot_sync(0xffffffffu, have && (__ffs(peers) - 1) == lane));
    if (lane == 0) { sdeg[v] = (int32_t)(end - beg - nm + nd); dirty[v] = nm == 0 ? 2 : 0; }
    __syncwarp();
  }
}

// Pass 2: the lists of the lone vertices counted in pass 1, at their coarse offsets.
// The coarse list merges two ascending sequences: the entries into lone vertices' clusters
// (in list order) and the nd distinct merged targets (sorted in s_dk).  An entry with key
// k lands at its rank among the lone entries plus t(k), the number of targets below k (a
// binary search of s_dk); target j lands at j plus the number of lone entries with
// t(k) <= j, counted in a histogram over t (one shared-memory add per run of equal t in
// a row) and summed by a scan over the targets.
template <typename WT>
__global__ void __launch_bounds__(256) sc_write_k(int64_t n, const int32_t* __restrict__ cidm,
                                                  const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                                  const WT* __restrict__ w, const int32_t* __restrict__ sdeg,
                                                  const unsigned char* __restrict__ dirty,
                                                  const int64_t* __restrict__ coff, int32_t* __restrict__ cadj,
                                                  long long* __restrict__ cw, int32_t* __restrict__ csrc) {
  __shared__ int32_t s_mk[8][kScMaxM];
  __shared__ long long s_mw[8][kScMaxM];
  __shared__ int32_t s_dk[8][kScMaxM];
  __shared__ long long s_dw[8][kScMaxM];
  __shared__ int s_ht[8][kScMaxM];  // lone entries per value of t below nd
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lower = (1u << lane) - 1u;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    if (sdeg[v] < 0) continue;  // the same in every lane
    const int64_t beg = off[v], end = off[v + 1];
    const int32_t x = cidm[v];  // lone: no sign bit
    const int64_t o = coff[x];
    if (dirty[v] == 2) {  // no entry into a merged cluster: the list renumbered in place
      for (int64_t b = beg; b < end; b += 32 * kScUnroll) {
        int32_t u[kScUnroll];
        long long wt[kScUnroll];
#pragma unroll
        for (int q = 0; q < kScUnroll; ++q) {
          const int64_t e = b + 32 * q + lane;
          u[q] = e < end ? __ldg(adj + e) : -1;
          wt[q] = e < end ? ldw(w, e) : 0;
        }
#pragma unroll
        for (int q = 0; q < kScUnroll; ++q)
          if (u[q] >= 0) {
            const int64_t at = o + (b + 32 * q + lane - beg);
            cadj[at] = __ldg(cidm + u[q]);
            cw[at] = wt[q];
            csrc[at] = x;
          }
      }
      continue;
    }
    const int nm = sc_collect<WT>(beg, end, lane, adj, w, cidm, true, s_mk[wid], s_mw[wid]);
    // distinct targets into merged groups: the lowest lane of each target sums it and
    // places it by its rank among the distinct targets
    const bool have = lane < nm;
    const int32_t key = have ? s_mk[wid][lane] : -1 - lane;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const bool first = have && (__ffs(peers) - 1) == lane;
    const unsigned firsts = __ballot_sync(0xffffffffu, first);
    const int nd = __popc(firsts);
    if (first) {
      long long sum = 0;
      for (unsigned m = peers; m; m &= m - 1u) sum += s_mw[wid][__ffs(m) - 1];
      int rank = 0;
      for (unsigned m = firsts; m; m &= m - 1u) rank += s_mk[wid][__ffs(m) - 1] < key;
      s_dk[wid][rank] = key;
      s_dw[wid][rank] = sum;
    }
    s_ht[wid][lane] = 0;
    __syncwarp();
    const int32_t* dk = s_dk[wid];
    int mbefore = 0;
    for (int64_t b = beg; b < end; b += 32 * kScUnroll) {
      int32_t u[kScUnroll], k[kScUnroll];
      long long wt[kScUnroll];
#pragma unroll
      for (int q = 0; q < kScUnroll; ++q) {
        const int64_t e = b + 32 * q + lane;
        u[q] = e < end ? __ldg(adj + e) : -1;
        wt[q] = e < end ? ldw(w, e) : 0;
      }
#pragma unroll
      for (int q = 0; q < kScUnroll; ++q) k[q] = u[q] >= 0 ? __ldg(cidm + u[q]) : 0;
#pragma unroll
      for (int q = 0; q < kScUnroll; ++q) {
        const bool m = u[q] >= 0 && k[q] < 0;
        const bool lone = u[q] >= 0 && k[q] >= 0;
        const unsigned balM = __ballot_sync(0xffffffffu, m);
        int t = 0;  // targets below k
        if (lone) {
          int hi = nd;
          while (t < hi) {
            const int mid = (t + hi) >> 1;
            if (dk[mid] < k[q]) t = mid + 1;
            else hi = mid;
          }
          const int64_t pos = (b + 32 * q - beg + lane) - (mbefore + __popc(balM & lower)) + t;
          cadj[o + pos] = k[q];
          cw[o + pos] = wt[q];
          csrc[o + pos] = x;
        }
        mbefore += __popc(balM);
        if (nd > 0) {
          const bool counted = lone && t < nd;
          const unsigned run = __match_any_sync(0xffffffffu, counted ? t : -1 - lane);
          if (counted && (__ffs(run) - 1) == lane) atomicAdd(&s_ht[wid][t], __popc(run));
        }
      }
    }
    __syncwarp();
    // target j: the lone entries with t <= j are below it
    int dbelow = lane < nd ? s_ht[wid][lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, dbelow, d);
      if (lane >= d) dbelow += y;
    }
    if (lane < nd) {
      cadj[o + lane + dbelow] = dk[lane];
      cw[o + lane + dbelow] = s_dw[wid][lane];
      csrc[o + lane + dbelow] = x;
    }
    __syncwarp();
  }
}

// The vertices left to the pre-merge, listed (in no particular order); *count their number.
__global__ void sc_list_k(int64_t n, const unsigned char* __restrict__ dirty, int32_t* __restrict__ list,
                          int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = b + lane;
    const bool d = v < n && dirty[v] == 1;
    const unsigned bal = __ballot_sync(0xffffffffu, d);
    int at = 0;
    if (lane == 0 && bal) at = atomicAdd(count, __popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (d) list[at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)v;
  }
}

// After the merge of the pre-merged clusters: the coarse degree of every cluster of a
// lone vertex handled here, and clean[x] marking those clusters.
__global__ void sc_clean_deg_k(int64_t n, const int32_t* __restrict__ sdeg, const int32_t* __restrict__ cid,
                               int32_t* __restrict__ ccount, unsigned char* __restrict__ clean) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (sdeg[v] < 0) continue;
    const int32_t x = cid[v];
    ccount[x] = sdeg[v];
    clean[x] = 1;
  }
}

template <typename F>
static void sc_by_weight(const GraphView& g, F f) {
  if (g.unit) f((const UnitW*)nullptr);
  else if (g.wbytes == 4) f((const int32_t*)g.w);
  else f((const long long*)g.w);
}

void sparse_mark(const GraphView& g, const int32_t* lab, const int32_t* cid, unsigned char* mflag, int32_t* cidm,
                 unsigned char* dirty, int32_t* sdeg, int32_t* list, int* count, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(mflag, 0, (size_t)g.n, s));
  VC_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s));
  const int grid = grid_for(g.n, 256, kSMs * 8);
  sc_merged_k<<<grid, 256, 0, s>>>(g.n, lab, cid, mflag);
  sc_pack_k<<<grid, 256, 0, s>>>(g.n, cid, mflag, cidm);
  sc_by_weight(g, [&](auto wp) {
    using WT = std::remove_cv_t<std::remove_pointer_t<decltype(wp)>>;
    sc_count_k<WT><<<grid_for(g.n, 8, kSMs * 16), 256, 0, s>>>(g.n, cidm, g.off, g.adj, wp, sdeg, dirty);
  });
  sc_list_k<<<grid, 256, 0, s>>>(g.n, dirty, list, count);
  count_launch(4);
  VC_CHECK_LAUNCH();
}

static void sparse_finish_degrees(const GraphView& g, const int32_t* cid, const int32_t* sdeg, int32_t* ccount,
                                  unsigned char* clean, int64_t c, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(clean, 0, (size_t)std::max<int64_t>(c, 1), s));
  sc_clean_deg_k<<<grid_for(g.n, 256, kSMs * 8), 256, 0, s>>>(g.n, sdeg, cid, ccount, clean);
  count_launch();
  VC_CHECK_LAUNCH();
}

static void sparse_copy(const GraphView& g, const int32_t* cidm, const int32_t* sdeg, const unsigned char* dirty,
                        const int64_t* coff, int32_t* cadj, long long* cw, int32_t* csrc, cudaStream_t s) {
  sc_by_weight(g, [&](auto wp) {
    using WT = std::remove_cv_t<std::remove_pointer_t<decltype(wp)>>;
    sc_write_k<WT><<<grid_for(g.n, 8, kSMs * 16), 256, 0, s>>>(g.n, cidm, g.off, g.adj, wp, sdeg, dirty, coff, cadj,
                                                               cw, csrc);
  });
  count_launch();
  VC_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- correcting step
// Sec. 4.1, "correcting algorithm" (fixMisplacedVertices of Algorithm 1), optional: in
// every cluster C of 2..lg vertices (lg = floor(log2 n)), d(C) = weight of the edges
// leaving C and, for a member v, d(C - v) = d(C) - c(v, V - C) + c(v, C - v); v is
// misplaced when d(C - v) < d(C), and each cluster gives up at most its misplaced
// vertex of smallest d(C - v) (ties: smallest id), which becomes a singleton with a
// cluster id after all others, in ascending vertex order.
__global__ void corr_size_k(int64_t n, const int32_t* __restrict__ cid, int* __restrict__ csize) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&csize[cid[v]], 1);
}

__device__ __forceinline__ bool corr_small(int sz, int lg) { return sz >= 2 && sz <= lg; }

// Eight lanes per vertex of a small cluster: its weight to the outside and to the rest
// of its cluster; the outside weights sum into d(C).
template <typename WT>
__global__ void corr_sums_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const WT* __restrict__ w, const int32_t* __restrict__ cid,
                            const int* __restrict__ csize, int lg, long long* __restrict__ vout,
                            long long* __restrict__ vin, long long* __restrict__ dc) {
  constexpr int G = 8;
  const int lane = threadIdx.x & 31, glane = lane & (G - 1);
  const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += groups) {
    const int32_t C = cid[v];
    if (!corr_small(csize[C], lg)) continue;  // the same in the group's lanes
    long long o = 0, i = 0;
    for (int64_t e = off[v] + glane; e < off[v + 1]; e += G) {
      const long long x = ldw(w, e);
      if (cid[adj[e]] == C) i += x;
      else o += x;
    }
#pragma unroll
    for (int k = G / 2; k > 0; k >>= 1) {
      o += __shfl_xor_sync(gmask, o, k);
      i += __shfl_xor_sync(gmask, i, k);
    }
    if (glane == 0) {
      vout[v] = o;
      vin[v] = i;
      if (o) atomicAdd((unsigned long long*)&dc[C], (unsigned long long)o);
    }
  }
}

// pass 0: the smallest d(C - v) below d(C) per cluster; pass 1: the smallest id
// attaining it; pass 2: flag[v] = v leaves its cluster.
__global__ void corr_pick_k(int64_t n, const int32_t* __restrict__ cid, const int* __restrict__ csize, int lg,
                            const long long* __restrict__ vout, const long long* __restrict__ vin,
                            const long long* __restrict__ dc, long long* __restrict__ bestv,
                            int* __restrict__ bestid, int* __restrict__ flag, int pass) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t C = cid[v];
    const bool small = corr_small(csize[C], lg);
    if (pass == 2) {
      flag[v] = small && bestid[C] == (int)v ? 1 : 0;
      continue;
    }
    if (!small) continue;
    const long long without = dc[C] - vout[v] + vin[v];
    if (without >= dc[C]) continue;
    if (pass == 0) atomicMin(&bestv[C], without);
    else if (without == bestv[C]) atomicMin(&bestid[C], (int)v);
  }
}

__global__ void corr_apply_k(int64_t n, const int* __restrict__ flag, const int* __restrict__ rank,
                             const int* __restrict__ c_dev, int32_t* __restrict__ cid) {
  const int c = *c_dev;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (flag[v]) cid[v] = c + rank[v];
}

__global__ void corr_count_k(int* __restrict__ c_dev, const int* __restrict__ moved) { *c_dev += *moved; }

void correct_clusters(const GraphView& g, int32_t* cid, int* c_dev, const CorrectScratch& cs, cudaStream_t s) {
  const int64_t n = g.n;
  if (n < 4) return;  // no cluster of 2..floor(log2 n) vertices below 4 vertices
  int lg = 0;
  while ((int64_t(2) << lg) <= n) ++lg;
  VC_CUDA(cudaMemsetAsync(cs.csize, 0, sizeof(int) * n, s));
  VC_CUDA(cudaMemsetAsync(cs.dc, 0, sizeof(long long) * n, s));
  VC_CUDA(cudaMemsetAsync(cs.bestv, 0x7f, sizeof(long long) * n, s));  // above every d(C - v)
  VC_CUDA(cudaMemsetAsync(cs.bestid, 0x7f, sizeof(int) * n, s));       // above every vertex id
  const int grid = grid_for(n, 256, kSMs * 8);
  corr_size_k<<<grid, 256, 0, s>>>(n, cid, cs.csize);
  const int gs = grid_for(n, 32, kSMs * 16);
  if (g.unit)
    corr_sums_k<UnitW><<<gs, 256, 0, s>>>(n, g.off, g.adj, nullptr, cid, cs.csize, lg, cs.vout, cs.vin, cs.dc);
  else if (g.wbytes == 4)
    corr_sums_k<int32_t><<<gs, 256, 0, s>>>(n, g.off, g.adj, (const int32_t*)g.w, cid, cs.csize, lg, cs.vout,
                                            cs.vin, cs.dc);
  else
    corr_sums_k<long long><<<gs, 256, 0, s>>>(n, g.off, g.adj, (const long long*)g.w, cid, cs.csize, lg, cs.vout,
                                              cs.vin, cs.dc);
  for (int pass = 0; pass < 3; ++pass)
    corr_pick_k<<<grid, 256, 0, s>>>(n, cid, cs.csize, lg, cs.vout, cs.vin, cs.dc, cs.bestv, cs.bestid, cs.flag,
                                     pass);
  count_launch(5);
  VC_CHECK_LAUNCH();
  exclusive_scan<int, int>(cs.flag, cs.rank, n, cs.moved, cs.scan_scr32, s);
  corr_apply_k<<<grid, 256, 0, s>>>(n, cs.flag, cs.rank, c_dev, cid);
  corr_count_k<<<1, 1, 0, s>>>(c_dev, cs.moved);
  count_launch(2);
  VC_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- giant clusters
__global__ void giant_list_k(int64_t c, const long long* __restrict__ cbase, int* __restrict__ gcount,
                             int32_t* __restrict__ glist, int32_t* __restrict__ gT) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < c; x += (int64_t)gridDim.x * blockDim.x) {
    const long long T = cbase[x + 1] - cbase[x];
    if (T > kMergeBlockMax) {
      const int j = atomicAdd(gcount, 1);
      glist[j] = (int32_t)x;
      gT[j] = (int32_t)T;
    }
  }
}

// The giant clusters' pairs, keyed (j << bits | target) for giant j.
__global__ void giant_gather_k(int ng, const int32_t* __restrict__ glist, const long long* __restrict__ gstart,
                               const long long* __restrict__ cbase, const int32_t* __restrict__ seg_key,
                               const long long* __restrict__ seg_val, int bits, unsigned long long* __restrict__ keys,
                               long long* __restrict__ vals) {
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, st = (int64_t)gridDim.x * blockDim.x;
  for (int j = 0; j < ng; ++j) {
    const long long b = cbase[glist[j]], o = gstart[j], T = gstart[j + 1] - o;
    for (int64_t e = t0; e < T; e += st) {
      keys[o + e] = ((unsigned long long)j << bits) | (unsigned long long)(uint32_t)seg_key[b + e];
      vals[o + e] = seg_val[b + e];
    }
  }
}

// Every run head of the sorted giant pairs sums its run and writes it at its rank within
// its cluster, at the front of the cluster's segment.
__global__ void giant_reduce_k(int64_t m, int bits, const unsigned long long* __restrict__ keys,
                               const long long* __restrict__ vals, const int32_t* __restrict__ heads,
                               const long long* __restrict__ hpos, const long long* __restrict__ gstart,
                               const int32_t* __restrict__ glist, const long long* __restrict__ cbase,
                               int32_t* __restrict__ seg_key, long long* __restrict__ seg_val) {
  const unsigned long long mask = (1ULL << bits) - 1ULL;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (!heads[i]) continue;
    const unsigned long long k = keys[i];
    long long sum = vals[i];
    for (int64_t q = i + 1; q < m && keys[q] == k; ++q) sum += vals[q];
    const int j = (int)(k >> bits);
    const long long at = cbase[glist[j]] + (hpos[i] - hpos[gstart[j]]);
    seg_key[at] = (int32_t)(k & mask);
    seg_val[at] = sum;
  }
}

__global__ void giant_count_k(int ng, const int32_t* __restrict__ glist, const long long* __restrict__ gstart,
                              const long long* __restrict__ hpos, int32_t* __restrict__ dcount) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ng; j += gridDim.x * blockDim.x)
    dcount[glist[j]] = (int32_t)(hpos[gstart[j + 1]] - hpos[gstart[j]]);
}

static void giant_merge(const GiantScratch& G, int64_t c, const long long* cbase, int32_t* seg_key,
                        long long* seg_val, int32_t* dcount, long long* scan_scr, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(G.gcount, 0, sizeof(int), s));
  giant_list_k<<<grid_for(c, 256, kSMs * 8), 256, 0, s>>>(c, cbase, G.gcount, G.glist, G.gT);
  count_launch();
  VC_CHECK_LAUNCH();
  exclusive_scan<int, long long>(G.gT, G.gstart, G.ngiant, G.gstart + G.ngiant, scan_scr, s);
  int bits = ceil_log2(c);
  if (bits < 1) bits = 1;
  int jbits = ceil_log2(G.ngiant);
  if (jbits < 1) jbits = 1;
  const int grid = grid_for(G.pairs, 256, kSMs * 8);
  giant_gather_k<<<grid, 256, 0, s>>>(G.ngiant, G.glist, G.gstart, cbase, seg_key, seg_val, bits, G.k0, G.v0);
  count_launch();
  VC_CHECK_LAUNCH();
  radix_sort_pairs(G.k0, G.v0, G.k1, G.v1, G.pairs, bits + jbits, G.hist, s);
  run_heads_k<<<grid, 256, 0, s>>>(G.k0, G.pairs, G.heads);
  count_launch();
  VC_CHECK_LAUNCH();
  exclusive_scan<int, long long>(G.heads, G.hpos, G.pairs, G.hpos + G.pairs, scan_scr, s);
  giant_reduce_k<<<grid, 256, 0, s>>>(G.pairs, bits, G.k0, G.v0, G.heads, G.hpos, G.gstart, G.glist, cbase, seg_key,
                                      seg_val);
  giant_count_k<<<grid_for(G.ngiant, 256, kSMs), 256, 0, s>>>(G.ngiant, G.glist, G.gstart, G.hpos, dcount);
  count_launch(2);
  VC_CHECK_LAUNCH();
}

void cluster_stats(int64_t n, const int32_t* ccount, int* maxt, long long* pairs, int* ngiant, long long* gpairs,
                   cudaStream_t s) {
  if (n <= 0) return;
  cluster_stats_k<<<grid_for(n, 256, kSMs * 4), 256, 0, s>>>(n, ccount, maxt, pairs, ngiant, gpairs);
  count_launch();
  VC_CHECK_LAUNCH();
}

// Opts cluster_merge_block_k into its shared-memory size, once per device.
static int merge_block_smem() {
  static std::mutex mu;
  static std::unordered_map<int, bool> ready;  // per device: the shared-memory limit was raised
  const int smem = kMergeBlockMax * (int)(sizeof(long long) + sizeof(int32_t));
  int dev = 0;
  VC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (!ready[dev]) {
    VC_CUDA(cudaFuncSetAttribute(cluster_merge_block_k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    ready[dev] = true;
  }
  return smem;
}

__global__ void block_class_list_k(int64_t c, const long long* __restrict__ cbase, int32_t* __restrict__ list,
                                   int* __restrict__ count) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < c; x += (int64_t)gridDim.x * blockDim.x) {
    const long long T = cbase[x + 1] - cbase[x];
    if (T > kMergeMax && T <= kMergeBlockMax) list[atomicAdd(count, 1)] = (int32_t)x;
  }
}

void cluster_merge(const GraphView& g, const int32_t* cid, const ContractScratch& cs, int32_t* ccount, int64_t c,
                   long long* cbase, long long* cursor, int32_t* seg_key, long long* seg_val, int64_t* coff,
                   int32_t* cadj, long long* cw, int32_t* csrc, long long* nnz_dev, bool big, bool sort_first,
                   const GiantScratch* giant, int32_t* blist, int* blist_n, cudaStream_t s, const SparseCtx* sp) {
  exclusive_scan<int, long long>(ccount, cbase, c, cbase + c, cs.scan_scr, s);
  VC_CUDA(cudaMemcpyAsync(cursor, cbase, sizeof(long long) * c, cudaMemcpyDeviceToDevice, s));
  const int gv = grid_for(g.n, 256, kSMs * 8), gc = grid_for(c, 8, kSMs * 16);
  const PairOut in{cs.tmp_key, cs.tmp_val, cs.cmp_key, cs.cmp_val};
  cluster_scatter_k<<<gv, 256, 0, s>>>(g.n, g.off, cid, cs.cnt, in, cursor, seg_key, seg_val);
  cluster_merge_k<<<gc, 256, 0, s>>>(c, cbase, seg_key, seg_val, ccount, sort_first);
  count_launch(2);
  VC_CHECK_LAUNCH();
  if (big) {
    // the clusters of kMergeMax < T <= kMergeBlockMax pairs listed first, so that the
    // blocks visit only them (blist: n ints no longer needed once the scatter ran)
    VC_CUDA(cudaMemsetAsync(blist_n, 0, sizeof(int), s));
    block_class_list_k<<<grid_for(c, 256, kSMs * 8), 256, 0, s>>>(c, cbase, blist, blist_n);
    const int smem = merge_block_smem();
    cluster_merge_block_k<<<kSMs, 256, smem, s>>>(c, cbase, seg_key, seg_val, ccount, blist, blist_n);
    count_launch(2);
    VC_CHECK_LAUNCH();
  }
  if (giant && giant->ngiant > 0) giant_merge(*giant, c, cbase, seg_key, seg_val, ccount, cs.scan_scr, s);
  if (sp) sparse_finish_degrees(g, cid, sp->sdeg, ccount, sp->clean, c, s);
  exclusive_scan<int, long long>(ccount, (long long*)coff, c, (long long*)coff + c, cs.scan_scr, s);
  cluster_place_k<<<grid_for(c, 256, kSMs * 8), 256, 0, s>>>(c, cbase, coff, seg_key, seg_val, cadj, cw, csrc,
                                                               sp ? sp->clean : nullptr);
  count_launch();
  VC_CHECK_LAUNCH();
  if (sp) sparse_copy(g, sp->cidm, sp->sdeg, sp->dirty, coff, cadj, cw, csrc, s);
  VC_CUDA(cudaMemcpyAsync(nnz_dev, coff + c, sizeof(long long), cudaMemcpyDeviceToDevice, s));
}


}  // namespace vc
