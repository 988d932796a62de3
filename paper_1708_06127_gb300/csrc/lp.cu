// Label propagation rounds and the pre-merge of cross-cluster edges.
//
// Both reduce, for every vertex v, the multiset {(key(u), c(v,u)) : u in N(v)} to
// per-key weight sums in an open-addressing table:
//   * label propagation (Sec. 4.1, "label propagation algorithm"): key = label of u,
//     then v takes the key of largest sum, ties by the larger tie hash;
//   * contraction pre-merge (Sec. 4.1, "contract it"): key = cluster id of u, keys
//     equal to v's own cluster dropped (intra-cluster edges vanish), every remaining
//     (key, sum) written out.
// Work is split by neighbour-list length: a warp per vertex with a shared-memory
// table for short lists, a block per vertex with a larger shared table, and a block
// per vertex with a table in global scratch for the few very long lists.
#include <limits.h>

#include "kernels.cuh"

namespace vc {

constexpr int kWarpsPerBlock = 8;
constexpr int kAggThreads = kWarpsPerBlock * 32;
constexpr int kEmptyKey = -1;

enum { kModeLP = 0, kModeEmit = 1 };

__global__ void bins_k(int64_t n, const int64_t* __restrict__ off, int32_t* __restrict__ blist,
                       int32_t* __restrict__ glist, int* __restrict__ counts) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t d = off[v + 1] - off[v];
    if (d > kWarpMaxDeg) {
      if (d <= kBlockMaxDeg) blist[atomicAdd(&counts[0], 1)] = (int32_t)v;
      else glist[atomicAdd(&counts[1], 1)] = (int32_t)v;
      atomicMax(&counts[2], (int)(d < INT_MAX ? d : INT_MAX));
    }
  }
}

void bins_build(const GraphView& g, Bins& b, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(b.counts, 0, 3 * sizeof(int), s));
  bins_k<<<grid_for(g.n, 256, kSMs * 8), 256, 0, s>>>(g.n, g.off, b.block_list, b.global_list, b.counts);
  count_launch();
  VC_CHECK_LAUNCH();
}

int64_t global_table_cap(int maxdeg) {
  int64_t c = 1;
  while (c < 2 * (int64_t)maxdeg) c <<= 1;
  return c < 64 ? 64 : c;
}

// Adds wt to the slot of key k (linear probing; capacity >= 2 x distinct keys).
__device__ __forceinline__ void tbl_add(int* tk, unsigned long long* tv, int lg, int k, long long wt) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = slot_hash(k, lg);
  // at most one probe per slot: the table always has room (capacity >= 2 x keys)
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int prev = atomicCAS(&tk[h], kEmptyKey, k);
    if (prev == kEmptyKey || prev == k) {
      atomicAdd(&tv[h], (unsigned long long)wt);
      return;
    }
    h = (h + 1) & mask;
  }
}

template <typename WT>
__device__ __forceinline__ long long ldw(const WT* w, int64_t e) { return (long long)__ldg(w + e); }

// key of neighbour u for vertex v; returns false when the entry is skipped
template <int MODE, bool FIRST>
__device__ __forceinline__ bool entry_key(const int32_t* __restrict__ lab, int32_t u, int32_t own, int32_t* k) {
  if (MODE == kModeLP) {
    *k = FIRST ? u : __ldg(lab + u);
    return true;
  } else {
    *k = __ldg(lab + u);
    return *k != own;
  }
}

// ------------------------------------------------------------------ warp class
template <typename WT, int MODE, bool FIRST>
__global__ void __launch_bounds__(kAggThreads) agg_warp_k(
    int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj, const WT* __restrict__ w,
    const int32_t* __restrict__ lab, int32_t* __restrict__ lab_out, uint64_t key,
    int32_t* __restrict__ tkey, long long* __restrict__ tval, int32_t* __restrict__ cnt) {
  __shared__ int s_keys[kWarpsPerBlock][kWarpCap];
  __shared__ unsigned long long s_vals[kWarpsPerBlock][kWarpCap];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* tk = s_keys[wib];
  unsigned long long* tv = s_vals[wib];
  for (int i = lane; i < kWarpCap; i += 32) { tk[i] = kEmptyKey; tv[i] = 0ULL; }
  __syncwarp();
  const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t v = (int64_t)blockIdx.x * kWarpsPerBlock + wib; v < n; v += stride) {
    const int64_t beg = __ldg(off + v), end = __ldg(off + v + 1);
    const int d = (int)(end - beg);
    if (d > kWarpMaxDeg) continue;
    const int32_t own = (MODE == kModeEmit) ? __ldg(lab + v) : 0;
    if (d == 0) {
      if (lane == 0) {
        if (MODE == kModeLP) lab_out[v] = FIRST ? (int32_t)v : __ldg(lab + v);
        else cnt[v] = 0;
      }
      continue;
    }
    int lg = ceil_log2(2 * (int64_t)d);
    if (lg < 5) lg = 5;
    const int cap = 1 << lg;
    for (int64_t e = beg + lane; e < end; e += 32) {
      int32_t k;
      if (entry_key<MODE, FIRST>(lab, __ldg(adj + e), own, &k)) tbl_add(tk, tv, lg, k, ldw(w, e));
    }
    __syncwarp();
    if (MODE == kModeLP) {
      Cand best{-1LL, 0ULL, INT_MAX};
      for (int i = lane; i < cap; i += 32) {
        int L = tk[i];
        if (L != kEmptyKey) {
          Cand c{(long long)tv[i], tie_hash(key, L), L};
          if (better(c, best)) best = c;
          tk[i] = kEmptyKey;
          tv[i] = 0ULL;
        }
      }
      best = warp_best(best);
      if (lane == 0) lab_out[v] = best.l;
    } else {
      int base = 0;
      for (int i0 = 0; i0 < cap; i0 += 32) {
        int i = i0 + lane;
        int L = tk[i];
        bool occ = L != kEmptyKey;
        unsigned bal = __ballot_sync(0xffffffffu, occ);
        if (occ) {
          int j = base + __popc(bal & ((1u << lane) - 1u));
          tkey[beg + j] = L;
          tval[beg + j] = (long long)tv[i];
          tk[i] = kEmptyKey;
          tv[i] = 0ULL;
        }
        base += __popc(bal);
      }
      if (lane == 0) cnt[v] = base;
    }
    __syncwarp();
  }
}

// --------------------------------------------------------- block / global class
// One block per listed vertex; the table is in shared memory (global == false) or
// in this block's region of global scratch (global == true).
template <typename WT, int MODE, bool FIRST, bool GLOBAL>
__global__ void __launch_bounds__(kAggThreads) agg_block_k(
    const int32_t* __restrict__ list, const int* __restrict__ count_ptr, const int64_t* __restrict__ off,
    const int32_t* __restrict__ adj, const WT* __restrict__ w, const int32_t* __restrict__ lab,
    int32_t* __restrict__ lab_out, uint64_t key, int32_t* __restrict__ tkey, long long* __restrict__ tval,
    int32_t* __restrict__ cnt, int32_t* __restrict__ gkeys, long long* __restrict__ gvals, int64_t gcap) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Cand s_best[kWarpsPerBlock];
  __shared__ int s_count;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* tk;
  unsigned long long* tv;
  int64_t table_cap;
  if (GLOBAL) {
    tk = gkeys + (int64_t)blockIdx.x * gcap;
    tv = (unsigned long long*)gvals + (int64_t)blockIdx.x * gcap;
    table_cap = gcap;
  } else {
    tv = (unsigned long long*)dyn;
    tk = (int*)(dyn + sizeof(unsigned long long) * kBlockCap);
    table_cap = kBlockCap;
  }
  for (int64_t i = threadIdx.x; i < table_cap; i += kAggThreads) { tk[i] = kEmptyKey; tv[i] = 0ULL; }
  __syncthreads();
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    const int64_t beg = off[v], end = off[v + 1];
    const int64_t d = end - beg;
    const int32_t own = (MODE == kModeEmit) ? lab[v] : 0;
    int lg = ceil_log2(2 * d);
    if (lg < 5) lg = 5;
    const int64_t cap = (int64_t)1 << lg;
    for (int64_t e = beg + threadIdx.x; e < end; e += kAggThreads) {
      int32_t k;
      if (entry_key<MODE, FIRST>(lab, adj[e], own, &k)) tbl_add(tk, tv, lg, k, ldw(w, e));
    }
    if (MODE == kModeEmit && threadIdx.x == 0) s_count = 0;
    __syncthreads();
    if (MODE == kModeLP) {
      Cand best{-1LL, 0ULL, INT_MAX};
      for (int64_t i = threadIdx.x; i < cap; i += kAggThreads) {
        int L = tk[i];
        if (L != kEmptyKey) {
          Cand c{(long long)tv[i], tie_hash(key, L), L};
          if (better(c, best)) best = c;
          tk[i] = kEmptyKey;
          tv[i] = 0ULL;
        }
      }
      best = warp_best(best);
      if (lane == 0) s_best[wib] = best;
      __syncthreads();
      if (threadIdx.x == 0) {
        Cand b = s_best[0];
        for (int q = 1; q < kWarpsPerBlock; ++q)
          if (better(s_best[q], b)) b = s_best[q];
        lab_out[v] = b.l;
      }
    } else {
      for (int64_t i = threadIdx.x; i < cap; i += kAggThreads) {
        int L = tk[i];
        if (L != kEmptyKey) {
          int j = atomicAdd(&s_count, 1);
          tkey[beg + j] = L;
          tval[beg + j] = (long long)tv[i];
          tk[i] = kEmptyKey;
          tv[i] = 0ULL;
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) cnt[v] = s_count;
    }
    __syncthreads();
  }
}

constexpr size_t kBlockDynSmem = (sizeof(unsigned long long) + sizeof(int)) * kBlockCap;

template <typename WT, int MODE, bool FIRST>
void launch_agg(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* lab,
                int32_t* lab_out, uint64_t key, int32_t* tkey, long long* tval, int32_t* cnt, cudaStream_t s) {
  const WT* w = (const WT*)g.w;
  // residency: 8 warps x 3 KB of tables per block
  int grid = grid_for(g.n, kWarpsPerBlock * 4, kSMs * 8);
  agg_warp_k<WT, MODE, FIRST><<<grid, kAggThreads, 0, s>>>(g.n, g.off, g.adj, w, lab, lab_out, key, tkey, tval, cnt);
  count_launch();
  VC_CHECK_LAUNCH();
  if (b.h_block > 0) {
    static bool attr_set = false;
    auto kfn = agg_block_k<WT, MODE, FIRST, false>;
    if (!attr_set) {
      VC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockDynSmem));
      attr_set = true;
    }
    kfn<<<grid_for(b.h_block, 1, kSMs * 4), kAggThreads, kBlockDynSmem, s>>>(
        b.block_list, b.counts + 0, g.off, g.adj, w, lab, lab_out, key, tkey, tval, cnt, nullptr, nullptr, 0);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_global > 0) {
    int grid_g = b.h_global < gt.blocks ? b.h_global : gt.blocks;
    agg_block_k<WT, MODE, FIRST, true><<<grid_g, kAggThreads, 0, s>>>(
        b.global_list, b.counts + 1, g.off, g.adj, w, lab, lab_out, key, tkey, tval, cnt, gt.keys, gt.vals, gt.cap);
    count_launch();
    VC_CHECK_LAUNCH();
  }
}

void lp_round(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* lab_in,
              int32_t* lab_out, uint64_t key, cudaStream_t s) {
  if (g.n <= 0) return;
  bool first = lab_in == nullptr;
  if (g.wbytes == 4) {
    if (first) launch_agg<int32_t, kModeLP, true>(g, b, gt, nullptr, lab_out, key, nullptr, nullptr, nullptr, s);
    else launch_agg<int32_t, kModeLP, false>(g, b, gt, lab_in, lab_out, key, nullptr, nullptr, nullptr, s);
  } else {
    if (first) launch_agg<long long, kModeLP, true>(g, b, gt, nullptr, lab_out, key, nullptr, nullptr, nullptr, s);
    else launch_agg<long long, kModeLP, false>(g, b, gt, lab_in, lab_out, key, nullptr, nullptr, nullptr, s);
  }
}

void emit_cross(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* cid,
                int32_t* tmp_key, long long* tmp_val, int32_t* cnt, cudaStream_t s) {
  if (g.n <= 0) return;
  if (g.wbytes == 4)
    launch_agg<int32_t, kModeEmit, false>(g, b, gt, cid, nullptr, 0, tmp_key, tmp_val, cnt, s);
  else
    launch_agg<long long, kModeEmit, false>(g, b, gt, cid, nullptr, 0, tmp_key, tmp_val, cnt, s);
}

}  // namespace vc
