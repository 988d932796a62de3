// Label propagation rounds and the pre-merge of cross-cluster edges.
//
// Both reduce, for every vertex v, the multiset {(key(u), c(v,u)) : u in N(v)} to
// per-key weight sums:
//   * label propagation (Sec. 4.1, "label propagation algorithm"): key = label of u,
//     then v takes the key of largest sum, ties by the larger tie hash;
//   * contraction pre-merge (Sec. 4.1, "contract it"): key = cluster id of u, keys
//     equal to v's own cluster dropped (intra-cluster edges vanish), every remaining
//     (key, sum) written out.
// A warp reads 32 neighbours at a time, groups the lanes holding equal keys with
// __match_any_sync and lets one leader per group add the group's weight to an
// open-addressing table (with unit weights the group weight is the group size).
// Lists of at most 32 entries need no table at all.  Work is split by list length:
//   small  (<= 128)  : a warp per vertex, 256-slot table in shared memory
//   mid    (<= 512)  : a warp per listed vertex, 1024-slot table in shared memory
//   block  (<= 4096) : a block per listed vertex, 8192-slot table in shared memory
//   global (larger)  : a block per listed vertex, table in global scratch.
#include <limits.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "kernels.cuh"
#include "prims.cuh"
#include "regvisit.cuh"

namespace vc {

constexpr int kWarpsPerBlock = 8;
constexpr int kAggThreads = kWarpsPerBlock * 32;
constexpr int kEmptyKey = -1;

enum { kModeLP = 0, kModeEmit = 1 };

// Binning in vertex order: each block takes a contiguous chunk, counts its classes
// (one global atomic per class and block reserves its positions), then writes the
// chunk's ids in order.
constexpr int kBinClasses = 5;  // small, reg, mid, block, global
__device__ __forceinline__ int bin_class(int64_t d) {
  return d <= 64 ? 0 : d <= kWarpMaxDeg ? 1 : d <= kMidMaxDeg ? 2 : d <= kBlockMaxDeg ? 3 : 4;
}
struct BinOut {
  int32_t* list[kBinClasses];
  int slot[kBinClasses];  // index of the class's count in Bins::counts
};

// With a vertex list (list_n not null), the listed vertices list[0, *list_n) are binned
// instead of [0, n) (n is then only the list's capacity).
__global__ void __launch_bounds__(256) bins_k(int64_t n, int64_t chunk, const int64_t* __restrict__ off, BinOut out,
                                              int* __restrict__ counts, const int32_t* __restrict__ list,
                                              const int* __restrict__ list_n) {
  __shared__ int s_cnt[kBinClasses], s_base[kBinClasses], s_run[kBinClasses], s_max;
  __shared__ int s_warp[8][kBinClasses];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (list_n) {  // the list's length is known on the device only: chunks follow from it
    n = *list_n;
    chunk = (n + gridDim.x - 1) / gridDim.x;
  }
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
  auto vert = [&](int64_t i) -> int64_t { return list_n ? (int64_t)list[i] : i; };
  if (tid < kBinClasses) { s_cnt[tid] = 0; s_run[tid] = 0; s_base[tid] = 0; }
  if (tid == 0) s_max = 0;
  __syncthreads();
  int c[kBinClasses] = {0, 0, 0, 0, 0};
  int dmax = 0;
  for (int64_t i = lo + tid; i < hi; i += 256) {
    const int64_t v = vert(i);
    const int64_t d = off[v + 1] - off[v];
    const int k = bin_class(d);
#pragma unroll
    for (int q = 0; q < kBinClasses; ++q) c[q] += k == q;
    if (k >= 2) dmax = max(dmax, (int)(d < INT_MAX ? d : INT_MAX));
  }
#pragma unroll
  for (int q = 0; q < kBinClasses; ++q) {
    const unsigned x = __reduce_add_sync(0xffffffffu, (unsigned)c[q]);
    if (lane == 0 && x) atomicAdd(&s_cnt[q], (int)x);
  }
  const unsigned m = __reduce_max_sync(0xffffffffu, (unsigned)dmax);
  if (lane == 0 && m) atomicMax(&s_max, (int)m);
  __syncthreads();
  if (tid < kBinClasses && s_cnt[tid]) s_base[tid] = atomicAdd(&counts[out.slot[tid]], s_cnt[tid]);
  if (tid == 0 && s_max) atomicMax(&counts[3], s_max);
  __syncthreads();
  for (int64_t b0 = lo; b0 < hi; b0 += 256) {  // the same trip count in every thread
    const int64_t i = b0 + tid;
    const int64_t v = i < hi ? vert(i) : -1;
    const int k = i < hi ? bin_class(off[v + 1] - off[v]) : -1;
    unsigned mine = 0;
#pragma unroll
    for (int q = 0; q < kBinClasses; ++q) {
      const unsigned bq = __ballot_sync(0xffffffffu, k == q);
      if (k == q) mine = bq;
      if (lane == 0) s_warp[wid][q] = __popc(bq);
    }
    __syncthreads();
    if (k >= 0) {
      int pos = s_base[k] + s_run[k] + __popc(mine & ((1u << lane) - 1u));
      for (int w2 = 0; w2 < wid; ++w2) pos += s_warp[w2][k];
      out.list[k][pos] = (int32_t)v;
    }
    __syncthreads();
    if (tid < kBinClasses) {
      int t = 0;
      for (int w2 = 0; w2 < 8; ++w2) t += s_warp[w2][tid];
      s_run[tid] += t;
    }
    __syncthreads();
  }
}

void bins_build(const GraphView& g, Bins& b, cudaStream_t s, const int32_t* list, const int* list_n) {
  VC_CUDA(cudaMemsetAsync(b.counts, 0, 6 * sizeof(int), s));
  if (g.n <= 0) return;
  const int64_t blocks = std::min<int64_t>((g.n + 255) / 256, (int64_t)kSMs * 8);
  const int64_t chunk = (g.n + blocks - 1) / blocks;
  BinOut out{{b.small_list, b.reg_list, b.mid_list, b.block_list, b.global_list}, {4, 5, 0, 1, 2}};
  bins_k<<<(int)blocks, 256, 0, s>>>(g.n, chunk, g.off, out, b.counts, list, list_n);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void hash_table_k(int64_t n, uint64_t key, const int32_t* __restrict__ gid,
                             const unsigned long long* __restrict__ gkey, const long long* __restrict__ gbase,
                             unsigned long long* __restrict__ hv) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (gid) {
      // batches: the label is hashed by its id inside its own graph
      const int g = gid[v];
      hv[v] = tie_hash(gkey[g], (int32_t)(v - gbase[g]));
    } else {
      hv[v] = tie_hash(key, (int32_t)v);
    }
  }
}

void hash_table(int64_t n, uint64_t key, const int32_t* gid, const unsigned long long* gkey, const long long* gbase,
                unsigned long long* hv, cudaStream_t s) {
  if (n <= 0) return;
  hash_table_k<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(n, key, gid, gkey, gbase, hv);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void count_changed_k(const int32_t* __restrict__ in, const int32_t* __restrict__ out, int64_t n,
                                long long* __restrict__ changed) {
  long long c = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    c += out[v] != (in ? in[v] : (int32_t)v);
  c = warp_sum(c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd((unsigned long long*)changed, (unsigned long long)c);
}

void count_changed(const int32_t* lab_in, const int32_t* lab_out, int64_t n, long long* changed, cudaStream_t s) {
  if (n <= 0) return;
  count_changed_k<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(lab_in, lab_out, n, changed);
  count_launch();
  VC_CHECK_LAUNCH();
}

// ------------------------------------------------------- asynchronous rounds
// Rounds in shuffled blocks of kAsyncBlock consecutive ids run in waves (see the
// declaration in kernels.cuh): the blocks' keys, each block's wave, each wave's members,
// and after a wave the members' new labels (with the first round's restriction).
__global__ void async_keys_k(int64_t nb, uint64_t key, uint64_t rk, unsigned long long* __restrict__ keys,
                             long long* __restrict__ vals) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
    keys[b] = mix64(key ^ rk ^ (uint64_t)b);
    vals[b] = b;
  }
}

// Position i of the ordered blocks belongs to wave k: the first nb % waves waves hold
// nb / waves + 1 blocks, the others nb / waves.
__global__ void async_waves_k(int64_t nb, int64_t waves, const long long* __restrict__ order,
                              unsigned char* __restrict__ wave_of) {
  const int64_t q = nb / waves, rmd = nb % waves;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i < rmd * (q + 1) ? i / (q + 1) : rmd + (i - rmd * (q + 1)) / q;
    wave_of[order[i]] = (unsigned char)k;
  }
}

__global__ void async_members_k(int64_t n, const unsigned char* __restrict__ wave_of, int k, int32_t* __restrict__ list,
                                int* __restrict__ count) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = b + lane;
    const bool in = v < n && wave_of[v / kAsyncBlock] == k;
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    int at = 0;
    if (lane == 0 && bal) at = atomicAdd(count, __popc(bal));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (in) list[at + __popc(bal & ((1u << lane) - 1u))] = (int32_t)v;
  }
}

// The wave's members take their new labels; in the first round a member some earlier
// wave moved into (joined) keeps its label.  Labels taken by a member that moved are
// recorded in took (marked into joined after the wave).
__global__ void async_apply_k(const int32_t* __restrict__ list, const int* __restrict__ count,
                              const int32_t* __restrict__ fresh, int32_t* __restrict__ lab,
                              const unsigned char* __restrict__ joined, int32_t* __restrict__ took) {
  const int c = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) {
    const int32_t v = list[i];
    int32_t L = fresh[v];
    if (joined && joined[v]) L = lab[v];
    if (took) took[i] = (L != lab[v] && L != v) ? L : -1;
    lab[v] = L;
  }
}

__global__ void async_mark_k(const int* __restrict__ count, const int32_t* __restrict__ took,
                             unsigned char* __restrict__ joined) {
  const int c = *count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x)
    if (took[i] >= 0) joined[took[i]] = 1;
}

void async_block_order(int64_t n, uint64_t key, int round, int64_t waves, unsigned long long* k0,
                       unsigned long long* k1, long long* v0, long long* v1, long long* hist, unsigned char* wave_of,
                       cudaStream_t s) {
  const int64_t nb = (n + kAsyncBlock - 1) / kAsyncBlock;
  async_keys_k<<<grid_for(nb, 256, kSMs * 4), 256, 0, s>>>(nb, key, mix64((uint64_t)round + 1), k0, v0);
  count_launch();
  VC_CHECK_LAUNCH();
  radix_sort_pairs(k0, v0, k1, v1, nb, 64, hist, s);
  async_waves_k<<<grid_for(nb, 256, kSMs * 4), 256, 0, s>>>(nb, waves < nb ? waves : nb, v0, wave_of);
  count_launch();
  VC_CHECK_LAUNCH();
}

void async_wave_members(int64_t n, const unsigned char* wave_of, int k, int32_t* list, int* count, cudaStream_t s) {
  VC_CUDA(cudaMemsetAsync(count, 0, sizeof(int), s));
  async_members_k<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(n, wave_of, k, list, count);
  count_launch();
  VC_CHECK_LAUNCH();
}

void async_apply(const int32_t* list, const int* count, int64_t cap, const int32_t* fresh, int32_t* lab,
                 unsigned char* joined, int32_t* took, cudaStream_t s) {
  const int grid = grid_for(cap, 256, kSMs * 8);
  async_apply_k<<<grid, 256, 0, s>>>(list, count, fresh, lab, joined, joined ? took : nullptr);
  count_launch();
  if (joined) {
    async_mark_k<<<grid, 256, 0, s>>>(count, took, joined);
    count_launch();
  }
  VC_CHECK_LAUNCH();
}

int64_t global_table_cap(int maxdeg) {
  int64_t c = 1;
  while (c < 2 * (int64_t)maxdeg) c <<= 1;
  return c < 64 ? 64 : c;
}

// Adds wt to the slot of key k (linear probing; capacity >= 2 x distinct keys, so a
// free slot always exists and the loop ends within one pass over the table).
// Returns the slot index if this call created the key, otherwise -1.
template <typename ACC>
__device__ __forceinline__ int tbl_add(int* tk, ACC* tv, int lg, int k, long long wt) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = slot_hash(k, lg);
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    int prev = atomicCAS(&tk[h], kEmptyKey, k);
    if (prev == kEmptyKey || prev == k) {
      atomicAdd(&tv[h], (ACC)wt);
      return prev == kEmptyKey ? (int)h : -1;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

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

// One chunk of up to 32 entries: every lane learns its key, whether it is used, and
// (on group leaders) the summed weight of the lanes sharing the key.
struct Chunk {
  int32_t k;
  bool use, leader;
  long long sum;
};

template <typename WT, int MODE, bool FIRST>
__device__ __forceinline__ Chunk load_chunk(int64_t e, int64_t end, const int32_t* __restrict__ adj,
                                            const WT* __restrict__ w, const int32_t* __restrict__ lab, int32_t own,
                                            long long* sw, int lane) {
  Chunk c;
  c.k = 0;
  c.use = false;
  long long wt = 0;
  if (e < end) {
    c.use = entry_key<MODE, FIRST>(lab, __ldg(adj + e), own, &c.k);
    wt = ldw(w, e);
  }
  // unused lanes get a unique negative key so they form singleton groups
  const int32_t km = c.use ? c.k : (-2 - lane);
  const unsigned peers = __match_any_sync(0xffffffffu, km);
  c.leader = c.use && (__ffs(peers) - 1) == lane;
  if (std::is_same<WT, UnitW>::value) {
    c.sum = __popc(peers);
  } else {
    sw[lane] = wt;
    __syncwarp();
    long long s = 0;
    if (c.leader)
      for (unsigned m = peers; m; m &= m - 1) s += sw[__ffs(m) - 1];
    __syncwarp();
    c.sum = s;
  }
  return c;
}

// Per-lane running best over (sum, hash, -label); the tie hash of a label is read
// from the level's table hv[L] = H(key, L), and only on ties.
struct LaneBest {
  long long s = -1;
  int l = INT_MAX;
  unsigned long long h = 0;
  bool hashed = false;
  __device__ __forceinline__ void add(long long sum, int L, const unsigned long long* __restrict__ hv) {
    if (sum > s) {
      s = sum;
      l = L;
      hashed = false;
    } else if (sum == s) {
      if (!hashed) { h = __ldg(hv + l); hashed = true; }
      unsigned long long hl = __ldg(hv + L);
      if (hl > h || (hl == h && L < l)) { l = L; h = hl; }
    }
  }
  __device__ __forceinline__ Cand done(const unsigned long long* __restrict__ hv) {
    if (!hashed && s >= 0) h = __ldg(hv + l);
    return Cand{s, h, l};
  }
};

// ------------------------------------------------------------------ warp classes
// Label propagation with a per-warp table.  LISTED = false: every vertex of list
// length <= CAP/2 (grid-stride over all vertices); LISTED = true: the listed vertices.
// The slots a vertex creates are recorded, so the final argmax visits only them.
template <typename WT, typename ACC, bool FIRST, int CAP, bool LISTED>
__global__ void __launch_bounds__(kAggThreads) lp_warp_k(
    int64_t n, const int32_t* __restrict__ list, const int* __restrict__ count_ptr,
    const int64_t* __restrict__ off, const int32_t* __restrict__ adj, const WT* __restrict__ w,
    const int32_t* __restrict__ lab, int32_t* __restrict__ lab_out, const unsigned long long* __restrict__ hv,
    const unsigned char* __restrict__ vact) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ long long s_w[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  ACC* tv = (ACC*)dyn + (size_t)wib * CAP;
  int* tk = (int*)((ACC*)dyn + (size_t)kWarpsPerBlock * CAP) + (size_t)wib * CAP;
  int* slots = (int*)((ACC*)dyn + (size_t)kWarpsPerBlock * CAP) + (size_t)kWarpsPerBlock * CAP + (size_t)wib * (CAP / 2);
  long long* sw = s_w[wib];
  for (int i = lane; i < CAP; i += 32) { tk[i] = kEmptyKey; tv[i] = 0; }
  __syncwarp();
  const int64_t total = LISTED ? (int64_t)*count_ptr : n;
  const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock;
  for (int64_t idx = (int64_t)blockIdx.x * kWarpsPerBlock + wib; idx < total; idx += stride) {
    const int64_t v = LISTED ? (int64_t)list[idx] : idx;
    if (vact && !vact[v]) continue;
    const int64_t beg = __ldg(off + v), end = __ldg(off + v + 1);
    const int d = (int)(end - beg);
    if (!LISTED && d > CAP / 2) continue;
    if (d == 0) {
      if (lane == 0) lab_out[v] = FIRST ? (int32_t)v : __ldg(lab + v);
      continue;
    }
    if (d <= 32) {
      // one chunk: the group sums are final, no table needed
      Chunk c = load_chunk<WT, kModeLP, FIRST>(beg + lane, end, adj, w, lab, 0, sw, lane);
      Cand cd = c.leader ? Cand{c.sum, __ldg(hv + c.k), c.k} : Cand{-1LL, 0ULL, INT_MAX};
      cd = warp_best(cd);
      if (lane == 0) lab_out[v] = cd.l;
      continue;
    }
    const int lg = ceil_log2(2 * (int64_t)d);
    int created = 0;  // warp-uniform count of recorded slots
    for (int64_t base = beg; base < end; base += 32) {
      Chunk c = load_chunk<WT, kModeLP, FIRST>(base + lane, end, adj, w, lab, 0, sw, lane);
      const int slot = c.leader ? tbl_add<ACC>(tk, tv, lg, c.k, c.sum) : -1;
      const unsigned bal = __ballot_sync(0xffffffffu, slot >= 0);
      if (slot >= 0) slots[created + __popc(bal & ((1u << lane) - 1u))] = slot;
      created += __popc(bal);
    }
    __syncwarp();
    LaneBest lb;
    for (int i = lane; i < created; i += 32) {
      const int slot = slots[i];
      lb.add((long long)tv[slot], tk[slot], hv);
      tk[slot] = kEmptyKey;
      tv[slot] = 0;
    }
    Cand cd = warp_best(lb.done(hv));
    if (lane == 0) lab_out[v] = cd.l;
    __syncwarp();
  }
}

// ------------------------------------------------------------ register class
// Lists of at most kWarpMaxDeg = 128 entries.  A group of G lanes (G = 16 for lists
// of at most 64 entries, two vertices per warp; G = 32 for 65..128) holds the whole
// list in registers (slot r of group lane i holds entry G r + i) and visits its
// distinct keys one at a time, slot by slot: the first lane whose slot r is still
// unvisited broadcasts its key, every lane marks its entries holding it (only slots
// >= r can), and a group reduction gives the key's count (unit weights) or weight
// sum.  No table and no shared memory: one short step per distinct key.  The groups
// of a warp step in lockstep (the loops run while any group has work; a group
// without work idles), so every warp-wide vote and shuffle has all lanes present.
//
// A vertex needs three dependent reads (its offsets, its neighbour ids, their keys),
// so the warp software-pipelines its vertices: while it works on one vertex per
// group it already holds the next vertex's ids and the offsets of the one after.

constexpr int kEmitBailKeys = 64;
constexpr int kEmitWalkKeys = 6;
constexpr int kEmitBlockPerVertexMax = kSMs * 8;  // block-class lists pre-merged a block each
constexpr int kLpBailKeys = 16;
constexpr int kLpWalkKeys = 8;      // short classes: labels walked before the table
constexpr int kLpTableMaxS = 4;     // classes of at most this many slots per lane
constexpr int kLpTableSlots = 256;  // table slots per warp (split between its groups)
// The table serves weighted graphs only: on unit weights its registers and shared
// memory cost an SM block of the kernel, and lists with many labels are rare there.
template <typename WT, int S>
constexpr bool lp_has_table() { return S <= kLpTableMaxS && !std::is_same<WT, UnitW>::value; }

// Neighbour ids (and weights) of one list in registers.
template <int S>
struct RegIds {
  int32_t u[S];
  long long wt[S];
};

template <typename WT, int G, int S>
__device__ __forceinline__ void reg_ids(RegIds<S>& R, int64_t beg, int64_t end, int glane,
                                        const int32_t* __restrict__ adj, const WT* __restrict__ w) {
  const int64_t dd = end - beg;
  const int d = dd > S * G ? 0 : (int)dd;
  const int32_t* a = adj + beg;
#pragma unroll
  for (int r = 0; r < S; ++r) {
    const int i = glane + G * r;
    R.u[r] = -1;
    R.wt[r] = 0;
    if (i < d) {
      R.u[r] = __ldcs(a + i);  // read once: evict first, keeping the gathered labels in L2
      R.wt[r] = ldw(w, beg + i);
    }
  }
}

template <int MODE, bool FIRST, int G, int S>
__device__ __forceinline__ void reg_keys(RegList<S>& L, const RegIds<S>& R, int deg, const int32_t* __restrict__ lab,
                                         int32_t own) {
  L.slots = (deg + G - 1) / G;
  L.todo = 0;
#pragma unroll
  for (int r = 0; r < S; ++r) {
    L.k[r] = -1;
    L.wt[r] = R.wt[r];
    if (R.u[r] >= 0) {
      int32_t kk;
      if (entry_key<MODE, FIRST>(lab, R.u[r], own, &kk)) L.todo |= 1u << r;
      L.k[r] = kk;
    }
  }
}

// The pipelined vertex loop of a warp over a vertex list.  Group g of the warp takes
// list entry i + g for i = first, first + stride, ... < total (the trip count is the
// same in every lane); body(v, valid, beg, end, pre, ids) runs with v's ids already
// in registers.  `pre(v)` is read with the offsets one entry ahead (e.g. v's own
// cluster id).
template <typename WT, int G, int S, typename PRE, typename BODY>
__device__ __forceinline__ void reg_pipeline(const int32_t* __restrict__ list, int64_t total, int64_t first,
                                             int64_t stride, int glane, int gi, const int64_t* __restrict__ off,
                                             const int32_t* __restrict__ adj, const WT* __restrict__ w, PRE pre,
                                             BODY body) {
  int64_t base = first;
  if (base >= total) return;  // the same in every lane (base is per warp)
  auto fetch = [&](int64_t b, int64_t& v, int64_t& bg, int64_t& en, int32_t& x) {
    v = -1;
    bg = en = 0;
    x = 0;
    if (b + gi < total) {
      v = __ldg(list + b + gi);
      bg = __ldg(off + v);
      en = __ldg(off + v + 1);
      x = pre(v);
    }
  };
  int64_t v, beg, end, vn, nbeg, nend;
  int32_t x, xn;
  fetch(base, v, beg, end, x);
  RegIds<S> cur;
  reg_ids<WT, G, S>(cur, beg, end, glane, adj, w);
  int64_t bn = base + stride;
  fetch(bn, vn, nbeg, nend, xn);
  for (;;) {
    RegIds<S> nxt;
    int64_t vnn = -1, nnbeg = 0, nnend = 0;
    int32_t xnn = 0;
    const int64_t bnn = bn + stride;
    if (bn < total) {
      reg_ids<WT, G, S>(nxt, nbeg, nend, glane, adj, w);
      fetch(bnn, vnn, nnbeg, nnend, xnn);
    }
    body(v, v >= 0, beg, end, x, cur);
    if (bn >= total) break;
    base = bn; v = vn; beg = nbeg; end = nend; x = xn; cur = nxt;
    bn = bnn; vn = vnn; nbeg = nnbeg; nend = nnend; xn = xnn;
  }
}

// The listed vertices (all of length <= S G), G lanes each, S slots per lane.
template <typename WT, typename ACC, bool FIRST, int G, int S>
__global__ void __launch_bounds__(kAggThreads) lp_reg_k(const int32_t* __restrict__ list,
                                                        const int* __restrict__ count_ptr,
                                                        const int64_t* __restrict__ off,
                                                        const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                        const int32_t* __restrict__ lab, int32_t* __restrict__ lab_out,
                                                        const unsigned long long* __restrict__ hv,
                                                        const unsigned char* __restrict__ vact,
                                                        int32_t* __restrict__ bail_list,
                                                        int* __restrict__ bail_count) {
  const int lane = threadIdx.x & 31, glane = lane & (G - 1), gi = lane / G;
  const unsigned gmask = group_mask<G>(lane);
  constexpr int kPer = 32 / G;  // vertices per warp
  // the short classes' tables (see below), one region of kLpTableSlots per warp
  __shared__ int32_t s_tab_k[lp_has_table<WT, S>() ? kWarpsPerBlock * kLpTableSlots : 1];
  __shared__ ACC s_tab_v[lp_has_table<WT, S>() ? kWarpsPerBlock * kLpTableSlots : 1];
  int32_t* tab_k = s_tab_k + (lp_has_table<WT, S>() ? (threadIdx.x >> 5) * kLpTableSlots : 0);
  ACC* tab_v = s_tab_v + (lp_has_table<WT, S>() ? (threadIdx.x >> 5) * kLpTableSlots : 0);
  if (lp_has_table<WT, S>()) {
    for (int i = lane; i < kLpTableSlots; i += 32) {
      tab_k[i] = kEmptyKey;
      tab_v[i] = 0;
    }
    __syncwarp();
  }
  const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock * kPer;
  const int64_t first = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kPer;
  // pre(v): v's own label from the previous round (INT_MIN: v is not active)
  reg_pipeline<WT, G, S>(list, *count_ptr, first, stride, glane, gi, off, adj, w,
                      [&](int64_t v) -> int32_t {
                        if (vact && !vact[v]) return INT_MIN;
                        return FIRST ? 0 : __ldg(lab + v);
                      },
                      [&](int64_t v, bool valid, int64_t beg, int64_t end, int32_t own, const RegIds<S>& ids) {
    const int64_t d = end - beg;
    const bool mine = valid && own != INT_MIN;
    if (mine && d == 0) {
      if (glane == 0) lab_out[v] = FIRST ? (int32_t)v : __ldg(lab + v);
    }
    RegList<S> L;
    reg_keys<kModeLP, FIRST, G, S>(L, ids, mine ? (int)d : 0, lab, 0);
    if (!mine) L.todo = 0;
    // running best (sum, hash, -label), the same in the group's lanes; the hash of
    // the best is read only once a tie needs it.  `left` is the weight of the keys not
    // visited yet: once the best exceeds it, no other key can reach the best, and the
    // walk stops (a majority label usually ends it after its own visit).
    ACC left;
    if (std::is_same<WT, UnitW>::value) {
      left = (ACC)(mine ? d : 0);
    } else {
      long long sum = 0;
#pragma unroll
      for (int r = 0; r < S; ++r)
        if (L.todo >> r & 1u) sum += L.wt[r];
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      left = (ACC)sum;
    }
    ACC bs = 0;
    int32_t bl = -1;
    unsigned long long bh = 0;
    bool hashed = false;
    if (!FIRST) {
      // the vertex's own label first: after one round most vertices see it on more than
      // half of their weight, and then no other label can reach it (the walk is skipped);
      // otherwise it seeds the best, and the walk visits only the other labels
      unsigned hit = 0;
#pragma unroll
      for (int r = 0; r < S; ++r)
        if (((L.todo >> r) & 1u) && L.k[r] == own) hit |= 1u << r;
      ACC t;
      if (std::is_same<WT, UnitW>::value) {
        t = (ACC)__reduce_add_sync(gmask, (unsigned)__popc(hit));
      } else {
        long long sum = 0;
#pragma unroll
        for (int r = 0; r < S; ++r)
          if ((hit >> r) & 1u) sum += L.wt[r];
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        t = (ACC)sum;
      }
      L.todo &= ~hit;
      if (t > 0) {
        left -= t;
        bs = t;
        bl = own;
        if (bs > left) L.todo = 0;
      }
    }
    // a vertex still undecided after a number of labels (a list whose neighbours carry
    // many different labels, where a step per label costs slots x compares) goes on
    // elsewhere: with a bail list (long class) to the hash-table kernel after
    // kLpBailKeys labels; in the short classes, after kLpWalkKeys labels, its remaining
    // entries are summed in the group's shared-memory table below
    int visited = 0;
    bool bailed = false;
    unsigned rest = 0;
    reg_visit<WT, ACC, G, S>(L, gmask, [&](int32_t kk, ACC t) {
      left -= t;
      if (bl < 0 || t > bs) {
        bs = t;
        bl = kk;
        hashed = false;
      } else if (t == bs) {
        if (!hashed) { bh = __ldg(hv + bl); hashed = true; }
        const unsigned long long h = __ldg(hv + kk);
        if (h > bh || (h == bh && kk < bl)) { bh = h; bl = kk; }
      }
      if (bs > left) return true;
      ++visited;
      if (bail_list) {
        if (visited >= kLpBailKeys) {
          bailed = true;
          return true;
        }
      } else if (lp_has_table<WT, S>() && visited >= kLpWalkKeys) {
        rest = L.todo;
        return true;
      }
      return false;
    });
    if constexpr (lp_has_table<WT, S>()) if (!bail_list && __any_sync(0xffffffffu, rest != 0u)) {
      // the group's table: CAPG slots (twice its list capacity); every remaining entry
      // adds its weight to its label's slot, then the group takes the best slot and
      // compares it with the walk's best; the slots are emptied for the next vertex
      constexpr int CAPG = kLpTableSlots / (32 / G);
      constexpr int LG = CAPG >= 256 ? 8 : 7;
      static_assert((1 << LG) == CAPG && CAPG >= 2 * S * G, "table of twice the list capacity");
      int32_t* tk = tab_k + gi * CAPG;
      ACC* tv = tab_v + gi * CAPG;
      const bool grest = (__ballot_sync(0xffffffffu, rest != 0u) & gmask) != 0u;
#pragma unroll
      for (int r = 0; r < S; ++r)
        if ((rest >> r) & 1u) tbl_add<ACC>(tk, tv, LG, L.k[r], L.wt[r]);
      __syncwarp();
      LaneBest lb;
      if (grest) {
        for (int i = glane; i < CAPG; i += G) {
          const int32_t key = tk[i];
          if (key != kEmptyKey) {
            lb.add((long long)tv[i], key, hv);
            tk[i] = kEmptyKey;
            tv[i] = 0;
          }
        }
      }
      Cand cd = lb.done(hv);
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        Cand e;
        e.s = __shfl_xor_sync(0xffffffffu, cd.s, o);
        e.h = __shfl_xor_sync(0xffffffffu, cd.h, o);
        e.l = __shfl_xor_sync(0xffffffffu, cd.l, o);
        if (better(e, cd)) cd = e;
      }
      if (grest) {
        if (bl >= 0) {
          const Cand wb{(long long)bs, hashed ? bh : __ldg(hv + bl), bl};
          if (better(wb, cd)) cd = wb;
        }
        bl = cd.l;
      }
      __syncwarp();
    }
    if (mine && d > 0 && glane == 0) {
      if (bailed) bail_list[atomicAdd(bail_count, 1)] = (int32_t)v;
      else lab_out[v] = bl;
    }
  });
}

// Pre-merge of the register class: one (key, sum) per distinct foreign cluster of the
// whole list; group lane i keeps the i-th pair of each run of G pairs, and a full run
// is written with one coalesced store.
template <typename WT, int G, int S>
__global__ void __launch_bounds__(kAggThreads) emit_reg_k(const int32_t* __restrict__ list,
                                                          const int* __restrict__ count_ptr,
                                                          const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                          const int32_t* __restrict__ cid, PairOut out,
                                                          int32_t* __restrict__ cnt, int32_t* __restrict__ bail_list,
                                                          int* __restrict__ bail_count) {
  const int lane = threadIdx.x & 31, glane = lane & (G - 1), gi = lane / G;
  const unsigned gmask = group_mask<G>(lane);
  constexpr int kPer = 32 / G;
  const int64_t stride = (int64_t)gridDim.x * kWarpsPerBlock * kPer;
  const int64_t first = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kPer;
  const bool rows = out.by_rows();
  reg_pipeline<WT, G, S>(list, *count_ptr, first, stride, glane, gi, off, adj, w,
                      [&](int64_t v) { return __ldg(cid + v); },
                      [&](int64_t v, bool valid, int64_t beg, int64_t end, int32_t own, const RegIds<S>& ids) {
    const int64_t d = end - beg;
    const bool mine = valid;
    RegList<S> L;
    reg_keys<kModeEmit, false, G, S>(L, ids, (mine && own >= 0) ? (int)d : 0, cid, own);
    if (!(mine && own >= 0)) L.todo = 0;
    int made = 0;  // the same in the group's lanes
    // one pass per row r (entries r G .. r G + G - 1) over the entries still to do:
    // lanes holding the same key (tagged with the group) match, the lowest of them sums
    // its peers' weights and writes the pair (a key met in several rows gives several
    // pairs, which the cluster merge sums)
    auto row_pass = [&]() {
      const int ws = __reduce_max_sync(0xffffffffu, L.slots);
#pragma unroll
      for (int r = 0; r < S; ++r) {
        if (r >= ws) break;
        const bool use = (L.todo >> r) & 1u;
        const unsigned long long tag =
            use ? ((unsigned long long)(uint32_t)L.k[r] | ((unsigned long long)gi << 32))
                : (0xffffffff00000000ull | (unsigned long long)lane);
        const unsigned peers = __match_any_sync(0xffffffffu, tag);
        const bool lead = use && (__ffs(peers) - 1) == lane;
        long long sum;
        if (std::is_same<WT, UnitW>::value) {
          sum = __popc(peers);
        } else {
          sum = L.wt[r];
          unsigned rest = lead ? (peers & (peers - 1u)) : 0u;
          while (__any_sync(0xffffffffu, rest != 0u)) {
            const long long x = __shfl_sync(0xffffffffu, L.wt[r], rest ? __ffs(rest) - 1 : lane);
            if (rest) {
              sum += x;
              rest &= rest - 1u;
            }
          }
        }
        const unsigned lb = __ballot_sync(0xffffffffu, lead) & gmask;
        if (lead) out.put(v, beg, made + __popc(lb & ((1u << lane) - 1u)), L.k[r], sum);
        made += __popc(lb);
      }
      L.todo = 0;
    };
    auto finish = [&]() {
      if (mine && glane == 0) {
        cnt[v] = made;
        if (out.ccount && made) atomicAdd(&out.ccount[own], made);
      }
    };
    if (rows) {
      row_pass();
      finish();
      return;
    }
    int32_t pk = 0;
    long long pv = 0;
    // the walk takes one step per distinct key.  In the short classes (no bail list) a
    // group still holding keys after kEmitWalkKeys steps (a list with many foreign
    // clusters) finishes with the row pass; in the long class a list reaching
    // kEmitBailKeys keys is handed to the chunk kernel.
    bool bailed = false;
    unsigned left = 0;
    reg_visit<WT, long long, G, S>(L, gmask, [&](int32_t kk, long long t) {
      if (glane == (made & (G - 1))) { pk = kk; pv = t; }
      if ((++made & (G - 1)) == 0) out.put(v, beg, made - G + glane, pk, pv);
      if (bail_list) {
        if (made >= kEmitBailKeys) { bailed = true; return true; }
      } else if (made >= kEmitWalkKeys) {
        left = L.todo;
        return true;
      }
      return false;
    });
    if (bailed) {
      if (glane == 0) bail_list[atomicAdd(bail_count, 1)] = (int32_t)v;
      return;
    }
    if (glane < (made & (G - 1))) out.put(v, beg, (made & ~(G - 1)) + glane, pk, pv);
    L.todo = left;
    if (__any_sync(0xffffffffu, left != 0u)) row_pass();
    finish();
  });
}

template <int CAP, typename ACC>
constexpr size_t warp_smem();
template <typename F>
void set_smem(F kfn, size_t bytes);

// The vertices a register-class kernel handed on: a warp per vertex with a hash table of
// CAP slots in shared memory (the bail list and its count are read on the device).
template <typename WT, typename ACC, bool FIRST, int CAP>
void launch_lp_bailed(const GraphView& g, const Bins& b, const WT* w, const int32_t* lab, int32_t* lab_out,
                      const unsigned long long* hv, cudaStream_t s) {
  constexpr size_t smem = warp_smem<CAP, ACC>();
  auto kfn = lp_warp_k<WT, ACC, FIRST, CAP, true>;
  set_smem(kfn, smem);
  kfn<<<kSMs * 2, kAggThreads, smem, s>>>(0, b.bail_list, b.counts + 7, g.off, g.adj, w, lab, lab_out, hv, g.vact);
  count_launch();
  VC_CHECK_LAUNCH();
}

// Register classes.  In rounds after the first, mid-class vertices (129..512 entries, 16
// slots per lane, where a step per distinct label is costly) with many distinct labels
// go on to the hash-table kernel (the bail list and counts[7] are free during label
// propagation: the pre-merge uses them later).  Lists of at most 128 entries keep the
// walk: four slots per lane make each step cheap, and measured, the table kernel did not
// beat it there.
template <typename WT, typename ACC, bool FIRST>
void launch_lp_reg(const GraphView& g, const Bins& b, const WT* w, const int32_t* lab, int32_t* lab_out,
                   const unsigned long long* hv, cudaStream_t s, bool mid_bail) {
  int32_t* bl = (FIRST || !mid_bail) ? nullptr : b.bail_list;
  int* bc = (FIRST || !mid_bail) ? nullptr : b.counts + 7;
  if (b.h_small > 0) {
    lp_reg_k<WT, ACC, FIRST, 16, 4><<<grid_for(b.h_small, kWarpsPerBlock * 2, kSMs * 16), kAggThreads, 0, s>>>(
        b.small_list, b.counts + 4, g.off, g.adj, w, lab, lab_out, hv, g.vact, nullptr, nullptr);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_reg > 0) {
    lp_reg_k<WT, ACC, FIRST, 32, 4><<<grid_for(b.h_reg, kWarpsPerBlock, kSMs * 16), kAggThreads, 0, s>>>(
        b.reg_list, b.counts + 5, g.off, g.adj, w, lab, lab_out, hv, g.vact, nullptr, nullptr);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_mid > 0) {
    if (bc) VC_CUDA(cudaMemsetAsync(bc, 0, sizeof(int), s));
    lp_reg_k<WT, ACC, FIRST, 32, kMidMaxDeg / 32><<<grid_for(b.h_mid, kWarpsPerBlock, kSMs * 16), kAggThreads, 0, s>>>(
        b.mid_list, b.counts + 0, g.off, g.adj, w, lab, lab_out, hv, g.vact, bl, bc);
    count_launch();
    VC_CHECK_LAUNCH();
    if (bc) launch_lp_bailed<WT, ACC, FIRST, kMidCap>(g, b, w, lab, lab_out, hv, s);
  }
}


// First round on a graph whose lists are strictly increasing: every neighbour is its
// own label, so S(u) = c(v,u) and the choice is the argmax of (c(v,u), hash(u), -u)
// over the list; no accumulation needed.  A warp per vertex (lengths <= MAXD) or, for
// the listed longer lists, a block per vertex.
template <typename WT>
__device__ __forceinline__ void first_scan(LaneBest& lb, int64_t a, int64_t end, int step,
                                           const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                           const unsigned long long* __restrict__ hv) {
  for (int64_t e = a; e < end; e += step) lb.add(ldw(w, e), __ldg(adj + e), hv);
}

// Group-wide best candidate over the G lanes of `gmask` (lane-local group of G lanes).
template <int G>
__device__ __forceinline__ Cand group_best(Cand c, unsigned gmask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    Cand d;
    d.s = __shfl_xor_sync(gmask, c.s, o);
    d.h = __shfl_xor_sync(gmask, c.h, o);
    d.l = __shfl_xor_sync(gmask, c.l, o);
    if (better(d, c)) c = d;
  }
  return c;
}

// G lanes per vertex (32 / G vertices per warp in flight).
template <typename WT, int G>
__global__ void __launch_bounds__(kAggThreads) lp_first_simple_k(int64_t n, int maxd,
                                                                 const int64_t* __restrict__ off,
                                                                 const int32_t* __restrict__ adj,
                                                                 const WT* __restrict__ w,
                                                                 int32_t* __restrict__ lab_out,
                                                                 const unsigned long long* __restrict__ hv,
                                                                 const unsigned char* __restrict__ vact) {
  const int lane = threadIdx.x & 31, glane = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += groups) {
    if (vact && !vact[v]) continue;
    const int64_t beg = __ldg(off + v), end = __ldg(off + v + 1);
    if (end - beg > maxd) continue;
    if (end == beg) {
      if (glane == 0) lab_out[v] = (int32_t)v;
      continue;
    }
    if (std::is_same<WT, UnitW>::value) {
      // unit weights: every neighbour has strength 1, so the choice is the neighbour
      // of largest tie hash
      // distinct ids have distinct hashes (mix64 is a bijection), so the largest
      // hash alone decides; bl < 0 marks a lane without entries.  Four entries per
      // lane in flight: ids first, then their hashes.
      unsigned long long bh = 0;
      int bl = -1;
      const int d = (int)(end - beg);
      const int32_t* a = adj + beg;
      for (int i0 = glane; i0 < d; i0 += 4 * G) {
        int u[4];
        unsigned long long h[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) u[r] = i0 + r * G < d ? __ldcs(a + i0 + r * G) : -1;  // read once
#pragma unroll
        for (int r = 0; r < 4; ++r) h[r] = u[r] >= 0 ? __ldg(hv + u[r]) : 0ULL;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (u[r] >= 0 && (h[r] > bh || bl < 0)) { bh = h[r]; bl = u[r]; }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        const unsigned long long oh = __shfl_xor_sync(gmask, bh, o);
        const int ol = __shfl_xor_sync(gmask, bl, o);
        if (ol >= 0 && (bl < 0 || oh > bh)) { bh = oh; bl = ol; }
      }
      if (glane == 0) lab_out[v] = bl;
    } else {
      LaneBest lb;
      first_scan(lb, beg + glane, end, G, adj, w, hv);
      Cand cd = group_best<G>(lb.done(hv), gmask);
      if (glane == 0) lab_out[v] = cd.l;
    }
  }
}

template <typename WT>
__global__ void __launch_bounds__(kAggThreads) lp_first_simple_block_k(const int32_t* __restrict__ list,
                                                                       const int* __restrict__ count_ptr,
                                                                       const int64_t* __restrict__ off,
                                                                       const int32_t* __restrict__ adj,
                                                                       const WT* __restrict__ w,
                                                                       int32_t* __restrict__ lab_out,
                                                                       const unsigned long long* __restrict__ hv,
                                                                       const unsigned char* __restrict__ vact) {
  __shared__ Cand s_best[kWarpsPerBlock];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    if (vact && !vact[v]) continue;
    LaneBest lb;
    first_scan(lb, off[v] + threadIdx.x, off[v + 1], kAggThreads, adj, w, hv);
    Cand cd = warp_best(lb.done(hv));
    if (lane == 0) s_best[wib] = cd;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b = s_best[0];
      for (int q = 1; q < kWarpsPerBlock; ++q)
        if (better(s_best[q], b)) b = s_best[q];
      lab_out[v] = b.l;
    }
    __syncthreads();
  }
}

// Pre-merge without a table: within each 32-entry chunk the warp walks the distinct
// foreign cluster ids (a chunk touches few of them: most neighbours share v's own
// cluster), summing each one's weight with a ballot (unit weights) or a warp sum, and
// the first lane holding the id writes the pair; the cluster merge that follows merges
// equal ids across chunks and across vertices.  `next_slot` yields the pair's index.
template <typename WT, int G, typename SLOT>
__device__ __forceinline__ void emit_chunk(int64_t e, int64_t end, const int32_t* __restrict__ adj,
                                           const WT* __restrict__ w, const int32_t* __restrict__ cid, int32_t own,
                                           int lane, unsigned gmask, const PairOut& out, int64_t v, int64_t beg,
                                           SLOT next_slot) {
  int32_t k = -1;
  long long wt = 0;
  bool use = false;
  if (e < end) {
    k = __ldg(cid + __ldg(adj + e));
    use = k != own;
    wt = ldw(w, e);
  }
  unsigned todo = __ballot_sync(gmask, use) & gmask;
  while (todo) {
    const int leader = __ffs(todo) - 1;
    const int32_t key = __shfl_sync(gmask, k, leader);
    const bool mine = use && k == key;
    const unsigned peers = __ballot_sync(gmask, mine) & gmask;
    long long sum;
    if (std::is_same<WT, UnitW>::value) {
      sum = __popc(peers);
    } else {
      sum = mine ? wt : 0LL;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(gmask, sum, o);
    }
    const int i = next_slot(leader);
    if (lane == leader) out.put(v, beg, i, key, sum);
    todo &= ~peers;
  }
}

// The same chunk, pre-merged with one match: the lowest lane holding each foreign key
// sums its peers' weights and writes the pair.  The cost does not grow with the
// distinct keys of the chunk (lists whose neighbours are nearly all in clusters of their
// own).  `reserve(k)` returns the index of the chunk's first of k pairs.
template <typename WT, int G, typename RESERVE>
__device__ __forceinline__ void emit_chunk_rows(int64_t e, int64_t end, const int32_t* __restrict__ adj,
                                                const WT* __restrict__ w, const int32_t* __restrict__ cid,
                                                int32_t own, int lane, unsigned gmask, const PairOut& out, int64_t v,
                                                int64_t beg, RESERVE reserve) {
  int32_t k = -1;
  long long wt = 0;
  bool use = false;
  if (e < end) {
    k = __ldg(cid + __ldg(adj + e));
    use = k != own;
    wt = ldw(w, e);
  }
  const unsigned long long tag = use ? (unsigned long long)(uint32_t)k : (0xffffffff00000000ull | (unsigned)lane);
  const unsigned peers = __match_any_sync(gmask, tag);
  const bool lead = use && (__ffs(peers) - 1) == lane;
  long long sum;
  if (std::is_same<WT, UnitW>::value) {
    sum = __popc(peers);
  } else {
    sum = wt;
    unsigned rest = lead ? (peers & (peers - 1u)) : 0u;
    while (__any_sync(gmask, rest != 0u)) {
      const long long x = __shfl_sync(gmask, wt, rest ? __ffs(rest) - 1 : lane);
      if (rest) {
        sum += x;
        rest &= rest - 1u;
      }
    }
  }
  const unsigned lb = __ballot_sync(gmask, lead) & gmask;
  if (lb == 0u) return;
  const int at = reserve(__popc(lb));
  if (lead) out.put(v, beg, at + __popc(lb & ((1u << lane) - 1u)), k, sum);
}

// Listed vertices (the mid and block classes), G lanes per vertex: 32 / G vertices
// per warp, each group walking its list in G-entry chunks.
template <typename WT, int G>
__global__ void __launch_bounds__(kAggThreads) emit_warp_k(const int32_t* __restrict__ list,
                                                           const int* __restrict__ count_ptr,
                                                           const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                           const int32_t* __restrict__ cid, PairOut out,
                                                           int32_t* __restrict__ cnt) {
  const int lane = threadIdx.x & 31, glane = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  const int64_t total = *count_ptr;
  const bool rows = out.by_rows();
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; i < total; i += groups) {
    const int32_t v = __ldg(list + i);
    const int64_t beg = __ldg(off + v), end = __ldg(off + v + 1);
    const int32_t own = __ldg(cid + v);
    int made = 0;  // group-uniform
    if (own >= 0) {
      if (rows)
        for (int64_t base = beg; base < end; base += G)
          emit_chunk_rows<WT, G>(base + glane, end, adj, w, cid, own, lane, gmask, out, v, beg, [&](int k) {
            const int at = made;
            made += k;
            return at;
          });
      else
        for (int64_t base = beg; base < end; base += G)
          emit_chunk<WT, G>(base + glane, end, adj, w, cid, own, lane, gmask, out, v, beg,
                            [&](int) { return made++; });
    }
    if (glane == 0) {
      cnt[v] = made;
      if (out.ccount && made) atomicAdd(&out.ccount[own], made);
    }
  }
}

template <typename WT>
__global__ void __launch_bounds__(kAggThreads) emit_block_k(const int32_t* __restrict__ list,
                                                            const int* __restrict__ count_ptr,
                                                            const int64_t* __restrict__ off,
                                                            const int32_t* __restrict__ adj,
                                                            const WT* __restrict__ w, const int32_t* __restrict__ cid,
                                                            PairOut out, int32_t* __restrict__ cnt) {
  __shared__ int s_made;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int count = *count_ptr;
  const bool rows = out.by_rows();
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    const int64_t beg = off[v], end = off[v + 1];
    const int32_t own = cid[v];
    if (threadIdx.x == 0) s_made = 0;
    __syncthreads();
    if (own >= 0) {
      if (rows)
        for (int64_t base = beg + 32 * wib; base < end; base += 32 * kWarpsPerBlock)
          emit_chunk_rows<WT, 32>(base + lane, end, adj, w, cid, own, lane, 0xffffffffu, out, v, beg, [&](int k) {
            int at = 0;
            if (lane == 0) at = atomicAdd(&s_made, k);
            return __shfl_sync(0xffffffffu, at, 0);
          });
      else
        for (int64_t base = beg + 32 * wib; base < end; base += 32 * kWarpsPerBlock)
          emit_chunk<WT, 32>(base + lane, end, adj, w, cid, own, lane, 0xffffffffu, out, v, beg, [&](int leader) {
            int at = 0;
            if (lane == leader) at = atomicAdd(&s_made, 1);
            return __shfl_sync(0xffffffffu, at, leader);
          });
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      cnt[v] = s_made;
      if (out.ccount && s_made) atomicAdd(&out.ccount[own], s_made);
    }
    __syncthreads();
  }
}

// --------------------------------------------------------- block / global classes
// Label propagation, one block per listed vertex; the table lives in shared memory
// (GLOBAL = false) or in this block's region of global scratch (GLOBAL = true).
template <typename WT, typename ACC, bool FIRST, bool GLOBAL>
__global__ void __launch_bounds__(kAggThreads) lp_block_k(
    const int32_t* __restrict__ list, const int* __restrict__ count_ptr, const int64_t* __restrict__ off,
    const int32_t* __restrict__ adj, const WT* __restrict__ w, const int32_t* __restrict__ lab,
    int32_t* __restrict__ lab_out, const unsigned long long* __restrict__ hv, int32_t* __restrict__ gkeys,
    long long* __restrict__ gvals, int64_t gcap, const unsigned char* __restrict__ vact) {
  extern __shared__ __align__(16) unsigned char dyn[];
  __shared__ Cand s_best[kWarpsPerBlock];
  __shared__ long long s_w[kWarpsPerBlock][32];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int* tk;
  ACC* tv;
  int64_t table_cap;
  if (GLOBAL) {
    tk = gkeys + (int64_t)blockIdx.x * gcap;
    tv = (ACC*)gvals + (int64_t)blockIdx.x * gcap;
    table_cap = gcap;
  } else {
    tv = (ACC*)dyn;
    tk = (int*)((ACC*)dyn + kBlockCap);
    table_cap = kBlockCap;
  }
  long long* sw = s_w[wib];
  for (int64_t i = threadIdx.x; i < table_cap; i += kAggThreads) { tk[i] = kEmptyKey; tv[i] = 0; }
  __syncthreads();
  const int count = *count_ptr;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int32_t v = list[idx];
    if (vact && !vact[v]) continue;
    const int64_t beg = off[v], end = off[v + 1];
    const int64_t d = end - beg;
    const int lg = ceil_log2(2 * d);
    const int64_t cap = (int64_t)1 << lg;
    for (int64_t base = beg + 32 * wib; base < end; base += 32 * kWarpsPerBlock) {
      Chunk c = load_chunk<WT, kModeLP, FIRST>(base + lane, end, adj, w, lab, 0, sw, lane);
      if (c.leader) tbl_add<ACC>(tk, tv, lg, c.k, c.sum);
    }
    __syncthreads();
    LaneBest lb;
    for (int64_t i = threadIdx.x; i < cap; i += kAggThreads) {
      const int L = tk[i];
      if (L != kEmptyKey) {
        lb.add((long long)tv[i], L, hv);
        tk[i] = kEmptyKey;
        tv[i] = 0;
      }
    }
    Cand cd = warp_best(lb.done(hv));
    if (lane == 0) s_best[wib] = cd;
    __syncthreads();
    if (threadIdx.x == 0) {
      Cand b = s_best[0];
      for (int q = 1; q < kWarpsPerBlock; ++q)
        if (better(s_best[q], b)) b = s_best[q];
      lab_out[v] = b.l;
    }
    __syncthreads();
  }
}

// Opts a kernel into more than 48 KB of dynamic shared memory, once per kernel.
template <typename F>
void set_smem(F kfn, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> done;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find((const void*)kfn);
  if (it != done.end() && it->second >= bytes) return;
  VC_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done[(const void*)kfn] = bytes;
}

template <int CAP, typename ACC>
constexpr size_t warp_smem() {
  return (size_t)kWarpsPerBlock * CAP * (sizeof(ACC) + sizeof(int)) + (size_t)kWarpsPerBlock * (CAP / 2) * sizeof(int);
}

template <typename WT, typename ACC, bool FIRST>
void launch_lp(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* lab, int32_t* lab_out,
               const unsigned long long* key, const LpTuning& tune, cudaStream_t s) {
  const WT* w = (const WT*)g.w;
  if (FIRST && g.simple) {
    const int G = tune.first_group;
    const int grid = grid_for(g.n, kAggThreads / G, kSMs * 16);
    if (G == 8)
      lp_first_simple_k<WT, 8><<<grid, kAggThreads, 0, s>>>(g.n, kBlockMaxDeg, g.off, g.adj, w, lab_out, key, g.vact);
    else if (G == 16)
      lp_first_simple_k<WT, 16><<<grid, kAggThreads, 0, s>>>(g.n, kBlockMaxDeg, g.off, g.adj, w, lab_out, key, g.vact);
    else
      lp_first_simple_k<WT, 32><<<grid, kAggThreads, 0, s>>>(g.n, kBlockMaxDeg, g.off, g.adj, w, lab_out, key, g.vact);
    count_launch();
    VC_CHECK_LAUNCH();
    if (b.h_global > 0) {
      lp_first_simple_block_k<WT><<<grid_for(b.h_global, 1, kSMs * 4), kAggThreads, 0, s>>>(
          b.global_list, b.counts + 2, g.off, g.adj, w, lab_out, key, g.vact);
      count_launch();
      VC_CHECK_LAUNCH();
    }
    return;
  }
  launch_lp_reg<WT, ACC, FIRST>(g, b, w, lab, lab_out, key, s, tune.mid_bail);
  if (b.h_block > 0) {
    const size_t smem = (size_t)kBlockCap * (sizeof(ACC) + sizeof(int));
    auto kfn = lp_block_k<WT, ACC, FIRST, false>;
    set_smem(kfn, smem);
    kfn<<<grid_for(b.h_block, 1, kSMs * 2), kAggThreads, smem, s>>>(b.block_list, b.counts + 1, g.off, g.adj, w,
                                                                   lab, lab_out, key, nullptr, nullptr, 0, g.vact);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_global > 0) {
    int grid_g = b.h_global < gt.blocks ? b.h_global : gt.blocks;
    lp_block_k<WT, ACC, FIRST, true><<<grid_g, kAggThreads, 0, s>>>(b.global_list, b.counts + 2, g.off, g.adj, w,
                                                                    lab, lab_out, key, gt.keys, gt.vals, gt.cap,
                                                                    g.vact);
    count_launch();
    VC_CHECK_LAUNCH();
  }
}

template <typename WT>
void launch_emit_reg(const GraphView& g, const Bins& b, const WT* w, const int32_t* cid, const PairOut& out,
                     int32_t* cnt, cudaStream_t s) {
  if (b.h_small > 0) {
    emit_reg_k<WT, 16, 4><<<grid_for(b.h_small, kWarpsPerBlock * 2, kSMs * 16), kAggThreads, 0, s>>>(
        b.small_list, b.counts + 4, g.off, g.adj, w, cid, out, cnt, nullptr, nullptr);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_reg > 0) {
    emit_reg_k<WT, 32, 4><<<grid_for(b.h_reg, kWarpsPerBlock, kSMs * 16), kAggThreads, 0, s>>>(
        b.reg_list, b.counts + 5, g.off, g.adj, w, cid, out, cnt, nullptr, nullptr);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_mid > 0) {
    VC_CUDA(cudaMemsetAsync(b.counts + 7, 0, sizeof(int), s));
    emit_reg_k<WT, 32, kMidMaxDeg / 32><<<grid_for(b.h_mid, kWarpsPerBlock, kSMs * 16), kAggThreads, 0, s>>>(
        b.mid_list, b.counts + 0, g.off, g.adj, w, cid, out, cnt, b.bail_list, b.counts + 7);
    emit_warp_k<WT, 32><<<grid_for(b.h_mid, kWarpsPerBlock, kSMs * 4), kAggThreads, 0, s>>>(
        b.bail_list, b.counts + 7, g.off, g.adj, w, cid, out, cnt);
    count_launch(2);
    VC_CHECK_LAUNCH();
  }
}

template <typename WT>
void launch_emit(const GraphView& g, const Bins& b, const int32_t* cid, const PairOut& out, int32_t* cnt, int G,
                 cudaStream_t s) {
  const WT* w = (const WT*)g.w;
  launch_emit_reg<WT>(g, b, w, cid, out, cnt, s);
  if (b.h_block > 0 && b.h_block <= kEmitBlockPerVertexMax) {
    // 513..4096 entries, few lists (hubs): a block per list, its warps on interleaved
    // chunks (a group walking a 4096-entry list alone would set the kernel's length)
    emit_block_k<WT><<<b.h_block, kAggThreads, 0, s>>>(b.block_list, b.counts + 1, g.off, g.adj, w, cid, out, cnt);
    count_launch();
    VC_CHECK_LAUNCH();
  } else if (b.h_block > 0) {  // many such lists: G lanes per vertex, in G-entry chunks
    const int grid = grid_for(b.h_block, kAggThreads / G, kSMs * 16);
    const int* cp = b.counts + 1;
    if (G == 8)
      emit_warp_k<WT, 8><<<grid, kAggThreads, 0, s>>>(b.block_list, cp, g.off, g.adj, w, cid, out, cnt);
    else if (G == 16)
      emit_warp_k<WT, 16><<<grid, kAggThreads, 0, s>>>(b.block_list, cp, g.off, g.adj, w, cid, out, cnt);
    else
      emit_warp_k<WT, 32><<<grid, kAggThreads, 0, s>>>(b.block_list, cp, g.off, g.adj, w, cid, out, cnt);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  if (b.h_global > 0) {
    emit_block_k<WT><<<grid_for(b.h_global, 1, kSMs * 4), kAggThreads, 0, s>>>(b.global_list, b.counts + 2, g.off,
                                                                               g.adj, w, cid, out, cnt);
    count_launch();
    VC_CHECK_LAUNCH();
  }
}

// Unit weights accumulate in 32 bits (a sum never exceeds the list length); stored
// weights accumulate in 64 bits.
void lp_round(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* lab_in,
              int32_t* lab_out, const unsigned long long* key, cudaStream_t s, const LpTuning& tune) {
  if (g.n <= 0) return;
  const bool first = lab_in == nullptr;
  if (g.unit) {
    if (first) launch_lp<UnitW, unsigned int, true>(g, b, gt, nullptr, lab_out, key, tune, s);
    else launch_lp<UnitW, unsigned int, false>(g, b, gt, lab_in, lab_out, key, tune, s);
  } else if (g.wbytes == 4) {
    if (first) launch_lp<int32_t, unsigned long long, true>(g, b, gt, nullptr, lab_out, key, tune, s);
    else launch_lp<int32_t, unsigned long long, false>(g, b, gt, lab_in, lab_out, key, tune, s);
  } else {
    if (first) launch_lp<long long, unsigned long long, true>(g, b, gt, nullptr, lab_out, key, tune, s);
    else launch_lp<long long, unsigned long long, false>(g, b, gt, lab_in, lab_out, key, tune, s);
  }
}

void emit_cross(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* cid, const PairOut& out,
                int32_t* cnt, cudaStream_t s, const LpTuning& tune) {
  (void)gt;
  if (g.n <= 0) return;
  const int G = tune.emit_group;
  if (g.unit) launch_emit<UnitW>(g, b, cid, out, cnt, G, s);
  else if (g.wbytes == 4) launch_emit<int32_t>(g, b, cid, out, cnt, G, s);
  else launch_emit<long long>(g, b, cid, out, cnt, G, s);
}

}  // namespace vc
