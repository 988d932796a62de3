// Final exact step: the minimum-cut algorithm of Nagamochi, Ono and Ibaraki (Sec. 3,
// "The Minimum Cut Algorithm of Nagamochi, Ono and Ibaraki"; used on the kernel in
// Sec. 4.1, "Final Step", and Algorithm 1).  A round is a maximum-adjacency scan
// from vertex 0 that always visits the unvisited vertex of largest attachment r
// (ties: smallest id); when x is visited every unvisited neighbour y gets
// r(y) += c(x,y) and q(x,y) = r(y) bounds the smallest x-y cut from below, so every
// edge with q >= lambda-hat (fixed for the round) is contracted.  Rounds repeat on
// the contracted graph until one vertex is left, the bound following the minimum
// degree after each contraction.
#include <limits.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>

#include "kernels.cuh"
#include "viecut.h"

namespace vc {

constexpr int kNoiThreads = 512;
constexpr int kNoiWarpMax = 32;  // kernels up to this size scan with one warp

__device__ __forceinline__ int sfind(volatile int* p, int x) {
  for (;;) {
    int px = p[x];
    if (px == x) return x;
    int ppx = p[px];
    if (ppx != px) p[x] = ppx;
    x = px;
  }
}

__device__ __forceinline__ void sunite(int* p, int a, int b) {
  for (;;) {
    a = sfind(p, a);
    b = sfind(p, b);
    if (a == b) return;
    if (a < b) { int t = a; a = b; b = t; }
    if (atomicCAS(&p[a], a, b) == a) return;
  }
}

// argmax of (r, -k) over unseen k < nk, by one warp
__device__ __forceinline__ int warp_argmax_unseen(const long long* r, const int* seen, int nk) {
  const int lane = threadIdx.x & 31;
  long long br = -1;
  int bx = INT_MAX;
  for (int k = lane; k < nk; k += 32)
    if (!seen[k]) {
      long long rv = r[k];
      if (rv > br || (rv == br && k < bx)) { br = rv; bx = k; }
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long orv = __shfl_xor_sync(0xffffffffu, br, o);
    int ox = __shfl_xor_sync(0xffffffffu, bx, o);
    if (orv > br || (orv == br && ox < bx)) { br = orv; bx = ox; }
  }
  return bx;
}

// Where one graph's exact-step results go: its bound, best-side kind, shape and
// trace (fields of DevState for single runs, per-graph arrays for batches).
struct NoiIO {
  long long* lam;
  int* best_kind;
  long long* n_out;
  long long* nnz_out;
  long long* dmin;
  long long* argmin;
  int* trace_len;
  TraceStep* trace;
  int trace_cap;
  int level;
};

// All rounds on one graph of n <= kDenseMax vertices, by one block, on a dense matrix.
// The graph's vertices are [base, base + n) of the CSR (off points at its first row).
template <typename WT>
__device__ __forceinline__ void noi_dense_body(int n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                               const WT* __restrict__ w, int32_t base, long long* M0, long long* M1,
                                               int32_t* curK, unsigned char* sideK, const NoiIO& io) {
  __shared__ long long r[kDenseMax];
  __shared__ int seen[kDenseMax];
  __shared__ int parent[kDenseMax];
  __shared__ int root[kDenseMax];
  __shared__ int rr[kDenseMax];
  __shared__ int wsum[kNoiThreads / 32];
  __shared__ long long red_d[kNoiThreads / 32];
  __shared__ int red_v[kNoiThreads / 32];
  __shared__ long long red_c[kNoiThreads / 32];
  __shared__ int s_x, s_stop, s_improved, s_nk2, s_arg, s_qt;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  constexpr int T = kNoiThreads;
  int nk = n;
  long long* M = M0;
  long long* Mn = M1;
  for (int i = tid; i < nk * nk; i += T) M[i] = 0;
  for (int k = tid; k < n; k += T) curK[k] = k;
  __syncthreads();
  for (int v = tid; v < nk; v += T)
    for (int64_t e = off[v]; e < off[v + 1]; ++e) M[v * nk + (adj[e] - base)] += (long long)w[e];
  __syncthreads();
  while (nk > 1) {
    const long long lam = *io.lam;
    for (int k = tid; k < nk; k += T) { r[k] = 0; seen[k] = 0; parent[k] = k; }
    __syncthreads();
    if (nk <= kNoiWarpMax) {
      // small kernels: warp 0 alone runs the scan (no block barrier per step)
      if (wid == 0) {
        for (int step = 0; step < nk; ++step) {
          const int x = warp_argmax_unseen(r, seen, nk);
          __syncwarp();
          if (lane == 0) seen[x] = 1;
          __syncwarp();
          const long long* row = M + (int64_t)x * nk;
          for (int y = lane; y < nk; y += 32) {
            if (!seen[y]) {
              const long long c = row[y];
              if (c != 0) {
                const long long ry = r[y] + c;
                r[y] = ry;
                if (ry >= lam) sunite(parent, x, y);
              }
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
    } else {
      // the round as closures (see noi_closure_warp below): each run's first vertex is the
      // untaken vertex of largest r (ties: smallest id); the run then grows level by
      // level, every thread relaxing matrix entries of the level's vertices, and takes
      // its smallest id as the label of all its vertices (rr holds the taken vertices)
      int qt = 0, qh = 0;
      while (qt < nk) {
        if (wid == 0) {
          const int x = warp_argmax_unseen(r, seen, nk);
          if (lane == 0) {
            rr[qt] = x;
            seen[x] = 1;
            s_qt = qt + 1;
          }
        }
        __syncthreads();
        const int rs = qt;
        qt = s_qt;
        while (qh < qt) {
          const int F = qt - qh;
          for (int idx = tid; idx < F * nk; idx += T) {
            const int f = idx / nk, y = idx - f * nk;
            if (seen[y]) continue;
            const long long c = M[(int64_t)rr[qh + f] * nk + y];
            if (c == 0) continue;
            const long long ry = (long long)atomicAdd((unsigned long long*)&r[y], (unsigned long long)c) + c;
            if (ry >= lam && (ry - c < lam || ry - c <= 0) && atomicExch(&seen[y], 1) == 0)
              rr[atomicAdd(&s_qt, 1)] = y;
          }
          __syncthreads();
          qh = qt;
          qt = s_qt;
          __syncthreads();  // every thread has read s_qt before the next level adds to it
        }
        int m = INT_MAX;
        for (int i = rs + tid; i < qt; i += T) m = rr[i] < m ? rr[i] : m;
        m = (int)__reduce_min_sync(0xffffffffu, (unsigned)m);
        if (lane == 0) red_v[wid] = m;
        __syncthreads();
        if (tid == 0) {
          for (int q = 1; q < T / 32; ++q) m = red_v[q] < m ? red_v[q] : m;
          s_arg = m;
        }
        __syncthreads();
        m = s_arg;
        for (int i = rs + tid; i < qt; i += T) root[rr[i]] = m;
        __syncthreads();
      }
    }
    if (nk <= kNoiWarpMax) {
      for (int k = tid; k < nk; k += T) root[k] = sfind(parent, k);
      __syncthreads();
    }
    // roots -> ranks (every root is the minimum of its component)
    {
      int flag = (tid < nk && root[tid] == tid) ? 1 : 0;  // nk <= T
      int inc = flag;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) wsum[wid] = inc;
      __syncthreads();
      if (tid == 0) {
        int acc = 0;
        for (int q = 0; q < T / 32; ++q) { int t = wsum[q]; wsum[q] = acc; acc += t; }
        s_nk2 = acc;
      }
      __syncthreads();
      if (tid < nk) rr[tid] = wsum[wid] + inc - flag;
      __syncthreads();
    }
    const int nk2 = s_nk2;
    if (nk2 == nk) break;  // no contraction (cannot happen while lambda-hat <= min degree)
    for (int i = tid; i < nk2 * nk2; i += T) Mn[i] = 0;
    __syncthreads();
    for (int i = tid; i < nk * nk; i += T) {
      long long c = M[i];
      if (c != 0) {
        int a = rr[root[i / nk]], b = rr[root[i % nk]];
        if (a != b) atomicAdd((unsigned long long*)&Mn[a * nk2 + b], (unsigned long long)c);
      }
    }
    for (int k = tid; k < n; k += T) curK[k] = rr[root[curK[k]]];
    __syncthreads();
    { long long* t = M; M = Mn; Mn = t; }
    nk = nk2;
    // degrees, minimum with smallest argmin, and entry count of the contracted graph
    long long bd = LLONG_MAX, cnt = 0;
    int bv = INT_MAX;
    for (int a = tid; a < nk; a += T) {
      long long d = 0;
      const long long* row = M + (int64_t)a * nk;
      for (int b = 0; b < nk; ++b) {
        long long c = row[b];
        d += c;
        cnt += c != 0;
      }
      if (d < bd || (d == bd && a < bv)) { bd = d; bv = a; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long od = __shfl_xor_sync(0xffffffffu, bd, o);
      int ov = __shfl_xor_sync(0xffffffffu, bv, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (od < bd || (od == bd && ov < bv)) { bd = od; bv = ov; }
    }
    if (lane == 0) { red_d[wid] = bd; red_v[wid] = bv; red_c[wid] = cnt; }
    __syncthreads();
    if (tid == 0) {
      long long tot = 0;
      for (int q = 0; q < T / 32; ++q) {
        tot += red_c[q];
        if (red_d[q] < bd || (red_d[q] == bd && red_v[q] < bv)) { bd = red_d[q]; bv = red_v[q]; }
      }
      s_stop = 0;
      s_improved = 0;
      *io.n_out = nk;
      *io.nnz_out = tot;
      if (nk > 1) {
        *io.dmin = bd;
        *io.argmin = bv;
        if (bd < *io.lam) {
          *io.lam = bd;
          *io.best_kind = 2;
          s_improved = 1;
          s_arg = bv;
        }
        if (*io.lam == 0) s_stop = 1;
      }
      int i = *io.trace_len;
      if (i < io.trace_cap) io.trace[i] = TraceStep{4, io.level, (long long)nk, tot, *io.lam};
      *io.trace_len = i + 1;
    }
    __syncthreads();
    if (s_improved) {
      const int b = s_arg;
      for (int k = tid; k < n; k += T) sideK[k] = curK[k] == b ? 1 : 0;
    }
    __syncthreads();
    if (s_stop) break;
  }
}

template <typename WT>
__global__ void __launch_bounds__(kNoiThreads) noi_dense_k(int n, const int64_t* __restrict__ off,
                                                           const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                           long long* M0, long long* M1, int32_t* curK,
                                                           unsigned char* sideK, DevState* st, TraceStep* trace,
                                                           int trace_cap, int level, int in_smem) {
  // small kernels keep the first round's matrix in shared memory (a round reads one
  // matrix row per scan step; shared memory answers in a few cycles); later rounds
  // are smaller and alternate between it and the global one
  extern __shared__ __align__(16) long long noi_dyn[];
  if (in_smem) M0 = noi_dyn;
  NoiIO io{&st->lambda_hat, &st->best_kind, &st->n, &st->nnz, &st->dmin, &st->argmin, &st->trace_len,
           trace, trace_cap, level};
  noi_dense_body<WT>(n, off, adj, w, 0, M0, M1, curK, sideK, io);
}

constexpr int kNoiSmemMaxN = 160;  // 160^2 x 8 B = 200 KiB of shared memory

template <typename WT>
static void noi_dense_launch(const GraphView& g, long long* M0, long long* M1, int32_t* curK, unsigned char* sideK,
                             DevState* st, TraceStep* trace, int trace_cap, int level, cudaStream_t s) {
  static std::mutex mu;
  static std::unordered_map<int, bool> ready;  // per device: the shared-memory limit was raised
  const int n = (int)g.n;
  const bool small = n <= kNoiSmemMaxN;
  const size_t smem = small ? sizeof(long long) * (size_t)n * n : 0;
  if (small) {
    int dev = 0;
    VC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
      VC_CUDA(cudaFuncSetAttribute(noi_dense_k<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(long long) * kNoiSmemMaxN * kNoiSmemMaxN)));
      ready[dev] = true;
    }
  }
  noi_dense_k<WT><<<1, kNoiThreads, smem, s>>>(n, g.off, g.adj, (const WT*)g.w, M0, M1, curK, sideK, st, trace,
                                               trace_cap, level, small ? 1 : 0);
  count_launch();
  VC_CHECK_LAUNCH();
}

void noi_dense(const GraphView& g, long long* M0, long long* M1, int32_t* curK, unsigned char* sideK,
               DevState* st, TraceStep* trace, int trace_cap, int level, cudaStream_t s) {
  if (g.wbytes == 4) noi_dense_launch<int32_t>(g, M0, M1, curK, sideK, st, trace, trace_cap, level, s);
  else noi_dense_launch<long long>(g, M0, M1, curK, sideK, st, trace, trace_cap, level, s);
}

// Batches: a persistent grid pulls the listed graphs; each block solves one at a time
// with its own matrices (mcap entries each).
template <typename WT>
__global__ void __launch_bounds__(kNoiThreads) noi_dense_batch_k(const int32_t* __restrict__ list, int count,
                                                                 const int64_t* __restrict__ off,
                                                                 const int32_t* __restrict__ adj,
                                                                 const WT* __restrict__ w, const long long* vbase,
                                                                 const long long* nv, long long* M, int64_t mcap,
                                                                 int32_t* curK, unsigned char* sideK, BatchNoi bn) {
  long long* M0 = M + (int64_t)blockIdx.x * 2 * mcap;
  long long* M1 = M0 + mcap;
  int32_t* ck = curK + (int64_t)blockIdx.x * kDenseMax;
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int g = list[idx];
    const int32_t base = (int32_t)vbase[g];
    NoiIO io{bn.lam + g, bn.best_kind + g, bn.n_out + g, bn.nnz_out + g, bn.dmin + g, bn.argmin + g,
             bn.trace_len + g, bn.trace + (int64_t)g * bn.trace_cap, bn.trace_cap, bn.level[g]};
    noi_dense_body<WT>((int)nv[g], off + base, adj, w, base, M0, M1, ck, sideK + (int64_t)g * kDenseMax, io);
    __syncthreads();
  }
}

void noi_dense_batch(const GraphView& u, const int32_t* list, int count, const long long* vbase, const long long* nv,
                     long long* M, int64_t mcap, int blocks, int32_t* curK, unsigned char* sideK, const BatchNoi& bn,
                     cudaStream_t s) {
  if (count <= 0) return;
  if (u.wbytes == 4)
    noi_dense_batch_k<int32_t><<<blocks, kNoiThreads, 0, s>>>(list, count, u.off, u.adj, (const int32_t*)u.w, vbase,
                                                               nv, M, mcap, curK, sideK, bn);
  else
    noi_dense_batch_k<long long><<<blocks, kNoiThreads, 0, s>>>(list, count, u.off, u.adj, (const long long*)u.w,
                                                                 vbase, nv, M, mcap, curK, sideK, bn);
  count_launch();
  VC_CHECK_LAUNCH();
}

// ------------------------------------------------------------ sparse single round
constexpr int kSparseThreads = 1024;

// One round on the vertices [lo, hi) (ids are global: r, seen, parent, labels are
// indexed by them); returns through *any whether something merged.
template <typename WT>
__device__ __forceinline__ void noi_round_body(int64_t lo, int64_t hi, const int64_t* __restrict__ off,
                                               const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                               long long lam, long long* r, unsigned char* seen, int32_t* parent,
                                               int32_t* labels, int* any_out) {
  __shared__ long long red_r[kSparseThreads / 32];
  __shared__ long long red_x[kSparseThreads / 32];
  __shared__ long long s_x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int64_t k = lo + tid; k < hi; k += kSparseThreads) { r[k] = 0; seen[k] = 0; parent[k] = (int32_t)k; }
  __syncthreads();
  for (int64_t step = lo; step < hi; ++step) {
    long long br = -1, bx = LLONG_MAX;
    for (int64_t k = lo + tid; k < hi; k += kSparseThreads)
      if (!seen[k]) {
        long long rv = r[k];
        if (rv > br || (rv == br && k < bx)) { br = rv; bx = k; }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long orv = __shfl_xor_sync(0xffffffffu, br, o);
      long long ox = __shfl_xor_sync(0xffffffffu, bx, o);
      if (orv > br || (orv == br && ox < bx)) { br = orv; bx = ox; }
    }
    if (lane == 0) { red_r[wid] = br; red_x[wid] = bx; }
    __syncthreads();
    if (tid == 0) {
      for (int q = 1; q < kSparseThreads / 32; ++q)
        if (red_r[q] > br || (red_r[q] == br && red_x[q] < bx)) { br = red_r[q]; bx = red_x[q]; }
      s_x = bx;
      seen[bx] = 1;
    }
    __syncthreads();
    const int64_t x = s_x;
    for (int64_t e = off[x] + tid; e < off[x + 1]; e += kSparseThreads) {
      const int y = adj[e];
      if (seen[y]) continue;
      const long long c = (long long)w[e];
      const long long ry = (long long)atomicAdd((unsigned long long*)&r[y], (unsigned long long)c) + c;
      if (ry >= lam) sunite(parent, (int)x, y);
    }
    __syncthreads();
  }
  int any = 0;
  for (int64_t k = lo + tid; k < hi; k += kSparseThreads) {
    int rt = sfind(parent, (int)k);
    labels[k] = rt;
    any |= rt != k;
  }
  if (__syncthreads_or(any) && tid == 0) atomicOr(any_out, 1);
  __syncthreads();
}

// ---- the same round by one warp, as closures.  Call a vertex "low" when it is visited
// with attachment r < max(lambda-hat, 1).  When a low vertex u is visited every
// unvisited r is at most r(u), so no unvisited vertex has reached lambda-hat; the
// vertices visited after u up to the next low vertex are then exactly the closure of
// u: the smallest set R holding u such that every vertex outside R and outside the
// earlier runs has fewer than lambda-hat of weight into the vertices visited so far.
// Adding a vertex only raises the weights into the set, so the closure does not depend
// on the order in which its vertices are added, and neither do the attachments of the
// vertices left afterwards; the next low vertex (the largest r, ties to the smallest
// id) is therefore the same as in the maximum-adjacency order.  The round unites every
// x, y with r(y) >= lambda-hat once x's edge is added; each such pair lies within one
// run, and every vertex of a run is joined to the vertex whose edge raised it to
// lambda-hat (visited inside the run), so the round's components are the runs and the
// union-find with smallest-id roots labels each run with its smallest id.
//
// So a round needs the exact order only to pick each run's first vertex (an argmax
// over the vertices not yet taken); a run then grows level by level, the warp relaxing
// up to 32 queued vertices at once: their lists are laid end to end over the lanes, a
// vertex whose attachment reaches lambda-hat joins the queue, and the run's labels are
// written when it stops growing.  queue (n entries from lo) holds the vertices in the
// order they were taken.

// argmax over the warp of (val, -idx) for val >= 0 (val < 0: no candidate); returns
// idx, or -1 if no lane has a candidate; *best = the value.
__device__ __forceinline__ int warp_argmax_vi(long long val, int idx, long long* best) {
  const unsigned long long u = (unsigned long long)(val + 1);  // 0 = none
  const unsigned hi = (unsigned)(u >> 32), lo = (unsigned)u;
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
  const unsigned long long mu = ((unsigned long long)mh << 32) | ml;
  const unsigned wi = __reduce_min_sync(0xffffffffu, (u == mu && u != 0) ? (unsigned)idx : 0xffffffffu);
  *best = (long long)mu - 1;
  return mu == 0 ? -1 : (int)wi;
}

// Taken flags of a round: an int per vertex at v - sb (global memory, where graphs of a
// union sit side by side), or a bit per vertex of the graph [lo, lo + n) in words the
// warp owns (shared memory).  claim(v) takes v and returns whether it was not taken
// yet: a vertex joins a queue at most once, whatever the weights.
struct WordSeen {
  int* p;
  int64_t sb;
  __device__ __forceinline__ void clear(int64_t lo, int64_t n, int lane) const {
    for (int64_t k = lane; k < n; k += 32) p[lo + k - sb] = 0;
  }
  __device__ __forceinline__ bool test(int64_t v) const { return ((volatile int*)p)[v - sb] != 0; }
  __device__ __forceinline__ bool claim(int64_t v) const { return atomicExch(&p[v - sb], 1) == 0; }
};
struct BitSeen {
  unsigned* bits;
  int64_t lo;
  __device__ __forceinline__ void clear(int64_t, int64_t n, int lane) const {
    for (int64_t k = lane; k < ((n + 31) >> 5); k += 32) bits[k] = 0;
  }
  __device__ __forceinline__ bool test(int64_t v) const {
    return (((volatile unsigned*)bits)[(v - lo) >> 5] >> ((v - lo) & 31)) & 1u;
  }
  __device__ __forceinline__ bool claim(int64_t v) const {
    const unsigned bit = 1u << ((v - lo) & 31);
    return (atomicOr(&bits[(v - lo) >> 5], bit) & bit) == 0u;
  }
};

constexpr int kNoiUnroll = 4;  // list entries in flight per lane while relaxing

// One round over the graph [lo, lo + n) (ids global: labels, queue and the lists use
// them); r holds vertex v at v - sb, queue the n taken vertices from lo (at q - qb for
// place q: qb = 0 for a queue over the whole id range, lo for the graph's own array).
// Writes every vertex's label; returns, in every lane, whether some run holds two or
// more vertices (the round unites).
template <typename WT, typename SEEN>
__device__ __forceinline__ bool noi_closure_warp(int64_t lo, int64_t n, const int64_t* __restrict__ off,
                                                 const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                 long long lam, long long* r, int64_t sb, SEEN seen,
                                                 long long* cmax, int32_t* queue, int64_t qb, int32_t* labels) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  const int64_t nc = (n + 31) >> 5;
  for (int64_t k = lane; k < n; k += 32) r[lo + k - sb] = 0;
  for (int64_t c = lane; c < nc; c += 32) cmax[c] = 0;
  seen.clear(lo, n, lane);
  __syncwarp();
  int32_t* q = queue + (lo - qb);  // q[i]: the i-th taken vertex
  int64_t qt = 0, qh = 0;          // taken / relaxed so far (the same in every lane)
  bool unites = false;
  while (qt < n) {
    // the run's first vertex: the untaken vertex of largest r, ties to the smallest id.
    // cmax[c] bounds the attachments of chunk c's untaken vertices from above (raised
    // with every relaxation; a taken vertex may leave it stale): the chunk of largest
    // bound (ties: lower chunk) is checked exactly, and a stale bound is lowered and the
    // choice made again.  A bound that holds is the largest attachment left.
    int u;
    for (;;) {
      long long bv = -1;
      int bc = -1;
      for (int64_t c = lane; c < nc; c += 32) {
        const long long m = cmax[c];
        if (m > bv) { bv = m; bc = (int)c; }
      }
      long long bound, best;
      const int C = warp_argmax_vi(bv, bc, &bound);
      const int64_t k = (int64_t)C * 32 + lane;
      const long long rv = (k < n && !seen.test(lo + k)) ? r[lo + k - sb] : -1;
      const int xl = warp_argmax_vi(rv, (int)k, &best);
      if (best == bound) {
        u = xl;
        break;
      }
      if (lane == 0) cmax[C] = best;  // -1: every vertex of the chunk is taken
      __syncwarp();
    }
    const int64_t rs = qt;
    int32_t runmin = (int32_t)(lo + u);
    if (lane == 0) {
      q[qt] = runmin;
      seen.claim(lo + u);
    }
    ++qt;
    __syncwarp();
    while (qh < qt) {
      // up to 32 taken vertices at once, their lists end to end over the lanes
      const int cnt = (int)(qt - qh < 32 ? qt - qh : 32);
      int64_t fb = 0, deg = 0;
      if (lane < cnt) {
        const int32_t x = q[qh + lane];
        fb = __ldg(off + x);
        deg = __ldg(off + x + 1) - fb;
      }
      qh += cnt;
      int64_t incl = deg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
      const int64_t excl = incl - deg;  // where lane j's list starts in the laid-out lists
      for (int64_t p0 = 0; p0 < total; p0 += 32 * kNoiUnroll) {
        int32_t y[kNoiUnroll];
        long long c[kNoiUnroll];
#pragma unroll
        for (int i = 0; i < kNoiUnroll; ++i) {
          const int64_t p = p0 + lane + 32 * i;
          // the list holding place p: the last lane j whose list starts at or before p
          int j = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int t = j + step;
            const int64_t ex = __shfl_sync(0xffffffffu, excl, t & 31);
            if (t < cnt && ex <= p) j = t;
          }
          const int64_t e = __shfl_sync(0xffffffffu, fb, j) + (p - __shfl_sync(0xffffffffu, excl, j));
          y[i] = -1;
          c[i] = 0;
          if (p < total) {
            y[i] = __ldg(adj + e);
            c[i] = (long long)__ldg(w + e);
          }
        }
#pragma unroll
        for (int i = 0; i < kNoiUnroll; ++i) {
          bool join = false;
          if (y[i] >= 0 && !seen.test(y[i])) {
            const long long ry =
                (long long)atomicAdd((unsigned long long*)&r[y[i] - sb], (unsigned long long)c[i]) + c[i];
            atomicMax(&cmax[(y[i] - lo) >> 5], ry);
            // the addition that first leaves r(y) >= lambda-hat: the one that crosses it,
            // or (lambda-hat <= 0) the first one
            join = ry >= lam && (ry - c[i] < lam || ry - c[i] <= 0);
          }
          join = join && seen.claim(y[i]);
          const unsigned b = __ballot_sync(0xffffffffu, join);
          if (join) q[qt + __popc(b & below)] = y[i];
          qt += __popc(b);
          const unsigned m = __reduce_min_sync(0xffffffffu, join ? (unsigned)y[i] : 0xffffffffu);
          if (m != 0xffffffffu && (int32_t)m < runmin) runmin = (int32_t)m;
          __syncwarp();
        }
      }
    }
    for (int64_t i = rs + lane; i < qt; i += 32) labels[q[i]] = runmin;
    if (qt - rs > 1) unites = true;
    __syncwarp();
  }
  return unites;
}

// The round with the graph's state (attachments, taken flags and queue) in shared
// memory.  One warp per block.
constexpr int kNoiSmemRoundMaxN = 16384;  // 16384 x 12.375 B < 227 KB
__host__ __device__ constexpr size_t noi_round_smem(int ncap) {
  return (size_t)ncap * 12 + ((size_t)ncap / 32 + 1) * 12 + 16;
}

template <typename WT>
__global__ void __launch_bounds__(32) noi_round_smem_k(int64_t n, const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                       const DevState* st, int32_t* labels, int* changed) {
  extern __shared__ __align__(16) unsigned char noi_rs[];
  long long* r = (long long*)noi_rs;
  long long* cmax = r + n;
  int32_t* queue = (int32_t*)(cmax + n / 32 + 1);
  unsigned* seen = (unsigned*)(queue + n);
  const bool any =
      noi_closure_warp<WT>(0, n, off, adj, w, st->lambda_hat, r, 0, BitSeen{seen, 0}, cmax, queue, 0, labels);
  if (any && threadIdx.x == 0) atomicOr(changed, 1);
}

// Above the shared-memory size: the same round on global arrays.
template <typename WT>
__global__ void __launch_bounds__(32) noi_round_k(int64_t n, const int64_t* __restrict__ off,
                                                  const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                  const DevState* st, long long* r, int* seen,
                                                  int32_t* queue, int32_t* labels, int* changed) {
  // r holds n attachments, then the chunk bounds
  const bool any =
      noi_closure_warp<WT>(0, n, off, adj, w, st->lambda_hat, r, 0, WordSeen{seen, 0}, r + n, queue, 0, labels);
  if (any && threadIdx.x == 0) atomicOr(changed, 1);
}

template <typename WT>
static void noi_round_launch(const GraphView& g, const DevState* st, long long* r, int* seen,
                             int32_t* queue, int32_t* labels, int* changed, cudaStream_t s) {
  if (g.n <= kNoiSmemRoundMaxN) {
    static std::mutex mu;
    static std::unordered_map<int, bool> ready;  // per device: the shared-memory limit was raised
    {
      int dev = 0;
      VC_CUDA(cudaGetDevice(&dev));
      std::lock_guard<std::mutex> lk(mu);
      if (!ready[dev]) {
        VC_CUDA(cudaFuncSetAttribute(noi_round_smem_k<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)noi_round_smem(kNoiSmemRoundMaxN)));
        ready[dev] = true;
      }
    }
    noi_round_smem_k<WT><<<1, 32, noi_round_smem((int)g.n), s>>>(g.n, g.off, g.adj, (const WT*)g.w, st, labels,
                                                                 changed);
  } else {
    noi_round_k<WT><<<1, 32, 0, s>>>(g.n, g.off, g.adj, (const WT*)g.w, st, r, seen, queue, labels, changed);
  }
  count_launch();
  VC_CHECK_LAUNCH();
}

void noi_round_sparse(const GraphView& g, const DevState* st, long long* r, int* seen,
                      int32_t* parent, int32_t* labels, int* changed, cudaStream_t s) {
  // parent (n entries) holds the queue of taken vertices
  if (g.wbytes == 4)
    noi_round_launch<int32_t>(g, st, r, seen, parent, labels, changed, s);
  else
    noi_round_launch<long long>(g, st, r, seen, parent, labels, changed, s);
}

// Batches: the round of each listed graph by a warp (persistent grid of 8-warp blocks
// pulling graphs from the list).  With ncap > 0 (every listed graph of at most ncap
// vertices) each warp keeps its graph's taken bits in shared memory; the attachments
// and queues stay in global memory (every graph of the list in flight at once).
__host__ __device__ constexpr size_t noi_batch_warp_smem(int ncap) { return (size_t)(ncap / 32 + 1) * 12; }
constexpr size_t kNoiBatchSmemMax = 160 * 1024;

template <typename WT>
__global__ void __launch_bounds__(256) noi_round_batch_k(const int32_t* __restrict__ list, int count,
                                                         const int64_t* __restrict__ off,
                                                         const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                         const long long* vbase, const long long* nv,
                                                         const long long* glam, long long* r, int* seen,
                                                         long long* cmax, int32_t* queue, int32_t* labels,
                                                         int* gchanged, int ncap) {
  extern __shared__ __align__(16) unsigned char noi_bs[];
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int words = ncap / 32 + 1;
  long long* wc = (long long*)noi_bs + (size_t)wid * words;
  unsigned* wb = (unsigned*)((long long*)noi_bs + (size_t)(blockDim.x >> 5) * words) + (size_t)wid * words;
  for (int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < count; idx += warps) {
    const int g = list[idx];
    const long long lo = vbase[g], n = nv[g];
    bool any;
    if (ncap > 0 && n <= ncap)
      any = noi_closure_warp<WT>(lo, n, off, adj, w, glam[g], r, 0, BitSeen{wb, lo}, wc, queue, 0, labels);
    else
      any = noi_closure_warp<WT>(lo, n, off, adj, w, glam[g], r, 0, WordSeen{seen, 0}, cmax + lo, queue, 0, labels);
    if (any && lane == 0) atomicOr(gchanged + g, 1);
    __syncwarp();
  }
}

template <typename WT>
static void noi_round_batch_launch(const GraphView& u, const int32_t* list, int count, const long long* vbase,
                                   const long long* nv, const long long* glam, long long* r, int* seen,
                                   long long* cmax, int32_t* queue, int32_t* labels, int* gchanged, int max_n,
                                   cudaStream_t s) {
  static std::mutex mu;
  static std::unordered_map<int, bool> ready;  // per device: the shared-memory limit was raised
  {
    int dev = 0;
    VC_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (!ready[dev]) {
      VC_CUDA(cudaFuncSetAttribute(noi_round_batch_k<WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kNoiBatchSmemMax));
      ready[dev] = true;
    }
  }
  const size_t smem = 8 * noi_batch_warp_smem(max_n);
  const bool in_smem = max_n > 0 && smem <= kNoiBatchSmemMax;
  const int blocks = grid_for(count, 8, kSMs * 4);
  noi_round_batch_k<WT><<<blocks, 256, in_smem ? smem : 0, s>>>(list, count, u.off, u.adj, (const WT*)u.w, vbase, nv,
                                                               glam, r, seen, cmax, queue, labels, gchanged,
                                                               in_smem ? max_n : 0);
  count_launch();
  VC_CHECK_LAUNCH();
}

void noi_round_batch(const GraphView& u, const int32_t* list, int count, const long long* vbase, const long long* nv,
                     const long long* glam, long long* r, int* seen, int32_t* parent, int32_t* labels,
                     int* gchanged, int max_n, cudaStream_t s) {
  if (count <= 0) return;
  // r holds noi_round_scratch(union size) entries: the attachments, then each graph's
  // chunk bounds at its own range; seen: the taken flags (union size); parent (union
  // size) holds the queues
  long long* cmax = r + u.n;
  if (u.wbytes == 4)
    noi_round_batch_launch<int32_t>(u, list, count, vbase, nv, glam, r, seen, cmax, parent, labels, gchanged, max_n,
                                    s);
  else
    noi_round_batch_launch<long long>(u, list, count, vbase, nv, glam, r, seen, cmax, parent, labels, gchanged, max_n,
                                      s);
}

// ------------------------------------------------------- allocation-free round
// Scratch of viecut_noi_round_noalloc: r (int64), parent (int32) and seen (byte) for
// at most kNoAllocMaxN vertices, in one array that every device loading the library
// keeps until the process exits (about 0.8 MB).  Host code must not pass the array's
// name to a kernel: on the host it is only a stand-in; its device address comes from
// cudaGetSymbolAddress, looked up once per device.
constexpr int64_t kNoAllocMaxN = 1 << 16;
constexpr size_t kNoAllocBytes = (size_t)kNoAllocMaxN * (sizeof(long long) + sizeof(int32_t) + 1);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__global__ void __launch_bounds__(kSparseThreads) noi_round_noalloc_k(int64_t n, const int64_t* __restrict__ off,
                                                                      const int32_t* __restrict__ adj,
                                                                      const long long* __restrict__ w, long long lam,
                                                                      unsigned char* scratch, int32_t* labels,
                                                                      int32_t* changed) {
  long long* r = (long long*)scratch;
  int32_t* parent = (int32_t*)(scratch + (size_t)kNoAllocMaxN * sizeof(long long));
  unsigned char* seen = scratch + (size_t)kNoAllocMaxN * (sizeof(long long) + sizeof(int32_t));
  if (threadIdx.x == 0) *changed = 0;
  __syncthreads();
  // the body clears r, seen and parent for [0, n) before using them
  noi_round_body<long long>(0, n, off, adj, w, lam, r, seen, parent, labels, changed);
}

static unsigned char* noalloc_scratch_address() {
  static std::mutex mu;
  static unsigned char* addr[256] = {nullptr};
  int dev = 0;
  VC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) throw Error{VIECUT_EINVAL, "device ordinal out of range"};
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    VC_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    addr[dev] = (unsigned char*)p;
  }
  return addr[dev];
}

void set_last_error(const std::string& msg);

}  // namespace vc

extern "C" int viecut_noi_round_noalloc(const int64_t* d_offsets, const int32_t* d_adj, const int64_t* d_weights,
                                        int64_t n, int64_t lambda_hat, int32_t* d_labels, int32_t* d_changed,
                                        void* stream) {
  try {
    if (n < 1 || n > vc::kNoAllocMaxN)
      throw vc::Error{VIECUT_EINVAL, "viecut_noi_round_noalloc: n = " + std::to_string(n) + " is outside [1, " +
                                         std::to_string(vc::kNoAllocMaxN) + "], the size of its static scratch"};
    // the host cannot see offsets[n], so a graph with edges cannot be told apart from an
    // edgeless one here: every array must be given
    if (!d_offsets || !d_adj || !d_weights || !d_labels || !d_changed)
      throw vc::Error{VIECUT_EINVAL, "viecut_noi_round_noalloc: null device pointer"};
    if (lambda_hat < 0) throw vc::Error{VIECUT_EINVAL, "lambda_hat must be >= 0"};
    unsigned char* scratch = vc::noalloc_scratch_address();
    vc::noi_round_noalloc_k<<<1, vc::kSparseThreads, 0, (cudaStream_t)stream>>>(
        n, d_offsets, d_adj, (const long long*)d_weights, lambda_hat, scratch, d_labels, d_changed);
    vc::count_launch();
    VC_CHECK_LAUNCH();
  } catch (const vc::Error& e) {
    vc::set_last_error(e.msg);
    return e.code;
  }
  return VIECUT_OK;
}
