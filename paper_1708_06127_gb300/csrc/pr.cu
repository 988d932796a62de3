// Padberg-Rinaldi reductions (Lemma "Padberg-Rinaldi", Sec. 4.1) with lock-free
// union-find.  Pass A tests conditions 1 and 2, pass B conditions 3 and 4, as the
// two passes of one "run" (Sec. 4.1, "Exact Reductions by Padberg and Rinaldi").
// Condition 2 marks only the edge to the designated partner p(v) = argmax over
// neighbours of (c(v,u), -u), and conditions 3/4 are checked on mutual partner
// pairs; the union of the marked edges is contracted in one step.
#include <limits.h>

#include "kernels.cuh"

namespace vc {

// Union-find whose representative is the smallest id of the component: a root is
// only ever linked below a smaller root (CAS on a root's own entry), so the final
// root of a component is its minimum.  Path halving writes only ancestors.
__device__ __forceinline__ int uf_find(volatile int32_t* p, int x) {
  for (;;) {
    int px = p[x];
    if (px == x) return x;
    int ppx = p[px];
    if (ppx != px) p[x] = ppx;
    x = px;
  }
}

__device__ __forceinline__ void uf_unite(int32_t* p, int a, int b) {
  for (;;) {
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (a < b) { int t = a; a = b; b = t; }
    if (atomicCAS(&p[a], a, b) == a) return;
  }
}

// A warp per vertex (kPartnerG lanes; 16, two vertices per warp, measured slower on
// the long lists of deep Padberg-Rinaldi levels); lists of more than kPartnerBlockMin
// entries (hubs that absorbed many vertices) take a block each in partners_long_k.
constexpr int kPartnerG = 32;
constexpr int64_t kPartnerBlockMin = 8192;

// Degree and designated partner of one list, folded into (s, bw, bu) (bu INT_MAX: none).
__device__ __forceinline__ void partner_fold(long long& s, long long& bw, int& bu, long long x, int u) {
  s += x;
  if (x > bw || (x == bw && u < bu)) { bw = x; bu = u; }
}

template <typename WT>
__global__ void partners_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const WT* __restrict__ w, int32_t* __restrict__ partner, long long* __restrict__ pw,
                           long long* __restrict__ deg) {
  constexpr int G = kPartnerG;
  const int lane = threadIdx.x & 31, glane = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << (G & 31)) - 1u) << (lane & ~(G - 1));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += groups) {
    const int64_t beg = off[v], end = off[v + 1];
    if (end - beg > kPartnerBlockMin) continue;  // partners_long_k
    long long s = 0, bw = -1;
    int bu = INT_MAX;
    for (int64_t e = beg + glane; e < end; e += G) partner_fold(s, bw, bu, (long long)w[e], adj[e]);
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const long long os = __shfl_xor_sync(gmask, s, o);
      const long long ow = __shfl_xor_sync(gmask, bw, o);
      const int ou = __shfl_xor_sync(gmask, bu, o);
      s += os;
      if (ow > bw || (ow == bw && ou < bu)) { bw = ow; bu = ou; }
    }
    if (glane == 0) {
      deg[v] = s;
      partner[v] = bw < 0 ? -1 : bu;
      pw[v] = bw;
    }
  }
}

// The lists of more than kPartnerBlockMin entries: each block lists the long ones among
// 256 consecutive vertices, then folds each of them with all its threads.
template <typename WT>
__global__ void __launch_bounds__(256) partners_long_k(int64_t n, const int64_t* __restrict__ off,
                                                       const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                                       int32_t* __restrict__ partner, long long* __restrict__ pw,
                                                       long long* __restrict__ deg) {
  __shared__ int32_t s_list[256];
  __shared__ int s_n;
  __shared__ long long s_s[8], s_bw[8];
  __shared__ int s_bu[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += (int64_t)gridDim.x * 256) {
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    const int64_t v0 = base + threadIdx.x;
    if (v0 < n && off[v0 + 1] - off[v0] > kPartnerBlockMin) s_list[atomicAdd(&s_n, 1)] = (int32_t)v0;
    __syncthreads();
    const int cnt = s_n;
    for (int i = 0; i < cnt; ++i) {
      const int32_t v = s_list[i];
      long long s = 0, bw = -1;
      int bu = INT_MAX;
      for (int64_t e = off[v] + threadIdx.x; e < off[v + 1]; e += 256) partner_fold(s, bw, bu, (long long)w[e], adj[e]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long os = __shfl_xor_sync(0xffffffffu, s, o);
        const long long ow = __shfl_xor_sync(0xffffffffu, bw, o);
        const int ou = __shfl_xor_sync(0xffffffffu, bu, o);
        s += os;
        if (ow > bw || (ow == bw && ou < bu)) { bw = ow; bu = ou; }
      }
      if (lane == 0) { s_s[wid] = s; s_bw[wid] = bw; s_bu[wid] = bu; }
      __syncthreads();
      if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) {
          s += s_s[k];
          if (s_bw[k] > bw || (s_bw[k] == bw && s_bu[k] < bu)) { bw = s_bw[k]; bu = s_bu[k]; }
        }
        deg[v] = s;
        partner[v] = bw < 0 ? -1 : bu;
        pw[v] = bw;
      }
      __syncthreads();
    }
  }
}

void pr_partners(const GraphView& g, int32_t* partner, long long* pw, long long* deg, cudaStream_t s) {
  const int grid = grid_for(g.n, 256 / kPartnerG, kSMs * 16), gl = grid_for(g.n, 256, kSMs * 4);
  if (g.wbytes == 4) {
    partners_k<int32_t><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, partner, pw, deg);
    partners_long_k<int32_t><<<gl, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, partner, pw, deg);
  } else {
    partners_k<long long><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, partner, pw, deg);
    partners_long_k<long long><<<gl, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, partner, pw, deg);
  }
  count_launch(2);
  VC_CHECK_LAUNCH();
}

__global__ void uf_init_k(int32_t* __restrict__ p, int64_t n) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    p[v] = (int32_t)v;
}

// Bound and activity of the graph vertex v belongs to (single graph: the run's bound).
__device__ __forceinline__ bool pr_graph(const BatchCtx& bc, const DevState* st, int64_t v, long long* lam) {
  if (!bc.gid) {
    *lam = st->lambda_hat;
    return true;
  }
  const int g = bc.gid[v];
  if (!bc.gact[g]) return false;
  *lam = bc.glam[g];
  return true;
}

// Condition 1 on every edge (once per undirected edge: u > v) and condition 2 on the
// designated-partner edge; both ends must have at least two distinct neighbours.
// Union-find finds are chains of dependent loads, so short lists take a thread each
// (all of them in flight at once) and only lists longer than kPrThreadMax a warp.
constexpr int kPrThreadMax = 64;

template <typename WT>
__global__ void pr_a_mark_thread_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                                   const WT* __restrict__ w, const int32_t* __restrict__ partner,
                                   const long long* __restrict__ pw, const long long* __restrict__ deg,
                                   const DevState* st, int32_t* parent, BatchCtx bc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    long long lam;
    if (!pr_graph(bc, st, v, &lam)) continue;
    const int64_t beg = off[v], end = off[v + 1];
    if (end - beg < 2 || end - beg > kPrThreadMax) continue;
    for (int64_t e = beg; e < end; ++e) {
      const int u = adj[e];
      if (u > v && (long long)w[e] >= lam && off[u + 1] - off[u] >= 2) uf_unite(parent, (int)v, u);
    }
    const int p = partner[v];
    if (p >= 0 && off[p + 1] - off[p] >= 2 && deg[v] <= 2 * pw[v]) uf_unite(parent, (int)v, p);
  }
}

// Contracted graphs carry each entry's source, so every entry takes a thread.
// The entry count is the graph's last offset, read on the device (a host-side count
// may be an upper bound).
template <typename WT>
__global__ void pr_a_edge_k(int64_t n, const int32_t* __restrict__ src, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ adj, const WT* __restrict__ w, const DevState* st,
                            int32_t* parent, BatchCtx bc) {
  const int64_t nnz = off[n];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const int v = src[e], u = adj[e];
    if (u <= v) continue;
    long long lam;
    if (!pr_graph(bc, st, v, &lam)) continue;
    if ((long long)w[e] < lam) continue;
    if (off[v + 1] - off[v] < 2 || off[u + 1] - off[u] < 2) continue;
    uf_unite(parent, v, u);
  }
}

// Union-find start for pass A on sorted lists: each vertex points at its smallest
// marked neighbour below it (or at itself).  Every such pointer is a union of a
// marked edge towards a smaller id, so this is a valid forest with min-id roots,
// shallow from the start; the per-entry pass then finds short paths.  Eight lanes per
// vertex read its list in rows of eight ascending entries (four rows at a time) and stop
// at the first row holding a marked entry below v or an entry at or above v.
constexpr int kInitMinG = 8;
constexpr int kInitMinRows = 4;
template <typename WT>
__global__ void uf_init_min_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                              const WT* __restrict__ w, const DevState* st, int32_t* __restrict__ parent,
                              BatchCtx bc) {
  constexpr int G = kInitMinG;
  const int lane = threadIdx.x & 31, glane = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << (G & 31)) - 1u) << (lane & ~(G - 1));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G; v < n; v += groups) {
    int32_t p = (int32_t)v;
    long long lam;
    const int64_t beg = off[v], end = off[v + 1];
    if (end - beg >= 2 && pr_graph(bc, st, v, &lam)) {
      bool found = false;
      for (int64_t b = beg; b < end && !found; b += kInitMinRows * G) {
        // kInitMinRows rows in flight: ids, then the weights of the entries below v,
        // then the list lengths of the heavy ones
        int u[kInitMinRows];
        bool mk[kInitMinRows];
#pragma unroll
        for (int r = 0; r < kInitMinRows; ++r) {
          const int64_t e = b + r * G + glane;
          u[r] = e < end ? adj[e] : INT_MAX;
        }
#pragma unroll
        for (int r = 0; r < kInitMinRows; ++r) mk[r] = u[r] < v && (long long)w[b + r * G + glane] >= lam;
#pragma unroll
        for (int r = 0; r < kInitMinRows; ++r) mk[r] = mk[r] && off[u[r] + 1] - off[u[r]] >= 2;
#pragma unroll
        for (int r = 0; r < kInitMinRows; ++r) {
          const unsigned mb = __ballot_sync(gmask, mk[r]);
          const unsigned past = __ballot_sync(gmask, !(u[r] < v));
          if (mb) {  // sorted: the lowest marked lane holds the smallest marked neighbour
            p = __shfl_sync(gmask, u[r], __ffs(mb) - 1);
            found = true;
            break;
          }
          if (past) {  // no smaller neighbour follows
            found = true;
            break;
          }
        }
      }
    }
    if (glane == 0) parent[v] = p;
  }
}

__global__ void pr_a_partner_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ partner,
                               const long long* __restrict__ pw, const long long* __restrict__ deg,
                               const DevState* st, int32_t* parent, BatchCtx bc) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    long long lam;
    if (!pr_graph(bc, st, v, &lam)) continue;
    if (off[v + 1] - off[v] < 2) continue;
    const int p = partner[v];
    if (p >= 0 && off[p + 1] - off[p] >= 2 && deg[v] <= 2 * pw[v]) uf_unite(parent, (int)v, p);
  }
}

template <typename WT>
__global__ void pr_a_mark_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                            const WT* __restrict__ w, const int32_t* __restrict__ partner,
                            const long long* __restrict__ pw, const long long* __restrict__ deg,
                            const DevState* st, int32_t* parent, BatchCtx bc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    long long lam;
    if (!pr_graph(bc, st, v, &lam)) continue;
    const int64_t beg = off[v], end = off[v + 1];
    if (end - beg <= kPrThreadMax) continue;
    for (int64_t e = beg + lane; e < end; e += 32) {
      int u = adj[e];
      if (u > v && (long long)w[e] >= lam && off[u + 1] - off[u] >= 2) uf_unite(parent, (int)v, u);
    }
    if (lane == 0) {
      int p = partner[v];
      if (p >= 0 && off[p + 1] - off[p] >= 2 && deg[v] <= 2 * pw[v]) uf_unite(parent, (int)v, p);
    }
  }
}

__global__ void uf_flatten_k(int32_t* parent, int64_t n, int32_t* __restrict__ labels, int* changed, BatchCtx bc) {
  int any = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    if (bc.gid && !bc.gact[bc.gid[v]]) continue;
    int r = uf_find(parent, (int)v);
    labels[v] = r;
    if (r != v) {
      any = 1;
      if (bc.gid) bc.gchanged[bc.gid[v]] = 1;
    }
  }
  if (__syncthreads_or(any) && threadIdx.x == 0 && changed) atomicOr(changed, 1);
}

void pr_pass_a(const GraphView& g, const int32_t* partner, const long long* pw, const long long* deg,
               const DevState* st, int32_t* parent, int32_t* labels, int* changed, cudaStream_t s,
               const BatchCtx* bcp) {
  BatchCtx bc = bcp ? *bcp : BatchCtx{};
  int grid1 = grid_for(g.n, 256, kSMs * 8);
  if (!g.src) uf_init_k<<<grid1, 256, 0, s>>>(parent, g.n);
  int grid = grid_for(g.n, 8, kSMs * 16);
  if (g.src) {  // contracted graph: sorted lists and entry sources
    const int ge = grid_for(g.nnz, 256, kSMs * 16);
    const int gi = grid_for(g.n, 256 / kInitMinG, kSMs * 16);
    if (g.wbytes == 4)
      uf_init_min_k<int32_t><<<gi, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, st, parent, bc);
    else
      uf_init_min_k<long long><<<gi, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, st, parent, bc);
    if (g.wbytes == 4)
      pr_a_edge_k<int32_t><<<ge, 256, 0, s>>>(g.n, g.src, g.off, g.adj, (const int32_t*)g.w, st, parent, bc);
    else
      pr_a_edge_k<long long><<<ge, 256, 0, s>>>(g.n, g.src, g.off, g.adj, (const long long*)g.w, st, parent, bc);
    pr_a_partner_k<<<grid1, 256, 0, s>>>(g.n, g.off, partner, pw, deg, st, parent, bc);
  } else if (g.wbytes == 4) {
    pr_a_mark_thread_k<int32_t><<<grid1, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, partner, pw, deg, st,
                                                      parent, bc);
    pr_a_mark_k<int32_t><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, partner, pw, deg, st, parent, bc);
  } else {
    pr_a_mark_thread_k<long long><<<grid1, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, partner, pw, deg,
                                                        st, parent, bc);
    pr_a_mark_k<long long><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, partner, pw, deg, st,
                                                parent, bc);
  }
  uf_flatten_k<<<grid1, 256, 0, s>>>(parent, g.n, labels, changed, bc);
  count_launch(4);
  VC_CHECK_LAUNCH();
}

// Conditions 3 and 4 on mutual partner pairs v < w = p(v), p(w) = v, through the
// common neighbourhood: the warp walks the shorter of the two lists and finds each entry
// in the longer one by binary search (a longer list of at most kPrBStage ids is first
// copied into the warp's shared memory, so the searches there wait on no global loads).
// Walking the shorter list keeps a pair of a hub and a small vertex as cheap as the
// small vertex's list.
constexpr int kPrBStage = 1024;
template <typename WT>
__global__ void __launch_bounds__(256) pr_b_k(int64_t n, const int64_t* __restrict__ off,
                                              const int32_t* __restrict__ adj, const WT* __restrict__ w,
                                              const int32_t* __restrict__ partner, const long long* __restrict__ pw,
                                              const long long* __restrict__ deg, const DevState* st,
                                              int32_t* __restrict__ labels, int* changed, BatchCtx bc) {
  __shared__ int32_t s_list[8][kPrBStage];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* sl = s_list[wid];
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    long long lam;
    if (!pr_graph(bc, st, v, &lam)) continue;
    const int p = partner[v];
    if (p <= v || partner[p] != v) continue;
    const int64_t vb = off[v], ve = off[v + 1], pb = off[p], pe = off[p + 1];
    if (ve - vb < 2 || pe - pb < 2) continue;
    const long long cvw = pw[v], dv = deg[v], dp = deg[p];
    // walk list s, search list l (s the shorter; ties: walk v's)
    const bool swap = pe - pb < ve - vb;
    const int64_t sb = swap ? pb : vb, se = swap ? pe : ve, lb = swap ? vb : pb, le = swap ? ve : pe;
    const bool staged = le - lb <= kPrBStage;
    if (staged)
      for (int64_t i = lane; i < le - lb; i += 32) sl[i] = adj[lb + i];
    __syncwarp();
    bool pr3 = false;
    long long sum = 0;
    for (int64_t e = sb + lane; e < se; e += 32) {
      const int u = adj[e];
      int64_t lo = lb, hi = le;
      if (staged) {
        int l = 0, h = (int)(le - lb);
        while (l < h) {
          const int mid = (l + h) >> 1;
          if (sl[mid] < u) l = mid + 1;
          else h = mid;
        }
        lo = lb + l;
      } else {
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (adj[mid] < u) lo = mid + 1;
          else hi = mid;
        }
      }
      if (lo < le && (staged ? sl[lo - lb] : adj[lo]) == u) {
        const long long cs = (long long)w[e], cl = (long long)w[lo];
        const long long cvu = swap ? cl : cs, cwu = swap ? cs : cl;  // c(v, u), c(p, u)
        if (dv <= 2 * (cvw + cvu) && dp <= 2 * (cvw + cwu)) pr3 = true;
        sum += cvu < cwu ? cvu : cwu;
      }
    }
    pr3 = __any_sync(0xffffffffu, pr3);
    sum = warp_sum(sum);
    if (lane == 0 && (pr3 || cvw + sum >= lam)) {
      labels[p] = (int32_t)v;
      if (changed) atomicOr(changed, 1);
      if (bc.gid) bc.gchanged[bc.gid[v]] = 1;
    }
    __syncwarp();  // the staged list is overwritten by the warp's next pair
  }
}

void pr_pass_b(const GraphView& g, const int32_t* partner, const long long* pw, const long long* deg,
               const DevState* st, int32_t* labels, int* changed, cudaStream_t s, const BatchCtx* bcp) {
  BatchCtx bc = bcp ? *bcp : BatchCtx{};
  if (!bc.gid) iota(labels, g.n, s);
  int grid = grid_for(g.n, 8, kSMs * 16);
  if (g.wbytes == 4)
    pr_b_k<int32_t><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const int32_t*)g.w, partner, pw, deg, st, labels,
                                         changed, bc);
  else
    pr_b_k<long long><<<grid, 256, 0, s>>>(g.n, g.off, g.adj, (const long long*)g.w, partner, pw, deg, st, labels,
                                           changed, bc);
  count_launch();
  VC_CHECK_LAUNCH();
}

}  // namespace vc
