// Batched solving: many graphs of uneven sizes solved together.
//
// The graphs are laid out as one disjoint union on the device (graph g owns the
// contiguous vertex range [vbase[g], vbase[g+1])).  Each graph carries its own state
// machine -- label-propagation level, Padberg-Rinaldi pass A, pass B, exact step
// (sparse rounds or the dense single-block kernel), done -- and the engine advances
// all graphs in lock-step "super-steps": one pass per graph (label propagation only
// touches graphs in that phase, each with its own tie-break key; the PR passes read
// each graph's own bound), then one contraction of the whole union serves every graph
// (clusters never cross graphs, so every graph's coarse ids stay contiguous; graphs
// that did not change pass through unchanged; finished graphs are dropped).  The
// exact step runs as persistent kernels that pull graphs from a list, a block per
// graph.  Per graph the arithmetic and the order of steps are exactly those of a
// single-graph run, so every result equals the graph's result alone.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>

#include "engine.cuh"

namespace vc {

enum BPhase { kBLP = 0, kBPRA = 1, kBPRB = 2, kBNoiS = 3, kBNoiD = 4, kBDone = 5, kBGone = 6 };
constexpr int kBTraceCap = 512;
constexpr int kSummaryInts = 16;

// Device arrays of the per-graph state (K graphs).
struct BState {
  int *phase, *level, *run, *any, *changed, *contracted, *first, *did, *best_kind, *trace_len;
  long long *vbase, *vbase_new, *nv, *nnz, *n_start, *lam, *best_vertex, *argmin, *dmin, *obase, *norig, *n1,
      *noi_base;
  long long* nv_new;
  unsigned long long* gkey;
  unsigned long long* seed;
  unsigned char* gact;
  TraceStep* trace;
  int* summary;  // [0..6] phase counts, [7] max n among NOI_D graphs, [8] contract or drop count
  int32_t *list_noid, *list_nois;
};

// ---------------------------------------------------------------- union setup
__global__ void b_rebase_k(int K, const long long* vbase, const long long* ebase, int64_t* off, int32_t* adj) {
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    const long long vb = vbase[g], ve = vbase[g + 1], eb = ebase[g], ee = ebase[g + 1];
    for (long long i = vb + threadIdx.x; i < ve; i += blockDim.x) off[i] += eb;
    for (long long e = eb + threadIdx.x; e < ee; e += blockDim.x) adj[e] += (int32_t)vb;
  }
}

// per-graph validation before the rebase: local ids in range, no self-loops, weights
// >= 1, offsets non-decreasing; bit 32 / 64 report non-unit weights / non-simple lists
__global__ void b_validate_k(int K, const long long* vbase, const long long* ebase, const int64_t* off,
                             const int32_t* adj, const int32_t* w, int* err) {
  int bad = 0;
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    const long long vb = vbase[g], n = vbase[g + 1] - vb, eb = ebase[g], m = ebase[g + 1] - eb;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      const long long a = off[vb + i], b = (i + 1 < n) ? off[vb + i + 1] : m;
      if (a > b || a < 0 || b > m) { bad |= 2; continue; }
      for (long long e = a; e < b; ++e) {
        const int32_t u = adj[eb + e];
        if (u < 0 || u >= n) bad |= 4;
        else if (u == i) bad |= 8;
        if (w[eb + e] < 1) bad |= 16;
        if (w[eb + e] != 1) bad |= 32;
        if (e + 1 < b && adj[eb + e + 1] <= u) bad |= 64;
      }
    }
  }
  if (bad) atomicOr(err, bad);
}

// vertex -> graph map for the graphs that just joined the union (first & 8)
__global__ void b_gid_init_k(int K, BState S, int32_t* gid) {
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    if (!(S.first[g] & 8)) continue;
    const long long vb = S.vbase[g], ve = vb + S.nv[g];
    for (long long v = vb + threadIdx.x; v < ve; v += blockDim.x) gid[v] = g;
  }
}

// ---------------------------------------------------------------- per-graph steps
// minimum degree with smallest argmin over each graph's range; mode 0 = initial
// bound, mode 1 = update of the graphs that contracted (did[g])
__global__ void b_segmin_k(int K, const long long* __restrict__ deg, BState S, int mode) {
  __shared__ long long sd[8], sv[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    if (mode == 1 && (!S.did[g] || S.nv[g] <= 1)) continue;
    if (mode == 0 && (!(S.first[g] & 8) || S.nv[g] < 1)) continue;
    const long long vb = S.vbase[g], ve = vb + S.nv[g];
    long long bd = LLONG_MAX, bv = LLONG_MAX;
    for (long long v = vb + threadIdx.x; v < ve; v += blockDim.x) {
      const long long d = deg[v];
      if (d < bd || (d == bd && v < bv)) { bd = d; bv = v; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      long long od = __shfl_xor_sync(0xffffffffu, bd, o), ov = __shfl_xor_sync(0xffffffffu, bv, o);
      if (od < bd || (od == bd && ov < bv)) { bd = od; bv = ov; }
    }
    if (lane == 0) { sd[wid] = bd; sv[wid] = bv; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
        if (sd[q] < bd || (sd[q] == bd && sv[q] < bv)) { bd = sd[q]; bv = sv[q]; }
      S.dmin[g] = bd;
      S.argmin[g] = bv;
      if (mode == 0) {
        S.lam[g] = bd;
        S.best_vertex[g] = bv - vb;
        S.best_kind[g] = 0;
      } else if (bd < S.lam[g]) {
        S.lam[g] = bd;
        S.best_kind[g] = 1;
        S.first[g] |= 2;  // improved: snapshot the side
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void b_push(BState& S, int g, int kind) {
  const int i = S.trace_len[g];
  if (i < kBTraceCap)
    S.trace[(int64_t)g * kBTraceCap + i] = TraceStep{kind, S.level[g], S.nv[g], S.nnz[g], S.lam[g]};
  S.trace_len[g] = i + 1;
}

__device__ __forceinline__ void b_enter_noi(BState& S, int g) { S.phase[g] = S.nv[g] > kDenseMax ? kBNoiS : kBNoiD; }

// initial phase of the graphs that just joined (first & 8), after their initial bound
__global__ void b_init_k(int K, BState S, long long n0) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    if (!(S.first[g] & 8)) continue;
    S.level[g] = 0;
    S.run[g] = 0;
    S.any[g] = 0;
    S.trace_len[g] = 0;
    S.contracted[g] = 0;
    S.n1[g] = 0;
    S.first[g] = 0;
    S.best_kind[g] = 0;
    S.noi_base[g] = 0;
    b_push(S, g, 0);
    if (S.lam[g] == 0) {
      S.phase[g] = kBDone;
    } else if (S.nv[g] > n0) {
      S.phase[g] = kBLP;
      S.n_start[g] = S.nv[g];
    } else {
      b_enter_noi(S, g);
      S.first[g] = 4;  // tier-1 is the graph itself
    }
  }
}

// tier-1 set-up and upkeep: identity for graphs entering the exact step uncontracted
// (first & 4), the first contraction's map (first & 1), map composition otherwise
__global__ void b_tier1_k(int K, BState S, const int32_t* __restrict__ cid, int32_t* map0, int32_t* cur1, int after) {
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    const long long ob = S.obase[g];
    if (!after) {
      if (!(S.first[g] & 4)) continue;
      const long long vb = S.vbase[g], n = S.nv[g];
      for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        map0[ob + i] = (int32_t)i;
        cur1[ob + i] = (int32_t)(vb + i);
      }
      if (threadIdx.x == 0) {
        S.n1[g] = n;
        S.contracted[g] = 1;
        S.first[g] &= ~4;
      }
      continue;
    }
    const int ph = S.phase[g];
    if (ph == kBGone || ph == kBDone) continue;  // dropped in this contraction
    if (S.did[g] && !S.contracted[g]) {
      // first contraction: original vertex i sat at vbase[g] + i
      const long long vb = S.vbase[g], nb = S.vbase_new[g], n = S.norig[g], c = S.nv_new[g];
      for (long long i = threadIdx.x; i < n; i += blockDim.x) map0[ob + i] = (int32_t)(cid[vb + i] - nb);
      for (long long j = threadIdx.x; j < c; j += blockDim.x) cur1[ob + j] = (int32_t)(nb + j);
      if (threadIdx.x == 0) {
        S.n1[g] = c;
        S.contracted[g] = 1;
      }
    } else if (S.contracted[g]) {
      // every union contraction renumbers the vertices, changed or not
      const long long n1 = S.n1[g];
      for (long long j = threadIdx.x; j < n1; j += blockDim.x) cur1[ob + j] = cid[cur1[ob + j]];
    }
  }
}

__global__ void b_snapshot_k(int K, BState S, const int32_t* __restrict__ cur1, unsigned char* side1) {
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    if (!(S.first[g] & 2)) continue;
    const long long ob = S.obase[g], n1 = S.n1[g], b = S.argmin[g];
    for (long long j = threadIdx.x; j < n1; j += blockDim.x) side1[ob + j] = cur1[ob + j] == b ? 1 : 0;
    __syncthreads();
    if (threadIdx.x == 0) S.first[g] &= ~2;
  }
}

// per graph: activity for the pass of phase `ph`; LP also gets its level key
__global__ void b_prepare_k(int K, BState S, int ph) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const bool a = S.phase[g] == ph;
    S.gact[g] = a ? 1 : 0;
    if (ph == kBLP) S.gkey[g] = level_key(S.seed[g], S.level[g]);
  }
}

__global__ void b_vact_k(int64_t n, const int32_t* __restrict__ gid, const unsigned char* __restrict__ gact,
                         unsigned char* vact) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    vact[v] = gact[gid[v]];
}

// phase counts, lists of the exact-step graphs, largest dense-step graph
__global__ void b_summary_k(int K, BState S) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const int ph = S.phase[g];
    atomicAdd(&S.summary[ph], 1);
    S.changed[g] = 0;
    S.did[g] = 0;
    if (ph == kBNoiD) {
      S.list_noid[atomicAdd(&S.summary[9], 1)] = g;
      atomicMax(&S.summary[7], (int)S.nv[g]);
      S.noi_base[g] = S.vbase[g];
    } else if (ph == kBNoiS) {
      S.list_nois[atomicAdd(&S.summary[10], 1)] = g;
      atomicMax(&S.summary[11], (int)S.nv[g]);
    }
  }
}

// which graphs contract (or are dropped) in this super-step
__global__ void b_decide_k(int K, BState S) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    int ph = S.phase[g];
    if (ph == kBNoiD) S.phase[g] = ph = kBDone;  // the dense kernel finished it
    const bool c = ph == kBLP || ((ph == kBPRA || ph == kBPRB || ph == kBNoiS) && S.changed[g]);
    S.did[g] = c ? 1 : 0;
    if (c || ph == kBDone) atomicAdd(&S.summary[8], 1);
  }
}

__global__ void b_drop_k(int64_t n, const int32_t* __restrict__ gid, const int* __restrict__ phase, int32_t* lab) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    if (phase[gid[v]] == kBDone) lab[v] = -1;
}

// new vertex ranges after a union contraction: a vertex id x of the old union maps to
// the rank of x among the kept labels (exclusive scan of the flags), so graph g's new
// range is [rank(vbase), rank(vbase + nv)); dropped graphs end up empty
__global__ void b_shape_k(int K, BState S, int64_t n_old, int64_t c_total, const int32_t* __restrict__ rank) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    if (S.phase[g] == kBGone) {
      S.vbase_new[g] = 0;
      S.nv_new[g] = 0;
      continue;
    }
    const long long vb = S.vbase[g], ve = vb + S.nv[g];
    const long long nb = vb < n_old ? (long long)rank[vb] : c_total;
    const long long ne = ve < n_old ? (long long)rank[ve] : c_total;
    S.vbase_new[g] = nb;
    S.nv_new[g] = ne - nb;
  }
}

__global__ void b_gid_update_k(int64_t n, const int32_t* __restrict__ cid, const int32_t* __restrict__ gid,
                               int32_t* gid_new) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cid[v];
    if (c >= 0) gid_new[c] = gid[v];
  }
}

__global__ void b_copy_shape_k(int K, BState S, const int64_t* __restrict__ coff) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const long long a = S.vbase_new[g], n = S.nv_new[g];
    S.vbase[g] = a;
    S.nv[g] = n;
    S.nnz[g] = n > 0 ? coff[a + n] - coff[a] : 0;
  }
}

__global__ void b_trace_k(int K, BState S) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    if (!S.did[g]) continue;
    const int ph = S.phase[g];
    b_push(S, g, ph == kBLP ? 1 : ph == kBPRA ? 2 : ph == kBPRB ? 3 : 4);
  }
}

// the per-graph control flow of Algorithm 1 (same order as a single-graph run)
__global__ void b_transition_k(int K, BState S, long long n0, int pr_runs_max) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const int ph = S.phase[g];
    if (ph == kBGone) continue;
    if (ph == kBDone) { S.phase[g] = kBGone; continue; }
    const bool did = S.did[g] != 0;
    const bool fin = did && (S.nv[g] <= 1 || S.lam[g] == 0);
    bool end_level = false;
    if (ph == kBLP) {
      if (fin) S.phase[g] = kBDone;
      else if (pr_runs_max == 0) end_level = true;
      else { S.phase[g] = kBPRA; S.run[g] = 0; S.any[g] = 0; }
    } else if (ph == kBPRA) {
      if (did) S.any[g] = 1;
      S.phase[g] = fin ? kBDone : kBPRB;
    } else if (ph == kBPRB) {
      if (did) S.any[g] = 1;
      if (fin) S.phase[g] = kBDone;
      else if (S.any[g] && S.run[g] + 1 < pr_runs_max) { S.run[g] += 1; S.any[g] = 0; S.phase[g] = kBPRA; }
      else end_level = true;
    } else if (ph == kBNoiS) {
      if (!did || fin) S.phase[g] = kBDone;
      else if (S.nv[g] <= kDenseMax) S.phase[g] = kBNoiD;
    }
    if (end_level) {
      S.level[g] += 1;
      if (S.nv[g] == S.n_start[g] || S.nv[g] <= n0) b_enter_noi(S, g);
      else { S.phase[g] = kBLP; S.n_start[g] = S.nv[g]; }
    }
  }
}

// final side bitmaps of the listed slots: slot list[i]'s words start at wbase[i]
__global__ void b_side_bits_k(const int32_t* __restrict__ list, int count, BState S, const long long* __restrict__ wbase,
                              const int32_t* __restrict__ map0, const unsigned char* __restrict__ side1,
                              const int32_t* __restrict__ cur1, const unsigned char* __restrict__ sideK,
                              unsigned long long* bits) {
  for (int idx = blockIdx.x; idx < count; idx += gridDim.x) {
    const int g = list ? list[idx] : idx;
    const long long n = S.norig[g], ob = S.obase[g];
    const int kind = S.best_kind[g];
    const long long bv = S.best_vertex[g], nb = S.noi_base[g];
    const unsigned char* sk = sideK + (int64_t)g * kDenseMax;
    auto side_of = [&](long long i) -> int {
      if (kind == 0) return i == bv;
      const int32_t t = map0[ob + i];
      if (kind == 1) return side1[ob + t];
      return sk[cur1[ob + t] - nb];
    };
    const int flip = side_of(0);
    const long long words = (n + 63) / 64;
    for (long long wd = threadIdx.x; wd < words; wd += blockDim.x) {
      unsigned long long x = 0;
      const long long lim = (wd + 1) * 64 < n ? (wd + 1) * 64 : n;
      for (long long i = wd * 64; i < lim; ++i)
        if (side_of(i) != flip) x |= 1ULL << (i & 63);
      bits[wbase[idx] + wd] = x;
    }
  }
}

// appends graphs to the union: graph j of the staged arrays (host CSR copied as is,
// local ids, int32 weights) lands at vertex base jv[j] / entry base je[j]
__global__ void b_join_k(int J, const long long* __restrict__ jv, const long long* __restrict__ je,
                         const long long* __restrict__ sv, const long long* __restrict__ se,
                         const long long* __restrict__ nn, const long long* __restrict__ mm,
                         const int64_t* __restrict__ st_off, const int32_t* __restrict__ st_adj,
                         const int32_t* __restrict__ st_w, int64_t* off, int32_t* adj, long long* w) {
  for (int j = blockIdx.x; j < J; j += gridDim.x) {
    const long long n = nn[j], m = mm[j];
    for (long long i = threadIdx.x; i < n; i += blockDim.x) off[jv[j] + i] = je[j] + st_off[sv[j] + i];
    for (long long e = threadIdx.x; e < m; e += blockDim.x) {
      adj[je[j] + e] = (int32_t)(jv[j] + st_adj[se[j] + e]);
      w[je[j] + e] = (long long)st_w[se[j] + e];
    }
  }
}

// Staged vertex -> index of its joining request.
__global__ void b_stage_gid_k(int J, const long long* __restrict__ sv, int32_t* __restrict__ sgid) {
  for (int j = blockIdx.x; j < J; j += gridDim.x)
    for (long long v = sv[j] + threadIdx.x; v < sv[j + 1]; v += blockDim.x) sgid[v] = j;
}

// Checks of the joining requests in the staging buffers (request-local offsets, n
// per request, the end of the last list being m), a warp per vertex; err[j] gathers
// request j's findings: 2 offsets, 4 id range, 8 self-loop, 16 weight < 1; 32 (not
// all weights 1) and 64 (a list not strictly increasing) are facts, not errors.
__global__ void b_validate_staged_k(long long sn, const int32_t* __restrict__ sgid, const long long* __restrict__ sv,
                                    const long long* __restrict__ se, const int64_t* __restrict__ off,
                                    const int32_t* __restrict__ adj, const int32_t* __restrict__ w, int* err) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < sn; v += warps) {
    const int j = sgid[v];
    const long long i = v - sv[j], n = sv[j + 1] - sv[j], m = se[j + 1] - se[j], eb = se[j];
    const long long a = off[v], b = (i + 1 < n) ? off[v + 1] : m;
    int bad = 0;
    if (a > b || a < 0 || b > m) {
      bad = 2;
    } else {
      for (long long e = a + lane; e < b; e += 32) {
        const int32_t u = adj[eb + e];
        if (u < 0 || u >= n) bad |= 4;
        else if (u == i) bad |= 8;
        const int32_t x = w[eb + e];
        if (x < 1) bad |= 16;
        if (x != 1) bad |= 32;
        if (e + 1 < b && adj[eb + e + 1] <= u) bad |= 64;
      }
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicOr(err + j, bad);
  }
}

// per-slot values of graphs joining the union
struct SlotInit {
  int slot;
  int pad;
  long long vbase, n, m, obase;
  unsigned long long seed;
};

__global__ void b_slot_init_k(int J, const SlotInit* __restrict__ in, BState S) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < J; j += gridDim.x * blockDim.x) {
    const SlotInit x = in[j];
    S.vbase[x.slot] = x.vbase;
    S.nv[x.slot] = x.n;
    S.nnz[x.slot] = x.m;
    S.norig[x.slot] = x.n;
    S.obase[x.slot] = x.obase;
    S.seed[x.slot] = x.seed;
    S.first[x.slot] = 8;
  }
}

__global__ void b_set_i64_k(int64_t* p, int64_t v) { *p = v; }

// ------------------------------------------------------------------ host side
// Grows a persistent device array, keeping its first `keep` bytes.
static void grow_keep(Buf& b, size_t bytes, size_t keep, cudaStream_t s) {
  if (bytes <= b.cap) return;
  void* p = nullptr;
  if (take_injected_alloc_failure())
    throw Error{VIECUT_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed (injected)"};
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{VIECUT_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
  }
  if (keep && b.p) VC_CUDA(cudaMemcpyAsync(p, b.p, keep, cudaMemcpyDeviceToDevice, s));
  VC_CUDA(cudaStreamSynchronize(s));
  b.release();
  b.p = p;
  b.cap = bytes;
}

// The engine shared by batches and the server: K slots of per-graph state, the
// current union, the per-original-vertex arrays (map0 / cur1 / side1, slot g's at
// [obase, obase + norig)) and the workspace.
struct Engine {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int K = 0;
  int64_t n0 = 10000;
  int pr_runs_max = 8;
  int lp_iters = 2;
  // per-slot state
  Buf phase, level, run, any, changed, contracted, first, did, best_kind, trace_len;
  Buf vbase, vbase_new, nv, nv_new, nnz, n_start, lam, best_vertex, argmin, dmin, obase, norig, n1, noi_base;
  Buf gkey, seed, gact, trace, summary, list_noid, list_nois;
  // union
  GraphView G;
  int slot = -1;  // coarse buffer of the workspace holding G (-1: in_*)
  Buf in_off, in_adj, in_w;
  Buf gidA, gidB;
  int32_t* gid = nullptr;
  Buf vact, sideK, noiM, noiCurK, noiQ;
  // the exact-step phases run on their own stream beside the other phases of a
  // super-step (they touch only their graphs' vertices and state)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Buf om0, oc1, os1;  // per original vertex
  int64_t ocap = 0;
  Workspace* ws = nullptr;
  int* h_summary = nullptr;
  int64_t steps = 0;
  ~Engine() {
    delete ws;
    if (h_summary) cudaFreeHost(h_summary);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  BState state() {
    BState S;
    S.phase = phase.as<int>(); S.level = level.as<int>(); S.run = run.as<int>(); S.any = any.as<int>();
    S.changed = changed.as<int>(); S.contracted = contracted.as<int>(); S.first = first.as<int>();
    S.did = did.as<int>(); S.best_kind = best_kind.as<int>(); S.trace_len = trace_len.as<int>();
    S.vbase = vbase.as<long long>(); S.vbase_new = vbase_new.as<long long>(); S.nv = nv.as<long long>();
    S.nv_new = nv_new.as<long long>(); S.nnz = nnz.as<long long>(); S.n_start = n_start.as<long long>();
    S.lam = lam.as<long long>(); S.best_vertex = best_vertex.as<long long>(); S.argmin = argmin.as<long long>();
    S.dmin = dmin.as<long long>(); S.obase = obase.as<long long>(); S.norig = norig.as<long long>();
    S.n1 = n1.as<long long>(); S.noi_base = noi_base.as<long long>(); S.gkey = gkey.as<unsigned long long>();
    S.seed = seed.as<unsigned long long>(); S.gact = gact.as<unsigned char>(); S.trace = trace.as<TraceStep>();
    S.summary = summary.as<int>(); S.list_noid = list_noid.as<int32_t>(); S.list_nois = list_nois.as<int32_t>();
    return S;
  }
};

static void engine_setup(Engine& E, int K, const viecut_opts& o) {
  E.K = K;
  E.n0 = o.n0;
  E.pr_runs_max = o.pr_runs_max;
  E.device = o.device;
  VC_CUDA(cudaSetDevice(E.device));
  if (o.stream) {
    E.stream = (cudaStream_t)o.stream;
  } else {
    VC_CUDA(cudaStreamCreateWithFlags(&E.stream, cudaStreamNonBlocking));
    E.own_stream = true;
  }
  VC_CUDA(cudaStreamCreateWithFlags(&E.side, cudaStreamNonBlocking));
  VC_CUDA(cudaEventCreateWithFlags(&E.ev_fork, cudaEventDisableTiming));
  VC_CUDA(cudaEventCreateWithFlags(&E.ev_join, cudaEventDisableTiming));
  for (Buf* b : {&E.phase, &E.level, &E.run, &E.any, &E.changed, &E.contracted, &E.first, &E.did, &E.best_kind,
                 &E.trace_len})
    b->ensure_n<int>(K);
  for (Buf* b : {&E.nv, &E.nv_new, &E.nnz, &E.n_start, &E.lam, &E.best_vertex, &E.argmin, &E.dmin, &E.obase,
                 &E.norig, &E.n1, &E.noi_base, &E.vbase, &E.vbase_new})
    b->ensure_n<long long>(K);
  E.gkey.ensure_n<unsigned long long>(K);
  E.seed.ensure_n<unsigned long long>(K);
  E.gact.ensure_n<unsigned char>(K);
  E.trace.ensure_n<TraceStep>((int64_t)K * kBTraceCap);
  E.summary.ensure_n<int>(kSummaryInts);
  E.list_noid.ensure_n<int32_t>(K);
  E.list_nois.ensure_n<int32_t>(K);
  E.sideK.ensure_n<unsigned char>((int64_t)K * kDenseMax);
  E.noiCurK.ensure_n<int32_t>((int64_t)kSMs * kNoiDenseBlocksPerSM * kDenseMax);  // per dense-step block
  VC_CUDA(cudaMemsetAsync(E.phase.p, 0, sizeof(int) * K, E.stream));
  {
    std::vector<int> gone(K, kBGone);
    VC_CUDA(cudaMemcpy(E.phase.p, gone.data(), sizeof(int) * K, cudaMemcpyHostToDevice));
  }
  VC_CUDA(cudaMallocHost(&E.h_summary, sizeof(int) * kSummaryInts));
  E.ws = new Workspace;
  E.ws->s = E.stream;
  E.ws->fix_groups(o.lp_group, o.emit_group);
}

static void read_summary(Engine& E) {
  VC_CUDA(cudaMemcpyAsync(E.h_summary, E.summary.p, sizeof(int) * kSummaryInts, cudaMemcpyDeviceToHost, E.stream));
  VC_CUDA(cudaStreamSynchronize(E.stream));
}

// Bound, phase and tier-1 set-up of the slots flagged new (first & 8); the union,
// gid, vbase, nv, nnz, norig, obase and seed of those slots must be in place.
static void engine_start_new(Engine& E) {
  cudaStream_t s = E.stream;
  Workspace& W = *E.ws;
  BState S = E.state();
  const int K = E.K;
  const int gK = (K + 255) / 256, gridK = K < 4 * kSMs ? K : 4 * kSMs;
  degrees(E.G, W.deg.as<long long>(), s);
  b_segmin_k<<<gridK, 256, 0, s>>>(K, W.deg.as<long long>(), S, 0);
  b_init_k<<<gK, 256, 0, s>>>(K, S, E.n0);
  b_tier1_k<<<gridK, 256, 0, s>>>(K, S, nullptr, E.om0.as<int32_t>(), E.oc1.as<int32_t>(), 0);
  count_launch(3);
  VC_CHECK_LAUNCH();
}

// One super-step for every slot; returns false when no slot is active.
static bool engine_step(Engine& E) {
  cudaStream_t s = E.stream;
  Workspace& W = *E.ws;
  BState S = E.state();
  const int K = E.K;
  const int gK = (K + 255) / 256, gridK = K < 4 * kSMs ? K : 4 * kSMs;
  GraphView& G = E.G;
  VC_CUDA(cudaMemsetAsync(S.summary, 0, sizeof(int) * kSummaryInts, s));
  b_summary_k<<<gK, 256, 0, s>>>(K, S);
  count_launch();
  read_summary(E);
  const int* cnt = E.h_summary;
  if (cnt[kBLP] + cnt[kBPRA] + cnt[kBPRB] + cnt[kBNoiS] + cnt[kBNoiD] + cnt[kBDone] == 0) return false;
  ++E.steps;
  int32_t* A = W.labA.as<int32_t>();
  int32_t* Bl = W.labB.as<int32_t>();
  iota(A, G.n, s);
  iota(Bl, G.n, s);
  // the super-step's labels: the last label-propagation round writes its graphs' into
  // bufs[(lp_iters - 1) & 1] (below), and every other phase writes its graphs' there too
  int32_t* F = (cnt[kBLP] > 0 && E.lp_iters > 0) ? ((E.lp_iters - 1) & 1 ? Bl : A) : A;
  // the exact-step phases (latency-bound scans of single graphs) on the side stream,
  // beside label propagation and Padberg-Rinaldi on the others; buffers grow first (a
  // reallocation waits for the device)
  const bool exact = cnt[kBNoiS] > 0 || cnt[kBNoiD] > 0;
  if (exact) {
    long long* M = nullptr;
    int64_t mcap = 0;
    int blocks = 0;
    if (cnt[kBNoiS] > 0) {
      W.noi_r.ensure_n<long long>(noi_round_scratch(G.n));
      W.noi_seen.ensure_n<int>(G.n);
      E.noiQ.ensure_n<int32_t>(G.n);
    }
    if (cnt[kBNoiD] > 0) {
      mcap = (int64_t)cnt[7] * cnt[7];
      // up to four blocks per SM (a dense round waits on a row read per scan step:
      // graphs in flight hide it); each block keeps its own two matrices
      blocks = std::min(cnt[kBNoiD], kSMs * kNoiDenseBlocksPerSM);
      M = E.noiM.ensure_n<long long>(2 * mcap * blocks);
    }
    VC_CUDA(cudaEventRecord(E.ev_fork, s));
    VC_CUDA(cudaStreamWaitEvent(E.side, E.ev_fork, 0));
    if (cnt[kBNoiS] > 0)
      noi_round_batch(G, S.list_nois, cnt[10], S.vbase, S.nv, S.lam, W.noi_r.as<long long>(),
                      W.noi_seen.as<int>(), E.noiQ.as<int32_t>(), F, S.changed, cnt[11], E.side);
    if (cnt[kBNoiD] > 0) {
      BatchNoi bn{S.lam, S.best_kind, S.nv, S.nnz, S.dmin, S.argmin, S.trace_len, S.trace, kBTraceCap, S.level};
      noi_dense_batch(G, S.list_noid, cnt[kBNoiD], S.vbase, S.nv, M, mcap, blocks, E.noiCurK.as<int32_t>(),
                      E.sideK.as<unsigned char>(), bn, E.side);
    }
    VC_CUDA(cudaEventRecord(E.ev_join, E.side));
  }
  BatchCtx bc;
  bc.gid = E.gid;
  bc.glam = S.lam;
  bc.gact = S.gact;
  bc.gchanged = S.changed;
  if (cnt[kBLP] > 0) {
    b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBLP);
    b_vact_k<<<grid_for(G.n, 256, kSMs * 8), 256, 0, s>>>(G.n, E.gid, S.gact, E.vact.as<unsigned char>());
    count_launch(2);
    hash_table(G.n, 0, E.gid, S.gkey, S.vbase, W.hv.as<unsigned long long>(), s);
    if (!W.bins_valid) W.build_bins(G);
    GraphView Ga = G;
    Ga.vact = E.vact.as<unsigned char>();
    int32_t* in = nullptr;
    int32_t* bufs[2] = {A, Bl};
    for (int r = 0; r < E.lp_iters; ++r) {
      if (!in) W.tune_first(Ga, bufs[r & 1]);
      lp_round(Ga, W.bins, W.gt, in, bufs[r & 1], W.hv.as<unsigned long long>(), s, W.tune);
      in = bufs[r & 1];
    }
  }
  if (cnt[kBPRA] > 0) {
    b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBPRA);
    count_launch();
    pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
    pr_pass_a(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(),
              W.parent.as<int32_t>(), F, nullptr, s, &bc);
  }
  if (cnt[kBPRB] > 0) {
    b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBPRB);
    count_launch();
    pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
    pr_pass_b(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(), F, nullptr, s, &bc);
  }
  if (exact) VC_CUDA(cudaStreamWaitEvent(s, E.ev_join, 0));
  b_decide_k<<<gK, 256, 0, s>>>(K, S);
  count_launch();
  read_summary(E);
  if (E.h_summary[8] > 0) {
    b_drop_k<<<grid_for(G.n, 256, kSMs * 8), 256, 0, s>>>(G.n, E.gid, S.phase, F);
    count_launch();
    const int dst = E.slot == 0 ? 1 : 0;
    int32_t* cid = W.cidT.as<int32_t>();
    const int64_t n_old = G.n;
    GraphView h = W.contract(G, F, cid, dst);
    int32_t* gid_new = (E.gid == E.gidA.as<int32_t>()) ? E.gidB.as<int32_t>() : E.gidA.as<int32_t>();
    b_shape_k<<<gK, 256, 0, s>>>(K, S, n_old, h.n, W.rank.as<int32_t>());
    b_gid_update_k<<<grid_for(n_old, 256, kSMs * 8), 256, 0, s>>>(n_old, cid, E.gid, gid_new);
    b_tier1_k<<<gridK, 256, 0, s>>>(K, S, cid, E.om0.as<int32_t>(), E.oc1.as<int32_t>(), 1);
    b_copy_shape_k<<<gK, 256, 0, s>>>(K, S, h.off);
    count_launch(4);
    VC_CHECK_LAUNCH();
    E.gid = gid_new;
    G = h;
    E.slot = dst;
    if (G.n > 0) {
      degrees(G, W.deg.as<long long>(), s);
      b_segmin_k<<<gridK, 256, 0, s>>>(K, W.deg.as<long long>(), S, 1);
      b_snapshot_k<<<gridK, 256, 0, s>>>(K, S, E.oc1.as<int32_t>(), E.os1.as<unsigned char>());
      count_launch(2);
    }
    b_trace_k<<<gK, 256, 0, s>>>(K, S);
    count_launch();
  }
  b_transition_k<<<gK, 256, 0, s>>>(K, S, E.n0, E.pr_runs_max);
  count_launch();
  VC_CHECK_LAUNCH();
  return true;
}

// ------------------------------------------------------------------ batches
struct Batch {
  Engine E;
  std::vector<int64_t> h_vbase, h_ebase, h_wbase;
  Buf d_vbase0, d_ebase, d_wbase, bits_out;
  bool unit = false, simple = false;
  viecut_batch_stats stats{};
};

static void batch_create(Batch& B, const viecut_graph_desc* gs, int K, const viecut_opts& o) {
  Engine& E = B.E;
  engine_setup(E, K, o);
  cudaStream_t s = E.stream;
  B.h_vbase.assign(K + 1, 0);
  B.h_ebase.assign(K + 1, 0);
  B.h_wbase.assign(K + 1, 0);
  for (int g = 0; g < K; ++g) {
    if (gs[g].n < 2 || gs[g].m < 0 || !gs[g].offsets || (gs[g].m > 0 && (!gs[g].adj || !gs[g].weights)))
      throw Error{VIECUT_EINVAL, "graph " + std::to_string(g) + ": n must be >= 2 and arrays non-null"};
    if (gs[g].offsets[0] != 0 || gs[g].offsets[gs[g].n] != gs[g].m)
      throw Error{VIECUT_EINVAL, "graph " + std::to_string(g) + ": offsets[0] != 0 or offsets[n] != m"};
    B.h_vbase[g + 1] = B.h_vbase[g] + gs[g].n;
    B.h_ebase[g + 1] = B.h_ebase[g] + gs[g].m;
    B.h_wbase[g + 1] = B.h_wbase[g] + (gs[g].n + 63) / 64;
  }
  const int64_t n_u = B.h_vbase[K], m_u = B.h_ebase[K];
  if (n_u > 0x7fffffffLL) throw Error{VIECUT_EINVAL, "the batch must hold fewer than 2^31 vertices"};
  int64_t* off = E.in_off.ensure_n<int64_t>(n_u + 1);
  int32_t* adj = E.in_adj.ensure_n<int32_t>(m_u);
  int32_t* w = E.in_w.ensure_n<int32_t>(m_u);
  for (int g = 0; g < K; ++g) {
    VC_CUDA(cudaMemcpyAsync(off + B.h_vbase[g], gs[g].offsets, sizeof(int64_t) * gs[g].n, cudaMemcpyHostToDevice, s));
    if (gs[g].m > 0) {
      VC_CUDA(cudaMemcpyAsync(adj + B.h_ebase[g], gs[g].adj, sizeof(int32_t) * gs[g].m, cudaMemcpyHostToDevice, s));
      VC_CUDA(cudaMemcpyAsync(w + B.h_ebase[g], gs[g].weights, sizeof(int32_t) * gs[g].m, cudaMemcpyHostToDevice, s));
    }
  }
  VC_CUDA(cudaMemcpyAsync(off + n_u, &m_u, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_vbase0.ensure_n<long long>(K + 1), B.h_vbase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_ebase.ensure_n<long long>(K + 1), B.h_ebase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_wbase.ensure_n<long long>(K + 1), B.h_wbase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  Workspace& W = *E.ws;
  int* err = &W.ctr()->changed;
  VC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  const int gridK = K < 4 * kSMs ? K : 4 * kSMs;
  if (o.validate >= 1) {
    b_validate_k<<<gridK, 256, 0, s>>>(K, B.d_vbase0.as<long long>(), B.d_ebase.as<long long>(), off, adj, w, err);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  b_rebase_k<<<gridK, 256, 0, s>>>(K, B.d_vbase0.as<long long>(), B.d_ebase.as<long long>(), off, adj);
  count_launch();
  VC_CHECK_LAUNCH();
  W.read_state();
  int bad = o.validate >= 1 ? W.h_counters->changed : (32 | 64);
  B.unit = (bad & 32) == 0;
  B.simple = (bad & 64) == 0;
  bad &= ~(32 | 64);
  if (bad) {
    std::string why;
    if (bad & 2) why += " offsets decrease or leave [0, m];";
    if (bad & 4) why += " neighbour id out of range;";
    if (bad & 8) why += " self-loop;";
    if (bad & 16) why += " weight < 1;";
    throw Error{VIECUT_EINVAL, "invalid graph in batch:" + why};
  }
  W.ensure_vertices(n_u);
  W.ensure_entries(m_u, n_u);
  E.gidA.ensure_n<int32_t>(n_u);
  E.gidB.ensure_n<int32_t>(n_u);
  E.vact.ensure_n<unsigned char>(n_u);
  E.om0.ensure_n<int32_t>(n_u);
  E.oc1.ensure_n<int32_t>(n_u);
  E.os1.ensure_n<unsigned char>(n_u);
  E.ocap = n_u;
  B.bits_out.ensure_n<unsigned long long>(B.h_wbase[K]);
  std::vector<long long> norig(K);
  for (int g = 0; g < K; ++g) norig[g] = gs[g].n;
  VC_CUDA(cudaMemcpyAsync(E.obase.p, B.h_vbase.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(E.norig.p, norig.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaStreamSynchronize(s));
}

static void batch_run(Batch& B, uint64_t seed, int lp_iters) {
  if (lp_iters < 0) throw Error{VIECUT_EINVAL, "lp_iters must be >= 0"};
  Engine& E = B.E;
  VC_CUDA(cudaSetDevice(E.device));
  cudaStream_t s = E.stream;
  E.ws->s = s;
  E.lp_iters = lp_iters;
  E.steps = 0;
  const unsigned long long launches0 = g_launches;
  cudaEvent_t e0, e1;
  VC_CUDA(cudaEventCreate(&e0));
  VC_CUDA(cudaEventCreate(&e1));
  VC_CUDA(cudaEventRecord(e0, s));
  const int K = E.K;
  const int64_t n_u = B.h_vbase[K], m_u = B.h_ebase[K];
  // every slot holds its graph of the input union
  E.G = GraphView();
  E.G.n = n_u;
  E.G.nnz = m_u;
  E.G.off = E.in_off.as<int64_t>();
  E.G.adj = E.in_adj.as<int32_t>();
  E.G.w = E.in_w.p;
  E.G.wbytes = 4;
  E.G.unit = B.unit;
  E.G.simple = B.simple;
  E.ws->bins_valid = false;
  E.slot = -1;
  E.gid = E.gidA.as<int32_t>();
  {
    std::vector<long long> nv(K), ne(K);
    std::vector<int> first(K, 8);
    std::vector<unsigned long long> sd(K, seed);
    for (int g = 0; g < K; ++g) {
      nv[g] = B.h_vbase[g + 1] - B.h_vbase[g];
      ne[g] = B.h_ebase[g + 1] - B.h_ebase[g];
    }
    VC_CUDA(cudaMemcpyAsync(E.vbase.p, B.d_vbase0.p, sizeof(long long) * K, cudaMemcpyDeviceToDevice, s));
    VC_CUDA(cudaMemcpyAsync(E.nv.p, nv.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
    VC_CUDA(cudaMemcpyAsync(E.nnz.p, ne.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
    VC_CUDA(cudaMemcpyAsync(E.first.p, first.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
    VC_CUDA(cudaMemcpyAsync(E.seed.p, sd.data(), sizeof(unsigned long long) * K, cudaMemcpyHostToDevice, s));
    VC_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  BState S = E.state();
  const int gridK = K < 4 * kSMs ? K : 4 * kSMs;
  b_gid_init_k<<<gridK, 256, 0, s>>>(K, S, E.gid);
  count_launch();
  engine_start_new(E);
  while (engine_step(E))
    if (E.steps > (int64_t)64 * (n_u + 16)) throw Error{VIECUT_ECUDA, "batch did not converge"};
  b_side_bits_k<<<gridK, 256, 0, s>>>(nullptr, K, S, B.d_wbase.as<long long>(), E.om0.as<int32_t>(),
                                      E.os1.as<unsigned char>(), E.oc1.as<int32_t>(), E.sideK.as<unsigned char>(),
                                      B.bits_out.as<unsigned long long>());
  count_launch();
  VC_CHECK_LAUNCH();
  VC_CUDA(cudaEventRecord(e1, s));
  VC_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  VC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  B.stats.ms_total = ms;
  B.stats.super_steps = E.steps;
  B.stats.kernel_launches = (int64_t)(g_launches - launches0);
  B.stats.graphs = K;
  B.stats.vertices = n_u;
  B.stats.entries = m_u;
}

static void copy_trace(Engine& E, int g, viecut_step* steps, int64_t cap, int64_t* len) {
  int tl = 0;
  VC_CUDA(cudaMemcpy(&tl, (int*)E.trace_len.p + g, sizeof(int), cudaMemcpyDeviceToHost));
  int cnt = tl < kBTraceCap ? tl : kBTraceCap;
  std::vector<TraceStep> t(cnt);
  if (cnt)
    VC_CUDA(cudaMemcpy(t.data(), (TraceStep*)E.trace.p + (int64_t)g * kBTraceCap, sizeof(TraceStep) * cnt,
                       cudaMemcpyDeviceToHost));
  *len = tl;
  for (int64_t i = 0; i < cap && i < cnt; ++i)
    steps[i] = viecut_step{t[i].kind, t[i].level, t[i].n, t[i].nnz, t[i].lambda_hat};
}

// ------------------------------------------------------------------ server
// Page-locked host blocks holding the requests that wait for the device, in
// power-of-two size classes reused across requests (pinning memory is slow, and a
// copy from pageable memory runs through the driver's own staging at a fraction of
// the bus rate).  Past `cap` pinned bytes a block comes from the ordinary heap.
struct HostPool {
  std::mutex mu;
  std::map<int, std::vector<void*>> free_blocks;
  std::vector<void*> pinned;
  int64_t pinned_bytes = 0, cap = int64_t(16) << 30;
  struct Block {
    void* p = nullptr;
    int cls = 0;
    bool is_pinned = false;
  };
  Block get(int64_t bytes) {
    int c = 20;
    while ((int64_t(1) << c) < bytes) ++c;
    std::lock_guard<std::mutex> lk(mu);
    auto& fl = free_blocks[c];
    if (!fl.empty()) {
      Block b{fl.back(), c, true};
      fl.pop_back();
      return b;
    }
    if (pinned_bytes + (int64_t(1) << c) <= cap) {
      void* p = nullptr;
      if (cudaMallocHost(&p, size_t(1) << c) == cudaSuccess) {
        pinned.push_back(p);
        pinned_bytes += int64_t(1) << c;
        return Block{p, c, true};
      }
      cudaGetLastError();
    }
    void* p = malloc(size_t(1) << c);
    if (!p) throw Error{VIECUT_ENOMEM, "host memory for a request"};
    return Block{p, c, false};
  }
  void put(Block& b) {
    if (!b.p) return;
    if (b.is_pinned) {
      std::lock_guard<std::mutex> lk(mu);
      free_blocks[b.cls].push_back(b.p);
    } else {
      free(b.p);
    }
    b.p = nullptr;
  }
  ~HostPool() {
    for (void* p : pinned) cudaFreeHost(p);
  }
};

// Copies a request's array into its page-locked block.  One core copies at about a
// tenth of what the host link carries (the device link of a Grace host reads pageable
// memory faster than one thread writes it), so large arrays are split over threads.
static void copy_parallel(void* dst, const void* src, size_t bytes) {
  constexpr size_t kPerThread = size_t(8) << 20;
  const size_t parts = std::min<size_t>(8, bytes / kPerThread);
  if (parts <= 1) {
    memcpy(dst, src, bytes);
    return;
  }
  const size_t per = (bytes + parts - 1) / parts;
  std::vector<std::thread> th;
  th.reserve(parts - 1);
  for (size_t i = 1; i < parts; ++i) {
    const size_t a = i * per, b = std::min(bytes, a + per);
    if (a < b) th.emplace_back([=] { memcpy((char*)dst + a, (const char*)src + a, b - a); });
  }
  memcpy(dst, src, std::min(per, bytes));
  for (auto& t : th) t.join();
}

// A request's copy of its graph lives in a host block until it reaches the device;
// its results (or the reason it was refused) are kept until the caller polls them.
struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, m = 0;
  uint64_t seed = 0;
  HostPool::Block blk;
  int64_t* off = nullptr;  // n + 1 entries
  int32_t* adj = nullptr;
  int32_t* w = nullptr;
  int err = 0;             // VIECUT_EINVAL once the device check refused the graph
  std::string err_msg;
  ~Request() {
    if (blk.p && !blk.is_pinned) free(blk.p);  // pinned blocks belong to the pool
  }
  int64_t est = 0;
  int slot = -1;
  int64_t obase = -1;
  std::chrono::steady_clock::time_point t_submit, t_start, t_done;
  int lane = 0;            // 0: the resident union, 1: the solo lane
  bool cancelled = false;  // viecut_server_cancel: the result is dropped
  bool done = false;
  int64_t cut = 0;
  std::vector<uint64_t> bits;
};

struct Server {
  Engine E;
  int64_t budget = 0;
  int lp_iters = 2;
  std::mutex mu;
  std::condition_variable cv;
  std::condition_variable cv_done;  // a request finished (viecut_server_wait)
  bool stopping = false;
  std::thread th;
  std::string error;  // set once the loop failed
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> tickets;
  std::vector<std::shared_ptr<Request>> slot_req;
  std::vector<int> free_slots;
  std::map<int64_t, int64_t> free_ranges;  // original-vertex arena: start -> length
  int64_t budget_used = 0;
  uint64_t next_ticket = 1;
  bool all_simple = true;
  int64_t admitted = 0, completed = 0, max_resident = 0, joins = 0;
  std::vector<int> h_phase;
  Buf d_join, d_list, d_wbase, d_bits, d_init, d_sgid, d_err;
  Buf st_off, st_adj, st_w;  // staging of joining graphs (grow-only)
  HostPool host;
  int64_t rejected = 0;
  int64_t cancelled = 0;
  int64_t failed = 0;  // requests answered with VIECUT_ENOMEM
  std::vector<long long> h_join;
  // solo lanes: requests of at least solo_min_n vertices (and, with solo_exact, those
  // whose whole run is the sequential exact step), each lane one request at a time on a
  // handle (and stream) of its own
  int64_t solo_min_n = 0;
  bool solo_exact = false;
  int64_t n0 = 10000;
  viecut_opts solo_opts{};
  std::deque<std::shared_ptr<Request>> solo_pending;
  std::condition_variable cv_solo;
  std::vector<std::thread> th_solo;
  int64_t solo_completed = 0;
};

static int64_t request_estimate(int64_t n, int64_t m) {
  // union CSR + workspace share per entry and per vertex (see DESIGN: memory layout)
  return 96 * (m + n) + 112 * n + (1 << 16);
}

static int64_t arena_alloc(Server& S, int64_t n) {
  for (;;) {
    for (auto it = S.free_ranges.begin(); it != S.free_ranges.end(); ++it) {
      if (it->second >= n) {
        const int64_t at = it->first, len = it->second;
        S.free_ranges.erase(it);
        if (len > n) S.free_ranges[at + n] = len - n;
        return at;
      }
    }
    Engine& E = S.E;
    const int64_t old = E.ocap, cap = std::max<int64_t>(2 * old, old + n);
    grow_keep(E.om0, sizeof(int32_t) * cap, sizeof(int32_t) * old, E.stream);
    grow_keep(E.oc1, sizeof(int32_t) * cap, sizeof(int32_t) * old, E.stream);
    grow_keep(E.os1, cap, old, E.stream);
    E.ocap = cap;
    // merge the new tail with a free range ending at the old capacity
    int64_t start = old, len = cap - old;
    auto it = S.free_ranges.lower_bound(old);
    if (it != S.free_ranges.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == old) { start = pv->first; len += pv->second; S.free_ranges.erase(pv); }
    }
    S.free_ranges[start] = len;
  }
}

static void arena_free(Server& S, int64_t at, int64_t n) {
  auto it = S.free_ranges.emplace(at, n).first;
  auto nx = std::next(it);
  if (nx != S.free_ranges.end() && at + n == nx->first) { it->second += nx->second; S.free_ranges.erase(nx); }
  if (it != S.free_ranges.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) { pv->second += it->second; S.free_ranges.erase(it); }
  }
}

static std::string invalid_reason(int bad) {
  std::string why = "invalid graph:";
  if (bad & 2) why += " offsets decrease or leave [0, m];";
  if (bad & 4) why += " neighbour id out of range;";
  if (bad & 8) why += " self-loop;";
  if (bad & 16) why += " weight < 1;";
  return why;
}

// Marks a request as refused (VIECUT_EINVAL: its graph failed the device check;
// VIECUT_ENOMEM: its admission could not get device memory) and gives back what
// admission took (under S.mu).
static void refuse(Server& S, const std::shared_ptr<Request>& r, const std::string& why, int code = VIECUT_EINVAL) {
  r->err = code;
  r->err_msg = why;
  r->t_done = std::chrono::steady_clock::now();
  r->done = true;
  S.host.put(r->blk);
  S.budget_used -= r->est;
  if (code == VIECUT_ENOMEM) S.failed += 1;
  else S.rejected += 1;
  S.completed += 1;
  S.cv_done.notify_all();
}

// A join whose device memory could not be had: its requests are answered with
// VIECUT_ENOMEM and their slots and arena ranges given back; the resident graphs are
// untouched (every allocation of a join comes before any change to them).
static void fail_join(Server& S, std::vector<std::shared_ptr<Request>>& add, const std::string& why) {
  std::lock_guard<std::mutex> lk(S.mu);
  for (auto& r : add) {
    if (r->obase >= 0) {
      arena_free(S, r->obase, r->n);
      r->obase = -1;
    }
    S.slot_req[r->slot].reset();
    S.free_slots.push_back(r->slot);
    refuse(S, r, why, VIECUT_ENOMEM);
  }
  add.clear();
}

// Copies the admitted requests to the device, checks them there (a refused request is
// answered with its reason and leaves the join), and appends the others to the union
// (a new union in the other coarse buffer: the old union first, unchanged, then the
// new graphs) and starts their state.
static void server_join(Server& S, std::vector<std::shared_ptr<Request>>& add) {
  Engine& E = S.E;
  Workspace& W = *E.ws;
  cudaStream_t s = E.stream;
  int J = (int)add.size();
  // staged host copies -> device (request-local offsets, n per request)
  std::vector<long long> sv(J + 1, 0), se(J + 1, 0);
  for (int j = 0; j < J; ++j) {
    sv[j + 1] = sv[j] + add[j]->n;
    se[j + 1] = se[j] + add[j]->m;
  }
  const int64_t sn = sv[J], sm = se[J];
  int64_t* d_off;
  int32_t *d_adj, *d_w, *sgid;
  long long* dsv;
  int* derr;
  try {
    d_off = S.st_off.ensure_n<int64_t>(sn);
    d_adj = S.st_adj.ensure_n<int32_t>(std::max<int64_t>(sm, 1));
    d_w = S.st_w.ensure_n<int32_t>(std::max<int64_t>(sm, 1));
    dsv = S.d_join.ensure_n<long long>(6 * (J + 1));
    sgid = S.d_sgid.ensure_n<int32_t>(std::max<int64_t>(sn, 1));
    derr = S.d_err.ensure_n<int>(J);
  } catch (const Error& e) {
    if (e.code != VIECUT_ENOMEM) throw;
    fail_join(S, add, e.msg);
    return;
  }
  for (int j = 0; j < J; ++j) {
    const auto& r = add[j];
    VC_CUDA(cudaMemcpyAsync(d_off + sv[j], r->off, sizeof(int64_t) * r->n, cudaMemcpyHostToDevice, s));
    if (r->m > 0) {
      VC_CUDA(cudaMemcpyAsync(d_adj + se[j], r->adj, sizeof(int32_t) * r->m, cudaMemcpyHostToDevice, s));
      VC_CUDA(cudaMemcpyAsync(d_w + se[j], r->w, sizeof(int32_t) * r->m, cudaMemcpyHostToDevice, s));
    }
  }
  VC_CUDA(cudaMemcpyAsync(dsv, sv.data(), sizeof(long long) * (J + 1), cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(dsv + (J + 1), se.data(), sizeof(long long) * (J + 1), cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * J, s));
  b_stage_gid_k<<<J < 4 * kSMs ? J : 4 * kSMs, 256, 0, s>>>(J, dsv, sgid);
  b_validate_staged_k<<<grid_for(sn, 8, kSMs * 16), 256, 0, s>>>(sn, sgid, dsv, dsv + (J + 1), d_off, d_adj, d_w,
                                                                 derr);
  count_launch(2);
  VC_CHECK_LAUNCH();
  std::vector<int> herr(J);
  VC_CUDA(cudaMemcpyAsync(herr.data(), derr, sizeof(int) * J, cudaMemcpyDeviceToHost, s));
  VC_CUDA(cudaStreamSynchronize(s));
  // the host blocks are free once the copies are done
  std::vector<std::shared_ptr<Request>> keep;
  std::vector<int> kj;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    for (int j = 0; j < J; ++j) {
      S.host.put(add[j]->blk);
      if (herr[j] & ~(32 | 64)) {
        S.slot_req[add[j]->slot].reset();
        S.free_slots.push_back(add[j]->slot);
        refuse(S, add[j], invalid_reason(herr[j]));
      } else {
        keep.push_back(add[j]);
        kj.push_back(j);
      }
    }
  }
  add.swap(keep);
  J = (int)add.size();
  if (J == 0) return;
  const int64_t n_u = E.G.n;
  int64_t m_u = 0;  // exact entry count of the resident union: its last offset
  if (n_u > 0) {
    VC_CUDA(cudaMemcpyAsync(&m_u, E.G.off + n_u, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    VC_CUDA(cudaStreamSynchronize(s));
  }
  int64_t kn = 0, km = 0;
  for (auto& r : add) { kn += r->n; km += r->m; }
  const int64_t n_new = n_u + kn, m_new = m_u + km;
  const int dst = E.slot == 0 ? 1 : 0;
  const bool onA = E.gid == E.gidA.as<int32_t>() || E.gid == nullptr;
  Buf& cur = onA ? E.gidA : E.gidB;
  Buf& alt = onA ? E.gidB : E.gidA;
  int64_t* off;
  int32_t* adj;
  long long* w;
  // every allocation of the join before any change to the resident graphs
  try {
    if (n_new > 0x7fffffffLL) throw Error{VIECUT_ENOMEM, "the resident graphs would exceed 2^31 vertices"};
    for (auto& r : add) r->obase = arena_alloc(S, r->n);
    S.d_join.ensure_n<long long>(6 * (J + 1));
    off = W.coff[dst].ensure_n<int64_t>(n_new + 1);
    adj = W.cadj[dst].ensure_n<int32_t>(std::max<int64_t>(m_new, 1));
    w = W.cw[dst].ensure_n<long long>(std::max<int64_t>(m_new, 1));
    grow_keep(cur, sizeof(int32_t) * std::max<int64_t>(n_new, 1), sizeof(int32_t) * n_u, s);
    E.gid = cur.as<int32_t>();
    alt.ensure_n<int32_t>(n_new);
    S.d_init.ensure(sizeof(SlotInit) * J);
    W.ensure_vertices(n_new);
    W.ensure_entries(m_new, n_new);
    E.vact.ensure_n<unsigned char>(n_new);
  } catch (const Error& e) {
    if (e.code != VIECUT_ENOMEM) throw;
    fail_join(S, add, e.msg);
    return;
  }
  // per kept request: union vertex and entry base, staged vertex and entry base, n, m
  S.h_join.assign(6 * (J + 1), 0);
  long long* jv = S.h_join.data();
  long long* je = jv + (J + 1);
  long long* ksv = je + (J + 1);
  long long* kse = ksv + (J + 1);
  long long* kn_ = kse + (J + 1);
  long long* km_ = kn_ + (J + 1);
  long long at_v = n_u, at_e = m_u;
  for (int i = 0; i < J; ++i) {
    jv[i] = at_v;
    je[i] = at_e;
    ksv[i] = sv[kj[i]];
    kse[i] = se[kj[i]];
    kn_[i] = add[i]->n;
    km_[i] = add[i]->m;
    at_v += add[i]->n;
    at_e += add[i]->m;
  }
  long long* dj = S.d_join.as<long long>();  // the checks above are done with it
  VC_CUDA(cudaMemcpyAsync(dj, jv, sizeof(long long) * 6 * (J + 1), cudaMemcpyHostToDevice, s));
  if (n_u > 0) {
    VC_CUDA(cudaMemcpyAsync(off, E.G.off, sizeof(int64_t) * n_u, cudaMemcpyDeviceToDevice, s));
    VC_CUDA(cudaMemcpyAsync(adj, E.G.adj, sizeof(int32_t) * m_u, cudaMemcpyDeviceToDevice, s));
    VC_CUDA(cudaMemcpyAsync(w, E.G.w, sizeof(long long) * m_u, cudaMemcpyDeviceToDevice, s));
  }
  long long* d6 = dj;
  b_join_k<<<J < 4 * kSMs ? J : 4 * kSMs, 256, 0, s>>>(J, d6, d6 + (J + 1), d6 + 2 * (J + 1), d6 + 3 * (J + 1),
                                                      d6 + 4 * (J + 1), d6 + 5 * (J + 1), d_off, d_adj, d_w, off,
                                                      adj, w);
  b_set_i64_k<<<1, 1, 0, s>>>(off + n_new, m_new);
  count_launch(2);
  VC_CHECK_LAUNCH();
  // slot records
  std::vector<SlotInit> init(J);
  for (int j = 0; j < J; ++j)
    init[j] = SlotInit{add[j]->slot, 0, jv[j], add[j]->n, add[j]->m, add[j]->obase, add[j]->seed};
  SlotInit* di = (SlotInit*)S.d_init.p;
  VC_CUDA(cudaMemcpyAsync(di, init.data(), sizeof(SlotInit) * J, cudaMemcpyHostToDevice, s));
  BState B = E.state();
  b_slot_init_k<<<(J + 255) / 256, 256, 0, s>>>(J, di, B);
  const int K = E.K, gridK = K < 4 * kSMs ? K : 4 * kSMs;
  b_gid_init_k<<<gridK, 256, 0, s>>>(K, B, E.gid);
  count_launch(2);
  VC_CHECK_LAUNCH();
  for (int i = 0; i < J; ++i) S.all_simple = S.all_simple && !(herr[kj[i]] & 64);
  E.G = GraphView();
  E.G.n = n_new;
  E.G.nnz = m_new;
  E.G.off = off;
  E.G.adj = adj;
  E.G.w = w;
  E.G.wbytes = 8;
  E.G.simple = S.all_simple;
  E.slot = dst;
  W.bins_valid = false;
  engine_start_new(E);
  VC_CUDA(cudaStreamSynchronize(s));
  S.joins += 1;
}

// Reads out every slot whose graph finished in the last super-step.
static void server_collect(Server& S) {
  Engine& E = S.E;
  cudaStream_t s = E.stream;
  const int K = E.K;
  S.h_phase.resize(K);
  VC_CUDA(cudaMemcpyAsync(S.h_phase.data(), E.phase.p, sizeof(int) * K, cudaMemcpyDeviceToHost, s));
  VC_CUDA(cudaStreamSynchronize(s));
  std::vector<int> fin;
  for (int g = 0; g < K; ++g)
    if (S.slot_req[g] && S.h_phase[g] == kBGone) fin.push_back(g);
  if (fin.empty()) return;
  const int F = (int)fin.size();
  std::vector<long long> wb(F + 1, 0);
  for (int i = 0; i < F; ++i) wb[i + 1] = wb[i] + (S.slot_req[fin[i]]->n + 63) / 64;
  int32_t* dl = S.d_list.ensure_n<int32_t>(F);
  long long* dw = S.d_wbase.ensure_n<long long>(F + 1);
  unsigned long long* db = S.d_bits.ensure_n<unsigned long long>(wb[F]);
  VC_CUDA(cudaMemcpyAsync(dl, fin.data(), sizeof(int32_t) * F, cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(dw, wb.data(), sizeof(long long) * (F + 1), cudaMemcpyHostToDevice, s));
  BState B = E.state();
  b_side_bits_k<<<F < 4 * kSMs ? F : 4 * kSMs, 256, 0, s>>>(dl, F, B, dw, E.om0.as<int32_t>(), E.os1.as<unsigned char>(),
                                                           E.oc1.as<int32_t>(), E.sideK.as<unsigned char>(), db);
  count_launch();
  VC_CHECK_LAUNCH();
  std::vector<uint64_t> bits(wb[F]);
  std::vector<long long> lam(K);
  VC_CUDA(cudaMemcpyAsync(bits.data(), db, sizeof(uint64_t) * wb[F], cudaMemcpyDeviceToHost, s));
  VC_CUDA(cudaMemcpyAsync(lam.data(), E.lam.p, sizeof(long long) * K, cudaMemcpyDeviceToHost, s));
  VC_CUDA(cudaStreamSynchronize(s));
  const auto now = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(S.mu);
  for (int i = 0; i < F; ++i) {
    auto r = S.slot_req[fin[i]];
    r->cut = lam[fin[i]];
    r->bits.assign(bits.begin() + wb[i], bits.begin() + wb[i + 1]);
    r->t_done = now;
    r->done = true;
    arena_free(S, r->obase, r->n);
    S.budget_used -= r->est;
    S.free_slots.push_back(fin[i]);
    S.slot_req[fin[i]].reset();
    S.completed += 1;
  }
  S.cv_solo.notify_one();  // budget came free
  S.cv_done.notify_all();
}

static void server_loop(Server& S) {
  Engine& E = S.E;
  try {
    VC_CUDA(cudaSetDevice(E.device));
    for (;;) {
      std::vector<std::shared_ptr<Request>> add;
      int resident = 0;
      {
        std::unique_lock<std::mutex> lk(S.mu);
        if (S.stopping) break;
        while (!S.pending.empty() && !S.free_slots.empty() && S.budget_used + S.pending.front()->est <= S.budget) {
          auto r = S.pending.front();
          S.pending.pop_front();
          r->slot = S.free_slots.back();
          S.free_slots.pop_back();
          S.budget_used += r->est;
          S.slot_req[r->slot] = r;
          r->t_start = std::chrono::steady_clock::now();
          add.push_back(r);
          S.admitted += 1;
        }
        for (auto& x : S.slot_req) resident += x ? 1 : 0;
        S.max_resident = std::max<int64_t>(S.max_resident, resident);
        if (add.empty() && resident == 0) {
          S.cv.wait_for(lk, std::chrono::milliseconds(20));
          continue;
        }
      }
      if (!add.empty()) server_join(S, add);
      engine_step(E);
      server_collect(S);
    }
  } catch (const Error& e) {
    std::lock_guard<std::mutex> lk(S.mu);
    S.error = e.msg.empty() ? "server failed" : e.msg;
  }
}

static void solo_check(int rc) {
  if (rc != VIECUT_OK) throw Error{rc, viecut_last_error()};
}

// The solo lane: takes the large requests in arrival order (each within the shared
// memory budget) and runs each alone through a reusable single-graph handle, whose
// load checks the graph on the device (a refused graph is answered with the reason).
static void solo_loop(Server& S) {
  viecut_t* h = nullptr;
  try {
    VC_CUDA(cudaSetDevice(S.E.device));
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(S.mu);
        S.cv_solo.wait(lk, [&] {
          return S.stopping || (!S.solo_pending.empty() && S.budget_used + S.solo_pending.front()->est <= S.budget);
        });
        if (S.stopping) break;
        r = S.solo_pending.front();
        S.solo_pending.pop_front();
        S.budget_used += r->est;
        S.admitted += 1;
        r->t_start = std::chrono::steady_clock::now();
        r->lane = 1;
      }
      int rc = h ? viecut_load(h, r->off, r->adj, r->n, r->m, r->w)
                 : viecut_create(&h, r->off, r->adj, r->n, r->m, r->w, &S.solo_opts);
      if (rc == VIECUT_EINVAL || rc == VIECUT_ENOMEM) {
        // a refused graph, or no device memory for it: this request fails, the lane goes on
        // (a handle whose load failed holds no graph until the next load)
        const std::string why = viecut_last_error();
        std::lock_guard<std::mutex> lk(S.mu);
        refuse(S, r, why, rc);
        S.cv.notify_one();
        continue;
      }
      solo_check(rc);
      S.host.put(r->blk);  // the graph is on the device now
      int64_t cut = 0;
      std::vector<uint64_t> bits((r->n + 63) / 64);
      rc = viecut_run(h, r->seed, S.lp_iters, &cut, bits.data());
      if (rc == VIECUT_ENOMEM) {
        const std::string why = viecut_last_error();
        std::lock_guard<std::mutex> lk(S.mu);
        refuse(S, r, why, rc);
        S.cv.notify_one();
        continue;
      }
      solo_check(rc);
      const auto now = std::chrono::steady_clock::now();
      {
        std::lock_guard<std::mutex> lk(S.mu);
        r->cut = cut;
        r->bits.swap(bits);
        r->t_done = now;
        r->done = true;
        S.budget_used -= r->est;
        S.completed += 1;
        S.solo_completed += 1;
      }
      S.cv_done.notify_all();
      S.cv.notify_one();  // budget came free for the union
    }
  } catch (const Error& e) {
    std::lock_guard<std::mutex> lk(S.mu);
    S.error = e.msg.empty() ? "server solo lane failed" : e.msg;
  }
  if (h) viecut_destroy(h);
}

}  // namespace vc
struct viecut_batch {
  vc::Batch b;
};

using vc::Error;

extern "C" {

int viecut_batch_create(viecut_batch** out, const viecut_graph_desc* graphs, int32_t k, const viecut_opts* opts) {
  VC_API_BEGIN
  if (!out || !graphs || k < 1) throw Error{VIECUT_EINVAL, "need at least one graph"};
  *out = nullptr;
  viecut_opts o;
  viecut_opts_init(&o);
  if (opts) o = *opts;
  if (o.n0 < 1 || o.pr_runs_max < 0) throw Error{VIECUT_EINVAL, "bad options"};
  if (o.correct) throw Error{VIECUT_EINVAL, "correct: the correcting step runs on single-graph handles only"};
  if (o.lp_converge) throw Error{VIECUT_EINVAL, "lp_converge: the convergence stop runs on single-graph handles only"};
  if (o.lp_async) throw Error{VIECUT_EINVAL, "lp_async: asynchronous rounds run on single-graph handles only"};
  auto* x = new viecut_batch;
  try {
    vc::batch_create(x->b, graphs, k, o);
  } catch (...) {
    delete x;
    throw;
  }
  *out = x;
  VC_API_END
}

int viecut_batch_run(viecut_batch* bt, uint64_t seed, int32_t lp_iters, int64_t* cut_values, uint64_t* side_bits) {
  VC_API_BEGIN
  if (!bt || !cut_values) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Batch& B = bt->b;
  vc::batch_run(B, seed, lp_iters);
  VC_CUDA(cudaMemcpyAsync(cut_values, B.E.lam.p, sizeof(int64_t) * B.E.K, cudaMemcpyDeviceToHost, B.E.stream));
  if (side_bits)
    VC_CUDA(cudaMemcpyAsync(side_bits, B.bits_out.p, sizeof(uint64_t) * B.h_wbase[B.E.K], cudaMemcpyDeviceToHost,
                            B.E.stream));
  VC_CUDA(cudaStreamSynchronize(B.E.stream));
  VC_API_END
}

int viecut_batch_side_words(const viecut_batch* bt, int64_t* words) {
  VC_API_BEGIN
  if (!bt || !words) throw Error{VIECUT_EINVAL, "null argument"};
  *words = bt->b.h_wbase[bt->b.E.K];
  VC_API_END
}

int viecut_batch_get_trace(const viecut_batch* bt, int32_t g, viecut_step* steps, int64_t cap, int64_t* len) {
  VC_API_BEGIN
  if (!bt || !len || g < 0 || g >= bt->b.E.K) throw Error{VIECUT_EINVAL, "bad graph index"};
  vc::Engine& E = const_cast<viecut_batch*>(bt)->b.E;
  VC_CUDA(cudaSetDevice(E.device));
  vc::copy_trace(E, g, steps, cap, len);
  VC_API_END
}

int viecut_batch_get_stats(const viecut_batch* bt, viecut_batch_stats* st) {
  VC_API_BEGIN
  if (!bt || !st) throw Error{VIECUT_EINVAL, "null argument"};
  *st = bt->b.stats;
  VC_API_END
}

int viecut_batch_destroy(viecut_batch* bt) {
  VC_API_BEGIN
  if (!bt) return VIECUT_OK;
  cudaSetDevice(bt->b.E.device);
  if (bt->b.E.stream) cudaStreamSynchronize(bt->b.E.stream);
  delete bt;
  VC_API_END
}


struct viecut_server {
  vc::Server s;
};

int viecut_server_opts_init(viecut_server_opts* o) {
  if (!o) return VIECUT_EINVAL;
  memset(o, 0, sizeof(*o));
  viecut_opts_init(&o->base);
  o->hbm_budget_bytes = (int64_t)120 << 30;
  o->max_slots = 1024;
  o->lp_iters = 2;
  o->solo_min_n = 65536;
  o->solo_lanes = 8;
  o->solo_exact = 1;
  return VIECUT_OK;
}

int viecut_server_start(viecut_server** out, const viecut_server_opts* opts) {
  VC_API_BEGIN
  if (!out) throw Error{VIECUT_EINVAL, "null server pointer"};
  *out = nullptr;
  viecut_server_opts o;
  viecut_server_opts_init(&o);
  if (opts) o = *opts;
  if (o.max_slots < 1 || o.hbm_budget_bytes < 1 || o.lp_iters < 0 || o.base.n0 < 1 || o.base.pr_runs_max < 0 ||
      o.solo_min_n < 0 || o.solo_lanes < 1 || o.solo_lanes > 64 || (o.solo_exact != 0 && o.solo_exact != 1))
    throw Error{VIECUT_EINVAL, "bad server options"};
  if (o.base.correct) throw Error{VIECUT_EINVAL, "correct: the correcting step runs on single-graph handles only"};
  if (o.base.lp_converge)
    throw Error{VIECUT_EINVAL, "lp_converge: the convergence stop runs on single-graph handles only"};
  if (o.base.lp_async) throw Error{VIECUT_EINVAL, "lp_async: asynchronous rounds run on single-graph handles only"};
  auto* x = new viecut_server;
  try {
    vc::Server& S = x->s;
    vc::engine_setup(S.E, o.max_slots, o.base);
    S.E.lp_iters = o.lp_iters;
    S.lp_iters = o.lp_iters;
    S.budget = o.hbm_budget_bytes;
    S.slot_req.assign(o.max_slots, nullptr);
    for (int g = o.max_slots - 1; g >= 0; --g) S.free_slots.push_back(g);
    S.solo_min_n = o.solo_min_n;
    S.solo_opts = o.base;
    S.solo_opts.stream = nullptr;  // a stream of its own, beside the union's
    S.solo_opts.validate = 1;      // already checked on submit; the device pass finds unit / simple
    S.solo_opts.timing = 0;
    S.th = std::thread(vc::server_loop, std::ref(S));
    S.solo_exact = o.solo_exact != 0;
    S.n0 = o.base.n0;
    if (S.solo_min_n > 0)
      for (int i = 0; i < o.solo_lanes; ++i) S.th_solo.emplace_back(vc::solo_loop, std::ref(S));
  } catch (...) {
    delete x;
    throw;
  }
  *out = x;
  VC_API_END
}

int viecut_server_submit(viecut_server* sv, const viecut_graph_desc* g, uint64_t seed, uint64_t* ticket) {
  VC_API_BEGIN
  if (!sv || !g || !ticket) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Server& S = sv->s;
  const int64_t n = g->n, m = g->m;
  if (n < 2 || m < 0 || !g->offsets || (m > 0 && (!g->adj || !g->weights)))
    throw Error{VIECUT_EINVAL, "graph: n must be >= 2 and arrays non-null"};
  if (g->offsets[0] != 0 || g->offsets[n] != m) throw Error{VIECUT_EINVAL, "graph: offsets[0] != 0 or offsets[n] != m"};
  auto r = std::make_shared<vc::Request>();
  r->n = n;
  r->m = m;
  r->seed = seed;
  r->est = vc::request_estimate(n, m);
  if (r->est > S.budget) throw Error{VIECUT_EINVAL, "graph needs more than the server's memory budget"};
  // one copy into a page-locked block; the per-entry checks run on the device
  const size_t b_off = sizeof(int64_t) * (n + 1), b_adj = sizeof(int32_t) * m;
  r->blk = S.host.get((int64_t)(b_off + 2 * b_adj));
  r->off = (int64_t*)r->blk.p;
  r->adj = (int32_t*)((char*)r->blk.p + b_off);
  r->w = (int32_t*)((char*)r->blk.p + b_off + b_adj);
  vc::copy_parallel(r->off, g->offsets, b_off);
  if (m > 0) {
    vc::copy_parallel(r->adj, g->adj, b_adj);
    vc::copy_parallel(r->w, g->weights, b_adj);
  }
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (!S.error.empty()) throw Error{VIECUT_ECUDA, S.error};
    r->ticket = S.next_ticket++;
    S.tickets[r->ticket] = r;
    // large graphs, and (solo_exact) graphs that go straight to the sequential exact step,
    // run alone: in the lock-step union a long exact-step scan would hold every graph back
    const bool solo = S.solo_min_n > 0 && (n >= S.solo_min_n || (S.solo_exact && n > vc::kDenseMax && n <= S.n0));
    if (solo) S.solo_pending.push_back(r);
    else S.pending.push_back(r);
  }
  S.cv.notify_one();
  S.cv_solo.notify_one();
  *ticket = r->ticket;
  VC_API_END
}

namespace {
// Hands a finished request's result out (and forgets the ticket), or says why not:
// EBUSY while it runs, the request's own error, ECANCELLED after viecut_server_cancel.
// timeout_ms < 0: no wait; otherwise waits up to that long (ETIMEOUT after it).
int take_result(viecut_server* sv, uint64_t ticket, double timeout_ms, int64_t* cut, uint64_t* side_bits,
                viecut_request_info* info) {
  if (!sv) throw Error{VIECUT_EINVAL, "null server"};
  vc::Server& S = sv->s;
  std::shared_ptr<vc::Request> r;
  {
    std::unique_lock<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) throw Error{VIECUT_EINVAL, "unknown ticket"};
    r = it->second;
    if (!r->done && timeout_ms >= 0) {
      S.cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms),
                         [&] { return r->done || !S.error.empty() || S.stopping; });
    }
    if (!r->done) {
      if (!S.error.empty()) throw Error{VIECUT_ECUDA, S.error};
      if (timeout_ms >= 0) throw Error{VIECUT_ETIMEOUT, "request not finished within the timeout"};
      return VIECUT_EBUSY;
    }
    S.tickets.erase(ticket);
  }
  if (r->cancelled) throw Error{VIECUT_ECANCELLED, "request cancelled"};
  if (r->err) throw Error{r->err, r->err_msg};
  if (cut) *cut = r->cut;
  if (side_bits && !r->bits.empty()) memcpy(side_bits, r->bits.data(), sizeof(uint64_t) * r->bits.size());
  if (info) {
    auto ms = [](std::chrono::steady_clock::duration d) { return std::chrono::duration<double, std::milli>(d).count(); };
    info->latency_ms = ms(r->t_done - r->t_submit);
    info->queue_ms = ms(r->t_start - r->t_submit);
    info->run_ms = ms(r->t_done - r->t_start);
    info->lane = r->lane;
    info->n = r->n;
    info->m = r->m;
  }
  return VIECUT_OK;
}
}  // namespace

int viecut_server_poll(viecut_server* sv, uint64_t ticket, int64_t* cut, uint64_t* side_bits, double* latency_ms) {
  VC_API_BEGIN
  viecut_request_info info{};
  const int rc = take_result(sv, ticket, -1.0, cut, side_bits, &info);
  if (rc != VIECUT_OK) return rc;
  if (latency_ms) *latency_ms = info.latency_ms;
  VC_API_END
}

int viecut_server_poll_info(viecut_server* sv, uint64_t ticket, int64_t* cut, uint64_t* side_bits,
                            viecut_request_info* info) {
  VC_API_BEGIN
  const int rc = take_result(sv, ticket, -1.0, cut, side_bits, info);
  if (rc != VIECUT_OK) return rc;
  VC_API_END
}

int viecut_server_wait(viecut_server* sv, uint64_t ticket, double timeout_ms, int64_t* cut, uint64_t* side_bits,
                       viecut_request_info* info) {
  VC_API_BEGIN
  if (!(timeout_ms >= 0)) throw Error{VIECUT_EINVAL, "timeout_ms must be >= 0"};
  const int rc = take_result(sv, ticket, timeout_ms, cut, side_bits, info);
  if (rc != VIECUT_OK) return rc;
  VC_API_END
}

int viecut_server_cancel(viecut_server* sv, uint64_t ticket) {
  VC_API_BEGIN
  if (!sv) throw Error{VIECUT_EINVAL, "null server"};
  vc::Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.tickets.find(ticket);
  if (it == S.tickets.end()) throw Error{VIECUT_EINVAL, "unknown ticket"};
  auto r = it->second;
  if (r->cancelled) return VIECUT_OK;
  r->cancelled = true;
  S.cancelled += 1;
  // still queued: it leaves the queue at once and never runs
  for (auto* q : {&S.pending, &S.solo_pending}) {
    for (auto qi = q->begin(); qi != q->end(); ++qi) {
      if (qi->get() == r.get()) {
        q->erase(qi);
        r->t_start = r->t_done = std::chrono::steady_clock::now();
        r->done = true;
        S.host.put(r->blk);
        S.completed += 1;
        S.cv_done.notify_all();
        return VIECUT_OK;
      }
    }
  }
  VC_API_END
}

int viecut_server_get_stats(viecut_server* sv, viecut_server_stats* st) {
  VC_API_BEGIN
  if (!sv || !st) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Server& S = sv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  st->admitted = S.admitted;
  st->completed = S.completed;
  st->pending = (int64_t)(S.pending.size() + S.solo_pending.size());
  st->max_resident = S.max_resident;
  st->super_steps = S.E.steps;
  st->joins = S.joins;
  st->budget_used = S.budget_used;
  st->solo_completed = S.solo_completed;
  st->rejected = S.rejected;
  st->cancelled = S.cancelled;
  st->failed = S.failed;
  VC_API_END
}

int viecut_server_stop(viecut_server* sv) {
  VC_API_BEGIN
  if (!sv) return VIECUT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->s.mu);
    sv->s.stopping = true;
  }
  sv->s.cv.notify_all();
  sv->s.cv_solo.notify_all();
  sv->s.cv_done.notify_all();
  if (sv->s.th.joinable()) sv->s.th.join();
  for (auto& t : sv->s.th_solo)
    if (t.joinable()) t.join();
  cudaSetDevice(sv->s.E.device);
  if (sv->s.E.stream) cudaStreamSynchronize(sv->s.E.stream);
  delete sv;
  VC_API_END
}

}  // extern "C"
