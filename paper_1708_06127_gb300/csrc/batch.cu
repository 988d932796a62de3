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

#include <numeric>

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
  unsigned long long* gkey;
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

__global__ void b_gid_init_k(int K, const long long* vbase, int32_t* gid) {
  for (int g = blockIdx.x; g < K; g += gridDim.x)
    for (long long v = vbase[g] + threadIdx.x; v < vbase[g + 1]; v += blockDim.x) gid[v] = g;
}

// ---------------------------------------------------------------- per-graph steps
// minimum degree with smallest argmin over each graph's range; mode 0 = initial
// bound, mode 1 = update of the graphs that contracted (did[g])
__global__ void b_segmin_k(int K, const long long* __restrict__ deg, BState S, int mode) {
  __shared__ long long sd[8], sv[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
    if (mode == 1 && (!S.did[g] || S.nv[g] <= 1)) continue;
    if (mode == 0 && S.nv[g] < 1) continue;
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

// initial phase of every graph (after the initial bound)
__global__ void b_init_k(int K, BState S, long long n0) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    S.level[g] = 0;
    S.run[g] = 0;
    S.any[g] = 0;
    S.trace_len[g] = 0;
    S.contracted[g] = 0;
    S.n1[g] = 0;
    S.first[g] = 0;
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
      const long long vb = S.vbase[g], nb = S.vbase_new[g], n = S.norig[g], c = S.nv[g];
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
__global__ void b_prepare_k(int K, BState S, int ph, uint64_t seed) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const bool a = S.phase[g] == ph;
    S.gact[g] = a ? 1 : 0;
    if (ph == kBLP) S.gkey[g] = level_key(seed, S.level[g]);
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

// new vertex ranges after a union contraction: the coarse base of graph g is the rank
// of its first vertex's id among the kept labels (exclusive scan of the flags)
__global__ void b_shape_k(int K, BState S, int64_t n_old, int64_t c_total, const int32_t* __restrict__ rank,
                          const int64_t* __restrict__ coff) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= K; g += gridDim.x * blockDim.x) {
    const long long vb = S.vbase[g];
    S.vbase_new[g] = vb < n_old ? (long long)rank[vb] : c_total;
  }
}

__global__ void b_shape2_k(int K, BState S, const int64_t* __restrict__ coff) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < K; g += gridDim.x * blockDim.x) {
    const long long a = S.vbase_new[g], b = S.vbase_new[g + 1];
    S.nv[g] = b - a;
    S.nnz[g] = coff[b] - coff[a];
  }
}

__global__ void b_gid_update_k(int64_t n, const int32_t* __restrict__ cid, const int32_t* __restrict__ gid,
                               int32_t* gid_new) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cid[v];
    if (c >= 0) gid_new[c] = gid[v];
  }
}

__global__ void b_copy_vbase_k(int K, BState S) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= K; g += gridDim.x * blockDim.x) S.vbase[g] = S.vbase_new[g];
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

// final side bitmaps: words of graph g start at wbase[g]
__global__ void b_side_bits_k(int K, BState S, const long long* __restrict__ wbase, const int32_t* __restrict__ map0,
                              const unsigned char* __restrict__ side1, const int32_t* __restrict__ cur1,
                              const unsigned char* __restrict__ sideK, unsigned long long* bits) {
  for (int g = blockIdx.x; g < K; g += gridDim.x) {
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
      bits[wbase[g] + wd] = x;
    }
  }
}

// ------------------------------------------------------------------ host side
struct Batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int K = 0;
  int64_t n_u = 0, m_u = 0;
  int64_t n0 = 10000;
  int pr_runs_max = 8;
  bool unit = false, simple = false;
  std::vector<int64_t> h_vbase, h_ebase, h_wbase;
  Buf in_off, in_adj, in_w;
  Buf d_vbase0, d_ebase, d_wbase;
  // per-graph state
  Buf phase, level, run, any, changed, contracted, first, did, best_kind, trace_len;
  Buf vbase, vbase_new, nv, nnz, n_start, lam, best_vertex, argmin, dmin, obase, norig, n1, noi_base;
  Buf gkey, gact, trace, summary, list_noid, list_nois;
  // union-wide
  Buf gid, gid2, vact, sideK, noiM, noiCurK, bits_out, cut_out;
  Workspace* ws = nullptr;
  int* h_summary = nullptr;
  viecut_batch_stats stats{};
  ~Batch() {
    delete ws;
    if (h_summary) cudaFreeHost(h_summary);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
  BState state() {
    BState S;
    S.phase = phase.as<int>(); S.level = level.as<int>(); S.run = run.as<int>(); S.any = any.as<int>();
    S.changed = changed.as<int>(); S.contracted = contracted.as<int>(); S.first = first.as<int>();
    S.did = did.as<int>(); S.best_kind = best_kind.as<int>(); S.trace_len = trace_len.as<int>();
    S.vbase = vbase.as<long long>(); S.vbase_new = vbase_new.as<long long>(); S.nv = nv.as<long long>();
    S.nnz = nnz.as<long long>(); S.n_start = n_start.as<long long>(); S.lam = lam.as<long long>();
    S.best_vertex = best_vertex.as<long long>(); S.argmin = argmin.as<long long>(); S.dmin = dmin.as<long long>();
    S.obase = obase.as<long long>(); S.norig = norig.as<long long>(); S.n1 = n1.as<long long>();
    S.noi_base = noi_base.as<long long>(); S.gkey = gkey.as<unsigned long long>(); S.gact = gact.as<unsigned char>();
    S.trace = trace.as<TraceStep>(); S.summary = summary.as<int>();
    S.list_noid = list_noid.as<int32_t>(); S.list_nois = list_nois.as<int32_t>();
    return S;
  }
};

static void batch_create(Batch& B, const viecut_graph_desc* gs, int K, const viecut_opts& o) {
  B.K = K;
  B.n0 = o.n0;
  B.pr_runs_max = o.pr_runs_max;
  B.device = o.device;
  VC_CUDA(cudaSetDevice(B.device));
  if (o.stream) {
    B.stream = (cudaStream_t)o.stream;
  } else {
    VC_CUDA(cudaStreamCreateWithFlags(&B.stream, cudaStreamNonBlocking));
    B.own_stream = true;
  }
  cudaStream_t s = B.stream;
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
  B.n_u = B.h_vbase[K];
  B.m_u = B.h_ebase[K];
  if (B.n_u > 0x7fffffffLL) throw Error{VIECUT_EINVAL, "the batch must hold fewer than 2^31 vertices"};
  int64_t* off = B.in_off.ensure_n<int64_t>(B.n_u + 1);
  int32_t* adj = B.in_adj.ensure_n<int32_t>(B.m_u);
  int32_t* w = B.in_w.ensure_n<int32_t>(B.m_u);
  for (int g = 0; g < K; ++g) {
    VC_CUDA(cudaMemcpyAsync(off + B.h_vbase[g], gs[g].offsets, sizeof(int64_t) * gs[g].n, cudaMemcpyHostToDevice, s));
    if (gs[g].m > 0) {
      VC_CUDA(cudaMemcpyAsync(adj + B.h_ebase[g], gs[g].adj, sizeof(int32_t) * gs[g].m, cudaMemcpyHostToDevice, s));
      VC_CUDA(cudaMemcpyAsync(w + B.h_ebase[g], gs[g].weights, sizeof(int32_t) * gs[g].m, cudaMemcpyHostToDevice, s));
    }
  }
  VC_CUDA(cudaMemcpyAsync(off + B.n_u, &B.m_u, sizeof(int64_t), cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_vbase0.ensure_n<long long>(K + 1), B.h_vbase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_ebase.ensure_n<long long>(K + 1), B.h_ebase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.d_wbase.ensure_n<long long>(K + 1), B.h_wbase.data(), sizeof(long long) * (K + 1),
                          cudaMemcpyHostToDevice, s));
  B.ws = new Workspace;
  B.ws->s = s;
  Workspace& W = *B.ws;
  int* err = &W.ctr()->changed;
  VC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  int gridK = K < 4 * kSMs ? K : 4 * kSMs;
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
  W.ensure_vertices(B.n_u);
  W.ensure_entries(B.m_u, B.n_u);
  for (Buf* b : {&B.phase, &B.level, &B.run, &B.any, &B.changed, &B.contracted, &B.first, &B.did, &B.best_kind,
                 &B.trace_len})
    b->ensure_n<int>(K);
  for (Buf* b : {&B.nv, &B.nnz, &B.n_start, &B.lam, &B.best_vertex, &B.argmin, &B.dmin, &B.obase, &B.norig, &B.n1,
                 &B.noi_base})
    b->ensure_n<long long>(K);
  B.vbase.ensure_n<long long>(K + 1);
  B.vbase_new.ensure_n<long long>(K + 1);
  B.gkey.ensure_n<unsigned long long>(K);
  B.gact.ensure_n<unsigned char>(K);
  B.trace.ensure_n<TraceStep>((int64_t)K * kBTraceCap);
  B.summary.ensure_n<int>(kSummaryInts);
  B.list_noid.ensure_n<int32_t>(K);
  B.list_nois.ensure_n<int32_t>(K);
  B.gid.ensure_n<int32_t>(B.n_u);
  B.gid2.ensure_n<int32_t>(B.n_u);
  B.vact.ensure_n<unsigned char>(B.n_u);
  B.sideK.ensure_n<unsigned char>((int64_t)K * kDenseMax);
  B.noiCurK.ensure_n<int32_t>((int64_t)kSMs * kDenseMax);
  B.bits_out.ensure_n<unsigned long long>(B.h_wbase[K]);
  B.cut_out.ensure_n<long long>(K);
  VC_CUDA(cudaMallocHost(&B.h_summary, sizeof(int) * kSummaryInts));
  // per-graph constants: original bases and sizes
  std::vector<long long> norig(K);
  for (int g = 0; g < K; ++g) norig[g] = gs[g].n;
  VC_CUDA(cudaMemcpyAsync(B.obase.p, B.h_vbase.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemcpyAsync(B.norig.p, norig.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaStreamSynchronize(s));
}

static void read_summary(Batch& B) {
  VC_CUDA(cudaMemcpyAsync(B.h_summary, B.summary.p, sizeof(int) * kSummaryInts, cudaMemcpyDeviceToHost, B.stream));
  VC_CUDA(cudaStreamSynchronize(B.stream));
}

static void batch_run(Batch& B, uint64_t seed, int lp_iters) {
  if (lp_iters < 0) throw Error{VIECUT_EINVAL, "lp_iters must be >= 0"};
  VC_CUDA(cudaSetDevice(B.device));
  cudaStream_t s = B.stream;
  Workspace& W = *B.ws;
  W.s = s;
  const unsigned long long launches0 = g_launches;
  cudaEvent_t e0, e1;
  VC_CUDA(cudaEventCreate(&e0));
  VC_CUDA(cudaEventCreate(&e1));
  VC_CUDA(cudaEventRecord(e0, s));
  const int K = B.K;
  BState S = B.state();
  const int gK = (K + 255) / 256;
  const int gridK = K < 4 * kSMs ? K : 4 * kSMs;

  // the input union
  GraphView G;
  G.n = B.n_u;
  G.nnz = B.m_u;
  G.off = B.in_off.as<int64_t>();
  G.adj = B.in_adj.as<int32_t>();
  G.w = B.in_w.p;
  G.wbytes = 4;
  G.unit = B.unit;
  G.simple = B.simple;
  W.bins_valid = false;
  int slot = -1;
  int32_t* gid = B.gid.as<int32_t>();
  int32_t* gid2 = B.gid2.as<int32_t>();
  VC_CUDA(cudaMemcpyAsync(S.vbase, B.d_vbase0.p, sizeof(long long) * (K + 1), cudaMemcpyDeviceToDevice, s));
  {
    std::vector<long long> nv(K);
    for (int g = 0; g < K; ++g) nv[g] = B.h_vbase[g + 1] - B.h_vbase[g];
    VC_CUDA(cudaMemcpyAsync(S.nv, nv.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
    std::vector<long long> ne(K);
    for (int g = 0; g < K; ++g) ne[g] = B.h_ebase[g + 1] - B.h_ebase[g];
    VC_CUDA(cudaMemcpyAsync(S.nnz, ne.data(), sizeof(long long) * K, cudaMemcpyHostToDevice, s));
    VC_CUDA(cudaMemsetAsync(S.noi_base, 0, sizeof(long long) * K, s));
    VC_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  b_gid_init_k<<<gridK, 256, 0, s>>>(K, S.vbase, gid);
  degrees(G, W.deg.as<long long>(), s);
  b_segmin_k<<<gridK, 256, 0, s>>>(K, W.deg.as<long long>(), S, 0);
  b_init_k<<<gK, 256, 0, s>>>(K, S, B.n0);
  b_tier1_k<<<gridK, 256, 0, s>>>(K, S, nullptr, W.map0.as<int32_t>(), W.cur1.as<int32_t>(), 0);
  count_launch(4);
  VC_CHECK_LAUNCH();

  int64_t steps = 0;
  for (;;) {
    VC_CUDA(cudaMemsetAsync(S.summary, 0, sizeof(int) * kSummaryInts, s));
    b_summary_k<<<gK, 256, 0, s>>>(K, S);
    count_launch();
    read_summary(B);
    const int* cnt = B.h_summary;
    if (cnt[kBLP] + cnt[kBPRA] + cnt[kBPRB] + cnt[kBNoiS] + cnt[kBNoiD] + cnt[kBDone] == 0) break;
    if (++steps > (int64_t)64 * (B.n_u + 16)) throw Error{VIECUT_ECUDA, "batch did not converge"};
    int32_t* A = W.labA.as<int32_t>();
    int32_t* Bl = W.labB.as<int32_t>();
    iota(A, G.n, s);
    iota(Bl, G.n, s);
    int32_t* F = A;
    BatchCtx bc;
    bc.gid = gid;
    bc.glam = S.lam;
    bc.gact = S.gact;
    bc.gchanged = S.changed;
    if (cnt[kBLP] > 0) {
      b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBLP, seed);
      b_vact_k<<<grid_for(G.n, 256, kSMs * 8), 256, 0, s>>>(G.n, gid, S.gact, B.vact.as<unsigned char>());
      count_launch(2);
      hash_table(G.n, 0, gid, S.gkey, S.vbase, W.hv.as<unsigned long long>(), s);
      if (!W.bins_valid) W.build_bins(G);
      GraphView Ga = G;
      Ga.vact = B.vact.as<unsigned char>();
      int32_t* in = nullptr;
      int32_t* bufs[2] = {A, Bl};
      for (int r = 0; r < lp_iters; ++r) {
        lp_round(Ga, W.bins, W.gt, in, bufs[r & 1], W.hv.as<unsigned long long>(), s);
        in = bufs[r & 1];
      }
      if (lp_iters > 0) F = in;
    }
    if (cnt[kBPRA] > 0) {
      b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBPRA, seed);
      count_launch();
      pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
      pr_pass_a(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(),
                W.parent.as<int32_t>(), F, nullptr, s, &bc);
    }
    if (cnt[kBPRB] > 0) {
      b_prepare_k<<<gK, 256, 0, s>>>(K, S, kBPRB, seed);
      count_launch();
      pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
      pr_pass_b(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(), F, nullptr, s, &bc);
    }
    if (cnt[kBNoiS] > 0) {
      W.noi_r.ensure_n<long long>(G.n);
      W.noi_seen.ensure_n<unsigned char>(G.n);
      noi_round_batch(G, S.list_nois, cnt[10], S.vbase, S.nv, S.lam, W.noi_r.as<long long>(),
                      W.noi_seen.as<unsigned char>(), W.parent.as<int32_t>(), F, S.changed, s);
    }
    if (cnt[kBNoiD] > 0) {
      const int64_t mcap = (int64_t)cnt[7] * cnt[7];
      const int blocks = cnt[kBNoiD] < kSMs ? cnt[kBNoiD] : kSMs;
      long long* M = B.noiM.ensure_n<long long>(2 * mcap * blocks);
      BatchNoi bn{S.lam, S.best_kind, S.nv, S.nnz, S.dmin, S.argmin, S.trace_len, S.trace, kBTraceCap, S.level};
      noi_dense_batch(G, S.list_noid, cnt[kBNoiD], S.vbase, S.nv, M, mcap, blocks, B.noiCurK.as<int32_t>(),
                      B.sideK.as<unsigned char>(), bn, s);
    }
    b_decide_k<<<gK, 256, 0, s>>>(K, S);
    count_launch();
    read_summary(B);
    if (B.h_summary[8] > 0) {
      b_drop_k<<<grid_for(G.n, 256, kSMs * 8), 256, 0, s>>>(G.n, gid, S.phase, F);
      count_launch();
      int dst = slot == 0 ? 1 : 0;
      int32_t* cid = W.cidT.as<int32_t>();
      const int64_t n_old = G.n;
      GraphView h = W.contract(G, F, cid, dst);
      b_shape_k<<<(K + 1 + 255) / 256, 256, 0, s>>>(K, S, n_old, h.n, W.rank.as<int32_t>(), h.off);
      b_shape2_k<<<gK, 256, 0, s>>>(K, S, h.off);
      b_gid_update_k<<<grid_for(n_old, 256, kSMs * 8), 256, 0, s>>>(n_old, cid, gid, gid2);
      b_tier1_k<<<gridK, 256, 0, s>>>(K, S, cid, W.map0.as<int32_t>(), W.cur1.as<int32_t>(), 1);
      b_copy_vbase_k<<<(K + 1 + 255) / 256, 256, 0, s>>>(K, S);
      count_launch(5);
      VC_CHECK_LAUNCH();
      std::swap(gid, gid2);
      G = h;
      G.nnz = W.h_counters->pairs;  // upper bound; lists are exact through the offsets
      slot = dst;
      if (G.n > 0) {
        degrees(G, W.deg.as<long long>(), s);
        b_segmin_k<<<gridK, 256, 0, s>>>(K, W.deg.as<long long>(), S, 1);
        b_snapshot_k<<<gridK, 256, 0, s>>>(K, S, W.cur1.as<int32_t>(), W.side1.as<unsigned char>());
        count_launch(2);
      }
      b_trace_k<<<gK, 256, 0, s>>>(K, S);
      count_launch();
    }
    b_transition_k<<<gK, 256, 0, s>>>(K, S, B.n0, B.pr_runs_max);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  b_side_bits_k<<<gridK, 256, 0, s>>>(K, S, B.d_wbase.as<long long>(), W.map0.as<int32_t>(),
                                      W.side1.as<unsigned char>(), W.cur1.as<int32_t>(), B.sideK.as<unsigned char>(),
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
  B.stats.super_steps = steps;
  B.stats.kernel_launches = (int64_t)(g_launches - launches0);
  B.stats.graphs = K;
  B.stats.vertices = B.n_u;
  B.stats.entries = B.m_u;
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
  VC_CUDA(cudaMemcpyAsync(cut_values, B.lam.p, sizeof(int64_t) * B.K, cudaMemcpyDeviceToHost, B.stream));
  if (side_bits)
    VC_CUDA(cudaMemcpyAsync(side_bits, B.bits_out.p, sizeof(uint64_t) * B.h_wbase[B.K], cudaMemcpyDeviceToHost,
                            B.stream));
  VC_CUDA(cudaStreamSynchronize(B.stream));
  VC_API_END
}

int viecut_batch_side_words(const viecut_batch* bt, int64_t* words) {
  VC_API_BEGIN
  if (!bt || !words) throw Error{VIECUT_EINVAL, "null argument"};
  *words = bt->b.h_wbase[bt->b.K];
  VC_API_END
}

int viecut_batch_get_trace(const viecut_batch* bt, int32_t g, viecut_step* steps, int64_t cap, int64_t* len) {
  VC_API_BEGIN
  if (!bt || !len || g < 0 || g >= bt->b.K) throw Error{VIECUT_EINVAL, "bad graph index"};
  const vc::Batch& B = bt->b;
  VC_CUDA(cudaSetDevice(B.device));
  int tl = 0;
  VC_CUDA(cudaMemcpy(&tl, (int*)B.trace_len.p + g, sizeof(int), cudaMemcpyDeviceToHost));
  int cnt = tl < vc::kBTraceCap ? tl : vc::kBTraceCap;
  std::vector<vc::TraceStep> t(cnt);
  if (cnt)
    VC_CUDA(cudaMemcpy(t.data(), (vc::TraceStep*)B.trace.p + (int64_t)g * vc::kBTraceCap, sizeof(vc::TraceStep) * cnt,
                       cudaMemcpyDeviceToHost));
  *len = tl;
  for (int64_t i = 0; i < cap && i < cnt; ++i)
    steps[i] = viecut_step{t[i].kind, t[i].level, t[i].n, t[i].nnz, t[i].lambda_hat};
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
  cudaSetDevice(bt->b.device);
  if (bt->b.stream) cudaStreamSynchronize(bt->b.stream);
  delete bt;
  VC_API_END
}

}  // extern "C"
