// Trivial-cut bound and solution tracking.
//
// The bound lambda-hat starts as the minimum weighted degree and, after every
// contraction, drops to the coarse graph's minimum degree when that is strictly
// smaller (Sec. 4, second paragraph; trivial cut, Sec. 3).  The side of the best
// cut is kept as a snapshot over the vertices of the first contracted graph
// ("tier 1"); the final side of each original vertex goes through the first map
// (solution transfer, Algorithm 1 and Appendix B).
#include <limits.h>

#include "kernels.cuh"

namespace vc {

template <typename WT>
__global__ void degrees_k(int64_t n, const int64_t* __restrict__ off, const WT* __restrict__ w,
                          long long* __restrict__ deg) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
    long long s = 0;
    for (int64_t e = off[v] + lane; e < off[v + 1]; e += 32) s += ldw(w, e);
    s = warp_sum(s);
    if (lane == 0) deg[v] = s;
  }
}

// unit weights: the degree is the list length
__global__ void degrees_unit_k(int64_t n, const int64_t* __restrict__ off, long long* __restrict__ deg) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    deg[v] = off[v + 1] - off[v];
}

void degrees(const GraphView& g, long long* deg, cudaStream_t s) {
  int grid = grid_for(g.n, 8, kSMs * 16);
  if (g.unit) degrees_unit_k<<<grid_for(g.n, 256, kSMs * 8), 256, 0, s>>>(g.n, g.off, deg);
  else if (g.wbytes == 4) degrees_k<int32_t><<<grid, 256, 0, s>>>(g.n, g.off, (const int32_t*)g.w, deg);
  else degrees_k<long long><<<grid, 256, 0, s>>>(g.n, g.off, (const long long*)g.w, deg);
  count_launch();
  VC_CHECK_LAUNCH();
}

struct DegArg {
  long long d, v;
};
__device__ __forceinline__ bool deg_less(const DegArg& a, const DegArg& b) {
  return a.d < b.d || (a.d == b.d && a.v < b.v);
}

template <int NT>
__device__ __forceinline__ DegArg block_min(DegArg x) {
  __shared__ long long sd[NT / 32], sv[NT / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DegArg y{__shfl_xor_sync(0xffffffffu, x.d, o), __shfl_xor_sync(0xffffffffu, x.v, o)};
    if (deg_less(y, x)) x = y;
  }
  if (lane == 0) { sd[wid] = x.d; sv[wid] = x.v; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < NT / 32; ++q) {
      DegArg y{sd[q], sv[q]};
      if (deg_less(y, x)) x = y;
    }
  }
  __syncthreads();
  return x;  // valid in thread 0
}

__global__ void min_partial_k(const long long* __restrict__ deg, int64_t n, long long* __restrict__ partial) {
  DegArg best{LLONG_MAX, LLONG_MAX};
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    DegArg c{deg[v], v};
    if (deg_less(c, best)) best = c;
  }
  best = block_min<256>(best);
  if (threadIdx.x == 0) { partial[2 * blockIdx.x] = best.d; partial[2 * blockIdx.x + 1] = best.v; }
}

__global__ void min_final_k(const long long* __restrict__ partial, int nb, DevState* st, int initial) {
  DegArg best{LLONG_MAX, LLONG_MAX};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    DegArg c{partial[2 * b], partial[2 * b + 1]};
    if (deg_less(c, best)) best = c;
  }
  best = block_min<256>(best);
  if (threadIdx.x == 0) {
    st->dmin = best.d;
    st->argmin = best.v;
    if (initial) {
      st->lambda_hat = best.d;
      st->best_vertex = best.v;
      st->best_kind = 0;
      st->improved = 0;
    } else if (best.d < st->lambda_hat) {
      st->lambda_hat = best.d;
      st->improved = 1;
    } else {
      st->improved = 0;
    }
  }
}

void bound_update_impl(const long long* deg, int64_t n, DevState* st, long long* partial, int initial,
                       cudaStream_t s) {
  int nb = grid_for(n, 256, 512);
  min_partial_k<<<nb, 256, 0, s>>>(deg, n, partial);
  min_final_k<<<1, 256, 0, s>>>(partial, nb, st, initial);
  count_launch(2);
  VC_CHECK_LAUNCH();
}

void bound_update(const long long* deg, int64_t n, DevState* st, long long* partial, cudaStream_t s) {
  bound_update_impl(deg, n, st, partial, 0, s);
}

void bound_init(const long long* deg, int64_t n, DevState* st, long long* partial, cudaStream_t s) {
  bound_update_impl(deg, n, st, partial, 1, s);
}

__global__ void snapshot_k(const int32_t* __restrict__ cur1, int64_t n1, unsigned char* __restrict__ side1,
                           DevState* st) {
  if (!st->improved) return;
  const long long b = st->argmin;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n1; j += (int64_t)gridDim.x * blockDim.x)
    side1[j] = cur1[j] == b ? 1 : 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) st->best_kind = 1;
}

void snapshot_side(const int32_t* cur1, int64_t n1, unsigned char* side1, DevState* st, cudaStream_t s) {
  snapshot_k<<<grid_for(n1, 256, kSMs * 8), 256, 0, s>>>(cur1, n1, side1, st);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void compose_k(int32_t* __restrict__ cur1, int64_t n1, const int32_t* __restrict__ cid) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n1; j += (int64_t)gridDim.x * blockDim.x)
    cur1[j] = cid[cur1[j]];
}

void compose_map(int32_t* cur1, int64_t n1, const int32_t* cid, cudaStream_t s) {
  compose_k<<<grid_for(n1, 256, kSMs * 8), 256, 0, s>>>(cur1, n1, cid);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void iota_k(int32_t* __restrict__ x, int64_t n) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    x[j] = (int32_t)j;
}

void iota(int32_t* x, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  iota_k<<<grid_for(n, 256, kSMs * 8), 256, 0, s>>>(x, n);
  count_launch();
  VC_CHECK_LAUNCH();
}

// Bit i = membership of original vertex i in the best side, flipped so that vertex 0
// is outside.  best_kind 0: single original vertex; 1: tier-1 snapshot; 2: snapshot
// over the vertices of the graph the final exact step started from.
__device__ __forceinline__ int side_of(int64_t i, const int32_t* orig_map, const unsigned char* side1,
                                       const int32_t* cur1, const unsigned char* sideK, int kind, long long bv) {
  if (kind == 0) return i == bv;
  int32_t t = orig_map[i];
  if (kind == 1) return side1[t];
  return sideK[cur1[t]];
}

__global__ void side_bits_k(const int32_t* __restrict__ orig_map, int64_t n, const unsigned char* __restrict__ side1,
                            const int32_t* __restrict__ cur1, const unsigned char* __restrict__ sideK,
                            const DevState* st, unsigned long long* __restrict__ bits) {
  const int kind = st->best_kind;
  const long long bv = st->best_vertex;
  const int flip = side_of(0, orig_map, side1, cur1, sideK, kind, bv);
  const int64_t words = (n + 63) / 64;
  for (int64_t wd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wd < words; wd += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long x = 0;
    int64_t lim = (wd + 1) * 64 < n ? (wd + 1) * 64 : n;
    for (int64_t i = wd * 64; i < lim; ++i)
      if (side_of(i, orig_map, side1, cur1, sideK, kind, bv) != flip) x |= 1ULL << (i & 63);
    bits[wd] = x;
  }
}

void side_bits2(const int32_t* orig_map, int64_t n, const unsigned char* side1, const int32_t* cur1,
                const unsigned char* sideK, const DevState* st, unsigned long long* bits, cudaStream_t s) {
  side_bits_k<<<grid_for((n + 63) / 64, 256, kSMs * 8), 256, 0, s>>>(orig_map, n, side1, cur1, sideK, st, bits);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void trace_push_k(DevState* st, TraceStep* trace, int cap, int kind, int level) {
  int i = st->trace_len;
  if (i < cap) trace[i] = TraceStep{kind, level, st->n, st->nnz, st->lambda_hat};
  st->trace_len = i + 1;
}

void trace_push(DevState* st, TraceStep* trace, int cap, int kind, int level, cudaStream_t s) {
  trace_push_k<<<1, 1, 0, s>>>(st, trace, cap, kind, level);
  count_launch();
  VC_CHECK_LAUNCH();
}

}  // namespace vc
