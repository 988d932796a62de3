// Cluster contraction (Sec. 4.1, "contract it"; contraction semantics, Sec. 3):
// every block of a labelling becomes one vertex, intra-block edges vanish and
// parallel edges between two blocks merge with summed weight.  Block ids are the
// ranks of the label values.  Steps: relabel (flag + scan), pre-merge per fine
// vertex (lp.cu), pair build, LSD radix sort on (cid v, cid u), run reduction.
#include "kernels.cuh"
#include "prims.cuh"

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

// One thread per fine vertex copies its pre-merged list (two entries on average at the
// level-0 contraction) into the contiguous pair arrays.
__global__ void build_pairs_k(int64_t n, const int64_t* __restrict__ off, const int32_t* __restrict__ cid,
                              const int32_t* __restrict__ cnt, const long long* __restrict__ pos,
                              const int32_t* __restrict__ tkey, const long long* __restrict__ tval, int bits,
                              unsigned long long* __restrict__ keys, long long* __restrict__ vals) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int k = cnt[v];
    if (k == 0) continue;
    const int64_t src = off[v];
    const long long dst = pos[v];
    const unsigned long long hi = (unsigned long long)cid[v] << bits;
    for (int j = 0; j < k; ++j) {
      keys[dst + j] = hi | (unsigned long long)(uint32_t)tkey[src + j];
      vals[dst + j] = tval[src + j];
    }
  }
}

void build_pairs(const GraphView& g, const int32_t* cid, const ContractScratch& cs, int bits,
                 unsigned long long* keys, long long* vals, cudaStream_t s) {
  build_pairs_k<<<grid_for(g.n, 256, kSMs * 8), 256, 0, s>>>(g.n, g.off, cid, cs.cnt, cs.pos, cs.tmp_key,
                                                           cs.tmp_val, bits, keys, vals);
  count_launch();
  VC_CHECK_LAUNCH();
}

__global__ void run_heads_k(const unsigned long long* __restrict__ keys, int64_t m, int32_t* __restrict__ heads) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    heads[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Each run head sums its run (runs are short: one entry per fine vertex of the
// source cluster that touches the target cluster).
__global__ void run_reduce_k(const unsigned long long* __restrict__ keys, const long long* __restrict__ vals,
                             int64_t m, int bits, const int32_t* __restrict__ heads,
                             const long long* __restrict__ hpos, int32_t* __restrict__ cadj,
                             long long* __restrict__ cw, int32_t* __restrict__ cv) {
  const unsigned long long mask = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1ULL);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    if (!heads[i]) continue;
    const unsigned long long k = keys[i];
    long long s = vals[i];
    for (int64_t j = i + 1; j < m && keys[j] == k; ++j) s += vals[j];
    const long long o = hpos[i];
    cadj[o] = (int32_t)(k & mask);
    cw[o] = s;
    cv[o] = (int32_t)(k >> bits);
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
    run_reduce_k<<<grid, 256, 0, s>>>(keys, vals, pairs, bits, heads, hpos, cadj, cw, cv_tmp);
    count_launch();
    VC_CHECK_LAUNCH();
  }
  build_offsets_k<<<grid_for(pairs + c + 1, 256, kSMs * 8), 256, 0, s>>>(cv_tmp, nnz_dev, c, (int64_t*)coff);
  count_launch();
  VC_CHECK_LAUNCH();
}

}  // namespace vc
