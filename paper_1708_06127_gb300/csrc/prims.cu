// Device-wide exclusive scan and stable LSD radix sort (reduce-then-scan design).
#include "prims.cuh"

namespace vc {

// ------------------------------------------------------------------- block scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <typename In, typename Out>
__global__ void scan_reduce_k(const In* __restrict__ in, int64_t n, Out* __restrict__ partial) {
  __shared__ Out red[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  Out s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t k = base + i * kScanThreads + threadIdx.x;
    if (k < n) s += (Out)in[k];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    Out v = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : (Out)0;
    v = warp_sum(v);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

// Single block: exclusive scan of partial[0..nb) in place; total to *total.
template <typename Out>
__global__ void scan_partials_k(Out* __restrict__ partial, int64_t nb, Out* __restrict__ total) {
  __shared__ Out wsum[32];
  __shared__ Out carry_s;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += 1024) {
    int64_t k = base + threadIdx.x;
    Out x = k < nb ? partial[k] : (Out)0;
    Out inc = warp_incl_scan(x);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      Out v = wsum[lane];
      Out vi = warp_incl_scan(v);
      wsum[lane] = vi - v;
    }
    __syncthreads();
    Out carry = carry_s;
    Out ex = carry + wsum[wid] + inc - x;
    if (k < nb) partial[k] = ex;
    __syncthreads();
    if (threadIdx.x == 1023) carry_s = ex + x;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry_s;
}

template <typename In, typename Out>
__global__ void scan_apply_k(const In* __restrict__ in, Out* __restrict__ out, int64_t n,
                             const Out* __restrict__ partial) {
  __shared__ Out tile[kScanTile];
  __shared__ Out wsum[kScanThreads / 32];
  int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int idx = i * kScanThreads + threadIdx.x;
    int64_t k = base + idx;
    tile[idx] = k < n ? (Out)in[k] : (Out)0;
  }
  __syncthreads();
  Out loc[kScanItems];
  Out s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = s;
    s += tile[threadIdx.x * kScanItems + i];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Out inc = warp_incl_scan(s);
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    Out v = lane < kScanThreads / 32 ? wsum[lane] : (Out)0;
    Out vi = warp_incl_scan(v);
    if (lane < kScanThreads / 32) wsum[lane] = vi - v;
  }
  __syncthreads();
  Out off = partial[blockIdx.x] + wsum[wid] + inc - s;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) tile[threadIdx.x * kScanItems + i] = off + loc[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int idx = i * kScanThreads + threadIdx.x;
    int64_t k = base + idx;
    if (k < n) out[k] = tile[idx];
  }
}

int64_t scan_scratch_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <typename In, typename Out>
void exclusive_scan(const In* in, Out* out, int64_t n, Out* total, Out* scratch, cudaStream_t s) {
  if (n <= 0) {
    if (total) VC_CUDA(cudaMemsetAsync(total, 0, sizeof(Out), s));
    return;
  }
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  scan_reduce_k<In, Out><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, scratch);
  scan_partials_k<Out><<<1, 1024, 0, s>>>(scratch, nb, total);
  scan_apply_k<In, Out><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, scratch);
  count_launch(3);
  VC_CHECK_LAUNCH();
}

template void exclusive_scan<int, long long>(const int*, long long*, int64_t, long long*, long long*, cudaStream_t);
template void exclusive_scan<long long, long long>(const long long*, long long*, int64_t, long long*, long long*, cudaStream_t);
template void exclusive_scan<int, int>(const int*, int*, int64_t, int*, int*, cudaStream_t);

// ------------------------------------------------------------------- radix sort
constexpr int kRadixBits = 8;
constexpr int kBuckets = 1 << kRadixBits;
constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kRTile = 2048;

int64_t radix_hist_elems(int64_t n) {
  int64_t nb = (n + kRTile - 1) / kRTile;
  return nb * kBuckets + scan_scratch_elems(nb * kBuckets) + 1;
}

__global__ void radix_hist_k(const unsigned long long* __restrict__ keys, int64_t n, int shift,
                             int64_t nb, long long* __restrict__ hist) {
  __shared__ int cnt[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += kRThreads) cnt[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRTile;
  for (int i = threadIdx.x; i < kRTile; i += kRThreads) {
    int64_t k = base + i;
    if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & (kBuckets - 1)], 1);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kBuckets; d += kRThreads) hist[(int64_t)d * nb + blockIdx.x] = cnt[d];
}

__global__ void radix_scatter_k(const unsigned long long* __restrict__ keys,
                                const long long* __restrict__ vals, int64_t n, int shift, int64_t nb,
                                const long long* __restrict__ ghist, unsigned long long* __restrict__ okeys,
                                long long* __restrict__ ovals) {
  __shared__ unsigned long long sk[kRTile];
  __shared__ long long sv[kRTile];
  __shared__ int wcnt[kRWarps][kBuckets];
  __shared__ int tstart[kBuckets];
  __shared__ int running[kBuckets];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRTile;
  const int tcount = (int)min((int64_t)kRTile, n - base);

  // digit counts of the whole tile -> tile-local bucket starts
  for (int d = threadIdx.x; d < kBuckets; d += kRThreads) { running[d] = 0; tstart[d] = 0; }
  __syncthreads();
  for (int i = threadIdx.x; i < tcount; i += kRThreads)
    atomicAdd(&tstart[(keys[base + i] >> shift) & (kBuckets - 1)], 1);
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of 256 counts by one warp, 8 per lane
    int v[kBuckets / 32];
    int s = 0;
#pragma unroll
    for (int j = 0; j < kBuckets / 32; ++j) { v[j] = tstart[lane * (kBuckets / 32) + j]; s += v[j]; }
    int inc = warp_incl_scan(s);
    int ex = inc - s;
#pragma unroll
    for (int j = 0; j < kBuckets / 32; ++j) { tstart[lane * (kBuckets / 32) + j] = ex; ex += v[j]; }
  }
  __syncthreads();

  // stable ranks, 256 keys per sub-round in input order
  for (int r0 = 0; r0 < tcount; r0 += kRThreads) {
    for (int d = lane; d < kBuckets; d += 32) wcnt[wid][d] = 0;
    int i = r0 + threadIdx.x;
    bool valid = i < tcount;
    unsigned long long k = valid ? keys[base + i] : 0ULL;
    long long val = valid ? vals[base + i] : 0LL;
    int d = valid ? (int)((k >> shift) & (kBuckets - 1)) : kBuckets;
    unsigned peers = __match_any_sync(0xffffffffu, d);
    int rank = __popc(peers & ((1u << lane) - 1));
    __syncwarp();
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    // per digit: exclusive prefix over warps, plus the running count of earlier rounds
    for (int dd = threadIdx.x; dd < kBuckets; dd += kRThreads) {
      int acc = running[dd];
#pragma unroll
      for (int w = 0; w < kRWarps; ++w) {
        int c = wcnt[w][dd];
        wcnt[w][dd] = acc;
        acc += c;
      }
      running[dd] = acc;
    }
    __syncthreads();
    if (valid) {
      int lp = tstart[d] + wcnt[wid][d] + rank;
      sk[lp] = k;
      sv[lp] = val;
    }
    __syncthreads();
  }
  // coalesced write-out of the locally sorted tile
  for (int i = threadIdx.x; i < tcount; i += kRThreads) {
    unsigned long long k = sk[i];
    int d = (int)((k >> shift) & (kBuckets - 1));
    long long pos = ghist[(int64_t)d * nb + blockIdx.x] + (i - tstart[d]);
    okeys[pos] = k;
    ovals[pos] = sv[i];
  }
}

void radix_sort_pairs(unsigned long long* keys, long long* vals, unsigned long long* keys_alt,
                      long long* vals_alt, int64_t n, int bits, long long* hist, cudaStream_t s) {
  if (n <= 1 || bits <= 0) return;
  int64_t nb = (n + kRTile - 1) / kRTile;
  long long* scan_scr = hist + nb * kBuckets;
  unsigned long long *src_k = keys, *dst_k = keys_alt;
  long long *src_v = vals, *dst_v = vals_alt;
  int passes = (bits + kRadixBits - 1) / kRadixBits;
  for (int p = 0; p < passes; ++p) {
    int shift = p * kRadixBits;
    radix_hist_k<<<(unsigned)nb, kRThreads, 0, s>>>(src_k, n, shift, nb, hist);
    count_launch();
    VC_CHECK_LAUNCH();
    exclusive_scan<long long, long long>(hist, hist, nb * kBuckets, nullptr, scan_scr, s);
    radix_scatter_k<<<(unsigned)nb, kRThreads, 0, s>>>(src_k, src_v, n, shift, nb, hist, dst_k, dst_v);
    count_launch();
    VC_CHECK_LAUNCH();
    std::swap(src_k, dst_k);
    std::swap(src_v, dst_v);
  }
  if (src_k != keys) {
    VC_CUDA(cudaMemcpyAsync(keys, src_k, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, s));
    VC_CUDA(cudaMemcpyAsync(vals, src_v, sizeof(long long) * n, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace vc
