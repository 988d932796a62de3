// Device-wide primitives (scan, radix sort) written for this library; no CUB.
#pragma once
#include "common.cuh"

namespace vc {

// Exclusive prefix sum out[i] = sum_{j<i} in[i]; *total (device pointer, may be
// null) receives the sum of all n inputs.  scratch must hold scan_scratch_elems(n)
// values of Out.
template <typename In, typename Out>
void exclusive_scan(const In* in, Out* out, int64_t n, Out* total, Out* scratch, cudaStream_t s);
int64_t scan_scratch_elems(int64_t n);

// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the keys.
// Sorted output lands in keys/vals (the alt buffers are scratch of the same size).
// hist must hold radix_hist_elems(n) int64 values.
void radix_sort_pairs(unsigned long long* keys, long long* vals, unsigned long long* keys_alt,
                      long long* vals_alt, int64_t n, int bits, long long* hist, cudaStream_t s);
int64_t radix_hist_elems(int64_t n);

}  // namespace vc
