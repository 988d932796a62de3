// Shared device/host utilities of the GB300 VieCut library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>

namespace vc {

// ------------------------------------------------------------ error handling
struct Error {
  int code;
  std::string msg;
};

#define VC_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      throw ::vc::Error{-3, std::string(#call) + ": " + cudaGetErrorString(e_)};        \
  } while (0)

#define VC_CHECK_LAUNCH() VC_CUDA(cudaGetLastError())

// ------------------------------------------------------------ launch shape
constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs

inline int grid_for(int64_t work, int per_block, int max_blocks) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > max_blocks) g = max_blocks;
  return (int)g;
}

// Number of kernels this library launched (process-wide), for the launch count
// reported beside timings.
extern std::atomic<unsigned long long> g_launches;  // host threads of servers count too
inline void count_launch(int k = 1) { g_launches += (unsigned long long)k; }

// ------------------------------------------------------------ device helpers
// SplitMix64 output function (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ULL;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebULL;
  z ^= z >> 31;
  return z;
}

// Per-level tie-break key: the SplitMix64 output after (level + 1) golden-gamma
// increments from the seed.
__host__ __device__ __forceinline__ uint64_t level_key(uint64_t seed, int64_t level) {
  return mix64(seed + 0x9e3779b97f4a7c15ULL * (uint64_t)(level + 1));
}

// Label-propagation tie-break value of label L under a level key.
__device__ __forceinline__ uint64_t tie_hash(uint64_t key, int32_t L) {
  return mix64(key ^ (uint64_t)(uint32_t)L);
}

// Slot hash for the open-addressing accumulation tables (any mixing works; this
// one is Fibonacci hashing on 32 bits).
__device__ __forceinline__ uint32_t slot_hash(int32_t k, int log2cap) {
  return ((uint32_t)k * 0x9E3779B1u) >> (32 - log2cap);
}

__host__ __device__ __forceinline__ int ceil_log2(int64_t x) {
  int r = 0;
  while (((int64_t)1 << r) < x) ++r;
  return r;
}

// Lexicographic "better" for label candidates: larger S, then larger hash.  The hash
// is a bijection of the label for a fixed key, so distinct labels never tie; the
// final comparison on the label keeps the order total for equal labels.
struct Cand {
  long long s;
  unsigned long long h;
  int l;
};
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
  if (a.s != b.s) return a.s > b.s;
  if (a.h != b.h) return a.h > b.h;
  return a.l < b.l;
}

__device__ __forceinline__ Cand warp_best(Cand c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand d;
    d.s = __shfl_xor_sync(0xffffffffu, c.s, o);
    d.h = __shfl_xor_sync(0xffffffffu, c.h, o);
    d.l = __shfl_xor_sync(0xffffffffu, c.l, o);
    if (better(d, c)) c = d;
  }
  return c;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Loads a weight stored as int32 (input graphs) or int64 (coarse graphs).
__device__ __forceinline__ long long load_w(const void* w, int wbytes, int64_t e) {
  return wbytes == 8 ? (long long)__ldg((const long long*)w + e) : (long long)__ldg((const int*)w + e);
}

// ------------------------------------------------------------ device state
// Small record in device memory that the kernels of one run read and update, so the
// host needs it only at decision points.
struct DevState {
  long long lambda_hat;   // current bound
  long long best_vertex;  // best_kind 0: original vertex of the trivial cut
  long long n, nnz;       // shape of the current graph
  long long c;            // cluster count of the last relabel
  long long pairs;        // pre-merged pair count of the last contraction
  long long dmin;         // last minimum degree
  long long argmin;       // last argmin
  int best_kind;          // 0: single original vertex, 1: snapshot over tier-1 vertices
  int improved;           // set when the last bound update improved
  int changed;            // set by PR passes / NOI rounds that merged something
  int maxdeg;             // largest list length of the current graph (clamped)
  int err;                // device-side error code (0 = ok)
  int trace_len;
  int pad[2];
};

struct TraceStep {
  int kind, level;
  long long n, nnz, lambda_hat;
};

}  // namespace vc
