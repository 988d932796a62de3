// Distinct-key aggregation in registers (shared by label propagation, the
// contraction pre-merge and the cluster merge).  A group of G lanes holds a list of
// at most S G (key, weight) entries, slot r of group lane i holding entry G r + i,
// and visits its distinct keys one at a time: one lane with an unvisited entry
// broadcasts that entry's key, every lane marks its entries holding it, and a group
// reduction gives the key's count (unit weights) or weight sum.  The groups of a warp
// step in lockstep, so warp-wide votes and shuffles always have every lane present.
#pragma once
#include <type_traits>

#include "kernels.cuh"

namespace vc {

template <int G>
__device__ __forceinline__ unsigned group_mask(int lane) {
  return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
}

template <int S>
struct RegList {
  int32_t k[S];
  long long wt[S];
  unsigned todo;  // bit r: slot r holds a used entry not yet visited
  int slots;      // slots in use: ceil(deg / G), the same in every lane of the group
};

// Lists of at most kVoteAllMaxS slots per lane take a key per step from any slot (one
// vote per step, no empty pass per slot; a lane finds its lowest unvisited slot with
// S - 1 selects); longer lists go slot by slot, where the selects would cost more
// than the empty passes they save.
constexpr int kVoteAllMaxS = 4;

// Calls visit(key, total) once per distinct used key of the group's list; total is
// the same in the group's lanes.  The order of the visits is not a contract: callers
// keep a total order over keys or sort afterwards.  A visit returning true ends the
// group's walk (its remaining keys are not visited).  Every lane of the warp must
// call it (groups without a list pass slots = todo = 0).
template <typename WT, typename ACC, int G, int S, typename F>
__device__ __forceinline__ void reg_visit(RegList<S>& L, unsigned gmask, F visit) {
  // one step: key kk (held by the group's first lane of the vote when gb != 0) is
  // marked visited in every slot >= r0 holding it, and visited with its total
  auto step = [&](unsigned gb, int32_t kk, int r0) {
    unsigned hit = 0;
#pragma unroll
    for (int q = 0; q < S; ++q)
      if (q >= r0 && L.k[q] == kk) hit |= 1u << q;
    hit = gb ? hit & L.todo : 0u;
    L.todo &= ~hit;
    ACC total;
    if (std::is_same<WT, UnitW>::value) {
      total = (ACC)__reduce_add_sync(gmask, (unsigned)__popc(hit));
    } else {
      long long sum = 0;
#pragma unroll
      for (int q = 0; q < S; ++q)
        if (hit >> q & 1u) sum += L.wt[q];
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      total = (ACC)sum;
    }
    if (gb && visit(kk, total)) L.todo = 0;
  };
  if (S <= kVoteAllMaxS) {
    for (;;) {
      const unsigned bal = __ballot_sync(0xffffffffu, L.todo != 0u);
      if (!bal) break;
      const unsigned gb = bal & gmask;
      int32_t lowest = L.k[S - 1];
#pragma unroll
      for (int q = S - 2; q >= 0; --q)
        if ((L.todo >> q) & 1u) lowest = L.k[q];
      step(gb, __shfl_sync(0xffffffffu, lowest, gb ? __ffs(gb) - 1 : 0), 0);
    }
  } else {
    // slot r's first occurrences in lane order; a key first seen in slot r sits in no
    // slot below r
    const int slots = (int)__reduce_max_sync(0xffffffffu, (unsigned)L.slots);  // the warp's longest list
#pragma unroll
    for (int r = 0; r < S; ++r) {
      if (r >= slots) break;
      for (;;) {
        const unsigned bal = __ballot_sync(0xffffffffu, (L.todo >> r) & 1u);
        if (!bal) break;
        const unsigned gb = bal & gmask;
        step(gb, __shfl_sync(0xffffffffu, L.k[r], gb ? __ffs(gb) - 1 : 0), r);
      }
    }
  }
}

}  // namespace vc
