// Host-side launchers of the library's kernels (one translation unit per family).
#pragma once
#include "common.cuh"

namespace vc {

// A CSR graph on the device.  Weights are int32 (input graphs, wbytes = 4) or int64
// (every contracted graph, wbytes = 8).  unit = every weight is 1: the kernels that
// support it (label propagation, pre-merge, degrees) then read no weights at all.
// simple = every list is strictly increasing (true for every contracted graph).
struct GraphView {
  int64_t n = 0, nnz = 0;
  const int64_t* off = nullptr;
  const int32_t* adj = nullptr;
  const void* w = nullptr;
  int wbytes = 8;
  bool unit = false;
  bool simple = false;  // every list strictly increasing (no parallel entries)
  // batches: label propagation touches only vertices v with vact[v] != 0 (null: all)
  const unsigned char* vact = nullptr;
  // source vertex of every entry (contracted graphs; null when not built)
  const int32_t* src = nullptr;
};

// Per-graph view of a batch (a disjoint union of graphs): vertex v belongs to graph
// gid[v]; the passes act only on graphs with gact[g] != 0, read their bound from
// glam[g] and report merges in gchanged[g].  Null in single-graph runs.
struct BatchCtx {
  const int32_t* gid = nullptr;
  const long long* glam = nullptr;
  const unsigned char* gact = nullptr;
  int* gchanged = nullptr;
};

// Weight loads for the three storage cases (UnitW: implicit weight 1).
struct UnitW {};
__device__ __forceinline__ long long ldw(const int32_t* w, int64_t e) { return (long long)__ldg(w + e); }
__device__ __forceinline__ long long ldw(const long long* w, int64_t e) { return __ldg(w + e); }
__device__ __forceinline__ long long ldw(const UnitW*, int64_t) { return 1; }

// Degree classes of one graph by neighbour-list length (see lp.cu):
//   small : length <= kWarpMaxDeg (every vertex not listed below)
//   mid   : kWarpMaxDeg < length <= kMidMaxDeg
//   block : kMidMaxDeg < length <= kBlockMaxDeg
//   global: length > kBlockMaxDeg (hash table in global scratch)
constexpr int kWarpMaxDeg = 128;
constexpr int kWarpCap = 256;
constexpr int kMidMaxDeg = 512;
constexpr int kMidCap = 1024;
constexpr int kBlockMaxDeg = 4096;
constexpr int kBlockCap = 8192;

// Vertices by list length: small (<= 64), reg (65..128), mid (129..512), block
// (513..4096), global (longer); each list in vertex order.
struct Bins {
  int32_t* small_list;   // [n]
  int32_t* reg_list;     // [n]
  int32_t* mid_list;     // [n]
  int32_t* block_list;   // [n]
  int32_t* global_list;  // [n]
  int32_t* bail_list;    // [n] mid-class lists the pre-merge's register walk handed on
  int* counts;           // device: [0] mid, [1] block, [2] global count, [3] max length above
                         // 128, [4] small, [5] reg, [7] bail count
  int h_mid = 0, h_block = 0, h_global = 0, h_maxdeg = 0, h_small = 0, h_reg = 0;  // host copies
};

// list_n not null: bins the vertices list[0, *list_n) (at most g.n of them) instead of all.
void bins_build(const GraphView& g, Bins& b, cudaStream_t s, const int32_t* list = nullptr,
                const int* list_n = nullptr);

// Scratch for the global-class tables: blocks x cap slots.
struct GlobalTables {
  int32_t* keys = nullptr;
  long long* vals = nullptr;
  int64_t cap = 0;  // slots per table (power of two)
  int blocks = 0;
};
int64_t global_table_cap(int maxdeg);

// Tie-break table of a level: hv[L] = mix64(key XOR L) for every label L < n.  With
// gid/gkey/gbase (batches) label L of graph g = gid[L] is hashed as mix64(gkey[g] XOR
// (L - gbase[g])), its id inside its own graph.
void hash_table(int64_t n, uint64_t key, const int32_t* gid, const unsigned long long* gkey, const long long* gbase,
                unsigned long long* hv, cudaStream_t s);

// Launch shapes an autotuner may change (results never depend on them).
struct LpTuning {
  int first_group = 32;  // lanes per vertex in the first round on simple graphs (8, 16, 32)
  int emit_group = 32;   // lanes per vertex in the pre-merge of the contraction (8, 16, 32)
  // rounds after the first: mid-class vertices with many distinct neighbouring labels
  // go to the hash-table kernel (pays on weakly clustered graphs, where lists carry
  // many labels; costs a launch per round elsewhere)
  bool mid_bail = false;
};

// Asynchronous rounds (optional; Sec. 4.1 in-place updates in random order, Sec. 4.3
// shuffled blocks): the n vertices form blocks of kAsyncBlock consecutive ids, ordered by
// mix64(key ^ mix64(round + 1) ^ b); the ordered blocks are cut into kAsyncWaves waves
// (the first nb % waves one block longer) that run one after another, every member of a
// wave choosing from the labels as they stand when the wave starts.  async_block_order
// writes each block's wave (wave_of, one byte per block; k0 / k1 / v0 / v1: nb elements,
// hist: radix_hist_elems(nb)); async_wave_members lists wave k (list[*count]);
// async_apply moves the members to their fresh labels, with joined (n bytes, zero at the
// round's start) applying the first round's restriction (a member that an earlier wave
// moved into keeps its label; took: cap ints).
constexpr int kAsyncBlock = 128;
constexpr int kAsyncWaves = 8;
void async_block_order(int64_t n, uint64_t key, int round, int64_t waves, unsigned long long* k0,
                       unsigned long long* k1, long long* v0, long long* v1, long long* hist, unsigned char* wave_of,
                       cudaStream_t s);
void async_wave_members(int64_t n, const unsigned char* wave_of, int k, int32_t* list, int* count, cudaStream_t s);
void async_apply(const int32_t* list, const int* count, int64_t cap, const int32_t* fresh, int32_t* lab,
                 unsigned char* joined, int32_t* took, cudaStream_t s);

// *changed += the number of v with lab_out[v] != lab_in[v] (lab_in null: the identity).
void count_changed(const int32_t* lab_in, const int32_t* lab_out, int64_t n, long long* changed, cudaStream_t s);

// One synchronous label-propagation round; lab_in == nullptr means the identity
// labelling (first round of a level).  hv: the level's tie-break table.
void lp_round(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* lab_in,
              int32_t* lab_out, const unsigned long long* hv, cudaStream_t s, const LpTuning& tune = LpTuning());

// Where the pre-merged pairs of fine vertex v go: pair i < kPairSlots at
// v kPairSlots + i of a dense strip (ckey, cval), so that readers of the few pairs of
// consecutive vertices touch consecutive memory; pair i >= kPairSlots at off[v] + i of
// (tkey, tval), which always has room (v has at most deg(v) pairs).
constexpr int kPairSlots = 4;
struct PairOut {
  int32_t* tkey;
  long long* tval;
  int32_t* ckey;
  long long* cval;
  int32_t* ccount = nullptr;  // if set: ccount[cid[v]] += the pairs of v (pairs per cluster)
  // If set: *nclust is the cluster count of this contraction (on the device), and a
  // contraction with at least nfine / 2 clusters (most clusters one or two vertices:
  // nearly every neighbour its own key) pre-merges each G-entry row of a list on its own
  // (one match per row instead of one step per distinct key); the pairs of a vertex may
  // then repeat a key across rows, which the cluster merge sums.
  const int* nclust = nullptr;
  int64_t nfine = 0;
  __device__ __forceinline__ bool by_rows() const { return nclust && 2LL * __ldg(nclust) >= nfine; }
  __device__ __forceinline__ void put(int64_t v, int64_t beg, int i, int32_t k, long long x) const {
    if (i < kPairSlots) {
      ckey[v * kPairSlots + i] = k;
      cval[v * kPairSlots + i] = x;
    } else {
      tkey[beg + i] = k;
      tval[beg + i] = x;
    }
  }
  __device__ __forceinline__ void get(int64_t v, int64_t beg, int i, int32_t* k, long long* x) const {
    if (i < kPairSlots) {
      *k = ckey[v * kPairSlots + i];
      *x = cval[v * kPairSlots + i];
    } else {
      *k = tkey[beg + i];
      *x = tval[beg + i];
    }
  }
};

// Pre-merge for contraction: for each vertex v, the distinct coarse neighbours cu =
// cid[u] != cid[v] with summed weights, cnt[v] pairs placed as PairOut says.
void emit_cross(const GraphView& g, const Bins& b, const GlobalTables& gt, const int32_t* cid, const PairOut& out,
                int32_t* cnt, cudaStream_t s, const LpTuning& tune = LpTuning());

// ------------------------------------------------------------------ contraction
struct ContractScratch {
  int32_t* flags;        // [n]
  int32_t* rank;         // [n]
  int32_t* cnt;          // [n]
  long long* pos;        // [n + 1]
  int32_t* tmp_key;      // [nnz]
  long long* tmp_val;    // [nnz]
  int32_t* cmp_key;      // [kPairSlots n]
  long long* cmp_val;    // [kPairSlots n]
  long long* scan_scr;   // scan scratch (sized for max(n, nnz))
  int* scan_scr32;
};

// Relabel: cid[v] = rank of lab[v] among the distinct labels; *c_dev = count.
void relabel(const int32_t* lab, int64_t n, int32_t* cid, ContractScratch& cs, int* c_dev, cudaStream_t s);

// The correcting step (Sec. 4.1, optional): the misplaced vertex of each cluster of 2 to
// floor(log2 n) vertices becomes a singleton (cid and *c_dev updated in place).  n-sized
// scratch: csize, bestid, flag, rank (int), dc, bestv, vout, vin (int64); moved: 1 int;
// scan_scr32: scan_scratch_elems(n) ints.
struct CorrectScratch {
  int *csize, *bestid, *flag, *rank, *moved, *scan_scr32;
  long long *dc, *bestv, *vout, *vin;
};
void correct_clusters(const GraphView& g, int32_t* cid, int* c_dev, const CorrectScratch& cs, cudaStream_t s);

// Cluster merge: a warp merges clusters of at most kMergeMax pre-merged pairs in
// registers, a block those of at most kMergeBlockMax; the few "giant" clusters beyond
// that (GiantScratch) are merged together by one radix sort of their pairs keyed by
// (giant index, target).  The pre-merge fills ccount[cid] (PairOut::ccount);
// cluster_stats reads its n entries (zero beyond the c clusters) into *maxt, *pairs and
// the giant clusters' count and pairs; cluster_merge writes the coarse CSR (coff[c + 1],
// sorted cadj, cw, entry sources csrc) and *nnz_dev; big = some cluster holds more than
// kMergeMax pairs.
constexpr int kMergeMax = 512;
constexpr int kMergeBlockMax = 4096;
struct GiantScratch {
  int ngiant = 0;      // clusters of more than kMergeBlockMax pairs
  int64_t pairs = 0;   // their pairs
  int* gcount;         // 1 int
  int32_t* glist;      // ngiant cluster ids
  int32_t* gT;         // ngiant pair counts
  long long* gstart;   // ngiant + 1 offsets into the gathered pairs
  unsigned long long *k0, *k1;  // pairs elements each
  long long *v0, *v1;
  int32_t* heads;      // pairs
  long long* hpos;     // pairs + 1
  long long* hist;     // radix_hist_elems(pairs)
};
void cluster_stats(int64_t n, const int32_t* ccount, int* maxt, long long* pairs, int* ngiant, long long* gpairs,
                   cudaStream_t s);
// Sparse contraction (most vertices alone in their cluster under their own id, on a graph
// of strictly increasing lists, see contract.cu): sparse_mark flags the merged clusters (mflag, n bytes), counts
// the coarse degree of every lone vertex it handles (sdeg[v], -1 for the others) and
// lists the others (dirty, n bytes; list[*count]) for the pre-merge.  With a SparseCtx,
// cluster_merge expects pairs from the listed vertices only (the rest with no pairs) and
// writes the handled vertices' lists itself; clean holds at least c bytes.
struct SparseCtx {
  const int32_t* cidm;  // cluster ids, sign bit set for members of merged groups (n)
  const int32_t* sdeg;
  unsigned char* clean;
  const unsigned char* dirty;  // 1: left to the pre-merge; 2: a lone list with no entry into a merged group
};
void sparse_mark(const GraphView& g, const int32_t* lab, const int32_t* cid, unsigned char* mflag, int32_t* cidm,
                 unsigned char* dirty, int32_t* sdeg, int32_t* list, int* count, cudaStream_t s);
void cluster_merge(const GraphView& g, const int32_t* cid, const ContractScratch& cs, int32_t* ccount, int64_t c,
                   long long* cbase, long long* cursor, int32_t* seg_key, long long* seg_val, int64_t* coff,
                   int32_t* cadj, long long* cw, int32_t* csrc, long long* nnz_dev, bool big, bool sort_first,
                   const GiantScratch* giant, int32_t* blist, int* blist_n, cudaStream_t s,
                   const SparseCtx* sparse = nullptr);

// Builds (cid[v] << bits | cu, weight) pairs from the pre-merged lists.
void build_pairs(const GraphView& g, const int32_t* cid, const ContractScratch& cs, int bits, int64_t pairs,
                 unsigned long long* keys, long long* vals, cudaStream_t s);

// From sorted pairs: merge equal keys, write the coarse CSR (offsets for c
// vertices).  Uses heads/hpos scratch of `pairs` elements; *nnz_dev gets the count.
void reduce_pairs(const unsigned long long* keys, const long long* vals, int64_t pairs, int bits,
                  int64_t c, int32_t* heads, long long* hpos, long long* scan_scr, int64_t* coff,
                  int32_t* cadj, long long* cw, int32_t* cv_tmp, long long* nnz_dev, cudaStream_t s);

// ------------------------------------------------------------------ bounds
void degrees(const GraphView& g, long long* deg, cudaStream_t s);
// Minimum degree with smallest argmin; if below st->lambda_hat the bound improves
// and st->improved is set (st->argmin/dmin always written).  partial: >= 1024 slots.
void bound_update(const long long* deg, int64_t n, DevState* st, long long* partial, cudaStream_t s);
// Initial bound on the input graph: lambda-hat = minimum degree, best = its argmin.
void bound_init(const long long* deg, int64_t n, DevState* st, long long* partial, cudaStream_t s);
// On improvement: side1[j] = (cur1[j] == st->argmin) and best_kind = 1.
void snapshot_side(const int32_t* cur1, int64_t n1, unsigned char* side1, DevState* st, cudaStream_t s);
void compose_map(int32_t* cur1, int64_t n1, const int32_t* cid, cudaStream_t s);
void iota(int32_t* x, int64_t n, cudaStream_t s);
// Final side bitmap of the input vertices (see side_of in bound.cu).
void side_bits2(const int32_t* orig_map, int64_t n, const unsigned char* side1, const int32_t* cur1,
                const unsigned char* sideK, const DevState* st, unsigned long long* bits, cudaStream_t s);
void trace_push(DevState* st, TraceStep* trace, int cap, int kind, int level, cudaStream_t s);

// ------------------------------------------------------------------ Padberg-Rinaldi
void pr_partners(const GraphView& g, int32_t* partner, long long* pw, long long* deg, cudaStream_t s);
// Pass A: PR1 edges and PR2 designated-partner edges, union-find, roots -> labels.
// With a batch context only active graphs are touched and `labels` must already
// hold the identity for every other vertex.
void pr_pass_a(const GraphView& g, const int32_t* partner, const long long* pw, const long long* deg,
               const DevState* st, int32_t* parent, int32_t* labels, int* changed, cudaStream_t s,
               const BatchCtx* bc = nullptr);
// Pass B: PR3 / PR4 on mutual partner pairs.
void pr_pass_b(const GraphView& g, const int32_t* partner, const long long* pw, const long long* deg,
               const DevState* st, int32_t* labels, int* changed, cudaStream_t s, const BatchCtx* bc = nullptr);

// ------------------------------------------------------------------ NOI
constexpr int kDenseMax = 512;
// All remaining rounds on a graph of n <= kDenseMax vertices inside one block.
// sideK[k] snapshots improvements over the graph's vertices (best_kind = 2).
void noi_dense(const GraphView& g, long long* M0, long long* M1, int32_t* curK, unsigned char* sideK,
               DevState* st, TraceStep* trace, int trace_cap, int level, cudaStream_t s);
// One round of the maximum-adjacency scan on a larger graph; labels = union-find roots.
// Scratch of a sparse exact-step round (r of noi_round_sparse / noi_round_batch), in
// int64 entries, for a graph (or union) of n vertices: attachments, then chunk bounds.
inline int64_t noi_round_scratch(int64_t n) { return 2 * n + 64; }
void noi_round_sparse(const GraphView& g, const DevState* st, long long* r, int* seen,
                      int32_t* parent, int32_t* labels, int* changed, cudaStream_t s);

// Per-graph result arrays of a batch's exact step (indexed by graph; trace holds
// trace_cap steps per graph).
struct BatchNoi {
  long long* lam;
  int* best_kind;
  long long* n_out;
  long long* nnz_out;
  long long* dmin;
  long long* argmin;
  int* trace_len;
  TraceStep* trace;
  int trace_cap;
  const int* level;
};
// Blocks per SM of the batches' dense exact step (512 threads and 32 registers each).
constexpr int kNoiDenseBlocksPerSM = 4;
// Dense rounds for the listed graphs of a union u (vertex range [vbase[g], +nv[g])),
// `blocks` persistent blocks with 2 x mcap matrix entries and kDenseMax curK each;
// sideK holds kDenseMax bytes per graph.
void noi_dense_batch(const GraphView& u, const int32_t* list, int count, const long long* vbase, const long long* nv,
                     long long* M, int64_t mcap, int blocks, int32_t* curK, unsigned char* sideK, const BatchNoi& bn,
                     cudaStream_t s);
// One sparse round for each listed graph; labels and gchanged written per graph.
// max_n: the largest listed graph (its state then fits in shared memory; 0 = unknown)
void noi_round_batch(const GraphView& u, const int32_t* list, int count, const long long* vbase, const long long* nv,
                     const long long* glam, long long* r, int* seen, int32_t* parent, int32_t* labels,
                     int* gchanged, int max_n, cudaStream_t s);
}  // namespace vc
