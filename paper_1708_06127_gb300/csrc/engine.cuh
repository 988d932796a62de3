// Host-side engine pieces shared by the single-graph driver and the batch driver:
// grow-only device buffers and the workspace of device arrays one run needs.
#pragma once
#include <string.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "kernels.cuh"
#include "prims.cuh"
#include "viecut.h"

namespace vc {

// Records the message of the last failure on this thread (viecut_last_error).
void set_last_error(const std::string& msg);

// Host-side fault injection for tests (viecut_debug_fail_device_allocs): true when the
// next device allocation is to fail as if cudaMalloc had run out of memory.
bool take_injected_alloc_failure();

// ------------------------------------------------------------- device buffers
struct Buf {
  void* p = nullptr;
  size_t cap = 0;
  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  ~Buf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  void* ensure(size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (bytes > cap) {
      release();
      if (take_injected_alloc_failure())
        throw Error{VIECUT_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed (injected)"};
      cudaError_t e = cudaMalloc(&p, bytes);
      if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        throw Error{VIECUT_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
      }
      cap = bytes;
    }
    return p;
  }
  template <typename T>
  T* ensure_n(int64_t count) { return (T*)ensure(sizeof(T) * (size_t)(count > 0 ? count : 1)); }
  template <typename T>
  T* as() const { return (T*)p; }
};

struct Counters {
  int c;
  int maxt;  // largest pre-merged pair count of one cluster
  long long pairs;
  int changed;
  int ngiant;         // clusters of more than kMergeBlockMax pairs
  long long gpairs;   // their pairs
  int blist_n;        // clusters listed for the block-level merge
};

enum Phase { kPhLP = 0, kPhContract, kPhPR, kPhNOI, kPhOther, kPhCount };

// Everything one run needs on the device.
struct Workspace {
  cudaStream_t s = nullptr;
  // vertex-sized
  Buf deg, labA, labB, map0, cidT, cur1, side1, flags, rank, cnt, pos, scan64, scan32, hv;
  Buf partner, pw, parent, slist, rlist, mlist, blist, glist, bl1, bcounts, noi_r, noi_seen;
  // entry-sized
  Buf tmpK, tmpV, cmpK, cmpV;
  // pair-sized
  Buf keysA, keysB, valsA, valsB, hist, heads, hpos, cvT, ccur, giantS, corrI, corrL;
  // coarse graphs (ping-pong)
  Buf coff[2], cadj[2], cw[2], csrc[2];
  // global-class tables
  Buf gkeys, gvals;
  GlobalTables gt;
  // exact step
  Buf M0, M1, curK, sideK;
  // state
  Buf state, trace, partial, counters;
  DevState* h_state = nullptr;
  Counters* h_counters = nullptr;
  int trace_cap = 4096;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> spans;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> lp_spans;
  long long lp_bytes_acc = 0, lp_nnz_acc = 0, lp_n_acc = 0;
  // contractions: device segments (the host reads the cluster and pair counts between
  // two of them, which is not device work) and the pre-merge launches alone
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ct_spans, pm_spans;
  long long ct_bytes_acc = 0, pm_bytes_acc = 0, ct_count = 0;

  Workspace() {
    VC_CUDA(cudaMallocHost(&h_state, sizeof(DevState)));
    VC_CUDA(cudaMallocHost(&h_counters, sizeof(Counters)));
    state.ensure(sizeof(DevState));
    trace.ensure_n<TraceStep>(trace_cap);
    partial.ensure_n<long long>(2 * 1024);
    counters.ensure(sizeof(Counters));
    bcounts.ensure_n<int>(8);
  }
  ~Workspace() {
    if (h_state) cudaFreeHost(h_state);
    if (h_counters) cudaFreeHost(h_counters);
    for (auto e : ev_pool) cudaEventDestroy(e);
  }
  DevState* st() { return state.as<DevState>(); }
  Counters* ctr() { return counters.as<Counters>(); }

  void ensure_vertices(int64_t n) {
    deg.ensure_n<long long>(n);
    labA.ensure_n<int32_t>(n);
    labB.ensure_n<int32_t>(n);
    hv.ensure_n<unsigned long long>(n);
    map0.ensure_n<int32_t>(n);
    cidT.ensure_n<int32_t>(n);
    cur1.ensure_n<int32_t>(n);
    side1.ensure_n<unsigned char>(n);
    flags.ensure_n<int32_t>(n);
    rank.ensure_n<int32_t>(n);
    cnt.ensure_n<int32_t>(n);
    pos.ensure_n<long long>(n + 1);
    partner.ensure_n<int32_t>(n);
    pw.ensure_n<long long>(n);
    parent.ensure_n<int32_t>(n);
    slist.ensure_n<int32_t>(n);
    rlist.ensure_n<int32_t>(n);
    bl1.ensure_n<int32_t>(n);
    cmpK.ensure_n<int32_t>(kPairSlots * n);
    cmpV.ensure_n<long long>(kPairSlots * n);
    mlist.ensure_n<int32_t>(n);
    blist.ensure_n<int32_t>(n);
    glist.ensure_n<int32_t>(n);
    scan32.ensure_n<int>(scan_scratch_elems(n) + 1);
  }
  void ensure_entries(int64_t nnz, int64_t n) {
    tmpK.ensure_n<int32_t>(nnz);
    tmpV.ensure_n<long long>(nnz);
    scan64.ensure_n<long long>(scan_scratch_elems(std::max(nnz, n)) + 1);
  }
  void ensure_noi() {
    M0.ensure_n<long long>((int64_t)kDenseMax * kDenseMax);
    M1.ensure_n<long long>((int64_t)kDenseMax * kDenseMax);
    curK.ensure_n<int32_t>(kDenseMax);
    sideK.ensure_n<unsigned char>(kDenseMax);
  }

  void sync() { VC_CUDA(cudaStreamSynchronize(s)); }
  void read_state() {
    VC_CUDA(cudaMemcpyAsync(h_state, st(), sizeof(DevState), cudaMemcpyDeviceToHost, s));
    VC_CUDA(cudaMemcpyAsync(h_counters, ctr(), sizeof(Counters), cudaMemcpyDeviceToHost, s));
    sync();
  }

  // ---------------------------------------------------------------- timing
  cudaEvent_t ev() {
    if (ev_used == ev_pool.size()) {
      cudaEvent_t e;
      VC_CUDA(cudaEventCreate(&e));
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
  cudaEvent_t mark() {
    if (!timing) return nullptr;
    cudaEvent_t e = ev();
    VC_CUDA(cudaEventRecord(e, s));
    return e;
  }
  void span(int ph, cudaEvent_t a) {
    if (!timing) return;
    spans.push_back({ph, {a, mark()}});
  }
  void reset_timing() {
    ev_used = 0;
    spans.clear();
    lp_spans.clear();
    lp_bytes_acc = lp_nnz_acc = lp_n_acc = 0;
    ct_spans.clear();
    pm_spans.clear();
    ct_bytes_acc = pm_bytes_acc = ct_count = 0;
  }

  // ---------------------------------------------------------------- launch shapes
  // Lanes per vertex of the first-round and pre-merge kernels, picked once per
  // workspace by timing each candidate on the first graph large enough to tell them
  // apart.  Every candidate writes the same output, so a trial run is repeated work.
  LpTuning tune;
  bool tuned_first = false, tuned_emit = false;
  static constexpr int64_t kTuneMinN = int64_t(1) << 16;

  template <typename F>
  int pick_group(F run) {
    cudaEvent_t a, b;
    VC_CUDA(cudaEventCreate(&a));
    VC_CUDA(cudaEventCreate(&b));
    float best = 3.0e38f;
    int pick = 32;
    for (int G : {32, 16, 8}) {
      run(G);  // warm-up
      float t = 3.0e38f;
      for (int rep = 0; rep < 2; ++rep) {
        VC_CUDA(cudaEventRecord(a, s));
        run(G);
        VC_CUDA(cudaEventRecord(b, s));
        VC_CUDA(cudaEventSynchronize(b));
        float ms = 0;
        VC_CUDA(cudaEventElapsedTime(&ms, a, b));
        t = std::min(t, ms);
      }
      if (t < best) { best = t; pick = G; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return pick;
  }
  // Fixed choices from the caller's options (0 keeps the timed pick).
  void fix_groups(int lp_group, int emit_group) {
    auto ok = [](int G) { return G == 0 || G == 8 || G == 16 || G == 32; };
    if (!ok(lp_group) || !ok(emit_group)) throw Error{VIECUT_EINVAL, "lp_group and emit_group must be 0, 8, 16 or 32"};
    if (lp_group) { tune.first_group = lp_group; tuned_first = true; }
    if (emit_group) { tune.emit_group = emit_group; tuned_emit = true; }
  }
  void tune_first(const GraphView& g, int32_t* out) {
    if (tuned_first || !g.simple || g.n < kTuneMinN) return;
    tuned_first = true;
    const unsigned long long* h = hv.as<unsigned long long>();
    tune.first_group = pick_group([&](int G) {
      LpTuning t = tune;
      t.first_group = G;
      lp_round(g, bins, gt, nullptr, out, h, s, t);
    });
  }
  void tune_emit(const GraphView& g, const int32_t* cid, const PairOut& po, int32_t* c) {
    if (tuned_emit || g.n < kTuneMinN || bins.h_block == 0) return;
    tuned_emit = true;
    tune.emit_group = pick_group([&](int G) {
      LpTuning t = tune;
      t.emit_group = G;
      emit_cross(g, bins, gt, cid, po, c, s, t);
    });
  }

  // ---------------------------------------------------------------- steps
  Bins bins;
  bool bins_valid = false;

  // Reads the class counts of bins b (and counts[6] into *extra when given) and sizes
  // the global-class tables for its longest list.
  void read_bins(Bins& b, int* extra = nullptr) {
    int hc[7];
    VC_CUDA(cudaMemcpyAsync(hc, b.counts, (extra ? 7 : 6) * sizeof(int), cudaMemcpyDeviceToHost, s));
    sync();
    b.h_mid = hc[0];
    b.h_block = hc[1];
    b.h_global = hc[2];
    b.h_maxdeg = hc[3];
    b.h_small = hc[4];
    b.h_reg = hc[5];
    if (extra) *extra = hc[6];
    if (b.h_global > 0) {
      int64_t cap = global_table_cap(b.h_maxdeg);
      int blocks = std::min(b.h_global, kSMs);
      // keep the scratch under ~2 GiB
      while (blocks > 1 && (int64_t)blocks * cap * 12 > (int64_t(2) << 30)) blocks /= 2;
      gt.keys = gkeys.ensure_n<int32_t>(blocks * cap);
      gt.vals = gvals.ensure_n<long long>(blocks * cap);
      gt.cap = cap;
      gt.blocks = blocks;
    }
  }

  void build_bins(const GraphView& g) {
    bins.small_list = slist.as<int32_t>();
    bins.reg_list = rlist.as<int32_t>();
    bins.mid_list = mlist.as<int32_t>();
    bins.block_list = blist.as<int32_t>();
    bins.global_list = glist.as<int32_t>();
    bins.bail_list = bl1.as<int32_t>();
    bins.counts = bcounts.as<int>();
    bins_build(g, bins, s);
    read_bins(bins);
    bins_valid = true;
  }

  // Sparse contraction by union-find roots: counts the coarse lists of the lone vertices
  // it handles and bins the others (members of merged groups, lone vertices with too
  // many entries into them).  True when those are at most half of g's vertices; then
  // dbins holds their bins.
  Bins dbins;
  Buf smflag, scidm, sdirty, sdeg, sclean, sdlist, dsl, drl, dml, dbl, dgl, dbail, dcounts;
  // dbins' lists, for at most n listed vertices
  void prepare_dbins(int64_t n) {
    dbins.small_list = dsl.ensure_n<int32_t>(n);
    dbins.reg_list = drl.ensure_n<int32_t>(n);
    dbins.mid_list = dml.ensure_n<int32_t>(n);
    dbins.block_list = dbl.ensure_n<int32_t>(n);
    dbins.global_list = dgl.ensure_n<int32_t>(n);
    dbins.bail_list = dbail.ensure_n<int32_t>(n);
    dbins.counts = dcounts.ensure_n<int>(8);
  }

  bool mark_sparse(const GraphView& g, const int32_t* labels, const int32_t* cid) {
    const int64_t n = g.n;
    prepare_dbins(n);
    int32_t* list = sdlist.ensure_n<int32_t>(n);
    sparse_mark(g, labels, cid, smflag.ensure_n<unsigned char>(n), scidm.ensure_n<int32_t>(n),
                sdirty.ensure_n<unsigned char>(n), sdeg.ensure_n<int32_t>(n), list, dbins.counts + 6, s);
    bins_build(g, dbins, s, list, dbins.counts + 6);
    int ndirty = 0;
    read_bins(dbins, &ndirty);
    sclean.ensure_n<unsigned char>(n);
    return 2 * (int64_t)ndirty <= n;
  }

  // Asynchronous rounds (lp_async 1, or 2 with the first round's restriction; see
  // async_block_order): the waves of each round run one after another, each binned and
  // propagated on its own members, then applied in place.
  Buf asK, asV, asH, asWave, asJoined, asTook, labC;
  void lp_rounds_async(const GraphView& g, uint64_t key, int rounds, int32_t** out_labels, bool converge,
                       int lp_async) {
    const int64_t n = g.n;
    int32_t* A = labA.as<int32_t>();
    int32_t* B = labB.as<int32_t>();
    iota(A, n, s);
    hash_table(n, key, nullptr, nullptr, nullptr, hv.as<unsigned long long>(), s);
    const int64_t nb = (n + kAsyncBlock - 1) / kAsyncBlock;
    const int64_t waves = std::min<int64_t>(kAsyncWaves, nb);
    auto* k0 = asK.ensure_n<unsigned long long>(2 * nb);
    auto* v0 = asV.ensure_n<long long>(2 * nb);
    long long* hist = asH.ensure_n<long long>(radix_hist_elems(nb));
    unsigned char* wave_of = asWave.ensure_n<unsigned char>(nb);
    unsigned char* joined = asJoined.ensure_n<unsigned char>(n);
    int32_t* took = asTook.ensure_n<int32_t>(n);
    int32_t* C = labC.ensure_n<int32_t>(n);
    prepare_dbins(n);
    int32_t* list = sdlist.ensure_n<int32_t>(n);
    int* count = dbins.counts + 6;
    for (int r = 0; r < rounds; ++r) {
      cudaEvent_t a = mark();
      if (converge) VC_CUDA(cudaMemcpyAsync(C, A, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, s));
      async_block_order(n, key, r, waves, k0, k0 + nb, v0, v0 + nb, hist, wave_of, s);
      const bool restrict_now = lp_async == 2 && r == 0;
      if (restrict_now) VC_CUDA(cudaMemsetAsync(joined, 0, (size_t)n, s));
      for (int k = 0; k < waves; ++k) {
        async_wave_members(n, wave_of, k, list, count, s);
        bins_build(g, dbins, s, list, count);
        read_bins(dbins);
        lp_round(g, dbins, gt, A, B, hv.as<unsigned long long>(), s, tune);
        async_apply(list, count, n, B, A, restrict_now ? joined : nullptr, took, s);
      }
      if (timing) {
        lp_spans.push_back({a, mark()});
        lp_bytes_acc += 8 * (n + 1) + g.nnz * (4 + (g.unit ? 0 : g.wbytes) + 4) + 4 * n;
        lp_nnz_acc += g.nnz;
        lp_n_acc += n;
      }
      if (converge) {
        long long* cnt = &ctr()->gpairs;  // free during label propagation
        VC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(long long), s));
        count_changed(C, A, n, cnt, s);
        long long changed = 0;
        VC_CUDA(cudaMemcpyAsync(&changed, cnt, sizeof(long long), cudaMemcpyDeviceToHost, s));
        sync();
        if (changed * 10000 <= n) break;
      }
    }
    *out_labels = A;
  }

  // `rounds` rounds; with converge, they end after the first round that changed at most
  // n / 10000 labels (one count and host read per round).
  void lp_rounds(const GraphView& g, uint64_t key, int rounds, int32_t** out_labels, int32_t* all_out,
                 bool converge = false, int lp_async = 0) {
    if (lp_async) {
      lp_rounds_async(g, key, rounds, out_labels, converge, lp_async);
      return;
    }
    int32_t* in = nullptr;
    int32_t* bufs[2] = {labA.as<int32_t>(), labB.as<int32_t>()};
    hash_table(g.n, key, nullptr, nullptr, nullptr, hv.as<unsigned long long>(), s);
    for (int r = 0; r < rounds; ++r) {
      int32_t* out = bufs[r & 1];
      if (!in) tune_first(g, out);
      cudaEvent_t a = mark();
      lp_round(g, bins, gt, in, out, hv.as<unsigned long long>(), s, tune);
      if (timing) {
        lp_spans.push_back({a, mark()});
        long long gather = in ? 4 : 0;
        lp_bytes_acc += 8 * (g.n + 1) + g.nnz * (4 + (g.unit ? 0 : g.wbytes) + gather) + 4 * g.n;
        lp_nnz_acc += g.nnz;
        lp_n_acc += g.n;
      }
      if (all_out)
        VC_CUDA(cudaMemcpyAsync(all_out + (int64_t)r * g.n, out, sizeof(int32_t) * g.n, cudaMemcpyDeviceToHost, s));
      const int32_t* prev = in;
      in = out;
      if (converge) {
        long long* cnt = &ctr()->gpairs;  // free during label propagation
        VC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(long long), s));
        count_changed(prev, out, g.n, cnt, s);
        long long changed = 0;
        VC_CUDA(cudaMemcpyAsync(&changed, cnt, sizeof(long long), cudaMemcpyDeviceToHost, s));
        sync();
        if (changed * 10000 <= g.n) break;
      }
    }
    *out_labels = in;
  }

  // Algorithmic bytes of one contraction of fine graph g into (cn vertices, cnnz
  // entries): the fine CSR read once (offsets, ids, weights unless all are 1), the
  // labels read and the cluster ids written (4 bytes per vertex each), the cluster id
  // of every neighbour gathered (4 bytes per entry), and the coarse CSR written
  // (offsets, int32 ids, int64 weights).
  void count_contract(const GraphView& g, int64_t cn, int64_t cnnz) {
    if (!timing) return;
    ct_bytes_acc += 8 * (g.n + 1) + g.nnz * (4 + (g.unit ? 0 : g.wbytes) + 4) + 8 * g.n + 8 * (cn + 1) + 12 * cnnz;
  }

  // Contracts g by labels into the coarse buffer `slot`; cid_out[n] receives the map.
  // Returns the coarse view; h_counters holds c and the pair count afterwards.
  // sparse_ok: try the sparse contraction on a graph of strictly increasing lists: a
  // vertex labelled by its own id and alone in its cluster ("lone": the cluster ids of
  // such vertices rise with their ids) is handled by a renumbering copy of its list.  It
  // pays when most vertices are lone (Padberg-Rinaldi passes, weakly clustered levels);
  // it is taken only when at most half of the vertices are left to the pre-merge.
  GraphView contract(const GraphView& g, const int32_t* labels, int32_t* cid_out, int slot, bool correct = false,
                     bool sparse_ok = false) {
    cudaEvent_t t0 = mark();
    ContractScratch cs;
    cs.flags = flags.as<int32_t>();
    cs.rank = rank.as<int32_t>();
    cs.cnt = cnt.as<int32_t>();
    cs.pos = pos.as<long long>();
    cs.tmp_key = tmpK.as<int32_t>();
    cs.tmp_val = tmpV.as<long long>();
    cs.cmp_key = cmpK.as<int32_t>();
    cs.cmp_val = cmpV.as<long long>();
    cs.scan_scr = scan64.as<long long>();
    cs.scan_scr32 = scan32.as<int>();
    relabel(labels, g.n, cid_out, cs, &ctr()->c, s);
    if (correct) {
      CorrectScratch cr;
      int* ci = corrI.ensure_n<int>(4 * g.n + 1);
      long long* cl = corrL.ensure_n<long long>(4 * g.n);
      cr.csize = ci;
      cr.bestid = ci + g.n;
      cr.flag = ci + 2 * g.n;
      cr.rank = ci + 3 * g.n;
      cr.moved = ci + 4 * g.n;
      cr.scan_scr32 = scan32.as<int>();
      cr.dc = cl;
      cr.bestv = cl + g.n;
      cr.vout = cl + 2 * g.n;
      cr.vin = cl + 3 * g.n;
      correct_clusters(g, cid_out, &ctr()->c, cr, s);
    }
    const bool sparse = sparse_ok && !correct && g.simple && g.n > 0 && mark_sparse(g, labels, cid_out);
    if (!sparse && !bins_valid) build_bins(g);
    const Bins& B = sparse ? dbins : bins;
    PairOut po{cs.tmp_key, cs.tmp_val, cs.cmp_key, cs.cmp_val};
    po.nclust = &ctr()->c;
    po.nfine = g.n;
    if (!sparse) tune_emit(g, cid_out, po, cs.cnt);  // trials: no counting
    // the pre-merge also counts pairs per cluster (flags is free again after the relabel)
    int32_t* ccount = cs.flags;
    VC_CUDA(cudaMemsetAsync(ccount, 0, sizeof(int32_t) * std::max<int64_t>(g.n, 1), s));
    if (sparse) VC_CUDA(cudaMemsetAsync(cs.cnt, 0, sizeof(int32_t) * g.n, s));  // clean vertices: no pairs
    po.ccount = ccount;
    cudaEvent_t e0 = mark();
    emit_cross(g, B, gt, cid_out, po, cs.cnt, s, tune);
    if (timing && !sparse) pm_spans.push_back({e0, mark()});  // the whole graph's pre-merge only
    VC_CUDA(cudaMemsetAsync(&ctr()->maxt, 0, sizeof(int), s));
    VC_CUDA(cudaMemsetAsync(&ctr()->pairs, 0, sizeof(long long), s));
    VC_CUDA(cudaMemsetAsync(&ctr()->ngiant, 0, sizeof(int), s));
    VC_CUDA(cudaMemsetAsync(&ctr()->gpairs, 0, sizeof(long long), s));
    cluster_stats(g.n, ccount, &ctr()->maxt, &ctr()->pairs, &ctr()->ngiant, &ctr()->gpairs, s);
    if (timing) ct_spans.push_back({t0, mark()});
    VC_CUDA(cudaMemcpyAsync(h_counters, ctr(), sizeof(Counters), cudaMemcpyDeviceToHost, s));
    sync();
    cudaEvent_t t1 = mark();
    const int64_t c = h_counters->c;
    const int64_t P = h_counters->pairs;
    if (timing) {
      // pre-merge: offsets, ids, weights (none when all are 1), the cluster id of every
      // neighbour and of v, the pair count of v and the pairs (int32 key + int64 sum)
      if (!sparse) pm_bytes_acc += 8 * (g.n + 1) + g.nnz * (4 + (g.unit ? 0 : g.wbytes) + 4) + 4 * g.n + 4 * g.n + 12 * P;
      ct_count += 1;
    }
    // coarse entries: at most the pairs, plus (sparse) the clean vertices' copied lists;
    // never more than the fine entries
    const int64_t E = sparse ? std::max<int64_t>(P, g.nnz) : P;
    int64_t* co = coff[slot].ensure_n<int64_t>(c + 1);
    int32_t* ca = cadj[slot].ensure_n<int32_t>(std::max<int64_t>(E, 1));
    long long* cwp = cw[slot].ensure_n<long long>(std::max<int64_t>(E, 1));
    int32_t* csp = csrc[slot].ensure_n<int32_t>(std::max<int64_t>(E, 1));
    // the cluster merge, with the few giant clusters radix-sorted together, unless
    // those hold most of the pairs (then one radix sort of all pairs)
    const int ng = h_counters->maxt > kMergeBlockMax ? h_counters->ngiant : 0;
    const int64_t GP = ng ? h_counters->gpairs : 0;
    if (2 * GP <= P || sparse) {
      long long* cbase = pos.as<long long>();  // n + 1 >= c + 1 entries
      long long* cur = ccur.ensure_n<long long>(std::max<int64_t>(c, 1));
      auto* sk = (int32_t*)keysA.ensure_n<unsigned long long>(std::max<int64_t>(P, 1));
      auto* sv = valsA.ensure_n<long long>(std::max<int64_t>(P, 1));
      scan64.ensure_n<long long>(scan_scratch_elems(std::max<int64_t>(std::max(c, GP), 1)) + 1);
      cs.scan_scr = scan64.as<long long>();
      GiantScratch gs;
      if (ng) {
        gs.ngiant = ng;
        gs.pairs = GP;
        auto* small = giantS.ensure_n<long long>(2 * ng + 4);
        gs.gstart = small;                               // ng + 1
        gs.gcount = (int*)(small + ng + 1);              // 1
        gs.glist = (int32_t*)(small + ng + 2);           // ng ints in ng / 2 + 1 slots
        gs.gT = gs.glist + ng + (ng & 1);                // ng ints
        gs.k0 = keysB.ensure_n<unsigned long long>(2 * GP);
        gs.k1 = gs.k0 + GP;
        gs.v0 = valsB.ensure_n<long long>(2 * GP);
        gs.v1 = gs.v0 + GP;
        gs.heads = heads.ensure_n<int32_t>(GP);
        gs.hpos = hpos.ensure_n<long long>(GP + 1);
        gs.hist = hist.ensure_n<long long>(radix_hist_elems(GP));
      }
      const SparseCtx sp{scidm.as<int32_t>(), sdeg.as<int32_t>(), sclean.as<unsigned char>(),
                         sdirty.as<unsigned char>()};
      cluster_merge(g, cid_out, cs, ccount, c, cbase, cur, sk, sv, co, ca, cwp, csp, &st()->nnz,
                    h_counters->maxt > kMergeMax, 2 * c >= g.n, ng ? &gs : nullptr, cs.cnt, &ctr()->blist_n, s,
                    sparse ? &sp : nullptr);
    } else {
      exclusive_scan<int, long long>(cs.cnt, cs.pos, g.n, &ctr()->pairs, cs.scan_scr, s);
      int bits = ceil_log2(c);
      if (bits < 1) bits = 1;
      auto* kA = keysA.ensure_n<unsigned long long>(P);
      auto* kB = keysB.ensure_n<unsigned long long>(P);
      auto* vA = valsA.ensure_n<long long>(P);
      auto* vB = valsB.ensure_n<long long>(P);
      auto* hs = hist.ensure_n<long long>(radix_hist_elems(P));
      auto* hd = heads.ensure_n<int32_t>(P);
      auto* hp = hpos.ensure_n<long long>(P + 1);
      scan64.ensure_n<long long>(scan_scratch_elems(std::max<int64_t>(P, 1)) + 1);
      build_pairs(g, cid_out, cs, bits, P, kA, vA, s);
      radix_sort_pairs(kA, vA, kB, vB, P, 2 * bits, hs, s);
      reduce_pairs(kA, vA, P, bits, c, hd, hp, scan64.as<long long>(), co, ca, cwp, csp, &st()->nnz, s);
    }
    if (timing) ct_spans.push_back({t1, mark()});
    GraphView h;
    h.n = c;
    h.nnz = E;  // upper bound until the state is read
    h.off = co;
    h.adj = ca;
    h.w = cwp;
    h.src = csp;
    h.wbytes = 8;
    h.simple = true;
    bins_valid = false;
    return h;
  }
};

}  // namespace vc

#define VC_API_BEGIN try {
#define VC_API_END                                   \
  }                                                  \
  catch (const vc::Error& e) {                       \
    vc::set_last_error(e.msg);                       \
    return e.code;                                   \
  }                                                  \
  catch (const std::bad_alloc&) {                    \
    vc::set_last_error("host allocation failed");    \
    return VIECUT_ENOMEM;                            \
  }                                                  \
  return VIECUT_OK;
