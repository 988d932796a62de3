// Host driver and C ABI of the GB300 VieCut library.
//
// Algorithm 1 of the paper (Appendix A) in the deterministic variant that
// include/viecut.h describes: levels of label propagation + cluster contraction +
// Padberg-Rinaldi runs while more than n0 vertices remain, then the exact step of
// Nagamochi, Ono and Ibaraki, with the trivial-cut bound tracked after every
// contraction.  Every step runs in this library's CUDA kernels; the host only
// sequences launches and reads a small state record at decision points.
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "engine.cuh"

namespace vc {

std::atomic<unsigned long long> g_launches{0};
static thread_local std::string t_last_error;
void set_last_error(const std::string& msg) { t_last_error = msg; }

// Injected allocation failures: the allocations after the next g_fail_skip ones fail,
// g_fail_count of them (process-wide, every thread).
static std::atomic<long long> g_fail_skip{0}, g_fail_count{0};
bool take_injected_alloc_failure() {
  if (g_fail_count.load() <= 0) return false;
  long long sk = g_fail_skip.load();
  while (sk > 0)
    if (g_fail_skip.compare_exchange_weak(sk, sk - 1)) return false;
  long long c = g_fail_count.load();
  while (c > 0)
    if (g_fail_count.compare_exchange_weak(c, c - 1)) return true;
  return false;
}

__global__ void set_n_k(DevState* st, long long n) { st->n = n; }

__global__ void validate_k(int64_t n, int64_t m, const int64_t* __restrict__ off, const int32_t* __restrict__ adj,
                           const int32_t* __restrict__ w, int* err) {
  int bad = 0;
  const int64_t T = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0 && (off[0] != 0 || off[n] != m)) bad |= 1;
  for (int64_t v = t0; v < n; v += T)
    if (off[v + 1] < off[v]) bad |= 2;
  // per-entry checks need the owning vertex for self-loops: warp per vertex
  const int lane = threadIdx.x & 31;
  const int64_t W = T >> 5;
  for (int64_t v = t0 >> 5; v < n; v += W) {
    int64_t a = off[v], b = off[v + 1];
    if (a < 0 || b > m || a > b) { bad |= 2; continue; }
    for (int64_t e = a + lane; e < b; e += 32) {
      int32_t u = adj[e];
      if (u < 0 || u >= n) bad |= 4;
      else if (u == v) bad |= 8;
      if (w) {  // null: the weights are checked apart (weight_check_k)
        if (w[e] < 1) bad |= 16;
        if (w[e] != 1) bad |= 32;  // not an error: the weights are not all 1
      }
      if (e + 1 < b && adj[e + 1] <= u) bad |= 64;  // not an error: a list is not strictly increasing
    }
  }
  if (bad) atomicOr(err, bad);
}

// Weights alone, an entry per thread: 16 = a weight < 1, 32 = not all weights 1.
__global__ void weight_check_k(int64_t m, const int32_t* __restrict__ w, int* err) {
  int bad = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = w[e];
    if (x < 1) bad |= 16;
    if (x != 1) bad |= 32;
  }
  bad = (int)__reduce_or_sync(0xffffffffu, (unsigned)bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(err, bad);
}

struct Handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0, m = 0;
  int64_t n0 = 10000;
  int pr_runs_max = 8;
  int validate = 1;
  bool correct = false;  // the correcting step on label-propagation clusterings
  bool lp_converge = false;  // rounds end once at most 1/10000 of the labels changed
  int lp_async = 0;          // asynchronous rounds in shuffled blocks (2: with the first round's restriction)
  bool unit = false;    // every input weight is 1 (found by validation)
  bool simple = false;  // every input list strictly increasing (found by validation)
  bool host_input = false;  // the graph was copied from host arrays into in_*
  bool bound = false;       // a graph passed validation and may run
  cudaStream_t cstream = nullptr;  // viecut_solve: the weights' copy and check
  cudaEvent_t wdone = nullptr;
  Buf werr;
  const int64_t* off0 = nullptr;
  const int32_t* adj0 = nullptr;
  const int32_t* w0 = nullptr;
  Buf in_off, in_adj, in_w, out_cut, out_bits;
  Workspace* ws = nullptr;
  viecut_stats stats{};
  std::vector<viecut_step> last_trace;
  ~Handle() {
    delete ws;
    if (wdone) cudaEventDestroy(wdone);
    if (cstream) cudaStreamDestroy(cstream);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

// with_weights = false: the weights are checked apart (viecut_solve); unit is then
// left as the caller set it.
static void device_validate(Handle& H, bool with_weights = true) {
  Workspace& W = *H.ws;
  int* err = &W.ctr()->changed;
  VC_CUDA(cudaMemsetAsync(err, 0, sizeof(int), H.stream));
  validate_k<<<grid_for(H.n, 256, kSMs * 8), 256, 0, H.stream>>>(H.n, H.m, H.off0, H.adj0,
                                                                with_weights ? H.w0 : nullptr, err);
  count_launch();
  VC_CHECK_LAUNCH();
  W.read_state();
  int bad = W.h_counters->changed;
  if (with_weights) H.unit = (bad & 32) == 0;
  H.simple = (bad & 64) == 0;
  bad &= ~(32 | 64);
  if (bad) {
    std::string why;
    if (bad & 1) why += " offsets[0] != 0 or offsets[n] != m;";
    if (bad & 2) why += " offsets decrease or leave [0, m];";
    if (bad & 4) why += " neighbour id out of range;";
    if (bad & 8) why += " self-loop;";
    if (bad & 16) why += " weight < 1;";
    throw Error{VIECUT_EINVAL, "invalid graph:" + why};
  }
}

// Returns true when every weight is 1; *simple = every list strictly increasing.
static bool host_validate(const int64_t* off, const int32_t* adj, const int32_t* w, int64_t n, int64_t m,
                          bool symmetric, bool* simple) {
  bool unit = true;
  *simple = true;
  if (off[0] != 0 || off[n] != m) throw Error{VIECUT_EINVAL, "invalid graph: offsets[0] != 0 or offsets[n] != m"};
  for (int64_t v = 0; v < n; ++v) {
    if (off[v + 1] < off[v]) throw Error{VIECUT_EINVAL, "invalid graph: offsets decrease at vertex " + std::to_string(v)};
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      if (adj[e] < 0 || adj[e] >= n) throw Error{VIECUT_EINVAL, "invalid graph: neighbour id out of range"};
      if (adj[e] == v) throw Error{VIECUT_EINVAL, "invalid graph: self-loop at vertex " + std::to_string(v)};
      if (w[e] < 1) throw Error{VIECUT_EINVAL, "invalid graph: weight < 1"};
      unit = unit && w[e] == 1;
      if (e + 1 < off[v + 1] && adj[e + 1] <= adj[e]) *simple = false;
    }
  }
  if (!symmetric) return unit;
  struct E { int64_t a, b; int32_t w; };
  std::vector<E> fwd, bwd;
  fwd.reserve(m);
  bwd.reserve(m);
  for (int64_t v = 0; v < n; ++v)
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      fwd.push_back({v, adj[e], w[e]});
      bwd.push_back({adj[e], v, w[e]});
    }
  auto lt = [](const E& x, const E& y) { return x.a < y.a || (x.a == y.a && (x.b < y.b || (x.b == y.b && x.w < y.w))); };
  std::sort(fwd.begin(), fwd.end(), lt);
  std::sort(bwd.begin(), bwd.end(), lt);
  for (int64_t i = 0; i < m; ++i)
    if (fwd[i].a != bwd[i].a || fwd[i].b != bwd[i].b || fwd[i].w != bwd[i].w)
      throw Error{VIECUT_EINVAL, "invalid graph: not symmetric (edge weights must match in both directions)"};
  return unit;
}

// ------------------------------------------------------------------- the run
static void run_impl(Handle& H, uint64_t seed, int lp_iters, long long* d_cut, unsigned long long* d_bits) {
  if (lp_iters < 0) throw Error{VIECUT_EINVAL, "lp_iters must be >= 0"};
  if (!H.bound) throw Error{VIECUT_EINVAL, "the handle holds no valid graph (its last viecut_load failed)"};
  Workspace& W = *H.ws;
  W.s = H.stream;
  cudaStream_t s = H.stream;
  const unsigned long long launches0 = g_launches;
  W.reset_timing();
  cudaEvent_t t_start = W.mark();
  DevState init{};
  init.n = H.n;
  init.nnz = H.m;
  VC_CUDA(cudaMemcpyAsync(W.st(), &init, sizeof(DevState), cudaMemcpyHostToDevice, s));
  VC_CUDA(cudaMemsetAsync(W.ctr(), 0, sizeof(Counters), s));
  DevState* st = W.st();
  TraceStep* tr = W.trace.as<TraceStep>();
  const int tcap = W.trace_cap;

  GraphView G;
  G.n = H.n;
  G.nnz = H.m;
  G.off = H.off0;
  G.adj = H.adj0;
  G.w = H.w0;
  G.wbytes = 4;
  G.unit = H.unit;
  G.simple = H.simple;
  W.bins_valid = false;

  cudaEvent_t a = W.mark();
  degrees(G, W.deg.as<long long>(), s);
  bound_init(W.deg.as<long long>(), G.n, st, W.partial.as<long long>(), s);
  trace_push(st, tr, tcap, 0, 0, s);
  W.span(kPhOther, a);
  W.read_state();

  int level = 0;
  int slot = -1;          // coarse buffer holding G (-1: the input)
  bool contracted = false;
  int64_t n1 = 0;         // tier-1 vertex count
  int64_t levels = 0;
  bool done = W.h_state->lambda_hat == 0;
  // W.partner / W.pw / W.deg hold the partners of the current G (a pass that merged
  // nothing leaves G, and so them, as they were)
  bool partners_ok = false;

  // contraction + bound update; returns false when the run ends
  auto step = [&](const int32_t* labels, int kind) -> bool {
    cudaEvent_t a0 = W.mark();
    int32_t* cid = contracted ? W.cidT.as<int32_t>() : W.map0.as<int32_t>();
    int dst = slot == 0 ? 1 : 0;
    const GraphView fine = G;
    // the sparse contraction for Padberg-Rinaldi passes and for levels the last one did
    // not halve (most vertices keep their own label there)
    GraphView h = W.contract(G, labels, cid, dst, kind == 1 && H.correct, kind >= 2 || W.tune.mid_bail);
    set_n_k<<<1, 1, 0, s>>>(st, h.n);
    count_launch();
    if (!contracted) {
      n1 = h.n;
      iota(W.cur1.as<int32_t>(), n1, s);
      contracted = true;
    } else {
      compose_map(W.cur1.as<int32_t>(), n1, cid, s);
    }
    G = h;
    slot = dst;
    W.span(kPhContract, a0);
    cudaEvent_t a1 = W.mark();
    partners_ok = false;
    if (G.n > 1) {
      // the weighted degrees for the bound, with the partners the next Padberg-Rinaldi
      // pass reads (the same scan of every list)
      pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
      partners_ok = true;
      bound_update(W.deg.as<long long>(), G.n, st, W.partial.as<long long>(), s);
      snapshot_side(W.cur1.as<int32_t>(), n1, W.side1.as<unsigned char>(), st, s);
    }
    trace_push(st, tr, tcap, kind, level, s);
    W.span(kPhOther, a1);
    W.read_state();
    G.nnz = W.h_state->nnz;
    W.count_contract(fine, G.n, G.nnz);
    return G.n > 1 && W.h_state->lambda_hat > 0;
  };

  auto read_changed = [&]() -> int {
    VC_CUDA(cudaMemcpyAsync(&W.h_counters->changed, &W.ctr()->changed, sizeof(int), cudaMemcpyDeviceToHost, s));
    W.sync();
    return W.h_counters->changed;
  };

  int64_t n_prev_level = 0;
  while (!done && G.n > H.n0) {
    const int64_t n_start = G.n;
    const uint64_t key = level_key(seed, level);
    // a graph the last level did not halve is weakly clustered: its lists carry many labels
    W.tune.mid_bail = n_prev_level > 0 && 2 * n_start > n_prev_level;
    n_prev_level = n_start;
    W.build_bins(G);
    int32_t* labels = nullptr;
    cudaEvent_t a0 = W.mark();
    if (lp_iters > 0) {
      W.lp_rounds(G, key, lp_iters, &labels, nullptr, H.lp_converge, H.lp_async);
    } else {
      labels = W.labA.as<int32_t>();
      iota(labels, G.n, s);
    }
    W.span(kPhLP, a0);
    ++levels;
    if (!step(labels, 1)) { done = true; break; }
    for (int run = 0; run < H.pr_runs_max && !done; ++run) {
      bool any = false;
      for (int pass = 0; pass < 2; ++pass) {
        cudaEvent_t ap = W.mark();
        VC_CUDA(cudaMemsetAsync(&W.ctr()->changed, 0, sizeof(int), s));
        if (!partners_ok) pr_partners(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), s);
        partners_ok = true;
        int32_t* lab = W.labA.as<int32_t>();
        if (pass == 0)
          pr_pass_a(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), st,
                    W.parent.as<int32_t>(), lab, &W.ctr()->changed, s);
        else
          pr_pass_b(G, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), st, lab,
                    &W.ctr()->changed, s);
        W.span(kPhPR, ap);
        if (read_changed()) {
          any = true;
          if (!step(lab, pass == 0 ? 2 : 3)) { done = true; break; }
        }
      }
      if (!any) break;
    }
    level += 1;
    if (done) break;
    if (G.n == n_start) break;
  }

  if (!done && G.n > 1) {
    cudaEvent_t a0 = W.mark();
    if (!contracted) {
      n1 = G.n;
      iota(W.map0.as<int32_t>(), G.n, s);
      iota(W.cur1.as<int32_t>(), G.n, s);
      contracted = true;
    }
    W.span(kPhOther, a0);
    while (!done && G.n > kDenseMax) {
      cudaEvent_t an = W.mark();
      W.noi_r.ensure_n<long long>(noi_round_scratch(G.n));
      W.noi_seen.ensure_n<int>(G.n);
      VC_CUDA(cudaMemsetAsync(&W.ctr()->changed, 0, sizeof(int), s));
      noi_round_sparse(G, st, W.noi_r.as<long long>(), W.noi_seen.as<int>(), W.parent.as<int32_t>(),
                       W.labA.as<int32_t>(), &W.ctr()->changed, s);
      W.span(kPhNOI, an);
      if (!read_changed()) { done = true; break; }
      if (!step(W.labA.as<int32_t>(), 4)) { done = true; break; }
    }
    if (!done && G.n > 1) {
      cudaEvent_t an = W.mark();
      W.ensure_noi();
      noi_dense(G, W.M0.as<long long>(), W.M1.as<long long>(), W.curK.as<int32_t>(), W.sideK.as<unsigned char>(),
                st, tr, tcap, level, s);
      W.span(kPhNOI, an);
    }
  }

  cudaEvent_t a1 = W.mark();
  // without any contraction the side is a single original vertex (best_kind 0)
  side_bits2(contracted ? W.map0.as<int32_t>() : nullptr, H.n, W.side1.as<unsigned char>(), W.cur1.as<int32_t>(),
             W.sideK.as<unsigned char>(), st, d_bits, s);
  VC_CUDA(cudaMemcpyAsync(d_cut, &st->lambda_hat, sizeof(long long), cudaMemcpyDeviceToDevice, s));
  W.span(kPhOther, a1);
  cudaEvent_t t_end = W.mark();

  // statistics
  viecut_stats& S = H.stats;
  memset(&S, 0, sizeof(S));
  S.levels = levels;
  if (W.timing) {
    VC_CUDA(cudaEventSynchronize(t_end));
    float ms;
    VC_CUDA(cudaEventElapsedTime(&ms, t_start, t_end));
    S.ms_total = ms;
    double ph[kPhCount] = {0, 0, 0, 0, 0};
    for (auto& sp : W.spans) {
      VC_CUDA(cudaEventElapsedTime(&ms, sp.second.first, sp.second.second));
      ph[sp.first] += ms;
    }
    S.ms_lp = ph[kPhLP];
    S.ms_contract = ph[kPhContract];
    S.ms_pr = ph[kPhPR];
    S.ms_noi = ph[kPhNOI];
    S.ms_other = ph[kPhOther];
    for (auto& sp : W.lp_spans) {
      VC_CUDA(cudaEventElapsedTime(&ms, sp.first, sp.second));
      S.ms_lp_kernel += ms;
    }
    S.lp_launches = (int64_t)W.lp_spans.size();
    S.lp_nnz = W.lp_nnz_acc;
    S.lp_n = W.lp_n_acc;
    S.lp_bytes = W.lp_bytes_acc;
    for (auto& sp : W.ct_spans) {
      VC_CUDA(cudaEventElapsedTime(&ms, sp.first, sp.second));
      S.ms_contract_kernel += ms;
    }
    for (auto& sp : W.pm_spans) {
      VC_CUDA(cudaEventElapsedTime(&ms, sp.first, sp.second));
      S.ms_premerge_kernel += ms;
    }
    S.contractions = W.ct_count;
    S.contract_bytes = W.ct_bytes_acc;
    S.premerge_bytes = W.pm_bytes_acc;
  }
  S.first_group = W.tune.first_group;
  S.emit_group = W.tune.emit_group;
  S.kernel_launches = (int64_t)(g_launches - launches0);
  (void)t_start;
}

static void fetch_trace(Handle& H) {
  Workspace& W = *H.ws;
  W.read_state();
  int len = W.h_state->trace_len;
  int cnt = std::min(len, W.trace_cap);
  std::vector<TraceStep> t(cnt);
  if (cnt) VC_CUDA(cudaMemcpy(t.data(), W.trace.p, sizeof(TraceStep) * cnt, cudaMemcpyDeviceToHost));
  H.last_trace.resize(cnt);
  for (int i = 0; i < cnt; ++i) {
    H.last_trace[i].kind = t[i].kind;
    H.last_trace[i].level = t[i].level;
    H.last_trace[i].n = t[i].n;
    H.last_trace[i].nnz = t[i].nnz;
    H.last_trace[i].lambda_hat = t[i].lambda_hat;
  }
  H.stats.trace_len = len;
}

// ---------------------------------------------------------------- step graphs
struct StepGraph {
  int device = 0;
  int64_t n = 0, nnz = 0;
  bool simple = false;
  bool unit = false;  // every weight is 1: the kernels that can then read no weights
  Buf off, adj, w;
  GraphView view() const {
    GraphView g;
    g.n = n;
    g.nnz = nnz;
    g.off = off.as<int64_t>();
    g.adj = adj.as<int32_t>();
    g.w = w.p;
    g.wbytes = 8;
    g.simple = simple;
    g.unit = unit;
    return g;
  }
};

}  // namespace vc

struct viecut_handle {
  vc::Handle h;
};
struct viecut_graph {
  vc::StepGraph g;
};

using vc::Error;

extern "C" {

const char* viecut_last_error(void) { return vc::t_last_error.c_str(); }

int viecut_struct_sizes(int64_t* sizes, int32_t count) {
  const int64_t known[] = {(int64_t)sizeof(viecut_opts),        (int64_t)sizeof(viecut_stats),
                           (int64_t)sizeof(viecut_step),        (int64_t)sizeof(viecut_graph_desc),
                           (int64_t)sizeof(viecut_batch_stats), (int64_t)sizeof(viecut_server_opts),
                           (int64_t)sizeof(viecut_server_stats), (int64_t)sizeof(viecut_request_info)};
  const int32_t nk = (int32_t)(sizeof(known) / sizeof(known[0]));
  if (count > 0 && !sizes) return VIECUT_EINVAL;
  for (int32_t i = 0; i < count && i < nk; ++i) sizes[i] = known[i];
  return nk;
}
int64_t viecut_launch_count(void) { return (int64_t)vc::g_launches; }

int viecut_debug_fail_device_allocs(int64_t after, int64_t count) {
  if (after < 0 || count < 0) return VIECUT_EINVAL;
  vc::g_fail_count.store(0);
  vc::g_fail_skip.store(after);
  vc::g_fail_count.store(count);
  return VIECUT_OK;
}

int viecut_opts_init(viecut_opts* o) {
  if (!o) return VIECUT_EINVAL;
  memset(o, 0, sizeof(*o));
  o->n0 = 10000;
  o->pr_runs_max = 8;
  o->device = 0;
  o->stream = nullptr;
  o->validate = 1;
  o->timing = 0;
  return VIECUT_OK;
}

static void check_shape(int64_t n, int64_t m, const int64_t* off, const int32_t* adj, const int32_t* w) {
  if (n < 2) throw Error{VIECUT_EINVAL, "n must be >= 2"};
  if (n > 0x7fffffffLL) throw Error{VIECUT_EINVAL, "n must fit int32 vertex ids"};
  if (m < 0) throw Error{VIECUT_EINVAL, "m must be >= 0"};
  if (!off || (m > 0 && (!adj || !w))) throw Error{VIECUT_EINVAL, "null graph array"};
}

// Points the handle at a graph: host arrays are copied into the handle's grow-only
// input buffers, device arrays are used in place; then validated per the handle's
// option (2: on the host before any copy; 1: one pass on the device).
// checked: the host check already ran (its findings in unit / simple).
static void bind_graph(vc::Handle& H, bool host_input, const int64_t* off, const int32_t* adj, const int32_t* w,
                       int64_t n, int64_t m, bool checked = false, bool unit = false, bool simple = false) {
  H.bound = false;
  if (host_input && H.validate >= 2 && !checked) unit = vc::host_validate(off, adj, w, n, m, true, &simple);
  VC_CUDA(cudaSetDevice(H.device));
  H.n = n;
  H.m = m;
  H.unit = unit;
  H.simple = simple;
  H.host_input = host_input;
  if (host_input) {
    H.off0 = H.in_off.ensure_n<int64_t>(n + 1);
    H.adj0 = H.in_adj.ensure_n<int32_t>(std::max<int64_t>(m, 1));
    H.w0 = H.in_w.ensure_n<int32_t>(std::max<int64_t>(m, 1));
    VC_CUDA(cudaMemcpyAsync((void*)H.off0, off, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, H.stream));
    if (m > 0) {
      VC_CUDA(cudaMemcpyAsync((void*)H.adj0, adj, sizeof(int32_t) * m, cudaMemcpyHostToDevice, H.stream));
      VC_CUDA(cudaMemcpyAsync((void*)H.w0, w, sizeof(int32_t) * m, cudaMemcpyHostToDevice, H.stream));
    }
  } else {
    H.off0 = off;
    H.adj0 = adj;
    H.w0 = w;
  }
  H.ws->ensure_vertices(n);
  H.ws->ensure_entries(m, n);
  H.out_cut.ensure_n<long long>(1);
  H.out_bits.ensure_n<unsigned long long>((n + 63) / 64);
  if (H.validate == 1 || (!host_input && H.validate >= 1)) vc::device_validate(H);
  VC_CUDA(cudaStreamSynchronize(H.stream));
  H.bound = true;
}

static int create_common(viecut_t** out, int64_t n, int64_t m, const viecut_opts* opts, bool host_input,
                         const int64_t* off, const int32_t* adj, const int32_t* w) {
  VC_API_BEGIN
  if (!out) throw Error{VIECUT_EINVAL, "null handle pointer"};
  *out = nullptr;
  check_shape(n, m, off, adj, w);
  viecut_opts o;
  viecut_opts_init(&o);
  if (opts) o = *opts;
  if (o.n0 < 1) throw Error{VIECUT_EINVAL, "n0 must be >= 1"};
  if (o.pr_runs_max < 0) throw Error{VIECUT_EINVAL, "pr_runs_max must be >= 0"};
  for (int G : {o.lp_group, o.emit_group})
    if (G != 0 && G != 8 && G != 16 && G != 32) throw Error{VIECUT_EINVAL, "lp_group and emit_group must be 0, 8, 16 or 32"};
  if (o.correct != 0 && o.correct != 1) throw Error{VIECUT_EINVAL, "correct must be 0 or 1"};
  if (o.lp_converge != 0 && o.lp_converge != 1) throw Error{VIECUT_EINVAL, "lp_converge must be 0 or 1"};
  if (o.lp_async < 0 || o.lp_async > 2) throw Error{VIECUT_EINVAL, "lp_async must be 0, 1 or 2"};
  // validate 2 rejects a malformed host graph before any device call
  const bool checked = host_input && o.validate >= 2;
  bool unit = false, simple = false;
  if (checked) unit = vc::host_validate(off, adj, w, n, m, true, &simple);
  auto* hh = new viecut_handle;
  vc::Handle& H = hh->h;
  try {
    H.device = o.device;
    VC_CUDA(cudaSetDevice(H.device));
    if (o.stream) {
      H.stream = (cudaStream_t)o.stream;
    } else {
      VC_CUDA(cudaStreamCreateWithFlags(&H.stream, cudaStreamNonBlocking));
      H.own_stream = true;
    }
    H.n0 = o.n0;
    H.pr_runs_max = o.pr_runs_max;
    H.validate = o.validate;
    H.correct = o.correct != 0;
    H.lp_converge = o.lp_converge != 0;
    H.lp_async = o.lp_async;
    H.ws = new vc::Workspace;
    H.ws->s = H.stream;
    H.ws->timing = o.timing != 0;
    H.ws->fix_groups(o.lp_group, o.emit_group);
    bind_graph(H, host_input, off, adj, w, n, m, checked, unit, simple);
  } catch (...) {
    delete hh;
    throw;
  }
  *out = hh;
  VC_API_END
}

int viecut_load(viecut_t* h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                const int32_t* weights) {
  VC_API_BEGIN
  if (!h) throw Error{VIECUT_EINVAL, "null handle"};
  if (!h->h.host_input) throw Error{VIECUT_EINVAL, "viecut_load needs a handle made by viecut_create"};
  check_shape(n, m, offsets, adj, weights);
  VC_CUDA(cudaSetDevice(h->h.device));
  VC_CUDA(cudaStreamSynchronize(h->h.stream));  // a previous run may still read the inputs
  bind_graph(h->h, true, offsets, adj, weights, n, m);
  VC_API_END
}

int viecut_create(viecut_t** h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                  const int32_t* weights, const viecut_opts* opts) {
  return create_common(h, n, m, opts, true, offsets, adj, weights);
}

int viecut_create_device(viecut_t** h, const int64_t* d_offsets, const int32_t* d_adj, int64_t n, int64_t m,
                         const int32_t* d_weights, const viecut_opts* opts) {
  return create_common(h, n, m, opts, false, d_offsets, d_adj, d_weights);
}

int viecut_run_device(viecut_t* h, uint64_t seed, int32_t lp_iters, int64_t* d_cut_value, uint64_t* d_side_bits) {
  VC_API_BEGIN
  if (!h || !d_cut_value) throw Error{VIECUT_EINVAL, "null argument"};
  VC_CUDA(cudaSetDevice(h->h.device));
  unsigned long long* bits = d_side_bits ? (unsigned long long*)d_side_bits : h->h.out_bits.as<unsigned long long>();
  vc::run_impl(h->h, seed, lp_iters, (long long*)d_cut_value, bits);
  VC_API_END
}

int viecut_run(viecut_t* h, uint64_t seed, int32_t lp_iters, int64_t* cut_value, uint64_t* side_bits) {
  VC_API_BEGIN
  if (!h || !cut_value) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Handle& H = h->h;
  VC_CUDA(cudaSetDevice(H.device));
  vc::run_impl(H, seed, lp_iters, H.out_cut.as<long long>(), H.out_bits.as<unsigned long long>());
  VC_CUDA(cudaMemcpyAsync(cut_value, H.out_cut.p, sizeof(int64_t), cudaMemcpyDeviceToHost, H.stream));
  if (side_bits)
    VC_CUDA(cudaMemcpyAsync(side_bits, H.out_bits.p, sizeof(uint64_t) * ((H.n + 63) / 64), cudaMemcpyDeviceToHost,
                            H.stream));
  VC_CUDA(cudaStreamSynchronize(H.stream));
  VC_API_END
}

// True when the first 256 weights and 4096 evenly spaced ones are all 1.
static bool sampled_unit(const int32_t* w, int64_t m) {
  for (int64_t e = 0; e < m && e < 256; ++e)
    if (w[e] != 1) return false;
  const int64_t stride = m / 4096 > 0 ? m / 4096 : 1;
  for (int64_t e = 0; e < m; e += stride)
    if (w[e] != 1) return false;
  return true;
}

int viecut_solve(viecut_t* h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                 const int32_t* weights, uint64_t seed, int32_t lp_iters, int64_t* cut_value, uint64_t* side_bits) {
  VC_API_BEGIN
  if (!h || !cut_value) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Handle& H = h->h;
  if (!H.host_input) throw Error{VIECUT_EINVAL, "viecut_solve needs a handle made by viecut_create"};
  if (lp_iters < 0) throw Error{VIECUT_EINVAL, "lp_iters must be >= 0"};
  check_shape(n, m, offsets, adj, weights);
  VC_CUDA(cudaSetDevice(H.device));
  VC_CUDA(cudaStreamSynchronize(H.stream));
  long long* d_cut = H.out_cut.ensure_n<long long>(1);
  if (H.validate != 1 || m == 0 || !sampled_unit(weights, m)) {
    bind_graph(H, true, offsets, adj, weights, n, m);
    vc::run_impl(H, seed, lp_iters, d_cut, H.out_bits.ensure_n<unsigned long long>((n + 63) / 64));
  } else {
    // the weights look like all 1: run with unit weights while they are copied and
    // checked on a second stream; run again with weights if the check disagrees
    H.bound = false;
    H.n = n;
    H.m = m;
    H.host_input = true;
    H.off0 = H.in_off.ensure_n<int64_t>(n + 1);
    H.adj0 = H.in_adj.ensure_n<int32_t>(m);
    H.w0 = H.in_w.ensure_n<int32_t>(m);
    if (!H.cstream) VC_CUDA(cudaStreamCreateWithFlags(&H.cstream, cudaStreamNonBlocking));
    if (!H.wdone) VC_CUDA(cudaEventCreateWithFlags(&H.wdone, cudaEventDisableTiming));
    int* werr = H.werr.ensure_n<int>(1);
    VC_CUDA(cudaMemcpyAsync((void*)H.off0, offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, H.stream));
    VC_CUDA(cudaMemcpyAsync((void*)H.adj0, adj, sizeof(int32_t) * m, cudaMemcpyHostToDevice, H.stream));
    VC_CUDA(cudaMemsetAsync(werr, 0, sizeof(int), H.cstream));
    VC_CUDA(cudaMemcpyAsync((void*)H.w0, weights, sizeof(int32_t) * m, cudaMemcpyHostToDevice, H.cstream));
    vc::weight_check_k<<<vc::grid_for(m, 256, vc::kSMs * 8), 256, 0, H.cstream>>>(m, H.w0, werr);
    vc::count_launch();
    VC_CHECK_LAUNCH();
    VC_CUDA(cudaEventRecord(H.wdone, H.cstream));
    int h_werr = 0;
    try {
      H.ws->ensure_vertices(n);
      H.ws->ensure_entries(m, n);
      H.out_bits.ensure_n<unsigned long long>((n + 63) / 64);
      vc::device_validate(H, false);
      H.unit = true;
      H.bound = true;
      vc::run_impl(H, seed, lp_iters, d_cut, H.out_bits.as<unsigned long long>());
      VC_CUDA(cudaMemcpyAsync(&h_werr, werr, sizeof(int), cudaMemcpyDeviceToHost, H.cstream));
      VC_CUDA(cudaStreamSynchronize(H.cstream));
    } catch (...) {
      cudaStreamSynchronize(H.cstream);  // the copy reads the caller's array
      H.bound = false;
      throw;
    }
    if (h_werr & 16) {
      H.bound = false;
      throw Error{VIECUT_EINVAL, "invalid graph: weight < 1;"};
    }
    if (h_werr & 32) {
      H.unit = false;
      vc::run_impl(H, seed, lp_iters, d_cut, H.out_bits.as<unsigned long long>());
    }
  }
  VC_CUDA(cudaMemcpyAsync(cut_value, d_cut, sizeof(int64_t), cudaMemcpyDeviceToHost, H.stream));
  if (side_bits)
    VC_CUDA(cudaMemcpyAsync(side_bits, H.out_bits.p, sizeof(uint64_t) * ((n + 63) / 64), cudaMemcpyDeviceToHost,
                            H.stream));
  VC_CUDA(cudaStreamSynchronize(H.stream));
  VC_API_END
}

int viecut_get_stats(const viecut_t* h, viecut_stats* stats) {
  VC_API_BEGIN
  if (!h || !stats) throw Error{VIECUT_EINVAL, "null argument"};
  *stats = h->h.stats;
  VC_API_END
}

int viecut_get_trace(const viecut_t* h, viecut_step* steps, int64_t cap, int64_t* len) {
  VC_API_BEGIN
  if (!h || !len) throw Error{VIECUT_EINVAL, "null argument"};
  vc::Handle& H = const_cast<viecut_t*>(h)->h;
  VC_CUDA(cudaSetDevice(H.device));
  vc::fetch_trace(H);
  *len = (int64_t)H.last_trace.size();
  for (int64_t i = 0; i < cap && i < *len; ++i) steps[i] = H.last_trace[i];
  VC_API_END
}

int viecut_destroy(viecut_t* h) {
  VC_API_BEGIN
  if (!h) return VIECUT_OK;
  cudaSetDevice(h->h.device);
  if (h->h.stream) cudaStreamSynchronize(h->h.stream);
  delete h;
  VC_API_END
}

// ------------------------------------------------------------------ step API
int viecut_graph_upload(viecut_graph** g, const int64_t* offsets, const int32_t* adj, const int64_t* weights,
                        int64_t n, int64_t nnz, int32_t device) {
  VC_API_BEGIN
  if (!g || !offsets || n < 1 || nnz < 0) throw Error{VIECUT_EINVAL, "bad graph arguments"};
  VC_CUDA(cudaSetDevice(device));
  auto* x = new viecut_graph;
  try {
    x->g.device = device;
    x->g.n = n;
    x->g.nnz = nnz;
    x->g.simple = true;
    for (int64_t v = 0; v < n && x->g.simple; ++v)
      for (int64_t e = offsets[v]; e + 1 < offsets[v + 1]; ++e)
        if (adj[e + 1] <= adj[e]) { x->g.simple = false; break; }
    x->g.unit = true;
    for (int64_t e = 0; e < nnz && x->g.unit; ++e) x->g.unit = weights[e] == 1;
    VC_CUDA(cudaMemcpy(x->g.off.ensure_n<int64_t>(n + 1), offsets, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
    x->g.adj.ensure_n<int32_t>(nnz);
    x->g.w.ensure_n<long long>(nnz);
    if (nnz > 0) {
      VC_CUDA(cudaMemcpy(x->g.adj.p, adj, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
      VC_CUDA(cudaMemcpy(x->g.w.p, weights, sizeof(int64_t) * nnz, cudaMemcpyHostToDevice));
    }
  } catch (...) {
    delete x;
    throw;
  }
  *g = x;
  VC_API_END
}

int viecut_graph_shape(const viecut_graph* g, int64_t* n, int64_t* nnz) {
  VC_API_BEGIN
  if (!g) throw Error{VIECUT_EINVAL, "null graph"};
  if (n) *n = g->g.n;
  if (nnz) *nnz = g->g.nnz;
  VC_API_END
}

int viecut_graph_download(const viecut_graph* g, int64_t* offsets, int32_t* adj, int64_t* weights) {
  VC_API_BEGIN
  if (!g) throw Error{VIECUT_EINVAL, "null graph"};
  VC_CUDA(cudaSetDevice(g->g.device));
  VC_CUDA(cudaMemcpy(offsets, g->g.off.p, sizeof(int64_t) * (g->g.n + 1), cudaMemcpyDeviceToHost));
  if (g->g.nnz > 0) {
    VC_CUDA(cudaMemcpy(adj, g->g.adj.p, sizeof(int32_t) * g->g.nnz, cudaMemcpyDeviceToHost));
    VC_CUDA(cudaMemcpy(weights, g->g.w.p, sizeof(int64_t) * g->g.nnz, cudaMemcpyDeviceToHost));
  }
  VC_API_END
}

int viecut_graph_free(viecut_graph* g) {
  VC_API_BEGIN
  if (g) {
    cudaSetDevice(g->g.device);
    delete g;
  }
  VC_API_END
}

namespace {
struct StepCtx {
  cudaStream_t s = nullptr;
  vc::Workspace* ws = nullptr;
  explicit StepCtx(const vc::StepGraph& g) {
    VC_CUDA(cudaSetDevice(g.device));
    VC_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ws = new vc::Workspace;
    ws->s = s;
    ws->ensure_vertices(g.n);
    ws->ensure_entries(g.nnz, g.n);
    VC_CUDA(cudaMemsetAsync(ws->state.p, 0, sizeof(vc::DevState), s));
    VC_CUDA(cudaMemsetAsync(ws->counters.p, 0, sizeof(vc::Counters), s));
  }
  ~StepCtx() {
    if (s) cudaStreamSynchronize(s);
    delete ws;
    if (s) cudaStreamDestroy(s);
  }
  void set_lambda(int64_t lam) {
    vc::DevState st{};
    st.lambda_hat = lam;
    VC_CUDA(cudaMemcpyAsync(ws->state.p, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  }
};
}  // namespace

int viecut_step_degrees(viecut_graph* g, int64_t* deg) {
  VC_API_BEGIN
  if (!g || !deg) throw Error{VIECUT_EINVAL, "null argument"};
  StepCtx c(g->g);
  vc::degrees(g->g.view(), c.ws->deg.as<long long>(), c.s);
  VC_CUDA(cudaMemcpyAsync(deg, c.ws->deg.p, sizeof(int64_t) * g->g.n, cudaMemcpyDeviceToHost, c.s));
  VC_CUDA(cudaStreamSynchronize(c.s));
  VC_API_END
}

// Labels are vertex ids of the graph: [0, n).
static void check_labels(const int32_t* lab, int64_t n) {
  for (int64_t v = 0; v < n; ++v)
    if (lab[v] < 0 || lab[v] >= n)
      throw Error{VIECUT_EINVAL, "label " + std::to_string(lab[v]) + " of vertex " + std::to_string(v) +
                                     " is outside [0, n)"};
}

int viecut_step_lp(viecut_graph* g, const int32_t* lab_in, uint64_t key, int32_t rounds, int32_t* lab_out) {
  VC_API_BEGIN
  if (!g || !lab_out || rounds < 1) throw Error{VIECUT_EINVAL, "bad argument"};
  if (lab_in) check_labels(lab_in, g->g.n);
  StepCtx c(g->g);
  vc::GraphView v = g->g.view();
  c.ws->build_bins(v);
  c.ws->tune.mid_bail = true;  // a launch choice only: the table kernel runs here for every
                                // mid-class list with many labels, so the tests see it
  int32_t* in = nullptr;
  if (lab_in) {
    vc::Buf tmp;
    in = tmp.ensure_n<int32_t>(v.n);
    VC_CUDA(cudaMemcpyAsync(in, lab_in, sizeof(int32_t) * v.n, cudaMemcpyHostToDevice, c.s));
    int32_t* bufs[2] = {c.ws->labA.as<int32_t>(), c.ws->labB.as<int32_t>()};
    vc::hash_table(v.n, key, nullptr, nullptr, nullptr, c.ws->hv.as<unsigned long long>(), c.s);
    for (int r = 0; r < rounds; ++r) {
      vc::lp_round(v, c.ws->bins, c.ws->gt, in, bufs[r & 1], c.ws->hv.as<unsigned long long>(), c.s, c.ws->tune);
      VC_CUDA(cudaMemcpyAsync(lab_out + (int64_t)r * v.n, bufs[r & 1], sizeof(int32_t) * v.n, cudaMemcpyDeviceToHost, c.s));
      in = bufs[r & 1];
    }
    VC_CUDA(cudaStreamSynchronize(c.s));
  } else {
    int32_t* last;
    c.ws->lp_rounds(v, key, rounds, &last, lab_out);
    VC_CUDA(cudaStreamSynchronize(c.s));
  }
  VC_API_END
}

int viecut_step_contract(viecut_graph* g, const int32_t* labels, viecut_graph** out, int32_t* cid) {
  VC_API_BEGIN
  if (!g || !labels || !out) throw Error{VIECUT_EINVAL, "null argument"};
  *out = nullptr;
  check_labels(labels, g->g.n);
  StepCtx c(g->g);
  vc::GraphView v = g->g.view();
  int32_t* lab = c.ws->labA.as<int32_t>();
  VC_CUDA(cudaMemcpyAsync(lab, labels, sizeof(int32_t) * v.n, cudaMemcpyHostToDevice, c.s));
  int32_t* cidd = c.ws->map0.as<int32_t>();
  vc::GraphView h = c.ws->contract(v, lab, cidd, 0, false, true);  // sparse path when it applies
  c.ws->read_state();
  const int64_t nnz = c.ws->h_state->nnz;
  auto* x = new viecut_graph;
  try {
    x->g.device = g->g.device;
    x->g.n = h.n;
    x->g.nnz = nnz;
    x->g.simple = true;
    VC_CUDA(cudaMemcpyAsync(x->g.off.ensure_n<int64_t>(h.n + 1), h.off, sizeof(int64_t) * (h.n + 1),
                            cudaMemcpyDeviceToDevice, c.s));
    VC_CUDA(cudaMemcpyAsync(x->g.adj.ensure_n<int32_t>(nnz), h.adj, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, c.s));
    VC_CUDA(cudaMemcpyAsync(x->g.w.ensure_n<long long>(nnz), h.w, sizeof(int64_t) * nnz, cudaMemcpyDeviceToDevice, c.s));
    if (cid) VC_CUDA(cudaMemcpyAsync(cid, cidd, sizeof(int32_t) * v.n, cudaMemcpyDeviceToHost, c.s));
    VC_CUDA(cudaStreamSynchronize(c.s));
  } catch (...) {
    delete x;
    throw;
  }
  *out = x;
  VC_API_END
}

static int step_labels(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed, int which) {
  VC_API_BEGIN
  if (!g || !labels) throw Error{VIECUT_EINVAL, "null argument"};
  StepCtx c(g->g);
  vc::GraphView v = g->g.view();
  vc::Workspace& W = *c.ws;
  c.set_lambda(lambda_hat);
  int* chg = &W.ctr()->changed;
  VC_CUDA(cudaMemsetAsync(chg, 0, sizeof(int), c.s));
  int32_t* lab = W.labA.as<int32_t>();
  if (which == 0 || which == 1) {
    vc::pr_partners(v, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), c.s);
    if (which == 0)
      vc::pr_pass_a(v, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(),
                    W.parent.as<int32_t>(), lab, chg, c.s);
    else
      vc::pr_pass_b(v, W.partner.as<int32_t>(), W.pw.as<long long>(), W.deg.as<long long>(), W.st(), lab, chg, c.s);
  } else {
    W.noi_r.ensure_n<long long>(vc::noi_round_scratch(v.n));
    W.noi_seen.ensure_n<int>(v.n);
    vc::noi_round_sparse(v, W.st(), W.noi_r.as<long long>(), W.noi_seen.as<int>(), W.parent.as<int32_t>(),
                         lab, chg, c.s);
  }
  W.read_state();
  VC_CUDA(cudaMemcpy(labels, lab, sizeof(int32_t) * v.n, cudaMemcpyDeviceToHost));
  if (changed) *changed = W.h_counters->changed;
  VC_API_END
}

int viecut_step_pr_a(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed) {
  return step_labels(g, lambda_hat, labels, changed, 0);
}
int viecut_step_pr_b(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed) {
  return step_labels(g, lambda_hat, labels, changed, 1);
}
int viecut_step_noi_round(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed) {
  return step_labels(g, lambda_hat, labels, changed, 2);
}

}  // extern "C"
