/*
 * viecut.h -- C ABI of the GB300 (sm_103a) implementation of VieCut, the inexact
 * near-linear minimum-cut method of "Practical Minimum Cut Algorithms" (Henzinger,
 * Noe, Schulz, Strash; arXiv 1708.06127).
 *
 * The method (Algorithm 1 of the paper, Appendix A): while the graph has more than n0
 * vertices, cluster it by label propagation (Sec. 4.1), contract the clusters
 * (Sec. 4.1, "contract it"), contract the edges that the Padberg-Rinaldi conditions
 * mark (Lemma "Padberg-Rinaldi", Sec. 4.1); then solve the remaining graph exactly
 * with the algorithm of Nagamochi, Ono and Ibaraki (Sec. 3).  Throughout, the bound
 * lambda-hat is the smallest trivial cut (minimum weighted degree) seen after any
 * contraction (Sec. 4, second paragraph).  The result is that bound and the side of
 * the cut that realises it, transferred back to the input vertices.
 *
 * Deterministic variant: label propagation is synchronous with ties broken by
 * mix64(key XOR label), key = mix64(seed + 0x9e3779b97f4a7c15 * (level + 1)),
 * mix64 = SplitMix64's output function; condition 2 of Padberg-Rinaldi marks only the
 * edge to each vertex's designated partner; conditions 3 and 4 run on mutual partner
 * pairs.  For a fixed (graph, seed, lp_iters, n0, pr_runs_max) every call returns
 * the same cut value and the same side, bit for bit.
 *
 * Conventions shared by all calls:
 *   - Graphs are undirected CSR: offsets int64[n+1] (offsets[0] = 0, non-decreasing,
 *     offsets[n] = m), adj int32[m] neighbour ids, weights int32[m] >= 1; every edge
 *     appears in both directions with equal weight; m counts directed entries (twice
 *     the paper's |E|).  Parallel entries are allowed and summed; self-loops are not.
 *   - Every call returns 0 on success or a negative VIECUT_E* code; the message of the
 *     last failure on the calling thread is available from viecut_last_error().
 *   - "Host" pointers are ordinary CPU memory (pinned memory makes copies faster);
 *     "device" pointers are CUDA global memory on the handle's device.
 *   - The library allocates its own device work space (cudaMalloc) at create time and
 *     grows it on first use; nothing is allocated by the caller except inputs/outputs.
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef VIECUT_H_
#define VIECUT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VIECUT_OK 0
#define VIECUT_EINVAL (-1)    /* invalid argument or malformed graph */
#define VIECUT_ENOMEM (-2)    /* device or host allocation failed */
#define VIECUT_ECUDA (-3)     /* CUDA runtime error (message names the call) */
#define VIECUT_ETIMEOUT (-4)  /* a bounded wait ran out (viecut_server_wait) */
#define VIECUT_ECANCELLED (-5) /* the request was cancelled (viecut_server_cancel) */
#define VIECUT_EBUSY (-6)     /* result not ready yet (server poll) */

typedef struct viecut_handle viecut_t;

/* Options fixed at create time.  viecut_opts_init fills the defaults. */
typedef struct viecut_opts {
  int64_t n0;          /* exact step once at most n0 vertices remain (default 10000, Sec. 5 setup) */
  int32_t pr_runs_max; /* Padberg-Rinaldi runs per level (default 8) */
  int32_t device;      /* CUDA device ordinal (default 0) */
  void* stream;        /* cudaStream_t for all work; NULL = the library creates one */
  int32_t validate;    /* 0 = trust input; 1 = range/loop/weight/offset checks, one pass on
                          the device (default); 2 = the same checks plus symmetry, on the
                          host (create from host arrays; O(m log m)) */
  int32_t timing;      /* 1 = record per-phase CUDA-event times (viecut_get_stats) */
  int32_t lp_group;    /* lanes per vertex of the first-round label-propagation kernel:
                          8, 16 or 32, or 0 = pick by timing once per handle (default);
                          results never depend on it */
  int32_t emit_group;  /* lanes per vertex of the contraction's pre-merge kernel (same) */
  int32_t correct;     /* 1 = the correcting step on every label-propagation clustering
                          (Sec. 4.1, "correcting algorithm"): in each cluster of 2 to
                          floor(log2 n) vertices, the vertex whose removal lowers the
                          cluster's weighted degree the most becomes a singleton; 0 = off
                          (default).  Single-graph handles only: viecut_batch_create and
                          viecut_server_start refuse it with VIECUT_EINVAL */
  int32_t lp_converge; /* 1 = lp_iters is an upper bound: a level's rounds end after the first
                          round in which at most 1/10000 of its vertices changed their label
                          (the VieCut25 configuration, App. D, with lp_iters = 25); 0 = exactly
                          lp_iters rounds (default).  Single-graph handles only (EINVAL for
                          batches and servers) */
  int32_t lp_async;    /* 0 = synchronous rounds (default); 1 = asynchronous rounds (Sec. 4.1
                          in-place updates, Sec. 4.3 shuffled blocks): the vertices form
                          blocks of 128 consecutive ids, ordered by mix64(key ^ mix64(round + 1)
                          ^ block) and cut into 8 waves that run one after another, each wave
                          choosing from the labels as they stand when it starts; 2 = the same
                          with the first round's restriction (Sec. 4.1: a vertex keeps its
                          label once a vertex of an earlier wave moved to its block).
                          Deterministic.  Single-graph handles only */
} viecut_opts;

/* Per-run statistics (valid after viecut_run / viecut_run_device completes). */
typedef struct viecut_stats {
  double ms_total;       /* device time of the whole run (timing = 1) */
  double ms_lp;          /* label-propagation rounds */
  double ms_contract;    /* cluster and edge contractions */
  double ms_pr;          /* Padberg-Rinaldi tests */
  double ms_noi;         /* exact final step */
  double ms_other;       /* bounds, side transfer */
  double ms_lp_kernel;   /* summed duration of the label-propagation launches */
  int64_t lp_launches;   /* label-propagation rounds timed in ms_lp_kernel */
  int64_t lp_nnz;        /* adjacency entries read by the timed label-propagation rounds */
  int64_t lp_n;          /* vertices processed by the timed label-propagation rounds */
  int64_t kernel_launches; /* kernels launched by this run */
  int64_t levels;        /* label-propagation levels run */
  int64_t trace_len;     /* contraction steps recorded (viecut_get_trace) */
  int64_t lp_bytes;      /* algorithmic bytes of the timed label-propagation rounds:
                            8(n+1) offsets + nnz (4 id + weight bytes + 4 label gather,
                            no gather in a level's first round) + 4n label writes */
  int32_t first_group;   /* lanes per vertex of the first-round label-propagation kernel
                            (8, 16 or 32; picked once per handle by timing each choice) */
  int32_t emit_group;    /* lanes per vertex of the contraction's pre-merge kernel (same) */
  double ms_contract_kernel; /* summed device time of the timed contractions (relabel,
                                pre-merge, cluster merge; the host's read of the cluster
                                and pair counts between them is not included) */
  double ms_premerge_kernel; /* summed duration of the pre-merge launches alone */
  int64_t contractions;      /* contractions timed in ms_contract_kernel */
  int64_t contract_bytes;    /* their algorithmic bytes: fine CSR read once (offsets, ids,
                                weights unless all are 1) + 4 per entry (cluster id of the
                                neighbour) + 8 per fine vertex (label read, cluster id
                                written) + coarse CSR written (offsets, int32 id + int64
                                weight per entry) */
  int64_t premerge_bytes;    /* the pre-merge's algorithmic bytes: 8(n+1) offsets + nnz (4 id
                                + weight bytes + 4 cluster id) + 8n (own cluster id, pair
                                count) + 12 per pre-merged pair written */
} viecut_stats;

/* One contraction step: kind 0 initial graph, 1 label-propagation contraction,
 * 2 Padberg-Rinaldi pass A, 3 pass B, 4 exact-step round; shape and bound after it. */
typedef struct viecut_step {
  int32_t kind, level;
  int64_t n, nnz, lambda_hat;
} viecut_step;

int viecut_opts_init(viecut_opts* opts);

/* Creates a handle from HOST arrays (copied to the device; the caller keeps them).
 * opts may be NULL (defaults).  EINVAL for n < 2, m < 0 or a malformed graph. */
int viecut_create(viecut_t** h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                  const int32_t* weights, const viecut_opts* opts);

/* Creates a handle over DEVICE arrays that stay owned by the caller and must
 * outlive the handle (no copy).  validate 2 is treated as 1. */
int viecut_create_device(viecut_t** h, const int64_t* d_offsets, const int32_t* d_adj, int64_t n, int64_t m,
                         const int32_t* d_weights, const viecut_opts* opts);

/* Replaces the graph of a handle made by viecut_create with another one from host
 * arrays (same layout and ownership rules as viecut_create), keeping the handle's
 * options, stream, chosen launch shapes and device buffers; buffers grow when the new
 * graph is larger and are never shrunk, so a loop over many graphs allocates only
 * while sizes grow.  Waits for the handle's previous work first.  EINVAL for a handle
 * made by viecut_create_device or a malformed graph (checked as viecut_create). */
int viecut_load(viecut_t* h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                const int32_t* weights);

/* viecut_load + viecut_run in one call, for a handle made by viecut_create: the host
 * arrays are read only during the call.  With validate = 1 and weights that look
 * like all 1 (the first 256 and 4096 evenly spaced ones are), the method runs with
 * unit weights while the weights are copied and checked on a second stream, and runs
 * again with the weights if the check finds one that is not 1; results are those of
 * viecut_load + viecut_run either way.  EINVAL as viecut_load (the handle then holds
 * no graph). */
int viecut_solve(viecut_t* h, const int64_t* offsets, const int32_t* adj, int64_t n, int64_t m,
                 const int32_t* weights, uint64_t seed, int32_t lp_iters, int64_t* cut_value, uint64_t* side_bits);

/* Runs the method and waits for it.  cut_value (host) receives the cut; side_bits
 * (host, ceil(n/64) words, may be NULL) receives bit i = 1 iff input vertex i is on
 * the returned side; vertex 0 is never on it.  lp_iters >= 0 (the paper uses 2). */
int viecut_run(viecut_t* h, uint64_t seed, int32_t lp_iters, int64_t* cut_value, uint64_t* side_bits);

/* As viecut_run, but the outputs are DEVICE pointers (d_side_bits may be NULL)
 * written on the handle's stream.  The level loop reads small shape records from the
 * device at its decision points, so the call returns when the last kernels are
 * enqueued; synchronise the stream before reading the outputs. */
int viecut_run_device(viecut_t* h, uint64_t seed, int32_t lp_iters, int64_t* d_cut_value,
                      uint64_t* d_side_bits);

int viecut_get_stats(const viecut_t* h, viecut_stats* stats);
/* Copies up to cap steps of the last run's contraction trace; *len = steps made. */
int viecut_get_trace(const viecut_t* h, viecut_step* steps, int64_t cap, int64_t* len);
int viecut_destroy(viecut_t* h);
const char* viecut_last_error(void);
/* Kernels launched by this library in this process so far. */
int64_t viecut_launch_count(void);

/* ---------------------------------------------------------------------------
 * Step entry points.  They run one step of the method on a device-resident graph,
 * with host inputs/outputs, so every step can be compared with a reference alone.
 * A viecut_graph owns its device CSR (int64 weights).
 * ------------------------------------------------------------------------- */
typedef struct viecut_graph viecut_graph;

/* Copies a host CSR (int64 weights) to the device.  A graph whose weights are all 1
 * is marked so, and the steps then run the kernels that read no weights, as they do on
 * an input graph of unit weights. */
int viecut_graph_upload(viecut_graph** g, const int64_t* offsets, const int32_t* adj, const int64_t* weights,
                        int64_t n, int64_t nnz, int32_t device);
int viecut_graph_shape(const viecut_graph* g, int64_t* n, int64_t* nnz);
/* Copies the CSR back (offsets n+1, adj nnz, weights nnz). */
int viecut_graph_download(const viecut_graph* g, int64_t* offsets, int32_t* adj, int64_t* weights);
int viecut_graph_free(viecut_graph* g);

/* Weighted degrees c(v) (Sec. 3): deg[n]. */
int viecut_step_degrees(viecut_graph* g, int64_t* deg);
/* `rounds` synchronous label-propagation rounds (Sec. 4.1) from lab_in (NULL = the
 * identity labelling; otherwise labels in [0, n), else EINVAL) with tie-break key `key`;
 * writes every round: lab_out[rounds*n]. */
int viecut_step_lp(viecut_graph* g, const int32_t* lab_in, uint64_t key, int32_t rounds, int32_t* lab_out);
/* Contraction by labels in [0, n) (Sec. 4.1, "contract it"; other labels: EINVAL): *out
 * receives the coarse graph, cid[n] the coarse id (rank of the label value) of every
 * vertex. */
int viecut_step_contract(viecut_graph* g, const int32_t* labels, viecut_graph** out, int32_t* cid);
/* Padberg-Rinaldi pass A (conditions 1, 2) / pass B (conditions 3, 4) with bound
 * lambda_hat: labels[n] = union-find representative (smallest id of each merged
 * group); *changed = 1 if anything merged.  The graph must have merged, sorted lists. */
int viecut_step_pr_a(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed);
int viecut_step_pr_b(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed);
/* One Nagamochi-Ono-Ibaraki round (Sec. 3) with bound lambda_hat: labels[n] as above. */
int viecut_step_noi_round(viecut_graph* g, int64_t lambda_hat, int32_t* labels, int32_t* changed);

/* One Nagamochi-Ono-Ibaraki round, like viecut_step_noi_round, that allocates no
 * memory at all.  The paper has no counterpart: this entry point exists for callers
 * that cannot call cudaMalloc -- code whose device memory is owned by another
 * allocator (a host framework that reserved the GPU for its own pool), or a serving
 * loop that must not hit cudaMalloc's implicit device synchronisation.  The caller
 * passes the graph (DEVICE CSR of n vertices with merged, sorted lists and int64
 * weights, as every contracted graph is), the bound, and the DEVICE outputs
 * d_labels[n] (union-find representative, smallest id of each merged group) and
 * *d_changed (1 if anything merged).  No pointer may be NULL, not even d_adj and
 * d_weights of a graph without edges (the host cannot read offsets[n]): EINVAL, and
 * nothing is launched.  Work space is a static device array sized
 * for n <= 65536 (about 0.8 MB, kept by every GPU that loads the library until the
 * process exits); larger n is rejected with VIECUT_EINVAL and nothing is launched.
 * The round runs on `stream` (NULL: the default stream) and the call returns without
 * waiting.  The first call on a device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current; make that first call before any
 * stream capture.  All calls share the one array (the kernel clears what it needs):
 * calls whose executions overlap on the GPU race and their results are undefined. */
int viecut_noi_round_noalloc(const int64_t* d_offsets, const int32_t* d_adj, const int64_t* d_weights, int64_t n,
                             int64_t lambda_hat, int32_t* d_labels, int32_t* d_changed, void* stream);

/* ---------------------------------------------------------------------------
 * Batches: many independent graphs solved together (same seed and options for all).
 * The graphs are laid out as one disjoint union on the device; each graph follows its
 * own sequence of steps (levels, Padberg-Rinaldi runs, exact step) and the union is
 * contracted once per super-step for all of them, so every graph's result is bit for
 * bit the result viecut_run gives for it alone.
 * ------------------------------------------------------------------------- */
typedef struct viecut_graph_desc {
  const int64_t* offsets; /* host, n+1 */
  const int32_t* adj;     /* host, m */
  const int32_t* weights; /* host, m, >= 1 */
  int64_t n, m;           /* vertices (>= 2), directed entries */
} viecut_graph_desc;

typedef struct viecut_batch_stats {
  double ms_total;         /* device time of the last viecut_batch_run */
  int64_t super_steps;     /* lock-step rounds the batch needed */
  int64_t kernel_launches; /* kernels launched by the last run */
  int64_t graphs, vertices, entries;
} viecut_batch_stats;

typedef struct viecut_batch viecut_batch;

/* Copies k host graphs to the device as one union (the caller keeps its arrays).
 * opts as for viecut_create (validate 2 acts as 1).  EINVAL names the bad graph. */
int viecut_batch_create(viecut_batch** b, const viecut_graph_desc* graphs, int32_t k, const viecut_opts* opts);
/* Solves all graphs: cut_values[k] (host); side_bits (host, may be NULL) receives the
 * graphs' bitmaps back to back, graph g's ceil(n_g/64) words after those of graphs
 * 0..g-1 (viecut_batch_side_words gives the total). */
int viecut_batch_run(viecut_batch* b, uint64_t seed, int32_t lp_iters, int64_t* cut_values, uint64_t* side_bits);
int viecut_batch_side_words(const viecut_batch* b, int64_t* words);
/* Contraction trace of graph g in the last run (as viecut_get_trace). */
int viecut_batch_get_trace(const viecut_batch* b, int32_t g, viecut_step* steps, int64_t cap, int64_t* len);
int viecut_batch_get_stats(const viecut_batch* b, viecut_batch_stats* stats);
int viecut_batch_destroy(viecut_batch* b);

/* ---------------------------------------------------------------------------
 * Serving: a request loop that keeps solving while requests arrive.  A host thread
 * admits submitted graphs whenever a slot is free and the memory budget allows,
 * appends them to the graphs resident on the device at the next super-step (their
 * contraction state stays on the device until they finish), advances all resident
 * graphs together, and hands each result back as soon as its graph finishes
 * (continuous batching).  Each result equals viecut_run's result for that graph with
 * the same seed, options and lp_iters.
 * ------------------------------------------------------------------------- */
typedef struct viecut_server_opts {
  viecut_opts base;         /* n0, pr_runs_max, device, stream (validate is not used) */
  int64_t hbm_budget_bytes; /* admission budget for resident graphs (default 120 GiB) */
  int32_t max_slots;        /* graphs resident at once (default 1024) */
  int32_t lp_iters;         /* label-propagation rounds per level for every request (default 2) */
  int64_t solo_min_n;       /* requests of at least this many vertices skip the union and run
                               on the solo lanes, beside the union (each has parallelism enough
                               alone); 0 = no solo lanes (default 65536) */
  int32_t solo_lanes;       /* solo lanes: threads, each running one request at a time on a handle
                               and stream of its own (1..64, default 8) */
  int32_t solo_exact;       /* 1 = requests of 513..n0 vertices (their whole run is the exact
                               step, a sequential scan per round) also go to the solo lanes, so that
                               the union's lock-step super-steps never wait for such a scan
                               (default); 0 = they join the union */
} viecut_server_opts;

typedef struct viecut_server_stats {
  int64_t admitted, completed, pending, max_resident, super_steps, joins, budget_used;
  int64_t solo_completed;   /* requests served on the solo lane */
  int64_t rejected;         /* requests refused by the device check (counted in completed) */
  int64_t cancelled;        /* requests cancelled by viecut_server_cancel */
  int64_t failed;           /* requests answered with VIECUT_ENOMEM (counted in completed) */
} viecut_server_stats;

/* Where a served request's time went (viecut_server_poll_info / viecut_server_wait). */
typedef struct viecut_request_info {
  double latency_ms;  /* submit -> result on the host */
  double queue_ms;    /* submit -> the request started on the device (admitted to the union or taken
                         by the solo lane) */
  double run_ms;      /* started -> result on the host */
  int32_t lane;       /* 0: batched in the resident union; 1: the solo lane */
  int32_t pad;
  int64_t n, m;       /* the request's graph */
} viecut_request_info;

typedef struct viecut_server viecut_server;

int viecut_server_opts_init(viecut_server_opts* o);
/* Starts the server thread (allocations happen here and as the resident set grows). */
int viecut_server_start(viecut_server** s, const viecut_server_opts* o);
/* Queues a graph (host arrays, copied into page-locked memory before the call
 * returns) with its seed; *ticket identifies the request.  EINVAL at once if n < 2, an
 * array is NULL, offsets[0] != 0, offsets[n] != m, or the graph alone exceeds the
 * budget.  The per-entry checks of validate 1 (offsets order, id range, self-loops,
 * weights >= 1) run on the device when the graph is copied there; a graph that fails
 * them never runs, and polling its ticket returns EINVAL with the reason. */
int viecut_server_submit(viecut_server* s, const viecut_graph_desc* g, uint64_t seed, uint64_t* ticket);
/* Non-blocking: VIECUT_EBUSY until the request finished; then writes the cut, the
 * side bitmap (ceil(n/64) words, may be NULL) and the latency from submit to the
 * moment the result reached the host, and forgets the ticket.  A request whose graph
 * the device check refused returns EINVAL (viecut_last_error gives the reason) and its
 * ticket is forgotten too. */
int viecut_server_poll(viecut_server* s, uint64_t ticket, int64_t* cut, uint64_t* side_bits, double* latency_ms);
/* As viecut_server_poll, with the request's timing breakdown in *info (may be NULL). */
int viecut_server_poll_info(viecut_server* s, uint64_t ticket, int64_t* cut, uint64_t* side_bits,
                            viecut_request_info* info);
/* As viecut_server_poll_info, but waits on the host for the request to finish, at most
 * timeout_ms milliseconds: VIECUT_ETIMEOUT when it has not (the ticket stays valid; poll
 * or wait again).  A host-side bounded wait: no device wait is involved.  EINVAL for a
 * negative timeout. */
int viecut_server_wait(viecut_server* s, uint64_t ticket, double timeout_ms, int64_t* cut, uint64_t* side_bits,
                       viecut_request_info* info);
/* Cancels a request.  A request still queued leaves the queue and never runs; one already
 * on the device runs to its end, but its result is dropped.  Either way the next poll or
 * wait on the ticket returns VIECUT_ECANCELLED and forgets it.  Cancelling twice is a
 * no-op; EINVAL for an unknown ticket (already polled, or never issued). */
int viecut_server_cancel(viecut_server* s, uint64_t ticket);
int viecut_server_get_stats(viecut_server* s, viecut_server_stats* st);
/* Stops the thread (requests still queued or resident are abandoned) and frees all. */
int viecut_server_stop(viecut_server* s);

/* Fault injection for tests (the paper has no counterpart): after the next `after`
 * device allocations of this library (any handle, batch, server or thread), the
 * following `count` fail on the host as if cudaMalloc had run out of memory, and the
 * call that needed them returns VIECUT_ENOMEM.  No GPU fault is involved.  count = 0
 * switches the injection off.  Handles, batches and servers stay usable afterwards: a
 * handle whose load failed holds no graph until the next successful load, and a server
 * answers the requests whose admission failed with VIECUT_ENOMEM.  EINVAL for negative
 * arguments. */
int viecut_debug_fail_device_allocs(int64_t after, int64_t count);

/* The library's sizes of its public structures, for bindings that restate them:
 * sizes[0..7] = sizeof viecut_opts, viecut_stats, viecut_step, viecut_graph_desc,
 * viecut_batch_stats, viecut_server_opts, viecut_server_stats, viecut_request_info (as
 * many as count allows).  Returns the number of sizes the library knows (8), or
 * VIECUT_EINVAL for a null array with count > 0.  Needs no device. */
int viecut_struct_sizes(int64_t* sizes, int32_t count);

#ifdef __cplusplus
}
#endif

#endif /* VIECUT_H_ */
