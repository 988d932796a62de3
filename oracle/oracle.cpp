// CPU ORACLE for the VieCut minimum-cut method — TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, single-threaded restatement of the method of "Practical Minimum
// Cut Algorithms" (Henzinger, Noe, Schulz, Strash; arXiv 1708.06127), in the
// deterministic variant that the GPU library must reproduce bit for bit.  Only the
// test suite, the package's smoke check and the benchmark's CPU-baseline leg load
// this file's library; the product path never does.  It shares no code with the
// CUDA implementation.
//
// Integer arithmetic throughout (weights are positive integers, Section 3; sums in
// int64).  Every function cites the passage it follows.  Where the paper is silent
// or its literal reading is unsafe, the reading taken is marked [R]:
//
//  [R1] Label propagation is synchronous (Jacobi): round r reads only the labels of
//       round r-1.  The paper's traversal is asynchronous in random order (Sec. 4.1,
//       "Label propagation", and Sec. 4.3).
//  [R2] Ties in label propagation are broken by the largest tie-break hash
//       H(key, L) = mix64(key XOR L), key = mix64(seed + G * (level + 1)), mix64 the
//       SplitMix64 output function (Steele, Lea, Flood 2014), G = 0x9e3779b97f4a7c15;
//       the paper breaks ties uniformly at random.  mix64 is a bijection, so (S, H)
//       totally orders distinct labels.
//  [R3] A fixed number of rounds, no first-round restriction (Sec. 4.1 notes the
//       restriction is not used in practice); the correcting step is off unless asked
//       for ([R10]), as in the paper's ER runs.  Optionally (converge) the rounds stop
//       early, as in the configuration VieCut25 of App. D (Table 3): after a round in
//       which at most 1/10000 of the vertices changed their label (changed * 10000 <=
//       n, n the current vertex count), no further round runs.
//  [R4] Cluster ids are ranks of the final label values, ascending.
//  [R5] Padberg-Rinaldi test 2 marks only the edge to each vertex's designated
//       partner p(v) = argmax over neighbours u of (c(v,u), -u); marking every
//       qualifying edge in bulk can merge both sides of a minimum cut.  Test 3 and
//       test 4 are applied to the mutual pairs p(v) = w, p(w) = v (a matching),
//       the scan order of the paper's "runs" replaced by this fixed matching.
//  [R6] "(v, w) is not the only edge adjacent to v or w" is read as: v and w both
//       have at least two distinct neighbours.
//  [R7] PR runs (pass A, then pass B) repeat until a run contracts nothing or
//       pr_runs_max runs were made.  A level that does not shrink the graph ends
//       the level loop.
//  [R8] The final Nagamochi-Ono-Ibaraki rounds start each maximum-adjacency scan at
//       vertex 0, break priority ties by smallest id and compare q(e) with the
//       bound fixed at the start of the round.
//  [R9] The bound improves only on a strictly smaller trivial cut (earliest found
//       wins); a contraction that leaves one vertex ends the run.  The returned
//       side is normalised so original vertex 0 is not in it.
//  [R10] The correcting step (Sec. 4.1, "correcting algorithm"; fixMisplacedVertices
//       of Algorithm 1) is optional and off unless asked for.  On a level's label
//       propagation clustering, a cluster C with 2 <= |C| <= floor(log2 n) (n the
//       current vertex count) has weighted degree d(C) (the weight of the edges
//       leaving C); removing v from C gives d(C - v) = d(C) - c(v, V - C) + c(v, C - v).
//       v is misplaced when d(C - v) < d(C) (its removal lowers the weighted degree of
//       C's vertex in the contracted graph).  Each cluster makes at most one vertex a
//       singleton ("single misplaced vertices"): the misplaced one of smallest
//       d(C - v), ties to the smallest id.  The singletons take the cluster ids after
//       all others, in ascending vertex order.
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <vector>

namespace {

struct Graph {
  int64_t n = 0;
  std::vector<int64_t> off;  // n + 1
  std::vector<int32_t> adj;  // nnz
  std::vector<int64_t> w;    // nnz
};

// SplitMix64 output function (Steele, Lea, Flood 2014), as published.
uint64_t mix64(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ULL;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebULL;
  z ^= z >> 31;
  return z;
}

uint64_t level_key(uint64_t seed, int64_t level) {
  return mix64(seed + 0x9e3779b97f4a7c15ULL * (uint64_t)(level + 1));
}

uint64_t tie_hash(uint64_t key, int32_t label) { return mix64(key ^ (uint64_t)(uint32_t)label); }

// Weighted degree c(v) = sum of the weights of v's incident edges (Sec. 3).
std::vector<int64_t> degrees(const Graph& g) {
  std::vector<int64_t> d(g.n, 0);
  for (int64_t v = 0; v < g.n; ++v)
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) d[v] += g.w[e];
  return d;
}

// Minimum weighted degree and the smallest vertex attaining it: the trivial cut
// that serves as the bound lambda-hat (Sec. 3, last paragraph of "Basic Concepts").
void min_degree(const Graph& g, int64_t* dmin, int64_t* arg) {
  std::vector<int64_t> d = degrees(g);
  *dmin = d[0];
  *arg = 0;
  for (int64_t v = 1; v < g.n; ++v)
    if (d[v] < *dmin) { *dmin = d[v]; *arg = v; }
}

// One round of label propagation (Sec. 4.1, "label propagation algorithm"): every
// vertex moves to the label L of strongest connection S(L) = sum of c(v,u) over
// neighbours u carrying L; [R1] reads lab_in only; [R2] ties by the hash.
void lp_round(const Graph& g, const int32_t* lab_in, uint64_t key, int32_t* lab_out) {
  std::vector<std::pair<int32_t, int64_t>> cand;
  for (int64_t v = 0; v < g.n; ++v) {
    cand.clear();
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) cand.push_back({lab_in[g.adj[e]], g.w[e]});
    if (cand.empty()) { lab_out[v] = lab_in[v]; continue; }
    std::sort(cand.begin(), cand.end());
    int32_t best = -1;
    int64_t best_s = -1;
    uint64_t best_h = 0;
    size_t i = 0;
    while (i < cand.size()) {
      int32_t L = cand[i].first;
      int64_t S = 0;
      while (i < cand.size() && cand[i].first == L) S += cand[i++].second;
      uint64_t H = tie_hash(key, L);
      if (S > best_s || (S == best_s && (H > best_h || (H == best_h && L < best)))) {
        best = L; best_s = S; best_h = H;
      }
    }
    lab_out[v] = best;
  }
}

// [R11] Asynchronous label propagation (optional): the paper visits the vertices in a
// random order and updates labels in place (Sec. 4.1), trading randomness for locality
// by shuffling blocks of consecutive vertex ids and traversing the shuffled blocks one
// after the other (Sec. 4.3; 128-vertex blocks, Sec. 5 setup).  Reading, deterministic:
// the n vertices form ceil(n / blk) blocks of blk consecutive ids; the blocks are
// ordered by the key mix64(key ^ mix64(round + 1) ^ b) of block b (a permutation drawn
// from the level key); the ordered blocks are cut into `waves` consecutive groups of
// equal count (the first B mod waves groups one block longer); the waves run one after
// another, every vertex of a wave choosing its label from the labels as they stand
// when the wave starts (updates of earlier waves of the round included), all vertices
// of a wave at once.  With waves = 1 this is the synchronous round [R1].  The first
// round's restriction (Sec. 4.1: a vertex does not change its label once another vertex
// moved to its block) is applied across waves: in round 0, a vertex keeps its own label
// when a vertex of an earlier wave took that label.
void lp_round_async(const Graph& g, std::vector<int32_t>& lab, uint64_t key, int32_t round, int64_t blk,
                    int64_t waves, bool restrict_first) {
  const int64_t nb = (g.n + blk - 1) / blk;
  std::vector<std::pair<uint64_t, int64_t>> order(nb);
  const uint64_t rk = mix64((uint64_t)round + 1);
  for (int64_t b = 0; b < nb; ++b) order[b] = {mix64(key ^ rk ^ (uint64_t)b), b};
  std::sort(order.begin(), order.end());
  if (waves > nb) waves = nb;
  std::vector<char> joined(restrict_first && round == 0 ? g.n : 0, 0);
  std::vector<int32_t> cur = lab;  // labels as they stand
  int64_t at = 0;
  for (int64_t k = 0; k < waves; ++k) {
    const int64_t len = nb / waves + (k < nb % waves ? 1 : 0);
    std::vector<int64_t> members;
    for (int64_t i = at; i < at + len; ++i)
      for (int64_t v = order[i].second * blk; v < std::min<int64_t>(g.n, (order[i].second + 1) * blk); ++v)
        members.push_back(v);
    at += len;
    // every member chooses from cur (one synchronous step on the members)
    std::vector<int32_t> all(g.n);
    lp_round(g, cur.data(), key, all.data());
    std::vector<int32_t> took;
    for (int64_t v : members) {
      int32_t L = all[v];
      if (!joined.empty() && joined[v]) L = cur[v];  // someone earlier moved to v's block
      if (L != cur[v] && L != (int32_t)v) took.push_back(L);
      cur[v] = L;
    }
    for (int32_t L : took)
      if (!joined.empty()) joined[L] = 1;
  }
  lab.swap(cur);
}

// Contraction of a clustering (Sec. 4.1, "contract it"; contraction semantics in
// Sec. 3): each block becomes one vertex, edges inside a block vanish, parallel
// edges between two blocks merge with summed weight.  [R4] block ids are the ranks
// of the label values.  The coarse lists come out sorted by neighbour id.
// Cluster ids [R4]: ranks of the label values; returns the number of clusters.
int64_t cluster_ids(const Graph& g, const int32_t* labels, std::vector<int32_t>& cid) {
  std::vector<int32_t> vals(labels, labels + g.n);
  std::sort(vals.begin(), vals.end());
  vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
  cid.assign(g.n, 0);
  for (int64_t v = 0; v < g.n; ++v)
    cid[v] = (int32_t)(std::lower_bound(vals.begin(), vals.end(), labels[v]) - vals.begin());
  return (int64_t)vals.size();
}

// The correcting step [R10] on cluster ids cid (c clusters); returns the new count.
int64_t correct_clusters(const Graph& g, std::vector<int32_t>& cid, int64_t c) {
  int64_t lg = 0;
  while ((int64_t(2) << lg) <= g.n) ++lg;  // floor(log2 n)
  std::vector<int64_t> size(c, 0), dc(c, 0), out(g.n, 0), in(g.n, 0);
  for (int64_t v = 0; v < g.n; ++v) size[cid[v]] += 1;
  for (int64_t v = 0; v < g.n; ++v)
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
      if (cid[g.adj[e]] == cid[v]) in[v] += g.w[e];
      else out[v] += g.w[e];
    }
  for (int64_t v = 0; v < g.n; ++v) dc[cid[v]] += out[v];
  std::vector<int64_t> best(c, -1);  // the vertex each cluster gives up, or -1
  for (int64_t v = 0; v < g.n; ++v) {
    const int32_t C = cid[v];
    if (size[C] < 2 || size[C] > lg) continue;
    const int64_t without = dc[C] - out[v] + in[v];
    if (without >= dc[C]) continue;
    const int64_t b = best[C];
    if (b < 0 || without < dc[C] - out[b] + in[b]) best[C] = v;  // ascending v keeps the smallest id on ties
  }
  std::vector<char> single(g.n, 0);
  for (int64_t C = 0; C < c; ++C)
    if (best[C] >= 0) single[best[C]] = 1;
  int64_t k = c;
  for (int64_t v = 0; v < g.n; ++v)
    if (single[v]) cid[v] = (int32_t)k++;
  return k;
}

// Contracts the clustering cid of c clusters.
Graph contract_ids(const Graph& g, const std::vector<int32_t>& cid, int64_t c) {
  struct T { int32_t a, b; int64_t w; };
  std::vector<T> t;
  for (int64_t v = 0; v < g.n; ++v)
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e) {
      int32_t a = cid[v], b = cid[g.adj[e]];
      if (a != b) t.push_back({a, b, g.w[e]});
    }
  std::sort(t.begin(), t.end(), [](const T& x, const T& y) { return x.a < y.a || (x.a == y.a && x.b < y.b); });
  Graph h;
  h.n = c;
  h.off.assign(h.n + 1, 0);
  for (size_t i = 0; i < t.size();) {
    size_t j = i;
    int64_t s = 0;
    while (j < t.size() && t[j].a == t[i].a && t[j].b == t[i].b) s += t[j++].w;
    h.adj.push_back(t[i].b);
    h.w.push_back(s);
    h.off[t[i].a + 1] += 1;
    i = j;
  }
  for (int64_t v = 0; v < h.n; ++v) h.off[v + 1] += h.off[v];
  return h;
}

Graph contract(const Graph& g, const int32_t* labels, std::vector<int32_t>& cid, bool correct = false) {
  int64_t c = cluster_ids(g, labels, cid);
  if (correct) c = correct_clusters(g, cid, c);
  return contract_ids(g, cid, c);
}

// Union-find with the smallest id as representative (Sec. 4.1 uses union-find to
// contract the marked edges; the representative choice makes the result unique).
struct UnionFind {
  std::vector<int32_t> p;
  explicit UnionFind(int64_t n) : p(n) { for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i; }
  int32_t find(int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  bool unite(int32_t a, int32_t b) {
    a = find(a); b = find(b);
    if (a == b) return false;
    if (a < b) p[b] = a; else p[a] = b;
    return true;
  }
};

// Designated partner p(v): the neighbour of heaviest connecting edge, ties to the
// smallest id [R5].  Lists are merged, so each neighbour appears once.
int32_t partner(const Graph& g, int64_t v, int64_t* cw) {
  int32_t best = -1;
  int64_t bw = -1;
  for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e)
    if (g.w[e] > bw || (g.w[e] == bw && g.adj[e] < best)) { bw = g.w[e]; best = g.adj[e]; }
  *cw = bw;
  return best;
}

// Padberg-Rinaldi pass A (Lemma "Padberg-Rinaldi", conditions 1 and 2; first pass of
// a run): mark every edge with c(v,w) >= lambda-hat and, [R5], the edge to the
// designated partner when c(v) <= 2 c(v, p(v)); [R6] both ends need two distinct
// neighbours; contract marked edges with union-find.  Returns the number of unions.
int64_t pr_pass_a(const Graph& g, int64_t lambda_hat, int32_t* labels) {
  std::vector<int64_t> d = degrees(g);
  UnionFind uf(g.n);
  int64_t unions = 0;
  auto ok = [&](int64_t x) { return g.off[x + 1] - g.off[x] >= 2; };
  for (int64_t v = 0; v < g.n; ++v) {
    if (!ok(v)) continue;
    for (int64_t e = g.off[v]; e < g.off[v + 1]; ++e)
      if (g.w[e] >= lambda_hat && ok(g.adj[e])) unions += uf.unite((int32_t)v, g.adj[e]);
    int64_t cw;
    int32_t p = partner(g, v, &cw);
    if (p >= 0 && ok(p) && d[v] <= 2 * cw) unions += uf.unite((int32_t)v, p);
  }
  for (int64_t v = 0; v < g.n; ++v) labels[v] = uf.find((int32_t)v);
  return unions;
}

// Padberg-Rinaldi pass B (conditions 3 and 4; second pass of a run): for each mutual
// pair p(v) = w, p(w) = v [R5], walk the common neighbourhood N(v) n N(w) of the
// sorted lists; condition 3 holds if some common u has c(v) <= 2(c(v,w) + c(v,u))
// and c(w) <= 2(c(v,w) + c(w,u)); condition 4 holds if c(v,w) + sum over common u of
// min(c(v,u), c(w,u)) >= lambda-hat.  Returns the number of contracted pairs.
int64_t pr_pass_b(const Graph& g, int64_t lambda_hat, int32_t* labels) {
  std::vector<int64_t> d = degrees(g);
  std::vector<int32_t> p(g.n);
  std::vector<int64_t> pw(g.n);
  for (int64_t v = 0; v < g.n; ++v) p[v] = partner(g, v, &pw[v]);
  for (int64_t v = 0; v < g.n; ++v) labels[v] = (int32_t)v;
  int64_t pairs = 0;
  for (int64_t v = 0; v < g.n; ++v) {
    int32_t w = p[v];
    if (w < 0 || w <= v || p[w] != v) continue;
    if (g.off[v + 1] - g.off[v] < 2 || g.off[w + 1] - g.off[w] < 2) continue;
    int64_t cvw = pw[v];
    bool pr3 = false;
    int64_t sum = cvw;
    int64_t i = g.off[v], j = g.off[w];
    while (i < g.off[v + 1] && j < g.off[w + 1]) {
      if (g.adj[i] < g.adj[j]) ++i;
      else if (g.adj[i] > g.adj[j]) ++j;
      else {
        int64_t cvu = g.w[i], cwu = g.w[j];
        if (d[v] <= 2 * (cvw + cvu) && d[w] <= 2 * (cvw + cwu)) pr3 = true;
        sum += std::min(cvu, cwu);
        ++i; ++j;
      }
    }
    if (pr3 || sum >= lambda_hat) { labels[w] = (int32_t)v; ++pairs; }
  }
  return pairs;
}

// One round of the Nagamochi-Ono-Ibaraki algorithm (Sec. 3, "The Minimum Cut
// Algorithm of Nagamochi, Ono and Ibaraki"): a maximum-adjacency scan visits next
// the unvisited vertex most strongly connected to the visited set; when x is visited
// each unvisited neighbour y gains r(y) += c(x,y) and q(x,y) = r(y) is a lower bound
// on the smallest x-y cut; every edge with q >= lambda-hat is contracted.  [R8].
int64_t noi_round(const Graph& g, int64_t lambda_hat, int32_t* labels) {
  std::vector<int64_t> r(g.n, 0);
  std::vector<char> seen(g.n, 0);
  UnionFind uf(g.n);
  int64_t unions = 0;
  for (int64_t step = 0; step < g.n; ++step) {
    int64_t x = -1;
    for (int64_t v = 0; v < g.n; ++v)
      if (!seen[v] && (x < 0 || r[v] > r[x])) x = v;
    seen[x] = 1;
    for (int64_t e = g.off[x]; e < g.off[x + 1]; ++e) {
      int32_t y = g.adj[e];
      if (seen[y]) continue;
      r[y] += g.w[e];
      if (r[y] >= lambda_hat) unions += uf.unite((int32_t)x, y);
    }
  }
  for (int64_t v = 0; v < g.n; ++v) labels[v] = uf.find((int32_t)v);
  return unions;
}

struct Step {
  int32_t kind;  // 0 initial, 1 label-propagation contraction, 2 PR pass A, 3 PR pass B, 4 NOI round
  int32_t level;
  int64_t n, nnz, lambda_hat;
};

struct Run {
  int64_t n0;
  std::vector<int32_t> cur;  // original vertex -> current coarse vertex
  std::vector<char> side;    // snapshot of the best trivial cut, per original vertex
  int64_t lambda_hat = 0;
  std::vector<Step> trace;
  int32_t level = 0;
};

// After a contraction: if the coarse graph has a strictly smaller trivial cut,
// record it as the new bound and snapshot its side (Sec. 4, second paragraph:
// "After every contraction ... minimum node degree ..."; [R9]).
void update_bound(Run& run, const Graph& g) {
  int64_t dmin, arg;
  min_degree(g, &dmin, &arg);
  if (dmin < run.lambda_hat) {
    run.lambda_hat = dmin;
    for (size_t i = 0; i < run.cur.size(); ++i) run.side[i] = run.cur[i] == arg;
  }
}

// Applies a contraction; returns false when the run must stop (one vertex left, or
// a zero bound: an isolated vertex means a cut of weight 0, Appendix B).
bool apply(Run& run, Graph& g, const int32_t* labels, int32_t kind, bool correct = false) {
  std::vector<int32_t> cid;
  Graph h = contract(g, labels, cid, correct);
  for (auto& c : run.cur) c = cid[c];
  g = std::move(h);
  if (g.n <= 1) {
    run.trace.push_back({kind, run.level, g.n, (int64_t)g.adj.size(), run.lambda_hat});
    return false;
  }
  update_bound(run, g);
  run.trace.push_back({kind, run.level, g.n, (int64_t)g.adj.size(), run.lambda_hat});
  return run.lambda_hat > 0;
}

// The label-propagation rounds of one level from the identity labelling: lp_iters
// rounds, or ([R3], converge) fewer when a round changes at most 1/10000 of the labels
// (VieCut25, App. D).  Returns the number of rounds run; lab holds the final labels.
// lp_async: 0 synchronous rounds [R1]; 1 asynchronous rounds [R11] (blocks of 128,
// eight waves); 2 the same with the first round's restriction.
int32_t lp_level(const Graph& g, uint64_t key, int32_t lp_iters, bool converge, std::vector<int32_t>& lab,
                 std::vector<int32_t>& nxt, int32_t lp_async = 0) {
  lab.resize(g.n);
  nxt.resize(g.n);
  for (int64_t v = 0; v < g.n; ++v) lab[v] = (int32_t)v;
  for (int32_t r = 0; r < lp_iters; ++r) {
    if (lp_async) {
      nxt = lab;
      lp_round_async(g, nxt, key, r, 128, 8, lp_async == 2);
    } else {
      lp_round(g, lab.data(), key, nxt.data());
    }
    int64_t changed = 0;
    for (int64_t v = 0; v < g.n; ++v) changed += nxt[v] != lab[v];
    lab.swap(nxt);
    if (converge && changed * 10000 <= g.n) return r + 1;
  }
  return lp_iters;
}

// Algorithm 1 (Appendix A) in the deterministic variant: levels of label
// propagation + cluster contraction + Padberg-Rinaldi runs while more than n0
// vertices remain, then Nagamochi-Ono-Ibaraki on the kernel; the bound is the
// smallest trivial cut seen (Sec. 4, "Throughout our algorithm we maintain ...").
void viecut(Graph g, uint64_t seed, int32_t lp_iters, int64_t n0, int32_t pr_runs_max, bool correct, bool converge,
            int32_t lp_async, Run& run) {
  int64_t n = g.n;
  run.cur.resize(n);
  run.side.assign(n, 0);
  for (int64_t i = 0; i < n; ++i) run.cur[i] = (int32_t)i;
  int64_t dmin, arg;
  min_degree(g, &dmin, &arg);
  run.lambda_hat = dmin;
  run.side[arg] = 1;
  run.trace.push_back({0, 0, g.n, (int64_t)g.adj.size(), dmin});
  if (dmin == 0) return;  // isolated vertex (Sec. 4.1, Appendix B)
  std::vector<int32_t> lab, nxt;
  while (g.n > n0) {
    int64_t n_start = g.n;
    uint64_t key = level_key(seed, run.level);
    lp_level(g, key, lp_iters, converge, lab, nxt, lp_async);
    if (!apply(run, g, lab.data(), 1, correct)) return;
    for (int32_t runi = 0; runi < pr_runs_max; ++runi) {
      bool any = false;
      lab.resize(g.n);
      if (pr_pass_a(g, run.lambda_hat, lab.data()) > 0) {
        if (!apply(run, g, lab.data(), 2)) return;
        any = true;
      }
      lab.resize(g.n);
      if (pr_pass_b(g, run.lambda_hat, lab.data()) > 0) {
        if (!apply(run, g, lab.data(), 3)) return;
        any = true;
      }
      if (!any) break;
    }
    run.level += 1;
    if (g.n == n_start) break;  // [R7] no progress
  }
  while (g.n > 1) {
    lab.resize(g.n);
    int64_t u = noi_round(g, run.lambda_hat, lab.data());
    if (u == 0) return;  // cannot happen while lambda-hat <= min degree (NOI, Sec. 3)
    if (!apply(run, g, lab.data(), 4)) return;
  }
}

Graph load(int64_t n, const int64_t* off, const int32_t* adj, const void* w, int32_t wbytes) {
  Graph g;
  g.n = n;
  g.off.assign(off, off + n + 1);
  int64_t nnz = off[n];
  g.adj.assign(adj, adj + nnz);
  g.w.resize(nnz);
  for (int64_t e = 0; e < nnz; ++e)
    g.w[e] = wbytes == 8 ? ((const int64_t*)w)[e] : (int64_t)((const int32_t*)w)[e];
  return g;
}

}  // namespace

extern "C" {

typedef struct {
  int32_t kind, level;
  int64_t n, nnz, lambda_hat;
} orc_step;

uint64_t orc_mix64(uint64_t z) { return mix64(z); }
uint64_t orc_level_key(uint64_t seed, int64_t level) { return level_key(seed, level); }

void orc_degrees(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w, int64_t* deg) {
  Graph g = load(n, off, adj, w, 8);
  std::vector<int64_t> d = degrees(g);
  memcpy(deg, d.data(), sizeof(int64_t) * n);
}

void orc_lp_round(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w,
                  const int32_t* lab_in, uint64_t key, int32_t* lab_out) {
  Graph g = load(n, off, adj, w, 8);
  lp_round(g, lab_in, key, lab_out);
}

// One asynchronous round [R11] from lab (in place) with the given block size and wave
// count; restrict_first applies the first round's restriction.
void orc_lp_round_async(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w, int32_t* lab,
                        uint64_t key, int32_t round, int64_t blk, int64_t waves, int32_t restrict_first) {
  Graph g = load(n, off, adj, w, 8);
  std::vector<int32_t> l(lab, lab + n);
  lp_round_async(g, l, key, round, blk, waves, restrict_first != 0);
  memcpy(lab, l.data(), sizeof(int32_t) * n);
}

// One level's rounds from the identity (lp_level): lab_out[n] the final labels; returns
// the rounds run.
int32_t orc_lp_level(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w, uint64_t key,
                     int32_t lp_iters, int32_t converge, int32_t* lab_out, int32_t lp_async) {
  Graph g = load(n, off, adj, w, 8);
  std::vector<int32_t> lab, nxt;
  int32_t r = lp_level(g, key, lp_iters, converge != 0, lab, nxt, lp_async);
  memcpy(lab_out, lab.data(), sizeof(int32_t) * n);
  return r;
}

// Contracts by labels.  Outputs: cid[n], coarse n in *cn, coarse CSR in coff (cap
// n+1), cadj / cw (cap nnz).  Returns the coarse nnz.
int64_t orc_contract(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w,
                     const int32_t* labels, int32_t* cid, int64_t* cn, int64_t* coff,
                     int32_t* cadj, int64_t* cw) {
  Graph g = load(n, off, adj, w, 8);
  std::vector<int32_t> c;
  Graph h = contract(g, labels, c);
  memcpy(cid, c.data(), sizeof(int32_t) * n);
  *cn = h.n;
  memcpy(coff, h.off.data(), sizeof(int64_t) * (h.n + 1));
  memcpy(cadj, h.adj.data(), sizeof(int32_t) * h.adj.size());
  memcpy(cw, h.w.data(), sizeof(int64_t) * h.w.size());
  return (int64_t)h.adj.size();
}

// The correcting step [R10] on the clustering `labels`: cid[n] receives the corrected
// cluster ids; returns their count.
int64_t orc_correct(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w, const int32_t* labels,
                    int32_t* cid) {
  Graph g = load(n, off, adj, w, 8);
  std::vector<int32_t> c;
  int64_t k = correct_clusters(g, c, cluster_ids(g, labels, c));
  memcpy(cid, c.data(), sizeof(int32_t) * n);
  return k;
}

int64_t orc_pr_pass_a(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w,
                      int64_t lambda_hat, int32_t* labels) {
  Graph g = load(n, off, adj, w, 8);
  return pr_pass_a(g, lambda_hat, labels);
}

int64_t orc_pr_pass_b(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w,
                      int64_t lambda_hat, int32_t* labels) {
  Graph g = load(n, off, adj, w, 8);
  return pr_pass_b(g, lambda_hat, labels);
}

int64_t orc_noi_round(int64_t n, const int64_t* off, const int32_t* adj, const int64_t* w,
                      int64_t lambda_hat, int32_t* labels) {
  Graph g = load(n, off, adj, w, 8);
  return noi_round(g, lambda_hat, labels);
}

// Whole method.  w has wbytes = 4 (int32) or 8 (int64) per entry.  side_bits holds
// ceil(n/64) words.  trace (nullable) receives up to trace_cap steps; the number of
// steps made is returned through *trace_len.
int orc_viecut(int64_t n, const int64_t* off, const int32_t* adj, const void* w, int32_t wbytes,
               uint64_t seed, int32_t lp_iters, int64_t n0, int32_t pr_runs_max,
               int64_t* cut, uint64_t* side_bits, orc_step* trace, int64_t trace_cap,
               int64_t* trace_len, int32_t correct, int32_t converge, int32_t lp_async) {
  if (n < 2 || lp_async < 0 || lp_async > 2) return -1;
  Run run;
  viecut(load(n, off, adj, w, wbytes), seed, lp_iters, n0, pr_runs_max, correct != 0, converge != 0, lp_async, run);
  *cut = run.lambda_hat;
  bool flip = run.side[0] != 0;
  int64_t words = (n + 63) / 64;
  for (int64_t k = 0; k < words; ++k) side_bits[k] = 0;
  for (int64_t i = 0; i < n; ++i)
    if ((run.side[i] != 0) != flip) side_bits[i >> 6] |= 1ULL << (i & 63);
  if (trace_len) *trace_len = (int64_t)run.trace.size();
  if (trace)
    for (int64_t k = 0; k < (int64_t)run.trace.size() && k < trace_cap; ++k) {
      trace[k].kind = run.trace[k].kind;
      trace[k].level = run.trace[k].level;
      trace[k].n = run.trace[k].n;
      trace[k].nnz = run.trace[k].nnz;
      trace[k].lambda_hat = run.trace[k].lambda_hat;
    }
  return 0;
}

}  // extern "C"
