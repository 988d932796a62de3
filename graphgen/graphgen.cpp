// Seeded synthetic graph generators for the minimum-cut workloads.
//
// This module only produces inputs. It holds none of the minimum-cut method's
// arithmetic and is shared by the CPU oracle, the tests and the benchmark.
//
// Families (shapes follow the paper's instances, Section 5 and Appendix C):
//   * random hyperbolic graphs, threshold model (Krioukov et al. 2010), generated
//     with a band decomposition of the disk in the spirit of von Looz et al. 2015;
//   * Erdos-Renyi G(n,p) by geometric edge skipping (Batagelj and Brandes 2005);
//   * planted-cut graphs: ER blocks joined by a few random bridges;
//   * k-core peeling (Batagelj and Zaversnik 2003) and largest-connected-component
//     restriction, the preprocessing of Appendix C.
//
// Determinism: every random number is a pure function of (seed, stream, counter)
// through the SplitMix64 output function (Steele, Lea and Flood 2014), and all
// floating point that decides an edge uses only +, -, *, /, sqrt and the series
// below (built with -ffp-contract=off), so x86-64 and aarch64 hosts produce the same
// graph bit for bit, whatever the number of threads.
#include <stdint.h>
#include <math.h>
#include <string.h>
#include <stdlib.h>
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- random numbers
inline uint64_t sm_mix(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ULL;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebULL;
  z ^= z >> 31;
  return z;
}
const uint64_t kGolden = 0x9e3779b97f4a7c15ULL;

// Counter-based stream: value number `i` of stream `s` under `seed`.
inline uint64_t rnd64(uint64_t seed, uint64_t s, uint64_t i) {
  return sm_mix(sm_mix(seed + kGolden * (s + 1)) + kGolden * (i + 1));
}
// Uniform double in [0, 1) from the top 53 bits.
inline double rnd01(uint64_t seed, uint64_t s, uint64_t i) {
  return (double)(rnd64(seed, s, i) >> 11) * (1.0 / 9007199254740992.0);
}

// ------------------------------------------------------ deterministic elementary math
const double kPi = 3.141592653589793;
const double kHalfPi = 1.5707963267948966;
const double kLn2Hi = 0.6931471803691238;     // high part of ln 2 (exact in 32 bits)
const double kLn2Lo = 1.9082149292705877e-10;  // ln 2 - kLn2Hi
const double kLn2 = 0.6931471805599453;

// exp(x) by Cody-Waite reduction x = k ln2 + r, |r| <= ln2/2, and a Taylor series.
double det_exp(double x) {
  double k = floor(x * (1.0 / kLn2) + 0.5);
  double r = (x - k * kLn2Hi) - k * kLn2Lo;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i <= 24; ++i) {
    term = term * r / (double)i;
    sum = sum + term;
  }
  return ldexp(sum, (int)k);
}
double det_cosh(double x) { double e = det_exp(x); return 0.5 * (e + 1.0 / e); }
double det_sinh(double x) { double e = det_exp(x); return 0.5 * (e - 1.0 / e); }

// log(x), x > 0: x = m 2^e with m in [sqrt(1/2), sqrt(2)); log m = 2 atanh((m-1)/(m+1)).
double det_log(double x) {
  int e;
  double m = frexp(x, &e);  // m in [0.5, 1)
  if (m < 0.7071067811865476) { m = m * 2.0; e = e - 1; }
  double z = (m - 1.0) / (m + 1.0);
  double z2 = z * z, p = z, sum = 0.0;
  for (int k = 0; k < 30; ++k) {
    sum = sum + p / (double)(2 * k + 1);
    p = p * z2;
  }
  return 2.0 * sum + (double)e * kLn2;
}

// atan(x) for x >= 0: fold x > 1 to pi/2 - atan(1/x), halve the angle twice with
// atan(x) = 2 atan(x / (1 + sqrt(1 + x^2))), then sum the Maclaurin series.
double det_atan_pos(double x) {
  bool inv = x > 1.0;
  if (inv) x = 1.0 / x;
  x = x / (1.0 + sqrt(1.0 + x * x));
  x = x / (1.0 + sqrt(1.0 + x * x));
  double x2 = x * x, p = x, sum = 0.0;
  for (int k = 0; k < 24; ++k) {
    double t = p / (double)(2 * k + 1);
    sum = (k & 1) ? sum - t : sum + t;
    p = p * x2;
  }
  sum = 4.0 * sum;
  return inv ? kHalfPi - sum : sum;
}
// acos(x), x in [-1, 1]: acos x = 2 atan(sqrt((1 - x) / (1 + x))).
double det_acos(double x) {
  if (x <= -1.0) return kPi;
  if (x >= 1.0) return 0.0;
  return 2.0 * det_atan_pos(sqrt((1.0 - x) / (1.0 + x)));
}

// sin and cos of 2 pi u for u in [0, 1): quadrant reduction on u (exact), fold to
// [0, pi/4], Taylor series.
void det_sincos2pi(double u, double* s, double* c) {
  double t = u * 4.0;
  double q = floor(t);
  double f = t - q;  // in [0, 1), exact
  bool comp = f > 0.5;
  double x = (comp ? (1.0 - f) : f) * kHalfPi;
  double x2 = x * x;
  double sn = 0.0, cs = 0.0, ps = x, pc = 1.0;
  for (int k = 0; k < 12; ++k) {
    sn = (k & 1) ? sn - ps : sn + ps;
    cs = (k & 1) ? cs - pc : cs + pc;
    ps = ps * x2 / (double)((2 * k + 2) * (2 * k + 3));
    pc = pc * x2 / (double)((2 * k + 1) * (2 * k + 2));
  }
  double sa = comp ? cs : sn, ca = comp ? sn : cs;  // sin, cos of f * pi/2
  switch ((int)q & 3) {
    case 0: *s = sa; *c = ca; break;
    case 1: *s = ca; *c = -sa; break;
    case 2: *s = -sa; *c = -ca; break;
    default: *s = -ca; *c = sa; break;
  }
}

// ------------------------------------------------------------------ threading
template <class F>
void parallel_ranges(int64_t n, F f) {
  unsigned hw = std::thread::hardware_concurrency();
  int64_t nt = hw ? (int64_t)hw : 4;
  if (nt > 64) nt = 64;
  if (n < 4096) nt = 1;
  if (nt == 1) { f((int64_t)0, n, 0); return; }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) {
    int64_t a = n * t / nt, b = n * (t + 1) / nt;
    th.emplace_back([=]() { f(a, b, (int)t); });
  }
  for (auto& x : th) x.join();
}

// Work-stealing loop over items [0, n) in chunks; f(i) must be independent per i.
template <class F>
void parallel_items(int64_t n, int64_t chunk, F f) {
  unsigned hw = std::thread::hardware_concurrency();
  int64_t nt = hw ? (int64_t)hw : 4;
  if (nt > 64) nt = 64;
  if (n < chunk * 2) nt = 1;
  std::atomic<int64_t> next(0);
  auto body = [&]() {
    for (;;) {
      int64_t a = next.fetch_add(chunk);
      if (a >= n) break;
      int64_t b = std::min(n, a + chunk);
      for (int64_t i = a; i < b; ++i) f(i);
    }
  };
  if (nt == 1) { body(); return; }
  std::vector<std::thread> th;
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(body);
  for (auto& x : th) x.join();
}

// ------------------------------------------------------------ CSR containers
struct Csr {
  int64_t n = 0;
  std::vector<int64_t> off;
  std::vector<int32_t> adj;
  std::vector<int32_t> w;
};

// Builds a CSR from per-vertex neighbour lists that are already complete in both
// directions.
Csr csr_from_lists(int64_t n, const std::vector<std::vector<int32_t>>& lists) {
  Csr g;
  g.n = n;
  g.off.assign(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) g.off[v + 1] = g.off[v] + (int64_t)lists[v].size();
  g.adj.resize(g.off[n]);
  parallel_ranges(n, [&](int64_t a, int64_t b, int) {
    for (int64_t v = a; v < b; ++v)
      std::copy(lists[v].begin(), lists[v].end(), g.adj.begin() + g.off[v]);
  });
  g.w.assign(g.off[n], 1);
  return g;
}

// ------------------------------------------------------ random hyperbolic graphs
// Points on a hyperbolic disk of radius R; radial density alpha sinh(alpha r) /
// (cosh(alpha R) - 1), angles uniform. Vertices u, v are adjacent iff their
// hyperbolic distance is below R, i.e.
//   cosh r_u cosh r_v - sinh r_u sinh r_v cos(theta_u - theta_v) < cosh R.
struct RhgPoint {
  double ch, sh, c, s, u;  // cosh r, sinh r, cos theta, sin theta, theta / 2pi
};

inline void rhg_radius(double alpha, double cosh_aR, double ur, double* ch, double* sh) {
  // inverse CDF: cosh(alpha r) = 1 + u (cosh(alpha R) - 1)
  double X = 1.0 + ur * (cosh_aR - 1.0);
  double r = det_log(X + sqrt((X - 1.0) * (X + 1.0))) / alpha;  // acosh(X) / alpha
  *ch = det_cosh(r);
  *sh = det_sinh(r);
}

// Expected number of neighbours of a vertex, times 1/(n-1): E over two independent
// points of Pr[adjacent] = dtheta_max(r1, r2) / pi, by a midpoint rule in the
// radial CDF variable.
double rhg_pair_prob(double R, double alpha, int M) {
  double C = det_cosh(R), cosh_aR = det_cosh(alpha * R);
  std::vector<double> ch(M), sh(M);
  for (int i = 0; i < M; ++i) rhg_radius(alpha, cosh_aR, (i + 0.5) / M, &ch[i], &sh[i]);
  double tot = 0.0;
  for (int i = 0; i < M; ++i) {
    double row = 0.0;
    for (int j = 0; j < M; ++j) {
      double den = sh[i] * sh[j];
      double T = den > 0 ? (ch[i] * ch[j] - C) / den : -2.0;
      row += det_acos(T < -1.0 ? -1.0 : (T > 1.0 ? 1.0 : T));
    }
    tot += row;
  }
  return tot / ((double)M * (double)M) / kPi;
}

// Disk radius giving the requested expected average degree: secant iteration on
// log(expected degree) as a function of R (nearly linear with slope -1/2), started
// from the asymptotic estimate R = 2 ln(n xi^2 (2/pi) / k), xi = alpha / (alpha - 1/2).
double rhg_radius_for_degree(int64_t n, double avg_deg, double alpha) {
  double xi = alpha / (alpha - 0.5);
  double R0 = 2.0 * det_log((double)n * xi * xi * (2.0 / kPi) / avg_deg);
  if (R0 < 1.0) R0 = 1.0;
  const int M = 384;
  auto f = [&](double R) { return det_log((double)(n - 1) * rhg_pair_prob(R, alpha, M)) - det_log(avg_deg); };
  double R1 = R0, f1 = f(R1);
  double R2 = R1 + 2.0 * f1, f2 = f(R2);
  for (int it = 0; it < 30; ++it) {
    if (f2 == f1) break;
    double R3 = R2 - f2 * (R2 - R1) / (f2 - f1);
    if (R3 < 0.1) R3 = 0.1;
    R1 = R2; f1 = f2; R2 = R3; f2 = f(R2);
    if (fabs(f2) < 1e-7) break;
  }
  return R2;
}

Csr gen_rhg(int64_t n, double avg_deg, double gamma, uint64_t seed) {
  double alpha = (gamma - 1.0) / 2.0;
  double R = rhg_radius_for_degree(n, avg_deg, alpha);
  double C = det_cosh(R), cosh_aR = det_cosh(alpha * R);
  // draw points; stream 0 = radial, stream 1 = angular
  std::vector<RhgPoint> raw(n);
  parallel_ranges(n, [&](int64_t a, int64_t b, int) {
    for (int64_t i = a; i < b; ++i) {
      RhgPoint p;
      rhg_radius(alpha, cosh_aR, rnd01(seed, 0, i), &p.ch, &p.sh);
      p.u = rnd01(seed, 1, i);
      det_sincos2pi(p.u, &p.s, &p.c);
      raw[i] = p;
    }
  });
  // vertex ids follow angular order (ties by draw index)
  std::vector<int64_t> ord(n);
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) {
    return raw[a].u < raw[b].u || (raw[a].u == raw[b].u && a < b);
  });
  std::vector<RhgPoint> P(n);
  for (int64_t i = 0; i < n; ++i) P[i] = raw[ord[i]];
  raw.clear();
  raw.shrink_to_fit();

  // radial bands of width 0.75 counted inwards from R; band 0 starts at r = 0
  const double width = 0.75;
  int K = (int)ceil(R / width);
  if (K < 1) K = 1;
  std::vector<double> lo(K), lo_ch(K), lo_sh(K);
  for (int j = 0; j < K; ++j) {
    lo[j] = (j == 0) ? 0.0 : R - (double)(K - j) * width;
    lo_ch[j] = det_cosh(lo[j]);
    lo_sh[j] = det_sinh(lo[j]);
  }
  std::vector<std::vector<int32_t>> band(K);
  std::vector<std::vector<double>> band_u(K);
  for (int64_t i = 0; i < n; ++i) {
    int j = (int)(std::upper_bound(lo_ch.begin(), lo_ch.end(), P[i].ch) - lo_ch.begin()) - 1;
    if (j < 0) j = 0;
    band[j].push_back((int32_t)i);
    band_u[j].push_back(P[i].u);
  }

  std::vector<std::vector<int32_t>> lists(n);
  const double margin = 1e-7;  // radians; covers rounding of the exact test
  parallel_items(n, 256, [&](int64_t i) {
    const RhgPoint& p = P[i];
    std::vector<int32_t>& out = lists[i];
    for (int j = 0; j < K; ++j) {
      const std::vector<int32_t>& B = band[j];
      if (B.empty()) continue;
      double du;
      if (j == 0 || lo_sh[j] <= 0.0 || p.sh <= 0.0) {
        du = 1.0;
      } else {
        double T = (p.ch * lo_ch[j] - C) / (p.sh * lo_sh[j]);
        if (T <= -1.0) du = 1.0;
        else du = (acos(T >= 1.0 ? 1.0 : T) + margin) / (2.0 * kPi);
      }
      auto test = [&](int32_t q) {
        if (q == (int32_t)i) return;
        const RhgPoint& o = P[q];
        double cd = p.c * o.c + p.s * o.s;
        if (p.ch * o.ch - p.sh * o.sh * cd < C) out.push_back(q);
      };
      const std::vector<double>& U = band_u[j];
      if (du >= 0.5) {
        for (int32_t q : B) test(q);
        continue;
      }
      double a = p.u - du, b = p.u + du;
      auto scan = [&](double x0, double x1) {
        size_t s = std::lower_bound(U.begin(), U.end(), x0) - U.begin();
        size_t e = std::upper_bound(U.begin(), U.end(), x1) - U.begin();
        for (size_t k = s; k < e; ++k) test(B[k]);
      };
      if (a < 0.0) { scan(a + 1.0, 1.0); scan(0.0, b); }
      else if (b >= 1.0) { scan(a, 1.0); scan(0.0, b - 1.0); }
      else scan(a, b);
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  });
  return csr_from_lists(n, lists);
}

// ---------------------------------------------------------------- Erdos-Renyi
// G(n, p) on vertex ids [base, base + n): row v draws its neighbours w < v by
// geometric skips; each accepted pair also draws its weight from the same stream.
struct EdgeRow {
  std::vector<int32_t> nbr;
  std::vector<int32_t> w;
};

void gen_er_rows(int64_t n, double p, uint64_t seed, uint64_t stream_base, int32_t wlo,
                 int32_t whi, std::vector<EdgeRow>& rows) {
  rows.assign(n, EdgeRow());
  if (p <= 0.0) return;
  double lq = det_log(1.0 - p);
  parallel_items(n, 1024, [&](int64_t v) {
    EdgeRow& r = rows[v];
    uint64_t s = stream_base + (uint64_t)v;
    uint64_t ctr = 0;
    int64_t w = -1;
    for (;;) {
      double u = rnd01(seed, s, ctr++);
      double skip = (p >= 1.0) ? 0.0 : floor(det_log(1.0 - u) / lq);
      if (skip > (double)n) break;
      w += (int64_t)skip + 1;
      if (w >= v) break;
      int32_t wt = wlo;
      if (whi > wlo) wt = wlo + (int32_t)(rnd01(seed, s, ctr++) * (double)(whi - wlo + 1));
      if (wt > whi) wt = whi;
      r.nbr.push_back((int32_t)w);
      r.w.push_back(wt);
    }
  });
}

// Assembles a symmetric CSR from rows of lower neighbours (row v holds w < v) plus
// an optional list of extra undirected edges; neighbour lists sorted by (id, weight).
Csr csr_from_rows(int64_t n, const std::vector<EdgeRow>& rows, int64_t base,
                  const std::vector<int64_t>& ex_u, const std::vector<int64_t>& ex_v,
                  const std::vector<int32_t>& ex_w, Csr* into = nullptr) {
  Csr g;
  g.n = n;
  std::vector<int64_t> deg(n, 0);
  for (int64_t v = 0; v < (int64_t)rows.size(); ++v) {
    deg[base + v] += (int64_t)rows[v].nbr.size();
    for (int32_t w : rows[v].nbr) deg[base + w] += 1;
  }
  for (size_t e = 0; e < ex_u.size(); ++e) { deg[ex_u[e]]++; deg[ex_v[e]]++; }
  g.off.assign(n + 1, 0);
  for (int64_t v = 0; v < n; ++v) g.off[v + 1] = g.off[v] + deg[v];
  g.adj.resize(g.off[n]);
  g.w.resize(g.off[n]);
  std::vector<int64_t> pos(g.off.begin(), g.off.end() - 1);
  for (int64_t v = 0; v < (int64_t)rows.size(); ++v) {
    int64_t gv = base + v;
    for (size_t k = 0; k < rows[v].nbr.size(); ++k) {
      int64_t gw = base + rows[v].nbr[k];
      g.adj[pos[gv]] = (int32_t)gw; g.w[pos[gv]++] = rows[v].w[k];
      g.adj[pos[gw]] = (int32_t)gv; g.w[pos[gw]++] = rows[v].w[k];
    }
  }
  for (size_t e = 0; e < ex_u.size(); ++e) {
    g.adj[pos[ex_u[e]]] = (int32_t)ex_v[e]; g.w[pos[ex_u[e]]++] = ex_w[e];
    g.adj[pos[ex_v[e]]] = (int32_t)ex_u[e]; g.w[pos[ex_v[e]]++] = ex_w[e];
  }
  (void)into;
  // sort each list by (neighbour, weight)
  parallel_items(n, 4096, [&](int64_t v) {
    int64_t a = g.off[v], b = g.off[v + 1];
    bool sorted = true;
    for (int64_t k = a + 1; k < b; ++k)
      if (g.adj[k - 1] > g.adj[k] || (g.adj[k - 1] == g.adj[k] && g.w[k - 1] > g.w[k])) { sorted = false; break; }
    if (sorted) return;
    std::vector<std::pair<int32_t, int32_t>> t(b - a);
    for (int64_t k = a; k < b; ++k) t[k - a] = {g.adj[k], g.w[k]};
    std::sort(t.begin(), t.end());
    for (int64_t k = a; k < b; ++k) { g.adj[k] = t[k - a].first; g.w[k] = t[k - a].second; }
  });
  return g;
}

Csr gen_er(int64_t n, double avg_deg, uint64_t seed, int32_t wlo, int32_t whi) {
  double p = n > 1 ? avg_deg / (double)(n - 1) : 0.0;
  if (p > 1.0) p = 1.0;
  std::vector<EdgeRow> rows;
  gen_er_rows(n, p, seed, 0, wlo, whi, rows);
  std::vector<int64_t> eu, ev;
  std::vector<int32_t> ew;
  return csr_from_rows(n, rows, 0, eu, ev, ew);
}

// k blocks of bn vertices, ER inside each block with the given average degree,
// plus `bridges` edges between two distinct uniformly chosen blocks at uniformly
// chosen vertices; all weights uniform in [wlo, whi].
Csr gen_planted(int64_t blocks, int64_t bn, double avg_deg, int64_t bridges, uint64_t seed,
                int32_t wlo, int32_t whi) {
  int64_t n = blocks * bn;
  double p = bn > 1 ? avg_deg / (double)(bn - 1) : 0.0;
  std::vector<EdgeRow> all(n);
  for (int64_t b = 0; b < blocks; ++b) {
    std::vector<EdgeRow> rows;
    gen_er_rows(bn, p, seed, (uint64_t)(b + 1) << 32, wlo, whi, rows);
    for (int64_t v = 0; v < bn; ++v) {
      EdgeRow& r = rows[v];
      for (auto& x : r.nbr) x = (int32_t)(x + b * bn);
      all[b * bn + v] = std::move(r);
    }
  }
  std::vector<int64_t> eu, ev;
  std::vector<int32_t> ew;
  const uint64_t s = 0xB1D9E5ULL;
  for (int64_t e = 0; e < bridges; ++e) {
    uint64_t c = (uint64_t)e * 8;
    int64_t b1 = (int64_t)(rnd01(seed, s, c) * (double)blocks);
    int64_t b2 = (int64_t)(rnd01(seed, s, c + 1) * (double)(blocks - 1));
    if (b2 >= b1) b2++;
    int64_t x = b1 * bn + (int64_t)(rnd01(seed, s, c + 2) * (double)bn);
    int64_t y = b2 * bn + (int64_t)(rnd01(seed, s, c + 3) * (double)bn);
    int32_t wt = wlo + (int32_t)(rnd01(seed, s, c + 4) * (double)(whi - wlo + 1));
    if (wt > whi) wt = whi;
    eu.push_back(x); ev.push_back(y); ew.push_back(wt);
  }
  return csr_from_rows(n, all, 0, eu, ev, ew);
}

// ------------------------------------------------------- k-core and components
// Vertices kept by peeling every vertex of (unweighted) degree < k, repeatedly.
std::vector<char> kcore_keep(const int64_t* off, const int32_t* adj, int64_t n, int64_t k) {
  std::vector<int64_t> deg(n);
  std::vector<char> keep(n, 1);
  std::vector<int64_t> stack;
  for (int64_t v = 0; v < n; ++v) {
    deg[v] = off[v + 1] - off[v];
    if (deg[v] < k) { keep[v] = 0; stack.push_back(v); }
  }
  while (!stack.empty()) {
    int64_t v = stack.back();
    stack.pop_back();
    for (int64_t e = off[v]; e < off[v + 1]; ++e) {
      int64_t u = adj[e];
      if (keep[u] && --deg[u] < k) { keep[u] = 0; stack.push_back(u); }
    }
  }
  return keep;
}

// Restricts `keep` to its largest connected component (ties: the one holding the
// smallest vertex id).
void largest_component(const int64_t* off, const int32_t* adj, int64_t n, std::vector<char>& keep) {
  std::vector<int64_t> comp(n, -1);
  std::vector<int64_t> q;
  int64_t best = -1, best_size = 0, ncomp = 0;
  for (int64_t s = 0; s < n; ++s) {
    if (!keep[s] || comp[s] >= 0) continue;
    int64_t id = ncomp++, size = 0;
    q.clear();
    q.push_back(s);
    comp[s] = id;
    for (size_t h = 0; h < q.size(); ++h) {
      int64_t v = q[h];
      ++size;
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        int64_t u = adj[e];
        if (keep[u] && comp[u] < 0) { comp[u] = id; q.push_back(u); }
      }
    }
    if (size > best_size) { best_size = size; best = id; }
  }
  for (int64_t v = 0; v < n; ++v) keep[v] = (keep[v] && comp[v] == best) ? 1 : 0;
}

Csr induced(const int64_t* off, const int32_t* adj, const int32_t* w, int64_t n,
            const std::vector<char>& keep) {
  std::vector<int64_t> id(n, -1);
  int64_t m = 0;
  for (int64_t v = 0; v < n; ++v) if (keep[v]) id[v] = m++;
  Csr g;
  g.n = m;
  g.off.assign(m + 1, 0);
  for (int64_t v = 0; v < n; ++v) {
    if (!keep[v]) continue;
    int64_t c = 0;
    for (int64_t e = off[v]; e < off[v + 1]; ++e) c += keep[adj[e]] ? 1 : 0;
    g.off[id[v] + 1] = c;
  }
  for (int64_t v = 0; v < m; ++v) g.off[v + 1] += g.off[v];
  g.adj.resize(g.off[m]);
  g.w.resize(g.off[m]);
  parallel_ranges(n, [&](int64_t a, int64_t b, int) {
    for (int64_t v = a; v < b; ++v) {
      if (!keep[v]) continue;
      int64_t p = g.off[id[v]];
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        if (!keep[adj[e]]) continue;
        g.adj[p] = (int32_t)id[adj[e]];
        g.w[p++] = w[e];
      }
    }
  });
  return g;
}

// Result registry: a generated graph lives here until the caller copies it out.
struct Handle {
  Csr g;
};

Handle* wrap(Csr&& g) {
  Handle* h = new Handle;
  h->g = std::move(g);
  return h;
}

}  // namespace

extern "C" {

// All generators return an opaque handle; read sizes with gg_info, copy with
// gg_copy, release with gg_free.
void* gg_rhg(int64_t n, double avg_deg, double gamma, uint64_t seed) {
  return wrap(gen_rhg(n, avg_deg, gamma, seed));
}
void* gg_er(int64_t n, double avg_deg, uint64_t seed, int32_t wlo, int32_t whi) {
  return wrap(gen_er(n, avg_deg, seed, wlo, whi));
}
void* gg_planted(int64_t blocks, int64_t block_n, double avg_deg, int64_t bridges,
                 uint64_t seed, int32_t wlo, int32_t whi) {
  return wrap(gen_planted(blocks, block_n, avg_deg, bridges, seed, wlo, whi));
}
// k-core (k <= 0: no peeling) then optional largest connected component.
void* gg_core_lcc(const int64_t* off, const int32_t* adj, const int32_t* w, int64_t n,
                  int64_t k, int32_t lcc) {
  std::vector<char> keep = k > 0 ? kcore_keep(off, adj, n, k) : std::vector<char>(n, 1);
  if (lcc) largest_component(off, adj, n, keep);
  return wrap(induced(off, adj, w, n, keep));
}
// Replaces every weight with a value uniform in [lo, hi] that depends only on the
// unordered endpoint pair, so both directions of an edge agree.
void gg_pair_weights(const int64_t* off, const int32_t* adj, int32_t* w, int64_t n,
                     uint64_t seed, int32_t lo, int32_t hi) {
  parallel_ranges(n, [&](int64_t a, int64_t b, int) {
    for (int64_t v = a; v < b; ++v)
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        uint64_t x = (uint64_t)std::min<int64_t>(v, adj[e]);
        uint64_t y = (uint64_t)std::max<int64_t>(v, adj[e]);
        double u = rnd01(seed, x, y);
        int32_t t = lo + (int32_t)(u * (double)(hi - lo + 1));
        w[e] = t > hi ? hi : t;
      }
  });
}
double gg_rhg_radius(int64_t n, double avg_deg, double gamma) {
  return rhg_radius_for_degree(n, avg_deg, (gamma - 1.0) / 2.0);
}
void gg_info(void* h, int64_t* n, int64_t* nnz) {
  Handle* x = (Handle*)h;
  *n = x->g.n;
  *nnz = (int64_t)x->g.adj.size();
}
void gg_copy(void* h, int64_t* off, int32_t* adj, int32_t* w) {
  Handle* x = (Handle*)h;
  memcpy(off, x->g.off.data(), sizeof(int64_t) * (x->g.n + 1));
  memcpy(adj, x->g.adj.data(), sizeof(int32_t) * x->g.adj.size());
  memcpy(w, x->g.w.data(), sizeof(int32_t) * x->g.w.size());
}
void gg_free(void* h) { delete (Handle*)h; }
// Uniform doubles from the shared counter-based stream (for Python-side sampling).
void gg_uniform(uint64_t seed, uint64_t stream, int64_t count, double* out) {
  for (int64_t i = 0; i < count; ++i) out[i] = rnd01(seed, stream, (uint64_t)i);
}

}  // extern "C"
