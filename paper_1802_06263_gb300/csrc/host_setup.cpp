// Host set-up arithmetic: mortar projections, KL roots, Gauss-Hermite rules,
// tensor and Smolyak grids. See host_setup.h.
#include "host_setup.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <stdexcept>

namespace sfb {

namespace {

// Antiderivatives on [0, 1] of the Lagrange basis of degree 1 (nodes 0, 1)
// and 2 (nodes 0, 1/2, 1).
double lagrange_antideriv(int deg, int a, double t) {
  if (deg == 1) return a == 0 ? t - 0.5 * t * t : 0.5 * t * t;
  const double t2 = t * t, t3 = t2 * t;
  if (a == 0) return 2.0 * t3 / 3.0 - 1.5 * t2 + t;   // 2t^2 - 3t + 1
  if (a == 1) return 2.0 * t2 - 4.0 * t3 / 3.0;       // 4t - 4t^2
  return 2.0 * t3 / 3.0 - 0.5 * t2;                   // 2t^2 - t
}

double lagrange_val(int deg, int a, double t) {
  if (deg == 1) return a == 0 ? 1.0 - t : t;
  if (a == 0) return 2.0 * (t - 0.5) * (t - 1.0);
  if (a == 1) return 4.0 * t * (1.0 - t);
  return 2.0 * t * (t - 0.5);
}

}  // namespace

void face_projection(const HostIface& itf, double f0, double h, int n_faces,
                     const std::vector<int>& cols, int ld, double* out) {
  const double H = (itf.s1 - itf.s0) / itf.n_el;
  const int nb = itf.deg + 1;
  for (int i = 0; i < n_faces; ++i) {
    const double a = f0 + i * h, b = f0 + (i + 1) * h;
    for (int e = 0; e < itf.n_el; ++e) {
      const double e0 = itf.s0 + e * H, e1 = itf.s0 + (e + 1) * H;
      const double lo = std::max(a, e0), hi = std::min(b, e1);
      if (!(hi > lo)) continue;
      const double ta = (lo - e0) / H, tb = (hi - e0) / H;
      for (int q = 0; q < nb; ++q) {
        const double v = H * (lagrange_antideriv(itf.deg, q, tb) - lagrange_antideriv(itf.deg, q, ta)) / h;
        out[(int64_t)i * ld + cols[e * nb + q]] += v;
      }
    }
  }
}

void mortar_times_p2(const HostIface& itf, double xa, double xb, int q, double* out) {
  // 5-point Gauss-Legendre on each piece between mortar breakpoints: exact
  // for the degree <= 4 products of a mortar function and a P2 shape.
  static const double gx[5] = {-0.9061798459386640, -0.5384693101056831, 0.0,
                               0.5384693101056831, 0.9061798459386640};
  static const double gw[5] = {0.2369268850561891, 0.4786286704993665, 0.5688888888888889,
                               0.4786286704993665, 0.2369268850561891};
  const double H = (itf.s1 - itf.s0) / itf.n_el;
  const int nb = itf.deg + 1;
  for (int k = 0; k < itf.n_dof; ++k) out[k] = 0.0;
  for (int e = 0; e < itf.n_el; ++e) {
    const double e0 = itf.s0 + e * H, e1 = itf.s0 + (e + 1) * H;
    const double lo = std::max(xa, e0), hi = std::min(xb, e1);
    if (!(hi > lo)) continue;
    const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
    for (int g = 0; g < 5; ++g) {
      const double s = mid + half * gx[g];
      const double shape = lagrange_val(2, q, (s - xa) / (xb - xa));
      const double t = (s - e0) / H;
      for (int a = 0; a < nb; ++a) out[e * nb + a] += gw[g] * half * shape * lagrange_val(itf.deg, a, t);
    }
  }
}

// ---- KL ------------------------------------------------------------------
namespace {

// Newton with bisection safeguard for f(theta) on [lo, hi] with a sign change.
template <typename F, typename DF>
double safe_newton(F f, DF df, double lo, double hi) {
  double flo = f(lo), fhi = f(hi);
  if (flo == 0.0) return lo;
  if (fhi == 0.0) return hi;
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    const double fx = f(x);
    if (fx == 0.0) return x;
    if ((fx < 0) == (flo < 0)) { lo = x; flo = fx; } else { hi = x; }
    const double d = df(x);
    double xn = x - fx / d;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 1e-16 * std::fabs(x) || hi - lo <= 2e-16 * std::fabs(x)) return xn;
    x = xn;
  }
  return x;
}

}  // namespace

void kl_1d_host(double L, double eta, int n, std::vector<double>& omega,
                std::vector<double>& lam, std::vector<int>& parity) {
  const double a = 0.5 * L, c = 1.0 / eta, ca = c * a;
  omega.clear(); lam.clear(); parity.clear();
  const double pi = M_PI;
  for (int k = 0; (int)omega.size() < n; ++k) {
    // even modes: c cos(th) - (th/a) sin(th) = 0 on (k pi, k pi + pi/2)
    auto fe = [&](double th) { return ca * std::cos(th) - th * std::sin(th); };
    auto dfe = [&](double th) { return -ca * std::sin(th) - std::sin(th) - th * std::cos(th); };
    double th = safe_newton(fe, dfe, k * pi, k * pi + 0.5 * pi);
    omega.push_back(th / a); parity.push_back(0);
    if ((int)omega.size() == n) break;
    // odd modes: (th/a) cos(th) + c sin(th) = 0 on (k pi + pi/2, (k+1) pi)
    auto fo = [&](double t) { return t * std::cos(t) + ca * std::sin(t); };
    auto dfo = [&](double t) { return std::cos(t) - t * std::sin(t) + ca * std::cos(t); };
    th = safe_newton(fo, dfo, k * pi + 0.5 * pi, (k + 1) * pi);
    omega.push_back(th / a); parity.push_back(1);
  }
  for (double w : omega) lam.push_back(2.0 * c / (w * w + c * c));
}

double kl_1d_eval_host(double x, double L, double w, int parity) {
  const double a = 0.5 * L;
  const double s = std::sin(2.0 * w * a) / (2.0 * w);
  return parity == 0 ? std::cos(w * x) / std::sqrt(a + s) : std::sin(w * x) / std::sqrt(a - s);
}

// ---- Gauss-Hermite ------------------------------------------------------------
void gauss_hermite_host(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0); w.assign(m, 0.0);
  if (m == 1) { w[0] = 1.0; return; }
  // Eigenvalues of the Jacobi matrix (zero diagonal, off-diagonal sqrt(k))
  // by bisection with Sturm counts, then Christoffel weights
  // w_i = 1 / sum_k p_k(x_i)^2 with the orthonormal p_k = He_k / sqrt(k!).
  auto count_below = [&](double t) {
    int cnt = 0;
    double q = -t;  // d_1 = a_1 - t
    if (q < 0) ++cnt;
    for (int k = 1; k < m; ++k) {
      if (q == 0.0) q = 1e-300;
      q = -t - (double)k / q;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  const double bound = 2.0 * std::sqrt((double)m) + 1.0;
  for (int i = 0; i < m; ++i) {
    double lo = -bound, hi = bound;
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(lo)); ++it) {
      const double mid = 0.5 * (lo + hi);
      if (count_below(mid) > i) hi = mid; else lo = mid;
    }
    double t = 0.5 * (lo + hi);
    // polish with Newton on He_m
    for (int it = 0; it < 3; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 1; k < m; ++k) { const double p2 = t * p1 - k * p0; p0 = p1; p1 = p2; }
      const double dp = m * p0;  // He_m' = m He_{m-1}
      if (dp != 0.0) t -= p1 / dp;
    }
    if (std::fabs(t) < 1e-14) t = 0.0;
    x[i] = t;
    double s = 1.0, pkm1 = 1.0, pk = t, fact = 1.0;
    for (int k = 1; k < m; ++k) {
      fact *= k;
      s += pk * pk / fact;
      const double pn = t * pk - k * pkm1;
      pkm1 = pk; pk = pn;
    }
    w[i] = 1.0 / s;
  }
  double tot = 0.0;
  for (double v : w) tot += v;
  for (double& v : w) v /= tot;
}

// ---- grids -----------------------------------------------------------------
void tensor_grid_host(const std::vector<int>& ms, Grid& out) {
  const int n = (int)ms.size();
  out.n_dim = n;
  out.y.clear(); out.w.clear();
  std::vector<std::vector<double>> xs(n), ws(n);
  for (int d = 0; d < n; ++d) gauss_hermite_host(ms[d], xs[d], ws[d]);
  std::vector<int> idx(n, 0);
  while (true) {
    double wt = 1.0;
    for (int d = 0; d < n; ++d) { out.y.push_back(xs[d][idx[d]]); wt *= ws[d][idx[d]]; }
    out.w.push_back(wt);
    int d = n - 1;
    while (d >= 0 && ++idx[d] == ms[d]) { idx[d] = 0; --d; }
    if (d < 0) break;
  }
}

int rule_size_host(int p, const std::vector<int>& rule) {
  if (rule.empty()) return (1 << (p + 1)) - 1;
  return p < (int)rule.size() ? rule[p] : rule.back();
}

namespace {
void enum_multi(int n_dim, int start, int remaining, std::vector<std::pair<int, int>>& cur,
                std::vector<std::vector<std::pair<int, int>>>& out) {
  if (remaining == 0) { out.push_back(cur); return; }
  for (int d = start; d < n_dim; ++d)
    for (int lev = 1; lev <= remaining; ++lev) {
      cur.push_back({d, lev});
      enum_multi(n_dim, d + 1, remaining - lev, cur, out);
      cur.pop_back();
    }
}
}  // namespace

void smolyak_grid_host(int n_dim, int lmax, const std::vector<int>& rule, Grid& out) {
  out.n_dim = n_dim;
  out.y.clear(); out.w.clear();
  const int lmin = std::max(0, lmax - n_dim + 1);
  // sparse point key: sorted (dim, quantised coordinate) of nonzero coordinates.
  // A point's weight adds up terms of both signs whose running sums far exceed
  // the result (level 3 over 64 dimensions: about 2e5 terms at the origin
  // against a coefficient of 39,711), so each sum carries Neumaier's
  // compensation term: the plain sum lost 1.2e-8 of the weights' total of 1.
  std::map<std::vector<int64_t>, std::pair<double, double>> acc;
  std::map<int, std::pair<std::vector<double>, std::vector<double>>> rules;
  auto get_rule = [&](int m) -> const std::pair<std::vector<double>, std::vector<double>>& {
    auto it = rules.find(m);
    if (it == rules.end()) {
      std::vector<double> x, w;
      gauss_hermite_host(m, x, w);
      it = rules.emplace(m, std::make_pair(x, w)).first;
    }
    return it->second;
  };
  for (int q = lmin; q <= lmax; ++q) {
    // coefficient (-1)^(lmax-q) C(n_dim-1, lmax-q)
    const int r = lmax - q;
    double binom = 1.0;
    for (int i = 0; i < r; ++i) binom = binom * (double)(n_dim - 1 - i) / (double)(i + 1);
    if (binom == 0.0) continue;
    const double coef = (r % 2 ? -1.0 : 1.0) * binom;
    std::vector<std::vector<std::pair<int, int>>> mis;
    std::vector<std::pair<int, int>> cur;
    enum_multi(n_dim, 0, q, cur, mis);
    for (const auto& mi : mis) {
      const int k = (int)mi.size();
      std::vector<int> sizes(k);
      for (int a = 0; a < k; ++a) sizes[a] = rule_size_host(mi[a].second, rule);
      std::vector<int> idx(k, 0);
      while (true) {
        std::vector<int64_t> key;
        double wt = coef;
        for (int a = 0; a < k; ++a) {
          const auto& R = get_rule(sizes[a]);
          const double v = R.first[idx[a]];
          wt *= R.second[idx[a]];
          const int64_t qv = qkey(v);
          if (qv != 0) { key.push_back(mi[a].first); key.push_back(qv); }
        }
        std::pair<double, double>& sc = acc[key];
        const double t = sc.first + wt;
        sc.second += std::fabs(sc.first) >= std::fabs(wt) ? (sc.first - t) + wt : (wt - t) + sc.first;
        sc.first = t;
        int a = k - 1;
        while (a >= 0 && ++idx[a] == sizes[a]) { idx[a] = 0; --a; }
        if (a < 0) break;
      }
    }
  }
  // dense points, sorted lexicographically by quantised coordinates
  std::vector<std::pair<std::vector<int64_t>, double>> pts;
  pts.reserve(acc.size());
  for (const auto& kv : acc) {
    std::vector<int64_t> dense(n_dim, 0);
    for (size_t i = 0; i < kv.first.size(); i += 2) dense[kv.first[i]] = kv.first[i + 1];
    pts.push_back({dense, kv.second.first + kv.second.second});
  }
  std::sort(pts.begin(), pts.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  for (const auto& p : pts) {
    for (int d = 0; d < n_dim; ++d) out.y.push_back((double)p.first[d] * 1e-12);
    out.w.push_back(p.second);
  }
  // restore full-precision coordinates from the 1-D rules
  std::map<int64_t, double> exact;
  for (const auto& kv : rules)
    for (double v : kv.second.first) exact[qkey(v)] = v;
  for (double& v : out.y) {
    auto it = exact.find(qkey(v));
    if (it != exact.end()) v = it->second;
  }
}

}  // namespace sfb
