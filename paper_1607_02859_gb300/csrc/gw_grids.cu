// Optimised imaginary-time and imaginary-frequency grids (Sec. II.A.2).
//
// The paper takes the grids from the minimisation of the discretisation error
// of the direct MP2 energy in imaginary time and in imaginary frequency.  For
// one transition energy x that energy needs 1/x, which both domains write as
// the integral of a squared propagator:
//   time:       1/x = int dtau exp(-x|tau|)^2            ~ sum_j alpha_j exp(-2 x tau_j)
//   frequency:  1/x = int dw/(2 pi) (2x/(x^2 + w^2))^2    ~ sum_k sigma_k (2x/(x^2 + omega_k^2))^2
// Each grid minimises the largest relative error |1 - x sum(...)| over
// x in [x_min, x_max] (a Chebyshev approximation).  It is computed by the
// Remez exchange: the error of the best n-term sum alternates in sign with
// equal magnitude at 2n+1 points; Newton's method solves for the 2n
// parameters (log-weights, log-nodes) and that magnitude on a reference set of
// 2n+1 points, and the reference then moves to the extrema of the new error.
// The n-term start comes from the (n-1)-term solution, its log-nodes and
// log-weights resampled over the term index, starting from a scan at n = 1.
// Host only, FP64; y = x / x_min in [1, R], R = x_max / x_min.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gw_common.cuh"

namespace {

using Vec = std::vector<double>;

// phi_j(y) = y * squared propagator of node v_j = exp(s_j), and d phi_j / d s_j
inline void mp2_basis(bool time, double y, double s, double* phi, double* dphi) {
  const double v = std::exp(s);
  if (time) {
    const double e = std::exp(-2.0 * y * v);
    *phi = y * e;
    *dphi = -2.0 * y * y * v * e;
  } else {
    const double d = y * y + v * v;
    *phi = 4.0 * y * y * y / (d * d);
    *dphi = -16.0 * y * y * y * v * v / (d * d * d);
  }
}

// 1 - y sum_j w_j phi_j(y); p = (log w_0..log w_{n-1}, s_0..s_{n-1})
double mp2_err(bool time, double y, const Vec& p, int n) {
  double acc = 0.0;
  for (int j = 0; j < n; ++j) {
    double phi, dphi;
    mp2_basis(time, y, p[n + j], &phi, &dphi);
    acc += std::exp(p[j]) * phi;
  }
  return 1.0 - acc;
}

// Dense solve with partial pivoting; a is m x m row-major (destroyed), b is overwritten by x.
bool dense_solve(Vec& a, Vec& b, int m) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(a[r * m + c]) > std::fabs(a[piv * m + c])) piv = r;
    if (a[piv * m + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) std::swap(a[c * m + k], a[piv * m + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = a[r * m + c] / a[c * m + c];
      if (f == 0.0) continue;
      for (int k = c; k < m; ++k) a[r * m + k] -= f * a[c * m + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double acc = b[r];
    for (int k = r + 1; k < m; ++k) acc -= a[r * m + k] * b[k];
    b[r] = acc / a[r * m + r];
  }
  return true;
}

// Solve err(ref_i) = (-1)^i E for (p, E) by damped Newton; false on failure.
bool newton_on_reference(bool time, Vec& p, const Vec& ref, double& e0, int n) {
  const int m = 2 * n + 1;
  Vec q(p);
  q.push_back(e0);
  Vec jac(size_t(m) * m), f(m);
  for (int it = 0; it < 30; ++it) {
    double fmax = 0.0;
    for (int i = 0; i < m; ++i) {
      const double sg = (i & 1) ? -1.0 : 1.0;
      double acc = 0.0;
      for (int j = 0; j < n; ++j) {
        double phi, dphi;
        mp2_basis(time, ref[i], q[n + j], &phi, &dphi);
        const double w = std::exp(q[j]);
        acc += w * phi;
        jac[size_t(i) * m + j] = -w * phi;
        jac[size_t(i) * m + n + j] = -w * dphi;
      }
      jac[size_t(i) * m + 2 * n] = -sg;
      f[i] = -(1.0 - acc - sg * q[2 * n]);
      fmax = std::max(fmax, std::fabs(f[i]));
    }
    if (!dense_solve(jac, f, m)) return false;
    double dmax = 0.0;
    for (int k = 0; k < 2 * n; ++k) dmax = std::max(dmax, std::fabs(f[k]));
    const double step = std::min(1.0, 0.3 / std::max(dmax, 1e-300));
    for (int k = 0; k < m; ++k) q[k] += step * f[k];
    if (step == 1.0 && fmax < 1e-14) break;
  }
  for (double v : q)
    if (!std::isfinite(v)) return false;
  p.assign(q.begin(), q.begin() + 2 * n);
  e0 = q[2 * n];
  return true;
}

Vec geomspace(double a, double b, int k) {
  Vec y(k);
  const double la = std::log(a), lb = std::log(b);
  for (int i = 0; i < k; ++i) y[i] = std::exp(la + (lb - la) * double(i) / double(k - 1));
  y[0] = a;
  y[k - 1] = b;
  return y;
}

// New reference: the largest |err| in each run of equal sign (2n+1 runs expected),
// interior ones refined on a local 41-point log grid.  false if the count is wrong.
bool extrema(bool time, const Vec& p, int n, const Vec& ref, double r, Vec& out) {
  Vec y = geomspace(1.0, r, 4000);
  y.insert(y.end(), ref.begin(), ref.end());
  std::sort(y.begin(), y.end());
  y.erase(std::unique(y.begin(), y.end()), y.end());
  const int ny = int(y.size());
  Vec e(ny);
  for (int i = 0; i < ny; ++i) e[i] = mp2_err(time, y[i], p, n);
  auto sgn = [](double v) { return (v > 0.0) - (v < 0.0); };
  std::vector<int> pos;
  for (int i = 0; i < ny;) {
    int j = i;
    while (j + 1 < ny && sgn(e[j + 1]) == sgn(e[i])) ++j;
    int best = i;
    for (int k = i; k <= j; ++k)
      if (std::fabs(e[k]) > std::fabs(e[best])) best = k;
    pos.push_back(best);
    i = j + 1;
  }
  if (int(pos.size()) != 2 * n + 1) return false;
  out.resize(pos.size());
  for (size_t m = 0; m < pos.size(); ++m) out[m] = y[pos[m]];
  for (size_t m = 1; m + 1 < pos.size(); ++m) {
    const int k = pos[m];
    const Vec yy = geomspace(y[k - 1], y[k + 1], 41);
    int best = 0;
    double bv = -1.0;
    for (int i = 0; i < 41; ++i) {
      const double v = std::fabs(mp2_err(time, yy[i], p, n));
      if (v > bv) {
        bv = v;
        best = i;
      }
    }
    out[m] = yy[best];
  }
  return true;
}

void remez(bool time, Vec& p, Vec& ref, int n, double r) {
  double e0 = 0.0;
  for (double y : ref) e0 += std::fabs(mp2_err(time, y, p, n));
  e0 /= double(ref.size());
  for (int it = 0; it < 40; ++it) {
    if (!newton_on_reference(time, p, ref, e0, n)) break;
    Vec nref;
    if (!extrema(time, p, n, ref, r, nref)) break;
    ref = nref;
    double amax = 0.0, amin = 1e300;
    for (double y : ref) {
      const double a = std::fabs(mp2_err(time, y, p, n));
      amax = std::max(amax, a);
      amin = std::min(amin, a);
    }
    if (amax - amin < 1e-4 * amax) break;
  }
}

// Linear interpolation of v (on an even grid of [0,1]) at m even points of [0,1].
Vec resample(const Vec& v, int m) {
  Vec out(m);
  const int k = int(v.size());
  for (int i = 0; i < m; ++i) {
    const double u = m > 1 ? double(i) / double(m - 1) : 0.0;
    const double t = u * double(k - 1);
    int lo = std::min(int(std::floor(t)), k - 2);
    if (k == 1) {
      out[i] = v[0];
      continue;
    }
    lo = std::max(lo, 0);
    const double f = t - double(lo);
    out[i] = v[lo] + f * (v[lo + 1] - v[lo]);
  }
  return out;
}

// Best n-term approximation of 1/y on [1, r]; nodes ascending, weights, largest relative error.
double mp2_minimax(bool time, int n, double r, Vec& nodes, Vec& weights) {
  const Vec y = geomspace(1.0, r, 2000);
  const double s_lo = time ? std::log(1e-3 / r) : std::log(0.1);
  const double s_hi = time ? std::log(10.0) : std::log(10.0 * r);
  double best_err = 1e300;
  Vec p(2);
  for (int k = 0; k < 400; ++k) {
    const double s = s_lo + (s_hi - s_lo) * double(k) / 399.0;
    double pmax = -1e300, pmin = 1e300;
    Vec phis(y.size());
    for (size_t i = 0; i < y.size(); ++i) {
      double phi, dphi;
      mp2_basis(time, y[i], s, &phi, &dphi);
      phis[i] = phi;
      pmax = std::max(pmax, phi);
      pmin = std::min(pmin, phi);
    }
    const double a = 2.0 / (pmax + pmin);          // the best single weight for this node
    double err = 0.0;
    for (double phi : phis) err = std::max(err, std::fabs(1.0 - a * phi));
    if (err < best_err) {
      best_err = err;
      p[0] = std::log(a);
      p[1] = s;
    }
  }
  Vec ref = {1.0, std::sqrt(r), r};
  remez(time, p, ref, 1, r);
  for (int m = 2; m <= n; ++m) {
    Vec lw(m), s(m);
    if (m == 2) {
      s[0] = p[1] - 1.0;
      s[1] = p[1] + 1.0;
      for (int j = 0; j < 2; ++j) lw[j] = p[0] - p[1] - std::log(2.0) + s[j];
    } else {
      Vec old_s(p.begin() + (m - 1), p.end()), ratio(m - 1);
      for (int j = 0; j < m - 1; ++j) ratio[j] = p[j] - old_s[j];
      s = resample(old_s, m);
      const Vec rr = resample(ratio, m);
      for (int j = 0; j < m; ++j) lw[j] = rr[j] + std::log(double(m - 1) / double(m)) + s[j];
    }
    p.assign(lw.begin(), lw.end());
    p.insert(p.end(), s.begin(), s.end());
    Vec lref(ref.size());
    for (size_t i = 0; i < ref.size(); ++i) lref[i] = std::log(ref[i]);
    const Vec nl = resample(lref, 2 * m + 1);
    ref.resize(nl.size());
    for (size_t i = 0; i < nl.size(); ++i) ref[i] = std::exp(nl[i]);
    remez(time, p, ref, m, r);
  }
  std::vector<int> order(n);
  for (int j = 0; j < n; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return p[n + a] < p[n + b]; });
  nodes.resize(n);
  weights.resize(n);
  for (int j = 0; j < n; ++j) {
    nodes[j] = std::exp(p[n + order[j]]);
    weights[j] = std::exp(p[order[j]]);
  }
  double err = 0.0;
  for (double yy : geomspace(1.0, r, 20000)) err = std::max(err, std::fabs(mp2_err(time, yy, p, n)));
  return err;
}

}  // namespace

extern "C" gw_status gw_mp2_grids(int n, double x_min, double x_max, double* tau_h, double* omega_h,
                                  double* alpha_h, double* sigma_h, double* err_h) {
  using gw::fail;
  if (n < 1 || n > 40) return fail(nullptr, GW_ERR_SHAPE, "need 1 <= n <= 40 grid points");
  if (!(x_min > 0.0) || !(x_max > x_min) || !(x_max / x_min <= 1e7))
    return fail(nullptr, GW_ERR_ARG, "need 0 < x_min < x_max with x_max / x_min <= 1e7");
  if (!tau_h || !omega_h) return fail(nullptr, GW_ERR_ARG, "NULL grid pointer");
  const double r = x_max / x_min;
  Vec t, a, w, sg;
  const double et = mp2_minimax(true, n, r, t, a);
  const double ew = mp2_minimax(false, n, r, w, sg);
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(t[j]) || !std::isfinite(w[j]) || !(t[j] > 0.0) || !(w[j] > 0.0))
      return fail(nullptr, GW_ERR_NUMERIC, "minimax grid iteration did not give finite positive nodes");
    tau_h[j] = t[j] / x_min;
    omega_h[j] = w[j] * x_min;
    if (alpha_h) alpha_h[j] = a[j] / x_min;
    if (sigma_h) sigma_h[j] = sg[j] / x_min;
  }
  if (err_h) {
    err_h[0] = et;
    err_h[1] = ew;
  }
  return GW_OK;
}
