// Host-side FP64 model set-up (see model.h).
#include "model.h"

#include <algorithm>
#include <limits>
#include <cmath>
#include <numeric>

namespace pqmc {

void build_hopping(const Lattice& lat, std::vector<double>& K, std::vector<double>& eps) {
  const int N = lat.n_sites();
  K.assign((size_t)N * N, 0.0);
  eps.assign(N, 0.0);
  auto add = [&](int i, int j, double amp) {
    K[(size_t)i * N + j] -= amp;
    K[(size_t)j * N + i] -= amp;
  };
  auto wrapx = [&](int x) { return ((x % lat.Lx) + lat.Lx) % lat.Lx; };
  auto wrapy = [&](int y) { return ((y % lat.Ly) + lat.Ly) % lat.Ly; };
  if (lat.kind == 0) {
    // unit cell (x, y) holds A = 2c and B = 2c + 1, c = x + Lx y; each A site
    // bonds to the B sites of cells (x, y), (x-1, y), (x, y-1)
    auto cell = [&](int x, int y) { return wrapx(x) + lat.Lx * wrapy(y); };
    for (int y = 0; y < lat.Ly; ++y)
      for (int x = 0; x < lat.Lx; ++x) {
        const int a = 2 * cell(x, y);
        eps[a] = 1.0;
        eps[a + 1] = -1.0;
        add(a, 2 * cell(x, y) + 1, lat.t);
        add(a, 2 * cell(x - 1, y) + 1, lat.t);
        add(a, 2 * cell(x, y - 1) + 1, lat.t);
      }
  } else {
    auto site = [&](int x, int y) { return wrapx(x) + lat.Lx * wrapy(y); };
    for (int y = 0; y < lat.Ly; ++y)
      for (int x = 0; x < lat.Lx; ++x) {
        const int i = site(x, y);
        eps[i] = ((x + y) % 2 == 0) ? 1.0 : -1.0;
        if (lat.t != 0.0) {
          add(i, site(x + 1, y), lat.t);
          add(i, site(x, y + 1), lat.t);
        }
        if (lat.tp != 0.0) {
          add(i, site(x + 1, y + 1), lat.tp);
          add(i, site(x + 1, y - 1), lat.tp);
        }
      }
  }
}

bool sym_eig(int n, const std::vector<double>& Ain, std::vector<double>& w, std::vector<double>& V) {
  std::vector<double> A(Ain);
  std::vector<double> Q((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  auto q = [&](int i, int j) -> double& { return Q[(size_t)i * n + j]; };

  // 1. Householder reduction to tridiagonal form: for column k, reflect
  //    x = A[k+1:, k] onto -sign(x0)|x| e_1 and apply H A H to the trailing
  //    block as a symmetric rank-2 update; accumulate Q <- Q H.
  std::vector<double> v(n), p(n), wv(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double nrm2 = 0.0;
    for (int i = 0; i < m; ++i) nrm2 += a(k + 1 + i, k) * a(k + 1 + i, k);
    if (nrm2 == 0.0) continue;
    double alpha = std::sqrt(nrm2);
    if (a(k + 1, k) > 0) alpha = -alpha;
    for (int i = 0; i < m; ++i) v[i] = a(k + 1 + i, k);
    v[0] -= alpha;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    double pv = 0.0;
    for (int i = 0; i < m; ++i) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += a(k + 1 + i, k + 1 + j) * v[j];
      p[i] = beta * s;
      pv += p[i] * v[i];
    }
    const double kk = 0.5 * beta * pv;
    for (int i = 0; i < m; ++i) wv[i] = p[i] - kk * v[i];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) a(k + 1 + i, k + 1 + j) -= v[i] * wv[j] + wv[i] * v[j];
    a(k + 1, k) = alpha;
    a(k, k + 1) = alpha;
    for (int i = 1; i < m; ++i) {
      a(k + 1 + i, k) = 0.0;
      a(k, k + 1 + i) = 0.0;
    }
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += q(r, k + 1 + j) * v[j];
      s *= beta;
      for (int j = 0; j < m; ++j) q(r, k + 1 + j) -= s * v[j];
    }
  }
  std::vector<double> d(n), e(std::max(n - 1, 0));
  for (int i = 0; i < n; ++i) d[i] = a(i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);

  // 2. Implicit symmetric QR steps with the Wilkinson shift on the unreduced
  //    trailing block; each step chases the bulge down with Givens rotations
  //    J (J_kk = J_k+1,k+1 = c, J_k,k+1 = s, J_k+1,k = -s), T <- J^T T J, and
  //    accumulates Q <- Q J.
  const double eps = std::numeric_limits<double>::epsilon();
  int hi = n - 1;
  long iters = 0;
  const long max_iters = 60L * n + 100;
  while (hi > 0) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi])) ||
        std::fabs(e[hi - 1]) < 1e-300) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && !(std::fabs(e[lo - 1]) <= eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo])) ||
                       std::fabs(e[lo - 1]) < 1e-300))
      --lo;
    if (++iters > max_iters) return false;
    const double delta = 0.5 * (d[hi - 1] - d[hi]);
    const double eh = e[hi - 1];
    const double sgn = delta >= 0 ? 1.0 : -1.0;
    const double mu = d[hi] - eh * eh / (delta + sgn * std::hypot(delta, eh));
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) {
        c = x / r;
        s = -z / r;
      }
      if (k > lo) e[k - 1] = r;
      const double ak = d[k], bk = e[k], dk = d[k + 1];
      d[k] = c * c * ak - 2.0 * c * s * bk + s * s * dk;
      d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * dk;
      e[k] = c * s * ak + (c * c - s * s) * bk - c * s * dk;
      if (k + 1 < hi) {
        z = -s * e[k + 1];      // bulge at (k, k+2)
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      for (int r2 = 0; r2 < n; ++r2) {
        const double qk = q(r2, k), qk1 = q(r2, k + 1);
        q(r2, k) = c * qk - s * qk1;
        q(r2, k + 1) = s * qk + c * qk1;
      }
    }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return d[i] < d[j]; });
  w.resize(n);
  V.assign((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c) {
    w[c] = d[order[c]];
    for (int r = 0; r < n; ++r) V[(size_t)r * n + c] = Q[(size_t)r * n + order[c]];
  }
  return true;
}

void expm_from_eig(int n, const std::vector<double>& w, const std::vector<double>& V, double x,
                   std::vector<double>& out) {
  out.assign((size_t)n * n, 0.0);
  std::vector<double> ew(n);
  for (int k = 0; k < n; ++k) ew[k] = std::exp(x * w[k]);
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) {
      const double vik = V[(size_t)i * n + k] * ew[k];
      if (vik == 0.0) continue;
      for (int j = 0; j < n; ++j) out[(size_t)i * n + j] += vik * V[(size_t)j * n + k];
    }
}

bool trial_orbitals(const Lattice& lat, const std::vector<double>& K, const std::vector<double>& eps,
                    double M_N, double tiebreak, int sigma, int n_sigma, std::vector<double>& P,
                    double& gap) {
  const int N = lat.n_sites();
  std::vector<double> h(K);
  if (lat.kind == 0) {
    const double tb = tiebreak < 0 ? 1e-4 : tiebreak;
    const double m = std::max(M_N, tb);
    for (int i = 0; i < N; ++i) h[(size_t)i * N + i] += sigma * m * eps[i];
  } else {
    // spin-independent on-site modulation w_i = cos(pi x/4) + cos(pi y/2)/2:
    // it has Fourier components at the momentum differences of the
    // degenerate plane-wave shells and so splits them at first order
    const double tb = tiebreak < 0 ? 0.2 : tiebreak;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < N; ++i) {
      const int x = i % lat.Lx, y = i / lat.Lx;
      const double w = std::cos(pi * x / 4.0) + 0.5 * std::cos(pi * y / 2.0);
      h[(size_t)i * N + i] += sigma * M_N * eps[i] + tb * w;
    }
  }
  std::vector<double> w, V;
  if (!sym_eig(N, h, w, V)) return false;
  P.assign((size_t)N * n_sigma, 0.0);
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < n_sigma; ++k) P[(size_t)i * n_sigma + k] = V[(size_t)i * N + k];
  gap = n_sigma < N ? w[n_sigma] - w[n_sigma - 1] : INFINITY;
  return true;
}

double hs_coupling(double x) { return std::acosh(std::exp(0.5 * x)); }

}  // namespace pqmc
