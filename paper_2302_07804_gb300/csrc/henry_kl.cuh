// Karhunen-Loeve basis of the squared-exponential covariance on the Henry box
// (host code, computed once per handle).
//
// Random-field model (configuration with random fields; the paper models
// porosity and permeability as random fields, Sec. 2.2): log K and phi are
// Gaussian fields with covariance sigma^2 exp(-r^2 / (2 l^2)), truncated to
// their n_terms leading KL terms.  The kernel separates in x and y, so the
// 2-D eigenpairs are products of 1-D eigenpairs on [0, Lx] and [0, Ly].  Each
// 1-D problem is discretised by the Nystrom method on an n-point
// Gauss-Legendre rule: the symmetric matrix A = W^1/2 K W^1/2 (W = diag of
// the weights) is diagonalised by the cyclic Jacobi method, u = W^-1/2 v is
// the eigenfunction at the nodes (sum_q w_q u_q^2 = 1), and the Nystrom
// interpolant psi(x) = (1/lam) sum_q w_q k(x, x_q) u_q evaluates it at cell
// centres.  Conventions: the sign of each u makes sum_q w_q (q + 1) u_q > 0;
// the 2-D terms are the n_terms largest products lam_x lam_y in decreasing
// order, with products within a relative 1e-9 ordered by (i + j, i).
#pragma once
#include <algorithm>
#include <cmath>
#include <vector>

namespace hkl {

// Gauss-Legendre nodes and weights on [a, b] (Newton iteration on P_n from
// the Chebyshev-like initial guess; Golub & Welsch give the same rule).
inline void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;  // P_0, P_1
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      // p1 = P_n(z), p0 = P_{n-1}(z)
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    const double wt = 2.0 / ((1.0 - z * z) * dp * dp);
    // node i is the i-th largest; store ascending
    x[n - 1 - i] = z;
    x[i] = -z;
    w[n - 1 - i] = wt;
    w[i] = wt;
  }
  for (int i = 0; i < n; ++i) {
    x[i] = 0.5 * (b - a) * x[i] + 0.5 * (b + a);
    w[i] = 0.5 * (b - a) * w[i];
  }
}

// Cyclic Jacobi eigenvalue algorithm for a symmetric n x n matrix (row-major,
// overwritten).  Returns eigenvalues in lam and eigenvectors as columns of V.
inline void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& lam, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = A[(size_t)i * n + j];
        if (i == j) diag += a * a;
        else off += a * a;
      }
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = A[(size_t)i * n + i];
}

struct Basis1D {
  std::vector<double> lam;  // m leading eigenvalues, decreasing
  std::vector<double> xq, wq;
  std::vector<double> U;    // [m][n]
  int m = 0, n = 0;
  double ell = 0.3;

  void build(double L, int nq, int modes, double corr) {
    n = nq;
    ell = corr;
    gauss_legendre(n, 0.0, L, xq, wq);
    std::vector<double> A((size_t)n * n), ev, V;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double d = xq[i] - xq[j];
        A[(size_t)i * n + j] = std::sqrt(wq[i]) * std::exp(-d * d / (2.0 * ell * ell)) * std::sqrt(wq[j]);
      }
    jacobi_eigen(n, A, ev, V);
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return ev[a] > ev[b]; });
    m = std::min(modes, n);
    lam.assign(m, 0.0);
    U.assign((size_t)m * n, 0.0);
    for (int i = 0; i < m; ++i) {
      lam[i] = ev[idx[i]];
      double sgn = 0.0;
      for (int q = 0; q < n; ++q) {
        const double u = V[(size_t)q * n + idx[i]] / std::sqrt(wq[q]);
        U[(size_t)i * n + q] = u;
        sgn += wq[q] * (q + 1.0) * u;
      }
      if (sgn < 0.0)
        for (int q = 0; q < n; ++q) U[(size_t)i * n + q] = -U[(size_t)i * n + q];
    }
  }
  // psi_i at x
  double eval(int i, double x) const {
    double s = 0.0;
    for (int q = 0; q < n; ++q) {
      const double d = x - xq[q];
      s += wq[q] * std::exp(-d * d / (2.0 * ell * ell)) * U[(size_t)i * n + q];
    }
    return s / lam[i];
  }
};

struct Basis2D {
  Basis1D bx, by;
  std::vector<int> ti, tj;       // term k = psi_x[ti[k]] * psi_y[tj[k]]
  std::vector<double> sqrt_lam;  // sqrt(lam_x lam_y)
  int terms = 0;

  void build(double Lx, double Ly, int n_terms, double corr, int nq = 256, int m1d = 40) {
    bx.build(Lx, nq, m1d, corr);
    by.build(Ly, nq, m1d, corr);
    struct Cand {
      double v;
      int i, j;
    };
    std::vector<Cand> c;
    for (int i = 0; i < bx.m; ++i)
      for (int j = 0; j < by.m; ++j) c.push_back({bx.lam[i] * by.lam[j], i, j});
    std::sort(c.begin(), c.end(), [](const Cand& a, const Cand& b) { return a.v > b.v; });
    const size_t top = std::min(c.size(), (size_t)n_terms + 8);
    std::vector<Cand> out;
    size_t k = 0;
    while (k < top) {
      size_t g = 1;
      while (k + g < top && std::fabs(c[k + g].v - c[k].v) <= 1e-9 * c[k].v) ++g;
      std::vector<Cand> grp(c.begin() + k, c.begin() + k + g);
      std::sort(grp.begin(), grp.end(), [](const Cand& a, const Cand& b) {
        return (a.i + a.j) != (b.i + b.j) ? (a.i + a.j) < (b.i + b.j) : a.i < b.i;
      });
      out.insert(out.end(), grp.begin(), grp.end());
      k += g;
    }
    terms = n_terms;
    ti.resize(terms);
    tj.resize(terms);
    sqrt_lam.resize(terms);
    for (int t = 0; t < terms; ++t) {
      ti[t] = out[t].i;
      tj[t] = out[t].j;
      sqrt_lam[t] = std::sqrt(out[t].v);
    }
  }
};

}  // namespace hkl
