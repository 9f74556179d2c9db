// Host-side finite-element tables: GLL rule, 1D element matrices, lumped mass.
//
// Spectral elements (Sec. 3.2.1): element nodes at the Gauss-Lobatto-Legendre
// points, Lagrange basis through them (Eq. 12), diagonal mass from GLL
// quadrature.  The kinetic part of Eq. 17 is integrated exactly with a
// (p+1)-point Gauss-Legendre rule, so the cell matrix is dense.
#include <cmath>

#include "internal.h"

namespace invdft {
namespace {

// P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double *P, double *dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = (std::fabs(1.0 - x * x) > 0.0) ? n * (p0 - x * p1) / (1.0 - x * x) : 0.0;
}

// GLL nodes: -1, 1 and the roots of P_p' (Newton from Chebyshev-Lobatto
// guesses, using P_p'' from Legendre's equation); weights 2/(p(p+1) P_p^2).
void gll(int p, std::vector<double> *x, std::vector<double> *w) {
  x->assign(p + 1, 0.0);
  w->assign(p + 1, 0.0);
  (*x)[0] = -1.0;
  (*x)[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    double xi = -std::cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, xi, &P, &dP);
      double d2P = (2.0 * xi * dP - p * (p + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    (*x)[i] = xi;
  }
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre(p, (*x)[i], &P, &dP);
    (*w)[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
}

// n-point Gauss-Legendre rule by Newton on P_n.
void gauss(int n, std::vector<double> *x, std::vector<double> *w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double xi = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double P = 0.0, dP = 1.0;
    for (int it = 0; it < 100; ++it) {
      legendre(n, xi, &P, &dP);
      double dx = P / dP;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    legendre(n, xi, &P, &dP);
    (*x)[i] = xi;
    (*w)[i] = 2.0 / ((1.0 - xi * xi) * dP * dP);
  }
}

}  // namespace

void build_reference(int p, Tables *t) {
  const int q = p + 1;
  gll(p, &t->gll_x, &t->gll_w);
  const std::vector<double> &xn = t->gll_x;
  // barycentric weights and the nodal differentiation matrix D_ij = l_j'(x_i)
  std::vector<double> lam(q, 1.0), Dm(q * q, 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      if (j != i) lam[i] /= (xn[i] - xn[j]);
  for (int i = 0; i < q; ++i) {
    double diag = 0.0;
    for (int j = 0; j < q; ++j)
      if (j != i) {
        Dm[i * q + j] = (lam[j] / lam[i]) / (xn[i] - xn[j]);
        diag -= Dm[i * q + j];
      }
    Dm[i * q + i] = diag;
  }
  std::vector<double> xq, wq;
  gauss(q, &xq, &wq);
  // basis values at the Gauss points by barycentric interpolation
  std::vector<double> V(q * q, 0.0), G(q * q, 0.0);   // [point][basis]
  for (int k = 0; k < q; ++k) {
    int hit = -1;
    for (int j = 0; j < q; ++j)
      if (xq[k] == xn[j]) hit = j;
    if (hit >= 0) {
      V[k * q + hit] = 1.0;
    } else {
      double den = 0.0;
      for (int j = 0; j < q; ++j) den += lam[j] / (xq[k] - xn[j]);
      for (int j = 0; j < q; ++j) V[k * q + j] = (lam[j] / (xq[k] - xn[j])) / den;
    }
    // l_j' is a polynomial of degree p-1: interpolate its nodal values
    for (int j = 0; j < q; ++j) {
      double s = 0.0;
      for (int i = 0; i < q; ++i) s += V[k * q + i] * Dm[i * q + j];
      G[k * q + j] = s;
    }
  }
  t->Dm = Dm;
  t->A.assign(q * q, 0.0);
  t->B.assign(q * q, 0.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < q; ++k) {
        a += wq[k] * G[k * q + i] * G[k * q + j];
        b += wq[k] * V[k * q + i] * V[k * q + j];
      }
      t->A[i * q + j] = a;
      t->B[i * q + j] = b;
    }
}

void gauss_lagrange(int p, int ng, std::vector<double> *xg, std::vector<double> *wg,
                    std::vector<double> *phi) {
  const int q = p + 1;
  std::vector<double> xn, wn;
  gll(p, &xn, &wn);
  gauss(ng, xg, wg);
  std::vector<double> lam(q, 1.0);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < q; ++j)
      if (j != i) lam[i] /= (xn[i] - xn[j]);
  phi->assign((size_t)ng * q, 0.0);
  for (int k = 0; k < ng; ++k) {
    // Gauss points are never GLL nodes (interior of [-1, 1], distinct roots)
    double den = 0.0;
    for (int j = 0; j < q; ++j) den += lam[j] / ((*xg)[k] - xn[j]);
    for (int j = 0; j < q; ++j) (*phi)[(size_t)k * q + j] = (lam[j] / ((*xg)[k] - xn[j])) / den;
  }
}

void build_axis(const Tables &ref, const std::vector<double> &breaks, int p, AxisTab *ax) {
  const int q = p + 1;
  const int ncell = (int)breaks.size() - 1;
  const int N = ncell * p + 1;
  ax->breaks = breaks;
  ax->h.assign(ncell, 0.0);
  ax->axis.assign(N, 0.0);
  ax->m1.assign(N, 0.0);
  ax->kdiag1_A.assign(N, 0.0);
  ax->kdiag1_B.assign(N, 0.0);
  ax->uniform = true;
  const double h0 = (breaks[ncell] - breaks[0]) / ncell;
  for (int e = 0; e < ncell; ++e) {
    const double h = breaks[e + 1] - breaks[e], s = 0.5 * h;
    ax->h[e] = h;
    if (std::fabs(h - h0) > 1e-12 * std::fabs(h0)) ax->uniform = false;
    for (int i = 0; i < q; ++i) {
      const int gi = e * p + i;
      ax->axis[gi] = breaks[e] + s * (ref.gll_x[i] + 1.0);
      ax->m1[gi] += s * ref.gll_w[i];
      ax->kdiag1_A[gi] += ref.A[i * q + i] / s;
      ax->kdiag1_B[gi] += ref.B[i * q + i] * s;
    }
  }
  ax->axis[0] = breaks[0];
  ax->axis[N - 1] = breaks[ncell];
}

}  // namespace invdft
