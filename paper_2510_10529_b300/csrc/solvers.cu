// Host orchestration of the solvers (kernels run on the caller's stream):
//   * Chebyshev filter (plain scaled recurrence; defect-corrected form for the
//     mixed path) and Chebyshev-filtered subspace iteration with FP64
//     Rayleigh-Ritz (Sec. 3.2.2, Eq. 23-24);
//   * batched projected preconditioned MINRES for all occupied adjoint
//     systems at once (Sec. 3.2.2), with FP64 iterative refinement;
//   * loss + gradient and the L-BFGS iteration (Eq. 1, 11, 21, 22).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "internal.h"
#include "solvers.h"
#include "batch.h"

namespace invdft {

namespace {

// Offsets (in doubles) inside the per-handle scalar area c->scal.

inline void set_tc(HxArgs<double> &, bool) {}
inline void set_tc(HxArgs<float> &a, bool on) { a.tc = on; }


double wall_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

invdft_status fetch(Ctx *c, const void *dev, size_t bytes, void *host, cudaStream_t s) {
  if (bytes > 16 * kMaxCols * sizeof(double)) {
    INV_CUDA(c, cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
    INV_CUDA(c, cudaStreamSynchronize(s));
    return INVDFT_OK;
  }
  INV_CUDA(c, cudaMemcpyAsync(c->hbuf, dev, bytes, cudaMemcpyDeviceToHost, s));
  INV_CUDA(c, cudaStreamSynchronize(s));
  std::memcpy(host, c->hbuf, bytes);
  return INVDFT_OK;
}

// Several small device reads with one synchronisation: the pieces are staged
// one after another in the pinned buffer (16 kMaxCols doubles in all).
struct Piece {
  const void *dev;
  size_t bytes;
  void *host;
};
invdft_status fetch_many(Ctx *c, std::initializer_list<Piece> pieces, cudaStream_t s) {
  size_t off = 0;
  for (const Piece &p : pieces) {
    if (off + p.bytes > 16 * kMaxCols * sizeof(double)) {
      c->err = "fetch_many: pieces exceed the staging buffer";
      return INVDFT_EINVAL;
    }
    INV_CUDA(c, cudaMemcpyAsync((char *)c->hbuf + off, p.dev, p.bytes, cudaMemcpyDeviceToHost, s));
    off += (p.bytes + 7) & ~(size_t)7;
  }
  INV_CUDA(c, cudaStreamSynchronize(s));
  off = 0;
  for (const Piece &p : pieces) {
    std::memcpy(p.host, (const char *)c->hbuf + off, p.bytes);
    off += (p.bytes + 7) & ~(size_t)7;
  }
  return INVDFT_OK;
}

// A kernel whose bounded wait gave up leaves its status word set; the solvers
// read the words back with their convergence data.
invdft_status check_waits(Ctx *c, const int *w) {
  static const char *const what[kStWaitCount] = {"H~X (tensor cores)", "H~X (sweep form)",
                                                 "deflation Gram", "deflation update"};
  for (int i = 0; i < kStWaitCount; ++i)
    if (w[i]) {
      c->err = std::string("a bounded device wait gave up in ") + what[i];
      return INVDFT_ETIMEOUT;
    }
  return INVDFT_OK;
}

invdft_status push(Ctx *c, void *dev, const void *host, size_t bytes, cudaStream_t s) {
  // synchronous w.r.t. the host buffer: the stream is synchronised before reuse
  INV_CUDA(c, cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s));
  INV_CUDA(c, cudaStreamSynchronize(s));
  return INVDFT_OK;
}

#define TRY(x)                             \
  do {                                     \
    invdft_status _st = (x);               \
    if (_st != INVDFT_OK) return _st;      \
  } while (0)
#define CU(x, what)                                             \
  do {                                                          \
    if (!cuda_ok(c, (x), what)) return INVDFT_ECUDA;            \
  } while (0)

// Largest eigenvalue of a symmetric tridiagonal matrix by Sturm bisection.
double tridiag_max_eig(const std::vector<double> &d, const std::vector<double> &e) {
  const int k = (int)d.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  auto count_below = [&](double x) {       // number of eigenvalues < x
    int cnt = 0;
    double q = d[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < k; ++i) {
      const double qq = (q == 0.0) ? 1e-300 : q;
      q = d[i] - x - e[i - 1] * e[i - 1] / qq;
      if (q < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-12 * std::max(1.0, std::fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= k) hi = mid; else lo = mid;
  }
  return hi;
}

// Upper bound of the spectrum of H~: k-step Lanczos, max Ritz value + |f|.
// With two or more states the chain runs on a two-column block, i.e. on
// H~ (+) H~, whose spectrum is that of H~: the block's H~X takes the
// owner-computes sweep form (deterministic, no scatter), which one FP64
// column cannot (its rows are narrower than a bulk copy's 16-byte unit).
invdft_status upper_bound(Ctx *c, cudaStream_t s, double *out) {
  const int nc = c->nv >= 2 ? 2 : 1;
  const long long L = c->L * nc;
  double *v0 = (double *)c->C0, *v = (double *)c->C1, *f = (double *)c->C2, *sc = c->scal + kScMisc;
  CU(launch_fill_random(v, L, c->o.seed ^ 0xA5A5A5A5ULL, s), "fill_random");
  CU(launch_dot(v, v, L, sc, c->partial, s), "dot");
  double nrm;
  TRY(fetch(c, sc, sizeof(double), &nrm, s));
  CU(launch_axpby(0.0, v, 1.0 / std::sqrt(nrm), v, L, s), "axpby");
  CU(cudaMemsetAsync(v0, 0, L * sizeof(double), s), "memset");
  const int k = 12;
  std::vector<double> d, e;
  double beta = 0.0;
  for (int j = 0; j < k; ++j) {
    HxArgs<double> a;
    a.X = v;
    a.Z = f;
    a.ncol = nc;
    a.W = v0;
    a.beta = -beta;                  // f = H v - beta v0
    CU(hx_op(c, a, s), "hx(lanczos)");
    CU(launch_dot(f, v, L, sc, c->partial, s), "dot");
    double alpha;
    TRY(fetch(c, sc, sizeof(double), &alpha, s));
    CU(launch_axpby(-alpha, v, 1.0, f, L, s), "axpby");
    CU(launch_dot(f, f, L, sc, c->partial, s), "dot");
    double ff;
    TRY(fetch(c, sc, sizeof(double), &ff, s));
    d.push_back(alpha);
    beta = std::sqrt(std::max(ff, 0.0));
    if (j < k - 1) {
      e.push_back(beta);
      std::swap(v0, v);                         // v0 <- v
      CU(launch_lincomb(1.0 / beta, f, 0.0, f, v, L, s), "lincomb");   // v <- f / beta
    }
  }
  e.resize(d.size() - 1);
  *out = tridiag_max_eig(d, e) + beta;
  return INVDFT_OK;
}

// Rayleigh-Ritz on (Y, HY): X = Y C, E = (HY C) - X diag(theta) (kept in Y,
// FP64) and E32; theta in c->eps.  Residual norms^2 of the Ritz pairs in
// c->scal[64 .. 64+nv).
invdft_status rayleigh_ritz(Ctx *c, cudaStream_t s) {
  const int n = c->nv;
  const long long L = c->L;
  double *S = c->small, *Hs = c->small + kMaxGram * kMaxGram, *Cm = c->small + 2 * kMaxGram * kMaxGram;
  double *work = c->small + 3 * kMaxGram * kMaxGram;
  CU(launch_gram_rr(c->Y, c->HY, n, L, S, Hs, c->partial, s), "gram(S, H)");
  CU(launch_rr_small(S, Hs, n, c->eps, Cm, c->status, work, s), "rr_small");
  int st = 0;
  TRY(fetch(c, c->status, sizeof(int), &st, s));
  if (st != 0) {
    c->err = "Rayleigh-Ritz: the filtered block is numerically rank deficient (Cholesky failed)";
    return INVDFT_ENOTSPD;
  }
  CU(launch_rotate(c->Y, n, Cm, n, L, c->X, s), "rotate(X)");
  CU(launch_rotate(c->HY, n, Cm, n, L, c->Y, s), "rotate(HX)");
  CU(launch_residual_block(c->Y, c->X, c->eps, n, L, c->Y, c->E32, s), "residual");
  CU(launch_coldot(c->Y, c->Y, n, L, c->scal + kScRes, c->partial, s), "coldot(res)");
  return INVDFT_OK;
}

invdft_status apply_h_f64(Ctx *c, const double *X, double *Z, int n, cudaStream_t s) {
  HxArgs<double> a;
  a.X = X;
  a.Z = Z;
  a.ncol = n;
  CU(hx_op(c, a, s), "hx");
  return INVDFT_OK;
}

// Adaptive tolerances of Sec. 4.2.4: t_eig = e_L2^2 / c_eig, t_ad = e_L2^2 / c_ad
// with e_L2 from the last loss evaluation; floors keep them reachable in FP64.
// Before any loss is known the solves use 1e-3 and 1e-6.
double eig_tolerance(const Ctx *c) {
  if (c->o.eig_tol > 0) return c->o.eig_tol;
  if (c->err_l2 <= 0) return 1e-3;
  return std::max(c->err_l2 * c->err_l2 / c->o.c_eig, 1e-10);
}
double adj_tolerance(const Ctx *c) {
  if (c->o.adj_tol > 0) return c->o.adj_tol;
  if (c->err_l2 <= 0) return 1e-6;
  return std::min(0.1, std::max(c->err_l2 * c->err_l2 / c->o.c_ad, 1e-10));
}

// Convergence weight of a state in the forward solve: with smearing, a state
// of occupation f changes the density in proportion to f, so its residual is
// weighted by min(1, f / 1e-4); states below f = 1e-8 are ignored.  (The
// highest Ritz vectors of the block converge slowest and, near a dense Fermi
// level, still carry small occupations.)
double conv_weight(const Ctx *c, double f) {
  if (c->o.kT <= 0) return f > 0.0 ? 1.0 : 0.0;
  if (!(f > 1e-8)) return 0.0;
  return std::min(1.0, f / 1e-4);
}
bool state_active(const Ctx *c, double f) { return c->o.kT > 0 ? f > 1e-8 : f > 0.0; }

}  // namespace

invdft_status run_filter(Ctx *c, const void *X, void *Y, int ncol, int m, double a, double b,
                         double a0, invdft_precision prec, const double *theta, const float *E,
                         cudaStream_t s) {
  const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
  const double sigma1 = e / (a0 - cc);
  void *bufs[3] = {c->C0, c->C1, c->C2};
  auto free_buf = [&](const void *p1, const void *p2) -> void * {
    for (void *q : bufs)
      if (q != p1 && q != p2) return q;
    return nullptr;
  };
  if (theta == nullptr) {
    const void *prev = nullptr, *cur = X;
    double sigma = sigma1;
    for (int k = 1; k <= m; ++k) {
      const double sn = (k == 1) ? sigma1 : 1.0 / (2.0 / sigma1 - sigma);
      void *Z = (k == m) ? Y : free_buf(prev, cur);
      const double alpha = (k == 1) ? sigma1 / e : 2.0 * sn / e;
      const double beta = (k == 1) ? 0.0 : -sigma * sn;
      cudaError_t err;
      if (prec == INVDFT_FP64) {
        HxArgs<double> h;
        h.X = (const double *)cur;
        h.Z = (double *)Z;
        h.ncol = ncol;
        h.alpha = alpha;
        h.shift = cc;
        h.W = (const double *)prev;
        h.beta = beta;
        err = hx_op(c, h, s);
      } else {
        HxArgs<float> h;
        h.tc = c->o.prec == INVDFT_MIXED_TF32;
        h.X = (const float *)cur;
        h.Z = (float *)Z;
        h.ncol = ncol;
        h.alpha = alpha;
        h.shift = cc;
        h.W = (const float *)prev;
        h.beta = beta;
        err = hx_op(c, h, s);
      }
      CU(err, "hx(filter)");
      prev = cur;
      cur = Z;
      if (k > 1) sigma = sn;
    }
    return INVDFT_OK;
  }
  // defect-corrected filter: Y = X diag(p_m(theta)) + D_m, D in FP32
  const int nk = m + 1;
  if ((size_t)nk * ncol > 128 * (size_t)kMaxCols) {
    c->err = "chebyshev filter: degree too high for the coefficient table";
    return INVDFT_EINVAL;
  }
  std::vector<double> pk((size_t)nk * ncol);
  std::vector<double> sig(nk + 1, 0.0);
  sig[1] = sigma1;
  for (int k = 1; k < m; ++k) sig[k + 1] = 1.0 / (2.0 / sigma1 - sig[k]);
  for (int j = 0; j < ncol; ++j) {
    double pm1 = 1.0, p = (sigma1 / e) * (theta[j] - cc);
    pk[j] = 1.0;
    if (m >= 1) pk[(size_t)ncol + j] = p;
    for (int k = 1; k < m; ++k) {
      const double pn = (2.0 * sig[k + 1] / e) * (theta[j] - cc) * p - sig[k] * sig[k + 1] * pm1;
      pm1 = p;
      p = pn;
      pk[(size_t)(k + 1) * ncol + j] = p;
    }
  }
  double *dpk = c->scal + kScPk;
  TRY(push(c, dpk, pk.data(), pk.size() * sizeof(double), s));
  const long long L = c->L;
  float *D1 = (float *)c->C0;
  CU(launch_scale_f32(E, nullptr, sigma1 / e, ncol, L, D1, s), "scale(D1)");
  const void *prev = nullptr, *cur = D1;
  // inside a batch step the passes of the batch's degree are batched; a pass
  // of another degree (a repeated pass) runs on its own
  const bool batched = c->batch && m >= 2 && m <= kMaxBatchDeg && batch_degree(c) == m;
  if (batched) {
    // batched step: phases 2..m of every waiting problem in one launch;
    // D_2, D_3 accumulate into zeroed buffers, later outputs are zeroed by
    // the owners of their nodes
    std::vector<double> al(m + 1, 0.0), be(m + 1, 0.0);
    for (int k = 2; k <= m; ++k) {
      al[k] = 2.0 * sig[k] / e;
      be[k] = k >= 3 ? -sig[k - 1] * sig[k] : 0.0;
    }
    CU(cudaMemsetAsync(bufs[1], 0, (size_t)L * ncol * sizeof(float), s), "memset");
    CU(cudaMemsetAsync(bufs[2], 0, (size_t)L * ncol * sizeof(float), s), "memset");
    TRY(batch_filter_submit(c, m, al.data(), be.data(), cc, s));
    cur = bufs[(m - 1) % 3];
  }
  for (int k = 2; k <= m && !batched; ++k) {
    const double sn = sig[k];
    void *Z = free_buf(prev, cur);
    HxArgs<float> h;
    h.tc = c->o.prec == INVDFT_MIXED_TF32;
    h.X = (const float *)cur;
    h.Z = (float *)Z;
    h.ncol = ncol;
    h.alpha = 2.0 * sn / e;
    h.shift = cc;
    h.W = (const float *)prev;
    h.beta = prev ? -sig[k - 1] * sn : 0.0;
    h.E = E;
    h.escale = dpk + (size_t)(k - 1) * ncol;
    CU(hx_op(c, h, s), "hx(defect filter)");
    prev = cur;
    cur = Z;
  }
  CU(launch_cheb_combine((const double *)X, dpk + (size_t)m * ncol, (const float *)cur, ncol, L,
                         (double *)Y, s),
     "cheb_combine");
  return INVDFT_OK;
}

// ---------------------------------------------------------------- forward
invdft_status forward_solve(Ctx *c, invdft_stats *stats, cudaStream_t s) {
  const double t0 = wall_ms();
  const int n = c->nv;
  const long long L = c->L;
  const size_t blk = (size_t)L * n;
  int hx_calls = 0;
  if (!c->have_orbitals) {
    CU(launch_fill_random(c->Y, (long long)blk, c->o.seed, s), "fill_random");
    TRY(apply_h_f64(c, c->Y, c->HY, n, s));
    ++hx_calls;
    TRY(rayleigh_ritz(c, s));
    c->have_orbitals = true;
  } else {
    CU(cudaMemcpyAsync(c->Y, c->X, blk * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    TRY(apply_h_f64(c, c->Y, c->HY, n, s));
    ++hx_calls;
    TRY(rayleigh_ritz(c, s));
  }
  if (!c->have_upper) {
    // Weyl: the potential enters H~ as diag(v), so a change of v moves the
    // top of the spectrum by at most max |dv|.  Up to kUbReuse solves reuse
    // the last Lanczos bound plus that shift; then the bound is taken again.
    constexpr int kUbReuse = 8;
    bool reused = false;
    if (c->have_ub_base && c->ub_reuse < kUbReuse) {
      double *dv = (double *)c->C2;     // free before the filter runs
      CU(launch_lincomb(1.0, c->v, -1.0, c->v_ub, dv, L, s), "dv");
      CU(launch_absmax(dv, L, c->scal + kScMisc, c->partial, s), "absmax(dv)");
      double shift = 0.0;
      TRY(fetch(c, c->scal + kScMisc, sizeof(double), &shift, s));
      if (std::isfinite(shift)) {
        c->upper_bound = c->ub_base + shift;
        ++c->ub_reuse;
        reused = true;
      }
    }
    if (!reused) {
      TRY(upper_bound(c, s, &c->upper_bound));
      hx_calls += 12;
      CU(cudaMemcpyAsync(c->v_ub, c->v, L * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
      c->ub_base = c->upper_bound;
      c->have_ub_base = true;
      c->ub_reuse = 0;
    }
    c->have_upper = true;
  }
  const double tol = eig_tolerance(c);
  c->eig_tol_used = tol;
  std::vector<double> theta(n), occ(n), res2(n);
  int pass = 0;
  double maxres = 0.0;
  invdft_status status = INVDFT_OK;
  for (;;) {
    CU(launch_occupations(c->eps, n, c->o.n_electrons, c->o.kT, c->occ, c->dfde, c->scal + kScMu,
                          c->status, s), "occupations");
    int occ_status = 0, waits[kStWaitCount];
    TRY(fetch_many(c, {{c->eps, n * sizeof(double), theta.data()},
                       {c->occ, n * sizeof(double), occ.data()},
                       {c->scal + kScRes, n * sizeof(double), res2.data()},
                       {c->status + 1, sizeof(int), &occ_status},
                       {c->status + kStWaitHxTc, sizeof(waits), waits}}, s));
    TRY(check_waits(c, waits));
    if (occ_status) {
      c->err = "occupations: kT = 0 needs an even electron count and nstates > N_e/2";
      return INVDFT_EINVAL;
    }
    maxres = 0.0;
    for (int i = 0; i < n; ++i)
      maxres = std::max(maxres, conv_weight(c, occ[i]) * std::sqrt(std::max(res2[i], 0.0)));
    if (maxres <= tol && pass >= 1) break;
    if (pass >= c->o.max_cheb_passes) {
      status = INVDFT_ENOCONV;
      c->err = "forward solve: Chebyshev pass cap reached";
      break;
    }
    const double a = theta[n - 1], a0 = theta[0];
    double b = c->upper_bound;
    if (!(b > a)) b = a + std::max(1.0, std::fabs(a));
    // a pass whose filtered block is numerically rank deficient (the filter
    // damps the top of a very wide wanted interval below FP64 resolution) is
    // repeated from the same Ritz vectors with half the degree; Rayleigh-Ritz
    // fails before it overwrites them
    // the first two passes of a solve use the configured degree m, the third
    // 2m and later ones 4m (at most kMaxFilterDeg): near the cut the filter's
    // gain grows with the square of the degree, so one pass of 2m does the
    // work of about four of m at twice the filter cost and one Rayleigh-Ritz
    // instead of four (the states that still need passes after two are those
    // close to the top of the block; Rayleigh-Ritz in FP64 costs about as much
    // as a degree-60 FP32 filter here)
    const int m1 = c->o.cheb_degree;
    const int m0 = pass < 2 ? m1 : std::max(m1, std::min((pass == 2 ? 2 : 4) * m1, kMaxFilterDeg));
    for (int m = m0;; m = std::max(1, m / 2)) {
      if (c->o.prec == INVDFT_FP64) {
        TRY(run_filter(c, c->X, c->Y, n, m, a, b, a0, INVDFT_FP64, nullptr, nullptr, s));
      } else {
        TRY(run_filter(c, c->X, c->Y, n, m, a, b, a0, INVDFT_MIXED, theta.data(), c->E32, s));
      }
      hx_calls += m;
      TRY(apply_h_f64(c, c->Y, c->HY, n, s));
      ++hx_calls;
      const invdft_status rr = rayleigh_ritz(c, s);
      if (rr == INVDFT_OK) break;
      if (rr != INVDFT_ENOTSPD || m == 1) return rr;
    }
    ++pass;
  }
  CU(launch_density(c->X, n, c->occ, c->mass, L, c->rho, s), "density");
  c->have_forward = true;
  if (stats) {
    stats->cheb_passes += pass;
    stats->hx_calls += hx_calls;
    stats->eig_resid_max = maxres;
    double mu = 0.0;
    TRY(fetch(c, c->scal + kScMu, sizeof(double), &mu, s));
    stats->mu = mu;
    stats->t_forward_ms += wall_ms() - t0;
  }
  return status;
}

// ---------------------------------------------------------------- adjoint
namespace {

// Columns of the batched adjoint solve: the occupied states, their shifts,
// and the coefficients of p~ along every computed Ritz vector.
struct AdjPlan {
  int no = 0;
  std::vector<int> idx;            // compact column -> state index
  int *d_idx = nullptr;
  double *d_eps_o = nullptr, *d_f_o = nullptr;
};

// Z <- Z - Psi (Psi^T Z): projection onto the complement of the deflation
// vectors (Psi [L][nv], Z [L][no], both in precision T).  With V != null the
// FP32 path also returns dot[j] = V_j . Z_j (after the projection) from the
// same pass.
template <typename T>
invdft_status deflate(Ctx *c, const T *Psi, int nv, T *Z, int no, cudaStream_t s,
                      const T *V = nullptr, double *dot = nullptr) {
  double *Cp = c->small + 4 * kMaxGram * kMaxGram;
  if (sizeof(T) == 8) {
    if (nv <= 64 && no <= 64)
      CU((launch_stripe_gram<double, double>((const double *)Psi, nv, (const double *)Z, no, c->L,
                                             Cp, c->partial, s)), "gram(deflate)");
    else
      CU(launch_gram((const double *)Psi, nv, (const double *)Z, no, c->L, Cp, c->partial, s),
         "gram(deflate)");
    CU(launch_stripe_rotate<T>(Psi, nv, Cp, no, c->L, Z, -1.0, s), "update(deflate)");
    if (V) CU(launch_coldot((const double *)V, (const double *)Z, no, c->L, dot, c->partial, s), "coldot");
    return INVDFT_OK;
  }
  if (nv > 64 || no > 64 || nv % 8 != 0 || no % 4 != 0) {
    CU(launch_gram_f32acc((const float *)Psi, nv, (const float *)Z, no, c->L, Cp, c->partial, s),
       "gram(deflate)");
    CU(launch_rotate_acc<T>(Psi, nv, Cp, no, c->L, Z, -1.0, s), "rotate(deflate)");
    if (V) CU(launch_coldot_f32((const float *)V, (const float *)Z, no, c->L, dot, c->partial, s), "coldot");
    return INVDFT_OK;
  }
  // padded FP32 blocks (Psi width a multiple of 8, Z width of 4)
  if (no >= 16) {
    // Gram and update on the tensor cores (tcgen05, operands split into two
    // TF32 terms), the column dot fused into the update; timed while the
    // handle's launch timing is on (algorithmic bytes: Psi and Z read for the
    // Gram; Psi, Z and V read and Z written for the update)
    const double L = (double)c->L;
    int k = prof_begin(c, 4, (nv + no) * 4.0 * L, 0.0, s);
    CU(launch_defl_gram_tc((const float *)Psi, nv, (const float *)Z, no, c->L, Cp, c->partial,
                           c->status + kStWaitGram, c->nsm, s), "gram(deflate)");
    prof_end(c, k, s);
    k = prof_begin(c, 5, (nv + (V ? 3 : 2) * no) * 4.0 * L, 0.0, s);
    CU(launch_defl_update_tc((const float *)Psi, nv, Cp, no, c->L, (float *)Z, -1.0,
                             (const float *)V, dot, c->partial, c->status + kStWaitUpdate,
                             c->nsm, s), "update(deflate)");
    prof_end(c, k, s);
  } else {
    // narrow blocks: one row per thread keeps every thread busy
    CU(launch_defl_gram_f32((const float *)Psi, nv, (const float *)Z, no, c->L, Cp, c->partial, s),
       "gram(deflate)");
    CU(launch_stripe_rotate<T>(Psi, nv, Cp, no, c->L, Z, -1.0, s), "update(deflate)");
    if (V) CU(launch_coldot_f32((const float *)V, (const float *)Z, no, c->L, dot, c->partial, s), "coldot");
  }
  return INVDFT_OK;
}

// Batched preconditioned MINRES (Paige & Saunders) on Q (H~ - eps_c) Q for
// every column at once, Q = I - Psi Psi^T, preconditioner Q T Q with T the
// inverse diagonal of the kinetic part (Sec. 3.2.2).  b must lie in range(Q).
template <typename T>
invdft_status minres_block(Ctx *c, const AdjPlan &pl, int n, const T *Psi, int nv, const T *b,
                           T *x, const std::vector<double> &tol, int maxit, int *iters_out,
                           cudaStream_t s) {
  // The legacy default stream cannot be captured into a graph: the solve then
  // runs on the handle's own non-blocking stream, ordered after the caller's
  // stream on entry and before it on every return.
  struct Join {
    Ctx *c;
    cudaStream_t caller = nullptr, own = nullptr;
    ~Join() {
      if (own && cudaEventRecord(c->aux_event, own) == cudaSuccess)
        cudaStreamWaitEvent(caller, c->aux_event, 0);
    }
  } join{c};
  if (!c->prof.on && (s == nullptr || s == cudaStreamLegacy)) {
    bool ok = true;
    if (!c->aux_stream)
      ok = cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&c->aux_event, cudaEventDisableTiming) == cudaSuccess;
    if (ok && cudaEventRecord(c->aux_event, s) == cudaSuccess &&
        cudaStreamWaitEvent(c->aux_stream, c->aux_event, 0) == cudaSuccess) {
      join.caller = s;
      join.own = c->aux_stream;
      s = c->aux_stream;
    }
    cudaGetLastError();
  }
  const long long L = c->L;
  const size_t blk = (size_t)L * n;
  // unnormalised Lanczos vectors qh, zh (current c, other o), w pair, H~ zh
  T *qc = (T *)c->mr[0], *qo = (T *)c->mr[1], *zc = (T *)c->mr[2], *zo = (T *)c->mr[3];
  T *wpp = (T *)c->mr[4], *wp = (T *)c->mr[5], *p = (T *)c->mr[6];
  double *st = c->scal + kScMr;    // kMrCount x n scalars
  CU(launch_prec_apply<T>(b, c->prec_diag, n, L, zc, s), "prec");
  TRY(deflate<T>(c, Psi, nv, zc, n, s));
  if (sizeof(T) == 8)
    CU(launch_coldot((const double *)b, (const double *)zc, n, L, st + kMrBeta1 * n, c->partial, s), "coldot");
  else
    CU(launch_coldot_f32((const float *)b, (const float *)zc, n, L, st + kMrBeta1 * n, c->partial, s), "coldot");
  std::vector<double> h((size_t)kMrCount * n, 0.0);
  TRY(fetch(c, st + kMrBeta1 * n, n * sizeof(double), h.data() + kMrBeta1 * n, s));
  for (int j = 0; j < n; ++j) {
    const double b1 = std::sqrt(std::max(h[kMrBeta1 * n + j], 0.0));
    h[kMrBeta1 * n + j] = b1;
    h[kMrPhibar * n + j] = b1;
    h[kMrActive * n + j] = b1 > 0.0 ? 1.0 : 0.0;
    h[kMrCpp * n + j] = 1.0;
    h[kMrCp * n + j] = 1.0;
    h[kMrTol * n + j] = tol[j];
    h[kMrRel * n + j] = b1 > 0.0 ? 1.0 : 0.0;
    h[kMrIb * n + j] = b1 > 0.0 ? 1.0 / b1 : 0.0;     // q_0 = b / beta_1, z_0 = zh_0 / beta_1
  }
  TRY(push(c, st, h.data(), h.size() * sizeof(double), s));
  CU(cudaMemcpyAsync(qc, b, blk * sizeof(T), cudaMemcpyDeviceToDevice, s), "copy");
  CU(cudaMemsetAsync(qo, 0, blk * sizeof(T), s), "memset");
  CU(cudaMemsetAsync(zo, 0, blk * sizeof(T), s), "memset");
  CU(cudaMemsetAsync(wpp, 0, blk * sizeof(T), s), "memset");
  CU(cudaMemsetAsync(wp, 0, blk * sizeof(T), s), "memset");
  CU(cudaMemsetAsync(x, 0, blk * sizeof(T), s), "memset");
  // one MINRES iteration on the current buffer roles (no host synchronisation)
  auto iteration = [&]() -> invdft_status {
    HxArgs<T> a;
    // the inner MINRES operator stays on the FP32 CUDA cores: with TF32
    // operands (relative error ~3e-4) the inner solves stall early and the
    // FP64 refinement needs several times more outer passes
    set_tc(a, false);
    a.X = zc;
    a.Z = p;
    a.ncol = n;
    a.shift_col = pl.d_eps_o;
    CU(hx_op(c, a, s), "hx(minres)");
    // p <- Q p, raw alpha = zh . p
    TRY(deflate<T>(c, Psi, nv, p, n, s, zc, st + kMrRaw * n));
    // qh_(k+1), zh_(k+1) = T qh_(k+1) (into qo, zo), pending solution update
    CU(launch_mr_step<T>(p, qc, qo, zo, wpp, wp, x, st, c->prec_diag, c->precf, n, L, s),
       "mr_step");
    // zh <- Q zh, beta_(k+1)^2 = qh . zh
    TRY(deflate<T>(c, Psi, nv, zo, n, s, qo, st + kMrBnext * n));
    CU(launch_mr_givens(n, st, s), "mr_givens");
    std::swap(qc, qo);
    std::swap(zc, zo);
    std::swap(wpp, wp);
    return INVDFT_OK;
  };
  // Iterations run in groups of kMrGroup between convergence checks.  Past
  // the first group, a group (two periods of the buffer rotation, so the
  // roles repeat) is captured once as a CUDA graph and replayed: small
  // problems are otherwise bound by launch latency.  Not while H~X launches
  // are being timed (their events would be captured too).
  constexpr int kMrGroup = 4;
  cudaGraphExec_t group = nullptr;
  long long group_kernels = 0;
  bool graphs = !c->prof.on;
  int it = 0;
  std::vector<double> act(n);
  invdft_status result = INVDFT_OK;
  while (it < maxit && result == INVDFT_OK) {
    result = fetch(c, st + kMrActive * n, n * sizeof(double), act.data(), s);
    if (result != INVDFT_OK) break;
    bool any = false;
    for (int j = 0; j < n; ++j) any |= act[j] != 0.0;
    if (!any) break;
    if (graphs && it >= kMrGroup && it + kMrGroup <= maxit) {
      if (!group) {
        T *roles[6] = {qc, qo, zc, zo, wpp, wp};
        const unsigned long long k0 = thread_launches();
        cudaGraph_t g = nullptr;
        bool ok = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          invdft_status cst = INVDFT_OK;
          for (int j = 0; j < kMrGroup && cst == INVDFT_OK; ++j) cst = iteration();
          ok = cudaStreamEndCapture(s, &g) == cudaSuccess && cst == INVDFT_OK;
        }
        if (ok) ok = cudaGraphInstantiate(&group, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        // nothing captured has run: restore the roles and the launch count
        qc = roles[0], qo = roles[1], zc = roles[2], zo = roles[3], wpp = roles[4], wp = roles[5];
        group_kernels = (long long)(thread_launches() - k0);
        count_launches(-group_kernels);
        count_graph(ok ? 0 : 2);
        if (!ok) {
          group = nullptr;
          graphs = false;
          continue;
        }
      }
      if (cudaGraphLaunch(group, s) != cudaSuccess) {
        c->err = "minres: graph launch failed";
        result = INVDFT_ECUDA;
        break;
      }
      count_launches(group_kernels);
      count_graph(1);
      it += kMrGroup;
      continue;
    }
    for (int j = 0; j < kMrGroup && it < maxit && result == INVDFT_OK; ++j, ++it)
      result = iteration();
  }
  if (group) cudaGraphExecDestroy(group);
  if (result != INVDFT_OK) return result;
  CU(launch_mr_finish<T>(zo, wpp, wp, x, st, n, L, s), "mr_finish");
  std::vector<double> itv(n);
  int waits[kStWaitCount];
  TRY(fetch_many(c, {{st + kMrIters * n, n * sizeof(double), itv.data()},
                     {c->status + kStWaitHxTc, sizeof(waits), waits}}, s));
  TRY(check_waits(c, waits));
  int mx = 0;
  for (int j = 0; j < n; ++j) mx = std::max(mx, (int)itv[j]);
  *iters_out = mx;
  return INVDFT_OK;
}

}  // namespace

// Adjoint functions p~ for the upstream dL/drho (device [L]) around the last
// forward solve (Eq. 7-10, 20).  The unique solution is assembled from
//   * the component along the degenerate set Psi_k of each state (Eq. 8-9);
//   * the components along the other converged Ritz vectors psi_j, which
//     (H~ - eps_i) maps to (eps_j - eps_i) psi_j, so psi_j^T p~_i =
//     psi_j^T g~_i / (eps_j - eps_i) exactly for eigenpairs;
//   * the component in the complement of those vectors, where
//     H~ - eps_i is positive definite, by batched preconditioned MINRES
//     (FP32 or FP64 inner iterations) inside FP64 iterative refinement.
// This deflation gives the same p~ as a solve on the complement of Psi_k
// alone (Sec. 3.2.2) but keeps the Krylov operator well conditioned when
// other levels lie close to eps_i.
// Output: compact P_o in c->P ([L][no]), Psi_o in c->HY; *plan_out the map.
invdft_status adjoint_solve(Ctx *c, const double *dLdrho, double *p_full, invdft_stats *stats,
                            AdjPlan *plan_out, cudaStream_t s) {
  const double t0 = wall_ms();
  if (!c->have_forward) {
    c->err = "adjoint_solve: no forward solve at the current potential";
    return INVDFT_EINVAL;
  }
  const int nv = c->nv;
  const long long L = c->L;
  std::vector<double> eps(nv), f(nv), dfde(nv);
  TRY(fetch(c, c->eps, nv * sizeof(double), eps.data(), s));
  TRY(fetch(c, c->occ, nv * sizeof(double), f.data(), s));
  TRY(fetch(c, c->dfde, nv * sizeof(double), dfde.data(), s));
  // adjoint columns: occupied states that are converged (residual <= 10
  // t_eig) or carry f >= 1e-4 (those are converged by the weighted test)
  std::vector<double> res2(nv);
  TRY(fetch(c, c->scal + kScRes, nv * sizeof(double), res2.data(), s));
  const double rtol = 10.0 * std::max(c->eig_tol_used, 1e-12);
  auto converged = [&](int i) { return std::sqrt(std::max(res2[i], 0.0)) <= rtol; };
  AdjPlan pl;
  for (int i = 0; i < nv; ++i)
    if (state_active(c, f[i]) && (converged(i) || conv_weight(c, f[i]) >= 1.0))
      pl.idx.push_back(i);
  pl.no = (int)pl.idx.size();
  const int no = pl.no;
  if (no == 0) {
    c->err = "adjoint_solve: no occupied states";
    return INVDFT_EINVAL;
  }
  // degenerate sets over all computed states (ascending eigenvalues)
  std::vector<int> grp(nv);
  int g = 0;
  for (int i = 0; i < nv; ++i) {
    if (i > 0 && !(eps[i] - eps[i - 1] < c->o.deg_tol)) ++g;
    grp[i] = g;
  }
  // deflation set: the active states and every other Ritz pair converged to
  // the eigen tolerance (an unconverged vector would carry its residual into
  // every column through the exact-ratio formula)
  std::vector<int> dset;
  {
    size_t k = 0;
    for (int i = 0; i < nv; ++i) {
      const bool col = k < pl.idx.size() && pl.idx[k] == i;
      if (col) ++k;
      if (col || converged(i)) dset.push_back(i);
    }
  }
  const int nd = (int)dset.size();
  int *ibase = reinterpret_cast<int *>(c->scal + kScInt);
  pl.d_idx = ibase;
  int *d_dset = ibase + kMaxDense;
  TRY(push(c, ibase, pl.idx.data(), no * sizeof(int), s));
  TRY(push(c, d_dset, dset.data(), nd * sizeof(int), s));
  double *dbase = c->scal + kScAdj;
  pl.d_eps_o = dbase;
  pl.d_f_o = dbase + kMaxDense;
  // the FP32 MINRES blocks are padded to a multiple of 4 columns with zero
  // (inactive) columns; their shifts repeat the last real one
  const int nop = (no + 3) / 4 * 4;
  std::vector<double> eo(nop), fo(no);
  for (int k = 0; k < nop; ++k) eo[k] = eps[pl.idx[std::min(k, no - 1)]];
  for (int k = 0; k < no; ++k) fo[k] = f[pl.idx[k]];
  TRY(push(c, pl.d_eps_o, eo.data(), nop * sizeof(double), s));
  TRY(push(c, pl.d_f_o, fo.data(), no * sizeof(double), s));
  // Psi_o (HY), b = 4 f omega psi (Rg), W = omega psi (Y); Psi_D (C1, FP64)
  double *Psi_o = c->HY, *R = c->Rg, *Wo = c->Y, *Po = c->P, *r64 = c->Y;
  double *PsiD = (double *)c->C1;
  CU(launch_adjoint_rhs(c->X, nv, pl.d_idx, no, pl.d_f_o, dLdrho, c->mass, L, Psi_o, R, Wo, s),
     "adjoint_rhs");
  CU(launch_gather_cols(c->X, nv, d_dset, nd, L, PsiD, s), "gather(psi_D)");
  // J[j][c] = psi_Dj^T diag(omega) psi_{s_c}
  double *J = c->small;
  CU(launch_gram(PsiD, nd, Wo, no, L, J, c->partial, s), "gram(J)");
  std::vector<double> Jh((size_t)nd * no), bn(no);
  TRY(fetch(c, J, Jh.size() * sizeof(double), Jh.data(), s));
  CU(launch_coldot(R, R, no, L, c->scal + kScCol, c->partial, s), "coldot");
  TRY(fetch(c, c->scal + kScCol, no * sizeof(double), bn.data(), s));
  std::vector<int> drow(nv, -1);
  for (int j = 0; j < nd; ++j) drow[dset[j]] = j;
  // eta (Eq. 9), component along the degenerate set (Eq. 8) and along the
  // other deflated vectors; A = Psi_D^T b removes b's part inside span(Psi_D)
  double sdf = 0.0, sdfI = 0.0;
  for (int k = 0; k < no; ++k) {
    sdf += dfde[pl.idx[k]];
    sdfI += dfde[pl.idx[k]] * Jh[(size_t)drow[pl.idx[k]] * no + k];
  }
  const double eta = sdf != 0.0 ? 2.0 * sdfI / sdf : 0.0;
  std::vector<double> Cm((size_t)nd * no), Am((size_t)nd * no), gn(no);
  for (int k = 0; k < no; ++k) {
    const int si = pl.idx[k];
    double along_grp = 0.0;
    for (int jj = 0; jj < nd; ++jj) {
      const int j = dset[jj];
      const double a = 4.0 * f[si] * Jh[(size_t)jj * no + k];
      Am[(size_t)jj * no + k] = a;
      if (grp[j] == grp[si]) {
        Cm[(size_t)jj * no + k] = dfde[si] * (-2.0 * Jh[(size_t)jj * no + k] + (j == si ? eta : 0.0));
        along_grp += a * a;
      } else {
        Cm[(size_t)jj * no + k] = a / (eps[j] - eps[si]);
      }
    }
    gn[k] = std::sqrt(std::max(bn[k] - along_grp, 0.0));     // |g~| of Eq. 10
  }
  double *dC = c->small + 5 * kMaxGram * kMaxGram, *dA = c->small + 6 * kMaxGram * kMaxGram;
  TRY(push(c, dC, Cm.data(), Cm.size() * sizeof(double), s));
  TRY(push(c, dA, Am.data(), Am.size() * sizeof(double), s));
  CU(launch_rotate_acc<double>(PsiD, nd, dA, no, L, R, -1.0, s), "deflate(rhs)");   // R = Q b
  // iterative refinement around the inner MINRES (FP32 or FP64)
  const double tad = adj_tolerance(c);
  const size_t blk = (size_t)L * no;
  CU(cudaMemsetAsync(Po, 0, blk * sizeof(double), s), "memset");
  CU(cudaMemcpyAsync(r64, R, blk * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  const bool mixed = c->o.prec != INVDFT_FP64;
  float *Psi32 = (float *)c->C0;
  const int ndp = (nd + 7) / 8 * 8;
  if (mixed) CU(launch_convert_pad_f32(PsiD, nd, ndp, L, Psi32, s), "convert(psi)");
  std::vector<double> rn(no), tol(no);
  int total_iters = 0, outer = 0;
  double relmax = 0.0;
  invdft_status status = INVDFT_OK;
  // block-normwise criterion: |r_c| <= t_ad max_k |g~_k|, so that every column
  // is accurate in proportion to its share of the gradient (columns of weakly
  // occupied states have small right-hand sides)
  double gmax = 0.0;
  for (int k = 0; k < no; ++k) gmax = std::max(gmax, gn[k]);
  for (;; ++outer) {
    CU(launch_coldot(r64, r64, no, L, c->scal + kScCol, c->partial, s), "coldot");
    TRY(fetch(c, c->scal + kScCol, no * sizeof(double), rn.data(), s));
    relmax = 0.0;
    for (int k = 0; k < no; ++k) {
      const double r = std::sqrt(std::max(rn[k], 0.0));
      const double rel = gmax > 0 ? r / gmax : 0.0;
      relmax = std::max(relmax, rel);
      const double floor_tol = mixed ? 1e-6 : 1e-14;
      // inner tolerance relative to this column's current residual
      tol[k] = rel > tad ? std::max(floor_tol, std::min(0.5, 0.5 * tad / rel)) : 1.0;
    }
    if (relmax <= tad) break;
    if (outer >= 12) {
      status = INVDFT_ENOCONV;
      c->err = "adjoint solve: refinement cap reached";
      break;
    }
    int its = 0;
    if (mixed) {
      float *b32 = (float *)c->mr[8], *x32 = (float *)c->mr[7];
      CU(launch_convert_pad_f32(r64, no, nop, L, b32, s), "convert");
      std::vector<double> tolp(nop, 1.0);
      std::copy(tol.begin(), tol.end(), tolp.begin());
      TRY(minres_block<float>(c, pl, nop, Psi32, ndp, b32, x32, tolp, c->o.max_minres_iters,
                              &its, s));
      CU(launch_add_unpad(x32, nop, Po, no, L, s), "add");
    } else {
      double *b64 = (double *)c->mr[8], *x64 = (double *)c->mr[7];
      CU(cudaMemcpyAsync(b64, r64, blk * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
      TRY(minres_block<double>(c, pl, no, PsiD, nd, b64, x64, tol, c->o.max_minres_iters, &its,
                               s));
      CU((launch_add_convert<double, double>(x64, Po, (long long)blk, s)), "add");
    }
    total_iters += its;
    // r = Q b - Q (H~ - eps) p: the inner solutions lie in range(Q) up to the
    // inner precision, and the part of p along Psi that this leaves changes
    // Q (H~ - eps) p only by Q (H~ Psi - Psi Lambda) c (the Ritz residuals
    // times that part), far below the refinement tolerance; p itself is
    // projected once after the loop
    HxArgs<double> a;
    a.X = Po;
    a.Z = r64;
    a.ncol = no;
    a.alpha = -1.0;
    a.shift_col = pl.d_eps_o;
    a.W = R;
    a.beta = 1.0;
    CU(hx_op(c, a, s), "hx(residual)");
    TRY(deflate<double>(c, PsiD, nd, r64, no, s));
  }
  TRY(deflate<double>(c, PsiD, nd, Po, no, s));
  // p~ = p_Q + Psi C  (Eq. 8 inside the degenerate set, exact ratios outside)
  CU(launch_rotate_acc<double>(PsiD, nd, dC, no, L, Po, 1.0, s), "along(psi)");
  if (p_full) {
    CU(cudaMemsetAsync(p_full, 0, (size_t)L * nv * sizeof(double), s), "memset");
    CU(launch_scatter_cols(Po, no, pl.d_idx, p_full, nv, L, s), "scatter");
  }
  if (stats) {
    stats->adj_resid_max = relmax;
    stats->eta = eta;
    stats->minres_iters_max = std::max(stats->minres_iters_max, total_iters);
    stats->refinements += outer;
    stats->t_adjoint_ms += wall_ms() - t0;
  }
  if (plan_out) *plan_out = pl;
  return status;
}

// ---------------------------------------------------------------- loss, gradient
invdft_status loss_grad(Ctx *c, const double *rd, const double *w, double *grad,
                        invdft_stats *stats, double *loss_out, cudaStream_t s) {
  invdft_status fst = forward_solve(c, stats, s);
  if (fst != INVDFT_OK && fst != INVDFT_ENOCONV) return fst;
  double out3[3];
  CU(launch_loss(c->rho, rd, w, c->mass, c->L, c->scal, c->dLdrho, c->partial, s), "loss");
  TRY(fetch(c, c->scal, 3 * sizeof(double), out3, s));
  c->loss = out3[0];
  c->err_l2 = std::sqrt(std::max(out3[1], 0.0));
  AdjPlan pl;
  invdft_status ast = adjoint_solve(c, c->dLdrho, nullptr, stats, &pl, s);
  if (ast != INVDFT_OK && ast != INVDFT_ENOCONV) return ast;
  CU(launch_gradient(c->P, c->HY, pl.no, rd, c->o.tau_bc, c->L, grad, s), "gradient");
  if (stats) {
    stats->loss = c->loss;
    stats->err_l2 = c->err_l2;
    stats->n_elec = out3[2];
  }
  if (loss_out) *loss_out = c->loss;
  return fst != INVDFT_OK ? fst : ast;
}

// loss only (line-search trial): forward + loss
invdft_status loss_only(Ctx *c, const double *rd, const double *w, invdft_stats *stats,
                        double *loss_out, double *err_out, cudaStream_t s) {
  invdft_status fst = forward_solve(c, stats, s);
  if (fst != INVDFT_OK && fst != INVDFT_ENOCONV) return fst;
  double out3[3];
  CU(launch_loss(c->rho, rd, w, c->mass, c->L, c->scal, nullptr, c->partial, s), "loss");
  TRY(fetch(c, c->scal, 3 * sizeof(double), out3, s));
  *loss_out = out3[0];
  *err_out = std::sqrt(std::max(out3[1], 0.0));
  if (stats) stats->n_elec = out3[2];
  return INVDFT_OK;
}

invdft_status set_v(Ctx *c, const double *vxc, cudaStream_t s) {
  CU(launch_lincomb(1.0, c->vfixed, 1.0, vxc, c->v, c->L, s), "set_v");
  CU(launch_convert_f64_to_f32(c->v, c->vf, c->L, s), "set_v(f32)");
  c->have_forward = false;
  c->have_upper = false;
  return INVDFT_OK;
}

double dot_host(Ctx *c, const double *x, const double *y, cudaStream_t s, invdft_status *st) {
  double r = 0.0;
  if (!cuda_ok(c, launch_dot(x, y, c->L, c->scal, c->partial, s), "dot")) {
    *st = INVDFT_ECUDA;
    return 0.0;
  }
  *st = fetch(c, c->scal, sizeof(double), &r, s);
  return r;
}

// one L-BFGS iteration (Eq. 21) with backtracking; readings match the oracle
invdft_status lbfgs_step(Ctx *c, const double *rd, const double *w, double *vxc,
                         invdft_stats *stats, cudaStream_t s) {
  const long long L = c->L;
  invdft_status st = INVDFT_OK;
  if (!c->have_grad) {
    TRY(set_v(c, vxc, s));
    double loss;
    invdft_status r = loss_grad(c, rd, w, c->grad, stats, &loss, s);
    if (r != INVDFT_OK && r != INVDFT_ENOCONV) return r;
    c->have_grad = true;
  }
  // direction by the two-loop recursion
  const int m = c->o.lbfgs_history;
  const int k = c->hist_n;
  double *d = c->dir;
  if (k == 0) {
    CU(launch_absmax(c->grad, L, c->scal, c->partial, s), "absmax");
    double gmax;
    TRY(fetch(c, c->scal, sizeof(double), &gmax, s));
    CU(launch_lincomb(gmax > 0 ? -0.1 / gmax : 0.0, c->grad, 0.0, c->grad, d, L, s), "lincomb");
  } else {
    CU(cudaMemcpyAsync(d, c->grad, L * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    std::vector<double> alpha(k), rho(k);
    auto slot = [&](int j) { return (c->hist_head - k + j + m) % m; };  // j = 0 oldest
    for (int j = k - 1; j >= 0; --j) {
      const double *Sj = c->Sh + (size_t)slot(j) * L, *Yj = c->Yh + (size_t)slot(j) * L;
      rho[j] = 1.0 / dot_host(c, Yj, Sj, s, &st);
      alpha[j] = rho[j] * dot_host(c, Sj, d, s, &st);
      TRY(st);
      CU(launch_axpby(-alpha[j], Yj, 1.0, d, L, s), "axpby");
    }
    const double *Sn = c->Sh + (size_t)slot(k - 1) * L, *Yn = c->Yh + (size_t)slot(k - 1) * L;
    const double gamma = dot_host(c, Sn, Yn, s, &st) / dot_host(c, Yn, Yn, s, &st);
    TRY(st);
    CU(launch_axpby(0.0, d, gamma, d, L, s), "scale");
    for (int j = 0; j < k; ++j) {
      const double *Sj = c->Sh + (size_t)slot(j) * L, *Yj = c->Yh + (size_t)slot(j) * L;
      const double beta = rho[j] * dot_host(c, Yj, d, s, &st);
      TRY(st);
      CU(launch_axpby(alpha[j] - beta, Sj, 1.0, d, L, s), "axpby");
    }
    CU(launch_axpby(0.0, d, -1.0, d, L, s), "negate");
  }
  const double slope = dot_host(c, c->grad, d, s, &st);
  TRY(st);
  double alpha = 1.0, L_try = 0.0, e_try = 0.0;
  int trials = 0;
  for (int t = 0; t < 10; ++t) {
    CU(launch_lincomb(1.0, vxc, alpha, d, c->vtry, L, s), "trial");
    TRY(set_v(c, c->vtry, s));
    invdft_status r = loss_only(c, rd, w, stats, &L_try, &e_try, s);
    if (r != INVDFT_OK && r != INVDFT_ENOCONV) return r;
    ++trials;
    if (L_try <= c->loss + 1e-4 * alpha * slope || t == 9) break;
    alpha *= 0.5;
  }
  // gradient at the accepted point (forward data of the last trial are current)
  {
    double out3[3];
    CU(launch_loss(c->rho, rd, w, c->mass, L, c->scal, c->dLdrho, c->partial, s), "loss");
    TRY(fetch(c, c->scal, 3 * sizeof(double), out3, s));
    c->loss = out3[0];
    c->err_l2 = std::sqrt(std::max(out3[1], 0.0));
    AdjPlan pl;
    invdft_status ast = adjoint_solve(c, c->dLdrho, nullptr, stats, &pl, s);
    if (ast != INVDFT_OK && ast != INVDFT_ENOCONV) return ast;
    CU(launch_gradient(c->P, c->HY, pl.no, rd, c->o.tau_bc, L, c->grad_new, s), "gradient");
    if (stats) {
      stats->n_elec = out3[2];
    }
  }
  // history: s = vtry - vxc, y = grad_new - grad
  double *Ss = c->Sh + (size_t)c->hist_head * L, *Ys = c->Yh + (size_t)c->hist_head * L;
  CU(launch_lincomb(1.0, c->vtry, -1.0, vxc, Ss, L, s), "s");
  CU(launch_lincomb(1.0, c->grad_new, -1.0, c->grad, Ys, L, s), "y");
  const double sy = dot_host(c, Ss, Ys, s, &st);
  const double ss = dot_host(c, Ss, Ss, s, &st);
  const double yy = dot_host(c, Ys, Ys, s, &st);
  TRY(st);
  if (sy > 1e-12 * std::sqrt(ss) * std::sqrt(yy)) {
    c->hist_head = (c->hist_head + 1) % m;
    c->hist_n = std::min(c->hist_n + 1, m);
  }
  CU(cudaMemcpyAsync(vxc, c->vtry, L * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  CU(cudaMemcpyAsync(c->grad, c->grad_new, L * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
  if (stats) {
    stats->loss = c->loss;
    stats->err_l2 = c->err_l2;
    stats->ls_trials = trials;
  }
  CU(cudaStreamSynchronize(s), "sync");
  return INVDFT_OK;
}

}  // namespace invdft

using namespace invdft;

extern "C" {

static bool ready(invdft_handle h, const char *who) {
  if (!h->bound || !h->have_potential) {
    h->err = std::string(who) + ": bind a workspace and set a potential first";
    return false;
  }
  return true;
}

invdft_status invdft_forward_solve(invdft_handle h, double *psi, double *eps, double *occ,
                                   double *rho, invdft_stats *stats, void *stream) {
  if (!h) return INVDFT_EINVAL;
  if (!ready(h, "forward_solve")) return INVDFT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  invdft_status st = forward_solve(h, stats, s);
  if (st != INVDFT_OK && st != INVDFT_ENOCONV) return st;
  const size_t n = h->nv;
  if (psi) INV_CUDA(h, cudaMemcpyAsync(psi, h->X, (size_t)h->L * n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (eps) INV_CUDA(h, cudaMemcpyAsync(eps, h->eps, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (occ) INV_CUDA(h, cudaMemcpyAsync(occ, h->occ, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (rho) INV_CUDA(h, cudaMemcpyAsync(rho, h->rho, (size_t)h->L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  INV_CUDA(h, cudaStreamSynchronize(s));
  return st;
}

invdft_status invdft_adjoint_solve(invdft_handle h, const double *dLdrho, double *p,
                                   invdft_stats *stats, void *stream) {
  if (!h || !dLdrho) return INVDFT_EINVAL;
  if (!ready(h, "adjoint_solve")) return INVDFT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  invdft_status st = adjoint_solve(h, dLdrho, p, stats, nullptr, s);
  INV_CUDA(h, cudaStreamSynchronize(s));
  return st;
}

invdft_status invdft_density_vjp(invdft_handle h, const double *dLdrho, double *grad_v,
                                 invdft_stats *stats, void *stream) {
  if (!h || !dLdrho || !grad_v) return INVDFT_EINVAL;
  if (!ready(h, "density_vjp")) return INVDFT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  AdjPlan pl;
  invdft_status st = adjoint_solve(h, dLdrho, nullptr, stats, &pl, s);
  if (st != INVDFT_OK && st != INVDFT_ENOCONV) return st;
  if (!cuda_ok(h, launch_gradient(h->P, h->HY, pl.no, nullptr, 0.0, h->L, grad_v, s), "gradient"))
    return INVDFT_ECUDA;
  INV_CUDA(h, cudaStreamSynchronize(s));
  return st;
}

invdft_status invdft_loss_grad(invdft_handle h, const double *rd, const double *w, double *loss_out,
                               double *grad, invdft_stats *stats, void *stream) {
  if (!h || !rd || !w || !grad) return INVDFT_EINVAL;
  if (!ready(h, "loss_grad")) return INVDFT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  invdft_status st = loss_grad(h, rd, w, grad, stats, loss_out, s);
  INV_CUDA(h, cudaStreamSynchronize(s));
  return st;
}

invdft_status invdft_step(invdft_handle h, const double *rd, const double *w, double *vxc,
                          invdft_stats *stats, void *stream) {
  if (!h || !rd || !w || !vxc) return INVDFT_EINVAL;
  if (!ready(h, "step")) return INVDFT_EINVAL;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return lbfgs_step(h, rd, w, vxc, stats, (cudaStream_t)stream);
}

}  // extern "C"
