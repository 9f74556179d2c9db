// Internal solver interfaces of libinvdft (host orchestration + kernel launchers).
#pragma once

#include "internal.h"

namespace invdft {

// Layout of the per-handle scalar area c->scal (doubles)
constexpr size_t kScMisc = 0;                       // dots, loss sums
constexpr size_t kScMu = 32;                        // chemical potential
constexpr size_t kScRes = 64;                       // Ritz residual norms^2 [nv]
constexpr size_t kScCol = 512;                      // column dots [<= 256]
constexpr size_t kScAdj = 200 * (size_t)kMaxCols;   // adjoint per-column tables
constexpr size_t kScMr = 256 * (size_t)kMaxCols;    // MINRES scalars
constexpr size_t kScInt = 400 * (size_t)kMaxCols;   // adjoint int tables
constexpr size_t kScPk = 512 * (size_t)kMaxCols;    // Chebyshev p_k(theta) table

// ---- dense.cu
cudaError_t launch_rr_small(const double *S, const double *H, int n, double *theta, double *C,
                            int *status, double *work, cudaStream_t s);
cudaError_t launch_occupations(const double *eps, int n, double ne, double kT, double *f,
                               double *dfde, double *mu, int *status, cudaStream_t s);

// ---- physics.cu
// rho[a] = sum_i occ[i] X[a][i]^2 / m[a]
cudaError_t launch_density(const double *X, int n, const double *occ, const double *mass,
                           long long L, double *rho, cudaStream_t s);
// out[0] = sum m w (rd - rho)^2, out[1] = sum m (rd - rho)^2, out[2] = sum m rho;
// dLdrho (optional) = -2 m w (rd - rho)
cudaError_t launch_loss(const double *rho, const double *rd, const double *w, const double *mass,
                        long long L, double *out3, double *dLdrho, double *partial, cudaStream_t s);
// Psi_o[a][c] = X[a][idx[c]];  R[a][c] = 4 f_c omega_a Psi_o[a][c],
// Wo[a][c] = omega_a Psi_o[a][c] with omega = -dLdrho / (2 m)
cudaError_t launch_adjoint_rhs(const double *X, int nv, const int *idx, int no, const double *f_o,
                               const double *dLdrho, const double *mass, long long L,
                               double *Psi_o, double *R, double *Wo, cudaStream_t s);
// coef[k] = sum_a A[a*lda + ia[k]] * B[a*ldb + ib[k]] for k < npairs (FP64 accumulate)
template <typename TA, typename TB>
cudaError_t launch_pairdot(const TA *A, int lda, const int *ia, const TB *B, int ldb, const int *ib,
                           int npairs, long long L, double *coef, double *partial, cudaStream_t s);
// X[a][ib[k]] -= coef[k] * Psi[a][ia[k]] for all pairs (pairs grouped by column)
template <typename T>
cudaError_t launch_project_apply(const double *Psi, int ldp, const int *col_start, const int *ia,
                                 const double *coef, T *X, int ncol, long long L, cudaStream_t s);
// grad[a] = sum_c P[a][c] Psi[a][c], 0 where rd < tau
cudaError_t launch_gradient(const double *P, const double *Psi, int ncol, const double *rd,
                            double tau, long long L, double *grad, cudaStream_t s);
// scalar reductions over [L] vectors: dot, max |x|
cudaError_t launch_dot(const double *x, const double *y, long long n, double *out, double *partial,
                       cudaStream_t s);
cudaError_t launch_absmax(const double *x, long long n, double *out, double *partial,
                          cudaStream_t s);
// y = a x + b y (+ c z), elementwise over n
cudaError_t launch_axpby(double a, const double *x, double b, double *y, long long n,
                         cudaStream_t s);
cudaError_t launch_lincomb(double a, const double *x, double b, const double *y, double *out,
                           long long n, cudaStream_t s);
// per-column elementwise helpers for the subspace and MINRES
cudaError_t launch_residual_block(const double *HX, const double *X, const double *theta, int n,
                                  long long L, double *E64, float *E32, cudaStream_t s);
cudaError_t launch_cheb_combine(const double *X, const double *pm, const float *D, int n,
                                long long L, double *Y, cudaStream_t s);
cudaError_t launch_scale_f32(const float *E, const double *scale_scalar, double alpha, int n,
                             long long L, float *D, cudaStream_t s);

// ---- MINRES (templated on the inner precision)
// Per-column scalars st[k * n + c] of the batched MINRES recurrence.  The
// Lanczos vectors are kept unnormalised (q_k = s_k qh_k, z_k = s_k zh_k with
// s_k = 1 / beta_k): kMrIb holds s_k, kMrIbp s_(k-1), kMrRaw the dot
// zh_k . (H~ - eps) zh_k, kMrAlpha alpha_k; kMrEps/Del/Ig/T are the Givens
// coefficients of the solution update of the last finished iteration.
enum { kMrAlpha = 0, kMrBeta, kMrBnext, kMrCpp, kMrSpp, kMrCp, kMrSp, kMrPhibar, kMrBeta1,
       kMrActive, kMrEps, kMrDel, kMrIg, kMrT, kMrIb, kMrRel, kMrTol, kMrIters, kMrIbp, kMrRaw,
       kMrCount };
// One fused pass of iteration k (all [L][n] blocks, in place where noted):
//   qh_(k+1) = s_k ph - alpha_k s_k qh_k - beta_k s_(k-1) qh_(k-1)   -> qo
//   zh_(k+1) = T qh_(k+1)                                           -> zo
//   w = (s_(k-1) zh_(k-1) - eps wpp - del wp) ig,  x += t w           -> wpp, x
// with alpha_k = s_k^2 raw_k (also stored to kMrAlpha), qo holding qh_(k-1)
// and zo holding zh_(k-1) on entry.  Inactive columns get qh = zh = 0.
// prec: T = inverse diagonal (FP64), precf its FP32 copy (FP32 blocks).
template <typename T>
cudaError_t launch_mr_step(const T *ph, const T *qh, T *qo, T *zo, T *wpp, const T *wp, T *x,
                           double *st, const double *prec, const float *precf, int n, long long L,
                           cudaStream_t s);
// The solution update alone (after the last iteration): w and x as above.
template <typename T>
cudaError_t launch_mr_finish(const T *zo, T *wpp, const T *wp, T *x, const double *st, int n,
                             long long L, cudaStream_t s);
cudaError_t launch_mr_givens(int n, double *st, cudaStream_t s);
template <typename T>
cudaError_t launch_prec_apply(const T *r, const double *prec, int n, long long L, T *z,
                              cudaStream_t s);
// p_o[a][c] += Psi_o[a][members] * d  for the component along the degenerate set
cudaError_t launch_add_along(const double *Psi_o, const int *col_start, const int *ia,
                             const double *dcoef, double *P, int n, long long L, cudaStream_t s);
cudaError_t launch_scatter_cols(const double *Po, int no, const int *idx, double *P, int nv,
                                long long L, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_add_convert(const TI *d, TO *p, long long n, cudaStream_t s);

// ---- solvers.cu
// Chebyshev filter of degree m on an [L][ncol] block in precision prec; with
// (theta, E) the defect-corrected form around Ritz pairs (mixed path).
invdft_status run_filter(Ctx *c, const void *X, void *Y, int ncol, int degree, double a, double b,
                         double a0, invdft_precision prec, const double *theta_host,
                         const float *E, cudaStream_t s);

}  // namespace invdft
