// Nodal kernels of the inverse-DFT step: density (Eq. 4), loss and L2 error
// (Eq. 1, Sec. 4.2.4), adjoint right-hand sides (Eq. 7, 10, 18), projections
// onto the complement of a degenerate set (Sec. 3.2.2), the gradient (Eq. 11,
// 22) with the far-field mask (Sec. 3.1.2), the elementwise steps of the
// batched preconditioned MINRES, and vector helpers for L-BFGS (Eq. 21).
#include "internal.h"
#include "solvers.h"

namespace invdft {
namespace {

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 8); }

#define GRID_STRIDE(i, n)                                                          \
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
       i += (long long)gridDim.x * blockDim.x)
// 32-bit grid stride over an [L][n] block (L * n < 2^31 is checked at handle creation)
#define GRID_STRIDE32(i, total)                                                         \
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < (uint32_t)(total);       \
       i += gridDim.x * blockDim.x)

__global__ void density_kernel(const double *__restrict__ X, int n, const double *__restrict__ occ,
                               const double *__restrict__ mass, long long L,
                               double *__restrict__ rho) {
  GRID_STRIDE(a, L) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
      const double x = X[a * n + i];
      s += occ[i] * x * x;
    }
    rho[a] = s / mass[a];
  }
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (blockDim.x + 31) / 32; ++k) t += red[k];
  return t;
}

__global__ void loss_partial(const double *__restrict__ rho, const double *__restrict__ rd,
                             const double *__restrict__ w, const double *__restrict__ mass,
                             long long L, double *__restrict__ partial,
                             double *__restrict__ dLdrho) {
  __shared__ double red[32];
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  GRID_STRIDE(a, L) {
    const double m = mass[a], d = rd[a] - rho[a], ww = w ? w[a] : 1.0;
    s0 += m * ww * d * d;
    s1 += m * d * d;
    s2 += m * rho[a];
    if (dLdrho) dLdrho[a] = -2.0 * m * ww * d;
  }
  const double t0 = block_sum(s0, red);
  const double t1 = block_sum(s1, red);
  const double t2 = block_sum(s2, red);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x + 0] = t0;
    partial[3 * blockIdx.x + 1] = t1;
    partial[3 * blockIdx.x + 2] = t2;
  }
}

__global__ void sum3(const double *__restrict__ partial, int nblk, double *__restrict__ out) {
  const int k = threadIdx.x;
  if (k >= 3) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[3 * b + k];
  out[k] = s;
}

__global__ void adjoint_rhs_kernel(const double *__restrict__ X, int nv, const int *__restrict__ idx,
                                   int no, const double *__restrict__ f_o,
                                   const double *__restrict__ dLdrho,
                                   const double *__restrict__ mass, long long L,
                                   double *__restrict__ Psi_o, double *__restrict__ R,
                                   double *__restrict__ Wo, FastDiv fd) {
  GRID_STRIDE32(e, L * no) {
    const uint32_t a = fdiv(e, fd);
    const int c = (int)(e - a * (uint32_t)no);
    const double psi = X[a * nv + idx[c]];
    const double omega = -dLdrho[a] / (2.0 * mass[a]);
    Psi_o[e] = psi;
    R[e] = 4.0 * f_o[c] * omega * psi;
    Wo[e] = omega * psi;
  }
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) pairdot_partial(const TA *__restrict__ A, int lda,
                                                       const int *__restrict__ ia,
                                                       const TB *__restrict__ B, int ldb,
                                                       const int *__restrict__ ib, int npairs,
                                                       long long L, double *__restrict__ partial) {
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int k0 = blockIdx.y * 256;
  const int np = min(256, npairs - k0);
  const int R = 256 / np;
  const int k = k0 + tid % np, r0 = tid / np;
  double s = 0.0;
  if (r0 < R) {
    const int ja = ia[k], jb = ib[k];
    for (long long a = (long long)blockIdx.x * R + r0; a < L; a += (long long)gridDim.x * R)
      s += (double)A[a * lda + ja] * (double)B[a * ldb + jb];
  }
  red[tid] = s;
  __syncthreads();
  if (tid < np) {
    double t = 0.0;
    for (int r = 0; r < R; ++r) t += red[r * np + tid];
    partial[(size_t)blockIdx.x * kMaxDense * kMaxGroup + k0 + tid] = t;
  }
}

__global__ void pair_sum(const double *__restrict__ partial, int nblk, int npairs,
                         double *__restrict__ coef) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= npairs) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kMaxDense * kMaxGroup + k];
  coef[k] = s;
}

template <typename T>
__global__ void project_apply_kernel(const double *__restrict__ Psi, int ldp,
                                     const int *__restrict__ cs, const int *__restrict__ ia,
                                     const double *__restrict__ coef, double scale,
                                     T *__restrict__ X, int ncol, long long L) {
  GRID_STRIDE(e, L * ncol) {
    const long long a = e / ncol;
    const int c = (int)(e - a * ncol);
    double s = 0.0;
    for (int k = cs[c]; k < cs[c + 1]; ++k) s += coef[k] * Psi[a * ldp + ia[k]];
    X[e] = (T)((double)X[e] + scale * s);
  }
}

__global__ void gradient_kernel(const double *__restrict__ P, const double *__restrict__ Psi,
                                int ncol, const double *__restrict__ rd, double tau, long long L,
                                double *__restrict__ grad) {
  GRID_STRIDE(a, L) {
    double s = 0.0;
    for (int c = 0; c < ncol; ++c) s += P[a * ncol + c] * Psi[a * ncol + c];
    grad[a] = (rd && rd[a] < tau) ? 0.0 : s;
  }
}

__global__ void dot_partial(const double *__restrict__ x, const double *__restrict__ y, long long n,
                            double *__restrict__ partial) {
  __shared__ double red[32];
  double s = 0.0;
  GRID_STRIDE(i, n) s += x[i] * y[i];
  const double t = block_sum(s, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = t;
}
__global__ void absmax_partial(const double *__restrict__ x, long long n,
                               double *__restrict__ partial) {
  __shared__ double red[32];
  double s = 0.0;
  GRID_STRIDE(i, n) s = fmax(s, fabs(x[i]));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (blockDim.x + 31) / 32; ++k) t = fmax(t, red[k]);
    partial[blockIdx.x] = t;
  }
}
__global__ void reduce_partials(const double *__restrict__ partial, int nblk, int op,
                                double *__restrict__ out) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s = op ? fmax(s, partial[b]) : s + partial[b];
  out[0] = s;
}

__global__ void axpby_kernel(double a, const double *__restrict__ x, double b,
                             double *__restrict__ y, long long n) {
  GRID_STRIDE(i, n) y[i] = a * x[i] + b * y[i];
}
__global__ void lincomb_kernel(double a, const double *__restrict__ x, double b,
                               const double *__restrict__ y, double *__restrict__ out, long long n) {
  GRID_STRIDE(i, n) out[i] = a * x[i] + b * y[i];
}

__global__ void residual_block_kernel(const double *__restrict__ HX, const double *__restrict__ X,
                                      const double *__restrict__ theta, int n, long long L,
                                      double *__restrict__ E64, float *__restrict__ E32,
                                      FastDiv fd) {
  GRID_STRIDE32(e, L * n) {
    const int j = (int)(e - fdiv(e, fd) * (uint32_t)n);
    const double r = HX[e] - theta[j] * X[e];
    if (E64) E64[e] = r;
    if (E32) E32[e] = (float)r;
  }
}

__global__ void cheb_combine_kernel(const double *__restrict__ X, const double *__restrict__ pm,
                                    const float *__restrict__ D, int n, long long L,
                                    double *__restrict__ Y, FastDiv fd) {
  GRID_STRIDE32(e, L * n) {
    const int j = (int)(e - fdiv(e, fd) * (uint32_t)n);
    Y[e] = X[e] * pm[j] + (double)D[e];
  }
}

__global__ void scale_f32_kernel(const float *__restrict__ E, double alpha, int n, long long L,
                                 float *__restrict__ D) {
  GRID_STRIDE(e, L * n) D[e] = (float)(alpha * (double)E[e]);
}

// st layout: st[k * n + c] for scalar k (kMr* in solvers.h) of column c
__global__ void mr_givens_kernel(int n, double *__restrict__ st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  auto S = [&](int k) -> double & { return st[(size_t)k * n + c]; };
  const double bn = sqrt(fmax(S(kMrBnext), 0.0));
  auto retire = [&]() {
    S(kMrEps) = S(kMrDel) = S(kMrIg) = S(kMrT) = 0.0;
    S(kMrIbp) = S(kMrIb);
    S(kMrIb) = 0.0;
  };
  if (S(kMrActive) == 0.0) {
    retire();
    return;
  }
  const double a = S(kMrAlpha), b = S(kMrBeta);
  const double eps_k = S(kMrSpp) * b;
  const double tmp = S(kMrCpp) * b;
  const double delta = S(kMrCp) * tmp + S(kMrSp) * a;
  const double gbar = -S(kMrSp) * tmp + S(kMrCp) * a;
  const double gamma = hypot(gbar, bn);
  if (!(gamma > 0.0)) {
    S(kMrActive) = 0.0;
    retire();
    return;
  }
  const double cs = gbar / gamma, sn = bn / gamma;
  const double t = cs * S(kMrPhibar);
  S(kMrPhibar) = -sn * S(kMrPhibar);
  S(kMrEps) = eps_k;
  S(kMrDel) = delta;
  S(kMrIg) = 1.0 / gamma;
  S(kMrT) = t;
  S(kMrCpp) = S(kMrCp);
  S(kMrSpp) = S(kMrSp);
  S(kMrCp) = cs;
  S(kMrSp) = sn;
  S(kMrBeta) = bn;
  S(kMrIbp) = S(kMrIb);
  S(kMrIb) = bn > 0.0 ? 1.0 / bn : 0.0;
  S(kMrRel) = fabs(S(kMrPhibar)) / S(kMrBeta1);
  S(kMrIters) += 1.0;
  if (S(kMrRel) <= S(kMrTol) || bn == 0.0) S(kMrActive) = 0.0;
}

template <typename T>
__global__ void mr_step_kernel(const T *__restrict__ ph, const T *__restrict__ qh,
                               T *__restrict__ qo, T *__restrict__ zo, T *__restrict__ wpp,
                               const T *__restrict__ wp, T *__restrict__ x,
                               double *__restrict__ st, const double *__restrict__ prec, int n,
                               long long L, FastDiv fd) {
  __shared__ T c1[kMaxCols], c2[kMaxCols], c3[kMaxCols], cz[kMaxCols];
  __shared__ T ce[kMaxCols], cd[kMaxCols], cg[kMaxCols], ct[kMaxCols];
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double sk = st[kMrIb * n + c], skm = st[kMrIbp * n + c], bk = st[kMrBeta * n + c];
    const bool on = st[kMrActive * n + c] != 0.0;
    const double alpha = sk * sk * st[kMrRaw * n + c];
    if (blockIdx.x == 0) st[kMrAlpha * n + c] = alpha;
    c1[c] = on ? (T)sk : (T)0;
    c2[c] = on ? (T)(-alpha * sk) : (T)0;
    c3[c] = on ? (T)(-bk * skm) : (T)0;
    cz[c] = (T)skm;
    ce[c] = (T)st[kMrEps * n + c];
    cd[c] = (T)st[kMrDel * n + c];
    cg[c] = (T)st[kMrIg * n + c];
    ct[c] = (T)st[kMrT * n + c];
  }
  __syncthreads();
  GRID_STRIDE32(e, L * n) {
    const uint32_t a = fdiv(e, fd);
    const int c = (int)(e - a * (uint32_t)n);
    const T w = (cz[c] * zo[e] - ce[c] * wpp[e] - cd[c] * wp[e]) * cg[c];
    wpp[e] = w;
    x[e] += ct[c] * w;
    const T q = c1[c] * ph[e] + c2[c] * qh[e] + c3[c] * qo[e];
    qo[e] = q;
    zo[e] = (T)prec[a] * q;
  }
}

// mr_step_kernel for FP32 blocks whose width is a multiple of 4: one thread
// per (node, column quad), float4 loads and stores
__global__ void mr_step_vec4_kernel(const float4 *__restrict__ ph, const float4 *__restrict__ qh,
                                    float4 *__restrict__ qo, float4 *__restrict__ zo,
                                    float4 *__restrict__ wpp, const float4 *__restrict__ wp,
                                    float4 *__restrict__ x, double *__restrict__ st,
                                    const float *__restrict__ prec, int n, long long L,
                                    FastDiv fd4) {
  __shared__ float4 c1[kMaxCols / 4], c2[kMaxCols / 4], c3[kMaxCols / 4], cz[kMaxCols / 4];
  __shared__ float4 ce[kMaxCols / 4], cd[kMaxCols / 4], cg[kMaxCols / 4], ct[kMaxCols / 4];
  float *f1 = reinterpret_cast<float *>(c1), *f2 = reinterpret_cast<float *>(c2);
  float *f3 = reinterpret_cast<float *>(c3), *fz = reinterpret_cast<float *>(cz);
  float *fe = reinterpret_cast<float *>(ce), *fdl = reinterpret_cast<float *>(cd);
  float *fg = reinterpret_cast<float *>(cg), *ft = reinterpret_cast<float *>(ct);
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    const double sk = st[kMrIb * n + c], skm = st[kMrIbp * n + c], bk = st[kMrBeta * n + c];
    const bool on = st[kMrActive * n + c] != 0.0;
    const double alpha = sk * sk * st[kMrRaw * n + c];
    if (blockIdx.x == 0) st[kMrAlpha * n + c] = alpha;
    f1[c] = on ? (float)sk : 0.f;
    f2[c] = on ? (float)(-alpha * sk) : 0.f;
    f3[c] = on ? (float)(-bk * skm) : 0.f;
    fz[c] = (float)skm;
    fe[c] = (float)st[kMrEps * n + c];
    fdl[c] = (float)st[kMrDel * n + c];
    fg[c] = (float)st[kMrIg * n + c];
    ft[c] = (float)st[kMrT * n + c];
  }
  __syncthreads();
  const int n4 = n / 4;
  GRID_STRIDE32(e, L * n4) {
    const uint32_t a = fdiv(e, fd4);
    const int c = (int)(e - a * (uint32_t)n4);
    const float4 z0 = zo[e], w2 = wpp[e], w1 = wp[e], x0 = x[e];
    const float4 p0 = ph[e], q1 = qh[e], q0 = qo[e];
    const float4 a1 = c1[c], a2 = c2[c], a3 = c3[c], az = cz[c];
    const float4 ae = ce[c], ad = cd[c], ag = cg[c], at = ct[c];
    const float pr = prec[a];
    float4 w, xn, q, z;
#define MR_LANE(k)                                                      \
  w.k = (az.k * z0.k - ae.k * w2.k - ad.k * w1.k) * ag.k;               \
  xn.k = fmaf(at.k, w.k, x0.k);                                         \
  q.k = a1.k * p0.k + a2.k * q1.k + a3.k * q0.k;                        \
  z.k = pr * q.k;
    MR_LANE(x) MR_LANE(y) MR_LANE(z) MR_LANE(w)
#undef MR_LANE
    wpp[e] = w;
    x[e] = xn;
    qo[e] = q;
    zo[e] = z;
  }
}

template <typename T>
__global__ void mr_finish_kernel(const T *__restrict__ zo, const T *__restrict__ wpp,
                                 const T *__restrict__ wp, T *__restrict__ x,
                                 const double *__restrict__ st, int n, long long L, FastDiv fd) {
  __shared__ T cz[kMaxCols], ce[kMaxCols], cd[kMaxCols], cg[kMaxCols], ct[kMaxCols];
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    cz[c] = (T)st[kMrIbp * n + c];
    ce[c] = (T)st[kMrEps * n + c];
    cd[c] = (T)st[kMrDel * n + c];
    cg[c] = (T)st[kMrIg * n + c];
    ct[c] = (T)st[kMrT * n + c];
  }
  __syncthreads();
  GRID_STRIDE32(e, L * n) {
    const int c = (int)(e - fdiv(e, fd) * (uint32_t)n);
    const T w = (cz[c] * zo[e] - ce[c] * wpp[e] - cd[c] * wp[e]) * cg[c];
    x[e] += ct[c] * w;
  }
}

template <typename T>
__global__ void prec_apply_kernel(const T *__restrict__ r, const double *__restrict__ prec, int n,
                                  long long L, T *__restrict__ z, FastDiv fd) {
  GRID_STRIDE32(e, L * n) z[e] = (T)prec[fdiv(e, fd)] * r[e];
}

__global__ void scatter_cols_kernel(const double *__restrict__ Po, int no,
                                    const int *__restrict__ idx, double *__restrict__ P, int nv,
                                    long long L, FastDiv fd) {
  GRID_STRIDE32(e, L * no) {
    const uint32_t a = fdiv(e, fd);
    const int c = (int)(e - a * (uint32_t)no);
    P[(size_t)a * nv + idx[c]] = Po[e];
  }
}

template <typename TI, typename TO>
__global__ void add_convert_kernel(const TI *__restrict__ d, TO *__restrict__ p, long long n) {
  GRID_STRIDE32(i, n) p[i] = p[i] + (TO)d[i];
}

}  // namespace

cudaError_t launch_density(const double *X, int n, const double *occ, const double *mass,
                           long long L, double *rho, cudaStream_t s) {
  ::invdft::count_launch();
  density_kernel<<<grid_for(L), 256, 0, s>>>(X, n, occ, mass, L, rho);
  return cudaGetLastError();
}

cudaError_t launch_loss(const double *rho, const double *rd, const double *w, const double *mass,
                        long long L, double *out3, double *dLdrho, double *partial,
                        cudaStream_t s) {
  ::invdft::count_launch();
  loss_partial<<<kGramBlocks, 256, 0, s>>>(rho, rd, w, mass, L, partial, dLdrho);
  ::invdft::count_launch();
  sum3<<<1, 32, 0, s>>>(partial, kGramBlocks, out3);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(const double *X, int nv, const int *idx, int no, const double *f_o,
                               const double *dLdrho, const double *mass, long long L,
                               double *Psi_o, double *R, double *Wo, cudaStream_t s) {
  ::invdft::count_launch();
  adjoint_rhs_kernel<<<grid_for(L * no), 256, 0, s>>>(X, nv, idx, no, f_o, dLdrho, mass, L, Psi_o,
                                                      R, Wo, make_fastdiv(no));
  return cudaGetLastError();
}

template <typename TA, typename TB>
cudaError_t launch_pairdot(const TA *A, int lda, const int *ia, const TB *B, int ldb, const int *ib,
                           int npairs, long long L, double *coef, double *partial,
                           cudaStream_t s) {
  if (npairs < 1 || npairs > kMaxDense * kMaxGroup) return cudaErrorInvalidValue;
  dim3 grid(kGramBlocks, (npairs + 255) / 256);
  ::invdft::count_launch();
  pairdot_partial<TA, TB><<<grid, 256, 0, s>>>(A, lda, ia, B, ldb, ib, npairs, L, partial);
  ::invdft::count_launch();
  pair_sum<<<(npairs + 255) / 256, 256, 0, s>>>(partial, kGramBlocks, npairs, coef);
  return cudaGetLastError();
}
template cudaError_t launch_pairdot<double, double>(const double *, int, const int *,
                                                    const double *, int, const int *, int,
                                                    long long, double *, double *, cudaStream_t);
template cudaError_t launch_pairdot<double, float>(const double *, int, const int *, const float *,
                                                   int, const int *, int, long long, double *,
                                                   double *, cudaStream_t);

template <typename T>
cudaError_t launch_project_apply(const double *Psi, int ldp, const int *col_start, const int *ia,
                                 const double *coef, T *X, int ncol, long long L, cudaStream_t s) {
  ::invdft::count_launch();
  project_apply_kernel<T><<<grid_for(L * ncol), 256, 0, s>>>(Psi, ldp, col_start, ia, coef, -1.0,
                                                             X, ncol, L);
  return cudaGetLastError();
}
template cudaError_t launch_project_apply<double>(const double *, int, const int *, const int *,
                                                  const double *, double *, int, long long,
                                                  cudaStream_t);
template cudaError_t launch_project_apply<float>(const double *, int, const int *, const int *,
                                                 const double *, float *, int, long long,
                                                 cudaStream_t);

cudaError_t launch_add_along(const double *Psi_o, const int *col_start, const int *ia,
                             const double *dcoef, double *P, int n, long long L, cudaStream_t s) {
  ::invdft::count_launch();
  project_apply_kernel<double><<<grid_for(L * n), 256, 0, s>>>(Psi_o, n, col_start, ia, dcoef, 1.0,
                                                               P, n, L);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const double *P, const double *Psi, int ncol, const double *rd,
                            double tau, long long L, double *grad, cudaStream_t s) {
  ::invdft::count_launch();
  gradient_kernel<<<grid_for(L), 256, 0, s>>>(P, Psi, ncol, rd, tau, L, grad);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double *x, const double *y, long long n, double *out, double *partial,
                       cudaStream_t s) {
  ::invdft::count_launch();
  dot_partial<<<kGramBlocks, 256, 0, s>>>(x, y, n, partial);
  ::invdft::count_launch();
  reduce_partials<<<1, 32, 0, s>>>(partial, kGramBlocks, 0, out);
  return cudaGetLastError();
}
cudaError_t launch_absmax(const double *x, long long n, double *out, double *partial,
                          cudaStream_t s) {
  ::invdft::count_launch();
  absmax_partial<<<kGramBlocks, 256, 0, s>>>(x, n, partial);
  ::invdft::count_launch();
  reduce_partials<<<1, 32, 0, s>>>(partial, kGramBlocks, 1, out);
  return cudaGetLastError();
}
cudaError_t launch_axpby(double a, const double *x, double b, double *y, long long n,
                         cudaStream_t s) {
  ::invdft::count_launch();
  axpby_kernel<<<grid_for(n), 256, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}
cudaError_t launch_lincomb(double a, const double *x, double b, const double *y, double *out,
                           long long n, cudaStream_t s) {
  ::invdft::count_launch();
  lincomb_kernel<<<grid_for(n), 256, 0, s>>>(a, x, b, y, out, n);
  return cudaGetLastError();
}
cudaError_t launch_residual_block(const double *HX, const double *X, const double *theta, int n,
                                  long long L, double *E64, float *E32, cudaStream_t s) {
  ::invdft::count_launch();
  residual_block_kernel<<<grid_for(L * n), 256, 0, s>>>(HX, X, theta, n, L, E64, E32,
                                                        make_fastdiv(n));
  return cudaGetLastError();
}
cudaError_t launch_cheb_combine(const double *X, const double *pm, const float *D, int n,
                                long long L, double *Y, cudaStream_t s) {
  ::invdft::count_launch();
  cheb_combine_kernel<<<grid_for(L * n), 256, 0, s>>>(X, pm, D, n, L, Y, make_fastdiv(n));
  return cudaGetLastError();
}
cudaError_t launch_scale_f32(const float *E, const double *, double alpha, int n, long long L,
                             float *D, cudaStream_t s) {
  ::invdft::count_launch();
  scale_f32_kernel<<<grid_for(L * n), 256, 0, s>>>(E, alpha, n, L, D);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mr_step(const T *ph, const T *qh, T *qo, T *zo, T *wpp, const T *wp, T *x,
                           double *st, const double *prec, const float *precf, int n, long long L,
                           cudaStream_t s) {
  ::invdft::count_launch();
  if (sizeof(T) == 4 && n % 4 == 0) {
    const int n4 = n / 4;
    mr_step_vec4_kernel<<<grid_for(L * n4), 256, 0, s>>>(
        reinterpret_cast<const float4 *>(ph), reinterpret_cast<const float4 *>(qh),
        reinterpret_cast<float4 *>(qo), reinterpret_cast<float4 *>(zo),
        reinterpret_cast<float4 *>(wpp), reinterpret_cast<const float4 *>(wp),
        reinterpret_cast<float4 *>(x), st, precf, n, L, make_fastdiv(n4));
    return cudaGetLastError();
  }
  mr_step_kernel<T><<<grid_for(L * n), 256, 0, s>>>(ph, qh, qo, zo, wpp, wp, x, st, prec, n, L,
                                                    make_fastdiv(n));
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_mr_finish(const T *zo, T *wpp, const T *wp, T *x, const double *st, int n,
                             long long L, cudaStream_t s) {
  ::invdft::count_launch();
  mr_finish_kernel<T><<<grid_for(L * n), 256, 0, s>>>(zo, wpp, wp, x, st, n, L, make_fastdiv(n));
  return cudaGetLastError();
}
cudaError_t launch_mr_givens(int n, double *st, cudaStream_t s) {
  ::invdft::count_launch();
  mr_givens_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, st);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prec_apply(const T *r, const double *prec, int n, long long L, T *z,
                              cudaStream_t s) {
  ::invdft::count_launch();
  prec_apply_kernel<T><<<grid_for(L * n), 256, 0, s>>>(r, prec, n, L, z, make_fastdiv(n));
  return cudaGetLastError();
}
cudaError_t launch_scatter_cols(const double *Po, int no, const int *idx, double *P, int nv,
                                long long L, cudaStream_t s) {
  ::invdft::count_launch();
  scatter_cols_kernel<<<grid_for(L * no), 256, 0, s>>>(Po, no, idx, P, nv, L, make_fastdiv(no));
  return cudaGetLastError();
}
template <typename TI, typename TO>
cudaError_t launch_add_convert(const TI *d, TO *p, long long n, cudaStream_t s) {
  ::invdft::count_launch();
  add_convert_kernel<TI, TO><<<grid_for(n), 256, 0, s>>>(d, p, n);
  return cudaGetLastError();
}

#define INST_MR(T)                                                                              \
  template cudaError_t launch_mr_step<T>(const T *, const T *, T *, T *, T *, const T *, T *,    \
                                         double *, const double *, const float *, int, long long, \
                                         cudaStream_t);                                          \
  template cudaError_t launch_mr_finish<T>(const T *, T *, const T *, T *, const double *, int,  \
                                           long long, cudaStream_t);                             \
  template cudaError_t launch_prec_apply<T>(const T *, const double *, int, long long, T *,     \
                                            cudaStream_t);
INST_MR(double)
INST_MR(float)
template cudaError_t launch_add_convert<float, double>(const float *, double *, long long,
                                                       cudaStream_t);
template cudaError_t launch_add_convert<double, double>(const double *, double *, long long,
                                                        cudaStream_t);

}  // namespace invdft
