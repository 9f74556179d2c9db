// Small dense FP64 kernels on the N_v x N_v subspace, one CTA each:
//   * Rayleigh-Ritz (Sec. 3.2.2, Eq. 23-24): Cholesky S_Y = L L^T, the standard
//     problem L^-1 H_Y L^-T v = eps v by cyclic parallel Jacobi rotations, and
//     the coefficient matrix C = L^-T V with X <- Y C.
//   * Fermi-Dirac occupations and the chemical potential (Eq. 4-5).
// The overlap is first scaled to unit diagonal (S' = D S D) so that the
// Cholesky works on a correlation matrix whatever the column norms of Y.
#include "internal.h"
#include "solvers.h"

namespace invdft {
namespace {

__global__ void __launch_bounds__(1024) rr_small(const double *__restrict__ S,
                                                 const double *__restrict__ H, int n,
                                                 double *__restrict__ theta,
                                                 double *__restrict__ Cout, int *__restrict__ status,
                                                 double *__restrict__ Lm, double *__restrict__ W,
                                                 int max_sweeps) {
  extern __shared__ double sm[];
  double *A = sm;               // n*n
  double *V = sm + n * n;       // n*n
  __shared__ double ds[kMaxDense];
  __shared__ double pc[kMaxDense / 2 + 1], ps[kMaxDense / 2 + 1];
  __shared__ int pp[kMaxDense / 2 + 1], pq[kMaxDense / 2 + 1];
  __shared__ int rank[kMaxDense];
  __shared__ int fail;
  __shared__ double red_off[32], red_all[32];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) fail = 0;
  __syncthreads();
  if (tid < n) {
    const double d = S[tid * n + tid];
    if (!(d > 0.0)) fail = 1;
    ds[tid] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  __syncthreads();
  if (fail) {
    if (tid == 0) status[0] = 1;
    return;
  }
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    Lm[e] = 0.5 * (S[e] + S[j * n + i]) * ds[i] * ds[j];
    A[e] = 0.5 * (H[e] + H[j * n + i]) * ds[i] * ds[j];
  }
  __syncthreads();
  // Cholesky, right-looking, lower triangle of Lm
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const double piv = Lm[k * n + k];
      if (!(piv > 1e-13)) fail = 1;
      Lm[k * n + k] = piv > 0.0 ? sqrt(piv) : 1.0;
    }
    __syncthreads();
    if (fail) break;
    const double lkk = Lm[k * n + k];
    for (int i = k + 1 + tid; i < n; i += nt) Lm[i * n + k] /= lkk;
    __syncthreads();
    const int m = n - k - 1;
    for (int e = tid; e < m * m; e += nt) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      if (j <= i) Lm[i * n + j] -= Lm[i * n + k] * Lm[j * n + k];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) status[0] = 1;
    return;
  }
  // W = L^-1 A (column c by forward substitution), then A <- L^-1 W^T
  for (int c = tid; c < n; c += nt) {
    for (int i = 0; i < n; ++i) {
      double s = A[i * n + c];
      for (int k = 0; k < i; ++k) s -= Lm[i * n + k] * W[k * n + c];
      W[i * n + c] = s / Lm[i * n + i];
    }
  }
  __syncthreads();
  for (int c = tid; c < n; c += nt) {
    for (int i = 0; i < n; ++i) {
      double s = W[c * n + i];
      for (int k = 0; k < i; ++k) s -= Lm[i * n + k] * V[k * n + c];
      V[i * n + c] = s / Lm[i * n + i];       // V used as scratch here
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    A[e] = 0.5 * (V[i * n + j] + V[j * n + i]);
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) V[e] = (e / n == e % n) ? 1.0 : 0.0;
  __syncthreads();

  // cyclic Jacobi with the round-robin (circle) ordering: m/2 disjoint pairs per round
  const int m = (n % 2) ? n + 1 : n;
  const int half = m / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const double a2 = A[e] * A[e];
      all += a2;
      if (e / n != e % n) off += a2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      all += __shfl_down_sync(0xffffffffu, all, o);
    }
    if ((tid & 31) == 0) {
      red_off[tid >> 5] = off;
      red_all[tid >> 5] = all;
    }
    __syncthreads();
    if (tid == 0) {
      double so = 0.0, sa = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        so += red_off[w];
        sa += red_all[w];
      }
      done = (so <= 1e-30 * sa) || so == 0.0;
    }
    __syncthreads();
    if (done) break;
    for (int r = 0; r < m - 1; ++r) {
      if (tid < half) {
        const int k = tid;
        int p = (k == 0) ? 0 : 1 + ((k - 1 + r) % (m - 1));
        const int kk = m - 1 - k;
        int q = 1 + ((kk - 1 + r) % (m - 1));
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[p * n + q];
          if (apq != 0.0) {
            const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pp[k] = p;
        pq[k] = q;
        pc[k] = c;
        ps[k] = s;
      }
      __syncthreads();
      for (int e = tid; e < n * half; e += nt) {      // columns: A <- A J, V <- V J
        const int i = e / half, k = e % half;
        const int p = pp[k], q = pq[k];
        if (q >= n || ps[k] == 0.0) continue;
        const double c = pc[k], s = ps[k];
        const double aip = A[i * n + p], aiq = A[i * n + q];
        A[i * n + p] = c * aip - s * aiq;
        A[i * n + q] = s * aip + c * aiq;
        const double vip = V[i * n + p], viq = V[i * n + q];
        V[i * n + p] = c * vip - s * viq;
        V[i * n + q] = s * vip + c * viq;
      }
      __syncthreads();
      for (int e = tid; e < n * half; e += nt) {      // rows: A <- J^T A
        const int j = e / half, k = e % half;
        const int p = pp[k], q = pq[k];
        if (q >= n || ps[k] == 0.0) continue;
        const double c = pc[k], s = ps[k];
        const double apj = A[p * n + j], aqj = A[q * n + j];
        A[p * n + j] = c * apj - s * aqj;
        A[q * n + j] = s * apj + c * aqj;
      }
      __syncthreads();
    }
  }
  // ascending order
  if (tid < n) {
    const double li = A[tid * n + tid];
    int rk = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = A[j * n + j];
      if (lj < li || (lj == li && j < tid)) ++rk;
    }
    rank[tid] = rk;
    theta[rk] = li;
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    W[i * n + rank[j]] = V[e];
  }
  __syncthreads();
  // C = D_s L^-T V (backward substitution per column)
  for (int c = tid; c < n; c += nt) {
    for (int i = n - 1; i >= 0; --i) {
      double s = W[i * n + c];
      for (int k = i + 1; k < n; ++k) s -= Lm[k * n + i] * V[k * n + c];
      V[i * n + c] = s / Lm[i * n + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) Cout[e] = ds[e / n] * V[e];
  if (tid == 0) status[0] = 0;
}

// Occupations f_i = 2 / (1 + exp((eps_i - mu)/kT)), mu by bisection on
// sum f = N_e; f'_i = df_i/deps_i.  kT = 0: the lowest N_e/2 states hold 2.
__global__ void occupations_kernel(const double *__restrict__ eps, int n, double ne, double kT,
                                   double *__restrict__ f, double *__restrict__ dfde,
                                   double *__restrict__ mu_out, int *__restrict__ status) {
  const int lane = threadIdx.x;
  if (kT <= 0.0) {
    const int nocc = (int)llround(ne / 2.0);
    for (int i = lane; i < n; i += 32) {
      f[i] = i < nocc ? 2.0 : 0.0;
      dfde[i] = 0.0;
    }
    if (lane == 0) {
      mu_out[0] = nocc <= 0 ? eps[0] : (nocc < n ? 0.5 * (eps[nocc - 1] + eps[nocc]) : eps[n - 1]);
      status[1] = (nocc > n || fabs(2.0 * nocc - ne) > 1e-12) ? 1 : 0;
    }
    return;
  }
  double lo = eps[0], hi = eps[0];
  for (int i = 0; i < n; ++i) {
    lo = fmin(lo, eps[i]);
    hi = fmax(hi, eps[i]);
  }
  lo -= 50.0 * kT + 1.0;
  hi += 50.0 * kT + 1.0;
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += 2.0 / (1.0 + exp((eps[i] - mid) / kT));
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (s < ne) lo = mid; else hi = mid;
    if (hi - lo <= 4e-16 * fmax(1.0, fabs(mid))) break;
  }
  const double mu = 0.5 * (lo + hi);
  for (int i = lane; i < n; i += 32) {
    const double sx = 1.0 / (1.0 + exp((eps[i] - mu) / kT));
    f[i] = 2.0 * sx;
    dfde[i] = -(2.0 / kT) * sx * (1.0 - sx);
  }
  if (lane == 0) {
    mu_out[0] = mu;
    status[1] = 0;
  }
}

}  // namespace

cudaError_t launch_rr_small(const double *S, const double *H, int n, double *theta, double *C,
                            int *status, double *work, cudaStream_t s) {
  if (n < 1 || n > kMaxDense) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)n * n * sizeof(double);
  cudaError_t e = raise_smem_limit(rr_small, (int)smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  rr_small<<<1, 1024, smem, s>>>(S, H, n, theta, C, status, work, work + (size_t)n * n, 60);
  return cudaGetLastError();
}

cudaError_t launch_occupations(const double *eps, int n, double ne, double kT, double *f,
                               double *dfde, double *mu, int *status, cudaStream_t s) {
  ::invdft::count_launch();
  occupations_kernel<<<1, 32, 0, s>>>(eps, n, ne, kT, f, dfde, mu, status);
  return cudaGetLastError();
}

}  // namespace invdft
