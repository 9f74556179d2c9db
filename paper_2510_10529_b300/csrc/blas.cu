// Tall-skinny block kernels: Gram matrices, rotations, column dot products and
// conversions over node-major [L][n] blocks.  All reductions accumulate in
// FP64 and sum per-CTA partials in a fixed order, so results are bitwise
// reproducible run to run.
#include "internal.h"

namespace invdft {
namespace {

constexpr int kTile = 64;    // Gram output tile (kTile x kTile per CTA column)
constexpr int kRows = 32;    // rows staged per step

// partial[b][i][j] over the rows owned by CTA b, for the (ty, tx) output tile.
template <typename TA, typename TC>
__global__ void __launch_bounds__(256) gram_partial(const TA *__restrict__ A, int n1,
                                                    const TA *__restrict__ B, int n2, long long L,
                                                    double *__restrict__ partial) {
  __shared__ TC sA[kRows][kTile + 1];
  __shared__ TC sB[kRows][kTile + 1];
  const int tid = threadIdx.x;
  const int ti = tid / 16, tj = tid % 16;
  const int i0 = blockIdx.y * kTile, j0 = blockIdx.z * kTile;
  TC acc[4][4] = {};
  const long long rows_per = (L + gridDim.x - 1) / gridDim.x;
  const long long r_begin = blockIdx.x * rows_per;
  const long long r_end = min(L, r_begin + rows_per);
  for (long long r0 = r_begin; r0 < r_end; r0 += kRows) {
    for (int idx = tid; idx < kRows * kTile; idx += 256) {
      const int r = idx / kTile, c = idx % kTile;
      const long long row = r0 + r;
      const bool ok = row < r_end;
      sA[r][c] = (ok && i0 + c < n1) ? (TC)A[row * n1 + i0 + c] : (TC)0;
      sB[r][c] = (ok && j0 + c < n2) ? (TC)B[row * n2 + j0 + c] : (TC)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kRows; ++r) {
      TC a[4], b[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        a[k] = sA[r][ti * 4 + k];
        b[k] = sB[r][tj * 4 + k];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  double *out = partial + (size_t)blockIdx.x * n1 * n2;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + ti * 4 + x, j = j0 + tj * 4 + y;
      if (i < n1 && j < n2) out[i * n2 + j] = (double)acc[x][y];
    }
}

__global__ void sum_partials(const double *__restrict__ partial, int nblk, int n1, int n2,
                             double *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n1 * n2) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * n1 * n2 + e];
  G[e] = s;
}

template <typename TA, typename TC>
cudaError_t gram_t(const TA *A, int n1, const TA *B, int n2, long long L, double *G,
                   double *partial, cudaStream_t s) {
  if (n1 < 1 || n2 < 1 || n1 > kMaxGram || n2 > kMaxGram) return cudaErrorInvalidValue;
  dim3 grid(kGramBlocks, (n1 + kTile - 1) / kTile, (n2 + kTile - 1) / kTile);
  ::invdft::count_launch();
  gram_partial<TA, TC><<<grid, 256, 0, s>>>(A, n1, B, n2, L, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  sum_partials<<<(n1 * n2 + 255) / 256, 256, 0, s>>>(partial, kGramBlocks, n1, n2, G);
  return cudaGetLastError();
}

// Xo[a][j] = sum_i Xi[a][i] Cm[i][j]; Cm staged in shared memory.
__global__ void __launch_bounds__(256) rotate_kernel(const double *__restrict__ Xi, int n1,
                                                     const double *__restrict__ Cm, int n2,
                                                     long long L, double *__restrict__ Xo) {
  extern __shared__ double sm[];
  double *sC = sm;                         // n1 * n2
  double *sX = sm + n1 * n2;               // rows_per_pass * n1
  const int tid = threadIdx.x;
  for (int e = tid; e < n1 * n2; e += 256) sC[e] = Cm[e];
  const int rpp = max(1, 256 / n2);        // rows per pass
  const int r = tid / n2, j = tid % n2;
  for (long long a0 = (long long)blockIdx.x * rpp; a0 < L; a0 += (long long)gridDim.x * rpp) {
    __syncthreads();
    for (int e = tid; e < rpp * n1; e += 256) {
      const int rr = e / n1, i = e % n1;
      const long long a = a0 + rr;
      sX[rr * n1 + i] = a < L ? Xi[a * n1 + i] : 0.0;
    }
    __syncthreads();
    if (r < rpp) {
      const long long a = a0 + r;
      if (a < L) {
        double s = 0.0;
        for (int i = 0; i < n1; ++i) s = fma(sX[r * n1 + i], sC[i * n2 + j], s);
        Xo[a * n2 + j] = s;
      }
    }
  }
}

// Xo[a][j] += alpha * sum_i Xi[a][i] Cm[i][j]  (storage and arithmetic in T)
template <typename T>
__global__ void __launch_bounds__(256) rotate_acc_kernel(const T *__restrict__ Xi, int n1,
                                                         const double *__restrict__ Cm, int n2,
                                                         long long L, T *__restrict__ Xo,
                                                         double alpha) {
  extern __shared__ unsigned char sm_raw[];
  T *sC = reinterpret_cast<T *>(sm_raw);   // n1 * n2
  T *sX = sC + n1 * n2;                     // rows_per_pass * n1
  const int tid = threadIdx.x;
  for (int e = tid; e < n1 * n2; e += 256) sC[e] = (T)(alpha * Cm[e]);
  const int rpp = max(1, 256 / n2);
  const int r = tid / n2, j = tid % n2;
  for (long long a0 = (long long)blockIdx.x * rpp; a0 < L; a0 += (long long)gridDim.x * rpp) {
    __syncthreads();
    for (int e = tid; e < rpp * n1; e += 256) {
      const int rr = e / n1, i = e % n1;
      const long long a = a0 + rr;
      sX[rr * n1 + i] = a < L ? Xi[a * n1 + i] : (T)0;
    }
    __syncthreads();
    if (r < rpp) {
      const long long a = a0 + r;
      if (a < L) {
        T s = 0;
        for (int i = 0; i < n1; ++i) s = fma(sX[r * n1 + i], sC[i * n2 + j], s);
        Xo[a * n2 + j] += s;
      }
    }
  }
}

template <typename TA>
__global__ void __launch_bounds__(256) coldot_partial(const TA *__restrict__ A,
                                                      const TA *__restrict__ B, int ncol,
                                                      long long L, double *__restrict__ partial) {
  __shared__ double red[256];
  const int tid = threadIdx.x;
  const int R = 256 / ncol;
  const int j = tid % ncol, r0 = tid / ncol;
  double s = 0.0;
  if (r0 < R) {
    for (long long a = (long long)blockIdx.x * R + r0; a < L; a += (long long)gridDim.x * R)
      s += (double)A[a * ncol + j] * (double)B[a * ncol + j];
  }
  red[tid] = s;
  __syncthreads();
  if (tid < ncol) {
    double t = 0.0;
    for (int r = 0; r < R; ++r) t += red[r * ncol + tid];
    partial[(size_t)blockIdx.x * kMaxCols + tid] = t;
  }
}

__global__ void sum_col_partials(const double *__restrict__ partial, int nblk, int ncol,
                                 double *__restrict__ d) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ncol) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * kMaxCols + j];
  d[j] = s;
}

template <typename TA>
cudaError_t coldot_t(const TA *A, const TA *B, int ncol, long long L, double *d, double *partial,
                     cudaStream_t s) {
  if (ncol < 1 || ncol > kMaxCols) return cudaErrorInvalidValue;
  ::invdft::count_launch();
  coldot_partial<TA><<<kGramBlocks, 256, 0, s>>>(A, B, ncol, L, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  sum_col_partials<<<(ncol + 127) / 128, 128, 0, s>>>(partial, kGramBlocks, ncol, d);
  return cudaGetLastError();
}

__global__ void gather_cols_kernel(const double *__restrict__ X, int nv, const int *__restrict__ idx,
                                   int n, long long L, double *__restrict__ Out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < L * n;
       e += (long long)gridDim.x * blockDim.x) {
    const long long a = e / n;
    Out[e] = X[a * nv + idx[e - a * n]];
  }
}

__global__ void conv_d2f(const double *__restrict__ x, float *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void conv_f2d(const float *__restrict__ x, double *__restrict__ y, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}

// Counter-based normal draws: splitmix64 of (seed, index) -> two uniforms ->
// Box-Muller.  Only the reproducibility of the start block matters.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
__global__ void fill_normal(double *__restrict__ X, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long h1 = splitmix64(seed * 0x100000001B3ULL + 2 * (unsigned long long)i);
    const unsigned long long h2 = splitmix64(h1 ^ (2 * (unsigned long long)i + 1));
    const double u1 = ((h1 >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    X[i] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 16); }

}  // namespace

cudaError_t launch_gram(const double *A, int n1, const double *B, int n2, long long L, double *G,
                        double *partial, cudaStream_t s) {
  return gram_t<double, double>(A, n1, B, n2, L, G, partial, s);
}
cudaError_t launch_gram_f32(const float *A, int n1, const float *B, int n2, long long L,
                            double *G, double *partial, cudaStream_t s) {
  return gram_t<float, double>(A, n1, B, n2, L, G, partial, s);
}
cudaError_t launch_rotate(const double *Xi, int n1, const double *Cm, int n2, long long L,
                          double *Xo, cudaStream_t s) {
  if (n1 < 1 || n2 < 1 || n1 > kMaxGram || n2 > kMaxGram) return cudaErrorInvalidValue;
  const int rpp = std::max(1, 256 / n2);
  const size_t smem = sizeof(double) * ((size_t)n1 * n2 + (size_t)rpp * n1);
  cudaError_t e = cudaFuncSetAttribute(rotate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  rotate_kernel<<<148 * 4, 256, smem, s>>>(Xi, n1, Cm, n2, L, Xo);
  return cudaGetLastError();
}
cudaError_t launch_gram_f32acc(const float *A, int n1, const float *B, int n2, long long L,
                               double *G, double *partial, cudaStream_t s) {
  return gram_t<float, float>(A, n1, B, n2, L, G, partial, s);
}
template <typename T>
cudaError_t launch_rotate_acc(const T *Xi, int n1, const double *Cm, int n2, long long L, T *Xo,
                              double alpha, cudaStream_t s) {
  if (n1 < 1 || n2 < 1 || n1 > kMaxGram || n2 > kMaxGram) return cudaErrorInvalidValue;
  const int rpp = std::max(1, 256 / n2);
  const size_t smem = sizeof(T) * ((size_t)n1 * n2 + (size_t)rpp * n1);
  cudaError_t e = cudaFuncSetAttribute(rotate_acc_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  rotate_acc_kernel<T><<<148 * 4, 256, smem, s>>>(Xi, n1, Cm, n2, L, Xo, alpha);
  return cudaGetLastError();
}
template cudaError_t launch_rotate_acc<double>(const double *, int, const double *, int, long long,
                                               double *, double, cudaStream_t);
template cudaError_t launch_rotate_acc<float>(const float *, int, const double *, int, long long,
                                              float *, double, cudaStream_t);
cudaError_t launch_coldot(const double *A, const double *B, int ncol, long long L, double *d,
                          double *partial, cudaStream_t s) {
  return coldot_t<double>(A, B, ncol, L, d, partial, s);
}
cudaError_t launch_coldot_f32(const float *A, const float *B, int ncol, long long L, double *d,
                              double *partial, cudaStream_t s) {
  return coldot_t<float>(A, B, ncol, L, d, partial, s);
}
cudaError_t launch_gather_cols(const double *X, int nv, const int *idx, int n, long long L,
                               double *Out, cudaStream_t s) {
  ::invdft::count_launch();
  gather_cols_kernel<<<grid_for(L * n), 256, 0, s>>>(X, nv, idx, n, L, Out);
  return cudaGetLastError();
}
cudaError_t launch_convert_f64_to_f32(const double *x, float *y, long long n, cudaStream_t s) {
  ::invdft::count_launch();
  conv_d2f<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_convert_f32_to_f64(const float *x, double *y, long long n, cudaStream_t s) {
  ::invdft::count_launch();
  conv_f2d<<<grid_for(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_fill_random(double *X, long long n, unsigned long long seed, cudaStream_t s) {
  ::invdft::count_launch();
  fill_normal<<<grid_for(n), 256, 0, s>>>(X, n, seed);
  return cudaGetLastError();
}

}  // namespace invdft
