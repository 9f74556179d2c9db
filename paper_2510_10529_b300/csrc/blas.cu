// Tall-skinny block kernels: Gram matrices, rotations, column dot products and
// conversions over node-major [L][n] blocks.  All reductions accumulate in
// FP64 and sum per-CTA partials in a fixed order, so results are bitwise
// reproducible run to run.
#include "internal.h"

namespace invdft {
namespace {

constexpr int kTile = 64;    // Gram output tile (kTile x kTile per CTA column)
constexpr int kColdotBlocks = 148 * 8;   // column-dot partials (more CTAs in flight)
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

// out[e] = sum_b partial[b * stride + e]: one warp per output, lanes take the
// blocks b = lane (mod 32), then a fixed shuffle tree (bitwise reproducible)
__global__ void warp_sum_partials(const double *__restrict__ partial, int nblk, size_t stride,
                                  int n, double *__restrict__ out) {
  const int e = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (e >= n) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[(size_t)b * stride + e];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[e] = s;
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
  warp_sum_partials<<<(n1 * n2 + 7) / 8, 256, 0, s>>>(partial, kGramBlocks, (size_t)n1 * n2,
                                                      n1 * n2, G);
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
    const long long step = (long long)gridDim.x * R;
    long long a = (long long)blockIdx.x * R + r0;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (; a + 3 * step < L; a += 4 * step) {
      const TA x0 = A[a * ncol + j], x1 = A[(a + step) * ncol + j];
      const TA x2 = A[(a + 2 * step) * ncol + j], x3 = A[(a + 3 * step) * ncol + j];
      const TA y0 = B[a * ncol + j], y1 = B[(a + step) * ncol + j];
      const TA y2 = B[(a + 2 * step) * ncol + j], y3 = B[(a + 3 * step) * ncol + j];
      s += (double)x0 * (double)y0;
      s1 += (double)x1 * (double)y1;
      s2 += (double)x2 * (double)y2;
      s3 += (double)x3 * (double)y3;
    }
    for (; a < L; a += step) s += (double)A[a * ncol + j] * (double)B[a * ncol + j];
    s += (s1 + s2) + s3;
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
  coldot_partial<TA><<<kColdotBlocks, 256, 0, s>>>(A, B, ncol, L, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  warp_sum_partials<<<(ncol + 7) / 8, 256, 0, s>>>(partial, kColdotBlocks, kMaxCols, ncol, d);
  return cudaGetLastError();
}

__global__ void gather_cols_kernel(const double *__restrict__ X, int nv, const int *__restrict__ idx,
                                   int n, long long L, double *__restrict__ Out, FastDiv fd) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < (uint32_t)(L * n);
       e += gridDim.x * blockDim.x) {
    const uint32_t a = fdiv(e, fd);
    Out[e] = X[(size_t)a * nv + idx[e - a * (uint32_t)n]];
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

template <typename T, typename TA>
cudaError_t launch_stripe_gram(const T *A, int n1, const T *B, int n2, long long L, double *G,
                               double *partial, cudaStream_t s);

cudaError_t launch_gram(const double *A, int n1, const double *B, int n2, long long L, double *G,
                        double *partial, cudaStream_t s) {
  if (n1 <= 64 && n2 <= 64) return launch_stripe_gram<double, double>(A, n1, B, n2, L, G, partial, s);
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
  cudaError_t e = raise_smem_limit(rotate_kernel, (int)smem);
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
  cudaError_t e = raise_smem_limit(rotate_acc_kernel<T>, (int)smem);
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
  gather_cols_kernel<<<grid_for(L * n), 256, 0, s>>>(X, nv, idx, n, L, Out, make_fastdiv(n));
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


// ---------------------------------------------------------------------------
// Row-striped tall-skinny Gram for any n1, n2 <= 64: a thread owns a 4x4
// output tile; when the n1 x n2 output has fewer tiles than the CTA has
// threads, the spare threads split the rows of each staged chunk ("stripes")
// and the stripes are summed in shared memory at the end.  T is the storage
// type, TA the accumulator (FP32 for the MINRES deflation, FP64 otherwise).
namespace invdft {
namespace {

constexpr int kSgRows = 32;

template <typename T, typename TA>
__global__ void __launch_bounds__(256) stripe_gram(const T *__restrict__ A, int n1,
                                                   const T *__restrict__ B, int n2, long long L,
                                                   double *__restrict__ partial) {
  extern __shared__ __align__(16) unsigned char sg_raw[];
  T *sA = reinterpret_cast<T *>(sg_raw);                       // [2][kSgRows][n1]
  T *sB = sA + 2 * kSgRows * n1;                               // [2][kSgRows][n2]
  const int tid = threadIdx.x;
  const int ntj = (n2 + 3) / 4, tiles = ((n1 + 3) / 4) * ntj;
  const int S = max(1, 256 / tiles);
  const int tile = tid % tiles, stripe = tid / tiles;
  const bool active = stripe < S && tid < S * tiles;
  const int i0 = (tile / ntj) * 4, j0 = (tile % ntj) * 4;
  const long long rows_per = ((L + gridDim.x - 1) / gridDim.x + kSgRows - 1) / kSgRows * kSgRows;
  const long long r_begin = blockIdx.x * rows_per;
  const long long r_end = min(L, r_begin + rows_per);
  TA acc[4][4] = {};
  auto stage = [&](int buf, long long r0) {
    const int rows = (int)min((long long)kSgRows, r_end - r0);
    T *da = sA + buf * kSgRows * n1;
    T *db = sB + buf * kSgRows * n2;
    for (int e = tid; e < kSgRows * n1; e += 256) {
      if (e < rows * n1) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                     :: "r"((unsigned)__cvta_generic_to_shared(da + e)), "l"(A + r0 * n1 + e),
                        "n"(sizeof(T)) : "memory");
      } else {
        da[e] = (T)0;
      }
    }
    for (int e = tid; e < kSgRows * n2; e += 256) {
      if (e < rows * n2) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                     :: "r"((unsigned)__cvta_generic_to_shared(db + e)), "l"(B + r0 * n2 + e),
                        "n"(sizeof(T)) : "memory");
      } else {
        db[e] = (T)0;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  if (r_begin < r_end) stage(0, r_begin);
  for (long long r0 = r_begin; r0 < r_end; r0 += kSgRows) {
    const bool more = r0 + kSgRows < r_end;
    if (more) {
      stage(buf ^ 1, r0 + kSgRows);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    if (active) {
      const T *ra = sA + buf * kSgRows * n1;
      const T *rb = sB + buf * kSgRows * n2;
      for (int r = stripe; r < kSgRows; r += S) {
        TA av[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          av[x] = i0 + x < n1 ? (TA)ra[r * n1 + i0 + x] : (TA)0;
          bv[x] = j0 + x < n2 ? (TA)rb[r * n2 + j0 + x] : (TA)0;
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(av[x], bv[y], acc[x][y]);
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  // sum the stripes (reuse the staging area)
  TA *red = reinterpret_cast<TA *>(sg_raw);                    // [S][tiles][16]
  if (active)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) red[((size_t)stripe * tiles + tile) * 16 + x * 4 + y] = acc[x][y];
  __syncthreads();
  double *out = partial + (size_t)blockIdx.x * n1 * n2;
  for (int e = tid; e < tiles * 16; e += 256) {
    const int tl = e / 16, xy = e % 16;
    const int i = (tl / ntj) * 4 + xy / 4, j = (tl % ntj) * 4 + xy % 4;
    if (i >= n1 || j >= n2) continue;
    double s = 0.0;
    for (int st = 0; st < S; ++st) s += (double)red[((size_t)st * tiles + tl) * 16 + xy];
    out[i * n2 + j] = s;
  }
}

// Z[a][j] += sum_i Psi[a][i] Cf[i][j]: a thread owns one row and NJ columns
template <typename T, int NJ>
__global__ void __launch_bounds__(256) stripe_rotate(const T *__restrict__ Psi, int n1,
                                                     const double *__restrict__ C, int n2,
                                                     long long L, T *__restrict__ Z,
                                                     double alpha) {
  extern __shared__ __align__(16) unsigned char sr_raw[];
  const int ncg = (n2 + NJ - 1) / NJ;
  const int rows_blk = 256 / ncg;
  T *sC = reinterpret_cast<T *>(sr_raw);                       // [n1][ncg * NJ]
  T *sP = sC + n1 * ncg * NJ;                                  // [rows_blk][n1 + 1]
  const int tid = threadIdx.x;
  const int ldc = ncg * NJ;
  for (int e = tid; e < n1 * ldc; e += 256) {
    const int i = e / ldc, j = e % ldc;
    sC[e] = j < n2 ? (T)(alpha * C[i * n2 + j]) : (T)0;
  }
  const int cg = tid % ncg, r = tid / ncg;
  const bool active = r < rows_blk;
  for (long long a0 = (long long)blockIdx.x * rows_blk; a0 < L;
       a0 += (long long)gridDim.x * rows_blk) {
    __syncthreads();
    const int rows = (int)min((long long)rows_blk, L - a0);
    for (int e = tid; e < rows * n1; e += 256) {
      const int rr = e / n1, i = e - rr * n1;
      sP[rr * (n1 + 1) + i] = Psi[(a0 + rr) * n1 + i];
    }
    __syncthreads();
    if (!active || r >= rows) continue;
    T acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = (T)0;
    for (int i = 0; i < n1; ++i) {
      const T psi = sP[r * (n1 + 1) + i];
#pragma unroll
      for (int j = 0; j < NJ; ++j) acc[j] = fma(psi, sC[i * ldc + cg * NJ + j], acc[j]);
    }
    T *zr = Z + (a0 + r) * n2 + cg * NJ;
#pragma unroll
    for (int j = 0; j < NJ; ++j)
      if (cg * NJ + j < n2) zr[j] += acc[j];
  }
}

}  // namespace

template <typename T, typename TA>
cudaError_t launch_stripe_gram(const T *A, int n1, const T *B, int n2, long long L, double *G,
                               double *partial, cudaStream_t s) {
  if (n1 < 1 || n2 < 1 || n1 > 64 || n2 > 64) return cudaErrorInvalidValue;
  const int tiles = ((n1 + 3) / 4) * ((n2 + 3) / 4);
  const int S = std::max(1, 256 / tiles);
  const size_t stage = 2 * (size_t)kSgRows * (n1 + n2) * sizeof(T);
  const size_t red = (size_t)S * tiles * 16 * sizeof(TA);
  const size_t smem = std::max(stage, red);
  cudaError_t e = raise_smem_limit(stripe_gram<T, TA>, smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  stripe_gram<T, TA><<<kGramBlocks, 256, smem, s>>>(A, n1, B, n2, L, partial);
  ::invdft::count_launch();
  warp_sum_partials<<<(n1 * n2 + 7) / 8, 256, 0, s>>>(partial, kGramBlocks, (size_t)n1 * n2,
                                                      n1 * n2, G);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_stripe_rotate(const T *Psi, int n1, const double *C, int n2, long long L, T *Z,
                                 double alpha, cudaStream_t s) {
  if (n1 < 1 || n2 < 1 || n1 > 128 || n2 > 128) return cudaErrorInvalidValue;
  auto run = [&](auto kern, int NJ) -> cudaError_t {
    const int ncg = (n2 + NJ - 1) / NJ;
    const int rows_blk = 256 / ncg;
    const size_t smem = sizeof(T) * ((size_t)n1 * ncg * NJ + (size_t)rows_blk * (n1 + 1));
    cudaError_t e = raise_smem_limit(kern, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<long long>((L + rows_blk - 1) / rows_blk, 148LL * 8);
    ::invdft::count_launch();
    kern<<<grid, 256, smem, s>>>(Psi, n1, C, n2, L, Z, alpha);
    return cudaGetLastError();
  };
  if (n2 <= 8) return run(stripe_rotate<T, 8>, 8);
  return run(stripe_rotate<T, 16>, 16);
}

template cudaError_t launch_stripe_gram<float, float>(const float *, int, const float *, int,
                                                      long long, double *, double *, cudaStream_t);
template cudaError_t launch_stripe_gram<double, double>(const double *, int, const double *, int,
                                                        long long, double *, double *,
                                                        cudaStream_t);
template cudaError_t launch_stripe_rotate<float>(const float *, int, const double *, int,
                                                 long long, float *, double, cudaStream_t);
template cudaError_t launch_stripe_rotate<double>(const double *, int, const double *, int,
                                                  long long, double *, double, cudaStream_t);

}  // namespace invdft

// ---------------------------------------------------------------------------
// Both Gram matrices of the Rayleigh-Ritz step (Eq. 23), S = Y^T Y and
// Hs = Y^T (H~Y), in FP64 from one pass over Y and H~Y.  Both are symmetric,
// so only the 4 x 4 tiles on or above the diagonal are formed (about half the
// FP64 FMAs of two full Grams); the final sum mirrors them.
namespace invdft {
namespace {

constexpr int kRrRows = 32;
constexpr int kRrTasks = 3;          // tiles per thread (n <= 96: 2 x 300 tiles)

__device__ __forceinline__ void tri_tile(int k, int T, int &ti, int &tj) {
  ti = 0;
  while (k >= T - ti) {
    k -= T - ti;
    ++ti;
  }
  tj = ti + k;
}

__global__ void __launch_bounds__(256) gram_rr_kernel(const double *__restrict__ Y,
                                                      const double *__restrict__ HY, int n,
                                                      long long L, double *__restrict__ partial) {
  extern __shared__ __align__(16) double rsm[];
  double *sY = rsm;                          // [2][kRrRows][n]
  double *sH = rsm + 2 * kRrRows * n;        // [2][kRrRows][n]
  const int tid = threadIdx.x;
  const int T = (n + 3) / 4, NT = T * (T + 1) / 2, ntask = 2 * NT;
  // ntask <= 256: one tile per thread, spare threads split the rows into
  // S stripes; otherwise up to kRrTasks tiles per thread
  const int S = ntask <= 256 ? min(kRrRows, 256 / ntask) : 1;
  const int stripe = ntask <= 256 ? tid / ntask : 0;
  const int tbase = ntask <= 256 ? tid - stripe * ntask : tid;
  int i0[kRrTasks], j0[kRrTasks];
  bool hs[kRrTasks], on[kRrTasks];
#pragma unroll
  for (int m = 0; m < kRrTasks; ++m) {
    const int t = tbase + 256 * m;
    on[m] = t < ntask && stripe < S;
    int ti = 0, tj = 0;
    if (on[m]) tri_tile(t % NT, T, ti, tj);
    i0[m] = 4 * ti;
    j0[m] = 4 * tj;
    hs[m] = t >= NT;
  }
  const long long per = ((L + gridDim.x - 1) / gridDim.x + kRrRows - 1) / kRrRows * kRrRows;
  const long long r_begin = (long long)blockIdx.x * per;
  const long long r_end = min(L, r_begin + per);
  double acc[kRrTasks][4][4];
#pragma unroll
  for (int m = 0; m < kRrTasks; ++m)
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[m][x][y] = 0.0;
  auto stage = [&](int buf, long long r0) {
    const int rows = (int)min((long long)kRrRows, r_end - r0);
    double *dy = sY + buf * kRrRows * n, *dh = sH + buf * kRrRows * n;
    for (int e = tid; e < kRrRows * n; e += 256) {
      if (e < rows * n) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                     :: "r"((unsigned)__cvta_generic_to_shared(dy + e)), "l"(Y + r0 * n + e)
                     : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;"
                     :: "r"((unsigned)__cvta_generic_to_shared(dh + e)), "l"(HY + r0 * n + e)
                     : "memory");
      } else {
        dy[e] = 0.0;
        dh[e] = 0.0;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int buf = 0;
  if (r_begin < r_end) stage(0, r_begin);
  for (long long r0 = r_begin; r0 < r_end; r0 += kRrRows) {
    const bool more = r0 + kRrRows < r_end;
    if (more) {
      stage(buf ^ 1, r0 + kRrRows);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const double *ry = sY + buf * kRrRows * n, *rh = sH + buf * kRrRows * n;
#pragma unroll
    for (int m = 0; m < kRrTasks; ++m) {
      if (!on[m]) continue;
      const double *rb = hs[m] ? rh : ry;
      for (int r = stripe; r < kRrRows; r += S) {
        double av[4], bv[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          av[x] = i0[m] + x < n ? ry[r * n + i0[m] + x] : 0.0;
          bv[x] = j0[m] + x < n ? rb[r * n + j0[m] + x] : 0.0;
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[m][x][y] = fma(av[x], bv[y], acc[m][x][y]);
      }
    }
    __syncthreads();
    buf ^= 1;
  }
  if (S > 1) {
    // stripes -> shared memory -> stripe 0 (the staging buffers are idle now)
    if (on[0])
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) rsm[(size_t)(stripe * ntask + tbase) * 16 + x * 4 + y] = acc[0][x][y];
    __syncthreads();
    if (stripe == 0 && on[0])
      for (int q = 1; q < S; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[0][x][y] += rsm[(size_t)(q * ntask + tbase) * 16 + x * 4 + y];
  }
  if (stripe != 0) return;
  double *out = partial + (size_t)blockIdx.x * ntask * 16;
#pragma unroll
  for (int m = 0; m < kRrTasks; ++m) {
    if (!on[m]) continue;
    const int t = tbase + 256 * m;
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) out[(size_t)t * 16 + x * 4 + y] = acc[m][x][y];
  }
}

// S[i][j], Hs[i][j] from the tile partials of all CTAs (mirrored below the
// diagonal); e < 2 n^2 indexes S then Hs
__global__ void gram_rr_sum(const double *__restrict__ partial, int nblk, int n,
                            double *__restrict__ S, double *__restrict__ Hs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * n * n) return;
  const int mat = e / (n * n), r = e - mat * n * n;
  int i = r / n, j = r - (r / n) * n;
  if (i / 4 > j / 4) {
    const int t = i;
    i = j;
    j = t;
  }
  const int T = (n + 3) / 4, NT = T * (T + 1) / 2, ti = i / 4, tj = j / 4;
  const int k = ti * T - ti * (ti - 1) / 2 + (tj - ti);
  const size_t task = (size_t)mat * NT + k, stride = (size_t)2 * NT * 16;
  const size_t off = task * 16 + (i % 4) * 4 + (j % 4);
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * stride + off];
  (mat == 0 ? S : Hs)[r] = s;
}

}  // namespace

cudaError_t launch_gram_rr(const double *Y, const double *HY, int n, long long L, double *S,
                           double *Hs, double *partial, cudaStream_t s) {
  const int T = (n + 3) / 4;
  if (n < 1 || 2 * T * (T + 1) / 2 > 256 * kRrTasks) return cudaErrorInvalidValue;
  // staging ring, and room for the stripe sums (at most 256 x 16 doubles)
  const size_t smem = std::max(4 * (size_t)kRrRows * n, (size_t)256 * 16) * sizeof(double);
  cudaError_t e =
      raise_smem_limit(gram_rr_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  gram_rr_kernel<<<kGramBlocks, 256, smem, s>>>(Y, HY, n, L, partial);
  ::invdft::count_launch();
  gram_rr_sum<<<(2 * n * n + 255) / 256, 256, 0, s>>>(partial, kGramBlocks, n, S, Hs);
  return cudaGetLastError();
}

}  // namespace invdft
