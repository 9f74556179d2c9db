// FP32 deflation of the MINRES blocks against the converged Ritz vectors,
//   Z <- Z - Psi (Psi^T Z)                                   (Sec. 3.2.2)
// with an optional fused column dot of the updated block.  Both blocks are
// node-major with widths n1p, n2p that are multiples of 4 (zero padding
// columns), so a run of rows is one contiguous, 16-byte aligned span that is
// staged with 16-byte cp.async copies and read back with float4 loads.
#include <algorithm>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kDgRows = 64;       // rows per staged chunk of the Gram
constexpr int kDgStages = 3;      // cp.async ring depth of the Gram
constexpr int kDuRows = 128;      // rows per tile of the update
constexpr int kDgCtasPerSm = 2;

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
               :: "r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory"); }

// partial[b][i * n2p + j] = sum over the rows of CTA b of A[a][i] B[a][j]
// (n1p a multiple of 8, n2p of 4).  A thread owns an 8 x 4 output tile; when
// the n1p x n2p output has fewer tiles than the CTA has threads, the rows of
// each chunk are split into S stripes whose sums meet in shared memory.
__global__ void __launch_bounds__(256, kDgCtasPerSm)
defl_gram_kernel(const float *__restrict__ A, int n1p, const float *__restrict__ B, int n2p,
                 long long L, double *__restrict__ partial) {
  extern __shared__ __align__(16) float dsm[];
  const int stage = kDgRows * (n1p + n2p);
  const int tid = threadIdx.x;
  const int T2 = n2p / 4, T = (n1p / 8) * T2;
  const int S = min(kDgRows, 256 / T);
  const int stripe = tid / T, t = tid - stripe * T;
  const int ti = t / T2, tj = t - ti * T2;
  const bool act = stripe < S;
  const long long per =
      ((L + gridDim.x - 1) / gridDim.x + kDgRows - 1) / kDgRows * kDgRows;
  const long long r0 = (long long)blockIdx.x * per;
  const long long r1 = min(L, r0 + per);
  const int nchunk = r0 < r1 ? (int)((r1 - r0 + kDgRows - 1) / kDgRows) : 0;
  auto load = [&](int k) {
    float *sa = dsm + (k % kDgStages) * stage;
    float *sb = sa + kDgRows * n1p;
    const long long a0 = r0 + (long long)k * kDgRows;
    const int rows = (int)min((long long)kDgRows, r1 - a0);
    const int na = rows * n1p / 4, nb = rows * n2p / 4;
    const float4 *ga = reinterpret_cast<const float4 *>(A + a0 * n1p);
    const float4 *gb = reinterpret_cast<const float4 *>(B + a0 * n2p);
    for (int e = tid; e < na; e += 256) cp_async16(sa + 4 * e, ga + e);
    for (int e = tid; e < nb; e += 256) cp_async16(sb + 4 * e, gb + e);
    if (rows < kDgRows) {   // last chunk of the range: zero rows past its end
      for (int e = 4 * na + tid; e < kDgRows * n1p; e += 256) sa[e] = 0.f;
      for (int e = 4 * nb + tid; e < kDgRows * n2p; e += 256) sb[e] = 0.f;
    }
  };
  float acc[8][4];
#pragma unroll
  for (int x = 0; x < 8; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) acc[x][y] = 0.f;
#pragma unroll
  for (int k = 0; k < kDgStages - 1; ++k) {
    if (k < nchunk) load(k);
    cp_commit();
  }
  for (int k = 0; k < nchunk; ++k) {
    if (k + kDgStages - 1 < nchunk) load(k + kDgStages - 1);
    cp_commit();
    cp_wait<kDgStages - 1>();
    __syncthreads();
    const float *sa = dsm + (k % kDgStages) * stage + ti * 8;
    const float *sb = dsm + (k % kDgStages) * stage + kDgRows * n1p + tj * 4;
    if (act) {
#pragma unroll 4
      for (int r = stripe; r < kDgRows; r += S) {
        const float4 a0 = *reinterpret_cast<const float4 *>(sa + r * n1p);
        const float4 a1 = *reinterpret_cast<const float4 *>(sa + r * n1p + 4);
        const float4 b = *reinterpret_cast<const float4 *>(sb + r * n2p);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
      }
    }
    __syncthreads();
  }
  double *out = partial + (size_t)blockIdx.x * n1p * n2p;
  if (S > 1) {
    // stripes -> shared memory -> stripe 0 (the ring is idle now)
    if (act)
#pragma unroll
      for (int x = 0; x < 8; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) dsm[(stripe * T + t) * 32 + x * 4 + y] = acc[x][y];
    __syncthreads();
    if (stripe == 0) {
      for (int qq = 1; qq < S; ++qq)
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] += dsm[(qq * T + t) * 32 + x * 4 + y];
    }
  }
  if (stripe == 0)
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y)
        out[(size_t)(ti * 8 + x) * n2p + tj * 4 + y] = (double)acc[x][y];
}

// out[e] = sum_b partial[b * n + e]: 32 outputs per CTA, 8 groups of CTAs
// summed with independent accumulators and met in shared memory.
__global__ void __launch_bounds__(256) defl_sum_partials(const double *__restrict__ partial,
                                                         int nblk, int n,
                                                         double *__restrict__ out) {
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int e = blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0;
  if (e < n) {
    int b = g;
    for (; b + 8 < nblk; b += 16) {
      s0 += partial[(size_t)b * n + e];
      s1 += partial[(size_t)(b + 8) * n + e];
    }
    if (b < nblk) s0 += partial[(size_t)b * n + e];
  }
  red[g][lane] = s0 + s1;
  __syncthreads();
  if (g == 0 && e < n) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += red[k][lane];
    out[e] = s;
  }
}

// Z[a][j] += sum_i Psi[a][i] (alpha C)[i][j] over 128-row tiles; with DOT,
// partial[b][j] = sum over the rows of CTA b of V[a][j] Z_new[a][j].
// Thread (tx, ty), ty < 16, owns columns 4 tx .. 4 tx + 3 of rows ty + 16 r,
// r < 8, of each tile.  The Psi tile is staged in shared memory with row
// stride ldp (ldp / 4 odd, so the three rows a warp reads at once fall in
// different banks) and double-buffered; Z of the tile is loaded into
// registers before the FMA loop so that its latency overlaps it.
template <bool DOT>
__global__ void __launch_bounds__(256, 2)
defl_update_kernel(const float *__restrict__ Psi, int n1p, int ldp, const double *__restrict__ C,
                   int n2p, long long L, float *__restrict__ Z, double alpha,
                   const float *__restrict__ V, double *__restrict__ partial) {
  extern __shared__ __align__(16) float usm[];
  float *sC = usm;                      // [n1p][n2p], alpha C in FP32
  float *sP = usm + n1p * n2p;          // 2 x [kDuRows][ldp]
  __shared__ double red[16][64];
  const int tid = threadIdx.x;
  const int T2 = n2p / 4;
  const int ty = tid / T2, tx = tid - ty * T2;
  const bool act = ty < 16;
  for (int e = tid; e < n1p * n2p; e += 256) sC[e] = (float)(alpha * C[e]);
  const long long ntile = (L + kDuRows - 1) / kDuRows;
  const int q1 = n1p / 4;
  auto load = [&](long long tile, int buf) {
    const long long a0 = tile * kDuRows;
    const int rows = (int)min((long long)kDuRows, L - a0);
    float *dst = sP + buf * kDuRows * ldp;
    const float4 *src = reinterpret_cast<const float4 *>(Psi + a0 * n1p);
    const int n4 = rows * q1;
    for (int e = tid; e < n4; e += 256) {
      const int r = e / q1, c = e - r * q1;
      cp_async16(dst + r * ldp + 4 * c, src + e);
    }
  };
  // dot partials: per-tile FP32 sums folded into a compensated FP32 total
  // (no FP64 work in the tile loop: FP64 issues at a small fraction of the
  // FP32 rate on this part)
  float dsum[4] = {0.f, 0.f, 0.f, 0.f}, dcmp[4] = {0.f, 0.f, 0.f, 0.f};
  long long tile = blockIdx.x;
  if (tile < ntile) load(tile, 0);
  cp_commit();
  int buf = 0;
  for (; tile < ntile; tile += gridDim.x) {
    const long long nxt = tile + gridDim.x;
    if (nxt < ntile) load(nxt, buf ^ 1);
    cp_commit();
    const long long a0 = tile * kDuRows;
    const int rows = (int)min((long long)kDuRows, L - a0);
    float4 z[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = ty + 16 * r;
      z[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (act && row < rows)
        z[r] = *reinterpret_cast<const float4 *>(Z + (size_t)(a0 + row) * n2p + tx * 4);
    }
    cp_wait<1>();
    __syncthreads();
    if (act) {
      const float *sp = sP + buf * kDuRows * ldp + ty * ldp;
      const float *sc = sC + tx * 4;
      float acc[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.f;
      for (int i = 0; i < n1p; i += 4) {
        const float4 c0 = *reinterpret_cast<const float4 *>(sc + (i + 0) * n2p);
        const float4 c1 = *reinterpret_cast<const float4 *>(sc + (i + 1) * n2p);
        const float4 c2 = *reinterpret_cast<const float4 *>(sc + (i + 2) * n2p);
        const float4 c3 = *reinterpret_cast<const float4 *>(sc + (i + 3) * n2p);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float4 p = *reinterpret_cast<const float4 *>(sp + 16 * r * ldp + i);
          acc[r][0] = fmaf(p.x, c0.x, fmaf(p.y, c1.x, fmaf(p.z, c2.x, fmaf(p.w, c3.x, acc[r][0]))));
          acc[r][1] = fmaf(p.x, c0.y, fmaf(p.y, c1.y, fmaf(p.z, c2.y, fmaf(p.w, c3.y, acc[r][1]))));
          acc[r][2] = fmaf(p.x, c0.z, fmaf(p.y, c1.z, fmaf(p.z, c2.z, fmaf(p.w, c3.z, acc[r][2]))));
          acc[r][3] = fmaf(p.x, c0.w, fmaf(p.y, c1.w, fmaf(p.z, c2.w, fmaf(p.w, c3.w, acc[r][3]))));
        }
      }
      float ds[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int row = ty + 16 * r;
        if (row < rows) {
          const size_t off = (size_t)(a0 + row) * n2p + tx * 4;
          float4 o;
          o.x = z[r].x + acc[r][0];
          o.y = z[r].y + acc[r][1];
          o.z = z[r].z + acc[r][2];
          o.w = z[r].w + acc[r][3];
          *reinterpret_cast<float4 *>(Z + off) = o;
          if (DOT) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(V + off));
            ds[0] = fmaf(v.x, o.x, ds[0]);
            ds[1] = fmaf(v.y, o.y, ds[1]);
            ds[2] = fmaf(v.z, o.z, ds[2]);
            ds[3] = fmaf(v.w, o.w, ds[3]);
          }
        }
      }
      if (DOT)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float y = ds[q] - dcmp[q];
          const float t = dsum[q] + y;
          dcmp[q] = (t - dsum[q]) - y;
          dsum[q] = t;
        }
    }
    __syncthreads();
    buf ^= 1;
  }
  if (DOT) {
    if (act)
#pragma unroll
      for (int q = 0; q < 4; ++q) red[ty][tx * 4 + q] = (double)dsum[q] - (double)dcmp[q];
    __syncthreads();
    if (tid < n2p) {
      double s = 0.0;
      for (int k = 0; k < 16; ++k) s += red[k][tid];
      partial[(size_t)blockIdx.x * n2p + tid] = s;
    }
  }
}

int num_sms() {
  static const int nsm = [] {
    int n = 148;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, 0);
    return n;
  }();
  return nsm;
}

bool padded_ok(int n) { return n >= 4 && n <= 64 && n % 4 == 0; }
bool padded8_ok(int n) { return n >= 8 && n <= 64 && n % 8 == 0; }

// [L][n] FP64 -> [L][np] FP32 with zero columns n .. np-1 (L * np < 2^31 is
// checked at handle creation)
__global__ void convert_pad_kernel(const double *__restrict__ X, int n, int np, uint32_t total,
                                   float *__restrict__ F, FastDiv fd) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += gridDim.x * blockDim.x) {
    const uint32_t a = fdiv(e, fd);
    const int j = (int)(e - a * (uint32_t)np);
    F[e] = j < n ? (float)X[(size_t)a * n + j] : 0.f;
  }
}

__global__ void add_unpad_kernel(const float *__restrict__ F, int np, double *__restrict__ P,
                                 int n, uint32_t total, FastDiv fd) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += gridDim.x * blockDim.x) {
    const uint32_t a = fdiv(e, fd);
    const int j = (int)(e - a * (uint32_t)n);
    P[e] += (double)F[(size_t)a * np + j];
  }
}

int elementwise_grid(long long n) {
  return (int)std::min<long long>((n + 255) / 256, (long long)num_sms() * 8);
}

}  // namespace

cudaError_t launch_sum_partials(const double *partial, int nblk, int n, double *out,
                                cudaStream_t s) {
  ::invdft::count_launch();
  defl_sum_partials<<<(n + 31) / 32, 256, 0, s>>>(partial, nblk, n, out);
  return cudaGetLastError();
}

cudaError_t launch_convert_pad_f32(const double *X, int n, int np, long long L, float *F,
                                   cudaStream_t s) {
  if (n < 1 || np < n || L < 1) return cudaErrorInvalidValue;
  const long long total = L * np;
  ::invdft::count_launch();
  convert_pad_kernel<<<elementwise_grid(total), 256, 0, s>>>(X, n, np, (uint32_t)total, F,
                                                             make_fastdiv(np));
  return cudaGetLastError();
}

cudaError_t launch_add_unpad(const float *F, int np, double *P, int n, long long L,
                             cudaStream_t s) {
  if (n < 1 || np < n || L < 1) return cudaErrorInvalidValue;
  const long long total = L * n;
  ::invdft::count_launch();
  add_unpad_kernel<<<elementwise_grid(total), 256, 0, s>>>(F, np, P, n, (uint32_t)total,
                                                           make_fastdiv(n));
  return cudaGetLastError();
}

cudaError_t launch_defl_gram_f32(const float *Psi, int n1p, const float *Z, int n2p, long long L,
                                 double *G, double *partial, cudaStream_t s) {
  if (!padded8_ok(n1p) || !padded_ok(n2p) || L < 1) return cudaErrorInvalidValue;
  const int nblk = kGramBlocks;
  const size_t smem =
      std::max((size_t)kDgStages * kDgRows * (n1p + n2p), (size_t)256 * 32) * sizeof(float);
  cudaError_t e = raise_smem_limit(defl_gram_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  defl_gram_kernel<<<nblk, 256, smem, s>>>(Psi, n1p, Z, n2p, L, partial);
  const int n = n1p * n2p;
  ::invdft::count_launch();
  defl_sum_partials<<<(n + 31) / 32, 256, 0, s>>>(partial, nblk, n, G);
  return cudaGetLastError();
}

cudaError_t launch_defl_update_f32(const float *Psi, int n1p, const double *C, int n2p,
                                   long long L, float *Z, double alpha, const float *V,
                                   double *dot_out, double *partial, cudaStream_t s) {
  if (!padded_ok(n1p) || !padded_ok(n2p) || L < 1) return cudaErrorInvalidValue;
  const int ldp = (n1p / 4) % 2 == 1 ? n1p : n1p + 4;
  const size_t smem = ((size_t)n1p * n2p + 2 * (size_t)kDuRows * ldp) * sizeof(float);
  const long long ntile = (L + kDuRows - 1) / kDuRows;
  const int grid = (int)std::min<long long>(ntile, (long long)num_sms() * 2);
  cudaError_t e;
  if (V) {
    e = raise_smem_limit(defl_update_kernel<true>, (int)smem);
    if (e != cudaSuccess) return e;
    ::invdft::count_launch();
    defl_update_kernel<true><<<grid, 256, smem, s>>>(Psi, n1p, ldp, C, n2p, L, Z, alpha, V,
                                                     partial);
    ::invdft::count_launch();
    defl_sum_partials<<<(n2p + 31) / 32, 256, 0, s>>>(partial, grid, n2p, dot_out);
  } else {
    e = raise_smem_limit(defl_update_kernel<false>, (int)smem);
    if (e != cudaSuccess) return e;
    ::invdft::count_launch();
    defl_update_kernel<false><<<grid, 256, smem, s>>>(Psi, n1p, ldp, C, n2p, L, Z, alpha,
                                                      nullptr, nullptr);
  }
  return cudaGetLastError();
}

}  // namespace invdft
