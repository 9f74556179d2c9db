// FP32 H~X on the CUDA cores for Q4 cells: the exact-FP32 operator of the
// inner MINRES iterations (the tensor-core TF32 kernel in hx_tc.cu is used by
// the Chebyshev filter).  Same contract as the tensor-core kernel: the
// launcher zeroes Z, every (cell, column chunk) tile gathers d o X_e with
// float4 loads, applies K_e in its Kronecker-factored form (seven 1D
// contractions of the 5x5x5 cell tensor in shared memory), and the epilogue
// adds the nodal term for the nodes the cell owns and scatter-adds with
// vector reductions.  Persistent CTAs walk the cells in the slab order of the
// tensor-core kernel.
#include <cstdint>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kSmThreads = 256;
constexpr int kQ = 5, kNe = 125;

struct SmArgs {
  const float *X;
  float *Z;
  const float *W;
  const double *v;
  const double *shift_col;
  const float *dm1f;
  const int *perm;
  float A[25], B[25];
  float kc_alpha, alpha, beta, shift;
  int ncol, ncell, Ni;
};

template <int C, bool HW>
__global__ void __launch_bounds__(kSmThreads, 3) hx_simt_kernel(SmArgs p) {
  constexpr int C4 = C / 4;
  extern __shared__ __align__(16) float sm[];
  float *u = sm;                 // [125][C]
  float *w = sm + kNe * C;       // [125][C]
  __shared__ float sA[25], sB[25];
  __shared__ float dlf[3][5];
  __shared__ int gi[3][5];
  __shared__ float sshift[kMaxCols];
  const int tid = threadIdx.x;
  const int nc = p.ncell, Ni = p.Ni;
  const int ncells = nc * nc * nc;
  const int nchunk = (p.ncol + C - 1) / C;
  const long long items = (long long)ncells * nchunk;
  if (tid < 25) {
    sA[tid] = p.A[tid];
    sB[tid] = p.B[tid];
  }
  for (int j = tid; j < p.ncol; j += kSmThreads)
    sshift[j] = (float)(p.shift_col ? p.shift_col[j] : p.shift);
  const bool vec = (p.ncol & 3) == 0;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int chunk = (int)(item % nchunk);
    const int cell = p.perm[item / nchunk];
    const int c0 = chunk * C;
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    __syncthreads();
    if (tid < 15) {
      const int d = tid / 5, l = tid % 5;
      const int g = (d == 0 ? cx : (d == 1 ? cy : cz)) * 4 + l;
      dlf[d][l] = p.dm1f[g];
      gi[d][l] = (g >= 1 && g <= Ni) ? g - 1 : -1;
    }
    __syncthreads();
    // gather u[a][c] = d_a X[node(a)][c0 + c]
    {
      constexpr int total = kNe * C4;
      constexpr int iters = (total + kSmThreads - 1) / kSmThreads;
      float4 vals[iters];
#pragma unroll
      for (int it = 0; it < iters; ++it) {
        const int idx = tid + it * kSmThreads;
        vals[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total) {
          const int a = idx / C4, c4 = idx - a * C4;
          const int lx = a % 5, ly = (a / 5) % 5, lz = a / 25;
          const int ix = gi[0][lx], iy = gi[1][ly], iz = gi[2][lz];
          const int col = c0 + c4 * 4;
          if (ix >= 0 && iy >= 0 && iz >= 0 && col < p.ncol) {
            const long long node = ix + (long long)Ni * (iy + (long long)Ni * iz);
            const float sc = dlf[0][lx] * dlf[1][ly] * dlf[2][lz];
            const float *src = p.X + node * p.ncol + col;
            float4 x;
            if (vec) {
              x = __ldg(reinterpret_cast<const float4 *>(src));
            } else {
              x.x = __ldg(src);
              x.y = col + 1 < p.ncol ? __ldg(src + 1) : 0.f;
              x.z = col + 2 < p.ncol ? __ldg(src + 2) : 0.f;
              x.w = col + 3 < p.ncol ? __ldg(src + 3) : 0.f;
            }
            vals[it] = make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
          }
        }
      }
#pragma unroll
      for (int it = 0; it < iters; ++it) {
        const int idx = tid + it * kSmThreads;
        if (idx < total) reinterpret_cast<float4 *>(u)[idx] = vals[it];
      }
    }
    __syncthreads();
    // x lines: u <- B_x u, w <- A_x u
    for (int idx = tid; idx < 25 * C; idx += kSmThreads) {
      const int j = idx % C, base = (idx / C) * kQ;
      float in[kQ];
#pragma unroll
      for (int x = 0; x < kQ; ++x) in[x] = u[(base + x) * C + j];
#pragma unroll
      for (int xo = 0; xo < kQ; ++xo) {
        float sb = 0.f, sa = 0.f;
#pragma unroll
        for (int x = 0; x < kQ; ++x) {
          sb = fmaf(sB[xo * kQ + x], in[x], sb);
          sa = fmaf(sA[xo * kQ + x], in[x], sa);
        }
        u[(base + xo) * C + j] = sb;
        w[(base + xo) * C + j] = sa;
      }
    }
    __syncthreads();
    // y lines: u <- B_y u, w <- A_y u + B_y w
    for (int idx = tid; idx < 25 * C; idx += kSmThreads) {
      const int j = idx % C, r = idx / C;
      const int x = r % kQ, z = r / kQ;
      float t1[kQ], t2[kQ];
#pragma unroll
      for (int y = 0; y < kQ; ++y) {
        t1[y] = u[(x + kQ * (y + kQ * z)) * C + j];
        t2[y] = w[(x + kQ * (y + kQ * z)) * C + j];
      }
#pragma unroll
      for (int yo = 0; yo < kQ; ++yo) {
        float s11 = 0.f, q = 0.f;
#pragma unroll
        for (int y = 0; y < kQ; ++y) {
          s11 = fmaf(sB[yo * kQ + y], t1[y], s11);
          q = fmaf(sA[yo * kQ + y], t1[y], fmaf(sB[yo * kQ + y], t2[y], q));
        }
        u[(x + kQ * (yo + kQ * z)) * C + j] = s11;
        w[(x + kQ * (yo + kQ * z)) * C + j] = q;
      }
    }
    __syncthreads();
    // z lines: u <- A_z u + B_z w
    for (int idx = tid; idx < 25 * C; idx += kSmThreads) {
      const int j = idx % C, r = idx / C;
      const int x = r % kQ, y = r / kQ;
      float t1[kQ], t2[kQ];
#pragma unroll
      for (int z = 0; z < kQ; ++z) {
        t1[z] = u[(x + kQ * (y + kQ * z)) * C + j];
        t2[z] = w[(x + kQ * (y + kQ * z)) * C + j];
      }
#pragma unroll
      for (int zo = 0; zo < kQ; ++zo) {
        float s = 0.f;
#pragma unroll
        for (int z = 0; z < kQ; ++z) s = fmaf(sA[zo * kQ + z], t1[z], fmaf(sB[zo * kQ + z], t2[z], s));
        u[(x + kQ * (y + kQ * zo)) * C + j] = s;
      }
    }
    __syncthreads();
    // epilogue: (node a, column quad) per thread; nodal term for owned nodes
    for (int idx = tid; idx < kNe * C4; idx += kSmThreads) {
      const int a = idx / C4, c4 = idx - a * C4;
      const int lx = a % 5, ly = (a / 5) % 5, lz = a / 25;
      const int ix = gi[0][lx], iy = gi[1][ly], iz = gi[2][lz];
      const int col = c0 + c4 * 4;
      if (ix < 0 || iy < 0 || iz < 0 || col >= p.ncol) continue;
      const long long node = ix + (long long)Ni * (iy + (long long)Ni * iz);
      const long long e0 = node * p.ncol + col;
      const float sc = p.kc_alpha * dlf[0][lx] * dlf[1][ly] * dlf[2][lz];
      const float4 y = reinterpret_cast<const float4 *>(u)[idx];
      float o[4] = {sc * y.x, sc * y.y, sc * y.z, sc * y.w};
      const int m = min(4, p.ncol - col);
      if (lx < 4 && ly < 4 && lz < 4) {
        const float va = (float)__ldg(p.v + node);
        float xs[4] = {0.f, 0.f, 0.f, 0.f}, ws[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec) {
          const float4 x4 = __ldg(reinterpret_cast<const float4 *>(p.X + e0));
          xs[0] = x4.x; xs[1] = x4.y; xs[2] = x4.z; xs[3] = x4.w;
          if (HW) {
            const float4 w4 = *reinterpret_cast<const float4 *>(p.W + e0);
            ws[0] = w4.x; ws[1] = w4.y; ws[2] = w4.z; ws[3] = w4.w;
          }
        } else {
          for (int t = 0; t < m; ++t) {
            xs[t] = p.X[e0 + t];
            if (HW) ws[t] = p.W[e0 + t];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          float tt = p.alpha * (va - sshift[min(col + t, p.ncol - 1)]) * xs[t];
          if (HW) tt = fmaf(p.beta, ws[t], tt);
          o[t] += tt;
        }
      }
      float *dst = p.Z + e0;
      if (vec) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                     :: "l"(dst), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]) : "memory");
      } else {
        for (int t = 0; t < m; ++t)
          asm volatile("red.global.add.f32 [%0], %1;" :: "l"(dst + t), "f"(o[t]) : "memory");
      }
    }
  }
}

template <int C, bool HW>
cudaError_t run_simt(const SmArgs &p, long long items, cudaStream_t s) {
  const size_t smem = 2 * (size_t)kNe * C * sizeof(float);
  auto k = hx_simt_kernel<C, HW>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  const int grid = (int)std::min<long long>(items, (long long)nsm * 3);
  ::invdft::count_launch();
  k<<<grid, kSmThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// FP32 CUDA-core H~X for Q4 meshes (no E term; W optional).  Z must not
// alias X or W; it is zeroed here.
cudaError_t launch_hx_simt_q4(const Geom &g, const double *v, const HxArgs<float> &a,
                              const int *perm, cudaStream_t s) {
  if (g.p != 4 || a.E) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.Z, 0, (size_t)g.L * a.ncol * sizeof(float), s);
  if (e != cudaSuccess) return e;
  SmArgs p;
  p.X = a.X;
  p.Z = a.Z;
  p.W = a.W;
  p.v = v;
  p.shift_col = a.shift_col;
  p.dm1f = g.dm1f;
  p.perm = perm;
  for (int i = 0; i < 25; ++i) {
    p.A[i] = (float)g.A[i];
    p.B[i] = (float)g.B[i];
  }
  p.kc_alpha = (float)(g.kc * a.alpha);
  p.alpha = (float)a.alpha;
  p.beta = (float)a.beta;
  p.shift = (float)a.shift;
  p.ncol = a.ncol;
  p.ncell = g.ncell;
  p.Ni = g.Ni;
  const int C = a.ncol <= 16 ? 16 : (a.ncol <= 32 ? 32 : 64);
  const long long items = (long long)g.ncell * g.ncell * g.ncell * ((a.ncol + C - 1) / C);
  if (C == 16) return a.W ? run_simt<16, true>(p, items, s) : run_simt<16, false>(p, items, s);
  if (C == 32) return a.W ? run_simt<32, true>(p, items, s) : run_simt<32, false>(p, items, s);
  return a.W ? run_simt<64, true>(p, items, s) : run_simt<64, false>(p, items, s);
}

}  // namespace invdft
