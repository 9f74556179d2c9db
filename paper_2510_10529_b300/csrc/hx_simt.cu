// FP32 H~X on the CUDA cores for Q4 cells: the exact-FP32 operator of the
// inner MINRES iterations (the tensor-core TF32 kernel in hx_tc.cu is used by
// the Chebyshev filter).  Same contract as the tensor-core kernel: the
// launcher zeroes Z, every (cell, column chunk) tile gathers d o X_e with
// float4 loads, applies K_e in its Kronecker-factored form (seven 1D
// contractions of the 5x5x5 cell tensor in shared memory), and the epilogue
// adds the nodal term for the nodes the cell owns and scatter-adds with
// vector reductions.  In each contraction phase a thread owns one 1D line of
// the cell for four adjacent columns (float4 shared-memory traffic), and the
// 5x5 element matrices are kernel parameters, so they enter the FMAs as
// constant operands.  Persistent CTAs walk the cells in the slab order of the
// tensor-core kernel.
#include <cstdint>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kQ = 5, kNe = 125;

struct SmArgs {
  const float *X;
  float *Z;
  const float *W;
  const float *E;           // optional defect block, added as alpha escale_j E
  const double *escale;
  const float *v;            // potential (FP32 copy)
  const double *shift_col;
  const float *dm1f;
  const int *perm;
  // even / odd blocks of the centrosymmetric 1D matrices (see eo_apply)
  float eA[9], oA[4], eB[9], oB[4];
  float kc_alpha, alpha, beta, shift;
  int ncol, ncell, Ni;
};

// Threads of a CTA for a chunk of C columns: one per (1D line, column quad)
// task of a contraction phase (25 lines x C/4 quads), rounded to whole warps.
template <int C>
__host__ __device__ constexpr int simt_threads() { return (25 * (C / 4) + 31) / 32 * 32; }

__device__ __forceinline__ float4 f4_fma(float a, const float4 &x, const float4 &y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 f4_add(const float4 &x, const float4 &y) {
  return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
}
__device__ __forceinline__ float4 f4_sub(const float4 &x, const float4 &y) {
  return make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
}

// A and B are centrosymmetric (M[i][j] = M[4-i][4-j]), so y = M u splits into
// an even part on e_k = u_k + u_(4-k) (3x3 block) and an odd part on
// o_k = u_k - u_(4-k) (2x2 block): y_i = ye_i + yo_i, y_(4-i) = ye_i - yo_i
// (i < 2), y_2 = ye_2; 13 FMAs instead of 25 per matrix.
__device__ __forceinline__ void eo_split4(const float4 *u, float4 *e, float4 *o) {
  e[0] = f4_add(u[0], u[4]);
  e[1] = f4_add(u[1], u[3]);
  e[2] = u[2];
  o[0] = f4_sub(u[0], u[4]);
  o[1] = f4_sub(u[1], u[3]);
}
// y = M1 u1 (+ M2 u2), each M given by its even (3x3) and odd (2x2) blocks
template <bool TWO>
__device__ __forceinline__ void eo_apply4(const float4 *e1, const float4 *o1, const float *eM1,
                                          const float *oM1, const float4 *e2, const float4 *o2,
                                          const float *eM2, const float *oM2, float4 *y) {
  float4 ye[3], yo[2];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      s = f4_fma(eM1[i * 3 + k], e1[k], s);
      if (TWO) s = f4_fma(eM2[i * 3 + k], e2[k], s);
    }
    ye[i] = s;
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      s = f4_fma(oM1[i * 2 + k], o1[k], s);
      if (TWO) s = f4_fma(oM2[i * 2 + k], o2[k], s);
    }
    yo[i] = s;
  }
  y[0] = f4_add(ye[0], yo[0]);
  y[4] = f4_sub(ye[0], yo[0]);
  y[1] = f4_add(ye[1], yo[1]);
  y[3] = f4_sub(ye[1], yo[1]);
  y[2] = ye[2];
}

template <int C, bool HW>
__global__ void __launch_bounds__(simt_threads<C>(), 2) hx_simt_kernel(const __grid_constant__ SmArgs p) {
  constexpr int Q4 = C / 4;                  // column quads of a chunk
  constexpr int NT = 25 * Q4;                // tasks of a contraction phase
  constexpr int NTH = simt_threads<C>();
  constexpr int NG = (kNe * Q4 + NTH - 1) / NTH;   // (node, quad) slots of a thread
  extern __shared__ __align__(16) float4 sm4[];
  float4 *u = sm4;                 // [125][Q4]
  float4 *w = sm4 + kNe * Q4;      // [125][Q4]
  __shared__ float dlf[3][5];
  __shared__ float sshift[kMaxCols], sesc[kMaxCols];
  const int tid = threadIdx.x;
  const int nc = p.ncell, Ni = p.Ni, ncol = p.ncol;
  const int ncells = nc * nc * nc;
  const int nchunk = (ncol + C - 1) / C;
  const int items = ncells * nchunk;
  for (int j = tid; j < ncol; j += NTH) {
    sshift[j] = (float)(p.shift_col ? p.shift_col[j] : p.shift);
    sesc[j] = p.E ? (float)(p.alpha * p.escale[j]) : 0.f;
  }
  const bool vec = (ncol & 3) == 0;
  const bool act = tid < NT;
  const int q = tid % Q4, l = tid / Q4;      // this thread's task: line l, quad q
  // The (node, quad) slots a thread gathers and scatters are the same for
  // every cell: cell-local node offset, quad, and the bits that make a slot
  // void on a boundary cell (1,2: x = 0 / 4; 4,8: y; 16,32: z), 64 = owned
  // (local index < 4 on every axis), 128 = no slot.
  int goff[NG], gq[NG], gflag[NG], gl[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    const int idx = tid + k * NTH;
    const int a = idx / Q4, c4 = idx - (idx / Q4) * Q4;
    const int lx = a % 5, ly = (a / 5) % 5, lz = a / 25;
    goff[k] = lx + Ni * (ly + Ni * lz);
    gq[k] = c4;
    gl[k] = lx | (ly << 4) | (lz << 8);
    gflag[k] = idx >= kNe * Q4 ? 128
             : (lx == 0) | ((lx == 4) << 1) | ((ly == 0) << 2) | ((ly == 4) << 3) |
                   ((lz == 0) << 4) | ((lz == 4) << 5) | ((lx < 4 && ly < 4 && lz < 4) << 6);
  }
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int chunk = item % nchunk;
    const int cell = p.perm[item / nchunk];
    const int c0 = chunk * C;
    const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
    // void slots of this cell; node index of local (0, 0, 0)
    const int edge = (cx == 0) | ((cx == nc - 1) << 1) | ((cy == 0) << 2) | ((cy == nc - 1) << 3) |
                     ((cz == 0) << 4) | ((cz == nc - 1) << 5) | 128;
    const int base = (4 * cx - 1) + Ni * ((4 * cy - 1) + Ni * (4 * cz - 1));
    __syncthreads();
    if (tid < 15) {
      const int d = tid / 5, t = tid % 5;
      const int g = (d == 0 ? cx : (d == 1 ? cy : cz)) * 4 + t;
      dlf[d][t] = p.dm1f[g];
    }
    __syncthreads();
    // gather u[a][quad] = d_a X[node(a)][c0 + 4 quad ...]
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      if (gflag[k] & 128) continue;
      const int col = c0 + 4 * gq[k];
      float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
      if (!(gflag[k] & edge) && col < ncol) {
        const uint32_t e0 = (uint32_t)(base + goff[k]) * (uint32_t)ncol + (uint32_t)col;
        const float sc = dlf[0][gl[k] & 15] * dlf[1][(gl[k] >> 4) & 15] * dlf[2][gl[k] >> 8];
        const float *src = p.X + e0;
        float4 x;
        if (vec) {
          x = __ldg(reinterpret_cast<const float4 *>(src));
        } else {
          x.x = __ldg(src);
          x.y = col + 1 < ncol ? __ldg(src + 1) : 0.f;
          x.z = col + 2 < ncol ? __ldg(src + 2) : 0.f;
          x.w = col + 3 < ncol ? __ldg(src + 3) : 0.f;
        }
        v4 = make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
      }
      u[tid + k * NTH] = v4;
    }
    __syncthreads();
    // x lines (nodes 5 l .. 5 l + 4): u <- B_x u, w <- A_x u
    if (act) {
      float4 in[kQ], e[3], o[2], yb[kQ], ya[kQ];
#pragma unroll
      for (int x = 0; x < kQ; ++x) in[x] = u[(5 * l + x) * Q4 + q];
      eo_split4(in, e, o);
      eo_apply4<false>(e, o, p.eB, p.oB, e, o, p.eB, p.oB, yb);
      eo_apply4<false>(e, o, p.eA, p.oA, e, o, p.eA, p.oA, ya);
#pragma unroll
      for (int xo = 0; xo < kQ; ++xo) {
        u[(5 * l + xo) * Q4 + q] = yb[xo];
        w[(5 * l + xo) * Q4 + q] = ya[xo];
      }
    }
    __syncthreads();
    // y lines (l = x + 5 z): u <- B_y u, w <- A_y u + B_y w
    if (act) {
      const int base = (l % 5) + 25 * (l / 5);
      float4 t[kQ], e1[3], o1[2], e2[3], o2[2], y1[kQ];
#pragma unroll
      for (int y = 0; y < kQ; ++y) t[y] = u[(base + 5 * y) * Q4 + q];
      eo_split4(t, e1, o1);
#pragma unroll
      for (int y = 0; y < kQ; ++y) t[y] = w[(base + 5 * y) * Q4 + q];
      eo_split4(t, e2, o2);
      eo_apply4<false>(e1, o1, p.eB, p.oB, e1, o1, p.eB, p.oB, y1);
#pragma unroll
      for (int yo = 0; yo < kQ; ++yo) u[(base + 5 * yo) * Q4 + q] = y1[yo];
      eo_apply4<true>(e1, o1, p.eA, p.oA, e2, o2, p.eB, p.oB, y1);
#pragma unroll
      for (int yo = 0; yo < kQ; ++yo) w[(base + 5 * yo) * Q4 + q] = y1[yo];
    }
    __syncthreads();
    // z lines (l = x + 5 y): u <- A_z u + B_z w
    if (act) {
      float4 t[kQ], e1[3], o1[2], e2[3], o2[2], yz[kQ];
#pragma unroll
      for (int z = 0; z < kQ; ++z) t[z] = u[(l + 25 * z) * Q4 + q];
      eo_split4(t, e1, o1);
#pragma unroll
      for (int z = 0; z < kQ; ++z) t[z] = w[(l + 25 * z) * Q4 + q];
      eo_split4(t, e2, o2);
      eo_apply4<true>(e1, o1, p.eA, p.oA, e2, o2, p.eB, p.oB, yz);
#pragma unroll
      for (int zo = 0; zo < kQ; ++zo) u[(l + 25 * zo) * Q4 + q] = yz[zo];
    }
    __syncthreads();
    // epilogue: the thread's (node, quad) slots; nodal term for owned nodes
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int col = c0 + 4 * gq[k];
      if ((gflag[k] & edge) || col >= ncol) continue;
      const uint32_t node = (uint32_t)(base + goff[k]);
      const uint32_t e0 = node * (uint32_t)ncol + (uint32_t)col;
      const float sc =
          p.kc_alpha * dlf[0][gl[k] & 15] * dlf[1][(gl[k] >> 4) & 15] * dlf[2][gl[k] >> 8];
      const float4 y = u[tid + k * NTH];
      float o[4] = {sc * y.x, sc * y.y, sc * y.z, sc * y.w};
      const int m = min(4, ncol - col);
      if (gflag[k] & 64) {
        const float va = __ldg(p.v + node);
        float xs[4] = {0.f, 0.f, 0.f, 0.f}, ws[4] = {0.f, 0.f, 0.f, 0.f};
        float es[4] = {0.f, 0.f, 0.f, 0.f};
        if (vec) {
          const float4 x4 = __ldg(reinterpret_cast<const float4 *>(p.X + e0));
          xs[0] = x4.x; xs[1] = x4.y; xs[2] = x4.z; xs[3] = x4.w;
          if (HW) {
            const float4 w4 = *reinterpret_cast<const float4 *>(p.W + e0);
            ws[0] = w4.x; ws[1] = w4.y; ws[2] = w4.z; ws[3] = w4.w;
          }
          if (p.E) {
            const float4 e4 = __ldg(reinterpret_cast<const float4 *>(p.E + e0));
            es[0] = e4.x; es[1] = e4.y; es[2] = e4.z; es[3] = e4.w;
          }
        } else {
          for (int t = 0; t < m; ++t) {
            xs[t] = p.X[e0 + t];
            if (HW) ws[t] = p.W[e0 + t];
            if (p.E) es[t] = p.E[e0 + t];
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int jc = min(col + t, ncol - 1);
          float tt = p.alpha * (va - sshift[jc]) * xs[t];
          if (HW) tt = fmaf(p.beta, ws[t], tt);
          tt = fmaf(sesc[jc], es[t], tt);
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
  int nsm = 148, per_sm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, simt_threads<C>(), smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)std::min<long long>(items, (long long)nsm * std::max(per_sm, 1));
  ::invdft::count_launch();
  k<<<grid, simt_threads<C>(), smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// FP32 CUDA-core H~X for Q4 meshes (W and E optional).  Z must not alias X,
// W or E; it is zeroed here.
cudaError_t launch_hx_simt_q4(const Geom &g, const float *v, const HxArgs<float> &a,
                              const int *perm, cudaStream_t s) {
  if (g.p != 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.Z, 0, (size_t)g.L * a.ncol * sizeof(float), s);
  if (e != cudaSuccess) return e;
  SmArgs p;
  p.X = a.X;
  p.Z = a.Z;
  p.W = a.W;
  p.E = a.E;
  p.escale = a.escale;
  p.v = v;
  p.shift_col = a.shift_col;
  p.dm1f = g.dm1f;
  p.perm = perm;
  // even / odd blocks of the (symmetrised) centrosymmetric 1D matrices
  for (int m = 0; m < 2; ++m) {
    const double *M = m == 0 ? g.A : g.B;
    float *e = m == 0 ? p.eA : p.eB, *o = m == 0 ? p.oA : p.oB;
    auto sym = [&](int i, int j) { return 0.5 * (M[i * 5 + j] + M[(4 - i) * 5 + (4 - j)]); };
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k)
        e[i * 3 + k] = (float)(k < 2 ? 0.5 * (sym(i, k) + sym(i, 4 - k)) : sym(i, 2));
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 2; ++k) o[i * 2 + k] = (float)(0.5 * (sym(i, k) - sym(i, 4 - k)));
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
