// FP32 H~X on the CUDA cores for Q4 cells: the exact-FP32 operator of the
// inner MINRES iterations and of the FP32 Chebyshev filter (the TF32
// tensor-core kernel in hx_tc.cu is the alternative for the filter).
//
// Persistent CTAs walk the cells in the slab order of the tensor-core kernel.
// For each (cell, chunk of C columns):
//   * one thread fetches the 5x5x5 x C brick of X with a single 4D TMA tiled
//     load (the unknowns form an Ni^3 grid of node rows, so a cell is a box
//     of that grid; coordinates outside it read as zero, which is the
//     Dirichlet boundary) into a staging buffer, one cell ahead;
//   * K_e = kc (B(x)B(x)A + B(x)A(x)B + A(x)B(x)B) is applied as seven 1D
//     contractions of the cell tensor in shared memory; in each phase a
//     thread owns one 1D line for four adjacent columns, and the 5x5 element
//     matrices (split into even / odd halves, they are centrosymmetric) are
//     kernel parameters that enter the FMAs as constant operands;
//   * the thread of x-line (y, z) scatter-adds that line's five nodes with
//     vector reductions into Z (zeroed by the launcher), adding the nodal
//     term alpha (v - shift) X (+ beta W + alpha escale E) for the nodes the
//     cell owns (local index < 4 on every axis) from the raw X it read.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kQ = 5, kNe = 125;
constexpr long long kSpinLimit = 1LL << 28;   // bounded mbarrier wait

struct SmArgs {
  float *Z;
  const float *X;           // for the W / E nodal terms' addressing only
  const float *W;
  const float *E;           // optional defect block, added as alpha escale_j E
  const double *escale;
  const float *v;           // potential (FP32 copy)
  const double *shift_col;
  const float *dm1f;
  const int *perm;
  int *err;                 // set to 2 when a wait for a TMA brick gives up
  // even / odd blocks of the centrosymmetric 1D matrices (see eo_acc4)
  float eA[9], oA[4], eB[9], oB[4];
  float kc_alpha, alpha, beta, shift;
  int ncol, ncell, Ni;
};

// Threads of a CTA for a chunk of C columns: one per (1D line, column quad)
// task of a contraction phase (25 lines x C/4 quads), rounded to whole warps.
template <int C>
__host__ __device__ constexpr int simt_threads() { return (25 * (C / 4) + 31) / 32 * 32; }

// Column-quad arithmetic on packed FP32 pairs (one instruction per two
// lanes; each lane is the IEEE round-to-nearest operation, so results are
// those of the scalar forms).
__device__ __forceinline__ float2 f4_lo(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 f4_hi(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 f4_cat(const float2 &a, const float2 &b) {
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 f4_fma(float a, const float4 &x, const float4 &y) {
  const float2 aa = make_float2(a, a);
  return f4_cat(__ffma2_rn(aa, f4_lo(x), f4_lo(y)), __ffma2_rn(aa, f4_hi(x), f4_hi(y)));
}
__device__ __forceinline__ float4 f4_add(const float4 &x, const float4 &y) {
  return f4_cat(__fadd2_rn(f4_lo(x), f4_lo(y)), __fadd2_rn(f4_hi(x), f4_hi(y)));
}
// x - y as x + (-1) y: the product is exact, so this is the rounded difference
__device__ __forceinline__ float4 f4_sub(const float4 &x, const float4 &y) {
  const float2 m1 = make_float2(-1.f, -1.f);
  return f4_cat(__ffma2_rn(m1, f4_lo(y), f4_lo(x)), __ffma2_rn(m1, f4_hi(y), f4_hi(x)));
}
__device__ __forceinline__ float4 f4_scale(float a, const float4 &x) {
  const float2 aa = make_float2(a, a);
  return f4_cat(__fmul2_rn(aa, f4_lo(x)), __fmul2_rn(aa, f4_hi(x)));
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
__device__ __forceinline__ uint32_t smem_addr(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}

// wait for phase `parity` of an mbarrier; false when the bounded wait gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  long long spins = 0;
  while (!done) {
    asm volatile(
        "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
        " selp.u32 %0, 1, 0, pw;\n}\n"
        : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (!done && ++spins > kSpinLimit) return false;
  }
  return true;
}

// y = M u for one or more lines u, accumulated on the even (3) and odd (2)
// parts: ye, yo; streamed so that few values stay live.
__device__ __forceinline__ void eo_acc4(const float4 *e, const float4 *o, const float *eM,
                                        const float *oM, float4 *ye, float4 *yo, bool first) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float4 s = first ? make_float4(0.f, 0.f, 0.f, 0.f) : ye[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) s = f4_fma(eM[i * 3 + k], e[k], s);
    ye[i] = s;
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    float4 s = first ? make_float4(0.f, 0.f, 0.f, 0.f) : yo[i];
#pragma unroll
    for (int k = 0; k < 2; ++k) s = f4_fma(oM[i * 2 + k], o[k], s);
    yo[i] = s;
  }
}
// y_i = ye_i + yo_i, y_(4-i) = ye_i - yo_i, y_2 = ye_2, stored at dst[i * stride]
__device__ __forceinline__ void eo_store4(const float4 *ye, const float4 *yo, float4 *dst,
                                          int stride) {
  dst[0] = f4_add(ye[0], yo[0]);
  dst[4 * stride] = f4_sub(ye[0], yo[0]);
  dst[stride] = f4_add(ye[1], yo[1]);
  dst[3 * stride] = f4_sub(ye[1], yo[1]);
  dst[2 * stride] = ye[2];
}

template <int C, bool HW>
__global__ void __launch_bounds__(simt_threads<C>(), 2)
hx_simt_kernel(const __grid_constant__ SmArgs p, const __grid_constant__ CUtensorMap tmx) {
  constexpr int Q4 = C / 4;                  // column quads of a chunk
  constexpr int NT = 25 * Q4;                // tasks of a contraction phase
  constexpr int NTH = simt_threads<C>();
  constexpr uint32_t kBrickBytes = kNe * C * 4;
  extern __shared__ unsigned char sm_raw[];
  // TMA destinations want 128-byte alignment
  float4 *stg = reinterpret_cast<float4 *>(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
  float4 *u = stg + kNe * Q4;      // [125][Q4]
  float4 *w = u + kNe * Q4;        // [125][Q4]
  __shared__ uint64_t mbar;
  __shared__ float dlf[2][3][5];   // d = m^-1/2 along each axis, per staged cell
  __shared__ int abort_flag;
  __shared__ float sshift[kMaxCols], sesc[kMaxCols];
  const int tid = threadIdx.x;
  const int nc = p.ncell, Ni = p.Ni, ncol = p.ncol;
  const int nchunk = (ncol + C - 1) / C;
  const int items = nc * nc * nc * nchunk;
  for (int j = tid; j < ncol; j += NTH) {
    sshift[j] = (float)(p.shift_col ? p.shift_col[j] : p.shift);
    sesc[j] = p.E ? (float)(p.alpha * p.escale[j]) : 0.f;
  }
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const bool act = tid < NT;
  const int q = tid % Q4, l = tid / Q4;      // this thread's line l = ly + 5 lz, quad q
  const int ly = l % 5, lz = l / 5;
  __syncthreads();
  auto locate = [&](int item, int &c0, int &cx, int &cy, int &cz) {
    const int cell = p.perm[item / nchunk];
    c0 = (item % nchunk) * C;
    cx = cell % nc;
    cy = (cell / nc) % nc;
    cz = cell / (nc * nc);
  };
  // stage an item: d tables, the brick by TMA, and the potential of the
  // nodes this thread owns on its x-line (into vn)
  float vn[4] = {0.f, 0.f, 0.f, 0.f};
  auto stage = [&](int item, int buf) {
    int c0, cx, cy, cz;
    locate(item, c0, cx, cy, cz);
    if (tid < 15) {
      const int d = tid / 5, t = tid % 5;
      dlf[buf][d][t] = p.dm1f[(d == 0 ? cx : (d == 1 ? cy : cz)) * 4 + t];
    }
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(smem_addr(&mbar)), "r"(kBrickBytes) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
          " [%0], [%1, {%2, %3, %4, %5}], [%6];"
          :: "r"(smem_addr(stg)), "l"(&tmx), "r"(c0), "r"(4 * cx - 1), "r"(4 * cy - 1),
             "r"(4 * cz - 1), "r"(smem_addr(&mbar))
          : "memory");
    }
    const int gy = 4 * cy - 1 + ly, gz = 4 * cz - 1 + lz;
#pragma unroll
    for (int x = 0; x < 4; ++x) vn[x] = 0.f;
    if (act && ly < 4 && lz < 4 && gy >= 0 && gz >= 0) {
      const int row = Ni * (gy + Ni * gz) + 4 * cx - 1;
#pragma unroll
      for (int x = 0; x < 4; ++x)
        vn[x] = (4 * cx - 1 + x >= 0) ? __ldg(p.v + row + x) : 0.f;
    }
  };
  if ((int)blockIdx.x < items) stage(blockIdx.x, 0);
  int it = 0;
  for (int item = blockIdx.x; item < items; item += gridDim.x, ++it) {
    const int buf = it & 1;
    int c0, cx, cy, cz;
    locate(item, c0, cx, cy, cz);
    if (!mbar_wait(&mbar, (uint32_t)(it & 1))) abort_flag = 1;
    __syncthreads();
    if (abort_flag) break;
    float vc[4] = {vn[0], vn[1], vn[2], vn[3]};
    // x lines (nodes 5 l .. 5 l + 4) from the raw brick, scaled by d:
    // u <- B_x u, w <- A_x u; the nodal term of the owned nodes is kept
    float4 nod[4];
    if (act) {
      const float syz = dlf[buf][1][ly] * dlf[buf][2][lz];
      float4 in[kQ], e[3], o[2];
#pragma unroll
      for (int x = 0; x < kQ; ++x) {
        const float4 r = stg[(5 * l + x) * Q4 + q];
        const float sc = dlf[buf][0][x] * syz;
        in[x] = f4_scale(sc, r);
        if (x < 4) {
          const int col = min(c0 + 4 * q, ncol - 4);
          nod[x] = make_float4(p.alpha * (vc[x] - sshift[col]) * r.x,
                               p.alpha * (vc[x] - sshift[col + 1]) * r.y,
                               p.alpha * (vc[x] - sshift[col + 2]) * r.z,
                               p.alpha * (vc[x] - sshift[col + 3]) * r.w);
        }
      }
      eo_split4(in, e, o);
      float4 ye[3], yo[2];
      eo_acc4(e, o, p.eB, p.oB, ye, yo, true);
      eo_store4(ye, yo, u + 5 * l * Q4 + q, Q4);
      eo_acc4(e, o, p.eA, p.oA, ye, yo, true);
      eo_store4(ye, yo, w + 5 * l * Q4 + q, Q4);
    }
    __syncthreads();
    // the staging buffer is free: fetch the next cell while this one finishes
    if (item + (int)gridDim.x < items) stage(item + gridDim.x, buf ^ 1);
    // y lines (l = x + 5 z): u <- B_y u, w <- A_y u + B_y w
    if (act) {
      const int lb = (l % 5) + 25 * (l / 5);
      float4 t[kQ], e[3], o[2], ye[3], yo[2];
#pragma unroll
      for (int y = 0; y < kQ; ++y) t[y] = u[(lb + 5 * y) * Q4 + q];
      eo_split4(t, e, o);
      eo_acc4(e, o, p.eB, p.oB, ye, yo, true);
      eo_store4(ye, yo, u + lb * Q4 + q, 5 * Q4);
      eo_acc4(e, o, p.eA, p.oA, ye, yo, true);
#pragma unroll
      for (int y = 0; y < kQ; ++y) t[y] = w[(lb + 5 * y) * Q4 + q];
      eo_split4(t, e, o);
      eo_acc4(e, o, p.eB, p.oB, ye, yo, false);
      eo_store4(ye, yo, w + lb * Q4 + q, 5 * Q4);
    }
    __syncthreads();
    // z lines (l = x + 5 y): u <- A_z u + B_z w
    if (act) {
      float4 t[kQ], e[3], o[2], ye[3], yo[2];
#pragma unroll
      for (int z = 0; z < kQ; ++z) t[z] = u[(l + 25 * z) * Q4 + q];
      eo_split4(t, e, o);
      eo_acc4(e, o, p.eA, p.oA, ye, yo, true);
#pragma unroll
      for (int z = 0; z < kQ; ++z) t[z] = w[(l + 25 * z) * Q4 + q];
      eo_split4(t, e, o);
      eo_acc4(e, o, p.eB, p.oB, ye, yo, false);
      eo_store4(ye, yo, u + l * Q4 + q, 25 * Q4);
    }
    __syncthreads();
    // epilogue: the five nodes of this thread's x-line
    if (act) {
      const int gy = 4 * cy - 1 + ly, gz = 4 * cz - 1 + lz;
      const int col = c0 + 4 * q;
      if (gy >= 0 && gy < Ni && gz >= 0 && gz < Ni && col < ncol) {
        const float syz = p.kc_alpha * dlf[buf][1][ly] * dlf[buf][2][lz];
        const bool own_yz = ly < 4 && lz < 4;
        const uint32_t row = (uint32_t)(Ni * (gy + Ni * gz) + 4 * cx - 1);
#pragma unroll
        for (int x = 0; x < kQ; ++x) {
          const int gx = 4 * cx - 1 + x;
          if (gx < 0 || gx >= Ni) continue;
          const uint32_t e0 = (row + x) * (uint32_t)ncol + (uint32_t)col;
          const float sc = syz * dlf[buf][0][x];
          const float4 y = u[(5 * l + x) * Q4 + q];
          float4 o = f4_scale(sc, y);
          if (x < 4 && own_yz) {
            o = f4_add(o, nod[x]);
            if (HW) {
              const float4 w4 = *reinterpret_cast<const float4 *>(p.W + e0);
              o.x = fmaf(p.beta, w4.x, o.x);
              o.y = fmaf(p.beta, w4.y, o.y);
              o.z = fmaf(p.beta, w4.z, o.z);
              o.w = fmaf(p.beta, w4.w, o.w);
            }
            if (p.E) {
              const float4 e4 = __ldg(reinterpret_cast<const float4 *>(p.E + e0));
              o.x = fmaf(sesc[col], e4.x, o.x);
              o.y = fmaf(sesc[col + 1], e4.y, o.y);
              o.z = fmaf(sesc[col + 2], e4.z, o.z);
              o.w = fmaf(sesc[col + 3], e4.w, o.w);
            }
          }
          // no "memory" clobber: nothing in this kernel reads Z
          asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                       :: "l"(p.Z + e0), "f"(o.x), "f"(o.y), "f"(o.z), "f"(o.w));
        }
      }
    }
  }
  if (abort_flag) {
    // a brick never arrived: report, and give a copy still in flight a
    // bounded chance to land before the CTA's shared memory is released
    if (tid == 0) {
      atomicExch(p.err, 2);
      mbar_wait(&mbar, (uint32_t)(it & 1));
    }
  }
}

template <int C, bool HW>
cudaError_t run_simt(const SmArgs &p, const CUtensorMap &tm, long long items, cudaStream_t s) {
  const size_t smem = 3 * (size_t)kNe * C * sizeof(float) + 128;
  auto k = hx_simt_kernel<C, HW>;
  cudaError_t e = raise_smem_limit(k, (int)smem);
  if (e != cudaSuccess) return e;
  // resident CTAs per SM: queried once per kernel variant (no device queries
  // while a stream may be capturing a graph)
  static const int resident = [&] {
    int nsm = 148, per_sm = 1;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, simt_threads<C>(), smem) !=
        cudaSuccess)
      per_sm = 1;
    return nsm * std::max(per_sm, 1);
  }();
  const int grid = (int)std::min<long long>(items, (long long)resident);
  ::invdft::count_launch();
  k<<<grid, simt_threads<C>(), smem, s>>>(p, tm);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled, looked up through the runtime so that the library
// loads on hosts without the driver (it is only called with a GPU present)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

}  // namespace

// FP32 CUDA-core H~X for Q4 meshes (W and E optional), ncol a multiple of 4
// (16-byte node rows for the TMA brick loads).  Z must not alias X, W or E;
// it is zeroed here.  err: device word set to 2 if a brick load timed out.
cudaError_t launch_hx_simt_q4(const Geom &g, const float *v, const HxArgs<float> &a,
                              const int *perm, int *err, cudaStream_t s) {
  if (g.p != 4 || a.ncol % 4 != 0 || a.ncol > kMaxCols) return cudaErrorInvalidValue;
  if (((uintptr_t)a.X & 15) != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(a.Z, 0, (size_t)g.L * a.ncol * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const int C = a.ncol <= 16 ? 16 : (a.ncol <= 32 ? 32 : 64);
  // X as a 4D tensor (column, x, y, z) of the interior node grid; box = one
  // cell's 5 x 5 x 5 nodes by C columns
  CUtensorMap tm;
  const cuuint64_t dims[4] = {(cuuint64_t)a.ncol, (cuuint64_t)g.Ni, (cuuint64_t)g.Ni,
                              (cuuint64_t)g.Ni};
  const cuuint64_t row = (cuuint64_t)a.ncol * sizeof(float);
  const cuuint64_t strides[3] = {row, row * g.Ni, row * g.Ni * g.Ni};
  const cuuint32_t box[4] = {(cuuint32_t)C, 5, 5, 5};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, (void *)a.X, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  SmArgs p;
  p.Z = a.Z;
  p.X = a.X;
  p.W = a.W;
  p.E = a.E;
  p.escale = a.escale;
  p.v = v;
  p.shift_col = a.shift_col;
  p.dm1f = g.dm1f;
  p.perm = perm;
  p.err = err;
  // even / odd blocks of the (symmetrised) centrosymmetric 1D matrices
  for (int m = 0; m < 2; ++m) {
    const double *M = m == 0 ? g.A : g.B;
    float *ev = m == 0 ? p.eA : p.eB, *ov = m == 0 ? p.oA : p.oB;
    auto sym = [&](int i, int j) { return 0.5 * (M[i * 5 + j] + M[(4 - i) * 5 + (4 - j)]); };
    for (int i = 0; i < 3; ++i)
      for (int k = 0; k < 3; ++k)
        ev[i * 3 + k] = (float)(k < 2 ? 0.5 * (sym(i, k) + sym(i, 4 - k)) : sym(i, 2));
    for (int i = 0; i < 2; ++i)
      for (int k = 0; k < 2; ++k) ov[i * 2 + k] = (float)(0.5 * (sym(i, k) - sym(i, 4 - k)));
  }
  p.kc_alpha = (float)(g.kc * a.alpha);
  p.alpha = (float)a.alpha;
  p.beta = (float)a.beta;
  p.shift = (float)a.shift;
  p.ncol = a.ncol;
  p.ncell = g.ncell;
  p.Ni = g.Ni;
  const long long items = (long long)g.ncell * g.ncell * g.ncell * ((a.ncol + C - 1) / C);
  if (C == 16) return a.W ? run_simt<16, true>(p, tm, items, s) : run_simt<16, false>(p, tm, items, s);
  if (C == 32) return a.W ? run_simt<32, true>(p, tm, items, s) : run_simt<32, false>(p, tm, items, s);
  return a.W ? run_simt<64, true>(p, tm, items, s) : run_simt<64, false>(p, tm, items, s);
}

}  // namespace invdft
