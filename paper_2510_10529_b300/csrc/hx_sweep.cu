// H~X in the owner-computes sweep form (Eq. 17, Eq. 19, Sec. 3.2.3), FP32 and
// FP64, for tensor-product meshes of order p in {2, 4, 6}, equal or graded cells.
//
// On a tensor-product mesh the cell matrix is a sum of Kronecker products,
// K_e = 1/2 (B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x),
// with per-axis 1D stiffness A = (2/h) A_ref and consistent mass B = (h/2) B_ref,
// and the cells form a product set.  So the *assembled* operator has the same
// form with the assembled 1D matrices (banded, one (p+1)x(p+1) block per cell,
// overlapping at the cell vertices), and with D = d1 (x) d1 (x) d1:
//   D K D X = 1/2 [B^z B^y A^x + B^z A^y B^x + A^z B^y B^x] X,
// hats meaning d1 M d1.  It is applied as seven banded sweeps:
//   Px = A^x X, Qx = B^x X;   R = B^y Px + A^y Qx, S = B^y Qx;
//   Y  = 1/2 (B^z R + A^z S)  (+ the nodal terms).
// This is the same matrix as the cell-by-cell gather / K_e X_e / scatter-add,
// up to rounding, but every node is computed once by its owner: no zero fill
// of the output, no atomics, no read-back of partial sums.
//
// Decomposition.  A CTA owns a TX x TY column of nodes and C columns of the
// block and streams through z one node plane at a time:
//   * one thread loads the plane's (TX+p+1) x (TY+p+1) x C tile (the owned
//     nodes, the low vertex and one cell of halo on the high side) with one 4D
//     TMA tiled load, NST planes ahead; coordinates outside the unknown grid
//     read as zero, which is the Dirichlet boundary;
//   * x sweep: each task takes one x-cell of one row (p+1 nodes, even/odd
//     halves of the centrosymmetric cell blocks) and writes Px, Qx at the cell's
//     nodes 1..p; node p (the vertex) also takes row 0 of the next cell;
//   * y sweep: each thread takes one y-cell of one owned x for a column pair,
//     the same way, and keeps R, S for its p nodes in registers;
//   * z: the thread accumulates Y for the p+1 planes of the current z-cell,
//     acc[i] += B^z[i][kz] R + A^z[i][kz] S, adds the nodal term
//     alpha (v - shift_j) X_j of the plane, and at each vertex plane writes the
//     finished planes of the cell (+ beta W + alpha escale_j E) with plain
//     coalesced stores and carries the vertex plane into the next cell.
// Optionally the z range is split into segments; a segment owns the planes
// above its bottom vertex up to and including its top vertex, which takes
// row 0 of the next cell from p extra planes.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "internal.h"

namespace invdft {
namespace {

constexpr long long kSweepSpin = 1LL << 28;   // polls before a TMA wait gives up

// The columns a thread carries: VW = 2 (a column pair, packed FP32 or two
// FP64 lanes) or VW = 1 (one column, scalar arithmetic).
template <typename T, int VW> struct VecOf;
template <> struct VecOf<float, 2> { using type = float2; };
template <> struct VecOf<double, 2> { using type = double2; };
template <> struct VecOf<float, 1> { using type = float; };
template <> struct VecOf<double, 1> { using type = double; };

// column-pair arithmetic: packed FP32 pairs (each lane an IEEE round-to-nearest
// operation) or two FP64 operations
__device__ __forceinline__ float2 vfma(float a, float2 x, float2 y) {
  return __ffma2_rn(make_float2(a, a), x, y);
}
__device__ __forceinline__ double2 vfma(double a, double2 x, double2 y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float2 vmul(float a, float2 x) { return __fmul2_rn(make_float2(a, a), x); }
__device__ __forceinline__ double2 vmul(double a, double2 x) { return make_double2(a * x.x, a * x.y); }
__device__ __forceinline__ float2 vadd(float2 x, float2 y) { return __fadd2_rn(x, y); }
__device__ __forceinline__ double2 vadd(double2 x, double2 y) {
  return make_double2(x.x + y.x, x.y + y.y);
}
// x - y as x + (-1) y: the product is exact
__device__ __forceinline__ float2 vsub(float2 x, float2 y) {
  return __ffma2_rn(make_float2(-1.f, -1.f), y, x);
}
__device__ __forceinline__ double2 vsub(double2 x, double2 y) {
  return make_double2(x.x - y.x, x.y - y.y);
}
// elementwise a * x + y
__device__ __forceinline__ float2 vfmav(float2 a, float2 x, float2 y) { return __ffma2_rn(a, x, y); }
__device__ __forceinline__ double2 vfmav(double2 a, double2 x, double2 y) {
  return make_double2(fma(a.x, x.x, y.x), fma(a.y, x.y, y.y));
}
// FP32 coefficients are stored as duplicated pairs so that a packed FMA takes
// them straight from the parameter space; FP64 ones as scalars
__device__ __forceinline__ float2 vfma(float2 a, float2 x, float2 y) { return __ffma2_rn(a, x, y); }
__device__ __forceinline__ float2 vmul(float2 a, float2 x) { return __fmul2_rn(a, x); }
template <typename T, int VW> struct CoefOf;
template <> struct CoefOf<float, 2> {
  using type = float2;
  static float2 make(double x) { return make_float2((float)x, (float)x); }
};
template <> struct CoefOf<float, 1> {
  using type = float;
  static float make(double x) { return (float)x; }
};
template <int VW> struct CoefOf<double, VW> {
  using type = double;
  static double make(double x) { return x; }
};
// scalar (one column per thread) forms
__device__ __forceinline__ float vfma(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ double vfma(double a, double x, double y) { return fma(a, x, y); }
__device__ __forceinline__ float vmul(float a, float x) { return a * x; }
__device__ __forceinline__ double vmul(double a, double x) { return a * x; }
__device__ __forceinline__ float vadd(float x, float y) { return x + y; }
__device__ __forceinline__ double vadd(double x, double y) { return x + y; }
__device__ __forceinline__ float vsub(float x, float y) { return x - y; }
__device__ __forceinline__ double vsub(double x, double y) { return x - y; }
__device__ __forceinline__ float vfmav(float a, float x, float y) { return fmaf(a, x, y); }
__device__ __forceinline__ double vfmav(double a, double x, double y) { return fma(a, x, y); }
// VW consecutive values of a per-column table / block as one V
template <typename V, typename T> __device__ __forceinline__ V vload(const T *p);
template <> __device__ __forceinline__ float2 vload<float2, float>(const float *p) {
  return make_float2(p[0], p[1]);
}
template <> __device__ __forceinline__ double2 vload<double2, double>(const double *p) {
  return make_double2(p[0], p[1]);
}
template <> __device__ __forceinline__ float vload<float, float>(const float *p) { return p[0]; }
template <> __device__ __forceinline__ double vload<double, double>(const double *p) { return p[0]; }
// s - v per lane
__device__ __forceinline__ float2 vrsub(float s, float2 v) { return make_float2(s - v.x, s - v.y); }
__device__ __forceinline__ double2 vrsub(double s, double2 v) { return make_double2(s - v.x, s - v.y); }
__device__ __forceinline__ float vrsub(float s, float v) { return s - v; }
__device__ __forceinline__ double vrsub(double s, double v) { return s - v; }
// the defect block E (FP32) at VW columns
template <typename V> __device__ __forceinline__ V eload(const float *p);
template <> __device__ __forceinline__ float2 eload<float2>(const float *p) {
  return __ldg(reinterpret_cast<const float2 *>(p));
}
template <> __device__ __forceinline__ float eload<float>(const float *p) { return __ldg(p); }
template <typename V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float vzero<float>() { return 0.f; }
template <> __device__ __forceinline__ double vzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 vzero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

// Coefficients passed by value (kernel parameter space).  x and y: even / odd
// blocks of the d-scaled centrosymmetric cell blocks (see split / apply);
// z: the dense d-scaled blocks with alpha / 2 folded in, [i][k].
template <typename CT, int P>
struct SweepCoef {
  static constexpr int H = P / 2, NE = (H + 1) * (H + 1), NO = H * H, Q = P + 1;
  CT eAx[NE], oAx[NO], eBx[NE], oBx[NO];
  CT eAy[NE], oAy[NO], eBy[NE], oBy[NO];
  CT Az[Q * Q], Bz[Q * Q];
  // row 0 of the (symmetrised) x and y blocks, for the contribution of the
  // next cell to a vertex node: applied to the raw values it needs no split
  CT rAx[Q], rBx[Q], rAy[Q], rBy[Q];
};

template <typename T, typename CT, int P>
struct SweepArgs {
  SweepCoef<CT, P> cf;
  T *Z;
  const T *W;
  const float *E;
  const double *escale;
  const T *v;                 // potential (FP32 copy on the FP32 path); null: none
  const double *shift_col;
  double shift, alpha, beta;
  int *err;                   // set to 3 when a wait for a TMA plane gives up
  int ncol, nx, ny, nz;       // columns; unknowns per axis
  int ncx, ncy, ncz;          // cells per axis
  int ntx, nty, nchunk, seglen;
  // graded meshes: per axis m1^-1/2 and m1 at every node (boundary included)
  // and the cell scalars 2/h_e (A) and h_e/2 (B)
  const double *dn[3], *m1[3], *cA[3], *cB[3];
};

// tile shape of a variant
template <typename T, int P, int C, int TX, int TY, int XPT, int VW>
struct SweepShape {
  using V = typename VecOf<T, VW>::type;
  static constexpr int H = P / 2, NCP = C / VW, RX = TX + P + 1, RY = TY + P + 1;
  static constexpr int NJX = TX / P, NJY = TY / P, NTH = TX * NJY * NCP;
  // x tasks: XPT consecutive x-cells of one row for one column pair
  static constexpr int NXT = NJX / XPT;
  static constexpr int NTASKX = RY * NXT * NCP;
  static constexpr int STAGE_V = RX * RY * NCP;            // V of one plane tile
  // stages start on 128-byte boundaries (TMA destinations)
  static constexpr int STAGE_STRIDE_V = ((STAGE_V * (int)sizeof(V) + 127) / 128 * 128) / (int)sizeof(V);
  // Px / Qx rows: pad so that consecutive rows start SEG_B bytes apart modulo
  // 128 (a warp holding several rows of SEG_B-byte node segments hits
  // distinct banks)
  static constexpr int SEG_B = NCP * (int)sizeof(V);
  static constexpr int ROW_B = TX * SEG_B;
  static constexpr int PAD_B = ((SEG_B - ROW_B % 128) % 128 + 128) % 128;
  static constexpr int PXS = (ROW_B + PAD_B) / (int)sizeof(V);
  static constexpr size_t smem(int nst) {
    return 128 + (size_t)nst * STAGE_STRIDE_V * sizeof(V) + 4 * (size_t)RY * PXS * sizeof(V);
  }
  static_assert(TX % P == 0 && TY % P == 0 && C % VW == 0 && (TX / P) % XPT == 0, "tile shape");
  static_assert((PAD_B % (int)sizeof(V)) == 0, "row padding");
};

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ bool wait_parity(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  long long spins = 0;
  while (!done) {
    asm volatile(
        "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
        " selp.u32 %0, 1, 0, pw;\n}\n"
        : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (!done && ++spins > kSweepSpin) return false;
  }
  return true;
}
__device__ __forceinline__ void load_plane(const CUtensorMap *tm, void *dst, uint64_t *bar,
                                           uint32_t bytes, int c0, int x, int y, int z) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               :: "r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];"
      :: "r"(smem_u32(dst)), "l"(tm), "r"(c0), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// even / odd halves of p+1 values: e_k = u_k + u_(p-k), o_k = u_k - u_(p-k)
// (k < p/2), e_(p/2) = u_(p/2)
template <int P, typename V>
__device__ __forceinline__ void split(const V *u, V *e, V *o) {
  constexpr int H = P / 2;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    e[k] = vadd(u[k], u[P - k]);
    o[k] = vsub(u[k], u[P - k]);
  }
  e[H] = u[H];
}
// y = M1 u1 (+ M2 u2) at local nodes 1..p (out[i-1]) from the even / odd
// halves: y_i = ye_i + yo_i, y_(p-i) = ye_i - yo_i, y_(p/2) = ye_(p/2); with
// LOC0 also local node 0 (*loc0 = ye_0 + yo_0)
template <int P, bool TWO, bool LOC0, typename CT, typename V>
__device__ __forceinline__ void apply_hi(const V *e1, const V *o1, const CT *eM1, const CT *oM1,
                                         const V *e2, const V *o2, const CT *eM2, const CT *oM2,
                                         V *out, V *loc0) {
  constexpr int H = P / 2;
  V ye[H + 1], yo[H > 0 ? H : 1];
#pragma unroll
  for (int i = 0; i <= H; ++i) {
    V s = vmul(eM1[i * (H + 1)], e1[0]);
#pragma unroll
    for (int k = 1; k <= H; ++k) s = vfma(eM1[i * (H + 1) + k], e1[k], s);
    if (TWO) {
#pragma unroll
      for (int k = 0; k <= H; ++k) s = vfma(eM2[i * (H + 1) + k], e2[k], s);
    }
    ye[i] = s;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    V s = vmul(oM1[i * H], o1[0]);
#pragma unroll
    for (int k = 1; k < H; ++k) s = vfma(oM1[i * H + k], o1[k], s);
    if (TWO) {
#pragma unroll
      for (int k = 0; k < H; ++k) s = vfma(oM2[i * H + k], o2[k], s);
    }
    yo[i] = s;
  }
#pragma unroll
  for (int i = 1; i <= P; ++i) {
    if (i < H) out[i - 1] = vadd(ye[i], yo[i]);
    else if (i == H) out[i - 1] = ye[H];
    else out[i - 1] = vsub(ye[P - i], yo[P - i]);
  }
  if (LOC0) *loc0 = vadd(ye[0], yo[0]);
}
// row 0 of M u from the raw values: sum_k r_k u_k
template <int P, typename CT, typename V>
__device__ __forceinline__ V row0d(const V *u, const CT *r, V acc) {
#pragma unroll
  for (int k = 0; k <= P; ++k) acc = vfma(r[k], u[k], acc);
  return acc;
}

// GR (graded meshes): the cell blocks are not all equal, so the coefficients
// are the reference blocks; X is scaled by D = d_x d_y d_z as it enters the x
// sweep, each cell's outputs by its scalars 2/h_e (A) or h_e/2 (B), and the
// result by D at the output (the nodal term is carried divided by D).
// BAL: the balanced schedule -- a persistent grid in which every CTA first
// takes whole (tile, chunk) units round-robin and then an equal share of the
// z-cells of the units left over; otherwise one (tile, chunk, z segment) item
// per CTA.
template <typename T, int P, int C, int TX, int TY, int NST, int XPT, int MINB, int VW, bool HW,
          bool HE, bool GR, bool BAL>
__global__ void __launch_bounds__(SweepShape<T, P, C, TX, TY, XPT, VW>::NTH, MINB)
hx_sweep_kernel(const __grid_constant__ SweepArgs<T, typename CoefOf<T, VW>::type, P> p,
                const __grid_constant__ CUtensorMap tmx) {
  using S = SweepShape<T, P, C, TX, TY, XPT, VW>;
  using V = typename S::V;
  using CT = typename CoefOf<T, VW>::type;
  constexpr int H = S::H, NCP = S::NCP, RX = S::RX, RY = S::RY, NTH = S::NTH, PXS = S::PXS;
  constexpr uint32_t kStageBytes = (uint32_t)(S::STAGE_V * sizeof(V));
  static_assert(!HE || std::is_same<T, float>::value, "the defect block is FP32");
  extern __shared__ unsigned char sm_raw[];
  V *stage0 = reinterpret_cast<V *>(((uintptr_t)sm_raw + 127) & ~(uintptr_t)127);
  // two Px / Qx buffers (plane it & 1), each Px followed by Qx
  V *Px = stage0 + NST * S::STAGE_STRIDE_V;
  V *Qx = Px + RY * PXS;
  __shared__ __align__(8) uint64_t full[NST];
  __shared__ T sash[C], sesc[C];
  __shared__ int abort_flag;
  // potential at the owned nodes of a plane, one plane ahead: element copies
  // (cp.async) into a two-plane ring, completed before the barrier that
  // precedes their use; zero where there is no potential or no unknown
  __shared__ __align__(16) T vring[2][TX * TY];
  const SweepCoef<CT, P> &cf = p.cf;
  const int tid = threadIdx.x;

  // Work: segments (unit, z-cells [n0, n1)), a unit being a (tile, column
  // chunk) pair numbered tile-fastest.  Per-item launches take one segment
  // from the block index; the balanced form walks its list.
  const int ntiles = p.ntx * p.nty;
  const int nunit = ntiles * p.nchunk;
  const int nfull = BAL ? nunit / (int)gridDim.x : 0;            // round-robin whole units
  int rlo = 0, rhi = 0;                                          // share of the rest, (unit, cell) order
  if constexpr (BAL) {
    const long long rest = (long long)(nunit - nfull * (int)gridDim.x) * p.ncz;
    rlo = (int)(rest * blockIdx.x / gridDim.x);
    rhi = (int)(rest * (blockIdx.x + 1) / gridDim.x);
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < NST; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // planes consumed by earlier segments: plane it of this segment is the
  // (gbase + it)-th load of the CTA, in stage (gbase + it) % NST, and its wait
  // parity is ((gbase + it) / NST) & 1
  int gbase = 0;
  int it = 0, nplanes = 0;
  for (int kseg = 0; BAL ? !abort_flag : kseg == 0; ++kseg) {
    int unit, n0, n1;
    if constexpr (!BAL) {
      int item = blockIdx.x;
      unit = item % ntiles;
      item /= ntiles;
      unit += ntiles * (item % p.nchunk);
      n0 = (item / p.nchunk) * p.seglen;
      n1 = min(p.ncz, n0 + p.seglen);
    } else if (kseg < nfull) {
      unit = blockIdx.x + kseg * gridDim.x;
      n0 = 0;
      n1 = p.ncz;
    } else {
      if (rlo >= rhi) break;
      unit = nfull * gridDim.x + rlo / p.ncz;
      n0 = rlo % p.ncz;
      n1 = min(p.ncz, n0 + (rhi - rlo));
      rlo += n1 - n0;
    }
    const int tile = unit % ntiles, chunk = unit / ntiles;
    const int gx0 = (tile % p.ntx) * TX, gy0 = (tile / p.ntx) * TY;  // owned index 0, unknown coords
    const int c0 = chunk * C;
    const int gz_begin = n0 == 0 ? 1 : n0 * P;            // node planes (0 = boundary)
    const int gz_end = n1 * P;
    const int extra = n1 < p.ncz ? P : 0;
    nplanes = gz_end + extra - gz_begin + 1;

    for (int j = tid; j < C; j += NTH) {
      const int col = c0 + j;
      const bool in = col < p.ncol;
      const double sh = in ? (p.shift_col ? p.shift_col[col] : p.shift) : 0.0;
      sash[j] = (T)(p.alpha * sh);
      sesc[j] = (HE && in) ? (T)(p.alpha * p.escale[col]) : (T)0;
    }
    auto fetch_v = [&](int gzp, int buf) {
      const int uz = gzp - 1;
      for (int e = tid; e < TX * TY; e += NTH) {
        const int lx = e % TX, ly = e / TX;
        const int vx = gx0 + lx, vy = gy0 + ly;
        T *dst = &vring[buf][e];
        if (p.v && uz >= 0 && uz < p.nz && vx < p.nx && vy < p.ny)
          asm volatile("cp.async.ca.shared.global [%0], [%1], %2;"
                       :: "r"(smem_u32(dst)),
                          "l"(p.v + (size_t)vx + (size_t)p.nx * ((size_t)vy + (size_t)p.ny * uz)),
                          "n"((int)sizeof(T)) : "memory");
        else
          *dst = (T)0;
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    fetch_v(gz_begin, 0);
    if (tid == 0) {
      // every stage is free: the previous segment's readers passed its last barrier
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int s = 0; s < NST && s < nplanes; ++s) {
        const int st = (gbase + s) % NST;
        load_plane(&tmx, stage0 + st * S::STAGE_STRIDE_V, &full[st], kStageBytes, c0, gx0 - 1,
                   gy0 - 1, gz_begin + s - 1);
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    // this thread's y/z task: owned x, a y-cell, a column pair
    const int cv = tid % NCP;
    const int ox = (tid / NCP) % TX;
    const int jy = tid / (NCP * TX);
    const int ux = gx0 + ox;
    const int colp = c0 + VW * cv;
    const bool cx_in = ux < p.nx && colp < p.ncol;
    const V ash = vload<V>(sash + VW * cv), esc = vload<V>(sesc + VW * cv);
    const T alpha = (T)p.alpha, beta = (T)p.beta;
    // graded meshes: D and D^-1 = sqrt(m) of the thread's nodes in x and y
    T dxy[P], sxy[P];
    if constexpr (GR) {
      const int gx = min(ux + 1, p.nx + 1);
#pragma unroll
      for (int yi = 0; yi < P; ++yi) {
        const int gy = min(gy0 + jy * P + yi + 1, p.ny + 1);
        dxy[yi] = (T)(p.dn[0][gx] * p.dn[1][gy]);
        sxy[yi] = (T)(p.m1[0][gx] * p.dn[0][gx] * p.m1[1][gy] * p.dn[1][gy]);
      }
    }
    V acc[P + 1][P];
#pragma unroll
    for (int i = 0; i <= P; ++i)
#pragma unroll
      for (int k = 0; k < P; ++k) acc[i][k] = vzero<V>();

    // store the finished plane g (node numbering) of the thread's nodes
    auto emit = [&](int g, const V *a) {
      const int uz = g - 1;
#pragma unroll
      for (int yi = 0; yi < P; ++yi) {
        const int uy = gy0 + jy * P + yi;
        if (cx_in && uy < p.ny) {
          const size_t off = ((size_t)ux + (size_t)p.nx * ((size_t)uy + (size_t)p.ny * uz)) * p.ncol + colp;
          V val = a[yi];
          if constexpr (GR) val = vmul((T)(dxy[yi] * p.dn[2][g]), val);
          // graded meshes add beta W + E here; uniform ones fold them into the
          // nodal term of their plane
          if constexpr (HW && GR) val = vfma(beta, *reinterpret_cast<const V *>(p.W + off), val);
          if constexpr (HE && GR) val = vfmav(esc, eload<V>(p.E + off), val);
          *reinterpret_cast<V *>(p.Z + off) = val;
        }
      }
    };

    // x sweep of one plane: Px = A^x X, Qx = B^x X at the owned x of every row;
    // a task takes XPT consecutive x-cells of a row (the shared vertices are
    // summed in registers) and row 0 of the cell after them
    auto xsweep = [&](const V *xs, V *Pw, V *Qw, int gzp) {
      const T dz = GR ? (T)p.dn[2][gzp] : (T)1;
      for (int t = tid; t < S::NTASKX; t += NTH) {
        const int xcv = t % NCP;
        const int rest = t / NCP;
        const int r = rest % RY;
        const int jt = rest / RY;
        const V *src = xs + (r * RX + jt * XPT * P) * NCP + xcv;
        // graded meshes: D of the inputs along this row, and the x-cells' scalars
        T drow = (T)1;
        int ex0 = 0;
        if constexpr (GR) {
          drow = (T)p.dn[1][min(gy0 + r, p.ny + 1)] * dz;
          ex0 = gx0 / P + jt * XPT;
        }
        auto load_in = [&](V *u, int c) {
#pragma unroll
          for (int i = 0; i <= P; ++i) {
            u[i] = src[(c + i) * NCP];
            if constexpr (GR)
              u[i] = vmul((T)(drow * p.dn[0][min(gx0 + jt * XPT * P + c + i, p.nx + 1)]), u[i]);
          }
        };
        V pa[XPT * P], qb[XPT * P];
#pragma unroll
        for (int q = 0; q < XPT; ++q) {
          V u[P + 1], e[H + 1], o[H > 0 ? H : 1];
          load_in(u, q * P);
          split<P>(u, e, o);
          V la, lb;
          apply_hi<P, false, true>(e, o, cf.eAx, cf.oAx, e, o, cf.eAx, cf.oAx, pa + q * P, &la);
          apply_hi<P, false, true>(e, o, cf.eBx, cf.oBx, e, o, cf.eBx, cf.oBx, qb + q * P, &lb);
          if constexpr (GR) {
            const int ec = min(ex0 + q, p.ncx - 1);
            const T sa = (T)p.cA[0][ec], sb = (T)p.cB[0][ec];
#pragma unroll
            for (int i = 0; i < P; ++i) {
              pa[q * P + i] = vmul(sa, pa[q * P + i]);
              qb[q * P + i] = vmul(sb, qb[q * P + i]);
            }
            la = vmul(sa, la);
            lb = vmul(sb, lb);
          }
          if (q > 0) {
            pa[q * P - 1] = vadd(pa[q * P - 1], la);
            qb[q * P - 1] = vadd(qb[q * P - 1], lb);
          }
        }
        {
          V u[P + 1];
          load_in(u, XPT * P);
          if constexpr (GR) {
            const int ec = min(ex0 + XPT, p.ncx - 1);
            pa[XPT * P - 1] = vfma((T)p.cA[0][ec], row0d<P>(u, cf.rAx, vzero<V>()), pa[XPT * P - 1]);
            qb[XPT * P - 1] = vfma((T)p.cB[0][ec], row0d<P>(u, cf.rBx, vzero<V>()), qb[XPT * P - 1]);
          } else {
            pa[XPT * P - 1] = row0d<P>(u, cf.rAx, pa[XPT * P - 1]);
            qb[XPT * P - 1] = row0d<P>(u, cf.rBx, qb[XPT * P - 1]);
          }
        }
        V *dp = Pw + r * PXS + jt * XPT * P * NCP + xcv;
        V *dq = Qw + r * PXS + jt * XPT * P * NCP + xcv;
#pragma unroll
        for (int i = 0; i < XPT * P; ++i) {
          dp[i * NCP] = pa[i];
          dq[i * NCP] = qb[i];
        }
      }
    };

    // prologue: x sweep of the first plane
    {
      const int st = gbase % NST;
      if (!wait_parity(&full[st], (uint32_t)((gbase / NST) & 1))) abort_flag = 1;
      xsweep(stage0 + st * S::STAGE_STRIDE_V, Px, Qx, gz_begin);
    }
    __syncthreads();
    // One barrier per plane: the y / z work of plane it (reading Px / Qx buffer
    // it & 1 and the X stage of plane it) and the x sweep of plane it + 1 (into
    // the other buffer) run between two barriers.
    for (it = 0; it < nplanes && !abort_flag; ++it) {
      const int gz = gz_begin + it;
      const int s = (gbase + it) % NST;
      const V *stg = stage0 + s * S::STAGE_STRIDE_V;
      const V *Pr = Px + (it & 1) * 2 * RY * PXS;
      const V *Qr = Pr + RY * PXS;
      // potential of the next plane into the other ring slot (its readers
      // passed the last barrier); this plane's from the ring
      if (it + 1 < nplanes) fetch_v(gz + 1, (it + 1) & 1);
      T vv[P];
#pragma unroll
      for (int yi = 0; yi < P; ++yi) vv[yi] = vring[it & 1][(jy * P + yi) * TX + ox];
      // uniform meshes: W and E of this plane at the thread's owned nodes, loaded
      // here and consumed with the nodal term after the y sweep
      constexpr bool kFold = (HW || HE) && !GR;
      V wr[kFold ? P : 1], er[kFold ? P : 1];
      if constexpr (kFold) {
        const int uz = gz - 1;
        const bool own = gz > n0 * P && gz <= gz_end && uz < p.nz;
#pragma unroll
        for (int yi = 0; yi < P; ++yi) {
          const int uy = gy0 + jy * P + yi;
          wr[yi] = vzero<V>();
          er[yi] = vzero<V>();
          if (own && cx_in && uy < p.ny) {
            const size_t off = ((size_t)ux + (size_t)p.nx * ((size_t)uy + (size_t)p.ny * uz)) * p.ncol + colp;
            if constexpr (HW) wr[yi] = *reinterpret_cast<const V *>(p.W + off);
            if constexpr (HE) er[yi] = eload<V>(p.E + off);
          }
        }
      }

      // ---- y sweep: R = B^y Px + A^y Qx, S = B^y Qx at this thread's p nodes
      V R[P], Sv[P];
      {
        const V *sp = Pr + jy * P * PXS + ox * NCP + cv;
        const V *sq = Qr + jy * P * PXS + ox * NCP + cv;
        V u[P + 1], w[P + 1], eu[H + 1], ou[H > 0 ? H : 1], ew[H + 1], ow[H > 0 ? H : 1];
#pragma unroll
        for (int i = 0; i <= P; ++i) {
          u[i] = sp[i * PXS];
          w[i] = sq[i * PXS];
        }
        split<P>(u, eu, ou);
        split<P>(w, ew, ow);
        if constexpr (GR) {
          // R = s_B B Px + s_A A Qx, S = s_B B Qx with the y-cell's scalars
          const int ey = min((gy0 + jy * P) / P, p.ncy - 1);
          const T sa = (T)p.cA[1][ey], sb = (T)p.cB[1][ey];
          V Ra[P], Rb[P];
          apply_hi<P, false, false>(eu, ou, cf.eBy, cf.oBy, eu, ou, cf.eBy, cf.oBy, Rb, Rb);
          apply_hi<P, false, false>(ew, ow, cf.eAy, cf.oAy, ew, ow, cf.eAy, cf.oAy, Ra, Ra);
          apply_hi<P, false, false>(ew, ow, cf.eBy, cf.oBy, ew, ow, cf.eBy, cf.oBy, Sv, Sv);
#pragma unroll
          for (int i = 0; i < P; ++i) {
            R[i] = vfma(sb, Rb[i], vmul(sa, Ra[i]));
            Sv[i] = vmul(sb, Sv[i]);
          }
        } else {
          apply_hi<P, true, false>(eu, ou, cf.eBy, cf.oBy, ew, ow, cf.eAy, cf.oAy, R, R);
          apply_hi<P, false, false>(ew, ow, cf.eBy, cf.oBy, ew, ow, cf.eBy, cf.oBy, Sv, Sv);
        }
        // row 0 of the next y-cell
#pragma unroll
        for (int i = 0; i <= P; ++i) {
          u[i] = sp[(P + i) * PXS];
          w[i] = sq[(P + i) * PXS];
        }
        if constexpr (GR) {
          const int ey = min((gy0 + jy * P) / P + 1, p.ncy - 1);
          const T sa = (T)p.cA[1][ey], sb = (T)p.cB[1][ey];
          R[P - 1] = vfma(sb, row0d<P>(u, cf.rBy, vzero<V>()), R[P - 1]);
          R[P - 1] = vfma(sa, row0d<P>(w, cf.rAy, vzero<V>()), R[P - 1]);
          Sv[P - 1] = vfma(sb, row0d<P>(w, cf.rBy, vzero<V>()), Sv[P - 1]);
        } else {
          R[P - 1] = row0d<P>(w, cf.rAy, row0d<P>(u, cf.rBy, R[P - 1]));
          Sv[P - 1] = row0d<P>(w, cf.rBy, Sv[P - 1]);
        }
      }
      // nodal term of this plane at the thread's nodes: alpha (v - shift_j) X_j
      V nod[P];
#pragma unroll
      for (int yi = 0; yi < P; ++yi) {
        const int oy = jy * P + yi;
        const V xv = stg[((oy + 1) * RX + ox + 1) * NCP + cv];
        nod[yi] = vfmav(vrsub(alpha * vv[yi], ash), xv, vzero<V>());
        // graded meshes: carried divided by D (restored at the output)
        if constexpr (GR) nod[yi] = vmul((T)(sxy[yi] * p.m1[2][gz] * p.dn[2][gz]), nod[yi]);
        if constexpr (kFold && HW) nod[yi] = vfma(beta, wr[yi], nod[yi]);
        if constexpr (kFold && HE) nod[yi] = vfmav(esc, er[yi], nod[yi]);
      }

      // ---- z: accumulate the planes of the current z-cell
      const int n = gz / P, kz = gz - n * P;
      // graded meshes: R, S of this plane scaled by the z-cell's scalars (the
      // vertex plane belongs to two cells)
      V Rz[P], Sz[P];
      auto zscale = [&](int cell) {
        if constexpr (GR) {
          const int ec = min(cell, p.ncz - 1);
          const T sb = (T)p.cB[2][ec], sa = (T)p.cA[2][ec];
#pragma unroll
          for (int yi = 0; yi < P; ++yi) {
            Rz[yi] = vmul(sb, R[yi]);
            Sz[yi] = vmul(sa, Sv[yi]);
          }
        }
      };
      const V *Ru = GR ? Rz : R, *Su = GR ? Sz : Sv;
      auto zall = [&](int k) {
#pragma unroll
        for (int i = 0; i <= P; ++i) {
          const CT b = cf.Bz[i * (P + 1) + k], a = cf.Az[i * (P + 1) + k];
#pragma unroll
          for (int yi = 0; yi < P; ++yi) acc[i][yi] = vfma(b, Ru[yi], vfma(a, Su[yi], acc[i][yi]));
        }
      };
      auto zrow0 = [&](int k) {
        const CT b = cf.Bz[k], a = cf.Az[k];
#pragma unroll
        for (int yi = 0; yi < P; ++yi) acc[0][yi] = vfma(b, Ru[yi], vfma(a, Su[yi], acc[0][yi]));
      };
      if (gz <= gz_end) {
        if (kz == 0 && gz > n0 * P) {
          // vertex plane: close cell n-1, write its planes, carry the vertex
          zscale(n - 1);
          zall(P);
#pragma unroll
          for (int i = 0; i < P; ++i) {
            const int g = (n - 1) * P + i;
            if (g > n0 * P) emit(g, acc[i]);
          }
#pragma unroll
          for (int yi = 0; yi < P; ++yi) {
            acc[0][yi] = vadd(acc[P][yi], nod[yi]);
#pragma unroll
            for (int i = 1; i <= P; ++i) acc[i][yi] = vzero<V>();
          }
          zscale(n);
          if (gz < gz_end) zall(0);
          else if (extra) zrow0(0);
        } else if (kz == 0) {
          zscale(n);
          zall(0);                      // bottom vertex of a segment: not owned here
        } else {
          zscale(n);
          zall(kz);
#pragma unroll
          for (int i = 1; i < P; ++i)
            if (i == kz) {
#pragma unroll
              for (int yi = 0; yi < P; ++yi) acc[i][yi] = vadd(acc[i][yi], nod[yi]);
            }
        }
      } else {
        // planes above the top vertex of the segment: row 0 of the next cell
        const int kk = gz - gz_end;
        zscale(n1);
        zrow0(kk);
        if (kk == P) emit(gz_end, acc[0]);
      }
      // x sweep of the next plane into the other buffer
      if (it + 1 < nplanes) {
        const int s1 = (gbase + it + 1) % NST;
        if (!wait_parity(&full[s1], (uint32_t)(((gbase + it + 1) / NST) & 1))) abort_flag = 1;
        V *Pw = Px + ((it + 1) & 1) * 2 * RY * PXS;
        xsweep(stage0 + s1 * S::STAGE_STRIDE_V, Pw, Pw + RY * PXS, gz + 1);
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
      // the stage of plane it is free: fetch the plane NST ahead into it
      if (tid == 0 && it + NST < nplanes) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        load_plane(&tmx, stage0 + s * S::STAGE_STRIDE_V, &full[s], kStageBytes, c0, gx0 - 1,
                   gy0 - 1, gz + NST - 1);
      }
    }
    if (abort_flag) break;
    gbase += nplanes;
  }  // segments
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (abort_flag && tid == 0) {
    // a plane never arrived: report, and give the loads still in flight a
    // bounded chance to land before the CTA's shared memory is released
    atomicExch(p.err, 3);
    for (int k = it; k < nplanes && k < it + NST; ++k)
      wait_parity(&full[(gbase + k) % NST], (uint32_t)(((gbase + k) / NST) & 1));
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled_fn() {
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

// d-scaled 1D cell blocks of one axis: Mh[i][j] = d_i M[i][j] d_j with the
// reference matrix scaled to the cell (A / s, B s, s = h/2) and d = m1^-1/2 at
// the cell's nodes (an interior vertex has m1 = 2 s w_0)
template <int P>
void scaled_blocks(const Geom &g, int axis, double *Ah, double *Bh) {
  constexpr int Q = P + 1;
  const double s = g.s[axis];
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j) {
      const double di = g.dl[axis][i], dj = g.dl[axis][j];
      Ah[i * Q + j] = di * (g.A[i * Q + j] / s) * dj;
      Bh[i * Q + j] = di * (g.B[i * Q + j] * s) * dj;
    }
}
// row 0 of a centrosymmetric matrix (symmetrised as in eo_blocks)
template <int P, typename T, int VW, typename CT>
void row0_block(const double *M, CT *r) {
  constexpr int Q = P + 1;
  for (int k = 0; k < Q; ++k) r[k] = CoefOf<T, VW>::make(0.5 * (M[k] + M[P * Q + (P - k)]));
}
// even / odd blocks of a centrosymmetric matrix (symmetrised first)
template <int P, typename T, int VW, typename CT>
void eo_blocks(const double *M, CT *e, CT *o) {
  constexpr int H = P / 2, Q = P + 1;
  auto sym = [&](int i, int j) { return 0.5 * (M[i * Q + j] + M[(P - i) * Q + (P - j)]); };
  for (int i = 0; i <= H; ++i)
    for (int k = 0; k <= H; ++k)
      e[i * (H + 1) + k] =
          CoefOf<T, VW>::make(k < H ? 0.5 * (sym(i, k) + sym(i, P - k)) : sym(i, H));
  for (int i = 0; i < H; ++i)
    for (int k = 0; k < H; ++k)
      o[i * H + k] = CoefOf<T, VW>::make(0.5 * (sym(i, k) - sym(i, P - k)));
}

template <typename T, int VW, int P, typename CT>
void make_coef(const Geom &g, double alpha, bool graded, SweepCoef<CT, P> *cf) {
  constexpr int Q = P + 1;
  double Ah[Q * Q], Bh[Q * Q];
  if (graded) {
    // the reference blocks; D and the cell scalars are applied in the kernel
    for (int i = 0; i < Q * Q; ++i) {
      Ah[i] = g.A[i];
      Bh[i] = g.B[i];
    }
    eo_blocks<P, T, VW>(Ah, cf->eAx, cf->oAx);
    eo_blocks<P, T, VW>(Bh, cf->eBx, cf->oBx);
    eo_blocks<P, T, VW>(Ah, cf->eAy, cf->oAy);
    eo_blocks<P, T, VW>(Bh, cf->eBy, cf->oBy);
    row0_block<P, T, VW>(Ah, cf->rAx);
    row0_block<P, T, VW>(Bh, cf->rBx);
    row0_block<P, T, VW>(Ah, cf->rAy);
    row0_block<P, T, VW>(Bh, cf->rBy);
    for (int i = 0; i < Q * Q; ++i) {
      cf->Az[i] = CoefOf<T, VW>::make(0.5 * alpha * Ah[i]);
      cf->Bz[i] = CoefOf<T, VW>::make(0.5 * alpha * Bh[i]);
    }
    return;
  }
  scaled_blocks<P>(g, 0, Ah, Bh);
  eo_blocks<P, T, VW>(Ah, cf->eAx, cf->oAx);
  eo_blocks<P, T, VW>(Bh, cf->eBx, cf->oBx);
  row0_block<P, T, VW>(Ah, cf->rAx);
  row0_block<P, T, VW>(Bh, cf->rBx);
  scaled_blocks<P>(g, 1, Ah, Bh);
  eo_blocks<P, T, VW>(Ah, cf->eAy, cf->oAy);
  eo_blocks<P, T, VW>(Bh, cf->eBy, cf->oBy);
  row0_block<P, T, VW>(Ah, cf->rAy);
  row0_block<P, T, VW>(Bh, cf->rBy);
  scaled_blocks<P>(g, 2, Ah, Bh);
  for (int i = 0; i < Q * Q; ++i) {
    cf->Az[i] = CoefOf<T, VW>::make(0.5 * alpha * Ah[i]);
    cf->Bz[i] = CoefOf<T, VW>::make(0.5 * alpha * Bh[i]);
  }
}

// CTAs of kernel k (nth threads, smem bytes) resident on the current device
// at once; cached per device (the shared-memory limit is raised before)
template <typename K>
int resident_grid(K *k, int nth, size_t smem) {
  static std::atomic<int> cache[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev < 16 && cache[dev].load() > 0) return cache[dev].load();
  int nsm = 0, occ = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, nth, smem) != cudaSuccess)
    return 0;
  const int g = nsm * std::max(occ, 1);
  if (dev < 16) cache[dev].store(g);
  return g;
}

template <typename T, int P, int C, int TX, int TY, int NST, int XPT, int MINB, int VW, bool HW,
          bool HE, bool GR, bool BAL = false>
cudaError_t run_sweep(const SweepArgs<T, typename CoefOf<T, VW>::type, P> &a, const CUtensorMap &tm,
                      int nitems, cudaStream_t s) {
  using Sh = SweepShape<T, P, C, TX, TY, XPT, VW>;
  auto k = hx_sweep_kernel<T, P, C, TX, TY, NST, XPT, MINB, VW, HW, HE, GR, BAL>;
  const size_t smem = Sh::smem(NST);
  cudaError_t e = raise_smem_limit(k, smem);
  if (e != cudaSuccess) return e;
  int grid = nitems;
  if (BAL) {
    // the persistent form: one CTA per resident slot
    grid = resident_grid(k, Sh::NTH, smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
  }
  ::invdft::count_launch();
  k<<<grid, Sh::NTH, smem, s>>>(a, tm);
  return cudaGetLastError();
}

// One tile variant: C columns per CTA, a TX x TY owned column of nodes, NST
// planes in flight, XPT x-cells per x task, MINB CTAs per SM for the
// register budget, VW columns per thread; GR: the graded-mesh form.
template <typename T, int P, int C, int TX, int TY, int NST, int XPT, int MINB, int VW, bool GR>
cudaError_t sweep_variant(const Geom &g, const T *v, const HxArgs<T> &a, int *err, int seglen,
                          cudaStream_t s) {
  using Sh = SweepShape<T, P, C, TX, TY, XPT, VW>;
  SweepArgs<T, typename CoefOf<T, VW>::type, P> sa;
  make_coef<T, VW>(g, a.alpha, GR, &sa.cf);
  for (int ax = 0; ax < 3; ++ax) {
    sa.dn[ax] = g.dnode[ax];
    sa.m1[ax] = g.m1node[ax];
    sa.cA[ax] = g.cellA[ax];
    sa.cB[ax] = g.cellB[ax];
  }
  sa.Z = a.Z;
  sa.W = a.W;
  sa.E = a.E;
  sa.escale = a.escale;
  sa.v = v;
  sa.shift_col = a.shift_col;
  sa.shift = a.shift;
  sa.alpha = a.alpha;
  sa.beta = a.beta;
  sa.err = err;
  sa.ncol = a.ncol;
  sa.nx = g.n[0];
  sa.ny = g.n[1];
  sa.nz = g.n[2];
  sa.ncx = g.nc[0];
  sa.ncy = g.nc[1];
  sa.ncz = g.nc[2];
  sa.ntx = (g.n[0] + TX - 1) / TX;
  sa.nty = (g.n[1] + TY - 1) / TY;
  sa.nchunk = (a.ncol + C - 1) / C;
  // the balanced schedule is built for the plain epilogue on uniform meshes
  // (the operator and the MINRES iterations); other launches with it fixed
  // run the whole z range per CTA
  const bool bal = seglen == kSegBalanced && !a.W && !a.E && !GR;
  if (seglen == kSegBalanced) seglen = g.nc[2];
  if (seglen < 0) {
    // the segment length that gives at least -seglen work items (CTAs)
    const long long per = (long long)sa.ntx * sa.nty * sa.nchunk;
    const long long nseg = std::min<long long>(g.nc[2], std::max<long long>(1, (-(long long)seglen + per - 1) / per));
    seglen = (int)((g.nc[2] + nseg - 1) / nseg);
  }
  sa.seglen = std::max(1, std::min(seglen, g.nc[2]));
  const int nseg = (g.nc[2] + sa.seglen - 1) / sa.seglen;
  const long long nitems = (long long)sa.ntx * sa.nty * sa.nchunk * nseg;
  if (nitems > 0x7fffffffLL) return cudaErrorInvalidValue;
  // X as a 4D tensor (column, x, y, z) of the unknown grid; box = one plane
  // of the tile with its halo
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap tm;
  const cuuint64_t dims[4] = {(cuuint64_t)a.ncol, (cuuint64_t)g.n[0], (cuuint64_t)g.n[1],
                              (cuuint64_t)g.n[2]};
  const cuuint64_t row = (cuuint64_t)a.ncol * sizeof(T);
  const cuuint64_t strides[3] = {row, row * g.n[0], row * g.n[0] * g.n[1]};
  const cuuint32_t box[4] = {(cuuint32_t)C, (cuuint32_t)Sh::RX, (cuuint32_t)Sh::RY, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  CUresult r = enc(&tm, sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                   4, (void *)a.X, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const bool hw = a.W != nullptr, he = a.E != nullptr;
  const int n = (int)nitems;
  if constexpr (!GR) {
    if (bal) return run_sweep<T, P, C, TX, TY, NST, XPT, MINB, VW, false, false, GR, true>(sa, tm, n, s);
  }
  if constexpr (std::is_same<T, float>::value) {
    if (hw && he) return run_sweep<T, P, C, TX, TY, NST, XPT, MINB, VW, true, true, GR>(sa, tm, n, s);
    if (he) return run_sweep<T, P, C, TX, TY, NST, XPT, MINB, VW, false, true, GR>(sa, tm, n, s);
  } else {
    if (he) return cudaErrorInvalidValue;
  }
  if (hw) return run_sweep<T, P, C, TX, TY, NST, XPT, MINB, VW, true, false, GR>(sa, tm, n, s);
  return run_sweep<T, P, C, TX, TY, NST, XPT, MINB, VW, false, false, GR>(sa, tm, n, s);
}

using SweepFn32 = cudaError_t (*)(const Geom &, const float *, const HxArgs<float> &, int *, int,
                                  cudaStream_t);
using SweepFn64 = cudaError_t (*)(const Geom &, const double *, const HxArgs<double> &, int *,
                                  int, cudaStream_t);
// Tile variants per (precision, order, mesh kind), the first one the default.
// Meshes of equal cells per axis (cubes or boxes of box cells) fold D and the
// cell size into the coefficients; graded meshes take the GR form.
const SweepFn32 kVar32q4[] = {
    sweep_variant<float, 4, 8, 16, 16, 4, 2, 2, 2, false>,   // 256 threads, two CTAs per SM
    sweep_variant<float, 4, 16, 16, 16, 3, 1, 1, 2, false>,  // 512 threads, one x-cell per task
    sweep_variant<float, 4, 16, 16, 16, 4, 2, 1, 2, false>,  // 512 threads, four planes in flight
    sweep_variant<float, 4, 8, 16, 32, 4, 2, 1, 2, false>,   // 512 threads, taller tile (less halo)
};
// (one column per thread in FP32 -- scalar FMAs instead of packed pairs -- was
// measured at 0.81 to 1.18 ms against 0.51 ms on the 32^3 x 64 case, and is not
// offered)
const SweepFn32 kVar32q2[] = {sweep_variant<float, 2, 16, 16, 8, 3, 2, 1, 2, false>};
const SweepFn32 kVar32q6[] = {sweep_variant<float, 6, 16, 12, 12, 3, 2, 1, 2, false>};
const SweepFn32 kVar32q4g[] = {sweep_variant<float, 4, 8, 16, 16, 4, 2, 2, 2, true>};
const SweepFn32 kVar32q2g[] = {sweep_variant<float, 2, 16, 16, 8, 3, 2, 1, 2, true>};
const SweepFn32 kVar32q6g[] = {sweep_variant<float, 6, 16, 12, 12, 3, 2, 1, 2, true>};
const SweepFn64 kVar64q4[] = {
    sweep_variant<double, 4, 8, 16, 16, 3, 2, 1, 1, false>,  // one column per thread, 512 threads
    sweep_variant<double, 4, 8, 16, 16, 3, 2, 1, 2, false>,  // column pairs, 256 threads
    sweep_variant<double, 4, 8, 16, 16, 3, 1, 1, 2, false>,
};
const SweepFn64 kVar64q2[] = {sweep_variant<double, 2, 8, 16, 8, 3, 2, 1, 2, false>};
const SweepFn64 kVar64q6[] = {sweep_variant<double, 6, 8, 12, 12, 3, 2, 1, 1, false>};
const SweepFn64 kVar64q4g[] = {sweep_variant<double, 4, 8, 16, 16, 3, 2, 1, 1, true>};
const SweepFn64 kVar64q2g[] = {sweep_variant<double, 2, 8, 16, 8, 3, 2, 1, 2, true>};
const SweepFn64 kVar64q6g[] = {sweep_variant<double, 6, 8, 12, 12, 3, 2, 1, 1, true>};
template <typename A, size_t N> constexpr int count_of(const A (&)[N]) { return (int)N; }

}  // namespace

bool sweep_supported(const Geom &g, int ncol, size_t elem, const void *X, const void *Z,
                     const void *W, const void *E) {
  if (!(g.p == 2 || g.p == 4 || g.p == 6)) return false;
  if (ncol < 2 || ncol > kMaxCols || (ncol * elem) % 16 != 0) return false;
  if (((uintptr_t)X & 15) != 0 || ((uintptr_t)Z & 15) != 0) return false;
  if (W && ((uintptr_t)W & 15) != 0) return false;
  if (E && ((uintptr_t)E & 7) != 0) return false;
  // the output is written while inputs of other tiles are still being read
  return Z != X && Z != W && Z != E;
}

namespace {
template <typename Fn, size_t A, size_t B, size_t C2, size_t D, size_t E2, size_t F>
std::pair<const Fn *, int> pick(const Geom &g, const Fn (&q2)[A], const Fn (&q4)[B],
                                const Fn (&q6)[C2], const Fn (&q2g)[D], const Fn (&q4g)[E2],
                                const Fn (&q6g)[F]) {
  if (g.graded) {
    if (g.p == 2) return {q2g, (int)D};
    if (g.p == 4) return {q4g, (int)E2};
    return {q6g, (int)F};
  }
  if (g.p == 2) return {q2, (int)A};
  if (g.p == 4) return {q4, (int)B};
  return {q6, (int)C2};
}
}  // namespace

int sweep_variants(const Geom &g, size_t elem) {
  if (elem == 4)
    return pick<SweepFn32>(g, kVar32q2, kVar32q4, kVar32q6, kVar32q2g, kVar32q4g, kVar32q6g).second;
  return pick<SweepFn64>(g, kVar64q2, kVar64q4, kVar64q6, kVar64q2g, kVar64q4g, kVar64q6g).second;
}

cudaError_t launch_hx_sweep(const Geom &g, const float *v, const HxArgs<float> &a, int *err,
                            int variant, int seglen, cudaStream_t s) {
  if (!sweep_supported(g, a.ncol, sizeof(float), a.X, a.Z, a.W, a.E)) return cudaErrorInvalidValue;
  auto t = pick<SweepFn32>(g, kVar32q2, kVar32q4, kVar32q6, kVar32q2g, kVar32q4g, kVar32q6g);
  if (variant < 0 || variant >= t.second) return cudaErrorInvalidValue;
  return t.first[variant](g, v, a, err, seglen, s);
}
cudaError_t launch_hx_sweep(const Geom &g, const double *v, const HxArgs<double> &a, int *err,
                            int variant, int seglen, cudaStream_t s) {
  if (!sweep_supported(g, a.ncol, sizeof(double), a.X, a.Z, a.W, nullptr) || a.E)
    return cudaErrorInvalidValue;
  auto t = pick<SweepFn64>(g, kVar64q2, kVar64q4, kVar64q6, kVar64q2g, kVar64q4g, kVar64q6g);
  if (variant < 0 || variant >= t.second) return cudaErrorInvalidValue;
  return t.first[variant](g, v, a, err, seglen, s);
}

}  // namespace invdft
