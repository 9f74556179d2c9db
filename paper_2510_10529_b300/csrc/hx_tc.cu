// H~X on the 5th-generation tensor cores (tcgen05, kind::tf32) for Q4 cells.
//
// For every cell e and a chunk of 64 columns the dense cell product
// Y_e = K_e (d_e o X_e) (Sec. 3.2.3: "cell-level dense-dense matrix products")
// is one M=128 (local nodes, 125 used) x N=64 (columns) x K=128 MMA sequence:
//   A = kc K_e, rounded to TF32, resident in shared memory for the CTA's life;
//   B = d o X_e, gathered from the node-major block, rounded to TF32 and
//       written transposed into the K-major (no-swizzle) UMMA layout;
//   D = FP32 accumulator in tensor memory (64 TMEM columns).
// The epilogue reads D row by row (one thread per local node), scales by
// alpha d_a, adds the nodal term alpha (v_a - shift) X_a + beta W_a +
// alpha s E_a for the nodes this cell owns (local index < 4 on every axis, so
// each interior node has exactly one owner) and scatter-adds into Z, which
// the launcher zeroes first.  Persistent CTAs walk the cells in x-fastest
// order so that concurrent CTAs touch neighbouring nodes and the atomics
// resolve in L2.
//
// Operands are TF32 (10-bit mantissa); the relative error of H~X is about
// 1e-3 of |K||X|, which the mixed solvers absorb (defect-corrected filter,
// FP64 refinement of the adjoint).
#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128, kTcK = 128, kTcN = 64;
constexpr int kTcNe = 125;
constexpr uint32_t kSmemA = kTcM * kTcK * 4;     // 64 KiB
constexpr uint32_t kSmemB = kTcN * kTcK * 4;     // 32 KiB
constexpr long long kSpinLimit = 1LL << 28;       // bounded mbarrier wait

// byte offset of element (row r, k) in the K-major no-swizzle layout:
// 8 x 16-byte core matrices, K-adjacent ones 128 B apart (LBO), 8-row groups
// (K/4) * 128 = 4096 B apart (SBO)
__host__ __device__ constexpr uint32_t kmajor_off(int r, int k) {
  return (uint32_t)((r >> 3) * 4096 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);          // start address
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;      // leading byte offset (K direction)
  d |= (uint64_t)((4096u >> 4) & 0x3FFF) << 32;     // stride byte offset (M/N direction)
  d |= (uint64_t)1 << 46;                           // descriptor version (sm_100 family)
  // base offset 0, LBO mode 0, layout type 0 = no swizzle
  return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) |
                            ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

struct TcArgs {
  const float *X;
  float *Z;
  const float *W;
  const float *E;
  const double *v;
  const double *shift_col;
  const double *escale;
  const float *Ke;          // 128 x 128 tf32 in the UMMA layout (kc included)
  const double *dm1;
  const int *perm;          // visiting order of the cells
  int *err;                 // device status word (set on a timed-out wait)
  double alpha, shift, beta;
  int ncol, ncell, Ni;
};

template <int C, bool HW, bool HE>
__global__ void __launch_bounds__(kTcThreads, 2) hx_tc_kernel(TcArgs p) {
  constexpr int G = kTcN / C;               // cells per tile (columns n = g*C + col)
  constexpr int C4 = C / 4;
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA = smem;
  unsigned char *sB = smem + kSmemA;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ float dlf[G][3][5];
  __shared__ float sshift[C], sesc[C];
  __shared__ int gi[G][3][5];
  __shared__ int abort_flag;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nc = p.ncell, Ni = p.Ni;
  const long long ncells = (long long)nc * nc * nc;
  const int nchunk = (p.ncol + C - 1) / C;
  const long long ngroups = (ncells + G - 1) / G;
  const long long items = ngroups * nchunk;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kTcN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // A: resident cell matrix; B: zero once (rows k >= 125 are never written)
  {
    const float4 *src = reinterpret_cast<const float4 *>(p.Ke);
    float4 *dst = reinterpret_cast<float4 *>(sA);
    for (int i = tid; i < (int)(kSmemA / 16); i += kTcThreads) dst[i] = src[i];
    float4 *b = reinterpret_cast<float4 *>(sB);
    for (int i = tid; i < (int)(kSmemB / 16); i += kTcThreads) b[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
  const float salpha = (float)p.alpha, sbeta = (float)p.beta;
  uint32_t phase = 0;

  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int chunk = (int)(item % nchunk);
    const long long grp = item / nchunk;
    const int c0 = chunk * C;
    if (tid < G * 15) {
      const int g = tid / 15, d = (tid % 15) / 5, l = tid % 5;
      const long long slot = grp * G + g;
      const long long cell = slot < ncells ? p.perm[slot] : ncells;
      int gidx = -1;
      double dv = 0.0;
      if (cell < ncells) {
        const int cx = (int)(cell % nc), cy = (int)((cell / nc) % nc),
                  cz = (int)(cell / ((long long)nc * nc));
        const int cc = d == 0 ? cx : (d == 1 ? cy : cz);
        const int gg = cc * 4 + l;
        dv = p.dm1[gg];
        gidx = (gg >= 1 && gg <= Ni) ? gg - 1 : -1;
      }
      dlf[g][d][l] = (float)dv;
      gi[g][d][l] = gidx;
    }
    if (tid >= 128 && tid < 128 + C) {
      const int j = tid - 128, col = c0 + j;
      const bool ok = col < p.ncol;
      sshift[j] = ok ? (float)(p.shift_col ? p.shift_col[col] : p.shift) : 0.f;
      sesc[j] = (ok && p.E) ? (float)(p.alpha * p.escale[col]) : 0.f;
    }
    __syncthreads();
    // ---- gather B = d o X_e (TF32), float4 loads; element (n = g*C + col, k)
    {
      constexpr int per_g = kTcNe * C4;
      constexpr int total = G * per_g;
      constexpr int iters = (total + kTcThreads - 1) / kTcThreads;
      float4 vals[iters];
      int offs[iters];
#pragma unroll
      for (int it = 0; it < iters; ++it) {
        const int idx = tid + it * kTcThreads;
        vals[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        offs[it] = -1;
        if (idx < total) {
          const int g = idx / per_g, r = idx % per_g;
          // lanes: 4 float4 along columns x 8 nodes; then column quads
          const int c4lo = r & 3, rest = r >> 2;
          const int k = rest % kTcNe, c4hi = rest / kTcNe;
          const int c4 = c4hi * 4 + c4lo;
          if (c4 < C4) {
            const int lx = k % 5, ly = (k / 5) % 5, lz = k / 25;
            const int ix = gi[g][0][lx], iy = gi[g][1][ly], iz = gi[g][2][lz];
            offs[it] = (g * C + c4 * 4) * 1024 + k;     // packed (n0, k)
            const int col = c0 + c4 * 4;
            if (ix >= 0 && iy >= 0 && iz >= 0 && col < p.ncol) {
              const long long node = ix + (long long)Ni * (iy + (long long)Ni * iz);
              const float sc = dlf[g][0][lx] * dlf[g][1][ly] * dlf[g][2][lz];
              const float *src = p.X + node * p.ncol + col;
              float4 x;
              if ((p.ncol & 3) == 0 && col + 3 < p.ncol) {
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
      }
#pragma unroll
      for (int it = 0; it < iters; ++it) {
        if (offs[it] < 0) continue;
        const int n0 = offs[it] >> 10, k = offs[it] & 1023;
        *reinterpret_cast<float *>(sB + kmajor_off(n0 + 0, k)) = to_tf32(vals[it].x);
        *reinterpret_cast<float *>(sB + kmajor_off(n0 + 1, k)) = to_tf32(vals[it].y);
        *reinterpret_cast<float *>(sB + kmajor_off(n0 + 2, k)) = to_tf32(vals[it].z);
        *reinterpret_cast<float *>(sB + kmajor_off(n0 + 3, k)) = to_tf32(vals[it].w);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // ---- one thread issues the 16 K-steps (K = 8 each)
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int j = 0; j < kTcK / 8; ++j) {
        const uint64_t ad = make_desc(a_base + j * 256);
        const uint64_t bd = make_desc(b_base + j * 256);
        const uint32_t acc = j > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n}\n"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_u32(&mbar)) : "memory");
    }
    // ---- wait for the accumulator (bounded)
    {
      uint32_t done = 0;
      long long spins = 0;
      while (!done) {
        asm volatile(
            "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
            " selp.u32 %0, 1, 0, pw;\n}\n"
            : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase) : "memory");
        if (!done && ++spins > kSpinLimit) {
          abort_flag = 1;
          break;
        }
      }
      phase ^= 1u;
    }
    __syncthreads();
    if (abort_flag) {
      if (tid == 0) atomicExch(p.err, 1);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // ---- epilogue: row a = TMEM lane (warp % 4) * 32 + lane, columns
    // [32 * (warp / 4), +32)
    {
      const int a = (warp & 3) * 32 + lane;
      const int nb = (warp >> 2) * 32;
      float acc[32];
      {
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + nb;
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = __uint_as_float(r[j]);
      }
      if (a < kTcNe) {
        const int lx = a % 5, ly = (a / 5) % 5, lz = a / 25;
        const bool owner = lx < 4 && ly < 4 && lz < 4;
        const bool vec = (p.ncol & 3) == 0;
#pragma unroll
        for (int hq = 0; hq < 8; hq += 4) {
        // phase 1: addresses and (for owned nodes) the nodal-term loads of 4 quads
        long long e0q[8];
        float4 xq[8], wq[8], eq[8];
        float vq[8];
#pragma unroll
        for (int qi = hq; qi < hq + 4; ++qi) {
          const int n = nb + qi * 4;
          const int g = n / C, col = c0 + (n % C);
          const int ix = gi[g][0][lx], iy = gi[g][1][ly], iz = gi[g][2][lz];
          e0q[qi] = -1;
          xq[qi] = wq[qi] = eq[qi] = make_float4(0.f, 0.f, 0.f, 0.f);
          vq[qi] = 0.f;
          if (ix < 0 || iy < 0 || iz < 0 || col >= p.ncol) continue;
          const long long node = ix + (long long)Ni * (iy + (long long)Ni * iz);
          e0q[qi] = node * p.ncol + col;
          if (owner) {
            vq[qi] = (float)p.v[node];
            if (vec) {
              xq[qi] = __ldg(reinterpret_cast<const float4 *>(p.X + e0q[qi]));
              if (HW) wq[qi] = *reinterpret_cast<const float4 *>(p.W + e0q[qi]);
              if (HE) eq[qi] = __ldg(reinterpret_cast<const float4 *>(p.E + e0q[qi]));
            } else {
              const int m = min(4, p.ncol - col);
              float tx[4] = {0.f, 0.f, 0.f, 0.f}, tw[4] = {0.f, 0.f, 0.f, 0.f},
                    te[4] = {0.f, 0.f, 0.f, 0.f};
              for (int t = 0; t < m; ++t) {
                tx[t] = p.X[e0q[qi] + t];
                if (HW) tw[t] = p.W[e0q[qi] + t];
                if (HE) te[t] = p.E[e0q[qi] + t];
              }
              xq[qi] = make_float4(tx[0], tx[1], tx[2], tx[3]);
              wq[qi] = make_float4(tw[0], tw[1], tw[2], tw[3]);
              eq[qi] = make_float4(te[0], te[1], te[2], te[3]);
            }
          }
        }
        // phase 2: combine and reduce into Z (fire-and-forget vector reductions)
#pragma unroll
        for (int qi = hq; qi < hq + 4; ++qi) {
          if (e0q[qi] < 0) continue;
          const int n = nb + qi * 4;
          const int g = n / C, cl = n % C;
          const float sc = salpha * dlf[g][0][lx] * dlf[g][1][ly] * dlf[g][2][lz];
          float o[4] = {sc * acc[qi * 4], sc * acc[qi * 4 + 1], sc * acc[qi * 4 + 2],
                        sc * acc[qi * 4 + 3]};
          if (owner) {
            const float xs[4] = {xq[qi].x, xq[qi].y, xq[qi].z, xq[qi].w};
            const float ws[4] = {wq[qi].x, wq[qi].y, wq[qi].z, wq[qi].w};
            const float es[4] = {eq[qi].x, eq[qi].y, eq[qi].z, eq[qi].w};
#pragma unroll
            for (int t = 0; t < 4; ++t)
            {
              float tt = salpha * (vq[qi] - sshift[cl + t]) * xs[t];
              if (HW) tt = fmaf(sbeta, ws[t], tt);
              if (HE) tt = fmaf(sesc[cl + t], es[t], tt);
              o[t] += tt;
            }
          }
          float *dst = p.Z + e0q[qi];
          if (vec) {
            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                         :: "l"(dst), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]) : "memory");
          } else {
            const int m = min(4, p.ncol - (c0 + cl));
            for (int t = 0; t < m; ++t)
              asm volatile("red.global.add.f32 [%0], %1;" :: "l"(dst + t), "f"(o[t]) : "memory");
          }
        }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (abort_flag) {
    // give an MMA still in flight a second bounded chance to land before the
    // accumulator is released
    uint32_t done = 0;
    for (long long spins = 0; !done && spins < kSpinLimit; ++spins)
      asm volatile(
          "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
          " selp.u32 %0, 1, 0, pw;\n}\n"
          : "=r"(done) : "r"(smem_u32(&mbar)), "r"(phase ^ 1u) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcN)
                 : "memory");
}

float round_tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;     // inf / nan
  u += 0x1000u;                                       // round to nearest on bit 13
  u &= 0xffffe000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

}  // namespace

// The 128 x 128 TF32 image of kc K_e in the UMMA layout (host side).
void build_tc_cell_matrix(const Geom &g, std::vector<float> *out) {
  out->assign(kTcM * kTcK, 0.f);
  const int q = 5;
  for (int a = 0; a < kTcNe; ++a) {
    const int ax = a % q, ay = (a / q) % q, az = a / (q * q);
    for (int b = 0; b < kTcNe; ++b) {
      const int bx = b % q, by = (b / q) % q, bz = b / (q * q);
      const double kab = g.kc * (g.B[az * q + bz] * g.B[ay * q + by] * g.A[ax * q + bx] +
                                 g.B[az * q + bz] * g.A[ay * q + by] * g.B[ax * q + bx] +
                                 g.A[az * q + bz] * g.B[ay * q + by] * g.B[ax * q + bx]);
      (*out)[kmajor_off(a, b) / 4] = round_tf32_host((float)kab);
    }
  }
}

size_t tc_cell_matrix_floats() { return (size_t)kTcM * kTcK; }

// Cell visiting order: z-slabs two cells thick; inside a slab the 8 parity
// classes (cx, cy, cz mod 2) one after the other.  Cells in flight at the same
// time then share no nodes (their reductions do not contend for the same L2
// lines) while the slab keeps the touched nodes inside L2.
void build_cell_order(int nc, std::vector<int> *perm) {
  perm->clear();
  for (int zs = 0; zs < nc; zs += 2)
    for (int color = 0; color < 8; ++color)
      for (int cz = zs; cz < std::min(nc, zs + 2); ++cz)
        for (int cy = 0; cy < nc; ++cy)
          for (int cx = 0; cx < nc; ++cx)
            if ((cx & 1) == (color & 1) && (cy & 1) == ((color >> 1) & 1) &&
                (cz & 1) == ((color >> 2) & 1))
              perm->push_back(cx + nc * (cy + nc * cz));
}

cudaError_t launch_hx_tc(const Geom &g, const double *v, const HxArgs<float> &a, const float *Ke,
                         const int *perm, int *err, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.Z, 0, (size_t)g.L * a.ncol * sizeof(float), s);
  if (e != cudaSuccess) return e;
  const size_t smem = kSmemA + kSmemB;
  const int C = a.ncol <= 16 ? 16 : (a.ncol <= 32 ? 32 : 64);
  const int mode = (a.W ? 1 : 0) + (a.E ? 2 : 0);
  using K = void (*)(TcArgs);
  static const K table[3][4] = {
      {hx_tc_kernel<16, false, false>, hx_tc_kernel<16, true, false>,
       hx_tc_kernel<16, false, true>, hx_tc_kernel<16, true, true>},
      {hx_tc_kernel<32, false, false>, hx_tc_kernel<32, true, false>,
       hx_tc_kernel<32, false, true>, hx_tc_kernel<32, true, true>},
      {hx_tc_kernel<64, false, false>, hx_tc_kernel<64, true, false>,
       hx_tc_kernel<64, false, true>, hx_tc_kernel<64, true, true>}};
  const K kern = table[C == 16 ? 0 : (C == 32 ? 1 : 2)][mode];
  e = raise_smem_limit(kern, (int)smem);
  if (e != cudaSuccess) return e;
  TcArgs p;
  p.X = a.X;
  p.Z = a.Z;
  p.W = a.W;
  p.E = a.E;
  p.v = v;
  p.shift_col = a.shift_col;
  p.escale = a.escale;
  p.Ke = Ke;
  p.dm1 = g.dm1;
  p.perm = perm;
  p.err = err;
  p.alpha = a.alpha;
  p.shift = a.shift;
  p.beta = a.beta;
  p.ncol = a.ncol;
  p.ncell = g.ncell;
  p.Ni = g.Ni;
  const long long cells = (long long)g.ncell * g.ncell * g.ncell;
  const long long items = ((cells + kTcN / C - 1) / (kTcN / C)) * ((a.ncol + C - 1) / C);
  const int grid = (int)std::min<long long>(items, 148LL * 2);
  ::invdft::count_launch();
  kern<<<grid, kTcThreads, smem, s>>>(p);
  return cudaGetLastError();
}


namespace {

// Tensor-pipe rate probe: chains of the H~X kernel's MMA shape (M = 128,
// N = 64, K = 128 as 16 steps of K = 8, kind::tf32) issued back to back by one
// thread per CTA on operands resident in shared memory; no memory traffic.
__global__ void __launch_bounds__(128, 1) tf32_probe_kernel(int chains, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char *sA = smem;
  unsigned char *sB = smem + kSmemA;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_slot)), "r"(kTcN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = tid; i < (int)((kSmemA + kSmemB) / 16); i += 128)
    reinterpret_cast<float4 *>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t a_base = smem_u32(sA), b_base = smem_u32(sB);
    for (int c = 0; c < chains; ++c) {
#pragma unroll
      for (int j = 0; j < kTcK / 8; ++j) {
        const uint64_t ad = make_desc(a_base + j * 256);
        const uint64_t bd = make_desc(b_base + j * 256);
        const uint32_t acc = (c | j) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n}\n"
            :: "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc) : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(&mbar)) : "memory");
    uint32_t done = 0;
    long long spins = 0;
    while (!done) {
      asm volatile(
          "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
          " selp.u32 %0, 1, 0, pw;\n}\n"
          : "=r"(done) : "r"(smem_u32(&mbar)), "r"(0u) : "memory");
      if (!done && ++spins > kSpinLimit) {
        atomicExch(err, 1);
        break;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcN)
                 : "memory");
}

}  // namespace

// flops of one probe launch: grid CTAs x chains x 2 M N K
cudaError_t launch_tf32_probe(int grid, int chains, int *err, double *flops, cudaStream_t s) {
  const size_t smem = kSmemA + kSmemB;
  cudaError_t e = raise_smem_limit(tf32_probe_kernel, smem);
  if (e != cudaSuccess) return e;
  ::invdft::count_launch();
  tf32_probe_kernel<<<grid, 128, smem, s>>>(chains, err);
  *flops = (double)grid * chains * 2.0 * kTcM * kTcN * kTcK;
  return cudaGetLastError();
}

}  // namespace invdft
