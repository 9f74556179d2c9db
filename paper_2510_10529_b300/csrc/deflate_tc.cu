// Deflation Gram of the FP32 MINRES blocks on the tensor cores (Sec. 3.2.2):
//   C = Psi^T Z,   Psi [L][n1p] (deflation vectors), Z [L][n2p] (MINRES block)
// as tcgen05 kind::tf32 MMAs, one 32-node tile = one K extent of 32, with
// TF32 splitting of both operands: x = hi + lo, hi the TF32 rounding of x and
// lo = x - hi (exact in FP32; the MMA takes its TF32 part).  The A operand
// stacks the hi rows (0..63) over the lo rows (64..127) of Psi^T, and two
// MMAs per K-step (B = Z_hi, then Z_lo) accumulate all four split products
// in TMEM: C = D[0:64] + D[64:128], summed in FP64 across CTAs.
//
// Persistent CTAs (two per SM, so that the barrier-separated phases of one
// overlap those of the other) walk 32-node tiles.  Psi and Z rows are staged
// node-major by 16-byte cp.async, one tile ahead, and transposed into the
// K-major no-swizzle operand layout by the threads that split them; the
// operand buffers are double-buffered so that the MMAs of a tile overlap the
// split of the next.  Waits on the MMA barriers are bounded: a wait that
// gives up sets the error word and the CTA leaves after a second bounded wait
// for its MMAs.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kTM = 128, kTN = 64;
constexpr long long kTSpin = 1LL << 28;

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (row r, k) in a K-major no-swizzle operand with K columns:
// core matrices of 8 rows x 16 bytes; K-adjacent ones 128 B apart, 8-row
// groups (K / 4) * 128 B apart
__host__ __device__ __forceinline__ uint32_t kmoff(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K / 4) * 128 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;       // K-adjacent core matrices
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;        // 8-row groups
  d |= (uint64_t)1 << 46;                             // descriptor version (sm_100 family)
  return d;
}

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 64
constexpr uint32_t kTIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                             ((uint32_t)(kTM >> 4) << 24);

// TF32 rounding (10 explicit mantissa bits), nearest with ties away from
// zero, on the bit pattern: add half the range of the 13 dropped bits, then
// clear them (finite x; a carry moves into the exponent as it should)
__device__ __forceinline__ float rna_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  long long spins = 0;
  while (!done) {
    asm volatile(
        "{\n .reg .pred pw;\n mbarrier.try_wait.parity.shared::cta.b64 pw, [%1], %2;\n"
        " selp.u32 %0, 1, 0, pw;\n}\n"
        : "=r"(done) : "r"(saddr(bar)), "r"(parity) : "memory");
    if (!done && ++spins > kTSpin) return false;
  }
  return true;
}

__device__ __forceinline__ void cp16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(saddr(dst)), "l"(src) : "memory");
}

// ---------------------------------------------------------------------------
// Gram C = Psi^T Z (partials per CTA), tensor cores
constexpr int kGK = 32;     // nodes per tile = MMA K extent of a tile
constexpr int kGThreads = 256;
constexpr int kGWarps = kGThreads / 32;
constexpr int kGPerSm = 2;  // resident CTAs per SM: one CTA's barrier phases overlap the other's

struct TcGram {
  const float *Psi;
  const float *Z;
  double *partial;     // [grid][n1p * n2p]
  int *err;
  int n1p, n2p;
  long long L;
};

constexpr int kGLd = 64;    // staging row stride (floats) of both Psi and Z
constexpr int kGStages = 2; // staging ring: loads run one tile ahead

__global__ void __launch_bounds__(kGThreads, kGPerSm) defl_gram_tc_kernel(const TcGram p) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  constexpr uint32_t szA = kTM * kGK * 4, szB = kTN * kGK * 4, szOp = szA + 2 * szB;
  float *raw = reinterpret_cast<float *>(gsm + 2 * szOp);
  constexpr int rawsz = 2 * kGK * kGLd;      // one stage: Psi rows, then Z rows
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(saddr(&tmem_slot)), "r"(kTN) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // operand padding (rows past n1p / n2p) stays zero
  for (int e = tid; e < (int)(2 * szOp / 16); e += kGThreads)
    reinterpret_cast<float4 *>(gsm)[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const long long ntile = (p.L + kGK - 1) / kGK;
  // node-major staging of the Psi and Z rows of a tile (zeros past L): each
  // warp copies 4 nodes, lanes 0..15 the Psi row, lanes 16..31 the Z row
  const bool cpsi = lane < 16;
  const int kq = cpsi ? lane : lane - 16;
  const bool cact = kq < (cpsi ? p.n1p : p.n2p) / 4;
  const int crow = warp * (kGK / kGWarps);
  const int cld = cpsi ? p.n1p : p.n2p;                 // global row stride
  const float *cbase = (cpsi ? p.Psi : p.Z) + 4 * kq + (long long)crow * cld;
  float *sbase = raw + (cpsi ? 0 : kGK * kGLd) + crow * kGLd + 4 * kq;
  auto load = [&](long long tile, int st) {
    const long long r0 = tile * kGK;
    const int rows = (int)min((long long)kGK, p.L - r0) - crow;
    if (cact) {
      const float *src = cbase + r0 * cld;
      float *dst = sbase + st * rawsz;
#pragma unroll
      for (int i = 0; i < kGK / kGWarps; ++i) {
        if (i < rows) cp16(dst + i * kGLd, src + i * cld);
        else *reinterpret_cast<float4 *>(dst + i * kGLd) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // transpose + split.  Work unit = 32 columns (lane = column) x 16 nodes: per
  // 4 nodes, four scalar staging reads (consecutive columns: conflict-free)
  // give the four K-adjacent values of one operand row, stored as one float4
  // each for hi and lo (a quarter-warp covers one 128-byte core-matrix row
  // block: no conflicts).  lo = x - hi is exact in FP32; the MMA takes its
  // TF32 part.
  const int cg1 = (p.n1p + 31) / 32, ncg = cg1 + (p.n2p + 31) / 32;
  auto split = [&](int st, int ob) {
    const float *stage = raw + st * rawsz;
    unsigned char *A = gsm + ob * szOp;
    for (int u = warp; u < ncg * (kGK / 16); u += kGWarps) {
      const int cgi = u / (kGK / 16), nb = (u % (kGK / 16)) * 16;
      const bool psi = cgi < cg1;
      const int col = (psi ? cgi : cgi - cg1) * 32 + lane;
      if (col >= (psi ? p.n1p : p.n2p)) continue;
      const float *src = stage + (psi ? 0 : kGK * kGLd) + nb * kGLd + col;
      unsigned char *dh = A + (psi ? 0 : szA) + kmoff(col, nb, kGK);
      const uint32_t lo_off = psi ? szA / 2 : szB;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float x0 = src[(4 * q + 0) * kGLd], x1 = src[(4 * q + 1) * kGLd];
        const float x2 = src[(4 * q + 2) * kGLd], x3 = src[(4 * q + 3) * kGLd];
        const float4 h = make_float4(rna_tf32(x0), rna_tf32(x1), rna_tf32(x2), rna_tf32(x3));
        *reinterpret_cast<float4 *>(dh + q * 128) = h;
        *reinterpret_cast<float4 *>(dh + q * 128 + lo_off) =
            make_float4(x0 - h.x, x1 - h.y, x2 - h.z, x3 - h.w);
      }
    }
  };
  uint32_t phase[2] = {0u, 0u};
  int last_s = -1;
  uint32_t last_par = 0;
  bool first = true;
  // operand descriptors of the two buffers at K-step 0 (8-row groups 2 KB apart)
  const uint64_t desc_a0 = umma_desc(saddr(gsm), (kGK / 4) * 128u);
  const uint64_t desc_a1 = umma_desc(saddr(gsm + szOp), (kGK / 4) * 128u);
  long long tile = blockIdx.x;
  // prologue: the first two tiles of this CTA (an empty group past the end)
  for (int i = 0; i < kGStages - 1; ++i) {
    const long long t = tile + (long long)i * gridDim.x;
    if (t < ntile) load(t, i);
    else asm volatile("cp.async.commit_group;" ::: "memory");
  }
  int st = 0;
  for (int it = 0; tile < ntile; tile += gridDim.x, ++it) {
    const int s = it & 1;
    // operand buffer s was read by the MMAs of iteration it - 2
    if (it >= 2) {
      if (!wait_bar(&mbar[s], phase[s])) abort_flag = 1;
      phase[s] ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    // the stage of iteration it - 1 was released by the barrier after its split
    const long long nxt = tile + (long long)(kGStages - 1) * gridDim.x;
    const int st_nxt = st == 0 ? kGStages - 1 : st - 1;
    if (nxt < ntile) load(nxt, st_nxt);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group %0;" :: "n"(kGStages - 1) : "memory");
    __syncthreads();
    if (abort_flag) break;
    split(st, s);
    st = st == kGStages - 1 ? 0 : st + 1;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // a K-step of 8 advances each operand by two core matrices (256 B),
      // i.e. 16 in the descriptor's address field
      const uint64_t da0 = s ? desc_a1 : desc_a0, dbh0 = da0 + (szA >> 4), dbl0 = dbh0 + (szB >> 4);
#pragma unroll
      for (int j = 0; j < kGK / 8; ++j) {
        const uint64_t da = da0 + 16 * j, dbh = dbh0 + 16 * j, dbl = dbl0 + 16 * j;
        const uint32_t acc0 = (first && j == 0) ? 0u : 1u;
        asm volatile(
            "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n}\n"
            :: "r"(tmem), "l"(da), "l"(dbh), "r"(kTIdesc), "r"(acc0) : "memory");
        asm volatile(
            "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n}\n"
            :: "r"(tmem), "l"(da), "l"(dbl), "r"(kTIdesc), "r"(1u) : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(saddr(&mbar[s])) : "memory");
    }
    first = false;
    last_s = s;
    last_par = phase[s];
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // the last commit tracks every MMA issued before it
  if (last_s >= 0 && !wait_bar(&mbar[last_s], last_par)) abort_flag = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag) {
    if (tid == 0) atomicExch(p.err, 4);
  } else {
    // D rows 0..63: Psi_hi^T Z, rows 64..127: Psi_lo^T Z; warps 0..7 read
    // 32 columns each (warps 8..15 only join the barriers)
    const int g = warp & 3, cb = ((warp >> 2) & 1) * 32;
    const bool rd = warp < 8;
    uint32_t r[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) r[j] = 0u;
    if (rd) {
      const uint32_t taddr = tmem + ((uint32_t)(g * 32) << 16) + cb;
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
    }
    double *red = reinterpret_cast<double *>(gsm);     // [64][65], in the operand buffers
    const int m = (g & 1) * 32 + lane;
    if (rd && g < 2) {
#pragma unroll
      for (int j = 0; j < 32; ++j) red[m * 65 + cb + j] = (double)__uint_as_float(r[j]);
    }
    __syncthreads();
    if (rd && g >= 2) {
#pragma unroll
      for (int j = 0; j < 32; ++j) red[m * 65 + cb + j] += (double)__uint_as_float(r[j]);
    }
    __syncthreads();
    const int nn = p.n1p * p.n2p;
    double *out = p.partial + (size_t)blockIdx.x * nn;
    for (int e = tid; e < nn; e += kGThreads) {
      const int i = e / p.n2p, j = e - i * p.n2p;
      out[e] = red[i * 65 + j];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTN)
                 : "memory");
}


// ---------------------------------------------------------------------------
// Update Z <- Z + Psi (alpha C) on the tensor cores, with the optional column
// dot of the updated block against V.
//
// One 128-node tile = one MMA of M = 128 rows, N = Np (n2p rounded up to 16),
// K = n1p, as three kind::tf32 products per K-step of 8:
//   Psi_hi B_hi + Psi_lo B_hi + Psi_hi B_lo,   B = (alpha C)^T split in TF32,
// which drops only the lo x lo term (relative 2^-22, the FP32 level).
// The Psi tile arrives by one TMA tensor copy already in the K-major
// no-swizzle operand layout: the tensor map views Psi [L][n1p] as (4 floats,
// node, group of 4 columns), so the box lands as [k / 4][row][k % 4], i.e.
// core matrices of 8 rows x 16 bytes with 8-row groups 128 B apart and
// K-adjacent core matrices 128 * 16 B apart.  The Z tile (a contiguous span
// of rows) arrives by a plain bulk copy, row-major.  The CTA splits Psi in
// place (hi) and into a second buffer (lo), one thread issues the MMAs, the
// eight warps read the accumulator back (warp w: TMEM lanes 32 (w % 4) ..,
// columns 32 (w / 4) ..), add it to the Z tile in shared memory, and one
// bulk copy writes the tile back.  Two stages: the copies of the next tile
// are in flight while this one is processed.  Every wait is bounded; a wait
// that gives up sets the error word, and the CTA drains its copies before it
// leaves.
constexpr int kUM = 128;           // rows per tile (MMA M)
constexpr int kUThreads = 256;
constexpr int kUStages = 2;

struct TcUpdate {
  const double *C;     // [n1p][n2p]
  float *Z;            // [L][n2p]
  const float *V;      // [L][n2p] or null
  double *partial;     // [grid][n2p]
  int *err;
  double alpha;
  int n1p, n2p, Np;
  long long L;
};

__device__ __forceinline__ uint64_t umma_desc_ls(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;        // K-adjacent core matrices
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;        // 8-row groups
  d |= (uint64_t)1 << 46;                             // descriptor version (sm_100 family)
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred pa;\n setp.ne.b32 pa, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, pa;\n}\n"
      :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc) : "memory");
}

__global__ void __launch_bounds__(kUThreads, 1)
defl_update_tc_kernel(const TcUpdate p, const __grid_constant__ CUtensorMap tmpsi) {
  extern __shared__ __align__(1024) unsigned char usm_raw[];
  unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)usm_raw + 1023) & ~(uintptr_t)1023);
  const int n1p = p.n1p, n2p = p.n2p, Np = p.Np;
  const uint32_t szA = (uint32_t)kUM * n1p * 4, szB = (uint32_t)Np * n1p * 4;
  const uint32_t szZ = (uint32_t)kUM * n2p * 4;
  unsigned char *Bhi = base, *Blo = base + szB, *Alo = base + 2 * szB;
  float *Vs = reinterpret_cast<float *>(Alo + szA);     // V rows of the current tile
  unsigned char *Ahi0 = Alo + szA + szZ;               // stage s: Ahi0 + s * (szA + szZ)
  __shared__ __align__(8) uint64_t full[kUStages], mmab, vbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  __shared__ float red[4][64];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto ahi = [&](int s) { return Ahi0 + s * (szA + szZ); };
  auto zs = [&](int s) { return reinterpret_cast<float *>(Ahi0 + s * (szA + szZ) + szA); };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(saddr(&tmem_slot)), "r"(64) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // B = (alpha C)^T, split, K-major: (n, k) at (k / 4) * Np * 16 + n * 16 + (k % 4) * 4;
  // rows n >= n2p stay zero
  for (int e = tid; e < Np * n1p; e += kUThreads) {
    const int k = e / Np, n = e - k * Np;
    const float x = n < n2p ? (float)(p.alpha * p.C[(size_t)k * n2p + n]) : 0.f;
    const float h = rna_tf32(x);
    const uint32_t off = (uint32_t)((k >> 2) * Np * 16 + n * 16 + (k & 3) * 4);
    *reinterpret_cast<float *>(Bhi + off) = h;
    *reinterpret_cast<float *>(Blo + off) = x - h;
  }
  const long long ntile = (p.L + kUM - 1) / kUM;
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < kUStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&full[s])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&mmab)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(saddr(&vbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  // copies of one tile into stage s (thread 0)
  auto issue = [&](long long tile, int s) {
    const long long r0 = tile * kUM;
    const int rows = (int)min((long long)kUM, p.L - r0);
    const uint32_t zbytes = (uint32_t)rows * n2p * 4;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(saddr(&full[s])), "r"(szA + zbytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];"
        :: "r"(saddr(ahi(s))), "l"(&tmpsi), "r"(0), "r"((int)r0), "r"(0), "r"(saddr(&full[s]))
        : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        :: "r"(saddr(zs(s))), "l"(p.Z + r0 * n2p), "r"(zbytes), "r"(saddr(&full[s]))
        : "memory");
  };
  // copies issued / consumed per stage (thread 0 issues; at most one of a
  // stage in flight): the k-th copy into a stage completes its phase k
  int nload[kUStages] = {}, nused[kUStages] = {};
  long long tile = blockIdx.x;
  if (tid == 0)
    for (int s = 0; s < kUStages; ++s) {
      const long long t = tile + (long long)s * gridDim.x;
      if (t < ntile) {
        issue(t, s);
        ++nload[s];
      }
    }
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Np >> 3) << 17) |
                         ((uint32_t)(kUM >> 4) << 24);
  // descriptors: A LBO = 128 rows x 16 B, SBO = 128 B; B LBO = Np x 16 B, SBO = 128 B
  const uint64_t dBh = umma_desc_ls(saddr(Bhi), (uint32_t)Np * 16, 128);
  const uint64_t dBl = umma_desc_ls(saddr(Blo), (uint32_t)Np * 16, 128);
  const uint64_t dAl = umma_desc_ls(saddr(Alo), kUM * 16, 128);
  const uint32_t advA = (2 * kUM * 16) >> 4, advB = (2 * (uint32_t)Np * 16) >> 4;
  float dsum = 0.f, dcmp = 0.f;                  // this thread's column, compensated
  const int dcol = tid & 63, dgrp = tid >> 6;    // dot pass: column, row group (4)
  uint32_t mma_par = 0, v_par = 0, v_issue_par = 0;
  bool stores_pending = false, mma_lost = false, v_pending = false;
  for (int it = 0; tile < ntile; tile += gridDim.x, ++it) {
    const int s = it % kUStages;
    const long long r0 = tile * kUM;
    const int rows = (int)min((long long)kUM, p.L - r0);
    // V rows of this tile (the buffer was released at the end of the last
    // tile): they land while the tile is split, multiplied and read back
    if (p.V && tid == 0) {
      const uint32_t vbytes = (uint32_t)rows * n2p * 4;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                   :: "r"(saddr(&vbar)), "r"(vbytes) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
          :: "r"(saddr(Vs)), "l"(p.V + r0 * n2p), "r"(vbytes), "r"(saddr(&vbar)) : "memory");
      v_pending = true;
      v_issue_par = v_par;
    }
    if (!wait_bar(&full[s], (uint32_t)((it / kUStages) & 1))) abort_flag = 1;
    else ++nused[s];
    __syncthreads();
    if (abort_flag) break;
    // split the Psi tile: hi in place, lo into Alo (same layout)
    {
      float4 *h4 = reinterpret_cast<float4 *>(ahi(s));
      float4 *l4 = reinterpret_cast<float4 *>(Alo);
      for (int e = tid; e < (int)(szA / 16); e += kUThreads) {
        const float4 x = h4[e];
        const float4 h = make_float4(rna_tf32(x.x), rna_tf32(x.y), rna_tf32(x.z), rna_tf32(x.w));
        h4[e] = h;
        l4[e] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dAh = umma_desc_ls(saddr(ahi(s)), kUM * 16, 128);
      for (int j = 0; j < n1p / 8; ++j) {
        mma_tf32(tmem, dAl + advA * j, dBh + advB * j, idesc, j > 0 ? 1u : 0u);
        mma_tf32(tmem, dAh + advA * j, dBl + advB * j, idesc, 1u);
        mma_tf32(tmem, dAh + advA * j, dBh + advB * j, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(saddr(&mmab)) : "memory");
    }
    if (!wait_bar(&mmab, mma_par)) {
      abort_flag = 1;
      mma_lost = true;
    }
    mma_par ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator rows -> Z tile in shared memory
    float *Zt = zs(s);
    {
      const int q = warp & 3, cb = (warp >> 2) * 32;
      const int row = q * 32 + lane;
      if (cb < Np) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)cb;
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
        if (row < rows) {
          float *zr = Zt + (size_t)row * n2p;
#pragma unroll
          for (int c = 0; c < 32; c += 4) {
            if (cb + c < n2p) {
              float4 z = *reinterpret_cast<float4 *>(zr + cb + c);
              z.x += __uint_as_float(r[c]);
              z.y += __uint_as_float(r[c + 1]);
              z.z += __uint_as_float(r[c + 2]);
              z.w += __uint_as_float(r[c + 3]);
              *reinterpret_cast<float4 *>(zr + cb + c) = z;
            }
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (abort_flag) break;
    if (tid == 0) {
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                   :: "l"(p.Z + r0 * n2p), "r"(saddr(Zt)), "r"((uint32_t)rows * n2p * 4)
                   : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      stores_pending = true;
    }
    if (p.V) {
      if (!wait_bar(&vbar, v_par)) abort_flag = 1;
      else if (tid == 0) v_pending = false;
      v_par ^= 1u;
      if (dcol < n2p) {
        float ds0 = 0.f, ds1 = 0.f;
        int r = dgrp;
        for (; r + 4 < rows; r += 8) {
          ds0 = fmaf(Vs[r * n2p + dcol], Zt[r * n2p + dcol], ds0);
          ds1 = fmaf(Vs[(r + 4) * n2p + dcol], Zt[(r + 4) * n2p + dcol], ds1);
        }
        if (r < rows) ds0 = fmaf(Vs[r * n2p + dcol], Zt[r * n2p + dcol], ds0);
        const float y = (ds0 + ds1) - dcmp;
        const float t = dsum + y;
        dcmp = (t - dsum) - y;
        dsum = t;
      }
    }
    __syncthreads();
    if (abort_flag) break;
    // stage s is free once the store has read it: refill it with the tile
    // kUStages ahead
    if (tid == 0) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      const long long t2 = tile + (long long)kUStages * gridDim.x;
      if (t2 < ntile) {
        issue(t2, s);
        ++nload[s];
      }
    }
  }
  if (tid == 0) {
    if (stores_pending) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (abort_flag) {
      atomicExch(p.err, 5);
      // copies still in flight land (bounded wait) before the CTA's shared
      // memory is released, and so do the MMAs of a lost commit
      for (int s = 0; s < kUStages; ++s)
        if (nload[s] > nused[s]) wait_bar(&full[s], (uint32_t)((nload[s] - 1) & 1));
      if (mma_lost) wait_bar(&mmab, mma_par ^ 1u);
      if (v_pending) wait_bar(&vbar, v_issue_par);
    }
  }
  if (p.V) {
    if (dcol < n2p) red[dgrp][dcol] = dsum - dcmp;
    __syncthreads();
    if (tid < n2p) {
      const double v = (double)red[0][tid] + (double)red[1][tid] + (double)red[2][tid] +
                       (double)red[3][tid];
      p.partial[(size_t)blockIdx.x * n2p + tid] = v;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(64)
                 : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
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

size_t defl_update_tc_smem(int n1p, int n2p) {
  const int Np = (n2p + 15) / 16 * 16;
  return 1024 + 2 * (size_t)Np * n1p * 4 + (size_t)kUM * n1p * 4 + (size_t)kUM * n2p * 4 +
         kUStages * ((size_t)kUM * n1p * 4 + (size_t)kUM * n2p * 4);
}

}  // namespace

size_t defl_gram_tc_smem() {
  const size_t ops = 2 * (size_t)(kTM * kGK + 2 * kTN * kGK) * 4;
  const size_t raw = kGStages * (size_t)(2 * kGK * kGLd) * 4;
  static_assert(2 * (kTM * kGK + 2 * kTN * kGK) * 4 >= 64 * 65 * 8, "reduction buffer");
  return ops + raw;
}

// G = Psi^T Z (FP32-accurate, summed in FP64 across CTAs); n1p a multiple of 8
// (<= 64), n2p a multiple of 4 (<= 64); partial holds 2 nsm * n1p * n2p doubles.
cudaError_t launch_defl_gram_tc(const float *Psi, int n1p, const float *Z, int n2p, long long L,
                                double *G, double *partial, int *err, int nsm, cudaStream_t s) {
  if (n1p < 8 || n1p > 64 || n1p % 8 != 0 || n2p < 4 || n2p > 64 || n2p % 4 != 0 || L < 1)
    return cudaErrorInvalidValue;
  const size_t smem = defl_gram_tc_smem();
  cudaError_t e = raise_smem_limit(defl_gram_tc_kernel, smem);
  if (e != cudaSuccess) return e;
  TcGram p;
  p.Psi = Psi;
  p.Z = Z;
  p.partial = partial;
  p.err = err;
  p.n1p = n1p;
  p.n2p = n2p;
  p.L = L;
  const long long ntile = (L + kGK - 1) / kGK;
  const int grid = (int)std::min<long long>(ntile, (long long)kGPerSm * nsm);
  ::invdft::count_launch();
  defl_gram_tc_kernel<<<grid, kGThreads, smem, s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_sum_partials(partial, grid, n1p * n2p, G, s);
}


// Z += alpha Psi C on the tensor cores (n1p a multiple of 8, n2p of 4, both
// <= 64; Psi and Z 16-byte aligned); with V also dot_out[j] = sum_a V[a][j]
// Z_new[a][j].  partial holds nsm * n2p doubles; err: device word set to 5 if
// a wait gave up.
cudaError_t launch_defl_update_tc(const float *Psi, int n1p, const double *C, int n2p,
                                  long long L, float *Z, double alpha, const float *V,
                                  double *dot_out, double *partial, int *err, int nsm,
                                  cudaStream_t s) {
  if (n1p < 8 || n1p > 64 || n1p % 8 != 0 || n2p < 4 || n2p > 64 || n2p % 4 != 0 || L < 1 ||
      ((uintptr_t)Psi & 15) != 0 || ((uintptr_t)Z & 15) != 0)
    return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  // Psi [L][n1p] as (4 floats, node, group of 4 columns): a box of (4, 128,
  // n1p / 4) lands in the K-major operand layout
  CUtensorMap tm;
  const cuuint64_t dims[3] = {4, (cuuint64_t)L, (cuuint64_t)(n1p / 4)};
  const cuuint64_t strides[2] = {(cuuint64_t)n1p * 4, 16};
  const cuuint32_t box[3] = {4, (cuuint32_t)kUM, (cuuint32_t)(n1p / 4)};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)Psi, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  const size_t smem = defl_update_tc_smem(n1p, n2p);
  cudaError_t e = raise_smem_limit(defl_update_tc_kernel, smem);
  if (e != cudaSuccess) return e;
  TcUpdate p;
  p.C = C;
  p.Z = Z;
  p.V = V;
  p.partial = partial;
  p.err = err;
  p.alpha = alpha;
  p.n1p = n1p;
  p.n2p = n2p;
  p.Np = (n2p + 15) / 16 * 16;
  p.L = L;
  const long long ntile = (L + kUM - 1) / kUM;
  const int grid = (int)std::min<long long>(ntile, (long long)nsm);
  ::invdft::count_launch();
  defl_update_tc_kernel<<<grid, kUThreads, smem, s>>>(p, tm);
  e = cudaGetLastError();
  if (e != cudaSuccess || !V) return e;
  return launch_sum_partials(partial, grid, n2p, dot_out, s);
}

}  // namespace invdft
