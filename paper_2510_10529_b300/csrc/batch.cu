// Batched multi-problem execution: the defect-corrected Chebyshev filter
// (Sec. 3.2.2; the FP32 recurrence of the mixed path) of many independent
// problems of uneven mesh size, element order and subspace width, run as one
// cooperative persistent kernel.
//
// Work queue.  An item is (phase k, problem b, cell, column chunk); phase k
// computes D_k = alpha_k (H~ - c) D_(k-1) + beta_k D_(k-2)
//                + alpha_k E diag(p_(k-1)(theta)) for k = 2..m (D_1 is formed
// before the launch).  Items are numbered phase-major, then problem, then
// tile; CTAs take the next number from a device counter.  An item of phase k
// of problem b starts once every item of phase k-1 of the same problem has
// finished (per-problem, per-phase completion counters; the wait is bounded
// and the launch is cooperative, so all CTAs are resident and every awaited
// item is held by a running CTA).  Problems do not wait on one another, so
// the phases of different problems overlap freely.
//
// Buffers.  D_k lives in buf[(k-1) % 3]: phase k gathers D_(k-1), reads
// D_(k-2) at the nodes its cell owns, and scatter-adds into buf[(k-1) % 3]
// (= the buffer of D_(k-3)).  That buffer was zeroed by the owners of its
// nodes during phase k-1, right after they read it as their W term; the first
// two outputs are zeroed before the launch.
//
// Per item, H~ on the cell is the Kronecker-factored element matrix (seven
// 1D contractions in shared memory, even/odd halves of the centrosymmetric
// 1D matrices) on float4 column quads, as in the single-problem FP32 kernel.
#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "batch.h"

namespace invdft {
namespace {

constexpr int kBThreads = 256;
// polls of a phase counter (with back-off) before a wait gives up: read from
// err[1], which the host sets (invdft_batch_set_wait_limit; 2^24 by default,
// 0 = give up at the first wait)

// column-quad arithmetic on packed FP32 pairs (each lane the IEEE
// round-to-nearest operation, as in the scalar forms)
__device__ __forceinline__ float4 f4cat(const float2 &a, const float2 &b) {
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 f4fma(float a, const float4 &x, const float4 &y) {
  const float2 aa = make_float2(a, a);
  return f4cat(__ffma2_rn(aa, make_float2(x.x, x.y), make_float2(y.x, y.y)),
               __ffma2_rn(aa, make_float2(x.z, x.w), make_float2(y.z, y.w)));
}
__device__ __forceinline__ float4 f4add(const float4 &x, const float4 &y) {
  return f4cat(__fadd2_rn(make_float2(x.x, x.y), make_float2(y.x, y.y)),
               __fadd2_rn(make_float2(x.z, x.w), make_float2(y.z, y.w)));
}
// x - y as x + (-1) y (exact product, one rounding)
__device__ __forceinline__ float4 f4sub(const float4 &x, const float4 &y) {
  const float2 m1 = make_float2(-1.f, -1.f);
  return f4cat(__ffma2_rn(m1, make_float2(y.x, y.y), make_float2(x.x, x.y)),
               __ffma2_rn(m1, make_float2(y.z, y.w), make_float2(x.z, x.w)));
}

// even / odd parts of a line of P+1 values (P even)
template <int P>
__device__ __forceinline__ void split_line(const float4 *u, float4 *e, float4 *o) {
  constexpr int H = P / 2;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    e[k] = f4add(u[k], u[P - k]);
    o[k] = f4sub(u[k], u[P - k]);
  }
  e[H] = u[H];
}
// ye, yo (+)= M (e, o) for M given by its even ((H+1)^2) and odd (H^2) blocks
template <int P>
__device__ __forceinline__ void acc_line(const float4 *e, const float4 *o, const float *eM,
                                         const float *oM, float4 *ye, float4 *yo, bool first) {
  constexpr int H = P / 2;
#pragma unroll
  for (int i = 0; i <= H; ++i) {
    float4 s = first ? make_float4(0.f, 0.f, 0.f, 0.f) : ye[i];
#pragma unroll
    for (int k = 0; k <= H; ++k) s = f4fma(eM[i * (H + 1) + k], e[k], s);
    ye[i] = s;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float4 s = first ? make_float4(0.f, 0.f, 0.f, 0.f) : yo[i];
#pragma unroll
    for (int k = 0; k < H; ++k) s = f4fma(oM[i * H + k], o[k], s);
    yo[i] = s;
  }
}
template <int P>
__device__ __forceinline__ void store_line(const float4 *ye, const float4 *yo, float4 *dst,
                                           int stride) {
  constexpr int H = P / 2;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    dst[i * stride] = f4add(ye[i], yo[i]);
    dst[(P - i) * stride] = f4sub(ye[i], yo[i]);
  }
  dst[H * stride] = ye[H];
}

struct Shared {
  float dl[3][5];            // d = m^-1/2 along each axis of the cell
  float tab[52];             // even/odd blocks: eA, oA, eB, oB
  int item;                  // broadcast of the dequeued item
  int abort;
};

// One (phase, cell, chunk) item of problem bp with C columns per chunk.
template <int P, int C>
__device__ void run_item(const BatchProb &bp, int k, int cell, int c0, float4 *u, float4 *w,
                         Shared &sh) {
  constexpr int Q = P + 1, NE = Q * Q * Q, Q4 = C / 4, NL = Q * Q;
  constexpr int H = P / 2, NEc = (H + 1) * (H + 1), NOc = H * H;
  const int tid = threadIdx.x;
  const int nc = bp.ncell, Ni = bp.Ni, ncol = bp.ncol;
  const int cx = cell % nc, cy = (cell / nc) % nc, cz = cell / (nc * nc);
  const float *X = bp.buf[(k - 2) % 3];
  float *Z = bp.buf[(k - 1) % 3];
  float *W = k >= 3 ? bp.buf[(k - 3) % 3] : nullptr;
  const float alpha = bp.alpha[k], beta = bp.beta[k];
  const bool vec = (ncol & 3) == 0;
  if (tid < 3 * Q) {
    const int d = tid / Q, t = tid % Q;
    sh.dl[d][t] = bp.dm1f[(d == 0 ? cx : (d == 1 ? cy : cz)) * P + t];
  }
  if (tid < 2 * (NEc + NOc)) sh.tab[tid] = bp.tab[tid];
  __syncthreads();
  const float *eA = sh.tab, *oA = sh.tab + NEc, *eB = oA + NOc, *oB = eB + NEc;
  // gather u = d o X over the cell (L2 loads: X was written by other CTAs)
  for (int idx = tid; idx < NE * Q4; idx += kBThreads) {
    const int a = idx / Q4, c4 = idx - (idx / Q4) * Q4;
    const int lx = a % Q, ly = (a / Q) % Q, lz = a / (Q * Q);
    const int gx = cx * P + lx, gy = cy * P + ly, gz = cz * P + lz;
    const int col = c0 + 4 * c4;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gx >= 1 && gx <= Ni && gy >= 1 && gy <= Ni && gz >= 1 && gz <= Ni && col < ncol) {
      const size_t e0 = ((size_t)(gx - 1) + (size_t)Ni * ((gy - 1) + (size_t)Ni * (gz - 1))) * ncol + col;
      if (vec) {
        x = __ldcg(reinterpret_cast<const float4 *>(X + e0));
      } else {
        x.x = __ldcg(X + e0);
        x.y = col + 1 < ncol ? __ldcg(X + e0 + 1) : 0.f;
        x.z = col + 2 < ncol ? __ldcg(X + e0 + 2) : 0.f;
        x.w = col + 3 < ncol ? __ldcg(X + e0 + 3) : 0.f;
      }
      const float sc = sh.dl[0][lx] * sh.dl[1][ly] * sh.dl[2][lz];
      x = make_float4(sc * x.x, sc * x.y, sc * x.z, sc * x.w);
    }
    u[idx] = x;
  }
  __syncthreads();
  // x lines: u <- B_x u, w <- A_x u
  for (int t = tid; t < NL * Q4; t += kBThreads) {
    const int l = t / Q4, q = t - l * Q4;
    float4 in[Q], e[H + 1], o[H > 0 ? H : 1], ye[H + 1], yo[H > 0 ? H : 1];
#pragma unroll
    for (int x = 0; x < Q; ++x) in[x] = u[(Q * l + x) * Q4 + q];
    split_line<P>(in, e, o);
    acc_line<P>(e, o, eB, oB, ye, yo, true);
    store_line<P>(ye, yo, u + Q * l * Q4 + q, Q4);
    acc_line<P>(e, o, eA, oA, ye, yo, true);
    store_line<P>(ye, yo, w + Q * l * Q4 + q, Q4);
  }
  __syncthreads();
  // y lines: u <- B_y u, w <- A_y u + B_y w
  for (int t = tid; t < NL * Q4; t += kBThreads) {
    const int l = t / Q4, q = t - l * Q4;
    const int lb = (l % Q) + Q * Q * (l / Q);
    float4 in[Q], e[H + 1], o[H > 0 ? H : 1], ye[H + 1], yo[H > 0 ? H : 1];
#pragma unroll
    for (int y = 0; y < Q; ++y) in[y] = u[(lb + Q * y) * Q4 + q];
    split_line<P>(in, e, o);
    acc_line<P>(e, o, eB, oB, ye, yo, true);
    store_line<P>(ye, yo, u + lb * Q4 + q, Q * Q4);
    acc_line<P>(e, o, eA, oA, ye, yo, true);
#pragma unroll
    for (int y = 0; y < Q; ++y) in[y] = w[(lb + Q * y) * Q4 + q];
    split_line<P>(in, e, o);
    acc_line<P>(e, o, eB, oB, ye, yo, false);
    store_line<P>(ye, yo, w + lb * Q4 + q, Q * Q4);
  }
  __syncthreads();
  // z lines: u <- A_z u + B_z w
  for (int t = tid; t < NL * Q4; t += kBThreads) {
    const int l = t / Q4, q = t - l * Q4;
    float4 in[Q], e[H + 1], o[H > 0 ? H : 1], ye[H + 1], yo[H > 0 ? H : 1];
#pragma unroll
    for (int z = 0; z < Q; ++z) in[z] = u[(l + Q * Q * z) * Q4 + q];
    split_line<P>(in, e, o);
    acc_line<P>(e, o, eA, oA, ye, yo, true);
#pragma unroll
    for (int z = 0; z < Q; ++z) in[z] = w[(l + Q * Q * z) * Q4 + q];
    split_line<P>(in, e, o);
    acc_line<P>(e, o, eB, oB, ye, yo, false);
    store_line<P>(ye, yo, u + l * Q4 + q, Q * Q * Q4);
  }
  __syncthreads();
  // epilogue: scatter-add; nodal, W and E terms (and zeroing of W) at the
  // nodes the cell owns (local index < P on every axis)
  for (int idx = tid; idx < NE * Q4; idx += kBThreads) {
    const int a = idx / Q4, c4 = idx - (idx / Q4) * Q4;
    const int lx = a % Q, ly = (a / Q) % Q, lz = a / (Q * Q);
    const int gx = cx * P + lx, gy = cy * P + ly, gz = cz * P + lz;
    const int col = c0 + 4 * c4;
    if (gx < 1 || gx > Ni || gy < 1 || gy > Ni || gz < 1 || gz > Ni || col >= ncol) continue;
    const size_t node = (size_t)(gx - 1) + (size_t)Ni * ((gy - 1) + (size_t)Ni * (gz - 1));
    const size_t e0 = node * ncol + col;
    const int m = min(4, ncol - col);
    const float sc = bp.kc * alpha * sh.dl[0][lx] * sh.dl[1][ly] * sh.dl[2][lz];
    const float4 y = u[idx];
    float o[4] = {sc * y.x, sc * y.y, sc * y.z, sc * y.w};
    if (lx < P && ly < P && lz < P) {
      const float va = __ldg(bp.v + node);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t >= m) break;
        const float xv = __ldcg(X + e0 + t);
        const float ev = __ldg(bp.E + e0 + t);
        float tt = alpha * (va - bp.shift) * xv;
        tt = fmaf(alpha * (float)bp.pk[(size_t)(k - 1) * ncol + col + t], ev, tt);
        if (W) {
          tt = fmaf(beta, __ldcg(W + e0 + t), tt);
          W[e0 + t] = 0.f;      // D_(k-2) is dead: it becomes the output of phase k+1
        }
        o[t] += tt;
      }
    }
    float *dst = Z + e0;
    if (vec) {
      asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};"
                   :: "l"(dst), "f"(o[0]), "f"(o[1]), "f"(o[2]), "f"(o[3]) : "memory");
    } else {
      for (int t = 0; t < m; ++t)
        asm volatile("red.global.add.f32 [%0], %1;" :: "l"(dst + t), "f"(o[t]) : "memory");
    }
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kBThreads)
batch_filter_kernel(const BatchProb *__restrict__ probs, int nprob, int m, int per_phase,
                    int *__restrict__ queue, unsigned *__restrict__ done, int *__restrict__ err) {
  extern __shared__ __align__(16) float4 bsm[];
  __shared__ Shared sh;
  const int tid = threadIdx.x;
  const int total = (m - 1) * per_phase;
  const long long wait_limit = (long long)ld_acquire((const unsigned *)err + 1);
  if (tid == 0) sh.abort = 0;
  for (;;) {
    __syncthreads();
    if (tid == 0) sh.item = atomicAdd(queue, 1);
    __syncthreads();
    const int it = sh.item;
    if (it >= total) break;
    const int k = 2 + it / per_phase;
    int r = it - (k - 2) * per_phase, b = 0;
    while (b + 1 < nprob && r >= probs[b + 1].item0) ++b;
    const BatchProb &bp = probs[b];
    r -= bp.item0;
    const int cell0 = r / bp.nchunk, chunk = r - cell0 * bp.nchunk;
    const int cell = bp.perm ? bp.perm[cell0] : cell0;
    // wait for phase k-1 of this problem (bounded, with back-off)
    if (tid == 0 && k >= 3) {
      const unsigned need = (unsigned)bp.items;
      const unsigned *cnt = done + (size_t)b * (m + 1) + (k - 1);
      long long polls = 0;
      for (;;) {
        // a zero limit gives up at the first wait, complete or not
        if (wait_limit > 0 && ld_acquire(cnt) >= need) break;
        if (++polls > wait_limit || ld_acquire((const unsigned *)err) != 0) {
          sh.abort = 1;
          break;
        }
        __nanosleep(256);
      }
      __threadfence();
    }
    __syncthreads();
    if (sh.abort) {
      if (tid == 0) atomicCAS(err, 0, 1);
      break;
    }
    float4 *u = bsm, *w = bsm + 125 * 8;
    const int c0 = chunk * bp.C;
    if (bp.p == 4) {
      if (bp.C == 8) run_item<4, 8>(bp, k, cell, c0, u, w, sh);
      else if (bp.C == 16) run_item<4, 16>(bp, k, cell, c0, u, w, sh);
      else run_item<4, 32>(bp, k, cell, c0, u, w, sh);
    } else {
      if (bp.C == 8) run_item<2, 8>(bp, k, cell, c0, u, w, sh);
      else if (bp.C == 16) run_item<2, 16>(bp, k, cell, c0, u, w, sh);
      else run_item<2, 32>(bp, k, cell, c0, u, w, sh);
    }
    // publish: every thread's reductions and stores, then the counter
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicAdd(done + (size_t)b * (m + 1) + k, 1u);
  }
}

}  // namespace

size_t batch_filter_smem() { return 2 * (size_t)125 * 8 * sizeof(float4); }

cudaError_t batch_filter_occupancy(int *per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_filter_kernel, kBThreads,
                                                       batch_filter_smem());
}

cudaError_t launch_batch_filter(const BatchProb *d_probs, int nprob, int m, int per_phase,
                                int *queue, unsigned *done, int *err, int grid, cudaStream_t s) {
  const size_t smem = batch_filter_smem();
  cudaError_t e = raise_smem_limit(batch_filter_kernel, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ::invdft::count_launch();
  return cudaLaunchKernelEx(&cfg, batch_filter_kernel, d_probs, nprob, m, per_phase, queue, done,
                            err);
}

}  // namespace invdft
