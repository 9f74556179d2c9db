// H~X: the finite-element Hamiltonian in standard form applied to a block of
// vectors, cell by cell (Sec. 3.2.3, Eq. 17, Eq. 19).
//
//   Z = alpha * (D K D X + (v - shift) o X) + beta * W + alpha * E diag(escale)
//
// Two launches: a nodal pass writes everything but the kinetic term, then the
// cell pass gathers X_e (scaled by d = m^-1/2) for each cell, applies the
// dense cell matrix K_e in its Kronecker-factored form and scatter-adds
// d o (K_e X_e) into Z.  K_e = kc (B(x)B(x)A + B(x)A(x)B + A(x)B(x)B) is the
// exact dense 125x125 (Q4) matrix; applying it as seven 1D contractions of the
// (p+1)^3 cell tensor gives the same product with 3.5x fewer FP64 operations,
// which matters because FP64 is the scarce pipe on this part.
#include <algorithm>

#include "internal.h"

namespace invdft {
namespace {

template <typename T>
__global__ void hx_nodal(const T *__restrict__ X, T *__restrict__ Z, const double *__restrict__ v,
                         long long L, int ncol, double alpha, double shift,
                         const double *__restrict__ shift_col, const T *__restrict__ W, double beta,
                         const float *__restrict__ E, const double *__restrict__ escale,
                         FastDiv fd) {
  const uint32_t n = (uint32_t)(L * (long long)ncol);
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint32_t a = fdiv(i, fd);
    const int j = (int)(i - a * (uint32_t)ncol);
    const double sh = shift_col ? shift_col[j] : shift;
    double z = alpha * ((v ? v[a] : 0.0) - sh) * (double)X[i];
    if (W) z += beta * (double)W[i];
    if (E) z += alpha * escale[j] * (double)E[i];
    Z[i] = (T)z;
  }
}

template <typename T>
__device__ __forceinline__ void atomic_add(T *p, T x) { atomicAdd(p, x); }

// The 1D matrices A and B are centrosymmetric (M[i][j] = M[P-i][P-j] for GLL
// nodes symmetric about the cell centre), so y = M u splits into an even part
// on e_k = u_k + u_(P-k) and an odd part on o_k = u_k - u_(P-k):
//   y_i = ye_i + yo_i,  y_(P-i) = ye_i - yo_i (i < P/2),  y_(P/2) = ye_(P/2),
// with (P/2+1)^2 + (P/2)^2 coefficients instead of (P+1)^2 (13 instead of 25
// FMAs for Q4).
template <int P>
struct EoTab {
  static constexpr int H = P / 2, NE = (H + 1) * (H + 1), NO = H * H;
  double eA[NE], oA[NO], eB[NE], oB[NO];
};

template <int P>
EoTab<P> make_eo(const Geom &g) {
  constexpr int Q = P + 1, H = P / 2;
  EoTab<P> t;
  auto sym = [&](const double *M, int i, int j) {
    return 0.5 * (M[i * Q + j] + M[(P - i) * Q + (P - j)]);
  };
  for (int m = 0; m < 2; ++m) {
    const double *M = m == 0 ? g.A : g.B;
    double *e = m == 0 ? t.eA : t.eB, *o = m == 0 ? t.oA : t.oB;
    for (int i = 0; i <= H; ++i)
      for (int k = 0; k <= H; ++k)
        e[i * (H + 1) + k] = k < H ? 0.5 * (sym(M, i, k) + sym(M, i, P - k)) : sym(M, i, H);
    for (int i = 0; i < H; ++i)
      for (int k = 0; k < H; ++k) o[i * H + k] = 0.5 * (sym(M, i, k) - sym(M, i, P - k));
  }
  return t;
}

template <typename T, int P>
__device__ __forceinline__ void eo_split(const T *u, T *e, T *o) {
  constexpr int H = P / 2;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    e[k] = u[k] + u[P - k];
    o[k] = u[k] - u[P - k];
  }
  e[H] = u[H];
}

// y = M1 u1 (+ M2 u2) from the even/odd parts of u1 (and u2)
template <typename T, int P, bool TWO>
__device__ __forceinline__ void eo_apply(const T *e1, const T *o1, const T *eM1, const T *oM1,
                                         const T *e2, const T *o2, const T *eM2, const T *oM2,
                                         T *y) {
  constexpr int H = P / 2;
  T ye[H + 1], yo[H > 0 ? H : 1];
#pragma unroll
  for (int i = 0; i <= H; ++i) {
    T s = 0;
#pragma unroll
    for (int k = 0; k <= H; ++k) {
      s += eM1[i * (H + 1) + k] * e1[k];
      if (TWO) s += eM2[i * (H + 1) + k] * e2[k];
    }
    ye[i] = s;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T s = 0;
#pragma unroll
    for (int k = 0; k < H; ++k) {
      s += oM1[i * H + k] * o1[k];
      if (TWO) s += oM2[i * H + k] * o2[k];
    }
    yo[i] = s;
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    y[i] = ye[i] + yo[i];
    y[P - i] = ye[i] - yo[i];
  }
  y[H] = ye[H];
}

// One CTA per (cell, chunk of C columns).  Two shared buffers of (p+1)^3 x C.
// The cell's per-axis scalars (2/h_a for A, h_a/2 for B) scale each 1D
// contraction, so box cells of any size (graded meshes) take the same path.
template <typename T, int P, int C>
__global__ void __launch_bounds__(256) hx_cells(const T *__restrict__ X, T *__restrict__ Z,
                                                int ncol, Geom g, EoTab<P> tab, double scale) {
  constexpr int Q = P + 1, NE = Q * Q * Q, H = P / 2;
  constexpr int NEC = EoTab<P>::NE, NOC = EoTab<P>::NO;
  extern __shared__ unsigned char smem_raw[];
  T *u = reinterpret_cast<T *>(smem_raw);
  T *w = u + NE * C;
  __shared__ T eA[NEC], oA[NOC > 0 ? NOC : 1], eB[NEC], oB[NOC > 0 ? NOC : 1];
  __shared__ double dl[3][Q];
  __shared__ int gidx[3][Q];

  const int cell = blockIdx.x;
  const int cx = cell % g.nc[0], cy = (cell / g.nc[0]) % g.nc[1], cz = cell / (g.nc[0] * g.nc[1]);
  const int c0 = blockIdx.y * C;
  const T sAx = (T)g.cellA[0][cx], sBx = (T)g.cellB[0][cx];
  const T sAy = (T)g.cellA[1][cy], sBy = (T)g.cellB[1][cy];
  const T sAz = (T)g.cellA[2][cz], sBz = (T)g.cellB[2][cz];
  const int tid = threadIdx.x;

  if (tid < NEC) {
    eA[tid] = (T)tab.eA[tid];
    eB[tid] = (T)tab.eB[tid];
  }
  if (tid < NOC) {
    oA[tid] = (T)tab.oA[tid];
    oB[tid] = (T)tab.oB[tid];
  }
  if (tid < 3 * Q) {
    const int d = tid / Q, l = tid % Q;
    const int c = d == 0 ? cx : (d == 1 ? cy : cz);
    const int gi = c * P + l;                 // full-grid index along the axis
    dl[d][l] = g.dnode[d][gi];                // 0 on the boundary
    gidx[d][l] = (gi >= 1 && gi <= g.n[d]) ? gi - 1 : -1;
  }
  __syncthreads();

  // gather: u[a][j] = d_a X[node(a)][c0 + j]
  for (int idx = tid; idx < NE * C; idx += blockDim.x) {
    const int a = idx / C, j = idx - a * C;
    const int lx = a % Q, ly = (a / Q) % Q, lz = a / (Q * Q);
    const int ix = gidx[0][lx], iy = gidx[1][ly], iz = gidx[2][lz];
    T val = (T)0;
    if (ix >= 0 && iy >= 0 && iz >= 0 && c0 + j < ncol) {
      const long long node = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
      val = (T)(dl[0][lx] * dl[1][ly] * dl[2][lz]) * X[node * ncol + c0 + j];
    }
    u[idx] = val;
  }
  __syncthreads();

  // x lines: u <- B_x u, w <- A_x u
  for (int idx = tid; idx < Q * Q * C; idx += blockDim.x) {
    const int j = idx % C, line = idx / C;
    const int base = line * Q;
    T in[Q], e[H + 1], o[H > 0 ? H : 1], yb[Q], ya[Q];
#pragma unroll
    for (int x = 0; x < Q; ++x) in[x] = u[(base + x) * C + j];
    eo_split<T, P>(in, e, o);
    eo_apply<T, P, false>(e, o, eB, oB, e, o, eB, oB, yb);
    eo_apply<T, P, false>(e, o, eA, oA, e, o, eA, oA, ya);
#pragma unroll
    for (int xo = 0; xo < Q; ++xo) {
      u[(base + xo) * C + j] = sBx * yb[xo];
      w[(base + xo) * C + j] = sAx * ya[xo];
    }
  }
  __syncthreads();

  // y lines: u <- B_y u (= B_y B_x X), w <- A_y u + B_y w (= A_y B_x X + B_y A_x X)
  for (int idx = tid; idx < Q * Q * C; idx += blockDim.x) {
    const int j = idx % C, r = idx / C;
    const int x = r % Q, z = r / Q;
    T t1[Q], t2[Q], e1[H + 1], o1[H > 0 ? H : 1], e2[H + 1], o2[H > 0 ? H : 1], y1[Q], y2[Q];
#pragma unroll
    for (int y = 0; y < Q; ++y) {
      t1[y] = u[(x + Q * (y + Q * z)) * C + j];
      t2[y] = w[(x + Q * (y + Q * z)) * C + j];
    }
    eo_split<T, P>(t1, e1, o1);
    eo_split<T, P>(t2, e2, o2);
    T ya[Q];
    eo_apply<T, P, false>(e1, o1, eB, oB, e1, o1, eB, oB, y1);
    eo_apply<T, P, false>(e1, o1, eA, oA, e1, o1, eA, oA, ya);
    eo_apply<T, P, false>(e2, o2, eB, oB, e2, o2, eB, oB, y2);
#pragma unroll
    for (int yo = 0; yo < Q; ++yo) {
      u[(x + Q * (yo + Q * z)) * C + j] = sBy * y1[yo];
      w[(x + Q * (yo + Q * z)) * C + j] = sAy * ya[yo] + sBy * y2[yo];
    }
  }
  __syncthreads();

  // z lines: u <- A_z u + B_z w
  for (int idx = tid; idx < Q * Q * C; idx += blockDim.x) {
    const int j = idx % C, r = idx / C;
    const int x = r % Q, y = r / Q;
    T t1[Q], t2[Q], e1[H + 1], o1[H > 0 ? H : 1], e2[H + 1], o2[H > 0 ? H : 1], yz[Q];
#pragma unroll
    for (int z = 0; z < Q; ++z) {
      t1[z] = u[(x + Q * (y + Q * z)) * C + j];
      t2[z] = w[(x + Q * (y + Q * z)) * C + j];
    }
    eo_split<T, P>(t1, e1, o1);
    eo_split<T, P>(t2, e2, o2);
    T yb[Q];
    eo_apply<T, P, false>(e1, o1, eA, oA, e1, o1, eA, oA, yz);
    eo_apply<T, P, false>(e2, o2, eB, oB, e2, o2, eB, oB, yb);
#pragma unroll
    for (int zo = 0; zo < Q; ++zo) u[(x + Q * (y + Q * zo)) * C + j] = sAz * yz[zo] + sBz * yb[zo];
  }
  __syncthreads();

  // scatter-add d_a * scale * (K_e X_e)_a
  for (int idx = tid; idx < NE * C; idx += blockDim.x) {
    const int a = idx / C, j = idx - a * C;
    const int lx = a % Q, ly = (a / Q) % Q, lz = a / (Q * Q);
    const int ix = gidx[0][lx], iy = gidx[1][ly], iz = gidx[2][lz];
    if (ix >= 0 && iy >= 0 && iz >= 0 && c0 + j < ncol) {
      const long long node = ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
      const T val = (T)(scale * dl[0][lx] * dl[1][ly] * dl[2][lz]) * u[idx];
      atomic_add(&Z[node * ncol + c0 + j], val);
    }
  }
}

template <typename T, int P, int C>
cudaError_t run_cells(const Geom &g, const T *X, T *Z, int ncol, double scale, cudaStream_t s) {
  constexpr int Q = P + 1, NE = Q * Q * Q;
  const size_t smem = 2 * (size_t)NE * C * sizeof(T);
  auto k = hx_cells<T, P, C>;
  cudaError_t e = raise_smem_limit(k, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(g.nc[0] * g.nc[1] * g.nc[2], (ncol + C - 1) / C);
  ::invdft::count_launch();
  k<<<grid, 256, smem, s>>>(X, Z, ncol, g, make_eo<P>(g), scale);
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t run_cells_p(const Geom &g, const T *X, T *Z, int ncol, double scale, cudaStream_t s) {
  if (ncol <= 8) return run_cells<T, P, 8>(g, X, Z, ncol, scale, s);
  if (ncol <= 16) return run_cells<T, P, 16>(g, X, Z, ncol, scale, s);
  return run_cells<T, P, 32>(g, X, Z, ncol, scale, s);
}

template <typename T>
cudaError_t launch_hx_t(const Geom &g, const double *v, const HxArgs<T> &a, cudaStream_t s) {
  if (a.ncol < 1 || a.ncol > kMaxCols) return cudaErrorInvalidValue;
  const long long n = g.L * a.ncol;
  int blocks = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
  ::invdft::count_launch();
  hx_nodal<T><<<blocks, 256, 0, s>>>(a.X, a.Z, v, g.L, a.ncol, a.alpha, a.shift, a.shift_col, a.W,
                                     a.beta, a.E, a.escale, make_fastdiv(a.ncol));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // K_e = 1/2 (B_z B_y A_x + B_z A_y B_x + A_z B_y B_x) with the cell scalars
  const double scale = 0.5 * a.alpha;
  if (g.p == 2) return run_cells_p<T, 2>(g, a.X, a.Z, a.ncol, scale, s);
  if (g.p == 4) return run_cells_p<T, 4>(g, a.X, a.Z, a.ncol, scale, s);
  if (g.p == 6) return run_cells_p<T, 6>(g, a.X, a.Z, a.ncol, scale, s);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_hx(const Geom &g, const double *v, const HxArgs<double> &a, cudaStream_t s) {
  return launch_hx_t<double>(g, v, a, s);
}
cudaError_t launch_hx(const Geom &g, const double *v, const HxArgs<float> &a, cudaStream_t s) {
  return launch_hx_t<float>(g, v, a, s);
}

}  // namespace invdft

namespace invdft {
namespace {

// route an FP32 block to the tensor-core kernel when the mesh is Q4, the
// caller asked for it and the output does not alias an input (the kernel
// zeroes Z before accumulating into it)
bool uses_tc(const Ctx *c, const HxArgs<double> &) { return false; }
bool uses_tc(const Ctx *c, const HxArgs<float> &a) {
  return a.tc && c->g.p == 4 && c->Ke_tc && a.Z != a.X && a.Z != a.W &&
         (const void *)a.Z != (const void *)a.E;
}
template <typename T>
bool uses_sweep(const Ctx *c, const HxArgs<T> &a) {
  return sweep_supported(c->g, a.ncol, sizeof(T), a.X, a.Z, a.W, a.E);
}

// Tile variant and z-segment length of the sweep kernel for this launch: the
// ones fixed by invdft_tune_hx, else the autotuned pair for (precision, ncol,
// W, E).  The autotuner times every candidate (each tile variant with the
// whole z range, halves, quarters, segments short enough for two CTAs per SM
// and the persistent balanced schedule) on the first such launch of a large
// mesh, writing into the launch's own output, and keeps the fastest; on small
// meshes, or while the stream is being captured, the defaults are used
// (variant 0, the whole z range).
template <typename T>
std::pair<int, int> sweep_config(Ctx *c, const T *v, const HxArgs<T> &a, cudaStream_t s) {
  const int nc = c->g.nc[2], nvar = sweep_variants(c->g, sizeof(T));
  const int fv = c->hx_variant_fixed < nvar ? c->hx_variant_fixed : -1;
  const int fs = c->hx_seglen_fixed == kSegBalanced ? kSegBalanced
                 : c->hx_seglen_fixed > 0             ? std::min(c->hx_seglen_fixed, nc)
                                                      : 0;
  if (fv >= 0 && fs > 0) return {fv, fs};
  const long long key = ((long long)a.ncol << 8) | (sizeof(T) << 2) | (a.W ? 2 : 0) | (a.E ? 1 : 0);
  auto it = c->hx_tuned.find(key);
  if (it != c->hx_tuned.end()) {
    return {fv >= 0 ? fv : it->second.first, fs > 0 ? fs : it->second.second};
  }
  // default: segments short enough for two CTAs per SM (a negative length is
  // resolved per launch from the variant's tile count)
  const int par = -2 * std::max(c->nsm, 1);
  const std::pair<int, int> dflt{fv >= 0 ? fv : 0, fs > 0 ? fs : par};
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return dflt;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return dflt;
  }
  std::pair<int, int> best = dflt;
  float best_ms = 1e30f;
  const int segs[5] = {nc, (nc + 1) / 2, (nc + 3) / 4, par, kSegBalanced};
  for (int var = 0; var < nvar; ++var) {
    if (fv >= 0 && var != fv) continue;
    for (int k = 0; k < 5; ++k) {
      const int seg = fs > 0 ? fs : segs[k];
      if (fs > 0 && k > 0) break;
      if (k > 0 && segs[k] == segs[k - 1]) continue;
      // the balanced schedule exists for the plain epilogue on uniform meshes
      if (segs[k] == kSegBalanced && (a.W || a.E || c->g.graded)) continue;
      int *err = c->status + kStWaitHxSweep;
      bool ok = launch_hx_sweep(c->g, v, a, err, var, seg, s) == cudaSuccess;
      ok = ok && cudaEventRecord(e0, s) == cudaSuccess;
      for (int r = 0; r < 2 && ok; ++r) ok = launch_hx_sweep(c->g, v, a, err, var, seg, s) == cudaSuccess;
      ok = ok && cudaEventRecord(e1, s) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
      float ms = 0.f;
      if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = {var, seg};
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  c->hx_tuned[key] = best;
  return best;
}

template <typename T>
cudaError_t sweep_op(Ctx *c, const T *v, const HxArgs<T> &a, cudaStream_t s) {
  const std::pair<int, int> cfg = sweep_config(c, v, a, s);
  return launch_hx_sweep(c->g, v, a, c->status + kStWaitHxSweep, cfg.first, cfg.second, s);
}

cudaError_t dispatch_hx(Ctx *c, const HxArgs<double> &a, cudaStream_t s) {
  if (uses_sweep(c, a)) return sweep_op(c, c->v, a, s);
  return launch_hx(c->g, c->v, a, s);
}
cudaError_t dispatch_hx(Ctx *c, const HxArgs<float> &a, cudaStream_t s) {
  if (uses_tc(c, a))
    return launch_hx_tc(c->g, c->v, a, c->Ke_tc, c->cell_perm, c->status + kStWaitHxTc, s);
  if (uses_sweep(c, a)) return sweep_op(c, c->vf, a, s);
  return launch_hx(c->g, c->v, a, s);
}

template <typename T>
cudaError_t hx_op_t(Ctx *c, const HxArgs<T> &a, cudaStream_t s) {
  HxProf &p = c->prof;
  if (!p.on) return dispatch_hx(c, a, s);
  const double L = (double)c->L, n = a.ncol, sz = sizeof(T);
  // kinds: 0 FP64, 1 FP32 with the filter's W / E terms, 2 other FP32 (the
  // MINRES operator), 3 TF32 tensor cores
  const bool tc = uses_tc(c, a);
  const int kind = sizeof(T) == 8 ? 0 : (tc ? 3 : ((a.W || a.E) ? 1 : 2));
  // X read, Z written, v read (the FP32 copy on the FP32 CUDA-core paths)
  double bytes = (2.0 * n * sz + ((sizeof(T) == 4 && !tc) ? 4.0 : 8.0)) * L;
  if (a.W) bytes += n * sz * L;
  if (a.E) bytes += n * 4.0 * L;
  const double ne = (double)c->g.q * c->g.q * c->g.q;
  const double cells = (double)c->g.nc[0] * c->g.nc[1] * c->g.nc[2];
  const int k = prof_begin(c, kind, bytes, 2.0 * ne * ne * n * cells, s);
  cudaError_t r = dispatch_hx(c, a, s);
  prof_end(c, k, s);
  return r;
}

}  // namespace

int prof_begin(Ctx *c, int kind, double bytes, double flops, cudaStream_t s) {
  HxProf &p = c->prof;
  if (!p.on) return -1;
  const int slots = 1024;
  if (p.ev.empty()) {
    p.ev.resize(2 * slots);
    p.kind.resize(slots);
    p.bytes.resize(slots);
    p.flops.resize(slots);
    for (auto &e : p.ev)
      if (cudaEventCreate(&e) != cudaSuccess) {
        p.on = false;      // no timing rather than a failed launch
        return -1;
      }
  }
  if (p.used == slots && prof_flush(c) != cudaSuccess) return -1;
  const int k = p.used++;
  p.kind[k] = kind;
  p.bytes[k] = bytes;
  p.flops[k] = flops;
  cudaEventRecord(p.ev[2 * k], s);
  return k;
}

void prof_end(Ctx *c, int slot, cudaStream_t s) {
  if (slot >= 0) cudaEventRecord(c->prof.ev[2 * slot + 1], s);
}

cudaError_t prof_flush(Ctx *c) {
  HxProf &p = c->prof;
  if (p.used == 0) return cudaSuccess;
  cudaError_t r = cudaEventSynchronize(p.ev[2 * (p.used - 1) + 1]);
  if (r != cudaSuccess) return r;
  for (int k = 0; k < p.used; ++k) {
    float ms = 0.f;
    r = cudaEventElapsedTime(&ms, p.ev[2 * k], p.ev[2 * k + 1]);
    if (r != cudaSuccess) return r;
    const int t = p.kind[k];
    p.ms[t] += ms;
    p.bytes_sum[t] += p.bytes[k];
    p.flops_sum[t] += p.flops[k];
    p.n[t] += 1;
  }
  p.used = 0;
  return cudaSuccess;
}

cudaError_t hx_op(Ctx *c, const HxArgs<double> &a, cudaStream_t s) { return hx_op_t(c, a, s); }

// D K D X (+ the shift, W and E terms) without the collocated potential: the
// kinetic part of an operator whose potential term is given elsewhere
cudaError_t hx_op_nopot(Ctx *c, const HxArgs<double> &a, cudaStream_t s) {
  if (uses_sweep(c, a)) {
    const std::pair<int, int> cfg = sweep_config(c, (const double *)nullptr, a, s);
    return launch_hx_sweep(c->g, (const double *)nullptr, a, c->status + kStWaitHxSweep,
                           cfg.first, cfg.second, s);
  }
  return launch_hx(c->g, nullptr, a, s);
}
cudaError_t hx_op_nopot(Ctx *c, const HxArgs<float> &a, cudaStream_t s) {
  if (uses_sweep(c, a)) {
    const std::pair<int, int> cfg = sweep_config(c, (const float *)nullptr, a, s);
    return launch_hx_sweep(c->g, (const float *)nullptr, a, c->status + kStWaitHxSweep,
                           cfg.first, cfg.second, s);
  }
  return launch_hx(c->g, nullptr, a, s);
}
cudaError_t hx_op(Ctx *c, const HxArgs<float> &a, cudaStream_t s) { return hx_op_t(c, a, s); }

}  // namespace invdft
