// Dense per-cell potential matrices: the Gauss-quadrature reading of the
// potential term of Eq. 17,
//   V_e[a][b] = sum_g W_g v(x_g) N_a(x_g) N_b(x_g),
//   W_g = (h_x/2)(h_y/2)(h_z/2) w_gx w_gy w_gz,  v(x_g) = sum_c v_c N_c(x_g),
// with n_g = 2p Gauss points per axis (exact for the interpolated v), one
// dense (p+1)^3 x (p+1)^3 matrix per cell; v is given on the full node grid
// (the Dirichlet boundary nodes included).  The standard form keeps the lumped
// GLL mass:  H~ = D (K + V) D,  D = M^-1/2.
//
// Building a cell's matrix is a sum factorisation: v at the Gauss points by
// three 1D interpolations, then V_e = sum over the Gauss points of
// W v psi_x psi_y psi_z with psi(g, a, b) = l_a(x_g) l_b(x_g), contracted
// one axis at a time.  Applying it (after the kinetic part, which the H~X
// kernels compute with the potential term switched off) is one dense product
// V_e (D X)_e per cell, scaled by D and added into the output.
#include <cmath>

#include "internal.h"

namespace invdft {
namespace {

constexpr int kVdMaxNg = 8;

struct VdGeom {
  int nc[3], n[3];
  const double *cellB[3];    // h_e / 2 per cell and axis
  const double *dnode[3];    // m1^-1/2 per node and axis (0 on the boundary)
  double phi[kVdMaxNg * kMaxQ];   // l_j(x_k), k < ng, j <= p
  double wg[kVdMaxNg];
};

// element (row a, column b) of a 128 x 128 FP32 tile in the no-swizzle
// K-major layout of the tensor-core kernels: 8 x 16-byte core matrices,
// K-adjacent ones 128 B apart, 8-row groups 4096 B apart (bytes / 4)
__host__ __device__ __forceinline__ int umma_index(int a, int b) {
  return ((a >> 3) * 4096 + (b >> 2) * 128 + (a & 7) * 16 + (b & 3) * 4) / 4;
}

template <int P>
struct BuildSmem {
  static constexpr int Q = P + 1, NG = 2 * P;
  static constexpr size_t doubles =
      Q * Q * Q + Q * Q * NG + Q * NG * NG + NG * NG * NG + NG * NG * Q * Q + NG * Q * Q * Q * Q;
};

template <int P>
__global__ void __launch_bounds__(256) build_ve_kernel(const double *__restrict__ vfull, VdGeom G,
                                                       double *__restrict__ out64,
                                                       float *__restrict__ out32) {
  constexpr int Q = P + 1, NG = 2 * P, NE = Q * Q * Q;
  extern __shared__ __align__(16) double bsm[];
  double *ve = bsm;                          // [z][y][x]
  double *t1 = ve + Q * Q * Q;               // [z][y][gx]
  double *t2 = t1 + Q * Q * NG;              // [z][gy][gx]
  double *wv = t2 + Q * NG * NG;             // [gz][gy][gx]
  double *u1 = wv + NG * NG * NG;            // [gz][gy][ax][bx]
  double *u2 = u1 + NG * NG * Q * Q;         // [gz][ay][by][ax][bx]
  const int tid = threadIdx.x;
  const int cell = blockIdx.x;
  const int cx = cell % G.nc[0], cy = (cell / G.nc[0]) % G.nc[1],
            cz = cell / (G.nc[0] * G.nc[1]);
  const int Nx = G.n[0] + 2, Ny = G.n[1] + 2;
  for (int i = tid; i < NE; i += 256) {
    const int lx = i % Q, ly = (i / Q) % Q, lz = i / (Q * Q);
    ve[i] = vfull[(cx * P + lx) + (long long)Nx * ((cy * P + ly) + (long long)Ny * (cz * P + lz))];
  }
  __syncthreads();
  // v at the Gauss points (x, then y, then z), times the weights
  for (int i = tid; i < Q * Q * NG; i += 256) {
    const int g = i % NG, yz = i / NG;
    double s = 0.0;
    for (int x = 0; x < Q; ++x) s += G.phi[g * Q + x] * ve[yz * Q + x];
    t1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < Q * NG * NG; i += 256) {
    const int gx = i % NG, gy = (i / NG) % NG, z = i / (NG * NG);
    double s = 0.0;
    for (int y = 0; y < Q; ++y) s += G.phi[gy * Q + y] * t1[(z * Q + y) * NG + gx];
    t2[i] = s;
  }
  __syncthreads();
  const double W = G.cellB[0][cx] * G.cellB[1][cy] * G.cellB[2][cz];
  for (int i = tid; i < NG * NG * NG; i += 256) {
    const int gx = i % NG, gy = (i / NG) % NG, gz = i / (NG * NG);
    double s = 0.0;
    for (int z = 0; z < Q; ++z) s += G.phi[gz * Q + z] * t2[(z * NG + gy) * NG + gx];
    wv[i] = W * G.wg[gx] * G.wg[gy] * G.wg[gz] * s;
  }
  __syncthreads();
  // V_e = sum_g wv psi_x psi_y psi_z, one axis at a time
  for (int i = tid; i < NG * NG * Q * Q; i += 256) {
    const int bx = i % Q, ax = (i / Q) % Q, gg = i / (Q * Q);    // gg = gz * NG + gy
    double s = 0.0;
    for (int g = 0; g < NG; ++g) s += G.phi[g * Q + ax] * G.phi[g * Q + bx] * wv[gg * NG + g];
    u1[i] = s;
  }
  __syncthreads();
  for (int i = tid; i < NG * Q * Q * Q * Q; i += 256) {
    const int xx = i % (Q * Q), by = (i / (Q * Q)) % Q, ay = (i / (Q * Q * Q)) % Q,
              gz = i / (Q * Q * Q * Q);
    double s = 0.0;
    for (int g = 0; g < NG; ++g)
      s += G.phi[g * Q + ay] * G.phi[g * Q + by] * u1[(gz * NG + g) * Q * Q + xx];
    u2[i] = s;
  }
  __syncthreads();
  const long long base = (long long)cell * (out32 ? 128 * 128 : NE * NE);
  if (out32) {
    // the whole 128 x 128 tile, zeros outside the (p+1)^3 block
    for (int i = tid; i < 128 * 128; i += 256) {
      const int a = i / 128, b = i % 128;
      float val = 0.f;
      if (a < NE && b < NE) {
        const int ax = a % Q, ay = (a / Q) % Q, az = a / (Q * Q);
        const int bx = b % Q, by = (b / Q) % Q, bz = b / (Q * Q);
        double s = 0.0;
        for (int g = 0; g < NG; ++g)
          s += G.phi[g * Q + az] * G.phi[g * Q + bz] *
               u2[(((g * Q + ay) * Q + by) * Q + ax) * Q + bx];
        val = (float)s;
      }
      out32[base + umma_index(a, b)] = val;
    }
  } else {
    for (int i = tid; i < NE * NE; i += 256) {
      const int a = i / NE, b = i % NE;
      const int ax = a % Q, ay = (a / Q) % Q, az = a / (Q * Q);
      const int bx = b % Q, by = (b / Q) % Q, bz = b / (Q * Q);
      double s = 0.0;
      for (int g = 0; g < NG; ++g)
        s += G.phi[g * Q + az] * G.phi[g * Q + bz] * u2[(((g * Q + ay) * Q + by) * Q + ax) * Q + bx];
      out64[base + i] = s;
    }
  }
}

// Z += alpha D (V_e (D X)_e) scattered over the cell's unknown nodes.  One CTA
// per (cell, chunk of C columns); the cell matrix and the gathered block are
// staged in shared memory.  V_e in FP64 (row-major) or FP32 (tensor-core tile
// layout).
template <typename T, int P, int C>
__global__ void __launch_bounds__(256) vdense_apply_kernel(const T *__restrict__ X, T *__restrict__ Z,
                                                           int ncol, VdGeom G, double alpha,
                                                           const double *__restrict__ Ve64,
                                                           const float *__restrict__ Ve32) {
  constexpr int Q = P + 1, NE = Q * Q * Q, RG = 256 / C;
  extern __shared__ __align__(16) unsigned char vd_sm[];
  T *sv = reinterpret_cast<T *>(vd_sm);           // [NE][NE]
  T *sx = sv + NE * NE;                           // [NE][C]
  __shared__ double dl[3][Q];
  __shared__ int gidx[3][Q];
  const int tid = threadIdx.x;
  const int cell = blockIdx.x, c0 = blockIdx.y * C;
  const int cx = cell % G.nc[0], cy = (cell / G.nc[0]) % G.nc[1],
            cz = cell / (G.nc[0] * G.nc[1]);
  if (tid < 3 * Q) {
    const int d = tid / Q, l = tid % Q;
    const int gi = (d == 0 ? cx : (d == 1 ? cy : cz)) * P + l;
    dl[d][l] = G.dnode[d][gi];
    gidx[d][l] = (gi >= 1 && gi <= G.n[d]) ? gi - 1 : -1;
  }
  for (int i = tid; i < NE * NE; i += 256) {
    const int a = i / NE, b = i % NE;
    sv[i] = Ve64 ? (T)Ve64[(long long)cell * NE * NE + i]
                 : (T)Ve32[(long long)cell * 128 * 128 + umma_index(a, b)];
  }
  __syncthreads();
  for (int i = tid; i < NE * C; i += 256) {
    const int b = i / C, j = i % C;
    const int lx = b % Q, ly = (b / Q) % Q, lz = b / (Q * Q);
    const int ix = gidx[0][lx], iy = gidx[1][ly], iz = gidx[2][lz];
    T val = (T)0;
    if (ix >= 0 && iy >= 0 && iz >= 0 && c0 + j < ncol) {
      const long long node = ix + (long long)G.n[0] * (iy + (long long)G.n[1] * iz);
      val = (T)(dl[0][lx] * dl[1][ly] * dl[2][lz]) * X[node * ncol + c0 + j];
    }
    sx[i] = val;
  }
  __syncthreads();
  const int j = tid % C;
  for (int a = tid / C; a < NE; a += RG) {
    T s = (T)0;
    for (int b = 0; b < NE; ++b) s += sv[a * NE + b] * sx[b * C + j];
    const int lx = a % Q, ly = (a / Q) % Q, lz = a / (Q * Q);
    const int ix = gidx[0][lx], iy = gidx[1][ly], iz = gidx[2][lz];
    if (ix >= 0 && iy >= 0 && iz >= 0 && c0 + j < ncol) {
      const long long node = ix + (long long)G.n[0] * (iy + (long long)G.n[1] * iz);
      atomicAdd(Z + node * ncol + c0 + j, (T)(alpha * dl[0][lx] * dl[1][ly] * dl[2][lz]) * s);
    }
  }
}

bool vd_geom(const Ctx *c, VdGeom *G) {
  const int p = c->g.p;
  if (!(p == 2 || p == 4)) return false;
  std::vector<double> xg, wg, phi;
  gauss_lagrange(p, 2 * p, &xg, &wg, &phi);
  for (int a = 0; a < 3; ++a) {
    G->nc[a] = c->g.nc[a];
    G->n[a] = c->g.n[a];
    G->cellB[a] = c->g.cellB[a];
    G->dnode[a] = c->g.dnode[a];
  }
  for (size_t i = 0; i < phi.size(); ++i) G->phi[i] = phi[i];
  for (size_t i = 0; i < wg.size(); ++i) G->wg[i] = wg[i];
  return true;
}

template <typename T, int P, int C>
cudaError_t run_vdense(const VdGeom &G, const T *X, T *Z, int ncol, double alpha, const double *V64,
                       const float *V32, cudaStream_t s) {
  constexpr int NE = (P + 1) * (P + 1) * (P + 1);
  const size_t smem = (size_t)(NE * NE + NE * C) * sizeof(T);
  auto k = vdense_apply_kernel<T, P, C>;
  cudaError_t e = raise_smem_limit(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(G.nc[0] * G.nc[1] * G.nc[2], (ncol + C - 1) / C);
  ::invdft::count_launch();
  k<<<grid, 256, smem, s>>>(X, Z, ncol, G, alpha, V64, V32);
  return cudaGetLastError();
}

}  // namespace
}  // namespace invdft

using namespace invdft;

extern "C" invdft_status invdft_cell_potential_bytes(invdft_handle h, invdft_precision prec,
                                                     size_t *bytes) {
  if (!h || !bytes || !(h->g.p == 2 || h->g.p == 4)) {
    if (h) h->err = "cell_potential_bytes: orders 2 and 4 only";
    return INVDFT_EINVAL;
  }
  const long long cells = (long long)h->g.nc[0] * h->g.nc[1] * h->g.nc[2];
  const long long ne = (long long)h->g.q * h->g.q * h->g.q;
  *bytes = prec == INVDFT_FP64 ? (size_t)(cells * ne * ne * 8) : (size_t)(cells * 128 * 128 * 4);
  return INVDFT_OK;
}

extern "C" invdft_status invdft_cell_potentials(invdft_handle h, const double *v_full, void *Ve,
                                                invdft_precision prec, void *stream) {
  VdGeom G;
  if (!h || !v_full || !Ve || !h->bound || !vd_geom(h, &G)) {
    if (h) h->err = "cell_potentials: bound handle of order 2 or 4 and device arrays needed";
    return INVDFT_EINVAL;
  }
  const int cells = h->g.nc[0] * h->g.nc[1] * h->g.nc[2];
  double *o64 = prec == INVDFT_FP64 ? (double *)Ve : nullptr;
  float *o32 = prec == INVDFT_FP64 ? nullptr : (float *)Ve;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->g.p == 2) {
    const size_t smem = BuildSmem<2>::doubles * sizeof(double);
    INV_CUDA(h, raise_smem_limit(build_ve_kernel<2>, smem));
    ::invdft::count_launch();
    build_ve_kernel<2><<<cells, 256, smem, s>>>(v_full, G, o64, o32);
  } else {
    const size_t smem = BuildSmem<4>::doubles * sizeof(double);
    INV_CUDA(h, raise_smem_limit(build_ve_kernel<4>, smem));
    ::invdft::count_launch();
    build_ve_kernel<4><<<cells, 256, smem, s>>>(v_full, G, o64, o32);
  }
  INV_LAUNCH(h, "build_ve_kernel");
  return INVDFT_OK;
}

extern "C" invdft_status invdft_apply_h_dense(invdft_handle h, const void *Ve, const void *X,
                                              void *Y, int ncol, invdft_precision prec,
                                              void *stream) {
  VdGeom G;
  if (!h || !Ve || !X || !Y || X == Y || ncol < 1 || ncol > kMaxCols || !h->bound ||
      !vd_geom(h, &G)) {
    if (h) h->err = "apply_h_dense: bad arguments (bound order-2/4 handle, ncol in [1, 256], Y != X)";
    return INVDFT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  // kinetic part with the collocated potential switched off, then + D V D X
  if (prec == INVDFT_FP64) {
    HxArgs<double> a;
    a.X = (const double *)X;
    a.Z = (double *)Y;
    a.ncol = ncol;
    e = hx_op_nopot(h, a, s);
    if (e == cudaSuccess) {
      if (h->g.p == 2)
        e = run_vdense<double, 2, 8>(G, (const double *)X, (double *)Y, ncol, 1.0,
                                     (const double *)Ve, nullptr, s);
      else
        e = run_vdense<double, 4, 8>(G, (const double *)X, (double *)Y, ncol, 1.0,
                                     (const double *)Ve, nullptr, s);
    }
  } else {
    HxArgs<float> a;
    a.X = (const float *)X;
    a.Z = (float *)Y;
    a.ncol = ncol;
    a.tc = false;
    e = hx_op_nopot(h, a, s);
    if (e == cudaSuccess) {
      if (h->g.p == 2)
        e = run_vdense<float, 2, 32>(G, (const float *)X, (float *)Y, ncol, 1.0, nullptr,
                                     (const float *)Ve, s);
      else
        e = run_vdense<float, 4, 32>(G, (const float *)X, (float *)Y, ncol, 1.0, nullptr,
                                     (const float *)Ve, s);
    }
  }
  if (!cuda_ok(h, e, "apply_h_dense")) return INVDFT_ECUDA;
  return INVDFT_OK;
}
