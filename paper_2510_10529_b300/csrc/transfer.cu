// Linear (Q1) v_xc mesh and the field transfer to and from the orbital mesh
// (Sec. 3.1.1, Sec. 3.2.2).  The Q1 mesh is a uniform mesh of nv cells per axis
// over the orbital mesh's box (equal or graded orbital cells), with v_xc on all of its (nv+1)^3 nodes (x
// fastest).  The transfer matrix T holds the trilinear weights of the Q1
// interpolant at the orbital mesh's unknown nodes (8 per node):
//   v_nodes = T v_q1                 (v_xc seen by the orbitals),
//   g_q1    = T^T g_nodes            (the nodal gradient of Eq. 22 pulled back
//                                     to the Q1 coefficients).
// T factorises by axis: T[a][b] = w(x_a, X_b) w(y_a, Y_b) w(z_a, Z_b) with the
// 1D hat function w(x, X) = max(0, 1 - |x - X| / h_v).  The first map is a
// gather of 8 values per node; the second is computed by its owner, each Q1
// node summing over the orbital nodes inside its support in a fixed order, so
// it is deterministic and needs no atomics.
#include <cmath>

#include "internal.h"

namespace invdft {
namespace {

struct AxisGeom {
  const double *x;         // orbital node coordinates along the axis, boundary included
  int nnodes;              // n + 2
};
struct TransferGeom {
  AxisGeom ax[3];
  int n[3];                // orbital unknowns per axis
  int nv;                  // Q1 cells per axis
  double vlo[3], hv[3];    // Q1 box start and cell size per axis
};

// coordinate of orbital node g (0 .. n + 1, the boundary included)
__device__ __forceinline__ double node_x(const AxisGeom &A, int g) { return A.x[g]; }

__global__ void q1_to_nodes_kernel(TransferGeom G, const double *__restrict__ vq,
                                   double *__restrict__ out) {
  const long long L = (long long)G.n[0] * G.n[1] * G.n[2];
  const int Nv = G.nv + 1;
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < L;
       a += (long long)gridDim.x * blockDim.x) {
    const int u[3] = {(int)(a % G.n[0]), (int)((a / G.n[0]) % G.n[1]),
                      (int)(a / ((long long)G.n[0] * G.n[1]))};
    int c[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
      const double t = (node_x(G.ax[d], u[d] + 1) - G.vlo[d]) / G.hv[d];
      int ci = (int)floor(t);
      ci = ci < 0 ? 0 : (ci > G.nv - 1 ? G.nv - 1 : ci);
      c[d] = ci;
      f[d] = t - ci;
    }
    double s = 0.0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                           (dz ? f[2] : 1.0 - f[2]);
          s += w * vq[(c[0] + dx) + (long long)Nv * ((c[1] + dy) + (long long)Nv * (c[2] + dz))];
        }
    out[a] = s;
  }
}

// orbital unknowns (0-based) whose coordinate lies within one Q1 cell of X:
// [*first, *last]; the hat weight is zero outside.  The node coordinates
// increase, so the first node right of X - hv is found by bisection.
__device__ __forceinline__ void support(const AxisGeom &A, int n, double X, double hv, int *first,
                                        int *last) {
  int lo = 0, hi = n + 1;               // x[lo] <= X - hv < x[hi] unless at the ends
  if (node_x(A, 0) > X - hv) hi = 0;
  while (hi - lo > 1) {
    const int mid = (lo + hi) / 2;
    if (node_x(A, mid) <= X - hv) lo = mid;
    else hi = mid;
  }
  int g = hi;
  int g1 = g;
  while (g1 + 1 <= n && node_x(A, g1 + 1) < X + hv) ++g1;
  *first = (g < 1 ? 1 : g) - 1;
  *last = (g1 > n ? n : g1) - 1;
}

__global__ void nodes_to_q1_kernel(TransferGeom G, const double *__restrict__ g,
                                   double *__restrict__ out) {
  const int Nv = G.nv + 1;
  const long long NQ = (long long)Nv * Nv * Nv;
  for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < NQ;
       b += (long long)gridDim.x * blockDim.x) {
    const int bi[3] = {(int)(b % Nv), (int)((b / Nv) % Nv), (int)(b / ((long long)Nv * Nv))};
    int lo[3], hi[3];
    double X[3];
    for (int d = 0; d < 3; ++d) {
      X[d] = G.vlo[d] + bi[d] * G.hv[d];
      support(G.ax[d], G.n[d], X[d], G.hv[d], &lo[d], &hi[d]);
    }
    double s = 0.0;
    for (int uz = lo[2]; uz <= hi[2]; ++uz) {
      const double wz = fmax(0.0, 1.0 - fabs(node_x(G.ax[2], uz + 1) - X[2]) / G.hv[2]);
      double sy = 0.0;
      for (int uy = lo[1]; uy <= hi[1]; ++uy) {
        const double wy = fmax(0.0, 1.0 - fabs(node_x(G.ax[1], uy + 1) - X[1]) / G.hv[1]);
        const double *row = g + (long long)G.n[0] * (uy + (long long)G.n[1] * uz);
        double sx = 0.0;
        for (int ux = lo[0]; ux <= hi[0]; ++ux) {
          const double wx = fmax(0.0, 1.0 - fabs(node_x(G.ax[0], ux + 1) - X[0]) / G.hv[0]);
          sx += wx * row[ux];
        }
        sy += wy * sx;
      }
      s += wz * sy;
    }
    out[b] = s;
  }
}

bool make_geom(invdft_handle h, int nv, TransferGeom *G) {
  if (nv < 1 || nv > 4096) return false;
  if (!h->bound) return false;
  for (int d = 0; d < 3; ++d) {
    G->ax[d].x = h->g.axis[d];
    G->ax[d].nnodes = h->g.n[d] + 2;
    G->n[d] = h->g.n[d];
    G->vlo[d] = h->mesh.lo[d];
    G->hv[d] = (h->mesh.hi[d] - h->mesh.lo[d]) / nv;
  }
  G->nv = nv;
  return true;
}

}  // namespace
}  // namespace invdft

using namespace invdft;

extern "C" invdft_status invdft_q1_to_nodes(invdft_handle h, int nv, const double *v_q1,
                                            double *v_nodes, void *stream) {
  TransferGeom G;
  if (!h || !v_q1 || !v_nodes || !make_geom(h, nv, &G)) {
    if (h) h->err = "q1_to_nodes: bad arguments (bound handle, nv in [1, 4096], device arrays)";
    return INVDFT_EINVAL;
  }
  const long long L = h->L;
  const int grid = (int)std::min<long long>((L + 255) / 256, 148LL * 16);
  ::invdft::count_launch();
  q1_to_nodes_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(G, v_q1, v_nodes);
  INV_LAUNCH(h, "q1_to_nodes_kernel");
  return INVDFT_OK;
}

extern "C" invdft_status invdft_grad_to_q1(invdft_handle h, int nv, const double *g_nodes,
                                           double *g_q1, void *stream) {
  TransferGeom G;
  if (!h || !g_nodes || !g_q1 || !make_geom(h, nv, &G)) {
    if (h) h->err = "grad_to_q1: bad arguments (bound handle, nv in [1, 4096], device arrays)";
    return INVDFT_EINVAL;
  }
  const long long NQ = (long long)(nv + 1) * (nv + 1) * (nv + 1);
  const int grid = (int)std::min<long long>((NQ + 127) / 128, 148LL * 16);
  ::invdft::count_launch();
  nodes_to_q1_kernel<<<grid, 128, 0, (cudaStream_t)stream>>>(G, g_nodes, g_q1);
  INV_LAUNCH(h, "nodes_to_q1_kernel");
  return INVDFT_OK;
}
