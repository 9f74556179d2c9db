// Initial guess of the exchange-correlation potential (Sec. 4.2.3, Eq. 25-26)
// on the device, at the unknown nodes:
//   v_init = f v0[rho] + (1 - f) alpha v_FA,   f = rho / (rho + tau),
//   v_FA   = -v_H / N_e (Fermi-Amaldi, v_H of the target density given),
//   v0     = v_x + v_c,  v_c the PW92 correlation potential of the
//            spin-unpolarised uniform gas, v_x the Slater exchange potential or
//            the LB94 exchange potential (closed shell, per-spin density rho/2,
//            needing |grad rho|).
// The density gradient is that of the finite-element interpolant at the GLL
// nodes: along each axis the derivative of the cell's degree-p polynomial
// through the node's line, and at a cell vertex the mean of the two cells'
// one-sided derivatives (the mean over all cells sharing the node reduces to
// this, since the other directions do not change the line).  rho is zero on
// the Dirichlet boundary.
#include <cmath>

#include "internal.h"

namespace invdft {
namespace {

// PW92 parameters of the spin-unpolarised correlation energy (Perdew and
// Wang 1992, Table I, p = 1)
constexpr double kA = 0.031091, kA1 = 0.21370;
constexpr double kB1 = 7.5957, kB2 = 3.5876, kB3 = 1.6382, kB4 = 0.49294;
constexpr double kLb94Beta = 0.05;

struct GuessGeom {
  int n[3];          // unknowns per axis (x, y, z)
  int p;
  const double *cellA[3];    // 2 / h_e per cell and axis (reference derivative to physical)
  double D[kMaxQ * kMaxQ];   // D[i][j] = l_j'(x_i) on [-1, 1]
};

// derivative along one axis at unknown index u (0-based) of the line values
// fetched by `at(g)` with g the node index including the boundary (at(0) =
// at(n+1) = 0 is the Dirichlet boundary)
template <typename F>
__device__ __forceinline__ double axis_derivative(const GuessGeom &G, int axis, int u, F at) {
  const int p = G.p, g = u + 1, q = p + 1;
  const int e = g / p, l = g - e * p;       // cell starting at node e p, local index l
  if (l != 0) {
    double s = 0.0;
    for (int j = 0; j < q; ++j) s += G.D[l * q + j] * at(e * p + j);
    return s * G.cellA[axis][e];
  }
  // a cell vertex (never the boundary: 1 <= g <= n): mean of the left cell's
  // derivative at its local node p and the right cell's at its local node 0
  double sl = 0.0, sr = 0.0;
  for (int j = 0; j < q; ++j) {
    sl += G.D[p * q + j] * at((e - 1) * p + j);
    sr += G.D[j] * at(e * p + j);
  }
  return 0.5 * (sl * G.cellA[axis][e - 1] + sr * G.cellA[axis][e]);
}

__global__ void gradnorm_kernel(const double *__restrict__ rho, GuessGeom G, double *__restrict__ gn) {
  const long long L = (long long)G.n[0] * G.n[1] * G.n[2];
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < L;
       a += (long long)gridDim.x * blockDim.x) {
    const int ux = (int)(a % G.n[0]);
    const int uy = (int)((a / G.n[0]) % G.n[1]);
    const int uz = (int)(a / ((long long)G.n[0] * G.n[1]));
    auto val = [&](int x, int y, int z) -> double {   // node indices incl. boundary
      if (x < 1 || y < 1 || z < 1 || x > G.n[0] || y > G.n[1] || z > G.n[2]) return 0.0;
      const double r = rho[(x - 1) + (long long)G.n[0] * ((y - 1) + (long long)G.n[1] * (z - 1))];
      return r > 0.0 ? r : 0.0;
    };
    const double gx = axis_derivative(G, 0, ux, [&](int g) { return val(g, uy + 1, uz + 1); });
    const double gy = axis_derivative(G, 1, uy, [&](int g) { return val(ux + 1, g, uz + 1); });
    const double gz = axis_derivative(G, 2, uz, [&](int g) { return val(ux + 1, uy + 1, g); });
    gn[a] = sqrt(gx * gx + gy * gy + gz * gz);
  }
}

// PW92 v_c = eps_c - (r_s / 3) d eps_c / d r_s (0 where rho <= 0)
__device__ __forceinline__ double pw92_vc(double rho) {
  if (!(rho > 0.0)) return 0.0;
  const double rs = cbrt(3.0 / (4.0 * M_PI * rho));
  const double srs = sqrt(rs);
  const double q0 = -2.0 * kA * (1.0 + kA1 * rs);
  const double q1 = 2.0 * kA * (kB1 * srs + kB2 * rs + kB3 * rs * srs + kB4 * rs * rs);
  const double dq1 = kA * (kB1 / srs + 2.0 * kB2 + 3.0 * kB3 * srs + 4.0 * kB4 * rs);
  const double lg = log1p(1.0 / q1);
  const double eps = q0 * lg;
  const double deps = -2.0 * kA * kA1 * lg - q0 * dq1 / (q1 * q1 + q1);
  return eps - rs / 3.0 * deps;
}

__global__ void guess_kernel(const double *__restrict__ rho_d, const double *__restrict__ v_H,
                             const double *__restrict__ gn, long long L, double n_elec,
                             double tau, double alpha, int lb94, double *__restrict__ v) {
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < L;
       a += (long long)gridDim.x * blockDim.x) {
    const double rho = rho_d[a] > 0.0 ? rho_d[a] : 0.0;
    double vx = -cbrt(3.0 * rho / M_PI);                    // Slater exchange
    if (lb94 && rho > 0.0) {
      const double rs = 0.5 * rho;                          // per-spin density
      const double x = 0.5 * gn[a] / pow(rs, 4.0 / 3.0);
      vx -= kLb94Beta * cbrt(rs) * x * x / (1.0 + 3.0 * kLb94Beta * x * asinh(x));
    }
    const double v0 = vx + pw92_vc(rho);
    const double vfa = -v_H[a] / n_elec;
    const double f = rho / (rho + tau);
    v[a] = f * v0 + (1.0 - f) * alpha * vfa;
  }
}

}  // namespace
}  // namespace invdft

using namespace invdft;

extern "C" invdft_status invdft_initial_guess(invdft_handle h, const double *rho_data,
                                              const double *v_H, double tau, double alpha,
                                              int exchange, double *v_out, void *stream) {
  if (!h || !rho_data || !v_H || !v_out || !(tau > 0.0) || (exchange != 0 && exchange != 1)) {
    if (h) h->err = "initial_guess: bad arguments (tau > 0, exchange 0 = Slater or 1 = LB94)";
    return INVDFT_EINVAL;
  }
  if (!h->bound) {
    h->err = "initial_guess: bind a workspace first";
    return INVDFT_EINVAL;
  }
  if (!(h->o.n_electrons > 0.0)) {
    h->err = "initial_guess: the options need n_electrons > 0 (Fermi-Amaldi term)";
    return INVDFT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long long L = h->L;
  const int grid = (int)std::min<long long>((L + 255) / 256, 148LL * 16);
  double *gn = h->grad_new;          // |grad rho| scratch ([L], free outside a step)
  if (exchange == 1) {
    GuessGeom G;
    G.p = h->g.p;
    for (int ax = 0; ax < 3; ++ax) {
      G.n[ax] = h->g.n[ax];
      G.cellA[ax] = h->g.cellA[ax];
    }
    const int q = h->g.p + 1;
    for (int i = 0; i < q * q; ++i) G.D[i] = h->tab.Dm[i];
    ::invdft::count_launch();
    gradnorm_kernel<<<grid, 256, 0, s>>>(rho_data, G, gn);
    INV_LAUNCH(h, "gradnorm_kernel");
  }
  ::invdft::count_launch();
  guess_kernel<<<grid, 256, 0, s>>>(rho_data, v_H, gn, L, h->o.n_electrons, tau, alpha, exchange,
                                    v_out);
  INV_LAUNCH(h, "guess_kernel");
  return INVDFT_OK;
}
