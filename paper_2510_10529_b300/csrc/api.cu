// C-ABI entry points of libinvdft (declared in include/invdft.h): handle
// life cycle, workspace binding, tables, potential, and the operator calls.
// The solver entry points (forward, adjoint, loss/gradient, step) live in
// solvers.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>

#include "internal.h"
#include "solvers.h"

using namespace invdft;

namespace invdft {

cudaError_t raise_smem_limit(const void *func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void *>, size_t> limit;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t &cur = limit[{dev, func}];
  if (bytes <= cur) return cudaSuccess;
  // the first time, raise the limit to the device's opt-in maximum, so that
  // it never has to change later (a change while a stream is being captured
  // into a CUDA graph would invalidate the capture)
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  size_t target = std::max(bytes, (size_t)optin);
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)target);
  if (e != cudaSuccess && target != bytes) {
    cudaGetLastError();
    target = bytes;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)target);
  }
  if (e == cudaSuccess) cur = target;
  return e;
}

static thread_local std::string g_create_error;
static std::atomic<unsigned long long> g_launches{0};

static thread_local unsigned long long t_launches = 0;   // launches issued by this thread
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void count_launches(long long n) {
  g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed);
  t_launches += (unsigned long long)n;
}
unsigned long long thread_launches() { return t_launches; }
static std::atomic<long long> g_graph_stats[3];            // captures, replays, refused captures
void count_graph(int what) { g_graph_stats[what].fetch_add(1, std::memory_order_relaxed); }
void set_global_error(const char *msg) { g_create_error = msg; }

bool cuda_ok(Ctx *c, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return true;
  char buf[512];
  std::snprintf(buf, sizeof(buf), "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  if (c) c->err = buf;
  return false;
}

namespace {

struct AxisTabs {
  const double *m1[3], *kA[3], *kB[3];
  int n[3];
};

__global__ void init_fields(AxisTabs t, double *__restrict__ mass, double *__restrict__ dvec,
                            double *__restrict__ prec, float *__restrict__ precf) {
  const long long L = (long long)t.n[0] * t.n[1] * t.n[2];
  for (long long a = blockIdx.x * (long long)blockDim.x + threadIdx.x; a < L;
       a += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(a % t.n[0]) + 1, iy = (int)((a / t.n[0]) % t.n[1]) + 1;
    const int iz = (int)(a / ((long long)t.n[0] * t.n[1])) + 1;
    const double m = t.m1[0][ix] * t.m1[1][iy] * t.m1[2][iz];
    const double kaa = 0.5 * (t.kB[2][iz] * t.kB[1][iy] * t.kA[0][ix] +
                              t.kB[2][iz] * t.kA[1][iy] * t.kB[0][ix] +
                              t.kA[2][iz] * t.kB[1][iy] * t.kB[0][ix]);
    mass[a] = m;
    dvec[a] = 1.0 / sqrt(m);
    prec[a] = m / kaa;          // inverse diagonal of D K D (Laplacian part)
    precf[a] = (float)(m / kaa);
  }
}

__global__ void add_fields(const double *__restrict__ a, const double *__restrict__ b,
                           double *__restrict__ out, float *__restrict__ outf, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double x = a[i] + (b ? b[i] : 0.0);
    out[i] = x;
    outf[i] = (float)x;
  }
}

int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 148LL * 16); }

// Lay out (or, with base == nullptr, only measure) the workspace.
size_t plan(Ctx *c, char *base) {
  Arena ar;
  ar.base = base;
  const long long L = c->L;
  const int nv = c->nv;
  const size_t blk = (size_t)L * nv;
  for (int a = 0; a < 3; ++a) {
    const int N = c->g.n[a] + 2, nc = c->g.nc[a];
    c->dnode[a] = ar.take<double>(N);
    c->m1tab[a] = ar.take<double>(N);
    c->kAtab[a] = ar.take<double>(N);
    c->kBtab[a] = ar.take<double>(N);
    c->axis[a] = ar.take<double>(N);
    c->cellA[a] = ar.take<double>(nc);
    c->cellB[a] = ar.take<double>(nc);
  }
  c->dm1f = ar.take<float>(c->g.n[0] + 2);
  c->mass = ar.take<double>(L);
  c->dvec = ar.take<double>(L);
  c->prec_diag = ar.take<double>(L);
  c->precf = ar.take<float>(L);
  c->Ke_tc = ar.take<float>(tc_cell_matrix_floats());
  c->cell_perm = ar.take<int>(c->g.cube ? (size_t)c->g.ncell * c->g.ncell * c->g.ncell : 1);
  c->v = ar.take<double>(L);
  c->vf = ar.take<float>(L);
  c->vfixed = ar.take<double>(L);
  c->rho = ar.take<double>(L);
  c->grad = ar.take<double>(L);
  c->grad_new = ar.take<double>(L);
  c->dir = ar.take<double>(L);
  c->vtry = ar.take<double>(L);
  c->v_ub = ar.take<double>(L);
  c->dLdrho = ar.take<double>(L);
  c->X = ar.take<double>(blk);
  c->Y = ar.take<double>(blk);
  c->HY = ar.take<double>(blk);
  c->P = ar.take<double>(blk);
  c->Rg = ar.take<double>(blk);
  // C0 and the MINRES buffers also hold FP32 blocks padded to a multiple of 4
  // columns (at most 2 nv floats per node once nv >= 2)
  const size_t blk2 = (size_t)L * std::max(nv, 2);
  c->C0 = ar.take<double>(blk2);
  c->C1 = ar.take<double>(blk);
  c->C2 = ar.take<double>(blk);
  c->E32 = ar.take<float>(blk);
  for (int k = 0; k < 9; ++k) c->mr[k] = ar.take<double>(blk2);
  const int hist = c->o.lbfgs_history;
  c->Sh = ar.take<double>((size_t)hist * L);
  c->Yh = ar.take<double>((size_t)hist * L);
  c->eps = ar.take<double>(kMaxGram);
  c->occ = ar.take<double>(kMaxGram);
  c->dfde = ar.take<double>(kMaxGram);
  c->small = ar.take<double>(16 * (size_t)kMaxGram * kMaxGram);
  c->partial = ar.take<double>((size_t)kGramBlocks * kMaxGram * kMaxGram);
  c->scal = ar.take<double>(1024 * (size_t)kMaxCols);
  c->status = ar.take<int>(16);
  return ar.off + 256;
}

}  // namespace
}  // namespace invdft

extern "C" {

invdft_status invdft_create_mesh(const invdft_mesh_desc *mesh, const invdft_opts *opts,
                                 invdft_handle *out, long long *n_nodes_out) {
  if (!mesh || !opts || !out) {
    g_create_error = "create_mesh: null argument";
    return INVDFT_EINVAL;
  }
  *out = nullptr;
  if (!(mesh->order == 2 || mesh->order == 4 || mesh->order == 6)) {
    g_create_error = "create_mesh: order must be 2, 4 or 6";
    return INVDFT_EINVAL;
  }
  long long nn[3];
  for (int a = 0; a < 3; ++a) {
    if (mesh->ncell[a] < 1 || !(mesh->hi[a] > mesh->lo[a])) {
      g_create_error = "create_mesh: every axis needs ncell >= 1 and hi > lo";
      return INVDFT_EINVAL;
    }
    nn[a] = (long long)mesh->ncell[a] * mesh->order - 1;
    if (nn[a] < 1 || nn[a] > 4095) {
      g_create_error = "create_mesh: an axis has no unknowns or more than 4095";
      return INVDFT_EINVAL;
    }
    if (mesh->breaks[a]) {
      const double *b = mesh->breaks[a];
      bool ok = b[0] == mesh->lo[a] && b[mesh->ncell[a]] == mesh->hi[a];
      for (int e = 0; e < mesh->ncell[a] && ok; ++e) ok = b[e + 1] > b[e];
      if (!ok) {
        g_create_error = "create_mesh: breaks must increase from lo to hi";
        return INVDFT_EINVAL;
      }
    }
  }
  if (nn[0] * nn[1] * nn[2] * (long long)kMaxCols >= (1LL << 31)) {
    g_create_error = "create_mesh: unknowns * 256 must stay below 2^31";
    return INVDFT_EINVAL;
  }
  if (opts->nstates < 1 || opts->nstates > kMaxDense) {
    g_create_error = "create_mesh: nstates must be in [1, 96]";
    return INVDFT_EINVAL;
  }
  invdft_ctx *c = new (std::nothrow) invdft_ctx();
  if (!c) {
    g_create_error = "create_mesh: out of host memory";
    return INVDFT_ENOMEM;
  }
  c->o = *opts;
  invdft_opts &o = c->o;
  if (o.cheb_degree <= 0) o.cheb_degree = 20;
  if (o.c_eig <= 0) o.c_eig = 1e2;
  if (o.c_ad <= 0) o.c_ad = 1e5;
  if (o.tau_bc <= 0) o.tau_bc = 1e-6;
  if (o.max_cheb_passes <= 0) o.max_cheb_passes = 60;
  if (o.max_minres_iters <= 0) o.max_minres_iters = 2000;
  if (o.lbfgs_history <= 0) o.lbfgs_history = 10;
  if (o.deg_tol <= 0) o.deg_tol = 1e-8;
  if (o.kT < 0) o.kT = 0;
  c->nv = o.nstates;
  build_reference(mesh->order, &c->tab);
  Geom &g = c->g;
  g.p = mesh->order;
  g.q = mesh->order + 1;
  for (int i = 0; i < g.q * g.q; ++i) {
    g.A[i] = c->tab.A[i];
    g.B[i] = c->tab.B[i];
  }
  g.graded = false;
  for (int a = 0; a < 3; ++a) {
    const int nc = mesh->ncell[a];
    std::vector<double> br(nc + 1);
    for (int e = 0; e <= nc; ++e)
      br[e] = mesh->breaks[a] ? mesh->breaks[a][e]
                              : (e == nc ? mesh->hi[a]
                                         : mesh->lo[a] + (mesh->hi[a] - mesh->lo[a]) * e / nc);
    build_axis(c->tab, br, g.p, &c->tab.ax[a]);
    g.nc[a] = nc;
    g.n[a] = (int)nn[a];
    g.graded |= !c->tab.ax[a].uniform;
    const double sh = 0.5 * (mesh->hi[a] - mesh->lo[a]) / nc;
    g.s[a] = sh;
    for (int i = 0; i <= g.p; ++i) {
      const double m = (i == 0 || i == g.p) ? 2.0 * sh * c->tab.gll_w[0] : sh * c->tab.gll_w[i];
      g.dl[a][i] = 1.0 / std::sqrt(m);
    }
  }
  g.cube = !g.graded && g.nc[0] == g.nc[1] && g.nc[1] == g.nc[2] &&
           std::fabs(g.s[0] - g.s[1]) <= 1e-14 * g.s[0] &&
           std::fabs(g.s[1] - g.s[2]) <= 1e-14 * g.s[0];
  g.ncell = g.nc[0];
  g.Ni = g.n[0];
  g.L = nn[0] * nn[1] * nn[2];
  g.kc = 0.5 * g.s[0];
  c->mesh = *mesh;
  for (int a = 0; a < 3; ++a) c->mesh.breaks[a] = nullptr;   // copied into the tables
  c->L = g.L;
  c->ws_bytes = plan(c, nullptr);
  *out = c;
  if (n_nodes_out) *n_nodes_out = c->L;
  return INVDFT_OK;
}

invdft_status invdft_destroy(invdft_handle h) {
  if (!h) return INVDFT_EINVAL;
  if (h->hbuf) cudaFreeHost(h->hbuf);
  for (auto e : h->prof.ev) cudaEventDestroy(e);
  if (h->aux_stream) {
    cudaStreamSynchronize(h->aux_stream);
    cudaStreamDestroy(h->aux_stream);
  }
  if (h->aux_event) cudaEventDestroy(h->aux_event);
  delete h;
  return INVDFT_OK;
}

invdft_status invdft_workspace_size(invdft_handle h, size_t *bytes) {
  if (!h || !bytes) return INVDFT_EINVAL;
  *bytes = h->ws_bytes;
  return INVDFT_OK;
}

invdft_status invdft_bind_workspace(invdft_handle h, void *device_ptr, size_t bytes, void *stream) {
  if (!h) return INVDFT_EINVAL;
  if (!device_ptr || bytes < h->ws_bytes) {
    h->err = "bind_workspace: workspace missing or smaller than invdft_workspace_size";
    return INVDFT_ENOMEM;
  }
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, 0);
  cudaStream_t s = (cudaStream_t)stream;
  char *base = reinterpret_cast<char *>(((uintptr_t)device_ptr + 255) & ~uintptr_t(255));
  if ((size_t)(base - (char *)device_ptr) + h->ws_bytes - 256 > bytes) {
    h->err = "bind_workspace: workspace too small after alignment";
    return INVDFT_ENOMEM;
  }
  plan(h, base);
  if (!h->hbuf) INV_CUDA(h, cudaHostAlloc((void **)&h->hbuf, 16 * kMaxCols * sizeof(double), 0));
  // 1D tables per axis: 1/sqrt(m1) (zero at the Dirichlet ends), m1, assembled
  // diagonals, node coordinates, and the cell scalars 2/h_e and h_e/2
  std::vector<std::vector<double>> host;     // kept alive until the stream sync below
  AxisTabs at;
  for (int a = 0; a < 3; ++a) {
    const AxisTab &t = h->tab.ax[a];
    const int N = h->g.n[a] + 2, nc = h->g.nc[a];
    std::vector<double> dn(N), ca(nc), cb(nc);
    for (int i = 0; i < N; ++i) dn[i] = (i == 0 || i == N - 1) ? 0.0 : 1.0 / std::sqrt(t.m1[i]);
    for (int e = 0; e < nc; ++e) {
      ca[e] = 2.0 / t.h[e];
      cb[e] = 0.5 * t.h[e];
    }
    host.push_back(dn);
    host.push_back(ca);
    host.push_back(cb);
    auto up = [&](double *dst, const std::vector<double> &src) {
      return cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice,
                             s);
    };
    INV_CUDA(h, up(h->dnode[a], host[host.size() - 3]));
    INV_CUDA(h, up(h->cellA[a], host[host.size() - 2]));
    INV_CUDA(h, up(h->cellB[a], host[host.size() - 1]));
    INV_CUDA(h, up(h->m1tab[a], t.m1));
    INV_CUDA(h, up(h->kAtab[a], t.kdiag1_A));
    INV_CUDA(h, up(h->kBtab[a], t.kdiag1_B));
    INV_CUDA(h, up(h->axis[a], t.axis));
    at.m1[a] = h->m1tab[a];
    at.kA[a] = h->kAtab[a];
    at.kB[a] = h->kBtab[a];
    at.n[a] = h->g.n[a];
    h->g.dnode[a] = h->dnode[a];
    h->g.m1node[a] = h->m1tab[a];
    h->g.cellA[a] = h->cellA[a];
    h->g.cellB[a] = h->cellB[a];
    h->g.axis[a] = h->axis[a];
  }
  std::vector<float> dm1f(host[0].begin(), host[0].end());
  INV_CUDA(h, cudaMemcpyAsync(h->dm1f, dm1f.data(), dm1f.size() * sizeof(float),
                              cudaMemcpyHostToDevice, s));
  ::invdft::count_launch();
  init_fields<<<grid_for(h->L), 256, 0, s>>>(at, h->mass, h->dvec, h->prec_diag, h->precf);
  INV_LAUNCH(h, "init_fields");
  std::vector<float> ke;
  std::vector<int> perm;
  if (h->g.p == 4 && h->g.cube) {
    build_tc_cell_matrix(h->g, &ke);
    INV_CUDA(h, cudaMemcpyAsync(h->Ke_tc, ke.data(), ke.size() * sizeof(float),
                                cudaMemcpyHostToDevice, s));
    build_cell_order(h->g.ncell, &perm);
    INV_CUDA(h, cudaMemcpyAsync(h->cell_perm, perm.data(), perm.size() * sizeof(int),
                                cudaMemcpyHostToDevice, s));
  } else {
    h->Ke_tc = nullptr;
    h->cell_perm = nullptr;
  }
  INV_CUDA(h, cudaMemsetAsync(h->status, 0, 16 * sizeof(int), s));
  INV_CUDA(h, cudaMemsetAsync(h->v, 0, h->L * sizeof(double), s));
  INV_CUDA(h, cudaMemsetAsync(h->vf, 0, h->L * sizeof(float), s));
  INV_CUDA(h, cudaMemsetAsync(h->vfixed, 0, h->L * sizeof(double), s));
  INV_CUDA(h, cudaStreamSynchronize(s));   // host tables above are freed on return
  h->g.dm1 = h->dnode[0];
  h->g.dm1f = h->dm1f;
  h->bound = true;
  h->have_potential = false;
  h->have_orbitals = false;
  h->have_forward = false;
  h->have_grad = false;
  h->have_upper = false;
  h->have_ub_base = false;
  h->hist_n = h->hist_head = 0;
  return INVDFT_OK;
}

invdft_status invdft_node_coords(invdft_handle h, double *xyz) {
  if (!h || !xyz) return INVDFT_EINVAL;
  const std::vector<double> &axx = h->tab.ax[0].axis, &axy = h->tab.ax[1].axis,
                            &axz = h->tab.ax[2].axis;
  long long a = 0;
  for (int iz = 1; iz <= h->g.n[2]; ++iz)
    for (int iy = 1; iy <= h->g.n[1]; ++iy)
      for (int ix = 1; ix <= h->g.n[0]; ++ix, ++a) {
        xyz[3 * a + 0] = axx[ix];
        xyz[3 * a + 1] = axy[iy];
        xyz[3 * a + 2] = axz[iz];
      }
  return INVDFT_OK;
}

invdft_status invdft_mass_diag(invdft_handle h, double *m_dev, void *stream) {
  if (!h || !m_dev) return INVDFT_EINVAL;
  if (!h->bound) {
    h->err = "mass_diag: bind a workspace first";
    return INVDFT_ENOMEM;
  }
  INV_CUDA(h, cudaMemcpyAsync(m_dev, h->mass, h->L * sizeof(double), cudaMemcpyDeviceToDevice,
                              (cudaStream_t)stream));
  return INVDFT_OK;
}

invdft_status invdft_set_potential(invdft_handle h, const double *v_fixed, const double *v_xc,
                                   void *stream) {
  if (!h || !v_fixed) return INVDFT_EINVAL;
  if (!h->bound) {
    h->err = "set_potential: bind a workspace first";
    return INVDFT_ENOMEM;
  }
  cudaStream_t s = (cudaStream_t)stream;
  INV_CUDA(h, cudaMemcpyAsync(h->vfixed, v_fixed, h->L * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ::invdft::count_launch();
  add_fields<<<grid_for(h->L), 256, 0, s>>>(v_fixed, v_xc, h->v, h->vf, h->L);
  INV_LAUNCH(h, "add_fields");
  h->have_potential = true;
  h->have_forward = false;
  h->have_grad = false;
  h->have_upper = false;
  return INVDFT_OK;
}

invdft_status invdft_apply_h(invdft_handle h, const void *X, void *Y, int ncol,
                             invdft_precision prec, void *stream) {
  if (!h || !X || !Y || ncol < 1 || ncol > kMaxCols || X == Y) {
    if (h) h->err = "apply_h: bad arguments (ncol in [1,256], X != Y)";
    return INVDFT_EINVAL;
  }
  if (!h->bound || !h->have_potential) {
    h->err = "apply_h: bind a workspace and set a potential first";
    return INVDFT_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  if (prec == INVDFT_FP64) {
    HxArgs<double> a;
    a.X = (const double *)X;
    a.Z = (double *)Y;
    a.ncol = ncol;
    e = hx_op(h, a, s);
  } else {
    HxArgs<float> a;
    a.X = (const float *)X;
    a.Z = (float *)Y;
    a.ncol = ncol;
    a.tc = prec == INVDFT_MIXED_TF32;
    e = hx_op(h, a, s);
  }
  if (!cuda_ok(h, e, "apply_h")) return INVDFT_ECUDA;
  return INVDFT_OK;
}

invdft_status invdft_chebyshev_filter(invdft_handle h, const void *X, void *Y, int ncol, int degree,
                                      double a, double b, double a0, invdft_precision prec,
                                      void *stream) {
  if (!h || !X || !Y || ncol < 1 || ncol > h->nv || degree < 1 || !(b > a) || !(a0 < a)) {
    if (h) h->err = "chebyshev_filter: bad arguments (ncol <= nstates, b > a > a0)";
    return INVDFT_EINVAL;
  }
  if (!h->bound || !h->have_potential) {
    h->err = "chebyshev_filter: bind a workspace and set a potential first";
    return INVDFT_EINVAL;
  }
  return run_filter(h, X, Y, ncol, degree, a, b, a0, prec, nullptr, nullptr, (cudaStream_t)stream);
}

invdft_status invdft_reset(invdft_handle h) {
  if (!h) return INVDFT_EINVAL;
  h->have_orbitals = false;
  h->have_forward = false;
  h->have_grad = false;
  h->have_upper = false;
  h->have_ub_base = false;
  h->hist_n = h->hist_head = 0;
  return INVDFT_OK;
}

invdft_status invdft_profile_hx(invdft_handle h, int enable, double *out16) {
  if (!h) return INVDFT_EINVAL;
  HxProf &p = h->prof;
  if (!cuda_ok(h, prof_flush(h), "profile flush")) return INVDFT_ECUDA;
  if (out16) {
    for (int t = 0; t < 4; ++t) {
      out16[4 * t + 0] = p.ms[t];
      out16[4 * t + 1] = p.bytes_sum[t];
      out16[4 * t + 2] = p.flops_sum[t];
      out16[4 * t + 3] = (double)p.n[t];
    }
  }
  if (enable) {
    for (int t = 0; t < kProfKinds; ++t) {
      p.ms[t] = p.bytes_sum[t] = p.flops_sum[t] = 0.0;
      p.n[t] = 0;
    }
  }
  p.on = enable != 0;
  return INVDFT_OK;
}

invdft_status invdft_profile_deflation(invdft_handle h, double *out8) {
  if (!h || !out8) return INVDFT_EINVAL;
  HxProf &p = h->prof;
  if (!cuda_ok(h, prof_flush(h), "profile flush")) return INVDFT_ECUDA;
  for (int t = 0; t < 2; ++t) {
    out8[4 * t + 0] = p.ms[4 + t];
    out8[4 * t + 1] = p.bytes_sum[4 + t];
    out8[4 * t + 2] = 0.0;
    out8[4 * t + 3] = (double)p.n[4 + t];
  }
  return INVDFT_OK;
}

invdft_status invdft_tune_hx(invdft_handle h, int variant, int seglen, int *nvariants) {
  if (!h || seglen < 0 || variant < -1) return INVDFT_EINVAL;
  const int n32 = sweep_variants(h->g, 4), n64 = sweep_variants(h->g, 8);
  if (variant >= std::max(n32, n64)) {
    h->err = "tune_hx: variant out of range";
    return INVDFT_EINVAL;
  }
  h->hx_variant_fixed = variant;
  h->hx_seglen_fixed = seglen;
  if (nvariants) {
    nvariants[0] = n32;
    nvariants[1] = n64;
  }
  return INVDFT_OK;
}

invdft_status invdft_hx_config(invdft_handle h, int ncol, int fp64, int *variant_seglen) {
  if (!h || !variant_seglen) return INVDFT_EINVAL;
  const long long key = ((long long)ncol << 8) | ((fp64 ? 8 : 4) << 2);
  for (int k = 0; k < 4; ++k) {
    auto it = h->hx_tuned.find(key | k);
    variant_seglen[2 * k] = it == h->hx_tuned.end() ? -1 : it->second.first;
    variant_seglen[2 * k + 1] = it == h->hx_tuned.end() ? -1 : it->second.second;
  }
  return INVDFT_OK;
}

invdft_status invdft_graph_stats(long long *out3) {
  if (!out3) return INVDFT_EINVAL;
  for (int k = 0; k < 3; ++k) out3[k] = g_graph_stats[k].load(std::memory_order_relaxed);
  return INVDFT_OK;
}

invdft_status invdft_kernel_launches(unsigned long long *count) {
  if (!count) return INVDFT_EINVAL;
  *count = g_launches.load(std::memory_order_relaxed);
  return INVDFT_OK;
}

const char *invdft_last_error(invdft_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

}  // extern "C"
