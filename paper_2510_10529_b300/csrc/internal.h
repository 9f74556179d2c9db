// Internal declarations of libinvdft: the handle, device-table layout and the
// launchers of every kernel.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/invdft.h"

namespace invdft {

constexpr int kMaxOrder = 6;
constexpr int kMaxQ = kMaxOrder + 1;
constexpr int kMaxCols = 256;       // widest block H~X accepts
constexpr int kMaxGram = 128;       // widest block of Gram / rotation work
constexpr int kMaxDense = 96;       // widest subspace of the one-CTA dense eigensolver
constexpr int kMaxGroup = 16;       // largest degenerate set handled by the projections
constexpr int kGramBlocks = 296;    // 2 x 148 SMs: partial sums of tall-skinny reductions
constexpr int kMaxFilterDeg = 128;  // highest Chebyshev degree a forward-solve pass raises to

// Device status words of the kernels with bounded waits (non-zero: a wait gave
// up; the solvers read them back with their convergence data)
constexpr int kStWaitHxTc = 8;      // H~X on the tensor cores
constexpr int kStWaitHxSweep = 9;    // H~X in the sweep form (TMA plane loads)
constexpr int kStWaitGram = 10;     // deflation Gram on the tensor cores
constexpr int kStWaitUpdate = 11;   // deflation update on the tensor cores
constexpr int kStWaitCount = 4;

// Geometry and 1D factors of the cell operator, passed to kernels by value.
// A cell is a box with sizes (h_x, h_y, h_z); with A, B the 1D GLL stiffness
// and consistent mass on [-1, 1] and per-axis A_a = (2/h_a) A, B_a = (h_a/2) B,
//   K_e = 1/2 (B_z (x) B_y (x) A_x + B_z (x) A_y (x) B_x + A_z (x) B_y (x) B_x);
// on a uniform cube this is kc (B (x) B (x) A + ...) with kc = h/4.
struct Geom {
  int p, q;                 // order, nodes per cell edge
  int nc[3], n[3];          // cells and unknowns per axis (x, y, z)
  int ncell, Ni;            // nc[0], n[0]: the cube-only kernels (tensor cores, batch)
  bool cube;                // equal cells, the same on every axis
  bool graded;              // some axis has unequal cells
  long long L;              // unknowns
  double kc;                // h/4 on a cube
  double A[kMaxQ * kMaxQ];
  double B[kMaxQ * kMaxQ];
  // per axis (x, y, z), for axes of equal cells: half the cell size s = h/2,
  // and d = m1^-1/2 at the local nodes of a cell away from the boundary (an
  // interior vertex has m1 = 2 s w_0, node i in between m1 = s w_i)
  double s[3];
  double dl[3][kMaxQ];
  // device tables per axis: d = m1^-1/2 at every node of the axis (0 at the two
  // boundary nodes), the cell scalars 2/h_e and h_e/2, the node coordinates
  const double *dnode[3] = {}, *m1node[3] = {}, *cellA[3] = {}, *cellB[3] = {}, *axis[3] = {};
  const double *dm1;        // dnode[0] (cube kernels)
  const float *dm1f;        // the same table in FP32 (tensor-core path)
};

// Host-side FE tables (tables.cu): per axis, the cell breaks and sizes, the
// node coordinates, the 1D lumped mass and the assembled 1D matrix diagonals,
// all over the axis's nodes including the two boundary nodes.
struct AxisTab {
  std::vector<double> breaks, h;      // ncell + 1, ncell
  std::vector<double> axis;           // node coordinates, ncell p + 1
  std::vector<double> m1;             // 1D lumped mass
  std::vector<double> kdiag1_A, kdiag1_B;  // assembled 1D diagonals (for the preconditioner)
  bool uniform = true;                // equal cells
};
struct Tables {
  std::vector<double> gll_x, gll_w;   // q
  std::vector<double> A, B;           // q x q
  std::vector<double> Dm;             // q x q: l_j'(x_i) at the GLL nodes on [-1, 1]
  AxisTab ax[3];                      // x, y, z
};
void build_reference(int p, Tables *t);
// ng-point Gauss-Legendre rule on [-1, 1] and the order-p GLL Lagrange basis at
// its points: phi[k * (p+1) + j] = l_j(x_k)
void gauss_lagrange(int p, int ng, std::vector<double> *xg, std::vector<double> *wg,
                    std::vector<double> *phi);
void build_axis(const Tables &ref, const std::vector<double> &breaks, int p, AxisTab *ax);

// Bump allocator over the caller's workspace.
struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  template <class T> T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = reinterpret_cast<T *>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

// CUDA-event timing of every H~X launch, and of the tensor-core deflation
// launches of the MINRES iterations, while enabled (benchmark evidence): per
// kind the summed device time, algorithmic bytes, nominal dense-cell flops
// (H~X) and launch count.
constexpr int kProfKinds = 6;
struct HxProf {
  bool on = false;
  std::vector<cudaEvent_t> ev;     // 2 per slot
  std::vector<int> kind;
  std::vector<double> bytes, flops;
  int used = 0;
  // kinds: 0 FP64, 1 FP32 with W / E terms (filter), 2 other FP32, 3 TF32;
  // 4 deflation Gram, 5 deflation update (tcgen05, FP32 blocks)
  double ms[kProfKinds] = {}, bytes_sum[kProfKinds] = {}, flops_sum[kProfKinds] = {};
  long long n[kProfKinds] = {};
};
// Bracket one launch of the given kind with CUDA events on stream s (a no-op
// returning -1 while timing is off); prof_end closes the slot prof_begin
// returned.
struct Ctx;
int prof_begin(Ctx *c, int kind, double bytes, double flops, cudaStream_t s);
void prof_end(Ctx *c, int slot, cudaStream_t s);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) that only ever raises a
// kernel's limit (api.cu).  Several host threads may launch the same kernel
// with different shared-memory sizes (problems of a batch); a smaller limit
// set by one thread must never undercut a launch of another.
cudaError_t raise_smem_limit(const void *func, size_t bytes);
template <typename F>
cudaError_t raise_smem_limit(F *func, size_t bytes) {
  return raise_smem_limit(reinterpret_cast<const void *>(func), bytes);
}

struct BatchState;                  // batch_api.cu

struct Ctx {
  HxProf prof;
  BatchState *batch = nullptr;      // set while a batch step runs this problem
  int batch_index = -1;
  invdft_mesh_desc mesh{};
  invdft_opts o{};
  Tables tab;
  Geom g{};
  long long L = 0;
  int nv = 0;                       // nstates
  std::string err;
  bool bound = false;
  bool have_potential = false;
  bool have_orbitals = false;       // warm start available
  bool have_forward = false;        // eps/occ/psi of the last forward solve valid
  size_t ws_bytes = 0;
  Arena ar;
  double upper_bound = 0.0;         // cached spectral upper bound of H~
  // the last Lanczos bound and the potential it was taken at: a later
  // potential v bounds the spectrum by ub_base + max |v - v_ub| (Weyl)
  double ub_base = 0.0;
  bool have_ub_base = false;
  int ub_reuse = 0;
  double *v_ub = nullptr;
  double eig_tol_used = 0.0;        // eigen tolerance of the last forward solve
  bool have_upper = false;

  // ---- device state (inside the workspace)
  double *dnode[3] = {};            // [n_a + 2] per axis: m1^-1/2 (0 at the boundary)
  float *dm1f = nullptr;            // [n_x + 2] FP32 copy of dnode[0] (cube kernels)
  double *m1tab[3] = {}, *kAtab[3] = {}, *kBtab[3] = {};  // [n_a + 2] 1D tables per axis
  double *cellA[3] = {}, *cellB[3] = {}, *axis[3] = {};    // per axis: 2/h_e, h_e/2; coordinates
  double *mass = nullptr;           // [L]
  double *dvec = nullptr;           // [L]  m^-1/2
  double *prec_diag = nullptr;      // [L]  1 / diag(D K D)
  float *precf = nullptr;           // [L]  FP32 copy (FP32 MINRES)
  float *Ke_tc = nullptr;           // 128 x 128 TF32 cell matrix in the UMMA layout (Q4)
  int *cell_perm = nullptr;         // [ncell^3] visiting order of the tensor-core kernel
  double *v = nullptr;              // [L]  total potential
  float *vf = nullptr;              // [L]  FP32 copy (FP32 CUDA-core H~X)
  double *vfixed = nullptr;         // [L]
  double *X = nullptr;              // [L][nv] orbitals (FP64)
  double *Y = nullptr;              // [L][nv]
  double *HY = nullptr;             // [L][nv]
  void *C0 = nullptr, *C1 = nullptr, *C2 = nullptr;  // filter buffers [L][nv] (prec)
  float *E32 = nullptr;             // [L][nv] residual copy for the defect-corrected filter
  double *eps = nullptr, *occ = nullptr, *dfde = nullptr, *rho = nullptr;
  double *small = nullptr;          // dense scratch: 8 * kMaxCols^2 doubles
  double *partial = nullptr;        // kGramBlocks * kMaxCols^2 doubles
  double *scal = nullptr;           // 1024 * kMaxCols doubles of per-column scalars and tables
  int *status = nullptr;            // device status words [16]
  // adjoint
  double *P = nullptr;              // [L][nv] adjoint output (FP64)
  double *Rg = nullptr;             // [L][nv] right-hand sides / residuals (FP64)
  void *mr[9] = {};                 // MINRES work blocks [L][nv] (FP32 or FP64)
  // inverse loop
  double *grad = nullptr, *grad_new = nullptr, *dir = nullptr, *vtry = nullptr, *dLdrho = nullptr;
  double *Sh = nullptr, *Yh = nullptr;   // [hist][L]
  int hist_n = 0, hist_head = 0;
  bool have_grad = false;
  double loss = 0.0, err_l2 = 0.0;
  // pinned host mirror for small read-backs
  double *hbuf = nullptr;           // 16 * kMaxCols doubles
  int nsm = 148;                    // SMs of the device (set at bind)
  // sweep H~X configuration: fixed by invdft_tune_hx (variant >= 0 and / or
  // seglen > 0), else autotuned per (ncol, precision, W, E) -> (variant, seglen)
  int hx_variant_fixed = -1, hx_seglen_fixed = 0;
  std::map<long long, std::pair<int, int>> hx_tuned;
  cudaStream_t aux_stream = nullptr;  // non-blocking stream for captured work (lazy)
  cudaEvent_t aux_event = nullptr;
};

}  // namespace invdft

// The opaque handle type of the C ABI is the context itself.
struct invdft_ctx : public invdft::Ctx {};

namespace invdft {

// ------------------------------------------------------------ error helpers
bool cuda_ok(Ctx *c, cudaError_t e, const char *what);
// text of invdft_last_error(NULL) (failures with no handle)
void set_global_error(const char *msg);
// process-wide count of kernels this library has launched (benchmark evidence)
void count_launch();
// n kernels run by a graph replay (negative: take back launches counted while
// capturing a graph); launches counted so far by this thread
void count_launches(long long n);
unsigned long long thread_launches();
// process-wide CUDA-graph counters: 0 captures, 1 replays, 2 refused captures
void count_graph(int what);
#define INV_CUDA(c, call)                                   \
  do {                                                      \
    if (!::invdft::cuda_ok((c), (call), #call)) return INVDFT_ECUDA; \
  } while (0)
#define INV_LAUNCH(c, what)                                 \
  do {                                                      \
    if (!::invdft::cuda_ok((c), cudaGetLastError(), what)) return INVDFT_ECUDA; \
  } while (0)

// Division by a runtime constant for 32-bit indices x < 2^31 (Granlund &
// Montgomery 1994): q = (umulhi(x, m) + x) >> s with s = ceil(log2 d),
// m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  uint32_t d = 1, m = 1, s = 0;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while ((1ull << f.s) < d) ++f.s;
  f.m = (uint32_t)(((1ull << 32) * ((1ull << f.s) - d)) / d + 1);
  return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv &f) {
  return (__umulhi(x, f.m) + x) >> f.s;
}
#endif

// ------------------------------------------------------------ H~X (hx.cu)
// Z = alpha * (H~ X - shift o X) + beta * W + alpha * E diag(escale)
//   shift: per-column (shift_col != nullptr) or the scalar shift;
//   W, E optional (nullptr); escale per column (device) for E.
template <typename T>
struct HxArgs {
  const T *X = nullptr;
  T *Z = nullptr;
  int ncol = 0;
  double alpha = 1.0;
  double shift = 0.0;
  const double *shift_col = nullptr;
  const T *W = nullptr;
  double beta = 0.0;
  const float *E = nullptr;
  const double *escale = nullptr;
  bool tc = true;            // FP32 blocks: TF32 tensor-core path where available
};
cudaError_t launch_hx(const Geom &g, const double *v, const HxArgs<double> &a, cudaStream_t s);
cudaError_t launch_hx(const Geom &g, const double *v, const HxArgs<float> &a, cudaStream_t s);
// launch_hx on the handle's operator, timed with CUDA events when profiling is on
cudaError_t hx_op(Ctx *c, const HxArgs<double> &a, cudaStream_t s);
cudaError_t hx_op(Ctx *c, const HxArgs<float> &a, cudaStream_t s);
// the same without the collocated potential term (dense cell potentials)
cudaError_t hx_op_nopot(Ctx *c, const HxArgs<double> &a, cudaStream_t s);
cudaError_t hx_op_nopot(Ctx *c, const HxArgs<float> &a, cudaStream_t s);
cudaError_t prof_flush(Ctx *c);
// tensor-core (tcgen05, TF32) H~X for Q4 cells (hx_tc.cu)
void build_tc_cell_matrix(const Geom &g, std::vector<float> *out);
size_t tc_cell_matrix_floats();
cudaError_t launch_hx_tc(const Geom &g, const double *v, const HxArgs<float> &a, const float *Ke,
                         const int *perm, int *err, cudaStream_t s);
void build_cell_order(int nc, std::vector<int> *perm);
// tensor-pipe rate probe (M = 128, N = 64, K = 128 TF32 MMA chains); err: set if
// the final wait gave up; flops: the launch's floating-point operations
cudaError_t launch_tf32_probe(int grid, int chains, int *err, double *flops, cudaStream_t s);
// Owner-computes sweep form of H~X (hx_sweep.cu): FP32 and FP64 blocks on
// orders 2, 4 and 6, ncol * elem a multiple of 16 bytes, 16-byte aligned
// blocks, Z not aliasing X, W or E.  variant in [0, sweep_variants) selects the
// tile shape; seglen = z-cells per CTA (the z range is split into segments of
// that many cells), or kSegBalanced for the persistent balanced schedule (one
// CTA per resident slot: whole (tile, chunk) units round-robin, then an equal
// share of the z-cells of the units left over; plain launches on uniform
// meshes, others run the whole z range).  err: device word set to 3 if a wait
// for a TMA plane gave up.
constexpr int kSegBalanced = INVDFT_HX_SEG_BALANCED;
bool sweep_supported(const Geom &g, int ncol, size_t elem, const void *X, const void *Z,
                     const void *W, const void *E);
int sweep_variants(const Geom &g, size_t elem);
cudaError_t launch_hx_sweep(const Geom &g, const float *v, const HxArgs<float> &a, int *err,
                            int variant, int seglen, cudaStream_t s);
cudaError_t launch_hx_sweep(const Geom &g, const double *v, const HxArgs<double> &a, int *err,
                            int variant, int seglen, cudaStream_t s);


// ------------------------------------------------------------ vector kernels (blas.cu)
// G[i*n2+j] = sum_a A[a*lda+i] B[a*ldb+j] in FP64 (partials then a fixed-order sum).
cudaError_t launch_gram(const double *A, int n1, const double *B, int n2, long long L,
                        double *G, double *partial, cudaStream_t s);
cudaError_t launch_gram_f32(const float *A, int n1, const float *B, int n2, long long L,
                            double *G, double *partial, cudaStream_t s);
// FP32 inputs, FP32 accumulation inside a CTA, FP64 across CTAs
cudaError_t launch_gram_f32acc(const float *A, int n1, const float *B, int n2, long long L,
                               double *G, double *partial, cudaStream_t s);
// Row-striped tall-skinny Gram (n1, n2 <= 64) and row-tiled update
// (n1, n2 <= 128): G = A^T B, Z += alpha Psi C
template <typename T, typename TA>
cudaError_t launch_stripe_gram(const T *A, int n1, const T *B, int n2, long long L, double *G,
                               double *partial, cudaStream_t s);
template <typename T>
cudaError_t launch_stripe_rotate(const T *Psi, int n1, const double *C, int n2, long long L, T *Z,
                                 double alpha, cudaStream_t s);
// S = Y^T Y and Hs = Y^T HY (both n x n, symmetric by construction: the upper
// 4 x 4 tiles are formed and mirrored), n <= 96
cudaError_t launch_gram_rr(const double *Y, const double *HY, int n, long long L, double *S,
                           double *Hs, double *partial, cudaStream_t s);
// FP32 deflation pair for MINRES blocks (deflate.cu).  Widths n1p (a multiple
// of 8) and n2p (a multiple of 4) are at most 64 (zero padding columns),
// blocks 16-byte aligned.
// G[i*n2p + j] = sum_a Psi[a][i] Z[a][j] (FP32 within a CTA, FP64 across CTAs)
cudaError_t launch_defl_gram_f32(const float *Psi, int n1p, const float *Z, int n2p, long long L,
                                 double *G, double *partial, cudaStream_t s);
// Z += alpha Psi C (C is n1p x n2p, FP64); with V != null also
// dot_out[j] = sum_a V[a][j] Z_new[a][j] (FP32 within a tile, FP64 across)
cudaError_t launch_defl_update_f32(const float *Psi, int n1p, const double *C, int n2p,
                                   long long L, float *Z, double alpha, const float *V,
                                   double *dot_out, double *partial, cudaStream_t s);
// Tensor-core version of launch_defl_gram_f32 (deflate_tc.cu): G[n1p][n2p] =
// Psi^T Z with two-term TF32 splitting of both operands, FP64 sums across
// CTAs; partial holds 2 nsm * n1p * n2p doubles; err: device word set to 4 if
// an MMA wait gave up.
cudaError_t launch_defl_gram_tc(const float *Psi, int n1p, const float *Z, int n2p, long long L,
                                double *G, double *partial, int *err, int nsm, cudaStream_t s);
// Tensor-core version of launch_defl_update_f32 (deflate_tc.cu): Z += alpha
// Psi C with C^T and Psi split in two TF32 terms (three products), Psi read by
// one TMA tensor copy per 128-node tile; partial holds nsm * n2p doubles; err:
// device word set to 5 if a wait gave up.
cudaError_t launch_defl_update_tc(const float *Psi, int n1p, const double *C, int n2p,
                                  long long L, float *Z, double alpha, const float *V,
                                  double *dot_out, double *partial, int *err, int nsm,
                                  cudaStream_t s);
// out[e] = sum_b partial[b * n + e], b < nblk
cudaError_t launch_sum_partials(const double *partial, int nblk, int n, double *out,
                                cudaStream_t s);
// F[a][j] = j < n ? X[a][j] : 0 for j < np (FP64 -> FP32 with zero padding)
cudaError_t launch_convert_pad_f32(const double *X, int n, int np, long long L, float *F,
                                   cudaStream_t s);
// P[a][j] += F[a][j] for j < n (FP32 padded block of width np into FP64)
cudaError_t launch_add_unpad(const float *F, int np, double *P, int n, long long L,
                             cudaStream_t s);
// Xo += alpha * Xi Cm  (n1 -> n2 columns) in the storage precision T
template <typename T>
cudaError_t launch_rotate_acc(const T *Xi, int n1, const double *Cm, int n2, long long L, T *Xo,
                              double alpha, cudaStream_t s);
// Xo[a][j] = sum_i Xi[a][i] Cm[i*n2 + j]   (n1 -> n2 columns), FP64
cudaError_t launch_rotate(const double *Xi, int n1, const double *Cm, int n2, long long L,
                          double *Xo, cudaStream_t s);
// column-wise dot products d[j] = sum_a A[a][j] B[a][j] (FP64 accumulate)
cudaError_t launch_coldot(const double *A, const double *B, int ncol, long long L, double *d,
                          double *partial, cudaStream_t s);
cudaError_t launch_coldot_f32(const float *A, const float *B, int ncol, long long L, double *d,
                              double *partial, cudaStream_t s);
// weighted scalar sums over nodes: out[k] = sum_a f_k(a) (see blas.cu)
// Out[a][c] = X[a*nv + idx[c]]
cudaError_t launch_gather_cols(const double *X, int nv, const int *idx, int n, long long L,
                               double *Out, cudaStream_t s);
cudaError_t launch_convert_f64_to_f32(const double *x, float *y, long long n, cudaStream_t s);
cudaError_t launch_convert_f32_to_f64(const float *x, double *y, long long n, cudaStream_t s);
cudaError_t launch_fill_random(double *X, long long n, unsigned long long seed, cudaStream_t s);

}  // namespace invdft
