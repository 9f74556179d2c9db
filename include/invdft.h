/*
 * invdft.h -- C ABI of the B300 inverse-DFT hot-path library (libinvdft.so).
 *
 * The library implements, on one GPU, the data-parallel hot path of the
 * adjoint-based inverse density-functional method of arXiv 2510.10529
 * ("invDFT"):
 *   - the finite-element Kohn-Sham Hamiltonian in standard form,
 *     H~ = M^-1/2 H M^-1/2 = D K D + diag(v)   (Eq. 17, Eq. 19),
 *     applied cell by cell to blocks of vectors (Sec. 3.2.3);
 *   - the Chebyshev-filtered subspace iteration with Rayleigh-Ritz
 *     (Sec. 3.2.2, Eq. 23-24) for the lowest eigenpairs;
 *   - Fermi-Dirac occupations and the density (Eq. 4, Eq. 5);
 *   - the loss (Eq. 1), the projected adjoint solves by preconditioned MINRES
 *     (Eq. 7-10, Eq. 20, Sec. 3.2.2) and the gradient dL/dv_xc (Eq. 11, 22)
 *     with the far-field mask (Sec. 3.1.2);
 *   - the limited-memory BFGS update of v_xc (Eq. 21).
 *
 * Discretisation (shared by every entry point): a box cut into a tensor
 * product of box cells of order p (2, 4 or 6) with nodes at the
 * Gauss-Lobatto-Legendre points (spectral elements, Sec. 3.2.1), equal cells
 * per axis or graded ones (invdft_mesh_desc).  Boundary nodes carry
 * psi = p = 0; the L = prod_a (ncell[a] p - 1) interior nodes are the
 * unknowns, numbered lexicographically with x fastest, then y, then z.
 *
 * Data layout: every nodal multivector is node-major ("row-major" in the
 * paper's words, Sec. 3.2.3): element (a, j) of an [L][ncol] block is at
 * a*ncol + j.  Nodal scalar fields are [L].  All arrays are C-contiguous.
 *
 * Ownership: the caller owns every array it passes.  Arrays documented as
 * "device" must be device pointers of the current CUDA device; "host" arrays
 * are host pointers.  The handle keeps pointers to nothing the caller owns
 * except the workspace bound by invdft_bind_workspace, which must stay valid
 * (and unused by anyone else) until the handle is destroyed or rebound.
 *
 * Streams: every call is enqueued on `stream` (a cudaStream_t passed as
 * void*; NULL is the legacy default stream).  Calls that return host values
 * (loss, stats, iteration counts) synchronise that stream before returning.
 *
 * Errors: every call returns an invdft_status and never throws across the
 * ABI.  On failure the text of the last error is available from
 * invdft_last_error(handle) (or invdft_last_error(NULL) for failures before a
 * handle exists).  INVDFT_ENOCONV leaves valid, flagged results.
 * INVDFT_ETIMEOUT is reported by the solves that read back the kernels' wait
 * status words (forward solve, adjoint MINRES, batch step): a kernel whose
 * bounded wait gave up set its word and left early, so the results of that
 * call are not valid.  The words of the H~X and Gram kernels stay set for
 * the handle, so every later solve on it reports the error again; destroy
 * the handle after it.  The batch kernel's word is cleared at each launch
 * (invdft_batch_set_wait_limit).
 *
 * Threading: a handle is not thread safe; distinct handles are independent.
 */
#ifndef INVDFT_H
#define INVDFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct invdft_ctx *invdft_handle;

typedef enum {
  INVDFT_OK = 0,
  INVDFT_EINVAL = 1,    /* bad argument, shape, order or state            */
  INVDFT_ENOMEM = 2,    /* workspace missing or too small                 */
  INVDFT_ECUDA = 3,     /* a CUDA runtime error; text in last_error       */
  INVDFT_ENOCONV = 4,   /* an iteration cap was reached; results flagged  */
  INVDFT_ETIMEOUT = 5,  /* a bounded device wait expired                  */
  INVDFT_ENOTSPD = 6    /* Cholesky of the subspace overlap failed        */
} invdft_status;

typedef enum {
  INVDFT_FP64 = 0,      /* every step in FP64                                     */
  INVDFT_MIXED = 1,     /* FP32 storage and FP32 cell products on the CUDA cores
                           in the Chebyshev filter and the inner MINRES
                           iterations; FP64 for Rayleigh-Ritz, Cholesky,
                           residuals, refinement and every reduction             */
  INVDFT_MIXED_TF32 = 2 /* as MIXED, but the Chebyshev filter's cell products
                           (Q4 meshes) run on the TF32 tensor cores (tcgen05)
                           with FP32 accumulation; MINRES stays in FP32         */
} invdft_precision;

/* Mesh: the box [lo[0],hi[0]] x [lo[1],hi[1]] x [lo[2],hi[2]] (x, y, z) cut
 * into ncell[0] x ncell[1] x ncell[2] box cells of element order 2, 4 or 6.
 * breaks[a] (optional, host, ncell[a] + 1 values, copied at create) gives the
 * cell breaks of axis a, increasing from lo[a] to hi[a], for meshes graded
 * towards features (Sec. 4.2.2: finer cells near the nuclei); NULL means equal
 * cells on that axis.  The nodes form a tensor-product grid, so the cell
 * stiffness keeps its Kronecker form with per-cell scalars (Eq. 17). */
typedef struct {
  double lo[3], hi[3];
  int ncell[3];
  int order;
  const double *breaks[3];
} invdft_mesh_desc;

/* Solver options.  Zero fields take the defaults given in brackets.
 * c_eig, c_ad, tau_bc default to the paper's values (Sec. 4.2.4). */
typedef struct {
  int nstates;            /* N_v in [1, 96]: Ritz vectors (occupied + buffer)  */
  double n_electrons;     /* N_e (Eq. 5)                                        */
  double kT;              /* k_B T in Ha; 0 = closed shell (N_e even)           */
  int cheb_degree;        /* Chebyshev filter degree m                  [20]   */
  double c_eig;           /* t_eig = e_L2^2 / c_eig                     [1e2]  */
  double c_ad;            /* t_ad  = e_L2^2 / c_ad                      [1e5]  */
  double tau_bc;          /* gradient mask threshold on rho_data        [1e-6] */
  double eig_tol;         /* fixed eigen-residual tolerance if > 0; else the
                             adaptive rule with floor 1e-10                     */
  double adj_tol;         /* fixed relative adjoint tolerance if > 0; else the
                             adaptive rule with floor 1e-10                     */
  int max_cheb_passes;    /* cap on filter + Rayleigh-Ritz passes       [60]   */
  int max_minres_iters;   /* cap on inner MINRES iterations per solve   [2000] */
  int lbfgs_history;      /* L-BFGS pairs kept                          [10]   */
  invdft_precision prec;  /* FP64, MIXED or MIXED_TF32                          */
  unsigned long long seed;/* seed of the random start block                     */
  double deg_tol;         /* eigenvalues closer than this form a degenerate
                             set (Ha)                                   [1e-8] */
} invdft_opts;

/* Per-call statistics (host struct filled by the calls that take it). */
typedef struct {
  double loss, err_l2, n_elec, mu;
  double eig_resid_max;   /* max standard-form residual over occupied states   */
  double adj_resid_max;   /* max relative true residual of the adjoint solves  */
  double eta;             /* multiplier of Eq. 9                               */
  int cheb_passes, hx_calls, minres_iters_max, ls_trials, refinements;
  double t_forward_ms, t_adjoint_ms;
} invdft_stats;

/* Create a handle for one problem.  Computes the GLL rule, the element
 * matrices and the lumped mass on the host; allocates nothing on the device.
 * n_nodes_out (optional) receives L.                                        */
invdft_status invdft_create_mesh(const invdft_mesh_desc *mesh, const invdft_opts *opts,
                                 invdft_handle *out, long long *n_nodes_out);
invdft_status invdft_destroy(invdft_handle h);

/* Device scratch needed by the solvers for this mesh and these options.
 * The caller allocates it (e.g. as a torch uint8 tensor) and binds it; the
 * handle then uploads its tables and keeps orbitals, the L-BFGS history and
 * every work vector there.  apply_h with ncol <= nstates needs the same
 * workspace.  Binding again moves the handle to the new region (state is
 * reset).                                                                   */
invdft_status invdft_workspace_size(invdft_handle h, size_t *bytes);
invdft_status invdft_bind_workspace(invdft_handle h, void *device_ptr, size_t bytes,
                                    void *stream);

/* Host output: xyz [L][3] coordinates (bohr) of the unknown nodes.          */
invdft_status invdft_node_coords(invdft_handle h, double *xyz_host);
/* Device output: m [L], the lumped (GLL) mass diagonal = quadrature weights.*/
invdft_status invdft_mass_diag(invdft_handle h, double *m_dev, void *stream);

/* Set the potential: v = v_fixed + v_xc at the unknown nodes (device [L]).
 * v_fixed = v_ext + v_H[rho_data] (Eq. 2); v_xc may be NULL (zero).        */
invdft_status invdft_set_potential(invdft_handle h, const double *v_fixed_dev,
                                   const double *v_xc_dev, void *stream);

/* Y = H~ X for an [L][ncol] block (Eq. 19, Sec. 3.2.3), device pointers.
 * prec = INVDFT_FP64: X, Y are double; INVDFT_MIXED (FP32 on the CUDA
 * cores) or INVDFT_MIXED_TF32 (TF32 tensor cores on uniform cubic Q4 meshes,
 * the CUDA cores elsewhere): X, Y are float.  Y must not alias X.
 * ncol in [1, 256].  The operator used is the one of the last
 * invdft_set_potential.                                                     */
invdft_status invdft_apply_h(invdft_handle h, const void *X_dev, void *Y_dev, int ncol,
                             invdft_precision prec, void *stream);

/* Chebyshev filter Y = p_m(H~) X with p_m(t) = T_m((t-c)/e)/T_m((a0-c)/e),
 * e = (b-a)/2, c = (b+a)/2, by the scaled three-term recurrence (Sec. 3.2.2).
 * X, Y: device [L][ncol] in the precision `prec` (double or float).  Exposed
 * for testing the filter on its own.                                        */
invdft_status invdft_chebyshev_filter(invdft_handle h, const void *X_dev, void *Y_dev,
                                      int ncol, int degree, double a, double b, double a0,
                                      invdft_precision prec, void *stream);

/* Forward Kohn-Sham solve at the current potential (Sec. 3.2.2):
 * Chebyshev-filtered subspace iteration with FP64 Rayleigh-Ritz until the
 * largest residual over occupied states is below the eigen tolerance.
 * psi: device [L][nstates] standard-form orbitals psi~ (out; also the warm
 * start kept inside the handle); eps, occ: device [nstates]; rho: device [L].
 * Any output pointer may be NULL.                                           */
invdft_status invdft_forward_solve(invdft_handle h, double *psi_dev, double *eps_dev,
                                   double *occ_dev, double *rho_dev, invdft_stats *stats,
                                   void *stream);

/* Adjoint solve for a generic upstream dL/drho (device [L]) around the last
 * forward solve: returns p~ (device [L][nstates], zero for empty states)
 * (Eq. 7-10, 20).  The paper's loss has dL/drho_a = -2 m_a w_a (rho_d-rho)_a.
 * The relative tolerance is opts.adj_tol if set, else the adaptive rule.    */
invdft_status invdft_adjoint_solve(invdft_handle h, const double *dL_drho_dev, double *p_dev,
                                   invdft_stats *stats, void *stream);

/* Vector-Jacobian product of the density map v -> rho(v) around the last
 * forward solve: grad_v = sum_i p~_i o psi~_i with p~ the adjoint functions
 * for the upstream dL/drho (device [L] in, device [L] out, no far-field
 * mask).  This is the backward of the Kohn-Sham solve (Eq. 7-11).          */
invdft_status invdft_density_vjp(invdft_handle h, const double *dL_drho_dev, double *grad_v_dev,
                                 invdft_stats *stats, void *stream);

/* Loss and masked gradient at the current potential: forward solve, loss
 * (Eq. 1), adjoint and grad_b = sum_i p~_bi psi~_bi, zero where
 * rho_data < tau_bc (Eq. 11, 22, Sec. 3.1.2).  rho_data, w, grad: device [L];
 * loss_out: host scalar (optional).                                          */
invdft_status invdft_loss_grad(invdft_handle h, const double *rho_data_dev, const double *w_dev,
                               double *loss_out, double *grad_dev, invdft_stats *stats,
                               void *stream);

/* One inverse iteration (Eq. 21): L-BFGS direction from the history kept in
 * the handle, backtracking line search (one forward solve per trial), then
 * loss, adjoint and gradient at the accepted point.  v_xc: device [L], in/out.
 * The potential of the handle becomes v_fixed + v_xc(new).  The first call
 * after set_potential/reset evaluates the gradient at the incoming v_xc.     */
invdft_status invdft_step(invdft_handle h, const double *rho_data_dev, const double *w_dev,
                          double *v_xc_dev, invdft_stats *stats, void *stream);

/* ---- Batched multi-problem execution.  The paper batches the shifted
 * adjoint systems of one problem into one block solve (Sec. 3.2.2); this
 * batches whole independent problems (no further counterpart in the paper).
 * invdft_batch_create: handles bound, in INVDFT_MIXED or INVDFT_MIXED_TF32
 * precision, on uniform cubic meshes (equal box, cells and sizes on every
 * axis) of order 2 or 4, with equal Chebyshev degree in [2, 64] and nstates
 * <= 256;
 * n in [1, 64], no handle twice.  The batch keeps the handle pointers: they
 * must outlive it, and no other call may use them while a batch step runs.
 * EINVAL on bad arguments, ECUDA if its streams or device tables cannot be
 * created.
 * invdft_batch_step: one invdft_step of every problem.  rho_data, w, v_xc
 * are host arrays of n device pointers (v_xc[b] in/out, [L_b] each); stats
 * and status (optional) are host arrays of n receiving each problem's
 * statistics and status.  The problems run concurrently, each on its own
 * stream; each pass of their Chebyshev filters (the defect-corrected FP32
 * recurrence) is combined with the passes of the other problems waiting at
 * that moment into one cooperative persistent kernel over a device work
 * queue of (phase, problem, cell tile) items, launched from a captured CUDA
 * graph per set of problems.  The first call autotunes the column chunk of
 * each (order, width) class.  Ordered after `stream`; `stream` waits for the
 * whole step; returns the worst status (ETIMEOUT if a phase wait of the
 * persistent kernel gave up).
 * invdft_batch_info: chunk_cols[b] (host, n; optional) = the column chunk of
 * problem b; info4 (optional) = {batched filter launches, of which CUDA-graph
 * replays, persistent CTAs per launch, autotuned (0/1)}.                    */
typedef struct invdft_batch_ctx *invdft_batch;
invdft_status invdft_batch_create(const invdft_handle *handles, int n, invdft_batch *out);
invdft_status invdft_batch_destroy(invdft_batch batch);
invdft_status invdft_batch_step(invdft_batch batch, const double *const *rho_data_dev,
                                const double *const *w_dev, double *const *v_xc_dev,
                                invdft_stats *stats, invdft_status *status, void *stream);
invdft_status invdft_batch_info(invdft_batch batch, int *chunk_cols, double *info4);
/* invdft_batch_set_wait_limit: the persistent filter kernel waits for the
 * previous phase of a problem by polling its phase counter, with a back-off
 * of 256 ns per poll, and gives up after `polls` polls: it sets its error
 * word, every CTA leaves, and the step returns INVDFT_ETIMEOUT for the
 * problems of that launch (the results of that step are not valid).
 * polls < 0 restores the default of 2^24 polls (seconds); polls = 0 makes
 * the first wait for a previous phase give up at once, whether that phase is
 * complete or not.  A zero or small limit makes a wait run out without any
 * device fault, which is how the timeout path is tested.  Call it between
 * steps.  EINVAL for a NULL batch, ECUDA if the limit cannot be copied to
 * the device.                                                               */
invdft_status invdft_batch_set_wait_limit(invdft_batch batch, int polls);

/* Instrumentation for benchmarks (no counterpart in the paper).
 * invdft_profile_hx: while enabled, every H~X launch of this handle is
 * bracketed by CUDA events on its stream.  Each call first drains pending
 * events (synchronising on them) and, if out16 != NULL, writes the totals
 * since the last enable: out16[0..3] = FP64 {device ms, algorithmic bytes
 * (X and v read, Z written, plus W/E when present), nominal dense-cell
 * flops 2 (p+1)^6 ncol cells, launches}, out16[4..7] the same for FP32
 * launches on the CUDA cores that carry the Chebyshev filter's W or E terms,
 * out16[8..11] for the other FP32 CUDA-core launches (the MINRES operator),
 * out16[12..15] for FP32 blocks on the TF32 tensor-core kernel.
 * enable = 1 resets the totals and turns timing on; 0 turns it off.
 * invdft_kernel_launches: process-wide count of kernels launched by this
 * library since it was loaded (kernels run by CUDA-graph replays included).
 * invdft_graph_stats: out3 = {graphs captured, graph replays, captures the
 * runtime refused (the work then ran as plain launches)}, process-wide.     */
invdft_status invdft_profile_hx(invdft_handle h, int enable, double *out16);
/* invdft_profile_deflation: while the timing of invdft_profile_hx is on, the
 * tensor-core deflation launches of the FP32 MINRES iterations (blocks of 16
 * or more columns) are timed the same way.  Drains pending events and writes
 * the totals since the last enable: out8[0..3] = Gram C = Psi^T Z {device ms,
 * algorithmic bytes ((n_psi + n_z) x 4 per node: Psi and Z read once), 0,
 * launches}, out8[4..7] = update Z -= Psi C {ms, bytes ((n_psi + 3 n_z) x 4
 * per node with the fused column dot: Psi, Z and V read, Z written), 0,
 * launches}.  EINVAL for a NULL handle or out8, ECUDA on a CUDA error.       */
invdft_status invdft_profile_deflation(invdft_handle h, double *out8);

/* Tuning of H~X (no counterpart in the paper).  On orders 2, 4 and 6, FP32
 * and FP64 blocks whose rows are a multiple of 16 bytes run in the sweep form: a
 * CTA owns a column of nodes of the x-y plane and a chunk of columns, and
 * walks a segment of the z range.  Several tile variants exist (columns per
 * CTA, tile height, planes in flight, x-cells per task).
 * invdft_tune_hx: variant >= 0 fixes the tile variant, seglen > 0 the segment
 * length (in cells) for every later H~X launch of this handle; -1 / 0 leave
 * them to the autotuner, which on the first launch of each (precision, ncol,
 * epilogue) on a mesh of 2^18 unknowns or more that is not being captured
 * into a graph times every variant with the whole z range, halves, quarters,
 * segments short enough for two CTAs per SM and the balanced schedule, and
 * keeps the fastest (smaller meshes, and launches inside a capture before
 * that, take variant 0 with the short segments).
 * seglen = INVDFT_HX_SEG_BALANCED fixes the balanced schedule: a persistent
 * grid of one CTA per resident slot that takes whole (tile, column chunk)
 * units round-robin and then an equal share of the z-cells of the units left
 * over, so that no second wave runs on part of the GPU (launches without the
 * W and E terms on meshes of equal cells; others then run the whole z range
 * per CTA).  nvariants (optional,
 * host int[2]) receives the number of FP32 and FP64 variants for this mesh
 * order.  EINVAL for a NULL handle, seglen < 0 or a variant out of range.
 * invdft_hx_config: the autotuned (variant, seglen) of this handle for a
 * width ncol and precision (fp64 != 0: FP64), for the four epilogues
 * {plain, E only, W only, W and E}: variant_seglen (host int[8]), -1 where
 * that configuration has not been tuned; a negative seglen -n means the
 * segment length is chosen per launch for at least n CTAs, and
 * INVDFT_HX_SEG_BALANCED the balanced schedule.                              */
#define INVDFT_HX_SEG_BALANCED 0x7fffffff
invdft_status invdft_tune_hx(invdft_handle h, int variant, int seglen, int *nvariants);
invdft_status invdft_hx_config(invdft_handle h, int ncol, int fp64, int *variant_seglen);
invdft_status invdft_kernel_launches(unsigned long long *count);
/* invdft_peak_probe: the arithmetic rate of this device in TFLOP/s, measured
 * at the clocks it runs at by a kernel that fills the GPU with independent
 * operations on register (or shared-memory) operands and no memory traffic:
 * kind 0 FP64 FMA, 1 FP32 FMA, 2 packed FP32 FMA pairs, 3 TF32 tensor-core
 * MMAs of the H~X kernel's shape (M = 128, N = 64, K = 128).  These are the
 * roofline denominators of kernels bound by arithmetic.  tflops (host) is
 * written; ms_out (optional, host) receives the timed launch's duration.
 * Synchronous; allocates a few bytes of scratch.  EINVAL for a bad kind,
 * ECUDA on a CUDA error, ETIMEOUT if the tensor-core probe's wait gave up. */
invdft_status invdft_peak_probe(int kind, double *tflops, double *ms_out, void *stream);
invdft_status invdft_graph_stats(long long *out3);

/* Allocation-free loss reduction.  The paper has no counterpart: this entry
 * point exists for callers that must not allocate device memory -- a host
 * application that owns all device memory through its own fixed pool and
 * forbids further cudaMalloc/cudaFree (to keep its footprint fixed, or
 * because an allocation would synchronise the device in the middle of its
 * pipeline), or a caller that simply has no workspace to bind.  It computes,
 * like the reduction inside invdft_loss_grad,
 *   out3[0] = sum_a m_a w_a (rho_data_a - rho_a)^2   (the weighted loss),
 *   out3[1] = sum_a m_a (rho_data_a - rho_a)^2       (the squared L2 error),
 *   out3[2] = sum_a m_a rho_a                        (the electron count),
 * and, if dLdrho != NULL, dLdrho_a = -2 m_a w_a (rho_data_a - rho_a).
 * All arrays are device arrays of length L (out3: 3 doubles) owned by the
 * caller; w may be NULL (w = 1).  No handle is needed.
 * Scratch: a fixed 192 KiB device array inside the library, which every GPU
 * that loads the library keeps until the process exits; it holds one partial
 * sum per 4096 nodes, so L is limited to 33,554,432 (larger L returns
 * INVDFT_EINVAL with a message in invdft_last_error(NULL)).  Every partial
 * used is rewritten by each call, so nothing needs clearing between calls,
 * and the array keeps the last call's partials afterwards.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture.  All calls share the one array: calls that may overlap on the GPU
 * (different streams, or different host threads) race and must be serialised
 * by the caller.  The call allocates nothing and is asynchronous on stream. */
invdft_status invdft_loss_reduce_noalloc(const double *rho, const double *rho_data,
                                         const double *w, const double *mass, long long L,
                                         double *out3, double *dLdrho, void *stream);

/* Initial guess of v_xc (Sec. 4.2.3, Eq. 25-26) at the unknown nodes:
 *   v_out = f v0[rho] + (1 - f) alpha v_FA,  f = rho / (rho + tau),
 *   v_FA = -v_H / N_e (Fermi-Amaldi; N_e = opts.n_electrons > 0),
 *   v0 = v_x + v_c, v_c the PW92 correlation potential (spin-unpolarised),
 *   v_x the Slater exchange potential (exchange = 0) or the LB94 exchange
 *   potential of the closed-shell density (exchange = 1), with rho = max(
 *   rho_data, 0) and |grad rho| from the finite-element interpolant of rho at
 *   the GLL nodes (at a cell vertex the mean of the two cells' one-sided
 *   derivatives; rho = 0 on the Dirichlet boundary).
 * rho_data, v_H (the Hartree potential of rho_data, the same one that enters
 * v_fixed), v_out: device [L].  tau > 0 (the paper suggests 1e-2); alpha
 * scales the Fermi-Amaldi tail (1 gives -1/r far out).  The LB94 form uses a
 * work vector of the bound workspace: do not run it concurrently with a step
 * of the same handle.  EINVAL for bad arguments or an unbound handle.        */
invdft_status invdft_initial_guess(invdft_handle h, const double *rho_data, const double *v_H,
                                   double tau, double alpha, int exchange, double *v_out,
                                   void *stream);

/* Dense per-cell potential matrices: the Gauss-quadrature reading of the
 * potential term of Eq. 17, V_e[a][b] = sum_g W_g v(x_g) N_a(x_g) N_b(x_g)
 * with 2p Gauss points per axis (exact for the interpolated v), and the
 * operator H~ = D (K + V) D with the lumped GLL mass (orders 2 and 4).
 * invdft_cell_potential_bytes: bytes of the cell-matrix buffer for prec
 *   (FP64: (p+1)^6 doubles per cell, row-major; MIXED: one 128 x 128 FP32
 *   tile per cell in the tensor-core operand layout).
 * invdft_cell_potentials: builds V_e of every cell into Ve (device, caller
 *   owned, the size above) from v_full, the potential on the FULL node grid
 *   including the Dirichlet boundary nodes (device, prod_a (ncell[a] p + 1)
 *   doubles, x fastest).
 * invdft_apply_h_dense: Y = D (K + V) D X for an [L][ncol] block (device;
 *   double for FP64, float for MIXED; Y must not alias X, ncol in [1, 256]):
 *   the kinetic part as in invdft_apply_h without the collocated potential,
 *   then each cell's dense product added in.  The potential set by
 *   invdft_set_potential is not used.
 * EINVAL for bad arguments, an unbound handle or another order.            */
invdft_status invdft_cell_potential_bytes(invdft_handle h, invdft_precision prec, size_t *bytes);
invdft_status invdft_cell_potentials(invdft_handle h, const double *v_full, void *Ve,
                                     invdft_precision prec, void *stream);
invdft_status invdft_apply_h_dense(invdft_handle h, const void *Ve, const void *X, void *Y,
                                   int ncol, invdft_precision prec, void *stream);

/* Linear (Q1) v_xc mesh and field transfer (Sec. 3.1.1, Sec. 3.2.2).  The Q1
 * mesh has nv cells per axis (nv in [1, 4096]) over the handle's box, with
 * values on all (nv+1)^3 nodes (x fastest); T is the matrix of trilinear
 * weights of the Q1 interpolant at the handle's unknown nodes (8 per node).
 * invdft_q1_to_nodes: v_nodes = T v_q1 (the potential seen by the orbitals;
 *   pass it to invdft_set_potential as v_xc).  v_q1 device [(nv+1)^3],
 *   v_nodes device [L].
 * invdft_grad_to_q1: g_q1 = T^T g_nodes, the nodal gradient of Eq. 22 (as
 *   returned by invdft_loss_grad) pulled back to the Q1 coefficients; each Q1
 *   node sums its support in a fixed order (deterministic, no atomics).
 *   g_nodes device [L], g_q1 device [(nv+1)^3].
 * Both are asynchronous on stream; EINVAL for bad arguments.                */
invdft_status invdft_q1_to_nodes(invdft_handle h, int nv, const double *v_q1, double *v_nodes,
                                 void *stream);
invdft_status invdft_grad_to_q1(invdft_handle h, int nv, const double *g_nodes, double *g_q1,
                                void *stream);

/* Forget the L-BFGS history and the warm-start orbitals.                   */
invdft_status invdft_reset(invdft_handle h);

/* Text of the last error on this handle (or of the last create failure if
 * h is NULL).  Valid until the next call on the handle.                     */
const char *invdft_last_error(invdft_handle h);

#ifdef __cplusplus
}
#endif
#endif /* INVDFT_H */
