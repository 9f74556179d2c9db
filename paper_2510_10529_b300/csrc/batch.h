// Batched multi-problem execution (batch.cu: kernel; batch_api.cu: host).
#pragma once

#include "internal.h"

namespace invdft {

constexpr int kMaxBatchDeg = 64;     // Chebyshev degree of a batched filter
constexpr int kMaxBatch = 64;        // problems in one batch

// One problem of a batched Chebyshev filter (device copy, built per launch).
struct BatchProb {
  int ncell, Ni, p, ncol;
  int C, nchunk, items, item0;       // column chunk, items per phase, offset in a phase
  float *buf[3];                     // D_k lives in buf[(k - 1) % 3]
  const float *E;                    // FP32 defect block E = H~X - X Lambda
  const float *v;                    // FP32 potential
  const float *dm1f;                 // [Ni + 2] m^-1/2 along an axis
  const int *perm;                   // cell visiting order (or null)
  const double *pk;                  // [m + 1][ncol] p_k(theta_j)
  float shift, kc;
  float tab[52];                     // even/odd blocks of A and B: eA, oA, eB, oB
  float alpha[kMaxBatchDeg + 1], beta[kMaxBatchDeg + 1];
};

size_t batch_filter_smem();
cudaError_t batch_filter_occupancy(int *per_sm);
cudaError_t launch_batch_filter(const BatchProb *d_probs, int nprob, int m, int per_phase,
                                int *queue, unsigned *done, int *err, int grid, cudaStream_t s);

// Fills the fields of a BatchProb that depend only on the problem (mesh,
// buffers, tables); C, item counts and the per-pass scalars are set later.
void batch_prob_static(const Ctx *c, BatchProb *bp);

// Chebyshev degree of the batch a problem belongs to (0 if none).
int batch_degree(const Ctx *c);

// Hands the defect-corrected filter of a problem taking part in a batch step
// to the batch (D_1 formed, outputs zeroed and p_k pushed on stream s), and
// returns once the batched launch is queued; s then waits for it.
invdft_status batch_filter_submit(Ctx *c, int m, const double *alpha, const double *beta,
                                  double shift, cudaStream_t s);

}  // namespace invdft
