// Allocation-free variant of the loss reduction, for callers that cannot
// allocate device memory (see invdft_loss_reduce_noalloc in include/invdft.h).
//
// The per-block partial sums live in a file-scope device array instead of a
// caller workspace.  Host code never passes the array's name to a kernel (on
// the host that name is only a stand-in, not a device address): the device
// address is looked up once per device with cudaGetSymbolAddress and cached.
#include <mutex>

#include "internal.h"

namespace invdft {
void set_global_error(const char *msg);

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocNodesPerBlock = 4096;          // nodes summed by one block
constexpr int kNoAllocMaxBlocks = 8192;              // scratch rows
constexpr long long kNoAllocMaxNodes =
    (long long)kNoAllocMaxBlocks * kNoAllocNodesPerBlock;   // 33,554,432 nodes
constexpr int kMaxDevices = 64;

// 8192 x 3 doubles = 192 KiB, held by every GPU that loads the library.
static __device__ __align__(256) double g_loss_scratch[kNoAllocMaxBlocks * 3];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

__global__ void __launch_bounds__(kNoAllocThreads)
loss_blocks(const double *__restrict__ rho, const double *__restrict__ rd,
            const double *__restrict__ w, const double *__restrict__ mass, long long L,
            double *__restrict__ partial, double *__restrict__ dLdrho) {
  __shared__ double red[3][kNoAllocThreads / 32];
  const long long a0 = (long long)blockIdx.x * kNoAllocNodesPerBlock;
  const long long a1 = a0 + kNoAllocNodesPerBlock < L ? a0 + kNoAllocNodesPerBlock : L;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long a = a0 + threadIdx.x; a < a1; a += kNoAllocThreads) {
    const double m = mass[a], d = rd[a] - rho[a], ww = w ? w[a] : 1.0;
    s0 += m * ww * d * d;
    s1 += m * d * d;
    s2 += m * rho[a];
    if (dLdrho) dLdrho[a] = -2.0 * m * ww * d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[0][warp] = s0;
    red[1][warp] = s1;
    red[2][warp] = s2;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int k = 0; k < kNoAllocThreads / 32; ++k) t += red[threadIdx.x][k];
    partial[3 * (size_t)blockIdx.x + threadIdx.x] = t;    // every used row is rewritten
  }
}

__global__ void loss_finish(const double *__restrict__ partial, int nblk,
                            double *__restrict__ out3) {
  const int k = threadIdx.x;
  if (k >= 3) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[3 * (size_t)b + k];
  out3[k] = s;
}

// Device address of the scratch array on the current device (set up once).
cudaError_t scratch_for_current_device(double **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double *>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace invdft

using namespace invdft;

extern "C" invdft_status invdft_loss_reduce_noalloc(const double *rho, const double *rho_data,
                                                    const double *w, const double *mass,
                                                    long long L, double *out3, double *dLdrho,
                                                    void *stream) {
  if (!rho || !rho_data || !mass || !out3 || L < 1) {
    set_global_error("loss_reduce_noalloc: null array or L < 1");
    return INVDFT_EINVAL;
  }
  if (L > kNoAllocMaxNodes) {
    set_global_error("loss_reduce_noalloc: L exceeds the fixed scratch limit of 33,554,432 "
                     "nodes; use invdft_loss_grad with a workspace instead");
    return INVDFT_EINVAL;
  }
  double *scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return INVDFT_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nblk = (int)((L + kNoAllocNodesPerBlock - 1) / kNoAllocNodesPerBlock);
  count_launch();
  loss_blocks<<<nblk, kNoAllocThreads, 0, s>>>(rho, rho_data, w, mass, L, scratch, dLdrho);
  count_launch();
  loss_finish<<<1, 32, 0, s>>>(scratch, nblk, out3);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_global_error(cudaGetErrorString(e));
    return INVDFT_ECUDA;
  }
  return INVDFT_OK;
}
