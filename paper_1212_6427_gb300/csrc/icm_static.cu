// Total fluid momentum of a device face field without allocating device memory.
//
// Some callers cannot call cudaMalloc: code running while another thread has a
// stream capture open (allocation is not permitted then), processes in which a
// framework has already reserved nearly all of the GPU's memory for its own pool,
// and latency-critical loops that must not take the device-wide synchronisation
// that cudaMalloc/cudaFree imply.  For them this file provides a variant of the
// library's FP64 compensated field sum (the reduction behind the momentum that
// icm_read_state reports) whose scratch lives in a fixed array in device memory
// that the module itself declares.  Every GPU that loads the library holds that
// array (3 * 16384 + 8 doubles, about 384 KB) until the process exits.
#include <mutex>

#include "../../include/icm.h"
#include "icm_internal.h"

namespace {

constexpr int kStaticPartials = 16384;                 // partial sums per component
constexpr long long kCellsPerPartial = 8192;           // cells reduced by one block
constexpr long long kStaticMaxCells = (long long)kStaticPartials * kCellsPerPartial;  // 512^3
constexpr int kMaxDevices = 64;

// Scratch of the reduction: partial sums [3][kStaticPartials], then 3 results.
// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) double g_momentum_scratch[3 * kStaticPartials + 8];

std::mutex g_lock;
double* g_scratch_dev[kMaxDevices] = {nullptr};

template <typename R>
__global__ void k_static_partial(const R* __restrict__ v, long long ncell, int nblk, double* __restrict__ scratch) {
  const int comp = blockIdx.y, b = blockIdx.x;
  const R* p = v + comp * ncell;
  const long long lo = (long long)b * kCellsPerPartial;
  const long long hi = lo + kCellsPerPartial < ncell ? lo + kCellsPerPartial : ncell;
  double s = 0.0, c = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const double y = (double)p[i] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[comp * kStaticPartials + b] = red[0];
}

__global__ void k_static_final(int nblk, double scale, double* __restrict__ scratch) {
  const int comp = blockIdx.x;
  double s = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    const double y = scratch[comp * kStaticPartials + i] - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) scratch[3 * kStaticPartials + comp] = scale * red[0];
}

icm_status say(icm_status st, const char* msg) { return (icm_status)icm::record_error((int)st, msg); }

// Device address of the scratch array for the current device, looked up once per
// device (the host-side name of a __device__ array is not a device address).  The
// cached address belongs to the device's primary context as it was at the lookup: a
// cudaDeviceReset (or a primary-context reset) in the process unloads the module and
// leaves a stale address behind, so the library must not be used across one.
icm_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return say(ICM_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return say(ICM_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> guard(g_lock);
  if (g_scratch_dev[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_momentum_scratch);
    if (e != cudaSuccess || p == nullptr) return say(ICM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
    g_scratch_dev[dev] = (double*)p;
  }
  *out = g_scratch_dev[dev];
  return ICM_OK;
}

}  // namespace

extern "C" icm_status icm_fluid_momentum_static(const void* fluid_v_dev, int32_t precision, int64_t ncell,
                                                double rho, double h, void* cuda_stream, double momentum[3]) {
  if (!fluid_v_dev || !momentum) return say(ICM_EINVAL, "fluid_v_dev and momentum must not be NULL");
  if (precision != 32 && precision != 64) return say(ICM_EINVAL, "precision must be 32 or 64");
  if (ncell < 1) return say(ICM_EINVAL, "ncell must be >= 1");
  if (ncell > kStaticMaxCells)
    return say(ICM_EINVAL, "ncell exceeds the 134217728 cells (512^3) the static scratch array can reduce");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // The call ends with a copy to the host and a wait, neither of which may enter a
  // graph: refuse a stream that is capturing.  The legacy default stream (NULL) also
  // reports an error here while a blocking stream of the process is capturing.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t ce = cudaStreamIsCapturing(s, &cap);
  if (ce != cudaSuccess) {
    (void)cudaGetLastError();
    return say(ICM_EINVAL, "cuda_stream cannot be used while a capture is open (use a non-blocking stream)");
  }
  if (cap != cudaStreamCaptureStatusNone)
    return say(ICM_EINVAL, "cuda_stream is capturing a graph: pass a stream that is not capturing");
  double* scratch = nullptr;
  const icm_status st = scratch_address(&scratch);
  if (st != ICM_OK) return st;
  const int nblk = (int)((ncell + kCellsPerPartial - 1) / kCellsPerPartial);
  // every partial slot read below is written first, so nothing needs clearing
  if (precision == 32)
    k_static_partial<float><<<dim3(nblk, 3), 256, 0, s>>>((const float*)fluid_v_dev, ncell, nblk, scratch);
  else
    k_static_partial<double><<<dim3(nblk, 3), 256, 0, s>>>((const double*)fluid_v_dev, ncell, nblk, scratch);
  k_static_final<<<3, 256, 0, s>>>(nblk, rho * h * h * h, scratch);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(momentum, scratch + 3 * kStaticPartials, 3 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return say(ICM_ECUDA, cudaGetErrorString(e));
  return ICM_OK;
}
