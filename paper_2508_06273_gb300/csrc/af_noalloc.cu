// af_noalloc.cu -- conserved totals of caller-owned cell averages, computed
// without the library allocating anything.
//
// Who needs this: callers that must not allocate device memory at the point
// of the call.  Examples are a time-stepping loop that cannot afford the
// device-wide synchronisation that cudaFree brings with it, and applications
// whose device memory all belongs to another allocator (a framework's caching
// pool, a fixed arena) that forbids side allocations.  af_conserved_totals
// needs a handle, and creating one allocates the whole grid state; this entry
// point works on arrays the caller already owns and keeps its scratch in a
// fixed static device array instead.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/af.h"
#include "af_kernels.h"

// One FP64 partial sum per grid row and conserved variable.  Every GPU that
// loads the library holds this array (AF_TOTALS_NOALLOC_MAX_ROWS x 4 doubles,
// 512 KiB) until the process exits.  All calls share it, and it keeps the
// last call's contents.
static __device__ __align__(256) double af_totals_scratch[AF_TOTALS_NOALLOC_MAX_ROWS * 4];

namespace {

constexpr int kThreads = 256;

// row j of [4][ny][nx]: a fixed-order sum per thread, then a fixed tree, so
// the result does not depend on scheduling
__global__ void row_sums_kernel(const float *__restrict__ hi, const float *__restrict__ lo, int nx,
                                int ny, double *rows) {
  __shared__ double sm[4][kThreads];
  const int j = blockIdx.x;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < nx; i += kThreads)
    for (int v = 0; v < 4; v++) {
      const long long e = ((long long)v * ny + j) * nx + i;
      acc[v] += (double)hi[e] + (lo ? (double)lo[e] : 0.0);
    }
  for (int v = 0; v < 4; v++) sm[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 4; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) rows[j * 4 + threadIdx.x] = sm[threadIdx.x][0];
}

__global__ void rows_total_kernel(const double *__restrict__ rows, int ny, double cell_area,
                                  double *out) {
  __shared__ double sm[4][kThreads];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int j = threadIdx.x; j < ny; j += kThreads)
    for (int v = 0; v < 4; v++) acc[v] += rows[j * 4 + v];
  for (int v = 0; v < 4; v++) sm[v][threadIdx.x] = acc[v];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int v = 0; v < 4; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[threadIdx.x] = sm[threadIdx.x][0] * cell_area;
}

// Device address of the scratch array, looked up once per device with that
// device current.  In host code the array's name is only a host-side stand-in,
// so kernels must be given this address, never the name.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch[kMaxDevices] = {};

cudaError_t scratch_on(int dev, double **ptr) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch[dev]) {
    int old = -1;
    cudaGetDevice(&old);
    if (old != dev) cudaSetDevice(dev);
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, af_totals_scratch);
    if (old != dev && old >= 0) cudaSetDevice(old);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<double *>(p);
  }
  *ptr = g_scratch[dev];
  return cudaSuccess;
}

// p is memory that kernels on device dev can read and write: device memory
// of that device, or managed memory
bool reachable_on(const void *p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

extern "C" int af_conserved_totals_noalloc(const float *avg, const float *avg_lo, int nx, int ny,
                                           double dx, double dy, double *out, void *stream) {
  char msg[160];
  if (!avg || !out || nx < 1 || ny < 1 || !(dx > 0.0) || !(dy > 0.0))
    return af::set_error(AF_ERR_ARG, "af_conserved_totals_noalloc: null array, empty grid or bad cell size");
  if (ny > AF_TOTALS_NOALLOC_MAX_ROWS) {
    std::snprintf(msg, sizeof(msg),
                  "af_conserved_totals_noalloc: ny = %d exceeds the static scratch limit of %d rows", ny,
                  AF_TOTALS_NOALLOC_MAX_ROWS);
    return af::set_error(AF_ERR_ARG, msg);
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, avg) != cudaSuccess ||
      (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device < 0 ||
      a.device >= kMaxDevices) {
    cudaGetLastError();
    return af::set_error(AF_ERR_ARG, "af_conserved_totals_noalloc: avg must be device memory");
  }
  // the kernels run on avg's device: out and avg_lo must be reachable there
  if (!reachable_on(out, a.device) || (avg_lo && !reachable_on(avg_lo, a.device)))
    return af::set_error(AF_ERR_ARG,
                         "af_conserved_totals_noalloc: out and avg_lo must be device memory on avg's device");
  double *rows = nullptr;
  cudaError_t e = scratch_on(a.device, &rows);
  if (e != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "af_conserved_totals_noalloc: cudaGetSymbolAddress: %s",
                  cudaGetErrorString(e));
    return af::set_error(AF_ERR_CUDA, msg);
  }
  int old = -1;
  cudaGetDevice(&old);
  if (old != a.device) cudaSetDevice(a.device);
  cudaStream_t s = (cudaStream_t)stream;
  row_sums_kernel<<<ny, kThreads, 0, s>>>(avg, avg_lo, nx, ny, rows);
  rows_total_kernel<<<1, kThreads, 0, s>>>(rows, ny, dx * dy, out);
  e = cudaGetLastError();
  if (old != a.device && old >= 0) cudaSetDevice(old);
  if (e != cudaSuccess) {
    std::snprintf(msg, sizeof(msg), "af_conserved_totals_noalloc: launch: %s", cudaGetErrorString(e));
    return af::set_error(AF_ERR_CUDA, msg);
  }
  return AF_OK;
}
