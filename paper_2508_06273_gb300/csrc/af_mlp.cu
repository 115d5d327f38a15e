// af_mlp.cu -- the surrogate network's parameters and its training on the
// GPU: forward and backward through the tcgen05 BF16 GEMM of af_gemm.cu
// (FP32 accumulation), GELU and loss kernels, and Adam (Kingma & Ba 2015)
// on FP32 master weights.
//
// One training step on a minibatch of B rows (B a multiple of 8):
//   Z1 = X W1^T + b1, H1 = gelu(Z1), ..., Y = H3 W4^T + b4     (forward)
//   dY = 2 (Y - T) / (8 B) on the 8 used outputs                (MSE loss)
//   dW4 = dY^T H3, db4 = sum dY, dH3 = dY W4, dZ3 = dH3 gelu'(Z3)
//   dW3 = dZ3^T H2, ..., dW1 = dZ1^T X                          (backward)
// Every product runs on the tensor cores with K-major operands, so the
// kernels that make H, dY and dZ also write their transposes.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/af.h"
#include "af_kernels.h"
#include "af_mlp.h"

using namespace af;
using namespace af::mlp;

namespace {

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__device__ __forceinline__ float uniform01(uint64_t h) {  // (0, 1]
  return ((float)(h >> 40) + 1.0f) * (1.0f / 16777216.0f);
}

// He-normal weights (Box-Muller on counter-based uniforms), zero biases,
// the last layer scaled by 0.1 and its unused rows zero; unit scales
__global__ void init_kernel(float *p, uint64_t seed) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NPARAM) return;
  float fan = 0.0f, mul = 1.0f;
  bool zero = false;
  if (k < OFF_B1) fan = NIN;
  else if (k < OFF_W2) zero = true;
  else if (k < OFF_B2) fan = NH;
  else if (k < OFF_W3) zero = true;
  else if (k < OFF_B3) fan = NH;
  else if (k < OFF_W4) zero = true;
  else if (k < OFF_B4) {
    fan = NH;
    mul = 0.1f;
    zero = (k - OFF_W4) / NH >= NOUT;
  } else if (k < NTRAIN) zero = true;
  if (k >= NTRAIN) {
    p[k] = 1.0f;
    return;
  }
  if (zero) {
    p[k] = 0.0f;
    return;
  }
  const float u1 = uniform01(mix64(seed ^ (2ull * k))), u2 = uniform01(mix64(seed ^ (2ull * k + 1)));
  const float g = sqrtf(-2.0f * logf(u1)) * cosf(6.283185307f * u2);
  p[k] = g * sqrtf(2.0f / fan) * mul;
}

// BF16 copies of the weights, row-major and transposed
__global__ void refresh_kernel(const float *p, __nv_bfloat16 *wb, __nv_bfloat16 *wbT) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NWB) return;
  int off, rows, cols, base;
  if (k < WB_W2) {
    off = OFF_W1; rows = NH; cols = NIN; base = WB_W1;
  } else if (k < WB_W3) {
    off = OFF_W2; rows = NH; cols = NH; base = WB_W2;
  } else if (k < WB_W4) {
    off = OFF_W3; rows = NH; cols = NH; base = WB_W3;
  } else {
    off = OFF_W4; rows = NOUT_PAD; cols = NH; base = WB_W4;
  }
  const int e = k - base, r = e / cols, c = e % cols;
  const __nv_bfloat16 w = __float2bfloat16_rn(p[off + e]);
  wb[k] = w;
  wbT[base + c * rows + r] = w;
}

// minibatch rows: row r of the batch is sample idx[r] (random when seed != 0,
// else r); features scaled by the input scales into BF16 (and transposed),
// targets divided by the output scales; rows >= nvalid are zero
__global__ void gather_kernel(const float *X, const float *T, int n, int B, int nvalid, uint64_t seed,
                              long long step, const float *p, __nv_bfloat16 *Xb, __nv_bfloat16 *XT, float *Tn) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr;
    float x = 0.0f;
    if (r < nvalid) {
      const long long src = seed ? (long long)(mix64(seed ^ mix64((uint64_t)step * 1315423911ull + r)) % n) : r;
      x = X[src * NIN + c0 + tx] * p[OFF_INS + c0 + tx];
      if (T && blockIdx.y == 0 && tx < NOUT) Tn[(long long)r * NOUT + tx] = T[src * NOUT + tx] / p[OFF_OUTS + tx];
    } else if (T && r < B && blockIdx.y == 0 && tx < NOUT) {
      Tn[(long long)r * NOUT + tx] = 0.0f;
    }
    if (r < B) Xb[(long long)r * NIN + c0 + tx] = __float2bfloat16_rn(x);
    tile[rr][tx] = x;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += blockDim.y) {
    const int r = r0 + tx;
    if (r < B) XT[(long long)(c0 + cc) * B + r] = __float2bfloat16_rn(tile[tx][cc]);
  }
}

// H = gelu(Z) in BF16, and H^T
__global__ void act_kernel(const float *Z, int B, __nv_bfloat16 *H, __nv_bfloat16 *HT) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int rr = ty; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr;
    float h = 0.0f;
    if (r < B) {
      h = gelu(Z[(long long)r * NH + c0 + tx]);
      H[(long long)r * NH + c0 + tx] = __float2bfloat16_rn(h);
    }
    tile[rr][tx] = h;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += blockDim.y) {
    const int r = r0 + tx;
    if (r < B) HT[(long long)(c0 + cc) * B + r] = __float2bfloat16_rn(tile[tx][cc]);
  }
}

// loss and dY = 2 (Y - T) / (8 nvalid) on the used outputs of the valid rows
// (BF16, and transposed), db4 += column sums
__global__ void loss_kernel(const float *Y, const float *Tn, int B, int nvalid, __nv_bfloat16 *dYb,
                            __nv_bfloat16 *dYT, float *db4, double *loss) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  float d[NOUT_PAD];
  float l = 0.0f;
#pragma unroll
  for (int k = 0; k < NOUT_PAD; k++) d[k] = 0.0f;
  if (r < nvalid) {
#pragma unroll
    for (int k = 0; k < NOUT; k++) {
      const float e = Y[(long long)r * NOUT_PAD + k] - Tn[(long long)r * NOUT + k];
      l += e * e;
      d[k] = 2.0f * e / (float)(NOUT * (long long)nvalid);
    }
  }
  if (r < B) {
#pragma unroll
    for (int k = 0; k < NOUT_PAD; k++) {
      const __nv_bfloat16 b = __float2bfloat16_rn(d[k]);
      dYb[(long long)r * NOUT_PAD + k] = b;
      dYT[(long long)k * B + r] = b;
    }
  }
  // block sums of the loss and of d (FP32 gradient of b4)
  __shared__ float sl[256];
  __shared__ float sd[NOUT][256];
  sl[threadIdx.x] = l;
#pragma unroll
  for (int k = 0; k < NOUT; k++) sd[k][threadIdx.x] = d[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sl[threadIdx.x] += sl[threadIdx.x + s];
#pragma unroll
      for (int k = 0; k < NOUT; k++) sd[k][threadIdx.x] += sd[k][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, (double)sl[0] / (double)(NOUT * (long long)nvalid));
  if (threadIdx.x < NOUT) atomicAdd(db4 + threadIdx.x, sd[threadIdx.x][0]);
}

// dZ = dH gelu'(Z) (BF16, and transposed); db += column sums
__global__ void dz_kernel(const float *dH, const float *Z, int B, __nv_bfloat16 *dZb, __nv_bfloat16 *dZT,
                          float *db) {
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  float colsum = 0.0f;
  for (int rr = ty; rr < 32; rr += blockDim.y) {
    const int r = r0 + rr;
    float g = 0.0f;
    if (r < B) {
      const long long e = (long long)r * NH + c0 + tx;
      g = dH[e] * gelu_grad(Z[e]);
      dZb[e] = __float2bfloat16_rn(g);
    }
    tile[rr][tx] = g;
    colsum += g;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += blockDim.y) {
    const int r = r0 + tx;
    if (r < B) dZT[(long long)(c0 + cc) * B + r] = __float2bfloat16_rn(tile[tx][cc]);
  }
  atomicAdd(db + c0 + tx, colsum);
}

// the 8 used outputs of each row times the output scales
__global__ void out_kernel(const float *Y, const float *p, int n, float *out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
#pragma unroll
  for (int k = 0; k < NOUT; k++) out[(long long)r * NOUT + k] = Y[(long long)r * NOUT_PAD + k] * p[OFF_OUTS + k];
}

__global__ void adam_kernel(float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= NTRAIN) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.0f - b1) * gk;
  const float vk = b2 * v[k] + (1.0f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// root mean square of each column of a row-major (n x cols) array
__global__ void colrms_kernel(const float *A, long long n, int cols, double *out) {
  const int c = blockIdx.y;
  double s = 0.0;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    const double a = A[r * cols + c];
    s += a * a;
  }
  __shared__ double sm[256];
  sm[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sm[threadIdx.x] += sm[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out + c, sm[0]);
}

int mfail(int code, const char *msg) { return set_error(code, msg); }
int mcuda(cudaError_t e, const char *where) {
  char m[400];
  std::snprintf(m, sizeof(m), "%s: %s", where, cudaGetErrorString(e));
  return set_error(AF_ERR_CUDA, m);
}
#define MCK(call, where)                              \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return mcuda(e_, where);   \
  } while (0)

struct MDev {
  int old = -1;
  explicit MDev(int d) {
    if (cudaGetDevice(&old) == cudaSuccess && old != d) cudaSetDevice(d);
    else old = -1;
  }
  ~MDev() {
    if (old >= 0) cudaSetDevice(old);
  }
};

int refresh(af_mlp *m, cudaStream_t s) {
  refresh_kernel<<<(NWB + 255) / 256, 256, 0, s>>>(m->params, m->wb, m->wbT);
  MCK(cudaGetLastError(), "af_mlp: refresh");
  return AF_OK;
}

// training scratch for B rows (B a multiple of 8)
int ensure_cap(af_mlp *m, int B) {
  if (m->cap >= B) return AF_OK;
  if (m->scratch) cudaFree(m->scratch);
  m->scratch = nullptr;
  m->cap = 0;
  const size_t b16 = sizeof(__nv_bfloat16), f32 = sizeof(float);
  const size_t sizes[] = {
      (size_t)B * NIN * b16,       (size_t)B * NIN * b16,                 // Xb, XT
      3 * (size_t)B * NH * b16,    3 * (size_t)B * NH * b16,              // H, HT
      (size_t)B * NH * b16,        (size_t)B * NH * b16,                  // dZb, dZT
      (size_t)B * NOUT_PAD * b16,  (size_t)B * NOUT_PAD * b16,            // dYb, dYT
      (size_t)B * NOUT * f32,      3 * (size_t)B * NH * f32,              // Tn, Z
      (size_t)B * NOUT_PAD * f32,  (size_t)B * NH * f32, 64};             // Y, dH, loss + flags
  size_t total = 0;
  for (size_t z : sizes) total += (z + 255) & ~size_t(255);
  MCK(cudaMalloc(&m->scratch, total), "af_mlp: cudaMalloc(scratch)");
  char *q = (char *)m->scratch;
  auto take = [&](size_t z) {
    char *r = q;
    q += (z + 255) & ~size_t(255);
    return r;
  };
  m->Xb = (__nv_bfloat16 *)take(sizes[0]);
  m->XT = (__nv_bfloat16 *)take(sizes[1]);
  char *h = take(sizes[2]), *ht = take(sizes[3]);
  for (int k = 0; k < 3; k++) {
    m->H[k] = (__nv_bfloat16 *)h + (size_t)k * B * NH;
    m->HT[k] = (__nv_bfloat16 *)ht + (size_t)k * B * NH;
  }
  m->dZb = (__nv_bfloat16 *)take(sizes[4]);
  m->dZT = (__nv_bfloat16 *)take(sizes[5]);
  m->dYb = (__nv_bfloat16 *)take(sizes[6]);
  m->dYT = (__nv_bfloat16 *)take(sizes[7]);
  m->Tn = (float *)take(sizes[8]);
  float *z = (float *)take(sizes[9]);
  for (int k = 0; k < 3; k++) m->Z[k] = z + (size_t)k * B * NH;
  m->Y = (float *)take(sizes[10]);
  m->dH = (float *)take(sizes[11]);
  char *tail = take(sizes[12]);
  m->loss = (double *)tail;
  m->err = (int *)(tail + 8);
  m->flag = (unsigned *)(tail + 16);
  m->cap = B;
  return AF_OK;
}

int gemm(const void *A, int lda, const void *B, int ldb, float *D, int ldd, int M, int N, int K, const float *bias,
         int splits, int *err, cudaStream_t s) {
  MCK(launch_gemm_bf16(A, lda, B, ldb, D, ldd, M, N, K, bias, splits, 0, err, s), "af_mlp: gemm");
  return AF_OK;
}

// forward of B rows already gathered into Xb / XT; Y = outputs (B x 16)
int forward(af_mlp *m, int B, cudaStream_t s) {
  const dim3 blk(32, 8), grd((B + 31) / 32, NH / 32);
  const __nv_bfloat16 *in = m->Xb;
  int K = NIN;
  const int offw[3] = {WB_W1, WB_W2, WB_W3}, offb[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 0; l < 3; l++) {
    int rc = gemm(in, K, m->wb + offw[l], K, m->Z[l], NH, B, NH, K, m->params + offb[l], 1, m->err, s);
    if (rc) return rc;
    act_kernel<<<grd, blk, 0, s>>>(m->Z[l], B, m->H[l], m->HT[l]);
    MCK(cudaGetLastError(), "af_mlp: act");
    in = m->H[l];
    K = NH;
  }
  return gemm(m->H[2], NH, m->wb + WB_W4, NH, m->Y, NOUT_PAD, B, NOUT_PAD, NH, m->params + OFF_B4, 1, m->err, s);
}

// gradient of the loss of the B gathered rows (nvalid of them real) into m->grads
int backward(af_mlp *m, int B, int nvalid, cudaStream_t s) {
  float *g = m->grads;
  MCK(cudaMemsetAsync(g, 0, sizeof(float) * NTRAIN, s), "af_mlp: memset");
  loss_kernel<<<(B + 255) / 256, 256, 0, s>>>(m->Y, m->Tn, B, nvalid, m->dYb, m->dYT, g + OFF_B4, m->loss);
  MCK(cudaGetLastError(), "af_mlp: loss");
  const int splits = B / 512 > 1 ? B / 512 : 1;
  // layer 4
  int rc = gemm(m->dYT, B, m->HT[2], B, g + OFF_W4, NH, NOUT_PAD, NH, B, nullptr, splits, m->err, s);
  if (rc) return rc;
  rc = gemm(m->dYb, NOUT_PAD, m->wbT + WB_W4, NOUT_PAD, m->dH, NH, B, NH, NOUT_PAD, nullptr, 1, m->err, s);
  if (rc) return rc;
  const dim3 blk(32, 8), grd((B + 31) / 32, NH / 32);
  const int offw[3] = {WB_W1, WB_W2, WB_W3}, offW[3] = {OFF_W1, OFF_W2, OFF_W3}, offb[3] = {OFF_B1, OFF_B2, OFF_B3};
  for (int l = 2; l >= 0; l--) {
    dz_kernel<<<grd, blk, 0, s>>>(m->dH, m->Z[l], B, m->dZb, m->dZT, g + offb[l]);
    MCK(cudaGetLastError(), "af_mlp: dz");
    const __nv_bfloat16 *inT = l > 0 ? m->HT[l - 1] : m->XT;
    const int nin = l > 0 ? NH : NIN;
    rc = gemm(m->dZT, B, inT, B, g + offW[l], nin, NH, nin, B, nullptr, splits, m->err, s);
    if (rc) return rc;
    if (l > 0) {
      // dH_{l-1} = dZ_l W_l: B operand W_l^T (in x out), K = out
      rc = gemm(m->dZb, NH, m->wbT + offw[l], NH, m->dH, NH, B, NH, NH, nullptr, 1, m->err, s);
      if (rc) return rc;
    }
  }
  return AF_OK;
}

int gather(af_mlp *m, const float *X, const float *T, int n, int B, int nvalid, uint64_t seed, long long step,
           cudaStream_t s) {
  gather_kernel<<<dim3((B + 31) / 32, NIN / 32), dim3(32, 8), 0, s>>>(X, T, n, B, nvalid, seed, step, m->params,
                                                                     m->Xb, m->XT, m->Tn);
  MCK(cudaGetLastError(), "af_mlp: gather");
  return AF_OK;
}

int check_err(af_mlp *m, cudaStream_t s) {
  int e = 0;
  MCK(cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, s), "af_mlp: err");
  MCK(cudaStreamSynchronize(s), "af_mlp: sync");
  if (e) return mfail(AF_ERR_CUDA, "af_mlp: a tensor-core wait timed out");
  return AF_OK;
}

void free_mlp(af_mlp *m) {
  cudaFree(m->params);
  cudaFree(m->grads);
  cudaFree(m->adam_m);
  cudaFree(m->adam_v);
  cudaFree(m->wb);
  cudaFree(m->wbT);
  if (m->scratch) cudaFree(m->scratch);
  delete m;
}

}  // namespace

extern "C" {

af_mlp *af_mlp_create(uint64_t seed) {
  af_mlp *m = new (std::nothrow) af_mlp();
  if (!m) {
    mfail(AF_ERR_ALLOC, "af_mlp_create: out of host memory");
    return nullptr;
  }
  cudaGetDevice(&m->device);
  cudaError_t e = prepare_gemm();
  if (e == cudaSuccess) e = cudaMalloc(&m->params, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMalloc(&m->grads, sizeof(float) * NTRAIN);
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_m, sizeof(float) * NTRAIN);
  if (e == cudaSuccess) e = cudaMalloc(&m->adam_v, sizeof(float) * NTRAIN);
  if (e == cudaSuccess) e = cudaMalloc(&m->wb, sizeof(__nv_bfloat16) * NWB);
  if (e == cudaSuccess) e = cudaMalloc(&m->wbT, sizeof(__nv_bfloat16) * NWB);
  if (e == cudaSuccess) e = cudaMemset(m->adam_m, 0, sizeof(float) * NTRAIN);
  if (e == cudaSuccess) e = cudaMemset(m->adam_v, 0, sizeof(float) * NTRAIN);
  if (e != cudaSuccess) {
    mcuda(e, "af_mlp_create");
    free_mlp(m);
    return nullptr;
  }
  init_kernel<<<(NPARAM + 255) / 256, 256>>>(m->params, seed);
  if (refresh(m, nullptr) != AF_OK || cudaDeviceSynchronize() != cudaSuccess) {
    free_mlp(m);
    return nullptr;
  }
  return m;
}

void af_mlp_destroy(af_mlp *m) {
  if (!m) return;
  MDev d(m->device);
  cudaDeviceSynchronize();
  free_mlp(m);
}

int af_mlp_set_params(af_mlp *m, const float *host) {
  if (!m || !host) return mfail(AF_ERR_ARG, "af_mlp_set_params: null argument");
  MDev d(m->device);
  MCK(cudaMemcpy(m->params, host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice), "af_mlp_set_params");
  MCK(cudaMemset(m->adam_m, 0, sizeof(float) * NTRAIN), "af_mlp_set_params");
  MCK(cudaMemset(m->adam_v, 0, sizeof(float) * NTRAIN), "af_mlp_set_params");
  m->adam_t = 0;
  int rc = refresh(m, nullptr);
  if (rc) return rc;
  MCK(cudaDeviceSynchronize(), "af_mlp_set_params");
  return AF_OK;
}

int af_mlp_get_params(af_mlp *m, float *host) {
  if (!m || !host) return mfail(AF_ERR_ARG, "af_mlp_get_params: null argument");
  MDev d(m->device);
  MCK(cudaDeviceSynchronize(), "af_mlp_get_params");
  MCK(cudaMemcpy(host, m->params, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost), "af_mlp_get_params");
  return AF_OK;
}

int af_mlp_fit_scales(af_mlp *m, const float *X, const float *T, long long n) {
  if (!m || !X || !T || n <= 0) return mfail(AF_ERR_ARG, "af_mlp_fit_scales: bad arguments");
  MDev d(m->device);
  double *acc = nullptr;
  MCK(cudaMalloc(&acc, sizeof(double) * (NIN + NOUT)), "af_mlp_fit_scales");
  cudaMemset(acc, 0, sizeof(double) * (NIN + NOUT));
  colrms_kernel<<<dim3(64, NIN), 256>>>(X, n, NIN, acc);
  colrms_kernel<<<dim3(64, NOUT), 256>>>(T, n, NOUT, acc + NIN);
  double h[NIN + NOUT];
  cudaError_t e = cudaMemcpy(h, acc, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(acc);
  MCK(e, "af_mlp_fit_scales");
  float sc[NIN + NOUT];
  for (int k = 0; k < NIN; k++) {
    const double r = std::sqrt(h[k] / (double)n);
    sc[k] = r > 1e-12 ? (float)(1.0 / r) : 0.0f;  // an input that is always 0 stays 0
  }
  for (int k = 0; k < NOUT; k++) {
    const double r = std::sqrt(h[NIN + k] / (double)n);
    sc[NIN + k] = r > 1e-30 ? (float)r : 1.0f;
  }
  MCK(cudaMemcpy(m->params + OFF_INS, sc, sizeof(sc), cudaMemcpyHostToDevice), "af_mlp_fit_scales");
  return AF_OK;
}

int af_mlp_forward(af_mlp *m, const float *X, float *Y, int n, void *stream) {
  if (!m || !X || !Y || n <= 0) return mfail(AF_ERR_ARG, "af_mlp_forward: bad arguments");
  MDev d(m->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int B = (n + 7) & ~7;
  int rc = ensure_cap(m, B);
  if (rc) return rc;
  MCK(cudaMemsetAsync(m->err, 0, sizeof(int), s), "af_mlp_forward");
  rc = gather(m, X, nullptr, n, B, n, 0, 0, s);
  if (rc) return rc;
  rc = forward(m, B, s);
  if (rc) return rc;
  out_kernel<<<(n + 255) / 256, 256, 0, s>>>(m->Y, m->params, n, Y);
  MCK(cudaGetLastError(), "af_mlp_forward");
  return check_err(m, s);
}

int af_mlp_loss_grad(af_mlp *m, const float *X, const float *T, int n, double *loss, float *grads) {
  if (!m || !X || !T || n <= 0) return mfail(AF_ERR_ARG, "af_mlp_loss_grad: bad arguments");
  MDev d(m->device);
  cudaStream_t s = nullptr;
  const int B = (n + 7) & ~7;
  int rc = ensure_cap(m, B);
  if (rc) return rc;
  MCK(cudaMemsetAsync(m->err, 0, sizeof(int), s), "af_mlp_loss_grad");
  MCK(cudaMemsetAsync(m->loss, 0, sizeof(double), s), "af_mlp_loss_grad");
  if ((rc = gather(m, X, T, n, B, n, 0, 0, s)) || (rc = forward(m, B, s)) || (rc = backward(m, B, n, s))) return rc;
  if ((rc = check_err(m, s))) return rc;
  if (loss) MCK(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost), "af_mlp_loss_grad");
  if (grads) MCK(cudaMemcpy(grads, m->grads, sizeof(float) * NTRAIN, cudaMemcpyDeviceToHost), "af_mlp_loss_grad");
  return AF_OK;
}

int af_mlp_train(af_mlp *m, const float *X, const float *T, long long n, int steps, int batch, double lr,
                 uint64_t seed, float *loss_hist) {
  if (!m || !X || !T || n <= 0 || steps < 0 || batch < 8 || (batch & 7) || !(lr > 0) || seed == 0)
    return mfail(AF_ERR_ARG, "af_mlp_train: bad arguments (batch a multiple of 8, lr > 0, seed != 0)");
  MDev d(m->device);
  cudaStream_t s = nullptr;
  int rc = ensure_cap(m, batch);
  if (rc) return rc;
  double *lh = nullptr;
  MCK(cudaMalloc(&lh, sizeof(double) * (steps > 0 ? steps : 1)), "af_mlp_train");
  MCK(cudaMemsetAsync(m->err, 0, sizeof(int), s), "af_mlp_train");
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int k = 0; k < steps && rc == AF_OK; k++) {
    m->adam_t += 1;
    const float c1 = 1.0f - std::pow(b1, (float)m->adam_t), c2 = 1.0f - std::pow(b2, (float)m->adam_t);
    cudaMemsetAsync(m->loss, 0, sizeof(double), s);
    if ((rc = gather(m, X, T, (int)(n > 0x7fffffff ? 0x7fffffff : n), batch, batch, seed, m->adam_t, s)) ||
        (rc = forward(m, batch, s)) || (rc = backward(m, batch, batch, s)))
      break;
    adam_kernel<<<(NTRAIN + 255) / 256, 256, 0, s>>>(m->params, m->grads, m->adam_m, m->adam_v, (float)lr, b1, b2,
                                                     eps, c1, c2);
    if ((rc = refresh(m, s))) break;
    cudaMemcpyAsync(lh + k, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, s);
  }
  if (rc == AF_OK) rc = check_err(m, s);
  if (rc == AF_OK && loss_hist && steps > 0) {
    std::vector<double> h(steps);
    cudaError_t e = cudaMemcpy(h.data(), lh, sizeof(double) * steps, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = mcuda(e, "af_mlp_train");
    for (int k = 0; k < steps; k++) loss_hist[k] = (float)h[k];
  }
  cudaFree(lh);
  return rc;
}

}  // extern "C"
