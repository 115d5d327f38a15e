// af_gemm.cu -- BF16 x BF16 -> FP32 matrix product on the tcgen05 tensor
// cores: D (+)= A B^T (+ bias), A (M x K) and B (N x K) row-major BF16.
// Used by the surrogate's training (weight gradients, backward products).
//
// One CTA of 128 threads owns 128 rows of D and all N <= 128 columns; the
// accumulator lives in tensor memory.  K is walked in chunks of 64: the
// threads stage the A and B chunks in shared memory in the K-major core-
// matrix layout (af_tc.cuh), one thread issues the four K = 16 MMAs and
// commits them to an mbarrier, and the chunk buffers are refilled once the
// MMAs have read them.  Split-K over gridDim.y adds partial products into D
// with atomics.
#include "../../include/af.h"
#include "af_kernels.h"
#include "af_tc.cuh"

namespace af {

namespace {

constexpr int GM = 128;  // rows per CTA
constexpr int GN_MAX = 128;
// chunk regions: exact sizes 16 KB (A) and N * 128 bytes (B), each padded to
// 48 KB so that any reading of the two descriptor offsets stays inside
constexpr unsigned REGION = 48 * 1024;
constexpr unsigned GEMM_SMEM = 2 * REGION + 1024;
constexpr unsigned GEMM_WAIT = 1u << 20;

struct GemmArgs {
  const __nv_bfloat16 *A, *B;
  float *D;
  const float *bias;
  int M, N, K, lda, ldb, ldd;
  int atomic;  // add into D
  int *err;
};

// stage rows [row0, row0 + R) x [k0, k0 + 64) of X (ld elements) into dst
__device__ __forceinline__ void stage_chunk(unsigned char *dst, const __nv_bfloat16 *X, int ld, int rows_total,
                                            int row0, int R, int K, int k0) {
  const int nvec = R * 8;
  for (int idx = threadIdx.x; idx < nvec; idx += blockDim.x) {
    const int r = idx >> 3, kv = idx & 7, k = k0 + 8 * kv, row = row0 + r;
    uint4 val = make_uint4(0u, 0u, 0u, 0u);
    if (row < rows_total && k < K) val = *reinterpret_cast<const uint4 *>(X + (long long)row * ld + k);
    *reinterpret_cast<uint4 *>(dst + tc::chunk_offset(R, r, 8 * kv)) = val;
  }
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs a) {
  extern __shared__ __align__(1024) unsigned char gsm[];
  __shared__ alignas(8) unsigned long long bar;
  __shared__ unsigned tslot;
  unsigned char *sA = gsm, *sB = gsm + REGION;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = blockIdx.x * GM;
  const int NP = (a.N + 15) & ~15;  // MMA N
  const unsigned ncols = NP <= 32 ? 32 : (NP <= 64 ? 64 : 128);
  // K chunks of this split
  const int nchunk = (a.K + tc::KCHUNK - 1) / tc::KCHUNK;
  const int per = (nchunk + gridDim.y - 1) / gridDim.y;
  const int c0 = blockIdx.y * per, c1 = min(nchunk, c0 + per);

  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  if (threadIdx.x == 0) tc::bar_init(&bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const unsigned tmem = tslot;
  const uint32_t idesc = tc::make_idesc(GM, NP);
  bool ok = true;
  unsigned phase = 0;
  for (int c = c0; c < c1 && ok; c++) {
    stage_chunk(sA, a.A, a.lda, a.M, row0, GM, a.K, c * tc::KCHUNK);
    stage_chunk(sB, a.B, a.ldb, a.N, 0, NP, a.K, c * tc::KCHUNK);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
      const unsigned ba = tc::smem_u32(sA), bb = tc::smem_u32(sB);
      const unsigned lboA = GM * 16, lboB = NP * 16;
#pragma unroll
      for (int s = 0; s < tc::KCHUNK / 16; s++) {
        const uint64_t da = tc::make_desc(ba + 2 * s * lboA, lboA, 128);
        const uint64_t db = tc::make_desc(bb + 2 * s * lboB, lboB, 128);
        tc::mma_bf16(tmem, da, db, idesc, (c > c0 || s > 0) ? 1 : 0);
      }
      tc::mma_commit(&bar);
    }
    // block-uniform outcome (the tensor-memory loads below are warp-collective)
    ok = __syncthreads_and(tc::bar_wait(&bar, phase, GEMM_WAIT)) != 0;
    phase ^= 1;
  }
  if (!ok) {
    // the MMAs did not complete in time: record it and give them one more
    // bounded wait before the tensor memory is released
    if (threadIdx.x == 0) atomicOr(a.err, 1);
    tc::bar_wait(&bar, phase ^ 1, GEMM_WAIT);
  } else if (c1 > c0) {
    tc::fence_after_sync();
    const int row = row0 + 32 * (warp & 3) + lane;
    for (int cb = 0; cb < a.N; cb += 32) {
      float v[32];
      tc::tmem_ld32(tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)cb, v);
      if (row < a.M) {
        float *d = a.D + (long long)row * a.ldd + cb;
#pragma unroll
        for (int j = 0; j < 32; j++) {
          if (cb + j >= a.N) break;
          float x = v[j];
          if (a.bias && blockIdx.y == 0) x += a.bias[cb + j];
          if (a.atomic) atomicAdd(d + j, x);
          else d[j] = x;
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

__device__ int g_gemm_err;

}  // namespace

int *gemm_default_err() {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_gemm_err) != cudaSuccess) return nullptr;
  return static_cast<int *>(p);
}

cudaError_t prepare_gemm() {
  return cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
}

cudaError_t launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, float *D, int ldd, int M, int N,
                             int K, const float *bias, int splits, int accumulate, int *err, cudaStream_t s) {
  if (M <= 0 || N <= 0 || N > GN_MAX || K <= 0 || (K & 7) || (lda & 7) || (ldb & 7) || lda < K || ldb < K ||
      ldd < N || splits < 1)
    return cudaErrorInvalidValue;
  if ((reinterpret_cast<size_t>(A) & 15) || (reinterpret_cast<size_t>(B) & 15)) return cudaErrorInvalidValue;
  const int nchunk = (K + tc::KCHUNK - 1) / tc::KCHUNK;
  if (splits > nchunk) splits = nchunk;
  const bool atomic = accumulate || splits > 1;
  if (atomic && !accumulate) {
    cudaError_t e = cudaMemset2DAsync(D, (size_t)ldd * sizeof(float), 0, (size_t)N * sizeof(float), M, s);
    if (e != cudaSuccess) return e;
  }
  GemmArgs a;
  a.A = static_cast<const __nv_bfloat16 *>(A);
  a.B = static_cast<const __nv_bfloat16 *>(B);
  a.D = D;
  a.bias = bias;
  a.M = M;
  a.N = N;
  a.K = K;
  a.lda = lda;
  a.ldb = ldb;
  a.ldd = ldd;
  a.atomic = atomic ? 1 : 0;
  a.err = err;
  dim3 grd((M + GM - 1) / GM, splits);
  gemm_bf16_kernel<<<grd, 128, GEMM_SMEM, s>>>(a);
  return cudaGetLastError();
}

}  // namespace af

extern "C" int af_gemm_bf16(const void *A, int lda, const void *B, int ldb, float *D, int ldd, int M, int N, int K,
                            const float *bias, int splits, int accumulate, int *err, void *stream) {
  static bool prepared = false;
  if (!prepared) {
    if (af::prepare_gemm() != cudaSuccess) return af::set_error(AF_ERR_CUDA, "af_gemm_bf16: kernel attributes");
    prepared = true;
  }
  if (!err) err = af::gemm_default_err();
  if (!err) return af::set_error(AF_ERR_CUDA, "af_gemm_bf16: error flag");
  cudaError_t e = af::launch_gemm_bf16(A, lda, B, ldb, D, ldd, M, N, K, bias, splits, accumulate, err,
                                       (cudaStream_t)stream);
  if (e == cudaErrorInvalidValue)
    return af::set_error(AF_ERR_ARG, "af_gemm_bf16: need 0 < N <= 128, K and the leading dimensions multiples "
                                     "of 8, 16-byte aligned A and B");
  if (e != cudaSuccess) return af::set_error(AF_ERR_CUDA, cudaGetErrorString(e));
  return AF_OK;
}
