// af_mlp.h -- the surrogate network: parameter layout and the device-side
// handle shared by its training (af_mlp.cu) and its fused inference
// (af_surrogate.cu).
//
// Network: 64 inputs -> 128 -> 128 -> 128 -> 16 outputs (the first 8 used),
// GELU (tanh form) on the hidden layers.  Inputs are multiplied by a fixed
// per-input scale before the first layer and the outputs by a per-output
// scale after the last one (both fitted to the training data, not trained).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace af {
namespace mlp {

constexpr int NIN = 64, NH = 128, NOUT = 8, NOUT_PAD = 16;
// packed FP32 parameters: W (out x in, row-major) then b, per layer, then
// the input and output scales
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH * NH;
constexpr int OFF_W4 = OFF_B3 + NH;
constexpr int OFF_B4 = OFF_W4 + NOUT_PAD * NH;
constexpr int NTRAIN = OFF_B4 + NOUT_PAD;  // trained parameters
constexpr int OFF_INS = NTRAIN;
constexpr int OFF_OUTS = OFF_INS + NIN;
constexpr int NPARAM = OFF_OUTS + NOUT;
// BF16 weight copies, row-major (out x in), packed in layer order
constexpr int WB_W1 = 0, WB_W2 = WB_W1 + NH * NIN, WB_W3 = WB_W2 + NH * NH, WB_W4 = WB_W3 + NH * NH;
constexpr int NWB = WB_W4 + NOUT_PAD * NH;

// tanh form of GELU and its derivative; tanh from the hardware approximation
__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float GELU_K = 0.7978845608028654f;  // sqrt(2/pi)
constexpr float GELU_C = 0.044715f;
__device__ __forceinline__ float gelu(float z) {
  const float t = tanh_approx(GELU_K * fmaf(GELU_C * z * z, z, z));
  return 0.5f * z * (1.0f + t);
}
__device__ __forceinline__ float gelu_grad(float z) {
  const float t = tanh_approx(GELU_K * fmaf(GELU_C * z * z, z, z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * GELU_K * fmaf(3.0f * GELU_C, z * z, 1.0f);
}

}  // namespace mlp
}  // namespace af

// the handle behind af_mlp* (include/af.h)
struct af_mlp {
  int device = 0;
  float *params = nullptr;  // NPARAM
  float *grads = nullptr;   // NTRAIN
  float *adam_m = nullptr, *adam_v = nullptr;
  __nv_bfloat16 *wb = nullptr;   // NWB, row-major weights
  __nv_bfloat16 *wbT = nullptr;  // NWB, transposed weights (in x out)
  long long adam_t = 0;
  // training scratch for up to `cap` rows
  int cap = 0;
  void *scratch = nullptr;
  __nv_bfloat16 *Xb, *XT, *H[3], *HT[3], *dZb, *dZT, *dYb, *dYT;
  float *Tn, *Z[3], *Y, *dH;
  double *loss;
  int *err;
  unsigned *flag;
};
