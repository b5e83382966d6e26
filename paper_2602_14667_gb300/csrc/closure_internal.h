// closure_internal.h -- shapes, parameter-blob layout and device buffers of
// the learned closure (not part of the public C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace mhd {

constexpr int kIn = 24, kInPad = 32, kHid = 64, kOut = 3, kOutPad = 8, kOutPadK = 16;
constexpr int kMaxWgradBlocks = 256;  // per-block partials of a weight gradient
// Flat FP32 parameter blob: mean[24] scale[24] out_scale[3] W1[24][64] b1[64]
// W2[64][64] b2[64] W3[64][3] b3[3]  (weights input-major, W[in][out]).
constexpr int kOffMean = 0, kOffScale = kOffMean + kIn, kOffOutScale = kOffScale + kIn;
constexpr int kOffW1 = kOffOutScale + kOut, kOffB1 = kOffW1 + kIn * kHid;
constexpr int kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kOut;
constexpr int kBlob = kOffB3 + kOut;  // 6006

// BF16 weights in both layouts (output-major for the forward pass,
// input-major for the backward pass), padded FP32 biases, and the per-batch
// work buffers of training.
struct MlpDev {
    __nv_bfloat16 *Wt1, *W1, *Wt2, *W2, *Wt3, *W3;
    float *b1, *b2, *b3;
    __nv_bfloat16* xb;
    float* tb;
    float *Z1, *Z2, *Y, *dYf, *dH2f, *dH1f;
    __nv_bfloat16 *H1, *H2, *dYb, *dH2b, *dH1b;
    float *part, *gW1, *gb1, *gW2, *gb2, *gW3, *gb3;
};

// What the closure step reads (a lattice-owned copy).
struct ClosureParamsDev {
    const __nv_bfloat16 *Wt1, *Wt2, *Wt3;
    const float *b1, *b2, *b3, *mean, *scale, *out_scale;
    int* err;  // set to 1 by the closure step if a tensor-core wait gave up
};

// The closure step: MLP on warp-level mma.sync fragments (kind 0) or on the
// tcgen05 tensor cores with tensor-memory accumulators (kind 1).
cudaError_t launch_step_closure(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st);
cudaError_t launch_step_closure_tc(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st);
cudaError_t launch_filter(const Layout& L, int prec, const void* prev, int r, float* out, cudaStream_t st);
cudaError_t launch_sgs(const Layout& L, int prec, const void* prev, int r, double tau_coarse, float* out,
                       cudaStream_t st);
cudaError_t launch_features(const float* state, int nx, int ny, float rho0, float* X, cudaStream_t st);
cudaError_t launch_targets(const float* sT, const float* sT1, int nx, int ny, double rho0, double omega,
                           float* out, cudaStream_t st);
cudaError_t mlp_forward_backward(const MlpDev& d, const float* prm, int rows, int nreal, bool backward,
                                 float* grad, double* lossp, int lossblocks, cudaStream_t st);
cudaError_t launch_gather_batch(const float* X, const float* T, const int* idx, int nreal, int rows,
                                const float* prm, const MlpDev& d, cudaStream_t st);
cudaError_t launch_refresh(const float* prm, const MlpDev& d, cudaStream_t st);
// Adam with the step count in device memory; then t += 1 and the batch's
// loss partials added to *acc (one thread, fixed order)
cudaError_t launch_adam_dev(float* prm, const float* grad, float* m, float* v, float lr, float b1, float b2,
                            float eps, const long long* t, cudaStream_t st);
cudaError_t launch_tick(long long* t, const double* lossp, int nb, double* acc, cudaStream_t st);
cudaError_t launch_stats(const float* X, const float* T, long long n, double* P, int nblocks, float* prm,
                         cudaStream_t st);
cudaError_t launch_mlp_predict(const MlpDev& d, int rows, int nreal, const float* prm, float* Yraw,
                               cudaStream_t st);

}  // namespace mhd
