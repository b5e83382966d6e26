// closure_internal.h -- shapes, parameter-blob layout and device buffers of
// the learned closure (not part of the public C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "internal.h"

namespace mhd {

constexpr int kIn = 24, kInPad = 32, kHid = 64, kOut = 3, kOutPad = 8, kOutPadK = 16;
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
    float *Z1, *Z2, *Y;
    __nv_bfloat16 *H1, *H2;
};

// What the closure step reads (a lattice-owned copy).
struct ClosureParamsDev {
    const __nv_bfloat16 *Wt1, *Wt2, *Wt3;
    const float *b1, *b2, *b3, *mean, *scale, *out_scale;
    int* err;  // set to 1 by the closure step if a tensor-core wait gave up
    // if set, the closure step also stores each node's correction here (3
    // planes of nx*ny floats: xx, xy, yy; node y*nx + x) for the steps that
    // reuse it (launch_step_da_cached)
    float* da_out = nullptr;
};

// The closure step: MLP on warp-level mma.sync fragments (kind 0) or on the
// tcgen05 tensor cores with tensor-memory accumulators (kind 1).
cudaError_t launch_step_closure(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st);
cudaError_t launch_step_closure_tc(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st);
// The fused step with a stored correction da (the layout of da_out) added to
// a1^(2) before the recursion: the steps between two evaluations of the MLP.
cudaError_t launch_step_da_cached(const StepLaunch& s, const float* da, cudaStream_t st);
cudaError_t launch_filter(const Layout& L, int prec, const void* prev, int r, float* out, cudaStream_t st);
cudaError_t launch_sgs(const Layout& L, int prec, const void* prev, int r, double tau_coarse, float* out,
                       cudaStream_t st);
cudaError_t launch_features(const float* state, int nx, int ny, float rho0, float* X, cudaStream_t st);
cudaError_t launch_targets(const float* sT, const float* sT1, int nx, int ny, double rho0, double omega,
                           float* out, cudaStream_t st);
cudaError_t launch_gather_batch(const float* X, const float* T, const int* idx, int nreal, int rows,
                                const float* prm, const MlpDev& d, cudaStream_t st);
cudaError_t launch_refresh(const float* prm, const MlpDev& d, cudaStream_t st);
cudaError_t launch_stats(const float* X, const float* T, long long n, double* P, int nblocks, float* prm,
                         cudaStream_t st);
cudaError_t launch_mlp_predict(const MlpDev& d, int rows, int nreal, const float* prm, float* Yraw,
                               cudaStream_t st);

// One training step (mlp_train.cu): a fused forward / backward / weight-
// gradient kernel over blocks of 128 rows writing per-block partials
// (train_blocks(rows) x kBlob floats in `part`, one loss sum per block in
// `lossp`), then a per-parameter kernel that sums them in block order and
// either applies Adam (adam: step += 1 first; the batch loss is added to
// *loss_acc) or stores the gradient in `grad`.  prepare_train_kernels sets
// the fused kernel's shared-memory size once per device.
int train_blocks(int rows);
// idx[0..n) = this epoch's order of the samples: a bijection of [0, n)
// keyed by seed and *step (the Adam step count when the epoch starts).
cudaError_t launch_epoch_permutation(int* idx, long long n, unsigned long long seed, const long long* step,
                                     cudaStream_t st);
cudaError_t prepare_train_kernels();
cudaError_t launch_train_step(const float* X, const float* T, const int* idx, int nreal, int rows, float* prm,
                              const MlpDev& d, float* part, double* lossp, long long* step, float* grad, float* m,
                              float* v, float lr, double* loss_acc, bool adam, cudaStream_t st);

}  // namespace mhd
