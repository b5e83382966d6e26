// closure.cu -- learned sub-grid closure for coarse lattices: data
// generation (box filter, features, one-step targets) and the BF16
// tensor-core MLP's layer-by-layer prediction.  The closure step itself
// (closure_rows.cu, closure_tc.cu) evaluates the MLP per node and adds its
// output to the projected a1^(2) before the recursion (task 3 of the
// paper's "Algorithm of computation"); training is in mlp_train.cu.  The
// closure is not part of the paper.
//
// MLP: 24 -> 64 -> 64 -> 3, ReLU, y = out_scale * (W3 h2 + b3) with
// h1 = relu(W1 xn + b1), h2 = relu(W2 h1 + b2), xn = (x - mean) * scale.
// All products run on mma.sync.m16n8k16 BF16 with FP32 accumulation; the
// layer input (features, activations, output gradients) and the weights are
// rounded to BF16 (round to nearest even), everything else is FP32.
//
// Feature columns (per node, from the pre-collision state):
//   0 rho - rho0, 1 u_x, 2 u_y, 3 b_x, 4 b_y, 5..7 a1^(2) xx, xy, yy,
//   then for q in (u_x, u_y, b_x, b_y): d_x q, d_y q (isotropic lattice
//   gradient), the 9-point lattice Laplacian, d_xy q   (8 + 16 = 24).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "closure_internal.h"
#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"
#include "closure_device.cuh"

namespace mhd {

// ---- data generation ---------------------------------------------------------
// Box filter of the fine pre-collision populations (gathered from the buffer
// the last step read) into a packed coarse state (FP32 deviations).
template <int PREC>
__global__ void filter_kernel(const void* prev, Layout L, int r, float* out) {
    using S = typename Prec<PREC>::S;
    const int ncx = L.nx / r, ncy = L.ny / r;
    const long long nc = (long long)ncx * ncy;
    const float inv = 1.0f / (float)(r * r);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nc;
         k += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(k % ncx), Y = (int)(k / ncx);
        float acc[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) acc[p] = 0.0f;
        for (int dy = 0; dy < r; ++dy)
            for (int dx = 0; dx < r; ++dx) {
                float f[9], g[10];
                gather_node<S, float>(static_cast<const S*>(prev), X * r + dx, Y * r + dy, L.nx, L.ny,
                                      L.pitch, L.plane, 0, 0, f, g);
#pragma unroll
                for (int i = 0; i < 9; ++i) acc[i] += f[i];
#pragma unroll
                for (int q = 0; q < 10; ++q) acc[9 + q] += g[q];
            }
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) out[(long long)p * nc + k] = acc[p] * inv;
    }
}

// Filtered sub-grid momentum flux of a fine lattice's pre-collision state
// (FP64 arithmetic): per coarse node the r x r block averages of rho,
// rho u, b and of rho u u + M(b); tau_sgs = <flux> - flux of the averaged
// fields (u = <rho u>/<rho>); out = tau_sgs / (1 - omega_coarse).
template <int PREC>
__global__ void sgs_kernel(const void* prev, Layout L, int r, double inv_om1, float* out) {
    using S = typename Prec<PREC>::S;
    const int ncx = L.nx / r, ncy = L.ny / r;
    const long long nc = (long long)ncx * ncy;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nc;
         k += (long long)gridDim.x * blockDim.x) {
        const int X = (int)(k % ncx), Y = (int)(k / ncx);
        double R = 0, MX = 0, MY = 0, BX = 0, BY = 0, Fxx = 0, Fxy = 0, Fyy = 0;
        const double rho0 = 1.0;
        for (int dy = 0; dy < r; ++dy)
            for (int dx = 0; dx < r; ++dx) {
                float f[9], g[10];
                gather_node<S, float>(static_cast<const S*>(prev), X * r + dx, Y * r + dy, L.nx, L.ny,
                                      L.pitch, L.plane, 0, 0, f, g);
                double fd[9], gd[10];
#pragma unroll
                for (int i = 0; i < 9; ++i) fd[i] = (double)f[i];
#pragma unroll
                for (int q = 0; q < 10; ++q) gd[q] = (double)g[q];
                const Moments<double> m = moments<double>(fd, gd, rho0);
                const double b2 = m.bx * m.bx + m.by * m.by;
                R += m.rho; MX += m.mx; MY += m.my; BX += m.bx; BY += m.by;
                Fxx += m.mx * m.ux + 0.5 * b2 - m.bx * m.bx;
                Fxy += m.mx * m.uy - m.bx * m.by;
                Fyy += m.my * m.uy + 0.5 * b2 - m.by * m.by;
            }
        const double a = 1.0 / (double)(r * r);
        R *= a; MX *= a; MY *= a; BX *= a; BY *= a; Fxx *= a; Fxy *= a; Fyy *= a;
        const double UX = MX / R, UY = MY / R, B2 = BX * BX + BY * BY;
        out[3 * k + 0] = (float)((Fxx - (R * UX * UX + 0.5 * B2 - BX * BX)) * inv_om1);
        out[3 * k + 1] = (float)((Fxy - (R * UX * UY - BX * BY)) * inv_om1);
        out[3 * k + 2] = (float)((Fyy - (R * UY * UY + 0.5 * B2 - BY * BY)) * inv_om1);
    }
}

constexpr int kFTX = 32, kFTY = 8, kFHX = kFTX + 2, kFHY = kFTY + 2;

// Features of a packed coarse pre-collision state (FP32 deviations).
__global__ void __launch_bounds__(256) features_kernel(const float* __restrict__ st, int nx, int ny,
                                                       float rho0, float* __restrict__ X) {
    __shared__ float sm[4][kFHY][kFHX];
    const long long n = (long long)nx * ny;
    const int tid = threadIdx.y * kFTX + threadIdx.x;
    const int x0 = blockIdx.x * kFTX, y0 = blockIdx.y * kFTY;
    for (int r = tid; r < kFHX * kFHY; r += kFTX * kFTY) {
        const int hx = r % kFHX, hy = r / kFHX;
        const int gx = ((x0 - 1 + hx) % nx + nx) % nx, gy = ((y0 - 1 + hy) % ny + ny) % ny;
        const long long o = (long long)gy * nx + gx;
        float f[9], g[10], pf[8];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const float v = st[(long long)p * n + o];
            if (p < 9) f[p] = v; else g[p - 9] = v;
        }
        point_features(f, g, rho0, pf);
        sm[0][hy][hx] = pf[1]; sm[1][hy][hx] = pf[2]; sm[2][hy][hx] = pf[3]; sm[3][hy][hx] = pf[4];
    }
    __syncthreads();
    const int lx = threadIdx.x, ly = threadIdx.y, x = x0 + lx, y = y0 + ly;
    if (x >= nx || y >= ny) return;
    const long long o = (long long)y * nx + x;
    float f[9], g[10], feat[kIn];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const float v = st[(long long)p * n + o];
        if (p < 9) f[p] = v; else g[p - 9] = v;
    }
    point_features(f, g, rho0, feat);
    stencil_features<kFHX, kFHY>(sm, lx, ly, feat + 8);
#pragma unroll
    for (int c = 0; c < kIn; ++c) X[o * kIn + c] = feat[c];
}

// One-step targets (FP64 arithmetic from FP32 states):
//   dA = (sum_i H2_i F*_i - a0^(2)) / (1 - omega) - a1^(2)(T),
//   F*_i(x) = F_i(x + c_i, T+1)   (periodic).
__global__ void targets_kernel(const float* __restrict__ sT, const float* __restrict__ sT1, int nx, int ny,
                               double rho0, double omega, float* __restrict__ out) {
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(k % nx), y = (int)(k / nx);
        double f[9], g[10];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const double v = (double)sT[(long long)p * n + k];
            if (p < 9) f[p] = v; else g[p - 9] = v;
        }
        const Moments<double> m = moments<double>(f, g, rho0);
        const double Mxx = 0.5 * (m.by * m.by - m.bx * m.bx), Mxy = -m.bx * m.by;
        const double a2xx = (f[1] + f[2] + f[3] + f[5] + f[6] + f[7]) - m.drho / 3.0 - m.mx * m.ux - Mxx;
        const double a2yy = (f[1] + f[3] + f[4] + f[5] + f[7] + f[8]) - m.drho / 3.0 - m.my * m.uy + Mxx;
        const double a2xy = ((f[3] + f[7]) - (f[1] + f[5])) - m.mx * m.uy - Mxy;
        double sxx = 0, sxy = 0, syy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cx = cx_of(i), cy = cy_of(i);
            const int xs = (x + cx + nx) % nx, ys = (y + cy + ny) % ny;
            const double v = (double)sT1[(long long)i * n + (long long)ys * nx + xs];
            sxx += (cx * cx - 1.0 / 3.0) * v;
            sxy += (double)(cx * cy) * v;
            syy += (cy * cy - 1.0 / 3.0) * v;
        }
        const double om1 = 1.0 - omega;
        out[3 * k + 0] = (float)((sxx - (m.mx * m.ux + Mxx)) / om1 - a2xx);
        out[3 * k + 1] = (float)((sxy - (m.mx * m.uy + Mxy)) / om1 - a2xy);
        out[3 * k + 2] = (float)((syy - (m.my * m.uy - Mxx)) / om1 - a2yy);
    }
}

// ---- MLP training kernels ------------------------------------------------------
// Layer forward on one warp per 16-row tile: out = A (M x K) * W^T + b with
// Wt stored output-major (N x K).  RELU: write Z (FP32) and H = bf16(relu(Z));
// else write Y (FP32).
template <int K, int N, bool RELU>
__global__ void mlp_fwd(const bf16* __restrict__ A, const bf16* __restrict__ Wt, const float* __restrict__ bias,
                        int M, float* __restrict__ Z, bf16* __restrict__ H) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int mt = warp; mt * 16 < M; mt += nwarps) {
        const int m0 = mt * 16;
        uint32_t a[K / 16][4];
#pragma unroll
        for (int c = 0; c < K / 16; ++c) {
            a[c][0] = ld2(A + (long long)(m0 + g) * K + 16 * c + 2 * t);
            a[c][1] = ld2(A + (long long)(m0 + g + 8) * K + 16 * c + 2 * t);
            a[c][2] = ld2(A + (long long)(m0 + g) * K + 16 * c + 2 * t + 8);
            a[c][3] = ld2(A + (long long)(m0 + g + 8) * K + 16 * c + 2 * t + 8);
        }
#pragma unroll
        for (int j = 0; j < N / 8; ++j) {
            const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
            float d[4] = {b0, b1, b0, b1};
#pragma unroll
            for (int c = 0; c < K / 16; ++c) {
                const uint32_t b[2] = {ld2(Wt + (8 * j + g) * K + 16 * c + 2 * t),
                                       ld2(Wt + (8 * j + g) * K + 16 * c + 2 * t + 8)};
                mma16816(d, a[c], b);
            }
            const long long r0 = (long long)(m0 + g) * N + 8 * j + 2 * t, r1 = r0 + 8LL * N;
            Z[r0] = d[0]; Z[r0 + 1] = d[1]; Z[r1] = d[2]; Z[r1 + 1] = d[3];
            if (RELU) {
                *reinterpret_cast<uint32_t*>(H + r0) = pack2(fmaxf(d[0], 0.f), fmaxf(d[1], 0.f));
                *reinterpret_cast<uint32_t*>(H + r1) = pack2(fmaxf(d[2], 0.f), fmaxf(d[3], 0.f));
            }
        }
    }
}

// Batch assembly: rows idx[r] of X (n x 24, raw) -> xb (rows x 32, bf16,
// normalised, zero padded), T (n x 3) -> tb (rows x 3); rows beyond nreal zero.
__global__ void gather_batch(const float* __restrict__ X, const float* __restrict__ T, const int* __restrict__ idx,
                             int nreal, int rows, const float* __restrict__ prm, bf16* __restrict__ xb,
                             float* __restrict__ tb) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const bool ok = r < nreal;
        const long long s = ok ? (idx ? idx[r] : r) : 0;
#pragma unroll
        for (int c = 0; c < kInPad; ++c) {
            float v = 0.f;
            if (ok && c < kIn) v = (X[s * kIn + c] - prm[kOffMean + c]) * prm[kOffScale + c];
            xb[(long long)r * kInPad + c] = __float2bfloat16_rn(v);
        }
#pragma unroll
        for (int c = 0; c < kOut; ++c) tb[(long long)r * kOut + c] = (ok && T) ? T[s * kOut + c] : 0.f;
    }
}

// BF16 weight copies in both layouts and padded FP32 biases from the blob.
__global__ void refresh_weights(const float* __restrict__ prm, MlpDev d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // layer 1: W1[in 24][out 64] -> Wt1 (64 x 32), W1b (32 x 64)
    if (i < kHid * kInPad) {
        const int o = i / kInPad, k = i % kInPad;
        const float w = k < kIn ? prm[kOffW1 + k * kHid + o] : 0.f;
        d.Wt1[o * kInPad + k] = __float2bfloat16_rn(w);
        d.W1[k * kHid + o] = __float2bfloat16_rn(w);
    }
    if (i < kHid * kHid) {
        const int o = i / kHid, k = i % kHid;
        const float w = prm[kOffW2 + k * kHid + o];
        d.Wt2[o * kHid + k] = __float2bfloat16_rn(w);
        d.W2[k * kHid + o] = __float2bfloat16_rn(w);
    }
    if (i < kOutPad * kHid) {  // Wt3: 8 x 64
        const int o = i / kHid, k = i % kHid;
        d.Wt3[o * kHid + k] = __float2bfloat16_rn(o < kOut ? prm[kOffW3 + k * kOut + o] : 0.f);
    }
    if (i < kHid * kOutPadK) {  // W3b: 64 x 16
        const int k = i / kOutPadK, o = i % kOutPadK;
        d.W3[k * kOutPadK + o] = __float2bfloat16_rn(o < kOut ? prm[kOffW3 + k * kOut + o] : 0.f);
    }
    if (i < kHid) {
        d.b1[i] = prm[kOffB1 + i];
        d.b2[i] = prm[kOffB2 + i];
    }
    if (i < kOutPad) d.b3[i] = i < kOut ? prm[kOffB3 + i] : 0.f;
}

// Per-column mean and scale (1 / std) of X (n x 24) and std of T (n x 3):
// per-block FP64 partial sums, then a one-block finish.
__global__ void stats_partials(const float* __restrict__ X, const float* __restrict__ T, long long n,
                               double* __restrict__ P) {
    constexpr int W = kIn + kOut;
    __shared__ double s1[W][8], s2[W][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double a1[W], a2[W];
#pragma unroll
    for (int c = 0; c < W; ++c) a1[c] = a2[c] = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < W; ++c) {
            const double v = c < kIn ? (double)X[r * kIn + c] : (double)T[r * kOut + c - kIn];
            a1[c] += v;
            a2[c] += v * v;
        }
    }
#pragma unroll
    for (int c = 0; c < W; ++c) {
        double v1 = a1[c], v2 = a2[c];
        for (int o = 16; o > 0; o >>= 1) {
            v1 += __shfl_down_sync(0xffffffffu, v1, o);
            v2 += __shfl_down_sync(0xffffffffu, v2, o);
        }
        if (lane == 0) { s1[c][warp] = v1; s2[c][warp] = v2; }
    }
    __syncthreads();
    if (threadIdx.x < W) {
        double v1 = 0, v2 = 0;
        for (int w = 0; w < 8; ++w) { v1 += s1[threadIdx.x][w]; v2 += s2[threadIdx.x][w]; }
        P[(long long)blockIdx.x * 2 * W + threadIdx.x] = v1;
        P[(long long)blockIdx.x * 2 * W + W + threadIdx.x] = v2;
    }
}

__global__ void stats_finish(const double* __restrict__ P, int nblocks, long long n, float* __restrict__ prm) {
    constexpr int W = kIn + kOut;
    const int c = threadIdx.x;
    if (c >= W) return;
    double v1 = 0, v2 = 0;
    for (int b = 0; b < nblocks; ++b) { v1 += P[(long long)b * 2 * W + c]; v2 += P[(long long)b * 2 * W + W + c]; }
    const double mean = v1 / (double)n;
    const double var = fmax(v2 / (double)n - mean * mean, 0.0);
    const double sd = sqrt(var);
    if (c < kIn) {
        prm[kOffMean + c] = (float)mean;
        prm[kOffScale + c] = (float)(sd > 0 ? 1.0 / sd : 1.0);
    } else {
        prm[kOffOutScale + c - kIn] = (float)(sd > 0 ? sd : 1.0);
    }
}

cudaError_t launch_filter(const Layout& L, int prec, const void* prev, int r, float* out, cudaStream_t st) {
    const long long nc = (long long)(L.nx / r) * (L.ny / r);
    const int blocks = (int)std::min<long long>((nc + 255) / 256, 16LL * device_sms());
    switch (prec) {
    case 0: filter_kernel<0><<<blocks, 256, 0, st>>>(prev, L, r, out); break;
    case 1: filter_kernel<1><<<blocks, 256, 0, st>>>(prev, L, r, out); break;
    case 2: filter_kernel<2><<<blocks, 256, 0, st>>>(prev, L, r, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_sgs(const Layout& L, int prec, const void* prev, int r, double tau_coarse, float* out,
                       cudaStream_t st) {
    const long long nc = (long long)(L.nx / r) * (L.ny / r);
    const int blocks = (int)std::min<long long>((nc + 255) / 256, 16LL * device_sms());
    const double inv = 1.0 / (1.0 - 1.0 / tau_coarse);
    switch (prec) {
    case 0: sgs_kernel<0><<<blocks, 256, 0, st>>>(prev, L, r, inv, out); break;
    case 1: sgs_kernel<1><<<blocks, 256, 0, st>>>(prev, L, r, inv, out); break;
    case 2: sgs_kernel<2><<<blocks, 256, 0, st>>>(prev, L, r, inv, out); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_features(const float* st_, int nx, int ny, float rho0, float* X, cudaStream_t st) {
    dim3 grid((nx + kFTX - 1) / kFTX, (ny + kFTY - 1) / kFTY);
    features_kernel<<<grid, dim3(kFTX, kFTY), 0, st>>>(st_, nx, ny, rho0, X);
    return cudaGetLastError();
}

cudaError_t launch_targets(const float* sT, const float* sT1, int nx, int ny, double rho0, double omega,
                           float* out, cudaStream_t st) {
    const long long n = (long long)nx * ny;
    const int blocks = (int)std::min<long long>((n + 255) / 256, 16LL * device_sms());
    targets_kernel<<<blocks, 256, 0, st>>>(sT, sT1, nx, ny, rho0, omega, out);
    return cudaGetLastError();
}

// ---- training driver pieces ------------------------------------------------------



cudaError_t launch_gather_batch(const float* X, const float* T, const int* idx, int nreal, int rows,
                                const float* prm, const MlpDev& d, cudaStream_t st) {
    const int blocks = std::max(1, std::min((rows + 255) / 256, 8 * device_sms()));
    gather_batch<<<blocks, 256, 0, st>>>(X, T, idx, nreal, rows, prm, d.xb, d.tb);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const float* prm, const MlpDev& d, cudaStream_t st) {
    refresh_weights<<<(kHid * kHid + 255) / 256, 256, 0, st>>>(prm, d);
    return cudaGetLastError();
}

cudaError_t launch_stats(const float* X, const float* T, long long n, double* P, int nblocks, float* prm,
                         cudaStream_t st) {
    stats_partials<<<nblocks, 256, 0, st>>>(X, T, n, P);
    stats_finish<<<1, 32, 0, st>>>(P, nblocks, n, prm);
    return cudaGetLastError();
}

__global__ void scale_outputs(const float* __restrict__ Y, int nreal, const float* __restrict__ prm,
                              float* __restrict__ out) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nreal; r += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < kOut; ++c) out[(long long)r * kOut + c] = Y[(long long)r * kOutPad + c] * prm[kOffOutScale + c];
}

cudaError_t launch_mlp_predict(const MlpDev& d, int rows, int nreal, const float* prm, float* Yraw, cudaStream_t st) {
    const int fwd_blocks = std::max(1, std::min((rows / 16 + 7) / 8, 8 * device_sms()));
    mlp_fwd<kInPad, kHid, true><<<fwd_blocks, 256, 0, st>>>(d.xb, d.Wt1, d.b1, rows, d.Z1, d.H1);
    mlp_fwd<kHid, kHid, true><<<fwd_blocks, 256, 0, st>>>(d.H1, d.Wt2, d.b2, rows, d.Z2, d.H2);
    mlp_fwd<kHid, kOutPad, false><<<fwd_blocks, 256, 0, st>>>(d.H2, d.Wt3, d.b3, rows, d.Y, nullptr);
    scale_outputs<<<std::max(1, std::min((nreal + 255) / 256, 8 * device_sms())), 256, 0, st>>>(d.Y, nreal, prm, Yraw);
    return cudaGetLastError();
}

}  // namespace mhd
