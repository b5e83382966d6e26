// mlp_train.cu -- one training step of the closure MLP (24 -> 64 -> 64 -> 3,
// ReLU, BF16 operands, FP32 accumulation) as two kernels.
//
// train_block: a block takes 128-row slices of the batch (one 16-row tile
// per warp), one slice per block up to one block per SM, several beyond.  A warp gathers and normalises its rows, runs the three layers on
// mma.sync fragments with the activations kept in registers (the
// accumulator fragment of one layer is the operand fragment of the next),
// forms the loss gradient, and back-propagates through the two hidden
// layers the same way, the ReLU masks kept as bits.  The activations and
// gradients of the block's rows are left in shared memory, from which the
// block adds the slice's share of the three weight gradients (Act^T dZ,
// loaded transposed by ldmatrix) to accumulators kept in registers, and at
// the end writes them, with the bias-gradient column sums and the loss, as
// one partial per block.
//
// train_update: every parameter sums the block partials in block order
// (deterministic), then either stores the gradient or applies Adam to the
// FP32 master weight and refreshes the BF16 copies the kernels read.
//
// The MSE loss and its gradient are those of the layer-by-layer kernels:
// dY = 2 (y - t / out_scale) / (n * 3) on real rows and outputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "closure_device.cuh"
#include "closure_internal.h"

namespace mhd {

namespace {

constexpr int kTR = 128;             // rows per block
constexpr int kTW = 8;               // warps per block (16 rows each)
constexpr int kSX = kInPad + 8;      // shared row strides (bf16), padded so
constexpr int kSH = kHid + 8;        // that the 8 rows of an ldmatrix fall
constexpr int kSY = 24;              // on distinct banks
constexpr int kBG = kHid + kHid + kOutPad;  // bias-gradient slots per warp

struct TrainShared {
    bf16 x[kTR][kSX];
    bf16 h1[kTR][kSH];
    bf16 h2[kTR][kSH];
    bf16 dy[kTR][kSY];
    bf16 dh2[kTR][kSH];
    bf16 dh1[kTR][kSH];
    float bg[kTW][kBG];
    double loss[kTW];
    // the weights and biases, staged once per block (rows padded as above)
    bf16 wt1[kHid][kSX];      // W1^T, output-major (forward)
    bf16 wt2[kHid][kSH];      // W2^T
    bf16 wt3[kOutPad][kSH];   // W3^T
    bf16 w3[kHid][kSY];       // W3, input-major (backward)
    bf16 w2[kHid][kSH];       // W2
    float b1[kHid], b2[kHid], b3[kOutPad];
};

__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const bf16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const bf16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(a)
                 : "memory");
}

// Sum over the 8 row groups g of a warp (lanes l, l^4, l^8, ...): the total
// of the 16 rows for columns 2t, 2t+1 ends up in lanes 0..3.
__device__ __forceinline__ float rows_sum(float v) {
    v += __shfl_xor_sync(kFull, v, 4);
    v += __shfl_xor_sync(kFull, v, 8);
    v += __shfl_xor_sync(kFull, v, 16);
    return v;
}

// One hidden layer on a 16-row tile: Z = A W^T + b (A as operand fragments
// over K, W^T output-major in shared memory), H = relu(Z) as the next
// layer's operand fragments and in shared memory, mask bit 4j+e = Z > 0.
template <int KC, int LD>
__device__ __forceinline__ void hidden_layer(const uint32_t (&a)[KC][4], const bf16 (*Wt)[LD],
                                             const float* bias, int g, int t, bf16 (*sh)[kSH],
                                             int r0, uint32_t (&h)[4][4], uint32_t& mask) {
    float d[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
        d[j][0] = b0; d[j][1] = b1; d[j][2] = b0; d[j][3] = b1;
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            const uint32_t b[2] = {ld2(&Wt[8 * j + g][16 * c + 2 * t]), ld2(&Wt[8 * j + g][16 * c + 2 * t + 8])};
            mma16816(d[j], a[c], b);
        }
    }
    mask = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            if (d[j][e] > 0.f) mask |= 1u << (4 * j + e);
            d[j][e] = fmaxf(d[j][e], 0.f);
        }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const uint32_t lo = pack2(d[j][0], d[j][1]), hi = pack2(d[j][2], d[j][3]);
        *reinterpret_cast<uint32_t*>(&sh[r0 + g][8 * j + 2 * t]) = lo;
        *reinterpret_cast<uint32_t*>(&sh[r0 + g + 8][8 * j + 2 * t]) = hi;
        h[j >> 1][(j & 1) * 2] = lo;
        h[j >> 1][(j & 1) * 2 + 1] = hi;
    }
}

// Back through a hidden layer: dH = (dZ W^T) masked by the layer's ReLU
// (W input-major in shared memory, dZ as operand fragments over KC chunks);
// writes BF16 dH to shared memory, its fragments for the layer below, and
// adds the column sums of the FP32 dH (bias gradient) to bg.
template <int KC, int LD>
__device__ __forceinline__ void hidden_back(const uint32_t (&a)[KC][4], const bf16 (*W)[LD], uint32_t mask,
                                            int g, int t, bf16 (*sh)[kSH], int r0, float* bg,
                                            uint32_t (&dh)[4][4]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            const uint32_t b[2] = {ld2(&W[8 * j + g][16 * c + 2 * t]), ld2(&W[8 * j + g][16 * c + 2 * t + 8])};
            mma16816(d, a[c], b);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (!((mask >> (4 * j + e)) & 1u)) d[e] = 0.f;
        const uint32_t lo = pack2(d[0], d[1]), hi = pack2(d[2], d[3]);
        *reinterpret_cast<uint32_t*>(&sh[r0 + g][8 * j + 2 * t]) = lo;
        *reinterpret_cast<uint32_t*>(&sh[r0 + g + 8][8 * j + 2 * t]) = hi;
        dh[j >> 1][(j & 1) * 2] = lo;
        dh[j >> 1][(j & 1) * 2 + 1] = hi;
        const float s0 = rows_sum(d[0] + d[2]), s1 = rows_sum(d[1] + d[3]);
        if (g == 0) {
            bg[8 * j + 2 * t] += s0;
            bg[8 * j + 2 * t + 1] += s1;
        }
    }
}

// acc += Act^T dZ over rows [0, nrows) of the block: Act (rows x KI, stride
// SA) gives the 16 x 16 operand tile (rows h0.., columns = batch rows),
// dZ (rows x n, stride SB) the 16 x 8 tile at column n0.
template <int SA, int SB>
__device__ __forceinline__ void wgrad_tile(const bf16 (*act)[SA], const bf16 (*dz)[SB], int h0, int n0, int nrows,
                                           int lane, float (&acc)[4]) {
    const int mi = lane >> 3, r = lane & 7;
    for (int k0 = 0; k0 < nrows; k0 += 16) {
        uint32_t a[4], b[2];
        ldsm_x4_t(a, &act[k0 + r + ((mi >> 1) << 3)][h0 + ((mi & 1) << 3)]);
        ldsm_x2_t(b, &dz[k0 + r + (((lane >> 3) & 1) << 3)][n0]);
        mma16816(acc, a, b);
    }
}

__global__ void __launch_bounds__(kTW * 32, 1) train_block(const float* __restrict__ X, const float* __restrict__ T,
                                                        const int* __restrict__ idx, int nreal, int rows,
                                                        const float* __restrict__ prm, const MlpDev d,
                                                        float* __restrict__ part, double* __restrict__ lossp,
                                                        long long* __restrict__ step) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainShared& S = *reinterpret_cast<TrainShared*>(smem_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int r0 = 16 * w;
    const int nslices = (rows + kTR - 1) / kTR;
    if (step && blockIdx.x == 0 && threadIdx.x == 0) *step += 1;  // Adam's step count

    // stage the weights and biases once (16-byte asynchronous copies, waited
    // for with the first slice's inputs in flight)
    {
        auto stage = [&](bf16* dst, int dld, const bf16* src, int nrow, int k) {
            const int chunks = k / 8;  // 8 bf16 per 16 bytes
            for (int q = threadIdx.x; q < nrow * chunks; q += blockDim.x)
                cp_async16(dst + (q / chunks) * dld + 8 * (q % chunks), src + (q / chunks) * k + 8 * (q % chunks));
        };
        stage(&S.wt1[0][0], kSX, d.Wt1, kHid, kInPad);
        stage(&S.wt2[0][0], kSH, d.Wt2, kHid, kHid);
        stage(&S.wt3[0][0], kSH, d.Wt3, kOutPad, kHid);
        stage(&S.w3[0][0], kSY, d.W3, kHid, kOutPadK);
        stage(&S.w2[0][0], kSH, d.W2, kHid, kHid);
        if (threadIdx.x < kHid / 4) {
            cp_async16(&S.b1[4 * threadIdx.x], d.b1 + 4 * threadIdx.x);
            cp_async16(&S.b2[4 * threadIdx.x], d.b2 + 4 * threadIdx.x);
        }
        if (threadIdx.x < kOutPad / 4) cp_async16(&S.b3[4 * threadIdx.x], d.b3 + 4 * threadIdx.x);
        cp_async_commit();
    }
    float* bg = S.bg[w];  // this warp's bias-gradient sums over the block's slices
    for (int c = lane; c < kBG; c += 32) bg[c] = 0.f;
    // this warp's weight-gradient tiles (tile w + 8 i), summed over the slices
    constexpr int kTilesPerWarp = (52 + kTW - 1) / kTW;
    float wacc[kTilesPerWarp][4];
#pragma unroll
    for (int i = 0; i < kTilesPerWarp; ++i) wacc[i][0] = wacc[i][1] = wacc[i][2] = wacc[i][3] = 0.f;
    double loss = 0.0;

    // a block walks the batch's 128-row slices (grid: at most one block per
    // SM, so the partials stay few whatever the batch size)
    for (int slice = blockIdx.x; slice < nslices; slice += gridDim.x) {
        const int blk_row = slice * kTR, m0 = blk_row + r0;
        const int nrows = min(kTR, rows - blk_row);  // a multiple of 16
        // sample index of each of the warp's 16 rows (lane r holds row r's),
        // then every load of the rows' inputs and targets issued together
        int my_s = 0;
        if (lane < 16 && m0 + lane < nreal) my_s = idx ? idx[m0 + lane] : m0 + lane;
        const int c = 2 * (lane & 15);  // this lane's column pair
        float xv[8][2];
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int rr = 2 * it + (lane >> 4);
            const long long sidx = __shfl_sync(kFull, my_s, rr);
            xv[it][0] = xv[it][1] = 0.f;
            if (m0 + rr < nreal && c < kIn) {
                xv[it][0] = X[sidx * kIn + c];
                xv[it][1] = X[sidx * kIn + c + 1];  // kIn is even
            }
        }
        float tv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int rr = g + ((e >> 1) << 3), col = 2 * t + (e & 1);
            const long long sidx = __shfl_sync(kFull, my_s, rr);
            tv[e] = (m0 + rr < nreal && col < kOut) ? T[sidx * kOut + col] : 0.f;
        }
        cp_async_wait<0>();
        __syncthreads();

        if (m0 < rows) {
            // normalise (padded columns and rows zero)
            const float mu0 = c < kIn ? prm[kOffMean + c] : 0.f, mu1 = c < kIn ? prm[kOffMean + c + 1] : 0.f;
            const float sc0 = c < kIn ? prm[kOffScale + c] : 0.f, sc1 = c < kIn ? prm[kOffScale + c + 1] : 0.f;
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int rr = 2 * it + (lane >> 4);
                const bool ok = m0 + rr < nreal && c < kIn;
                const float v0 = ok ? (xv[it][0] - mu0) * sc0 : 0.f, v1 = ok ? (xv[it][1] - mu1) * sc1 : 0.f;
                *reinterpret_cast<uint32_t*>(&S.x[r0 + rr][c]) = pack2(v0, v1);
            }
            __syncwarp();
            uint32_t a1[2][4];
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
                ldsm_x4(a1[kc], &S.x[r0 + (lane & 7) + (((lane >> 3) & 1) << 3)][16 * kc + ((lane >> 4) << 3)]);
            uint32_t h1[4][4], h2[4][4], mask1, mask2;
            hidden_layer<2, kSX>(a1, S.wt1, S.b1, g, t, S.h1, r0, h1, mask1);
            hidden_layer<4, kSH>(h1, S.wt2, S.b2, g, t, S.h2, r0, h2, mask2);
            // output layer and loss gradient (columns 2t, 2t+1 of rows g, g+8)
            float y[4] = {S.b3[2 * t], S.b3[2 * t + 1], S.b3[2 * t], S.b3[2 * t + 1]};
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const uint32_t b[2] = {ld2(&S.wt3[g][16 * cc + 2 * t]), ld2(&S.wt3[g][16 * cc + 2 * t + 8])};
                mma16816(y, h2[cc], b);
            }
            const float inv = 2.0f / (float)(nreal * kOut);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gr = m0 + g + ((e >> 1) << 3), col = 2 * t + (e & 1);
                float gy = 0.f;
                if (gr < nreal && col < kOut) {
                    const float dd = y[e] - tv[e] / prm[kOffOutScale + col];
                    loss += (double)dd * (double)dd;
                    gy = inv * dd;
                }
                y[e] = gy;
            }
            const uint32_t dy_lo = pack2(y[0], y[1]), dy_hi = pack2(y[2], y[3]);
            *reinterpret_cast<uint32_t*>(&S.dy[r0 + g][2 * t]) = dy_lo;
            *reinterpret_cast<uint32_t*>(&S.dy[r0 + g + 8][2 * t]) = dy_hi;
            {
                const float s0 = rows_sum(y[0] + y[2]), s1 = rows_sum(y[1] + y[3]);
                if (g == 0) {
                    bg[2 * kHid + 2 * t] += s0;
                    bg[2 * kHid + 2 * t + 1] += s1;
                }
            }
            // back through layer 2 (dZ = dY, 8 real of 16 operand columns) and layer 1
            const uint32_t ady[1][4] = {{dy_lo, dy_hi, 0u, 0u}};
            uint32_t dh2[4][4], dh1[4][4];
            hidden_back<1, kSY>(ady, S.w3, mask2, g, t, S.dh2, r0, bg + kHid, dh2);
            hidden_back<4, kSH>(dh2, S.w2, mask1, g, t, S.dh1, r0, bg, dh1);
        }
        __syncthreads();

        // weight gradients of the slice: 16 tiles of W1 (32 x 64), 32 of W2
        // (64 x 64), 4 of W3 (64 x 8); warp w takes tiles w, w + 8, ...
#pragma unroll
        for (int i = 0; i < kTilesPerWarp; ++i) {
            const int tile = w + kTW * i;
            if (tile < 16)
                wgrad_tile<kSX, kSH>(S.x, S.dh1, 16 * (tile >> 3), 8 * (tile & 7), nrows, lane, wacc[i]);
            else if (tile < 48)
                wgrad_tile<kSH, kSH>(S.h1, S.dh2, 16 * ((tile - 16) >> 3), 8 * ((tile - 16) & 7), nrows, lane,
                                     wacc[i]);
            else if (tile < 52)
                wgrad_tile<kSH, kSY>(S.h2, S.dy, 16 * (tile - 48), 0, nrows, lane, wacc[i]);
        }
        __syncthreads();  // the next slice overwrites the shared rows
    }

    // the block's partial: weight-gradient tiles, bias sums (warps in order), loss
    float* out = part + (long long)blockIdx.x * kBlob;
#pragma unroll
    for (int i = 0; i < kTilesPerWarp; ++i) {
        const int tile = w + kTW * i;
        if (tile >= 52) break;
        int h0, n0, off, ld, kmax, nmax;
        if (tile < 16) {
            h0 = 16 * (tile >> 3); n0 = 8 * (tile & 7); off = kOffW1; ld = kHid; kmax = kIn; nmax = kHid;
        } else if (tile < 48) {
            h0 = 16 * ((tile - 16) >> 3); n0 = 8 * ((tile - 16) & 7); off = kOffW2; ld = kHid; kmax = kHid; nmax = kHid;
        } else {
            h0 = 16 * (tile - 48); n0 = 0; off = kOffW3; ld = kOut; kmax = kHid; nmax = kOut;
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = h0 + g + ((e >> 1) << 3), n = n0 + 2 * t + (e & 1);
            if (k < kmax && n < nmax) out[off + k * ld + n] = wacc[i][e];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(kFull, loss, o);
    if (lane == 0) S.loss[w] = loss;
    __syncthreads();
    for (int c = threadIdx.x; c < kBG; c += blockDim.x) {
        float s = 0.f;
        for (int ww = 0; ww < kTW; ++ww) s += S.bg[ww][c];
        if (c < kHid) out[kOffB1 + c] = s;
        else if (c < 2 * kHid) out[kOffB2 + c - kHid] = s;
        else if (c - 2 * kHid < kOut) out[kOffB3 + c - 2 * kHid] = s;
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int ww = 0; ww < kTW; ++ww) s += S.loss[ww];
        lossp[blockIdx.x] = s;
    }
}

// Sum of the block partials per parameter; ADAM: update the master weight
// and its BF16 / bias copies and add the batch loss to *loss_acc; else
// store the gradient (zero for the untrained normalisation entries).  A
// block takes 32 parameters; warp w sums the partials of blocks w, w + 8,
// ... and the eight warp sums are added in warp order (a fixed order).
template <bool ADAM>
__global__ void __launch_bounds__(256) train_update(const float* __restrict__ part, int nblk, float* __restrict__ prm,
                                                    float* __restrict__ grad, float* __restrict__ m,
                                                    float* __restrict__ v, float lr,
                                                    const long long* __restrict__ step,
                                                    const double* __restrict__ lossp, double* __restrict__ loss_acc,
                                                    const MlpDev d) {
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    if (ADAM && blockIdx.x == 0 && threadIdx.x == 0) {
        double s = *loss_acc;
        for (int b = 0; b < nblk; ++b) s += lossp[b];
        *loss_acc = s;
    }
    float part_sum = 0.f;
    if (i >= kOffW1 && i < kBlob) {
#pragma unroll 4
        for (int b = w; b < nblk; b += 8) part_sum += part[(long long)b * kBlob + i];
    }
    red[w][lane] = part_sum;
    __syncthreads();
    if (w != 0 || i >= kBlob) return;
    if (i < kOffW1) {
        if (!ADAM) grad[i] = 0.f;
        return;
    }
    float gi = red[0][lane];
#pragma unroll
    for (int ww = 1; ww < 8; ++ww) gi += red[ww][lane];
    if (!ADAM) {
        grad[i] = gi;
        return;
    }
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float tn = (float)(*step);
    const float c1 = 1.f - powf(b1, tn), c2 = 1.f - powf(b2, tn);
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wv = prm[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    prm[i] = wv;
    const bf16 wb = __float2bfloat16_rn(wv);
    if (i < kOffB1) {
        const int k = (i - kOffW1) / kHid, o = (i - kOffW1) % kHid;
        d.Wt1[o * kInPad + k] = wb;
        d.W1[k * kHid + o] = wb;
    } else if (i < kOffW2) {
        d.b1[i - kOffB1] = wv;
    } else if (i < kOffB2) {
        const int k = (i - kOffW2) / kHid, o = (i - kOffW2) % kHid;
        d.Wt2[o * kHid + k] = wb;
        d.W2[k * kHid + o] = wb;
    } else if (i < kOffW3) {
        d.b2[i - kOffB2] = wv;
    } else if (i < kOffB3) {
        const int k = (i - kOffW3) / kOut, o = (i - kOffW3) % kOut;
        d.Wt3[o * kHid + k] = wb;
        d.W3[k * kOutPadK + o] = wb;
    } else {
        d.b3[i - kOffB3] = wv;
    }
}

// ---- the epoch's sample order ---------------------------------------------
// A pseudo-random permutation of [0, n) without a sort: a balanced 4-round
// Feistel network is a bijection on [0, 4^h) (h-bit halves, 4^h the
// smallest power of four >= n, so below 4n), and cycle-walking (apply it
// again while the image is >= n) restricts it to a bijection on [0, n).
// The round function is a 32-bit integer mix of the right half and a round
// key; the keys come from SplitMix64 of the seed and the Adam step count at
// the start of the epoch (one different order per epoch).
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

__global__ void epoch_permutation(int* __restrict__ idx, long long n, int h, unsigned long long seed,
                                  const long long* __restrict__ step) {
    const unsigned long long k64 = splitmix64(seed ^ splitmix64((unsigned long long)*step));
    const uint32_t key[4] = {(uint32_t)k64, (uint32_t)(k64 >> 32), (uint32_t)splitmix64(k64),
                             (uint32_t)(splitmix64(k64) >> 32)};
    const uint32_t mask = (1u << h) - 1u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        unsigned long long x = (unsigned long long)i;
        do {
            uint32_t L = (uint32_t)(x >> h), R = (uint32_t)x & mask;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const uint32_t nl = R, nr = L ^ (mix32(R ^ key[r]) & mask);
                L = nl;
                R = nr;
            }
            x = ((unsigned long long)L << h) | R;
        } while (x >= (unsigned long long)n);
        idx[i] = (int)x;
    }
}

}  // namespace

cudaError_t launch_epoch_permutation(int* idx, long long n, unsigned long long seed, const long long* step,
                                     cudaStream_t st) {
    int h = 1;
    while ((1LL << (2 * h)) < n) ++h;
    const long long blocks = std::max(1LL, std::min((n + 255) / 256, 16LL * device_sms()));
    epoch_permutation<<<(unsigned)blocks, 256, 0, st>>>(idx, n, h, seed, step);
    return cudaGetLastError();
}

// Blocks of the fused kernel: one per 128-row slice, at most one per SM
// (it holds 120 KB of shared memory); each block writes one partial.
int train_blocks(int rows) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, std::min((rows + kTR - 1) / kTR, sms));
}

cudaError_t prepare_train_kernels() {
    return cudaFuncSetAttribute(train_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrainShared));
}

cudaError_t launch_train_step(const float* X, const float* T, const int* idx, int nreal, int rows, float* prm,
                              const MlpDev& d, float* part, double* lossp, long long* step, float* grad, float* m,
                              float* v, float lr, double* loss_acc, bool adam, cudaStream_t st) {
    const int nblk = train_blocks(rows);
    train_block<<<nblk, kTW * 32, sizeof(TrainShared), st>>>(X, T, idx, nreal, rows, prm, d, part, lossp,
                                                             adam ? step : nullptr);
    const int ub = (kBlob + 31) / 32;
    if (adam)
        train_update<true><<<ub, 256, 0, st>>>(part, nblk, prm, grad, m, v, lr, step, lossp, loss_acc, d);
    else
        train_update<false><<<ub, 256, 0, st>>>(part, nblk, prm, grad, m, v, lr, step, lossp, loss_acc, d);
    return cudaGetLastError();
}

}  // namespace mhd
