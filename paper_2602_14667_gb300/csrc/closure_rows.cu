// closure_rows.cu -- the closure step (learned correction of a1^(2), the
// closure is not part of the paper) with one warp per tile of rows and the
// MLP on warp-level mma.sync.
//
// A warp walks one tile: a strip of 30 output columns (lanes 1..30; lanes
// 0 and 31 hold the neighbouring columns, so x neighbours arrive by warp
// shuffles) and a stack of rows, downwards in even row segments and upwards
// in odd ones.  The pull of every row of the walk (the pre-collision
// populations of its 32 nodes, one node per lane) is copied with cp.async
// into a per-warp stage of three row slots one row ahead of its use (the
// next row of the tile, or the first row of the warp's next tile), so the
// loads of one row overlap the work on the previous one.  The warp keeps u
// and b of the last three rows in registers; for the row before the newest
// one it forms the 24 features (point values and the 3 x 3 stencils), runs
// the 24 -> 64 -> 64 -> 3 MLP on its 32 feature rows as two M tiles sharing
// every weight fragment (BF16 operands, FP32 accumulation; bias in the
// accumulator, ReLU and the BF16 packing of the next layer's operand in one
// conversion), adds the output to the projected a1^(2) and collides (tasks
// 3-5 of the paper's "Algorithm of computation").  The only block-wide
// barrier is the one after the weights are staged in shared memory; the
// stage, the feature rows and the outputs are per warp.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "closure_device.cuh"
#include "closure_internal.h"

namespace mhd {

namespace {

constexpr int kRWarps = 8;      // warps per block, each on its own tiles
constexpr int kRFeat = 40;      // bf16 per feature row (80 bytes: conflict-free ldmatrix rows)
constexpr int kRW1 = 40;        // padded weight rows (bf16): strides of 20 and 36 words put
constexpr int kRW2 = 72;        // the 32 lanes of a B-fragment load in 32 banks

struct RowsShared {
    bf16 Wt1[kHid * kRW1];
    bf16 Wt2[kHid * kRW2];
    bf16 Wt3[kOutPad * kRW2];
    float b1[kHid], b2[kHid], b3[kOutPad];
    alignas(16) float mean[kIn];
    alignas(16) float scale[kIn];
    float out_scale[kOut];
    alignas(16) bf16 feat[kRWarps][32 * kRFeat];
    float da[kRWarps][32][4];
    float stage[kRWarps][3][kPlanes][32];  // per warp: three pulled rows, plane-major, a column per lane
};
static_assert(offsetof(RowsShared, Wt1) % 16 == 0 && offsetof(RowsShared, Wt2) % 16 == 0 &&
                  offsetof(RowsShared, Wt3) % 16 == 0 && offsetof(RowsShared, feat) % 16 == 0,
              "ldmatrix sources must be 16-byte aligned");
static_assert((kRW1 * sizeof(bf16)) % 16 == 0 && (kRW2 * sizeof(bf16)) % 16 == 0 &&
                  (kRFeat * sizeof(bf16)) % 16 == 0,
              "ldmatrix row strides must be multiples of 16 bytes");
static_assert(offsetof(RowsShared, b1) % 8 == 0 && offsetof(RowsShared, b2) % 8 == 0 &&
                  offsetof(RowsShared, b3) % 8 == 0,
              "bias pairs are read as float2");

// MLP of the warp's 32 feature rows (two M tiles sharing every B fragment);
// out_scale * y into da.
__device__ __forceinline__ void mlp32(const RowsShared& sh, const bf16* feat, float (*da)[4], int lane) {
    const int t = lane & 3, lr = lane & 7, lm = lane >> 3;
    uint32_t h[2][4][4];  // layer 2's A fragments (K = 64) of both M tiles
    {
        uint32_t a1[2][2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int c = 0; c < 2; ++c)
                ldsm_x4(a1[mt][c], feat + (16 * mt + lr + 8 * (lm & 1)) * kRFeat + 16 * c + 8 * (lm >> 1));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 bb = *reinterpret_cast<const float2*>(sh.b1 + 8 * j + 2 * t);
            uint32_t w[4];
            ldsm_x4(w, sh.Wt1 + (8 * j + lr) * kRW1 + 8 * lm);
            const uint32_t b0[2] = {w[0], w[1]}, b1[2] = {w[2], w[3]};
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                float d[4] = {bb.x, bb.y, bb.x, bb.y};
                mma16816(d, a1[mt][0], b0);
                mma16816(d, a1[mt][1], b1);
                // the accumulator of n-tile j is half of k-chunk j/2 of the next A
                h[mt][j >> 1][(j & 1) * 2 + 0] = relu_pack2(d[0], d[1]);
                h[mt][j >> 1][(j & 1) * 2 + 1] = relu_pack2(d[2], d[3]);
            }
        }
    }
    uint32_t h2[2][4][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 bb = *reinterpret_cast<const float2*>(sh.b2 + 8 * j + 2 * t);
        float d[2][4] = {{bb.x, bb.y, bb.x, bb.y}, {bb.x, bb.y, bb.x, bb.y}};
#pragma unroll
        for (int c = 0; c < 4; c += 2) {
            uint32_t w[4];
            ldsm_x4(w, sh.Wt2 + (8 * j + lr) * kRW2 + 16 * c + 8 * lm);
            const uint32_t b0[2] = {w[0], w[1]}, b1[2] = {w[2], w[3]};
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma16816(d[mt], h[mt][c], b0);
                mma16816(d[mt], h[mt][c + 1], b1);
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            h2[mt][j >> 1][(j & 1) * 2 + 0] = relu_pack2(d[mt][0], d[mt][1]);
            h2[mt][j >> 1][(j & 1) * 2 + 1] = relu_pack2(d[mt][2], d[mt][3]);
        }
    }
    const float2 bb = *reinterpret_cast<const float2*>(sh.b3 + 2 * t);
    float d[2][4] = {{bb.x, bb.y, bb.x, bb.y}, {bb.x, bb.y, bb.x, bb.y}};
#pragma unroll
    for (int c = 0; c < 4; c += 2) {
        uint32_t w[4];
        ldsm_x4(w, sh.Wt3 + lr * kRW2 + 16 * c + 8 * lm);
        const uint32_t b0[2] = {w[0], w[1]}, b1[2] = {w[2], w[3]};
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            mma16816(d[mt], h2[mt][c], b0);
            mma16816(d[mt], h2[mt][c + 1], b1);
        }
    }
    // d0: (row g, col 2t), d1: (g, 2t+1), d2: (g+8, 2t), d3: (g+8, 2t+1)
    const int g = lane >> 2;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        if (2 * t < kOut) {
            da[16 * mt + g][2 * t] = d[mt][0] * sh.out_scale[2 * t];
            da[16 * mt + g + 8][2 * t] = d[mt][2] * sh.out_scale[2 * t];
        }
        if (2 * t + 1 < kOut) {
            da[16 * mt + g][2 * t + 1] = d[mt][1] * sh.out_scale[2 * t + 1];
            da[16 * mt + g + 8][2 * t + 1] = d[mt][3] * sh.out_scale[2 * t + 1];
        }
    }
}

template <typename Off>
__global__ void __launch_bounds__(kRWarps * 32, 2) step_closure_rows(const StepArgs<float> a,
                                                                     const ClosureParamsDev cp, int strips,
                                                                     int rows, int ntiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RowsShared& sh = *reinterpret_cast<RowsShared*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float* src = static_cast<const float*>(a.src);
    float* dst = static_cast<float*>(a.dst);
    // the network: weight rows in 16-byte pieces into the padded shared rows
    constexpr int kC1 = kInPad * 2 / 16, kC2 = kHid * 2 / 16;  // 16-byte pieces per weight row
    for (int i = tid; i < kHid * kC1; i += kRWarps * 32)
        cp_async16(sh.Wt1 + (i / kC1) * kRW1 + (i % kC1) * 8, cp.Wt1 + (i / kC1) * kInPad + (i % kC1) * 8);
    for (int i = tid; i < kHid * kC2; i += kRWarps * 32)
        cp_async16(sh.Wt2 + (i / kC2) * kRW2 + (i % kC2) * 8, cp.Wt2 + (i / kC2) * kHid + (i % kC2) * 8);
    for (int i = tid; i < kOutPad * kC2; i += kRWarps * 32)
        cp_async16(sh.Wt3 + (i / kC2) * kRW2 + (i % kC2) * 8, cp.Wt3 + (i / kC2) * kHid + (i % kC2) * 8);
    cp_async_commit();
    if (tid < kHid) { sh.b1[tid] = cp.b1[tid]; sh.b2[tid] = cp.b2[tid]; }
    if (tid < kOutPad) sh.b3[tid] = cp.b3[tid];
    if (tid < kIn) { sh.mean[tid] = cp.mean[tid]; sh.scale[tid] = cp.scale[tid]; }
    if (tid < kOut) sh.out_scale[tid] = cp.out_scale[tid];

    // tile t: strip t % strips of 30 output columns (lane l holds column
    // 30 * strip - 1 + l, wrapped), rows [y0, y1) of segment t / strips; row
    // i of its walk is y0 - 1 + i (even segments) or y1 - i (odd ones)
    struct Tile {
        int xl, xw, y0, y1;
        bool up;
    };
    auto tile_of = [&](int t) {
        Tile T;
        const int strip = t % strips, seg = t / strips;
        T.xl = strip * 30 - 1 + lane;
        T.xw = T.xl % a.nx;
        if (T.xw < 0) T.xw += a.nx;
        T.y0 = seg * rows;
        T.y1 = min(a.ny, T.y0 + rows);
        T.up = seg & 1;
        return T;
    };
    // the pull of row i of tile T into stage slot sl: each lane copies its
    // own node's 19 cells into its own column of the slot
    auto issue_row = [&](const Tile& T, int i, int sl) {
        const int m = T.up ? T.y1 - i : T.y0 - 1 + i;
        const int my = m < 0 ? m + a.ny : (m >= a.ny ? m - a.ny : m);
        const int ym = my == 0 ? a.ny - 1 : my - 1, yp = my + 1 == a.ny ? 0 : my + 1;
        const int xm = T.xw == 0 ? a.nx - 1 : T.xw - 1, xp = T.xw + 1 == a.nx ? 0 : T.xw + 1;
        const Off pt = (Off)a.pitch, pl = (Off)a.plane;
        const Off r_m = (Off)ym * pt, r_0 = (Off)my * pt, r_p = (Off)yp * pt;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int cx = pcx(p), cy = pcy(p);
            const Off o = (Off)p * pl + (cy > 0 ? r_m : (cy < 0 ? r_p : r_0)) + (cx > 0 ? xm : (cx < 0 ? xp : T.xw));
            cp_async4(&sh.stage[warp][sl][p][lane], src + o);
        }
    };
    const int stride = gridDim.x * kRWarps;
    int t = blockIdx.x * kRWarps + warp;
    // the first row of the warp's first tile is in flight while the weights land
    if (t < ntiles) issue_row(tile_of(t), 0, 0);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's weight pieces (the older group)
    __syncthreads();

    bf16* feat = sh.feat[warp];
    float(*da)[4] = sh.da[warp];
    const bool out_lane = lane >= 1 && lane <= 30;
    const float rho0 = a.np.rho0;
    int sl = 0;  // stage slot of the row about to be used
    for (; t < ntiles; t += stride) {
        const Tile T = tile_of(t);
        const float sgn = T.up ? -1.f : 1.f;
        float wnd[3][4] = {};  // u_x, u_y, b_x, b_y of the last three rows (slot 2 newest)
        const int nrow = T.y1 - T.y0 + 2;
        for (int i = 0; i < nrow; ++i) {
            // three slots: the row in flight (next of this tile, or the first
            // of the warp's next tile), the newest row, and the row before it
            const int sl_next = sl == 2 ? 0 : sl + 1, sl_prev = sl == 0 ? 2 : sl - 1;
            if (i + 1 < nrow)
                issue_row(T, i + 1, sl_next);
            else if (t + stride < ntiles)
                issue_row(tile_of(t + stride), 0, sl_next);
            cp_async_commit();
            cp_async_wait<1>();
            const float(*nxt)[32] = sh.stage[warp][sl];
            const float(*cur)[32] = sh.stage[warp][sl_prev];
            sl = sl_next;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                wnd[0][q] = wnd[1][q];
                wnd[1][q] = wnd[2][q];
            }
            {
                float f[9], g[10];
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = nxt[k][lane];
#pragma unroll
                for (int k = 0; k < 10; ++k) g[k] = nxt[9 + k][lane];
                const Moments<float> mm = moments(f, g, rho0);
                wnd[2][0] = mm.ux;
                wnd[2][1] = mm.uy;
                wnd[2][2] = mm.bx;
                wnd[2][3] = mm.by;
            }
            if (i < 2) continue;  // warp-uniform
            const int o = T.up ? T.y1 - i + 1 : T.y0 - 2 + i;  // the row of cur: y0 <= o < y1
            float fe[kIn];
            {
                float f[9], g[10];
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = cur[k][lane];
#pragma unroll
                for (int k = 0; k < 10; ++k) g[k] = cur[9 + k][lane];
                point_features(f, g, rho0, fe);
            }
            stencil_rows(wnd, sgn, fe + 8);
            {
                uint32_t pk[kInPad / 2];
#pragma unroll
                for (int c4 = 0; c4 < kIn / 4; ++c4) {
                    const float4 mu = *reinterpret_cast<const float4*>(sh.mean + 4 * c4);
                    const float4 sc = *reinterpret_cast<const float4*>(sh.scale + 4 * c4);
                    pk[2 * c4] = pack2((fe[4 * c4] - mu.x) * sc.x, (fe[4 * c4 + 1] - mu.y) * sc.y);
                    pk[2 * c4 + 1] = pack2((fe[4 * c4 + 2] - mu.z) * sc.z, (fe[4 * c4 + 3] - mu.w) * sc.w);
                }
#pragma unroll
                for (int c = kIn / 2; c < kInPad / 2; ++c) pk[c] = 0u;
                uint4* row = reinterpret_cast<uint4*>(feat + lane * kRFeat);
#pragma unroll
                for (int c = 0; c < kInPad / 8; ++c)
                    row[c] = make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
            }
            __syncwarp();
            mlp32(sh, feat, da, lane);
            __syncwarp();
            if (out_lane && T.xl < a.nx) {
                float f[9], g[10];
#pragma unroll
                for (int k = 0; k < 9; ++k) f[k] = cur[k][lane];
#pragma unroll
                for (int k = 0; k < 10; ++k) g[k] = cur[9 + k][lane];
                const float d3[3] = {da[lane][0], da[lane][1], da[lane][2]};
                if (cp.da_out) {
                    const Off nn = (Off)a.nx * (Off)a.ny, node = (Off)o * (Off)a.nx + T.xl;
#pragma unroll
                    for (int k = 0; k < 3; ++k) cp.da_out[(Off)k * nn + node] = d3[k];
                }
                collide_impl<true, float>(f, g, a.np, d3);
                const Off off = (Off)o * (Off)a.pitch + T.xl, pl = (Off)a.plane;
#pragma unroll
                for (int k = 0; k < 9; ++k) dst[(Off)k * pl + off] = f[k];
#pragma unroll
                for (int k = 0; k < 10; ++k) dst[(Off)(9 + k) * pl + off] = g[k];
            }
            __syncwarp();  // the next row rewrites the warp's feature and output tiles
        }
    }
    cp_async_wait<0>();
}

// The steps between two evaluations of the MLP: the fused step (the pull
// gather of step_row, four nodes per lane) with each node's stored
// correction added to a1^(2); 12 bytes per node more than the plain step.
template <typename Off>
__global__ void __launch_bounds__(512) step_da_cached(const StepArgs<float> a, const float* __restrict__ da,
                                                      int nxb, int ntiles) {
    constexpr int V = 4;
    const Off nn = (Off)a.nx * (Off)a.ny;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = (t / nxb) * blockDim.y + threadIdx.y;
        if (y >= a.ny) continue;  // whole warp
        const int lane = threadIdx.x, xb = t % nxb;
        float v[kPlanes][V];
        const bool active = gather_row<1, V, false, Off>(static_cast<const float*>(a.src), a.nx, a.ny, a.pitch,
                                                          a.plane, xb, y, lane, v);
        if (!active) continue;
        const int x0 = (xb * 32 + lane) * V;
        float d[3][V];
        const Off node = (Off)y * (Off)a.nx + x0;
#pragma unroll
        for (int k = 0; k < 3; ++k) VecIO<float, V>::load(da + (Off)k * nn + node, d[k]);
        float* dst = static_cast<float*>(a.dst);
        const Off o_0 = (Off)y * (Off)a.pitch + x0, pl = (Off)a.plane;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float f[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = v[i][k];
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = v[9 + q][k];
            const float d3[3] = {d[0][k], d[1][k], d[2][k]};
            collide_impl<true, float>(f, g, a.np, d3);
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i][k] = f[i];
#pragma unroll
            for (int q = 0; q < 10; ++q) v[9 + q][k] = g[q];
        }
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) VecIO<float, V>::store(dst + ((Off)p * pl + o_0), v[p]);
    }
}

}  // namespace

cudaError_t launch_step_da_cached(const StepLaunch& s, const float* da, cudaStream_t st) {
    constexpr int V = 4;
    if (s.prec != 1 || s.wall_x || s.wall_y || s.L.nx % V) return cudaErrorInvalidValue;
    if (reinterpret_cast<uintptr_t>(da) % 16 || ((long long)s.L.nx * s.L.ny) % V) return cudaErrorInvalidValue;
    StepArgs<float> a;
    a.src = s.src;
    a.dst = s.dst;
    a.nx = s.L.nx;
    a.ny = s.L.ny;
    a.pitch = s.L.pitch;
    a.plane = s.L.plane;
    a.np.omega = (float)s.omega;
    a.np.omega_m = (float)s.omega_m;
    a.np.rho0 = (float)s.rho0;
    a.np.variant = s.variant;
    a.np.collision = s.collision;
    a.np.mag_collision = s.mag_collision;
    a.wall_x = 0;
    a.wall_y = 0;
    const int nxb = (s.L.nx + 32 * V - 1) / (32 * V), ntiles = nxb * s.L.ny;  // one-warp blocks, one row each
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto kernel = small ? step_da_cached<int> : step_da_cached<long long>;
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32, 0);
    if (e != cudaSuccess) return e;
    // the residency of the plain FP32 step: about 4 KB of every plane in flight per SM
    per_sm = std::min(std::max(1, per_sm), 4096 / (32 * V * (int)sizeof(float)));
    const int blocks = std::max(1, std::min(ntiles, per_sm * sms));
    kernel<<<blocks, dim3(32, 1), 0, st>>>(a, da, nxb, ntiles);
    return cudaGetLastError();
}

cudaError_t launch_step_closure(const StepLaunch& s, const ClosureParamsDev& cp, cudaStream_t st) {
    if (s.prec != 1 || s.wall_x || s.wall_y) return cudaErrorInvalidValue;
    // the weight blocks are staged in 16-byte pieces
    for (const void* w : {(const void*)cp.Wt1, (const void*)cp.Wt2, (const void*)cp.Wt3})
        if (reinterpret_cast<uintptr_t>(w) % 16) return cudaErrorInvalidValue;
    StepArgs<float> a;
    a.src = s.src;
    a.dst = s.dst;
    a.nx = s.L.nx;
    a.ny = s.L.ny;
    a.pitch = s.L.pitch;
    a.plane = s.L.plane;
    a.np.omega = (float)s.omega;
    a.np.omega_m = (float)s.omega_m;
    a.np.rho0 = (float)s.rho0;
    a.np.variant = s.variant;
    a.np.collision = s.collision;
    a.np.mag_collision = s.mag_collision;
    a.wall_x = 0;
    a.wall_y = 0;
    const size_t smem = sizeof(RowsShared);
    // int element offsets while the 19 planes hold fewer than 2^31 elements
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto kernel = small ? step_closure_rows<int> : step_closure_rows<long long>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0, dev = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kRWarps * 32, smem);
    if (e != cudaSuccess) return e;
    // tiles: strips of 30 columns, row segments so that the tiles are about
    // as many as the resident warps
    const long long strips = (s.L.nx + 29) / 30;
    const long long maxb = (long long)std::max(1, per_sm) * sms;
    const long long segs_want = std::max(1LL, maxb * kRWarps / strips);
    const long long rows = ((long long)s.L.ny + segs_want - 1) / segs_want;
    const long long segs = ((long long)s.L.ny + rows - 1) / rows;
    const long long ntiles = strips * segs;
    if (ntiles > (1LL << 30)) return cudaErrorInvalidValue;
    const int blocks = (int)std::max(1LL, std::min(maxb, (ntiles + kRWarps - 1) / kRWarps));
    kernel<<<blocks, kRWarps * 32, smem, st>>>(a, cp, (int)strips, (int)rows, (int)ntiles);
    return cudaGetLastError();
}

}  // namespace mhd
