// closure_device.cuh -- device pieces shared by the learned-closure kernels:
// warp-level BF16 MMA fragments, the feature stencils, and the tile gather
// of the closure step (32 x 8 nodes plus a one-node halo ring, fetched by
// cp.async into a double-buffered shared layout).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "closure_internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

using bf16 = __nv_bfloat16;

// ---- MMA helpers -------------------------------------------------------------
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}
// two consecutive bf16 (4-byte aligned)
__device__ __forceinline__ uint32_t ld2(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
// Four 8x8 bf16 matrices from shared memory in one instruction: lanes
// 8m .. 8m+7 give the 16-byte-aligned row addresses of matrix m, and r[m]
// receives this lane's share of matrix m in the mma fragment layout (row
// lane/4, columns 2(lane%4), 2(lane%4)+1).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const bf16* p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a)
                 : "memory");
}
// two separate bf16
__device__ __forceinline__ uint32_t ld11(const bf16* lo, const bf16* hi) {
    return (uint32_t)__bfloat16_as_ushort(*lo) | ((uint32_t)__bfloat16_as_ushort(*hi) << 16);
}

// relu(lo), relu(hi) rounded to BF16 (nearest even) and packed: lo in the
// low half, as the next layer's A fragment wants it.
__device__ __forceinline__ uint32_t relu_pack2(float lo, float hi) {
    uint32_t u;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(u) : "f"(hi), "f"(lo));
    return u;
}

// ---- feature stencils -------------------------------------------------------
// s[q][r][c] holds q in (u_x, u_y, b_x, b_y) for a tile plus a one-node
// halo; (r, c) = (ly + 1, lx + 1) is the node.
template <int HX, int HY>
__device__ __forceinline__ void stencil_features(const float (*s)[HY][HX], int lx, int ly, float* out16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float C = s[q][ly + 1][lx + 1];
        const float E = s[q][ly + 1][lx + 2], W = s[q][ly + 1][lx];
        const float N = s[q][ly + 2][lx + 1], S = s[q][ly][lx + 1];
        const float NE = s[q][ly + 2][lx + 2], NW = s[q][ly + 2][lx];
        const float SE = s[q][ly][lx + 2], SW = s[q][ly][lx];
        out16[4 * q + 0] = (1.0f / 3.0f) * (E - W) + (1.0f / 12.0f) * ((NE - NW) + (SE - SW));
        out16[4 * q + 1] = (1.0f / 3.0f) * (N - S) + (1.0f / 12.0f) * ((NE - SE) + (NW - SW));
        out16[4 * q + 2] = (4.0f * ((E + W) + (N + S)) + ((NE + NW) + (SE + SW)) - 20.0f * C) * (1.0f / 6.0f);
        out16[4 * q + 3] = 0.25f * ((NE - NW) - (SE - SW));
    }
}

// rho - rho0, u, b, projected a1^(2) of pre-collision deviations (FP32)
__device__ __forceinline__ void point_features(const float (&f)[9], const float (&g)[10], float rho0,
                                               float* out8) {
    const Moments<float> m = moments(f, g, rho0);
    const float Mxx = 0.5f * (m.by * m.by - m.bx * m.bx), Mxy = -m.bx * m.by;
    const float Sxx = f[1] + f[2] + f[3] + f[5] + f[6] + f[7];
    const float Syy = f[1] + f[3] + f[4] + f[5] + f[7] + f[8];
    const float Sxy = (f[3] + f[7]) - (f[1] + f[5]);
    out8[0] = m.drho;
    out8[1] = m.ux;
    out8[2] = m.uy;
    out8[3] = m.bx;
    out8[4] = m.by;
    out8[5] = Sxx - (1.0f / 3.0f) * m.drho - m.mx * m.ux - Mxx;
    out8[6] = Sxy - m.mx * m.uy - Mxy;
    out8[7] = Syy - (1.0f / 3.0f) * m.drho - m.my * m.uy + Mxx;
}

// ---- closure-step tiles ----------------------------------------------------
constexpr int kCTX = 32, kCTY = 8, kCHX = kCTX + 2, kCHY = kCTY + 2;
constexpr int kTile = kCTX * kCTY;          // 256 nodes
constexpr int kHalo = kCHX * kCHY - kTile;  // 84 ring positions

// 4-byte asynchronous global -> shared copy (completes at cp_async_wait)
__device__ __forceinline__ void cp_async4(float* smem, const float* gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// 16-byte asynchronous copy (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem) : "memory");
}
// wait until at most N of this thread's committed groups are still in flight
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }


// d_x, d_y (isotropic gradient), the 9-point Laplacian and d_xy of the four
// fields (u_x, u_y, b_x, b_y) at the lane's node, from w[r][q] with slot 1
// the node's row and slots 2 / 0 the rows on either side (sgn = +1 when
// slot 2 is the row above, -1 when it is the row below); x neighbours come
// from the neighbouring lanes.  Same stencils as stencil_features.
__device__ __forceinline__ void stencil_rows(const float (&w)[3][4], float sgn, float* out16) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float C = w[1][q], N = w[2][q], S = w[0][q];
        const float E = __shfl_down_sync(kFull, C, 1), W = __shfl_up_sync(kFull, C, 1);
        const float NE = __shfl_down_sync(kFull, N, 1), NW = __shfl_up_sync(kFull, N, 1);
        const float SE = __shfl_down_sync(kFull, S, 1), SW = __shfl_up_sync(kFull, S, 1);
        out16[4 * q + 0] = (1.0f / 3.0f) * (E - W) + (1.0f / 12.0f) * ((NE - NW) + (SE - SW));
        out16[4 * q + 1] = sgn * ((1.0f / 3.0f) * (N - S) + (1.0f / 12.0f) * ((NE - SE) + (NW - SW)));
        out16[4 * q + 2] = (4.0f * ((E + W) + (N + S)) + ((NE + NW) + (SE + SW)) - 20.0f * C) * (1.0f / 6.0f);
        out16[4 * q + 3] = sgn * (0.25f * ((NE - NW) - (SE - SW)));
    }
}

// Ring position h (0..83) of a tile: top row (34), bottom row (34), left
// column (8), right column (8), as (column, row) of the 34 x 10 halo tile.
__device__ __forceinline__ void ring_pos(int h, int& hx, int& hy) {
    if (h < kCHX) { hx = h; hy = 0; }
    else if (h < 2 * kCHX) { hx = h - kCHX; hy = kCHY - 1; }
    else if (h < 2 * kCHX + kCTY) { hx = 0; hy = 1 + h - 2 * kCHX; }
    else { hx = kCHX - 1; hy = 1 + h - 2 * kCHX - kCTY; }
}

// Issue the pull gather of tile tl (every thread its node, threads < 84 one
// ring node; periodic) into buffer b, as one cp.async group.
// Sh: any shared layout with pop[2][kPlanes][kTile] and hpop[2][kPlanes][kHalo].
template <typename Sh>
__device__ __forceinline__ void closure_prefetch(Sh& sh, const float* src, const StepArgs<float>& a, int ntx,
                                                 int tl, int b, int tid, int lane, int ly) {
    const int x0 = (tl % ntx) * kCTX, y0 = (tl / ntx) * kCTY;
    // a thread past the lattice edge gathers its periodic image: it is the
    // neighbour of the last in-range nodes
    const int x = (x0 + lane) % a.nx, y = (y0 + ly) % a.ny;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        int sx = x - pcx(p), sy = y - pcy(p);
        sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
        sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
        cp_async4(&sh.pop[b][p][tid], src + (long long)p * a.plane + (long long)sy * a.pitch + sx);
    }
    if (tid < kHalo) {
        int hx, hy;
        ring_pos(tid, hx, hy);
        const int gx = ((x0 - 1 + hx) % a.nx + a.nx) % a.nx, gy = ((y0 - 1 + hy) % a.ny + a.ny) % a.ny;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            int sx = gx - pcx(p), sy = gy - pcy(p);
            sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
            sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
            cp_async4(&sh.hpop[b][p][tid], src + (long long)p * a.plane + (long long)sy * a.pitch + sx);
        }
    }
    cp_async_commit();
}

}  // namespace mhd
