// inplace.cu -- kernels of the single-buffer (in-place) step: phase A
// (pull-gather, collide, write back into the gathered cells), phase B
// (local read, collide, canonical write) and the conversion of a streamed
// state back to the canonical layout without a collision.  The row bodies
// and the layout argument are in inplace_row.cuh.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "inplace.h"
#include "inplace_row.cuh"

namespace mhd {

// FP16S phase A (node pairs on FP32x2 beside the x-shift logic of both the
// gather and the write-back) runs in blocks of at most 256 threads, two of
// them per SM, i.e. at most 128 registers; at four nodes per lane it holds
// the populations as packed halves (aa_row_a_h4), which spills least under
// that cap (4096^2 in place: 71.6k MLUPS, against 70.7k with all four nodes
// in FP32 and about 150 registers, 68.0k with those capped at 128).
constexpr int aa_a_max_threads(int prec) { return prec == 2 ? 256 : 512; }

template <int PREC, int V, bool WALLY, typename Off>
__global__ void __launch_bounds__(aa_a_max_threads(PREC), PREC == 2 ? 2 : 1) aa_step_a(const StepArgs<typename Prec<PREC>::C> a, int nxb,
                                                 int ntiles) {
    using S = typename Prec<PREC>::S;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = (t / nxb) * blockDim.y + threadIdx.y;
        if (y < a.ny) {  // whole warp
            if constexpr (PREC == 2 && V == 4)
                aa_row_a_h4<WALLY, Off>(static_cast<S*>(a.dst), a.nx, a.ny, a.pitch, a.plane, a.np, t % nxb, y,
                                        threadIdx.x);
            else
                aa_row_a<PREC, V, WALLY, Off>(static_cast<S*>(a.dst), a.nx, a.ny, a.pitch, a.plane, a.np,
                                              t % nxb, y, threadIdx.x);
        }
    }
}

template <int PREC, int V, typename Off>
__global__ void __launch_bounds__(512) aa_step_b(const StepArgs<typename Prec<PREC>::C> a, int nxb,
                                                 int ntiles) {
    using S = typename Prec<PREC>::S;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = (t / nxb) * blockDim.y + threadIdx.y;
        if (y < a.ny)
            aa_row_b<PREC, V, Off>(static_cast<S*>(a.dst), a.nx, a.pitch, a.plane, a.np, t % nxb, y,
                                   threadIdx.x);
    }
}

// Streamed -> canonical without a collision: the canonical f*_q(x) sits in
// plane opp(q) at x + c_q, or in plane q at x where x + c_q crosses a y wall.
// Cell (x + c_q, opp(q)) and cell (x, q) trade places; taking q from the
// half of the directions that point "forward" visits every pair once.
template <int PREC>
__global__ void aa_unstream_kernel(Layout L, void* buf, int wall_y) {
    using S = typename Prec<PREC>::S;
    S* b = static_cast<S*>(buf);
    const long long n = (long long)L.nx * L.ny;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
#pragma unroll
        for (int q = 1; q < kPlanes; ++q) {
            const int cx = pcx(q), cy = pcy(q);
            if (!(cx > 0 || (cx == 0 && cy > 0))) continue;
            int xs = x + cx, ys = y + cy;
            if (wall_y && (ys < 0 || ys >= L.ny)) continue;
            xs = xs < 0 ? xs + L.nx : (xs >= L.nx ? xs - L.nx : xs);
            ys = ys < 0 ? ys + L.ny : (ys >= L.ny ? ys - L.ny : ys);
            S* c1 = b + (long long)popp(q) * L.plane + (long long)ys * L.pitch + xs;
            S* c2 = b + (long long)q * L.plane + (long long)y * L.pitch + x;
            const S t = *c1;
            *c1 = *c2;
            *c2 = t;
        }
    }
}

template <int PREC>
static cudaError_t launch_aa_t(const StepLaunch& s, int phase, cudaStream_t st) {
    using C = typename Prec<PREC>::C;
    StepArgs<C> a;
    a.src = s.dst;
    a.dst = s.dst;
    a.nx = s.L.nx;
    a.ny = s.L.ny;
    a.pitch = s.L.pitch;
    a.plane = s.L.plane;
    a.np.omega = C(s.omega);
    a.np.omega_m = C(s.omega_m);
    a.np.rho0 = C(s.rho0);
    a.np.variant = s.variant;
    a.np.collision = s.collision;
    a.np.mag_collision = s.mag_collision;
    a.wall_x = 0;
    a.wall_y = s.wall_y;
    const dim3 block(32, s.BY);
    const int nxb = (s.L.nx + 32 * s.V - 1) / (32 * s.V);
    const int ntiles = nxb * ((s.L.ny + s.BY - 1) / s.BY);
    // persistent grid: as many blocks as are resident at once, with the
    // resident warps capped as for the pull step (by default about 4 KB of
    // every plane in flight per SM; FP64 uncapped; s.W sets another depth)
    const int max_warps = s.W > 0 ? s.W : step_rule_warps(PREC, s.V);
    const int warp_cap = std::max(1, max_warps / s.BY);
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0, sms = 0, dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * s.BY, 0);
        if (e != cudaSuccess) return e;
        per_sm = std::min(std::max(1, per_sm), warp_cap);
        const int blocks = std::max(1, std::min(ntiles, per_sm * sms));
        kernel<<<blocks, block, 0, st>>>(a, nxb, ntiles);
        return cudaGetLastError();
    };
    auto pick = [&](auto a_periodic, auto a_wall, auto b) -> cudaError_t {
        if (phase == 1) return go(b);
        return s.wall_y ? go(a_wall) : go(a_periodic);
    };
    // 32-bit element offsets while the state has fewer than 2^31 elements
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto pick_v = [&](auto v) -> cudaError_t {
        constexpr int V = decltype(v)::value;
        if (small)
            return pick(aa_step_a<PREC, V, false, int>, aa_step_a<PREC, V, true, int>, aa_step_b<PREC, V, int>);
        return pick(aa_step_a<PREC, V, false, long long>, aa_step_a<PREC, V, true, long long>,
                    aa_step_b<PREC, V, long long>);
    };
    switch (s.V) {
    case 1: return pick_v(std::integral_constant<int, 1>{});
    case 2: return pick_v(std::integral_constant<int, 2>{});
    case 4:
        if constexpr (PREC != 0) return pick_v(std::integral_constant<int, 4>{});
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_aa_step(const StepLaunch& s, int phase, cudaStream_t st) {
    if (s.wall_x || s.src != s.dst || (phase != 0 && phase != 1)) return cudaErrorInvalidValue;
    if (!step_shape_ok(s.L, s.prec, 0, s.V, s.BY)) return cudaErrorInvalidValue;
    if (32 * s.BY > aa_a_max_threads(s.prec)) return cudaErrorInvalidValue;
    switch (s.prec) {
    case 0: return launch_aa_t<0>(s, phase, st);
    case 1: return launch_aa_t<1>(s, phase, st);
    case 2: return launch_aa_t<2>(s, phase, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_aa_unstream(const Layout& L, int prec, void* buf, int wall_y, cudaStream_t st) {
    long long blocks = ((long long)L.nx * L.ny + 255) / 256;
    blocks = std::max(1LL, std::min(blocks, 16LL * device_sms()));
    switch (prec) {
    case 0: aa_unstream_kernel<0><<<(unsigned)blocks, 256, 0, st>>>(L, buf, wall_y); break;
    case 1: aa_unstream_kernel<1><<<(unsigned)blocks, 256, 0, st>>>(L, buf, wall_y); break;
    case 2: aa_unstream_kernel<2><<<(unsigned)blocks, 256, 0, st>>>(L, buf, wall_y); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mhd
