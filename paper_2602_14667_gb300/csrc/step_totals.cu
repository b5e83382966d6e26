// step_totals.cu -- the fused step of a sample step: the step of step_vec
// (the pull gather of step_row, the collision, aligned vector stores) that
// also reduces the point totals of the pre-collision state it gathers.
// These are the global diagnostics that need no neighbour of a node: mass,
// momentum, kinetic and magnetic energy, cross helicity, the sum of b and
// the largest |j_z| (Eq. current).  They are formed from the populations
// the warp already holds in registers for the collision, so a sample step
// reads and writes the state once, like every other step; div b and the
// vorticity need the 3 x 3 neighbourhood and stay with the diagnostics pass.
// Arithmetic and partial slots are the diagnostics' (diag_device.cuh): the
// per-node quantities in the compute type (FP32 for FP32 and FP16S
// storage), compensated FP32 sums per lane, FP64 only in the warp, block
// and fixed-order final reductions.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "diag_device.cuh"
#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

namespace {

constexpr int kTotWarps = 8;  // warps (rows) per block at most

// The persistent row walk of step_vec; slots as in the diagnostics:
// 0 sum (rho - rho0), 1 mom_x, 2 mom_y, 3 sum |u|^2/2, 4 sum |b|^2/2,
// 5 sum u.b, 6 sum b_x, 7 sum b_y, 11 max |j_z|; 8, 9, 10, 12 zero.
template <int PREC, int V, bool WALLY, typename Off>
__global__ void __launch_bounds__(kTotWarps * 32) step_vec_totals(const StepArgs<typename Prec<PREC>::C> a,
                                                                   int nxb, int ntiles,
                                                                   double* __restrict__ partials) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    using MB = AbsBits<C>;
    __shared__ double red[kTotWarps][kDiagSlots];
    const int lane = threadIdx.x, warp = threadIdx.y;
    // FP16S populations stay in the storage units (2^12 x deviation)
    const C unit = PREC == 2 ? C(kHalfInvScale) : C(1);
    constexpr bool kScaled = PREC == 2;
    constexpr int kMode = PREC == 2 ? kPairs : kNative;
    LaneSum<C> ls[8];
    typename MB::T mjz = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = (t / nxb) * blockDim.y + threadIdx.y;
        if (y >= a.ny) continue;  // whole warp (one row per warp)
        const int xb = t % nxb;
        C v[kPlanes][V];
        if (!gather_row<PREC, V, WALLY, Off>(static_cast<const S*>(a.src), a.nx, a.ny, a.pitch, a.plane, xb, y,
                                             lane, v))
            continue;
        // the point quantities of the V nodes before they collide
        C ps[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) ps[q] = C(0);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            C f[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = v[i][k];
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = v[9 + q][k];
            const NodeMom<C> n = node_moments(f, g, unit, a.np.rho0);
            add_point_sums(n, ps);
            mjz = max(mjz, MB::of(node_current(n, a.np.omega_m, C(1))));
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) ls[q].add(ps[q]);
        collide_nodes<C, V, kScaled, kMode>(v, a.np);
        const int x0 = (xb * 32 + lane) * V;
        const Off o_0 = (Off)y * (Off)a.pitch, pl = (Off)a.plane;
        using Codec = StepCodec<S, V>;
        S* dst = static_cast<S*>(a.dst);
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            S r[V];
            Codec::to_storage(v[p], r);
            VecIO<S, V>::store(dst + ((Off)p * pl + o_0 + x0), r);
        }
    }
    // warp sums and maxima, then the block's warps in order
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double s = warp_sum(ls[q].take());
        if (lane == 0) red[warp][q] = s;
    }
    const unsigned long long m11 = warp_max_bits(dbits(MB::value(mjz)));
    if (lane == 0) {
        red[warp][8] = red[warp][9] = red[warp][10] = red[warp][12] = 0.0;
        red[warp][11] = __longlong_as_double((long long)m11);
    }
    __syncthreads();
    const int tid = threadIdx.y * 32 + lane;
    if (tid < kDiagSlots) {
        const int q = tid;
        double s = red[0][q];
        for (int w = 1; w < (int)blockDim.y; ++w)
            s = q < 10 ? s + red[w][q] : __longlong_as_double((long long)max_bits(dbits(s), dbits(red[w][q])));
        partials[(long long)blockIdx.x * kDiagSlots + q] = s;
    }
}

}  // namespace

template <int PREC>
static cudaError_t launch_step_totals_t(const StepLaunch& s, double* partials, int capacity, double* totals,
                                        cudaStream_t st) {
    using C = typename Prec<PREC>::C;
    if (s.wall_x || capacity < 1) return cudaErrorInvalidValue;
    if (!step_shape_ok(s.L, PREC, 0, s.V, s.BY)) return cudaErrorInvalidValue;
    StepArgs<C> a;
    a.src = s.src;
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
    // the lattice's launch shape with at most kTotWarps rows per block (the
    // row-to-block map does not change the populations a step writes)
    const int BY = std::min(s.BY, kTotWarps);
    const dim3 block(32, BY);
    const int cols = 32 * s.V;
    const int nxb = (s.L.nx + cols - 1) / cols, ntiles = nxb * ((s.L.ny + BY - 1) / BY);
    const int max_warps = s.W > 0 ? s.W : step_rule_warps(PREC, s.V);
    const int warp_cap = std::max(1, max_warps / BY);
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 32 * BY, 0);
        if (e != cudaSuccess) return e;
        per_sm = std::min(std::max(1, per_sm), warp_cap);
        const int blocks = std::max(1, std::min({ntiles, per_sm * device_sms(), capacity}));
        kernel<<<blocks, block, 0, st>>>(a, nxb, ntiles, partials);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_diag_final(partials, blocks, s.rho0 * (double)s.L.nx * (double)s.L.ny, totals, st);
    };
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto pick = [&](auto k32, auto k64) -> cudaError_t { return small ? go(k32) : go(k64); };
    switch (s.V) {
    case 1:
        return s.wall_y ? pick(step_vec_totals<PREC, 1, true, int>, step_vec_totals<PREC, 1, true, long long>)
                        : pick(step_vec_totals<PREC, 1, false, int>, step_vec_totals<PREC, 1, false, long long>);
    case 2:
        return s.wall_y ? pick(step_vec_totals<PREC, 2, true, int>, step_vec_totals<PREC, 2, true, long long>)
                        : pick(step_vec_totals<PREC, 2, false, int>, step_vec_totals<PREC, 2, false, long long>);
    case 4:
        if constexpr (PREC != 0)
            return s.wall_y ? pick(step_vec_totals<PREC, 4, true, int>, step_vec_totals<PREC, 4, true, long long>)
                            : pick(step_vec_totals<PREC, 4, false, int>, step_vec_totals<PREC, 4, false, long long>);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_totals(const StepLaunch& s, double* partials, int capacity, double* totals,
                               cudaStream_t st) {
    switch (s.prec) {
    case 0: return launch_step_totals_t<0>(s, partials, capacity, totals, st);
    case 1: return launch_step_totals_t<1>(s, partials, capacity, totals, st);
    case 2: return launch_step_totals_t<2>(s, partials, capacity, totals, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mhd
