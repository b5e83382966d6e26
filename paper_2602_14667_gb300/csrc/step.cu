// step.cu -- the sm_103a kernels of the fused RR-MHD lattice Boltzmann step
// and their launcher.
//
// One kernel launch per time step (pull scheme): each thread gathers the
// post-collision populations f*_i(x - c_i, t-1), g*_j(x - e_j, t-1) of the
// previous step (task 6, streaming, read in pull form), runs tasks 1-5 of
// the paper's "Algorithm of computation" in registers, and writes f*(x, t),
// g*(x, t) to the other buffer.  Half-way bounce-back on wall axes:
// a population whose source node lies outside the lattice is the node's own
// post-collision population of the opposite direction.
//
// step_vec: periodic x axis, V consecutive x nodes per thread, one warp per
// row segment of 32*V nodes (step_row.cuh).  HBM traffic is one read and
// one write of the 19 planes.
// step_gen: x walls (any boundary), one node per thread, scalar loads.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

// Persistent: the grid holds as many blocks as are resident on the GPU at
// once and each block walks the tiles (rows_per_block rows x 32*V columns)
// with a fixed stride, so warps of one SM drift apart and the loads of one
// tile overlap the arithmetic of another.
// Off: int offsets when the state has fewer than 2^31 elements per buffer.
template <int PREC, int V, bool WALLY, typename Off>
__global__ void __launch_bounds__(512) step_vec(const StepArgs<typename Prec<PREC>::C> a, int nxb,
                                                int ntiles) {
    using S = typename Prec<PREC>::S;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int y = (t / nxb) * blockDim.y + threadIdx.y;
        if (y < a.ny)  // whole warp (one row per warp)
            step_row<PREC, V, WALLY, Off>(static_cast<const S*>(a.src), static_cast<S*>(a.dst), a.nx,
                                          a.ny, a.pitch, a.plane, a.np, t % nxb, y, threadIdx.x);
    }
}

template <int PREC>
__global__ void __launch_bounds__(512) step_gen(const StepArgs<typename Prec<PREC>::C> a) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= a.nx || y >= a.ny) return;
    C f[9], g[10];
    gather_node(static_cast<const S*>(a.src), x, y, a.nx, a.ny, a.pitch, a.plane, a.wall_x, a.wall_y,
                f, g);
    collide(f, g, a.np);
    S* dst = static_cast<S*>(a.dst);
    const long long o = (long long)y * a.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) encode(f[i], dst[(long long)i * a.plane + o]);
#pragma unroll
    for (int q = 0; q < 10; ++q) encode(g[q], dst[(long long)(9 + q) * a.plane + o]);
}

template <int PREC>
static cudaError_t launch_step_t(const StepLaunch& s, cudaStream_t st) {
    using C = typename Prec<PREC>::C;
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
    a.wall_x = s.wall_x;
    a.wall_y = s.wall_y;
    dim3 block(32, s.BY);
    const int cols = 32 * s.V;
    dim3 grid((s.L.nx + cols - 1) / cols, (s.L.ny + s.BY - 1) / s.BY);
    if (s.V == 1 && s.wall_x) {
        step_gen<PREC><<<grid, block, 0, st>>>(a);
        return cudaGetLastError();
    }
    const int nxb = grid.x, ntiles = grid.x * grid.y;
    // Resident warps per SM (the staging depth: how many row tiles, and
    // bytes of every plane, are in flight): the DRAM throughput of the
    // storage-bound kernels peaks with about 4 KB of every plane in flight
    // per SM (warps x 32 lanes x V elements); more concurrent row streams
    // lose bandwidth (FP32: 8 warps at V = 4 or 16 at V = 2; FP16S: 16 at
    // V = 4).  FP64 is bound by its arithmetic and keeps every resident
    // block.  The launch shape may set another depth (s.W).
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
    const bool small = (long long)kPlanes * s.L.plane < (1LL << 31);
    auto pick = [&](auto k32, auto k64) -> cudaError_t { return small ? go(k32) : go(k64); };
    switch (s.V) {
    case 1:
        return s.wall_y ? pick(step_vec<PREC, 1, true, int>, step_vec<PREC, 1, true, long long>)
                        : pick(step_vec<PREC, 1, false, int>, step_vec<PREC, 1, false, long long>);
    case 2:
        return s.wall_y ? pick(step_vec<PREC, 2, true, int>, step_vec<PREC, 2, true, long long>)
                        : pick(step_vec<PREC, 2, false, int>, step_vec<PREC, 2, false, long long>);
    case 4:
        if constexpr (PREC != 0)
            return s.wall_y ? pick(step_vec<PREC, 4, true, int>, step_vec<PREC, 4, true, long long>)
                            : pick(step_vec<PREC, 4, false, int>, step_vec<PREC, 4, false, long long>);
        return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

int step_rule_warps(int prec, int V) {
    const int esize = prec == 0 ? 8 : (prec == 1 ? 4 : 2);
    return prec == 0 ? 64 : std::max(1, 4096 / (32 * V * esize));
}

bool step_shape_ok(const Layout& L, int prec, int wall_x, int V, int BY) {
    if (BY < 1 || BY > 16) return false;
    if (V != 1 && V != 2 && V != 4) return false;
    if (prec == 0 && V > 2) return false;
    if (wall_x && V != 1) return false;
    if (L.nx % V) return false;
    return true;
}

cudaError_t launch_step(const StepLaunch& s, cudaStream_t st) {
    if (!step_shape_ok(s.L, s.prec, s.wall_x, s.V, s.BY)) return cudaErrorInvalidValue;
    switch (s.prec) {
    case 0: return launch_step_t<0>(s, st);
    case 1: return launch_step_t<1>(s, st);
    case 2: return launch_step_t<2>(s, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace mhd
