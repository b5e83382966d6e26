// diag.cu -- the global diagnostics of a lattice: mass, momentum, kinetic
// and magnetic energy, cross helicity, sum of b, div b (rms and max) and the
// maxima of the current density and the vorticity, reduced on the device in
// a fixed order.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

// ---- diagnostics ----------------------------------------------------------
// Persistent grid (the blocks resident at once, at most one per tile); each
// block walks 32 x 8 node tiles with a fixed stride.  The moments of a tile
// plus a one-node halo are staged in shared memory for the isotropic
// gradient stencil.  Per-node contributions are accumulated in FP64 in
// registers over all the block's tiles, then reduced once with warp
// shuffles and across warps in shared memory into kDiagSlots partials per
// block:
//   0 mass, 1 mom_x, 2 mom_y, 3 sum |u|^2/2, 4 sum |b|^2/2, 5 sum u.b,
//   6 sum b_x, 7 sum b_y, 8 sum (div b)^2, 9 #gradient nodes,
//   10 max |div b|, 11 max |j_z|, 12 max |omega_z|.
// The FP64 units are the bound (two FP64 instructions per clock per SM), so
// the count is kept as an integer and the three maxima, all of
// non-negative values, are taken on the bit patterns of the doubles with
// integer instructions (a NaN, whose pattern is above every finite value's,
// reaches the totals).
constexpr int kDTX = 32, kDTY = 8, kDHX = kDTX + 2, kDHY = kDTY + 2;

template <typename C> struct DiagArgs {
    const void* prev;
    const void* cur;
    int nx, ny;
    long long pitch, plane;
    C omega_m, rho0, neq_scale;
    int wall_x, wall_y;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_max_bits(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_down_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}
__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}
__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

template <int PREC, int MODE>
__global__ void __launch_bounds__(256) diag_kernel(const DiagArgs<typename Prec<PREC>::C> a, int tiles_x,
                                                   int ntiles, double* __restrict__ partials) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    __shared__ C sm[4][kDHY][kDHX];  // ux, uy, bx, by
    __shared__ double red[8][kDiagSlots];
    const int tid = threadIdx.y * kDTX + threadIdx.x;
    double acc[8];  // slots 0..7
    double div2 = 0.0;
    long long cnt = 0;
    unsigned long long mdiv = 0, mjz = 0, mvort = 0;
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[s] = 0.0;

    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int tx0 = (t % tiles_x) * kDTX, ty0 = (t / tiles_x) * kDTY;
        for (int r = tid; r < kDHX * kDHY; r += kDTX * kDTY) {
            const int hx = r % kDHX, hy = r / kDHX;
            int gx = tx0 - 1 + hx, gy = ty0 - 1 + hy;
            const bool interior = hx >= 1 && hx <= kDTX && hy >= 1 && hy <= kDTY && gx < a.nx && gy < a.ny;
            bool have = true;
            // (a tile may reach several periods past a lattice narrower than it)
            if (a.wall_x) have = have && gx >= 0 && gx < a.nx;
            else gx = ((gx % a.nx) + a.nx) % a.nx;
            if (a.wall_y) have = have && gy >= 0 && gy < a.ny;
            else gy = ((gy % a.ny) + a.ny) % a.ny;
            C ux = 0, uy = 0, bx = 0, by = 0;
            if (have) {
                C f[9], g[10];
                if (MODE == 0) {
                    gather_node(static_cast<const S*>(a.prev), gx, gy, a.nx, a.ny, a.pitch, a.plane,
                                a.wall_x, a.wall_y, f, g);
                } else {
                    const S* b = static_cast<const S*>(a.cur);
                    const long long o = (long long)gy * a.pitch + gx;
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) {
                        const C val = decode(b[(long long)p * a.plane + o]);
                        if (p < 9) f[p] = val; else g[p - 9] = val;
                    }
                }
                const Moments<C> m = moments(f, g, a.rho0);
                ux = m.ux; uy = m.uy; bx = m.bx; by = m.by;
                if (interior) {
                    const double rho = (double)m.rho, dux = (double)ux, duy = (double)uy;
                    const double dbx = (double)bx, dby = (double)by;
                    acc[0] += rho;
                    acc[1] += rho * dux;
                    acc[2] += rho * duy;
                    acc[3] += 0.5 * (dux * dux + duy * duy);
                    acc[4] += 0.5 * (dbx * dbx + dby * dby);
                    acc[5] += dux * dbx + duy * dby;
                    acc[6] += dbx;
                    acc[7] += dby;
                    const C jz = current_density(g, ux, uy, bx, by, a.omega_m, a.neq_scale);
                    mjz = max_bits(mjz, abs_bits((double)jz));
                }
            }
            sm[0][hy][hx] = ux; sm[1][hy][hx] = uy; sm[2][hy][hx] = bx; sm[3][hy][hx] = by;
        }
        __syncthreads();
        {
            const int lx = threadIdx.x, ly = threadIdx.y;
            const int x = tx0 + lx, y = ty0 + ly;
            bool ok = x < a.nx && y < a.ny;
            if (a.wall_x) ok = ok && x >= 1 && x <= a.nx - 2;
            if (a.wall_y) ok = ok && y >= 1 && y <= a.ny - 2;
            if (ok) {
                // d_a phi = 3 sum_i w_i phi(x + c_i) c_ia
                auto dx = [&](int q) {
                    const C e = sm[q][ly + 1][lx + 2] - sm[q][ly + 1][lx];
                    const C d = (sm[q][ly + 2][lx + 2] - sm[q][ly + 2][lx]) + (sm[q][ly][lx + 2] - sm[q][ly][lx]);
                    return (double)(C(1.0 / 3.0) * e + C(1.0 / 12.0) * d);
                };
                auto dy = [&](int q) {
                    const C e = sm[q][ly + 2][lx + 1] - sm[q][ly][lx + 1];
                    const C d = (sm[q][ly + 2][lx + 2] - sm[q][ly][lx + 2]) + (sm[q][ly + 2][lx] - sm[q][ly][lx]);
                    return (double)(C(1.0 / 3.0) * e + C(1.0 / 12.0) * d);
                };
                const double div = dx(2) + dy(3);
                const double vort = dx(1) - dy(0);
                div2 += div * div;
                ++cnt;
                mdiv = max_bits(mdiv, abs_bits(div));
                mvort = max_bits(mvort, abs_bits(vort));
            }
        }
        __syncthreads();  // the next tile overwrites sm
    }
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const double v = warp_sum(acc[s]);
        if (lane == 0) red[warp][s] = v;
    }
    {
        const double v8 = warp_sum(div2), v9 = warp_sum((double)cnt);
        const unsigned long long m10 = warp_max_bits(mdiv), m11 = warp_max_bits(mjz), m12 = warp_max_bits(mvort);
        if (lane == 0) {
            red[warp][8] = v8;
            red[warp][9] = v9;
            red[warp][10] = __longlong_as_double((long long)m10);
            red[warp][11] = __longlong_as_double((long long)m11);
            red[warp][12] = __longlong_as_double((long long)m12);
        }
    }
    __syncthreads();
    if (tid < kDiagSlots) {
        double v = red[0][tid];
        for (int w = 1; w < 8; ++w)
            v = tid < 10 ? v + red[w][tid]
                         : __longlong_as_double((long long)max_bits(abs_bits(v), abs_bits(red[w][tid])));
        partials[(long long)blockIdx.x * kDiagSlots + tid] = v;
    }
}

// Fixed-order final reduction of the per-block partials (one block).
__global__ void __launch_bounds__(256) diag_final(const double* __restrict__ partials, int nblocks,
                                                  double* __restrict__ totals) {
    __shared__ double red[8][kDiagSlots];
    double acc[10];
    unsigned long long mx[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < 10; ++s) acc[s] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int s = 0; s < 10; ++s) acc[s] += partials[(long long)b * kDiagSlots + s];
#pragma unroll
        for (int s = 0; s < 3; ++s) mx[s] = max_bits(mx[s], abs_bits(partials[(long long)b * kDiagSlots + 10 + s]));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 10; ++s) {
        const double v = warp_sum(acc[s]);
        if (lane == 0) red[warp][s] = v;
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const unsigned long long v = warp_max_bits(mx[s]);
        if (lane == 0) red[warp][10 + s] = __longlong_as_double((long long)v);
    }
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int s = threadIdx.x;
        double v = red[0][s];
        for (int w = 1; w < 8; ++w)
            v = s < 10 ? v + red[w][s] : __longlong_as_double((long long)max_bits(abs_bits(v), abs_bits(red[w][s])));
        totals[s] = v;
    }
}

int diag_blocks(const Layout& L) {
    return ((L.nx + kDTX - 1) / kDTX) * ((L.ny + kDTY - 1) / kDTY);
}

template <int PREC>
static cudaError_t launch_diag_t(const DiagLaunch& d, double* partials, int* nblocks, cudaStream_t st) {
    using C = typename Prec<PREC>::C;
    DiagArgs<C> a;
    a.prev = d.prev;
    a.cur = d.cur;
    a.nx = d.L.nx;
    a.ny = d.L.ny;
    a.pitch = d.L.pitch;
    a.plane = d.L.plane;
    a.omega_m = C(d.omega_m);
    a.rho0 = C(d.rho0);
    a.neq_scale = C(d.neq_scale);
    a.wall_x = d.wall_x;
    a.wall_y = d.wall_y;
    const int tiles_x = (d.L.nx + kDTX - 1) / kDTX;
    const int ntiles = diag_blocks(d.L);
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0, sms = 0, dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDTX * kDTY, 0);
        if (e != cudaSuccess) return e;
        *nblocks = std::max(1, std::min(ntiles, std::max(1, per_sm) * sms));
        kernel<<<*nblocks, dim3(kDTX, kDTY), 0, st>>>(a, tiles_x, ntiles, partials);
        return cudaGetLastError();
    };
    return d.mode == 0 ? go(diag_kernel<PREC, 0>) : go(diag_kernel<PREC, 1>);
}

cudaError_t launch_diag(const DiagLaunch& d, double* partials, double* totals, cudaStream_t st) {
    cudaError_t e;
    int nblocks = 0;
    switch (d.prec) {
    case 0: e = launch_diag_t<0>(d, partials, &nblocks, st); break;
    case 1: e = launch_diag_t<1>(d, partials, &nblocks, st); break;
    case 2: e = launch_diag_t<2>(d, partials, &nblocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    diag_final<<<1, 256, 0, st>>>(partials, nblocks, totals);
    return cudaGetLastError();
}

}  // namespace mhd
