// state.cu -- kernels that convert between the stored state and host-side
// quantities (initial equilibrium, fields, single planes, the unstreamed
// pre-collision state), the slab exchange's row copies, the storage layout
// and the SM-count query the grid-stride launchers use.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

// ---- state conversion kernels ------------------------------------------

__device__ __forceinline__ void encode_d(double v, double& s) { s = v; }
__device__ __forceinline__ void encode_d(double v, float& s) { s = __double2float_rn(v); }
__device__ __forceinline__ void encode_d(double v, __half& s) { s = __double2half(v * 4096.0); }

// The initial equilibrium and the moments read back are evaluated in the
// compute type of the storage (FP64 for FP64, FP32 for FP32 and FP16S), as
// the step evaluates its collision: on GB300 FP64 arithmetic would make
// these memory-bound conversions bound by the FP64 units instead.
// T: the type of the field arrays (double, or float for the FP32 field
// calls: converted exactly to double or as the FP32 value); they may live in
// device memory or in pinned host memory mapped into the device's address
// space (one pass over the host link).  flags (may be null): the input
// checks of mhd_set_fields on the values read (bit 0 a non-finite field,
// bit 1 rho <= 0 or non-finite); the state is written either way.
template <int PREC, typename T>
__global__ void init_kernel(Layout L, void* buf, const T* rho, const T* ux, const T* uy, const T* bx,
                            const T* by, double rho0, int variant, int* flags) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    const long long n = (long long)L.nx * L.ny;
    int fl = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        const T vx = ux[k], vy = uy[k], wx = bx[k], wy = by[k];
        const double r = rho ? (double)rho[k] : rho0;
        if (flags) {
            if (!(isfinite(vx) && isfinite(vy) && isfinite(wx) && isfinite(wy))) fl |= 1;
            if (rho) fl |= !isfinite(r) ? 1 : (r > 0 ? 0 : 2);
        }
        C f[9], g[10];
        equilibrium<C>(C(r), C(vx), C(vy), C(wx), C(wy), C(rho0), variant, f, g);
        S* b = static_cast<S*>(buf);
        const long long o = (long long)y * L.pitch + x;
        for (int i = 0; i < 9; ++i) encode(f[i], b[(long long)i * L.plane + o]);
        for (int q = 0; q < 10; ++q) encode(g[q], b[(long long)(9 + q) * L.plane + o]);
    }
    if (flags) {
        fl = __reduce_or_sync(0xffffffffu, fl);
        if ((threadIdx.x & 31) == 0 && fl) atomicOr(flags, fl);
    }
}

template <int PREC, typename T>
__global__ void fields_kernel(Layout L, const void* buf, double rho0, T* rho, T* ux, T* uy, T* bx, T* by) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    const long long n = (long long)L.nx * L.ny;
    const S* b = static_cast<const S*>(buf);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        const long long o = (long long)y * L.pitch + x;
        C f[9], g[10];
        for (int i = 0; i < 9; ++i) f[i] = decode(b[(long long)i * L.plane + o]);
        for (int q = 0; q < 10; ++q) g[q] = decode(b[(long long)(9 + q) * L.plane + o]);
        const Moments<C> m = moments<C>(f, g, C(rho0));
        // the deviation keeps its relative precision; a float output is the
        // double value rounded to nearest
        if (rho) rho[k] = T(rho0 + (double)m.drho);
        if (ux) ux[k] = T(m.ux);
        if (uy) uy[k] = T(m.uy);
        if (bx) bx[k] = T(m.bx);
        if (by) by[k] = T(m.by);
    }
}

template <int PREC>
__global__ void plane_out_kernel(Layout L, const void* buf, int p, double shift, double* out) {
    using S = typename Prec<PREC>::S;
    const long long n = (long long)L.nx * L.ny;
    const S* b = static_cast<const S*>(buf) + (long long)p * L.plane;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        out[k] = (double)decode(b[(long long)y * L.pitch + x]) + shift;
    }
}

template <int PREC>
__global__ void plane_in_kernel(Layout L, void* buf, int p, double shift, const double* in) {
    using S = typename Prec<PREC>::S;
    const long long n = (long long)L.nx * L.ny;
    S* b = static_cast<S*>(buf) + (long long)p * L.plane;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
        encode_d(in[k] - shift, b[(long long)y * L.pitch + x]);
    }
}

// S_p(x) = F_p(x + c_p) (periodic): a stored state whose pull-gather gives
// back the pre-collision state F (packed FP32 deviations) at every node.
template <int PREC>
__global__ void unstream_kernel(Layout L, void* buf, const float* F) {
    using S = typename Prec<PREC>::S;
    const long long n = (long long)L.nx * L.ny;
    S* b = static_cast<S*>(buf);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(k / L.nx), x = (int)(k % L.nx);
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int xs = (x + pcx(p) + L.nx) % L.nx, ys = (y + pcy(p) + L.ny) % L.ny;
            encode_d((double)F[(long long)p * n + (long long)ys * L.nx + xs],
                     b[(long long)p * L.plane + (long long)y * L.pitch + x]);
        }
    }
}

int device_sms() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 152;
        cached[dev] = sms;
    }
    return cached[dev];
}

// grid-stride launches: at most 16 blocks of 256 threads per SM
static dim3 flat_grid(long long n) {
    long long b = (n + 255) / 256;
    const long long cap = 16LL * device_sms();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return dim3((unsigned)b);
}

#define MHD_DISPATCH(prec, KERNEL, grid, block, st, ...)                  \
    do {                                                                  \
        switch (prec) {                                                   \
        case 0: KERNEL<0><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        case 1: KERNEL<1><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        case 2: KERNEL<2><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        default: return cudaErrorInvalidValue;                            \
        }                                                                 \
    } while (0)

#define MHD_DISPATCH_T(prec, KERNEL, T, grid, block, st, ...)               \
    do {                                                                     \
        switch (prec) {                                                      \
        case 0: KERNEL<0, T><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        case 1: KERNEL<1, T><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        case 2: KERNEL<2, T><<<grid, block, 0, st>>>(__VA_ARGS__); break;    \
        default: return cudaErrorInvalidValue;                               \
        }                                                                    \
    } while (0)

template <typename T>
static cudaError_t launch_init_t(const Layout& L, int prec, void* buf, const T* rho, const T* ux, const T* uy,
                                 const T* bx, const T* by, double rho0, int variant, cudaStream_t st, int* flags) {
    MHD_DISPATCH_T(prec, init_kernel, T, flat_grid((long long)L.nx * L.ny), 256, st, L, buf, rho, ux, uy, bx,
                   by, rho0, variant, flags);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fields_t(const Layout& L, int prec, const void* buf, double rho0, T* rho, T* ux,
                                   T* uy, T* bx, T* by, cudaStream_t st) {
    MHD_DISPATCH_T(prec, fields_kernel, T, flat_grid((long long)L.nx * L.ny), 256, st, L, buf, rho0, rho, ux,
                   uy, bx, by);
    return cudaGetLastError();
}

cudaError_t launch_init(const Layout& L, int prec, void* buf, const double* rho, const double* ux,
                        const double* uy, const double* bx, const double* by, double rho0,
                        int variant, cudaStream_t st, int* flags) {
    return launch_init_t(L, prec, buf, rho, ux, uy, bx, by, rho0, variant, st, flags);
}

cudaError_t launch_init(const Layout& L, int prec, void* buf, const float* rho, const float* ux,
                        const float* uy, const float* bx, const float* by, double rho0, int variant,
                        cudaStream_t st, int* flags) {
    return launch_init_t(L, prec, buf, rho, ux, uy, bx, by, rho0, variant, st, flags);
}

cudaError_t launch_fields(const Layout& L, int prec, const void* buf, double rho0, double* rho,
                          double* ux, double* uy, double* bx, double* by, cudaStream_t st) {
    return launch_fields_t(L, prec, buf, rho0, rho, ux, uy, bx, by, st);
}

cudaError_t launch_fields(const Layout& L, int prec, const void* buf, double rho0, float* rho, float* ux,
                          float* uy, float* bx, float* by, cudaStream_t st) {
    return launch_fields_t(L, prec, buf, rho0, rho, ux, uy, bx, by, st);
}

// The row copies of a slab exchange on one device: for each listed plane p,
// `bytes` from src + p * src_plane + src_off to dst + p * dst_plane +
// dst_off, in 16-byte pieces (every address and size a multiple of 16).
__global__ void halo_rows_kernel(const char* __restrict__ src, char* __restrict__ dst, long long src_plane,
                                 long long dst_plane, long long src_off, long long dst_off, long long bytes,
                                 HaloPlanes hp) {
    const long long n16 = bytes / 16;
    for (int j = blockIdx.y; j < hp.n; j += gridDim.y) {
        const long long p = hp.p[j];
        const uint4* s = reinterpret_cast<const uint4*>(src + p * src_plane + src_off);
        uint4* d = reinterpret_cast<uint4*>(dst + p * dst_plane + dst_off);
        for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n16;
             k += (long long)gridDim.x * blockDim.x)
            d[k] = s[k];
    }
}

cudaError_t launch_halo_rows(const void* src, void* dst, long long src_plane, long long dst_plane, long long src_off,
                             long long dst_off, long long bytes, const HaloPlanes& hp, cudaStream_t st) {
    if (hp.n < 1 || hp.n > kStatePlanes || bytes % 16 || src_plane % 16 || dst_plane % 16 || src_off % 16 ||
        dst_off % 16 || reinterpret_cast<uintptr_t>(src) % 16 || reinterpret_cast<uintptr_t>(dst) % 16)
        return cudaErrorInvalidValue;
    const long long bx = std::max(1LL, std::min((bytes / 16 + 255) / 256, 64LL));
    halo_rows_kernel<<<dim3((unsigned)bx, (unsigned)hp.n), 256, 0, st>>>(
        static_cast<const char*>(src), static_cast<char*>(dst), src_plane, dst_plane, src_off, dst_off, bytes, hp);
    return cudaGetLastError();
}

// The exchanges of a whole slab group in one launch: block (x, job, k)
// copies a share of plane planes[k] of job's row, in 16-byte pieces.
__global__ void halo_jobs_kernel(const HaloJob* __restrict__ jobs, long long n16) {
    const HaloJob& j = jobs[blockIdx.y];
    const long long p = j.planes[blockIdx.z];
    const uint4* s = reinterpret_cast<const uint4*>(j.src + p * j.src_plane);
    uint4* d = reinterpret_cast<uint4*>(j.dst + p * j.dst_plane);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n16; k += (long long)gridDim.x * blockDim.x)
        d[k] = s[k];
}

cudaError_t launch_halo_jobs(const HaloJob* jobs, int njobs, long long row_bytes, cudaStream_t st) {
    if (njobs < 1 || njobs > 65535 || row_bytes % 16 || reinterpret_cast<uintptr_t>(jobs) % alignof(HaloJob))
        return cudaErrorInvalidValue;
    const long long n16 = row_bytes / 16;
    const long long bx = std::max(1LL, std::min((n16 + 255) / 256, 16LL));
    halo_jobs_kernel<<<dim3((unsigned)bx, (unsigned)njobs, 5), 256, 0, st>>>(jobs, n16);
    return cudaGetLastError();
}

cudaError_t launch_unstream(const Layout& L, int prec, void* buf, const float* F, cudaStream_t st) {
    MHD_DISPATCH(prec, unstream_kernel, flat_grid((long long)L.nx * L.ny), 256, st, L, buf, F);
    return cudaGetLastError();
}

static double plane_shift(int p, double rho0) { return p < 9 ? w_of(p) * rho0 : 0.0; }

cudaError_t launch_plane_out(const Layout& L, int prec, const void* buf, int p, double rho0,
                             double* out, cudaStream_t st) {
    MHD_DISPATCH(prec, plane_out_kernel, flat_grid((long long)L.nx * L.ny), 256, st, L, buf, p,
                 plane_shift(p, rho0), out);
    return cudaGetLastError();
}

cudaError_t launch_plane_in(const Layout& L, int prec, void* buf, int p, double rho0,
                            const double* in, cudaStream_t st) {
    MHD_DISPATCH(prec, plane_in_kernel, flat_grid((long long)L.nx * L.ny), 256, st, L, buf, p,
                 plane_shift(p, rho0), in);
    return cudaGetLastError();
}


Layout make_layout(int nx, int ny, int prec) {
    Layout L;
    L.nx = nx;
    L.ny = ny;
    L.esize = prec == 0 ? 8 : (prec == 1 ? 4 : 2);
    const long long row_align = 128 / L.esize;
    L.pitch = (nx + row_align - 1) / row_align * row_align;
    const long long pl_align = 256 / L.esize;
    L.plane = ((long long)ny * L.pitch + pl_align - 1) / pl_align * pl_align;
    return L;
}

}  // namespace mhd
