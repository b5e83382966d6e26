// noalloc.cu -- allocation-free variant of the global diagnostics.
//
// mhd_get_totals reduces through a per-lattice device buffer of per-block
// partial sums that mhd_create allocates.  Some callers cannot allocate
// device memory when they need the diagnostics: a host framework that has
// already reserved the whole GPU for its own memory pool and only lends out
// pointers it owns, or a latency-critical loop that must not call cudaMalloc
// because it synchronises the device and stalls the other streams.
// mhd_totals_noalloc serves them: it takes the state from caller-owned device
// memory, reduces through a fixed scratch array compiled into the library,
// and writes the totals to a caller-owned struct.  It allocates nothing.
//
// The scratch is one file-scope __device__ array (kNoallocScratchDoubles
// doubles, about 1.7 MB), created when the library is loaded and held by
// every GPU that loads the library until the process exits.  It holds the
// per-block partials of at most kNoallocMaxBlocks blocks; the diagnostics
// grid is persistent (its blocks walk the lattice's tiles) and is capped at
// that count, so the array bounds no lattice size.  In host code the
// array's name is only a host-side stand-in, so each device's address is
// looked up with cudaGetSymbolAddress, with that device current, on the
// first call made in the device's current context, and passed to the
// kernels.  The lookup is keyed on the context's unique id: after a
// cudaDeviceReset the runtime creates a new context, in which the module
// holding the array may sit at another address, and the first call there
// looks it up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mhd.h"
#include "internal.h"

namespace {

// Per-block partials of the diagnostics kernel (kDiagSlots doubles for each
// of at most kNoallocMaxBlocks blocks), then kDiagSlots doubles of totals.
constexpr long long kNoallocMaxBlocks = 16384;
constexpr long long kNoallocScratchDoubles = kNoallocMaxBlocks * mhd::kDiagSlots + 16;

static __device__ __align__(256) double g_noalloc_scratch[kNoallocScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct ScratchCache {
    unsigned long long ctx_id;  // id of the context the address belongs to
    double* ptr;
};
ScratchCache g_scratch[kMaxDevices] = {};

mhd_status nfail(mhd_status s, const std::string& m) {
    mhd::set_last_error(m);
    return s;
}

mhd_status ncuda(cudaError_t e, const char* what) {
    return nfail(MHD_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

// Unique id of the calling thread's current context (0 if the driver
// cannot tell).  The two driver calls are reached through the runtime's
// entry-point query, so the library needs no link against the driver.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* fc = nullptr;
        void* fi = nullptr;
        cudaDriverEntryPointQueryResult qc, qi;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fc, 12000, cudaEnableDefault, &qc) == cudaSuccess &&
            qc == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &fi, 12000, cudaEnableDefault, &qi) == cudaSuccess &&
            qi == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(fc);
            get_id = reinterpret_cast<GetId>(fi);
        }
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current device's current
// context: looked up on the first call made in that context (with the
// device current) and kept; a context the driver cannot identify gets a
// fresh lookup on every call.
mhd_status scratch_on_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return ncuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return nfail(MHD_ECUDA, "device ordinal out of range");
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (id == 0 || g_scratch[dev].ctx_id != id || !g_scratch[dev].ptr) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return ncuda(e, "cudaGetSymbolAddress(scratch)");
        g_scratch[dev].ctx_id = id;
        g_scratch[dev].ptr = static_cast<double*>(ptr);
    }
    *out = g_scratch[dev].ptr;
    return MHD_OK;
}

}  // namespace

extern "C" mhd_status mhd_totals_noalloc(const void* state, const void* prev_state, int nx, int ny,
                                         const mhd_params* p, void* stream, mhd_totals* out) {
    if (!state || !p || !out) return nfail(MHD_EINVAL, "NULL argument");
    if (nx < 2 || ny < 2) return nfail(MHD_EINVAL, "nx and ny must be >= 2");
    if (!(p->tau_m > 0.5) || !std::isfinite(p->tau_m) || !(p->rho0 > 0) || !std::isfinite(p->rho0))
        return nfail(MHD_EINVAL, "tau_m must be > 1/2 and rho0 > 0");
    if (p->precision < MHD_FP64 || p->precision > MHD_FP16S) return nfail(MHD_EINVAL, "unknown precision");
    if ((p->bc_x != MHD_PERIODIC && p->bc_x != MHD_WALL) || (p->bc_y != MHD_PERIODIC && p->bc_y != MHD_WALL))
        return nfail(MHD_EINVAL, "bc_x / bc_y must be MHD_PERIODIC or MHD_WALL");
    // Packed layout of mhd_get_state: plane after plane, nx*ny elements each.
    mhd::Layout L;
    L.nx = nx;
    L.ny = ny;
    L.esize = p->precision == MHD_FP64 ? 8 : (p->precision == MHD_FP32 ? 4 : 2);
    L.pitch = nx;
    L.plane = (long long)nx * ny;
    // A state larger than the device's memory cannot be valid: reject it
    // before anything is launched (a smaller wrong size cannot be told from
    // a right one; the caller must pass the state's true extent).
    {
        size_t free_b = 0, total = 0;
        const cudaError_t e = cudaMemGetInfo(&free_b, &total);
        if (e != cudaSuccess) return ncuda(e, "cudaMemGetInfo");
        const double bytes = (double)mhd::kStatePlanes * (double)L.plane * (double)L.esize;
        if (bytes > (double)total)
            return nfail(MHD_EINVAL, "lattice too large for mhd_totals_noalloc: its state (" + std::to_string(bytes) +
                                         " bytes) exceeds the device's memory");
    }
    double* scratch = nullptr;
    mhd_status s = scratch_on_current_device(&scratch);
    if (s != MHD_OK) return s;
    double* totals_d = scratch + kNoallocMaxBlocks * mhd::kDiagSlots;

    mhd::DiagLaunch d;
    d.L = L;
    d.prec = p->precision;
    d.prev = prev_state;
    d.cur = state;
    d.mode = prev_state ? 0 : 1;
    d.omega_m = 1.0 / p->tau_m;
    d.rho0 = p->rho0;
    const double om1 = 1.0 - d.omega_m;
    d.neq_scale = prev_state ? 1.0 : (std::fabs(om1) < 1e-12 ? 0.0 : 1.0 / om1);
    d.wall_x = p->bc_x == MHD_WALL;
    d.wall_y = p->bc_y == MHD_WALL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // Every per-block slot that diag_final reads is written by the first
    // kernel of this call and the totals slots by diag_final, so nothing left
    // in the array by an earlier call is read and nothing needs clearing.
    // The grid is capped at the blocks the array has room for.
    cudaError_t e = mhd::launch_diag(d, scratch, (int)kNoallocMaxBlocks, totals_d, st);
    if (e == cudaErrorInvalidValue)
        return nfail(MHD_EINVAL, "lattice too large for mhd_totals_noalloc: its tile count exceeds the int range");
    if (e != cudaSuccess) return ncuda(e, "diagnostics kernel");
    double t[mhd::kDiagSlots];
    e = cudaMemcpyAsync(t, totals_d, sizeof t, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ncuda(e, "D2H totals");
    const double n = (double)nx * ny;
    out->mass = t[0];
    out->mom_x = t[1];
    out->mom_y = t[2];
    out->e_kin = t[3] / n;
    out->e_mag = t[4] / n;
    out->cross_hel = t[5] / n;
    out->bsum_x = t[6];
    out->bsum_y = t[7];
    out->divb_rms = t[9] > 0 ? std::sqrt(t[8] / t[9]) : 0.0;
    out->divb_max = t[10];
    out->jz_max = t[11];
    out->omega_max = t[12];
    out->step = 0;
    for (int k = 0; k < mhd::kDiagSlots; ++k)
        if (!std::isfinite(t[k])) return nfail(MHD_EUNSTABLE, "non-finite diagnostics: the run blew up");
    return MHD_OK;
}
