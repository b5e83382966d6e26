// api.cu -- C ABI of the single-lattice RR-MHD solver (declared in
// include/mhd.h): argument checking, device buffers, CUDA-graph capture of
// the step loop, diagnostics, checkpointing and the launch-shape autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "closure_internal.h"
#include "inplace.h"
#include "internal.h"
#include "lbm_device.cuh"

namespace {

thread_local std::string g_err;

mhd_status fail(mhd_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

mhd_status cuda_fail(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? MHD_ENOMEM : MHD_ECUDA, m);
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int kGraphSteps = 64;  // steps per captured graph (even: ends on the same buffer)

bool finite_array(const double* a, long long n) {
    for (long long k = 0; k < n; ++k)
        if (!std::isfinite(a[k])) return false;
    return true;
}

// Input check of mhd_set_fields on the device copies: bit 0 of *flags for a
// non-finite field value, bit 1 for rho <= 0 (or non-finite rho).
template <typename T>
__global__ void check_fields_kernel(const T* ux, const T* uy, const T* bx, const T* by, const T* rho, long long n,
                                    int* flags) {
    int f = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        if (!(isfinite(ux[k]) && isfinite(uy[k]) && isfinite(bx[k]) && isfinite(by[k]))) f |= 1;
        if (rho) f |= !isfinite(rho[k]) ? 1 : (rho[k] > 0 ? 0 : 2);
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

}  // namespace

void mhd::set_last_error(const std::string& msg) { g_err = msg; }

void mhd_internal_closure_params(const mhd_mlp* m, mhd::ClosureParamsDev* cp);

struct mhd_lattice {
    int nx = 0, ny = 0;
    mhd_params p{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    mhd::Layout L{};
    void* buf[2] = {nullptr, nullptr};  // in place: buf[0] only
    // slab (bc_y = MHD_HALO): each buffer holds ny + 2 rows, ghost rows
    // first and last; buf[] point at row 0, alloc[] at the ghost row below,
    // and Lx describes the ny + 2 rows the step runs over
    bool halo = false;
    mhd::Layout Lx{};
    void* alloc[2] = {nullptr, nullptr};
    cudaEvent_t xev = nullptr;  // marks the state a slab exchange copies from
    int cur = 0;
    bool in_place = false;
    bool aa_streamed = false;  // in place, after an odd number of steps: streamed layout
    bool fields_set = false;
    bool prev_valid = false;  // buf[cur^1] holds the state the last step read
    bool state_is_eq = false; // current state has zero non-equilibrium
    long long step = 0;
    double* io = nullptr;     // 5*n doubles, lazily allocated
    double* partials = nullptr;
    double* totals_d = nullptr;
    double* totals_h = nullptr;  // pinned
    int* flags_d = nullptr;      // device word of the input checks
    mhd_kernel_config cfg{1, 8};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    void* closure_buf = nullptr;  // lattice-owned copy of the closure's inference parameters
    int closure_kind = MHD_CLOSURE_WARP_MMA;
    mhd::ClosureParamsDev closure{};
    // the MLP runs on every closure_interval-th step (counted by
    // closure_count since the last change of state or closure) and its
    // output, kept in da (3 planes of nx*ny floats), serves the steps between
    int closure_interval = 1;
    long long closure_count = 0;
    float* da = nullptr;

    long long n() const { return (long long)nx * ny; }
    size_t buf_bytes() const { return (size_t)mhd::kStatePlanes * L.plane * L.esize; }
};

namespace {

mhd::StepLaunch step_launch(const mhd_lattice* l, int from) {
    mhd::StepLaunch s;
    s.L = l->L;
    s.prec = l->p.precision;
    s.src = l->buf[from];
    s.dst = l->buf[from ^ 1];
    s.omega = 1.0 / l->p.tau_f;
    s.omega_m = 1.0 / l->p.tau_m;
    s.rho0 = l->p.rho0;
    s.variant = l->p.eq_variant;
    s.collision = l->p.collision;
    s.mag_collision = l->p.mag_collision;
    s.wall_x = l->p.bc_x == MHD_WALL;
    s.wall_y = l->p.bc_y == MHD_WALL;
    s.V = l->cfg.nodes_per_thread;
    s.BY = l->cfg.rows_per_block;
    s.W = l->cfg.warps_per_sm;
    if (l->halo) {
        // A slab steps as a periodic lattice of its ny + 2 rows: rows 0..ny-1
        // pull from the ghost rows, which hold the neighbours' edge rows; the
        // ghost rows' own update reads stale values and is overwritten by the
        // next exchange.
        s.L = l->Lx;
        s.src = l->alloc[from];
        s.dst = l->alloc[from ^ 1];
    }
    return s;
}

// One step from buffer `from`.  A closure lattice evaluates its MLP when
// `count` (its closure step count) is a multiple of the interval, and
// otherwise reuses the stored correction.
cudaError_t launch_lattice_step(const mhd_lattice* l, int from, cudaStream_t st, long long count = 0) {
    const mhd::StepLaunch s = step_launch(l, from);
    if (l->closure_buf) {
        if (l->closure_interval > 1 && count % l->closure_interval != 0) return mhd::launch_step_da_cached(s, l->da, st);
        mhd::ClosureParamsDev cp = l->closure;
        cp.da_out = l->closure_interval > 1 ? l->da : nullptr;
        return l->closure_kind == MHD_CLOSURE_TCGEN05 ? mhd::launch_step_closure_tc(s, cp, st)
                                                      : mhd::launch_step_closure(s, cp, st);
    }
    return mhd::launch_step(s, st);
}

// In place: one step on `buf` (phase 0 from the canonical layout, 1 from
// the streamed one).
cudaError_t launch_inplace_step(const mhd_lattice* l, void* buf, int phase, cudaStream_t st) {
    mhd::StepLaunch s = step_launch(l, 0);
    s.src = buf;
    s.dst = buf;
    return mhd::launch_aa_step(s, phase, st);
}

// A closure step whose tensor-core wait gave up leaves a flag behind.
mhd_status closure_status(mhd_lattice* l) {
    if (!l->closure_buf || !l->closure.err) return MHD_OK;
    int err = 0;
    CK(cudaMemcpyAsync(&err, l->closure.err, sizeof(int), cudaMemcpyDeviceToHost, l->stream), "closure status");
    CK(cudaStreamSynchronize(l->stream), "closure status");
    if (err) return fail(MHD_ECUDA, "closure step: a tensor-core MMA did not complete (wait limit reached)");
    return MHD_OK;
}

// Bring an in-place lattice to the canonical layout (same time step).
cudaError_t normalize(mhd_lattice* l) {
    if (!l->in_place || !l->aa_streamed) return cudaSuccess;
    cudaError_t e = mhd::launch_aa_unstream(l->L, l->p.precision, l->buf[0], l->p.bc_y == MHD_WALL, l->stream);
    if (e == cudaSuccess) l->aa_streamed = false;
    return e;
}

void drop_graphs(mhd_lattice* l) {
    for (auto& g : l->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

mhd_kernel_config default_config(const mhd::Layout& L, int prec, int wall_x) {
    mhd_kernel_config c;
    int V = prec == 0 ? 2 : 4;
    while (V > 1 && !mhd::step_shape_ok(L, prec, wall_x, V, 4)) V >>= 1;
    c.nodes_per_thread = V;
    c.rows_per_block = V == 1 ? 8 : 4;
    c.warps_per_sm = 0;
    return c;
}

bool config_ok(const mhd_lattice* l, const mhd_kernel_config& c) {
    if (c.warps_per_sm < 0 || c.warps_per_sm > 64) return false;
    if (l->p.precision == 0 && c.rows_per_block > 8) return false;
    // the FP16S in-place phase A kernel takes blocks of at most 256 threads
    if (l->in_place && l->p.precision == MHD_FP16S && c.rows_per_block > 8) return false;
    return mhd::step_shape_ok(l->L, l->p.precision, l->p.bc_x == MHD_WALL, c.nodes_per_thread,
                              c.rows_per_block);
}

mhd_status ensure_io(mhd_lattice* l) {
    if (l->io) return MHD_OK;
    CK(cudaMalloc(&l->io, sizeof(double) * 5 * (size_t)l->n()), "cudaMalloc(io)");
    return MHD_OK;
}

// ---- tune cache: one JSON object, one "key": [V, BY] entry per line ----
std::string cache_key(const mhd_lattice* l) {
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, l->dev) == cudaSuccess) name = prop.name;
    char buf[256];
    snprintf(buf, sizeof buf, "%s|p%d|%dx%d|bc%d%d%s", name.c_str(), l->p.precision, l->nx, l->ny,
             l->p.bc_x, l->p.bc_y, l->in_place ? "|inplace" : "");
    return buf;
}

// entries "key": [nodes_per_thread, rows_per_block, warps_per_sm] (a
// two-number entry has the built-in staging depth, warps_per_sm = 0)
using TuneCache = std::map<std::string, mhd_kernel_config>;

TuneCache read_cache(const char* path) {
    TuneCache m;
    FILE* fp = fopen(path, "r");
    if (!fp) return m;
    char line[512];
    while (fgets(line, sizeof line, fp)) {
        char* q1 = strchr(line, '"');
        if (!q1) continue;
        char* q2 = strchr(q1 + 1, '"');
        if (!q2) continue;
        int v = 0, by = 0, w = 0;
        const int got = sscanf(q2 + 1, " : [%d , %d , %d]", &v, &by, &w);
        if (got >= 2) m[std::string(q1 + 1, q2)] = mhd_kernel_config{v, by, got == 3 ? w : 0};
    }
    fclose(fp);
    return m;
}

void write_cache(const char* path, const TuneCache& m) {
    std::string tmp = std::string(path) + ".tmp";
    FILE* fp = fopen(tmp.c_str(), "w");
    if (!fp) return;
    fprintf(fp, "{\n");
    size_t i = 0;
    for (auto& kv : m)
        fprintf(fp, "  \"%s\": [%d, %d, %d]%s\n", kv.first.c_str(), kv.second.nodes_per_thread,
                kv.second.rows_per_block, kv.second.warps_per_sm, ++i < m.size() ? "," : "");
    fprintf(fp, "}\n");
    fclose(fp);
    rename(tmp.c_str(), path);
}

mhd_status check_params(const mhd_params* p) {
    if (!p) return fail(MHD_EINVAL, "params is NULL");
    if (!(std::isfinite(p->tau_f) && p->tau_f > 0.5)) return fail(MHD_EINVAL, "tau_f must be > 1/2");
    if (!(std::isfinite(p->tau_m) && p->tau_m > 0.5)) return fail(MHD_EINVAL, "tau_m must be > 1/2");
    if (!(std::isfinite(p->rho0) && p->rho0 > 0)) return fail(MHD_EINVAL, "rho0 must be > 0");
    if ((p->bc_x != MHD_PERIODIC && p->bc_x != MHD_WALL) ||
        (p->bc_y != MHD_PERIODIC && p->bc_y != MHD_WALL && p->bc_y != MHD_HALO))
        return fail(MHD_EINVAL, "bc_x must be MHD_PERIODIC or MHD_WALL, bc_y one of those or MHD_HALO");
    if (p->bc_y == MHD_HALO && p->streaming != MHD_TWO_BUFFERS)
        return fail(MHD_EINVAL, "slabs (bc_y = MHD_HALO) use two-buffer streaming");
    if (p->precision < MHD_FP64 || p->precision > MHD_FP16S)
        return fail(MHD_EINVAL, "unknown precision");
    if (p->eq_variant != 0 && p->eq_variant != 1) return fail(MHD_EINVAL, "eq_variant must be 0 or 1");
    if (p->collision != MHD_RR && p->collision != MHD_BGK) return fail(MHD_EINVAL, "unknown collision");
    if (p->mag_collision != MHD_MAG_BGK && p->mag_collision != MHD_MAG_REGULARISED)
        return fail(MHD_EINVAL, "unknown mag_collision");
    if (p->streaming != MHD_TWO_BUFFERS && p->streaming != MHD_IN_PLACE)
        return fail(MHD_EINVAL, "unknown streaming");
    if (p->streaming == MHD_IN_PLACE && p->bc_x != MHD_PERIODIC)
        return fail(MHD_EINVAL, "in-place streaming needs a periodic x axis");
    return MHD_OK;
}

}  // namespace

extern "C" {

const char* mhd_last_error(void) { return g_err.c_str(); }

mhd_status mhd_create(int nx, int ny, const mhd_params* p, void* stream, mhd_lattice** out) {
    if (!out) return fail(MHD_EINVAL, "out is NULL");
    *out = nullptr;
    mhd_status s = check_params(p);
    if (s != MHD_OK) return s;
    if (nx < 2 || ny < 2) return fail(MHD_EINVAL, "nx and ny must be >= 2");
    if ((long long)nx * ny > (1LL << 31)) return fail(MHD_EINVAL, "nx*ny must be <= 2^31");
    auto* l = new (std::nothrow) mhd_lattice();
    if (!l) return fail(MHD_ENOMEM, "host allocation failed");
    l->nx = nx;
    l->ny = ny;
    l->p = *p;
    l->stream = static_cast<cudaStream_t>(stream);
    l->in_place = p->streaming == MHD_IN_PLACE;
    l->halo = p->bc_y == MHD_HALO;
    if (l->halo) {
        l->Lx = mhd::make_layout(nx, ny + 2, p->precision);
        l->L = l->Lx;  // the interior: rows 1..ny of each plane
        l->L.ny = ny;
    } else {
        l->L = mhd::make_layout(nx, ny, p->precision);
    }
    cudaError_t e = cudaGetDevice(&l->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&l->cap, cudaStreamNonBlocking);
    for (int b = 0; b < (l->in_place ? 1 : 2) && e == cudaSuccess; ++b) {
        e = cudaMalloc(&l->alloc[b], l->buf_bytes());
        if (e == cudaSuccess && l->halo) e = cudaMemset(l->alloc[b], 0, l->buf_bytes());
        l->buf[b] = l->halo ? static_cast<char*>(l->alloc[b]) + l->L.pitch * l->L.esize : l->alloc[b];
    }
    if (e == cudaSuccess)
        e = cudaMalloc(&l->partials, sizeof(double) * mhd::kDiagSlots * mhd::diag_blocks(l->L));
    if (e == cudaSuccess) e = cudaMalloc(&l->totals_d, sizeof(double) * mhd::kDiagSlots);
    if (e == cudaSuccess) e = cudaMallocHost(&l->totals_h, sizeof(double) * mhd::kDiagSlots);
    if (e == cudaSuccess) e = cudaMalloc(&l->flags_d, 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mhd_destroy(l);
        return cuda_fail(e, "mhd_create");
    }
    l->cfg = default_config(l->L, p->precision, p->bc_x == MHD_WALL);
    if (const char* path = getenv("MHD_TUNE_CACHE")) {
        auto m = read_cache(path);
        auto it = m.find(cache_key(l));
        if (it != m.end() && config_ok(l, it->second)) l->cfg = it->second;
    }
    *out = l;
    return MHD_OK;
}

mhd_status mhd_destroy(mhd_lattice* l) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    cudaSetDevice(l->dev);
    if (l->stream || l->buf[0]) cudaStreamSynchronize(l->stream);
    drop_graphs(l);
    for (auto& b : l->alloc)
        if (b) cudaFree(b);
    if (l->io) cudaFree(l->io);
    if (l->closure_buf) cudaFree(l->closure_buf);
    if (l->da) cudaFree(l->da);
    if (l->partials) cudaFree(l->partials);
    if (l->totals_d) cudaFree(l->totals_d);
    if (l->totals_h) cudaFreeHost(l->totals_h);
    if (l->flags_d) cudaFree(l->flags_d);
    if (l->cap) cudaStreamDestroy(l->cap);
    if (l->xev) cudaEventDestroy(l->xev);
    delete l;
    return MHD_OK;
}

// Whether the device reads and writes host array p in place: pinned memory
// mapped at the same address (a NULL optional array counts as mapped).
static bool host_mapped(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer == p;
}

// mhd_set_fields / mhd_set_fields_f32: T is the host (and device copy) type
// of the fields.  Pinned host arrays on a two-buffer lattice are read in
// place by the initial-equilibrium kernel, which checks them on the way and
// writes the other buffer (kept only if every value passed: one pass over
// the host link); otherwise they are staged in the lattice's io buffer
// (5 x nx*ny doubles), checked there, and then converted.
extern "C++" {
template <typename T>
static mhd_status set_fields_t(mhd_lattice* l, const T* ux, const T* uy, const T* bx, const T* by, const T* rho) {
    if (!l || !ux || !uy || !bx || !by) return fail(MHD_EINVAL, "NULL argument");
    const long long n = l->n();
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    if (!l->in_place && host_mapped(ux) && host_mapped(uy) && host_mapped(bx) && host_mapped(by) &&
        host_mapped(rho)) {
        int flags = 0;
        CK(cudaMemsetAsync(l->flags_d, 0, sizeof(int), l->stream), "clear input flags");
        CK(mhd::launch_init(l->L, l->p.precision, l->buf[l->cur ^ 1], rho, ux, uy, bx, by, l->p.rho0,
                            l->p.eq_variant, l->stream, l->flags_d),
           "init kernel");
        CK(cudaMemcpyAsync(&flags, l->flags_d, sizeof(int), cudaMemcpyDeviceToHost, l->stream), "input flags");
        CK(cudaStreamSynchronize(l->stream), "mhd_set_fields");
        if (flags) {
            // the state is unchanged, but the other buffer no longer holds
            // the state the last step read
            l->prev_valid = false;
            return fail(MHD_EINVAL, (flags & 1) ? "non-finite input field" : "rho must be > 0");
        }
        l->cur ^= 1;
        l->step = 0;
        l->fields_set = true;
        l->prev_valid = false;
        l->closure_count = 0;  // the next closure step evaluates the MLP
        l->state_is_eq = true;
        l->aa_streamed = false;
        return MHD_OK;
    }
    mhd_status s = ensure_io(l);
    if (s != MHD_OK) return s;
    const size_t bytes = sizeof(T) * n;
    T* io = reinterpret_cast<T*>(l->io);
    T* d[5] = {io, io + n, io + 2 * n, io + 3 * n, io + 4 * n};
    const T* h[5] = {ux, uy, bx, by, rho};
    for (int q = 0; q < 5; ++q)
        if (h[q]) CK(cudaMemcpyAsync(d[q], h[q], bytes, cudaMemcpyHostToDevice, l->stream), "H2D fields");
    // the inputs are checked on the device copies, before the state is touched
    {
        int flags = 0;
        CK(cudaMemsetAsync(l->flags_d, 0, sizeof(int), l->stream), "clear input flags");
        const long long blocks = std::max(1LL, std::min((n + 255) / 256, 8LL * mhd::device_sms()));
        check_fields_kernel<T><<<(unsigned)blocks, 256, 0, l->stream>>>(d[0], d[1], d[2], d[3],
                                                                         rho ? d[4] : nullptr, n, l->flags_d);
        CK(cudaGetLastError(), "input check kernel");
        CK(cudaMemcpyAsync(&flags, l->flags_d, sizeof(int), cudaMemcpyDeviceToHost, l->stream), "input flags");
        CK(cudaStreamSynchronize(l->stream), "mhd_set_fields");
        if (flags & 1) return fail(MHD_EINVAL, "non-finite input field");
        if (flags & 2) return fail(MHD_EINVAL, "rho must be > 0");
    }
    CK(mhd::launch_init(l->L, l->p.precision, l->buf[l->cur], rho ? d[4] : nullptr, d[0], d[1], d[2],
                        d[3], l->p.rho0, l->p.eq_variant, l->stream),
       "init kernel");
    CK(cudaStreamSynchronize(l->stream), "mhd_set_fields");
    l->step = 0;
    l->fields_set = true;
    l->prev_valid = false;
    l->closure_count = 0;  // the next closure step evaluates the MLP
    l->state_is_eq = true;
    l->aa_streamed = false;
    return MHD_OK;
}
}  // extern "C++"

mhd_status mhd_set_fields(mhd_lattice* l, const double* ux, const double* uy, const double* bx,
                          const double* by, const double* rho) {
    return set_fields_t(l, ux, uy, bx, by, rho);
}

mhd_status mhd_set_fields_f32(mhd_lattice* l, const float* ux, const float* uy, const float* bx, const float* by,
                              const float* rho) {
    return set_fields_t(l, ux, uy, bx, by, rho);
}

// Graph of kGraphSteps steps starting from buffer `from` (two buffers) or
// from phase `from` (in place); kGraphSteps is even, so it ends where it began.
static mhd_status capture_graph(mhd_lattice* l, int from) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(l->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int c = from;
    cudaError_t le = cudaSuccess;
    // (a closure lattice with an interval > 1 captures only from a step
    // count that is a multiple of the interval, which divides kGraphSteps)
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) {
        le = l->in_place ? launch_inplace_step(l, l->buf[0], c, l->cap) : launch_lattice_step(l, c, l->cap, k);
        c ^= 1;
    }
    cudaError_t ee = cudaStreamEndCapture(l->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(le, "step launch during capture");
    }
    if (ee != cudaSuccess) return cuda_fail(ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&l->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(ie, "graph instantiate");
    return MHD_OK;
}

mhd_status mhd_advance(mhd_lattice* l, long long nsteps) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    if (nsteps < 0) return fail(MHD_EINVAL, "nsteps must be >= 0");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    if (nsteps == 0) return MHD_OK;
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    if (l->in_place) {
        while (nsteps >= kGraphSteps) {
            const int ph = l->aa_streamed ? 1 : 0;
            if (!l->graph[ph]) {
                mhd_status s = capture_graph(l, ph);
                if (s != MHD_OK) return s;
            }
            CK(cudaGraphLaunch(l->graph[ph], l->stream), "graph launch");
            nsteps -= kGraphSteps;
            l->step += kGraphSteps;
        }
        while (nsteps > 0) {
            CK(launch_inplace_step(l, l->buf[0], l->aa_streamed ? 1 : 0, l->stream), "step launch");
            l->aa_streamed = !l->aa_streamed;
            --nsteps;
            ++l->step;
        }
        l->state_is_eq = false;
        return MHD_OK;
    }
    auto single = [&]() -> mhd_status {
        CK(launch_lattice_step(l, l->cur, l->stream, l->closure_count), "step launch");
        l->cur ^= 1;
        --nsteps;
        ++l->step;
        ++l->closure_count;
        return MHD_OK;
    };
    while (nsteps >= kGraphSteps) {
        if (l->closure_buf && l->closure_count % l->closure_interval != 0) {
            mhd_status s = single();  // step up to the next evaluation of the MLP first
            if (s != MHD_OK) return s;
            continue;
        }
        if (!l->graph[l->cur]) {
            mhd_status s = capture_graph(l, l->cur);
            if (s != MHD_OK) return s;
        }
        CK(cudaGraphLaunch(l->graph[l->cur], l->stream), "graph launch");
        nsteps -= kGraphSteps;
        l->step += kGraphSteps;
        l->closure_count += kGraphSteps;
    }
    while (nsteps > 0) {
        mhd_status s = single();
        if (s != MHD_OK) return s;
    }
    l->prev_valid = true;
    l->state_is_eq = false;
    return MHD_OK;
}

extern "C++" {
// mhd_get_fields / mhd_get_fields_f32: pinned host arrays are written in
// place by the fields kernel (one pass over the host link); others through
// the io buffer and a copy.
template <typename T>
static mhd_status get_fields_t(mhd_lattice* l, T* rho, T* ux, T* uy, T* bx, T* by) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(normalize(l), "unstream kernel");
    {
        const mhd_status cs = closure_status(l);
        if (cs != MHD_OK) return cs;
    }
    if (host_mapped(rho) && host_mapped(ux) && host_mapped(uy) && host_mapped(bx) && host_mapped(by)) {
        CK(mhd::launch_fields(l->L, l->p.precision, l->buf[l->cur], l->p.rho0, rho, ux, uy, bx, by, l->stream),
           "fields kernel");
        CK(cudaStreamSynchronize(l->stream), "mhd_get_fields");
        return MHD_OK;
    }
    mhd_status s = ensure_io(l);
    if (s != MHD_OK) return s;
    const long long n = l->n();
    T* io = reinterpret_cast<T*>(l->io);
    T* d[5] = {io, io + n, io + 2 * n, io + 3 * n, io + 4 * n};
    T* h[5] = {rho, ux, uy, bx, by};
    CK(mhd::launch_fields(l->L, l->p.precision, l->buf[l->cur], l->p.rho0, h[0] ? d[0] : nullptr,
                          h[1] ? d[1] : nullptr, h[2] ? d[2] : nullptr, h[3] ? d[3] : nullptr,
                          h[4] ? d[4] : nullptr, l->stream),
       "fields kernel");
    for (int q = 0; q < 5; ++q)
        if (h[q]) CK(cudaMemcpyAsync(h[q], d[q], sizeof(T) * n, cudaMemcpyDeviceToHost, l->stream), "D2H fields");
    CK(cudaStreamSynchronize(l->stream), "mhd_get_fields");
    return MHD_OK;
}
}  // extern "C++"

mhd_status mhd_get_fields(mhd_lattice* l, double* rho, double* ux, double* uy, double* bx, double* by) {
    return get_fields_t(l, rho, ux, uy, bx, by);
}

mhd_status mhd_get_fields_f32(mhd_lattice* l, float* rho, float* ux, float* uy, float* bx, float* by) {
    return get_fields_t(l, rho, ux, uy, bx, by);
}

mhd_status mhd_get_totals(mhd_lattice* l, mhd_totals* out) {
    if (!l || !out) return fail(MHD_EINVAL, "NULL argument");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(normalize(l), "unstream kernel");
    {
        const mhd_status cs = closure_status(l);
        if (cs != MHD_OK) return cs;
    }
    mhd::DiagLaunch d;
    d.L = l->L;
    d.prec = l->p.precision;
    d.prev = l->buf[l->cur ^ 1];
    d.cur = l->buf[l->cur];
    // (a slab reads the moments of its ghost rows for the stencil at its
    // edge rows, so it reduces the stored state)
    d.mode = (l->prev_valid && !l->halo) ? 0 : 1;
    d.omega_m = 1.0 / l->p.tau_m;
    d.rho0 = l->p.rho0;
    const double om1 = 1.0 - d.omega_m;
    // gather mode reads the pre-collision g itself; the stored-state mode
    // recovers g - g_eq = (g* - g_eq) / (1 - omega_m)
    d.neq_scale = d.mode == 0 ? 1.0 : ((l->state_is_eq || std::fabs(om1) < 1e-12) ? 0.0 : 1.0 / om1);
    d.wall_x = l->p.bc_x == MHD_WALL;
    d.wall_y = l->p.bc_y == MHD_WALL;
    d.halo_y = l->halo;
    CK(mhd::launch_diag(d, l->partials, mhd::diag_blocks(l->L), l->totals_d, l->stream), "diagnostics kernel");
    CK(cudaMemcpyAsync(l->totals_h, l->totals_d, sizeof(double) * mhd::kDiagSlots,
                       cudaMemcpyDeviceToHost, l->stream),
       "D2H totals");
    CK(cudaStreamSynchronize(l->stream), "mhd_get_totals");
    const double* t = l->totals_h;
    const double n = (double)l->n();
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
    out->step = l->step;
    for (int s = 0; s < mhd::kDiagSlots; ++s)
        if (!std::isfinite(t[s])) return fail(MHD_EUNSTABLE, "non-finite diagnostics: the run blew up");
    return MHD_OK;
}

mhd_status mhd_advance_totals(mhd_lattice* l, long long nsteps, mhd_totals* out) {
    if (!l || !out) return fail(MHD_EINVAL, "NULL argument");
    if (nsteps < 1) return fail(MHD_EINVAL, "nsteps must be >= 1");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    // the fused step is the periodic-x two-buffer step of a whole lattice
    const bool fused = !l->in_place && !l->closure_buf && !l->halo && l->p.bc_x != MHD_WALL;
    mhd_status s = mhd_advance(l, fused ? nsteps - 1 : nsteps);
    if (s != MHD_OK) return s;
    if (!fused) return mhd_get_totals(l, out);
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(mhd::launch_step_totals(step_launch(l, l->cur), l->partials, mhd::diag_blocks(l->L), l->totals_d,
                               l->stream),
       "step with totals");
    l->cur ^= 1;
    ++l->step;
    l->prev_valid = true;
    l->state_is_eq = false;
    CK(cudaMemcpyAsync(l->totals_h, l->totals_d, sizeof(double) * mhd::kDiagSlots, cudaMemcpyDeviceToHost,
                       l->stream),
       "D2H totals");
    CK(cudaStreamSynchronize(l->stream), "mhd_advance_totals");
    const double* t = l->totals_h;
    const double n = (double)l->n();
    out->mass = t[0];
    out->mom_x = t[1];
    out->mom_y = t[2];
    out->e_kin = t[3] / n;
    out->e_mag = t[4] / n;
    out->cross_hel = t[5] / n;
    out->bsum_x = t[6];
    out->bsum_y = t[7];
    out->divb_rms = out->divb_max = out->omega_max = std::nan("");
    out->jz_max = t[11];
    out->step = l->step;
    for (int q : {0, 1, 2, 3, 4, 5, 6, 7, 11})
        if (!std::isfinite(t[q])) return fail(MHD_EUNSTABLE, "non-finite point totals: the run blew up");
    return MHD_OK;
}

mhd_status mhd_get_populations(mhd_lattice* l, double* f, double* g) {
    if (!l || !f || !g) return fail(MHD_EINVAL, "NULL argument");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(normalize(l), "unstream kernel");
    {
        const mhd_status cs = closure_status(l);
        if (cs != MHD_OK) return cs;
    }
    mhd_status s = ensure_io(l);
    if (s != MHD_OK) return s;
    const long long n = l->n();
    for (int p = 0; p < mhd::kStatePlanes; ++p) {
        double* host = p < 9 ? f + (long long)p * n : g + (long long)(p - 9) * n;
        CK(mhd::launch_plane_out(l->L, l->p.precision, l->buf[l->cur], p, l->p.rho0, l->io, l->stream),
           "plane out kernel");
        CK(cudaMemcpyAsync(host, l->io, sizeof(double) * n, cudaMemcpyDeviceToHost, l->stream),
           "D2H populations");
        CK(cudaStreamSynchronize(l->stream), "mhd_get_populations");
    }
    return MHD_OK;
}

mhd_status mhd_set_populations(mhd_lattice* l, const double* f, const double* g) {
    if (!l || !f || !g) return fail(MHD_EINVAL, "NULL argument");
    const long long n = l->n();
    if (!finite_array(f, 9 * n) || !finite_array(g, 10 * n))
        return fail(MHD_EINVAL, "non-finite populations");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    mhd_status s = ensure_io(l);
    if (s != MHD_OK) return s;
    for (int p = 0; p < mhd::kStatePlanes; ++p) {
        const double* host = p < 9 ? f + (long long)p * n : g + (long long)(p - 9) * n;
        CK(cudaMemcpyAsync(l->io, host, sizeof(double) * n, cudaMemcpyHostToDevice, l->stream),
           "H2D populations");
        CK(mhd::launch_plane_in(l->L, l->p.precision, l->buf[l->cur], p, l->p.rho0, l->io, l->stream),
           "plane in kernel");
        CK(cudaStreamSynchronize(l->stream), "mhd_set_populations");
    }
    l->fields_set = true;
    l->prev_valid = false;
    l->closure_count = 0;  // the next closure step evaluates the MLP
    l->state_is_eq = false;
    l->aa_streamed = false;
    return MHD_OK;
}

mhd_status mhd_set_closure(mhd_lattice* l, const mhd_mlp* mlp) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(cudaStreamSynchronize(l->stream), "mhd_set_closure");
    if (!mlp) {
        if (l->closure_buf) cudaFree(l->closure_buf);
        l->closure_buf = nullptr;
        drop_graphs(l);
        return MHD_OK;
    }
    if (l->p.precision != MHD_FP32 || l->p.bc_x != MHD_PERIODIC || l->p.bc_y != MHD_PERIODIC || l->in_place)
        return fail(MHD_EINVAL, "the closure runs on FP32 periodic two-buffer lattices");
    using namespace mhd;
    const size_t nbf = (size_t)kHid * kInPad + (size_t)kHid * kHid + (size_t)kOutPad * kHid;
    const size_t nfl = 2 * kHid + kOutPad + 2 * kIn + kOut;
    const size_t err_off = (nbf * sizeof(__nv_bfloat16) + nfl * sizeof(float) + 15) / 16 * 16;
    const size_t bytes = err_off + 16;
    if (!l->closure_buf) CK(cudaMalloc(&l->closure_buf, bytes), "cudaMalloc(closure)");
    ClosureParamsDev src;
    mhd_internal_closure_params(mlp, &src);
    auto* bf = static_cast<__nv_bfloat16*>(l->closure_buf);
    auto* fl = reinterpret_cast<float*>(bf + nbf);
    ClosureParamsDev& cp = l->closure;
    cp.Wt1 = bf;
    cp.Wt2 = bf + kHid * kInPad;
    cp.Wt3 = bf + kHid * kInPad + kHid * kHid;
    cp.b1 = fl;
    cp.b2 = fl + kHid;
    cp.b3 = fl + 2 * kHid;
    cp.mean = fl + 2 * kHid + kOutPad;
    cp.scale = fl + 2 * kHid + kOutPad + kIn;
    cp.out_scale = fl + 2 * kHid + kOutPad + 2 * kIn;
    cp.err = reinterpret_cast<int*>(static_cast<char*>(l->closure_buf) + err_off);
    CK(cudaMemsetAsync(cp.err, 0, sizeof(int), l->stream), "clear closure status");
    struct { const void* s; const void* d; size_t b; } parts[] = {
        {src.Wt1, cp.Wt1, sizeof(__nv_bfloat16) * kHid * kInPad},
        {src.Wt2, cp.Wt2, sizeof(__nv_bfloat16) * kHid * kHid},
        {src.Wt3, cp.Wt3, sizeof(__nv_bfloat16) * kOutPad * kHid},
        {src.b1, cp.b1, sizeof(float) * kHid},
        {src.b2, cp.b2, sizeof(float) * kHid},
        {src.b3, cp.b3, sizeof(float) * kOutPad},
        {src.mean, cp.mean, sizeof(float) * kIn},
        {src.scale, cp.scale, sizeof(float) * kIn},
        {src.out_scale, cp.out_scale, sizeof(float) * kOut}};
    for (auto& q : parts)
        CK(cudaMemcpyAsync(const_cast<void*>(q.d), q.s, q.b, cudaMemcpyDeviceToDevice, l->stream), "copy closure");
    CK(cudaStreamSynchronize(l->stream), "mhd_set_closure");
    drop_graphs(l);
    l->closure_count = 0;
    return MHD_OK;
}

mhd_status mhd_set_closure_interval(mhd_lattice* l, int k) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    if (k < 1 || k > kGraphSteps || kGraphSteps % k != 0)
        return fail(MHD_EINVAL, "the closure interval must divide 64");
    if (k > 1 && (l->nx % 4 || l->p.precision != MHD_FP32 || l->p.bc_x != MHD_PERIODIC ||
                  l->p.bc_y != MHD_PERIODIC || l->in_place))
        return fail(MHD_EINVAL, "a closure interval > 1 needs an FP32 periodic two-buffer lattice with nx % 4 == 0");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(cudaStreamSynchronize(l->stream), "mhd_set_closure_interval");
    if (k > 1 && !l->da) CK(cudaMalloc(&l->da, sizeof(float) * 3 * (size_t)l->n()), "cudaMalloc(closure correction)");
    if (k != l->closure_interval) drop_graphs(l);
    l->closure_interval = k;
    l->closure_count = 0;
    return MHD_OK;
}

mhd_status mhd_get_closure_interval(const mhd_lattice* l, int* k) {
    if (!l || !k) return fail(MHD_EINVAL, "NULL argument");
    *k = l->closure_interval;
    return MHD_OK;
}

mhd_status mhd_set_closure_kernel(mhd_lattice* l, int kind) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    if (kind != MHD_CLOSURE_WARP_MMA && kind != MHD_CLOSURE_TCGEN05) return fail(MHD_EINVAL, "unknown closure kernel");
    if (kind != l->closure_kind) {
        CK(cudaSetDevice(l->dev), "cudaSetDevice");
        CK(cudaStreamSynchronize(l->stream), "mhd_set_closure_kernel");
        drop_graphs(l);
        l->closure_kind = kind;
        l->closure_count = 0;
    }
    return MHD_OK;
}

mhd_status mhd_get_closure_kernel(const mhd_lattice* l, int* kind) {
    if (!l || !kind) return fail(MHD_EINVAL, "NULL argument");
    *kind = l->closure_kind;
    return MHD_OK;
}

mhd_status mhd_closure_filter(mhd_lattice* l, int factor, float* coarse_state) {
    if (!l || !coarse_state) return fail(MHD_EINVAL, "NULL argument");
    if (factor < 1 || l->nx % factor || l->ny % factor) return fail(MHD_EINVAL, "factor must divide nx and ny");
    if (l->p.bc_x != MHD_PERIODIC || l->p.bc_y != MHD_PERIODIC) return fail(MHD_EINVAL, "periodic lattices only");
    if (l->in_place) return fail(MHD_EINVAL, "in-place lattices keep no previous state");
    if (!l->prev_valid) return fail(MHD_ESTATE, "needs the state after a step (advance first)");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(mhd::launch_filter(l->L, l->p.precision, l->buf[l->cur ^ 1], factor, coarse_state, l->stream), "filter kernel");
    CK(cudaStreamSynchronize(l->stream), "mhd_closure_filter");
    return MHD_OK;
}

mhd_status mhd_closure_sgs_targets(mhd_lattice* l, int factor, double tau_coarse, float* targets) {
    if (!l || !targets) return fail(MHD_EINVAL, "NULL argument");
    if (factor < 1 || l->nx % factor || l->ny % factor) return fail(MHD_EINVAL, "factor must divide nx and ny");
    if (l->p.bc_x != MHD_PERIODIC || l->p.bc_y != MHD_PERIODIC) return fail(MHD_EINVAL, "periodic lattices only");
    if (!(tau_coarse > 0.5) || std::fabs(1.0 - 1.0 / tau_coarse) < 1e-12)
        return fail(MHD_EINVAL, "tau_coarse must be > 1/2 and != 1");
    if (l->in_place) return fail(MHD_EINVAL, "in-place lattices keep no previous state");
    if (!l->prev_valid) return fail(MHD_ESTATE, "needs the state after a step (advance first)");
    if (l->p.rho0 != 1.0) return fail(MHD_EINVAL, "rho0 = 1 only");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(mhd::launch_sgs(l->L, l->p.precision, l->buf[l->cur ^ 1], factor, tau_coarse, targets, l->stream),
       "sgs kernel");
    CK(cudaStreamSynchronize(l->stream), "mhd_closure_sgs_targets");
    return MHD_OK;
}

mhd_status mhd_set_precollision_state(mhd_lattice* l, const float* state) {
    if (!l || !state) return fail(MHD_EINVAL, "NULL argument");
    if (l->p.bc_x != MHD_PERIODIC || l->p.bc_y != MHD_PERIODIC) return fail(MHD_EINVAL, "periodic lattices only");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(mhd::launch_unstream(l->L, l->p.precision, l->buf[l->cur], state, l->stream), "unstream kernel");
    CK(cudaStreamSynchronize(l->stream), "mhd_set_precollision_state");
    l->fields_set = true;
    l->prev_valid = false;
    l->closure_count = 0;  // the next closure step evaluates the MLP
    l->state_is_eq = false;
    l->aa_streamed = false;
    return MHD_OK;
}

mhd_status mhd_state_bytes(const mhd_lattice* l, size_t* bytes) {
    if (!l || !bytes) return fail(MHD_EINVAL, "NULL argument");
    *bytes = (size_t)mhd::kStatePlanes * (size_t)l->n() * (size_t)l->L.esize;
    return MHD_OK;
}

mhd_status mhd_slab_exchange(mhd_lattice* lower, mhd_lattice* upper, int all_planes) {
    if (!lower || !upper) return fail(MHD_EINVAL, "lattice is NULL");
    if (!lower->halo || !upper->halo) return fail(MHD_EINVAL, "slab exchange needs bc_y = MHD_HALO lattices");
    if (lower->nx != upper->nx || lower->p.precision != upper->p.precision || lower->p.bc_x != upper->p.bc_x)
        return fail(MHD_EINVAL, "the slabs of one lattice share nx, precision and bc_x");
    for (mhd_lattice* l : {lower, upper})
        if (!l->xev) {
            CK(cudaSetDevice(l->dev), "cudaSetDevice");
            CK(cudaEventCreateWithFlags(&l->xev, cudaEventDisableTiming), "exchange event");
        }
    // the edge rows are final once each lattice's queued steps are done
    CK(cudaSetDevice(lower->dev), "cudaSetDevice");
    CK(cudaEventRecord(lower->xev, lower->stream), "exchange event");
    CK(cudaSetDevice(upper->dev), "cudaSetDevice");
    CK(cudaEventRecord(upper->xev, upper->stream), "exchange event");
    const size_t es = lower->L.esize, row = (size_t)lower->nx * es;
    // from `from`'s interior row `src_row` into `to`'s row `dst_row` (-1 or
    // ny: a ghost row), the planes whose c_y equals `cy` (all with all_planes):
    // on one device one copy kernel for all of them (whole padded rows: the
    // row pitch is a multiple of 128 bytes), across devices one copy each
    auto copy = [&](mhd_lattice* from, int src_row, mhd_lattice* to, int dst_row, int cy) -> mhd_status {
        CK(cudaSetDevice(to->dev), "cudaSetDevice");
        CK(cudaStreamWaitEvent(to->stream, from->xev, 0), "exchange wait");
        const char* sb = static_cast<const char*>(from->buf[from->cur]);
        char* db = static_cast<char*>(to->buf[to->cur]);
        if (from->dev == to->dev) {
            mhd::HaloPlanes hp{};
            for (int p = 0; p < mhd::kStatePlanes; ++p)
                if (all_planes || mhd::pcy(p) == cy) hp.p[hp.n++] = p;
            const long long pb = (long long)from->L.pitch * (long long)es;
            CK(mhd::launch_halo_rows(sb, db, from->L.plane * (long long)es, to->L.plane * (long long)es,
                                     (long long)src_row * pb, (long long)dst_row * pb, pb, hp, to->stream),
               "halo copy kernel");
            return MHD_OK;
        }
        for (int p = 0; p < mhd::kStatePlanes; ++p) {
            if (!all_planes && mhd::pcy(p) != cy) continue;
            const char* src = sb + ((long long)p * from->L.plane + (long long)src_row * from->L.pitch) * (long long)es;
            char* dst = db + ((long long)p * to->L.plane + (long long)dst_row * to->L.pitch) * (long long)es;
            CK(cudaMemcpyAsync(dst, src, row, cudaMemcpyDefault, to->stream), "halo copy");
        }
        return MHD_OK;
    };
    mhd_status s = copy(lower, lower->ny - 1, upper, -1, +1);
    if (s == MHD_OK) s = copy(upper, 0, lower, lower->ny, -1);
    return s;
}

// ---- slab groups ------------------------------------------------------------
struct mhd_slab_group {
    std::vector<mhd_lattice*> slabs;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;              // capture stream of the group's graphs
    mhd::HaloJob* jobs[2] = {nullptr, nullptr};  // per buffer parity: 2 copies per boundary
    int njobs = 0;
    long long row_bytes = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};  // kGraphSteps rounds from parity 0 / 1
    std::vector<mhd_kernel_config> graph_cfg;       // the slabs' launch shapes at capture
};

static void group_drop_graphs(mhd_slab_group* g) {
    for (auto& x : g->graph)
        if (x) {
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
}

mhd_status mhd_slab_group_create(mhd_lattice* const* slabs, int n, mhd_slab_group** out) {
    if (!out) return fail(MHD_EINVAL, "out is NULL");
    *out = nullptr;
    if (!slabs || n < 1) return fail(MHD_EINVAL, "need at least one slab");
    const mhd_lattice* a = slabs[0];
    for (int i = 0; i < n; ++i) {
        const mhd_lattice* l = slabs[i];
        if (!l) return fail(MHD_EINVAL, "slab is NULL");
        if (!l->halo) return fail(MHD_EINVAL, "a slab group needs bc_y = MHD_HALO lattices");
        if (l->nx != a->nx || l->p.precision != a->p.precision || l->p.bc_x != a->p.bc_x)
            return fail(MHD_EINVAL, "the slabs of one lattice share nx, precision and bc_x");
        if (l->dev != a->dev || l->stream != a->stream)
            return fail(MHD_EINVAL, "the slabs of a group share one device and one stream");
        if (l->closure_buf) return fail(MHD_EINVAL, "a slab group steps slabs without a closure");
    }
    CK(cudaSetDevice(a->dev), "cudaSetDevice");
    auto* g = new mhd_slab_group;
    g->slabs.assign(slabs, slabs + n);
    g->stream = a->stream;
    g->row_bytes = (long long)a->L.pitch * a->L.esize;  // a multiple of 128 bytes
    g->njobs = 2 * n;
    std::vector<mhd::HaloJob> host(g->njobs);
    cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
        for (int i = 0; i < n; ++i) {
            mhd_lattice* lo = slabs[i];
            mhd_lattice* up = slabs[(i + 1) % n];
            const char* lb = static_cast<const char*>(lo->buf[par]);
            const char* ub = static_cast<const char*>(up->buf[par]);
            const long long lp = lo->L.plane * (long long)lo->L.esize, upl = up->L.plane * (long long)up->L.esize;
            // the top row of `lo` into the ghost row below `up` (c_y = +1) ...
            mhd::HaloJob& j0 = host[2 * i];
            j0.src = lb + (long long)(lo->ny - 1) * g->row_bytes;
            j0.dst = const_cast<char*>(ub) - g->row_bytes;
            j0.src_plane = lp;
            j0.dst_plane = upl;
            // ... and the bottom row of `up` into the ghost row above `lo` (c_y = -1)
            mhd::HaloJob& j1 = host[2 * i + 1];
            j1.src = ub;
            j1.dst = const_cast<char*>(lb) + (long long)lo->ny * g->row_bytes;
            j1.src_plane = upl;
            j1.dst_plane = lp;
            int k0 = 0, k1 = 0;
            for (int p = 0; p < mhd::kStatePlanes; ++p) {
                if (mhd::pcy(p) > 0) j0.planes[k0++] = p;
                if (mhd::pcy(p) < 0) j1.planes[k1++] = p;
            }
        }
        e = cudaMalloc(&g->jobs[par], sizeof(mhd::HaloJob) * g->njobs);
        if (e == cudaSuccess)
            e = cudaMemcpy(g->jobs[par], host.data(), sizeof(mhd::HaloJob) * g->njobs, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        mhd_slab_group_destroy(g);
        return cuda_fail(e, "mhd_slab_group_create");
    }
    *out = g;
    return MHD_OK;
}

// One round from buffer parity `par` on stream st: every slab's step, then
// the exchanges of every boundary into the buffers the steps wrote.
static cudaError_t group_round(const mhd_slab_group* g, int par, cudaStream_t st) {
    for (const mhd_lattice* l : g->slabs) {
        const cudaError_t e = launch_lattice_step(l, par, st);
        if (e != cudaSuccess) return e;
    }
    return mhd::launch_halo_jobs(g->jobs[par ^ 1], g->njobs, g->row_bytes, st);
}

mhd_status mhd_slab_group_advance(mhd_slab_group* g, long long nsteps) {
    if (!g) return fail(MHD_EINVAL, "group is NULL");
    if (nsteps < 0) return fail(MHD_EINVAL, "nsteps must be >= 0");
    const int par0 = g->slabs[0]->cur;
    for (const mhd_lattice* l : g->slabs) {
        if (!l->fields_set) return fail(MHD_ESTATE, "set the fields of every slab first");
        if (l->cur != par0) return fail(MHD_ESTATE, "the slabs have taken different numbers of steps");
        if (l->closure_buf) return fail(MHD_EINVAL, "a slab group steps slabs without a closure");
    }
    if (nsteps == 0) return MHD_OK;
    CK(cudaSetDevice(g->slabs[0]->dev), "cudaSetDevice");
    // graphs captured with other launch shapes are stale
    std::vector<mhd_kernel_config> cfg;
    for (const mhd_lattice* l : g->slabs) cfg.push_back(l->cfg);
    if (cfg.size() != g->graph_cfg.size() ||
        !std::equal(cfg.begin(), cfg.end(), g->graph_cfg.begin(), [](const mhd_kernel_config& x, const mhd_kernel_config& y) {
            return x.nodes_per_thread == y.nodes_per_thread && x.rows_per_block == y.rows_per_block &&
                   x.warps_per_sm == y.warps_per_sm;
        })) {
        CK(cudaStreamSynchronize(g->stream), "mhd_slab_group_advance");
        group_drop_graphs(g);
        g->graph_cfg = cfg;
    }
    int par = par0;
    long long done = 0;
    while (nsteps - done >= kGraphSteps) {
        if (!g->graph[par]) {
            cudaGraph_t gr = nullptr;
            CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
            cudaError_t le = cudaSuccess;
            for (int k = 0, c = par; k < kGraphSteps && le == cudaSuccess; ++k, c ^= 1) le = group_round(g, c, g->cap);
            const cudaError_t ee = cudaStreamEndCapture(g->cap, &gr);
            if (le != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return cuda_fail(le, "slab group capture");
            }
            if (ee != cudaSuccess) return cuda_fail(ee, "end capture");
            const cudaError_t ie = cudaGraphInstantiate(&g->graph[par], gr, 0);
            cudaGraphDestroy(gr);
            if (ie != cudaSuccess) return cuda_fail(ie, "graph instantiate");
        }
        CK(cudaGraphLaunch(g->graph[par], g->stream), "graph launch");
        done += kGraphSteps;  // kGraphSteps is even: the parity is unchanged
    }
    for (; done < nsteps; ++done, par ^= 1) CK(group_round(g, par, g->stream), "slab group round");
    for (mhd_lattice* l : g->slabs) {
        l->cur = par;
        l->step += nsteps;
        l->prev_valid = true;
        l->state_is_eq = false;
    }
    return MHD_OK;
}

mhd_status mhd_slab_group_destroy(mhd_slab_group* g) {
    if (!g) return MHD_OK;
    cudaSetDevice(g->slabs[0]->dev);
    if (g->stream) cudaStreamSynchronize(g->stream);
    group_drop_graphs(g);
    for (auto& j : g->jobs)
        if (j) cudaFree(j);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
    return MHD_OK;
}

mhd_status mhd_get_state(mhd_lattice* l, void* host, size_t bytes) {
    size_t need = 0;
    if (!host || mhd_state_bytes(l, &need) != MHD_OK) return fail(MHD_EINVAL, "NULL argument");
    if (bytes != need) return fail(MHD_EINVAL, "state buffer has the wrong size");
    if (!l->fields_set) return fail(MHD_ESTATE, "set fields or populations first");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    CK(normalize(l), "unstream kernel");
    {
        const mhd_status cs = closure_status(l);
        if (cs != MHD_OK) return cs;
    }
    const size_t es = l->L.esize, row = (size_t)l->nx * es;
    for (int p = 0; p < mhd::kStatePlanes; ++p) {
        char* dst = static_cast<char*>(host) + (size_t)p * l->n() * es;
        const char* src = static_cast<const char*>(l->buf[l->cur]) + (size_t)p * l->L.plane * es;
        CK(cudaMemcpy2DAsync(dst, row, src, (size_t)l->L.pitch * es, row, l->ny,
                             cudaMemcpyDeviceToHost, l->stream),
           "D2H state");
    }
    CK(cudaStreamSynchronize(l->stream), "mhd_get_state");
    return MHD_OK;
}

mhd_status mhd_set_state(mhd_lattice* l, const void* host, size_t bytes) {
    size_t need = 0;
    if (!host || mhd_state_bytes(l, &need) != MHD_OK) return fail(MHD_EINVAL, "NULL argument");
    if (bytes != need) return fail(MHD_EINVAL, "state buffer has the wrong size");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    const size_t es = l->L.esize, row = (size_t)l->nx * es;
    for (int p = 0; p < mhd::kStatePlanes; ++p) {
        const char* src = static_cast<const char*>(host) + (size_t)p * l->n() * es;
        char* dst = static_cast<char*>(l->buf[l->cur]) + (size_t)p * l->L.plane * es;
        CK(cudaMemcpy2DAsync(dst, (size_t)l->L.pitch * es, src, row, row, l->ny,
                             cudaMemcpyHostToDevice, l->stream),
           "H2D state");
    }
    CK(cudaStreamSynchronize(l->stream), "mhd_set_state");
    l->fields_set = true;
    l->prev_valid = false;
    l->closure_count = 0;  // the next closure step evaluates the MLP
    l->state_is_eq = false;
    l->aa_streamed = false;
    return MHD_OK;
}

mhd_status mhd_get_kernel_config(const mhd_lattice* l, mhd_kernel_config* out) {
    if (!l || !out) return fail(MHD_EINVAL, "NULL argument");
    *out = l->cfg;
    return MHD_OK;
}

mhd_status mhd_set_kernel_config(mhd_lattice* l, const mhd_kernel_config* cfg) {
    if (!l || !cfg) return fail(MHD_EINVAL, "NULL argument");
    if (!config_ok(l, *cfg)) return fail(MHD_EINVAL, "launch shape not valid for this lattice");
    if (cfg->nodes_per_thread != l->cfg.nodes_per_thread || cfg->rows_per_block != l->cfg.rows_per_block ||
        cfg->warps_per_sm != l->cfg.warps_per_sm) {
        CK(cudaStreamSynchronize(l->stream), "mhd_set_kernel_config");
        drop_graphs(l);
        l->cfg = *cfg;
    }
    return MHD_OK;
}

// With a closure the step is the closure kernel (fixed 32 x 8-node tiles):
// time its two MLP kernels (reading the current buffer, writing the spare
// one) and keep the faster.
static mhd_status autotune_closure(mhd_lattice* l, mhd_kernel_config* best) {
    CK(cudaStreamSynchronize(l->stream), "mhd_autotune");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    const mhd::StepLaunch s = step_launch(l, l->cur);
    float ms[2] = {0.f, 0.f};
    cudaError_t err = cudaSuccess;
    for (int kind = 0; kind < 2 && err == cudaSuccess; ++kind) {
        auto one = [&]() {
            return kind == MHD_CLOSURE_TCGEN05 ? mhd::launch_step_closure_tc(s, l->closure, l->stream)
                                               : mhd::launch_step_closure(s, l->closure, l->stream);
        };
        for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = one();
        if (err == cudaSuccess) err = cudaEventRecord(e0, l->stream);
        for (int k = 0; k < 20 && err == cudaSuccess; ++k) err = one();
        if (err == cudaSuccess) err = cudaEventRecord(e1, l->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[kind], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "closure autotune");
    l->prev_valid = false;  // the spare buffer was overwritten
    mhd_status st = closure_status(l);
    if (st != MHD_OK) return st;
    if (getenv("MHD_TUNE_VERBOSE"))
        fprintf(stderr, "mhd_autotune closure %dx%d: warp-MMA %.4f ms/step, tcgen05 %.4f ms/step\n", l->nx, l->ny,
                ms[0] / 20, ms[1] / 20);
    st = mhd_set_closure_kernel(l, ms[1] < ms[0] ? MHD_CLOSURE_TCGEN05 : MHD_CLOSURE_WARP_MMA);
    if (best) *best = l->cfg;
    return st;
}

mhd_status mhd_autotune(mhd_lattice* l, mhd_kernel_config* best) {
    if (!l) return fail(MHD_EINVAL, "lattice is NULL");
    CK(cudaSetDevice(l->dev), "cudaSetDevice");
    if (l->closure_buf) return autotune_closure(l, best);
    const char* path = getenv("MHD_TUNE_CACHE");
    const std::string key = cache_key(l);
    if (path) {
        auto m = read_cache(path);
        auto it = m.find(key);
        if (it != m.end() && config_ok(l, it->second)) {
            mhd_status s = mhd_set_kernel_config(l, &it->second);
            if (best) *best = l->cfg;
            return s;
        }
    }
    CK(cudaStreamSynchronize(l->stream), "mhd_autotune");
    // In place there is no spare buffer: candidates run on a scratch copy of
    // the state (held only while tuning), one phase-0 / phase-1 pair per step pair.
    void* scratch = nullptr;
    if (l->in_place) {
        CK(normalize(l), "unstream kernel");
        CK(cudaMalloc(&scratch, l->buf_bytes()), "cudaMalloc(autotune scratch)");
        cudaError_t ce = cudaMemcpyAsync(scratch, l->buf[0], l->buf_bytes(), cudaMemcpyDeviceToDevice, l->stream);
        if (ce != cudaSuccess) {
            cudaFree(scratch);
            return cuda_fail(ce, "autotune scratch copy");
        }
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    mhd_kernel_config chosen = l->cfg;
    float best_ms = 1e30f;
    const mhd_kernel_config saved = l->cfg;
    const int iters = 20;
    // time one candidate shape (ms for `iters` steps after 4 untimed ones)
    auto time_config = [&](const mhd_kernel_config& c, float* ms) -> cudaError_t {
        l->cfg = c;
        mhd::StepLaunch s = step_launch(l, l->cur);  // reads cur, writes the spare buffer
        auto one = [&](int k) {
            return l->in_place ? launch_inplace_step(l, scratch, k & 1, l->stream) : mhd::launch_step(s, l->stream);
        };
        cudaError_t err = cudaSuccess;
        for (int k = 0; k < 4 && err == cudaSuccess; ++k) err = one(k);
        if (err == cudaSuccess) err = cudaEventRecord(e0, l->stream);
        for (int k = 0; k < iters && err == cudaSuccess; ++k) err = one(k);
        if (err == cudaSuccess) err = cudaEventRecord(e1, l->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
        if (err == cudaSuccess && getenv("MHD_TUNE_VERBOSE"))
            fprintf(stderr, "mhd_autotune %dx%d p%d V=%d BY=%d W=%d: %.4f ms/step\n", l->nx, l->ny, l->p.precision,
                    c.nodes_per_thread, c.rows_per_block, c.warps_per_sm, *ms / iters);
        return err;
    };
    auto give_up = [&](cudaError_t err) {
        l->cfg = saved;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (scratch) cudaFree(scratch);
        return cuda_fail(err, "autotune candidate");
    };
    // every shape at the built-in staging depth ...
    for (int V : {1, 2, 4}) {
        for (int BY : {1, 2, 4, 8, 16}) {
            mhd_kernel_config c{V, BY, 0};
            if (!config_ok(l, c)) continue;
            float ms = 0;
            const cudaError_t err = time_config(c, &ms);
            if (err != cudaSuccess) return give_up(err);
            if (ms < best_ms) {
                best_ms = ms;
                chosen = c;
            }
        }
    }
    // ... then the fastest one at other depths (the x-wall kernel has none)
    if (l->p.bc_x != MHD_WALL) {
        const int rule = mhd::step_rule_warps(l->p.precision, chosen.nodes_per_thread);
        const mhd_kernel_config shape = chosen;
        float depth_ms = best_ms;
        for (int num : {2, 3, 6, 8}) {  // quarters of the rule's depth
            const int W = std::min(64, std::max(shape.rows_per_block, rule * num / 4));
            if (W / shape.rows_per_block == rule / shape.rows_per_block) continue;  // the same grid
            mhd_kernel_config c{shape.nodes_per_thread, shape.rows_per_block, W};
            float ms = 0;
            const cudaError_t err = time_config(c, &ms);
            if (err != cudaSuccess) return give_up(err);
            if (ms < depth_ms) {
                depth_ms = ms;
                if (ms < 0.99f * best_ms) chosen = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (scratch) {
        CK(cudaStreamSynchronize(l->stream), "mhd_autotune");
        cudaFree(scratch);
    }
    l->cfg = saved;
    l->prev_valid = false;  // the spare buffer was overwritten
    mhd_status s = mhd_set_kernel_config(l, &chosen);
    if (s != MHD_OK) return s;
    if (path) {
        auto m = read_cache(path);
        m[key] = chosen;
        write_cache(path, m);
    }
    if (best) *best = l->cfg;
    return MHD_OK;
}

}  // extern "C"
