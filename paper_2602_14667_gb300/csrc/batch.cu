// batch.cu -- ensemble of independent periodic lattices (uneven sizes, own
// nu and eta) advanced by ONE persistent kernel launch per time step.
//
// All lattices live in one pair of FP32 population buffers (19 planes each,
// lattice after lattice).  The host builds a work-list of tiles -- one tile
// is rows_per_block rows x 32*V columns of one lattice -- and the kernel is
// launched with as many blocks as fit on the GPU at once; every block walks
// the tile list with a fixed stride.  Each warp of a block updates one row
// segment of its tile with the same fused pull-stream + RR-MHD collision
// as the single-lattice kernel (step_row.cuh), so a batched lattice is
// bitwise identical to the same lattice advanced alone with the same shape.
// The step loop is captured in a CUDA graph (64 steps per graph).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include "../../include/mhd.h"
#include "diag_device.cuh"
#include "internal.h"
#include "step_row.cuh"

namespace mhd {

struct BatchLattice {
    long long offset;  // first element of the lattice in each buffer
    long long pitch, plane;
    int nx, ny;
    NodeParams<float> np;
};

struct BatchTile {
    int lat, xblock, y0, pad;
};

// Off: int offsets when every lattice's state has fewer than 2^31 elements.
template <int V, typename Off>
__global__ void __launch_bounds__(512) batch_step(const BatchLattice* __restrict__ lats,
                                                  const BatchTile* __restrict__ tiles, int ntiles,
                                                  const float* __restrict__ src, float* __restrict__ dst) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tile = tiles[t];
        const BatchLattice L = lats[tile.lat];
        const int y = tile.y0 + threadIdx.y;
        if (y < L.ny)  // uniform over the warp
            step_row<1, V, false, Off>(src + L.offset, dst + L.offset, L.nx, L.ny, L.pitch, L.plane,
                                       L.np, tile.xblock, y, threadIdx.x);
    }
}

// A sample step of the ensemble: batch_step that also reduces the point
// totals of every lattice's pre-collision state (mass, momentum, energies,
// cross helicity, sum b, max |j_z|; the arithmetic of the diagnostics,
// diag_device.cuh) from the populations each warp collides.  Each block
// takes a contiguous run of the tile list (the tiles come lattice by
// lattice), adds its rows into compensated FP32 lane sums and, when the
// lattice changes and at the end, reduces them in FP64 into the partial of
// the first tile of that lattice's run; the block's other tiles get zero
// partials (kDiagSlots doubles per tile; the gradient slots 8, 9, 10, 12
// zero), which launch_diag_batch_final reduces per lattice in tile order.
// The populations are batch_step's.
template <int V, typename Off>
__global__ void __launch_bounds__(512) batch_step_totals(const BatchLattice* __restrict__ lats,
                                                         const BatchTile* __restrict__ tiles, int ntiles,
                                                         const float* __restrict__ src, float* __restrict__ dst,
                                                         double* __restrict__ tile_partials) {
    using MB = AbsBits<float>;
    __shared__ double red[16][kDiagSlots];
    const int lane = threadIdx.x, warp = threadIdx.y, tid = threadIdx.y * 32 + lane;
    const int chunk = (ntiles + gridDim.x - 1) / gridDim.x;
    const int t0 = blockIdx.x * chunk, t1 = min(ntiles, t0 + chunk);
    LaneSum<float> ls[8];
    MB::T mjz = 0;
    // the block's sums so far into the partial of tile `slot` (block-uniform)
    auto flush = [&](int slot) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const double w = warp_sum(ls[q].take());
            if (lane == 0) red[warp][q] = w;
        }
        const unsigned long long m = warp_max_bits(dbits(MB::value(mjz)));
        mjz = 0;
        if (lane == 0) {
            red[warp][8] = red[warp][9] = red[warp][10] = red[warp][12] = 0.0;
            red[warp][11] = __longlong_as_double((long long)m);
        }
        __syncthreads();
        if (tid < kDiagSlots) {
            double a = red[0][tid];
            for (int w = 1; w < (int)blockDim.y; ++w)
                a = tid < 10 ? a + red[w][tid] : __longlong_as_double((long long)max_bits(dbits(a), dbits(red[w][tid])));
            tile_partials[(long long)slot * kDiagSlots + tid] = a;
        }
        __syncthreads();  // red is rewritten by the next flush
    };
    int cur = -1, first = t0;
    for (int t = t0; t < t1; ++t) {
        const BatchTile tile = tiles[t];
        if (tile.lat != cur) {  // uniform over the block
            if (cur >= 0) flush(first);
            cur = tile.lat;
            first = t;
        } else if (tid < kDiagSlots) {
            tile_partials[(long long)t * kDiagSlots + tid] = 0.0;
        }
        const BatchLattice L = lats[tile.lat];
        const int y = tile.y0 + threadIdx.y;
        if (y < L.ny) {  // uniform over the warp
            float v[kPlanes][V];
            if (gather_row<1, V, false, Off>(src + L.offset, L.nx, L.ny, L.pitch, L.plane, tile.xblock, y, lane, v)) {
                float ps[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) ps[q] = 0.f;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    float f[9], g[10];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = v[i][k];
#pragma unroll
                    for (int q = 0; q < 10; ++q) g[q] = v[9 + q][k];
                    const NodeMom<float> n = node_moments(f, g, 1.f, L.np.rho0);
                    add_point_sums(n, ps);
                    mjz = max(mjz, MB::of(node_current(n, L.np.omega_m, 1.f)));
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) ls[q].add(ps[q]);
                collide_nodes<float, V, false, kNative>(v, L.np);
                const int x0 = (tile.xblock * 32 + lane) * V;
                const Off o_0 = (Off)y * (Off)L.pitch, pl = (Off)L.plane;
                float* d = dst + L.offset;
#pragma unroll
                for (int p = 0; p < kPlanes; ++p) {
                    float r[V];
                    StepCodec<float, V>::to_storage(v[p], r);
                    VecIO<float, V>::store(d + ((Off)p * pl + o_0 + x0), r);
                }
            }
        }
    }
    if (cur >= 0) flush(first);
}

}  // namespace mhd

namespace {

mhd_status bfail(mhd_status s, const std::string& m) {
    mhd::set_last_error(m);
    return s;
}
mhd_status bcuda(cudaError_t e, const char* what) {
    return bfail(e == cudaErrorMemoryAllocation ? MHD_ENOMEM : MHD_ECUDA,
                 std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}
#define BCK(call, what)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return bcuda(e_, what);  \
    } while (0)

constexpr int kBatchGraphSteps = 64;

}  // namespace

struct mhd_batch {
    int count = 0;
    int dev = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;
    std::vector<mhd_params> params;
    std::vector<mhd::Layout> layouts;
    std::vector<long long> offsets;
    std::vector<char> set;        // fields set for lattice i
    std::vector<char> prev_valid; // the spare buffer holds the state the last step read
    std::vector<char> is_eq;      // lattice i holds an equilibrium state (no step since set)
    long long total_elems = 0, nodes = 0;
    bool wide = false;            // some lattice's state has 2^31 elements or more
    float* buf[2] = {nullptr, nullptr};
    int cur = 0;
    long long step = 0;
    mhd::BatchLattice* d_lats = nullptr;
    mhd::BatchTile* d_tiles = nullptr;
    int ntiles = 0;
    int grid = 0;
    mhd_kernel_config cfg{4, 4};
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    double* io = nullptr;
    long long io_elems = 0;
    double* partials = nullptr;
    double* totals_d = nullptr;
    double* totals_h = nullptr;
    mhd::DiagEnsemble diag;  // the all-lattice diagnostics tables (built on first use)
    // the sample step's per-tile partials and each lattice's first tile
    double* tile_partials = nullptr;
    int* d_tile_first = nullptr;
    double* d_mass = nullptr;  // rho0 * nodes of each lattice
};

namespace {

void batch_drop_graphs(mhd_batch* b) {
    for (auto& g : b->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

bool batch_shape_ok(const mhd_batch* b, const mhd_kernel_config& c) {
    if (c.rows_per_block < 1 || c.rows_per_block > 16) return false;
    if (c.warps_per_sm < 0 || c.warps_per_sm > 64) return false;
    if (c.nodes_per_thread != 1 && c.nodes_per_thread != 2 && c.nodes_per_thread != 4) return false;
    for (auto& L : b->layouts)
        if (L.nx % c.nodes_per_thread) return false;
    return true;
}

using BatchKernel = void (*)(const mhd::BatchLattice*, const mhd::BatchTile*, int, const float*, float*);

BatchKernel batch_kernel(bool wide, int V) {
    switch (V) {
    case 1: return wide ? mhd::batch_step<1, long long> : mhd::batch_step<1, int>;
    case 2: return wide ? mhd::batch_step<2, long long> : mhd::batch_step<2, int>;
    case 4: return wide ? mhd::batch_step<4, long long> : mhd::batch_step<4, int>;
    }
    return nullptr;
}

using BatchTotalsKernel = void (*)(const mhd::BatchLattice*, const mhd::BatchTile*, int, const float*, float*,
                                  double*);

BatchTotalsKernel batch_totals_kernel(bool wide, int V) {
    switch (V) {
    case 1: return wide ? mhd::batch_step_totals<1, long long> : mhd::batch_step_totals<1, int>;
    case 2: return wide ? mhd::batch_step_totals<2, long long> : mhd::batch_step_totals<2, int>;
    case 4: return wide ? mhd::batch_step_totals<4, long long> : mhd::batch_step_totals<4, int>;
    }
    return nullptr;
}

cudaError_t launch_batch(const mhd_batch* b, int from, int V, cudaStream_t st) {
    dim3 block(32, b->cfg.rows_per_block);
    const float* src = b->buf[from];
    float* dst = b->buf[from ^ 1];
    const BatchKernel k = batch_kernel(b->wide, V);
    if (!k) return cudaErrorInvalidValue;
    k<<<b->grid, block, 0, st>>>(b->d_lats, b->d_tiles, b->ntiles, src, dst);
    return cudaGetLastError();
}

// Tile list and persistent grid for a launch shape.
mhd_status batch_configure(mhd_batch* b, const mhd_kernel_config& c) {
    std::vector<mhd::BatchTile> tiles;
    const int cols = 32 * c.nodes_per_thread, rows = c.rows_per_block;
    for (int l = 0; l < b->count; ++l) {
        const auto& L = b->layouts[l];
        for (int y0 = 0; y0 < L.ny; y0 += rows)
            for (int xb = 0; xb * cols < L.nx; ++xb) tiles.push_back({l, xb, y0, 0});
    }
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    BCK(cudaMalloc(&b->d_tiles, sizeof(mhd::BatchTile) * tiles.size()), "cudaMalloc(tiles)");
    BCK(cudaMemcpy(b->d_tiles, tiles.data(), sizeof(mhd::BatchTile) * tiles.size(),
                   cudaMemcpyHostToDevice),
        "H2D tiles");
    b->ntiles = (int)tiles.size();
    // the tiles of lattice l are [first[l], first[l + 1]) (they come lattice by lattice)
    std::vector<int> first(b->count + 1, 0);
    for (size_t k = tiles.size(); k-- > 0;) first[tiles[k].lat] = (int)k;
    first[b->count] = b->ntiles;
    if (b->tile_partials) cudaFree(b->tile_partials);
    if (b->d_tile_first) cudaFree(b->d_tile_first);
    b->tile_partials = nullptr;
    b->d_tile_first = nullptr;
    BCK(cudaMalloc(&b->tile_partials, sizeof(double) * mhd::kDiagSlots * tiles.size()), "cudaMalloc(tile partials)");
    BCK(cudaMalloc(&b->d_tile_first, sizeof(int) * (b->count + 1)), "cudaMalloc(tile ranges)");
    BCK(cudaMemcpy(b->d_tile_first, first.data(), sizeof(int) * (b->count + 1), cudaMemcpyHostToDevice),
        "H2D tile ranges");
    if (!b->d_mass) {
        std::vector<double> mass(b->count);
        for (int l = 0; l < b->count; ++l)
            mass[l] = b->params[l].rho0 * (double)b->layouts[l].nx * (double)b->layouts[l].ny;
        BCK(cudaMalloc(&b->d_mass, sizeof(double) * b->count), "cudaMalloc(mass)");
        BCK(cudaMemcpy(b->d_mass, mass.data(), sizeof(double) * b->count, cudaMemcpyHostToDevice), "H2D mass");
    }
    int per_sm = 0, sms = 0;
    const int threads = 32 * rows;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel(b->wide, c.nodes_per_thread),
                                                      threads, 0),
        "occupancy");
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev), "SM count");
    per_sm = std::max(1, per_sm);
    // staging depth: every resident block unless the shape caps the warps per SM
    if (c.warps_per_sm > 0) per_sm = std::min(per_sm, std::max(1, c.warps_per_sm / rows));
    b->grid = std::max(1, std::min(b->ntiles, per_sm * sms));
    batch_drop_graphs(b);
    b->cfg = c;
    return MHD_OK;
}

mhd_status batch_index(const mhd_batch* b, int i) {
    if (!b) return bfail(MHD_EINVAL, "batch is NULL");
    if (i < 0 || i >= b->count) return bfail(MHD_EINVAL, "lattice index out of range");
    return MHD_OK;
}

mhd_status batch_io(mhd_batch* b, long long n) {
    if (b->io && b->io_elems >= n) return MHD_OK;
    if (b->io) cudaFree(b->io);
    b->io = nullptr;
    BCK(cudaMalloc(&b->io, sizeof(double) * n), "cudaMalloc(io)");
    b->io_elems = n;
    return MHD_OK;
}

}  // namespace

extern "C" {

mhd_status mhd_batch_create(int count, const int* nx, const int* ny, const mhd_params* params,
                            void* stream, mhd_batch** out) {
    if (!out) return bfail(MHD_EINVAL, "out is NULL");
    *out = nullptr;
    if (count < 1 || !nx || !ny || !params) return bfail(MHD_EINVAL, "count >= 1 and non-NULL arrays required");
    for (int i = 0; i < count; ++i) {
        const mhd_params& p = params[i];
        if (nx[i] < 2 || ny[i] < 2 || (long long)nx[i] * ny[i] > (1LL << 31))
            return bfail(MHD_EINVAL, "lattice " + std::to_string(i) + ": bad size");
        if (!(p.tau_f > 0.5) || !(p.tau_m > 0.5) || !std::isfinite(p.tau_f) || !std::isfinite(p.tau_m))
            return bfail(MHD_EINVAL, "lattice " + std::to_string(i) + ": tau must be > 1/2");
        if (!(p.rho0 > 0) || !std::isfinite(p.rho0)) return bfail(MHD_EINVAL, "rho0 must be > 0");
        if (p.precision != MHD_FP32 || p.bc_x != MHD_PERIODIC || p.bc_y != MHD_PERIODIC)
            return bfail(MHD_EINVAL, "batched lattices are FP32 and periodic");
        if ((p.eq_variant != 0 && p.eq_variant != 1) || (p.collision != MHD_RR && p.collision != MHD_BGK) ||
            (p.mag_collision != MHD_MAG_BGK && p.mag_collision != MHD_MAG_REGULARISED))
            return bfail(MHD_EINVAL, "unknown eq_variant / collision / mag_collision");
        if (p.streaming != MHD_TWO_BUFFERS) return bfail(MHD_EINVAL, "batched lattices use two buffers");
    }
    auto* b = new (std::nothrow) mhd_batch();
    if (!b) return bfail(MHD_ENOMEM, "host allocation failed");
    b->count = count;
    b->stream = static_cast<cudaStream_t>(stream);
    b->params.assign(params, params + count);
    b->set.assign(count, 0);
    b->prev_valid.assign(count, 0);
    b->is_eq.assign(count, 0);
    std::vector<mhd::BatchLattice> lats(count);
    long long maxn = 0;
    for (int i = 0; i < count; ++i) {
        mhd::Layout L = mhd::make_layout(nx[i], ny[i], MHD_FP32);
        b->layouts.push_back(L);
        b->offsets.push_back(b->total_elems);
        lats[i].offset = b->total_elems;
        lats[i].pitch = L.pitch;
        lats[i].plane = L.plane;
        lats[i].nx = nx[i];
        lats[i].ny = ny[i];
        lats[i].np.omega = (float)(1.0 / params[i].tau_f);
        lats[i].np.omega_m = (float)(1.0 / params[i].tau_m);
        lats[i].np.rho0 = (float)params[i].rho0;
        lats[i].np.variant = params[i].eq_variant;
        lats[i].np.collision = params[i].collision;
        lats[i].np.mag_collision = params[i].mag_collision;
        b->total_elems += (long long)mhd::kStatePlanes * L.plane;
        if ((long long)mhd::kStatePlanes * L.plane >= (1LL << 31)) b->wide = true;
        b->nodes += (long long)nx[i] * ny[i];
        maxn = std::max(maxn, (long long)nx[i] * ny[i]);
    }
    cudaError_t e = cudaGetDevice(&b->dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&b->buf[k], sizeof(float) * b->total_elems);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_lats, sizeof(mhd::BatchLattice) * count);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_lats, lats.data(), sizeof(mhd::BatchLattice) * count, cudaMemcpyHostToDevice);
    int maxblocks = 0;
    for (auto& L : b->layouts) maxblocks = std::max(maxblocks, mhd::diag_blocks(L));
    if (e == cudaSuccess) e = cudaMalloc(&b->partials, sizeof(double) * mhd::kDiagSlots * maxblocks);
    // one slot set of totals per lattice (mhd_batch_get_all_totals)
    if (e == cudaSuccess) e = cudaMalloc(&b->totals_d, sizeof(double) * mhd::kDiagSlots * b->count);
    if (e == cudaSuccess) e = cudaMallocHost(&b->totals_h, sizeof(double) * mhd::kDiagSlots * b->count);
    if (e != cudaSuccess) {
        cudaGetLastError();
        mhd_batch_destroy(b);
        return bcuda(e, "mhd_batch_create");
    }
    mhd_kernel_config c{4, 4};
    while (!batch_shape_ok(b, c) && c.nodes_per_thread > 1) c.nodes_per_thread >>= 1;
    mhd_status s = batch_configure(b, c);
    if (s != MHD_OK) {
        mhd_batch_destroy(b);
        return s;
    }
    (void)maxn;
    *out = b;
    return MHD_OK;
}

mhd_status mhd_batch_destroy(mhd_batch* b) {
    if (!b) return bfail(MHD_EINVAL, "batch is NULL");
    cudaSetDevice(b->dev);
    cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (auto& p : b->buf)
        if (p) cudaFree(p);
    if (b->d_lats) cudaFree(b->d_lats);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->io) cudaFree(b->io);
    if (b->partials) cudaFree(b->partials);
    if (b->totals_d) cudaFree(b->totals_d);
    if (b->totals_h) cudaFreeHost(b->totals_h);
    mhd::diag_ensemble_destroy(b->diag);
    if (b->tile_partials) cudaFree(b->tile_partials);
    if (b->d_tile_first) cudaFree(b->d_tile_first);
    if (b->d_mass) cudaFree(b->d_mass);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return MHD_OK;
}

mhd_status mhd_batch_nodes(const mhd_batch* b, long long* nodes) {
    if (!b || !nodes) return bfail(MHD_EINVAL, "NULL argument");
    *nodes = b->nodes;
    return MHD_OK;
}

mhd_status mhd_batch_set_fields(mhd_batch* b, int index, const double* ux, const double* uy,
                                const double* bx, const double* by, const double* rho) {
    mhd_status s = batch_index(b, index);
    if (s != MHD_OK) return s;
    if (!ux || !uy || !bx || !by) return bfail(MHD_EINVAL, "NULL field");
    const mhd::Layout& L = b->layouts[index];
    const long long n = (long long)L.nx * L.ny;
    for (const double* a : {ux, uy, bx, by, rho})
        if (a)
            for (long long k = 0; k < n; ++k)
                if (!std::isfinite(a[k])) return bfail(MHD_EINVAL, "non-finite input field");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    s = batch_io(b, 5 * n);
    if (s != MHD_OK) return s;
    double* d[5] = {b->io, b->io + n, b->io + 2 * n, b->io + 3 * n, b->io + 4 * n};
    const double* h[5] = {ux, uy, bx, by, rho};
    for (int q = 0; q < 5; ++q)
        if (h[q]) BCK(cudaMemcpyAsync(d[q], h[q], sizeof(double) * n, cudaMemcpyHostToDevice, b->stream), "H2D");
    BCK(mhd::launch_init(L, MHD_FP32, b->buf[b->cur] + b->offsets[index], rho ? d[4] : nullptr, d[0], d[1],
                         d[2], d[3], b->params[index].rho0, b->params[index].eq_variant, b->stream),
        "init kernel");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_set_fields");
    b->set[index] = 1;
    b->prev_valid[index] = 0;
    b->is_eq[index] = 1;
    return MHD_OK;
}

static mhd_status batch_capture(mhd_batch* b, int from) {
    cudaGraph_t g = nullptr;
    BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    int c = from;
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kBatchGraphSteps && le == cudaSuccess; ++k) {
        le = launch_batch(b, c, b->cfg.nodes_per_thread, b->cap);
        c ^= 1;
    }
    cudaError_t ee = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(le, "batch launch during capture");
    }
    if (ee != cudaSuccess) return bcuda(ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&b->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return bcuda(ie, "graph instantiate");
    return MHD_OK;
}

mhd_status mhd_batch_advance(mhd_batch* b, long long nsteps) {
    if (!b) return bfail(MHD_EINVAL, "batch is NULL");
    if (nsteps < 0) return bfail(MHD_EINVAL, "nsteps must be >= 0");
    for (int i = 0; i < b->count; ++i)
        if (!b->set[i]) return bfail(MHD_ESTATE, "set the fields of every lattice first");
    if (nsteps == 0) return MHD_OK;
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    while (nsteps >= kBatchGraphSteps) {
        if (!b->graph[b->cur]) {
            mhd_status s = batch_capture(b, b->cur);
            if (s != MHD_OK) return s;
        }
        BCK(cudaGraphLaunch(b->graph[b->cur], b->stream), "graph launch");
        nsteps -= kBatchGraphSteps;
        b->step += kBatchGraphSteps;
    }
    while (nsteps > 0) {
        BCK(launch_batch(b, b->cur, b->cfg.nodes_per_thread, b->stream), "batch launch");
        b->cur ^= 1;
        --nsteps;
        ++b->step;
    }
    std::fill(b->prev_valid.begin(), b->prev_valid.end(), 1);
    std::fill(b->is_eq.begin(), b->is_eq.end(), 0);
    return MHD_OK;
}

mhd_status mhd_batch_advance_totals(mhd_batch* b, long long nsteps, mhd_totals* out) {
    if (!b || !out) return bfail(MHD_EINVAL, "NULL argument");
    if (nsteps < 1) return bfail(MHD_EINVAL, "nsteps must be >= 1");
    mhd_status s = mhd_batch_advance(b, nsteps - 1);
    if (s != MHD_OK) return s;
    const BatchTotalsKernel k = batch_totals_kernel(b->wide, b->cfg.nodes_per_thread);
    if (!k) return bfail(MHD_EINVAL, "launch shape");
    const float* src = b->buf[b->cur];
    float* dst = b->buf[b->cur ^ 1];
    // one resident wave of this kernel (its blocks take contiguous runs of tiles)
    const int threads = 32 * b->cfg.rows_per_block;
    int per_sm = 0;
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, 0), "occupancy");
    const int grid = std::max(1, std::min(b->ntiles, std::max(1, per_sm) * mhd::device_sms()));
    k<<<grid, dim3(32, b->cfg.rows_per_block), 0, b->stream>>>(b->d_lats, b->d_tiles, b->ntiles, src, dst,
                                                              b->tile_partials);
    BCK(cudaGetLastError(), "ensemble step with totals");
    b->cur ^= 1;
    ++b->step;
    std::fill(b->prev_valid.begin(), b->prev_valid.end(), 1);
    std::fill(b->is_eq.begin(), b->is_eq.end(), 0);
    BCK(mhd::launch_diag_batch_final(b->tile_partials, b->d_tile_first, b->d_mass, b->count, b->totals_d, b->stream),
        "ensemble point totals");
    BCK(cudaMemcpyAsync(b->totals_h, b->totals_d, sizeof(double) * mhd::kDiagSlots * b->count,
                        cudaMemcpyDeviceToHost, b->stream),
        "D2H totals");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_advance_totals");
    int bad = -1;
    for (int i = 0; i < b->count; ++i) {
        const double* t = b->totals_h + (long long)mhd::kDiagSlots * i;
        const mhd::Layout& L = b->layouts[i];
        const double n = (double)L.nx * L.ny;
        mhd_totals& o = out[i];
        o.mass = t[0]; o.mom_x = t[1]; o.mom_y = t[2];
        o.e_kin = t[3] / n; o.e_mag = t[4] / n; o.cross_hel = t[5] / n;
        o.bsum_x = t[6]; o.bsum_y = t[7];
        o.divb_rms = o.divb_max = o.omega_max = std::nan("");
        o.jz_max = t[11];
        o.step = b->step;
        for (int q : {0, 1, 2, 3, 4, 5, 6, 7, 11})
            if (!std::isfinite(t[q]) && bad < 0) bad = i;
    }
    if (bad >= 0)
        return bfail(MHD_EUNSTABLE, "non-finite point totals in lattice " + std::to_string(bad) + ": the run blew up");
    return MHD_OK;
}

mhd_status mhd_batch_get_fields(mhd_batch* b, int index, double* rho, double* ux, double* uy,
                                double* bx, double* by) {
    mhd_status s = batch_index(b, index);
    if (s != MHD_OK) return s;
    if (!b->set[index]) return bfail(MHD_ESTATE, "fields of this lattice were not set");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    const mhd::Layout& L = b->layouts[index];
    const long long n = (long long)L.nx * L.ny;
    s = batch_io(b, 5 * n);
    if (s != MHD_OK) return s;
    double* d[5] = {b->io, b->io + n, b->io + 2 * n, b->io + 3 * n, b->io + 4 * n};
    double* h[5] = {rho, ux, uy, bx, by};
    BCK(mhd::launch_fields(L, MHD_FP32, b->buf[b->cur] + b->offsets[index], b->params[index].rho0,
                           h[0] ? d[0] : nullptr, h[1] ? d[1] : nullptr, h[2] ? d[2] : nullptr,
                           h[3] ? d[3] : nullptr, h[4] ? d[4] : nullptr, b->stream),
        "fields kernel");
    for (int q = 0; q < 5; ++q)
        if (h[q]) BCK(cudaMemcpyAsync(h[q], d[q], sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream), "D2H");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_get_fields");
    return MHD_OK;
}

// The diagnostics pass of lattice `index` into slot set `slot` of totals_d.
static cudaError_t batch_diag(mhd_batch* b, int index, int slot) {
    const mhd::Layout& L = b->layouts[index];
    mhd::DiagLaunch d;
    d.L = L;
    d.prec = MHD_FP32;
    d.prev = b->buf[b->cur ^ 1] + b->offsets[index];
    d.cur = b->buf[b->cur] + b->offsets[index];
    d.mode = b->prev_valid[index] ? 0 : 1;
    d.omega_m = 1.0 / b->params[index].tau_m;
    d.rho0 = b->params[index].rho0;
    const double om1 = 1.0 - d.omega_m;
    d.neq_scale = d.mode == 0 ? 1.0 : ((b->is_eq[index] || std::fabs(om1) < 1e-12) ? 0.0 : 1.0 / om1);
    d.wall_x = d.wall_y = 0;
    return mhd::launch_diag(d, b->partials, mhd::diag_blocks(L), b->totals_d + (long long)mhd::kDiagSlots * slot,
                            b->stream);
}

static bool batch_totals_out(const mhd_batch* b, int index, const double* t, mhd_totals* out) {
    const mhd::Layout& L = b->layouts[index];
    const double n = (double)L.nx * L.ny;
    out->mass = t[0]; out->mom_x = t[1]; out->mom_y = t[2];
    out->e_kin = t[3] / n; out->e_mag = t[4] / n; out->cross_hel = t[5] / n;
    out->bsum_x = t[6]; out->bsum_y = t[7];
    out->divb_rms = t[9] > 0 ? std::sqrt(t[8] / t[9]) : 0.0;
    out->divb_max = t[10]; out->jz_max = t[11]; out->omega_max = t[12];
    out->step = b->step;
    for (int k = 0; k < mhd::kDiagSlots; ++k)
        if (!std::isfinite(t[k])) return false;
    return true;
}

mhd_status mhd_batch_get_totals(mhd_batch* b, int index, mhd_totals* out) {
    mhd_status s = batch_index(b, index);
    if (s != MHD_OK) return s;
    if (!out) return bfail(MHD_EINVAL, "out is NULL");
    if (!b->set[index]) return bfail(MHD_ESTATE, "fields of this lattice were not set");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    BCK(batch_diag(b, index, 0), "diagnostics kernel");
    BCK(cudaMemcpyAsync(b->totals_h, b->totals_d, sizeof(double) * mhd::kDiagSlots, cudaMemcpyDeviceToHost,
                        b->stream),
        "D2H totals");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_get_totals");
    if (!batch_totals_out(b, index, b->totals_h, out))
        return bfail(MHD_EUNSTABLE, "non-finite diagnostics: the run blew up");
    return MHD_OK;
}

mhd_status mhd_batch_get_all_totals(mhd_batch* b, mhd_totals* out) {
    if (!b || !out) return bfail(MHD_EINVAL, "NULL argument");
    for (int i = 0; i < b->count; ++i)
        if (!b->set[i]) return bfail(MHD_ESTATE, "the fields of every lattice must be set");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    // one launch over the tiles of every lattice; where a lattice's rows do
    // not allow its vector loads, every lattice's pass queued back to back
    // (the partials are reused in stream order); then one copy, one wait
    if (!b->diag.d_args) {
        std::vector<double> rho0(b->count);
        for (int i = 0; i < b->count; ++i) rho0[i] = b->params[i].rho0;
        BCK(mhd::diag_ensemble_create(b->diag, b->layouts.data(), rho0.data(), b->count), "ensemble diagnostics tables");
    }
    std::vector<mhd::DiagLatticeState> st(b->count);
    for (int i = 0; i < b->count; ++i) {
        mhd::DiagLatticeState& d = st[i];
        d.prev = b->buf[b->cur ^ 1] + b->offsets[i];
        d.cur = b->buf[b->cur] + b->offsets[i];
        d.mode = b->prev_valid[i] ? 0 : 1;
        d.omega_m = 1.0 / b->params[i].tau_m;
        d.rho0 = b->params[i].rho0;
        const double om1 = 1.0 - d.omega_m;
        d.neq_scale = d.mode == 0 ? 1.0 : ((b->is_eq[i] || std::fabs(om1) < 1e-12) ? 0.0 : 1.0 / om1);
    }
    const cudaError_t le = mhd::diag_ensemble_launch(b->diag, b->layouts.data(), st.data(), b->totals_d, b->stream);
    if (le == cudaErrorNotSupported) {
        for (int i = 0; i < b->count; ++i) BCK(batch_diag(b, i, i), "diagnostics kernel");
    } else {
        BCK(le, "ensemble diagnostics kernel");
    }
    BCK(cudaMemcpyAsync(b->totals_h, b->totals_d, sizeof(double) * mhd::kDiagSlots * b->count,
                        cudaMemcpyDeviceToHost, b->stream),
        "D2H totals");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_get_all_totals");
    int bad = -1;
    for (int i = 0; i < b->count; ++i)
        if (!batch_totals_out(b, i, b->totals_h + (long long)mhd::kDiagSlots * i, out + i) && bad < 0) bad = i;
    if (bad >= 0)
        return bfail(MHD_EUNSTABLE, "non-finite diagnostics in lattice " + std::to_string(bad) + ": the run blew up");
    return MHD_OK;
}

mhd_status mhd_batch_get_kernel_config(const mhd_batch* b, mhd_kernel_config* out) {
    if (!b || !out) return bfail(MHD_EINVAL, "NULL argument");
    *out = b->cfg;
    return MHD_OK;
}

mhd_status mhd_batch_set_kernel_config(mhd_batch* b, const mhd_kernel_config* cfg) {
    if (!b || !cfg) return bfail(MHD_EINVAL, "NULL argument");
    if (!batch_shape_ok(b, *cfg)) return bfail(MHD_EINVAL, "launch shape not valid for these lattices");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_set_kernel_config");
    return batch_configure(b, *cfg);
}

mhd_status mhd_batch_autotune(mhd_batch* b, mhd_kernel_config* best) {
    if (!b) return bfail(MHD_EINVAL, "batch is NULL");
    for (int i = 0; i < b->count; ++i)
        if (!b->set[i]) return bfail(MHD_ESTATE, "set the fields of every lattice first");
    BCK(cudaSetDevice(b->dev), "cudaSetDevice");
    BCK(cudaStreamSynchronize(b->stream), "mhd_batch_autotune");
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0), "event");
    BCK(cudaEventCreate(&e1), "event");
    mhd_kernel_config chosen = b->cfg;
    float best_ms = 1e30f;
    // one candidate: configure, two untimed and five timed steps
    auto time_config = [&](const mhd_kernel_config& c, float* ms) -> mhd_status {
        mhd_status s = batch_configure(b, c);
        if (s != MHD_OK) return s;
        const int V = c.nodes_per_thread;
        cudaError_t err = cudaSuccess;
        for (int k = 0; k < 2 && err == cudaSuccess; ++k) err = launch_batch(b, b->cur, V, b->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 5 && err == cudaSuccess; ++k) err = launch_batch(b, b->cur, V, b->stream);
        if (err == cudaSuccess) err = cudaEventRecord(e1, b->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(ms, e0, e1);
        if (err != cudaSuccess) return bcuda(err, "batch autotune candidate");
        if (getenv("MHD_TUNE_VERBOSE"))
            fprintf(stderr, "mhd_batch_autotune V=%d BY=%d W=%d grid=%d tiles=%d: %.4f ms/step\n", V,
                    c.rows_per_block, c.warps_per_sm, b->grid, b->ntiles, *ms / 5);
        return MHD_OK;
    };
    auto done = [&](mhd_status s) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return s;
    };
    for (int V : {1, 2, 4})
        for (int BY : {1, 2, 4, 8, 16}) {
            mhd_kernel_config c{V, BY, 0};
            if (!batch_shape_ok(b, c)) continue;
            float ms = 0;
            const mhd_status s = time_config(c, &ms);
            if (s != MHD_OK) return done(s);
            if (ms < best_ms) {
                best_ms = ms;
                chosen = c;
            }
        }
    // the fastest shape with fewer warps in flight per SM than fit (kept
    // only if at least 1 % faster)
    {
        const mhd_kernel_config shape = chosen;
        float depth_ms = best_ms;
        for (int W : {8, 16, 32}) {
            if (W < shape.rows_per_block) continue;
            mhd_kernel_config c{shape.nodes_per_thread, shape.rows_per_block, W};
            float ms = 0;
            const mhd_status s = time_config(c, &ms);
            if (s != MHD_OK) return done(s);
            if (ms < depth_ms) {
                depth_ms = ms;
                if (ms < 0.99f * best_ms) chosen = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::fill(b->prev_valid.begin(), b->prev_valid.end(), 0);  // the spare buffer was overwritten
    mhd_status s = batch_configure(b, chosen);
    if (s != MHD_OK) return s;
    if (best) *best = b->cfg;
    return MHD_OK;
}

}  // extern "C"
