// diag.cu -- the global diagnostics of a lattice: mass, momentum, kinetic
// and magnetic energy, cross helicity, sum of b, div b (rms and max) and the
// maxima of the current density and the vorticity, reduced on the device in
// a fixed order.
//
// Definitions: the moments of task 1 of the "Algorithm of computation";
// j_z of Eq. current; the isotropic lattice gradient, the vorticity and the
// energies E_k = mean |u|^2/2, E_m = mean |b|^2/2 of the Orszag-Tang
// section.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <vector>

#include "diag_device.cuh"
#include "internal.h"
#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

// ---- tiles ------------------------------------------------------------------
// One warp walks one tile: a strip of 30 V output columns and up to H
// output rows [y0, y1) (H picked by the launcher so that the tiles are
// about as many as the resident warps).  Lane l holds the V nodes starting at
// x0s + l V with x0s = strip * 30 V - V: lanes 1..30 are the tile's own
// columns, lanes 0 and 31 the one-vector halo on either side, so the x
// neighbours of every output node arrive by warp shuffles and every load
// is an aligned vector (periodic x wraps the halo lanes around).  The warp
// forms the moments of rows y0 - 1 .. y1 one after the other (downwards
// in even row segments, upwards in odd ones) from the row's 19 planes --
// read with vector loads, and for the state the last step read with the
// step's pull gather -- adds the point sums of its output nodes, and keeps
// u and b of the last three rows in registers; once a row is formed the
// isotropic gradient stencil of the row before it is evaluated.  Each node
// is read by one tile, apart from the halo lanes and the two halo rows of
// each tile, which the neighbouring tiles read at about the same time.  No
// shared memory and no barrier is needed until the block's final
// reduction.
//
// Arithmetic: FP64 storage keeps every per-node quantity in FP64.  FP32 and
// FP16S storage form the per-node quantities in FP32; each lane adds them
// into an FP32 sum with an FP32 compensation term (Knuth's TwoSum recovers
// the rounding error of every addition exactly), and FP64 enters only in
// the warp, block and final reductions.  Mass is rho0 times the node count
// plus the sum of the density deviations, and the momentum is the sum of
// the first moments sum_i f_i c_i themselves.
//
// Per-block partials (kDiagSlots doubles):
//   0 sum (rho - rho0), 1 mom_x, 2 mom_y, 3 sum |u|^2/2, 4 sum |b|^2/2,
//   5 sum u.b, 6 sum b_x, 7 sum b_y, 8 sum (div b)^2, 9 #gradient nodes,
//   10 max |div b|, 11 max |j_z|, 12 max |omega_z|.
// The maxima of non-negative values are taken on their bit patterns with
// integer instructions (a NaN, whose pattern is above every finite value's,
// reaches the totals).
constexpr int kDWarps = 8;                 // warps per block (independent tiles)
constexpr int kDiagMaxBlocks = 4096;       // upper bound of any grid the launcher picks

template <typename C> struct DiagArgs {
    const void* src;   // mode 0: the buffer the last step read (gathered); mode 1: the stored state
    int nx, ny;
    long long pitch, plane;
    C omega_m, rho0, neq_scale;
    int wall_x, wall_y;
    int halo_y;        // rows -1 and ny are read from the ghost rows (a slab)
    int strips;        // tiles along x (30 V output columns each)
    int rows;          // output rows per tile (H)
    int ntiles;
    int mode = 0;      // ensembles: 0 gathered, 1 stored (the per-lattice choice of src above)
};

// u, b of one node (x, y) inside the lattice, one population at a time:
// mode 0 gathers the pre-collision state, mode 1 reads the stored one.
template <int PREC, int MODE>
__device__ __forceinline__ NodeMom<typename Prec<PREC>::C> scalar_node(
    const DiagArgs<typename Prec<PREC>::C>& a, int x, int y) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    const S* src = static_cast<const S*>(a.src);
    C f[9], g[10];
    if (MODE == 0) {
        gather_node(src, x, y, a.nx, a.ny, a.pitch, a.plane, a.wall_x, a.wall_y, f, g);
    } else {
        const long long o = (long long)y * a.pitch + x;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const C v = decode(src[(long long)p * a.plane + o]);
            if (p < 9) f[p] = v; else g[p - 9] = v;
        }
    }
    return node_moments(f, g, C(1), a.rho0);
}

// The accumulators of one warp: the lane sums of slots 0..8, the count of
// gradient nodes and the three maxima (as bit patterns).
template <typename C> struct DiagAcc {
    LaneSum<C> ls[9];
    long long cnt = 0;
    typename AbsBits<C>::T mdiv = 0, mjz = 0, mvort = 0;
    // the warp's 13 slot values (valid in lane 0); the sums restart
    __device__ __forceinline__ void warp_slots(double (&out)[kDiagSlots]) {
        using MB = AbsBits<C>;
#pragma unroll
        for (int q = 0; q < 9; ++q) out[q] = warp_sum(ls[q].take());
        out[9] = warp_sum((double)cnt);
        out[10] = __longlong_as_double((long long)warp_max_bits(dbits(MB::value(mdiv))));
        out[11] = __longlong_as_double((long long)warp_max_bits(dbits(MB::value(mjz))));
        out[12] = __longlong_as_double((long long)warp_max_bits(dbits(MB::value(mvort))));
    }
};

// ---- the tile kernel --------------------------------------------------------
// V: nodes per lane (vector loads; V = 1 also for lattices whose nx is not
// a multiple of the vector width).  GEN: x walls, one node per lane, every
// node gathered one population at a time (nodes outside the lattice are
// left at zero and never enter a valid stencil).  WALLY: y walls in the
// vector gather of mode 0.
// One tile t of lattice a into the warp's accumulators.
template <int PREC, int V, int MODE, bool WALLY, bool GEN>
__device__ __forceinline__ void diag_tile(const DiagArgs<typename Prec<PREC>::C>& a, int t, int lane,
                                          DiagAcc<typename Prec<PREC>::C>& acc) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    using MB = AbsBits<C>;
    constexpr int WO = 30 * V;  // output columns per tile
    // FP16S vector loads keep the step's storage units (2^12 x deviation)
    const C unit = (PREC == 2 && !GEN) ? C(kHalfInvScale) : C(1);
    const bool out_lane = lane >= 1 && lane <= 30;
    auto& ls = acc.ls;
    long long& cnt = acc.cnt;
    auto& mdiv = acc.mdiv;
    auto& mjz = acc.mjz;
    auto& mvort = acc.mvort;
    const int strip = t % a.strips, seg = t / a.strips;
    const int xl = strip * WO - V + lane * V;  // the lane's first node (may lie outside)
    int xw = xl;                               // ... wrapped (periodic x)
    if (!GEN) {
        xw %= a.nx;
        if (xw < 0) xw += a.nx;
    }
    const int y0 = seg * a.rows, y1 = min(a.ny, y0 + a.rows);
    // Odd segments walk upwards, so that the halo rows two neighbouring
    // tiles share are read by both at about the same time (the second
    // read then hits L2).
    const bool up = seg & 1;
    const C sgn = up ? C(-1) : C(1);  // orientation of the window in y
    // u_x, u_y, b_x, b_y of the last three rows formed (slots 0, 1, 2;
    // slot 2 the newest)
    C wnd[3][4][V];
    const int nrow = y1 - y0 + 2;
    for (int i = 0; i < nrow; ++i) {
        const int m = up ? y1 - i : y0 - 1 + i;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int k = 0; k < V; ++k) {
                wnd[0][q][k] = wnd[1][q][k];
                wnd[1][q][k] = wnd[2][q][k];
                wnd[2][q][k] = C(0);
            }
        int my = m;
        bool have = true;
        if ((my < 0 || my >= a.ny) && !a.halo_y) {
            if (a.wall_y) have = false;
            else my = my < 0 ? my + a.ny : my - a.ny;
        }
        if (have) {  // warp-uniform
            NodeMom<C> nm[V];
            bool inside = true;  // the lane's nodes lie inside the lattice
            if (GEN) {
                inside = xl >= 0 && xl < a.nx;
                if (inside) nm[0] = scalar_node<PREC, MODE>(a, xl, my);
            } else {
                C v[kPlanes][V];
                if (MODE == 0) {
                    gather_row_wrapped<PREC, V, WALLY>(static_cast<const S*>(a.src), a.nx, a.ny, a.pitch,
                                                       a.plane, xw, my, lane, v);
                } else {
                    const S* src = static_cast<const S*>(a.src) + (long long)my * a.pitch + xw;
                    S r[kPlanes][V];
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) VecIO<S, V>::load(src + (long long)p * a.plane, r[p]);
#pragma unroll
                    for (int p = 0; p < kPlanes; ++p) StepCodec<S, V>::to_compute(r[p], v[p]);
                }
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    C f[9], g[10];
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = v[i][k];
#pragma unroll
                    for (int q = 0; q < 10; ++q) g[q] = v[9 + q][k];
                    nm[k] = node_moments(f, g, unit, a.rho0);
                }
            }
            if (inside) {
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    wnd[2][0][k] = nm[k].ux;
                    wnd[2][1][k] = nm[k].uy;
                    wnd[2][2][k] = nm[k].bx;
                    wnd[2][3][k] = nm[k].by;
                }
                if (m >= y0 && m < y1 && out_lane) {
                    C ps[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) ps[q] = C(0);
#pragma unroll
                    for (int k = 0; k < V; ++k) {
                        if (xl + k < a.nx) {
                            const NodeMom<C>& n = nm[k];
                            add_point_sums(n, ps);
                            mjz = max(mjz, MB::of(node_current(n, a.omega_m, a.neq_scale)));
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) ls[q].add(ps[q]);
                }
            }
        }
        // gradient stencil on the row before m (window slot 1)
        const int o = up ? m + 1 : m - 1;
        if (i >= 2) {  // warp-uniform; y0 <= o < y1
            // x - 1 and x + 1 neighbours of the lane's first and last node
            C lft[3][4], rgt[3][4];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    lft[r][q] = __shfl_up_sync(kFull, wnd[r][q][V - 1], 1);
                    rgt[r][q] = __shfl_down_sync(kFull, wnd[r][q][0], 1);
                }
            auto at = [&](int r, int q, int j) -> C {  // field q of row slot r at node j (-1 .. V)
                return j < 0 ? lft[r][q] : (j >= V ? rgt[r][q] : wnd[r][q][j]);
            };
            bool rowok = out_lane;
            if (a.wall_y) rowok = rowok && o >= 1 && o <= a.ny - 2;
            C d2 = C(0);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int x = xl + k;
                bool ok = rowok && x < a.nx;
                if (a.wall_x) ok = ok && x >= 1 && x <= a.nx - 2;
                // isotropic gradient: d_a phi = 3 sum_i w_i phi(x + c_i) c_ia
                // (walking upwards slot 2 is the row below: d_y changes
                // sign, which is exact)
                const C dxbx = C(1.0 / 3.0) * (at(1, 2, k + 1) - at(1, 2, k - 1)) +
                               C(1.0 / 12.0) * ((at(2, 2, k + 1) - at(2, 2, k - 1)) +
                                                (at(0, 2, k + 1) - at(0, 2, k - 1)));
                const C dyby = sgn * (C(1.0 / 3.0) * (at(2, 3, k) - at(0, 3, k)) +
                                      C(1.0 / 12.0) * ((at(2, 3, k + 1) - at(0, 3, k + 1)) +
                                                       (at(2, 3, k - 1) - at(0, 3, k - 1))));
                const C dxuy = C(1.0 / 3.0) * (at(1, 1, k + 1) - at(1, 1, k - 1)) +
                               C(1.0 / 12.0) * ((at(2, 1, k + 1) - at(2, 1, k - 1)) +
                                                (at(0, 1, k + 1) - at(0, 1, k - 1)));
                const C dyux = sgn * (C(1.0 / 3.0) * (at(2, 0, k) - at(0, 0, k)) +
                                      C(1.0 / 12.0) * ((at(2, 0, k + 1) - at(0, 0, k + 1)) +
                                                       (at(2, 0, k - 1) - at(0, 0, k - 1))));
                if (ok) {
                    const C div = dxbx + dyby;
                    const C vort = dxuy - dyux;
                    d2 += div * div;
                    ++cnt;
                    mdiv = max(mdiv, MB::of(div));
                    mvort = max(mvort, MB::of(vort));
                }
            }
            ls[8].add(d2);
        }
    }
}

// The tile kernel: a persistent grid whose warps walk tiles t, t + warps, ...
// Launch bounds: FP32 and FP16S keep two blocks per SM (at most 128
// registers, twice the rows in flight), FP16S with four nodes per lane
// (8-byte loads; its register cap spills a little: 0.23 against 0.29 ms per
// totals call at 4096^2 with one block per SM), FP32 with two (at four:
// 0.29 against 0.26 ms).  FP64 is bound by its arithmetic.
template <int PREC, int V, int MODE, bool WALLY, bool GEN>
__global__ void __launch_bounds__(kDWarps * 32, PREC == 0 ? 1 : 2) diag_kernel(const DiagArgs<typename Prec<PREC>::C> a,
                                                            double* __restrict__ partials) {
    using C = typename Prec<PREC>::C;
    __shared__ double red[kDWarps][kDiagSlots];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kDWarps + warp, nw = gridDim.x * kDWarps;
    DiagAcc<C> acc;
    for (int t = gw; t < a.ntiles; t += nw) diag_tile<PREC, V, MODE, WALLY, GEN>(a, t, lane, acc);
    double w[kDiagSlots];
    acc.warp_slots(w);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < kDiagSlots; ++q) red[warp][q] = w[q];
    __syncthreads();
    if (threadIdx.x < kDiagSlots) {
        const int q = threadIdx.x;
        double v = red[0][q];
        for (int w = 1; w < kDWarps; ++w)
            v = q < 10 ? v + red[w][q] : __longlong_as_double((long long)max_bits(dbits(v), dbits(red[w][q])));
        partials[(long long)blockIdx.x * kDiagSlots + q] = v;
    }
}

// Fixed-order final reduction of the per-block partials (one block); slot 0
// becomes the mass rho0 * nodes + sum (rho - rho0).
__global__ void __launch_bounds__(256) diag_final(const double* __restrict__ partials, int nblocks,
                                                  double mass_base, double* __restrict__ totals) {
    __shared__ double red[8][kDiagSlots];
    double acc[10];
    unsigned long long mx[3] = {0, 0, 0};
#pragma unroll
    for (int s = 0; s < 10; ++s) acc[s] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
        for (int s = 0; s < 10; ++s) acc[s] += partials[(long long)b * kDiagSlots + s];
#pragma unroll
        for (int s = 0; s < 3; ++s) mx[s] = max_bits(mx[s], dbits(partials[(long long)b * kDiagSlots + 10 + s]));
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
            v = s < 10 ? v + red[w][s] : __longlong_as_double((long long)max_bits(dbits(v), dbits(red[w][s])));
        totals[s] = s == 0 ? mass_base + v : v;
    }
}

// ---- ensembles ---------------------------------------------------------------
// The diagnostics of every lattice of an ensemble (FP32 storage, periodic,
// two nodes per lane) in one launch: the warps walk a list of (lattice,
// tile) pairs, each tile's 13 slot values go to a partial of its own, and
// the final kernel adds each lattice's tile partials in tile order (fixed:
// bitwise reproducible).
__global__ void __launch_bounds__(kDWarps * 32, 2) diag_batch_kernel(const DiagArgs<float>* __restrict__ lats,
                                                                      const int2* __restrict__ tiles, int ntiles,
                                                                      double* __restrict__ tile_partials) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gw = blockIdx.x * kDWarps + warp, nw = gridDim.x * kDWarps;
    for (int k = gw; k < ntiles; k += nw) {
        const int2 tl = tiles[k];
        const DiagArgs<float> a = lats[tl.x];
        DiagAcc<float> acc;
        if (a.mode == 0)  // warp-uniform: one lattice per tile
            diag_tile<1, 2, 0, false, false>(a, tl.y, lane, acc);
        else
            diag_tile<1, 2, 1, false, false>(a, tl.y, lane, acc);
        double w[kDiagSlots];
        acc.warp_slots(w);
        if (lane == 0)
#pragma unroll
            for (int q = 0; q < kDiagSlots; ++q) tile_partials[(long long)k * kDiagSlots + q] = w[q];
    }
}

// One block of kFinalThreads per lattice: thread j adds the partials of the
// lattice's tiles first[l] + j, + j + kFinalThreads, ... (in that order),
// then thread q adds slot q of the threads' sums in thread order (a fixed
// order: bitwise reproducible); slot 0 plus mass_base[l] is the mass.
constexpr int kFinalThreads = 256;
__global__ void __launch_bounds__(kFinalThreads) diag_batch_final(const double* __restrict__ tile_partials,
                                                                  const int* __restrict__ first,
                                                                  const double* __restrict__ mass_base,
                                                                  double* __restrict__ totals) {
    __shared__ double red[kFinalThreads][kDiagSlots];
    const int l = blockIdx.x, j = threadIdx.x;
    const int t0 = first[l], t1 = first[l + 1];
    double acc[kDiagSlots];
#pragma unroll
    for (int q = 0; q < kDiagSlots; ++q) acc[q] = 0.0;
    for (int k = t0 + j; k < t1; k += kFinalThreads) {
        const double* p = tile_partials + (long long)k * kDiagSlots;
#pragma unroll
        for (int q = 0; q < kDiagSlots; ++q)
            acc[q] = q < 10 ? acc[q] + p[q] : __longlong_as_double((long long)max_bits(dbits(acc[q]), dbits(p[q])));
    }
#pragma unroll
    for (int q = 0; q < kDiagSlots; ++q) red[j][q] = acc[q];
    __syncthreads();
    if (j < kDiagSlots) {
        const int q = j;
        double v = red[0][q];
        for (int w = 1; w < kFinalThreads; ++w)
            v = q < 10 ? v + red[w][q] : __longlong_as_double((long long)max_bits(dbits(v), dbits(red[w][q])));
        totals[(long long)l * kDiagSlots + q] = q == 0 ? mass_base[l] + v : v;
    }
}

int diag_blocks(const Layout& L) {
    (void)L;
    return kDiagMaxBlocks;
}

template <int PREC>
static cudaError_t launch_diag_t(const DiagLaunch& d, double* partials, int capacity, int* nblocks,
                                 cudaStream_t st) {
    using C = typename Prec<PREC>::C;
    constexpr int VF = PREC == 2 ? 4 : 2;  // nodes per lane of the vector path
    const bool gen = d.wall_x != 0;
    // vector loads need every row of every plane to start on a vector boundary
    const long long vb = (long long)VF * d.L.esize;
    const void* src = d.mode == 0 ? d.prev : d.cur;
    const bool aligned = (reinterpret_cast<uintptr_t>(src) % vb == 0) && (d.L.pitch * d.L.esize) % vb == 0 &&
                         (d.L.plane * d.L.esize) % vb == 0;
    const int V = (!gen && aligned && d.L.nx % VF == 0) ? VF : 1;
    DiagArgs<C> a;
    a.src = src;
    a.nx = d.L.nx;
    a.ny = d.L.ny;
    a.pitch = d.L.pitch;
    a.plane = d.L.plane;
    a.omega_m = C(d.omega_m);
    a.rho0 = C(d.rho0);
    a.neq_scale = C(d.neq_scale);
    a.wall_x = d.wall_x;
    a.wall_y = d.wall_y;
    a.halo_y = d.halo_y;
    if (d.halo_y && d.mode != 1) return cudaErrorInvalidValue;
    const long long strips = (d.L.nx + 30LL * V - 1) / (30LL * V);
    if (strips > INT_MAX) return cudaErrorInvalidValue;
    a.strips = (int)strips;
    auto go = [&](auto kernel) -> cudaError_t {
        int per_sm = 0, sms = 0, dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kDWarps * 32, 0);
        if (e != cudaSuccess) return e;
        const int maxb = std::max(1, std::min({std::max(1, per_sm) * sms, capacity, kDiagMaxBlocks}));
        // tile height: at most one tile per resident warp (tall tiles keep
        // the halo rows few)
        const long long warps = (long long)maxb * kDWarps;
        const long long segs_want = std::max(1LL, warps / strips);
        const long long rows = ((long long)d.L.ny + segs_want - 1) / segs_want;
        const long long segs = ((long long)d.L.ny + rows - 1) / rows;
        if (strips * segs > INT_MAX) return cudaErrorInvalidValue;
        a.rows = (int)rows;
        a.ntiles = (int)(strips * segs);
        *nblocks = (int)std::max(1LL, std::min<long long>(maxb, (a.ntiles + kDWarps - 1) / kDWarps));
        kernel<<<*nblocks, kDWarps * 32, 0, st>>>(a, partials);
        return cudaGetLastError();
    };
    if (gen) return d.mode == 0 ? go(diag_kernel<PREC, 1, 0, false, true>) : go(diag_kernel<PREC, 1, 1, false, true>);
    if (V == 1) {
        if (d.mode == 1) return go(diag_kernel<PREC, 1, 1, false, false>);
        return d.wall_y ? go(diag_kernel<PREC, 1, 0, true, false>) : go(diag_kernel<PREC, 1, 0, false, false>);
    }
    if (d.mode == 1) return go(diag_kernel<PREC, VF, 1, false, false>);
    return d.wall_y ? go(diag_kernel<PREC, VF, 0, true, false>) : go(diag_kernel<PREC, VF, 0, false, false>);
}

cudaError_t launch_diag(const DiagLaunch& d, double* partials, int capacity, double* totals, cudaStream_t st) {
    if (capacity < 1) return cudaErrorInvalidValue;
    cudaError_t e;
    int nblocks = 0;
    switch (d.prec) {
    case 0: e = launch_diag_t<0>(d, partials, capacity, &nblocks, st); break;
    case 1: e = launch_diag_t<1>(d, partials, capacity, &nblocks, st); break;
    case 2: e = launch_diag_t<2>(d, partials, capacity, &nblocks, st); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    return launch_diag_final(partials, nblocks, d.rho0 * (double)d.L.nx * (double)d.L.ny, totals, st);
}

cudaError_t launch_diag_final(const double* partials, int nblocks, double mass_base, double* totals,
                              cudaStream_t st) {
    if (nblocks < 1) return cudaErrorInvalidValue;
    diag_final<<<1, 256, 0, st>>>(partials, nblocks, mass_base, totals);
    return cudaGetLastError();
}

constexpr int kEnsembleRows = 16;  // output rows per tile of an ensemble lattice

cudaError_t diag_ensemble_create(DiagEnsemble& e, const Layout* layouts, const double* rho0, int count) {
    diag_ensemble_destroy(e);
    std::vector<int2> tiles;
    std::vector<int> first(count + 1);
    std::vector<double> mass(count);
    for (int i = 0; i < count; ++i) {
        const Layout& L = layouts[i];
        const long long strips = (L.nx + 59) / 60, segs = (L.ny + kEnsembleRows - 1) / kEnsembleRows;
        if ((long long)tiles.size() + strips * segs > INT_MAX / kDiagSlots) return cudaErrorInvalidValue;
        first[i] = (int)tiles.size();
        for (int t = 0; t < (int)(strips * segs); ++t) tiles.push_back(make_int2(i, t));
        mass[i] = rho0[i] * (double)L.nx * (double)L.ny;
    }
    first[count] = (int)tiles.size();
    e.count = count;
    e.ntiles = (int)tiles.size();
    cudaError_t err = cudaMalloc(&e.d_args, sizeof(DiagArgs<float>) * count);
    if (err == cudaSuccess) err = cudaMallocHost(&e.h_args, sizeof(DiagArgs<float>) * count);
    if (err == cudaSuccess) err = cudaMalloc(&e.d_tiles, sizeof(int2) * tiles.size());
    if (err == cudaSuccess) err = cudaMalloc(&e.d_first, sizeof(int) * (count + 1));
    if (err == cudaSuccess) err = cudaMalloc(&e.d_mass, sizeof(double) * count);
    if (err == cudaSuccess) err = cudaMalloc(&e.d_partials, sizeof(double) * kDiagSlots * tiles.size());
    if (err == cudaSuccess)
        err = cudaMemcpy(e.d_tiles, tiles.data(), sizeof(int2) * tiles.size(), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e.d_first, first.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemcpy(e.d_mass, mass.data(), sizeof(double) * count, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) diag_ensemble_destroy(e);
    return err;
}

void diag_ensemble_destroy(DiagEnsemble& e) {
    if (e.d_args) cudaFree(e.d_args);
    if (e.h_args) cudaFreeHost(e.h_args);
    if (e.d_tiles) cudaFree(e.d_tiles);
    if (e.d_first) cudaFree(e.d_first);
    if (e.d_mass) cudaFree(e.d_mass);
    if (e.d_partials) cudaFree(e.d_partials);
    e = DiagEnsemble();
}

cudaError_t diag_ensemble_launch(DiagEnsemble& e, const Layout* layouts, const DiagLatticeState* states,
                                 double* totals, cudaStream_t st) {
    if (e.count < 1 || !e.d_args) return cudaErrorInvalidValue;
    DiagArgs<float>* h = static_cast<DiagArgs<float>*>(e.h_args);
    for (int i = 0; i < e.count; ++i) {
        const Layout& L = layouts[i];
        const DiagLatticeState& d = states[i];
        const void* src = d.mode == 0 ? d.prev : d.cur;
        // the two-node vector loads need every row of every plane on an 8-byte boundary
        if (L.nx % 2 || reinterpret_cast<uintptr_t>(src) % 8 || (L.pitch * L.esize) % 8 || (L.plane * L.esize) % 8)
            return cudaErrorNotSupported;
        DiagArgs<float> a;
        a.src = src;
        a.nx = L.nx;
        a.ny = L.ny;
        a.pitch = L.pitch;
        a.plane = L.plane;
        a.omega_m = (float)d.omega_m;
        a.rho0 = (float)d.rho0;
        a.neq_scale = (float)d.neq_scale;
        a.wall_x = a.wall_y = 0;
        a.halo_y = 0;
        a.strips = (L.nx + 59) / 60;
        a.rows = kEnsembleRows;
        a.ntiles = a.strips * ((L.ny + kEnsembleRows - 1) / kEnsembleRows);
        a.mode = d.mode;
        h[i] = a;
    }
    cudaError_t err = cudaMemcpyAsync(e.d_args, e.h_args, sizeof(DiagArgs<float>) * e.count, cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, diag_batch_kernel, kDWarps * 32, 0);
    if (err != cudaSuccess) return err;
    const int blocks = std::max(1, std::min(std::max(1, per_sm) * device_sms(), (e.ntiles + kDWarps - 1) / kDWarps));
    diag_batch_kernel<<<blocks, kDWarps * 32, 0, st>>>(static_cast<const DiagArgs<float>*>(e.d_args),
                                                        static_cast<const int2*>(e.d_tiles), e.ntiles, e.d_partials);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return launch_diag_batch_final(e.d_partials, e.d_first, e.d_mass, e.count, totals, st);
}

cudaError_t launch_diag_batch_final(const double* tile_partials, const int* first, const double* mass_base,
                                    int count, double* totals, cudaStream_t st) {
    if (count < 1) return cudaErrorInvalidValue;
    diag_batch_final<<<count, kFinalThreads, 0, st>>>(tile_partials, first, mass_base, totals);
    return cudaGetLastError();
}

}  // namespace mhd
