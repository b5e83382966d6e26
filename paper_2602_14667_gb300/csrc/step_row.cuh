// step_row.cuh -- the per-row body of the fused pull-scheme step, shared by
// the single-lattice kernel and the batched persistent kernel.
//
// One warp updates 32*V consecutive x nodes of row y: every plane is read
// with aligned V-wide vector loads, all issued before the first shuffle;
// the +-1 x shift of the moving populations is then done with warp shuffles
// (lane l takes the neighbour lane's edge element) and only the lanes at a
// warp or lattice edge issue one extra scalar load.  Pull streaming with half-way bounce-back on y walls; the x
// axis is periodic.  Stores are aligned V-wide vectors.
#pragma once

#include "lbm_device.cuh"

namespace mhd {

constexpr unsigned kFull = 0xffffffffu;

template <typename C> struct StepArgs {
    const void* src;
    void* dst;
    int nx, ny;
    long long pitch, plane;
    NodeParams<C> np;
    int wall_x, wall_y;
};

// Pre-collision populations of the V nodes x0 .. x0+V-1 (x0 = (32 xblock +
// lane) V) of row y, pulled from the post-collision buffer src: v[p][k] in
// the compute type (FP16S values stay in storage units, 2^12 times the
// deviation).  Returns whether the lane's nodes lie inside the lattice
// (false: nothing was loaded and v is unset).
// Requires nx % V == 0, all 32 lanes of the warp present, y < ny.  WALLY:
// half-way bounce-back walls below row 0 and above row ny-1 (compile-time,
// so that the periodic kernel has no branch between its 19 plane loads).
// Off: the type of element offsets into the state; int when the 19 planes
// hold fewer than 2^31 elements (fewer address instructions per plane),
// long long otherwise.
template <int PREC, int V, bool WALLY, typename Off = long long>
__device__ __forceinline__ bool gather_row(const typename Prec<PREC>::S* __restrict__ src, int nx, int ny,
                                           long long pitch, long long plane, int xblock, int y, int lane,
                                           typename Prec<PREC>::C (&v)[kPlanes][V]) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    const int x0 = (xblock * 32 + lane) * V;
    const bool active = x0 < nx;

    int ym = y - 1, yp = y + 1;
    bool bm = false, bp = false;
    if (WALLY) {
        bm = ym < 0;
        bp = yp >= ny;
    } else {
        if (ym < 0) ym += ny;
        if (yp >= ny) yp -= ny;
    }
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;          // source column for c_x = +1 at x0
    const int xr = (x0 + V >= nx) ? x0 + V - nx : x0 + V;  // source column for c_x = -1 at x0+V-1
    const bool right_by_shfl = (lane < 31) && (x0 + V < nx);
    const Off pl = (Off)plane, pt = (Off)pitch;
    const Off o_m = (Off)ym * pt, o_0 = (Off)y * pt, o_p = (Off)yp * pt;

    // Phase 1: issue every load of the 19 planes (aligned vectors, plus the
    // edge element for the lanes at a warp / lattice edge) before any
    // shuffle, so that all of them are in flight together.
    S r[kPlanes][V];
    S edge[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p), cy = pcy(p);
        const bool bounce = WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));  // warp-uniform
        const S* row = src + (bounce ? (Off)popp(p) * pl + o_0
                                     : (Off)p * pl + (cy > 0 ? o_m : (cy < 0 ? o_p : o_0)));
#pragma unroll
        for (int k = 0; k < V; ++k) r[p][k] = S(0);
        edge[p] = S(0);
        if (active) VecIO<S, V>::load(row + x0, r[p]);
        if (cx > 0 && !bounce && lane == 0 && active) edge[p] = row[xl];
        if (cx < 0 && !bounce && !right_by_shfl && active) edge[p] = row[xr];
    }
    // Phase 2: decode and apply the +-1 x shift of the moving populations
    // (FP16S values stay in storage units).
    using Codec = StepCodec<S, V>;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p), cy = pcy(p);
        const bool bounce = WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));
        C c[V];
        Codec::to_compute(r[p], c);
        if (cx == 0 || bounce) {
#pragma unroll
            for (int k = 0; k < V; ++k) v[p][k] = c[k];
        } else if (cx > 0) {  // source x - 1
            C left = __shfl_up_sync(kFull, c[V - 1], 1);
            if (lane == 0) left = Codec::template one<C>(edge[p]);
            v[p][0] = left;
#pragma unroll
            for (int k = 1; k < V; ++k) v[p][k] = c[k - 1];
        } else {  // source x + 1
            C right = __shfl_down_sync(kFull, c[0], 1);
            if (!right_by_shfl) right = Codec::template one<C>(edge[p]);
#pragma unroll
            for (int k = 0; k < V - 1; ++k) v[p][k] = c[k + 1];
            v[p][V - 1] = right;
        }
    }
    return active;
}

// One warp updates 32*V consecutive x nodes of row y: the pull gather above,
// the collision, aligned V-wide vector stores.  Same requirements.
template <int PREC, int V, bool WALLY, typename Off = long long>
__device__ __forceinline__ void step_row(const typename Prec<PREC>::S* __restrict__ src,
                                         typename Prec<PREC>::S* __restrict__ dst, int nx, int ny,
                                         long long pitch, long long plane,
                                         const NodeParams<typename Prec<PREC>::C>& np, int xblock,
                                         int y, int lane) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    C v[kPlanes][V];
    if (!gather_row<PREC, V, WALLY, Off>(src, nx, ny, pitch, plane, xblock, y, lane, v)) return;
    // FP16S collides in storage units, node pairs on FP32x2
    constexpr bool kScaled = PREC == 2;
    constexpr int kMode = PREC == 2 ? kPairs : kNative;
    collide_nodes<C, V, kScaled, kMode>(v, np);
    const int x0 = (xblock * 32 + lane) * V;
    const Off o_0 = (Off)y * (Off)pitch, pl = (Off)plane;
    using Codec = StepCodec<S, V>;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        S r[V];
        Codec::to_storage(v[p], r);
        VecIO<S, V>::store(dst + ((Off)p * pl + o_0 + x0), r);
    }
}

// Pre-collision populations of the V nodes x0 .. x0+V-1 of row y pulled
// from the post-collision buffer src, where the lanes of the warp hold
// consecutive vectors modulo nx (x0 wrapped into [0, nx), nx % V == 0):
// gather_row with the warp's edge elements taken at the wrapped neighbours.
// FP16S values stay in storage units.  Off as in gather_row.
template <int PREC, int V, bool WALLY, typename Off = long long>
__device__ __forceinline__ void gather_row_wrapped(const typename Prec<PREC>::S* __restrict__ src, int nx,
                                                   int ny, long long pitch, long long plane, int x0, int y,
                                                   int lane, typename Prec<PREC>::C (&v)[kPlanes][V]) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    int ym = y - 1, yp = y + 1;
    bool bm = false, bp = false;
    if (WALLY) {
        bm = ym < 0;
        bp = yp >= ny;
    } else {
        if (ym < 0) ym += ny;
        if (yp >= ny) yp -= ny;
    }
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;
    const int xr = x0 + V >= nx ? x0 + V - nx : x0 + V;
    const Off pl = (Off)plane, pt = (Off)pitch;
    const Off o_m = (Off)ym * pt, o_0 = (Off)y * pt, o_p = (Off)yp * pt;
    S r[kPlanes][V];
    S edge[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p), cy = pcy(p);
        const bool bounce = WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));  // warp-uniform
        const S* row = src + (bounce ? (Off)popp(p) * pl + o_0 : (Off)p * pl + (cy > 0 ? o_m : (cy < 0 ? o_p : o_0)));
        VecIO<S, V>::load(row + x0, r[p]);
        edge[p] = S(0);
        if (cx > 0 && !bounce && lane == 0) edge[p] = row[xl];
        if (cx < 0 && !bounce && lane == 31) edge[p] = row[xr];
    }
    using Codec = StepCodec<S, V>;
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p), cy = pcy(p);
        const bool bounce = WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));
        C c[V];
        Codec::to_compute(r[p], c);
        if (cx == 0 || bounce) {
#pragma unroll
            for (int k = 0; k < V; ++k) v[p][k] = c[k];
        } else if (cx > 0) {  // source x - 1
            C left = __shfl_up_sync(kFull, c[V - 1], 1);
            if (lane == 0) left = Codec::template one<C>(edge[p]);
            v[p][0] = left;
#pragma unroll
            for (int k = 1; k < V; ++k) v[p][k] = c[k - 1];
        } else {  // source x + 1
            C right = __shfl_down_sync(kFull, c[0], 1);
            if (lane == 31) right = Codec::template one<C>(edge[p]);
#pragma unroll
            for (int k = 0; k < V - 1; ++k) v[p][k] = c[k + 1];
            v[p][V - 1] = right;
        }
    }
}

// Pre-collision populations of node (x, y) gathered from a post-collision
// buffer (pull streaming with half-way bounce-back on wall axes).
template <typename S, typename C>
__device__ __forceinline__ void gather_node(const S* __restrict__ src, int x, int y, int nx, int ny,
                                            long long pitch, long long plane, int wall_x,
                                            int wall_y, C (&f)[9], C (&g)[10]) {
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        int sx = x - pcx(p), sy = y - pcy(p);
        const bool out = (wall_x && (sx < 0 || sx >= nx)) || (wall_y && (sy < 0 || sy >= ny));
        long long off;
        if (out) {
            off = (long long)popp(p) * plane + (long long)y * pitch + x;
        } else {
            sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            off = (long long)p * plane + (long long)sy * pitch + sx;
        }
        const C val = decode(src[off]);
        if (p < 9) f[p] = val; else g[p - 9] = val;
    }
}

}  // namespace mhd
