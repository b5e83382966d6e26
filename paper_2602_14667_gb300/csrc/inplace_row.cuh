// inplace_row.cuh -- the fused step on ONE state buffer (in-place streaming).
//
// The two-buffer pull scheme reads f*(t) from one buffer and writes f*(t+1)
// to the other.  Here a pair of kernels updates a single buffer in place
// (the "AA" access pattern), so a lattice needs half the memory for the
// same bytes moved per step:
//
//   phase A (buffer holds the canonical state f*_p(x) at plane p):
//     gather f_p(x) exactly as the pull step does (plane p at x - c_p, or
//     plane opp(p) at x across a half-way bounce-back wall), collide, and
//     write every post-collision population back into the cell its
//     opposite's slot was read from: slot p receives f*_opp(p)(x).  After
//     it, plane opp(q) at x + c_q holds f*_q(x) = f_q(x + c_q, t+1), the
//     pre-collision state of the next step, stored in the opposite plane.
//   phase B (buffer holds that streamed state): every node reads its own
//     pre-collision populations locally (population q from plane opp(q)),
//     collides, and writes f*_q(x) to plane q: the canonical layout again.
//
// Each node writes exactly the cells it read, so no two threads touch the
// same cell and the update needs no second buffer.  Both phases evaluate
// the same collision on the same inputs as the two-buffer step, so the
// state after an even number of steps is bitwise that of the pull scheme.
// In phase A the warp-edge lanes own one cell of the neighbouring warp's
// aligned vector: they write it with a scalar store and the neighbour's
// vector store leaves it out (the neighbour's vector load of that cell is
// discarded).  Loads are plain (coherent) loads: the buffer is written by
// the same kernel.
#pragma once

#include "step_row.cuh"

namespace mhd {

template <typename S, int V> struct VecRW {
    using Raw = typename RawT<sizeof(S) * V>::T;
    __device__ __forceinline__ static void load(const S* p, S (&out)[V]) {
        const Raw r = *reinterpret_cast<const Raw*>(p);
        memcpy(out, &r, sizeof(Raw));
    }
    // Aligned store of the V elements, except the first and/or the last.
    __device__ __forceinline__ static void store(S* p, const S (&in)[V], bool skip_first,
                                                 bool skip_last) {
        if (!skip_first && !skip_last) {
            Raw r;
            memcpy(&r, in, sizeof(Raw));
            *reinterpret_cast<Raw*>(p) = r;
            return;
        }
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (!((k == 0 && skip_first) || (k == V - 1 && skip_last))) p[k] = in[k];
    }
};

// One value into the step's storage units (FP16S: the stored half of a
// value already in 2^12 units; otherwise the storage type itself).
__device__ __forceinline__ double step_store_one(double c, double) { return c; }
__device__ __forceinline__ float step_store_one(float c, float) { return c; }
__device__ __forceinline__ __half step_store_one(float c, __half) { return __float2half_rn(c); }

// Phase A for one warp: 32*V consecutive nodes of row y (requires nx % V
// == 0, all 32 lanes present, y < ny; periodic in x).  Off: the element
// offset type (int when the state has fewer than 2^31 elements).
template <int PREC, int V, bool WALLY, typename Off = long long>
__device__ __forceinline__ void aa_row_a(typename Prec<PREC>::S* buf, int nx, int ny,
                                         long long pitch, long long plane,
                                         const NodeParams<typename Prec<PREC>::C>& np, int xblock,
                                         int y, int lane) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    constexpr bool kScaled = PREC == 2;
    // FP16S: node pairs on FP32x2, as in the two-buffer step (same bits)
    constexpr int kMode = PREC == 2 ? kPairs : kNative;
    using Codec = StepCodec<S, V>;
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
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const int xr = (x0 + V >= nx) ? x0 + V - nx : x0 + V;
    const bool right_by_shfl = (lane < 31) && (x0 + V < nx);
    const Off pl = (Off)plane, pt = (Off)pitch;
    const Off o_m = (Off)ym * pt, o_0 = (Off)y * pt, o_p = (Off)yp * pt;

    auto slot_off = [&](int p) -> Off {  // offset of the cells slot p reads and writes
        const int cy = pcy(p);
        const bool bounce = WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));
        return bounce ? (Off)popp(p) * pl + o_0 : (Off)p * pl + (cy > 0 ? o_m : (cy < 0 ? o_p : o_0));
    };
    auto slot_row = [&](int p) -> S* { return buf + slot_off(p); };
    auto slot_bounce = [&](int p) -> bool {
        const int cy = pcy(p);
        return WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));
    };

    // gather: all loads first, then the shuffles (as in step_row)
    S r[kPlanes][V];
    S edge[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        const bool bounce = slot_bounce(p);
        const S* row = slot_row(p);
#pragma unroll
        for (int k = 0; k < V; ++k) r[p][k] = S(0);
        edge[p] = S(0);
        if (active) VecRW<S, V>::load(row + x0, r[p]);
        if (cx > 0 && !bounce && lane == 0 && active) edge[p] = row[xl];
        if (cx < 0 && !bounce && !right_by_shfl && active) edge[p] = row[xr];
    }
    C v[kPlanes][V];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        const bool bounce = slot_bounce(p);
        C c[V];
        Codec::to_compute(r[p], c);
        if (cx == 0 || bounce) {
#pragma unroll
            for (int k = 0; k < V; ++k) v[p][k] = c[k];
        } else if (cx > 0) {
            C left = __shfl_up_sync(kFull, c[V - 1], 1);
            if (lane == 0) left = Codec::template one<C>(edge[p]);
            v[p][0] = left;
#pragma unroll
            for (int k = 1; k < V; ++k) v[p][k] = c[k - 1];
        } else {
            C right = __shfl_down_sync(kFull, c[0], 1);
            if (!right_by_shfl) right = Codec::template one<C>(edge[p]);
#pragma unroll
            for (int k = 0; k < V - 1; ++k) v[p][k] = c[k + 1];
            v[p][V - 1] = right;
        }
    }
    // collide (inactive lanes hold zero deviations: a harmless rest state;
    // they stay in the warp for the shuffles below)
    collide_nodes<C, V, kScaled, kMode>(v, np);
    // write back: slot p's cells receive f*_opp(p) of the nodes that read them.
    // A fresh copy of the base pointer makes the compiler recompute the 19
    // slot addresses here instead of keeping them live across the collision.
    S* wbuf;
    asm volatile("mov.b64 %0, %1;" : "=l"(wbuf) : "l"(buf));
    auto wslot_row = [&](int p) -> S* { return wbuf + slot_off(p); };
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        const bool bounce = slot_bounce(p);
        S* row = wslot_row(p);
        const int q = popp(p);
        if (cx == 0 || bounce) {
            S w[V];
            Codec::to_storage(v[q], w);
            if (active) VecRW<S, V>::store(row + x0, w, false, false);
        } else if (cx > 0) {
            // slot read x - 1: node x0+k owns cell x0+k-1
            C u[V];
#pragma unroll
            for (int k = 0; k < V - 1; ++k) u[k] = v[q][k + 1];
            u[V - 1] = __shfl_down_sync(kFull, v[q][0], 1);
            S w[V];
            Codec::to_storage(u, w);
            if (active) VecRW<S, V>::store(row + x0, w, false, !right_by_shfl);
            if (active && lane == 0) row[xl] = step_store_one(v[q][0], S());
        } else {
            // slot read x + 1: node x0+k owns cell x0+k+1
            C u[V];
            u[0] = __shfl_up_sync(kFull, v[q][V - 1], 1);
#pragma unroll
            for (int k = 1; k < V; ++k) u[k] = v[q][k - 1];
            S w[V];
            Codec::to_storage(u, w);
            if (active) VecRW<S, V>::store(row + x0, w, lane == 0, false);
            if (active && !right_by_shfl) row[xr] = step_store_one(v[q][V - 1], S());
        }
    }
}

// Phase A for FP16S storage at four nodes per lane, with the populations
// held as packed halves (two nodes per 32-bit register) except while a
// node pair collides: the x shifts of the gather and of the write-back move
// packed halves with byte permutes, and each pair of nodes is decoded,
// collided on FP32x2 in storage units and re-encoded before the next pair
// is decoded.  The conversions, the pairs and the arithmetic are those of
// the two-buffer step, so the bits are the same; about half the registers
// of holding all four nodes' populations as FP32.  Same requirements as
// aa_row_a.
template <bool WALLY, typename Off = long long>
__device__ __forceinline__ void aa_row_a_h4(__half* buf, int nx, int ny, long long pitch, long long plane,
                                            const NodeParams<float>& np, int xblock, int y, int lane) {
    constexpr int V = 4;
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
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const int xr = (x0 + V >= nx) ? x0 + V - nx : x0 + V;
    const bool right_by_shfl = (lane < 31) && (x0 + V < nx);
    const Off pl = (Off)plane, pt = (Off)pitch;
    const Off o_m = (Off)ym * pt, o_0 = (Off)y * pt, o_p = (Off)yp * pt;
    auto slot_bounce = [&](int p) -> bool {
        const int cy = pcy(p);
        return WALLY && (cy > 0 ? bm : (cy < 0 ? bp : false));
    };
    auto slot_off = [&](int p) -> Off {
        return slot_bounce(p) ? (Off)popp(p) * pl + o_0
                              : (Off)p * pl + (pcy(p) > 0 ? o_m : (pcy(p) < 0 ? o_p : o_0));
    };

    // gather: halves (x0, x0+1) in lo, (x0+2, x0+3) in hi; every load first
    uint32_t lo[kPlanes], hi[kPlanes];
    unsigned short edge[kPlanes];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        const bool bounce = slot_bounce(p);
        const __half* row = buf + slot_off(p);
        lo[p] = hi[p] = 0u;
        edge[p] = 0;
        if (active) {
            const uint2 u = *reinterpret_cast<const uint2*>(row + x0);
            lo[p] = u.x;
            hi[p] = u.y;
        }
        if (cx > 0 && !bounce && lane == 0 && active) edge[p] = __half_as_ushort(row[xl]);
        if (cx < 0 && !bounce && !right_by_shfl && active) edge[p] = __half_as_ushort(row[xr]);
    }
    // x shifts: source x - 1 -> (left, h0, h1, h2); source x + 1 -> (h1, h2, h3, right)
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        if (cx == 0 || slot_bounce(p)) continue;
        if (cx > 0) {
            uint32_t L = __shfl_up_sync(kFull, hi[p], 1);  // the left lane's h3 in the high half
            if (lane == 0) L = (uint32_t)edge[p] << 16;
            const uint32_t l2 = __byte_perm(L, lo[p], 0x5432), h2 = __byte_perm(lo[p], hi[p], 0x5432);
            lo[p] = l2;
            hi[p] = h2;
        } else {
            uint32_t R = __shfl_down_sync(kFull, lo[p], 1);  // the right lane's h0 in the low half
            if (!right_by_shfl) R = (uint32_t)edge[p];
            const uint32_t l2 = __byte_perm(lo[p], hi[p], 0x5432), h2 = __byte_perm(hi[p], R, 0x5432);
            lo[p] = l2;
            hi[p] = h2;
        }
    }
    // collide pair (0, 1), then pair (2, 3); the results replace the inputs
    NodeParams<F2> p2;
    p2.omega = F2(np.omega);
    p2.omega_m = F2(np.omega_m);
    p2.rho0 = F2(np.rho0);
    p2.variant = np.variant;
    p2.collision = np.collision;
    p2.mag_collision = np.mag_collision;
    auto collide_pair = [&](uint32_t (&w)[kPlanes]) {
        F2 f[9], g[10];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            __half2 h;
            memcpy(&h, &w[i], 4);
            f[i] = F2(__half22float2(h));
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            __half2 h;
            memcpy(&h, &w[9 + q], 4);
            g[q] = F2(__half22float2(h));
        }
        collide_impl<false, F2, true>(f, g, p2, nullptr);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const __half2 h = __floats2half2_rn(f[i].v.x, f[i].v.y);
            memcpy(&w[i], &h, 4);
        }
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const __half2 h = __floats2half2_rn(g[q].v.x, g[q].v.y);
            memcpy(&w[9 + q], &h, 4);
        }
    };
    collide_pair(lo);
    collide_pair(hi);
    // write back: slot p's cells receive f*_opp(p) of the nodes that read them
    __half* wbuf;
    asm volatile("mov.b64 %0, %1;" : "=l"(wbuf) : "l"(buf));
    auto store4 = [&](__half* dst, uint32_t a, uint32_t b, bool skip_first, bool skip_last) {
        if (!skip_first && !skip_last) {
            *reinterpret_cast<uint2*>(dst) = make_uint2(a, b);
            return;
        }
        unsigned short* d = reinterpret_cast<unsigned short*>(dst);
        if (!skip_first) d[0] = (unsigned short)(a & 0xffffu);
        d[1] = (unsigned short)(a >> 16);
        d[2] = (unsigned short)(b & 0xffffu);
        if (!skip_last) d[3] = (unsigned short)(b >> 16);
    };
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = pcx(p);
        const bool bounce = slot_bounce(p);
        __half* row = wbuf + slot_off(p);
        const int q = popp(p);
        if (cx == 0 || bounce) {
            if (active) store4(row + x0, lo[q], hi[q], false, false);
        } else if (cx > 0) {
            // slot read x - 1: node x0+k owns cell x0+k-1 -> (w1, w2, w3, right lane's w0)
            const uint32_t N = __shfl_down_sync(kFull, lo[q], 1);
            const uint32_t a = __byte_perm(lo[q], hi[q], 0x5432), b = __byte_perm(hi[q], N, 0x5432);
            if (active) store4(row + x0, a, b, false, !right_by_shfl);
            if (active && lane == 0) row[xl] = __ushort_as_half((unsigned short)(lo[q] & 0xffffu));
        } else {
            // slot read x + 1: node x0+k owns cell x0+k+1 -> (left lane's w3, w0, w1, w2)
            const uint32_t P = __shfl_up_sync(kFull, hi[q], 1);
            const uint32_t a = __byte_perm(P, lo[q], 0x5432), b = __byte_perm(lo[q], hi[q], 0x5432);
            if (active) store4(row + x0, a, b, lane == 0, false);
            if (active && !right_by_shfl) row[xr] = __ushort_as_half((unsigned short)(hi[q] >> 16));
        }
    }
}

// Phase B for one thread: V consecutive nodes of row y, all accesses local.
template <int PREC, int V, typename Off = long long>
__device__ __forceinline__ void aa_row_b(typename Prec<PREC>::S* buf, int nx, long long pitch,
                                         long long plane,
                                         const NodeParams<typename Prec<PREC>::C>& np, int xblock,
                                         int y, int lane) {
    using S = typename Prec<PREC>::S;
    using C = typename Prec<PREC>::C;
    constexpr bool kScaled = PREC == 2;
    // FP16S: node pairs on FP32x2
    constexpr int kMode = PREC == 2 ? kPairs : kNative;
    using Codec = StepCodec<S, V>;
    const int x0 = (xblock * 32 + lane) * V;
    if (x0 >= nx) return;
    const Off pl = (Off)plane;
    S* base = buf + ((Off)y * (Off)pitch + x0);
    S r[kPlanes][V];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) VecRW<S, V>::load(base + (Off)p * pl, r[p]);
    C v[kPlanes][V];  // v[q]: population q, read from plane opp(q)
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) Codec::to_compute(r[p], v[popp(p)]);
    collide_nodes<C, V, kScaled, kMode>(v, np);
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        S w[V];
        Codec::to_storage(v[p], w);
        VecRW<S, V>::store(base + (Off)p * pl, w, false, false);
    }
}

}  // namespace mhd
