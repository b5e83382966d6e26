// diag_device.cuh -- per-node pieces of the global diagnostics, shared by
// the diagnostics pass (diag.cu) and the step that reduces the point totals
// on a sample step (step_totals.cu): the node's moments and current density
// (task 1 of the "Algorithm of computation", Eq. current), FP32 sums with
// exact compensation, and warp reductions in FP64.
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"
#include "step_row.cuh"

namespace mhd {

// ---- accumulation helpers -------------------------------------------------
template <typename C> struct LaneSum {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double take() {
        const double v = s;
        s = 0.0;
        return v;
    }
};
template <> struct LaneSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x;
        const float bv = t - s;
        const float e = (s - (t - bv)) + (x - bv);
        s = t;
        c += e;
    }
    __device__ __forceinline__ double take() {
        const double v = (double)s + (double)c;
        s = c = 0.f;
        return v;
    }
};

template <typename C> struct AbsBits;
template <> struct AbsBits<double> {
    using T = unsigned long long;
    __device__ __forceinline__ static T of(double v) {
        return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
    }
    __device__ __forceinline__ static double value(T b) { return __longlong_as_double((long long)b); }
};
template <> struct AbsBits<float> {
    using T = unsigned int;
    __device__ __forceinline__ static T of(float v) { return __float_as_uint(v) & 0x7fffffffu; }
    __device__ __forceinline__ static double value(T b) { return (double)__uint_as_float(b); }
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
__device__ __forceinline__ unsigned long long dbits(double v) {
    return (unsigned long long)__double_as_longlong(fabs(v));
}
__device__ __forceinline__ unsigned long long max_bits(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// ---- one node's moments -----------------------------------------------------
template <typename C> struct NodeMom {
    C drho, mx, my, bx, by, ux, uy;
    C dg;  // (g_3y - g_1y) - (g_4x - g_2x): the e-weighted antisymmetric part entering j_z
};

// Every product of the point quantities is rounded on its own (never
// contracted into an FMA): the step that reduces the point totals forms
// them beside its collision of the same values, and products shared with
// the collision would change how the compiler fuses the collision's own
// multiply-adds (its populations must stay those of the plain step).
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// From populations in `unit`s of the deviation (FP16S storage units: 2^-12).
template <typename C>
__device__ __forceinline__ NodeMom<C> node_moments(const C (&f)[9], const C (&g)[10], C unit, C rho0) {
    Moments<C> m;
    moment_sums(f, g, m);
    NodeMom<C> n;
    n.drho = rmul(m.drho, unit);
    n.mx = rmul(m.mx, unit);
    n.my = rmul(m.my, unit);
    n.bx = rmul(m.bx, unit);
    n.by = rmul(m.by, unit);
    const C inv = C(1) / (rho0 + n.drho);
    n.ux = rmul(n.mx, inv);
    n.uy = rmul(n.my, inv);
    n.dg = rmul((g[7] - g[3]) - (g[8] - g[4]), unit);
    return n;
}

// Eq. current with g_eq of the node substituted: for D2Q5,
// sum_j (e_jx g_neq_jy - e_jy g_neq_jx) = dg - 2 (u_x b_y - u_y b_x).
template <typename C>
__device__ __forceinline__ C node_current(const NodeMom<C>& n, C omega_m, C neq_scale) {
    const C e = rmul(n.ux, n.by) - rmul(n.uy, n.bx);
    return rmul(rmul(rmul(-C(3), omega_m), neq_scale), n.dg - rmul(C(2), e));
}

// The point sums of one node into ps (slots 0..7 of the partials):
// rho - rho0, m_x, m_y, |u|^2/2, |b|^2/2, u.b, b_x, b_y.
template <typename C>
__device__ __forceinline__ void add_point_sums(const NodeMom<C>& n, C (&ps)[8]) {
    ps[0] += n.drho;
    ps[1] += n.mx;
    ps[2] += n.my;
    ps[3] += rmul(C(0.5), rmul(n.ux, n.ux) + rmul(n.uy, n.uy));
    ps[4] += rmul(C(0.5), rmul(n.bx, n.bx) + rmul(n.by, n.by));
    ps[5] += rmul(n.ux, n.bx) + rmul(n.uy, n.by);
    ps[6] += n.bx;
    ps[7] += n.by;
}

}  // namespace mhd
