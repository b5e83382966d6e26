// lbm_device.cuh -- device building blocks of the fused RR-MHD step (sm_103a).
//
// Method: De Rosis, "Recursive regularised lattice Boltzmann method for
// magnetohydrodynamics", Section "Algorithm of computation", tasks 1-6.
//
// Storage: 19 structure-of-arrays planes per buffer, each ny rows of `pitch`
// elements (pitch a multiple of 128 bytes):
//   planes 0..8   fluid populations f_i (D2Q9, the paper's ordering), stored
//                 as deviations f_i - w_i rho0 (Eq. feq_4th rest weights);
//   planes 9..18  magnetic populations g_{j,a}, plane 9 + 2j + a (D2Q5,
//                 component a = x, y), stored unshifted.
// FP16S stores 2^12 times the FP32 value in IEEE half (power-of-two scale,
// exact apart from the half rounding itself).
//
// The node update below is the algorithm's tasks 1-5 with the Hermite sums
// contracted by hand: f*_i = w_i sum_n [a0^(n) + (1-omega) a1^(n)] : H_i^(n)
// / (n! cs^2n) (Eq. fistar_acoeff) over the D2Q9-supported components
// (orders 0-2, xxy, xyy, xxyy), which is the same as Eq. feq_4th plus
// (1-omega) Eq. fineq_reg.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "f32x2.cuh"

namespace mhd {

constexpr int kQ = 9;        // D2Q9
constexpr int kQM = 5;       // D2Q5
constexpr int kPlanes = 19;  // 9 f + 5 x 2 g

// D2Q9 in the paper's (Latt's) ordering; opposite of i >= 1 is ((i+3)%8)+1.
__host__ __device__ constexpr int cx_of(int i) { return i == 0 ? 0 : (i <= 3 ? -1 : (i == 4 || i == 8 ? 0 : 1)); }
__host__ __device__ constexpr int cy_of(int i) {
    return i == 0 ? 0 : (i == 1 || i == 7 || i == 8 ? 1 : (i == 2 || i == 6 ? 0 : -1));
}
__host__ __device__ constexpr int opp_f(int i) { return i == 0 ? 0 : ((i + 3) % 8) + 1; }
__host__ __device__ constexpr double w_of(int i) {
    return i == 0 ? 4.0 / 9.0 : ((i & 1) ? 1.0 / 36.0 : 1.0 / 9.0);
}
// D2Q5: e = (0,0), (-1,0), (0,-1), (1,0), (0,1); opposite of j >= 1 is ((j+1)%4)+1.
__host__ __device__ constexpr int ex_of(int j) { return j == 1 ? -1 : (j == 3 ? 1 : 0); }
__host__ __device__ constexpr int ey_of(int j) { return j == 2 ? -1 : (j == 4 ? 1 : 0); }
__host__ __device__ constexpr int opp_g(int j) { return j == 0 ? 0 : ((j + 1) % 4) + 1; }

// plane index of population p = 0..18 and its x / y velocity components
__host__ __device__ constexpr int pcx(int p) { return p < 9 ? cx_of(p) : ex_of((p - 9) >> 1); }
__host__ __device__ constexpr int pcy(int p) { return p < 9 ? cy_of(p) : ey_of((p - 9) >> 1); }
__host__ __device__ constexpr int popp(int p) {
    return p < 9 ? opp_f(p) : 9 + 2 * opp_g((p - 9) >> 1) + ((p - 9) & 1);
}

constexpr float kHalfScale = 4096.0f;
constexpr float kHalfInvScale = 1.0f / 4096.0f;

// ---- storage precision traits --------------------------------------------
template <int PREC> struct Prec;
template <> struct Prec<0> { using S = double; using C = double; };  // MHD_FP64
template <> struct Prec<1> { using S = float;  using C = float;  };  // MHD_FP32
template <> struct Prec<2> { using S = __half; using C = float;  };  // MHD_FP16S

__device__ __forceinline__ double decode(double s) { return s; }
__device__ __forceinline__ float decode(float s) { return s; }
__device__ __forceinline__ float decode(__half s) { return __half2float(s) * kHalfInvScale; }
// round-to-nearest-even into the storage type
__device__ __forceinline__ void encode(double v, double& s) { s = v; }
__device__ __forceinline__ void encode(float v, float& s) { s = v; }
__device__ __forceinline__ void encode(float v, __half& s) { s = __float2half_rn(v * kHalfScale); }

// Storage <-> compute values of V consecutive elements inside the fused
// step.  FP16S values stay in storage units there (2^12 times the value; the
// step's collision runs in those units), converted two at a time.
template <typename S, int V> struct StepCodec {
    template <typename C>
    __device__ __forceinline__ static void to_compute(const S (&r)[V], C (&c)[V]) {
#pragma unroll
        for (int k = 0; k < V; ++k) c[k] = decode(r[k]);
    }
    template <typename C>
    __device__ __forceinline__ static C one(S r) { return decode(r); }
    template <typename C>
    __device__ __forceinline__ static void to_storage(const C (&c)[V], S (&r)[V]) {
#pragma unroll
        for (int k = 0; k < V; ++k) encode(c[k], r[k]);
    }
};
template <int V> struct StepCodec<__half, V> {
    __device__ __forceinline__ static void to_compute(const __half (&r)[V], float (&c)[V]) {
        if constexpr (V % 2 == 0) {
#pragma unroll
            for (int k = 0; k < V; k += 2) {
                __half2 h;
                memcpy(&h, &r[k], sizeof(h));
                const float2 t = __half22float2(h);
                c[k] = t.x;
                c[k + 1] = t.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) c[k] = __half2float(r[k]);
        }
    }
    template <typename C>
    __device__ __forceinline__ static float one(__half r) { return __half2float(r); }
    __device__ __forceinline__ static void to_storage(const float (&c)[V], __half (&r)[V]) {
        if constexpr (V % 2 == 0) {
#pragma unroll
            for (int k = 0; k < V; k += 2) {
                const __half2 h = __floats2half2_rn(c[k], c[k + 1]);
                memcpy(&r[k], &h, sizeof(h));
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) r[k] = __float2half_rn(c[k]);
        }
    }
};

template <int BYTES> struct RawT;
template <> struct RawT<2> { using T = unsigned short; };
template <> struct RawT<4> { using T = unsigned int; };
template <> struct RawT<8> { using T = uint2; };
template <> struct RawT<16> { using T = uint4; };

// V consecutive storage elements as one aligned vector access.
template <typename S, int V> struct VecIO {
    using Raw = typename RawT<sizeof(S) * V>::T;
    __device__ __forceinline__ static void load(const S* p, S (&out)[V]) {
        Raw r = __ldg(reinterpret_cast<const Raw*>(p));
        memcpy(out, &r, sizeof(Raw));
    }
    __device__ __forceinline__ static void store(S* p, const S (&in)[V]) {
        Raw r;
        memcpy(&r, in, sizeof(Raw));
        *reinterpret_cast<Raw*>(p) = r;
    }
};

// ---- physical parameters of one lattice -----------------------------------
template <typename C> struct NodeParams {
    C omega;    // 1 / tau_f
    C omega_m;  // 1 / tau_m
    C rho0;
    int variant;    // 0: Eq. feq_4th; 1: + u (x) M terms of Eq. a0_4
    int collision;  // 0: recursive regularised; 1: BGK
    int mag_collision;  // 0: BGK (Eq. collide_g); 1: first Hermite moment of g - g_eq only
};

// Moments of one node (task 1): rho = rho0 + sum df, m = sum df c, b = sum g.
template <typename C> struct Moments {
    C drho, mx, my, rho, ux, uy, bx, by;
};

// The linear sums drho, mx, my, bx, by of the populations as given.
template <typename C>
__device__ __forceinline__ void moment_sums(const C (&f)[9], const C (&g)[10], Moments<C>& m) {
    // cx = -1: 1,2,3; cx = +1: 5,6,7; cy = +1: 1,7,8; cy = -1: 3,4,5
    C left = f[1] + f[2] + f[3], right = f[5] + f[6] + f[7];
    C up = f[1] + f[7] + f[8], down = f[3] + f[4] + f[5];
    m.drho = f[0] + f[4] + f[8] + left + right;
    m.mx = right - left;
    m.my = up - down;
    m.bx = g[0] + g[2] + g[4] + g[6] + g[8];
    m.by = g[1] + g[3] + g[5] + g[7] + g[9];
}

template <typename C>
__device__ __forceinline__ Moments<C> moments(const C (&f)[9], const C (&g)[10], C rho0) {
    Moments<C> m;
    moment_sums(f, g, m);
    m.rho = rho0 + m.drho;
    C inv = C(1) / m.rho;
    m.ux = m.mx * inv;
    m.uy = m.my * inv;
    return m;
}

// Hermite coefficients of the post-collision state (Eq. fistar_acoeff):
// A_n = a0^(n) + om1 * a1^(n) on the supported components.
template <typename C> struct Coeffs {
    C drho, mx, my, A2xx, A2xy, A2yy, A3xxy, A3xyy, A4;
};

// Evaluate w_i sum_n A_n : H_i^(n) / (n! cs^2n) - w_i rho0 for all nine i.
template <typename C>
__device__ __forceinline__ void hermite_eval(const Coeffs<C>& a, C (&out)[9]) {
    const C w0 = C(4.0 / 9.0), wa = C(1.0 / 9.0), wd = C(1.0 / 36.0);
    const C s = a.A2xx + a.A2yy;
    // rest: H_xx = H_yy = -1/3, H_xxyy = 1/9
    out[0] = w0 * (a.drho - C(1.5) * s + C(2.25) * a.A4);
    // axis x (cx = -+1): H_xx = 2/3, H_yy = -1/3, H_xyy = -cx/3, H_xxyy = -2/9
    const C ax = a.drho + C(3) * a.A2xx - C(1.5) * a.A2yy - C(4.5) * a.A4;
    out[2] = wa * (ax - C(3) * a.mx + C(4.5) * a.A3xyy);
    out[6] = wa * (ax + C(3) * a.mx - C(4.5) * a.A3xyy);
    // axis y (cy = -+1): H_yy = 2/3, H_xx = -1/3, H_xxy = -cy/3, H_xxyy = -2/9
    const C ay = a.drho - C(1.5) * a.A2xx + C(3) * a.A2yy - C(4.5) * a.A4;
    out[4] = wa * (ay - C(3) * a.my + C(4.5) * a.A3xxy);
    out[8] = wa * (ay + C(3) * a.my - C(4.5) * a.A3xxy);
    // diagonals: H_xx = H_yy = 2/3, H_xy = cx cy, H_xxy = 2cy/3, H_xyy = 2cx/3, H_xxyy = 4/9
    const C dg = a.drho + C(3) * s + C(9) * a.A4;
    const C pp = C(3) * (a.mx + a.my) + C(9) * (a.A3xxy + a.A3xyy);  // cx = cy = +1 odd part
    const C pm = C(3) * (a.mx - a.my) + C(9) * (a.A3xyy - a.A3xxy);  // cx = +1, cy = -1 odd part
    const C xy = C(9) * a.A2xy;
    out[7] = wd * (dg + xy + pp);  // (+1, +1)
    out[3] = wd * (dg + xy - pp);  // (-1, -1)
    out[5] = wd * (dg - xy + pm);  // (+1, -1)
    out[1] = wd * (dg - xy - pm);  // (-1, +1)
}

// Tasks 2-5 at one node, in place.  f holds deviations f_i - w_i rho0 of the
// pre-collision populations, g the pre-collision g_{j,a} (index 2j + a).
// With DA, da (xx, xy, yy) is added to the projected a1^(2) before the
// recursion (the learned closure; mass and momentum are untouched).
// SCALED: f and g (in and out) are 2^12 times the deviations (the FP16S
// storage units).  Every quantity linear in the populations (the moment
// sums, a1^(2) and its recursion, the Hermite coefficients, g) is then
// carried in those units and only u and the b entering the Maxwell stress
// are brought back; scaling by a power of two commutes with rounding, so the
// result is the unscaled one times 2^12, without a multiply per population.
template <bool DA, typename C, bool SCALED = false>
__device__ __forceinline__ void collide_impl(C (&f)[9], C (&g)[10], const NodeParams<C>& p,
                                             const C* da);

template <typename C>
__device__ __forceinline__ void collide(C (&f)[9], C (&g)[10], const NodeParams<C>& p) {
    collide_impl<false, C>(f, g, p, nullptr);
}

template <bool DA, typename C, bool SCALED>
__device__ __forceinline__ void collide_impl(C (&f)[9], C (&g)[10], const NodeParams<C>& p,
                                             const C* da) {
    Moments<C> m;  // sums in the units of f, g; rho and u physical
    moment_sums(f, g, m);
    C bx = m.bx, by = m.by;  // physical b (Maxwell stress only)
    if constexpr (SCALED) {
        m.rho = p.rho0 + m.drho * C(kHalfInvScale);
        const C inv = C(1) / m.rho;
        m.ux = (m.mx * C(kHalfInvScale)) * inv;
        m.uy = (m.my * C(kHalfInvScale)) * inv;
        bx = m.bx * C(kHalfInvScale);
        by = m.by * C(kHalfInvScale);
    } else {
        m.rho = p.rho0 + m.drho;
        const C inv = C(1) / m.rho;
        m.ux = m.mx * inv;
        m.uy = m.my * inv;
    }
    const C ux = m.ux, uy = m.uy;
    // Maxwell stress M = |b|^2 I / 2 - b b (traceless in 2-D), in the units of f
    const C Mxx = C(0.5) * (by * m.by - bx * m.bx);
    const C Mxy = -bx * m.by;
    // task 3: projection a1^(2) = sum H2 (f - f_eq) = sum cc df - cs^2 drho I - rho uu - M
    const C Sxx = f[1] + f[2] + f[3] + f[5] + f[6] + f[7];
    const C Syy = f[1] + f[3] + f[4] + f[5] + f[7] + f[8];
    const C Sxy = (f[3] + f[7]) - (f[1] + f[5]);
    const C third = C(1.0 / 3.0);
    const C ruxx = m.mx * ux, ruyy = m.my * uy, ruxy = m.mx * uy;
    C a2xx = Sxx - third * m.drho - ruxx - Mxx;
    C a2yy = Syy - third * m.drho - ruyy + Mxx;
    C a2xy = Sxy - ruxy - Mxy;
    if constexpr (DA) {
        const C u = SCALED ? C(kHalfScale) : C(1);
        a2xx += u * da[0];
        a2xy += u * da[1];
        a2yy += u * da[2];
    }
    // recursion (task 3) on the supported components
    const C a3xxy = C(2) * ux * a2xy + uy * a2xx;
    const C a3xyy = C(2) * uy * a2xy + ux * a2yy;
    const C a4 = C(2) * ux * a3xyy + C(2) * uy * a3xxy - ux * ux * a2yy - C(4) * ux * uy * a2xy -
                 uy * uy * a2xx;
    const C om1 = C(1) - p.omega;
    const C k = p.collision == 0 ? om1 : C(0);
    Coeffs<C> A;
    A.drho = m.drho;
    A.mx = m.mx;
    A.my = m.my;
    A.A2xx = ruxx + Mxx + k * a2xx;
    A.A2yy = ruyy - Mxx + k * a2yy;
    A.A2xy = ruxy + Mxy + k * a2xy;
    C e3x = ruxy * ux, e3y = ruxy * uy, e4 = ruxy * ux * uy;  // rho ux^2 uy, rho ux uy^2, rho ux^2 uy^2
    if (p.variant == 1) {
        e3x += C(2) * ux * Mxy + uy * Mxx;
        e3y += -ux * Mxx + C(2) * uy * Mxy;
        e4 += -ux * ux * Mxx + C(4) * ux * uy * Mxy + uy * uy * Mxx;
    }
    A.A3xxy = e3x + k * a3xxy;
    A.A3xyy = e3y + k * a3xyy;
    A.A4 = e4 + k * a4;
    if (p.collision == 0) {
        hermite_eval(A, f);
    } else {
        C feq[9];
        hermite_eval(A, feq);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = feq[i] + om1 * (f[i] - feq[i]);
    }
    // Mass and momentum are collision invariants (a1^(0) = a1^(1) = 0).  The
    // weights 1/9, 1/36 are not representable, so the evaluated populations
    // carry a systematic relative bias of ~1e-8 (FP32) in their mass and
    // momentum; left alone it accumulates step after step.  Fold the
    // (algebraically zero) residuals back: x / y momentum into the axis pairs
    // (2, 6) / (4, 8), mass into the rest population.  In FP64 the residual
    // is ~1e-16 and the fold (about 20 FP64 instructions on units that bound
    // the FP64 step) is left out.
    constexpr bool kFold = !std::is_same<C, double>::value;
    if constexpr (kFold) {
        const C rx = m.mx - ((f[5] + f[6] + f[7]) - (f[1] + f[2] + f[3]));
        f[6] += C(0.5) * rx;
        f[2] -= C(0.5) * rx;
        const C ry = m.my - ((f[1] + f[7] + f[8]) - (f[3] + f[4] + f[5]));
        f[8] += C(0.5) * ry;
        f[4] -= C(0.5) * ry;
        f[0] = m.drho - (((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8])));
    }
    // magnetic BGK (Eq. collide_g): g* = omega_m g_eq + (1 - omega_m) g,
    // g_eq_{j,a} = psi_j [b_a + 3 e_{j,c} (u_c b_a - u_a b_c)], E = ux by - uy bx
    // (linear in b: evaluated in the units of g)
    const C Bx = m.bx, By = m.by;
    const C E3 = C(3) * (ux * By - uy * Bx);
    const C om = p.omega_m, omm1 = C(1) - p.omega_m;
    const C q1 = C(1.0 / 6.0);
    const C gbx = q1 * Bx, gby = q1 * By;
    if (p.mag_collision == 0) {
        g[2] = om * gbx + omm1 * g[2];               // j=1 (-1,0): x
        g[3] = om * (q1 * (By - E3)) + omm1 * g[3];  // j=1: y
        g[4] = om * (q1 * (Bx + E3)) + omm1 * g[4];  // j=2 (0,-1): x
        g[5] = om * gby + omm1 * g[5];               // j=2: y
        g[6] = om * gbx + omm1 * g[6];               // j=3 (+1,0): x
        g[7] = om * (q1 * (By + E3)) + omm1 * g[7];  // j=3: y
        g[8] = om * (q1 * (Bx - E3)) + omm1 * g[8];  // j=4 (0,+1): x
        g[9] = om * gby + omm1 * g[9];               // j=4: y
    } else {
        // Regularised: psi_j e_{j,a} Lambda_ab / cs^2 with Lambda the first
        // moment of g - g_eq keeps, on D2Q5, the antisymmetric half h of
        // each opposite pair's non-equilibrium (-h on j = 1, 2; +h on
        // j = 3, 4) and none on j = 0.
        const C e1y = q1 * (By - E3), e2x = q1 * (Bx + E3);
        const C e3y = q1 * (By + E3), e4x = q1 * (Bx - E3);
        const C h13x = C(0.5) * (g[6] - g[2]);  // g_eq equal on the pair
        const C h13y = C(0.5) * ((g[7] - e3y) - (g[3] - e1y));
        const C h24x = C(0.5) * ((g[8] - e4x) - (g[4] - e2x));
        const C h24y = C(0.5) * (g[9] - g[5]);
        g[2] = gbx - omm1 * h13x;
        g[6] = gbx + omm1 * h13x;
        g[3] = e1y - omm1 * h13y;
        g[7] = e3y + omm1 * h13y;
        g[4] = e2x - omm1 * h24x;
        g[8] = e4x + omm1 * h24x;
        g[5] = gby - omm1 * h24y;
        g[9] = gby + omm1 * h24y;
    }
    // rest population by difference: sum_j g*_j = b exactly (psi_0 + 4 psi_1
    // = 1 + 6e-8 in FP32 would otherwise grow b by ~1e-7 per step); FP64
    // relaxes it directly (psi_0 = 1/3; no non-equilibrium kept at j = 0
    // by the regularised collision)
    if constexpr (kFold) {
        g[0] = Bx - ((g[2] + g[4]) + (g[6] + g[8]));
        g[1] = By - ((g[3] + g[5]) + (g[7] + g[9]));
    } else {
        const C q0 = C(1.0 / 3.0);
        if (p.mag_collision == 0) {
            g[0] = om * (q0 * Bx) + omm1 * g[0];
            g[1] = om * (q0 * By) + omm1 * g[1];
        } else {
            g[0] = q0 * Bx;
            g[1] = q0 * By;
        }
    }
}

// How collide_nodes evaluates the collision of a thread's V nodes.
enum CollideMode {
    kNative = 0,    // C as given, products fused where the compiler chooses
    kPairs = 1,     // FP32: nodes (k, k+1) as one F2 on the packed FP32x2 instructions
    kExplicit = 2,  // FP32: one node at a time as F1, bitwise equal to kPairs
};

// Tasks 2-5 for the V nodes of one thread, held as v[plane][k].  kPairs
// does the arithmetic of two nodes in one instruction stream (about half
// the FP32 instructions, more registers live); it pays where the step is
// issue-bound (FP16S storage: half the bytes per node).  kExplicit is its
// one-node form (used for odd V), so that every FP16S kernel produces the
// same bits whatever its launch shape.
template <typename C, int V, bool SCALED, int MODE>
__device__ __forceinline__ void collide_nodes(C (&v)[kPlanes][V], const NodeParams<C>& np) {
    if constexpr (MODE == kNative) {
#pragma unroll
        for (int k = 0; k < V; ++k) {
            C f[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = v[i][k];
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = v[9 + q][k];
            collide_impl<false, C, SCALED>(f, g, np, nullptr);
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i][k] = f[i];
#pragma unroll
            for (int q = 0; q < 10; ++q) v[9 + q][k] = g[q];
        }
    } else if constexpr (MODE == kPairs && V % 2 == 0) {
        static_assert(std::is_same<C, float>::value, "packed pairs are FP32");
        NodeParams<F2> p2;
        p2.omega = F2(np.omega);
        p2.omega_m = F2(np.omega_m);
        p2.rho0 = F2(np.rho0);
        p2.variant = np.variant;
        p2.collision = np.collision;
        p2.mag_collision = np.mag_collision;
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            F2 f[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = F2(v[i][k], v[i][k + 1]);
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = F2(v[9 + q][k], v[9 + q][k + 1]);
            collide_impl<false, F2, SCALED>(f, g, p2, nullptr);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                v[i][k] = f[i].v.x;
                v[i][k + 1] = f[i].v.y;
            }
#pragma unroll
            for (int q = 0; q < 10; ++q) {
                v[9 + q][k] = g[q].v.x;
                v[9 + q][k + 1] = g[q].v.y;
            }
        }
    } else {
        static_assert(std::is_same<C, float>::value, "explicit fusion is FP32");
        NodeParams<F1> p1;
        p1.omega = F1(np.omega);
        p1.omega_m = F1(np.omega_m);
        p1.rho0 = F1(np.rho0);
        p1.variant = np.variant;
        p1.collision = np.collision;
        p1.mag_collision = np.mag_collision;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            F1 f[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = F1(v[i][k]);
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = F1(v[9 + q][k]);
            collide_impl<false, F1, SCALED>(f, g, p1, nullptr);
#pragma unroll
            for (int i = 0; i < 9; ++i) v[i][k] = f[i].v;
#pragma unroll
            for (int q = 0; q < 10; ++q) v[9 + q][k] = g[q].v;
        }
    }
}

// Equilibrium deviations for given fields (initial state; a1 = 0).
template <typename C>
__device__ __forceinline__ void equilibrium(C rho, C ux, C uy, C bx, C by, C rho0, int variant,
                                            C (&f)[9], C (&g)[10]) {
    const C Mxx = C(0.5) * (by * by - bx * bx);
    const C Mxy = -bx * by;
    const C mx = rho * ux, my = rho * uy;
    Coeffs<C> A;
    A.drho = rho - rho0;
    A.mx = mx;
    A.my = my;
    A.A2xx = mx * ux + Mxx;
    A.A2yy = my * uy - Mxx;
    A.A2xy = mx * uy + Mxy;
    A.A3xxy = mx * uy * ux;
    A.A3xyy = mx * uy * uy;
    A.A4 = mx * uy * ux * uy;
    if (variant == 1) {
        A.A3xxy += C(2) * ux * Mxy + uy * Mxx;
        A.A3xyy += -ux * Mxx + C(2) * uy * Mxy;
        A.A4 += -ux * ux * Mxx + C(4) * ux * uy * Mxy + uy * uy * Mxx;
    }
    hermite_eval(A, f);
    const C E3 = C(3) * (ux * by - uy * bx);
    const C q0 = C(1.0 / 3.0), q1 = C(1.0 / 6.0);
    g[0] = q0 * bx; g[1] = q0 * by;
    g[2] = q1 * bx; g[3] = q1 * (by - E3);
    g[4] = q1 * (bx + E3); g[5] = q1 * by;
    g[6] = q1 * bx; g[7] = q1 * (by + E3);
    g[8] = q1 * (bx - E3); g[9] = q1 * by;
}

// Current density of Eq. current from the pre-collision g of one node:
// j_z = -(omega_m / cs^2) [sum_j e_jx (g - g_eq)_jy - e_jy (g - g_eq)_jx].
// Only the j = 1..4 terms carry e != 0; g_eq for those is as in collide().
template <typename C>
__device__ __forceinline__ C current_density(const C (&g)[10], C ux, C uy, C bx, C by, C omega_m,
                                             C neq_scale) {
    const C E3 = C(3) * (ux * by - uy * bx);
    const C q1 = C(1.0 / 6.0);
    const C n1y = g[3] - q1 * (by - E3);
    const C n3y = g[7] - q1 * (by + E3);
    const C n2x = g[4] - q1 * (bx + E3);
    const C n4x = g[8] - q1 * (bx - E3);
    const C s = (n3y - n1y) - (n4x - n2x);
    return -C(3) * omega_m * neq_scale * s;
}

}  // namespace mhd
