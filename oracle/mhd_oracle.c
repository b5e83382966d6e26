/*
 * mhd_oracle.c -- plain, slow FP64 CPU oracle of the recursive regularised
 * lattice Boltzmann method for 2-D incompressible MHD (De Rosis,
 * "Recursive regularised lattice Boltzmann method for magnetohydrodynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is what the CUDA path is checked
 * against.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA library: the lattice constants below are typed in again from the
 * paper, and every quantity is evaluated the long way, in the paper's order
 * and notation:
 *
 *   Section "Algorithm of computation", tasks 1-6:
 *     1. moments rho, u, b                      (Eq. for rho, u, b)
 *     2. f_eq as the Hermite series w_i sum_n a0^(n):H^(n)/(n! cs^2n)
 *        (Eq. fistar_acoeff / Eq. a0_4), g_eq (Dellar's magnetic equilibrium)
 *     3. a1^(2) by projection sum_i H2_i (f_i - f_eq_i); a1^(3), a1^(4) by
 *        the recursion, as full tensors over {x,y}^n
 *     4. f_neq,reg by Eq. fineq_reg (full contraction over the supported set)
 *     5. collide: f* = f_eq + (1-omega) f_neq,reg;  g* = g_eq + (1-omega_m) g_neq
 *        (optionally with g_neq regularised onto its first Hermite moment)
 *     6. stream, push form f_i(x + c_i, t+1) = f*_i(x, t)
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *   - nu = cs^2 (tau_f - 1/2), eta = cs^2 (tau_m - 1/2); the printed transport
 *     relation drops cs^2.  Only tau_f, tau_m enter this file.
 *   - The fourth-order H_xxyy equilibrium term carries 1/(4 cs^8): it is what
 *     the Hermite series of Eq. fistar_acoeff gives for the six permutations
 *     of xxyy, and it is what the series below produces.
 *   - Third and fourth orders keep only the D2Q9-supported classes xxy, xyy
 *     and xxyy (the same set as Eq. feq_4th); xxxx, yyyy (aliased onto H2 on
 *     D2Q9) and the classes that vanish on D2Q9 are left out.
 *   - Equilibrium variant A (default) is Eq. feq_4th as printed: the Maxwell
 *     stress enters only at second order.  Variant B takes a0^(3), a0^(4) of
 *     Eq. a0_4 with their u (x) M cross terms.
 *   - Walls (the paper is periodic only): half-way bounce-back of f and g.
 *   - j_z (Eq. current) uses the pre-collision g and g_eq of the same node,
 *     with eps_xy = +1, eps_yx = -1.
 *   - Gradients use the isotropic lattice stencil of the Orszag-Tang section.
 *
 * Array layout (this file's own): f[i*n + k] for i = 0..8, g[(2j+a)*n + k]
 * for j = 0..4, a = 0 (x), 1 (y); node k = y*nx + x, x fastest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice definitions (Section "BGK lattice Boltzmann formulation") ---- */
/* D2Q9 velocities in the ordering the paper gives (Latt's ordering). */
static const int CX[9] = {0, -1, -1, -1, 0, 1, 1, 1, 0};
static const int CY[9] = {0, 1, 0, -1, -1, -1, 0, 1, 1};
/* D2Q9 weights: rest 4/9, odd i (diagonals) 1/36, even i >= 2 (axes) 1/9. */
static const double W[9] = {4.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 9.0};
/* D2Q5 magnetic velocities and weights. */
static const int EX[5] = {0, -1, 0, 1, 0};
static const int EY[5] = {0, 0, -1, 0, 1};
static const double PSI[5] = {1.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0, 1.0 / 6.0};
/* lattice sound speed squared, cs = 1/sqrt(3) */
static const double CS2 = 1.0 / 3.0;

typedef struct {
    int nx, ny;
    double rho0, tau_f, tau_m;
    int wall_x, wall_y; /* 0: periodic axis, 1: half-way bounce-back walls */
    int eq_variant;     /* 0: A (Eq. feq_4th as printed), 1: B (Eq. a0_4 in full) */
    int collision;      /* 0: recursive regularised, 1: BGK (Eq. collide_f) */
    int mag_collision;  /* 0: BGK (Eq. collide_g); 1: regularised -- only the first
                           Hermite moment of g - g_eq relaxes (the extension of the
                           regularisation to the magnetic populations that the
                           Conclusions name as the next step) */
} orc_params;

static int opposite_f(int i) {
    for (int k = 0; k < 9; ++k)
        if (CX[k] == -CX[i] && CY[k] == -CY[i]) return k;
    return -1;
}
static int opposite_g(int j) {
    for (int k = 0; k < 5; ++k)
        if (EX[k] == -EX[j] && EY[k] == -EY[j]) return k;
    return -1;
}

void orc_lattice(int* cx, int* cy, double* w, int* ex, int* ey, double* psi) {
    for (int i = 0; i < 9; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = W[i]; }
    for (int j = 0; j < 5; ++j) { ex[j] = EX[j]; ey[j] = EY[j]; psi[j] = PSI[j]; }
}

/* ---- Hermite tensors (Section "BGK lattice Boltzmann formulation") ----
 * idx[k] in {0 (x), 1 (y)}; H^(n)_i evaluated from the definition. */
static double cvec(int i, int a) { return a == 0 ? (double)CX[i] : (double)CY[i]; }
static double kd(int a, int b) { return a == b ? 1.0 : 0.0; }

double orc_hermite(int n, const int* idx, int i) {
    if (n == 0) return 1.0;
    if (n == 1) return cvec(i, idx[0]);
    if (n == 2) {
        int a = idx[0], b = idx[1];
        return cvec(i, a) * cvec(i, b) - CS2 * kd(a, b);
    }
    if (n == 3) {
        int a = idx[0], b = idx[1], g = idx[2];
        return cvec(i, a) * cvec(i, b) * cvec(i, g) -
               CS2 * (cvec(i, a) * kd(b, g) + cvec(i, b) * kd(a, g) + cvec(i, g) * kd(a, b));
    }
    if (n == 4) {
        int a = idx[0], b = idx[1], g = idx[2], d = idx[3];
        double c4 = cvec(i, a) * cvec(i, b) * cvec(i, g) * cvec(i, d);
        double c2 = cvec(i, a) * cvec(i, b) * kd(g, d) + cvec(i, a) * cvec(i, g) * kd(b, d) +
                    cvec(i, a) * cvec(i, d) * kd(b, g) + cvec(i, b) * cvec(i, g) * kd(a, d) +
                    cvec(i, b) * cvec(i, d) * kd(a, g) + cvec(i, g) * cvec(i, d) * kd(a, b);
        double c0 = kd(a, b) * kd(g, d) + kd(a, g) * kd(b, d) + kd(a, d) * kd(b, g);
        return c4 - CS2 * c2 + CS2 * CS2 * c0;
    }
    return 0.0;
}

/* Components kept in the truncated expansion on D2Q9: all of orders 0-2, the
 * xxy / xyy classes at order 3 and the xxyy class at order 4. */
int orc_supported(int n, const int* idx) {
    if (n <= 2) return 1;
    int nxc = 0;
    for (int k = 0; k < n; ++k) nxc += (idx[k] == 0);
    if (n == 3) return nxc == 1 || nxc == 2;
    if (n == 4) return nxc == 2;
    return 0;
}

static void tuple_of(int n, int t, int* idx) {
    for (int k = 0; k < n; ++k) idx[k] = (t >> k) & 1;
}

static double factorial(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= k;
    return r;
}

/* Maxwell stress M_ab = |b|^2 delta_ab / 2 - b_a b_b. */
static double maxwell(const double* b, int a, int c) {
    return 0.5 * (b[0] * b[0] + b[1] * b[1]) * kd(a, c) - b[a] * b[c];
}

/* Equilibrium Hermite coefficient a0^(n) for one index tuple (Eq. a0_4).
 * Variant A drops the u (x) M terms at orders 3 and 4 (Eq. feq_4th). */
static double a0_coeff(int n, const int* id, double rho, const double* u, const double* b,
                       int variant) {
    switch (n) {
    case 0: return rho;
    case 1: return rho * u[id[0]];
    case 2: return rho * u[id[0]] * u[id[1]] + maxwell(b, id[0], id[1]);
    case 3: {
        double v = rho * u[id[0]] * u[id[1]] * u[id[2]];
        if (variant == 1)
            v += u[id[0]] * maxwell(b, id[1], id[2]) + u[id[1]] * maxwell(b, id[0], id[2]) +
                 u[id[2]] * maxwell(b, id[0], id[1]);
        return v;
    }
    case 4: {
        int a = id[0], bb = id[1], g = id[2], d = id[3];
        double v = rho * u[a] * u[bb] * u[g] * u[d];
        if (variant == 1)
            v += u[a] * u[bb] * maxwell(b, g, d) + u[a] * u[g] * maxwell(b, bb, d) +
                 u[a] * u[d] * maxwell(b, bb, g) + u[bb] * u[g] * maxwell(b, a, d) +
                 u[bb] * u[d] * maxwell(b, a, g) + u[g] * u[d] * maxwell(b, a, bb);
        return v;
    }
    }
    return 0.0;
}

/* H^(n)_i for every index tuple, tabulated once from orc_hermite, and the
 * series factors 1/(n! cs^(2n)).  Filled before any parallel region. */
static double HT[5][16][9];
static double SERIES[5];
static int tables_ready = 0;

static void ensure_tables(void) {
    if (tables_ready) return;
    int idx[4];
    for (int n = 0; n <= 4; ++n) {
        SERIES[n] = 1.0 / (factorial(n) * pow(CS2, n));
        for (int t = 0; t < (1 << n); ++t) {
            tuple_of(n, t, idx);
            for (int i = 0; i < 9; ++i) HT[n][t][i] = orc_hermite(n, idx, i);
        }
    }
    tables_ready = 1;
}

/* Task 2: f_eq_i = w_i sum_{n=0}^{4} a0^(n) : H_i^(n) / (n! cs^(2n)). */
void orc_feq(double rho, double ux, double uy, double bx, double by, int variant, double* feq) {
    ensure_tables();
    double u[2] = {ux, uy}, b[2] = {bx, by};
    double a0[5][16];
    int keep[5][16];
    int idx[4];
    for (int n = 0; n <= 4; ++n)
        for (int t = 0; t < (1 << n); ++t) {
            tuple_of(n, t, idx);
            keep[n][t] = orc_supported(n, idx);
            a0[n][t] = keep[n][t] ? a0_coeff(n, idx, rho, u, b, variant) : 0.0;
        }
    for (int i = 0; i < 9; ++i) {
        double s = 0.0;
        for (int n = 0; n <= 4; ++n) {
            double acc = 0.0;
            for (int t = 0; t < (1 << n); ++t)
                if (keep[n][t]) acc += a0[n][t] * HT[n][t][i];
            s += acc * SERIES[n];
        }
        feq[i] = W[i] * s;
    }
}

/* Task 2: g_eq_{j,a} = psi_j [ b_a + e_{j,c} (u_c b_a - u_a b_c) / cs^2 ]. */
void orc_geq(double ux, double uy, double bx, double by, double* geq) {
    double u[2] = {ux, uy}, b[2] = {bx, by};
    for (int j = 0; j < 5; ++j) {
        double e[2] = {(double)EX[j], (double)EY[j]};
        for (int a = 0; a < 2; ++a) {
            double s = 0.0;
            for (int c = 0; c < 2; ++c) s += e[c] * (u[c] * b[a] - u[a] * b[c]);
            geq[2 * j + a] = PSI[j] * (b[a] + s / CS2);
        }
    }
}

/* Task 1: rho = sum_i f_i, u = sum_i f_i c_i / rho, b = sum_j g_j. */
void orc_moments(const double* f, const double* g, double* out5) {
    double rho = 0.0, mx = 0.0, my = 0.0, bx = 0.0, by = 0.0;
    for (int i = 0; i < 9; ++i) { rho += f[i]; mx += f[i] * CX[i]; my += f[i] * CY[i]; }
    for (int j = 0; j < 5; ++j) { bx += g[2 * j]; by += g[2 * j + 1]; }
    out5[0] = rho; out5[1] = mx / rho; out5[2] = my / rho; out5[3] = bx; out5[4] = by;
}

/* Tasks 1-5 at one node.  da (may be NULL) is a learned correction
 * (xx, xy, yy) added to the projected a1^(2) before the recursion (the
 * closure; only the second- and higher-order non-equilibrium content changes,
 * so mass and momentum stay exact).  info (may be NULL) receives
 * [rho, ux, uy, bx, by, a2_xx, a2_xy, a2_yy, a3_xxy, a3_xyy, a4_xxyy,
 *  fneq_reg[0..8]] -- 20 doubles, with a2 before the correction. */
void orc_collide_node_da(const orc_params* p, const double* f, const double* g, const double* da,
                         double* fs, double* gs, double* info);

void orc_collide_node(const orc_params* p, const double* f, const double* g, double* fs,
                      double* gs, double* info) {
    orc_collide_node_da(p, f, g, NULL, fs, gs, info);
}

void orc_collide_node_da(const orc_params* p, const double* f, const double* g, const double* da,
                         double* fs, double* gs, double* info) {
    ensure_tables();
    double mom[5];
    orc_moments(f, g, mom);
    double rho = mom[0], u[2] = {mom[1], mom[2]}, b[2] = {mom[3], mom[4]};
    double feq[9], geq[10];
    orc_feq(rho, u[0], u[1], b[0], b[1], p->eq_variant, feq);
    orc_geq(u[0], u[1], b[0], b[1], geq);

    /* Task 3: projection of the second-order non-equilibrium coefficient. */
    double a2[2][2], a3[2][2][2], a4[2][2][2][2];
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            int id[2] = {a, c};
            double s = 0.0;
            for (int i = 0; i < 9; ++i) s += HT[2][id[0] | (id[1] << 1)][i] * (f[i] - feq[i]);
            a2[a][c] = s;
        }
    double a2_proj[3] = {a2[0][0], a2[0][1], a2[1][1]};
    if (da) {
        a2[0][0] += da[0];
        a2[0][1] += da[1];
        a2[1][0] += da[1];
        a2[1][1] += da[2];
    }
    /* recursion, third order: a3_abg = u_a a2_bg + u_b a2_ag + u_g a2_ab */
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c)
            for (int g3 = 0; g3 < 2; ++g3)
                a3[a][c][g3] = u[a] * a2[c][g3] + u[c] * a2[a][g3] + u[g3] * a2[a][c];
    /* recursion, fourth order: four u (x) a3 terms minus six u u (x) a2 terms */
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c)
            for (int g3 = 0; g3 < 2; ++g3)
                for (int d = 0; d < 2; ++d)
                    a4[a][c][g3][d] =
                        u[a] * a3[c][g3][d] + u[c] * a3[a][g3][d] + u[g3] * a3[a][c][d] +
                        u[d] * a3[a][c][g3] -
                        (u[a] * u[c] * a2[g3][d] + u[a] * u[g3] * a2[c][d] +
                         u[a] * u[d] * a2[c][g3] + u[c] * u[g3] * a2[a][d] +
                         u[c] * u[d] * a2[a][g3] + u[g3] * u[d] * a2[a][c]);

    /* Task 4: f_neq,reg (Eq. fineq_reg) over the supported components. */
    double fneq[9];
    int idx[4];
    for (int i = 0; i < 9; ++i) {
        double s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (int t = 0; t < 4; ++t) {
            tuple_of(2, t, idx);
            s2 += a2[idx[0]][idx[1]] * HT[2][t][i];
        }
        for (int t = 0; t < 8; ++t) {
            tuple_of(3, t, idx);
            if (!orc_supported(3, idx)) continue;
            s3 += a3[idx[0]][idx[1]][idx[2]] * HT[3][t][i];
        }
        for (int t = 0; t < 16; ++t) {
            tuple_of(4, t, idx);
            if (!orc_supported(4, idx)) continue;
            s4 += a4[idx[0]][idx[1]][idx[2]][idx[3]] * HT[4][t][i];
        }
        fneq[i] = W[i] * (s2 * SERIES[2] + s3 * SERIES[3] + s4 * SERIES[4]);
    }

    /* Task 5: collision. */
    double omega = 1.0 / p->tau_f, omega_m = 1.0 / p->tau_m;
    for (int i = 0; i < 9; ++i) {
        if (p->collision == 1)
            fs[i] = feq[i] + (1.0 - omega) * (f[i] - feq[i]);
        else
            fs[i] = feq[i] + (1.0 - omega) * fneq[i];
    }
    if (p->mag_collision == 1) {
        /* Regularised magnetic collision: project g - g_eq onto the first
         * Hermite moment, Lambda_ac = sum_j e_{j,a} (g_{j,c} - g_eq_{j,c}), and
         * rebuild g_neq,reg_{j,c} = psi_j e_{j,a} Lambda_ac / cs^2 (the zeroth
         * moment of g - g_eq is zero: b is conserved). */
        double lam[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
        for (int j = 0; j < 5; ++j) {
            double e[2] = {(double)EX[j], (double)EY[j]};
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) lam[a][c] += e[a] * (g[2 * j + c] - geq[2 * j + c]);
        }
        for (int j = 0; j < 5; ++j) {
            double e[2] = {(double)EX[j], (double)EY[j]};
            for (int c = 0; c < 2; ++c) {
                double reg = PSI[j] * (e[0] * lam[0][c] + e[1] * lam[1][c]) / CS2;
                gs[2 * j + c] = geq[2 * j + c] + (1.0 - omega_m) * reg;
            }
        }
    } else {
        for (int k = 0; k < 10; ++k) gs[k] = geq[k] + (1.0 - omega_m) * (g[k] - geq[k]);
    }

    if (info) {
        info[0] = rho; info[1] = u[0]; info[2] = u[1]; info[3] = b[0]; info[4] = b[1];
        info[5] = a2_proj[0]; info[6] = a2_proj[1]; info[7] = a2_proj[2];
        info[8] = a3[0][0][1]; info[9] = a3[0][1][1]; info[10] = a4[0][0][1][1];
        for (int i = 0; i < 9; ++i) info[11 + i] = fneq[i];
    }
}

static void gather_node(long n, long k, const double* f, const double* g, double* fl, double* gl) {
    for (int i = 0; i < 9; ++i) fl[i] = f[i * n + k];
    for (int q = 0; q < 10; ++q) gl[q] = g[q * n + k];
}

/* Task 5 over the lattice: fs, gs receive the post-collision populations. */
void orc_collide(const orc_params* p, const double* f, const double* g, double* fs, double* gs) {
    ensure_tables();
    long n = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double fl[9], gl[10], fo[9], go[10];
        gather_node(n, k, f, g, fl, gl);
        orc_collide_node(p, fl, gl, fo, go, NULL);
        for (int i = 0; i < 9; ++i) fs[i * n + k] = fo[i];
        for (int q = 0; q < 10; ++q) gs[q * n + k] = go[q];
    }
}

/* Task 5 over the lattice with a per-node correction da[3*k + (xx, xy, yy)]
 * of a1^(2) (NULL: none). */
void orc_collide_da(const orc_params* p, const double* f, const double* g, const double* da,
                    double* fs, double* gs) {
    ensure_tables();
    long n = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double fl[9], gl[10], fo[9], go[10];
        gather_node(n, k, f, g, fl, gl);
        orc_collide_node_da(p, fl, gl, da ? da + 3 * k : NULL, fo, go, NULL);
        for (int i = 0; i < 9; ++i) fs[i * n + k] = fo[i];
        for (int q = 0; q < 10; ++q) gs[q * n + k] = go[q];
    }
}

/* Per-node info of orc_collide_node for the whole lattice: info[20*k + .]. */
void orc_node_info(const orc_params* p, const double* f, const double* g, double* info) {
    ensure_tables();
    long n = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static)
    for (long k = 0; k < n; ++k) {
        double fl[9], gl[10], fo[9], go[10];
        gather_node(n, k, f, g, fl, gl);
        orc_collide_node(p, fl, gl, fo, go, info + 20 * k);
    }
}

/* Task 6: push streaming f_i(x + c_i) = f*_i(x).  On a wall axis a population
 * whose destination lies outside the lattice is reflected back into the
 * opposite direction of the node it left (half-way bounce-back). */
void orc_stream(const orc_params* p, const double* fs, const double* gs, double* f, double* g) {
    int nx = p->nx, ny = p->ny;
    long n = (long)nx * ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            for (int i = 0; i < 9; ++i) {
                int dx = x + CX[i], dy = y + CY[i];
                int out = (p->wall_x && (dx < 0 || dx >= nx)) || (p->wall_y && (dy < 0 || dy >= ny));
                if (out) {
                    f[(long)opposite_f(i) * n + k] = fs[(long)i * n + k];
                } else {
                    dx = (dx + nx) % nx; dy = (dy + ny) % ny;
                    f[(long)i * n + (long)dy * nx + dx] = fs[(long)i * n + k];
                }
            }
            for (int j = 0; j < 5; ++j) {
                int dx = x + EX[j], dy = y + EY[j];
                int out = (p->wall_x && (dx < 0 || dx >= nx)) || (p->wall_y && (dy < 0 || dy >= ny));
                for (int a = 0; a < 2; ++a) {
                    if (out) {
                        g[(long)(2 * opposite_g(j) + a) * n + k] = gs[(long)(2 * j + a) * n + k];
                    } else {
                        int ddx = (dx + nx) % nx, ddy = (dy + ny) % ny;
                        g[(long)(2 * j + a) * n + (long)ddy * nx + ddx] = gs[(long)(2 * j + a) * n + k];
                    }
                }
            }
        }
}

/* Initial state: f = f_eq(rho, u, b), g = g_eq(u, b) (zero non-equilibrium).
 * rho may be NULL, meaning rho = rho0 everywhere. */
void orc_init(const orc_params* p, const double* rho, const double* ux, const double* uy,
              const double* bx, const double* by, double* f, double* g) {
    long n = (long)p->nx * p->ny;
    for (long k = 0; k < n; ++k) {
        double feq[9], geq[10];
        double r = rho ? rho[k] : p->rho0;
        orc_feq(r, ux[k], uy[k], bx[k], by[k], p->eq_variant, feq);
        orc_geq(ux[k], uy[k], bx[k], by[k], geq);
        for (int i = 0; i < 9; ++i) f[i * n + k] = feq[i];
        for (int q = 0; q < 10; ++q) g[q * n + k] = geq[q];
    }
}

/* nsteps full time steps (collide, then stream), in place on f, g (which hold
 * the pre-collision populations).  Returns 0, or -1 if scratch could not be
 * allocated. */
int orc_run(const orc_params* p, double* f, double* g, long nsteps) {
    long n = (long)p->nx * p->ny;
    double* fs = (double*)malloc(sizeof(double) * 9 * n);
    double* gs = (double*)malloc(sizeof(double) * 10 * n);
    if (!fs || !gs) { free(fs); free(gs); return -1; }
    for (long s = 0; s < nsteps; ++s) {
        orc_collide(p, f, g, fs, gs);
        orc_stream(p, fs, gs, f, g);
    }
    free(fs); free(gs);
    return 0;
}

void orc_fields(const orc_params* p, const double* f, const double* g, double* rho, double* ux,
                double* uy, double* bx, double* by) {
    long n = (long)p->nx * p->ny;
    for (long k = 0; k < n; ++k) {
        double fl[9], gl[10], m[5];
        gather_node(n, k, f, g, fl, gl);
        orc_moments(fl, gl, m);
        rho[k] = m[0]; ux[k] = m[1]; uy[k] = m[2]; bx[k] = m[3]; by[k] = m[4];
    }
}

/* Eq. current: j_z = -(omega_m / cs^2) eps_ab sum_j e_{j,a} (g_{j,b} - g_eq_{j,b}),
 * from the pre-collision populations held in f, g. */
void orc_current(const orc_params* p, const double* f, const double* g, double* jz) {
    long n = (long)p->nx * p->ny;
    double omega_m = 1.0 / p->tau_m;
    for (long k = 0; k < n; ++k) {
        double fl[9], gl[10], m[5], geq[10];
        gather_node(n, k, f, g, fl, gl);
        orc_moments(fl, gl, m);
        orc_geq(m[1], m[2], m[3], m[4], geq);
        double s = 0.0;
        for (int j = 0; j < 5; ++j)
            for (int a = 0; a < 2; ++a)
                for (int c = 0; c < 2; ++c) {
                    double eps = (a == 0 && c == 1) ? 1.0 : (a == 1 && c == 0) ? -1.0 : 0.0;
                    double e = a == 0 ? EX[j] : EY[j];
                    s += eps * e * (gl[2 * j + c] - geq[2 * j + c]);
                }
        jz[k] = -(omega_m / CS2) * s;
    }
}

/* Isotropic lattice gradient (Orszag-Tang section):
 * d_a phi(x) = cs^-2 sum_i w_i phi(x + c_i) c_{i,a}.  Periodic axes wrap; on a
 * wall axis a node whose stencil leaves the lattice is marked invalid (0) and
 * its gradient set to 0. */
void orc_gradient(const orc_params* p, const double* phi, double* dx, double* dy,
                  unsigned char* valid) {
    int nx = p->nx, ny = p->ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            long k = (long)y * nx + x;
            double sx = 0.0, sy = 0.0;
            int ok = 1;
            for (int i = 0; i < 9; ++i) {
                int xx = x + CX[i], yy = y + CY[i];
                if ((p->wall_x && (xx < 0 || xx >= nx)) || (p->wall_y && (yy < 0 || yy >= ny))) {
                    ok = 0;
                    break;
                }
                xx = (xx + nx) % nx; yy = (yy + ny) % ny;
                double v = phi[(long)yy * nx + xx];
                sx += W[i] * v * CX[i];
                sy += W[i] * v * CY[i];
            }
            valid[k] = (unsigned char)ok;
            dx[k] = ok ? sx / CS2 : 0.0;
            dy[k] = ok ? sy / CS2 : 0.0;
        }
}

/* Global diagnostics of the pre-collision state (f, g):
 * out[0..11] = mass, mom_x, mom_y, e_kin, e_mag, cross_hel, bsum_x, bsum_y,
 *              divb_max, divb_rms, jz_max, omega_max
 * with e_kin = mean |u|^2/2 and e_mag = mean |b|^2/2 (the energy definitions
 * of the Orszag-Tang section, 1/(2L^2) int |.|^2), cross_hel = mean u.b,
 * divb_rms over the nodes whose gradient stencil is valid.
 * Returns 0, or -1 on allocation failure. */
int orc_totals(const orc_params* p, const double* f, const double* g, double* out) {
    long n = (long)p->nx * p->ny;
    double* buf = (double*)malloc(sizeof(double) * 14 * n);
    unsigned char* valid = (unsigned char*)malloc((size_t)n);
    if (!buf || !valid) { free(buf); free(valid); return -1; }
    double *rho = buf, *ux = buf + n, *uy = buf + 2 * n, *bx = buf + 3 * n, *by = buf + 4 * n;
    double *jz = buf + 5 * n, *d1 = buf + 6 * n, *d2 = buf + 7 * n, *d3 = buf + 8 * n,
           *d4 = buf + 9 * n, *d5 = buf + 10 * n, *d6 = buf + 11 * n, *d7 = buf + 12 * n,
           *d8 = buf + 13 * n;
    orc_fields(p, f, g, rho, ux, uy, bx, by);
    orc_current(p, f, g, jz);
    orc_gradient(p, ux, d1, d2, valid); /* d_x u_x, d_y u_x */
    orc_gradient(p, uy, d3, d4, valid); /* d_x u_y, d_y u_y */
    orc_gradient(p, bx, d5, d6, valid); /* d_x b_x, d_y b_x */
    orc_gradient(p, by, d7, d8, valid); /* d_x b_y, d_y b_y */
    double mass = 0, mxs = 0, mys = 0, ek = 0, em = 0, hc = 0, bxs = 0, bys = 0;
    double dmax = 0, dsq = 0, jmax = 0, wmax = 0;
    long nvalid = 0;
    for (long k = 0; k < n; ++k) {
        mass += rho[k];
        mxs += rho[k] * ux[k];
        mys += rho[k] * uy[k];
        ek += 0.5 * (ux[k] * ux[k] + uy[k] * uy[k]);
        em += 0.5 * (bx[k] * bx[k] + by[k] * by[k]);
        hc += ux[k] * bx[k] + uy[k] * by[k];
        bxs += bx[k];
        bys += by[k];
        if (fabs(jz[k]) > jmax) jmax = fabs(jz[k]);
        if (valid[k]) {
            double div = d5[k] + d8[k];
            double vort = d3[k] - d2[k];
            if (fabs(div) > dmax) dmax = fabs(div);
            if (fabs(vort) > wmax) wmax = fabs(vort);
            dsq += div * div;
            ++nvalid;
        }
    }
    out[0] = mass; out[1] = mxs; out[2] = mys;
    out[3] = ek / n; out[4] = em / n; out[5] = hc / n;
    out[6] = bxs; out[7] = bys;
    out[8] = dmax; out[9] = nvalid ? sqrt(dsq / nvalid) : 0.0;
    out[10] = jmax; out[11] = wmax;
    free(buf); free(valid);
    return 0;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
