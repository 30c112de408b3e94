/*
 * oracle_sp.c -- plain FP64 CPU oracle of the single-phase model of Remark 3
 * (Sec. 2.3) of arXiv:1902.08933: the generalized lattice Boltzmann model with
 * rho~ = rho_0 and a constant density rho (= 1), which recovers the
 * incompressible Navier-Stokes equations with a mass source,
 *   div u = S,
 *   d_t u + div(u u) = -grad p + div[nu (grad u + grad u^T)] + div[-(2/3) nu div u I] + F.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Build: gcc -O2 -ffp-contract=off.
 *
 * One time step on the D2Q9 lattice (Sec. 2.2), following Remark 3:
 *   u = sum_i c_i g_i + F/2                                   (Eq. 27a, rho = 1)
 *   G_i = w_i { S + c_i.F / c_s^2
 *              + (c_i c_i - c_s^2 I) : (u F + F u + Q S I) / (2 c_s^4) },
 *   Q = (2/d) rho c_s^2 - xi / (tau_g - 1/2)                  (after Eq. 27)
 *   p = c_s^2 / (1 - w_0) [ sum_{i != 0} g_i + S/2 + s_0(u) + (tau_g - 1/2) G_0 ]   (Eq. 28)
 *   g_i^eq = rho_0 + (p / c_s^2)(w_0 - 1) + s_0(u)  (i = 0),  (p / c_s^2) w_i + s_i(u)  (i != 0)
 *   g_i(x + c_i, t + 1) = g_i - (g_i - g_i^eq) / tau_g + (1 - 1/(2 tau_g)) G_i   (Eq. 24)
 * with tau_g = nu / c_s^2 + 1/2, a source field S(x) and a uniform force F;
 * x periodic, y periodic or halfway bounce-back walls. Layout as oracle.c.
 *
 * model = 1: the nearly incompressible form of Remark 1 (rho~ = rho, p = rho c_s^2):
 *   rho = sum_i g_i + S/2                                     (Eq. 27aa)
 *   u = (sum_i c_i g_i + F/2) / rho                           (Eq. 27a)
 *   g_i^eq = rho (w_i + s_i(u))                               (Eq. 29bb)
 *   G_i = w_i { S + c_i.F / c_s^2
 *              + (c_i c_i - c_s^2 I) : (u F + F u - u u S + Q div(u) I) / (2 c_s^4) },
 *   Q = (2/d) rho c_s^2 - xi / (tau_g - 1/2),
 * div u by the isotropic gradient of Eq. 30a (mirror at walls, reading Q7);
 * the u u S term is kept as printed.
 *
 * Remark 2 (orc_sp2_*): Eq. 29bb multiplied by c_s^2 with the O(Ma^2) part of
 * the density in front of s_i dropped, g in units of pressure:
 *   g_i^eq = w_i p + p_0 s_i(u)                                (Eq. 29bd)
 *   G_i = w_i { p_0 S_1 + p_0 c_i.F_1 / c_s^2
 *              + (c_i c_i - c_s^2 I) : [p_0 (u F_1 + F_1 u) + Q_2 div(u) I] / (2 c_s^4) },
 *   Q_2 = (2/d) p_0 c_s^2 - xi / (tau_g - 1/2)  (as printed),
 *   p = sum_i g_i + p_0 S_1 / 2,   p_0 u = sum_i c_i g_i + p_0 F_1 / 2,
 * with the constant p_0, the source S_1 and the force F_1 (S = p_0 S_1 and
 * F = p_0 F_1 in the notation of the other remarks); div u as for Remark 1.
 *
 * Remark 4 (orc_sp4_*): the Remark 3 model with a velocity-dependent force
 * F(u) = F_0 - (lambda + beta |u|) u, evolved without the shift of Eq. 23a and
 * with the explicit discretization of D_i G_i the remark gives:
 *   f_i(x + c_i, t + 1) = f_i - (f_i - f_i^eq) / tau_g
 *                        + G_i(x, t) + [G_i(x + c_i, t) - G_i(x, t - 1)] / 2,
 * u = sum_i c_i f_i (rho = 1; explicit: the moments of the unshifted f are the
 * equilibrium's, sum f = rho_0, sum c f = u), G_i of Remark 3 with F = F(u), and
 * the pressure of Eq. 28 rewritten for the unshifted f (f_0 - f_0^eq = tau G_0
 * to first order, the argument of App. B):
 *   p = c_s^2 / (1 - w_0) [ sum_{i != 0} f_i + s_0(u) + tau_g G_0 ].
 * G_i(x + c_i, t) across a wall is taken at the mirrored cell (as the stencils
 * of the phase-field model), and G_i(x, -1) = G_i(x, 0). G at t - 1 is kept as
 * the remark says (nine planes). Halfway bounce-back acts on g = f - G/2 of
 * Eq. 23a (the variable the rule is stated for): the population i that left x
 * towards the wall returns as f_opp = f_i^post - G_i(x + c_i, t)/2 + G_opp(x, t)/2,
 * so a fluid at rest under a uniform force stays at rest.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define QS 9
static const int SX[QS] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int SY[QS] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double SW[QS] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double SCS2 = 1.0 / 3.0;

static int sp_opposite(int i) {
    for (int k = 0; k < QS; ++k)
        if (SX[k] == -SX[i] && SY[k] == -SY[i]) return k;
    return -1;
}

static double sp_s(int i, double ux, double uy) {
    const double cu = SX[i] * ux + SY[i] * uy, uu = ux * ux + uy * uy;
    return SW[i] * (cu / SCS2 + cu * cu / (2.0 * SCS2 * SCS2) - uu / (2.0 * SCS2));
}

double orc_sp_tau(const orc_sp_params* P) { return P->nu / SCS2 + 0.5; }

/* Remark 3 equilibrium (Eq. 25 with rho~ = rho_0, rho = 1). */
void orc_sp_geq(double p, double ux, double uy, double rho0, double* geq) {
    for (int i = 0; i < QS; ++i)
        geq[i] = (i == 0 ? rho0 + p / SCS2 * (SW[0] - 1.0) : p / SCS2 * SW[i]) + sp_s(i, ux, uy);
}

/* Remark 3 force distribution, the contraction written out over alpha, beta. */
void orc_sp_force(const orc_sp_params* P, double S, double Fx, double Fy, double ux, double uy,
                  double* G) {
    const double rho = 1.0, tau = orc_sp_tau(P);
    const double Qc = (2.0 / 2.0) * rho * SCS2 - P->xi / (tau - 0.5);
    const double u[2] = {ux, uy}, F[2] = {Fx, Fy};
    double A[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) A[a][b] = u[a] * F[b] + F[a] * u[b] + (a == b ? Qc * S : 0.0);
    for (int i = 0; i < QS; ++i) {
        const double c[2] = {(double)SX[i], (double)SY[i]};
        double contraction = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) contraction += (c[a] * c[b] - (a == b ? SCS2 : 0.0)) * A[a][b];
        G[i] = SW[i] * (S + (c[0] * Fx + c[1] * Fy) / SCS2 + contraction / (2.0 * SCS2 * SCS2));
    }
}

/* u (Eq. 27a) and p (Eq. 28) of one cell from its populations. */
void orc_sp_moments(const orc_sp_params* P, const double* g, double S, double* ux, double* uy,
                    double* p) {
    double jx = 0.0, jy = 0.0, rest = 0.0;
    for (int i = 0; i < QS; ++i) {
        jx += SX[i] * g[i];
        jy += SY[i] * g[i];
        if (i) rest += g[i];
    }
    *ux = jx + 0.5 * P->force_x;
    *uy = jy + 0.5 * P->force_y;
    double G[QS];
    orc_sp_force(P, S, P->force_x, P->force_y, *ux, *uy, G);
    const double tau = orc_sp_tau(P);
    *p = SCS2 / (1.0 - SW[0]) * (rest + 0.5 * S + sp_s(0, *ux, *uy) + (tau - 0.5) * G[0]);
}

/* ---- Remark 1 ---- */
static double sp_at(const orc_sp_params* P, const double* f, int x, int y) {
    const int nx = P->nx, ny = P->ny;
    x = ((x % nx) + nx) % nx;
    if (P->walls_y) {
        if (y < 0) y = -1 - y;
        if (y >= ny) y = 2 * ny - 1 - y;
    } else {
        y = ((y % ny) + ny) % ny;
    }
    return f[(long)y * nx + x];
}

/* rho (Eq. 27aa) and u (Eq. 27a) of one cell. */
void orc_sp1_moments(const orc_sp_params* P, const double* g, double S, double* rho, double* ux, double* uy) {
    double m0 = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < QS; ++i) {
        m0 += g[i];
        jx += SX[i] * g[i];
        jy += SY[i] * g[i];
    }
    *rho = m0 + 0.5 * S;
    *ux = (jx + 0.5 * P->force_x) / *rho;
    *uy = (jy + 0.5 * P->force_y) / *rho;
}

/* Remark 1 force distribution with div u supplied. */
void orc_sp1_force(const orc_sp_params* P, double S, double rho, double ux, double uy, double divu,
                   double* G) {
    const double tau = orc_sp_tau(P);
    const double Qc = (2.0 / 2.0) * rho * SCS2 - P->xi / (tau - 0.5);
    const double u[2] = {ux, uy}, F[2] = {P->force_x, P->force_y};
    double A[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            A[a][b] = u[a] * F[b] + F[a] * u[b] - u[a] * u[b] * S + (a == b ? Qc * divu : 0.0);
    for (int i = 0; i < QS; ++i) {
        const double c[2] = {(double)SX[i], (double)SY[i]};
        double contraction = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) contraction += (c[a] * c[b] - (a == b ? SCS2 : 0.0)) * A[a][b];
        G[i] = SW[i] * (S + (c[0] * F[0] + c[1] * F[1]) / SCS2 + contraction / (2.0 * SCS2 * SCS2));
    }
}

/* Eq. 29bb. */
void orc_sp1_geq(double rho, double ux, double uy, double* geq) {
    for (int i = 0; i < QS; ++i) geq[i] = rho * (SW[i] + sp_s(i, ux, uy));
}

int orc_sp1_init(const orc_sp_params* P, double rho_init, double* g) {
    const long N = (long)P->nx * P->ny;
    double geq[QS];
    orc_sp1_geq(rho_init, 0.0, 0.0, geq);
    for (int i = 0; i < QS; ++i)
        for (long c = 0; c < N; ++c) g[i * N + c] = geq[i];
    return 0;
}

int orc_sp1_step(const orc_sp_params* P, const double* S, double* g, int nsteps) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    const double tau = orc_sp_tau(P);
    double* post = (double*)malloc((size_t)(QS * N) * sizeof(double));
    double* rho = (double*)malloc((size_t)N * sizeof(double));
    double* ux = (double*)malloc((size_t)N * sizeof(double));
    double* uy = (double*)malloc((size_t)N * sizeof(double));
    if (!post || !rho || !ux || !uy) {
        free(post); free(rho); free(ux); free(uy);
        return 2;
    }
    for (int step = 0; step < nsteps; ++step) {
        /* rho and u on the whole grid first (div u needs the neighbours') */
        for (long c = 0; c < N; ++c) {
            double gc[QS];
            for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
            orc_sp1_moments(P, gc, S[c], &rho[c], &ux[c], &uy[c]);
        }
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            const int x = (int)(c % nx), y = (int)(c / nx);
            double divu = 0.0;   /* Eq. 30a applied to u */
            for (int i = 1; i < QS; ++i)
                divu += SW[i] * (SX[i] * sp_at(P, ux, x + SX[i], y + SY[i]) +
                                 SY[i] * sp_at(P, uy, x + SX[i], y + SY[i])) / SCS2;
            double geq[QS], G[QS];
            orc_sp1_geq(rho[c], ux[c], uy[c], geq);
            orc_sp1_force(P, S[c], rho[c], ux[c], uy[c], divu, G);
            for (int i = 0; i < QS; ++i) {
                const double gi = g[i * N + c];
                post[i * N + c] = gi - (gi - geq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * G[i];
            }
        }
        for (int i = 0; i < QS; ++i) {
            const int oi = sp_opposite(i);
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long here = (long)y * nx + x;
                    const int ys = y - SY[i];
                    if (P->walls_y && (ys < 0 || ys >= ny)) {
                        g[i * N + here] = post[oi * N + here];
                    } else {
                        const int xs = ((x - SX[i]) % nx + nx) % nx, yw = (ys % ny + ny) % ny;
                        g[i * N + here] = post[i * N + (long)yw * nx + xs];
                    }
                }
        }
    }
    free(post); free(rho); free(ux); free(uy);
    return 0;
}

int orc_sp1_fields(const orc_sp_params* P, const double* S, const double* g, double* rho, double* ux,
                   double* uy) {
    const long N = (long)P->nx * P->ny;
    for (long c = 0; c < N; ++c) {
        double gc[QS], r, a, b;
        for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
        orc_sp1_moments(P, gc, S[c], &r, &a, &b);
        if (rho) rho[c] = r;
        if (ux) ux[c] = a;
        if (uy) uy[c] = b;
    }
    return 0;
}

int orc_sp_init(const orc_sp_params* P, double* g) {
    const long N = (long)P->nx * P->ny;
    double geq[QS];
    orc_sp_geq(0.0, 0.0, 0.0, P->rho0, geq);
    for (int i = 0; i < QS; ++i)
        for (long c = 0; c < N; ++c) g[i * N + c] = geq[i];
    return 0;
}

int orc_sp_step(const orc_sp_params* P, const double* S, double* g, int nsteps) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    const double tau = orc_sp_tau(P);
    double* post = (double*)malloc((size_t)(QS * N) * sizeof(double));
    if (!post) return 2;
    for (int step = 0; step < nsteps; ++step) {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            double gc[QS], geq[QS], G[QS], ux, uy, p;
            for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
            orc_sp_moments(P, gc, S[c], &ux, &uy, &p);
            orc_sp_geq(p, ux, uy, P->rho0, geq);
            orc_sp_force(P, S[c], P->force_x, P->force_y, ux, uy, G);
            for (int i = 0; i < QS; ++i)
                post[i * N + c] = gc[i] - (gc[i] - geq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * G[i];
        }
        /* streaming (pull), halfway bounce-back at y walls */
        for (int i = 0; i < QS; ++i) {
            const int oi = sp_opposite(i);
#pragma omp parallel for schedule(static)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long here = (long)y * nx + x;
                    const int ys = y - SY[i];
                    if (P->walls_y && (ys < 0 || ys >= ny)) {
                        g[i * N + here] = post[oi * N + here];
                    } else {
                        const int xs = ((x - SX[i]) % nx + nx) % nx, yw = (ys % ny + ny) % ny;
                        g[i * N + here] = post[i * N + (long)yw * nx + xs];
                    }
                }
        }
    }
    free(post);
    return 0;
}

int orc_sp_fields(const orc_sp_params* P, const double* S, const double* g, double* ux, double* uy,
                  double* p) {
    const long N = (long)P->nx * P->ny;
    for (long c = 0; c < N; ++c) {
        double gc[QS], a, b, q;
        for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
        orc_sp_moments(P, gc, S[c], &a, &b, &q);
        if (ux) ux[c] = a;
        if (uy) uy[c] = b;
        if (p) p[c] = q;
    }
    return 0;
}

/* ---- Remark 4 ---- */
void orc_sp4_force_of_u(const orc_sp_params* P, double ux, double uy, double* Fx, double* Fy) {
    const double k = P->drag_lin + P->drag_quad * sqrt(ux * ux + uy * uy);
    *Fx = P->force_x - k * ux;
    *Fy = P->force_y - k * uy;
}

/* u = sum c f, F(u), G_i(x, t) (Remark 3 with F(u)) and p of one cell. */
static void sp4_cell(const orc_sp_params* P, const double* f, double S, double* ux, double* uy,
                     double* p, double* G) {
    double jx = 0.0, jy = 0.0, rest = 0.0;
    for (int i = 0; i < QS; ++i) {
        jx += SX[i] * f[i];
        jy += SY[i] * f[i];
        if (i) rest += f[i];
    }
    *ux = jx;
    *uy = jy;
    double Fx, Fy;
    orc_sp4_force_of_u(P, jx, jy, &Fx, &Fy);
    orc_sp_force(P, S, Fx, Fy, jx, jy, G);
    *p = SCS2 / (1.0 - SW[0]) * (rest + sp_s(0, jx, jy) + orc_sp_tau(P) * G[0]);
}

void orc_sp4_moments(const orc_sp_params* P, const double* f, double S, double* ux, double* uy,
                     double* p) {
    double G[QS];
    sp4_cell(P, f, S, ux, uy, p, G);
}

int orc_sp4_init(const orc_sp_params* P, const double* S, double* f, double* Gprev) {
    const long N = (long)P->nx * P->ny;
    double geq[QS];
    orc_sp_geq(0.0, 0.0, 0.0, P->rho0, geq);
    for (int i = 0; i < QS; ++i)
        for (long c = 0; c < N; ++c) f[i * N + c] = geq[i];
    for (long c = 0; c < N; ++c) {   /* G at the initial state stands in for G at t = -1 */
        double G[QS], ux, uy, p, fc[QS];
        for (int i = 0; i < QS; ++i) fc[i] = f[i * N + c];
        sp4_cell(P, fc, S[c], &ux, &uy, &p, G);
        for (int i = 0; i < QS; ++i) Gprev[i * N + c] = G[i];
    }
    return 0;
}

int orc_sp4_step(const orc_sp_params* P, const double* S, double* f, double* Gprev, int nsteps) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    const double tau = orc_sp_tau(P);
    double* post = (double*)malloc((size_t)(QS * N) * sizeof(double));
    double* Gnow = (double*)malloc((size_t)(QS * N) * sizeof(double));
    double* pc = (double*)malloc((size_t)N * sizeof(double));
    double* uxc = (double*)malloc((size_t)N * sizeof(double));
    double* uyc = (double*)malloc((size_t)N * sizeof(double));
    if (!post || !Gnow || !pc || !uxc || !uyc) {
        free(post); free(Gnow); free(pc); free(uxc); free(uyc);
        return 2;
    }
    for (int step = 0; step < nsteps; ++step) {
        /* G_i(x, t) everywhere first: the update at x needs it at x + c_i */
        for (long c = 0; c < N; ++c) {
            double fc[QS], G[QS];
            for (int i = 0; i < QS; ++i) fc[i] = f[i * N + c];
            sp4_cell(P, fc, S[c], &uxc[c], &uyc[c], &pc[c], G);
            for (int i = 0; i < QS; ++i) Gnow[i * N + c] = G[i];
        }
        for (long c = 0; c < N; ++c) {
            const int x = (int)(c % nx), y = (int)(c / nx);
            double geq[QS];
            orc_sp_geq(pc[c], uxc[c], uyc[c], P->rho0, geq);
            for (int i = 0; i < QS; ++i) {
                const int xn = ((x + SX[i]) % nx + nx) % nx;
                int yn = y + SY[i];
                if (P->walls_y) {
                    if (yn < 0 || yn >= ny) yn = y;   /* mirror about the wall */
                } else {
                    yn = (yn % ny + ny) % ny;
                }
                const double Gdst = Gnow[i * N + (long)yn * nx + xn];
                const double fi = f[i * N + c];
                post[i * N + c] = fi - (fi - geq[i]) / tau + Gnow[i * N + c] +
                                  0.5 * (Gdst - Gprev[i * N + c]);
            }
        }
        for (int i = 0; i < QS; ++i) {
            const int oi = sp_opposite(i);
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long here = (long)y * nx + x;
                    const int ys = y - SY[i];
                    if (P->walls_y && (ys < 0 || ys >= ny)) {
                        /* halfway bounce-back of g = f - G/2 (Eq. 23a): the
                         * population oi left here towards the wall, whose
                         * G_oi(x + c_oi) is at the mirrored cell (x + c_oi,x, y) */
                        const int xm = ((x + SX[oi]) % nx + nx) % nx;
                        f[i * N + here] = post[oi * N + here] - 0.5 * Gnow[oi * N + (long)y * nx + xm] +
                                          0.5 * Gnow[i * N + here];
                    } else {
                        const int xs = ((x - SX[i]) % nx + nx) % nx, yw = (ys % ny + ny) % ny;
                        f[i * N + here] = post[i * N + (long)yw * nx + xs];
                    }
                }
        }
        memcpy(Gprev, Gnow, (size_t)(QS * N) * sizeof(double));
    }
    free(post); free(Gnow); free(pc); free(uxc); free(uyc);
    return 0;
}

int orc_sp4_fields(const orc_sp_params* P, const double* S, const double* f, double* ux, double* uy,
                   double* p) {
    const long N = (long)P->nx * P->ny;
    for (long c = 0; c < N; ++c) {
        double fc[QS], a, b, q;
        for (int i = 0; i < QS; ++i) fc[i] = f[i * N + c];
        orc_sp4_moments(P, fc, S[c], &a, &b, &q);
        if (ux) ux[c] = a;
        if (uy) uy[c] = b;
        if (p) p[c] = q;
    }
    return 0;
}

/* ---- Remark 2 ---- */
void orc_sp2_moments(const orc_sp_params* P, const double* g, double S1, double* p, double* ux,
                     double* uy) {
    double m0 = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < QS; ++i) {
        m0 += g[i];
        jx += SX[i] * g[i];
        jy += SY[i] * g[i];
    }
    *p = m0 + 0.5 * P->p0 * S1;
    *ux = (jx + 0.5 * P->p0 * P->force_x) / P->p0;
    *uy = (jy + 0.5 * P->p0 * P->force_y) / P->p0;
}

void orc_sp2_force(const orc_sp_params* P, double S1, double ux, double uy, double divu, double* G) {
    const double tau = orc_sp_tau(P), p0 = P->p0;
    const double Q2 = (2.0 / 2.0) * p0 * SCS2 - P->xi / (tau - 0.5);
    const double u[2] = {ux, uy}, F[2] = {P->force_x, P->force_y};
    double A[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) A[a][b] = p0 * (u[a] * F[b] + F[a] * u[b]) + (a == b ? Q2 * divu : 0.0);
    for (int i = 0; i < QS; ++i) {
        const double c[2] = {(double)SX[i], (double)SY[i]};
        double contraction = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) contraction += (c[a] * c[b] - (a == b ? SCS2 : 0.0)) * A[a][b];
        G[i] = SW[i] * (p0 * S1 + p0 * (c[0] * F[0] + c[1] * F[1]) / SCS2 + contraction / (2.0 * SCS2 * SCS2));
    }
}

void orc_sp2_geq(double p, double p0, double ux, double uy, double* geq) {
    for (int i = 0; i < QS; ++i) geq[i] = SW[i] * p + p0 * sp_s(i, ux, uy);
}

int orc_sp2_init(const orc_sp_params* P, double* g) {   /* p = p_0, u = 0 */
    const long N = (long)P->nx * P->ny;
    double geq[QS];
    orc_sp2_geq(P->p0, P->p0, 0.0, 0.0, geq);
    for (int i = 0; i < QS; ++i)
        for (long c = 0; c < N; ++c) g[i * N + c] = geq[i];
    return 0;
}

int orc_sp2_step(const orc_sp_params* P, const double* S1, double* g, int nsteps) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    const double tau = orc_sp_tau(P);
    if (!(P->p0 > 0.0)) return 1;
    double* post = (double*)malloc((size_t)(QS * N) * sizeof(double));
    double* pc = (double*)malloc((size_t)N * sizeof(double));
    double* ux = (double*)malloc((size_t)N * sizeof(double));
    double* uy = (double*)malloc((size_t)N * sizeof(double));
    if (!post || !pc || !ux || !uy) {
        free(post); free(pc); free(ux); free(uy);
        return 2;
    }
    for (int step = 0; step < nsteps; ++step) {
        for (long c = 0; c < N; ++c) {   /* p and u everywhere first (div u) */
            double gc[QS];
            for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
            orc_sp2_moments(P, gc, S1[c], &pc[c], &ux[c], &uy[c]);
        }
        for (long c = 0; c < N; ++c) {
            const int x = (int)(c % nx), y = (int)(c / nx);
            double divu = 0.0;   /* Eq. 30a applied to u */
            for (int i = 1; i < QS; ++i)
                divu += SW[i] * (SX[i] * sp_at(P, ux, x + SX[i], y + SY[i]) +
                                 SY[i] * sp_at(P, uy, x + SX[i], y + SY[i])) / SCS2;
            double geq[QS], G[QS];
            orc_sp2_geq(pc[c], P->p0, ux[c], uy[c], geq);
            orc_sp2_force(P, S1[c], ux[c], uy[c], divu, G);
            for (int i = 0; i < QS; ++i) {
                const double gi = g[i * N + c];
                post[i * N + c] = gi - (gi - geq[i]) / tau + (1.0 - 1.0 / (2.0 * tau)) * G[i];
            }
        }
        for (int i = 0; i < QS; ++i) {
            const int oi = sp_opposite(i);
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long here = (long)y * nx + x;
                    const int ys = y - SY[i];
                    if (P->walls_y && (ys < 0 || ys >= ny)) {
                        g[i * N + here] = post[oi * N + here];
                    } else {
                        const int xs = ((x - SX[i]) % nx + nx) % nx, yw = (ys % ny + ny) % ny;
                        g[i * N + here] = post[i * N + (long)yw * nx + xs];
                    }
                }
        }
    }
    free(post); free(pc); free(ux); free(uy);
    return 0;
}

int orc_sp2_fields(const orc_sp_params* P, const double* S1, const double* g, double* p, double* ux,
                   double* uy) {
    const long N = (long)P->nx * P->ny;
    for (long c = 0; c < N; ++c) {
        double gc[QS], a, b, q;
        for (int i = 0; i < QS; ++i) gc[i] = g[i * N + c];
        orc_sp2_moments(P, gc, S1[c], &q, &a, &b);
        if (p) p[c] = q;
        if (ux) ux[c] = a;
        if (uy) uy[c] = b;
    }
    return 0;
}
