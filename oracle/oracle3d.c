/*
 * oracle3d.c -- plain FP64 CPU oracle of the same phase-field lattice Boltzmann
 * model (arXiv:1902.08933, Sec. 3) on the three-dimensional D3Q15 lattice that
 * Sec. 2.2 lists after Eq. 25. The model is written for a DdQq lattice (d
 * enters Eq. 34 and the printed G_0); this file is the 2-D oracle's step
 * sequence with d = 3 and the D3Q15 velocities and weights.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Build: gcc -O2 -ffp-contract=off.
 *
 * Geometry: nx x ny x nz, x and z periodic, y periodic or bounded by halfway
 * bounce-back walls (walls_y), exactly as the 2-D oracle treats x and y; the
 * stencils see the field mirrored about a wall (reading Q7). Buoyancy acts
 * along -y. Layout: a[(z * ny + y) * nx + x]; populations a[i * N + cell].
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* D3Q15, Sec. 2.2: omega_0 = 2/9, omega_1-6 = 1/9, omega_7-14 = 1/72, c_s^2 = 1/3. */
#define Q3 15
#define D3 3
static const int CX3[Q3] = {0, 1, 0, 0, -1, 0, 0, 1, 1, 1, -1, -1, -1, -1, 1};
static const int CY3[Q3] = {0, 0, 1, 0, 0, -1, 0, 1, 1, -1, 1, -1, -1, 1, -1};
static const int CZ3[Q3] = {0, 0, 0, 1, 0, 0, -1, 1, -1, 1, 1, -1, 1, -1, -1};
static const double W3[Q3] = {2.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0,
                              1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0, 1.0 / 72.0};
static const double CS2_3 = 1.0 / 3.0;

static int opposite3(int i) {
    for (int k = 0; k < Q3; ++k)
        if (CX3[k] == -CX3[i] && CY3[k] == -CY3[i] && CZ3[k] == -CZ3[i]) return k;
    return -1;
}

void orc3_lattice(int* cx, int* cy, int* cz, double* w, int* opp) {
    for (int i = 0; i < Q3; ++i) {
        if (cx) cx[i] = CX3[i];
        if (cy) cy[i] = CY3[i];
        if (cz) cz[i] = CZ3[i];
        if (w) w[i] = W3[i];
        if (opp) opp[i] = opposite3(i);
    }
}

static double dot3(int i, const double* v) { return CX3[i] * v[0] + CY3[i] * v[1] + CZ3[i] * v[2]; }

/* s_i(u), Sec. 2.2 after Eq. 25. */
double orc3_s(int i, const double* u) {
    const double cu = dot3(i, u);
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W3[i] * (cu / CS2_3 + cu * cu / (2.0 * CS2_3 * CS2_3) - uu / (2.0 * CS2_3));
}

/* Eq. 33. */
void orc3_geq(double p, double rho, const double* u, double rho0, double* geq) {
    for (int i = 0; i < Q3; ++i) {
        if (i == 0)
            geq[i] = rho0 + p / CS2_3 * (W3[i] - 1.0) + rho * orc3_s(i, u);
        else
            geq[i] = p / CS2_3 * W3[i] + rho * orc3_s(i, u);
    }
}

/* Eq. 11, with phi u = phi * u. */
void orc3_heq(double phi, double mu, double eta, const double* u, double* heq) {
    for (int i = 0; i < Q3; ++i) {
        if (i == 0)
            heq[i] = phi + (W3[i] - 1.0) * eta * mu;
        else
            heq[i] = W3[i] * eta * mu + W3[i] * phi * dot3(i, u) / CS2_3;
    }
}

/* Eq. 34 with d = 3, the double contraction written out over alpha, beta. */
void orc3_force_dist(double S, double rho, double S1, const double* F, const double* Ft,
                     const double* u, double* G) {
    double A[D3][D3];
    for (int a = 0; a < D3; ++a)
        for (int b = 0; b < D3; ++b)
            A[a][b] = u[a] * Ft[b] + Ft[a] * u[b] + (a == b ? (2.0 / D3) * rho * CS2_3 * S1 : 0.0);
    for (int i = 0; i < Q3; ++i) {
        const double c[D3] = {(double)CX3[i], (double)CY3[i], (double)CZ3[i]};
        double contraction = 0.0;
        for (int a = 0; a < D3; ++a)
            for (int b = 0; b < D3; ++b)
                contraction += (c[a] * c[b] - (a == b ? CS2_3 : 0.0)) * A[a][b];
        G[i] = W3[i] * (S + dot3(i, F) / CS2_3 + contraction / (2.0 * CS2_3 * CS2_3));
    }
}

/* The simplified G_0 printed after Eq. 34, with d = 3. */
double orc3_G0_printed(double rho, double S1, const double* F, const double* dp, const double* u) {
    const double uFp = u[0] * (F[0] - dp[0]) + u[1] * (F[1] - dp[1]) + u[2] * (F[2] - dp[2]);
    return W3[0] * ((1.0 - 1.0 / D3) * rho * S1 - uFp / CS2_3);
}

/* Eq. 14 with d_t(phi u) supplied. */
void orc3_source_R(double tau_h, const double* dphiu, double* R) {
    for (int i = 0; i < Q3; ++i) R[i] = (1.0 - 1.0 / (2.0 * tau_h)) * W3[i] * dot3(i, dphiu) / CS2_3;
}

/* Eq. 28 (schemes 0, 1 with the caller's G_0) or Eq. 29 (scheme 2). */
double orc3_pressure(int scheme, const double* g, double S, double rho, const double* u,
                     double tau_g, double G0) {
    double sum = 0.0;
    for (int i = 1; i < Q3; ++i) sum += g[i];
    double bracket = sum + 0.5 * S + rho * orc3_s(0, u);
    if (scheme != 2) bracket += (tau_g - 0.5) * G0;
    return CS2_3 / (1.0 - W3[0]) * bracket;
}

/* Neighbour access: x, z periodic; y periodic or mirrored about the walls. */
static double at3(const orc_params* P, int nz, const double* f, int x, int y, int z) {
    const int nx = P->nx, ny = P->ny;
    x = ((x % nx) + nx) % nx;
    z = ((z % nz) + nz) % nz;
    if (P->walls_y) {
        if (y < 0) y = -1 - y;
        if (y >= ny) y = 2 * ny - 1 - y;
    } else {
        y = ((y % ny) + ny) % ny;
    }
    return f[((long)z * ny + y) * nx + x];
}

/* Eq. 30a. */
void orc3_grad(const orc_params* P, int nz, const double* f, double* gx, double* gy, double* gz) {
    const int nx = P->nx, ny = P->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                double s[3] = {0.0, 0.0, 0.0};
                for (int i = 1; i < Q3; ++i) {
                    const double v = at3(P, nz, f, x + CX3[i], y + CY3[i], z + CZ3[i]);
                    s[0] += W3[i] * CX3[i] * v / CS2_3;
                    s[1] += W3[i] * CY3[i] * v / CS2_3;
                    s[2] += W3[i] * CZ3[i] * v / CS2_3;
                }
                const long c = ((long)z * ny + y) * nx + x;
                gx[c] = s[0];
                gy[c] = s[1];
                gz[c] = s[2];
            }
}

/* Eq. 30b. */
void orc3_lap(const orc_params* P, int nz, const double* f, double* lap) {
    const int nx = P->nx, ny = P->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const long c = ((long)z * ny + y) * nx + x;
                double s = 0.0;
                for (int i = 1; i < Q3; ++i)
                    s += 2.0 * W3[i] * (at3(P, nz, f, x + CX3[i], y + CY3[i], z + CZ3[i]) - f[c]) / CS2_3;
                lap[c] = s;
            }
}

/* Streaming (pull form), halfway bounce-back at the y walls. */
void orc3_stream(const orc_params* P, int nz, const double* post, double* pre) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny * nz;
    for (int i = 0; i < Q3; ++i) {
        const int oi = opposite3(i);
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    const long here = ((long)z * ny + y) * nx + x;
                    const int ys = y - CY3[i];
                    if (P->walls_y && (ys < 0 || ys >= ny)) {
                        pre[i * N + here] = post[oi * N + here];
                    } else {
                        const int xs = ((x - CX3[i]) % nx + nx) % nx;
                        const int zs = ((z - CZ3[i]) % nz + nz) % nz;
                        const int yw = ((ys % ny) + ny) % ny;
                        pre[i * N + here] = post[i * N + ((long)zs * ny + yw) * nx + xs];
                    }
                }
    }
}

/* Whole-grid fields of the macroscopic stage. */
typedef struct {
    double *phi, *rho, *lap_phi, *mu, *dphi[3], *dmu[3], *lap_mu, *dp[3];
    double *S1, *F[3], *u[3], *S, *tau_g, *Ft[3], *G0, *p;
} fields3_t;

static double** slot3(fields3_t* F, int k) {
    double** s[] = {&F->phi, &F->rho, &F->lap_phi, &F->mu, &F->dphi[0], &F->dphi[1], &F->dphi[2],
                    &F->dmu[0], &F->dmu[1], &F->dmu[2], &F->lap_mu, &F->dp[0], &F->dp[1], &F->dp[2],
                    &F->S1, &F->F[0], &F->F[1], &F->F[2], &F->u[0], &F->u[1], &F->u[2], &F->S,
                    &F->tau_g, &F->Ft[0], &F->Ft[1], &F->Ft[2], &F->G0, &F->p};
    return k < (int)(sizeof(s) / sizeof(s[0])) ? s[k] : NULL;
}

static int fields3_alloc(fields3_t* F, long N) {
    memset(F, 0, sizeof(*F));
    int bad = 0;
    for (int k = 0; slot3(F, k); ++k) {
        *slot3(F, k) = (double*)calloc((size_t)N, sizeof(double));
        if (!*slot3(F, k)) bad = 1;
    }
    return bad;
}

static void fields3_free(fields3_t* F) {
    for (int k = 0; slot3(F, k); ++k) free(*slot3(F, k));
}

static double density3(const orc_params* P, double phi) {
    return P->rho_B + phi * (P->rho_A - P->rho_B);   /* Eq. 3aa, phi_A = 1, phi_B = 0 */
}

static double chem3(const orc_derived* Dd, double phi, double lap_phi) {
    return 4.0 * Dd->beta * phi * (phi - 1.0) * (phi - 0.5) - Dd->kappa * lap_phi;   /* Eq. 8 */
}

/* Steps 1-6 of a time step, as in the 2-D oracle (grad p from p_prev, Q2). */
static void macroscopic3(const orc_params* P, int nz, const orc_derived* Dd, const double* h,
                         const double* g, const double* p_prev, fields3_t* F) {
    const long N = (long)P->nx * P->ny * nz;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        double phi = 0.0;
        for (int i = 0; i < Q3; ++i) phi += h[i * N + c];   /* Eq. 18 */
        F->phi[c] = phi;
        F->rho[c] = density3(P, phi);
    }
    orc3_lap(P, nz, F->phi, F->lap_phi);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) F->mu[c] = chem3(Dd, F->phi[c], F->lap_phi[c]);
    orc3_grad(P, nz, F->phi, F->dphi[0], F->dphi[1], F->dphi[2]);
    orc3_grad(P, nz, F->mu, F->dmu[0], F->dmu[1], F->dmu[2]);
    orc3_lap(P, nz, F->mu, F->lap_mu);
    orc3_grad(P, nz, p_prev, F->dp[0], F->dp[1], F->dp[2]);
    const double drho_dphi = P->rho_A - P->rho_B;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        const double phi = F->phi[c], rho = F->rho[c], mu = F->mu[c];
        double dr[3], Fo[3], u[3], Ft[3], dp[3];
        for (int a = 0; a < 3; ++a) {
            dr[a] = drho_dphi * F->dphi[a][c];
            dp[a] = F->dp[a][c];
        }
        const double S1 = P->qim ? -Dd->gamma * P->M * F->lap_mu[c] : 0.0;   /* Sec. 3.2.1 */
        for (int a = 0; a < 3; ++a)                                             /* Secs. 3.1, 4.2 */
            Fo[a] = P->surface_force == 0 ? mu * F->dphi[a][c] : -phi * F->dmu[a][c];
        Fo[0] += P->force_x;
        Fo[1] += P->force_y - (rho - P->rho_A) * P->gravity;                    /* Sec. 4.4 */
        double j[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q3; ++i) {
            const double gi = g[i * N + c];
            j[0] += CX3[i] * gi;
            j[1] += CY3[i] * gi;
            j[2] += CZ3[i] * gi;
        }
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * Fo[a]) / rho;          /* Eq. 27a */
        const double S = u[0] * dr[0] + u[1] * dr[1] + u[2] * dr[2] + rho * S1;
        const double tau_g = orc_tau_g(P, phi, rho);
        for (int a = 0; a < 3; ++a) Ft[a] = Fo[a] - dp[a] + CS2_3 * dr[a];
        double G0 = 0.0;
        if (P->pressure == 0) {
            G0 = orc3_G0_printed(rho, S1, Fo, dp, u);
        } else if (P->pressure == 1) {
            double G[Q3];
            orc3_force_dist(S, rho, S1, Fo, Ft, u, G);
            G0 = G[0];
        }
        double gc[Q3];
        for (int i = 0; i < Q3; ++i) gc[i] = g[i * N + c];
        F->S1[c] = S1;
        for (int a = 0; a < 3; ++a) {
            F->F[a][c] = Fo[a];
            F->u[a][c] = u[a];
            F->Ft[a][c] = Ft[a];
        }
        F->S[c] = S;
        F->tau_g[c] = tau_g;
        F->G0[c] = G0;
        F->p[c] = orc3_pressure(P->pressure, gc, S, rho, u, tau_g, G0);   /* Eq. 28 / 29 */
    }
}

/* Initial state, reading Q6 (as the 2-D oracle). phiu_prev holds 3 planes. */
int orc3_init(const orc_params* P, int nz, const double* phi0, double* h, double* g,
              double* phiu_prev, double* p_prev) {
    orc_derived Dd;
    if (nz < 1 || orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny * nz;
    double* lap = (double*)malloc((size_t)N * sizeof(double));
    if (!lap) return 2;
    orc3_lap(P, nz, phi0, lap);
    const double zero[3] = {0.0, 0.0, 0.0};
    for (long c = 0; c < N; ++c) {
        double heq[Q3], geq[Q3];
        orc3_heq(phi0[c], chem3(&Dd, phi0[c], lap[c]), Dd.eta, zero, heq);
        orc3_geq(0.0, density3(P, phi0[c]), zero, P->rho0, geq);
        for (int i = 0; i < Q3; ++i) {
            h[i * N + c] = heq[i];
            g[i * N + c] = geq[i];
        }
        for (int a = 0; a < 3; ++a) phiu_prev[a * N + c] = 0.0;
        p_prev[c] = 0.0;
    }
    free(lap);
    return 0;
}

/* Time steps: Eqs. 24 and 10, then streaming. */
int orc3_step(const orc_params* P, int nz, double* h, double* g, double* phiu_prev, double* p_prev,
              int nsteps) {
    orc_derived Dd;
    if (nz < 1 || orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny * nz;
    fields3_t F;
    double* hpost = (double*)malloc((size_t)(Q3 * N) * sizeof(double));
    double* gpost = (double*)malloc((size_t)(Q3 * N) * sizeof(double));
    if (fields3_alloc(&F, N) || !hpost || !gpost) {
        fields3_free(&F);
        free(hpost);
        free(gpost);
        return 2;
    }
    for (int step = 0; step < nsteps; ++step) {
        macroscopic3(P, nz, &Dd, h, g, p_prev, &F);
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            const double phi = F.phi[c], rho = F.rho[c], tau_g = F.tau_g[c];
            const double u[3] = {F.u[0][c], F.u[1][c], F.u[2][c]};
            const double Fo[3] = {F.F[0][c], F.F[1][c], F.F[2][c]};
            const double Ft[3] = {F.Ft[0][c], F.Ft[1][c], F.Ft[2][c]};
            double geq[Q3], G[Q3], heq[Q3], R[Q3];
            orc3_geq(F.p[c], rho, u, P->rho0, geq);
            orc3_force_dist(F.S[c], rho, F.S1[c], Fo, Ft, u, G);
            for (int i = 0; i < Q3; ++i) {
                const double gi = g[i * N + c];
                gpost[i * N + c] = gi - (gi - geq[i]) / tau_g + (1.0 - 1.0 / (2.0 * tau_g)) * G[i];
            }
            orc3_heq(phi, F.mu[c], Dd.eta, u, heq);
            double dphiu[3];
            for (int a = 0; a < 3; ++a) dphiu[a] = phi * u[a] - phiu_prev[a * N + c];
            orc3_source_R(P->tau_h, dphiu, R);
            for (int i = 0; i < Q3; ++i) {
                const double hi = h[i * N + c];
                hpost[i * N + c] = hi - (hi - heq[i]) / P->tau_h + R[i];
            }
            for (int a = 0; a < 3; ++a) phiu_prev[a * N + c] = phi * u[a];
            p_prev[c] = F.p[c];
        }
        orc3_stream(P, nz, hpost, h);
        orc3_stream(P, nz, gpost, g);
    }
    fields3_free(&F);
    free(hpost);
    free(gpost);
    return 0;
}

/* Laplace-law pressure of Sec. 4.2 in 3-D. */
static double laplace_P3(const orc_derived* Dd, double phi, double lap_phi, const double* gphi, double p) {
    const double psi = Dd->beta * phi * phi * (phi - 1.0) * (phi - 1.0);
    const double dpsi = 2.0 * Dd->beta * phi * (phi - 1.0) * (2.0 * phi - 1.0);
    const double g2 = gphi[0] * gphi[0] + gphi[1] * gphi[1] + gphi[2] * gphi[2];
    return phi * dpsi - psi - Dd->kappa * phi * lap_phi + 0.5 * Dd->kappa * g2 + p;
}

int orc3_fields(const orc_params* P, int nz, const double* h, const double* g, const double* p_prev,
                double* phi, double* ux, double* uy, double* uz, double* p, double* rho, double* mu,
                double* Plap) {
    orc_derived Dd;
    if (nz < 1 || orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny * nz;
    fields3_t F;
    if (fields3_alloc(&F, N)) {
        fields3_free(&F);
        return 2;
    }
    macroscopic3(P, nz, &Dd, h, g, p_prev, &F);
    for (long c = 0; c < N; ++c) {
        const double gphi[3] = {F.dphi[0][c], F.dphi[1][c], F.dphi[2][c]};
        if (phi) phi[c] = F.phi[c];
        if (ux) ux[c] = F.u[0][c];
        if (uy) uy[c] = F.u[1][c];
        if (uz) uz[c] = F.u[2][c];
        if (p) p[c] = F.p[c];
        if (rho) rho[c] = F.rho[c];
        if (mu) mu[c] = F.mu[c];
        if (Plap) Plap[c] = laplace_P3(&Dd, F.phi[c], F.lap_phi[c], gphi, F.p[c]);
    }
    fields3_free(&F);
    return 0;
}

/* Diagnostics as in 2-D; the centroids are given in x and y. */
int orc3_diagnostics(const orc_params* P, int nz, const double* h, const double* g,
                     const double* p_prev, orc_diag* out) {
    orc_derived Dd;
    if (nz < 1 || orc_derive(P, &Dd)) return 1;
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny * nz;
    fields3_t F;
    if (fields3_alloc(&F, N)) {
        fields3_free(&F);
        return 2;
    }
    macroscopic3(P, nz, &Dd, h, g, p_prev, &F);
    memset(out, 0, sizeof(*out));
    double sAx = 0, sAy = 0, sBx = 0, sBy = 0, PA = 0, PB = 0;
    for (long c = 0; c < N; ++c) {
        for (int i = 0; i < Q3; ++i)
            if (!isfinite(h[i * N + c]) || !isfinite(g[i * N + c])) out->nonfinite = 1;
        const double x = (double)(c % nx), y = (double)((c / nx) % ny);
        const double phi = F.phi[c], rho = F.rho[c];
        const double uu = F.u[0][c] * F.u[0][c] + F.u[1][c] * F.u[1][c] + F.u[2][c] * F.u[2][c];
        const double gphi[3] = {F.dphi[0][c], F.dphi[1][c], F.dphi[2][c]};
        out->sum_phi += phi;
        out->sum_rho += rho;
        out->kinetic_energy += 0.5 * rho * uu;
        if (sqrt(uu) > out->max_u) out->max_u = sqrt(uu);
        out->mass_A += phi;
        out->mass_B += 1.0 - phi;
        sAx += phi * x;
        sAy += phi * y;
        sBx += (1.0 - phi) * x;
        sBy += (1.0 - phi) * y;
        const double Pl = laplace_P3(&Dd, phi, F.lap_phi[c], gphi, F.p[c]);
        if (phi > 1.0 - 1e-3) {
            PA += Pl;
            out->n_bulk_A += 1.0;
        }
        if (phi < 1e-3) {
            PB += Pl;
            out->n_bulk_B += 1.0;
        }
    }
    out->centroid_A_x = sAx / out->mass_A;
    out->centroid_A_y = sAy / out->mass_A;
    out->centroid_B_x = sBx / out->mass_B;
    out->centroid_B_y = sBy / out->mass_B;
    out->P_bulk_A = out->n_bulk_A > 0 ? PA / out->n_bulk_A : 0.0;
    out->P_bulk_B = out->n_bulk_B > 0 ? PB / out->n_bulk_B : 0.0;
    fields3_free(&F);
    return 0;
}
