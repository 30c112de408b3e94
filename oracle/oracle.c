/*
 * oracle.c -- plain FP64 CPU oracle of the phase-field lattice Boltzmann model
 * of arXiv:1902.08933 (Yuan, Chai, Wang, Shi), Sec. 3 with the boundary and
 * forcing choices of Sec. 4.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h). Build: gcc -O2 -ffp-contract=off.
 * The OpenMP pragmas only split independent per-cell loops across threads; no
 * reduction runs in parallel, so results do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* D2Q9 lattice, Sec. 2.2 (after Eq. 25): velocities c_i, weights omega_i,    */
/* c_s^2 = c^2/3 with c = dx/dt = 1.                                          */
/* ------------------------------------------------------------------------- */
#define Q 9
#define D 2
static const int    CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int    CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double OMEGA[Q] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                                1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
static const double PHI_A = 1.0, PHI_B = 0.0; /* Sec. 3.1, after Eq. 3aa */

/* Direction that points the opposite way; used by halfway bounce-back. */
static int opposite(int i) {
    for (int k = 0; k < Q; ++k)
        if (CX[k] == -CX[i] && CY[k] == -CY[i]) return k;
    return -1;
}

void orc_lattice(int* cx, int* cy, double* w, int* opp) {
    for (int i = 0; i < Q; ++i) {
        if (cx) cx[i] = CX[i];
        if (cy) cy[i] = CY[i];
        if (w) w[i] = OMEGA[i];
        if (opp) opp[i] = opposite(i);
    }
}

/* ------------------------------------------------------------------------- */
/* Derived parameters.                                                        */
/*   Eqs. 6-7: W = sqrt(8 kappa / beta), sigma = sqrt(2 kappa beta) / 6.      */
/*   Solving: kappa / beta = W^2 / 8 and kappa * beta = 18 sigma^2, so        */
/*   kappa = 3 sigma W / 2 and beta = 12 sigma / W.                           */
/*   Eq. 17: M_phi = eta c_s^2 (tau_h - 1/2) dt  =>  eta = M / (c_s^2 (tau_h - 1/2)). */
/*   Sec. 3.2: gamma = (rho_A - rho_B) / (phi_A rho_B - phi_B rho_A).          */
/* ------------------------------------------------------------------------- */
int orc_derive(const orc_params* P, orc_derived* Dd) {
    if (P->W <= 0.0 || P->tau_h <= 0.5 || P->rho_B <= 0.0 || P->rho_A <= 0.0) return 1;
    Dd->kappa = 1.5 * P->sigma * P->W;
    Dd->beta = 12.0 * P->sigma / P->W;
    Dd->eta = P->M / (CS2 * (P->tau_h - 0.5));
    Dd->gamma = (P->rho_A - P->rho_B) / (PHI_A * P->rho_B - PHI_B * P->rho_A);
    return 0;
}

/* s_i(u), Sec. 2.2 after Eq. 25. */
double orc_s(int i, double ux, double uy) {
    double cu = CX[i] * ux + CY[i] * uy;
    double uu = ux * ux + uy * uy;
    return OMEGA[i] * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* Equilibrium of the flow distribution, Eq. 33 (Eq. 25 with rho~ = rho_0). */
void orc_geq(double p, double rho, double ux, double uy, double rho0, double* geq) {
    for (int i = 0; i < Q; ++i) {
        if (i == 0)
            geq[i] = rho0 + p / CS2 * (OMEGA[i] - 1.0) + rho * orc_s(i, ux, uy);
        else
            geq[i] = p / CS2 * OMEGA[i] + rho * orc_s(i, ux, uy);
    }
}

/* Equilibrium of the order-parameter distribution, Eq. 11. */
void orc_heq(double phi, double mu, double eta, double ux, double uy, double* heq) {
    for (int i = 0; i < Q; ++i) {
        if (i == 0)
            heq[i] = phi + (OMEGA[i] - 1.0) * eta * mu;
        else
            heq[i] = OMEGA[i] * eta * mu + OMEGA[i] * (CX[i] * phi * ux + CY[i] * phi * uy) / CS2;
    }
}

/* Force distribution of the phase-field model, Eq. 34:
 *   G_i = omega_i [ S + c_i.F / c_s^2
 *                   + (c_i c_i - c_s^2 I) : (u Ft + Ft u + (2/d) rho c_s^2 S1 I) / (2 c_s^4) ]
 * with S = u.grad(rho) + rho S1 passed in, Ft the modified force F~ (Sec. 2.2,
 * after Eq. 27). The double contraction is written out over alpha, beta. */
void orc_force_dist(double S, double rho, double S1, double Fx, double Fy,
                    double Ftx, double Fty, double ux, double uy, double* G) {
    const double u[D] = {ux, uy};
    const double Ft[D] = {Ftx, Fty};
    double A[D][D]; /* u Ft + Ft u + (2/d) rho c_s^2 S1 I */
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b)
            A[a][b] = u[a] * Ft[b] + Ft[a] * u[b] + (a == b ? (2.0 / D) * rho * CS2 * S1 : 0.0);
    for (int i = 0; i < Q; ++i) {
        const double c[D] = {(double)CX[i], (double)CY[i]};
        double contraction = 0.0;
        for (int a = 0; a < D; ++a)
            for (int b = 0; b < D; ++b)
                contraction += (c[a] * c[b] - (a == b ? CS2 : 0.0)) * A[a][b];
        G[i] = OMEGA[i] * (S + (c[0] * Fx + c[1] * Fy) / CS2 + contraction / (2.0 * CS2 * CS2));
    }
}

/* The simplified G_0 printed after Eq. 34 (last line of that derivation):
 *   G_0 = omega_0 { (1 - 1/d) rho S1 - [u.(F - grad p)] / c_s^2 }. */
double orc_G0_printed(double rho, double S1, double Fx, double Fy,
                      double dpx, double dpy, double ux, double uy) {
    return OMEGA[0] * ((1.0 - 1.0 / D) * rho * S1 - (ux * (Fx - dpx) + uy * (Fy - dpy)) / CS2);
}

/* Source of the C-H equation, Eq. 14, with d_t(phi u) supplied by the caller
 * (first-order backward difference, Sec. 3.2.2). */
void orc_source_R(double tau_h, double dphiux, double dphiuy, double* R) {
    for (int i = 0; i < Q; ++i)
        R[i] = (1.0 - 1.0 / (2.0 * tau_h)) * OMEGA[i] * (CX[i] * dphiux + CY[i] * dphiuy) / CS2;
}

/* Pressure, Eq. 28 (scheme 0 or 1: the caller passes the G_0 it chose) or the
 * previous scheme Eq. 29 (scheme 2, no G_0 term). dt = 1. */
double orc_pressure(int scheme, const double* g, double S, double rho, double ux, double uy,
                    double tau_g, double G0) {
    double sum = 0.0;
    for (int i = 1; i < Q; ++i) sum += g[i];
    double bracket = sum + 0.5 * S + rho * orc_s(0, ux, uy);
    if (scheme != 2) bracket += (tau_g - 0.5) * G0;
    return CS2 / (1.0 - OMEGA[0]) * bracket;
}

/* Relaxation time of the flow distribution from the local viscosity:
 * nu = c_s^2 (tau_g - 1/2) dt (Sec. 2.2); nu from the inverse-linear rule of
 * Sec. 3.2.2 or, for viscosity == 1, the step dynamic viscosity of Sec. 4.3. */
double orc_tau_g(const orc_params* P, double phi, double rho) {
    double nu;
    if (P->viscosity == 0) {
        double phin = (phi - PHI_B) / (PHI_A - PHI_B);
        double inv_nu = phin * (1.0 / P->nu_A - 1.0 / P->nu_B) + 1.0 / P->nu_B;
        nu = 1.0 / inv_nu;
    } else {
        double mu_dyn = (phi >= 0.5) ? P->rho_A * P->nu_A : P->rho_B * P->nu_B;
        nu = mu_dyn / rho;
    }
    return nu / CS2 + 0.5;
}

/* ------------------------------------------------------------------------- */
/* Neighbour access for the finite-difference stencils. x is periodic. In y: */
/* periodic, or, next to a halfway bounce-back wall, the field is mirrored    */
/* about the wall (zeta(x,-1) = zeta(x,0), zeta(x,ny) = zeta(x,ny-1)); the    */
/* paper does not state the wall treatment of the stencils (reading Q7).       */
/* ------------------------------------------------------------------------- */
static double at(const orc_params* P, const double* f, int x, int y) {
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

/* Isotropic gradient, Eq. 30a. */
void orc_grad(const orc_params* P, const double* f, double* gx, double* gy) {
    const int nx = P->nx, ny = P->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double sx = 0.0, sy = 0.0;
            for (int i = 1; i < Q; ++i) {
                double z = at(P, f, x + CX[i], y + CY[i]);
                sx += OMEGA[i] * CX[i] * z / CS2;
                sy += OMEGA[i] * CY[i] * z / CS2;
            }
            gx[(long)y * nx + x] = sx;
            gy[(long)y * nx + x] = sy;
        }
}

/* Isotropic Laplacian, Eq. 30b. */
void orc_lap(const orc_params* P, const double* f, double* lap) {
    const int nx = P->nx, ny = P->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            double z0 = f[(long)y * nx + x];
            double s = 0.0;
            for (int i = 1; i < Q; ++i)
                s += 2.0 * OMEGA[i] * (at(P, f, x + CX[i], y + CY[i]) - z0) / CS2;
            lap[(long)y * nx + x] = s;
        }
}

/* Streaming, the left-hand side of Eqs. 10 and 24: a population moves from x
 * to x + c_i. Written as a pull: pre_i(x) = post_i(x - c_i). If x - c_i lies
 * beyond a halfway bounce-back wall (Sec. 4.3), the population that left x in
 * the opposite direction comes back: pre_i(x) = post_opp(i)(x). */
void orc_stream(const orc_params* P, const double* post, double* pre) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    for (int i = 0; i < Q; ++i) {
        const int oi = opposite(i);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int xs = x - CX[i], ys = y - CY[i];
                long dst = i * N + (long)y * nx + x;
                if (P->walls_y && (ys < 0 || ys >= ny)) {
                    pre[dst] = post[oi * N + (long)y * nx + x];
                } else {
                    xs = ((xs % nx) + nx) % nx;
                    ys = ((ys % ny) + ny) % ny;
                    pre[dst] = post[i * N + (long)ys * nx + xs];
                }
            }
    }
}

/* ------------------------------------------------------------------------- */
/* Macroscopic stage of one step: everything the collision needs, as whole-   */
/* grid arrays.                                                               */
/* ------------------------------------------------------------------------- */
typedef struct {
    double *phi, *rho, *lap_phi, *mu, *dphix, *dphiy, *dmux, *dmuy, *lap_mu, *dpx, *dpy;
    double *S1, *Fx, *Fy, *ux, *uy, *S, *tau_g, *Ftx, *Fty, *G0, *p;
} fields_t;

static int fields_alloc(fields_t* F, long N) {
    double** slots[] = {&F->phi, &F->rho, &F->lap_phi, &F->mu, &F->dphix, &F->dphiy, &F->dmux,
                        &F->dmuy, &F->lap_mu, &F->dpx, &F->dpy, &F->S1, &F->Fx, &F->Fy,
                        &F->ux, &F->uy, &F->S, &F->tau_g, &F->Ftx, &F->Fty, &F->G0, &F->p};
    int n = (int)(sizeof(slots) / sizeof(slots[0]));
    int bad = 0;
    for (int k = 0; k < n; ++k) {
        *slots[k] = (double*)calloc((size_t)N, sizeof(double));
        if (!*slots[k]) bad = 1;
    }
    return bad;
}

static void fields_free(fields_t* F) {
    double* slots[] = {F->phi, F->rho, F->lap_phi, F->mu, F->dphix, F->dphiy, F->dmux, F->dmuy,
                       F->lap_mu, F->dpx, F->dpy, F->S1, F->Fx, F->Fy, F->ux, F->uy,
                       F->S, F->tau_g, F->Ftx, F->Fty, F->G0, F->p};
    for (size_t k = 0; k < sizeof(slots) / sizeof(slots[0]); ++k) free(slots[k]);
}

/* Density from the order parameter, Eq. 3aa. */
static double density(const orc_params* P, double phi) {
    return P->rho_B + (phi - PHI_B) * (P->rho_A - P->rho_B) / (PHI_A - PHI_B);
}

/* Chemical potential, Eq. 8: mu = 4 beta phi (phi - 1)(phi - 1/2) - kappa lap(phi). */
static double chem_potential(const orc_derived* Dd, double phi, double lap_phi) {
    return 4.0 * Dd->beta * phi * (phi - 1.0) * (phi - 0.5) - Dd->kappa * lap_phi;
}

/* Steps 1-6 of a time step (reading of the step order: moments, phi stencil,
 * mu stencil, forces and velocity, pressure). grad p uses the pressure of the
 * previous step, p_prev (reading Q2: the paper leaves the p / grad p circularity
 * of Eqs. 28 and 34 open). */
static void macroscopic(const orc_params* P, const orc_derived* Dd, const double* h,
                        const double* g, const double* p_prev, fields_t* F) {
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;

    /* phi = sum_i h_i (Eq. 18); rho from phi (Eq. 3aa). */
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        double phi = 0.0;
        for (int i = 0; i < Q; ++i) phi += h[i * N + c];
        F->phi[c] = phi;
        F->rho[c] = density(P, phi);
    }
    /* lap(phi) (Eq. 30b), then mu (Eq. 8) on the whole grid. */
    orc_lap(P, F->phi, F->lap_phi);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) F->mu[c] = chem_potential(Dd, F->phi[c], F->lap_phi[c]);
    /* grad(phi), grad(mu), lap(mu), grad(p_prev) (Eq. 30). */
    orc_grad(P, F->phi, F->dphix, F->dphiy);
    orc_grad(P, F->mu, F->dmux, F->dmuy);
    orc_lap(P, F->mu, F->lap_mu);
    orc_grad(P, p_prev, F->dpx, F->dpy);

    const double drho_dphi = (P->rho_A - P->rho_B) / (PHI_A - PHI_B);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
        const double phi = F->phi[c], rho = F->rho[c], mu = F->mu[c];
        const double drx = drho_dphi * F->dphix[c], dry = drho_dphi * F->dphiy[c];
        /* S1 = -gamma div(M grad mu) for the QIM, 0 for the IM (Sec. 3.2.1). */
        const double S1 = P->qim ? -Dd->gamma * P->M * F->lap_mu[c] : 0.0;
        /* Total force F = F_s + G (Sec. 3.1); F_s = mu grad(phi) or -phi grad(mu)
         * (Sec. 4.2); body force: uniform density plus buoyancy (Sec. 4.4). */
        double Fsx, Fsy;
        if (P->surface_force == 0) {
            Fsx = mu * F->dphix[c];
            Fsy = mu * F->dphiy[c];
        } else {
            Fsx = -phi * F->dmux[c];
            Fsy = -phi * F->dmuy[c];
        }
        const double Fx = Fsx + P->force_x;
        const double Fy = Fsy + P->force_y - (rho - P->rho_A) * P->gravity;
        /* Velocity, Eq. 27a. */
        double jx = 0.0, jy = 0.0;
        for (int i = 0; i < Q; ++i) {
            jx += CX[i] * g[i * N + c];
            jy += CY[i] * g[i * N + c];
        }
        const double ux = (jx + 0.5 * Fx) / rho;
        const double uy = (jy + 0.5 * Fy) / rho;
        /* Mass source S = u.grad(rho) + rho S1 (Sec. 3.1). */
        const double S = ux * drx + uy * dry + rho * S1;
        const double tau_g = orc_tau_g(P, phi, rho);
        /* Modified force F~ = F - grad(p - rho c_s^2) (Sec. 2.2 after Eq. 27). */
        const double Ftx = Fx - F->dpx[c] + CS2 * drx;
        const double Fty = Fy - F->dpy[c] + CS2 * dry;
        /* G_0 for the pressure: printed simplification, or Eq. 34 at i = 0. */
        double G0 = 0.0;
        if (P->pressure == 0) {
            G0 = orc_G0_printed(rho, S1, Fx, Fy, F->dpx[c], F->dpy[c], ux, uy);
        } else if (P->pressure == 1) {
            double G[Q];
            orc_force_dist(S, rho, S1, Fx, Fy, Ftx, Fty, ux, uy, G);
            G0 = G[0];
        }
        double gc[Q];
        for (int i = 0; i < Q; ++i) gc[i] = g[i * N + c];
        F->S1[c] = S1;
        F->Fx[c] = Fx;
        F->Fy[c] = Fy;
        F->ux[c] = ux;
        F->uy[c] = uy;
        F->S[c] = S;
        F->tau_g[c] = tau_g;
        F->Ftx[c] = Ftx;
        F->Fty[c] = Fty;
        F->G0[c] = G0;
        /* Pressure, Eq. 28 (or Eq. 29). */
        F->p[c] = orc_pressure(P->pressure, gc, S, rho, ux, uy, tau_g, G0);
    }
}

/* ------------------------------------------------------------------------- */
/* Initial state (the paper does not state the LB initialisation, reading Q6): */
/* u = 0, p = 0, mu_0 from Eq. 8, h = h^eq(phi_0, mu_0, 0) (Eq. 11),          */
/* g = g^eq(p = 0, u = 0) (Eq. 33), phi u at t - dt = 0 (reading Q5).          */
/* ------------------------------------------------------------------------- */
int orc_init(const orc_params* P, const double* phi0, double* h, double* g,
             double* phiu_prev, double* p_prev) {
    orc_derived Dd;
    if (orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny;
    double* lap = (double*)malloc((size_t)N * sizeof(double));
    if (!lap) return 2;
    orc_lap(P, phi0, lap);
    for (long c = 0; c < N; ++c) {
        const double mu = chem_potential(&Dd, phi0[c], lap[c]);
        double heq[Q], geq[Q];
        orc_heq(phi0[c], mu, Dd.eta, 0.0, 0.0, heq);
        orc_geq(0.0, density(P, phi0[c]), 0.0, 0.0, P->rho0, geq);
        for (int i = 0; i < Q; ++i) {
            h[i * N + c] = heq[i];
            g[i * N + c] = geq[i];
        }
        phiu_prev[c] = 0.0;
        phiu_prev[N + c] = 0.0;
        p_prev[c] = 0.0;
    }
    free(lap);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Time stepping: macroscopic stage, collisions (Eqs. 24 and 10), streaming.   */
/* ------------------------------------------------------------------------- */
int orc_step(const orc_params* P, double* h, double* g, double* phiu_prev, double* p_prev,
             int nsteps) {
    orc_derived Dd;
    if (orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny;
    fields_t F;
    double* hpost = (double*)malloc((size_t)(Q * N) * sizeof(double));
    double* gpost = (double*)malloc((size_t)(Q * N) * sizeof(double));
    if (fields_alloc(&F, N) || !hpost || !gpost) {
        fields_free(&F);
        free(hpost);
        free(gpost);
        return 2;
    }
    for (int step = 0; step < nsteps; ++step) {
        macroscopic(P, &Dd, h, g, p_prev, &F);
#pragma omp parallel for schedule(static)
        for (long c = 0; c < N; ++c) {
            const double rho = F.rho[c], ux = F.ux[c], uy = F.uy[c], tau_g = F.tau_g[c];
            const double phi = F.phi[c];
            /* Flow distribution: Eq. 24 with g^eq (Eq. 33) and G_i (Eq. 34). */
            double geq[Q], G[Q];
            orc_geq(F.p[c], rho, ux, uy, P->rho0, geq);
            orc_force_dist(F.S[c], rho, F.S1[c], F.Fx[c], F.Fy[c], F.Ftx[c], F.Fty[c], ux, uy, G);
            for (int i = 0; i < Q; ++i) {
                const double gi = g[i * N + c];
                gpost[i * N + c] = gi - (gi - geq[i]) / tau_g + (1.0 - 1.0 / (2.0 * tau_g)) * G[i];
            }
            /* Order-parameter distribution: Eq. 10 with h^eq (Eq. 11) and R_i
             * (Eq. 14), d_t(phi u) by the first-order backward difference. */
            double heq[Q], R[Q];
            orc_heq(phi, F.mu[c], Dd.eta, ux, uy, heq);
            orc_source_R(P->tau_h, phi * ux - phiu_prev[c], phi * uy - phiu_prev[N + c], R);
            for (int i = 0; i < Q; ++i) {
                const double hi = h[i * N + c];
                hpost[i * N + c] = hi - (hi - heq[i]) / P->tau_h + R[i];
            }
            phiu_prev[c] = phi * ux;
            phiu_prev[N + c] = phi * uy;
            p_prev[c] = F.p[c];
        }
        orc_stream(P, hpost, h);
        orc_stream(P, gpost, g);
    }
    fields_free(&F);
    free(hpost);
    free(gpost);
    return 0;
}

/* Laplace-law pressure of Sec. 4.2:
 *   P = p_0 - kappa phi lap(phi) + kappa |grad phi|^2 / 2 + p,
 *   p_0 = phi psi'(phi) - psi(phi), psi = beta phi^2 (phi - 1)^2 (Eq. 5). */
static double laplace_P(const orc_derived* Dd, double phi, double lap_phi, double gx, double gy,
                        double p) {
    const double psi = Dd->beta * phi * phi * (phi - 1.0) * (phi - 1.0);
    const double dpsi = 2.0 * Dd->beta * phi * (phi - 1.0) * (2.0 * phi - 1.0);
    const double p0 = phi * dpsi - psi;
    return p0 - Dd->kappa * phi * lap_phi + 0.5 * Dd->kappa * (gx * gx + gy * gy) + p;
}

int orc_fields(const orc_params* P, const double* h, const double* g, const double* p_prev,
               double* phi, double* ux, double* uy, double* p, double* rho, double* mu,
               double* Plap) {
    orc_derived Dd;
    if (orc_derive(P, &Dd)) return 1;
    const long N = (long)P->nx * P->ny;
    fields_t F;
    if (fields_alloc(&F, N)) {
        fields_free(&F);
        return 2;
    }
    macroscopic(P, &Dd, h, g, p_prev, &F);
    for (long c = 0; c < N; ++c) {
        if (phi) phi[c] = F.phi[c];
        if (ux) ux[c] = F.ux[c];
        if (uy) uy[c] = F.uy[c];
        if (p) p[c] = F.p[c];
        if (rho) rho[c] = F.rho[c];
        if (mu) mu[c] = F.mu[c];
        if (Plap) Plap[c] = laplace_P(&Dd, F.phi[c], F.lap_phi[c], F.dphix[c], F.dphiy[c], F.p[c]);
    }
    fields_free(&F);
    return 0;
}

int orc_diagnostics(const orc_params* P, const double* h, const double* g, const double* p_prev,
                    orc_diag* out) {
    orc_derived Dd;
    if (orc_derive(P, &Dd)) return 1;
    const int nx = P->nx, ny = P->ny;
    const long N = (long)nx * ny;
    fields_t F;
    if (fields_alloc(&F, N)) {
        fields_free(&F);
        return 2;
    }
    macroscopic(P, &Dd, h, g, p_prev, &F);
    memset(out, 0, sizeof(*out));
    double sAx = 0, sAy = 0, sBx = 0, sBy = 0, PA = 0, PB = 0;
    for (long c = 0; c < N; ++c) {
        for (int i = 0; i < Q; ++i)
            if (!isfinite(h[i * N + c]) || !isfinite(g[i * N + c])) out->nonfinite = 1;
        const double x = (double)(c % nx), y = (double)(c / nx);
        const double phi = F.phi[c], rho = F.rho[c];
        const double uu = F.ux[c] * F.ux[c] + F.uy[c] * F.uy[c];
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
        const double Pl = laplace_P(&Dd, phi, F.lap_phi[c], F.dphix[c], F.dphiy[c], F.p[c]);
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
    fields_free(&F);
    return 0;
}

/* Eq. 37 with mu_A -> mu_up (0 < y <= h) and mu_B -> mu_down (-h <= y <= 0). */
double orc_layered_ux(double y, double hh, double Gdrive, double mu_up, double mu_down) {
    const double r = y / hh;
    const double a = (mu_up - mu_down) / (mu_up + mu_down);
    if (y > 0.0)
        return Gdrive * hh * hh / (2.0 * mu_up) * (-r * r - r * a + 2.0 * mu_up / (mu_up + mu_down));
    return Gdrive * hh * hh / (2.0 * mu_down) * (-r * r - r * a + 2.0 * mu_down / (mu_up + mu_down));
}
