/*
 * oracle.h -- plain FP64 CPU oracle of the phase-field lattice Boltzmann model
 * of Yuan, Chai, Wang and Shi, "A generalized lattice Boltzmann model for fluid
 * flow system and its application in two-phase flows" (arXiv:1902.08933), Sec. 3.
 *
 * TEST INFRASTRUCTURE. Only the test suite, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library. It shares no
 * code, header, table or helper with the CUDA path, and it never reads a value
 * produced by the CUDA path.
 *
 * The code is written to be checked against the paper by eye, not to be fast:
 * every field is materialised over the whole grid before the stencil that
 * consumes it, and each step follows the paper's equations in order.
 *
 * Units: lattice units, dx = dt = 1, so c = 1 and c_s^2 = 1/3 (Sec. 2.2, D2Q9).
 * Order parameter: phi_A = 1 (phase A), phi_B = 0 (phase B) (Sec. 3.1, Eq. 3aa).
 *
 * Grid layout of every array: a[y * nx + x], x fastest; population arrays hold
 * nine such planes, a[i * nx * ny + y * nx + x], i in the D2Q9 order of Sec. 2.2.
 *
 * Pinning: every function here is checked by the "not gpu" tests against
 * closed-form moment identities, conservation, symmetry, analytic solutions
 * (Laplace's law, layered Poiseuille flow, planar interface) and brute force.
 * Parts with no such pin are listed as "parity unpinned" in the design notes:
 * the late-time spinodal morphology and the rising-bubble trajectory are only
 * checked for agreement between oracle and GPU.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Model and boundary parameters of one simulation (Sec. 3, Sec. 4). */
typedef struct {
    int nx, ny;            /* grid; x is always periodic (Sec. 4)                         */
    int walls_y;           /* 0: periodic in y; 1: halfway bounce-back walls at y=-1/2 and
                              y=ny-1/2 (Sec. 4.3)                                          */
    int qim;               /* 0: incompressible model, S1 = 0; 1: quasi-incompressible,
                              S1 = -gamma div(M grad mu) (Sec. 3.2, Sec. 4 intro)           */
    int pressure;          /* 0: Eq. 28 with the simplified G_0 printed after Eq. 34;
                              1: Eq. 28 with G_0 taken from Eq. 34 at i = 0 (= Eq. 28aa);
                              2: the previous scheme, Eq. 29                                 */
    int surface_force;     /* 0: F_s = mu grad(phi) (Sec. 3.1); 1: F_s = -phi grad(mu) (Sec. 4.2) */
    int viscosity;         /* 0: inverse-linear 1/nu (Sec. 3.2); 1: step dynamic viscosity
                              mu = mu_A if phi >= 1/2 else mu_B (Sec. 4.3)                   */
    double rho_A, rho_B;   /* densities of phase A (phi=1) and B (phi=0)                    */
    double nu_A, nu_B;     /* kinematic viscosities of the two phases                        */
    double sigma, W;       /* surface tension and interface width (Eqs. 6-7)                 */
    double tau_h;          /* relaxation time of the C-H distribution (Eq. 10)              */
    double M;              /* mobility M_phi (Eq. 17)                                        */
    double force_x, force_y; /* uniform body-force density (e.g. the driving G of Sec. 4.3)  */
    double gravity;        /* buoyancy F_b,y = -(rho - rho_A) g (Sec. 4.4)                  */
    double rho0;           /* the constant rho~ = rho_0 of Eq. 33                            */
} orc_params;

/* Quantities derived from the parameters (Eqs. 6-7, 17, and gamma of Sec. 3.2). */
typedef struct {
    double beta, kappa, eta, gamma;
} orc_derived;

/* Per-grid diagnostics (Sec. 4.2 pressure P; sums for conservation checks). */
typedef struct {
    double sum_phi, sum_rho, kinetic_energy, max_u;
    double centroid_A_x, centroid_A_y;   /* phi-weighted centroid              */
    double centroid_B_x, centroid_B_y;   /* (1-phi)-weighted centroid          */
    double mass_A, mass_B;               /* sum phi, sum (1-phi)               */
    double P_bulk_A, P_bulk_B;           /* mean P over phi > 1-1e-3 / phi < 1e-3 */
    double n_bulk_A, n_bulk_B;           /* number of cells in each bulk       */
    int nonfinite;                        /* any non-finite population          */
} orc_diag;

/* ---- lattice and building blocks (pinned one by one) ---- */
void   orc_lattice(int* cx, int* cy, double* w, int* opposite);
int    orc_derive(const orc_params* P, orc_derived* D);
double orc_s(int i, double ux, double uy);
void   orc_geq(double p, double rho, double ux, double uy, double rho0, double* geq);
void   orc_heq(double phi, double mu, double eta, double ux, double uy, double* heq);
void   orc_force_dist(double S, double rho, double S1, double Fx, double Fy,
                      double Ftx, double Fty, double ux, double uy, double* G);
double orc_G0_printed(double rho, double S1, double Fx, double Fy,
                      double dpx, double dpy, double ux, double uy);
void   orc_source_R(double tau_h, double dphiux, double dphiuy, double* R);
double orc_pressure(int scheme, const double* g, double S, double rho, double ux, double uy,
                    double tau_g, double G0);
double orc_tau_g(const orc_params* P, double phi, double rho);
void   orc_grad(const orc_params* P, const double* f, double* gx, double* gy);
void   orc_lap(const orc_params* P, const double* f, double* lap);
void   orc_stream(const orc_params* P, const double* post, double* pre);

/* ---- whole-grid driver ---- */
/* state: h[9N], g[9N], phiu_prev[2N] (phi*ux plane then phi*uy), p_prev[N], N = nx*ny */
int  orc_init(const orc_params* P, const double* phi0, double* h, double* g,
              double* phiu_prev, double* p_prev);
int  orc_step(const orc_params* P, double* h, double* g, double* phiu_prev, double* p_prev,
              int nsteps);
/* Macroscopic fields at the current time, as one step would compute them before
 * collision. Any output pointer may be NULL. mu and P (Sec. 4.2) are extras. */
int  orc_fields(const orc_params* P, const double* h, const double* g, const double* p_prev,
                double* phi, double* ux, double* uy, double* p, double* rho,
                double* mu, double* Plap);
int  orc_diagnostics(const orc_params* P, const double* h, const double* g,
                     const double* p_prev, orc_diag* out);

/* ---- the same model on the D3Q15 lattice (Sec. 2.2 after Eq. 25; d = 3 in
 * Eq. 34 and in the printed G_0), oracle3d.c. Grid nx x ny x nz with x and z
 * periodic and y as in 2-D (walls_y); buoyancy along -y. Layout
 * a[(z * ny + y) * nx + x]; populations 15 planes in the paper's D3Q15 order;
 * phiu_prev 3 planes; velocities passed as u[3]. ---- */
void   orc3_lattice(int* cx, int* cy, int* cz, double* w, int* opposite);
double orc3_s(int i, const double* u);
void   orc3_geq(double p, double rho, const double* u, double rho0, double* geq);
void   orc3_heq(double phi, double mu, double eta, const double* u, double* heq);
void   orc3_force_dist(double S, double rho, double S1, const double* F, const double* Ft,
                       const double* u, double* G);
double orc3_G0_printed(double rho, double S1, const double* F, const double* dp, const double* u);
void   orc3_source_R(double tau_h, const double* dphiu, double* R);
double orc3_pressure(int scheme, const double* g, double S, double rho, const double* u,
                     double tau_g, double G0);
void   orc3_grad(const orc_params* P, int nz, const double* f, double* gx, double* gy, double* gz);
void   orc3_lap(const orc_params* P, int nz, const double* f, double* lap);
void   orc3_stream(const orc_params* P, int nz, const double* post, double* pre);
int    orc3_init(const orc_params* P, int nz, const double* phi0, double* h, double* g,
                 double* phiu_prev, double* p_prev);
int    orc3_step(const orc_params* P, int nz, double* h, double* g, double* phiu_prev,
                 double* p_prev, int nsteps);
int    orc3_fields(const orc_params* P, int nz, const double* h, const double* g,
                   const double* p_prev, double* phi, double* ux, double* uy, double* uz,
                   double* p, double* rho, double* mu, double* Plap);
int    orc3_diagnostics(const orc_params* P, int nz, const double* h, const double* g,
                        const double* p_prev, orc_diag* out);

/* ---- single-phase model of Remark 3 (Sec. 2.3): incompressible flow with a
 * mass source S(x) (div u = S), rho~ = rho_0, rho = 1, D2Q9; oracle_sp.c ---- */
typedef struct {
    int nx, ny;
    int walls_y;          /* 0 periodic in y, 1 halfway bounce-back walls        */
    double nu;            /* kinematic viscosity: tau_g = nu / c_s^2 + 1/2       */
    double xi;            /* bulk viscosity in Q = (2/d) rho c_s^2 - xi/(tau_g - 1/2) */
    double force_x, force_y;
    double rho0;          /* rho~ = rho_0 of the equilibrium                     */
    /* velocity-dependent force of the Remark 4 scheme:
     * F(u) = (force_x, force_y) - (drag_lin + drag_quad |u|) u                   */
    double drag_lin, drag_quad;
    double p0;            /* Remark 2: the constant p_0 (> 0)                    */
} orc_sp_params;

double orc_sp_tau(const orc_sp_params* P);
void   orc_sp_geq(double p, double ux, double uy, double rho0, double* geq);
void   orc_sp_force(const orc_sp_params* P, double S, double Fx, double Fy, double ux, double uy,
                    double* G);
void   orc_sp_moments(const orc_sp_params* P, const double* g, double S, double* ux, double* uy,
                      double* p);
int    orc_sp_init(const orc_sp_params* P, double* g);
/* S: source field, nx*ny; g: 9 planes of nx*ny */
int    orc_sp_step(const orc_sp_params* P, const double* S, double* g, int nsteps);
int    orc_sp_fields(const orc_sp_params* P, const double* S, const double* g, double* ux, double* uy,
                     double* p);
/* Remark 1, the nearly incompressible form (rho~ = rho, p = rho c_s^2): */
void   orc_sp1_moments(const orc_sp_params* P, const double* g, double S, double* rho, double* ux,
                       double* uy);
void   orc_sp1_force(const orc_sp_params* P, double S, double rho, double ux, double uy, double divu,
                     double* G);
void   orc_sp1_geq(double rho, double ux, double uy, double* geq);
int    orc_sp1_init(const orc_sp_params* P, double rho_init, double* g);
int    orc_sp1_step(const orc_sp_params* P, const double* S, double* g, int nsteps);
int    orc_sp1_fields(const orc_sp_params* P, const double* S, const double* g, double* rho,
                      double* ux, double* uy);

/* Remark 4: the Remark 3 model evolved with the explicit discretization of
 * D_i G_i (f_bar not shifted by G/2, u = sum c f_bar explicit even when F
 * depends on u). Gprev: the 9 planes of G_i at t - 1. */
void   orc_sp4_force_of_u(const orc_sp_params* P, double ux, double uy, double* Fx, double* Fy);
void   orc_sp4_moments(const orc_sp_params* P, const double* f, double S, double* ux, double* uy,
                       double* p);
int    orc_sp4_init(const orc_sp_params* P, const double* S, double* f, double* Gprev);
int    orc_sp4_step(const orc_sp_params* P, const double* S, double* f, double* Gprev, int nsteps);
int    orc_sp4_fields(const orc_sp_params* P, const double* S, const double* f, double* ux,
                      double* uy, double* p);

/* Remark 2 (He-type incompressible form with a source S_1): g in units of
 * pressure, p = sum g + p_0 S_1 / 2, p_0 u = sum c g + p_0 F_1 / 2 (force_x,
 * force_y are F_1; the source field is S_1). */
void   orc_sp2_moments(const orc_sp_params* P, const double* g, double S1, double* p, double* ux,
                       double* uy);
void   orc_sp2_force(const orc_sp_params* P, double S1, double ux, double uy, double divu, double* G);
void   orc_sp2_geq(double p, double p0, double ux, double uy, double* geq);
int    orc_sp2_init(const orc_sp_params* P, double* g);
int    orc_sp2_step(const orc_sp_params* P, const double* S1, double* g, int nsteps);
int    orc_sp2_fields(const orc_sp_params* P, const double* S1, const double* g, double* p, double* ux,
                      double* uy);

/* Analytic layered Poiseuille profile, Eq. 37: y measured from the interface,
 * walls at y = -hh and y = +hh, dynamic viscosity mu_up for 0 < y <= hh and
 * mu_down for -hh <= y <= 0 (Eq. 37 names them mu_A and mu_B). */
double orc_layered_ux(double y, double hh, double Gdrive, double mu_up, double mu_down);

#ifdef __cplusplus
}
#endif
#endif
