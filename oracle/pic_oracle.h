/*
 * Plain, slow FP64 CPU oracle for the explicit electromagnetic particle-in-cell
 * (PIC) cycle of patch-based PIC codes (Sec. 3, "The importance of computational
 * load-management", and Sec. 3.1 "Dynamic load balancing": a PIC code whose cost is
 * the per-super-particle (SP) loop plus the field update).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may include, link, call or
 * execute this code; only the test suite, the smoke check and the bench's CPU
 * baseline do. It shares no code with the CUDA implementation.
 *
 * The paper identifies the field solver only as a standard second-order scheme (Sec. 2.1)
 * and prints no PIC equations, so every formula here is the standard published form:
 *   - Yee (1966) staggered FDTD for Faraday and Ampere,
 *   - quadratic B-spline (order-2) shape functions,
 *   - the relativistic Boris (1970) rotation,
 *   - Esirkepov (2001) charge-conserving current deposition.
 * Each function below says which of these it follows. Units are normalised:
 * c = eps0 = 1; dE/dt = curl B - J, dB/dt = -curl E, div E = rho.
 *
 * Layout: every field component is a plain row-major array [nz][ny][nx] (x fastest;
 * nz = 1 in 2D) with NO guard cells. Array index i of a component stands for the
 * position (i + s/2) * d, where s is that component's stagger bit along the axis:
 *      Ex (1,0,0)  Ey (0,1,0)  Ez (0,0,1)   (J like E)
 *      Bx (0,1,1)  By (1,0,1)  Bz (1,1,0)   (rho on nodes: (0,0,0))
 * Periodic axes wrap indices; along a moving-window x axis a value outside [0, nx)
 * is zero (fields) or dropped (current).
 */
#ifndef PIC_ORACLE_H
#define PIC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_config {
    int dims;           /* 2 (2D3V) or 3 (3D3V) */
    int n[3];           /* cells per axis (n[2] = 1 in 2D) */
    double d[3];        /* cell sizes */
    double dt;          /* time step */
    int window;         /* 0: x periodic; 1: x is a moving window at c (y, z periodic) */
    double q, m;        /* species charge and mass (electrons: -1, 1) */
    double n0;          /* injected plasma density (window only) */
    double ramp_x0;     /* lab-frame x where the linear density ramp starts */
    double ramp_len;    /* ramp length; n(x) = n0 * clamp((x - ramp_x0)/ramp_len, 0, 1) */
    int inject_ppc[3];  /* injected lattice per cell (window only) */
    int order;          /* Maxwell solver: 2 (or 0) = Yee; 6 = sixth-order staggered space
                           derivatives, leapfrog (second order) in time */
} orc_config;

typedef struct orc_sim orc_sim;

/* ---- building blocks (each used by the full step and pinned on its own) ---- */

/* Quadratic B-spline weights of a particle at coordinate xi (in cell units, already
 * shifted by -1/2 for a dual axis): nearest node i = floor(xi + 1/2),
 * delta = xi - i, S[0..2] = weights of nodes i-1, i, i+1. Returns i. */
long orc_shape2(double xi, double S[3]);

/* Relativistic Boris rotation: u^{n-1/2} -> u^{n+1/2} in the fields E, B. */
void orc_boris(double q, double m, double dt, const double E[3], const double B[3],
               double u[3]);

/* Order-2 interpolation of the six staggered components at a position.
 * F = {Ex,Ey,Ez,Bx,By,Bz}; out = the six values. */
void orc_interp(const orc_config* c, const double* const F[6], const double pos[3],
                double out[6]);

/* Esirkepov deposition of one particle moving pos0 -> pos1 (physical units,
 * |displacement| < one cell per axis), charge*weight qw, in-plane-unresolved
 * velocity vz (2D only). Adds into J = {Jx,Jy,Jz}. */
void orc_deposit(const orc_config* c, const double pos0[3], const double pos1[3],
                 double vz, double qw, double* const J[3]);

/* Order-2 charge density of n particles (adds into rho). */
void orc_rho(const orc_config* c, long long n, const double* x, const double* y,
             const double* z, const double* w, double q, double* rho);

/* Yee half-updates: E += dt (curl B - J); B -= dt curl E. In place. The curl takes
 * staggered differences of the configured order: order 2 is Yee's two-point difference;
 * order 6 is the centred staggered difference over six points,
 *   D f(x) = sum_{l=1..3} c_l [f(x + (l - 1/2) h) - f(x - (l - 1/2) h)] / h,
 * with c_l the unique coefficients exact for polynomials up to degree 6 (the
 * higher-order scheme of the paper's Photon-Plasma runs, Sec. 2.1). */
void orc_yee_e(const orc_config* c, double* const E[3], const double* const B[3],
               const double* const J[3]);
void orc_yee_b(const orc_config* c, const double* const E[3], double* const B[3]);

/* div E on nodes (two-point backward differences of the staggered E, whatever the
 * solver order: the difference under which Esirkepov's current conserves charge). */
void orc_div_e(const orc_config* c, const double* const E[3], double* out);

/* Number of window shifts after `step` steps: floor(step * dt / dx[0]). */
long long orc_shift_count(const orc_config* c, long long step);

/* ---- a whole simulation ---- */
orc_sim* orc_create(const orc_config* c, long long capacity);
void orc_destroy(orc_sim* s);
/* Particles: physical positions (z ignored in 2D), momenta u = gamma v, weights, ids. */
int orc_set_particles(orc_sim* s, long long n, const double* x, const double* y,
                      const double* z, const double* ux, const double* uy,
                      const double* uz, const double* w, const int* id);
long long orc_num_particles(const orc_sim* s);
int orc_get_particles(const orc_sim* s, double* x, double* y, double* z, double* ux,
                      double* uy, double* uz, double* w, int* id);
/* E at t = 0 and B at t = +dt/2; the first push uses that B at integer time too. */
int orc_set_fields(orc_sim* s, const double* Ex, const double* Ey, const double* Ez,
                   const double* Bx, const double* By, const double* Bz);
/* Copies out E^n, B^{n+1/2}, B^n (= the average used by the push) and the last
 * step's J^{n-1/2}: 12 arrays of ncell each, in that order. */
int orc_get_fields(const orc_sim* s, double* out12);
/* Background (immobile ion) charge density on nodes; NULL = minus the electron
 * density at the time of the call. */
int orc_set_rho_bg(orc_sim* s, const double* rho_bg);
int orc_step(orc_sim* s, int nsteps);
/* The same steps on up to `nthreads` host threads, with results identical bit for bit
 * to orc_step: particles are pushed in parallel, and each thread deposits every
 * particle's current (in particle order) into its own band of rows of J only, so each
 * element of J sums the same terms in the same order. Returns as orc_step (-4 if a
 * host allocation fails). */
int orc_step_mt(orc_sim* s, int nsteps, int nthreads);
long long orc_steps_done(const orc_sim* s);
long long orc_shifts_done(const orc_sim* s);
/* {W_E, W_B, W_kin} at integer time (B^n for W_B). */
void orc_energy(const orc_sim* s, double out[3]);
/* div E - rho_e - rho_bg on nodes (ncell values). */
void orc_gauss(const orc_sim* s, double* out);

/* ---- load limiting by particle merging ----
 * The paper bounds the SP count of overloaded regions by merging SP (Sec. 3.2, and
 * Sec. 3, where regions holding up to 40x the initial count are the load problem). It
 * prints no merge algorithm; this follows the published energy- and momentum-conserving
 * merge of Vranic et al., Comput. Phys. Commun. 191 (2015) 65:
 *   a group of N >= 3 particles sharing one cell and one momentum bin becomes two
 *   particles a, b with w_a = w_b = W/2 (W = sum w), gamma_a = gamma_b = E/W
 *   (E = sum w gamma), and momenta symmetric about P = sum w u, at the half angle
 *   theta with cos(theta) = |P| / (W |u_ab|), so that W, P and E are kept exactly.
 * Choices of this implementation (the published method leaves them free):
 *   - members are taken in increasing id; a and b keep the ids and positions of the two
 *     smallest ids;
 *   - the plane of u_a, u_b is spanned by P and the momentum of the smallest-id member
 *     (when that is parallel to P, by P and the coordinate axis least aligned with P);
 *     when P = 0, u_a = -u_b lies along that member's momentum (else the x axis);
 *   - the momentum bin of a particle is floor(u_a / dp) on each axis. */

/* Two-particle replacement of one group of n members. Returns 0 (nothing to do) when
 * n < 3; else 1 with the new momenta out_u[0..2] (a) and out_u[3..5] (b), the common
 * weight *out_w, and the member indices of a and b in keep[0], keep[1]. */
int orc_merge_group(long long n, const double* ux, const double* uy, const double* uz,
                    const double* w, const int* id, double out_u[6], double* out_w,
                    long long keep[2]);

/* Merge every group (same cell, same momentum bin of width dp, N >= 3) inside each
 * patch (patch[a] cells per axis) holding more than `above` particles and more than
 * 5/4 of its count after its previous merge pass (the sim remembers that count per
 * patch; an implementation choice, so that patches merging cannot bring below the
 * threshold are not reprocessed every step). Removed particles are compacted away,
 * order otherwise kept. Returns the number removed. */
long long orc_merge(orc_sim* s, const int patch[3], long long above, double dp);

/* ---- load limiting by particle splitting ----
 * The paper splits SP in cells of low SP number density and merges them in cells of
 * high density, conserving the physics (Sec. 3.2); the algorithm itself is in a reference
 * that is not available, so this rule is built from the conservation laws:
 *   a cell holding n particles, 1 <= n < below, is under-populated; its particles of
 *   weight w >= 2 wmin, taken in increasing id, are split one by one until the cell
 *   holds `below` particles or each of them has been split once. A split replaces
 *   (x, u, w) by (x + delta, u, w/2), keeping the id, and (x - delta, u, w/2), with a new
 *   id; delta_a = min(f_a, 1 - f_a) d_a / 2 on every axis, f_a the in-cell offset.
 * Halving is exact, so the total weight (charge), momentum sum w u and kinetic energy
 * sum w (gamma - 1) are kept exactly; both halves stay in the parent's cell (and patch),
 * the charge centroid is kept, and the second moment of the charge grows by w delta_a^2
 * per axis. New ids are next_id + the split's rank in (patch, cell, parent id) order,
 * patches numbered x fastest and cells in increasing local index (x fastest); next_id
 * then advances by the number of splits. Returns the number of splits, -1 on error
 * (capacity or allocation). */
long long orc_split(orc_sim* s, const int patch[3], long long below, double wmin);

#ifdef __cplusplus
}
#endif
#endif
