/*
 * Plain FP64 CPU oracle of the explicit PIC cycle (test infrastructure only; see
 * pic_oracle.h). Loops are written in the order of the published definitions with
 * no blocking, fusion or reordering, so that each function can be checked by eye:
 *
 *   step:  B^n = (B^{n-1/2} + B^{n+1/2})/2 (kept from the previous step)
 *          for every particle: order-2 interpolation of E^n, B^n at x^n,
 *                              Boris  u^{n-1/2} -> u^{n+1/2},
 *                              move   x^{n+1} = x^n + dt u/gamma,
 *                              Esirkepov deposit of J^{n+1/2} from x^n -> x^{n+1}
 *          particle boundaries (periodic wrap; window: absorb outside [0, Lx))
 *          Ampere   E^{n+1}   = E^n + dt (curl B^{n+1/2} - J^{n+1/2})
 *          Faraday  B^{n+3/2} = B^{n+1/2} - dt curl E^{n+1};  B^{n+1} = average
 *          moving window: shift by one cell when floor(step dt/dx) increments,
 *          drop particles with x < 0, inject a cold lattice column on the right.
 *
 * The paper (Sec. 2.1) identifies only a standard second-order field scheme; the
 * schemes are the textbook ones: Yee 1966; Boris 1970; Esirkepov 2001 (Comput. Phys. Commun.
 * 135, 144), Eqs. for W and the cumulative current; quadratic B-spline shapes.
 */
#include "pic_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* stagger bits (x, y, z) of Ex, Ey, Ez, Bx, By, Bz; J uses the first three */
static const int STAG[6][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {0, 1, 1}, {1, 0, 1}, {1, 1, 0}};

struct orc_sim {
    orc_config c;
    long long ncell;
    double* E[3];
    double* Bh[3]; /* B^{n+1/2} */
    double* Bn[3]; /* B^n, used by the push */
    double* J[3];
    double* rho_bg;
    long long np, cap;
    double *x, *y, *z, *ux, *uy, *uz, *w;
    int* id;
    long long step, nshift, next_id;
    long long* mlast;  /* per patch: count after its last merge pass (0 = none yet) */
    long long mlast_n;
};

/* ------------------------------------------------------------------ helpers */

static long wrap(long i, long n) {
    if (i < 0) i += n;
    else if (i >= n) i -= n;
    if (i < 0 || i >= n) i = ((i % n) + n) % n;  /* more than one period away */
    return i;
}

/* flat index of (i, j, k) with the boundary rule; -1 = outside a window x axis */
static long long flat(const orc_config* c, long i, long j, long k) {
    if (c->window) {
        if (i < 0 || i >= c->n[0]) return -1;
    } else {
        i = wrap(i, c->n[0]);
    }
    j = wrap(j, c->n[1]);
    k = wrap(k, c->n[2]);
    return ((long long)k * c->n[1] + j) * c->n[0] + i;
}

static double at(const orc_config* c, const double* a, long i, long j, long k) {
    long long t = flat(c, i, j, k);
    return t < 0 ? 0.0 : a[t];
}

static void add_at(const orc_config* c, double* a, long i, long j, long k, double v) {
    long long t = flat(c, i, j, k);
    if (t >= 0) a[t] += v;
}

/* Index along the slowest array axis (y in 2D, z in 3D; always a periodic axis) of
 * flat index t. */
static long slow_index(const orc_config* c, long long t) {
    return c->dims == 3 ? (long)(t / ((long long)c->n[0] * c->n[1])) : (long)(t / c->n[0]);
}

static long slow_extent(const orc_config* c) { return c->dims == 3 ? c->n[2] : c->n[1]; }

/* add_at restricted to the elements whose slow-axis index lies in [band[0], band[1]).
 * The plain step passes the whole axis, so it is add_at; the threaded step gives each
 * thread its own band of the current, so every element still receives the same
 * additions in the same order. */
static void add_band(const orc_config* c, const long band[2], double* a, long i, long j,
                     long k, double v) {
    long long t = flat(c, i, j, k);
    if (t < 0) return;
    long sl = slow_index(c, t);
    if (sl >= band[0] && sl < band[1]) a[t] += v;
}

long long orc_shift_count(const orc_config* c, long long step) {
    return (long long)floor((double)step * c->dt / c->d[0]);
}

/* ------------------------------------------------------------------ shapes */

long orc_shape2(double xi, double S[3]) {
    double node = floor(xi + 0.5);
    double delta = xi - node; /* in [-1/2, 1/2] */
    S[0] = 0.5 * (0.5 - delta) * (0.5 - delta);
    S[1] = 0.75 - delta * delta;
    S[2] = 0.5 * (0.5 + delta) * (0.5 + delta);
    return (long)node;
}

/* ------------------------------------------------------------------ Boris */

void orc_boris(double q, double m, double dt, const double E[3], const double B[3],
               double u[3]) {
    double eps = q * dt / (2.0 * m);
    double um[3], t[3], s[3], up[3], uq[3];
    for (int a = 0; a < 3; a++) um[a] = u[a] + eps * E[a];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int a = 0; a < 3; a++) t[a] = eps * B[a] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int a = 0; a < 3; a++) s[a] = 2.0 * t[a] / (1.0 + t2);
    /* u' = u- + u- x t */
    up[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);
    up[1] = um[1] + (um[2] * t[0] - um[0] * t[2]);
    up[2] = um[2] + (um[0] * t[1] - um[1] * t[0]);
    /* u+ = u- + u' x s */
    uq[0] = um[0] + (up[1] * s[2] - up[2] * s[1]);
    uq[1] = um[1] + (up[2] * s[0] - up[0] * s[2]);
    uq[2] = um[2] + (up[0] * s[1] - up[1] * s[0]);
    for (int a = 0; a < 3; a++) u[a] = uq[a] + eps * E[a];
}

/* ------------------------------------------------------------------ interpolation */

void orc_interp(const orc_config* c, const double* const F[6], const double pos[3],
                double out[6]) {
    for (int comp = 0; comp < 6; comp++) {
        long node[3] = {0, 0, 0};
        double S[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
        for (int a = 0; a < c->dims; a++) {
            double xi = pos[a] / c->d[a] - 0.5 * STAG[comp][a];
            node[a] = orc_shape2(xi, S[a]);
        }
        int kz = c->dims == 3 ? 1 : 0;
        double sum = 0.0;
        for (int k = -kz; k <= kz; k++)
            for (int j = -1; j <= 1; j++)
                for (int i = -1; i <= 1; i++)
                    sum += S[0][i + 1] * S[1][j + 1] * S[2][k + 1] *
                           at(c, F[comp], node[0] + i, node[1] + j, node[2] + k);
        out[comp] = sum;
    }
}

/* ------------------------------------------------------------------ Esirkepov */

/* S0, S1 on the five primal nodes node0-2 .. node0+2 around the old nearest node;
 * returns 0, or -1 if the particle moved by more than one node. */
static int esirkepov_shapes(double xi0, double xi1, long* node0, double S0[5],
                            double DS[5]) {
    double s[3], S1[5] = {0, 0, 0, 0, 0};
    *node0 = orc_shape2(xi0, s);
    S0[0] = 0.0;
    S0[1] = s[0];
    S0[2] = s[1];
    S0[3] = s[2];
    S0[4] = 0.0;
    long node1 = orc_shape2(xi1, s);
    long shift = node1 - *node0;
    if (shift < -1 || shift > 1) return -1;
    for (int b = 0; b < 3; b++) S1[shift + 1 + b] = s[b];
    for (int k = 0; k < 5; k++) DS[k] = S1[k] - S0[k];
    return 0;
}

static int deposit2d(const orc_config* c, const double pos0[3], const double pos1[3],
                     double vz, double qw, double* const J[3], const long band[2]) {
    long n0[2];
    double S0[2][5], DS[2][5];
    for (int a = 0; a < 2; a++)
        if (esirkepov_shapes(pos0[a] / c->d[a], pos1[a] / c->d[a], &n0[a], S0[a], DS[a]))
            return -1;
    double dV = c->d[0] * c->d[1];
    double cx = -qw / dV * c->d[0] / c->dt;
    double cy = -qw / dV * c->d[1] / c->dt;
    double cz = qw / dV * vz;
    /* Jx at (i+1/2, j): running sum of Wx = DSx (S0y + DSy/2) along +x */
    for (int l = 0; l < 5; l++) {
        double acc = 0.0;
        for (int k = 0; k < 4; k++) {
            acc += DS[0][k] * (S0[1][l] + 0.5 * DS[1][l]);
            add_band(c, band, J[0], n0[0] + k - 2, n0[1] + l - 2, 0, cx * acc);
        }
    }
    /* Jy at (i, j+1/2): running sum of Wy = DSy (S0x + DSx/2) along +y */
    for (int k = 0; k < 5; k++) {
        double acc = 0.0;
        for (int l = 0; l < 4; l++) {
            acc += DS[1][l] * (S0[0][k] + 0.5 * DS[0][k]);
            add_band(c, band, J[1], n0[0] + k - 2, n0[1] + l - 2, 0, cy * acc);
        }
    }
    /* Jz at nodes: vz times the path-averaged shape Wz */
    for (int l = 0; l < 5; l++)
        for (int k = 0; k < 5; k++) {
            double wz = S0[0][k] * S0[1][l] + 0.5 * DS[0][k] * S0[1][l] +
                        0.5 * S0[0][k] * DS[1][l] + DS[0][k] * DS[1][l] / 3.0;
            add_band(c, band, J[2], n0[0] + k - 2, n0[1] + l - 2, 0, cz * wz);
        }
    return 0;
}

/* 3D: W_a = DS_a (S0_b S0_c + DS_b S0_c/2 + S0_b DS_c/2 + DS_b DS_c/3) for the two
 * other axes b, c; J_a is the running sum of -(qw/dV)(d_a/dt) W_a along +a. */
static int deposit3d(const orc_config* c, const double pos0[3], const double pos1[3],
                     double qw, double* const J[3], const long band[2]) {
    long n0[3];
    double S0[3][5], DS[3][5];
    for (int a = 0; a < 3; a++)
        if (esirkepov_shapes(pos0[a] / c->d[a], pos1[a] / c->d[a], &n0[a], S0[a], DS[a]))
            return -1;
    double dV = c->d[0] * c->d[1] * c->d[2];
    for (int a = 0; a < 3; a++) {
        int b = (a + 1) % 3, e = (a + 2) % 3;
        double coef = -qw / dV * c->d[a] / c->dt;
        for (int ie = 0; ie < 5; ie++)
            for (int ib = 0; ib < 5; ib++) {
                double acc = 0.0;
                for (int ia = 0; ia < 4; ia++) {
                    double w = DS[a][ia] *
                               (S0[b][ib] * S0[e][ie] + 0.5 * DS[b][ib] * S0[e][ie] +
                                0.5 * S0[b][ib] * DS[e][ie] + DS[b][ib] * DS[e][ie] / 3.0);
                    acc += w;
                    long idx[3];
                    idx[a] = n0[a] + ia - 2;
                    idx[b] = n0[b] + ib - 2;
                    idx[e] = n0[e] + ie - 2;
                    add_band(c, band, J[a], idx[0], idx[1], idx[2], coef * acc);
                }
            }
    }
    return 0;
}

void orc_deposit(const orc_config* c, const double pos0[3], const double pos1[3],
                 double vz, double qw, double* const J[3]) {
    const long all[2] = {0, slow_extent(c)};
    if (c->dims == 2)
        deposit2d(c, pos0, pos1, vz, qw, J, all);
    else
        deposit3d(c, pos0, pos1, qw, J, all);
}

void orc_rho(const orc_config* c, long long n, const double* x, const double* y,
             const double* z, const double* w, double q, double* rho) {
    double dV = c->d[0] * c->d[1] * (c->dims == 3 ? c->d[2] : 1.0);
    for (long long p = 0; p < n; p++) {
        double pos[3] = {x[p], y[p], c->dims == 3 ? z[p] : 0.0};
        long node[3] = {0, 0, 0};
        double S[3][3] = {{0, 1, 0}, {0, 1, 0}, {0, 1, 0}};
        for (int a = 0; a < c->dims; a++) node[a] = orc_shape2(pos[a] / c->d[a], S[a]);
        int kz = c->dims == 3 ? 1 : 0;
        for (int k = -kz; k <= kz; k++)
            for (int j = -1; j <= 1; j++)
                for (int i = -1; i <= 1; i++)
                    add_at(c, rho, node[0] + i, node[1] + j, node[2] + k,
                           q * w[p] / dV * S[0][i + 1] * S[1][j + 1] * S[2][k + 1]);
    }
}

/* ------------------------------------------------------------------ Yee */

/* Coefficients c_l of the staggered first difference of the configured order.
 * Order 2: c_1 = 1 (Yee 1966). Order 6: the c_l solving
 *   sum_l c_l (2l - 1)^(2m+1) = [m == 0],  m = 0, 1, 2,
 * i.e. the Taylor conditions that make the difference exact up to degree 6:
 * 75/64, -25/384, 3/640. Returns the number of terms. */
static int stag_coef(const orc_config* c, const double** coef) {
    static const double C2[1] = {1.0};
    static const double C6[3] = {75.0 / 64.0, -25.0 / 384.0, 3.0 / 640.0};
    if (c->order == 6) {
        *coef = C6;
        return 3;
    }
    *coef = C2;
    return 1;
}

/* d/dx_a of F at the integer position (i, j, k) from values at the half-integer
 * positions below it: F stored at index m sits at m + 1/2 along axis a, so the
 * difference pairs are F(m = i + l - 1) and F(m = i - l). */
static double dminus(const orc_config* c, const double* F, int a, long i, long j, long k) {
    const double* cf;
    int R = stag_coef(c, &cf);
    double s = 0.0;
    for (int l = 1; l <= R; l++) {
        long p[3] = {i, j, k}, m[3] = {i, j, k};
        p[a] += l - 1;
        m[a] -= l;
        s += cf[l - 1] * (at(c, F, p[0], p[1], p[2]) - at(c, F, m[0], m[1], m[2]));
    }
    return s / c->d[a];
}

/* d/dx_a of F at the half-integer position (i + 1/2) along axis a from values at the
 * integer positions: pairs F(i + l) and F(i - l + 1). */
static double dplus(const orc_config* c, const double* F, int a, long i, long j, long k) {
    const double* cf;
    int R = stag_coef(c, &cf);
    double s = 0.0;
    for (int l = 1; l <= R; l++) {
        long p[3] = {i, j, k}, m[3] = {i, j, k};
        p[a] += l;
        m[a] -= l - 1;
        s += cf[l - 1] * (at(c, F, p[0], p[1], p[2]) - at(c, F, m[0], m[1], m[2]));
    }
    return s / c->d[a];
}

/* The field updates over the cells whose slow-axis index lies in [lo, hi) (the whole
 * grid for the plain step; one band per thread for the threaded one: every cell's new
 * value depends only on the old arrays, so the bands are independent). */
static void yee_e_band(const orc_config* c, double* const E[3], const double* const B[3],
                       const double* const J[3], long lo, long hi) {
    double dt = c->dt;
    int d3 = c->dims == 3;
    long k0 = d3 ? lo : 0, k1 = d3 ? hi : 1, j0 = d3 ? 0 : lo, j1 = d3 ? c->n[1] : hi;
    for (long k = k0; k < k1; k++)
        for (long j = j0; j < j1; j++)
            for (long i = 0; i < c->n[0]; i++) {
                long long t = flat(c, i, j, k);
                const double *Bx = B[0], *By = B[1], *Bz = B[2];
                /* curl B at the E positions: each derivative crosses the stagger of
                   the B component along its own axis */
                double cx = dminus(c, Bz, 1, i, j, k);
                double cy = -dminus(c, Bz, 0, i, j, k);
                double cz = dminus(c, By, 0, i, j, k) - dminus(c, Bx, 1, i, j, k);
                if (d3) {
                    cx -= dminus(c, By, 2, i, j, k);
                    cy += dminus(c, Bx, 2, i, j, k);
                }
                E[0][t] += dt * (cx - J[0][t]);
                E[1][t] += dt * (cy - J[1][t]);
                E[2][t] += dt * (cz - J[2][t]);
            }
}

void orc_yee_e(const orc_config* c, double* const E[3], const double* const B[3],
               const double* const J[3]) {
    yee_e_band(c, E, B, J, 0, slow_extent(c));
}

static void yee_b_band(const orc_config* c, const double* const E[3], double* const B[3],
                       long lo, long hi) {
    double dt = c->dt;
    int d3 = c->dims == 3;
    long k0 = d3 ? lo : 0, k1 = d3 ? hi : 1, j0 = d3 ? 0 : lo, j1 = d3 ? c->n[1] : hi;
    for (long k = k0; k < k1; k++)
        for (long j = j0; j < j1; j++)
            for (long i = 0; i < c->n[0]; i++) {
                long long t = flat(c, i, j, k);
                const double *Ex = E[0], *Ey = E[1], *Ez = E[2];
                double cx = dplus(c, Ez, 1, i, j, k);
                double cy = -dplus(c, Ez, 0, i, j, k);
                double cz = dplus(c, Ey, 0, i, j, k) - dplus(c, Ex, 1, i, j, k);
                if (d3) {
                    cx -= dplus(c, Ey, 2, i, j, k);
                    cy += dplus(c, Ex, 2, i, j, k);
                }
                B[0][t] -= dt * cx;
                B[1][t] -= dt * cy;
                B[2][t] -= dt * cz;
            }
}

void orc_yee_b(const orc_config* c, const double* const E[3], double* const B[3]) {
    yee_b_band(c, E, B, 0, slow_extent(c));
}

void orc_div_e(const orc_config* c, const double* const E[3], double* out) {
    for (long k = 0; k < c->n[2]; k++)
        for (long j = 0; j < c->n[1]; j++)
            for (long i = 0; i < c->n[0]; i++) {
                double v = (at(c, E[0], i, j, k) - at(c, E[0], i - 1, j, k)) / c->d[0] +
                           (at(c, E[1], i, j, k) - at(c, E[1], i, j - 1, k)) / c->d[1];
                if (c->dims == 3)
                    v += (at(c, E[2], i, j, k) - at(c, E[2], i, j, k - 1)) / c->d[2];
                out[flat(c, i, j, k)] = v;
            }
}

/* ------------------------------------------------------------------ simulation */

static int valid_config(const orc_config* c) {
    if (c->dims != 2 && c->dims != 3) return 0;
    if (c->dims == 2 && c->n[2] != 1) return 0;
    for (int a = 0; a < c->dims; a++)
        if (c->n[a] < 1 || !(c->d[a] > 0)) return 0;
    if (!(c->dt > 0) || !(c->m > 0)) return 0;
    for (int a = 0; a < c->dims; a++)
        if (c->dt >= c->d[a]) return 0; /* displacement must stay below one cell */
    if (c->order != 0 && c->order != 2 && c->order != 6) return 0;
    return 1;
}

orc_sim* orc_create(const orc_config* c, long long capacity) {
    if (!valid_config(c) || capacity < 0) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->c = *c;
    s->ncell = (long long)c->n[0] * c->n[1] * c->n[2];
    for (int a = 0; a < 3; a++) {
        s->E[a] = (double*)calloc(s->ncell, sizeof(double));
        s->Bh[a] = (double*)calloc(s->ncell, sizeof(double));
        s->Bn[a] = (double*)calloc(s->ncell, sizeof(double));
        s->J[a] = (double*)calloc(s->ncell, sizeof(double));
    }
    s->rho_bg = (double*)calloc(s->ncell, sizeof(double));
    s->cap = capacity;
    long long m = capacity > 0 ? capacity : 1;
    s->x = (double*)calloc(m, sizeof(double));
    s->y = (double*)calloc(m, sizeof(double));
    s->z = (double*)calloc(m, sizeof(double));
    s->ux = (double*)calloc(m, sizeof(double));
    s->uy = (double*)calloc(m, sizeof(double));
    s->uz = (double*)calloc(m, sizeof(double));
    s->w = (double*)calloc(m, sizeof(double));
    s->id = (int*)calloc(m, sizeof(int));
    return s;
}

void orc_destroy(orc_sim* s) {
    if (!s) return;
    for (int a = 0; a < 3; a++) {
        free(s->E[a]);
        free(s->Bh[a]);
        free(s->Bn[a]);
        free(s->J[a]);
    }
    free(s->rho_bg);
    free(s->mlast);
    free(s->x);
    free(s->y);
    free(s->z);
    free(s->ux);
    free(s->uy);
    free(s->uz);
    free(s->w);
    free(s->id);
    free(s);
}

int orc_set_particles(orc_sim* s, long long n, const double* x, const double* y,
                      const double* z, const double* ux, const double* uy,
                      const double* uz, const double* w, const int* id) {
    if (n < 0 || n > s->cap) return -1;
    s->np = n;
    if (s->mlast)  /* a new particle set: no patch has been merged yet */
        for (long long q = 0; q < s->mlast_n; q++) s->mlast[q] = 0;
    int maxid = -1;
    for (long long p = 0; p < n; p++) {
        s->x[p] = x[p];
        s->y[p] = y[p];
        s->z[p] = z ? z[p] : 0.0;
        s->ux[p] = ux[p];
        s->uy[p] = uy[p];
        s->uz[p] = uz[p];
        s->w[p] = w[p];
        s->id[p] = id[p];
        if (id[p] > maxid) maxid = id[p];
    }
    s->next_id = (long long)maxid + 1;
    return 0;
}

long long orc_num_particles(const orc_sim* s) { return s->np; }
long long orc_steps_done(const orc_sim* s) { return s->step; }
long long orc_shifts_done(const orc_sim* s) { return s->nshift; }

int orc_get_particles(const orc_sim* s, double* x, double* y, double* z, double* ux,
                      double* uy, double* uz, double* w, int* id) {
    for (long long p = 0; p < s->np; p++) {
        x[p] = s->x[p];
        y[p] = s->y[p];
        z[p] = s->z[p];
        ux[p] = s->ux[p];
        uy[p] = s->uy[p];
        uz[p] = s->uz[p];
        w[p] = s->w[p];
        id[p] = s->id[p];
    }
    return 0;
}

int orc_set_fields(orc_sim* s, const double* Ex, const double* Ey, const double* Ez,
                   const double* Bx, const double* By, const double* Bz) {
    const double* E[3] = {Ex, Ey, Ez};
    const double* B[3] = {Bx, By, Bz};
    size_t bytes = (size_t)s->ncell * sizeof(double);
    for (int a = 0; a < 3; a++) {
        memcpy(s->E[a], E[a], bytes);
        memcpy(s->Bh[a], B[a], bytes);
        memcpy(s->Bn[a], B[a], bytes);
    }
    return 0;
}

int orc_get_fields(const orc_sim* s, double* out12) {
    size_t nc = (size_t)s->ncell;
    for (int a = 0; a < 3; a++) {
        memcpy(out12 + (0 + a) * nc, s->E[a], nc * sizeof(double));
        memcpy(out12 + (3 + a) * nc, s->Bh[a], nc * sizeof(double));
        memcpy(out12 + (6 + a) * nc, s->Bn[a], nc * sizeof(double));
        memcpy(out12 + (9 + a) * nc, s->J[a], nc * sizeof(double));
    }
    return 0;
}

int orc_set_rho_bg(orc_sim* s, const double* rho_bg) {
    if (rho_bg) {
        memcpy(s->rho_bg, rho_bg, (size_t)s->ncell * sizeof(double));
    } else {
        memset(s->rho_bg, 0, (size_t)s->ncell * sizeof(double));
        orc_rho(&s->c, s->np, s->x, s->y, s->z, s->w, s->c.q, s->rho_bg);
        for (long long t = 0; t < s->ncell; t++) s->rho_bg[t] = -s->rho_bg[t];
    }
    return 0;
}

/* stable compaction: keep particle p iff keep[p] != 0 */
static void compact(orc_sim* s, const unsigned char* keep) {
    long long o = 0;
    for (long long p = 0; p < s->np; p++) {
        if (!keep[p]) continue;
        s->x[o] = s->x[p];
        s->y[o] = s->y[p];
        s->z[o] = s->z[p];
        s->ux[o] = s->ux[p];
        s->uy[o] = s->uy[p];
        s->uz[o] = s->uz[p];
        s->w[o] = s->w[p];
        s->id[o] = s->id[p];
        o++;
    }
    s->np = o;
}

static double density(const orc_config* c, double x_lab) {
    double f = (x_lab - c->ramp_x0) / c->ramp_len;
    if (f < 0.0) f = 0.0;
    if (f > 1.0) f = 1.0;
    return c->n0 * f;
}

/* Window shift by one cell: fields move one cell towards -x, the uncovered column
 * is zero; particles move by -dx, those with x < 0 are dropped; the new rightmost
 * cell column is filled with a cold lattice weighted by the lab-frame density. */
static int window_shift(orc_sim* s) {
    const orc_config* c = &s->c;
    long nx = c->n[0], ny = c->n[1], nz = c->n[2];
    double* arrays[9] = {s->E[0], s->E[1], s->E[2], s->Bh[0], s->Bh[1],
                         s->Bh[2], s->Bn[0], s->Bn[1], s->Bn[2]};
    for (int a = 0; a < 9; a++)
        for (long k = 0; k < nz; k++)
            for (long j = 0; j < ny; j++) {
                double* row = arrays[a] + ((long long)k * ny + j) * nx;
                for (long i = 0; i < nx - 1; i++) row[i] = row[i + 1];
                row[nx - 1] = 0.0;
            }
    s->nshift++;
    unsigned char* keep = (unsigned char*)malloc((size_t)(s->np > 0 ? s->np : 1));
    for (long long p = 0; p < s->np; p++) {
        s->x[p] -= c->d[0];
        keep[p] = s->x[p] >= 0.0;
    }
    compact(s, keep);
    free(keep);
    int px = c->inject_ppc[0], py = c->inject_ppc[1];
    int pz = c->dims == 3 ? c->inject_ppc[2] : 1;
    long nzz = c->dims == 3 ? nz : 1;
    double dV = c->d[0] * c->d[1] * (c->dims == 3 ? c->d[2] : 1.0);
    double ppc = (double)px * py * pz;
    for (long k = 0; k < nzz; k++)
        for (long j = 0; j < ny; j++)
            for (int cz = 0; cz < pz; cz++)
                for (int b = 0; b < py; b++)
                    for (int a = 0; a < px; a++) {
                        double xw = ((double)(nx - 1) + ((double)a + 0.5) / px) * c->d[0];
                        double xl = xw + (double)s->nshift * c->d[0];
                        double dens = density(c, xl);
                        if (!(dens > 0.0)) continue;
                        if (s->np >= s->cap) return -1;
                        long long lat = (((long long)(k * ny + j) * pz + cz) * py + b) * px + a;
                        long long p = s->np++;
                        s->x[p] = xw;
                        s->y[p] = ((double)j + ((double)b + 0.5) / py) * c->d[1];
                        s->z[p] = c->dims == 3
                                      ? ((double)k + ((double)cz + 0.5) / pz) * c->d[2]
                                      : 0.0;
                        s->ux[p] = s->uy[p] = s->uz[p] = 0.0;
                        s->w[p] = dens * dV / ppc;
                        s->id[p] = (int)(s->next_id + lat);
                    }
    s->next_id += (long long)nzz * ny * pz * py * px;
    return 0;
}

static void wrap_pos(double* v, double L) {
    if (*v < 0.0) *v += L;
    if (*v >= L) *v -= L;
}

int orc_step(orc_sim* s, int nsteps) {
    const orc_config* c = &s->c;
    int dims = c->dims;
    double L[3] = {c->n[0] * c->d[0], c->n[1] * c->d[1], c->n[2] * c->d[2]};
    double* Bold[3];
    for (int a = 0; a < 3; a++) Bold[a] = (double*)malloc((size_t)s->ncell * sizeof(double));
    const long all[2] = {0, slow_extent(c)};
    int rc = 0;
    for (int it = 0; it < nsteps && rc == 0; it++) {
        for (int a = 0; a < 3; a++) memset(s->J[a], 0, (size_t)s->ncell * sizeof(double));
        const double* F[6] = {s->E[0], s->E[1], s->E[2], s->Bn[0], s->Bn[1], s->Bn[2]};
        for (long long p = 0; p < s->np; p++) {
            double pos0[3] = {s->x[p], s->y[p], s->z[p]};
            double EB[6];
            orc_interp(c, F, pos0, EB);
            double u[3] = {s->ux[p], s->uy[p], s->uz[p]};
            orc_boris(c->q, c->m, c->dt, EB, EB + 3, u);
            double gamma = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
            double pos1[3] = {pos0[0], pos0[1], pos0[2]};
            for (int a = 0; a < dims; a++) pos1[a] = pos0[a] + c->dt * u[a] / gamma;
            int bad = dims == 2 ? deposit2d(c, pos0, pos1, u[2] / gamma, c->q * s->w[p], s->J, all)
                                : deposit3d(c, pos0, pos1, c->q * s->w[p], s->J, all);
            if (bad) rc = -2;
            s->x[p] = pos1[0];
            s->y[p] = pos1[1];
            s->z[p] = pos1[2];
            s->ux[p] = u[0];
            s->uy[p] = u[1];
            s->uz[p] = u[2];
        }
        unsigned char* keep = (unsigned char*)malloc((size_t)(s->np > 0 ? s->np : 1));
        for (long long p = 0; p < s->np; p++) {
            keep[p] = 1;
            if (c->window)
                keep[p] = s->x[p] >= 0.0 && s->x[p] < L[0];
            else
                wrap_pos(&s->x[p], L[0]);
            wrap_pos(&s->y[p], L[1]);
            if (dims == 3) wrap_pos(&s->z[p], L[2]);
        }
        compact(s, keep);
        free(keep);
        orc_yee_e(c, s->E, (const double* const*)s->Bh, (const double* const*)s->J);
        for (int a = 0; a < 3; a++) memcpy(Bold[a], s->Bh[a], (size_t)s->ncell * sizeof(double));
        orc_yee_b(c, (const double* const*)s->E, s->Bh);
        for (int a = 0; a < 3; a++)
            for (long long t = 0; t < s->ncell; t++) s->Bn[a][t] = 0.5 * (Bold[a][t] + s->Bh[a][t]);
        s->step++;
        if (c->window && orc_shift_count(c, s->step) > orc_shift_count(c, s->step - 1))
            if (window_shift(s)) rc = -3;
    }
    for (int a = 0; a < 3; a++) free(Bold[a]);
    return rc;
}

/* ------------------------------------------------------------------ threaded step
 *
 * orc_step_mt computes exactly what orc_step computes, on several host threads, with
 * results identical bit for bit (it is the oracle's all-core timing and long-run
 * form; tests check the identity). Each phase of the step is split so that no value
 * is summed in a different order:
 *   - the particle update (interpolation, Boris, move) is independent per particle:
 *     threads take contiguous particle ranges;
 *   - the current: thread t owns a band of rows along the slowest axis of J (y in 2D,
 *     z in 3D) and walks ALL particles in index order, depositing only into its band.
 *     Every element of J thus receives the same additions in the same order as in the
 *     single-thread loop (per-thread copies of J summed afterwards would not: the
 *     association of the sums would change);
 *   - the field updates are independent per cell: threads take bands;
 *   - particle boundaries, the window shift and the diagnostics stay single-threaded. */

#define ORC_MAX_THREADS 256

typedef struct {
    void (*fn)(void*, int, int);
    void* arg;
    int tid, nt;
} par_job;

static void* par_entry(void* p) {
    par_job* j = (par_job*)p;
    j->fn(j->arg, j->tid, j->nt);
    return NULL;
}

/* runs fn(arg, t, nt) for t = 0..nt-1, thread 0 on the calling thread */
static void par_run(int nt, void (*fn)(void*, int, int), void* arg) {
    pthread_t th[ORC_MAX_THREADS];
    par_job job[ORC_MAX_THREADS];
    int started[ORC_MAX_THREADS];
    for (int t = 0; t < nt; t++) {
        job[t].fn = fn;
        job[t].arg = arg;
        job[t].tid = t;
        job[t].nt = nt;
        started[t] = 0;
    }
    for (int t = 1; t < nt; t++)
        started[t] = pthread_create(&th[t], NULL, par_entry, &job[t]) == 0;
    fn(arg, 0, nt);
    for (int t = 1; t < nt; t++) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            fn(arg, t, nt); /* no thread: do its share here */
    }
}

static void range_of(long long n, int t, int nt, long long* lo, long long* hi) {
    *lo = n * t / nt;
    *hi = n * (t + 1) / nt;
}

typedef struct {
    orc_sim* s;
    double *x0, *y0, *z0, *vz, *qw; /* per particle: old position, v_z, q w */
    double* Bold[3];
    int bad;                        /* a particle moved by more than one node */
} mt_ctx;

static void mt_push(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    orc_sim* s = m->s;
    const orc_config* c = &s->c;
    const double* F[6] = {s->E[0], s->E[1], s->E[2], s->Bn[0], s->Bn[1], s->Bn[2]};
    long long lo, hi;
    range_of(s->np, t, nt, &lo, &hi);
    for (long long p = lo; p < hi; p++) {
        double pos0[3] = {s->x[p], s->y[p], s->z[p]};
        double EB[6];
        orc_interp(c, F, pos0, EB);
        double u[3] = {s->ux[p], s->uy[p], s->uz[p]};
        orc_boris(c->q, c->m, c->dt, EB, EB + 3, u);
        double gamma = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double pos1[3] = {pos0[0], pos0[1], pos0[2]};
        for (int a2 = 0; a2 < c->dims; a2++) pos1[a2] = pos0[a2] + c->dt * u[a2] / gamma;
        m->x0[p] = pos0[0];
        m->y0[p] = pos0[1];
        m->z0[p] = pos0[2];
        m->vz[p] = u[2] / gamma;
        m->qw[p] = c->q * s->w[p];
        s->x[p] = pos1[0];
        s->y[p] = pos1[1];
        s->z[p] = pos1[2];
        s->ux[p] = u[0];
        s->uy[p] = u[1];
        s->uz[p] = u[2];
    }
}

static void mt_deposit(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    orc_sim* s = m->s;
    const orc_config* c = &s->c;
    const int sa = c->dims == 3 ? 2 : 1; /* slow axis */
    const long ns = slow_extent(c);
    long long lo, hi;
    range_of(ns, t, nt, &lo, &hi);
    const long band[2] = {(long)lo, (long)hi};
    if (lo >= hi) return;
    int bad = 0;
    for (long long p = 0; p < s->np; p++) {
        const double pos0[3] = {m->x0[p], m->y0[p], m->z0[p]};
        /* the deposit touches slow-axis nodes node0 - 2 .. node0 + 2 (wrapped) */
        const long node0 = (long)floor(pos0[sa] / c->d[sa] + 0.5);
        int touches = 0;
        for (long r = node0 - 2; r <= node0 + 2 && !touches; r++) {
            long rw = wrap(r, ns);
            touches = rw >= band[0] && rw < band[1];
        }
        if (!touches) continue;
        const double pos1[3] = {s->x[p], s->y[p], s->z[p]};
        int b = c->dims == 2 ? deposit2d(c, pos0, pos1, m->vz[p], m->qw[p], s->J, band)
                             : deposit3d(c, pos0, pos1, m->qw[p], s->J, band);
        if (b) bad = 1;
    }
    if (bad) m->bad = 1; /* every writer stores the same value */
}

static void mt_zero_j(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    long long lo, hi;
    range_of(m->s->ncell, t, nt, &lo, &hi);
    for (int k = 0; k < 3; k++)
        memset(m->s->J[k] + lo, 0, (size_t)(hi - lo) * sizeof(double));
}

static void mt_yee_e(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    orc_sim* s = m->s;
    long long lo, hi;
    range_of(slow_extent(&s->c), t, nt, &lo, &hi);
    yee_e_band(&s->c, s->E, (const double* const*)s->Bh, (const double* const*)s->J, (long)lo,
               (long)hi);
    /* keep B^{n+1/2} for the average (the cells of this band only) */
    long long c0 = lo * (s->ncell / slow_extent(&s->c)), c1 = hi * (s->ncell / slow_extent(&s->c));
    for (int k = 0; k < 3; k++)
        memcpy(m->Bold[k] + c0, s->Bh[k] + c0, (size_t)(c1 - c0) * sizeof(double));
}

static void mt_yee_b(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    orc_sim* s = m->s;
    long long lo, hi;
    range_of(slow_extent(&s->c), t, nt, &lo, &hi);
    yee_b_band(&s->c, (const double* const*)s->E, s->Bh, (long)lo, (long)hi);
}

static void mt_average(void* a, int t, int nt) {
    mt_ctx* m = (mt_ctx*)a;
    orc_sim* s = m->s;
    long long lo, hi;
    range_of(s->ncell, t, nt, &lo, &hi);
    for (int k = 0; k < 3; k++)
        for (long long i = lo; i < hi; i++) s->Bn[k][i] = 0.5 * (m->Bold[k][i] + s->Bh[k][i]);
}

int orc_step_mt(orc_sim* s, int nsteps, int nthreads) {
    const orc_config* c = &s->c;
    int nt = nthreads < 1 ? 1 : (nthreads > ORC_MAX_THREADS ? ORC_MAX_THREADS : nthreads);
    if (nt > slow_extent(c)) nt = (int)slow_extent(c);
    double L[3] = {c->n[0] * c->d[0], c->n[1] * c->d[1], c->n[2] * c->d[2]};
    mt_ctx m;
    memset(&m, 0, sizeof m);
    m.s = s;
    long long cap = s->cap > 0 ? s->cap : 1;
    m.x0 = (double*)malloc((size_t)cap * sizeof(double));
    m.y0 = (double*)malloc((size_t)cap * sizeof(double));
    m.z0 = (double*)malloc((size_t)cap * sizeof(double));
    m.vz = (double*)malloc((size_t)cap * sizeof(double));
    m.qw = (double*)malloc((size_t)cap * sizeof(double));
    for (int a = 0; a < 3; a++) m.Bold[a] = (double*)malloc((size_t)s->ncell * sizeof(double));
    int rc = 0;
    if (!m.x0 || !m.y0 || !m.z0 || !m.vz || !m.qw || !m.Bold[0] || !m.Bold[1] || !m.Bold[2])
        rc = -4;
    for (int it = 0; it < nsteps && rc == 0; it++) {
        par_run(nt, mt_zero_j, &m);
        par_run(nt, mt_push, &m);
        m.bad = 0;
        par_run(nt, mt_deposit, &m);
        if (m.bad) rc = -2;
        /* particle boundaries: as in orc_step */
        unsigned char* keep = (unsigned char*)malloc((size_t)(s->np > 0 ? s->np : 1));
        for (long long p = 0; p < s->np; p++) {
            keep[p] = 1;
            if (c->window)
                keep[p] = s->x[p] >= 0.0 && s->x[p] < L[0];
            else
                wrap_pos(&s->x[p], L[0]);
            wrap_pos(&s->y[p], L[1]);
            if (c->dims == 3) wrap_pos(&s->z[p], L[2]);
        }
        compact(s, keep);
        free(keep);
        par_run(nt, mt_yee_e, &m);
        par_run(nt, mt_yee_b, &m);
        par_run(nt, mt_average, &m);
        s->step++;
        if (c->window && orc_shift_count(c, s->step) > orc_shift_count(c, s->step - 1))
            if (window_shift(s)) rc = -3;
    }
    free(m.x0), free(m.y0), free(m.z0), free(m.vz), free(m.qw);
    for (int a = 0; a < 3; a++) free(m.Bold[a]);
    return rc;
}

void orc_energy(const orc_sim* s, double out[3]) {
    const orc_config* c = &s->c;
    double dV = c->d[0] * c->d[1] * (c->dims == 3 ? c->d[2] : 1.0);
    double we = 0, wb = 0, wk = 0;
    for (long long t = 0; t < s->ncell; t++) {
        for (int a = 0; a < 3; a++) {
            we += s->E[a][t] * s->E[a][t];
            wb += s->Bn[a][t] * s->Bn[a][t];
        }
    }
    for (long long p = 0; p < s->np; p++) {
        double g = sqrt(1.0 + s->ux[p] * s->ux[p] + s->uy[p] * s->uy[p] + s->uz[p] * s->uz[p]);
        wk += s->w[p] * c->m * (g - 1.0);
    }
    out[0] = 0.5 * we * dV;
    out[1] = 0.5 * wb * dV;
    out[2] = wk;
}

void orc_gauss(const orc_sim* s, double* out) {
    const orc_config* c = &s->c;
    double* rho = (double*)calloc((size_t)s->ncell, sizeof(double));
    orc_rho(c, s->np, s->x, s->y, s->z, s->w, c->q, rho);
    orc_div_e(c, (const double* const*)s->E, out);
    for (long long t = 0; t < s->ncell; t++) out[t] -= rho[t] + s->rho_bg[t];
    free(rho);
}

/* ------------------------------------------------------------------ merging */

int orc_merge_group(long long n, const double* ux, const double* uy, const double* uz,
                    const double* w, const int* id, double out_u[6], double* out_w,
                    long long keep[2]) {
    if (n < 3) return 0;
    /* the two smallest ids */
    long long a = -1, b = -1;
    for (long long k = 0; k < n; k++) {
        if (a < 0 || id[k] < id[a]) {
            b = a;
            a = k;
        } else if (b < 0 || id[k] < id[b]) {
            b = k;
        }
    }
    keep[0] = a;
    keep[1] = b;
    /* totals, members in increasing id */
    double W = 0.0, P[3] = {0.0, 0.0, 0.0}, E = 0.0;
    int last = -2147483647 - 1;
    for (long long done = 0; done < n; done++) {
        long long k = -1;
        for (long long j = 0; j < n; j++)
            if (id[j] > last && (k < 0 || id[j] < id[k])) k = j;
        if (k < 0) break; /* ids repeat: not a valid group */
        last = id[k];
        const double g = sqrt(1.0 + ux[k] * ux[k] + uy[k] * uy[k] + uz[k] * uz[k]);
        W += w[k];
        P[0] += w[k] * ux[k];
        P[1] += w[k] * uy[k];
        P[2] += w[k] * uz[k];
        E += w[k] * g;
    }
    *out_w = 0.5 * W;
    const double gn = E / W;
    const double un = sqrt(gn * gn - 1.0 > 0.0 ? gn * gn - 1.0 : 0.0);
    const double pm = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
    double e1[3], e2[3];
    const double r[3] = {ux[a], uy[a], uz[a]};
    const double rm = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (pm > 0.0) {
        for (int i = 0; i < 3; i++) e1[i] = P[i] / pm;
    } else if (rm > 0.0) {
        for (int i = 0; i < 3; i++) e1[i] = r[i] / rm;
    } else {
        e1[0] = 1.0, e1[1] = 0.0, e1[2] = 0.0;
    }
    /* e2: the reference momentum's part normal to e1, else an axis's */
    double v[3] = {r[0], r[1], r[2]};
    double dot = v[0] * e1[0] + v[1] * e1[1] + v[2] * e1[2];
    double t[3] = {v[0] - dot * e1[0], v[1] - dot * e1[1], v[2] - dot * e1[2]};
    double tm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    if (!(tm > 1e-12 * (rm > 0.0 ? rm : 1.0))) {
        int ax = 0;
        for (int i = 1; i < 3; i++)
            if (fabs(e1[i]) < fabs(e1[ax])) ax = i;
        v[0] = v[1] = v[2] = 0.0;
        v[ax] = 1.0;
        dot = e1[ax];
        t[0] = v[0] - dot * e1[0];
        t[1] = v[1] - dot * e1[1];
        t[2] = v[2] - dot * e1[2];
        tm = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    }
    for (int i = 0; i < 3; i++) e2[i] = t[i] / tm;
    double ct = (un > 0.0) ? pm / (W * un) : 0.0;
    if (ct > 1.0) ct = 1.0;
    const double st = sqrt(1.0 - ct * ct);
    for (int i = 0; i < 3; i++) {
        out_u[i] = un * (ct * e1[i] + st * e2[i]);
        out_u[3 + i] = un * (ct * e1[i] - st * e2[i]);
    }
    return 1;
}

/* cell and patch of particle p (window or periodic, positions in [0, L)) */
static void cell_of(const orc_sim* s, long long p, long ic[3]) {
    const orc_config* c = &s->c;
    const double pos[3] = {s->x[p], s->y[p], s->z[p]};
    for (int a = 0; a < 3; a++) {
        if (a >= c->dims) {
            ic[a] = 0;
            continue;
        }
        long i = (long)floor(pos[a] / c->d[a]);
        if (i < 0) i = 0;
        if (i >= c->n[a]) i = c->n[a] - 1;
        ic[a] = i;
    }
}

long long orc_merge(orc_sim* s, const int patch[3], long long above, double dp) {
    const orc_config* c = &s->c;
    long np_[3];
    for (int a = 0; a < 3; a++) np_[a] = a < c->dims ? c->n[a] / patch[a] : 1;
    const long long npatch = (long long)np_[0] * np_[1] * np_[2];
    if (s->mlast_n != npatch) {
        free(s->mlast);
        s->mlast = (long long*)calloc((size_t)npatch, sizeof(long long));
        s->mlast_n = s->mlast ? npatch : 0;
        if (!s->mlast) return -1;
    }
    long long* count = (long long*)calloc((size_t)npatch, sizeof(long long));
    long long* prem = (long long*)calloc((size_t)npatch, sizeof(long long));
    long long* pidx = (long long*)malloc((size_t)(s->np > 0 ? s->np : 1) * sizeof(long long));
    long long* key = (long long*)malloc((size_t)(s->np > 0 ? s->np : 1) * 4 * sizeof(long long));
    unsigned char* keep = (unsigned char*)malloc((size_t)(s->np > 0 ? s->np : 1));
    if (!count || !prem || !pidx || !key || !keep) {
        free(count), free(prem), free(pidx), free(key), free(keep);
        return -1;
    }
    for (long long p = 0; p < s->np; p++) {
        long ic[3];
        cell_of(s, p, ic);
        const long pc = ic[0] / (c->dims > 0 ? patch[0] : 1);
        const long pcy = ic[1] / patch[1];
        const long pcz = c->dims == 3 ? ic[2] / patch[2] : 0;
        pidx[p] = (long long)pc + np_[0] * ((long long)pcy + np_[1] * pcz);
        count[pidx[p]]++;
        key[4 * p + 0] = ((long long)ic[2] * c->n[1] + ic[1]) * c->n[0] + ic[0];
        key[4 * p + 1] = (long long)floor(s->ux[p] / dp);
        key[4 * p + 2] = (long long)floor(s->uy[p] / dp);
        key[4 * p + 3] = (long long)floor(s->uz[p] / dp);
        keep[p] = 1;
    }
    /* a patch is merged when it holds more than `above` particles and more than 5/4 of
     * its count after its previous merge pass (so a patch that merging cannot bring
     * below the threshold is not reprocessed every step) */
    unsigned char* hot = (unsigned char*)calloc((size_t)npatch, 1);
    for (long long q = 0; q < npatch && hot; q++)
        hot[q] = count[q] > above && count[q] > s->mlast[q] + s->mlast[q] / 4;
    /* plain grouping: for each unvisited particle of an overloaded patch, collect the
     * members sharing its cell and bin (quadratic, fine for an oracle) */
    unsigned char* seen = (unsigned char*)calloc((size_t)(s->np > 0 ? s->np : 1), 1);
    long long* mem = (long long*)malloc((size_t)(s->np > 0 ? s->np : 1) * sizeof(long long));
    double *gx = (double*)malloc((size_t)(s->np > 0 ? s->np : 1) * 4 * sizeof(double));
    int* gid = (int*)malloc((size_t)(s->np > 0 ? s->np : 1) * sizeof(int));
    long long removed = 0;
    if (seen && mem && gx && gid && hot) {
        for (long long p = 0; p < s->np; p++) {
            if (seen[p] || !hot[pidx[p]]) continue;
            long long m = 0;
            for (long long q = p; q < s->np; q++) {
                if (seen[q] || pidx[q] != pidx[p]) continue;
                if (key[4 * q] != key[4 * p] || key[4 * q + 1] != key[4 * p + 1] ||
                    key[4 * q + 2] != key[4 * p + 2] || key[4 * q + 3] != key[4 * p + 3])
                    continue;
                seen[q] = 1;
                mem[m++] = q;
            }
            if (m < 3) continue;
            double* gux = gx;
            double* guy = gx + m;
            double* guz = gx + 2 * m;
            double* gw = gx + 3 * m;
            for (long long k = 0; k < m; k++) {
                gux[k] = s->ux[mem[k]];
                guy[k] = s->uy[mem[k]];
                guz[k] = s->uz[mem[k]];
                gw[k] = s->w[mem[k]];
                gid[k] = s->id[mem[k]];
            }
            double nu[6], nw;
            long long kp[2];
            orc_merge_group(m, gux, guy, guz, gw, gid, nu, &nw, kp);
            for (long long k = 0; k < m; k++) keep[mem[k]] = 0;
            for (int j = 0; j < 2; j++) {
                const long long q = mem[kp[j]];
                keep[q] = 1;
                s->ux[q] = nu[3 * j + 0];
                s->uy[q] = nu[3 * j + 1];
                s->uz[q] = nu[3 * j + 2];
                s->w[q] = nw;
            }
            removed += m - 2;
            prem[pidx[p]] += m - 2;
        }
        compact(s, keep);
        for (long long q = 0; q < npatch; q++)
            if (hot[q]) s->mlast[q] = count[q] - prem[q];
    } else {
        removed = -1;
    }
    free(count), free(prem), free(pidx), free(key), free(keep), free(seen), free(mem), free(gx),
        free(gid), free(hot);
    return removed;
}

/* ------------------------------------------------------------------ splitting */

long long orc_split(orc_sim* s, const int patch[3], long long below, double wmin) {
    const orc_config* c = &s->c;
    if (below <= 1) return 0;
    long np_[3];
    for (int a = 0; a < 3; a++) np_[a] = a < c->dims ? c->n[a] / patch[a] : 1;
    const long P[3] = {patch[0], c->dims >= 2 ? patch[1] : 1, c->dims == 3 ? patch[2] : 1};
    const long long ncell = s->ncell;
    const long long n0 = s->np;
    /* cell of every particle, and particles per cell */
    long long* cnt = (long long*)calloc((size_t)ncell, sizeof(long long));
    long long* pc = (long long*)malloc((size_t)(n0 > 0 ? n0 : 1) * sizeof(long long));
    if (!cnt || !pc) {
        free(cnt), free(pc);
        return -1;
    }
    for (long long p = 0; p < n0; p++) {
        long ic[3];
        cell_of(s, p, ic);
        pc[p] = ((long long)ic[2] * c->n[1] + ic[1]) * c->n[0] + ic[0];
        cnt[pc[p]]++;
    }
    long long done = 0;
    /* patches in index order, cells in local order, parents in increasing id */
    for (long pz = 0; pz < np_[2]; pz++)
        for (long py = 0; py < np_[1]; py++)
            for (long px = 0; px < np_[0]; px++)
                for (long lz = 0; lz < P[2]; lz++)
                    for (long ly = 0; ly < P[1]; ly++)
                        for (long lx = 0; lx < P[0]; lx++) {
                            const long long cell =
                                ((long long)(pz * P[2] + lz) * c->n[1] + (py * P[1] + ly)) * c->n[0] +
                                (px * P[0] + lx);
                            const long long n = cnt[cell];
                            if (n < 1 || n >= below) continue;
                            long long room = below - n;
                            int last = -2147483647 - 1;
                            while (room > 0) {
                                /* the next eligible particle of this cell by id */
                                long long q = -1;
                                for (long long p = 0; p < n0; p++)
                                    if (pc[p] == cell && s->id[p] > last && s->w[p] >= 2.0 * wmin &&
                                        (q < 0 || s->id[p] < s->id[q]))
                                        q = p;
                                if (q < 0) break;
                                last = s->id[q];
                                if (s->np >= s->cap) {
                                    free(cnt), free(pc);
                                    return -1;
                                }
                                const double pos[3] = {s->x[q], s->y[q], s->z[q]};
                                double d[3] = {0.0, 0.0, 0.0};
                                for (int a = 0; a < c->dims; a++) {
                                    const double xi = pos[a] / c->d[a];
                                    const double f = xi - floor(xi);
                                    d[a] = 0.5 * (f < 1.0 - f ? f : 1.0 - f) * c->d[a];
                                }
                                const long long k = s->np++;
                                s->x[k] = pos[0] - d[0];
                                s->y[k] = pos[1] - d[1];
                                s->z[k] = pos[2] - d[2];
                                s->x[q] = pos[0] + d[0];
                                s->y[q] = pos[1] + d[1];
                                s->z[q] = pos[2] + d[2];
                                s->ux[k] = s->ux[q];
                                s->uy[k] = s->uy[q];
                                s->uz[k] = s->uz[q];
                                s->w[q] *= 0.5;
                                s->w[k] = s->w[q];
                                s->id[k] = (int)(s->next_id + done);
                                done++;
                                room--;
                            }
                        }
    s->next_id += done;
    free(cnt), free(pc);
    return done;
}
