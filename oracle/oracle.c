/*
 * oracle.c -- plain, slow, unfused CPU FP64 oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (HFAV, arXiv 1710.08774):
 *   The fused, contracted loop nests HFAV emits reorder side-effect-free,
 *   order-agnostic kernels (Sec. 3.1 "Fundamentals") and elide intermediate
 *   storage (Sec. 3.5 "Variables and storage").  They therefore reach the same
 *   values as calling every kernel in its own loop nest over fully
 *   materialised arrays, in topological order of the dataflow DAG (Sec. 3.2).
 *   That plain definition is what this file writes out: one loop nest per
 *   kernel, every intermediate stored in full, FP64 throughout, compiled with
 *   -ffp-contract=off so no FMA contraction happens.
 *
 * Workloads:
 *   - 2D three-stage chain  L = 5-pt Laplacian(u); G = |central grad L| / 2;
 *     out = G / (1 + G), periodic or caller-given halo of width 2.  The 5-pt
 *     Laplacian is the paper's running example (Sec. 3, Listing "laplace5").
 *   - 2D Euler Godunov step, directionally split, with the nine kernels
 *     Hydro2D is built from (Sec. 5.4: make_boundary, constoprim,
 *     equation_of_state, slope, trace, qleftright, riemann, cmpflx,
 *     update_cons_vars) plus the CFL time-step reduction.  The paper names the
 *     kernels only; the physics written here is the textbook MUSCL-Hancock /
 *     two-shock Godunov scheme, in the reading stated beside each function.
 *   - 3D four-stage 7-point chain (Laplacian, Laplacian, |grad|/2, x/(1+x)).
 *   - the COSMO horizontal-diffusion micro-kernels (Sec. 5.3: ulapstage,
 *     flux_x, flux_y, ustage) over 3D data with no dependency in k.
 *
 * Parity status: every function here is pinned by tests/test_oracle_*.py
 * against closed forms, invariants, an exact Riemann solution or brute force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL -1
#define ORACLE_ENOMEM -2

/* ------------------------------------------------------------------------- */
/* 2D three-stage chain                                                       */
/* ------------------------------------------------------------------------- */

/* Periodic wrap of an index in [-h, n+h) onto [0, n). */
static long wrap(long a, long n) {
    long r = a % n;
    return r < 0 ? r + n : r;
}

/*
 * oracle_chain2d
 *   u    : (ny+4) x (nx+4) array, row pitch pu >= nx+4, interior at (2,2).
 *   periodic != 0 : the halo is filled by periodic wrap of the interior
 *                   (halo index h maps to h mod n) into a private copy;
 *                   otherwise the caller's halo values are used as given.
 *   L    : (ny+2) x (nx+2) output (halo 1, pitch nx+2) or NULL.
 *   G    : ny x nx output (pitch nx) or NULL.
 *   out  : ny x nx output (pitch nx).
 * Stage formulas (one loop nest each, in DAG order):
 *   L(i,j)  = u(i+1,j) + u(i-1,j) + u(i,j+1) + u(i,j-1) - 4 u(i,j)
 *   G(i,j)  = sqrt((L(i+1,j)-L(i-1,j))^2 + (L(i,j+1)-L(i,j-1))^2) / 2
 *   out     = G / (1 + G)
 */
int oracle_chain2d(const double* u, long nx, long ny, long pu, int periodic,
                   double* L, double* G, double* out) {
    if (nx < 1 || ny < 1 || pu < nx + 4) return ORACLE_EINVAL;
    const long px = nx + 4, py = ny + 4;
    double* w = (double*)malloc(sizeof(double) * px * py);
    double* Lw = (double*)malloc(sizeof(double) * (nx + 2) * (ny + 2));
    double* Gw = (double*)malloc(sizeof(double) * nx * ny);
    if (!w || !Lw || !Gw) { free(w); free(Lw); free(Gw); return ORACLE_ENOMEM; }
    /* make_boundary: copy (and wrap) the input into a private padded array */
    for (long j = -2; j < ny + 2; ++j)
        for (long i = -2; i < nx + 2; ++i) {
            long si = periodic ? wrap(i, nx) : i;
            long sj = periodic ? wrap(j, ny) : j;
            w[(j + 2) * px + (i + 2)] = u[(sj + 2) * pu + (si + 2)];
        }
#define W_(i, j) w[((j) + 2) * px + ((i) + 2)]
#define L_(i, j) Lw[((j) + 1) * (nx + 2) + ((i) + 1)]
    /* stage 1: L over the halo-1 ring */
    for (long j = -1; j < ny + 1; ++j)
        for (long i = -1; i < nx + 1; ++i)
            L_(i, j) = W_(i + 1, j) + W_(i - 1, j) + W_(i, j + 1) + W_(i, j - 1) - 4.0 * W_(i, j);
    /* stage 2: G over the interior */
    for (long j = 0; j < ny; ++j)
        for (long i = 0; i < nx; ++i) {
            double gx = L_(i + 1, j) - L_(i - 1, j);
            double gy = L_(i, j + 1) - L_(i, j - 1);
            Gw[j * nx + i] = sqrt(gx * gx + gy * gy) / 2.0;
        }
    /* stage 3: out over the interior */
    for (long j = 0; j < ny; ++j)
        for (long i = 0; i < nx; ++i) {
            double g = Gw[j * nx + i];
            out[j * nx + i] = g / (1.0 + g);
        }
    if (L) memcpy(L, Lw, sizeof(double) * (nx + 2) * (ny + 2));
    if (G) memcpy(G, Gw, sizeof(double) * nx * ny);
#undef W_
#undef L_
    free(w); free(Lw); free(Gw);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* 3D four-stage 7-point chain                                                */
/* ------------------------------------------------------------------------- */

/*
 * oracle_chain3d
 *   u   : (nz+6) x (ny+6) x (nx+6) array, contiguous, interior at (3,3,3).
 *   periodic != 0 : halo filled by wrap; else used as given.
 *   out : nz x ny x nx.
 *   s1 = D7(u)   (sum of the 6 face neighbours minus 6 u), over halo-2 box
 *   s2 = D7(s1)  over halo-1 box
 *   s3 = sqrt(sum over axes (s2(+1) - s2(-1))^2) / 2 over the interior
 *   out = s3 / (1 + s3)
 */
int oracle_chain3d(const double* u, long nx, long ny, long nz, int periodic, double* out) {
    if (nx < 1 || ny < 1 || nz < 1) return ORACLE_EINVAL;
    const long H = 3;
    const long px = nx + 2 * H, py = ny + 2 * H, pz = nz + 2 * H;
    const long n = px * py * pz;
    double* w = (double*)malloc(sizeof(double) * n);
    double* s1 = (double*)calloc(n, sizeof(double));
    double* s2 = (double*)calloc(n, sizeof(double));
    double* s3 = (double*)calloc(n, sizeof(double));
    if (!w || !s1 || !s2 || !s3) { free(w); free(s1); free(s2); free(s3); return ORACLE_ENOMEM; }
#define I3(i, j, k) ((((k) + H) * py + ((j) + H)) * px + ((i) + H))
    for (long k = -H; k < nz + H; ++k)
        for (long j = -H; j < ny + H; ++j)
            for (long i = -H; i < nx + H; ++i) {
                long si = periodic ? wrap(i, nx) : i;
                long sj = periodic ? wrap(j, ny) : j;
                long sk = periodic ? wrap(k, nz) : k;
                w[I3(i, j, k)] = u[I3(si, sj, sk)];
            }
    for (long k = -2; k < nz + 2; ++k)
        for (long j = -2; j < ny + 2; ++j)
            for (long i = -2; i < nx + 2; ++i)
                s1[I3(i, j, k)] = w[I3(i + 1, j, k)] + w[I3(i - 1, j, k)] + w[I3(i, j + 1, k)] +
                                  w[I3(i, j - 1, k)] + w[I3(i, j, k + 1)] + w[I3(i, j, k - 1)] -
                                  6.0 * w[I3(i, j, k)];
    for (long k = -1; k < nz + 1; ++k)
        for (long j = -1; j < ny + 1; ++j)
            for (long i = -1; i < nx + 1; ++i)
                s2[I3(i, j, k)] = s1[I3(i + 1, j, k)] + s1[I3(i - 1, j, k)] + s1[I3(i, j + 1, k)] +
                                  s1[I3(i, j - 1, k)] + s1[I3(i, j, k + 1)] + s1[I3(i, j, k - 1)] -
                                  6.0 * s1[I3(i, j, k)];
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double gx = s2[I3(i + 1, j, k)] - s2[I3(i - 1, j, k)];
                double gy = s2[I3(i, j + 1, k)] - s2[I3(i, j - 1, k)];
                double gz = s2[I3(i, j, k + 1)] - s2[I3(i, j, k - 1)];
                s3[I3(i, j, k)] = sqrt(gx * gx + gy * gy + gz * gz) / 2.0;
            }
    for (long k = 0; k < nz; ++k)
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double s = s3[I3(i, j, k)];
                out[(k * ny + j) * nx + i] = s / (1.0 + s);
            }
#undef I3
    free(w); free(s1); free(s2); free(s3);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------- */
/* 2D Euler, directionally split Godunov (Hydro2D kernel list, Sec. 5.4)      */
/* ------------------------------------------------------------------------- */

#define RHO_FLOOR 1e-10
#define P_FLOOR 1e-10
#define NEWTON_MAX 10
#define NEWTON_TOL 1e-10

typedef struct {
    long floor_hits;        /* density / pressure floors applied in eos or riemann */
    long newton_nonconv;    /* faces whose Newton loop hit NEWTON_MAX without converging */
    long newton_iters;      /* total Newton iterations over all faces */
    long faces;             /* Riemann problems solved */
    long iters_hist[NEWTON_MAX + 1];
} oracle_godunov_stats;

static double minmod(double a, double b) {
    if (a * b <= 0.0) return 0.0;
    return fabs(a) < fabs(b) ? a : b;
}

/*
 * Two-shock Riemann solver, Newton iteration on the star pressure, sampled at
 * x/t = 0.  qL, qR, gdnv: primitive states (rho, u_normal, u_transverse, p).
 * Reading (the paper only names "riemann"): Lagrangian wave speeds
 * W_k = C_k sqrt(1 + (g+1)/(2g) (p* - p_k)/p_k), C_k = sqrt(g p_k rho_k);
 * Newton on u*_R(p) - u*_L(p) = 0 with slopes 1/Z_k, Z_k = 2 W_k^3/(W_k^2 + C_k^2);
 * stop after an update with |dp| <= 1e-10 p_new, at most 10 iterations.
 * Returns the number of Newton iterations taken; *nonconv set when the
 * tolerance was not reached.
 */
int oracle_riemann(const double* qL, const double* qR, double g, double* gdnv,
                   int* nonconv, long* floor_hits) {
    const double rl = qL[0], ul = qL[1], vl = qL[2], pl = qL[3];
    const double rr = qR[0], ur = qR[1], vr = qR[2], pr = qR[3];
    const double cl = sqrt(g * pl * rl);
    const double cr = sqrt(g * pr * rr);
    const double a = (g + 1.0) / (2.0 * g);
    double pstar = (cr * pl + cl * pr - cl * cr * (ur - ul)) / (cl + cr);
    if (pstar < P_FLOOR) { pstar = P_FLOOR; if (floor_hits) ++*floor_hits; }
    int it = 0, conv = 0;
    while (it < NEWTON_MAX) {
        ++it;
        double wl = cl * sqrt(1.0 + a * (pstar - pl) / pl);
        double wr = cr * sqrt(1.0 + a * (pstar - pr) / pr);
        double zl = 2.0 * wl * wl * wl / (wl * wl + cl * cl);
        double zr = 2.0 * wr * wr * wr / (wr * wr + cr * cr);
        double usl = ul - (pstar - pl) / wl;
        double usr = ur + (pstar - pr) / wr;
        double pnew = pstar - zl * zr * (usr - usl) / (zl + zr);
        if (pnew < P_FLOOR) { pnew = P_FLOOR; if (floor_hits) ++*floor_hits; }
        double dp = fabs(pnew - pstar);
        pstar = pnew;
        if (dp <= NEWTON_TOL * pnew) { conv = 1; break; }
    }
    if (nonconv) *nonconv = !conv;
    const double wl = cl * sqrt(1.0 + a * (pstar - pl) / pl);
    const double wr = cr * sqrt(1.0 + a * (pstar - pr) / pr);
    const double ustar = (wl * ul + wr * ur + pl - pr) / (wl + wr);
    /* sample at x/t = 0: the contact moves right (u* > 0) -> left side governs */
    double rs, us, vs, ps, ws, sgn;
    if (ustar > 0.0) { rs = rl; us = ul; vs = vl; ps = pl; ws = wl; sgn = -1.0; }
    else             { rs = rr; us = ur; vs = vr; ps = pr; ws = wr; sgn = 1.0; }
    double rstar = 1.0 / (1.0 / rs - (pstar - ps) / (ws * ws));
    if (rstar < RHO_FLOOR) { rstar = RHO_FLOOR; if (floor_hits) ++*floor_hits; }
    const double cs = sqrt(g * ps / rs);
    const double cstar = sqrt(g * pstar / rstar);
    double ro, uo, po;
    if (pstar > ps) {
        /* shock on side s */
        double S = us + sgn * ws / rs;
        if (sgn * S < 0.0) { ro = rs; uo = us; po = ps; }
        else { ro = rstar; uo = ustar; po = pstar; }
    } else {
        /* rarefaction on side s, linear interpolation across the fan */
        double head = us + sgn * cs;
        double tail = ustar + sgn * cstar;
        if (sgn * head < 0.0) { ro = rs; uo = us; po = ps; }
        else if (sgn * tail > 0.0 || head == tail) { ro = rstar; uo = ustar; po = pstar; }
        else {
            double f = (0.0 - tail) / (head - tail);
            ro = f * rs + (1.0 - f) * rstar;
            uo = f * us + (1.0 - f) * ustar;
            po = f * ps + (1.0 - f) * pstar;
        }
    }
    gdnv[0] = ro; gdnv[1] = uo; gdnv[2] = vs; gdnv[3] = po;
    return it;
}

/*
 * trace: characteristic tracing of one cell, MUSCL-Hancock form (the Hydro2D
 * kernel "trace", Sec. 5.4; the paper names it only).  W = (rho, u_n, u_t, p),
 * c its sound speed, dW its limited slopes, dtdx = dt/dx.  Wave strengths
 * alpha = L dW, eigenvalues (u-c, u, u, u+c), right eigenvectors r_k;
 *   face-right state (at a+1/2): qp = W + 1/2 sum (1 - nu_k) alpha_k r_k,
 *   face-left state (at a-1/2):  qm = W - 1/2 sum (1 + nu_k) alpha_k r_k,
 * with nu_k = lambda_k dt/dx.
 */
void oracle_trace(const double* W, double c, const double* dW, double dtdx, double* qm, double* qp) {
    const double r = W[0], u = W[1];
    const double dr = dW[0], du = dW[1], dv = dW[2], dp = dW[3];
    double alpha[4], lam[4], rv[4][4];
    alpha[0] = (dp / c - r * du) / (2.0 * c);
    alpha[1] = dr - dp / (c * c);
    alpha[2] = dv;
    alpha[3] = (dp / c + r * du) / (2.0 * c);
    lam[0] = u - c; lam[1] = u; lam[2] = u; lam[3] = u + c;
    rv[0][0] = 1.0; rv[0][1] = -c / r; rv[0][2] = 0.0; rv[0][3] = c * c;
    rv[1][0] = 1.0; rv[1][1] = 0.0;    rv[1][2] = 0.0; rv[1][3] = 0.0;
    rv[2][0] = 0.0; rv[2][1] = 0.0;    rv[2][2] = 1.0; rv[2][3] = 0.0;
    rv[3][0] = 1.0; rv[3][1] = c / r;  rv[3][2] = 0.0; rv[3][3] = c * c;
    for (int f = 0; f < 4; ++f) {
        double sp = 0.0, sm = 0.0;
        for (int m = 0; m < 4; ++m) {
            double nu = lam[m] * dtdx;
            sp += (1.0 - nu) * alpha[m] * rv[m][f];
            sm += (1.0 + nu) * alpha[m] * rv[m][f];
        }
        qp[f] = W[f] + 0.5 * sp;
        qm[f] = W[f] - 0.5 * sm;
    }
}

/* Godunov work arrays: every intermediate of one sweep, fully materialised
 * over the padded (ny+4) x (nx+4) grid.  4 (U) + 4 (W) + 1 (c) + 4 (dW)
 * + 8 (face-left/right traces) + 8 (qL/qR) + 4 (Riemann state) + 4 (flux)
 * = 37 full arrays. */
typedef struct {
    long nx, ny, px, py, n;
    double *U[4], *W[4], *c, *dW[4], *qm[4], *qp[4], *qL[4], *qR[4], *gd[4], *F[4];
    double* pool;
} gwork;

static int gwork_init(gwork* w, long nx, long ny) {
    w->nx = nx; w->ny = ny; w->px = nx + 4; w->py = ny + 4; w->n = w->px * w->py;
    w->pool = (double*)calloc((size_t)37 * w->n, sizeof(double));
    if (!w->pool) return ORACLE_ENOMEM;
    double* p = w->pool;
    for (int f = 0; f < 4; ++f) { w->U[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->W[f] = p; p += w->n; }
    w->c = p; p += w->n;
    for (int f = 0; f < 4; ++f) { w->dW[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->qm[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->qp[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->qL[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->qR[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->gd[f] = p; p += w->n; }
    for (int f = 0; f < 4; ++f) { w->F[f] = p; p += w->n; }
    return ORACLE_OK;
}

/* Address of padded cell (a along the sweep, b across it) for a sweep
 * direction: dir 0 = x (a = i), dir 1 = y (a = j). */
static long gidx(const gwork* w, int dir, long a, long b) {
    long i = dir == 0 ? a : b;
    long j = dir == 0 ? b : a;
    return (j + 2) * w->px + (i + 2);
}

/*
 * One directional sweep over all lines, every kernel its own loop nest.
 * Conserved components: U0 = rho, U1 = rho u, U2 = rho v, U3 = E.
 * For dir 0 the normal momentum is U1 and the transverse U2; for dir 1 the
 * roles swap (the paper notes the rules are given once per pass, Sec. 5.4).
 * Cells run over a in [0, na); the sweep needs W on [-2, na+2).
 */
static void godunov_sweep(gwork* w, int dir, double dt, double dx, double g,
                          oracle_godunov_stats* st) {
    const long na = dir == 0 ? w->nx : w->ny;   /* length along the sweep */
    const long nb = dir == 0 ? w->ny : w->nx;   /* number of lines */
    const int mn = dir == 0 ? 1 : 2;            /* normal momentum component */
    const int mt = dir == 0 ? 2 : 1;            /* transverse momentum component */
    const double dtdx = dt / dx;

    /* make_boundary: periodic halo of width 2 in both directions */
    for (int f = 0; f < 4; ++f)
        for (long j = -2; j < w->ny + 2; ++j)
            for (long i = -2; i < w->nx + 2; ++i) {
                if (i >= 0 && i < w->nx && j >= 0 && j < w->ny) continue;
                w->U[f][(j + 2) * w->px + (i + 2)] =
                    w->U[f][(wrap(j, w->ny) + 2) * w->px + (wrap(i, w->nx) + 2)];
            }

    /* constoprim: W = (rho, u_n, u_t, e) with e the specific internal energy
     * (e is kept in W[3] until equation_of_state replaces it by p) */
    for (long b = 0; b < nb; ++b)
        for (long a = -2; a < na + 2; ++a) {
            long k = gidx(w, dir, a, b);
            double r = w->U[0][k];
            double un = w->U[mn][k] / r;
            double ut = w->U[mt][k] / r;
            double e = w->U[3][k] / r - 0.5 * (un * un + ut * ut);
            w->W[0][k] = r; w->W[1][k] = un; w->W[2][k] = ut; w->W[3][k] = e;
        }

    /* equation_of_state: p = (g-1) rho e, c = sqrt(g p / rho), with floors */
    for (long b = 0; b < nb; ++b)
        for (long a = -2; a < na + 2; ++a) {
            long k = gidx(w, dir, a, b);
            double r = w->W[0][k];
            if (r < RHO_FLOOR) { r = RHO_FLOOR; w->W[0][k] = r; ++st->floor_hits; }
            double p = (g - 1.0) * r * w->W[3][k];
            if (p < P_FLOOR) { p = P_FLOOR; ++st->floor_hits; }
            w->W[3][k] = p;
            w->c[k] = sqrt(g * p / r);
        }

    /* slope: minmod-limited differences of the primitives */
    for (int f = 0; f < 4; ++f)
        for (long b = 0; b < nb; ++b)
            for (long a = -1; a < na + 1; ++a) {
                double qm1 = w->W[f][gidx(w, dir, a - 1, b)];
                double q0 = w->W[f][gidx(w, dir, a, b)];
                double qp1 = w->W[f][gidx(w, dir, a + 1, b)];
                w->dW[f][gidx(w, dir, a, b)] = minmod(q0 - qm1, qp1 - q0);
            }

    /* trace: characteristic tracing (oracle_trace), cell by cell */
    for (long b = 0; b < nb; ++b)
        for (long a = -1; a < na + 1; ++a) {
            long k = gidx(w, dir, a, b);
            double Wc[4], dWc[4], qm[4], qp[4];
            for (int f = 0; f < 4; ++f) { Wc[f] = w->W[f][k]; dWc[f] = w->dW[f][k]; }
            oracle_trace(Wc, w->c[k], dWc, dtdx, qm, qp);
            for (int f = 0; f < 4; ++f) { w->qm[f][k] = qm[f]; w->qp[f][k] = qp[f]; }
        }

    /* qleftright: the face a+1/2 is stored at index a, for a in [-1, na) */
    for (int f = 0; f < 4; ++f)
        for (long b = 0; b < nb; ++b)
            for (long a = -1; a < na; ++a) {
                w->qL[f][gidx(w, dir, a, b)] = w->qp[f][gidx(w, dir, a, b)];
                w->qR[f][gidx(w, dir, a, b)] = w->qm[f][gidx(w, dir, a + 1, b)];
            }

    /* riemann: Godunov state at every face */
    for (long b = 0; b < nb; ++b)
        for (long a = -1; a < na; ++a) {
            long k = gidx(w, dir, a, b);
            double ql[4], qr[4], gs[4];
            for (int f = 0; f < 4; ++f) { ql[f] = w->qL[f][k]; qr[f] = w->qR[f][k]; }
            int nonconv = 0;
            int it = oracle_riemann(ql, qr, g, gs, &nonconv, &st->floor_hits);
            st->faces++; st->newton_iters += it; st->iters_hist[it]++;
            if (nonconv) st->newton_nonconv++;
            for (int f = 0; f < 4; ++f) w->gd[f][k] = gs[f];
        }

    /* cmpflx: Euler flux of the Godunov state */
    for (long b = 0; b < nb; ++b)
        for (long a = -1; a < na; ++a) {
            long k = gidx(w, dir, a, b);
            double r = w->gd[0][k], un = w->gd[1][k], ut = w->gd[2][k], p = w->gd[3][k];
            double mflux = r * un;
            double etot = p / (g - 1.0) + 0.5 * r * (un * un + ut * ut);
            w->F[0][k] = mflux;
            w->F[1][k] = mflux * un + p;
            w->F[2][k] = mflux * ut;
            w->F[3][k] = un * (etot + p);
        }

    /* update_cons_vars: U -= dt/dx (F(a+1/2) - F(a-1/2)) */
    for (long b = 0; b < nb; ++b)
        for (long a = 0; a < na; ++a) {
            long k = gidx(w, dir, a, b);
            long km = gidx(w, dir, a - 1, b);
            w->U[0][k] -= dtdx * (w->F[0][k] - w->F[0][km]);
            w->U[mn][k] -= dtdx * (w->F[1][k] - w->F[1][km]);
            w->U[mt][k] -= dtdx * (w->F[2][k] - w->F[2][km]);
            w->U[3][k] -= dtdx * (w->F[3][k] - w->F[3][km]);
        }
}

/* CFL reduction: dt = cfl dx / max over interior cells of max(|u|+c, |v|+c). */
static double godunov_dt(const gwork* w, double cfl, double dx, double g) {
    double smax = 0.0;
    for (long j = 0; j < w->ny; ++j)
        for (long i = 0; i < w->nx; ++i) {
            long k = (j + 2) * w->px + (i + 2);
            double r = w->U[0][k];
            double u = w->U[1][k] / r, v = w->U[2][k] / r;
            double e = w->U[3][k] / r - 0.5 * (u * u + v * v);
            double p = (g - 1.0) * r * e;
            if (p < P_FLOOR) p = P_FLOOR;
            double c = sqrt(g * p / r);
            double s = fabs(u) + c;
            double t = fabs(v) + c;
            if (t > s) s = t;
            if (s > smax) smax = s;
        }
    return cfl * dx / smax;
}

static void gload(gwork* w, const double* U) {
    for (int f = 0; f < 4; ++f)
        for (long j = 0; j < w->ny; ++j)
            for (long i = 0; i < w->nx; ++i)
                w->U[f][(j + 2) * w->px + (i + 2)] = U[(f * w->ny + j) * w->nx + i];
}

static void gstore(const gwork* w, double* U) {
    for (int f = 0; f < 4; ++f)
        for (long j = 0; j < w->ny; ++j)
            for (long i = 0; i < w->nx; ++i)
                U[(f * w->ny + j) * w->nx + i] = w->U[f][(j + 2) * w->px + (i + 2)];
}

/*
 * oracle_godunov: nsteps of (dt from CFL; x sweep; y sweep) on a periodic grid.
 *   U       : 4 x ny x nx interior, field-major (rho, rho u, rho v, E); in/out.
 *   dx      : 1/nx (domain [0,1] x [0, ny/nx]).
 *   dt_fixed: if > 0, that dt is used every step instead of the CFL value.
 *   sweeps  : bit 0 = do the x sweep, bit 1 = do the y sweep (3 = both).
 *   dt_hist : nsteps entries, the dt used at each step (may be NULL).
 */
int oracle_godunov(double* U, long nx, long ny, int nsteps, double cfl, double g,
                   double dt_fixed, int sweeps, double* dt_hist, oracle_godunov_stats* st) {
    if (nx < 3 || ny < 3 || nsteps < 0) return ORACLE_EINVAL;
    gwork w;
    if (gwork_init(&w, nx, ny) != ORACLE_OK) return ORACLE_ENOMEM;
    oracle_godunov_stats local;
    if (!st) st = &local;
    memset(st, 0, sizeof(*st));
    gload(&w, U);
    const double dx = 1.0 / (double)nx;
    for (int s = 0; s < nsteps; ++s) {
        double dt = dt_fixed > 0.0 ? dt_fixed : godunov_dt(&w, cfl, dx, g);
        if (dt_hist) dt_hist[s] = dt;
        if (sweeps & 1) godunov_sweep(&w, 0, dt, dx, g, st);
        if (sweeps & 2) godunov_sweep(&w, 1, dt, dx, g, st);
    }
    gstore(&w, U);
    free(w.pool);
    return ORACLE_OK;
}

/* CFL time step of a state (same reduction as inside oracle_godunov). */
double oracle_godunov_cfl_dt(const double* U, long nx, long ny, double cfl, double g) {
    gwork w;
    if (gwork_init(&w, nx, ny) != ORACLE_OK) return -1.0;
    gload(&w, U);
    double dt = godunov_dt(&w, cfl, 1.0 / (double)nx, g);
    free(w.pool);
    return dt;
}

/* ------------------------------------------------------------------------- */
/* timing helper for the CPU baseline                                         */
/* ------------------------------------------------------------------------- */
int oracle_version(void) { return 1; }

/* ------------------------------------------------------------------------- */
/* COSMO horizontal diffusion (Sec. 5.3)                                      */
/* ------------------------------------------------------------------------- */

/*
 * oracle_cosmo
 *   The paper lists the four kernels and the operands each reads (a cell's u
 *   and its i / j neighbours for ulapstage; u and ulapstage at two
 *   neighbouring cells in i (j) for flux_x (flux_y); u and the four
 *   neighbouring fluxes for ustage) but not their formulas.  Written here:
 *   the fourth-order horizontal diffusion with a flux limiter of the stencil
 *   benchmark the paper takes the example from:
 *     lap(i,j) = u(i+1,j) + u(i-1,j) + u(i,j+1) + u(i,j-1) - 4 u(i,j)
 *     flx(i,j) = lap(i+1,j) - lap(i,j), or 0 where flx (u(i+1,j) - u(i,j)) > 0
 *     fly(i,j) = lap(i,j+1) - lap(i,j), or 0 where fly (u(i,j+1) - u(i,j)) > 0
 *     out(i,j) = u(i,j) - c ((flx(i,j) - flx(i-1,j)) + (fly(i,j) - fly(i,j-1)))
 *   (the flux at index i is the face i+1/2), every k plane on its own.
 *   u    : (nz+4) x (ny+4) x (nx+4) array, row pitch pu >= nx+4, plane pitch
 *          pp >= pu (ny+4), interior at (2,2,2); the k halo is never read.
 *   periodic != 0 : i and j wrap onto the interior; otherwise the caller's
 *          halo of width 2 in i and j is used as given.
 *   lap  : nz x (ny+2) x (nx+2) (halo 1) or NULL;  flx : nz x ny x (nx+1)
 *          (i = -1 .. nx-1) or NULL;  fly : nz x (ny+1) x nx (j = -1 .. ny-1)
 *          or NULL;  out : nz x ny x nx.
 */
int oracle_cosmo(const double* u, long nx, long ny, long nz, long pu, long pp, int periodic, double c,
                 double* lap, double* flx, double* fly, double* out) {
    if (nx < 1 || ny < 1 || nz < 1 || pu < nx + 4 || pp < pu * (ny + 4)) return ORACLE_EINVAL;
    const long px = nx + 4, py = ny + 4;
    double* w = (double*)malloc(sizeof(double) * px * py);
    double* Lw = (double*)malloc(sizeof(double) * (nx + 2) * (ny + 2));
    double* Fx = (double*)malloc(sizeof(double) * (nx + 1) * ny);
    double* Fy = (double*)malloc(sizeof(double) * nx * (ny + 1));
    if (!w || !Lw || !Fx || !Fy) { free(w); free(Lw); free(Fx); free(Fy); return ORACLE_ENOMEM; }
#define W_(i, j) w[((j) + 2) * px + ((i) + 2)]
#define L_(i, j) Lw[((j) + 1) * (nx + 2) + ((i) + 1)]
#define FX_(i, j) Fx[(j) * (nx + 1) + ((i) + 1)]
#define FY_(i, j) Fy[((j) + 1) * nx + (i)]
    for (long k = 0; k < nz; ++k) {
        const double* uk = u + (k + 2) * pp;
        /* make_boundary: copy (and wrap) the plane into a private padded array */
        for (long j = -2; j < ny + 2; ++j)
            for (long i = -2; i < nx + 2; ++i) {
                long si = periodic ? wrap(i, nx) : i;
                long sj = periodic ? wrap(j, ny) : j;
                W_(i, j) = uk[(sj + 2) * pu + (si + 2)];
            }
        /* ulapstage over the halo-1 ring */
        for (long j = -1; j < ny + 1; ++j)
            for (long i = -1; i < nx + 1; ++i)
                L_(i, j) = W_(i + 1, j) + W_(i - 1, j) + W_(i, j + 1) + W_(i, j - 1) - 4.0 * W_(i, j);
        /* flux_x on faces i = -1 .. nx-1 of the interior rows */
        for (long j = 0; j < ny; ++j)
            for (long i = -1; i < nx; ++i) {
                double f = L_(i + 1, j) - L_(i, j);
                if (f * (W_(i + 1, j) - W_(i, j)) > 0.0) f = 0.0;
                FX_(i, j) = f;
            }
        /* flux_y on faces j = -1 .. ny-1 of the interior columns */
        for (long j = -1; j < ny; ++j)
            for (long i = 0; i < nx; ++i) {
                double f = L_(i, j + 1) - L_(i, j);
                if (f * (W_(i, j + 1) - W_(i, j)) > 0.0) f = 0.0;
                FY_(i, j) = f;
            }
        /* ustage */
        for (long j = 0; j < ny; ++j)
            for (long i = 0; i < nx; ++i)
                out[(k * ny + j) * nx + i] =
                    W_(i, j) - c * ((FX_(i, j) - FX_(i - 1, j)) + (FY_(i, j) - FY_(i, j - 1)));
        if (lap) memcpy(lap + k * (nx + 2) * (ny + 2), Lw, sizeof(double) * (nx + 2) * (ny + 2));
        if (flx) memcpy(flx + k * (nx + 1) * ny, Fx, sizeof(double) * (nx + 1) * ny);
        if (fly) memcpy(fly + k * nx * (ny + 1), Fy, sizeof(double) * nx * (ny + 1));
    }
#undef W_
#undef L_
#undef FX_
#undef FY_
    free(w); free(Lw); free(Fx); free(Fy);
    return ORACLE_OK;
}
