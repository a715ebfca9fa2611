/*
 * khydro_oracle.c -- plain, slow, FP64 CPU oracle for one explicit Godunov
 * finite-volume step of the Euler equations on a uniform Cartesian mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or helper
 * with the CUDA library; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  The product path never calls it.
 *
 * What it computes (arXiv:2501.02317, Kratos hydrodynamics module):
 *   - conserved state U = (rho, rho v, eps), eps = eps_g + rho v^2/2 (Sec. 3, Eq. 2)
 *   - conserved -> primitive recovery, then the CFL time step on the first
 *     sub-step only (Sec. 3.1)
 *   - ghost zones of width n_gh = 2 filled by the physical boundary rules
 *     free / outflow / reflecting (Sec. 3.1.1) or by periodic wrap (Sec. 3.1.1,
 *     periodic domains become communication boundaries)
 *   - slope-limited piecewise-linear reconstruction with the minmod limiter
 *     (Eq. 3, Sec. 3.1.2; used by PLM per Sec. 3.2.2) on primitive variables
 *   - the HLLC Riemann solver with the contact speed of Eq. 4 and the
 *     subtraction-safe wave speeds of Eq. 5 (Sec. 3.2.2)
 *   - the conservative flux-difference update inside the Heun (RK2)
 *     predictor-corrector (Sec. 3.3), or inside the memory-optimized van Leer
 *     predictor-corrector (Sec. 3.3, last paragraph)
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - HLLC p* estimate: the pressure-based (PVRS) estimate clamped at 0, the
 *     estimate Eq. 5's q_i belongs to in Toro's textbook (ch. 10).
 *   - HLLC star states: the state-based form U*_K with F*_K = F_K + s_K (U*_K - U_K).
 *   - Unsplit method of lines: every direction reads the same stage state and
 *     the direction contributions are summed (fluxes "from the pre-update
 *     primitive variables", Sec. 4.2).
 *   - PLM: minmod is positively homogeneous, so
 *     minmod(D-/dx, D+/dx) * dx/2 == minmod(D-, D+) / 2 exactly in real
 *     arithmetic; the undivided form is evaluated and dx never appears as a
 *     difference of cell-centre coordinates (the concern of Sec. 3.2.2).
 *   - minmod(a,b) = 0 when a*b <= 0; the sign test is done on the signs, not on
 *     the product, so it cannot underflow.
 *   - dt = C * min over cells and directions of dx_d / (|v_d| + c_s), computed
 *     from U^n before stage 1, reused by stage 2, clipped to hit t_end.
 *   - van Leer integrator (the paper names it only): the predictor advances
 *     U^n by dt/2 with first-order (piecewise-constant) face states, and only
 *     the primitives of that half-step state are kept; the corrector advances
 *     U^n by the full dt with PLM face states of those primitives.  The final
 *     state is U^n plus flux differences only, so it is conservative.
 *   - floors rho_floor, p_floor act on the recovered primitives only.
 *
 * Canonical operation order.  Every floating-point operation below is written
 * out in the order it is evaluated; the file must be compiled with
 * -ffp-contract=off (no fused multiply-add contraction) and without
 * -ffast-math, so that IEEE-754 double rounding applies to each operation.
 *
 * Array layout: field-major [nvar][nz][ny][nx], x fastest, interior cells
 * only.  nvar = 2 + ndim: (rho, m_1..m_ndim, E) conserved, (rho, v_1..v_ndim,
 * p) primitive.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_BC_PERIODIC 0
#define ORC_BC_OUTFLOW  1
#define ORC_BC_FREE     2
#define ORC_BC_REFLECT  3

#define ORC_FLAG_NONPHYSICAL 1u
#define ORC_FLAG_FLOOR       2u

#define NG 2 /* ghost width = reconstruction order (Sec. 3.1) */

typedef struct {
    int ndim;          /* 1, 2 or 3 */
    int n[3];          /* interior cells per axis (1 for unused axes) */
    double lo[3];      /* domain lower corner */
    double hi[3];      /* domain upper corner */
    double gamma;      /* adiabatic index */
    double cfl;        /* Courant number C */
    double rho_floor;  /* floor on the recovered density */
    double p_floor;    /* floor on the recovered pressure */
    int bc[3][2];      /* ORC_BC_* per axis, [0]=low side, [1]=high side */
} orc_mesh;

/* ---------------------------------------------------------------- helpers */

static long ncell(const orc_mesh *m) { return (long)m->n[0] * m->n[1] * m->n[2]; }

static double cell_width(const orc_mesh *m, int d) { return (m->hi[d] - m->lo[d]) / (double)m->n[d]; }

/* Padded primitive grid: NG ghost cells on both sides of every active axis. */
typedef struct {
    int np[3];  /* padded extents */
    int off[3]; /* offset of interior index 0 */
} pad_t;

static pad_t make_pad(const orc_mesh *m) {
    pad_t p;
    for (int d = 0; d < 3; ++d) {
        if (d < m->ndim) { p.np[d] = m->n[d] + 2 * NG; p.off[d] = NG; }
        else { p.np[d] = 1; p.off[d] = 0; }
    }
    return p;
}

/* index of interior cell (i,j,k) in the padded grid; i,j,k may be ghosts */
static long pidx(const pad_t *p, int i, int j, int k) {
    return ((long)(k + p->off[2]) * p->np[1] + (j + p->off[1])) * p->np[0] + (i + p->off[0]);
}

static long uidx(const orc_mesh *m, int i, int j, int k) {
    return ((long)k * m->n[1] + j) * m->n[0] + i;
}

/* ------------------------------------------------- Eq. 2: state variables */

/* primitive (rho, v_1..v_ndim, p) -> conserved (rho, m_1..m_ndim, E):
 * m_d = rho v_d, E = p/(gamma-1) + rho |v|^2 / 2 (Sec. 3, text under Eq. 2) */
void orc_prim_to_cons(const orc_mesh *m, const double *W, double *U) {
    const long N = ncell(m);
    const int nd = m->ndim, nv = 2 + nd;
    const double gm1 = m->gamma - 1.0;
    for (long c = 0; c < N; ++c) {
        double rho = W[c];
        double v[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < nd; ++d) v[d] = W[(long)(1 + d) * N + c];
        double p = W[(long)(nv - 1) * N + c];
        double vsq = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        U[c] = rho;
        for (int d = 0; d < nd; ++d) U[(long)(1 + d) * N + c] = rho * v[d];
        U[(long)(nv - 1) * N + c] = p / gm1 + 0.5 * rho * vsq;
    }
}

/* Sec. 3.1: conserved -> primitive for one cell.  w[0..4] = (rho, v_x, v_y,
 * v_z, p) with unused velocity components set to 0.  Floors act on the
 * primitive only; *flags collects NONPHYSICAL / FLOOR events. */
static void recover_cell(const orc_mesh *m, const double *u, double *w, unsigned *flags) {
    const int nd = m->ndim;
    const double gm1 = m->gamma - 1.0;
    double rho = u[0];
    if (!(rho > 0.0)) *flags |= ORC_FLAG_NONPHYSICAL;
    if (rho < m->rho_floor) { rho = m->rho_floor; *flags |= ORC_FLAG_FLOOR; }
    double v[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < nd; ++d) v[d] = u[1 + d] / rho;
    double ke = 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double eint = u[1 + nd] - ke;
    if (!(eint >= 0.0)) *flags |= ORC_FLAG_NONPHYSICAL;
    double p = gm1 * eint;
    if (p < m->p_floor) { p = m->p_floor; *flags |= ORC_FLAG_FLOOR; }
    w[0] = rho; w[1] = v[0]; w[2] = v[1]; w[3] = v[2]; w[4] = p;
}

static void gather_cons(const orc_mesh *m, const double *U, long c, double *u) {
    const long N = ncell(m);
    const int nv = 2 + m->ndim;
    for (int q = 0; q < nv; ++q) u[q] = U[(long)q * N + c];
}

void orc_cons_to_prim(const orc_mesh *m, const double *U, double *W, unsigned *flags) {
    const long N = ncell(m);
    const int nd = m->ndim, nv = 2 + nd;
    unsigned f = 0;
    for (long c = 0; c < N; ++c) {
        double u[5], w[5];
        gather_cons(m, U, c, u);
        recover_cell(m, u, w, &f);
        W[c] = w[0];
        for (int d = 0; d < nd; ++d) W[(long)(1 + d) * N + c] = w[1 + d];
        W[(long)(nv - 1) * N + c] = w[4];
    }
    if (flags) *flags |= f;
}

/* ------------------------------------------------------ Sec. 3.1: CFL step */

/* C * min over interior cells and active directions of dx_d / (|v_d| + c_s),
 * c_s = sqrt(gamma p / rho).  Not yet clipped to t_end. */
double orc_cfl_dt(const orc_mesh *m, const double *U, unsigned *flags) {
    const long N = ncell(m);
    const int nd = m->ndim;
    double dx[3];
    for (int d = 0; d < 3; ++d) dx[d] = cell_width(m, d);
    double wmin = INFINITY;
    unsigned f = 0;
#pragma omp parallel for schedule(static) reduction(min:wmin) reduction(|:f)
    for (long c = 0; c < N; ++c) {
        double u[5], w[5];
        gather_cons(m, U, c, u);
        recover_cell(m, u, w, &f);
        double cs = sqrt(m->gamma * w[4] / w[0]);
        for (int d = 0; d < nd; ++d) {
            double t = dx[d] / (fabs(w[1 + d]) + cs);
            if (t < wmin) wmin = t;
        }
    }
    if (flags) *flags |= f;
    return m->cfl * wmin;
}

/* --------------------------------------------------- Eq. 3: minmod limiter */

double orc_minmod(double a, double b) {
    int same_sign = (a > 0.0 && b > 0.0) || (a < 0.0 && b < 0.0); /* ab > 0 */
    if (!same_sign) return 0.0;
    return (fabs(a) < fabs(b)) ? a : b;
}

/* ------------------------------------------- Sec. 3.2.2: HLLC Riemann flux */

/* Physical flux along the normal of a primitive state w = (rho, u, t1, t2, p)
 * in the rotated frame, and the matching conserved state. */
static void euler_flux(double gamma, const double *w, double *U, double *F) {
    double rho = w[0], u = w[1], t1 = w[2], t2 = w[3], p = w[4];
    double E = p / (gamma - 1.0) + 0.5 * rho * (u * u + t1 * t1 + t2 * t2);
    double mf = rho * u;
    U[0] = rho; U[1] = rho * u; U[2] = rho * t1; U[3] = rho * t2; U[4] = E;
    F[0] = mf; F[1] = mf * u + p; F[2] = mf * t1; F[3] = mf * t2; F[4] = (E + p) * u;
}

/* HLLC flux between left state wl and right state wr, both (rho, u, t1, t2, p)
 * with u the velocity normal to the face.  Output F in the same rotated
 * order (mass, normal momentum, t1 momentum, t2 momentum, energy). */
void orc_hllc(double gamma, const double *wl, const double *wr, double *F) {
    double rl = wl[0], ul = wl[1], pl = wl[4];
    double rr = wr[0], ur = wr[1], pr = wr[4];
    double cl = sqrt(gamma * pl / rl);
    double cr = sqrt(gamma * pr / rr);
    /* estimate of p*: the linearised (PVRS) value, clamped at zero; when it
     * exceeds both input pressures (both waves are shocks) it is replaced by
     * the two-shock estimate built on it.  Without the switch, colliding
     * flows faster than about Mach 1.8 give s_L > s_R. */
    double ppv = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr);
    double pstar = ppv > 0.0 ? ppv : 0.0;
    double pmax = pl > pr ? pl : pr;
    if (pstar > pmax) {
        double gl = sqrt((2.0 / ((gamma + 1.0) * rl)) / (pstar + (gamma - 1.0) / (gamma + 1.0) * pl));
        double gr = sqrt((2.0 / ((gamma + 1.0) * rr)) / (pstar + (gamma - 1.0) / (gamma + 1.0) * pr));
        pstar = (gl * pl + gr * pr - (ur - ul)) / (gl + gr);
    }
    /* Eq. 5: q_K and the subtraction-safe speed offsets ds_K = s_K - u_K */
    double g1 = (gamma + 1.0) / (2.0 * gamma);
    double ratl = pstar / pl, ratr = pstar / pr;
    if (ratl < 1.0) ratl = 1.0;
    if (ratr < 1.0) ratr = 1.0;
    double ql = sqrt(1.0 + g1 * (ratl - 1.0));
    double qr = sqrt(1.0 + g1 * (ratr - 1.0));
    double dsl = -cl * ql;
    double dsr = cr * qr;
    double sl = ul + dsl;
    double sr = ur + dsr;
    /* Eq. 4 with s_K - u_K replaced by ds_K */
    double sstar = ((pr - rr * ur * dsr) - (pl - rl * ul * dsl)) / (rl * dsl - rr * dsr);

    double UL[5], FL[5], UR[5], FR[5];
    euler_flux(gamma, wl, UL, FL);
    euler_flux(gamma, wr, UR, FR);

    if (0.0 <= sl) {
        for (int q = 0; q < 5; ++q) F[q] = FL[q];
    } else if (0.0 <= sstar) {
        double fac = rl * dsl / (sl - sstar);
        double Us[5];
        Us[0] = fac;
        Us[1] = fac * sstar;
        Us[2] = fac * wl[2];
        Us[3] = fac * wl[3];
        Us[4] = fac * (UL[4] / rl + (sstar - ul) * (sstar + pl / (rl * dsl)));
        for (int q = 0; q < 5; ++q) F[q] = FL[q] + sl * (Us[q] - UL[q]);
    } else if (0.0 < sr) {
        double fac = rr * dsr / (sr - sstar);
        double Us[5];
        Us[0] = fac;
        Us[1] = fac * sstar;
        Us[2] = fac * wr[2];
        Us[3] = fac * wr[3];
        Us[4] = fac * (UR[4] / rr + (sstar - ur) * (sstar + pr / (rr * dsr)));
        for (int q = 0; q < 5; ++q) F[q] = FR[q] + sr * (Us[q] - UR[q]);
    } else {
        for (int q = 0; q < 5; ++q) F[q] = FR[q];
    }
}

/* ---------------------------------- Sec. 3.1.1: ghost zones on primitives */

/* Fill the NG ghost layers of axis d (both sides) for every cell whose other
 * coordinates are interior.  Wp holds 5 primitive fields (rho, vx, vy, vz, p)
 * on the padded grid.  Ghost index g = 1..NG counts outward from the face. */
static void fill_ghosts_axis(const orc_mesh *m, const pad_t *P, double *Wp, int d) {
    const long NP = (long)P->np[0] * P->np[1] * P->np[2];
    const int n = m->n[d];
    int lim[3] = {m->n[0], m->n[1], m->n[2]};
    lim[d] = 1;
    for (int k = 0; k < lim[2]; ++k)
        for (int j = 0; j < lim[1]; ++j)
            for (int i = 0; i < lim[0]; ++i)
                for (int side = 0; side < 2; ++side) {
                    int bc = m->bc[d][side];
                    for (int g = 1; g <= NG; ++g) {
                        int ghost = side == 0 ? -g : n - 1 + g;
                        int src; /* interior source index along d */
                        if (bc == ORC_BC_PERIODIC) src = side == 0 ? n - g : g - 1;
                        else if (bc == ORC_BC_REFLECT) src = side == 0 ? g - 1 : n - g;
                        else src = side == 0 ? 0 : n - 1; /* free, outflow */
                        int gi[3] = {i, j, k}, si[3] = {i, j, k};
                        gi[d] = ghost; si[d] = src;
                        long gdst = pidx(P, gi[0], gi[1], gi[2]);
                        long gsrc = pidx(P, si[0], si[1], si[2]);
                        for (int q = 0; q < 5; ++q) Wp[(long)q * NP + gdst] = Wp[(long)q * NP + gsrc];
                        double *vn = &Wp[(long)(1 + d) * NP + gdst];
                        if (bc == ORC_BC_REFLECT) *vn = -*vn;
                        else if (bc == ORC_BC_OUTFLOW) {
                            /* no inflow: the normal velocity may only point out */
                            if (side == 0) { if (*vn > 0.0) *vn = 0.0; }
                            else { if (*vn < 0.0) *vn = 0.0; }
                        }
                    }
                }
}

/* --------------------------------------------- one stage right-hand side */

/* dU = -sum_d (dt/dx_d) (F_{i+1/2} - F_{i-1/2}), directions summed x, y, z.
 * Each direction term is (F_hi - F_lo) first, then times dt/dx_d.  The face
 * states are the PLM states (order 2) or the two adjacent cell values
 * themselves (order 1, the van Leer predictor). */
static void rhs_order(const orc_mesh *m, const double *U, double dt, int order, double *dU, unsigned *flags) {
    const long N = ncell(m);
    const int nd = m->ndim, nv = 2 + nd;
    const pad_t P = make_pad(m);
    const long NP = (long)P.np[0] * P.np[1] * P.np[2];
    double *Wp = (double *)calloc((size_t)5 * NP, sizeof(double));
    unsigned f = 0;

    /* 1. recover primitives on the interior */
#pragma omp parallel for schedule(static) reduction(|:f)
    for (int k = 0; k < m->n[2]; ++k)
        for (int j = 0; j < m->n[1]; ++j)
            for (int i = 0; i < m->n[0]; ++i) {
                double u[5], w[5];
                gather_cons(m, U, uidx(m, i, j, k), u);
                recover_cell(m, u, w, &f);
                long pc = pidx(&P, i, j, k);
                for (int q = 0; q < 5; ++q) Wp[(long)q * NP + pc] = w[q];
            }
    /* 2. ghost zones */
    for (int d = 0; d < nd; ++d) fill_ghosts_axis(m, &P, Wp, d);

    /* 3. per-direction PLM + HLLC; accumulate flux differences */
#pragma omp parallel for schedule(static)
    for (long q = 0; q < (long)nv * N; ++q) dU[q] = 0.0;
    for (int d = 0; d < nd; ++d) {
        const double dtdx = dt / cell_width(m, d);
        const int n = m->n[d];
        /* transverse velocity slots in increasing axis order */
        int t1 = d == 0 ? 1 : 0;
        int t2 = d == 2 ? 1 : 2;
        int lim[3] = {m->n[0], m->n[1], m->n[2]};
        lim[d] = 1;
        const long npencil = (long)lim[0] * lim[1] * lim[2];
#pragma omp parallel
        {
        double *Fl = (double *)malloc(sizeof(double) * 5 * (size_t)(n + 1));
#pragma omp for schedule(static)
        for (long pen = 0; pen < npencil; ++pen) {
                    /* the pencil's fixed coordinates; coordinate d is swept below */
                    int i = (int)(pen % lim[0]);
                    int j = (int)((pen / lim[0]) % lim[1]);
                    int k = (int)(pen / ((long)lim[0] * lim[1]));
                    /* faces f = 0..n; face f lies between cells f-1 and f */
                    for (int fc = 0; fc <= n; ++fc) {
                        double wl[5], wr[5];
                        /* rotated primitives (rho, v_n, v_t1, v_t2, p) of cells fc-2..fc+1 */
                        double s[4][5];
                        for (int o = 0; o < 4; ++o) {
                            int ci[3] = {i, j, k};
                            ci[d] = fc - 2 + o;
                            long pc = pidx(&P, ci[0], ci[1], ci[2]);
                            s[o][0] = Wp[pc];
                            s[o][1] = Wp[(long)(1 + d) * NP + pc];
                            s[o][2] = Wp[(long)(1 + t1) * NP + pc];
                            s[o][3] = Wp[(long)(1 + t2) * NP + pc];
                            s[o][4] = Wp[(long)4 * NP + pc];
                        }
                        for (int q = 0; q < 5; ++q) {
                            if (order == 1) {
                                wl[q] = s[1][q];
                                wr[q] = s[2][q];
                                continue;
                            }
                            /* left state: cell fc-1 at its upper face */
                            double sl = orc_minmod(s[1][q] - s[0][q], s[2][q] - s[1][q]);
                            wl[q] = s[1][q] + 0.5 * sl;
                            /* right state: cell fc at its lower face */
                            double sr = orc_minmod(s[2][q] - s[1][q], s[3][q] - s[2][q]);
                            wr[q] = s[2][q] - 0.5 * sr;
                        }
                        orc_hllc(m->gamma, wl, wr, &Fl[5 * fc]);
                    }
                    for (int c = 0; c < n; ++c) {
                        int ci[3] = {i, j, k};
                        ci[d] = c;
                        long uc = uidx(m, ci[0], ci[1], ci[2]);
                        const double *Flo = &Fl[5 * c], *Fhi = &Fl[5 * (c + 1)];
                        /* rotated flux slot -> conserved field */
                        double dif[5];
                        for (int q = 0; q < 5; ++q) dif[q] = Fhi[q] - Flo[q];
                        dU[uc] = dU[uc] - dtdx * dif[0];
                        dU[(long)(1 + d) * N + uc] = dU[(long)(1 + d) * N + uc] - dtdx * dif[1];
                        if (t1 < nd) dU[(long)(1 + t1) * N + uc] = dU[(long)(1 + t1) * N + uc] - dtdx * dif[2];
                        if (t2 < nd) dU[(long)(1 + t2) * N + uc] = dU[(long)(1 + t2) * N + uc] - dtdx * dif[3];
                        dU[(long)(nv - 1) * N + uc] = dU[(long)(nv - 1) * N + uc] - dtdx * dif[4];
                    }
        }
        free(Fl);
        }
    }
    free(Wp);
    if (flags) *flags |= f;
}

void orc_rhs(const orc_mesh *m, const double *U, double dt, double *dU, unsigned *flags) {
    rhs_order(m, U, dt, 2, dU, flags);
}

/* --------------------------------------------- Sec. 3.3: one Heun step */

/* Advances U in place by one Heun step and t by dt.  dt comes from U^n
 * (first sub-step only) and is clipped so that t lands exactly on t_end.
 * Returns the dt used. */
double orc_heun_step(const orc_mesh *m, double *U, double *t, double t_end, unsigned *flags) {
    const long NV = (long)(2 + m->ndim) * ncell(m);
    double dt = orc_cfl_dt(m, U, flags);
    int last = 0;
    double rem = t_end - *t;
    if (dt >= rem) { dt = rem; last = 1; }
    double *dU = (double *)malloc(sizeof(double) * (size_t)NV);
    double *U1 = (double *)malloc(sizeof(double) * (size_t)NV);
    /* predictor: U1 = U^n + dt L(U^n) */
    orc_rhs(m, U, dt, dU, flags);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < NV; ++q) U1[q] = U[q] + dU[q];
    /* corrector: U^{n+1} = (U^n + (U1 + dt L(U1))) / 2 */
    orc_rhs(m, U1, dt, dU, flags);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < NV; ++q) U[q] = 0.5 * (U[q] + (U1[q] + dU[q]));
    *t = last ? t_end : *t + dt;
    free(dU);
    free(U1);
    return dt;
}

/* ------------------------------ Sec. 3.3: one memory-optimized van Leer step */

/* Advances U in place by one van Leer predictor-corrector step and t by dt
 * (dt from U^n as in orc_heun_step).
 *   predictor: U^{n+1/2} = U^n + (dt/2) L_1(U^n), first-order face states;
 *              only its primitives W^{n+1/2} are used afterwards
 *   corrector: U^{n+1} = U^n + dt L_2(W^{n+1/2}), PLM face states
 * Returns the dt used. */
double orc_vl2_step(const orc_mesh *m, double *U, double *t, double t_end, unsigned *flags) {
    const long NV = (long)(2 + m->ndim) * ncell(m);
    double dt = orc_cfl_dt(m, U, flags);
    int last = 0;
    double rem = t_end - *t;
    if (dt >= rem) { dt = rem; last = 1; }
    double *dU = (double *)malloc(sizeof(double) * (size_t)NV);
    double *Uh = (double *)malloc(sizeof(double) * (size_t)NV);
    /* predictor: half step with piecewise-constant face states */
    rhs_order(m, U, 0.5 * dt, 1, dU, flags);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < NV; ++q) Uh[q] = U[q] + dU[q];
    /* corrector: PLM on the primitives of U^{n+1/2} (rhs_order recovers them,
     * floors included), full step from U^n */
    rhs_order(m, Uh, dt, 2, dU, flags);
#pragma omp parallel for schedule(static)
    for (long q = 0; q < NV; ++q) U[q] = U[q] + dU[q];
    *t = last ? t_end : *t + dt;
    free(dU);
    free(Uh);
    return dt;
}

/* Steps with the given integrator (0 Heun, 1 van Leer) until t reaches t_end
 * or max_steps steps were taken.  Returns the number of steps; *t is updated. */
long orc_run_with(const orc_mesh *m, double *U, double *t, double t_end, long max_steps, int integrator,
                  unsigned *flags) {
    long s = 0;
    while (*t < t_end && s < max_steps) {
        if (integrator == 1) orc_vl2_step(m, U, t, t_end, flags);
        else orc_heun_step(m, U, t, t_end, flags);
        ++s;
    }
    return s;
}

/* Heun steps until t reaches t_end or max_steps steps were taken. */
long orc_run(const orc_mesh *m, double *U, double *t, double t_end, long max_steps, unsigned *flags) {
    return orc_run_with(m, U, t, t_end, max_steps, 0, flags);
}

/* ------------------------------------ conservation totals (diagnostic) */

/* Neumaier-compensated sum of every conserved field over interior cells. */
void orc_totals(const orc_mesh *m, const double *U, double *out) {
    const long N = ncell(m);
    const int nv = 2 + m->ndim;
    for (int q = 0; q < nv; ++q) {
        double s = 0.0, comp = 0.0;
        for (long c = 0; c < N; ++c) {
            double x = U[(long)q * N + c];
            double t = s + x;
            if (fabs(s) >= fabs(x)) comp += (s - t) + x;
            else comp += (x - t) + s;
            s = t;
        }
        out[q] = s + comp;
    }
}

int orc_abi_version(void) { return 1; }

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP).
 * Per-cell work is independent, the minimum is exact and the totals are
 * serial, so results do not depend on the thread count. */
int orc_set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
