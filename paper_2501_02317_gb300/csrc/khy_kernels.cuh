// khy_kernels.cuh -- device building blocks of the Godunov hydro step
// (sm_103a): geometry and clock records, the ghost-zone index map
// (Sec. 3.1.1), the FP64 primitive recovery and CFL candidate (Sec. 3.1), the
// minmod limiter (Eq. 3), the HLLC flux (Eq. 4, Eq. 5) and the PLM face flux
// (Sec. 3.2.2).  The stage kernel that puts them together is khy_stage.cuh.
//
// Everything here evaluates floating-point operations in the same order as
// the CPU reference.  In the FP64 translation unit (built with -fmad=false)
// that makes the two agree to the last bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace khy {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_FREE = 2, BC_REFLECT = 3 };
enum : unsigned { FLAG_NONPHYSICAL = 1u, FLAG_FLOOR = 2u, FLAG_DT_UNDERFLOW = 4u };

// Mesh geometry and method constants, passed by value to every kernel.
struct Geom {
    int ndim;
    int n[3];
    int bc[3][2];
    long long ncell;
    double dx[3];
    double gamma;
    double gm1;          // gamma - 1
    double g1;           // (gamma + 1) / (2 gamma)        (Eq. 5)
    double gp1;          // gamma + 1
    double gm1_gp1;      // (gamma - 1) / (gamma + 1)      (two-shock estimate)
    double cfl;
    double rho_floor;
    double p_floor;
    // the same constants rounded to FP32 on the host (for the FP32 kernels:
    // read from the parameter bank instead of converted on the device)
    float f_gamma, f_gm1, f_g1, f_gp1, f_gm1_gp1, f_igm1;  // f_igm1 = 1 / (gamma - 1)
    float f_rho_floor, f_p_floor;
    float f_dx[3];
};

// Device-resident step state.  Written only by clock_kernel (and the host
// between launches); read by the stage kernels.
struct Clock {
    double t;
    double t_end;
    double dt;
    double dtdx[3];                  // dt / dx_d of the current step
    unsigned long long wmin_bits;    // atomicMin target: bits of min dx/(|v|+c) (> 0)
    long long steps;                 // steps taken
    long long max_steps;             // absolute step limit
    int active;                      // 1 while the current step runs
    unsigned status;                 // FLAG_* bits, latched
    unsigned long long floor_hits;   // floor applications on interior cells
};

constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

// Start of a Heun step for one grid (Sec. 3.1: dt on the first sub-step
// only): dt = C * (accumulated CFL minimum), clipped so the step lands on
// t_end; advances t and the step counter, arms the stage kernels and resets
// the minimum for the stage-2 launch.  Inactive once t >= t_end, the step
// limit is reached or dt underflowed.
__device__ __forceinline__ void clock_step(Clock *c, const Geom &g) {
    if (!(c->t < c->t_end) || c->steps >= c->max_steps || (c->status & FLAG_DT_UNDERFLOW)) {
        c->active = 0;
        return;
    }
    const double w = __longlong_as_double((long long)c->wmin_bits);
    double dt = g.cfl * w;
    int last = 0;
    const double rem = c->t_end - c->t;
    if (dt >= rem) {
        dt = rem;
        last = 1;
    }
    if (!(dt > 1e-300) || !(dt < INFINITY)) {
        c->status |= FLAG_DT_UNDERFLOW;
        c->active = 0;
        return;
    }
    c->dt = dt;
    c->dtdx[0] = dt / g.dx[0];
    c->dtdx[1] = dt / g.dx[1];
    c->dtdx[2] = dt / g.dx[2];
    c->t = last ? c->t_end : c->t + dt;
    c->steps += 1;
    c->active = 1;
    c->wmin_bits = kInfBits;
}

// ------------------------------------------------------------ Sec. 3.1.1
// Maps coordinate x (possibly a ghost) onto an interior index along an axis
// with n cells and boundary rules (lo, hi).  *act receives the velocity rule
// for the normal component: 0 none, 1 negate (reflect), 2 min(v,0) (outflow,
// low side), 3 max(v,0) (outflow, high side).  Ghosts within two cells follow
// the boundary rules exactly; farther cells (only used by faces outside the
// interior) are clamped into range.  Callers pass -n <= x < 2n (a halo of two
// cells around a tile of an axis with n >= 2 cells), so the periodic wrap is
// one add or subtract.
__device__ __forceinline__ int bc_map(int x, int n, int lo, int hi, int *act) {
    *act = 0;
    if (x >= 0 && x < n) return x;
    if (x < 0) {
        if (lo == BC_PERIODIC) return x + n;
        if (lo == BC_REFLECT) { *act = 1; int s = -x - 1; return s < n ? s : n - 1; }
        if (lo == BC_OUTFLOW) *act = 2;
        return 0;
    }
    if (hi == BC_PERIODIC) return x - n;
    if (hi == BC_REFLECT) { *act = 1; int s = 2 * n - 1 - x; return s >= 0 ? s : 0; }
    if (hi == BC_OUTFLOW) *act = 3;
    return n - 1;
}

__device__ __forceinline__ double apply_vrule(double v, int act) {
    if (act == 1) return -v;
    if (act == 2) return v > 0.0 ? 0.0 : v;
    if (act == 3) return v < 0.0 ? 0.0 : v;
    return v;
}

// ------------------------------------------------------------ Sec. 3.1
// Conserved -> primitive, FP64, floors on the primitive only.  Operation
// order: v_d = m_d / rho; ke = (0.5 rho) ((v_0^2 + v_1^2) + v_2^2);
// p = (gamma - 1)(E - ke).
template <int ND>
__device__ __forceinline__ void recover(const double (&u)[ND + 2], const Geom &g, double (&w)[ND + 2],
                                        unsigned &flags, unsigned &floors) {
    double rho = u[0];
    if (!(rho > 0.0)) flags |= FLAG_NONPHYSICAL;
    if (rho < g.rho_floor) { rho = g.rho_floor; flags |= FLAG_FLOOR; ++floors; }
    double v[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) v[d] = u[1 + d] / rho;
    double s = v[0] * v[0];
#pragma unroll
    for (int d = 1; d < ND; ++d) s = s + v[d] * v[d];
    double ke = 0.5 * rho * s;
    double eint = u[ND + 1] - ke;
    if (!(eint >= 0.0)) flags |= FLAG_NONPHYSICAL;
    double p = g.gm1 * eint;
    if (p < g.p_floor) { p = g.p_floor; flags |= FLAG_FLOOR; ++floors; }
    w[0] = rho;
#pragma unroll
    for (int d = 0; d < ND; ++d) w[1 + d] = v[d];
    w[ND + 1] = p;
}

// CFL candidate of one cell: min_d dx_d / (|v_d| + c_s), c_s = sqrt(gamma p / rho).
template <int ND>
__device__ __forceinline__ double cfl_candidate(const double (&w)[ND + 2], const Geom &g) {
    double cs = sqrt(g.gamma * w[ND + 1] / w[0]);
    double m = g.dx[0] / (fabs(w[1]) + cs);
#pragma unroll
    for (int d = 1; d < ND; ++d) {
        double t = g.dx[d] / (fabs(w[1 + d]) + cs);
        if (t < m) m = t;
    }
    return m;
}

// ------------------------------------------------------------ Eq. 3
template <class R>
__device__ __forceinline__ R minmod(R a, R b) {
    bool same = (a > R(0) && b > R(0)) || (a < R(0) && b < R(0));
    if (!same) return R(0);
    return fabs(a) < fabs(b) ? a : b;
}

template <class R>
struct Consts {
    R gamma, gm1, g1, gp1, gm1_gp1;
    R igm1;  // 1 / (gamma - 1), FP32 path only
    R hgp1;  // (gamma + 1) / 2, FP32 path only
};

template <class R>
__device__ __forceinline__ Consts<R> make_consts(const Geom &g) {
    Consts<R> c;
    if constexpr (sizeof(R) == 4) {
        c.gamma = g.f_gamma; c.gm1 = g.f_gm1; c.g1 = g.f_g1; c.gp1 = g.f_gp1; c.gm1_gp1 = g.f_gm1_gp1;
        c.igm1 = g.f_igm1;
        c.hgp1 = 0.5f * g.f_gp1;  // exact
    } else {
        c.gamma = g.gamma; c.gm1 = g.gm1; c.g1 = g.g1; c.gp1 = g.gp1; c.gm1_gp1 = g.gm1_gp1;
        c.igm1 = 0.0;  // the FP64 flux divides by gamma - 1, as the reference does
        c.hgp1 = 0.0;
    }
    return c;
}

// ------------------------------------------------------------ pinned arithmetic
// Every floating-point operation of the face flux goes through these
// round-to-nearest intrinsics, so the compiler cannot fuse or reorder them:
// a face flux computed by two different CTAs (or two unrolled copies of a
// loop) from the same inputs has the same bits, which is what makes the
// flux-difference update conservative to round-off.
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rroot(double a) { return __dsqrt_rn(a); }
// FP32 (mixed path): division and square root use the special-function
// unit's approximate reciprocal (max error 1 ulp) and reciprocal square root
// (relative error below 2^-22.9), one instruction each, with subnormals
// flushed (PTX rcp.approx.ftz / rsqrt.approx.ftz); far inside the mixed
// path's tolerance, and still pure functions of their inputs, so redundant
// face fluxes stay bitwise identical.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fmul_rn(a, rcp_approx(b)); }
__device__ __forceinline__ float rroot(float a) { return a > 0.f ? __fmul_rn(a, rsqrt_approx(a)) : 0.f; }
// square root of an argument known to be >= 1 (no zero guard)
__device__ __forceinline__ float rroot_ge1(float a) { return __fmul_rn(a, rsqrt_approx(a)); }

// ------------------------------------------------------------ Sec. 3.2.2
// HLLC flux for rotated primitive states w = (rho, u, t_1..t_NT, p), NT
// transverse velocity components.  Output F = (mass, normal momentum,
// transverse momenta, energy).  Operation order as in the CPU reference.
template <class R, int NT>
__device__ __forceinline__ void hllc(const Consts<R> &k, const R (&wl)[NT + 3], const R (&wr)[NT + 3],
                                     R (&F)[NT + 3]) {
    constexpr int P = NT + 2;  // pressure slot
    const R rl = wl[0], ul = wl[1], pl = wl[P];
    const R rr = wr[0], ur = wr[1], pr = wr[P];
    const R cl = rroot(rdiv(rmul(k.gamma, pl), rl));
    const R cr = rroot(rdiv(rmul(k.gamma, pr), rr));
    // p* estimate: PVRS clamped at 0; the two-shock estimate when both waves are shocks
    const R ppv = rsub(rmul(R(0.5), radd(pl, pr)),
                       rmul(rmul(rmul(R(0.125), rsub(ur, ul)), radd(rl, rr)), radd(cl, cr)));
    R pstar = ppv > R(0) ? ppv : R(0);
    const R pmax = pl > pr ? pl : pr;
    if (pstar > pmax) {
        const R gl = rroot(rdiv(rdiv(R(2), rmul(k.gp1, rl)), radd(pstar, rmul(k.gm1_gp1, pl))));
        const R gr = rroot(rdiv(rdiv(R(2), rmul(k.gp1, rr)), radd(pstar, rmul(k.gm1_gp1, pr))));
        pstar = rdiv(rsub(radd(rmul(gl, pl), rmul(gr, pr)), rsub(ur, ul)), radd(gl, gr));
    }
    R ratl = rdiv(pstar, pl), ratr = rdiv(pstar, pr);
    if (ratl < R(1)) ratl = R(1);
    if (ratr < R(1)) ratr = R(1);
    // Eq. 5: q_K and the subtraction-safe offsets ds_K = s_K - u_K
    const R ql = rroot(radd(R(1), rmul(k.g1, rsub(ratl, R(1)))));
    const R qr = rroot(radd(R(1), rmul(k.g1, rsub(ratr, R(1)))));
    const R dsl = rmul(-cl, ql);
    const R dsr = rmul(cr, qr);
    const R sl = radd(ul, dsl);
    const R sr = radd(ur, dsr);
    // Eq. 4 with s_K - u_K replaced by ds_K
    const R sstar = rdiv(rsub(rsub(pr, rmul(rmul(rr, ur), dsr)), rsub(pl, rmul(rmul(rl, ul), dsl))),
                         rsub(rmul(rl, dsl), rmul(rr, dsr)));

    // Branches in the reference order: 0 <= s_L -> F_L; 0 <= s* -> F*_L;
    // 0 < s_R -> F*_R; else F_R.  Only the selected side's states are built.
    const bool left = (R(0) <= sl) || (R(0) <= sstar);
    const bool outside = left ? (R(0) <= sl) : !(R(0) < sr);
    R w[NT + 3];
#pragma unroll
    for (int j = 0; j < NT + 3; ++j) w[j] = left ? wl[j] : wr[j];
    const R rk = w[0], uk = w[1], pk = w[P];
    const R sk = left ? sl : sr;
    const R dsk = left ? dsl : dsr;
    R vsq = rmul(uk, uk);
#pragma unroll
    for (int j = 0; j < NT; ++j) vsq = radd(vsq, rmul(w[2 + j], w[2 + j]));
    const R E = radd(rdiv(pk, k.gm1), rmul(rmul(R(0.5), rk), vsq));
    const R mf = rmul(rk, uk);
    R Uk[NT + 3], Fk[NT + 3];
    Uk[0] = rk;
    Uk[1] = rmul(rk, uk);
    Fk[0] = mf;
    Fk[1] = radd(rmul(mf, uk), pk);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        Uk[2 + j] = rmul(rk, w[2 + j]);
        Fk[2 + j] = rmul(mf, w[2 + j]);
    }
    Uk[P] = E;
    Fk[P] = rmul(radd(E, pk), uk);
    if (outside) {
#pragma unroll
        for (int q = 0; q < NT + 3; ++q) F[q] = Fk[q];
        return;
    }
    const R fac = rdiv(rmul(rk, dsk), rsub(sk, sstar));
    R Us[NT + 3];
    Us[0] = fac;
    Us[1] = rmul(fac, sstar);
#pragma unroll
    for (int j = 0; j < NT; ++j) Us[2 + j] = rmul(fac, w[2 + j]);
    Us[P] = rmul(fac, radd(rdiv(Uk[P], rk), rmul(rsub(sstar, uk), radd(sstar, rdiv(pk, rmul(rk, dsk))))));
#pragma unroll
    for (int q = 0; q < NT + 3; ++q) F[q] = radd(Fk[q], rmul(sk, rsub(Us[q], Uk[q])));
}

// Face flux from the four primitive cells around a face along direction dir
// (cells f-2, f-1 | f, f+1), primitives in storage order (rho, v_0.., p).
// Minmod PLM per primitive (undivided differences: minmod is positively
// homogeneous, so the dx factors of the slope cancel), then HLLC in the frame
// rotated onto dir.  F is returned in conserved order (mass, m_0.., E).
// PLM = false: first-order face states (the two adjacent cells themselves),
// as in the predictor of the van Leer integrator (Sec. 3.3).
template <int ND, class R, bool PLM = true>
__device__ __forceinline__ void face_flux(const R (&s)[4][ND + 2], int dir, const Consts<R> &k, R (&F)[ND + 2]) {
    constexpr int NT = ND - 1;
    // rotation: storage slot of rotated component j (0 rho, 1 normal, 2.. transverse, last p)
    int slot[ND + 2];
    slot[0] = 0;
    slot[1] = 1 + dir;
    if (ND >= 2) slot[2] = 1 + (dir == 0 ? 1 : 0);
    if (ND >= 3) slot[3] = 1 + (dir == 2 ? 1 : 2);
    slot[ND + 1] = ND + 1;
    R wl[NT + 3], wr[NT + 3];
#pragma unroll
    for (int j = 0; j < ND + 2; ++j) {
        const int q = slot[j];
        const R s0 = s[0][q], s1 = s[1][q], s2 = s[2][q], s3 = s[3][q];
        if (!PLM) {
            wl[j] = s1;
            wr[j] = s2;
            continue;
        }
        const R a = minmod<R>(rsub(s1, s0), rsub(s2, s1));
        wl[j] = radd(s1, rmul(R(0.5), a));
        const R b = minmod<R>(rsub(s2, s1), rsub(s3, s2));
        wr[j] = rsub(s2, rmul(R(0.5), b));
    }
    R Fr[NT + 3];
    hllc<R, NT>(k, wl, wr, Fr);
#pragma unroll
    for (int j = 0; j < ND + 2; ++j) F[slot[j]] = Fr[j];
}

}  // namespace khy
