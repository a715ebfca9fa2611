// khy_packed.cuh -- two face fluxes per thread with Blackwell's packed FP32
// instructions (mixed path).
//
// The FP32 part of the mixed stage (PLM + HLLC, Sec. 3.2.2) is most of its
// instructions.  sm_100+ executes FADD2 / FMUL2 / FFMA2: one instruction for
// two independent FP32 operations.  Every face of the mixed path is computed
// by face_flux2 below, two faces per call (the x and y lanes of float2
// values); lanes never mix, so a face has the same bits whichever thread,
// lane or CTA computes it.  Divisions and square roots are per lane on the
// special-function unit; comparisons and branch choices are per-lane selects.
#pragma once

#include "khy_kernels.cuh"

namespace khy {
namespace pk {

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b == a + b * (-1), rounded once: identical to a rounded subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a / b: two special-function reciprocals, one packed multiply
__device__ __forceinline__ float2 div2(float2 a, float2 b) {
    return __fmul2_rn(a, make_float2(rcp_approx(b.x), rcp_approx(b.y)));
}
// sqrt(a) for a >= 1
__device__ __forceinline__ float2 root2_ge1(float2 a) {
    return __fmul2_rn(a, make_float2(rsqrt_approx(a.x), rsqrt_approx(a.y)));
}
__device__ __forceinline__ float2 splat(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sel2(bool cx, bool cy, float2 a, float2 b) {
    return make_float2(cx ? a.x : b.x, cy ? a.y : b.y);
}
__device__ __forceinline__ float2 max2(float2 a, float2 b) { return make_float2(a.x > b.x ? a.x : b.x, a.y > b.y ? a.y : b.y); }

// Float-float pairs of two independent sums (lanes): the same round-to-nearest
// operations as the scalar Knuth TwoSum, so each lane has the scalar's bits.
struct FF2 {
    float2 hi, lo;
};
__device__ __forceinline__ FF2 two_sum2(float2 a, float2 b) {
    const float2 s = add2(a, b);
    const float2 bb = sub2(s, a);
    return {s, add2(sub2(a, sub2(s, bb)), sub2(b, bb))};
}
// exact a - b as a float-float pair: TwoSum(a, -b) without the negation
// (round-to-nearest is symmetric, so the bits are those of TwoSum(a, -b))
__device__ __forceinline__ FF2 two_diff2(float2 a, float2 b) {
    const float2 s = sub2(a, b);
    const float2 bb = sub2(s, a);
    return {s, sub2(sub2(a, sub2(s, bb)), add2(b, bb))};
}
__device__ __forceinline__ FF2 ff_add2(FF2 a, FF2 b) {
    const FF2 s = two_sum2(a.hi, b.hi);
    const float2 e = add2(s.lo, add2(a.lo, b.lo));
    const float2 hi = add2(s.hi, e);
    return {hi, sub2(e, sub2(hi, s.hi))};
}
// a + b + c of three exact pairs as hi + lo without the renormalisation
// (|lo| stays within a few units of hi's last place): the leading parts are
// summed by two TwoSums and every error term is collected in lo -- for an
// FP64 update that adds the two parts as separate doubles.
__device__ __forceinline__ FF2 ff_sum3_unnorm(FF2 a, FF2 b, FF2 c) {
    const FF2 t = two_sum2(a.hi, b.hi), u = two_sum2(t.hi, c.hi);
    return {u.hi, add2(add2(add2(a.lo, b.lo), add2(c.lo, t.lo)), u.lo)};
}
__device__ __forceinline__ FF2 ff_sum2_unnorm(FF2 a, FF2 b) {
    const FF2 t = two_sum2(a.hi, b.hi);
    return {t.hi, add2(add2(a.lo, b.lo), t.lo)};
}

// a clamped to [lo, hi] per lane: with lo = min(b, 0), hi = max(b, 0) this is
// minmod(a, b) of Eq. 3 (the value of the smaller magnitude when a and b share
// a sign, otherwise 0; b when |a| = |b|) in two min/max operations per lane
// once the bounds, which both sides of a face share, are formed
__device__ __forceinline__ float2 clamp2(float2 a, float2 lo, float2 hi) {
    return make_float2(fminf(fmaxf(a.x, lo.x), hi.x), fminf(fmaxf(a.y, lo.y), hi.y));
}

// HLLC flux of two faces (lanes), rotated primitives (rho, u, t_1..t_NT, p):
// the same estimate of p* (PVRS, two-shock above both pressures), the same
// Eq. 4 / Eq. 5 speeds and the same branch order as the scalar hllc(), with
// the algebra arranged for few instructions: the star-state energy
// rho*_K E*_K / rho*_K = rho_K Delta s_K / (s_K - s*) (E_K / rho_K + (s* - u_K)
// (s* + p_K / (rho_K Delta s_K))) is formed as (Delta s_K E_K + (s* - u_K)
// (m_K s* + p_K)) / (s_K - s*) with m_K = rho_K Delta s_K (no reciprocal of
// rho_K or m_K), the transverse momentum fluxes are the mass flux times the
// upwind transverse velocity, and the two-shock weights are reciprocal
// square roots of (p* + B_K) / A_K.
template <int NT>
__device__ __forceinline__ void hllc2(const Consts<float> &k, const float2 (&wl)[NT + 3], const float2 (&wr)[NT + 3],
                                      float2 (&F)[NT + 3]) {
    constexpr int P = NT + 2;
    const float2 rl = wl[0], ul = wl[1], pl = wl[P];
    const float2 rr = wr[0], ur = wr[1], pr = wr[P];
    // c = sqrt(gamma p / rho) = a rsqrt(a rho) with a = gamma p: one
    // special-function operation per lane (a rho is clamped to the smallest
    // normal float, so a = 0 gives c = 0)
    const float2 g = splat(k.gamma);
    const float2 al = mul2(g, pl), ar = mul2(g, pr);
    const float2 xl = max2(mul2(al, rl), splat(1.17549435e-38f)), xr = max2(mul2(ar, rr), splat(1.17549435e-38f));
    const float2 cl = mul2(al, make_float2(rsqrt_approx(xl.x), rsqrt_approx(xl.y)));
    const float2 cr = mul2(ar, make_float2(rsqrt_approx(xr.x), rsqrt_approx(xr.y)));
    const float2 du = sub2(ur, ul);
    // p_pvrs = (p_L + p_R)/2 - (u_R - u_L)(rho_L + rho_R)(c_L + c_R)/8
    const float2 ppv = mul2(splat(0.5f), fma2(mul2(du, add2(rl, rr)), mul2(splat(-0.25f), add2(cl, cr)), add2(pl, pr)));
    float2 pstar = max2(ppv, splat(0.f));
    const float2 pmax = max2(pl, pr);
    const bool tx = pstar.x > pmax.x, ty = pstar.y > pmax.y;
    if (tx || ty) {  // both waves shocks in at least one lane: two-shock estimate
        // g_K = sqrt(A_K / (p* + B_K)), A_K = 2 / ((gamma + 1) rho_K), B_K = (gamma - 1)/(gamma + 1) p_K
        const float2 hgp1 = splat(k.hgp1), gg = splat(k.gm1_gp1);
        const float2 yl = mul2(fma2(gg, pl, pstar), mul2(hgp1, rl));
        const float2 yr = mul2(fma2(gg, pr, pstar), mul2(hgp1, rr));
        const float2 gl = make_float2(rsqrt_approx(yl.x), rsqrt_approx(yl.y));
        const float2 gr = make_float2(rsqrt_approx(yr.x), rsqrt_approx(yr.y));
        const float2 pts = div2(sub2(fma2(gl, pl, mul2(gr, pr)), du), add2(gl, gr));
        pstar = sel2(tx, ty, pts, pstar);
    }
    const float2 one = splat(1.f);
    const float2 ratl = max2(div2(pstar, pl), one);
    const float2 ratr = max2(div2(pstar, pr), one);
    const float2 ql = root2_ge1(fma2(splat(k.g1), sub2(ratl, one), one));  // rat >= 1
    const float2 qr = root2_ge1(fma2(splat(k.g1), sub2(ratr, one), one));
    // Eq. 4: Delta s_K = s_K - u_K straight from c_K q_K
    const float2 dsl = mul2(mul2(splat(-1.f), cl), ql);
    const float2 dsr = mul2(cr, qr);
    const float2 sl = add2(ul, dsl);
    const float2 sr = add2(ur, dsr);
    // m_K = rho_K Delta s_K, then Eq. 5:
    // s* = (p_R - p_L + u_L m_L - u_R m_R) / (m_L - m_R)
    const float2 ml = mul2(rl, dsl), mr = mul2(rr, dsr);
    const float2 sstar = div2(sub2(fma2(ul, ml, sub2(pr, pl)), mul2(ur, mr)), sub2(ml, mr));
    // branch order: 0 <= s_L -> F_L; 0 <= s* -> F*_L; 0 < s_R -> F*_R; else F_R
    const bool lx = (0.f <= sl.x) || (0.f <= sstar.x), ly = (0.f <= sl.y) || (0.f <= sstar.y);
    const bool ox = lx ? (0.f <= sl.x) : !(0.f < sr.x), oy = ly ? (0.f <= sl.y) : !(0.f < sr.y);
    float2 w[NT + 3];
#pragma unroll
    for (int j = 0; j < NT + 3; ++j) w[j] = sel2(lx, ly, wl[j], wr[j]);
    const float2 rk = w[0], uk = w[1], pk = w[P];
    const float2 sk = sel2(lx, ly, sl, sr);
    const float2 mk = sel2(lx, ly, ml, mr);
    const float2 dsk = sel2(lx, ly, dsl, dsr);
    float2 vsq = mul2(uk, uk);
#pragma unroll
    for (int j = 0; j < NT; ++j) vsq = fma2(w[2 + j], w[2 + j], vsq);
    const float2 E = fma2(mul2(splat(0.5f), rk), vsq, mul2(pk, splat(k.igm1)));
    const float2 mf = mul2(rk, uk);
    // F_K, and F = F_K + s_K (U*_K - U_K) with s_K and r = 1 / (s_K - s*)
    // zeroed where F_K itself is the flux (supersonic lanes: the correction
    // vanishes exactly and stays finite)
    const float2 zero = splat(0.f);
    const float2 skm = sel2(ox, oy, zero, sk);
    const float2 dss = sub2(sk, sstar);
    const float2 r = sel2(ox, oy, zero, make_float2(rcp_approx(dss.x), rcp_approx(dss.y)));
    const float2 fac = mul2(mk, r);  // rho*_K
    const float2 sd0 = mul2(skm, sub2(fac, rk));
    F[0] = add2(mf, sd0);
    F[1] = fma2(skm, sub2(mul2(fac, sstar), mf), fma2(mf, uk, pk));
#pragma unroll
    for (int j = 0; j < NT; ++j) F[2 + j] = mul2(F[0], w[2 + j]);
    // rho*_K E*_K / rho*_K as (Delta s_K E_K + (s* - u_K)(m_K s* + p_K)) r
    const float2 facX = mul2(r, fma2(sub2(sstar, uk), fma2(mk, sstar, pk), mul2(dsk, E)));
    F[P] = fma2(skm, sub2(facX, E), mul2(add2(E, pk), uk));
}

// Storage slot of rotated component j (0 rho, 1 normal velocity, 2..ND
// transverse velocities in increasing axis order, ND+1 pressure) for a face
// normal to direction dir.
template <int ND>
__device__ __forceinline__ int rot_slot(int dir, int j) {
    if (j == 0) return 0;
    if (j == ND + 1) return ND + 1;
    if (j == 1) return 1 + dir;
    if (j == 2) return 1 + (dir == 0 ? 1 : 0);
    return 1 + (dir == 2 ? 1 : 2);
}

// Two face fluxes (lanes) from two four-cell stencils already rotated onto
// their face normals: packed minmod PLM (or, PLM = false, the first-order
// states of the van Leer predictor), then packed HLLC.  Fr is in rotated
// order (mass, normal momentum, transverse momenta, energy).
template <int ND, bool PLM = true>
__device__ __forceinline__ void face_flux2(const float2 (&st)[4][ND + 2], const Consts<float> &k, float2 (&Fr)[ND + 2]) {
    constexpr int NT = ND - 1;
    float2 wl[NT + 3], wr[NT + 3];
    const float2 half = splat(0.5f), mhalf = splat(-0.5f);
#pragma unroll
    for (int j = 0; j < ND + 2; ++j) {
        if (!PLM) {
            wl[j] = st[1][j];
            wr[j] = st[2][j];
            continue;
        }
        // minmod (Eq. 3) of the difference across the face with the one on
        // either side, as clamps to the interval between 0 and the face
        // difference (the bounds are shared by both sides)
        const float2 d12 = sub2(st[2][j], st[1][j]);
        const float2 lo = make_float2(fminf(d12.x, 0.f), fminf(d12.y, 0.f));
        const float2 hi = make_float2(fmaxf(d12.x, 0.f), fmaxf(d12.y, 0.f));
        wl[j] = fma2(clamp2(sub2(st[1][j], st[0][j]), lo, hi), half, st[1][j]);
        wr[j] = fma2(clamp2(sub2(st[3][j], st[2][j]), lo, hi), mhalf, st[2][j]);
    }
    hllc2<NT>(k, wl, wr, Fr);
}

}  // namespace pk
}  // namespace khy
