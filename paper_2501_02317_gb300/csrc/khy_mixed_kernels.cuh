// khy_mixed_kernels.cuh -- device functions of the mixed-precision path (Sec. 3.2.2),
// shaped for GB300, whose FP64 pipe retires about 1.6 operations per clock
// per SM against about 117 FP32 FMAs.  Every FP64 operation that the method
// does not need is moved off that pipe:
//
//   * FP64 <-> FP32 conversions are done with integer instructions (the
//     hardware conversions issue on the FP64 pipe).
//   * Primitive recovery (Sec. 3.1) keeps the cancellation-prone internal
//     energy E - |m|^2/(2 rho) at FP64 accuracy without FP64 instructions:
//     the FP64 conserved values are split into FP32 pairs with integer
//     operations, |m|^2 and the kinetic energy are formed as pairs from
//     exact FMA errors and an error-free sum, and the cancelling difference
//     is exact (Sterbenz); the density, velocities and the pressure leave it
//     as FP32 primitives.
//   * Flux differences: per cell and field, the six FP32 face fluxes are
//     summed error-free as a float-float pair (Knuth TwoSum); the first
//     stage turns the pair into one double with integer operations and a
//     scaled conversion of lo, and costs one fused multiply-add per field
//     (U + c S); the Heun average adds the pair's two exact doubles to the
//     stored V = (Un + U1)/2 with two; each face flux still enters its two
//     cells with opposite signs to full FP64 precision.
//   * The CFL minimum for the next step is taken in FP32 from the recovered
//     primitives of the new state.
//
// The stage kernel that uses these functions is khy_stage.cuh.
#pragma once

#include "khy_kernels.cuh"

namespace khy {
namespace mx {

// ---------------------------------------------------------------- conversions
// double -> float, round to nearest even; results below the float normal
// range flush to zero, above it become +-inf; NaN stays NaN.
__device__ __forceinline__ float d2f(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu) - 896;  // float biased exponent
    const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1FFFFFFFu;
    unsigned f = sign | ((unsigned)e << 23) | m;
    f += (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));  // carry may reach the exponent
    if (e <= 0) f = sign;                                           // underflow: flush to zero
    if (e >= 255) f = sign | 0x7F800000u | ((((hi & 0x7FF00000u) == 0x7FF00000u) && ((hi & 0xFFFFFu) | lo)) ? 0x400000u : 0u);
    return __uint_as_float(f);
}

// float -> double for the flux sums and reciprocals of the update: exact for
// zero and normal floats; a subnormal float (below 1.2e-38) maps to a double
// of the same sign below 2^-126, and inf / NaN to a finite double of magnitude
// >= 2^128 (a non-finite flux only comes from a state the recovery has
// already flagged).  Four integer operations instead of the FP64 pipe's
// conversion.
__device__ __forceinline__ double f2d_fast(float x) {
    const unsigned f = __float_as_uint(x);
    const unsigned a = f & 0x7FFFFFFFu;
    // exponent re-bias 127 -> 1023 is + (896 << 20) on the high word
    const unsigned hi = (a == 0u ? 0u : (a >> 3) + 0x38000000u) | (f & 0x80000000u);
    return __hiloint2double((int)hi, (int)(f << 29));
}

// hi + lo of a float-float pair (|lo| <= ulp(hi)/2, as TwoSum and its
// renormalisation produce) as one double: lo is scaled by a power of two
// into units of the last place of the double of hi (the scale carries hi's
// sign, so the count is signed relative to hi's magnitude), rounded to an
// integer (exact when the exponents differ by at most 29, otherwise the
// nearest unit: the sum rounded below 2^-52 relative) and added to the
// double's bits; from an exact power of two a negative count drops a binade,
// where the unit halves.  For |hi| below 2^-75 (the scale would leave FP32's
// range) lo is dropped.  Replaces an FP64 add in the update.
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
    const unsigned H = __float_as_uint(hi);
    // scale 2^(52 - e) with e hi's unbiased exponent: biased 306 - eh, at most 254
    const unsigned es = min(306u - ((H >> 23) & 0xFFu), 254u);
    int m = __float2int_rn(__fmul_rn(lo, __uint_as_float((es << 23) | (H & 0x80000000u))));
    if ((H & 0x7FFFFFu) == 0u && m < 0) m += m;
    return __longlong_as_double(__double_as_longlong(f2d_fast(hi)) + (long long)m);
}

// x / 2 by decrementing the exponent with integer operations: exact for
// |x| >= 2^-1021 (where halving is exact in FP64 as well); zeros keep their
// sign, smaller magnitudes flush to a signed zero; Inf and NaN pass through.
// Replaces an FP64 multiply in the Heun average.
__device__ __forceinline__ double half_exact(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned e = (unsigned)hi & 0x7FF00000u;
    int h = hi - 0x00100000, l = lo;
    if (e <= 0x00100000u) {
        h = hi & (int)0x80000000u;
        l = 0;
    }
    if (e == 0x7FF00000u) h = hi;
    return __hiloint2double(h, l);
}

// |x| -> float rounded toward zero, for estimates only (the CFL candidate of
// the van Leer corrector): magnitudes below 2^-126 flush to zero; |x| must
// stay below 2^128.
__device__ __forceinline__ float abs_d2f_rz(double x) {
    const unsigned a = (unsigned)__double2hiint(x) & 0x7FFFFFFFu;
    const unsigned lo = (unsigned)__double2loint(x);
    const unsigned f = ((a - 0x38000000u) << 3) | (lo >> 29);
    return __uint_as_float(a < 0x38100000u ? 0u : f);
}
__device__ __forceinline__ float abs_d2f_rz(float x) { return fabsf(x); }

// float -> double, exact for normal floats (subnormals flush to zero).
__device__ __forceinline__ double f2d(float x) {
    const unsigned f = __float_as_uint(x);
    const unsigned sign = f & 0x80000000u;
    const unsigned e = (f >> 23) & 0xFFu;
    const unsigned m = f & 0x7FFFFFu;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    if (e == 0) hi = sign;
    if (e == 255) hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
    const unsigned lo = (e == 0) ? 0u : (m << 29);
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// ---------------------------------------------------------------- float-float
struct FF {
    float hi, lo;
};

// exact: a + b == hi + lo
__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    FF s = two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s.hi, e);
    return {hi, __fsub_rn(e, __fsub_rn(hi, s.hi))};
}

// FP64 value -> pair of FP32 values with integer operations only: hi is x
// truncated to FP32's 24 significant bits, lo holds the next 23 bits, so
// x = hi + lo + d with |d| < 2^-46 |x| (hi and lo carry x's sign; |lo| <
// ulp(hi)).  |x| below 2^-126 gives hi = lo = 0 and below 2^-103 lo = 0;
// |x| must stay below 2^128 -- the recovery flags larger and non-finite
// states before it uses the pair.
__device__ __forceinline__ FF split_d(double x) {
    const unsigned H = (unsigned)__double2hiint(x), L = (unsigned)__double2loint(x);
    const unsigned sgn = H & 0x80000000u, a = H & 0x7FFFFFFFu;
    // exponent re-bias 1023 -> 127 on the high word, then 20 + 3 mantissa bits
    const unsigned fh = __funnelshift_l(L, a - 0x38000000u, 3);
    const float hi = __uint_as_float((a < 0x38100000u ? 0u : fh) | sgn);
    // the 29 bits below hi: their top 23 as a float in [0, 1) (exact
    // subtraction of the implicit one), scaled by 2^(e - 1046), e the
    // biased FP64 exponent
    const float f = __fsub_rn(__uint_as_float(0x3F800000u | ((L >> 6) & 0x7FFFFFu)), 1.0f);
    const int eb = (int)(a >> 20) - 919;
    const float sc = __uint_as_float(((unsigned)max(eb, 0) << 23) | sgn);
    return {hi, __fmul_rn(f, sc)};
}

// ---------------------------------------------------------------- constants
struct MixConsts {
    float gamma, gm1, g1, gp1, gm1_gp1;
    float rho_floor, p_floor;
    long long rho_floor_bits;
    double rho_floor_d;
    float rho_floor_hi, rho_floor_lo;  // the FP64 density floor as an FP32 pair (split_d)
    float dx[3];
};

__device__ __forceinline__ MixConsts make_mix(const Geom &g) {
    MixConsts k;
    k.gamma = g.f_gamma; k.gm1 = g.f_gm1; k.g1 = g.f_g1; k.gp1 = g.f_gp1;
    k.gm1_gp1 = g.f_gm1_gp1;
    k.rho_floor = g.f_rho_floor; k.p_floor = g.f_p_floor;
    k.rho_floor_d = g.rho_floor;
    k.rho_floor_bits = __double_as_longlong(g.rho_floor);
    const FF fl = split_d(g.rho_floor);
    k.rho_floor_hi = fl.hi;
    k.rho_floor_lo = fl.lo;
    k.dx[0] = g.f_dx[0]; k.dx[1] = g.f_dx[1]; k.dx[2] = g.f_dx[2];
    return k;
}

// ---------------------------------------------------------------- Sec. 3.1
// Conserved (FP64) -> primitive (FP32), with the internal energy
// E - |m|^2 / (2 rho) at FP64 accuracy and no FP64 instruction: every
// conserved value is split exactly enough into an FP32 pair (split_d,
// 2^-46), |m|^2 is formed as a pair from the exact errors of the squares
// (FMA) and an error-free sum, 1/rho is the special-function reciprocal r0
// with its Newton residual e = 1 - rho r0 applied to the kinetic energy, and
// E - ke is taken with its leading difference exact (where the two cancel
// they are within a factor of two: Sterbenz' lemma).  The internal energy
// carries a few units of 2^-24 eint + 2^-44 |m|^2 / rho, the error of an
// FP64 recovery with a one-step Newton reciprocal.  Floors on the primitive
// only; the density floor is compared on the FP64 value.
template <int ND>
__device__ __forceinline__ void recover(const double (&u)[ND + 2], const MixConsts &k, float (&w)[ND + 2],
                                        unsigned &flags, unsigned &floors) {
    FF s[ND + 2];
    unsigned amax = 0u;
#pragma unroll
    for (int q = 0; q < ND + 2; ++q) {
        s[q] = split_d(u[q]);
        amax = max(amax, (unsigned)__double2hiint(u[q]) & 0x7FFFFFFFu);
    }
    // |q| >= 2^128, Inf or NaN anywhere: not a physical state
    if (amax >= 0x47F00000u) flags |= FLAG_NONPHYSICAL;
    const long long rb = __double_as_longlong(u[0]);
    if (rb <= 0) flags |= FLAG_NONPHYSICAL;  // rho <= 0 (NaN is caught above)
    float rh = s[0].hi, rl = s[0].lo;
    if (rb < k.rho_floor_bits) {  // positive doubles order like their bits
        rh = k.rho_floor_hi;
        rl = k.rho_floor_lo;
        flags |= FLAG_FLOOR;
        ++floors;
    }
    const float rho32 = __fadd_rn(rh, rl);
    const float r0 = rcp_approx(rho32);
    const float hr = __fmul_rn(0.5f, r0);
    const float e = __fmaf_rn(-rl, r0, __fmaf_rn(-rh, r0, 1.0f));  // 1 - rho r0, |e| ~ 2^-22
    // |m|^2 = Sh + Sl: the squares of the high parts with their exact errors
    // plus the cross terms 2 m_hi m_lo (m_lo^2 < 2^-46 m^2 is dropped)
    float Sh = 0.f, Sl = 0.f;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        const float mh = s[1 + d].hi, ml = s[1 + d].lo;
        const float P = __fmul_rn(mh, mh);
        const float Q = __fmaf_rn(__fmul_rn(2.f, mh), ml, __fmaf_rn(mh, mh, -P));
        if (d == 0) {
            Sh = P;
            Sl = Q;
        } else {  // TwoSum of the high parts
            const float t = __fadd_rn(Sh, P);
            const float bb = __fsub_rn(t, Sh);
            const float err = __fadd_rn(__fsub_rn(Sh, __fsub_rn(t, bb)), __fsub_rn(P, bb));
            Sh = t;
            Sl = __fadd_rn(Sl, __fadd_rn(err, Q));
        }
    }
    // ke = |m|^2 r0 (1 + e) / 2 = kh + kl
    const float kh = __fmul_rn(Sh, hr);
    const float kl = __fmaf_rn(kh, e, __fmaf_rn(Sl, hr, __fmaf_rn(Sh, hr, -kh)));
    const float eint = __fadd_rn(__fsub_rn(s[ND + 1].hi, kh), __fsub_rn(s[ND + 1].lo, kl));
    if (!(eint >= 0.0f)) flags |= FLAG_NONPHYSICAL;
    float p = __fmul_rn(k.gm1, eint);
    if (p < k.p_floor) {
        p = k.p_floor;
        flags |= FLAG_FLOOR;
        ++floors;
    }
    w[0] = rho32;
#pragma unroll
    for (int d = 0; d < ND; ++d) w[1 + d] = __fmul_rn(__fadd_rn(s[1 + d].hi, s[1 + d].lo), r0);
    w[ND + 1] = p;
}

// CFL candidate min_d dx_d / (|v_d| + c_s), c_s = sqrt(gamma p / rho), of one
// cell from its recovered FP32 primitives (Sec. 3.1: the step length comes
// out of the variable conversion).  An estimate: division and square root
// use the special-function unit.  Written with explicit round-to-nearest
// intrinsics (no contraction), so every kernel that calls it produces the
// same bits for the same primitives.
template <int ND>
__device__ __forceinline__ float cfl_from_prim(const float (&w)[ND + 2], const MixConsts &k) {
    const float c = rroot(rdiv(__fmul_rn(k.gamma, w[ND + 1]), w[0]));
    float m = rdiv(k.dx[0], __fadd_rn(fabsf(w[1]), c));
#pragma unroll
    for (int d = 1; d < ND; ++d) {
        const float t = rdiv(k.dx[d], __fadd_rn(fabsf(w[1 + d]), c));
        m = t < m ? t : m;
    }
    return m;
}

// CFL candidate straight from a conserved state (FP64 or FP32 storage), for
// the van Leer corrector, which stores no primitives of the new state: FP32
// estimate of rho, |v_d| and p; with an FP64 state the internal energy falls
// back to FP64 where E - ke cancels by more than a factor of four.
template <int ND, class S>
__device__ __forceinline__ float cfl_from_state(const S (&u)[ND + 2], const MixConsts &k) {
    float rho = abs_d2f_rz(u[0]);
    if (!(rho >= k.rho_floor)) rho = k.rho_floor;
    const float r = rcp_approx(rho);
    float v[ND];
    float vsq = 0.f;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        v[d] = __fmul_rn(abs_d2f_rz(u[1 + d]), r);
        vsq = __fmaf_rn(v[d], v[d], vsq);
    }
    const float E = abs_d2f_rz(u[ND + 1]);
    float eint = __fsub_rn(E, __fmul_rn(__fmul_rn(0.5f, rho), vsq));
    if constexpr (sizeof(S) == 8) {
        if (eint < __fmul_rn(0.25f, E)) {
            double msq = __dmul_rn(u[1], u[1]);
#pragma unroll
            for (int d = 1; d < ND; ++d) msq = __fma_rn(u[1 + d], u[1 + d], msq);
            eint = d2f(__dsub_rn(u[ND + 1], __ddiv_rn(__dmul_rn(0.5, msq), u[0])));
        }
    }
    float p = __fmul_rn(k.gm1, eint);
    if (!(p >= k.p_floor)) p = k.p_floor;
    const float c = rroot(__fmul_rn(__fmul_rn(k.gamma, p), r));
    float m = rdiv(k.dx[0], __fadd_rn(v[0], c));
#pragma unroll
    for (int d = 1; d < ND; ++d) {
        const float t = rdiv(k.dx[d], __fadd_rn(v[d], c));
        m = t < m ? t : m;
    }
    return m;
}

}  // namespace mx
}  // namespace khy
