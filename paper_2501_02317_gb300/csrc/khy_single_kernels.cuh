// khy_single_kernels.cuh -- device functions of the all-FP32 path: the
// paper's compile-time choice of single precision for both float_t and
// float2_t (Sec. 3.2.2, "Single" in its speed tables).  The conserved state
// is stored in FP32 and every operation is FP32; conservation then holds to
// FP32 round-off.  Explicit round-to-nearest intrinsics keep every kernel
// that calls these functions bit-for-bit consistent.
#pragma once

#include "khy_mixed_kernels.cuh"

namespace khy {
namespace sg {

// Conserved (FP32) -> primitive (FP32), floors on the primitive only.
template <int ND>
__device__ __forceinline__ void recover(const float (&u)[ND + 2], const mx::MixConsts &k, float (&w)[ND + 2],
                                        unsigned &flags, unsigned &floors) {
    float rho = u[0];
    if (!(rho > 0.f)) flags |= FLAG_NONPHYSICAL;
    if (rho < k.rho_floor) {
        rho = k.rho_floor;
        flags |= FLAG_FLOOR;
        ++floors;
    }
    const float r = rcp_approx(rho);
    float msq = __fmul_rn(u[1], u[1]);
#pragma unroll
    for (int d = 1; d < ND; ++d) msq = __fmaf_rn(u[1 + d], u[1 + d], msq);
    const float eint = __fmaf_rn(-0.5f, __fmul_rn(msq, r), u[ND + 1]);
    if (!(eint >= 0.f)) flags |= FLAG_NONPHYSICAL;
    float p = __fmul_rn(k.gm1, eint);
    if (p < k.p_floor) {
        p = k.p_floor;
        flags |= FLAG_FLOOR;
        ++floors;
    }
    w[0] = rho;
#pragma unroll
    for (int d = 0; d < ND; ++d) w[1 + d] = __fmul_rn(u[1 + d], r);
    w[ND + 1] = p;
}

}  // namespace sg
}  // namespace khy
