// khy_stage.cuh -- the fused stage kernel of the Godunov hydro step and the
// CFL-minimum kernel (sm_103a).
//
// One Heun step (Sec. 3.3) is three launches on one stream:
//   clock kernel   : dt = C * min dx_d/(|v_d|+c_s) from the minimum the
//                    previous stage-2 launch (or dt_kernel) accumulated, clipped
//                    to t_end; t and the step counter advance (khy_runtime.cu).
//   stage_kernel 1 : U1 = Un + dt L(Un)
//   stage_kernel 2 : Un+1 = (Un + (U1 + dt L(U1))) / 2 written over Un, plus the
//                    CFL minimum of Un+1 for the next step (Sec. 3.1: the step
//                    length comes out of the variable conversion).
// The memory-optimized van Leer integrator (Sec. 3.3) replaces the two stage
// launches with
//   stage_kernel 3 : predictor, U^{n+1/2} = Un + (dt/2) L_1(Un) with
//                    first-order face states; only its primitives W^{n+1/2}
//                    are stored (in the flux precision R: FP32 in the mixed
//                    path), in place of U1
//   stage_kernel 4 : corrector, Un+1 = Un + dt L(W^{n+1/2}) with PLM face
//                    states of W^{n+1/2}, written over Un, plus the CFL minimum.
// Single-grid Heun steps keep the primitives of the current state in HBM
// (in the flux precision) so that no CTA recovers halo cells:
//   stage_kernel 5 : as stage 1, fluxes from the stored primitives of Un;
//                    writes the primitives of U1 and, in the U1 buffer, U1
//                    (all-FP64) or V = (Un + U1)/2 (mixed and all-FP32)
//   stage_kernel 6 : as stage 2, fluxes from the stored primitives of U1;
//                    writes Un+1 (from V alone where V was stored) and its
//                    primitives.
// Every stored primitive comes from the same recovery function as an on-the-
// fly one, so stages 5, 6 give the same bits as stages 1, 2.
//
// Work decomposition.  The grid is cut into tiles of TX x TY columns along
// the slowest ("march") axis -- z in 3D, y in 2D; a 1D grid is one row.  On
// large grids every tile column is cut at the same plane boundaries into
// runs (StageArgs::kb), one CTA per run, numbered chunk-major, so CTAs that
// run at the same time hold neighbouring tiles at the same planes and share
// their halo rows through L2; smaller grids use a persistent launch, one CTA
// per resident slot, CTA b owning the b-th equal share of the (tile, plane)
// sequence.  A CTA walks each of its tile segments plane by plane: a plane
// of primitives with a two-cell halo on every side -- copied from the stored
// primitives (cp.async, one plane ahead) or recovered from the state (Sec.
// 3.1) -- with the ghost-zone rules applied by index mapping (Sec. 3.1.1) is
// kept in a four-plane ring in shared memory (the row staging of Sec. 3.2.1
// extended to a 2.5D march).  FP32 fluxes: the march, x and y faces of a
// plane are consecutive task ranges, two faces per task (packed FP32x2);
// FP64 fluxes: in-plane faces as one task list, the march face by the
// column's thread.  Each face flux is computed once per CTA and enters its
// two cells with opposite signs; faces on a tile edge are recomputed by the
// neighbouring CTA from the same inputs by the same code, so both cells see
// the same value.
//
// Precision (Sec. 3.2.2) is the template parameter R (fluxes) with S (state):
//   R = double : all-FP64, every operation in the CPU reference's order
//                (compiled with -fmad=false: bitwise equal to the reference);
//   R = float  : mixed (S = double) -- FP32 reconstruction and HLLC, FP64
//                state, FP64 internal energy in the recovery and FP64
//                flux-difference accumulation (khy_mixed_kernels.cuh); or
//                all-FP32 (S = float).
#pragma once

#include <type_traits>

#include "khy_kernels.cuh"
#include "khy_mixed_kernels.cuh"
#include "khy_packed.cuh"
#include "khy_single_kernels.cuh"

namespace khy {

constexpr int kMaxChunks = 96;  // runs of planes per tile column (stage_kernel work split)

struct StageArgs {
    Geom g;
    const double *Uin;    // state the stage adds to: Un (1, 3, 5) or U1 (2, 6); unused in 4
    const double *Ubase;  // Un (stages 2, 4, 6)
    double *Uout;         // U1 (1, 5) or Un+1 (2, 4, 6; may alias Ubase); unused in 3
    const void *Win;      // stored primitives the fluxes come from (4: W^{n+1/2}, 5: W^n, 6: W^1)
    void *Wout;           // primitives written (3: W^{n+1/2}, 5: W^1, 6: W^{n+1})
    Clock *clk;
    int cubic;            // mixed path: all active dx equal (one dt/dx factor)
    int nchunk;           // work split (stage_kernel): 0 = one contiguous share of the
                          // (tile, plane) sequence per CTA; > 0 = each tile column cut
                          // into nchunk runs of planes [kb[c], kb[c + 1]), one run per
                          // CTA, chunk-major
    int kb[kMaxChunks + 1];
};

template <int ND, int TX, int TY>
struct Tile {
    static constexpr int NV = ND + 2;
    static constexpr int PX = TX + 4;
    static constexpr int PY = (ND == 3) ? TY + 4 : 1;
    static constexpr int PC = PX * PY;
    static constexpr int NSLOT = (ND == 1) ? 1 : 4;
    static constexpr int NT = TX * TY;
    static constexpr int NXF = (TX + 1) * TY;
    static constexpr int NYF = (ND == 3) ? TX * (TY + 1) : 0;
    // mixed path: march-axis fluxes of the last two planes also live in shared memory
    static constexpr int NFM = (ND >= 2) ? 2 * NV * NT : 0;
    // buffer offsets in elements, each a multiple of 4 (16 bytes for FP32): the
    // FP32 face loop reads and writes float2 pairs at even offsets within them
    static constexpr int up4(int v) { return (v + 3) / 4 * 4; }
    static constexpr int OFF_FX = up4(NSLOT * NV * PC);
    static constexpr int OFF_FY = OFF_FX + up4(NV * NXF);
    static constexpr int OFF_FM = OFF_FY + up4(NV * NYF);
    template <class R>
    static constexpr size_t smem_bytes() {
        return sizeof(R) * ((size_t)OFF_FM + (std::is_same<R, float>::value ? (size_t)NFM : 0));
    }
    static_assert(PX % 2 == 0 && PC % 2 == 0 && NYF % 2 == 0 && NT % 2 == 0,
                  "float2 accesses need even row, plane, flux-row and column strides");
};

// Threads per CTA.  The FP32 face loop of a 2D tile has TX + 1 face pairs
// per row (TX/2 march-face pairs, TX/2 + 1 x-face pairs); with the TX cell
// threads rounded up to whole warps for each range they all run in one
// round.  Every other tile uses one thread per cell.
template <class R, int ND, int TX, int TY>
__host__ __device__ constexpr int cta_threads() {
    return (std::is_same<R, float>::value && ND == 2)
               ? ((TX / 2 + 31) / 32 * 32 + ((TX + 2) / 2 + 31) / 32 * 32 > TX * TY
                      ? (TX / 2 + 31) / 32 * 32 + ((TX + 2) / 2 + 31) / 32 * 32
                      : TX * TY)
               : TX * TY;
}

// Asynchronous 4-byte global -> shared copy (no registers, no wait) and the
// wait for all of this thread's outstanding copies.
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One segment: tile (x0, y0) of one grid, planes [k0, k1) of its march axis.
// Shared by the single-grid and the multi-grid kernels.  Accumulates the
// status bits, the floor count and (stage 2) the CFL minimum into the
// caller's registers.
// S is the storage type of the conserved state: double (all-FP64 and mixed
// paths) or float (all-FP32 path, S = R = float).
template <class R, int ND, int STAGE, int TX, int TY, class S = double>
__device__ __forceinline__ void run_segment(const Geom &g, const S *__restrict__ Uin, const S *Ubase,
                                            S *Uout, const R *__restrict__ Win, R *Wout,
                                            const double (&dtdx)[3], int cubic, int x0, int y0,
                                            int k0, int k1, R *sW, R *sFx, R *sFy, unsigned &flags,
                                            unsigned &floors, double &wmin) {
    constexpr bool MIX = std::is_same<R, float>::value;
    constexpr bool SINGLE = std::is_same<S, float>::value;
    static_assert(!SINGLE || MIX, "an FP32 state needs FP32 fluxes");
    static_assert(STAGE >= 1 && STAGE <= 6, "stages 1, 2, 5, 6 (Heun) and 3, 4 (van Leer)");
    constexpr bool HEUN2 = STAGE == 2 || STAGE == 6;             // Heun average with Ubase
    constexpr bool PLM = STAGE != 3;                             // the predictor uses first-order face states
    constexpr bool CFL = STAGE == 2 || STAGE == 4 || STAGE == 6; // last stage of a step: CFL minimum of Un+1
    constexpr bool FROM_W = STAGE == 4 || STAGE >= 5;            // fluxes from stored primitives (type R)
    constexpr bool WRITE_U = STAGE != 3;                         // stores the new state
    constexpr bool WRITE_W = STAGE == 3 || STAGE >= 5;           // stores the new state's primitives
    using T = Tile<ND, TX, TY>;
    constexpr int NV = T::NV, PX = T::PX, PC = T::PC, NT = T::NT;
    constexpr int NTH = cta_threads<R, ND, TX, TY>();  // threads (>= NT; cells use the first NT)
    constexpr int DM = ND - 1;  // march axis (ND >= 2)
    const Consts<R> kc = make_consts<R>(g);
    const Consts<float> kc_f = make_consts<float>(g);
    const mx::MixConsts mk = mx::make_mix(g);
    const long long N = g.ncell;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    float wmin_f = __int_as_float(0x7F800000);  // FP32 CFL minimum of this segment (mixed / FP32)
    // active extent of this tile (ragged tiles and grids narrower than a tile)
    const int wact = min(TX, g.n[0] - x0);
    const int hact = (ND == 3) ? min(TY, g.n[1] - y0) : 1;

    // the step's dt/dx, halved for the van Leer predictor (a power-of-two
    // scaling: the same bits as (dt/2)/dx)
    double dtq[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) dtq[d] = STAGE == 3 ? 0.5 * dtdx[d] : dtdx[d];
    // dt/(2 dx) for the mixed Heun average; dt/dx_d rounded to FP32 once for
    // the all-FP32 update
    const double hcd = 0.5 * dtq[0];
    const float c32x = mx::d2f(dtq[0]), c32y = mx::d2f(dtq[1]), c32m = mx::d2f(dtq[DM < 0 ? 0 : DM]);

    // tiles whose halo box lies inside the grid skip the ghost-zone index map
    const bool x_inside = x0 >= 2 && x0 + wact + 2 <= g.n[0];
    const bool y_inside = ND != 3 || (y0 >= 2 && y0 + hact + 2 <= g.n[1]);

    // plane L of the march axis (ignored in 1D) -> ring slot
    auto load_plane = [&](int L, int slot) {
        R *dst = sW + (size_t)slot * NV * PC;
        int actm = 0;  // the march-axis index map is the same for the whole plane
        const int cm = (ND >= 2) ? bc_map(L, g.n[DM], g.bc[DM][0], g.bc[DM][1], &actm) : 0;
        for (int e = tid; e < PC; e += NTH) {
            const int hx = e % PX, hy = e / PX;
            if (hx >= wact + 4 || (ND == 3 && hy >= hact + 4)) continue;  // outside the active halo box
            int act[3] = {0, 0, 0};
            int c[3] = {0, 0, 0};
            if (x_inside) c[0] = x0 - 2 + hx;
            else c[0] = bc_map(x0 - 2 + hx, g.n[0], g.bc[0][0], g.bc[0][1], &act[0]);
            if (ND == 3) {
                if (y_inside) c[1] = y0 - 2 + hy;
                else c[1] = bc_map(y0 - 2 + hy, g.n[1], g.bc[1][0], g.bc[1][1], &act[1]);
                c[2] = cm;
                act[2] = actm;
            } else if (ND == 2) {
                c[1] = cm;
                act[1] = actm;
            }
            const long long idx = ((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
            R w[NV];
            unsigned fl = 0;
            if constexpr (FROM_W) {  // stored primitives: no recovery
#pragma unroll
                for (int q = 0; q < NV; ++q) w[q] = __ldg(Win + (long long)q * N + idx);
            } else if constexpr (SINGLE) {
                float u[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) u[q] = __ldg(Uin + (long long)q * N + idx);
                sg::recover<ND>(u, mk, w, flags, fl);
            } else {
                double u[NV];
#pragma unroll
                for (int q = 0; q < NV; ++q) u[q] = __ldg(Uin + (long long)q * N + idx);
                if constexpr (MIX) {
                    mx::recover<ND>(u, mk, w, flags, fl);
                } else {
                    recover<ND>(u, g, w, flags, fl);
                }
            }
            const bool interior = hx >= 2 && hx < TX + 2 && x0 - 2 + hx < g.n[0] &&
                                  (ND != 3 || (hy >= 2 && hy < TY + 2 && y0 - 2 + hy < g.n[1])) &&
                                  (ND == 1 || (L >= k0 && L < k1));
            if (interior) floors += fl;
#pragma unroll
            for (int d = 0; d < ND; ++d) {  // ghost-zone velocity rules (Sec. 3.1.1)
                R v = w[1 + d];
                if (act[d] == 1) v = -v;
                else if (act[d] == 2) v = v > R(0) ? R(0) : v;
                else if (act[d] == 3) v = v < R(0) ? R(0) : v;
                w[1 + d] = v;
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) dst[(size_t)q * PC + e] = w[q];
        }
    };

    // mixed / FP32 stages that read stored primitives: plane L is copied with
    // cp.async (issued one plane ahead, while the previous plane's cells are
    // updated); the ghost-zone velocity rules are applied by the copying
    // thread after its copies have landed (fix_plane).
    // tiles whose halo box lies inside the grid copy whole rows in 8-byte
    // pairs (the row start x0 - 2 is even, and so is every row and field
    // offset when nx is even) -- provided the grid's primitive array itself
    // starts on 8 bytes, which a grid packed after one with an odd cell
    // count in a many-grid pool does not; the others copy cell by cell
    // through the ghost-zone index map
    const bool rows8 = x_inside && y_inside && (g.n[0] % 2 == 0) &&
                       (reinterpret_cast<unsigned long long>(Win) % 8 == 0);
    auto load_plane_async = [&](int L, int slot) {
        if constexpr (MIX && FROM_W) {
            R *dst = sW + (size_t)slot * NV * PC;
            int actm = 0;
            const int cm = (ND >= 2) ? bc_map(L, g.n[DM], g.bc[DM][0], g.bc[DM][1], &actm) : 0;
            if (rows8) {
                constexpr int CH = PX / 2;                        // 8-byte pairs per halo row
                constexpr int NTASK = ((ND == 3) ? T::PY : 1) * CH;
                // first halo cell (x0 - 2, y0 - 2) of plane cm; ND == 2: row cm
                const long long row0 = ((ND == 3) ? ((long long)cm * g.n[1] + y0 - 2) * g.n[0]
                                                  : (ND == 2 ? (long long)cm * g.n[0] : 0LL)) + x0 - 2;
                for (int t = tid; t < NTASK; t += NTH) {
                    const int hy = t / CH, ch = t % CH;
                    const long long gi = row0 + (long long)hy * g.n[0] + 2 * ch;
                    R *d = dst + hy * PX + 2 * ch;
#pragma unroll
                    for (int q = 0; q < NV; ++q) cp_async8(d + (size_t)q * PC, Win + (long long)q * N + gi);
                }
                return;
            }
            for (int e = tid; e < PC; e += NTH) {
                const int hx = e % PX, hy = e / PX;
                if (hx >= wact + 4 || (ND == 3 && hy >= hact + 4)) continue;
                int act = 0;
                int c[3] = {0, 0, 0};
                if (x_inside) c[0] = x0 - 2 + hx;
                else c[0] = bc_map(x0 - 2 + hx, g.n[0], g.bc[0][0], g.bc[0][1], &act);
                if (ND == 3) {
                    if (y_inside) c[1] = y0 - 2 + hy;
                    else c[1] = bc_map(y0 - 2 + hy, g.n[1], g.bc[1][0], g.bc[1][1], &act);
                    c[2] = cm;
                } else if (ND == 2) {
                    c[1] = cm;
                }
                const long long idx = ((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
#pragma unroll
                for (int q = 0; q < NV; ++q) cp_async4(dst + (size_t)q * PC + e, Win + (long long)q * N + idx);
            }
        }
    };
    const bool x_rules = !x_inside && (g.bc[0][0] != BC_PERIODIC || g.bc[0][1] != BC_PERIODIC);
    const bool y_rules = ND == 3 && !y_inside && (g.bc[1][0] != BC_PERIODIC || g.bc[1][1] != BC_PERIODIC);
    auto fix_plane = [&](int L, int slot) {
        if constexpr (MIX && FROM_W) {
            int actm = 0;
            if (ND >= 2) bc_map(L, g.n[DM], g.bc[DM][0], g.bc[DM][1], &actm);
            if (!x_rules && !y_rules && actm == 0) return;  // no ghost cell with a velocity rule
            // (a CTA-uniform condition) every thread has waited for its own copies;
            // the row copies of interior tiles assign elements to threads other than
            // this loop does, so all of them must have landed before any is fixed
            __syncthreads();
            R *dst = sW + (size_t)slot * NV * PC;
            for (int e = tid; e < PC; e += NTH) {
                const int hx = e % PX, hy = e / PX;
                if (hx >= wact + 4 || (ND == 3 && hy >= hact + 4)) continue;
                int act[3] = {0, 0, 0};
                if (x_rules) bc_map(x0 - 2 + hx, g.n[0], g.bc[0][0], g.bc[0][1], &act[0]);
                if (y_rules) bc_map(y0 - 2 + hy, g.n[1], g.bc[1][0], g.bc[1][1], &act[1]);
                act[DM] = actm;
#pragma unroll
                for (int d = 0; d < ND; ++d) {  // ghost-zone velocity rules (Sec. 3.1.1)
                    if (act[d] == 0) continue;
                    R v = dst[(size_t)(1 + d) * PC + e];
                    if (act[d] == 1) v = -v;
                    else if (act[d] == 2) v = v > R(0) ? R(0) : v;
                    else v = v < R(0) ? R(0) : v;
                    dst[(size_t)(1 + d) * PC + e] = v;
                }
            }
        }
    };

    auto gather = [&](const R *base, int e0, int stride, R (&s)[4][NV]) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
            for (int q = 0; q < NV; ++q) s[o][q] = base[(size_t)q * PC + e0 + o * stride];
    };

    auto inplane_faces = [&](int slot) {
        const R *pl = sW + (size_t)slot * NV * PC;
        for (int f = tid; f < T::NXF + T::NYF; f += NT) {
            R s[4][NV], F[NV];
            if (f < T::NXF) {
                const int fx = f % (TX + 1), fy = f / (TX + 1);
                if (fx > wact || fy >= hact) continue;
                const int hy = (ND == 3) ? fy + 2 : 0;
                gather(pl, hy * PX + fx, 1, s);
                face_flux<ND, R, PLM>(s, 0, kc, F);
#pragma unroll
                for (int q = 0; q < NV; ++q) sFx[(size_t)q * T::NXF + f] = F[q];
            } else {
                const int f2 = f - T::NXF;
                const int fxx = f2 % TX, fyy = f2 / TX;
                if (fxx >= wact || fyy > hact) continue;
                gather(pl, fyy * PX + fxx + 2, PX, s);
                face_flux<ND, R, PLM>(s, 1, kc, F);
#pragma unroll
                for (int q = 0; q < NV; ++q) sFy[(size_t)q * T::NYF + f2] = F[q];
            }
        }
    };

    // mixed path: the faces of one plane as three direction-specific task
    // ranges -- march-axis faces, x faces, y faces -- back to back: each
    // branch's rotation is a compile-time constant, a warp that straddles two
    // ranges diverges only in its gather and its stores and runs the one
    // flux call site for both (no warp runs the flux for a few lanes of
    // padding).  A task computes two neighbouring faces of one
    // direction as the two lanes of the packed face_flux2, from one shared
    // stencil: x faces f, f+1 of one row share a five-cell stencil (three
    // float2 loads); y faces and march faces of the column pair (2c, 2c+1)
    // are read as float2 pairs (along y within the plane, along the march
    // axis from the four ring planes).  March fluxes go to sFm[cur & 1],
    // in-plane ones to sFx / sFy.  The last pair of an x row (faces TX, TX+1)
    // has one valid lane; its idle lane reads shared memory past the row
    // (other fields or the flux buffers) and stores nothing.
    R *sFm = sW + T::OFF_FM;  // [2][NV][NT], mixed path only
    constexpr int XPR = (TX + 2) / 2;                  // x-face pairs per row (faces 0..TX)
    constexpr int YPC = (ND == 3) ? TY + 1 : 0;        // y faces per column pair (faces 0..TY)
    constexpr int TY_ = (ND == 3) ? TY : 1;
    constexpr int NMP = (ND >= 2) ? NT / 2 : 0;        // march-face column pairs
    constexpr int M_END = NMP;
    constexpr int X_END = M_END + XPR * TY_;
    constexpr int Y_END = X_END + YPC * (TX / 2);
    static_assert(TX % 2 == 0, "face pairs need an even tile width");
    static_assert(NT % 4 == 0, "16-byte flux stores need a cell count divisible by 4");
    // FP32 flux layout (mixed and FP32 paths), per direction: the fields in
    // pairs (0,1), (2,3) as float2 arrays of nelem elements, an odd last
    // field as a float array -- a cell reads two fields per 8-byte load
    constexpr int NPR = NV / 2;
    auto pread = [&](const float *base, int nelem, int p, int i) -> float2 {
        if (p < NPR) return *reinterpret_cast<const float2 *>(base + (size_t)2 * nelem * p + 2 * i);
        const float v = base[(size_t)2 * NPR * nelem + i];
        return make_float2(v, v);
    };
    auto fread = [&](const float *base, int nelem, int q, int i) -> float {
        if (q < 2 * NPR) return base[(size_t)2 * nelem * (q / 2) + 2 * i + (q & 1)];
        return base[(size_t)2 * NPR * nelem + i];
    };
    auto faces_mix = [&](int cur, bool inplane) {
        const float *cp = reinterpret_cast<const float *>(sW);
        float *fm = reinterpret_cast<float *>(sFm) + (size_t)(cur & 1) * NV * NT;
        float *fxo = reinterpret_cast<float *>(sFx);
        float *fyo = reinterpret_cast<float *>(sFy);
        const float *plane = cp + (size_t)(cur & 3) * NV * PC;
        const int ntask = inplane ? Y_END : M_END;
        for (int k = tid; k < ntask; k += NTH) {
            // gather: direction-specific, rotations fixed at compile time;
            // then one flux call site (keeps the kernel's code small)
            float2 st[4][NV];
            int kind, a0, a1;  // 0 march (column col), 1 x (row ty, face p2), 2 y (column tx, face fy)
            bool vy = true;
            if (k < M_END) {  // march faces between planes cur and cur + 1 of columns 2c, 2c + 1
                if (k >= NMP) continue;
                const int col = 2 * k, ctx = col % TX, cty = col / TX;
                if (ctx >= wact || cty >= hact) continue;
                kind = 0;
                a0 = col;
                a1 = 0;
                const int e = ((ND == 3) ? (cty + 2) * PX : 0) + ctx + 2;
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const float *pl = cp + (size_t)((cur - 1 + o) & 3) * NV * PC + e;
#pragma unroll
                    for (int j = 0; j < NV; ++j)
                        st[o][j] = *reinterpret_cast<const float2 *>(pl + (size_t)pk::rot_slot<ND>(DM, j) * PC);
                }
            } else if (k < X_END) {  // x faces 2p, 2p + 1 of row ty: cells 2p .. 2p + 4
                const int x = k - M_END;
                if (x >= XPR * TY_) continue;
                const int ty_ = x / XPR, p2 = 2 * (x % XPR);
                if (p2 > wact || ty_ >= hact) continue;
                kind = 1;
                a0 = ty_;
                a1 = p2;
                vy = p2 + 1 <= wact;
                const float *pl = plane + ((ND == 3) ? (ty_ + 2) * PX : 0) + p2;
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    const float *c = pl + (size_t)j * PC;  // rotation onto x is the identity
                    const float2 va = *reinterpret_cast<const float2 *>(c);
                    const float2 vb = *reinterpret_cast<const float2 *>(c + 2);
                    const float2 vd = *reinterpret_cast<const float2 *>(c + 4);
                    st[0][j] = va;
                    st[1][j] = make_float2(va.y, vb.x);
                    st[2][j] = vb;
                    st[3][j] = make_float2(vb.y, vd.x);
                }
            } else {  // y face fy of columns 2c, 2c + 1: rows fy .. fy + 3
                const int y = k - X_END;
                if (y >= YPC * (TX / 2)) continue;
                const int tx_ = 2 * (y % (TX / 2)), fy = y / (TX / 2);
                if (tx_ >= wact || fy > hact) continue;
                kind = 2;
                a0 = tx_;
                a1 = fy;
                const float *pl = plane + fy * PX + tx_ + 2;
#pragma unroll
                for (int o = 0; o < 4; ++o)
#pragma unroll
                    for (int j = 0; j < NV; ++j)
                        st[o][j] = *reinterpret_cast<const float2 *>(pl + (size_t)pk::rot_slot<ND>(1, j) * PC + o * PX);
            }
            float2 Fr[NV], Fq[NV];  // rotated order / field order
            pk::face_flux2<ND, PLM>(st, kc_f, Fr);
            if (kind == 0) {  // columns a0, a0 + 1: one 16-byte store per field pair
#pragma unroll
                for (int j = 0; j < NV; ++j) Fq[pk::rot_slot<ND>(DM, j)] = Fr[j];
#pragma unroll
                for (int p = 0; p < NPR; ++p)
                    *reinterpret_cast<float4 *>(fm + (size_t)2 * NT * p + 2 * a0) =
                        make_float4(Fq[2 * p].x, Fq[2 * p + 1].x, Fq[2 * p].y, Fq[2 * p + 1].y);
                if (NV % 2) *reinterpret_cast<float2 *>(fm + (size_t)2 * NPR * NT + a0) = Fq[NV - 1];
            } else if (kind == 1) {  // faces a1, a1 + 1 of row a0
#pragma unroll
                for (int j = 0; j < NV; ++j) Fq[j] = Fr[j];  // rotation onto x is the identity
                const int i = a0 * (TX + 1) + a1;
#pragma unroll
                for (int p = 0; p < NPR; ++p) {
                    float *d = fxo + (size_t)2 * T::NXF * p + 2 * i;
                    *reinterpret_cast<float2 *>(d) = make_float2(Fq[2 * p].x, Fq[2 * p + 1].x);
                    if (vy) *reinterpret_cast<float2 *>(d + 2) = make_float2(Fq[2 * p].y, Fq[2 * p + 1].y);
                }
                if (NV % 2) {
                    float *d = fxo + (size_t)2 * NPR * T::NXF + i;
                    d[0] = Fq[NV - 1].x;
                    if (vy) d[1] = Fq[NV - 1].y;
                }
            } else {  // face a1 of columns a0, a0 + 1
#pragma unroll
                for (int j = 0; j < NV; ++j) Fq[pk::rot_slot<ND>(1, j)] = Fr[j];
                const int i = a1 * TX + a0;
#pragma unroll
                for (int p = 0; p < NPR; ++p)
                    *reinterpret_cast<float4 *>(fyo + (size_t)2 * T::NYF * p + 2 * i) =
                        make_float4(Fq[2 * p].x, Fq[2 * p + 1].x, Fq[2 * p].y, Fq[2 * p + 1].y);
                if (NV % 2) *reinterpret_cast<float2 *>(fyo + (size_t)2 * NPR * T::NYF + i) = Fq[NV - 1];
            }
        }
    };

    // conservative update of cell (tx, ty) of plane cur (Sec. 3.3): stages
    // 1, 3, 4, 5 add dt L (or dt/2 L) to a state, stages 2, 6 take the Heun
    // average; then the new state's primitives (stages 3, 5, 6) and its CFL
    // candidate (last stage of a step).
    // the cell's state values, loaded ahead of the barrier that precedes the
    // update: uc = the state this stage adds to; for the Heun average, ub = Un
    // (all-FP64: kept apart for the reference operation order), or in the
    // mixed and FP32 stage 2 uc = Un + U1 already summed (fewer live
    // registers), or in stage 6 uc = V.
    // Stage 5 of the mixed and all-FP32 paths stores V = (Un + U1) / 2
    // (exact halving) in place of U1 -- the primitives of U1 are stored as
    // well -- so stage 6 adds to V and reads no Un: V + acc/2 equals the
    // lean stage 2's half(Un + U1) + acc/2 bit for bit.
    constexpr bool STORE_V = MIX && STAGE == 5;
    constexpr bool FROM_V = MIX && STAGE == 6;
    constexpr bool SUM_A = MIX && HEUN2 && !FROM_V;
    auto prefetch_cell = [&](int cur, S (&uc)[NV], S (&ub)[NV]) {
        const int gx = x0 + tx;
        const int gy = (ND == 3) ? y0 + ty : (ND == 2 ? cur : 0);
        const int gz = (ND == 3) ? cur : 0;
        if (gx >= g.n[0] || (ND == 3 && gy >= g.n[1])) return;
        const long long idx = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
        const S *Ucell = (STAGE == 4) ? Ubase : Uin;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const S u = Ucell[(long long)q * N + idx];
            if constexpr (SUM_A) {
                const S b = Ubase[(long long)q * N + idx];
                if constexpr (SINGLE) uc[q] = __fadd_rn(b, u);
                else uc[q] = __dadd_rn(b, u);
            } else {
                uc[q] = u;
                if constexpr (HEUN2 && !FROM_V) ub[q] = Ubase[(long long)q * N + idx];
            }
        }
    };

    auto update_cell = [&](int cur, const R (&Fmlo)[NV], const R (&Fmhi)[NV], const S (&uc)[NV], const S (&ub)[NV]) {
        const int gx = x0 + tx;
        const int gy = (ND == 3) ? y0 + ty : (ND == 2 ? cur : 0);
        const int gz = (ND == 3) ? cur : 0;
        if (gx >= g.n[0] || (ND == 3 && gy >= g.n[1])) return;
        const long long idx = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
        // FP32 flux buffers (pair layout) around this cell
        const float *fxs = reinterpret_cast<const float *>(sFx);
        const float *fys = reinterpret_cast<const float *>(sFy);
        const float *fml = reinterpret_cast<const float *>(sW + T::OFF_FM) + (size_t)((cur - 1) & 1) * NV * NT;
        const float *fmh = reinterpret_cast<const float *>(sW + T::OFF_FM) + (size_t)(cur & 1) * NV * NT;
        const int ix = ty * (TX + 1) + tx, iy = ty * TX + tx;
        (void)fml; (void)fmh; (void)iy;
        // mixed, equal dx: the six face fluxes of each field summed exactly as
        // a float-float pair, two fields per packed operation (lanes), then
        // the FP64 update of those two fields
        S un[NV];
        bool packed_done = false;
        if constexpr (MIX && !SINGLE) {
            if (cubic) {
#pragma unroll
                for (int p = 0; p < (NV + 1) / 2; ++p) {
                    const float2 xl = pread(fxs, T::NXF, p, ix), xh = pread(fxs, T::NXF, p, ix + 1);
                    pk::FF2 Fs = pk::two_diff2(xl, xh);
                    if constexpr (HEUN2 && ND >= 2) {
                        // the Heun average adds hi and lo as two doubles, so the
                        // pair needs no renormalisation
                        const float2 ml = pread(fml, NT, p, tid), mh = pread(fmh, NT, p, tid);
                        if constexpr (ND == 3) {
                            const float2 yl = pread(fys, T::NYF, p, iy), yh = pread(fys, T::NYF, p, iy + TX);
                            Fs = pk::ff_sum3_unnorm(Fs, pk::two_diff2(yl, yh), pk::two_diff2(ml, mh));
                        } else {
                            Fs = pk::ff_sum2_unnorm(Fs, pk::two_diff2(ml, mh));
                        }
                    } else {
                        if (ND == 3) {
                            const float2 yl = pread(fys, T::NYF, p, iy), yh = pread(fys, T::NYF, p, iy + TX);
                            Fs = pk::ff_add2(Fs, pk::two_diff2(yl, yh));
                        }
                        if (ND >= 2) {
                            const float2 ml = pread(fml, NT, p, tid), mh = pread(fmh, NT, p, tid);
                            Fs = pk::ff_add2(Fs, pk::two_diff2(ml, mh));
                        }
                    }
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        const int q = 2 * p + l;
                        if (q >= NV) break;
                        const float fhi = l ? Fs.hi.y : Fs.hi.x, flo = l ? Fs.lo.y : Fs.lo.x;
                        const double u = uc[q];
                        double r;
                        if constexpr (HEUN2) {
                            // Heun average: V + (dt/2)(S_hi + S_lo) as two FP64
                            // FMAs with the exact doubles of the pair, which
                            // need not be renormalised (this stage has FP64
                            // issue to spare; in stage 1, whose FP64 pipe also
                            // forms V, the same form is 2 % slower)
                            const double v = FROM_V ? u : mx::half_exact(u);  // V, or (Un + U1)/2
                            r = __fma_rn(hcd, mx::f2d_fast(fhi), __fma_rn(hcd, mx::f2d_fast(flo), v));
                        } else {
                            // one FP64 operation: the flux sum as one double
                            // built with integer operations
                            r = __fma_rn(dtq[0], mx::ff_to_double(fhi, flo), u);
                        }
                        un[q] = r;
                        if constexpr (STORE_V) Uout[(long long)q * N + idx] = mx::half_exact(__dadd_rn(u, r));
                        else if (WRITE_U) Uout[(long long)q * N + idx] = r;
                    }
                }
                packed_done = true;
            }
        }
        if constexpr (SINGLE) {  // all-FP32: dt L(U) of two fields per packed operation
#pragma unroll
            for (int p = 0; p < (NV + 1) / 2; ++p) {
                const float2 xl = pread(fxs, T::NXF, p, ix), xh = pread(fxs, T::NXF, p, ix + 1);
                float2 acc = pk::mul2(pk::splat(c32x), pk::sub2(xl, xh));
                if (ND == 3) {
                    const float2 yl = pread(fys, T::NYF, p, iy), yh = pread(fys, T::NYF, p, iy + TX);
                    acc = pk::fma2(pk::splat(c32y), pk::sub2(yl, yh), acc);
                }
                if (ND >= 2) {
                    const float2 ml = pread(fml, NT, p, tid), mh = pread(fmh, NT, p, tid);
                    acc = pk::fma2(pk::splat(c32m), pk::sub2(ml, mh), acc);
                }
#pragma unroll
                for (int l = 0; l < 2; ++l) {
                    const int q = 2 * p + l;
                    if (q >= NV) break;
                    const float a = l ? acc.y : acc.x;
                    const float u = uc[q];
                    float r;
                    if (!HEUN2) r = __fadd_rn(u, a);
                    else if (FROM_V) r = __fadd_rn(u, __fmul_rn(0.5f, a));  // u = V
                    else r = __fmaf_rn(0.5f, u, __fmul_rn(0.5f, a));        // u = Un + U1
                    un[q] = r;
                    if constexpr (STORE_V) Uout[(long long)q * N + idx] = __fmul_rn(0.5f, __fadd_rn(u, r));
                    else if (WRITE_U) Uout[(long long)q * N + idx] = r;
                }
            }
            packed_done = true;
        }
#pragma unroll
        for (int q = 0; q < NV && !packed_done; ++q) {
            const R *fx = sFx + (size_t)q * T::NXF + ty * (TX + 1) + tx;
            const R *fy = sFy + (size_t)q * T::NYF + ty * TX + tx;
            S r;
            if constexpr (SINGLE) {  // (the packed path above handles every FP32 update)
                float acc = __fmul_rn(c32x, __fsub_rn(fread(fxs, T::NXF, q, ix), fread(fxs, T::NXF, q, ix + 1)));
                if (ND == 3) acc = __fmaf_rn(c32y, __fsub_rn(fread(fys, T::NYF, q, iy), fread(fys, T::NYF, q, iy + TX)), acc);
                if (ND >= 2) acc = __fmaf_rn(c32m, __fsub_rn(fread(fml, NT, q, tid), fread(fmh, NT, q, tid)), acc);
                if (!HEUN2) r = __fadd_rn(uc[q], acc);
                else if (FROM_V) r = __fadd_rn(uc[q], __fmul_rn(0.5f, acc));  // uc = V
                else r = __fmaf_rn(0.5f, uc[q], __fmul_rn(0.5f, acc));   // uc = Un + U1
            } else if constexpr (!MIX) {
                const double u = uc[q];
                // dU = -sum_d (dt/dx_d)(F_hi - F_lo), directions in x, y, z order
                double acc = 0.0 - dtq[0] * (fx[1] - fx[0]);
                if (ND == 3) acc = acc - dtq[1] * (fy[TX] - fy[0]);
                if (ND >= 2) acc = acc - dtq[DM] * (Fmhi[q] - Fmlo[q]);
                if (!HEUN2) r = u + acc;
                else r = 0.5 * (ub[q] + (u + acc));
            } else {
                const double u = uc[q];
                {  // unequal dx (equal dx is the packed path above)
                    // F_lo - F_hi per direction, exact as float-float pairs
                    const mx::FF Dx = mx::two_sum(fread(fxs, T::NXF, q, ix), -fread(fxs, T::NXF, q, ix + 1));
                    mx::FF Dy = {0.f, 0.f}, Dm = {0.f, 0.f};
                    if (ND == 3) Dy = mx::two_sum(fread(fys, T::NYF, q, iy), -fread(fys, T::NYF, q, iy + TX));
                    if (ND >= 2) Dm = mx::two_sum(fread(fml, NT, q, tid), -fread(fmh, NT, q, tid));
                    double acc = __fma_rn(dtq[0], mx::f2d_fast(Dx.hi), __dmul_rn(dtq[0], mx::f2d_fast(Dx.lo)));
                    if (ND == 3) acc = __fma_rn(dtq[1], mx::f2d_fast(Dy.hi), __fma_rn(dtq[1], mx::f2d_fast(Dy.lo), acc));
                    if (ND >= 2) acc = __fma_rn(dtq[DM], mx::f2d_fast(Dm.hi), __fma_rn(dtq[DM], mx::f2d_fast(Dm.lo), acc));
                    if (!HEUN2) r = __dadd_rn(u, acc);
                    else if (FROM_V) r = __fma_rn(0.5, acc, u);                // u = V
                    else r = __fma_rn(0.5, acc, mx::half_exact(u));            // u = Un + U1
                }
            }
            un[q] = r;
            if constexpr (STORE_V) {
                if constexpr (SINGLE) Uout[(long long)q * N + idx] = __fmul_rn(0.5f, __fadd_rn(uc[q], r));
                else Uout[(long long)q * N + idx] = mx::half_exact(__dadd_rn(uc[q], r));
            } else if (WRITE_U) {
                Uout[(long long)q * N + idx] = r;
            }
        }
        // CFL estimate of the van Leer corrector (mixed / FP32): straight from
        // the state, which it does not recover
        constexpr bool CFL_STATE = MIX && STAGE == 4;
        R w[NV];
        if (WRITE_W || (CFL && !CFL_STATE)) {  // primitives of the new state
            unsigned fl = 0;   // floors count once per stored recovery
            if constexpr (SINGLE) sg::recover<ND>(un, mk, w, flags, fl);
            else if constexpr (MIX) mx::recover<ND>(un, mk, w, flags, fl);
            else recover<ND>(un, g, w, flags, fl);
            if (WRITE_W) {
                floors += fl;
#pragma unroll
                for (int q = 0; q < NV; ++q) Wout[(long long)q * N + idx] = w[q];
            }
        }
        if (CFL) {  // CFL candidate of the new state for the next step
            if constexpr (MIX) {  // FP32 minimum (no FP64 compare per cell)
                float c;
                if constexpr (CFL_STATE) c = mx::cfl_from_state<ND>(un, mk);
                else c = mx::cfl_from_prim<ND>(w, mk);
                wmin_f = c < wmin_f ? c : wmin_f;
            } else {
                const double c = cfl_candidate<ND>(w, g);
                wmin = c < wmin ? c : wmin;
            }
        }
    };

    if (ND == 1) {
        load_plane(0, 0);
        __syncthreads();
        if constexpr (MIX) faces_mix(0, true);
        else inplane_faces(0);
        __syncthreads();
        R dummy[NV];
        S uc[NV], ub[NV];
        prefetch_cell(0, uc, ub);
        update_cell(0, dummy, dummy, uc, ub);
        __syncthreads();
    } else if constexpr (MIX && FROM_W) {
        // planes arrive by cp.async one plane ahead; the cell's state values
        // are loaded before the barrier that precedes its update
        const bool own = tx < wact && ty < hact;
        S uc[NV], ub[NV];
        for (int L = k0 - 2; L <= k0 + 1; ++L) load_plane_async(L, L & 3);
        for (int L = k0 + 1; L <= k1 + 1; ++L) {
            cp_async_wait_all();
            if (L == k0 + 1) {
                for (int Lp = k0 - 2; Lp <= k0 + 1; ++Lp) fix_plane(Lp, Lp & 3);
            } else {
                fix_plane(L, L & 3);
            }
            __syncthreads();
            const int cur = L - 2;
            faces_mix(cur, cur >= k0);
            if (cur >= k0 && own) prefetch_cell(cur, uc, ub);
            __syncthreads();
            if (L + 1 <= k1 + 1) load_plane_async(L + 1, (L + 1) & 3);  // slot of plane cur - 1, now free
            if (cur >= k0 && own) {
                R unused[NV];  // the FP32 update reads the march fluxes from sFm itself
                update_cell(cur, unused, unused, uc, ub);
            }
        }
    } else if constexpr (MIX) {
        for (int L = k0 - 2; L <= k1 + 1; ++L) {
            load_plane(L, L & 3);
            __syncthreads();
            if (L >= k0 + 1) {
                const int cur = L - 2;
                faces_mix(cur, cur >= k0);
                __syncthreads();
                if (cur >= k0 && tx < wact && ty < hact) {
                    R unused[NV];  // the FP32 update reads the march fluxes from sFm itself
                    S uc[NV], ub[NV];
                    prefetch_cell(cur, uc, ub);
                    update_cell(cur, unused, unused, uc, ub);
                }
            } else {
                __syncthreads();
            }
        }
    } else {
        R Fmlo[NV], Fmhi[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { Fmlo[q] = R(0); Fmhi[q] = R(0); }
        for (int L = k0 - 2; L <= k1 + 1; ++L) {
            load_plane(L, L & 3);
            __syncthreads();
            if (L >= k0 + 1) {
                const int cur = L - 2;
                if (tx < wact && ty < hact) {  // march-axis face between cur and cur+1, planes cur-1 .. cur+2
                    R s[4][NV];
                    const int e = (ND == 3) ? (ty + 2) * PX + tx + 2 : tx + 2;
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const R *pl = sW + (size_t)((cur - 1 + o) & 3) * NV * PC;
#pragma unroll
                        for (int q = 0; q < NV; ++q) s[o][q] = pl[(size_t)q * PC + e];
                    }
                    face_flux<ND, R, PLM>(s, DM, kc, Fmhi);
                }
                if (cur >= k0) inplane_faces(cur & 3);
                __syncthreads();
                if (cur >= k0) {
                    S uc[NV], ub[NV];
                    prefetch_cell(cur, uc, ub);
                    update_cell(cur, Fmlo, Fmhi, uc, ub);
                }
#pragma unroll
                for (int q = 0; q < NV; ++q) Fmlo[q] = Fmhi[q];
            } else {
                __syncthreads();
            }
        }
    }
    if constexpr (MIX) {
        const double c = mx::f2d(wmin_f);
        wmin = c < wmin ? c : wmin;
    }
}

// Block-wide reduction of the status bits, floor count and (stage 2) CFL
// minimum into one clock.  Every thread of the block must call it.
template <int STAGE, int NT>
__device__ __forceinline__ void reduce_to_clock(Clock *clk, unsigned flags, unsigned floors, double wmin) {
    __shared__ unsigned s_flags;
    __shared__ unsigned long long s_floors;
    __shared__ double s_wmin[32];
    const int tid = threadIdx.x;
    __syncthreads();
    if (tid == 0) { s_flags = 0; s_floors = 0; }
    __syncthreads();
    const unsigned wf = __reduce_or_sync(0xffffffffu, flags);
    const unsigned wc = __reduce_add_sync(0xffffffffu, floors);
    double wm = wmin;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, wm, o);
        wm = other < wm ? other : wm;
    }
    if ((tid & 31) == 0) {
        if (wf) atomicOr(&s_flags, wf);
        if (wc) atomicAdd(&s_floors, (unsigned long long)wc);
        s_wmin[tid >> 5] = wm;
    }
    __syncthreads();
    if (tid == 0) {
        if (s_flags) atomicOr(&clk->status, s_flags);
        if (s_floors) atomicAdd(&clk->floor_hits, s_floors);
        if (STAGE == 2 || STAGE == 4 || STAGE == 6) {
            double m = s_wmin[0];
            for (int i = 1; i < NT / 32; ++i) m = s_wmin[i] < m ? s_wmin[i] : m;
            if (m < __longlong_as_double((long long)kInfBits))
                atomicMin(&clk->wmin_bits, (unsigned long long)__double_as_longlong(m));
        }
    }
}

// Mixed path: cap registers at 64 per thread so that 1024 threads per SM stay
// resident (four 256-thread CTAs of a 3D tile); the all-FP64 path is limited
// by shared memory instead.
template <class R, int NT>  // NT: threads per CTA
struct MinBlocks {
    static constexpr int value = std::is_same<R, float>::value ? (1024 / NT > 0 ? 1024 / NT : 1) : 1;
};

template <class R, int ND, int STAGE, int TX, int TY, class S = double>
__global__ void __launch_bounds__(cta_threads<R, ND, TX, TY>(), MinBlocks<R, cta_threads<R, ND, TX, TY>()>::value)
    stage_kernel(StageArgs a) {
    using T = Tile<ND, TX, TY>;
    constexpr int NTH = cta_threads<R, ND, TX, TY>();
    constexpr int DM = ND - 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sW = reinterpret_cast<R *>(smem_raw);   // [NSLOT][NV][PC] primitives
    R *sFx = sW + T::OFF_FX;  // [NV][TY][TX+1] x-face fluxes
    R *sFy = sW + T::OFF_FY;  // [NV][TY+1][TX] y-face fluxes (3D)

    const Geom &g = a.g;
    const Clock *clk = a.clk;
    if (!clk->active) return;
    const double dtdx[3] = {clk->dtdx[0], clk->dtdx[1], clk->dtdx[2]};

    const int ntx = (g.n[0] + TX - 1) / TX;
    const int nty = (ND == 3) ? (g.n[1] + TY - 1) / TY : 1;
    const int nm = (ND >= 2) ? g.n[DM] : 1;
    const long long total = (long long)ntx * nty * nm;

    unsigned flags = 0, floors = 0;
    double wmin = __longlong_as_double((long long)kInfBits);
    if (a.nchunk > 0 && ND >= 2) {
        // unit = one run of planes [kb[c], kb[c + 1]) of one tile column,
        // numbered chunk-major: CTAs that run at the same
        // time hold neighbouring tiles at the same planes, so the halo rows
        // they share are read from HBM once and from L2 after that, and the
        // hardware hands the units to CTA slots as they free up
        const long long ntile = (long long)ntx * nty;
        const int nch = a.nchunk;
        const long long units = ntile * nch;
        for (long long u = blockIdx.x; u < units; u += gridDim.x) {
            const long long tile = u % ntile;
            const int c = (int)(u / ntile);
            const int k0 = a.kb[c], k1 = a.kb[c + 1];
            const int x0 = (int)(tile % ntx) * TX;
            const int y0 = (ND == 3) ? (int)(tile / ntx) * TY : 0;
            run_segment<R, ND, STAGE, TX, TY, S>(g, reinterpret_cast<const S *>(a.Uin), reinterpret_cast<const S *>(a.Ubase),
                                                 reinterpret_cast<S *>(a.Uout), reinterpret_cast<const R *>(a.Win),
                                                 reinterpret_cast<R *>(a.Wout), dtdx, a.cubic, x0, y0, k0, k1, sW, sFx,
                                                 sFy, flags, floors, wmin);
        }
        reduce_to_clock<STAGE, NTH>(a.clk, flags, floors, wmin);
        return;
    }
    const long long s0 = total * blockIdx.x / gridDim.x;
    const long long s1 = total * (blockIdx.x + 1) / gridDim.x;
    for (long long pos = s0; pos < s1;) {
        const long long tile = pos / nm;
        const int k0 = (int)(pos % nm);
        const int k1 = (int)((long long)nm < k0 + (s1 - pos) ? (long long)nm : k0 + (s1 - pos));
        const int x0 = (int)(tile % ntx) * TX;
        const int y0 = (ND == 3) ? (int)(tile / ntx) * TY : 0;
        pos += k1 - k0;
        run_segment<R, ND, STAGE, TX, TY, S>(g, reinterpret_cast<const S *>(a.Uin), reinterpret_cast<const S *>(a.Ubase),
                                             reinterpret_cast<S *>(a.Uout), reinterpret_cast<const R *>(a.Win),
                                             reinterpret_cast<R *>(a.Wout), dtdx, a.cubic, x0, y0, k0, k1, sW, sFx,
                                             sFy, flags, floors, wmin);
    }
    reduce_to_clock<STAGE, NTH>(a.clk, flags, floors, wmin);
}

// ---------------------------------------------------------------- many grids
// Batched and served workloads: many independent grids (one dimensionality,
// one precision) in one pooled state, each with its own clock and dt.  One
// launch per stage covers all grids; CTA b runs its precomputed list of
// segments (tile runs), balanced by cells on the host.

struct GridDesc {
    Geom g;
    long long off;  // offset (in doubles) of the grid's state in the pools
    int cubic;
    int pad;
};

struct SegDesc {
    int grid;
    int x0, y0;  // tile origin
    int k0, k1;  // march-axis planes [k0, k1)
};

struct MultiArgs {
    const GridDesc *grids;
    const SegDesc *segs;
    const int *cta_seg;  // CTA b runs segments [cta_seg[b], cta_seg[b + 1])
    const double *Uin;   // pool the stage adds to (U or U1)
    const double *Ubase; // U pool (Heun average)
    double *Uout;        // U1 pool (stage 5) or U pool (stage 6)
    const void *Win;     // primitive pool the fluxes come from (W0 or W1, flux precision)
    void *Wout;          // primitive pool written (W1 or W0)
    Clock *clocks;       // one per grid
    int *queue;          // non-null: persistent CTAs take segments 0 .. nseg - 1 in order from
                         // this counter (zeroed before the launch) instead of cta_seg
    int nseg;
};

template <class R, int ND, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(cta_threads<R, ND, TX, TY>(), MinBlocks<R, cta_threads<R, ND, TX, TY>()>::value)
    multi_stage_kernel(MultiArgs a) {
    using T = Tile<ND, TX, TY>;
    constexpr int NTH = cta_threads<R, ND, TX, TY>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sW = reinterpret_cast<R *>(smem_raw);
    R *sFx = sW + T::OFF_FX;
    R *sFy = sW + T::OFF_FY;
    auto run_one = [&](int si) {
        const SegDesc sd = a.segs[si];
        Clock *clk = a.clocks + sd.grid;
        if (!clk->active) return;  // same value for every thread of the CTA
        const GridDesc *gd = a.grids + sd.grid;
        const Geom g = gd->g;
        const double dtdx[3] = {clk->dtdx[0], clk->dtdx[1], clk->dtdx[2]};
        unsigned flags = 0, floors = 0;
        double wmin = __longlong_as_double((long long)kInfBits);
        run_segment<R, ND, STAGE, TX, TY>(g, a.Uin + gd->off, a.Ubase + gd->off, a.Uout + gd->off,
                                          reinterpret_cast<const R *>(a.Win) + gd->off,
                                          reinterpret_cast<R *>(a.Wout) + gd->off, dtdx, gd->cubic,
                                          sd.x0, sd.y0, sd.k0, sd.k1, sW, sFx, sFy, flags, floors, wmin);
        reduce_to_clock<STAGE, NTH>(clk, flags, floors, wmin);
    };
    if (a.queue != nullptr) {
        // persistent CTA: the next segment from the shared counter (segments
        // are ordered longest first, so the last ones to start are short)
        __shared__ int s_next;
        for (;;) {
            __syncthreads();  // every thread has read the previous s_next
            if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
            __syncthreads();
            const int si = s_next;
            if (si >= a.nseg) break;
            run_one(si);
        }
        return;
    }
    const int sb = a.cta_seg[blockIdx.x], se = a.cta_seg[blockIdx.x + 1];
    for (int si = sb; si < se; ++si) run_one(si);
}

// Per-grid CFL minimum of every grid over the same segments (after the
// states were set from outside); also stores every cell's primitives in the
// pool W (flux precision) for the stages that read stored primitives.
template <class R, int ND>
__global__ void __launch_bounds__(256) multi_dt_kernel(MultiArgs a, int TX, int TY, R *W) {
    constexpr bool MIX = std::is_same<R, float>::value;
    constexpr int NV = ND + 2;
    const int sb = a.cta_seg[blockIdx.x], se = a.cta_seg[blockIdx.x + 1];
    for (int si = sb; si < se; ++si) {
        const SegDesc sd = a.segs[si];
        const GridDesc *gd = a.grids + sd.grid;
        const Geom g = gd->g;
        const mx::MixConsts mk = mx::make_mix(g);
        const long long N = g.ncell;
        const double *U = a.Uin + gd->off;
        const int w = min(TX, g.n[0] - sd.x0);
        const int h = (ND == 3) ? min(TY, g.n[1] - sd.y0) : 1;
        const long long cnt = (long long)w * h * (sd.k1 - sd.k0);
        unsigned flags = 0, floors = 0;
        double wmin = __longlong_as_double((long long)kInfBits);
        for (long long i = threadIdx.x; i < cnt; i += blockDim.x) {
            const int cx = sd.x0 + (int)(i % w);
            const int cy = (ND == 3) ? sd.y0 + (int)((i / w) % h) : 0;
            const int cm = sd.k0 + (int)(i / ((long long)w * h));
            const long long c = (ND == 3) ? ((long long)cm * g.n[1] + cy) * g.n[0] + cx
                                          : (ND == 2 ? (long long)cm * g.n[0] + cx : (long long)cx);
            double u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = U[(long long)q * N + c];
            double m;
            R wv[NV];
            if constexpr (MIX) {
                mx::recover<ND>(u, mk, wv, flags, floors);
                m = mx::f2d(mx::cfl_from_prim<ND>(wv, mk));
            } else {
                recover<ND>(u, g, wv, flags, floors);
                m = cfl_candidate<ND>(wv, g);
            }
#pragma unroll
            for (int q = 0; q < NV; ++q) W[gd->off + (long long)q * N + c] = wv[q];
            wmin = m < wmin ? m : wmin;
        }
        reduce_to_clock<2, 256>(a.clocks + sd.grid, flags, 0u, wmin);
    }
}

// CFL minimum over all cells of U (used when the state was set from outside);
// the same per-cell candidate as the fused one in stage_kernel<..., 2, ...>.
// When W is not null it also stores the primitives of U (type R) for the
// stages that read stored primitives.
// from_state (mixed / FP32 van Leer): the corrector's estimate from the state.
template <class R, int ND, class S = double>
__global__ void __launch_bounds__(256) dt_kernel(Geom g, const double *U, Clock *clk, R *W, int from_state) {
    constexpr bool MIX = std::is_same<R, float>::value;
    constexpr bool SINGLE = std::is_same<S, float>::value;
    constexpr int NV = ND + 2;
    const mx::MixConsts mk = mx::make_mix(g);
    const long long N = g.ncell;
    unsigned flags = 0, floors = 0;
    double wmin = __longlong_as_double((long long)kInfBits);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double m;
        if constexpr (SINGLE) {
            const float *Uf = reinterpret_cast<const float *>(U);
            float u[NV], w[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = Uf[(long long)q * N + c];
            sg::recover<ND>(u, mk, w, flags, floors);
            m = from_state ? mx::f2d(mx::cfl_from_state<ND>(u, mk)) : mx::f2d(mx::cfl_from_prim<ND>(w, mk));
            if (W) {
#pragma unroll
                for (int q = 0; q < NV; ++q) W[(long long)q * N + c] = w[q];
            }
        } else if constexpr (MIX) {
            double u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = U[(long long)q * N + c];
            float w[NV];
            mx::recover<ND>(u, mk, w, flags, floors);
            m = from_state ? mx::f2d(mx::cfl_from_state<ND>(u, mk)) : mx::f2d(mx::cfl_from_prim<ND>(w, mk));
            if (W) {
#pragma unroll
                for (int q = 0; q < NV; ++q) W[(long long)q * N + c] = w[q];
            }
        } else {
            double u[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = U[(long long)q * N + c];
            double w[NV];
            recover<ND>(u, g, w, flags, floors);
            m = cfl_candidate<ND>(w, g);
            if (W) {
#pragma unroll
                for (int q = 0; q < NV; ++q) W[(long long)q * N + c] = w[q];
            }
        }
        wmin = m < wmin ? m : wmin;
    }
    __shared__ double s_w[8];
    __shared__ unsigned s_f;
    if (threadIdx.x == 0) s_f = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double other = __shfl_xor_sync(0xffffffffu, wmin, o);
        wmin = other < wmin ? other : wmin;
    }
    const unsigned wf = __reduce_or_sync(0xffffffffu, flags);
    if ((threadIdx.x & 31) == 0) {
        s_w[threadIdx.x >> 5] = wmin;
        if (wf) atomicOr(&s_f, wf);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = s_w[0];
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = s_w[i] < m ? s_w[i] : m;
        atomicMin(&clk->wmin_bits, (unsigned long long)__double_as_longlong(m));
        if (s_f) atomicOr(&clk->status, s_f);
    }
}

}  // namespace khy
