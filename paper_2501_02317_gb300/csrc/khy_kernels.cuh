// khy_kernels.cuh -- device code of the Godunov hydro step (sm_103a).
//
// One Heun step (Sec. 3.3) is three launches on one stream:
//   clock_kernel    : dt = C * min dx_d/(|v_d|+c_s) from the minimum that the
//                     previous stage-2 launch (or dt_kernel) accumulated; dt is
//                     clipped to t_end; t and the step counter advance.
//   stage_kernel<1> : U1 = Un + dt L(Un)
//   stage_kernel<2> : Un+1 = (Un + (U1 + dt L(U1))) / 2, written over Un, and
//                     the CFL minimum of Un+1 for the next step (Sec. 3.1: the
//                     step length is computed during the variable conversion).
//
// The stage kernel fuses the whole spatial operator: each CTA owns a tile of
// columns along the slowest ("march") axis -- z in 3D, y in 2D -- and walks
// it plane by plane.  Each plane of the conserved state, with two halo cells
// on every side, is loaded once, converted to primitives (Sec. 3.1) with the
// ghost-zone rules applied by index mapping (Sec. 3.1.1), and kept in a
// four-plane ring in shared memory (the row staging of Sec. 3.2.1, extended
// to a 2.5D march).  In-plane face fluxes are computed as a flat task list
// over the CTA's threads; the face along the march axis is computed by the
// thread that owns the column.  Each face flux is computed once per CTA and
// used with + on one cell and - on the other; faces on a tile edge are
// recomputed by the neighbouring CTA from the same inputs by the same code,
// so both sides see the identical value.
//
// Precision (Sec. 3.2.2): template parameter R is the reconstruction/Riemann
// type: double for the all-FP64 path, float for the mixed path.  The
// conserved state, the primitive recovery and the flux-difference
// accumulation are always FP64.
//
// The FP64 instantiation is compiled with -fmad=false and evaluates every
// floating-point operation in the same order as the CPU reference, so the
// two agree to the last bit.
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

// ------------------------------------------------------------ Sec. 3.1.1
// Maps coordinate x (possibly a ghost) onto an interior index along an axis
// with n cells and boundary rules (lo, hi).  *act receives the velocity rule
// for the normal component: 0 none, 1 negate (reflect), 2 min(v,0) (outflow,
// low side), 3 max(v,0) (outflow, high side).  Ghosts within two cells follow
// the boundary rules exactly; farther cells (only used by faces outside the
// interior) are clamped into range.
__device__ __forceinline__ int bc_map(int x, int n, int lo, int hi, int *act) {
    *act = 0;
    if (x >= 0 && x < n) return x;
    if (x < 0) {
        if (lo == BC_PERIODIC) { int r = x % n; return r < 0 ? r + n : r; }
        if (lo == BC_REFLECT) { *act = 1; int s = -x - 1; return s < n ? s : n - 1; }
        if (lo == BC_OUTFLOW) *act = 2;
        return 0;
    }
    if (hi == BC_PERIODIC) return x % n;
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
};

template <class R>
__device__ __forceinline__ Consts<R> make_consts(const Geom &g) {
    Consts<R> c;
    c.gamma = (R)g.gamma; c.gm1 = (R)g.gm1; c.g1 = (R)g.g1; c.gp1 = (R)g.gp1; c.gm1_gp1 = (R)g.gm1_gp1;
    return c;
}

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
    const R cl = sqrt(k.gamma * pl / rl);
    const R cr = sqrt(k.gamma * pr / rr);
    R ppv = R(0.5) * (pl + pr) - R(0.125) * (ur - ul) * (rl + rr) * (cl + cr);
    R pstar = ppv > R(0) ? ppv : R(0);
    R pmax = pl > pr ? pl : pr;
    if (pstar > pmax) {  // both waves are shocks: two-shock estimate
        R gl = sqrt((R(2) / (k.gp1 * rl)) / (pstar + k.gm1_gp1 * pl));
        R gr = sqrt((R(2) / (k.gp1 * rr)) / (pstar + k.gm1_gp1 * pr));
        pstar = (gl * pl + gr * pr - (ur - ul)) / (gl + gr);
    }
    R ratl = pstar / pl, ratr = pstar / pr;
    if (ratl < R(1)) ratl = R(1);
    if (ratr < R(1)) ratr = R(1);
    const R ql = sqrt(R(1) + k.g1 * (ratl - R(1)));
    const R qr = sqrt(R(1) + k.g1 * (ratr - R(1)));
    const R dsl = -cl * ql;
    const R dsr = cr * qr;
    const R sl = ul + dsl;
    const R sr = ur + dsr;
    const R sstar = ((pr - rr * ur * dsr) - (pl - rl * ul * dsl)) / (rl * dsl - rr * dsr);

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
    R vsq = uk * uk;
#pragma unroll
    for (int j = 0; j < NT; ++j) vsq = vsq + w[2 + j] * w[2 + j];
    const R E = pk / k.gm1 + R(0.5) * rk * vsq;
    const R mf = rk * uk;
    R Uk[NT + 3], Fk[NT + 3];
    Uk[0] = rk; Uk[1] = rk * uk;
    Fk[0] = mf; Fk[1] = mf * uk + pk;
#pragma unroll
    for (int j = 0; j < NT; ++j) { Uk[2 + j] = rk * w[2 + j]; Fk[2 + j] = mf * w[2 + j]; }
    Uk[P] = E;
    Fk[P] = (E + pk) * uk;
    if (outside) {
#pragma unroll
        for (int q = 0; q < NT + 3; ++q) F[q] = Fk[q];
        return;
    }
    const R fac = rk * dsk / (sk - sstar);
    R Us[NT + 3];
    Us[0] = fac;
    Us[1] = fac * sstar;
#pragma unroll
    for (int j = 0; j < NT; ++j) Us[2 + j] = fac * w[2 + j];
    Us[P] = fac * (Uk[P] / rk + (sstar - uk) * (sstar + pk / (rk * dsk)));
#pragma unroll
    for (int q = 0; q < NT + 3; ++q) F[q] = Fk[q] + sk * (Us[q] - Uk[q]);
}

// Face flux from the four primitive cells around a face along direction dir
// (cells f-2, f-1 | f, f+1), primitives in storage order (rho, v_0.., p).
// Minmod PLM per primitive (undivided differences: minmod is positively
// homogeneous, so the dx factors of the slope cancel), then HLLC in the frame
// rotated onto dir.  F is returned in conserved order (mass, m_0.., E).
template <int ND, class R>
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
        R a = minmod<R>(s1 - s0, s2 - s1);
        wl[j] = s1 + R(0.5) * a;
        R b = minmod<R>(s2 - s1, s3 - s2);
        wr[j] = s2 - R(0.5) * b;
    }
    R Fr[NT + 3];
    hllc<R, NT>(k, wl, wr, Fr);
#pragma unroll
    for (int j = 0; j < ND + 2; ++j) F[slot[j]] = Fr[j];
}

// ---------------------------------------------------------- kernels

struct StageArgs {
    Geom g;
    const double *Uin;    // state the fluxes are computed from (Un or U1)
    const double *Ubase;  // Un (stage 2 average); unused in stage 1
    double *Uout;         // U1 (stage 1) or Un+1 (stage 2, may alias Ubase)
    Clock *clk;
    int kchunk;           // planes per CTA along the march axis
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
    template <class R>
    static constexpr size_t smem_bytes() {
        return sizeof(R) * ((size_t)NSLOT * NV * PC + (size_t)NV * NXF + (size_t)NV * NYF);
    }
};

template <int ND, class R, int STAGE, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) stage_kernel(StageArgs a) {
    using T = Tile<ND, TX, TY>;
    constexpr int NV = T::NV, PX = T::PX, PC = T::PC, NT = T::NT;
    constexpr int DM = ND - 1;  // march axis for ND >= 2
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sW = reinterpret_cast<R *>(smem_raw);          // [NSLOT][NV][PC]
    R *sFx = sW + (size_t)T::NSLOT * NV * PC;         // [NV][TY][TX+1]
    R *sFy = sFx + (size_t)NV * T::NXF;               // [NV][TY+1][TX]

    const Geom &g = a.g;
    const Clock *clk = a.clk;
    if (!clk->active) return;
    double dtdx[3] = {clk->dtdx[0], clk->dtdx[1], clk->dtdx[2]};
    const Consts<R> kc = make_consts<R>(g);
    const long long N = g.ncell;

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX;
    const int y0 = (ND == 3) ? blockIdx.y * TY : 0;
    const int chunk = (ND == 3) ? blockIdx.z : (ND == 2 ? blockIdx.y : 0);
    const int nm = (ND >= 2) ? g.n[DM] : 1;
    const int k0 = chunk * a.kchunk;
    const int k1 = min(k0 + a.kchunk, nm);

    unsigned flags = 0, floors = 0;
    double wmin = __longlong_as_double((long long)kInfBits);

    // load plane L (march coordinate; ignored in 1D) into ring slot
    auto load_plane = [&](int L, int slot) {
        R *dst = sW + (size_t)slot * NV * PC;
        for (int e = tid; e < PC; e += NT) {
            const int hx = e % PX, hy = e / PX;
            int act[3] = {0, 0, 0};
            int c[3] = {0, 0, 0};
            c[0] = bc_map(x0 - 2 + hx, g.n[0], g.bc[0][0], g.bc[0][1], &act[0]);
            if (ND == 3) {
                c[1] = bc_map(y0 - 2 + hy, g.n[1], g.bc[1][0], g.bc[1][1], &act[1]);
                c[2] = bc_map(L, g.n[2], g.bc[2][0], g.bc[2][1], &act[2]);
            } else if (ND == 2) {
                c[1] = bc_map(L, g.n[1], g.bc[1][0], g.bc[1][1], &act[1]);
            }
            const long long idx = ((long long)c[2] * g.n[1] + c[1]) * g.n[0] + c[0];
            double u[NV], w[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) u[q] = __ldg(a.Uin + (long long)q * N + idx);
            unsigned fl = 0;
            recover<ND>(u, g, w, flags, fl);
            const bool interior = hx >= 2 && hx < TX + 2 && x0 - 2 + hx < g.n[0] &&
                                  (ND != 3 || (hy >= 2 && hy < TY + 2 && y0 - 2 + hy < g.n[1])) &&
                                  (ND == 1 || (L >= k0 && L < k1));
            if (interior) floors += fl;
#pragma unroll
            for (int d = 0; d < ND; ++d) w[1 + d] = apply_vrule(w[1 + d], act[d]);
#pragma unroll
            for (int q = 0; q < NV; ++q) dst[(size_t)q * PC + e] = (R)w[q];
        }
    };

    // stencil gather along direction dir from a ring slot
    auto gather = [&](const R *base, int e0, int stride, R (&s)[4][NV]) {
#pragma unroll
        for (int o = 0; o < 4; ++o)
#pragma unroll
            for (int q = 0; q < NV; ++q) s[o][q] = base[(size_t)q * PC + e0 + o * stride];
    };

    // in-plane face fluxes of the plane in ring slot `slot` into sFx / sFy
    auto inplane_faces = [&](int slot) {
        const R *pl = sW + (size_t)slot * NV * PC;
        for (int f = tid; f < T::NXF + T::NYF; f += NT) {
            R s[4][NV], F[NV];
            if (f < T::NXF) {
                const int fx = f % (TX + 1), fy = f / (TX + 1);
                const int hy = (ND == 3) ? fy + 2 : 0;
                gather(pl, hy * PX + fx, 1, s);
                face_flux<ND, R>(s, 0, kc, F);
#pragma unroll
                for (int q = 0; q < NV; ++q) sFx[(size_t)q * T::NXF + f] = F[q];
            } else {
                const int f2 = f - T::NXF;
                const int fxx = f2 % TX, fyy = f2 / TX;
                gather(pl, fyy * PX + fxx + 2, PX, s);
                face_flux<ND, R>(s, 1, kc, F);
#pragma unroll
                for (int q = 0; q < NV; ++q) sFy[(size_t)q * T::NYF + f2] = F[q];
            }
        }
    };

    // update of the cell (tx, ty) of plane `cur` given the march-face fluxes
    auto update_cell = [&](int cur, const R (&Fmlo)[NV], const R (&Fmhi)[NV]) {
        const int gx = x0 + tx;
        const int gy = (ND == 3) ? y0 + ty : (ND == 2 ? cur : 0);
        const int gz = (ND == 3) ? cur : 0;
        if (gx >= g.n[0] || (ND == 3 && gy >= g.n[1])) return;
        const long long idx = ((long long)gz * g.n[1] + gy) * g.n[0] + gx;
        double acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const R *fx = sFx + (size_t)q * T::NXF + ty * (TX + 1) + tx;
            acc[q] = 0.0 - dtdx[0] * ((double)fx[1] - (double)fx[0]);
        }
        if (ND == 3) {
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const R *fy = sFy + (size_t)q * T::NYF + ty * TX + tx;
                acc[q] = acc[q] - dtdx[1] * ((double)fy[TX] - (double)fy[0]);
            }
        }
        if (ND >= 2) {
#pragma unroll
            for (int q = 0; q < NV; ++q) acc[q] = acc[q] - dtdx[DM] * ((double)Fmhi[q] - (double)Fmlo[q]);
        }
        double un[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const double u = a.Uin[(long long)q * N + idx];
            double r;
            if (STAGE == 1) r = u + acc[q];
            else r = 0.5 * (a.Ubase[(long long)q * N + idx] + (u + acc[q]));
            un[q] = r;
            a.Uout[(long long)q * N + idx] = r;
        }
        if (STAGE == 2) {
            double w[NV];
            unsigned fl = 0;
            recover<ND>(un, g, w, flags, fl);
            const double c = cfl_candidate<ND>(w, g);
            if (c < wmin) wmin = c;
        }
    };

    if (ND == 1) {
        load_plane(0, 0);
        __syncthreads();
        inplane_faces(0);
        __syncthreads();
        R dummy[NV];
        update_cell(0, dummy, dummy);
    } else {
        R Fmlo[NV], Fmhi[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) { Fmlo[q] = R(0); Fmhi[q] = R(0); }
        for (int L = k0 - 2; L <= k1 + 1; ++L) {
            load_plane(L, L & 3);
            __syncthreads();
            if (L >= k0 + 1) {
                const int cur = L - 2;
                // march face between cur and cur+1 from planes cur-1 .. cur+2
                {
                    R s[4][NV];
                    const int e = (ND == 3) ? (ty + 2) * PX + tx + 2 : tx + 2;
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const R *pl = sW + (size_t)((cur - 1 + o) & 3) * NV * PC;
#pragma unroll
                        for (int q = 0; q < NV; ++q) s[o][q] = pl[(size_t)q * PC + e];
                    }
                    face_flux<ND, R>(s, DM, kc, Fmhi);
                }
                if (cur >= k0) inplane_faces(cur & 3);
                __syncthreads();
                if (cur >= k0) update_cell(cur, Fmlo, Fmhi);
#pragma unroll
                for (int q = 0; q < NV; ++q) Fmlo[q] = Fmhi[q];
            } else {
                __syncthreads();
            }
        }
    }

    // block reductions: status bits, floor count, CFL minimum
    __shared__ unsigned s_flags;
    __shared__ unsigned long long s_floors;
    __shared__ double s_wmin[32];
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
        if (s_flags) atomicOr(&a.clk->status, s_flags);
        if (s_floors) atomicAdd(&a.clk->floor_hits, s_floors);
        if (STAGE == 2) {
            double m = s_wmin[0];
            for (int i = 1; i < NT / 32; ++i) m = s_wmin[i] < m ? s_wmin[i] : m;
            atomicMin(&a.clk->wmin_bits, (unsigned long long)__double_as_longlong(m));
        }
    }
}

// CFL minimum over all cells of U (used when the state was set from outside).
template <int ND>
__global__ void __launch_bounds__(256) dt_kernel(Geom g, const double *U, Clock *clk) {
    constexpr int NV = ND + 2;
    const long long N = g.ncell;
    unsigned flags = 0, floors = 0;
    double wmin = __longlong_as_double((long long)kInfBits);
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        double u[NV], w[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) u[q] = U[(long long)q * N + c];
        recover<ND>(u, g, w, flags, floors);
        const double m = cfl_candidate<ND>(w, g);
        if (m < wmin) wmin = m;
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
