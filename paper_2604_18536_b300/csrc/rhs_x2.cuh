// FP32 stage evaluation with two cells per thread along x (paper App. A discrete momentum
// equation, App. B kernels; the RK stage boundary of Sec. 2.6.1): the same arithmetic per cell
// as k_rhs_div / k_update_rhs_div, with fewer instructions per cell.
//
// A CTA of 32 x 8 threads owns a 64 x 8 column of cells; thread (tx, ty) owns the cells
// i0 + 2 tx and i0 + 2 tx + 1 of row j0 + ty. Planes are staged as pairs of cells (8-byte
// loads and shared-memory accesses): columns i0 - 2 .. i0 + 65 (34 pairs), rows j0 - 2 ..
// j0 + 8. Because nx is even and tiles start at multiples of 64, a pair never straddles the
// periodic wrap. The neighbour values of the two cells are shared: of the 34 values the two F
// evaluations read per plane, 17 pair loads come from shared memory, the rest from registers
// (the previous plane's values and the partner cell's).
//
// The z march keeps five planes in a shared ring (m = k - 1, o = k, p = k + 1, the staged
// plane k + 2 and plane k + 3 being staged) and exchanges F^y across rows through a
// double-buffered row array, so one barrier per plane suffices: iteration k stages plane k + 3
// from the registers loaded in iteration k - 1 into the slot of plane k - 2, which no thread
// reads after the previous barrier, then issues the loads of plane k + 4 (every load has a
// whole plane iteration to arrive, with one plane's inputs in flight); the F^y rows of plane k
// are read after this plane's barrier and rewritten two planes later. F^x of the left
// neighbour comes from the neighbouring lane (shuffle); F^x left of the tile and F^y below it
// are computed by lanes of warps 1 and 0.
//
// STAGE = false: the stage evaluation of a stored field u (stage 1 of a step).
// STAGE = true:  the fused RK stage boundary: plane cells are staged from F_s, p_s and u_0 as
//   u_{s+1} = u_0 + dt a_{s+1,s} (F_s - G p_s), and the RK accumulator is updated at the
//   own cells (acc = b_s k or acc += b_s k), as in k_update_rhs_div.
// STS (with STAGE): no accumulator; the staged u_{s+1} of the own cells is stored to fa.ust
//   (the stage states of the step VJP's recomputation).
// Requirements (checked by the caller): nx even, every field 8-byte aligned, 3 x cells < 2^31.
#pragma once

#include "rhs.cuh"

namespace ins {

constexpr int PX = RBX + 2;                  // pairs of a staged row
constexpr int PSX = 2 * PX;                  // floats of a staged row
constexpr int PLN = PX * RSY;                // pairs of a staged plane
constexpr int PH = 3 * PX + 2 * (RSY - 3);   // halo pairs of a plane: rows 0, 1, RSY - 1 and the
                                             // first and last pair of rows 2 .. RSY - 2 (118)
static_assert(RNT / 2 + PH <= RNT, "halo pairs are staged by threads 128 .. 245");

using PairPlane = const float (*)[2 * PLN];  // flat float view of a ring slot: [comp][row * PSX + column]

struct PairMap {
    int off[2];      // in-plane offset of the pair's first cell (mirror row for a wall ghost)
    int sidx[2];     // pair index in the shared plane
    int dxp[2];      // offset from the first cell to the +x neighbour of the second (wrap)
    int dyp[2];      // offset of the +y neighbour row (wrap; unused on the top wall row)
    int gj[2];       // source row
    bool ghost[2];   // wall ghost row: u^x, u^z negated, u^y = 0
    bool has[2];     // element 1 exists for threads 128 .. 128 + PH - 1
};

template <bool WALL>
__device__ __forceinline__ PairMap pair_map(int nx, int ny, int i0, int j0) {
    PairMap pm;
    const int t = threadIdx.x + threadIdx.y * RBX;
    const int h = t - RNT / 2;
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        int q = threadIdx.x + 1, lj = threadIdx.y + 2;
        pm.has[e] = e == 0 || (h >= 0 && h < PH);
        if (e == 1 && pm.has[1]) {
            if (h < 3 * PX) {
                const int rr = h / PX;
                lj = rr == 2 ? RSY - 1 : rr;
                q = h - rr * PX;
            } else {
                const int hh = h - 3 * PX;
                lj = 2 + (hh >> 1);
                q = (hh & 1) ? PX - 1 : 0;
            }
        }
        pm.sidx[e] = lj * PX + q;
        int gi = (i0 - 2 + 2 * q) % nx;
        if (gi < 0) gi += nx;
        int gj = j0 - 2 + lj;
        pm.ghost[e] = false;
        if (!WALL) {
            gj %= ny;
            if (gj < 0) gj += ny;
        } else if (gj < 0 || gj >= ny) {
            const int mj = gj < 0 ? -gj - 1 : 2 * ny - 1 - gj;
            gj = mj < 0 ? 0 : (mj >= ny ? ny - 1 : mj);
            pm.ghost[e] = true;
        }
        pm.gj[e] = gj;
        pm.off[e] = gj * nx + gi;
        pm.dxp[e] = gi + 2 == nx ? -gi : 2;
        pm.dyp[e] = gj + 1 == ny ? -(ny - 1) * nx : nx;
    }
    return pm;
}

__device__ __forceinline__ float2 ld2(const float* __restrict__ b, int a) {
    return *reinterpret_cast<const float2*>(b + a);
}
__device__ __forceinline__ void st2(float* __restrict__ b, int a, float x, float y) {
    *reinterpret_cast<float2*>(b + a) = make_float2(x, y);
}

// Packed FP32 pairs: the two cells of a thread run the same arithmetic, so the F evaluations
// use the paired instructions add/sub/mul/fma.rn.f32x2 (each lane rounds like the scalar
// instruction, so the results are those of nb_Fx / nb_Fy / nb_Fz bit for bit).
union P2 {
    float2 f;
    unsigned long long u;
};
__device__ __forceinline__ float2 p2add(float2 a, float2 b) {
    P2 A, B, R;
    A.f = a;
    B.f = b;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(R.u) : "l"(A.u), "l"(B.u));
    return R.f;
}
__device__ __forceinline__ float2 p2mul(float2 a, float2 b) {
    P2 A, B, R;
    A.f = a;
    B.f = b;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(R.u) : "l"(A.u), "l"(B.u));
    return R.f;
}
__device__ __forceinline__ float2 p2fma(float2 a, float2 b, float2 c) {
    P2 A, B, C, R;
    A.f = a;
    B.f = b;
    C.f = c;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(R.u) : "l"(A.u), "l"(B.u), "l"(C.u));
    return R.f;
}
__device__ __forceinline__ float2 p2neg(float2 a) {   // exact: flips both sign bits
    P2 A;
    A.f = a;
    A.u ^= 0x8000000080000000ull;
    return A.f;
}
__device__ __forceinline__ float2 p2b(float x) { return make_float2(x, x); }

// The register neighbourhood of the two cells as pairs (field f = (cell a, cell b)).
struct NbP {
    float2 X0, X0e, X0w, X0n, X0s, X0wn;
    float2 Y0, Y0e, Y0w, Y0n, Y0s, Y0es;
    float2 Z0, Z0e, Z0w, Z0n, Z0s;
    float2 Xp, Xpw, Yp, Yps, Zp;
    float2 Xm, Ym, Zm, Zme, Zmn;
    float2 cx, cy, cz;
};

// Per-thread constants of the packed evaluations (the row coefficients do not change along z).
struct NbPC {
    float2 dx, dz, fx, fy, fz, bp, bm, ap, am, wl, wr;
    float2 ncx, ncz, ncx2, ncz2, nyf, nys;   // negated convection coefficients
    float2 ndsx, ndsy, ndsz;                 // negated diagonal diffusion sums of F^x, F^y, F^z
};

template <bool WALL>
__device__ __forceinline__ NbPC nbp_consts(const RhsCoef<float>& c, const YRow<float>& y) {
    NbPC k;
    k.dx = p2b(c.dx);
    k.dz = p2b(c.dz);
    k.fx = p2b(c.fx);
    k.fy = p2b(c.fy);
    k.fz = p2b(c.fz);
    k.bp = p2b(y.bp);
    k.bm = p2b(y.bm);
    k.ap = p2b(y.ap);
    k.am = p2b(y.am);
    k.wl = p2b(y.wl);
    k.wr = p2b(y.wr);
    k.ncx = p2b(-c.cx);
    k.ncz = p2b(-c.cz);
    k.ncx2 = p2b(-(WALL ? 2.f * c.cx : c.cx));
    k.ncz2 = p2b(-(WALL ? 2.f * c.cz : c.cz));
    k.nyf = p2b(-y.f);
    k.nys = p2b(-y.s);
    // the same sums as nb_Fx / nb_Fy / nb_Fz form
    float dsx = 2.f * c.dx + y.bp + y.bm;
    dsx += 2.f * c.dz;
    float dsy = 2.f * c.dx + y.ap + y.am;
    dsy += 2.f * c.dz;
    k.ndsx = p2b(-dsx);
    k.ndsy = p2b(-dsy);
    k.ndsz = p2b(-(2.f * (c.dx + c.dz) + y.bp + y.bm));
    return k;
}

__device__ __forceinline__ float2 nbp_Fx(const NbPC& k, NbP& v) {
    const float2 uc = v.X0, ue = v.X0e, uw = v.X0w, un = v.X0n, us = v.X0s;
    const float2 s1 = p2add(uc, ue), s2 = p2add(uw, uc);
    const float2 X = p2fma(s1, s1, p2neg(p2mul(s2, s2)));
    const float2 vp = p2add(v.Y0, v.Y0e), vm = p2add(v.Y0s, v.Y0es);
    const float2 Y = p2fma(vp, p2add(uc, un), p2neg(p2mul(vm, p2add(us, uc))));
    float2 acc = p2fma(k.dx, p2add(ue, uw), k.fx);
    acc = p2fma(k.bp, un, acc);
    acc = p2fma(k.bm, us, acc);
    const float2 ut = v.Xp, ub = v.Xm;
    const float2 wp = p2add(v.Z0, v.Z0e), sup = p2add(uc, ut);
    const float2 Z = p2fma(wp, sup, p2neg(v.cx));
    v.cx = p2mul(wp, sup);
    acc = p2fma(k.dz, p2add(ut, ub), acc);
    acc = p2fma(k.ncz, Z, acc);
    acc = p2fma(k.ndsx, uc, acc);
    acc = p2fma(k.ncx, X, acc);
    return p2fma(k.nyf, Y, acc);
}

template <bool WALL>
__device__ __forceinline__ float2 nbp_Fy(const NbPC& k, NbP& v) {
    const float2 uc = v.Y0, un = v.Y0n, us = v.Y0s, ue = v.Y0e, uw = v.Y0w;
    const float2 s1 = p2add(uc, un), s2 = p2add(us, uc);
    const float2 Ys = p2fma(s1, s1, p2neg(p2mul(s2, s2)));
    float2 vp, vm, wp;
    if constexpr (WALL) {
        vp = p2fma(k.wl, v.X0, p2mul(k.wr, v.X0n));
        vm = p2fma(k.wl, v.X0w, p2mul(k.wr, v.X0wn));
        wp = p2fma(k.wl, v.Z0, p2mul(k.wr, v.Z0n));
    } else {
        vp = p2add(v.X0, v.X0n);
        vm = p2add(v.X0w, v.X0wn);
        wp = p2add(v.Z0, v.Z0n);
    }
    const float2 X = p2fma(vp, p2add(uc, ue), p2neg(p2mul(vm, p2add(uw, uc))));
    float2 acc = p2fma(k.dx, p2add(ue, uw), k.fy);
    acc = p2fma(k.ap, un, acc);
    acc = p2fma(k.am, us, acc);
    const float2 ut = v.Yp, ub = v.Ym;
    const float2 sup = p2add(uc, ut);
    const float2 Z = p2fma(wp, sup, p2neg(v.cy));
    v.cy = p2mul(wp, sup);
    acc = p2fma(k.dz, p2add(ut, ub), acc);
    acc = p2fma(k.ncz2, Z, acc);
    acc = p2fma(k.ndsy, uc, acc);
    acc = p2fma(k.nys, Ys, acc);
    return p2fma(k.ncx2, X, acc);
}

__device__ __forceinline__ float2 nbp_Fz(const NbPC& k, NbP& v) {
    const float2 uc = v.Z0, ut = v.Zp, ub = v.Zm, ue = v.Z0e, uw = v.Z0w, un = v.Z0n, us = v.Z0s;
    const float2 s1 = p2add(uc, ut);
    const float2 Zs = p2fma(s1, s1, p2neg(v.cz));
    v.cz = p2mul(s1, s1);
    const float2 vp = p2add(v.X0, v.Xp), vm = p2add(v.X0w, v.Xpw);
    const float2 X = p2fma(vp, p2add(uc, ue), p2neg(p2mul(vm, p2add(uw, uc))));
    const float2 wp = p2add(v.Y0, v.Yp), wm = p2add(v.Y0s, v.Yps);
    const float2 Y = p2fma(wp, p2add(uc, un), p2neg(p2mul(wm, p2add(us, uc))));
    float2 acc = p2fma(k.dx, p2add(ue, uw), k.fz);
    acc = p2fma(k.dz, p2add(ut, ub), acc);
    acc = p2fma(k.bp, un, acc);
    acc = p2fma(k.bm, us, acc);
    acc = p2fma(k.ndsz, uc, acc);
    acc = p2fma(k.ncz, Zs, acc);
    acc = p2fma(k.ncx, X, acc);
    return p2fma(k.nyf, Y, acc);
}

// Register neighbourhood of the two cells from a ring slot (pair index idx of the own pair): the
// o-plane values not carried from the previous plane, the p plane, and the m plane with the
// carried o values of the first plane of a march.
__device__ __forceinline__ void nbp_load_o(NbP& v, const float2 (*o)[PLN], int idx) {
    const float* of0 = reinterpret_cast<const float*>(o[0]);
    const float* of1 = reinterpret_cast<const float*>(o[1]);
    const float* of2 = reinterpret_cast<const float*>(o[2]);
    const int f = 2 * idx;
    const float2 xn = o[0][idx + PX];
    v.X0e = make_float2(v.X0.y, of0[f + 2]);
    v.X0n = xn;
    v.X0s = o[0][idx - PX];
    v.X0wn = make_float2(of0[f + PSX - 1], xn.x);
    v.Y0e = make_float2(v.Y0.y, of1[f + 2]);
    v.Y0w = make_float2(of1[f - 1], v.Y0.x);
    v.Y0n = o[1][idx + PX];
    v.Y0es = make_float2(v.Y0s.y, of1[f - PSX + 2]);
    v.Z0e = make_float2(v.Z0.y, of2[f + 2]);
    v.Z0w = make_float2(of2[f - 1], v.Z0.x);
    v.Z0n = o[2][idx + PX];
    v.Z0s = o[2][idx - PX];
}

__device__ __forceinline__ void nbp_load_p(NbP& v, const float2 (*p)[PLN], int idx) {
    const float* pf0 = reinterpret_cast<const float*>(p[0]);
    v.Xp = p[0][idx];
    v.Xpw = make_float2(pf0[2 * idx - 1], v.Xp.x);
    v.Yp = p[1][idx];
    v.Yps = p[1][idx - PX];
    v.Zp = p[2][idx];
}

__device__ __forceinline__ void nbp_init(NbP& v, const float2 (*m)[PLN], const float2 (*o)[PLN], int idx) {
    const float* mf2 = reinterpret_cast<const float*>(m[2]);
    const float* of0 = reinterpret_cast<const float*>(o[0]);
    v.Xm = m[0][idx];
    v.Ym = m[1][idx];
    v.Zm = m[2][idx];
    v.Zme = make_float2(v.Zm.y, mf2[2 * idx + 2]);
    v.Zmn = m[2][idx + PX];
    v.X0 = o[0][idx];
    v.X0w = make_float2(of0[2 * idx - 1], v.X0.x);
    v.Y0 = o[1][idx];
    v.Y0s = o[1][idx - PX];
    v.Z0 = o[2][idx];
}

template <bool WALL>
__device__ __forceinline__ void nbp_carry_init(NbP& v, const NbPC& k) {
    v.cx = p2mul(p2add(v.Zm, v.Zme), p2add(v.Xm, v.X0));
    const float2 wm = WALL ? p2fma(k.wl, v.Zm, p2mul(k.wr, v.Zmn)) : p2add(v.Zm, v.Zmn);
    v.cy = p2mul(wm, p2add(v.Ym, v.Y0));
    const float2 s2 = p2add(v.Zm, v.Z0);
    v.cz = p2mul(s2, s2);
}

__device__ __forceinline__ void nbp_rotate(NbP& v) {
    v.Xm = v.X0;
    v.Ym = v.Y0;
    v.Zm = v.Z0;
    v.Zme = v.Z0e;
    v.Zmn = v.Z0n;
    v.X0 = v.Xp;
    v.X0w = v.Xpw;
    v.Y0 = v.Yp;
    v.Y0s = v.Yps;
    v.Z0 = v.Zp;
}

// Grid (ceil(nx/64), ceil(ny/8), ceil(nz/kchunk)), block (32, 8), dynamic shared memory
// PairRegSmem::BYTES: CTAs that are resident together march neighbouring columns of the same
// z chunk in step, so the halo re-reads hit in L2.
struct PairRegSmem {
    static constexpr int RING = 0;
    static constexpr int FY = 5 * 3 * PLN;
    static constexpr int FXH = FY + 2 * (RBY + 1) * RBX;
    static constexpr int BYTES = FXH * 8 + 2 * RBY * 4;
};

// Resident CTAs per SM the kernel is compiled for: the plain periodic evaluation fits 80
// registers (three CTAs); the staged and the wall variants keep 128 (two CTAs, no spills).
constexpr int pair_ctas_per_sm(bool wall, bool stage) { return (stage || wall) ? 2 : 3; }

template <bool WALL, bool STAGE, bool STS = false>
__global__ void __launch_bounds__(RNT, pair_ctas_per_sm(WALL, STAGE))
    k_rhs_div_x2(RhsCoef<float> c, float ihx, float ihz, const float* __restrict__ ihy, const float* __restrict__ Fs,
                  const float* __restrict__ p, const float* __restrict__ u0, float* __restrict__ acc,
                  float* __restrict__ F, float* __restrict__ r, FusedArgs fa, int kchunk) {
    extern __shared__ __align__(16) float2 smem2[];
    float2 (*const su)[3][PLN] = reinterpret_cast<float2 (*)[3][PLN]>(smem2 + PairRegSmem::RING);
    float2 (*const sFy)[RBY + 1][RBX] = reinterpret_cast<float2 (*)[RBY + 1][RBX]>(smem2 + PairRegSmem::FY);
    float (*const sFxh)[RBY] = reinterpret_cast<float (*)[RBY]>(smem2 + PairRegSmem::FXH);
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const int N = nx * ny * nz;   // component stride: offsets of all three components fit in 32 bits
    const int iplane = nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y;
    float dta = 0.f, bb = 0.f;
    if constexpr (STAGE) {
        const double dt = fa.dt_dev ? *fa.dt_dev : fa.dt_host;
        dta = (float)(dt * fa.a_next);
        bb = (float)fa.b;
    }
    auto wrapz = [nz](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    const int kb = blockIdx.z * kchunk;
    const int ke = min(kb + kchunk, nz);
    const int i0 = blockIdx.x * (2 * RBX), j0 = blockIdx.y * RBY;
    const int i = i0 + 2 * tx, j = j0 + ty;
    const bool inside = i < nx && j < ny;
    const int idx = (ty + 2) * PX + tx + 1;   // own pair in a ring slot
    const YRow<float> yr = yrow<float, WALL>(c, j < ny ? j : ny - 1);
    const bool hy = ty == 0;
    const bool hx = ty == 1 && tx < RBY;
    const bool hy_wall = WALL && j0 == 0;
    const int jhy = j0 - 1 < 0 ? ny - 1 : j0 - 1;
    const int jhx = j0 + tx < ny ? j0 + tx : ny - 1;
    const YRow<float> yh = yrow<float, WALL>(c, hy ? jhy : jhx);
    const int f0hy = 1 * PSX + 2 + 2 * tx;
    const int f0hx = (tx + 2) * PSX + 1;
    const PairMap pm = pair_map<WALL>(nx, ny, i0, j0);
    auto slot = [kb](int q) { return (q - kb + 2) % 5; };

    float ihy_e[2];
    bool top_e[2];
    float2 pself[2];
    if constexpr (STAGE) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            ihy_e[e] = __ldg(&ihy[pm.gj[e]]);
            top_e[e] = WALL && pm.gj[e] == ny - 1;
            pself[e] = pm.has[e] ? ld2(p, wrapz(kb - 2) * iplane + pm.off[e]) : make_float2(0.f, 0.f);
        }
    }
    float2 lF[3][2], lU[3][2], lpy[2], lpz[2];
    float2 lA[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    float lpx[2];
    int la0 = 0;
    bool lown = false;
    auto stage_load = [&](int q) {
        const int base = wrapz(q) * iplane;
        lown = STAGE && q >= kb && q < ke && inside;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!pm.has[e]) continue;
            const int a = base + pm.off[e];
            if (e == 0) la0 = a;
            lU[0][e] = ld2(u0, a);
            lU[1][e] = ld2(u0, a + N);
            lU[2][e] = ld2(u0, a + 2 * N);
            if constexpr (STAGE) {
                lF[0][e] = ld2(Fs, a);
                lF[1][e] = ld2(Fs, a + N);
                lF[2][e] = ld2(Fs, a + 2 * N);
                lpx[e] = p[a + pm.dxp[e]];
                lpy[e] = ld2(p, a + pm.dyp[e]);
                lpz[e] = ld2(p, wrapz(q + 1) * iplane + pm.off[e]);
            }
        }
        if constexpr (STAGE && !STS) {
            if (lown && fa.stage > 0) {
                lA[0] = ld2(acc, la0);
                lA[1] = ld2(acc, la0 + N);
                lA[2] = ld2(acc, la0 + 2 * N);
            }
        }
    };
    // u_{s+1} of the loaded plane into ring slot s (and the accumulator at the own cells)
    auto stage_finish = [&](int s) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (!pm.has[e]) continue;
            float2 ux = lU[0][e], uy = lU[1][e], uz = lU[2][e];
            if constexpr (STAGE) {
                const float2 p0 = pself[e];
                pself[e] = lpz[e];
                const float kx0 = fmaf(p0.x - p0.y, ihx, lF[0][e].x);
                const float kx1 = fmaf(p0.y - lpx[e], ihx, lF[0][e].y);
                const float ky0 = top_e[e] ? 0.f : fmaf(p0.x - lpy[e].x, ihy_e[e], lF[1][e].x);
                const float ky1 = top_e[e] ? 0.f : fmaf(p0.y - lpy[e].y, ihy_e[e], lF[1][e].y);
                const float kz0 = fmaf(p0.x - lpz[e].x, ihz, lF[2][e].x);
                const float kz1 = fmaf(p0.y - lpz[e].y, ihz, lF[2][e].y);
                ux = make_float2(fmaf(dta, kx0, ux.x), fmaf(dta, kx1, ux.y));
                uy = make_float2(fmaf(dta, ky0, uy.x), fmaf(dta, ky1, uy.y));
                uz = make_float2(fmaf(dta, kz0, uz.x), fmaf(dta, kz1, uz.y));
                if constexpr (STS) {
                    if (e == 0 && lown) {
                        st2(fa.ust, la0, ux.x, ux.y);
                        st2(fa.ust, la0 + N, uy.x, uy.y);
                        st2(fa.ust, la0 + 2 * N, uz.x, uz.y);
                    }
                } else if (e == 0 && lown) {
                    if (fa.stage == 0) {
                        st2(acc, la0, bb * kx0, bb * kx1);
                        st2(acc, la0 + N, bb * ky0, bb * ky1);
                        st2(acc, la0 + 2 * N, bb * kz0, bb * kz1);
                    } else {
                        st2(acc, la0, fmaf(bb, kx0, lA[0].x), fmaf(bb, kx1, lA[0].y));
                        st2(acc, la0 + N, fmaf(bb, ky0, lA[1].x), fmaf(bb, ky1, lA[1].y));
                        st2(acc, la0 + 2 * N, fmaf(bb, kz0, lA[2].x), fmaf(bb, kz1, lA[2].y));
                    }
                }
            }
            if (WALL && pm.ghost[e]) {
                ux = make_float2(-ux.x, -ux.y);
                uy = make_float2(0.f, 0.f);
                uz = make_float2(-uz.x, -uz.y);
            }
            su[s][0][pm.sidx[e]] = ux;
            su[s][1][pm.sidx[e]] = uy;
            su[s][2][pm.sidx[e]] = uz;
        }
    };
    auto flat = [&](int s) { return reinterpret_cast<PairPlane>(su[s]); };

    // prologue: planes kb - 2 .. kb + 2, F^z one plane below the chunk, loads of plane kb + 3
    for (int q = kb - 2; q <= kb + 2 && q <= ke; ++q) {
        stage_load(q);
        stage_finish(slot(q));
    }
    if (kb + 3 <= ke) stage_load(kb + 3);
    __syncthreads();
    float fzp0, fzp1;
    {
        const PairPlane m = flat(slot(kb - 2)), o = flat(slot(kb - 1)), pp = flat(slot(kb));
        fzp0 = eval_Fz<float, WALL, PSX, PairPlane>(c, yr, m, o, pp, 2 * idx);
        fzp1 = eval_Fz<float, WALL, PSX, PairPlane>(c, yr, m, o, pp, 2 * idx + 1);
    }
    const NbPC kp = nbp_consts<WALL>(c, yr);
    NbP nv;
    nbp_init(nv, su[slot(kb - 1)], su[slot(kb)], idx);
    nbp_carry_init<WALL>(nv, kp);
    __syncthreads();   // the slot of plane kb - 2 is refilled in the first iteration

    int buf = 0;
    for (int k = kb; k < ke; ++k) {
        if (k + 3 <= ke) {
            stage_finish(slot(k + 3));
            if (k + 4 <= ke) stage_load(k + 4);
        }
        const int sm = slot(k - 1), so = slot(k), sp = slot(k + 1);
        nbp_load_o(nv, su[so], idx);
        nbp_load_p(nv, su[sp], idx);
        const float2 fxp = nbp_Fx(kp, nv), fyp = nbp_Fy<WALL>(kp, nv), fzp = nbp_Fz(kp, nv);
        const float fx0 = fxp.x, fx1 = fxp.y, fz0 = fzp.x, fz1 = fzp.y;
        float fy0 = fyp.x, fy1 = fyp.y;
        if (WALL && j == ny - 1) fy0 = fy1 = 0.f;
        sFy[buf][ty + 1][tx] = make_float2(fy0, fy1);
        if (hy) {
            float h0 = 0.f, h1 = 0.f;
            if (!hy_wall) {
                const PairPlane m = flat(sm), o = flat(so), pp = flat(sp);
                h0 = eval_Fy<float, 3, WALL, PSX, PairPlane>(c, yh, m, o, pp, f0hy);
                h1 = eval_Fy<float, 3, WALL, PSX, PairPlane>(c, yh, m, o, pp, f0hy + 1);
            }
            sFy[buf][0][tx] = make_float2(h0, h1);
        }
        if (hx) sFxh[buf][tx] = eval_Fx<float, 3, WALL, PSX, PairPlane>(c, yh, flat(sm), flat(so), flat(sp), f0hx);
        __syncthreads();
        float fxm = __shfl_up_sync(0xffffffffu, fx1, 1);
        if (tx == 0) fxm = sFxh[buf][ty];
        const float2 fys = sFy[buf][ty][tx];
        if (inside) {
            const int a = k * iplane + j * nx + i;
            st2(F, a, fx0, fx1);
            st2(F, a + N, fy0, fy1);
            st2(F, a + 2 * N, fz0, fz1);
            st2(r, a, (fx0 - fxm) * c.ix + (fy0 - fys.x) * yr.i + (fz0 - fzp0) * c.iz,
                (fx1 - fx0) * c.ix + (fy1 - fys.y) * yr.i + (fz1 - fzp1) * c.iz);
        }
        fzp0 = fz0;
        fzp1 = fz1;
        nbp_rotate(nv);
        buf ^= 1;
    }
}

}  // namespace ins
