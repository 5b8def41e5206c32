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

// Register neighbourhoods of the two cells from a ring slot (pair index idx of the own pair):
// values of the o plane not carried from the previous plane, and the p plane.
__device__ __forceinline__ void nb2_load_o(Nb<float>& a, Nb<float>& b, const float2 (*o)[PLN], int idx) {
    const float* of0 = reinterpret_cast<const float*>(o[0]);
    const float* of1 = reinterpret_cast<const float*>(o[1]);
    const float* of2 = reinterpret_cast<const float*>(o[2]);
    const int f = 2 * idx;   // flat index of the first cell
    const float2 xn = o[0][idx + PX], xs = o[0][idx - PX];
    a.X0e = b.X0;
    b.X0e = of0[f + 2];
    a.X0n = xn.x;
    b.X0n = xn.y;
    a.X0s = xs.x;
    b.X0s = xs.y;
    a.X0wn = of0[f + PSX - 1];
    b.X0wn = xn.x;
    const float2 yn = o[1][idx + PX];
    a.Y0e = b.Y0;
    b.Y0e = of1[f + 2];
    a.Y0w = of1[f - 1];
    b.Y0w = a.Y0;
    a.Y0n = yn.x;
    b.Y0n = yn.y;
    a.Y0es = b.Y0s;
    b.Y0es = of1[f - PSX + 2];
    const float2 zn = o[2][idx + PX], zs = o[2][idx - PX];
    a.Z0e = b.Z0;
    b.Z0e = of2[f + 2];
    a.Z0w = of2[f - 1];
    b.Z0w = a.Z0;
    a.Z0n = zn.x;
    b.Z0n = zn.y;
    a.Z0s = zs.x;
    b.Z0s = zs.y;
}

__device__ __forceinline__ void nb2_load_p(Nb<float>& a, Nb<float>& b, const float2 (*p)[PLN], int idx) {
    const float* pf0 = reinterpret_cast<const float*>(p[0]);
    const float2 xp = p[0][idx], yp = p[1][idx], yps = p[1][idx - PX], zp = p[2][idx];
    a.Xp = xp.x;
    b.Xp = xp.y;
    a.Xpw = pf0[2 * idx - 1];
    b.Xpw = xp.x;
    a.Yp = yp.x;
    b.Yp = yp.y;
    a.Yps = yps.x;
    b.Yps = yps.y;
    a.Zp = zp.x;
    b.Zp = zp.y;
}

// m plane and the carried o values of the first plane of a march
__device__ __forceinline__ void nb2_init(Nb<float>& a, Nb<float>& b, const float2 (*m)[PLN], const float2 (*o)[PLN],
                                         int idx) {
    const float* mf2 = reinterpret_cast<const float*>(m[2]);
    const float* of0 = reinterpret_cast<const float*>(o[0]);
    const float2 xm = m[0][idx], ym = m[1][idx], zm = m[2][idx], zmn = m[2][idx + PX];
    a.Xm = xm.x;
    b.Xm = xm.y;
    a.Ym = ym.x;
    b.Ym = ym.y;
    a.Zm = zm.x;
    b.Zm = zm.y;
    a.Zme = zm.y;
    b.Zme = mf2[2 * idx + 2];
    a.Zmn = zmn.x;
    b.Zmn = zmn.y;
    const float2 x0 = o[0][idx], y0 = o[1][idx], y0s = o[1][idx - PX], z0 = o[2][idx];
    a.X0 = x0.x;
    b.X0 = x0.y;
    a.X0w = of0[2 * idx - 1];
    b.X0w = x0.x;
    a.Y0 = y0.x;
    b.Y0 = y0.y;
    a.Y0s = y0s.x;
    b.Y0s = y0s.y;
    a.Z0 = z0.x;
    b.Z0 = z0.y;
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

template <bool WALL, bool STAGE>
__global__ void __launch_bounds__(RNT, 2)
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
        if constexpr (STAGE) {
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
                if (e == 0 && lown) {
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
    Nb<float> na, nb;
    nb2_init(na, nb, su[slot(kb - 1)], su[slot(kb)], idx);
    nb_carry_init<float, WALL>(na, yr);
    nb_carry_init<float, WALL>(nb, yr);
    __syncthreads();   // the slot of plane kb - 2 is refilled in the first iteration

    int buf = 0;
    for (int k = kb; k < ke; ++k) {
        if (k + 3 <= ke) {
            stage_finish(slot(k + 3));
            if (k + 4 <= ke) stage_load(k + 4);
        }
        const int sm = slot(k - 1), so = slot(k), sp = slot(k + 1);
        nb2_load_o(na, nb, su[so], idx);
        nb2_load_p(na, nb, su[sp], idx);
        const float fx0 = nb_Fx<float, WALL>(c, yr, na), fx1 = nb_Fx<float, WALL>(c, yr, nb);
        float fy0 = nb_Fy<float, WALL>(c, yr, na), fy1 = nb_Fy<float, WALL>(c, yr, nb);
        const float fz0 = nb_Fz<float, WALL>(c, yr, na), fz1 = nb_Fz<float, WALL>(c, yr, nb);
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
        nb_rotate<float>(na);
        nb_rotate<float>(nb);
        buf ^= 1;
    }
}

}  // namespace ins
