// FP32 pullback J_F^T w of a 3-D periodic grid with two x cells per thread (paper Sec. 3.4,
// pullback equation; App. B pullbacks), the same gather form and stage finish as k_adj_rhs_z.
//
// A CTA of 32 x 8 threads owns a 64 x 8 column (thread (tx, ty): cells i0 + 2 tx and
// i0 + 2 tx + 1 of row j0 + ty) and a chunk of planes. Planes k-1, k, k+1 of u and w (all
// three components) sit in a four-slot shared ring of 10 rows x 68 floats (cells i0-2 ..
// i0+65, rows j0-1 .. j0+8; pairs of even-aligned cells, so every shared and global access
// is one 8-byte load). The two cells' values at an x offset of -1 / +1 come from the
// neighbouring pairs (3 pair loads serve dx = -1, 0, +1), and the arithmetic of both cells
// runs in the paired FP32 instructions (each lane rounds like the scalar instruction).
// Plane k+2 is loaded into registers while plane k is computed and stored into the slot of
// plane k-2 before the iteration's single barrier.
// Needs nx even and 8-byte aligned fields; x and y wrap periodically for every staged cell.
#pragma once

#include "adjoint.cuh"
#include "rhs_x2.cuh"

namespace ins {

constexpr int AX2_ROW = 68;                    // floats per staged row (34 pairs)
constexpr int AX2_PL = AX2_ROW * 10;           // floats per component plane
constexpr int AX2_HALO = 2 * 34 + 2 * 8;       // halo pairs per plane (rows j0-1, j0+8; pair columns 0, 33)
constexpr int ax2_smem() { return 4 * 6 * AX2_PL * (int)sizeof(float); }

__device__ __forceinline__ float2 p2sub(float2 a, float2 b) { return p2add(a, p2neg(b)); }

static __global__ void __launch_bounds__(256, 2) k_adj_rhs_z2(AdjCoef<float> c, const float* __restrict__ u,
                                                       const float* __restrict__ w, const float* __restrict__ ybar,
                                                       float* __restrict__ ubar0, float* __restrict__ kb,
                                                       double* __restrict__ nu_part, const float* __restrict__ extra,
                                                       int kchunk, const float* __restrict__ uin) {
    extern __shared__ __align__(16) float ax2s[];   // [slot 4][comp 6][AX2_PL]
    const int nx = c.nx, ny = c.ny, nz = c.nz;
    const int N = nx * ny * nz;   // 3 N < 2^31 (checked by the caller)
    const int plane = nx * ny;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + 32 * ty;
    const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 8;
    const int i = i0 + 2 * tx, j = j0 + ty;
    const bool ok = i < nx && j < ny;
    const int kb0 = blockIdx.z * kchunk, ke = min(kb0 + kchunk, nz);
    const double dt = c.dt_dev ? *c.dt_dev : c.dt_host;
    const float2 dtb = p2b((float)(dt * c.bn)), dta = p2b((float)(dt * c.an));
    // staged pairs of this thread: its own and (tid < AX2_HALO) one halo pair
    int soff[2], goff[2];
    bool has[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        int row = ty + 1, pc = tx + 1;
        has[e] = e == 0 || tid < AX2_HALO;
        if (e == 1 && has[1]) {
            if (tid < 68) {
                row = tid < 34 ? 0 : 9;
                pc = tid < 34 ? tid : tid - 34;
            } else {
                const int h = tid - 68;
                row = 1 + (h >> 1);
                pc = (h & 1) ? 33 : 0;
            }
        }
        soff[e] = row * AX2_ROW + 2 * pc;
        int gi = (i0 - 2 + 2 * pc) % nx;   // even, so the pair (gi, gi + 1) is contiguous
        if (gi < 0) gi += nx;
        int gj = (j0 - 1 + row) % ny;
        if (gj < 0) gj += ny;
        goff[e] = gj * nx + gi;
    }
    float2 v[2][6];
    auto fetch = [&](int kk) {
        const int base = kk * plane;
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (has[e]) {
#pragma unroll
                for (int f = 0; f < 3; ++f) {
                    v[e][f] = ld2(u, f * N + base + goff[e]);
                    v[e][3 + f] = ld2(w, f * N + base + goff[e]);
                }
            }
    };
    auto commit = [&](int slot) {
        float* s = ax2s + slot * 6 * AX2_PL;
#pragma unroll
        for (int e = 0; e < 2; ++e)
            if (has[e]) {
#pragma unroll
                for (int f = 0; f < 6; ++f) *reinterpret_cast<float2*>(s + f * AX2_PL + soff[e]) = v[e][f];
            }
    };
    auto wz = [nz](int k) { return k < 0 ? k + nz : (k >= nz ? k - nz : k); };
    auto slot = [kb0](int q) { return (q - kb0 + 1) & 3; };
    fetch(wz(kb0 - 1));
    commit(slot(kb0 - 1));
    fetch(wz(kb0));
    commit(slot(kb0));
    fetch(wz(kb0 + 1));
    commit(slot(kb0 + 1));
    __syncthreads();
    const int r0 = (ty + 1) * AX2_ROW + 2 * tx + 2;   // the own pair in a staged plane
    const float2 nu2 = p2b(c.nu), two = p2b(2.f);
    double nup = 0.0;
    for (int k = kb0; k < ke; ++k) {
        const bool more = k + 1 < ke;
        if (more) fetch(wz(k + 2));
        if (ok) {
            const float* Pz[3] = {ax2s + slot(k - 1) * 6 * AX2_PL, ax2s + slot(k) * 6 * AX2_PL,
                                  ax2s + slot(k + 1) * 6 * AX2_PL};   // planes k-1, k, k+1
            // the finish's own-cell values first, so their loads overlap the stencil arithmetic
            const int J = k * plane + j * nx + i;
            float2 oldv[3], yv[3], xv[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                oldv[a] = ld2(uin, a * N + J);   // the accumulator's previous value (ubar0, or ybar first)
                yv[a] = ybar ? ld2(ybar, a * N + J) : oldv[a];
                xv[a] = extra ? ld2(extra, a * N + J) : make_float2(0.f, 0.f);
            }
            // the two cells' values of field f (0-2 u, 3-5 w) at offset (dx, dy, dz)
            auto at = [&](int f, int dx, int dy, int dz) -> float2 {
                const float* q = Pz[dz + 1] + f * AX2_PL + r0 + dy * AX2_ROW;
                if (dx == 0) return *reinterpret_cast<const float2*>(q);
                const float2 lo = *reinterpret_cast<const float2*>(dx > 0 ? q : q - 2);
                const float2 hi = *reinterpret_cast<const float2*>(dx > 0 ? q + 2 : q);
                return make_float2(lo.y, hi.x);
            };
            float2 lpart = make_float2(0.f, 0.f);   // u . diffusion(w) / nu over the three faces
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int ea[3] = {0, 0, 0};
                ea[a] = 1;
                const float2 ua0 = at(a, 0, 0, 0), uap = at(a, ea[0], ea[1], ea[2]),
                             uam = at(a, -ea[0], -ea[1], -ea[2]);
                const float2 wa0 = at(3 + a, 0, 0, 0), wap = at(3 + a, ea[0], ea[1], ea[2]),
                             wam = at(3 + a, -ea[0], -ea[1], -ea[2]);
                float2 acc = p2mul(p2b(c.c1[a]), p2fma(p2add(ua0, uap), p2sub(wap, wa0),
                                                       p2mul(p2add(uam, ua0), p2sub(wa0, wam))));
                float2 lap = p2mul(p2b(c.l2[a]), p2sub(p2add(wap, wam), p2mul(two, wa0)));
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if (b == a) continue;
                    int eb[3] = {0, 0, 0};
                    eb[b] = 1;
                    const float2 S0 = p2add(at(b, 0, 0, 0), at(b, ea[0], ea[1], ea[2]));
                    const float2 S1 = p2add(at(b, -eb[0], -eb[1], -eb[2]),
                                            at(b, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]));
                    const float2 wabp = at(3 + a, eb[0], eb[1], eb[2]), wabm = at(3 + a, -eb[0], -eb[1], -eb[2]);
                    const float2 wb0 = at(3 + b, 0, 0, 0), wbpa = at(3 + b, ea[0], ea[1], ea[2]);
                    const float2 wbm = at(3 + b, -eb[0], -eb[1], -eb[2]);
                    const float2 wbpam = at(3 + b, ea[0] - eb[0], ea[1] - eb[1], ea[2] - eb[2]);
                    acc = p2fma(p2b(c.c2[b]), p2fma(S0, p2sub(wabp, wa0), p2mul(S1, p2sub(wa0, wabm))), acc);
                    acc = p2fma(p2b(c.c2[a]), p2fma(S0, p2sub(wbpa, wb0), p2mul(S1, p2sub(wbpam, wbm))), acc);
                    lap = p2fma(p2b(c.l2[b]), p2sub(p2add(wabp, wabm), p2mul(two, wa0)), lap);
                }
                float2 ubs = p2fma(nu2, lap, acc);
                if (extra) ubs = p2add(ubs, xv[a]);
                lpart = p2fma(ua0, lap, lpart);
                const float2 nv = p2add(oldv[a], ubs);
                st2(ubar0, a * N + J, nv.x, nv.y);
                if (kb) {
                    const float2 kv = p2fma(dtb, yv[a], p2mul(dta, ubs));
                    st2(kb, a * N + J, kv.x, kv.y);
                }
            }
            nup += (double)lpart.x + (double)lpart.y;
        }
        // plane k + 2 into the slot of plane k - 2, which no thread reads after the previous barrier
        if (more) commit(slot(k + 2));
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) nup += __shfl_xor_sync(0xffffffffu, nup, o);
    __shared__ double red[8];
    if (tx == 0) red[ty] = nup;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int r = 0; r < 8; ++r) t += red[r];
        nu_part[((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
    }
}

}  // namespace ins
