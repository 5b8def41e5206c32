// 3x3x3 circular convolutions of the CNN closure on the 5th-generation tensor
// cores (tcgen05, kind::f16: BF16 operands, FP32 accumulation in TMEM).
//
// Implicit GEMM without an im2col buffer. One MMA tile = 128 output voxels (8 in x by 16 in y of
// one z plane) by N output channels. Input planes (with a one-voxel periodic halo) are staged in
// shared memory as 16-byte entries of 8 channels, a ring slot per plane laid out
// [channel group][y (18)][x (10)]. For tap (dx, dy) of a staged plane the A operand of the MMA is
// a shared-memory descriptor pointing at entry (1+dy, 1+dx) of the slot: its 8-row core matrices
// are 8 consecutive x voxels (16 B apart) and consecutive core matrices are consecutive y rows
// (SBO = one padded row, 160 B); the two core matrices of a K=16 step are two channel groups
// (LBO = one channel-group block). The B operand is a weight block [rows x K channels], K-major.
// D lives in TMEM; the epilogue reads it with tcgen05.ld (one voxel per thread).
//
// A CTA owns one 8 x 16 column of one z chunk and computes it in groups of four output planes
// z0 .. z0+3, which read input planes z0-1 .. z0+4. The weights of one (dx, dy) are stored as the
// N rows of dz = +1, 0, -1 stacked (3N rows), and output plane z0+o reads input plane z0+r with
// dz = r - o: one MMA of (number of outputs) x N columns applies a staged plane to every output
// plane of the group that reads it, writing adjacent N-column blocks of the group's accumulator
// (4N TMEM columns): 27 MMAs per output plane for 32 input channels instead of 54 with one plane
// per tile. Measured on this part: an MMA of 128 x N x 16 from one issuing thread takes about 58
// cycles for N <= 64 and 61 for N = 96, bound by its shared-memory operand reads (A is 4 KB per
// MMA whatever N), so wider MMAs do more work per operand byte. Three roles synchronise through
// mbarriers only:
//  * two loader warps stage the planes of the chunk into a 12-slot ring with cp.async (offsets
//    formed once per CTA) and publish each plane on its slot's barrier; a slot is refilled once the
//    MMAs of the last group that reads it have completed (a commit of that group arrives on the
//    slot's release barrier). The weights arrive by one bulk copy at the start;
//  * an MMA warp waits for the group's planes and for a free accumulator (two alternate), and one
//    lane issues the group's MMAs and commits them to the accumulator's barrier;
//  * eight epilogue warps wait for the accumulator, read its four planes with tcgen05.ld (two warps
//    per TMEM lane quarter split the channels), release it, and form and store the outputs.
// Every wait is bounded and reports through an error flag instead of hanging.
//
// The same kernel runs the backward data gradient (a convolution with the taps
// reversed and the channel roles swapped) with a different epilogue.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace ins {

constexpr int CV_TX = 8, CV_TY = 16;           // output tile: 8 x 16 voxels = 128 rows
constexpr int CV_PX = CV_TX + 2, CV_PY = CV_TY + 2;
constexpr int CV_ROW = CV_PX * 16;              // bytes per padded row of 16-byte entries
constexpr int CV_CGB = CV_PY * CV_ROW;          // bytes of one channel group of a staged plane
constexpr int CV_G = 4;                         // output planes per MMA group
constexpr int CV_LAG = 2;                       // plane copies in flight beyond the one published
constexpr int CV_SLOTS = 12;                    // plane ring (>= 10 + CV_LAG: see the loader warps)
constexpr int CV_EPI_WARPS = 8;                 // epilogue warps
constexpr int CV_LD_WARPS = 2;                  // plane-loader warps
constexpr int CV_THREADS = 32 * (CV_EPI_WARPS + CV_LD_WARPS + 1);   // + one MMA warp
constexpr long CV_SPIN = 1L << 24;              // bound on every mbarrier wait

enum ConvEpi {
    EPI_GELU = 0,      // y = bf16(gelu(acc + b)) channels-last; z = acc + b (FP32) if zout
    EPI_OUT = 1,       // out_T[c][v] = acc + b for c < nreal (the closure output m, SoA)
    EPI_DGELU = 2,     // y = bf16(acc * gelu'(zin)) channels-last (data gradient through GELU)
    EPI_ACCUM = 3      // out_T[c][v] += acc for c < nreal (data gradient of the input, SoA)
};

struct ConvArgs {
    const void* x;          // input activations, bf16 channels-last [vox][8 * cin_g]
    const void* wblob;      // packed weights (bf16), CV taps x N x (8 * kg) in the B layout
    const float* bias;      // [N] (EPI_GELU / EPI_OUT), may be null
    void* y;                // EPI_GELU / EPI_DGELU: bf16 channels-last [vox][N]
    float* zout;            // EPI_GELU: FP32 pre-activation [vox][N] or null
    const float* zin;       // EPI_DGELU: FP32 pre-activation of the layer below [vox][N]
    void* out;              // EPI_OUT / EPI_ACCUM: SoA field (float or double) [nreal][vox]
    int out_f64;            // out holds doubles
    int nreal;              // real output channels for EPI_OUT / EPI_ACCUM
    int nx, ny, nz;         // grid (periodic in all directions)
    int zchunk;
    unsigned int* err;      // bit 1: an mbarrier wait gave up
};

__device__ __forceinline__ uint32_t cv_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: no swizzle, K-major canonical layout.
__device__ __forceinline__ uint64_t cv_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ void cv_cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// erf(x) and exp(-x^2) by the rational approximation of Hastings as given by Abramowitz and Stegun,
// Handbook of Mathematical Functions, formula 7.1.26: for x >= 0,
//   erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2),  t = 1 / (1 + p x),
// with |error| <= 1.5e-7, extended to x < 0 by oddness. The exponential is shared with the GELU
// derivative. The error is far below the BF16 resolution (2^-8) of the activations written.
__device__ __forceinline__ float cv_erf(float x, float& ex2) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    float q = fmaf(1.061405429f, t, -1.453152027f);
    q = fmaf(q, t, 1.421413741f);
    q = fmaf(q, t, -0.284496736f);
    q = fmaf(q, t, 0.254829592f);
    ex2 = __expf(-ax * ax);
    return copysignf(fmaf(-q * t, ex2, 1.0f), x);
}
// GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2 and its derivative Phi(z) + z phi(z)
__device__ __forceinline__ float cv_gelu(float z) {
    float e;
    const float er = cv_erf(z * 0.70710678118654752440f, e);
    return 0.5f * z * (1.0f + er);
}
__device__ __forceinline__ float cv_gelu_grad(float z) {
    float e;   // exp(-z^2 / 2)
    const float er = cv_erf(z * 0.70710678118654752440f, e);
    return fmaf(z * 0.39894228040143267794f, e, 0.5f * (1.0f + er));
}

// Ring-slot layout of a staged plane: CG blocks of CV_CGB bytes, block cg holding [y (18)][x (10)]
// 16-byte entries of channels 8 cg .. 8 cg + 7 (the A operand's core matrices), with the periodic
// wrap in x and y applied. CvPlaneCopy holds the entries e = first + COUNT k (k < K) one thread
// copies of every plane, ordered [y][x][channel group] so that a warp's reads are contiguous, with
// their byte offsets within a z plane of the input (g) and within a slot (s): they are the same
// for every plane, so a plane costs one cp.async per entry.
template <int CG, int COUNT>
struct CvPlaneCopy {
    static constexpr int EPP = CG * CV_PY * CV_PX;    // entries per plane
    static constexpr int K = (EPP + COUNT - 1) / COUNT;
    uint32_t g[K], s[K];
    bool last;                                        // entry K-1 exists for this thread
    __device__ __forceinline__ CvPlaneCopy(int first, int x0, int y0, int nx, int ny) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int e = min(first + COUNT * k, EPP - 1);
            const int cg = e % CG;
            const int r = e / CG;
            const int yy = r / CV_PX, xx = r - yy * CV_PX;
            int gx = x0 - 1 + xx, gy = y0 - 1 + yy;
            gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
            gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
            g[k] = (uint32_t)((gy * nx + gx) * (CG * 16) + cg * 16);
            s[k] = (uint32_t)(cg * CV_CGB + yy * CV_ROW + xx * 16);
        }
        last = first + COUNT * (K - 1) < EPP;
    }
    // plane gz of x (bytes) into the slot at shared address dst, as one cp.async group
    __device__ __forceinline__ void load(const unsigned char* x, int gz, int nx, int ny, uint32_t dst) const {
        const unsigned char* src = x + (size_t)gz * nx * ny * (CG * 16);
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (k < K - 1 || last) cv_cp_async16(dst + s[k], src + g[k]);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
};

// CG: channel groups of 8 in the input (1 or 4); N: MMA N (16 or 32); KG: K channel groups in
// the weight blob (2 when CG == 1, the second group being zero; else CG).
template <int CG, int N, int EPI>
__global__ void __launch_bounds__(CV_THREADS, 1) k_conv3d_tc(ConvArgs a) {
    constexpr int KG = CG == 1 ? 2 : CG;
    constexpr int KSTEPS = KG / 2;                   // MMAs (K = 16) per tap
    constexpr int XYB = 3 * N * KG * 16;             // weight bytes per (dx, dy): rows dz = +1, 0, -1
    constexpr int SBO_B = KG * 128;                  // byte stride of 8-row groups in a weight block
    constexpr int NH = N / (CV_EPI_WARPS / 4);       // channels per epilogue warp
    constexpr int ACC = CV_G * N;                    // TMEM columns per accumulator (one group)
    constexpr uint32_t TCOLS = 2 * ACC < 32 ? 32 : 2 * ACC;
    extern __shared__ __align__(1024) unsigned char smem[];
    constexpr int SLOTB = CG * CV_CGB;               // bytes per ring slot
    unsigned char* sA = smem;                        // CV_SLOTS * SLOTB bytes
    unsigned char* sB = smem + CV_SLOTS * SLOTB;     // 9 * XYB bytes
    __shared__ __align__(8) uint64_t full[2];        // accumulator b holds a finished group (MMA commit)
    __shared__ __align__(8) uint64_t empty[2];       // the epilogue warps have read accumulator b
    __shared__ __align__(8) uint64_t pfull[CV_SLOTS];    // ring slot s holds its plane (loader warps)
    __shared__ __align__(8) uint64_t pempty[CV_SLOTS];   // the MMAs that read slot s's plane have completed
    __shared__ __align__(8) uint64_t wbar;               // the weights have landed (bulk copy)
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int x0 = blockIdx.x * CV_TX, y0 = blockIdx.y * CV_TY;
    const int zb = blockIdx.z * a.zchunk, ze = min(zb + a.zchunk, nz);
    const int ngroups = (ze - zb + CV_G - 1) / CV_G;
    const long nvox = (long)nx * ny * nz;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cv_smem(&tbase)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&full[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cv_smem(&empty[b])), "r"(CV_EPI_WARPS));
        }
        for (int q = 0; q < CV_SLOTS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cv_smem(&pfull[q])), "r"(CV_LD_WARPS));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&pempty[q])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&wbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // weights: 9 (dx, dy) blocks of 3N rows (dz = +1, 0, -1), one bulk copy (the blob is
        // 256-byte aligned and a multiple of 16 bytes long) completing on wbar
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cv_smem(&wbar)), "r"(9 * XYB)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                cv_smem(sB)),
            "l"(a.wblob), "r"(9 * XYB), "r"(cv_smem(&wbar))
            : "memory");
    }
    // plane p (p >= zb - 1) has ring index i = p - zb + 1 and sits in slot i % CV_SLOTS
    auto slot_of = [zb](int p) { return (p - zb + 1) % CV_SLOTS; };
    auto wrapz = [nz](int z) { return ((z % nz) + nz) % nz; };
    // Launched as a programmatic dependent of the previous kernel in the stream: the set-up above
    // (barriers, TMEM, the weights, which no kernel of the closure writes) overlaps that kernel's
    // tail; everything below reads or writes activations, so it waits for the previous grid to
    // have completed and flushed. Dependents of this grid may be scheduled at once: they wait the
    // same way before touching its outputs.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // prologue: the first group's planes (ring indices 0 .. 5), by every thread
    const unsigned char* xin = reinterpret_cast<const unsigned char*>(a.x);
    {
        const CvPlaneCopy<CG, CV_THREADS> pc(tid, x0, y0, nx, ny);
        for (int i = 0; i < CV_G + 2; ++i) pc.load(xin, wrapz(zb - 1 + i), nx, ny, cv_smem(sA + i * SLOTB));
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    // instruction descriptors for MMAs of N, 2N and 3N columns (BF16 x BF16 -> FP32, M = 128)
    auto idesc_n = [](int n) {
        return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((128u >> 4) << 24);
    };
    const uint64_t adesc0 = cv_desc(cv_smem(sA), CG == 1 ? 0 : CV_CGB, CV_ROW);
    const uint64_t bdesc0 = cv_desc(cv_smem(sB), 128, SBO_B);
    // a descriptor = base descriptor + operand byte offset / 16 in the start-address field (bits
    // 0..13): shared addresses stay below 256 KB, so the sum never carries out of the field and
    // only the low word changes (one 32-bit add per operand)
    auto desc_at = [](uint64_t base, uint32_t off16) {
        uint64_t d;
        asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "r"((uint32_t)base + off16), "r"((uint32_t)(base >> 32)));
        return d;
    };
    // MMAs of the group of output planes z0 .. z0+3 into accumulator acc (one thread). Input plane
    // z0 + r (r = -1 .. 4) contributes to outputs o = max(0, r-1) .. min(3, r+1) with dz = r - o; their
    // weight rows (dz = +1, 0, -1 stacked) are contiguous, so one MMA of N (o_last - o_first + 1)
    // columns covers them, into columns N o_first of the accumulator. r = 1 (outputs 0..2) and r = 4
    // (output 3) go first: their first MMAs overwrite every column, all later ones accumulate.
    auto issue_group = [&](int z0, int acc) {
        const uint32_t dbase = tmem + (uint32_t)(acc * ACC);
        const int rorder[6] = {1, 4, -1, 0, 2, 3};
#pragma unroll
        for (int ri = 0; ri < 6; ++ri) {
            const int r = rorder[ri];
            const int of = r - 1 > 0 ? r - 1 : 0, ol = r + 1 < CV_G - 1 ? r + 1 : CV_G - 1;
            const uint32_t idesc = idesc_n(N * (ol - of + 1));
            const uint32_t ap = (uint32_t)((slot_of(z0 + r) * SLOTB) >> 4);
            const uint32_t dcol = dbase + (uint32_t)(N * of);
            const int rowb = N * (1 - r + of);   // first weight row of the block
#pragma unroll
            for (int xy = 0; xy < 9; ++xy) {
                const int dy = xy / 3 - 1, dx = xy % 3 - 1;
#pragma unroll
                for (int s = 0; s < KSTEPS; ++s) {
                    const uint64_t ad =
                        desc_at(adesc0, ap + (uint32_t)(((1 + dy) * CV_ROW + (1 + dx) * 16 + 2 * s * CV_CGB) >> 4));
                    const uint64_t bd = desc_at(bdesc0, (uint32_t)((xy * XYB + (rowb / 8) * SBO_B + 2 * s * 128) >> 4));
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(idesc), "r"((ri >= 2 || xy > 0 || s > 0) ? 1u : 0u));
                }
            }
        }
    };
    // planes z0-1 .. z0+2 are not read by later groups: their slots are free once the group's MMAs
    // complete. The accumulator's commit goes last, so its completion implies the others'.
    auto commit_group = [&](int z0, int acc) {
#pragma unroll
        for (int p = -1; p <= 2; ++p)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             cv_smem(&pempty[slot_of(z0 + p)]))
                         : "memory");
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         cv_smem(&full[acc]))
                     : "memory");
    };
    // bounded wait for the completion of the phase of parity `par` (false: gave up)
    auto wait_par = [](uint64_t* bar, uint32_t par) {
        uint32_t done = 0;
        for (long it = 0; it < CV_SPIN && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(cv_smem(bar)), "r"(par)
                : "memory");
        }
        return done != 0;
    };
    const int plast = zb + CV_G * ngroups;   // the last plane any group reads
    const int nplanes = plast - zb + 2;        // ring indices 0 .. plast - zb + 1
    if (warp >= CV_EPI_WARPS && warp < CV_EPI_WARPS + CV_LD_WARPS) {
        // ---- loader warps: planes 6, 7, ... (ring index i) in order, each warp a fixed share of
        // every plane's entries, CV_LAG + 1 planes in flight. Plane i goes into the slot of plane
        // i - CV_SLOTS, free once the group whose MMAs read that plane last has completed (pempty).
        // A warp's share of a plane counts on the plane's barrier (pfull, one arrival per loader
        // warp) once its copies have landed and been fenced for the tensor cores' (async-proxy)
        // reads. A warp waits for the slot of plane i before it publishes planes i - CV_LAG .. i - 1;
        // with 10 + CV_LAG or more slots none of those is read before the group after the one that
        // frees the slot, so the MMA warp always has a complete group queued while the loaders wait.
        const int lw = warp - CV_EPI_WARPS;
        const CvPlaneCopy<CG, 32 * CV_LD_WARPS> pc(lw * 32 + lane, x0, y0, nx, ny);
        bool alive = true;
        for (int i = CV_G + 2; i < nplanes + CV_LAG && alive; ++i) {
            if (i < nplanes) {
                const int slot = i % CV_SLOTS;
                if (i >= CV_SLOTS) {
                    alive = __all_sync(0xffffffffu,
                                       wait_par(&pempty[slot], (uint32_t)(((i - CV_SLOTS) / CV_SLOTS) & 1)));
                    if (!alive) break;
                }
                pc.load(xin, wrapz(zb - 1 + i), nx, ny, cv_smem(sA + slot * SLOTB));
            } else {
                asm volatile("cp.async.commit_group;" ::: "memory");   // empty group: keeps the count
            }
            asm volatile("cp.async.wait_group %0;" ::"n"(CV_LAG) : "memory");   // plane i - CV_LAG has landed
            const int q = i - CV_LAG;
            if (q >= CV_G + 2) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0)
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cv_smem(&pfull[q % CV_SLOTS]))
                                 : "memory");
            }
        }
        if (!alive && lane == 0) atomicOr(a.err, 2u);
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == CV_EPI_WARPS + CV_LD_WARPS) {
        // ---- MMA warp: group g needs accumulator g & 1 free (group g-2 read out) and its new planes
        // z0+1 .. z0+4 published (ring indices 4g+2 .. 4g+5; those of group 0 come from the
        // prologue; planes z0-1, z0 were waited for by group g-1). The loaders publish ring indices
        // 6, 7, ..., so plane i is the ((i - 6) / CV_SLOTS)-th published in its slot. Lane 0 issues
        // the group's MMAs.
        bool alive = __all_sync(0xffffffffu, wait_par(&wbar, 0u));
        for (int g = 0; g < ngroups && alive; ++g) {
            const int z0 = zb + CV_G * g, b = g & 1, u = g >> 1;
            bool ok = true;
            if (g >= 2) ok = wait_par(&empty[b], (uint32_t)((u - 1) & 1));
            for (int i = CV_G * g + 2; g > 0 && ok && i <= CV_G * g + CV_G + 1; ++i)
                ok = wait_par(&pfull[i % CV_SLOTS], (uint32_t)(((i - CV_G - 2) / CV_SLOTS) & 1));
            alive = __all_sync(0xffffffffu, ok);
            if (!alive) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (lane == 0) {
                issue_group(z0, b);
                commit_group(z0, b);
            }
            __syncwarp();
        }
        // no MMA may still write TMEM when it is freed: wait for the last group issued
        if (alive && ngroups > 0) alive = wait_par(&full[(ngroups - 1) & 1], (uint32_t)(((ngroups - 1) >> 1) & 1));
        if (!alive && lane == 0) atomicOr(a.err, 2u);
    } else {
        // ---- epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (voxel rows) and channels
        // (w / 4) NH .. +NH of each output plane of a group, releases the accumulator, then forms and
        // stores the outputs
        const int q4 = warp & 3, part = warp >> 2;
        const int m = q4 * 32 + lane;
        const int vx = x0 + (m & 7), vy = y0 + (m >> 3);
        const bool inside = vx < nx && vy < ny;
        const int c0 = part * NH;
        float bv[NH];
#pragma unroll
        for (int c = 0; c < NH; ++c) bv[c] = (a.bias && (EPI == EPI_GELU || EPI == EPI_OUT)) ? a.bias[c0 + c] : 0.f;
        for (int g = 0; g < ngroups; ++g) {
            const int z0 = zb + CV_G * g, b = g & 1, u = g >> 1;
            if (!__all_sync(0xffffffffu, wait_par(&full[b], (uint32_t)(u & 1)))) {
                if (lane == 0) atomicOr(a.err, 2u);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t rr[CV_G][NH];
#pragma unroll
            for (int o = 0; o < CV_G; ++o) {
                const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * ACC + o * N + c0);
                uint32_t* r = rr[o];
                if constexpr (NH == 16) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                          "=r"(r[15])
                        : "r"(taddr));
                } else if constexpr (NH == 4) {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                                 : "r"(taddr));
                } else {
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                                   "=r"(r[7])
                                 : "r"(taddr));
                }
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            // release the accumulator to the MMA warp (its next MMAs into it follow these reads)
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(cv_smem(&empty[b])) : "memory");
            // one copy of the per-plane code (instruction cache): plane o is always rr[0], and the
            // planes move down one register block after each
#pragma unroll 1
            for (int o = 0; o < CV_G; ++o) {
                const int z = z0 + o;
                if (z >= ze) break;
                if (o > 0) {
#pragma unroll
                    for (int q = 0; q + 1 < CV_G; ++q)
#pragma unroll
                        for (int c = 0; c < NH; ++c) rr[q][c] = rr[q + 1][c];
                }
                const uint32_t* r = rr[0];
                // epilogue: D row m -> voxel (vx, vy, z), channels c0 .. c0 + NH
                if (inside) {
                    const long v = ((long)z * ny + vy) * nx + vx;
                    if (EPI == EPI_GELU) {
                        __align__(16) __nv_bfloat16 ob[NH];
                        __align__(16) float zz[NH];
#pragma unroll
                        for (int c = 0; c < NH; ++c) {
                            zz[c] = __uint_as_float(r[c]) + bv[c];
                            ob[c] = __float2bfloat16_rn(cv_gelu(zz[c]));
                        }
                        if (a.zout) {
                            float4* zd = reinterpret_cast<float4*>(a.zout + v * N + c0);
#pragma unroll
                            for (int q = 0; q < NH / 4; ++q) zd[q] = reinterpret_cast<const float4*>(zz)[q];
                        }
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.y) + v * N + c0);
#pragma unroll
                        for (int q = 0; q < NH / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(ob)[q];
                    } else if (EPI == EPI_DGELU) {
                        __align__(16) float zi[NH];
                        const float4* zs = reinterpret_cast<const float4*>(a.zin + v * N + c0);
#pragma unroll
                        for (int q = 0; q < NH / 4; ++q) reinterpret_cast<float4*>(zi)[q] = zs[q];
                        __align__(16) __nv_bfloat16 ob[NH];
#pragma unroll
                        for (int c = 0; c < NH; ++c) ob[c] = __float2bfloat16_rn(__uint_as_float(r[c]) * cv_gelu_grad(zi[c]));
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.y) + v * N + c0);
#pragma unroll
                        for (int q = 0; q < NH / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(ob)[q];
                    } else {
#pragma unroll
                        for (int cc = 0; cc < NH; ++cc) {
                            const int c = c0 + cc;
                            if (c >= a.nreal) continue;
                            float val = __uint_as_float(r[cc]);
                            if (EPI == EPI_OUT) val += bv[cc];
                            if (a.out_f64) {
                                double* od = reinterpret_cast<double*>(a.out) + c * nvox + v;
                                *od = EPI == EPI_ACCUM ? *od + (double)val : (double)val;
                            } else {
                                float* of = reinterpret_cast<float*>(a.out) + c * nvox + v;
                                *of = EPI == EPI_ACCUM ? *of + val : val;
                            }
                        }
                    }
                }
            }
        }
    }
    // the weight copy has landed before the CTA leaves, even on a path that gave up
    if (tid == 0) wait_par(&wbar, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
}

// Pack weights W[27][cin][cout] (FP32 master copy) into the B layout of k_conv3d_tc as BF16:
// 9 (dx, dy) blocks of 3N rows, the N rows of dz = +1, 0, -1 stacked.
// forward: row n = co, channel k = ci, tap t; data gradient: row n = ci, channel k = co, tap 26 - t.
static __global__ void k_pack_weights(const float* __restrict__ W, int cin, int cout, int N, int KG, int transpose,
                               __nv_bfloat16* __restrict__ blob) {
    const int K = 8 * KG;
    const int total = 27 * N * K;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int t = e / (N * K);
        const int rem = e - t * N * K;
        const int n = rem / K, k = rem - n * K;
        float v = 0.f;
        if (!transpose) {
            if (n < cout && k < cin) v = W[((long)t * cin + k) * cout + n];
        } else {
            if (n < cin && k < cout) v = W[((long)(26 - t) * cin + n) * cout + k];
        }
        // the taps of one (dx, dy) are stacked as rows dz = +1, 0, -1 (3N rows, t = 9 (dz + 1) + xy)
        const int xy = t % 9, ns = (2 - t / 9) * N + n;
        const long off = (long)xy * 3 * N * K + (ns / 8) * (KG * 64) + (k / 8) * 64 + (ns % 8) * 8 + (k % 8);
        blob[off] = __float2bfloat16_rn(v);
    }
}

// Velocity (SoA, float or double) -> BF16 channels-last with 8 channels (3 used, 5 zero).
template <typename T>
__global__ void k_pack_input(const T* __restrict__ u, long nvox, __nv_bfloat16* __restrict__ x) {
    for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nvox; v += (long)gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16_rn(c < 3 ? (float)u[c * nvox + v] : 0.f);
        reinterpret_cast<uint4*>(x)[v] = *reinterpret_cast<const uint4*>(o);
    }
}

// ---------------------------------------------------------------------------------------
// Weight and bias gradients on the tensor cores:
//   dW[t][ci][co] = sum_v x[v + off_t][ci] gq[v][co],   db[co] = sum_v gq[v][co]
// (gq = BF16 gradient of the layer's pre-activation, x = BF16 layer input, both channels-last).
// GEMM with M = (tap, ci) (128 / CX taps per CTA), N = co, K = voxels. Channels-last rows hold
// M (resp. N) contiguously for each voxel, so both operands are read MN-major: the canonical
// no-swizzle MN-major layout has core matrices of 8 K-rows of 16 bytes (8 consecutive M or N
// values); LBO = stride between core matrices along K, SBO = along M / N (checked on the
// device against a host product). Per stage, 64 voxels of A (16 M-groups of 1 KB) and B are
// staged with 16-byte cp.async gathers (tap shift with periodic wrap) into a 4-stage ring,
// two stages ahead of the MMAs (a buffer is refilled once the MMAs that read it two stages
// earlier have committed); one thread issues the 4 MMAs (K = 16 each) of a stage into the
// TMEM accumulator. A CTA reduces
// its voxel range and adds its 128 x N block to dW with atomics; CTAs of the first tap group
// also sum gq for db. Zero-filled taps >= 27, voxels >= nvox and padding channels.
constexpr int WG_S = 64;                   // voxels per stage
constexpr int WG_NS = 4;                   // stages in the ring
constexpr int WG_PD = 2;                   // stages loaded ahead of the MMAs
constexpr int WG_THREADS = 256;

template <int N>
struct WgShape {
    static constexpr int KGRP = WG_S / 8;                     // K groups (8 voxels) per stage
    static constexpr int A_BYTES = 16 * KGRP * 128;          // 16 M-groups x KGRP x 128 B
    static constexpr int B_BYTES = (N / 8) * KGRP * 128;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int SMEM = WG_NS * STAGE;
};

template <int CX, int CY>
__global__ void __launch_bounds__(WG_THREADS) k_wgrad_tc(const __nv_bfloat16* __restrict__ X,
                                                         const __nv_bfloat16* __restrict__ dY, int nx, int ny, int nz,
                                                         int cin, int cout, long vchunk, float* __restrict__ dW,
                                                         float* __restrict__ db, unsigned int* __restrict__ err) {
    constexpr int N = CY < 16 ? 16 : CY;
    constexpr int TAPS = 128 / CX;         // taps per CTA (M = TAPS * CX = 128)
    constexpr int CGX = CX / 8;            // 16-byte channel groups per input voxel
    constexpr int TPV = WG_THREADS / WG_S; // threads per staged voxel
    using Sh = WgShape<N>;
    constexpr int MSTR = Sh::KGRP * 128;   // byte stride between M (or N) groups
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[WG_NS];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long nvox = (long)nx * ny * nz;
    const int tg = blockIdx.x;             // tap group
    const long v0 = (long)blockIdx.y * vchunk;
    const long v1 = v0 + vchunk < nvox ? v0 + vchunk : nvox;
    const int nst = v1 > v0 ? (int)((v1 - v0 + WG_S - 1) / WG_S) : 0;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cv_smem(&tbase)), "r"(32));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0)
        for (int q = 0; q < WG_NS; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&mbar[q])));
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
                           ((128u >> 4) << 24);
    // staging: thread t handles voxel k = t % WG_S of the stage and every TPV-th M-group / N-group;
    // its M-groups' tap offsets are fixed, the voxel coordinates are 32-bit (grids hold < 2^31 voxels)
    const int kk = tid % WG_S, part = tid / WG_S;
    constexpr int MPT = 16 / TPV;          // M-groups per thread
    int tdx[MPT], tdy[MPT], tdz[MPT], tcg[MPT];
    bool tok[MPT];
#pragma unroll
    for (int j = 0; j < MPT; ++j) {
        const int mg = part + TPV * j;
        const int tl = mg / CGX;
        const int t = tg * TAPS + tl;
        tok[j] = t < 27;
        tdz[j] = t / 9 - 1;
        tdy[j] = (t / 3) % 3 - 1;
        tdx[j] = t % 3 - 1;
        tcg[j] = mg - tl * CGX;
    }
    const int nxy = nx * ny;
    // coordinates of this thread's voxel of the next stage to issue: stages are issued in
    // order, each WG_S voxels after the previous one, so the coordinates advance without divisions
    int cvx, cvy, cvz;
    {
        const long vl = v0 + kk;
        const int v = vl < nvox ? (int)vl : 0;
        cvz = v / nxy;
        const int rxy = v - cvz * nxy;
        cvy = rxy / nx;
        cvx = rxy - cvy * nx;
    }
    auto issue = [&](int st, int b) {
        unsigned char* sa = smem + b * Sh::STAGE;
        unsigned char* sbb = sa + Sh::A_BYTES;
        const long vl = v0 + (long)st * WG_S + kk;
        const bool okv = vl < v1;
        const int x = cvx, y = cvy, z = cvz;
        const int v = okv ? (z * ny + y) * nx + x : 0;
        cvx += WG_S;
        while (cvx >= nx) {
            cvx -= nx;
            if (++cvy == ny) {
                cvy = 0;
                ++cvz;
            }
        }
        const uint32_t kofs = (uint32_t)((kk >> 3) * 128 + (kk & 7) * 16);
#pragma unroll
        for (int j = 0; j < MPT; ++j) {
            const int mg = part + TPV * j;
            const bool ok = okv && tok[j];
            const unsigned char* src = reinterpret_cast<const unsigned char*>(X);
            if (ok) {
                int xs = x + tdx[j], ys = y + tdy[j], zs = z + tdz[j];
                xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
                ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
                zs = zs < 0 ? zs + nz : (zs >= nz ? zs - nz : zs);
                const int vs = zs * nxy + ys * nx + xs;
                src += ((size_t)vs * CX + tcg[j] * 8) * 2;
            }
            const uint32_t dst = cv_smem(sa) + (uint32_t)mg * MSTR + kofs;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
        }
        for (int ng = part; ng < N / 8; ng += TPV) {
            const bool ok = okv && ng < CY / 8;
            const unsigned char* src = reinterpret_cast<const unsigned char*>(dY);
            if (ok) src += ((size_t)v * CY + ng * 8) * 2;
            const uint32_t dst = cv_smem(sbb) + (uint32_t)ng * MSTR + kofs;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto wait_mbar = [&](int b, uint32_t parity) -> bool {
        uint32_t done = 0;
        for (long it = 0; it < CV_SPIN && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(cv_smem(&mbar[b])), "r"(parity)
                : "memory");
        }
        return done != 0;
    };
    uint32_t uses[WG_NS];                  // commits issued on each buffer's barrier
#pragma unroll
    for (int q = 0; q < WG_NS; ++q) uses[q] = 0u;
    bool alive = true;
    float bsum = 0.f;                      // db partial (first tap group; thread n < CY sums column n)
    for (int q = 0; q < WG_PD; ++q) {      // prologue: stages 0 .. PD - 1, one commit group each
        if (q < nst) issue(q, q);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < nst && alive; ++i) {
        const int b = i % WG_NS;
        const int nxt = i + WG_PD;
        if (nxt < nst) {
            // buffer of stage i - 2: its MMAs were issued two iterations ago, its db sums are
            // behind two barriers
            const int nb = nxt % WG_NS;
            if (uses[nb] > 0 && !wait_mbar(nb, (uses[nb] - 1) & 1)) {
                if (tid == 0) atomicOr(err, 2u);
                alive = false;
            }
            issue(nxt, nb);
        } else {
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(WG_PD) : "memory");   // stage i has landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (__syncthreads_or(!alive)) break;
        const unsigned char* sa = smem + b * Sh::STAGE;
        if (tg == 0 && tid < CY) {
            const unsigned char* sbb = sa + Sh::A_BYTES;
            const int ng = tid >> 3, w = tid & 7;
            for (int k = 0; k < WG_S; ++k) {
                const __nv_bfloat16 h =
                    *reinterpret_cast<const __nv_bfloat16*>(sbb + ng * MSTR + (k >> 3) * 128 + (k & 7) * 16 + w * 2);
                bsum += __bfloat162float(h);
            }
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t abase = cv_smem(sa), bbase = abase + Sh::A_BYTES;
#pragma unroll
            for (int s2 = 0; s2 < WG_S / 16; ++s2) {
                const uint64_t ad = cv_desc(abase + s2 * 256, 128, MSTR);
                const uint64_t bd = cv_desc(bbase + s2 * 256, 128, MSTR);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"((i > 0 || s2 > 0) ? 1 : 0));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             cv_smem(&mbar[b]))
                         : "memory");
        }
        ++uses[b];
    }
    // the last stage's MMAs, then the accumulator block
    if (alive && nst > 0) {
        const int b = (nst - 1) % WG_NS;
        if (!wait_mbar(b, (uses[b] - 1) & 1)) {
            if (tid == 0) atomicOr(err, 2u);
            alive = false;
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(!alive)) alive = false;
    if (alive && nst > 0 && warp < 4) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        if (N == 32) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
        } else {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int m = warp * 32 + lane;
        const int tl = m / CX, ci = m - tl * CX;
        const int t = tg * TAPS + tl;
        if (t < 27 && ci < cin) {
            for (int co = 0; co < cout; ++co) atomicAdd(&dW[((long)t * cin + ci) * cout + co], __uint_as_float(r[co]));
        }
    }
    if (alive && tg == 0 && tid < cout && db) atomicAdd(&db[tid], bsum);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32));
}

// Weight and bias gradients of a layer with 32 input channels without gathers:
//   dW[t][ci][co] = sum_v x[v + tap t][ci] dY[v][co],  db[co] = sum_v dY[v][co].
// A CTA owns a 16 x 8 column of voxels (x, y) and a chunk of z planes. Input planes are
// staged once, with a one-voxel halo in x and rows y0 - 1 .. y0 + 9, as 16-byte entries of
// 8 channels laid out [row][channel group][x]; inside a row the four channel groups are
// 288 bytes apart and consecutive rows 4 x 288 bytes apart, so the 16 M groups (channel
// group, dy) of one MMA (M = 128 rows = (dy = -1 .. +2) x 32 channels) sit at one constant
// stride: the tap shift in y is part of the A descriptor's M stride, the shifts in x and z
// are its start address. Both operands are MN-major (8 voxels x 16 bytes per core matrix;
// K = 16 voxels = one row of the tile). Per plane: 9 (dx, dz) accumulators x 8 rows = 72
// MMAs of 128 x N x 16 into TMEM regions (dx, dz) that persist over the CTA's planes; the
// rows dy = +2 are computed and discarded. The dY plane of the tile is staged [row][group][x]
// (zero-filled beyond the real channels). At the end each CTA writes its accumulators as one
// partial block part[cta][27][32][N] (k_wgrad_reduce sums the blocks into dW; an error leaves
// the block unwritten and sets the flag).
// Input planes z - 1 .. z + 1 come from a 5-slot ring, dY from a 3-slot ring; plane slots
// are reused only after the MMAs of the tile two planes back have completed (one commit
// group per tile on alternating mbarriers, bounded waits with an error flag).
constexpr int WP_TX = 16, WP_TY = 8;
constexpr int WP_XE = WP_TX + 2;                 // x entries of a staged row
constexpr int WP_ROWS = WP_TY + 3;               // rows y0 - 1 .. y0 + 9
constexpr int WP_CGS = WP_XE * 16;               // channel-group stride in a row (288 B)
constexpr int WP_ROWB = 4 * WP_CGS;              // row stride (1152 B)
constexpr int WP_XPLANE = WP_ROWS * WP_ROWB;     // 12672 B
constexpr int WP_XSLOTS = 5, WP_DSLOTS = 3;
template <int N>
struct WpShape {
    static constexpr int DROW = (N / 8) * 256;   // dY row: N/8 groups x 16 x-entries
    static constexpr int DPLANE = WP_TY * DROW;
    static constexpr int SMEM = WP_XSLOTS * WP_XPLANE + WP_DSLOTS * DPLANE;
    static constexpr uint32_t TCOLS = 9 * N <= 256 ? 256 : 512;
};

template <int CY>
__global__ void __launch_bounds__(256, 1) k_wgrad_plane(const __nv_bfloat16* __restrict__ X,
                                                        const __nv_bfloat16* __restrict__ dY, int nx, int ny, int nz,
                                                        int cout, int zchunk, float* __restrict__ part,
                                                        float* __restrict__ db, unsigned int* __restrict__ err) {
    constexpr int N = CY < 16 ? 16 : CY;
    using Sh = WpShape<N>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* const sx = smem;
    unsigned char* const sd = smem + WP_XSLOTS * WP_XPLANE;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * WP_TX, y0 = blockIdx.y * WP_TY;
    const int zb = blockIdx.z * zchunk, ze = min(zb + zchunk, nz);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(cv_smem(&tbase)),
                     "r"(Sh::TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cv_smem(&mbar[1])));
    }
    auto wrapz = [nz](int z) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); };
    auto xslot = [zb](int z) { return (z - zb + 1) % WP_XSLOTS; };   // z >= zb - 1
    auto dslot = [zb](int z) { return (z - zb) % WP_DSLOTS; };       // z >= zb
    // staging of input plane z: 11 rows x 4 groups x 18 entries
    auto load_x = [&](int z) {
        const unsigned char* xb = reinterpret_cast<const unsigned char*>(X);
        const int gz = wrapz(z);
        unsigned char* dst = sx + xslot(z) * WP_XPLANE;
        for (int e = tid; e < WP_ROWS * 4 * WP_XE; e += 256) {
            const int row = e / (4 * WP_XE), r2 = e - row * (4 * WP_XE);
            const int cg = r2 / WP_XE, xe = r2 - cg * WP_XE;
            int gx = x0 - 1 + xe, gy = y0 - 1 + row;
            gx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
            gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
            const long vox = ((long)gz * ny + gy) * nx + gx;
            cv_cp_async16(cv_smem(dst + row * WP_ROWB + cg * WP_CGS + xe * 16), xb + vox * 64 + cg * 16);
        }
    };
    // staging of dY plane z: 8 rows x N/8 groups x 16 entries (groups beyond CY zero-filled)
    auto load_d = [&](int z) {
        const unsigned char* db8 = reinterpret_cast<const unsigned char*>(dY);
        unsigned char* dst = sd + dslot(z) * Sh::DPLANE;
        for (int e = tid; e < WP_TY * (N / 8) * WP_TX; e += 256) {
            const int row = e / ((N / 8) * WP_TX), r2 = e - row * ((N / 8) * WP_TX);
            const int ng = r2 / WP_TX, xe = r2 - ng * WP_TX;
            const long vox = ((long)z * ny + (y0 + row)) * nx + (x0 + xe);
            const bool ok = ng < CY / 8;
            const unsigned sa = cv_smem(dst + row * Sh::DROW + ng * 256 + xe * 16);
            const void* src = ok ? (const void*)(db8 + (vox * CY + ng * 8) * 2) : (const void*)db8;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(src), "r"(ok ? 16 : 0) : "memory");
        }
    };
    for (int z = zb - 1; z <= zb + 1 && z <= ze; ++z) load_x(z);
    if (zb < ze) load_d(zb);
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tbase;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
                           ((128u >> 4) << 24);
    // descriptors: base + (byte offset / 16) in the address field (shared addresses < 256 KB)
    const uint64_t adesc0 = cv_desc(cv_smem(sx), 128, WP_CGS);
    const uint64_t bdesc0 = cv_desc(cv_smem(sd), 128, 256);
    auto issue_tile = [&](int z, bool first) {
        const uint64_t as[3] = {adesc0 + (uint64_t)((xslot(z - 1) * WP_XPLANE) >> 4),
                                adesc0 + (uint64_t)((xslot(z) * WP_XPLANE) >> 4),
                                adesc0 + (uint64_t)((xslot(z + 1) * WP_XPLANE) >> 4)};
        const uint64_t bs = bdesc0 + (uint64_t)((dslot(z) * Sh::DPLANE) >> 4);
#pragma unroll
        for (int dz = 0; dz < 3; ++dz)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint32_t dcol = tmem + (uint32_t)((dz * 3 + dx) * N);
#pragma unroll
                for (int r = 0; r < WP_TY; ++r) {
                    const uint64_t ad = as[dz] + (uint64_t)((r * WP_ROWB + dx * 16) >> 4);
                    const uint64_t bd = bs + (uint64_t)((r * Sh::DROW) >> 4);
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(idesc), "r"((first && r == 0) ? 0 : 1));
                }
            }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         cv_smem(&mbar[(z - zb) & 1]))
                     : "memory");
    };
    auto wait_tile = [&](int t) -> bool {   // the MMAs of tile t (t >= zb) have completed
        const uint32_t parity = (uint32_t)(((t - zb) >> 1) & 1);
        uint32_t done = 0;
        for (long it = 0; it < CV_SPIN && !done; ++it) {
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(cv_smem(&mbar[(t - zb) & 1])), "r"(parity)
                : "memory");
        }
        return done != 0;
    };
    bool alive = true;
    // db partials: the dY tile of a plane is 8 rows x N/8 groups x 16 voxels of 16-byte entries;
    // thread t sums entries t, t + 256, ..., all of channel group (t / 16) % (N / 8), into 8
    // channel sums (16-byte shared loads, every warp an equal share)
    float bsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    constexpr int DB_ENT = WP_TY * (N / 8) * WP_TX;   // 512 or 256
    const int dbg = (tid >> 4) % (N / 8);
    for (int z = zb; z < ze; ++z) {
        // slots of plane z + 2 (input) and z + 1 (dY) were last read by tile z - 2
        if (z - 2 >= zb && !wait_tile(z - 2)) alive = false;
        if (z + 1 < ze) {
            load_x(z + 2);
            load_d(z + 1);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");   // plane z + 1 and dY z have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!alive)) {
            alive = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) issue_tile(z, z == zb);
        if (db && dbg < CY / 8) {
            const unsigned char* p = sd + dslot(z) * Sh::DPLANE;
#pragma unroll
            for (int e = tid; e < DB_ENT; e += 256) {
                const int row = e / ((N / 8) * WP_TX), r2 = e - row * ((N / 8) * WP_TX);
                const int xe = r2 - (r2 / WP_TX) * WP_TX;
                const uint4 q = *reinterpret_cast<const uint4*>(p + row * Sh::DROW + dbg * 256 + xe * 16);
                const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
                for (int c2 = 0; c2 < 4; ++c2) {
                    const float2 f = __bfloat1622float2(h[c2]);
                    bsum[2 * c2] += f.x;
                    bsum[2 * c2 + 1] += f.y;
                }
            }
        }
    }
    // the last two tiles
    if (alive) {
        for (int t = ze - 2 < zb ? zb : ze - 2; t < ze; ++t)
            if (!wait_tile(t)) alive = false;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(!alive)) alive = false;
    if (!alive && tid == 0) atomicOr(err, 2u);
    if (alive && zb < ze) {
        const long cta = ((long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 of regions (w / 4) * 5 .. : 0..4 and 5..8
        const int m = (warp & 3) * 32 + lane;
        const int g = m >> 3, ci = (g & 3) * 8 + (m & 7), dyi = g >> 2;
        const int rb = (warp >> 2) * 5, re = (warp >> 2) ? 9 : 5;
        for (int reg = rb; reg < re; ++reg) {
            uint32_t r[N];
            const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(reg * N);
            if constexpr (N == 32) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
            } else {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr));
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (dyi < 3) {
                const int dz = reg / 3, dx = reg - dz * 3;
                const int t = dz * 9 + dyi * 3 + dx;
                float4* dst = reinterpret_cast<float4*>(part + (cta * 27L * 32 + (long)t * 32 + ci) * N);
#pragma unroll
                for (int q = 0; q < N / 4; ++q)
                    dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            }
        }
        if (db) {
            // lanes 0..15 and 16..31 of a warp share a channel group
#pragma unroll
            for (int c = 0; c < 8; ++c)
                for (int o = 8; o > 0; o >>= 1) bsum[c] += __shfl_xor_sync(0xffffffffu, bsum[c], o);
            if ((lane & 15) == 0 && dbg < CY / 8) {
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (dbg * 8 + c < cout) atomicAdd(&db[dbg * 8 + c], bsum[c]);
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::TCOLS));
}

// dW[t][ci][co] += sum over the CTAs' partial blocks part[c][t][ci][0..N) (co < cout). A block of
// 256 threads takes 32 consecutive weights (one per lane); warp w sums the blocks c = w, w + 8, ...
// in order and the eight warp sums are added in warp order: a fixed summation order, with eight
// times the loads in flight of one thread per weight.
static __global__ void __launch_bounds__(256) k_wgrad_reduce(const float* __restrict__ part, int ncta, int N, int cout,
                                                             float* __restrict__ dW) {
    __shared__ float ws[8][32];
    const int total = 27 * 32 * cout;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + lane;
    float sum = 0.f;
    if (e < total) {
        const int tci = e / cout, co = e - tci * cout;
        const float* p = part + (long)tci * N + co;
        for (int c = warp; c < ncta; c += 8) sum += p[(long)c * 27 * 32 * N];
    }
    ws[warp][lane] = sum;
    __syncthreads();
    if (warp == 0 && e < total) {
        float t = ws[0][lane];
#pragma unroll
        for (int w = 1; w < 8; ++w) t += ws[w][lane];
        dW[e] += t;
    }
}

}  // namespace ins
