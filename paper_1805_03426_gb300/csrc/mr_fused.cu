// MR_VEL_FUSED: the FP32 step kernel with every stage of the refinement
// (Section 3.2) inside it, from the coarse faces.  The refined velocity, and
// every intermediate of the refinement, lives in shared memory and registers
// only; per step the kernel reads the coarse faces, T^s and T^{s-1} and
// writes T^{s+1}.
//
// The work is cut into chunks: a run of coarse slabs of a 64 x TY column of
// dense cells (TY = 8 or 16).  The step launches one CTA per resident slot,
// and each CTA marches its chunks one after the other without a break in its
// pipelines (the next chunk's coarse faces, first slab and first planes
// arrive while the current chunk's last layers are stepped); the reductions
// launch one CTA per chunk.  A CTA has three kinds of warps:
//   - a producer warp streams, through TMA onto mbarriers, the two scalar
//     planes of every dense layer with the layer's constants (a ring of NB
//     slots), and the coarse faces of every coarse slab (two buffers: the R_z
//     window planes of U and V and the slab's two W planes, for the tile's
//     coarse rows and columns with their neighbours, from a copy of the coarse
//     faces padded with their periodic images so that every box is in bounds);
//   - three builder warps form, from those coarse faces, the slab's refinement
//     stages at coarse resolution in x (two buffers: slab K+1 while slab K is
//     stepped; the first slab of a chunk is built by every consumer and
//     builder thread together):
//       stage Z  the full-area W on the slab's inner dense planes by the slab
//                balance, top-down, written as W(K+1) + sum_q Z[c][q] D_q with
//                D_q the horizontal divergence of coarse plane q of the R_z
//                window and Z[c][q] = sum_{c' >= c} dz_c' R_z[c'][q] (the same
//                linear map as the layer-by-layer balance, reassociated);
//       WY       R_y of the full-area W on the slab's M + 1 dense planes;
//       UO       the outer U sub-faces (R_y R_z of U), in units of U / (2 dx);
//       VR       the full-coarse-width V on every dense y-face of the tile: R_z
//                of V on the coarse faces, the row balance of stage Y (south
//                to north) on the inner ones, in units of V / (2 dy);
//   - the consumer warps run every dense layer: stage X (R_x splits of W and
//     V, the west-to-east cell balance for U) in registers, then the
//     finite-volume update of Eq. 5 with the Euler-leapfrog coefficients of
//     Section 2.2, on packed FP32 pairs.
// The hand-overs are full/empty mbarrier pairs (ring slots, coarse buffers,
// slab buffers); every wait is bounded, and a time-out records MR_ERR_TIMEOUT
// in a device flag.  Before the CTA exits, the producer waits for every copy
// it issued, so that none is in flight even after a time-out.
//
// Supported: FP32, periodic x and y, mx = my = mz = M in {2, 4},
// Nx % 64 == 0, Ny % 16 == 0, explicit diffusion, second-order faces.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "mr_internal.cuh"
#include "mr_ptx.cuh"

namespace mr {
namespace {

using namespace ptx;

constexpr int kTX = 64;                 // tile width (cells)
constexpr int kLCW = 32;                // layer-constant row (floats)
constexpr int kSCW = 32;                // slab-constant row (floats)
#ifndef MR_FUSED_IDLE_NS
#define MR_FUSED_IDLE_NS 256
#endif
constexpr unsigned kIdleNs = MR_FUSED_IDLE_NS;   // sleep between the polls of the producer and builder warps
// builder warps: three measured 0.379 ms per step on 512 x 512 x 384 (7.66 on
// 1536 x 1536 x 1024) against 0.397 (8.19) with two and 0.392 (7.87) with four
#ifndef MR_FUSED_BUILDER_WARPS
#define MR_FUSED_BUILDER_WARPS 3
#endif

__host__ __device__ constexpr int up32(int n) { return (n + 31) / 32 * 32; }

// Registers per thread of the step on 64 x 16 tiles (256 threads, two CTAs per
// SM): at launch, and after the split between the consumer warpgroup and the
// producer / builder warpgroup (128 kRegCons + 128 kRegOther = 256 kRegLaunch).
#ifndef MR_FUSED_REG_CONS
#define MR_FUSED_REG_CONS 184     // compile-time override for tuning sweeps
#endif
constexpr int kRegLaunch = 128, kRegCons = MR_FUSED_REG_CONS, kRegOther = 2 * kRegLaunch - kRegCons;
static_assert(kRegCons + kRegOther == 2 * kRegLaunch, "register split exceeds the launch");

// Shared-memory layout (offsets in floats; every TMA destination on a
// 128-byte boundary).  DIV: the reductions, which stream no scalar planes.
template <int M, int TY, bool DIV>
struct FL {
    // consumer threads: 4-cell segments of one dense row (the reductions) or
    // of two rows (the step)
    static constexpr int CONS = DIV ? 16 * TY : 8 * TY;
    static constexpr int NCW = CONS / 32;                   // consumer warps
    static constexpr int NBT = 32 * MR_FUSED_BUILDER_WARPS;  // builder threads
    static constexpr int THREADS = CONS + 32 + NBT;         // + producer warp + builder warps
    // resident CTAs per SM the layout is sized for (the step at M = 2, two rows
    // per consumer thread, runs two so that its registers need not spill)
    static constexpr int CTAS = (TY == 16 || (!DIV && M == 2)) ? 2 : 3;
    // registers move from warpgroup 1 (producer, builders) to warpgroup 0 (consumers)
    static constexpr bool RS = !DIV && CONS == 128 && NBT == 96;
#ifndef MR_FUSED_NB16
#define MR_FUSED_NB16 6           // ring slots of the step on 64 x 16 tiles (tuning override)
#endif
    static constexpr int NB = DIV ? 8 : (TY == 16 ? MR_FUSED_NB16 : (M == 4 ? 7 : 6));   // ring slots
    static constexpr int CX = kTX / M, CY = TY / M;         // coarse cells of the tile
    static constexpr int BXC = CX + 8;                      // coarse box columns I0-4 .. I0+CX+3
    static constexpr int SXC = CX + 4;                      // slab buffer columns I0-1 .. I0+CX+2
    // one scalar level (T^s or T^{s-1}) of one plane in a ring slot, each part a
    // TMA box on a 128-byte boundary: the tile's TY rows (64 wide), the row
    // south and the row north of them, the 4 columns west and east of them (the
    // periodic images at the domain's x edges, the periodic images or a
    // y-slab's halo rows at its y edges)
    static constexpr int fYS = kTX * TY, fYN = fYS + kTX, fXW = fYN + kTX, fXE = fXW + 4 * TY;
    static constexpr int FW = DIV ? 0 : fXE + 4 * TY;
    static_assert(FW % 32 == 0 && fXE % 32 == 0, "TMA boxes of a slot start on 128-byte boundaries");
    // ring slot: T^s, T^{s-1}, the layer constants
    static constexpr int oTn = 0, oTm = FW, oLC = 2 * FW;
    static constexpr int slot = up32(oLC + kLCW);
    // slab buffer: WY [M+1][TY][SXC], UO [M][TY][SXC], VR [M][TY+1][SXC]
    static constexpr int bWY = 0, bUO = (M + 1) * TY * SXC, bVR = bUO + M * TY * SXC;
    static constexpr int SLAB = up32(bVR + M * (TY + 1) * SXC);
    static constexpr int oSlab = NB * slot;
    // coarse buffer: U [3][NUR][BXC] (R_z window planes, coarse rows J0-1 .. J0+CY),
    // V [3][NVR][BXC] (rows J0-1 .. J0+CY+1), W [2][NUR][BXC] (planes K, K+1)
    static constexpr int NUR = CY + 2, NVR = CY + 3;
    static constexpr int cU = 0, cV = up32(3 * NUR * BXC), cW = cV + up32(3 * NVR * BXC);
    // then the slab's constants (fused_slab_constants)
    static constexpr int cSC = cW + up32(2 * NUR * BXC);
    static constexpr int CBOX = cSC + kSCW;
    static constexpr uint32_t cu_bytes = 3 * NUR * BXC * 4, cv_bytes = 3 * NVR * BXC * 4,
                              cw_bytes = 2 * NUR * BXC * 4;
    static constexpr int oCoarse = oSlab + 2 * SLAB;
    static constexpr int oZ = oCoarse + 2 * CBOX;           // stage Z: [M-1][NUR][BXC]
    static constexpr int oTcb = oZ + up32((M - 1) * NUR * BXC);   // upscale sums: [2][TY][CX]
    static constexpr int oRed = oTcb + (DIV ? 0 : up32(2 * TY * CX));   // 64 floats: reduction, failure flag
    static constexpr int oBar = (oRed + 64) / 2;            // in uint64
    // full[NB], empty[NB], cfull[2], cempty[2], built[2], freed[2]
    static constexpr size_t bytes = (size_t)(oBar + 2 * NB + 8) * 8;
};

// Tensor maps of the step: per scalar level (n: T^s, m: T^{s-1}) the tile's
// rows (64 x TY boxes), single rows (64 x 1), four columns (4 x TY), and single
// rows of the arrays holding the rows south of row 0 (s) and north of row Ny-1
// (h); then the layer constants, the padded coarse faces and the slab constants.
struct FLMaps {
    CUtensorMap tn, tm, rn, rm, xn, xm, sn, smp, hn, hm, lc, cu, cv, cw, sc;
};

struct FLArgs {
    Grid<float> g;
    float* Tp1;          // T^{s+1}
    float a, b, gdt;
    int kcs;             // coarse slabs per chunk
    int nch, zch, tpx;   // chunks in all, chunks per 64 x TY column, columns in x
    int nfull, sp, ps;   // chunks below nfull are whole; each later one is a part of ps slabs, sp per whole chunk
    int* err;
    unsigned long long* divmax;
    float rx[4][3];      // R_x rows of the 4 cells of a segment (uniform periodic x)
    float ry[4][3];      // R_y rows of the sub-rows of a coarse row (uniform periodic y)
    float iDX, iDY;      // 1 / DX, 1 / DY (coarse)
    float hx, hy;        // 1 / (2 dx), 1 / (2 dy)
    unsigned long long wait_ns;   // time limit of every bounded wait
    int stop_ring;       // test hook: the producer of CTA (0,0,0) issues nothing from this ring on (-1: none)
    double* Tc;          // NULL, or the upscaled coarse scalar of the new level [nz][ny][nx]
    const double* tcinv; // with Tc: per coarse slab, 1 / (mx my sum of its dz)
};

// R_x split of three coarse values by one row of R (rows sum to one).
__device__ __forceinline__ float rsplit3(const float (&r)[3], float c0, float c1, float c2)
{
    return c1 + r[0] * (c0 - c1) + r[2] * (c2 - c1);
}
// The same split negated, in as many operations.
__device__ __forceinline__ float nrsplit3(const float (&r)[3], float c0, float c1, float c2)
{
    return -c1 + r[0] * (c1 - c0) + r[2] * (c1 - c2);
}
// Packed FP32 pairs: one instruction updates two cells (sm_100 and later).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Named barriers of the builder group (id 2, the builder warps) and of the
// first slab's build (id 3, consumers and builders); each agrees on failure
// first, so that either every participant builds or none does.
template <int N>
__device__ __forceinline__ void named_sync(int id)
{
    asm volatile("barrier.cta.sync %0, %1;" ::"r"(id), "n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ bool named_or(int id, bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "barrier.cta.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "n"(N)
        : "memory");
    return r != 0;
}

// VR of the slab on the columns I0-1 .. I0+CX: the coarse face of rows
// J0 .. J0+CY from R_z of V, then, inside the tile, the row balance of stage Y
// south to north.  The UO and WY it reads and the VR it writes are disjoint
// regions of the slab buffer (separate restrict pointers, so that every load
// of an item can be issued ahead of its running balance).
template <int M, int TY, int NT>
__device__ __forceinline__ void build_vr(const float* __restrict__ cv, const float* __restrict__ uo_all,
                                         const float* __restrict__ wy_all, float* __restrict__ vr_all,
                                         const float (&rz)[M][3], const float (&hz)[M], float hy, int t0)
{
    using L = FL<M, TY, false>;
    constexpr int BXC = L::BXC, SXC = L::SXC, NVR = L::NVR, CX = L::CX, CY = L::CY, NZC = CX + 2;
    constexpr float iM = 1.f / (float)M;
    for (int t = t0; t < NZC * (CY + 1); t += NT) {
        const int Jr = t / NZC, xs = t - Jr * NZC, x = xs + 3;     // slab column xs, coarse box column x
        const float v0 = cv[(0 * NVR + Jr + 1) * BXC + x], v1 = cv[(1 * NVR + Jr + 1) * BXC + x],
                    v2 = cv[(2 * NVR + Jr + 1) * BXC + x];
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float du[M - 1], dw[M - 1];
            if (Jr < CY) {
                const float* uo = uo_all + (i * TY + Jr * M) * SXC + xs;
                const float* wb = wy_all + (i * TY + Jr * M) * SXC + xs;
#pragma unroll
                for (int b = 0; b < M - 1; ++b) {
                    du[b] = uo[b * SXC + 1] - uo[b * SXC];
                    dw[b] = wb[(TY + b) * SXC] - wb[b * SXC];
                }
            }
            float vr = (rz[i][0] * v0 + rz[i][1] * v1 + rz[i][2] * v2) * hy;
            float* dst = vr_all + (i * (TY + 1) + Jr * M) * SXC + xs;
            dst[0] = vr;
            if (Jr < CY) {
#pragma unroll
                for (int b = 0; b < M - 1; ++b) {
                    vr = vr - du[b] * iM - dw[b] * hz[i];
                    dst[(b + 1) * SXC] = vr;
                }
            }
        }
    }
}

// One coarse slab's refinement stages (see the file comment) from the coarse
// buffer cb into the slab buffer sb (sz: stage-Z scratch), by NT threads
// (this one t0) that meet at named barrier bar between the stages.  scg: the
// slab's constants, which come with its coarse faces (R_z rows of its M
// layers, 1/(2 dz) of each, the stage-Z weights Z[c][q]).
template <int M, int TY, int NT>
__device__ void build_slab(const FLArgs& A, const float* __restrict__ cb, float* __restrict__ sb,
                           float* __restrict__ sz, const float* __restrict__ scg, int t0, int bar)
{
    using L = FL<M, TY, false>;
    constexpr int BXC = L::BXC, SXC = L::SXC, NUR = L::NUR, NVR = L::NVR, CX = L::CX, CY = L::CY;
    const float* cu = cb + L::cU;
    const float* cv = cb + L::cV;
    const float* cw = cb + L::cW;
    float rz[M][3], hz[M], zc[M - 1][3];
#pragma unroll
    for (int i = 0; i < M; ++i) {
#pragma unroll
        for (int q = 0; q < 3; ++q) rz[i][q] = scg[3 * i + q];
        hz[i] = scg[3 * M + i];
    }
#pragma unroll
    for (int c = 0; c < M - 1; ++c)
#pragma unroll
        for (int q = 0; q < 3; ++q) zc[c][q] = scg[4 * M + 3 * c + q];
    const float iDX = A.iDX, iDY = A.iDY, hx = A.hx;
    // one pass over two kinds of items (so that the builder lanes stay busy):
    // stage Z on the columns I0-1 .. I0+CX of coarse rows J0-1 .. J0+CY, and
    // UO of the slab's M layers on the columns I0-1 .. I0+CX+1 (from the
    // coarse faces alone, so before the barrier): the z split of the three
    // window rows is shared by the coarse row's M dense rows
    constexpr int NZC = CX + 2, NUC = CX + 3, NZI = NUR * NZC;
    for (int t = t0; t < NZI + NUC * CY; t += NT) {
        if (t < NZI) {
            const int r = t / NZC, x = 3 + t - r * NZC;
            float D[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float uw = cu[(q * NUR + r) * BXC + x], ue = cu[(q * NUR + r) * BXC + x + 1];
                const float vs = cv[(q * NVR + r) * BXC + x], vn = cv[(q * NVR + r + 1) * BXC + x];
                D[q] = (ue - uw) * iDX + (vn - vs) * iDY;
            }
            const float wtop = cw[(NUR + r) * BXC + x];
#pragma unroll
            for (int c = 0; c < M - 1; ++c)
                sz[(c * NUR + r) * BXC + x] = wtop + zc[c][0] * D[0] + zc[c][1] * D[1] + zc[c][2] * D[2];
        } else {
            const int u0 = t - NZI, Jc = u0 / NUC, x = 3 + u0 - Jc * NUC;
            float u[3][3];
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int p = 0; p < 3; ++p) u[q][p] = cu[(q * NUR + Jc + p) * BXC + x];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                float a[3];
#pragma unroll
                for (int p = 0; p < 3; ++p)
                    a[p] = (rz[i][0] * u[0][p] + rz[i][1] * u[1][p] + rz[i][2] * u[2][p]) * hx;
                float* dst = sb + L::bUO + (i * TY + Jc * M) * SXC + x - 3;
#pragma unroll
                for (int b = 0; b < M; ++b) dst[b * SXC] = A.ry[b][0] * a[0] + A.ry[b][1] * a[1] + A.ry[b][2] * a[2];
            }
        }
    }
    named_sync<NT>(bar);
    // WY on the slab's M + 1 dense planes: per (plane, coarse row, column)
    for (int t = t0; t < NZC * CY * (M + 1); t += NT) {
        const int i = t / (NZC * CY), rem = t - i * (NZC * CY), Jc = rem / NZC, x = 3 + rem - Jc * NZC;
        const float* src = (i == 0) ? cw : (i == M ? cw + NUR * BXC : sz + (i - 1) * NUR * BXC);
        const float c0 = src[Jc * BXC + x], c1 = src[(Jc + 1) * BXC + x], c2 = src[(Jc + 2) * BXC + x];
        float* dst = sb + L::bWY + (i * TY + Jc * M) * SXC + x - 3;
#pragma unroll
        for (int b = 0; b < M; ++b) dst[b * SXC] = A.ry[b][0] * c0 + A.ry[b][1] * c1 + A.ry[b][2] * c2;
    }
    named_sync<NT>(bar);
    build_vr<M, TY, NT>(cv, sb + L::bUO, sb + L::bWY, sb + L::bVR, rz, hz, A.hy, t0);
    named_sync<NT>(bar);
}

// KIND 0: the step; 1: max |divergence| of the dense velocity; 2: max CFL rate.
// LF: a plain leapfrog step (a = 1, b = 0).  TC: the step also writes the
// upscaled coarse scalar of the new level (A.Tc), which a coupled coarse solver
// takes back every step: the consumers leave each row's dz-weighted sums of a
// slab in shared memory, and once the slab is freed the builder warps add the
// M rows of each coarse cell and scale them (Section 3.3).
template <int M, int TY, int KIND, bool LF, bool TC = false>
__global__ void __launch_bounds__(FL<M, TY, (KIND != 0)>::THREADS, FL<M, TY, (KIND != 0)>::CTAS)
k_fused(const __grid_constant__ FLMaps T, const FLArgs A)
{
    constexpr bool DIVONLY = KIND != 0;
    using L = FL<M, TY, DIVONLY>;
    constexpr int NB = L::NB, SXC = L::SXC, NC = 4 / M, NCW = L::NCW, CONS = L::CONS;
    extern __shared__ __align__(128) float sm[];
    float* red = sm + L::oRed;
    volatile int* s_fail = reinterpret_cast<volatile int*>(sm + L::oRed + 32);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm) + L::oBar;
    uint64_t* empty = full + NB;
    uint64_t* cfull = empty + NB;
    uint64_t* cempty = cfull + 2;
    uint64_t* built = cempty + 2;
    uint64_t* freed = built + 2;

    const Grid<float>& g = A.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Chunk c: the coarse slabs K0 .. K1-1 of the 64 x TY column at (i0, j0).
    // A CTA steps the chunks blockIdx.x, blockIdx.x + gridDim.x, ... (the
    // step launches one CTA per resident slot, the reductions one per chunk);
    // the chunks of a column are consecutive, so that the CTAs resident at one
    // time cover neighbouring columns at the same heights.  Every counter of
    // ring slots, coarse buffers and slab buffers runs on across the chunks of
    // a CTA, so that the next chunk's coarse faces, first slab and first planes
    // are fetched and built while the current chunk's last layers are stepped.
    // The chunks from A.nfull on are parts of the last whole chunks, sp parts
    // of ps slabs each (some may be empty: K0 >= K1, skipped by every warp),
    // so that the CTAs' shares of the last round differ by one part at most.
    struct Chunk { int K0, K1, i0, j0; };
    auto chunk = [&](int c) {
        int cw = c, q = -1;
        if (c >= A.nfull) {
            cw = A.nfull + (c - A.nfull) / A.sp;
            q = (c - A.nfull) % A.sp;
        }
        const int cz = cw % A.zch, t = cw / A.zch;
        Chunk h;
        h.K0 = cz * A.kcs;
        h.K1 = min(h.K0 + A.kcs, g.nz);
        if (q >= 0) {
            h.K0 += q * A.ps;
            h.K1 = min(h.K0 + A.ps, h.K1);
        }
        h.i0 = (t % A.tpx) * kTX;
        h.j0 = (t / A.tpx) * TY;
        return h;
    };

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CONS);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&cfull[s], 1);
            mbar_init(&cempty[s], L::NBT);
            mbar_init(&built[s], L::NBT);
            mbar_init(&freed[s], CONS);
        }
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    int rings_issued = 0, slabs_issued = 0;       // producer lane 0: for the final drain
    // the step on 64 x 16 tiles: the consumer warps (warpgroup 0) take
    // registers from the producer and builder warps (warpgroup 1); the launch
    // gives every thread kRegLaunch (checked on the host before the launch)
    if (warp >= NCW) {
        if constexpr (L::RS) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kRegOther));
        if (warp == NCW) {
            // ------------------------------------------------------------ producer warp
            if (lane == 0) {
                const bool stopper = (A.stop_ring >= 0 && blockIdx.x == 0);
                int R = 0;                                // rings of the CTA's earlier chunks
                bool ok = true, stopped = stopper && A.stop_ring == 0;
                for (int c = blockIdx.x; ok && !stopped && c < A.nch; c += gridDim.x) {
                    const Chunk h = chunk(c);
                    if (h.K0 >= h.K1) continue;
                    const int K0 = h.K0, K1 = h.K1, i0 = h.i0, j0 = h.j0, I0 = i0 / M, J0 = j0 / M;
                    const int k0 = K0 * M, k1 = K1 * M;
                    const int nrings = k1 - k0 + 2;      // ring R + r: plane k0-1+r and the constants of layer k0+r-2
                    // the coarse faces of slab K into buffer S & 1, S counting the
                    // slabs of every chunk of the CTA
                    auto issue_coarse = [&](int K) {
                        const int S = slabs_issued, bb = S & 1, use = S >> 1;
                        if (use > 0 && !mbar_wait_idle(&cempty[bb], (use - 1) & 1, A.wait_ns, kIdleNs)) return false;
                        float* dst = sm + L::oCoarse + bb * L::CBOX;
                        const int wz0 = min(max(K - 1, 0), g.nz - 3);     // first plane of the R_z window
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        mbar_expect_tx(&cfull[bb], L::cu_bytes + L::cv_bytes + L::cw_bytes + kSCW * 4);
                        tma_3d(dst + L::cU, &T.cu, I0, J0, wz0, &cfull[bb]);
                        tma_3d(dst + L::cV, &T.cv, I0, J0, wz0, &cfull[bb]);
                        tma_3d(dst + L::cW, &T.cw, I0, J0, K, &cfull[bb]);
                        tma_3d(dst + L::cSC, &T.sc, 0, K, 0, &cfull[bb]);
                        ++slabs_issued;
                        return true;
                    };
                    // the rows south / north of the tile: inside the domain from the
                    // level itself, beyond its y edges from the arrays of those rows;
                    // the columns west / east: periodic in x
                    const bool s_edge = (j0 == 0), n_edge = (j0 + TY == g.Ny);
                    const CUtensorMap* ys_n = s_edge ? &T.sn : &T.rn;
                    const CUtensorMap* ys_m = s_edge ? &T.smp : &T.rm;
                    const CUtensorMap* yn_n = n_edge ? &T.hn : &T.rn;
                    const CUtensorMap* yn_m = n_edge ? &T.hm : &T.rm;
                    const int ys_y = s_edge ? 0 : j0 - 1, yn_y = n_edge ? 0 : j0 + TY;
                    const int xw_x = (i0 == 0) ? g.Nx - 4 : i0 - 4, xe_x = (i0 + kTX == g.Nx) ? 0 : i0 + kTX;
                    ok = issue_coarse(K0);
                    if (ok && K0 + 1 < K1) ok = issue_coarse(K0 + 1);
                    for (int r = 0; ok && r < nrings; ++r) {
                        const int G = R + r, s = G % NB;  // the CTA's ring G: slot G % NB, phase G / NB
                        if (stopper && G == A.stop_ring) {   // every copy issued so far is waited for
                            stopped = true;
                            break;
                        }
                        if (G >= NB && !mbar_wait_idle(&empty[s], ((G / NB) - 1) & 1, A.wait_ns, kIdleNs)) {
                            ok = false;
                            break;
                        }
                        float* slot = sm + s * L::slot;
                        const int p = k0 - 1 + r;
                        const bool lc = (r >= 2);
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        mbar_expect_tx(&full[s], (uint32_t)(2 * L::FW + (lc ? kLCW : 0)) * 4u);
                        if (!DIVONLY) {
                            // per level: the tile's rows, the rows beyond its y edges, the
                            // columns beyond its x edges (wrapped at the domain's edges,
                            // so that every box is in bounds in x and y)
                            tma_3d(slot + L::oTn, &T.tn, i0, j0, p, &full[s]);
                            tma_3d(slot + L::oTm, &T.tm, i0, j0, p, &full[s]);
                            tma_3d(slot + L::oTn + L::fYS, ys_n, i0, ys_y, p, &full[s]);
                            tma_3d(slot + L::oTm + L::fYS, ys_m, i0, ys_y, p, &full[s]);
                            tma_3d(slot + L::oTn + L::fYN, yn_n, i0, yn_y, p, &full[s]);
                            tma_3d(slot + L::oTm + L::fYN, yn_m, i0, yn_y, p, &full[s]);
                            tma_3d(slot + L::oTn + L::fXW, &T.xn, xw_x, j0, p, &full[s]);
                            tma_3d(slot + L::oTm + L::fXW, &T.xm, xw_x, j0, p, &full[s]);
                            tma_3d(slot + L::oTn + L::fXE, &T.xn, xe_x, j0, p, &full[s]);
                            tma_3d(slot + L::oTm + L::fXE, &T.xm, xe_x, j0, p, &full[s]);
                        }
                        if (lc) tma_3d(slot + L::oLC, &T.lc, 0, p - 1, 0, &full[s]);
                        rings_issued = G + 1;
                        // the first plane of slab K (K > K0) goes out with the coarse faces of slab K + 1
                        if (p > k0 && p < k1 && (p - k0) % M == 0 && p / M + 1 < K1) ok = issue_coarse(p / M + 1);
                    }
                    R += nrings;
                }
                if (!ok) *s_fail = 1;
            }
        } else {
            // ------------------------------------------------------------ builder warps
            const int bt = tid - CONS - 32;              // 0 .. NBT-1
            bool fail = false;
            int S = 0;                                   // slabs of the CTA built so far (every chunk)
            // TC: coarse slab and chunk of the slabs in buffers 0 and 1
            int hK0 = 0, hc0 = 0, hK1 = 0, hc1 = 0;
            // TC: the coarse cells of a freed slab Sx (sums over its M dense rows, in
            // the rows' order, in FP32; the scaling in FP64)
            auto upscale = [&](int Sx) {
                constexpr int CX = L::CX, CY = L::CY;
                const int bb = Sx & 1, K = bb ? hK1 : hK0;
                const Chunk h = chunk(bb ? hc1 : hc0);
                const int I0 = h.i0 / M, J0 = h.j0 / M;
                const float* tb = sm + L::oTcb + bb * TY * CX;
                const double inv = A.tcinv[K];
                for (int t = bt; t < CY * CX; t += L::NBT) {
                    const int Jc = t / CX, I = t - Jc * CX;
                    float v = 0.f;
    #pragma unroll
                    for (int b = 0; b < M; ++b) v += tb[(Jc * M + b) * CX + I];
                    A.Tc[((size_t)K * g.ny + J0 + Jc) * g.nx + I0 + I] = (double)v * inv;
                }
            };
            for (int c = blockIdx.x; !fail && c < A.nch; c += gridDim.x) {
                const Chunk h = chunk(c);
                for (int K = h.K0; K < h.K1; ++K, ++S) {
                    const int bb = S & 1, use = S >> 1;
                    if (S == 0) {
                        // the CTA's first slab, with the consumers
                        fail = !mbar_wait(&cfull[0], 0, A.wait_ns);
                        fail = named_or<CONS + L::NBT>(3, fail);
                        if (!fail)
                            build_slab<M, TY, CONS + L::NBT>(A, sm + L::oCoarse, sm + L::oSlab, sm + L::oZ,
                                                             sm + L::oCoarse + L::cSC, CONS + bt, 3);
                    } else {
                        bool f = !mbar_wait_idle(&cfull[bb], use & 1, A.wait_ns, kIdleNs);
                        if (!f && use > 0) f = !mbar_wait_idle(&freed[bb], (use - 1) & 1, A.wait_ns, kIdleNs);
                        fail = named_or<L::NBT>(2, f);
                        if (!fail) {
                            if constexpr (TC) {
                                if (use > 0) upscale(S - 2);
                            }
                            build_slab<M, TY, L::NBT>(A, sm + L::oCoarse + bb * L::CBOX, sm + L::oSlab + bb * L::SLAB,
                                                      sm + L::oZ, sm + L::oCoarse + bb * L::CBOX + L::cSC, bt, 2);
                        }
                    }
                    if (fail) break;
                    mbar_arrive(&cempty[bb]);
                    mbar_arrive(&built[bb]);
                    if (bb) {
                        hK1 = K;
                        hc1 = c;
                    } else {
                        hK0 = K;
                        hc0 = c;
                    }
                }
            }
            if constexpr (TC) {
                // the last two slabs, once the consumers have freed them
                for (int Sx = max(0, S - 2); Sx < S && !fail; ++Sx) {
                    fail = named_or<L::NBT>(2, !mbar_wait_idle(&freed[Sx & 1], (Sx >> 1) & 1, A.wait_ns, kIdleNs));
                    if (!fail) upscale(Sx);
                }
            }
            if (fail && bt == 0) *s_fail = 1;
        }
    } else {
        if constexpr (L::RS) asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kRegCons));
        if constexpr (DIVONLY) {
            // ------------------------------------------------------------ consumer warps (the reductions)
            // this thread's 4-cell segment of dense row jl; the half-warps take rows
            // four apart (slab rows 4 SXC floats apart fall 16 banks apart, so the
            // half-warps' coarse-column reads do not conflict)
            const int seg = tid & 15, jl = ((warp >> 2) << 3) + (warp & 3) + 4 * ((tid >> 4) & 1);
            const int cb0 = seg * 4 / M;                 // first coarse column of the segment (tile-local)
            const auto& rx = A.rx;
            // one chunk per CTA (the reductions launch one CTA per chunk)
            const Chunk h = chunk(blockIdx.x);
            const int k0 = h.K0 * M, k1 = h.K1 * M;
            bool fail = false;
            float dmax = 0.f;
            float wcar[4] = {0.f, 0.f, 0.f, 0.f};        // R_x split of W on plane k (from layer k-1)
            // the chunk's first slab, with the builder warps
            fail = !mbar_wait(&cfull[0], 0, A.wait_ns);
            fail = named_or<CONS + L::NBT>(3, fail);
            if (!fail)
                build_slab<M, TY, CONS + L::NBT>(A, sm + L::oCoarse, sm + L::oSlab, sm + L::oZ, sm + L::oCoarse + L::cSC,
                                                 tid, 3);
            for (int r = 0; r < 2; ++r)
                if (!fail && !mbar_wait(&full[r], 0, A.wait_ns)) fail = true;
            auto layer = [&](const int k, const int i, const int Kr, const int sb, const int st, const int tpar) {
                const int bb = Kr & 1;
                if (i == 0 && Kr > 0 && !fail && !mbar_wait(&built[bb], (Kr >> 1) & 1, A.wait_ns)) fail = true;
                if (!fail && !mbar_wait(&full[st], tpar, A.wait_ns)) fail = true;
                if (!fail) {
                    const float* slab = sm + L::oSlab + bb * L::SLAB;
                    const float* lcp = sm + st * L::slot + L::oLC;
                    const float2 c0 = *reinterpret_cast<const float2*>(lcp);
                    const float inv_dz = c0.x, hz = c0.y;
                    float wb[4], wt[4], vs[4], vn[4], us[5];
                    // R_x splits of the full-width W (planes k, k+1) and V (faces jl, jl+1);
                    // slab column c holds coarse column I0 - 1 + c
                    const float* yt = slab + L::bWY + ((i + 1) * TY + jl) * SXC + cb0;
                    const float* rs = slab + L::bVR + (i * (TY + 1) + jl) * SXC + cb0;
                    const float* rn = rs + SXC;
                    const float* ur = slab + L::bUO + (i * TY + jl) * SXC + cb0 + 1;   // outer face of column cb0
                    constexpr int NV = NC + 2;
                    float ytv[NV], rsv[NV], rnv[NV], urv[NC + 1];
                    if (k == k0) {
                        const float* yb = slab + L::bWY + jl * SXC + cb0;            // plane k0 (i = 0)
    #pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int cb = a / M;
                            wcar[a] = rsplit3(rx[a], yb[cb], yb[cb + 1], yb[cb + 2]);
                        }
                    }
    #pragma unroll
                    for (int c = 0; c < NV; ++c) {
                        ytv[c] = yt[c];
                        rsv[c] = rs[c];
                        rnv[c] = rn[c];
                    }
    #pragma unroll
                    for (int q = 0; q <= NC; ++q) urv[q] = ur[q];
    #pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int cb = a / M;
                        wb[a] = wcar[a];
                        wt[a] = rsplit3(rx[a], ytv[cb], ytv[cb + 1], ytv[cb + 2]);
                        vs[a] = rsplit3(rx[a], rsv[cb], rsv[cb + 1], rsv[cb + 2]);
                        vn[a] = rsplit3(rx[a], rnv[cb], rnv[cb + 1], rnv[cb + 2]);
                    }
                    // stage X: cell balance, west to east, in units of U / (2 dx)
    #pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        float h = urv[q];
                        us[q * M] = h;
    #pragma unroll
                        for (int a = 0; a < M - 1; ++a) {
                            const int m = q * M + a;
                            h = h - (vn[m] - vs[m]) - (wt[m] - wb[m]) * hz;
                            us[m + 1] = h;
                        }
                    }
                    us[4] = urv[NC];
    #pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        wcar[a] = wt[a];
                        const float d = KIND == 2 ? 2.f * (fmaxf(fabsf(us[a]), fabsf(us[a + 1])) +
                                                           fmaxf(fabsf(vs[a]), fabsf(vn[a]))) +
                                                        fmaxf(fabsf(wb[a]), fabsf(wt[a])) * inv_dz
                                                  : 2.f * ((us[a + 1] - us[a]) + (vn[a] - vs[a])) +
                                                        (wt[a] - wb[a]) * inv_dz;
                        dmax = fmaxf(dmax, fabsf(d));
                    }
                }
                // ring slot sb (plane k-1) and, after the slab's last layer, the
                // slab's intermediates are no longer needed by this thread
                mbar_arrive(&empty[sb]);
                if (i == M - 1) mbar_arrive(&freed[bb]);
            };
            {
                int sb = 0, st = 2, tpar = 0;
                for (int k = k0; k < k1; ++k) {
                    layer(k, k & (M - 1), (k - k0) / M, sb, st, tpar);
                    sb = (sb + 1 == NB) ? 0 : sb + 1;
                    if (++st == NB) {
                        st = 0;
                        tpar ^= 1;
                    }
                }
            }
            if (fail) *s_fail = 1;
            for (int d = 16; d > 0; d >>= 1) dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, d));
            if (lane == 0) red[warp] = dmax;
        } else {
            // ------------------------------------------------------------ consumer warps (the step)
            // this thread's 4-cell segment of the dense rows jl and jl + 1; the
            // half-warps take row pairs four rows apart (slab rows 4 SXC floats
            // apart fall 16 banks apart, so the half-warps' coarse-column reads do
            // not conflict).  Per layer a thread loads from the ring its two rows
            // of plane k + 1 and the rows jl - 1 and jl + 2 of plane k, and splits
            // the V face between its rows once.  Carried from layer to layer
            // (Carry): the rows of T^s and T^{s-1} on plane k, the advective flux
            // through the layer's bottom face (w T_f), the diffusive term of the
            // plane below (cdn T^{s-1}_{k-1}) and the R_x split of W on plane k.
            // Layers run in pairs with both rings waited for first, so that the
            // pair's body has no branch: the two Carry sets alternate and no
            // register is copied between layers.
            const int seg = tid & 15, jl = ((warp >> 1) << 3) + ((warp & 1) << 1) + 4 * ((tid >> 4) & 1);
            const int il0 = seg * 4, cb0 = il0 / M;      // first coarse column of the segment (tile-local)
            const auto& rx = A.rx;
            bool fail = false;
            const float2 kx2p = make_float2(g.kx2, g.kx2), ky2p = make_float2(g.ky2, g.ky2);
            const float2 gdtp = make_float2(A.gdt, A.gdt), cap = make_float2(A.a, A.a), cbp = make_float2(A.b, A.b);
            const size_t plane = (size_t)g.Nx * g.Ny;
            // offsets in a level of a ring slot: the segment's first cell of row jl
            // (row jl + 1 follows kTX floats on), of rows jl - 1 and jl + 2, and the
            // west / east neighbours of row jl (row jl + 1: 4 floats on)
            const int om = jl * kTX + il0;
            const int osr = (jl == 0) ? L::fYS + il0 : om - kTX;
            const int onr = (jl + 2 == TY) ? L::fYN + il0 : om + 2 * kTX;
            const int oxw = L::fXW + jl * 4 + 3, oxe = L::fXE + jl * 4;
            struct Carry {
                float4 t[2], d[2];     // T^s, T^{s-1} of rows jl, jl + 1 on plane k
                float2 ab[2][2];       // advective flux w T_f through the bottom face of layer k (pairs)
                float2 pd[2][2];       // cdn_k T^{s-1} on plane k - 1 (pairs)
                float w[2][4];         // R_x split of W on plane k
            };
            Carry S0, S1;
            int R = 0, S = 0;                            // rings and slabs of the CTA's earlier chunks
            for (int c = blockIdx.x; !fail && c < A.nch; c += gridDim.x) {
                const Chunk h = chunk(c);
                if (h.K0 >= h.K1) continue;
                const int k0 = h.K0 * M, k1 = h.K1 * M, nrings = k1 - k0 + 2;
                float* outp = A.Tp1 + (size_t)k0 * plane + (size_t)(h.j0 + jl) * g.Nx + h.i0 + il0;
                float tcs[2][NC] = {};                       // upscale partials of the segment's coarse columns
                if (S == 0) {
                    // the CTA's first slab, with the builder warps (measured faster than
                    // waiting for the builders alone)
                    fail = !mbar_wait(&cfull[0], 0, A.wait_ns);
                    fail = named_or<CONS + L::NBT>(3, fail);
                    if (!fail)
                        build_slab<M, TY, CONS + L::NBT>(A, sm + L::oCoarse, sm + L::oSlab, sm + L::oZ,
                                                         sm + L::oCoarse + L::cSC, tid, 3);
                } else if (!mbar_wait(&built[S & 1], (S >> 1) & 1, A.wait_ns)) {
                    fail = true;                             // a later chunk's first slab, from the builder warps
                }
                // planes k0 - 1, k0, k0 + 1 (rings R, R + 1, R + 2; ring R + 2 holds
                // the constants of layer k0): the state at the chunk's first layer
                const int s0 = R % NB, s1 = (R + 1) % NB, s2 = (R + 2) % NB;
                for (int r = 0; r < 3; ++r)
                    if (!fail && !mbar_wait(&full[(R + r) % NB], ((R + r) / NB) & 1, A.wait_ns)) fail = true;
                if (!fail) {
                    const float* lc0 = sm + s2 * L::slot + L::oLC;
                    const float dzk = lc0[2], bwlo = lc0[12], bwhi = lc0[14], cdn = lc0[20];
                    const float* yb = sm + L::oSlab + (S & 1) * L::SLAB + L::bWY + jl * SXC + cb0;   // plane k0 (i = 0)
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const float4 tb = *reinterpret_cast<const float4*>(sm + s0 * L::slot + L::oTn + om + r * kTX);
                        const float4 db = *reinterpret_cast<const float4*>(sm + s0 * L::slot + L::oTm + om + r * kTX);
                        S0.t[r] = *reinterpret_cast<const float4*>(sm + s1 * L::slot + L::oTn + om + r * kTX);
                        S0.d[r] = *reinterpret_cast<const float4*>(sm + s1 * L::slot + L::oTm + om + r * kTX);
                        const float tbv[4] = {tb.x, tb.y, tb.z, tb.w};
                        const float tcv[4] = {S0.t[r].x, S0.t[r].y, S0.t[r].z, S0.t[r].w};
                        const float dbv[4] = {db.x, db.y, db.z, db.w};
                        float ab[4], pd[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int cb = r * SXC + a / M;
                            S0.w[r][a] = rsplit3(rx[a], yb[cb], yb[cb + 1], yb[cb + 2]);
                            ab[a] = S0.w[r][a] * (dzk * (bwlo * tbv[a] + bwhi * tcv[a]));
                            pd[a] = cdn * dbv[a];
                        }
                        S0.ab[r][0] = make_float2(ab[0], ab[1]);
                        S0.ab[r][1] = make_float2(ab[2], ab[3]);
                        S0.pd[r][0] = make_float2(pd[0], pd[1]);
                        S0.pd[r][1] = make_float2(pd[2], pd[3]);
                    }
                }
                mbar_arrive(&empty[s0]);
                // one layer, no waits: sc, st the ring slots of planes k, k + 1; bb the
                // slab buffer; in the state at layer k, out the state at layer k + 1
                auto layer = [&](const int k, const int i, const int bb, const int sc, const int st, const Carry& in,
                                 Carry& out) {
                    const float* slab = sm + L::oSlab + bb * L::SLAB;
                    const float* lcp = sm + st * L::slot + L::oLC;
                    const float hz = lcp[1];
                    float vf[3][4], us[2][5];
                    {
                        // R_x splits of the full-width W (plane k+1, rows jl, jl+1) and V
                        // (faces jl, jl+1, jl+2); slab column c holds coarse column I0 - 1 + c
                        constexpr int NV = NC + 2;
                        const float* yt = slab + L::bWY + ((i + 1) * TY + jl) * SXC + cb0;
                        const float* rs = slab + L::bVR + (i * (TY + 1) + jl) * SXC + cb0;
                        const float* ur = slab + L::bUO + (i * TY + jl) * SXC + cb0 + 1;   // outer face of column cb0
                        float ytv[2][NV], vv[3][NV], urv[2][NC + 1];
#pragma unroll
                        for (int c = 0; c < NV; ++c) {
                            ytv[0][c] = yt[c];
                            ytv[1][c] = yt[SXC + c];
                            vv[0][c] = rs[c];
                            vv[1][c] = rs[SXC + c];
                            vv[2][c] = rs[2 * SXC + c];
                        }
#pragma unroll
                        for (int q = 0; q <= NC; ++q) {
                            urv[0][q] = ur[q];
                            urv[1][q] = ur[SXC + q];
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int cb = a / M;
#pragma unroll
                            for (int r = 0; r < 2; ++r)
                                out.w[r][a] = rsplit3(rx[a], ytv[r][cb], ytv[r][cb + 1], ytv[r][cb + 2]);
#pragma unroll
                            for (int f = 0; f < 3; ++f)
                                vf[f][a] = rsplit3(rx[a], vv[f][cb], vv[f][cb + 1], vv[f][cb + 2]);
                        }
                        // stage X: cell balance, west to east, in units of U / (2 dx)
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
#pragma unroll
                            for (int q = 0; q < NC; ++q) {
                                float h = urv[r][q];
                                us[r][q * M] = h;
#pragma unroll
                                for (int a = 0; a < M - 1; ++a) {
                                    const int m = q * M + a;
                                    h = h - (vf[r + 1][m] - vf[r][m]) - (out.w[r][m] - in.w[r][m]) * hz;
                                    us[r][m + 1] = h;
                                }
                            }
                            us[r][4] = urv[r][NC];
                        }
                    }
                    const float* Pn_c = sm + sc * L::slot + L::oTn;
                    const float* Pm_c = sm + sc * L::slot + L::oTm;
                    const float* Pn_t = sm + st * L::slot + L::oTn;
                    const float* Pm_t = sm + st * L::slot + L::oTm;
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        out.t[r] = *reinterpret_cast<const float4*>(Pn_t + om + r * kTX);
                        out.d[r] = *reinterpret_cast<const float4*>(Pm_t + om + r * kTX);
                    }
                    // rows jl - 1 and jl + 2 of plane k
                    const float4 ts4 = *reinterpret_cast<const float4*>(Pn_c + osr);
                    const float4 ds4 = *reinterpret_cast<const float4*>(Pm_c + osr);
                    const float4 tn4 = *reinterpret_cast<const float4*>(Pn_c + onr);
                    const float4 dn4 = *reinterpret_cast<const float4*>(Pm_c + onr);
                    // x neighbours: shuffles inside the tile, the slot's edge columns at its edges
                    float tw[2], te[2], dw[2], de[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        tw[r] = __shfl_up_sync(0xffffffffu, in.t[r].w, 1);
                        te[r] = __shfl_down_sync(0xffffffffu, in.t[r].x, 1);
                        dw[r] = __shfl_up_sync(0xffffffffu, in.d[r].w, 1);
                        de[r] = __shfl_down_sync(0xffffffffu, in.d[r].x, 1);
                        if (seg == 0) {
                            tw[r] = Pn_c[oxw + 4 * r];
                            dw[r] = Pm_c[oxw + 4 * r];
                        }
                        if (seg == 15) {
                            te[r] = Pn_c[oxe + 4 * r];
                            de[r] = Pm_c[oxe + 4 * r];
                        }
                    }
                    // x fluxes in scalar form (adjacent cells share a face), then the
                    // rest on the pairs (0, 1), (2, 3) with the pair constants of the layer:
                    // D = kx2 (dw + de) + ky2 (ds + dn) + cdn db + cup dt - diag dc + plate,
                    // the z advective terms as (w T_f)(bottom) - (w T_f)(top) over dz; the
                    // planes beyond the plates are zero-filled, where W is zero and the plate
                    // value enters D through `plate`
                    const float4 qf = *reinterpret_cast<const float4*>(lcp + 4);    // f_lo, f_hi (top face)
                    const float4 qn = *reinterpret_cast<const float4*>(lcp + 8);    // 1/dz, cdn of layer k+1
                    const float4 q2 = *reinterpret_cast<const float4*>(lcp + 20);   // cdn, cup
                    const float4 q3 = *reinterpret_cast<const float4*>(lcp + 24);   // -diag, plate
                    float4 out4[2];
#pragma unroll
                    for (int r = 0; r < 2; ++r) {
                        const float4 tc4 = in.t[r], dc4 = in.d[r];
                        const float4 tsr = r ? in.t[0] : ts4, tnr = r ? tn4 : in.t[1];
                        const float4 dsr = r ? in.d[0] : ds4, dnr = r ? dn4 : in.d[1];
                        const float tcv[6] = {tw[r], tc4.x, tc4.y, tc4.z, tc4.w, te[r]};
                        const float dcv[6] = {dw[r], dc4.x, dc4.y, dc4.z, dc4.w, de[r]};
                        float F[5], cxv[4], sdx[4];
#pragma unroll
                        for (int a = 0; a < 5; ++a) F[a] = us[r][a] * (tcv[a] + tcv[a + 1]);
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            cxv[a] = F[a] - F[a + 1];
                            sdx[a] = dcv[a] + dcv[a + 2];
                        }
                        float2 res[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 tcp = h ? hi2(tc4) : lo2(tc4), dcp = h ? hi2(dc4) : lo2(dc4);
                            const float2 tsp = h ? hi2(tsr) : lo2(tsr), tnp = h ? hi2(tnr) : lo2(tnr);
                            const float2 dsp = h ? hi2(dsr) : lo2(dsr), dnp = h ? hi2(dnr) : lo2(dnr);
                            const float2 ttp = h ? hi2(out.t[r]) : lo2(out.t[r]);
                            const float2 dtp = h ? hi2(out.d[r]) : lo2(out.d[r]);
                            const int a = 2 * h;
                            // the top face: T_f = f_lo T_k + f_hi T_{k+1}, its advective flux
                            const float2 atop = mul2(make_float2(out.w[r][a], out.w[r][a + 1]),
                                                     fma2(lo2(qf), tcp, mul2(hi2(qf), ttp)));
                            float2 acc = fma2(kx2p, make_float2(sdx[a], sdx[a + 1]), hi2(q3));
                            acc = fma2(ky2p, add2(dsp, dnp), acc);
                            acc = add2(acc, in.pd[r][h]);
                            acc = fma2(hi2(q2), dtp, acc);
                            acc = fma2(lo2(q3), dcp, acc);
                            acc = add2(acc, make_float2(cxv[a], cxv[a + 1]));
                            acc = fma2(make_float2(vf[r][a], vf[r][a + 1]), add2(tsp, tcp), acc);
                            acc = fma2(make_float2(-vf[r + 1][a], -vf[r + 1][a + 1]), add2(tcp, tnp), acc);
                            acc = fma2(lo2(qn), add2(in.ab[r][h], make_float2(-atop.x, -atop.y)), acc);
                            res[h] = LF ? fma2(gdtp, acc, dcp) : fma2(gdtp, acc, fma2(cap, dcp, mul2(cbp, tcp)));
                            out.ab[r][h] = atop;
                            out.pd[r][h] = mul2(hi2(qn), dcp);
                        }
                        out4[r] = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
                    }
                    float* op = outp + (size_t)(k - k0) * plane;
                    *reinterpret_cast<float4*>(op) = out4[0];
                    *reinterpret_cast<float4*>(op + g.Nx) = out4[1];
                    if constexpr (TC) {
                        // the upscale integration (Section 3.3): dz-weighted sums over the
                        // slab's layers of each coarse column's cells in these rows
                        const float dzk = lcp[2];
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const float4 v = out4[r];
                            if (NC == 1) {
                                tcs[r][0] += dzk * ((v.x + v.y) + (v.z + v.w));
                            } else {
                                tcs[r][0] += dzk * (v.x + v.y);
                                tcs[r][NC - 1] += dzk * (v.z + v.w);
                            }
                        }
                    }
                };
                // the layers in pairs (chunks hold whole coarse slabs of M = 2 or 4
                // layers); ring R + r holds plane k0 - 1 + r in slot (R + r) % NB with
                // parity ((R + r) / NB) & 1, the chunk's coarse slab Kr is the CTA's
                // slab S + Kr, in buffer (S + Kr) & 1
                {
                    int sc = s1, st = s2, su = (R + 3) % NB, pt = ((R + 2) / NB) & 1, pu = ((R + 3) / NB) & 1;
                    for (int k = k0; k < k1; k += 2) {
                        const int i = k & (M - 1), Sg = S + (k - k0) / M, bb = Sg & 1;
                        if (i == 0 && k > k0 && !fail && !mbar_wait(&built[bb], (Sg >> 1) & 1, A.wait_ns)) fail = true;
                        if (!fail && !mbar_wait(&full[st], pt, A.wait_ns)) fail = true;
                        if (!fail && !mbar_wait(&full[su], pu, A.wait_ns)) fail = true;
                        if (!fail) {
                            layer(k, i, bb, sc, st, S0, S1);
                            layer(k + 1, i + 1, bb, st, su, S1, S0);
                        }
                        // planes k and k + 1 are no longer needed by this thread; nor,
                        // after the slab's last layer, the slab's intermediates
                        mbar_arrive(&empty[sc]);
                        mbar_arrive(&empty[st]);
                        if (i + 1 == M - 1) {
                            if constexpr (TC) {
#pragma unroll
                                for (int r = 0; r < 2; ++r) {
                                    float* tp = sm + L::oTcb + (bb * TY + jl + r) * L::CX + cb0;
#pragma unroll
                                    for (int q = 0; q < NC; ++q) {
                                        tp[q] = tcs[r][q];
                                        tcs[r][q] = 0.f;
                                    }
                                }
                            }
                            mbar_arrive(&freed[bb]);
                        }
                        sc = su;
                        st = su + 1;
                        pt = pu;
                        if (st == NB) {
                            st = 0;
                            pt ^= 1;
                        }
                        su = st + 1;
                        pu = pt;
                        if (su == NB) {
                            su = 0;
                            pu ^= 1;
                        }
                    }
                    // the chunk's last ring (plane k1), which no layer releases
                    mbar_arrive(&empty[(R + nrings - 1) % NB]);
                }
                R += nrings;
                S += h.K1 - h.K0;
            }
            if (fail) *s_fail = 1;
        }
    }
    __syncthreads();
    if (warp == NCW && lane == 0) {
        // no copy may still be in flight when the CTA exits: wait for the last
        // phase issued on every ring slot and coarse buffer (already complete
        // unless a wait gave up)
        bool ok = true;
        for (int s = 0; s < NB && s < rings_issued; ++s) {
            const int last = s + NB * ((rings_issued - 1 - s) / NB);
            ok &= mbar_wait(&full[s], (last / NB) & 1, A.wait_ns);
        }
        for (int bb = 0; bb < 2 && bb < slabs_issued; ++bb) {
            const int last = bb + 2 * ((slabs_issued - 1 - bb) / 2);
            ok &= mbar_wait(&cfull[bb], (last >> 1) & 1, A.wait_ns);
        }
        if (!ok || *s_fail) atomicExch(A.err, MR_ERR_TIMEOUT);
    }
    if (DIVONLY && tid == 0 && !*s_fail) {
        float m = 0.f;
        for (int w = 0; w < NCW; ++w) m = fmaxf(m, red[w]);
        atomicMax(A.divmax, (unsigned long long)__double_as_longlong((double)m));
    }
}

// The coarse faces padded with their periodic images: U and W with one ghost
// row each side in y, V with one below and two above, all with four ghost
// columns each side in x, so that every coarse box of k_fused is in bounds and
// starts on a 16-byte boundary.  out: padded U, V, W one after the other, for
// the ny coarse rows from j0 of a domain of nyg rows (a y-slab: its padded
// rows come from the neighbouring slabs' rows).
__global__ void k_pad_coarse(const float* __restrict__ U, const float* __restrict__ V, const float* __restrict__ W,
                             float* __restrict__ out, int nx, int nyg, int nz, int j0, int ny)
{
    const int px = nx + 8;
    const size_t nU = (size_t)nz * (ny + 2) * px, nV = (size_t)nz * (ny + 3) * px, nW = (size_t)(nz + 1) * (ny + 2) * px;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nU + nV + nW;
         t += (size_t)gridDim.x * blockDim.x) {
        const float* src;
        size_t e;
        int rows;
        if (t < nU) { src = U; e = t; rows = ny + 2; }
        else if (t < nU + nV) { src = V; e = t - nU; rows = ny + 3; }
        else { src = W; e = t - nU - nV; rows = ny + 2; }
        const int x = (int)(e % px);
        const size_t zr = e / px;
        const int r = (int)(zr % rows), z = (int)(zr / rows);
        int I = x - 4, J = j0 + r - 1;
        I = I < 0 ? I + nx : (I >= nx ? I - nx : I);
        J = J < 0 ? J + nyg : (J >= nyg ? J - nyg : J);
        out[t] = src[((size_t)z * nyg + J) * nx + I];
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// Tensor maps of (buffer, shape, row and layer strides in floats, box),
// encoded once each.
bool map_fx3(CUtensorMap* out, const float* base, int d0, int d1, int d2, size_t s1, size_t s2, int b0, int b1,
             int b2)
{
    struct Entry { const float* p; long long d[8]; CUtensorMap m; };
    constexpr int kCache = 128;
    static Entry cache[kCache];
    static int n = 0, next = 0;
    static std::mutex mu;
    const long long key[8] = {d0, d1, d2, (long long)s1, (long long)s2, b0, b1, b2};
    {
        std::lock_guard<std::mutex> lock(mu);
        for (int q = 0; q < n; ++q)
            if (cache[q].p == base && !memcmp(cache[q].d, key, sizeof key)) {
                *out = cache[q].m;
                return true;
            }
    }
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
    cuuint64_t strides[2] = {(cuuint64_t)s1 * 4, (cuuint64_t)s2 * 4};
    cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    std::lock_guard<std::mutex> lock(mu);
    Entry& e = cache[n < kCache ? n++ : (next = (next + 1) % kCache)];
    e.p = base;
    memcpy(e.d, key, sizeof key);
    e.m = *out;
    return true;
}
// A contiguous [d2][d1][d0] array.
bool map_fx(CUtensorMap* out, const float* base, int d0, int d1, int d2, int b0, int b1, int b2)
{
    return map_fx3(out, base, d0, d1, d2, (size_t)d0, (size_t)d0 * d1, b0, b1, b2);
}

template <int M, int TY, int KIND, bool LF, bool TC = false>
cudaError_t launch_fl(const Grid<float>& g, const FusedInputs& in, const float* Tm1, const float* T, float* Tp1,
                      StepCoef c, int* err, unsigned long long* divmax, cudaStream_t st)
{
    using L = FL<M, TY, (KIND != 0)>;
    static unsigned long long attr = 0;                   // one bit per device
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_fused<M, TY, KIND, LF, TC>), (int)L::bytes, &attr);
    if (e != cudaSuccess) return e;
    if constexpr (L::RS) {
        // the register split inside the kernel adds up only to a launch of
        // exactly kRegLaunch registers per thread: refuse any other build
        static int regs = -1;
        if (regs < 0) {
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k_fused<M, TY, KIND, LF, TC>));
            if (e != cudaSuccess) return e;
            regs = fa.numRegs;
        }
        if (regs != kRegLaunch) return cudaErrorInvalidConfiguration;
    }
    FLMaps maps;
    memset(&maps, 0, sizeof maps);
    if (KIND == 0) {
        // per level: the tile's rows, single rows, four columns; the rows beyond
        // the y edges: [Nz][Nx] at layer stride hstride
        const float* lv[2] = {T, Tm1};
        CUtensorMap* mt[2] = {&maps.tn, &maps.tm};
        CUtensorMap* mr1[2] = {&maps.rn, &maps.rm};
        CUtensorMap* mx4[2] = {&maps.xn, &maps.xm};
        CUtensorMap* ms[2] = {&maps.sn, &maps.smp};
        CUtensorMap* mh[2] = {&maps.hn, &maps.hm};
        for (int q = 0; q < 2; ++q)
            if (!map_fx(mt[q], lv[q], g.Nx, g.Ny, g.Nz, kTX, TY, 1) || !map_fx(mr1[q], lv[q], g.Nx, g.Ny, g.Nz, kTX, 1, 1) ||
                !map_fx(mx4[q], lv[q], g.Nx, g.Ny, g.Nz, 4, TY, 1) ||
                !map_fx3(ms[q], in.hs[q], g.Nx, 1, g.Nz, (size_t)g.Nx, in.hstride, kTX, 1, 1) ||
                !map_fx3(mh[q], in.hn[q], g.Nx, 1, g.Nz, (size_t)g.Nx, in.hstride, kTX, 1, 1))
                return cudaErrorInvalidValue;
    }
    const int px = g.nx + 8;
    const float* pU = in.pad;
    const float* pV = pU + (size_t)g.nz * (g.ny + 2) * px;
    const float* pW = pV + (size_t)g.nz * (g.ny + 3) * px;
    if (!map_fx(&maps.lc, in.lc, kLCW, g.Nz, 1, kLCW, 1, 1) ||
        !map_fx(&maps.cu, pU, px, g.ny + 2, g.nz, L::BXC, L::NUR, 3) ||
        !map_fx(&maps.cv, pV, px, g.ny + 3, g.nz, L::BXC, L::NVR, 3) ||
        !map_fx(&maps.cw, pW, px, g.ny + 2, g.nz + 1, L::BXC, L::NUR, 2) ||
        !map_fx(&maps.sc, in.sc, kSCW, g.nz, 1, kSCW, 1, 1))
        return cudaErrorInvalidValue;
    // ~6 chunks per resident CTA, chunks of at most 96 dense layers
#ifndef MR_FUSED_WAVES
#define MR_FUSED_WAVES 6                  // compile-time override for tuning sweeps
#endif
    const int tpx = g.Nx / kTX, tiles = tpx * (g.Ny / TY);
    const int want = 152 * L::CTAS * MR_FUSED_WAVES;
    int chunks = max(1, min((want + tiles - 1) / tiles, g.nz));
    int kcs = (g.nz + chunks - 1) / chunks;
    kcs = max(1, min(kcs, 96 / M));
    chunks = (g.nz + kcs - 1) / kcs;      // every chunk holds at least one coarse slab
    const int nch = chunks * tiles;
    // the step: one CTA per resident slot, each stepping every gridDim.x-th
    // chunk; the reductions: one CTA per chunk
    int grid = nch;
    if (KIND == 0) {
        static int slots[64] = {};        // resident CTAs of this kernel on all SMs, per device
        int dev = 0;
        e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!slots[dev]) {
            int sms = 0, per = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fused<M, TY, KIND, LF, TC>, L::THREADS,
                                                              L::bytes);
            if (e != cudaSuccess) return e;
            if (per < 1) return cudaErrorInvalidConfiguration;
            slots[dev] = sms * per;
        }
        grid = min(nch, slots[dev]);
    }
    // the last round of chunks, which not every CTA gets, in sp parts of ps
    // slabs: sp minimises the slabs of the busiest CTA, counting each part's two
    // extra planes as half a slab
    int nfull = nch, sp = 1, ps = kcs;
    if (KIND == 0 && nch > grid && nch % grid) {
        const int F = nch / grid, rem = nch - F * grid;
        double best = 1e30;
        for (int q = 1; q <= kcs; ++q) {
            const int p = (kcs + q - 1) / q;
            const double cost = (double)((rem * q + grid - 1) / grid) * (p + 0.5);
            if (cost < best - 1e-9) {
                best = cost;
                sp = q;
                ps = p;
            }
        }
        nfull = F * grid;
    }
    FLArgs A;
    memset(&A, 0, sizeof A);
    A.g = g;
    A.Tp1 = Tp1;
    A.a = (float)c.a;
    A.b = (float)c.b;
    A.gdt = (float)c.gdt;
    A.kcs = kcs;
    A.nch = nfull + (nch - nfull) * sp;
    A.zch = chunks;
    A.tpx = tpx;
    A.nfull = nfull;
    A.sp = sp;
    A.ps = ps;
    A.err = err;
    A.divmax = divmax;
    memcpy(A.rx, in.rx12, sizeof A.rx);
    memcpy(A.ry, in.ry12, sizeof A.ry);
    A.iDX = (float)(1.0 / (double)g.DX);
    A.iDY = (float)(1.0 / (double)g.DY);
    A.hx = g.hx;
    A.hy = g.hy;
    A.wait_ns = ptx::kWaitNs;
    A.stop_ring = -1;
    if (KIND == 0) {
        take_wait_injection(&A.stop_ring, &A.wait_ns);
        A.Tc = in.Tc;
        A.tcinv = in.tcinv;
    }
    k_fused<M, TY, KIND, LF, TC><<<grid, L::THREADS, L::bytes, st>>>(maps, A);
    return cudaGetLastError();
}

// The step on 64x16 tiles at M = 4 (two CTAs per SM; measured on 512 x 512 x
// 384: 0.432 ms per step against 0.491 on 64x8 tiles, on 1536 x 1536 x 1024
// 8.77 against 10.2 ms), on 64x8 tiles at M = 2 (its 64x16 layout would not
// fit two CTAs per SM); the reductions, which stream no scalar, on 64x8 tiles.
template <int KIND, bool LF, bool TC>
cudaError_t launch_fl_any(const Grid<float>& g, const FusedInputs& in, const float* Tm1, const float* T, float* Tp1,
                          StepCoef c, int* err, unsigned long long* divmax, cudaStream_t st)
{
    if (g.mx == 2) return launch_fl<2, 8, KIND, LF, TC>(g, in, Tm1, T, Tp1, c, err, divmax, st);
    if constexpr (KIND == 0) return launch_fl<4, 16, KIND, LF, TC>(g, in, Tm1, T, Tp1, c, err, divmax, st);
    else return launch_fl<4, 8, KIND, LF, TC>(g, in, Tm1, T, Tp1, c, err, divmax, st);
}

// The same padding from the FP64 coarse faces, rounding them to FP32 once;
// on a whole-domain grid (j0 = 0, ny = nyg) the interior of the padded copy
// also goes to the unpadded FP32 faces U32, V32, W32 (one pass instead of a
// conversion and a padding).
__global__ void k_pad_coarse64(const double* __restrict__ U, const double* __restrict__ V,
                               const double* __restrict__ W, float* __restrict__ out, float* __restrict__ U32,
                               float* __restrict__ V32, float* __restrict__ W32, int nx, int nyg, int nz, int j0,
                               int ny)
{
    const int px = nx + 8;
    const size_t nU = (size_t)nz * (ny + 2) * px, nV = (size_t)nz * (ny + 3) * px, nW = (size_t)(nz + 1) * (ny + 2) * px;
    const bool whole = (j0 == 0 && ny == nyg);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < nU + nV + nW;
         t += (size_t)gridDim.x * blockDim.x) {
        const double* src;
        float* dst;
        size_t e;
        int rows;
        if (t < nU) { src = U; dst = U32; e = t; rows = ny + 2; }
        else if (t < nU + nV) { src = V; dst = V32; e = t - nU; rows = ny + 3; }
        else { src = W; dst = W32; e = t - nU - nV; rows = ny + 2; }
        const int x = (int)(e % px);
        const size_t zr = e / px;
        const int r = (int)(zr % rows), z = (int)(zr / rows);
        int I = x - 4, J = j0 + r - 1;
        const bool interior = (I >= 0 && I < nx && J >= 0 && J < nyg && r >= 1 && r <= ny);
        I = I < 0 ? I + nx : (I >= nx ? I - nx : I);
        J = J < 0 ? J + nyg : (J >= nyg ? J - nyg : J);
        const size_t m = ((size_t)z * nyg + J) * nx + I;
        const float v = (float)src[m];
        out[t] = v;
        if (whole && interior) dst[m] = v;
    }
}

// The plate Nusselt numbers of a new level (Section 4.1) in one launch: each
// of kCRNu blocks adds the conductive fluxes of a fixed set of plate cells in
// FP64 and stores its two sums; the last to finish (an atomic count) adds them
// in a fixed order -- so the result never changes from run to run -- and
// resets the count.
constexpr int kCRThreads = 256, kCRNu = 304;
__device__ __forceinline__ void cr_block_sum(double& a, double& b, double (*s)[kCRThreads / 32])
{
    for (int d = 16; d > 0; d >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, d);
        b += __shfl_down_sync(0xffffffffu, b, d);
    }
    if ((threadIdx.x & 31) == 0) {
        s[0][threadIdx.x >> 5] = a;
        s[1][threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int w = 0; w < kCRThreads / 32; ++w) {
            a += s[0][w];
            b += s[1][w];
        }
    }
}
__device__ __forceinline__ void cr_plate_nu(const float* __restrict__ T, size_t plane, size_t top, double izb,
                                            double izt, double inv_plane, double* __restrict__ work,
                                            double* __restrict__ nu2, unsigned nb)
{
    double a = 0.0, b = 0.0;
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < plane; m += (size_t)nb * blockDim.x) {
        a += 0.5 - (double)T[m];
        b += (double)T[top + m] + 0.5;
    }
    __shared__ double s[2][kCRThreads / 32];
    __shared__ bool last;
    unsigned* count = reinterpret_cast<unsigned*>(work);
    double* part = work + 1;
    cr_block_sum(a, b, s);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = b;
        __threadfence();                     // this block's sums before its count
        last = atomicAdd(count, 1u) == nb - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    a = 0.0;
    b = 0.0;
    for (unsigned q = threadIdx.x; q < nb; q += blockDim.x) {
        a += __ldcg(part + 2 * q);
        b += __ldcg(part + 2 * q + 1);
    }
    __syncthreads();                         // s is reused
    cr_block_sum(a, b, s);
    if (threadIdx.x == 0) {
        nu2[0] = a * izb * inv_plane;
        nu2[1] = b * izt * inv_plane;
        *count = 0u;
    }
}
__global__ void __launch_bounds__(kCRThreads)
k_coupled_nu(const float* __restrict__ T, size_t plane, size_t top, double izb, double izt, double inv_plane,
             double* __restrict__ work, double* __restrict__ nu2)
{
    cr_plate_nu(T, plane, top, izb, izt, inv_plane, work, nu2, gridDim.x);
}

}  // namespace

cudaError_t launch_fused_pad64(const double* U, const double* V, const double* W, float* out, float* U32, float* V32,
                               float* W32, int nx, int nyg, int nz, int j0, int ny, cudaStream_t st)
{
    const size_t n = fused_pad_floats(nx, ny, nz);
    const size_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    k_pad_coarse64<<<blocks, 256, 0, st>>>(U, V, W, out, U32, V32, W32, nx, nyg, nz, j0, ny);
    return cudaGetLastError();
}

cudaError_t launch_fused_plate_nu(const Grid<float>& g, const float* T, double izb, double izt, double* work,
                                  double* nu2, cudaStream_t st)
{
    const size_t plane = (size_t)g.Nx * g.Ny;
    const unsigned blocks = (unsigned)std::min((plane + kCRThreads - 1) / kCRThreads, (size_t)kCRNu);
    k_coupled_nu<<<blocks, kCRThreads, 0, st>>>(T, plane, (size_t)(g.Nz - 1) * plane, izb, izt, 1.0 / (double)plane,
                                               work, nu2);
    return cudaGetLastError();
}

size_t fused_plate_nu_work() { return 1 + 2 * (size_t)kCRNu; }

size_t fused_pad_floats(int nx, int ny, int nz)
{
    const size_t px = (size_t)nx + 8;
    return (size_t)nz * (ny + 2) * px + (size_t)nz * (ny + 3) * px + (size_t)(nz + 1) * (ny + 2) * px;
}

cudaError_t launch_fused_pad(const float* U, const float* V, const float* W, float* out, int nx, int nyg, int nz,
                             int j0, int ny, cudaStream_t st)
{
    const size_t n = fused_pad_floats(nx, ny, nz);
    const size_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    k_pad_coarse<<<blocks, 256, 0, st>>>(U, V, W, out, nx, nyg, nz, j0, ny);
    return cudaGetLastError();
}

// Per coarse slab K, 32 floats (FP64 on the host, rounded once): the R_z rows
// of its M dense layers (3M), 1/(2 dz) of each (M), and the stage-Z weights
// Z[c][q] = sum_{c' = c}^{M-1} dz_{KM+c'} R_z[KM+c'][q], c = 1 .. M-1 (3(M-1)).
std::vector<float> fused_slab_constants(int nz, int M, const double* Rz, const double* dz)
{
    std::vector<float> t((size_t)nz * kSCW, 0.f);
    for (int K = 0; K < nz; ++K) {
        float* q = &t[(size_t)K * kSCW];
        for (int i = 0; i < M; ++i) {
            const int k = K * M + i;
            for (int c = 0; c < 3; ++c) q[3 * i + c] = (float)Rz[3 * (size_t)k + c];
            q[3 * M + i] = (float)(0.5 / dz[k]);
        }
        for (int c = 1; c < M; ++c)
            for (int r = 0; r < 3; ++r) {
                double s = 0.0;
                for (int cc = c; cc < M; ++cc) s += dz[K * M + cc] * Rz[3 * (size_t)(K * M + cc) + r];
                q[4 * M + 3 * (c - 1) + r] = (float)s;
            }
    }
    return t;
}

cudaError_t launch_step_fused_f32(const Grid<float>& g, const FusedInputs& in, const float* Tm1, const float* T,
                                  float* Tp1, StepCoef c, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    const bool lf = (c.a == 1.0 && c.b == 0.0);
    if (in.Tc)
        return lf ? launch_fl_any<0, true, true>(g, in, Tm1, T, Tp1, c, err, nullptr, st)
                  : launch_fl_any<0, false, true>(g, in, Tm1, T, Tp1, c, err, nullptr, st);
    return lf ? launch_fl_any<0, true, false>(g, in, Tm1, T, Tp1, c, err, nullptr, st)
              : launch_fl_any<0, false, false>(g, in, Tm1, T, Tp1, c, err, nullptr, st);
}

cudaError_t launch_fused_max_f32(const Grid<float>& g, int kind, const FusedInputs& in, double* partials, int blocks,
                                 cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(partials, 0, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return e;
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(partials);
    const StepCoef c{0, 0, 0};
    return kind == 2 ? launch_fl_any<2, false, false>(g, in, nullptr, nullptr, nullptr, c, err, dm, st)
                     : launch_fl_any<1, false, false>(g, in, nullptr, nullptr, nullptr, c, err, dm, st);
}

// Raise a kernel's dynamic shared-memory limit once per device; *done holds
// one bit per device index.
cudaError_t smem_optin(const void* kernel, int bytes, unsigned long long* done)
{
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (*done >> dev & 1ull) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) *done |= 1ull << dev;
    return e;
}

bool fused_supported(const mr_config& cfg, std::string* why)
{
    if (cfg.precision != MR_F32) { *why = "MR_VEL_FUSED needs MR_F32"; return false; }
    if (cfg.bc_horizontal != MR_PERIODIC) { *why = "MR_VEL_FUSED needs periodic x and y"; return false; }
    if (cfg.mx != cfg.my || cfg.my != cfg.mz || (cfg.mx != 2 && cfg.mx != 4)) {
        *why = "MR_VEL_FUSED needs mx = my = mz in {2, 4}";
        return false;
    }
    if ((cfg.nx * cfg.mx) % kTX || (cfg.ny * cfg.my) % 16) {
        *why = "MR_VEL_FUSED needs Nx % 64 == 0 and Ny % 16 == 0";
        return false;
    }
    if (cfg.diffz_implicit) { *why = "MR_VEL_FUSED does not support diffz_implicit"; return false; }
    if (!encode_fn()) { *why = "cuTensorMapEncodeTiled unavailable"; return false; }
    return true;
}

// Device error flag of the fused kernels (MR_ERR_TIMEOUT after a bounded wait
// gave up).  One per device, allocated on first use; read and cleared by
// fused_take_error on the caller's stream.
static int* g_err[64] = {};
static std::mutex g_err_mu;

static int** err_slot()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    return &g_err[dev];
}

int* fused_error_flag()
{
    std::lock_guard<std::mutex> lock(g_err_mu);
    int** slot = err_slot();
    if (!slot) return nullptr;
    if (!*slot) {
        int* p = nullptr;
        if (dev_malloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) { dev_free(p); return nullptr; }
        *slot = p;
    }
    return *slot;
}

int fused_take_error(cudaStream_t st)
{
    int* flag = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_err_mu);
        int** slot = err_slot();
        if (slot) flag = *slot;
    }
    if (!flag) return 0;
    int v = 0;
    if (cudaMemcpyAsync(&v, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MR_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MR_ERR_CUDA;
    if (v) cudaMemsetAsync(flag, 0, sizeof(int), st);
    return v;
}

}  // namespace mr
