// MR_VEL_FUSED: the FP32 step kernel with every stage of the refinement
// (Section 3.2) inside it, from the coarse faces.  The refined velocity, and
// every intermediate of the refinement, lives in shared memory and registers
// only; per step the kernel reads the coarse faces, T^s and T^{s-1} and
// writes T^{s+1}.
//
// One CTA owns a 64 x 8 column of dense cells and marches a chunk of coarse
// slabs.  At the start of each slab K its 128 consumer threads compute, from
// the coarse U, V, W (global, L1/L2-resident), the slab's refinement stages at
// coarse resolution in x, for the tile's rows and the bundle columns
// I0-4 .. I0+CX+3 (periodic images):
//   - stage Z: the slab balance of every coarse column (full-area W on the
//     slab's inner dense planes), top-down;
//   - WY: R_y of the full-area W on the slab's M+1 dense planes;
//   - UO: the outer U sub-faces (R_y R_z of U) in units of U / (2 dx);
//   - VR: the full-coarse-width V on every dense y-face of the tile (R_z of V
//     on the coarse faces, row balance of stage Y on the inner ones) in units
//     of V / (2 dy);
// separated by consumer-only barriers.  Each dense layer then runs exactly the
// split-x step (stage X -- R_x splits and the west-to-east cell balance -- in
// registers, then the finite-volume update of Eq. 5 with the Euler-leapfrog
// coefficients of Section 2.2), with T^s, T^{s-1} and the layer constants
// streamed by one producer warp through a TMA ring on full/empty mbarriers.
// Every wait is bounded: on time-out the kernel records MR_ERR_TIMEOUT in a
// device flag.
//
// Supported: FP32, periodic x and y, mx = my = mz = M in {2, 4},
// Nx % 64 == 0, Ny % 16 == 0, explicit diffusion, second-order faces.
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "mr_internal.cuh"
#include "mr_ptx.cuh"

namespace mr {
namespace {

using namespace ptx;

constexpr int kTX = 64, kTY = 8;                        // tile (cells)
constexpr int kBX = kTX + 8, kBY = kTY + 2;             // scalar plane box (floats)
constexpr int kCons = 16 * kTY;                         // consumer threads: 4-cell segments
constexpr int kThreadsAll = kCons + 32;                 // + one producer warp
constexpr int kLCW = 32;                                // layer-constant row (floats)

template <int M>
struct FX {
    static constexpr int CX = kTX / M, CY = kTY / M;    // coarse cells of the tile
    static constexpr int BXC = CX + 8;                  // bundle columns I0-4 .. I0+CX+3
    static constexpr int NB = 6;                        // ring slots
    static constexpr uint32_t plane_bytes = (uint32_t)(kBX * kBY) * 4;
    static constexpr int PS = (int)((plane_bytes + 127) / 128) * 128 / 4;
    // ring slot (floats): T^s plane, T^{s-1} plane, the layer constants
    static constexpr int oTn = 0, oTm = PS, oLC = 2 * PS;
    static constexpr int slot = (((oLC + kLCW) * 4 + 127) / 128) * 128 / 4;
    // the slab's intermediates: WY [M+1][TY][BXC], UO [M][TY][BXC],
    // VR [M][TY+1][BXC], and the slab balance [M-1][CY+2][BXC]
    static constexpr int oWY = NB * slot;
    static constexpr int oUO = oWY + (M + 1) * kTY * BXC;
    static constexpr int oVR = oUO + M * kTY * BXC;
    static constexpr int oSW = oVR + M * (kTY + 1) * BXC;
    // the slab's coarse faces (periodic images), staged by cp.async: U on the
    // three R_z window planes, coarse rows J0-1 .. J0+CY, columns I0-4 .. I0+CX+4;
    // V likewise with rows up to J0+CY+1; W on the slab's two coarse planes
    static constexpr int NUX = BXC + 1, NUY = CY + 2, NVY = CY + 3, NWY = CY + 2;
    static constexpr int NU = 3 * NUY * NUX, NV = 3 * NVY * BXC, NW = 2 * NWY * BXC;
    static constexpr int oSU = oSW + (M - 1) * (CY + 2) * BXC;
    static constexpr int oSV = oSU + NU;
    static constexpr int oSWc = oSV + NV;
    // R_y rows of the tile's dense rows [TY][3]; R_z rows and widths of the slab's layers
    static constexpr int oRy = oSWc + NW;
    static constexpr int oRz = oRy + 3 * kTY;
    static constexpr int oDz = oRz + 3 * M;
    static constexpr int oRed = (oDz + M + 3) / 4 * 4;
    static constexpr int oBar = ((oRed + 64) * 4 + 7) / 8;
    static constexpr size_t bytes = (size_t)(oBar + 2 * NB) * 8;
};

struct FXArgs {
    Grid<float> g;
    const float* U;      // coarse faces, FP32: [nz][ny][nx]
    const float* V;      // [nz][ny][nx]
    const float* W;      // [nz+1][ny][nx]
    const float* Tn;     // T^s (global, for the periodic halo of edge threads)
    const float* Tm;     // T^{s-1}
    float* Tp1;          // T^{s+1}
    float a, b, gdt;
    int kcs;             // coarse slabs per CTA chunk
    int* err;
    unsigned long long* divmax;
    float rx[4][3];      // R_x rows of the 4 cells of a segment (uniform periodic x)
    unsigned long long wait_ns;   // time limit of every bounded wait
    int stop_ring;       // test hook: the producer of CTA (0,0,0) issues no ring from this one on (-1: none)
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

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

// The slab's refinement intermediates (see the file comment), written by the
// kCons consumer threads from the coarse faces staged in shared memory; ends
// with every value visible to all of them.
template <int M>
__device__ void slab_prep(const FXArgs& A, float* sm, int K, int I0, int J0, int j0, int tid)
{
    using L = FX<M>;
    constexpr int BXC = L::BXC, CY = L::CY, NUX = L::NUX, NUY = L::NUY, NVY = L::NVY, NWY = L::NWY;
    const Grid<float>& g = A.g;
    float* sWY = sm + L::oWY;
    float* sUO = sm + L::oUO;
    float* sVR = sm + L::oVR;
    float* sSW = sm + L::oSW;
    float* sU = sm + L::oSU;
    float* sV = sm + L::oSV;
    float* sW = sm + L::oSWc;
    const size_t cpl = (size_t)g.ny * g.nx;                 // coarse plane
    // stage the coarse faces: U, V on the R_z window planes of K, W on K, K+1
#pragma unroll 4
    for (int u = 0; u < (L::NU + kCons - 1) / kCons; ++u) {
        const int t = tid + u * kCons;
        if (t < L::NU) {
            const int q = t / (NUY * NUX), r = t - q * NUY * NUX, jr = r / NUX, xc = r - jr * NUX;
            const int I = wrapi(I0 - 4 + xc, g.nx), J = wrapi(J0 - 1 + jr, g.ny);
            cp_async4(sU + t, A.U + (size_t)g.wz[3 * K + q] * cpl + (size_t)J * g.nx + I);
        }
    }
#pragma unroll 4
    for (int u = 0; u < (L::NV + kCons - 1) / kCons; ++u) {
        const int t = tid + u * kCons;
        if (t < L::NV) {
            const int q = t / (NVY * BXC), r = t - q * NVY * BXC, jr = r / BXC, xc = r - jr * BXC;
            const int I = wrapi(I0 - 4 + xc, g.nx), J = wrapi(J0 - 1 + jr, g.ny);
            cp_async4(sV + t, A.V + (size_t)g.wz[3 * K + q] * cpl + (size_t)J * g.nx + I);
        }
    }
#pragma unroll 4
    for (int u = 0; u < (L::NW + kCons - 1) / kCons; ++u) {
        const int t = tid + u * kCons;
        if (t < L::NW) {
            const int q = t / (NWY * BXC), r = t - q * NWY * BXC, jr = r / BXC, xc = r - jr * BXC;
            const int I = wrapi(I0 - 4 + xc, g.nx), J = wrapi(J0 - 1 + jr, g.ny);
            cp_async4(sW + t, A.W + (size_t)(K + q) * cpl + (size_t)J * g.nx + I);
        }
    }
    if (tid < 3 * M) sm[L::oRz + tid] = g.Rz[3 * K * M + tid];
    if (tid < M) sm[L::oDz + tid] = g.dz[K * M + tid];
    cp_async_commit();
    cp_async_wait_all();
    asm volatile("barrier.cta.sync 1, %0;" ::"n"(kCons) : "memory");
    const float* sRy = sm + L::oRy;
    const float* sRz = sm + L::oRz;
    const float* sDz = sm + L::oDz;
    // stage Z: slab balance of every coarse column, top-down (full-area W on
    // the inner dense planes K M + c, c = M-1 .. 1), coarse rows J0-1 .. J0+CY
    for (int t = tid; t < (CY + 2) * BXC; t += kCons) {
        const int jr = t / BXC, xb = t - jr * BXC;
        float F = sW[(NWY + jr) * BXC + xb] * g.DX * g.DY;      // W on coarse plane K+1
#pragma unroll
        for (int c = M - 1; c >= 1; --c) {
            float uw = 0.f, ue = 0.f, vs = 0.f, vn = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float r = sRz[3 * c + q];
                uw += r * sU[(q * NUY + jr) * NUX + xb];
                ue += r * sU[(q * NUY + jr) * NUX + xb + 1];
                vs += r * sV[(q * NVY + jr) * BXC + xb];
                vn += r * sV[(q * NVY + jr + 1) * BXC + xb];
            }
            F = F + (ue - uw) * g.DY * sDz[c] + (vn - vs) * g.DX * sDz[c];
            sSW[((c - 1) * (CY + 2) + jr) * BXC + xb] = F / (g.DX * g.DY);
        }
    }
    asm volatile("barrier.cta.sync 1, %0;" ::"n"(kCons) : "memory");
    // WY on the slab's M + 1 dense planes, per (dense row, bundle column)
    for (int e = tid; e < kTY * BXC; e += kCons) {
        const int jl = e / BXC, xb = e - jl * BXC;
        const int jr = (j0 + jl) / M - J0;                         // coarse row, relative to J0
        const float r0 = sRy[3 * jl], r1 = sRy[3 * jl + 1], r2 = sRy[3 * jl + 2];
#pragma unroll
        for (int i = 0; i <= M; ++i) {
            const float* src = (i == 0 || i == M) ? sW + (i == M ? NWY : 0) * BXC : sSW + (i - 1) * (CY + 2) * BXC;
            const float c0 = src[jr * BXC + xb], c1 = src[(jr + 1) * BXC + xb], c2 = src[(jr + 2) * BXC + xb];
            sWY[(i * kTY + jl) * BXC + xb] = r0 * c0 + r1 * c1 + r2 * c2;
        }
    }
    // UO of the slab's M layers, per (coarse row, bundle column): the z split
    // of the three window rows is shared by the row's M dense rows
    const float hix = 0.5f * g.inv_dx;
    for (int e = tid; e < CY * BXC; e += kCons) {
        const int Jr = e / BXC, xb = e - Jr * BXC;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float a[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) s += sRz[3 * i + q] * sU[(q * NUY + Jr + p) * NUX + xb];
                a[p] = s;
            }
#pragma unroll
            for (int b = 0; b < M; ++b) {
                const int jl = Jr * M + b;
                sUO[(i * kTY + jl) * BXC + xb] =
                    (sRy[3 * jl] * a[0] + sRy[3 * jl + 1] * a[1] + sRy[3 * jl + 2] * a[2]) * hix;
            }
        }
    }
    asm volatile("barrier.cta.sync 1, %0;" ::"n"(kCons) : "memory");
    // VR: per layer and coarse row J0 .. J0+CY, the coarse face from R_z of V,
    // then (rows inside the tile) the row balance, south to north; the last
    // bundle column is never read and is skipped (its east neighbour is absent)
    const float hiy = 0.5f * g.inv_dy, two_dx = 2.f * g.dx;
    for (int e = tid; e < (CY + 1) * (BXC - 1); e += kCons) {
        const int Jr = e / (BXC - 1), xb = e - Jr * (BXC - 1);
#pragma unroll
        for (int i = 0; i < M; ++i) {
            float vz = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) vz += sRz[3 * i + q] * sV[(q * NVY + Jr + 1) * BXC + xb];
            float* vr = sVR + (i * (kTY + 1) + Jr * M) * BXC + xb;
            vr[0] = vz * hiy;
            if (Jr < CY) {
                const float dzk = sDz[i];
                const float* uo = sUO + (i * kTY + Jr * M) * BXC + xb;
                const float* wyb = sWY + (i * kTY + Jr * M) * BXC + xb;
                const float* wyt = wyb + kTY * BXC;
                float G = vz * g.DX * dzk;
#pragma unroll
                for (int b = 0; b < M - 1; ++b) {
                    const float uw = uo[b * BXC] * two_dx, ue = uo[b * BXC + 1] * two_dx;
                    G = G - (ue - uw) * g.dy * dzk - (wyt[b * BXC] - wyb[b * BXC]) * g.DX * g.dy;
                    vr[(b + 1) * BXC] = G / (g.DX * dzk) * hiy;
                }
            }
        }
    }
    asm volatile("barrier.cta.sync 1, %0;" ::"n"(kCons) : "memory");
}

// KIND 0: the step; 1: max |divergence| of the dense velocity; 2: max CFL rate.
// LF: a plain leapfrog step (a = 1, b = 0).
template <int M, int KIND, bool LF>
__global__ void __launch_bounds__(kThreadsAll, 4)
k_fused(const __grid_constant__ CUtensorMap tmn, const __grid_constant__ CUtensorMap tmm,
         const __grid_constant__ CUtensorMap tlc, const FXArgs A)
{
    using L = FX<M>;
    constexpr int NB = L::NB, BXC = L::BXC, NC = 4 / M, NW = kCons / 32;
    constexpr bool DIVONLY = KIND != 0;
    extern __shared__ __align__(128) float sm[];
    float* red = sm + L::oRed;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm) + L::oBar;
    uint64_t* empty = full + NB;

    const Grid<float>& g = A.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * kTX, j0 = blockIdx.z * kTY;
    const int I0 = i0 / M, J0 = j0 / M;
    const int K0 = blockIdx.x * A.kcs, K1 = min(K0 + A.kcs, g.nz);
    if (K0 >= K1) return;
    const int k0 = K0 * M, k1 = K1 * M;
    const int nrings = k1 - k0 + 2;              // ring r: plane k0-1+r and the constants of layer k0+r-2

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kCons);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---------------------------------------------------------------- producer warp
    if (warp == NW) {
        if (lane != 0) return;
        const bool stopper = (A.stop_ring >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
        for (int r = 0; r < nrings; ++r) {
            const int s = r % NB;
            if (stopper && r == A.stop_ring) break;  // every ring issued so far is waited for by the consumers
            if (r >= NB && !mbar_wait(&empty[s], ((r / NB) - 1) & 1, A.wait_ns)) {
                atomicExch(A.err, MR_ERR_TIMEOUT);   // consumers then time out on full[]
                break;
            }
            float* slot = sm + s * L::slot;
            const int p = k0 - 1 + r;
            const bool lc = (r >= 2);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&full[s], (DIVONLY ? 0u : 2 * L::plane_bytes) + (lc ? (uint32_t)kLCW * 4 : 0u));
            if (!DIVONLY) {
                tma_3d(slot + L::oTn, &tmn, i0 - 4, j0 - 1, p, &full[s]);
                tma_3d(slot + L::oTm, &tmm, i0 - 4, j0 - 1, p, &full[s]);
            }
            if (lc) tma_3d(slot + L::oLC, &tlc, 0, p - 1, 0, &full[s]);
        }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    // this thread's 4-cell segment of dense row jl (half-warps on rows two apart)
    const int seg = tid & 15, jl = ((warp >> 1) << 2) + (warp & 1) + 2 * ((tid >> 4) & 1);
    const int il0 = seg * 4, cb0 = il0 / M;      // first coarse column of the segment (tile-local)
    const auto& rx = A.rx;
    const bool wrap_w = (i0 == 0 && seg == 0), wrap_e = (i0 + kTX == g.Nx && seg == 15);
    const bool wrap_s = (j0 == 0 && jl == 0), wrap_n = (j0 + kTY == g.Ny && jl == kTY - 1);

    bool fail = false;
    float dmax = 0.f;
    const float kx2 = g.kx2, ky2 = g.ky2;
    const float ca = A.a, cbb = A.b, gdt = A.gdt;
    const float2 kx2p = make_float2(kx2, kx2), ky2p = make_float2(ky2, ky2), gdtp = make_float2(gdt, gdt);
    const float2 cap = make_float2(ca, ca), cbp = make_float2(cbb, cbb);
    // PK: the update runs on packed pairs of cells (0, 1), (2, 3); vn then holds
    // the negated V split, the sign its flux enters with
    constexpr bool PK = !DIVONLY;
    const size_t plane = (size_t)g.Nx * g.Ny;
    float* outp = A.Tp1 + (size_t)k0 * plane + (size_t)(j0 + jl) * g.Nx + i0 + il0;
    const int o = (jl + 1) * kBX + il0 + 4;      // this segment's first cell in a plane box
    const float* sWY = sm + L::oWY;
    const float* sUO = sm + L::oUO;
    const float* sVR = sm + L::oVR;

    if (tid < 3 * kTY) sm[L::oRy + tid] = g.Ry[3 * j0 + tid];   // the tile's R_y rows (read after a barrier)
    float wcar[4] = {0.f, 0.f, 0.f, 0.f};        // R_x split of W on plane k (from layer k-1)
    // rings 0 and 1 (planes k0-1, k0) before the layer loop; then layer k waits
    // for the ring of plane k+1 only
    for (int r = 0; r < 2; ++r)
        if (!fail && !mbar_wait(&full[r], 0, A.wait_ns)) fail = true;
    // one layer; sb, sc, st: the ring slots of planes k-1, k, k+1, tpar: the
    // parity of the ring of plane k+1
    auto layer = [&](const int k, const int sb, const int sc, const int st, const int tpar) {
        const int K = k / M, i = k - K * M;
        if (i == 0) {
            // the previous slab's intermediates are no longer read: build this slab's
            asm volatile("barrier.cta.sync 1, %0;" ::"n"(kCons) : "memory");
            slab_prep<M>(A, sm, K, I0, J0, j0, tid);
        }
        // the ring of plane k+1 and of this layer's constants
        if (!fail && !mbar_wait(&full[st], tpar, A.wait_ns)) fail = true;
        if (!fail) {
            const float* lcp = sm + st * L::slot + L::oLC;
            const float2 c0 = *reinterpret_cast<const float2*>(lcp);
            const float inv_dz = c0.x, hz = c0.y;
            float wb[4], wt[4], vs[4], vn[4], us[5];
            {
                // R_x splits of the full-width W (planes k, k+1) and V (faces jl, jl+1)
                const float* yb = sWY + (i * kTY + jl) * BXC + cb0 + 3;
                const float* yt = yb + kTY * BXC;
                const float* rs = sVR + (i * (kTY + 1) + jl) * BXC + cb0 + 3;
                const float* rn = rs + BXC;
                const float* ur = sUO + (i * kTY + jl) * BXC + cb0 + 4;   // outer face of coarse column cb0
                constexpr int NV = NC + 2;
                float ytv[NV], rsv[NV], rnv[NV], urv[NC + 1];
                if (k == k0) {
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
                    vn[a] = PK ? nrsplit3(rx[a], rnv[cb], rnv[cb + 1], rnv[cb + 2])
                               : rsplit3(rx[a], rnv[cb], rnv[cb + 1], rnv[cb + 2]);
                }
                // stage X: cell balance, west to east, in units of U / (2 dx)
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    float h = urv[q];
                    us[q * M] = h;
#pragma unroll
                    for (int a = 0; a < M - 1; ++a) {
                        const int m = q * M + a;
                        h = (PK ? h + (vn[m] + vs[m]) : h - (vn[m] - vs[m])) - (wt[m] - wb[m]) * hz;
                        us[m + 1] = h;
                    }
                }
                us[4] = urv[NC];
#pragma unroll
                for (int a = 0; a < 4; ++a) wcar[a] = wt[a];
            }
            if (DIVONLY) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float d = KIND == 2 ? 2.f * (fmaxf(fabsf(us[a]), fabsf(us[a + 1])) + fmaxf(fabsf(vs[a]), fabsf(vn[a]))) +
                                                    fmaxf(fabsf(wb[a]), fabsf(wt[a])) * inv_dz
                                              : 2.f * ((us[a + 1] - us[a]) + (vn[a] - vs[a])) + (wt[a] - wb[a]) * inv_dz;
                    dmax = fmaxf(dmax, fabsf(d));
                }
            } else {
                const float* Pn_b = sm + sb * L::slot + L::oTn;
                const float* Pm_b = sm + sb * L::slot + L::oTm;
                const float* Pn_c = sm + sc * L::slot + L::oTn;
                const float* Pm_c = sm + sc * L::slot + L::oTm;
                const float* Pn_t = sm + st * L::slot + L::oTn;
                const float* Pm_t = sm + st * L::slot + L::oTm;
                const float4 tc4 = *reinterpret_cast<const float4*>(Pn_c + o);
                float4 ts4 = *reinterpret_cast<const float4*>(Pn_c + o - kBX);
                float4 tn4 = *reinterpret_cast<const float4*>(Pn_c + o + kBX);
                const float4 dc4 = *reinterpret_cast<const float4*>(Pm_c + o);
                float4 ds4 = *reinterpret_cast<const float4*>(Pm_c + o - kBX);
                float4 dn4 = *reinterpret_cast<const float4*>(Pm_c + o + kBX);
                float tw = __shfl_up_sync(0xffffffffu, tc4.w, 1), te = __shfl_down_sync(0xffffffffu, tc4.x, 1);
                float dw = __shfl_up_sync(0xffffffffu, dc4.w, 1), de = __shfl_down_sync(0xffffffffu, dc4.x, 1);
                if (seg == 0) { tw = Pn_c[o - 1]; dw = Pm_c[o - 1]; }
                if (seg == 15) { te = Pn_c[o + 4]; de = Pm_c[o + 4]; }
                if (wrap_w | wrap_e | wrap_s | wrap_n) {
                    // the box holds zeros beyond the domain: fetch the periodic images
                    const float* gn = A.Tn + (size_t)k * plane;
                    const float* gm = A.Tm + (size_t)k * plane;
                    const size_t row = (size_t)(j0 + jl) * g.Nx;
                    if (wrap_w) { tw = gn[row + g.Nx - 1]; dw = gm[row + g.Nx - 1]; }
                    if (wrap_e) { te = gn[row]; de = gm[row]; }
                    if (wrap_s) {
                        const size_t r2 = (size_t)(g.Ny - 1) * g.Nx + i0 + il0;
                        ts4 = *reinterpret_cast<const float4*>(gn + r2);
                        ds4 = *reinterpret_cast<const float4*>(gm + r2);
                    }
                    if (wrap_n) {
                        tn4 = *reinterpret_cast<const float4*>(gn + i0 + il0);
                        dn4 = *reinterpret_cast<const float4*>(gm + i0 + il0);
                    }
                }
                // planes below / above: zero-filled beyond the plates, where W is zero
                // and the plate value enters D through `plate`
                const float4 tb4 = *reinterpret_cast<const float4*>(Pn_b + o);
                const float4 db4 = *reinterpret_cast<const float4*>(Pm_b + o);
                const float4 tt4 = *reinterpret_cast<const float4*>(Pn_t + o);
                const float4 dt4 = *reinterpret_cast<const float4*>(Pm_t + o);
                const float tcv[6] = {tw, tc4.x, tc4.y, tc4.z, tc4.w, te};
                const float dcv[6] = {dw, dc4.x, dc4.y, dc4.z, dc4.w, de};
                // x fluxes in scalar form (adjacent cells share a face), then the
                // rest on the pairs (0, 1), (2, 3) with the pair constants of the row:
                // D = kx2 (dw + de) + ky2 (ds + dn) + cdn db + cup dt - diag dc + plate
                const float4 q0 = *reinterpret_cast<const float4*>(lcp + 12);   // bwlo, bwhi
                const float4 q1 = *reinterpret_cast<const float4*>(lcp + 16);   // -twlo, -twhi
                const float4 q2 = *reinterpret_cast<const float4*>(lcp + 20);   // cdn, cup
                const float4 q3 = *reinterpret_cast<const float4*>(lcp + 24);   // -diag, plate
                float F[5], cxv[4], sdx[4];
#pragma unroll
                for (int a = 0; a < 5; ++a) F[a] = us[a] * (tcv[a] + tcv[a + 1]);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    cxv[a] = F[a] - F[a + 1];
                    sdx[a] = dcv[a] + dcv[a + 2];
                }
                float2 res[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 tc = h ? hi2(tc4) : lo2(tc4), dc = h ? hi2(dc4) : lo2(dc4);
                    const float2 ts = h ? hi2(ts4) : lo2(ts4), tn = h ? hi2(tn4) : lo2(tn4);
                    const float2 ds = h ? hi2(ds4) : lo2(ds4), dn = h ? hi2(dn4) : lo2(dn4);
                    const float2 tb = h ? hi2(tb4) : lo2(tb4), tt = h ? hi2(tt4) : lo2(tt4);
                    const float2 db = h ? hi2(db4) : lo2(db4), dt = h ? hi2(dt4) : lo2(dt4);
                    const int a = 2 * h;
                    float2 acc = fma2(kx2p, make_float2(sdx[a], sdx[a + 1]), hi2(q3));
                    acc = fma2(ky2p, add2(ds, dn), acc);
                    acc = fma2(lo2(q2), db, acc);
                    acc = fma2(hi2(q2), dt, acc);
                    acc = fma2(lo2(q3), dc, acc);
                    acc = add2(acc, make_float2(cxv[a], cxv[a + 1]));
                    acc = fma2(make_float2(vs[a], vs[a + 1]), add2(ts, tc), acc);
                    acc = fma2(make_float2(vn[a], vn[a + 1]), add2(tc, tn), acc);
                    acc = fma2(make_float2(wb[a], wb[a + 1]), fma2(lo2(q0), tb, mul2(hi2(q0), tc)), acc);
                    acc = fma2(make_float2(wt[a], wt[a + 1]), fma2(lo2(q1), tc, mul2(hi2(q1), tt)), acc);
                    res[h] = LF ? fma2(gdtp, acc, dc) : fma2(gdtp, acc, fma2(cap, dc, mul2(cbp, tc)));
                }
                *reinterpret_cast<float4*>(outp) = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
            }
        }
        // plane k-1 is no longer needed by this thread
        mbar_arrive(&empty[sb]);
        outp += plane;
    };
    // the slots rotate (a loop unrolled by the ring length would copy the slab
    // build into every layer and outgrow the instruction cache)
    int sb = 0, sc = 1, st = 2, tpar = 0;
    for (int k = k0; k < k1; ++k) {
        layer(k, sb, sc, st, tpar);
        sb = sc;
        sc = st;
        if (++st == NB) {
            st = 0;
            tpar ^= 1;
        }
    }
    if (consumers_sync_or<kCons>(fail)) {
        if (tid == 0) atomicExch(A.err, MR_ERR_TIMEOUT);
        return;
    }
    if (DIVONLY) {
        for (int d = 16; d > 0; d >>= 1) dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, d));
        if (lane == 0) red[warp] = dmax;
        consumers_sync<kCons>();
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < NW; ++w) m = fmaxf(m, red[w]);
            atomicMax(A.divmax, (unsigned long long)__double_as_longlong((double)m));
        }
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

// Tensor maps of (buffer, shape, box), encoded once each.
bool map_fx(CUtensorMap* out, const float* base, int d0, int d1, int d2, int b0, int b1, int b2)
{
    struct Entry { const float* p; int d[6]; CUtensorMap m; };
    static Entry cache[16];
    static int n = 0, next = 0;
    static std::mutex mu;
    const int key[6] = {d0, d1, d2, b0, b1, b2};
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
    cuuint64_t strides[2] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * d1 * 4};
    cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2};
    cuuint32_t es[3] = {1, 1, 1};
    if (fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
        return false;
    std::lock_guard<std::mutex> lock(mu);
    Entry& e = cache[n < 16 ? n++ : (next = (next + 1) % 16)];
    e.p = base;
    memcpy(e.d, key, sizeof key);
    e.m = *out;
    return true;
}

template <int M, int KIND, bool LF>
cudaError_t launch_fx(const Grid<float>& g, const float* U, const float* V, const float* W, const float* lc,
                      const float* rx12, const float* Tm1, const float* T, float* Tp1, StepCoef c, int* err,
                      unsigned long long* divmax, cudaStream_t st)
{
    using L = FX<M>;
    static unsigned long long attr = 0;                   // one bit per device
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_fused<M, KIND, LF>), (int)L::bytes, &attr);
    if (e != cudaSuccess) return e;
    CUtensorMap mn, mm, mlc;
    memset(&mn, 0, sizeof mn);
    memset(&mm, 0, sizeof mm);
    if (KIND == 0 && (!map_fx(&mn, T, g.Nx, g.Ny, g.Nz, kBX, kBY, 1) || !map_fx(&mm, Tm1, g.Nx, g.Ny, g.Nz, kBX, kBY, 1)))
        return cudaErrorInvalidValue;
    if (!map_fx(&mlc, lc, kLCW, g.Nz, 1, kLCW, 1, 1)) return cudaErrorInvalidValue;
    // ~12 waves of four CTAs per SM, chunks of at most 96 dense layers
    const int tiles = (g.Nx / kTX) * (g.Ny / kTY);
    const int want = 152 * 4 * 12;
    int chunks = max(1, min((want + tiles - 1) / tiles, g.nz));
    int kcs = (g.nz + chunks - 1) / chunks;
    kcs = max(1, min(kcs, 96 / M));
    chunks = (g.nz + kcs - 1) / kcs;
    FXArgs A{g, U, V, W, T, Tm1, Tp1, (float)c.a, (float)c.b, (float)c.gdt, kcs, err, divmax, {}, ptx::kWaitNs, -1};
    memcpy(A.rx, rx12, sizeof A.rx);
    if (KIND == 0) take_wait_injection(&A.stop_ring, &A.wait_ns);
    dim3 grid(chunks, g.Nx / kTX, g.Ny / kTY);
    k_fused<M, KIND, LF><<<grid, kThreadsAll, L::bytes, st>>>(mn, mm, mlc, A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_fused_f32(const Grid<float>& g, const float* U, const float* V, const float* W,
                                   const float* lc, const float* rx12, const float* Tm1, const float* T, float* Tp1,
                                   StepCoef c, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    const bool lf = (c.a == 1.0 && c.b == 0.0);
    if (g.mx == 4)
        return lf ? launch_fx<4, 0, true>(g, U, V, W, lc, rx12, Tm1, T, Tp1, c, err, nullptr, st)
                  : launch_fx<4, 0, false>(g, U, V, W, lc, rx12, Tm1, T, Tp1, c, err, nullptr, st);
    return lf ? launch_fx<2, 0, true>(g, U, V, W, lc, rx12, Tm1, T, Tp1, c, err, nullptr, st)
              : launch_fx<2, 0, false>(g, U, V, W, lc, rx12, Tm1, T, Tp1, c, err, nullptr, st);
}

cudaError_t launch_fused_max_f32(const Grid<float>& g, int kind, const float* U, const float* V, const float* W,
                                  const float* lc, const float* rx12, double* partials, int blocks, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(partials, 0, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return e;
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(partials);
    const StepCoef c{0, 0, 0};
    if (g.mx == 4)
        return kind == 2 ? launch_fx<4, 2, false>(g, U, V, W, lc, rx12, nullptr, nullptr, nullptr, c, err, dm, st)
                         : launch_fx<4, 1, false>(g, U, V, W, lc, rx12, nullptr, nullptr, nullptr, c, err, dm, st);
    return kind == 2 ? launch_fx<2, 2, false>(g, U, V, W, lc, rx12, nullptr, nullptr, nullptr, c, err, dm, st)
                     : launch_fx<2, 1, false>(g, U, V, W, lc, rx12, nullptr, nullptr, nullptr, c, err, dm, st);
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
    if ((cfg.nx * cfg.mx) % kTX || (cfg.ny * cfg.my) % kTY) {
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
