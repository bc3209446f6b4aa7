// Fused FP32 refine + scalar-step kernel (MR_VEL_FUSED).
//
// One CTA owns a 64 x 16 column of dense cells (x by y) and marches up a chunk
// of coarse layers.  Per coarse layer K it loads the coarse U, V, W it needs
// (a one-coarse-cell halo, periodic wrap) with cp.async, forms the z-splits
// and the full-area vertical fluxes of every column by slab balance (stage Z
// of the refinement, Section 3.2); per dense layer it then builds, entirely
// in shared memory, the refined W on the layer's top plane (R_y then R_x),
// the outer U sub-faces, the full-width V of every dense row by row balance
// (stage Y), the refined V (R_x), and the inner U by cell balance (stage X),
// and finally applies the second-order finite-volume update (Eq. 5) with the
// Euler-leapfrog coefficients (Section 2.2).  The refined velocity never
// touches HBM.
//
// The two scalar levels T^n and T^{n-1} stream through a ring of NB dense
// planes per field, each a (64+8) x (16+2) box fetched by TMA
// (cp.async.bulk.tensor) onto an mbarrier; the x box starts 4 cells left of
// the tile so that the copy stays 16-byte aligned.  Where the tile touches the
// periodic edge, the wrapped halo column / row is patched in with plain loads.
// Every mbarrier wait is bounded: on time-out the CTA records MR_ERR_TIMEOUT
// in a device flag and leaves.
//
// Supported: FP32, periodic x and y, mx = my = mz = M in {2, 4},
// Nx % 64 == 0, Ny % 16 == 0, explicit diffusion.
#include <cuda.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "mr_internal.cuh"
#include "mr_ptx.cuh"

namespace mr {
namespace {

using namespace ptx;

constexpr int kTX = 64, kTY = 16;
constexpr int kBX = kTX + 8, kBY = kTY + 2;           // TMA box (floats)
constexpr int kPlaneFloats = kBX * kBY;                // 1296
constexpr int kSlotFloats = ((kPlaneFloats * 4 + 127) / 128) * 128 / 4;  // 128-byte aligned slot
constexpr int kThreads = 256;                          // consumer threads (8 warps)
constexpr int kThreadsAll = kThreads + 32;             // + one producer warp
constexpr uint32_t kPlaneBytes = kPlaneFloats * 4;
constexpr float kTBottom = 0.5f, kTTop = -0.5f;

template <int M>
struct Tile {
    static constexpr int CX = kTX / M, CY = kTY / M;
    static constexpr int UX = CX + 3, UY = CY + 2;     // U faces I0-1..I0+CX+1, rows J0-1..J0+CY
    static constexpr int VX = CX + 2, VY = CY + 3;     // V cells I0-1..I0+CX, faces J0-1..J0+CY+1
    static constexpr int WX = CX + 2, WY = CY + 2;     // W columns I0-1..I0+CX, J0-1..J0+CY
    static constexpr int NB = (M == 4) ? 6 : 5;        // dense planes resident per field
    // shared-memory layout (floats), T ring first (128-byte aligned slots)
    static constexpr int oT = 0;
    static constexpr int oCU = oT + NB * 2 * kSlotFloats;
    static constexpr int oCV = oCU + 2 * 3 * UY * UX;
    static constexpr int oCW = oCV + 2 * 3 * VY * VX;
    static constexpr int oUz = oCW + 2 * 2 * WY * WX;
    static constexpr int oVz = oUz + M * UY * UX;
    static constexpr int oWc = oVz + M * VY * VX;
    static constexpr int oWy = oWc + (M + 1) * WY * WX;
    static constexpr int oUo = oWy + (M + 1) * kTY * WX;
    static constexpr int oVr = oUo + M * kTY * UX;
    static constexpr int oRy = oVr + M * (kTY + 1) * VX;
    static constexpr int oLc = oRy + kTY * 3;          // [M][kLc] per-layer constants of the slab
    static constexpr int oRed = oLc + M * 12;
    static constexpr int oBar = ((oRed + 64) * 4 + 7) / 8;  // in uint64 units: full[NB], empty[NB]
    static constexpr size_t bytes = (size_t)(oBar + 2 * NB) * 8;
};

struct FusedArgs {
    Grid<float> g;
    const float* U;      // coarse faces [nz][ny][nx], [nz+1][ny][nx] for W
    const float* V;
    const float* W;
    const float* Tn;     // T^s (global, for halo patches)
    const float* Tm;     // T^{s-1}
    float* Tp1;          // T^{s+1}
    float a, b, gdt;
    int kc;              // coarse layers per chunk
    int* err;
    unsigned long long* divmax;   // DIVONLY: max |div| as FP64 bits
};

// Issue the TMA copies of dense plane z (both fields) into ring slot s.
__device__ __forceinline__ void issue_plane(float* sT, uint64_t* bar, const CUtensorMap* mn, const CUtensorMap* mm,
                                            int s, int i0, int j0, int z)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[s], 2 * kPlaneBytes);
    tma_3d(sT + (2 * s + 0) * kSlotFloats, mn, i0 - 4, j0 - 1, z, &bar[s]);
    tma_3d(sT + (2 * s + 1) * kSlotFloats, mm, i0 - 4, j0 - 1, z, &bar[s]);
}

template <int M, bool DIVONLY>
__global__ void __launch_bounds__(kThreadsAll, 2)
k_fused(const __grid_constant__ CUtensorMap tmn, const __grid_constant__ CUtensorMap tmm, const FusedArgs A)
{
    using L = Tile<M>;
    constexpr int UX = L::UX, UY = L::UY, VX = L::VX, VY = L::VY, WX = L::WX, WY = L::WY, NB = L::NB;
    constexpr int NC = 4 / M;                  // coarse cells per 4-cell segment
    constexpr int NW = kThreads / 32;          // consumer warps
    extern __shared__ __align__(128) float sm[];
    float* sT = sm + L::oT;
    float* cu = sm + L::oCU;   // [2][3][UY][UX]  coarse U of the slab's z-window
    float* cv = sm + L::oCV;   // [2][3][VY][VX]
    float* cw = sm + L::oCW;   // [2][2][WY][WX]  coarse W below / above the slab
    float* Uz = sm + L::oUz;   // [M][UY][UX]     z-split of U per dense layer (R_z)
    float* Vz = sm + L::oVz;   // [M][VY][VX]
    float* Wc = sm + L::oWc;   // [M+1][WY][WX]   full-area W per dense plane of the slab
    float* Wy = sm + L::oWy;   // [M+1][TY][WX]   y-split of Wc
    float* Uo = sm + L::oUo;   // [M][TY][UX]     outer U sub-faces (R_y of Uz)
    float* Vr = sm + L::oVr;   // [M][TY+1][VX]   full-coarse-width V of every dense row
    float* sRy = sm + L::oRy;  // [TY][3]
    float* Lc = sm + L::oLc;   // [M][12] layer constants: dz, 1/dz, wlo_b, whi_b, wlo_t, whi_t, cdn, cup, dx/dz
    float* red = sm + L::oRed;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm) + L::oBar;
    uint64_t* empty = full + NB;

    const Grid<float>& g = A.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * kTX, j0 = blockIdx.z * kTY;
    const int I0 = i0 / M, J0 = j0 / M;
    const int K0 = blockIdx.x * A.kc;
    const int K1 = min(K0 + A.kc, g.nz);
    if (K0 >= K1) return;
    const int k0 = K0 * M, k1 = K1 * M;          // dense layers [k0, k1)
    const int nplanes = k1 - k0 + 2;             // ring planes k0-1 .. k1

    if (!DIVONLY && tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---------------------------------------------------------------- producer warp
    if (warp == NW) {
        if (DIVONLY || lane != 0) return;
        for (int r = 0; r < nplanes; ++r) {
            const int s = r % NB;
            if (r >= NB && !mbar_wait(&empty[s], ((r / NB) - 1) & 1)) {
                atomicExch(A.err, MR_ERR_TIMEOUT);    // consumers then time out on full[]
                break;
            }
            issue_plane(sT, full, &tmn, &tmm, s, i0, j0, k0 - 1 + r);
        }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    const float DX = g.DX, DY = g.DY, dx = g.dx, dy = g.dy;
    const int seg = tid & 15, jl = tid >> 4;     // this thread's 4-cell segment of dense row jl
    const int il0 = seg * 4;
    float rx[4][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int p = 0; p < 3; ++p) rx[a][p] = g.Rx[(size_t)(i0 + il0 + a) * 3 + p];
    for (int t = tid; t < kTY * 3; t += kThreads) sRy[t] = g.Ry[(size_t)j0 * 3 + t];
    // periodic wrap of the in-plane halo, for the threads on the domain edge
    const bool wrap_w = (i0 == 0 && seg == 0), wrap_e = (i0 + kTX == g.Nx && seg == 15);
    const bool wrap_s = (j0 == 0 && jl == 0), wrap_n = (j0 + kTY == g.Ny && jl == kTY - 1);
    const size_t plane = (size_t)g.Nx * g.Ny;

    // coarse tile of layer K into buffer bb (cp.async; one warp per row)
    auto load_coarse = [&](int K, int bb) {
        constexpr int RU = 3 * UY, RV = 3 * VY, RW = 2 * WY;
        for (int row = warp; row < RU + RV + RW; row += NW) {
            if (row < RU) {
                const int q = row / UY, uj = row % UY;
                const float* src = A.U + ((size_t)g.wz[3 * K + q] * g.ny + wrap(J0 - 1 + uj, g.ny)) * g.nx;
                float* dst = cu + (bb * RU + row) * UX;
                for (int x = lane; x < UX; x += 32) cp_async4(dst + x, src + wrap(I0 - 1 + x, g.nx));
            } else if (row < RU + RV) {
                const int r2 = row - RU, q = r2 / VY, vj = r2 % VY;
                const float* src = A.V + ((size_t)g.wz[3 * K + q] * g.ny + wrap(J0 - 1 + vj, g.ny)) * g.nx;
                float* dst = cv + (bb * RV + r2) * VX;
                for (int x = lane; x < VX; x += 32) cp_async4(dst + x, src + wrap(I0 - 1 + x, g.nx));
            } else {
                const int r2 = row - RU - RV, q = r2 / WY, wj = r2 % WY;
                const float* src = A.W + ((size_t)(K + q) * g.ny + wrap(J0 - 1 + wj, g.ny)) * g.nx;
                float* dst = cw + (bb * RW + r2) * WX;
                for (int x = lane; x < WX; x += 32) cp_async4(dst + x, src + wrap(I0 - 1 + x, g.nx));
            }
        }
        cp_async_commit();
    };

    load_coarse(K0, 0);
    int waited = 0;            // ring planes this thread has waited for
    bool fail = false;
    float dmax = 0.f;

    for (int K = K0; K < K1; ++K) {
        const int bb = (K - K0) & 1;
        cp_async_wait_all();
        if (consumers_sync_or<kThreads>(fail)) break;       // uniform exit of every consumer
        if (K + 1 < K1) load_coarse(K + 1, bb ^ 1);
        const float* ccu = cu + bb * 3 * UY * UX;
        const float* ccv = cv + bb * 3 * VY * VX;
        const float* ccw = cw + bb * 2 * WY * WX;
        // per-layer constants of the slab, read by every thread of every layer
        if (tid < M) {
            const int k = K * M + tid;
            float* lc = Lc + tid * 12;
            lc[0] = g.dz[k]; lc[1] = g.inv_dz[k];
            lc[2] = g.wlo[k]; lc[3] = g.whi[k]; lc[4] = g.wlo[k + 1]; lc[5] = g.whi[k + 1];
            lc[6] = g.cdn[k]; lc[7] = g.cup[k]; lc[8] = dx / g.dz[k];
        }
        // A1: z-splits of the U and V faces for the M dense layers (R_z)
        for (int row = warp; row < M * UY + M * VY; row += NW) {
            if (row < M * UY) {
                const int c = row / UY, uj = row % UY;
                const float* rz = g.Rz + 3 * (K * M + c);
                const float r0 = rz[0], r1 = rz[1], r2 = rz[2];
                for (int x = lane; x < UX; x += 32)
                    Uz[row * UX + x] = r0 * ccu[uj * UX + x] + r1 * ccu[(UY + uj) * UX + x] + r2 * ccu[(2 * UY + uj) * UX + x];
            } else {
                const int rr = row - M * UY, c = rr / VY, vj = rr % VY;
                const float* rz = g.Rz + 3 * (K * M + c);
                const float r0 = rz[0], r1 = rz[1], r2 = rz[2];
                for (int x = lane; x < VX; x += 32)
                    Vz[rr * VX + x] = r0 * ccv[vj * VX + x] + r1 * ccv[(VY + vj) * VX + x] + r2 * ccv[(2 * VY + vj) * VX + x];
            }
        }
        consumers_sync<kThreads>();
        // A2: stage Z slab balance, top-down, one thread per coarse column
        for (int t = tid; t < WY * WX; t += kThreads) {
            const int wj = t / WX, wi = t % WX;
            const float wtop = ccw[WY * WX + t];
            Wc[t] = ccw[t];
            Wc[M * WY * WX + t] = wtop;
            float F = wtop * DX * DY;
#pragma unroll
            for (int c = M - 1; c >= 1; --c) {
                const float dzk = g.dz[K * M + c];
                const float* uz = Uz + c * UY * UX + wj * UX + wi;
                const float* vz = Vz + c * VY * VX + wj * VX + wi;
                F = F + (uz[1] - uz[0]) * DY * dzk + (vz[VX] - vz[0]) * DX * dzk;
                Wc[c * WY * WX + t] = F / (DX * DY);
            }
        }
        consumers_sync<kThreads>();
        // S1: y-split of Wc on the M+1 planes; outer U sub-faces of the M layers (R_y)
        for (int row = warp; row < (M + 1) * kTY + M * kTY; row += NW) {
            if (row < (M + 1) * kTY) {
                const int c = row / kTY, j = row % kTY;
                const float* ry = sRy + 3 * j;
                const float* wc = Wc + c * WY * WX + (j / M) * WX;
                for (int x = lane; x < WX; x += 32)
                    Wy[row * WX + x] = ry[0] * wc[x] + ry[1] * wc[WX + x] + ry[2] * wc[2 * WX + x];
            } else {
                const int rr = row - (M + 1) * kTY, c = rr / kTY, j = rr % kTY;
                const float* ry = sRy + 3 * j;
                const float* uz = Uz + c * UY * UX + (j / M) * UX;
                for (int x = lane; x < UX; x += 32)
                    Uo[rr * UX + x] = ry[0] * uz[x] + ry[1] * uz[UX + x] + ry[2] * uz[2 * UX + x];
            }
        }
        consumers_sync<kThreads>();
        // S2: stage Y, full-width V of every dense row by row balance (running
        // sum from the coarse south face), for the M layers
        for (int row = warp; row < M * (kTY + 1); row += NW) {
            const int c = row / (kTY + 1), jr = row % (kTY + 1);
            const int Jl = jr / M, b = jr % M;
            const float dzk = g.dz[K * M + c];
            const float* vz = Vz + (c * VY + Jl + 1) * VX;
            const float* uo = Uo + c * kTY * UX;
            const float* wyb = Wy + c * kTY * WX;
            const float* wyt = Wy + (c + 1) * kTY * WX;
            for (int x = lane; x < VX; x += 32) {
                float G = vz[x] * DX * dzk;
                for (int q = 0; q < b; ++q) {
                    const int j2 = Jl * M + q;
                    G = G - (uo[j2 * UX + x + 1] - uo[j2 * UX + x]) * dy * dzk
                          - (wyt[j2 * WX + x] - wyb[j2 * WX + x]) * DX * dy;
                }
                Vr[row * VX + x] = b == 0 ? vz[x] : G / (DX * dzk);
            }
        }
        consumers_sync<kThreads>();

        // the M dense layers of the slab, free-running (no block barrier)
        for (int c = 0; c < M; ++c) {
            const int k = K * M + c;
            if (!DIVONLY && !fail) {
                const int need = k + 1 - (k0 - 1);             // ring index of plane k+1
                while (waited <= need) {
                    if (!mbar_wait(&full[waited % NB], (waited / NB) & 1)) { fail = true; break; }
                    ++waited;
                }
            }
            if (!fail) {
            const float* lc = Lc + c * 12;
            // refined faces of this thread's 4 cells, in registers
            float wb[4], wt[4], vs[4], vn[4], us[5];
            {
                const float* yb = Wy + (c * kTY + jl) * WX;
                const float* yt = Wy + ((c + 1) * kTY + jl) * WX;
                const float* rs = Vr + (c * (kTY + 1) + jl) * VX;
                const float* rn = rs + VX;
                const int cb0 = il0 / M;                      // first coarse column of the window
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int cb = cb0 + a / M;
                    wb[a] = rx[a][0] * yb[cb] + rx[a][1] * yb[cb + 1] + rx[a][2] * yb[cb + 2];
                    wt[a] = rx[a][0] * yt[cb] + rx[a][1] * yt[cb + 1] + rx[a][2] * yt[cb + 2];
                    vs[a] = rx[a][0] * rs[cb] + rx[a][1] * rs[cb + 1] + rx[a][2] * rs[cb + 2];
                    vn[a] = rx[a][0] * rn[cb] + rx[a][1] * rn[cb + 1] + rx[a][2] * rn[cb + 2];
                }
                // stage X: cell balance, west to east (velocity units: h = H / (dy dz))
                const float* ur = Uo + (c * kTY + jl) * UX;
                const float fx_y = dx / dy, fx_z = lc[8];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    float h = ur[cb0 + q + 1];                // outer west face of the coarse cell
                    us[q * M] = h;
#pragma unroll
                    for (int a = 0; a < M - 1; ++a) {
                        const int m = q * M + a;
                        h = h - (vn[m] - vs[m]) * fx_y - (wt[m] - wb[m]) * fx_z;
                        us[m + 1] = h;
                    }
                }
                us[4] = ur[cb0 + NC + 1];                     // outer east face of the segment
            }
            const float inv_dz = lc[1];
            if (DIVONLY) {
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float d = (us[a + 1] - us[a]) * g.inv_dx + (vn[a] - vs[a]) * g.inv_dy + (wt[a] - wb[a]) * inv_dz;
                    dmax = fmaxf(dmax, fabsf(d));
                }
                continue;
            }
            const int rb = k - k0, rc = rb + 1, rt = rb + 2;   // ring indices of planes k-1, k, k+1
            const float* Pn_b = sT + (2 * (rb % NB) + 0) * kSlotFloats;
            const float* Pm_b = sT + (2 * (rb % NB) + 1) * kSlotFloats;
            const float* Pn_c = sT + (2 * (rc % NB) + 0) * kSlotFloats;
            const float* Pm_c = sT + (2 * (rc % NB) + 1) * kSlotFloats;
            const float* Pn_t = sT + (2 * (rt % NB) + 0) * kSlotFloats;
            const float* Pm_t = sT + (2 * (rt % NB) + 1) * kSlotFloats;
            const int o = (jl + 1) * kBX + il0 + 4;
            float4 tc4 = *reinterpret_cast<const float4*>(Pn_c + o);
            float4 ts4 = *reinterpret_cast<const float4*>(Pn_c + o - kBX);
            float4 tn4 = *reinterpret_cast<const float4*>(Pn_c + o + kBX);
            float4 dc4 = *reinterpret_cast<const float4*>(Pm_c + o);
            float4 ds4 = *reinterpret_cast<const float4*>(Pm_c + o - kBX);
            float4 dn4 = *reinterpret_cast<const float4*>(Pm_c + o + kBX);
            float tw = Pn_c[o - 1], te = Pn_c[o + 4], dw = Pm_c[o - 1], de = Pm_c[o + 4];
            if (wrap_w | wrap_e | wrap_s | wrap_n) {
                // the box holds zeros beyond the domain: fetch the periodic images
                const size_t row = (size_t)k * plane + (size_t)(j0 + jl) * g.Nx;
                if (wrap_w) { tw = A.Tn[row + g.Nx - 1]; dw = A.Tm[row + g.Nx - 1]; }
                if (wrap_e) { te = A.Tn[row]; de = A.Tm[row]; }
                if (wrap_s) {
                    const size_t r2 = (size_t)k * plane + (size_t)(g.Ny - 1) * g.Nx + i0 + il0;
                    ts4 = *reinterpret_cast<const float4*>(A.Tn + r2);
                    ds4 = *reinterpret_cast<const float4*>(A.Tm + r2);
                }
                if (wrap_n) {
                    const size_t r2 = (size_t)k * plane + i0 + il0;
                    tn4 = *reinterpret_cast<const float4*>(A.Tn + r2);
                    dn4 = *reinterpret_cast<const float4*>(A.Tm + r2);
                }
            }
            const float tcv[6] = {tw, tc4.x, tc4.y, tc4.z, tc4.w, te};
            const float dcv[6] = {dw, dc4.x, dc4.y, dc4.z, dc4.w, de};
            const float tsv[4] = {ts4.x, ts4.y, ts4.z, ts4.w}, tnv[4] = {tn4.x, tn4.y, tn4.z, tn4.w};
            const float dsv[4] = {ds4.x, ds4.y, ds4.z, ds4.w}, dnv[4] = {dn4.x, dn4.y, dn4.z, dn4.w};
            float tbv[4] = {0.f, 0.f, 0.f, 0.f}, dbv[4] = {0.f, 0.f, 0.f, 0.f};
            float ttv[4] = {0.f, 0.f, 0.f, 0.f}, dtv[4] = {0.f, 0.f, 0.f, 0.f};
            const bool bot = (k == 0), top = (k == g.Nz - 1);
            if (!bot) {
                const float4 b4 = *reinterpret_cast<const float4*>(Pn_b + o);
                const float4 e4 = *reinterpret_cast<const float4*>(Pm_b + o);
                tbv[0] = b4.x; tbv[1] = b4.y; tbv[2] = b4.z; tbv[3] = b4.w;
                dbv[0] = e4.x; dbv[1] = e4.y; dbv[2] = e4.z; dbv[3] = e4.w;
            }
            if (!top) {
                const float4 b4 = *reinterpret_cast<const float4*>(Pn_t + o);
                const float4 e4 = *reinterpret_cast<const float4*>(Pm_t + o);
                ttv[0] = b4.x; ttv[1] = b4.y; ttv[2] = b4.z; ttv[3] = b4.w;
                dtv[0] = e4.x; dtv[1] = e4.y; dtv[2] = e4.z; dtv[3] = e4.w;
            }
            // plane k-1 is no longer needed by this thread: release its ring slot
            mbar_arrive(&empty[rb % NB]);
            const float wlo_b = lc[2], whi_b = lc[3], wlo_t = lc[4], whi_t = lc[5];
            const float cdn = lc[6], cup = lc[7];
            float res[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float tc = tcv[a + 1], dc = dcv[a + 1];
                float cz = 0.f, dz_ = 0.f;
                if (!bot) {
                    cz += wb[a] * (wlo_b * tbv[a] + whi_b * tc);
                    dz_ -= cdn * (dc - dbv[a]);
                } else {
                    dz_ -= cdn * (dc - kTBottom);
                }
                if (!top) {
                    cz -= wt[a] * (wlo_t * tc + whi_t * ttv[a]);
                    dz_ += cup * (dtv[a] - dc);
                } else {
                    dz_ += cup * (kTTop - dc);
                }
                const float cx = us[a] * 0.5f * (tcv[a] + tc) - us[a + 1] * 0.5f * (tc + tcv[a + 2]);
                const float cy = vs[a] * 0.5f * (tsv[a] + tc) - vn[a] * 0.5f * (tc + tnv[a]);
                const float C = cx * g.inv_dx + cy * g.inv_dy + cz * inv_dz;
                const float D = g.kx2 * ((dcv[a + 2] - dc) - (dc - dcv[a])) + g.ky2 * ((dnv[a] - dc) - (dc - dsv[a])) + dz_;
                res[a] = A.a * dc + A.b * tc + A.gdt * (C + D);
            }
            *reinterpret_cast<float4*>(A.Tp1 + (size_t)k * plane + (size_t)(j0 + jl) * g.Nx + i0 + il0) =
                make_float4(res[0], res[1], res[2], res[3]);
            } else if (!DIVONLY) {
                mbar_arrive(&empty[(k - k0) % NB]);
            }
        }
    }
    if (consumers_sync_or<kThreads>(fail)) {
        if (tid == 0) atomicExch(A.err, MR_ERR_TIMEOUT);
        return;
    }
    if (DIVONLY) {
        // block max -> device max (non-negative doubles order as their bit patterns)
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
        if (lane == 0) red[warp] = dmax;
        consumers_sync<kThreads>();
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

bool make_map(CUtensorMap* m, const float* base, const Grid<float>& g)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)g.Nx, (cuuint64_t)g.Ny, (cuuint64_t)g.Nz};
    cuuint64_t strides[2] = {(cuuint64_t)g.Nx * 4, (cuuint64_t)g.Nx * g.Ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)kBX, (cuuint32_t)kBY, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

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

namespace {

// Tensor maps of the (few) scalar buffers in use, encoded once each.
bool cached_map(CUtensorMap* m, const float* base, const Grid<float>& g)
{
    struct Entry { const float* p; int nx, ny, nz; CUtensorMap map; };
    static Entry cache[16];
    static int n = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    for (int q = 0; q < n; ++q)
        if (cache[q].p == base && cache[q].nx == g.Nx && cache[q].ny == g.Ny && cache[q].nz == g.Nz) {
            *m = cache[q].map;
            return true;
        }
    if (!make_map(m, base, g)) return false;
    Entry& e = cache[n < 16 ? n++ : (n = 1, 0)];
    e.p = base; e.nx = g.Nx; e.ny = g.Ny; e.nz = g.Nz; e.map = *m;
    return true;
}

// Coarse layers per CTA chunk; MR_FUSED_KC in the environment overrides the
// automatic choice (used for tuning).
int chunk_override()
{
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("MR_FUSED_KC");
        v = e ? atoi(e) : 0;
    }
    return v;
}

template <int M, bool DIVONLY>
cudaError_t launch_fused(const Grid<float>& g, const float* U, const float* V, const float* W, const float* Tm1,
                         const float* T, float* Tp1, StepCoef c, int* err, unsigned long long* divmax,
                         cudaStream_t st)
{
    using L = Tile<M>;
    static unsigned long long attr = 0;                   // one bit per device
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_fused<M, DIVONLY>), (int)L::bytes, &attr);
    if (e != cudaSuccess) return e;
    CUtensorMap mn, mm;
    if (!DIVONLY) {
        if (!cached_map(&mn, T, g) || !cached_map(&mm, Tm1, g)) return cudaErrorInvalidValue;
    } else {
        memset(&mn, 0, sizeof mn);
        memset(&mm, 0, sizeof mm);
    }
    // chunk the z march so that the grid fills the GPU several times over
    const int tiles = (g.Nx / kTX) * (g.Ny / kTY);
    int kc = chunk_override();
    if (kc <= 0) {
        const int want = 152 * 2 * 8;                     // ~8 waves at 2 CTAs / SM
        int chunks = (want + tiles - 1) / tiles;
        chunks = max(1, min(chunks, g.nz));
        kc = (g.nz + chunks - 1) / chunks;
        kc = max(kc, 2);
    }
    const int chunks = (g.nz + kc - 1) / kc;
    FusedArgs A{g, U, V, W, T, Tm1, Tp1, (float)c.a, (float)c.b, (float)c.gdt, kc, err, divmax};
    dim3 grid(chunks, g.Nx / kTX, g.Ny / kTY);
    k_fused<M, DIVONLY><<<grid, kThreadsAll, L::bytes, st>>>(mn, mm, A);
    return cudaGetLastError();
}

}  // namespace

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
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) { cudaFree(p); return nullptr; }
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

cudaError_t launch_step_fused_f32(const Grid<float>& g, const float* U, const float* V, const float* W,
                                  const float* Tm1, const float* T, float* Tp1, StepCoef c, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    if (g.mx == 4) return launch_fused<4, false>(g, U, V, W, Tm1, T, Tp1, c, err, nullptr, st);
    return launch_fused<2, false>(g, U, V, W, Tm1, T, Tp1, c, err, nullptr, st);
}

cudaError_t launch_maxdiv_fused_f32(const Grid<float>& g, const float* U, const float* V, const float* W,
                                    double* partials, int blocks, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(partials, 0, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return e;
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(partials);
    StepCoef c{0, 0, 0};
    if (g.mx == 4) return launch_fused<4, true>(g, U, V, W, nullptr, nullptr, nullptr, c, err, dm, st);
    return launch_fused<2, true>(g, U, V, W, nullptr, nullptr, nullptr, c, err, dm, st);
}

}  // namespace mr
