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

#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr int kTX = 64, kTY = 16;
constexpr int kBX = kTX + 8, kBY = kTY + 2;           // TMA box (floats)
constexpr int kPlaneFloats = kBX * kBY;                // 1296
constexpr int kSlotFloats = ((kPlaneFloats * 4 + 127) / 128) * 128 / 4;  // 128-byte aligned slot
constexpr int kNB = 5;                                 // planes resident per field
constexpr int kThreads = 256;
constexpr uint32_t kPlaneBytes = kPlaneFloats * 4;
constexpr long kWaitLimit = 1L << 26;                  // bounded mbarrier wait: iterations ...
constexpr unsigned long long kWaitNs = 1000000000ull;  // ... and wall time (1 s)
constexpr float kTBottom = 0.5f, kTTop = -0.5f;

template <int M>
struct Tile {
    static constexpr int CX = kTX / M, CY = kTY / M;
    static constexpr int UX = CX + 3, UY = CY + 2;     // U faces I0-1..I0+CX+1, rows J0-1..J0+CY
    static constexpr int VX = CX + 2, VY = CY + 3;     // V cells I0-1..I0+CX, faces J0-1..J0+CY+1
    static constexpr int WX = CX + 2, WY = CY + 2;     // W columns I0-1..I0+CX, J0-1..J0+CY
    // shared-memory layout (floats), T ring first (128-byte aligned slots)
    static constexpr int oT = 0;
    static constexpr int oCU = oT + kNB * 2 * kSlotFloats;
    static constexpr int oCV = oCU + 2 * 3 * UY * UX;
    static constexpr int oCW = oCV + 2 * 3 * VY * VX;
    static constexpr int oUz = oCW + 2 * 2 * WY * WX;
    static constexpr int oVz = oUz + M * UY * UX;
    static constexpr int oWc = oVz + M * VY * VX;
    static constexpr int oWy = oWc + (M + 1) * WY * WX;
    static constexpr int oWs = oWy + 2 * kTY * WX;
    static constexpr int oUo = oWs + 2 * kTY * kTX;
    static constexpr int oUs = oUo + kTY * UX;
    static constexpr int oVr = oUs + kTY * (kTX + 1);
    static constexpr int oVs = oVr + (kTY + 1) * VX;
    static constexpr int oRx = oVs + (kTY + 1) * kTX;
    static constexpr int oRy = oRx + kTX * 3;
    static constexpr int oRed = oRy + kTY * 3;
    static constexpr int oBar = ((oRed + 64) * 4 + 7) / 8;  // in uint64 units
    static constexpr size_t bytes = (size_t)(oBar + kNB) * 8;
};

__device__ __forceinline__ uint32_t sa(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sa(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sa(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sa(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait (iteration count and wall time); true on success.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity)
{
    if (mbar_test(b, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long it = 0; it < kWaitLimit; ++it) {
        if (mbar_test(b, parity)) return true;
        if ((it & 255) == 0 && global_ns() - t0 > kWaitNs) break;
    }
    return false;
}
__device__ __forceinline__ void tma_plane(float* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(sa(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(sa(bar))
        : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

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
    tma_plane(sT + (2 * s + 0) * kSlotFloats, mn, i0 - 4, j0 - 1, z, &bar[s]);
    tma_plane(sT + (2 * s + 1) * kSlotFloats, mm, i0 - 4, j0 - 1, z, &bar[s]);
}

template <int M, bool DIVONLY>
__global__ void __launch_bounds__(kThreads, 2)
k_fused(const __grid_constant__ CUtensorMap tmn, const __grid_constant__ CUtensorMap tmm, const FusedArgs A)
{
    using L = Tile<M>;
    constexpr int CX = L::CX, CY = L::CY, UX = L::UX, UY = L::UY, VX = L::VX, VY = L::VY, WX = L::WX, WY = L::WY;
    extern __shared__ __align__(128) float sm[];
    float* sT = sm + L::oT;
    float* cu = sm + L::oCU;   // [2][3][UY][UX]
    float* cv = sm + L::oCV;   // [2][3][VY][VX]
    float* cw = sm + L::oCW;   // [2][2][WY][WX]
    float* Uz = sm + L::oUz;   // [M][UY][UX]
    float* Vz = sm + L::oVz;   // [M][VY][VX]
    float* Wc = sm + L::oWc;   // [M+1][WY][WX]
    float* Wy = sm + L::oWy;   // [2][TY][WX]
    float* Ws = sm + L::oWs;   // [2][TY][TX]
    float* Uo = sm + L::oUo;   // [TY][UX]
    float* Us = sm + L::oUs;   // [TY][TX+1]
    float* Vr = sm + L::oVr;   // [TY+1][VX]
    float* Vs = sm + L::oVs;   // [TY+1][TX]
    float* sRx = sm + L::oRx;  // [TX][3]
    float* sRy = sm + L::oRy;  // [TY][3]
    float* red = sm + L::oRed;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm) + L::oBar;

    const Grid<float>& g = A.g;
    const int tid = threadIdx.x;
    const int chunk = blockIdx.x;
    const int i0 = blockIdx.y * kTX, j0 = blockIdx.z * kTY;
    const int I0 = i0 / M, J0 = j0 / M;
    const int K0 = chunk * A.kc;
    const int K1 = min(K0 + A.kc, g.nz);
    if (K0 >= K1) return;
    const int k0 = K0 * M, k1 = K1 * M;          // dense layers [k0, k1)
    const int nplanes = k1 - k0 + 2;             // planes k0-1 .. k1
    const float DX = g.DX, DY = g.DY, dx = g.dx, dy = g.dy;
    const bool xedge = (i0 == 0) || (i0 + kTX == g.Nx);
    const bool yedge = (j0 == 0) || (j0 + kTY == g.Ny);

    for (int t = tid; t < kTX * 3; t += kThreads) sRx[t] = g.Rx[(size_t)i0 * 3 + t];
    for (int t = tid; t < kTY * 3; t += kThreads) sRy[t] = g.Ry[(size_t)j0 * 3 + t];
    if (!DIVONLY && tid == 0) {
        for (int s = 0; s < kNB; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (!DIVONLY && tid == 0)
        for (int r = 0; r < kNB && r < nplanes; ++r) issue_plane(sT, bar, &tmn, &tmm, r, i0, j0, k0 - 1 + r);

    // coarse tile of layer K into buffer bb (cp.async, periodic wrap in x, y)
    auto load_coarse = [&](int K, int bb) {
        constexpr int nU = 3 * UY * UX, nV = 3 * VY * VX, nW = 2 * WY * WX;
        for (int t = tid; t < nU + nV + nW; t += kThreads) {
            if (t < nU) {
                const int q = t / (UY * UX), r = t % (UY * UX), uj = r / UX, ui = r % UX;
                const int Kq = g.wz[3 * K + q];
                const int I = wrap(I0 - 1 + ui, g.nx), J = wrap(J0 - 1 + uj, g.ny);
                cp_async4(cu + bb * nU + t, A.U + ((size_t)Kq * g.ny + J) * g.nx + I);
            } else if (t < nU + nV) {
                const int u = t - nU;
                const int q = u / (VY * VX), r = u % (VY * VX), vj = r / VX, vi = r % VX;
                const int Kq = g.wz[3 * K + q];
                const int I = wrap(I0 - 1 + vi, g.nx), J = wrap(J0 - 1 + vj, g.ny);
                cp_async4(cv + bb * nV + u, A.V + ((size_t)Kq * g.ny + J) * g.nx + I);
            } else {
                const int u = t - nU - nV;
                const int q = u / (WY * WX), r = u % (WY * WX), wj = r / WX, wi = r % WX;
                const int I = wrap(I0 - 1 + wi, g.nx), J = wrap(J0 - 1 + wj, g.ny);
                cp_async4(cw + bb * nW + u, A.W + ((size_t)(K + q) * g.ny + J) * g.nx + I);
            }
        }
        cp_async_commit();
    };

    load_coarse(K0, 0);
    int waited = 0;            // ring planes waited for and patched
    bool fail = false;
    float dmax = 0.f;

    for (int K = K0; K < K1; ++K) {
        const int bb = (K - K0) & 1;
        cp_async_wait_all();
        __syncthreads();
        if (K + 1 < K1) load_coarse(K + 1, bb ^ 1);
        const float* ccu = cu + bb * 3 * UY * UX;
        const float* ccv = cv + bb * 3 * VY * VX;
        const float* ccw = cw + bb * 2 * WY * WX;
        // A1: z-splits of the U and V faces for the M dense layers of the slab
        for (int t = tid; t < M * UY * UX + M * VY * VX; t += kThreads) {
            if (t < M * UY * UX) {
                const int c = t / (UY * UX), r = t % (UY * UX);
                const float* rz = g.Rz + 3 * (K * M + c);
                Uz[t] = rz[0] * ccu[r] + rz[1] * ccu[UY * UX + r] + rz[2] * ccu[2 * UY * UX + r];
            } else {
                const int u = t - M * UY * UX;
                const int c = u / (VY * VX), r = u % (VY * VX);
                const float* rz = g.Rz + 3 * (K * M + c);
                Vz[u] = rz[0] * ccv[r] + rz[1] * ccv[VY * VX + r] + rz[2] * ccv[2 * VY * VX + r];
            }
        }
        __syncthreads();
        // A2: stage Z slab balance, top-down, one thread per column
        for (int t = tid; t < WY * WX; t += kThreads) {
            const int wj = t / WX, wi = t % WX;
            const float wbot = ccw[t], wtop = ccw[WY * WX + t];
            Wc[t] = wbot;
            Wc[M * WY * WX + t] = wtop;
            float F = wtop * DX * DY;
            for (int c = M - 1; c >= 1; --c) {
                const float dzk = g.dz[K * M + c];
                const float* uz = Uz + c * UY * UX + wj * UX + wi;
                const float* vz = Vz + c * VY * VX + wj * VX + wi;
                F = F + (uz[1] - uz[0]) * DY * dzk + (vz[VX] - vz[0]) * DX * dzk;
                Wc[c * WY * WX + t] = F / (DX * DY);
            }
        }
        __syncthreads();

        for (int c = 0; c < M; ++c) {
            const int k = K * M + c;
            const int pb = k & 1, pt = pb ^ 1;       // Wy / Ws buffers of the bottom / top plane
            const float dzk = g.dz[k];
            // B1: y-split of the full-area W on the top plane (and the bottom
            // plane at the start of the chunk)
            const int first = (k == k0) ? 0 : 1;
            for (int t = tid; t < (2 - first) * kTY * WX; t += kThreads) {
                const int pp = first + t / (kTY * WX);            // 0 bottom, 1 top
                const int r = t % (kTY * WX), jl = r / WX, wi = r % WX;
                const float* wc = Wc + (c + pp) * WY * WX + (jl / M) * WX + wi;
                const float* ry = sRy + 3 * jl;
                Wy[(pp ? pt : pb) * kTY * WX + r] = ry[0] * wc[0] + ry[1] * wc[WX] + ry[2] * wc[2 * WX];
            }
            __syncthreads();
            if (!DIVONLY && tid == 0 && k > k0) {
                // the ring slot of plane k-2 is free: fetch plane k-2+NB
                const int r = (k - 2) - (k0 - 1) + kNB;
                if (r < nplanes) issue_plane(sT, bar, &tmn, &tmm, r % kNB, i0, j0, k0 - 1 + r);
            }
            // B2: x-split into the refined W; B3: outer U sub-faces (R_y of the z-split)
            for (int t = tid; t < (2 - first) * kTY * kTX + kTY * UX; t += kThreads) {
                if (t < (2 - first) * kTY * kTX) {
                    const int pp = first + t / (kTY * kTX);
                    const int r = t % (kTY * kTX), jl = r / kTX, il = r % kTX;
                    const float* wy = Wy + (pp ? pt : pb) * kTY * WX + jl * WX + il / M;
                    const float* rx = sRx + 3 * il;
                    Ws[(pp ? pt : pb) * kTY * kTX + r] = rx[0] * wy[0] + rx[1] * wy[1] + rx[2] * wy[2];
                } else {
                    const int u = t - (2 - first) * kTY * kTX;
                    const int jl = u / UX, ui = u % UX;
                    const float* uz = Uz + c * UY * UX + (jl / M) * UX + ui;
                    const float* ry = sRy + 3 * jl;
                    Uo[u] = ry[0] * uz[0] + ry[1] * uz[UX] + ry[2] * uz[2 * UX];
                }
            }
            __syncthreads();
            // B4: stage Y row balance, south to north, per (column, coarse row)
            for (int t = tid; t < VX * CY; t += kThreads) {
                const int Jl = t / VX, vi = t % VX;
                const float vs0 = Vz[c * VY * VX + (Jl + 1) * VX + vi];
                float G = vs0 * DX * dzk;
                Vr[(Jl * M) * VX + vi] = vs0;
                for (int b = 0; b < M - 1; ++b) {
                    const int jl = Jl * M + b;
                    const float uw = Uo[jl * UX + vi], ue = Uo[jl * UX + vi + 1];
                    const float wb = Wy[pb * kTY * WX + jl * WX + vi] * DX;
                    const float wt = Wy[pt * kTY * WX + jl * WX + vi] * DX;
                    G = G - (ue - uw) * dy * dzk - (wt - wb) * dy;
                    Vr[(jl + 1) * VX + vi] = G / (DX * dzk);
                }
                if (Jl == CY - 1) Vr[kTY * VX + vi] = Vz[c * VY * VX + (CY + 1) * VX + vi];
            }
            __syncthreads();
            // B5: refined V (R_x over the neighbouring columns' rows)
            for (int t = tid; t < (kTY + 1) * kTX; t += kThreads) {
                const int jl = t / kTX, il = t % kTX;
                const float* vr = Vr + jl * VX + il / M;
                const float* rx = sRx + 3 * il;
                Vs[t] = rx[0] * vr[0] + rx[1] * vr[1] + rx[2] * vr[2];
            }
            __syncthreads();
            // B6: stage X cell balance, west to east, per (coarse column, dense row)
            for (int t = tid; t < CX * kTY; t += kThreads) {
                const int jl = t / CX, Il = t % CX;
                const float uo = Uo[jl * UX + Il + 1];
                float H = uo * dy * dzk;
                Us[jl * (kTX + 1) + Il * M] = uo;
                for (int a = 0; a < M - 1; ++a) {
                    const int il = Il * M + a;
                    H = H - (Vs[(jl + 1) * kTX + il] - Vs[jl * kTX + il]) * dx * dzk
                          - (Ws[pt * kTY * kTX + jl * kTX + il] - Ws[pb * kTY * kTX + jl * kTX + il]) * dx * dy;
                    Us[jl * (kTX + 1) + il + 1] = H / (dy * dzk);
                }
                if (Il == CX - 1) Us[jl * (kTX + 1) + kTX] = Uo[jl * UX + CX + 1];
            }
            if (!DIVONLY) {
                // planes k-1, k, k+1 must be resident: wait (bounded) and patch the wrap halo
                const int need = k + 1 - (k0 - 1);             // ring index of plane k+1
                while (waited <= need && !fail) {
                    const int s = waited % kNB;
                    if (!mbar_wait(&bar[s], (waited / kNB) & 1)) { fail = true; break; }
                    const int z = k0 - 1 + waited;
                    if ((xedge || yedge) && z >= 0 && z < g.Nz) {
                        for (int f = 0; f < 2; ++f) {
                            float* P = sT + (2 * s + f) * kSlotFloats;
                            const float* src = (f == 0 ? A.Tn : A.Tm) + (size_t)z * g.Nx * g.Ny;
                            if (xedge)
                                for (int t = tid; t < kBY; t += kThreads) {
                                    const int j = wrap(j0 - 1 + t, g.Ny);
                                    if (i0 == 0) P[t * kBX + 3] = src[(size_t)j * g.Nx + g.Nx - 1];
                                    if (i0 + kTX == g.Nx) P[t * kBX + kTX + 4] = src[(size_t)j * g.Nx];
                                }
                            if (yedge)
                                for (int t = tid; t < kBX; t += kThreads) {
                                    const int i = wrap(i0 - 4 + t, g.Nx);
                                    if (j0 == 0) P[t] = src[(size_t)(g.Ny - 1) * g.Nx + i];
                                    if (j0 + kTY == g.Ny) P[(kTY + 1) * kBX + t] = src[i];
                                }
                        }
                    }
                    ++waited;
                }
                // generic writes above precede later asynchronous (TMA) writes of the slot
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            if (__syncthreads_or(fail)) {
                if (tid == 0) atomicExch(A.err, MR_ERR_TIMEOUT);
                return;
            }
            // B7: the finite-volume update of this dense layer (or its divergence)
            const float inv_dz = g.inv_dz[k];
            const int rb = k - 1 - (k0 - 1), rc = k - (k0 - 1), rt = k + 1 - (k0 - 1);
            const float* Pn_b = sT + (2 * (rb % kNB) + 0) * kSlotFloats;
            const float* Pm_b = sT + (2 * (rb % kNB) + 1) * kSlotFloats;
            const float* Pn_c = sT + (2 * (rc % kNB) + 0) * kSlotFloats;
            const float* Pm_c = sT + (2 * (rc % kNB) + 1) * kSlotFloats;
            const float* Pn_t = sT + (2 * (rt % kNB) + 0) * kSlotFloats;
            const float* Pm_t = sT + (2 * (rt % kNB) + 1) * kSlotFloats;
            const float wlo_b = g.wlo[k], whi_b = g.whi[k], wlo_t = g.wlo[k + 1], whi_t = g.whi[k + 1];
            const float cdn = g.cdn[k], cup = g.cup[k];
            const bool bot = (k == 0), top = (k == g.Nz - 1);
            const int il = tid % kTX;
            for (int jl = tid / kTX; jl < kTY; jl += kThreads / kTX) {
                const float uw = Us[jl * (kTX + 1) + il], ue = Us[jl * (kTX + 1) + il + 1];
                const float vs = Vs[jl * kTX + il], vn = Vs[(jl + 1) * kTX + il];
                const float wb = Ws[pb * kTY * kTX + jl * kTX + il], wt = Ws[pt * kTY * kTX + jl * kTX + il];
                if (DIVONLY) {
                    const float d = (ue - uw) * g.inv_dx + (vn - vs) * g.inv_dy + (wt - wb) * inv_dz;
                    dmax = fmaxf(dmax, fabsf(d));
                    continue;
                }
                const int o = (jl + 1) * kBX + il + 4;
                const float tc = Pn_c[o], tw = Pn_c[o - 1], te = Pn_c[o + 1], ts = Pn_c[o - kBX], tn = Pn_c[o + kBX];
                const float dc = Pm_c[o], dw = Pm_c[o - 1], de = Pm_c[o + 1], ds = Pm_c[o - kBX], dn = Pm_c[o + kBX];
                float cz = 0.f, dz_ = 0.f;
                if (!bot) {
                    cz += wb * (wlo_b * Pn_b[o] + whi_b * tc);
                    dz_ -= cdn * (dc - Pm_b[o]);
                } else {
                    dz_ -= cdn * (dc - kTBottom);
                }
                if (!top) {
                    cz -= wt * (wlo_t * tc + whi_t * Pn_t[o]);
                    dz_ += cup * (Pm_t[o] - dc);
                } else {
                    dz_ += cup * (kTTop - dc);
                }
                const float cx = uw * 0.5f * (tw + tc) - ue * 0.5f * (tc + te);
                const float cy = vs * 0.5f * (ts + tc) - vn * 0.5f * (tc + tn);
                const float C = cx * g.inv_dx + cy * g.inv_dy + cz * inv_dz;
                const float D = g.kx2 * ((de - dc) - (dc - dw)) + g.ky2 * ((dn - dc) - (dc - ds)) + dz_;
                A.Tp1[((size_t)k * g.Ny + j0 + jl) * g.Nx + i0 + il] = A.a * dc + A.b * tc + A.gdt * (C + D);
            }
            // next layer reuses Ws/Wy of this top plane as its bottom plane
        }
    }
    if (DIVONLY) {
        // block max -> device max (non-negative doubles order as their bit patterns)
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
        if ((tid & 31) == 0) red[tid >> 5] = dmax;
        __syncthreads();
        if (tid == 0) {
            float m = 0.f;
            for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
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
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_fused<M, DIVONLY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)L::bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap mn, mm;
    if (!DIVONLY) {
        if (!make_map(&mn, T, g) || !make_map(&mm, Tm1, g)) return cudaErrorInvalidValue;
    } else {
        memset(&mn, 0, sizeof mn);
        memset(&mm, 0, sizeof mm);
    }
    // chunk the z march so that the grid fills the GPU several times over
    const int tiles = (g.Nx / kTX) * (g.Ny / kTY);
    int kc = chunk_override();
    if (kc <= 0) {
        const int want = 152 * 2 * 4;                     // ~4 waves at 2 CTAs / SM
        int chunks = (want + tiles - 1) / tiles;
        chunks = max(1, min(chunks, g.nz));
        kc = (g.nz + chunks - 1) / chunks;
        kc = max(kc, 2);
    }
    const int chunks = (g.nz + kc - 1) / kc;
    FusedArgs A{g, U, V, W, T, Tm1, Tp1, (float)c.a, (float)c.b, (float)c.gdt, kc, err, divmax};
    dim3 grid(chunks, g.Nx / kTX, g.Ny / kTY);
    k_fused<M, DIVONLY><<<grid, kThreads, L::bytes, st>>>(mn, mm, A);
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
// gave up).  One per process; read and cleared by fused_take_error.
static int* g_err = nullptr;
int* fused_error_flag()
{
    if (!g_err) {
        if (cudaMalloc(&g_err, sizeof(int)) != cudaSuccess) return nullptr;
        cudaMemset(g_err, 0, sizeof(int));
    }
    return g_err;
}

int fused_take_error(cudaStream_t st)
{
    if (!g_err) return 0;
    int v = 0;
    if (cudaMemcpyAsync(&v, g_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MR_ERR_CUDA;
    cudaStreamSynchronize(st);
    if (v) cudaMemsetAsync(g_err, 0, sizeof(int), st);
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
