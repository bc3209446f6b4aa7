// MR_VEL_XFUSED: the FP32 step kernel with the x-stage of the refinement fused
// in, fed by stored coarse-x intermediates of the z- and y-stages.
//
// The refinement (Section 3.2) is separable by stage.  Its z- and y-stages
// (slab balance, y-splits, row balance) produce, at coarse resolution in x,
//   WY[k][j][I]  full-coarse-width W on dense plane k, dense row j (R_y of the
//                slab-balanced full-area W),
//   UO[k][j][I]  the outer U sub-face of coarse x-face I (R_y R_z of U),
//   VR[k][j][I]  the full-coarse-width V on dense y-face j (row balance),
// which depend on the coarse velocity only (UO and VR are stored multiplied by
// 1/(2 dx) and 1/(2 dy), the factors with which they enter the advective
// fluxes, so the x balance runs in those units); they are computed once per
// mr_refine_velocity (1/M_x of the dense face count, with 4 periodic ghost
// columns each side so that every TMA box stays in bounds and 16-byte
// aligned).  The step kernel streams them with the two scalar levels through
// one TMA ring (one producer warp, full/empty mbarriers) and performs the
// x-stage -- R_x splits of W and V and the west-to-east cell balance for U --
// in registers, followed by the finite-volume update (Eq. 5) with the
// Euler-leapfrog coefficients (Section 2.2).  The dense velocity is never
// stored and the layer loop has no block-wide barrier.
//
// Supported: FP32, periodic x and y, mx = my = mz = M in {2, 4},
// Nx % 64 == 0, Ny % 16 == 0, explicit diffusion.
#include <stdlib.h>
#include <string.h>

#include <mutex>

#include "mr_internal.cuh"
#include "mr_ptx.cuh"

namespace mr {
namespace {

using namespace ptx;

constexpr int kTX = 64;                                // tile width (cells); the height TY is 16 or 8
constexpr float kTBottom = 0.5f, kTTop = -0.5f;
#ifndef MR_XFUSED_IDLE_NS
#define MR_XFUSED_IDLE_NS 256
#endif
constexpr unsigned kIdleNs = MR_XFUSED_IDLE_NS;  // sleep between the producer warp's polls

// O4: fourth-order face values of T^s (Section 2.2): T^s has two halo rows
// each side and the layer constants carry the z-face weights.
// TY: tile height; 16 consumer threads (4-cell segments) per row, one producer
// warp; 64x16 tiles run two CTAs per SM, 64x8 tiles four (small grids).
// DIV: the layout of the reductions (divergence, CFL), which stream only the
// velocity sets: no scalar boxes, 16 slots, so that about four times the bytes
// are in flight per CTA.
template <int M, bool MT, bool O4 = false, int TY = 16, bool DIV = false>
struct XT {
    static constexpr int CONS = 16 * TY;                // consumer threads
    static constexpr int THREADS = CONS + 32;           // + one producer warp
    static constexpr int CTAS = TY == 16 ? 2 : (O4 ? 3 : 4);   // resident CTAs per SM the layout is sized for
    // one scalar level of one plane in a ring slot, each part a TMA box on a
    // 128-byte boundary: the tile's TY rows (64 wide), H rows south and H rows
    // north of them, the 4 columns west and east of them (periodic images at
    // the domain's edges); T^s has H = HN (two rows with O4), T^{s-1} H = 1
    static constexpr int HN = O4 ? 2 : 1;
    static constexpr int nYS = kTX * TY, nYN = nYS + kTX * HN, nXW = nYN + kTX * HN, nXE = nXW + 4 * TY;
    static constexpr int mYS = kTX * TY, mYN = mYS + kTX, mXW = mYN + kTX, mXE = mXW + 4 * TY;
    static constexpr int PN = DIV ? 0 : nXE + 4 * TY, PM = DIV ? 0 : mXE + 4 * TY;
    static_assert(PN % 32 == 0 && PM % 32 == 0 && nXE % 32 == 0 && mXE % 32 == 0, "128-byte TMA boxes");
    static constexpr uint32_t tn_bytes = (uint32_t)PN * 4, tm_bytes = (uint32_t)PM * 4;
    static constexpr int CX = kTX / M;
    static constexpr int BXC = CX + 8;                  // coarse box width: columns I0-4 .. I0+CX+3
    // ring slots; MT (two velocity sets per slot) keeps two CTAs per SM with fewer
    // slots.  O4 keeps five planes live at a chunk's first layer (k0-2 .. k0+2),
    // so it needs at least five slots (at M = 2 with MT that leaves one CTA per SM).
    static constexpr int NB0 = MT ? ((M == 4) ? 5 : 4) : ((M == 4 && TY == 16) ? 7 : 6);
    static constexpr int NB = DIV ? 16 : ((O4 && TY == 8 && !MT) ? 7 : ((O4 && NB0 < 5) ? 5 : NB0));
    // one ring slot (floats): T^n plane, T^{n-1} plane, then the velocity set of
    // one layer k: WY of its upper plane k+1 (its lower plane k is the previous
    // slot's), UO and VR of layer k; with MT the set of the second coarse time
    // level follows at offset DS; then the layer constants
    static constexpr int LCW = 32;                      // floats of one row of layer constants
    static constexpr int oTn = 0, oTm = PN;
    static constexpr int oWY = PN + PM;                 // [TY][BXC]      plane k+1
    static constexpr int oUO = oWY + TY * BXC;          // [TY][BXC]
    static constexpr int oVR = oUO + TY * BXC;          // [TY+1][BXC]
    static constexpr int SET = ((2 * TY + TY + 1) * BXC + 31) / 32 * 32;     // one set, 128-B multiple
    static constexpr int DS = MT ? SET : 0;
    static constexpr int oLC = oWY + (MT ? 2 : 1) * SET;                     // [LCW] layer constants
    static constexpr int slot = (((oLC + LCW) * 4 + 127) / 128) * 128 / 4;
    static constexpr int NSET = MT ? 2 : 1;
    static constexpr uint32_t wy_bytes = (uint32_t)(NSET * TY * BXC) * 4;
    static constexpr uint32_t bundle_bytes = (uint32_t)(NSET * (TY * BXC + (TY + 1) * BXC) + LCW) * 4;  // UO, VR, LC
    static constexpr int oRed = NB * slot;              // 64 floats
    static constexpr int oBar = ((oRed + 64) * 4 + 7) / 8;
    static constexpr size_t bytes = (size_t)(oBar + 2 * NB) * 8;
};

// Tensor maps of the step: per scalar level (n: T^s, m: T^{s-1}) the tile's
// rows (64 x TY boxes), the rows beyond its y edges (64 x H), the columns beyond
// its x edges (4 x TY); the intermediates of one or two coarse time levels and
// the layer constants.
struct XMaps {
    CUtensorMap tn, tm, rn, rm, xn, xm, wy, uo, vr, lc, wy1, uo1, vr1;
};

struct XArgs {
    Grid<float> g;
    float* Tp1;          // T^{s+1}
    const float* lc;     // [Nz][32] per-layer constants
    float a, b, gdt;
    int kcl;             // dense layers per CTA chunk
    int* err;
    unsigned long long* divmax;
    float rx[4][3];      // R_x rows of the 4 cells of a segment (x is uniform and the
                         // segment starts on a coarse cell boundary, so these are the
                         // same for every thread: kept in the constant bank)
    float alpha;         // MT: weight of the second velocity set, i / M_t (Section 3.4)
    float w4x[4], w4y[4];  // O4: twice the fourth-order face weights of cells f-2..f+1 (uniform, periodic)
    unsigned long long wait_ns;   // time limit of every bounded wait
    int stop_ring;       // test hook: the producer of CTA (0,0,0) issues no ring from this one on (-1: none)
};

// R_x split of three coarse values by one row of R (rows sum to one):
// c1 + r0 (c0 - c1) + r2 (c2 - c1)
__device__ __forceinline__ float rsplit(const float (&r)[3], float c0, float c1, float c2)
{
    return c1 + r[0] * (c0 - c1) + r[2] * (c2 - c1);
}

// The same split negated, in as many operations: -c1 + r0 (c1 - c0) + r2 (c1 - c2).
__device__ __forceinline__ float nrsplit(const float (&r)[3], float c0, float c1, float c2)
{
    return -c1 + r[0] * (c1 - c0) + r[2] * (c1 - c2);
}

// Packed FP32 pairs: one instruction updates two cells (sm_100 and later).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// LF: a plain leapfrog step (a = 1, b = 0), by far the most frequent kind.
// MT: the velocity is A + alpha (B - A) between the intermediates of two
// coarse time levels (temporal refinement; the refinement is linear, so
// interpolating the intermediates interpolates the dense velocity).
// KIND 0: the step; 1: max |divergence| of the dense velocity; 2: max CFL
// rate |u|/dx + |v|/dy + |w|/dz (the last two read no scalar).
// O4: fourth-order face values of T^s (Section 2.2).  Ring r then carries plane
// k0-2+r (one more plane below and above the chunk) and the consumers carry the
// z-face advective flux of plane k+1 to the next layer.
template <int M, int KIND, bool LF, bool MT, bool O4, int TY>
__global__ void __launch_bounds__(XT<M, MT, O4, TY, (KIND != 0)>::THREADS, XT<M, MT, O4, TY, (KIND != 0)>::CTAS)
k_xfused(const __grid_constant__ XMaps T, const XArgs A)
{
    using L = XT<M, MT, O4, TY, (KIND != 0)>;
    constexpr int kThreads = L::CONS;
    constexpr int NB = L::NB, BXC = L::BXC, NC = 4 / M, NW = kThreads / 32;
    constexpr bool DIVONLY = KIND != 0;
    // PK: the update runs on packed pairs of cells (0, 1), (2, 3); vn then
    // holds the negated V split, the sign its flux enters with
    constexpr bool PK = !DIVONLY;
    constexpr int OFF = O4 ? 2 : 1;                  // ring r carries plane k0 - OFF + r
    extern __shared__ __align__(128) float sm[];
    float* red = sm + L::oRed;
    uint64_t* full = reinterpret_cast<uint64_t*>(sm) + L::oBar;
    uint64_t* empty = full + NB;

    const Grid<float>& g = A.g;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * kTX, j0 = blockIdx.z * TY;
    const int I0 = i0 / M;
    const int k0 = blockIdx.x * A.kcl;
    const int k1 = min(k0 + A.kcl, g.Nz);
    if (k0 >= k1) return;
    const int nrings = k1 - k0 + 2 * OFF;        // ring r: plane p = k0-OFF+r, WY of plane p (k0 <= p <= k1)
                                                 // and the bundle of layer p-1 (k0 <= p-1 < k1)

    if (tid == 0) {
        for (int s = 0; s < NB; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kThreads);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    // ---------------------------------------------------------------- producer warp
    if (warp == NW) {
        if (lane != 0) return;
        const bool stopper = (A.stop_ring >= 0 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0);
        // the rows and columns beyond the tile's edges, periodic in x and y
        const int ysn = (j0 == 0) ? g.Ny - L::HN : j0 - L::HN, ysm = (j0 == 0) ? g.Ny - 1 : j0 - 1;
        const int yn = (j0 + TY == g.Ny) ? 0 : j0 + TY;
        const int xw = (i0 == 0) ? g.Nx - 4 : i0 - 4, xe = (i0 + kTX == g.Nx) ? 0 : i0 + kTX;
        for (int r = 0; r < nrings; ++r) {
            const int s = r % NB;
            if (stopper && r == A.stop_ring) break;  // every ring issued so far is waited for by the consumers
            if (r >= NB && !mbar_wait_idle(&empty[s], ((r / NB) - 1) & 1, A.wait_ns, kIdleNs)) {
                atomicExch(A.err, MR_ERR_TIMEOUT);   // consumers then time out on full[]
                break;
            }
            float* slot = sm + s * L::slot;
            const int p = k0 - OFF + r;              // plane of this ring
            const bool wy = (p >= k0 && p <= k1), bundle = (p - 1 >= k0 && p - 1 < k1);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(&full[s], (DIVONLY ? 0u : L::tn_bytes + L::tm_bytes) + (wy ? L::wy_bytes : 0u) +
                                         (bundle ? L::bundle_bytes : 0u));
            if (!DIVONLY) {
                float* sn = slot + L::oTn;
                float* smm = slot + L::oTm;
                tma_3d(sn, &T.tn, i0, j0, p, &full[s]);
                tma_3d(sn + L::nYS, &T.rn, i0, ysn, p, &full[s]);
                tma_3d(sn + L::nYN, &T.rn, i0, yn, p, &full[s]);
                tma_3d(sn + L::nXW, &T.xn, xw, j0, p, &full[s]);
                tma_3d(sn + L::nXE, &T.xn, xe, j0, p, &full[s]);
                tma_3d(smm, &T.tm, i0, j0, p, &full[s]);
                tma_3d(smm + L::mYS, &T.rm, i0, ysm, p, &full[s]);
                tma_3d(smm + L::mYN, &T.rm, i0, yn, p, &full[s]);
                tma_3d(smm + L::mXW, &T.xm, xw, j0, p, &full[s]);
                tma_3d(smm + L::mXE, &T.xm, xe, j0, p, &full[s]);
            }
            if (wy) {
                tma_3d(slot + L::oWY, &T.wy, I0, j0, p, &full[s]);   // WY plane p
                if (MT) tma_3d(slot + L::oWY + L::DS, &T.wy1, I0, j0, p, &full[s]);
            }
            if (bundle) {
                const int kb = p - 1;
                tma_3d(slot + L::oUO, &T.uo, I0, j0, kb, &full[s]);
                tma_3d(slot + L::oVR, &T.vr, I0, j0, kb, &full[s]);
                if (MT) {
                    tma_3d(slot + L::oUO + L::DS, &T.uo1, I0, j0, kb, &full[s]);
                    tma_3d(slot + L::oVR + L::DS, &T.vr1, I0, j0, kb, &full[s]);
                }
                tma_3d(slot + L::oLC, &T.lc, 0, kb, 0, &full[s]);
            }
        }
        return;
    }

    // ---------------------------------------------------------------- consumer warps
    // this thread's 4-cell segment of dense row jl; the two half-warps take rows
    // two apart (bundle rows 2 BXC floats apart fall 16 banks apart, so the
    // half-warps' coarse-column reads do not conflict at M = 4)
    const int seg = tid & 15, jl = ((warp >> 1) << 2) + (warp & 1) + 2 * ((tid >> 4) & 1);
    const int il0 = seg * 4, cb0 = il0 / M;      // first coarse column of the segment (tile-local)
    const auto& rx = A.rx;

    bool fail = false;
    float dmax = 0.f;
    const float kx2 = g.kx2, ky2 = g.ky2;
    const float ca = A.a, cbb = A.b, gdt = A.gdt, alpha = A.alpha;
    const float2 kx2p = make_float2(kx2, kx2), ky2p = make_float2(ky2, ky2), gdtp = make_float2(gdt, gdt);
    const float2 cap = make_float2(ca, ca), cbp = make_float2(cbb, cbb);
    // O4: twice the y-face weights of rows j-2 .. j+1 (uniform), as pairs
    const float2 wy0p = make_float2(A.w4y[0], A.w4y[0]), wy1p = make_float2(A.w4y[1], A.w4y[1]);
    const float2 wy2p = make_float2(A.w4y[2], A.w4y[2]), wy3p = make_float2(A.w4y[3], A.w4y[3]);
    // ring bookkeeping without divisions: slots of planes k-1, k, k+1 (and, with
    // O4, k-2 and k+2).  Rings 0 .. 2 OFF - 1 (planes k0-OFF .. k0+OFF-1) are
    // waited for before the layer loop; then layer k waits for one ring, that of
    // plane k+OFF, in slot st (O4: s2) with parity tpar (2 OFF < NB)
#pragma unroll
    for (int r = 0; r < 2 * OFF; ++r)
        if (!fail && !mbar_wait(&full[r], 0, A.wait_ns)) fail = true;
    const size_t plane = (size_t)g.Nx * g.Ny;
    float* outp = A.Tp1 + (size_t)k0 * plane + (size_t)(j0 + jl) * g.Nx + i0 + il0;
    // offsets in a scalar level of a ring slot: the segment's first cell (both
    // levels), rows jl - 1 and jl + 1 of T^s (n) and T^{s-1} (m), rows jl - 2 and
    // jl + 2 of T^s (O4), the west and east neighbours of the row
    const int om = jl * kTX + il0;
    const int osn = jl >= 1 ? om - kTX : L::nYS + (L::HN - 1) * kTX + il0;
    const int onn = jl + 1 < TY ? om + kTX : L::nYN + il0;
    const int osn2 = jl >= 2 ? om - 2 * kTX : L::nYS + jl * kTX + il0;
    const int onn2 = jl + 2 < TY ? om + 2 * kTX : L::nYN + (jl + 2 - TY) * kTX + il0;
    const int osm = jl >= 1 ? om - kTX : L::mYS + il0;
    const int onm = jl + 1 < TY ? om + kTX : L::mYN + il0;
    const int oxwn = L::nXW + jl * 4 + 3, oxen = L::nXE + jl * 4;
    const int oxwm = L::mXW + jl * 4 + 3, oxem = L::mXE + jl * 4;

    float wcar[4] = {0.f, 0.f, 0.f, 0.f};            // R_x split of W on plane k (from layer k-1)
    float2 fcar[2] = {};                             // O4: advective flux W T_f through face k (from layer k-1)
    // one layer; sm2, sb, sc, st, s2: the slots of planes k-2 (O4), k-1, k, k+1
    // and k+2 (O4); tpar: the parity of the ring of plane k+OFF
    auto layer = [&](const int k, const int sm2, const int sb, const int sc, const int st, const int s2,
                     const int tpar) {
        // the ring of plane k+1 and of this layer's bundle (O4: of plane k+2)
        if (!fail && !mbar_wait(&full[O4 ? s2 : st], tpar, A.wait_ns)) fail = true;
        if (!fail) {
            const float* bun = sm + st * L::slot;
            // layer constants (from the bundle, see xfused_layer_constants)
            const float2 c0 = *reinterpret_cast<const float2*>(bun + L::oLC);
            const float inv_dz = c0.x, hz = c0.y;
            float wb[4], wt[4], vs[4], vn[4], us[5];
            {
                // R_x splits of the full-width W (planes k, k+1) and V (faces jl, jl+1);
                // bundle column xb holds coarse column I0 - 4 + xb
                const float* yb = sm + sc * L::slot + L::oWY + jl * BXC + cb0 + 3;   // plane k (previous slot)
                const float* yt = bun + L::oWY + jl * BXC + cb0 + 3;                  // plane k+1
                const float* rs = bun + L::oVR + jl * BXC + cb0 + 3;
                const float* rn = rs + BXC;
                const float* ur = bun + L::oUO + jl * BXC + cb0 + 4;   // outer face of coarse column cb0
                // the coarse columns a segment touches (interpolated in time with MT)
                constexpr int NV = NC + 2;
                float ybv[NV], ytv[NV], rsv[NV], rnv[NV], urv[NC + 1];
                if (k == k0) {
#pragma unroll
                    for (int c = 0; c < NV; ++c) {
                        ybv[c] = yb[c];
                        if (MT) ybv[c] += alpha * (yb[c + L::DS] - ybv[c]);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int cb = a / M;
                        wcar[a] = rsplit(rx[a], ybv[cb], ybv[cb + 1], ybv[cb + 2]);
                    }
                }
#pragma unroll
                for (int c = 0; c < NV; ++c) {
                    ytv[c] = yt[c];
                    rsv[c] = rs[c];
                    rnv[c] = rn[c];
                    if (MT) {
                        ytv[c] += alpha * (yt[c + L::DS] - ytv[c]);
                        rsv[c] += alpha * (rs[c + L::DS] - rsv[c]);
                        rnv[c] += alpha * (rn[c + L::DS] - rnv[c]);
                    }
                }
#pragma unroll
                for (int q = 0; q <= NC; ++q) {
                    urv[q] = ur[q];
                    if (MT) urv[q] += alpha * (ur[q + L::DS] - urv[q]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int cb = a / M;
                    wb[a] = wcar[a];
                    wt[a] = rsplit(rx[a], ytv[cb], ytv[cb + 1], ytv[cb + 2]);
                    vs[a] = rsplit(rx[a], rsv[cb], rsv[cb + 1], rsv[cb + 2]);
                    vn[a] = PK ? nrsplit(rx[a], rnv[cb], rnv[cb + 1], rnv[cb + 2])
                               : rsplit(rx[a], rnv[cb], rnv[cb + 1], rnv[cb + 2]);
                }
                // stage X: cell balance, west to east, in units of U / (2 dx) (V is in
                // units of V / (2 dy): the dx/dy factor of the balance cancels)
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
                    // us, vs, vn hold U/(2 dx), V/(2 dy)
                    const float d = KIND == 2 ? 2.f * (fmaxf(fabsf(us[a]), fabsf(us[a + 1])) + fmaxf(fabsf(vs[a]), fabsf(vn[a]))) +
                                                    fmaxf(fabsf(wb[a]), fabsf(wt[a])) * inv_dz
                                              : 2.f * ((us[a + 1] - us[a]) + (vn[a] - vs[a])) + (wt[a] - wb[a]) * inv_dz;
                    dmax = fmaxf(dmax, fabsf(d));
                }
            } else if constexpr (O4) {
                const float* Pn_b = sm + sb * L::slot + L::oTn;
                const float* Pm_b = sm + sb * L::slot + L::oTm;
                const float* Pn_c = sm + sc * L::slot + L::oTn;
                const float* Pm_c = sm + sc * L::slot + L::oTm;
                const float* Pn_t = sm + st * L::slot + L::oTn;
                const float* Pm_t = sm + st * L::slot + L::oTm;
                const float* Pn_2 = sm + s2 * L::slot + L::oTn;
                const float4 tc4 = *reinterpret_cast<const float4*>(Pn_c + om);
                const float4 ts4 = *reinterpret_cast<const float4*>(Pn_c + osn);
                const float4 tn4 = *reinterpret_cast<const float4*>(Pn_c + onn);
                const float4 ts24 = *reinterpret_cast<const float4*>(Pn_c + osn2);
                const float4 tn24 = *reinterpret_cast<const float4*>(Pn_c + onn2);
                const float4 dc4 = *reinterpret_cast<const float4*>(Pm_c + om);
                const float4 ds4 = *reinterpret_cast<const float4*>(Pm_c + osm);
                const float4 dn4 = *reinterpret_cast<const float4*>(Pm_c + onm);
                // in-row neighbours: two of T^s, one of T^{s-1} on each side
                float tw1 = __shfl_up_sync(0xffffffffu, tc4.w, 1), tw2 = __shfl_up_sync(0xffffffffu, tc4.z, 1);
                float te1 = __shfl_down_sync(0xffffffffu, tc4.x, 1), te2 = __shfl_down_sync(0xffffffffu, tc4.y, 1);
                float dw = __shfl_up_sync(0xffffffffu, dc4.w, 1), de = __shfl_down_sync(0xffffffffu, dc4.x, 1);
                if (seg == 0) { tw1 = Pn_c[oxwn]; tw2 = Pn_c[oxwn - 1]; dw = Pm_c[oxwm]; }
                if (seg == 15) { te1 = Pn_c[oxen]; te2 = Pn_c[oxen + 1]; de = Pm_c[oxem]; }
                const float4 db4 = *reinterpret_cast<const float4*>(Pm_b + om);
                const float4 dt4 = *reinterpret_cast<const float4*>(Pm_t + om);
                const float4 tb4 = *reinterpret_cast<const float4*>(Pn_b + om);
                const float4 tt4 = *reinterpret_cast<const float4*>(Pn_t + om);
                const float4 t24 = *reinterpret_cast<const float4*>(Pn_2 + om);
                const float t8[8] = {tw2, tw1, tc4.x, tc4.y, tc4.z, tc4.w, te1, te2};
                const float dcv[6] = {dw, dc4.x, dc4.y, dc4.z, dc4.w, de};
                const auto& wx = A.w4x;
                // twice the face values of the segment's five x faces (us holds U / (2 dx)),
                // and the x fluxes in scalar form (adjacent cells share a face)
                float F[5], cxv[4], sdx[4];
#pragma unroll
                for (int a = 0; a < 5; ++a)
                    F[a] = us[a] * (wx[0] * t8[a] + wx[1] * t8[a + 1] + wx[2] * t8[a + 2] + wx[3] * t8[a + 3]);
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    cxv[a] = F[a] - F[a + 1];
                    sdx[a] = dcv[a] + dcv[a + 2];
                }
                if (k == k0) {
                    // the chunk's first layer: face k from planes k-2 .. k+1
                    const float* Pn_m2 = sm + sm2 * L::slot + L::oTn;
                    const float4 tm4 = *reinterpret_cast<const float4*>(Pn_m2 + om);
                    const float4 zb = *reinterpret_cast<const float4*>(bun + L::oLC + 4);
                    const float tmv[4] = {tm4.x, tm4.y, tm4.z, tm4.w}, tbv[4] = {tb4.x, tb4.y, tb4.z, tb4.w};
                    const float ttv[4] = {tt4.x, tt4.y, tt4.z, tt4.w};
                    float f[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        f[a] = wb[a] * (zb.x * tmv[a] + zb.y * tbv[a] + zb.z * t8[a + 2] + zb.w * ttv[a]);
                    fcar[0] = make_float2(f[0], f[1]);
                    fcar[1] = make_float2(f[2], f[3]);
                }
                // the rest on the pairs (0, 1), (2, 3) with the pair constants of the row:
                // face-(k+1) weights of planes k-1 .. k+2, cdn, cup, -diag, plate, 1/dz, -1/dz
                const float4 q0 = *reinterpret_cast<const float4*>(bun + L::oLC + 12);
                const float4 q1 = *reinterpret_cast<const float4*>(bun + L::oLC + 16);
                const float4 q2 = *reinterpret_cast<const float4*>(bun + L::oLC + 20);
                const float4 q3 = *reinterpret_cast<const float4*>(bun + L::oLC + 24);
                const float4 q4 = *reinterpret_cast<const float4*>(bun + L::oLC + 28);
                float2 res[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 tc = h ? hi2(tc4) : lo2(tc4), dc = h ? hi2(dc4) : lo2(dc4);
                    const float2 ts = h ? hi2(ts4) : lo2(ts4), tn = h ? hi2(tn4) : lo2(tn4);
                    const float2 ts2 = h ? hi2(ts24) : lo2(ts24), tn2 = h ? hi2(tn24) : lo2(tn24);
                    const float2 ds = h ? hi2(ds4) : lo2(ds4), dn = h ? hi2(dn4) : lo2(dn4);
                    const float2 tb = h ? hi2(tb4) : lo2(tb4), tt = h ? hi2(tt4) : lo2(tt4);
                    const float2 t2 = h ? hi2(t24) : lo2(t24);
                    const float2 db = h ? hi2(db4) : lo2(db4), dt = h ? hi2(dt4) : lo2(dt4);
                    const int a = 2 * h;
                    float2 acc = fma2(kx2p, make_float2(sdx[a], sdx[a + 1]), hi2(q3));
                    acc = fma2(ky2p, add2(ds, dn), acc);
                    acc = fma2(lo2(q2), db, acc);
                    acc = fma2(hi2(q2), dt, acc);
                    acc = fma2(lo2(q3), dc, acc);
                    acc = add2(acc, make_float2(cxv[a], cxv[a + 1]));
                    const float2 fs = fma2(wy0p, ts2, fma2(wy1p, ts, fma2(wy2p, tc, mul2(wy3p, tn))));
                    const float2 fn = fma2(wy0p, ts, fma2(wy1p, tc, fma2(wy2p, tn, mul2(wy3p, tn2))));
                    acc = fma2(make_float2(vs[a], vs[a + 1]), fs, acc);
                    acc = fma2(make_float2(vn[a], vn[a + 1]), fn, acc);
                    const float2 ft = mul2(make_float2(wt[a], wt[a + 1]),
                                           fma2(lo2(q0), tb, fma2(hi2(q0), tc, fma2(lo2(q1), tt, mul2(hi2(q1), t2)))));
                    acc = fma2(lo2(q4), fcar[h], acc);
                    acc = fma2(hi2(q4), ft, acc);
                    fcar[h] = ft;
                    res[h] = LF ? fma2(gdtp, acc, dc) : fma2(gdtp, acc, fma2(cap, dc, mul2(cbp, tc)));
                }
                *reinterpret_cast<float4*>(outp) = make_float4(res[0].x, res[0].y, res[1].x, res[1].y);
            } else {
                const float* Pn_b = sm + sb * L::slot + L::oTn;
                const float* Pm_b = sm + sb * L::slot + L::oTm;
                const float* Pn_c = sm + sc * L::slot + L::oTn;
                const float* Pm_c = sm + sc * L::slot + L::oTm;
                const float* Pn_t = sm + st * L::slot + L::oTn;
                const float* Pm_t = sm + st * L::slot + L::oTm;
                const float4 tc4 = *reinterpret_cast<const float4*>(Pn_c + om);
                const float4 ts4 = *reinterpret_cast<const float4*>(Pn_c + osn);
                const float4 tn4 = *reinterpret_cast<const float4*>(Pn_c + onn);
                const float4 dc4 = *reinterpret_cast<const float4*>(Pm_c + om);
                const float4 ds4 = *reinterpret_cast<const float4*>(Pm_c + osm);
                const float4 dn4 = *reinterpret_cast<const float4*>(Pm_c + onm);
                // in-row neighbours from the adjacent segments (16 lanes per row)
                float tw = __shfl_up_sync(0xffffffffu, tc4.w, 1), te = __shfl_down_sync(0xffffffffu, tc4.x, 1);
                float dw = __shfl_up_sync(0xffffffffu, dc4.w, 1), de = __shfl_down_sync(0xffffffffu, dc4.x, 1);
                if (seg == 0) { tw = Pn_c[oxwn]; dw = Pm_c[oxwm]; }
                if (seg == 15) { te = Pn_c[oxen]; de = Pm_c[oxem]; }
                // planes below / above: zero-filled beyond the plates, where the plate
                // W is exactly zero and the plate value enters D through `plate`
                const float4 tb4 = *reinterpret_cast<const float4*>(Pn_b + om);
                const float4 db4 = *reinterpret_cast<const float4*>(Pm_b + om);
                const float4 tt4 = *reinterpret_cast<const float4*>(Pn_t + om);
                const float4 dt4 = *reinterpret_cast<const float4*>(Pm_t + om);
                const float tcv[6] = {tw, tc4.x, tc4.y, tc4.z, tc4.w, te};
                const float dcv[6] = {dw, dc4.x, dc4.y, dc4.z, dc4.w, de};
                // x fluxes in scalar form (adjacent cells share a face), then the rest
                // of the update on the pairs (0, 1), (2, 3):
                // D = kx2 (dw + de) + ky2 (ds + dn) + cdn db + cup dt - diag dc + plate,
                // the pair constants of the row (each value twice) with -diag and the
                // top-face weights negated, vn negated
                const float4 q0 = *reinterpret_cast<const float4*>(bun + L::oLC + 12);   // bwlo, bwhi
                const float4 q1 = *reinterpret_cast<const float4*>(bun + L::oLC + 16);   // -twlo, -twhi
                const float4 q2 = *reinterpret_cast<const float4*>(bun + L::oLC + 20);   // cdn, cup
                const float4 q3 = *reinterpret_cast<const float4*>(bun + L::oLC + 24);   // -diag, plate
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
        // plane k-1 (and the bundle of layer k-2) are no longer needed by this thread
        if constexpr (O4) {
            if (k == k0) mbar_arrive(&empty[sm2]);   // plane k0-2 served the first layer only
            mbar_arrive(&empty[sb]);
        } else {
            mbar_arrive(&empty[sb]);
        }
        outp += plane;
    };
    if constexpr (!O4 && !DIVONLY) {
        // unrolled by the ring length: layer k0 + i uses the slots i, i+1, i+2
        // (mod NB), constants in the inner loop
        for (int kb = k0, opar = 0; kb < k1; kb += NB, opar ^= 1) {
#pragma unroll
            for (int u = 0; u < NB; ++u) {
                if (kb + u >= k1) break;
                layer(kb + u, 0, u % NB, (u + 1) % NB, (u + 2) % NB, 0, opar ^ (((u + 2) / NB) & 1));
            }
        }
    } else {
        // fourth order (an unrolled loop would outgrow the instruction cache) and
        // the reductions (16 slots): the slots rotate; the waited slot is s2
        // (O4) or st, its parity flips when it wraps
        int sm2 = 0, sb = OFF - 1, sc = OFF, st = OFF + 1, s2 = OFF + 2, tpar = 0;
        for (int k = k0; k < k1; ++k) {
            layer(k, sm2, sb, sc, st, s2, tpar);
            sm2 = sb;
            sb = sc;
            sc = st;
            if constexpr (O4) {
                st = s2;
                if (++s2 == NB) {
                    s2 = 0;
                    tpar ^= 1;
                }
            } else {
                if (++st == NB) {
                    st = 0;
                    tpar ^= 1;
                }
            }
        }
    }
    if (consumers_sync_or<kThreads>(fail)) {
        if (tid == 0) atomicExch(A.err, MR_ERR_TIMEOUT);
        return;
    }
    if (DIVONLY) {
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

// ------------------------------------------------------------- intermediates (once per velocity)

// Periodic wrap of a coarse column index that is at most one period outside.
__device__ __forceinline__ int wrapc(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// The kernels below run one thread per (gx, coarse row J) of one dense layer
// k = blockIdx.y (32-bit index arithmetic; gx is the bundle column, coarse
// column I = gx - 4 wrapped).

// UO[k][j][gx], the outer U sub-face of coarse x-face I (R_y R_z of U: the z
// split first, shared by the M_y dense rows of J) times 1/(2 dx), and WY[k][j][gx], R_y of
// the full-area W on dense plane k (coarse W on the coarse planes,
// slab-balanced scrW on the inner ones); the top layer also writes plane Nz.
template <int MY>
__global__ void k_xprep_uowy(Grid<float> g, const float* __restrict__ U, const float* __restrict__ W,
                             const float* __restrict__ scrW, float* __restrict__ UO, float* __restrict__ WY, int nxg)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nxg * g.ny) return;
    const int k = blockIdx.y, J = t / nxg, gx = t - J * nxg;
    const int I = wrapc(gx - 4, g.nx), K = k / g.mz;
    float a[3];
    for (int p = 0; p < 3; ++p) {
        const int Jp = g.wy[3 * J + p];
        float s = 0.f;
        for (int q = 0; q < 3; ++q) s += g.Rz[3 * k + q] * U[((size_t)g.wz[3 * K + q] * g.ny + Jp) * g.nx + I];
        a[p] = s;
    }
#pragma unroll
    for (int b = 0; b < MY; ++b) {
        const int j = J * MY + b;
        UO[((size_t)k * g.Ny + j) * nxg + gx] =
            (g.Ry[3 * j] * a[0] + g.Ry[3 * j + 1] * a[1] + g.Ry[3 * j + 2] * a[2]) * (0.5f * g.inv_dx);
    }
    for (int kp = k; kp <= (k == g.Nz - 1 ? g.Nz : k); ++kp) {
        const int Kp = kp / g.mz;
        const float* src = (kp == Kp * g.mz) ? W + (size_t)Kp * g.ny * g.nx : scrW + (size_t)kp * g.ny * g.nx;
        float c[3];
        for (int p = 0; p < 3; ++p) c[p] = src[(size_t)g.wy[3 * J + p] * g.nx + I];
#pragma unroll
        for (int b = 0; b < MY; ++b) {
            const int j = J * MY + b;
            WY[((size_t)kp * g.Ny + j) * nxg + gx] = g.Ry[3 * j] * c[0] + g.Ry[3 * j + 1] * c[1] + g.Ry[3 * j + 2] * c[2];
        }
    }
}

// VR[k][j][gx]: full-coarse-width V on every dense y-face times 1/(2 dy), by
// the row balance (south to north) of stage Y; one thread per coarse row J
// (0..ny, row ny repeating row 0, periodic) walks its M_y - 1 inner faces.
template <int MY>
__global__ void k_xprep_vr(Grid<float> g, const float* __restrict__ V, const float* __restrict__ UO,
                           const float* __restrict__ WY, float* __restrict__ VR, int nxg)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nxg * (g.ny + 1)) return;
    const int k = blockIdx.y, J = t / nxg, gx = t - J * nxg;
    const int I = wrapc(gx - 4, g.nx), K = k / g.mz, Jf = (J == g.ny) ? 0 : J;
    float vz = 0.f;
    for (int q = 0; q < 3; ++q) vz += g.Rz[3 * k + q] * V[((size_t)g.wz[3 * K + q] * g.ny + Jf) * g.nx + I];
    const size_t vrow = (size_t)g.Ny + 1;
    const float hiy = 0.5f * g.inv_dy, two_dx = 2.f * g.dx;   // UO holds U / (2 dx)
    VR[((size_t)k * vrow + (size_t)J * MY) * nxg + gx] = vz * hiy;
    if (J == g.ny) return;
    const float dzk = g.dz[k];
    const int xi = I + 4, xe = wrapc(I + 1, g.nx) + 4;
    // the loads of all inner faces first (independent of the running balance)
    float uw[MY], ue[MY], wb[MY], wt[MY];
#pragma unroll
    for (int b = 0; b < MY - 1; ++b) {
        const size_t r = (size_t)k * g.Ny + J * MY + b;
        uw[b] = UO[r * nxg + xi] * two_dx;
        ue[b] = UO[r * nxg + xe] * two_dx;
        wb[b] = WY[r * nxg + xi];
        wt[b] = WY[(r + g.Ny) * nxg + xi];
    }
    float G = vz * g.DX * dzk;
#pragma unroll
    for (int b = 0; b < MY - 1; ++b) {
        const int j = J * MY + b;
        G = G - (ue[b] - uw[b]) * g.dy * dzk - (wt[b] - wb[b]) * g.DX * g.dy;
        VR[((size_t)k * vrow + j + 1) * nxg + gx] = G / (g.DX * dzk) * hiy;
    }
}

// All three intermediates of one coarse slab K (dense layers K M .. K M + M - 1)
// and one coarse row J (dense rows J M .. J M + M - 1): one block, M = mx = my = mz.
// Phase 1 forms UO and WY of the slab at the interior coarse columns in shared
// memory, the 3 x 3 coarse U values of a column (R_z x R_y windows) loaded once
// for the M layers, WY also on the next slab's first plane; phase 2 stores them
// for every bundle column (periodic ghosts included) and runs the row balance
// of VR from shared memory, so that UO and WY are not read back from HBM.  The
// arithmetic is that of k_xprep_uowy and k_xprep_vr, operation for operation.
template <int M>
__global__ void __launch_bounds__(128) k_xprep_slab(Grid<float> g, const float* __restrict__ U,
                                                     const float* __restrict__ V, const float* __restrict__ W,
                                                     const float* __restrict__ scrW, float* __restrict__ UO,
                                                     float* __restrict__ WY, float* __restrict__ VR, int nxg)
{
    extern __shared__ float s[];
    const int nx = g.nx, J = blockIdx.x, K = blockIdx.y, k0 = K * M;
    float* suo = s;                       // [M layers][M rows][nx]  U / (2 dx)
    float* swy = s + M * M * nx;          // [M + 1 planes][M rows][nx]
    int wz[3], wy[3];
    float rz[M][3], ry[M][3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        wz[q] = g.wz[3 * K + q];
        wy[q] = g.wy[3 * J + q];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            rz[m][q] = g.Rz[3 * (k0 + m) + q];
            ry[m][q] = g.Ry[3 * (J * M + m) + q];
        }
    }
    const float hx = 0.5f * g.inv_dx;
    const size_t cplane = (size_t)g.ny * nx;
    for (int I = threadIdx.x; I < nx; I += blockDim.x) {
        float u[3][3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int p = 0; p < 3; ++p) u[q][p] = U[((size_t)wz[q] * g.ny + wy[p]) * nx + I];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float a[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                float t = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) t += rz[m][q] * u[q][p];
                a[p] = t;
            }
#pragma unroll
            for (int b = 0; b < M; ++b)
                suo[(m * M + b) * nx + I] = (ry[b][0] * a[0] + ry[b][1] * a[1] + ry[b][2] * a[2]) * hx;
        }
#pragma unroll
        for (int mp = 0; mp <= M; ++mp) {
            // coarse W on the coarse planes, the slab-balanced scrW on the inner ones
            const float* src = (mp == 0 || mp == M) ? W + (size_t)(K + mp / M) * cplane : scrW + (size_t)(k0 + mp) * cplane;
            float c[3];
#pragma unroll
            for (int p = 0; p < 3; ++p) c[p] = src[(size_t)wy[p] * nx + I];
#pragma unroll
            for (int b = 0; b < M; ++b)
                swy[(mp * M + b) * nx + I] = ry[b][0] * c[0] + ry[b][1] * c[1] + ry[b][2] * c[2];
        }
    }
    __syncthreads();
    const size_t vrow = (size_t)g.Ny + 1;
    const float hiy = 0.5f * g.inv_dy, two_dx = 2.f * g.dx;
    const bool last_row = (J == g.ny - 1), top = (K == g.nz - 1);
    for (int gx = threadIdx.x; gx < nxg; gx += blockDim.x) {
        const int I = wrapc(gx - 4, nx), Ie = wrapc(I + 1, nx);
#pragma unroll
        for (int m = 0; m < M; ++m)
#pragma unroll
            for (int b = 0; b < M; ++b) {
                const size_t r = (size_t)(k0 + m) * g.Ny + J * M + b;
                UO[r * nxg + gx] = suo[(m * M + b) * nx + I];
                WY[r * nxg + gx] = swy[(m * M + b) * nx + I];
            }
        if (top)
#pragma unroll
            for (int b = 0; b < M; ++b)
                WY[((size_t)g.Nz * g.Ny + J * M + b) * nxg + gx] = swy[(M * M + b) * nx + I];
        float v[3], v0[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            v[q] = V[((size_t)wz[q] * g.ny + J) * nx + I];
            v0[q] = last_row ? V[(size_t)wz[q] * g.ny * nx + I] : 0.f;   // row ny repeats row 0
        }
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const int k = k0 + m;
            float vz = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) vz += rz[m][q] * v[q];
            VR[((size_t)k * vrow + (size_t)J * M) * nxg + gx] = vz * hiy;
            if (last_row) {
                float vz0 = 0.f;
#pragma unroll
                for (int q = 0; q < 3; ++q) vz0 += rz[m][q] * v0[q];
                VR[((size_t)k * vrow + (size_t)g.Ny) * nxg + gx] = vz0 * hiy;
            }
            const float dzk = g.dz[k];
            float G = vz * g.DX * dzk;
#pragma unroll
            for (int b = 0; b < M - 1; ++b) {
                const float uw = suo[(m * M + b) * nx + I] * two_dx, ue = suo[(m * M + b) * nx + Ie] * two_dx;
                const float wb = swy[(m * M + b) * nx + I], wt = swy[((m + 1) * M + b) * nx + I];
                G = G - (ue - uw) * g.dy * dzk - (wt - wb) * g.DX * g.dy;
                VR[((size_t)k * vrow + J * M + b + 1) * nxg + gx] = G / (g.DX * dzk) * hiy;
            }
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3-D FP32 tensor map of a [d2][d1][d0] array with a (b0, b1, b2) box.
bool map3(CUtensorMap* m, const float* base, int d0, int d1, int d2, int b0, int b1, int b2)
{
    EncodeTiledFn fn = encode();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
    cuuint64_t strides[2] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * d1 * 4};
    cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, (cuuint32_t)b2};
    cuuint32_t es[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps encoded once per (buffer, shape, box); the scalar buffers rotate
// through a handful of pointers, the intermediates are fixed.
bool cached_map3(CUtensorMap* out, const float* base, int d0, int d1, int d2, int b0, int b1, int b2)
{
    struct Entry { const float* p; int d[6]; CUtensorMap m; };
    constexpr int kCache = 128;
    static Entry cache[kCache];
    static int n = 0, next = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    const int key[6] = {d0, d1, d2, b0, b1, b2};
    for (int q = 0; q < n; ++q)
        if (cache[q].p == base && !memcmp(cache[q].d, key, sizeof key)) {
            *out = cache[q].m;
            return true;
        }
    if (!map3(out, base, d0, d1, d2, b0, b1, b2)) return false;
    Entry& e = cache[n < kCache ? n++ : (next = (next + 1) % kCache)];
    e.p = base;
    memcpy(e.d, key, sizeof key);
    e.m = *out;
    return true;
}

// Velocity intermediates of one coarse time level.
struct XSet {
    const float *wy, *uo, *vr;
};

template <int M, int KIND, bool LF, bool MT, bool O4, int TY>
cudaError_t launch_xt(const Grid<float>& g, XSet v0, XSet v1, float alpha, int nxg, const float* lc, int lcw,
                      const float* rx12, const float* w4, const float* Tm1, const float* T, float* Tp1, StepCoef c,
                      int* err, unsigned long long* divmax, cudaStream_t st)
{
    using L = XT<M, MT, O4, TY, (KIND != 0)>;
    if (lcw < L::LCW) return cudaErrorInvalidValue;
    static unsigned long long attr = 0;                   // one bit per device
    constexpr bool DIVONLY = KIND != 0;
    cudaError_t e = smem_optin(reinterpret_cast<const void*>(k_xfused<M, KIND, LF, MT, O4, TY>), (int)L::bytes, &attr);
    if (e != cudaSuccess) return e;
    XMaps maps;
    memset(&maps, 0, sizeof maps);
    if (!DIVONLY && (!cached_map3(&maps.tn, T, g.Nx, g.Ny, g.Nz, kTX, TY, 1) ||
                     !cached_map3(&maps.rn, T, g.Nx, g.Ny, g.Nz, kTX, L::HN, 1) ||
                     !cached_map3(&maps.xn, T, g.Nx, g.Ny, g.Nz, 4, TY, 1) ||
                     !cached_map3(&maps.tm, Tm1, g.Nx, g.Ny, g.Nz, kTX, TY, 1) ||
                     !cached_map3(&maps.rm, Tm1, g.Nx, g.Ny, g.Nz, kTX, 1, 1) ||
                     !cached_map3(&maps.xm, Tm1, g.Nx, g.Ny, g.Nz, 4, TY, 1)))
        return cudaErrorInvalidValue;
    auto set_maps = [&](const XSet& v, CUtensorMap* wy, CUtensorMap* uo, CUtensorMap* vr) {
        return cached_map3(wy, v.wy, nxg, g.Ny, g.Nz + 1, L::BXC, TY, 1) &&
               cached_map3(uo, v.uo, nxg, g.Ny, g.Nz, L::BXC, TY, 1) &&
               cached_map3(vr, v.vr, nxg, g.Ny + 1, g.Nz, L::BXC, TY + 1, 1);
    };
    if (!set_maps(v0, &maps.wy, &maps.uo, &maps.vr) || (MT && !set_maps(v1, &maps.wy1, &maps.uo1, &maps.vr1)) ||
        !cached_map3(&maps.lc, lc, lcw, g.Nz, 1, L::LCW, 1, 1))
        return cudaErrorInvalidValue;
    const int tiles = (g.Nx / kTX) * (g.Ny / TY);
    // ~20 waves of resident CTAs, but no chunk longer than 96 layers: on large
    // grids long chunks leave the resident CTAs far apart in z (measured on
    // 1536 x 1536 x 1024: 512 layers 8.8 ms, 64-128 layers 7.0 ms, 96 layers
    // 6.8 ms per step; on 512 x 512 x 384, 64x8 tiles: 8 layers 0.300 ms,
    // 12: 0.287, 16: 0.284, 26: 0.286, 48: 0.305)
    const int want = 152 * L::CTAS * 20;
    int nch = (want + tiles - 1) / tiles;
    nch = max(1, min(nch, g.Nz / 4));
    const int kcl = min((g.Nz + nch - 1) / nch, 96);
    const int chunks = (g.Nz + kcl - 1) / kcl;
    XArgs A{g, Tp1, lc, (float)c.a, (float)c.b, (float)c.gdt, kcl, err, divmax, {}, alpha, {}, {},
            ptx::kWaitNs, -1};
    if (KIND == 0) take_wait_injection(&A.stop_ring, &A.wait_ns);
    memcpy(A.rx, rx12, sizeof A.rx);
    if (O4) {
        memcpy(A.w4x, w4, sizeof A.w4x);
        memcpy(A.w4y, w4 + 4, sizeof A.w4y);
    }
    dim3 grid(chunks, g.Nx / kTX, g.Ny / TY);
    k_xfused<M, KIND, LF, MT, O4, TY><<<grid, L::THREADS, L::bytes, st>>>(maps, A);
    return cudaGetLastError();
}

// Tile height: 64x16 tiles (two CTAs per SM) when the grid offers at least
// ~8 waves of them in chunks of 96 layers, else 64x8 tiles (four CTAs per SM,
// so that a small grid still overlaps the chunks' start-up; 512 x 512 x 384:
// 0.315 -> 0.306 ms per step, while 1536 x 1536 x 1024 prefers 64x16).
int tile_rows(const Grid<float>& g)
{
    const long long tiles16 = (long long)(g.Nx / kTX) * (g.Ny / 16), chunks96 = (g.Nz + 95) / 96;
    return tiles16 * chunks96 >= 152LL * 2 * 8 ? 16 : 8;
}

template <int M, int KIND, bool LF, bool MT, bool O4>
cudaError_t launch_x(const Grid<float>& g, XSet v0, XSet v1, float alpha, int nxg, const float* lc, int lcw,
                     const float* rx12, const float* w4, const float* Tm1, const float* T, float* Tp1, StepCoef c,
                     int* err, unsigned long long* divmax, cudaStream_t st)
{
    // fourth order with two velocity levels keeps 64x16 tiles (its 64x8 ring
    // would be too shallow for the five live planes); single-level fourth order
    // on 64x8 tiles runs three CTAs per SM with a 7-slot ring and 128 registers
    // (512 x 512 x 384: 0.39 ms per step, vs 0.46 on 64x16 tiles)
    if constexpr (O4 && MT) {
        return launch_xt<M, KIND, LF, MT, O4, 16>(g, v0, v1, alpha, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, divmax,
                                                  st);
    } else {
        if (tile_rows(g) == 16)
            return launch_xt<M, KIND, LF, MT, O4, 16>(g, v0, v1, alpha, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err,
                                                      divmax, st);
        return launch_xt<M, KIND, LF, MT, O4, 8>(g, v0, v1, alpha, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, divmax,
                                                 st);
    }
}

template <int M, bool O4>
cudaError_t launch_step_m(const Grid<float>& g, XSet v0, const XSet* v1, float alpha, int nxg, const float* lc, int lcw,
                          const float* rx12, const float* w4, const float* Tm1, const float* T, float* Tp1, StepCoef c,
                          int* err, cudaStream_t st)
{
    const bool lf = (c.a == 1.0 && c.b == 0.0);
    if (v1) {
        return lf ? launch_x<M, 0, true, true, O4>(g, v0, *v1, alpha, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, nullptr, st)
                  : launch_x<M, 0, false, true, O4>(g, v0, *v1, alpha, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, nullptr, st);
    }
    return lf ? launch_x<M, 0, true, false, O4>(g, v0, v0, 0.f, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, nullptr, st)
              : launch_x<M, 0, false, false, O4>(g, v0, v0, 0.f, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, nullptr, st);
}

}  // namespace

cudaError_t launch_xfused_prep(const Grid<float>& g, const float* U, const float* V, const float* W, float* scrW,
                               float* WY, float* UO, float* VR, int nxg, cudaStream_t st)
{
    cudaError_t e = launch_column_balance<float>(g, U, V, W, scrW, st);
    if (e != cudaSuccess) return e;
    // one block per (coarse row, coarse slab) while the slab's UO and WY fit in
    // shared memory; else the two per-layer kernels (MR_XFUSED_PREP_LAYERS=1 in
    // the environment, read at every call, selects them on any grid so that
    // they stay tested)
    const int M = g.mz;
    const size_t smem = (size_t)(2 * M + 1) * M * g.nx * sizeof(float);
    const char* force = getenv("MR_XFUSED_PREP_LAYERS");
    if (g.mx == M && g.my == M && smem <= 200 * 1024 && !(force && force[0] == '1')) {
        static unsigned long long attr[2] = {0, 0};
        const void* kern = M == 4 ? reinterpret_cast<const void*>(k_xprep_slab<4>)
                                  : reinterpret_cast<const void*>(k_xprep_slab<2>);
        e = smem_optin(kern, 200 * 1024, &attr[M == 4]);   // the cap, once per device
        if (e != cudaSuccess) return e;
        if (M == 4)
            k_xprep_slab<4><<<dim3(g.ny, g.nz), 128, smem, st>>>(g, U, V, W, scrW, UO, WY, VR, nxg);
        else
            k_xprep_slab<2><<<dim3(g.ny, g.nz), 128, smem, st>>>(g, U, V, W, scrW, UO, WY, VR, nxg);
        return cudaGetLastError();
    }
    const unsigned row = (unsigned)((nxg * g.ny + 127) / 128), rowc = (unsigned)((nxg * (g.ny + 1) + 127) / 128);
    if (g.my == 4) k_xprep_uowy<4><<<dim3(row, g.Nz), 128, 0, st>>>(g, U, W, scrW, UO, WY, nxg);
    else k_xprep_uowy<2><<<dim3(row, g.Nz), 128, 0, st>>>(g, U, W, scrW, UO, WY, nxg);
    if (g.my == 4) k_xprep_vr<4><<<dim3(rowc, g.Nz), 128, 0, st>>>(g, V, UO, WY, VR, nxg);
    else k_xprep_vr<2><<<dim3(rowc, g.Nz), 128, 0, st>>>(g, V, UO, WY, VR, nxg);
    return cudaGetLastError();
}

cudaError_t launch_step_xfused_f32(const Grid<float>& g, const float* const setA[3], const float* const setB[3],
                                   double alpha, int nxg, const float* lc, int lcw, const float* rx12, const float* w4,
                                   const float* Tm1, const float* T, float* Tp1, StepCoef c, cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    const XSet v0{setA[0], setA[1], setA[2]};
    XSet v1{};
    const XSet* pv1 = nullptr;
    if (setB && alpha != 0.0) {
        v1 = XSet{setB[0], setB[1], setB[2]};
        pv1 = &v1;
    }
    const float a = (float)alpha;
    if (g.order4)
        return g.mx == 4 ? launch_step_m<4, true>(g, v0, pv1, a, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, st)
                         : launch_step_m<2, true>(g, v0, pv1, a, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, st);
    return g.mx == 4 ? launch_step_m<4, false>(g, v0, pv1, a, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, st)
                     : launch_step_m<2, false>(g, v0, pv1, a, nxg, lc, lcw, rx12, w4, Tm1, T, Tp1, c, err, st);
}

// kind 1: max |divergence|, kind 2: max CFL rate, as a double in partials[0]
// (the other blocks - 1 partials are zeroed).
cudaError_t launch_xfused_max_f32(const Grid<float>& g, int kind, const float* WY, const float* UO, const float* VR,
                                  int nxg, const float* lc, int lcw, const float* rx12, double* partials, int blocks,
                                  cudaStream_t st)
{
    int* err = fused_error_flag();
    if (!err) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(partials, 0, (size_t)blocks * sizeof(double), st);
    if (e != cudaSuccess) return e;
    unsigned long long* dm = reinterpret_cast<unsigned long long*>(partials);
    StepCoef c{0, 0, 0};
    const XSet v{WY, UO, VR};
    if (g.mx == 4)
        return kind == 2 ? launch_x<4, 2, false, false, false>(g, v, v, 0.f, nxg, lc, lcw, rx12, nullptr, nullptr, nullptr,
                                                               nullptr, c, err, dm, st)
                         : launch_x<4, 1, false, false, false>(g, v, v, 0.f, nxg, lc, lcw, rx12, nullptr, nullptr, nullptr,
                                                               nullptr, c, err, dm, st);
    return kind == 2 ? launch_x<2, 2, false, false, false>(g, v, v, 0.f, nxg, lc, lcw, rx12, nullptr, nullptr, nullptr,
                                                           nullptr, c, err, dm, st)
                     : launch_x<2, 1, false, false, false>(g, v, v, 0.f, nxg, lc, lcw, rx12, nullptr, nullptr, nullptr,
                                                           nullptr, c, err, dm, st);
}

// Per-layer constants of the split-x and fully fused kernels, [Nz][32] floats,
// all folded on the host in FP64.  The pair entries hold each value twice, for
// the packed pair arithmetic of the update:
//   0: 1/dz, 1: 1/(2 dz), 2: dz, 4..7: fourth order only, the weights of planes
//   k-2 .. k+1 at face k (the first layer of a chunk); second order (read by the
//   fully fused kernel, pairs): 4..7 the linear-interpolation weights of T_k and
//   T_{k+1} at face k+1, 8..11 1/dz and cdn of layer k+1 (zero on the last layer);
//   12..19 (pairs): second order, the linear-interpolation weights of T_{k-1},
//   T_k at face k and the negated weights of T_k, T_{k+1} at face k+1, each
//   times 1/dz; fourth order, the weights of planes k-1 .. k+2 at face k+1;
//   20..27 (pairs): kappa/(dz d) toward the centre (or plate) below and above,
//   the negated diagonal 2 kappa/dx^2 + 2 kappa/dy^2 + cdn + cup, the plate term
//   (Dirichlet plates: cdn T_bottom on the first layer, cup T_top on the last);
//   28..31: fourth order only, the pairs 1/dz and -1/dz.
// The kernels read zeros for the planes beyond the plates, where W is zero.
std::vector<float> xfused_layer_constants(int Nz, const double* zf, const double* zc, const double* dz, double kappa,
                                          double dx, double dy, bool dirichlet, const double* f4z, int* lcw)
{
    *lcw = 32;
    std::vector<float> lc((size_t)Nz * *lcw, 0.f);
    const double kx2 = kappa / (dx * dx), ky2 = kappa / (dy * dy);
    for (int k = 0; k < Nz; ++k) {
        float* q = &lc[(size_t)k * *lcw];
        const double dzk = dz[k], idz = 1.0 / dzk;
        const double below = k > 0 ? zc[k] - zc[k - 1] : zc[0] - zf[0];
        const double above = k < Nz - 1 ? zc[k + 1] - zc[k] : zf[Nz] - zc[Nz - 1];
        const double cdn = (k > 0 || dirichlet) ? kappa / (dzk * below) : 0.0;
        const double cup = (k < Nz - 1 || dirichlet) ? kappa / (dzk * above) : 0.0;
        double zw[4] = {0.0, 0.0, 0.0, 0.0};
        if (f4z) {
            for (int c = 0; c < 4; ++c) {
                zw[c] = f4z[4 * (size_t)(k + 1) + c];             // face k+1: planes k-1 .. k+2
                q[4 + c] = (float)f4z[4 * (size_t)k + c];       // face k: planes k-2 .. k+1
            }
            q[28] = q[29] = (float)idz;
            q[30] = q[31] = (float)-idz;
        } else {
            if (k < Nz - 1) {
                const double dn = dz[k + 1], cnext = kappa / (dn * (zc[k + 1] - zc[k]));
                q[4] = q[5] = (float)(dn / (dzk + dn));
                q[6] = q[7] = (float)(dzk / (dzk + dn));
                q[10] = q[11] = (float)cnext;
            }
            q[8] = q[9] = (float)idz;
            if (k > 0) {
                zw[0] = dzk / (dz[k - 1] + dzk) * idz;
                zw[1] = dz[k - 1] / (dz[k - 1] + dzk) * idz;
            }
            if (k < Nz - 1) {
                zw[2] = -(dz[k + 1] / (dzk + dz[k + 1]) * idz);
                zw[3] = -(dzk / (dzk + dz[k + 1]) * idz);
            }
        }
        double plate = 0.0;
        if (dirichlet && k == 0) plate += cdn * (double)kTBottom;
        if (dirichlet && k == Nz - 1) plate += cup * (double)kTTop;
        q[0] = (float)idz;
        q[1] = (float)(0.5 * idz);
        q[2] = (float)dzk;
        const double pv[8] = {zw[0], zw[1], zw[2], zw[3], cdn, cup, -(2.0 * kx2 + 2.0 * ky2 + cdn + cup), plate};
        for (int c = 0; c < 8; ++c) q[12 + 2 * c] = q[13 + 2 * c] = (float)pv[c];
    }
    return lc;
}

}  // namespace mr
