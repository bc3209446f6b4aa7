// Hand-written discrete adjoint of the scalar path (stored-velocity mode).
//
// Loss L = sum_s wnu[s] Nu_bot(T^s) + wvar[s] Var(T^s) over the levels
// s = 0..S of an S-step run.  The forward scheme (Section 2.2, Eq. 5) is
//   T^{s+1} = a_s T^{s-1} + b_s T^s + g_s dt [C(u; T^s) + D(T^{s-1})],
// affine in T for fixed u and bilinear in (u, T) through C.  The backward sweep
// carries mu = lambda / Vol (adjoint per unit volume):
//   mu^s     += b_s mu^{s+1} + g_s dt C^T mu^{s+1}
//   mu^{s-1}  = direct_{s-1} + a_s mu^{s+1} + g_s dt D^T mu^{s+1}
// (Euler start: mu^0 += mu^1 + dt (C^T + D^T) mu^1).  In this form D^T is the
// forward diffusion stencil itself (D is symmetric in the volume-weighted inner
// product, plate values zero), and C^T is gathered per cell:
//   (C^T mu)_c = sum_faces (A_f / Vol_c) u_f w_{c,f} (mu_R - mu_L),
// w_{c,f} being the weight of T_c in the face value T_f.  The face gradient is
//   dL/du_f += g_s dt A_f T^s_f (mu_R - mu_L),
// accumulated by the cell that owns the face (its west, south and bottom
// faces), so no atomics are needed: in the working precision over one
// checkpoint segment, then added into FP64 totals (GB300's FP64 pipe is a
// small fraction of its FP32 one).  The coarse gradient is the
// transpose of the refinement (Section 3.2), applied once at the end (it is
// linear and fixed, so sum_s P^T g_s = P^T sum_s g_s).
//
// Checkpoints: the forward stores (T^{s-1}, T^s) every k steps; the backward
// recomputes each segment's levels from its checkpoint before sweeping it.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr int kThreads = 256;
inline unsigned nblk(size_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// direct term of one level: mu = s_nu * (k == 0) + s_var * (T - mean)
template <typename P>
__global__ void k_adj_direct(Grid<P> g, const P* __restrict__ T, double s_nu_bottom, double s_var, double mean,
                             P* __restrict__ mu)
{
    const size_t plane = (size_t)g.Nx * g.Ny, n = plane * g.Nz;
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x) {
        double v = 0.0;
        if (m < plane) v += s_nu_bottom;
        if (s_var != 0.0) v += s_var * ((double)T[m] - mean);
        mu[m] = (P)v;
    }
}

// One backward step (thread per cell).  Mn = mu^{s+1} (complete), Mc = mu^s
// (accumulated), Mp = mu^{s-1} (written: its direct term -- s_nu on the bottom
// layer, s_var (T^{s-1} - mean) everywhere -- plus this step's share);
// EULER: the s = 0 start, which feeds everything into Mc.
template <typename P, bool EULER>
__global__ void __launch_bounds__(256) k_adj_step(Grid<P> g, const P* __restrict__ Us, const P* __restrict__ Vs,
                                                  const P* __restrict__ Ws, const P* __restrict__ T,
                                                  const P* __restrict__ Tprev, const P* __restrict__ Mn,
                                                  P* __restrict__ Mc, P* __restrict__ Mp, double s_nu, double s_var,
                                                  double mean_prev, P* __restrict__ gU,
                                                  P* __restrict__ gV, P* __restrict__ gW, P a, P b, P gdt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.Nx || j >= g.Ny) return;
    const size_t plane = (size_t)g.Nx * g.Ny;
    const size_t m = (size_t)k * plane + (size_t)j * g.Nx + i;
    const P half = P(0.5);
    const P mc = Mn[m], tc = T[m];
    P ct = 0, dxs = 0, dys = 0, dzs = 0, cy = 0, cz = 0;
    const size_t urow = ((size_t)k * g.Ny + j) * g.ufx;
    // x faces
    if (!(g.walls && i == 0)) {
        const int iw = (i == 0) ? g.Nx - 1 : i - 1;
        const size_t mw = m - i + iw;
        const P uw = Us[urow + i], mw_ = Mn[mw];
        ct += uw * half * (mc - mw_);
        dxs -= mc - mw_;
        gU[urow + i] += gdt * (g.dy * g.dz[k]) * (half * (T[mw] + tc)) * (mc - mw_);
    }
    if (!(g.walls && i == g.Nx - 1)) {
        const int ie = (i == g.Nx - 1) ? 0 : i + 1;
        const int fe = g.walls ? i + 1 : ie;
        const P me_ = Mn[m - i + ie];
        ct += Us[urow + fe] * half * (me_ - mc);
        dxs += me_ - mc;
    }
    // y faces
    const size_t vrow = ((size_t)k * g.vfy + j) * g.Nx + i;
    if (!(g.walls && j == 0)) {
        const int js = (j == 0) ? g.Ny - 1 : j - 1;
        const size_t ms = m + ((ptrdiff_t)js - j) * g.Nx;
        const P ms_ = Mn[ms];
        cy += Vs[vrow] * half * (mc - ms_);
        dys -= mc - ms_;
        gV[vrow] += gdt * (g.dx * g.dz[k]) * (half * (T[ms] + tc)) * (mc - ms_);
    }
    if (!(g.walls && j == g.Ny - 1)) {
        const int jn = (j == g.Ny - 1) ? 0 : j + 1;
        const int fn = g.walls ? j + 1 : jn;
        const P mn_ = Mn[m + ((ptrdiff_t)jn - j) * g.Nx];
        cy += Vs[((size_t)k * g.vfy + fn) * g.Nx + i] * half * (mn_ - mc);
        dys += mn_ - mc;
    }
    // z faces (plates: no advective flux, Dirichlet / zero-flux diffusion with zero plate value)
    if (k > 0) {
        const P mb_ = Mn[m - plane];
        cz += Ws[m] * g.whi[k] * (mc - mb_);
        dzs -= g.cdn[k] * (mc - mb_);
        gW[m] += gdt * (g.dx * g.dy) * (g.wlo[k] * T[m - plane] + g.whi[k] * tc) * (mc - mb_);
    } else {
        dzs -= g.cdn[0] * mc;
    }
    if (k < g.Nz - 1) {
        const P mt_ = Mn[m + plane];
        cz += Ws[m + plane] * g.wlo[k + 1] * (mt_ - mc);
        dzs += g.cup[k] * (mt_ - mc);
    } else {
        dzs -= g.cup[k] * mc;
    }
    const P CT = ct * g.inv_dx + cy * g.inv_dy + cz * g.inv_dz[k];
    const P DT = g.kx2 * dxs + g.ky2 * dys + dzs;
    if (EULER) {
        Mc[m] = Mc[m] + mc + gdt * (CT + DT);
    } else {
        Mc[m] = Mc[m] + b * mc + gdt * CT;
        double d = (k == 0) ? s_nu : 0.0;
        if (s_var != 0.0) d += s_var * ((double)Tprev[m] - mean_prev);
        Mp[m] = (P)d + a * mc + gdt * DT;
    }
}

// The same backward step for periodic x and y, folded for the FP64 pipe
// like the forward's k_step_periodic (about 42 FP operations per cell instead
// of 60): the adjoint differences of the six neighbours are formed once, the
// planes beyond the plates read as zero (which gives the plate terms of D^T),
// the z weights times 1/dz come from g.lz, and the face-gradient factors
// gdt A_f / 2 (x, y) and gdt A_z arrive as cx, cy, cz per unit dz.
template <typename P, bool EULER>
__global__ void __launch_bounds__(256) k_adj_step_periodic(Grid<P> g, const P* __restrict__ Us,
                                                           const P* __restrict__ Vs, const P* __restrict__ Ws,
                                                           const P* __restrict__ T, const P* __restrict__ Tprev,
                                                           const P* __restrict__ Mn, P* __restrict__ Mc,
                                                           P* __restrict__ Mp, double s_nu, double s_var,
                                                           double mean_prev, P* __restrict__ gU, P* __restrict__ gV,
                                                           P* __restrict__ gW, P a, P b, P gdt, P cx, P cy, P cz)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.Nx || j >= g.Ny) return;
    const size_t plane = (size_t)g.Nx * g.Ny;
    const size_t row = (size_t)j * g.Nx, m = (size_t)k * plane + row + i;
    const P* L = g.lz + 8 * k;
    const int iw = i == 0 ? g.Nx - 1 : i - 1, ie = i == g.Nx - 1 ? 0 : i + 1;
    const int js = j == 0 ? g.Ny - 1 : j - 1, jn = j == g.Ny - 1 ? 0 : j + 1;
    const size_t mw = m - i + iw, me = m - i + ie;
    const size_t ms = m - row + (size_t)js * g.Nx, mn = m - row + (size_t)jn * g.Nx;
    const bool lo = k > 0, hi = k < g.Nz - 1;
    const P mc = Mn[m], tc = T[m];
    const P dw = mc - Mn[mw], de = Mn[me] - mc, ds = mc - Mn[ms], dn = Mn[mn] - mc;
    const P db = mc - (lo ? Mn[m - plane] : P(0)), dt = (hi ? Mn[m + plane] : P(0)) - mc;
    const size_t urow = ((size_t)k * g.Ny + j) * g.Nx, vrow = (size_t)k * plane;
    const P uw = Us[urow + i], wb = Ws[m];
    const P CT = g.hx * (uw * dw + Us[urow + ie] * de) + g.hy * (Vs[vrow + row + i] * ds + Vs[vrow + (size_t)jn * g.Nx + i] * dn) +
                 ((wb * L[1]) * db - (Ws[m + plane] * L[2]) * dt);
    const P DT = g.kx2 * (de - dw) + g.ky2 * (dn - ds) + L[5] * dt - L[4] * db;
    // face gradients of the cell's west, south and bottom faces
    const P dzk = g.dz[k];
    gU[urow + i] += (cx * dzk) * (T[mw] + tc) * dw;
    gV[vrow + row + i] += (cy * dzk) * (T[ms] + tc) * ds;
    if (lo) gW[m] += (cz * dzk) * (L[0] * T[m - plane] + L[1] * tc) * db;
    if (EULER) {
        Mc[m] = Mc[m] + mc + gdt * (CT + DT);
    } else {
        Mc[m] = Mc[m] + b * mc + gdt * CT;
        double d = (k == 0) ? s_nu : 0.0;
        if (s_var != 0.0) d += s_var * ((double)Tprev[m] - mean_prev);
        Mp[m] = (P)d + a * mc + gdt * DT;
    }
}

// totals (FP64) += segment sums (FP32), which are cleared
__global__ void k_flush_faces(float* __restrict__ seg, double* __restrict__ tot, size_t n)
{
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x) {
        tot[m] += (double)seg[m];
        seg[m] = 0.f;
    }
}

template <typename P>
__global__ void k_times_volume(Grid<P> g, const P* __restrict__ mu, int dst_f64, void* __restrict__ out)
{
    const size_t plane = (size_t)g.Nx * g.Ny, n = plane * g.Nz;
    const double dxdy = (double)g.dx * (double)g.dy;
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x) {
        const double v = (double)mu[m] * dxdy * (double)g.dz[m / plane];
        if (dst_f64) ((double*)out)[m] = v;
        else ((float*)out)[m] = (float)v;
    }
}

// ------------------------------------------------------------- refinement transpose (FP64)
// The passes of the refinement in reverse order, each replaced by its
// adjoint; scatter-adds use FP64 atomics.

__global__ void k_t_stage_x(Grid<double> g, double* aUs, double* aVs, double* aWs)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.Ny * g.nx;
    if (t >= n) return;
    const int I = (int)(t % g.nx), j = (int)((t / g.nx) % g.Ny), k = (int)(t / ((size_t)g.nx * g.Ny));
    const int jn = g.walls ? j + 1 : (j + 1) % g.Ny;
    const double dzk = g.dz[k];
    const size_t urow = ((size_t)k * g.Ny + j) * g.ufx;
    double aH = 0.0;
    for (int a = g.mx - 2; a >= 0; --a) {
        const int i = I * g.mx + a;
        aH += aUs[urow + i + 1] / (g.dy * dzk);
        aUs[urow + i + 1] = 0.0;
        atomicAdd(&aVs[((size_t)k * g.vfy + jn) * g.Nx + i], -aH * g.dx * dzk);
        atomicAdd(&aVs[((size_t)k * g.vfy + j) * g.Nx + i], aH * g.dx * dzk);
        atomicAdd(&aWs[((size_t)(k + 1) * g.Ny + j) * g.Nx + i], -aH * g.dx * g.dy);
        atomicAdd(&aWs[((size_t)k * g.Ny + j) * g.Nx + i], aH * g.dx * g.dy);
    }
    atomicAdd(&aUs[urow + (size_t)I * g.mx], aH * g.dy * dzk);
}

__global__ void k_t_split_v(Grid<double> g, double* aVs, double* aVrow)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t rows = (size_t)g.ny * (g.my - 1), n = (size_t)g.Nz * rows * g.Nx;
    if (t >= n) return;
    const int i = (int)(t % g.Nx), jj = (int)((t / g.Nx) % rows), k = (int)(t / ((size_t)g.Nx * rows));
    const int j = (jj / (g.my - 1)) * g.my + jj % (g.my - 1) + 1;
    const int I = i / g.mx;
    const size_t f = ((size_t)k * g.vfy + j) * g.Nx + i;
    const double v = aVs[f];
    aVs[f] = 0.0;
    for (int p = 0; p < 3; ++p)
        atomicAdd(&aVrow[((size_t)k * g.vfy + j) * g.nx + g.wx[3 * I + p]], g.Rx[3 * i + p] * v);
}

__global__ void k_t_row_balance(Grid<double> g, double* aUs, double* aVs, double* aWs, const double* aVrow)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.ny * g.nx;
    if (t >= n) return;
    const int I = (int)(t % g.nx), J = (int)((t / g.nx) % g.ny), k = (int)(t / ((size_t)g.nx * g.ny));
    const int Ie = g.walls ? I + 1 : (I + 1) % g.nx;
    const double dzk = g.dz[k];
    double aG = 0.0;
    for (int b = g.my - 2; b >= 0; --b) {
        const int j = J * g.my + b;
        aG += aVrow[((size_t)k * g.vfy + j + 1) * g.nx + I] / (g.DX * dzk);
        const size_t urow = ((size_t)k * g.Ny + j) * g.ufx;
        atomicAdd(&aUs[urow + (size_t)Ie * g.mx], -aG * g.dy * dzk);
        atomicAdd(&aUs[urow + (size_t)I * g.mx], aG * g.dy * dzk);
        for (int a = 0; a < g.mx; ++a) {
            atomicAdd(&aWs[((size_t)(k + 1) * g.Ny + j) * g.Nx + I * g.mx + a], -aG * g.dy * g.dx);
            atomicAdd(&aWs[((size_t)k * g.Ny + j) * g.Nx + I * g.mx + a], aG * g.dy * g.dx);
        }
    }
    for (int a = 0; a < g.mx; ++a)
        atomicAdd(&aVs[((size_t)k * g.vfy + (size_t)J * g.my) * g.Nx + I * g.mx + a], aG * dzk * g.dx);
}

__global__ void k_t_split_w(Grid<double> g, double* aWs, double* aWc)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t planes = (size_t)g.nz * (g.mz - 1), n = planes * g.Ny * g.Nx;
    if (t >= n) return;
    const int i = (int)(t % g.Nx), j = (int)((t / g.Nx) % g.Ny), kk = (int)(t / ((size_t)g.Nx * g.Ny));
    const int k = (kk / (g.mz - 1)) * g.mz + kk % (g.mz - 1) + 1;
    const int I = i / g.mx, J = j / g.my;
    const size_t f = ((size_t)k * g.Ny + j) * g.Nx + i;
    const double v = aWs[f];
    aWs[f] = 0.0;
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            atomicAdd(&aWc[((size_t)k * g.ny + g.wy[3 * J + q]) * g.nx + g.wx[3 * I + p]],
                      g.Rx[3 * i + p] * g.Ry[3 * j + q] * v);
}

__global__ void k_t_column_balance(Grid<double> g, const double* aWc, double* gU, double* gV, double* gW)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.nz * g.ny * g.nx;
    if (t >= n) return;
    const int I = (int)(t % g.nx), J = (int)((t / g.nx) % g.ny), K = (int)(t / ((size_t)g.nx * g.ny));
    const int Ie = g.walls ? I + 1 : (I + 1) % g.nx;
    const int Jn = g.walls ? J + 1 : (J + 1) % g.ny;
    double aF = 0.0;
    for (int c = 1; c <= g.mz - 1; ++c) {
        const int k = K * g.mz + c;
        aF += aWc[((size_t)k * g.ny + J) * g.nx + I] / (g.DX * g.DY);
        const double au = aF * g.DY * g.dz[k], av = aF * g.DX * g.dz[k];
        for (int q = 0; q < 3; ++q) {
            const double r = g.Rz[3 * k + q];
            const int Kq = g.wz[3 * K + q];
            atomicAdd(&gU[((size_t)Kq * g.ny + J) * g.cux + Ie], r * au);
            atomicAdd(&gU[((size_t)Kq * g.ny + J) * g.cux + I], -r * au);
            atomicAdd(&gV[((size_t)Kq * g.cvy + Jn) * g.nx + I], r * av);
            atomicAdd(&gV[((size_t)Kq * g.cvy + J) * g.nx + I], -r * av);
        }
    }
    atomicAdd(&gW[((size_t)(K + 1) * g.ny + J) * g.nx + I], aF * g.DX * g.DY);
}

__global__ void k_t_outer_u(Grid<double> g, const double* aUs, double* gU)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.Ny * g.cux;
    if (t >= n) return;
    const int I = (int)(t % g.cux), j = (int)((t / g.cux) % g.Ny), k = (int)(t / ((size_t)g.cux * g.Ny));
    const int J = j / g.my, K = k / g.mz;
    const double v = aUs[((size_t)k * g.Ny + j) * g.ufx + (size_t)I * g.mx];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            atomicAdd(&gU[((size_t)g.wz[3 * K + q] * g.ny + g.wy[3 * J + p]) * g.cux + I], g.Ry[3 * j + p] * g.Rz[3 * k + q] * v);
}

__global__ void k_t_outer_v(Grid<double> g, const double* aVs, double* gV)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.cvy * g.Nx;
    if (t >= n) return;
    const int i = (int)(t % g.Nx), J = (int)((t / g.Nx) % g.cvy), k = (int)(t / ((size_t)g.Nx * g.cvy));
    const int I = i / g.mx, K = k / g.mz;
    const double v = aVs[((size_t)k * g.vfy + (size_t)J * g.my) * g.Nx + i];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            atomicAdd(&gV[((size_t)g.wz[3 * K + q] * g.cvy + J) * g.nx + g.wx[3 * I + p]], g.Rx[3 * i + p] * g.Rz[3 * k + q] * v);
}

__global__ void k_t_outer_w(Grid<double> g, const double* aWs, double* gW)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)(g.nz + 1) * g.Ny * g.Nx;
    if (t >= n) return;
    const int i = (int)(t % g.Nx), j = (int)((t / g.Nx) % g.Ny), K = (int)(t / ((size_t)g.Nx * g.Ny));
    const int I = i / g.mx, J = j / g.my;
    const double v = aWs[((size_t)K * g.mz * g.Ny + j) * g.Nx + i];
    for (int p = 0; p < 3; ++p)
        for (int q = 0; q < 3; ++q)
            atomicAdd(&gW[((size_t)K * g.ny + g.wy[3 * J + q]) * g.nx + g.wx[3 * I + p]], g.Rx[3 * i + p] * g.Ry[3 * j + q] * v);
}

}  // namespace

// P^T: dense face gradients (consumed) -> coarse gradients (zeroed first).
cudaError_t launch_refine_transpose(const Grid<double>& g, double* aUs, double* aVs, double* aWs, double* aWc,
                                    double* aVrow, double* gU, double* gV, double* gW, size_t ncU, size_t ncV,
                                    size_t ncW, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(gU, 0, ncU * 8, st)) || (e = cudaMemsetAsync(gV, 0, ncV * 8, st)) ||
        (e = cudaMemsetAsync(gW, 0, ncW * 8, st)))
        return e;
    if ((e = cudaMemsetAsync(aWc, 0, (size_t)(g.Nz + 1) * g.ny * g.nx * 8, st)) ||
        (e = cudaMemsetAsync(aVrow, 0, (size_t)g.Nz * g.vfy * g.nx * 8, st)))
        return e;
    size_t n;
    if (g.mx > 1) { n = (size_t)g.Nz * g.Ny * g.nx; k_t_stage_x<<<nblk(n), kThreads, 0, st>>>(g, aUs, aVs, aWs); }
    if (g.my > 1) {
        n = (size_t)g.Nz * g.ny * (g.my - 1) * g.Nx;
        k_t_split_v<<<nblk(n), kThreads, 0, st>>>(g, aVs, aVrow);
        n = (size_t)g.Nz * g.ny * g.nx;
        k_t_row_balance<<<nblk(n), kThreads, 0, st>>>(g, aUs, aVs, aWs, aVrow);
    }
    if (g.mz > 1) {
        n = (size_t)g.nz * (g.mz - 1) * g.Ny * g.Nx;
        k_t_split_w<<<nblk(n), kThreads, 0, st>>>(g, aWs, aWc);
        n = (size_t)g.nz * g.ny * g.nx;
        k_t_column_balance<<<nblk(n), kThreads, 0, st>>>(g, aWc, gU, gV, gW);
    }
    n = (size_t)g.Nz * g.Ny * g.cux;
    k_t_outer_u<<<nblk(n), kThreads, 0, st>>>(g, aUs, gU);
    n = (size_t)g.Nz * g.cvy * g.Nx;
    k_t_outer_v<<<nblk(n), kThreads, 0, st>>>(g, aVs, gV);
    n = (size_t)(g.nz + 1) * g.Ny * g.Nx;
    k_t_outer_w<<<nblk(n), kThreads, 0, st>>>(g, aWs, gW);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_adj_direct(const Grid<P>& g, const P* T, double s_nu_bottom, double s_var, double mean, P* mu,
                              cudaStream_t st)
{
    k_adj_direct<P><<<152 * 8, kThreads, 0, st>>>(g, T, s_nu_bottom, s_var, mean, mu);
    return cudaGetLastError();
}

cudaError_t launch_flush_faces(float* seg, double* tot, size_t n, cudaStream_t st)
{
    k_flush_faces<<<152 * 8, kThreads, 0, st>>>(seg, tot, n);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_adj_step(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, const P* T, const P* Tprev,
                            const P* Mn, P* Mc, P* Mp, double s_nu, double s_var, double mean_prev, P* gU,
                            P* gV, P* gW, StepCoef c, bool euler, cudaStream_t st)
{
    dim3 blk(64, 4);
    dim3 grd((g.Nx + blk.x - 1) / blk.x, (g.Ny + blk.y - 1) / blk.y, g.Nz);
    if (!g.walls) {
        // face-gradient factors: gdt dy / 2 and gdt dx / 2 per unit dz_k (x and y
        // faces), gdt dx dy (z faces, times dz_k in the kernel to undo the 1/dz_k
        // of the g.lz weights)
        const double dx = (double)g.dx, dy = (double)g.dy;
        const P cx = (P)(c.gdt * 0.5 * dy), cy = (P)(c.gdt * 0.5 * dx), cz = (P)(c.gdt * dx * dy);
        if (euler)
            k_adj_step_periodic<P, true><<<grd, blk, 0, st>>>(g, Us, Vs, Ws, T, Tprev, Mn, Mc, Mp, s_nu, s_var,
                                                              mean_prev, gU, gV, gW, (P)c.a, (P)c.b, (P)c.gdt,
                                                              cx, cy, cz);
        else
            k_adj_step_periodic<P, false><<<grd, blk, 0, st>>>(g, Us, Vs, Ws, T, Tprev, Mn, Mc, Mp, s_nu, s_var,
                                                               mean_prev, gU, gV, gW, (P)c.a, (P)c.b, (P)c.gdt,
                                                               cx, cy, cz);
        return cudaGetLastError();
    }
    if (euler)
        k_adj_step<P, true><<<grd, blk, 0, st>>>(g, Us, Vs, Ws, T, Tprev, Mn, Mc, Mp, s_nu, s_var, mean_prev, gU, gV,
                                                 gW, (P)c.a, (P)c.b, (P)c.gdt);
    else
        k_adj_step<P, false><<<grd, blk, 0, st>>>(g, Us, Vs, Ws, T, Tprev, Mn, Mc, Mp, s_nu, s_var, mean_prev, gU,
                                                  gV, gW, (P)c.a, (P)c.b, (P)c.gdt);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_times_volume(const Grid<P>& g, const P* mu, int dst_dtype, void* out, cudaStream_t st)
{
    k_times_volume<P><<<152 * 8, kThreads, 0, st>>>(g, mu, dst_dtype == MR_F64 ? 1 : 0, out);
    return cudaGetLastError();
}

#define MR_INST(P)                                                                                                 \
    template cudaError_t launch_adj_direct<P>(const Grid<P>&, const P*, double, double, double, P*, cudaStream_t); \
    template cudaError_t launch_adj_step<P>(const Grid<P>&, const P*, const P*, const P*, const P*, const P*,        \
                                            const P*, P*, P*, double, double, double, P*, P*, P*,                  \
                                            StepCoef, bool, cudaStream_t);                                         \
    template cudaError_t launch_times_volume<P>(const Grid<P>&, const P*, int, void*, cudaStream_t);
MR_INST(double)
MR_INST(float)
#undef MR_INST

}  // namespace mr
