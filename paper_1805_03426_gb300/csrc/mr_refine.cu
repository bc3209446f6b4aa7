// Divergence-free refinement of the coarse staggered velocity onto the dense
// grid (Section 3.2), as a chain of small kernels; used by MR_VEL_STORED and
// to export dense faces.  The fused FP32 step kernel (mr_fused.cu) performs
// the same stages inside shared memory instead.
//
// Stages (3-D reading of the paper's 2-D procedure, z first, then y, then x):
//   0  every coarse face value is split over its sub-faces with the tensor
//      product of the two tangential R matrices (V_s = R V, R = A_s A^-1);
//   Z  per coarse cell, the full-area W on the inner dense z-planes follows
//      from the mass balance of each dense slab, top-down, and is split over
//      the sub-faces with R_x (x) R_y applied to the neighbouring columns;
//   Y  per dense layer, the full-width V on the inner y-planes follows from
//      the balance of each row, south to north, and is split along x with R_x;
//   X  per dense row, U on the inner x-faces follows from each dense cell's
//      balance, west to east.
#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(size_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// Stage 0, x-normal faces on the coarse x-planes: thread per (k, j, I).
template <typename P>
__global__ void k_outer_u(Grid<P> g, const P* __restrict__ U, P* __restrict__ Us)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.Ny * g.cux;
    if (t >= n) return;
    int I = (int)(t % g.cux);
    int j = (int)((t / g.cux) % g.Ny);
    int k = (int)(t / ((size_t)g.cux * g.Ny));
    int J = j / g.my, K = k / g.mz;
    P s = P(0);
    for (int p = 0; p < 3; ++p) {
        int Jp = g.wy[3 * J + p];
        for (int q = 0; q < 3; ++q) {
            int Kq = g.wz[3 * K + q];
            s += g.Ry[3 * j + p] * g.Rz[3 * k + q] * U[((size_t)Kq * g.ny + Jp) * g.cux + I];
        }
    }
    Us[((size_t)k * g.Ny + j) * g.ufx + (size_t)I * g.mx] = s;
}

// Stage 0, y-normal faces on the coarse y-planes: thread per (k, J, i).
template <typename P>
__global__ void k_outer_v(Grid<P> g, const P* __restrict__ V, P* __restrict__ Vs)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.cvy * g.Nx;
    if (t >= n) return;
    int i = (int)(t % g.Nx);
    int J = (int)((t / g.Nx) % g.cvy);
    int k = (int)(t / ((size_t)g.Nx * g.cvy));
    int I = i / g.mx, K = k / g.mz;
    P s = P(0);
    for (int p = 0; p < 3; ++p) {
        int Ip = g.wx[3 * I + p];
        for (int q = 0; q < 3; ++q) {
            int Kq = g.wz[3 * K + q];
            s += g.Rx[3 * i + p] * g.Rz[3 * k + q] * V[((size_t)Kq * g.cvy + J) * g.nx + Ip];
        }
    }
    Vs[((size_t)k * g.vfy + (size_t)J * g.my) * g.Nx + i] = s;
}

// Stage 0, z-normal faces on the coarse z-planes: thread per (K, j, i).
template <typename P>
__global__ void k_outer_w(Grid<P> g, const P* __restrict__ W, P* __restrict__ Ws)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)(g.nz + 1) * g.Ny * g.Nx;
    if (t >= n) return;
    int i = (int)(t % g.Nx);
    int j = (int)((t / g.Nx) % g.Ny);
    int K = (int)(t / ((size_t)g.Nx * g.Ny));
    int I = i / g.mx, J = j / g.my;
    P s = P(0);
    for (int p = 0; p < 3; ++p) {
        int Ip = g.wx[3 * I + p];
        for (int q = 0; q < 3; ++q) {
            int Jq = g.wy[3 * J + q];
            s += g.Rx[3 * i + p] * g.Ry[3 * j + q] * W[((size_t)K * g.ny + Jq) * g.nx + Ip];
        }
    }
    Ws[((size_t)K * g.mz * g.Ny + j) * g.Nx + i] = s;
}

// Stage Z balance: thread per coarse cell; writes the full-area inner-plane W.
// MZ > 0: the refinement factor in z known at compile time (the loop unrolls
// and every load is issued before the running balance); 0: any factor.
template <typename P, int MZ = 0>
__global__ void k_column_balance(Grid<P> g, const P* __restrict__ U, const P* __restrict__ V,
                                 const P* __restrict__ W, P* __restrict__ scrW)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.nz * g.ny * g.nx;
    if (t >= n) return;
    int I = (int)(t % g.nx);
    int J = (int)((t / g.nx) % g.ny);
    int K = (int)(t / ((size_t)g.nx * g.ny));
    int Ie = g.walls ? I + 1 : (I + 1) % g.nx;
    int Jn = g.walls ? J + 1 : (J + 1) % g.ny;
    P F = W[((size_t)(K + 1) * g.ny + J) * g.nx + I] * g.DX * g.DY;
    const int mz = MZ > 0 ? MZ : g.mz;
#pragma unroll
    for (int c = mz - 1; c >= 1; --c) {
        int k = K * mz + c;
        P uw = 0, ue = 0, vs = 0, vn = 0;
        for (int q = 0; q < 3; ++q) {
            P r = g.Rz[3 * k + q];
            int Kq = g.wz[3 * K + q];
            uw += r * U[((size_t)Kq * g.ny + J) * g.cux + I];
            ue += r * U[((size_t)Kq * g.ny + J) * g.cux + Ie];
            vs += r * V[((size_t)Kq * g.cvy + J) * g.nx + I];
            vn += r * V[((size_t)Kq * g.cvy + Jn) * g.nx + I];
        }
        F = F + (ue - uw) * g.DY * g.dz[k] + (vn - vs) * g.DX * g.dz[k];
        scrW[((size_t)k * g.ny + J) * g.nx + I] = F / (g.DX * g.DY);
    }
}

// Stage Z split: thread per dense face on an inner z-plane.
template <typename P>
__global__ void k_split_w(Grid<P> g, const P* __restrict__ scrW, P* __restrict__ Ws)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t planes = (size_t)g.nz * (g.mz - 1);
    size_t n = planes * g.Ny * g.Nx;
    if (t >= n) return;
    int i = (int)(t % g.Nx);
    int j = (int)((t / g.Nx) % g.Ny);
    int kk = (int)(t / ((size_t)g.Nx * g.Ny));
    int k = (kk / (g.mz - 1)) * g.mz + kk % (g.mz - 1) + 1;
    int I = i / g.mx, J = j / g.my;
    P s = P(0);
    for (int p = 0; p < 3; ++p) {
        int Ip = g.wx[3 * I + p];
        for (int q = 0; q < 3; ++q) {
            int Jq = g.wy[3 * J + q];
            s += g.Rx[3 * i + p] * g.Ry[3 * j + q] * scrW[((size_t)k * g.ny + Jq) * g.nx + Ip];
        }
    }
    Ws[((size_t)k * g.Ny + j) * g.Nx + i] = s;
}

// Stage Y balance: thread per (I, J, dense layer k); writes the full-width
// inner-row V.
template <typename P>
__global__ void k_row_balance(Grid<P> g, const P* __restrict__ Us, const P* __restrict__ Vs,
                              const P* __restrict__ Ws, P* __restrict__ scrV)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.ny * g.nx;
    if (t >= n) return;
    int I = (int)(t % g.nx);
    int J = (int)((t / g.nx) % g.ny);
    int k = (int)(t / ((size_t)g.nx * g.ny));
    int Ie = g.walls ? I + 1 : (I + 1) % g.nx;
    P dzk = g.dz[k];
    P G = 0;
    for (int a = 0; a < g.mx; ++a) G += Vs[((size_t)k * g.vfy + (size_t)J * g.my) * g.Nx + I * g.mx + a] * g.dx;
    G *= dzk;
    for (int b = 0; b < g.my - 1; ++b) {
        int j = J * g.my + b;
        P uw = Us[((size_t)k * g.Ny + j) * g.ufx + (size_t)I * g.mx];
        P ue = Us[((size_t)k * g.Ny + j) * g.ufx + (size_t)Ie * g.mx];
        P wb = 0, wt = 0;
        for (int a = 0; a < g.mx; ++a) {
            wb += Ws[((size_t)k * g.Ny + j) * g.Nx + I * g.mx + a] * g.dx;
            wt += Ws[((size_t)(k + 1) * g.Ny + j) * g.Nx + I * g.mx + a] * g.dx;
        }
        G = G - (ue - uw) * g.dy * dzk - (wt - wb) * g.dy;
        scrV[((size_t)k * g.vfy + j + 1) * g.nx + I] = G / (g.DX * dzk);
    }
}

// Stage Y split: thread per dense face on an inner y-row.
template <typename P>
__global__ void k_split_v(Grid<P> g, const P* __restrict__ scrV, P* __restrict__ Vs)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t rows = (size_t)g.ny * (g.my - 1);
    size_t n = (size_t)g.Nz * rows * g.Nx;
    if (t >= n) return;
    int i = (int)(t % g.Nx);
    int jj = (int)((t / g.Nx) % rows);
    int k = (int)(t / ((size_t)g.Nx * rows));
    int j = (jj / (g.my - 1)) * g.my + jj % (g.my - 1) + 1;
    int I = i / g.mx;
    P s = P(0);
    for (int p = 0; p < 3; ++p) s += g.Rx[3 * i + p] * scrV[((size_t)k * g.vfy + j) * g.nx + g.wx[3 * I + p]];
    Vs[((size_t)k * g.vfy + j) * g.Nx + i] = s;
}

// Stage X: thread per (I, dense row j, dense layer k).
template <typename P>
__global__ void k_stage_x(Grid<P> g, P* __restrict__ Us, const P* __restrict__ Vs, const P* __restrict__ Ws)
{
    size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t n = (size_t)g.Nz * g.Ny * g.nx;
    if (t >= n) return;
    int I = (int)(t % g.nx);
    int j = (int)((t / g.nx) % g.Ny);
    int k = (int)(t / ((size_t)g.nx * g.Ny));
    int jn = g.walls ? j + 1 : (j + 1) % g.Ny;
    P dzk = g.dz[k];
    size_t urow = ((size_t)k * g.Ny + j) * g.ufx;
    P H = Us[urow + (size_t)I * g.mx] * g.dy * dzk;
    for (int a = 0; a < g.mx - 1; ++a) {
        int i = I * g.mx + a;
        H = H - (Vs[((size_t)k * g.vfy + jn) * g.Nx + i] - Vs[((size_t)k * g.vfy + j) * g.Nx + i]) * g.dx * dzk
              - (Ws[((size_t)(k + 1) * g.Ny + j) * g.Nx + i] - Ws[((size_t)k * g.Ny + j) * g.Nx + i]) * g.dx * g.dy;
        Us[urow + i + 1] = H / (g.dy * dzk);
    }
}

}  // namespace

template <typename P>
cudaError_t launch_refine(const Grid<P>& g, const P* U, const P* V, const P* W, P* Us, P* Vs, P* Ws,
                          P* scrW, P* scrV, cudaStream_t st)
{
    size_t n;
    n = (size_t)g.Nz * g.Ny * g.cux;
    k_outer_u<P><<<blocks_for(n), kThreads, 0, st>>>(g, U, Us);
    n = (size_t)g.Nz * g.cvy * g.Nx;
    k_outer_v<P><<<blocks_for(n), kThreads, 0, st>>>(g, V, Vs);
    n = (size_t)(g.nz + 1) * g.Ny * g.Nx;
    k_outer_w<P><<<blocks_for(n), kThreads, 0, st>>>(g, W, Ws);
    if (g.mz > 1) {
        n = (size_t)g.nz * g.ny * g.nx;
        k_column_balance<P><<<blocks_for(n), kThreads, 0, st>>>(g, U, V, W, scrW);
        n = (size_t)g.nz * (g.mz - 1) * g.Ny * g.Nx;
        k_split_w<P><<<blocks_for(n), kThreads, 0, st>>>(g, scrW, Ws);
    }
    if (g.my > 1) {
        n = (size_t)g.Nz * g.ny * g.nx;
        k_row_balance<P><<<blocks_for(n), kThreads, 0, st>>>(g, Us, Vs, Ws, scrV);
        n = (size_t)g.Nz * g.ny * (g.my - 1) * g.Nx;
        k_split_v<P><<<blocks_for(n), kThreads, 0, st>>>(g, scrV, Vs);
    }
    if (g.mx > 1) {
        n = (size_t)g.Nz * g.Ny * g.nx;
        k_stage_x<P><<<blocks_for(n), kThreads, 0, st>>>(g, Us, Vs, Ws);
    }
    return cudaGetLastError();
}

// Stage Z slab balance alone (full-area W on the inner planes), for the
// split-x fused path.
template <typename P>
cudaError_t launch_column_balance(const Grid<P>& g, const P* U, const P* V, const P* W, P* scrW, cudaStream_t st)
{
    if (g.mz > 1) {
        const size_t n = (size_t)g.nz * g.ny * g.nx;
        if (g.mz == 4) k_column_balance<P, 4><<<blocks_for(n), kThreads, 0, st>>>(g, U, V, W, scrW);
        else if (g.mz == 2) k_column_balance<P, 2><<<blocks_for(n), kThreads, 0, st>>>(g, U, V, W, scrW);
        else k_column_balance<P><<<blocks_for(n), kThreads, 0, st>>>(g, U, V, W, scrW);
    }
    return cudaGetLastError();
}
template cudaError_t launch_column_balance<float>(const Grid<float>&, const float*, const float*, const float*,
                                                  float*, cudaStream_t);

template cudaError_t launch_refine<double>(const Grid<double>&, const double*, const double*, const double*,
                                           double*, double*, double*, double*, double*, cudaStream_t);
template cudaError_t launch_refine<float>(const Grid<float>&, const float*, const float*, const float*,
                                          float*, float*, float*, float*, float*, cudaStream_t);

}  // namespace mr
