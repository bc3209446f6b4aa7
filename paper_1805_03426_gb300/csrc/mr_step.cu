// Scalar time step with the dense velocity read from HBM (MR_VEL_STORED),
// FP64 or FP32.  Eq. (5) in flux form, second-order (linear) face values,
// Euler-leapfrog with the averaging step (Section 2.2):
//   T^{s+1} = a T^{s-1} + b T^s + gdt [C(T^s) + D(T^{s-1})]
// C = -(1/Vol) sum_faces u_f T_f A_f (outward), D = (1/Vol) sum kappa A dT/dn.
// Per-layer coefficients (1/dz, interpolation weights, kappa/(dz d)) come
// from the handle's grid, so a stretched z costs no extra arithmetic.
#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr double kTBottom = 0.5;
constexpr double kTTop = -0.5;

// Dense face velocity of a step: one stored field, or (LERP) the linear
// interpolation A + alpha (B - A) between the fields of two coarse time
// levels (temporal refinement, Section 3.4).
template <typename P, bool LERP>
struct FaceVel {
    const P* __restrict__ A;
    const P* __restrict__ B;
    P alpha;
    __device__ __forceinline__ P operator[](size_t f) const
    {
        if (!LERP) return A[f];
        const P a = A[f];
        return a + alpha * (B[f] - a);
    }
};

// Fourth-order value at face f of an axis of N cells (Section 2.2): the cells
// f-2 .. f+1 at T[base + c * stride] with the grid's weights; periodic cells
// wrap, cells beyond a wall carry zero weight and are not read.
template <typename P>
__device__ __forceinline__ P face4(const P* __restrict__ w, int f, int N, bool periodic, const P* __restrict__ T,
                                   size_t base, size_t stride)
{
    P s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int c = f - 2 + q;
        if (periodic) c = c < 0 ? c + N : (c >= N ? c - N : c);
        else if (c < 0 || c >= N) continue;
        s += w[4 * f + q] * T[base + (size_t)c * stride];
    }
    return s;
}

// One thread per dense cell.  IMPLZ: vertical diffusion enters as
// (D_z(T^{s-1}) + plate terms) / 2; the implicit half follows in k_zsolve.
// O4: fourth-order face values of the advected scalar.
template <typename P, bool IMPLZ, bool LERP, bool O4>
__global__ void __launch_bounds__(256) k_step_stored(Grid<P> g, const FaceVel<P, LERP> Us,
                                                     const FaceVel<P, LERP> Vs, const FaceVel<P, LERP> Ws,
                                                     const P* __restrict__ Tm1, const P* __restrict__ T,
                                                     P* __restrict__ Tp1, P a, P b, P gdt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = blockIdx.z;
    if (i >= g.Nx || j >= g.Ny) return;
    const size_t plane = (size_t)g.Nx * g.Ny;
    const size_t m = (size_t)k * plane + (size_t)j * g.Nx + i;
    const P Tc = T[m], Dc = Tm1[m];
    const P half = P(0.5);
    P cx = 0, dx_ = 0, cy = 0, dy_ = 0;
    // x faces
    const size_t urow = ((size_t)k * g.Ny + j) * g.ufx;
    if (!(g.walls && i == 0)) {
        const int iw = (i == 0) ? g.Nx - 1 : i - 1;
        const size_t mw = m - i + iw;
        cx += Us[urow + i] * (O4 ? face4(g.f4x, i, g.Nx, !g.walls, T, m - i, 1) : half * (T[mw] + Tc));
        dx_ -= Dc - Tm1[mw];
    }
    if (!(g.walls && i == g.Nx - 1)) {
        const int ie = (i == g.Nx - 1) ? 0 : i + 1;
        const int fe = g.walls ? i + 1 : ie;
        const size_t me = m - i + ie;
        cx -= Us[urow + fe] * (O4 ? face4(g.f4x, i + 1, g.Nx, !g.walls, T, m - i, 1) : half * (Tc + T[me]));
        dx_ += Tm1[me] - Dc;
    }
    // y faces
    if (!(g.walls && j == 0)) {
        const int js = (j == 0) ? g.Ny - 1 : j - 1;
        const size_t ms = m + ((ptrdiff_t)js - j) * g.Nx;
        cy += Vs[((size_t)k * g.vfy + j) * g.Nx + i] *
              (O4 ? face4(g.f4y, j, g.Ny, !g.walls, T, m - (size_t)j * g.Nx, g.Nx) : half * (T[ms] + Tc));
        dy_ -= Dc - Tm1[ms];
    }
    if (!(g.walls && j == g.Ny - 1)) {
        const int jn = (j == g.Ny - 1) ? 0 : j + 1;
        const int fn = g.walls ? j + 1 : jn;
        const size_t mn = m + ((ptrdiff_t)jn - j) * g.Nx;
        cy -= Vs[((size_t)k * g.vfy + fn) * g.Nx + i] *
              (O4 ? face4(g.f4y, j + 1, g.Ny, !g.walls, T, m - (size_t)j * g.Nx, g.Nx) : half * (Tc + T[mn]));
        dy_ += Tm1[mn] - Dc;
    }
    // z faces (plates: no advective flux; Dirichlet or zero diffusive flux)
    P cz = 0, dz_ = 0;
    if (k > 0) {
        const P Tb = T[m - plane];
        cz += Ws[m] * (O4 ? face4(g.f4z, k, g.Nz, false, T, m - k * plane, plane) : g.wlo[k] * Tb + g.whi[k] * Tc);
        dz_ -= g.cdn[k] * (Dc - Tm1[m - plane]);
    } else {
        dz_ -= g.cdn[0] * (Dc - P(kTBottom));    // cdn[0] = 0 when adiabatic
    }
    if (k < g.Nz - 1) {
        const P Tt = T[m + plane];
        cz -= Ws[m + plane] *
              (O4 ? face4(g.f4z, k + 1, g.Nz, false, T, m - k * plane, plane) : g.wlo[k + 1] * Tc + g.whi[k + 1] * Tt);
        dz_ += g.cup[k] * (Tm1[m + plane] - Dc);
    } else {
        dz_ += g.cup[k] * (P(kTTop) - Dc);        // cup[Nz-1] = 0 when adiabatic
    }
    if (IMPLZ) {
        // (Lz T^{s-1} + bz)/2 + bz/2: the plate terms count in full
        P bz = 0;
        if (k == 0) bz += g.cdn[0] * P(kTBottom);
        if (k == g.Nz - 1) bz += g.cup[k] * P(kTTop);
        dz_ = half * dz_ + half * bz;
    }
    const P C = cx * g.inv_dx + cy * g.inv_dy + cz * g.inv_dz[k];
    const P D = g.kx2 * dx_ + g.ky2 * dy_ + dz_;
    Tp1[m] = a * Dc + b * Tc + gdt * (C + D);
}

// The same step (Eq. 5) for the common case -- periodic x and y, explicit
// diffusion, second-order faces, one velocity level -- with the arithmetic
// folded for the FP64 pipe (25 FP operations per cell instead of 39):
// 1/(2 dx), 1/(2 dy) scale the summed x and y flux differences, the z-face
// weights carry 1/dz_k (the top face's negated), the opposite diffusion
// neighbours are summed before kx2, ky2, and the diagonal and the plate
// terms come from the per-layer table g.lz.  LF: a plain leapfrog step.
template <typename P, bool LF>
__global__ void __launch_bounds__(256) k_step_periodic(Grid<P> g, const P* __restrict__ Us,
                                                       const P* __restrict__ Vs, const P* __restrict__ Ws,
                                                       const P* __restrict__ Tm1, const P* __restrict__ T,
                                                       P* __restrict__ Tp1, P a, P b, P gdt)
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
    const P Tc = T[m], Dc = Tm1[m];
    // beyond the plates: zero (W is zero there; the plate values enter through L[7])
    const bool lo = k > 0, hi = k < g.Nz - 1;
    const P Tb = lo ? T[m - plane] : P(0), Db = lo ? Tm1[m - plane] : P(0);
    const P Tt = hi ? T[m + plane] : P(0), Dt = hi ? Tm1[m + plane] : P(0);
    const size_t urow = ((size_t)k * g.Ny + j) * g.Nx, vrow = (size_t)k * g.Ny * g.Nx;
    const P ax = Us[urow + i] * (T[mw] + Tc) - Us[urow + ie] * (Tc + T[me]);
    const P ay = Vs[vrow + row + i] * (T[ms] + Tc) - Vs[vrow + (size_t)jn * g.Nx + i] * (Tc + T[mn]);
    const P az = Ws[m] * (L[0] * Tb + L[1] * Tc) + Ws[m + plane] * (L[2] * Tc + L[3] * Tt);
    const P D = L[7] + g.kx2 * (Tm1[mw] + Tm1[me]) + g.ky2 * (Tm1[ms] + Tm1[mn]) + L[4] * Db + L[5] * Dt + L[6] * Dc;
    const P C = g.hx * ax + g.hy * ay + az;
    Tp1[m] = LF ? Dc + gdt * (C + D) : a * Dc + b * Tc + gdt * (C + D);
}

// Opt-in implicit vertical diffusion: per (x, y) column solve
//   (1 + h (cup + cdn)) x_k - h cdn_k x_{k-1} - h cup_k x_{k+1} = r_k,
// h = gdt / 2, by the Thomas algorithm; work holds the eliminated
// super-diagonal (one value per cell).
template <typename P>
__global__ void k_zsolve(Grid<P> g, P* __restrict__ X, P h, P* __restrict__ work)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= g.Nx) return;
    const size_t plane = (size_t)g.Nx * g.Ny;
    const size_t base = (size_t)j * g.Nx + i;
    const int N = g.Nz;
    P prev_c = 0, prev_x = 0;
    for (int k = 0; k < N; ++k) {
        const P lo = (k > 0) ? -h * g.cdn[k] : P(0);
        const P up = (k < N - 1) ? -h * g.cup[k] : P(0);
        const P di = P(1) + h * (g.cup[k] + g.cdn[k]);
        const P den = di - lo * prev_c;
        const P c = up / den;
        const P x = (X[base + k * plane] - lo * prev_x) / den;
        work[base + k * plane] = c;
        X[base + k * plane] = x;
        prev_c = c;
        prev_x = x;
    }
    for (int k = N - 2; k >= 0; --k) {
        prev_x = X[base + k * plane] - work[base + k * plane] * prev_x;
        X[base + k * plane] = prev_x;
    }
}

template <typename P, bool LERP>
cudaError_t step_stored(const Grid<P>& g, const FaceVel<P, LERP>& u, const FaceVel<P, LERP>& v,
                        const FaceVel<P, LERP>& w, const P* Tm1, const P* T, P* Tp1, StepCoef c, bool implz,
                        cudaStream_t st)
{
    dim3 blk(64, 4);
    dim3 grd((g.Nx + blk.x - 1) / blk.x, (g.Ny + blk.y - 1) / blk.y, g.Nz);
    const P a = (P)c.a, b = (P)c.b, gdt = (P)c.gdt;
    if (!LERP && !implz && !g.order4 && !g.walls) {
        if (c.a == 1.0 && c.b == 0.0)
            k_step_periodic<P, true><<<grd, blk, 0, st>>>(g, u.A, v.A, w.A, Tm1, T, Tp1, a, b, gdt);
        else
            k_step_periodic<P, false><<<grd, blk, 0, st>>>(g, u.A, v.A, w.A, Tm1, T, Tp1, a, b, gdt);
        return cudaGetLastError();
    }
    if (g.order4) {
        if (implz) k_step_stored<P, true, LERP, true><<<grd, blk, 0, st>>>(g, u, v, w, Tm1, T, Tp1, a, b, gdt);
        else k_step_stored<P, false, LERP, true><<<grd, blk, 0, st>>>(g, u, v, w, Tm1, T, Tp1, a, b, gdt);
    } else {
        if (implz) k_step_stored<P, true, LERP, false><<<grd, blk, 0, st>>>(g, u, v, w, Tm1, T, Tp1, a, b, gdt);
        else k_step_stored<P, false, LERP, false><<<grd, blk, 0, st>>>(g, u, v, w, Tm1, T, Tp1, a, b, gdt);
    }
    return cudaGetLastError();
}

__global__ void k_lerp(const float* __restrict__ A, const float* __restrict__ B, float alpha, float* __restrict__ out,
                       size_t n)
{
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const float a = A[t];
        out[t] = a + alpha * (B[t] - a);
    }
}

}  // namespace

cudaError_t launch_lerp_f32(const float* A, const float* B, double alpha, float* out, size_t n, cudaStream_t st)
{
    if (!n) return cudaSuccess;
    const size_t want = (n + 255) / 256;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    k_lerp<<<blocks, 256, 0, st>>>(A, B, (float)alpha, out, n);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_step_stored(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, const P* Tm1,
                               const P* T, P* Tp1, StepCoef c, bool implz, cudaStream_t st)
{
    return step_stored<P, false>(g, {Us, nullptr, P(0)}, {Vs, nullptr, P(0)}, {Ws, nullptr, P(0)}, Tm1, T, Tp1,
                                 c, implz, st);
}

template <typename P>
cudaError_t launch_step_stored_lerp(const Grid<P>& g, const P* const velA[3], const P* const velB[3], double alpha,
                                    const P* Tm1, const P* T, P* Tp1, StepCoef c, bool implz, cudaStream_t st)
{
    const P al = (P)alpha;
    return step_stored<P, true>(g, {velA[0], velB[0], al}, {velA[1], velB[1], al}, {velA[2], velB[2], al}, Tm1,
                                T, Tp1, c, implz, st);
}

template <typename P>
cudaError_t launch_zsolve(const Grid<P>& g, P* Tp1, double half_gdt, P* work, cudaStream_t st)
{
    dim3 blk(128);
    dim3 grd((g.Nx + 127) / 128, g.Ny);
    k_zsolve<P><<<grd, blk, 0, st>>>(g, Tp1, (P)half_gdt, work);
    return cudaGetLastError();
}

template cudaError_t launch_step_stored<double>(const Grid<double>&, const double*, const double*,
                                                const double*, const double*, const double*, double*,
                                                StepCoef, bool, cudaStream_t);
template cudaError_t launch_step_stored<float>(const Grid<float>&, const float*, const float*, const float*,
                                               const float*, const float*, float*, StepCoef, bool,
                                               cudaStream_t);
template cudaError_t launch_step_stored_lerp<double>(const Grid<double>&, const double* const[3],
                                                     const double* const[3], double, const double*,
                                                     const double*, double*, StepCoef, bool, cudaStream_t);
template cudaError_t launch_step_stored_lerp<float>(const Grid<float>&, const float* const[3], const float* const[3],
                                                    double, const float*, const float*, float*, StepCoef, bool,
                                                    cudaStream_t);
template cudaError_t launch_zsolve<double>(const Grid<double>&, double*, double, double*, cudaStream_t);
template cudaError_t launch_zsolve<float>(const Grid<float>&, float*, double, float*, cudaStream_t);

}  // namespace mr
