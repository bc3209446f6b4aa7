// FP64 reductions (Section 4.1 plate Nusselt numbers, volume moments, the
// divergence check of Section 3.2, the CFL limit) and dtype conversion.
// Each block reduces with warp shuffles into one FP64 partial; the host sums
// the partials in block order, so every result is deterministic.
#include <math.h>

#include "mr_internal.cuh"

namespace mr {
namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of NV values per thread (sum or max); thread 0 writes them.
template <int NV, bool MAX>
__device__ void block_reduce_store(double (&v)[NV], double* out)
{
    __shared__ double sh[NV][kRedThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = 0; q < NV; ++q) {
        double r = MAX ? warp_max(v[q]) : warp_sum(v[q]);
        if (lane == 0) sh[q][wid] = r;
    }
    __syncthreads();
    if (wid == 0) {
        for (int q = 0; q < NV; ++q) {
            double r = (lane < kRedThreads / 32) ? sh[q][lane] : (MAX ? 0.0 : 0.0);
            r = MAX ? warp_max(r) : warp_sum(r);
            if (lane == 0) out[q] = r;
        }
    }
}

// pass 0: (sum T vol, count of non-finite T); pass 1: sum (T - mean)^2 vol.
// vol is dx dy dz_k; the dx dy factor is applied on the host.  Work units are
// slices of one dense plane (8 per plane), so dz_k is common to a unit; a
// thread loads 16 cells at a time (16 independent loads in flight), adds them
// in precision P and each group into its FP64 sum, which is scaled by dz_k
// once per unit.
template <typename P>
__global__ void __launch_bounds__(kRedThreads) k_moments(Grid<P> g, const P* __restrict__ T, double mean,
                                                         int pass, double* __restrict__ partials)
{
    constexpr int kSlices = 8, kGroup = 16;
    const size_t plane = (size_t)g.Nx * g.Ny, per = (plane + kSlices - 1) / kSlices;
    const int units = g.Nz * kSlices;
    const P mp = (P)mean;
    double v[2] = {0.0, 0.0};
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int k = u / kSlices, sl = u - k * kSlices;
        const P* r = T + (size_t)k * plane;
        const size_t lo = (size_t)sl * per, hi = lo + per < plane ? lo + per : plane;
        const size_t step = blockDim.x;
        double acc = 0.0;
        int bad = 0;
        size_t m = lo + threadIdx.x;
        for (; m + (kGroup - 1) * step < hi; m += kGroup * step) {
            P t[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; ++q) t[q] = r[m + q * step];
            P grp = 0;
#pragma unroll
            for (int q = 0; q < kGroup; ++q) {
                if (pass == 0) {
                    if (isfinite(t[q])) grp += t[q];
                    else ++bad;
                } else {
                    const P d = t[q] - mp;
                    grp += d * d;
                }
            }
            acc += (double)grp;
        }
        P grp = 0;
        for (; m < hi; m += step) {
            const P t = r[m];
            if (pass == 0) {
                if (isfinite(t)) grp += t;
                else ++bad;
            } else {
                const P d = t - mp;
                grp += d * d;
            }
        }
        acc += (double)grp;
        v[0] += acc * (double)g.dz[k];
        v[1] += (double)bad;
    }
    block_reduce_store<2, false>(v, partials + 2 * blockIdx.x);
}

// Plate Nusselt numbers: every block sums a fixed slice of both plates,
// sum (T_bottom - T) and sum (T - T_top), into two FP64 partials; the block
// that finishes last (an atomic count, nothing waits) adds the partials --
// thread t the partials t, t + 256, ..., then the block's fixed reduction tree,
// so the order of the additions never changes -- divides by the centre
// distance and the cell count, and resets the count for the next launch.
template <typename P>
__global__ void __launch_bounds__(256) k_plate_nu(Grid<P> g, const P* __restrict__ T, double zb, double zt,
                                                  double inv_plane, double* __restrict__ partials,
                                                  unsigned* __restrict__ count, double* __restrict__ out2)
{
    const size_t plane = (size_t)g.Nx * g.Ny;
    const P* top = T + (size_t)(g.Nz - 1) * plane;
    double v[2] = {0.0, 0.0};
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < plane; m += (size_t)gridDim.x * blockDim.x) {
        v[0] += 0.5 - (double)T[m];
        v[1] += (double)top[m] + 0.5;
    }
    block_reduce_store<2, false>(v, partials + 2 * blockIdx.x);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();                     // this block's partials before its count
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s2[2] = {0.0, 0.0};
    for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        s2[0] += __ldcg(partials + 2 * q);
        s2[1] += __ldcg(partials + 2 * q + 1);
    }
    __shared__ double tot[2];
    block_reduce_store<2, false>(s2, tot);
    if (threadIdx.x == 0) {                  // the thread that wrote tot
        out2[0] = tot[0] / zb * inv_plane;
        out2[1] = tot[1] / zt * inv_plane;
        *count = 0u;
    }
}

// FP64 values from mapped pinned host memory (read by the SMs over the host
// link) into the FP64 device copy and, where d32 is given, its FP32 rounding.
__global__ void k_fetch_f64(const double* __restrict__ src, double* __restrict__ d64, float* __restrict__ d32,
                            size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t n2 = n / 2;
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* o2 = reinterpret_cast<double2*>(d64);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n2; t += stride) {
        const double2 v = s2[t];
        o2[t] = v;
        if (d32) reinterpret_cast<float2*>(d32)[t] = make_float2((float)v.x, (float)v.y);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        d64[n - 1] = src[n - 1];
        if (d32) d32[n - 1] = (float)src[n - 1];
    }
}

// Max |divergence| of the dense refined faces (outward flux sum / volume).
// Blocks stride over dense rows (j, k), threads over x.
template <typename P>
__global__ void __launch_bounds__(kRedThreads) k_maxdiv(Grid<P> g, const P* __restrict__ Us,
                                                        const P* __restrict__ Vs, const P* __restrict__ Ws,
                                                        double* __restrict__ partials)
{
    const size_t plane = (size_t)g.Nx * g.Ny;
    const int rows = g.Ny * g.Nz;
    double v[1] = {0.0};
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = row / g.Ny, j = row - k * g.Ny;
        const int fn = g.walls ? j + 1 : (j + 1 == g.Ny ? 0 : j + 1);
        const P* ur = Us + ((size_t)k * g.Ny + j) * g.ufx;
        const P* vs = Vs + ((size_t)k * g.vfy + j) * g.Nx;
        const P* vn = Vs + ((size_t)k * g.vfy + fn) * g.Nx;
        const P* wb = Ws + (size_t)row * g.Nx;
        const P* wt = wb + plane;
        const double idz = (double)g.inv_dz[k];
        for (int i = threadIdx.x; i < g.Nx; i += blockDim.x) {
            const int fe = g.walls ? i + 1 : (i + 1 == g.Nx ? 0 : i + 1);
            const double d = ((double)ur[fe] - (double)ur[i]) * (double)g.inv_dx +
                             ((double)vn[i] - (double)vs[i]) * (double)g.inv_dy + ((double)wt[i] - (double)wb[i]) * idz;
            v[0] = fmax(v[0], fabs(d));
        }
    }
    block_reduce_store<1, true>(v, partials + blockIdx.x);
}

// CFL rate max(|u|)/dx + max(|v|)/dy + max(|w|)/dz over the cell's faces, in
// precision P (|.| and max are exact; the rate is one sum of three products).
template <typename P>
__global__ void __launch_bounds__(kRedThreads) k_cfl(Grid<P> g, const P* __restrict__ Us,
                                                     const P* __restrict__ Vs, const P* __restrict__ Ws,
                                                     double* __restrict__ partials)
{
    const size_t plane = (size_t)g.Nx * g.Ny;
    const int rows = g.Ny * g.Nz;
    P m = 0;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int k = row / g.Ny, j = row - k * g.Ny;
        const int fn = g.walls ? j + 1 : (j + 1 == g.Ny ? 0 : j + 1);
        const P* ur = Us + ((size_t)k * g.Ny + j) * g.ufx;
        const P* vs = Vs + ((size_t)k * g.vfy + j) * g.Nx;
        const P* vn = Vs + ((size_t)k * g.vfy + fn) * g.Nx;
        const P* wb = Ws + (size_t)row * g.Nx;
        const P* wt = wb + plane;
        const P idz = g.inv_dz[k];
        for (int i = threadIdx.x; i < g.Nx; i += blockDim.x) {
            const int fe = g.walls ? i + 1 : (i + 1 == g.Nx ? 0 : i + 1);
            const P u = fmax(fabs(ur[i]), fabs(ur[fe]));
            const P vv = fmax(fabs(vs[i]), fabs(vn[i]));
            const P w = fmax(fabs(wb[i]), fabs(wt[i]));
            m = fmax(m, u * g.inv_dx + vv * g.inv_dy + w * idz);
        }
    }
    double v[1] = {(double)m};
    block_reduce_store<1, true>(v, partials + blockIdx.x);
}

// Upscale integration (Section 3.3): volume average over every coarse cell.
template <typename P>
__global__ void k_upscale(Grid<P> g, const P* __restrict__ T, double* __restrict__ Tc)
{
    const size_t n = (size_t)g.nz * g.ny * g.nx;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (size_t)gridDim.x * blockDim.x) {
        const int I = (int)(t % g.nx), J = (int)((t / g.nx) % g.ny), K = (int)(t / ((size_t)g.nx * g.ny));
        // the sum over each dense layer in the working precision (GB300's FP64
        // pipe is 1/64 of its FP32 rate), the volume weighting in FP64
        double s = 0.0, h = 0.0;
        for (int k = K * g.mz; k < (K + 1) * g.mz; ++k) {
            P r = P(0);
            for (int j = J * g.my; j < (J + 1) * g.my; ++j) {
                const P* row = T + ((size_t)k * g.Ny + j) * g.Nx + (size_t)I * g.mx;
                for (int i = 0; i < g.mx; ++i) r += row[i];
            }
            s += (double)r * (double)g.dz[k];
            h += (double)g.dz[k];
        }
        Tc[t] = s / (h * g.mx * g.my);
    }
}

// Nu(z) (Section 4.1) on dense z-face k = blockIdx.x: plane average of
// w T_f / kappa - dT/dz (the plates: conductive flux only).
template <typename P>
__global__ void __launch_bounds__(256) k_nu_profile(Grid<P> g, const P* __restrict__ T, const P* __restrict__ Ws,
                                                    const double* __restrict__ zc, double inv_kappa, double zb,
                                                    double zt, double* __restrict__ nu_z)
{
    const int k = blockIdx.x;
    const size_t plane = (size_t)g.Nx * g.Ny;
    double v[1] = {0.0};
    for (size_t m = threadIdx.x; m < plane; m += blockDim.x) {
        if (k == 0) {
            v[0] += (0.5 - (double)T[m]) / zb;
        } else if (k == g.Nz) {
            v[0] += ((double)T[(size_t)(g.Nz - 1) * plane + m] + 0.5) / zt;
        } else {
            const double tl = (double)T[(size_t)(k - 1) * plane + m], tr = (double)T[(size_t)k * plane + m];
            double tf = (double)g.wlo[k] * tl + (double)g.whi[k] * tr;
            if (g.order4) {                      // the step's fourth-order face value
                tf = 0.0;
                for (int q = 0; q < 4; ++q) {
                    const int c = k - 2 + q;
                    if (c >= 0 && c < g.Nz) tf += (double)g.f4z[4 * k + q] * (double)T[(size_t)c * plane + m];
                }
            }
            v[0] += (double)Ws[(size_t)k * plane + m] * tf * inv_kappa - (tr - tl) / (zc[k] - zc[k - 1]);
        }
    }
    block_reduce_store<1, false>(v, nu_z + k);
}

// <|grad T|^2> from face gradients weighted by the face's dual volume (A d),
// plates at their Dirichlet values: partial sums per block.
template <typename P>
__global__ void __launch_bounds__(kRedThreads) k_grad2(Grid<P> g, const P* __restrict__ T, const double* __restrict__ zc,
                                                       double zb, double zt, double* __restrict__ partials)
{
    const size_t plane = (size_t)g.Nx * g.Ny, n = plane * g.Nz;
    const double dx = (double)g.dx, dy = (double)g.dy;
    double v[1] = {0.0};
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(m % g.Nx), j = (int)((m / g.Nx) % g.Ny), k = (int)(m / plane);
        const double t = (double)T[m], dzk = (double)g.dz[k];
        if (!(g.walls && i == 0)) {
            const double d = t - (double)T[m - i + (i == 0 ? g.Nx - 1 : i - 1)];
            v[0] += d * d * dy * dzk / dx;
        }
        if (!(g.walls && j == 0)) {
            const double d = t - (double)T[m + ((ptrdiff_t)(j == 0 ? g.Ny - 1 : j - 1) - j) * g.Nx];
            v[0] += d * d * dx * dzk / dy;
        }
        if (k > 0) {
            const double d = t - (double)T[m - plane];
            v[0] += d * d * dx * dy / (zc[k] - zc[k - 1]);
        } else if (g.dirichlet) {
            const double d = t - 0.5;
            v[0] += d * d * dx * dy / zb;
        }
        if (k == g.Nz - 1 && g.dirichlet) {
            const double d = -0.5 - t;
            v[0] += d * d * dx * dy / zt;
        }
    }
    block_reduce_store<1, false>(v, partials + blockIdx.x);
}

template <typename S, typename D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, size_t n)
{
    for (size_t m = (size_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (size_t)gridDim.x * blockDim.x)
        dst[m] = (D)src[m];
}

}  // namespace

template <typename P>
cudaError_t launch_moments(const Grid<P>& g, const P* T, double mean, int pass, double* partials, int blocks,
                           cudaStream_t st)
{
    k_moments<P><<<blocks, kRedThreads, 0, st>>>(g, T, mean, pass, partials);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_plate_nu(const Grid<P>& g, const P* T, const double* zb_zt, double* out2, cudaStream_t st)
{
    // out2 holds 3 + 2 * kPlateBlocks doubles: the two means, the block count
    // (zero between launches) and the partials
    k_plate_nu<P><<<kPlateBlocks, 256, 0, st>>>(g, T, zb_zt[0], zb_zt[1], 1.0 / ((double)g.Nx * g.Ny), out2 + 3,
                                                reinterpret_cast<unsigned*>(out2 + 2), out2);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_upscale(const Grid<P>& g, const P* T, double* Tc, cudaStream_t st)
{
    k_upscale<P><<<152 * 8, kRedThreads, 0, st>>>(g, T, Tc);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_nu_profile(const Grid<P>& g, const P* T, const P* Ws, const double* zc, double inv_kappa, double zb,
                              double zt, double* nu_z, double* partials, int blocks, cudaStream_t st)
{
    k_nu_profile<P><<<g.Nz + 1, 256, 0, st>>>(g, T, Ws, zc, inv_kappa, zb, zt, nu_z);
    k_grad2<P><<<blocks, kRedThreads, 0, st>>>(g, T, zc, zb, zt, partials);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_maxdiv(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, double* partials, int blocks,
                          cudaStream_t st)
{
    k_maxdiv<P><<<blocks, kRedThreads, 0, st>>>(g, Us, Vs, Ws, partials);
    return cudaGetLastError();
}

template <typename P>
cudaError_t launch_cfl(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, double* partials, int blocks,
                       cudaStream_t st)
{
    k_cfl<P><<<blocks, kRedThreads, 0, st>>>(g, Us, Vs, Ws, partials);
    return cudaGetLastError();
}

// src/dst dtypes: MR_F64 or MR_F32.  P is unused (kept for a uniform launcher signature).
template <typename P>
cudaError_t launch_convert(const void* src, int sd, void* dst, int dd, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const int threads = 256;
    size_t want = (n + threads - 1) / threads;
    const unsigned blocks = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    if (sd == MR_F64 && dd == MR_F32)
        k_convert<double, float><<<blocks, threads, 0, st>>>((const double*)src, (float*)dst, n);
    else if (sd == MR_F32 && dd == MR_F64)
        k_convert<float, double><<<blocks, threads, 0, st>>>((const float*)src, (double*)dst, n);
    else if (sd == MR_F64 && dd == MR_F64)
        return cudaMemcpyAsync(dst, src, n * 8, cudaMemcpyDeviceToDevice, st);
    else
        return cudaMemcpyAsync(dst, src, n * 4, cudaMemcpyDeviceToDevice, st);
    return cudaGetLastError();
}

#define MR_INST(P)                                                                                           \
    template cudaError_t launch_moments<P>(const Grid<P>&, const P*, double, int, double*, int, cudaStream_t); \
    template cudaError_t launch_plate_nu<P>(const Grid<P>&, const P*, const double*, double*, cudaStream_t);    \
    template cudaError_t launch_maxdiv<P>(const Grid<P>&, const P*, const P*, const P*, double*, int,          \
                                          cudaStream_t);                                                     \
    template cudaError_t launch_cfl<P>(const Grid<P>&, const P*, const P*, const P*, double*, int, cudaStream_t);    \
    template cudaError_t launch_upscale<P>(const Grid<P>&, const P*, double*, cudaStream_t);                       \
    template cudaError_t launch_nu_profile<P>(const Grid<P>&, const P*, const P*, const double*, double, double,   \
                                              double, double*, double*, int, cudaStream_t);
MR_INST(double)
MR_INST(float)
#undef MR_INST
template cudaError_t launch_convert<double>(const void*, int, void*, int, size_t, cudaStream_t);

cudaError_t launch_fetch_f64(const double* src, double* d64, float* d32, size_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    // 16-byte alignment for the pair loads and stores
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(d64)) & 15 ||
        reinterpret_cast<uintptr_t>(d32) & 7)
        return cudaErrorInvalidValue;
    k_fetch_f64<<<152 * 8, 256, 0, st>>>(src, d64, d32, n);
    return cudaGetLastError();
}

}  // namespace mr
