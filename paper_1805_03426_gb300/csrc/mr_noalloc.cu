// mr_refine_velocity_noalloc: the divergence-free refinement (FP64) for callers
// that cannot allocate device memory.  Everything the refinement needs beyond
// the caller's inputs and outputs -- the grid, the R matrices and the two
// refinement work arrays -- lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process exits.
// The grid and R matrices are rebuilt on the device by a set-up kernel at every
// call, so the call touches no host heap either.
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "mr_internal.cuh"

#define MR_NOALLOC_SCRATCH_BYTES (32u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[MR_NOALLOC_SCRATCH_BYTES];

namespace mr {
namespace {

constexpr int kMaxDevices = 64;
constexpr double kMinLayer = 1e-12;   // narrowest dense z-layer accepted (domain height 1)
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch on the current device (host code must not use
// the symbol itself: on the host it is only a stand-in).
int scratch_address(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check(e, "mr_refine_velocity_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_check(e, "mr_refine_velocity_noalloc: cudaGetSymbolAddress");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return MR_OK;
}

struct AxisDesc {
    int n, m;          // coarse cells, refinement
    int kind;          // 0: uniform faces length*i/N; 1: tanh-clustered z faces
    double length, gamma;
    int periodic;
};

__device__ double face_coord(const AxisDesc& a, int i)
{
    const int N = a.n * a.m;
    if (i <= 0) return 0.0;
    if (i >= N) return a.length;
    const double eta = (double)i / (double)N;
    if (a.kind == 0 || a.gamma <= 0.0) return a.length * eta;
    return 0.5 * (1.0 + tanh(a.gamma * (2.0 * eta - 1.0)) / tanh(a.gamma));
}

// Row of the mass-conserving third-order interpolation (Section 3.2) for the
// dense index d of an axis, in coordinates local to its coarse cell, and the
// window of that coarse cell (written by its first sub-cell).
__device__ void axis_row(const AxisDesc& a, int d, double* R, int* win)
{
    const int i = d / a.m, s = d % a.m;
    int first = i - 1;
    if (!a.periodic) first = min(max(first, 0), max(a.n - 3, 0));
    if (a.n < 3) first = i;
    const double lo_i = face_coord(a, i * a.m), hi_i = face_coord(a, (i + 1) * a.m);
    const double ctr = 0.5 * (lo_i + hi_i), wid = hi_i - lo_i;
    double A[3][3];
    int centre = 1;
    for (int r = 0; r < 3; ++r) {
        int cell = first + r;
        double off = 0.0;
        if (a.periodic) {
            if (cell < 0) { cell += a.n; off = -a.length; }
            if (cell >= a.n) { cell -= a.n; off = a.length; }
        }
        if (a.n < 3) cell = i;
        if (s == 0) win[3 * i + r] = cell;
        if (first + r == i) centre = r;
        const double x0 = (face_coord(a, cell * a.m) + off - ctr) / wid;
        const double x1 = (face_coord(a, (cell + 1) * a.m) + off - ctr) / wid;
        A[r][0] = 1.0;
        A[r][1] = 0.5 * (x0 + x1);
        A[r][2] = (x0 * x0 + x0 * x1 + x1 * x1) / 3.0;
    }
    double* row = R + 3 * (size_t)d;
    if (a.m == 1) {
        row[0] = row[1] = row[2] = 0.0;
        row[centre] = 1.0;
        return;
    }
    // inverse of A by cofactors
    const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    double inv[3][3];
    inv[0][0] = c00 / det;
    inv[1][0] = c01 / det;
    inv[2][0] = c02 / det;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    const double x0 = (face_coord(a, d) - ctr) / wid, x1 = (face_coord(a, d + 1) - ctr) / wid;
    const double As[3] = {1.0, 0.5 * (x0 + x1), (x0 * x0 + x0 * x1 + x1 * x1) / 3.0};
    for (int c = 0; c < 3; ++c) row[c] = As[0] * inv[0][c] + As[1] * inv[1][c] + As[2] * inv[2][c];
}

__global__ void k_noalloc_metric(AxisDesc ax, AxisDesc ay, AxisDesc az, double* Rx, double* Ry, double* Rz,
                                 int* wx, int* wy, int* wz, double* dz)
{
    const int Nx = ax.n * ax.m, Ny = ay.n * ay.m, Nz = az.n * az.m;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Nx + Ny + 2 * Nz; t += gridDim.x * blockDim.x) {
        if (t < Nx) axis_row(ax, t, Rx, wx);
        else if (t < Nx + Ny) axis_row(ay, t - Nx, Ry, wy);
        else if (t < Nx + Ny + Nz) axis_row(az, t - Nx - Ny, Rz, wz);
        else {
            const int k = t - Nx - Ny - Nz;
            dz[k] = face_coord(az, k + 1) - face_coord(az, k);
        }
    }
}

inline size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mr

using namespace mr;

extern "C" int mr_refine_velocity_noalloc(const mr_config* c, const double* U, const double* V, const double* W,
                                          double* Us, double* Vs, double* Ws, mr_stream stream)
{
    if (!c || !U || !V || !W || !Us || !Vs || !Ws) return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: NULL argument");
    if (c->struct_size != sizeof(mr_config)) return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: bad struct_size");
    const int n[3] = {c->nx, c->ny, c->nz}, m[3] = {c->mx, c->my, c->mz};
    const bool periodic = c->bc_horizontal == MR_PERIODIC;
    if (c->bc_horizontal != MR_PERIODIC && c->bc_horizontal != MR_WALLS)
        return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: bad bc_horizontal");
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || m[a] < 1 || m[a] > 8 || (m[a] > 1 && n[a] < 3) || (a < 2 && periodic && n[a] < 3) ||
            (long long)n[a] * m[a] > (1 << 20))
            return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: bad grid sizes");
    }
    if (!(c->lx > 0) || !(c->ly > 0) || !(c->stretch_gamma >= 0) || c->stretch_gamma > 20)
        return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: bad extents or stretching");
    // the narrowest dense z-layers of a tanh-clustered grid are the two at the
    // plates: a clustering that collapses them (tanh saturating in double
    // precision) would make the R matrices and the layer balance divide by zero
    {
        const int Nzd = c->nz * c->mz;
        const double gam = c->stretch_gamma;
        auto zface = [&](int i) {
            if (gam <= 0.0) return (double)i / (double)Nzd;
            return 0.5 * (1.0 + tanh(gam * (2.0 * ((double)i / (double)Nzd) - 1.0)) / tanh(gam));
        };
        const double lo = zface(1) - 0.0, hi = 1.0 - zface(Nzd - 1);
        if (!(lo > kMinLayer) || !(hi > kMinLayer))
            return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: stretching collapses the dense z-layers at the "
                                         "plates (width <= 1e-12)");
    }
    const void* ptrs[6] = {U, V, W, Us, Vs, Ws};
    for (const void* p : ptrs)
        if (!is_device_pointer(p)) return set_error(MR_ERR_ARG, "mr_refine_velocity_noalloc: pointers must be device memory");
    const int w = periodic ? 0 : 1;
    const int Nx = c->nx * c->mx, Ny = c->ny * c->my, Nz = c->nz * c->mz;
    // scratch layout: R rows, windows, dz, then the two refinement work arrays
    size_t off = 0;
    const size_t oRx = off; off += up256(3 * (size_t)Nx * 8);
    const size_t oRy = off; off += up256(3 * (size_t)Ny * 8);
    const size_t oRz = off; off += up256(3 * (size_t)Nz * 8);
    const size_t oDz = off; off += up256((size_t)Nz * 8);
    const size_t oWin = off; off += up256(3 * ((size_t)c->nx + c->ny + c->nz) * 4);
    const size_t oSW = off; off += up256((size_t)(Nz + 1) * c->ny * c->nx * 8);
    const size_t oSV = off; off += up256((size_t)Nz * (Ny + w) * c->nx * 8);
    if (off > MR_NOALLOC_SCRATCH_BYTES) {
        char msg[160];
        snprintf(msg, sizeof msg, "mr_refine_velocity_noalloc: grid needs %zu bytes of scratch, limit is %u", off,
                 (unsigned)MR_NOALLOC_SCRATCH_BYTES);
        return set_error(MR_ERR_ARG, msg);
    }
    void* base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    char* b = (char*)base;
    cudaStream_t st = (cudaStream_t)stream;
    AxisDesc ax{c->nx, c->mx, 0, c->lx, 0.0, periodic ? 1 : 0};
    AxisDesc ay{c->ny, c->my, 0, c->ly, 0.0, periodic ? 1 : 0};
    AxisDesc az{c->nz, c->mz, 1, 1.0, c->stretch_gamma, 0};
    int* wx = (int*)(b + oWin);
    k_noalloc_metric<<<64, 256, 0, st>>>(ax, ay, az, (double*)(b + oRx), (double*)(b + oRy), (double*)(b + oRz), wx,
                                         wx + 3 * c->nx, wx + 3 * (c->nx + c->ny), (double*)(b + oDz));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, "mr_refine_velocity_noalloc: metric kernel");
    Grid<double> g{};
    g.nx = c->nx; g.ny = c->ny; g.nz = c->nz; g.mx = c->mx; g.my = c->my; g.mz = c->mz;
    g.Nx = Nx; g.Ny = Ny; g.Nz = Nz; g.walls = w;
    g.ufx = Nx + w; g.vfy = Ny + w; g.cux = c->nx + w; g.cvy = c->ny + w;
    g.dx = c->lx / Nx; g.dy = c->ly / Ny; g.DX = c->lx / c->nx; g.DY = c->ly / c->ny;
    g.dz = (const double*)(b + oDz);
    g.Rx = (const double*)(b + oRx); g.Ry = (const double*)(b + oRy); g.Rz = (const double*)(b + oRz);
    g.wx = wx; g.wy = wx + 3 * c->nx; g.wz = wx + 3 * (c->nx + c->ny);
    e = launch_refine<double>(g, U, V, W, Us, Vs, Ws, (double*)(b + oSW), (double*)(b + oSV), st);
    return cuda_check(e, "mr_refine_velocity_noalloc: refinement launch");
}
