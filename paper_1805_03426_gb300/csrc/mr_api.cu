// C-ABI entry points (include/mr.h) and the host-side metric setup.
//
// Metric setup (Sections 3.1, 3.2): the dense grid is generated first (z by
// tanh clustering toward both plates, x and y uniform); coarse faces are every
// M-th dense face.  For every coarse cell of every axis the mass-conserving
// third-order interpolation matrix R = A_s A^-1 is formed once, in FP64, in
// coordinates local to the cell ((x - x_centre) / dX, the same matrix as in
// absolute coordinates but well conditioned).  The 3x3 system is inverted by
// its adjugate.  Near a wall the three-cell window is one-sided.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mr_internal.cuh"

namespace mr {

static thread_local std::string g_last_error;

int set_error(int code, const std::string& msg)
{
    g_last_error = msg;
    return code;
}

int cuda_check(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return MR_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_error(MR_ERR_OOM, m);
    return set_error(MR_ERR_CUDA, m);
}

// The device address of mapped pinned host memory (page-locked by the CUDA
// runtime, so addressable from kernels), else NULL.
static const double* host_mapped(const double* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? (const double*)a.devicePointer : nullptr;
}

bool is_device_pointer(const void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

StepCoef step_coef(const mr_config& cfg, int64_t s)
{
    // Section 2.2: leapfrog, averaging every N_p steps; s = 0 starts with Euler.
    if (s == 0) return {0.0, 1.0, cfg.dt};
    if (cfg.np_average > 0 && (s + 1) % cfg.np_average == 0) return {0.5, 0.5, 1.5 * cfg.dt};
    return {1.0, 0.0, 2.0 * cfg.dt};
}

// ---------------------------------------------------------------- metric setup

static void dense_z_faces(int N, double gamma, std::vector<double>& zf)
{
    zf.resize(N + 1);
    const double tg = gamma > 0.0 ? tanh(gamma) : 1.0;
    for (int k = 0; k <= N; ++k) {
        const double eta = (double)k / (double)N;
        zf[k] = gamma > 0.0 ? 0.5 * (1.0 + tanh(gamma * (2.0 * eta - 1.0)) / tg) : eta;
    }
    zf[0] = 0.0;
    zf[N] = 1.0;
}

// Row of cell means of 1, t, t^2 over [a, b] (the rows of A and A_s).
static void means3(double a, double b, double out[3])
{
    out[0] = 1.0;
    out[1] = 0.5 * (a + b);
    out[2] = (a * a + a * b + b * b) / 3.0;
}

static bool invert3(const double A[3][3], double inv[3][3])
{
    const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
    const double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
    const double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (det == 0.0 || !isfinite(det)) return false;
    const double r = 1.0 / det;
    inv[0][0] = c00 * r;
    inv[1][0] = c01 * r;
    inv[2][0] = c02 * r;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * r;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * r;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * r;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * r;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * r;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * r;
    return true;
}

// R for every coarse cell of one axis; R out [n*m][3] (one row per dense
// index), window out [n][3].
static bool axis_r(int n, int m, const std::vector<double>& dense_faces, bool periodic, double length,
                   std::vector<double>& R, std::vector<int>& win)
{
    R.assign((size_t)n * m * 3, 0.0);
    win.assign((size_t)n * 3, 0);
    for (int i = 0; i < n; ++i) {
        int first = i - 1;
        if (!periodic) first = std::min(std::max(first, 0), std::max(n - 3, 0));
        if (n < 3) first = i;  // only reachable with m == 1
        const double lo_i = dense_faces[(size_t)i * m], hi_i = dense_faces[(size_t)(i + 1) * m];
        const double ctr = 0.5 * (lo_i + hi_i), wid = hi_i - lo_i;
        double A[3][3];
        int centre_pos = 1;
        for (int r = 0; r < 3; ++r) {
            int cell = first + r;
            double off = 0.0;
            if (periodic) {
                if (cell < 0) { cell += n; off = -length; }
                if (cell >= n) { cell -= n; off = length; }
            }
            if (n < 3) cell = i;
            win[3 * i + r] = cell;
            if (first + r == i) centre_pos = r;
            const double a = (dense_faces[(size_t)cell * m] + off - ctr) / wid;
            const double b = (dense_faces[(size_t)(cell + 1) * m] + off - ctr) / wid;
            means3(a, b, A[r]);
        }
        if (m == 1) {
            R[3 * (size_t)i + centre_pos] = 1.0;
            continue;
        }
        double inv[3][3];
        if (!invert3(A, inv)) return false;
        for (int s = 0; s < m; ++s) {
            double As[3];
            means3((dense_faces[(size_t)i * m + s] - ctr) / wid, (dense_faces[(size_t)i * m + s + 1] - ctr) / wid, As);
            for (int c = 0; c < 3; ++c)
                R[((size_t)i * m + s) * 3 + c] = As[0] * inv[0][c] + As[1] * inv[1][c] + As[2] * inv[2][c];
        }
    }
    return true;
}

// Fourth-order face values (Section 2.2) along one axis of N cells with faces
// X[0..N]: w[4 f + q] weighs cell f - 2 + q at face f.  The face value is the
// derivative at X_f of the polynomial interpolating the primitive
// P(X_m) = sum_{c < m} h_c T_c at the stencil's faces, which is the
// polynomial whose cell averages over the stencil are the cell values:
//   T_f = sum_c T_c h_c sum_{m > c} L_m'(X_f)
// with L_m the Lagrange basis on the stencil faces.  Stencil: cells f-2..f+1;
// next to a wall (faces 1, N-1) the three domain-side cells; wall faces none.
static bool face4_axis(int N, const std::vector<double>& X, bool periodic, double length, std::vector<double>& w)
{
    w.assign(4 * ((size_t)N + 1), 0.0);
    if (N < (periodic ? 4 : 3)) return false;
    for (int f = 0; f <= N; ++f) {
        int first, n;
        if (periodic) {
            first = f - 2;
            n = 4;
        } else if (f == 0 || f == N) {
            continue;
        } else if (f == 1 || f == N - 1) {
            first = (f == 1) ? 0 : N - 3;
            n = 3;
        } else {
            first = f - 2;
            n = 4;
        }
        // stencil faces x_0..x_n relative to X_f, scaled by the stencil width
        double x[5];
        auto face = [&](int m) {            // unwrapped face m (may be < 0 or > N when periodic)
            double off = 0.0;
            while (m < 0) { m += N; off -= length; }
            while (m > N) { m -= N; off += length; }
            return X[m] + off;
        };
        const double xf = face(f), scale = face(first + n) - face(first);
        for (int m = 0; m <= n; ++m) x[m] = (face(first + m) - xf) / scale;
        const int t = f - first;            // the face is stencil node t
        double dL[5];
        for (int m = 0; m <= n; ++m) {
            if (m == t) {
                double sum = 0.0;
                for (int j = 0; j <= n; ++j)
                    if (j != t) sum += 1.0 / (x[t] - x[j]);
                dL[m] = sum;
            } else {
                double num = 1.0, den = 1.0;
                for (int j = 0; j <= n; ++j) {
                    if (j != m) den *= x[m] - x[j];
                    if (j != m && j != t) num *= x[t] - x[j];
                }
                dL[m] = num / den;
            }
        }
        for (int c = 0; c < n; ++c) {
            double tail = 0.0;
            for (int m = c + 1; m <= n; ++m) tail += dL[m];
            w[4 * (size_t)f + (first + c) - (f - 2)] = (x[c + 1] - x[c]) * tail;
        }
    }
    return true;
}

template <typename P>
static size_t metric_bytes(const mr_handle_s* h)
{
    const size_t nP = (size_t)h->Nz * 4 + 2 * ((size_t)h->Nz + 1) + 3 * ((size_t)h->Nx + h->Ny + h->Nz) +
                      4 * ((size_t)h->Nx + h->Ny + h->Nz + 3) + 8 * (size_t)h->Nz;
    return ((nP * sizeof(P) + 255) / 256) * 256;
}

// Copy the FP64 host metric, cast to P, into dst (device) and point g at it.
template <typename P>
static int upload_metric(mr_handle_s* h, char* dst, const int* dwin, Grid<P>& g)
{
    const mr_config& c = h->cfg;
    const int Nz = h->Nz;
    std::vector<P> host;
    host.reserve(metric_bytes<P>(h) / sizeof(P));
    std::vector<size_t> off;
    auto push = [&](const std::vector<double>& v) {
        off.push_back(host.size());
        for (double x : v) host.push_back((P)x);
    };
    std::vector<double> inv_dz(Nz), wlo(Nz + 1, 0.0), whi(Nz + 1, 0.0), cdn(Nz), cup(Nz);
    for (int k = 0; k < Nz; ++k) inv_dz[k] = 1.0 / h->dz[k];
    for (int k = 1; k < Nz; ++k) {
        wlo[k] = h->dz[k] / (h->dz[k - 1] + h->dz[k]);
        whi[k] = h->dz[k - 1] / (h->dz[k - 1] + h->dz[k]);
    }
    const bool dir = c.bc_plates == MR_DIRICHLET;
    for (int k = 0; k < Nz; ++k) {
        const double below = k > 0 ? h->zc[k] - h->zc[k - 1] : h->zc[0] - h->zf[0];
        const double above = k < Nz - 1 ? h->zc[k + 1] - h->zc[k] : h->zf[Nz] - h->zc[Nz - 1];
        cdn[k] = (k > 0 || dir) ? h->kappa / (h->dz[k] * below) : 0.0;
        cup[k] = (k < Nz - 1 || dir) ? h->kappa / (h->dz[k] * above) : 0.0;
    }
    const double dx = c.lx / h->Nx, dy = c.ly / h->Ny;
    const double kx2 = h->kappa / (dx * dx), ky2 = h->kappa / (dy * dy);
    std::vector<double> lz(8 * (size_t)Nz);
    for (int k = 0; k < Nz; ++k) {
        double* q = &lz[8 * (size_t)k];
        q[0] = wlo[k] * inv_dz[k];
        q[1] = whi[k] * inv_dz[k];
        q[2] = -(wlo[k + 1] * inv_dz[k]);
        q[3] = -(whi[k + 1] * inv_dz[k]);
        q[4] = cdn[k];
        q[5] = cup[k];
        q[6] = -(2.0 * kx2 + 2.0 * ky2 + cdn[k] + cup[k]);
        // plates at T = +0.5 (bottom) and -0.5 (top); cdn[0] = cup[Nz-1] = 0 when adiabatic
        q[7] = (k == 0 ? cdn[0] * 0.5 : 0.0) + (k == Nz - 1 ? cup[Nz - 1] * -0.5 : 0.0);
    }
    push(h->dz); push(inv_dz); push(wlo); push(whi); push(cdn); push(cup);
    push(h->Rx); push(h->Ry); push(h->Rz);
    push(h->f4x); push(h->f4y); push(h->f4z);
    push(lz);
    cudaError_t e = cudaMemcpy(dst, host.data(), host.size() * sizeof(P), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_check(e, "upload metric");
    const P* base = (const P*)dst;
    // the kernels see the rows the handle stores (a y-slab's, or the whole domain's)
    g.nx = c.nx; g.ny = h->nys; g.nz = c.nz; g.mx = c.mx; g.my = c.my; g.mz = c.mz;
    g.Nx = h->Nx; g.Ny = h->Nys; g.Nz = h->Nz; g.walls = h->w;
    g.ufx = h->Nx + h->w; g.vfy = h->Ny + h->w; g.cux = c.nx + h->w; g.cvy = c.ny + h->w;
    g.dirichlet = dir ? 1 : 0;
    g.dx = (P)dx; g.dy = (P)dy; g.DX = (P)(c.lx / c.nx); g.DY = (P)(c.ly / c.ny);
    g.inv_dx = (P)(1.0 / dx); g.inv_dy = (P)(1.0 / dy);
    g.kx2 = (P)kx2; g.ky2 = (P)ky2;
    g.hx = (P)(0.5 / dx); g.hy = (P)(0.5 / dy);
    g.dz = base + off[0]; g.inv_dz = base + off[1]; g.wlo = base + off[2]; g.whi = base + off[3];
    g.cdn = base + off[4]; g.cup = base + off[5]; g.Rx = base + off[6]; g.Ry = base + off[7]; g.Rz = base + off[8];
    g.f4x = base + off[9]; g.f4y = base + off[10]; g.f4z = base + off[11];
    g.lz = base + off[12];
    g.order4 = c.face_order == 4 ? 1 : 0;
    g.wx = dwin; g.wy = dwin + 3 * c.nx; g.wz = dwin + 3 * (c.nx + c.ny);
    return MR_OK;
}

static int validate(const mr_config* c, std::string* why)
{
    char b[256];
    if (c->struct_size != sizeof(mr_config)) {
        snprintf(b, sizeof b, "mr_config.struct_size %u != %zu", c->struct_size, sizeof(mr_config));
        *why = b;
        return MR_ERR_ARG;
    }
    const int n[3] = {c->nx, c->ny, c->nz}, m[3] = {c->mx, c->my, c->mz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || m[a] < 1 || m[a] > 8) { *why = "coarse sizes must be >= 1 and refinement in 1..8"; return MR_ERR_ARG; }
        if (m[a] > 1 && n[a] < 3) { *why = "an axis with refinement > 1 needs >= 3 coarse cells (R window)"; return MR_ERR_ARG; }
        if (a < 2 && c->bc_horizontal == MR_PERIODIC && n[a] < 3) { *why = "periodic axes need >= 3 coarse cells"; return MR_ERR_ARG; }
        if ((long long)n[a] * m[a] > (1LL << 20)) { *why = "dense size too large"; return MR_ERR_ARG; }
    }
    const long long cells = (long long)c->nx * c->mx * c->ny * c->my * c->nz * c->mz;
    if (cells > (1LL << 36)) { *why = "dense grid too large"; return MR_ERR_ARG; }
    if (!(c->lx > 0) || !(c->ly > 0) || !isfinite(c->lx) || !isfinite(c->ly)) { *why = "lx, ly must be positive"; return MR_ERR_ARG; }
    if (!(c->stretch_gamma >= 0) || c->stretch_gamma > 20) { *why = "stretch_gamma must be in [0, 20]"; return MR_ERR_ARG; }
    if (!(c->ra > 0) || !(c->pr_or_sc > 0) || !isfinite(c->ra * c->pr_or_sc)) { *why = "ra and pr_or_sc must be positive"; return MR_ERR_ARG; }
    if (!(c->dt > 0) || !isfinite(c->dt)) { *why = "dt must be positive"; return MR_ERR_ARG; }
    if (c->precision != MR_F64 && c->precision != MR_F32) { *why = "precision must be MR_F64 or MR_F32"; return MR_ERR_ARG; }
    if (c->velocity_mode != MR_VEL_STORED && c->velocity_mode != MR_VEL_FUSED && c->velocity_mode != MR_VEL_XFUSED) {
        *why = "bad velocity_mode";
        return MR_ERR_ARG;
    }
    if (c->bc_plates != MR_DIRICHLET && c->bc_plates != MR_ADIABATIC) { *why = "bad bc_plates"; return MR_ERR_ARG; }
    if (c->bc_horizontal != MR_PERIODIC && c->bc_horizontal != MR_WALLS) { *why = "bad bc_horizontal"; return MR_ERR_ARG; }
    if (c->diffz_implicit != 0 && c->diffz_implicit != 1) { *why = "diffz_implicit must be 0 or 1"; return MR_ERR_ARG; }
    if (c->face_order != 2 && c->face_order != 4) { *why = "face_order must be 2 or 4"; return MR_ERR_ARG; }
    if (c->face_order == 4) {
        const bool per = c->bc_horizontal == MR_PERIODIC;
        const int need = per ? 4 : 3;
        if ((long long)c->nx * c->mx < need || (long long)c->ny * c->my < need || (long long)c->nz * c->mz < 3) {
            *why = "face_order 4 needs >= 4 dense cells on periodic axes and >= 3 between walls";
            return MR_ERR_ARG;
        }
        if (c->velocity_mode == MR_VEL_FUSED) { *why = "MR_VEL_FUSED supports face_order 2 only"; return MR_ERR_ARG; }
    }
    if (c->velocity_mode != MR_VEL_STORED && !fused_supported(*c, why)) return MR_ERR_ARG;
    if (c->slab_ny != 0) {
        if (c->velocity_mode != MR_VEL_FUSED) { *why = "a y-slab handle needs MR_VEL_FUSED"; return MR_ERR_ARG; }
        if (c->slab_ny < 0 || c->slab_j0 < 0 || c->slab_j0 + c->slab_ny > c->ny) {
            *why = "y-slab rows out of range (0 <= slab_j0, slab_j0 + slab_ny <= ny)";
            return MR_ERR_ARG;
        }
        if ((c->slab_ny * c->my) % 16) { *why = "a y-slab needs slab_ny * my % 16 == 0"; return MR_ERR_ARG; }
    } else if (c->slab_j0 != 0) {
        *why = "slab_j0 without slab_ny";
        return MR_ERR_ARG;
    }
    return MR_OK;
}

}  // namespace mr

using namespace mr;

// ---------------------------------------------------------------- ABI

extern "C" {

const char* mr_last_error(void) { return g_last_error.c_str(); }

int mr_config_default(mr_config* c)
{
    if (!c) return set_error(MR_ERR_ARG, "mr_config_default: NULL");
    memset(c, 0, sizeof(*c));
    c->struct_size = sizeof(mr_config);
    c->nx = c->ny = c->nz = 16;
    c->mx = c->my = c->mz = 2;
    c->lx = c->ly = 1.0;
    c->stretch_gamma = 0.0;
    c->ra = 1e6;
    c->pr_or_sc = 7.0;
    c->dt = 1e-3;
    c->precision = MR_F64;
    c->velocity_mode = MR_VEL_STORED;
    c->np_average = 50;
    c->bc_plates = MR_DIRICHLET;
    c->bc_horizontal = MR_PERIODIC;
    c->diffz_implicit = 0;
    c->face_order = 2;
    return MR_OK;
}

void mr_destroy(mr_handle h)
{
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    DeviceBuffers& b = h->buf;
    void* ptrs[] = {b.T[0], b.T[1], b.T[2], b.U64, b.V64, b.W64, b.Us, b.Vs, b.Ws, b.scrW, b.scrV,
                    b.metric, b.red, b.nu2, b.stage, b.tri};
    for (void* p : ptrs)
        if (p) dev_free(p);
    DeviceBuffers::Level& n = b.next;
    void* nptrs[] = {n.U64, n.V64, n.W64, n.Us, n.Vs, n.Ws, n.xwy, n.xuo, n.xvr, b.lerpc};
    for (void* p : nptrs)
        if (p) dev_free(p);
    if (h->elt == 4) {
        void* cptrs[] = {n.Uc, n.Vc, n.Wc};
        for (void* p : cptrs)
            if (p) dev_free(p);
    }
    void* xptrs[] = {b.xwy, b.xuo, b.xvr, b.xlc, b.diag, b.cpad, b.fsc, n.cpad, b.halo, b.tcinv, b.nup};
    for (void* p : xptrs)
        if (p) dev_free(p);
    for (int q = 0; q < 2; ++q) {
        void* sptrs[] = {b.sU[q], b.sV[q], b.sW[q]};
        for (void* p : sptrs)
            if (p) dev_free(p);
        if (b.stg_copied[q]) cudaEventDestroy(b.stg_copied[q]);
        if (b.stg_free[q]) cudaEventDestroy(b.stg_free[q]);
    }
    void* aptrs[] = {h->adj.cp, h->adj.seg, h->adj.mu, h->adj.face, h->adj.scr, h->adj.out};
    for (void* p : aptrs)
        if (p) dev_free(p);
    if (h->elt == 4) {
        if (b.Uc) dev_free(b.Uc);
        if (b.Vc) dev_free(b.Vc);
        if (b.Wc) dev_free(b.Wc);
    }
    cudaSetDevice(cur);
    delete h;
}

int mr_create(const mr_config* cfg, mr_handle* out)
{
    if (!cfg || !out) return set_error(MR_ERR_ARG, "mr_create: NULL argument");
    *out = nullptr;
    std::string why;
    int rc = validate(cfg, &why);
    if (rc) return set_error(rc, "mr_create: " + why);
    mr_handle_s* h = new mr_handle_s();
    h->cfg = *cfg;
    cudaGetDevice(&h->device);
    const mr_config& c = h->cfg;
    h->w = c.bc_horizontal == MR_WALLS ? 1 : 0;
    h->Nx = c.nx * c.mx; h->Ny = c.ny * c.my; h->Nz = c.nz * c.mz;
    h->slab = c.slab_ny > 0;
    h->nys = h->slab ? c.slab_ny : c.ny;
    h->Nys = h->nys * c.my;
    h->ncell = (size_t)h->Nx * h->Nys * h->Nz;
    h->nU = (size_t)h->Nz * h->Ny * (h->Nx + h->w);
    h->nV = (size_t)h->Nz * (h->Ny + h->w) * h->Nx;
    h->nW = (size_t)(h->Nz + 1) * h->Ny * h->Nx;
    h->ncU = (size_t)c.nz * c.ny * (c.nx + h->w);
    h->ncV = (size_t)c.nz * (c.ny + h->w) * c.nx;
    h->ncW = (size_t)(c.nz + 1) * c.ny * c.nx;
    h->elt = c.precision == MR_F64 ? 8 : 4;
    h->kappa = 1.0 / sqrt(c.ra * c.pr_or_sc);

    // Section 3.1 grid, Section 3.2 R matrices (FP64, host)
    dense_z_faces(h->Nz, c.stretch_gamma, h->zf);
    h->zc.resize(h->Nz);
    h->dz.resize(h->Nz);
    for (int k = 0; k < h->Nz; ++k) {
        h->zc[k] = 0.5 * (h->zf[k] + h->zf[k + 1]);
        h->dz[k] = h->zf[k + 1] - h->zf[k];
        if (!(h->dz[k] > 1e-12)) {
            // tanh clustering saturating in double precision collapses the layers at the plates
            delete h;
            return set_error(MR_ERR_ARG, "mr_create: stretching collapses a dense z-layer (width <= 1e-12)");
        }
    }
    std::vector<double> xf(h->Nx + 1), yf(h->Ny + 1);
    for (int i = 0; i <= h->Nx; ++i) xf[i] = c.lx * i / h->Nx;
    for (int j = 0; j <= h->Ny; ++j) yf[j] = c.ly * j / h->Ny;
    const bool per = c.bc_horizontal == MR_PERIODIC;
    if (!axis_r(c.nx, c.mx, xf, per, c.lx, h->Rx, h->wx) || !axis_r(c.ny, c.my, yf, per, c.ly, h->Ry, h->wy) ||
        !axis_r(c.nz, c.mz, h->zf, false, 1.0, h->Rz, h->wz)) {
        delete h;
        return set_error(MR_ERR_ARG, "mr_create: singular interpolation matrix (degenerate grid)");
    }
    h->f4x.assign(4 * ((size_t)h->Nx + 1), 0.0);
    h->f4y.assign(4 * ((size_t)h->Ny + 1), 0.0);
    h->f4z.assign(4 * ((size_t)h->Nz + 1), 0.0);
    if (c.face_order == 4 && (!face4_axis(h->Nx, xf, per, c.lx, h->f4x) || !face4_axis(h->Ny, yf, per, c.ly, h->f4y) ||
                              !face4_axis(h->Nz, h->zf, false, 1.0, h->f4z))) {
        delete h;
        return set_error(MR_ERR_ARG, "mr_create: fourth-order face stencil does not fit the grid");
    }

    DeviceBuffers& b = h->buf;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess && bytes) e = dev_malloc(p, bytes);
    };
    for (int q = 0; q < 3; ++q) alloc(&b.T[q], h->ncell * h->elt);
    alloc((void**)&b.U64, h->ncU * 8);
    alloc((void**)&b.V64, h->ncV * 8);
    alloc((void**)&b.W64, h->ncW * 8);
    if (h->elt == 4) {
        alloc(&b.Uc, h->ncU * 4);
        alloc(&b.Vc, h->ncV * 4);
        alloc(&b.Wc, h->ncW * 4);
    } else {
        b.Uc = b.U64; b.Vc = b.V64; b.Wc = b.W64;
    }
    if (c.velocity_mode == MR_VEL_STORED) {
        alloc(&b.Us, h->nU * h->elt);
        alloc(&b.Vs, h->nV * h->elt);
        alloc(&b.Ws, h->nW * h->elt);
        alloc(&b.scrW, (size_t)(h->Nz + 1) * c.ny * c.nx * h->elt);
        alloc(&b.scrV, (size_t)h->Nz * (h->Ny + h->w) * c.nx * h->elt);
    }
    const size_t mb64 = metric_bytes<double>(h), mb32 = metric_bytes<float>(h);
    const size_t nwin = 3 * ((size_t)c.nx + c.ny + c.nz);
    alloc(&b.metric, mb64 + mb32 + nwin * sizeof(int));
    h->red_blocks = 152 * 8;
    alloc((void**)&b.red, (size_t)h->red_blocks * 2 * sizeof(double));
    alloc((void**)&b.nu2, (3 + 2 * kPlateBlocks) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(b.nu2, 0, (3 + 2 * kPlateBlocks) * sizeof(double));   // the block count
    h->stage_bytes = std::min<size_t>((size_t)64 << 20, std::max<size_t>(h->ncell * 8, 1 << 16));
    alloc(&b.stage, h->stage_bytes);
    if (c.diffz_implicit) alloc(&b.tri, h->ncell * h->elt);
    if (c.velocity_mode == MR_VEL_XFUSED) {
        b.nxg = c.nx + 8;
        alloc((void**)&b.xwy, (size_t)(h->Nz + 1) * h->Ny * b.nxg * 4);
        alloc((void**)&b.xuo, (size_t)h->Nz * h->Ny * b.nxg * 4);
        alloc((void**)&b.xvr, (size_t)h->Nz * (h->Ny + 1) * b.nxg * 4);
        alloc((void**)&b.xlc, (size_t)h->Nz * 32 * 4);
        alloc(&b.scrW, (size_t)(h->Nz + 1) * c.ny * c.nx * h->elt);
    } else if (c.velocity_mode == MR_VEL_FUSED) {
        alloc((void**)&b.xlc, (size_t)h->Nz * 32 * 4);   // layer constants of the fused step
        alloc((void**)&b.fsc, (size_t)c.nz * 32 * 4);    // slab constants
        alloc((void**)&b.cpad, fused_pad_floats(c.nx, h->nys, c.nz) * 4);
        if (h->slab) alloc((void**)&b.halo, (size_t)6 * h->Nz * h->Nx * 4);
    }
    if (e != cudaSuccess) {
        int r = cuda_check(e, "mr_create: device allocation");
        mr_destroy(h);
        return r;
    }
    std::vector<int> win;
    win.insert(win.end(), h->wx.begin(), h->wx.end());
    win.insert(win.end(), h->wy.begin(), h->wy.end());
    win.insert(win.end(), h->wz.begin(), h->wz.end());
    int* dwin = (int*)((char*)b.metric + mb64 + mb32);
    e = cudaMemcpy(dwin, win.data(), win.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        int r = cuda_check(e, "mr_create: upload windows");
        mr_destroy(h);
        return r;
    }
    rc = upload_metric<double>(h, (char*)b.metric, dwin, h->g64);
    if (!rc) rc = upload_metric<float>(h, (char*)b.metric + mb64, dwin, h->g32);
    if (!rc && b.xlc) {
        const std::vector<float> lc =
            xfused_layer_constants(h->Nz, h->zf.data(), h->zc.data(), h->dz.data(), h->kappa, c.lx / h->Nx,
                                   c.ly / h->Ny, c.bc_plates == MR_DIRICHLET,
                                   c.face_order == 4 ? h->f4z.data() : nullptr, &b.xlcw);
        // periodic uniform x and y: every face has the same fourth-order weights
        for (int q = 0; q < 4; ++q) {
            b.xw4[q] = (float)(2.0 * h->f4x[q]);
            b.xw4[4 + q] = (float)(2.0 * h->f4y[q]);
        }
        rc = cuda_check(cudaMemcpy(b.xlc, lc.data(), lc.size() * 4, cudaMemcpyHostToDevice), "mr_create: layer constants");
        // x is uniform and periodic: every coarse cell has the same R_x rows
        for (int q = 0; q < 12; ++q) b.xrx[q] = (float)h->Rx[(size_t)(q / 3) * 3 + q % 3];
        for (int q = 0; q < 12 && (size_t)q < h->Ry.size(); ++q) b.xry[q] = (float)h->Ry[(size_t)(q / 3) * 3 + q % 3];
    }
    if (!rc && b.fsc) {
        const std::vector<float> sc = fused_slab_constants(c.nz, c.mz, h->Rz.data(), h->dz.data());
        rc = cuda_check(cudaMemcpy(b.fsc, sc.data(), sc.size() * 4, cudaMemcpyHostToDevice), "mr_create: slab constants");
    }
    if (rc) {
        mr_destroy(h);
        return rc;
    }
    *out = h;
    return MR_OK;
}

int mr_grid(mr_handle h, int32_t* dims3, double* zf_host)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_grid: NULL handle");
    if (dims3) { dims3[0] = h->Nx; dims3[1] = h->Nys; dims3[2] = h->Nz; }
    if (zf_host) memcpy(zf_host, h->zf.data(), h->zf.size() * sizeof(double));
    return MR_OK;
}

int mr_set_dt(mr_handle h, double dt)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_set_dt: NULL handle");
    if (!(dt > 0) || !isfinite(dt)) return set_error(MR_ERR_ARG, "mr_set_dt: dt must be positive");
    h->cfg.dt = dt;
    return MR_OK;
}

int mr_step_index(mr_handle h, int64_t* s)
{
    if (!h || !s) return set_error(MR_ERR_ARG, "mr_step_index: NULL argument");
    *s = h->step;
    return MR_OK;
}

// Copy n elements of dtype sd at src (host or device) into the device buffer
// dst of dtype dd, converting through the staging buffer when needed.
static int copy_in(mr_handle h, const void* src, int sd, void* dst, int dd, size_t n, cudaStream_t st)
{
    const size_t se = sd == MR_F64 ? 8 : 4, de = dd == MR_F64 ? 8 : 4;
    cudaError_t e;
    if (sd == dd) {
        e = cudaMemcpyAsync(dst, src, n * se, cudaMemcpyDefault, st);
        return cuda_check(e, "copy in");
    }
    if (is_device_pointer(src)) return cuda_check(launch_convert<double>(src, sd, dst, dd, n, st), "convert");
    const size_t chunk = h->stage_bytes / se;
    for (size_t o = 0; o < n; o += chunk) {
        const size_t c = std::min(chunk, n - o);
        e = cudaMemcpyAsync(h->buf.stage, (const char*)src + o * se, c * se, cudaMemcpyDefault, st);
        if (e != cudaSuccess) return cuda_check(e, "copy in (stage)");
        e = launch_convert<double>(h->buf.stage, sd, (char*)dst + o * de, dd, c, st);
        if (e != cudaSuccess) return cuda_check(e, "convert (stage)");
    }
    return MR_OK;
}

static int copy_out(mr_handle h, const void* src, int sd, void* dst, int dd, size_t n, cudaStream_t st)
{
    const size_t se = sd == MR_F64 ? 8 : 4, de = dd == MR_F64 ? 8 : 4;
    cudaError_t e;
    if (sd == dd) return cuda_check(cudaMemcpyAsync(dst, src, n * se, cudaMemcpyDefault, st), "copy out");
    if (is_device_pointer(dst)) return cuda_check(launch_convert<double>(src, sd, dst, dd, n, st), "convert");
    const size_t chunk = h->stage_bytes / de;
    for (size_t o = 0; o < n; o += chunk) {
        const size_t c = std::min(chunk, n - o);
        e = launch_convert<double>((const char*)src + o * se, sd, h->buf.stage, dd, c, st);
        if (e != cudaSuccess) return cuda_check(e, "convert (stage)");
        e = cudaMemcpyAsync((char*)dst + o * de, h->buf.stage, c * de, cudaMemcpyDefault, st);
        if (e != cudaSuccess) return cuda_check(e, "copy out (stage)");
    }
    return MR_OK;
}

// Refine the handle's coarse faces into device dense-face buffers (Section 3.2).
static int refine_into(mr_handle h, void* dUs, void* dVs, void* dWs, cudaStream_t st)
{
    DeviceBuffers& b = h->buf;
    cudaError_t e = cudaSuccess;
    if (!b.scrW) e = dev_malloc(&b.scrW, (size_t)(h->Nz + 1) * h->cfg.ny * h->cfg.nx * h->elt);
    if (e == cudaSuccess && !b.scrV) e = dev_malloc(&b.scrV, (size_t)h->Nz * (h->Ny + h->w) * h->cfg.nx * h->elt);
    if (e != cudaSuccess) return cuda_check(e, "refinement scratch");
    if (h->cfg.precision == MR_F64)
        e = launch_refine<double>(h->g64, (const double*)b.Uc, (const double*)b.Vc, (const double*)b.Wc,
                                  (double*)dUs, (double*)dVs, (double*)dWs, (double*)b.scrW, (double*)b.scrV, st);
    else
        e = launch_refine<float>(h->g32, (const float*)b.Uc, (const float*)b.Vc, (const float*)b.Wc,
                                 (float*)dUs, (float*)dVs, (float*)dWs, (float*)b.scrW, (float*)b.scrV, st);
    return cuda_check(e, "refinement launch");
}

}  // extern "C"

// Load a coarse velocity into the handle's current level: FP64 copy, the
// precision-P coarse faces, and what the velocity mode steps from (dense faces
// for MR_VEL_STORED, the split-x intermediates for MR_VEL_XFUSED).
static int derive_velocity(mr_handle h, bool convert, cudaStream_t st);

static int load_velocity(mr_handle h, const double* U, const double* V, const double* W, cudaStream_t st)
{
    DeviceBuffers& b = h->buf;
    int rc;
    const bool f32 = h->cfg.precision == MR_F32;
    bool fetched = false;
    const double *mU = host_mapped(U), *mV = host_mapped(V), *mW = host_mapped(W);
    if (mU && mV && mW) {
        // pinned host faces: the SMs read them over the host link, writing the
        // FP64 copy and the FP32 faces in the same pass
        cudaError_t e = launch_fetch_f64(mU, b.U64, f32 ? (float*)b.Uc : nullptr, h->ncU, st);
        if (e == cudaSuccess) e = launch_fetch_f64(mV, b.V64, f32 ? (float*)b.Vc : nullptr, h->ncV, st);
        if (e == cudaSuccess) e = launch_fetch_f64(mW, b.W64, f32 ? (float*)b.Wc : nullptr, h->ncW, st);
        if (e == cudaErrorInvalidValue) cudaGetLastError();   // unaligned: the copy path below
        else if (e != cudaSuccess) return cuda_check(e, "fetch coarse faces");
        else fetched = true;
    }
    if (!fetched) {
        if ((rc = copy_in(h, U, MR_F64, b.U64, MR_F64, h->ncU, st))) return rc;
        if ((rc = copy_in(h, V, MR_F64, b.V64, MR_F64, h->ncV, st))) return rc;
        if ((rc = copy_in(h, W, MR_F64, b.W64, MR_F64, h->ncW, st))) return rc;
    }
    return derive_velocity(h, !fetched, st);
}

// What the velocity mode steps from, given the FP64 coarse faces in U64/V64/W64
// (and, unless convert, their FP32 rounding already in Uc/Vc/Wc).
static int derive_velocity(mr_handle h, bool convert, cudaStream_t st)
{
    DeviceBuffers& b = h->buf;
    h->maxdiv_valid = false;
    if (h->cfg.velocity_mode == MR_VEL_FUSED && convert) {
        // the FP64 faces straight to the padded FP32 copy (and the FP32 faces)
        cudaError_t e = launch_fused_pad64(b.U64, b.V64, b.W64, b.cpad, (float*)b.Uc, (float*)b.Vc, (float*)b.Wc,
                                           h->cfg.nx, h->cfg.ny, h->cfg.nz, h->slab ? h->cfg.slab_j0 : 0, h->nys, st);
        return cuda_check(e, "padded coarse faces");
    }
    if (h->cfg.precision == MR_F32 && convert) {
        // the handle's own FP64 device faces: no pointer queries
        cudaError_t e = launch_convert<double>(b.U64, MR_F64, b.Uc, MR_F32, h->ncU, st);
        if (e == cudaSuccess) e = launch_convert<double>(b.V64, MR_F64, b.Vc, MR_F32, h->ncV, st);
        if (e == cudaSuccess) e = launch_convert<double>(b.W64, MR_F64, b.Wc, MR_F32, h->ncW, st);
        if (e != cudaSuccess) return cuda_check(e, "coarse faces to FP32");
    }
    if (h->cfg.velocity_mode == MR_VEL_XFUSED) {
        cudaError_t e = launch_xfused_prep(h->g32, (const float*)b.Uc, (const float*)b.Vc, (const float*)b.Wc,
                                           (float*)b.scrW, b.xwy, b.xuo, b.xvr, b.nxg, st);
        if (e != cudaSuccess) return cuda_check(e, "split-x intermediates");
    }
    if (h->cfg.velocity_mode == MR_VEL_FUSED) {
        cudaError_t e = launch_fused_pad((const float*)b.Uc, (const float*)b.Vc, (const float*)b.Wc, b.cpad,
                                         h->cfg.nx, h->cfg.ny, h->cfg.nz, h->slab ? h->cfg.slab_j0 : 0, h->nys, st);
        if (e != cudaSuccess) return cuda_check(e, "padded coarse faces");
    }
    if (h->cfg.velocity_mode == MR_VEL_STORED) return refine_into(h, b.Us, b.Vs, b.Ws, st);
    return MR_OK;
}

// One time step of the scalar.  alpha = 0: the current velocity; otherwise the
// velocity (1 - alpha) U^{n-1} + alpha U^n between the current level and the
// next one (temporal refinement, Section 3.4).
static int one_step(mr_handle h, double alpha, cudaStream_t st, double* Tc = nullptr)
{
    DeviceBuffers& b = h->buf;
    const DeviceBuffers::Level& nx = b.next;
    const bool lerp = alpha != 0.0, implz = h->cfg.diffz_implicit != 0;
    const StepCoef c = step_coef(h->cfg, h->step);
    const int in = 3 - h->ip - h->ic;
    const void* Tm1 = h->step == 0 ? b.T[h->ic] : b.T[h->ip];
    cudaError_t e;
    if (h->cfg.precision == MR_F64) {
        const double* A[3] = {(const double*)b.Us, (const double*)b.Vs, (const double*)b.Ws};
        const double* B[3] = {(const double*)nx.Us, (const double*)nx.Vs, (const double*)nx.Ws};
        e = lerp ? launch_step_stored_lerp<double>(h->g64, A, B, alpha, (const double*)Tm1, (const double*)b.T[h->ic],
                                                   (double*)b.T[in], c, implz, st)
                 : launch_step_stored<double>(h->g64, A[0], A[1], A[2], (const double*)Tm1, (const double*)b.T[h->ic],
                                              (double*)b.T[in], c, implz, st);
        if (e == cudaSuccess && implz) e = launch_zsolve<double>(h->g64, (double*)b.T[in], 0.5 * c.gdt, (double*)b.tri, st);
    } else if (h->cfg.velocity_mode == MR_VEL_XFUSED) {
        const float* A[3] = {b.xwy, b.xuo, b.xvr};
        const float* B[3] = {nx.xwy, nx.xuo, nx.xvr};
        e = launch_step_xfused_f32(h->g32, A, lerp ? B : nullptr, alpha, b.nxg, b.xlc, b.xlcw, b.xrx, b.xw4,
                                   (const float*)Tm1,
                                   (const float*)b.T[h->ic], (float*)b.T[in], c, st);
    } else if (h->cfg.velocity_mode == MR_VEL_FUSED) {
        FusedInputs fin{b.cpad, {}, {}, 0, b.fsc, b.xlc, b.xrx, b.xry, Tc, b.tcinv};
        // the rows beyond the y edges of T^s and T^{s-1}
        const int lm = h->step == 0 ? h->ic : h->ip;
        if (h->slab) {
            const size_t hp = (size_t)h->Nz * h->Nx;
            fin.hs[0] = b.halo + (2 * h->ic) * hp;
            fin.hn[0] = b.halo + (2 * h->ic + 1) * hp;
            fin.hs[1] = b.halo + (2 * lm) * hp;
            fin.hn[1] = b.halo + (2 * lm + 1) * hp;
            fin.hstride = h->Nx;
        } else {
            const size_t row = (size_t)(h->Nys - 1) * h->Nx;
            fin.hs[0] = (const float*)b.T[h->ic] + row;
            fin.hn[0] = (const float*)b.T[h->ic];
            fin.hs[1] = (const float*)b.T[lm] + row;
            fin.hn[1] = (const float*)b.T[lm];
            fin.hstride = (size_t)h->Nx * h->Nys;
        }
        e = cudaSuccess;
        if (lerp) {
            // the refinement is linear: refining the interpolated coarse faces
            // interpolates the refined ones (the periodic images interpolate too)
            e = launch_lerp_f32(b.cpad, nx.cpad, alpha, b.lerpc, fused_pad_floats(h->cfg.nx, h->nys, h->cfg.nz), st);
            fin.pad = b.lerpc;
        }
        if (e == cudaSuccess)
            e = launch_step_fused_f32(h->g32, fin, (const float*)Tm1, (const float*)b.T[h->ic], (float*)b.T[in], c, st);
    } else {
        const float* A[3] = {(const float*)b.Us, (const float*)b.Vs, (const float*)b.Ws};
        const float* B[3] = {(const float*)nx.Us, (const float*)nx.Vs, (const float*)nx.Ws};
        e = lerp ? launch_step_stored_lerp<float>(h->g32, A, B, alpha, (const float*)Tm1, (const float*)b.T[h->ic],
                                                  (float*)b.T[in], c, implz, st)
                 : launch_step_stored<float>(h->g32, A[0], A[1], A[2], (const float*)Tm1, (const float*)b.T[h->ic],
                                             (float*)b.T[in], c, implz, st);
        if (e == cudaSuccess && implz) e = launch_zsolve<float>(h->g32, (float*)b.T[in], 0.5 * c.gdt, (float*)b.tri, st);
    }
    if (e != cudaSuccess) return cuda_check(e, "scalar step launch");
    h->ip = h->ic;
    h->ic = in;
    h->halo_set[in] = false;       // a y-slab's new level has no halo rows yet
    ++h->step;
    return MR_OK;
}

// Exchange the current velocity level with the next one.
static void swap_levels(DeviceBuffers& b)
{
    DeviceBuffers::Level& n = b.next;
    std::swap(b.U64, n.U64); std::swap(b.V64, n.V64); std::swap(b.W64, n.W64);
    std::swap(b.Uc, n.Uc); std::swap(b.Vc, n.Vc); std::swap(b.Wc, n.Wc);
    std::swap(b.Us, n.Us); std::swap(b.Vs, n.Vs); std::swap(b.Ws, n.Ws);
    std::swap(b.xwy, n.xwy); std::swap(b.xuo, n.xuo); std::swap(b.xvr, n.xvr);
    std::swap(b.cpad, n.cpad);
}

// Allocate the next velocity level (once per handle).
static int alloc_next(mr_handle h)
{
    DeviceBuffers& b = h->buf;
    DeviceBuffers::Level& n = b.next;
    if (n.U64) return MR_OK;
    cudaError_t e = cudaSuccess;
    auto alloc = [&](void** p, size_t bytes) {
        if (e == cudaSuccess && bytes) e = dev_malloc(p, bytes);
    };
    alloc((void**)&n.U64, h->ncU * 8);
    alloc((void**)&n.V64, h->ncV * 8);
    alloc((void**)&n.W64, h->ncW * 8);
    if (h->elt == 4) {
        alloc(&n.Uc, h->ncU * 4);
        alloc(&n.Vc, h->ncV * 4);
        alloc(&n.Wc, h->ncW * 4);
    }
    const int mode = h->cfg.velocity_mode;
    if (mode == MR_VEL_STORED) {
        alloc(&n.Us, h->nU * h->elt);
        alloc(&n.Vs, h->nV * h->elt);
        alloc(&n.Ws, h->nW * h->elt);
    } else if (mode == MR_VEL_XFUSED) {
        alloc((void**)&n.xwy, (size_t)(h->Nz + 1) * h->Ny * b.nxg * 4);
        alloc((void**)&n.xuo, (size_t)h->Nz * h->Ny * b.nxg * 4);
        alloc((void**)&n.xvr, (size_t)h->Nz * (h->Ny + 1) * b.nxg * 4);
    } else {
        const size_t np = fused_pad_floats(h->cfg.nx, h->nys, h->cfg.nz);
        alloc((void**)&n.cpad, np * 4);
        alloc((void**)&b.lerpc, np * 4);
    }
    if (e != cudaSuccess) {
        void* ptrs[] = {n.U64, n.V64, n.W64, n.Us, n.Vs, n.Ws, n.xwy, n.xuo, n.xvr, n.cpad, b.lerpc};
        for (void* p : ptrs)
            if (p) dev_free(p);
        if (h->elt == 4) {
            void* cptrs[] = {n.Uc, n.Vc, n.Wc};
            for (void* p : cptrs)
                if (p) dev_free(p);
        }
        n = DeviceBuffers::Level();
        b.lerpc = nullptr;
        return cuda_check(e, "mr_scalar_coarse_step: device allocation");
    }
    if (h->elt == 8) {
        n.Uc = n.U64; n.Vc = n.V64; n.Wc = n.W64;
    }
    return MR_OK;
}

extern "C" {

int mr_refine_velocity(mr_handle h, const double* U, const double* V, const double* W, void* Us, void* Vs,
                       void* Ws, mr_stream stream)
{
    if (!h || !U || !V || !W) return set_error(MR_ERR_ARG, "mr_refine_velocity: NULL argument");
    if ((Us || Vs || Ws) && !(Us && Vs && Ws))
        return set_error(MR_ERR_ARG, "mr_refine_velocity: Us, Vs, Ws must be all NULL or all set");
    if (Us && h->cfg.velocity_mode != MR_VEL_STORED &&
        (!is_device_pointer(Us) || !is_device_pointer(Vs) || !is_device_pointer(Ws)))
        return set_error(MR_ERR_ARG, "mr_refine_velocity: in fused mode Us, Vs, Ws must be device memory");
    if (Us && h->slab) return set_error(MR_ERR_ARG, "mr_refine_velocity: no dense faces from a y-slab handle");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    int rc = load_velocity(h, U, V, W, st);
    if (rc) return rc;
    h->have_velocity = true;
    if (!Us) return MR_OK;
    const int P = h->cfg.precision;
    if (h->cfg.velocity_mode != MR_VEL_STORED) return refine_into(h, Us, Vs, Ws, st);
    if ((rc = copy_out(h, b.Us, P, Us, P, h->nU, st))) return rc;
    if ((rc = copy_out(h, b.Vs, P, Vs, P, h->nV, st))) return rc;
    return copy_out(h, b.Ws, P, Ws, P, h->nW, st);
}

int mr_stage_velocity(mr_handle h, const double* U, const double* V, const double* W, mr_stream copy_stream)
{
    if (!h || !U || !V || !W) return set_error(MR_ERR_ARG, "mr_stage_velocity: NULL argument");
    DeviceBuffers& b = h->buf;
    cudaStream_t cs = (cudaStream_t)copy_stream;
    cudaError_t e = cudaSuccess;
    if (!b.stg_free[1]) {
        // both slots and their events, or nothing (a failed call leaves no half state)
        double* p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        const size_t n[3] = {h->ncU, h->ncV, h->ncW};
        for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = dev_malloc((void**)&p[k], n[k % 3] * 8);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (double* x : p)
                if (x) dev_free(x);
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            return cuda_check(e, "mr_stage_velocity: staging slots");
        }
        for (int q = 0; q < 2; ++q) {
            b.sU[q] = p[3 * q];
            b.sV[q] = p[3 * q + 1];
            b.sW[q] = p[3 * q + 2];
            b.stg_copied[q] = ev[2 * q];
            b.stg_free[q] = ev[2 * q + 1];
        }
    }
    const int q = b.stg_next;
    // the slot's memory may still be read by work queued before the refinement
    // that released it, or written by an earlier copy on another stream (a wait
    // on a never-recorded event passes at once)
    e = cudaStreamWaitEvent(cs, b.stg_free[q], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b.stg_copied[q], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.sU[q], U, h->ncU * 8, cudaMemcpyDefault, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.sV[q], V, h->ncV * 8, cudaMemcpyDefault, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.sW[q], W, h->ncW * 8, cudaMemcpyDefault, cs);
    if (e == cudaSuccess) e = cudaEventRecord(b.stg_copied[q], cs);
    if (e != cudaSuccess) return cuda_check(e, "mr_stage_velocity: copy");
    b.stg_ready = q;
    b.stg_next = q ^ 1;
    return MR_OK;
}

int mr_refine_velocity_staged(mr_handle h, mr_stream stream)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_refine_velocity_staged: NULL argument");
    DeviceBuffers& b = h->buf;
    if (b.stg_ready < 0) return set_error(MR_ERR_STATE, "mr_refine_velocity_staged: call mr_stage_velocity first");
    cudaStream_t st = (cudaStream_t)stream;
    const int q = b.stg_ready;
    cudaError_t e = cudaStreamWaitEvent(st, b.stg_copied[q], 0);
    if (e != cudaSuccess) return cuda_check(e, "mr_refine_velocity_staged: wait");
    // the staged slot becomes the handle's FP64 faces; the old faces' memory
    // becomes the slot, free once the work queued so far has run
    std::swap(b.U64, b.sU[q]);
    std::swap(b.V64, b.sV[q]);
    std::swap(b.W64, b.sW[q]);
    if (h->elt == 8) {
        b.Uc = b.U64;
        b.Vc = b.V64;
        b.Wc = b.W64;
    }
    b.stg_ready = -1;
    int rc = derive_velocity(h, true, st);
    e = cudaEventRecord(b.stg_free[q], st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_check(e, "mr_refine_velocity_staged: record");
    h->have_velocity = true;
    return MR_OK;
}

int mr_scalar_coarse_step(mr_handle h, const double* U, const double* V, const double* W, int32_t mt,
                          mr_stream stream)
{
    if (!h || !U || !V || !W) return set_error(MR_ERR_ARG, "mr_scalar_coarse_step: NULL argument");
    if (mt < 1) return set_error(MR_ERR_ARG, "mr_scalar_coarse_step: mt must be >= 1");
    if (h->slab && mt > 1)
        return set_error(MR_ERR_ARG, "mr_scalar_coarse_step: a y-slab handle takes one step per call (mt = 1)");
    if (h->slab && !(h->halo_set[h->ic] && (h->step == 0 || h->halo_set[h->ip])))
        return set_error(MR_ERR_STATE, "mr_scalar_coarse_step: set the y-slab's halo rows first");
    if (!h->have_velocity || !h->have_scalar)
        return set_error(MR_ERR_STATE, "mr_scalar_coarse_step: call mr_refine_velocity and mr_set_scalar first");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    int rc = alloc_next(h);
    if (rc) return rc;
    swap_levels(b);                    // load U^n into the next level's buffers
    rc = load_velocity(h, U, V, W, st);
    swap_levels(b);
    if (rc) return rc;
    for (int32_t i = 0; i < mt; ++i)
        if ((rc = one_step(h, (double)i / (double)mt, st))) return rc;
    swap_levels(b);                    // U^n is now the current velocity
    h->maxdiv_valid = false;
    return MR_OK;
}

int mr_set_scalar(mr_handle h, const void* T0, int32_t dtype, mr_stream stream)
{
    if (!h || !T0) return set_error(MR_ERR_ARG, "mr_set_scalar: NULL argument");
    if (dtype != MR_F64 && dtype != MR_F32) return set_error(MR_ERR_ARG, "mr_set_scalar: bad dtype");
    cudaStream_t st = (cudaStream_t)stream;
    h->ip = 0;
    h->ic = 1;
    int rc = copy_in(h, T0, dtype, h->buf.T[h->ic], h->cfg.precision, h->ncell, st);
    if (rc) return rc;
    rc = cuda_check(cudaMemcpyAsync(h->buf.T[h->ip], h->buf.T[h->ic], h->ncell * h->elt,
                                    cudaMemcpyDeviceToDevice, st), "mr_set_scalar");
    if (rc) return rc;
    h->step = 0;
    h->have_scalar = true;
    for (bool& f : h->halo_set) f = false;
    return MR_OK;
}

int mr_get_scalar(mr_handle h, void* T, void* Tprev, int32_t dtype, mr_stream stream)
{
    if (!h || (!T && !Tprev)) return set_error(MR_ERR_ARG, "mr_get_scalar: NULL argument");
    if (dtype != MR_F64 && dtype != MR_F32) return set_error(MR_ERR_ARG, "mr_get_scalar: bad dtype");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_get_scalar: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if (h->cfg.velocity_mode != MR_VEL_STORED && fused_take_error(st) == MR_ERR_TIMEOUT)
        return set_error(MR_ERR_TIMEOUT, "mr_get_scalar: a fused step kernel gave up a bounded wait");
    if (T && (rc = copy_out(h, h->buf.T[h->ic], h->cfg.precision, T, dtype, h->ncell, st))) return rc;
    if (Tprev && (rc = copy_out(h, h->buf.T[h->ip], h->cfg.precision, Tprev, dtype, h->ncell, st))) return rc;
    return MR_OK;
}

int mr_scalar_step(mr_handle h, int64_t nsteps, mr_stream stream)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_scalar_step: NULL handle");
    if (nsteps < 0) return set_error(MR_ERR_ARG, "mr_scalar_step: nsteps < 0");
    if (!h->have_velocity || !h->have_scalar)
        return set_error(MR_ERR_STATE, "mr_scalar_step: call mr_refine_velocity and mr_set_scalar first");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->slab && nsteps > 1)
        return set_error(MR_ERR_ARG, "mr_scalar_step: a y-slab handle takes one step per call (halo rows between)");
    if (h->slab && nsteps == 1 && !(h->halo_set[h->ic] && (h->step == 0 || h->halo_set[h->ip])))
        return set_error(MR_ERR_STATE, "mr_scalar_step: set the y-slab's halo rows (mr_set_halo_rows) first");
    for (int64_t q = 0; q < nsteps; ++q) {
        const int rc = one_step(h, 0.0, st);
        if (rc) return rc;
    }
    return MR_OK;
}

// The device address of a device pointer, or of pinned host memory; NULL for
// pageable host memory.
static void* device_alias(void* p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

int mr_scalar_step_coupled(mr_handle h, double* nu2, double* Tc, mr_stream stream)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_scalar_step_coupled: NULL handle");
    double* dnu = nullptr;
    double* dtc = nullptr;
    if (nu2 && !(dnu = (double*)device_alias(nu2)))
        return set_error(MR_ERR_ARG, "mr_scalar_step_coupled: nu2 must be device or pinned host memory");
    if (Tc && !(dtc = (double*)device_alias(Tc)))
        return set_error(MR_ERR_ARG, "mr_scalar_step_coupled: Tc must be device or pinned host memory");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    const bool fused = h->cfg.velocity_mode == MR_VEL_FUSED;
    int rc;
    if (fused && (dtc || dnu) && !b.nup) {
        // the fused step writes Tc itself (per coarse slab, 1 / (mx my sum of its
        // dz) in FP64); one launch forms the plate Nusselt numbers of the new level
        const mr_config& c = h->cfg;
        cudaError_t e = dev_malloc(&b.tcinv, (size_t)c.nz * sizeof(double));
        if (e == cudaSuccess) e = dev_malloc(&b.nup, fused_plate_nu_work() * sizeof(double));
        std::vector<double> inv(c.nz);
        for (int K = 0; K < c.nz; ++K) {
            double z = 0.0;
            for (int k = K * c.mz; k < (K + 1) * c.mz; ++k) z += h->dz[k];
            inv[K] = 1.0 / (z * c.mx * c.my);
        }
        if (e == cudaSuccess) e = cudaMemcpy(b.tcinv, inv.data(), inv.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(b.nup, 0, sizeof(double));      // the launch's block count
        if (e != cudaSuccess) {
            dev_free(b.tcinv);
            dev_free(b.nup);
            b.tcinv = nullptr;
            b.nup = nullptr;
            return cuda_check(e, "mr_scalar_step_coupled: coupled outputs");
        }
    }
    if (fused && dtc) {
        // the step kernel writes the upscaled coarse scalar of the new level itself
        if (h->slab && !(h->halo_set[h->ic] && (h->step == 0 || h->halo_set[h->ip])))
            return set_error(MR_ERR_STATE, "mr_scalar_step_coupled: set the y-slab's halo rows first");
        if (!h->have_velocity || !h->have_scalar)
            return set_error(MR_ERR_STATE, "mr_scalar_step_coupled: call mr_refine_velocity and mr_set_scalar first");
        rc = one_step(h, 0.0, st, dtc);
    } else {
        rc = mr_scalar_step(h, 1, stream);
    }
    if (rc) return rc;
    cudaError_t e = cudaSuccess;
    if (fused) {
        if (dnu)
            e = launch_fused_plate_nu(h->g32, (const float*)h->buf.T[h->ic], 1.0 / (h->zc[0] - h->zf[0]),
                                      1.0 / (h->zf[h->Nz] - h->zc[h->Nz - 1]), b.nup, dnu, st);
    } else {
        if (dnu) {
            const double zz[2] = {h->zc[0] - h->zf[0], h->zf[h->Nz] - h->zc[h->Nz - 1]};
            e = h->cfg.precision == MR_F64
                    ? launch_plate_nu<double>(h->g64, (const double*)h->buf.T[h->ic], zz, h->buf.nu2, st)
                    : launch_plate_nu<float>(h->g32, (const float*)h->buf.T[h->ic], zz, h->buf.nu2, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dnu, h->buf.nu2, 2 * sizeof(double), cudaMemcpyDefault, st);
        }
        if (e == cudaSuccess && dtc)
            e = h->cfg.precision == MR_F64 ? launch_upscale<double>(h->g64, (const double*)h->buf.T[h->ic], dtc, st)
                                           : launch_upscale<float>(h->g32, (const float*)h->buf.T[h->ic], dtc, st);
    }
    return cuda_check(e, "mr_scalar_step_coupled");
}

int mr_get_boundary_rows(mr_handle h, void* south, void* north, mr_stream stream)
{
    if (!h || (!south && !north)) return set_error(MR_ERR_ARG, "mr_get_boundary_rows: NULL argument");
    if (!h->slab) return set_error(MR_ERR_ARG, "mr_get_boundary_rows: not a y-slab handle");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_get_boundary_rows: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t row = (size_t)h->Nx * h->elt, plane = row * h->Nys;
    const char* T = (const char*)h->buf.T[h->ic];
    cudaError_t e = cudaSuccess;
    if (south) e = cudaMemcpy2DAsync(south, row, T, plane, row, h->Nz, cudaMemcpyDefault, st);
    if (e == cudaSuccess && north)
        e = cudaMemcpy2DAsync(north, row, T + (size_t)(h->Nys - 1) * row, plane, row, h->Nz, cudaMemcpyDefault, st);
    return cuda_check(e, "mr_get_boundary_rows");
}

int mr_set_halo_rows(mr_handle h, const void* below, const void* above, mr_stream stream)
{
    if (!h || !below || !above) return set_error(MR_ERR_ARG, "mr_set_halo_rows: NULL argument");
    if (!h->slab) return set_error(MR_ERR_ARG, "mr_set_halo_rows: not a y-slab handle");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_set_halo_rows: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t n = (size_t)h->Nz * h->Nx;
    float* dst = h->buf.halo + 2 * (size_t)h->ic * n;
    cudaError_t e = cudaMemcpyAsync(dst, below, n * h->elt, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst + n, above, n * h->elt, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_set_halo_rows");
    h->halo_set[h->ic] = true;
    return MR_OK;
}

int mr_plate_nu(mr_handle h, double* nu2, mr_stream stream)
{
    if (!h || !nu2) return set_error(MR_ERR_ARG, "mr_plate_nu: NULL argument");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_plate_nu: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    const double zz[2] = {h->zc[0] - h->zf[0], h->zf[h->Nz] - h->zc[h->Nz - 1]};
    cudaError_t e = h->cfg.precision == MR_F64
                        ? launch_plate_nu<double>(h->g64, (const double*)h->buf.T[h->ic], zz, h->buf.nu2, st)
                        : launch_plate_nu<float>(h->g32, (const float*)h->buf.T[h->ic], zz, h->buf.nu2, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_plate_nu: launch");
    return cuda_check(cudaMemcpyAsync(nu2, h->buf.nu2, 2 * sizeof(double), cudaMemcpyDefault, st), "mr_plate_nu: copy");
}

static int reduce_partials(mr_handle h, int nper, std::vector<double>& out, cudaStream_t st)
{
    out.resize((size_t)h->red_blocks * nper);
    cudaError_t e = cudaMemcpyAsync(out.data(), h->buf.red, out.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_check(e, "reduction");
}

static int max_divergence(mr_handle h, double* out, cudaStream_t st)
{
    cudaError_t e;
    const DeviceBuffers& b = h->buf;
    if (h->cfg.velocity_mode == MR_VEL_XFUSED)
        e = launch_xfused_max_f32(h->g32, 1, b.xwy, b.xuo, b.xvr, b.nxg, b.xlc, b.xlcw, b.xrx, b.red, h->red_blocks, st);
    else if (h->cfg.velocity_mode == MR_VEL_FUSED)
        e = launch_fused_max_f32(h->g32, 1, FusedInputs{b.cpad, {}, {}, 0, b.fsc, b.xlc, b.xrx, b.xry, nullptr, nullptr}, b.red,
                                 h->red_blocks, st);
    else if (h->cfg.precision == MR_F64)
        e = launch_maxdiv<double>(h->g64, (const double*)b.Us, (const double*)b.Vs, (const double*)b.Ws, b.red,
                                  h->red_blocks, st);
    else
        e = launch_maxdiv<float>(h->g32, (const float*)b.Us, (const float*)b.Vs, (const float*)b.Ws, b.red,
                                 h->red_blocks, st);
    if (e != cudaSuccess) return cuda_check(e, "max divergence: launch");
    std::vector<double> p;
    int rc = reduce_partials(h, 1, p, st);
    if (rc) return rc;
    double m = 0.0;
    for (double v : p) m = std::max(m, v);
    *out = m;
    return MR_OK;
}

int mr_scalar_stats(mr_handle h, mr_stats* out, mr_stream stream)
{
    if (!h || !out) return set_error(MR_ERR_ARG, "mr_scalar_stats: NULL argument");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_scalar_stats: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    if (h->cfg.velocity_mode != MR_VEL_STORED && fused_take_error(st) == MR_ERR_TIMEOUT)
        return set_error(MR_ERR_TIMEOUT, "mr_scalar_stats: a fused step kernel gave up a bounded wait");
    const void* T = h->buf.T[h->ic];
    const double dxdy = (h->cfg.lx / h->Nx) * (h->cfg.ly / h->Ny);
    double vtot = 0.0;
    for (int k = 0; k < h->Nz; ++k) vtot += h->dz[k];
    vtot *= dxdy * (double)h->Nx * (double)h->Nys;
    std::vector<double> p;
    cudaError_t e;
    e = h->cfg.precision == MR_F64 ? launch_moments<double>(h->g64, (const double*)T, 0.0, 0, h->buf.red, h->red_blocks, st)
                                   : launch_moments<float>(h->g32, (const float*)T, 0.0, 0, h->buf.red, h->red_blocks, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_scalar_stats: launch");
    int rc = reduce_partials(h, 2, p, st);
    if (rc) return rc;
    double s = 0.0, bad = 0.0;
    for (int q = 0; q < h->red_blocks; ++q) { s += p[2 * q]; bad += p[2 * q + 1]; }
    out->integral = s * dxdy;
    out->mean = out->integral / vtot;
    e = h->cfg.precision == MR_F64
            ? launch_moments<double>(h->g64, (const double*)T, out->mean, 1, h->buf.red, h->red_blocks, st)
            : launch_moments<float>(h->g32, (const float*)T, out->mean, 1, h->buf.red, h->red_blocks, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_scalar_stats: launch");
    if ((rc = reduce_partials(h, 2, p, st))) return rc;
    double v = 0.0;
    for (int q = 0; q < h->red_blocks; ++q) v += p[2 * q];
    out->var = v * dxdy / vtot;
    double nu[2];
    if ((rc = mr_plate_nu(h, nu, stream))) return rc;
    if ((rc = cuda_check(cudaStreamSynchronize(st), "mr_scalar_stats: sync"))) return rc;
    out->nu_bot = nu[0];
    out->nu_top = nu[1];
    out->max_div = 0.0;
    if (h->have_velocity) {
        // the divergence depends on the velocity alone: once per velocity
        if (!h->maxdiv_valid) {
            if ((rc = max_divergence(h, &h->maxdiv, st))) return rc;
            h->maxdiv_valid = true;
        }
        out->max_div = h->maxdiv;
    }
    if (bad > 0.0) return set_error(MR_ERR_NONFINITE, "mr_scalar_stats: the scalar holds NaN or Inf");
    return MR_OK;
}

int mr_cfl_dt(mr_handle h, double cfl, double* dt_out, mr_stream stream)
{
    if (!h || !dt_out) return set_error(MR_ERR_ARG, "mr_cfl_dt: NULL argument");
    if (!(cfl > 0)) return set_error(MR_ERR_ARG, "mr_cfl_dt: cfl must be positive");
    if (!h->have_velocity) return set_error(MR_ERR_STATE, "mr_cfl_dt: call mr_refine_velocity first");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    const void *us = b.Us, *vs = b.Vs, *ws = b.Ws;
    bool tmp = false;
    cudaError_t e = cudaSuccess;
    if (h->cfg.velocity_mode == MR_VEL_XFUSED) {
        // the split-x kernel forms the dense faces in registers: one pass, no dense storage
        e = launch_xfused_max_f32(h->g32, 2, b.xwy, b.xuo, b.xvr, b.nxg, b.xlc, b.xlcw, b.xrx, b.red, h->red_blocks, st);
    } else if (h->cfg.velocity_mode == MR_VEL_FUSED) {
        // the fused kernel forms the dense faces in registers from the coarse ones
        e = launch_fused_max_f32(h->g32, 2, FusedInputs{b.cpad, {}, {}, 0, b.fsc, b.xlc, b.xrx, b.xry, nullptr, nullptr}, b.red,
                                 h->red_blocks, st);
    } else if (h->cfg.velocity_mode != MR_VEL_STORED) {
        // dense faces are not kept: refine into temporary buffers once
        void *a = nullptr, *bb = nullptr, *c = nullptr;
        e = dev_malloc(&a, h->nU * h->elt);
        if (e == cudaSuccess) e = dev_malloc(&bb, h->nV * h->elt);
        if (e == cudaSuccess) e = dev_malloc(&c, h->nW * h->elt);
        if (e != cudaSuccess) {
            dev_free(a); dev_free(bb); dev_free(c);
            return cuda_check(e, "mr_cfl_dt: temporary dense faces");
        }
        int rc = refine_into(h, a, bb, c, st);
        if (rc) { dev_free(a); dev_free(bb); dev_free(c); return rc; }
        us = a; vs = bb; ws = c;
        tmp = true;
    }
    if (h->cfg.velocity_mode == MR_VEL_STORED || tmp)
        e = h->cfg.precision == MR_F64
                ? launch_cfl<double>(h->g64, (const double*)us, (const double*)vs, (const double*)ws, b.red, h->red_blocks, st)
                : launch_cfl<float>(h->g32, (const float*)us, (const float*)vs, (const float*)ws, b.red, h->red_blocks, st);
    std::vector<double> p;
    int rc = e != cudaSuccess ? cuda_check(e, "mr_cfl_dt: launch") : reduce_partials(h, 1, p, st);
    if (tmp) { dev_free((void*)us); dev_free((void*)vs); dev_free((void*)ws); }
    if (rc) return rc;
    if (h->cfg.velocity_mode != MR_VEL_STORED && fused_take_error(st) == MR_ERR_TIMEOUT)
        return set_error(MR_ERR_TIMEOUT, "mr_cfl_dt: a fused kernel gave up a bounded wait");
    double m = 0.0;
    for (double v : p) m = std::max(m, v);
    if (!(m > 0)) return set_error(MR_ERR_ARG, "mr_cfl_dt: zero velocity");
    *dt_out = cfl / m;
    return MR_OK;
}

int mr_debug_index_maps(mr_handle h, int32_t* out, size_t cap)
{
    if (!h || !out) return set_error(MR_ERR_ARG, "mr_debug_index_maps: NULL argument");
    const mr_config& c = h->cfg;
    const size_t need = (size_t)h->Nx + h->Ny + h->Nz + 3 * ((size_t)c.nx + c.ny + c.nz);
    if (cap < need) return set_error(MR_ERR_ARG, "mr_debug_index_maps: buffer too small");
    // the maps are read back from the device copy the kernels use
    std::vector<int> win(3 * ((size_t)c.nx + c.ny + c.nz));
    const char* base = (const char*)h->buf.metric + metric_bytes<double>(h) + metric_bytes<float>(h);
    cudaError_t e = cudaMemcpy(win.data(), base, win.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_check(e, "mr_debug_index_maps");
    int32_t* p = out;
    for (int i = 0; i < h->Nx; ++i) *p++ = i / c.mx;
    for (int j = 0; j < h->Ny; ++j) *p++ = j / c.my;
    for (int k = 0; k < h->Nz; ++k) *p++ = k / c.mz;
    for (int v : win) *p++ = v;
    return MR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- adjoint (host orchestration)

namespace {

using namespace mr;

// FP64 volume mean and variance of a dense field in precision P (two-pass).
int field_moments(mr_handle h, const void* T, double* mean, double* var, cudaStream_t st)
{
    const double dxdy = (h->cfg.lx / h->Nx) * (h->cfg.ly / h->Ny);
    double vtot = 0.0;
    for (int k = 0; k < h->Nz; ++k) vtot += h->dz[k];
    vtot *= dxdy * (double)h->Nx * (double)h->Nys;
    std::vector<double> p;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = h->cfg.precision == MR_F64
                            ? launch_moments<double>(h->g64, (const double*)T, *mean, pass, h->buf.red, h->red_blocks, st)
                            : launch_moments<float>(h->g32, (const float*)T, *mean, pass, h->buf.red, h->red_blocks, st);
        if (e != cudaSuccess) return cuda_check(e, "moments");
        int rc = reduce_partials(h, 2, p, st);
        if (rc) return rc;
        double s = 0.0;
        for (int q = 0; q < h->red_blocks; ++q) s += p[2 * q];
        if (pass == 0) *mean = s * dxdy / vtot;
        else *var = s * dxdy / vtot;
    }
    return MR_OK;
}

int field_nu(mr_handle h, const void* T, double nu[2], cudaStream_t st)
{
    const double zz[2] = {h->zc[0] - h->zf[0], h->zf[h->Nz] - h->zc[h->Nz - 1]};
    cudaError_t e = h->cfg.precision == MR_F64 ? launch_plate_nu<double>(h->g64, (const double*)T, zz, h->buf.nu2, st)
                                               : launch_plate_nu<float>(h->g32, (const float*)T, zz, h->buf.nu2, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nu, h->buf.nu2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_check(e, "plate Nusselt");
}

cudaError_t step_buffers(mr_handle h, const void* Tm1, const void* T, void* Tp1, int64_t s, cudaStream_t st)
{
    const StepCoef c = step_coef(h->cfg, s);
    const void* tm = s == 0 ? T : Tm1;
    const DeviceBuffers& b = h->buf;
    if (h->cfg.precision == MR_F64)
        return launch_step_stored<double>(h->g64, (const double*)b.Us, (const double*)b.Vs, (const double*)b.Ws,
                                          (const double*)tm, (const double*)T, (double*)Tp1, c, false, st);
    return launch_step_stored<float>(h->g32, (const float*)b.Us, (const float*)b.Vs, (const float*)b.Ws,
                                     (const float*)tm, (const float*)T, (float*)Tp1, c, false, st);
}

void adj_free(mr_handle h)
{
    auto& a = h->adj;
    void* ptrs[] = {a.cp, a.seg, a.mu, a.face, a.scr, a.out, a.face32};
    for (void* p : ptrs)
        if (p) dev_free(p);
    a.cp = a.seg = a.mu = nullptr;
    a.face = a.scr = a.out = nullptr;
    a.face32 = nullptr;
    a.cp_pairs = 0;
    a.ready = false;
}

}  // namespace

extern "C" {

int mr_adjoint_forward(mr_handle h, int64_t nsteps, int32_t ck, const double* wnu, const double* wvar, double* loss,
                       mr_stream stream)
{
    if (!h || !loss) return set_error(MR_ERR_ARG, "mr_adjoint_forward: NULL argument");
    if (nsteps < 1 || ck < 1) return set_error(MR_ERR_ARG, "mr_adjoint_forward: nsteps and checkpoint_every must be >= 1");
    if (h->cfg.velocity_mode != MR_VEL_STORED || h->cfg.diffz_implicit || h->cfg.face_order != 2)
        return set_error(MR_ERR_ARG, "mr_adjoint_forward: needs MR_VEL_STORED, explicit diffusion and face_order 2");
    if (!h->have_velocity || !h->have_scalar || h->step != 0)
        return set_error(MR_ERR_STATE, "mr_adjoint_forward: call mr_refine_velocity and mr_set_scalar first");
    cudaStream_t st = (cudaStream_t)stream;
    auto& a = h->adj;
    const size_t cpairs = (size_t)((nsteps + ck - 1) / ck);
    const size_t fb = h->ncell * h->elt;
    if (a.cp && (a.cp_pairs < cpairs || a.ck < ck)) adj_free(h);
    cudaError_t e = cudaSuccess;
    if (!a.cp) {
        e = dev_malloc(&a.cp, cpairs * 2 * fb);
        if (e == cudaSuccess) e = dev_malloc(&a.seg, ((size_t)ck + 1) * fb);
        if (e == cudaSuccess) e = dev_malloc(&a.mu, 3 * fb);
        if (e == cudaSuccess) e = dev_malloc((void**)&a.face, (h->nU + h->nV + h->nW) * sizeof(double));
        const size_t nscr = (size_t)(h->Nz + 1) * h->cfg.ny * h->cfg.nx + (size_t)h->Nz * (h->Ny + h->w) * h->cfg.nx;
        if (e == cudaSuccess) e = dev_malloc((void**)&a.scr, nscr * sizeof(double));
        if (e == cudaSuccess) e = dev_malloc((void**)&a.out, (h->ncell + h->ncU + h->ncV + h->ncW) * sizeof(double));
        if (e == cudaSuccess && h->cfg.precision == MR_F32) {
            e = dev_malloc((void**)&a.face32, (h->nU + h->nV + h->nW) * sizeof(float));
            if (e == cudaSuccess) e = cudaMemset(a.face32, 0, (h->nU + h->nV + h->nW) * sizeof(float));
        }
        if (e != cudaSuccess) {
            adj_free(h);
            return cuda_check(e, "mr_adjoint_forward: checkpoint store");
        }
        a.cp_pairs = cpairs;
        a.ck = ck;
    }
    a.ready = false;
    a.S = nsteps;
    a.ck = ck;
    a.wnu.assign(wnu ? wnu : nullptr, wnu ? wnu + nsteps + 1 : nullptr);
    a.wvar.assign(wvar ? wvar : nullptr, wvar ? wvar + nsteps + 1 : nullptr);
    if (a.wnu.empty()) a.wnu.assign(nsteps + 1, 0.0);
    if (a.wvar.empty()) a.wvar.assign(nsteps + 1, 0.0);
    a.mean.assign(nsteps + 1, 0.0);
    double L = 0.0;
    for (int64_t s = 0; s <= nsteps; ++s) {
        const void* Tc = h->buf.T[h->ic];
        if (s < nsteps && s % ck == 0) {
            char* pair = (char*)a.cp + (size_t)(s / ck) * 2 * fb;
            e = cudaMemcpyAsync(pair, h->buf.T[h->ip], fb, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(pair + fb, Tc, fb, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_forward: checkpoint");
        }
        int rc;
        if (a.wnu[s] != 0.0) {
            double nu[2];
            if ((rc = field_nu(h, Tc, nu, st))) return rc;
            L += a.wnu[s] * nu[0];
        }
        if (a.wvar[s] != 0.0) {
            double mean = 0.0, var = 0.0;
            if ((rc = field_moments(h, Tc, &mean, &var, st))) return rc;
            a.mean[s] = mean;
            L += a.wvar[s] * var;
        }
        if (s < nsteps && (rc = mr_scalar_step(h, 1, stream))) return rc;
    }
    *loss = L;
    a.ready = true;
    return cuda_check(cudaStreamSynchronize(st), "mr_adjoint_forward");
}

int mr_adjoint_backward(mr_handle h, double gscale, void* gT0, int32_t gT0_dtype, double* gU, double* gV, double* gW,
                        mr_stream stream)
{
    if (!h) return set_error(MR_ERR_ARG, "mr_adjoint_backward: NULL handle");
    if (gT0 && gT0_dtype != MR_F64 && gT0_dtype != MR_F32) return set_error(MR_ERR_ARG, "mr_adjoint_backward: bad dtype");
    auto& a = h->adj;
    if (!a.ready) return set_error(MR_ERR_STATE, "mr_adjoint_backward: call mr_adjoint_forward first");
    cudaStream_t st = (cudaStream_t)stream;
    const int P = h->cfg.precision;
    const size_t fb = h->ncell * h->elt;
    const int64_t S = a.S;
    const int ck = a.ck;
    const double dxdy = (h->cfg.lx / h->Nx) * (h->cfg.ly / h->Ny);
    double vtot = 0.0;
    for (int k = 0; k < h->Nz; ++k) vtot += h->dz[k];
    vtot *= dxdy * (double)h->Nx * (double)h->Nys;
    const double zb = h->zc[0] - h->zf[0];
    // direct terms in adjoint-density units (per unit volume)
    auto s_nu = [&](int64_t s) { return -gscale * a.wnu[s] / ((double)h->Nx * h->Ny * zb * dxdy * h->dz[0]); };
    auto s_var = [&](int64_t s) { return gscale * a.wvar[s] * 2.0 / vtot; };
    char* mu[3] = {(char*)a.mu, (char*)a.mu + fb, (char*)a.mu + 2 * fb};
    int in = 0, ic = 1, ip = 2;     // mu^{s+1}, mu^s, mu^{s-1}
    cudaError_t e = cudaMemsetAsync(a.face, 0, (h->nU + h->nV + h->nW) * sizeof(double), st);
    if (e == cudaSuccess && a.face32) e = cudaMemsetAsync(a.face32, 0, (h->nU + h->nV + h->nW) * sizeof(float), st);
    // levels S and S-1 start from their direct terms (T^S, T^{S-1} are the handle's current pair)
    auto direct = [&](const void* T, int64_t s, void* out) {
        return P == MR_F64 ? launch_adj_direct<double>(h->g64, (const double*)T, s_nu(s), s_var(s), a.mean[s], (double*)out, st)
                           : launch_adj_direct<float>(h->g32, (const float*)T, s_nu(s), s_var(s), a.mean[s], (float*)out, st);
    };
    if (e == cudaSuccess) e = direct(h->buf.T[h->ic], S, mu[in]);
    if (e == cudaSuccess) e = direct(h->buf.T[h->ip], S - 1, mu[ic]);
    if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: init");
    double* fU = a.face;
    double* fV = a.face + h->nU;
    double* fW = a.face + h->nU + h->nV;
    const DeviceBuffers& b = h->buf;
    const int64_t nseg = (S + ck - 1) / ck;
    for (int64_t c = nseg - 1; c >= 0; --c) {
        const int64_t c0 = c * ck, e1 = std::min<int64_t>(c0 + ck, S);
        // recompute T^{c0-1} .. T^{e1-1} into seg[0 .. e1-c0]
        char* seg = (char*)a.seg;
        const char* pair = (const char*)a.cp + (size_t)c * 2 * fb;
        e = cudaMemcpyAsync(seg, pair, 2 * fb, cudaMemcpyDeviceToDevice, st);
        for (int64_t s = c0; e == cudaSuccess && s < e1 - 1; ++s)
            e = step_buffers(h, seg + (s - c0) * fb, seg + (s - c0 + 1) * fb, seg + (s - c0 + 2) * fb, s, st);
        if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: recompute");
        for (int64_t s = e1 - 1; s >= c0; --s) {
            const void* Ts = seg + (s - c0 + 1) * fb;
            const void* Tsm = seg + (s - c0) * fb;
            const StepCoef co = step_coef(h->cfg, s);
            const bool euler = (s == 0);
            const int64_t sp = euler ? 0 : s - 1;
            if (P == MR_F64)
                e = launch_adj_step<double>(h->g64, (const double*)b.Us, (const double*)b.Vs, (const double*)b.Ws,
                                            (const double*)Ts, (const double*)Tsm, (const double*)mu[in],
                                            (double*)mu[ic], (double*)mu[ip], s_nu(sp), s_var(sp), a.mean[sp], fU, fV,
                                            fW, co, euler, st);
            else
                e = launch_adj_step<float>(h->g32, (const float*)b.Us, (const float*)b.Vs, (const float*)b.Ws,
                                           (const float*)Ts, (const float*)Tsm, (const float*)mu[in], (float*)mu[ic],
                                           (float*)mu[ip], s_nu(sp), s_var(sp), a.mean[sp], a.face32,
                                           a.face32 + h->nU, a.face32 + h->nU + h->nV, co, euler, st);
            if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: launch");
            if (!euler) {
                const int t = in;
                in = ic;
                ic = ip;
                ip = t;
            }
        }
        if (P == MR_F32) {
            // the segment's FP32 face-gradient sums into the FP64 totals
            e = launch_flush_faces(a.face32, a.face, h->nU + h->nV + h->nW, st);
            if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: flush");
        }
    }
    // after the Euler step the level-0 adjoint density is mu[ic]
    int rc;
    double* out = a.out;
    if (gT0) {
        const bool dev = is_device_pointer(gT0);
        void* dst = dev ? gT0 : (void*)out;
        const int dd = dev ? gT0_dtype : MR_F64;
        e = P == MR_F64 ? launch_times_volume<double>(h->g64, (const double*)mu[ic], dd, dst, st)
                        : launch_times_volume<float>(h->g32, (const float*)mu[ic], dd, dst, st);
        if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: dL/dT0");
        if (!dev && (rc = copy_out(h, out, MR_F64, gT0, gT0_dtype, h->ncell, st))) return rc;
    }
    if (gU || gV || gW) {
        double* cU = out + h->ncell;
        double* cV = cU + h->ncU;
        double* cW = cV + h->ncV;
        double* aWc = a.scr;
        double* aVrow = a.scr + (size_t)(h->Nz + 1) * h->cfg.ny * h->cfg.nx;
        e = launch_refine_transpose(h->g64, fU, fV, fW, aWc, aVrow, cU, cV, cW, h->ncU, h->ncV, h->ncW, st);
        if (e != cudaSuccess) return cuda_check(e, "mr_adjoint_backward: refinement transpose");
        if (gU && (rc = copy_out(h, cU, MR_F64, gU, MR_F64, h->ncU, st))) return rc;
        if (gV && (rc = copy_out(h, cV, MR_F64, gV, MR_F64, h->ncV, st))) return rc;
        if (gW && (rc = copy_out(h, cW, MR_F64, gW, MR_F64, h->ncW, st))) return rc;
    }
    return cuda_check(cudaStreamSynchronize(st), "mr_adjoint_backward");
}

}  // extern "C"

// ---------------------------------------------------------------- diagnostics

extern "C" {

int mr_upscale_scalar(mr_handle h, double* Tc, mr_stream stream)
{
    if (!h || !Tc) return set_error(MR_ERR_ARG, "mr_upscale_scalar: NULL argument");
    if (!h->have_scalar) return set_error(MR_ERR_STATE, "mr_upscale_scalar: no scalar set");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    const size_t nc = (size_t)h->cfg.nx * h->nys * h->cfg.nz;
    const size_t need = nc + (size_t)h->Nz + 1 + (size_t)h->Nz;
    if (!b.diag) {
        cudaError_t e = dev_malloc((void**)&b.diag, need * sizeof(double));
        if (e != cudaSuccess) return cuda_check(e, "mr_upscale_scalar: buffer");
    }
    const bool dev = is_device_pointer(Tc);
    double* out = dev ? Tc : b.diag;
    cudaError_t e = h->cfg.precision == MR_F64 ? launch_upscale<double>(h->g64, (const double*)b.T[h->ic], out, st)
                                               : launch_upscale<float>(h->g32, (const float*)b.T[h->ic], out, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_upscale_scalar: launch");
    if (!dev) e = cudaMemcpyAsync(Tc, out, nc * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_check(e, "mr_upscale_scalar");
}

int mr_scalar_profiles(mr_handle h, double* nu_z, double* nu_T, mr_stream stream)
{
    if (!h || (!nu_z && !nu_T)) return set_error(MR_ERR_ARG, "mr_scalar_profiles: NULL argument");
    if (!h->have_scalar || !h->have_velocity)
        return set_error(MR_ERR_STATE, "mr_scalar_profiles: call mr_refine_velocity and mr_set_scalar first");
    cudaStream_t st = (cudaStream_t)stream;
    DeviceBuffers& b = h->buf;
    const size_t nc = (size_t)h->cfg.nx * h->nys * h->cfg.nz;
    if (h->slab) return set_error(MR_ERR_ARG, "mr_scalar_profiles: not on a y-slab handle");
    if (!b.diag) {
        cudaError_t e = dev_malloc((void**)&b.diag, (nc + 2 * (size_t)h->Nz + 1) * sizeof(double));
        if (e != cudaSuccess) return cuda_check(e, "mr_scalar_profiles: buffer");
    }
    double* dnu = b.diag + nc;
    double* dzc = dnu + h->Nz + 1;
    cudaError_t e = cudaMemcpyAsync(dzc, h->zc.data(), h->Nz * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_check(e, "mr_scalar_profiles: centres");
    // dense W of the refinement: stored, or refined into a temporary for the fused modes
    const void* ws = b.Ws;
    void *tu = nullptr, *tv = nullptr, *tw = nullptr;
    if (h->cfg.velocity_mode != MR_VEL_STORED) {
        e = dev_malloc(&tu, h->nU * h->elt);
        if (e == cudaSuccess) e = dev_malloc(&tv, h->nV * h->elt);
        if (e == cudaSuccess) e = dev_malloc(&tw, h->nW * h->elt);
        int rc = e != cudaSuccess ? cuda_check(e, "mr_scalar_profiles: temporary faces") : refine_into(h, tu, tv, tw, st);
        if (rc) { dev_free(tu); dev_free(tv); dev_free(tw); return rc; }
        ws = tw;
    }
    const double zb = h->zc[0] - h->zf[0], zt = h->zf[h->Nz] - h->zc[h->Nz - 1];
    e = h->cfg.precision == MR_F64
            ? launch_nu_profile<double>(h->g64, (const double*)b.T[h->ic], (const double*)ws, dzc, 1.0 / h->kappa, zb, zt,
                                        dnu, b.red, h->red_blocks, st)
            : launch_nu_profile<float>(h->g32, (const float*)b.T[h->ic], (const float*)ws, dzc, 1.0 / h->kappa, zb, zt,
                                       dnu, b.red, h->red_blocks, st);
    std::vector<double> p;
    int rc = e != cudaSuccess ? cuda_check(e, "mr_scalar_profiles: launch") : reduce_partials(h, 1, p, st);
    if (tu) { dev_free(tu); dev_free(tv); dev_free(tw); }
    if (rc) return rc;
    if (nu_T) {
        double s = 0.0, vt = 0.0;
        for (int q = 0; q < h->red_blocks; ++q) s += p[q];
        for (int k = 0; k < h->Nz; ++k) vt += h->dz[k];
        vt *= h->cfg.lx * h->cfg.ly;
        *nu_T = s / vt;
    }
    if (nu_z) {
        e = cudaMemcpy(nu_z, dnu, (h->Nz + 1) * sizeof(double), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_check(e, "mr_scalar_profiles: copy");
        for (int k = 0; k <= h->Nz; ++k) nu_z[k] /= (double)h->Nx * (double)h->Ny;
    }
    return MR_OK;
}

}  // extern "C"
