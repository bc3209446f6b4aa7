// Internal declarations of the multiple-resolution scalar library (sm_103a).
// The public boundary is include/mr.h; everything here is private.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mr.h"

namespace mr {

constexpr int kPlateBlocks = 304;  // blocks of the plate Nusselt reduction

// Device view of the grid and of the per-layer coefficients, in precision P.
// Built once per handle from the FP64 host grid (Sections 3.1, 3.2).
template <typename P>
struct Grid {
    int nx, ny, nz, mx, my, mz;  // coarse cells, refinement factors
    int Nx, Ny, Nz;              // dense cells
    int walls;                   // 1: impermeable adiabatic side walls
    int ufx, vfy;                // dense U row length (Nx+w), V rows (Ny+w)
    int cux, cvy;                // coarse U row length, V rows
    int dirichlet;               // plates: 1 Dirichlet (+-0.5), 0 adiabatic
    P dx, dy, DX, DY;
    P inv_dx, inv_dy;            // A_x / Vol and A_y / Vol
    P kx2, ky2;                  // kappa / dx^2, kappa / dy^2
    const P* dz;                 // [Nz] dense layer widths
    const P* inv_dz;             // [Nz] A_z / Vol
    const P* wlo;                // [Nz+1] weight of T_{k-1} at z-face k (linear interpolation)
    const P* whi;                // [Nz+1] weight of T_k at z-face k
    const P* cdn;                // [Nz] kappa / (dz_k * distance to the centre or plate below)
    const P* cup;                // [Nz] kappa / (dz_k * distance to the centre or plate above)
    const P* Rx;                 // [Nx][3] R row of every dense x index (Section 3.2)
    const P* Ry;                 // [Ny][3]
    const P* Rz;                 // [Nz][3]
    const int* wx;               // [nx][3] coarse cells of the R window
    const int* wy;               // [ny][3]
    const int* wz;               // [nz][3]
    const P* f4x;                // [Nx+1][4] fourth-order face weights of cells f-2..f+1
    const P* f4y;                // [Ny+1][4]
    const P* f4z;                // [Nz+1][4]
    int order4;                  // 1: fourth-order face values of the advected scalar
    P hx, hy;                    // 1 / (2 dx), 1 / (2 dy)
    // [Nz][8] per-layer constants of the periodic second-order step: the
    // weights of T_{k-1}, T_k at z-face k times 1/dz_k, the negated weights of
    // T_k, T_{k+1} at z-face k+1 times 1/dz_k, cdn, cup, the negated diagonal
    // 2 kx2 + 2 ky2 + cdn + cup, and the plate term (cdn T_bottom on the first
    // layer, cup T_top on the last, Dirichlet plates)
    const P* lz;
};

// Coefficients of one step: T^{s+1} = a T^{s-1} + b T^s + gdt [C(T^s) + D(T^{s-1})].
struct StepCoef {
    double a, b, gdt;
};

struct DeviceBuffers {
    void* T[3] = {nullptr, nullptr, nullptr};  // rotating scalar levels, precision P
    double* U64 = nullptr;                     // coarse faces, FP64 copy
    double* V64 = nullptr;
    double* W64 = nullptr;
    void* Uc = nullptr;                        // coarse faces in precision P (alias of *64 for FP64)
    void* Vc = nullptr;
    void* Wc = nullptr;
    void* Us = nullptr;                        // dense faces (MR_VEL_STORED)
    void* Vs = nullptr;
    void* Ws = nullptr;
    void* scrW = nullptr;                      // refinement scratch: full-coarse-area W per dense plane
    void* scrV = nullptr;                      // refinement scratch: full-coarse-width V per dense row
    void* metric = nullptr;                    // one block holding every Grid array
    double* red = nullptr;                     // reduction partials
    double* nu2 = nullptr;                     // plate Nusselt numbers (2 doubles + partials)
    void* stage = nullptr;                     // conversion staging buffer
    void* tri = nullptr;                       // implicit-z work (2 * Nz per column)
    // MR_VEL_XFUSED: coarse-x intermediates of the z- and y-stages (FP32,
    // nxg = nx + 8 columns with 4 periodic ghosts each side) and layer constants
    float* xwy = nullptr;                      // [Nz+1][Ny][nxg]
    float* xuo = nullptr;                      // [Nz][Ny][nxg]
    float* xvr = nullptr;                      // [Nz][Ny+1][nxg]
    float* xlc = nullptr;                      // [Nz][32] layer constants of the fused steps
    float xrx[12] = {0};                       // R_x rows of the 4 cells of a 4-cell segment
    float xry[12] = {0};                       // R_y rows of dense rows 0..3 (MR_VEL_FUSED)
    float* cpad = nullptr;                     // MR_VEL_FUSED: padded FP32 coarse faces
    float* fsc = nullptr;                      // MR_VEL_FUSED: [nz][32] slab constants
    float* halo = nullptr;                     // y-slab: [3 levels][below, above][Nz][Nx] halo rows
    double* tcinv = nullptr;                   // MR_VEL_FUSED: 1 / (mx my sum of each slab's dz) (lazy)
    double* nup = nullptr;                     // MR_VEL_FUSED: work of the plate-Nu launch (lazy)
    float xw4[8] = {0};                        // fourth order: twice the x and y face weights (uniform)
    int xlcw = 12;                             // row length of xlc
    double* diag = nullptr;                    // diagnostics: coarse T, Nu(z), dense z centres (lazy)
    int nxg = 0;
    // Temporal refinement (Section 3.4): the velocity of the next coarse time
    // level, in the same layout as the current one above (allocated by the
    // first mr_scalar_coarse_step; swapped with the current level after it).
    struct Level {
        double *U64 = nullptr, *V64 = nullptr, *W64 = nullptr;
        void *Uc = nullptr, *Vc = nullptr, *Wc = nullptr;
        void *Us = nullptr, *Vs = nullptr, *Ws = nullptr;
        float *xwy = nullptr, *xuo = nullptr, *xvr = nullptr;
        float* cpad = nullptr;
    } next;
    float* lerpc = nullptr;                    // MR_VEL_FUSED: interpolated padded coarse faces
    // staged coarse faces (mr_stage_velocity): two FP64 slots; a refinement
    // swaps the slot with U64/V64/W64 instead of copying it
    double *sU[2] = {nullptr, nullptr}, *sV[2] = {nullptr, nullptr}, *sW[2] = {nullptr, nullptr};
    cudaEvent_t stg_copied[2] = {nullptr, nullptr};   // on the copy stream: the slot's copy is done
    cudaEvent_t stg_free[2] = {nullptr, nullptr};     // on the compute stream: the slot's memory is free
    int stg_next = 0;                                 // slot the next mr_stage_velocity fills
    int stg_ready = -1;                               // slot holding staged faces not yet refined
};

}  // namespace mr

struct mr_handle_s {
    mr_config cfg;
    int device = 0;
    int Nx = 0, Ny = 0, Nz = 0, w = 0;
    // stored dense and coarse rows: the whole domain's Ny, ny, or a y-slab's
    int Nys = 0, nys = 0;
    bool slab = false;
    bool halo_set[3] = {false, false, false};   // y-slab: halo rows given for each scalar level
    size_t ncell = 0, nU = 0, nV = 0, nW = 0, ncU = 0, ncV = 0, ncW = 0;
    size_t elt = 8;          // bytes per element of precision P
    double kappa = 0.0;
    int64_t step = 0;        // steps taken since mr_set_scalar
    int ip = 0, ic = 1;      // indices of T^{n-1}, T^n in buf.T
    bool have_velocity = false, have_scalar = false;
    // maximum divergence of the current refined velocity, computed by the
    // first mr_scalar_stats after the velocity changed
    bool maxdiv_valid = false;
    double maxdiv = 0.0;
    // host FP64 grid (Section 3.1) and R matrices (Section 3.2)
    std::vector<double> zf, zc, dz, Rx, Ry, Rz;
    std::vector<double> f4x, f4y, f4z;   // fourth-order face weights (zeros at face_order 2)
    std::vector<int> wx, wy, wz;
    mr::DeviceBuffers buf;
    mr::Grid<double> g64;
    mr::Grid<float> g32;
    size_t stage_bytes = 0;
    int red_blocks = 0;
    // adjoint state between mr_adjoint_forward and mr_adjoint_backward
    struct Adjoint {
        bool ready = false;
        int64_t S = 0;
        int ck = 0;
        std::vector<double> wnu, wvar, mean;   // weights and FP64 means of every level (s = 0..S)
        void* cp = nullptr;                    // checkpoints: pairs (T^{s-1}, T^s) every ck steps
        size_t cp_pairs = 0;
        void* seg = nullptr;                   // recomputed levels of one segment (ck + 1)
        void* mu = nullptr;                    // three adjoint levels
        double* face = nullptr;                // dense face gradients (U, V, W), FP64
        float* face32 = nullptr;               // MR_F32: per-segment FP32 sums, flushed into face
        double* scr = nullptr;                 // transpose scratch (full-area W, full-width V), FP64
        double* out = nullptr;                 // FP64 staging of the outputs (dense T0, coarse U, V, W)
    } adj;
};

namespace mr {

int set_error(int code, const std::string& msg);
int cuda_check(cudaError_t e, const char* what);
bool is_device_pointer(const void* p);
StepCoef step_coef(const mr_config& cfg, int64_t s);

// launchers (return cudaError_t of the launch)
template <typename P>
cudaError_t launch_refine(const Grid<P>& g, const P* U, const P* V, const P* W, P* Us, P* Vs, P* Ws,
                          P* scrW, P* scrV, cudaStream_t st);
template <typename P>
cudaError_t launch_step_stored(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, const P* Tm1,
                               const P* T, P* Tp1, StepCoef c, bool implz, cudaStream_t st);
// the same step with the velocity A + alpha (B - A) of two stored dense fields
template <typename P>
cudaError_t launch_step_stored_lerp(const Grid<P>& g, const P* const velA[3], const P* const velB[3], double alpha,
                                    const P* Tm1, const P* T, P* Tp1, StepCoef c, bool implz, cudaStream_t st);
// out = A + alpha (B - A), elementwise (coarse faces of two time levels)
cudaError_t launch_lerp_f32(const float* A, const float* B, double alpha, float* out, size_t n, cudaStream_t st);
template <typename P>
cudaError_t launch_zsolve(const Grid<P>& g, P* Tp1, double half_gdt, P* work, cudaStream_t st);
template <typename P>
cudaError_t launch_convert(const void* src, int src_dtype, void* dst, int dst_dtype, size_t n,
                           cudaStream_t st);
template <typename P>
cudaError_t launch_moments(const Grid<P>& g, const P* T, double mean, int pass, double* partials,
                           int blocks, cudaStream_t st);
template <typename P>
cudaError_t launch_plate_nu(const Grid<P>& g, const P* T, const double* zb_zt, double* out2,
                            cudaStream_t st);
template <typename P>
cudaError_t launch_maxdiv(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, double* partials,
                          int blocks, cudaStream_t st);
template <typename P>
cudaError_t launch_upscale(const Grid<P>& g, const P* T, double* Tc, cudaStream_t st);
template <typename P>
cudaError_t launch_nu_profile(const Grid<P>& g, const P* T, const P* Ws, const double* zc, double inv_kappa, double zb,
                              double zt, double* nu_z, double* partials, int blocks, cudaStream_t st);
template <typename P>
cudaError_t launch_cfl(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, double* partials,
                       int blocks, cudaStream_t st);
bool fused_supported(const mr_config& cfg, std::string* why);
// FP64 values from mapped pinned host memory into an FP64 device array and,
// where d32 is given, an FP32 one (16-byte aligned src and d64, 8-byte d32).
cudaError_t launch_fetch_f64(const double* src, double* d64, float* d32, size_t n, cudaStream_t st);
// MR_VEL_FUSED: what the fused step kernel reads besides the scalar levels
struct FusedInputs {
    const float* pad;    // coarse U, V, W padded with their periodic images (launch_fused_pad)
    // the dense rows south of row 0 and north of row Ny-1 of T^s and T^{s-1}
    // (hs, hn), element (k, i) at k * hstride + i: the periodic images on a
    // whole-domain grid, the halo rows of a y-slab
    const float* hs[2];
    const float* hn[2];
    size_t hstride;
    const float* sc;     // [nz][32] slab constants (fused_slab_constants)
    const float* lc;     // [Nz][32] layer constants (xfused_layer_constants)
    const float* rx12;   // R_x rows of the 4 cells of a 4-cell segment (uniform, periodic x)
    const float* ry12;   // R_y rows of dense rows 0..3 (uniform, periodic y)
    // NULL, or where the step writes the upscaled coarse scalar of the new level
    // ([nz][ny][nx], FP64, device or mapped host memory); then tcinv[K] = 1 / (mx my
    // sum of slab K's dz)
    double* Tc;
    const double* tcinv;
};
// every refinement stage in the step kernel
cudaError_t launch_step_fused_f32(const Grid<float>& g, const FusedInputs& in, const float* Tm1, const float* T,
                                  float* Tp1, StepCoef c, cudaStream_t st);
// kind 1: max |divergence| of the dense velocity, kind 2: max CFL rate (into partials[0])
cudaError_t launch_fused_max_f32(const Grid<float>& g, int kind, const FusedInputs& in, double* partials, int blocks,
                                 cudaStream_t st);
// The plate Nusselt numbers of the level T (nu2[0] bottom, nu2[1] top) in one launch;
// izb, izt the inverse plate-to-centre distances; work: fused_plate_nu_work() doubles,
// the first one zero before the first launch (each launch leaves it zero).
cudaError_t launch_fused_plate_nu(const Grid<float>& g, const float* T, double izb, double izt, double* work,
                                  double* nu2, cudaStream_t st);
size_t fused_plate_nu_work();
// floats of the padded coarse faces, and the kernel that forms them from the FP32 coarse faces
size_t fused_pad_floats(int nx, int ny, int nz);
// (the coarse rows j0-1 .. j0+ny+1 of a domain of nyg rows, periodic)
cudaError_t launch_fused_pad(const float* U, const float* V, const float* W, float* out, int nx, int nyg, int nz,
                             int j0, int ny, cudaStream_t st);
// the same from the FP64 coarse faces, also writing the FP32 faces on a whole-domain grid
cudaError_t launch_fused_pad64(const double* U, const double* V, const double* W, float* out, float* U32, float* V32,
                               float* W32, int nx, int nyg, int nz, int j0, int ny, cudaStream_t st);
// per coarse slab: R_z rows, 1/(2 dz) and the stage-Z weights, [nz][32]
std::vector<float> fused_slab_constants(int nz, int M, const double* Rz, const double* dz);
int* fused_error_flag();
// per-layer constant table [Nz][32] of the split-x and fully fused kernels
// (layout owned by mr_xfused.cu)
std::vector<float> xfused_layer_constants(int Nz, const double* zf, const double* zc, const double* dz, double kappa,
                                          double dx, double dy, bool dirichlet, const double* f4z, int* lcw);
// Raise a kernel's dynamic shared-memory limit once per device (*done: one bit per device).
cudaError_t smem_optin(const void* kernel, int bytes, unsigned long long* done);
template <typename P>
cudaError_t launch_column_balance(const Grid<P>& g, const P* U, const P* V, const P* W, P* scrW, cudaStream_t st);
cudaError_t launch_xfused_prep(const Grid<float>& g, const float* U, const float* V, const float* W, float* scrW,
                               float* WY, float* UO, float* VR, int nxg, cudaStream_t st);
// setA = {WY, UO, VR} of the current velocity; setB (or NULL) those of the next
// coarse time level, interpolated with weight alpha (temporal refinement)
cudaError_t launch_step_xfused_f32(const Grid<float>& g, const float* const setA[3], const float* const setB[3],
                                   double alpha, int nxg, const float* lc, int lcw, const float* rx12, const float* w4,
                                   const float* Tm1, const float* T, float* Tp1, StepCoef c, cudaStream_t st);
// kind 1: max |divergence| of the dense velocity, kind 2: max CFL rate (into partials[0])
cudaError_t launch_xfused_max_f32(const Grid<float>& g, int kind, const float* WY, const float* UO, const float* VR,
                                  int nxg, const float* lc, int lcw, const float* rx12, double* partials, int blocks,
                                  cudaStream_t st);
cudaError_t launch_refine_transpose(const Grid<double>& g, double* aUs, double* aVs, double* aWs, double* aWc,
                                    double* aVrow, double* gU, double* gV, double* gW, size_t ncU, size_t ncV,
                                    size_t ncW, cudaStream_t st);
template <typename P>
cudaError_t launch_adj_step(const Grid<P>& g, const P* Us, const P* Vs, const P* Ws, const P* T, const P* Tprev,
                            const P* Mn, P* Mc, P* Mp, double s_nu, double s_var, double mean_prev, P* gU,
                            P* gV, P* gW, StepCoef c, bool euler, cudaStream_t st);
cudaError_t launch_flush_faces(float* seg, double* tot, size_t n, cudaStream_t st);
template <typename P>
cudaError_t launch_adj_direct(const Grid<P>& g, const P* T, double s_nu_bottom, double s_var, double mean, P* mu,
                              cudaStream_t st);
template <typename P>
cudaError_t launch_times_volume(const Grid<P>& g, const P* mu, int dst_dtype, void* out, cudaStream_t st);
int fused_take_error(cudaStream_t st);   // MR_ERR_TIMEOUT if a fused kernel gave up a wait
// Test hook (mr_debug_inject_wait_timeout): if armed, hand the next TMA step
// launch its stop ring and wait limit, and disarm; else leave both unchanged.
void take_wait_injection(int* stop_ring, unsigned long long* wait_ns);
// Device allocations of the library, counted so that a test can cap them
// (mr_debug_alloc_cap) and check that a failed call leaks nothing.
cudaError_t dev_malloc(void** p, size_t bytes);
template <typename T>
cudaError_t dev_malloc(T** p, size_t bytes)
{
    return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
cudaError_t dev_free(void* p);

}  // namespace mr
