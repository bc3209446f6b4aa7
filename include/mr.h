/*
 * mr.h -- C-ABI of the GB300 (sm_103a) multiple-resolution scalar library.
 *
 * The library advances a scalar (temperature or concentration) on a dense
 * staggered grid whose velocity is held on an M-times coarser grid, following
 * Chong, Ding & Xia, "Multiple-resolution scheme in finite-volume code for
 * active or passive scalar turbulence" (arXiv:1805.03426):
 *   - Section 3.1: the dense grid is generated first (tanh clustering toward
 *     the plates in z, uniform in x and y); coarse faces are every M-th face.
 *   - Section 3.2: the coarse face velocity is refined onto the dense faces by
 *     the mass-conserving third-order interpolation R = A_s A^-1 and the
 *     stepwise flux balance of the inner faces (divergence-free to round-off).
 *   - Eq. (2)/(5): finite-volume advection-diffusion with second-order face
 *     values (or, opt-in, the fourth-order face values of Section 2.2),
 *     kappa = (Ra Pr)^-1/2 (or Sc in place of Pr for a passive scalar).
 *   - Section 2.2: Euler-leapfrog time integration with the averaging step
 *     every N_p steps; the first step after mr_set_scalar is forward Euler.
 *
 * Conventions shared by every call
 *   Arrays are [z][y][x] with x contiguous (row-major, no padding).
 *     dense cells   Nz x Ny x Nx            Nx = mx*nx, Ny = my*ny, Nz = mz*nz
 *     U faces       nz x ny x (nx + w)      x-normal; face i is the west face
 *     V faces       nz x (ny + w) x nx      y-normal; face j is the south face
 *     W faces       (nz + 1) x ny x nx      z-normal; planes 0 and nz are plates
 *   (dense face arrays likewise with Nx, Ny, Nz); w = 1 with MR_WALLS, 0 with
 *   MR_PERIODIC.  The domain is [0,lx] x [0,ly] x [0,1].
 *   Plates: T = +0.5 at z = 0 and -0.5 at z = 1 (MR_DIRICHLET) or zero flux.
 *   Every pointer may be host or device memory unless stated; the library
 *   detects which and copies on the given stream.  Device pointers must be
 *   on the handle's device.  The library keeps no caller pointer after a call.
 *   A stream argument of NULL means the legacy default stream.  Calls are
 *   asynchronous on the stream except where "synchronises" is stated.
 *   Return value: MR_OK (0) or a negative MR_ERR_* code; mr_last_error() then
 *   holds a message for the calling thread.
 */
#ifndef MR_H
#define MR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mr_handle_s* mr_handle;
typedef void* mr_stream; /* a cudaStream_t */

enum {
    MR_OK = 0,
    MR_ERR_ARG = -1,       /* invalid argument or configuration            */
    MR_ERR_CUDA = -2,      /* a CUDA runtime call or kernel launch failed  */
    MR_ERR_NONFINITE = -3, /* a reduction met NaN or Inf                   */
    MR_ERR_TIMEOUT = -4,   /* a bounded device wait gave up                */
    MR_ERR_OOM = -5,       /* device allocation failed                     */
    MR_ERR_STATE = -6      /* call out of order (e.g. step before set)     */
};
enum { MR_F64 = 0, MR_F32 = 1 };               /* precision / buffer dtype */
enum { MR_VEL_STORED = 0, MR_VEL_FUSED = 1, MR_VEL_XFUSED = 2 };  /* dense velocity handling */
enum { MR_DIRICHLET = 0, MR_ADIABATIC = 1 };   /* plates                   */
enum { MR_PERIODIC = 0, MR_WALLS = 1 };        /* x and y boundaries       */

/* Problem statement (Sections 2.1, 3.1).  Fill with mr_config_default first. */
typedef struct {
    uint32_t struct_size;     /* sizeof(mr_config): ABI version check         */
    int32_t nx, ny, nz;       /* coarse cells (>= 3 along any refined axis)   */
    int32_t mx, my, mz;       /* refinement factors M_x, M_y, M_z (1..8)      */
    double lx, ly;            /* horizontal extent; height is 1               */
    double stretch_gamma;     /* 0: uniform z; > 0: tanh clustering of the
                                 dense z faces, z_k = (1 + tanh(g(2k/Nz-1))/tanh g)/2 */
    double ra, pr_or_sc;      /* kappa = (ra * pr_or_sc)^-1/2                  */
    double dt;                /* time step (see mr_cfl_dt / mr_set_dt)        */
    int32_t precision;        /* MR_F64: FP64 storage and flux arithmetic;
                                 MR_F32: FP32 storage and flux arithmetic.
                                 Reductions are FP64 in both.                 */
    int32_t velocity_mode;    /* MR_VEL_STORED: dense faces kept in HBM;
                                 MR_VEL_FUSED: every stage of the refinement
                                 inside the step kernel, from the coarse faces;
                                 MR_VEL_XFUSED: the z- and y-stages are kept at
                                 coarse resolution in x (1/mx of the dense face
                                 count, computed by mr_refine_velocity) and the
                                 x-stage runs inside the step kernel.  In both
                                 fused modes the dense faces are never stored
                                 (MR_F32, MR_PERIODIC, mx=my=mz in {2,4},
                                 Nx % 64 == 0, Ny % 16 == 0).                 */
    int32_t np_average;       /* N_p of the averaging step (Section 2.2);
                                 <= 0 disables it; default 50                 */
    int32_t bc_plates;        /* MR_DIRICHLET | MR_ADIABATIC                  */
    int32_t bc_horizontal;    /* MR_PERIODIC | MR_WALLS (impermeable, adiabatic) */
    int32_t diffz_implicit;   /* 0: explicit (the paper's scheme); 1: opt-in
                                 Crank-Nicolson for vertical diffusion with one
                                 tridiagonal solve per (x, y) column           */
    int32_t face_order;       /* face values of the advected scalar: 2 (linear
                                 between centres, default) or 4 (Section 2.2:
                                 the cubic with the four nearest cell averages
                                 along the face normal, evaluated at the face;
                                 the three domain-side cells next to a wall).
                                 Diffusive fluxes are two-point in both.  4 is
                                 supported by MR_VEL_STORED and MR_VEL_XFUSED,
                                 not by the adjoint; it needs >= 4 dense cells
                                 on periodic axes and >= 3 between walls.     */
    int32_t slab_j0, slab_ny; /* y-slab decomposition over GPUs (the data
                                 partition of the paper's parallel solver,
                                 Section 2.4, in slabs of whole coarse rows):
                                 slab_ny = 0 (default) gives the whole domain;
                                 otherwise the handle owns coarse rows
                                 slab_j0 .. slab_j0 + slab_ny - 1 of the
                                 periodic domain of ny coarse rows (ly is the
                                 whole domain's): its scalar arrays hold the
                                 slab's slab_ny * my dense rows, the coarse
                                 velocity it takes is the whole domain's, and
                                 the dense rows just outside the slab come
                                 from mr_set_halo_rows instead of the periodic
                                 wrap.  MR_VEL_FUSED only; slab_ny * my % 16
                                 == 0; one step per mr_scalar_step call; the
                                 reductions cover the slab (the caller sums
                                 over slabs).                                 */
} mr_config;

typedef struct {
    double nu_bot;    /* <(0.5 - T(z_c0)) / z_c0>_xy: bottom-plate Nusselt number  */
    double nu_top;    /* <(T(z_cN-1) + 0.5) / (1 - z_cN-1)>_xy: top-plate Nusselt  */
    double mean;      /* volume-weighted mean of T                                 */
    double var;       /* volume-weighted variance of T (two-pass)                  */
    double integral;  /* sum of T * cell volume                                    */
    double max_div;   /* max over dense cells of |sum of outward face fluxes|/volume
                         of the refined velocity (Section 3.2 divergence check)   */
} mr_stats;

/* Fill *cfg with defaults: 16^3 coarse, M = 2, uniform, Ra = 1e6, Pr = 7,
 * dt = 1e-3, MR_F64, MR_VEL_STORED, N_p = 50, Dirichlet plates, periodic. */
int mr_config_default(mr_config* cfg);

/* Validate *cfg, build the grid and R matrices (Section 3.2: R depends on the
 * grid only and is computed once), and allocate every device buffer on the
 * current CUDA device.  *out receives the handle; mr_destroy frees it.
 * Errors: MR_ERR_ARG (bad sizes, unsupported combination), MR_ERR_OOM. */
int mr_create(const mr_config* cfg, mr_handle* out);

/* Free every buffer of the handle (synchronises the device first).  NULL is ignored. */
void mr_destroy(mr_handle h);

/* Message of the last failed call on this thread ("" if none). */
const char* mr_last_error(void);

/* Dense sizes and the dense z-face coordinates (host array of Nz + 1 doubles,
 * may be NULL).  dims3 (may be NULL) receives Nx, Ny, Nz. */
int mr_grid(mr_handle h, int32_t* dims3, double* zf_host);

/* Refinement, Section 3.2.  U, V, W: coarse face velocities in FP64 (host or
 * device).  The handle keeps its own copy.  In MR_VEL_STORED mode the dense
 * faces are computed now and kept; Us, Vs, Ws (device, handle precision, may
 * be NULL) receive a copy of them.  In MR_VEL_FUSED mode the step kernel
 * refines on the fly; non-NULL Us, Vs, Ws are still filled for inspection.
 * The coarse field must be discretely divergence-free and zero on the plates;
 * the library does not check this (mr_scalar_stats reports max_div). */
int mr_refine_velocity(mr_handle h, const double* U, const double* V, const double* W,
                       void* Us, void* Vs, void* Ws, mr_stream stream);

/* The refinement of mr_refine_velocity split in two, so that the hand-over of
 * the next coarse velocity overlaps the current steps (the paper has no such
 * call: it is the pipelining of the host-to-device copy).
 * mr_stage_velocity copies U, V, W (FP64, host or device, the layout of
 * mr_refine_velocity) into one of two device slots owned by the handle, on
 * copy_stream, and returns at once; the caller must not change U, V, W until
 * copy_stream has passed the copy (pinned host memory keeps it asynchronous).
 * A second call before a refinement replaces the staged faces.
 * mr_refine_velocity_staged refines the last staged faces on stream (which
 * waits for their copy): the same result as mr_refine_velocity with them.
 * A slot is reused only after the work queued on the refining stream before
 * its release has run.  Errors: MR_ERR_ARG (NULL), MR_ERR_STATE (nothing
 * staged), MR_ERR_CUDA, MR_ERR_OOM (slots are allocated at the first call). */
int mr_stage_velocity(mr_handle h, const double* U, const double* V, const double* W,
                      mr_stream copy_stream);
int mr_refine_velocity_staged(mr_handle h, mr_stream stream);

/* Copy the scalar in (dtype MR_F64 or MR_F32, host or device) and restart the
 * time integration: the next step is the forward-Euler start. */
int mr_set_scalar(mr_handle h, const void* T0, int32_t dtype, mr_stream stream);

/* Copy T^n (and T^{n-1} if Tprev != NULL) out, converted to dtype. */
int mr_get_scalar(mr_handle h, void* T, void* Tprev, int32_t dtype, mr_stream stream);

/* Advance nsteps time steps (Section 2.2, Eq. 5): one fused kernel launch per
 * step.  Needs mr_refine_velocity and mr_set_scalar first (MR_ERR_STATE). */
int mr_scalar_step(mr_handle h, int64_t nsteps, mr_stream stream);

/* One time step (as mr_scalar_step) followed by what a coupled coarse solver
 * takes back every step: the plate Nusselt numbers of the new T^n into nu2
 * (2 doubles, bottom then top, Section 4.1) and the volume-weighted average of
 * T^n over every coarse cell into Tc (nz x ny x nx doubles, [z][y][x]; a
 * y-slab handle: its slab's coarse rows), the upscale integration of Section
 * 3.3.  Either may be NULL.  Each must be device memory or pinned host memory,
 * which the kernels write directly (MR_ERR_ARG for pageable host memory).
 * Asynchronous on stream; the other rules are mr_scalar_step's. */
int mr_scalar_step_coupled(mr_handle h, double* nu2, double* Tc, mr_stream stream);

/* One coarse time step with temporal refinement (Section 3.4, Eq. 18): the
 * velocity set by mr_refine_velocity (or by the previous call) is U^{n-1};
 * U, V, W (FP64, host or device, coarse layout as in mr_refine_velocity) are
 * U^n.  Refines U^n, then advances mt >= 1 scalar steps, step i = 0..mt-1
 * using the velocity U^{n-1} + (i/mt)(U^n - U^{n-1}) (a convex combination of
 * two divergence-free fields, so divergence-free), with the handle's dt as the
 * dense step (the coarse step being mt dt).  On return U^n is the current
 * velocity.  The step count and the leapfrog state carry over.  The first
 * call allocates a second velocity level (MR_ERR_OOM/MR_ERR_CUDA if that
 * fails).  MR_ERR_ARG on NULL or mt < 1; MR_ERR_STATE before mr_refine_velocity
 * and mr_set_scalar.  Asynchronous on stream. */
int mr_scalar_coarse_step(mr_handle h, const double* U, const double* V, const double* W, int32_t mt,
                          mr_stream stream);

/* Number of steps taken since the last mr_set_scalar. */
int mr_step_index(mr_handle h, int64_t* s);

/* FP64 reductions of T^n and the refined velocity (Section 4.1 plate Nusselt
 * numbers, volume moments, divergence check).  Synchronises the stream.
 * Returns MR_ERR_NONFINITE (and still fills *out) if T holds NaN or Inf. */
int mr_scalar_stats(mr_handle h, mr_stats* out, mr_stream stream);

/* Plate Nusselt numbers only (nu2[0] bottom, nu2[1] top; host or device
 * pointer to 2 doubles).  Asynchronous; a cheap reduction over two planes. */
int mr_plate_nu(mr_handle h, double* nu2, mr_stream stream);

/* dt = cfl / max over dense cells of (max(|u_w|,|u_e|)/dx + max(|v_s|,|v_n|)/dy
 * + max(|w_b|,|w_t|)/dz) on the refined velocity.  Synchronises.  Does not
 * change the handle's dt (use mr_set_dt). */
int mr_cfl_dt(mr_handle h, double cfl, double* dt_out, mr_stream stream);

/* Replace the time step. */
int mr_set_dt(mr_handle h, double dt);

/* Upscale integration (Section 3.3): Tc (nz x ny x nx doubles, host or
 * device) receives the volume-weighted average of T^n over every coarse cell,
 * the value the coarse momentum solver of a coupled run consumes.  Synchronises. */
int mr_upscale_scalar(mr_handle h, double* Tc, mr_stream stream);

/* Heat-flux diagnostics (Section 4.1).  nu_z (host, Nz + 1 doubles, may be
 * NULL): the plane average of Nu(z) = (Ra Pr)^1/2 w T - dT/dz on every dense
 * z-face, with the face value and gradient of the step's discretisation (at the
 * plates the conductive flux alone).  nu_T (host, may be NULL): Nu_T =
 * eps_T (Ra Pr)^1/2 = <|grad T|^2>, the volume average of the squared face
 * gradients weighted by each face's dual volume, plates at their Dirichlet
 * values.  FP64; synchronises.  Fused modes refine into temporary dense faces. */
int mr_scalar_profiles(mr_handle h, double* nu_z, double* nu_T, mr_stream stream);

/* Gradients (hand-written discrete adjoint of the scheme above).
 * mr_adjoint_forward runs nsteps steps from the scalar just set by
 * mr_set_scalar (MR_ERR_STATE otherwise), storing the pair (T^{s-1}, T^s)
 * every checkpoint_every steps in library memory, and returns
 *   L = sum_{s=0..nsteps} wnu[s] Nu_bot(T^s) + wvar[s] Var(T^s)
 * (wnu, wvar: host arrays of nsteps + 1 doubles; either may be NULL = 0).
 * mr_adjoint_backward then recomputes each segment from its checkpoint,
 * sweeps the adjoint back to s = 0 and writes gscale * dL/dT^0 (dense, dtype
 * MR_F64 or MR_F32) and gscale * dL/dU, dL/dV, dL/dW (coarse, FP64, through
 * the transpose of the refinement of Section 3.2); any output may be NULL.
 * Pointers may be host or device.  Both synchronise.  Needs MR_VEL_STORED,
 * explicit diffusion and face_order 2 (MR_ERR_ARG otherwise).  The time step is not
 * differentiated.  After the backward the handle holds T^nsteps. */
int mr_adjoint_forward(mr_handle h, int64_t nsteps, int32_t checkpoint_every, const double* wnu,
                       const double* wvar, double* loss, mr_stream stream);
int mr_adjoint_backward(mr_handle h, double gscale, void* gT0, int32_t gT0_dtype, double* gU, double* gV,
                        double* gW, mr_stream stream);

/* Allocation-free refinement.  The paper has no counterpart: this is an
 * interface for callers that cannot allocate device memory, e.g. code running
 * inside a framework whose caching allocator owns the whole device, or a
 * plug-in forbidden to call cudaMalloc.  It computes the same dense faces as
 * mr_refine_velocity (FP64 in, FP64 out) from *cfg alone -- no handle -- using
 * only a file-scope device scratch array of 32 MiB that every GPU loading this
 * library holds until the process exits; it allocates nothing.  Its grid and R
 * matrices are rebuilt into that array at every call.  Sizes whose grid, R
 * matrices and work arrays exceed the 32 MiB give MR_ERR_ARG with the needed
 * size in mr_last_error(), and so does a stretching that collapses the dense
 * z-layers at the plates (width <= 1e-12).  U, V, W, Us, Vs, Ws must be device
 * memory (MR_ERR_ARG otherwise); cfg's precision, velocity_mode, Ra, Pr, dt
 * and plate settings are ignored.  The first call on a device looks the
 * array's device address up (cudaGetSymbolAddress, with that device current),
 * so make that first call before any stream capture.  Each device has its own
 * copy of the array, shared by every call on that device: calls that overlap
 * on the same device (on any streams) race and corrupt each other's results;
 * calls on different devices do not interact. */
int mr_refine_velocity_noalloc(const mr_config* cfg, const double* U, const double* V, const double* W,
                               double* Us, double* Vs, double* Ws, mr_stream stream);

/* Halo exchange of a y-slab handle (mr_config.slab_ny > 0): the paper's
 * parallel solver swaps ghost layers between subdomains every step (Section
 * 2.4); here a slab needs one dense row of T^n and of T^{n-1} beyond each of
 * its two y edges.  mr_get_boundary_rows copies the slab's first (south) and
 * last (north) dense rows of T^n, each as [Nz][Nx] values in the handle's
 * precision (host or device pointers, either may be NULL); they are the
 * north halo of the southern neighbour and the south halo of the northern
 * one.  mr_set_halo_rows gives T^n its halo rows: below (the row south of row
 * 0, i.e. the southern neighbour's last row) and above (the row north of the
 * last row, the northern neighbour's first), [Nz][Nx] each, copied in.  The
 * halo rows of T^n become those of T^{n-1} at the next step, so after
 * mr_set_scalar and after every step the caller exchanges and sets them once;
 * mr_scalar_step returns MR_ERR_STATE if they are missing.  Asynchronous on
 * stream.  MR_ERR_ARG on a whole-domain handle or NULL arguments. */
int mr_get_boundary_rows(mr_handle h, void* south, void* north, mr_stream stream);
int mr_set_halo_rows(mr_handle h, const void* below, const void* above, mr_stream stream);

/* Measurement aid (no counterpart in the paper): the FP64 arithmetic rate of
 * the current device in TFLOP/s (an FMA counts two), from a kernel of
 * independent FMA chains in registers timed with CUDA events on stream (best
 * of three launches after one untimed).  The FP64 stored-velocity step is
 * bound by this rate rather than by HBM.  Synchronises.  Errors: MR_ERR_ARG
 * (NULL), MR_ERR_CUDA. */
int mr_fp64_fma_rate(double* tflops, mr_stream stream);

/* Test hooks of the failure paths (no counterpart in the paper; neither
 * faults the GPU).
 * mr_debug_inject_wait_timeout arms a one-shot injection: in the next launch
 * of a TMA-fed step kernel (MR_VEL_XFUSED or MR_VEL_FUSED), every bounded
 * wait gives up after wait_seconds (0 < wait_seconds <= 1, instead of 1 s), and
 * the producer warp of the first CTA issues none of its ring loads from ring
 * stop_ring on.  Every load it did issue is still waited for, so nothing is
 * in flight when the CTA exits; the consumers' wait for ring stop_ring runs
 * out and the launch records MR_ERR_TIMEOUT, which the next synchronising
 * call on a handle in a fused mode returns.  The scalar that launch wrote is
 * then invalid (restart with mr_set_scalar).
 * mr_debug_alloc_cap caps the bytes of device memory the library may hold
 * (cap_bytes >= 0; -1 removes the cap; -2 leaves it unchanged); a refused
 * allocation fails like an exhausted device (MR_ERR_OOM).  live_bytes (may be
 * NULL) receives the bytes the library holds now.  Process-wide, thread-safe. */
int mr_debug_inject_wait_timeout(int32_t stop_ring, double wait_seconds);
int mr_debug_alloc_cap(int64_t cap_bytes, int64_t* live_bytes);

/* Integer index maps for testing (synchronous, host buffer): coarse cell of
 * every dense cell along x, y, z, then the three coarse cells of the R window
 * of every coarse cell along x, y, z: Nx+Ny+Nz+3(nx+ny+nz) int32 values.
 * MR_ERR_ARG if cap (in elements) is too small. */
int mr_debug_index_maps(mr_handle h, int32_t* out, size_t cap);

#ifdef __cplusplus
}
#endif
#endif /* MR_H */
