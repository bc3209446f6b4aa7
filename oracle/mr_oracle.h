/*
 * Plain FP64 CPU oracle for the multiple-resolution scalar path of
 * Chong, Ding & Xia, "Multiple-resolution scheme in finite-volume code for
 * active or passive scalar turbulence" (arXiv:1805.03426).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA library under paper_1805_03426_gb300/csrc.
 *
 * Layout of every 3-D array: [z][y][x], x contiguous.
 *   dense cells       Nz x Ny x Nx           (Nx = mx*nx, ...)
 *   U faces (x-normal) Nz x Ny x (Nx + w)    w = 1 with side walls, 0 periodic
 *   V faces (y-normal) Nz x (Ny + w) x Nx
 *   W faces (z-normal) (Nz + 1) x Ny x Nx    planes 0 and Nz are the plates
 * Coarse arrays use the same layout with nx, ny, nz.
 */
#ifndef MR_ORACLE_H
#define MR_ORACLE_H
#include <stdint.h>

typedef struct {
    int32_t nx, ny, nz;       /* coarse cells                                   */
    int32_t mx, my, mz;       /* refinement factors M_x, M_y, M_z (Section 3.1) */
    double  lx, ly;           /* horizontal extent; the height is 1             */
    double  gamma;            /* tanh clustering of the dense z faces, 0=uniform */
    double  kappa;            /* (Ra Pr)^-1/2 or (Ra Sc)^-1/2, Eq. (2)          */
    double  dt;
    int32_t np_average;       /* N_p of the averaging step, Section 2.2; <=0 off */
    int32_t plates_dirichlet; /* 1: T=+0.5 at z=0, -0.5 at z=1; 0: adiabatic    */
    int32_t walls_xy;         /* 0: periodic in x,y; 1: impermeable adiabatic   */
    int32_t implicit_z;       /* 1: vertical diffusion Crank-Nicolson (opt-in)  */
    int32_t face_order;       /* 2: linear face values; 4: fourth-order face
                                 values of the advected scalar (Section 2.2)    */
} or_cfg;

/* Fourth-order face value (Section 2.2) on one axis: weights w[f][0..3] of the
 * cells f-2 .. f+1 for every face f = 0..N (periodic: face N is face 0), from
 * the polynomial whose averages over the stencil cells equal the cell values,
 * evaluated at the face.  Stencil: the four cells f-2..f+1; next to a wall
 * (faces 1 and N-1) the three cells on the domain side, {0,1,2} or
 * {N-3,N-2,N-1}; wall faces 0 and N get zero weights.  X: N+1 faces. */
int  or_face4_weights(int32_t N, const double* X, int32_t periodic, double length, double* w);

/* Grid (Section 3.1): dense faces first, coarse faces = every M-th dense face. */
int  or_zfaces(int32_t nz_dense, double gamma, double* zf /* nz_dense+1 */);
/* R = A_s A^-1 for every coarse cell of one axis (Section 3.2).
 * Xc: n+1 coarse faces, Xd: n*m+1 dense faces, R out [n][m][3], win out [n][3]. */
int  or_rmatrix(int32_t n, int32_t m, const double* Xc, const double* Xd,
                int32_t periodic, double length, double* R, int32_t* win);

/* Divergence-free refinement coarse -> dense (Section 3.2). */
int  or_refine(const or_cfg* c, const double* U, const double* V, const double* W,
               double* Us, double* Vs, double* Ws);
/* Transpose of or_refine: coarse gradient from dense face gradient. */
int  or_refine_adjoint(const or_cfg* c, const double* gUs, const double* gVs,
                       const double* gWs, double* gU, double* gV, double* gW);

/* One time step s (s = 0 is the forward-Euler start), Section 2.2. */
int  or_step(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
             const double* Tm1, const double* T, int64_t s, double* Tp1);
/* Explicit right-hand sides: C(Tc) (advection) and D(Td) (diffusion), Eq. (5). */
int  or_rhs(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
            const double* Tc, const double* Td, double* rhsC, double* rhsD);
/* nsteps steps from T0; on return Tprev = T^{n-1}, Tcur = T^n. */
int  or_run(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
            const double* T0, int64_t nsteps, double* Tprev, double* Tcur);

/* Continue from the pair (Tprev, Tcur) = (T^{s0-1}, T^{s0}) for nsteps steps
 * with global indices s0 .. s0+nsteps-1; the pair is updated in place. */
int  or_run_from(const or_cfg* c, const double* Us, const double* Vs, const double* Ws, int64_t s0,
                 int64_t nsteps, double* Tprev, double* Tcur);

/* out[0..5] = Nu_bottom, Nu_top, volume mean, volume variance, integral,
 * max |div u| over dense cells (Section 4.1 and the divergence check, 3.2). */
int  or_stats(const or_cfg* c, const double* T, const double* Us, const double* Vs,
              const double* Ws, double* out);
double or_max_divergence(const or_cfg* c, const double* Us, const double* Vs,
                         const double* Ws);
double or_cfl_dt(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
                 double cfl);

/* Discrete adjoint of or_run for L = sum_s wnu[s] Nu_bot(T^s) + wvar[s] Var(T^s),
 * s = 0..nsteps.  Returns dL/dT^0 and dL/d(dense faces); the coarse gradient is
 * or_refine_adjoint of the latter.  Stores every state (small grids only).    */
int  or_adjoint(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
                const double* T0, int64_t nsteps, const double* wnu, const double* wvar,
                double* loss, double* gT0, double* gUs, double* gVs, double* gWs);

/* Upscale integration (Section 3.3): the volume-weighted average of the dense
 * scalar over every coarse cell.  Tc: nz x ny x nx. */
int  or_upscale(const or_cfg* c, const double* T, double* Tc);
/* Heat-flux diagnostics (Section 4.1): nu_z[k], k = 0..Nz, the plane-averaged
 * Nu(z) = (Ra Pr)^1/2 <w T> - <dT/dz> on every dense z-face (plates: the
 * conductive flux only), and Nu_T = eps_T (Ra Pr)^1/2 with eps_T the volume-
 * averaged thermal dissipation kappa <|grad T|^2> from face gradients. */
int  or_nusselt_profile(const or_cfg* c, const double* T, const double* Ws, double* nu_z, double* nu_T);

/* Integer maps for the bit-exact comparison: the coarse cell of every dense
 * cell along x, y, z, then the three coarse cells of the R window of every
 * coarse cell along x, y, z.  out: Nx + Ny + Nz + 3*(nx + ny + nz) ints.     */
int  or_index_maps(const or_cfg* c, int32_t* out);

#endif
