/*
 * Plain FP64 CPU oracle of the multiple-resolution scalar path
 * (Chong, Ding & Xia, arXiv:1805.03426).
 *
 * TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg are the only users.  Nothing here is shared with the CUDA
 * library: grid, R matrices, refinement, step, statistics and adjoint are all
 * written out again, directly from the paper, loop by loop, in double precision.
 *
 * Readings of the paper that this file fixes (the paper is silent or garbled):
 *  - Dense z faces z_k = (1 + tanh(gamma (2k/Nz - 1)) / tanh gamma) / 2; the
 *    paper only asks for wall clustering (Section 3.1).  Cell centres are face
 *    midpoints.
 *  - R windows at a wall are one-sided ({0,1,2} / {n-3,n-2,n-1}); periodic axes
 *    wrap with unwrapped coordinates.  R is built in coordinates local to the
 *    coarse cell, (x - x_centre) / dX, which gives the same matrix.
 *  - The 3-D stepwise refinement runs z (top-down slab balance), then y
 *    (south-to-north row balance), then x (west-to-east cell balance); the
 *    garbled 2-D balance formula of Section 3.2 is read as plain flux balance.
 *  - Face values of the advected scalar: linear interpolation between cell
 *    centres (second order), or, with face_order 4, the fourth-order
 *    reconstruction of Section 2.2 read as: the cubic whose averages over the
 *    four cells f-2..f+1 equal their values, evaluated at face f; next to a
 *    wall the three cells on the domain side (quadratic).  Diffusive fluxes
 *    stay two-point in both cases.
 *  - The leapfrog starts with one forward-Euler step; the averaging step is
 *    taken when (s+1) mod N_p == 0, with D kept at level n-1.
 */
#include "mr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    int Nx, Ny, Nz;        /* dense cells                                      */
    int ufx, vfy;          /* dense U row length (Nx+w), V rows (Ny+w)          */
    int cux, cvy;          /* coarse U row length (nx+w), V rows (ny+w)         */
    double dx, dy;         /* dense widths (uniform horizontally)              */
    double DX, DY;         /* coarse widths                                     */
    double *zf, *zc, *dz;  /* dense z faces (Nz+1), centres (Nz), widths (Nz)   */
    double *Rx, *Ry, *Rz;  /* [n][m][3]                                         */
    int32_t *wx, *wy, *wz; /* [n][3] window cells                               */
    double *f4x, *f4y, *f4z; /* face_order 4: [N+1][4] weights of cells f-2..f+1 */
} geom;

static void geom_free(geom* g)
{
    free(g->zf); free(g->zc); free(g->dz);
    free(g->Rx); free(g->Ry); free(g->Rz);
    free(g->wx); free(g->wy); free(g->wz);
    free(g->f4x); free(g->f4y); free(g->f4z);
    memset(g, 0, sizeof(*g));
}

int or_zfaces(int32_t N, double gamma, double* zf)
{
    if (N < 1) return -1;
    for (int k = 0; k <= N; ++k) {
        double eta = (double)k / (double)N;          /* 0..1 */
        if (gamma == 0.0) zf[k] = eta;
        else zf[k] = 0.5 * (1.0 + tanh(gamma * (2.0 * eta - 1.0)) / tanh(gamma));
    }
    zf[0] = 0.0;
    zf[N] = 1.0;
    return 0;
}

/* Mean of s^0, s^1, s^2 over [a, b]: one row of the paper's matrix A (or A_s),
 * i.e. (1/(b-a)) * integral of x^(n-1) dx, Section 3.2. */
/* Fourth-order face values (Section 2.2).  For face f the stencil cells c
 * (lo..lo+n-1) define the polynomial p of degree n-1 with
 *   (1/h_c) int_c p = T_c,
 * in the coordinate t = (x - X_f) / h_f; the face value is p(0) = a_0, a linear
 * form sum_c w_c T_c with w the first row of A^-1, A[c][q] = mean of t^q over
 * cell c.  Solved as A^T w = e_0 by Gaussian elimination with pivoting. */
static int face_weights_one(int n, const double* lo, const double* hi, double* w)
{
    double M[4][5];
    for (int q = 0; q < n; ++q) {          /* row q of A^T: means of t^q over each cell */
        for (int c = 0; c < n; ++c) {
            double a = lo[c], b = hi[c];
            M[q][c] = (pow(b, q + 1) - pow(a, q + 1)) / ((q + 1) * (b - a));
        }
        M[q][n] = (q == 0) ? 1.0 : 0.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (M[piv][col] == 0.0) return -1;
        for (int k = 0; k <= n; ++k) { double t = M[col][k]; M[col][k] = M[piv][k]; M[piv][k] = t; }
        for (int r = col + 1; r < n; ++r) {
            double f = M[r][col] / M[col][col];
            for (int k = col; k <= n; ++k) M[r][k] -= f * M[col][k];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double v = M[r][n];
        for (int k = r + 1; k < n; ++k) v -= M[r][k] * w[k];
        w[r] = v / M[r][r];
    }
    return 0;
}

int or_face4_weights(int32_t N, const double* X, int32_t periodic, double length, double* w)
{
    memset(w, 0, sizeof(double) * 4 * (N + 1));
    if (N < (periodic ? 4 : 3)) return -1;
    for (int f = 0; f <= N; ++f) {
        int first, n;
        if (periodic) { if (f == N) continue; first = f - 2; n = 4; }
        else if (f == 0 || f == N) continue;
        else if (f == 1) { first = 0; n = 3; }
        else if (f == N - 1) { first = N - 3; n = 3; }
        else { first = f - 2; n = 4; }
        double lo[4], hi[4], cw[4];
        const double h = X[f + 1 <= N ? f + 1 : f] - X[f > 0 ? f - 1 : f];   /* a local length scale */
        for (int c = 0; c < n; ++c) {
            int cell = first + c;
            double shift = 0.0;                      /* unwrap periodic cells */
            if (cell < 0) { cell += N; shift = -length; }
            if (cell >= N) { cell -= N; shift = length; }
            lo[c] = (X[cell] + shift - X[f]) / h;
            hi[c] = (X[cell + 1] + shift - X[f]) / h;
        }
        if (face_weights_one(n, lo, hi, cw)) return -1;
        for (int c = 0; c < n; ++c) w[4 * f + (first + c) - (f - 2)] = cw[c];
    }
    if (periodic) memcpy(w + 4 * N, w, 4 * sizeof(double));
    return 0;
}

static void monomial_means(double a, double b, double row[3])
{
    row[0] = 1.0;
    row[1] = 0.5 * (a + b);
    row[2] = (a * a + a * b + b * b) / 3.0;
}

/* Solve M x = r for a 3x3 system by Gaussian elimination, partial pivoting. */
static int solve3(double M[3][3], double r[3], double x[3])
{
    for (int col = 0; col < 3; ++col) {
        int piv = col;
        for (int row = col + 1; row < 3; ++row)
            if (fabs(M[row][col]) > fabs(M[piv][col])) piv = row;
        if (M[piv][col] == 0.0) return -1;
        if (piv != col) {
            for (int k = 0; k < 3; ++k) { double t = M[col][k]; M[col][k] = M[piv][k]; M[piv][k] = t; }
            double t = r[col]; r[col] = r[piv]; r[piv] = t;
        }
        for (int row = col + 1; row < 3; ++row) {
            double f = M[row][col] / M[col][col];
            for (int k = col; k < 3; ++k) M[row][k] -= f * M[col][k];
            r[row] -= f * r[col];
        }
    }
    for (int row = 2; row >= 0; --row) {
        double s = r[row];
        for (int k = row + 1; k < 3; ++k) s -= M[row][k] * x[k];
        x[row] = s / M[row][row];
    }
    return 0;
}

int or_rmatrix(int32_t n, int32_t m, const double* Xc, const double* Xd,
               int32_t periodic, double length, double* R, int32_t* win)
{
    if (n < 1 || m < 1) return -1;
    if (m > 1 && n < 3) return -1;
    for (int i = 0; i < n; ++i) {
        /* window of three coarse cells around i (one-sided at a wall) */
        int w0 = i - 1;
        if (!periodic) { if (w0 < 0) w0 = 0; if (w0 > n - 3) w0 = n - 3; }
        if (n < 3) w0 = i;                 /* m == 1 only */
        double xc = 0.5 * (Xc[i] + Xc[i + 1]);
        double DXi = Xc[i + 1] - Xc[i];
        double A[3][3];
        for (int r = 0; r < 3; ++r) {
            int cell = w0 + r, shift = 0;
            if (periodic) {
                while (cell < 0) { cell += n; --shift; }
                while (cell >= n) { cell -= n; ++shift; }
            }
            win[3 * i + r] = (n < 3) ? i : cell;
            double lo = (Xc[cell] + shift * length - xc) / DXi;
            double hi = (Xc[cell + 1] + shift * length - xc) / DXi;
            monomial_means(lo, hi, A[r]);
        }
        for (int s = 0; s < m; ++s) {
            double* Rrow = R + ((size_t)i * m + s) * 3;
            if (m == 1) {             /* no refinement: the cell itself */
                Rrow[0] = Rrow[1] = Rrow[2] = 0.0;
                Rrow[i - w0] = 1.0;
                continue;
            }
            double As[3];
            monomial_means((Xd[i * m + s] - xc) / DXi, (Xd[i * m + s + 1] - xc) / DXi, As);
            /* R row satisfies  R_row . A = As  <=>  A^T R_row^T = As^T */
            double At[3][3], rhs[3] = {As[0], As[1], As[2]};
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) At[a][b] = A[b][a];
            if (solve3(At, rhs, Rrow)) return -2;
        }
    }
    return 0;
}

static int geom_init(const or_cfg* c, geom* g)
{
    memset(g, 0, sizeof(*g));
    if (c->nx < 1 || c->ny < 1 || c->nz < 1 || c->mx < 1 || c->my < 1 || c->mz < 1) return -1;
    int w = c->walls_xy ? 1 : 0;
    g->Nx = c->nx * c->mx; g->Ny = c->ny * c->my; g->Nz = c->nz * c->mz;
    g->ufx = g->Nx + w; g->vfy = g->Ny + w;
    g->cux = c->nx + w; g->cvy = c->ny + w;
    g->dx = c->lx / g->Nx; g->dy = c->ly / g->Ny;
    g->DX = c->lx / c->nx; g->DY = c->ly / c->ny;
    g->zf = malloc(sizeof(double) * (g->Nz + 1));
    g->zc = malloc(sizeof(double) * g->Nz);
    g->dz = malloc(sizeof(double) * g->Nz);
    g->Rx = malloc(sizeof(double) * 3 * g->Nx);
    g->Ry = malloc(sizeof(double) * 3 * g->Ny);
    g->Rz = malloc(sizeof(double) * 3 * g->Nz);
    g->wx = malloc(sizeof(int32_t) * 3 * c->nx);
    g->wy = malloc(sizeof(int32_t) * 3 * c->ny);
    g->wz = malloc(sizeof(int32_t) * 3 * c->nz);
    or_zfaces(g->Nz, c->gamma, g->zf);
    for (int k = 0; k < g->Nz; ++k) {
        g->zc[k] = 0.5 * (g->zf[k] + g->zf[k + 1]);
        g->dz[k] = g->zf[k + 1] - g->zf[k];
    }
    /* horizontal faces: uniform; coarse faces are every M-th dense face */
    double* xd = malloc(sizeof(double) * (g->Nx + 1));
    double* xc = malloc(sizeof(double) * (c->nx + 1));
    double* yd = malloc(sizeof(double) * (g->Ny + 1));
    double* yc = malloc(sizeof(double) * (c->ny + 1));
    double* zcf = malloc(sizeof(double) * (c->nz + 1));
    for (int i = 0; i <= g->Nx; ++i) xd[i] = c->lx * i / g->Nx;
    for (int j = 0; j <= g->Ny; ++j) yd[j] = c->ly * j / g->Ny;
    for (int I = 0; I <= c->nx; ++I) xc[I] = xd[I * c->mx];
    for (int J = 0; J <= c->ny; ++J) yc[J] = yd[J * c->my];
    for (int K = 0; K <= c->nz; ++K) zcf[K] = g->zf[K * c->mz];
    int periodic = !c->walls_xy;
    int rc = 0;
    rc |= or_rmatrix(c->nx, c->mx, xc, xd, periodic, c->lx, g->Rx, g->wx);
    rc |= or_rmatrix(c->ny, c->my, yc, yd, periodic, c->ly, g->Ry, g->wy);
    rc |= or_rmatrix(c->nz, c->mz, zcf, g->zf, 0, 1.0, g->Rz, g->wz);
    if (c->face_order == 4) {
        g->f4x = malloc(sizeof(double) * 4 * (g->Nx + 1));
        g->f4y = malloc(sizeof(double) * 4 * (g->Ny + 1));
        g->f4z = malloc(sizeof(double) * 4 * (g->Nz + 1));
        rc |= or_face4_weights(g->Nx, xd, periodic, c->lx, g->f4x);
        rc |= or_face4_weights(g->Ny, yd, periodic, c->ly, g->f4y);
        rc |= or_face4_weights(g->Nz, g->zf, 0, 1.0, g->f4z);
    } else if (c->face_order != 2) {
        rc = -1;
    }
    free(xd); free(xc); free(yd); free(yc); free(zcf);
    if (rc) { geom_free(g); return -1; }
    return 0;
}

/* index helpers (64-bit) */
#define IDX_C(g, k, j, i)  (((size_t)(k) * (g)->Ny + (j)) * (g)->Nx + (i))
#define IDX_U(g, k, j, i)  (((size_t)(k) * (g)->Ny + (j)) * (g)->ufx + (i))
#define IDX_V(g, k, j, i)  (((size_t)(k) * (g)->vfy + (j)) * (g)->Nx + (i))
#define IDX_W(g, k, j, i)  (((size_t)(k) * (g)->Ny + (j)) * (g)->Nx + (i))
#define CIDX_U(c, g, K, J, I) (((size_t)(K) * (c)->ny + (J)) * (g)->cux + (I))
#define CIDX_V(c, g, K, J, I) (((size_t)(K) * (g)->cvy + (J)) * (c)->nx + (I))
#define CIDX_W(c, K, J, I)    (((size_t)(K) * (c)->ny + (J)) * (c)->nx + (I))

/* ------------------------------------------------------------------------ */
/* Refinement, Section 3.2                                                   */
/* ------------------------------------------------------------------------ */

int or_refine(const or_cfg* c, const double* U, const double* V, const double* W,
              double* Us, double* Vs, double* Ws)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    const int nx = c->nx, ny = c->ny, nz = c->nz, mx = c->mx, my = c->my, mz = c->mz;
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    const int walls = c->walls_xy;
    double* Wc = calloc((size_t)(Nz + 1) * ny * nx, sizeof(double));   /* full-coarse-area W per dense plane */
    double* Vrow = calloc((size_t)Nz * g->vfy * nx, sizeof(double));    /* full-coarse-width V per dense row  */
    if (!Wc || !Vrow) { free(Wc); free(Vrow); geom_free(g); return -3; }

    /* Pass 1 (stage 0): every coarse face value split into its sub-faces by
     * the tensor product of the two tangential R matrices, Eq. V_s = R V. */
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < g->cux; ++I)
                for (int cz = 0; cz < mz; ++cz)
                    for (int b = 0; b < my; ++b) {
                        double s = 0.0;
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                s += g->Ry[(J * my + b) * 3 + p] * g->Rz[(K * mz + cz) * 3 + q] *
                                     U[CIDX_U(c, g, g->wz[3 * K + q], g->wy[3 * J + p], I)];
                        Us[IDX_U(g, K * mz + cz, J * my + b, I * mx)] = s;
                    }
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < g->cvy; ++J)
            for (int I = 0; I < nx; ++I)
                for (int cz = 0; cz < mz; ++cz)
                    for (int a = 0; a < mx; ++a) {
                        double s = 0.0;
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                s += g->Rx[(I * mx + a) * 3 + p] * g->Rz[(K * mz + cz) * 3 + q] *
                                     V[CIDX_V(c, g, g->wz[3 * K + q], J, g->wx[3 * I + p])];
                        Vs[IDX_V(g, K * mz + cz, J * my, I * mx + a)] = s;
                    }
    #pragma omp parallel for schedule(static)
    for (int K = 0; K <= nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I)
                for (int b = 0; b < my; ++b)
                    for (int a = 0; a < mx; ++a) {
                        double s = 0.0;
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                s += g->Rx[(I * mx + a) * 3 + p] * g->Ry[(J * my + b) * 3 + q] *
                                     W[CIDX_W(c, K, g->wy[3 * J + q], g->wx[3 * I + p])];
                        Ws[IDX_W(g, K * mz, J * my + b, I * mx + a)] = s;
                    }

    /* Pass 2 (stage Z): full-area vertical flux at the inner planes of each
     * coarse cell from the mass balance of each dense slab, top-down. */
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I) {
                int Ie = walls ? I + 1 : (I + 1) % nx;
                int Jn = walls ? J + 1 : (J + 1) % ny;
                Wc[CIDX_W(c, K * mz, J, I)] = W[CIDX_W(c, K, J, I)];
                if (K == nz - 1) Wc[CIDX_W(c, Nz, J, I)] = W[CIDX_W(c, nz, J, I)];
                double F = W[CIDX_W(c, K + 1, J, I)] * g->DX * g->DY;
                for (int cz = mz - 1; cz >= 1; --cz) {
                    int k = K * mz + cz;
                    double uw = 0, ue = 0, vs = 0, vn = 0;
                    for (int q = 0; q < 3; ++q) {
                        double r = g->Rz[(K * mz + cz) * 3 + q];
                        int Kq = g->wz[3 * K + q];
                        uw += r * U[CIDX_U(c, g, Kq, J, I)];
                        ue += r * U[CIDX_U(c, g, Kq, J, Ie)];
                        vs += r * V[CIDX_V(c, g, Kq, J, I)];
                        vn += r * V[CIDX_V(c, g, Kq, Jn, I)];
                    }
                    F = F + (ue - uw) * g->DY * g->dz[k] + (vn - vs) * g->DX * g->dz[k];
                    Wc[CIDX_W(c, k, J, I)] = F / (g->DX * g->DY);
                }
            }

    /* Pass 3: split the inner-plane W of each column with the tangential R's
     * using the same plane of the neighbouring columns. */
    #pragma omp parallel for schedule(static)
    for (int k = 0; k <= Nz; ++k) {
        if (k % mz == 0) continue;
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                int I = i / mx, J = j / my;
                double s = 0.0;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q)
                        s += g->Rx[i * 3 + p] * g->Ry[j * 3 + q] *
                             Wc[CIDX_W(c, k, g->wy[3 * J + q], g->wx[3 * I + p])];
                Ws[IDX_W(g, k, j, i)] = s;
            }
    }

    /* Pass 4 (stage Y): in each dense layer of a coarse cell, the full-width
     * V flux at the inner y-planes from the balance of each row, south to north. */
    #pragma omp parallel for schedule(static)
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I) {
                int Ie = walls ? I + 1 : (I + 1) % nx;
                for (int cz = 0; cz < mz; ++cz) {
                    int k = K * mz + cz;
                    double dzk = g->dz[k];
                    double G = 0.0;
                    for (int a = 0; a < mx; ++a) G += Vs[IDX_V(g, k, J * my, I * mx + a)] * g->dx;
                    G *= dzk;
                    for (int b = 0; b < my - 1; ++b) {
                        int j = J * my + b;
                        double uw = Us[IDX_U(g, k, j, I * mx)];
                        double ue = Us[IDX_U(g, k, j, Ie * mx)];
                        double wb = 0.0, wt = 0.0;
                        for (int a = 0; a < mx; ++a) {
                            wb += Ws[IDX_W(g, k, j, I * mx + a)] * g->dx;
                            wt += Ws[IDX_W(g, k + 1, j, I * mx + a)] * g->dx;
                        }
                        G = G - (ue - uw) * g->dy * dzk - (wt - wb) * g->dy;
                        Vrow[((size_t)k * g->vfy + (j + 1)) * nx + I] = G / (g->DX * dzk);
                    }
                }
            }

    /* Pass 5: split the inner-row V along x with R_x over the neighbouring
     * columns' rows. */
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j) {
            if (j % my == 0) continue;
            for (int i = 0; i < Nx; ++i) {
                int I = i / mx;
                double s = 0.0;
                for (int p = 0; p < 3; ++p)
                    s += g->Rx[i * 3 + p] * Vrow[((size_t)k * g->vfy + j) * nx + g->wx[3 * I + p]];
                Vs[IDX_V(g, k, j, i)] = s;
            }
        }

    /* Pass 6 (stage X): U at the inner x-faces from each dense cell's balance,
     * west to east. */
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j) {
            int jn = walls ? j + 1 : (j + 1) % Ny;
            for (int I = 0; I < nx; ++I) {
                double H = Us[IDX_U(g, k, j, I * mx)] * g->dy * g->dz[k];
                for (int a = 0; a < mx - 1; ++a) {
                    int i = I * mx + a;
                    H = H - (Vs[IDX_V(g, k, jn, i)] - Vs[IDX_V(g, k, j, i)]) * g->dx * g->dz[k]
                          - (Ws[IDX_W(g, k + 1, j, i)] - Ws[IDX_W(g, k, j, i)]) * g->dx * g->dy;
                    Us[IDX_U(g, k, j, i + 1)] = H / (g->dy * g->dz[k]);
                }
            }
        }

    free(Wc); free(Vrow); geom_free(g);
    return 0;
}

/* Transpose of or_refine: the passes above in reverse order, each replaced by
 * its adjoint (every assignment y = sum a_i x_i becomes x_i += a_i y). */
int or_refine_adjoint(const or_cfg* c, const double* gUs, const double* gVs,
                      const double* gWs, double* gU, double* gV, double* gW)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    const int nx = c->nx, ny = c->ny, nz = c->nz, mx = c->mx, my = c->my, mz = c->mz;
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    const int walls = c->walls_xy;
    size_t nU = (size_t)Nz * Ny * g->ufx, nV = (size_t)Nz * g->vfy * Nx, nW = (size_t)(Nz + 1) * Ny * Nx;
    double* aUs = malloc(nU * sizeof(double));
    double* aVs = malloc(nV * sizeof(double));
    double* aWs = malloc(nW * sizeof(double));
    double* aWc = calloc((size_t)(Nz + 1) * ny * nx, sizeof(double));
    double* aVrow = calloc((size_t)Nz * g->vfy * nx, sizeof(double));
    memcpy(aUs, gUs, nU * sizeof(double));
    memcpy(aVs, gVs, nV * sizeof(double));
    memcpy(aWs, gWs, nW * sizeof(double));
    memset(gU, 0, sizeof(double) * (size_t)nz * ny * g->cux);
    memset(gV, 0, sizeof(double) * (size_t)nz * g->cvy * nx);
    memset(gW, 0, sizeof(double) * (size_t)(nz + 1) * ny * nx);

    /* adjoint of pass 6 */
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j) {
            int jn = walls ? j + 1 : (j + 1) % Ny;
            for (int I = 0; I < nx; ++I) {
                double aH = 0.0;
                for (int a = mx - 2; a >= 0; --a) {
                    int i = I * mx + a;
                    aH += aUs[IDX_U(g, k, j, i + 1)] / (g->dy * g->dz[k]);
                    aUs[IDX_U(g, k, j, i + 1)] = 0.0;
                    aVs[IDX_V(g, k, jn, i)] -= aH * g->dx * g->dz[k];
                    aVs[IDX_V(g, k, j, i)] += aH * g->dx * g->dz[k];
                    aWs[IDX_W(g, k + 1, j, i)] -= aH * g->dx * g->dy;
                    aWs[IDX_W(g, k, j, i)] += aH * g->dx * g->dy;
                }
                aUs[IDX_U(g, k, j, I * mx)] += aH * g->dy * g->dz[k];
            }
        }
    /* adjoint of pass 5 */
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j) {
            if (j % my == 0) continue;
            for (int i = 0; i < Nx; ++i) {
                int I = i / mx;
                double a = aVs[IDX_V(g, k, j, i)];
                aVs[IDX_V(g, k, j, i)] = 0.0;
                for (int p = 0; p < 3; ++p)
                    aVrow[((size_t)k * g->vfy + j) * nx + g->wx[3 * I + p]] += g->Rx[i * 3 + p] * a;
            }
        }
    /* adjoint of pass 4 */
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I) {
                int Ie = walls ? I + 1 : (I + 1) % nx;
                for (int cz = 0; cz < mz; ++cz) {
                    int k = K * mz + cz;
                    double dzk = g->dz[k];
                    double aG = 0.0;
                    for (int b = my - 2; b >= 0; --b) {
                        int j = J * my + b;
                        aG += aVrow[((size_t)k * g->vfy + (j + 1)) * nx + I] / (g->DX * dzk);
                        aUs[IDX_U(g, k, j, Ie * mx)] -= aG * g->dy * dzk;
                        aUs[IDX_U(g, k, j, I * mx)] += aG * g->dy * dzk;
                        for (int a = 0; a < mx; ++a) {
                            aWs[IDX_W(g, k + 1, j, I * mx + a)] -= aG * g->dy * g->dx;
                            aWs[IDX_W(g, k, j, I * mx + a)] += aG * g->dy * g->dx;
                        }
                    }
                    for (int a = 0; a < mx; ++a) aVs[IDX_V(g, k, J * my, I * mx + a)] += aG * dzk * g->dx;
                }
            }
    /* adjoint of pass 3 */
    for (int k = 0; k <= Nz; ++k) {
        if (k % mz == 0) continue;
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                int I = i / mx, J = j / my;
                double a = aWs[IDX_W(g, k, j, i)];
                aWs[IDX_W(g, k, j, i)] = 0.0;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q)
                        aWc[CIDX_W(c, k, g->wy[3 * J + q], g->wx[3 * I + p])] += g->Rx[i * 3 + p] * g->Ry[j * 3 + q] * a;
            }
    }
    /* adjoint of pass 2 */
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I) {
                int Ie = walls ? I + 1 : (I + 1) % nx;
                int Jn = walls ? J + 1 : (J + 1) % ny;
                double aF = 0.0;
                for (int cz = 1; cz <= mz - 1; ++cz) {
                    int k = K * mz + cz;
                    aF += aWc[CIDX_W(c, k, J, I)] / (g->DX * g->DY);
                    double au = aF * g->DY * g->dz[k], av = aF * g->DX * g->dz[k];
                    for (int q = 0; q < 3; ++q) {
                        double r = g->Rz[(K * mz + cz) * 3 + q];
                        int Kq = g->wz[3 * K + q];
                        gU[CIDX_U(c, g, Kq, J, Ie)] += r * au;
                        gU[CIDX_U(c, g, Kq, J, I)] -= r * au;
                        gV[CIDX_V(c, g, Kq, Jn, I)] += r * av;
                        gV[CIDX_V(c, g, Kq, J, I)] -= r * av;
                    }
                }
                gW[CIDX_W(c, K + 1, J, I)] += aF * g->DX * g->DY;
            }
    /* adjoint of pass 1 */
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < g->cux; ++I)
                for (int cz = 0; cz < mz; ++cz)
                    for (int b = 0; b < my; ++b) {
                        double a = aUs[IDX_U(g, K * mz + cz, J * my + b, I * mx)];
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                gU[CIDX_U(c, g, g->wz[3 * K + q], g->wy[3 * J + p], I)] +=
                                    g->Ry[(J * my + b) * 3 + p] * g->Rz[(K * mz + cz) * 3 + q] * a;
                    }
    for (int K = 0; K < nz; ++K)
        for (int J = 0; J < g->cvy; ++J)
            for (int I = 0; I < nx; ++I)
                for (int cz = 0; cz < mz; ++cz)
                    for (int a = 0; a < mx; ++a) {
                        double v = aVs[IDX_V(g, K * mz + cz, J * my, I * mx + a)];
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                gV[CIDX_V(c, g, g->wz[3 * K + q], J, g->wx[3 * I + p])] +=
                                    g->Rx[(I * mx + a) * 3 + p] * g->Rz[(K * mz + cz) * 3 + q] * v;
                    }
    for (int K = 0; K <= nz; ++K)
        for (int J = 0; J < ny; ++J)
            for (int I = 0; I < nx; ++I)
                for (int b = 0; b < my; ++b)
                    for (int a = 0; a < mx; ++a) {
                        double v = aWs[IDX_W(g, K * mz, J * my + b, I * mx + a)];
                        for (int p = 0; p < 3; ++p)
                            for (int q = 0; q < 3; ++q)
                                gW[CIDX_W(c, K, g->wy[3 * J + q], g->wx[3 * I + p])] +=
                                    g->Rx[(I * mx + a) * 3 + p] * g->Ry[(J * my + b) * 3 + q] * v;
                    }
    free(aUs); free(aVs); free(aWs); free(aWc); free(aVrow); geom_free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Scalar step, Eq. (5) with the Euler-leapfrog scheme of Section 2.2        */
/* ------------------------------------------------------------------------ */

#define T_BOTTOM  0.5
#define T_TOP    -0.5

/* Fourth-order value at face f of one axis: cells f-2 .. f+1 along the axis,
 * starting at T[base] with the given stride; periodic cells wrap, cells
 * outside a walled axis carry zero weight and are not read. */
static double face4(const double* w, int f, int N, int periodic, const double* T, size_t base, size_t stride)
{
    double s = 0.0;
    for (int q = 0; q < 4; ++q) {
        double wq = w[4 * f + q];
        if (wq == 0.0) continue;
        int cell = f - 2 + q;
        if (periodic) cell = ((cell % N) + N) % N;
        s += wq * T[base + (size_t)cell * stride];
    }
    return s;
}

/* Per cell: rC = advection of Tc, rDh / rDz = horizontal / vertical diffusion
 * of Td (outward flux sums over the six faces divided by the cell volume).
 * Fluxes are positive in the +axis direction: P = u T_f A, G = kappa A dT/dn. */
static void rhs_fields(const or_cfg* c, const geom* g, const double* Us, const double* Vs,
                       const double* Ws, const double* Tc, const double* Td,
                       double* rC, double* rDh, double* rDz)
{
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    const int walls = c->walls_xy, dir = c->plates_dirichlet, o4 = c->face_order == 4;
    const double kap = c->kappa, dx = g->dx, dy = g->dy;
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                const size_t xrow = IDX_C(g, k, j, 0), ycol = IDX_C(g, k, 0, i), zcol = IDX_C(g, 0, j, i);
                const size_t m = IDX_C(g, k, j, i);
                const double dzk = g->dz[k], vol = dx * dy * dzk;
                double Pw = 0, Pe = 0, Ps = 0, Pn = 0, Pb = 0, Pt = 0;
                double Gw = 0, Ge = 0, Gs = 0, Gn = 0, Gb = 0, Gt = 0;
                /* x faces */
                double Ax = dy * dzk;
                if (!(walls && i == 0)) {
                    int iw = walls ? i - 1 : (i - 1 + Nx) % Nx;
                    size_t mw = IDX_C(g, k, j, iw);
                    double Tf = o4 ? face4(g->f4x, i, Nx, !walls, Tc, xrow, 1) : 0.5 * (Tc[mw] + Tc[m]);
                    Pw = Us[IDX_U(g, k, j, i)] * Tf * Ax;
                    Gw = kap * Ax * (Td[m] - Td[mw]) / dx;
                }
                if (!(walls && i == Nx - 1)) {
                    int ie = (i + 1) % Nx;
                    int fe = walls ? i + 1 : ie;
                    size_t me = IDX_C(g, k, j, ie);
                    double Tf = o4 ? face4(g->f4x, i + 1, Nx, !walls, Tc, xrow, 1) : 0.5 * (Tc[m] + Tc[me]);
                    Pe = Us[IDX_U(g, k, j, fe)] * Tf * Ax;
                    Ge = kap * Ax * (Td[me] - Td[m]) / dx;
                }
                /* y faces */
                double Ay = dx * dzk;
                if (!(walls && j == 0)) {
                    int js = walls ? j - 1 : (j - 1 + Ny) % Ny;
                    size_t ms = IDX_C(g, k, js, i);
                    double Tf = o4 ? face4(g->f4y, j, Ny, !walls, Tc, ycol, Nx) : 0.5 * (Tc[ms] + Tc[m]);
                    Ps = Vs[IDX_V(g, k, j, i)] * Tf * Ay;
                    Gs = kap * Ay * (Td[m] - Td[ms]) / dy;
                }
                if (!(walls && j == Ny - 1)) {
                    int jn = (j + 1) % Ny;
                    int fn = walls ? j + 1 : jn;
                    size_t mn = IDX_C(g, k, jn, i);
                    double Tf = o4 ? face4(g->f4y, j + 1, Ny, !walls, Tc, ycol, Nx) : 0.5 * (Tc[m] + Tc[mn]);
                    Pn = Vs[IDX_V(g, k, fn, i)] * Tf * Ay;
                    Gn = kap * Ay * (Td[mn] - Td[m]) / dy;
                }
                /* z faces: linear interpolation between the two cell centres */
                double Az = dx * dy;
                if (k == 0) {
                    if (dir) Gb = kap * Az * (Td[m] - T_BOTTOM) / (g->zc[0] - g->zf[0]);
                } else {
                    size_t mb = IDX_C(g, k - 1, j, i);
                    double Tf = o4 ? face4(g->f4z, k, Nz, 0, Tc, zcol, (size_t)Nx * Ny)
                                   : (g->dz[k] * Tc[mb] + g->dz[k - 1] * Tc[m]) / (g->dz[k - 1] + g->dz[k]);
                    Pb = Ws[IDX_W(g, k, j, i)] * Tf * Az;
                    Gb = kap * Az * (Td[m] - Td[mb]) / (g->zc[k] - g->zc[k - 1]);
                }
                if (k == Nz - 1) {
                    if (dir) Gt = kap * Az * (T_TOP - Td[m]) / (g->zf[Nz] - g->zc[Nz - 1]);
                } else {
                    size_t mt = IDX_C(g, k + 1, j, i);
                    double Tf = o4 ? face4(g->f4z, k + 1, Nz, 0, Tc, zcol, (size_t)Nx * Ny)
                                   : (g->dz[k + 1] * Tc[m] + g->dz[k] * Tc[mt]) / (g->dz[k] + g->dz[k + 1]);
                    Pt = Ws[IDX_W(g, k + 1, j, i)] * Tf * Az;
                    Gt = kap * Az * (Td[mt] - Td[m]) / (g->zc[k + 1] - g->zc[k]);
                }
                rC[m] = (Pw - Pe + Ps - Pn + Pb - Pt) / vol;
                rDh[m] = (Ge - Gw + Gn - Gs) / vol;
                rDz[m] = (Gt - Gb) / vol;
            }
}

int or_rhs(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
           const double* Tc, const double* Td, double* rhsC, double* rhsD)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    size_t n = (size_t)g->Nx * g->Ny * g->Nz;
    double* rz = malloc(n * sizeof(double));
    rhs_fields(c, g, Us, Vs, Ws, Tc, Td, rhsC, rhsD, rz);
    for (size_t m = 0; m < n; ++m) rhsD[m] += rz[m];
    free(rz); geom_free(g);
    return 0;
}

/* Coefficients of step s: T^{s+1} = a T^{s-1} + b T^s + g dt [C(T^s) + D(T^{s-1})].
 * s = 0 is the forward-Euler start (T^{-1} taken as T^0). */
static void step_coeffs(const or_cfg* c, int64_t s, double* a, double* b, double* gc)
{
    if (s == 0) { *a = 0.0; *b = 1.0; *gc = 1.0; return; }
    if (c->np_average > 0 && (s + 1) % c->np_average == 0) { *a = 0.5; *b = 0.5; *gc = 1.5; return; }
    *a = 1.0; *b = 0.0; *gc = 2.0;
}

/* Thomas algorithm for one tridiagonal system (lo, di, up) x = r; r is overwritten. */
static void thomas(int n, const double* lo, const double* di, const double* up, double* r, double* work)
{
    work[0] = up[0] / di[0];
    r[0] = r[0] / di[0];
    for (int k = 1; k < n; ++k) {
        double den = di[k] - lo[k] * work[k - 1];
        work[k] = up[k] / den;
        r[k] = (r[k] - lo[k] * r[k - 1]) / den;
    }
    for (int k = n - 2; k >= 0; --k) r[k] -= work[k] * r[k + 1];
}

static void step_impl(const or_cfg* c, const geom* g, const double* Us, const double* Vs,
                      const double* Ws, const double* Tm1, const double* T, int64_t s,
                      double* Tp1, double* rC, double* rDh, double* rDz)
{
    const size_t n = (size_t)g->Nx * g->Ny * g->Nz;
    double a, b, gc;
    step_coeffs(c, s, &a, &b, &gc);
    const double* Told = (s == 0) ? T : Tm1;
    rhs_fields(c, g, Us, Vs, Ws, T, Told, rC, rDh, rDz);
    const double dt = c->dt;
    if (!c->implicit_z) {
        #pragma omp parallel for schedule(static)
        for (size_t m = 0; m < n; ++m) {
            double rhs = rC[m] + (rDh[m] + rDz[m]);
            if (s == 0) Tp1[m] = T[m] + dt * rhs;
            else if (a == 1.0) Tp1[m] = Tm1[m] + 2.0 * dt * rhs;
            else Tp1[m] = 0.5 * Tm1[m] + 0.5 * T[m] + 1.5 * dt * rhs;
        }
        return;
    }
    /* Opt-in: vertical diffusion by Crank-Nicolson over the step's interval,
     *   (I - g dt/2 Lz) T^{s+1} = a T^{s-1} + b T^s + g dt [C + Dh + Dz(T^{s-1})/2 + bz/2],
     * Dz(T) = Lz T + bz (bz: the Dirichlet plate terms).  One tridiagonal
     * system per (x, y) column. */
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    const double kap = c->kappa, half = 0.5 * gc * dt;
    #pragma omp parallel
    {
        double *lo = calloc(Nz, sizeof(double)), *di = calloc(Nz, sizeof(double));
        double *up = calloc(Nz, sizeof(double)), *r = calloc(Nz, sizeof(double));
        double *wk = calloc(Nz, sizeof(double));
        #pragma omp for schedule(static)
        for (int jj = 0; jj < Nx * Ny; ++jj) {
            int j = jj / Nx, i = jj % Nx;
            for (int k = 0; k < Nz; ++k) {
                size_t m = IDX_C(g, k, j, i);
                double bz = 0.0;
                double cb = 0.0, ct = 0.0;   /* kappa/(dz d) toward bottom / top neighbour */
                if (k > 0) cb = kap / (g->dz[k] * (g->zc[k] - g->zc[k - 1]));
                else if (c->plates_dirichlet) { cb = kap / (g->dz[0] * (g->zc[0] - g->zf[0])); bz += cb * T_BOTTOM; }
                if (k < Nz - 1) ct = kap / (g->dz[k] * (g->zc[k + 1] - g->zc[k]));
                else if (c->plates_dirichlet) { ct = kap / (g->dz[k] * (g->zf[Nz] - g->zc[k])); bz += ct * T_TOP; }
                lo[k] = (k > 0) ? -half * cb : 0.0;
                up[k] = (k < Nz - 1) ? -half * ct : 0.0;
                di[k] = 1.0 + half * (cb + ct);
                double base = (s == 0) ? T[m] : a * Tm1[m] + b * T[m];
                r[k] = base + gc * dt * (rC[m] + rDh[m] + 0.5 * rDz[m] + 0.5 * bz);
            }
            thomas(Nz, lo, di, up, r, wk);
            for (int k = 0; k < Nz; ++k) Tp1[IDX_C(g, k, j, i)] = r[k];
        }
        free(lo); free(di); free(up); free(r); free(wk);
    }
}

int or_step(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
            const double* Tm1, const double* T, int64_t s, double* Tp1)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    size_t n = (size_t)g->Nx * g->Ny * g->Nz;
    double* w = malloc(3 * n * sizeof(double));
    step_impl(c, g, Us, Vs, Ws, Tm1, T, s, Tp1, w, w + n, w + 2 * n);
    free(w); geom_free(g);
    return 0;
}

int or_run(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
           const double* T0, int64_t nsteps, double* Tprev, double* Tcur)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    size_t n = (size_t)g->Nx * g->Ny * g->Nz;
    double* w = malloc(4 * n * sizeof(double));
    double *a = Tprev, *b = Tcur, *nxt = w + 3 * n;
    memcpy(a, T0, n * sizeof(double));
    memcpy(b, T0, n * sizeof(double));
    for (int64_t s = 0; s < nsteps; ++s) {
        step_impl(c, g, Us, Vs, Ws, a, b, s, nxt, w, w + n, w + 2 * n);
        memcpy(a, b, n * sizeof(double));
        memcpy(b, nxt, n * sizeof(double));
    }
    free(w); geom_free(g);
    return 0;
}

int or_run_from(const or_cfg* c, const double* Us, const double* Vs, const double* Ws, int64_t s0,
                int64_t nsteps, double* Tprev, double* Tcur)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    size_t n = (size_t)g->Nx * g->Ny * g->Nz;
    double* w = malloc(4 * n * sizeof(double));
    /* the three levels rotate through Tprev, Tcur and one work array */
    double *a = Tprev, *b = Tcur, *nxt = w + 3 * n;
    for (int64_t s = s0; s < s0 + nsteps; ++s) {
        step_impl(c, g, Us, Vs, Ws, a, b, s, nxt, w, w + n, w + 2 * n);
        double* t = a; a = b; b = nxt; nxt = t;
    }
    if (a != Tprev) memcpy(w, a, n * sizeof(double));       /* a may alias Tcur: stage it */
    if (b != Tcur) memcpy(Tcur, b, n * sizeof(double));
    if (a != Tprev) memcpy(Tprev, w, n * sizeof(double));
    free(w); geom_free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Statistics, Section 4.1                                                    */
/* ------------------------------------------------------------------------ */

static double cell_divergence(const or_cfg* c, const geom* g, const double* Us, const double* Vs,
                              const double* Ws, int k, int j, int i)
{
    int fe = c->walls_xy ? i + 1 : (i + 1) % g->Nx;
    int fn = c->walls_xy ? j + 1 : (j + 1) % g->Ny;
    double out = (Us[IDX_U(g, k, j, fe)] - Us[IDX_U(g, k, j, i)]) * g->dy * g->dz[k]
               + (Vs[IDX_V(g, k, fn, i)] - Vs[IDX_V(g, k, j, i)]) * g->dx * g->dz[k]
               + (Ws[IDX_W(g, k + 1, j, i)] - Ws[IDX_W(g, k, j, i)]) * g->dx * g->dy;
    return out / (g->dx * g->dy * g->dz[k]);
}

double or_max_divergence(const or_cfg* c, const double* Us, const double* Vs, const double* Ws)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1.0;
    double mx = 0.0;
    for (int k = 0; k < g->Nz; ++k)
        for (int j = 0; j < g->Ny; ++j)
            for (int i = 0; i < g->Nx; ++i) {
                double d = fabs(cell_divergence(c, g, Us, Vs, Ws, k, j, i));
                if (d > mx) mx = d;
            }
    geom_free(g);
    return mx;
}

int or_stats(const or_cfg* c, const double* T, const double* Us, const double* Vs,
             const double* Ws, double* out)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    /* plate Nusselt numbers: conductive flux at the plates over the conductive
     * flux of the linear profile (Delta T = H = 1), area-averaged */
    double nb = 0.0, nt = 0.0;
    for (int j = 0; j < Ny; ++j)
        for (int i = 0; i < Nx; ++i) {
            nb += (T_BOTTOM - T[IDX_C(g, 0, j, i)]) / (g->zc[0] - g->zf[0]);
            nt += (T[IDX_C(g, Nz - 1, j, i)] - T_TOP) / (g->zf[Nz] - g->zc[Nz - 1]);
        }
    out[0] = nb / ((double)Nx * Ny);
    out[1] = nt / ((double)Nx * Ny);
    double vt = 0.0, s = 0.0;
    for (int k = 0; k < Nz; ++k) {
        double vol = g->dx * g->dy * g->dz[k];
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) { s += T[IDX_C(g, k, j, i)] * vol; vt += vol; }
    }
    double mean = s / vt, v = 0.0;
    for (int k = 0; k < Nz; ++k) {
        double vol = g->dx * g->dy * g->dz[k];
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) { double d = T[IDX_C(g, k, j, i)] - mean; v += d * d * vol; }
    }
    out[2] = mean;
    out[3] = v / vt;
    out[4] = s;
    geom_free(g);
    out[5] = (Us && Vs && Ws) ? or_max_divergence(c, Us, Vs, Ws) : 0.0;
    return 0;
}

double or_cfl_dt(const or_cfg* c, const double* Us, const double* Vs, const double* Ws, double cfl)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1.0;
    double mx = 0.0;
    for (int k = 0; k < g->Nz; ++k)
        for (int j = 0; j < g->Ny; ++j)
            for (int i = 0; i < g->Nx; ++i) {
                int fe = c->walls_xy ? i + 1 : (i + 1) % g->Nx;
                int fn = c->walls_xy ? j + 1 : (j + 1) % g->Ny;
                double u = fmax(fabs(Us[IDX_U(g, k, j, i)]), fabs(Us[IDX_U(g, k, j, fe)]));
                double v = fmax(fabs(Vs[IDX_V(g, k, j, i)]), fabs(Vs[IDX_V(g, k, fn, i)]));
                double w = fmax(fabs(Ws[IDX_W(g, k, j, i)]), fabs(Ws[IDX_W(g, k + 1, j, i)]));
                double r = u / g->dx + v / g->dy + w / g->dz[k];
                if (r > mx) mx = r;
            }
    geom_free(g);
    return mx > 0.0 ? cfl / mx : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of or_run                                                */
/* ------------------------------------------------------------------------ */

/* out += alpha * C(u)^T lam ; out += beta * D_lin^T lam (either may be NULL).
 * With <lam, C T> = sum_faces P_f (lam_R/V_R - lam_L/V_L) and
 *      <lam, D T> = sum_faces G_f (lam_L/V_L - lam_R/V_R) + plate terms. */
static void transpose_ops(const or_cfg* c, const geom* g, const double* Us, const double* Vs,
                          const double* Ws, const double* lam, double alpha, double* outC,
                          double beta, double* outD)
{
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz, walls = c->walls_xy;
    const double kap = c->kappa, dx = g->dx, dy = g->dy;
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                const size_t mR = IDX_C(g, k, j, i);
                const double vR = dx * dy * g->dz[k];
                /* x face between (i-1) and i */
                if (!(walls && i == 0)) {
                    size_t mL = IDX_C(g, k, j, walls ? i - 1 : (i - 1 + Nx) % Nx);
                    double A = dy * g->dz[k], vL = vR;
                    double dl = lam[mR] / vR - lam[mL] / vL;
                    if (outC) { double q = alpha * Us[IDX_U(g, k, j, i)] * A * dl;
                                outC[mL] += 0.5 * q; outC[mR] += 0.5 * q; }
                    if (outD) { double q = beta * kap * A / dx * (-dl);
                                outD[mR] += q; outD[mL] -= q; }
                }
                /* y face between (j-1) and j */
                if (!(walls && j == 0)) {
                    size_t mL = IDX_C(g, k, walls ? j - 1 : (j - 1 + Ny) % Ny, i);
                    double A = dx * g->dz[k], vL = vR;
                    double dl = lam[mR] / vR - lam[mL] / vL;
                    if (outC) { double q = alpha * Vs[IDX_V(g, k, j, i)] * A * dl;
                                outC[mL] += 0.5 * q; outC[mR] += 0.5 * q; }
                    if (outD) { double q = beta * kap * A / dy * (-dl);
                                outD[mR] += q; outD[mL] -= q; }
                }
                /* z face between (k-1) and k, or the bottom plate */
                double A = dx * dy;
                if (k > 0) {
                    size_t mL = IDX_C(g, k - 1, j, i);
                    double vL = dx * dy * g->dz[k - 1];
                    double dl = lam[mR] / vR - lam[mL] / vL;
                    double wL = g->dz[k] / (g->dz[k - 1] + g->dz[k]);
                    double wR = g->dz[k - 1] / (g->dz[k - 1] + g->dz[k]);
                    if (outC) { double q = alpha * Ws[IDX_W(g, k, j, i)] * A * dl;
                                outC[mL] += wL * q; outC[mR] += wR * q; }
                    if (outD) { double q = beta * kap * A / (g->zc[k] - g->zc[k - 1]) * (-dl);
                                outD[mR] += q; outD[mL] -= q; }
                } else if (outD && c->plates_dirichlet) {
                    outD[mR] -= beta * kap * A / (g->zc[0] - g->zf[0]) * lam[mR] / vR;
                }
                if (k == Nz - 1 && outD && c->plates_dirichlet)
                    outD[mR] -= beta * kap * A / (g->zf[Nz] - g->zc[Nz - 1]) * lam[mR] / vR;
            }
}

/* gface += coef * dC/du_f contracted with lam: A_f T_f (lam_R/V_R - lam_L/V_L). */
static void velocity_grad(const or_cfg* c, const geom* g, const double* T, const double* lam,
                          double coef, double* gUs, double* gVs, double* gWs)
{
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz, walls = c->walls_xy;
    const double dx = g->dx, dy = g->dy;
    for (int k = 0; k < Nz; ++k)
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                const size_t mR = IDX_C(g, k, j, i);
                const double vR = dx * dy * g->dz[k];
                if (!(walls && i == 0)) {
                    size_t mL = IDX_C(g, k, j, walls ? i - 1 : (i - 1 + Nx) % Nx);
                    gUs[IDX_U(g, k, j, i)] += coef * dy * g->dz[k] * 0.5 * (T[mL] + T[mR]) *
                                              (lam[mR] / vR - lam[mL] / vR);
                }
                if (!(walls && j == 0)) {
                    size_t mL = IDX_C(g, k, walls ? j - 1 : (j - 1 + Ny) % Ny, i);
                    gVs[IDX_V(g, k, j, i)] += coef * dx * g->dz[k] * 0.5 * (T[mL] + T[mR]) *
                                              (lam[mR] / vR - lam[mL] / vR);
                }
                if (k > 0) {
                    size_t mL = IDX_C(g, k - 1, j, i);
                    double vL = dx * dy * g->dz[k - 1];
                    double Tf = (g->dz[k] * T[mL] + g->dz[k - 1] * T[mR]) / (g->dz[k - 1] + g->dz[k]);
                    gWs[IDX_W(g, k, j, i)] += coef * dx * dy * Tf * (lam[mR] / vR - lam[mL] / vL);
                }
            }
}

int or_adjoint(const or_cfg* c, const double* Us, const double* Vs, const double* Ws,
               const double* T0, int64_t S, const double* wnu, const double* wvar,
               double* loss, double* gT0, double* gUs, double* gVs, double* gWs)
{
    if (c->implicit_z || c->face_order != 2) return -4;   /* adjoint of the explicit second-order scheme */
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz;
    const size_t n = (size_t)Nx * Ny * Nz;
    double* st = malloc((size_t)(S + 1) * n * sizeof(double));    /* T^0 .. T^S */
    double* lam = calloc((size_t)(S + 1) * n, sizeof(double));
    double* w = malloc(3 * n * sizeof(double));
    double* vol = malloc(n * sizeof(double));
    if (!st || !lam || !w || !vol) { free(st); free(lam); free(w); free(vol); geom_free(g); return -3; }
    for (int k = 0; k < Nz; ++k)
        for (size_t m = 0; m < (size_t)Nx * Ny; ++m) vol[(size_t)k * Nx * Ny + m] = g->dx * g->dy * g->dz[k];
    double vt = 0.0;
    for (size_t m = 0; m < n; ++m) vt += vol[m];

    memcpy(st, T0, n * sizeof(double));
    for (int64_t s = 0; s < S; ++s) {
        const double* Tm1 = (s == 0) ? st : st + (size_t)(s - 1) * n;
        step_impl(c, g, Us, Vs, Ws, Tm1, st + (size_t)s * n, s, st + (size_t)(s + 1) * n,
                  w, w + n, w + 2 * n);
    }
    /* loss and its direct derivative at every level */
    double L = 0.0;
    const double zb = g->zc[0] - g->zf[0];
    for (int64_t s = 0; s <= S; ++s) {
        const double* T = st + (size_t)s * n;
        double* l = lam + (size_t)s * n;
        if (wnu && wnu[s] != 0.0) {
            double nb = 0.0;
            for (size_t m = 0; m < (size_t)Nx * Ny; ++m) {
                nb += (T_BOTTOM - T[m]) / zb;
                l[m] += -wnu[s] / (zb * (double)Nx * Ny);
            }
            L += wnu[s] * nb / ((double)Nx * Ny);
        }
        if (wvar && wvar[s] != 0.0) {
            double mean = 0.0, var = 0.0;
            for (size_t m = 0; m < n; ++m) mean += T[m] * vol[m];
            mean /= vt;
            for (size_t m = 0; m < n; ++m) { double d = T[m] - mean; var += d * d * vol[m]; }
            L += wvar[s] * var / vt;
            for (size_t m = 0; m < n; ++m) l[m] += wvar[s] * 2.0 * vol[m] * (T[m] - mean) / vt;
        }
    }
    *loss = L;
    memset(gUs, 0, sizeof(double) * (size_t)Nz * Ny * g->ufx);
    memset(gVs, 0, sizeof(double) * (size_t)Nz * g->vfy * Nx);
    memset(gWs, 0, sizeof(double) * (size_t)(Nz + 1) * Ny * Nx);
    /* backward sweep */
    double* ct = w;
    double* dt_ = w + n;
    for (int64_t s = S - 1; s >= 0; --s) {
        double a, b, gc;
        step_coeffs(c, s, &a, &b, &gc);
        const double* l1 = lam + (size_t)(s + 1) * n;
        memset(ct, 0, n * sizeof(double));
        memset(dt_, 0, n * sizeof(double));
        transpose_ops(c, g, Us, Vs, Ws, l1, 1.0, ct, 1.0, dt_);
        velocity_grad(c, g, st + (size_t)s * n, l1, gc * c->dt, gUs, gVs, gWs);
        double* ls = lam + (size_t)s * n;
        if (s == 0) {
            for (size_t m = 0; m < n; ++m) ls[m] += l1[m] + c->dt * (ct[m] + dt_[m]);
        } else {
            double* lm = lam + (size_t)(s - 1) * n;
            for (size_t m = 0; m < n; ++m) {
                lm[m] += a * l1[m] + gc * c->dt * dt_[m];
                ls[m] += b * l1[m] + gc * c->dt * ct[m];
            }
        }
    }
    memcpy(gT0, lam, n * sizeof(double));
    free(st); free(lam); free(w); free(vol); geom_free(g);
    return 0;
}

int or_index_maps(const or_cfg* c, int32_t* out)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    int32_t* p = out;
    for (int i = 0; i < g->Nx; ++i) *p++ = i / c->mx;
    for (int j = 0; j < g->Ny; ++j) *p++ = j / c->my;
    for (int k = 0; k < g->Nz; ++k) *p++ = k / c->mz;
    for (int I = 0; I < 3 * c->nx; ++I) *p++ = g->wx[I];
    for (int J = 0; J < 3 * c->ny; ++J) *p++ = g->wy[J];
    for (int K = 0; K < 3 * c->nz; ++K) *p++ = g->wz[K];
    geom_free(g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Upscale integration and heat-flux diagnostics                             */
/* ------------------------------------------------------------------------ */

int or_upscale(const or_cfg* c, const double* T, double* Tc)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    for (int K = 0; K < c->nz; ++K)
        for (int J = 0; J < c->ny; ++J)
            for (int I = 0; I < c->nx; ++I) {
                double s = 0.0, v = 0.0;
                for (int k = K * c->mz; k < (K + 1) * c->mz; ++k)
                    for (int j = J * c->my; j < (J + 1) * c->my; ++j)
                        for (int i = I * c->mx; i < (I + 1) * c->mx; ++i) {
                            double vol = g->dx * g->dy * g->dz[k];
                            s += T[IDX_C(g, k, j, i)] * vol;
                            v += vol;
                        }
                Tc[((size_t)K * c->ny + J) * c->nx + I] = s / v;
            }
    geom_free(g);
    return 0;
}

int or_nusselt_profile(const or_cfg* c, const double* T, const double* Ws, double* nu_z, double* nu_T)
{
    geom G, *g = &G;
    if (geom_init(c, g)) return -1;
    const int Nx = g->Nx, Ny = g->Ny, Nz = g->Nz, walls = c->walls_xy;
    const double inv_area = 1.0 / ((double)Nx * Ny);
    /* Nu(z) on every z-face: advective heat flux / kappa minus the mean gradient */
    for (int k = 0; k <= Nz; ++k) {
        double s = 0.0;
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                if (k == 0) s += (T_BOTTOM - T[IDX_C(g, 0, j, i)]) / (g->zc[0] - g->zf[0]);
                else if (k == Nz) s += (T[IDX_C(g, Nz - 1, j, i)] - T_TOP) / (g->zf[Nz] - g->zc[Nz - 1]);
                else {
                    double Tl = T[IDX_C(g, k - 1, j, i)], Tr = T[IDX_C(g, k, j, i)];
                    double Tf = c->face_order == 4
                                    ? face4(g->f4z, k, Nz, 0, T, IDX_C(g, 0, j, i), (size_t)Nx * Ny)
                                    : (g->dz[k] * Tl + g->dz[k - 1] * Tr) / (g->dz[k - 1] + g->dz[k]);
                    double grad = (Tr - Tl) / (g->zc[k] - g->zc[k - 1]);
                    s += Ws[IDX_W(g, k, j, i)] * Tf / c->kappa - grad;
                }
            }
        nu_z[k] = s * inv_area;
    }
    /* thermal dissipation: kappa sum_faces A d (dT/d)^2 / V, plates at their Dirichlet values */
    double e = 0.0, vt = 0.0;
    for (int k = 0; k < Nz; ++k) {
        vt += g->dx * g->dy * g->dz[k] * Nx * Ny;
        for (int j = 0; j < Ny; ++j)
            for (int i = 0; i < Nx; ++i) {
                double t = T[IDX_C(g, k, j, i)];
                if (!(walls && i == 0)) {
                    double d = t - T[IDX_C(g, k, j, walls ? i - 1 : (i - 1 + Nx) % Nx)];
                    e += d * d / (g->dx * g->dx) * g->dx * g->dy * g->dz[k];
                }
                if (!(walls && j == 0)) {
                    double d = t - T[IDX_C(g, k, walls ? j - 1 : (j - 1 + Ny) % Ny, i)];
                    e += d * d / (g->dy * g->dy) * g->dx * g->dy * g->dz[k];
                }
                double dist, d;
                if (k > 0) {
                    dist = g->zc[k] - g->zc[k - 1];
                    d = t - T[IDX_C(g, k - 1, j, i)];
                    e += d * d / (dist * dist) * g->dx * g->dy * dist;
                } else if (c->plates_dirichlet) {
                    dist = g->zc[0] - g->zf[0];
                    d = t - T_BOTTOM;
                    e += d * d / (dist * dist) * g->dx * g->dy * dist;
                }
                if (k == Nz - 1 && c->plates_dirichlet) {
                    dist = g->zf[Nz] - g->zc[Nz - 1];
                    d = T_TOP - t;
                    e += d * d / (dist * dist) * g->dx * g->dy * dist;
                }
            }
    }
    /* Nu_T = eps_T (Ra Pr)^1/2 = kappa <|grad T|^2> / kappa */
    *nu_T = e / vt;
    geom_free(g);
    return 0;
}
