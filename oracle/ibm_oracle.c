/*
 * Oracle for the discrete-forcing IBM step (arXiv 2301.09349), plain FP64 C.
 *
 * TEST INFRASTRUCTURE ONLY.  Loaded by tests/, by __graft_entry__.smoke() and
 * by the benchmark's CPU-baseline leg; never by the product path.  It shares
 * no code with the CUDA library.  Every routine follows the definition it
 * cites, written out with plain loops; parallel loops (OpenMP) only split
 * independent per-cell work and never change the arithmetic of a cell.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *  - the multi-D kernel is the tensor product of the 1D kernel with r in
 *    units of h, delta_h = Phi / h^d, so with the Eulerian quadrature h^d the
 *    interpolation weight is Phi (Sec. 2.2, Eq. interp);
 *  - A and eps are taken in dimensionless form A~_kl = sum_j Phi_k Phi_l,
 *    A~ eps~ = 1, eps = h^d eps~, so that interpolating a spread unit field
 *    returns 1 (Sec. 2.2, partition of unity);
 *  - the explicit scheme has a_s = a_e = 1/dt (Eqs. forceMomentum, corr3.8);
 *  - the forcing is applied once per time step after the SSP-RK2 predictor
 *    (App. B steps 1-3) and the heat source acts on internal energy
 *    (Eq. e_centralF2), the f.u work term being dropped (Sec. 2.2.1);
 *  - fluid scheme: MUSCL on primitives with the van Leer limiter, Rusanov
 *    convective flux, central viscous and heat fluxes (Sec. 2.2.2 names
 *    second-order centred schemes with a van Leer limiter; the Rusanov flux
 *    and SSP-RK2 are the explicit density-based stand-in for rhoCentralFoam).
 */
#include "ibm_oracle.h"

/* Largest fraction of a forced cell's internal energy the heat source may
 * remove in one step (positivity reading of the forced update). */
#define HEAT_SOURCE_CAP 0.9

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_BC_FREESTREAM 0
#define OR_BC_ZEROGRAD 1
#define OR_BC_SLIP 2
#define OR_BC_PERIODIC 3

static int g_threads = 1;
void or_set_threads(int nthreads) { g_threads = nthreads < 1 ? 1 : nthreads; }
int or_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------------ */
/* grid helpers                                                              */
/* ------------------------------------------------------------------------ */

static long n_cells(const or_desc *g) {
    long N = 1;
    for (int d = 0; d < g->dim; ++d) N *= g->n[d];
    return N;
}
static int n_comp(const or_desc *g) { return g->dim + 2; }
static double cell_center(const or_desc *g, int d, int i) { return g->lo[d] + (i + 0.5) * g->h; }

/* gas constants in units rho_inf = U_inf = T_inf = 1 */
static double gas_R(const or_desc *g) { return 1.0 / (g->gamma * g->Mach * g->Mach); }
static double gas_cv(const or_desc *g) { return gas_R(g) / (g->gamma - 1.0); }
static double gas_cp(const or_desc *g) { return g->gamma * gas_cv(g); }

/* Sutherland's law (Sec. 2.1), mu_inf = 1/Re at T = 1 */
static double viscosity(const or_desc *g, double T) {
    if (g->Re <= 0.0) return 0.0;
    return (1.0 / g->Re) * pow(T, 1.5) * (1.0 + g->S) / (T + g->S);
}

/* ------------------------------------------------------------------------ */
/* the regularised 3-point delta (Sec. 2.2, Pinelli et al.)                  */
/* ------------------------------------------------------------------------ */

double or_phi(double r) {
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a <= 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
    return 0.0;
}

void or_phi_many(const double *r, long n, double *out) {
    for (long i = 0; i < n; ++i) out[i] = or_phi(r[i]);
}

/* Phi_k(j): tensor-product weight of marker position X at cell (i0,i1,i2) */
static double weight(const or_desc *g, const double *X, const int *c) {
    double w = 1.0;
    for (int d = 0; d < g->dim; ++d) w *= or_phi((cell_center(g, d, c[d]) - X[d]) / g->h);
    return w;
}

/* ------------------------------------------------------------------------ */
/* markers: owner cell, dedup, binning                                       */
/* ------------------------------------------------------------------------ */

/* owner cell floor((X - lo)/h); returns 0, or -1 when a marker sits closer
 * than two cells to the domain edge (its support plus the MUSCL halo must
 * stay inside). */
int or_owner_cells(const or_desc *g, int n, const double *X, int *cell) {
    int bad = 0;
    for (int k = 0; k < n; ++k)
        for (int d = 0; d < g->dim; ++d) {
            double x = X[(long)k * g->dim + d];
            if (!isfinite(x)) { bad = 1; cell[(long)k * g->dim + d] = 0; continue; }
            double c = floor((x - g->lo[d]) / g->h);
            if (c < 2.0 || c > (double)(g->n[d] - 3)) bad = 1;
            cell[(long)k * g->dim + d] = (c < -1e9 || c > 1e9) ? 0 : (int)c;
        }
    return bad ? -1 : 0;
}

typedef struct { long key; double dist; int idx; } dd_item;

static int dd_cmp(const void *a, const void *b) {
    const dd_item *x = (const dd_item *)a, *y = (const dd_item *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->dist != y->dist) return x->dist < y->dist ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}
static int int_cmp(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return x < y ? -1 : (x > y);
}

/* Sec. 3.1: of the markers falling in one mesh element keep only the one
 * closest to the element centre (ties: lowest input index).  `keep` receives
 * the kept input indices in ascending order. */
int or_dedup(const or_desc *g, int n, const double *X, int *keep, int *n_kept) {
    int *cell = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1) * g->dim);
    int rc = or_owner_cells(g, n, X, cell);
    dd_item *it = (dd_item *)malloc(sizeof(dd_item) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) {
        long key = 0;
        double dist = 0.0;
        for (int d = g->dim - 1; d >= 0; --d) {
            int c = cell[(long)k * g->dim + d];
            key = key * (long)g->n[d] + c;
            double dx = X[(long)k * g->dim + d] - cell_center(g, d, c);
            dist += dx * dx;
        }
        it[k].key = key;
        it[k].dist = dist;
        it[k].idx = k;
    }
    qsort(it, (size_t)n, sizeof(dd_item), dd_cmp);
    int m = 0;
    for (int k = 0; k < n; ++k)
        if (k == 0 || it[k].key != it[k - 1].key) keep[m++] = it[k].idx;
    qsort(keep, (size_t)m, sizeof(int), int_cmp);
    *n_kept = m;
    free(it);
    free(cell);
    return rc;
}

long or_num_tiles(const or_desc *g) {
    long t = 1;
    for (int d = 0; d < g->dim; ++d) t *= (g->n[d] + g->tile[d] - 1) / g->tile[d];
    return t;
}

typedef struct { unsigned key; int idx; } kv_item;
static int kv_cmp(const void *a, const void *b) {
    const kv_item *x = (const kv_item *)a, *y = (const kv_item *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

/* Marker-to-cell bins: sort markers by (tile id, cell within tile, index);
 * tile_off[t] .. tile_off[t+1] is the range of tile t in `perm`. */
int or_bin(const or_desc *g, int n, const double *X, int *tile_off, int *perm, unsigned *keys) {
    int *cell = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1) * g->dim);
    int rc = or_owner_cells(g, n, X, cell);
    int T[3] = {1, 1, 1}, nt[3] = {1, 1, 1};
    for (int d = 0; d < g->dim; ++d) {
        T[d] = g->tile[d];
        nt[d] = (g->n[d] + T[d] - 1) / T[d];
    }
    unsigned cells_per_tile = (unsigned)(T[0] * T[1] * T[2]);
    kv_item *it = (kv_item *)malloc(sizeof(kv_item) * (size_t)(n > 0 ? n : 1));
    for (int k = 0; k < n; ++k) {
        int c[3] = {0, 0, 0};
        for (int d = 0; d < g->dim; ++d) c[d] = cell[(long)k * g->dim + d];
        unsigned tid = (unsigned)(c[0] / T[0] + nt[0] * (c[1] / T[1] + nt[1] * (c[2] / T[2])));
        unsigned cin = (unsigned)(c[0] % T[0] + T[0] * (c[1] % T[1] + T[1] * (c[2] % T[2])));
        it[k].key = tid * cells_per_tile + cin;
        it[k].idx = k;
    }
    qsort(it, (size_t)n, sizeof(kv_item), kv_cmp);
    long ntiles = or_num_tiles(g);
    for (long t = 0; t <= ntiles; ++t) tile_off[t] = 0;
    for (int k = 0; k < n; ++k) tile_off[it[k].key / cells_per_tile + 1] += 1;
    for (long t = 0; t < ntiles; ++t) tile_off[t + 1] += tile_off[t];
    for (int k = 0; k < n; ++k) {
        perm[k] = it[k].idx;
        if (keys) keys[k] = it[k].key;
    }
    free(it);
    free(cell);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* interpolation and spreading (Eqs. interp and force2)                      */
/* ------------------------------------------------------------------------ */

/* enumerate the 3^d support cells of a marker (owner cell +-1 per axis) */
static int support_cells(const or_desc *g, const double *X, int cells[27][3]) {
    int c0[3] = {0, 0, 0};
    for (int d = 0; d < g->dim; ++d) c0[d] = (int)floor((X[d] - g->lo[d]) / g->h);
    int m = 0;
    int oz_lo = g->dim == 3 ? -1 : 0, oz_hi = g->dim == 3 ? 1 : 0;
    for (int oz = oz_lo; oz <= oz_hi; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                cells[m][0] = c0[0] + ox;
                cells[m][1] = c0[1] + oy;
                cells[m][2] = c0[2] + oz;
                ++m;
            }
    return m;
}

static long lin_index(const or_desc *g, const int *c) {
    return c[0] + (long)g->n[0] * (c[1] + (long)g->n[1] * c[2]);
}

/* I[p]_k = sum_{j in D_k} p_j Phi_k(j)  (Eq. interp with Delta x = h^d) */
void or_interp(const or_desc *g, int ns, const double *X, const double *field, int nc,
               double *out) {
    long N = n_cells(g);
    for (int k = 0; k < ns; ++k) {
        const double *Xk = X + (long)k * g->dim;
        int cells[27][3];
        int m = support_cells(g, Xk, cells);
        for (int c = 0; c < nc; ++c) out[(long)k * nc + c] = 0.0;
        for (int s = 0; s < m; ++s) {
            double w = weight(g, Xk, cells[s]);
            long j = lin_index(g, cells[s]);
            for (int c = 0; c < nc; ++c) out[(long)k * nc + c] += w * field[(long)c * N + j];
        }
    }
}

/* the same sum taken over every cell of the grid (brute force, tiny grids) */
void or_interp_dense(const or_desc *g, int ns, const double *X, const double *field, int nc,
                     double *out) {
    long N = n_cells(g);
    int nz = g->dim == 3 ? g->n[2] : 1;
    for (int k = 0; k < ns; ++k) {
        for (int c = 0; c < nc; ++c) out[(long)k * nc + c] = 0.0;
        for (int i2 = 0; i2 < nz; ++i2)
            for (int i1 = 0; i1 < g->n[1]; ++i1)
                for (int i0 = 0; i0 < g->n[0]; ++i0) {
                    int cc[3] = {i0, i1, i2};
                    double w = weight(g, X + (long)k * g->dim, cc);
                    if (w == 0.0) continue;
                    long j = lin_index(g, cc);
                    for (int c = 0; c < nc; ++c) out[(long)k * nc + c] += w * field[(long)c * N + j];
                }
    }
}

/* r_j = sum_{k : j in D_k} R_k Phi_k(j) eps~_k  (Eq. force2, eps = h^d eps~) */
void or_spread(const or_desc *g, int ns, const double *X, const double *eps_t, const double *R,
               int nc, double *out) {
    long N = n_cells(g);
    memset(out, 0, sizeof(double) * (size_t)N * nc);
    for (int k = 0; k < ns; ++k) {
        const double *Xk = X + (long)k * g->dim;
        int cells[27][3];
        int m = support_cells(g, Xk, cells);
        for (int s = 0; s < m; ++s) {
            double w = weight(g, Xk, cells[s]);
            long j = lin_index(g, cells[s]);
            for (int c = 0; c < nc; ++c) out[(long)c * N + j] += R[(long)k * nc + c] * w * eps_t[k];
        }
    }
}

void or_spread_dense(const or_desc *g, int ns, const double *X, const double *eps_t,
                     const double *R, int nc, double *out) {
    long N = n_cells(g);
    int nz = g->dim == 3 ? g->n[2] : 1;
    for (int i2 = 0; i2 < nz; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                int cc[3] = {i0, i1, i2};
                long j = lin_index(g, cc);
                for (int c = 0; c < nc; ++c) out[(long)c * N + j] = 0.0;
                for (int k = 0; k < ns; ++k) {
                    double w = weight(g, X + (long)k * g->dim, cc);
                    if (w == 0.0) continue;
                    for (int c = 0; c < nc; ++c) out[(long)c * N + j] += R[(long)k * nc + c] * w * eps_t[k];
                }
            }
}

/* ------------------------------------------------------------------------ */
/* Lagrangian quadrature: A~ eps~ = 1 (Sec. 2.2)                             */
/* ------------------------------------------------------------------------ */

void or_assemble_A_dense(const or_desc *g, int ns, const double *X, double *A) {
    int nz = g->dim == 3 ? g->n[2] : 1;
    for (long q = 0; q < (long)ns * ns; ++q) A[q] = 0.0;
    for (int i2 = 0; i2 < nz; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                int cc[3] = {i0, i1, i2};
                for (int k = 0; k < ns; ++k) {
                    double wk = weight(g, X + (long)k * g->dim, cc);
                    if (wk == 0.0) continue;
                    for (int l = 0; l < ns; ++l) {
                        double wl = weight(g, X + (long)l * g->dim, cc);
                        A[(long)k * ns + l] += wk * wl;
                    }
                }
            }
}

/* sparse rows: A~_kl = sum over k's support cells of Phi_k Phi_l, kept when
 * the owner cells of k and l are within two cells on every axis (otherwise
 * the supports are disjoint). */
typedef struct { int *ptr; int *col; double *val; } or_csr;

static void assemble_sparse(const or_desc *g, int ns, const double *X, or_csr *A) {
    int *cell = (int *)malloc(sizeof(int) * (size_t)(ns > 0 ? ns : 1) * g->dim);
    or_owner_cells(g, ns, X, cell);
    int *cnt = (int *)calloc((size_t)ns + 1, sizeof(int));
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 16)
    for (int k = 0; k < ns; ++k) {
        int c = 0;
        for (int l = 0; l < ns; ++l) {
            int near = 1;
            for (int d = 0; d < g->dim; ++d)
                if (abs(cell[(long)k * g->dim + d] - cell[(long)l * g->dim + d]) > 2) near = 0;
            c += near;
        }
        cnt[k + 1] = c;
    }
    A->ptr = (int *)malloc(sizeof(int) * ((size_t)ns + 1));
    A->ptr[0] = 0;
    for (int k = 0; k < ns; ++k) A->ptr[k + 1] = A->ptr[k] + cnt[k + 1];
    A->col = (int *)malloc(sizeof(int) * (size_t)(A->ptr[ns] > 0 ? A->ptr[ns] : 1));
    A->val = (double *)malloc(sizeof(double) * (size_t)(A->ptr[ns] > 0 ? A->ptr[ns] : 1));
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 16)
    for (int k = 0; k < ns; ++k) {
        int p = A->ptr[k];
        int cells[27][3];
        int m = support_cells(g, X + (long)k * g->dim, cells);
        for (int l = 0; l < ns; ++l) {
            int near = 1;
            for (int d = 0; d < g->dim; ++d)
                if (abs(cell[(long)k * g->dim + d] - cell[(long)l * g->dim + d]) > 2) near = 0;
            if (!near) continue;
            double a = 0.0;
            for (int s = 0; s < m; ++s)
                a += weight(g, X + (long)k * g->dim, cells[s]) * weight(g, X + (long)l * g->dim, cells[s]);
            A->col[p] = l;
            A->val[p] = a;
            ++p;
        }
    }
    free(cnt);
    free(cell);
}

static void csr_mv(const or_csr *A, int ns, const double *x, double *y) {
    for (int k = 0; k < ns; ++k) {
        double s = 0.0;
        for (int p = A->ptr[k]; p < A->ptr[k + 1]; ++p) s += A->val[p] * x[A->col[p]];
        y[k] = s;
    }
}

/* Jacobi-preconditioned conjugate gradients on A~ eps~ = 1; stops when the
 * true residual max|1 - A~ eps~| <= tol.  Returns 0, or -2 on no convergence
 * within maxit iterations.  warm != 0 starts from the given eps_t. */
int or_quadrature(const or_desc *g, int ns, const double *X, double *eps_t, double tol,
                  int maxit, int warm, int *iters, double *resid) {
    if (ns <= 0) { if (iters) *iters = 0; if (resid) *resid = 0.0; return 0; }
    or_csr A;
    assemble_sparse(g, ns, X, &A);
    double *diag = (double *)malloc(sizeof(double) * ns);
    for (int k = 0; k < ns; ++k) {
        diag[k] = 0.0;
        for (int p = A.ptr[k]; p < A.ptr[k + 1]; ++p)
            if (A.col[p] == k) diag[k] = A.val[p];
    }
    double *x = eps_t, *r = malloc(sizeof(double) * ns), *z = malloc(sizeof(double) * ns);
    double *p = malloc(sizeof(double) * ns), *q = malloc(sizeof(double) * ns);
    if (!warm)
        for (int k = 0; k < ns; ++k) x[k] = 0.0;
    int it = 0, rc = -2;
    double rmax = 0.0;
    for (int restart = 0; restart < 50 && it < maxit; ++restart) {
        /* true residual */
        csr_mv(&A, ns, x, q);
        rmax = 0.0;
        for (int k = 0; k < ns; ++k) {
            r[k] = 1.0 - q[k];
            if (fabs(r[k]) > rmax) rmax = fabs(r[k]);
        }
        if (rmax <= tol) { rc = 0; break; }
        double rz = 0.0;
        for (int k = 0; k < ns; ++k) { z[k] = r[k] / diag[k]; p[k] = z[k]; rz += r[k] * z[k]; }
        for (; it < maxit; ++it) {
            csr_mv(&A, ns, p, q);
            double pq = 0.0;
            for (int k = 0; k < ns; ++k) pq += p[k] * q[k];
            double alpha = rz / pq;
            double rm = 0.0;
            for (int k = 0; k < ns; ++k) {
                x[k] += alpha * p[k];
                r[k] -= alpha * q[k];
                if (fabs(r[k]) > rm) rm = fabs(r[k]);
            }
            if (rm <= tol) { ++it; break; }
            double rz_new = 0.0;
            for (int k = 0; k < ns; ++k) { z[k] = r[k] / diag[k]; rz_new += r[k] * z[k]; }
            double beta = rz_new / rz;
            rz = rz_new;
            for (int k = 0; k < ns; ++k) p[k] = z[k] + beta * p[k];
        }
    }
    if (rc != 0) {
        csr_mv(&A, ns, x, q);
        rmax = 0.0;
        for (int k = 0; k < ns; ++k)
            if (fabs(1.0 - q[k]) > rmax) rmax = fabs(1.0 - q[k]);
        if (rmax <= tol) rc = 0;
    }
    if (iters) *iters = it;
    if (resid) *resid = rmax;
    free(r); free(z); free(p); free(q); free(diag);
    free(A.ptr); free(A.col); free(A.val);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* fluid: ghost cells, primitives, fluxes, SSP-RK2                           */
/* ------------------------------------------------------------------------ */

/* padded storage: 2 ghost layers on every axis of the grid's dimension */
static void pad_dims(const or_desc *g, int P[3]) {
    for (int d = 0; d < 3; ++d) P[d] = d < g->dim ? g->n[d] + 4 : 1;
}

/* map an index along one axis to its interior source under the face BCs */
static int map_axis(const or_desc *g, int d, int idx, int *flip, int *freestream) {
    int n = g->n[d];
    if (idx >= 0 && idx < n) return idx;
    int bc = idx < 0 ? g->bc[2 * d] : g->bc[2 * d + 1];
    switch (bc) {
    case OR_BC_FREESTREAM: *freestream = 1; return idx < 0 ? 0 : n - 1;
    case OR_BC_ZEROGRAD: return idx < 0 ? 0 : n - 1;
    case OR_BC_SLIP: *flip ^= (1 << d); return idx < 0 ? -1 - idx : 2 * n - 1 - idx;
    default: return ((idx % n) + n) % n; /* periodic */
    }
}

static void freestream_state(const or_desc *g, double *u) {
    double p = 1.0 / (g->gamma * g->Mach * g->Mach);
    u[0] = 1.0;
    for (int d = 0; d < g->dim; ++d) u[1 + d] = d == 0 ? 1.0 : 0.0;
    u[g->dim + 1] = p / (g->gamma - 1.0) + 0.5;
}

void or_fill_ghosts(const or_desc *g, const double *U, double *Pd) {
    int P[3];
    pad_dims(g, P);
    long Np = (long)P[0] * P[1] * P[2], N = n_cells(g);
    int nc = n_comp(g);
    double Uinf[5];
    freestream_state(g, Uinf);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long q = 0; q < Np; ++q) {
        int pq[3] = {(int)(q % P[0]), (int)((q / P[0]) % P[1]), (int)(q / ((long)P[0] * P[1]))};
        int src[3] = {0, 0, 0}, flip = 0, fs = 0;
        for (int d = 0; d < g->dim; ++d) src[d] = map_axis(g, d, pq[d] - 2, &flip, &fs);
        if (fs) {
            for (int c = 0; c < nc; ++c) Pd[c * Np + q] = Uinf[c];
            continue;
        }
        long j = lin_index(g, src);
        for (int c = 0; c < nc; ++c) {
            double v = U[(long)c * N + j];
            if (c >= 1 && c <= g->dim && (flip & (1 << (c - 1)))) v = -v;
            Pd[c * Np + q] = v;
        }
    }
}

/* primitives (rho, u.., p) and temperature of one conserved vector */
static void to_primitive(const or_desc *g, const double *u, double *w, double *T) {
    double rho = u[0], ke = 0.0;
    w[0] = rho;
    for (int d = 0; d < g->dim; ++d) {
        w[1 + d] = u[1 + d] / rho;
        ke += w[1 + d] * w[1 + d];
    }
    double p = (g->gamma - 1.0) * (u[g->dim + 1] - 0.5 * rho * ke);
    w[g->dim + 1] = p;
    *T = p / (rho * gas_R(g));
}

static double van_leer(double a, double b) {
    double ab = a * b;
    if (ab <= 0.0) return 0.0;
    return 2.0 * ab / (a + b);
}

/* Euler flux along axis d of a primitive state, with its conserved vector */
static void euler_flux(const or_desc *g, const double *w, int d, double *U, double *F) {
    int dim = g->dim;
    double rho = w[0], p = w[dim + 1], ke = 0.0;
    for (int m = 0; m < dim; ++m) ke += w[1 + m] * w[1 + m];
    double E = p / (g->gamma - 1.0) + 0.5 * rho * ke;
    double un = w[1 + d];
    U[0] = rho;
    F[0] = rho * un;
    for (int m = 0; m < dim; ++m) {
        U[1 + m] = rho * w[1 + m];
        F[1 + m] = rho * w[1 + m] * un + (m == d ? p : 0.0);
    }
    U[dim + 1] = E;
    F[dim + 1] = (E + p) * un;
}

/* numerical flux through the face between padded cells a and a + s (axis d):
 * Rusanov flux of the MUSCL/van Leer states minus the viscous and heat flux */
static void face_flux(const or_desc *g, const double *W, const double *Tc, long Np, long a,
                      int d, const long *stride, double *Fhat) {
    int dim = g->dim, nw = dim + 2;
    long s = stride[d], b = a + s;
    double wl[5], wr[5];
    for (int m = 0; m < nw; ++m) {
        double wa = W[m * Np + a], wb = W[m * Np + b];
        double wam = W[m * Np + a - s], wbp = W[m * Np + b + s];
        wl[m] = wa + 0.5 * van_leer(wa - wam, wb - wa);
        wr[m] = wb - 0.5 * van_leer(wb - wa, wbp - wb);
    }
    double UL[5], UR[5], FL[5], FR[5];
    euler_flux(g, wl, d, UL, FL);
    euler_flux(g, wr, d, UR, FR);
    double cl = sqrt(g->gamma * wl[dim + 1] / wl[0]);
    double cr = sqrt(g->gamma * wr[dim + 1] / wr[0]);
    double sl = fabs(wl[1 + d]) + cl, sr = fabs(wr[1 + d]) + cr;
    double smax = sl > sr ? sl : sr;
    for (int m = 0; m < nw; ++m) Fhat[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * smax * (UR[m] - UL[m]);

    if (g->Re <= 0.0) return;
    /* viscous stress and heat flux (Sec. 2.1), face values from the two cells */
    double h = g->h;
    double Tf = 0.5 * (Tc[a] + Tc[b]);
    double mu = viscosity(g, Tf);
    double lam = mu * gas_cp(g) / g->Pr;
    double grad[3][3]; /* grad[m][e] = d u_m / d x_e at the face */
    for (int m = 0; m < dim; ++m) {
        const double *um = W + (long)(1 + m) * Np;
        for (int e = 0; e < dim; ++e) {
            if (e == d) {
                grad[m][e] = (um[b] - um[a]) / h;
            } else {
                long t = stride[e];
                grad[m][e] = (um[a + t] - um[a - t] + um[b + t] - um[b - t]) / (4.0 * h);
            }
        }
    }
    double div = 0.0;
    for (int m = 0; m < dim; ++m) div += grad[m][m];
    double work = 0.0;
    for (int m = 0; m < dim; ++m) {
        double tau = mu * (grad[d][m] + grad[m][d]) - (m == d ? (2.0 / 3.0) * mu * div : 0.0);
        double uf = 0.5 * (W[(long)(1 + m) * Np + a] + W[(long)(1 + m) * Np + b]);
        Fhat[1 + m] -= tau;
        work += uf * tau;
    }
    double dTdn = (Tc[b] - Tc[a]) / h;
    Fhat[dim + 1] -= work + lam * dTdn;
}

/* L(U) = -(1/h) sum_d (Fhat_{i+1/2} - Fhat_{i-1/2}) on every interior cell */
void or_rhs(const or_desc *g, const double *U, double *L) {
    int P[3];
    pad_dims(g, P);
    long Np = (long)P[0] * P[1] * P[2], N = n_cells(g);
    int nc = n_comp(g);
    double *Pd = (double *)malloc(sizeof(double) * (size_t)Np * nc);
    double *W = (double *)malloc(sizeof(double) * (size_t)Np * nc);
    double *Tc = (double *)malloc(sizeof(double) * (size_t)Np);
    or_fill_ghosts(g, U, Pd);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long q = 0; q < Np; ++q) {
        double u[5] = {0, 0, 0, 0, 0}, w[5], T;
        for (int c = 0; c < nc; ++c) u[c] = Pd[c * Np + q];
        to_primitive(g, u, w, &T);
        for (int c = 0; c < nc; ++c) W[c * Np + q] = w[c];
        Tc[q] = T;
    }
    long stride[3] = {1, P[0], (long)P[0] * P[1]};
    int nz = g->dim == 3 ? g->n[2] : 1;
#pragma omp parallel for num_threads(g_threads) schedule(static) collapse(2)
    for (int i2 = 0; i2 < nz; ++i2)
        for (int i1 = 0; i1 < g->n[1]; ++i1)
            for (int i0 = 0; i0 < g->n[0]; ++i0) {
                long a = (i0 + 2) + stride[1] * (i1 + 2) + stride[2] * (g->dim == 3 ? i2 + 2 : 0);
                long j = i0 + (long)g->n[0] * (i1 + (long)g->n[1] * i2);
                double acc[5] = {0, 0, 0, 0, 0};
                for (int d = 0; d < g->dim; ++d) {
                    double Fhi[5], Flo[5];
                    face_flux(g, W, Tc, Np, a, d, stride, Fhi);
                    face_flux(g, W, Tc, Np, a - stride[d], d, stride, Flo);
                    for (int c = 0; c < nc; ++c) acc[c] -= (Fhi[c] - Flo[c]) / g->h;
                }
                for (int c = 0; c < nc; ++c) L[(long)c * N + j] = acc[c];
            }
    free(Pd);
    free(W);
    free(Tc);
}

/* explicit step size: dt = CFL / max_j s_j, s_j = sum_d (|u_d| + c)/h
 * + sum_d 2 nu_j / h^2, nu_j = max(4/3, gamma/Pr) mu(T_j) / rho_j */
double or_dt(const or_desc *g, const double *U) {
    long N = n_cells(g);
    int nc = n_comp(g);
    double smax = 0.0;
    double kvisc = (4.0 / 3.0) > (g->gamma / g->Pr) ? (4.0 / 3.0) : (g->gamma / g->Pr);
#pragma omp parallel for num_threads(g_threads) schedule(static) reduction(max : smax)
    for (long j = 0; j < N; ++j) {
        double u[5] = {0, 0, 0, 0, 0}, w[5], T;
        for (int c = 0; c < nc; ++c) u[c] = U[(long)c * N + j];
        to_primitive(g, u, w, &T);
        double c = sqrt(g->gamma * w[g->dim + 1] / w[0]);
        double nu = kvisc * viscosity(g, T) / w[0];
        double s = 0.0;
        for (int d = 0; d < g->dim; ++d) s += (fabs(w[1 + d]) + c) / g->h + 2.0 * nu / (g->h * g->h);
        if (!(s <= smax)) smax = s; /* NaN propagates */
    }
    return g->cfl / smax;
}

/* SSP-RK2 predictor without sources (App. B step 1):
 * U1 = U + dt L(U); U* = U/2 + (U1 + dt L(U1))/2.  Returns dt. */
double or_fluid_predictor(const or_desc *g, const double *U, double *Ustar, double dt_fixed) {
    long N = n_cells(g), M = N * n_comp(g);
    double dt = dt_fixed > 0.0 ? dt_fixed : or_dt(g, U);
    double *L = (double *)malloc(sizeof(double) * (size_t)M);
    double *U1 = (double *)malloc(sizeof(double) * (size_t)M);
    or_rhs(g, U, L);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long q = 0; q < M; ++q) U1[q] = U[q] + dt * L[q];
    or_rhs(g, U1, L);
#pragma omp parallel for num_threads(g_threads) schedule(static)
    for (long q = 0; q < M; ++q) Ustar[q] = 0.5 * U[q] + 0.5 * (U1[q] + dt * L[q]);
    free(L);
    free(U1);
    return dt;
}

/* ------------------------------------------------------------------------ */
/* direct forcing (Eqs. forceMomentum, corr3.8) and its application (App. B) */
/* ------------------------------------------------------------------------ */

/* rho_L = I[rho*], (rho_L U)bar = I[(rho u)*], (rho_L Theta)^l c_v = I[(rho e)*];
 * F_k = a_s (rho_L U_b - I[rho u]), Q_k = a_e (rho_L c_v T_w - I[rho e]) with
 * a_s = a_e = 1/dt.  Outputs rhoL (ns), G = dt F (ns*dim) and H = dt Q (ns):
 * the explicit update adds dt f = S[dt F], so dt cancels from the state. */
void or_interp_force(const or_desc *g, int ns, const double *X, const double *Ub,
                     const double *Tw, const double *Ustar, double *rhoL, double *G, double *H) {
    long N = n_cells(g);
    int dim = g->dim, nf = dim + 2;
    double *fields = (double *)malloc(sizeof(double) * (size_t)N * nf);
    for (long j = 0; j < N; ++j) {
        double rho = Ustar[j], ke = 0.0;
        fields[j] = rho;
        for (int d = 0; d < dim; ++d) {
            double m = Ustar[(long)(1 + d) * N + j];
            fields[(long)(1 + d) * N + j] = m;
            ke += m * m;
        }
        fields[(long)(dim + 1) * N + j] = Ustar[(long)(dim + 1) * N + j] - 0.5 * ke / rho;
    }
    double *I = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * nf);
    or_interp(g, ns, X, fields, nf, I);
    double cv = gas_cv(g);
    for (int k = 0; k < ns; ++k) {
        double rk = I[(long)k * nf];
        rhoL[k] = rk;
        for (int d = 0; d < dim; ++d) {
            double ub = Ub ? Ub[(long)k * dim + d] : 0.0;
            G[(long)k * dim + d] = rk * ub - I[(long)k * nf + 1 + d];
        }
        H[k] = rk * cv * Tw[k] - I[(long)k * nf + dim + 1];
    }
    free(I);
    free(fields);
}

/* cells in the union of the marker supports D_k */
int or_band_mask(const or_desc *g, int ns, const double *X, unsigned char *mask) {
    long N = n_cells(g);
    memset(mask, 0, (size_t)N);
    int cnt = 0;
    for (int k = 0; k < ns; ++k) {
        int cells[27][3];
        int m = support_cells(g, X + (long)k * g->dim, cells);
        for (int s = 0; s < m; ++s) {
            long j = lin_index(g, cells[s]);
            if (!mask[j]) { mask[j] = 1; ++cnt; }
        }
    }
    return cnt;
}

/* App. B step 3 for an explicit scheme: (rho u)^{n+1} = (rho u)* + dt f,
 * (rho e)^{n+1} = (rho e)* + dt q, rho unchanged, rho E rebuilt from the new
 * momentum (energy reading 0) or rho E += dt q (reading 1).  Applied on the
 * band cells only.  G = dt F and H = dt Q per marker, so dt f = S[G]. */
void or_spread_apply(const or_desc *g, int ns, const double *X, const double *eps_t,
                     const double *G, const double *H, double *U) {
    long N = n_cells(g);
    int dim = g->dim, nr = dim + 1;
    double *R = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * nr);
    for (int k = 0; k < ns; ++k) {
        for (int d = 0; d < dim; ++d) R[(long)k * nr + d] = G[(long)k * dim + d];
        R[(long)k * nr + dim] = H[k];
    }
    double *r = (double *)malloc(sizeof(double) * (size_t)N * nr);
    or_spread(g, ns, X, eps_t, R, nr, r);
    unsigned char *mask = (unsigned char *)malloc((size_t)N);
    or_band_mask(g, ns, X, mask);
    for (long j = 0; j < N; ++j) {
        if (!mask[j]) continue;
        double rho = U[j], ke0 = 0.0, ke1 = 0.0;
        for (int d = 0; d < dim; ++d) {
            double m0 = U[(long)(1 + d) * N + j];
            double m1 = m0 + r[(long)d * N + j];
            ke0 += m0 * m0;
            ke1 += m1 * m1;
            U[(long)(1 + d) * N + j] = m1;
        }
        double E = U[(long)(dim + 1) * N + j];
        double q = r[(long)dim * N + j];
        /* positivity reading (the paper is silent): the heat source removes
         * at most HEAT_SOURCE_CAP of the cell's internal energy in one step,
         * dt q >= -HEAT_SOURCE_CAP rho e*.  Inactive unless a cold wall
         * would otherwise drive a forced cell to non-positive pressure. */
        double rhoe0 = E - 0.5 * ke0 / rho;
        if (q < -HEAT_SOURCE_CAP * rhoe0) q = -HEAT_SOURCE_CAP * rhoe0;
        if (g->energy_reading == 1)
            U[(long)(dim + 1) * N + j] = E + q;
        else
            U[(long)(dim + 1) * N + j] = (E - 0.5 * ke0 / rho + q) + 0.5 * ke1 / rho;
    }
    free(mask);
    free(r);
    free(R);
}

/* One IBM step: predictor (f = q = 0), interpolate and force, spread and
 * re-solve with the sources (App. B).  Returns dt; G, H (dt F, dt Q) and
 * rhoL per marker are returned for diagnostics.
 *
 * Variant forcing_per_stage = 1: the direct forcing is applied after EACH
 * SSP-RK2 stage instead of once after the predictor:
 *   U1 = U + dt L(U);            U1 <- forced(U1)   (sources G1, H1)
 *   U* = U/2 + (U1 + dt L(U1))/2; U^{n+1} = forced(U*) (sources G2, H2).
 * The forcing of the first stage reaches U^{n+1} with weight 1/2, so the
 * sources of the step (what the body exerts over dt) are G = G1/2 + G2 and
 * H = H1/2 + H2; rhoL is the second stage's. */
double or_step(const or_desc *g, int ns, const double *X, const double *Ub, const double *Tw,
               const double *eps_t, const double *U, double *Unew, double dt_fixed,
               double *G, double *H, double *rhoL) {
    if (!g->forcing_per_stage || ns == 0) {
        double dt = or_fluid_predictor(g, U, Unew, dt_fixed);
        if (ns > 0) {
            or_interp_force(g, ns, X, Ub, Tw, Unew, rhoL, G, H);
            or_spread_apply(g, ns, X, eps_t, G, H, Unew);
        }
        return dt;
    }
    long N = n_cells(g), M = N * n_comp(g);
    int dim = g->dim;
    double dt = dt_fixed > 0.0 ? dt_fixed : or_dt(g, U);
    double *L = (double *)malloc(sizeof(double) * (size_t)M);
    double *U1 = (double *)malloc(sizeof(double) * (size_t)M);
    double *G1 = (double *)malloc(sizeof(double) * (size_t)ns * dim);
    double *H1 = (double *)malloc(sizeof(double) * (size_t)ns);
    double *r1 = (double *)malloc(sizeof(double) * (size_t)ns);
    or_rhs(g, U, L);
    for (long q = 0; q < M; ++q) U1[q] = U[q] + dt * L[q];
    or_interp_force(g, ns, X, Ub, Tw, U1, r1, G1, H1);
    or_spread_apply(g, ns, X, eps_t, G1, H1, U1);
    or_rhs(g, U1, L);
    for (long q = 0; q < M; ++q) Unew[q] = 0.5 * U[q] + 0.5 * (U1[q] + dt * L[q]);
    or_interp_force(g, ns, X, Ub, Tw, Unew, rhoL, G, H);
    or_spread_apply(g, ns, X, eps_t, G, H, Unew);
    for (long k = 0; k < (long)ns * dim; ++k) G[k] += 0.5 * G1[k];
    for (int k = 0; k < ns; ++k) H[k] += 0.5 * H1[k];
    free(L);
    free(U1);
    free(G1);
    free(H1);
    free(r1);
    return dt;
}

/* Body force and heat rate from the markers (Sec. 3.1, Eq. Bulk):
 * F_body = -h^d sum_k eps~_k F_k, Qdot = h^d sum_k eps~_k Q_k with F = G/dt,
 * Q = H/dt.  C = 2F/(rho U^2 Lref), Lref = D (2D) or pi D^2/4 (3D);
 * Nu = Qdot D / (lambda_inf A_s (mean T_w - 1)), A_s = pi D or pi D^2. */
void or_forces(const or_desc *g, int ns, const double *eps_t, const double *G, const double *H,
               const double *Tw, double dt, double *force, double *heat, double *Cd, double *Cl,
               double *Nu) {
    int dim = g->dim;
    double hd = pow(g->h, dim);
    double f[3] = {0, 0, 0}, q = 0.0, tw = 0.0;
    for (int k = 0; k < ns; ++k) {
        for (int d = 0; d < dim; ++d) f[d] += eps_t[k] * (G[(long)k * dim + d] / dt);
        q += eps_t[k] * (H[k] / dt);
        tw += Tw[k];
    }
    for (int d = 0; d < 3; ++d) force[d] = d < dim ? -hd * f[d] : 0.0;
    *heat = hd * q;
    double pi = 3.14159265358979323846;
    double lref = dim == 2 ? g->D : pi * g->D * g->D / 4.0;
    *Cd = 2.0 * force[0] / lref;
    *Cl = 2.0 * force[1] / lref;
    double As = dim == 2 ? pi * g->D : pi * g->D * g->D;
    double lam_inf = g->Re > 0.0 ? (1.0 / g->Re) * gas_cp(g) / g->Pr : 0.0;
    double dT = (ns > 0 ? tw / ns : 0.0) - 1.0;
    *Nu = (lam_inf > 0.0 && dT != 0.0) ? (*heat) * g->D / (lam_inf * As * dT) : NAN;
}

/* Prescribed oscillation (Sec. 5): X = X0 + amp sin(2 pi f t) e_axis,
 * U_b = dX/dt. */
void or_motion(int ns, int dim, const double *X0, double amp, double freq, int axis, double t,
               double *X, double *Ub) {
    double pi = 3.14159265358979323846;
    double s = amp * sin(2.0 * pi * freq * t);
    double v = amp * 2.0 * pi * freq * cos(2.0 * pi * freq * t);
    for (int k = 0; k < ns; ++k)
        for (int d = 0; d < dim; ++d) {
            X[(long)k * dim + d] = X0[(long)k * dim + d] + (d == axis ? s : 0.0);
            Ub[(long)k * dim + d] = d == axis ? v : 0.0;
        }
}
