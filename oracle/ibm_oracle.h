/*
 * Oracle for the discrete-forcing IBM step of Riahi, Goncalves da Silva and
 * Meldi (arXiv 2301.09349): a plain, slow, FP64 CPU restatement of what the
 * GPU path computes.  TEST INFRASTRUCTURE ONLY: it is loaded by the test
 * suite, by the smoke check and by the benchmark's CPU-baseline leg, and by
 * nothing on the product path.  It shares no code, header or constant with
 * the CUDA library.
 *
 * Every function works on host arrays.  Conserved state arrays are
 * component-major: ncomp planes of N cells, cell (i,j,k) at i + nx*(j + ny*k),
 * ncomp = dim + 2, components (rho, rho u, rho v, [rho w], rho E).
 */
#ifndef IBM_ORACLE_H
#define IBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;          /* 2 or 3 */
    int n[3];         /* cells per axis (n[2] = 1 in 2D) */
    double lo[3];     /* lower domain corner */
    double h;         /* uniform spacing */
    double gamma, Pr, Re, Mach, S, cfl;  /* Re <= 0: inviscid */
    int bc[6];        /* x-, x+, y-, y+, z-, z+ : 0 freestream 1 zerograd 2 slip 3 periodic */
    int tile[3];      /* binning tile (cells per axis) */
    double D;         /* reference length */
    int energy_reading; /* 0: forcing on internal energy (default); 1: on total energy */
    int forcing_per_stage; /* 0: forcing once after the predictor (default); 1: after each stage */
} or_desc;

/* --- regularised delta (Sec. 2.2) --- */
double or_phi(double r);
void   or_phi_many(const double *r, long n, double *out);

/* --- markers: owner cells, dedup (Sec. 3.1), binning --- */
int  or_owner_cells(const or_desc *g, int n, const double *X, int *cell /* n*dim */);
int  or_dedup(const or_desc *g, int n, const double *X, int *keep /* n */, int *n_kept);
int  or_bin(const or_desc *g, int n, const double *X, int *tile_off /* n_tiles+1 */,
            int *perm /* n */, unsigned *keys /* n, sorted */);
long or_num_tiles(const or_desc *g);

/* --- interpolation I and spreading S (Eqs. interp, force2) --- */
void or_interp(const or_desc *g, int ns, const double *X, const double *field, int nc,
               double *out /* ns*nc */);
void or_interp_dense(const or_desc *g, int ns, const double *X, const double *field, int nc,
                     double *out);
void or_spread(const or_desc *g, int ns, const double *X, const double *eps_t, const double *R,
               int nc, double *out /* nc*N */);
void or_spread_dense(const or_desc *g, int ns, const double *X, const double *eps_t,
                     const double *R, int nc, double *out);

/* --- Lagrangian quadrature A eps = 1 --- */
void or_assemble_A_dense(const or_desc *g, int ns, const double *X, double *A /* ns*ns */);
int  or_quadrature(const or_desc *g, int ns, const double *X, double *eps_t, double tol,
                   int maxit, int warm, int *iters, double *resid);

/* --- fluid (Sec. 2.1 equations; explicit FV scheme) --- */
void   or_set_threads(int nthreads);
int    or_get_threads(void);
void   or_rhs(const or_desc *g, const double *U, double *L);
double or_dt(const or_desc *g, const double *U);
void   or_fill_ghosts(const or_desc *g, const double *U, double *P /* padded */);
double or_fluid_predictor(const or_desc *g, const double *U, double *Ustar, double dt_fixed);

/* --- forcing (Eqs. forceMomentum, corr3.8; App. B) --- */
void or_interp_force(const or_desc *g, int ns, const double *X, const double *Ub,
                     const double *Tw, const double *Ustar, double *rhoL /* ns */,
                     double *G /* ns*dim */, double *H /* ns */);
void or_spread_apply(const or_desc *g, int ns, const double *X, const double *eps_t,
                     const double *G, const double *H, double *U /* in/out */);
int  or_band_mask(const or_desc *g, int ns, const double *X, unsigned char *mask /* N */);

/* --- one full IBM step: predictor, interpolate/force, spread/apply --- */
double or_step(const or_desc *g, int ns, const double *X, const double *Ub, const double *Tw,
               const double *eps_t, const double *U, double *Unew, double dt_fixed,
               double *G, double *H, double *rhoL);

/* --- body force and heat rate (Eq. Bulk and its Nusselt analogue) --- */
void or_forces(const or_desc *g, int ns, const double *eps_t, const double *G, const double *H,
               const double *Tw, double dt, double *force /* 3 */, double *heat,
               double *Cd, double *Cl, double *Nu);

/* --- prescribed motion (Sec. 5) --- */
void or_motion(int ns, int dim, const double *X0, double amp, double freq, int axis, double t,
               double *X, double *Ub);

#ifdef __cplusplus
}
#endif
#endif
