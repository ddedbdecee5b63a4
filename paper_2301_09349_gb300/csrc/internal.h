// Host-side declarations shared by the library's translation units
// (internal; the public ABI is include/ibm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ibmk {

// Opt `func` in to `smem` bytes of dynamic shared memory on the current
// device (and, with carveout >= 0, set its preferred shared-memory carveout
// in percent).  Kernel attributes belong to one device, so the applied limit
// is recorded per (kernel, device ordinal) under a mutex (api.cu); requests of
// at most 48 KB need no opt-in and return at once.
cudaError_t func_smem_attr(const void *func, size_t smem, int carveout = -1);

// ---- fluid stages (flux.cu, flux_zm.cu) ------------------------------------
// Stage 1: out = U1 = U + dt L(U), dt = dt_fixed if > 0 else *dt.
// Stage 2: out = U* = Un/2 + (U1 + dt L(U1))/2; per-CTA maximum of the
//          step-size rate s_j(U*) over the cells the forcing leaves alone
//          (band_bits clear) into blockmax[].
// dt_init: *dt = cfl / max_j s_j(U) over every cell (last-block reduction).
// The next step's dt = cfl / max(stage-2 maxima, band-cell maxima after the
// forcing) is formed by the finish kernel, so dt always follows from the
// state at the start of the step.
struct FluidBuffers {
    double *blockmax;            // per-CTA maxima (stage 2, dt_init)
    unsigned *counter;           // last-block tickets (zero between launches): [0] dt_init,
                                 // [1] the finish kernel
    double *dt;                  // device step size of the next step
    int *err;                    // device error word
    const unsigned *band_bits;   // one bit per cell changed by the forcing
};

constexpr int DT_CELLS_PER_CTA = 2048;   // dt_init: 256 threads x 8 cells

size_t fluid_stage_blocks(const GridParams &g, int fp_bytes);
size_t dt_init_blocks(const GridParams &g);
size_t fluid_blockmax_count(const GridParams &g, int fp_bytes);
cudaError_t launch_stage1(const GridParams &g, int fp_bytes, const void *U, void *U1,
                          const FluidBuffers &fb, double dt_fixed, cudaStream_t s);
cudaError_t launch_stage2(const GridParams &g, int fp_bytes, const void *Un, const void *U1,
                          void *out, const FluidBuffers &fb, double dt_fixed, cudaStream_t s);
// L(U) only, for the diagnostic ibm_rhs
cudaError_t launch_rhs(const GridParams &g, int fp_bytes, const void *U, void *L,
                       const FluidBuffers &fb, cudaStream_t s);
cudaError_t launch_dt_init(const GridParams &g, int fp_bytes, const void *U,
                           const FluidBuffers &fb, cudaStream_t s);
// the z-marching form used for 3D FP32 grids (flux_zm.cu); mode 0/1/2 as above
cudaError_t launch_zmarch(int mode, const GridParams &g, const void *Uin, const void *Un,
                          void *out, const FluidBuffers &fb, double dt_fixed, cudaStream_t s);
size_t zmarch_blocks(const GridParams &g);

// Step-size rate of one cell from its conserved state (DIM+2 values):
// s = sum_d (|u_d| + c)/h + 2 DIM nu / h^2, nu = max(4/3, gamma/Pr) mu(T)/rho.
// ok is cleared for a non-positive density or pressure or a non-finite s.
template <int DIM, typename T>
__device__ __forceinline__ T step_rate(const GridParams &g, const T *u, bool &ok);

// FP32 grids: single precision throughout, from the host-rounded constants.
template <int DIM>
__device__ __forceinline__ float step_rate_f(const GridParams &g, const float *u, bool &ok) {
    const FloatConsts &c = g.f;
    const float rho = u[0], inv = __fdividef(1.0f, rho);
    float ke = 0.0f, sabs = 0.0f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const float v = u[1 + d] * inv;
        ke += v * v;
        sabs += fabsf(v);
    }
    const float p = c.gm1 * (u[DIM + 1] - 0.5f * rho * ke);
    const float c2 = c.gamma * p * inv;
    const float snd = c2 * rsqrtf(c2);
    float mu = 0.0f;
    if (c.viscous) {
        const float Tt = p * inv * c.invR;
        mu = __fdividef(c.mu_inf * Tt * (Tt * rsqrtf(Tt)) * c.onepS, Tt + c.S);
    }
    const float s = (sabs + (float)DIM * snd) * c.inv_h +
                    (float)(2 * DIM) * (c.kvisc * mu * inv) * c.inv_h * c.inv_h;
    if (!(rho > 0.0f && p > 0.0f && s <= 3.0e38f)) ok = false;
    return s;
}
template <>
__device__ __forceinline__ float step_rate<3, float>(const GridParams &g, const float *u, bool &ok) {
    return step_rate_f<3>(g, u, ok);
}

template <int DIM, typename T>
__device__ __forceinline__ T step_rate_generic(const GridParams &g, const T *u, bool &ok) {
    const T rho = u[0];
    T ke = T(0), sabs = T(0);
    for (int d = 0; d < DIM; ++d) {
        const T v = u[1 + d] / rho;
        ke += v * v;
        sabs += v < T(0) ? -v : v;
    }
    const T p = (T)(g.gamma - 1.0) * (u[DIM + 1] - T(0.5) * rho * ke);
    const T c = sqrt((T)g.gamma * p / rho);
    T mu = T(0);
    if (g.mu_inf > 0.0) {
        const T Tt = p / (rho * (T)g.R), S = (T)g.S;
        mu = (T)g.mu_inf * Tt * sqrt(Tt) * (T(1) + S) / (Tt + S);
    }
    const T nu = (T)g.kvisc * mu / rho;
    const T s = (sabs + T(DIM) * c) * (T)g.inv_h + T(2 * DIM) * nu * (T)(g.inv_h * g.inv_h);
    if (!(rho > T(0) && p > T(0) && (double)s <= 1.0e300)) ok = false;
    return s;
}
template <>
__device__ __forceinline__ double step_rate<3, double>(const GridParams &g, const double *u, bool &ok) {
    return step_rate_generic<3, double>(g, u, ok);
}
template <>
__device__ __forceinline__ double step_rate<2, double>(const GridParams &g, const double *u, bool &ok) {
    return step_rate_generic<2, double>(g, u, ok);
}
template <>
__device__ __forceinline__ float step_rate<2, float>(const GridParams &g, const float *u, bool &ok) {
    return step_rate_f<2>(g, u, ok);
}

__device__ __forceinline__ bool band_bit(const unsigned *bits, long long j) {
    return (__ldg(bits + (j >> 5)) >> (j & 31)) & 1u;
}

// ---- markers (markers.cu) --------------------------------------------------
// One forced cell of the precomputed spreading operator of static markers:
// its global index and its run [start, start + n) of (marker, weight)
// entries.
struct SpreadCell {
    long long j;
    int start, n;
};

struct MarkerBuffers {
    int ns;                  // kept markers
    double *X0, *X;          // ns*dim positions at t = 0 and now
    double *Ub0, *Ub;        // ns*dim body velocity (prescribed part, current)
    double *Tw;              // ns wall temperatures
    double *eps;             // ns quadrature weights eps~
    int *cell;               // ns*3 owner cells floor((X - lo)/h) (bins kernel)
    double *frac_d;          // ns*3 offsets (X - lo)/h - cell, in [0, 1)
    float *frac_f;           // the same offsets in single precision
    double *wphi;            // ns*9: phi((i - 1) + 1/2 - frac_d) for i = 0..2 per axis, the
                             // marker's 1D weights at its owner cell and the two beside it
    double *rhoL, *G, *H;    // last forcing: rho_L, dt*F (ns*dim), dt*Q
    double *cp;              // ns surface pressure coefficients (ibm_surface_pressure)
    unsigned *keys[2];       // radix-sort ping-pong
    int *perm[2];
    int sorted;              // which of keys/perm holds the sorted order
    int *tile_off;           // n_tiles + 1
    int *occ_flag, *band_flag;  // n_tiles
    int *occ_list, *band_list;  // n_tiles
    int *counts;             // [0] occupied tiles, [1] band tiles, [2] operator cells,
                             // [3] operator entries
    double *sums;            // [0..2] sum eps~ G, [3] sum eps~ H, [4] dt of those sums;
                             // [8..11] the first stage's sums (forcing per stage)
    double *bandmax;         // per-CTA step-size maxima of the spread kernel
    double *finpart;         // kFinishCtas x 5 partials of the split finish kernel
    void *gs;                // ns x 4 eps~-scaled forcing in the field precision: eps~ G_d
                             // (d < dim), eps~ H at [3] (written by the interpolation)
    SpreadCell *sp_cell;     // forced cells of the spreading operator (counts[2] of them)
    int *sp_k;               // marker of each operator entry (counts[3] of them)
    void *sp_w;              // weight of each entry, field precision
    int sp_cap;              // capacity of cells and of entries: 3^dim x marker capacity
    int sp_ready;            // the operator matches the current (static) markers
    unsigned *band_bits;     // one bit per cell inside some marker support
    double *t;               // simulated time
    long long *steps;        // step counter
    int *err;
};

cudaError_t launch_motion(const GridParams &g, const MarkerBuffers &m, double amp, double freq,
                          int axis, const double *dt, double dt_fixed, cudaStream_t s);
// the per-step marker pipeline of a moving body with at most kSmallRebuildNs
// markers in one launch (motion, bins, forced cells, tile lists); the
// quadrature follows separately
constexpr int kSmallRebuildNs = 512;
cudaError_t launch_small_rebuild(const GridParams &g, MarkerBuffers &m, double amp, double freq,
                                 int axis, const double *dt, double dt_fixed, cudaStream_t s);
// forced-cell bits and band-tile flags scattered from the markers' supports,
// then the ordered occupied and band tile lists (after launch_bin)
cudaError_t launch_band_mask(const GridParams &g, const MarkerBuffers &m, cudaStream_t s);
cudaError_t launch_bin(const GridParams &g, MarkerBuffers &m, cudaStream_t s);
cudaError_t launch_interp_force(const GridParams &g, int fp_bytes, const void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s);
// What the step's finish needs when it runs inside the spreading launch.
struct FinishArgs {
    const double *blockmax;   // stage-2 per-CTA maxima
    int nb;                   // their count
    double *dt;               // the next step size (device)
    int *err;                 // the device error word
    double dt_fixed;          // > 0: the step size used
    double *part;             // kFinishCtas x 5 chunk partials
    unsigned *ticket;         // last-CTA ticket (zero between launches)
};
FinishArgs finish_args(const MarkerBuffers &m, const FluidBuffers &fb, int nb, double dt_fixed);

// spreading and forced update: through the precomputed operator when
// m.sp_ready, else gathering straight from the binned markers; with fin
// (operator path only) the step's finish runs in the same launch
cudaError_t launch_spread_apply(const GridParams &g, int fp_bytes, void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s,
                                const FinishArgs *fin = nullptr);
// the spreading operator of the current (static) markers, from their bins
cudaError_t launch_spread_build(const GridParams &g, int fp_bytes, const MarkerBuffers &m,
                                int grid_ctas, cudaStream_t s);
// sums[8..11] = sum eps~ G, sum eps~ H of the current G, H (fixed order)
cudaError_t launch_partial_sums(const GridParams &g, const MarkerBuffers &m, cudaStream_t s);
// force/heat sums, the time update and the next dt from the stage-2 and
// band maxima (nbs = 0 when the spread kernel did not run), split over up to
// kFinishCtas CTAs with a fixed-order combine
constexpr int kFinishCtas = 32;
cudaError_t launch_finish(const GridParams &g, const MarkerBuffers &m, const FluidBuffers &fb,
                          int nb, int nbs, double dt_fixed, cudaStream_t s);
// cp[k] = (I[p]_k - p_inf) / (rho_inf U_inf^2 / 2) at every marker
cudaError_t launch_surface_pressure(const GridParams &g, int fp_bytes, const void *U,
                                    const MarkerBuffers &m, cudaStream_t s);
cudaError_t launch_interpolate_op(const GridParams &g, int fp_bytes, const void *field, int nc,
                                  const MarkerBuffers &m, double *out, cudaStream_t s);
cudaError_t launch_spread_op(const GridParams &g, int fp_bytes, const double *R, int nc,
                             const MarkerBuffers &m, void *out, cudaStream_t s);

// ---- batches of 2D grids (batch.cu drives; kernels in flux.cu, markers.cu) --
// One case of a batch as the batched kernels see it.  Two tables exist, one
// per step parity, so that Un and Us swap without rewriting the table.
struct BatchCase {
    GridParams g;
    const void *Un;              // state at the start of the step
    void *Us;                    // state at the end of the step (stage 2 output, forced in place)
    void *U1;                    // stage-1 output
    double *dt;                  // this case's step size
    int *err;                    // this case's error word
    const unsigned *band_bits;   // this case's band mask
    MarkerBuffers m;             // this case's markers
    int item0, nitems;           // its (case, tile) stage items, for the tile shape in use
    int band0, nband;            // its (case, band tile) spread items
};

constexpr int kBatchShapes = 4;   // 2D tile shapes of the batched stage kernel
void batch_tile_shape(int shape, int *bx, int *by);
// mode 1 or 2 as launch_stage1/2; items are (case, tile) pairs in the
// shape's tile numbering; mode 2 writes item_max[item]
cudaError_t launch_batch_stage(int mode, int shape, int fp_bytes, const BatchCase *cases,
                               const int2 *items, int n_items, double *item_max, double dt_fixed,
                               int n_sm, cudaStream_t s);
// interpolation + forcing: items are (case, marker); warps = markers per CTA
cudaError_t launch_batch_interp(int fp_bytes, const BatchCase *cases, const int2 *items,
                                int n_items, int warps, cudaStream_t s);
// spreading + forced update: items are (case, index into the case's band
// list); band_max[item] receives the step-size maximum of the forced cells
// the spreading of a batch through its cases' operators (static markers):
// items (case, first of 32 forced cells)
cudaError_t launch_batch_spread_static(int fp_bytes, const BatchCase *cases, const int2 *items,
                                       int n_items, double *band_max, cudaStream_t s);
cudaError_t launch_batch_spread(int fp_bytes, size_t smem, const BatchCase *cases,
                                const int2 *items, int n_items, double *band_max, int n_sm,
                                cudaStream_t s);
size_t batch_spread_smem(const GridParams &g, int fp_bytes);
// per-case sums, time update and next step size (one CTA per case)
// sums[0..4], t and the error word of every case into out[c * 8 + 0..6]
cudaError_t launch_batch_gather(const BatchCase *cases, int ncases, double *out, cudaStream_t s);
// wall temperatures of a batch: slot c copies vals[off, off + n) to dst
struct BatchTwSlot {
    double *dst;
    long long off, n;
};
cudaError_t launch_batch_tw(const BatchTwSlot *slots, int ncases, const double *vals,
                            cudaStream_t s);
cudaError_t launch_batch_finish(const BatchCase *cases, int ncases, const double *item_max,
                                const double *band_max, double dt_fixed, cudaStream_t s);

// ---- discrete adjoint (adjoint.cu) -------------------------------------------
// Device buffers of ibm_record / ibm_backward, carved from the caller's
// adjoint workspace.  States are (dim+2) x N elements of the grid's type.
struct AdjBuffers {
    int max_steps = 0, every = 0, n_ckpt = 0, cap = 0;
    void *ckpt = nullptr;        // n_ckpt states: U at steps 0, every, 2 every, ...
    double *dt_hist = nullptr;   // step size of every recorded step
    void *seg = nullptr;         // every states: one replayed segment
    void *seg1 = nullptr;        // every states: U1 of each step of the segment
    void *segs = nullptr;        // every states: U* (before forcing) of each step
    double *segf = nullptr;      // every x cap x 5: rho_L, G (3), H of each step
    void *A = nullptr;           // U1 of the step being reversed
    void *B = nullptr;           // U* of the step being reversed
    void *lam = nullptr;         // adjoint state
    void *mu = nullptr;          // adjoint of U1
    void *jtv = nullptr;         // scratch state
    void *lfq = nullptr;         // (dim+1) x N: adjoints of the spread sources
    void *lamW = nullptr;        // (dim+2) x N doubles of FP64 scratch (band-cell passes)
    void *tbuf = nullptr;        // flux transpose: tile-plus-halo sums of every tile
    double *lamX = nullptr;      // cap x 3 marker-position gradient
    double *lamTw = nullptr;     // cap wall-temperature gradient
    double *lamEps = nullptr;    // cap adjoint of eps~
    double *mr = nullptr;        // cap x 5: adjoints of rho_L, I[rho u] (3), I[rho e]
    double *z = nullptr;         // cap: A~ z = lamEps
    double *save = nullptr;      // cap x 5: rho_L, G (3), H of the last forward step
};

// out = J_L(U)^T V (tbuf: the per-tile accumulators of the adjoint workspace)
cudaError_t launch_rhs_vjp(const GridParams &g, int fp_bytes, const void *U, const void *V,
                           void *tbuf, void *out, cudaStream_t s);
// one step reversed: a.A = U1, a.B = U* and the marker forcing of the step
// must be current; a.lam holds the adjoint of U^{n+1} and receives that of
// U^n; cd, nu: the direct terms of J (last step only)
cudaError_t launch_reverse_step(const GridParams &g, int fp_bytes, const MarkerBuffers &m,
                                const AdjBuffers &a, const void *Un, double dt, double cd,
                                double nu, int n_sm, cudaStream_t s);
// dJ/dX through eps~: a.z = A~^{-1} dJ/deps~ must be current
cudaError_t launch_eps_adjoint_x(const GridParams &g, const MarkerBuffers &m, const AdjBuffers &a,
                                 int n_sm, cudaStream_t s);

// ---- quadrature (quadrature.cu) --------------------------------------------
struct QuadBuffers {
    int width;               // row capacity of the ELL storage
    int cap;                 // marker capacity (ELL column stride)
    int *cnt;                // cap
    int *col;                // width * cap, column-major
    double *val;             // width * cap
    double *diag;            // cap
    double *r, *z, *p, *q;   // cap each
    int *iters;              // CG iterations of the last solve
    double *resid;           // true residual of the last solve
};

int quad_row_width(int dim);
// A~ assembly and the solve A~ eps~ = 1 (warm: start from the current eps~;
// have_weights: m.wphi already holds the current positions' support weights)
cudaError_t launch_quadrature(const GridParams &g, const MarkerBuffers &m, const QuadBuffers &qb,
                              double tol, int maxit, int warm, cudaStream_t s, int have_weights = 0);
cudaError_t launch_quadrature_solve(int ns, const QuadBuffers &qb, const double *rhs, double *x,
                                    double tol, int maxit, int *err, cudaStream_t s);

}  // namespace ibmk
