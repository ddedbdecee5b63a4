// Host-side declarations shared by the library's translation units
// (internal; the public ABI is include/ibm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace ibmk {

// ---- fluid stages (flux.cu) ------------------------------------------------
// Stage 1: L = L(U), per-block maximum of the step-size rate, and (by the
// last block) dt = cfl / max s, or dt_fixed when > 0, written to *dt.
// Stage 2: out = U/2 + (U1 + dt L(U1))/2 with U1 = U + dt Lprev built on load.
struct FluidBuffers {
    double *blockmax;       // one per CTA of the stage-1 grid
    unsigned *counter;      // last-block ticket (zero between launches)
    double *dt;             // device step size
    int *err;               // device error word
};

size_t fluid_blockmax_count(const GridParams &g, int fp_bytes);
cudaError_t launch_stage1(const GridParams &g, int fp_bytes, const void *U, void *L,
                          const FluidBuffers &fb, double dt_fixed, cudaStream_t s);
cudaError_t launch_stage2(const GridParams &g, int fp_bytes, const void *U, const void *Lprev,
                          void *out, const FluidBuffers &fb, cudaStream_t s);
// L(U) only (no step size), for the diagnostic ibm_rhs
cudaError_t launch_rhs(const GridParams &g, int fp_bytes, const void *U, void *L,
                       const FluidBuffers &fb, cudaStream_t s);
// the z-marching form used for 3D FP32 grids (flux_zm.cu); mode 0/1/2 as above
cudaError_t launch_zmarch(int mode, const GridParams &g, const void *U, const void *Lp, void *out,
                          const FluidBuffers &fb, double dt_fixed, cudaStream_t s);
size_t zmarch_blocks(const GridParams &g);

// ---- markers (markers.cu) --------------------------------------------------
struct MarkerBuffers {
    int ns;                  // kept markers
    double *X0, *X;          // ns*dim positions at t = 0 and now
    double *Ub0, *Ub;        // ns*dim body velocity (prescribed part, current)
    double *Tw;              // ns wall temperatures
    double *eps;             // ns quadrature weights eps~
    int *cell;               // ns*3 owner cells floor((X - lo)/h) (bins kernel)
    double *frac_d;          // ns*3 offsets (X - lo)/h - cell, in [0, 1)
    float *frac_f;           // the same offsets in single precision
    double *rhoL, *G, *H;    // last forcing: rho_L, dt*F (ns*dim), dt*Q
    unsigned *keys[2];       // radix-sort ping-pong
    int *perm[2];
    int sorted;              // which of keys/perm holds the sorted order
    int *tile_off;           // n_tiles + 1
    int *occ_flag, *band_flag;  // n_tiles
    int *occ_list, *band_list;  // n_tiles
    int *counts;             // [0] occupied tiles, [1] band tiles
    double *sums;            // [0..2] sum eps~ G, [3] sum eps~ H, [4] dt of those sums
    double *t;               // simulated time
    long long *steps;        // step counter
    int *err;
};

cudaError_t launch_motion(const GridParams &g, const MarkerBuffers &m, double amp, double freq,
                          int axis, const double *dt, cudaStream_t s);
cudaError_t launch_bin(const GridParams &g, MarkerBuffers &m, cudaStream_t s);
cudaError_t launch_interp_force(const GridParams &g, int fp_bytes, const void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s);
cudaError_t launch_spread_apply(const GridParams &g, int fp_bytes, void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s);
cudaError_t launch_finish(const GridParams &g, const MarkerBuffers &m, const double *dt,
                          cudaStream_t s);
cudaError_t launch_interpolate_op(const GridParams &g, int fp_bytes, const void *field, int nc,
                                  const MarkerBuffers &m, double *out, cudaStream_t s);
cudaError_t launch_spread_op(const GridParams &g, int fp_bytes, const double *R, int nc,
                             const MarkerBuffers &m, void *out, cudaStream_t s);

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
cudaError_t launch_quadrature(const GridParams &g, const MarkerBuffers &m, const QuadBuffers &qb,
                              double tol, int maxit, int warm, cudaStream_t s);

}  // namespace ibmk
