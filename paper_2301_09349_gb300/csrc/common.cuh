// Device-side definitions shared by the library's kernels (internal header).
//
// Grid parameters are passed to every kernel by value in one POD struct; the
// physics follows Sec. 2.1 of the paper (perfect gas, Sutherland viscosity,
// Newtonian stress, Fourier heat flux) in units rho_inf = U_inf = T_inf = 1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ibmk {

// error bits recorded on the device, decoded by the host at sync points
enum : int {
    ERR_NONFINITE = 1,      // non-finite or non-positive density/pressure
    ERR_NOCONV = 2,         // quadrature CG did not converge
    ERR_MARKER_RANGE = 4,   // a (moving) marker left the admissible region
    ERR_CAPACITY = 8,       // a quadrature row exceeded its storage
    ERR_TIMEOUT = 16,       // a bounded wait gave up
    ERR_BOUNDS = 32,        // (bounds-checked build) an index outside its array
};

enum : int { BC_FREESTREAM = 0, BC_ZEROGRAD = 1, BC_SLIP = 2, BC_PERIODIC = 3 };

// Positivity reading of the forced update (the paper is silent on it): the
// heat source of one step removes at most this fraction of a forced cell's
// internal energy, dt q_j >= -0.9 (rho e)*_j.  It never binds in the Mach 0.3
// cases or with a hot wall; it keeps the pressure positive when a cold wall
// meets an impulsive Mach 2 start.
constexpr double kHeatSourceCap = 0.9;

// Single-precision copies of the gas and grid constants, each rounded once
// from its double value on the host, for kernels that compute in FP32
// (double arithmetic runs at a small fraction of the FP32 rate on this GPU,
// so no FP32 kernel converts or divides doubles per cell or per face).
struct FloatConsts {
    float gamma, inv_gm1, gm1, invR, mu_inf, S, onepS, lam_fac, inv_h, qinv_h, kvisc, E_inf;
    int viscous;
};

struct GridParams {
    int dim;
    int n[3];
    long long N;          // cells
    double lo[3];
    double h, inv_h;
    double gamma, Pr, Re, Mach, S, cfl;
    double R, cv, cp;     // gas constant r = 1/(gamma Ma^2), c_v, c_p
    double mu_inf;        // 1/Re, or 0 when inviscid
    double kvisc;         // max(4/3, gamma/Pr) for the viscous step limit
    double p_inf;         // free-stream pressure
    int bc[6];
    int tile[3];
    int ntile[3];
    int n_tiles;
    int cells_per_tile;
    int energy_reading;
    int forcing_per_stage;
    FloatConsts f;        // FP32 copies of the constants above
};

inline FloatConsts float_consts(const GridParams &g) {
    FloatConsts c;
    c.gamma = (float)g.gamma;
    c.inv_gm1 = (float)(1.0 / (g.gamma - 1.0));
    c.gm1 = (float)(g.gamma - 1.0);
    c.invR = (float)(1.0 / g.R);
    c.mu_inf = (float)g.mu_inf;
    c.S = (float)g.S;
    c.onepS = (float)(1.0 + g.S);
    c.lam_fac = (float)(g.cp / g.Pr);
    c.inv_h = (float)g.inv_h;
    c.qinv_h = (float)(0.25 * g.inv_h);
    c.kvisc = (float)g.kvisc;
    c.E_inf = (float)(g.p_inf / (g.gamma - 1.0) + 0.5);
    c.viscous = g.mu_inf > 0.0;
    return c;
}

// The 1D regularised 3-point delta of Sec. 2.2 (Pinelli et al.); r in cells.
__device__ __forceinline__ double phi_d(double r) {
    double a = fabs(r);
    if (a <= 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) * (1.0 / 3.0);
    if (a <= 1.5) {
        double b = 1.0 - a;
        return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * b * b)) * (1.0 / 6.0);
    }
    return 0.0;
}

// Owner cell floor((X - lo)/h) per axis, rounded exactly as IEEE double
// subtraction and division (no contraction), so every implementation that
// evaluates the same two IEEE operations bins identically.
__device__ __forceinline__ int owner_cell(double x, double lo, double h) {
    return (int)floor(__ddiv_rn(__dsub_rn(x, lo), h));
}

__device__ __forceinline__ double cell_center(const GridParams &g, int d, int i) {
    return g.lo[d] + (i + 0.5) * g.h;
}

// Interior source index of an index along one axis under that axis's face
// boundary conditions.  Slip mirrors and toggles `flip` for the axis;
// freestream sets `fs`.  Matches the boundary description of ibm.h.
__device__ __forceinline__ int map_axis(int idx, int n, int bc_lo, int bc_hi, int axis, int &flip,
                                        int &fs) {
    if (idx >= 0 && idx < n) return idx;
    int bc = idx < 0 ? bc_lo : bc_hi;
    if (bc == BC_FREESTREAM) { fs = 1; return idx < 0 ? 0 : n - 1; }
    if (bc == BC_ZEROGRAD) return idx < 0 ? 0 : n - 1;
    if (bc == BC_SLIP) {
        flip ^= (1 << axis);
        int s = idx < 0 ? -1 - idx : 2 * n - 1 - idx;
        return s < 0 ? 0 : (s >= n ? n - 1 : s);
    }
    int m = idx % n;
    return m < 0 ? m + n : m;
}

// key of a cell for the marker bins: tile id * cells_per_tile + cell in tile
__device__ __forceinline__ unsigned cell_key(const GridParams &g, int cx, int cy, int cz) {
    int tx = cx / g.tile[0], ty = cy / g.tile[1], tz = cz / g.tile[2];
    int lx = cx - tx * g.tile[0], ly = cy - ty * g.tile[1], lz = cz - tz * g.tile[2];
    unsigned tid = (unsigned)(tx + g.ntile[0] * (ty + g.ntile[1] * tz));
    unsigned cin = (unsigned)(lx + g.tile[0] * (ly + g.tile[1] * lz));
    return tid * (unsigned)g.cells_per_tile + cin;
}

__device__ __forceinline__ void record_error(int *err, int bits) { atomicOr(err, bits); }

// Larger of two non-negative doubles through their bit patterns, which order
// like the values from +0 to +inf (a NaN with a clear sign bit orders above
// them all, so it propagates where fmax would drop it): integer ALU work
// instead of the FP64 pipe, which retires about two operations per SM cycle
// on this GPU with a 64-cycle dependent latency.
__device__ __forceinline__ double dmax_nonneg(double a, double b) {
    const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
    return __longlong_as_double(x > y ? x : y);
}

// Bounds-checked build (compiled with IBM_CHECKED, the stand-in for a memory
// checker on this GPU): a global index outside [0, n) is recorded in the
// device error word (ERR_BOUNDS, reported as IBM_ERR_BOUNDS) and the caller
// skips the access; nothing traps.  The regular build compiles the checks
// away.
#ifdef IBM_CHECKED
__device__ __forceinline__ bool in_bounds(long long i, long long n, int *err) {
    if (i >= 0 && i < n) return true;
    record_error(err, ERR_BOUNDS);
    return false;
}
#else
__device__ __forceinline__ bool in_bounds(long long, long long, int *) { return true; }
#endif

// a - b on both lanes of an FP32 pair in one packed instruction, rounded to
// nearest, subnormal results flushed (the FP32 stage units are built with
// flushing on).  Adding the negated pair instead costs two scalar negations.
__device__ __forceinline__ float2 fsub2_ftz(float2 a, float2 b) {
    float2 r;
    asm("{ .reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.ftz.f32x2 pd, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pd; }"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

}  // namespace ibmk
