// Fluid stages for 3D FP32 grids: the same discretisation as flux.cu
// (MUSCL/van Leer + Rusanov + central viscous/heat fluxes, SSP-RK2 stages),
// organised as a z-march for GB300.
//
// A CTA of 256 threads owns a 32 x 16 column of cells and walks up a chunk of
// z-planes; each thread owns two neighbouring cells of one row, (2t, r) and
// (2t+1, r).  Shared memory holds a ring of four primitive planes (z-1 ..
// z+2) with a two-cell halo in x and y, so every cell is loaded from memory
// and converted to primitives once per chunk.  Per plane and thread:
//   - the x-faces 2t-1/2 and 2t+1/2 of its row as one packed FP32x2 pair:
//     the five cells 2t-2 .. 2t+2 give the three limited slopes of cells
//     2t-1, 2t, 2t+1 (the middle one serves both faces);
//   - the y-faces below its two cells (row r-1/2) as a pair;
//   - the z-faces above its two cells (z+1/2) as a pair; the limited z-slope
//     of plane z+1 and the z-face fluxes are carried in registers to the
//     next plane, where they are the lower plane's;
//   - warp 7 also evaluates the tile's upper x- and y-edge faces;
// one barrier, then each thread forms the flux divergence of its two cells
// from its own faces (registers), the x-face of its right neighbour (a warp
// shuffle), the y-faces of the row above (shared memory), and writes both
// cells with 8-byte accesses; the next plane is converted into the ring and
// a second barrier closes the plane.  Neighbouring cells sit in adjacent
// 32-bit words of the ring, so most stencil loads are 8-byte (two cells).
// All constants are single precision: the kernel issues no FP64 work except
// the per-CTA step-size maximum.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>
#include <stdint.h>
#include <string.h>

#include "internal.h"

namespace ibmk {
namespace {

constexpr int TX = 32, TY = 16, NTH = 256;               // tile cells; 16 threads per row
constexpr int PX = TX + 4, PY = TY + 4, PP = PX * PY;    // plane with a 2-cell halo
constexpr int NW = 6;                                     // rho, u, v, w, p, T
constexpr int NC = 5;
constexpr int RING = 4;
constexpr int SLOT = NW * PP;
// TMA staging box of one plane: x from ox-4 (16-byte aligned) over 40 cells,
// y from oy-2 over 20 rows, the five conserved components
constexpr int SBX = TX + 8, SBY = TY + 4;
constexpr int STAGE = NC * SBX * SBY;                     // floats
constexpr int FYN = NC * (TY + 1) * TX;                   // y-face fluxes, row r = face r-1/2
constexpr int FXE = NC * TY;                              // x-face fluxes of the upper x edge
constexpr size_t SMEM_BASE = sizeof(float) * (size_t)(RING * SLOT + FYN + FXE);
constexpr size_t SMEM_TMA_OFF = (SMEM_BASE + 127) / 128 * 128;
constexpr size_t SMEM = SMEM_TMA_OFF + sizeof(float) * STAGE + 16;   // + mbarrier
constexpr long long TMA_WAIT_LIMIT = 1ll << 20;           // bounded mbarrier waits
static_assert(PX % 2 == 0 && PP % 2 == 0 && SLOT % 2 == 0, "8-byte ring loads need even strides");

using FC = FloatConsts;

// step-size rate of one cell from its conserved state, single precision
// throughout (same formula as the shared step_rate helper)
__device__ __forceinline__ float rate_f(const FC &c, const float *u, bool &ok) {
    const float rho = u[0], inv = __fdividef(1.0f, rho);
    const float vx = u[1] * inv, vy = u[2] * inv, vz = u[3] * inv;
    const float p = c.gm1 * (u[4] - 0.5f * rho * (vx * vx + vy * vy + vz * vz));
    const float c2 = c.gamma * p * inv;
    const float snd = c2 * rsqrtf(c2);
    float mu = 0.0f;
    if (c.viscous) {
        const float Tt = p * inv * c.invR;
        mu = __fdividef(c.mu_inf * Tt * (Tt * rsqrtf(Tt)) * c.onepS, Tt + c.S);
    }
    const float s = (fabsf(vx) + fabsf(vy) + fabsf(vz) + 3.0f * snd) * c.inv_h +
                    6.0f * (c.kvisc * mu * inv) * c.inv_h * c.inv_h;
    if (!(rho > 0.0f && p > 0.0f && s <= 3.0e38f)) ok = false;
    return s;
}

FC make_fc(const GridParams &g) { return float_consts(g); }

// ---- packed pairs: two faces evaluated by one FP32x2 instruction stream ----
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return fsub2_ftz(a, b); }
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sp(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 rcp2(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}
__device__ __forceinline__ float2 rsqrt2(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 abs2(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 max2(float2 a, float2 b) {
    return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
// half the van Leer slope, ab / (a + b) where ab > 0: the face states are
// w +- psi/2, and the factor 2 of psi = 2ab/(a+b) and the 1/2 cancel exactly
__device__ __forceinline__ float2 vlh2(float2 a, float2 b) {
    const float2 ab = a * b;
    const float2 q = ab * rcp2(a + b);
    return make_float2(ab.x > 0.0f ? q.x : 0.0f, ab.y > 0.0f ? q.y : 0.0f);
}
__device__ __forceinline__ float vlh1(float a, float b) {
    const float ab = a * b;
    const float q = ab * __fdividef(1.0f, a + b);
    return ab > 0.0f ? q : 0.0f;
}
// two neighbouring ring cells (the first at an even index)
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }

// Rusanov flux of two faces from their reconstructed states in the face
// frame (rho, u_n, u_t1, u_t2, p): F = (mass, normal momentum, t1 momentum,
// t2 momentum, energy).
__device__ __forceinline__ void euler_pair(const FC &c, const float2 (&wl)[NC],
                                           const float2 (&wr)[NC], float2 (&F)[NC]) {
    const float2 keL = fma2(wl[1], wl[1], fma2(wl[2], wl[2], wl[3] * wl[3]));
    const float2 keR = fma2(wr[1], wr[1], fma2(wr[2], wr[2], wr[3] * wr[3]));
    const float2 EL = fma2(wl[4], sp(c.inv_gm1), sp(0.5f) * wl[0] * keL);
    const float2 ER = fma2(wr[4], sp(c.inv_gm1), sp(0.5f) * wr[0] * keR);
    const float2 unL = wl[1], unR = wr[1];
    const float2 c2L = sp(c.gamma) * wl[4] * rcp2(wl[0]);
    const float2 c2R = sp(c.gamma) * wr[4] * rcp2(wr[0]);
    const float2 sL = fma2(c2L, rsqrt2(c2L), abs2(unL));
    const float2 sR = fma2(c2R, rsqrt2(c2R), abs2(unR));
    const float2 hs = sp(-0.5f) * max2(sL, sR);      // -smax/2
    const float2 mLn = wl[0] * unL, mRn = wr[0] * unR;
    const float2 mL1 = wl[0] * wl[2], mR1 = wr[0] * wr[2];
    const float2 mL2 = wl[0] * wl[3], mR2 = wr[0] * wr[3];
    F[0] = fma2(hs, wr[0] - wl[0], sp(0.5f) * (mLn + mRn));
    F[1] = fma2(hs, mRn - mLn, sp(0.5f) * (fma2(mLn, unL, wl[4]) + fma2(mRn, unR, wr[4])));
    F[2] = fma2(hs, mR1 - mL1, sp(0.5f) * fma2(mL1, unL, mR1 * unR));
    F[3] = fma2(hs, mR2 - mL2, sp(0.5f) * fma2(mL2, unL, mR2 * unR));
    F[4] = fma2(hs, ER - EL, sp(0.5f) * fma2(EL + wl[4], unL, (ER + wr[4]) * unR));
}

// Viscous stress and heat flux of two faces, subtracted from F (face frame).
// Cell values of the velocity components (n, t1, t2) and T on the two sides
// a and b; d1n, d11: the sums over the two cells of the central differences
// (w[+1] - w[-1], unscaled) of u_n and u_t1 along t1; d2n, d22: of u_n and
// u_t2 along t2.  Tangential derivatives are those sums / (4h) (reading 11).
__device__ __forceinline__ void visc_pair(const FC &c, float2 na, float2 nb, float2 t1a,
                                          float2 t1b, float2 t2a, float2 t2b, float2 Ta,
                                          float2 Tb, float2 d1n, float2 d11, float2 d2n,
                                          float2 d22, float2 (&F)[NC]) {
    const float2 Tf = sp(0.5f) * (Ta + Tb);
    const float2 mu = sp(c.mu_inf * c.onepS) * Tf * (Tf * rsqrt2(Tf)) * rcp2(Tf + sp(c.S));
    const float2 lam = mu * sp(c.lam_fac);
    const float2 ih = sp(c.inv_h), qh = sp(c.qinv_h);
    const float2 dn_n = (nb - na) * ih;
    const float2 dn_1 = (t1b - t1a) * ih;
    const float2 dn_2 = (t2b - t2a) * ih;
    const float2 dn_T = (Tb - Ta) * ih;
    const float2 div = fma2(d11 + d22, qh, dn_n);
    const float2 tNN = mu * fma2(sp(2.0f), dn_n, sp(-2.0f / 3.0f) * div);
    const float2 tN1 = mu * fma2(d1n, qh, dn_1);
    const float2 tN2 = mu * fma2(d2n, qh, dn_2);
    const float2 ufn = sp(0.5f) * (na + nb);
    const float2 uf1 = sp(0.5f) * (t1a + t1b);
    const float2 uf2 = sp(0.5f) * (t2a + t2b);
    F[1] = F[1] - tNN;
    F[2] = F[2] - tN1;
    F[3] = F[3] - tN2;
    F[4] = F[4] - fma2(ufn, tNN, fma2(uf1, tN1, fma2(uf2, tN2, lam * dn_T)));
}

// central differences (unscaled) along x of a field at cells 2t, 2t+1 of one
// row: w[x+1] - w[x-1] from the pairs at x-2, x (given) and x+2
__device__ __forceinline__ float2 cdx2(const float *f, float2 mid) {
    const float2 lo = ld2(f - 2), hi = ld2(f + 2);
    return make_float2(mid.y, hi.x) - make_float2(lo.y, mid.x);
}

// x-faces 2t-1/2 (.x) and 2t+1/2 (.y) of one row; b: ring index of cell 2t
// in the plane slot R points at; up, dn: offsets to the planes above and
// below.  Output in (rho, rho u, rho v, rho w, rho E) order.
__device__ __forceinline__ void x_pair(const FC &c, const float *__restrict__ R, int b, int up,
                                       int dn, float2 (&F)[NC]) {
    float2 wl[NC], wr[NC];
    float2 va[3], vb[3];     // u, v, w on the a side (cells 2t-1, 2t) and b side (2t, 2t+1)
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *f = R + m * PP + b;
        const float2 lo = ld2(f - 2), mid = ld2(f);
        const float w2 = f[2];
        const float2 dA = make_float2(lo.y, mid.y) - make_float2(lo.x, mid.x);   // d(-3/2), d(1/2)
        const float2 dB = make_float2(mid.x, w2) - make_float2(lo.y, mid.y);     // d(-1/2), d(3/2)
        const float2 so = vlh2(dA, dB);                                          // slopes of 2t-1, 2t+1
        const float s0 = vlh1(dB.x, dA.y);                                       // slope of 2t
        wl[m] = make_float2(lo.y, mid.x) + make_float2(so.x, s0);
        wr[m] = mid - make_float2(s0, so.y);
        if (m >= 1 && m <= 3) {
            va[m - 1] = make_float2(lo.y, mid.x);
            vb[m - 1] = mid;
        }
    }
    euler_pair(c, wl, wr, F);
    if (!c.viscous) return;
    const float *T = R + 5 * PP + b;
    const float2 Tmid = ld2(T);
    const float2 Ta = make_float2(T[-1], Tmid.x), Tb = Tmid;
    // central differences of cells 2t-1, 2t, 2t+1 along an axis of stride o
    // (o = PX: y) summed pairwise per face
    auto cd = [&](const float *f, int o) {
        const float cm = f[o - 1] - f[-o - 1];
        const float2 c01 = ld2(f + o) - ld2(f - o);
        return make_float2(cm, c01.x) + c01;
    };
    const float *U = R + PP + b, *V = R + 2 * PP + b, *W = R + 3 * PP + b;
    const float2 d1n = cd(U, PX), d11 = cd(V, PX);   // along y: u (normal), v (t1)
    // along z (planes above and below): u (normal) and w (t2)
    const float um = U[up - 1] - U[dn - 1];
    const float2 u01 = ld2(U + up) - ld2(U + dn);
    const float wm = W[up - 1] - W[dn - 1];
    const float2 w01 = ld2(W + up) - ld2(W + dn);
    const float2 d2n = make_float2(um, u01.x) + u01;
    const float2 d22 = make_float2(wm, w01.x) + w01;
    visc_pair(c, va[0], vb[0], va[1], vb[1], va[2], vb[2], Ta, Tb, d1n, d11, d2n, d22, F);
}

// y-faces at row r-1/2 of cells 2t (.x) and 2t+1 (.y); b: ring index of cell
// (2t, r).  Output in (rho, rho u, rho v, rho w, rho E) order.
__device__ __forceinline__ void y_pair(const FC &c, const float *__restrict__ R, int b, int up,
                                       int dn, float2 (&Fo)[NC]) {
    constexpr int fy[NC] = {0, 2, 1, 3, 4};   // face frame (rho, v, u, w, p)
    float2 wl[NC], wr[NC], ca[NC], cb[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *f = R + fy[m] * PP + b;
        const float2 x0 = ld2(f - 2 * PX), x1 = ld2(f - PX), x2 = ld2(f), x3 = ld2(f + PX);
        const float2 d0 = x1 - x0, d1 = x2 - x1, d2 = x3 - x2;
        wl[m] = x1 + vlh2(d0, d1);
        wr[m] = x2 - vlh2(d1, d2);
        ca[m] = x1;
        cb[m] = x2;
    }
    float2 F[NC];
    euler_pair(c, wl, wr, F);
    if (c.viscous) {
        const float *T = R + 5 * PP + b;
        const float2 Ta = ld2(T - PX), Tb = ld2(T);
        const float *U = R + PP + b, *V = R + 2 * PP + b, *W = R + 3 * PP + b;
        // along x: v (normal) and u (t1) at rows r-1 and r
        const float2 d1n = cdx2(V - PX, ca[1]) + cdx2(V, cb[1]);
        const float2 d11 = cdx2(U - PX, ca[2]) + cdx2(U, cb[2]);
        // along z: v (normal) and w (t2)
        const float2 d2n = (ld2(V - PX + up) - ld2(V - PX + dn)) + (ld2(V + up) - ld2(V + dn));
        const float2 d22 = (ld2(W - PX + up) - ld2(W - PX + dn)) + (ld2(W + up) - ld2(W + dn));
        visc_pair(c, ca[1], cb[1], ca[2], cb[2], ca[3], cb[3], Ta, Tb, d1n, d11, d2n, d22, F);
    }
    Fo[0] = F[0]; Fo[1] = F[2]; Fo[2] = F[1]; Fo[3] = F[3]; Fo[4] = F[4];
}

// halved limited z-slopes of cells 2t, 2t+1 at the plane of slot sm, from the
// planes below (sl) and above (sh); b: ring index of cell (2t, r)
__device__ __forceinline__ void z_slopes(const float *__restrict__ ring, int sl, int sm, int sh,
                                         int b, float2 (&sig)[NC]) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *f = ring + m * PP + b;
        const float2 lo = ld2(f + sl), mid = ld2(f + sm), hi = ld2(f + sh);
        sig[m] = vlh2(mid - lo, hi - mid);
    }
}

// z-faces between the planes of slots sa (below) and sb (above) for cells
// 2t (.x) and 2t+1 (.y): siga, sigb are the halved limited z-slopes of the
// two planes (lab field order).  Output in (rho, rho u, rho v, rho w, rho E)
// order.
__device__ __forceinline__ void z_pair(const FC &c, const float *__restrict__ ring, int sa, int sb,
                                       int b, const float2 (&siga)[NC], const float2 (&sigb)[NC],
                                       float2 (&Fo)[NC]) {
    constexpr int fz[NC] = {0, 3, 1, 2, 4};   // face frame (rho, w, u, v, p)
    float2 wl[NC], wr[NC], ca[NC], cb[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const int f = fz[m];
        ca[m] = ld2(ring + sa + f * PP + b);
        cb[m] = ld2(ring + sb + f * PP + b);
        wl[m] = ca[m] + siga[f];
        wr[m] = cb[m] - sigb[f];
    }
    float2 F[NC];
    euler_pair(c, wl, wr, F);
    if (c.viscous) {
        const float *A = ring + sa + b, *B = ring + sb + b;
        const float2 Ta = ld2(A + 5 * PP), Tb = ld2(B + 5 * PP);
        // along x: w (normal) and u (t1); along y: w (normal) and v (t2)
        const float2 d1n = cdx2(A + 3 * PP, ca[1]) + cdx2(B + 3 * PP, cb[1]);
        const float2 d11 = cdx2(A + PP, ca[2]) + cdx2(B + PP, cb[2]);
        const float2 d2n = (ld2(A + 3 * PP + PX) - ld2(A + 3 * PP - PX)) +
                           (ld2(B + 3 * PP + PX) - ld2(B + 3 * PP - PX));
        const float2 d22 = (ld2(A + 2 * PP + PX) - ld2(A + 2 * PP - PX)) +
                           (ld2(B + 2 * PP + PX) - ld2(B + 2 * PP - PX));
        visc_pair(c, ca[1], cb[1], ca[2], cb[2], ca[3], cb[3], Ta, Tb, d1n, d11, d2n, d22, F);
    }
    Fo[0] = F[0]; Fo[1] = F[2]; Fo[2] = F[3]; Fo[3] = F[1]; Fo[4] = F[4];
}

// Two faces of the tile's upper edges (warp 7), one per pair lane: the x-face
// between cells 31 and 32 of a row or the y-face between rows 15 and 16 of a
// column.  aA, aB: ring index of each face's lower cell; sn: the cell stride
// along the face normal (1 for x, PX for y), st the stride along the other
// in-plane axis; nf: the normal velocity field (1 = u, 2 = v).  Output in
// (rho, rho u, rho v, rho w, rho E) order.
__device__ __forceinline__ void edge_pair(const FC &c, const float *__restrict__ R, int aA, int aB,
                                          int sn, int st, int nf, int up, int dn,
                                          float2 (&Fo)[NC]) {
    // face frame (rho, normal, in-plane tangent, w, p)
    const int f[NC] = {0, nf, 3 - nf, 3, 4};
    float2 wl[NC], wr[NC], ca[NC], cb[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *X = R + f[m] * PP + aA, *Y = R + f[m] * PP + aB;
        const float2 x0 = make_float2(X[-sn], Y[-sn]);
        const float2 x1 = make_float2(X[0], Y[0]);
        const float2 x2 = make_float2(X[sn], Y[sn]);
        const float2 x3 = make_float2(X[2 * sn], Y[2 * sn]);
        const float2 d0 = x1 - x0, d1 = x2 - x1, d2 = x3 - x2;
        wl[m] = x1 + vlh2(d0, d1);
        wr[m] = x2 - vlh2(d1, d2);
        ca[m] = x1;
        cb[m] = x2;
    }
    float2 F[NC];
    euler_pair(c, wl, wr, F);
    if (c.viscous) {
        const float *TA = R + 5 * PP + aA, *TB = R + 5 * PP + aB;
        const float2 Ta = make_float2(TA[0], TB[0]), Tb = make_float2(TA[sn], TB[sn]);
        const float *NA = R + f[1] * PP + aA, *NB = R + f[1] * PP + aB;   // normal velocity
        const float *PA = R + f[2] * PP + aA, *PB = R + f[2] * PP + aB;   // in-plane tangent
        const float *WA = R + 3 * PP + aA, *WB = R + 3 * PP + aB;
        auto cd = [&](const float *A, const float *B, int o, int mo) {   // both cells of each face
            return make_float2(A[o] - A[mo], B[o] - B[mo]) +
                   make_float2(A[sn + o] - A[sn + mo], B[sn + o] - B[sn + mo]);
        };
        const float2 d1n = cd(NA, NB, st, -st), d11 = cd(PA, PB, st, -st);
        const float2 d2n = cd(NA, NB, up, dn), d22 = cd(WA, WB, up, dn);
        visc_pair(c, ca[1], cb[1], ca[2], cb[2], ca[3], cb[3], Ta, Tb, d1n, d11, d2n, d22, F);
    }
    // back to lab order: the normal momentum goes to u (x-face) or v (y-face)
    const bool xf = nf == 1;
    Fo[0] = F[0];
    Fo[1] = xf ? F[1] : F[2];
    Fo[2] = xf ? F[2] : F[1];
    Fo[3] = F[3];
    Fo[4] = F[4];
}

// ---- TMA: one bulk tensor copy per plane into the staging box -------------
__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// issue the copy of plane gz (thread 0 only)
__device__ __forceinline__ void tma_issue(const CUtensorMap *tmap, unsigned dst, unsigned mbar,
                                          int x0, int y0, int gz) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(mbar), "r"((unsigned)(sizeof(float) * STAGE)) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"((unsigned long long)tmap), "r"(x0), "r"(y0), "r"(gz), "r"(0), "r"(mbar)
        : "memory");
}
// wait for the phase with the given parity; bounded: after TMA_WAIT_LIMIT
// polls it gives up, sets the error flag and returns false
__device__ __forceinline__ bool tma_wait(unsigned mbar, unsigned parity, int *err) {
    for (long long it = 0; it < TMA_WAIT_LIMIT; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;"
            " selp.u32 %0, 1, 0, p; }"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    record_error(err, ERR_TIMEOUT);
    return false;
}

// primitives (rho, u, v, w, p, T) of one conserved cell into ring cell q
__device__ __forceinline__ void to_primitive(const FC &c, const float (&u)[NC],
                                             float *__restrict__ slot, int q) {
    const float rho = u[0];
    const float inv = __fdividef(1.0f, rho);
    const float vx = u[1] * inv, vy = u[2] * inv, vz = u[3] * inv;
    const float p = c.gm1 * (u[4] - 0.5f * rho * (vx * vx + vy * vy + vz * vz));
    slot[q] = rho;
    slot[PP + q] = vx;
    slot[2 * PP + q] = vy;
    slot[3 * PP + q] = vz;
    slot[4 * PP + q] = p;
    slot[5 * PP + q] = p * inv * c.invR;
}

// conserved state of a ghost or interior cell through the boundary maps
__device__ __forceinline__ void mapped_cell(const GridParams &g, const FC &c,
                                            const float *__restrict__ U, int gx, int gy, int gz,
                                            float (&u)[NC], int *err) {
    int flip = 0, fs = 0;
    const int sx = map_axis(gx, g.n[0], g.bc[0], g.bc[1], 0, flip, fs);
    const int sy = map_axis(gy, g.n[1], g.bc[2], g.bc[3], 1, flip, fs);
    const int sz = map_axis(gz, g.n[2], g.bc[4], g.bc[5], 2, flip, fs);
    if (fs) {
        u[0] = 1.0f;
        u[1] = 1.0f;
        u[2] = 0.0f;
        u[3] = 0.0f;
        u[4] = c.E_inf;
        return;
    }
    const long long N = g.N;
    const long long j = sx + (long long)g.n[0] * (sy + (long long)g.n[1] * sz);
    const bool okj = in_bounds(j, N, err);
#pragma unroll
    for (int m = 0; m < NC; ++m) u[m] = okj ? __ldg(U + m * N + j) : 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d)
        if ((flip >> d) & 1) u[1 + d] = -u[1 + d];
}

// Convert the staged plane gz into one ring slot.  Cells outside the domain in
// x or y (zero-filled by the copy) are taken through the boundary conditions.
__device__ __forceinline__ void convert_staged(const GridParams &g, const FC &c,
                                               const float *__restrict__ U,
                                               const float *__restrict__ st,
                                               float *__restrict__ slot, int ox, int oy, int gz,
                                               bool xy_interior, int *err) {
    for (int q = threadIdx.x; q < PP; q += NTH) {
        const int lx = q % PX, ly = q / PX;
        const int gx = ox + lx - 2, gy = oy + ly - 2;
        float u[NC];
        if (xy_interior || (gx >= 0 && gx < g.n[0] && gy >= 0 && gy < g.n[1])) {
#pragma unroll
            for (int m = 0; m < NC; ++m) u[m] = st[(m * SBY + ly) * SBX + lx + 2];
        } else {
            mapped_cell(g, c, U, gx, gy, gz, u, err);
        }
        to_primitive(c, u, slot, q);
    }
}

// Load plane gz (ghosts through the boundary conditions) and convert it to
// primitives into one ring slot.
__device__ __forceinline__ void load_plane(const GridParams &g, const FC &c,
                                           const float *__restrict__ U, float *__restrict__ slot,
                                           int ox, int oy, int gz, bool xy_interior, int *err) {
    const long long N = g.N;
    const bool fast = xy_interior && gz >= 0 && gz < g.n[2];
    for (int q = threadIdx.x; q < PP; q += NTH) {
        const int lx = q % PX, ly = q / PX;
        float u[NC];
        if (fast) {
            const long long j =
                (ox + lx - 2) + (long long)g.n[0] * ((oy + ly - 2) + (long long)g.n[1] * gz);
            const bool okj = in_bounds(j, N, err);
#pragma unroll
            for (int m = 0; m < NC; ++m) u[m] = okj ? __ldg(U + m * N + j) : 0.0f;
        } else {
            mapped_cell(g, c, U, ox + lx - 2, oy + ly - 2, gz, u, err);
        }
        to_primitive(c, u, slot, q);
    }
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

#ifndef IBM_ZM_MIN_BLOCKS
#define IBM_ZM_MIN_BLOCKS 2
#endif
#ifndef IBM_ZM_PREFETCH
#define IBM_ZM_PREFETCH 1
#endif

// MODE 0: out = L(Uin).  MODE 1: out = U1 = Uin + dt L(Uin).
// MODE 2: out = U* = Un/2 + (Uin + dt L(Uin))/2 with Uin = U1, plus the
// per-CTA maximum of s_j(U*) over the cells outside the band.
// TMA: the planes of Uin inside the domain arrive by bulk tensor copies,
// each prefetched one plane ahead while the faces of the current plane are
// evaluated (needs nx % 4 == 0); otherwise every plane is loaded by threads.
template <int MODE, bool TMA>
__global__ void __launch_bounds__(NTH, IBM_ZM_MIN_BLOCKS)
zmarch_kernel(const __grid_constant__ CUtensorMap tmap, const GridParams g, const FC c, int zc,
              const float *__restrict__ Uin, const float *__restrict__ Un,
              float *__restrict__ out, double *__restrict__ blockmax,
              const double *__restrict__ dt_ptr, int *__restrict__ err,
              const unsigned *__restrict__ band_bits, double dt_fixed) {
    extern __shared__ __align__(128) float smem_zm[];
    float *ring = smem_zm;
    float *FY = ring + RING * SLOT;           // [NC][TY+1][TX]: y-faces, row r = face r-1/2
    float *FXe = FY + FYN;                    // [NC][TY]: x-faces between cells 31 and 32
    __shared__ double s_red[NTH / 32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r = tid >> 4, t = tid & 15;     // row of the thread, its cells 2t and 2t+1
    const int ox = blockIdx.x * TX, oy = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.n[2]);
    const long long N = g.N;
    const float dt = MODE == 0 ? 0.0f : (float)(dt_fixed > 0.0 ? dt_fixed : *dt_ptr);
    const bool xyint = ox >= 2 && oy >= 2 && ox + TX + 2 <= g.n[0] && oy + TY + 2 <= g.n[1];
    auto slot_of = [](int z) { return ((z + RING) & (RING - 1)) * SLOT; };   // z >= -2
    const int b = (2 * t + 2) + PX * (r + 2);   // ring index of cell (2t, r)

    float *stage = reinterpret_cast<float *>(reinterpret_cast<char *>(smem_zm) + SMEM_TMA_OFF);
    const unsigned st_addr = smem_u32(stage);
    const unsigned mbar = smem_u32(stage + STAGE);
    unsigned parity = 0;
    const int nz = g.n[2];
    // A copy that does not complete within the bounded wait switches the CTA
    // to thread loads.  Each thread decides for the cells it converts: a
    // thread whose wait gave up loads its own cells of the plane from global
    // memory, one whose wait completed converts the staged copy; both give
    // the same values, so threads may decide differently within one plane.
    // The shared flag only stops further copies; thread 0 reads it after the
    // plane's barrier.  Thread 0 tracks the copy it issued last and, if it
    // never saw that copy complete, drains it (bounded) before the CTA exits.
    __shared__ int s_tma_dead;
    volatile int *tma_dead = &s_tma_dead;
    bool outstanding = false;   // thread 0 only
    if (TMA) {
        if (tid == 0) {
            *tma_dead = 0;
            mbar_init(mbar);
            if (z0 + 2 < nz) {
                tma_issue(&tmap, st_addr, mbar, ox - 4, oy - 2, z0 + 2);
                outstanding = true;
            }

        }
        __syncthreads();
    }
    // planes z0-2 .. z0+1 by threads; z0+2 comes from the copy just issued
    for (int zz = z0 - 2; zz <= z0 + 1; ++zz)
        load_plane(g, c, Uin, ring + slot_of(zz), ox, oy, zz, xyint, err);
    __syncthreads();

    // carried from plane to plane: the halved limited z-slopes of the current
    // plane and the z-face fluxes below it
    float2 sig[NC], Fzl[NC];
    {
        float2 sgm[NC];
        z_slopes(ring, slot_of(z0 - 2), slot_of(z0 - 1), slot_of(z0), b, sgm);
        z_slopes(ring, slot_of(z0 - 1), slot_of(z0), slot_of(z0 + 1), b, sig);
        z_pair(c, ring, slot_of(z0 - 1), slot_of(z0), b, sgm, sig, Fzl);
    }
    __syncthreads();   // plane z0-2's slot is about to take plane z0+2
    // plane z0+2 (the ring needs planes z-1 .. z+2 at plane z)
    {
        bool use_stage = TMA && z0 + 2 < nz;
        if (use_stage && !tma_wait(mbar, parity, err)) {
            use_stage = false;
            *tma_dead = 1;
        }
        if (use_stage) {
            parity ^= 1u;
            if (tid == 0) outstanding = false;
            convert_staged(g, c, Uin, stage, ring + slot_of(z0 + 2), ox, oy, z0 + 2, xyint, err);
        } else {
            load_plane(g, c, Uin, ring + slot_of(z0 + 2), ox, oy, z0 + 2, xyint, err);
        }
    }
    __syncthreads();
    if (TMA && tid == 0 && !*tma_dead && z0 + 1 < z1 && z0 + 3 < nz) {
        tma_issue(&tmap, st_addr, mbar, ox - 4, oy - 2, z0 + 3);
        outstanding = true;
    }

    // the edge lanes of warp 7: 0-15 the y-faces above row 15 (columns 2l,
    // 2l+1), 16-23 the x-faces right of column 31 (rows q and q + 8)
    const bool edge = warp == 7 && lane < 24;
    int eA = 0, eB = 0, esn = 1, est = PX, enf = 1;
    if (warp == 7) {
        if (lane < 16) {
            eA = (2 * lane + 2) + PX * (TY - 1 + 2);
            eB = eA + 1;
            esn = PX;
            est = 1;
            enf = 2;
        } else if (lane < 24) {
            const int q = lane - 16;
            eA = (TX - 1 + 2) + PX * (q + 2);
            eB = eA + 8 * PX;
        }
    }

    const int gx = ox + 2 * t, gy = oy + r;
    const bool row_in = gy < g.n[1];
    const bool in0 = row_in && gx < g.n[0], in1 = row_in && gx + 1 < g.n[0];
    const bool vec = in1 && (g.n[0] % 2 == 0);   // both cells, 8-byte aligned
    float smaxf = 0.0f;
    bool ok = true;
    for (int z = z0; z < z1; ++z) {
        const int sm1 = slot_of(z - 1), s0 = slot_of(z), s1 = slot_of(z + 1), s2 = slot_of(z + 2);
        const int up = s1 - s0, dn = sm1 - s0;
#if IBM_ZM_PREFETCH
        // stage 2 reads U^n at its output cells, which nothing has touched:
        // start those lines toward L2 two planes ahead
        if (MODE == 2 && z + 2 < z1 && in0) {
            const long long jp = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * (z + 2));
#pragma unroll
            for (int m = 0; m < NC; ++m)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Un + m * N + jp));
        }
#endif
        // faces of plane z: x pair, y pair (stored for the row below), z pair
        float2 Fx[NC], Fy[NC], Fzh[NC];
        x_pair(c, ring + s0, b, up, dn, Fx);
        y_pair(c, ring + s0, b, up, dn, Fy);
#pragma unroll
        for (int m = 0; m < NC; ++m) st2(FY + (m * (TY + 1) + r) * TX + 2 * t, Fy[m]);
        {
            float2 sgh[NC];
            z_slopes(ring, s0, s1, s2, b, sgh);
            z_pair(c, ring, s0, s1, b, sig, sgh, Fzh);
#pragma unroll
            for (int m = 0; m < NC; ++m) sig[m] = sgh[m];
        }
        if (edge) {
            float2 Fe[NC];
            edge_pair(c, ring + s0, eA, eB, esn, est, enf, up, dn, Fe);
            if (lane < 16) {
#pragma unroll
                for (int m = 0; m < NC; ++m) st2(FY + (m * (TY + 1) + TY) * TX + 2 * lane, Fe[m]);
            } else {
                const int q = lane - 16;
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    FXe[m * TY + q] = Fe[m].x;
                    FXe[m * TY + q + 8] = Fe[m].y;
                }
            }
        }
        __syncthreads();

        // flux divergence of the two cells
        float2 acc[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            // x-face right of cell 2t+1: the neighbour's first face, or the edge
            float fr = __shfl_down_sync(0xffffffffu, Fx[m].x, 1);
            if (t == 15) fr = FXe[m * TY + r];
            const float2 Fyu = ld2(FY + (m * (TY + 1) + r + 1) * TX + 2 * t);
            acc[m] = ((Fx[m] - make_float2(Fx[m].y, fr)) + (Fy[m] - Fyu)) + (Fzl[m] - Fzh[m]);
            Fzl[m] = Fzh[m];
        }
        // output operands of the two cells: U^n (stage 2) is issued now and
        // used after the next plane's conversion, so its latency overlaps it;
        // the input state at the cells is rebuilt from the ring at the output
        const long long j = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * z);
        float2 o1[NC], o2[NC];
        if (MODE == 2 && vec && in_bounds(j + 1, N, err)) {
#pragma unroll
            for (int m = 0; m < NC; ++m) o2[m] = ld2(Un + m * N + j);
        }

        // plane z+3 into the slot of z-1 (read only before the barrier above)
        if (z + 1 < z1) {
            bool use_stage = TMA && z + 3 < nz && !*tma_dead;
            if (use_stage && !tma_wait(mbar, parity, err)) {
                use_stage = false;
                *tma_dead = 1;
            }
            if (use_stage) {
                parity ^= 1u;
                if (tid == 0) outstanding = false;
                convert_staged(g, c, Uin, stage, ring + slot_of(z + 3), ox, oy, z + 3, xyint, err);
            } else {
                load_plane(g, c, Uin, ring + slot_of(z + 3), ox, oy, z + 3, xyint, err);
            }
        }

        if (in0 && in_bounds(j + (vec ? 1 : 0), N, err)) {
            const float2 ih = sp(c.inv_h), dt2 = sp(dt);
            // the input state at the two cells, rebuilt from the primitives
            // of plane z in the ring (a few FP32 roundings from the stored
            // values; saves holding them in registers across the conversion).
            // Cells of a ragged tile edge or an odd nx load it instead.
            auto u_from_ring = [&](float2 (&u)[NC]) {
                const float *P = ring + s0 + b;
                const float2 rh = ld2(P), vu = ld2(P + PP), vv = ld2(P + 2 * PP),
                             vw = ld2(P + 3 * PP), pr = ld2(P + 4 * PP);
                const float2 ke = fma2(vu, vu, fma2(vv, vv, vw * vw));
                u[0] = rh;
                u[1] = rh * vu;
                u[2] = rh * vv;
                u[3] = rh * vw;
                u[4] = fma2(pr, sp(c.inv_gm1), sp(0.5f) * rh * ke);
            };
            if (vec) {
                if (MODE != 0) u_from_ring(o1);
                if (MODE == 0) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) st2(out + m * N + j, acc[m] * ih);
                } else if (MODE == 1) {
#pragma unroll
                    for (int m = 0; m < NC; ++m) st2(out + m * N + j, fma2(dt2, acc[m] * ih, o1[m]));
                } else {
                    float ua[NC], ub[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        const float2 us =
                            fma2(sp(0.5f), o2[m], sp(0.5f) * fma2(dt2, acc[m] * ih, o1[m]));
                        st2(out + m * N + j, us);
                        ua[m] = us.x;
                        ub[m] = us.y;
                    }
                    if (!band_bit(band_bits, j)) smaxf = fmaxf(smaxf, rate_f(c, ua, ok));
                    if (!band_bit(band_bits, j + 1)) smaxf = fmaxf(smaxf, rate_f(c, ub, ok));
                }
            } else {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (k == 1 && !in1) break;
                    const long long jk = j + k;
                    float us[NC];
#pragma unroll
                    for (int m = 0; m < NC; ++m) {
                        const float a = (k == 0 ? acc[m].x : acc[m].y) * c.inv_h;
                        if (MODE == 0) {
                            out[m * N + jk] = a;
                        } else if (MODE == 1) {
                            out[m * N + jk] = fmaf(dt, a, __ldg(Uin + m * N + jk));
                        } else {
                            const float un = __ldg(Un + m * N + jk);
                            const float u1 = __ldg(Uin + m * N + jk);
                            us[m] = 0.5f * un + 0.5f * fmaf(dt, a, u1);
                            out[m * N + jk] = us[m];
                        }
                    }
                    if (MODE == 2 && !band_bit(band_bits, jk)) smaxf = fmaxf(smaxf, rate_f(c, us, ok));
                }
            }
        }
        __syncthreads();
        if (TMA && tid == 0 && !*tma_dead && z + 2 < z1 && z + 4 < nz) {
            tma_issue(&tmap, st_addr, mbar, ox - 4, oy - 2, z + 4);
            outstanding = true;
        }

    }

    // thread 0 flips its parity only on copies it saw complete, so `parity`
    // is the phase of a copy still outstanding
    if (TMA && tid == 0 && outstanding) tma_wait(mbar, parity, err);


    if (MODE == 2) {
        const double smax = warp_max_d((double)smaxf);
        const int bad = __syncthreads_or(!ok);
        if (lane == 0) s_red[warp] = smax;
        __syncthreads();
        if (tid == 0) {
            double m = s_red[0];
            for (int w = 1; w < NTH / 32; ++w) m = fmax(m, s_red[w]);
            blockmax[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = m;
            if (bad) record_error(err, ERR_NONFINITE);
        }
    }
}

}  // namespace

#ifndef IBM_ZM_WAVES
#define IBM_ZM_WAVES 3
#endif
#ifndef IBM_ZM_CHUNK
#define IBM_ZM_CHUNK 19
#endif

int zmarch_chunk(const GridParams &g) {
    // planes per CTA: enough CTAs to fill the GPU several times over (two
    // resident per SM).  At 256^3 (bench, ms per step): 16: 1.236, 19:
    // 1.220, 21: 1.251, 24: 1.227, 32: 1.27 - the wave count of the grid
    // (128 columns x 14 chunks = 5.9 waves at 19) matters as much as the
    // four-plane prologue of each chunk
    const long long cols = (long long)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY);
    int zc = IBM_ZM_CHUNK;
    while (zc > 4 && cols * ((g.n[2] + zc - 1) / zc) < IBM_ZM_WAVES * 2 * 152) zc /= 2;
    return zc;
}

size_t zmarch_blocks(const GridParams &g) {
    const int zc = zmarch_chunk(g);
    return (size_t)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY) * ((g.n[2] + zc - 1) / zc);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point
// (a driver function, the same for every device; resolved once, thread-safe)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuTensorMapEncodeTiled_v12000)p;
        return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
    }();
    return fn;
}

// 4D map over a conserved state: (x, y, z, component), box 40 x 20 x 1 x 5
static bool make_state_map(const GridParams &g, const void *U, CUtensorMap *map) {
    if (g.n[0] % 4 != 0 || ((uintptr_t)U) % 16 != 0) return false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.n[0], (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], NC};
    const cuuint64_t strides[3] = {(cuuint64_t)g.n[0] * 4, (cuuint64_t)g.n[0] * g.n[1] * 4,
                                   (cuuint64_t)g.N * 4};
    const cuuint32_t box[4] = {SBX, SBY, 1, NC};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(U), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MODE, bool TMA>
static cudaError_t zm_launch_t(const GridParams &g, const CUtensorMap &map, const void *Uin,
                               const void *Un, void *out, const FluidBuffers &fb, double dt_fixed,
                               cudaStream_t s) {
    cudaError_t e = func_smem_attr((const void *)zmarch_kernel<MODE, TMA>, SMEM, 100);
    if (e != cudaSuccess) return e;
    const int zc = zmarch_chunk(g);
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + zc - 1) / zc);
    zmarch_kernel<MODE, TMA><<<grid, NTH, SMEM, s>>>(map, g, make_fc(g), zc,
                                                     (const float *)Uin,
                                                     (const float *)Un, (float *)out, fb.blockmax,
                                                     fb.dt, fb.err, fb.band_bits, dt_fixed);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t zm_launch(const GridParams &g, const void *Uin, const void *Un, void *out,
                             const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (make_state_map(g, Uin, &map))
        return zm_launch_t<MODE, true>(g, map, Uin, Un, out, fb, dt_fixed, s);
    return zm_launch_t<MODE, false>(g, map, Uin, Un, out, fb, dt_fixed, s);
}

cudaError_t launch_zmarch(int mode, const GridParams &g, const void *Uin, const void *Un,
                          void *out, const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    if (mode == 1) return zm_launch<1>(g, Uin, Un, out, fb, dt_fixed, s);
    if (mode == 2) return zm_launch<2>(g, Uin, Un, out, fb, dt_fixed, s);
    return zm_launch<0>(g, Uin, Un, out, fb, dt_fixed, s);
}

}  // namespace ibmk
