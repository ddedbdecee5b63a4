// Fluid stages for 3D FP32 grids: the same discretisation as flux.cu
// (MUSCL/van Leer + Rusanov + central viscous/heat fluxes, SSP-RK2 stages),
// organised as a z-march for GB300.
//
// A CTA of 32 x 8 threads owns a 32 x 8 column of cells and walks up a chunk
// of z-planes.  Shared memory holds a ring of four primitive planes
// (z-1 .. z+2) with a two-cell halo in x and y, so every cell is loaded from
// memory and converted to primitives once per chunk (1.7x halo overhead
// instead of 3.4x for a cubic tile).  Per plane:
//   - one new plane is loaded (ghost cells through the boundary conditions),
//   - x- and y-faces of the plane are evaluated once each into shared face
//     rows (one warp per row, consecutive lanes on consecutive cells, so the
//     stencil loads are free of bank conflicts),
//   - the z-faces above the plane are evaluated by warps 0-3 (two columns
//     per thread as a packed pair) into a face buffer kept by plane parity,
//     so each plane's upper faces serve the next plane as its lower faces,
//   - each thread forms its cell's flux divergence and writes its output.
// All constants are single precision: the kernel issues no FP64 work
// except the per-CTA step-size maximum.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>
#include <stdint.h>
#include <string.h>

#include "internal.h"

namespace ibmk {
namespace {

constexpr int TX = 32, TY = 8, NTH = TX * TY;
constexpr int PX = TX + 4, PY = TY + 4, PP = PX * PY;   // plane with a 2-cell halo
constexpr int NW = 6;                                    // rho, u, v, w, p, T
constexpr int NC = 5;
constexpr int RING = 4;
constexpr int SLOT = NW * PP;
constexpr int FXW = TX + 1;                              // x-faces per row
// TMA staging box of one plane: x from ox-4 (16-byte aligned) over 40 cells,
// y from oy-2 over 12 rows, the five conserved components
constexpr int SBX = TX + 8, SBY = TY + 4;
constexpr int STAGE = NC * SBX * SBY;                    // floats
constexpr size_t SMEM_BASE =
    sizeof(float) * (size_t)(RING * SLOT + NC * TY * FXW + NC * (TY + 1) * TX + 2 * NC * TY * TX);
constexpr size_t SMEM_TMA_OFF = (SMEM_BASE + 127) / 128 * 128;
constexpr size_t SMEM = SMEM_TMA_OFF + sizeof(float) * STAGE + 16;   // + mbarrier
constexpr long long TMA_WAIT_LIMIT = 1ll << 20;          // bounded mbarrier waits

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

// ---- packed pairs: the x-face (.x) and the y-face (.y) of one thread ------
// Both faces run the same arithmetic once their velocity components are
// ordered (normal, tangential 1, tangential 2): the x-face takes (u, v, w),
// the y-face (v, u, w).  Each pair operation is one packed FP32x2
// instruction on sm_100-class GPUs.
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

// x-face between ring cells ax and ax+1 and y-face between ay and ay+PX of
// the same plane; up / dn move to the planes above and below.  Outputs in
// (rho, rho u, rho v, rho w, rho E) order.
__device__ __forceinline__ void face_xy(const FC &c, const float *__restrict__ R, int ax, int ay,
                                        int up, int dn, float (&Fx)[NC], float (&Fy)[NC]) {
    // field of (rho, normal, tangential 1, tangential 2, p) for each face
    constexpr int fx[NC] = {0, 1, 2, 3, 4};
    constexpr int fy[NC] = {0, 2, 1, 3, 4};
    float2 wl[NC], wr[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *X = R + fx[m] * PP;
        const float *Y = R + fy[m] * PP;
        const float2 x0 = make_float2(X[ax - 1], Y[ay - PX]);
        const float2 x1 = make_float2(X[ax], Y[ay]);
        const float2 x2 = make_float2(X[ax + 1], Y[ay + PX]);
        const float2 x3 = make_float2(X[ax + 2], Y[ay + 2 * PX]);
        const float2 d0 = x1 - x0, d1 = x2 - x1, d2 = x3 - x2;
        wl[m] = x1 + vlh2(d0, d1);
        wr[m] = x2 - vlh2(d1, d2);
    }
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
    const float2 mL1 = wl[0] * unL, mR1 = wr[0] * unR;
    const float2 mL2 = wl[0] * wl[2], mR2 = wr[0] * wr[2];
    const float2 mL3 = wl[0] * wl[3], mR3 = wr[0] * wr[3];
    float2 F0 = fma2(hs, wr[0] - wl[0], sp(0.5f) * (mL1 + mR1));
    float2 Fn = fma2(hs, mR1 - mL1, sp(0.5f) * (fma2(mL1, unL, wl[4]) + fma2(mR1, unR, wr[4])));
    float2 F1 = fma2(hs, mR2 - mL2, sp(0.5f) * fma2(mL2, unL, mR2 * unR));
    float2 F2 = fma2(hs, mR3 - mL3, sp(0.5f) * fma2(mL3, unL, mR3 * unR));
    float2 FE = fma2(hs, ER - EL, sp(0.5f) * fma2(EL + wl[4], unL, (ER + wr[4]) * unR));

    if (c.viscous) {
        const float *T = R + 5 * PP;
        const float2 Ta = make_float2(T[ax], T[ay]), Tb = make_float2(T[ax + 1], T[ay + PX]);
        const float2 Tf = sp(0.5f) * (Ta + Tb);
        const float2 mu = sp(c.mu_inf * c.onepS) * Tf * (Tf * rsqrt2(Tf)) * rcp2(Tf + sp(c.S));
        const float2 lam = mu * sp(c.lam_fac);
        const float *Xn = R + PP, *Yn = R + 2 * PP;       // normal velocity: u / v
        const float *X1 = R + 2 * PP, *Y1 = R + PP;       // tangential 1: v / u
        const float *W3 = R + 3 * PP;                     // tangential 2: w
        const int bx = ax + 1, by = ay + PX;
        const float2 ih = sp(c.inv_h), qh = sp(c.qinv_h);
        const float2 dn_n = (make_float2(Xn[bx], Yn[by]) - make_float2(Xn[ax], Yn[ay])) * ih;
        const float2 dn_1 = (make_float2(X1[bx], Y1[by]) - make_float2(X1[ax], Y1[ay])) * ih;
        const float2 dn_2 = (make_float2(W3[bx], W3[by]) - make_float2(W3[ax], W3[ay])) * ih;
        const float2 dn_T = (Tb - Ta) * ih;
        // along tangential 1 (y for the x-face, x for the y-face)
        const float2 d1_n = ((make_float2(Xn[ax + PX], Yn[ay + 1]) - make_float2(Xn[ax - PX], Yn[ay - 1])) +
                             (make_float2(Xn[bx + PX], Yn[by + 1]) - make_float2(Xn[bx - PX], Yn[by - 1]))) * qh;
        const float2 d1_1 = ((make_float2(X1[ax + PX], Y1[ay + 1]) - make_float2(X1[ax - PX], Y1[ay - 1])) +
                             (make_float2(X1[bx + PX], Y1[by + 1]) - make_float2(X1[bx - PX], Y1[by - 1]))) * qh;
        // along z
        const float2 d2_n = ((make_float2(Xn[ax + up], Yn[ay + up]) - make_float2(Xn[ax + dn], Yn[ay + dn])) +
                             (make_float2(Xn[bx + up], Yn[by + up]) - make_float2(Xn[bx + dn], Yn[by + dn]))) * qh;
        const float2 d2_2 = ((make_float2(W3[ax + up], W3[ay + up]) - make_float2(W3[ax + dn], W3[ay + dn])) +
                             (make_float2(W3[bx + up], W3[by + up]) - make_float2(W3[bx + dn], W3[by + dn]))) * qh;
        const float2 div = dn_n + d1_1 + d2_2;
        const float2 tNN = mu * fma2(sp(2.0f), dn_n, sp(-2.0f / 3.0f) * div);
        const float2 tN1 = mu * (d1_n + dn_1);
        const float2 tN2 = mu * (d2_n + dn_2);
        const float2 ufn = sp(0.5f) * (make_float2(Xn[ax], Yn[ay]) + make_float2(Xn[bx], Yn[by]));
        const float2 uf1 = sp(0.5f) * (make_float2(X1[ax], Y1[ay]) + make_float2(X1[bx], Y1[by]));
        const float2 uf2 = sp(0.5f) * (make_float2(W3[ax], W3[ay]) + make_float2(W3[bx], W3[by]));
        Fn = Fn - tNN;
        F1 = F1 - tN1;
        F2 = F2 - tN2;
        FE = FE - fma2(ufn, tNN, fma2(uf1, tN1, fma2(uf2, tN2, lam * dn_T)));
    }
    Fx[0] = F0.x; Fx[1] = Fn.x; Fx[2] = F1.x; Fx[3] = F2.x; Fx[4] = FE.x;
    Fy[0] = F0.y; Fy[1] = F1.y; Fy[2] = Fn.y; Fy[3] = F2.y; Fy[4] = FE.y;
}

// Two z-faces (columns A -> .x, B -> .y) between planes z (cells aA, aB) and
// z+1 (bA, bB) from given reconstructed states; tangential neighbours are
// +-1 (x) and +-PX (y) within each plane.
__device__ __forceinline__ void face_zz(const FC &c, const float *__restrict__ R, int aA, int bA,
                                        int aB, int bB, const float2 (&wl)[NC],
                                        const float2 (&wr)[NC], float2 (&F)[NC]) {
    const float2 keL = fma2(wl[1], wl[1], fma2(wl[2], wl[2], wl[3] * wl[3]));
    const float2 keR = fma2(wr[1], wr[1], fma2(wr[2], wr[2], wr[3] * wr[3]));
    const float2 EL = fma2(wl[4], sp(c.inv_gm1), sp(0.5f) * wl[0] * keL);
    const float2 ER = fma2(wr[4], sp(c.inv_gm1), sp(0.5f) * wr[0] * keR);
    const float2 unL = wl[3], unR = wr[3];
    const float2 c2L = sp(c.gamma) * wl[4] * rcp2(wl[0]);
    const float2 c2R = sp(c.gamma) * wr[4] * rcp2(wr[0]);
    const float2 sL = fma2(c2L, rsqrt2(c2L), abs2(unL));
    const float2 sR = fma2(c2R, rsqrt2(c2R), abs2(unR));
    const float2 hs = sp(-0.5f) * max2(sL, sR);
    const float2 mLn = wl[0] * unL, mRn = wr[0] * unR;
    const float2 mLu = wl[0] * wl[1], mRu = wr[0] * wr[1];
    const float2 mLv = wl[0] * wl[2], mRv = wr[0] * wr[2];
    F[0] = fma2(hs, wr[0] - wl[0], sp(0.5f) * (mLn + mRn));
    F[1] = fma2(hs, mRu - mLu, sp(0.5f) * fma2(mLu, unL, mRu * unR));
    F[2] = fma2(hs, mRv - mLv, sp(0.5f) * fma2(mLv, unL, mRv * unR));
    F[3] = fma2(hs, mRn - mLn, sp(0.5f) * (fma2(mLn, unL, wl[4]) + fma2(mRn, unR, wr[4])));
    F[4] = fma2(hs, ER - EL, sp(0.5f) * fma2(EL + wl[4], unL, (ER + wr[4]) * unR));
    if (!c.viscous) return;
    const float *T = R + 5 * PP, *U = R + PP, *V = R + 2 * PP, *Wz = R + 3 * PP;
    const float2 Ta = make_float2(T[aA], T[aB]), Tb = make_float2(T[bA], T[bB]);
    const float2 Tf = sp(0.5f) * (Ta + Tb);
    const float2 mu = sp(c.mu_inf * c.onepS) * Tf * (Tf * rsqrt2(Tf)) * rcp2(Tf + sp(c.S));
    const float2 lam = mu * sp(c.lam_fac);
    const float2 ih = sp(c.inv_h), qh = sp(c.qinv_h);
    auto P2 = [&](const float *f, int oA, int oB) { return make_float2(f[oA], f[oB]); };
    const float2 dn_w = (P2(Wz, bA, bB) - P2(Wz, aA, aB)) * ih;
    const float2 dn_u = (P2(U, bA, bB) - P2(U, aA, aB)) * ih;
    const float2 dn_v = (P2(V, bA, bB) - P2(V, aA, aB)) * ih;
    const float2 dn_T = (Tb - Ta) * ih;
    const float2 dx_w = ((P2(Wz, aA + 1, aB + 1) - P2(Wz, aA - 1, aB - 1)) +
                         (P2(Wz, bA + 1, bB + 1) - P2(Wz, bA - 1, bB - 1))) * qh;
    const float2 dy_w = ((P2(Wz, aA + PX, aB + PX) - P2(Wz, aA - PX, aB - PX)) +
                         (P2(Wz, bA + PX, bB + PX) - P2(Wz, bA - PX, bB - PX))) * qh;
    const float2 dx_u = ((P2(U, aA + 1, aB + 1) - P2(U, aA - 1, aB - 1)) +
                         (P2(U, bA + 1, bB + 1) - P2(U, bA - 1, bB - 1))) * qh;
    const float2 dy_v = ((P2(V, aA + PX, aB + PX) - P2(V, aA - PX, aB - PX)) +
                         (P2(V, bA + PX, bB + PX) - P2(V, bA - PX, bB - PX))) * qh;
    const float2 div = dn_w + dx_u + dy_v;
    const float2 tzz = mu * fma2(sp(2.0f), dn_w, sp(-2.0f / 3.0f) * div);
    const float2 tzx = mu * (dx_w + dn_u);
    const float2 tzy = mu * (dy_w + dn_v);
    const float2 ufw = sp(0.5f) * (P2(Wz, aA, aB) + P2(Wz, bA, bB));
    const float2 ufu = sp(0.5f) * (P2(U, aA, aB) + P2(U, bA, bB));
    const float2 ufv = sp(0.5f) * (P2(V, aA, aB) + P2(V, bA, bB));
    F[3] = F[3] - tzz;
    F[1] = F[1] - tzx;
    F[2] = F[2] - tzy;
    F[4] = F[4] - fma2(ufw, tzz, fma2(ufu, tzx, fma2(ufv, tzy, lam * dn_T)));
}

// half the limited z-slopes of two columns (A -> .x, B -> .y) at the middle plane
__device__ __forceinline__ void column_slope2(const float *__restrict__ R, int loA, int midA,
                                              int hiA, int loB, int midB, int hiB,
                                              float2 (&sig)[NC]) {
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *w = R + m * PP;
        const float2 lo = make_float2(w[loA], w[loB]), mid = make_float2(w[midA], w[midB]),
                     hi = make_float2(w[hiA], w[hiB]);
        sig[m] = vlh2(mid - lo, hi - mid);
    }
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

// Convert the staged plane gz into one ring slot.  Cells outside the domain in
// x or y (zero-filled by the copy) are taken through the boundary conditions.
__device__ __forceinline__ void convert_staged(const GridParams &g, const FC &c,
                                               const float *__restrict__ U,
                                               const float *__restrict__ st,
                                               float *__restrict__ slot, int ox, int oy, int gz,
                                               bool xy_interior) {
    const long long N = g.N;
    for (int q = threadIdx.x; q < PP; q += NTH) {
        const int lx = q % PX, ly = q / PX;
        const int gx = ox + lx - 2, gy = oy + ly - 2;
        float u[NC];
        if (xy_interior || (gx >= 0 && gx < g.n[0] && gy >= 0 && gy < g.n[1])) {
#pragma unroll
            for (int m = 0; m < NC; ++m) u[m] = st[(m * SBY + ly) * SBX + lx + 2];
        } else {
            int flip = 0, fs = 0;
            const int sx = map_axis(gx, g.n[0], g.bc[0], g.bc[1], 0, flip, fs);
            const int sy = map_axis(gy, g.n[1], g.bc[2], g.bc[3], 1, flip, fs);
            if (fs) {
                u[0] = 1.0f;
                u[1] = 1.0f;
                u[2] = 0.0f;
                u[3] = 0.0f;
                u[4] = c.E_inf;
            } else {
                const long long j = sx + (long long)g.n[0] * (sy + (long long)g.n[1] * gz);
#pragma unroll
                for (int m = 0; m < NC; ++m) u[m] = __ldg(U + m * N + j);
#pragma unroll
                for (int d = 0; d < 2; ++d)
                    if ((flip >> d) & 1) u[1 + d] = -u[1 + d];
            }
        }
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
}

// Load plane gz (ghosts through the boundary conditions) and convert it to
// primitives into one ring slot.
__device__ __forceinline__ void load_plane(const GridParams &g, const FC &c,
                                           const float *__restrict__ U, float *__restrict__ slot,
                                           int ox, int oy, int gz, bool xy_interior) {
    const long long N = g.N;
    const bool fast = xy_interior && gz >= 0 && gz < g.n[2];
    for (int q = threadIdx.x; q < PP; q += NTH) {
        const int lx = q % PX, ly = q / PX;
        float u[NC];
        if (fast) {
            const long long j = (ox + lx - 2) + (long long)g.n[0] * ((oy + ly - 2) + (long long)g.n[1] * gz);
#pragma unroll
            for (int m = 0; m < NC; ++m) u[m] = __ldg(U + m * N + j);
        } else {
            int flip = 0, fs = 0;
            const int sx = map_axis(ox + lx - 2, g.n[0], g.bc[0], g.bc[1], 0, flip, fs);
            const int sy = map_axis(oy + ly - 2, g.n[1], g.bc[2], g.bc[3], 1, flip, fs);
            const int sz = map_axis(gz, g.n[2], g.bc[4], g.bc[5], 2, flip, fs);
            if (fs) {
                u[0] = 1.0f;
                u[1] = 1.0f;
                u[2] = 0.0f;
                u[3] = 0.0f;
                u[4] = c.E_inf;
            } else {
                const long long j = sx + (long long)g.n[0] * (sy + (long long)g.n[1] * sz);
#pragma unroll
                for (int m = 0; m < NC; ++m) u[m] = __ldg(U + m * N + j);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if ((flip >> d) & 1) u[1 + d] = -u[1 + d];
            }
        }
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
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

#ifndef IBM_ZM_MIN_BLOCKS
#define IBM_ZM_MIN_BLOCKS 3
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
    float *FXb = ring + RING * SLOT;          // [NC][TY][FXW]
    float *FYb = FXb + NC * TY * FXW;         // [NC][TY+1][TX]
    float *FZb = FYb + NC * (TY + 1) * TX;    // [2][NC][TY][TX] upper z-faces by plane parity
    __shared__ double s_red[NTH / 32];

    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    const int ox = blockIdx.x * TX, oy = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.n[2]);
    const long long N = g.N;
    const float dt = MODE == 0 ? 0.0f : (float)(dt_fixed > 0.0 ? dt_fixed : *dt_ptr);
    const bool xyint = ox >= 2 && oy >= 2 && ox + TX + 2 <= g.n[0] && oy + TY + 2 <= g.n[1];
    auto slot_of = [](int z) { return ((z % RING) + RING) % RING * SLOT; };

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
    for (int zz = z0 - 2; zz <= z0 + 1; ++zz)
        load_plane(g, c, Uin, ring + slot_of(zz), ox, oy, zz, xyint);
    __syncthreads();

    // warps 0-3 own the z-faces of two cell rows each (2w -> .x, 2w+1 -> .y)
    const bool zwarp = ly < TY / 2;
    const int cA = (lx + 2) + PX * (2 * ly + 2), cB = cA + PX;
    if (zwarp) {       // z-face below the first plane (z0 - 1/2)
        const int sam = slot_of(z0 - 2), sa = slot_of(z0 - 1), sb = slot_of(z0), sbp = slot_of(z0 + 1);
        float2 sgA[NC], sig0[NC], wl[NC], wr[NC], F[NC];
        column_slope2(ring, sam + cA, sa + cA, sb + cA, sam + cB, sa + cB, sb + cB, sgA);
        column_slope2(ring, sa + cA, sb + cA, sbp + cA, sa + cB, sb + cB, sbp + cB, sig0);
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            wl[m] = make_float2(ring[sa + m * PP + cA], ring[sa + m * PP + cB]) + sgA[m];
            wr[m] = make_float2(ring[sb + m * PP + cA], ring[sb + m * PP + cB]) - sig0[m];
        }
        face_zz(c, ring, sa + cA, sb + cA, sa + cB, sb + cB, wl, wr, F);
        float *Fz = FZb + ((z0 - 1) & 1) * NC * TY * TX;
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            Fz[(m * TY + 2 * ly) * TX + lx] = F[m].x;
            Fz[(m * TY + 2 * ly + 1) * TX + lx] = F[m].y;
        }
    }
    __syncthreads();

    float smaxf = 0.0f;
    bool ok = true;
    for (int z = z0; z < z1; ++z) {
        bool use_stage = TMA && z + 2 < nz && !*tma_dead;
        if (use_stage && !tma_wait(mbar, parity, err)) {
            use_stage = false;
            *tma_dead = 1;
        }
        if (use_stage) {
            parity ^= 1u;
            if (tid == 0) outstanding = false;
            convert_staged(g, c, Uin, stage, ring + slot_of(z + 2), ox, oy, z + 2, xyint);
        } else {
            load_plane(g, c, Uin, ring + slot_of(z + 2), ox, oy, z + 2, xyint);
        }
        __syncthreads();
        if (TMA && tid == 0 && !*tma_dead && z + 1 < z1 && z + 3 < nz) {
            tma_issue(&tmap, st_addr, mbar, ox - 4, oy - 2, z + 3);
            outstanding = true;
        }
#if IBM_ZM_PREFETCH
        // stage 2 reads U^n at its output cells, which nothing has touched:
        // start those lines toward L2 two planes ahead
        if (MODE == 2 && z + 2 < z1 && ox + lx < g.n[0] && oy + ly < g.n[1]) {
            const long long jp = (ox + lx) + (long long)g.n[0] * ((oy + ly) + (long long)g.n[1] * (z + 2));
#pragma unroll
            for (int m = 0; m < NC; ++m)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(Un + m * N + jp));
        }
#endif
        const int sm1 = slot_of(z - 1), s0 = slot_of(z), s1 = slot_of(z + 1), s2 = slot_of(z + 2);
        const int up = s1 - s0, dn = sm1 - s0;
        // x-face lx of row ly (between cells lx-1 and lx) paired with y-face
        // row ly (between cell rows ly-1 and ly) of column lx
        {
            float Fx[NC], Fy[NC];
            face_xy(c, ring, s0 + (lx + 1) + PX * (ly + 2), s0 + (lx + 2) + PX * (ly + 1), up, dn,
                    Fx, Fy);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                FXb[(m * TY + ly) * FXW + lx] = Fx[m];
                FYb[(m * (TY + 1) + ly) * TX + lx] = Fy[m];
            }
        }
        if (zwarp) {
            // z-faces above two columns (between planes z and z+1).  The
            // plane-z slopes are taken again from the ring (planes z-1..z+1)
            // rather than carried from the previous plane: ten fewer registers
            // live through the loop (fewer spills; stage 2 0.735 -> 0.707 ms
            // at 256^3)
            float2 sig0[NC], sig1[NC], wl[NC], wr[NC], F[NC];
            column_slope2(ring, sm1 + cA, s0 + cA, s1 + cA, sm1 + cB, s0 + cB, s1 + cB, sig0);
            column_slope2(ring, s0 + cA, s1 + cA, s2 + cA, s0 + cB, s1 + cB, s2 + cB, sig1);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                wl[m] = make_float2(ring[s0 + m * PP + cA], ring[s0 + m * PP + cB]) + sig0[m];
                wr[m] = make_float2(ring[s1 + m * PP + cA], ring[s1 + m * PP + cB]) - sig1[m];
            }
            face_zz(c, ring, s0 + cA, s1 + cA, s0 + cB, s1 + cB, wl, wr, F);
            float *Fz = FZb + (z & 1) * NC * TY * TX;
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                Fz[(m * TY + 2 * ly) * TX + lx] = F[m].x;
                Fz[(m * TY + 2 * ly + 1) * TX + lx] = F[m].y;
            }
        } else if (ly == TY / 2) {
            // the last x-face of each row paired with the last y-face row
            float Fx[NC], Fy[NC];
            const int r = lx < TY ? lx : 0;
            face_xy(c, ring, s0 + (TX + 1) + PX * (r + 2), s0 + (lx + 2) + PX * (TY + 1), up, dn,
                    Fx, Fy);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                if (lx < TY) FXb[(m * TY + lx) * FXW + TX] = Fx[m];
                FYb[(m * (TY + 1) + TY) * TX + lx] = Fy[m];
            }
        }
        __syncthreads();

        float acc[NC];
        {
            const float *Fzl = FZb + ((z - 1) & 1) * NC * TY * TX;
            const float *Fzh = FZb + (z & 1) * NC * TY * TX;
#pragma unroll
            for (int m = 0; m < NC; ++m)
                acc[m] = (FXb[(m * TY + ly) * FXW + lx] - FXb[(m * TY + ly) * FXW + lx + 1]) +
                         (FYb[(m * (TY + 1) + ly) * TX + lx] - FYb[(m * (TY + 1) + ly + 1) * TX + lx]) +
                         (Fzl[(m * TY + ly) * TX + lx] - Fzh[(m * TY + ly) * TX + lx]);
        }
        const int gx = ox + lx, gy = oy + ly;
        if (gx < g.n[0] && gy < g.n[1]) {
            const long long j = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * z);
            if (MODE == 0) {
#pragma unroll
                for (int m = 0; m < NC; ++m) out[m * N + j] = acc[m] * c.inv_h;
            } else if (MODE == 1) {
#pragma unroll
                for (int m = 0; m < NC; ++m) out[m * N + j] = fmaf(dt, acc[m] * c.inv_h, __ldg(Uin + m * N + j));
            } else {
                float us[NC];
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const float un = __ldg(Un + m * N + j);
                    const float u1 = __ldg(Uin + m * N + j);
                    us[m] = 0.5f * un + 0.5f * fmaf(dt, acc[m] * c.inv_h, u1);
                    out[m * N + j] = us[m];
                }
                if (!band_bit(band_bits, j)) smaxf = fmaxf(smaxf, rate_f(c, us, ok));
            }
        }
    }

    // thread 0 flips its parity only on copies it saw complete, so `parity`
    // is the phase of a copy still outstanding
    if (TMA && tid == 0 && outstanding) tma_wait(mbar, parity, err);

    if (MODE == 2) {
        const double smax = warp_max_d((double)smaxf);
        const int bad = __syncthreads_or(!ok);
        if ((tid & 31) == 0) s_red[tid >> 5] = smax;
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

int zmarch_chunk(const GridParams &g) {
    // planes per CTA: enough CTAs to fill the GPU several times over.  At
    // 256^3, chunks of 19-24 planes measured 2.6 % faster per step than 32
    // (8 was 5 % slower, 43 3 %)
    const long long cols = (long long)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY);
    int zc = 24;
    while (zc > 8 && cols * ((g.n[2] + zc - 1) / zc) < 8 * 152) zc /= 2;
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

// 4D map over a conserved state: (x, y, z, component), box 40 x 12 x 1 x 5
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
    zmarch_kernel<MODE, TMA><<<grid, NTH, SMEM, s>>>(map, g, make_fc(g), zc, (const float *)Uin,
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
