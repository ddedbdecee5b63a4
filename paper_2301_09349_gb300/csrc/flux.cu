// Fluid stages of the IBM step: the explicit finite-volume discretisation of
// the compressible Navier-Stokes equations of Sec. 2.1 on a uniform grid.
//
//   L(U) = -(1/h) sum_d (Fhat_{i+1/2} - Fhat_{i-1/2}),
//   Fhat = Rusanov(MUSCL/van Leer states of (rho, u, p)) - viscous/heat flux,
//
// advanced by SSP-RK2 as the source-free predictor of App. B (step 1):
//   stage 1:  U^1 = U^n + dt L(U^n)
//   stage 2:  U* = U^n/2 + (U^1 + dt L(U^1))/2
// with dt = cfl / max_j s_j(U^n), formed at the end of the previous step (or
// by dt_init after a new state) so that stage 1 can write U^1 directly.
//
// Each CTA owns a BX x BY x BZ tile of cells.  It loads the tile plus a
// two-cell halo once (ghost cells mapped through the boundary conditions on
// the fly), converts to primitives in shared memory, then evaluates every
// face of the tile exactly once per direction into a shared face buffer and
// accumulates the flux differences in registers.
#include <atomic>
#include <float.h>

#include <type_traits>

#include "internal.h"

// the pair tiles leave some of BoxT's stride constants unused
#pragma nv_diag_suppress 177

namespace ibmk {
namespace {

constexpr int NT = 256;

constexpr int cmax(int a, int b) { return a > b ? a : b; }

// A BX x BY x BZ tile of cells with its two-cell halo, 256 threads.
template <int DIM_, typename T, int BX_, int BY_, int BZ_>
struct BoxT {
    static constexpr int DIM = DIM_;
    static constexpr int BX = BX_, BY = BY_, BZ = DIM_ == 3 ? BZ_ : 1;
    static constexpr int PX = BX + 4, PY = BY + 4, PZ = DIM == 3 ? BZ + 4 : 1;
    static constexpr int PN = PX * PY * PZ;          // cells in tile + halo
    static constexpr int NC = DIM + 2;               // conserved components
    static constexpr int NW = DIM + 3;               // rho, u.., p, T
    static constexpr int SX = 1, SY = PX, SZ = PX * PY;
    static constexpr int NCELL = BX * BY * BZ;
    static constexpr int CPT = (NCELL + NT - 1) / NT;
    static constexpr int NF0 = (BX + 1) * BY * BZ;
    static constexpr int NF1 = BX * (BY + 1) * BZ;
    static constexpr int NF2 = DIM == 3 ? BX * BY * (BZ + 1) : 0;
    static constexpr int NFMAX = cmax(NF0, cmax(NF1, NF2));
    // 2D FP32 tiles evaluate x- and y-faces together (pair layout: all x-face
    // rows, then all y-face rows)
    static constexpr bool PAIRS = DIM == 2 && sizeof(T) == 4;
    static constexpr int NFP = PAIRS ? NF0 + NF1 : 0;
    static constexpr size_t SMEM = sizeof(T) * (size_t)(NW * PN + NC * cmax(NFMAX, NFP));
};

// Tile of the single-grid kernels.
template <int DIM, typename T> struct DefaultBox;
template <> struct DefaultBox<3, float> { using type = BoxT<3, float, 8, 8, 8>; };
template <> struct DefaultBox<3, double> { using type = BoxT<3, double, 8, 8, 4>; };
template <> struct DefaultBox<2, float> { using type = BoxT<2, float, 16, 16, 1>; };
template <> struct DefaultBox<2, double> { using type = BoxT<2, double, 16, 16, 1>; };
template <int DIM, typename T> using Box = typename DefaultBox<DIM, T>::type;

// Small 2D FP64 grids: FP64 arithmetic runs at a small fraction of the FP32
// rate on this GPU, so the stage time of a grid with few 16 x 16 tiles is set
// by how many SMs take part; 8 x 8 tiles spread it over four times as many.
using SmallBox2D = BoxT<2, double, 8, 8, 1>;
inline bool small_2d_fp64(const GridParams &g) {
    return g.dim == 2 && (long long)((g.n[0] + 15) / 16) * ((g.n[1] + 15) / 16) < 256;
}
template <int DIM, typename T, bool SMALL>
using StageBox = typename std::conditional<SMALL, SmallBox2D, Box<DIM, T>>::type;

// 2D tile shapes of the batched kernel (all 256 cells): the autotuner's
// choices.  Every face is evaluated by the same arithmetic whatever the
// tile, so the shape changes the speed, never the result.
template <typename T, int S> struct Shape2;
template <typename T> struct Shape2<T, 0> { using type = BoxT<2, T, 16, 16, 1>; };
template <typename T> struct Shape2<T, 1> { using type = BoxT<2, T, 32, 8, 1>; };
template <typename T> struct Shape2<T, 2> { using type = BoxT<2, T, 64, 4, 1>; };
template <typename T> struct Shape2<T, 3> { using type = BoxT<2, T, 8, 32, 1>; };

// Arithmetic helpers.  FP32 uses the hardware approximations (MUFU
// reciprocal / reciprocal square root, ~2 ulp), which are far inside the
// FP32 parity tolerance; FP64 keeps correctly rounded division and sqrt.
template <typename T> __device__ __forceinline__ T fdiv(T a, T b);
template <> __device__ __forceinline__ float fdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv<double>(double a, double b) { return a / b; }

// sqrt of a positive argument
template <typename T> __device__ __forceinline__ T psqrt(T x);
template <> __device__ __forceinline__ float psqrt<float>(float x) { return x * rsqrtf(x); }
template <> __device__ __forceinline__ double psqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ T van_leer(T a, T b) {
    T ab = a * b;
    return ab > T(0) ? fdiv<T>(T(2) * ab, a + b) : T(0);
}

// The constants of the face flux in the compute type: FP32 kernels read the
// host-rounded copies, FP64 kernels the doubles (same values either way as
// converting in the kernel).
template <typename T> struct FluxK;
template <> struct FluxK<float> {
    float gam, inv_gm1, inv_h, S, mu_inf, lam_fac, gm1, invR, E_inf;
    bool viscous;
    __device__ __forceinline__ explicit FluxK(const GridParams &g)
        : gam(g.f.gamma), inv_gm1(g.f.inv_gm1), inv_h(g.f.inv_h), S(g.f.S), mu_inf(g.f.mu_inf),
          lam_fac(g.f.lam_fac), gm1(g.f.gm1), invR(g.f.invR), E_inf(g.f.E_inf),
          viscous(g.f.viscous != 0) {}
};
template <> struct FluxK<double> {
    double gam, inv_gm1, inv_h, S, mu_inf, lam_fac, gm1, invR, E_inf;
    bool viscous;
    __device__ __forceinline__ explicit FluxK(const GridParams &g)
        : gam(g.gamma), inv_gm1(1.0 / (g.gamma - 1.0)), inv_h(g.inv_h), S(g.S), mu_inf(g.mu_inf),
          lam_fac(g.cp / g.Pr), gm1(g.gamma - 1.0), invR(1.0 / g.R),
          E_inf(g.p_inf / (g.gamma - 1.0) + 0.5), viscous(g.mu_inf > 0.0) {}
};

// Numerical flux through the face between box cells a and a + s_D.
template <typename B, typename T, int D>
__device__ __forceinline__ void face_flux(const FluxK<T> &k, const T *__restrict__ sW, int a,
                                          T (&F)[B::DIM + 2]) {
    constexpr int DIM = B::DIM;
    constexpr int s = D == 0 ? B::SX : (D == 1 ? B::SY : B::SZ);
    constexpr int NC = DIM + 2;
    const int b = a + s;
    const T gam = k.gam;
    const T inv_gm1 = k.inv_gm1;

    // MUSCL reconstruction of (rho, u.., p) with the van Leer limiter
    T wl[NC], wr[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const T *w = sW + m * B::PN;
        T wam = w[a - s], wa = w[a], wb = w[b], wbp = w[b + s];
        T d0 = wa - wam, d1 = wb - wa, d2 = wbp - wb;
        wl[m] = wa + T(0.5) * van_leer(d0, d1);
        wr[m] = wb - T(0.5) * van_leer(d1, d2);
    }

    // Rusanov flux: (F_L + F_R)/2 - s_max (U_R - U_L)/2
    T keL = 0, keR = 0;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        keL += wl[1 + m] * wl[1 + m];
        keR += wr[1 + m] * wr[1 + m];
    }
    const T EL = wl[NC - 1] * inv_gm1 + T(0.5) * wl[0] * keL;
    const T ER = wr[NC - 1] * inv_gm1 + T(0.5) * wr[0] * keR;
    const T unL = wl[1 + D], unR = wr[1 + D];
    const T cL = psqrt<T>(fdiv<T>(gam * wl[NC - 1], wl[0]));
    const T cR = psqrt<T>(fdiv<T>(gam * wr[NC - 1], wr[0]));
    const T sL = fabs(unL) + cL, sR = fabs(unR) + cR;
    const T smax = sL > sR ? sL : sR;
    F[0] = T(0.5) * (wl[0] * unL + wr[0] * unR) - T(0.5) * smax * (wr[0] - wl[0]);
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        T mL = wl[0] * wl[1 + m], mR = wr[0] * wr[1 + m];
        T fL = mL * unL + (m == D ? wl[NC - 1] : T(0));
        T fR = mR * unR + (m == D ? wr[NC - 1] : T(0));
        F[1 + m] = T(0.5) * (fL + fR) - T(0.5) * smax * (mR - mL);
    }
    F[NC - 1] = T(0.5) * ((EL + wl[NC - 1]) * unL + (ER + wr[NC - 1]) * unR) -
                T(0.5) * smax * (ER - EL);

    if (!k.viscous) return;

    // viscous stress and heat flux; face values from the two adjacent cells,
    // tangential derivatives from the average of the two cells' central
    // differences
    const T inv_h = k.inv_h;
    const T *Tc = sW + (DIM + 2) * B::PN;
    const T Tf = T(0.5) * (Tc[a] + Tc[b]);
    const T Sv = k.S;
    const T mu = fdiv<T>(k.mu_inf * Tf * psqrt<T>(Tf) * (T(1) + Sv), Tf + Sv);
    const T lam = mu * k.lam_fac;
    T grad[DIM][DIM];
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        const T *um = sW + (1 + m) * B::PN;
#pragma unroll
        for (int e = 0; e < DIM; ++e) {
            if (e == D) {
                grad[m][e] = (um[b] - um[a]) * inv_h;
            } else {
                const int t = e == 0 ? B::SX : (e == 1 ? B::SY : B::SZ);
                grad[m][e] = (um[a + t] - um[a - t] + um[b + t] - um[b - t]) * (T(0.25) * inv_h);
            }
        }
    }
    T div = 0;
#pragma unroll
    for (int m = 0; m < DIM; ++m) div += grad[m][m];
    T work = 0;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        T tau = mu * (grad[D][m] + grad[m][D]);
        if (m == D) tau -= T(2.0 / 3.0) * mu * div;
        const T *um = sW + (1 + m) * B::PN;
        const T uf = T(0.5) * (um[a] + um[b]);
        F[1 + m] -= tau;
        work += uf * tau;
    }
    F[NC - 1] -= work + lam * (Tc[b] - Tc[a]) * inv_h;
}

// ---- 2D FP32: the x-face (.x) and the y-face (.y) of a thread as one pair --
// Both faces run the same arithmetic with their velocities ordered (normal,
// tangential); every pair operation is one packed FP32x2 instruction.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return fsub2_ftz(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_s(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 p_rcp(float2 a) {
    return make_float2(__fdividef(1.0f, a.x), __fdividef(1.0f, a.y));
}
__device__ __forceinline__ float2 p_rsqrt(float2 a) { return make_float2(rsqrtf(a.x), rsqrtf(a.y)); }
__device__ __forceinline__ float2 p_abs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 p_max(float2 a, float2 b) {
    return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
// half the van Leer slope, ab / (a + b) where ab > 0: the face states are
// w +- psi/2, and the factor 2 of psi = 2ab/(a+b) and the 1/2 cancel exactly
__device__ __forceinline__ float2 p_vlh(float2 a, float2 b) {
    const float2 ab = p_mul(a, b);
    const float2 q = p_mul(ab, p_rcp(p_add(a, b)));
    return make_float2(ab.x > 0.0f ? q.x : 0.0f, ab.y > 0.0f ? q.y : 0.0f);
}

// x-face between box cells ax, ax+1 and y-face between ay, ay+PX; outputs in
// (rho, rho u, rho v, rho E) order.  The same flux as face_flux: MUSCL/van
// Leer states, Rusanov, central viscous stress and heat flux.
template <int PX, int PN>
__device__ __forceinline__ void face_pair2d(const FluxK<float> &k, const float *__restrict__ sW,
                                            int ax, int ay, float (&Fx)[4], float (&Fy)[4]) {
    constexpr int fx[4] = {0, 1, 2, 3};   // rho, normal, tangential, p
    constexpr int fy[4] = {0, 2, 1, 3};
    float2 wl[4], wr[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float *X = sW + fx[m] * PN;
        const float *Y = sW + fy[m] * PN;
        const float2 x0 = make_float2(X[ax - 1], Y[ay - PX]);
        const float2 x1 = make_float2(X[ax], Y[ay]);
        const float2 x2 = make_float2(X[ax + 1], Y[ay + PX]);
        const float2 x3 = make_float2(X[ax + 2], Y[ay + 2 * PX]);
        const float2 d0 = p_sub(x1, x0), d1 = p_sub(x2, x1), d2 = p_sub(x3, x2);
        wl[m] = p_add(x1, p_vlh(d0, d1));
        wr[m] = p_sub(x2, p_vlh(d1, d2));
    }
    const float2 keL = p_fma(wl[1], wl[1], p_mul(wl[2], wl[2]));
    const float2 keR = p_fma(wr[1], wr[1], p_mul(wr[2], wr[2]));
    const float2 EL = p_fma(wl[3], p_s(k.inv_gm1), p_mul(p_mul(p_s(0.5f), wl[0]), keL));
    const float2 ER = p_fma(wr[3], p_s(k.inv_gm1), p_mul(p_mul(p_s(0.5f), wr[0]), keR));
    const float2 unL = wl[1], unR = wr[1];
    const float2 c2L = p_mul(p_mul(p_s(k.gam), wl[3]), p_rcp(wl[0]));
    const float2 c2R = p_mul(p_mul(p_s(k.gam), wr[3]), p_rcp(wr[0]));
    const float2 sL = p_fma(c2L, p_rsqrt(c2L), p_abs(unL));
    const float2 sR = p_fma(c2R, p_rsqrt(c2R), p_abs(unR));
    const float2 hs = p_mul(p_s(-0.5f), p_max(sL, sR));   // -smax/2
    const float2 mLn = p_mul(wl[0], unL), mRn = p_mul(wr[0], unR);
    const float2 mLt = p_mul(wl[0], wl[2]), mRt = p_mul(wr[0], wr[2]);
    float2 F0 = p_fma(hs, p_sub(wr[0], wl[0]), p_mul(p_s(0.5f), p_add(mLn, mRn)));
    float2 Fn = p_fma(hs, p_sub(mRn, mLn),
                      p_mul(p_s(0.5f), p_add(p_fma(mLn, unL, wl[3]), p_fma(mRn, unR, wr[3]))));
    float2 Ft = p_fma(hs, p_sub(mRt, mLt), p_mul(p_s(0.5f), p_fma(mLt, unL, p_mul(mRt, unR))));
    float2 FE = p_fma(hs, p_sub(ER, EL),
                      p_mul(p_s(0.5f), p_fma(p_add(EL, wl[3]), unL, p_mul(p_add(ER, wr[3]), unR))));
    if (k.viscous) {
        const float *T = sW + 4 * PN;
        const int bx = ax + 1, by = ay + PX;
        const float2 Ta = make_float2(T[ax], T[ay]), Tb = make_float2(T[bx], T[by]);
        const float2 Tf = p_mul(p_s(0.5f), p_add(Ta, Tb));
        const float2 mu = p_mul(p_mul(p_mul(p_s(k.mu_inf), Tf), p_mul(Tf, p_rsqrt(Tf))),
                                p_mul(p_s(1.0f + k.S), p_rcp(p_add(Tf, p_s(k.S)))));
        const float2 lam = p_mul(mu, p_s(k.lam_fac));
        const float *Xn = sW + PN, *Yn = sW + 2 * PN;     // normal velocity: u / v
        const float *Xt = sW + 2 * PN, *Yt = sW + PN;     // tangential velocity: v / u
        const float2 ih = p_s(k.inv_h), qh = p_s(0.25f * k.inv_h);
        const float2 na = make_float2(Xn[ax], Yn[ay]), nb = make_float2(Xn[bx], Yn[by]);
        const float2 ta = make_float2(Xt[ax], Yt[ay]), tb = make_float2(Xt[bx], Yt[by]);
        const float2 dn_n = p_mul(p_sub(nb, na), ih);
        const float2 dn_t = p_mul(p_sub(tb, ta), ih);
        const float2 dn_T = p_mul(p_sub(Tb, Ta), ih);
        // along the tangent (y for the x-face, x for the y-face)
        const float2 d1_n = p_mul(p_add(p_sub(make_float2(Xn[ax + PX], Yn[ay + 1]),
                                              make_float2(Xn[ax - PX], Yn[ay - 1])),
                                        p_sub(make_float2(Xn[bx + PX], Yn[by + 1]),
                                              make_float2(Xn[bx - PX], Yn[by - 1]))), qh);
        const float2 d1_t = p_mul(p_add(p_sub(make_float2(Xt[ax + PX], Yt[ay + 1]),
                                              make_float2(Xt[ax - PX], Yt[ay - 1])),
                                        p_sub(make_float2(Xt[bx + PX], Yt[by + 1]),
                                              make_float2(Xt[bx - PX], Yt[by - 1]))), qh);
        const float2 div = p_add(dn_n, d1_t);
        const float2 tNN = p_mul(mu, p_fma(p_s(2.0f), dn_n, p_mul(p_s(-2.0f / 3.0f), div)));
        const float2 tNT = p_mul(mu, p_add(d1_n, dn_t));
        const float2 ufn = p_mul(p_s(0.5f), p_add(na, nb));
        const float2 uft = p_mul(p_s(0.5f), p_add(ta, tb));
        Fn = p_sub(Fn, tNN);
        Ft = p_sub(Ft, tNT);
        FE = p_sub(FE, p_fma(ufn, tNN, p_fma(uft, tNT, p_mul(lam, dn_T))));
    }
    Fx[0] = F0.x; Fx[1] = Fn.x; Fx[2] = Ft.x; Fx[3] = FE.x;
    Fy[0] = F0.y; Fy[1] = Ft.y; Fy[2] = Fn.y; Fy[3] = FE.y;
}

// All faces of a 2D FP32 tile in one pass: thread (cx, cy) evaluates the
// x-face on the left of its cell and the y-face below it; the BY faces on
// the right edge and the BX faces on the top edge follow as further pairs
// on the first warps.  acc receives each cell's flux differences.
template <typename B>
__device__ __forceinline__ void pair_faces_2d(const FluxK<float> &k, const float *__restrict__ sW,
                                              float *__restrict__ sF, float (&acc)[1][4]) {
    constexpr int BX = B::BX, BY = B::BY, PX = B::PX, PN = B::PN;
    constexpr int FXW = BX + 1, NXF = FXW * BY, NYF = BX * (BY + 1);
    float *FX = sF, *FY = sF + 4 * NXF;     // [4][BY][BX+1], [4][BY+1][BX]
    const int tid = threadIdx.x;
    const int cx = tid % BX, cy = tid / BX;
    {
        float Fx[4], Fy[4];
        face_pair2d<PX, PN>(k, sW, (cx + 1) + PX * (cy + 2), (cx + 2) + PX * (cy + 1), Fx, Fy);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            FX[c * NXF + cy * FXW + cx] = Fx[c];
            FY[c * NYF + cy * BX + cx] = Fy[c];
        }
    }
    constexpr int NE = BX > BY ? BX : BY;
    if (tid < NE) {
        const int ex = tid < BY ? tid : 0, ey = tid < BX ? tid : 0;
        float Fx[4], Fy[4];
        face_pair2d<PX, PN>(k, sW, (BX + 1) + PX * (ex + 2), (ey + 2) + PX * (BY + 1), Fx, Fy);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (tid < BY) FX[c * NXF + ex * FXW + BX] = Fx[c];
            if (tid < BX) FY[c * NYF + BY * BX + ey] = Fy[c];
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 4; ++c)
        acc[0][c] = (FX[c * NXF + cy * FXW + cx] - FX[c * NXF + cy * FXW + cx + 1]) +
                    (FY[c * NYF + cy * BX + cx] - FY[c * NYF + (cy + 1) * BX + cx]);
    __syncthreads();
}

// One direction: evaluate all faces of the tile normal to axis D, then add
// each cell's flux difference to its accumulator.
template <typename B, typename T, int D>
__device__ __forceinline__ void direction_pass(const FluxK<T> &k, const T *__restrict__ sW,
                                               T *__restrict__ sF, T (&acc)[B::CPT][B::DIM + 2]) {
    constexpr int DIM = B::DIM;
    constexpr int NC = DIM + 2;
    constexpr int dx = D == 0, dy = D == 1, dz = (D == 2 && DIM == 3);
    constexpr int FX = B::BX + dx, FY = B::BY + dy, FZ = B::BZ + dz;
    constexpr int NF = FX * FY * FZ;
    for (int f = threadIdx.x; f < NF; f += NT) {
        const int fx = f % FX;
        const int r = f / FX;
        const int fy = r % FY;
        const int fz = r / FY;
        const int a = (fx - dx + 2) + B::PX * (fy - dy + 2) +
                      (DIM == 3 ? B::PX * B::PY * (fz - dz + 2) : 0);
        T F[NC];
        face_flux<B, T, D>(k, sW, a, F);
#pragma unroll
        for (int c = 0; c < NC; ++c) sF[c * B::NFMAX + f] = F[c];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < B::CPT; ++i) {
        const int cell = threadIdx.x + i * NT;
        if (cell < B::NCELL) {
            const int cx = cell % B::BX;
            const int cy = (cell / B::BX) % B::BY;
            const int cz = cell / (B::BX * B::BY);
            const int flo = cx + FX * (cy + FY * cz);
            const int fhi = (cx + dx) + FX * ((cy + dy) + FY * (cz + dz));
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[i][c] += sF[c * B::NFMAX + flo] - sF[c * B::NFMAX + fhi];
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One tile of one stage.  MODE 0: out = L(Uin).  MODE 1: out = U1 = Uin +
// dt L(Uin).  MODE 2: out = U* = Un/2 + (Uin + dt L(Uin))/2 with Uin = U1,
// and the maximum of s_j(U*) over the tile's cells outside the band is
// returned to thread 0 (every thread must call; the function synchronises;
// a later call may reuse s_red only after its own first barrier).
template <typename B, typename T, int MODE>
__device__ __forceinline__ double stage_tile(const GridParams &g, int ox, int oy, int oz,
                                             const T *__restrict__ Uin, const T *__restrict__ Un,
                                             T *__restrict__ out, const T dt,
                                             const unsigned *__restrict__ band_bits,
                                             unsigned char *smem_raw, double *s_red, bool &bad,
                                             int *err) {
    constexpr int DIM = B::DIM;
    constexpr int NC = DIM + 2;
    T *sW = reinterpret_cast<T *>(smem_raw);
    T *sF = sW + B::NW * B::PN;

    const int tid = threadIdx.x;
    const long long N = g.N;
    const FluxK<T> k(g);
    const T gm1 = k.gm1;
    const T invR = k.invR;

    // ---- load tile + halo, to primitives
    // Tiles whose halo lies inside the domain index directly; the others map
    // every halo index through the boundary conditions.
    const bool interior = ox >= 2 && oy >= 2 && ox + B::BX + 2 <= g.n[0] &&
                          oy + B::BY + 2 <= g.n[1] &&
                          (DIM == 2 || (oz >= 2 && oz + B::BZ + 2 <= g.n[2]));
    const T p_inf_E = k.E_inf;
    for (int q = tid; q < B::PN; q += NT) {
        const int lx = q % B::PX;
        const int r = q / B::PX;
        const int ly = r % B::PY;
        const int lz = r / B::PY;
        T u[NC];
        if (interior) {
            const long long j = (ox + lx - 2) +
                                (long long)g.n[0] * ((oy + ly - 2) + (long long)g.n[1] * (oz + lz - 2 * (DIM == 3)));
            const bool okj = in_bounds(j, N, err);
#pragma unroll
            for (int c = 0; c < NC; ++c) u[c] = okj ? __ldg(Uin + c * N + j) : T(0);
        } else {
            int flip = 0, fs = 0;
            const int sx = map_axis(ox + lx - 2, g.n[0], g.bc[0], g.bc[1], 0, flip, fs);
            const int sy = map_axis(oy + ly - 2, g.n[1], g.bc[2], g.bc[3], 1, flip, fs);
            const int sz = DIM == 3 ? map_axis(oz + lz - 2, g.n[2], g.bc[4], g.bc[5], 2, flip, fs) : 0;
            if (fs) {
                u[0] = T(1);
                u[1] = T(1);
#pragma unroll
                for (int d = 1; d < DIM; ++d) u[1 + d] = T(0);
                u[NC - 1] = p_inf_E;
            } else {
                const long long j = sx + (long long)g.n[0] * (sy + (long long)g.n[1] * sz);
                const bool okj = in_bounds(j, N, err);
#pragma unroll
                for (int c = 0; c < NC; ++c) u[c] = okj ? __ldg(Uin + c * N + j) : T(0);
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    if ((flip >> d) & 1) u[1 + d] = -u[1 + d];
            }
        }
        const T rho = u[0];
        const T inv = fdiv<T>(T(1), rho);
        T ke = 0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T v = u[1 + d] * inv;
            sW[(1 + d) * B::PN + q] = v;
            ke += v * v;
        }
        const T p = gm1 * (u[NC - 1] - T(0.5) * rho * ke);
        sW[q] = rho;
        sW[(DIM + 1) * B::PN + q] = p;
        sW[(DIM + 2) * B::PN + q] = p * inv * invR;
    }
    __syncthreads();

    // ---- faces, one direction at a time
    T acc[B::CPT][NC];
#pragma unroll
    for (int i = 0; i < B::CPT; ++i)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[i][c] = T(0);
    if constexpr (B::PAIRS) {
        static_assert(B::NCELL == NT, "pair tiles hold one cell per thread");
        pair_faces_2d<B>(k, sW, sF, acc);
    } else {
        direction_pass<B, T, 0>(k, sW, sF, acc);
        direction_pass<B, T, 1>(k, sW, sF, acc);
        if constexpr (DIM == 3) direction_pass<B, T, 2>(k, sW, sF, acc);
    }

    // ---- outputs
    const T inv_h = k.inv_h;
    T smax_t = T(0);   // in the compute type: one conversion per tile, not per cell
    bool ok = true;
#pragma unroll
    for (int i = 0; i < B::CPT; ++i) {
        const int cell = tid + i * NT;
        if (cell >= B::NCELL) continue;
        const int cx = cell % B::BX;
        const int cy = (cell / B::BX) % B::BY;
        const int cz = cell / (B::BX * B::BY);
        const int gx = ox + cx, gy = oy + cy, gz = oz + cz;
        if (gx >= g.n[0] || gy >= g.n[1] || (DIM == 3 && gz >= g.n[2])) continue;
        const long long j = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
        if (!in_bounds(j, N, err)) continue;
        if (MODE == 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c * N + j] = acc[i][c] * inv_h;
        } else if (MODE == 1) {
#pragma unroll
            for (int c = 0; c < NC; ++c) out[c * N + j] = __ldg(Uin + c * N + j) + dt * (acc[i][c] * inv_h);
        } else {
            T us[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const T un = __ldg(Un + c * N + j);
                const T u1 = __ldg(Uin + c * N + j);
                us[c] = T(0.5) * un + T(0.5) * (u1 + dt * (acc[i][c] * inv_h));
                out[c * N + j] = us[c];
            }
            if (!band_bit(band_bits, j)) {
                const T sj = step_rate<DIM, T>(g, us, ok);
                smax_t = fmax(smax_t, sj);
            }
        }
    }

    if (MODE == 2) {
        // the tile's maximum in the compute type (exact), widened once
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax_t = fmax(smax_t, __shfl_xor_sync(0xffffffffu, smax_t, o));
        bad = __syncthreads_or(!ok) != 0;
        if ((tid & 31) == 0) s_red[tid >> 5] = (double)smax_t;
        __syncthreads();
        if (tid != 0) return 0.0;
        double m = s_red[0];
        for (int w = 1; w < NT / 32; ++w) m = fmax(m, s_red[w]);
        return m;
    }
    return 0.0;
}

template <int DIM, typename T, int MODE, bool SMALL>
__global__ void __launch_bounds__(NT)
stage_kernel(const GridParams g, const T *__restrict__ Uin, const T *__restrict__ Un,
             T *__restrict__ out, double *__restrict__ blockmax, const double *__restrict__ dt_ptr,
             int *__restrict__ err, const unsigned *__restrict__ band_bits, double dt_fixed) {
    using B = StageBox<DIM, T, SMALL>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[NT / 32];
    const int ox = blockIdx.x * B::BX, oy = blockIdx.y * B::BY;
    const int oz = DIM == 3 ? blockIdx.z * B::BZ : 0;
    const T dt = MODE == 0 ? T(0) : (T)(dt_fixed > 0.0 ? dt_fixed : *dt_ptr);
    bool bad = false;
    const double m = stage_tile<B, T, MODE>(g, ox, oy, oz, Uin, Un, out, dt, band_bits, smem_raw,
                                            s_red, bad, err);
    if (MODE == 2 && threadIdx.x == 0) {
        blockmax[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = m;
        if (bad) record_error(err, ERR_NONFINITE);
    }
}

// The same stages over a batch of 2D grids: one persistent launch walks a
// list of (case, tile) work items; every case keeps its own parameters,
// state, step size and error word.  MODE 2 writes one maximum per item.
// FP32: five CTAs per SM (48 registers, a few bytes of spill): measured
// faster on the 64-case batch than four (64 registers) or three
#ifndef IBM_BATCH_MIN_BLOCKS
#define IBM_BATCH_MIN_BLOCKS 5
#endif
template <typename T, int S, int MODE>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? IBM_BATCH_MIN_BLOCKS : 1)
batch_stage_kernel(const BatchCase *__restrict__ cases, const int2 *__restrict__ items,
                   int n_items, double *__restrict__ item_max, double dt_fixed) {
    using B = typename Shape2<T, S>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double s_red[NT / 32];
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = items[it];
        const BatchCase &bc = cases[w.x];
        const GridParams g = bc.g;
        const int ntx = (g.n[0] + B::BX - 1) / B::BX;
        const int ox = (w.y % ntx) * B::BX, oy = (w.y / ntx) * B::BY;
        const T dt = MODE == 0 ? T(0) : (T)(dt_fixed > 0.0 ? dt_fixed : *bc.dt);
        const T *Uin = (const T *)(MODE == 2 ? bc.U1 : bc.Un);
        T *out = (T *)(MODE == 2 ? bc.Us : bc.U1);
        bool bad = false;
        const double m = stage_tile<B, T, MODE>(g, ox, oy, 0, Uin, (const T *)bc.Un, out, dt,
                                                bc.band_bits, smem_raw, s_red, bad, bc.err);
        if (MODE == 2 && threadIdx.x == 0) {
            item_max[it] = m;
            if (bad) record_error(bc.err, ERR_NONFINITE);
        }
    }
}

// *dt = cfl / max_j s_j(U) over every cell: per-CTA maxima, then the last
// CTA to finish reduces them.
template <int DIM, typename T>
__global__ void __launch_bounds__(NT)
dt_init_kernel(const GridParams g, const T *__restrict__ U, double *__restrict__ blockmax,
               unsigned *__restrict__ counter, double *__restrict__ dt, int *__restrict__ err) {
    constexpr int NC = DIM + 2;
    __shared__ double s_red[NT / 32];
    __shared__ int s_last;
    const long long N = g.N;
    const long long j0 = (long long)blockIdx.x * DT_CELLS_PER_CTA;
    const long long j1 = j0 + DT_CELLS_PER_CTA < N ? j0 + DT_CELLS_PER_CTA : N;
    double smax = 0.0;
    bool ok = true;
    for (long long j = j0 + threadIdx.x; j < j1; j += NT) {
        T u[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = U[c * N + j];
        smax = fmax(smax, (double)step_rate<DIM, T>(g, u, ok));
    }
    smax = warp_max(smax);
    const int bad = __syncthreads_or(!ok);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = smax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = s_red[0];
        for (int w = 1; w < NT / 32; ++w) m = fmax(m, s_red[w]);
        blockmax[blockIdx.x] = m;
        if (bad) record_error(err, ERR_NONFINITE);
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double m = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += NT) m = fmax(m, __ldcg(blockmax + b));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = s_red[0];
        for (int w = 1; w < NT / 32; ++w) mm = fmax(mm, s_red[w]);
        const bool good = mm > 0.0 && mm <= DBL_MAX && !(__ldcg(err) & ERR_NONFINITE);
        if (!good) record_error(err, ERR_NONFINITE);
        *dt = good ? g.cfl / mm : 0.0;
        *counter = 0u;
    }
}

template <int DIM, typename T, bool SMALL = false>
dim3 stage_grid(const GridParams &g) {
    using B = StageBox<DIM, T, SMALL>;
    return dim3((g.n[0] + B::BX - 1) / B::BX, (g.n[1] + B::BY - 1) / B::BY,
                DIM == 3 ? (g.n[2] + B::BZ - 1) / B::BZ : 1);
}

template <int DIM, typename T, int MODE, bool SMALL>
cudaError_t launch_box(const GridParams &g, const void *Uin, const void *Un, void *out,
                       const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    using B = StageBox<DIM, T, SMALL>;
    cudaError_t e = func_smem_attr((const void *)stage_kernel<DIM, T, MODE, SMALL>, B::SMEM);
    if (e != cudaSuccess) return e;
    stage_kernel<DIM, T, MODE, SMALL><<<stage_grid<DIM, T, SMALL>(g), NT, B::SMEM, s>>>(
        g, (const T *)Uin, (const T *)Un, (T *)out, fb.blockmax, fb.dt, fb.err, fb.band_bits,
        dt_fixed);
    return cudaGetLastError();
}

template <int DIM, typename T, int MODE>
cudaError_t launch_one(const GridParams &g, const void *Uin, const void *Un, void *out,
                       const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    if (DIM == 2 && sizeof(T) == 8 && small_2d_fp64(g))
        return launch_box<DIM, T, MODE, DIM == 2 && sizeof(T) == 8>(g, Uin, Un, out, fb, dt_fixed, s);
    return launch_box<DIM, T, MODE, false>(g, Uin, Un, out, fb, dt_fixed, s);
}

template <int MODE>
cudaError_t dispatch(const GridParams &g, int fp_bytes, const void *Uin, const void *Un, void *out,
                     const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    if (g.dim == 3) {
        if (fp_bytes == 4) return launch_zmarch(MODE, g, Uin, Un, out, fb, dt_fixed, s);
        return launch_one<3, double, MODE>(g, Uin, Un, out, fb, dt_fixed, s);
    }
    if (fp_bytes == 4) return launch_one<2, float, MODE>(g, Uin, Un, out, fb, dt_fixed, s);
    return launch_one<2, double, MODE>(g, Uin, Un, out, fb, dt_fixed, s);
}

template <typename T, int S, int MODE>
cudaError_t batch_stage_t(const BatchCase *cases, const int2 *items, int n_items,
                          double *item_max, double dt_fixed, int n_sm, cudaStream_t s) {
    using B = typename Shape2<T, S>::type;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = func_smem_attr((const void *)batch_stage_kernel<T, S, MODE>, B::SMEM);
    if (e != cudaSuccess) return e;
    // resident blocks per SM, per device ordinal (0: not yet asked)
    static std::atomic<int> per_sm_of[64];
    int per_sm = dev < 64 ? per_sm_of[dev].load() : 0;
    if (per_sm == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_stage_kernel<T, S, MODE>,
                                                          NT, B::SMEM);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        if (dev < 64) per_sm_of[dev].store(per_sm);
    }
    long long ctas = (long long)per_sm * (n_sm > 0 ? n_sm : 1);
    if (ctas > n_items) ctas = n_items;
    if (ctas < 1) return cudaSuccess;
    batch_stage_kernel<T, S, MODE><<<(unsigned)ctas, NT, B::SMEM, s>>>(cases, items, n_items,
                                                                        item_max, dt_fixed);
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t batch_stage_shape(int shape, const BatchCase *cases, const int2 *items, int n_items,
                              double *item_max, double dt_fixed, int n_sm, cudaStream_t s) {
    switch (shape) {
    case 0: return batch_stage_t<T, 0, MODE>(cases, items, n_items, item_max, dt_fixed, n_sm, s);
    case 1: return batch_stage_t<T, 1, MODE>(cases, items, n_items, item_max, dt_fixed, n_sm, s);
    case 2: return batch_stage_t<T, 2, MODE>(cases, items, n_items, item_max, dt_fixed, n_sm, s);
    case 3: return batch_stage_t<T, 3, MODE>(cases, items, n_items, item_max, dt_fixed, n_sm, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

void batch_tile_shape(int shape, int *bx, int *by) {
    static const int X[kBatchShapes] = {16, 32, 64, 8}, Y[kBatchShapes] = {16, 8, 4, 32};
    *bx = X[shape];
    *by = Y[shape];
}

cudaError_t launch_batch_stage(int mode, int shape, int fp_bytes, const BatchCase *cases,
                               const int2 *items, int n_items, double *item_max, double dt_fixed,
                               int n_sm, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (mode == 1)
        return fp_bytes == 4
                   ? batch_stage_shape<float, 1>(shape, cases, items, n_items, item_max, dt_fixed, n_sm, s)
                   : batch_stage_shape<double, 1>(shape, cases, items, n_items, item_max, dt_fixed, n_sm, s);
    if (mode == 2)
        return fp_bytes == 4
                   ? batch_stage_shape<float, 2>(shape, cases, items, n_items, item_max, dt_fixed, n_sm, s)
                   : batch_stage_shape<double, 2>(shape, cases, items, n_items, item_max, dt_fixed, n_sm, s);
    return cudaErrorInvalidValue;
}

size_t fluid_stage_blocks(const GridParams &g, int fp_bytes) {
    dim3 d;
    if (g.dim == 3 && fp_bytes == 4) return zmarch_blocks(g);
    if (g.dim == 3) d = stage_grid<3, double>(g);
    else if (fp_bytes == 4) d = stage_grid<2, float>(g);
    else d = small_2d_fp64(g) ? stage_grid<2, double, true>(g) : stage_grid<2, double>(g);
    return (size_t)d.x * d.y * d.z;
}

size_t dt_init_blocks(const GridParams &g) {
    return (size_t)((g.N + DT_CELLS_PER_CTA - 1) / DT_CELLS_PER_CTA);
}

size_t fluid_blockmax_count(const GridParams &g, int fp_bytes) {
    const size_t a = fluid_stage_blocks(g, fp_bytes), b = dt_init_blocks(g);
    return a > b ? a : b;
}

cudaError_t launch_stage1(const GridParams &g, int fp_bytes, const void *U, void *U1,
                          const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    return dispatch<1>(g, fp_bytes, U, U, U1, fb, dt_fixed, s);
}

cudaError_t launch_stage2(const GridParams &g, int fp_bytes, const void *Un, const void *U1,
                          void *out, const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    return dispatch<2>(g, fp_bytes, U1, Un, out, fb, dt_fixed, s);
}

cudaError_t launch_rhs(const GridParams &g, int fp_bytes, const void *U, void *L,
                       const FluidBuffers &fb, cudaStream_t s) {
    return dispatch<0>(g, fp_bytes, U, U, L, fb, 0.0, s);
}

cudaError_t launch_dt_init(const GridParams &g, int fp_bytes, const void *U,
                           const FluidBuffers &fb, cudaStream_t s) {
    const unsigned nb = (unsigned)dt_init_blocks(g);
    if (g.dim == 3) {
        if (fp_bytes == 4) dt_init_kernel<3, float><<<nb, NT, 0, s>>>(g, (const float *)U, fb.blockmax, fb.counter, fb.dt, fb.err);
        else dt_init_kernel<3, double><<<nb, NT, 0, s>>>(g, (const double *)U, fb.blockmax, fb.counter, fb.dt, fb.err);
    } else {
        if (fp_bytes == 4) dt_init_kernel<2, float><<<nb, NT, 0, s>>>(g, (const float *)U, fb.blockmax, fb.counter, fb.dt, fb.err);
        else dt_init_kernel<2, double><<<nb, NT, 0, s>>>(g, (const double *)U, fb.blockmax, fb.counter, fb.dt, fb.err);
    }
    return cudaGetLastError();
}

}  // namespace ibmk
