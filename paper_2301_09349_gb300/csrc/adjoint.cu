// Discrete adjoint of the IBM step: gradients of J = a C_d + b Nu (the last
// recorded step's drag coefficient and Nusselt number, Eq. Bulk) with respect
// to the marker positions X and the wall temperatures T_w, by reverse
// accumulation through every recorded step.
//
// Conventions (the derivative of the discrete map actually computed):
//   - the step sizes are those of the forward run (held fixed);
//   - bins, the kept marker set and the band mask do not move;
//   - the van Leer limiter, the Rusanov max and |u| take the branch of the
//     forward evaluation;
//   - eps~ = A~^{-1} 1 is differentiated exactly: one extra solve A~ z =
//     dJ/deps~ with the forward solver and dA~/dX from the kernel derivative.
//
// One forward step (App. B) is U1 = U + dt L(U), U* = U/2 + (U1 + dt L(U1))/2,
// G = rho_L U_b - I[rho u], H = rho_L c_v T_w - I[rho e] (Eqs. interp,
// forceMomentum, corr3.8), f = S[eps~ G], q = S[eps~ H] (Eq. force2) and the
// forced update of the band cells (Eqs. u_centralF2, e_centralF2).  Its
// reverse, with lam the adjoint of U^{n+1}:
//   1. forced update   -> lam* (adjoint of U*), lam_f, lam_q at band cells;
//   2. spreading       -> adjoints of G, H, eps~ and X (through Phi);
//   3. forcing         -> adjoints of rho_L, I[rho u], I[rho e] and T_w;
//   4. interpolation   -> lam* += S-type gather, X (through Phi);
//   5. predictor       -> mu = lam*/2 + dt/2 J_L(U1)^T lam*,
//                         lam^n = lam*/2 + mu + dt J_L(U)^T mu.
// J_L^T v is evaluated face by face: the reverse of the face flux (MUSCL /
// van Leer states, Rusanov flux, central viscous stress and heat flux with
// Sutherland's law) is scattered into accumulators of the primitive
// adjoints of its stencil cells (ghost cells mapped to their sources, with
// the slip flips; free-stream ghosts are constants), then chained to the
// conserved variables cell by cell (the sums in the grid's type: FP32 grids
// run the reverse sweep in FP32, with the per-marker gradient accumulators
// in FP64).  The forward states of each segment are replayed from
// checkpoints taken every `every` steps.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "handle.h"
#include "internal.h"
#include "marker_ops.cuh"

namespace ibmk {
namespace {

constexpr int AT = 256;

// constants of the flux in the compute type R (the forward's own values)
template <typename R> struct AdjK;
template <> struct AdjK<double> {
    double gam, inv_gm1, gm1, invR, mu_inf, S, lam_fac, inv_h, E_inf;
    bool viscous;
    __device__ __forceinline__ explicit AdjK(const GridParams &g)
        : gam(g.gamma), inv_gm1(1.0 / (g.gamma - 1.0)), gm1(g.gamma - 1.0), invR(1.0 / g.R),
          mu_inf(g.mu_inf), S(g.S), lam_fac(g.cp / g.Pr), inv_h(g.inv_h),
          E_inf(g.p_inf / (g.gamma - 1.0) + 0.5), viscous(g.mu_inf > 0.0) {}
};
template <> struct AdjK<float> {
    float gam, inv_gm1, gm1, invR, mu_inf, S, lam_fac, inv_h, E_inf;
    bool viscous;
    __device__ __forceinline__ explicit AdjK(const GridParams &g)
        : gam(g.f.gamma), inv_gm1(g.f.inv_gm1), gm1(g.f.gm1), invR(g.f.invR), mu_inf(g.f.mu_inf),
          S(g.f.S), lam_fac(g.f.lam_fac), inv_h(g.f.inv_h), E_inf(g.f.E_inf),
          viscous(g.f.viscous != 0) {}
};

template <typename R> __device__ __forceinline__ R sgn(R x) {
    return x > R(0) ? R(1) : (x < R(0) ? R(-1) : R(0));
}

// primitives (rho, u.., p) of the (ghost-mapped) cell (x, y, z); its source
// cell, slip flips and free-stream flag are returned for the scatter
template <int DIM, typename T, typename R>
__device__ __forceinline__ void load_prim(const GridParams &g, const AdjK<R> &k,
                                          const T *__restrict__ U, int x, int y, int z,
                                          R (&w)[DIM + 2], long long &src, int &flip, int &fs) {
    constexpr int NC = DIM + 2;
    flip = 0;
    fs = 0;
    const int sx = map_axis(x, g.n[0], g.bc[0], g.bc[1], 0, flip, fs);
    const int sy = map_axis(y, g.n[1], g.bc[2], g.bc[3], 1, flip, fs);
    const int sz = DIM == 3 ? map_axis(z, g.n[2], g.bc[4], g.bc[5], 2, flip, fs) : 0;
    src = sx + (long long)g.n[0] * (sy + (long long)g.n[1] * sz);
    R u[NC];
    if (fs) {
        u[0] = R(1);
        u[1] = R(1);
#pragma unroll
        for (int d = 1; d < DIM; ++d) u[1 + d] = R(0);
        u[NC - 1] = k.E_inf;
    } else {
#pragma unroll
        for (int c = 0; c < NC; ++c) u[c] = (R)U[c * g.N + src];
#pragma unroll
        for (int d = 0; d < DIM; ++d)
            if ((flip >> d) & 1) u[1 + d] = -u[1 + d];
    }
    const R rho = u[0];
    R ke = R(0);
    w[0] = rho;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        w[1 + d] = u[1 + d] / rho;
        ke += w[1 + d] * w[1 + d];
    }
    w[NC - 1] = k.gm1 * (u[NC - 1] - R(0.5) * rho * ke);
}

template <typename R>
__device__ __forceinline__ R vl(R a, R b) {
    const R ab = a * b;
    return ab > R(0) ? R(2) * ab / (a + b) : R(0);
}
// partial derivatives of vl(a, b) (zero off the branch taken)
template <typename R>
__device__ __forceinline__ void vl_grad(R a, R b, R &da, R &db) {
    if (a * b > R(0)) {
        const R s = a + b, s2 = s * s;
        da = R(2) * b * b / s2;
        db = R(2) * a * a / s2;
    } else {
        da = db = R(0);
    }
}

// Reverse of one side's Euler flux and conserved vector: Fx = dJ/dF_side,
// Ux = dJ/dU_side; adds to wxb (rho, u.., p) and returns the adjoint of u_n
// separately (the caller adds the wave-speed part first).
template <int DIM, int D, typename R>
__device__ __forceinline__ void side_vjp(const AdjK<R> &k, const R (&wx)[DIM + 2],
                                         const R (&Fx)[DIM + 2], const R (&Ux)[DIM + 2],
                                         R (&wxb)[DIM + 2], R &unb) {
    constexpr int NC = DIM + 2;
    const R rho = wx[0], p = wx[NC - 1], un = wx[1 + D];
    R ke = R(0);
#pragma unroll
    for (int m = 0; m < DIM; ++m) ke += wx[1 + m] * wx[1 + m];
    const R E = p * k.inv_gm1 + R(0.5) * rho * ke;
    R rhob = Fx[0] * un + Ux[0], pb = R(0), Eb = R(0);
    unb += Fx[0] * rho;
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        const R um = wx[1 + m];
        rhob += Fx[1 + m] * um * un + Ux[1 + m] * um;
        wxb[1 + m] += Fx[1 + m] * rho * un + Ux[1 + m] * rho;
        unb += Fx[1 + m] * rho * um;
        if (m == D) pb += Fx[1 + m];
    }
    Eb += Fx[NC - 1] * un + Ux[NC - 1];
    pb += Fx[NC - 1] * un;
    unb += Fx[NC - 1] * (E + p);
    pb += Eb * k.inv_gm1;
    rhob += Eb * R(0.5) * ke;
#pragma unroll
    for (int m = 0; m < DIM; ++m) wxb[1 + m] += Eb * rho * wx[1 + m];
    wxb[0] += rhob;
    wxb[NC - 1] += pb;
}

__host__ __device__ constexpr int ntan(int dim) { return dim > 1 ? dim - 1 : 1; }

// Reverse of the face flux between stencil cells a = w[1] and b = w[2]
// along axis D.  w[0..3]: primitives of a - s, a, b, b + s; ut[ti][0..3]:
// velocities of a - t, a + t, b - t, b + t for the ti-th tangential axis.
template <int DIM, int D, typename R>
__device__ __forceinline__ void face_vjp(const AdjK<R> &k, const R (&w)[4][DIM + 2],
                                         const R (&ut)[ntan(DIM)][4][DIM],
                                         const R (&Fb)[DIM + 2], R (&wb)[4][DIM + 2],
                                         R (&utb)[ntan(DIM)][4][DIM]) {
    constexpr int NC = DIM + 2;
    // ---- forward: MUSCL states
    R wl[NC], wr[NC], d0[NC], d1[NC], d2[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        d0[m] = w[1][m] - w[0][m];
        d1[m] = w[2][m] - w[1][m];
        d2[m] = w[3][m] - w[2][m];
        wl[m] = w[1][m] + R(0.5) * vl(d0[m], d1[m]);
        wr[m] = w[2][m] - R(0.5) * vl(d1[m], d2[m]);
    }
    // ---- forward: Rusanov
    R UL[NC], UR[NC];
    R keL = R(0), keR = R(0);
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        keL += wl[1 + m] * wl[1 + m];
        keR += wr[1 + m] * wr[1 + m];
    }
    UL[0] = wl[0];
    UR[0] = wr[0];
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
        UL[1 + m] = wl[0] * wl[1 + m];
        UR[1 + m] = wr[0] * wr[1 + m];
    }
    UL[NC - 1] = wl[NC - 1] * k.inv_gm1 + R(0.5) * wl[0] * keL;
    UR[NC - 1] = wr[NC - 1] * k.inv_gm1 + R(0.5) * wr[0] * keR;
    const R cL = sqrt(k.gam * wl[NC - 1] / wl[0]), cR = sqrt(k.gam * wr[NC - 1] / wr[0]);
    const R unL = wl[1 + D], unR = wr[1 + D];
    const R sL = fabs(unL) + cL, sR = fabs(unR) + cR;
    const bool left = sL > sR;
    const R smax = left ? sL : sR;

    R wlb[NC], wrb[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) wlb[m] = wrb[m] = R(0);

    // ---- reverse: viscous stress and heat flux
    if (k.viscous) {
        const R Ta = w[1][NC - 1] * k.invR / w[1][0], Tb = w[2][NC - 1] * k.invR / w[2][0];
        const R Tf = R(0.5) * (Ta + Tb);
        const R mu = k.mu_inf * Tf * sqrt(Tf) * (R(1) + k.S) / (Tf + k.S);
        const R lam = mu * k.lam_fac;
        const R q = R(0.25) * k.inv_h;
        R grad[DIM][DIM];
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
            int ti = 0;
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
                if (e == D) {
                    grad[m][e] = (w[2][1 + m] - w[1][1 + m]) * k.inv_h;
                } else {
                    grad[m][e] = (ut[ti][1][m] - ut[ti][0][m] + ut[ti][3][m] - ut[ti][2][m]) * q;
                    ++ti;
                }
            }
        }
        R div = R(0);
#pragma unroll
        for (int m = 0; m < DIM; ++m) div += grad[m][m];
        R tau[DIM], uf[DIM];
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
            tau[m] = mu * (grad[D][m] + grad[m][D]) - (m == D ? R(2.0 / 3.0) * mu * div : R(0));
            uf[m] = R(0.5) * (w[1][1 + m] + w[2][1 + m]);
        }
        const R workb = -Fb[NC - 1];
        const R lamb = -Fb[NC - 1] * (Tb - Ta) * k.inv_h;
        R Tbb = -Fb[NC - 1] * lam * k.inv_h, Tab = Fb[NC - 1] * lam * k.inv_h;
        R mub = lamb * k.lam_fac, divb = R(0);
        R gb[DIM][DIM];
#pragma unroll
        for (int m = 0; m < DIM; ++m)
#pragma unroll
            for (int e = 0; e < DIM; ++e) gb[m][e] = R(0);
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
            const R taub = -Fb[1 + m] + workb * uf[m];
            const R ufb = workb * tau[m];
            wb[1][1 + m] += R(0.5) * ufb;
            wb[2][1 + m] += R(0.5) * ufb;
            mub += taub * (grad[D][m] + grad[m][D]);
            gb[D][m] += mu * taub;
            gb[m][D] += mu * taub;
            if (m == D) {
                mub -= R(2.0 / 3.0) * div * taub;
                divb -= R(2.0 / 3.0) * mu * taub;
            }
        }
#pragma unroll
        for (int m = 0; m < DIM; ++m) gb[m][m] += divb;
        const R Tfb = mub * mu * (R(1.5) / Tf - R(1) / (Tf + k.S));
        Tab += R(0.5) * Tfb;
        Tbb += R(0.5) * Tfb;
#pragma unroll
        for (int m = 0; m < DIM; ++m) {
            int ti = 0;
#pragma unroll
            for (int e = 0; e < DIM; ++e) {
                if (e == D) {
                    wb[2][1 + m] += gb[m][e] * k.inv_h;
                    wb[1][1 + m] -= gb[m][e] * k.inv_h;
                } else {
                    utb[ti][1][m] += gb[m][e] * q;
                    utb[ti][0][m] -= gb[m][e] * q;
                    utb[ti][3][m] += gb[m][e] * q;
                    utb[ti][2][m] -= gb[m][e] * q;
                    ++ti;
                }
            }
        }
        // T = p r^-1 / rho at a and b
        wb[1][NC - 1] += Tab * k.invR / w[1][0];
        wb[1][0] -= Tab * Ta / w[1][0];
        wb[2][NC - 1] += Tbb * k.invR / w[2][0];
        wb[2][0] -= Tbb * Tb / w[2][0];
    }

    // ---- reverse: Rusanov, F = (F_L + F_R)/2 - smax (U_R - U_L)/2
    R FxL[NC], FxR[NC], UxL[NC], UxR[NC];
    R sb = R(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        FxL[c] = FxR[c] = R(0.5) * Fb[c];
        UxL[c] = R(0.5) * smax * Fb[c];
        UxR[c] = -R(0.5) * smax * Fb[c];
        sb -= R(0.5) * Fb[c] * (UR[c] - UL[c]);
    }
    R unLb = R(0), unRb = R(0);
    side_vjp<DIM, D, R>(k, wl, FxL, UxL, wlb, unLb);
    side_vjp<DIM, D, R>(k, wr, FxR, UxR, wrb, unRb);
    // smax = max(sL, sR), s = |u_n| + c, c = sqrt(gamma p / rho)
    const R sLb = left ? sb : R(0), sRb = left ? R(0) : sb;
    unLb += sgn(unL) * sLb;
    unRb += sgn(unR) * sRb;
    wlb[NC - 1] += sLb * k.gam / (R(2) * wl[0] * cL);
    wlb[0] -= sLb * cL / (R(2) * wl[0]);
    wrb[NC - 1] += sRb * k.gam / (R(2) * wr[0] * cR);
    wrb[0] -= sRb * cR / (R(2) * wr[0]);
    wlb[1 + D] += unLb;
    wrb[1 + D] += unRb;

    // ---- reverse: MUSCL
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        wb[1][m] += wlb[m];
        wb[2][m] += wrb[m];
        R a01, b01, a12, b12;
        vl_grad(d0[m], d1[m], a01, b01);
        vl_grad(d1[m], d2[m], a12, b12);
        const R g01 = R(0.5) * wlb[m], g12 = -R(0.5) * wrb[m];
        const R d0b = g01 * a01, d1b = g01 * b01 + g12 * a12, d2b = g12 * b12;
        wb[1][m] += d0b - d1b;
        wb[0][m] -= d0b;
        wb[2][m] += d1b - d2b;
        wb[3][m] += d2b;
    }
}

// flux-reverse CTA: 256 threads, three per SM (80 registers, a few bytes of
// spill; 69 KB of shared memory each); measured faster than 128 x 3 (115
// registers) and 256 x 2 on the 128^3 adjoint
#ifndef IBM_ADJ_FT
#define IBM_ADJ_FT 256
#endif
#ifndef IBM_ADJ_FT_MIN
#define IBM_ADJ_FT_MIN 3
#endif
constexpr int FT = IBM_ADJ_FT;

// ---- tiled form: one CTA per tile of cells -------------------------------
// The CTA stages the primitives of its tile plus a two-cell halo (ghosts
// through the boundary maps) in shared memory, reverses every face it owns
// - the faces whose upper cell b lies in the tile, and on the last tile of an
// axis also the domain face b = n - accumulating the stencil adjoints in
// shared memory, then adds the tile-plus-halo accumulators to the source
// cells in global memory (slip flips applied, free-stream ghosts dropped).
template <int DIM, typename T> struct AdjTile;
template <> struct AdjTile<3, float> { static constexpr int BX = 8, BY = 8, BZ = 8; };
template <> struct AdjTile<3, double> { static constexpr int BX = 8, BY = 8, BZ = 4; };
template <> struct AdjTile<2, float> { static constexpr int BX = 16, BY = 16, BZ = 1; };
template <> struct AdjTile<2, double> { static constexpr int BX = 16, BY = 16, BZ = 1; };

template <int DIM, typename T>
struct AdjBox {
    static constexpr int BX = AdjTile<DIM, T>::BX, BY = AdjTile<DIM, T>::BY,
                         BZ = AdjTile<DIM, T>::BZ;
    static constexpr int PX = BX + 4, PY = BY + 4, PZ = DIM == 3 ? BZ + 4 : 1;
    static constexpr int PN = PX * PY * PZ;
    static constexpr size_t SMEM = 2 * sizeof(T) * (size_t)(DIM + 2) * PN;
};

template <int DIM, int D, typename T>
__device__ __forceinline__ void tile_faces(const GridParams &g, const AdjK<T> &k,
                                           const T *__restrict__ V, const T *__restrict__ Wsm,
                                           T *__restrict__ Acc, int ox, int oy, int oz) {
    using B = AdjBox<DIM, T>;
    using R = T;
    constexpr int NC = DIM + 2;
    constexpr int NT2 = ntan(DIM);
    constexpr int PN = B::PN;
    const int o[3] = {ox, oy, oz};
    const int bsz[3] = {B::BX, B::BY, B::BZ};
    const int str[3] = {1, B::PX, B::PX * B::PY};
    int cnt[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int n = e < DIM ? g.n[e] : 1;
        const int b = e < DIM ? bsz[e] : 1;
        cnt[e] = min(b, n - o[e]);
    }
    if (o[D] + bsz[D] >= g.n[D]) cnt[D] += 1;   // the last tile owns the domain face b = n
    const int nf = cnt[0] * cnt[1] * cnt[2];
    const long long N = g.N;
    // Faces go in batches of one per thread.  Each face adds to 4 cells along
    // its normal and 4 cells per tangent; for one such stencil slot the map
    // face -> cell is one-to-one, so the slots are added in a fixed order
    // with a barrier between them and no two faces of a batch ever touch the
    // same accumulator at once: the sums are bitwise reproducible.
    for (int base = 0; base < nf; base += FT) {
        const int f = base + threadIdx.x;
        bool act = false;
        int qs[4];
        int qt[NT2][4];
        R wb[4][NC];
        R utb[NT2][4][DIM];
        if (f < nf) {
            int l[3];
            l[0] = f % cnt[0];
            l[1] = (f / cnt[0]) % cnt[1];
            l[2] = f / (cnt[0] * cnt[1]);
            const int gb = o[D] + l[D];
            const bool b_in = gb < g.n[D], a_in = gb >= 1;
            long long jb = 0, ja = 0;
            {
                int c[3] = {o[0] + l[0], o[1] + l[1], o[2] + l[2]};
                jb = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
                c[D] -= 1;
                ja = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
            }
            R Fb[NC];
            bool any = false;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                const R vb = b_in ? V[q * N + jb] : R(0);
                const R va = a_in ? V[q * N + ja] : R(0);
                Fb[q] = (vb - va) * k.inv_h;
                any |= Fb[q] != R(0);
            }
            if (any) {
                act = true;
                const int qb =
                    (l[0] + 2) + B::PX * ((l[1] + 2) + B::PY * (DIM == 3 ? l[2] + 2 : 0));
                const int sD = str[D];
                R w[4][NC];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    qs[i] = qb + (i - 2) * sD;
#pragma unroll
                    for (int c = 0; c < NC; ++c) {
                        w[i][c] = Wsm[c * PN + qs[i]];
                        wb[i][c] = R(0);
                    }
                }
                R ut[NT2][4][DIM];
                {
                    int ti = 0;
#pragma unroll
                    for (int e = 0; e < DIM; ++e) {
                        if (e == D) continue;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            qt[ti][i] = (i < 2 ? qb - sD : qb) + ((i & 1) ? str[e] : -str[e]);
#pragma unroll
                            for (int m = 0; m < DIM; ++m) {
                                ut[ti][i][m] = Wsm[(1 + m) * PN + qt[ti][i]];
                                utb[ti][i][m] = R(0);
                            }
                        }
                        ++ti;
                    }
                }
                face_vjp<DIM, D, R>(k, w, ut, Fb, wb, utb);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (act) {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    if (wb[i][c] != R(0)) Acc[c * PN + qs[i]] += wb[i][c];
            }
            __syncthreads();
        }
#pragma unroll
        for (int ti = 0; ti < (DIM > 1 ? DIM - 1 : 0); ++ti)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (act) {
#pragma unroll
                    for (int m = 0; m < DIM; ++m)
                        if (utb[ti][i][m] != R(0)) Acc[(1 + m) * PN + qt[ti][i]] += utb[ti][i][m];
                }
                __syncthreads();
            }
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(FT, IBM_ADJ_FT_MIN)
adj_flux_tile_kernel(const GridParams g, const T *__restrict__ U, const T *__restrict__ V,
                     T *__restrict__ tbuf) {
    using B = AdjBox<DIM, T>;
    using R = T;
    constexpr int NC = DIM + 2;
    constexpr int PN = B::PN;
    extern __shared__ __align__(16) unsigned char smem_adj[];
    R *Wsm = reinterpret_cast<R *>(smem_adj);   // [NC][PN] primitives
    R *Acc = Wsm + NC * PN;                      // [NC][PN] adjoint sums
    const AdjK<R> k(g);
    const int ox = blockIdx.x * B::BX, oy = blockIdx.y * B::BY;
    const int oz = DIM == 3 ? blockIdx.z * B::BZ : 0;
    for (int q = threadIdx.x; q < PN; q += FT) {
        const int lx = q % B::PX, ly = (q / B::PX) % B::PY, lz = q / (B::PX * B::PY);
        R w[NC];
        long long src;
        int flip, fs;
        load_prim<DIM, T, R>(g, k, U, ox + lx - 2, oy + ly - 2, DIM == 3 ? oz + lz - 2 : 0, w, src,
                             flip, fs);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            Wsm[c * PN + q] = w[c];
            Acc[c * PN + q] = R(0);
        }
    }
    __syncthreads();
    tile_faces<DIM, 0, T>(g, k, V, Wsm, Acc, ox, oy, oz);
    tile_faces<DIM, 1, T>(g, k, V, Wsm, Acc, ox, oy, oz);
    if constexpr (DIM == 3) tile_faces<DIM, (DIM == 3 ? 2 : 0), T>(g, k, V, Wsm, Acc, ox, oy, oz);
    __syncthreads();
    // the tile-plus-halo sums go to this tile's own slice of the buffer; the
    // chain kernel gathers them per cell in a fixed order
    const size_t tile = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
    T *dst = tbuf + tile * NC * PN;
    for (int q = threadIdx.x; q < NC * PN; q += FT) dst[q] = Acc[q];
}

// The primitive adjoints of cell c from the tile buffers: every tile whose
// halo-extended box holds the cell, or a ghost image of it (slip mirror,
// zero gradient or periodic image; free-stream ghosts are constants and drop
// out), summed in a fixed order - per axis the boxes holding the cell itself
// by ascending tile, then those holding its ghost images - with the slip
// flips of the momentum components applied.  Up to six candidates per axis
// (a ragged last tile of one cell adds a box), kept in registers as packed
// (tile << 8 | position << 1 | flip) words and picked by selects.
struct AxisCands {
    unsigned v0 = 0, v1 = 0, v2 = 0, v3 = 0, v4 = 0, v5 = 0;
    int n = 0;
    __device__ __forceinline__ void add(unsigned w) {
        v5 = n == 5 ? w : v5;
        v4 = n == 4 ? w : v4;
        v3 = n == 3 ? w : v3;
        v2 = n == 2 ? w : v2;
        v1 = n == 1 ? w : v1;
        v0 = n == 0 ? w : v0;
        n = n < 6 ? n + 1 : 6;
    }
    __device__ __forceinline__ unsigned get(int k) const {
        unsigned r = v0;
        r = k == 1 ? v1 : r;
        r = k == 2 ? v2 : r;
        r = k == 3 ? v3 : r;
        r = k == 4 ? v4 : r;
        r = k == 5 ? v5 : r;
        return r;
    }
};

template <int DIM, typename T>
__device__ __forceinline__ void gather_tiles(const GridParams &g, const T *__restrict__ tbuf,
                                             const int (&c)[3], T (&wv)[DIM + 2]) {
    using B = AdjBox<DIM, T>;
    constexpr int NC = DIM + 2;
    constexpr int PN = B::PN;
    const int bs[3] = {B::BX, B::BY, B::BZ};
    const int ps[3] = {B::PX, B::PY, B::PZ};
    int nt[3] = {1, 1, 1};
    AxisCands ax[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        if (e >= DIM) {
            ax[e].add(0u);
            continue;
        }
        const int n = g.n[e], be = bs[e];
        nt[e] = (n + be - 1) / be;
        // the cell itself, then the ghost positions whose image it is
        const int cand[5] = {c[e], -2, -1, n, n + 1};
#pragma unroll
        for (int pi = 0; pi < 5; ++pi) {
            const int p = cand[pi];
            int flip = 0;
            if (pi > 0) {
                int fs = 0;
                const int src = map_axis(p, n, g.bc[2 * e], g.bc[2 * e + 1], e, flip, fs);
                if (fs || src != c[e]) continue;
            }
            // tiles te whose box [te be - 2, te be + be + 1] holds p (p >= -2;
            // at most two, since be >= 4)
            const int thi = (p + 2) / be;
#pragma unroll
            for (int te = thi - 1; te <= thi; ++te) {
                const int l = p - te * be + 2;
                if (te < 0 || te >= nt[e] || l < 0 || l >= ps[e]) continue;
                ax[e].add(((unsigned)te << 8) | ((unsigned)l << 1) | (flip ? 1u : 0u));
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NC; ++q) wv[q] = T(0);
    for (int iz = 0; iz < ax[2].n; ++iz) {
        const unsigned wz = ax[2].get(iz);
        for (int iy = 0; iy < ax[1].n; ++iy) {
            const unsigned wy = ax[1].get(iy);
            for (int ix = 0; ix < ax[0].n; ++ix) {
                const unsigned wx = ax[0].get(ix);
                const size_t tile =
                    (wx >> 8) + (size_t)nt[0] * ((wy >> 8) + (size_t)nt[1] * (wz >> 8));
                const int q = (int)((wx >> 1) & 127u) +
                              B::PX * ((int)((wy >> 1) & 127u) + B::PY * (int)((wz >> 1) & 127u));
                const int flip = (int)(wx & 1u) | ((int)(wy & 1u) << 1) | ((int)(wz & 1u) << 2);
                const T *src = tbuf + tile * NC * PN + q;
#pragma unroll
                for (int cc = 0; cc < NC; ++cc) {
                    T v = src[(size_t)cc * PN];
                    if (cc >= 1 && cc <= DIM && ((flip >> (cc - 1)) & 1)) v = -v;
                    wv[cc] += v;
                }
            }
        }
    }
}

// w = (dW/dU)^T W-bar at every cell, W-bar gathered from the tile buffers:
// rho-bar = W_rho - sum_m W_um u_m / rho + W_p (gamma-1) |u|^2/2,
// m-bar = W_u / rho - W_p (gamma-1) u, E-bar = W_p (gamma-1).
// MODE -1 stores w in out; the reverse sweep's two SSP-RK2 updates take w
// directly: MODE 0 mu = lam/2 + (dt/2) w, MODE 1 lam = lam/2 + mu + dt w.
// In the grid's type throughout (double arithmetic is slow on this GPU).
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(AT)
adj_prim_kernel(const GridParams g, const T *__restrict__ U, const T *__restrict__ tbuf,
                T *__restrict__ out, T *__restrict__ lam, T *__restrict__ mu, double dt_d) {
    using R = T;
    constexpr int NC = DIM + 2;
    const long long N = g.N;
    const AdjK<R> k(g);
    const R dt = (R)dt_d, half = R(0.5);
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < N;
         j += (long long)gridDim.x * blockDim.x) {
        // all of a cell's loads are issued before its stores
        R uc[DIM + 1], wbv[NC], lv[NC], mv[NC];
#pragma unroll
        for (int q = 0; q <= DIM; ++q) uc[q] = __ldg(U + q * N + j);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            lv[q] = MODE >= 0 ? lam[q * N + j] : R(0);
            mv[q] = MODE == 1 ? mu[q * N + j] : R(0);
        }
        {
            const long long nxy = (long long)g.n[0] * g.n[1];
            const int c[3] = {(int)(j % g.n[0]), (int)((j / g.n[0]) % g.n[1]),
                              DIM == 3 ? (int)(j / nxy) : 0};
            gather_tiles<DIM, T>(g, tbuf, c, wbv);
        }
        const R rho = uc[0], inv = R(1) / rho;
        R v[DIM], ke = R(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            v[d] = uc[1 + d] * inv;
            ke += v[d] * v[d];
        }
        const R pb = wbv[NC - 1] * k.gm1;
        R w[NC];
        R rb = wbv[0] + pb * R(0.5) * ke;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            rb -= wbv[1 + d] * v[d] * inv;
            w[1 + d] = wbv[1 + d] * inv - pb * v[d];
        }
        w[0] = rb;
        w[NC - 1] = pb;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            if (MODE < 0) out[q * N + j] = w[q];
            else if (MODE == 0) mu[q * N + j] = half * lv[q] + half * dt * w[q];
            else lam[q * N + j] = half * lv[q] + mv[q] + dt * w[q];
        }
    }
}


// One warp per band cell (cells of the band tiles in order, warps strided
// over the grid); fn(c, j, lane) runs on every lane of the warp.
template <int DIM, typename F>
__device__ __forceinline__ void for_band_cells_warp(const GridParams &g, const MarkerBuffers &m,
                                                    F &&fn) {
    const int lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    const long long nw = (long long)gridDim.x * wpb;
    const long long total = (long long)m.counts[1] * g.cells_per_tile;
    for (long long it = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); it < total; it += nw) {
        const int t = m.band_list[it / g.cells_per_tile];
        const int q = (int)(it % g.cells_per_tile);
        const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
                  tz = t / (g.ntile[0] * g.ntile[1]);
        const int c[3] = {tx * g.tile[0] + q % g.tile[0],
                          ty * g.tile[1] + (q / g.tile[0]) % g.tile[1],
                          DIM == 3 ? tz * g.tile[2] + q / (g.tile[0] * g.tile[1]) : 0};
        if (c[0] >= g.n[0] || c[1] >= g.n[1] || (DIM == 3 && c[2] >= g.n[2])) continue;
        const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
        if (!((m.band_bits[j >> 5] >> (j & 31)) & 1u)) continue;
        fn(c, j, lane);
    }
}

// Lane n < 3^DIM visits the markers owned by neighbour n of c (the order of
// gather_markers: z, y, x offsets ascending); the warp then sums the lanes'
// partials with warp_sum_d, a fixed tree.  The weights Phi_k(j) are taken in
// precision R: the field precision where the pass reverses the forward
// interpolation or spreading (the forward evaluates them in that precision,
// and FP64 square roots run at a small fraction of the FP32 rate on this
// GPU), double for the quadrature's FP64 fields.
template <int DIM, typename R, typename F>
__device__ __forceinline__ void gather_markers_lane(const GridParams &g, const MarkerBuffers &m,
                                                    const unsigned *__restrict__ keys,
                                                    const int *__restrict__ perm, const int c[3],
                                                    int lane, F &&visit) {
    constexpr int NT3 = DIM == 3 ? 27 : 9;
    if (lane >= NT3) return;
    gather_cell<DIM, R>(g, m, keys, perm, c, lane % 3 - 1, (lane / 3) % 3 - 1,
                        DIM == 3 ? lane / 9 - 1 : 0, visit);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// 1. reverse of the forced update at the band cells: lam (adjoint of
//    U^{n+1}) -> lam* in place, and lam_f, lam_q into lfq.  Sums and
//    arithmetic in the field precision T, like the forward spreading (a
//    warp-wide FP64 instruction costs the FP64 pipe ~16 cycles on this GPU
//    whatever the active lanes); the change of |rho u|^2 is taken as
//    sum_d f_d (2 m_d + f_d), free of cancellation.
template <int DIM, typename T>
__global__ void __launch_bounds__(AT)
adj_apply_kernel(const GridParams g, const MarkerBuffers m, const unsigned *__restrict__ keys,
                 const int *__restrict__ perm, const T *__restrict__ Us, T *__restrict__ lam,
                 T *__restrict__ lfq) {
    const long long N = g.N;
    for_band_cells_warp<DIM>(g, m, [&](const int *c, long long j, int lane) {
        T f[DIM], q = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) f[d] = T(0);
        gather_markers_lane<DIM, T>(g, m, keys, perm, c, lane, [&](int kk, T w) {
            const T ew = (T)m.eps[kk] * w;
#pragma unroll
            for (int d = 0; d < DIM; ++d) f[d] += (T)m.G[(long long)kk * DIM + d] * ew;
            q += (T)m.H[kk] * ew;
        });
#pragma unroll
        for (int d = 0; d < DIM; ++d) f[d] = warp_sum_r<T>(f[d]);
        q = warp_sum_r<T>(q);
        if (lane != 0) return;
        const T irho = T(1) / Us[j];
        const T lE = lam[(DIM + 1) * N + j];
        const T lEr = lE * irho;
        // the heat-source cap of the forward update: where it binds, q is
        // replaced by -cap (rho e)* = -cap (E* - |m*|^2 / (2 rho)), so the
        // adjoint of q is 0 and E*, m* and rho receive the cap's terms
        T ke0 = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) ke0 += Us[(1 + d) * N + j] * Us[(1 + d) * N + j];
        const T cap = (T)kHeatSourceCap;
        const bool act = q < -cap * (Us[(DIM + 1) * N + j] - T(0.5) * ke0 * irho);
        const T a = act ? cap : T(0);
        T dk = T(0);   // |m1|^2 - |m0|^2
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T ms = Us[(1 + d) * N + j];
            const T m1 = ms + f[d];
            const T lm = lam[(1 + d) * N + j];
            dk += f[d] * (ms + m1);
            if (g.energy_reading == 1) {
                lfq[d * N + j] = lm;
                if (act) lam[(1 + d) * N + j] = lm + lEr * a * ms;
            } else {
                lfq[d * N + j] = lm + lEr * m1;
                lam[(1 + d) * N + j] = lm + lEr * (f[d] + a * ms);
            }
        }
        lfq[DIM * N + j] = act ? T(0) : lE;
        if (g.energy_reading != 1)
            lam[j] = lam[j] - T(0.5) * lEr * irho * (dk + a * ke0);
        else if (act)
            lam[j] = lam[j] - T(0.5) * lEr * irho * a * ke0;
        if (act) lam[(DIM + 1) * N + j] = lE * (T(1) - a);
    });
}

// derivative of the 1D kernel, in precision R
template <typename R> __device__ __forceinline__ R dphi_r(R r) {
    const R a = r < R(0) ? -r : r, s = r < R(0) ? R(-1) : R(1);
    if (a <= R(0.5)) return -r / sqrt(R(1) - R(3) * a * a);
    if (a <= R(1.5)) {
        const R b = R(1) - a;
        return s * (R(-3) - R(3) * b / sqrt(R(1) - R(3) * b * b)) / R(6);
    }
    return R(0);
}

// Phi_k and dPhi_k/dX_k at the support cell `lane` of marker k, in
// precision R (the field precision where the pass reverses the forward
// interpolation or spreading, double for the quadrature)
template <int DIM, typename R>
__device__ __forceinline__ R lane_weight_grad(const GridParams &g, const MarkerBuffers &m, int k,
                                              int lane, R (&gw)[DIM], long long &j) {
    const int o[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, DIM == 3 ? lane / 9 - 1 : 0};
    R ph[DIM], dp[DIM];
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        c[d] = m.cell[(long long)k * 3 + d] + o[d];
        const R r = cell_offset<R>(o[d], marker_frac<R>(m, k, d));
        ph[d] = phi_r<R>(r);
        dp[d] = dphi_r<R>(r);
    }
    R w = R(1);
#pragma unroll
    for (int d = 0; d < DIM; ++d) w *= ph[d];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        R pr = -dp[d] * (R)g.inv_h;   // dr/dX = -1/h
#pragma unroll
        for (int e = 0; e < DIM; ++e)
            if (e != d) pr *= ph[e];
        gw[d] = pr;
    }
    j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    return w;
}

// 2.-3. one warp per marker: spreading and forcing reversed, the X parts of
// spreading and interpolation, and the per-marker adjoints mr for step 4.
// cd, nu: the direct terms of J at the last step (zero before it).
template <int DIM, typename T>
__global__ void __launch_bounds__(AT)
adj_marker_kernel(const GridParams g, const MarkerBuffers m, const AdjBuffers a,
                  const T *__restrict__ Us, double cd, double nu) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    const long long N = g.N;
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= m.ns) return;
    const double e = m.eps[k];
    double G[DIM], H = m.H[k];
#pragma unroll
    for (int d = 0; d < DIM; ++d) G[d] = m.G[(long long)k * DIM + d];
    // the weights, their X derivatives and the lane sums in the field
    // precision T (the forward spreading and interpolation use the same
    // weights); the per-marker terms and the interpolation part, which
    // cancels where the wall and fluid temperatures are close, in double
    T gw[DIM], w = T(0), sfT[DIM], sqT = T(0), gxT[DIM];
    long long j = 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) sfT[d] = gxT[d] = gw[d] = T(0);
    if (lane < NS) {
        w = lane_weight_grad<DIM, T>(g, m, k, lane, gw, j);
        T dot = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T lf = ((const T *)a.lfq)[d * N + j];
            sfT[d] = w * lf;
            dot += (T)G[d] * lf;
        }
        const T lq = ((const T *)a.lfq)[DIM * N + j];
        sqT = w * lq;
        dot += (T)H * lq;
#pragma unroll
        for (int d = 0; d < DIM; ++d) gxT[d] = gw[d] * dot;
    }
    double sf[DIM], gxs[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        sf[d] = (double)warp_sum_r<T>(sfT[d]);
        gxs[d] = (double)warp_sum_r<T>(gxT[d]);
    }
    const double sq = (double)warp_sum_r<T>(sqT);
    double lG[DIM], lH = e * sq + nu * e;
#pragma unroll
    for (int d = 0; d < DIM; ++d) lG[d] = e * sf[d] + (d == 0 ? cd * e : 0.0);
    const double rk = m.rhoL[k];
    double lrho = lH * g.cv * m.Tw[k];
#pragma unroll
    for (int d = 0; d < DIM; ++d) lrho += lG[d] * m.Ub[(long long)k * DIM + d];
    // interpolation part of dJ/dX: sum_j dPhi (l_rhoL rho + l_m . m + l_e rho e)
    double gxi[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) gxi[d] = 0.0;
    if (lane < NS) {
        const double rho = (double)Us[j];
        double msq = 0.0, dotm = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double md = (double)Us[(1 + d) * N + j];
            msq += md * md;
            dotm += -lG[d] * md;
        }
        const double rhoe = (double)Us[(DIM + 1) * N + j] - 0.5 * msq / rho;
        const double s = lrho * rho + dotm - lH * rhoe;
#pragma unroll
        for (int d = 0; d < DIM; ++d) gxi[d] = (double)gw[d] * s;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) gxi[d] = warp_sum_d(gxi[d]);
    if (lane == 0) {
        double le = cd * G[0] + nu * H + H * sq;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            le += G[d] * sf[d];
            a.lamX[(long long)k * 3 + d] += e * gxs[d] + gxi[d];
        }
        a.lamEps[k] += le;
        a.lamTw[k] += lH * rk * g.cv;
        double *mr = a.mr + (long long)k * 5;
        mr[0] = lrho;
#pragma unroll
        for (int d = 0; d < 3; ++d) mr[1 + d] = d < DIM ? -lG[d] : 0.0;
        mr[4] = -lH;
    }
}

// 4. interpolation reversed: lam* += sum_k Phi_k(j) d(rho, rho u, rho e)/dU^T mr_k
//    (sums and arithmetic in the field precision T, as in step 1)
template <int DIM, typename T>
__global__ void __launch_bounds__(AT)
adj_interp_kernel(const GridParams g, const MarkerBuffers m, const unsigned *__restrict__ keys,
                  const int *__restrict__ perm, const AdjBuffers a, const T *__restrict__ Us,
                  T *__restrict__ lam) {
    const long long N = g.N;
    for_band_cells_warp<DIM>(g, m, [&](const int *c, long long j, int lane) {
        T sr = T(0), sm[DIM], se = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) sm[d] = T(0);
        gather_markers_lane<DIM, T>(g, m, keys, perm, c, lane, [&](int kk, T w) {
            const double *mr = a.mr + (long long)kk * 5;
            sr += w * (T)mr[0];
#pragma unroll
            for (int d = 0; d < DIM; ++d) sm[d] += w * (T)mr[1 + d];
            se += w * (T)mr[4];
        });
        sr = warp_sum_r<T>(sr);
#pragma unroll
        for (int d = 0; d < DIM; ++d) sm[d] = warp_sum_r<T>(sm[d]);
        se = warp_sum_r<T>(se);
        if (lane != 0) return;
        const T irho = T(1) / Us[j];
        const T ser = se * irho;
        T msq = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T md = Us[(1 + d) * N + j];
            msq += md * md;
            lam[(1 + d) * N + j] = lam[(1 + d) * N + j] + sm[d] - ser * md;
        }
        lam[j] = lam[j] + sr + T(0.5) * ser * irho * msq;
        lam[(DIM + 1) * N + j] = lam[(DIM + 1) * N + j] + se;
    });
}

// S(eps~)_j and S(z)_j = sum_l v_l Phi_l(j) at the band cells into lamW[0], lamW[1]
template <int DIM>
__global__ void __launch_bounds__(AT)
adj_eps_fields_kernel(const GridParams g, const MarkerBuffers m, const unsigned *__restrict__ keys,
                      const int *__restrict__ perm, const AdjBuffers a) {
    const long long N = g.N;
    for_band_cells_warp<DIM>(g, m, [&](const int *c, long long j, int lane) {
        double se = 0.0, sz = 0.0;
        gather_markers_lane<DIM, double>(g, m, keys, perm, c, lane, [&](int kk, double w) {
            se += w * m.eps[kk];
            sz += w * a.z[kk];
        });
        se = warp_sum_d(se);
        sz = warp_sum_d(sz);
        if (lane != 0) return;
        double *w = (double *)a.lamW;   // FP64 scratch here
        w[j] = se;
        w[N + j] = sz;
    });
}

// dJ/dX_k -= sum_j dPhi_k(j)/dX_k (z_k S(eps~)_j + eps~_k S(z)_j)
template <int DIM>
__global__ void __launch_bounds__(AT)
adj_eps_x_kernel(const GridParams g, const MarkerBuffers m, const AdjBuffers a) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    const long long N = g.N;
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= m.ns) return;
    double gx[DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) gx[d] = 0.0;
    if (lane < NS) {
        double gw[DIM];
        long long j;
        lane_weight_grad<DIM, double>(g, m, k, lane, gw, j);
        const double *w = (const double *)a.lamW;
        const double s = a.z[k] * w[j] + m.eps[k] * w[N + j];
#pragma unroll
        for (int d = 0; d < DIM; ++d) gx[d] = gw[d] * s;
    }
#pragma unroll
    for (int d = 0; d < DIM; ++d) gx[d] = warp_sum_d(gx[d]);
    if (lane == 0)
#pragma unroll
        for (int d = 0; d < DIM; ++d) a.lamX[(long long)k * 3 + d] -= gx[d];
}

int grid_for(long long work, int per_block = AT) {
    long long b = (work + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > 16384) b = 16384;
    return (int)b;
}

// out = J_L(U)^T V (tbuf: the per-tile accumulators, adj_tile_buf_bytes)
template <int DIM, typename T>
cudaError_t rhs_vjp_t(const GridParams &g, const void *U, const void *V, void *tbuf_, void *out,
                      cudaStream_t s, int mode = -1, void *lam = nullptr, void *mu = nullptr,
                      double dt = 0.0) {
    const T *u = (const T *)U, *v = (const T *)V;
    T *tbuf = (T *)tbuf_;
    using B = AdjBox<DIM, T>;
    {
        cudaError_t e = func_smem_attr((const void *)adj_flux_tile_kernel<DIM, T>, B::SMEM);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid((g.n[0] + B::BX - 1) / B::BX, (g.n[1] + B::BY - 1) / B::BY,
                    DIM == 3 ? (g.n[2] + B::BZ - 1) / B::BZ : 1);
    adj_flux_tile_kernel<DIM, T><<<grid, FT, B::SMEM, s>>>(g, u, v, tbuf);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nb = grid_for(g.N);
    if (mode == 0)
        adj_prim_kernel<DIM, T, 0><<<nb, AT, 0, s>>>(g, u, tbuf, nullptr, (T *)lam, (T *)mu, dt);
    else if (mode == 1)
        adj_prim_kernel<DIM, T, 1><<<nb, AT, 0, s>>>(g, u, tbuf, nullptr, (T *)lam, (T *)mu, dt);
    else
        adj_prim_kernel<DIM, T, -1><<<nb, AT, 0, s>>>(g, u, tbuf, (T *)out, nullptr, nullptr, 0.0);
    return cudaGetLastError();
}

template <int DIM, typename T>
cudaError_t reverse_step_t(const GridParams &g, const MarkerBuffers &m, const AdjBuffers &a,
                           const void *Un, double dt, double cd, double nu, int n_sm,
                           cudaStream_t s) {
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    const int bc = 4 * (n_sm > 0 ? n_sm : 1);
    T *lam = (T *)a.lam, *mu = (T *)a.mu;
    cudaError_t e = cudaSuccess;
    if (m.ns > 0) {
        adj_apply_kernel<DIM, T><<<bc, AT, 0, s>>>(g, m, keys, perm, (const T *)a.B, lam,
                                                    (T *)a.lfq);
        adj_marker_kernel<DIM, T><<<(m.ns * 32 + AT - 1) / AT, AT, 0, s>>>(g, m, a,
                                                                            (const T *)a.B, cd, nu);
        adj_interp_kernel<DIM, T><<<bc, AT, 0, s>>>(g, m, keys, perm, a, (const T *)a.B, lam);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // mu = lam/2 + (dt/2) J_L(U1)^T lam, then lam = lam/2 + mu + dt J_L(U)^T mu
    e = rhs_vjp_t<DIM, T>(g, a.A, lam, a.tbuf, nullptr, s, 0, lam, mu, dt);
    if (e != cudaSuccess) return e;
    return rhs_vjp_t<DIM, T>(g, Un, mu, a.tbuf, nullptr, s, 1, lam, mu, dt);
}

template <int DIM>
cudaError_t eps_adjoint_x(const GridParams &g, const MarkerBuffers &m, const AdjBuffers &a,
                          int n_sm, cudaStream_t s) {
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    adj_eps_fields_kernel<DIM><<<4 * (n_sm > 0 ? n_sm : 1), AT, 0, s>>>(g, m, keys, perm, a);
    adj_eps_x_kernel<DIM><<<(m.ns * 32 + AT - 1) / AT, AT, 0, s>>>(g, m, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // lamW[0..1] held the two spread fields; clear them for the next use
    return cudaMemsetAsync(a.lamW, 0, sizeof(double) * 2 * (size_t)g.N, s);
}

}  // namespace

cudaError_t launch_rhs_vjp(const GridParams &g, int fp_bytes, const void *U, const void *V,
                           void *tbuf, void *out, cudaStream_t s) {
    if (g.dim == 3)
        return fp_bytes == 4 ? rhs_vjp_t<3, float>(g, U, V, tbuf, out, s)
                             : rhs_vjp_t<3, double>(g, U, V, tbuf, out, s);
    return fp_bytes == 4 ? rhs_vjp_t<2, float>(g, U, V, tbuf, out, s)
                         : rhs_vjp_t<2, double>(g, U, V, tbuf, out, s);
}

cudaError_t launch_reverse_step(const GridParams &g, int fp_bytes, const MarkerBuffers &m,
                                const AdjBuffers &a, const void *Un, double dt, double cd,
                                double nu, int n_sm, cudaStream_t s) {
    if (g.dim == 3)
        return fp_bytes == 4 ? reverse_step_t<3, float>(g, m, a, Un, dt, cd, nu, n_sm, s)
                             : reverse_step_t<3, double>(g, m, a, Un, dt, cd, nu, n_sm, s);
    return fp_bytes == 4 ? reverse_step_t<2, float>(g, m, a, Un, dt, cd, nu, n_sm, s)
                         : reverse_step_t<2, double>(g, m, a, Un, dt, cd, nu, n_sm, s);
}

cudaError_t launch_eps_adjoint_x(const GridParams &g, const MarkerBuffers &m, const AdjBuffers &a,
                                 int n_sm, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    return g.dim == 3 ? eps_adjoint_x<3>(g, m, a, n_sm, s) : eps_adjoint_x<2>(g, m, a, n_sm, s);
}

}  // namespace ibmk

// ---------------------------------------------------------------------------
// C ABI: recording, the reverse sweep, and the transpose-Jacobian diagnostic
// ---------------------------------------------------------------------------

using namespace ibmk;

namespace {

size_t aup(size_t x) { return (x + 255) / 256 * 256; }

// bytes of the flux transpose's per-tile accumulators: every tile of the
// reverse flux kernel keeps its tile-plus-halo sums (dim+2 fields)
template <int DIM, typename T> size_t tile_buf_bytes_t(const int *n) {
    using B = AdjBox<DIM, T>;
    const size_t tiles = (size_t)((n[0] + B::BX - 1) / B::BX) * ((n[1] + B::BY - 1) / B::BY) *
                         (DIM == 3 ? (n[2] + B::BZ - 1) / B::BZ : 1);
    return tiles * (DIM + 2) * B::PN * sizeof(T);
}
size_t adj_tile_buf_bytes(const ibm_grid_desc &d) {
    if (d.dim == 3)
        return d.fp_bytes == 4 ? tile_buf_bytes_t<3, float>(d.n) : tile_buf_bytes_t<3, double>(d.n);
    return d.fp_bytes == 4 ? tile_buf_bytes_t<2, float>(d.n) : tile_buf_bytes_t<2, double>(d.n);
}

size_t state_bytes_of(const ibm_grid_desc &d) {
    long long N = 1;
    for (int i = 0; i < d.dim; ++i) N *= d.n[i];
    return (size_t)N * (d.dim + 2) * d.fp_bytes;
}

// carve (base != nullptr) or measure the adjoint workspace
size_t adj_layout(const ibm_grid_desc &d, int cap, int max_steps, int every, char *base,
                  AdjBuffers *a) {
    long long N = 1;
    for (int i = 0; i < d.dim; ++i) N *= d.n[i];
    const size_t SB = aup(state_bytes_of(d));
    const int n_ckpt = (max_steps + every - 1) / every;
    const size_t c1 = cap > 0 ? (size_t)cap : 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += aup(bytes > 0 ? bytes : 1);
        return p;
    };
    AdjBuffers b;
    b.max_steps = max_steps;
    b.every = every;
    b.n_ckpt = n_ckpt;
    b.cap = cap;
    b.ckpt = take(SB * n_ckpt);
    b.dt_hist = (double *)take(sizeof(double) * max_steps);
    b.seg = take(SB * every);
    b.seg1 = take(SB * every);
    b.segs = take(SB * every);
    b.segf = (double *)take(sizeof(double) * 5 * c1 * every);
    b.A = take(SB);
    b.B = take(SB);
    b.lam = take(SB);
    b.mu = take(SB);
    b.jtv = take(SB);
    b.lfq = take(SB);
    b.lamW = take(sizeof(double) * (size_t)N * (d.dim + 2));
    b.tbuf = take(adj_tile_buf_bytes(d));
    b.lamX = (double *)take(sizeof(double) * 3 * c1);
    b.lamTw = (double *)take(sizeof(double) * c1);
    b.lamEps = (double *)take(sizeof(double) * c1);
    b.mr = (double *)take(sizeof(double) * 5 * c1);
    b.z = (double *)take(sizeof(double) * c1);
    b.save = (double *)take(sizeof(double) * 5 * c1);
    if (a) *a = b;
    return off;
}

ibm_status afail(ibm_grid *g, ibm_status st, const std::string &msg) {
    g->err = msg;
    return st;
}

#define ACU(call, where)                                                                      \
    do {                                                                                      \
        cudaError_t _e = (call);                                                              \
        if (_e != cudaSuccess)                                                                \
            return afail(g, IBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
    } while (0)

int marker_ctas(const ibm_grid *g) {
    const int c = 4 * (g->n_sm > 0 ? g->n_sm : 1);
    return c < 4096 ? c : 4096;
}

// one forward step from Un into Unext with a given dt (no finish: the
// handle's time, sums and step size are left alone)
// The marker buffers with the forcing (rho_L, G, H) of segment step i
// redirected into the segment store.
MarkerBuffers seg_markers(const ibm_grid *g, int i) {
    MarkerBuffers m = g->mb;
    const size_t c1 = g->adj.cap > 0 ? (size_t)g->adj.cap : 1;
    double *f = g->adj.segf + (size_t)i * 5 * c1;
    m.rhoL = f;
    m.G = f + c1;
    m.H = f + 4 * c1;
    return m;
}

// One recorded step again (its recorded dt), keeping what its reverse needs:
// U1 into U1s, U* before the forcing into Uss, the marker forcing into m.
ibm_status replay_step(ibm_grid *g, const void *Un, void *Unext, double dt, void *U1s,
                       void *Uss, const MarkerBuffers &m) {
    const int fpb = g->desc.fp_bytes;
    ACU(launch_stage1(g->gp, fpb, Un, U1s, g->fb, dt, g->stream), "replay stage 1");
    ACU(launch_stage2(g->gp, fpb, Un, U1s, Unext, g->fb, dt, g->stream), "replay stage 2");
    ACU(cudaMemcpyAsync(Uss, Unext, state_bytes_of(g->desc), cudaMemcpyDeviceToDevice, g->stream),
        "keep U*");
    if (g->mb.ns > 0) {
        ACU(launch_interp_force(g->gp, fpb, Unext, m, marker_ctas(g), g->stream), "replay interp");
        ACU(launch_spread_apply(g->gp, fpb, Unext, m, marker_ctas(g), g->stream), "replay spread");
    }
    return IBM_OK;
}

ibm_status sync_errors(ibm_grid *g) {
    ibm_status st = ibm_sync(g);
    return st;
}

}  // namespace

extern "C" {

size_t ibm_adjoint_workspace_bytes(const ibm_grid_desc *desc, int max_markers, int max_steps,
                                   int every) {
    if (!desc || ibm_workspace_bytes(desc, max_markers < 0 ? 0 : max_markers) == 0) return 0;
    if (max_markers < 0 || max_steps < 1 || every < 1) return 0;
    return adj_layout(*desc, max_markers, max_steps, every, nullptr, nullptr);
}

ibm_status ibm_record(ibm_grid *g, int max_steps, int every, void *dev_workspace, size_t bytes) {
    if (!g) return IBM_ERR_ARG;
    if (max_steps < 1 || every < 1) return afail(g, IBM_ERR_ARG, "max_steps and every must be >= 1");
    if (!dev_workspace || ((uintptr_t)dev_workspace) % 256 != 0)
        return afail(g, IBM_ERR_ARG, "adjoint workspace must be non-null and 256-byte aligned");
    if (g->moving && g->mb.ns > 0)
        return afail(g, IBM_ERR_UNSUPPORTED, "the adjoint takes static markers only");
    if (g->desc.forcing_per_stage)
        return afail(g, IBM_ERR_UNSUPPORTED, "the adjoint reverses the once-per-step forcing only");
    const size_t need = adj_layout(g->desc, g->max_markers, max_steps, every, nullptr, nullptr);
    if (bytes < need)
        return afail(g, IBM_ERR_WORKSPACE,
                     "adjoint workspace too small: need " + std::to_string(need) + " bytes");
    adj_layout(g->desc, g->max_markers, max_steps, every, (char *)dev_workspace, &g->adj);
    long long N = g->gp.N;
    ACU(cudaMemsetAsync(g->adj.lamW, 0, sizeof(double) * (size_t)N * (g->desc.dim + 2), g->stream),
        "clear accumulators");
    g->recording = true;
    g->rec_steps = 0;
    return IBM_OK;
}

ibm_status ibm_rhs_vjp(ibm_grid *g, const void *U, const void *V, void *out) {
    if (!g) return IBM_ERR_ARG;
    if (!U || !V || !out) return afail(g, IBM_ERR_ARG, "null buffer");
    if (!g->recording) return afail(g, IBM_ERR_STATE, "ibm_record must come first (it holds the scratch)");
    ACU(launch_rhs_vjp(g->gp, g->desc.fp_bytes, U, V, g->adj.tbuf, out, g->stream), "rhs vjp");
    return IBM_OK;
}

ibm_status ibm_backward(ibm_grid *g, double dJ_dCd, double dJ_dNu, double *dJ_dX, double *dJ_dTw) {
    if (!g) return IBM_ERR_ARG;
    if (!g->recording || g->rec_steps < 1)
        return afail(g, IBM_ERR_STATE, "no recorded steps: ibm_record, then ibm_step");
    if (g->moving && g->mb.ns > 0)
        return afail(g, IBM_ERR_UNSUPPORTED, "the adjoint takes static markers only");
    const int ns = g->mb.ns, dim = g->desc.dim;
    if (ns < 1) return afail(g, IBM_ERR_ARG, "no markers");
    if (!isfinite(dJ_dCd) || !isfinite(dJ_dNu)) return afail(g, IBM_ERR_ARG, "non-finite weights");
    const AdjBuffers &a = g->adj;
    const int S = g->rec_steps, K = a.every;
    const size_t SB = aup(state_bytes_of(g->desc));
    const size_t sb = state_bytes_of(g->desc);
    cudaStream_t s = g->stream;

    std::vector<double> dts((size_t)S), sums(8, 0.0);
    ACU(cudaMemcpyAsync(dts.data(), a.dt_hist, sizeof(double) * S, cudaMemcpyDeviceToHost, s), "read dt");
    ACU(cudaMemcpyAsync(sums.data(), g->mb.sums, sizeof(double) * 8, cudaMemcpyDeviceToHost, s), "read sums");
    ibm_status st = sync_errors(g);
    if (st != IBM_OK) return st;

    // direct terms of J at the last step (Eq. Bulk, with the coefficients
    // and Nu of ibm_forces_and_nusselt)
    double f3[3], heat, Cd, Cl, Nu;
    forces_from_sums(g, sums.data(), f3, &heat, &Cd, &Cl, &Nu);
    const double pi = 3.14159265358979323846;
    const double hd = pow(g->desc.h, dim), dtN = sums[4];
    const double lref = dim == 2 ? g->desc.D : pi * g->desc.D * g->desc.D / 4.0;
    const double As = dim == 2 ? pi * g->desc.D : pi * g->desc.D * g->desc.D;
    const double lam_inf = g->desc.Re > 0.0 ? g->gp.mu_inf * g->gp.cp / g->desc.Pr : 0.0;
    double tw = 0.0;
    for (double v : g->Tw_h) tw += v;
    const double dT = tw / ns - 1.0;
    if (!(dtN > 0.0)) return afail(g, IBM_ERR_STATE, "the last step size is not positive");
    const double cd = dJ_dCd * (2.0 / lref) * (-hd / dtN);
    double nu = 0.0, tw_direct = 0.0;
    if (dJ_dNu != 0.0) {
        if (!(lam_inf > 0.0) || dT == 0.0)
            return afail(g, IBM_ERR_ARG, "Nu is undefined (inviscid, or mean T_w = T_inf)");
        nu = dJ_dNu * g->desc.D * hd / (dtN * lam_inf * As * dT);
        tw_direct = -dJ_dNu * Nu / (dT * ns);
    }

    // the last forward step's marker forcing is recomputed below; keep it
    ACU(cudaMemcpyAsync(a.save, g->mb.rhoL, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "save");
    ACU(cudaMemcpyAsync(a.save + ns, g->mb.G, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, s), "save");
    ACU(cudaMemcpyAsync(a.save + (size_t)ns * (dim + 1), g->mb.H, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "save");
    ACU(cudaMemsetAsync(a.lam, 0, sb, s), "clear adjoint");
    ACU(cudaMemsetAsync(a.lamX, 0, sizeof(double) * 3 * ns, s), "clear");
    ACU(cudaMemsetAsync(a.lamTw, 0, sizeof(double) * ns, s), "clear");
    ACU(cudaMemsetAsync(a.lamEps, 0, sizeof(double) * ns, s), "clear");

    const int fpb = g->desc.fp_bytes;
    for (int seg = (S - 1) / K; seg >= 0; --seg) {
        const int s0 = seg * K, s1 = S < s0 + K ? S : s0 + K;
        char *segb = (char *)a.seg;
        ACU(cudaMemcpyAsync(segb, (char *)a.ckpt + (size_t)seg * SB, sb, cudaMemcpyDeviceToDevice, s),
            "restore checkpoint");
        // replay the segment, keeping each step's U1, U* and marker forcing
        // (the last step's successor state is not needed: it goes to the
        // scratch state jtv)
        for (int n = s0; n < s1; ++n) {
            const size_t i = (size_t)(n - s0);
            void *next = n + 1 < s1 ? (void *)(segb + (i + 1) * SB) : a.jtv;
            st = replay_step(g, segb + i * SB, next, dts[n], (char *)a.seg1 + i * SB,
                             (char *)a.segs + i * SB, seg_markers(g, (int)i));
            if (st != IBM_OK) return st;
        }
        for (int n = s1 - 1; n >= s0; --n) {
            const size_t i = (size_t)(n - s0);
            const void *Un = segb + i * SB;
            AdjBuffers an = a;
            an.A = (char *)a.seg1 + i * SB;
            an.B = (char *)a.segs + i * SB;
            const bool last = n == S - 1;
            ACU(launch_reverse_step(g->gp, fpb, seg_markers(g, (int)i), an, Un, dts[n],
                                    last ? cd : 0.0, last ? nu : 0.0, g->n_sm, s),
                "reverse step");
        }
    }

    // eps~ = A~^{-1} 1: dJ/dX += -sum_j dPhi (z_k S(eps~) + eps~_k S(z)), A~ z = dJ/deps~
    std::vector<double> le((size_t)ns);
    ACU(cudaMemcpyAsync(le.data(), a.lamEps, sizeof(double) * ns, cudaMemcpyDeviceToHost, s), "read");
    ACU(cudaStreamSynchronize(s), "stream synchronize");
    double scale = 0.0;
    for (double v : le) scale = fmax(scale, fabs(v));
    if (scale > 0.0) {
        ACU(launch_quadrature_solve(ns, g->qb, a.lamEps, a.z, 1e-12 * scale, g->cg_maxit, g->err_d, s),
            "adjoint quadrature solve");
        ACU(launch_eps_adjoint_x(g->gp, g->mb, a, g->n_sm, s), "weights adjoint");
    }

    std::vector<double> gx((size_t)ns * 3), gt((size_t)ns);
    ACU(cudaMemcpyAsync(gx.data(), a.lamX, sizeof(double) * 3 * ns, cudaMemcpyDeviceToHost, s), "read");
    ACU(cudaMemcpyAsync(gt.data(), a.lamTw, sizeof(double) * ns, cudaMemcpyDeviceToHost, s), "read");
    ACU(cudaMemcpyAsync(g->mb.rhoL, a.save, sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "restore");
    ACU(cudaMemcpyAsync(g->mb.G, a.save + ns, sizeof(double) * ns * dim, cudaMemcpyDeviceToDevice, s), "restore");
    ACU(cudaMemcpyAsync(g->mb.H, a.save + (size_t)ns * (dim + 1), sizeof(double) * ns, cudaMemcpyDeviceToDevice, s), "restore");
    st = sync_errors(g);
    if (st != IBM_OK) return st;
    if (dJ_dX)
        for (int k = 0; k < ns; ++k)
            for (int d = 0; d < dim; ++d) dJ_dX[(size_t)k * dim + d] = gx[(size_t)k * 3 + d];
    if (dJ_dTw)
        for (int k = 0; k < ns; ++k) dJ_dTw[k] = gt[k] + tw_direct;
    return IBM_OK;
}

}  // extern "C"
