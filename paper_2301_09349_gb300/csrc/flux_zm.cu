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
//   - the z-face above each column is evaluated by the column's thread and
//     kept in registers as the next plane's lower face,
//   - each thread forms its cell's flux divergence and writes its output.
// All constants are single precision: the kernel issues no FP64 work
// except the step-size reduction.
#include <float.h>

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
constexpr size_t SMEM = sizeof(float) * (size_t)(RING * SLOT + NC * TY * FXW + NC * (TY + 1) * TX);

struct FC {
    float gamma, inv_gm1, gm1, invR, mu_inf, S, onepS, lam_fac, inv_h, qinv_h, kvisc, E_inf;
    int viscous;
};

FC make_fc(const GridParams &g) {
    FC c;
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

__device__ __forceinline__ float vl(float a, float b) {
    const float ab = a * b;
    return ab > 0.0f ? __fdividef(2.0f * ab, a + b) : 0.0f;
}

// Numerical flux through the face between ring cells a and b (normal axis
// D).  am / bp are the next cells outward along the normal; t1* and t2* are
// the neighbours of a and b along the two tangential axes E1 < E2.
template <int D>
__device__ __forceinline__ void face(const FC &c, const float *__restrict__ R, int am, int a, int b,
                                     int bp, int t1ap, int t1am, int t1bp, int t1bm, int t2ap,
                                     int t2am, int t2bp, int t2bm, float (&F)[NC]) {
    constexpr int E1 = D == 0 ? 1 : 0;
    constexpr int E2 = D == 2 ? 1 : 2;
    float wl[NC], wr[NC];
#pragma unroll
    for (int m = 0; m < NC; ++m) {
        const float *w = R + m * PP;
        const float x0 = w[am], x1 = w[a], x2 = w[b], x3 = w[bp];
        const float d0 = x1 - x0, d1 = x2 - x1, d2 = x3 - x2;
        wl[m] = x1 + 0.5f * vl(d0, d1);
        wr[m] = x2 - 0.5f * vl(d1, d2);
    }
    const float keL = wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3];
    const float keR = wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
    const float EL = wl[4] * c.inv_gm1 + 0.5f * wl[0] * keL;
    const float ER = wr[4] * c.inv_gm1 + 0.5f * wr[0] * keR;
    const float unL = wl[1 + D], unR = wr[1 + D];
    const float cL2 = __fdividef(c.gamma * wl[4], wl[0]);
    const float cR2 = __fdividef(c.gamma * wr[4], wr[0]);
    const float sL = fabsf(unL) + cL2 * rsqrtf(cL2);
    const float sR = fabsf(unR) + cR2 * rsqrtf(cR2);
    const float smax = fmaxf(sL, sR);
    F[0] = 0.5f * (wl[0] * unL + wr[0] * unR) - 0.5f * smax * (wr[0] - wl[0]);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const float mL = wl[0] * wl[1 + m], mR = wr[0] * wr[1 + m];
        const float fL = mL * unL + (m == D ? wl[4] : 0.0f);
        const float fR = mR * unR + (m == D ? wr[4] : 0.0f);
        F[1 + m] = 0.5f * (fL + fR) - 0.5f * smax * (mR - mL);
    }
    F[4] = 0.5f * ((EL + wl[4]) * unL + (ER + wr[4]) * unR) - 0.5f * smax * (ER - EL);

    if (!c.viscous) return;
    const float *Tc = R + 5 * PP;
    const float Ta = Tc[a], Tb = Tc[b];
    const float Tf = 0.5f * (Ta + Tb);
    const float mu = __fdividef(c.mu_inf * Tf * (Tf * rsqrtf(Tf)) * c.onepS, Tf + c.S);
    const float lam = mu * c.lam_fac;
    const float *uD = R + (1 + D) * PP;
    const float *u1 = R + (1 + E1) * PP;
    const float *u2 = R + (1 + E2) * PP;
    const float dn_uD = (uD[b] - uD[a]) * c.inv_h;
    const float dn_u1 = (u1[b] - u1[a]) * c.inv_h;
    const float dn_u2 = (u2[b] - u2[a]) * c.inv_h;
    const float dn_T = (Tb - Ta) * c.inv_h;
    const float d1_uD = (uD[t1ap] - uD[t1am] + uD[t1bp] - uD[t1bm]) * c.qinv_h;
    const float d2_uD = (uD[t2ap] - uD[t2am] + uD[t2bp] - uD[t2bm]) * c.qinv_h;
    const float d1_u1 = (u1[t1ap] - u1[t1am] + u1[t1bp] - u1[t1bm]) * c.qinv_h;
    const float d2_u2 = (u2[t2ap] - u2[t2am] + u2[t2bp] - u2[t2bm]) * c.qinv_h;
    const float div = dn_uD + d1_u1 + d2_u2;
    const float tDD = mu * (2.0f * dn_uD - (2.0f / 3.0f) * div);
    const float tD1 = mu * (d1_uD + dn_u1);
    const float tD2 = mu * (d2_uD + dn_u2);
    const float ufD = 0.5f * (uD[a] + uD[b]);
    const float uf1 = 0.5f * (u1[a] + u1[b]);
    const float uf2 = 0.5f * (u2[a] + u2[b]);
    F[1 + D] -= tDD;
    F[1 + E1] -= tD1;
    F[1 + E2] -= tD2;
    F[4] -= ufD * tDD + uf1 * tD1 + uf2 * tD2 + lam * dn_T;
}

// Load plane gz (ghosts through the boundary conditions), build U1 on the
// fly in stage 2, convert to primitives into one ring slot.
template <int MODE>
__device__ __forceinline__ void load_plane(const GridParams &g, const FC &c,
                                           const float *__restrict__ U,
                                           const float *__restrict__ Lp, float dt,
                                           float *__restrict__ slot, int ox, int oy, int gz,
                                           bool xy_interior) {
    const long long N = g.N;
    const bool fast = xy_interior && gz >= 0 && gz < g.n[2];
    for (int q = threadIdx.x; q < PP; q += NTH) {
        const int lx = q % PX, ly = q / PX;
        float u[NC];
        if (fast) {
            const long long j = (ox + lx - 2) + (long long)g.n[0] * ((oy + ly - 2) + (long long)g.n[1] * gz);
#pragma unroll
            for (int m = 0; m < NC; ++m) {
                float v = __ldg(U + m * N + j);
                if (MODE == 2) v = fmaf(dt, __ldg(Lp + m * N + j), v);
                u[m] = v;
            }
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
                for (int m = 0; m < NC; ++m) {
                    float v = __ldg(U + m * N + j);
                    if (MODE == 2) v = fmaf(dt, __ldg(Lp + m * N + j), v);
                    u[m] = v;
                }
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

// MODE 0: L only.  MODE 1: stage 1 (L and the step size).  MODE 2: stage 2.
template <int MODE>
__global__ void __launch_bounds__(NTH, 2)
zmarch_kernel(const GridParams g, const FC c, int zc, const float *__restrict__ U,
              const float *__restrict__ Lp, float *__restrict__ out,
              double *__restrict__ blockmax, unsigned *__restrict__ counter,
              double *__restrict__ dt_ptr, int *__restrict__ err, double dt_fixed) {
    extern __shared__ __align__(16) float smem_zm[];
    float *ring = smem_zm;
    float *FXb = ring + RING * SLOT;          // [NC][TY][FXW]
    float *FYb = FXb + NC * TY * FXW;         // [NC][TY+1][TX]
    __shared__ double s_red[NTH / 32];
    __shared__ int s_flag;

    const int tid = threadIdx.x, lx = tid & 31, ly = tid >> 5;
    const int ox = blockIdx.x * TX, oy = blockIdx.y * TY;
    const int z0 = blockIdx.z * zc, z1 = min(z0 + zc, g.n[2]);
    const long long N = g.N;
    const float dt = MODE == 2 ? (float)(*dt_ptr) : 0.0f;
    const bool xyint = ox >= 2 && oy >= 2 && ox + TX + 2 <= g.n[0] && oy + TY + 2 <= g.n[1];
    auto slot_of = [](int z) { return ((z % RING) + RING) % RING * SLOT; };

    for (int zz = z0 - 2; zz <= z0 + 1; ++zz)
        load_plane<MODE>(g, c, U, Lp, dt, ring + slot_of(zz), ox, oy, zz, xyint);
    __syncthreads();

    const int cxy = (lx + 2) + PX * (ly + 2);   // own column inside a plane
    float Fz[NC];
    {
        const int sa = slot_of(z0 - 1), sb = slot_of(z0), sam = slot_of(z0 - 2), sbp = slot_of(z0 + 1);
        face<2>(c, ring, sam + cxy, sa + cxy, sb + cxy, sbp + cxy, sa + cxy + 1, sa + cxy - 1,
                sb + cxy + 1, sb + cxy - 1, sa + cxy + PX, sa + cxy - PX, sb + cxy + PX,
                sb + cxy - PX, Fz);
    }
    __syncthreads();

    double smax = 0.0;
    int bad = 0;
    for (int z = z0; z < z1; ++z) {
        load_plane<MODE>(g, c, U, Lp, dt, ring + slot_of(z + 2), ox, oy, z + 2, xyint);
        __syncthreads();
        const int sm1 = slot_of(z - 1), s0 = slot_of(z), s1 = slot_of(z + 1), s2 = slot_of(z + 2);
        const int up = s1 - s0, dn = sm1 - s0;
        // x-faces of row ly: face lx lies between cells lx-1 and lx
        {
            float F[NC];
            const int a = s0 + (lx + 1) + PX * (ly + 2), b = a + 1;
            face<0>(c, ring, a - 1, a, b, b + 1, a + PX, a - PX, b + PX, b - PX, a + up, a + dn,
                    b + up, b + dn, F);
#pragma unroll
            for (int m = 0; m < NC; ++m) FXb[(m * TY + ly) * FXW + lx] = F[m];
            if (ly == 0 && lx < TY) {   // the last face of each row
                const int a2 = s0 + (TX + 1) + PX * (lx + 2), b2 = a2 + 1;
                face<0>(c, ring, a2 - 1, a2, b2, b2 + 1, a2 + PX, a2 - PX, b2 + PX, b2 - PX,
                        a2 + up, a2 + dn, b2 + up, b2 + dn, F);
#pragma unroll
                for (int m = 0; m < NC; ++m) FXb[(m * TY + lx) * FXW + TX] = F[m];
            }
        }
        // y-faces: face row ly lies between cell rows ly-1 and ly
        {
            float F[NC];
            const int a = s0 + (lx + 2) + PX * (ly + 1), b = a + PX;
            face<1>(c, ring, a - PX, a, b, b + PX, a + 1, a - 1, b + 1, b - 1, a + up, a + dn,
                    b + up, b + dn, F);
#pragma unroll
            for (int m = 0; m < NC; ++m) FYb[(m * (TY + 1) + ly) * TX + lx] = F[m];
            if (ly == 1) {   // the last face row
                const int a2 = s0 + (lx + 2) + PX * (TY + 1), b2 = a2 + PX;
                face<1>(c, ring, a2 - PX, a2, b2, b2 + PX, a2 + 1, a2 - 1, b2 + 1, b2 - 1,
                        a2 + up, a2 + dn, b2 + up, b2 + dn, F);
#pragma unroll
                for (int m = 0; m < NC; ++m) FYb[(m * (TY + 1) + TY) * TX + lx] = F[m];
            }
        }
        // z-face above the column (between planes z and z+1)
        float Fh[NC];
        face<2>(c, ring, sm1 + cxy, s0 + cxy, s1 + cxy, s2 + cxy, s0 + cxy + 1, s0 + cxy - 1,
                s1 + cxy + 1, s1 + cxy - 1, s0 + cxy + PX, s0 + cxy - PX, s1 + cxy + PX,
                s1 + cxy - PX, Fh);
        __syncthreads();

        float acc[NC];
#pragma unroll
        for (int m = 0; m < NC; ++m) {
            acc[m] = (FXb[(m * TY + ly) * FXW + lx] - FXb[(m * TY + ly) * FXW + lx + 1]) +
                     (FYb[(m * (TY + 1) + ly) * TX + lx] - FYb[(m * (TY + 1) + ly + 1) * TX + lx]) +
                     (Fz[m] - Fh[m]);
            Fz[m] = Fh[m];
        }
        const int gx = ox + lx, gy = oy + ly;
        if (gx < g.n[0] && gy < g.n[1]) {
            const long long j = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * z);
            if (MODE == 2) {
#pragma unroll
                for (int m = 0; m < NC; ++m) {
                    const float un = __ldg(U + m * N + j);
                    const float u1 = fmaf(dt, __ldg(Lp + m * N + j), un);
                    out[m * N + j] = 0.5f * un + 0.5f * fmaf(dt, acc[m] * c.inv_h, u1);
                }
            } else {
#pragma unroll
                for (int m = 0; m < NC; ++m) out[m * N + j] = acc[m] * c.inv_h;
            }
            if (MODE == 1) {
                const float *P = ring + s0;
                const float rho = P[cxy], p = P[4 * PP + cxy], Tt = P[5 * PP + cxy];
                const float c2 = __fdividef(c.gamma * p, rho);
                const float snd = c2 * rsqrtf(c2);
                float mu = 0.0f;
                if (c.viscous) mu = __fdividef(c.mu_inf * Tt * (Tt * rsqrtf(Tt)) * c.onepS, Tt + c.S);
                const float nu = __fdividef(c.kvisc * mu, rho);
                const float s = (fabsf(P[PP + cxy]) + fabsf(P[2 * PP + cxy]) + fabsf(P[3 * PP + cxy]) +
                                 3.0f * snd) * c.inv_h + 6.0f * nu * c.inv_h * c.inv_h;
                if (!(rho > 0.0f && p > 0.0f && s <= FLT_MAX)) bad = 1;
                else smax = fmax(smax, (double)s);
            }
        }
    }

    if (MODE == 1) {
        smax = warp_max_d(smax);
        bad = __syncthreads_or(bad);
        if ((tid & 31) == 0) s_red[tid >> 5] = smax;
        __syncthreads();
        const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
        const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        if (tid == 0) {
            double m = s_red[0];
            for (int w = 1; w < NTH / 32; ++w) m = fmax(m, s_red[w]);
            blockmax[bid] = m;
            if (bad) record_error(err, ERR_NONFINITE);
            __threadfence();
            const unsigned ticket = atomicAdd(counter, 1u);
            s_flag = ticket == nblocks - 1;
        }
        __syncthreads();
        if (s_flag) {
            __threadfence();
            double m = 0.0;
            for (unsigned b = tid; b < nblocks; b += NTH) m = fmax(m, __ldcg(blockmax + b));
            m = warp_max_d(m);
            if ((tid & 31) == 0) s_red[tid >> 5] = m;
            __syncthreads();
            if (tid == 0) {
                double mm = s_red[0];
                for (int w = 1; w < NTH / 32; ++w) mm = fmax(mm, s_red[w]);
                double dtv;
                if (dt_fixed > 0.0) {
                    dtv = dt_fixed;
                } else if (mm > 0.0 && mm <= DBL_MAX) {
                    dtv = g.cfl / mm;
                } else {
                    dtv = 0.0;
                    record_error(err, ERR_NONFINITE);
                }
                if (__ldcg(err) & ERR_NONFINITE) dtv = 0.0;
                *dt_ptr = dtv;
                *counter = 0u;
            }
        }
    }
}

}  // namespace

int zmarch_chunk(const GridParams &g) {
    // planes per CTA: enough CTAs to fill the GPU several times over
    const long long cols = (long long)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY);
    int zc = 32;
    while (zc > 8 && cols * ((g.n[2] + zc - 1) / zc) < 8 * 152) zc /= 2;
    return zc;
}

size_t zmarch_blocks(const GridParams &g) {
    const int zc = zmarch_chunk(g);
    return (size_t)((g.n[0] + TX - 1) / TX) * ((g.n[1] + TY - 1) / TY) * ((g.n[2] + zc - 1) / zc);
}

template <int MODE>
static cudaError_t zm_launch(const GridParams &g, const void *U, const void *Lp, void *out,
                             const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(zmarch_kernel<MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int zc = zmarch_chunk(g);
    dim3 grid((g.n[0] + TX - 1) / TX, (g.n[1] + TY - 1) / TY, (g.n[2] + zc - 1) / zc);
    zmarch_kernel<MODE><<<grid, NTH, SMEM, s>>>(g, make_fc(g), zc, (const float *)U,
                                                (const float *)Lp, (float *)out, fb.blockmax,
                                                fb.counter, fb.dt, fb.err, dt_fixed);
    return cudaGetLastError();
}

cudaError_t launch_zmarch(int mode, const GridParams &g, const void *U, const void *Lp, void *out,
                          const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    if (mode == 1) return zm_launch<1>(g, U, Lp, out, fb, dt_fixed, s);
    if (mode == 2) return zm_launch<2>(g, U, Lp, out, fb, dt_fixed, s);
    return zm_launch<0>(g, U, Lp, out, fb, dt_fixed, s);
}

}  // namespace ibmk
