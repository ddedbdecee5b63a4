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
#include <float.h>

#include "internal.h"

namespace ibmk {
namespace {

constexpr int NT = 256;

template <int DIM, typename T> struct TileShape;
template <> struct TileShape<3, float> { static constexpr int BX = 8, BY = 8, BZ = 8; };
template <> struct TileShape<3, double> { static constexpr int BX = 8, BY = 8, BZ = 4; };
template <> struct TileShape<2, float> { static constexpr int BX = 16, BY = 16, BZ = 1; };
template <> struct TileShape<2, double> { static constexpr int BX = 16, BY = 16, BZ = 1; };

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int DIM, typename T>
struct Box {
    static constexpr int BX = TileShape<DIM, T>::BX, BY = TileShape<DIM, T>::BY,
                         BZ = TileShape<DIM, T>::BZ;
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
    static constexpr size_t SMEM = sizeof(T) * (size_t)(NW * PN + NC * NFMAX);
};

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

// Numerical flux through the face between box cells a and a + s_D.
template <int DIM, typename T, int D>
__device__ __forceinline__ void face_flux(const GridParams &g, const T *__restrict__ sW, int a,
                                          T (&F)[DIM + 2]) {
    using B = Box<DIM, T>;
    constexpr int s = D == 0 ? B::SX : (D == 1 ? B::SY : B::SZ);
    constexpr int NC = DIM + 2;
    const int b = a + s;
    const T gam = (T)g.gamma;
    const T inv_gm1 = (T)(1.0 / (g.gamma - 1.0));

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

    if (g.mu_inf <= 0.0) return;

    // viscous stress and heat flux; face values from the two adjacent cells,
    // tangential derivatives from the average of the two cells' central
    // differences
    const T inv_h = (T)g.inv_h;
    const T *Tc = sW + (DIM + 2) * B::PN;
    const T Tf = T(0.5) * (Tc[a] + Tc[b]);
    const T Sv = (T)g.S;
    const T mu = fdiv<T>((T)g.mu_inf * Tf * psqrt<T>(Tf) * (T(1) + Sv), Tf + Sv);
    const T lam = mu * (T)(g.cp / g.Pr);
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

// One direction: evaluate all faces of the tile normal to axis D, then add
// each cell's flux difference to its accumulator.
template <int DIM, typename T, int D>
__device__ __forceinline__ void direction_pass(const GridParams &g, const T *__restrict__ sW,
                                               T *__restrict__ sF,
                                               T (&acc)[Box<DIM, T>::CPT][DIM + 2]) {
    using B = Box<DIM, T>;
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
        face_flux<DIM, T, D>(g, sW, a, F);
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

// MODE 0: out = L(Uin).  MODE 1: out = U1 = Uin + dt L(Uin).
// MODE 2: out = U* = Un/2 + (Uin + dt L(Uin))/2 with Uin = U1, plus the
// per-CTA maximum of s_j(U*) over the cells outside the band.
template <int DIM, typename T, int MODE>
__global__ void __launch_bounds__(NT)
stage_kernel(const GridParams g, const T *__restrict__ Uin, const T *__restrict__ Un,
             T *__restrict__ out, double *__restrict__ blockmax, const double *__restrict__ dt_ptr,
             int *__restrict__ err, const unsigned *__restrict__ band_bits, double dt_fixed) {
    using B = Box<DIM, T>;
    constexpr int NC = DIM + 2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sW = reinterpret_cast<T *>(smem_raw);
    T *sF = sW + B::NW * B::PN;
    __shared__ double s_red[NT / 32];

    const int tid = threadIdx.x;
    const int ox = blockIdx.x * B::BX, oy = blockIdx.y * B::BY;
    const int oz = DIM == 3 ? blockIdx.z * B::BZ : 0;
    const long long N = g.N;
    const T dt = MODE == 0 ? T(0) : (T)(dt_fixed > 0.0 ? dt_fixed : *dt_ptr);
    const T gm1 = (T)(g.gamma - 1.0);
    const T invR = (T)(1.0 / g.R);

    // ---- load tile + halo, to primitives
    // Tiles whose halo lies inside the domain index directly; the others map
    // every halo index through the boundary conditions.
    const bool interior = ox >= 2 && oy >= 2 && ox + B::BX + 2 <= g.n[0] &&
                          oy + B::BY + 2 <= g.n[1] &&
                          (DIM == 2 || (oz >= 2 && oz + B::BZ + 2 <= g.n[2]));
    const T p_inf_E = (T)(g.p_inf / (g.gamma - 1.0) + 0.5);
    for (int q = tid; q < B::PN; q += NT) {
        const int lx = q % B::PX;
        const int r = q / B::PX;
        const int ly = r % B::PY;
        const int lz = r / B::PY;
        T u[NC];
        if (interior) {
            const long long j = (ox + lx - 2) +
                                (long long)g.n[0] * ((oy + ly - 2) + (long long)g.n[1] * (oz + lz - 2 * (DIM == 3)));
#pragma unroll
            for (int c = 0; c < NC; ++c) u[c] = __ldg(Uin + c * N + j);
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
#pragma unroll
                for (int c = 0; c < NC; ++c) u[c] = __ldg(Uin + c * N + j);
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
    direction_pass<DIM, T, 0>(g, sW, sF, acc);
    direction_pass<DIM, T, 1>(g, sW, sF, acc);
    if constexpr (DIM == 3) direction_pass<DIM, T, 2>(g, sW, sF, acc);

    // ---- outputs
    const T inv_h = (T)g.inv_h;
    double smax = 0.0;
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
                smax = fmax(smax, (double)sj);
            }
        }
    }

    if (MODE == 2) {
        smax = warp_max(smax);
        const int bad = __syncthreads_or(!ok);
        if ((tid & 31) == 0) s_red[tid >> 5] = smax;
        __syncthreads();
        if (tid == 0) {
            double m = s_red[0];
            for (int w = 1; w < NT / 32; ++w) m = fmax(m, s_red[w]);
            blockmax[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z)] = m;
            if (bad) record_error(err, ERR_NONFINITE);
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

template <int DIM, typename T>
dim3 stage_grid(const GridParams &g) {
    using B = Box<DIM, T>;
    return dim3((g.n[0] + B::BX - 1) / B::BX, (g.n[1] + B::BY - 1) / B::BY,
                DIM == 3 ? (g.n[2] + B::BZ - 1) / B::BZ : 1);
}

template <int DIM, typename T, int MODE>
cudaError_t launch_one(const GridParams &g, const void *Uin, const void *Un, void *out,
                       const FluidBuffers &fb, double dt_fixed, cudaStream_t s) {
    using B = Box<DIM, T>;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(stage_kernel<DIM, T, MODE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)B::SMEM);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    stage_kernel<DIM, T, MODE><<<stage_grid<DIM, T>(g), NT, B::SMEM, s>>>(
        g, (const T *)Uin, (const T *)Un, (T *)out, fb.blockmax, fb.dt, fb.err, fb.band_bits,
        dt_fixed);
    return cudaGetLastError();
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

}  // namespace

size_t fluid_stage_blocks(const GridParams &g, int fp_bytes) {
    dim3 d;
    if (g.dim == 3 && fp_bytes == 4) return zmarch_blocks(g);
    if (g.dim == 3) d = stage_grid<3, double>(g);
    else d = fp_bytes == 4 ? stage_grid<2, float>(g) : stage_grid<2, double>(g);
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
