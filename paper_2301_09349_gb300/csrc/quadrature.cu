// Lagrangian quadrature of Sec. 2.2: the weights eps solve A eps = 1 with
// A_kl the overlap of the k-th and l-th interpolation kernels, so that
// interpolating a spread unit field returns 1 at every marker.  Taken in
// dimensionless form A~_kl = sum_j Phi_k(j) Phi_l(j), A~ eps~ = 1,
// eps = h^d eps~.
//
// Because Phi is a tensor product, A~_kl = prod_d sum_i phi(r_k,d(i))
// phi(r_l,d(i)) over the three support columns of k on each axis.  Rows are
// assembled in ELL form (column-major, one warp per marker, neighbours
// found through the marker bins in a fixed order).  Up to 160 markers a
// single CTA factors the dense matrix (Cholesky, FP64); above, a single CTA
// runs Jacobi-preconditioned CG in FP64 with fixed-order block reductions.
// Either way the result is bitwise reproducible; every loop is bounded.
#include "internal.h"

namespace ibmk {
namespace {

// Row k of A~: one warp per marker, one lane per neighbour cell of its owner
// cell (the 5^d cells whose markers can overlap its support), visited in
// (z, y, x) order and bin order within a cell; a warp scan of the per-cell
// counts places every entry where a serial walk would, so the rows are the
// same whatever the warp size.
template <int DIM>
__global__ void __launch_bounds__(128)
assemble_kernel(const GridParams g, const MarkerBuffers m, const QuadBuffers q,
                const unsigned *__restrict__ keys, const int *__restrict__ perm) {
    constexpr int NCELLS = DIM == 3 ? 125 : 25;
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= m.ns) return;
    int ck[3] = {0, 0, 0};
    double wk[3][3];
    for (int d = 0; d < DIM; ++d) {
        ck[d] = m.cell[(long long)k * 3 + d];
        const double fk = m.frac_d[(long long)k * 3 + d];
        for (int i = 0; i < 3; ++i) wk[d][i] = phi_d(((double)(i - 1) + 0.5) - fk);
    }
    int base = 0;
    bool overflow = false;
    for (int r0 = 0; r0 < NCELLS; r0 += 32) {
        const int c = r0 + lane;
        int lo = 0, end = 0;
        if (c < NCELLS) {
            const int ox = c % 5 - 2, oy = (c / 5) % 5 - 2, oz = DIM == 3 ? c / 25 - 2 : 0;
            const int x = ck[0] + ox, y = ck[1] + oy, z = (DIM == 3 ? ck[2] : 0) + oz;
            const bool in = x >= 0 && y >= 0 && z >= 0 && x < g.n[0] && y < g.n[1] &&
                            (DIM == 2 || z < g.n[2]);
            if (in) {
                const unsigned key = cell_key(g, x, y, z);
                const int tc = (int)(key / (unsigned)g.cells_per_tile);
                int a = m.tile_off[tc], b = m.tile_off[tc + 1];
                const int tend = b;
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if (keys[mid] < key) a = mid + 1;
                    else b = mid;
                }
                lo = a;
                end = a;
                while (end < tend && keys[end] == key) ++end;
            }
        }
        const int cnt = end - lo;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int w = base + incl - cnt;
        for (int p = lo; p < end; ++p, ++w) {
            const int l = perm[p];
            double a = 1.0;
            for (int d = 0; d < DIM; ++d) {
                const int cl = m.cell[(long long)l * 3 + d];
                const double fl = m.frac_d[(long long)l * 3 + d];
                double sum = 0.0;
                for (int i = 0; i < 3; ++i)
                    sum += wk[d][i] * phi_d(((double)(ck[d] - 1 + i - cl) + 0.5) - fl);
                a *= sum;
            }
            if (l == k) q.diag[k] = a;
            if (w < q.width) {
                q.col[(long long)w * q.cap + k] = l;
                q.val[(long long)w * q.cap + k] = a;
            } else {
                overflow = true;
            }
        }
        base += tot;
    }
    overflow = __any_sync(0xffffffffu, overflow);
    if (lane == 0) {
        q.cnt[k] = base < q.width ? base : q.width;
        if (overflow) record_error(m.err, ERR_CAPACITY);
    }
}

template <int NTH>
__device__ __forceinline__ double block_sum(double v, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double r = lane < NTH / 32 ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

template <int NTH>
__device__ __forceinline__ double block_max(double v, double *s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double r = lane < NTH / 32 ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

template <int NTH>
__device__ __forceinline__ void spmv(int ns, const QuadBuffers &q, const double *x, double *y) {
    for (int k = threadIdx.x; k < ns; k += NTH) {
        const int c = q.cnt[k];
        double s = 0.0;
        for (int i = 0; i < c; ++i) s += q.val[(long long)i * q.cap + k] * x[q.col[(long long)i * q.cap + k]];
        y[k] = s;
    }
}

template <int NTH>
__global__ void __launch_bounds__(NTH)
pcg_kernel(int ns, const QuadBuffers q, double *x, const double *__restrict__ rhs, double tol,
           int maxit, int warm, int *err) {
    __shared__ double s_red[32];
    double *r = q.r, *z = q.z, *p = q.p, *qv = q.q;
    if (!warm)
        for (int k = threadIdx.x; k < ns; k += NTH) x[k] = 0.0;
    __syncthreads();
    int it = 0;
    bool converged = false;
    double rmax = 0.0;
    for (int restart = 0; restart < 50 && it < maxit && !converged; ++restart) {
        spmv<NTH>(ns, q, x, qv);
        __syncthreads();
        double lm = 0.0;
        for (int k = threadIdx.x; k < ns; k += NTH) {
            r[k] = (rhs ? rhs[k] : 1.0) - qv[k];
            lm = fmax(lm, fabs(r[k]));
        }
        rmax = block_max<NTH>(lm, s_red);
        if (rmax <= tol) { converged = true; break; }
        double lrz = 0.0;
        for (int k = threadIdx.x; k < ns; k += NTH) {
            z[k] = r[k] / q.diag[k];
            p[k] = z[k];
            lrz += r[k] * z[k];
        }
        double rz = block_sum<NTH>(lrz, s_red);
        while (it < maxit) {
            __syncthreads();
            spmv<NTH>(ns, q, p, qv);
            __syncthreads();
            double lpq = 0.0;
            for (int k = threadIdx.x; k < ns; k += NTH) lpq += p[k] * qv[k];
            const double alpha = rz / block_sum<NTH>(lpq, s_red);
            double lr = 0.0;
            for (int k = threadIdx.x; k < ns; k += NTH) {
                x[k] += alpha * p[k];
                r[k] -= alpha * qv[k];
                lr = fmax(lr, fabs(r[k]));
            }
            const double rm = block_max<NTH>(lr, s_red);
            ++it;
            if (rm <= tol) break;
            double lrz2 = 0.0;
            for (int k = threadIdx.x; k < ns; k += NTH) {
                z[k] = r[k] / q.diag[k];
                lrz2 += r[k] * z[k];
            }
            const double rzn = block_sum<NTH>(lrz2, s_red);
            const double beta = rzn / rz;
            rz = rzn;
            for (int k = threadIdx.x; k < ns; k += NTH) p[k] = z[k] + beta * p[k];
        }
        __syncthreads();
    }
    if (!converged) {
        __syncthreads();
        spmv<NTH>(ns, q, x, qv);
        __syncthreads();
        double lm = 0.0;
        for (int k = threadIdx.x; k < ns; k += NTH) lm = fmax(lm, fabs((rhs ? rhs[k] : 1.0) - qv[k]));
        rmax = block_max<NTH>(lm, s_red);
        converged = rmax <= tol;
    }
    if (threadIdx.x == 0) {
        *q.iters = it;
        *q.resid = rmax;
        if (!converged) record_error(err, ERR_NOCONV);
    }
}

// Small systems: A~ is assembled dense in shared memory from the ELL rows and
// factored A~ = L L^T by a right-looking Cholesky (FP64, fixed order, one
// CTA), then the two triangular solves.  ~ns^3/6 multiply-adds against a
// few hundred latency-bound CG iterations; the residual max|rhs - A~ x| is
// checked against tol like the CG's.  A non-positive pivot (A~ not positive
// definite) records ERR_NOCONV.
constexpr int CHOL_T = 512;
#ifndef IBM_CHOL_MAX
#define IBM_CHOL_MAX 160
#endif
constexpr int CHOL_MAX = IBM_CHOL_MAX;   // (ns^2 + ns) doubles of shared memory

__global__ void __launch_bounds__(CHOL_T)
chol_kernel(int ns, const QuadBuffers q, double *x, const double *__restrict__ rhs, double tol,
            int *err) {
    extern __shared__ __align__(16) double sA[];   // [ns][ns] row-major, then b[ns]
    double *b = sA + (size_t)ns * ns;
    __shared__ double s_red[CHOL_T / 32];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    for (int i = tid; i < ns * ns; i += CHOL_T) sA[i] = 0.0;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int k = tid; k < ns; k += CHOL_T) {
        const int c = q.cnt[k];
        for (int i = 0; i < c; ++i)
            sA[(size_t)k * ns + q.col[(long long)i * q.cap + k]] = q.val[(long long)i * q.cap + k];
        b[k] = rhs ? rhs[k] : 1.0;
    }
    __syncthreads();
    // factor: column j of L, then the trailing lower triangle
    for (int j = 0; j < ns; ++j) {
        if (tid == 0) {
            const double d = sA[(size_t)j * ns + j];
            if (!(d > 0.0)) s_bad = 1;
            sA[(size_t)j * ns + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double inv = 1.0 / sA[(size_t)j * ns + j];
        for (int i = j + 1 + tid; i < ns; i += CHOL_T) sA[(size_t)i * ns + j] *= inv;
        __syncthreads();
        // trailing lower triangle: one warp per row, lanes along the row
        for (int i = j + 1 + (tid >> 5); i < ns; i += CHOL_T / 32) {
            const double lij = sA[(size_t)i * ns + j];
            for (int kk = j + 1 + (tid & 31); kk <= i; kk += 32)
                sA[(size_t)i * ns + kk] -= lij * sA[(size_t)kk * ns + j];
        }
        __syncthreads();
    }
    // L y = b (forward), L^T x = y (backward), one unknown per step
    for (int j = 0; j < ns; ++j) {
        if (tid == 0) b[j] /= sA[(size_t)j * ns + j];
        __syncthreads();
        const double yj = b[j];
        for (int i = j + 1 + tid; i < ns; i += CHOL_T) b[i] -= sA[(size_t)i * ns + j] * yj;
        __syncthreads();
    }
    for (int j = ns - 1; j >= 0; --j) {
        if (tid == 0) b[j] /= sA[(size_t)j * ns + j];
        __syncthreads();
        const double xj = b[j];
        for (int i = tid; i < j; i += CHOL_T) b[i] -= sA[(size_t)j * ns + i] * xj;
        __syncthreads();
    }
    for (int k = tid; k < ns; k += CHOL_T) x[k] = b[k];
    __syncthreads();
    // true residual with the ELL matrix
    double lm = 0.0;
    for (int k = tid; k < ns; k += CHOL_T) {
        const int c = q.cnt[k];
        double sum = 0.0;
        for (int i = 0; i < c; ++i)
            sum += q.val[(long long)i * q.cap + k] * x[q.col[(long long)i * q.cap + k]];
        lm = fmax(lm, fabs((rhs ? rhs[k] : 1.0) - sum));
    }
    const double rmax = block_max<CHOL_T>(lm, s_red);
    if (tid == 0) {
        *q.iters = 0;
        *q.resid = rmax;
        if (s_bad || !(rmax <= tol)) record_error(err, ERR_NOCONV);
    }
}

}  // namespace

int quad_row_width(int dim) { return dim == 3 ? 125 * 4 : 25 * 4; }

// A~ x = rhs (rhs == nullptr: all ones): dense Cholesky up to CHOL_MAX
// markers, Jacobi-PCG (warm start if asked) above
static cudaError_t launch_quadrature_solve_w(int ns, const QuadBuffers &qb, const double *rhs,
                                            double *x, double tol, int maxit, int warm, int *err,
                                            cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    if (ns <= CHOL_MAX) {
        const size_t smem = sizeof(double) * ((size_t)ns * ns + ns);
        static bool configured = false;
        if (!configured) {
            cudaError_t e = cudaFuncSetAttribute(
                chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                (int)(sizeof(double) * ((size_t)CHOL_MAX * CHOL_MAX + CHOL_MAX)));
            if (e != cudaSuccess) return e;
            configured = true;
        }
        chol_kernel<<<1, CHOL_T, smem, s>>>(ns, qb, x, rhs, tol, err);
    } else if (ns <= 2048) {
        pcg_kernel<256><<<1, 256, 0, s>>>(ns, qb, x, rhs, tol, maxit, warm, err);
    } else {
        pcg_kernel<1024><<<1, 1024, 0, s>>>(ns, qb, x, rhs, tol, maxit, warm, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_quadrature(const GridParams &g, const MarkerBuffers &m, const QuadBuffers &qb,
                              double tol, int maxit, int warm, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    const int nb = (m.ns * 32 + 127) / 128;   // one warp per marker
    if (g.dim == 3) assemble_kernel<3><<<nb, 128, 0, s>>>(g, m, qb, keys, perm);
    else assemble_kernel<2><<<nb, 128, 0, s>>>(g, m, qb, keys, perm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_quadrature_solve_w(m.ns, qb, nullptr, m.eps, tol, maxit, warm, m.err, s);
}

// A~ x = rhs with the matrix assembled by the last launch_quadrature (the
// adjoint of the weights); x starts from zero.
cudaError_t launch_quadrature_solve(int ns, const QuadBuffers &qb, const double *rhs, double *x,
                                    double tol, int maxit, int *err, cudaStream_t s) {
    return launch_quadrature_solve_w(ns, qb, rhs, x, tol, maxit, 0, err, s);
}

}  // namespace ibmk
