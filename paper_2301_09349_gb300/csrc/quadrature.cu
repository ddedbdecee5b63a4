// Lagrangian quadrature of Sec. 2.2: the weights eps solve A eps = 1 with
// A_kl the overlap of the k-th and l-th interpolation kernels, so that
// interpolating a spread unit field returns 1 at every marker.  Taken in
// dimensionless form A~_kl = sum_j Phi_k(j) Phi_l(j), A~ eps~ = 1,
// eps = h^d eps~.
//
// Because Phi is a tensor product, A~_kl = prod_d sum_i phi(r_k,d(i))
// phi(r_l,d(i)) over the three support columns of k on each axis.  Rows are
// assembled in ELL form (column-major, one thread per marker, neighbours
// found through the marker bins in a fixed order), then a single CTA runs
// Jacobi-preconditioned CG in FP64 with fixed-order block reductions, so the
// result is bitwise reproducible.  Every loop is bounded by maxit.
#include "internal.h"

namespace ibmk {
namespace {

template <int DIM>
__global__ void assemble_kernel(const GridParams g, const MarkerBuffers m, const QuadBuffers q,
                                const unsigned *__restrict__ keys, const int *__restrict__ perm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m.ns) return;
    int ck[3] = {0, 0, 0};
    double wk[3][3];
    for (int d = 0; d < DIM; ++d) {
        ck[d] = m.cell[(long long)k * 3 + d];
        const double fk = m.frac_d[(long long)k * 3 + d];
        for (int i = 0; i < 3; ++i) wk[d][i] = phi_d(((double)(i - 1) + 0.5) - fk);
    }
    int cnt = 0;
    bool overflow = false;
    const int zr = DIM == 3 ? 2 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
        for (int oy = -2; oy <= 2; ++oy)
            for (int ox = -2; ox <= 2; ++ox) {
                const int x = ck[0] + ox, y = ck[1] + oy, z = (DIM == 3 ? ck[2] : 0) + oz;
                if (x < 0 || y < 0 || z < 0 || x >= g.n[0] || y >= g.n[1]) continue;
                if (DIM == 3 && z >= g.n[2]) continue;
                const unsigned key = cell_key(g, x, y, z);
                const int tc = (int)(key / (unsigned)g.cells_per_tile);
                int lo = m.tile_off[tc], hi = m.tile_off[tc + 1];
                const int end = hi;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (keys[mid] < key) lo = mid + 1;
                    else hi = mid;
                }
                for (int p = lo; p < end && keys[p] == key; ++p) {
                    const int l = perm[p];
                    double a = 1.0;
                    for (int d = 0; d < DIM; ++d) {
                        const int cl = m.cell[(long long)l * 3 + d];
                        const double fl = m.frac_d[(long long)l * 3 + d];
                        double s = 0.0;
                        for (int i = 0; i < 3; ++i)
                            s += wk[d][i] * phi_d(((double)(ck[d] - 1 + i - cl) + 0.5) - fl);
                        a *= s;
                    }
                    if (l == k) q.diag[k] = a;
                    if (cnt < q.width) {
                        q.col[(long long)cnt * q.cap + k] = l;
                        q.val[(long long)cnt * q.cap + k] = a;
                        ++cnt;
                    } else {
                        overflow = true;
                    }
                }
            }
    q.cnt[k] = cnt;
    if (overflow) record_error(m.err, ERR_CAPACITY);
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

}  // namespace

int quad_row_width(int dim) { return dim == 3 ? 125 * 4 : 25 * 4; }

cudaError_t launch_quadrature(const GridParams &g, const MarkerBuffers &m, const QuadBuffers &qb,
                              double tol, int maxit, int warm, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    const int nb = (m.ns + 127) / 128;
    if (g.dim == 3) assemble_kernel<3><<<nb, 128, 0, s>>>(g, m, qb, keys, perm);
    else assemble_kernel<2><<<nb, 128, 0, s>>>(g, m, qb, keys, perm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (m.ns <= 2048) pcg_kernel<256><<<1, 256, 0, s>>>(m.ns, qb, m.eps, nullptr, tol, maxit, warm, m.err);
    else pcg_kernel<1024><<<1, 1024, 0, s>>>(m.ns, qb, m.eps, nullptr, tol, maxit, warm, m.err);
    return cudaGetLastError();
}

// A~ x = rhs with the matrix assembled by the last launch_quadrature (the
// adjoint of the weights); x starts from zero.
cudaError_t launch_quadrature_solve(int ns, const QuadBuffers &qb, const double *rhs, double *x,
                                    double tol, int maxit, int *err, cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    if (ns <= 2048) pcg_kernel<256><<<1, 256, 0, s>>>(ns, qb, x, rhs, tol, maxit, 0, err);
    else pcg_kernel<1024><<<1, 1024, 0, s>>>(ns, qb, x, rhs, tol, maxit, 0, err);
    return cudaGetLastError();
}

}  // namespace ibmk
