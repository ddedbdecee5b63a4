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
// single CTA factors the dense matrix (Cholesky in FP32, refined to the FP64
// solution); above, a single CTA
// runs Jacobi-preconditioned CG in FP64 with fixed-order block reductions.
// Either way the result is bitwise reproducible; every loop is bounded.
#include "internal.h"

namespace ibmk {
namespace {

// The 1D weights of every marker at its owner cell and the two beside it,
// per axis: wphi[k][d][i] = phi((i - 1) + 1/2 - frac_d[k][d]) (Eq. 3-point
// delta), one thread per (marker, axis).  FP64 runs at a small fraction of
// the FP32 rate on this GPU, so the assembly multiplies these tabulated
// weights instead of evaluating phi for every pair of markers.
__global__ void support_weights_kernel(const MarkerBuffers m, int dim) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = t / 3, d = t - 3 * k;
    if (k >= m.ns || d >= dim) return;
    const double fk = m.frac_d[(long long)k * 3 + d];
#pragma unroll
    for (int i = 0; i < 3; ++i) m.wphi[(long long)k * 9 + d * 3 + i] = phi_d(((double)(i - 1) + 0.5) - fk);
}

// Row k of A~: one warp per marker, one lane per neighbour cell of its owner
// cell (the 5^d cells whose markers can overlap its support), visited in
// (z, y, x) order and bin order within a cell; a warp scan of the per-cell
// counts places every entry where a serial walk would, so the rows are the
// same whatever the warp size.  A~_kl = prod_d sum_i phi_k,d(i) phi_l,d(i)
// over the cells of both supports, from the tabulated weights: cell
// ck - 1 + i of marker k is cell j = ck - cl + i of marker l, and the terms
// with j outside [0, 2] are zero (|r| >= 3/2), so skipping them leaves every
// sum as it was with phi evaluated per pair.
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
        for (int i = 0; i < 3; ++i) wk[d][i] = m.wphi[(long long)k * 9 + d * 3 + i];
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
                const int off = ck[d] - m.cell[(long long)l * 3 + d];
                const double *wl = m.wphi + (long long)l * 9 + d * 3;
                double sum = 0.0;
                for (int i = 0; i < 3; ++i) {
                    const int j = off + i;
                    if (j >= 0 && j <= 2) sum += wk[d][i] * wl[j];
                }
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
    for (int o = 16; o > 0; o >>= 1) v = dmax_nonneg(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) s_red[w] = v;
    __syncthreads();
    double r = lane < NTH / 32 ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = dmax_nonneg(r, __shfl_xor_sync(0xffffffffu, r, o));
    return r;
}

template <int NTH>
__device__ __forceinline__ void spmv(int ns, const QuadBuffers &q, const double *x, double *y,
                                     int *err) {
    for (int k = threadIdx.x; k < ns; k += NTH) {
        const int c = q.cnt[k];
        double s = 0.0;
        for (int i = 0; i < c; ++i) {
            const int l = q.col[(long long)i * q.cap + k];
            if (in_bounds(l, ns, err)) s += q.val[(long long)i * q.cap + k] * x[l];
        }
        y[k] = s;
    }
}

// Jacobi-PCG on A~ x = rhs (all ones when rhs is null) by one CTA of NTH
// threads, from x (warm) or from zero; restarts from the true residual.
// Returns whether max|rhs - A~ x| <= tol; *iters and *resid report the run.
template <int NTH>
__device__ bool pcg_solve(int ns, const QuadBuffers &q, double *x, const double *__restrict__ rhs,
                          double tol, int maxit, int warm, double *s_red, int *iters,
                          double *resid, int *err) {
    double *r = q.r, *z = q.z, *p = q.p, *qv = q.q;
    if (!warm)
        for (int k = threadIdx.x; k < ns; k += NTH) x[k] = 0.0;
    __syncthreads();
    int it = 0;
    bool converged = false;
    double rmax = 0.0;
    for (int restart = 0; restart < 50 && it < maxit && !converged; ++restart) {
        spmv<NTH>(ns, q, x, qv, err);
        __syncthreads();
        double lm = 0.0;
        for (int k = threadIdx.x; k < ns; k += NTH) {
            r[k] = (rhs ? rhs[k] : 1.0) - qv[k];
            lm = dmax_nonneg(lm, fabs(r[k]));
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
            spmv<NTH>(ns, q, p, qv, err);
            __syncthreads();
            double lpq = 0.0;
            for (int k = threadIdx.x; k < ns; k += NTH) lpq += p[k] * qv[k];
            const double alpha = rz / block_sum<NTH>(lpq, s_red);
            double lr = 0.0;
            for (int k = threadIdx.x; k < ns; k += NTH) {
                x[k] += alpha * p[k];
                r[k] -= alpha * qv[k];
                lr = dmax_nonneg(lr, fabs(r[k]));
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
        spmv<NTH>(ns, q, x, qv, err);
        __syncthreads();
        double lm = 0.0;
        for (int k = threadIdx.x; k < ns; k += NTH) lm = dmax_nonneg(lm, fabs((rhs ? rhs[k] : 1.0) - qv[k]));
        rmax = block_max<NTH>(lm, s_red);
        converged = rmax <= tol;
    }
    *iters = it;
    *resid = rmax;
    return converged;
}

template <int NTH>
__global__ void __launch_bounds__(NTH)
pcg_kernel(int ns, const QuadBuffers q, double *x, const double *__restrict__ rhs, double tol,
           int maxit, int warm, int *err) {
    __shared__ double s_red[32];
    int it = 0;
    double rmax = 0.0;
    const bool converged =
        pcg_solve<NTH>(ns, q, x, rhs, tol, maxit, warm, s_red, &it, &rmax, err);
    if (threadIdx.x == 0) {
        *q.iters = it;
        *q.resid = rmax;
        if (!converged) record_error(err, ERR_NOCONV);
    }
}

// Small systems: A~ is copied dense, in FP32, into shared memory from the
// ELL rows.  FP64 runs at a small fraction of the FP32 rate on this GPU, so
// the O(ns^3) work is done in FP32: a blocked right-looking Cholesky
// A~ = L L^T over 32-column panels (one warp factors the panel's diagonal
// block without block barriers, one thread per row solves the rows below
// it, 4 x 4 register tiles update the trailing matrix: three barriers per
// panel), then the inverses of the 32 x 32 diagonal blocks of L, one warp
// each.  The FP64 solution comes from iterative refinement,
// x += L^-T L^-1 (rhs - A~ x), with the residual taken in FP64 from the
// ELL rows (only their nonzeros) and the two triangular solves blocked by
// the same panels (each diagonal block applied through its inverse); it
// contracts by about cond(A~) times the FP32 rounding per pass and stops
// at the FP64 residual's rounding floor: when the residual is within
// CHOL_FLOOR of the right-hand side's size, stops falling, or reaches zero
// (the first test saves the pass that would only confirm the floor).  Fixed
// order throughout, so the result is bitwise reproducible.
// If the refinement stops above tol or a pivot is not positive (a system
// too ill-conditioned for the FP32 factor), the same CTA runs the FP64
// Jacobi-PCG instead; ERR_NOCONV only if that fails too.
constexpr int CHOL_T = 512;
constexpr int CHOL_W = CHOL_T / 32;
#ifndef IBM_CHOL_MAX
#define IBM_CHOL_MAX 160
#endif
constexpr int CHOL_MAX = IBM_CHOL_MAX;
constexpr int CHOL_PB = 32;                                  // panel width
static_assert((CHOL_MAX + CHOL_PB - 1) / CHOL_PB <= CHOL_W, "one warp per diagonal block");
constexpr int CHOL_REFINE_MAX = 40;
constexpr double CHOL_FLOOR = 4.0 * 2.220446049250313e-16;   // 4 ulp of 1

// the first CHOL_EC entries of every row of A~ are kept in shared memory for
// the residuals of the refinement (rows hold ~10-60 entries; the rest are
// read from the ELL arrays in global memory)
constexpr int CHOL_EC = 32;

// x [ns] and the cached row values [CHOL_EC][ns] in FP64, then the FP32
// factors [ns][ns | 1], 1/L_jj, r and t, then the cached columns [CHOL_EC][ns]
// and the row lengths [ns]
size_t chol_smem(int ns) {
    return sizeof(double) * (size_t)ns * (1 + CHOL_EC) +
           sizeof(float) * ((size_t)ns * (ns | 1) + 3 * (size_t)ns) +
           sizeof(int) * (size_t)ns * (CHOL_EC + 1);
}

// Cholesky of the diagonal block [c0, c0 + w) in place, by one warp: lane r
// holds row c0 + r of the block in registers; 1 / L_kk into dinv, *bad set
// on a pivot that is not positive.  The row shifts left by one column per
// step (a[l] holds column k + l at step k), so the pivot column is always
// a[0] and every step runs the same compact loop body.  Step k hands the
// pivot column L_{k+l,k} to the lanes through col (32 floats, 16-byte
// aligned, this warp's alone): each lane stores its entry at l = lane - k
// and reads the column back as eight 16-byte broadcast loads, where 31
// shuffles (one per entry) set the step's latency.  Same operations in the
// same order as a shuffle form.
__device__ __forceinline__ void chol_diag_block(float *__restrict__ F, int ld, int c0, int w,
                                                float *__restrict__ dinv, int lane, int *bad,
                                                float *__restrict__ col) {
    float a[CHOL_PB];
#pragma unroll
    for (int l = 0; l < CHOL_PB; ++l)
        a[l] = (lane < w && l <= lane) ? F[(size_t)(c0 + lane) * ld + c0 + l] : 0.0f;
#pragma unroll 1
    for (int k = 0; k < w; ++k) {
        const float d = __shfl_sync(0xffffffffu, a[0], k);
        // pivots from the hardware reciprocal square root (a few ulp; the
        // factor only has to make the FP64 refinement contract): 18.7 k ->
        // 13.5 k cycles per 32-column block against IEEE sqrt and division
        const bool good = d > 0.0f;
        const float inv = good ? rsqrtf(d) : 1.0f;
        const float sd = good ? d * inv : 1.0f;
        float lk = a[0];   // zero on the lanes above the diagonal
        if (lane == k) {
            lk = sd;
            dinv[c0 + k] = inv;
            if (!good) *bad = 1;
        } else if (lane > k) {
            lk = a[0] * inv;
        }
        if (lane >= k && lane < w) F[(size_t)(c0 + lane) * ld + c0 + k] = lk;
        // col[l] = L_{k+l,k}; the entries past 31 - k are stale and unused
        if (lane >= k) col[lane - k] = lk;
        __syncwarp();
        float c[CHOL_PB];
#pragma unroll
        for (int v = 0; v < CHOL_PB / 4; ++v) {
            const float4 q = reinterpret_cast<const float4 *>(col)[v];
            c[4 * v] = q.x;
            c[4 * v + 1] = q.y;
            c[4 * v + 2] = q.z;
            c[4 * v + 3] = q.w;
        }
        __syncwarp();   // every lane has read col before the next step writes it
#pragma unroll
        for (int l = 1; l < CHOL_PB; ++l)
            if (lane >= k + l) a[l] -= lk * c[l];
#pragma unroll
        for (int l = 0; l < CHOL_PB - 1; ++l) a[l] = a[l + 1];
        a[CHOL_PB - 1] = 0.0f;
    }
}

// rows i >= c0 + w of panel [c0, c0 + w): L_i = A_i L_D^-T, one thread per row
__device__ __forceinline__ void chol_panel_rows(float *__restrict__ F, int ld, int c0, int w,
                                                int ns, const float *__restrict__ dinv, int tid) {
    for (int i = c0 + w + tid; i < ns; i += CHOL_T) {
        float *row = F + (size_t)i * ld + c0;
        float v[CHOL_PB];
#pragma unroll
        for (int k = 0; k < CHOL_PB; ++k) v[k] = k < w ? row[k] : 0.0f;
#pragma unroll
        for (int k = 0; k < CHOL_PB; ++k) {
            if (k < w) {
                const float *lk = F + (size_t)(c0 + k) * ld + c0;
                float acc = v[k];
#pragma unroll
                for (int l = 0; l < k; ++l) acc -= v[l] * lk[l];
                v[k] = acc * dinv[c0 + k];
            }
        }
#pragma unroll
        for (int k = 0; k < CHOL_PB; ++k)
            if (k < w) row[k] = v[k];
    }
}

// trailing update A_ij -= sum_k L_ik L_jk over the panel's columns, for
// c1 <= j <= i < ns, in 2 x 2 tiles (tile pairs tj <= ti, one per thread;
// 4 x 4 tiles kept fewer warps busy: 2.6 us more per moving-cylinder step)
__device__ __forceinline__ void chol_trailing(float *__restrict__ F, int ld, int c0, int w, int ns,
                                              int tid) {
    const int c1 = c0 + w, m = ns - c1, nt = (m + 1) / 2, npairs = nt * (nt + 1) / 2;
    for (int p = tid; p < npairs; p += CHOL_T) {
        int ti = (int)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= p) ++ti;
        while (ti * (ti + 1) / 2 > p) --ti;
        const int tj = p - ti * (ti + 1) / 2;
        const int i0 = c1 + 2 * ti, j0 = c1 + 2 * tj;
        float acc[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) acc[r][q] = 0.0f;
        for (int k = 0; k < w; ++k) {
            float a[2], b[2];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                a[r] = i0 + r < ns ? F[(size_t)(i0 + r) * ld + c0 + k] : 0.0f;
                b[r] = j0 + r < ns ? F[(size_t)(j0 + r) * ld + c0 + k] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int q = 0; q < 2; ++q) acc[r][q] += a[r] * b[q];
        }
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = i0 + r, j = j0 + q;
                if (i < ns && j <= i) F[(size_t)i * ld + j] -= acc[r][q];
            }
    }
}

// inverse of the diagonal block [b0, b0 + wb) of L by one warp (lane =
// column c): X_rc for r > c goes to F[c][r], above the diagonal; X_cc is
// dinv[c] already
__device__ __forceinline__ void chol_diag_inverse(float *__restrict__ F, int ld, int b0, int wb,
                                                  const float *__restrict__ dinv, int lane) {
    float xc[CHOL_PB];
#pragma unroll
    for (int r = 0; r < CHOL_PB; ++r) {
        float acc = r == lane ? 1.0f : 0.0f;
        if (r < wb) {
            const float *lr = F + (size_t)(b0 + r) * ld + b0;
#pragma unroll
            for (int l = 0; l < r; ++l) acc -= lr[l] * xc[l];
            acc *= dinv[b0 + r];
        }
        xc[r] = acc;
    }
    if (lane < wb) {
        float *out = F + (size_t)(b0 + lane) * ld + b0;
#pragma unroll
        for (int r = 0; r < CHOL_PB; ++r)
            if (r > lane && r < wb) out[r] = xc[r];
    }
}

// one CTA per launch: the register file is the CTA's alone, so the
// registers a thread may take are bounded for one resident block (the
// diagonal-block factor keeps a 32-float row per lane)
__global__ void __launch_bounds__(CHOL_T, 1)
chol_kernel(int ns, const QuadBuffers q, double *x, const double *__restrict__ rhs, double tol,
            int maxit, int warm, int *err) {
    // rows have an odd stride, so a warp walking a column (consecutive rows)
    // or threads walking their own rows hit distinct banks
    const int ld = ns | 1;
    extern __shared__ __align__(16) double sD[];
    double *sx = sD;                                 // [ns] solution
    double *ev = sx + ns;                            // [CHOL_EC][ns] cached row values
    float *F = reinterpret_cast<float *>(ev + (size_t)CHOL_EC * ns);
                                                     // [ns][ld]: L on and below the diagonal,
                                                     // the inverses X_II of its 32 x 32
                                                     // diagonal blocks transposed above it
    float *dinv = F + (size_t)ns * ld;               // [ns] 1 / L_jj, the diagonal of X_II
    float *r32 = dinv + ns;                          // [ns] residual in FP32
    float *st = r32 + ns;                            // [ns] the triangular solves' vector
    int *ec = reinterpret_cast<int *>(st + ns);      // [CHOL_EC][ns] cached row columns
    int *ecnt = ec + (size_t)CHOL_EC * ns;           // [ns] row lengths
    __shared__ double s_red[CHOL_T / 32];
    __shared__ int s_bad;
    __shared__ __align__(16) float s_col[CHOL_PB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < ns * ld; i += CHOL_T) F[i] = 0.0f;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    // lower triangle of A~ (the upper triangle stays zero); the rows' first
    // CHOL_EC entries and their lengths kept for the residuals
    for (int k = tid; k < ns; k += CHOL_T) {
        const int c = q.cnt[k];
        ecnt[k] = c;
        for (int i = 0; i < c; ++i) {
            const int l = q.col[(long long)i * q.cap + k];
            const double v = q.val[(long long)i * q.cap + k];
            if (i < CHOL_EC) {
                ec[(size_t)i * ns + k] = l;
                ev[(size_t)i * ns + k] = v;
            }
            if (in_bounds(l, ns, err) && l <= k) F[(size_t)k * ld + l] = (float)v;
        }
        sx[k] = warm ? x[k] : 0.0;
    }
    // the right-hand side's size, the scale of the residual's floor
    double rscale = 1.0;
    if (rhs) {
        double lr = 0.0;
        for (int k = tid; k < ns; k += CHOL_T) lr = dmax_nonneg(lr, fabs(rhs[k]));
        rscale = block_max<CHOL_T>(lr, s_red);   // synchronizes
    }
    __syncthreads();
    // blocked Cholesky over 32-column panels, then the diagonal blocks' inverses
    for (int c0 = 0; c0 < ns; c0 += CHOL_PB) {
        const int w = min(CHOL_PB, ns - c0);
        if (warp == 0) chol_diag_block(F, ld, c0, w, dinv, lane, &s_bad, s_col);
        __syncthreads();
        if (c0 + w < ns) {
            chol_panel_rows(F, ld, c0, w, ns, dinv, tid);
            __syncthreads();
            chol_trailing(F, ld, c0, w, ns, tid);
            __syncthreads();
        }
    }
    if (warp * CHOL_PB < ns)
        chol_diag_inverse(F, ld, warp * CHOL_PB, min(CHOL_PB, ns - warp * CHOL_PB), dinv, lane);
    __syncthreads();
    // refinement: r = rhs - A~ x in FP64 from the ELL rows (one thread per
    // row), x += L^-T L^-1 r in FP32
    double rmax = 0.0, rprev = 0.0;
    int it = 0;
    for (;; ++it) {
        double lm = 0.0;
        for (int k = tid; k < ns; k += CHOL_T) {
            const int c = ecnt[k];
            const int cc = min(c, CHOL_EC);
            double sum = 0.0;
            // the cached entries in batches of four (loads first, then the
            // terms in row order), the rest from the ELL arrays
            for (int i0 = 0; i0 < cc; i0 += 4) {
                int l[4];
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const bool in = i0 + u < cc;
                    l[u] = in ? ec[(size_t)(i0 + u) * ns + k] : 0;
                    v[u] = in ? ev[(size_t)(i0 + u) * ns + k] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (i0 + u < cc && in_bounds(l[u], ns, err)) sum += v[u] * sx[l[u]];
            }
            for (int i = CHOL_EC; i < c; ++i) {
                const int l = q.col[(long long)i * q.cap + k];
                if (in_bounds(l, ns, err)) sum += q.val[(long long)i * q.cap + k] * sx[l];
            }
            const double r = (rhs ? rhs[k] : 1.0) - sum;
            r32[k] = (float)r;
            lm = dmax_nonneg(lm, fabs(r));
        }
        rmax = block_max<CHOL_T>(lm, s_red);   // synchronizes
        if (!(rmax > 0.0) || rmax <= CHOL_FLOOR * rscale || (it > 0 && !(rmax < 0.5 * rprev)) ||
            it == CHOL_REFINE_MAX)
            break;
        rprev = rmax;
        // t = L^-1 r: per panel, t_I = X_II t_I (warp 0), then the rows
        // below take -L_iI t_I
        for (int i = tid; i < ns; i += CHOL_T) st[i] = r32[i];
        __syncthreads();
        for (int b0 = 0; b0 < ns; b0 += CHOL_PB) {
            const int b1 = min(b0 + CHOL_PB, ns);
            // (loops of the panel width with predicated terms: the loads of
            // every term issue together; same terms in the same order as
            // loops that stop at the ragged end)
            if (warp == 0) {
                const int i = b0 + lane;
                float y = 0.0f;
                if (i < b1) {
                    y = dinv[i] * st[i];
#pragma unroll
                    for (int j = 0; j < CHOL_PB - 1; ++j) {
                        const int cq = b0 + j;
                        if (cq < i) y += F[(size_t)cq * ld + i] * st[cq];
                    }
                }
                __syncwarp();
                if (i < b1) st[i] = y;
            }
            __syncthreads();
            for (int i = b1 + tid; i < ns; i += CHOL_T) {
                const float *row = F + (size_t)i * ld;
                float a0 = st[i], a1 = 0.0f;
#pragma unroll
                for (int j = 0; j < CHOL_PB / 2; ++j) {
                    const int cq = b0 + 2 * j;
                    if (cq + 2 <= b1) {
                        a0 -= row[cq] * st[cq];
                        a1 -= row[cq + 1] * st[cq + 1];
                    } else if (cq < b1) {
                        a0 -= row[cq] * st[cq];
                    }
                }
                st[i] = a0 + a1;
            }
            __syncthreads();
        }
        // z = L^-T t: per panel from the last, z_I = X_II^T t_I (warp 0),
        // then the rows above take -L_Ic^T z_I
        for (int b0 = ((ns - 1) / CHOL_PB) * CHOL_PB; b0 >= 0; b0 -= CHOL_PB) {
            const int b1 = min(b0 + CHOL_PB, ns);
            if (warp == 0) {
                const int c = b0 + lane;
                float z = 0.0f;
                if (c < b1) {
                    const float *row = F + (size_t)c * ld;
                    z = dinv[c] * st[c];
#pragma unroll
                    for (int j = 1; j < CHOL_PB; ++j) {
                        const int i = b0 + j;
                        if (i > c && i < b1) z += row[i] * st[i];
                    }
                }
                __syncwarp();
                if (c < b1) st[c] = z;
            }
            __syncthreads();
            for (int c = tid; c < b0; c += CHOL_T) {
                float a0 = st[c], a1 = 0.0f;
#pragma unroll
                for (int j = 0; j < CHOL_PB / 2; ++j) {
                    const int i = b0 + 2 * j;
                    if (i + 2 <= b1) {
                        a0 -= F[(size_t)i * ld + c] * st[i];
                        a1 -= F[(size_t)(i + 1) * ld + c] * st[i + 1];
                    } else if (i < b1) {
                        a0 -= F[(size_t)i * ld + c] * st[i];
                    }
                }
                st[c] = a0 + a1;
            }
            __syncthreads();
        }
        for (int c = tid; c < ns; c += CHOL_T) sx[c] += (double)st[c];
        __syncthreads();
    }
    for (int k = tid; k < ns; k += CHOL_T) x[k] = sx[k];
    bool ok = !s_bad && rmax <= tol;
    if (!ok) {
        // too ill-conditioned for the FP32 factor (e.g. two markers in one
        // cell, placed without dedup): the FP64 Jacobi-PCG takes over, from
        // the refined x when it is finite
        __shared__ double s_red32[32];
        const bool warm_x = !s_bad && rmax < 1.0;
        ok = pcg_solve<CHOL_T>(ns, q, x, rhs, tol, maxit, warm_x, s_red32, &it, &rmax, err);
    }
    if (tid == 0) {
        *q.iters = it;
        *q.resid = rmax;
        if (!ok) record_error(err, ERR_NOCONV);
    }
}

}  // namespace

int quad_row_width(int dim) { return dim == 3 ? 125 * 4 : 25 * 4; }

// A~ x = rhs (rhs == nullptr: all ones): dense Cholesky with refinement up
// to CHOL_MAX markers, Jacobi-PCG above (either warm-started if asked)
static cudaError_t launch_quadrature_solve_w(int ns, const QuadBuffers &qb, const double *rhs,
                                            double *x, double tol, int maxit, int warm, int *err,
                                            cudaStream_t s) {
    if (ns <= 0) return cudaSuccess;
    if (ns <= CHOL_MAX) {
        cudaError_t e = func_smem_attr((const void *)chol_kernel, chol_smem(CHOL_MAX));
        if (e != cudaSuccess) return e;
        chol_kernel<<<1, CHOL_T, chol_smem(ns), s>>>(ns, qb, x, rhs, tol, maxit, warm, err);
    } else if (ns <= 2048) {
        pcg_kernel<256><<<1, 256, 0, s>>>(ns, qb, x, rhs, tol, maxit, warm, err);
    } else {
        pcg_kernel<1024><<<1, 1024, 0, s>>>(ns, qb, x, rhs, tol, maxit, warm, err);
    }
    return cudaGetLastError();
}

cudaError_t launch_quadrature(const GridParams &g, const MarkerBuffers &m, const QuadBuffers &qb,
                              double tol, int maxit, int warm, cudaStream_t s, int have_weights) {
    if (m.ns <= 0) return cudaSuccess;
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    if (!have_weights) support_weights_kernel<<<(m.ns * 3 + 127) / 128, 128, 0, s>>>(m, g.dim);
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
