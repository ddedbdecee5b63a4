// Lagrangian side of the IBM step (Sec. 2.2): marker motion, marker-to-cell
// bins, interpolation + direct forcing, and the cell-centric spreading that
// applies the sources.
//
//  - Bins: markers sorted by key = (tile id, cell in tile) and input index
//    with a stable LSD radix sort in one CTA (warp __match_any_sync ranks and
//    a block-wide scan of the digit histograms), then tile_off[] by binary
//    search, then the lists of occupied tiles and of "band" tiles (tiles
//    within one tile of an occupied one).  Integer work only: bit-exact.
//  - Interpolation (Eq. interp): one CTA per occupied tile stages the tile
//    plus a one-cell halo of (rho, rho u, rho e) in shared memory; one warp
//    per marker, one lane per support cell, warp butterfly sum.
//  - Forcing (Eqs. forceMomentum, corr3.8, a = 1/dt): G = dt F =
//    rho_L U_b - I[rho u], H = dt Q = rho_L c_v T_w - I[rho e].
//  - Spreading (Eq. force2) as a gather: each cell of a band tile visits its
//    3^d neighbour cells in a fixed order and the markers binned there in
//    sorted order, so the sum order is fixed and no float atomics are used.
//    The forced update (App. B, Eqs. u_centralF2 and e_centralF2) follows in
//    the same thread.
#include "internal.h"

namespace ibmk {
namespace {

constexpr int SORT_T = 1024;
constexpr int SORT_W = SORT_T / 32;
constexpr int RADIX = 256;
constexpr int HSTRIDE = SORT_W + 1;

// exclusive scan of one int per thread over a 1024-thread block
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int &total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
        int xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += y;
        }
        s_warp[lane] = xi - x;          // exclusive prefix of warp totals
        if (lane == 31) s_warp[32] = xi;
    }
    __syncthreads();
    const int excl = s_warp[w] + incl - v;
    total = s_warp[32];
    __syncthreads();
    return excl;
}

// ---------------------------------------------------------------------------
// bins
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(SORT_T)
bin_sort_kernel(const GridParams g, int ns, const double *__restrict__ X, unsigned *keys0,
                int *vals0, unsigned *keys1, int *vals1, int passes, int *err) {
    __shared__ int hist[RADIX * HSTRIDE];
    __shared__ int s_warp[33];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int bad = 0;
    for (int k = tid; k < ns; k += SORT_T) {
        int c[3] = {0, 0, 0};
        for (int d = 0; d < g.dim; ++d) {
            int cd = owner_cell(X[(long long)k * g.dim + d], g.lo[d], g.h);
            if (!(cd >= 2 && cd <= g.n[d] - 3)) {
                bad = 1;
                cd = cd < 0 ? 0 : (cd >= g.n[d] ? g.n[d] - 1 : cd);
            }
            c[d] = cd;
        }
        keys0[k] = cell_key(g, c[0], c[1], c[2]);
        vals0[k] = k;
    }
    if (bad) record_error(err, ERR_MARKER_RANGE);
    __syncthreads();

    const int seg = (ns + SORT_W - 1) / SORT_W;
    const int s0 = w * seg, s1 = min(ns, s0 + seg);
    unsigned *kin = keys0, *kout = keys1;
    int *vin = vals0, *vout = vals1;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        for (int i = tid; i < RADIX * HSTRIDE; i += SORT_T) hist[i] = 0;
        __syncthreads();
        // per-warp digit histogram of the warp's contiguous segment
        for (int base = s0; base < s1; base += 32) {
            const int i = base + lane;
            const bool valid = i < s1;
            const unsigned dig = valid ? (kin[i] >> shift) & (RADIX - 1) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, dig);
            if (valid && lane == __ffs(peers) - 1) hist[dig * HSTRIDE + w] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // exclusive scan in (digit, warp) order: 8 consecutive entries per thread
        int vals[8], sum = 0;
        const int dg = tid >> 2, wb = (tid & 3) * 8;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            vals[r] = hist[dg * HSTRIDE + wb + r];
            sum += vals[r];
        }
        int total;
        int run = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            hist[dg * HSTRIDE + wb + r] = run;
            run += vals[r];
        }
        __syncthreads();
        // stable scatter
        for (int base = s0; base < s1; base += 32) {
            const int i = base + lane;
            const bool valid = i < s1;
            const unsigned key = valid ? kin[i] : 0u;
            const int v = valid ? vin[i] : 0;
            const unsigned dig = valid ? (key >> shift) & (RADIX - 1) : 0xffffffffu;
            const unsigned peers = __match_any_sync(0xffffffffu, dig);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            if (valid) {
                const int pos = hist[dig * HSTRIDE + w] + rank;
                kout[pos] = key;
                vout[pos] = v;
            }
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) hist[dig * HSTRIDE + w] += __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        unsigned *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
}

// tile_off[t] = number of sorted keys below t * cells_per_tile
__global__ void tile_offsets_kernel(const GridParams g, int ns, const unsigned *__restrict__ keys,
                                    int *__restrict__ tile_off) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > g.n_tiles) return;
    const unsigned target = (unsigned)t * (unsigned)g.cells_per_tile;
    int lo = 0, hi = ns;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    tile_off[t] = lo;
}

__global__ void tile_flags_kernel(const GridParams g, const int *__restrict__ tile_off,
                                  int *__restrict__ occ, int *__restrict__ band) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_tiles) return;
    const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
              tz = t / (g.ntile[0] * g.ntile[1]);
    occ[t] = tile_off[t + 1] > tile_off[t];
    int b = 0;
    const int zr = g.dim == 3 ? 1 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int x = tx + ox, y = ty + oy, z = tz + oz;
                if (x < 0 || y < 0 || z < 0 || x >= g.ntile[0] || y >= g.ntile[1] || z >= g.ntile[2])
                    continue;
                const int u = x + g.ntile[0] * (y + g.ntile[1] * z);
                b |= tile_off[u + 1] > tile_off[u];
            }
    band[t] = b;
}

// ordered compaction of the two flag arrays (single CTA)
__global__ void __launch_bounds__(SORT_T)
tile_lists_kernel(int n_tiles, const int *__restrict__ occ, const int *__restrict__ band,
                  int *__restrict__ occ_list, int *__restrict__ band_list, int *__restrict__ counts) {
    __shared__ int s_warp[33];
    const int chunk = (n_tiles + SORT_T - 1) / SORT_T;
    const int t0 = threadIdx.x * chunk, t1 = min(n_tiles, t0 + chunk);
    int co = 0, cb = 0;
    for (int t = t0; t < t1; ++t) {
        co += occ[t];
        cb += band[t];
    }
    int to, tb;
    int eo = block_exclusive_scan(co, s_warp, to);
    int eb = block_exclusive_scan(cb, s_warp, tb);
    for (int t = t0; t < t1; ++t) {
        if (occ[t]) occ_list[eo++] = t;
        if (band[t]) band_list[eb++] = t;
    }
    if (threadIdx.x == 0) {
        counts[0] = to;
        counts[1] = tb;
    }
}

// ---------------------------------------------------------------------------
// motion (Sec. 5): positions and body velocity at t^{n+1} = t^n + dt
// ---------------------------------------------------------------------------

__global__ void motion_kernel(const GridParams g, int ns, const double *__restrict__ X0,
                              const double *__restrict__ Ub0, double *__restrict__ X,
                              double *__restrict__ Ub, double amp, double freq, int axis,
                              const double *__restrict__ t, const double *__restrict__ dt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    const double pi = 3.14159265358979323846;
    const double tn = *t + *dt;
    const double sv = amp * sin(2.0 * pi * freq * tn);
    const double vv = amp * 2.0 * pi * freq * cos(2.0 * pi * freq * tn);
    for (int d = 0; d < g.dim; ++d) {
        const long long q = (long long)k * g.dim + d;
        X[q] = X0[q] + (d == axis ? sv : 0.0);
        Ub[q] = Ub0[q] + (d == axis ? vv : 0.0);
    }
}

// ---------------------------------------------------------------------------
// interpolation + forcing
// ---------------------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// support-cell weight Phi_k(j) for lane l of 3^DIM (offsets in z,y,x order)
template <int DIM>
__device__ __forceinline__ double lane_weight(const GridParams &g, const double *Xk, const int *ck,
                                              int l, int *cell) {
    const int o[3] = {l % 3 - 1, (l / 3) % 3 - 1, DIM == 3 ? l / 9 - 1 : 0};
    double w = 1.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        cell[d] = ck[d] + o[d];
        w *= phi_d((cell_center(g, d, cell[d]) - Xk[d]) * g.inv_h);
    }
    if (DIM == 2) cell[2] = 0;
    return w;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256)
interp_force_kernel(const GridParams g, const T *__restrict__ U, const MarkerBuffers m,
                    const int *__restrict__ perm) {
    constexpr int NF = DIM + 2;   // rho, rho u.., rho e
    constexpr int NS = DIM == 3 ? 27 : 9;
    extern __shared__ __align__(16) double sS[];
    const int bx = g.tile[0] + 2, by = g.tile[1] + 2, bz = DIM == 3 ? g.tile[2] + 2 : 1;
    const int bn = bx * by * bz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const long long N = g.N;
    const int n_occ = m.counts[0];
    for (int it = blockIdx.x; it < n_occ; it += gridDim.x) {
        const int t = m.occ_list[it];
        const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
                  tz = t / (g.ntile[0] * g.ntile[1]);
        const int ox = tx * g.tile[0] - 1, oy = ty * g.tile[1] - 1,
                  oz = DIM == 3 ? tz * g.tile[2] - 1 : 0;
        for (int q = threadIdx.x; q < bn; q += blockDim.x) {
            const int lx = q % bx, ly = (q / bx) % by, lz = q / (bx * by);
            const int gx = ox + lx, gy = oy + ly, gz = oz + lz;
            const bool in = gx >= 0 && gy >= 0 && gz >= 0 && gx < g.n[0] && gy < g.n[1] &&
                            (DIM == 2 || gz < g.n[2]);
            double v[NF];
            if (in) {
                const long long j = gx + (long long)g.n[0] * (gy + (long long)g.n[1] * gz);
                const double rho = (double)U[j];
                double ke = 0.0;
#pragma unroll
                for (int d = 0; d < DIM; ++d) {
                    const double md = (double)U[(1 + d) * N + j];
                    v[1 + d] = md;
                    ke += md * md;
                }
                v[0] = rho;
                v[NF - 1] = (double)U[(DIM + 1) * N + j] - 0.5 * ke / rho;
            } else {
#pragma unroll
                for (int f = 0; f < NF; ++f) v[f] = 0.0;
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) sS[f * bn + q] = v[f];
        }
        __syncthreads();
        const int p0 = m.tile_off[t], p1 = m.tile_off[t + 1];
        for (int p = p0 + warp; p < p1; p += nwarps) {
            const int k = perm[p];
            double Xk[3] = {0, 0, 0};
            int ck[3] = {0, 0, 0};
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                Xk[d] = m.X[(long long)k * DIM + d];
                ck[d] = owner_cell(Xk[d], g.lo[d], g.h);
            }
            double acc[NF];
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = 0.0;
            if (lane < NS) {
                int cell[3];
                const double w = lane_weight<DIM>(g, Xk, ck, lane, cell);
                const int li = (cell[0] - ox) + bx * ((cell[1] - oy) + by * (cell[2] - oz));
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] = w * sS[f * bn + li];
            }
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = warp_sum(acc[f]);
            if (lane == 0) {
                const double rk = acc[0];
                m.rhoL[k] = rk;
#pragma unroll
                for (int d = 0; d < DIM; ++d)
                    m.G[(long long)k * DIM + d] = rk * m.Ub[(long long)k * DIM + d] - acc[1 + d];
                m.H[k] = rk * g.cv * m.Tw[k] - acc[NF - 1];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// spreading as a cell-centric gather
// ---------------------------------------------------------------------------

// Visit, in a fixed order, every marker whose support contains cell c:
// neighbour owner cells (z, y, x offsets ascending), then sorted bin order.
template <int DIM, typename F>
__device__ __forceinline__ bool gather_markers(const GridParams &g, const MarkerBuffers &m,
                                               const unsigned *__restrict__ keys,
                                               const int *__restrict__ perm, const int c[3],
                                               F &&visit) {
    bool any = false;
    const int zr = DIM == 3 ? 1 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int x = c[0] + ox, y = c[1] + oy, z = c[2] + oz;
                if (x < 0 || y < 0 || x >= g.n[0] || y >= g.n[1]) continue;
                if (DIM == 3 && (z < 0 || z >= g.n[2])) continue;
                const unsigned key = cell_key(g, x, y, z);
                const int tc = (int)(key / (unsigned)g.cells_per_tile);
                int lo = m.tile_off[tc], hi = m.tile_off[tc + 1];
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (keys[mid] < key) lo = mid + 1;
                    else hi = mid;
                }
                const int end = m.tile_off[tc + 1];
                for (int p = lo; p < end && keys[p] == key; ++p) {
                    const int k = perm[p];
                    double w = 1.0;
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
                        w *= phi_d((cell_center(g, d, c[d]) - m.X[(long long)k * DIM + d]) * g.inv_h);
                    visit(k, w);
                    any = true;
                }
            }
    return any;
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256)
spread_apply_kernel(const GridParams g, T *__restrict__ U, const MarkerBuffers m,
                    const unsigned *__restrict__ keys, const int *__restrict__ perm) {
    const long long N = g.N;
    const int n_band = m.counts[1];
    const int cpt = g.cells_per_tile;
    for (int it = blockIdx.x; it < n_band; it += gridDim.x) {
        const int t = m.band_list[it];
        const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
                  tz = t / (g.ntile[0] * g.ntile[1]);
        for (int q = threadIdx.x; q < cpt; q += blockDim.x) {
            const int c[3] = {tx * g.tile[0] + q % g.tile[0],
                              ty * g.tile[1] + (q / g.tile[0]) % g.tile[1],
                              DIM == 3 ? tz * g.tile[2] + q / (g.tile[0] * g.tile[1]) : 0};
            if (c[0] >= g.n[0] || c[1] >= g.n[1] || (DIM == 3 && c[2] >= g.n[2])) continue;
            double f[DIM], qh = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) f[d] = 0.0;
            const bool band = gather_markers<DIM>(g, m, keys, perm, c, [&](int k, double w) {
                const double we = w * m.eps[k];
#pragma unroll
                for (int d = 0; d < DIM; ++d) f[d] += m.G[(long long)k * DIM + d] * we;
                qh += m.H[k] * we;
            });
            if (!band) continue;
            const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
            const double rho = (double)U[j];
            double ke0 = 0.0, ke1 = 0.0;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const double m0 = (double)U[(1 + d) * N + j];
                const double m1 = m0 + f[d];
                ke0 += m0 * m0;
                ke1 += m1 * m1;
                U[(1 + d) * N + j] = (T)m1;
            }
            const double E = (double)U[(DIM + 1) * N + j];
            const double En = g.energy_reading == 1 ? E + qh
                                                    : (E - 0.5 * ke0 / rho + qh) + 0.5 * ke1 / rho;
            U[(DIM + 1) * N + j] = (T)En;
        }
    }
}

// ---------------------------------------------------------------------------
// forces/heat sums (fixed-order reduction) and the time update
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256)
finish_kernel(int dim, int ns, const MarkerBuffers m, const double *__restrict__ dt) {
    __shared__ double s[4][256];
    double a[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < ns; k += 256) {
        const double e = m.eps[k];
        for (int d = 0; d < dim; ++d) a[d] += e * m.G[(long long)k * dim + d];
        a[3] += e * m.H[k];
    }
    for (int i = 0; i < 4; ++i) s[i][threadIdx.x] = a[i];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int i = 0; i < 4; ++i) s[i][threadIdx.x] += s[i][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) m.sums[i] = s[i][0];
        m.sums[4] = *dt;
        *m.t += *dt;
        *m.steps += 1;
    }
}

// ---------------------------------------------------------------------------
// operators for the diagnostic entry points
// ---------------------------------------------------------------------------

template <int DIM, typename T>
__global__ void interpolate_op_kernel(const GridParams g, const T *__restrict__ field, int nc,
                                      const MarkerBuffers m, double *__restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m.ns) return;
    double Xk[3] = {0, 0, 0};
    int ck[3] = {0, 0, 0};
    for (int d = 0; d < DIM; ++d) {
        Xk[d] = m.X[(long long)k * DIM + d];
        ck[d] = owner_cell(Xk[d], g.lo[d], g.h);
    }
    for (int c = 0; c < nc; ++c) out[(long long)k * nc + c] = 0.0;
    constexpr int NS = DIM == 3 ? 27 : 9;
    for (int l = 0; l < NS; ++l) {
        int cell[3];
        const double w = lane_weight<DIM>(g, Xk, ck, l, cell);
        const long long j = cell[0] + (long long)g.n[0] * (cell[1] + (long long)g.n[1] * cell[2]);
        for (int c = 0; c < nc; ++c) out[(long long)k * nc + c] += w * (double)field[c * g.N + j];
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256)
spread_op_kernel(const GridParams g, const double *__restrict__ R, int nc, const MarkerBuffers m,
                 const unsigned *__restrict__ keys, const int *__restrict__ perm,
                 T *__restrict__ out) {
    const int n_band = m.counts[1];
    const int cpt = g.cells_per_tile;
    for (int it = blockIdx.x; it < n_band; it += gridDim.x) {
        const int t = m.band_list[it];
        const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
                  tz = t / (g.ntile[0] * g.ntile[1]);
        for (int q = threadIdx.x; q < cpt; q += blockDim.x) {
            const int c[3] = {tx * g.tile[0] + q % g.tile[0],
                              ty * g.tile[1] + (q / g.tile[0]) % g.tile[1],
                              DIM == 3 ? tz * g.tile[2] + q / (g.tile[0] * g.tile[1]) : 0};
            if (c[0] >= g.n[0] || c[1] >= g.n[1] || (DIM == 3 && c[2] >= g.n[2])) continue;
            const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
            for (int cc = 0; cc < nc; ++cc) {
                double acc = 0.0;
                gather_markers<DIM>(g, m, keys, perm, c, [&](int k, double w) {
                    acc += R[(long long)k * nc + cc] * (w * m.eps[k]);
                });
                out[cc * g.N + j] = (T)acc;
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------

cudaError_t launch_motion(const GridParams &g, const MarkerBuffers &m, double amp, double freq,
                          int axis, const double *dt, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    motion_kernel<<<(m.ns + 127) / 128, 128, 0, s>>>(g, m.ns, m.X0, m.Ub0, m.X, m.Ub, amp, freq,
                                                      axis, m.t, dt);
    return cudaGetLastError();
}

static int radix_passes(const GridParams &g) {
    unsigned long long maxkey = (unsigned long long)g.n_tiles * g.cells_per_tile - 1ull;
    int bits = 0;
    while (bits < 32 && (maxkey >> bits) != 0ull) ++bits;
    int p = (bits + 7) / 8;
    return p < 1 ? 1 : p;
}

cudaError_t launch_bin(const GridParams &g, MarkerBuffers &m, cudaStream_t s) {
    const int passes = radix_passes(g);
    m.sorted = passes & 1;
    if (m.ns > 0) {
        bin_sort_kernel<<<1, SORT_T, 0, s>>>(g, m.ns, m.X, m.keys[0], m.perm[0], m.keys[1],
                                             m.perm[1], passes, m.err);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    tile_offsets_kernel<<<(g.n_tiles + 1 + 255) / 256, 256, 0, s>>>(g, m.ns, m.keys[m.sorted],
                                                                     m.tile_off);
    tile_flags_kernel<<<(g.n_tiles + 255) / 256, 256, 0, s>>>(g, m.tile_off, m.occ_flag,
                                                              m.band_flag);
    tile_lists_kernel<<<1, SORT_T, 0, s>>>(g.n_tiles, m.occ_flag, m.band_flag, m.occ_list,
                                           m.band_list, m.counts);
    return cudaGetLastError();
}

static size_t interp_smem(const GridParams &g) {
    size_t bn = (size_t)(g.tile[0] + 2) * (g.tile[1] + 2) * (g.dim == 3 ? g.tile[2] + 2 : 1);
    return bn * (g.dim + 2) * sizeof(double);
}

template <int DIM, typename T>
static cudaError_t interp_force_t(const GridParams &g, const void *U, const MarkerBuffers &m,
                                  int grid_ctas, cudaStream_t s) {
    const size_t smem = interp_smem(g);
    static size_t configured = 0;
    if (smem > 48 * 1024 && configured < smem) {
        cudaError_t e = cudaFuncSetAttribute(interp_force_kernel<DIM, T>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    interp_force_kernel<DIM, T><<<grid_ctas, 256, smem, s>>>(g, (const T *)U, m, m.perm[m.sorted]);
    return cudaGetLastError();
}

cudaError_t launch_interp_force(const GridParams &g, int fp_bytes, const void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    if (g.dim == 3)
        return fp_bytes == 4 ? interp_force_t<3, float>(g, U, m, grid_ctas, s)
                             : interp_force_t<3, double>(g, U, m, grid_ctas, s);
    return fp_bytes == 4 ? interp_force_t<2, float>(g, U, m, grid_ctas, s)
                         : interp_force_t<2, double>(g, U, m, grid_ctas, s);
}

cudaError_t launch_spread_apply(const GridParams &g, int fp_bytes, void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    if (g.dim == 3) {
        if (fp_bytes == 4)
            spread_apply_kernel<3, float><<<grid_ctas, 256, 0, s>>>(g, (float *)U, m, keys, perm);
        else
            spread_apply_kernel<3, double><<<grid_ctas, 256, 0, s>>>(g, (double *)U, m, keys, perm);
    } else {
        if (fp_bytes == 4)
            spread_apply_kernel<2, float><<<grid_ctas, 256, 0, s>>>(g, (float *)U, m, keys, perm);
        else
            spread_apply_kernel<2, double><<<grid_ctas, 256, 0, s>>>(g, (double *)U, m, keys, perm);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish(const GridParams &g, const MarkerBuffers &m, const double *dt,
                          cudaStream_t s) {
    finish_kernel<<<1, 256, 0, s>>>(g.dim, m.ns, m, dt);
    return cudaGetLastError();
}

cudaError_t launch_interpolate_op(const GridParams &g, int fp_bytes, const void *field, int nc,
                                  const MarkerBuffers &m, double *out, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    const int nb = (m.ns + 127) / 128;
    if (g.dim == 3) {
        if (fp_bytes == 4)
            interpolate_op_kernel<3, float><<<nb, 128, 0, s>>>(g, (const float *)field, nc, m, out);
        else
            interpolate_op_kernel<3, double><<<nb, 128, 0, s>>>(g, (const double *)field, nc, m, out);
    } else {
        if (fp_bytes == 4)
            interpolate_op_kernel<2, float><<<nb, 128, 0, s>>>(g, (const float *)field, nc, m, out);
        else
            interpolate_op_kernel<2, double><<<nb, 128, 0, s>>>(g, (const double *)field, nc, m, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_spread_op(const GridParams &g, int fp_bytes, const double *R, int nc,
                             const MarkerBuffers &m, void *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, (size_t)nc * g.N * fp_bytes, s);
    if (e != cudaSuccess || m.ns <= 0) return e;
    const unsigned *keys = m.keys[m.sorted];
    const int *perm = m.perm[m.sorted];
    const int nb = 4 * 152;
    if (g.dim == 3) {
        if (fp_bytes == 4)
            spread_op_kernel<3, float><<<nb, 256, 0, s>>>(g, R, nc, m, keys, perm, (float *)out);
        else
            spread_op_kernel<3, double><<<nb, 256, 0, s>>>(g, R, nc, m, keys, perm, (double *)out);
    } else {
        if (fp_bytes == 4)
            spread_op_kernel<2, float><<<nb, 256, 0, s>>>(g, R, nc, m, keys, perm, (float *)out);
        else
            spread_op_kernel<2, double><<<nb, 256, 0, s>>>(g, R, nc, m, keys, perm, (double *)out);
    }
    return cudaGetLastError();
}

}  // namespace ibmk
