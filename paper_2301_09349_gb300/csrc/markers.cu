// Lagrangian side of the IBM step (Sec. 2.2): marker motion, marker-to-cell
// bins, interpolation + direct forcing, and the cell-centric spreading that
// applies the sources.
//
//  - Bins: markers sorted by key = (tile id, cell in tile) and input index
//    with a stable LSD radix sort in one CTA (warp __match_any_sync ranks and
//    a block-wide scan of the digit histograms), then tile_off[] by binary
//    search; the forced cells scattered from the markers' supports, and the
//    lists of occupied tiles and of "band" tiles (tiles holding a forced
//    cell).  Integer work only: bit-exact.  Small moving bodies do all of
//    it in one launch (small_rebuild_kernel).
//  - Interpolation (Eq. interp): one warp per marker, one lane per support
//    cell read straight from the state, warp butterfly sum.
//  - Forcing (Eqs. forceMomentum, corr3.8, a = 1/dt): G = dt F =
//    rho_L U_b - I[rho u], H = dt Q = rho_L c_v T_w - I[rho e].
//  - Spreading (Eq. force2) as a gather: each cell of a band tile visits its
//    3^d neighbour cells in a fixed order and the markers binned there in
//    sorted order, so the sum order is fixed and no float atomics are used;
//    static markers keep that per-cell list of (marker, weight) entries as
//    their spreading operator and gather through it.  The forced update
//    (App. B, Eqs. u_centralF2 and e_centralF2) follows in the same thread.
#include <float.h>

#include <algorithm>

#include "internal.h"
#include "marker_ops.cuh"

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

// Owner cell floor(xi) and offset xi - cell of marker k, xi = (X - lo)/h with
// IEEE subtraction and division (they feed every weight evaluation); its
// sort key.  A marker closer than two cells to the grid's edge sets bad.
__device__ __forceinline__ unsigned owner_cell(const GridParams &g, const double *__restrict__ X,
                                               int k, int *__restrict__ cell_out,
                                               double *__restrict__ frac_d,
                                               float *__restrict__ frac_f, int &bad) {
    int c[3] = {0, 0, 0};
    for (int d = 0; d < 3; ++d) {
        double fr = 0.0;
        if (d < g.dim) {
            const double xi = __ddiv_rn(__dsub_rn(X[(long long)k * g.dim + d], g.lo[d]), g.h);
            int cd = (int)floor(xi);
            fr = xi - (double)cd;
            if (!(cd >= 2 && cd <= g.n[d] - 3)) {
                bad = 1;
                cd = cd < 0 ? 0 : (cd >= g.n[d] ? g.n[d] - 1 : cd);
                fr = 0.5;
            }
            c[d] = cd;
        }
        cell_out[(long long)k * 3 + d] = c[d];
        frac_d[(long long)k * 3 + d] = fr;
        frac_f[(long long)k * 3 + d] = (float)fr;
    }
    return cell_key(g, c[0], c[1], c[2]);
}

__global__ void __launch_bounds__(SORT_T)
bin_sort_kernel(const GridParams g, int ns, const double *__restrict__ X, unsigned *keys0,
                int *vals0, unsigned *keys1, int *vals1, int passes, int *err,
                int *__restrict__ cell_out, double *__restrict__ frac_d, float *__restrict__ frac_f) {
    __shared__ int hist[RADIX * HSTRIDE];
    __shared__ int s_warp[33];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int bad = 0;
    for (int k = tid; k < ns; k += SORT_T) {
        keys0[k] = owner_cell(g, X, k, cell_out, frac_d, frac_f, bad);
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

// occ[t] = tile t holds an owner cell; band[t] cleared for the scatter of
// the forced cells
__global__ void tile_flags_kernel(const GridParams g, const int *__restrict__ tile_off,
                                  int *__restrict__ occ, int *__restrict__ band) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.n_tiles) return;
    occ[t] = tile_off[t + 1] > tile_off[t];
    band[t] = 0;
}

// ordered compaction of the two flag arrays by one CTA of SORT_T threads
__device__ __forceinline__ void tile_lists(int n_tiles, const int *__restrict__ occ,
                                           const int *__restrict__ band, int *__restrict__ occ_list,
                                           int *__restrict__ band_list, int *__restrict__ counts,
                                           int *s_warp) {
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

__global__ void __launch_bounds__(SORT_T)
tile_lists_kernel(int n_tiles, const int *__restrict__ occ, const int *__restrict__ band,
                  int *__restrict__ occ_list, int *__restrict__ band_list, int *__restrict__ counts) {
    __shared__ int s_warp[33];
    tile_lists(n_tiles, occ, band, occ_list, band_list, counts, s_warp);
}

// ---------------------------------------------------------------------------
// motion (Sec. 5): positions and body velocity at t^{n+1} = t^n + dt
// ---------------------------------------------------------------------------

// body offset and velocity along the motion axis at t^{n+1} (rigid
// transverse or streamwise oscillation X = X0 + A sin(2 pi f t))
__device__ __forceinline__ void motion_offset(double amp, double freq,
                                              const double *__restrict__ t,
                                              const double *__restrict__ dt, double dt_fixed,
                                              double &sv, double &vv) {
    const double pi = 3.14159265358979323846;
    const double tn = *t + (dt_fixed > 0.0 ? dt_fixed : *dt);
    sv = amp * sin(2.0 * pi * freq * tn);
    vv = amp * 2.0 * pi * freq * cos(2.0 * pi * freq * tn);
}

__global__ void motion_kernel(const GridParams g, int ns, const double *__restrict__ X0,
                              const double *__restrict__ Ub0, double *__restrict__ X,
                              double *__restrict__ Ub, double amp, double freq, int axis,
                              const double *__restrict__ t, const double *__restrict__ dt,
                              double dt_fixed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ns) return;
    double sv, vv;
    motion_offset(amp, freq, t, dt, dt_fixed, sv, vv);
    for (int d = 0; d < g.dim; ++d) {
        const long long q = (long long)k * g.dim + d;
        X[q] = X0[q] + (d == axis ? sv : 0.0);
        Ub[q] = Ub0[q] + (d == axis ? vv : 0.0);
    }
}

// The per-step marker pipeline of a small moving body (ns <= SMALL_NS) in one
// CTA: the motion, owner cells and keys, a stable sort by key (rank of each
// key: the keys below it plus the equal keys before it, the order a stable
// radix sort gives), tile offsets and occupancy, the forced-cell scatter and
// the tile lists - the work of motion_kernel, bin_sort_kernel,
// tile_offsets_kernel, tile_flags_kernel, band_scatter_kernel and
// tile_lists_kernel, and the support weights of support_weights_kernel, with
// barriers in place of seven launches.  band_bits
// must hold exactly the previous marker set's forced cells on entry (it
// clears them first, from the previous owner cells, instead of a memset of
// the whole mask); the sorted order goes to keys[0] / perm[0].
// Support cell sc (0 .. 3^d - 1, x fastest) of marker k from its owner cell:
// its index in j, false when it lies outside the grid.
__device__ __forceinline__ bool support_cell(const GridParams &g, const MarkerBuffers &m, int k,
                                             int sc, long long &j) {
    const int o[3] = {sc % 3 - 1, (sc / 3) % 3 - 1, g.dim == 3 ? sc / 9 - 1 : 0};
    int c[3] = {0, 0, 0};
    for (int d = 0; d < g.dim; ++d) {
        c[d] = m.cell[(long long)k * 3 + d] + o[d];
        if (c[d] < 0 || c[d] >= g.n[d]) return false;
    }
    j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    return in_bounds(j, g.N, m.err);
}

constexpr int SMALL_NS = kSmallRebuildNs;
static_assert(SMALL_NS <= SORT_T, "one marker per thread");
__global__ void __launch_bounds__(SORT_T)
small_rebuild_kernel(const GridParams g, const MarkerBuffers m, double amp, double freq, int axis,
                     const double *__restrict__ dt, double dt_fixed) {
    __shared__ unsigned s_key[SMALL_NS];
    __shared__ unsigned s_sorted[SMALL_NS];
    __shared__ int s_warp[33];
    __shared__ double s_mv[2];
    const int tid = threadIdx.x, ns = m.ns;
    const int nsc = g.dim == 3 ? 27 : 9;
    if (tid == 0) motion_offset(amp, freq, m.t, dt, dt_fixed, s_mv[0], s_mv[1]);
    // the previous forced cells off (the same support cells the scatter
    // below sets, from the owner cells of the previous step)
    for (int i = tid; i < ns * nsc; i += SORT_T) {
        long long j;
        if (support_cell(g, m, i / nsc, i % nsc, j)) atomicAnd(m.band_bits + (j >> 5), ~(1u << (j & 31)));
    }
    __syncthreads();
    int bad = 0;
    if (tid < ns) {
        const int k = tid;
        for (int d = 0; d < g.dim; ++d) {
            const long long q = (long long)k * g.dim + d;
            m.X[q] = m.X0[q] + (d == axis ? s_mv[0] : 0.0);
            m.Ub[q] = m.Ub0[q] + (d == axis ? s_mv[1] : 0.0);
        }
        s_key[k] = owner_cell(g, m.X, k, m.cell, m.frac_d, m.frac_f, bad);
        // the marker's 1D support weights for the assembly (those of
        // support_weights_kernel, which the quadrature then skips)
        for (int d = 0; d < g.dim; ++d) {
            const double fk = m.frac_d[(long long)k * 3 + d];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                m.wphi[(long long)k * 9 + d * 3 + i] = phi_d(((double)(i - 1) + 0.5) - fk);
        }
    }
    if (bad) record_error(m.err, ERR_MARKER_RANGE);
    __syncthreads();
    if (tid < ns) {
        const unsigned key = s_key[tid];
        int r = 0;
        for (int j = 0; j < ns; ++j) {
            const unsigned kj = s_key[j];
            r += kj < key || (kj == key && j < tid);
        }
        s_sorted[r] = key;
        m.keys[0][r] = key;
        m.perm[0][r] = tid;
    }
    __syncthreads();
    // tile offsets (lower bounds in the sorted keys), occupancy; band flags
    // cleared for the scatter
    const unsigned cpt = (unsigned)g.cells_per_tile;
    for (int t = tid; t <= g.n_tiles; t += SORT_T) {
        const unsigned target = (unsigned)t * cpt;
        int lo = 0, hi = ns;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_sorted[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        m.tile_off[t] = lo;
        if (t < g.n_tiles) {
            // occupied: some key in [t cpt, (t+1) cpt)
            m.occ_flag[t] = lo < ns && s_sorted[lo] < target + cpt;
            m.band_flag[t] = 0;
        }
    }
    __syncthreads();
    // forced cells: the 3^d support cells of every marker
    for (int i = tid; i < ns * nsc; i += SORT_T) {
        long long j;
        if (!support_cell(g, m, i / nsc, i % nsc, j)) continue;
        atomicOr(m.band_bits + (j >> 5), 1u << (j & 31));
        const int cx = (int)(j % g.n[0]), cy = (int)((j / g.n[0]) % g.n[1]),
                  cz = (int)(j / ((long long)g.n[0] * g.n[1]));
        m.band_flag[cell_key(g, cx, cy, cz) / cpt] = 1;
    }
    __syncthreads();
    tile_lists(g.n_tiles, m.occ_flag, m.band_flag, m.occ_list, m.band_list, m.counts, s_warp);
}

// ---------------------------------------------------------------------------
// interpolation + forcing
// ---------------------------------------------------------------------------

// The interpolated fields of cell j: rho, rho u.., rho e = rho E - |rho u|^2/(2 rho).
template <int DIM, typename R>
__device__ __forceinline__ void interp_fields(const R *__restrict__ U, long long N, long long j,
                                              R (&v)[DIM + 2]) {
    const R rho = U[j];
    R ke = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const R md = U[(1 + d) * N + j];
        v[1 + d] = md;
        ke += md * md;
    }
    v[0] = rho;
    v[DIM + 1] = U[(DIM + 1) * N + j] - R(0.5) * rdiv<R>(ke, rho);
}

// rho_L and the forcing of marker k from its interpolated sums (lane 0):
// G = dt F = rho_L U_b - I[rho u], H = dt Q = rho_L c_v T_w - I[rho e].
template <int DIM, typename R>
__device__ __forceinline__ void store_forcing(const GridParams &g, const MarkerBuffers &m, int k,
                                              const R (&acc)[DIM + 2]) {
    const double rk = (double)acc[0];
    const double e = m.eps[k];
    R *gs = reinterpret_cast<R *>(m.gs) + 4 * (long long)k;
    m.rhoL[k] = rk;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const double Gd = rk * m.Ub[(long long)k * DIM + d] - (double)acc[1 + d];
        m.G[(long long)k * DIM + d] = Gd;
        gs[d] = (R)(Gd * e);
    }
    if (DIM == 2) gs[2] = R(0);
    const double H = rk * g.cv * m.Tw[k] - (double)acc[DIM + 1];
    m.H[k] = H;
    gs[3] = (R)(H * e);
}

// Batched form: one warp per (case, marker) item, the 3^DIM support cells
// read straight from the case's state; the terms and warp sums of
// interp_direct_kernel, so the results are bitwise the per-case step's.
template <int DIM, typename T>
__global__ void __launch_bounds__(512)
batch_interp_kernel(const BatchCase *__restrict__ cases, const int2 *__restrict__ items,
                    int n_items) {
    using R = T;
    constexpr int NF = DIM + 2;
    constexpr int NS = DIM == 3 ? 27 : 9;
    const int lane = threadIdx.x & 31;
    const int nw = blockDim.x >> 5;
    for (int it = blockIdx.x * nw + (threadIdx.x >> 5); it < n_items; it += gridDim.x * nw) {
        const int2 w = items[it];
        const BatchCase &bc = cases[w.x];
        const GridParams &g = bc.g;
        const MarkerBuffers &m = bc.m;
        const R *U = (const R *)bc.Us;
        const int k = w.y;
        R fr[3] = {R(0), R(0), R(0)};
        int ck[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            ck[d] = m.cell[(long long)k * 3 + d];
            fr[d] = marker_frac<R>(m, k, d);
        }
        R acc[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = R(0);
        if (lane < NS) {
            int cell[3];
            const R wgt = lane_weight<DIM, R>(fr, ck, lane, cell);
            const long long j = cell[0] + (long long)g.n[0] * (cell[1] + (long long)g.n[1] * cell[2]);
            R v[NF];
            if (in_bounds(j, g.N, m.err)) {
                interp_fields<DIM, R>(U, g.N, j, v);
#pragma unroll
                for (int f = 0; f < NF; ++f) acc[f] = wgt * v[f];
            }
        }
#pragma unroll
        for (int f = 0; f < NF; ++f) acc[f] = warp_sum_r<R>(acc[f]);
        if (lane == 0) store_forcing<DIM, R>(g, m, k, acc);
    }
}

// Interpolation and forcing of one grid (Eqs. interp, forceMomentum,
// corr3.8) with one warp per marker, lane l on support cell l, the cells read
// straight from the state (L2): every SM gets markers at once, where a form
// staging each occupied tile in shared memory ran one CTA per tile in a
// single short wave (3D sphere at 256^3: 18.6 -> 10.5 us; moving cylinder
// 12.5 -> 8.3 us, heated cylinder 18.6 -> 12.4 us per step, results bitwise
// the same).  The warp sums run in a fixed order.
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
interp_direct_kernel(const GridParams g, const T *__restrict__ U, const MarkerBuffers m) {
    using R = T;
    constexpr int NF = DIM + 2;
    constexpr int NS = DIM == 3 ? 27 : 9;
    const int lane = threadIdx.x & 31;
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
    if (k >= m.ns) return;
    R fr[3] = {R(0), R(0), R(0)};
    int ck[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        ck[d] = m.cell[(long long)k * 3 + d];
        fr[d] = marker_frac<R>(m, k, d);
    }
    R acc[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = R(0);
    if (lane < NS) {
        int cell[3];
        const R wgt = lane_weight<DIM, R>(fr, ck, lane, cell);
        const long long j = cell[0] + (long long)g.n[0] * (cell[1] + (long long)g.n[1] * cell[2]);
        R v[NF];
        if (in_bounds(j, g.N, m.err)) {
            interp_fields<DIM, R>(U, g.N, j, v);
#pragma unroll
            for (int f = 0; f < NF; ++f) acc[f] = wgt * v[f];
        }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) acc[f] = warp_sum_r<R>(acc[f]);
    if (lane == 0) store_forcing<DIM, R>(g, m, k, acc);
}

// ---------------------------------------------------------------------------
// spreading as a cell-centric gather
// ---------------------------------------------------------------------------

// threads of a spreading CTA (one band tile at a time): a 3D body has a few
// dozen 8^3 band tiles, whose candidate staging and gathers finish sooner with
// 512 threads; the many small 2D tiles of a batch run best at 256
template <int DIM> constexpr int SP_T = DIM == 3 ? 512 : 256;
constexpr int SP_MAXC = 1024;   // staged candidates per band tile

template <typename R>
size_t spread_smem_bytes(const GridParams &g) {
    const size_t bn = (size_t)(g.tile[0] + 2) * (g.tile[1] + 2) * (g.dim == 3 ? g.tile[2] + 2 : 1);
    return SP_MAXC * (7 * sizeof(R) + 2 * sizeof(int)) + 2 * bn * sizeof(int);
}

// Forced update of one band cell (App. B, Eqs. u_centralF2 and e_centralF2;
// f.u dropped): momentum += dt f, internal energy += dt q, rho unchanged, so
// rho E gains dt q + (|m1|^2 - |m0|^2) / (2 rho), the difference taken as
// sum_d f_d (m0_d + m1_d) (no cancellation).  The heat source is capped at
// kHeatSourceCap of the cell's internal energy (positivity reading).  In the
// spreading precision R (the field precision).
template <int DIM, typename R>
__device__ __forceinline__ void force_cell(const GridParams &g, R (&u)[DIM + 2], const R *f, R qh) {
    const R rho = u[0];
    R dke = R(0), ke0 = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const R m0 = u[1 + d];
        const R m1 = m0 + f[d];
        dke += f[d] * (m0 + m1);
        ke0 += m0 * m0;
        u[1 + d] = m1;
    }
    const R E = u[DIM + 1];
    const R qmin = -(R)kHeatSourceCap * (E - R(0.5) * ke0 / rho);
    if (qh < qmin) qh = qmin;
    u[DIM + 1] = g.energy_reading == 1 ? E + qh : E + (qh + R(0.5) * dke / rho);
}

template <int DIM, typename T, typename R>
__device__ __forceinline__ void apply_forcing(const GridParams &g, T *__restrict__ U, long long j,
                                              const R *f, R qh) {
    const long long N = g.N;
    R u[DIM + 2];
#pragma unroll
    for (int c = 0; c < DIM + 2; ++c) u[c] = (R)U[c * N + j];
    force_cell<DIM, R>(g, u, f, qh);
#pragma unroll
    for (int c = 1; c < DIM + 2; ++c) U[c * N + j] = (T)u[c];
}

// Shared memory of the spreading kernels: staged candidate markers (dynamic)
// and the small per-tile tables (static, declared by the kernel).
template <typename R>
struct SpreadSmem {
    R *fr, *g, *h;                // [3][SP_MAXC] offsets, [3][SP_MAXC] eps~ G, [SP_MAXC] eps~ H
    int *cell, *k;                // [SP_MAXC] owner cell in box, [SP_MAXC] marker
    int *head, *len;              // [bn], [bn]
    int *cnt, *start, *warp;      // [NT3 + 1], [NT3], [33]
};

template <typename R>
__device__ __forceinline__ SpreadSmem<R> spread_smem(unsigned char *raw, const GridParams &g,
                                                     int *cnt, int *start, int *warp) {
    const int bn = (g.tile[0] + 2) * (g.tile[1] + 2) * (g.dim == 3 ? g.tile[2] + 2 : 1);
    SpreadSmem<R> sm;
    sm.fr = reinterpret_cast<R *>(raw);
    sm.g = sm.fr + 3 * SP_MAXC;
    sm.h = sm.g + 3 * SP_MAXC;
    sm.cell = reinterpret_cast<int *>(sm.h + SP_MAXC);
    sm.k = sm.cell + SP_MAXC;
    sm.head = sm.k + SP_MAXC;
    sm.len = sm.head + bn;
    sm.cnt = cnt;
    sm.start = start;
    sm.warp = warp;
    return sm;
}

// Candidates of marker tile t: stage, in bin order, the markers whose owner
// cell lies in the tile grown by one cell (their supports reach the tile),
// then the runs of candidates per owner cell.  o receives the tile's first
// cell; returns true when the candidates overflowed the staging area (the
// caller then gathers from global memory).  Every thread calls it; it ends
// with a barrier.
template <int DIM, typename R>
__device__ __forceinline__ bool spread_stage(const GridParams &g, const MarkerBuffers &m,
                                             const unsigned *__restrict__ keys,
                                             const int *__restrict__ perm, int t,
                                             const SpreadSmem<R> &sm, int o[3]) {
    constexpr int NT3 = DIM == 3 ? 27 : 9;
    const int bx = g.tile[0] + 2, by = g.tile[1] + 2, bz = DIM == 3 ? g.tile[2] + 2 : 1;
    const int bn = bx * by * bz;
    R *s_fr = sm.fr, *s_g = sm.g, *s_h = sm.h;
    int *s_cell = sm.cell, *s_head = sm.head, *s_len = sm.len;
    int *s_cnt = sm.cnt, *s_start = sm.start, *s_warp = sm.warp;
    const int tid = threadIdx.x;
    const int cpt = g.cells_per_tile;
    const int tx = t % g.ntile[0], ty = (t / g.ntile[0]) % g.ntile[1],
              tz = t / (g.ntile[0] * g.ntile[1]);
    o[0] = tx * g.tile[0];
    o[1] = ty * g.tile[1];
    o[2] = DIM == 3 ? tz * g.tile[2] : 0;
    // 1. bin ranges of the neighbour tiles (z, y, x order)
    if (tid < NT3) {
        const int ux = tx + tid % 3 - 1, uy = ty + (tid / 3) % 3 - 1,
                  uz = tz + (DIM == 3 ? tid / 9 - 1 : 0);
        int st = 0, cnt = 0;
        if (ux >= 0 && uy >= 0 && uz >= 0 && ux < g.ntile[0] && uy < g.ntile[1] &&
            uz < g.ntile[2]) {
            const int u = ux + g.ntile[0] * (uy + g.ntile[1] * uz);
            st = m.tile_off[u];
            cnt = m.tile_off[u + 1] - st;
        }
        s_start[tid] = st;
        s_cnt[tid + 1] = cnt;
    }
    __syncthreads();
    if (tid == 0) {
        s_cnt[0] = 0;
        for (int i = 1; i <= NT3; ++i) s_cnt[i] += s_cnt[i - 1];
    }
    __syncthreads();
    const int total = s_cnt[NT3];
    // 2. stage, in order, the markers whose owner cell lies in the tile
    //    grown by one cell (their supports reach the tile)
    int kept = 0;
    for (int base = 0; base < total; base += SP_T<DIM>) {
        const int i = base + tid;
        int keep = 0, p = 0, lc = 0;
        if (i < total) {
            int nt = 0;
            while (s_cnt[nt + 1] <= i) ++nt;
            p = s_start[nt] + (i - s_cnt[nt]);
            const unsigned key = keys[p];
            const int tu = (int)(key / (unsigned)cpt);
            const int cin = (int)(key - (unsigned)tu * (unsigned)cpt);
            const int cu[3] = {(tu % g.ntile[0]) * g.tile[0] + cin % g.tile[0],
                               ((tu / g.ntile[0]) % g.ntile[1]) * g.tile[1] +
                                   (cin / g.tile[0]) % g.tile[1],
                               (tu / (g.ntile[0] * g.ntile[1])) * g.tile[2] +
                                   cin / (g.tile[0] * g.tile[1])};
            const int d0 = cu[0] - o[0] + 1, d1 = cu[1] - o[1] + 1,
                      d2 = DIM == 3 ? cu[2] - o[2] + 1 : 0;
            keep = d0 >= 0 && d0 < bx && d1 >= 0 && d1 < by && d2 >= 0 && d2 < bz;
            lc = d0 + bx * (d1 + by * d2);
        }
        int tot;
        const int pos = block_exclusive_scan(keep, s_warp, tot) + kept;
        if (keep && pos < SP_MAXC && in_bounds(perm[p], m.ns, m.err)) {
            const int k = perm[p];
            const double e = m.eps[k];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                s_fr[d * SP_MAXC + pos] = marker_frac<R>(m, k, d);
                s_g[d * SP_MAXC + pos] = d < DIM ? (R)(m.G[(long long)k * DIM + d] * e) : R(0);
            }
            s_h[pos] = (R)(m.H[k] * e);
            s_cell[pos] = lc;
            sm.k[pos] = k;
        }
        kept += tot;
    }
    const bool overflow = kept > SP_MAXC;
    // 3. runs of candidates per owner cell (contiguous in bin order)
    if (!overflow) {
        for (int q = tid; q < bn; q += SP_T<DIM>) s_head[q] = -1;
        __syncthreads();
        for (int i = tid; i < kept; i += SP_T<DIM>) {
            const int c = s_cell[i];
            if (i == 0 || s_cell[i - 1] != c) {
                int j = i + 1;
                while (j < kept && s_cell[j] == c) ++j;
                s_head[c] = i;
                s_len[c] = j - i;
            }
        }
    }
    __syncthreads();
    return overflow;
}

// The staged candidates of local cell l of a tile (l in [0, tile)) in the
// gather order - owner cells by z, y, x offset from -1 to +1, then bin order
// - as visit(slot, w) with w the weight of that marker at the cell.  Returns
// whether there was any.
template <int DIM, typename R, typename F>
__device__ __forceinline__ bool visit_staged(const GridParams &g, const SpreadSmem<R> &sm,
                                             const int l[3], F &&visit) {
    const int bx = g.tile[0] + 2, by = g.tile[1] + 2;
    bool any = false;
    const int zr = DIM == 3 ? 1 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int lc = (l[0] + 1 + ox) +
                               bx * ((l[1] + 1 + oy) + by * (DIM == 3 ? l[2] + 1 + oz : 0));
                const int h0 = sm.head[lc];
                if (h0 < 0) continue;
                const int h1 = h0 + sm.len[lc];
                const int oo[3] = {-ox, -oy, -oz};   // this cell seen from the owner cell
                for (int i = h0; i < h1; ++i) {
                    R w = R(1);
#pragma unroll
                    for (int d = 0; d < DIM; ++d)
                        w *= phi_r<R>(cell_offset<R>(oo[d], sm.fr[d * SP_MAXC + i]));
                    visit(i, w);
                    any = true;
                }
            }
    return any;
}

// Spreading and the forced update of the cells of marker tile t; smax
// collects the step-size rates of the forced cells.  Every thread calls it.
template <int DIM, typename T>
__device__ __forceinline__ void spread_tile(const GridParams &g, T *__restrict__ U,
                                            const MarkerBuffers &m,
                                            const unsigned *__restrict__ keys,
                                            const int *__restrict__ perm, int t,
                                            const SpreadSmem<T> &sm, T &smax, bool &ok) {
    using R = T;
    const R *s_g = sm.g, *s_h = sm.h;
    const int tid = threadIdx.x;
    const int cpt = g.cells_per_tile;
    int o[3];
    const bool overflow = spread_stage<DIM, R>(g, m, keys, perm, t, sm, o);
    // 4. gather per cell in the fixed order, then the forced update
    for (int q = tid; q < cpt; q += SP_T<DIM>) {
        const int l[3] = {q % g.tile[0], (q / g.tile[0]) % g.tile[1],
                          DIM == 3 ? q / (g.tile[0] * g.tile[1]) : 0};
        const int c[3] = {o[0] + l[0], o[1] + l[1], o[2] + l[2]};
        if (c[0] >= g.n[0] || c[1] >= g.n[1] || (DIM == 3 && c[2] >= g.n[2])) continue;
        R f[DIM], qh = R(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) f[d] = R(0);
        bool band = false;
        if (!overflow) {
            band = visit_staged<DIM, R>(g, sm, l, [&](int i, R w) {
#pragma unroll
                for (int d = 0; d < DIM; ++d) f[d] += s_g[d * SP_MAXC + i] * w;
                qh += s_h[i] * w;
            });
        } else {
            band = gather_markers<DIM, R>(g, m, keys, perm, c, [&](int k, R w) {
                const double e = m.eps[k];
#pragma unroll
                for (int d = 0; d < DIM; ++d) f[d] += (R)(m.G[(long long)k * DIM + d] * e) * w;
                qh += (R)(m.H[k] * e) * w;
            });
        }
        if (!band) continue;
        const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
        if (!in_bounds(j, g.N, m.err)) continue;
        apply_forcing<DIM, T, R>(g, U, j, f, qh);
        T u[DIM + 2];
#pragma unroll
        for (int cc = 0; cc < DIM + 2; ++cc) u[cc] = U[cc * g.N + j];
        smax = fmax(smax, step_rate<DIM, T>(g, u, ok));
    }
    __syncthreads();
}

template <int DIM, typename T>
__global__ void __launch_bounds__(SP_T<DIM>)
spread_apply_kernel(const GridParams g, T *__restrict__ U, const MarkerBuffers m,
                    const unsigned *__restrict__ keys, const int *__restrict__ perm) {
    constexpr int NT3 = DIM == 3 ? 27 : 9;
    extern __shared__ __align__(16) unsigned char smem_sp[];
    __shared__ int s_cnt[NT3 + 1], s_start[NT3], s_warp[33];
    __shared__ double s_max[SP_T<DIM> / 32];
    const SpreadSmem<T> sm = spread_smem<T>(smem_sp, g, s_cnt, s_start, s_warp);
    const int tid = threadIdx.x;
    const int n_band = m.counts[1];
    T smax = T(0);   // step-size rate of the forced cells, for the next dt
    bool ok = true;
    for (int it = blockIdx.x; it < n_band; it += gridDim.x)
        spread_tile<DIM, T>(g, U, m, keys, perm, m.band_list[it], sm, smax, ok);
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o2));
    const int bad = __syncthreads_or(!ok);
    if ((tid & 31) == 0) s_max[tid >> 5] = (double)smax;
    __syncthreads();
    if (tid == 0) {
        double mx = s_max[0];
        for (int w = 1; w < SP_T<DIM> / 32; ++w) mx = dmax_nonneg(mx, s_max[w]);
        m.bandmax[blockIdx.x] = mx;
        if (bad) record_error(m.err, ERR_NONFINITE);
    }
}


// The spreading operator of static markers, built once per marker set: for
// every forced cell its (marker, weight) entries in the gather order of
// spread_tile, so that the spreading of a step is a plain gather over them.
// Cells and entry runs are allocated by atomics per block of cells, so their
// placement varies between builds but no cell's run does.  counts[2..3]
// must be zero on entry.  A marker reaches 3^dim cells, so 3^dim x markers
// (sp_cap) bounds both the cells and the entries; a block that would pass
// it records ERR_BOUNDS and writes nothing (its records stay empty).
template <int DIM, typename T>
__global__ void __launch_bounds__(SP_T<DIM>)
spread_build_kernel(const GridParams g, const MarkerBuffers m, const unsigned *__restrict__ keys,
                    const int *__restrict__ perm) {
    using R = T;
    constexpr int NT3 = DIM == 3 ? 27 : 9;
    extern __shared__ __align__(16) unsigned char smem_sp[];
    __shared__ int s_cnt[NT3 + 1], s_start[NT3], s_warp[33];
    __shared__ int s_base[2];
    const SpreadSmem<R> sm = spread_smem<R>(smem_sp, g, s_cnt, s_start, s_warp);
    const int tid = threadIdx.x;
    const int cpt = g.cells_per_tile;
    R *w_out = reinterpret_cast<R *>(m.sp_w);
    const int n_band = m.counts[1];
    for (int it = blockIdx.x; it < n_band; it += gridDim.x) {
        int o[3];
        const bool overflow = spread_stage<DIM, R>(g, m, keys, perm, m.band_list[it], sm, o);
        for (int q0 = 0; q0 < cpt; q0 += SP_T<DIM>) {
            const int q = q0 + tid;
            const int l[3] = {q % g.tile[0], (q / g.tile[0]) % g.tile[1],
                              DIM == 3 ? q / (g.tile[0] * g.tile[1]) : 0};
            const int c[3] = {o[0] + l[0], o[1] + l[1], o[2] + l[2]};
            const bool inside = q < cpt && c[0] < g.n[0] && c[1] < g.n[1] &&
                                (DIM == 2 || c[2] < g.n[2]);
            int n = 0;
            if (inside) {
                if (!overflow) visit_staged<DIM, R>(g, sm, l, [&](int, R) { ++n; });
                else gather_markers<DIM, R>(g, m, keys, perm, c, [&](int, R) { ++n; });
            }
            int tot_c, tot_e;
            const int co = block_exclusive_scan(n > 0 ? 1 : 0, s_warp, tot_c);
            const int eo = block_exclusive_scan(n, s_warp, tot_e);
            if (tid == 0) {
                s_base[0] = tot_c > 0 ? atomicAdd(m.counts + 2, tot_c) : 0;
                s_base[1] = tot_e > 0 ? atomicAdd(m.counts + 3, tot_e) : 0;
            }
            __syncthreads();
            const long long bc = s_base[0], be = s_base[1];
            if (bc + tot_c > m.sp_cap || be + tot_e > m.sp_cap) {
                if (tid == 0) record_error(m.err, ERR_BOUNDS);
            } else if (n > 0) {
                const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
                int p = (int)be + eo;
                m.sp_cell[bc + co] = SpreadCell{j, p, n};
                if (!overflow) {
                    visit_staged<DIM, R>(g, sm, l, [&](int i, R w) {
                        m.sp_k[p] = sm.k[i];
                        w_out[p] = w;
                        ++p;
                    });
                } else {
                    gather_markers<DIM, R>(g, m, keys, perm, c, [&](int k, R w) {
                        m.sp_k[p] = k;
                        w_out[p] = w;
                        ++p;
                    });
                }
            }
            __syncthreads();   // s_base is taken again by the next block of cells
        }
    }
}

__device__ __forceinline__ void load4(const float *p, float v[4]) {
    const float4 x = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
__device__ __forceinline__ void load4(const double *p, double v[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

constexpr int SPS_B = 8;   // operator entries whose loads issue together

// Forced cell i of the spreading operator: its entries summed in the stored
// order, the forced update, its step-size rate into smax.
template <int DIM, typename T>
__device__ __forceinline__ void spread_static_cell(const GridParams &g, T *__restrict__ U,
                                                   const MarkerBuffers &m, int i, T &smax,
                                                   bool &ok) {
    using R = T;
    const R *gs = reinterpret_cast<const R *>(m.gs);
    const R *ew = reinterpret_cast<const R *>(m.sp_w);
    const SpreadCell rc = m.sp_cell[i];
    if (rc.n <= 0 || !in_bounds(rc.j, g.N, m.err)) return;
    // the cell's state is loaded ahead of its entries
    T u[DIM + 2];
#pragma unroll
    for (int cc = 0; cc < DIM + 2; ++cc) u[cc] = U[cc * g.N + rc.j];
    R f[DIM], qh = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) f[d] = R(0);
    // entries in batches of SPS_B: their loads issue together, then
    // the terms in the stored order
    const int pe = rc.start + rc.n;
    for (int p0 = rc.start; p0 < pe; p0 += SPS_B) {
        int k[SPS_B];
        R w[SPS_B], v[SPS_B][4];
#pragma unroll
        for (int b = 0; b < SPS_B; ++b) {
            const int p = p0 + b;
            const bool in = p < pe && in_bounds(p, m.sp_cap, m.err);
            k[b] = in ? __ldg(m.sp_k + p) : -1;
            w[b] = in ? __ldg(ew + p) : R(0);
        }
#pragma unroll
        for (int b = 0; b < SPS_B; ++b) {
            if (k[b] >= 0 && in_bounds(k[b], m.ns, m.err)) {
                load4(gs + 4 * (long long)k[b], v[b]);
            } else {
                k[b] = -1;
                v[b][0] = v[b][1] = v[b][2] = v[b][3] = R(0);
            }
        }
#pragma unroll
        for (int b = 0; b < SPS_B; ++b) {
            if (k[b] < 0) continue;
#pragma unroll
            for (int d = 0; d < DIM; ++d) f[d] += v[b][d] * w[b];
            qh += v[b][3] * w[b];
        }
    }
    // the forced update (as apply_forcing), the rate from the new state
    force_cell<DIM, T>(g, u, f, qh);
#pragma unroll
    for (int cc = 1; cc < DIM + 2; ++cc) U[cc * g.N + rc.j] = u[cc];
    smax = fmax(smax, step_rate<DIM, T>(g, u, ok));
}

// Spreading and forced update of static markers through their operator:
// one thread per forced cell sums its entries in the stored order (the
// terms and the order of spread_tile, so the results are bitwise the same),
// then applies the forcing.  One step-size maximum per CTA in bandmax.
constexpr int SPS_T = 256;
template <int DIM, typename T>
__global__ void __launch_bounds__(SPS_T)
spread_static_kernel(const GridParams g, T *__restrict__ U, const MarkerBuffers m) {
    __shared__ double s_max[SPS_T / 32];
    const int nc = min(m.counts[2], m.sp_cap);
    T smax = T(0);
    bool ok = true;
    for (int i = blockIdx.x * SPS_T + threadIdx.x; i < nc; i += gridDim.x * SPS_T)
        spread_static_cell<DIM, T>(g, U, m, i, smax, ok);
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o2));
    const int bad = __syncthreads_or(!ok);
    if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = (double)smax;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = s_max[0];
        for (int w = 1; w < SPS_T / 32; ++w) mx = dmax_nonneg(mx, s_max[w]);
        m.bandmax[blockIdx.x] = mx;
        if (bad) record_error(m.err, ERR_NONFINITE);
    }
}

// Batched form of the operator spreading (static markers): items are (case,
// first of a run of 32 of the case's forced cells), one warp each; one
// step-size maximum per item.  The cells are formed as in
// spread_static_kernel, so a batch step stays bitwise the per-case step.
template <typename T>
__global__ void __launch_bounds__(256)
batch_spread_static_kernel(const BatchCase *__restrict__ cases, const int2 *__restrict__ items,
                           int n_items, double *__restrict__ band_max) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < n_items; it += nw) {
        const int2 w = items[it];
        const BatchCase &bc = cases[w.x];
        const int nc = min(bc.m.counts[2], bc.m.sp_cap);
        T smax = T(0);
        bool ok = true;
        if (w.y + lane < nc) spread_static_cell<2, T>(bc.g, (T *)bc.Us, bc.m, w.y + lane, smax, ok);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        const bool bad = __any_sync(0xffffffffu, !ok);
        if (lane == 0) {
            band_max[it] = (double)smax;
            if (bad) record_error(bc.err, ERR_NONFINITE);
        }
    }
}

// Batched form: items are (case, position in the case's band list); one
// step-size maximum per item.
template <int DIM, typename T>
__global__ void __launch_bounds__(SP_T<DIM>)
batch_spread_kernel(const BatchCase *__restrict__ cases, const int2 *__restrict__ items,
                    int n_items, double *__restrict__ band_max) {
    constexpr int NT3 = DIM == 3 ? 27 : 9;
    extern __shared__ __align__(16) unsigned char smem_sp[];
    __shared__ int s_cnt[NT3 + 1], s_start[NT3], s_warp[33];
    __shared__ double s_max[SP_T<DIM> / 32];
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
        const int2 w = items[it];
        const BatchCase &bc = cases[w.x];
        const GridParams g = bc.g;
        const MarkerBuffers m = bc.m;
        const SpreadSmem<T> sm = spread_smem<T>(smem_sp, g, s_cnt, s_start, s_warp);
        T smax = T(0);
        bool ok = true;
        spread_tile<DIM, T>(g, (T *)bc.Us, m, m.keys[m.sorted], m.perm[m.sorted],
                            m.band_list[w.y], sm, smax, ok);
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o2));
        const int bad = __syncthreads_or(!ok);
        if ((tid & 31) == 0) s_max[tid >> 5] = (double)smax;
        __syncthreads();
        if (tid == 0) {
            double mx = s_max[0];
            for (int w2 = 1; w2 < SP_T<DIM> / 32; ++w2) mx = dmax_nonneg(mx, s_max[w2]);
            band_max[it] = mx;
            if (bad) record_error(bc.err, ERR_NONFINITE);
        }
    }
}

// The forced cells, scattered from the markers: the support of marker k is
// the 3^d cells around its owner cell (per axis the owner and its two
// neighbours; the 3-point delta vanishes beyond), so one thread per (marker,
// support cell) sets that cell's bit in band_bits and the flag of its tile in
// band_flag - the set the spreading's cell-centric gather visits, with bit
// OR and flag stores that do not depend on order.  Both must be clear on
// entry.
template <int DIM>
__global__ void __launch_bounds__(256)
band_scatter_kernel(const GridParams g, const MarkerBuffers m) {
    constexpr int NSC = DIM == 3 ? 27 : 9;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int k = (int)(t / NSC), sc = (int)(t - (long long)k * NSC);
    if (k >= m.ns) return;
    const int o[3] = {sc % 3 - 1, (sc / 3) % 3 - 1, DIM == 3 ? sc / 9 - 1 : 0};
    int c[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        c[d] = m.cell[(long long)k * 3 + d] + o[d];
        if (c[d] < 0 || c[d] >= g.n[d]) return;
    }
    const long long j = c[0] + (long long)g.n[0] * (c[1] + (long long)g.n[1] * c[2]);
    if (!in_bounds(j, g.N, m.err)) return;
    atomicOr(m.band_bits + (j >> 5), 1u << (j & 31));
    m.band_flag[cell_key(g, c[0], c[1], c[2]) / (unsigned)g.cells_per_tile] = 1;
}

// ---------------------------------------------------------------------------
// forces/heat sums (fixed-order reduction) and the time update
// ---------------------------------------------------------------------------

constexpr int FIN_T = 256;   // threads of the batch finish and of the stage-1 sums

// A warp's five partials (sums 0..3, maximum 4) combined as a fixed
// shuffle tree; the result in every lane.
__device__ __forceinline__ void finish_combine(double a[5]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
        a[4] = dmax_nonneg(a[4], __shfl_xor_sync(0xffffffffu, a[4], o));
    }
}

// The finish of a grid splits its markers (and its maxima) into C chunks,
// chunk c covering [n c / C, n (c+1) / C), C = ceil(n_s / FIN_CHUNK) <= 32.
// One warp forms a chunk's partial: lane l sums markers k0 + l, k0 + l + 32,
// ... in order, then a shuffle tree; the C partials are combined by a second
// fixed tree.  FP64 is the limiter here (this GPU's FP64 pipe retires about
// two operations per SM cycle), so the chunks run on separate SMs with one
// warp each, and C depends on the marker count alone: the split kernel of
// one grid and the one-CTA finish of a batch case add the same partials in
// the same trees.
constexpr int FIN_CHUNK = 128;
__host__ __device__ __forceinline__ int finish_chunks(int ns) {
    const int c = (ns + FIN_CHUNK - 1) / FIN_CHUNK;
    return c < 1 ? 1 : (c > kFinishCtas ? kFinishCtas : c);
}
__host__ __device__ __forceinline__ int finish_cut(int n, int c, int C) {
    return (int)((long long)n * c / C);
}

// One warp: a[0..dim) = sum eps~ G, a[3] = sum eps~ H over markers [k0, k1)
// and a[4] = the largest of blockmax[b0, b1) and bandmax[c0, c1), in every
// lane on return.
__device__ __forceinline__ void finish_chunk(const GridParams &g, const MarkerBuffers &m, int k0,
                                             int k1, const double *__restrict__ blockmax, int b0,
                                             int b1, const double *__restrict__ bandmax, int c0,
                                             int c1, int lane, double a[5]) {
    const int dim = g.dim;
#pragma unroll
    for (int i = 0; i < 5; ++i) a[i] = 0.0;
    // the loads of FIN_B markers issue together, then their terms in order
    constexpr int FIN_B = 4;
    for (int kb = k0 + lane; kb < k1; kb += FIN_B * 32) {
        double e[FIN_B], gq[FIN_B][4];
#pragma unroll
        for (int i = 0; i < FIN_B; ++i) {
            const int k = kb + i * 32;
            e[i] = 0.0;
            gq[i][0] = gq[i][1] = gq[i][2] = gq[i][3] = 0.0;
            if (k < k1) {
                e[i] = __ldg(m.eps + k);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (d < dim) gq[i][d] = __ldg(m.G + (long long)k * dim + d);
                gq[i][3] = __ldg(m.H + k);
            }
        }
#pragma unroll
        for (int i = 0; i < FIN_B; ++i) {
            if (kb + i * 32 >= k1) break;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (d < dim) a[d] += e[i] * gq[i][d];
            a[3] += e[i] * gq[i][3];
        }
    }
    // maxima (the order does not matter), eight loads issued together
    for (int b = b0 + lane; b < b1; b += 8 * 32) {
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = b + i * 32 < b1 ? __ldg(blockmax + b + i * 32) : 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) a[4] = dmax_nonneg(a[4], v[i]);
    }
    for (int b = c0 + lane; b < c1; b += 8 * 32) {
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = b + i * 32 < c1 ? __ldg(bandmax + b + i * 32) : 0.0;
#pragma unroll
        for (int i = 0; i < 8; ++i) a[4] = dmax_nonneg(a[4], v[i]);
    }
    finish_combine(a);
}

// The sums of a step, its time update and the next step size from the
// largest rate mx (one thread).
__device__ __forceinline__ void finish_update(const GridParams &g, const MarkerBuffers &m,
                                              const double a[5], double *__restrict__ dt_ptr,
                                              int *__restrict__ err, double dt_fixed) {
    for (int i = 0; i < 4; ++i) {
        // forcing per stage: the first stage's sources count with weight 1/2
        m.sums[i] = g.forcing_per_stage ? a[i] + 0.5 * m.sums[8 + i] : a[i];
    }
    const double mx = a[4];
    const double dt_used = dt_fixed > 0.0 ? dt_fixed : *dt_ptr;
    m.sums[4] = dt_used;
    *m.t += dt_used;
    *m.steps += 1;
    const bool good = mx > 0.0 && mx <= DBL_MAX && !(__ldcg(err) & ERR_NONFINITE);
    if (!good) record_error(err, ERR_NONFINITE);
    *dt_ptr = good ? g.cfl / mx : 0.0;
}

// One CTA of FIN_T threads: the force/heat sums of one grid, its time update
// and its next step size from the stage-2 maxima (blockmax[0..nb)) and the
// forced-cell maxima (bandmax[0..nbs)); warp w forms chunks w, w + 8, ...
__device__ __forceinline__ void finish_grid(const GridParams &g, int ns, const MarkerBuffers &m,
                                            const double *__restrict__ blockmax, int nb,
                                            const double *__restrict__ bandmax, int nbs,
                                            double *__restrict__ dt_ptr, int *__restrict__ err,
                                            double dt_fixed, double (*part)[5]) {
    const int C = finish_chunks(ns);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = w; c < C; c += FIN_T / 32) {
        double a[5];
        finish_chunk(g, m, finish_cut(ns, c, C), finish_cut(ns, c + 1, C), blockmax,
                     finish_cut(nb, c, C), finish_cut(nb, c + 1, C), bandmax,
                     finish_cut(nbs, c, C), finish_cut(nbs, c + 1, C), lane, a);
        if (lane == 0)
            for (int i = 0; i < 5; ++i) part[c][i] = a[i];
    }
    __syncthreads();
    if (w != 0) return;
    double a[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) a[i] = lane < C ? part[lane][i] : 0.0;
    finish_combine(a);
    if (lane == 0) finish_update(g, m, a, dt_ptr, err, dt_fixed);
}

// sum eps~ G and sum eps~ H of the current marker forcing into sums[8..11],
// in the finish kernel's fixed order
__global__ void __launch_bounds__(FIN_T)
partial_sums_kernel(const GridParams g, const MarkerBuffers m) {
    __shared__ double s[4][FIN_T / 32];
    const int dim = g.dim;
    double a[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < m.ns; k += FIN_T) {
        const double e = __ldg(m.eps + k);
        for (int d = 0; d < dim; ++d) a[d] += e * __ldg(m.G + (long long)k * dim + d);
        a[3] += e * __ldg(m.H + k);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0)
        for (int i = 0; i < 4; ++i) s[i][w] = a[i];
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = lane < FIN_T / 32 ? s[i][lane] : 0.0;
#pragma unroll
    for (int o = FIN_T / 64; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
    if (lane == 0)
        for (int i = 0; i < 4; ++i) m.sums[8 + i] = a[i];
}

// The forced update of static markers with the step's finish in the same
// launch (one kernel less per step): CTAs c < C_m also form marker chunk c's
// force/heat partial (one warp, as finish_kernel's CTA c does), every CTA
// its forced cells' step-size maximum; the last CTA to finish (ticket)
// combines the partials in finish_kernel's tree (so the sums are bitwise
// those of the separate finish), takes the largest rate over the stage-2
// and forced-cell maxima, updates the time and the next step size, and
// resets the ticket.
template <int DIM, typename T>
__global__ void __launch_bounds__(SPS_T)
spread_static_finish_kernel(const GridParams g, T *__restrict__ U, const MarkerBuffers m,
                            const FinishArgs f) {
    __shared__ double s_max[SPS_T / 32];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int ns = m.ns, Cm = finish_chunks(ns);
    if ((int)blockIdx.x < Cm && w == 0) {
        double a[5];
        finish_chunk(g, m, finish_cut(ns, blockIdx.x, Cm), finish_cut(ns, blockIdx.x + 1, Cm),
                     f.blockmax, 0, 0, m.bandmax, 0, 0, lane, a);
        if (lane == 0)
            for (int i = 0; i < 5; ++i) f.part[blockIdx.x * 5 + i] = a[i];
    }
    const int nc = min(m.counts[2], m.sp_cap);
    T smax = T(0);
    bool ok = true;
    for (int i = blockIdx.x * SPS_T + tid; i < nc; i += gridDim.x * SPS_T)
        spread_static_cell<DIM, T>(g, U, m, i, smax, ok);
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o2));
    const int bad = __syncthreads_or(!ok);
    if (lane == 0) s_max[w] = (double)smax;
    __syncthreads();
    if (tid == 0) {
        double mx = s_max[0];
        for (int v = 1; v < SPS_T / 32; ++v) mx = dmax_nonneg(mx, s_max[v]);
        m.bandmax[blockIdx.x] = mx;
        if (bad) record_error(m.err, ERR_NONFINITE);
        __threadfence();
        s_last = atomicAdd(f.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // the largest rate: the stage-2 block maxima and every CTA's forced cells
    double mx = 0.0;
    for (int b = tid; b < f.nb; b += SPS_T) mx = dmax_nonneg(mx, __ldcg(f.blockmax + b));
    for (int b = tid; b < (int)gridDim.x; b += SPS_T) mx = dmax_nonneg(mx, __ldcg(m.bandmax + b));
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) mx = dmax_nonneg(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
    if (lane == 0) s_max[w] = mx;
    __syncthreads();
    if (w != 0) return;
    double a[5];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = lane < Cm ? __ldcg(f.part + lane * 5 + i) : 0.0;
    a[4] = 0.0;
    finish_combine(a);
    if (lane == 0) {
        for (int v = 0; v < SPS_T / 32; ++v) a[4] = dmax_nonneg(a[4], s_max[v]);
        finish_update(g, m, a, f.dt, f.err, f.dt_fixed);
        *f.ticket = 0u;
    }
}

// Split form: one warp per chunk (CTA c forms chunk c's partial into
// part[c]); the last CTA to finish (ticket) combines the C partials as the
// fixed tree of finish_combine, so the sums do not depend on which CTA comes
// last, and resets the ticket for the next launch.
__global__ void __launch_bounds__(32)
finish_kernel(const GridParams g, int ns, const MarkerBuffers m, const double *__restrict__ blockmax,
              int nb, int nbs, double *__restrict__ dt_ptr, int *__restrict__ err, double dt_fixed,
              double *__restrict__ part, unsigned *__restrict__ ticket) {
    // CTAs c < Cm form the marker chunks (as the batch finish does); the
    // maxima are shared over all C >= Cm CTAs, and CTAs past Cm add exact
    // zeros to the sums, as the empty lanes of the batch's combine do
    const int C = gridDim.x, c = blockIdx.x, lane = threadIdx.x;
    const int Cm = finish_chunks(ns);
    const int k0 = c < Cm ? finish_cut(ns, c, Cm) : ns, k1 = c < Cm ? finish_cut(ns, c + 1, Cm) : ns;
    double a[5];
    finish_chunk(g, m, k0, k1, blockmax, finish_cut(nb, c, C), finish_cut(nb, c + 1, C), m.bandmax,
                 finish_cut(nbs, c, C), finish_cut(nbs, c + 1, C), lane, a);
    unsigned last = 0;
    if (lane == 0) {
        for (int i = 0; i < 5; ++i) part[c * 5 + i] = a[i];
        __threadfence();
        last = atomicAdd(ticket, 1u) == (unsigned)C - 1;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
#pragma unroll
    for (int i = 0; i < 5; ++i) a[i] = lane < C ? __ldcg(part + lane * 5 + i) : 0.0;
    finish_combine(a);
    if (lane == 0) {
        finish_update(g, m, a, dt_ptr, err, dt_fixed);
        *ticket = 0u;
    }
}

// Batched form: CTA c finishes case c over its own stage and band items.
__global__ void __launch_bounds__(FIN_T)
batch_finish_kernel(const BatchCase *__restrict__ cases, const double *__restrict__ item_max,
                    const double *__restrict__ band_max, double dt_fixed) {
    __shared__ double part[kFinishCtas][5];
    const BatchCase &bc = cases[blockIdx.x];
    finish_grid(bc.g, bc.m.ns, bc.m, item_max + bc.item0, bc.nitems, band_max + bc.band0,
                bc.nband, bc.dt, bc.err, dt_fixed, part);
}

// The force sums, the step size they belong to and the time of every case
// of a batch, gathered for one read: out[c * 6 + i].
__global__ void batch_gather_kernel(const BatchCase *__restrict__ cases, int ncases,
                                    double *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncases) return;
    const MarkerBuffers &m = cases[c].m;
    for (int i = 0; i < 5; ++i) out[c * 8 + i] = m.sums[i];
    out[c * 8 + 5] = *m.t;
    out[c * 8 + 6] = (double)*cases[c].err;
    out[c * 8 + 7] = 0.0;
}

__global__ void batch_tw_kernel(const BatchTwSlot *__restrict__ slots,
                                const double *__restrict__ vals) {
    const BatchTwSlot sl = slots[blockIdx.x];
    for (long long k = threadIdx.x; k < sl.n; k += blockDim.x) sl.dst[k] = vals[sl.off + k];
}

// ---------------------------------------------------------------------------
// operators for the diagnostic entry points
// ---------------------------------------------------------------------------

// C_p at the markers: p = (gamma - 1)(rho E - |rho u|^2 / (2 rho)) interpolated
// with the weights of Eq. interp (FP64, one warp per marker, lane per cell).
template <int DIM, typename T>
__global__ void __launch_bounds__(256)
surface_pressure_kernel(const GridParams g, const T *__restrict__ U, const MarkerBuffers m) {
    constexpr int NS = DIM == 3 ? 27 : 9;
    const int lane = threadIdx.x & 31;
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= m.ns) return;
    double acc = 0.0;
    if (lane < NS) {
        double fr[3] = {0.0, 0.0, 0.0};
        int ck[3] = {0, 0, 0};
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            ck[d] = m.cell[(long long)k * 3 + d];
            fr[d] = m.frac_d[(long long)k * 3 + d];
        }
        int cell[3];
        const double w = lane_weight<DIM, double>(fr, ck, lane, cell);
        const long long j = cell[0] + (long long)g.n[0] * (cell[1] + (long long)g.n[1] * cell[2]);
        const double rho = (double)U[j];
        double msq = 0.0;
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const double md = (double)U[(1 + d) * g.N + j];
            msq += md * md;
        }
        const double p = (g.gamma - 1.0) * ((double)U[(DIM + 1) * g.N + j] - 0.5 * msq / rho);
        acc = w * p;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) m.cp[k] = 2.0 * (acc - g.p_inf);
}

template <int DIM, typename T>
__global__ void interpolate_op_kernel(const GridParams g, const T *__restrict__ field, int nc,
                                      const MarkerBuffers m, double *__restrict__ out) {
    using R = T;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m.ns) return;
    R fr[3] = {R(0), R(0), R(0)};
    int ck[3] = {0, 0, 0};
    for (int d = 0; d < DIM; ++d) {
        ck[d] = m.cell[(long long)k * 3 + d];
        fr[d] = marker_frac<R>(m, k, d);
    }
    for (int c = 0; c < nc; ++c) out[(long long)k * nc + c] = 0.0;
    constexpr int NS = DIM == 3 ? 27 : 9;
    for (int l = 0; l < NS; ++l) {
        int cell[3];
        const double w = (double)lane_weight<DIM, R>(fr, ck, l, cell);
        const long long j = cell[0] + (long long)g.n[0] * (cell[1] + (long long)g.n[1] * cell[2]);
        for (int c = 0; c < nc; ++c) out[(long long)k * nc + c] += w * (double)field[c * g.N + j];
    }
}

template <int DIM, typename T>
__global__ void __launch_bounds__(256)
spread_op_kernel(const GridParams g, const double *__restrict__ R_, int nc, const MarkerBuffers m,
                 const unsigned *__restrict__ keys, const int *__restrict__ perm,
                 T *__restrict__ out) {
    using R = T;
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
                gather_markers<DIM, R>(g, m, keys, perm, c, [&](int k, R w) {
                    acc += R_[(long long)k * nc + cc] * ((double)w * m.eps[k]);
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
                          int axis, const double *dt, double dt_fixed, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    motion_kernel<<<(m.ns + 127) / 128, 128, 0, s>>>(g, m.ns, m.X0, m.Ub0, m.X, m.Ub, amp, freq,
                                                      axis, m.t, dt, dt_fixed);
    return cudaGetLastError();
}

cudaError_t launch_small_rebuild(const GridParams &g, MarkerBuffers &m, double amp, double freq,
                                 int axis, const double *dt, double dt_fixed, cudaStream_t s) {
    if (m.ns <= 0 || m.ns > SMALL_NS) return cudaErrorInvalidValue;
    m.sorted = 0;
    small_rebuild_kernel<<<1, SORT_T, 0, s>>>(g, m, amp, freq, axis, dt, dt_fixed);
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
                                             m.perm[1], passes, m.err, m.cell, m.frac_d, m.frac_f);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    tile_offsets_kernel<<<(g.n_tiles + 1 + 255) / 256, 256, 0, s>>>(g, m.ns, m.keys[m.sorted],
                                                                     m.tile_off);
    tile_flags_kernel<<<(g.n_tiles + 255) / 256, 256, 0, s>>>(g, m.tile_off, m.occ_flag,
                                                              m.band_flag);
    return cudaGetLastError();
}

template <int DIM, typename T>
static cudaError_t interp_force_t(const GridParams &g, const void *U, const MarkerBuffers &m,
                                  int grid_ctas, cudaStream_t s) {
    (void)grid_ctas;
    const long long threads = 32ll * m.ns;
    interp_direct_kernel<DIM, T><<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(
        g, (const T *)U, m);
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

template <int DIM, typename T>
static cudaError_t spread_apply_t(const GridParams &g, void *U, const MarkerBuffers &m,
                                  int grid_ctas, cudaStream_t s, const FinishArgs *fin) {
    if (m.sp_ready) {
        if (fin)
            spread_static_finish_kernel<DIM, T><<<grid_ctas, SPS_T, 0, s>>>(g, (T *)U, m, *fin);
        else
            spread_static_kernel<DIM, T><<<grid_ctas, SPS_T, 0, s>>>(g, (T *)U, m);
        return cudaGetLastError();
    }
    if (fin) return cudaErrorInvalidValue;
    const size_t smem = spread_smem_bytes<T>(g);
    cudaError_t e = func_smem_attr((const void *)spread_apply_kernel<DIM, T>, smem);
    if (e != cudaSuccess) return e;
    spread_apply_kernel<DIM, T><<<grid_ctas, SP_T<DIM>, smem, s>>>(g, (T *)U, m, m.keys[m.sorted],
                                                                m.perm[m.sorted]);
    return cudaGetLastError();
}

cudaError_t launch_spread_apply(const GridParams &g, int fp_bytes, void *U,
                                const MarkerBuffers &m, int grid_ctas, cudaStream_t s,
                                const FinishArgs *fin) {
    if (m.ns <= 0) return cudaSuccess;
    if (g.dim == 3)
        return fp_bytes == 4 ? spread_apply_t<3, float>(g, U, m, grid_ctas, s, fin)
                             : spread_apply_t<3, double>(g, U, m, grid_ctas, s, fin);
    return fp_bytes == 4 ? spread_apply_t<2, float>(g, U, m, grid_ctas, s, fin)
                         : spread_apply_t<2, double>(g, U, m, grid_ctas, s, fin);
}

FinishArgs finish_args(const MarkerBuffers &m, const FluidBuffers &fb, int nb, double dt_fixed) {
    return FinishArgs{fb.blockmax, nb, fb.dt, fb.err, dt_fixed, m.finpart, fb.counter + 1};
}

template <int DIM, typename T>
static cudaError_t spread_build_t(const GridParams &g, const MarkerBuffers &m, int grid_ctas,
                                  cudaStream_t s) {
    // counts to zero; every cell record empty (n = 0), so a record that a
    // failed block reserved but did not write is skipped
    cudaError_t e = cudaMemsetAsync(m.counts + 2, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m.sp_cell, 0, sizeof(SpreadCell) * m.sp_cap, s);
    if (e != cudaSuccess) return e;
    const size_t smem = spread_smem_bytes<T>(g);
    e = func_smem_attr((const void *)spread_build_kernel<DIM, T>, smem);
    if (e != cudaSuccess) return e;
    spread_build_kernel<DIM, T><<<grid_ctas, SP_T<DIM>, smem, s>>>(g, m, m.keys[m.sorted],
                                                                m.perm[m.sorted]);
    return cudaGetLastError();
}

cudaError_t launch_spread_build(const GridParams &g, int fp_bytes, const MarkerBuffers &m,
                                int grid_ctas, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    if (g.dim == 3)
        return fp_bytes == 4 ? spread_build_t<3, float>(g, m, grid_ctas, s)
                             : spread_build_t<3, double>(g, m, grid_ctas, s);
    return fp_bytes == 4 ? spread_build_t<2, float>(g, m, grid_ctas, s)
                         : spread_build_t<2, double>(g, m, grid_ctas, s);
}

cudaError_t launch_finish(const GridParams &g, const MarkerBuffers &m, const FluidBuffers &fb,
                          int nb, int nbs, double dt_fixed, cudaStream_t s) {
    // the marker chunks, and at least one CTA per 512 maxima (up to kFinishCtas)
    const int C = std::max(finish_chunks(m.ns), std::min(kFinishCtas, (nb + nbs + 511) / 512));
    finish_kernel<<<C, 32, 0, s>>>(g, m.ns, m, fb.blockmax, nb, nbs, fb.dt, fb.err, dt_fixed,
                                      m.finpart, fb.counter + 1);
    return cudaGetLastError();
}

cudaError_t launch_batch_interp(int fp_bytes, const BatchCase *cases, const int2 *items,
                                int n_items, int warps, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    if (warps < 1 || warps > 16) return cudaErrorInvalidValue;
    const int nb = (n_items + warps - 1) / warps;
    if (fp_bytes == 4)
        batch_interp_kernel<2, float><<<nb, 32 * warps, 0, s>>>(cases, items, n_items);
    else
        batch_interp_kernel<2, double><<<nb, 32 * warps, 0, s>>>(cases, items, n_items);
    return cudaGetLastError();
}

size_t batch_spread_smem(const GridParams &g, int fp_bytes) {
    return fp_bytes == 4 ? spread_smem_bytes<float>(g) : spread_smem_bytes<double>(g);
}

template <typename T>
static cudaError_t batch_spread_t(size_t smem, const BatchCase *cases, const int2 *items,
                                  int n_items, double *band_max, int ctas, cudaStream_t s) {
    cudaError_t e = func_smem_attr((const void *)batch_spread_kernel<2, T>, smem);
    if (e != cudaSuccess) return e;
    batch_spread_kernel<2, T><<<ctas, SP_T<2>, smem, s>>>(cases, items, n_items, band_max);
    return cudaGetLastError();
}

cudaError_t launch_batch_spread_static(int fp_bytes, const BatchCase *cases, const int2 *items,
                                       int n_items, double *band_max, cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    const unsigned nb = (unsigned)((n_items + 7) / 8);   // eight warps per CTA
    if (fp_bytes == 4) batch_spread_static_kernel<float><<<nb, 256, 0, s>>>(cases, items, n_items, band_max);
    else batch_spread_static_kernel<double><<<nb, 256, 0, s>>>(cases, items, n_items, band_max);
    return cudaGetLastError();
}

cudaError_t launch_batch_spread(int fp_bytes, size_t smem, const BatchCase *cases,
                                const int2 *items, int n_items, double *band_max, int n_sm,
                                cudaStream_t s) {
    if (n_items <= 0) return cudaSuccess;
    int ctas = 4 * (n_sm > 0 ? n_sm : 1);
    if (ctas > n_items) ctas = n_items;
    return fp_bytes == 4 ? batch_spread_t<float>(smem, cases, items, n_items, band_max, ctas, s)
                         : batch_spread_t<double>(smem, cases, items, n_items, band_max, ctas, s);
}

cudaError_t launch_partial_sums(const GridParams &g, const MarkerBuffers &m, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    partial_sums_kernel<<<1, FIN_T, 0, s>>>(g, m);
    return cudaGetLastError();
}

cudaError_t launch_batch_finish(const BatchCase *cases, int ncases, const double *item_max,
                                const double *band_max, double dt_fixed, cudaStream_t s) {
    if (ncases <= 0) return cudaSuccess;
    batch_finish_kernel<<<ncases, FIN_T, 0, s>>>(cases, item_max, band_max, dt_fixed);
    return cudaGetLastError();
}

cudaError_t launch_batch_gather(const BatchCase *cases, int ncases, double *out, cudaStream_t s) {
    if (ncases <= 0) return cudaSuccess;
    batch_gather_kernel<<<(ncases + 127) / 128, 128, 0, s>>>(cases, ncases, out);
    return cudaGetLastError();
}

cudaError_t launch_batch_tw(const BatchTwSlot *slots, int ncases, const double *vals,
                            cudaStream_t s) {
    if (ncases <= 0) return cudaSuccess;
    batch_tw_kernel<<<ncases, 128, 0, s>>>(slots, vals);
    return cudaGetLastError();
}

cudaError_t launch_band_mask(const GridParams &g, const MarkerBuffers &m, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(m.band_bits, 0, sizeof(unsigned) * (size_t)(g.N / 32 + 1), s);
    if (e != cudaSuccess) return e;
    if (m.ns > 0) {
        const long long threads = (long long)m.ns * (g.dim == 3 ? 27 : 9);
        const unsigned nb = (unsigned)((threads + 255) / 256);
        if (g.dim == 3) band_scatter_kernel<3><<<nb, 256, 0, s>>>(g, m);
        else band_scatter_kernel<2><<<nb, 256, 0, s>>>(g, m);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    tile_lists_kernel<<<1, SORT_T, 0, s>>>(g.n_tiles, m.occ_flag, m.band_flag, m.occ_list,
                                           m.band_list, m.counts);
    return cudaGetLastError();
}

cudaError_t launch_surface_pressure(const GridParams &g, int fp_bytes, const void *U,
                                    const MarkerBuffers &m, cudaStream_t s) {
    if (m.ns <= 0) return cudaSuccess;
    const int nb = (m.ns * 32 + 255) / 256;
    if (g.dim == 3) {
        if (fp_bytes == 4) surface_pressure_kernel<3, float><<<nb, 256, 0, s>>>(g, (const float *)U, m);
        else surface_pressure_kernel<3, double><<<nb, 256, 0, s>>>(g, (const double *)U, m);
    } else {
        if (fp_bytes == 4) surface_pressure_kernel<2, float><<<nb, 256, 0, s>>>(g, (const float *)U, m);
        else surface_pressure_kernel<2, double><<<nb, 256, 0, s>>>(g, (const double *)U, m);
    }
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
