// Marker-side device helpers shared by the forward kernels (markers.cu) and
// the adjoint (adjoint.cu): the regularised delta in the field precision,
// the marker-to-cell offsets, warp sums and the fixed-order cell-centric
// visit of the markers whose support holds a cell.
#pragma once

#include "internal.h"

namespace ibmk {

// The 1D kernel evaluated in the field precision R: float on FP32 grids
// (weights within ~1e-7 relative), double on FP64 grids.
template <typename R> __device__ __forceinline__ R phi_r(R r);
template <> __device__ __forceinline__ float phi_r<float>(float r) {
    const float a = fabsf(r);
    if (a <= 0.5f) return (1.0f + sqrtf(1.0f - 3.0f * a * a)) * (1.0f / 3.0f);
    if (a <= 1.5f) {
        const float b = 1.0f - a;
        return (5.0f - 3.0f * a - sqrtf(1.0f - 3.0f * b * b)) * (1.0f / 6.0f);
    }
    return 0.0f;
}
template <> __device__ __forceinline__ double phi_r<double>(double r) { return phi_d(r); }

// Offset in cells from marker k to the centre of the cell o cells away from
// its owner cell on one axis: (o + 1/2) - frac, frac = (X - lo)/h - owner.
// Every kernel evaluates the weights through this one expression (in the
// field precision), so interpolation and spreading use identical weights.
template <typename R> __device__ __forceinline__ R marker_frac(const MarkerBuffers &m, int k, int d);
template <> __device__ __forceinline__ float marker_frac<float>(const MarkerBuffers &m, int k, int d) {
    return m.frac_f[(long long)k * 3 + d];
}
template <> __device__ __forceinline__ double marker_frac<double>(const MarkerBuffers &m, int k, int d) {
    return m.frac_d[(long long)k * 3 + d];
}
template <typename R> __device__ __forceinline__ R cell_offset(int o, R frac) {
    return ((R)o + R(0.5)) - frac;
}

template <typename R>
__device__ __forceinline__ R warp_sum_r(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R> __device__ __forceinline__ R rdiv(R a, R b);
template <> __device__ __forceinline__ float rdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double rdiv<double>(double a, double b) { return a / b; }

// Phi_k(j) for the support cell `l` of 3^DIM (offsets in z, y, x order)
template <int DIM, typename R>
__device__ __forceinline__ R lane_weight(const R *fr, const int *ck, int l, int *cell) {
    const int o[3] = {l % 3 - 1, (l / 3) % 3 - 1, DIM == 3 ? l / 9 - 1 : 0};
    R w = R(1);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        cell[d] = ck[d] + o[d];
        w *= phi_r<R>(cell_offset<R>(o[d], fr[d]));
    }
    if (DIM == 2) cell[2] = 0;
    return w;
}

// Visit, in sorted bin order (ascending marker index), the markers owned by
// the neighbour (c + (ox, oy, oz)) of cell c.  Global-memory form.
template <int DIM, typename R, typename F>
__device__ __forceinline__ bool gather_cell(const GridParams &g, const MarkerBuffers &m,
                                            const unsigned *__restrict__ keys,
                                            const int *__restrict__ perm, const int c[3], int ox,
                                            int oy, int oz, F &&visit) {
    const int x = c[0] + ox, y = c[1] + oy, z = c[2] + oz;
    if (x < 0 || y < 0 || x >= g.n[0] || y >= g.n[1]) return false;
    if (DIM == 3 && (z < 0 || z >= g.n[2])) return false;
    const unsigned key = cell_key(g, x, y, z);
    const int tc = (int)(key / (unsigned)g.cells_per_tile);
    int lo = m.tile_off[tc], hi = m.tile_off[tc + 1];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    const int end = m.tile_off[tc + 1];
    const int oo[3] = {-ox, -oy, -oz};   // cell c seen from owner cell (x, y, z)
    bool any = false;
    for (int p = lo; p < end && keys[p] == key; ++p) {
        const int k = perm[p];
        if (!in_bounds(k, m.ns, m.err)) continue;
        R w = R(1);
#pragma unroll
        for (int d = 0; d < DIM; ++d) w *= phi_r<R>(cell_offset<R>(oo[d], marker_frac<R>(m, k, d)));
        visit(k, w);
        any = true;
    }
    return any;
}

// Visit, in a fixed order, every marker whose support contains cell c:
// neighbour owner cells (z, y, x offsets ascending), then sorted bin order
// (ascending marker index within a cell).  Global-memory form.
template <int DIM, typename R, typename F>
__device__ __forceinline__ bool gather_markers(const GridParams &g, const MarkerBuffers &m,
                                               const unsigned *__restrict__ keys,
                                               const int *__restrict__ perm, const int c[3],
                                               F &&visit) {
    bool any = false;
    const int zr = DIM == 3 ? 1 : 0;
    for (int oz = -zr; oz <= zr; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox)
                any |= gather_cell<DIM, R>(g, m, keys, perm, c, ox, oy, oz, visit);
    return any;
}

}  // namespace ibmk
