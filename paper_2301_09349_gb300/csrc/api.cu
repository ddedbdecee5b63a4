// C ABI of the library (include/ibm.h): handle management, argument checks,
// workspace carving, marker set-up (dedup of Sec. 3.1, bins, quadrature) and
// the stream-ordered step driver.  No exception crosses the boundary and no
// device memory is allocated here: every device buffer is a slice of the
// caller's workspace.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/ibm.h"
#include <nvtx3/nvToolsExt.h>
#include "device_table.h"
#include "handle.h"
#include "internal.h"

using namespace ibmk;

namespace {

thread_local std::string g_create_error;

// upper bound of the persistent marker-kernel grids (4 CTAs per SM)
constexpr int kMaxPersistentCtas = 4096;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t state_bytes(const ibm_grid_desc &d) {
    long long N = 1;
    for (int i = 0; i < d.dim; ++i) N *= d.n[i];
    return (size_t)N * (d.dim + 2) * d.fp_bytes;
}

const char *check_desc(const ibm_grid_desc *d) {
    if (!d) return "null grid description";
    if (d->dim != 2 && d->dim != 3) return "dim must be 2 or 3";
    for (int i = 0; i < d->dim; ++i) {
        if (d->n[i] < 4) return "each axis needs at least 4 cells";
        if (d->tile[i] < 1 || d->tile[i] > 64) return "tile sizes must be in [1, 64]";
    }
    if (d->dim == 2 && (d->n[2] != 1 || d->tile[2] != 1)) return "2D grids need n[2] = tile[2] = 1";
    if (d->fp_bytes != 4 && d->fp_bytes != 8) return "fp_bytes must be 4 or 8";
    if (!(d->h > 0.0) || !isfinite(d->h)) return "spacing h must be positive";
    if (!(d->gamma > 1.0) || !(d->Mach > 0.0) || !(d->Pr > 0.0) || !(d->cfl > 0.0))
        return "gamma > 1, Mach > 0, Pr > 0, cfl > 0 required";
    if (!(d->sutherland_S >= 0.0)) return "Sutherland constant must be >= 0";
    if (!(d->D > 0.0)) return "reference length D must be positive";
    for (int i = 0; i < 6; ++i) {
        if (d->bc[i] < 0 || d->bc[i] > 3) return "unknown boundary condition";
        if (i >= 2 * d->dim) continue;
    }
    for (int a = 0; a < d->dim; ++a)
        if ((d->bc[2 * a] == IBM_BC_PERIODIC) != (d->bc[2 * a + 1] == IBM_BC_PERIODIC))
            return "periodic boundaries must be paired on an axis";
    long long N = 1;
    for (int i = 0; i < d->dim; ++i) N *= d->n[i];
    if (N * (d->dim + 2) > (1ll << 40)) return "grid too large";
    long long tiles = 1, cpt = 1;
    for (int i = 0; i < d->dim; ++i) {
        tiles *= (d->n[i] + d->tile[i] - 1) / d->tile[i];
        cpt *= d->tile[i];
    }
    if (tiles * cpt >= (1ll << 32)) return "tile key space exceeds 32 bits";
    size_t staged = (size_t)(d->tile[0] + 2) * (d->tile[1] + 2) * (d->dim == 3 ? d->tile[2] + 2 : 1);
    if (staged * (d->dim + 2) * sizeof(double) > 160 * 1024) return "tile too large for staging";
    if (d->energy_reading != 0 && d->energy_reading != 1) return "energy_reading must be 0 or 1";
    if (d->forcing_per_stage != 0 && d->forcing_per_stage != 1)
        return "forcing_per_stage must be 0 or 1";
    return nullptr;
}

GridParams make_params(const ibm_grid_desc &d) {
    GridParams g{};
    g.dim = d.dim;
    g.N = 1;
    for (int i = 0; i < 3; ++i) {
        g.n[i] = i < d.dim ? d.n[i] : 1;
        g.lo[i] = d.lo[i];
        g.tile[i] = i < d.dim ? d.tile[i] : 1;
        g.ntile[i] = (g.n[i] + g.tile[i] - 1) / g.tile[i];
    }
    for (int i = 0; i < d.dim; ++i) g.N *= d.n[i];
    g.h = d.h;
    g.inv_h = 1.0 / d.h;
    g.gamma = d.gamma;
    g.Pr = d.Pr;
    g.Re = d.Re;
    g.Mach = d.Mach;
    g.S = d.sutherland_S;
    g.cfl = d.cfl;
    g.R = 1.0 / (d.gamma * d.Mach * d.Mach);
    g.cv = g.R / (d.gamma - 1.0);
    g.cp = d.gamma * g.cv;
    g.mu_inf = d.Re > 0.0 ? 1.0 / d.Re : 0.0;
    g.kvisc = std::max(4.0 / 3.0, d.gamma / d.Pr);
    g.p_inf = 1.0 / (d.gamma * d.Mach * d.Mach);
    for (int i = 0; i < 6; ++i) g.bc[i] = d.bc[i];
    g.n_tiles = g.ntile[0] * g.ntile[1] * g.ntile[2];
    g.cells_per_tile = g.tile[0] * g.tile[1] * g.tile[2];
    g.energy_reading = d.energy_reading;
    g.forcing_per_stage = d.forcing_per_stage;
    g.f = float_consts(g);
    return g;
}

// Carves the workspace; with base == nullptr only measures it.
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};

void layout(ibm_grid *g, const ibm_grid_desc &d, int cap, char *base, size_t *total) {
    GridParams gp = make_params(d);
    Carver c{base};
    const size_t sb = state_bytes(d);
    void *U0 = c.take<char>(sb);
    void *U1 = c.take<char>(sb);
    void *L = c.take<char>(sb);
    const size_t nbm = fluid_blockmax_count(gp, d.fp_bytes);
    double *blockmax = c.take<double>(nbm);
    unsigned *counter = c.take<unsigned>(4);
    double *scal = c.take<double>(8);
    int *err = c.take<int>(4);
    const int dim = d.dim;
    MarkerBuffers m{};
    m.X0 = c.take<double>((size_t)cap * dim);
    m.X = c.take<double>((size_t)cap * dim);
    m.Ub0 = c.take<double>((size_t)cap * dim);
    m.Ub = c.take<double>((size_t)cap * dim);
    m.Tw = c.take<double>(cap);
    m.eps = c.take<double>(cap);
    m.cell = c.take<int>((size_t)cap * 3);
    m.frac_d = c.take<double>((size_t)cap * 3);
    m.frac_f = c.take<float>((size_t)cap * 3);
    m.wphi = c.take<double>((size_t)cap * 9);
    m.rhoL = c.take<double>(cap);
    m.G = c.take<double>((size_t)cap * dim);
    m.H = c.take<double>(cap);
    m.cp = c.take<double>(cap);
    m.keys[0] = c.take<unsigned>(cap);
    m.keys[1] = c.take<unsigned>(cap);
    m.perm[0] = c.take<int>(cap);
    m.perm[1] = c.take<int>(cap);
    m.tile_off = c.take<int>((size_t)gp.n_tiles + 1);
    m.occ_flag = c.take<int>(gp.n_tiles);
    m.band_flag = c.take<int>(gp.n_tiles);
    m.occ_list = c.take<int>(gp.n_tiles);
    m.band_list = c.take<int>(gp.n_tiles);
    m.counts = c.take<int>(4);
    m.sums = c.take<double>(16);
    m.bandmax = c.take<double>(kMaxPersistentCtas);
    m.finpart = c.take<double>((size_t)kFinishCtas * 5);
    m.gs = c.take<double>((size_t)cap * 4);
    m.sp_cap = (dim == 3 ? 27 : 9) * (cap > 0 ? cap : 1);
    m.sp_cell = c.take<SpreadCell>((size_t)m.sp_cap);
    m.sp_k = c.take<int>((size_t)m.sp_cap);
    m.sp_w = c.take<double>((size_t)m.sp_cap);
    m.band_bits = c.take<unsigned>((size_t)(gp.N / 32 + 1));
    m.t = c.take<double>(1);
    m.steps = c.take<long long>(1);
    QuadBuffers q{};
    q.width = quad_row_width(dim);
    q.cap = cap > 0 ? cap : 1;
    q.cnt = c.take<int>(cap);
    q.col = c.take<int>((size_t)q.width * q.cap);
    q.val = c.take<double>((size_t)q.width * q.cap);
    q.diag = c.take<double>(cap);
    q.r = c.take<double>(cap);
    q.z = c.take<double>(cap);
    q.p = c.take<double>(cap);
    q.q = c.take<double>(cap);
    q.iters = c.take<int>(2);
    q.resid = c.take<double>(1);
    *total = align_up(c.off, 256);
    if (!g) return;
    g->U[0] = U0;
    g->U[1] = U1;
    g->L = L;
    g->fb.blockmax = blockmax;
    g->fb.counter = counter;
    g->fb.dt = scal;
    g->fb.err = err;
    g->fb.band_bits = m.band_bits;
    g->scratch_d = scal;
    g->err_d = err;
    m.err = err;
    m.ns = 0;
    g->mb = m;
    g->qb = q;
}

ibm_status fail(ibm_grid *g, ibm_status st, const std::string &msg) {
    if (g) g->err = msg;
    else g_create_error = msg;
    return st;
}

ibm_status cuda_fail(ibm_grid *g, cudaError_t e, const char *where) {
    return fail(g, IBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CU(call, where)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return cuda_fail(g, _e, where); \
    } while (0)

// Synchronize and decode the device error word.
ibm_status check_device(ibm_grid *g) {
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    int e = 0;
    CU(cudaMemcpy(&e, g->err_d, sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (e & ERR_NONFINITE) return fail(g, IBM_ERR_NONFINITE, "non-finite or non-positive state");
    if (e & ERR_NOCONV) return fail(g, IBM_ERR_NOCONV, "quadrature A eps = 1 did not converge");
    if (e & ERR_MARKER_RANGE)
        return fail(g, IBM_ERR_ARG, "a marker left the admissible region (2 cells from the edges)");
    if (e & ERR_CAPACITY) return fail(g, IBM_ERR_WORKSPACE, "quadrature row capacity exceeded");
    if (e & ERR_TIMEOUT) return fail(g, IBM_ERR_TIMEOUT, "a bounded device wait gave up");
    if (e & ERR_BOUNDS)
        return fail(g, IBM_ERR_BOUNDS, "a kernel met an index outside its array (checked build)");
    return IBM_OK;
}

int persistent_ctas(const ibm_grid *g) {
    return std::min(kMaxPersistentCtas, std::max(1, g->n_sm) * 4);
}

// Event pair around a kernel group (no-op unless profiling is on).
// Kernel groups of a step as named NVTX ranges (host-side markers for a
// timeline profiler; the header-only NVTX v3 API costs nothing when no tool
// is attached), opened and closed with the event pair of the group.
// (indexed by IBM_PROF_*)
const char *const kProfNames[IBM_PROF_GROUPS] = {"ibm: fluid stage 1", "ibm: fluid stage 2",
                                                 "ibm: moving markers (bins, weights)",
                                                 "ibm: interpolation + forcing",
                                                 "ibm: spreading + forced update",
                                                 "ibm: force sums, next dt"};

cudaError_t prof_begin(ibm_grid *g, int group, int launches, long *rec,
                       cudaStream_t on = nullptr) {
    *rec = -1;
    if (!g->prof) return cudaSuccess;
    nvtxRangePushA(kProfNames[group]);
    while (g->ev_pool.size() < g->ev_used + 2) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        g->ev_pool.push_back(e);
    }
    const size_t i = g->ev_used;
    g->ev_used += 2;
    g->recs.push_back({group, launches, i});
    *rec = (long)g->recs.size() - 1;
    return cudaEventRecord(g->ev_pool[i], on ? on : g->stream);
}

cudaError_t prof_end(ibm_grid *g, long rec, cudaStream_t on = nullptr) {
    if (rec < 0) return cudaSuccess;
    const cudaError_t e = cudaEventRecord(g->ev_pool[g->recs[rec].ev + 1], on ? on : g->stream);
    nvtxRangePop();
    return e;
}

// fold recorded pairs into the totals (requires the stream to be idle)
cudaError_t prof_collect(ibm_grid *g) {
    for (const auto &r : g->recs) {
        float ms = 0.0f;
        cudaError_t e = cudaEventElapsedTime(&ms, g->ev_pool[r.ev], g->ev_pool[r.ev + 1]);
        if (e != cudaSuccess) return e;
        g->prof_ms[r.group] += ms;
        g->prof_n[r.group] += r.launches;
    }
    g->recs.clear();
    g->ev_used = 0;
    return cudaSuccess;
}

// Marker pipeline on the device: bins, then quadrature (warm start if asked).
ibm_status rebuild_markers(ibm_grid *g, int warm, cudaStream_t s) {
    CU(launch_bin(g->gp, g->mb, s), "bin markers");
    CU(launch_band_mask(g->gp, g->mb, s), "band mask");
    if (g->mb.ns > 0)
        CU(launch_quadrature(g->gp, g->mb, g->qb, g->cg_tol, g->cg_maxit, warm, s), "quadrature");
    // static markers: their spreading operator, once per marker set
    g->mb.sp_ready = 0;
    if (!g->moving && g->mb.ns > 0) {
        CU(launch_spread_build(g->gp, g->desc.fp_bytes, g->mb, persistent_ctas(g), s),
           "spreading operator");
        g->mb.sp_ready = 1;
    }
    return IBM_OK;
}
ibm_status rebuild_markers(ibm_grid *g, int warm) { return rebuild_markers(g, warm, g->stream); }

}  // namespace

namespace ibmk {
cudaError_t func_smem_attr(const void *func, size_t smem, int carveout) {
    if (smem <= 48 * 1024 && carveout < 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static DeviceAttrTable table;
    const int rc = table.ensure(func, dev, smem, [&]() -> int {
        cudaError_t r = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (r == cudaSuccess && carveout >= 0)
            r = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     carveout);
        return (int)r;
    });
    return (cudaError_t)rc;
}

GridParams params_from_desc(const ibm_grid_desc &d) { return make_params(d); }
const char *desc_problem(const ibm_grid_desc *d) { return check_desc(d); }
void set_handle_free_error(const char *msg) { g_create_error = msg; }

// Eq. Bulk: F_body = -h^d sum_k eps~_k F_k, Q_body = h^d sum_k eps~_k Q_k with
// F = G/dt, Q = H/dt; coefficients and Nu as documented in include/ibm.h.
void forces_from_sums(const ibm_grid *g, const double *sums, double force[3], double *heat_rate,
                      double *Cd, double *Cl, double *Nu) {
    const int dim = g->desc.dim;
    const double hd = pow(g->desc.h, dim);
    const double dt = sums[4];
    double f[3] = {0, 0, 0}, q = 0.0;
    if (dt > 0.0) {
        for (int d = 0; d < dim; ++d) f[d] = -hd * sums[d] / dt;
        q = hd * sums[3] / dt;
    }
    const double pi = 3.14159265358979323846;
    const double Dr = g->desc.D;
    const double lref = dim == 2 ? Dr : pi * Dr * Dr / 4.0;
    const double As = dim == 2 ? pi * Dr : pi * Dr * Dr;
    const double lam_inf = g->desc.Re > 0.0 ? g->gp.mu_inf * g->gp.cp / g->desc.Pr : 0.0;
    double tw = 0.0;
    for (double v : g->Tw_h) tw += v;
    const double dT = (g->Tw_h.empty() ? 0.0 : tw / g->Tw_h.size()) - 1.0;
    if (force)
        for (int d = 0; d < 3; ++d) force[d] = f[d];
    if (heat_rate) *heat_rate = q;
    if (Cd) *Cd = 2.0 * f[0] / lref;
    if (Cl) *Cl = 2.0 * f[1] / lref;
    if (Nu) *Nu = (lam_inf > 0.0 && dT != 0.0) ? q * Dr / (lam_inf * As * dT) : NAN;
}
}  // namespace ibmk

extern "C" {

size_t ibm_workspace_bytes(const ibm_grid_desc *desc, int max_markers) {
    if (check_desc(desc) || max_markers < 0) return 0;
    size_t total = 0;
    layout(nullptr, *desc, max_markers, nullptr, &total);
    return total;
}

ibm_status ibm_create_grid(const ibm_grid_desc *desc, int max_markers, void *dev_workspace,
                           size_t bytes, void *stream, ibm_grid **out) {
    if (!out) return fail(nullptr, IBM_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    if (const char *why = check_desc(desc)) return fail(nullptr, IBM_ERR_ARG, why);
    if (max_markers < 0) return fail(nullptr, IBM_ERR_ARG, "negative marker capacity");
    if (!dev_workspace) return fail(nullptr, IBM_ERR_ARG, "null workspace");
    if (((uintptr_t)dev_workspace) % 256 != 0)
        return fail(nullptr, IBM_ERR_ARG, "workspace must be 256-byte aligned");
    size_t need = ibm_workspace_bytes(desc, max_markers);
    if (bytes < need)
        return fail(nullptr, IBM_ERR_WORKSPACE,
                    "workspace too small: need " + std::to_string(need) + " bytes");
    ibm_grid *g = new (std::nothrow) ibm_grid();
    if (!g) return fail(nullptr, IBM_ERR_ARG, "host allocation failed");
    g->desc = *desc;
    g->gp = make_params(*desc);
    g->stream = (cudaStream_t)stream;
    g->max_markers = max_markers;
    g->ws = (char *)dev_workspace;
    g->ws_bytes = bytes;
    size_t total = 0;
    layout(g, *desc, max_markers, g->ws, &total);
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) {
        cudaPointerAttributes pa;
        e = cudaPointerGetAttributes(&pa, dev_workspace);
        if (e == cudaSuccess && pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) {
            delete g;
            return fail(nullptr, IBM_ERR_ARG, "workspace is not device memory");
        }
    }
    // zero the small control block (counters, error word, time, sums)
    if (e == cudaSuccess) e = cudaMemsetAsync(g->fb.counter, 0, 4 * sizeof(unsigned), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->err_d, 0, 4 * sizeof(int), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->scratch_d, 0, 8 * sizeof(double), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mb.sums, 0, 16 * sizeof(double), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mb.t, 0, sizeof(double), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mb.steps, 0, sizeof(long long), g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->mb.counts, 0, 4 * sizeof(int), g->stream);
    if (e == cudaSuccess) e = launch_bin(g->gp, g->mb, g->stream);  // empty bins
    if (e == cudaSuccess) e = launch_band_mask(g->gp, g->mb, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("CUDA: ") + cudaGetErrorString(e);
        delete g;
        return IBM_ERR_CUDA;
    }
    *out = g;
    return IBM_OK;
}

ibm_status ibm_destroy(ibm_grid *g) {
    if (!g) return IBM_ERR_ARG;
    if (g->in_batch) return fail(g, IBM_ERR_ARG, "this grid belongs to a batch: destroy the batch");
    delete g;
    return IBM_OK;
}

const char *ibm_last_error(const ibm_grid *g) {
    return g ? g->err.c_str() : g_create_error.c_str();
}

ibm_status ibm_set_state(ibm_grid *g, const void *U) {
    if (!g) return IBM_ERR_ARG;
    if (!U) return fail(g, IBM_ERR_ARG, "null state pointer");
    CU(cudaMemcpyAsync(g->U[g->cur], U, state_bytes(g->desc), cudaMemcpyDeviceToDevice, g->stream),
       "set_state copy");
    CU(launch_dt_init(g->gp, g->desc.fp_bytes, g->U[g->cur], g->fb, g->stream), "initial dt");
    CU(cudaMemsetAsync(g->mb.t, 0, sizeof(double), g->stream), "reset time");
    CU(cudaMemsetAsync(g->mb.steps, 0, sizeof(long long), g->stream), "reset steps");
    g->has_state = true;
    g->rec_steps = 0;
    return IBM_OK;
}

ibm_status ibm_set_state_host(ibm_grid *g, const void *U_host) {
    if (!g) return IBM_ERR_ARG;
    if (!U_host) return fail(g, IBM_ERR_ARG, "null state pointer");
    CU(cudaMemcpyAsync(g->U[g->cur], U_host, state_bytes(g->desc), cudaMemcpyHostToDevice,
                       g->stream),
       "set_state_host copy");
    CU(launch_dt_init(g->gp, g->desc.fp_bytes, g->U[g->cur], g->fb, g->stream), "initial dt");
    CU(cudaMemsetAsync(g->mb.t, 0, sizeof(double), g->stream), "reset time");
    CU(cudaMemsetAsync(g->mb.steps, 0, sizeof(long long), g->stream), "reset steps");
    g->has_state = true;
    g->rec_steps = 0;
    return IBM_OK;
}

ibm_status ibm_get_state(ibm_grid *g, void *U) {
    if (!g) return IBM_ERR_ARG;
    if (!U) return fail(g, IBM_ERR_ARG, "null state pointer");
    if (!g->has_state) return fail(g, IBM_ERR_STATE, "no state set");
    CU(cudaMemcpyAsync(U, g->U[g->cur], state_bytes(g->desc), cudaMemcpyDeviceToDevice, g->stream),
       "get_state copy");
    return check_device(g);
}

ibm_status ibm_get_state_host(ibm_grid *g, void *U_host) {
    if (!g) return IBM_ERR_ARG;
    if (!U_host) return fail(g, IBM_ERR_ARG, "null state pointer");
    if (!g->has_state) return fail(g, IBM_ERR_STATE, "no state set");
    CU(cudaMemcpyAsync(U_host, g->U[g->cur], state_bytes(g->desc), cudaMemcpyDeviceToHost,
                       g->stream),
       "get_state_host copy");
    return check_device(g);
}

ibm_status ibm_set_markers(ibm_grid *g, int n, const double *X0, const double *Ub,
                           const double *Tw, const ibm_motion *motion, int dedup, int *n_kept) {
    if (!g) return IBM_ERR_ARG;
    if (n < 0) return fail(g, IBM_ERR_ARG, "negative marker count");
    if (n > 0 && (!X0 || !Tw)) return fail(g, IBM_ERR_ARG, "null marker arrays");
    const int dim = g->desc.dim;
    if (motion) {
        if (motion->axis < 0 || motion->axis >= dim || !isfinite(motion->amp) ||
            !isfinite(motion->freq))
            return fail(g, IBM_ERR_ARG, "invalid motion");
    }
    // owner cells and the admissible region (support + MUSCL halo inside)
    std::vector<long long> cell((size_t)n);
    std::vector<double> dist((size_t)n);
    for (int k = 0; k < n; ++k) {
        long long key = 0;
        double dd = 0.0;
        for (int d = dim - 1; d >= 0; --d) {
            const double x = X0[(size_t)k * dim + d];
            if (!isfinite(x)) return fail(g, IBM_ERR_ARG, "non-finite marker position");
            const double c = floor((x - g->desc.lo[d]) / g->desc.h);
            if (c < 2.0 || c > (double)(g->desc.n[d] - 3))
                return fail(g, IBM_ERR_ARG, "marker " + std::to_string(k) +
                                                " closer than two cells to the domain edge");
            key = key * g->desc.n[d] + (long long)c;
            const double dx = x - (g->desc.lo[d] + (c + 0.5) * g->desc.h);
            dd += dx * dx;
        }
        if (!isfinite(Tw[k]) || Tw[k] <= 0.0)
            return fail(g, IBM_ERR_ARG, "wall temperature must be finite and positive");
        if (Ub)
            for (int d = 0; d < dim; ++d)
                if (!isfinite(Ub[(size_t)k * dim + d]))
                    return fail(g, IBM_ERR_ARG, "non-finite body velocity");
        cell[k] = key;
        dist[k] = dd;
    }
    // Sec. 3.1: one marker per mesh element, the one closest to its centre
    std::vector<int> keep;
    if (dedup) {
        std::vector<int> order((size_t)n);
        for (int k = 0; k < n; ++k) order[k] = k;
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            if (cell[a] != cell[b]) return cell[a] < cell[b];
            if (dist[a] != dist[b]) return dist[a] < dist[b];
            return a < b;
        });
        for (int i = 0; i < n; ++i)
            if (i == 0 || cell[order[i]] != cell[order[i - 1]]) keep.push_back(order[i]);
        std::sort(keep.begin(), keep.end());
    } else {
        keep.resize((size_t)n);
        for (int k = 0; k < n; ++k) keep[k] = k;
    }
    const int ns = (int)keep.size();
    if (ns > g->max_markers)
        return fail(g, IBM_ERR_WORKSPACE, "kept markers " + std::to_string(ns) +
                                              " exceed capacity " + std::to_string(g->max_markers));
    std::vector<double> Xh((size_t)ns * dim), Ubh((size_t)ns * dim, 0.0), Twh((size_t)ns);
    for (int i = 0; i < ns; ++i) {
        const int k = keep[i];
        for (int d = 0; d < dim; ++d) {
            Xh[(size_t)i * dim + d] = X0[(size_t)k * dim + d];
            if (Ub) Ubh[(size_t)i * dim + d] = Ub[(size_t)k * dim + d];
        }
        Twh[i] = Tw[k];
    }
    // the uploads read host vectors: wait for them before returning
    if (ns > 0) {
        const size_t bx = sizeof(double) * (size_t)ns * dim;
        CU(cudaMemcpyAsync(g->mb.X0, Xh.data(), bx, cudaMemcpyHostToDevice, g->stream), "upload X0");
        CU(cudaMemcpyAsync(g->mb.X, Xh.data(), bx, cudaMemcpyHostToDevice, g->stream), "upload X");
        CU(cudaMemcpyAsync(g->mb.Ub0, Ubh.data(), bx, cudaMemcpyHostToDevice, g->stream), "upload Ub0");
        CU(cudaMemcpyAsync(g->mb.Ub, Ubh.data(), bx, cudaMemcpyHostToDevice, g->stream), "upload Ub");
        CU(cudaMemcpyAsync(g->mb.Tw, Twh.data(), sizeof(double) * ns, cudaMemcpyHostToDevice,
                           g->stream),
           "upload Tw");
        CU(cudaMemsetAsync(g->mb.rhoL, 0, sizeof(double) * ns, g->stream), "clear rhoL");
        CU(cudaMemsetAsync(g->mb.G, 0, bx, g->stream), "clear G");
        CU(cudaMemsetAsync(g->mb.H, 0, sizeof(double) * ns, g->stream), "clear H");
    }
    CU(cudaMemsetAsync(g->mb.sums, 0, 16 * sizeof(double), g->stream), "clear sums");
    g->mb.ns = ns;
    g->kept = keep;
    g->Tw_h = Twh;
    ++g->marker_gen;
    g->drop_graphs();
    g->rec_steps = 0;
    g->moving = motion != nullptr;
    if (motion) g->motion = *motion;
    ibm_status st = rebuild_markers(g, 0);
    if (st == IBM_OK) st = check_device(g);
    if (st != IBM_OK) {
        g->mb.sp_ready = 0;
        return st;
    }
    if (n_kept) *n_kept = ns;
    return IBM_OK;
}

ibm_status ibm_set_quadrature(ibm_grid *g, double tol, int maxit) {
    if (!g) return IBM_ERR_ARG;
    if (!(tol > 0.0 && tol < 1.0) || maxit < 1)
        return fail(g, IBM_ERR_ARG, "quadrature tolerance must be in (0, 1) and maxit >= 1");
    g->cg_tol = tol;
    g->cg_maxit = maxit;
    return IBM_OK;
}

ibm_status ibm_set_wall_temperature(ibm_grid *g, const double *Tw) {
    if (!g) return IBM_ERR_ARG;
    if (g->mb.ns > 0 && !Tw) return fail(g, IBM_ERR_ARG, "null wall temperatures");
    for (int k = 0; k < g->mb.ns; ++k)
        if (!isfinite(Tw[k]) || Tw[k] <= 0.0)
            return fail(g, IBM_ERR_ARG, "wall temperature must be finite and positive");
    if (g->mb.ns > 0) {
        g->Tw_h.assign(Tw, Tw + g->mb.ns);
        CU(cudaMemcpyAsync(g->mb.Tw, Tw, sizeof(double) * g->mb.ns, cudaMemcpyHostToDevice,
                           g->stream),
           "upload Tw");
    }
    return IBM_OK;
}

}  // extern "C"

namespace {
// the side stream and fork/join events of the small-body marker pipeline
cudaError_t ensure_side(ibm_grid *g) {
    cudaError_t e = cudaSuccess;
    if (!g->side) e = cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&g->ev_fork, &g->ev_bins, &g->ev_quad})
        if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    return e;
}

// nsteps IBM steps launched on stream s (the handle's stream, or the private
// stream a graph is captured on)
ibm_status run_steps(ibm_grid *g, int nsteps, double dt_fixed, cudaStream_t s) {
    const int fpb = g->desc.fp_bytes;
    const int ctas = persistent_ctas(g);
    long rec;
    const int nb = (int)fluid_stage_blocks(g->gp, fpb);
    for (int step = 0; step < nsteps; ++step) {
        void *Un = g->U[g->cur];
        void *Us = g->U[1 - g->cur];
        void *U1 = g->L;
        if (g->recording && g->rec_steps % g->adj.every == 0)
            CU(cudaMemcpyAsync((char *)g->adj.ckpt +
                                   (size_t)(g->rec_steps / g->adj.every) * align_up(state_bytes(g->desc), 256),
                               Un, state_bytes(g->desc), cudaMemcpyDeviceToDevice, s),
               "checkpoint");
        // A small moving body's marker pipeline (positions at t^{n+1}, bins,
        // forced cells, weights) depends only on the time and the step
        // size: it runs on a side stream beside stage 1; stage 2 (which
        // skips the forced cells) waits for the bins, the interpolation for
        // the weights.
        const bool fork = g->moving && g->mb.ns > 0 && g->mb.ns <= kSmallRebuildNs;
        if (fork) {
            CU(ensure_side(g), "side stream");
            CU(cudaEventRecord(g->ev_fork, s), "fork");
            CU(cudaStreamWaitEvent(g->side, g->ev_fork, 0), "fork");
            CU(prof_begin(g, IBM_PROF_MARKERS, 3, &rec, g->side), "profile");
            CU(launch_small_rebuild(g->gp, g->mb, g->motion.amp, g->motion.freq, g->motion.axis,
                                    g->fb.dt, dt_fixed, g->side),
               "motion + bins");
            CU(cudaEventRecord(g->ev_bins, g->side), "bins");
            CU(launch_quadrature(g->gp, g->mb, g->qb, g->cg_tol, g->cg_maxit, 1, g->side, 1),
               "quadrature");
            CU(prof_end(g, rec, g->side), "profile");
            CU(cudaEventRecord(g->ev_quad, g->side), "weights");
        }
        CU(prof_begin(g, IBM_PROF_STAGE1, 1, &rec), "profile");
        CU(launch_stage1(g->gp, fpb, Un, U1, g->fb, dt_fixed, s), "stage 1");
        CU(prof_end(g, rec), "profile");
        if (fork) {
            CU(cudaStreamWaitEvent(s, g->ev_bins, 0), "join bins");
        } else if (g->moving && g->mb.ns > 0) {
            CU(prof_begin(g, IBM_PROF_MARKERS, 9, &rec), "profile");
            CU(launch_motion(g->gp, g->mb, g->motion.amp, g->motion.freq, g->motion.axis,
                             g->fb.dt, dt_fixed, s),
               "motion");
            ibm_status st = rebuild_markers(g, 1, s);
            if (st != IBM_OK) return st;
            CU(prof_end(g, rec), "profile");
        }
        bool joined = !fork;
        if (g->desc.forcing_per_stage && g->mb.ns > 0) {
            if (!joined) {
                CU(cudaStreamWaitEvent(s, g->ev_quad, 0), "join weights");
                joined = true;
            }
            // variant: the first stage is forced too; its sources are summed now
            CU(prof_begin(g, IBM_PROF_INTERP, 2, &rec), "profile");
            CU(launch_interp_force(g->gp, fpb, U1, g->mb, ctas, s), "interp/force (stage 1)");
            CU(launch_partial_sums(g->gp, g->mb, s), "stage-1 sums");
            CU(prof_end(g, rec), "profile");
            CU(prof_begin(g, IBM_PROF_SPREAD, 1, &rec), "profile");
            CU(launch_spread_apply(g->gp, fpb, U1, g->mb, ctas, s), "spread/apply (stage 1)");
            CU(prof_end(g, rec), "profile");
        }
        CU(prof_begin(g, IBM_PROF_STAGE2, 1, &rec), "profile");
        CU(launch_stage2(g->gp, fpb, Un, U1, Us, g->fb, dt_fixed, s), "stage 2");
        CU(prof_end(g, rec), "profile");
        if (!joined) CU(cudaStreamWaitEvent(s, g->ev_quad, 0), "join weights");
        // static markers: the finish runs inside the spreading launch
        const bool fused_finish = g->mb.ns > 0 && g->mb.sp_ready;
        if (g->mb.ns > 0) {
            CU(prof_begin(g, IBM_PROF_INTERP, 1, &rec), "profile");
            CU(launch_interp_force(g->gp, fpb, Us, g->mb, ctas, s), "interp/force");
            CU(prof_end(g, rec), "profile");
            const FinishArgs fa = finish_args(g->mb, g->fb, nb, dt_fixed);
            CU(prof_begin(g, IBM_PROF_SPREAD, 1, &rec), "profile");
            CU(launch_spread_apply(g->gp, fpb, Us, g->mb, ctas, s, fused_finish ? &fa : nullptr),
               "spread/apply");
            CU(prof_end(g, rec), "profile");
        }
        if (!fused_finish) {
            CU(prof_begin(g, IBM_PROF_FINISH, 1, &rec), "profile");
            CU(launch_finish(g->gp, g->mb, g->fb, nb, g->mb.ns > 0 ? ctas : 0, dt_fixed, s),
               "finish");
            CU(prof_end(g, rec), "profile");
        }
        if (g->recording) {
            CU(cudaMemcpyAsync(g->adj.dt_hist + g->rec_steps, g->mb.sums + 4, sizeof(double),
                               cudaMemcpyDeviceToDevice, s),
               "record dt");
            ++g->rec_steps;
        }
        g->cur = 1 - g->cur;
    }
    return IBM_OK;
}

}  // namespace

extern "C" {

ibm_status ibm_step(ibm_grid *g, int nsteps, double dt_fixed) {
    if (!g) return IBM_ERR_ARG;
    if (nsteps < 0 || !isfinite(dt_fixed)) return fail(g, IBM_ERR_ARG, "invalid step arguments");
    if (!g->has_state) return fail(g, IBM_ERR_STATE, "ibm_set_state must come first");
    if (g->recording) {
        if (g->moving && g->mb.ns > 0)
            return fail(g, IBM_ERR_UNSUPPORTED, "the adjoint records static markers only");
        if ((long long)g->rec_steps + nsteps > g->adj.max_steps)
            return fail(g, IBM_ERR_WORKSPACE, "more steps than the adjoint workspace records (" +
                                                  std::to_string(g->adj.max_steps) + ")");
    }
    // graphs: whole chunks of graph_steps steps (an even number, so the
    // buffers end where they started); not while profiling or recording
    const int k = g->graph_steps;
    if (k > 0 && !g->prof && !g->recording) {
        while (nsteps >= k) {
            const int p = g->cur;
            if (!g->gexec[p] || g->gexec_dt[p] != dt_fixed) {
                if (g->gexec[p]) cudaGraphExecDestroy(g->gexec[p]);
                g->gexec[p] = nullptr;
                if (!g->cap) CU(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking), "stream");
                CU(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeRelaxed), "begin capture");
                const ibm_status st = run_steps(g, k, dt_fixed, g->cap);
                cudaGraph_t graph = nullptr;
                const cudaError_t e = cudaStreamEndCapture(g->cap, &graph);
                g->cur = p;
                if (st != IBM_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (e != cudaSuccess) return cuda_fail(g, e, "end capture");
                const cudaError_t e2 = cudaGraphInstantiate(&g->gexec[p], graph, 0);
                cudaGraphDestroy(graph);
                if (e2 != cudaSuccess) {
                    g->gexec[p] = nullptr;
                    return cuda_fail(g, e2, "instantiate step graph");
                }
                g->gexec_dt[p] = dt_fixed;
            }
            CU(cudaGraphLaunch(g->gexec[p], g->stream), "graph launch");
            nsteps -= k;
        }
    }
    return run_steps(g, nsteps, dt_fixed, g->stream);
}

ibm_status ibm_step_graphs(ibm_grid *g, int steps_per_graph) {
    if (!g) return IBM_ERR_ARG;
    if (steps_per_graph < 0 || (steps_per_graph & 1))
        return fail(g, IBM_ERR_ARG, "steps_per_graph must be 0 or a positive even number");
    if (steps_per_graph != g->graph_steps) g->drop_graphs();
    g->graph_steps = steps_per_graph;
    return IBM_OK;
}

ibm_status ibm_profile(ibm_grid *g, int enable) {
    if (!g) return IBM_ERR_ARG;
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    g->recs.clear();
    g->ev_used = 0;
    for (int i = 0; i < IBM_PROF_GROUPS; ++i) {
        g->prof_ms[i] = 0.0;
        g->prof_n[i] = 0;
    }
    g->prof = enable != 0;
    return IBM_OK;
}

ibm_status ibm_profile_read(ibm_grid *g, double *ms, long long *launches) {
    if (!g) return IBM_ERR_ARG;
    CU(cudaStreamSynchronize(g->stream), "stream synchronize");
    CU(prof_collect(g), "event timing");
    for (int i = 0; i < IBM_PROF_GROUPS; ++i) {
        if (ms) ms[i] = g->prof_ms[i];
        if (launches) launches[i] = g->prof_n[i];
        g->prof_ms[i] = 0.0;
        g->prof_n[i] = 0;
    }
    return IBM_OK;
}

ibm_status ibm_sync(ibm_grid *g) {
    if (!g) return IBM_ERR_ARG;
    return check_device(g);
}

ibm_status ibm_forces_and_nusselt(ibm_grid *g, double force[3], double *heat_rate, double *Cd,
                                  double *Cl, double *Nu) {
    if (!g) return IBM_ERR_ARG;
    double sums[8] = {0};
    CU(cudaMemcpyAsync(sums, g->mb.sums, sizeof(sums), cudaMemcpyDeviceToHost, g->stream),
       "read force sums");
    ibm_status st = check_device(g);
    if (st != IBM_OK) return st;
    forces_from_sums(g, sums, force, heat_rate, Cd, Cl, Nu);
    return IBM_OK;
}


ibm_status ibm_get_markers(ibm_grid *g, double *X, double *eps_t, int *input_index) {
    if (!g) return IBM_ERR_ARG;
    const int ns = g->mb.ns, dim = g->desc.dim;
    if (ns > 0 && X)
        CU(cudaMemcpyAsync(X, g->mb.X, sizeof(double) * ns * dim, cudaMemcpyDeviceToHost, g->stream),
           "read X");
    if (ns > 0 && eps_t)
        CU(cudaMemcpyAsync(eps_t, g->mb.eps, sizeof(double) * ns, cudaMemcpyDeviceToHost, g->stream),
           "read eps");
    ibm_status st = check_device(g);
    if (st != IBM_OK) return st;
    if (input_index)
        for (int i = 0; i < ns; ++i) input_index[i] = g->kept[i];
    return IBM_OK;
}

ibm_status ibm_get_marker_forcing(ibm_grid *g, double *rhoL, double *F, double *Q) {
    if (!g) return IBM_ERR_ARG;
    const int ns = g->mb.ns, dim = g->desc.dim;
    double dt = 0.0;
    CU(cudaMemcpyAsync(&dt, g->mb.sums + 4, sizeof(double), cudaMemcpyDeviceToHost, g->stream),
       "read dt");
    if (ns > 0 && rhoL)
        CU(cudaMemcpyAsync(rhoL, g->mb.rhoL, sizeof(double) * ns, cudaMemcpyDeviceToHost, g->stream),
           "read rhoL");
    if (ns > 0 && F)
        CU(cudaMemcpyAsync(F, g->mb.G, sizeof(double) * ns * dim, cudaMemcpyDeviceToHost, g->stream),
           "read G");
    if (ns > 0 && Q)
        CU(cudaMemcpyAsync(Q, g->mb.H, sizeof(double) * ns, cudaMemcpyDeviceToHost, g->stream),
           "read H");
    ibm_status st = check_device(g);
    if (st != IBM_OK) return st;
    const double a = dt > 0.0 ? 1.0 / dt : 0.0;
    if (F)
        for (int i = 0; i < ns * dim; ++i) F[i] *= a;
    if (Q)
        for (int i = 0; i < ns; ++i) Q[i] *= a;
    return IBM_OK;
}

ibm_status ibm_surface_pressure(ibm_grid *g, double *cp) {
    if (!g) return IBM_ERR_ARG;
    if (!g->has_state) return fail(g, IBM_ERR_STATE, "no state set");
    const int ns = g->mb.ns;
    if (ns > 0 && !cp) return fail(g, IBM_ERR_ARG, "null output");
    if (ns > 0) {
        CU(launch_surface_pressure(g->gp, g->desc.fp_bytes, g->U[g->cur], g->mb, g->stream),
           "surface pressure");
        CU(cudaMemcpyAsync(cp, g->mb.cp, sizeof(double) * ns, cudaMemcpyDeviceToHost, g->stream),
           "read cp");
    }
    return check_device(g);
}

ibm_status ibm_get_bins(ibm_grid *g, int *tile_off, int *perm, unsigned *keys, int *n_tiles) {
    if (!g) return IBM_ERR_ARG;
    const int ns = g->mb.ns;
    if (tile_off)
        CU(cudaMemcpyAsync(tile_off, g->mb.tile_off, sizeof(int) * (g->gp.n_tiles + 1),
                           cudaMemcpyDeviceToHost, g->stream),
           "read tile_off");
    if (ns > 0 && perm)
        CU(cudaMemcpyAsync(perm, g->mb.perm[g->mb.sorted], sizeof(int) * ns, cudaMemcpyDeviceToHost,
                           g->stream),
           "read perm");
    if (ns > 0 && keys)
        CU(cudaMemcpyAsync(keys, g->mb.keys[g->mb.sorted], sizeof(unsigned) * ns,
                           cudaMemcpyDeviceToHost, g->stream),
           "read keys");
    if (n_tiles) *n_tiles = g->gp.n_tiles;
    return check_device(g);
}

ibm_status ibm_get_time(ibm_grid *g, double *dt, double *t, long long *steps) {
    if (!g) return IBM_ERR_ARG;
    double dtv = 0.0, tv = 0.0;
    long long sv = 0;
    CU(cudaMemcpyAsync(&dtv, g->mb.sums + 4, sizeof(double), cudaMemcpyDeviceToHost, g->stream),
       "read dt");
    CU(cudaMemcpyAsync(&tv, g->mb.t, sizeof(double), cudaMemcpyDeviceToHost, g->stream), "read t");
    CU(cudaMemcpyAsync(&sv, g->mb.steps, sizeof(long long), cudaMemcpyDeviceToHost, g->stream),
       "read steps");
    ibm_status st = check_device(g);
    if (dt) *dt = dtv;
    if (t) *t = tv;
    if (steps) *steps = sv;
    return st;
}

ibm_status ibm_rhs(ibm_grid *g, const void *U, void *L) {
    if (!g) return IBM_ERR_ARG;
    if (!U || !L) return fail(g, IBM_ERR_ARG, "null buffer");
    CU(launch_rhs(g->gp, g->desc.fp_bytes, U, L, g->fb, g->stream), "rhs");
    return IBM_OK;
}

ibm_status ibm_interpolate(ibm_grid *g, const void *field, int nc, double *out) {
    if (!g) return IBM_ERR_ARG;
    if (!field || !out || nc < 1) return fail(g, IBM_ERR_ARG, "invalid interpolate arguments");
    CU(launch_interpolate_op(g->gp, g->desc.fp_bytes, field, nc, g->mb, out, g->stream),
       "interpolate");
    return IBM_OK;
}

ibm_status ibm_spread(ibm_grid *g, const double *R, int nc, void *out) {
    if (!g) return IBM_ERR_ARG;
    if (!R || !out || nc < 1) return fail(g, IBM_ERR_ARG, "invalid spread arguments");
    CU(launch_spread_op(g->gp, g->desc.fp_bytes, R, nc, g->mb, out, g->stream), "spread");
    return IBM_OK;
}

}  // extern "C"
