// Batches of independent 2D grids (include/ibm.h, "batches"): host side.
//
// Every case is an ordinary grid handle carved from the batch workspace; the
// batch adds device tables that let one kernel launch per stage serve all
// cases:
//   - BatchCase[2][ncases]: per case its parameters, state buffers (one table
//     per step parity, so Un and Us swap without a rewrite), step size, error
//     word, band mask and marker buffers;
//   - stage items (case, tile) in the tile numbering of the chosen shape, one
//     step-size maximum per item;
//   - marker items (case, marker) for the interpolation;
//   - band items (case, band-tile position) for the spreading, one maximum each.
// A step is five launches: stage 1, stage 2, interpolation + forcing,
// spreading + forced update, finish (one CTA per case: sums, time, next dt).
// Optionally the five are captured once per parity in a CUDA graph and
// replayed.  Each case's arithmetic is the single-grid kernels' own device
// code, so a batch step is bitwise a per-case ibm_step.
#include <math.h>
#include <cmath>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "handle.h"
#include "internal.h"

using namespace ibmk;

struct ibm_batch {
    int ncases = 0;
    int fp_bytes = 4;
    cudaStream_t stream = nullptr;   // all device work and graph launches
    cudaStream_t cap = nullptr;      // private stream, used only to capture graphs
    int n_sm = 0;
    std::vector<ibm_grid *> grids;

    // device tables (slices of the workspace)
    BatchCase *tbl[2] = {nullptr, nullptr};
    int2 *stage_items = nullptr;
    double *item_max = nullptr;
    int2 *band_items = nullptr;
    double *band_max = nullptr;
    int2 *mk_items = nullptr;
    double *save = nullptr;     // autotune: the last marker forcing of every case
    double *gather = nullptr;   // ncases * 8: force sums, dt, t and the error word
    // wall temperatures: ncases slots, then the values of all kept markers
    BatchTwSlot *tw_slots = nullptr;
    double *tw_vals = nullptr;
    std::vector<BatchTwSlot> tw_slots_h;   // what tw_slots holds on the device
    size_t stage_cap = 0, band_cap = 0, mk_cap = 0;

    // what the tables were built from
    bool built = false;
    int built_shape = -1;
    std::vector<int> tbl_cur;
    std::vector<long long> tbl_gen;
    int n_stage = 0, n_band = 0, n_mk = 0;
    size_t spread_smem = 0;
    bool spread_op = false;   // spreading through the cases' operators
    ibm_batch_tuning tune{0, 4, 1};

    // kernel timing (ibm_batch_profile): event pairs around each group;
    // steps are launched directly, not from graphs, while it is on
    struct ProfRec {
        int group;
        int launches;
        size_t ev;
    };
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> recs;
    double prof_ms[IBM_PROF_GROUPS] = {0};
    long long prof_n[IBM_PROF_GROUPS] = {0};

    // one captured step per parity
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    double exec_dt[2] = {0.0, 0.0};
    std::string err;

    void drop_graphs() {
        for (int p = 0; p < 2; ++p) {
            if (exec[p]) cudaGraphExecDestroy(exec[p]);
            exec[p] = nullptr;
        }
    }
    ~ibm_batch() {
        drop_graphs();
        for (ibm_grid *g : grids) {
            if (!g) continue;
            g->in_batch = false;
            ibm_destroy(g);
        }
        if (cap) cudaStreamDestroy(cap);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    }
};

namespace {

thread_local std::string g_batch_create_error;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

ibm_status fail(ibm_batch *b, ibm_status st, const std::string &msg) {
    if (b) b->err = msg;
    else g_batch_create_error = msg;
    return st;
}

#define BCU(call, where)                                                                    \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess)                                                              \
            return fail(b, IBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(_e)); \
    } while (0)

int tiles_of_shape(const ibm_grid_desc &d, int shape) {
    int bx = 0, by = 0;
    batch_tile_shape(shape, &bx, &by);
    return ((d.n[0] + bx - 1) / bx) * ((d.n[1] + by - 1) / by);
}

int marker_tiles(const ibm_grid_desc &d) {
    return ((d.n[0] + d.tile[0] - 1) / d.tile[0]) * ((d.n[1] + d.tile[1] - 1) / d.tile[1]);
}

struct BatchLayout {
    std::vector<size_t> case_off, case_bytes;
    size_t tbl = 0, stage_items = 0, item_max = 0, band_items = 0, band_max = 0, mk_items = 0,
           save = 0, gather = 0, tw = 0, total = 0;
    size_t stage_cap = 0, band_cap = 0, mk_cap = 0;
};

// Why the batch description is invalid, or nullptr.
const char *check_batch(int ncases, const ibm_grid_desc *descs, const int *max_markers,
                        ibm_status *st) {
    *st = IBM_ERR_ARG;
    if (ncases < 1 || ncases > (1 << 20)) return "ncases must be in [1, 2^20]";
    if (!descs) return "null descriptions";
    for (int c = 0; c < ncases; ++c) {
        const int mm = max_markers ? max_markers[c] : 0;
        if (mm < 0) return "negative marker capacity";
        if (ibm_workspace_bytes(&descs[c], mm) == 0) return "invalid grid description";
        if (descs[c].dim != 2) {
            *st = IBM_ERR_UNSUPPORTED;
            return "batches hold 2D grids only";
        }
        if (descs[c].forcing_per_stage) {
            *st = IBM_ERR_UNSUPPORTED;
            return "batches force once per step (forcing_per_stage = 0)";
        }
        if (descs[c].fp_bytes != descs[0].fp_bytes) {
            *st = IBM_ERR_UNSUPPORTED;
            return "all cases of a batch need the same fp_bytes";
        }
    }
    return nullptr;
}

BatchLayout batch_layout(int ncases, const ibm_grid_desc *descs, const int *max_markers) {
    BatchLayout L;
    size_t off = 0;
    for (int c = 0; c < ncases; ++c) {
        const int mm = max_markers ? max_markers[c] : 0;
        const size_t wb = ibm_workspace_bytes(&descs[c], mm);
        L.case_off.push_back(off);
        L.case_bytes.push_back(wb);
        off = align_up(off + wb, 256);
        int most = 0;
        for (int s = 0; s < kBatchShapes; ++s) most = std::max(most, tiles_of_shape(descs[c], s));
        L.stage_cap += most;
        // band items: band tiles, or runs of 32 forced cells (at most 3^2 per marker)
        L.band_cap += std::max(marker_tiles(descs[c]), (9 * mm + 31) / 32);
        L.mk_cap += mm;
    }
    auto take = [&](size_t bytes) {
        off = align_up(off, 256);
        const size_t at = off;
        off += bytes > 0 ? bytes : 1;
        return at;
    };
    L.tbl = take(2 * sizeof(BatchCase) * (size_t)ncases);
    L.stage_items = take(sizeof(int2) * L.stage_cap);
    L.item_max = take(sizeof(double) * L.stage_cap);
    L.band_items = take(sizeof(int2) * L.band_cap);
    L.band_max = take(sizeof(double) * L.band_cap);
    L.mk_items = take(sizeof(int2) * L.mk_cap);
    L.save = take(sizeof(double) * 4 * L.mk_cap);
    L.gather = take(sizeof(double) * 8 * (size_t)ncases);
    L.tw = take(sizeof(BatchTwSlot) * (size_t)ncases + sizeof(double) * L.mk_cap);
    L.total = align_up(off, 256);
    return L;
}

// Rebuild every table from the cases as they are now (synchronizes).
ibm_status build_tables(ibm_batch *b) {
    const int nc = b->ncases;
    b->drop_graphs();
    std::vector<int> counts((size_t)nc * 4, 0);
    for (int c = 0; c < nc; ++c)
        BCU(cudaMemcpyAsync(&counts[(size_t)c * 4], b->grids[c]->mb.counts, 4 * sizeof(int),
                            cudaMemcpyDeviceToHost, b->stream),
            "read tile counts");
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");

    const int shape = b->tune.tile_shape;
    // every case's spreading operator built (static markers): the batch
    // spreads through them, in runs of 32 forced cells
    bool use_op = true;
    for (int c = 0; c < nc; ++c)
        if (b->grids[c]->mb.ns > 0 && !b->grids[c]->mb.sp_ready) use_op = false;
    std::vector<int2> st, bd, mk;
    std::vector<BatchCase> tb((size_t)2 * nc);
    size_t smem = 0;
    for (int c = 0; c < nc; ++c) {
        ibm_grid *g = b->grids[c];
        BatchCase bc{};
        bc.g = g->gp;
        bc.U1 = g->L;
        bc.dt = g->fb.dt;
        bc.err = g->err_d;
        bc.band_bits = g->mb.band_bits;
        bc.m = g->mb;
        bc.item0 = (int)st.size();
        bc.nitems = tiles_of_shape(g->desc, shape);
        for (int t = 0; t < bc.nitems; ++t) st.push_back(make_int2(c, t));
        const int ns = g->mb.ns;
        const int ncell = ns > 0 ? counts[(size_t)c * 4 + 2] : 0;
        const int nband = ns <= 0 ? 0 : use_op ? (ncell + 31) / 32 : counts[(size_t)c * 4 + 1];
        bc.band0 = (int)bd.size();
        bc.nband = nband;
        for (int i = 0; i < nband; ++i) bd.push_back(make_int2(c, use_op ? 32 * i : i));
        for (int k = 0; k < ns; ++k) mk.push_back(make_int2(c, k));
        if (ns > 0) smem = std::max(smem, batch_spread_smem(g->gp, b->fp_bytes));
        for (int p = 0; p < 2; ++p) {
            const int un = g->cur ^ p;
            bc.Un = g->U[un];
            bc.Us = g->U[1 - un];
            tb[(size_t)p * nc + c] = bc;
        }
    }
    if (st.size() > b->stage_cap || bd.size() > b->band_cap || mk.size() > b->mk_cap)
        return fail(b, IBM_ERR_WORKSPACE, "batch work lists exceed their capacity");
    BCU(cudaMemcpyAsync(b->tbl[0], tb.data(), sizeof(BatchCase) * (size_t)2 * nc,
                        cudaMemcpyHostToDevice, b->stream),
        "upload case tables");
    if (!st.empty())
        BCU(cudaMemcpyAsync(b->stage_items, st.data(), sizeof(int2) * st.size(),
                            cudaMemcpyHostToDevice, b->stream),
            "upload stage items");
    if (!bd.empty())
        BCU(cudaMemcpyAsync(b->band_items, bd.data(), sizeof(int2) * bd.size(),
                            cudaMemcpyHostToDevice, b->stream),
            "upload band items");
    if (!mk.empty())
        BCU(cudaMemcpyAsync(b->mk_items, mk.data(), sizeof(int2) * mk.size(),
                            cudaMemcpyHostToDevice, b->stream),
            "upload marker items");
    // the uploads read the host vectors above
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    b->n_stage = (int)st.size();
    b->n_band = (int)bd.size();
    b->n_mk = (int)mk.size();
    b->spread_smem = smem;
    b->spread_op = use_op;
    b->tbl_cur.resize(nc);
    b->tbl_gen.resize(nc);
    for (int c = 0; c < nc; ++c) {
        b->tbl_cur[c] = b->grids[c]->cur;
        b->tbl_gen[c] = b->grids[c]->marker_gen;
    }
    b->built_shape = shape;
    b->built = true;
    return IBM_OK;
}

// Parity of the table that matches the cases' current buffers, or -1 when
// the tables are stale (markers changed, a case stepped alone, new tuning).
int table_parity(const ibm_batch *b) {
    if (!b->built || b->built_shape != b->tune.tile_shape) return -1;
    int p = -1;
    for (int c = 0; c < b->ncases; ++c) {
        const ibm_grid *g = b->grids[c];
        if (g->marker_gen != b->tbl_gen[c]) return -1;
        const int pc = g->cur ^ b->tbl_cur[c];
        if (p < 0) p = pc;
        else if (pc != p) return -1;
    }
    return p;
}

ibm_status current_parity(ibm_batch *b, int *p) {
    *p = table_parity(b);
    if (*p >= 0) return IBM_OK;
    ibm_status st = build_tables(b);
    if (st != IBM_OK) return st;
    *p = table_parity(b);
    return *p >= 0 ? IBM_OK : fail(b, IBM_ERR_STATE, "batch tables inconsistent");
}

// One kernel group of a batch step (IBM_PROF_STAGE1, _STAGE2, _INTERP,
// _SPREAD or _FINISH).
cudaError_t launch_group(ibm_batch *b, int p, int group, double dt_fixed, cudaStream_t s) {
    const BatchCase *t = b->tbl[p];
    const int sh = b->tune.tile_shape, fp = b->fp_bytes;
    switch (group) {
    case IBM_PROF_STAGE1:
        return launch_batch_stage(1, sh, fp, t, b->stage_items, b->n_stage, b->item_max, dt_fixed,
                                  b->n_sm, s);
    case IBM_PROF_STAGE2:
        return launch_batch_stage(2, sh, fp, t, b->stage_items, b->n_stage, b->item_max, dt_fixed,
                                  b->n_sm, s);
    case IBM_PROF_INTERP:
        return launch_batch_interp(fp, t, b->mk_items, b->n_mk, b->tune.markers_per_block, s);
    case IBM_PROF_SPREAD:
        if (b->spread_op)
            return launch_batch_spread_static(fp, t, b->band_items, b->n_band, b->band_max, s);
        return launch_batch_spread(fp, b->spread_smem, t, b->band_items, b->n_band, b->band_max,
                                   b->n_sm, s);
    case IBM_PROF_FINISH:
        return launch_batch_finish(t, b->ncases, b->item_max, b->band_max, dt_fixed, s);
    default:
        return cudaErrorInvalidValue;
    }
}

constexpr int kStepGroups[5] = {IBM_PROF_STAGE1, IBM_PROF_STAGE2, IBM_PROF_INTERP,
                                IBM_PROF_SPREAD, IBM_PROF_FINISH};

cudaError_t launch_stages(ibm_batch *b, int p, double dt_fixed, cudaStream_t s) {
    cudaError_t e = launch_group(b, p, IBM_PROF_STAGE1, dt_fixed, s);
    if (e == cudaSuccess) e = launch_group(b, p, IBM_PROF_STAGE2, dt_fixed, s);
    return e;
}

// launches of a group in one step (0 when it has no work items)
int group_launches(const ibm_batch *b, int group) {
    switch (group) {
    case IBM_PROF_STAGE1:
    case IBM_PROF_STAGE2: return b->n_stage > 0;
    case IBM_PROF_INTERP: return b->n_mk > 0;
    case IBM_PROF_SPREAD: return b->n_band > 0;
    default: return 1;
    }
}

cudaError_t launch_step(ibm_batch *b, int p, double dt_fixed, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
        const int grp = kStepGroups[i];
        if (!b->prof) {
            e = launch_group(b, p, grp, dt_fixed, s);
            continue;
        }
        while (b->ev_pool.size() < b->ev_used + 2) {
            cudaEvent_t ev;
            e = cudaEventCreate(&ev);
            if (e != cudaSuccess) return e;
            b->ev_pool.push_back(ev);
        }
        const size_t k = b->ev_used;
        b->ev_used += 2;
        b->recs.push_back({grp, group_launches(b, grp), k});
        e = cudaEventRecord(b->ev_pool[k], s);
        if (e == cudaSuccess) e = launch_group(b, p, grp, dt_fixed, s);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev_pool[k + 1], s);
    }
    return e;
}

// Capture one step of parity p into a graph (once per parity and dt_fixed).
ibm_status ensure_graph(ibm_batch *b, int p, double dt_fixed) {
    if (b->exec[p] && b->exec_dt[p] == dt_fixed) return IBM_OK;
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
    b->exec[p] = nullptr;
    BCU(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed), "begin capture");
    const cudaError_t e = launch_step(b, p, dt_fixed, b->cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(b, IBM_ERR_CUDA,
                    std::string("capture step: ") +
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    const cudaError_t e3 = cudaGraphInstantiate(&b->exec[p], graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        b->exec[p] = nullptr;
        return fail(b, IBM_ERR_CUDA, std::string("instantiate step graph: ") + cudaGetErrorString(e3));
    }
    b->exec_dt[p] = dt_fixed;
    return IBM_OK;
}

ibm_status check_cases_ready(ibm_batch *b) {
    for (int c = 0; c < b->ncases; ++c) {
        const ibm_grid *g = b->grids[c];
        if (!g->has_state)
            return fail(b, IBM_ERR_STATE, "case " + std::to_string(c) + " has no state");
        if (g->moving && g->mb.ns > 0)
            return fail(b, IBM_ERR_UNSUPPORTED,
                        "case " + std::to_string(c) + " has moving markers; batches take static markers");
    }
    return IBM_OK;
}

}  // namespace

extern "C" {

size_t ibm_batch_workspace_bytes(int ncases, const ibm_grid_desc *descs, const int *max_markers) {
    ibm_status st;
    if (check_batch(ncases, descs, max_markers, &st)) return 0;
    return batch_layout(ncases, descs, max_markers).total;
}

ibm_status ibm_create_batch(int ncases, const ibm_grid_desc *descs, const int *max_markers,
                            void *dev_workspace, size_t bytes, void *stream, ibm_batch **out) {
    if (!out) return fail(nullptr, IBM_ERR_ARG, "null output handle pointer");
    *out = nullptr;
    ibm_status st;
    if (const char *why = check_batch(ncases, descs, max_markers, &st)) return fail(nullptr, st, why);
    if (!dev_workspace) return fail(nullptr, IBM_ERR_ARG, "null workspace");
    if (((uintptr_t)dev_workspace) % 256 != 0)
        return fail(nullptr, IBM_ERR_ARG, "workspace must be 256-byte aligned");
    const BatchLayout L = batch_layout(ncases, descs, max_markers);
    if (bytes < L.total)
        return fail(nullptr, IBM_ERR_WORKSPACE,
                    "workspace too small: need " + std::to_string(L.total) + " bytes");
    ibm_batch *b = new (std::nothrow) ibm_batch();
    if (!b) return fail(nullptr, IBM_ERR_ARG, "host allocation failed");
    b->ncases = ncases;
    b->fp_bytes = descs[0].fp_bytes;
    b->stream = (cudaStream_t)stream;
    char *base = (char *)dev_workspace;
    for (int c = 0; c < ncases; ++c) {
        ibm_grid *g = nullptr;
        const int mm = max_markers ? max_markers[c] : 0;
        const ibm_status s2 = ibm_create_grid(&descs[c], mm, base + L.case_off[c], L.case_bytes[c],
                                              stream, &g);
        if (s2 != IBM_OK) {
            const std::string msg = "case " + std::to_string(c) + ": " + ibm_last_error(nullptr);
            delete b;
            return fail(nullptr, s2, msg);
        }
        g->in_batch = true;
        b->grids.push_back(g);
    }
    b->tbl[0] = (BatchCase *)(base + L.tbl);
    b->tbl[1] = b->tbl[0] + ncases;
    b->stage_items = (int2 *)(base + L.stage_items);
    b->item_max = (double *)(base + L.item_max);
    b->band_items = (int2 *)(base + L.band_items);
    b->band_max = (double *)(base + L.band_max);
    b->mk_items = (int2 *)(base + L.mk_items);
    b->save = (double *)(base + L.save);
    b->gather = (double *)(base + L.gather);
    b->tw_slots = (BatchTwSlot *)(base + L.tw);
    b->tw_vals = (double *)(b->tw_slots + ncases);
    b->stage_cap = L.stage_cap;
    b->band_cap = L.band_cap;
    b->mk_cap = L.mk_cap;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        const std::string msg = std::string("CUDA: ") + cudaGetErrorString(e);
        delete b;
        return fail(nullptr, IBM_ERR_CUDA, msg);
    }
    *out = b;
    return IBM_OK;
}

ibm_status ibm_batch_destroy(ibm_batch *b) {
    if (!b) return IBM_ERR_ARG;
    delete b;
    return IBM_OK;
}

ibm_grid *ibm_batch_case(ibm_batch *b, int c) {
    if (!b || c < 0 || c >= b->ncases) return nullptr;
    return b->grids[c];
}

const char *ibm_batch_last_error(const ibm_batch *b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

ibm_status ibm_batch_get_tuning(const ibm_batch *b, ibm_batch_tuning *t) {
    if (!b || !t) return IBM_ERR_ARG;
    *t = b->tune;
    return IBM_OK;
}

ibm_status ibm_batch_set_tuning(ibm_batch *b, const ibm_batch_tuning *t) {
    if (!b) return IBM_ERR_ARG;
    if (!t) return fail(b, IBM_ERR_ARG, "null tuning");
    if (t->tile_shape < 0 || t->tile_shape >= kBatchShapes)
        return fail(b, IBM_ERR_ARG, "tile_shape must be in [0, 3]");
    if (t->markers_per_block < 1 || t->markers_per_block > 16)
        return fail(b, IBM_ERR_ARG, "markers_per_block must be in [1, 16]");
    if (t->tile_shape != b->tune.tile_shape || t->markers_per_block != b->tune.markers_per_block)
        b->drop_graphs();
    b->tune = *t;
    return IBM_OK;
}

ibm_status ibm_batch_step(ibm_batch *b, int nsteps, double dt_fixed) {
    if (!b) return IBM_ERR_ARG;
    if (nsteps < 0 || !isfinite(dt_fixed)) return fail(b, IBM_ERR_ARG, "invalid step arguments");
    ibm_status st = check_cases_ready(b);
    if (st != IBM_OK) return st;
    if (nsteps == 0) return IBM_OK;
    int p = 0;
    st = current_parity(b, &p);
    if (st != IBM_OK) return st;
    for (int s = 0; s < nsteps; ++s) {
        if (b->tune.use_graph && !b->prof) {
            st = ensure_graph(b, p, dt_fixed);
            if (st != IBM_OK) return st;
            BCU(cudaGraphLaunch(b->exec[p], b->stream), "graph launch");
        } else {
            BCU(launch_step(b, p, dt_fixed, b->stream), "batch step");
        }
        for (ibm_grid *g : b->grids) g->cur = 1 - g->cur;
        p ^= 1;
    }
    return IBM_OK;
}

ibm_status ibm_batch_profile(ibm_batch *b, int enable) {
    if (!b) return IBM_ERR_ARG;
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    b->recs.clear();
    b->ev_used = 0;
    for (int i = 0; i < IBM_PROF_GROUPS; ++i) {
        b->prof_ms[i] = 0.0;
        b->prof_n[i] = 0;
    }
    b->prof = enable != 0;
    return IBM_OK;
}

ibm_status ibm_batch_profile_read(ibm_batch *b, double *ms, long long *launches) {
    if (!b) return IBM_ERR_ARG;
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    for (const auto &r : b->recs) {
        float f = 0.0f;
        BCU(cudaEventElapsedTime(&f, b->ev_pool[r.ev], b->ev_pool[r.ev + 1]), "event timing");
        b->prof_ms[r.group] += f;
        b->prof_n[r.group] += r.launches;
    }
    b->recs.clear();
    b->ev_used = 0;
    for (int i = 0; i < IBM_PROF_GROUPS; ++i) {
        if (ms) ms[i] = b->prof_ms[i];
        if (launches) launches[i] = b->prof_n[i];
        b->prof_ms[i] = 0.0;
        b->prof_n[i] = 0;
    }
    return IBM_OK;
}

ibm_status ibm_batch_sync(ibm_batch *b, int *bad_case) {
    if (!b) return IBM_ERR_ARG;
    if (bad_case) *bad_case = -1;
    std::vector<int> errs((size_t)b->ncases, 0);
    for (int c = 0; c < b->ncases; ++c)
        BCU(cudaMemcpyAsync(&errs[c], b->grids[c]->err_d, sizeof(int), cudaMemcpyDeviceToHost,
                            b->stream),
            "read error words");
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    for (int c = 0; c < b->ncases; ++c) {
        if (!errs[c]) continue;
        const ibm_status st = ibm_sync(b->grids[c]);
        if (bad_case) *bad_case = c;
        return fail(b, st == IBM_OK ? IBM_ERR_STATE : st,
                    "case " + std::to_string(c) + ": " + ibm_last_error(b->grids[c]));
    }
    return IBM_OK;
}

ibm_status ibm_batch_set_wall_temperature(ibm_batch *b, const double *Tw) {
    if (!b) return IBM_ERR_ARG;
    const int nc = b->ncases;
    std::vector<BatchTwSlot> slots((size_t)nc);
    long long total = 0;
    for (int c = 0; c < nc; ++c) {
        ibm_grid *g = b->grids[c];
        slots[c] = BatchTwSlot{g->mb.Tw, total, (long long)g->mb.ns};
        total += g->mb.ns;
    }
    if (total == 0) return IBM_OK;
    if (!Tw) return fail(b, IBM_ERR_ARG, "null wall temperatures");
    for (long long k = 0; k < total; ++k)
        if (!std::isfinite(Tw[k]) || Tw[k] <= 0.0)
            return fail(b, IBM_ERR_ARG,
                        "wall temperature " + std::to_string(k) + " must be finite and positive");
    for (int c = 0; c < nc; ++c) {
        ibm_grid *g = b->grids[c];
        g->Tw_h.assign(Tw + slots[c].off, Tw + slots[c].off + slots[c].n);
    }
    // the slot table changes only with the kept-marker counts
    bool same = b->tw_slots_h.size() == slots.size();
    for (size_t c = 0; same && c < slots.size(); ++c)
        same = b->tw_slots_h[c].dst == slots[c].dst && b->tw_slots_h[c].off == slots[c].off &&
               b->tw_slots_h[c].n == slots[c].n;
    if (!same) {
        BCU(cudaMemcpyAsync(b->tw_slots, slots.data(), sizeof(BatchTwSlot) * nc,
                            cudaMemcpyHostToDevice, b->stream),
            "upload wall-temperature slots");
        BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
        b->tw_slots_h = slots;
    }
    BCU(cudaMemcpyAsync(b->tw_vals, Tw, sizeof(double) * total, cudaMemcpyHostToDevice, b->stream),
        "upload wall temperatures");
    BCU(launch_batch_tw(b->tw_slots, nc, b->tw_vals, b->stream), "scatter wall temperatures");
    return IBM_OK;
}

ibm_status ibm_batch_forces(ibm_batch *b, double *out) {
    if (!b) return IBM_ERR_ARG;
    if (!out) return fail(b, IBM_ERR_ARG, "null output");
    int p = 0;
    ibm_status st = current_parity(b, &p);
    if (st != IBM_OK) return st;
    const int nc = b->ncases;
    std::vector<double> sums((size_t)nc * 8);
    BCU(launch_batch_gather(b->tbl[p], nc, b->gather, b->stream), "gather sums");
    BCU(cudaMemcpyAsync(sums.data(), b->gather, sizeof(double) * 8 * nc, cudaMemcpyDeviceToHost,
                        b->stream),
        "read sums");
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    // the error words came with the sums; a failing case reports as
    // ibm_batch_sync would
    for (int c = 0; c < nc; ++c)
        if (sums[(size_t)c * 8 + 6] != 0.0) return ibm_batch_sync(b, nullptr);
    for (int c = 0; c < nc; ++c) {
        double f[3], q, cd, cl, nu;
        const double *sc = &sums[(size_t)c * 8];
        forces_from_sums(b->grids[c], sc, f, &q, &cd, &cl, &nu);
        double *o = out + (size_t)c * 8;
        o[0] = f[0];
        o[1] = f[1];
        o[2] = q;
        o[3] = cd;
        o[4] = cl;
        o[5] = nu;
        o[6] = sc[4];
        o[7] = sc[5];
    }
    return IBM_OK;
}

ibm_status ibm_batch_autotune(ibm_batch *b, int reps, double *stage_ms, double *interp_ms) {
    if (!b) return IBM_ERR_ARG;
    if (reps < 1 || reps > 10000) return fail(b, IBM_ERR_ARG, "reps must be in [1, 10000]");
    ibm_status st = check_cases_ready(b);
    if (st != IBM_OK) return st;
    int p = 0;
    st = current_parity(b, &p);
    if (st != IBM_OK) return st;
    // keep the last marker forcing: the interpolation passes overwrite it
    size_t off = 0;
    for (ibm_grid *g : b->grids) {
        const size_t ns = (size_t)g->mb.ns;
        if (ns == 0) continue;
        BCU(cudaMemcpyAsync(b->save + off, g->mb.rhoL, sizeof(double) * ns, cudaMemcpyDeviceToDevice, b->stream), "save");
        BCU(cudaMemcpyAsync(b->save + off + ns, g->mb.G, sizeof(double) * 2 * ns, cudaMemcpyDeviceToDevice, b->stream), "save");
        BCU(cudaMemcpyAsync(b->save + off + 3 * ns, g->mb.H, sizeof(double) * ns, cudaMemcpyDeviceToDevice, b->stream), "save");
        off += 4 * ns;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCU(cudaEventCreate(&e0), "event");
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(b, IBM_ERR_CUDA, "event");
    }
    auto timed = [&](auto &&body, double *ms) -> cudaError_t {
        cudaError_t e = body();   // warm-up pass
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = body();
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float f = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
        *ms = (double)f / reps;
        return e;
    };
    const ibm_batch_tuning keep = b->tune;
    double sms[kBatchShapes] = {0}, ims[5] = {0};
    const int warps[5] = {1, 2, 4, 8, 16};
    cudaError_t e = cudaSuccess;
    for (int s = 0; s < kBatchShapes && st == IBM_OK && e == cudaSuccess; ++s) {
        b->tune.tile_shape = s;
        st = current_parity(b, &p);
        if (st == IBM_OK)
            e = timed([&]() { return launch_stages(b, p, 0.0, b->stream); }, &sms[s]);
    }
    for (int i = 0; i < 5 && st == IBM_OK && e == cudaSuccess; ++i) {
        const BatchCase *t = b->tbl[p];
        e = timed([&]() {
            return launch_batch_interp(b->fp_bytes, t, b->mk_items, b->n_mk, warps[i], b->stream);
        }, &ims[i]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == IBM_OK && e != cudaSuccess)
        st = fail(b, IBM_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    if (st == IBM_OK) {
        int bs = 0, bi = 0;
        for (int s = 1; s < kBatchShapes; ++s)
            if (sms[s] < sms[bs]) bs = s;
        for (int i = 1; i < 5; ++i)
            if (ims[i] < ims[bi]) bi = i;
        b->tune.tile_shape = bs;
        b->tune.markers_per_block = warps[bi];
        st = current_parity(b, &p);
    } else {
        b->tune = keep;
    }
    // put the last marker forcing back
    off = 0;
    for (ibm_grid *g : b->grids) {
        const size_t ns = (size_t)g->mb.ns;
        if (ns == 0) continue;
        BCU(cudaMemcpyAsync(g->mb.rhoL, b->save + off, sizeof(double) * ns, cudaMemcpyDeviceToDevice, b->stream), "restore");
        BCU(cudaMemcpyAsync(g->mb.G, b->save + off + ns, sizeof(double) * 2 * ns, cudaMemcpyDeviceToDevice, b->stream), "restore");
        BCU(cudaMemcpyAsync(g->mb.H, b->save + off + 3 * ns, sizeof(double) * ns, cudaMemcpyDeviceToDevice, b->stream), "restore");
        off += 4 * ns;
    }
    BCU(cudaStreamSynchronize(b->stream), "stream synchronize");
    if (st != IBM_OK) return st;
    b->drop_graphs();
    if (stage_ms)
        for (int s = 0; s < kBatchShapes; ++s) stage_ms[s] = sms[s];
    if (interp_ms)
        for (int i = 0; i < 5; ++i) interp_ms[i] = ims[i];
    return IBM_OK;
}

}  // extern "C"
