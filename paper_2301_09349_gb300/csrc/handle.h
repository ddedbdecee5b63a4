// The grid handle behind the opaque ibm_grid of include/ibm.h (internal:
// shared by api.cu and batch.cu).
#pragma once

#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "internal.h"

struct ibm_grid {
    using GridParams = ibmk::GridParams;
    using FluidBuffers = ibmk::FluidBuffers;
    using MarkerBuffers = ibmk::MarkerBuffers;
    using QuadBuffers = ibmk::QuadBuffers;
    ibm_grid_desc desc;
    GridParams gp;
    cudaStream_t stream = nullptr;
    int device = 0;
    int n_sm = 0;
    int max_markers = 0;
    char *ws = nullptr;
    size_t ws_bytes = 0;

    void *U[2] = {nullptr, nullptr};
    int cur = 0;
    void *L = nullptr;
    FluidBuffers fb{};
    MarkerBuffers mb{};
    QuadBuffers qb{};
    int *err_d = nullptr;
    double *scratch_d = nullptr;   // small device scalars: dt, t

    bool has_state = false;
    bool moving = false;
    long long marker_gen = 0;   // bumped by every ibm_set_markers
    bool recording = false;     // ibm_record: checkpoints taken by ibm_step
    int rec_steps = 0;          // steps recorded since ibm_record / the last new state
    ibmk::AdjBuffers adj{};
    bool in_batch = false;      // owned by an ibm_batch (ibm_destroy refuses it)
    ibm_motion motion{};
    std::vector<int> kept;
    std::vector<double> Tw_h;
    int cg_maxit = 4000;
    double cg_tol = 1e-12;
    std::string err;

    // kernel timing: event pairs recorded around kernel groups
    struct ProfRec {
        int group;
        int launches;
        size_t ev;   // index of the start event; the stop event follows
    };
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRec> recs;
    double prof_ms[IBM_PROF_GROUPS] = {0};
    long long prof_n[IBM_PROF_GROUPS] = {0};

    // ibm_step_graphs: steps replayed from captured CUDA graphs of graph_steps
    // steps each, one graph per starting buffer (cur)
    int graph_steps = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};

    // small moving bodies: the marker pipeline runs on a side stream beside
    // fluid stage 1 (forked and joined by events, also inside a capture)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_bins = nullptr, ev_quad = nullptr;
    double gexec_dt[2] = {0.0, 0.0};

    void drop_graphs() {
        for (int p = 0; p < 2; ++p) {
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
            gexec[p] = nullptr;
        }
    }
    ~ibm_grid() {
        drop_graphs();
        if (cap) cudaStreamDestroy(cap);
        if (side) cudaStreamDestroy(side);
        for (cudaEvent_t e : {ev_fork, ev_bins, ev_quad})
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    }
};

namespace ibmk {
// Cd, Cl, Nu and the force/heat rate from the device sums (sums[0..4]).
void forces_from_sums(const ibm_grid *g, const double *sums, double force[3], double *heat_rate,
                      double *Cd, double *Cl, double *Nu);
}  // namespace ibmk
