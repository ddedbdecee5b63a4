// Allocation-free fluid stage 1: L(U) and the stable step size, for callers
// that cannot allocate device memory.
//
// The regular API takes every device buffer from a workspace the caller
// allocates.  Some callers cannot do even that: a module loaded into a host
// application that owns the whole device-memory budget and forbids its
// plug-ins to call cudaMalloc, or a control loop that may not pay for an
// allocation (cudaMalloc can synchronise the device) in the middle of a run.
// They can still hand over the arrays they already own: the state U, the
// output L and the output step size.  The only scratch needed beyond those -
// one double per CTA of the step-size reduction, the last-block ticket and an
// error word - lives in the file-scope device array below.  It is
// statically sized, so every GPU that loads the library holds it until the
// process exits.
#include <mutex>
#include <vector>

#include "../../include/ibm.h"
#include "internal.h"

namespace ibmk {
GridParams params_from_desc(const ibm_grid_desc &d);
const char *desc_problem(const ibm_grid_desc *d);
void set_handle_free_error(const char *msg);
}  // namespace ibmk

using namespace ibmk;

namespace {

// Largest step-size reduction served: 65536 CTAs of 2048 cells (2^27 cells).
constexpr int kMaxCtas = IBM_NOALLOC_MAX_CTAS;
constexpr size_t kMaxCtaBytes = sizeof(double) * (size_t)kMaxCtas;
// block maxima, then the ticket counter and the error word (one 256-byte line)
constexpr size_t kScratchBytes = kMaxCtaBytes + 256;

static __device__ __align__(256) unsigned char g_stage1_scratch[kScratchBytes];

// Device address of g_stage1_scratch, resolved once per device.  In host
// code the symbol names a host-side stand-in, not device memory, so kernels
// must receive the address from cudaGetSymbolAddress.
std::mutex g_mutex;
std::vector<void *> g_addr;   // indexed by device ordinal; nullptr = not yet resolved

cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mutex);
    if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_stage1_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

ibm_status fail(ibm_status st, const char *msg) {
    set_handle_free_error(msg);
    return st;
}

}  // namespace

extern "C" ibm_status ibm_rhs_dt_noalloc(const ibm_grid_desc *desc, const void *U, void *L,
                                         double *dt, void *stream) {
    if (const char *why = desc_problem(desc)) return fail(IBM_ERR_ARG, why);
    if (!U || !L || !dt) return fail(IBM_ERR_ARG, "null buffer");
    const GridParams g = params_from_desc(*desc);
    const size_t ctas = dt_init_blocks(g);
    if (ctas > (size_t)kMaxCtas)
        return fail(IBM_ERR_ARG,
                    "grid too large for ibm_rhs_dt_noalloc: its step-size reduction needs more "
                    "than IBM_NOALLOC_MAX_CTAS (65536) thread blocks of 2048 cells");
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return fail(IBM_ERR_CUDA, cudaGetErrorString(e));
    char *p = (char *)base;
    FluidBuffers fb;
    fb.blockmax = (double *)p;
    fb.counter = (unsigned *)(p + kMaxCtaBytes);
    fb.err = (int *)(p + kMaxCtaBytes + 16);
    fb.dt = dt;
    fb.band_bits = nullptr;
    // the ticket counter and the error word must start at zero; the block
    // maxima are all written before they are read
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemsetAsync(p + kMaxCtaBytes, 0, 256, s);
    if (e == cudaSuccess) e = launch_rhs(g, desc->fp_bytes, U, L, fb, s);
    if (e == cudaSuccess) e = launch_dt_init(g, desc->fp_bytes, U, fb, s);
    if (e != cudaSuccess) return fail(IBM_ERR_CUDA, cudaGetErrorString(e));
    set_handle_free_error("");   // no stale message after a successful call
    return IBM_OK;
}
