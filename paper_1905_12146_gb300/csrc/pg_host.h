// Host-side internals of the library shared by its translation units (not part of the C ABI):
// the context and handle records, where an upload places its device block, and the entry points
// the serving runtime (pg_server.cu) builds on.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <pthread.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "phylograd.h"
#include "pg_internal.cuh"

struct pg_ctx {
    int device = 0;
    int n_sm = 1;
    int blocks_per_sm[2][pg::kMaxCat + 1] = {};   // tree kernel occupancy [precision][C]
    int max_range = 0;                            // cap on patterns per block (0 = kMaxRange)
    uint64_t budget = 0;
    uint64_t used = 0;
    uint32_t flags = 0;
    std::mutex mu;   // guards used and handles (a serving worker uploads and frees concurrently)
    std::vector<pg_handle *> handles;
};

struct pg_handle {
    pg_ctx *ctx = nullptr;
    pg::ProbDesc desc{};     // device pointers; b and outputs are set per evaluation
    void *block = nullptr;   // one device allocation holding every array of the problem
    size_t bytes = 0;
    int max_tiles = 0;       // blocks one evaluation of this problem may use
    int cut = 0;             // levels [0, cut) run as level kernels when evaluated alone
    std::vector<int> level_off;   // host copy of the level offsets
    std::vector<uint8_t> level_cherry;   // 1 when every node of the level has two tip children
    int timing = 0;                // phase-timing mode: 0 off, 1 every phase, 2 the pre-order levels,
                                   // 3 those of every kTimingEvery-th evaluation
    long long timing_count = 0;    // full evaluations enqueued since the mode was set
    std::vector<cudaEvent_t> events;   // 6 per timed evaluation
    uint64_t post_levels_bytes = 0, fused_bytes = 0, pre_levels_bytes = 0;
    double *io_b = nullptr, *io_logL = nullptr, *io_grad = nullptr, *io_hess = nullptr,
           *io_site = nullptr;   // device staging for the host-pointer pg_eval
    // pinned host staging of pg_eval (allocated on its first call, freed with the handle): the branch
    // lengths, the status word and the device span io_logL .. io_site + P, each 16-byte aligned
    char *io_host = nullptr;
    size_t io_host_bytes = 0;
    pg_handle_info info{};
    cudaStream_t last_stream = nullptr;
    bool have_post = false;   // an enqueued post-order left partials a backward pass can use
    bool mstate = false;      // a general state space (pg_mstate.cu): md holds its layout
    pg::MDesc md{};
    CUtensorMap tm_post, tm_pre, tm_tab;   // TMA descriptors of the tensor-core kernels (the type is 64-byte aligned)
    bool external = false;    // the device block belongs to a caller's arena (not freed here)
    // nodes as the caller numbers them: 2N-1, or fewer for a tree with multifurcations, which the
    // handle holds resolved into a binary tree with added nodes n_user .. 2N-2 (branches of length 0)
    int n_user = 0;
    // A problem whose arrays exceed the context's budget, evaluated in pattern chunks: the chunks'
    // handles (contiguous pattern slices starting at chunk_p0) share one region for their
    // per-evaluation arrays and run one after another on the evaluation's stream; their logL,
    // gradient and Hessian land in part_out ([K], [K][n], [K][n]) and are summed in a fixed order.
    std::vector<pg_handle *> chunks;
    std::vector<int> chunk_p0;
    void *scratch_block = nullptr;
    size_t scratch_bytes = 0;
    double *part_out = nullptr;
    double *b_fwd = nullptr;   // [n] the branch lengths of the last forward pass (chunked backward)
    const pg::ProbDesc *d_desc = nullptr;   // device copy of desc (batched level kernels read it)
    const int *d_parent = nullptr;          // [n] parent index on the device (the clock kernels)
};

namespace pg {
namespace host {

extern thread_local std::string g_err;
pg_status fail(pg_status s, const char *fmt, ...);
// the calling thread's error text, as fail() records it (for messages built elsewhere)
void set_error(const std::string &msg);
// Records, without allocating, that `msg` (a static buffer that outlives the call) is the last error
// of thread `tid`: pg_last_error on that thread returns it until the thread records another error.
void publish_static_error(const char *msg, pthread_t tid);

// Where an upload puts its one device block and how it copies into it: cudaMalloc under the
// context's budget and blocking copies (pg_upload), or a caller's allocator (the serving arena)
// and copies enqueued on a stream.
struct Placement {
    void *(*alloc)(void *self, size_t bytes) = nullptr;   // nullptr: no room
    void (*release)(void *self, void *block) = nullptr;
    void *self = nullptr;
    cudaStream_t stream = nullptr;
};

// validation, layout and upload of one problem; pl = nullptr: cudaMalloc + blocking copies
pg_status upload(pg_ctx *ctx, const pg_problem *pr, pg_handle **out, const Placement *pl);
// enqueue one evaluation (skip: kSkipPost / kSkipPre bits) on stream s
pg_status enqueue(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad, double *d_hess,
                  double *d_site_logL, const double *d_gscale, cudaStream_t s);

}  // namespace host
}  // namespace pg
