// Host side of the C ABI declared in include/phylograd.h: validation of a problem (Section 2.1
// assumptions: rooted binary tree, CTMC generators, root distribution, rate categories of
// Section 2.5), level scheduling of the tree, the device layout of one problem and the launches
// of one (or a batch of) evaluation(s).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "phylograd.h"
#include "pg_internal.cuh"
#include <nvtx3/nvToolsExt.h>
#include "pg_host.h"

namespace pg {
namespace host {

thread_local std::string g_err;
// Errors are ordered by one sequence: a thread's own last error (g_err, at g_err_at) or the static
// message that pg_eval_noalloc published for it, whichever came later.
std::atomic<uint64_t> g_err_seq{0};
thread_local uint64_t g_err_at = 0;
std::mutex g_static_mu;
const char *g_static_msg = nullptr;
pthread_t g_static_tid;
uint64_t g_static_at = 0;

void set_error(const std::string &msg) {
    g_err = msg;
    g_err_at = ++g_err_seq;
}

pg_status fail(pg_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error(buf);
    return s;
}

void publish_static_error(const char *msg, pthread_t tid) {
    std::lock_guard<std::mutex> g(g_static_mu);
    g_static_msg = msg;
    g_static_tid = tid;
    g_static_at = ++g_err_seq;
}

const char *last_error() {
    {
        std::lock_guard<std::mutex> g(g_static_mu);
        if (g_static_msg && pthread_equal(g_static_tid, pthread_self()) && g_static_at > g_err_at) return g_static_msg;
    }
    return g_err.c_str();
}

}  // namespace host
}  // namespace pg

using pg::host::fail;
using pg::host::Placement;

namespace {

#define PG_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return fail(PG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Makes ctx's device current for the duration of a call and restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

// ------------------------------------------------------------------------------------------
// validation and tree preparation
// ------------------------------------------------------------------------------------------

namespace {

struct TreePlan {
    int root = -1;
    std::vector<int4> ops;        // internal nodes sorted by height: {k, c0, c1, 0}
    std::vector<int> level_off;   // [H + 1]
};

pg_status plan_tree(int n_tips, const int32_t *parent, TreePlan &tp) {
    const int n = 2 * n_tips - 1;
    std::vector<int> kid0(n, -1), kid1(n, -1);
    for (int i = 0; i < n; ++i) {
        const int p = parent[i];
        if (p == -1) {
            if (tp.root >= 0) return fail(PG_ERR_INVALID, "more than one root (nodes %d and %d)", tp.root, i);
            tp.root = i;
            continue;
        }
        if (p < n_tips || p >= n || p == i)
            return fail(PG_ERR_INVALID, "parent[%d] = %d is not an internal node", i, p);
        if (kid0[p] < 0) kid0[p] = i;
        else if (kid1[p] < 0) kid1[p] = i;
        else return fail(PG_ERR_INVALID, "node %d has more than two children (binary tree required)", p);
    }
    if (tp.root < 0) return fail(PG_ERR_INVALID, "no root (no node with parent -1)");
    if (tp.root < n_tips) return fail(PG_ERR_INVALID, "the root %d is a tip", tp.root);
    for (int k = n_tips; k < n; ++k)
        if (kid1[k] < 0) return fail(PG_ERR_INVALID, "internal node %d has fewer than two children", k);
    // depth-first order from the root; every node must be reached exactly once (no cycles)
    std::vector<int> order;
    order.reserve(n);
    std::vector<int> stack{tp.root};
    while (!stack.empty()) {
        const int k = stack.back();
        stack.pop_back();
        if ((int)order.size() >= n) return fail(PG_ERR_INVALID, "the parent array contains a cycle");
        order.push_back(k);
        if (k >= n_tips) { stack.push_back(kid1[k]); stack.push_back(kid0[k]); }
    }
    if ((int)order.size() != n) return fail(PG_ERR_INVALID, "the parent array contains a cycle");
    std::vector<int> height(n, 0);
    int H = 0;
    for (int o = n - 1; o >= 0; --o) {
        const int k = order[o];
        if (k < n_tips) continue;
        height[k] = 1 + std::max(height[kid0[k]], height[kid1[k]]);
        H = std::max(H, height[k]);
    }
    // counting sort of internal nodes by height (level h-1 holds height h)
    tp.level_off.assign(H + 1, 0);
    for (int k = n_tips; k < n; ++k) tp.level_off[height[k]]++;
    for (int h = 1; h <= H; ++h) tp.level_off[h] += tp.level_off[h - 1];
    tp.ops.assign(n_tips - 1, int4{});
    std::vector<int> fill(tp.level_off.begin(), tp.level_off.end() - 1);
    for (int k = n_tips; k < n; ++k) {
        const int lv = height[k] - 1;
        tp.ops[fill[lv]++] = int4{k, kid0[k], kid1[k], 0};
    }
    return PG_OK;
}

pg_status check_model(const pg_problem *pr) {
    const int m = pr->n_states, C = pr->n_categories, M = pr->n_models;
    if (!pr->Q || !pr->root_freqs || !pr->cat_rates || !pr->cat_weights)
        return fail(PG_ERR_INVALID, "Q, root_freqs, cat_rates and cat_weights are required");
    for (int md = 0; md < M; ++md) {
        const double *Q = pr->Q + (size_t)md * m * m;
        double mx = 0.0;
        for (int t = 0; t < m * m; ++t) {
            if (!std::isfinite(Q[t])) return fail(PG_ERR_INVALID, "Q[%d] has a non-finite entry", md);
            mx = std::max(mx, std::fabs(Q[t]));
        }
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) {
                if (i != j && Q[i * m + j] < 0.0)
                    return fail(PG_ERR_INVALID, "Q[%d][%d][%d] < 0 off the diagonal", md, i, j);
                s += Q[i * m + j];
            }
            if (std::fabs(s) > 1e-10 * std::max(mx, 1e-300) && mx > 0.0)
                return fail(PG_ERR_INVALID, "row %d of Q[%d] sums to %g, not 0", i, md, s);
        }
    }
    double s = 0.0;
    for (int i = 0; i < m; ++i) {
        if (!(pr->root_freqs[i] >= 0.0) || !std::isfinite(pr->root_freqs[i]))
            return fail(PG_ERR_INVALID, "root_freqs[%d] is negative or not finite", i);
        s += pr->root_freqs[i];
    }
    if (std::fabs(s - 1.0) > 1e-10) return fail(PG_ERR_INVALID, "root_freqs sum to %.17g, not 1", s);
    s = 0.0;
    for (int l = 0; l < C; ++l) {
        if (!(pr->cat_weights[l] >= 0.0) || !std::isfinite(pr->cat_weights[l]))
            return fail(PG_ERR_INVALID, "cat_weights[%d] is negative or not finite", l);
        if (!(pr->cat_rates[l] >= 0.0) || !std::isfinite(pr->cat_rates[l]))
            return fail(PG_ERR_INVALID, "cat_rates[%d] is negative or not finite", l);
        s += pr->cat_weights[l];
    }
    if (std::fabs(s - 1.0) > 1e-10) return fail(PG_ERR_INVALID, "cat_weights sum to %.17g, not 1", s);
    const int K = pr->n_tip_partials;
    if (K < 0 || m + K > 256) return fail(PG_ERR_INVALID, "n_tip_partials = %d (0 .. %d)", K, 256 - m);
    if (K > 0 && !pr->tip_partials) return fail(PG_ERR_INVALID, "tip_partials is NULL");
    for (int v = 0; v < K; ++v) {
        bool positive = false;
        for (int i = 0; i < m; ++i) {
            const double x = pr->tip_partials[(size_t)v * m + i];
            if (!(x >= 0.0) || !std::isfinite(x))
                return fail(PG_ERR_INVALID, "tip_partials[%d][%d] is negative or not finite", v, i);
            positive = positive || x > 0.0;
        }
        if (!positive) return fail(PG_ERR_INVALID, "tip_partials[%d] has no positive entry", v);
    }
    const int n = 2 * pr->n_tips - 1;
    if (pr->branch_model)
        for (int i = 0; i < n; ++i)
            if (pr->branch_model[i] < 0 || pr->branch_model[i] >= M)
                return fail(PG_ERR_INVALID, "branch_model[%d] = %d outside [0, %d)", i, pr->branch_model[i], M);
    for (int p = 0; p < pr->n_patterns; ++p)
        if (!(pr->pattern_weights[p] >= 0.0) || !std::isfinite(pr->pattern_weights[p]))
            return fail(PG_ERR_INVALID, "pattern_weights[%d] is negative or not finite", p);
    return PG_OK;
}

// Blocks for one problem evaluated alone: every SM filled to the tree kernel's occupancy.
int single_target(const pg_ctx *ctx, const pg::ProbDesc &d) {
    return std::min(4 * ctx->n_sm, ctx->n_sm * ctx->blocks_per_sm[d.precision][d.C]);
}

// The pattern factor r_p in [1, 2) of the FP32 kernels (pg_device.cuh: pattern_factor): the
// lowbias32 integer hash (C. Wellons) of p as a 23-bit mantissa, the same bits on the host.
float host_pattern_factor(uint32_t p) {
    uint32_t x = p + 0x9E3779B9u;
    x ^= x >> 16; x *= 0x21F0AAADu;
    x ^= x >> 15; x *= 0x735A2D97u;
    x ^= x >> 15;
    const uint32_t bits = 0x3F800000u | (x >> 9);
    float r;
    std::memcpy(&r, &bits, sizeof r);
    return r;
}

// Carves one device allocation into aligned arrays.
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count) {
        const size_t at = align_up(off, 256);
        off = at + count * sizeof(T);
        return at;
    }
};

// The per-evaluation arrays of a problem (partials, their exponents, per-branch slot sums, per-site
// values): in the problem's own block, or in an external region shared by the pattern chunks of a
// problem that is evaluated chunk by chunk (the chunks run one after another on one stream).
struct Scratch {
    char *base = nullptr;
    size_t bytes = 0;
};

// Splits the P patterns of a problem into `target` blocks of contiguous ranges (fewer when the
// ranges would otherwise hold less than one pattern or more than max_range).
void set_tiling(pg::ProbDesc &d, int target, int max_range) {
    const int P = d.P;
    if (P <= 0) {
        d.n_tiles = d.range_len = d.pieces = d.n_tg = 0;
        return;
    }
    int T = std::max(1, std::min(target, P));
    T = std::max(T, (P + max_range - 1) / max_range);
    const int L = (P + T - 1) / T;
    T = (P + L - 1) / L;
    d.n_tiles = T;
    d.range_len = L;
    d.pieces = (L + 31) / 32 + 1;
    d.n_tg = T * d.pieces;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------

namespace {

// Uniformisation of one generator (m states): mu = max_i -Q_ii (1 for Q = 0), B = I + Q / mu
// (entrywise non-negative for a generator), and B^k for k = 1 .. kUnifK in FP64, stored FP32 in
// the padded kMP x kMP layout; QT the transposed generator in FP32.
void uniformise(const double *Q, int m, float *Bpow, float *QT, double *mu_out) {
    double mu = 0.0;
    for (int i = 0; i < m; ++i) mu = std::max(mu, -Q[(size_t)i * m + i]);
    if (!(mu > 0.0)) mu = 1.0;
    std::vector<double> B((size_t)m * m), Bk((size_t)m * m), next((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) B[(size_t)i * m + j] = (i == j ? 1.0 : 0.0) + Q[(size_t)i * m + j] / mu;
    Bk = B;
    const int KP = pg::kMP;
    for (int k = 1; k <= pg::kUnifK; ++k) {
        float *dst = Bpow + (size_t)(k - 1) * KP * KP;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) dst[(size_t)i * KP + j] = (float)Bk[(size_t)i * m + j];
        if (k == pg::kUnifK) break;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < m; ++j) {
                double acc = 0.0;
                for (int t = 0; t < m; ++t) acc += Bk[(size_t)i * m + t] * B[(size_t)t * m + j];
                next[(size_t)i * m + j] = acc;
            }
        Bk.swap(next);
    }
    for (int k = 0; k < m; ++k)
        for (int s = 0; s < m; ++s) QT[(size_t)k * KP + s] = (float)Q[(size_t)s * m + k];
    *mu_out = mu;
}

pg_status acquire_block(pg_ctx *ctx, const Placement *pl, size_t bytes, void **block) {
    *block = nullptr;
    if (pl) {
        *block = pl->alloc(pl->self, bytes);
        return *block ? PG_OK : fail(PG_ERR_OOM, "no room for %zu bytes in the arena", bytes);
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (ctx->budget && ctx->used + bytes > ctx->budget)
            return fail(PG_ERR_OOM, "problem needs %zu bytes, %llu of %llu budget in use", bytes,
                        (unsigned long long)ctx->used, (unsigned long long)ctx->budget);
    }
    cudaError_t ce = cudaMalloc(block, bytes);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        *block = nullptr;
        return fail(PG_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(ce));
    }
    return PG_OK;
}
void release_block(const Placement *pl, void *block) {
    if (!block) return;
    if (pl) pl->release(pl->self, block);
    else cudaFree(block);
}
cudaError_t h2d(const Placement *pl, void *dst, const void *src, size_t n) {
    if (n == 0) return cudaSuccess;
    return pl ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, pl->stream)
              : cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
}
cudaError_t h2d_rows(const Placement *pl, void *dst, size_t dpitch, const void *src, size_t spitch, size_t w, size_t h) {
    return pl ? cudaMemcpy2DAsync(dst, dpitch, src, spitch, w, h, cudaMemcpyHostToDevice, pl->stream)
              : cudaMemcpy2D(dst, dpitch, src, spitch, w, h, cudaMemcpyHostToDevice);
}
cudaError_t dzero(const Placement *pl, void *dst, size_t n) {
    return pl ? cudaMemsetAsync(dst, 0, n, pl->stream) : cudaMemset(dst, 0, n);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// FP32 tiled tensor map with 32-float (128-byte, swizzled) inner boxes; rows beyond a dimension's
// extent read as zero and are not written
pg_status encode_map(CUtensorMap *m, void *base, int rank, const cuuint64_t *dims, const cuuint64_t *strides,
                     const cuuint32_t *box) {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q{};
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            return fail(PG_ERR_CUDA, "the driver provides no cuTensorMapEncodeTiled");
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims, strides, box, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(PG_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return PG_OK;
}

// upload of a problem on the general path (pg_mstate.cu, pg_mtc.cu, pg_mcherry.cu kernels): any
// state count but 4, and 4-state problems with tip partial vectors
pg_status upload_m(pg_ctx *ctx, const pg_problem *pr, const TreePlan &tp, pg_handle **out, const Placement *pl,
                   const Scratch *ext, size_t *scratch_need) {
    const int N = pr->n_tips, m = pr->n_states, P = pr->n_patterns, C = pr->n_categories, M = pr->n_models;
    const int n = 2 * N - 1, H = (int)tp.level_off.size() - 1;
    const int KP = pg::kMP;
    std::vector<float> Bpow((size_t)M * pg::kUnifK * KP * KP, 0.f), QT((size_t)M * KP * KP, 0.f);
    std::vector<double> mu(M, 1.0);
    for (int md = 0; md < M; ++md)
        uniformise(pr->Q + (size_t)md * m * m, m, Bpow.data() + (size_t)md * pg::kUnifK * KP * KP,
                   QT.data() + (size_t)md * KP * KP, &mu[md]);
    const int Ps = (P + 15) / 16 * 16;
    const int n_pt = (P + pg::kMTile - 1) / pg::kMTile, n_lb = (P + pg::kMRootPatterns - 1) / pg::kMRootPatterns;
    Carver cv;
    const size_t o_ops = cv.take<int4>(N - 1), o_lv = cv.take<int>(H + 1);
    const size_t o_tips = cv.take<uint8_t>((size_t)N * Ps), o_w = cv.take<double>(Ps);
    const int K = pr->n_tip_partials;
    // FP32 rows, pads 0, each scaled exactly by 2^-e_v so that its largest entry is 1 (any finite
    // row then neither overflows nor underflows the FP32 products); a site's likelihood is the
    // scaled one times 2^(sum of e over its tips), added back at the root
    std::vector<float> tipv((size_t)std::max(K, 1) * KP, 0.f);
    std::vector<int> tv_e(std::max(K, 1), 0);
    for (int v = 0; v < K; ++v) {
        double mx = 0.0;
        for (int i = 0; i < m; ++i) mx = std::max(mx, pr->tip_partials[(size_t)v * m + i]);
        int e = 0;
        std::frexp(mx, &e);
        tv_e[v] = e - 1;   // mx = f 2^e with f in [0.5, 1): mx 2^-(e-1) in [1, 2)
        for (int i = 0; i < m; ++i)
            tipv[(size_t)v * KP + i] = (float)std::ldexp(pr->tip_partials[(size_t)v * m + i], -tv_e[v]);
    }
    std::vector<int> tip_E;
    bool any_scale = false;
    for (int v = 0; v < K; ++v) any_scale = any_scale || tv_e[v] != 0;
    if (any_scale && P > 0) {
        tip_E.assign(Ps, 0);
        const size_t stride = pr->tip_stride ? (size_t)pr->tip_stride : (size_t)P;
        for (int t = 0; t < N; ++t) {
            const uint8_t *row = pr->tip_states + (size_t)t * stride;
            for (int p = 0; p < P; ++p) {
                const int y = row[p];
                if (y >= m && y < m + K) tip_E[p] += tv_e[y - m];
            }
        }
    }
    const size_t o_tv = cv.take<float>(tipv.size());
    const size_t o_tE = tip_E.empty() ? 0 : cv.take<int>(tip_E.size());
    const size_t o_Bp = cv.take<float>(Bpow.size()), o_QT = cv.take<float>(QT.size());
    const size_t o_mu = cv.take<double>(mu.size());
    const size_t o_bm = pr->branch_model ? cv.take<int>(n) : 0;
    const bool tc = !(ctx->flags & PG_FLAG_SIMT_MSTATE);
    Carver sc;   // per-evaluation arrays (see Scratch)
    const size_t o_tab = sc.take<float>((size_t)n * C * (tc ? (size_t)pg::kTcKinds * KP * KP
                                                              : (size_t)pg::kTabKinds * pg::kTabFloats));
    const size_t part = (size_t)(N - 1) * C * Ps * KP;
    const size_t o_post = sc.take<float>(part), o_pre = sc.take<float>(part);
    const size_t o_pe = sc.take<int>((size_t)(N - 1) * C * Ps), o_qe = sc.take<int>((size_t)(N - 1) * C * Ps);
    // gradient slots per branch: the SIMT kernel's pattern tiles, or the tensor-core kernel's
    // 128-pattern tiles x category groups (at most one group per category)
    const int n_gslots = tc ? ((P + pg::kTcTile - 1) / pg::kTcTile) * C : n_pt;
    const size_t o_gp = sc.take<double>((size_t)n * std::max(n_gslots, 1));
    const size_t o_hp = sc.take<double>((size_t)n * std::max(n_gslots, 1));
    const size_t o_lp = sc.take<double>(std::max(n_lb, 1)), o_st = cv.take<int>(1);
    const size_t o_sinv = sc.take<float>(std::max(Ps, 16)), o_ser = sc.take<int>(std::max(Ps, 16));
    const size_t scratch_bytes = align_up(sc.off, 256);
    if (ext && ext->bytes < scratch_bytes) return fail(PG_ERR_INVALID, "shared scratch too small");
    const size_t o_scr = ext ? 0 : cv.take<char>(scratch_bytes);
    if (scratch_need) {
        *scratch_need = scratch_bytes;
        return PG_OK;
    }
    const size_t o_par = cv.take<int>(n);
    const size_t o_ib = cv.take<double>(n), o_il = cv.take<double>(1), o_ig = cv.take<double>(n);
    const size_t o_ih = cv.take<double>(n), o_is = cv.take<double>(std::max(P, 1));
    const size_t bytes = align_up(cv.off, 256);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", ctx->device);
    void *block = nullptr;
    if (pg_status st = acquire_block(ctx, pl, bytes, &block); st != PG_OK) return st;
    char *base = static_cast<char *>(block);
    pg_handle *h = new (std::nothrow) pg_handle;
    if (!h) { release_block(pl, block); return fail(PG_ERR_OOM, "host allocation failed"); }
    h->ctx = ctx;
    h->block = block;
    h->bytes = bytes;
    h->mstate = true;
    h->external = pl != nullptr;
    auto cp = [&](size_t off, const void *src, size_t nbytes) -> cudaError_t {
        return h2d(pl, base + off, src, nbytes);
    };
    cudaError_t e = cp(o_ops, tp.ops.data(), sizeof(int4) * tp.ops.size());
    if (e == cudaSuccess) e = cp(o_lv, tp.level_off.data(), sizeof(int) * tp.level_off.size());
    if (e == cudaSuccess && P > 0)
        e = h2d_rows(pl, base + o_tips, Ps, pr->tip_states, pr->tip_stride ? pr->tip_stride : P, P, N);
    if (e == cudaSuccess && P > 0) e = cp(o_w, pr->pattern_weights, sizeof(double) * P);
    if (e == cudaSuccess) e = cp(o_tv, tipv.data(), sizeof(float) * tipv.size());
    if (e == cudaSuccess && !tip_E.empty()) e = cp(o_tE, tip_E.data(), sizeof(int) * tip_E.size());
    if (e == cudaSuccess) e = cp(o_Bp, Bpow.data(), sizeof(float) * Bpow.size());
    if (e == cudaSuccess) e = cp(o_QT, QT.data(), sizeof(float) * QT.size());
    if (e == cudaSuccess) e = cp(o_mu, mu.data(), sizeof(double) * mu.size());
    if (e == cudaSuccess && pr->branch_model) e = cp(o_bm, pr->branch_model, sizeof(int) * n);
    if (e == cudaSuccess) e = cp(o_par, pr->parent, sizeof(int) * n);
    if (e == cudaSuccess) e = dzero(pl, base + o_st, sizeof(int));
    // padded states of every partial stay zero: the kernels write whole columns, pads included
    if (e != cudaSuccess) {
        release_block(pl, block);
        delete h;
        return fail(PG_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    pg::MDesc &d = h->md;
    char *scr = ext ? ext->base : base + o_scr;
    d.ops = reinterpret_cast<const int4 *>(base + o_ops);
    d.level_off = reinterpret_cast<const int *>(base + o_lv);
    d.tips = reinterpret_cast<const uint8_t *>(base + o_tips);
    d.tipv = reinterpret_cast<const float *>(base + o_tv);
    d.tip_E = tip_E.empty() ? nullptr : reinterpret_cast<const int *>(base + o_tE);
    d.n_tv = K;
    d.weights = reinterpret_cast<const double *>(base + o_w);
    d.Bpow = reinterpret_cast<const float *>(base + o_Bp);
    d.QT = reinterpret_cast<const float *>(base + o_QT);
    d.mu = reinterpret_cast<const double *>(base + o_mu);
    d.bmodel = pr->branch_model ? reinterpret_cast<const int *>(base + o_bm) : nullptr;
    d.tabs = reinterpret_cast<float *>(scr + o_tab);
    d.post = reinterpret_cast<float *>(scr + o_post);
    d.pre = reinterpret_cast<float *>(scr + o_pre);
    d.pe = reinterpret_cast<int *>(scr + o_pe);
    d.qe = reinterpret_cast<int *>(scr + o_qe);
    d.gpart = reinterpret_cast<double *>(scr + o_gp);
    d.hpart = reinterpret_cast<double *>(scr + o_hp);
    d.lpart = reinterpret_cast<double *>(scr + o_lp);
    d.status = reinterpret_cast<int *>(base + o_st);
    d.site_invL = reinterpret_cast<float *>(scr + o_sinv);
    d.site_Er = reinterpret_cast<int *>(scr + o_ser);
    d.n_tips = N;
    d.n_nodes = n;
    d.root = tp.root;
    d.n_levels = H;
    d.P = P;
    d.Ps = Ps;
    d.m = m;
    d.C = C;
    d.n_models = M;
    d.n_ptiles = n_pt;
    d.tc = tc ? 1 : 0;
    d.n_gslots = n_gslots;
    if (tc && P > 0) {
        const cuuint64_t pdims[3] = {(cuuint64_t)KP, (cuuint64_t)P, (cuuint64_t)(N - 1) * C};
        const cuuint64_t pstr[2] = {(cuuint64_t)KP * 4, (cuuint64_t)Ps * KP * 4};
        const cuuint32_t pbox[3] = {32, (cuuint32_t)pg::kTcTile, 1};
        const cuuint64_t tdims[2] = {(cuuint64_t)KP, (cuuint64_t)n * C * pg::kTcKinds * KP};
        const cuuint64_t tstr[1] = {(cuuint64_t)KP * 4};
        const cuuint32_t tbox[2] = {32, (cuuint32_t)KP};
        pg_status st = encode_map(&h->tm_post, d.post, 3, pdims, pstr, pbox);
        if (st == PG_OK) st = encode_map(&h->tm_pre, d.pre, 3, pdims, pstr, pbox);
        if (st == PG_OK) st = encode_map(&h->tm_tab, d.tabs, 2, tdims, tstr, tbox);
        if (st != PG_OK) {
            release_block(pl, block);
            delete h;
            return st;
        }
    }
    for (int l = 0; l < pg::kMaxCat; ++l) {
        d.cw[l] = l < C ? pr->cat_weights[l] : 0.0;
        d.rates[l] = l < C ? pr->cat_rates[l] : 0.0;
    }
    for (int s = 0; s < KP; ++s) {
        d.pi[s] = s < m ? pr->root_freqs[s] : 0.0;
        d.pif[s] = (float)d.pi[s];
    }
    // the fields the shared entry points read (status, sizes, tree) mirror into desc
    pg::ProbDesc &pd = h->desc;
    pd.ops = d.ops;
    pd.level_off = d.level_off;
    h->d_parent = reinterpret_cast<const int *>(base + o_par);
    pd.status = d.status;
    pd.n_tips = N;
    pd.n_nodes = n;
    pd.root = tp.root;
    pd.n_levels = H;
    pd.P = P;
    pd.Ps = Ps;
    pd.C = C;
    pd.n_models = M;
    h->level_off = tp.level_off;
    h->io_b = reinterpret_cast<double *>(base + o_ib);
    h->io_logL = reinterpret_cast<double *>(base + o_il);
    h->io_grad = reinterpret_cast<double *>(base + o_ig);
    h->io_hess = reinterpret_cast<double *>(base + o_ih);
    h->io_site = reinterpret_cast<double *>(base + o_is);
    pg_handle_info &I = h->info;
    I.n_tips = N;
    I.n_nodes = n;
    I.n_states = m;
    I.n_patterns = P;
    I.n_categories = C;
    I.n_levels = H;
    I.n_tiles = n_pt;
    I.patterns_per_tile = pg::kMTile;
    I.device_bytes = bytes;
    // the same node streams as the 4-state path with kMP FP32 states and one exponent per column
    const uint64_t node_stream = (uint64_t)P * C * ((uint64_t)KP * 4ull + 4ull);
    I.stream_bytes = 5ull * (uint64_t)(N - 2) * node_stream + 2ull * (uint64_t)N * P;
    // post P x, pre P x, G x and P^T q per internal child branch and column (2 kMP^2 each)
    I.flops = (uint64_t)(N - 2) * P * C * 4ull * 2ull * KP * KP;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!pl) ctx->used += bytes;
        ctx->handles.push_back(h);
    }
    *out = h;
    return PG_OK;
}

// an NVTX range around the launches of one phase (host timeline; tools that follow NVTX attribute
// the kernels launched inside it to the phase)
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

pg_status enqueue_m(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad, double *d_hess,
                    double *d_site_logL, const double *d_gscale, cudaStream_t s) {
    pg::MDesc d = h->md;
    d.b = d_b;
    d.out_logL = d_logL;
    d.out_grad = d_grad;
    d.out_hess = d_hess;
    d.out_site = d_site_logL;
    d.gscale = d_gscale;
    d.skip = skip;
    const bool fwd = !(skip & pg::kSkipPost), bwd = !(skip & pg::kSkipPre);
    const bool hess = bwd && d_hess != nullptr;
    if (hess && !fwd) return fail(PG_ERR_UNSUPPORTED, "the Hessian diagonal of a %d-state problem needs a full evaluation", d.m);
    cudaError_t e = cudaSuccess;
    Range range(fwd && !(skip & pg::kSkipPre) ? "pg evaluation (general states)"
                                               : (fwd ? "pg forward (general states)" : "pg backward (general states)"));
    if (fwd) {
        e = pg::launch_m_pmatrix(d, hess, s);
        for (int lv = 0; e == cudaSuccess && lv < d.n_levels; ++lv) {
            const int o0 = h->level_off[lv], nd = h->level_off[lv + 1] - o0;
            // level 0 holds exactly the nodes whose children are both tips
            e = !d.tc ? pg::launch_m_post_level(d, o0, nd, s)
                : lv == 0 ? pg::launch_m_post_cherry(d, o0, nd, s)
                          : pg::launch_m_post_level_tc(d, &h->tm_post, &h->tm_tab, o0, nd, s);
        }
        if (e == cudaSuccess) e = pg::launch_m_root(d, s);
    }
    for (int lv = d.n_levels - 1; bwd && e == cudaSuccess && lv >= 0; --lv) {
        const int o0 = h->level_off[lv], nd = h->level_off[lv + 1] - o0;
        e = !d.tc ? pg::launch_m_pre_level(d, o0, nd, hess, s)
            : (lv == 0 && !hess) ? pg::launch_m_pre_cherry(d, o0, nd, s)
                                 : pg::launch_m_pre_level_tc(d, &h->tm_post, &h->tm_pre, &h->tm_tab, o0, nd, hess, h->ctx->n_sm, s);
    }
    if (e == cudaSuccess) e = pg::launch_m_reduce(d, hess, s);
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    h->last_stream = s;
    if (fwd) h->have_post = true;
    return PG_OK;
}

}  // namespace

extern "C" {

const char *pg_status_string(pg_status s) {
    switch (s) {
        case PG_OK: return "ok";
        case PG_ERR_INVALID: return "invalid argument";
        case PG_ERR_OOM: return "out of device memory or over the context budget";
        case PG_ERR_CUDA: return "CUDA runtime error";
        case PG_ERR_TIMEOUT: return "device-side wait timed out";
        case PG_ERR_NUMERIC: return "a site likelihood was zero or not finite";
        case PG_ERR_UNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

const char *pg_last_error(void) { return pg::host::last_error(); }

pg_status pg_create(const pg_options *opt, pg_ctx **out) {
    if (!out) return fail(PG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    pg_options o{};
    if (opt) o = *opt;
    int ndev = 0;
    PG_CUDA(cudaGetDeviceCount(&ndev));
    if (o.device < 0 || o.device >= ndev) return fail(PG_ERR_INVALID, "device %d not present (%d devices)", o.device, ndev);
    if (o.patterns_per_tile < 0 || o.patterns_per_tile > pg::kMaxRange)
        return fail(PG_ERR_INVALID, "patterns_per_tile must be in [0, %d]", pg::kMaxRange);
    pg_ctx *c = new (std::nothrow) pg_ctx;
    if (!c) return fail(PG_ERR_OOM, "host allocation failed");
    c->device = o.device;
    c->max_range = o.patterns_per_tile;
    c->budget = o.hbm_budget_bytes;
    c->flags = o.flags;
    DeviceGuard g(c->device);
    if (!g.ok) { delete c; return fail(PG_ERR_CUDA, "cannot select device %d", o.device); }
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->n_sm < 1) {
        delete c;
        return fail(PG_ERR_CUDA, "cannot read the SM count of device %d", o.device);
    }
    for (int f = 0; f < 2; ++f)
        for (int C = 1; C <= pg::kMaxCat; ++C) c->blocks_per_sm[f][C] = pg::tree_blocks_per_sm(C, f == 1);
    *out = c;
    return PG_OK;
}

pg_status pg_free(pg_handle *h) {
    if (!h) return PG_OK;
    pg_ctx *c = h->ctx;
    DeviceGuard g(c->device);
    for (pg_handle *ch : h->chunks) pg_free(ch);   // a problem evaluated in pattern chunks
    if (h->scratch_block) {
        cudaFree(h->scratch_block);
        std::lock_guard<std::mutex> gl(c->mu);
        c->used -= h->scratch_bytes;
    }
    for (cudaEvent_t x : h->events) cudaEventDestroy(x);
    if (h->io_host) cudaFreeHost(h->io_host);
    if (h->block && !h->external) cudaFree(h->block);
    {
        std::lock_guard<std::mutex> gl(c->mu);
        if (h->block && !h->external) c->used -= h->bytes;
        c->handles.erase(std::remove(c->handles.begin(), c->handles.end(), h), c->handles.end());
    }
    delete h;
    return PG_OK;
}

pg_status pg_destroy(pg_ctx *ctx) {
    if (!ctx) return PG_OK;
    while (!ctx->handles.empty()) pg_free(ctx->handles.back());
    delete ctx;
    return PG_OK;
}

pg_status pg_upload(pg_ctx *ctx, const pg_problem *pr, pg_handle **out) { return pg::host::upload(ctx, pr, out, nullptr); }

}  // extern "C"

// upload of a binary tree (n = 2N-1 nodes); pg::host::upload resolves multifurcations first
// (scratch_need: only compute the bytes of the per-evaluation arrays, allocate nothing)
static pg_status upload_binary(pg_ctx *ctx, const pg_problem *pr, pg_handle **out, const Placement *pl,
                               const Scratch *ext = nullptr, size_t *scratch_need = nullptr) {
    if (!ctx || !pr || !out) return fail(PG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const int N = pr->n_tips, m = pr->n_states, P = pr->n_patterns, C = pr->n_categories;
    if (N < 2) return fail(PG_ERR_INVALID, "n_tips = %d (at least 2 required)", N);
    if (m < 2) return fail(PG_ERR_INVALID, "n_states = %d (at least 2 required)", m);
    if (P < 0) return fail(PG_ERR_INVALID, "n_patterns = %d", P);
    if (C < 1) return fail(PG_ERR_INVALID, "n_categories = %d", C);
    if (pr->n_models < 1) return fail(PG_ERR_INVALID, "n_models = %d", pr->n_models);
    if (pr->precision != PG_PRECISION_FP32 && pr->precision != PG_PRECISION_FP64)
        return fail(PG_ERR_INVALID, "precision = %d", pr->precision);
    const bool f64 = pr->precision == PG_PRECISION_FP64;
    if (m > pg::kMP) return fail(PG_ERR_UNSUPPORTED, "n_states = %d: at most %d", m, pg::kMP);
    if (m != pg::kStates && f64)
        return fail(PG_ERR_UNSUPPORTED, "FP64 partials are implemented for 4 states only");
    if (pr->n_tip_partials > 0 && f64)
        return fail(PG_ERR_UNSUPPORTED, "FP64 partials are implemented without tip partial vectors only");
    if (C > pg::kMaxCat) return fail(PG_ERR_UNSUPPORTED, "n_categories = %d: at most %d", C, pg::kMaxCat);
    if (!pr->parent) return fail(PG_ERR_INVALID, "parent is NULL");
    if (P > 0 && (!pr->tip_states || !pr->pattern_weights))
        return fail(PG_ERR_INVALID, "tip_states and pattern_weights are required when n_patterns > 0");
    if (pr->tip_stride != 0 && pr->tip_stride < P)
        return fail(PG_ERR_INVALID, "tip_stride = %d is smaller than n_patterns = %d", pr->tip_stride, P);
    if ((int64_t)N * 2 - 1 > (int64_t)1 << 30) return fail(PG_ERR_UNSUPPORTED, "tree too large");
    TreePlan tp;
    pg_status st = plan_tree(N, pr->parent, tp);
    if (st != PG_OK) return st;
    st = check_model(pr);
    if (st != PG_OK) return st;
    // the 4-state kernels take state codes and missing data only; tip partial vectors run on the
    // general path
    if (m != pg::kStates || pr->n_tip_partials > 0) return upload_m(ctx, pr, tp, out, pl, ext, scratch_need);

    const int n = 2 * N - 1;
    const int H = (int)tp.level_off.size() - 1;
    // a launch uses at most max_tiles blocks for this problem, each a range of <= kMaxRange
    // patterns; its slot arrays hold n_tiles * (ceil(range/32) + 1) <= P/32 + 3 * max_tiles
    const int max_tiles = 4 * ctx->n_sm;
    const int max_range = ctx->max_range ? ctx->max_range : pg::kMaxRange;
    if ((int64_t)max_tiles * max_range < (int64_t)P)
        return fail(PG_ERR_UNSUPPORTED, "n_patterns = %d exceeds %d on this device", P, max_tiles * max_range);
    const int Ps = (P + 15) / 16 * 16;   // row stride of per-pattern arrays (16-byte rows for TMA)
    const int level_ranges = (P + pg::level_range(C) - 1) / pg::level_range(C);
    // wide branches use one slot per (range, consumer warp) of the level kernels
    const int slot_cap = std::max((P + 31) / 32 + 3 * max_tiles + 2, level_ranges * (pg::kLevelRange / 32));
    // FP32 problems evaluated alone run every level with at least two blocks per SM of
    // (node, 256-pattern) work as its own launch; the narrower levels near the root stay fused
    int cut = 0;
    if (!f64) {
        while (cut < H - 1 && (int64_t)(tp.level_off[cut + 1] - tp.level_off[cut]) * level_ranges >= 2 * ctx->n_sm)
            ++cut;
    }
    std::vector<int> plevel(n, -1);   // level index of each node's parent
    for (int lv = 0; lv < H; ++lv)
        for (int o = tp.level_off[lv]; o < tp.level_off[lv + 1]; ++o) {
            plevel[tp.ops[o].y] = lv;
            plevel[tp.ops[o].z] = lv;
        }
    // ops[].w: bit 0 (bit 1) when c0 (c1) is an internal node on the level just below, whose row the
    // post-order level kernels copy only after waiting for the previous launch
    {
        std::vector<int> lev(n, -1);
        for (int lv = 0; lv < H; ++lv)
            for (int o = tp.level_off[lv]; o < tp.level_off[lv + 1]; ++o) lev[tp.ops[o].x] = lv;
        for (int lv = 1; lv < H; ++lv)
            for (int o = tp.level_off[lv]; o < tp.level_off[lv + 1]; ++o)
                tp.ops[o].w = (lev[tp.ops[o].y] == lv - 1 ? 1 : 0) | (lev[tp.ops[o].z] == lv - 1 ? 2 : 0);
    }
    // the top part (levels >= cut) for the shared-memory top kernel: children of top nodes coded
    // as -1 - slot (a tip), their top index, or n_top + their boundary index
    const int o_cut = tp.level_off[cut];
    const int n_top = (N - 1) - o_cut;
    std::vector<int> top_index(n, -1), bnd_index(n, -1);
    for (int o = o_cut; o < N - 1; ++o) top_index[tp.ops[o].x] = o - o_cut;
    std::vector<int2> top_code(std::max(n_top, 1));
    std::vector<int> bnd_node;
    int n_tip_children = 0;
    for (int o = o_cut; o < N - 1; ++o) {
        int cc[2];
        for (int side = 0; side < 2; ++side) {
            const int c = side ? tp.ops[o].z : tp.ops[o].y;
            if (c < N) cc[side] = -1 - n_tip_children++;   // a tip: its slot among the top's tips
            else if (top_index[c] >= 0) cc[side] = top_index[c];
            else {
                if (bnd_index[c] < 0) { bnd_index[c] = (int)bnd_node.size(); bnd_node.push_back(c); }
                cc[side] = n_top + bnd_index[c];
            }
        }
        top_code[o - o_cut] = int2{cc[0], cc[1]};
    }
    const int n_bnd = (int)bnd_node.size();
    const int M = pr->n_models;

    Carver cv;
    const size_t o_ops = cv.take<int4>(N - 1), o_lv = cv.take<int>(H + 1);
    const size_t o_tips = cv.take<uint8_t>((size_t)N * Ps), o_w = cv.take<double>(Ps);
    const size_t o_wf = cv.take<float>(Ps), o_rl = f64 ? 0 : cv.take<double>(Ps);
    const size_t o_Qd = cv.take<double>((size_t)M * 16), o_Qf = cv.take<float4>((size_t)M * 4);
    const size_t o_Mp = cv.take<double>((size_t)M * (pg::kTaylorDeg + 1) * 16), o_qn = cv.take<double>(M);
    const size_t o_bm = pr->branch_model ? cv.take<int>(n) : 0;
    Carver sc;   // per-evaluation arrays (see Scratch)
    const size_t o_P = f64 ? sc.take<double2>((size_t)n * C * pg::kPtab64Pairs)
                           : sc.take<float4>((size_t)n * C * pg::kPtabCols);
    const size_t part = (size_t)(N - 1) * C * Ps * (f64 ? 2 : 1);   // float4 or 2 x double2
    const size_t o_post = f64 ? sc.take<double2>(part) : sc.take<float4>(part);
    const size_t o_pre = f64 ? sc.take<double2>(part) : sc.take<float4>(part);
    const size_t o_pe = sc.take<int>((size_t)(N - 1) * Ps), o_qe = sc.take<int>((size_t)(N - 1) * Ps);
    const size_t o_gp = sc.take<double>((size_t)n * slot_cap), o_hp = sc.take<double>((size_t)n * slot_cap);
    const size_t o_lp = sc.take<double>(slot_cap), o_st = cv.take<int>(1);
    const size_t o_plv = cv.take<int>(n), o_sinv = sc.take<float>(std::max(Ps, 16));
    const size_t o_desc = cv.take<pg::ProbDesc>(1);
    const size_t o_ser = sc.take<int>(std::max(Ps, 16));
    const size_t scratch_bytes = align_up(sc.off, 256);
    if (ext && ext->bytes < scratch_bytes) return fail(PG_ERR_INVALID, "shared scratch too small");
    const size_t o_scr = ext ? 0 : cv.take<char>(scratch_bytes);
    if (scratch_need) {
        *scratch_need = scratch_bytes;
        return PG_OK;
    }
    const size_t o_tc = cv.take<int2>(top_code.size()), o_bn = cv.take<int>(std::max(n_bnd, 1));
    const size_t o_par = cv.take<int>(n);
    const size_t o_ib = cv.take<double>(n), o_il = cv.take<double>(1), o_ig = cv.take<double>(n);
    const size_t o_ih = cv.take<double>(n), o_is = cv.take<double>(std::max(P, 1));
    const size_t bytes = align_up(cv.off, 256);

    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", ctx->device);
    void *block = nullptr;
    if (pg_status st = acquire_block(ctx, pl, bytes, &block); st != PG_OK) return st;
    char *base = static_cast<char *>(block);
    pg_handle *h = new (std::nothrow) pg_handle;
    if (!h) { release_block(pl, block); return fail(PG_ERR_OOM, "host allocation failed"); }
    h->ctx = ctx;
    h->block = block;
    h->bytes = bytes;
    h->external = pl != nullptr;
    h->max_tiles = max_tiles;

    // Taylor coefficients Q^k / k! and ||Q||_1 per model (FP64, host, once per upload)
    std::vector<double> Mpow((size_t)M * (pg::kTaylorDeg + 1) * 16), qnorm(M);
    for (int md = 0; md < M; ++md) {
        const double *Q = pr->Q + (size_t)md * 16;
        double *Mk = Mpow.data() + (size_t)md * (pg::kTaylorDeg + 1) * 16;
        for (int u = 0; u < 16; ++u) Mk[u] = (u % 5 == 0) ? 1.0 : 0.0;
        for (int k = 1; k <= pg::kTaylorDeg; ++k)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int t = 0; t < 4; ++t) acc += Mk[(k - 1) * 16 + r * 4 + t] * Q[t * 4 + c];
                    Mk[k * 16 + r * 4 + c] = acc / (double)k;
                }
        double nrm = 0.0;
        for (int c = 0; c < 4; ++c)
            nrm = std::max(nrm, std::fabs(Q[c]) + std::fabs(Q[4 + c]) + std::fabs(Q[8 + c]) + std::fabs(Q[12 + c]));
        qnorm[md] = nrm;
    }
    std::vector<float4> Qf((size_t)M * 4);
    for (int md = 0; md < M; ++md)
        for (int c = 0; c < 4; ++c) {
            const double *Q = pr->Q + (size_t)md * 16;
            Qf[md * 4 + c] = make_float4((float)Q[c], (float)Q[4 + c], (float)Q[8 + c], (float)Q[12 + c]);
        }
    auto cp = [&](size_t off, const void *src, size_t nbytes) -> cudaError_t {
        return h2d(pl, base + off, src, nbytes);
    };
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cp(o_ops, tp.ops.data(), sizeof(int4) * tp.ops.size());
    if (e == cudaSuccess) e = cp(o_lv, tp.level_off.data(), sizeof(int) * tp.level_off.size());
    std::vector<float> wf(Ps, 0.f);
    for (int p = 0; p < P; ++p) wf[p] = (float)pr->pattern_weights[p];
    if (e == cudaSuccess && P > 0)
        e = h2d_rows(pl, base + o_tips, Ps, pr->tip_states, pr->tip_stride ? pr->tip_stride : P, P, N);
    if (e == cudaSuccess && P > 0) e = cp(o_w, pr->pattern_weights, sizeof(double) * P);
    if (e == cudaSuccess && P > 0) e = cp(o_wf, wf.data(), sizeof(float) * Ps);
    if (!f64 && P > 0) {   // N log r_p of the FP32 kernels' pattern factors
        std::vector<double> rl(Ps, 0.0);
        for (int p = 0; p < P; ++p) rl[p] = (double)N * std::log((double)host_pattern_factor((uint32_t)p));
        if (e == cudaSuccess) e = cp(o_rl, rl.data(), sizeof(double) * Ps);
    }
    if (e == cudaSuccess) e = cp(o_Qd, pr->Q, sizeof(double) * 16 * M);
    if (e == cudaSuccess) e = cp(o_Qf, Qf.data(), sizeof(float4) * Qf.size());
    if (e == cudaSuccess) e = cp(o_Mp, Mpow.data(), sizeof(double) * Mpow.size());
    if (e == cudaSuccess) e = cp(o_qn, qnorm.data(), sizeof(double) * M);
    if (e == cudaSuccess && pr->branch_model) e = cp(o_bm, pr->branch_model, sizeof(int) * n);
    if (e == cudaSuccess) e = cp(o_plv, plevel.data(), sizeof(int) * plevel.size());
    if (e == cudaSuccess) e = cp(o_tc, top_code.data(), sizeof(int2) * top_code.size());
    if (e == cudaSuccess && n_bnd > 0) e = cp(o_bn, bnd_node.data(), sizeof(int) * n_bnd);
    if (e == cudaSuccess) e = cp(o_par, pr->parent, sizeof(int) * n);
    if (e == cudaSuccess) e = dzero(pl, base + o_st, sizeof(int));
    if (e != cudaSuccess) {
        release_block(pl, block);
        delete h;
        return fail(PG_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }

    pg::ProbDesc &d = h->desc;
    d.ops = reinterpret_cast<const int4 *>(base + o_ops);
    d.level_off = reinterpret_cast<const int *>(base + o_lv);
    d.tips = reinterpret_cast<const uint8_t *>(base + o_tips);
    d.weights = reinterpret_cast<const double *>(base + o_w);
    d.wf = reinterpret_cast<const float *>(base + o_wf);
    d.rlog = (f64 || P == 0) ? nullptr : reinterpret_cast<const double *>(base + o_rl);
    d.Qd = reinterpret_cast<const double *>(base + o_Qd);
    d.Qf = reinterpret_cast<const float4 *>(base + o_Qf);
    d.Mpow = reinterpret_cast<const double *>(base + o_Mp);
    d.qnorm = reinterpret_cast<const double *>(base + o_qn);
    d.bmodel = pr->branch_model ? reinterpret_cast<const int *>(base + o_bm) : nullptr;
    char *scr = ext ? ext->base : base + o_scr;
    d.Ptab = f64 ? nullptr : reinterpret_cast<float4 *>(scr + o_P);
    d.Ptab64 = f64 ? reinterpret_cast<double2 *>(scr + o_P) : nullptr;
    d.post = scr + o_post;
    d.pre = scr + o_pre;
    d.pe = reinterpret_cast<int *>(scr + o_pe);
    d.qe = reinterpret_cast<int *>(scr + o_qe);
    d.gpart = reinterpret_cast<double *>(scr + o_gp);
    d.hpart = reinterpret_cast<double *>(scr + o_hp);
    d.lpart = reinterpret_cast<double *>(scr + o_lp);
    d.status = reinterpret_cast<int *>(base + o_st);
    d.plevel = reinterpret_cast<const int *>(base + o_plv);
    d.site_invL = reinterpret_cast<float *>(scr + o_sinv);
    d.site_Er = reinterpret_cast<int *>(scr + o_ser);
    d.level_ranges = level_ranges;
    d.n_top = n_top;
    d.n_bnd = n_bnd;
    d.top_code = reinterpret_cast<const int2 *>(base + o_tc);
    d.bnd_node = reinterpret_cast<const int *>(base + o_bn);
    h->d_parent = reinterpret_cast<const int *>(base + o_par);
    d.cut = 0;
    h->cut = cut;
    h->level_off = tp.level_off;
    h->level_cherry.assign(H, 1);
    for (int lv = 0; lv < H; ++lv)
        for (int o = tp.level_off[lv]; o < tp.level_off[lv + 1]; ++o)
            if (tp.ops[o].y >= N || tp.ops[o].z >= N) h->level_cherry[lv] = 0;
    {
        // algorithmic bytes per node: partial + log2 scale per internal node stream, tip codes
        const uint64_t row = (uint64_t)P * ((f64 ? 32ull : 16ull) * C + 4ull), tiprow = (uint64_t)P;
        for (int lv = 0; lv < H; ++lv) {
            uint64_t post_b = 0, pre_b = 0;
            for (int o = tp.level_off[lv]; o < tp.level_off[lv + 1]; ++o) {
                const int4 op = tp.ops[o];
                const bool root = op.x == tp.root;
                post_b += root ? 0 : row;                     // write p_k (the root's is not stored)
                pre_b += root ? 0 : row;                      // read q_k
                for (int c : {op.y, op.z}) {
                    post_b += c < N ? tiprow : row;           // read p_c or the tip codes
                    pre_b += c < N ? tiprow : 2 * row;        // read p_c and write q_c, or tip codes
                }
            }
            if (lv < cut) { h->post_levels_bytes += post_b; h->pre_levels_bytes += pre_b; }
            else h->fused_bytes += post_b + pre_b;
        }
    }
    h->io_b = reinterpret_cast<double *>(base + o_ib);
    h->io_logL = reinterpret_cast<double *>(base + o_il);
    h->io_grad = reinterpret_cast<double *>(base + o_ig);
    h->io_hess = reinterpret_cast<double *>(base + o_ih);
    h->io_site = reinterpret_cast<double *>(base + o_is);
    d.n_tips = N;
    d.n_nodes = n;
    d.root = tp.root;
    d.n_levels = H;
    d.P = P;
    d.Ps = Ps;
    d.slot_cap = slot_cap;
    d.C = C;
    d.n_models = M;
    d.precision = pr->precision;
    for (int s = 0; s < pg::kStates; ++s) { d.pi[s] = pr->root_freqs[s]; d.pif[s] = (float)pr->root_freqs[s]; }
    for (int l = 0; l < pg::kMaxCat; ++l) {
        const bool on = l < C;
        d.cw[l] = on ? pr->cat_weights[l] : 0.0;
        d.rates[l] = on ? pr->cat_rates[l] : 0.0;
        d.gw[l] = on ? (float)(pr->cat_rates[l] * pr->cat_weights[l]) : 0.f;
        d.gw2[l] = on ? (float)(pr->cat_rates[l] * pr->cat_rates[l] * pr->cat_weights[l]) : 0.f;
    }

    pg_handle_info &I = h->info;
    I.n_tips = N;
    I.n_nodes = n;
    I.n_states = m;
    I.n_patterns = P;
    I.n_categories = C;
    I.n_levels = H;
    {
        pg::ProbDesc tmp = d;
        set_tiling(tmp, single_target(ctx, tmp), max_range);
        I.n_tiles = tmp.n_tiles;
        I.patterns_per_tile = tmp.range_len;
    }
    I.device_bytes = bytes;
    // post: write N-2 non-root internal partials, read them once as children; pre: read q of the
    // N-2 non-root internal nodes, read their p again, write their q; plus the tip codes twice.
    const uint64_t node_stream = (uint64_t)P * ((f64 ? 32ull : 16ull) * C + 4ull);   // partial + exponent
    I.stream_bytes = 5ull * (uint64_t)(N - 2) * node_stream + 2ull * (uint64_t)N * P;
    I.flops = (uint64_t)(N - 1) * P * C * (68ull + 216ull);

    // the static descriptor in device memory, for launches that cover several problems
    h->d_desc = reinterpret_cast<const pg::ProbDesc *>(base + o_desc);
    if (h2d(pl, base + o_desc, &h->desc, sizeof(pg::ProbDesc)) != cudaSuccess) {
        release_block(pl, block);
        delete h;
        return fail(PG_ERR_CUDA, "upload of the descriptor failed");
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!pl) ctx->used += bytes;
        ctx->handles.push_back(h);
    }
    *out = h;
    return PG_OK;
}

namespace {

// A tree with multifurcations as a binary tree.  The caller's nodes keep their ids 0..n_user-1; a
// node k with children c_0 < c_1 < ... < c_{d-1}, d > 2, keeps c_0 and gets the added node x_1, x_1
// takes c_1 and x_2, ..., x_{d-2} takes c_{d-2} and c_{d-1}.  The added nodes get ids n_user ..
// 2N-2, model 0 and (at evaluation) branch length 0, so that P = I on their branches: every site
// likelihood, and the gradient and Hessian entries of every original branch, are those of the
// multifurcating tree (a branch of length 0 multiplies the partial vector below it by I).
pg_status resolve_multifurcations(const pg_problem *pr, int n_user, std::vector<int32_t> &par,
                                  std::vector<int32_t> &bm) {
    const int N = pr->n_tips, n = 2 * N - 1;
    if (n_user < N + 1 || n_user > n)
        return fail(PG_ERR_INVALID, "n_nodes = %d: between n_tips + 1 = %d and 2 n_tips - 1 = %d", n_user, N + 1, n);
    if (!pr->parent) return fail(PG_ERR_INVALID, "parent is NULL");
    std::vector<std::vector<int>> kids(n_user);
    int root = -1;
    for (int i = 0; i < n_user; ++i) {
        const int p = pr->parent[i];
        if (p == -1) {
            if (root >= 0) return fail(PG_ERR_INVALID, "more than one root (nodes %d and %d)", root, i);
            root = i;
            continue;
        }
        if (p < N || p >= n_user || p == i)
            return fail(PG_ERR_INVALID, "parent[%d] = %d is not an internal node", i, p);
        kids[p].push_back(i);
    }
    if (root < 0) return fail(PG_ERR_INVALID, "no root (no node with parent -1)");
    for (int k = N; k < n_user; ++k)
        if (kids[k].size() < 2) return fail(PG_ERR_INVALID, "internal node %d has fewer than two children", k);
    par.assign(n, -1);
    for (int i = 0; i < n_user; ++i) par[i] = pr->parent[i];
    int next = n_user;
    for (int k = N; k < n_user; ++k) {
        const int d = (int)kids[k].size();
        int host = k;
        for (int j = 1; j < d - 1; ++j) {
            const int x = next++;
            par[x] = host;
            par[kids[k][j]] = x;
            host = x;
        }
        par[kids[k][d - 1]] = host;
    }
    if (next != n) return fail(PG_ERR_INVALID, "the parent array does not describe a tree");
    if (pr->branch_model) {
        bm.assign(n, 0);
        for (int i = 0; i < n_user; ++i) bm[i] = pr->branch_model[i];
    }
    return PG_OK;
}

}  // namespace

namespace {

// A problem whose arrays do not fit the context's budget (or the device) as a whole.  Sites are
// i.i.d. (Section 2.1): the log-likelihood, gradient and Hessian diagonal of the alignment are the
// sums of those of contiguous pattern slices.  The problem is uploaded as K chunks of Pc patterns (a
// multiple of 128, K doubling until it fits) whose per-evaluation arrays (partials, exponents, slot
// sums) share one region sized for one chunk, so the device holds one chunk's partials at a time;
// the parent handle runs the chunks one after another and sums their results in a fixed order.
pg_status upload_chunked(pg_ctx *ctx, const pg_problem *pr, pg_handle **out) {
    const int P = pr->n_patterns, n = 2 * pr->n_tips - 1;
    const size_t stride = pr->tip_stride ? (size_t)pr->tip_stride : (size_t)P;
    const std::string whole = pg::host::g_err;   // why the whole problem did not fit
    auto add_used = [&](long long bytes) {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->used += bytes;
    };
    for (int K = 2;; K *= 2) {
        const int Pc = ((P + K - 1) / K + 127) / 128 * 128;
        if (Pc >= P) {
            if (Pc <= 128) break;
            continue;
        }
        const int nk = (P + Pc - 1) / Pc;
        pg_problem c0 = *pr;
        c0.n_patterns = Pc;
        c0.tip_stride = (int32_t)stride;
        size_t need = 0;
        pg_handle *unused = nullptr;
        pg_status st = upload_binary(ctx, &c0, &unused, nullptr, nullptr, &need);
        if (st != PG_OK) return st;
        // the shared scratch, then the parent's block: io arrays, b of the last forward, parts
        DeviceGuard g(ctx->device);
        void *scratch = nullptr, *pblock = nullptr;
        if (acquire_block(ctx, nullptr, need, &scratch) != PG_OK) {
            if (Pc <= 128) break;
            continue;
        }
        add_used((long long)need);
        Carver cv;
        const size_t o_ib = cv.take<double>(n), o_il = cv.take<double>(1), o_ig = cv.take<double>(n);
        const size_t o_ih = cv.take<double>(n), o_is = cv.take<double>(std::max(P, 1)), o_bf = cv.take<double>(n);
        const size_t o_pt = cv.take<double>((size_t)nk * (1 + 2 * (size_t)n));
        const size_t pbytes = align_up(cv.off, 256);
        std::vector<pg_handle *> chunks;
        auto undo = [&]() {
            for (pg_handle *c : chunks) pg_free(c);
            if (pblock) {
                cudaFree(pblock);
                add_used(-(long long)pbytes);
            }
            cudaFree(scratch);
            add_used(-(long long)need);
        };
        if (acquire_block(ctx, nullptr, pbytes, &pblock) != PG_OK) {
            pblock = nullptr;
            undo();
            if (Pc <= 128) break;
            continue;
        }
        add_used((long long)pbytes);
        Scratch ext;
        ext.base = static_cast<char *>(scratch);
        ext.bytes = need;
        bool room = true;
        for (int j = 0; j < nk; ++j) {
            pg_problem cj = *pr;
            cj.n_patterns = std::min(Pc, P - j * Pc);
            cj.tip_stride = (int32_t)stride;
            cj.tip_states = pr->tip_states + (size_t)j * Pc;
            cj.pattern_weights = pr->pattern_weights + (size_t)j * Pc;
            pg_handle *ch = nullptr;
            st = upload_binary(ctx, &cj, &ch, nullptr, &ext);
            if (st == PG_ERR_OOM) {
                room = false;
                break;
            }
            if (st != PG_OK) {
                undo();
                return st;
            }
            ch->n_user = n;
            chunks.push_back(ch);
        }
        if (!room) {
            undo();
            if (Pc <= 128) break;
            continue;
        }
        pg_handle *h = new (std::nothrow) pg_handle;
        if (!h) {
            undo();
            return fail(PG_ERR_OOM, "host allocation failed");
        }
        {
            std::lock_guard<std::mutex> gl(ctx->mu);   // the parent owns its chunks
            for (pg_handle *c : chunks)
                ctx->handles.erase(std::remove(ctx->handles.begin(), ctx->handles.end(), c), ctx->handles.end());
            ctx->handles.push_back(h);
        }
        pg_handle *c0h = chunks[0];
        h->ctx = ctx;
        h->block = pblock;
        h->bytes = pbytes;
        h->desc = c0h->desc;   // tree, sizes and model of the problem (pointers of chunk 0)
        h->d_parent = c0h->d_parent;
        h->desc.P = P;
        h->mstate = c0h->mstate;
        h->md = c0h->md;
        h->n_user = n;
        h->chunks = chunks;
        for (int j = 0; j < nk; ++j) h->chunk_p0.push_back(j * Pc);
        h->scratch_block = scratch;
        h->scratch_bytes = need;
        char *base = static_cast<char *>(pblock);
        h->io_b = reinterpret_cast<double *>(base + o_ib);
        h->io_logL = reinterpret_cast<double *>(base + o_il);
        h->io_grad = reinterpret_cast<double *>(base + o_ig);
        h->io_hess = reinterpret_cast<double *>(base + o_ih);
        h->io_site = reinterpret_cast<double *>(base + o_is);
        h->b_fwd = reinterpret_cast<double *>(base + o_bf);
        h->part_out = reinterpret_cast<double *>(base + o_pt);
        h->info = c0h->info;
        h->info.n_patterns = P;
        h->info.device_bytes = pbytes + need;
        h->info.stream_bytes = 0;
        h->info.flops = 0;
        for (pg_handle *c : chunks) {
            h->info.device_bytes += c->bytes;
            h->info.stream_bytes += c->info.stream_bytes;
            h->info.flops += c->info.flops;
        }
        *out = h;
        return PG_OK;
    }
    return fail(PG_ERR_OOM, "%s; not even in pattern chunks of 128 patterns", whole.c_str());
}

// upload_binary, and in pattern chunks when the whole problem does not fit (not for a caller's arena)
pg_status upload_fit(pg_ctx *ctx, const pg_problem *pr, pg_handle **out, const Placement *pl) {
    pg_status st = upload_binary(ctx, pr, out, pl);
    if (st == PG_ERR_OOM && !pl && pr->n_patterns > 128) st = upload_chunked(ctx, pr, out);
    return st;
}

}  // namespace

pg_status pg::host::upload(pg_ctx *ctx, const pg_problem *pr, pg_handle **out, const Placement *pl) {
    if (!ctx || !pr || !out) return fail(PG_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const int N = pr->n_tips;
    if (N < 2) return fail(PG_ERR_INVALID, "n_tips = %d (at least 2 required)", N);
    const int n = 2 * N - 1, n_user = pr->n_nodes ? pr->n_nodes : n;
    if (n_user == n) {
        pg_status st = upload_fit(ctx, pr, out, pl);
        if (st == PG_OK) (*out)->n_user = n;
        return st;
    }
    std::vector<int32_t> par, bm;
    pg_status st = resolve_multifurcations(pr, n_user, par, bm);
    if (st != PG_OK) return st;
    pg_problem rb = *pr;
    rb.parent = par.data();
    rb.branch_model = pr->branch_model ? bm.data() : nullptr;
    rb.n_nodes = n;
    st = upload_fit(ctx, &rb, out, pl);
    if (st != PG_OK) return st;
    pg_handle *h = *out;
    h->n_user = n_user;
    h->info.n_nodes = n_user;
    // the added nodes' branch lengths stay 0: the caller's lengths fill entries 0 .. n_user-1
    DeviceGuard g(ctx->device);
    cudaError_t e = dzero(pl, h->io_b, sizeof(double) * n);
    if (e != cudaSuccess) {
        pg_free(h);
        *out = nullptr;
        return fail(PG_ERR_CUDA, "upload: %s", cudaGetErrorString(e));
    }
    return PG_OK;
}

extern "C" {

pg_status pg_get_info(const pg_handle *h, pg_handle_info *out) {
    if (!h || !out) return fail(PG_ERR_INVALID, "NULL argument");
    *out = h->info;
    return PG_OK;
}

}  // extern "C"

namespace {

void fill_args_one(pg::BatchArgs<1> &a, const pg::ProbDesc &d) {
    a.n = 1;
    a.tile_base[0] = 0;
    a.tile_base[1] = d.n_tiles;
    a.mat_base[0] = 0;
    a.mat_base[1] = d.n_nodes * d.C;
    a.red_base[0] = 0;
    a.red_base[1] = d.n_nodes + 1;
    a.d[0] = d;
}

}  // namespace

namespace {

// One problem alone: the P build and the wide post-order levels as level kernels, the levels from
// the cut up in the shared-memory top kernel (or the fused kernel), the pre-order levels, the
// fixed-order reduction.  skip = kSkipPre enqueues the forward part (logL), kSkipPost the backward
// part (gradient, Hessian diagonal) on the partials the last forward part left in the handle.
pg_status enqueue_chunked(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad,
                          double *d_hess, double *d_site_logL, const double *d_gscale, cudaStream_t s);

// phase-timing mode 3 times the pre-order levels of one evaluation in this many
constexpr long long kTimingEvery = 8;

pg_status enqueue_single(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad,
                         double *d_hess, double *d_site_logL, const double *d_gscale, cudaStream_t s) {
    if (!h->chunks.empty()) return enqueue_chunked(h, skip, d_b, d_logL, d_grad, d_hess, d_site_logL, d_gscale, s);
    if (h->mstate) return enqueue_m(h, skip, d_b, d_logL, d_grad, d_hess, d_site_logL, d_gscale, s);
    pg::BatchArgs<1> a;
    pg::ProbDesc d = h->desc;
    d.b = d_b;
    d.out_logL = d_logL;
    d.out_grad = d_grad;
    d.out_hess = d_hess;
    d.out_site = d_site_logL;
    d.gscale = d_gscale;
    d.skip = skip;
    const bool fwd = !(skip & pg::kSkipPost), bwd = !(skip & pg::kSkipPre);
    const int max_range = h->ctx->max_range ? h->ctx->max_range : pg::kMaxRange;
    d.cut = d.P > 0 ? h->cut : 0;
    // FP32: the levels from the cut up run in the shared-memory top kernel when its per-block
    // partials fit (two blocks per SM, else one); otherwise in the fused kernel
    bool use_top = false;
    if (d.precision == PG_PRECISION_FP32 && d.P > 0) {
        for (int k = 2; k >= 1 && !use_top; --k) {
            set_tiling(d, k * h->ctx->n_sm, max_range);
            use_top = (size_t)k * (pg::top_smem_bytes(d) + 1024) <= (size_t)228 * 1024;   // 1 KB reserved per block
        }
    }
    // FP64: the whole tree pass in the shared-memory latency kernel when a block's vectors fit at
    // one block per SM (one slot per block and branch); otherwise in the fused kernel
    if (d.precision == PG_PRECISION_FP64 && d.P > 0 && !(h->ctx->flags & PG_FLAG_FP64_DEVICE_PARTIALS)) {
        set_tiling(d, h->ctx->n_sm, max_range);
        d.pieces = 1;
        d.n_tg = d.n_tiles;
        d.small64 = pg::small64_smem_bytes(d) != 0;
    }
    if (!use_top && !d.small64) set_tiling(d, single_target(h->ctx, d), max_range);
    fill_args_one(a, d);
    const bool hess = bwd && d_hess != nullptr;
    // phase timing: events at the six phase boundaries (mode 1), or only around the pre-order
    // levels (mode 2: marks 3 and 4; a timed event waits for all earlier work, so each one also
    // ends the programmatic overlap of the launches on either side)
    int tmode = (fwd && bwd) ? h->timing : 0;
    if (tmode == 3) tmode = (h->timing_count % kTimingEvery == 0) ? 2 : 0;   // sampled
    if (fwd && bwd) ++h->timing_count;
    const int n_ev = tmode == 1 ? 6 : (tmode == 2 ? 2 : 0);
    cudaEvent_t ev[6] = {};
    for (int i = 0; i < n_ev; ++i)
        if (cudaEventCreate(&ev[i]) != cudaSuccess) return fail(PG_ERR_CUDA, "cudaEventCreate failed");
    h->events.insert(h->events.end(), ev, ev + n_ev);
    auto mark = [&](int i) {
        if (tmode == 1) cudaEventRecord(ev[i], s);
        else if (tmode == 2 && (i == 3 || i == 4)) cudaEventRecord(ev[i - 3], s);
    };
    Range range(fwd && bwd ? "pg evaluation" : (fwd ? "pg forward" : "pg backward"));
    cudaError_t e = cudaSuccess;
    mark(0);
    if (fwd) e = pg::launch_pmatrix<1>(a, s);
    mark(1);
    for (int lv = 0; fwd && e == cudaSuccess && lv < d.cut; ++lv)
        e = pg::launch_post_level(d, h->level_off[lv], h->level_off[lv + 1] - h->level_off[lv], h->ctx->n_sm,
                                  h->level_cherry[lv] != 0, s);
    mark(2);
    if (e == cudaSuccess) e = use_top ? pg::launch_top(a, hess, h->ctx->n_sm, s) : pg::launch_tree<1>(a, hess, s);
    mark(3);
    // The first pre-order level is a plain launch: scheduled while the top kernel ran (programmatic
    // launch), it made the evaluation slower, 0.730 against 0.694 ms in the nucleotide configuration.
    for (int lv = d.cut - 1; bwd && e == cudaSuccess && lv >= 0; --lv)
        e = pg::launch_pre_level(d, h->level_off[lv], h->level_off[lv + 1] - h->level_off[lv], hess, h->ctx->n_sm,
                                 h->level_cherry[lv] != 0, s, lv != d.cut - 1);
    mark(4);
    if (e == cudaSuccess) e = pg::launch_reduce<1>(a, hess, s);
    mark(5);
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    h->last_stream = s;
    if (fwd) h->have_post = true;
    return PG_OK;
}

// A problem evaluated in pattern chunks (see upload_chunked): the chunks run one after another on
// stream s, each writing its logL, gradient and Hessian diagonal to its slot of part_out (its site
// log-likelihoods straight to its slice of d_site_logL), then fixed-order sums give the outputs.
// The forward part keeps no partials (the next chunk overwrites them): it stores b for the backward
// part, which runs each chunk's whole evaluation again -- the post-order partials of the chunk are
// recomputed before its pre-order pass.
pg_status enqueue_chunked(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad,
                          double *d_hess, double *d_site_logL, const double *d_gscale, cudaStream_t s) {
    const int K = (int)h->chunks.size(), n = h->desc.n_nodes;
    const bool fwd = !(skip & pg::kSkipPost), bwd = !(skip & pg::kSkipPre);
    double *p_l = h->part_out, *p_g = p_l + K, *p_h = p_g + (size_t)K * n;
    const double *b = d_b;
    if (fwd && !bwd) PG_CUDA(cudaMemcpyAsync(h->b_fwd, d_b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    if (!fwd) b = h->b_fwd;
    for (int j = 0; j < K; ++j) {
        pg_handle *c = h->chunks[j];
        const int sk = (fwd && !bwd) ? pg::kSkipPre : 0;
        pg_status st = enqueue_single(c, sk, b, p_l + j, (bwd && d_grad) ? p_g + (size_t)j * n : nullptr,
                                      (bwd && d_hess) ? p_h + (size_t)j * n : nullptr,
                                      (fwd && d_site_logL) ? d_site_logL + h->chunk_p0[j] : nullptr,
                                      bwd ? d_gscale : nullptr, s);
        if (st != PG_OK) return st;
    }
    cudaError_t e = cudaSuccess;
    if (fwd && d_logL) e = pg::launch_chunk_sum(p_l, K, 1, d_logL, s);
    if (e == cudaSuccess && bwd && d_grad) e = pg::launch_chunk_sum(p_g, K, n, d_grad, s);
    if (e == cudaSuccess && bwd && d_hess) e = pg::launch_chunk_sum(p_h, K, n, d_hess, s);
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    h->last_stream = s;
    if (fwd) h->have_post = true;
    return PG_OK;
}

// k problems in as few launches as possible: grouped by category count and precision, each
// launch covers every tile of every problem of the group, every level in the fused kernel
// patterns per tile of the fused kernel when it runs only the root's level of a batch
constexpr int kRootRange = 512;

pg_status enqueue_batch(pg_handle *const *hs, int32_t k, int skip, const double *const *d_b, double *d_logL,
                        double *const *d_grad, double *const *d_hess, const double *d_gscale, cudaStream_t s) {
    const bool fwd = !(skip & pg::kSkipPost), bwd = !(skip & pg::kSkipPre);
    DeviceGuard g(hs[0]->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", hs[0]->ctx->device);
    for (int i = 0; i < k; ++i) {   // general state spaces and chunked problems: their own launches
        if (!hs[i]->mstate && hs[i]->chunks.empty()) continue;
        if (!hs[i]->chunks.empty()) {
            pg_status st = enqueue_chunked(hs[i], skip, d_b ? d_b[i] : nullptr, d_logL ? d_logL + i : nullptr,
                                           (bwd && d_grad) ? d_grad[i] : nullptr, (bwd && d_hess) ? d_hess[i] : nullptr,
                                           nullptr, d_gscale ? d_gscale + i : nullptr, s);
            if (st != PG_OK) return st;
            continue;
        }
        pg_status st = enqueue_m(hs[i], skip, d_b ? d_b[i] : nullptr, d_logL ? d_logL + i : nullptr,
                                 (bwd && d_grad) ? d_grad[i] : nullptr, (bwd && d_hess) ? d_hess[i] : nullptr,
                                 nullptr, d_gscale ? d_gscale + i : nullptr, s);
        if (st != PG_OK) return st;
    }
    for (int key = 0; key < 2 * pg::kMaxCat; ++key) {
        const int C = 1 + key / 2, prec = key % 2;
        std::vector<int> idx;
        for (int i = 0; i < k; ++i)
            if (!hs[i]->mstate && hs[i]->chunks.empty() && hs[i]->desc.C == C && hs[i]->desc.precision == prec)
                idx.push_back(i);
        if (idx.empty()) continue;
        // the fused-kernel, P-build and reduction launches take groups of up to kMaxBatch problems
        // (descriptors by value); the level launches cover every problem of the key at once
        const size_t n_groups = (idx.size() + pg::kMaxBatch - 1) / pg::kMaxBatch;
        std::vector<pg::BatchArgs<pg::kMaxBatch>> groups;
        try {
            groups.resize(n_groups);
        } catch (...) {
            return fail(PG_ERR_OOM, "host allocation failed");
        }
        std::vector<int> cut_of(idx.size());
        bool hess = false;
        for (size_t gi = 0; gi < n_groups; ++gi) {
            pg::BatchArgs<pg::kMaxBatch> &a = groups[gi];
            const size_t at = gi * pg::kMaxBatch;
            const int cnt = (int)std::min<size_t>(pg::kMaxBatch, idx.size() - at);
            a.n = cnt;
            a.tile_base[0] = a.mat_base[0] = a.red_base[0] = 0;
            // blocks in proportion to each problem's partial-stream work, one wave in total
            double work = 0.0;
            for (int j = 0; j < cnt; ++j) work += (double)hs[idx[at + j]]->info.stream_bytes + 1.0;
            const pg_ctx *cx = hs[0]->ctx;
            const int slots = cx->n_sm * cx->blocks_per_sm[prec][C];
            const int max_range = cx->max_range ? cx->max_range : pg::kMaxRange;
            for (int j = 0; j < cnt; ++j) {
                const int i = idx[at + j];
                pg::ProbDesc d = hs[i]->desc;
                const double share = ((double)hs[i]->info.stream_bytes + 1.0) / work;
                int target = std::max(1, (int)(slots * share));
                // FP32: the fused kernel runs the root's level alone, one short step per tile, so
                // the tiles are many and small rather than one wave of long ones
                if (prec == PG_PRECISION_FP32) target = std::max(target, (d.P + kRootRange - 1) / kRootRange);
                set_tiling(d, std::min(hs[i]->max_tiles, target), max_range);
                d.b = d_b ? d_b[i] : nullptr;
                d.out_logL = d_logL ? d_logL + i : nullptr;
                d.out_grad = (bwd && d_grad) ? d_grad[i] : nullptr;
                d.out_hess = (bwd && d_hess) ? d_hess[i] : nullptr;
                d.out_site = nullptr;
                d.gscale = d_gscale ? d_gscale + i : nullptr;
                d.skip = skip;
                // FP32: every level below the root's in batched level kernels, the root's level
                // in the fused kernel; FP64: every level in the fused kernel
                d.cut = (prec == PG_PRECISION_FP32 && d.P > 0) ? d.n_levels - 1 : 0;
                cut_of[at + j] = d.cut;
                hess = hess || d.out_hess;
                a.d[j] = d;
                a.tile_base[j + 1] = a.tile_base[j] + d.n_tiles;
                a.mat_base[j + 1] = a.mat_base[j] + d.n_nodes * d.C;
                a.red_base[j + 1] = a.red_base[j] + d.n_nodes + 1;
                hs[i]->last_stream = s;
                if (fwd) hs[i]->have_post = true;
            }
        }
        int max_cut = 0;
        for (int cu : cut_of) max_cut = std::max(max_cut, cu);
        const int n_sm = hs[0]->ctx->n_sm;
        // one launch per level index over every problem that takes part (L < its cut), up to
        // kMaxLevelBatch problems per launch
        auto levels = [&](int L, bool post) -> cudaError_t {
            pg::LevelBatch lb;
            lb.n = 0;
            lb.base[0] = 0;
            for (size_t j = 0; j <= idx.size(); ++j) {
                if (j == idx.size() || lb.n == pg::kMaxLevelBatch) {
                    if (lb.n) {
                        cudaError_t e = post ? pg::launch_post_level_batch(lb, C, n_sm, L == 0, s)
                                             : pg::launch_pre_level_batch(lb, C, hess, n_sm, L == 0, s);
                        if (e != cudaSuccess) return e;
                    }
                    lb.n = 0;
                    if (j == idx.size()) break;
                }
                if (L >= cut_of[j]) continue;
                const pg_handle *hj = hs[idx[j]];
                const int o0 = hj->level_off[L], nd = hj->level_off[L + 1] - o0;
                // level 0 holds the cherries, whose items take several ranges
                const int nr = L > 0 ? hj->desc.level_ranges
                                     : pg::level_items_per_node(hj->desc.P, C, post ? pg::post_cherry_ranges(C)
                                                                                    : pg::pre_cherry_ranges(C));
                lb.d[lb.n] = hj->d_desc;
                lb.o0[lb.n] = o0;
                lb.nr[lb.n] = nr;
                lb.base[lb.n + 1] = lb.base[lb.n] + nd * nr;
                ++lb.n;
            }
            return cudaSuccess;
        };
        cudaError_t e = cudaSuccess;
        for (size_t gi = 0; fwd && e == cudaSuccess && gi < n_groups; ++gi) e = pg::launch_pmatrix<pg::kMaxBatch>(groups[gi], s);
        for (int L = 0; fwd && e == cudaSuccess && L < max_cut; ++L) e = levels(L, true);
        for (size_t gi = 0; e == cudaSuccess && gi < n_groups; ++gi) e = pg::launch_tree<pg::kMaxBatch>(groups[gi], hess, s);
        for (int L = max_cut - 1; bwd && e == cudaSuccess && L >= 0; --L) e = levels(L, false);
        for (size_t gi = 0; e == cudaSuccess && gi < n_groups; ++gi) e = pg::launch_reduce<pg::kMaxBatch>(groups[gi], hess, s);
        if (e != cudaSuccess) return fail(PG_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    }
    return PG_OK;
}

pg_status check_batch(pg_handle *const *hs, int32_t k) {
    if (k < 0 || (k > 0 && !hs)) return fail(PG_ERR_INVALID, "bad batch arguments");
    for (int i = 0; i < k; ++i) {
        if (!hs[i]) return fail(PG_ERR_INVALID, "batch entry %d is NULL", i);
        if (hs[i]->ctx != hs[0]->ctx) return fail(PG_ERR_INVALID, "batch mixes contexts");
    }
    return PG_OK;
}

// The public entry points take per-node arrays of the caller's n_user nodes.  A handle that holds a
// resolved multifurcating tree evaluates on its full-size buffers: the branch lengths are copied
// into io_b (whose added entries stay 0), the gradient and Hessian diagonal are written to io_grad
// and io_hess and their first n_user entries (the caller's nodes) copied out.
pg_status enqueue_user(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad, double *d_hess,
                       double *d_site_logL, const double *d_gscale, cudaStream_t s) {
    const int nu = h->n_user;
    if (nu == h->desc.n_nodes)
        return enqueue_single(h, skip, d_b, d_logL, d_grad, d_hess, d_site_logL, d_gscale, s);
    const size_t bytes = sizeof(double) * nu;
    if (d_b) PG_CUDA(cudaMemcpyAsync(h->io_b, d_b, bytes, cudaMemcpyDeviceToDevice, s));
    pg_status st = enqueue_single(h, skip, d_b ? h->io_b : nullptr, d_logL, d_grad ? h->io_grad : nullptr,
                                  d_hess ? h->io_hess : nullptr, d_site_logL, d_gscale, s);
    if (st != PG_OK) return st;
    if (d_grad) PG_CUDA(cudaMemcpyAsync(d_grad, h->io_grad, bytes, cudaMemcpyDeviceToDevice, s));
    if (d_hess) PG_CUDA(cudaMemcpyAsync(d_hess, h->io_hess, bytes, cudaMemcpyDeviceToDevice, s));
    return PG_OK;
}

// The same for a batch: per-problem pointer arrays with the resolved handles' entries replaced by
// their full-size buffers (remap_in), and the caller's entries copied out afterwards (remap_out).
struct BatchPtrs {
    std::vector<const double *> b;
    std::vector<double *> g, h;
};
pg_status remap_in(pg_handle *const *hs, int32_t k, const double *const *d_b, double *const *d_grad,
                   double *const *d_hess, cudaStream_t s, BatchPtrs &bp) {
    if (d_b) bp.b.assign(d_b, d_b + k);
    if (d_grad) bp.g.assign(d_grad, d_grad + k);
    if (d_hess) bp.h.assign(d_hess, d_hess + k);
    for (int i = 0; i < k; ++i) {
        pg_handle *h = hs[i];
        if (h->n_user == h->desc.n_nodes) continue;
        if (d_b && d_b[i]) {
            PG_CUDA(cudaMemcpyAsync(h->io_b, d_b[i], sizeof(double) * h->n_user, cudaMemcpyDeviceToDevice, s));
            bp.b[i] = h->io_b;
        }
        if (d_grad && d_grad[i]) bp.g[i] = h->io_grad;
        if (d_hess && d_hess[i]) bp.h[i] = h->io_hess;
    }
    return PG_OK;
}
pg_status remap_out(pg_handle *const *hs, int32_t k, double *const *d_grad, double *const *d_hess, cudaStream_t s) {
    for (int i = 0; i < k; ++i) {
        pg_handle *h = hs[i];
        if (h->n_user == h->desc.n_nodes) continue;
        const size_t bytes = sizeof(double) * h->n_user;
        if (d_grad && d_grad[i]) PG_CUDA(cudaMemcpyAsync(d_grad[i], h->io_grad, bytes, cudaMemcpyDeviceToDevice, s));
        if (d_hess && d_hess[i]) PG_CUDA(cudaMemcpyAsync(d_hess[i], h->io_hess, bytes, cudaMemcpyDeviceToDevice, s));
    }
    return PG_OK;
}

}  // namespace

pg_status pg::host::enqueue(pg_handle *h, int skip, const double *d_b, double *d_logL, double *d_grad,
                           double *d_hess, double *d_site_logL, const double *d_gscale, cudaStream_t s) {
    DeviceGuard g(h->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", h->ctx->device);
    return enqueue_single(h, skip, d_b, d_logL, d_grad, d_hess, d_site_logL, d_gscale, s);
}

extern "C" {

pg_status pg_eval_async(pg_handle *h, const double *d_b, double *d_logL, double *d_grad,
                        double *d_hess, double *d_site_logL, void *stream) {
    if (!h || !d_b) return fail(PG_ERR_INVALID, "NULL handle or branch lengths");
    DeviceGuard g(h->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", h->ctx->device);
    return enqueue_user(h, 0, d_b, d_logL, d_grad, d_hess, d_site_logL, nullptr, static_cast<cudaStream_t>(stream));
}

pg_status pg_forward_async(pg_handle *h, const double *d_b, double *d_logL, double *d_site_logL, void *stream) {
    if (!h || !d_b) return fail(PG_ERR_INVALID, "NULL handle or branch lengths");
    DeviceGuard g(h->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", h->ctx->device);
    return enqueue_user(h, pg::kSkipPre, d_b, d_logL, nullptr, nullptr, d_site_logL, nullptr,
                        static_cast<cudaStream_t>(stream));
}

pg_status pg_backward_async(pg_handle *h, const double *d_gscale, double *d_grad, double *d_hess, void *stream) {
    if (!h) return fail(PG_ERR_INVALID, "NULL handle");
    if (!h->have_post) return fail(PG_ERR_INVALID, "no forward pass has been enqueued on this handle");
    DeviceGuard g(h->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", h->ctx->device);
    return enqueue_user(h, pg::kSkipPost, nullptr, nullptr, d_grad, d_hess, nullptr, d_gscale,
                        static_cast<cudaStream_t>(stream));
}

pg_status pg_eval_batch_async(pg_handle *const *hs, int32_t k, const double *const *d_b,
                              double *d_logL, double *const *d_grad, double *const *d_hess,
                              void *stream) {
    if (pg_status st = check_batch(hs, k); st != PG_OK) return st;
    if (k > 0 && (!d_b || !d_logL)) return fail(PG_ERR_INVALID, "bad batch arguments");
    for (int i = 0; i < k; ++i)
        if (!d_b[i]) return fail(PG_ERR_INVALID, "batch entry %d is NULL", i);
    if (k == 0) return PG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard g(hs[0]->ctx->device);
    BatchPtrs bp;
    if (pg_status st = remap_in(hs, k, d_b, d_grad, d_hess, s, bp); st != PG_OK) return st;
    pg_status st = enqueue_batch(hs, k, 0, bp.b.data(), d_logL, d_grad ? bp.g.data() : nullptr,
                                 d_hess ? bp.h.data() : nullptr, nullptr, s);
    return st != PG_OK ? st : remap_out(hs, k, d_grad, d_hess, s);
}

pg_status pg_forward_batch_async(pg_handle *const *hs, int32_t k, const double *const *d_b, double *d_logL,
                                 void *stream) {
    if (pg_status st = check_batch(hs, k); st != PG_OK) return st;
    if (k > 0 && (!d_b || !d_logL)) return fail(PG_ERR_INVALID, "bad batch arguments");
    for (int i = 0; i < k; ++i)
        if (!d_b[i]) return fail(PG_ERR_INVALID, "batch entry %d is NULL", i);
    if (k == 0) return PG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard g(hs[0]->ctx->device);
    BatchPtrs bp;
    if (pg_status st = remap_in(hs, k, d_b, nullptr, nullptr, s, bp); st != PG_OK) return st;
    return enqueue_batch(hs, k, pg::kSkipPre, bp.b.data(), d_logL, nullptr, nullptr, nullptr, s);
}

pg_status pg_backward_batch_async(pg_handle *const *hs, int32_t k, const double *d_gscale,
                                  double *const *d_grad, double *const *d_hess, void *stream) {
    if (pg_status st = check_batch(hs, k); st != PG_OK) return st;
    for (int i = 0; i < k; ++i)
        if (!hs[i]->have_post) return fail(PG_ERR_INVALID, "batch entry %d has no forward pass", i);
    if (k == 0) return PG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceGuard g(hs[0]->ctx->device);
    BatchPtrs bp;
    if (pg_status st = remap_in(hs, k, nullptr, d_grad, d_hess, s, bp); st != PG_OK) return st;
    pg_status st = enqueue_batch(hs, k, pg::kSkipPost, nullptr, nullptr, d_grad ? bp.g.data() : nullptr,
                                 d_hess ? bp.h.data() : nullptr, d_gscale, s);
    return st != PG_OK ? st : remap_out(hs, k, d_grad, d_hess, s);
}

namespace {

pg_status enqueue_clock(pg_handle *const *hs, int32_t k, bool grad, const double *const *d_eps,
                        const double *d_mu, const double *const *d_t, double *const *d_b,
                        const double *const *d_grad_b, double *const *d_grad_eps, double *d_grad_mu,
                        double *const *d_grad_t, double *const *d_grad_rate, cudaStream_t s) {
    if (pg_status st = check_batch(hs, k); st != PG_OK) return st;
    if (k > 0 && (!d_eps || !d_mu || !d_t || (grad ? !d_grad_b : !d_b)))
        return fail(PG_ERR_INVALID, "bad clock arguments");
    for (int i = 0; i < k; ++i)
        if (!d_eps[i] || !d_t[i] || (grad ? !d_grad_b[i] : !d_b[i]))
            return fail(PG_ERR_INVALID, "clock entry %d has a NULL array", i);
    if (k == 0) return PG_OK;
    for (int i = 0; i < k; ++i)
        if (hs[i]->n_user != hs[i]->desc.n_nodes)
            return fail(PG_ERR_UNSUPPORTED, "clock entry %d: the clock parameterisation takes binary trees only", i);
    DeviceGuard g(hs[0]->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", hs[0]->ctx->device);
    auto *a = new (std::nothrow) pg::ClockArgs<pg::kMaxClock>;
    if (!a) return fail(PG_ERR_OOM, "host allocation failed");
    for (int at = 0; at < k; at += pg::kMaxClock) {
        a->n = std::min(pg::kMaxClock, k - at);
        for (int j = 0; j < a->n; ++j) {
            const int i = at + j;
            const pg::ProbDesc &d = hs[i]->desc;
            pg::ClockDesc c{};
            c.parent = hs[i]->d_parent;
            c.ops = d.ops;
            c.n_tips = d.n_tips;
            c.n_nodes = d.n_nodes;
            c.root = d.root;
            c.eps = d_eps[i];
            c.mu = d_mu + i;
            c.t = d_t[i];
            if (grad) {
                c.g = d_grad_b[i];
                c.g_eps = d_grad_eps ? d_grad_eps[i] : nullptr;
                c.g_mu = d_grad_mu ? d_grad_mu + i : nullptr;
                c.g_t = d_grad_t ? d_grad_t[i] : nullptr;
                c.g_rate = d_grad_rate ? d_grad_rate[i] : nullptr;
            } else {
                c.b = d_b[i];
            }
            a->c[j] = c;
        }
        cudaError_t e = pg::launch_clock(*a, grad, s);
        if (e != cudaSuccess) { delete a; return fail(PG_ERR_CUDA, "launch: %s", cudaGetErrorString(e)); }
    }
    delete a;
    return PG_OK;
}

}  // namespace

pg_status pg_clock_lengths_async(pg_handle *const *hs, int32_t k, const double *const *d_eps,
                                 const double *d_mu, const double *const *d_t, double *const *d_b,
                                 void *stream) {
    return enqueue_clock(hs, k, false, d_eps, d_mu, d_t, d_b, nullptr, nullptr, nullptr, nullptr, nullptr,
                         static_cast<cudaStream_t>(stream));
}

pg_status pg_clock_grad_async(pg_handle *const *hs, int32_t k, const double *const *d_eps, const double *d_mu,
                              const double *const *d_t, const double *const *d_grad_b,
                              double *const *d_grad_eps, double *d_grad_mu, double *const *d_grad_t,
                              double *const *d_grad_rate, void *stream) {
    return enqueue_clock(hs, k, true, d_eps, d_mu, d_t, nullptr, d_grad_b, d_grad_eps, d_grad_mu, d_grad_t,
                         d_grad_rate, static_cast<cudaStream_t>(stream));
}

pg_status pg_set_phase_timing(pg_handle *h, int enable) {
    if (!h) return fail(PG_ERR_INVALID, "NULL handle");
    if (!h->chunks.empty()) return fail(PG_ERR_UNSUPPORTED, "phase timing of a problem evaluated in pattern chunks");
    DeviceGuard g(h->ctx->device);
    for (cudaEvent_t x : h->events) cudaEventDestroy(x);
    h->events.clear();
    if (enable < 0 || enable > 3) return fail(PG_ERR_INVALID, "phase-timing mode %d: 0, 1, 2 or 3", enable);
    h->timing = enable;
    h->timing_count = 0;
    return PG_OK;
}

pg_status pg_get_phase_times(pg_handle *h, pg_phase_times *out) {
    if (!h || !out) return fail(PG_ERR_INVALID, "NULL argument");
    DeviceGuard g(h->ctx->device);
    pg_phase_times t{};
    double *ph[5] = {&t.pmatrix_ms, &t.post_levels_ms, &t.fused_ms, &t.pre_levels_ms, &t.reduce_ms};
    if (h->timing >= 2) {   // the pre-order levels only
        for (size_t b = 0; b + 2 <= h->events.size(); b += 2) {
            PG_CUDA(cudaEventSynchronize(h->events[b + 1]));
            float ms = 0.f;
            PG_CUDA(cudaEventElapsedTime(&ms, h->events[b], h->events[b + 1]));
            t.pre_levels_ms += ms;
            t.evals += 1;
        }
    }
    for (size_t b = 0; h->timing == 1 && b + 6 <= h->events.size(); b += 6) {
        PG_CUDA(cudaEventSynchronize(h->events[b + 5]));
        for (int i = 0; i < 5; ++i) {
            float ms = 0.f;
            PG_CUDA(cudaEventElapsedTime(&ms, h->events[b + i], h->events[b + i + 1]));
            *ph[i] += ms;
        }
        float ms = 0.f;
        PG_CUDA(cudaEventElapsedTime(&ms, h->events[b], h->events[b + 5]));
        t.total_ms += ms;
        t.evals += 1;
    }
    t.launches_per_eval = h->desc.P > 0 ? 3 + 2 * h->cut : 2;
    t.post_levels_bytes = h->post_levels_bytes;
    t.fused_bytes = h->fused_bytes;
    t.pre_levels_bytes = h->pre_levels_bytes;
    *out = t;
    return PG_OK;
}

// The API status of a handle's sticky device status word (kStatus* bits; 0 = PG_OK).
static pg_status status_result(int st) {
    if (st & pg::kStatusBadLength) return fail(PG_ERR_INVALID, "a branch length was negative or not finite");
    if (st & pg::kStatusNumeric) return fail(PG_ERR_NUMERIC, "a site likelihood was zero or not finite");
    if (st & pg::kStatusUnsettled)
        return fail(PG_ERR_TIMEOUT, "a device-side wait gave up and a block left before the copies or products it "
                                    "issued were confirmed complete: the device state is suspect, destroy the context");
    if (st & pg::kStatusTimeout) return fail(PG_ERR_TIMEOUT, "a device-side wait for staged data gave up");
    return PG_OK;
}

pg_status pg_eval_status(pg_handle *h) {
    if (!h) return fail(PG_ERR_INVALID, "NULL handle");
    DeviceGuard g(h->ctx->device);
    PG_CUDA(cudaStreamSynchronize(h->last_stream));
    int st = 0;
    if (h->chunks.empty()) {
        PG_CUDA(cudaMemcpy(&st, h->desc.status, sizeof(int), cudaMemcpyDeviceToHost));
        if (st) PG_CUDA(cudaMemset(h->desc.status, 0, sizeof(int)));
    }
    for (pg_handle *c : h->chunks) {   // every chunk's status word
        int cs = 0;
        PG_CUDA(cudaMemcpy(&cs, c->desc.status, sizeof(int), cudaMemcpyDeviceToHost));
        if (cs) PG_CUDA(cudaMemset(c->desc.status, 0, sizeof(int)));
        st |= cs;
    }
    return status_result(st);
}

// Host arrays through one pinned staging buffer: the lengths go in with one copy, the outputs and
// the status word come back with two, and the call waits on the stream once.
pg_status pg_eval(pg_handle *h, const double *b, double *logL, double *grad, double *hess,
                  double *site_logL) {
    if (!h || !b) return fail(PG_ERR_INVALID, "NULL handle or branch lengths");
    DeviceGuard g(h->ctx->device);
    if (!g.ok) return fail(PG_ERR_CUDA, "cannot select device %d", h->ctx->device);
    const int n = h->n_user, P = h->desc.P;   // the caller's nodes; added nodes keep b = 0 in io_b
    // the outputs were carved in this order from one block: one copy covers the requested ones
    const char *lo = reinterpret_cast<const char *>(h->io_logL);
    const auto end_of = [lo](const double *p, size_t count) {
        return (size_t)(reinterpret_cast<const char *>(p + count) - lo);
    };
    size_t span = sizeof(double);
    if (grad) span = std::max(span, end_of(h->io_grad, n));
    if (hess) span = std::max(span, end_of(h->io_hess, n));
    if (site_logL && P > 0) span = std::max(span, end_of(h->io_site, P));
    const size_t o_st = align_up(sizeof(double) * n, 16), o_out = o_st + 16;
    const size_t need = o_out + align_up(end_of(h->io_site, std::max(P, 1)), 16);   // every output
    if (!h->io_host) {
        void *p = nullptr;
        PG_CUDA(cudaHostAlloc(&p, need, cudaHostAllocDefault));
        h->io_host = static_cast<char *>(p);
        h->io_host_bytes = need;
    }
    double *hb = reinterpret_cast<double *>(h->io_host);
    int *hst = reinterpret_cast<int *>(h->io_host + o_st);
    const char *hout = h->io_host + o_out;
    std::memcpy(hb, b, sizeof(double) * n);
    *hst = 0;
    PG_CUDA(cudaMemcpyAsync(h->io_b, hb, sizeof(double) * n, cudaMemcpyHostToDevice, nullptr));
    pg_status st = enqueue_single(h, 0, h->io_b, h->io_logL, grad ? h->io_grad : nullptr, hess ? h->io_hess : nullptr,
                                  site_logL ? h->io_site : nullptr, nullptr, nullptr);
    if (st != PG_OK) return st;
    PG_CUDA(cudaMemcpyAsync(h->io_host + o_out, lo, span, cudaMemcpyDeviceToHost, nullptr));
    const bool chunked = !h->chunks.empty();
    if (!chunked) PG_CUDA(cudaMemcpyAsync(hst, h->desc.status, sizeof(int), cudaMemcpyDeviceToHost, nullptr));
    PG_CUDA(cudaStreamSynchronize(nullptr));
    const auto at = [&](const double *p) { return reinterpret_cast<const double *>(hout + (reinterpret_cast<const char *>(p) - lo)); };
    if (logL) *logL = *at(h->io_logL);
    if (grad) std::memcpy(grad, at(h->io_grad), sizeof(double) * n);
    if (hess) std::memcpy(hess, at(h->io_hess), sizeof(double) * n);
    if (site_logL && P > 0) std::memcpy(site_logL, at(h->io_site), sizeof(double) * P);
    if (chunked) return pg_eval_status(h);
    if (*hst) PG_CUDA(cudaMemset(h->desc.status, 0, sizeof(int)));
    return status_result(*hst);
}

}  // extern "C"
