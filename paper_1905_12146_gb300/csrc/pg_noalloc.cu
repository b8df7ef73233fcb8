// pg_eval_noalloc: one evaluation of a small problem that allocates no memory at all.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocator) at the point where they
// evaluate -- for example code that must not trigger the device-wide synchronisation and latency
// of an allocation inside a latency-critical loop, code running under an external memory manager
// that owns every device allocation of the process, or plug-ins whose host application forbids
// allocation after start-up.  They pass host arrays in and out; every intermediate array lives in
// the fixed device array below, and host-side planning uses fixed static buffers.  The inputs are
// laid out at the start of the array and go in with one copy from a static host image; the status
// word and the outputs follow them and come back with one copy (array by array when a problem's
// regions exceed the static images).
//
// The scratch array is g_noalloc_scratch (PG_NOALLOC_SCRATCH_BYTES, 64 MiB).  Being a file-scope
// __device__ variable it is created on every GPU that loads this library's code and stays there
// until the process exits.  In host code its name is only a host-side stand-in, so its device
// address is taken with cudaGetSymbolAddress, once per device, with that device current, on the
// first call made on that device (thread-safely).  That cached address belongs to the device's
// current CUDA context: after cudaDeviceReset on a device, do not call this entry point on that
// device again in the same process.  All calls share the array (and the static host buffers): calls
// that overlap -- on the GPU or from several host threads -- race and must be serialised by the
// caller.  An error message is formatted into a fixed static buffer (no allocation) and is what
// pg_last_error() returns on the failing call's thread until that thread records another error.  The array keeps the last call's contents; the only value that must start at zero, the
// device status word, is cleared at the start of every call, and every partial and partial sum the
// kernels read is written by the same call first.
#include <cuda_runtime.h>
#include <pthread.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "phylograd.h"
#include "pg_host.h"
#include "pg_internal.cuh"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PG_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxTips = 8192;                 // host planning buffers
constexpr int kMaxNodes = 2 * kMaxTips - 1;
constexpr int kMaxModels = 64;

pg::DeviceOnce g_scratch_once;   // the array's device address, looked up once per device
void *g_scratch_addr[pg::kMaxDevices];

// static host buffers for validation and planning (no heap)
int g_kid0[kMaxNodes], g_kid1[kMaxNodes], g_order[kMaxNodes], g_height[kMaxNodes], g_fill[kMaxNodes];
int4 g_ops[kMaxTips];
int g_level_off[kMaxTips + 1];
float4 g_qf[kMaxModels * 4];
double g_mpow[kMaxModels * (pg::kTaylorDeg + 1) * 16];
double g_qnorm[kMaxModels];
// host images of the input and output regions of the scratch array (one copy each way when the
// problem's regions fit; larger problems copy array by array)
alignas(256) unsigned char g_stage_in[4u << 20];
alignas(256) unsigned char g_stage_out[1u << 20];

// the message of the last failure: a fixed buffer, formatted with vsnprintf (integer and string
// conversions only, which allocate nothing), then published to pg_last_error
char g_msg[256];
pg_status noalloc_fail(pg_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof g_msg, fmt, ap);
    va_end(ap);
    pg::host::publish_static_error(g_msg, pthread_self());
    return s;
}

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// Levels by height (tips 0, a node one above its higher child), written to g_ops / g_level_off.
pg_status plan(int N, const int32_t *parent, int &root, int &H) {
    const int n = 2 * N - 1;
    root = -1;
    for (int i = 0; i < n; ++i) g_kid0[i] = g_kid1[i] = -1;
    for (int i = 0; i < n; ++i) {
        const int p = parent[i];
        if (p == -1) {
            if (root >= 0) return noalloc_fail(PG_ERR_INVALID, "more than one root");
            root = i;
            continue;
        }
        if (p < N || p >= n || p == i) return noalloc_fail(PG_ERR_INVALID, "parent[%d] = %d is not an internal node", i, p);
        if (g_kid0[p] < 0) g_kid0[p] = i;
        else if (g_kid1[p] < 0) g_kid1[p] = i;
        else return noalloc_fail(PG_ERR_INVALID, "node %d has more than two children", p);
    }
    if (root < N) return noalloc_fail(PG_ERR_INVALID, "no internal root");
    for (int k = N; k < n; ++k)
        if (g_kid1[k] < 0) return noalloc_fail(PG_ERR_INVALID, "internal node %d has fewer than two children", k);
    int cnt = 0, top = 0;
    g_fill[top++] = root;   // g_fill doubles as the traversal stack
    while (top > 0) {
        const int k = g_fill[--top];
        if (cnt >= n) return noalloc_fail(PG_ERR_INVALID, "the parent array contains a cycle");
        g_order[cnt++] = k;
        if (k >= N) { g_fill[top++] = g_kid1[k]; g_fill[top++] = g_kid0[k]; }
    }
    if (cnt != n) return noalloc_fail(PG_ERR_INVALID, "the parent array contains a cycle");
    H = 0;
    for (int i = 0; i < n; ++i) g_height[i] = 0;
    for (int o = n - 1; o >= 0; --o) {
        const int k = g_order[o];
        if (k < N) continue;
        g_height[k] = 1 + (g_height[g_kid0[k]] > g_height[g_kid1[k]] ? g_height[g_kid0[k]] : g_height[g_kid1[k]]);
        if (g_height[k] > H) H = g_height[k];
    }
    for (int h = 0; h <= H; ++h) g_level_off[h] = 0;
    for (int k = N; k < n; ++k) g_level_off[g_height[k]]++;
    for (int h = 1; h <= H; ++h) g_level_off[h] += g_level_off[h - 1];
    for (int h = 0; h < H; ++h) g_fill[h] = g_level_off[h];
    for (int k = N; k < n; ++k) g_ops[g_fill[g_height[k] - 1]++] = int4{k, g_kid0[k], g_kid1[k], 0};
    return PG_OK;
}

pg_status check_inputs(const pg_problem *pr) {
    const int m = pr->n_states, C = pr->n_categories, M = pr->n_models, N = pr->n_tips, P = pr->n_patterns;
    if (N < 2 || m < 2 || P < 0 || C < 1 || M < 1) return noalloc_fail(PG_ERR_INVALID, "bad problem sizes");
    if (m != pg::kStates || C > pg::kMaxCat) return noalloc_fail(PG_ERR_UNSUPPORTED, "4 states and at most 4 categories");
    if (pr->n_tip_partials != 0) return noalloc_fail(PG_ERR_UNSUPPORTED, "tip partial vectors need pg_upload");
    if (pr->n_nodes != 0 && pr->n_nodes != 2 * N - 1)
        return noalloc_fail(PG_ERR_UNSUPPORTED, "multifurcating trees (n_nodes = %d) need pg_upload", pr->n_nodes);
    if (N > kMaxTips || M > kMaxModels)
        return noalloc_fail(PG_ERR_UNSUPPORTED, "at most %d tips and %d models without allocation", kMaxTips, kMaxModels);
    if (pr->precision != PG_PRECISION_FP32 && pr->precision != PG_PRECISION_FP64)
        return noalloc_fail(PG_ERR_INVALID, "precision = %d", pr->precision);
    if (!pr->parent || !pr->Q || !pr->root_freqs || !pr->cat_rates || !pr->cat_weights ||
        (P > 0 && (!pr->tip_states || !pr->pattern_weights)) || (pr->tip_stride != 0 && pr->tip_stride < P))
        return noalloc_fail(PG_ERR_INVALID, "a required input is NULL");
    for (int md = 0; md < M; ++md) {
        const double *Q = pr->Q + (size_t)md * 16;
        double mx = 0.0;
        for (int t = 0; t < 16; ++t) {
            if (!std::isfinite(Q[t])) return noalloc_fail(PG_ERR_INVALID, "Q has a non-finite entry");
            mx = std::fmax(mx, std::fabs(Q[t]));
        }
        for (int i = 0; i < 4; ++i) {
            double s = 0.0;
            for (int j = 0; j < 4; ++j) {
                if (i != j && Q[i * 4 + j] < 0.0) return noalloc_fail(PG_ERR_INVALID, "negative off-diagonal of Q");
                s += Q[i * 4 + j];
            }
            if (mx > 0.0 && std::fabs(s) > 1e-10 * mx) return noalloc_fail(PG_ERR_INVALID, "a row of Q does not sum to 0");
        }
    }
    double s = 0.0;
    for (int i = 0; i < 4; ++i) {
        if (!(pr->root_freqs[i] >= 0.0)) return noalloc_fail(PG_ERR_INVALID, "negative root frequency");
        s += pr->root_freqs[i];
    }
    if (std::fabs(s - 1.0) > 1e-10) return noalloc_fail(PG_ERR_INVALID, "root_freqs do not sum to 1");
    s = 0.0;
    for (int l = 0; l < C; ++l) {
        if (!(pr->cat_weights[l] >= 0.0) || !(pr->cat_rates[l] >= 0.0) || !std::isfinite(pr->cat_rates[l]))
            return noalloc_fail(PG_ERR_INVALID, "bad rate category");
        s += pr->cat_weights[l];
    }
    if (std::fabs(s - 1.0) > 1e-10) return noalloc_fail(PG_ERR_INVALID, "cat_weights do not sum to 1");
    if (pr->branch_model)
        for (int i = 0; i < 2 * N - 1; ++i)
            if (pr->branch_model[i] < 0 || pr->branch_model[i] >= M) return noalloc_fail(PG_ERR_INVALID, "bad branch_model");
    for (int p = 0; p < P; ++p)
        if (!(pr->pattern_weights[p] >= 0.0) || !std::isfinite(pr->pattern_weights[p]))
            return noalloc_fail(PG_ERR_INVALID, "bad pattern weight");
    return PG_OK;
}

#define NOALLOC_CUDA(call)                                                                        \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return noalloc_fail(PG_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" pg_status pg_eval_noalloc(const pg_problem *pr, const double *b, double *logL, double *grad,
                                     double *hess, double *site_logL, void *stream) {
    if (!pr || !b) return noalloc_fail(PG_ERR_INVALID, "NULL problem or branch lengths");
    pg_status st = check_inputs(pr);
    if (st != PG_OK) return st;
    int root = -1, H = 0;
    st = plan(pr->n_tips, pr->parent, root, H);
    if (st != PG_OK) return st;

    const int N = pr->n_tips, n = 2 * N - 1, P = pr->n_patterns, C = pr->n_categories, M = pr->n_models;
    const bool f64 = pr->precision == PG_PRECISION_FP64;
    const int Ps = (P + 15) / 16 * 16;
    int dev = 0, n_sm = 1;
    NOALLOC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= pg::kMaxDevices) return noalloc_fail(PG_ERR_UNSUPPORTED, "device ordinal %d", dev);
    NOALLOC_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    // set-up on this device's first call, with the device current: the array's device address
    NOALLOC_CUDA(pg::device_once(g_scratch_once, [dev](int &) {
        return cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
    }));
    char *base = static_cast<char *>(g_scratch_addr[dev]);

    // tiling of the fused kernel over the patterns, as a single-problem evaluation
    const int max_tiles = 4 * n_sm;
    int T = 0, L = 0, pieces = 0;
    if (P > 0) {
        T = n_sm * pg::tree_blocks_per_sm(C, f64);
        if (T > max_tiles) T = max_tiles;
        if (T > P) T = P;
        const int min_T = (P + pg::kMaxRange - 1) / pg::kMaxRange;
        if (T < min_T) T = min_T;
        L = (P + T - 1) / T;
        T = (P + L - 1) / L;
        pieces = (L + 31) / 32 + 1;
    }
    const int slot_cap = (P + 31) / 32 + 3 * max_tiles + 2;

    // layout of the scratch array
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = up256(off + bytes); return at; };
    const size_t o_ops = take(sizeof(int4) * (N - 1)), o_lv = take(sizeof(int) * (H + 1));
    const size_t o_tips = take((size_t)N * Ps), o_w = take(sizeof(double) * Ps);
    const size_t o_Qd = take(sizeof(double) * 16 * M), o_Qf = take(sizeof(float4) * 4 * M);
    const size_t o_Mp = take(sizeof(double) * (pg::kTaylorDeg + 1) * 16 * M), o_qn = take(sizeof(double) * M);
    const size_t o_bm = take(pr->branch_model ? sizeof(int) * n : 0);
    const size_t o_ib = take(sizeof(double) * n);
    // the status word ends the inputs (it goes in as zero) and starts the outputs
    const size_t o_st = take(sizeof(int)), o_il = take(sizeof(double)), o_ig = take(sizeof(double) * n);
    const size_t o_ih = take(sizeof(double) * n), o_is = take(sizeof(double) * (P > 0 ? P : 1));
    const size_t in_bytes = o_st + sizeof(int), out_bytes = o_is + sizeof(double) * (P > 0 ? P : 1) - o_st;
    const size_t o_P = take(f64 ? sizeof(double2) * n * C * pg::kPtab64Pairs : sizeof(float4) * n * C * pg::kPtabCols);
    const size_t part = (size_t)(N - 1) * C * Ps * (f64 ? 2 * sizeof(double2) : sizeof(float4));
    const size_t o_post = take(part), o_pre = take(part);
    const size_t o_pe = take(sizeof(int) * (N - 1) * Ps), o_qe = take(sizeof(int) * (N - 1) * Ps);
    const size_t o_gp = take(sizeof(double) * n * slot_cap), o_hp = take(sizeof(double) * n * slot_cap);
    const size_t o_lp = take(sizeof(double) * slot_cap);
    const size_t o_sinv = take(sizeof(float) * (Ps > 16 ? Ps : 16)), o_ser = take(sizeof(int) * (Ps > 16 ? Ps : 16));
    if (off > (size_t)PG_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(PG_ERR_UNSUPPORTED, "problem needs %zu bytes of scratch; the fixed array holds %u",
                            off, (unsigned)PG_NOALLOC_SCRATCH_BYTES);

    for (int md = 0; md < M; ++md) {
        const double *Q = pr->Q + (size_t)md * 16;
        for (int c = 0; c < 4; ++c)
            g_qf[md * 4 + c] = make_float4((float)Q[c], (float)Q[4 + c], (float)Q[8 + c], (float)Q[12 + c]);
        double *Mk = g_mpow + (size_t)md * (pg::kTaylorDeg + 1) * 16;   // Q^k / k!
        for (int u = 0; u < 16; ++u) Mk[u] = (u % 5 == 0) ? 1.0 : 0.0;
        for (int k = 1; k <= pg::kTaylorDeg; ++k)
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    double acc = 0.0;
                    for (int t = 0; t < 4; ++t) acc += Mk[(k - 1) * 16 + r * 4 + t] * Q[t * 4 + c];
                    Mk[k * 16 + r * 4 + c] = acc / (double)k;
                }
        double nrm = 0.0;
        for (int c = 0; c < 4; ++c) {
            const double cs = std::fabs(Q[c]) + std::fabs(Q[4 + c]) + std::fabs(Q[8 + c]) + std::fabs(Q[12 + c]);
            nrm = cs > nrm ? cs : nrm;
        }
        g_qnorm[md] = nrm;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t tip_stride = pr->tip_stride > 0 ? (size_t)pr->tip_stride : (size_t)P;
    if (in_bytes <= sizeof g_stage_in) {   // the inputs as laid out on the device: one copy
        unsigned char *h = g_stage_in;
        std::memcpy(h + o_ops, g_ops, sizeof(int4) * (N - 1));
        std::memcpy(h + o_lv, g_level_off, sizeof(int) * (H + 1));
        for (int t = 0; t < N && P > 0; ++t) std::memcpy(h + o_tips + (size_t)t * Ps, pr->tip_states + t * tip_stride, P);
        if (P > 0) std::memcpy(h + o_w, pr->pattern_weights, sizeof(double) * P);
        std::memcpy(h + o_Qd, pr->Q, sizeof(double) * 16 * M);
        std::memcpy(h + o_Qf, g_qf, sizeof(float4) * 4 * M);
        std::memcpy(h + o_Mp, g_mpow, sizeof(double) * (pg::kTaylorDeg + 1) * 16 * M);
        std::memcpy(h + o_qn, g_qnorm, sizeof(double) * M);
        if (pr->branch_model) std::memcpy(h + o_bm, pr->branch_model, sizeof(int) * n);
        std::memcpy(h + o_ib, b, sizeof(double) * n);
        std::memset(h + o_st, 0, sizeof(int));   // the sticky status starts clear
        NOALLOC_CUDA(cudaMemcpyAsync(base, h, in_bytes, cudaMemcpyHostToDevice, s));
    } else {
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_ops, g_ops, sizeof(int4) * (N - 1), cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_lv, g_level_off, sizeof(int) * (H + 1), cudaMemcpyHostToDevice, s));
        if (P > 0) {
            NOALLOC_CUDA(cudaMemcpy2DAsync(base + o_tips, Ps, pr->tip_states, tip_stride, P, N, cudaMemcpyHostToDevice, s));
            NOALLOC_CUDA(cudaMemcpyAsync(base + o_w, pr->pattern_weights, sizeof(double) * P, cudaMemcpyHostToDevice, s));
        }
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_Qd, pr->Q, sizeof(double) * 16 * M, cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_Qf, g_qf, sizeof(float4) * 4 * M, cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_Mp, g_mpow, sizeof(double) * (pg::kTaylorDeg + 1) * 16 * M,
                                     cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_qn, g_qnorm, sizeof(double) * M, cudaMemcpyHostToDevice, s));
        if (pr->branch_model)
            NOALLOC_CUDA(cudaMemcpyAsync(base + o_bm, pr->branch_model, sizeof(int) * n, cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemcpyAsync(base + o_ib, b, sizeof(double) * n, cudaMemcpyHostToDevice, s));
        NOALLOC_CUDA(cudaMemsetAsync(base + o_st, 0, sizeof(int), s));   // the sticky status starts clear
    }

    pg::BatchArgs<1> a;
    pg::ProbDesc &d = a.d[0];
    d = pg::ProbDesc{};
    d.ops = reinterpret_cast<const int4 *>(base + o_ops);
    d.level_off = reinterpret_cast<const int *>(base + o_lv);
    d.tips = reinterpret_cast<const uint8_t *>(base + o_tips);
    d.weights = reinterpret_cast<const double *>(base + o_w);
    d.Qd = reinterpret_cast<const double *>(base + o_Qd);
    d.Qf = reinterpret_cast<const float4 *>(base + o_Qf);
    d.Mpow = reinterpret_cast<const double *>(base + o_Mp);
    d.qnorm = reinterpret_cast<const double *>(base + o_qn);
    d.bmodel = pr->branch_model ? reinterpret_cast<const int *>(base + o_bm) : nullptr;
    d.Ptab = f64 ? nullptr : reinterpret_cast<float4 *>(base + o_P);
    d.Ptab64 = f64 ? reinterpret_cast<double2 *>(base + o_P) : nullptr;
    d.post = base + o_post;
    d.pre = base + o_pre;
    d.pe = reinterpret_cast<int *>(base + o_pe);
    d.qe = reinterpret_cast<int *>(base + o_qe);
    d.gpart = reinterpret_cast<double *>(base + o_gp);
    d.hpart = reinterpret_cast<double *>(base + o_hp);
    d.lpart = reinterpret_cast<double *>(base + o_lp);
    d.status = reinterpret_cast<int *>(base + o_st);
    d.cut = 0;
    d.plevel = nullptr;
    d.site_invL = reinterpret_cast<float *>(base + o_sinv);
    d.site_Er = reinterpret_cast<int *>(base + o_ser);
    d.b = reinterpret_cast<const double *>(base + o_ib);
    d.out_logL = reinterpret_cast<double *>(base + o_il);
    d.out_grad = grad ? reinterpret_cast<double *>(base + o_ig) : nullptr;
    d.out_hess = hess ? reinterpret_cast<double *>(base + o_ih) : nullptr;
    d.out_site = site_logL ? reinterpret_cast<double *>(base + o_is) : nullptr;
    d.n_tips = N;
    d.n_nodes = n;
    d.root = root;
    d.n_levels = H;
    d.P = P;
    d.Ps = Ps;
    d.slot_cap = slot_cap;
    d.n_tiles = T;
    d.range_len = L;
    d.pieces = pieces;
    d.n_tg = T * pieces;
    d.C = C;
    d.n_models = M;
    d.precision = pr->precision;
    for (int i = 0; i < pg::kStates; ++i) { d.pi[i] = pr->root_freqs[i]; d.pif[i] = (float)pr->root_freqs[i]; }
    for (int l = 0; l < pg::kMaxCat; ++l) {
        const bool on = l < C;
        d.cw[l] = on ? pr->cat_weights[l] : 0.0;
        d.rates[l] = on ? pr->cat_rates[l] : 0.0;
        d.gw[l] = on ? (float)(pr->cat_rates[l] * pr->cat_weights[l]) : 0.f;
        d.gw2[l] = on ? (float)(pr->cat_rates[l] * pr->cat_rates[l] * pr->cat_weights[l]) : 0.f;
    }
    if (f64 && P > 0) {   // the shared-memory latency kernel when a block's vectors fit at one block per SM
        pg::ProbDesc ds = d;
        ds.range_len = (P + n_sm - 1) / n_sm;
        if (ds.range_len > pg::kMaxRange) ds.range_len = pg::kMaxRange;
        ds.n_tiles = (P + ds.range_len - 1) / ds.range_len;
        ds.pieces = 1;
        ds.n_tg = ds.n_tiles;
        ds.small64 = 1;
        if (pg::small64_smem_bytes(ds) != 0) {
            d = ds;
            T = ds.n_tiles;
        }
    }
    a.n = 1;
    a.tile_base[0] = 0;
    a.tile_base[1] = T;
    a.mat_base[0] = 0;
    a.mat_base[1] = n * C;
    a.red_base[0] = 0;
    a.red_base[1] = n + 1;
    NOALLOC_CUDA(pg::launch_eval_nt<1>(a, hess != nullptr, s));

    int status = 0;
    if (out_bytes <= sizeof g_stage_out) {   // status and outputs as laid out on the device: one copy
        const unsigned char *h = g_stage_out;
        NOALLOC_CUDA(cudaMemcpyAsync(g_stage_out, base + o_st, out_bytes, cudaMemcpyDeviceToHost, s));
        NOALLOC_CUDA(cudaStreamSynchronize(s));
        std::memcpy(&status, h, sizeof(int));
        if (logL) std::memcpy(logL, h + (o_il - o_st), sizeof(double));
        if (grad) std::memcpy(grad, h + (o_ig - o_st), sizeof(double) * n);
        if (hess) std::memcpy(hess, h + (o_ih - o_st), sizeof(double) * n);
        if (site_logL && P > 0) std::memcpy(site_logL, h + (o_is - o_st), sizeof(double) * P);
    } else {
        if (logL) NOALLOC_CUDA(cudaMemcpyAsync(logL, base + o_il, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (grad) NOALLOC_CUDA(cudaMemcpyAsync(grad, base + o_ig, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (hess) NOALLOC_CUDA(cudaMemcpyAsync(hess, base + o_ih, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
        if (site_logL && P > 0)
            NOALLOC_CUDA(cudaMemcpyAsync(site_logL, base + o_is, sizeof(double) * P, cudaMemcpyDeviceToHost, s));
        NOALLOC_CUDA(cudaMemcpyAsync(&status, base + o_st, sizeof(int), cudaMemcpyDeviceToHost, s));
        NOALLOC_CUDA(cudaStreamSynchronize(s));
    }
    if (status & pg::kStatusBadLength) return noalloc_fail(PG_ERR_INVALID, "a branch length was negative or not finite");
    if (status & pg::kStatusNumeric) return noalloc_fail(PG_ERR_NUMERIC, "a site likelihood was zero or not finite");
    if (status & pg::kStatusUnsettled)
        return noalloc_fail(PG_ERR_TIMEOUT, "a device-side wait gave up and a block left with copies unconfirmed");
    if (status & pg::kStatusTimeout) return noalloc_fail(PG_ERR_TIMEOUT, "a device-side wait gave up");
    return PG_OK;
}
