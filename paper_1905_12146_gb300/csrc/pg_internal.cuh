// Internal structures shared by the host side (pg_api.cu) and the kernels (pg_nt.cu).
// Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

namespace pg {

// One-time set-up of a kernel on each device.  cudaFuncSetAttribute and the occupancy queries apply
// to the device current at the call, so every device ordinal runs the set-up once (thread-safely:
// a serving worker and the caller's thread may launch at the same time); later calls on that device
// return the set-up's status and the value it produced (e.g. resident blocks per SM).
constexpr int kMaxDevices = 64;
struct DeviceOnce {
    std::once_flag flag[kMaxDevices];
    cudaError_t err[kMaxDevices] = {};
    int value[kMaxDevices] = {};
};
template <class F>
cudaError_t device_once(DeviceOnce &o, F &&setup, int *value = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(o.flag[dev], [&] {
        int v = 0;
        o.err[dev] = setup(v);
        o.value[dev] = v;
    });
    if (value) *value = o.value[dev];
    return o.err[dev];
}

constexpr int kStates = 4;      // nucleotide state space handled by the kernels in pg_nt.cu
constexpr int kMaxCat = 4;      // rate categories held in registers per pattern
// problems per batched launch (kernel-parameter descriptors): BatchArgs<64> is 32,528 bytes, within
// the 32,764 bytes a kernel's parameters may take
constexpr int kMaxBatch = 64;
constexpr int kMaxRange = 1024;  // patterns per thread block of the tree kernel (shared arrays)
constexpr int kBlock = 256;      // threads per block of the tree kernel
constexpr int kLevelRange = 128; // consumer threads per block of the level kernels (4 warps)
// patterns per item of the level kernels for C rate categories: an item's copies and barrier round
// trips cost the same whatever its size, so with fewer categories (smaller rows) an item takes more
// patterns (each consumer thread kLevelRange apart), keeping items at several KB
__host__ __device__ constexpr int level_range(int C) { return C <= 2 ? 2 * kLevelRange : kLevelRange; }
// A cherry level's item (both children tips: a few table lookups per pattern, no child rows) covers
// this many consecutive ranges of level_range(C) patterns, so its fixed costs are spread over more
// patterns; the pre-order step still stores one slot per (range, consumer warp).  With C <= 2 a
// range's rows are small; with more categories larger cherry items measured no faster.
__host__ __device__ constexpr int post_cherry_ranges(int C) { return C <= 2 ? 4 : 1; }
__host__ __device__ constexpr int pre_cherry_ranges(int C) { return C <= 2 ? 4 : 1; }
// items of one node of a level: ranges of level_range(C) patterns, or of `ranges` such ranges
__host__ __device__ constexpr int level_items_per_node(int P, int C, int ranges) {
    return (P + level_range(C) * ranges - 1) / (level_range(C) * ranges);
}
constexpr int kTaylorDeg = 12;   // degree of the Taylor polynomial of e^{Q t} (||Q t||_1 <= 1/4)
// FP32 transition table per (branch, category), float4 columns of the 4x4 matrices:
//   [0..4]   P hi (columns 0..3, then the row sums = P applied to the all-ones vector)
//   [5..9]   G = Q P in the same column layout (the generator applied to a column of P)
//   [10..14] P lo (the FP32 residual P - hi of the same entries)
//   [15..18] D hi, [19..22] D lo, with D = P - I
constexpr int kPtabCols = 23;
constexpr int kColG = 5, kColPlo = 10, kColDhi = 15, kColDlo = 19;
// FP64 transition table per (branch, category): 5 columns of 4 doubles as double2 pairs
constexpr int kPtab64Pairs = 10;

// device status bits (sticky until read by pg_eval_status / pg_eval)
constexpr int kStatusBadLength = 1;
constexpr int kStatusNumeric = 2;
constexpr int kStatusTimeout = 4;
// a block that gave up left before every copy or product it issued was confirmed complete
constexpr int kStatusUnsettled = 8;
// bound on a block's wait for its own bulk copies (SM clocks, about one second)
constexpr long long kWaitLimitCycles = 2000000000LL;

// Everything one problem's kernels need.  Lives in kernel parameter space (by value), so a
// launch never depends on host memory that may change afterwards.
struct ProbDesc {
    // tree: internal-node operations sorted by height, {k, c0, c1, flags} (node ids); flags bit 0
    // (bit 1) when c0 (c1) is internal and on the level just below k's (read by the post-order
    // level kernels to split a stage's copies around their programmatic-launch wait)
    const int4 *ops;
    const int *level_off;          // [n_levels + 1] offsets into ops
    // data
    const uint8_t *tips;           // [N][P], code >= 4 = all-ones
    const double *weights;         // [P]
    // model
    const double *b;               // [n] branch lengths of this evaluation (device)
    const double *Qd;              // [n_models][4][4] FP64 row-major
    const double *Mpow;            // [n_models][kTaylorDeg + 1][16]: Q^k / k!, FP64 row-major
    const double *qnorm;           // [n_models] ||Q||_1
    const float4 *Qf;              // [n_models][4] FP32 columns of Q
    const int *bmodel;             // [n] or nullptr (model 0)
    float4 *Ptab;                  // FP32: [n][C][kPtabCols]
    double2 *Ptab64;               // FP64: [n][C][kPtab64Pairs]
    // pass buffers: FP32 float4 [N-1][C][P], FP64 double2 [N-1][C][P][2]
    void *post;                    // post-order partials of internal nodes
    void *pre;                     // pre-order partials of internal nodes
    int *pe;                       // [N-1][P] log2 scale of post partials
    int *qe;                       // [N-1][P] log2 scale of pre partials
    double *gpart;                 // [n][slot_cap] per-(block, piece) gradient sums
    double *hpart;                 // [n][slot_cap] per-(block, piece) Hessian-diagonal sums
    double *lpart;                 // [slot_cap] per-(block, piece) log-likelihood sums
    int *status;
    // levels [0, cut) run as one launch per level (level kernels), [cut, n_levels) in the fused
    // tree kernel
    int cut;
    float *site_invL;              // [P] 1 / Lhat_p, written at the root for the level kernels
    int *site_Er;                  // [P] log2 scale of L_p
    int level_ranges;              // ceil(P / level_range(C)); a wide branch has 4 slots per range
    // shared-memory-resident top part (levels >= cut) for the top kernel (pg_top.cu): n_top nodes
    // ops[level_off[cut] ..], children coded per top node: -1 - s for the s-th tip child,
    // [0, n_top) a top node, n_top + b the b-th boundary node (internal, below the cut;
    // bnd_node[b] its node id)
    int n_top, n_bnd;
    const int2 *top_code;
    const int *bnd_node;
    // outputs of this evaluation (device, may be null)
    double *out_logL, *out_grad, *out_hess, *out_site;
    // parts of the evaluation this launch leaves out (kSkipPost / kSkipPre bits; 0 = all of it).
    // A launch that skips the post-order reads the partials and site arrays that an earlier
    // launch left in the handle; gscale (device scalar, may be null = 1) multiplies the gradient
    int skip;
    const double *gscale;
    // [Ps] N log r_p, the log of the pattern factors the FP32 post-order multiplies into L_p
    // (computed once on upload; null: the kernels compute it)
    const double *rlog;
    // [n] level index of each node's parent (-1 at the root): a branch whose parent lies below
    // the cut was summed in level-kernel slots, the others in fused-kernel slots
    const int *plevel;
    // sizes
    int n_tips, n_nodes, root, n_levels;
    int P;                         // site patterns
    int Ps;                        // row stride of every per-pattern array: P rounded up to 16
    const float *wf;               // [Ps] pattern weights in FP32 (gradient terms)
    int slot_cap;                  // capacity of the per-branch slot arrays
    // tiling of this launch: n_tiles blocks, each a contiguous range of range_len patterns
    // (the last one shorter); a node's pairs in one block span at most pieces 32-lane chunks
    int n_tiles, range_len, pieces, n_tg;   // n_tg = n_tiles * pieces used slots
    int C, n_models;
    int precision;                 // 0 FP32 partials, 1 FP64 partials
    int small64;                   // 1: the tree pass of this FP64 problem runs in the shared-memory
                                   // latency kernel (pg_small64.cu), tiled for it with pieces = 1
    double pi[kStates], cw[kMaxCat], rates[kMaxCat];
    float pif[kStates], gw[kMaxCat], gw2[kMaxCat];   // FP32 pi, r_l w_l, r_l^2 w_l
};

constexpr int kSkipPost = 1;   // forward part: P build, post-order levels, root and logL
constexpr int kSkipPre = 2;    // backward part: pre-order levels, gradient and Hessian diagonal

template <int MAXB>
struct BatchArgs {
    int n;
    int tile_base[MAXB + 1];   // prefix sums of n_tiles   (tree kernel blocks)
    int mat_base[MAXB + 1];    // prefix sums of n * C     (P-build threads)
    int red_base[MAXB + 1];    // prefix sums of n + 1     (reduce warps)
    ProbDesc d[MAXB];
};
static_assert(sizeof(BatchArgs<kMaxBatch>) + sizeof(int) <= 32764, "batched launch parameters exceed 32,764 bytes");

// one problem of the clock parameterisation b_i = mu eps_i (t_i - t_parent(i)) (pg_clock.cu);
// every array is [n_nodes] on the device, mu and g_mu are device scalars
struct ClockDesc {
    const int *parent;
    const int4 *ops;               // internal nodes {k, c0, c1, 0}
    int n_tips, n_nodes, root;
    const double *eps, *mu, *t;
    double *b;                     // lengths (forward)
    const double *g;               // dlogL/db (backward)
    double *g_eps, *g_mu, *g_t, *g_rate;   // outputs of the chain rule (each may be null)
};

constexpr int kMaxClock = 64;   // problems per clock launch

template <int MAXB>
struct ClockArgs {
    int n;
    ClockDesc c[MAXB];
};

cudaError_t launch_clock(const ClockArgs<kMaxClock> &a, bool grad, cudaStream_t s);

// ---- general state spaces (pg_mstate.cu): 5 <= m <= 64 states, padded to kMP ---------------------
// Transition matrices by uniformisation: with mu = max_i -Q_ii and B = I + Q / mu (entrywise
// non-negative), P(t) = e^{-mu t} sum_k (mu t)^k / k! B^k.  The host forms B^k, k = 1 .. kUnifK,
// in FP64 once per upload; per branch and category the device forms (t = b r, halved s times until
// mu t <= 4 and squared back in the D form D <- 2 D + D D)
//   D = P - I = expm1(-mu t) I + e^{-mu t} sum_{k>=1} (mu t)^k / k! B^k,  G = r Q P,  H = r^2 Q^2 P,
// where every off-diagonal term is positive: small transition probabilities keep their relative
// accuracy and never turn negative.
// Partials are FP32 [node - N][C][Ps][kMP] (a column = (pattern, category) holds kMP states, pads
// zero) with one power-of-two exponent per column [node - N][C][Ps].
constexpr int kMP = 64;                 // padded state count
constexpr int kMTile = 64;              // patterns per item of the m-state kernels
constexpr int kTabRows = kMP + 1;       // table rows: kMP, then the ambiguous-code row
constexpr int kTabFloats = kTabRows * kMP;
constexpr int kTabDT = 0, kTabD = 1, kTabGT = 2, kTabHT = 3, kTabKinds = 4;
constexpr int kUnifK = 32;              // powers of B held per model (covers mu t <= 4 to ~1e-13)
constexpr int kMRootPatterns = 16;   // patterns per block of the general-state root kernel (16 lanes each)

struct MDesc {
    const int4 *ops;
    const int *level_off;
    const uint8_t *tips;           // [N][Ps] codes: < m a state, m .. m + n_tv - 1 a row of tipv,
                                   // larger the all-ones (missing) code
    const float *tipv;             // [n_tv][kMP] partial vectors of partially observed tips, pads 0,
                                   // each row scaled by a power of two so that its largest entry is 1
    const int *tip_E;              // [Ps] or null: sum over the tips of pattern p of their rows' log2
                                   // scales (added back to the site log-likelihoods only: the
                                   // gradient and Hessian are ratios in which the scales cancel)
    int n_tv;
    const double *weights;         // [P]
    const double *b;               // [n] branch lengths of this evaluation
    const float *Bpow;             // [n_models][kUnifK][kMP][kMP]: B^k (k = 1 ..), FP32, pads 0
    const float *QT;               // [n_models][kMP][kMP]: QT[k][s] = Q[s][k], FP32, pads 0
    const double *mu;              // [n_models] uniformisation rates
    const int *bmodel;
    float *tabs;                   // [n][C][kTabKinds][kTabRows][kMP]
    float *post, *pre;             // [n_int][C][Ps][kMP]
    int *pe, *qe;                  // [n_int][C][Ps]
    double *gpart, *hpart;         // [n][n_ptiles]
    double *lpart;                 // [n_ptiles]
    int *status;
    float *site_invL;              // [Ps] 1 / Lhat_p
    int *site_Er;                  // [Ps]
    double *out_logL, *out_grad, *out_hess, *out_site;
    const double *gscale;
    int skip;
    int n_tips, n_nodes, root, n_levels, P, Ps, m, C, n_models, n_ptiles;
    int n_gslots;                  // per-branch gradient slots: pattern tiles (x categories, tensor-core path)
    int tc;                        // 1: tensor-core kernels and table layout, 0: SIMT
    double cw[kMaxCat], rates[kMaxCat];
    float pif[kMP];                // root frequencies, FP32 (pads 0)
    double pi[kMP];
};

// Tensor-core layout of the transition tables (pg_mtc.cu): per (branch, category) kTcKinds tables
// of kMP x kMP FP32, row-major W[s][k] (the K-major B operand of Y[p][s] = sum_k X[p][k] W[s][k]):
// D = P - I, G, their TF32 remainders (W - trunc_tf32(W)), D^T and remainder, H and remainder.
// The identity part of P x and P^T q is added to the products in FP32 by the kernels.
constexpr int kTcD = 0, kTcG = 1, kTcDlo = 2, kTcGlo = 3, kTcDT = 4, kTcDTlo = 5, kTcH = 6, kTcHlo = 7, kTcKinds = 8;
constexpr int kTcTile = 128;   // patterns per item of the tensor-core kernels (the MMA's M)

cudaError_t launch_m_pmatrix(const MDesc &d, bool hess, cudaStream_t s);
cudaError_t launch_m_post_level(const MDesc &d, int o0, int nd, cudaStream_t s);
cudaError_t launch_m_root(const MDesc &d, cudaStream_t s);
cudaError_t launch_m_pre_level(const MDesc &d, int o0, int nd, bool hess, cudaStream_t s);
cudaError_t launch_m_reduce(const MDesc &d, bool hess, cudaStream_t s);
// tensor-core level kernels; the maps describe d.post, d.pre (3-D: state, pattern, node * C +
// category) and d.tabs (2-D: state, table row) with 128-byte swizzled 32-float boxes
// level 0 of the tensor-core layout (both children tips): column lookups, no products
cudaError_t launch_m_post_cherry(const MDesc &d, int o0, int nd, cudaStream_t s);
cudaError_t launch_m_pre_cherry(const MDesc &d, int o0, int nd, cudaStream_t s);
cudaError_t launch_m_post_level_tc(const MDesc &d, const void *tm_post, const void *tm_tab, int o0, int nd,
                                   cudaStream_t s);
cudaError_t launch_m_pre_level_tc(const MDesc &d, const void *tm_post, const void *tm_pre, const void *tm_tab,
                                  int o0, int nd, bool hess, int n_sm, cudaStream_t s);

// launchers (pg_nt.cu); every problem of one launch shares C and precision
template <int MAXB>
cudaError_t launch_eval_nt(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s);
template <int MAXB>
cudaError_t launch_pmatrix(const BatchArgs<MAXB> &args, cudaStream_t s);
template <int MAXB>
cudaError_t launch_tree(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s);
template <int MAXB>
cudaError_t launch_reduce(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s);
// the fixed-order sum of k per-chunk results of length n (a problem evaluated in pattern chunks)
cudaError_t launch_chunk_sum(const double *parts, int k, int n, double *out, cudaStream_t s);
// resident blocks per SM of the tree kernel for C categories and the given precision
int tree_blocks_per_sm(int C, bool f64);
// the whole tree pass of a single small FP64 problem with its per-block vectors in shared memory
// (pg_small64.cu): the shared bytes one block of d's tiling needs, 0 when the kernel does not take
// d: not an FP64 problem with patterns, more than kSmall64MaxRange patterns per block (there the
// FP64 pipe, not the dependent chain, bounds a level, and the fused kernel's wider blocks keep it
// busier: measured 143 us against 94 us at 33 patterns per block), or more than kSmall64MaxSmem
constexpr size_t kSmall64MaxSmem = 200 * 1024;
constexpr int kSmall64MaxRange = 16;
size_t small64_smem_bytes(const ProbDesc &d);
cudaError_t launch_small64(const BatchArgs<1> &args, bool hess, cudaStream_t s);
// the levels [cut, n_levels) of a single FP32 problem with shared-memory-resident partials
// (pg_top.cu); returns cudaErrorNotSupported when they do not fit
cudaError_t launch_top(const BatchArgs<1> &args, bool hess, int n_sm, cudaStream_t s);
size_t top_smem_bytes(const ProbDesc &d);
// one level index of up to kMaxBatch problems in one launch: segment i covers problem
// d[i]'s nodes [o0[i], o0[i] + nd) x nr[i] pattern ranges, items [base[i], base[i + 1]); d[i] is
// the problem's descriptor in device memory
constexpr int kMaxLevelBatch = 128;   // problems per batched level launch (device descriptors)
struct LevelBatch {
    int n;
    int base[kMaxLevelBatch + 1];
    int o0[kMaxLevelBatch], nr[kMaxLevelBatch];
    const ProbDesc *d[kMaxLevelBatch];
};
cudaError_t launch_post_level_batch(const LevelBatch &lb, int C, int n_sm, bool cherry, cudaStream_t s);
cudaError_t launch_pre_level_batch(const LevelBatch &lb, int C, bool hess, int n_sm, bool cherry, cudaStream_t s);
// one post-order (pre-order) level [o0, o0 + nd) of a single FP32 problem (pg_levels.cu)
// (cherry: every node of the level has two tip children)
cudaError_t launch_post_level(const ProbDesc &d, int o0, int nd, int n_sm, bool cherry, cudaStream_t s);
// programmatic = false: a plain launch (it starts once the previous kernel has completed)
cudaError_t launch_pre_level(const ProbDesc &d, int o0, int nd, bool hess, int n_sm, bool cherry, cudaStream_t s,
                             bool programmatic = true);

}  // namespace pg
