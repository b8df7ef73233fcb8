// Level kernels for the wide tree levels of a single FP32 problem.
//
// Near the tips a level holds hundreds of nodes, so one launch per level has enough independent
// (node, pattern) work to fill the GPU by itself.  An item is one node of the level and a range of
// kLevelRange patterns.  Blocks are persistent and warp-specialised: they walk the items
// blockIdx.x, blockIdx.x + gridDim.x, ... through a ring of STAGES shared-memory stages.  A producer
// warp stages each item with a handful of 1-D bulk copies (TMA), one per contiguous row segment (the
// children's partial rows per rate category, q_k's rows, the log2 scales, tip codes, the per-pattern
// site values and the node's two branch tables), signalling a "full" mbarrier; kConsumerWarps
// consumer warps each compute 32 patterns of the item and release the stage on an "empty" mbarrier.
// No block-wide barrier is taken inside the loop.  Bytes in flight are bounded by shared memory, not
// by registers, and no block depends on another within a launch.
//
// The arithmetic is that of the fused tree kernel (pg_nt.cu): the exact-product post-order update
// of Section 2.3, and the pre-order step of Section 2.4 with the branch gradient (Section 2.5) and
// Hessian diagonal (Section 2.6).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

// CHERRY: every node of the level has two tip children (height-1 nodes), so a stage carries no
// child partial rows or scales.  A stage holds one item of R patterns: level_range(C), or that many
// times post_cherry_ranges(C) / pre_cherry_ranges(C) for a cherry level.  Every bulk-copy
// destination starts on a 16-byte boundary.
template <int C, bool CHERRY = false>
struct PostStage {
    static constexpr int R = level_range(C) * (CHERRY ? post_cherry_ranges(C) : 1);
    static constexpr int RX = CHERRY ? 1 : R;   // child rows and scales (none for a cherry level)
    alignas(16) float4 x0[C][RX];
    alignas(16) float4 x1[C][RX];   // children's partial rows
    alignas(16) int e0[RX];
    alignas(16) int e1[RX];         // children's log2 scales
    alignas(16) uint8_t y0[R];
    alignas(16) uint8_t y1[R];      // tip codes
    alignas(16) float4 tab[2][C][kPtabCols];   // both branches' tables
};

template <int C, bool CHERRY = false>
struct PreStage {
    static constexpr int R = level_range(C) * (CHERRY ? pre_cherry_ranges(C) : 1);
    static constexpr int RX = CHERRY ? 1 : R;
    alignas(16) float4 qk[C][R];
    alignas(16) float4 x0[C][RX];
    alignas(16) float4 x1[C][RX];
    alignas(16) int eq[R];
    alignas(16) int e0[RX];
    alignas(16) int e1[RX];
    alignas(16) int er[R];          // log2 scale of L_p
    alignas(16) float inv[R];       // 1 / Lhat_p
    alignas(16) float w[R];         // pattern weights
    alignas(16) uint8_t y0[R];
    alignas(16) uint8_t y1[R];
    // both branches' tables: P hi columns and row sums, then G = Q P alike (the first 10 columns),
    // staged with one copy per branch (all C tables, which for C > 1 includes the other columns)
    static constexpr int TC = C == 1 ? 10 : kPtabCols;
    alignas(16) float4 tab[2][C][TC];
    alignas(16) float4 qtab[2][4];           // Q columns of both children's models (not staged for a cherry level
                                 // without the Hessian: tips take G's columns)
};

constexpr int kConsumerWarps = kLevelRange / 32;
constexpr int kLevelThreads = kLevelRange + 32;   // consumers + one producer warp

template <class Stage, int STAGES>
struct Ring {
    Stage st[STAGES];
    uint64_t full[STAGES];    // producer: arrive with the stage's transaction bytes
    uint64_t empty[STAGES];   // consumers: one arrival per consumer warp when done reading
};

__device__ __forceinline__ unsigned round16(unsigned b) { return (b + 15u) & ~15u; }

struct Item {
    const ProbDesc *pd;   // the item's problem
    int4 op;
    int rg, p0, cnt;
};

// item j of a level whose nodes (from ops[o0]) have nr items each of KC ranges of level_range(C)
// patterns; it.rg counts items, i.e. KC ranges
template <int KC>
__device__ __forceinline__ Item item_of(const ProbDesc &d, int o0, int nr, int j) {
    Item it;
    it.pd = &d;
    const int u = j / nr;
    it.rg = j - u * nr;
    it.op = __ldg(d.ops + o0 + u);
    const int RL = level_range(d.C) * KC;
    it.p0 = it.rg * RL;
    it.cnt = min(RL, d.P - it.p0);
    return it;
}

// part 0: every copy of the item; part 1: the stage's byte count and the copies that do not depend
// on the previous post-order launch (tables, tip codes, and the rows and scales of internal children
// two or more levels below: a post-order level above level 0 starts only after its predecessor's
// wait, i.e. after every earlier launch completed); part 2: the rows and scales of children on the
// level just below (op.w bits 0 and 1)
template <int C, bool CHERRY>
__device__ void issue_post(const ProbDesc &d, const Item &it, PostStage<C, CHERRY> &sm, uint64_t *bar, int part = 0) {
    const int N = d.n_tips, Ps = d.Ps, c0 = it.op.y, c1 = it.op.z, p0 = it.p0;
    const bool t0 = c0 < N, t1 = c1 < N;
    const float4 *post = static_cast<const float4 *>(d.post);
    const unsigned rowb = (unsigned)it.cnt * 16u, eb = round16(it.cnt * 4u), yb = round16((unsigned)it.cnt);
    // which copies this call makes: part 1 the independent ones, part 2 the rest
    const int fl = it.op.w;
    const bool late0 = (fl & 1) != 0, late1 = (fl & 2) != 0;
    const bool rows0 = !t0 && (part == 0 || (part == 1) != late0), rows1 = !t1 && (part == 0 || (part == 1) != late1);
    if (part != 2) {
        unsigned bytes = 2u * C * kPtabCols * 16u;
        bytes += t0 ? yb : (C * rowb + eb);
        bytes += t1 ? yb : (C * rowb + eb);
        mbar_arrive_expect(bar, bytes);
        bulk_load(sm.tab[0], d.Ptab + (size_t)c0 * C * kPtabCols, C * kPtabCols * 16u, bar);
        bulk_load(sm.tab[1], d.Ptab + (size_t)c1 * C * kPtabCols, C * kPtabCols * 16u, bar);
        if (t0) bulk_load(sm.y0, d.tips + (size_t)c0 * Ps + p0, yb, bar);
        if (t1) bulk_load(sm.y1, d.tips + (size_t)c1 * Ps + p0, yb, bar);
    }
    if constexpr (!CHERRY) {
        if (rows0) {
            bulk_load(sm.e0, d.pe + (size_t)(c0 - N) * Ps + p0, eb, bar);
            for (int l = 0; l < C; ++l) bulk_load(sm.x0[l], post + ((size_t)(c0 - N) * C + l) * Ps + p0, rowb, bar);
        }
        if (rows1) {
            bulk_load(sm.e1, d.pe + (size_t)(c1 - N) * Ps + p0, eb, bar);
            for (int l = 0; l < C; ++l) bulk_load(sm.x1[l], post + ((size_t)(c1 - N) * C + l) * Ps + p0, rowb, bar);
        }
    }
}

// part 0: every copy of the item; part 1: the stage's byte count and the copies that do not depend
// on the previous pre-order launch (tables, the children's post-order rows and scales, tip codes,
// weights: complete before any pre-order launch starts); part 2: the rest (q_k and its scales, the
// per-site values written by the root's kernel)
template <int C, bool HESS, bool CHERRY>
__device__ void issue_pre(const ProbDesc &d, const Item &it, PreStage<C, CHERRY> &sm, uint64_t *bar, int part = 0) {
    const int N = d.n_tips, Ps = d.Ps, k = it.op.x, c0 = it.op.y, c1 = it.op.z, p0 = it.p0;
    const bool t0 = c0 < N, t1 = c1 < N;
    const float4 *post = static_cast<const float4 *>(d.post);
    const float4 *pre = static_cast<const float4 *>(d.pre);
    const unsigned rowb = (unsigned)it.cnt * 16u, eb = round16(it.cnt * 4u), yb = round16((unsigned)it.cnt);
    constexpr bool kQ = HESS || !CHERRY;   // the Q columns are read by some product
    constexpr unsigned tb = C * PreStage<C, CHERRY>::TC * 16u;   // a branch's staged tables
    unsigned bytes = C * rowb + eb + 3u * eb + 2u * tb + (kQ ? 2u * 64u : 0u);
    bytes += t0 ? yb : (C * rowb + eb);
    bytes += t1 ? yb : (C * rowb + eb);
    if (part == 2) {
        bulk_load(sm.eq, d.qe + (size_t)(k - N) * Ps + p0, eb, bar);
        for (int l = 0; l < C; ++l) bulk_load(sm.qk[l], pre + ((size_t)(k - N) * C + l) * Ps + p0, rowb, bar);
        bulk_load(sm.er, d.site_Er + p0, eb, bar);
        bulk_load(sm.inv, d.site_invL + p0, eb, bar);
        return;
    }
    mbar_arrive_expect(bar, bytes);
    for (int side = 0; side < 2; ++side) {   // one copy per branch: its C tables are contiguous
        const int c = side ? c1 : c0;
        bulk_load(sm.tab[side], d.Ptab + (size_t)c * C * kPtabCols, tb, bar);
        if (kQ) bulk_load(sm.qtab[side], d.Qf + 4 * (d.bmodel ? d.bmodel[c] : 0), 64u, bar);
    }
    if (part == 0) {
        bulk_load(sm.eq, d.qe + (size_t)(k - N) * Ps + p0, eb, bar);
        for (int l = 0; l < C; ++l) bulk_load(sm.qk[l], pre + ((size_t)(k - N) * C + l) * Ps + p0, rowb, bar);
        bulk_load(sm.er, d.site_Er + p0, eb, bar);
        bulk_load(sm.inv, d.site_invL + p0, eb, bar);
    }
    bulk_load(sm.w, d.wf + p0, eb, bar);
    if (t0) bulk_load(sm.y0, d.tips + (size_t)c0 * Ps + p0, yb, bar);
    else if constexpr (!CHERRY) {
        bulk_load(sm.e0, d.pe + (size_t)(c0 - N) * Ps + p0, eb, bar);
        for (int l = 0; l < C; ++l) bulk_load(sm.x0[l], post + ((size_t)(c0 - N) * C + l) * Ps + p0, rowb, bar);
    }
    if (t1) bulk_load(sm.y1, d.tips + (size_t)c1 * Ps + p0, yb, bar);
    else if constexpr (!CHERRY) {
        bulk_load(sm.e1, d.pe + (size_t)(c1 - N) * Ps + p0, eb, bar);
        for (int l = 0; l < C; ++l) bulk_load(sm.x1[l], post + ((size_t)(c1 - N) * C + l) * Ps + p0, rowb, bar);
    }
}

// post-order update (Section 2.3) of pattern t of one item from its stage
template <int C, bool CHERRY>
__device__ __forceinline__ void compute_post_one(const ProbDesc &d, const Item &it, const PostStage<C, CHERRY> &sm, int t) {
    if (t >= it.cnt) return;
    const int N = d.n_tips, Ps = d.Ps, k = it.op.x, c0 = it.op.y, c1 = it.op.z;
    const bool t0 = CHERRY || c0 < N, t1 = CHERRY || c1 < N;
    const int p = it.p0 + t;
    const float r = pattern_factor((uint32_t)p);
    const int y0 = t0 ? min((int)sm.y0[t], 4) : 0, y1 = t1 ? min((int)sm.y1[t], 4) : 0;
    const int E = (t0 ? 0 : sm.e0[t]) + (t1 ? 0 : sm.e1[t]);
    float4 v[C];
    float mx = 0.0f;
    if (CHERRY || (t0 && t1)) {   // a cherry: both contributions are (hi + lo) columns times r, one product each
#pragma unroll
        for (int l = 0; l < C; ++l) {
            const float4 h0 = sm.tab[0][l][y0], l0 = sm.tab[0][l][kColPlo + y0];
            const float4 h1 = sm.tab[1][l][y1], l1 = sm.tab[1][l][kColPlo + y1];
            const float4 x0 = f4(fmaf(h0.x, r, l0.x * r), fmaf(h0.y, r, l0.y * r), fmaf(h0.z, r, l0.z * r), fmaf(h0.w, r, l0.w * r));
            const float4 x1 = f4(fmaf(h1.x, r, l1.x * r), fmaf(h1.y, r, l1.y * r), fmaf(h1.z, r, l1.z * r), fmaf(h1.w, r, l1.w * r));
            v[l] = mul(x0, x1);
            mx = fmaxf(mx, hmax(v[l]));
        }
    } else if constexpr (!CHERRY) {
#pragma unroll
        for (int l = 0; l < C; ++l) {
            float4 x0, x1, s0 = f4(0.f, 0.f, 0.f, 0.f), s1 = f4(0.f, 0.f, 0.f, 0.f);
            if (t0) {
                const float4 hi = sm.tab[0][l][y0], lo = sm.tab[0][l][kColPlo + y0];
                x0 = f4(fmaf(hi.x, r, lo.x * r), fmaf(hi.y, r, lo.y * r), fmaf(hi.z, r, lo.z * r), fmaf(hi.w, r, lo.w * r));
            } else {
                x0 = sm.x0[l][t];
                s0 = matvec_hilo_v(&sm.tab[0][l][kColDhi], &sm.tab[0][l][kColDlo], x0);
            }
            if (t1) {
                const float4 hi = sm.tab[1][l][y1], lo = sm.tab[1][l][kColPlo + y1];
                x1 = f4(fmaf(hi.x, r, lo.x * r), fmaf(hi.y, r, lo.y * r), fmaf(hi.z, r, lo.z * r), fmaf(hi.w, r, lo.w * r));
            } else {
                x1 = sm.x1[l][t];
                s1 = matvec_hilo_v(&sm.tab[1][l][kColDhi], &sm.tab[1][l][kColDlo], x1);
            }
            v[l] = f4(prod_split(x0.x, s0.x, x1.x, s1.x), prod_split(x0.y, s0.y, x1.y, s1.y),
                      prod_split(x0.z, s0.z, x1.z, s1.z), prod_split(x0.w, s0.w, x1.w, s1.w));
            mx = fmaxf(mx, hmax(v[l]));
        }
    }
    const int e = scale_exponent(mx);
    float4 *out = static_cast<float4 *>(d.post);
#pragma unroll
    for (int l = 0; l < C; ++l) __stcg(out + ((size_t)(k - N) * C + l) * Ps + p, scale4(v[l], e));
    __stcg(d.pe + (size_t)(k - N) * Ps + p, E + e);
}
// the item's patterns t, t + kLevelRange, ... of consumer thread t
template <int C, bool CHERRY>
__device__ __forceinline__ void compute_post(const ProbDesc &d, const Item &it, const PostStage<C, CHERRY> &sm, int t) {
#pragma unroll 1
    for (int tt = t; tt < PostStage<C, CHERRY>::R; tt += kLevelRange) compute_post_one<C, CHERRY>(d, it, sm, tt);
}

// pre-order step (Section 2.4) with the branch gradient (2.5) and Hessian diagonal (2.6) of pattern
// t of one item: writes q of internal children, returns the pattern's weighted branch terms
template <int C, bool HESS, bool CHERRY>
__device__ __forceinline__ void compute_pre_one(const ProbDesc &d, const Item &it, const PreStage<C, CHERRY> &sm, int t,
                                                float (&sums)[4]) {
    const int N = d.n_tips, Ps = d.Ps, c0 = it.op.y, c1 = it.op.z;
    const bool t0 = CHERRY || c0 < N, t1 = CHERRY || c1 < N;
    const bool active = t < it.cnt;
    const int tt = active ? t : it.cnt - 1;
    const int p = it.p0 + tt;
    const float r = pattern_factor((uint32_t)p);
    const int y0 = t0 ? min((int)sm.y0[tt], 4) : 0, y1 = t1 ? min((int)sm.y1[tt], 4) : 0;
    const int Eq = sm.eq[tt], E0 = t0 ? 0 : sm.e0[tt], E1 = t1 ? 0 : sm.e1[tt];
    const float inv = sm.inv[tt], wt = active ? sm.w[tt] : 0.f;
    const int dE = Eq + E0 + E1 - sm.er[tt];
    float4 q0[C], q1[C];
    float m0 = 0.f, m1 = 0.f, g0 = 0.f, g1 = 0.f, h0 = 0.f, h1 = 0.f;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        const float4 a0 = t0 ? scal(sm.tab[0][l][y0], r) : matvec_p(sm.tab[0][l], sm.x0[l][CHERRY ? 0 : tt]);
        const float4 a1 = t1 ? scal(sm.tab[1][l][y1], r) : matvec_p(sm.tab[1][l], sm.x1[l][CHERRY ? 0 : tt]);
        const float4 qk = sm.qk[l][tt];
        const float4 qt0 = mul(qk, a1), qt1 = mul(qk, a0);   // top of branches c0 and c1
        // Q a_c: a gathered column of G = Q P for tips, a matvec otherwise
        const float4 u0 = t0 ? scal(sm.tab[0][l][kColG + y0], r) : matvec_p(sm.qtab[0], a0);
        const float4 u1 = t1 ? scal(sm.tab[1][l][kColG + y1], r) : matvec_p(sm.qtab[1], a1);
        g0 = fmaf(d.gw[l], dot(qt0, u0), g0);
        g1 = fmaf(d.gw[l], dot(qt1, u1), g1);
        if (HESS) {
            h0 = fmaf(d.gw2[l], dot(qt0, matvec_p(sm.qtab[0], u0)), h0);
            h1 = fmaf(d.gw2[l], dot(qt1, matvec_p(sm.qtab[1], u1)), h1);
        }
        if (!t0) { q0[l] = matvec_tp(sm.tab[0][l], qt0); m0 = fmaxf(m0, hmax(q0[l])); }
        if (!t1) { q1[l] = matvec_tp(sm.tab[1][l], qt1); m1 = fmaxf(m1, hmax(q1[l])); }
    }
    float4 *pre = static_cast<float4 *>(d.pre);
    if (!t0 && active) {
        const int e = scale_exponent(m0);
#pragma unroll
        for (int l = 0; l < C; ++l) __stcg(pre + ((size_t)(c0 - N) * C + l) * Ps + p, scale4(q0[l], e));
        __stcg(d.qe + (size_t)(c0 - N) * Ps + p, Eq + E1 + e);
    }
    if (!t1 && active) {
        const int e = scale_exponent(m1);
#pragma unroll
        for (int l = 0; l < C; ++l) __stcg(pre + ((size_t)(c1 - N) * C + l) * Ps + p, scale4(q1[l], e));
        __stcg(d.qe + (size_t)(c1 - N) * Ps + p, Eq + E0 + e);
    }
    const float d0 = ldexp2f(g0, dE) * inv, d1 = ldexp2f(g1, dE) * inv;
    sums[0] = wt != 0.f ? wt * d0 : 0.f;
    sums[1] = wt != 0.f ? wt * d1 : 0.f;
    sums[2] = (HESS && wt != 0.f) ? wt * (ldexp2f(h0, dE) * inv - d0 * d0) : 0.f;
    sums[3] = (HESS && wt != 0.f) ? wt * (ldexp2f(h1, dE) * inv - d1 * d1) : 0.f;
}
// the warp's sums of one range into its slot of both child branches (lane 0; slot = 4 * range + warp;
// the reduction adds the slots in FP64 in a fixed order)
template <bool HESS>
__device__ __forceinline__ void store_slot_sums(const ProbDesc &d, const int4 op, int slot, int lane, const float (&acc)[4]) {
#pragma unroll
    for (int s = 0; s < (HESS ? 4 : 2); ++s) {
        const float v = warp_sum_f(acc[s]);
        if (lane == 0) {
            double *dst = (s < 2) ? d.gpart : d.hpart;
            dst[(size_t)((s & 1) ? op.z : op.y) * d.slot_cap + slot] = (double)v;
        }
    }
}

// the item's patterns t, t + kLevelRange, ... of consumer thread t; per range of level_range(C)
// patterns each thread adds its patterns' terms, then the warp adds its 32 lanes (all in FP32:
// level_range(C) / 4 patterns per slot, no FP64 instruction, which this GPU issues at a small
// fraction of the FP32 rate) and stores the sums in its slot.  A cherry item of KC > 1 ranges does
// this range by range.
template <int C, bool HESS, bool CHERRY>
__device__ __forceinline__ void compute_pre(const ProbDesc &d, const Item &it, const PreStage<C, CHERRY> &sm, int t) {
    constexpr int LR = level_range(C), KC = PreStage<C, CHERRY>::R / LR;
    const int lane = t & 31;
    if constexpr (KC == 1 && LR == kLevelRange) {   // one pattern per thread
        float sums[4];
        compute_pre_one<C, HESS, CHERRY>(d, it, sm, t, sums);
        store_slot_sums<HESS>(d, it.op, it.rg * kConsumerWarps + (t >> 5), lane, sums);
    } else if constexpr (KC == 1) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int tt = t; tt < LR; tt += kLevelRange) {
            float sums[4];
            compute_pre_one<C, HESS, CHERRY>(d, it, sm, tt, sums);
#pragma unroll
            for (int s = 0; s < (HESS ? 4 : 2); ++s) acc[s] += sums[s];
        }
        store_slot_sums<HESS>(d, it.op, it.rg * kConsumerWarps + (t >> 5), lane, acc);
    } else {
#pragma unroll 1
        for (int h = 0; h < KC; ++h) {
            const int g = it.rg * KC + h;   // the range whose slots this pass fills
            if (g >= d.level_ranges) break; // (the last item's ranges past the last pattern)
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
            for (int tt = t + h * LR; tt < (h + 1) * LR; tt += kLevelRange) {
                float sums[4];
                compute_pre_one<C, HESS, CHERRY>(d, it, sm, tt, sums);
#pragma unroll
                for (int s = 0; s < (HESS ? 4 : 2); ++s) acc[s] += sums[s];
            }
            store_slot_sums<HESS>(d, it.op, g * kConsumerWarps + (t >> 5), lane, acc);
        }
    }
}

// The persistent, warp-specialised walk over a level's items shared by both passes.  Warp
// kConsumerWarps is the producer: its lane 0 refills stage s once the consumers released it and
// issues the item's bulk copies.  Consumer warps wait for the stage to be full, compute their 32
// patterns and release it.  Every wait is bounded; a warp that gives up records PG_ERR_TIMEOUT and
// leaves (the producer first lets the copies it issued land).
// PREFETCH: the producer loads the next item's record one item ahead (measured: faster for the
// post-order levels, slower for the pre-order levels)
// EARLY: before waiting for the previous launch, the producer issues the part of its first STAGES
// items' copies that does not depend on that launch (issue part 1), and the rest after the wait
// (part 2); the copies of later items are issued whole (part 0).
template <bool PREFETCH, bool EARLY, bool LATE_TRIGGER, class Stage, int STAGES, class ItemFn, class Issue, class Compute>
__device__ __forceinline__ void staged_walk(int n_items, Ring<Stage, STAGES> &ring, ItemFn &&item_at, Issue &&issue,
                                            Compute &&compute) {
    const int G = gridDim.x, b = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&ring.full[s], 1);
            mbar_init(&ring.empty[s], kConsumerWarps);
        }
    }
    __syncthreads();   // barriers initialised before anyone uses them
    // LATE_TRIGGER (post-order levels): a thread lets the next launch be scheduled only after its own
    // wait, so a launch that has started knows every launch but its predecessor complete (the next
    // post-order level copies older children's rows early; the top kernel its P tables)
    if constexpr (!LATE_TRIGGER) pdl_launch_dependents();
    if (warp == kConsumerWarps) {   // producer
        if (lane != 0) return;
        int i = 0;
        if constexpr (EARLY) {
            for (; i < STAGES && b + i * G < n_items; ++i) issue(item_at(b + i * G), ring.st[i], &ring.full[i], 1);
        }
        pdl_wait();   // the previous level's partials are complete and visible
        if constexpr (LATE_TRIGGER) pdl_launch_dependents();
        for (int q = 0; q < i; ++q) issue(item_at(b + q * G), ring.st[q], &ring.full[q], 2);
        Item nxt = (PREFETCH && b + i * G < n_items) ? item_at(b + i * G) : Item{};
        for (;; ++i) {
            const int j = b + i * G;
            if (j >= n_items) break;
            const int s = i % STAGES, use = i / STAGES;
            const Item it = PREFETCH ? nxt : item_at(j);
            if (PREFETCH && j + G < n_items) nxt = item_at(j + G);
            if (use > 0 && !mbar_wait_bounded(&ring.empty[s], (unsigned)(use - 1) & 1u, kWaitLimitCycles)) {
                atomicOr(it.pd->status, kStatusTimeout);
                break;
            }
            issue(it, ring.st[s], &ring.full[s], 0);
        }
        // let every copy issued by this warp land before the block may leave
        for (int q = (i > STAGES ? i - STAGES : 0); q < i; ++q)
            if (!mbar_wait_bounded(&ring.full[q % STAGES], (unsigned)(q / STAGES) & 1u, kWaitLimitCycles))
                atomicOr(item_at(b + q * G).pd->status, kStatusTimeout | kStatusUnsettled);
        return;
    }
    pdl_wait();   // (the consumers read only the stages; kept so no thread runs ahead of the launch order)
    if constexpr (LATE_TRIGGER) pdl_launch_dependents();
    for (int i = 0;; ++i) {   // consumers
        const int j = b + i * G;
        if (j >= n_items) break;
        const int s = i % STAGES;
        const Item it = item_at(j);
        if (!mbar_wait_bounded(&ring.full[s], (unsigned)(i / STAGES) & 1u, kWaitLimitCycles)) {
            if (lane == 0) atomicOr(it.pd->status, kStatusTimeout);
            return;
        }
        compute(it, ring.st[s], threadIdx.x);
        __syncwarp();
        if (lane == 0) mbar_arrive(&ring.empty[s]);
    }
}

// the item source of one problem's level, or of one level index across a batch of problems
// (KC ranges of level_range(C) patterns per item)
template <int KC>
struct OneLevel {
    const ProbDesc &d;
    int o0, nr;
    __device__ Item operator()(int j) const { return item_of<KC>(d, o0, nr, j); }
};
template <int KC>
struct BatchLevel {
    const LevelBatch &lb;
    __device__ Item operator()(int j) const {
        int lo = 0, hi = lb.n - 1;   // the segment holding item j: base[lo] <= j < base[lo + 1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (lb.base[mid] <= j) lo = mid;
            else hi = mid - 1;
        }
        return item_of<KC>(*lb.d[lo], lb.o0[lo], lb.nr[lo], j - lb.base[lo]);
    }
};

template <int C, int STAGES, bool CHERRY, class Src>
__device__ __forceinline__ void post_walk(int n_items, const Src &src) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using St = PostStage<C, CHERRY>;
    auto &ring = *reinterpret_cast<Ring<St, STAGES> *>(smem_raw);
    staged_walk<true, !CHERRY, true>(n_items, ring, src,
                [&](const Item &it, St &st, uint64_t *bar, int part) { issue_post<C, CHERRY>(*it.pd, it, st, bar, part); },
                [&](const Item &it, const St &st, int t) { compute_post<C, CHERRY>(*it.pd, it, st, t); });
}
template <int C, bool HESS, int STAGES, bool CHERRY, class Src>
__device__ __forceinline__ void pre_walk(int n_items, const Src &src) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using St = PreStage<C, CHERRY>;
    auto &ring = *reinterpret_cast<Ring<St, STAGES> *>(smem_raw);
    staged_walk<false, true, false>(n_items, ring, src,
                [&](const Item &it, St &st, uint64_t *bar, int part) { issue_pre<C, HESS, CHERRY>(*it.pd, it, st, bar, part); },
                [&](const Item &it, const St &st, int t) { compute_pre<C, HESS, CHERRY>(*it.pd, it, st, t); });
}

template <int C, int STAGES, bool CHERRY>
__global__ void __launch_bounds__(kLevelThreads) post_level_kernel(const __grid_constant__ ProbDesc d, int o0, int nr, int n_items) {
    post_walk<C, STAGES, CHERRY>(n_items, OneLevel<CHERRY ? post_cherry_ranges(C) : 1>{d, o0, nr});
}
template <int C, bool HESS, int STAGES, bool CHERRY>
__global__ void __launch_bounds__(kLevelThreads) pre_level_kernel(const __grid_constant__ ProbDesc d, int o0, int nr, int n_items) {
    pre_walk<C, HESS, STAGES, CHERRY>(n_items, OneLevel<CHERRY ? pre_cherry_ranges(C) : 1>{d, o0, nr});
}
// one level index of every problem of a batch (descriptors in device memory)
template <int C, int STAGES, bool CHERRY>
__global__ void __launch_bounds__(kLevelThreads) post_level_batch_kernel(const __grid_constant__ LevelBatch lb, int n_items) {
    post_walk<C, STAGES, CHERRY>(n_items, BatchLevel<CHERRY ? post_cherry_ranges(C) : 1>{lb});
}
template <int C, bool HESS, int STAGES, bool CHERRY>
__global__ void __launch_bounds__(kLevelThreads) pre_level_batch_kernel(const __grid_constant__ LevelBatch lb, int n_items) {
    pre_walk<C, HESS, STAGES, CHERRY>(n_items, BatchLevel<CHERRY ? pre_cherry_ranges(C) : 1>{lb});
}

constexpr int kPostStages = 2, kPreStages = 2, kPostCherryStages = 3;
// the pre-order cherry stage holds q_k's rows and four per-pattern arrays; for C <= 2, items of four
// ranges in two stages (three blocks per SM) measured slightly faster than two ranges in three
constexpr int pre_cherry_stages(int C) { return C <= 2 ? 2 : 3; }

// blocks of a persistent level launch: every resident slot, at most one per item
// (the attribute and the occupancy are set up once per device and instantiation)
template <class K>
int persistent_blocks(K kernel, size_t smem, int n_sm, int n_items, DeviceOnce &once) {
    int per_sm = 1;
    const cudaError_t e = device_once(once, [&](int &v) {
        cudaError_t r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r == cudaSuccess) r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kLevelThreads, smem);
        if (v < 1) v = 1;
        return r;
    }, &per_sm);
    if (e != cudaSuccess) return -1;
    return n_items < n_sm * per_sm ? n_items : n_sm * per_sm;
}

// launch with programmatic stream serialisation: the kernel may be scheduled while the previous
// one drains, and waits for it in pdl_wait() (programmatic = false: a plain launch, pdl_wait() then
// returns at once)
template <class K>
cudaError_t launch_pdl(K kernel, int blocks, size_t smem, cudaStream_t s, const ProbDesc &d, int o0, int nr, int n_items,
                       bool programmatic = true) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kLevelThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = programmatic ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, d, o0, nr, n_items);
}

template <class K, class A>
cudaError_t launch_pdl_batch(K kernel, int blocks, size_t smem, cudaStream_t s, const A &lb, int n_items) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kLevelThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, lb, n_items);
}

template <int C, bool CHERRY>
cudaError_t post_batch_c(const LevelBatch &lb, int n_sm, cudaStream_t s) {
    static DeviceOnce once;
    constexpr int ST = CHERRY ? kPostCherryStages : kPostStages;
    const int n_items = lb.base[lb.n];
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = sizeof(Ring<PostStage<C, CHERRY>, ST>);
    const int blocks = persistent_blocks(post_level_batch_kernel<C, ST, CHERRY>, smem, n_sm, n_items, once);
    if (blocks < 0) return cudaErrorInvalidConfiguration;
    return launch_pdl_batch(post_level_batch_kernel<C, ST, CHERRY>, blocks, smem, s, lb, n_items);
}

template <int C, bool HESS, bool CHERRY>
cudaError_t pre_batch_c(const LevelBatch &lb, int n_sm, cudaStream_t s) {
    static DeviceOnce once;
    constexpr int ST = CHERRY ? pre_cherry_stages(C) : kPreStages;
    const int n_items = lb.base[lb.n];
    if (n_items <= 0) return cudaSuccess;
    const size_t smem = sizeof(Ring<PreStage<C, CHERRY>, ST>);
    const int blocks = persistent_blocks(pre_level_batch_kernel<C, HESS, ST, CHERRY>, smem, n_sm, n_items, once);
    if (blocks < 0) return cudaErrorInvalidConfiguration;
    return launch_pdl_batch(pre_level_batch_kernel<C, HESS, ST, CHERRY>, blocks, smem, s, lb, n_items);
}

template <int C, bool CHERRY>
cudaError_t post_c(const ProbDesc &d, int o0, int nd, int n_sm, cudaStream_t s) {
    static DeviceOnce once;   // attribute and occupancy, once per device and instantiation
    constexpr int ST = CHERRY ? kPostCherryStages : kPostStages;
    const int nr = CHERRY ? level_items_per_node(d.P, C, post_cherry_ranges(C)) : d.level_ranges, n_items = nd * nr;
    const size_t smem = sizeof(Ring<PostStage<C, CHERRY>, ST>);
    const int blocks = persistent_blocks(post_level_kernel<C, ST, CHERRY>, smem, n_sm, n_items, once);
    if (blocks < 0) return cudaErrorInvalidConfiguration;
    return launch_pdl(post_level_kernel<C, ST, CHERRY>, blocks, smem, s, d, o0, nr, n_items);
}

template <int C, bool HESS, bool CHERRY>
cudaError_t pre_c(const ProbDesc &d, int o0, int nd, int n_sm, cudaStream_t s, bool programmatic) {
    static DeviceOnce once;
    constexpr int ST = CHERRY ? pre_cherry_stages(C) : kPreStages;
    const int nr = CHERRY ? level_items_per_node(d.P, C, pre_cherry_ranges(C)) : d.level_ranges, n_items = nd * nr;
    const size_t smem = sizeof(Ring<PreStage<C, CHERRY>, ST>);
    const int blocks = persistent_blocks(pre_level_kernel<C, HESS, ST, CHERRY>, smem, n_sm, n_items, once);
    if (blocks < 0) return cudaErrorInvalidConfiguration;
    return launch_pdl(pre_level_kernel<C, HESS, ST, CHERRY>, blocks, smem, s, d, o0, nr, n_items, programmatic);
}

}  // namespace

cudaError_t launch_post_level(const ProbDesc &d, int o0, int nd, int n_sm, bool cherry, cudaStream_t s) {
    switch (d.C * 2 + (cherry ? 1 : 0)) {
        case 2: return post_c<1, false>(d, o0, nd, n_sm, s);
        case 3: return post_c<1, true>(d, o0, nd, n_sm, s);
        case 4: return post_c<2, false>(d, o0, nd, n_sm, s);
        case 5: return post_c<2, true>(d, o0, nd, n_sm, s);
        case 6: return post_c<3, false>(d, o0, nd, n_sm, s);
        case 7: return post_c<3, true>(d, o0, nd, n_sm, s);
        case 8: return post_c<4, false>(d, o0, nd, n_sm, s);
        case 9: return post_c<4, true>(d, o0, nd, n_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pre_level(const ProbDesc &d, int o0, int nd, bool hess, int n_sm, bool cherry, cudaStream_t s,
                             bool programmatic) {
    switch (d.C * 4 + (hess ? 2 : 0) + (cherry ? 1 : 0)) {
        case 4: return pre_c<1, false, false>(d, o0, nd, n_sm, s, programmatic);
        case 5: return pre_c<1, false, true>(d, o0, nd, n_sm, s, programmatic);
        case 6: return pre_c<1, true, false>(d, o0, nd, n_sm, s, programmatic);
        case 7: return pre_c<1, true, true>(d, o0, nd, n_sm, s, programmatic);
        case 8: return pre_c<2, false, false>(d, o0, nd, n_sm, s, programmatic);
        case 9: return pre_c<2, false, true>(d, o0, nd, n_sm, s, programmatic);
        case 10: return pre_c<2, true, false>(d, o0, nd, n_sm, s, programmatic);
        case 11: return pre_c<2, true, true>(d, o0, nd, n_sm, s, programmatic);
        case 12: return pre_c<3, false, false>(d, o0, nd, n_sm, s, programmatic);
        case 13: return pre_c<3, false, true>(d, o0, nd, n_sm, s, programmatic);
        case 14: return pre_c<3, true, false>(d, o0, nd, n_sm, s, programmatic);
        case 15: return pre_c<3, true, true>(d, o0, nd, n_sm, s, programmatic);
        case 16: return pre_c<4, false, false>(d, o0, nd, n_sm, s, programmatic);
        case 17: return pre_c<4, false, true>(d, o0, nd, n_sm, s, programmatic);
        case 18: return pre_c<4, true, false>(d, o0, nd, n_sm, s, programmatic);
        case 19: return pre_c<4, true, true>(d, o0, nd, n_sm, s, programmatic);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_post_level_batch(const LevelBatch &lb, int C, int n_sm, bool cherry, cudaStream_t s) {
    switch (C * 2 + (cherry ? 1 : 0)) {
        case 2: return post_batch_c<1, false>(lb, n_sm, s);
        case 3: return post_batch_c<1, true>(lb, n_sm, s);
        case 4: return post_batch_c<2, false>(lb, n_sm, s);
        case 5: return post_batch_c<2, true>(lb, n_sm, s);
        case 6: return post_batch_c<3, false>(lb, n_sm, s);
        case 7: return post_batch_c<3, true>(lb, n_sm, s);
        case 8: return post_batch_c<4, false>(lb, n_sm, s);
        case 9: return post_batch_c<4, true>(lb, n_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_pre_level_batch(const LevelBatch &lb, int C, bool hess, int n_sm, bool cherry, cudaStream_t s) {
    switch (C * 4 + (hess ? 2 : 0) + (cherry ? 1 : 0)) {
        case 4: return pre_batch_c<1, false, false>(lb, n_sm, s);
        case 5: return pre_batch_c<1, false, true>(lb, n_sm, s);
        case 6: return pre_batch_c<1, true, false>(lb, n_sm, s);
        case 7: return pre_batch_c<1, true, true>(lb, n_sm, s);
        case 8: return pre_batch_c<2, false, false>(lb, n_sm, s);
        case 9: return pre_batch_c<2, false, true>(lb, n_sm, s);
        case 10: return pre_batch_c<2, true, false>(lb, n_sm, s);
        case 11: return pre_batch_c<2, true, true>(lb, n_sm, s);
        case 12: return pre_batch_c<3, false, false>(lb, n_sm, s);
        case 13: return pre_batch_c<3, false, true>(lb, n_sm, s);
        case 14: return pre_batch_c<3, true, false>(lb, n_sm, s);
        case 15: return pre_batch_c<3, true, true>(lb, n_sm, s);
        case 16: return pre_batch_c<4, false, false>(lb, n_sm, s);
        case 17: return pre_batch_c<4, false, true>(lb, n_sm, s);
        case 18: return pre_batch_c<4, true, false>(lb, n_sm, s);
        case 19: return pre_batch_c<4, true, true>(lb, n_sm, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pg
