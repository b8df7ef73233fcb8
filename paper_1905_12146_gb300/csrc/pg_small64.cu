// Nucleotide (m = 4) FP64 latency kernel: the whole tree of a small problem in shared memory.
//
// A problem of a few dozen taxa and a few hundred patterns (the plain FP64 method of Sections
// 2.3-2.5 at the scale of a per-iteration call of an optimiser or sampler) is bound neither by
// memory nor by arithmetic throughput but by the chain of dependent steps: one tree level after
// another, each a few dozen FP64 operations deep, and on this GPU the FP64 pipe takes a warp
// instruction only every few dozen cycles.  This kernel shortens that chain twice over:
//   * every block keeps the per-pattern vectors of its pattern range in shared memory for the
//     whole evaluation (the transition tables, the tip codes, for each non-root internal node c
//     the branch-top vector a_c = P_c p_c of its post-order partial, its pre-order partial, both
//     log2 scales), so a level reads nothing from device memory;
//   * four lanes share one (node, pattern) unit, lane s holding state s, so a level's dependent
//     chain is one row of each 4x4 product; the 4-vectors a row needs are read from shared memory
//     (a_c, the tables) or exchanged with shuffles within the four lanes (p_k, q_k * a_sibling).
// The arithmetic is that of the FP64 tree kernel: post-order p_k = (P_c0 p_c0) * (P_c1 p_c1),
// rescaled by a power of two per (node, pattern); the root's L = sum_l w_l pi . p_root,l; the
// pre-order q_c = P_c^T (q_k * a_sibling); the branch terms r_l w_l (q_k * a_sib) . Q a_c and
// r_l^2 w_l (q_k * a_sib) . Q Q a_c, divided by L (Sections 2.4-2.5).  Per-pattern sums go to one
// slot per (block, branch), written in pattern order, so the result does not depend on timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

constexpr int kSmallThreads = 128;               // four warps: one per SM sub-partition
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kUnitsPerPass = kSmallWarps * 8;   // (node, pattern) units per pass, four lanes each
constexpr int kTab = 2 * kPtab64Pairs;           // doubles per (branch, category) table: P columns, row sums

// Byte offsets of the shared arrays of one block (cnt = patterns per block).
struct Small64Layout {
    size_t ops, top, pre, tab, gq, hq, lq, invL, w, pe, qe, Er, tips, bytes;
};

__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Small64Layout small64_layout(int N, int n, int C, int cnt) {
    Small64Layout L;
    size_t o = 0;
    const size_t nint = (size_t)(N - 1);
    L.ops = o;  o = up16(o + 16 * nint);
    L.top = o;  o = up16(o + 8 * nint * C * cnt * 4);
    L.pre = o;  o = up16(o + 8 * nint * C * cnt * 4);
    L.tab = o;  o = up16(o + 8 * (size_t)n * C * kTab);
    L.gq = o;   o = up16(o + 8 * (size_t)n * cnt);
    L.hq = o;   o = up16(o + 8 * (size_t)n * cnt);
    L.lq = o;   o = up16(o + 8 * (size_t)cnt);
    L.invL = o; o = up16(o + 8 * (size_t)cnt);
    L.w = o;    o = up16(o + 8 * (size_t)cnt);
    L.pe = o;   o = up16(o + 4 * nint * cnt);
    L.qe = o;   o = up16(o + 4 * nint * cnt);
    L.Er = o;   o = up16(o + 4 * (size_t)cnt);
    L.tips = o; o = up16(o + (size_t)N * cnt);
    L.bytes = o;
    return L;
}

// FP64 helpers that keep FP64 instructions off the dependent chain where integer ones do: on this
// GPU each FP64 warp instruction holds an SM sub-partition's FP64 pipe for dozens of cycles.

// x * 2^e: one multiplication by an exact power of two for e in [-1022, 1023] (exact for a normal
// result, one rounding for a subnormal one, as ldexp), ldexp beyond
__device__ __forceinline__ double ldexp2(double x, int e) {
    if (e >= -1022 && e <= 1023) return x * __longlong_as_double((long long)(1023 + e) << 52);
    return ldexp(x, e);
}
// v * 2^-e exactly (e from scale_exp)
__device__ __forceinline__ double unscale(double v, int e) { return ldexp2(v, -e); }

// The maximum of non-negative doubles is the maximum of their bit patterns as signed integers
// (a negative value, which products of these tables can only be through rounding, loses to any
// non-negative one; a NaN wins and then gets scale 0, as the root reports it).
__device__ __forceinline__ long long max_bits(long long a, double v) { return max(a, __double_as_longlong(v)); }
__device__ __forceinline__ long long grp_max(long long b) {   // over the four lanes of a unit
    b = max(b, __shfl_xor_sync(0xffffffffu, b, 1));
    return max(b, __shfl_xor_sync(0xffffffffu, b, 2));
}
// scale_exponent64 of the double with bit pattern b, from its exponent field: mx * 2^-e in [1, 2)
// for a positive normal mx; 0 for zero, negative, infinite or NaN; frexp for a subnormal one
__device__ __forceinline__ int scale_exp(long long b) {
    const int eb = (int)((b >> 52) & 0x7ff);
    if (b <= 0 || eb == 0x7ff) return 0;
    if (eb == 0) return scale_exponent64(__longlong_as_double(b));
    return eb - 1023;
}

__device__ __forceinline__ double grp_sum(double v) {   // over the four lanes of a unit
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    return v + __shfl_xor_sync(0xffffffffu, v, 2);
}

template <int C, bool HESS>
__global__ void __launch_bounds__(kSmallThreads) small64_kernel(const __grid_constant__ BatchArgs<1> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const ProbDesc &d = a.d[0];
    const int N = d.n_tips, n = d.n_nodes, root = d.root;
    const int cm = d.range_len;   // patterns per block: the stride of every per-pattern shared array
    const int tile = (int)blockIdx.x;
    const int p0 = tile * cm;
    const int cnt = min(cm, d.P - p0);
    const Small64Layout Ly = small64_layout(N, n, C, cm);
    int4 *ops = reinterpret_cast<int4 *>(smem + Ly.ops);
    double *top = reinterpret_cast<double *>(smem + Ly.top);    // [N-1][C][cm][4]: a_c = P_c p_c
    double *pre = reinterpret_cast<double *>(smem + Ly.pre);    // [N-1][C][cm][4]: q_c
    double *tab = reinterpret_cast<double *>(smem + Ly.tab);    // [n][C][kTab]: entry (i, j) at 4j + i
    double *gq = reinterpret_cast<double *>(smem + Ly.gq);      // [n][cm]: weighted gradient terms
    double *hq = reinterpret_cast<double *>(smem + Ly.hq);      // [n][cm]: weighted Hessian terms
    double *lq = reinterpret_cast<double *>(smem + Ly.lq);      // [cm]: w_p log L_p
    double *invL = reinterpret_cast<double *>(smem + Ly.invL);  // [cm]: 1 / mantissa of L_p
    double *wq = reinterpret_cast<double *>(smem + Ly.w);       // [cm]: pattern weights
    int *pe = reinterpret_cast<int *>(smem + Ly.pe);            // [N-1][cm]: log2 scale of p_c (and a_c)
    int *qe = reinterpret_cast<int *>(smem + Ly.qe);            // [N-1][cm]: log2 scale of q_c
    int *Er = reinterpret_cast<int *>(smem + Ly.Er);            // [cm]: log2 scale of L_p
    uint8_t *tips = reinterpret_cast<uint8_t *>(smem + Ly.tips);   // [N][cm]: tip codes, 4 = all-ones
    const int tid = (int)threadIdx.x;

    // what does not depend on the transition tables of this evaluation
    for (int i = tid; i < N - 1; i += kSmallThreads) ops[i] = __ldg(d.ops + i);
    for (int i = tid; i < N * cm; i += kSmallThreads) {
        const int t = i / cm, q = i - t * cm;
        tips[i] = (uint8_t)(q < cnt ? min((int)__ldg(d.tips + (size_t)t * d.Ps + p0 + q), 4) : 4);
    }
    for (int i = tid; i < n * cm; i += kSmallThreads) {
        gq[i] = 0.0;
        if (HESS) hq[i] = 0.0;
    }
    for (int q = tid; q < cm; q += kSmallThreads) wq[q] = q < cnt ? __ldg(d.weights + p0 + q) : 0.0;
    pdl_launch_dependents();
    pdl_wait();   // the P build of this evaluation has completed and its tables are visible
    {
        const double *src = reinterpret_cast<const double *>(d.Ptab64);
        for (int i = tid; i < n * C * kTab; i += kSmallThreads) tab[i] = __ldcg(src + i);
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31, s = lane & 3, gb = lane & ~3;
    const int unit = (lane >> 2) * kSmallWarps + warp;   // this lane group's unit within a pass
    constexpr unsigned kAll = 0xffffffffu;

    // post-order, tips to root (Section 2.3); the root gives L_p (Section 2.1)
    for (int lv = 0; lv < d.n_levels; ++lv) {
        const int o0 = __ldg(d.level_off + lv), U = (__ldg(d.level_off + lv + 1) - o0) * cnt;
        for (int base = 0; base < U; base += kUnitsPerPass) {   // the same passes in every thread
            const int j = base + unit;
            const bool active = j < U;
            const int jj = active ? j : U - 1;
            const int u = jj / cnt, q = jj - u * cnt;
            const int4 op = ops[o0 + u];
            const int k = op.x, c0 = op.y, c1 = op.z;
            const bool t0 = c0 < N, t1 = c1 < N;
            double v[C];
            long long mx = 0;   // bit pattern of the largest v
#pragma unroll
            for (int l = 0; l < C; ++l) {
                double A0, A1;   // state s of a_c0 and a_c1
                if (t0) A0 = tab[((size_t)c0 * C + l) * kTab + 4 * tips[c0 * cm + q] + s];
                else A0 = top[((((size_t)(c0 - N) * C + l) * cm + q) << 2) + s];
                if (t1) A1 = tab[((size_t)c1 * C + l) * kTab + 4 * tips[c1 * cm + q] + s];
                else A1 = top[((((size_t)(c1 - N) * C + l) * cm + q) << 2) + s];
                v[l] = A0 * A1;
                mx = max_bits(mx, v[l]);
            }
            const int E = (t0 ? 0 : pe[(c0 - N) * cm + q]) + (t1 ? 0 : pe[(c1 - N) * cm + q]);
            if (k == root) {   // the root is alone on its level: the same branch in every lane
                double r = 0.0;
#pragma unroll
                for (int l = 0; l < C; ++l) r = fma(d.cw[l], v[l], r);
                const double Lp = grp_sum(d.pi[s] * r);
                int e2 = 0;
                const double f = (Lp > 0.0 && isfinite(Lp)) ? frexp(Lp, &e2) : Lp;
                const int Erq = E + e2;
                const double lp = log(f) + (double)Erq * 0.69314718055994530942;
                if (active && s == 0) {
                    invL[q] = 1.0 / f;
                    Er[q] = Erq;
                    if (!(f > 0.0) || !isfinite(lp)) atomicOr(d.status, kStatusNumeric);
                    if (d.out_site) d.out_site[p0 + q] = lp;
                    lq[q] = wq[q] != 0.0 ? wq[q] * lp : 0.0;
                }
                continue;
            }
            const int e = scale_exp(grp_max(mx));
#pragma unroll
            for (int l = 0; l < C; ++l) {
                const double x = unscale(v[l], e);   // state s of p_k
                const double *Pk = tab + ((size_t)k * C + l) * kTab;
                double t = Pk[s] * __shfl_sync(kAll, x, gb);
                t = fma(Pk[4 + s], __shfl_sync(kAll, x, gb + 1), t);
                t = fma(Pk[8 + s], __shfl_sync(kAll, x, gb + 2), t);
                t = fma(Pk[12 + s], __shfl_sync(kAll, x, gb + 3), t);
                if (active) top[((((size_t)(k - N) * C + l) * cm + q) << 2) + s] = t;
            }
            if (active && s == 0) pe[(k - N) * cm + q] = E + e;
        }
        __syncthreads();
    }
    if (tid == 0) {   // this block's share of logL, summed in pattern order
        double sl = 0.0;
        for (int q = 0; q < cnt; ++q) sl += lq[q];
        const int slot0 = tile * d.pieces;
        d.lpart[slot0] = sl;
        for (int pc = 1; pc < d.pieces; ++pc) d.lpart[slot0 + pc] = 0.0;
    }
    if (d.skip & kSkipPre) return;

    // pre-order, root to tips (Section 2.4), with the branch terms of Section 2.5
    for (int lv = d.n_levels - 1; lv >= 0; --lv) {
        const int o0 = __ldg(d.level_off + lv), U = (__ldg(d.level_off + lv + 1) - o0) * cnt;
        for (int base = 0; base < U; base += kUnitsPerPass) {
            const int j = base + unit;
            const bool active = j < U;
            const int jj = active ? j : U - 1;
            const int u = jj / cnt, q = jj - u * cnt;
            const int4 op = ops[o0 + u];
            const int k = op.x, c0 = op.y, c1 = op.z;
            const bool t0 = c0 < N, t1 = c1 < N, rt = (k == root);
            const int Eq = rt ? 0 : qe[(k - N) * cm + q];
            const int E0 = t0 ? 0 : pe[(c0 - N) * cm + q], E1 = t1 ? 0 : pe[(c1 - N) * cm + q];
            double Q0[4], Q1[4];   // row s of each child's generator
            {
                const double *r0 = d.Qd + 16 * (d.bmodel ? __ldg(d.bmodel + c0) : 0) + 4 * s;
                const double *r1 = d.Qd + 16 * (d.bmodel ? __ldg(d.bmodel + c1) : 0) + 4 * s;
#pragma unroll
                for (int i = 0; i < 4; ++i) { Q0[i] = __ldg(r0 + i); Q1[i] = __ldg(r1 + i); }
            }
            double g0 = 0.0, g1 = 0.0, h0 = 0.0, h1 = 0.0;
            long long m0 = 0, m1 = 0;   // bit patterns of the largest q_c0, q_c1 entries
            double x0[C], x1[C];   // state s of q_c0 and q_c1 before rescaling
#pragma unroll
            for (int l = 0; l < C; ++l) {
                const double qk = rt ? d.pi[s] : pre[((((size_t)(k - N) * C + l) * cm + q) << 2) + s];
                const double *T0 = tab + ((size_t)c0 * C + l) * kTab, *T1 = tab + ((size_t)c1 * C + l) * kTab;
                const double *a0, *a1;   // a_c0, a_c1: a column of P (tip) or the branch-top vector
                if (t0) a0 = T0 + 4 * tips[c0 * cm + q];
                else a0 = top + ((((size_t)(c0 - N) * C + l) * cm + q) << 2);
                if (t1) a1 = T1 + 4 * tips[c1 * cm + q];
                else a1 = top + ((((size_t)(c1 - N) * C + l) * cm + q) << 2);
                const double qt0 = qk * a1[s], qt1 = qk * a0[s];   // (q_k * a_sibling), state s
                double u0 = Q0[0] * a0[0], u1 = Q1[0] * a1[0];     // (Q a_c), state s
#pragma unroll
                for (int i = 1; i < 4; ++i) { u0 = fma(Q0[i], a0[i], u0); u1 = fma(Q1[i], a1[i], u1); }
                const double rc = d.rates[l] * d.cw[l];
                g0 = fma(rc, qt0 * u0, g0);
                g1 = fma(rc, qt1 * u1, g1);
                if (HESS) {   // (Q Q a_c), state s, from the four lanes' (Q a_c)
                    double w0 = Q0[0] * __shfl_sync(kAll, u0, gb), w1 = Q1[0] * __shfl_sync(kAll, u1, gb);
#pragma unroll
                    for (int i = 1; i < 4; ++i) {
                        w0 = fma(Q0[i], __shfl_sync(kAll, u0, gb + i), w0);
                        w1 = fma(Q1[i], __shfl_sync(kAll, u1, gb + i), w1);
                    }
                    const double rc2 = d.rates[l] * d.rates[l] * d.cw[l];
                    h0 = fma(rc2, qt0 * w0, h0);
                    h1 = fma(rc2, qt1 * w1, h1);
                }
                // q_c = P_c^T (q_k * a_sibling): column s of P_c against the four lanes' values
                const double *S0 = T0 + 4 * s, *S1 = T1 + 4 * s;
                double y0 = S0[0] * __shfl_sync(kAll, qt0, gb), y1 = S1[0] * __shfl_sync(kAll, qt1, gb);
#pragma unroll
                for (int i = 1; i < 4; ++i) {
                    y0 = fma(S0[i], __shfl_sync(kAll, qt0, gb + i), y0);
                    y1 = fma(S1[i], __shfl_sync(kAll, qt1, gb + i), y1);
                }
                x0[l] = y0;
                x1[l] = y1;
                m0 = max_bits(m0, y0);
                m1 = max_bits(m1, y1);
            }
            g0 = grp_sum(g0);
            g1 = grp_sum(g1);
            if (HESS) {
                h0 = grp_sum(h0);
                h1 = grp_sum(h1);
            }
            const int e0 = scale_exp(grp_max(m0)), e1 = scale_exp(grp_max(m1));
            if (active && !t0) {
#pragma unroll
                for (int l = 0; l < C; ++l) pre[((((size_t)(c0 - N) * C + l) * cm + q) << 2) + s] = unscale(x0[l], e0);
                if (s == 0) qe[(c0 - N) * cm + q] = Eq + E1 + e0;
            }
            if (active && !t1) {
#pragma unroll
                for (int l = 0; l < C; ++l) pre[((((size_t)(c1 - N) * C + l) * cm + q) << 2) + s] = unscale(x1[l], e1);
                if (s == 0) qe[(c1 - N) * cm + q] = Eq + E0 + e1;
            }
            if (active && (s < 2 || HESS)) {   // lanes 0, 1: gradient of c0, c1; lanes 2, 3: Hessian
                const int side = s & 1;
                const int c = side ? c1 : c0;
                const int dE = Eq + E0 + E1 - Er[q];
                const double inv = invL[q], wt = wq[q];
                const double dd = ldexp2(side ? g1 : g0, dE) * inv;
                if (s < 2) gq[c * cm + q] = wt != 0.0 ? wt * dd : 0.0;
                else hq[c * cm + q] = wt != 0.0 ? wt * (ldexp2(side ? h1 : h0, dE) * inv - dd * dd) : 0.0;
            }
        }
        __syncthreads();
    }

    // this block's share of each branch's gradient and Hessian diagonal, summed in pattern order
    const int slot0 = tile * d.pieces;
    for (int i = tid; i < n; i += kSmallThreads) {
        if (i == root) continue;
        double sg = 0.0, sh = 0.0;
        for (int q = 0; q < cnt; ++q) {
            sg += gq[i * cm + q];
            if (HESS) sh += hq[i * cm + q];
        }
        double *gp = d.gpart + (size_t)i * d.slot_cap + slot0;
        gp[0] = sg;
        for (int pc = 1; pc < d.pieces; ++pc) gp[pc] = 0.0;
        if (HESS) {
            double *hp = d.hpart + (size_t)i * d.slot_cap + slot0;
            hp[0] = sh;
            for (int pc = 1; pc < d.pieces; ++pc) hp[pc] = 0.0;
        }
    }
}

template <int C, bool HESS>
cudaError_t launch_small64_c(const BatchArgs<1> &a, cudaStream_t s) {
    const ProbDesc &d = a.d[0];
    const size_t smem = small64_layout(d.n_tips, d.n_nodes, C, d.range_len).bytes;
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) {
            return cudaFuncSetAttribute(small64_kernel<C, HESS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kSmall64MaxSmem);
        });
        e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch: the prologue overlaps the P build
    cfg.gridDim = dim3((unsigned)d.n_tiles);
    cfg.blockDim = dim3(kSmallThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, small64_kernel<C, HESS>, a);
}

template <bool HESS>
cudaError_t launch_small64_h(const BatchArgs<1> &a, cudaStream_t s) {
    switch (a.d[0].C) {
        case 1: return launch_small64_c<1, HESS>(a, s);
        case 2: return launch_small64_c<2, HESS>(a, s);
        case 3: return launch_small64_c<3, HESS>(a, s);
        case 4: return launch_small64_c<4, HESS>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t small64_smem_bytes(const ProbDesc &d) {
    if (d.precision != 1 || d.P <= 0 || d.n_tiles <= 0 || d.range_len <= 0 || d.range_len > kSmall64MaxRange ||
        d.C < 1 || d.C > kMaxCat)
        return 0;
    const size_t b = small64_layout(d.n_tips, d.n_nodes, d.C, d.range_len).bytes;
    return b <= kSmall64MaxSmem ? b : 0;
}

cudaError_t launch_small64(const BatchArgs<1> &a, bool hess, cudaStream_t s) {
    if (a.n != 1 || small64_smem_bytes(a.d[0]) == 0) return cudaErrorInvalidValue;
    return hess ? launch_small64_h<true>(a, s) : launch_small64_h<false>(a, s);
}

}  // namespace pg
