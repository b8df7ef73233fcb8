// Nucleotide (m = 4) kernels: FP64 transition matrices, the fused post-order / root /
// pre-order / gradient pass, and the deterministic per-branch reduction.
//
// Work decomposition.  Site patterns are independent (Section 2.1), so the tree kernel gives each
// thread block a tile of 32*G patterns and lets it walk the WHOLE tree for that tile: the
// post-order pass level by level from the tips (Section 2.3), the root likelihood, then the
// pre-order pass level by level from the root (Section 2.4) with the branch gradient
// (Section 2.5) computed on the way down.  Levels are synchronised with __syncthreads only; no
// block ever waits for another block, so an evaluation is three launches whatever the tree
// height.  Inside a level a warp takes (node, group of 32 patterns) tasks; a lane owns one
// pattern and all C rate categories of it, so the per-pattern power-of-two rescaling needs no
// cross-lane traffic.
//
// FP32 numerics.  Partials are stored in FP32.  Round-to-nearest is unbiased only when the
// discarded bits are uniformly distributed; in the pruning update the bulk of each state's
// value is one large term (the transition matrix is close to I for short branches) to which
// small terms of widely spread magnitudes are added, and those additions lose slightly more
// than they gain.  Over a thousand nodes that bias, not random rounding, dominates the error
// of logL.  Three measures remove it:
//   * P = I + D, so a child's contribution is a = p + S with S = D p small and computed from
//     an FP32 hi/lo split of D; the parent's value (p0 + S0)(p1 + S1) is formed as the exact
//     product p0 p1 (value + FMA residual) plus the small cross terms, and rounded once;
//   * tip children use P's columns as an FP32 hi/lo pair (P applied to a 0/1 vector is a column,
//     or the row sums for the all-ones vector);
//   * every tip vector of pattern p is multiplied by a pattern-specific factor r_p in [1, 2)
//     (the lowbias32 integer hash of p), so exactly representable sub-patterns shared by many
//     sites get different mantissas at different sites.  Each tip contributes r_p once, so L_p
//     carries r_p^N and log L_p loses N log r_p, subtracted in FP64.
// The root's state products are rounded once in FP32 like every node's; the root inner product
// with pi, the mixture over categories, the logarithm and all sums over patterns and tiles are
// FP64.  The pre-order pass feeds only the gradient and uses plain FP32.
//
// FP64 numerics.  Every partial, product and sum in FP64 (no dither, no splitting).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

template <int MAXB>
__device__ __forceinline__ int find_problem(const int (&base)[MAXB + 1], int n, int x) {
    int lo = 0, hi = n;   // base[lo] <= x < base[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (base[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------------------------------
// K1: transition matrices in FP64 (Sections 2.1, 2.5): P = e^{Q b r} by the truncated Taylor
// series of degree 12 with scaling and squaring, ||Q x||_1 <= 1/4 with x = b r / 2^s (truncation
// < 3e-18), and G = Q P.  The matrix coefficients Q^k / k! are computed once per model on upload,
// so each entry of e^{Q x} is a scalar polynomial in x (12 FP64 FMAs) before the squarings.
// ------------------------------------------------------------------------------------------

// Sixteen lanes hold one 4x4 FP64 matrix, lane 4i+j holding entry (i, j); X (the scaled
// generator) is kept whole in every lane, so a product X E needs four shuffles of E per entry.
__device__ __forceinline__ double col_entry(double e, int k, int j, unsigned mask) {   // E[k][j]
    return __shfl_sync(mask, e, k * 4 + j, 16);
}

// entry (i, j) of P = e^{Q b r} in the 16 lanes of one matrix (model row Qr of Q), of G = Q P, and
// the row sums of both; a negative, infinite or NaN branch length is taken as 0 (the caller flags it)
__device__ __forceinline__ void form_pmatrix(const ProbDesc &d, int model, const double (&Qr)[4], double bl, int l,
                                             int lane16, int i, int j, unsigned mask, double &E, double &g, double &rs,
                                             double &gs) {
    if (!(bl >= 0.0) || isinf(bl)) bl = 0.0;
    const double t = bl * d.rates[l];
    double nrm = d.qnorm[model] * fabs(t);
    int sq = 0;
    while (nrm > 0.25 && sq < 1100) { nrm *= 0.5; ++sq; }
    const double x = t * ldexp(1.0, -sq);
    // entry (i, j) of e^{Q x} = sum_k (Q^k / k!)_ij x^k, the Q^k / k! precomputed per model
    const double *Mk = d.Mpow + (size_t)model * (kTaylorDeg + 1) * 16 + lane16;
    E = Mk[kTaylorDeg * 16];
#pragma unroll
    for (int k = kTaylorDeg - 1; k >= 0; --k) E = fma(E, x, Mk[k * 16]);
#pragma unroll 1
    for (int q = 0; q < sq; ++q) {   // squaring: E[i][j] = sum_k E[i][k] E[k][j]
        const double r0 = __shfl_sync(mask, E, i * 4 + 0, 16), r1 = __shfl_sync(mask, E, i * 4 + 1, 16);
        const double r2 = __shfl_sync(mask, E, i * 4 + 2, 16), r3 = __shfl_sync(mask, E, i * 4 + 3, 16);
        double s = r0 * col_entry(E, 0, j, mask);
        s = fma(r1, col_entry(E, 1, j, mask), s);
        s = fma(r2, col_entry(E, 2, j, mask), s);
        E = fma(r3, col_entry(E, 3, j, mask), s);
    }
    // G = Q P (entry (i, j)); row sums of P and of G (P and G applied to the all-ones vector)
    g = Qr[0] * col_entry(E, 0, j, mask);
    g = fma(Qr[1], col_entry(E, 1, j, mask), g);
    g = fma(Qr[2], col_entry(E, 2, j, mask), g);
    g = fma(Qr[3], col_entry(E, 3, j, mask), g);
    rs = E + __shfl_xor_sync(mask, E, 1, 16);
    rs += __shfl_xor_sync(mask, rs, 2, 16);
    gs = g + __shfl_xor_sync(mask, g, 1, 16);
    gs += __shfl_xor_sync(mask, gs, 2, 16);
}

// Launched with programmatic serialisation: the matrices are formed while the previous launch (the
// last evaluation's reduction) drains, and stored only after waiting for it, since until then the
// tables they replace may still be read.  The branch length read before the wait is read again
// after it and the matrix formed again if it changed (an input the previous launch wrote).  Every
// thread waits before it leaves, so this launch completes only after the previous one.
template <int MAXB>
__global__ void __launch_bounds__(128) pmatrix4_kernel(const __grid_constant__ BatchArgs<MAXB> a) {
    pdl_launch_dependents();   // the first level kernel may be scheduled now; it waits for these tables
    const int gid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int mat = gid >> 4, lane16 = gid & 15, i = lane16 >> 2, j = lane16 & 3;
    const int total = a.mat_base[a.n];
    // whole 16-lane groups stay together; groups past the end leave together
    if (mat >= total) {
        pdl_wait();
        return;
    }
    const unsigned mask = 0xFFFFu << (threadIdx.x & 16);
    const int pid = find_problem<MAXB>(a.mat_base, a.n, mat);
    const ProbDesc &d = a.d[pid];
    const int item = mat - a.mat_base[pid];
    const int br = item / d.C, l = item - br * d.C;
    if (br == d.root) {   // uniform within the group
        pdl_wait();
        return;
    }
    const int model = d.bmodel ? d.bmodel[br] : 0;
    const double *Qm = d.Qd + model * 16;
    double Qr[4];   // row i of Q
#pragma unroll
    for (int k = 0; k < 4; ++k) Qr[k] = Qm[i * 4 + k];
    const double b0 = d.b[br];
    double E, g, rs, gs;
    form_pmatrix(d, model, Qr, b0, l, lane16, i, j, mask, E, g, rs, gs);
    pdl_wait();
    const double bl = __ldcg(d.b + br);   // (the same for the group's 16 lanes)
    if (__double_as_longlong(bl) != __double_as_longlong(b0)) form_pmatrix(d, model, Qr, bl, l, lane16, i, j, mask, E, g, rs, gs);
    if (!(bl >= 0.0) || isinf(bl)) {
        if (lane16 == 0) atomicOr(d.status, kStatusBadLength);
    }
    const double id = (i == j) ? 1.0 : 0.0;
    if (d.precision == 1) {   // FP64 table: column c as two double2 = P[0..3][c]
        double *out = reinterpret_cast<double *>(d.Ptab64 + ((size_t)br * d.C + l) * kPtab64Pairs);
        out[j * 4 + i] = E;
        if (j == 0) out[16 + i] = rs;
        return;
    }
    float *out = reinterpret_cast<float *>(d.Ptab + ((size_t)br * d.C + l) * kPtabCols);
    const float hi = (float)E, lo = (float)(E - (double)hi);
    const double dd = E - id;
    const float dhi = (float)dd, dlo = (float)(dd - (double)dhi);
    out[j * 4 + i] = hi;
    out[(kColPlo + j) * 4 + i] = lo;
    out[(kColG + j) * 4 + i] = (float)g;
    out[(kColDhi + j) * 4 + i] = dhi;
    out[(kColDlo + j) * 4 + i] = dlo;
    if (j == 0) {
        const float rhi = (float)rs;
        out[4 * 4 + i] = rhi;
        out[(kColPlo + 4) * 4 + i] = (float)(rs - (double)rhi);
        out[(kColG + 4) * 4 + i] = (float)gs;
    }
}

// ------------------------------------------------------------------------------------------
// K2-K4: the tree pass for one contiguous range of patterns per thread block
// ------------------------------------------------------------------------------------------
//
// A block owns patterns [p0, p0 + cnt).  At a level with nd nodes its work is the nd * cnt
// (node, pattern) pairs, pattern-fastest; warps take 32 consecutive pairs at a time, so lanes stay
// busy for any range length and a warp may straddle node boundaries.  Sums over patterns (logL,
// branch gradients) are reduced per node segment of the warp and written to a fixed slot
// (block, piece), piece = the warp's 32-pair chunk counted from the node's first chunk; the
// reduction kernel adds the slots of a branch in a fixed order.

// ---- FP64 partials ------------------------------------------------------------------------

struct D4 {
    double v[4];
};

__device__ __forceinline__ D4 ld_d4(const double2 *base, size_t idx) {
    const double2 a = base[2 * idx], b = base[2 * idx + 1];
    return D4{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ void st_d4(double2 *base, size_t idx, const D4 &x) {
    base[2 * idx] = make_double2(x.v[0], x.v[1]);
    base[2 * idx + 1] = make_double2(x.v[2], x.v[3]);
}
// column c of a P64 table: P[0..3][c]
__device__ __forceinline__ D4 col64(const double2 *P, int c) {
    const double2 a = __ldg(P + 2 * c), b = __ldg(P + 2 * c + 1);
    return D4{{a.x, a.y, b.x, b.y}};
}
__device__ __forceinline__ D4 matvec64(const double2 *P, const D4 &x) {
    D4 a{{0, 0, 0, 0}};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const D4 col = col64(P, c);
#pragma unroll
        for (int s = 0; s < 4; ++s) a.v[s] = fma(col.v[s], x.v[c], a.v[s]);
    }
    return a;
}
__device__ __forceinline__ D4 matvec64_t(const double2 *P, const D4 &x) {
    D4 a;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const D4 col = col64(P, c);
        a.v[c] = fma(col.v[3], x.v[3], fma(col.v[2], x.v[2], fma(col.v[1], x.v[1], col.v[0] * x.v[0])));
    }
    return a;
}
__device__ __forceinline__ D4 matvecQ64(const double *Q, const D4 &x) {   // row-major Q
    D4 a;
#pragma unroll
    for (int s = 0; s < 4; ++s)
        a.v[s] = fma(Q[s * 4 + 3], x.v[3], fma(Q[s * 4 + 2], x.v[2], fma(Q[s * 4 + 1], x.v[1], Q[s * 4] * x.v[0])));
    return a;
}
__device__ __forceinline__ double dot64(const D4 &a, const D4 &b) {
    return fma(a.v[3], b.v[3], fma(a.v[2], b.v[2], fma(a.v[1], b.v[1], a.v[0] * b.v[0])));
}

template <int C>
__device__ __forceinline__ void post_pair64(const ProbDesc &d, const int4 op, const int p, const bool active,
                                           double &L, int &E) {
    const int N = d.n_tips, Pn = d.Ps;
    const int k = op.x, c0 = op.y, c1 = op.z;
    const bool t0 = c0 < N, t1 = c1 < N;
    const bool root = (k == d.root);
    const double2 *post = static_cast<const double2 *>(d.post);
    int y0 = 0, y1 = 0;
    E = 0;
    if (t0) y0 = min((int)d.tips[(size_t)c0 * Pn + p], 4); else E += d.pe[(size_t)(c0 - N) * Pn + p];
    if (t1) y1 = min((int)d.tips[(size_t)c1 * Pn + p], 4); else E += d.pe[(size_t)(c1 - N) * Pn + p];
    D4 v[C];
    double mx = 0.0;
    L = 0.0;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        const double2 *P0 = d.Ptab64 + ((size_t)c0 * C + l) * kPtab64Pairs;
        const double2 *P1 = d.Ptab64 + ((size_t)c1 * C + l) * kPtab64Pairs;
        const D4 a0 = t0 ? col64(P0, y0) : matvec64(P0, ld_d4(post, ((size_t)(c0 - N) * C + l) * Pn + p));
        const D4 a1 = t1 ? col64(P1, y1) : matvec64(P1, ld_d4(post, ((size_t)(c1 - N) * C + l) * Pn + p));
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            v[l].v[s] = a0.v[s] * a1.v[s];
            mx = fmax(mx, v[l].v[s]);
        }
        if (root) {
            double s = 0.0;
#pragma unroll
            for (int t = 0; t < 4; ++t) s = fma(d.pi[t], v[l].v[t], s);
            L = fma(d.cw[l], s, L);
        }
    }
    if (root || !active) return;
    const int e = scale_exponent64(mx);
    double2 *out = static_cast<double2 *>(d.post);
#pragma unroll
    for (int l = 0; l < C; ++l) {
        D4 w;
#pragma unroll
        for (int s = 0; s < 4; ++s) w.v[s] = ldexp(v[l].v[s], -e);
        st_d4(out, ((size_t)(k - N) * C + l) * Pn + p, w);
    }
    d.pe[(size_t)(k - N) * Pn + p] = E + e;
}

template <int C, bool HESS>
__device__ __forceinline__ void pre_pair64(const ProbDesc &d, const int4 op, const int p, const bool active,
                                          double (&g)[2], double (&h)[2], int &dEsum) {
    const int N = d.n_tips, Pn = d.Ps;
    const int k = op.x, c0 = op.y, c1 = op.z;
    const bool t0 = c0 < N, t1 = c1 < N;
    const bool root = (k == d.root);
    const double2 *post = static_cast<const double2 *>(d.post);
    double2 *pre = static_cast<double2 *>(d.pre);
    const int Eq = root ? 0 : d.qe[(size_t)(k - N) * Pn + p];
    int E0 = 0, E1 = 0, y0 = 0, y1 = 0;
    if (t0) y0 = min((int)d.tips[(size_t)c0 * Pn + p], 4); else E0 = d.pe[(size_t)(c0 - N) * Pn + p];
    if (t1) y1 = min((int)d.tips[(size_t)c1 * Pn + p], 4); else E1 = d.pe[(size_t)(c1 - N) * Pn + p];
    const double *Q0 = d.Qd + 16 * (d.bmodel ? d.bmodel[c0] : 0);
    const double *Q1 = d.Qd + 16 * (d.bmodel ? d.bmodel[c1] : 0);
    double m0 = 0, m1 = 0;
    g[0] = g[1] = h[0] = h[1] = 0.0;
    D4 q0[C], q1[C];
#pragma unroll
    for (int l = 0; l < C; ++l) {
        const D4 qk = root ? D4{{d.pi[0], d.pi[1], d.pi[2], d.pi[3]}}
                           : ld_d4(pre, ((size_t)(k - N) * C + l) * Pn + p);
        const double2 *P0 = d.Ptab64 + ((size_t)c0 * C + l) * kPtab64Pairs;
        const double2 *P1 = d.Ptab64 + ((size_t)c1 * C + l) * kPtab64Pairs;
        const D4 a0 = t0 ? col64(P0, y0) : matvec64(P0, ld_d4(post, ((size_t)(c0 - N) * C + l) * Pn + p));
        const D4 a1 = t1 ? col64(P1, y1) : matvec64(P1, ld_d4(post, ((size_t)(c1 - N) * C + l) * Pn + p));
        D4 qt0, qt1;
#pragma unroll
        for (int s = 0; s < 4; ++s) { qt0.v[s] = qk.v[s] * a1.v[s]; qt1.v[s] = qk.v[s] * a0.v[s]; }
        const D4 u0 = matvecQ64(Q0, a0), u1 = matvecQ64(Q1, a1);
        g[0] = fma(d.rates[l] * d.cw[l], dot64(qt0, u0), g[0]);
        g[1] = fma(d.rates[l] * d.cw[l], dot64(qt1, u1), g[1]);
        if (HESS) {
            h[0] = fma(d.rates[l] * d.rates[l] * d.cw[l], dot64(qt0, matvecQ64(Q0, u0)), h[0]);
            h[1] = fma(d.rates[l] * d.rates[l] * d.cw[l], dot64(qt1, matvecQ64(Q1, u1)), h[1]);
        }
        if (!t0) {
            q0[l] = matvec64_t(P0, qt0);
#pragma unroll
            for (int s = 0; s < 4; ++s) m0 = fmax(m0, q0[l].v[s]);
        }
        if (!t1) {
            q1[l] = matvec64_t(P1, qt1);
#pragma unroll
            for (int s = 0; s < 4; ++s) m1 = fmax(m1, q1[l].v[s]);
        }
    }
    if (!t0 && active) {
        const int e = scale_exponent64(m0);
#pragma unroll
        for (int l = 0; l < C; ++l) {
            D4 w;
#pragma unroll
            for (int s = 0; s < 4; ++s) w.v[s] = ldexp(q0[l].v[s], -e);
            st_d4(pre, ((size_t)(c0 - N) * C + l) * Pn + p, w);
        }
        d.qe[(size_t)(c0 - N) * Pn + p] = Eq + E1 + e;
    }
    if (!t1 && active) {
        const int e = scale_exponent64(m1);
#pragma unroll
        for (int l = 0; l < C; ++l) {
            D4 w;
#pragma unroll
            for (int s = 0; s < 4; ++s) w.v[s] = ldexp(q1[l].v[s], -e);
            st_d4(pre, ((size_t)(c1 - N) * C + l) * Pn + p, w);
        }
        d.qe[(size_t)(c1 - N) * Pn + p] = Eq + E0 + e;
    }
    dEsum = Eq + E0 + E1;
}

// ---- FP32 kernel: per-warp double-buffered cp.async prefetch of the partials ------------------
//
// A warp's next 32 pairs are independent of the pairs it is computing (same level), so their
// partial vectors are copied global -> shared (cp.async, 16 B per copy, L2 only) while the current
// ones are processed.  Shared memory, not registers, holds the bytes in flight.

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// where a lane's pair lives and its small inputs (loaded into registers at prefetch time)
struct PairMeta {
    int4 op;
    int u, q, p;
    int e0, e1, eq;   // log2 scales of the children's post partials and of q_k
    int y0, y1;       // tip codes of tip children
    bool active;
};

// items per lane in a stage: post needs both children (2C float4), pre also q_k (3C)
template <int C>
__host__ __device__ constexpr int stage_items() { return 3 * C; }

template <int C>
__host__ __device__ constexpr size_t f32_stage_bytes(int warps) {
    return (size_t)warps * 2 * stage_items<C>() * 32 * sizeof(float4);
}

template <int C, bool PRE>
__device__ __forceinline__ void prefetch_pair(const ProbDesc &d, int o0, int cnt, int p0, int npairs, int chunk,
                                              float4 *slot, PairMeta &m) {
    const int lane = threadIdx.x & 31;
    const int N = d.n_tips, Pn = d.Ps;
    const int j = chunk * 32 + lane;
    m.active = j < npairs;
    const int jj = m.active ? j : npairs - 1;
    m.u = jj / cnt;
    m.q = jj - m.u * cnt;
    m.p = p0 + m.q;
    m.op = __ldg(d.ops + o0 + m.u);
    const float4 *post = static_cast<const float4 *>(d.post);
    const int c0 = m.op.y, c1 = m.op.z, k = m.op.x;
    m.e0 = m.e1 = m.eq = m.y0 = m.y1 = 0;
    if (c0 < N) m.y0 = min((int)__ldg(d.tips + (size_t)c0 * Pn + m.p), 4);
    else {
        m.e0 = __ldcg(d.pe + (size_t)(c0 - N) * Pn + m.p);
#pragma unroll
        for (int l = 0; l < C; ++l) cp_async16(slot + l * 32, post + ((size_t)(c0 - N) * C + l) * Pn + m.p);
    }
    if (c1 < N) m.y1 = min((int)__ldg(d.tips + (size_t)c1 * Pn + m.p), 4);
    else {
        m.e1 = __ldcg(d.pe + (size_t)(c1 - N) * Pn + m.p);
#pragma unroll
        for (int l = 0; l < C; ++l) cp_async16(slot + (C + l) * 32, post + ((size_t)(c1 - N) * C + l) * Pn + m.p);
    }
    if (PRE && k != d.root) {
        const float4 *pre = static_cast<const float4 *>(d.pre);
        m.eq = __ldcg(d.qe + (size_t)(k - N) * Pn + m.p);
#pragma unroll
        for (int l = 0; l < C; ++l) cp_async16(slot + (2 * C + l) * 32, pre + ((size_t)(k - N) * C + l) * Pn + m.p);
    }
}

// Post-order update of internal node m.op.x for pattern m.p (Section 2.3); at the root returns
// the site likelihood L (Section 2.3 root inner product with the Section 2.5 mixture) and its
// log2 scale E instead of storing a partial.
template <int C>
__device__ __forceinline__ void post_compute32(const ProbDesc &d, const PairMeta &m, const float4 *slot,
                                               double &L, int &E) {
    const int N = d.n_tips, Pn = d.Ps;
    const int k = m.op.x, c0 = m.op.y, c1 = m.op.z;
    const bool t0 = c0 < N, t1 = c1 < N;
    const bool root = (k == d.root);
    const float r = pattern_factor((uint32_t)m.p);
    E = m.e0 + m.e1;
    float4 v[C];
    float mx = 0.0f;
    L = 0.0;
#pragma unroll
    for (int l = 0; l < C; ++l) {
        const float4 *P0 = d.Ptab + ((size_t)c0 * C + l) * kPtabCols;
        const float4 *P1 = d.Ptab + ((size_t)c1 * C + l) * kPtabCols;
        float4 x0, x1, s0 = f4(0.f, 0.f, 0.f, 0.f), s1 = f4(0.f, 0.f, 0.f, 0.f);
        if (t0) {
            const float4 hi = __ldg(P0 + m.y0), lo = __ldg(P0 + kColPlo + m.y0);
            x0 = f4(fmaf(hi.x, r, lo.x * r), fmaf(hi.y, r, lo.y * r), fmaf(hi.z, r, lo.z * r), fmaf(hi.w, r, lo.w * r));
        } else {
            x0 = slot[l * 32];
            s0 = matvec_hilo(P0 + kColDhi, P0 + kColDlo, x0);
        }
        if (t1) {
            const float4 hi = __ldg(P1 + m.y1), lo = __ldg(P1 + kColPlo + m.y1);
            x1 = f4(fmaf(hi.x, r, lo.x * r), fmaf(hi.y, r, lo.y * r), fmaf(hi.z, r, lo.z * r), fmaf(hi.w, r, lo.w * r));
        } else {
            x1 = slot[(C + l) * 32];
            s1 = matvec_hilo(P1 + kColDhi, P1 + kColDlo, x1);
        }
        v[l] = f4(prod_split(x0.x, s0.x, x1.x, s1.x), prod_split(x0.y, s0.y, x1.y, s1.y),
                  prod_split(x0.z, s0.z, x1.z, s1.z), prod_split(x0.w, s0.w, x1.w, s1.w));
        if (root) {   // the root's products rounded once in FP32, as every node's; their sums in FP64
            double s = d.pi[0] * (double)v[l].x;
            s = fma(d.pi[1], (double)v[l].y, s);
            s = fma(d.pi[2], (double)v[l].z, s);
            s = fma(d.pi[3], (double)v[l].w, s);
            L = fma(d.cw[l], s, L);
        } else {
            mx = fmaxf(mx, hmax(v[l]));
        }
    }
    if (root || !m.active) return;
    const int e = scale_exponent(mx);
    float4 *out = static_cast<float4 *>(d.post);
#pragma unroll
    for (int l = 0; l < C; ++l) __stcg(out + ((size_t)(k - N) * C + l) * Pn + m.p, scale4(v[l], e));
    __stcg(d.pe + (size_t)(k - N) * Pn + m.p, E + e);
}

// Pre-order step at internal node k for pattern p (Section 2.4): the top-of-branch vectors
// qt_c = q_k o (P_s p_s) of both children, their gradient terms (Section 2.5) and Hessian terms
// (Section 2.6), and q_c = P_c' qt_c stored for internal children.  The terms are relative to
// 2^{Eq + E0 + E1} (returned in dEsum).
template <int C, bool HESS>
__device__ __forceinline__ void pre_compute32(const ProbDesc &d, const PairMeta &m, const float4 *slot,
                                              float (&g)[2], float (&h)[2], int &dEsum) {
    const int N = d.n_tips, Pn = d.Ps;
    const int k = m.op.x, c0 = m.op.y, c1 = m.op.z;
    const bool t0 = c0 < N, t1 = c1 < N;
    const bool root = (k == d.root);
    const float r = pattern_factor((uint32_t)m.p);
    float4 *pre = static_cast<float4 *>(d.pre);
    float4 a0[C], a1[C];
#pragma unroll
    for (int l = 0; l < C; ++l) {
        const float4 *P0 = d.Ptab + ((size_t)c0 * C + l) * kPtabCols;
        const float4 *P1 = d.Ptab + ((size_t)c1 * C + l) * kPtabCols;
        if (t0) a0[l] = scal(__ldg(P0 + m.y0), r);
        else { float4 H[4]; load_cols(P0, H); a0[l] = matvec(H, slot[l * 32]); }
        if (t1) a1[l] = scal(__ldg(P1 + m.y1), r);
        else { float4 H[4]; load_cols(P1, H); a1[l] = matvec(H, slot[(C + l) * 32]); }
    }
    g[0] = g[1] = h[0] = h[1] = 0.f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int c = side ? c1 : c0;
        const bool tip = side ? t1 : t0;
        float4 Qc[4];
        load_cols(d.Qf + 4 * (d.bmodel ? d.bmodel[c] : 0), Qc);
        float4 q[C];
        float mq = 0.f, gs = 0.f, hs = 0.f;
#pragma unroll
        for (int l = 0; l < C; ++l) {
            const float4 qk = root ? f4(d.pif[0], d.pif[1], d.pif[2], d.pif[3]) : slot[(2 * C + l) * 32];
            const float4 qt = mul(qk, side ? a0[l] : a1[l]);   // top of branch c
            const float4 u = matvec(Qc, side ? a1[l] : a0[l]);
            gs = fmaf(d.gw[l], dot(qt, u), gs);
            if (HESS) hs = fmaf(d.gw2[l], dot(qt, matvec(Qc, u)), hs);
            if (!tip) {
                float4 H[4];
                load_cols(d.Ptab + ((size_t)c * C + l) * kPtabCols, H);
                q[l] = matvec_t(H, qt);
                mq = fmaxf(mq, hmax(q[l]));
            }
        }
        g[side] = gs;
        h[side] = hs;
        if (!tip && m.active) {
            const int e = scale_exponent(mq);
#pragma unroll
            for (int l = 0; l < C; ++l) __stcg(pre + ((size_t)(c - N) * C + l) * Pn + m.p, scale4(q[l], e));
            __stcg(d.qe + (size_t)(c - N) * Pn + m.p, m.eq + (side ? m.e0 : m.e1) + e);
        }
    }
    dEsum = m.eq + m.e0 + m.e1;
}

// per-pattern values of the block's range, after the stage buffers in dynamic shared memory
struct RangeArrays {
    float *invL;   // 1 / Lhat_p  (Lhat in [0.5, 1))
    int *Eroot;    // log2 scale of L_p (with the r_p^N factor inside)
    float *w;      // pattern weight
};

template <int C>
__device__ __forceinline__ void post_level_chunk(const ProbDesc &d, const PairMeta &m, const float4 *slot,
                                                 int chunk, int cnt, int pieces, int slot0, RangeArrays &ra) {
    double L;
    int E;
    post_compute32<C>(d, m, slot, L, E);
    if (m.op.x != d.root) return;   // uniform: the root is alone on its level
    int e2 = 0;
    const double f = split_exponent(L, e2);   // (integer instructions: FP64 bounds this level)
    const int Er = E + e2;
    const double wgt = d.weights[m.p];
    const double lp = log(f) + (double)Er * 0.69314718055994530942 -
                      (d.rlog ? __ldg(d.rlog + m.p) : (double)d.n_tips * log((double)pattern_factor((uint32_t)m.p)));
    const float rf = __frcp_rn((float)f);   // 1 / Lhat_p for the FP32 branch terms
    if (m.active) {
        ra.invL[m.q] = rf;
        ra.Eroot[m.q] = Er;
        ra.w[m.q] = (float)wgt;
        d.site_invL[m.p] = rf;
        d.site_Er[m.p] = Er;
        if (!(f > 0.0) || !isfinite(lp)) atomicOr(d.status, kStatusNumeric);
        if (d.out_site) d.out_site[m.p] = lp;
    }
    segment_sums(m.u, m.active, (m.active && wgt != 0.0) ? wgt * lp : 0.0, chunk, cnt, pieces,
                 [&](int, int pc, double s) { d.lpart[slot0 + pc] = s; });
}

template <int C, bool HESS>
__device__ __forceinline__ void pre_level_chunk(const ProbDesc &d, const PairMeta &m, const float4 *slot,
                                                int o0, int chunk, int cnt, int pieces, int slot0,
                                                const RangeArrays &ra) {
    float g[2], h[2];
    int dEsum;
    pre_compute32<C, HESS>(d, m, slot, g, h, dEsum);
    const double wt = m.active ? (double)ra.w[m.q] : 0.0;
    const int dE = dEsum - ra.Eroot[m.q];
    const float inv = ra.invL[m.q];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const float dd = ldexp2f(g[s], dE) * inv;
        const double dg = wt != 0.0 ? wt * (double)dd : 0.0;
        segment_sums(m.u, m.active, dg, chunk, cnt, pieces, [&](int us, int pc, double v) {
            const int4 o = __ldg(d.ops + o0 + us);
            d.gpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
        });
        if (HESS) {
            const double dh = wt != 0.0 ? wt * (double)(ldexp2f(h[s], dE) * inv - dd * dd) : 0.0;
            segment_sums(m.u, m.active, dh, chunk, cnt, pieces, [&](int us, int pc, double v) {
                const int4 o = __ldg(d.ops + o0 + us);
                d.hpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
            });
        }
    }
}

template <int C, bool HESS, int MAXB>
__global__ void __launch_bounds__(kBlock, 2) tree4f_kernel(const __grid_constant__ BatchArgs<MAXB> a) {
    extern __shared__ float4 dyn[];
    const int pid = (MAXB == 1) ? 0 : find_problem<MAXB>(a.tile_base, a.n, (int)blockIdx.x);
    const ProbDesc &d = a.d[pid];
    const int tile = (int)blockIdx.x - a.tile_base[pid];
    const int p0 = tile * d.range_len;
    const int cnt = min(d.range_len, d.P - p0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const int pieces = d.pieces;
    const int slot0 = tile * pieces;
    constexpr int IT = stage_items<C>();
    float4 *st0 = dyn + (size_t)(warp * 2) * IT * 32 + lane;
    float4 *st1 = st0 + IT * 32;
    RangeArrays ra;
    {
        char *tail = reinterpret_cast<char *>(dyn + (size_t)W * 2 * IT * 32);
        ra.invL = reinterpret_cast<float *>(tail);
        ra.Eroot = reinterpret_cast<int *>(tail + sizeof(float) * d.range_len);
        ra.w = reinterpret_cast<float *>(tail + 2 * sizeof(float) * d.range_len);
    }
    PairMeta m0, m1;

    // post-order, tips to root (Section 2.3); levels below d.cut were done by the level kernels
    for (int lv = (d.skip & kSkipPost) ? d.n_levels : d.cut; lv < d.n_levels; ++lv) {
        const int o0 = d.level_off[lv], npairs = (d.level_off[lv + 1] - o0) * cnt;
        int chunk = warp;
        if (chunk * 32 < npairs) prefetch_pair<C, false>(d, o0, cnt, p0, npairs, chunk, st0, m0);
        cp_async_commit();
        while (chunk * 32 < npairs) {
            int next = chunk + W;
            if (next * 32 < npairs) prefetch_pair<C, false>(d, o0, cnt, p0, npairs, next, st1, m1);
            cp_async_commit();
            cp_async_wait1();
            __syncwarp();
            post_level_chunk<C>(d, m0, st0, chunk, cnt, pieces, slot0, ra);
            chunk = next;
            if (chunk * 32 >= npairs) break;
            next = chunk + W;
            if (next * 32 < npairs) prefetch_pair<C, false>(d, o0, cnt, p0, npairs, next, st0, m0);
            cp_async_commit();
            cp_async_wait1();
            __syncwarp();
            post_level_chunk<C>(d, m1, st1, chunk, cnt, pieces, slot0, ra);
            chunk = next;
        }
        cp_async_wait0();
        __syncthreads();
    }
    if (d.skip & kSkipPre) return;
    if (d.skip & kSkipPost) {   // the root's per-pattern values from the earlier post-order launch
        for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
            ra.invL[q] = __ldcg(d.site_invL + p0 + q);
            ra.Eroot[q] = __ldcg(d.site_Er + p0 + q);
            ra.w[q] = (float)d.weights[p0 + q];
        }
        __syncthreads();
    }
    // pre-order, root to tips (Section 2.4) with the gradient (Section 2.5), down to d.cut
    for (int lv = d.n_levels - 1; lv >= d.cut; --lv) {
        const int o0 = d.level_off[lv], npairs = (d.level_off[lv + 1] - o0) * cnt;
        int chunk = warp;
        if (chunk * 32 < npairs) prefetch_pair<C, true>(d, o0, cnt, p0, npairs, chunk, st0, m0);
        cp_async_commit();
        while (chunk * 32 < npairs) {
            int next = chunk + W;
            if (next * 32 < npairs) prefetch_pair<C, true>(d, o0, cnt, p0, npairs, next, st1, m1);
            cp_async_commit();
            cp_async_wait1();
            __syncwarp();
            pre_level_chunk<C, HESS>(d, m0, st0, o0, chunk, cnt, pieces, slot0, ra);
            chunk = next;
            if (chunk * 32 >= npairs) break;
            next = chunk + W;
            if (next * 32 < npairs) prefetch_pair<C, true>(d, o0, cnt, p0, npairs, next, st0, m0);
            cp_async_commit();
            cp_async_wait1();
            __syncwarp();
            pre_level_chunk<C, HESS>(d, m1, st1, o0, chunk, cnt, pieces, slot0, ra);
            chunk = next;
        }
        cp_async_wait0();
        __syncthreads();
    }
}

// ---- FP64 kernel: direct loads ------------------------------------------------------------

struct TileShared64 {
    int Eroot[kMaxRange];
    double w[kMaxRange];
    double invL64[kMaxRange];
};

template <int C, bool HESS, int MAXB>
__global__ void __launch_bounds__(kBlock, 1) tree4d_kernel(const __grid_constant__ BatchArgs<MAXB> a) {
    __shared__ TileShared64 sh;
    const int pid = (MAXB == 1) ? 0 : find_problem<MAXB>(a.tile_base, a.n, (int)blockIdx.x);
    const ProbDesc &d = a.d[pid];
    const int tile = (int)blockIdx.x - a.tile_base[pid];
    const int p0 = tile * d.range_len;
    const int cnt = min(d.range_len, d.P - p0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int W = blockDim.x >> 5;
    const int pieces = d.pieces;
    const int slot0 = tile * pieces;

    for (int lv = 0; lv < d.n_levels; ++lv) {
        const int o0 = d.level_off[lv], nd = d.level_off[lv + 1] - o0;
        const int npairs = nd * cnt;
        for (int chunk = warp; chunk * 32 < npairs; chunk += W) {
            const int j = chunk * 32 + lane;
            const bool active = j < npairs;
            const int jj = active ? j : npairs - 1;
            const int u = jj / cnt, q = jj - u * cnt;
            const int p = p0 + q;
            const int4 op = __ldg(d.ops + o0 + u);
            double L;
            int E;
            post_pair64<C>(d, op, p, active, L, E);
            if (op.x != d.root) continue;   // uniform: the root is alone on its level
            int e2 = 0;
            const double f = (L > 0.0 && isfinite(L)) ? frexp(L, &e2) : L;
            const int Er = E + e2;
            const double wgt = d.weights[p];
            const double lp = log(f) + (double)Er * 0.69314718055994530942;
            if (active) {
                sh.invL64[q] = 1.0 / f;
                sh.Eroot[q] = Er;
                sh.w[q] = wgt;
                if (!(f > 0.0) || !isfinite(lp)) atomicOr(d.status, kStatusNumeric);
                if (d.out_site) d.out_site[p] = lp;
            }
            segment_sums(u, active, (active && wgt != 0.0) ? wgt * lp : 0.0, chunk, cnt, pieces,
                         [&](int, int pc, double s) { d.lpart[slot0 + pc] = s; });
        }
        __syncthreads();
    }
    if (d.skip & kSkipPre) return;   // (the FP64 kernel always recomputes the post-order)
    for (int lv = d.n_levels - 1; lv >= 0; --lv) {
        const int o0 = d.level_off[lv], nd = d.level_off[lv + 1] - o0;
        const int npairs = nd * cnt;
        for (int chunk = warp; chunk * 32 < npairs; chunk += W) {
            const int j = chunk * 32 + lane;
            const bool active = j < npairs;
            const int jj = active ? j : npairs - 1;
            const int u = jj / cnt, q = jj - u * cnt;
            const int p = p0 + q;
            const int4 op = __ldg(d.ops + o0 + u);
            int dEsum;
            double g[2], h[2];
            pre_pair64<C, HESS>(d, op, p, active, g, h, dEsum);
            const double wt = active ? sh.w[q] : 0.0;
            const int dE = dEsum - sh.Eroot[q];
            const double inv = sh.invL64[q];
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const double dd = ldexp(g[s], dE) * inv;
                const double dg = wt != 0.0 ? wt * dd : 0.0;
                segment_sums(u, active, dg, chunk, cnt, pieces, [&](int us, int pc, double v) {
                    const int4 o = __ldg(d.ops + o0 + us);
                    d.gpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
                });
                if (HESS) {
                    const double dh = wt != 0.0 ? wt * (ldexp(h[s], dE) * inv - dd * dd) : 0.0;
                    segment_sums(u, active, dh, chunk, cnt, pieces, [&](int us, int pc, double v) {
                        const int4 o = __ldg(d.ops + o0 + us);
                        d.hpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
                    });
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// K5: fixed-order reduction over tile groups: one warp per branch (grad, hess), one per logL
// ------------------------------------------------------------------------------------------

// sum of v[lane], v[lane + 32], ... below ns in a fixed order: four accumulators, each pass of the
// loop issuing its (up to) four loads independently, so a short row is one round trip
__device__ __forceinline__ double lane_sum(const double *v, int ns, int lane) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll 2
    for (int j = lane; j < ns; j += 128) {
        const double x0 = v[j];
        const double x1 = j + 32 < ns ? v[j + 32] : 0.0;
        const double x2 = j + 64 < ns ? v[j + 64] : 0.0;
        const double x3 = j + 96 < ns ? v[j + 96] : 0.0;
        a0 += x0;
        a1 += x1;
        a2 += x2;
        a3 += x3;
    }
    return (a0 + a1) + (a2 + a3);
}

// one warp per (problem, branch) and one per problem's logL: blockIdx.y is the problem, so a block's
// descriptor is uniform and no warp searches for its problem
template <int MAXB>
__global__ void __launch_bounds__(256) reduce_kernel(const __grid_constant__ BatchArgs<MAXB> a, int want_hess) {
    // The next evaluation's transition-matrix launch may start now: it forms its matrices and waits
    // for this launch before it stores them.
    pdl_launch_dependents();
    pdl_wait();   // launched while the last pass drains: its slot sums are complete and visible after this
    const ProbDesc &d = a.d[blockIdx.y];
    const int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (item > d.n_nodes) return;
    if (item == d.n_nodes) {
        const double s = warp_sum(lane_sum(d.lpart, d.n_tg, lane));
        if (lane == 0 && d.out_logL) *d.out_logL = s;
        return;
    }
    double g = 0.0, h = 0.0;
    if (item != d.root) {
        // branches below the cut were reduced per level-kernel block, the others per fused slot
        const int ns = (d.cut > 0 && d.plevel[item] < d.cut) ? d.level_ranges * (kLevelRange / 32) : d.n_tg;
        g = warp_sum(lane_sum(d.gpart + (size_t)item * d.slot_cap, ns, lane));
        if (want_hess) h = warp_sum(lane_sum(d.hpart + (size_t)item * d.slot_cap, ns, lane));
    }
    if (lane == 0) {
        if (d.gscale) g *= *d.gscale;
        if (d.out_grad) d.out_grad[item] = g;
        if (want_hess && d.out_hess) d.out_hess[item] = h;
    }
}

// logL alone (a forward part): warp i sums problem i's slots in the order reduce_kernel does
template <int MAXB>
__global__ void __launch_bounds__(256) reduce_logl_kernel(const __grid_constant__ BatchArgs<MAXB> a) {
    pdl_wait();
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (gw >= a.n) return;
    const ProbDesc &d = a.d[gw];
    const double s = warp_sum(lane_sum(d.lpart, d.n_tg, lane));
    if (lane == 0 && d.out_logL) *d.out_logL = s;
}

template <int C>
size_t f32_dyn_smem(int range_len) {
    return f32_stage_bytes<C>(kBlock / 32) + (size_t)range_len * (2 * sizeof(float) + sizeof(int));
}

template <int C, bool HESS, int MAXB>
cudaError_t launch_tree_cc(const BatchArgs<MAXB> &args, bool f64, cudaStream_t s) {
    const int blocks = args.tile_base[args.n];
    if (f64) {
        tree4d_kernel<C, HESS, MAXB><<<blocks, kBlock, 0, s>>>(args);
    } else {
        int rl = 0;
        for (int i = 0; i < args.n; ++i) rl = rl > args.d[i].range_len ? rl : args.d[i].range_len;
        const size_t smem = f32_dyn_smem<C>(rl);
        static DeviceOnce once;   // the shared-memory attribute, once per device
        if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(tree4f_kernel<C, HESS, MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32_dyn_smem<C>(kMaxRange)); }); e != cudaSuccess)
            return e;
        tree4f_kernel<C, HESS, MAXB><<<blocks, kBlock, smem, s>>>(args);
    }
    return cudaGetLastError();
}

template <int MAXB, bool HESS>
cudaError_t launch_tree_c(const BatchArgs<MAXB> &args, int C, bool f64, cudaStream_t s) {
    switch (C) {
        case 1: return launch_tree_cc<1, HESS, MAXB>(args, f64, s);
        case 2: return launch_tree_cc<2, HESS, MAXB>(args, f64, s);
        case 3: return launch_tree_cc<3, HESS, MAXB>(args, f64, s);
        case 4: return launch_tree_cc<4, HESS, MAXB>(args, f64, s);
        default: return cudaErrorInvalidValue;
    }
}

// resident blocks per SM of the fused kernel, queried once per device
template <int C, bool F64>
int occupancy_of() {
    static DeviceOnce once;
    int k = 1;
    const cudaError_t e = device_once(once, [](int &v) {
        cudaError_t r;
        if (F64) {
            r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, tree4d_kernel<C, true, kMaxBatch>, kBlock, 0);
        } else {
            const size_t smem = f32_dyn_smem<C>(64);
            r = cudaFuncSetAttribute(tree4f_kernel<C, true, kMaxBatch>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)f32_dyn_smem<C>(kMaxRange));
            if (r == cudaSuccess)
                r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, tree4f_kernel<C, true, kMaxBatch>, kBlock, smem);
        }
        if (v < 1) v = 1;
        return r;
    }, &k);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return k;
}

}  // namespace

int tree_blocks_per_sm(int C, bool f64) {
    switch (C * 2 + (f64 ? 1 : 0)) {
        case 2: return occupancy_of<1, false>();
        case 3: return occupancy_of<1, true>();
        case 4: return occupancy_of<2, false>();
        case 5: return occupancy_of<2, true>();
        case 6: return occupancy_of<3, false>();
        case 7: return occupancy_of<3, true>();
        case 8: return occupancy_of<4, false>();
        case 9: return occupancy_of<4, true>();
        default: return 1;
    }
}

// All problems in args share the category count args.d[0].C and the precision args.d[0].precision.
template <int MAXB>
cudaError_t launch_pmatrix(const BatchArgs<MAXB> &args, cudaStream_t s) {
    const int nmat = args.mat_base[args.n];
    if (args.n <= 0 || nmat <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch (the kernel waits before storing)
    cfg.gridDim = dim3((unsigned)((nmat * 16 + 127) / 128));
    cfg.blockDim = dim3(128);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pmatrix4_kernel<MAXB>, args);
}

template <int MAXB>
cudaError_t launch_tree(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s) {
    if (args.n <= 0 || args.tile_base[args.n] <= 0) return cudaSuccess;
    if constexpr (MAXB == 1) {
        if (args.d[0].small64) return launch_small64(args, hess, s);
    }
    const bool f64 = args.d[0].precision == 1;
    return hess ? launch_tree_c<MAXB, true>(args, args.d[0].C, f64, s)
                : launch_tree_c<MAXB, false>(args, args.d[0].C, f64, s);
}

template <int MAXB>
cudaError_t launch_reduce(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s) {
    if (args.n <= 0) return cudaSuccess;
    bool branches = false, logl = false;   // what the launch's problems want
    for (int i = 0; i < args.n; ++i) {
        branches = branches || args.d[i].out_grad || (hess && args.d[i].out_hess);
        logl = logl || args.d[i].out_logL;
    }
    if (!branches && !logl) return cudaSuccess;
    // a forward part (logL only) needs one warp per problem; else a row of blocks per problem with
    // a warp per branch and one for logL
    int per = 0;
    for (int i = 0; i < args.n; ++i) {
        const int w = args.red_base[i + 1] - args.red_base[i];
        per = per > w ? per : w;
    }
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch (the kernel waits in pdl_wait)
    cfg.gridDim = branches ? dim3((unsigned)((per + 7) / 8), (unsigned)args.n) : dim3((unsigned)((args.n + 7) / 8));
    cfg.blockDim = dim3(256);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!branches) return cudaLaunchKernelEx(&cfg, reduce_logl_kernel<MAXB>, args);
    return cudaLaunchKernelEx(&cfg, reduce_kernel<MAXB>, args, hess ? 1 : 0);
}

template <int MAXB>
cudaError_t launch_eval_nt(const BatchArgs<MAXB> &args, bool hess, cudaStream_t s) {
    cudaError_t e = launch_pmatrix<MAXB>(args, s);
    if (e == cudaSuccess) e = launch_tree<MAXB>(args, hess, s);
    if (e == cudaSuccess) e = launch_reduce<MAXB>(args, hess, s);
    return e;
}

// out[i] = sum over j = 0 .. k-1, in that order, of parts[j n + i]
__global__ void __launch_bounds__(256) chunk_sum_kernel(const double *parts, int k, int n, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = 0.0;
    for (int j = 0; j < k; ++j) v += parts[(size_t)j * n + i];
    out[i] = v;
}

cudaError_t launch_chunk_sum(const double *parts, int k, int n, double *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    chunk_sum_kernel<<<(n + 255) / 256, 256, 0, s>>>(parts, k, n, out);
    return cudaGetLastError();
}

template cudaError_t launch_eval_nt<1>(const BatchArgs<1> &, bool, cudaStream_t);
template cudaError_t launch_pmatrix<1>(const BatchArgs<1> &, cudaStream_t);
template cudaError_t launch_tree<1>(const BatchArgs<1> &, bool, cudaStream_t);
template cudaError_t launch_reduce<1>(const BatchArgs<1> &, bool, cudaStream_t);
template cudaError_t launch_eval_nt<kMaxBatch>(const BatchArgs<kMaxBatch> &, bool, cudaStream_t);
template cudaError_t launch_pmatrix<kMaxBatch>(const BatchArgs<kMaxBatch> &, cudaStream_t);
template cudaError_t launch_tree<kMaxBatch>(const BatchArgs<kMaxBatch> &, bool, cudaStream_t);
template cudaError_t launch_reduce<kMaxBatch>(const BatchArgs<kMaxBatch> &, bool, cudaStream_t);

}  // namespace pg
