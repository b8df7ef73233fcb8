// General state spaces (any of 2..64 states but 4, e.g. the 61 sense codons or 20 amino acids;
// also 4-state problems with tip partial vectors): the transition
// tables, the post-order pass (Section 2.3), the root mixture (Section 2.5), the pre-order pass
// (Section 2.4) with the branch gradient (Section 2.5) and Hessian diagonal (Section 2.6), and the
// fixed-order reduction.  SIMT FP32 products; every column (pattern, category) carries its own
// power-of-two exponent.
//
// Work item = (node, tile of kMTile patterns), one thread block of 256 threads; thread (tp, ts)
// owns patterns 4 tp .. 4 tp + 3 of the tile and states 4 ts .. 4 ts + 3.  A product of a table T
// (rows k = input state, columns s = output state) with a tile X (pattern-major rows of kMP states)
// runs as a register-tiled outer-product loop over k from shared memory.
#include <cuda_runtime.h>

#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

constexpr int kMThreads = 256;
constexpr int kLDX = kMP + 4;                 // row stride (floats) of pattern-major tiles
constexpr int kTileFloats = kMTile * kLDX;
constexpr int kRootThreads = 256;

__device__ __forceinline__ const float *tab_of(const MDesc &d, int c, int l, int kind) {
    return d.tabs + ((size_t)(c * d.C + l) * kTabKinds + kind) * kTabFloats;
}
__device__ __forceinline__ size_t row_of(const MDesc &d, int node, int l, int p) {   // column start
    return (((size_t)(node - d.n_tips) * d.C + l) * d.Ps + p) * kMP;
}
__device__ __forceinline__ size_t col_of(const MDesc &d, int node, int l, int p) {   // exponent index
    return ((size_t)(node - d.n_tips) * d.C + l) * d.Ps + p;
}

__device__ __forceinline__ void load_table(float *dst, const float *src) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int i = threadIdx.x; i < kTabFloats / 4; i += blockDim.x) d4[i] = __ldg(s4 + i);
}

// cnt columns (contiguous kMP-float rows in global memory) into a pattern-major tile; rows >= cnt
// are zero
__device__ __forceinline__ void load_rows(float *dst, const float *src, int cnt) {
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    for (int i = threadIdx.x; i < kMTile * kMP / 4; i += blockDim.x) {
        const int p = i / (kMP / 4), q = i - p * (kMP / 4);
        const float4 v = p < cnt ? __ldcg(s4 + i) : f4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4 *>(dst + p * kLDX + 4 * q) = v;
    }
}

// y[i][j] = sum_k T[k][4 ts + j] * X[4 tp + i][k]
__device__ __forceinline__ void gemm_tile(const float *T, const float *X, int tp, int ts, float y[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) y[i][j] = 0.f;
#pragma unroll 8
    for (int k = 0; k < kMP; ++k) {
        const float4 a = *reinterpret_cast<const float4 *>(T + k * kMP + 4 * ts);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = X[(4 * tp + i) * kLDX + k];
            y[i][0] = fmaf(a.x, x, y[i][0]);
            y[i][1] = fmaf(a.y, x, y[i][1]);
            y[i][2] = fmaf(a.z, x, y[i][2]);
            y[i][3] = fmaf(a.w, x, y[i][3]);
        }
    }
}

// the identity part of P = I + D: y += X (own rows)
__device__ __forceinline__ void add_tile(const float *X, int tp, int ts, float y[4][4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float4 x = *reinterpret_cast<const float4 *>(X + (4 * tp + i) * kLDX + 4 * ts);
        y[i][0] += x.x;
        y[i][1] += x.y;
        y[i][2] += x.z;
        y[i][3] += x.w;
    }
}

// a tip child: y[i][.] = column code_i of the table (+1 on the diagonal for P = I + D), the
// table's ambiguous-code row (row sums) for missing data, or for a partially observed tip (a row v
// of d.tipv) the columns weighted by v (+ v for P = I + D)
__device__ __forceinline__ void tip_tile(const float *T, const int code[4], const MDesc &d, int ts, bool ident,
                                         float y[4][4]) {
    const int m = d.m;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (code[i] >= m && code[i] < m + d.n_tv) {
            const float *v = d.tipv + (size_t)(code[i] - m) * kMP;
            float4 a = ident ? __ldg(reinterpret_cast<const float4 *>(v) + ts) : f4(0.f, 0.f, 0.f, 0.f);
            for (int k = 0; k < m; ++k) {
                const float vk = __ldg(v + k);
                if (vk == 0.f) continue;
                const float4 c = *reinterpret_cast<const float4 *>(T + k * kMP + 4 * ts);
                a = f4(fmaf(vk, c.x, a.x), fmaf(vk, c.y, a.y), fmaf(vk, c.z, a.z), fmaf(vk, c.w, a.w));
            }
            y[i][0] = a.x;
            y[i][1] = a.y;
            y[i][2] = a.z;
            y[i][3] = a.w;
            continue;
        }
        const int r = code[i] < m ? code[i] : kMP;
        const float4 a = *reinterpret_cast<const float4 *>(T + r * kMP + 4 * ts);
        y[i][0] = a.x;
        y[i][1] = a.y;
        y[i][2] = a.z;
        y[i][3] = a.w;
        if (ident && r < m) {
            const int jj = r - 4 * ts;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (jj == j) y[i][j] += 1.f;
        }
    }
}

__device__ __forceinline__ void tip_codes(const MDesc &d, int c, int p0, int cnt, int tp, int code[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = 4 * tp + i;
        code[i] = q < cnt ? (int)__ldg(d.tips + (size_t)c * d.Ps + p0 + q) : 0;
    }
}

__device__ __forceinline__ float max16(float v) {   // over the 16 lanes sharing tp
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float sum16(float v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one exponent per column: the column's largest state scaled into [1, 2); writes rows + exponents
__device__ __forceinline__ void store_scaled(float *rows, int *exps, const MDesc &d, int node, int l, int p0,
                                             int cnt, int tp, int ts, float v[4][4], const int E[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float mx = max16(fmaxf(fmaxf(v[i][0], v[i][1]), fmaxf(v[i][2], v[i][3])));
        const int q = 4 * tp + i;
        if (q >= cnt) continue;
        const int e = scale_exponent(mx);
        __stcg(reinterpret_cast<float4 *>(rows + row_of(d, node, l, p0 + q)) + ts,
               scale4(f4(v[i][0], v[i][1], v[i][2], v[i][3]), e));
        if (ts == 0) __stcg(exps + col_of(d, node, l, p0 + q), E[i] + e);
    }
}

// ---- transition tables ------------------------------------------------------------------------
// Block (branch c, category l), thread (ts, tj) owns rows s = 4 ts + a and columns j = 4 tj + b of
// the 64 x 64 tables.  D by uniformisation (see MDesc), then G = r (Q + Q D) and H = r Q G as
// products from shared memory.  SIMT layout: DT, GT, HT transposed (row j = column j) with the row
// sums as the ambiguous-code row (1 + row sums of D for P) and D row-major for P^T q.  With TC the
// tensor-core layout instead: row-major D, G, H and D^T, each with its TF32 remainder
// W - trunc_tf32(W) (kTcKinds tables of kMP x kMP per branch and category).
__device__ __forceinline__ float tf32_rem(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u); }

// acc[a][b] = sum_k A[k][4 ts + a] * Bm[k][4 tj + b]  (A = left operand transposed, Bm row-major)
__device__ __forceinline__ void smem_product(const float *A, const float *Bm, int ts, int tj, float acc[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 8
    for (int k = 0; k < kMP; ++k) {
        const float4 w = *reinterpret_cast<const float4 *>(A + k * kMP + 4 * ts);
        const float4 u = *reinterpret_cast<const float4 *>(Bm + k * kMP + 4 * tj);
        const float wa[4] = {w.x, w.y, w.z, w.w}, ub[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(wa[a], ub[b], acc[a][b]);
    }
}
__device__ __forceinline__ void put_rowmajor(float *M, int ts, int tj, const float acc[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4 *>(M + (4 * ts + a) * kMP + 4 * tj) = f4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
}
__device__ __forceinline__ void put_transposed(float *M, int ts, int tj, const float acc[4][4]) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
        *reinterpret_cast<float4 *>(M + (4 * tj + b) * kMP + 4 * ts) = f4(acc[0][b], acc[1][b], acc[2][b], acc[3][b]);
}
__device__ __forceinline__ void put_rem(float *M, const float acc[4][4], int ts, int tj, bool transposed) {
    float r[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) r[a][b] = tf32_rem(acc[a][b]);
    if (transposed) put_transposed(M, ts, tj, r);
    else put_rowmajor(M, ts, tj, r);
}

// kind 0: D, 1: G, 2: H of (c, l) into the table layout
template <bool TC>
// (stage: a free kMP x kMP shared-memory tile, used by the tensor-core layout's transposed D; all
// threads of the block call this)
__device__ __forceinline__ void store_tables(const MDesc &d, int c, int l, int kind, const float acc[4][4], int ts, int tj,
                                             float *stage) {
    if constexpr (TC) {
        float *base = d.tabs + (size_t)(c * d.C + l) * kTcKinds * kMP * kMP;
        const int hk = kind == 0 ? kTcD : (kind == 1 ? kTcG : kTcH);
        const int lk = kind == 0 ? kTcDlo : (kind == 1 ? kTcGlo : kTcHlo);
        put_rowmajor(base + (size_t)hk * kMP * kMP, ts, tj, acc);
        put_rem(base + (size_t)lk * kMP * kMP, acc, ts, tj, false);
        if (kind == 0) {   // D^T and its remainder through shared memory, so the rows go out whole
            put_transposed(stage, ts, tj, acc);
            __syncthreads();
            float4 *dt = reinterpret_cast<float4 *>(base + (size_t)kTcDT * kMP * kMP);
            float4 *dtlo = reinterpret_cast<float4 *>(base + (size_t)kTcDTlo * kMP * kMP);
            for (int i = threadIdx.x; i < kMP * kMP / 4; i += blockDim.x) {
                const float4 v = reinterpret_cast<const float4 *>(stage)[i];
                dt[i] = v;
                dtlo[i] = f4(tf32_rem(v.x), tf32_rem(v.y), tf32_rem(v.z), tf32_rem(v.w));
            }
            __syncthreads();
        }
    } else {
        float rs[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) rs[a] = sum16(acc[a][0] + acc[a][1] + acc[a][2] + acc[a][3]);
        float *T = d.tabs + ((size_t)(c * d.C + l) * kTabKinds + (kind == 0 ? kTabDT : (kind == 1 ? kTabGT : kTabHT))) * kTabFloats;
        put_transposed(T, ts, tj, acc);
        if (tj == 0) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int s = 4 * ts + a;
                T[kMP * kMP + s] = kind == 0 ? (s < d.m ? 1.f + rs[a] : 0.f) : rs[a];
            }
        }
        if (kind == 0) put_rowmajor(d.tabs + ((size_t)(c * d.C + l) * kTabKinds + kTabD) * kTabFloats, ts, tj, acc);
    }
}

template <bool TC>
__global__ void __launch_bounds__(kMThreads) m_pmatrix_kernel(const __grid_constant__ MDesc d, int kinds) {
    __shared__ __align__(16) float A[kMP * kMP];    // left operand, transposed
    __shared__ __align__(16) float Bm[kMP * kMP];   // right operand, row-major
    __shared__ float ck[kUnifK + 1];
    __shared__ float e0;
    __shared__ int nk, nsq;
    const int c = blockIdx.x / d.C, l = blockIdx.x - c * d.C;
    if (c == d.root) return;
    const double bl = d.b[c];
    if (!(bl >= 0.0) || isinf(bl)) {
        if (threadIdx.x == 0) atomicOr(d.status, kStatusBadLength);
        return;
    }
    const int md = d.bmodel ? d.bmodel[c] : 0;
    const float r = (float)d.rates[l];
    if (threadIdx.x < 32) {   // Poisson weights w_k = e^{-x} x^k / k! of the (halved) interval, FP64
        static_assert(kUnifK <= 32, "one lane per power");
        const int lane = threadIdx.x;
        double x = d.mu[md] * bl * d.rates[l];
        int s = 0;
        while (x > 4.0 && s < 1000) {
            x *= 0.5;
            ++s;
        }
        const int K = min(kUnifK, (int)ceil(x + 6.0 * sqrt(x) + 10.0));
        // lane k - 1 holds x / k; an inclusive prefix product over the lanes gives x^k / k!
        double f = x / (double)(lane + 1);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double g = __shfl_up_sync(0xffffffffu, f, o);
            if (lane >= o) f *= g;
        }
        if (lane < K) ck[lane + 1] = (float)(exp(-x) * f);
        if (lane == 0) {
            e0 = (float)expm1(-x);
            nk = K;
            nsq = s;
        }
    }
    __syncthreads();
    const int ts = threadIdx.x >> 4, tj = threadIdx.x & 15;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    const float *Bp = d.Bpow + (size_t)md * kUnifK * kMP * kMP;
    for (int k = 1; k <= nk; ++k) {
        const float w = ck[k];
        const float *Bk = Bp + (size_t)(k - 1) * kMP * kMP;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(Bk + (4 * ts + a) * kMP + 4 * tj));
            acc[a][0] = fmaf(w, v.x, acc[a][0]);
            acc[a][1] = fmaf(w, v.y, acc[a][1]);
            acc[a][2] = fmaf(w, v.z, acc[a][2]);
            acc[a][3] = fmaf(w, v.w, acc[a][3]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            if (4 * ts + a == 4 * tj + b && 4 * ts + a < d.m) acc[a][b] += e0;
    for (int i = 0; i < nsq; ++i) {   // P(2t) = P(t)^2 in the D form: D <- 2 D + D D
        put_transposed(A, ts, tj, acc);
        put_rowmajor(Bm, ts, tj, acc);
        __syncthreads();
        float sq[4][4];
        smem_product(A, Bm, ts, tj, sq);
        __syncthreads();
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(2.f, acc[a][b], sq[a][b]);
    }
    store_tables<TC>(d, c, l, 0, acc, ts, tj, A);
    // G = r (Q + Q D)
    {
        const float4 *src = reinterpret_cast<const float4 *>(d.QT + (size_t)md * kMP * kMP);
        for (int i = threadIdx.x; i < kMP * kMP / 4; i += blockDim.x) reinterpret_cast<float4 *>(A)[i] = __ldg(src + i);
    }
    put_rowmajor(Bm, ts, tj, acc);
    __syncthreads();
    float g[4][4];
    smem_product(A, Bm, ts, tj, g);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) g[a][b] = r * (g[a][b] + A[(4 * tj + b) * kMP + 4 * ts + a]);
    store_tables<TC>(d, c, l, 1, g, ts, tj, nullptr);
    if (kinds > 2) {   // H = r Q G
        __syncthreads();
        put_rowmajor(Bm, ts, tj, g);
        __syncthreads();
        float h[4][4];
        smem_product(A, Bm, ts, tj, h);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) h[a][b] *= r;
        store_tables<TC>(d, c, l, 2, h, ts, tj, nullptr);
    }
}

// ---- post-order level ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMThreads) m_post_kernel(const __grid_constant__ MDesc d, int o0, int n_pt) {
    extern __shared__ __align__(16) float msm[];
    float *T = msm, *X = msm + kTabFloats;
    const int u = blockIdx.x / n_pt, pt = blockIdx.x - u * n_pt;
    const int4 op = __ldg(d.ops + o0 + u);
    const int N = d.n_tips, k = op.x;
    const int p0 = pt * kMTile, cnt = min(kMTile, d.P - p0);
    const int tp = threadIdx.x >> 4, ts = threadIdx.x & 15;
    for (int l = 0; l < d.C; ++l) {
        float v[4][4];
        int E[4] = {0, 0, 0, 0};
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int c = side ? op.z : op.y;
            __syncthreads();   // the previous readers of T and X are done
            load_table(T, tab_of(d, c, l, kTabDT));
            if (c >= N) load_rows(X, d.post + row_of(d, c, l, p0), cnt);
            __syncthreads();
            float y[4][4];
            if (c >= N) {
                gemm_tile(T, X, tp, ts, y);
                add_tile(X, tp, ts, y);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int q = 4 * tp + i;
                    if (q < cnt) E[i] += __ldcg(d.pe + col_of(d, c, l, p0 + q));
                }
            } else {
                int code[4];
                tip_codes(d, c, p0, cnt, tp, code);
                tip_tile(T, code, d, ts, true, y);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) v[i][j] = side ? v[i][j] * y[i][j] : y[i][j];
        }
        store_scaled(d.post, d.pe, d, k, l, p0, cnt, tp, ts, v, E);
    }
}

// ---- root: L_p = sum_l w_l 2^{E_l} pi . x_l (Section 2.5) ----------------------------------------
// 16 lanes per pattern (4 states each, FP64 products and a fixed shuffle tree), kMRootPatterns
// patterns per block: the FP64 work spreads over the SMs, and the block's weighted sum of log L_p is
// one slot of lpart.
__global__ void __launch_bounds__(kRootThreads) m_root_kernel(const __grid_constant__ MDesc d) {
    __shared__ double wsum[kRootThreads / 32];
    const int sub = threadIdx.x & 15, p = blockIdx.x * kMRootPatterns + (threadIdx.x >> 4);
    const bool on = p < d.P;
    double term = 0.0, s[kMaxCat];
    int Ec[kMaxCat], Emax = -0x7fffffff;
    for (int l = 0; l < d.C; ++l) {   // every lane takes part in the shuffles
        const float4 v = on ? __ldcg(reinterpret_cast<const float4 *>(d.post + row_of(d, d.root, l, p)) + sub)
                            : f4(0.f, 0.f, 0.f, 0.f);
        double a = d.pi[4 * sub] * (double)v.x;
        a = fma(d.pi[4 * sub + 1], (double)v.y, a);
        a = fma(d.pi[4 * sub + 2], (double)v.z, a);
        a = fma(d.pi[4 * sub + 3], (double)v.w, a);
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o, 16);
        s[l] = a;
        Ec[l] = on ? __ldcg(d.pe + col_of(d, d.root, l, p)) : 0;
        Emax = max(Emax, Ec[l]);
    }
    if (on && sub == 0) {
        double S = 0.0;
        for (int l = 0; l < d.C; ++l) S = fma(d.cw[l], ldexp(s[l], Ec[l] - Emax), S);
        int e2 = 0;
        const double f = (S > 0.0 && isfinite(S)) ? frexp(S, &e2) : S;
        const int Er = Emax + e2;
        const int Et = d.tip_E ? __ldg(d.tip_E + p) : 0;   // the tip rows' scales
        const double lp = log(f) + (double)(Er + Et) * 0.69314718055994530942;
        d.site_invL[p] = (float)(1.0 / f);
        d.site_Er[p] = Er;
        if (!(f > 0.0) || !isfinite(lp)) atomicOr(d.status, kStatusNumeric);
        if (d.out_site) d.out_site[p] = lp;
        const double w = d.weights[p];
        term = w != 0.0 ? w * lp : 0.0;
    }
    term = warp_sum(term);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRootThreads / 32; ++w) t += wsum[w];
        d.lpart[blockIdx.x] = t;
    }
}

// ---- pre-order level with the gradient -----------------------------------------------------------
// Node k with children c0, c1, per category: a_c = P_c x_c; the top of branch c is
// qt_c = q_k o a_other (q_root = pi); the branch term qt_c . (G_c x_c) 2^{E} / L_p (Section 2.5,
// top-of-branch form); q_c = P_c^T qt_c for an internal child (Section 2.4).
template <bool HESS>
__global__ void __launch_bounds__(kMThreads) m_pre_kernel(const __grid_constant__ MDesc d, int o0, int n_pt) {
    extern __shared__ __align__(16) float msm[];
    float *T = msm;
    float *Xs[2] = {msm + kTabFloats, msm + kTabFloats + kTileFloats};
    float *Qk = msm + kTabFloats + 2 * kTileFloats, *Qt = Qk + kTileFloats;
    __shared__ double red[2][2][kMThreads / 16];
    const int u = blockIdx.x / n_pt, pt = blockIdx.x - u * n_pt;
    const int4 op = __ldg(d.ops + o0 + u);
    const int N = d.n_tips, k = op.x;
    const bool root = k == d.root;
    const int p0 = pt * kMTile, cnt = min(kMTile, d.P - p0);
    const int tp = threadIdx.x >> 4, ts = threadIdx.x & 15;
    const int cs[2] = {op.y, op.z};
    float inv[4], dsum[2][4], hsum[2][4];
    int Er[4], code[2][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = 4 * tp + i;
        inv[i] = q < cnt ? __ldcg(d.site_invL + p0 + q) : 0.f;
        Er[i] = q < cnt ? __ldcg(d.site_Er + p0 + q) : 0;
        dsum[0][i] = dsum[1][i] = hsum[0][i] = hsum[1][i] = 0.f;
    }
#pragma unroll
    for (int side = 0; side < 2; ++side)
        if (cs[side] < N) tip_codes(d, cs[side], p0, cnt, tp, code[side]);
    for (int l = 0; l < d.C; ++l) {
        __syncthreads();   // the previous category's readers of the tiles are done
        if (!root) load_rows(Qk, d.pre + row_of(d, k, l, p0), cnt);
#pragma unroll
        for (int side = 0; side < 2; ++side)
            if (cs[side] >= N) load_rows(Xs[side], d.post + row_of(d, cs[side], l, p0), cnt);
        int Eq[4], Ex[2][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = 4 * tp + i;
            const bool on = q < cnt;
            Eq[i] = (on && !root) ? __ldcg(d.qe + col_of(d, k, l, p0 + q)) : 0;
#pragma unroll
            for (int side = 0; side < 2; ++side)
                Ex[side][i] = (on && cs[side] >= N) ? __ldcg(d.pe + col_of(d, cs[side], l, p0 + q)) : 0;
        }
        float a[2][4][4];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            __syncthreads();
            load_table(T, tab_of(d, cs[side], l, kTabDT));
            __syncthreads();
            if (cs[side] >= N) {
                gemm_tile(T, Xs[side], tp, ts, a[side]);
                add_tile(Xs[side], tp, ts, a[side]);
            } else {
                tip_tile(T, code[side], d, ts, true, a[side]);
            }
        }
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int c = cs[side];
            float qt[4][4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float4 qk = root ? f4(d.pif[4 * ts], d.pif[4 * ts + 1], d.pif[4 * ts + 2], d.pif[4 * ts + 3])
                                       : *reinterpret_cast<const float4 *>(Qk + (4 * tp + i) * kLDX + 4 * ts);
                qt[i][0] = qk.x * a[1 - side][i][0];
                qt[i][1] = qk.y * a[1 - side][i][1];
                qt[i][2] = qk.z * a[1 - side][i][2];
                qt[i][3] = qk.w * a[1 - side][i][3];
            }
            for (int kind = 0; kind < (HESS ? 2 : 1); ++kind) {
                __syncthreads();
                load_table(T, tab_of(d, c, l, kind ? kTabHT : kTabGT));
                __syncthreads();
                float uu[4][4];
                if (c >= N) gemm_tile(T, Xs[side], tp, ts, uu);
                else tip_tile(T, code[side], d, ts, false, uu);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float t = qt[i][0] * uu[i][0];
                    t = fmaf(qt[i][1], uu[i][1], t);
                    t = fmaf(qt[i][2], uu[i][2], t);
                    t = fmaf(qt[i][3], uu[i][3], t);
                    t = sum16(t);
                    const int dE = Eq[i] + Ex[1 - side][i] + Ex[side][i] - Er[i];
                    const float term = (float)d.cw[l] * ldexp2f(t, dE) * inv[i];
                    if (kind == 0) dsum[side][i] += term;
                    else hsum[side][i] += term;
                }
            }
            if (c >= N) {   // q_c = P_c^T qt = qt + D^T qt
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    *reinterpret_cast<float4 *>(Qt + (4 * tp + i) * kLDX + 4 * ts) = f4(qt[i][0], qt[i][1], qt[i][2], qt[i][3]);
                __syncthreads();
                load_table(T, tab_of(d, c, l, kTabD));
                __syncthreads();
                float qq[4][4];
                gemm_tile(T, Qt, tp, ts, qq);
                add_tile(Qt, tp, ts, qq);
                int E[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) E[i] = Eq[i] + Ex[1 - side][i];
                store_scaled(d.pre, d.qe, d, c, l, p0, cnt, tp, ts, qq, E);
            }
        }
    }
    // per child branch: sum over the tile's patterns of w_p d_p and w_p (h_p - d_p^2), fixed order
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        double g = 0.0, h = 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int q = 4 * tp + i;
            if (q >= cnt) continue;
            const double w = d.weights[p0 + q];
            if (w == 0.0) continue;
            g += w * (double)dsum[side][i];
            if (HESS) h += w * ((double)hsum[side][i] - (double)dsum[side][i] * (double)dsum[side][i]);
        }
        if (ts == 0) {
            red[side][0][tp] = g;
            red[side][1][tp] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        const int side = threadIdx.x;
        double g = 0.0, h = 0.0;
        for (int j = 0; j < kMThreads / 16; ++j) {
            g += red[side][0][j];
            h += red[side][1][j];
        }
        d.gpart[(size_t)cs[side] * d.n_gslots + pt] = g;
        if (HESS) d.hpart[(size_t)cs[side] * d.n_gslots + pt] = h;
    }
}

// ---- fixed-order reduction: one warp per branch, one for logL --------------------------------------
__global__ void __launch_bounds__(256) m_reduce_kernel(const __grid_constant__ MDesc d, int want_hess, int n_lblocks) {
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gw > d.n_nodes) return;
    if (gw == d.n_nodes) {
        double s = 0.0;
        for (int j = lane; j < n_lblocks; j += 32) s += d.lpart[j];
        s = warp_sum(s);
        if (lane == 0 && d.out_logL) *d.out_logL = s;
        return;
    }
    double g = 0.0, h = 0.0;
    if (gw != d.root) {
        for (int j = lane; j < d.n_gslots; j += 32) g += d.gpart[(size_t)gw * d.n_gslots + j];
        g = warp_sum(g);
        if (want_hess) {
            for (int j = lane; j < d.n_gslots; j += 32) h += d.hpart[(size_t)gw * d.n_gslots + j];
            h = warp_sum(h);
        }
    }
    if (lane == 0) {
        if (d.gscale) g *= *d.gscale;
        if (d.out_grad) d.out_grad[gw] = g;
        if (want_hess && d.out_hess) d.out_hess[gw] = h;
    }
}

constexpr size_t kPostSmem = sizeof(float) * (kTabFloats + kTileFloats);
constexpr size_t kPreSmem = sizeof(float) * (kTabFloats + 4 * kTileFloats);

}  // namespace

cudaError_t launch_m_pmatrix(const MDesc &d, bool hess, cudaStream_t s) {
    if (d.n_nodes * d.C <= 0) return cudaSuccess;
    if (d.tc) m_pmatrix_kernel<true><<<d.n_nodes * d.C, kMThreads, 0, s>>>(d, hess ? 3 : 2);
    else m_pmatrix_kernel<false><<<d.n_nodes * d.C, kMThreads, 0, s>>>(d, hess ? 3 : 2);
    return cudaGetLastError();
}

cudaError_t launch_m_post_level(const MDesc &d, int o0, int nd, cudaStream_t s) {
    if (nd <= 0 || d.n_ptiles <= 0) return cudaSuccess;
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_post_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPostSmem); }); e != cudaSuccess)
        return e;
    m_post_kernel<<<nd * d.n_ptiles, kMThreads, kPostSmem, s>>>(d, o0, d.n_ptiles);
    return cudaGetLastError();
}

cudaError_t launch_m_root(const MDesc &d, cudaStream_t s) {
    if (d.P <= 0) return cudaSuccess;
    m_root_kernel<<<(d.P + kMRootPatterns - 1) / kMRootPatterns, kRootThreads, 0, s>>>(d);
    return cudaGetLastError();
}

template <bool HESS>
cudaError_t launch_m_pre_h(const MDesc &d, int o0, int nd, cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_pre_kernel<HESS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPreSmem); }); e != cudaSuccess)
        return e;
    m_pre_kernel<HESS><<<nd * d.n_ptiles, kMThreads, kPreSmem, s>>>(d, o0, d.n_ptiles);
    return cudaGetLastError();
}

cudaError_t launch_m_pre_level(const MDesc &d, int o0, int nd, bool hess, cudaStream_t s) {
    if (nd <= 0 || d.n_ptiles <= 0) return cudaSuccess;
    return hess ? launch_m_pre_h<true>(d, o0, nd, s) : launch_m_pre_h<false>(d, o0, nd, s);
}

cudaError_t launch_m_reduce(const MDesc &d, bool hess, cudaStream_t s) {
    const int warps = d.n_nodes + 1;
    const int n_lblocks = (d.P + kMRootPatterns - 1) / kMRootPatterns;
    m_reduce_kernel<<<(warps + 7) / 8, 256, 0, s>>>(d, hess ? 1 : 0, n_lblocks);
    return cudaGetLastError();
}

}  // namespace pg
