// Cherry level of the general-state path (tensor-core table layout): nodes whose two children are
// both tips.  A tip's state vector x is one-hot (or all-ones over the m states for an ambiguous
// code), so P x is a column of P = I + D and G x a column of G: the post-order product (Section 2.3)
// and the pre-order branch terms (Sections 2.4-2.5) are table lookups, done here in FP32 without
// the tensor core.  The rare partially observed tip (a row of the problem's tip-vector table)
// takes the sum of the columns weighted by its vector.  The tables of one (node, category) are copied into shared memory once as
// column tables, with the row sums (the all-ones case) as an extra column, and a block then walks a
// chunk of patterns: 16 lanes per pattern, 4 states per lane.
#include <cuda_runtime.h>

#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

constexpr int kChThreads = 256;            // 16 patterns x 16 lanes per step
constexpr int kChChunk = 1024;             // patterns per block
constexpr int kS = 68;                     // row stride (floats) of a column table in shared memory
constexpr int kColFloats = (kMP + 1) * kS;

// Column tables in shared memory: row k holds column k of the matrix (states contiguous, so a
// lane reads its 4 states of a column as one float4), row kMP the row sums (the column of an
// all-ones vector).
// from a transposed table in global memory (row k = column k already)
__device__ void columns_from_transposed(float *Cb, const MDesc &d, int c, int l, int kind) {
    const float4 *src = reinterpret_cast<const float4 *>(d.tabs + ((size_t)(c * d.C + l) * kTcKinds + kind) * kMP * kMP);
    for (int i = threadIdx.x; i < kMP * kMP / 4; i += blockDim.x)
        *reinterpret_cast<float4 *>(Cb + (i / (kMP / 4)) * kS + 4 * (i % (kMP / 4))) = __ldg(src + i);
}
// from a row-major table in global memory (transposed on the way in)
__device__ void columns_from_rows(float *Cb, const MDesc &d, int c, int l, int kind) {
    const float4 *src = reinterpret_cast<const float4 *>(d.tabs + ((size_t)(c * d.C + l) * kTcKinds + kind) * kMP * kMP);
    for (int i = threadIdx.x; i < kMP * kMP / 4; i += blockDim.x) {
        const float4 v = __ldg(src + i);
        const int s = i / (kMP / 4), k = 4 * (i % (kMP / 4));
        Cb[k * kS + s] = v.x;
        Cb[(k + 1) * kS + s] = v.y;
        Cb[(k + 2) * kS + s] = v.z;
        Cb[(k + 3) * kS + s] = v.w;
    }
}
__device__ void row_sums(float *Cb, int s) {   // one thread per state, fixed order
    float a = 0.f;
    for (int k = 0; k < kMP; ++k) a += Cb[k * kS + s];
    Cb[kMP * kS + s] = a;
}

// W v at this lane's states 4 j .. 4 j + 3 for the partial vector v of a partially observed tip
// (row y - m of d.tipv): the columns of W weighted by v, in state order
__device__ __forceinline__ float4 weighted_columns(const float *Wc, const MDesc &d, int y, int j) {
    const float *v = d.tipv + (size_t)(y - d.m) * kMP;
    float4 a = f4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < d.m; ++k) {
        const float vk = __ldg(v + k);
        if (vk == 0.f) continue;
        const float4 c = *reinterpret_cast<const float4 *>(Wc + k * kS + 4 * j);
        a = f4(fmaf(vk, c.x, a.x), fmaf(vk, c.y, a.y), fmaf(vk, c.z, a.z), fmaf(vk, c.w, a.w));
    }
    return a;
}

// P x = x + D x at this lane's states 4 j .. 4 j + 3 for the tip vector x of code y: column y of P
// for a state, P 1 (the row sums) for missing data, x + D x for a partially observed tip (TV: the
// problem has tip vectors)
template <bool TV>
__device__ __forceinline__ void p_column(const float *Dc, int y, const MDesc &d, int j, float a[4]) {
    const int m = d.m;
    if (TV && y >= m && y < m + d.n_tv) {
        const float4 dv = weighted_columns(Dc, d, y, j);
        const float4 x = __ldg(reinterpret_cast<const float4 *>(d.tipv + (size_t)(y - m) * kMP) + j);
        a[0] = x.x + dv.x;
        a[1] = x.y + dv.y;
        a[2] = x.z + dv.z;
        a[3] = x.w + dv.w;
        return;
    }
    const bool amb = y >= m;
    const float4 v = *reinterpret_cast<const float4 *>(Dc + (amb ? kMP : y) * kS + 4 * j);
    const float dv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int s = 4 * j + i;
        a[i] = (amb ? (s < m ? 1.f : 0.f) : (s == y ? 1.f : 0.f)) + dv[i];
    }
}
template <bool TV>
__device__ __forceinline__ void g_column(const float *Gc, int y, const MDesc &d, int j, float u[4]) {
    const float4 v = (TV && y >= d.m && y < d.m + d.n_tv) ? weighted_columns(Gc, d, y, j)
                                                          : *reinterpret_cast<const float4 *>(Gc + (y >= d.m ? kMP : y) * kS + 4 * j);
    u[0] = v.x;
    u[1] = v.y;
    u[2] = v.z;
    u[3] = v.w;
}
__device__ __forceinline__ float sum16(float v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
    return v;
}
__device__ __forceinline__ float max16(float v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o, 16));
    return v;
}

// The pattern loop: a step covers 256 patterns, 16 consecutive ones per 16-lane group.  Lane j
// first loads what belongs to pattern 16 g + j of the step (tip codes; for the pre-order its
// exponents, 1 / L_p and weight), so those loads are independent and in flight together; the group
// then takes its 16 patterns in turn with the codes broadcast by shuffles, and lane r keeps the
// result of pattern r.

// ---- post-order: p_k = (P_0 x_0) o (P_1 x_1), scaled by its largest state -------------------------
template <bool TV>
__global__ void __launch_bounds__(kChThreads) m_post_cherry_kernel(const __grid_constant__ MDesc d, int o0, int n_ch) {
    extern __shared__ float chs[];
    float *D0 = chs, *D1 = chs + kColFloats;
    const int item = blockIdx.x, pair = item / n_ch, ci = item - pair * n_ch;
    const int u = pair / d.C, l = pair - u * d.C;
    const int4 op = __ldg(d.ops + o0 + u);
    const int k = op.x, N = d.n_tips;
    columns_from_transposed(D0, d, op.y, l, kTcDT);
    columns_from_transposed(D1, d, op.z, l, kTcDT);
    __syncthreads();
    if (threadIdx.x < kMP) row_sums(D0, threadIdx.x);
    else if (threadIdx.x < 2 * kMP) row_sums(D1, threadIdx.x - kMP);
    __syncthreads();
    const int g = threadIdx.x >> 4, j = threadIdx.x & 15;
    const int pend = min(d.P, (ci + 1) * kChChunk);
    float *rows = d.post + ((size_t)(k - N) * d.C + l) * d.Ps * kMP;
    int *exps = d.pe + ((size_t)(k - N) * d.C + l) * d.Ps;
    for (int base = ci * kChChunk + 16 * g; base < ci * kChChunk + kChChunk; base += kChThreads) {   // uniform
        const int pl = base + j;
        const bool onl = pl < pend;
        const int y0l = onl ? (int)__ldg(d.tips + (size_t)op.y * d.Ps + pl) : 0;
        const int y1l = onl ? (int)__ldg(d.tips + (size_t)op.z * d.Ps + pl) : 0;
        int my_e = 0;
#pragma unroll 4
        for (int r = 0; r < 16; ++r) {
            const int y0 = __shfl_sync(0xffffffffu, y0l, r, 16), y1 = __shfl_sync(0xffffffffu, y1l, r, 16);
            float a0[4], a1[4], v[4];
            p_column<TV>(D0, y0, d, j, a0);
            p_column<TV>(D1, y1, d, j, a1);
            float mx = 0.f;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                v[i] = a0[i] * a1[i];
                mx = fmaxf(mx, v[i]);
            }
            const int e = scale_exponent(max16(mx));
            if (j == r) my_e = e;
            if (base + r < pend)
                __stcg(reinterpret_cast<float4 *>(rows + (size_t)(base + r) * kMP) + j, scale4(f4(v[0], v[1], v[2], v[3]), e));
        }
        if (onl) __stcg(exps + pl, my_e);
    }
}

// ---- pre-order branch terms of both children: qt_c . (G_c x_c) 2^{E} / L_p per category ---------------
// qt_0 = q_k o P_1 x_1, qt_1 = q_k o P_0 x_0 (q_root = pi); the block's weighted sum for category l
// and chunk ci goes to gradient slot l * n_pt + ci of each child (slots ci >= n_ch are zeroed).
template <bool TV>
__global__ void __launch_bounds__(kChThreads) m_pre_cherry_kernel(const __grid_constant__ MDesc d, int o0, int n_ch,
                                                                   int n_pt) {
    extern __shared__ float chs[];
    float *D0 = chs, *D1 = chs + kColFloats, *G0 = chs + 2 * kColFloats, *G1 = chs + 3 * kColFloats;
    __shared__ double red[2][kChThreads / 32];
    const int item = blockIdx.x, pair = item / n_ch, ci = item - pair * n_ch;
    const int u = pair / d.C, l = pair - u * d.C;
    const int4 op = __ldg(d.ops + o0 + u);
    const int k = op.x, N = d.n_tips;
    const bool root = k == d.root;
    columns_from_transposed(D0, d, op.y, l, kTcDT);
    columns_from_transposed(D1, d, op.z, l, kTcDT);
    columns_from_rows(G0, d, op.y, l, kTcG);
    columns_from_rows(G1, d, op.z, l, kTcG);
    __syncthreads();
    {
        const int r = threadIdx.x & (kMP - 1), which = threadIdx.x / kMP;   // 4 tables x 64 rows
        row_sums(which == 0 ? D0 : which == 1 ? D1 : which == 2 ? G0 : G1, r);
    }
    __syncthreads();
    const int g = threadIdx.x >> 4, j = threadIdx.x & 15;
    const int pend = min(d.P, (ci + 1) * kChChunk);
    const float *qrows = root ? nullptr : d.pre + ((size_t)(k - N) * d.C + l) * d.Ps * kMP;
    const int *qexp = root ? nullptr : d.qe + ((size_t)(k - N) * d.C + l) * d.Ps;
    const float cw = (float)d.cw[l];
    float4 pi4 = f4(0.f, 0.f, 0.f, 0.f);
    if (root) pi4 = f4(d.pif[4 * j], d.pif[4 * j + 1], d.pif[4 * j + 2], d.pif[4 * j + 3]);
    double acc[2] = {0.0, 0.0};
    for (int base = ci * kChChunk + 16 * g; base < ci * kChChunk + kChChunk; base += kChThreads) {   // uniform
        const int pl = base + j;
        const bool onl = pl < pend;
        const int y0l = onl ? (int)__ldg(d.tips + (size_t)op.y * d.Ps + pl) : 0;
        const int y1l = onl ? (int)__ldg(d.tips + (size_t)op.z * d.Ps + pl) : 0;
        const int dEl = onl ? (root ? 0 : __ldcg(qexp + pl)) - __ldcg(d.site_Er + pl) : 0;
        const float invl = onl ? __ldcg(d.site_invL + pl) : 0.f;
        const double wl = onl ? d.weights[pl] : 0.0;
        float my0 = 0.f, my1 = 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float4 qv[8];   // q_k rows of patterns 8 h .. 8 h + 7 of the group, this lane's states
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int p = base + 8 * h + r;
                qv[r] = (root || p >= pend) ? pi4 : __ldcs(reinterpret_cast<const float4 *>(qrows + (size_t)p * kMP) + j);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int rr = 8 * h + r;
                const int y0 = __shfl_sync(0xffffffffu, y0l, rr, 16), y1 = __shfl_sync(0xffffffffu, y1l, rr, 16);
                float a0[4], a1[4], u0[4], u1[4];
                p_column<TV>(D0, y0, d, j, a0);
                p_column<TV>(D1, y1, d, j, a1);
                g_column<TV>(G0, y0, d, j, u0);
                g_column<TV>(G1, y1, d, j, u1);
                const float q[4] = {qv[r].x, qv[r].y, qv[r].z, qv[r].w};
                float dot0 = 0.f, dot1 = 0.f;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    dot0 = fmaf(q[i] * a1[i], u0[i], dot0);   // top of branch 0: q_k o P_1 x_1
                    dot1 = fmaf(q[i] * a0[i], u1[i], dot1);
                }
                dot0 = sum16(dot0);
                dot1 = sum16(dot1);
                if (j == rr) {
                    my0 = dot0;
                    my1 = dot1;
                }
            }
        }
        if (onl && wl != 0.0) {
            acc[0] += wl * (double)(cw * ldexp2f(my0, dEl) * invl);
            acc[1] += wl * (double)(cw * ldexp2f(my1, dEl) * invl);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int side = 0; side < 2; ++side) {
        const double v = warp_sum(acc[side]);
        if (lane == 0) red[side][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double v = 0.0;
        for (int w = 0; w < kChThreads / 32; ++w) v += red[threadIdx.x][w];
        double *slots = d.gpart + (size_t)(threadIdx.x ? op.z : op.y) * d.n_gslots + (size_t)l * n_pt;
        slots[ci] = v;
        if (ci == 0)
            for (int c2 = n_ch; c2 < n_pt; ++c2) slots[c2] = 0.0;
    }
}

constexpr size_t kPostChSmem = 2 * kColFloats * sizeof(float);
constexpr size_t kPreChSmem = 4 * kColFloats * sizeof(float);

template <bool TV>
cudaError_t launch_pre_cherry(const MDesc &d, int o0, int nd, int n_ch, int n_pt, cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_pre_cherry_kernel<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPreChSmem); }); e != cudaSuccess)
        return e;
    m_pre_cherry_kernel<TV><<<nd * d.C * n_ch, kChThreads, kPreChSmem, s>>>(d, o0, n_ch, n_pt);
    return cudaGetLastError();
}

}  // namespace

// problems with tip vectors take the instantiations that look them up; the others keep the plain
// state and missing-data lookups
cudaError_t launch_m_post_cherry(const MDesc &d, int o0, int nd, cudaStream_t s) {
    const int n_ch = (d.P + kChChunk - 1) / kChChunk;
    if (nd <= 0 || n_ch <= 0) return cudaSuccess;
    if (d.n_tv > 0) m_post_cherry_kernel<true><<<nd * d.C * n_ch, kChThreads, kPostChSmem, s>>>(d, o0, n_ch);
    else m_post_cherry_kernel<false><<<nd * d.C * n_ch, kChThreads, kPostChSmem, s>>>(d, o0, n_ch);
    return cudaGetLastError();
}

cudaError_t launch_m_pre_cherry(const MDesc &d, int o0, int nd, cudaStream_t s) {
    const int n_ch = (d.P + kChChunk - 1) / kChChunk, n_pt = (d.P + kTcTile - 1) / kTcTile;
    if (nd <= 0 || n_ch <= 0) return cudaSuccess;
    return d.n_tv > 0 ? launch_pre_cherry<true>(d, o0, nd, n_ch, n_pt, s) : launch_pre_cherry<false>(d, o0, nd, n_ch, n_pt, s);
}

}  // namespace pg
