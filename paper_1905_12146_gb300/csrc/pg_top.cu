// The top part of the tree (levels >= cut, the root, and their pre-order steps) of a single FP32
// problem, with every partial kept in shared memory.
//
// Near the root the levels hold a handful of nodes, so each level is a short dependent step and the
// cost of a level is its latency.  Here a block owns a contiguous range of patterns and keeps, for
// that range, the post- and pre-order partials of every top node and the post-order partials of the
// boundary nodes (internal children of top nodes below the cut, prefetched once with cp.async) in
// shared memory.  Between two levels there is only a block barrier; the only global traffic is the
// boundary prefetch, the tip codes, the pre-order vectors of boundary nodes (read next by the
// pre-order level kernels) and the per-site values.  The arithmetic is that of the fused kernel
// (pg_nt.cu): Section 2.3 post-order update, Section 2.4 pre-order step with the Section 2.5
// gradient and Section 2.6 Hessian diagonal.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

constexpr size_t kTopSmemLimit = 227 * 1024;

// partial rows and scales of top and boundary nodes, site values, the top ops and codes, and the
// tip codes of the top nodes' tip children (at most n_top + 1 of them)
__host__ __device__ size_t top_bytes(int n_top, int n_bnd, int C, int L) {
    const size_t tabs = (size_t)n_top * 2 * (C * kPtabCols + 4) * 16;   // child-branch tables and Q columns
    const size_t rows = tabs + (size_t)(2 * n_top + n_bnd) * L * (16 * C + 4) + (size_t)L * 12;
    const size_t meta = (size_t)n_top * (sizeof(int4) + sizeof(int2)) + (size_t)(n_bnd + n_top + 1) * sizeof(int);
    const size_t tipc = (size_t)(n_top + 1) * ((L + 15) / 16 * 16);
    return rows + meta + tipc + 64;
}

__device__ __forceinline__ void cols_from_smem(const float4 *p, float4 (&c)[4]) {   // load_cols for shared memory
#pragma unroll
    for (int t = 0; t < 4; ++t) c[t] = p[t];
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}

template <int C, bool HESS>
__global__ void __launch_bounds__(kBlock, 2) top_kernel(const __grid_constant__ BatchArgs<1> a) {
    extern __shared__ float4 dyn[];
    const ProbDesc &d = a.d[0];
    const int N = d.n_tips, Ps = d.Ps, L = d.range_len;
    const int tile = blockIdx.x;
    const int p0 = tile * L, cnt = min(L, d.P - p0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    const int pieces = d.pieces, slot0 = tile * pieces;
    const int n_top = d.n_top, n_bnd = d.n_bnd;
    const int o_cut = d.level_off[d.cut];
    // shared layout: the top nodes' child-branch tables [node][side][C][kPtabCols], float4 rows
    // [node][C][L], then int scales [node][L], then site values [L]
    float4 *Tt = dyn;                                   // tables (each read many times per level)
    float4 *Qs = Tt + (size_t)n_top * 2 * C * kPtabCols; // [node][side][4] Q columns of the child's model
    float4 *Pt = Qs + (size_t)n_top * 2 * 4;            // post partials of top nodes
    float4 *Qt = Pt + (size_t)n_top * C * L;            // pre partials of top nodes
    float4 *Bt = Qt + (size_t)n_top * C * L;            // post partials of boundary nodes
    int *EP = reinterpret_cast<int *>(Bt + (size_t)n_bnd * C * L);
    int *EQ = EP + (size_t)n_top * L;
    int *EB = EQ + (size_t)n_top * L;
    float *invL = reinterpret_cast<float *>(EB + (size_t)n_bnd * L);
    int *Er = reinterpret_cast<int *>(invL + L);
    float *wv = reinterpret_cast<float *>(Er + L);
    int4 *ops_s = reinterpret_cast<int4 *>(reinterpret_cast<uintptr_t>(wv + L + 3) & ~(uintptr_t)15);
    int2 *code_s = reinterpret_cast<int2 *>(ops_s + n_top);
    int *bnd_s = reinterpret_cast<int *>(code_s + n_top);            // boundary node ids
    int *lvo_s = bnd_s + n_bnd;                                      // level offsets from the cut
    const int n_lv = d.n_levels - d.cut;                             // (at most n_top levels)
    uint8_t *tips_s = reinterpret_cast<uint8_t *>(lvo_s + n_lv + 1); // [n_top + 1][L16]
    const int L16 = (L + 15) / 16 * 16;
    const float4 *post_g = static_cast<const float4 *>(d.post);
    float4 *pre_g = static_cast<float4 *>(d.pre);

    // What does not depend on the previous kernels (the tree, the tip codes, the models' Q
    // columns) is loaded while the last post-order level drains; then the tables of this
    // evaluation and the boundary nodes' rows.
    for (int t = threadIdx.x; t < n_top; t += blockDim.x) {
        ops_s[t] = __ldg(d.ops + o_cut + t);
        code_s[t] = __ldg(d.top_code + t);
    }
    for (int t = threadIdx.x; t < n_bnd; t += blockDim.x) bnd_s[t] = __ldg(d.bnd_node + t);
    for (int t = threadIdx.x; t <= n_lv; t += blockDim.x) lvo_s[t] = __ldg(d.level_off + d.cut + t);
    __syncthreads();
    // tip codes of the top nodes' tip children (code -1 - slot)
    for (int t = threadIdx.x; t < n_top * 2 * cnt; t += blockDim.x) {
        const int nb = t / cnt, q = t - nb * cnt;
        const int4 op = ops_s[nb >> 1];
        const int2 code = code_s[nb >> 1];
        const int cc = (nb & 1) ? code.y : code.x, c = (nb & 1) ? op.z : op.y;
        if (cc < 0) tips_s[(size_t)(-1 - cc) * L16 + q] = min((int)__ldg(d.tips + (size_t)c * Ps + p0 + q), 4);
    }
    for (int t = threadIdx.x; t < n_top * 2 * 4; t += blockDim.x) {   // Q columns of each child branch's model
        const int nb = t >> 2, col = t & 3;
        const int4 op = ops_s[nb >> 1];
        const int c = (nb & 1) ? op.z : op.y;
        Qs[t] = __ldg(d.Qf + 4 * (d.bmodel ? __ldg(d.bmodel + c) : 0) + col);
    }
    // The tables of this evaluation.  Every post-order level lets its successor start only after its
    // own wait, so when this kernel runs behind a post-order level, every launch before that level
    // (the P build among them) has completed and the tables can be copied before the wait; not
    // when the P build itself precedes this kernel (no level kernels: cut = 0).
    auto copy_tables = [&]() {   // (the copies' node ids come from shared memory)
        for (int t = threadIdx.x; t < n_top * 2 * C * kPtabCols; t += blockDim.x) {
            const int per = C * kPtabCols, nb = t / per, e = t - nb * per;
            const int4 op = ops_s[nb >> 1];
            cp_async16(Tt + (size_t)nb * per + e, d.Ptab + (size_t)((nb & 1) ? op.z : op.y) * per + e);
        }
    };
    const bool tables_early = d.cut > 0 || (d.skip & kSkipPost);
    if (tables_early) copy_tables();
    pdl_wait();                // the last post-order level has completed and its rows are visible
    pdl_launch_dependents();   // a programmatic successor (a forward part's reduction) may be scheduled
    if (!tables_early) copy_tables();

    // boundary nodes' post-order rows and scales
    for (int idx = threadIdx.x; idx < n_bnd * C * cnt; idx += blockDim.x) {
        const int bl = idx / cnt, q = idx - bl * cnt, b = bl / C, l = bl - b * C;
        cp_async16(Bt + (size_t)bl * L + q, post_g + ((size_t)(bnd_s[b] - N) * C + l) * Ps + p0 + q);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int idx = threadIdx.x; idx < n_bnd * cnt; idx += blockDim.x) {
        const int b = idx / cnt, q = idx - b * cnt;
        EB[b * L + q] = __ldcg(d.pe + (size_t)(bnd_s[b] - N) * Ps + p0 + q);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();

    // post-order, levels cut .. top (Section 2.3); the last level is the root alone
    for (int lv = d.cut; lv < d.n_levels; ++lv) {
        const int o0 = lvo_s[lv - d.cut], npairs = (lvo_s[lv - d.cut + 1] - o0) * cnt;
        for (int chunk = warp; chunk * 32 < npairs; chunk += W) {
            const int j = chunk * 32 + lane;
            const bool active = j < npairs;
            const int jj = active ? j : npairs - 1;
            const int u = jj / cnt, q = jj - u * cnt, p = p0 + q;
            const int ti = o0 + u - o_cut;
            const int4 op = ops_s[ti];
            const int2 code = code_s[ti];
            const int k = op.x;
            const bool root = (k == d.root);
            const float r = pattern_factor((uint32_t)p);
            int E = 0;
            float4 v[C];
            float mx = 0.f;
            double Lsite = 0.0;
#pragma unroll
            for (int l = 0; l < C; ++l) {
                float4 x[2], sm[2];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    const int cc = side ? code.y : code.x;
                    const float4 *T = Tt + ((size_t)(2 * ti + side) * C + l) * kPtabCols;
                    sm[side] = f4(0.f, 0.f, 0.f, 0.f);
                    if (cc < 0) {
                        const int y = tips_s[(size_t)(-1 - cc) * L16 + q];
                        const float4 hi = T[y], lo = T[kColPlo + y];
                        x[side] = f4(fmaf(hi.x, r, lo.x * r), fmaf(hi.y, r, lo.y * r), fmaf(hi.z, r, lo.z * r),
                                     fmaf(hi.w, r, lo.w * r));
                    } else {
                        x[side] = cc < n_top ? Pt[((size_t)cc * C + l) * L + q] : Bt[((size_t)(cc - n_top) * C + l) * L + q];
                        sm[side] = matvec_hilo_v(T + kColDhi, T + kColDlo, x[side]);
                        if (l == 0) E += cc < n_top ? EP[cc * L + q] : EB[(cc - n_top) * L + q];
                    }
                }
                v[l] = f4(prod_split(x[0].x, sm[0].x, x[1].x, sm[1].x), prod_split(x[0].y, sm[0].y, x[1].y, sm[1].y),
                          prod_split(x[0].z, sm[0].z, x[1].z, sm[1].z), prod_split(x[0].w, sm[0].w, x[1].w, sm[1].w));
                if (root) {   // the root's products rounded once in FP32, as every node's; their sums in FP64
                    double s = d.pi[0] * (double)v[l].x;
                    s = fma(d.pi[1], (double)v[l].y, s);
                    s = fma(d.pi[2], (double)v[l].z, s);
                    s = fma(d.pi[3], (double)v[l].w, s);
                    Lsite = fma(d.cw[l], s, Lsite);
                } else {
                    mx = fmaxf(mx, hmax(v[l]));
                }
            }
            if (!root) {
                if (active) {
                    const int e = scale_exponent(mx);
#pragma unroll
                    for (int l = 0; l < C; ++l) Pt[((size_t)ti * C + l) * L + q] = scale4(v[l], e);
                    EP[ti * L + q] = E + e;
                }
                continue;
            }
            // the site likelihood (Section 2.3 root inner product, Section 2.5 mixture).  This GPU
            // issues FP64 at a small fraction of the FP32 rate and the root level is bound by its FP64
            // work per SM, so the exponent split and the stored reciprocal avoid FP64 instructions.
            int e2 = 0;
            const double f = split_exponent(Lsite, e2);
            const int Erq = E + e2;
            const double wgt = d.weights[p];
            const double lp = log(f) + (double)Erq * 0.69314718055994530942 -
                              (d.rlog ? d.rlog[p] : (double)N * log((double)r));
            const float rf = __frcp_rn((float)f);   // 1 / Lhat_p for the FP32 branch terms
            if (active) {
                invL[q] = rf;
                Er[q] = Erq;
                wv[q] = (float)wgt;
            }
            if (d.skip & kSkipPost) continue;   // recomputed for the pre-order only
            if (active) {
                d.site_invL[p] = rf;
                d.site_Er[p] = Erq;
                if (!(f > 0.0) || !isfinite(lp)) atomicOr(d.status, kStatusNumeric);
                if (d.out_site) d.out_site[p] = lp;
            }
            segment_sums(u, active, (active && wgt != 0.0) ? wgt * lp : 0.0, chunk, cnt, pieces,
                         [&](int, int pc, double s) { d.lpart[slot0 + pc] = s; });
        }
        __syncthreads();
    }

    if (d.skip & kSkipPre) return;
    // pre-order, top .. cut (Section 2.4) with the gradient (2.5) and Hessian diagonal (2.6)
    for (int lv = d.n_levels - 1; lv >= d.cut; --lv) {
        const int o0 = lvo_s[lv - d.cut], npairs = (lvo_s[lv - d.cut + 1] - o0) * cnt;
        for (int chunk = warp; chunk * 32 < npairs; chunk += W) {
            const int j = chunk * 32 + lane;
            const bool active = j < npairs;
            const int jj = active ? j : npairs - 1;
            const int u = jj / cnt, q = jj - u * cnt, p = p0 + q;
            const int ti = o0 + u - o_cut;
            const int4 op = ops_s[ti];
            const int2 code = code_s[ti];
            const bool root = (op.x == d.root);
            const float r = pattern_factor((uint32_t)p);
            const int Eq = root ? 0 : EQ[ti * L + q];
            int Ec[2] = {0, 0}, y[2] = {0, 0};
            float4 aa[2][C];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int cc = side ? code.y : code.x;
                if (cc < 0) y[side] = tips_s[(size_t)(-1 - cc) * L16 + q];
                else Ec[side] = cc < n_top ? EP[cc * L + q] : EB[(cc - n_top) * L + q];
#pragma unroll
                for (int l = 0; l < C; ++l) {
                    const float4 *T = Tt + ((size_t)(2 * ti + side) * C + l) * kPtabCols;
                    if (cc < 0) {
                        aa[side][l] = scal(T[y[side]], r);
                    } else {
                        const float4 xv = cc < n_top ? Pt[((size_t)cc * C + l) * L + q]
                                                     : Bt[((size_t)(cc - n_top) * C + l) * L + q];
                        float4 H[4];
                        cols_from_smem(T, H);
                        aa[side][l] = matvec(H, xv);
                    }
                }
            }
            float dg[2], dh[2];
            const float inv = invL[q], wt = active ? wv[q] : 0.f;
            const int dE = Eq + Ec[0] + Ec[1] - Er[q];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const int c = side ? op.z : op.y, cc = side ? code.y : code.x;
                float4 Qc[4];
                cols_from_smem(Qs + (size_t)(2 * ti + side) * 4, Qc);
                float4 qv[C];
                float mq = 0.f, gs = 0.f, hs = 0.f;
#pragma unroll
                for (int l = 0; l < C; ++l) {
                    const float4 qk = root ? f4(d.pif[0], d.pif[1], d.pif[2], d.pif[3]) : Qt[((size_t)ti * C + l) * L + q];
                    const float4 qt = mul(qk, aa[1 - side][l]);   // top of branch c
                    const float4 uu = matvec(Qc, aa[side][l]);
                    gs = fmaf(d.gw[l], dot(qt, uu), gs);
                    if (HESS) hs = fmaf(d.gw2[l], dot(qt, matvec(Qc, uu)), hs);
                    if (cc >= 0) {
                        float4 H[4];
                        cols_from_smem(Tt + ((size_t)(2 * ti + side) * C + l) * kPtabCols, H);
                        qv[l] = matvec_t(H, qt);
                        mq = fmaxf(mq, hmax(qv[l]));
                    }
                }
                if (cc >= 0 && active) {
                    const int e = scale_exponent(mq);
                    const int eq_c = Eq + Ec[1 - side] + e;
                    if (cc < n_top) {
#pragma unroll
                        for (int l = 0; l < C; ++l) Qt[((size_t)cc * C + l) * L + q] = scale4(qv[l], e);
                        EQ[cc * L + q] = eq_c;
                    } else {   // a boundary node: its pre-order vector goes on to the level kernels
#pragma unroll
                        for (int l = 0; l < C; ++l) __stcg(pre_g + ((size_t)(c - N) * C + l) * Ps + p, scale4(qv[l], e));
                        __stcg(d.qe + (size_t)(c - N) * Ps + p, eq_c);
                    }
                }
                const float dd = ldexp2f(gs, dE) * inv;
                dg[side] = wt != 0.f ? wt * dd : 0.f;
                dh[side] = (HESS && wt != 0.f) ? wt * (ldexp2f(hs, dE) * inv - dd * dd) : 0.f;
            }
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                segment_sums_f(u, active, dg[s], chunk, cnt, pieces, [&](int us, int pc, double v) {
                    const int4 o = ops_s[o0 + us - o_cut];
                    d.gpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
                });
                if (HESS)
                    segment_sums_f(u, active, dh[s], chunk, cnt, pieces, [&](int us, int pc, double v) {
                        const int4 o = ops_s[o0 + us - o_cut];
                        d.hpart[(size_t)(s ? o.z : o.y) * d.slot_cap + slot0 + pc] = v;
                    });
            }
        }
        __syncthreads();
    }
}

template <int C, bool HESS>
cudaError_t launch_top_c(const BatchArgs<1> &args, size_t smem, cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(top_kernel<C, HESS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTopSmemLimit); }); e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch (the kernel waits in pdl_wait)
    cfg.gridDim = dim3((unsigned)args.d[0].n_tiles);
    cfg.blockDim = dim3(kBlock);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, top_kernel<C, HESS>, args);
}

}  // namespace

size_t top_smem_bytes(const ProbDesc &d) { return top_bytes(d.n_top, d.n_bnd, d.C, d.range_len); }

cudaError_t launch_top(const BatchArgs<1> &args, bool hess, int, cudaStream_t s) {
    const ProbDesc &d = args.d[0];
    if (d.n_tiles <= 0) return cudaSuccess;
    const size_t smem = top_smem_bytes(d);
    if (smem > kTopSmemLimit) return cudaErrorNotSupported;
    switch (d.C * 2 + (hess ? 1 : 0)) {
        case 2: return launch_top_c<1, false>(args, smem, s);
        case 3: return launch_top_c<1, true>(args, smem, s);
        case 4: return launch_top_c<2, false>(args, smem, s);
        case 5: return launch_top_c<2, true>(args, smem, s);
        case 6: return launch_top_c<3, false>(args, smem, s);
        case 7: return launch_top_c<3, true>(args, smem, s);
        case 8: return launch_top_c<4, false>(args, smem, s);
        case 9: return launch_top_c<4, true>(args, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pg
