// Device helpers shared by the nucleotide kernels (pg_nt.cu, pg_levels.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pg {
namespace dev {

__device__ __forceinline__ float4 f4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ float4 mul(float4 a, float4 b) { return f4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }
__device__ __forceinline__ float4 scal(float4 a, float s) { return f4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float dot(float4 a, float4 b) { return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x))); }
__device__ __forceinline__ float hmax(float4 a) { return fmaxf(fmaxf(a.x, a.y), fmaxf(a.z, a.w)); }
__device__ __forceinline__ float4 fma4(float4 col, float s, float4 acc) {
    return f4(fmaf(col.x, s, acc.x), fmaf(col.y, s, acc.y), fmaf(col.z, s, acc.z), fmaf(col.w, s, acc.w));
}

// y = M v with M given by its four columns
__device__ __forceinline__ float4 matvec(const float4 (&col)[4], float4 v) {
    float4 a = scal(col[0], v.x);
    a = fma4(col[1], v.y, a);
    a = fma4(col[2], v.z, a);
    return fma4(col[3], v.w, a);
}
// y = M' v with M given by its four columns
__device__ __forceinline__ float4 matvec_t(const float4 (&col)[4], float4 v) {
    return f4(dot(col[0], v), dot(col[1], v), dot(col[2], v), dot(col[3], v));
}
// y = (Mhi + Mlo) v, the small half first
__device__ __forceinline__ float4 matvec_hilo(const float4 *hi, const float4 *lo, float4 v) {
    float4 a = scal(__ldg(lo), v.x);
    a = fma4(__ldg(lo + 1), v.y, a);
    a = fma4(__ldg(lo + 2), v.z, a);
    a = fma4(__ldg(lo + 3), v.w, a);
    a = fma4(__ldg(hi), v.x, a);
    a = fma4(__ldg(hi + 1), v.y, a);
    a = fma4(__ldg(hi + 2), v.z, a);
    return fma4(__ldg(hi + 3), v.w, a);
}

// y = (Mhi + Mlo) v from register/shared copies of the columns, the small half first
__device__ __forceinline__ float4 matvec_hilo_v(const float4 *hi, const float4 *lo, float4 v) {
    float4 a = scal(lo[0], v.x);
    a = fma4(lo[1], v.y, a);
    a = fma4(lo[2], v.z, a);
    a = fma4(lo[3], v.w, a);
    a = fma4(hi[0], v.x, a);
    a = fma4(hi[1], v.y, a);
    a = fma4(hi[2], v.z, a);
    return fma4(hi[3], v.w, a);
}
__device__ __forceinline__ float4 matvec_p(const float4 *col, float4 v) {
    float4 a = scal(col[0], v.x);
    a = fma4(col[1], v.y, a);
    a = fma4(col[2], v.z, a);
    return fma4(col[3], v.w, a);
}
__device__ __forceinline__ float4 matvec_tp(const float4 *col, float4 v) {
    return f4(dot(col[0], v), dot(col[1], v), dot(col[2], v), dot(col[3], v));
}

__device__ __forceinline__ void load_cols(const float4 *p, float4 (&c)[4]) {
#pragma unroll
    for (int t = 0; t < 4; ++t) c[t] = __ldg(p + t);
}

// (x0 + s0)(x1 + s1) rounded once: exact product x0*x1 (value + FMA residual) plus cross terms
__device__ __forceinline__ float prod_split(float x0, float s0, float x1, float s1) {
    const float h = x0 * x1;
    const float res = fmaf(x0, x1, -h);
    const float small = fmaf(s0, x1 + s1, x0 * s1);
    return h + (res + small);
}

// Pattern-specific factor in [1, 2): lowbias32 integer hash (C. Wellons) of the pattern index
// as a 23-bit mantissa.
__device__ __forceinline__ float pattern_factor(uint32_t p) {
    uint32_t x = p + 0x9E3779B9u;
    x ^= x >> 16; x *= 0x21F0AAADu;
    x ^= x >> 15; x *= 0x735A2D97u;
    x ^= x >> 15;
    return __uint_as_float(0x3F800000u | (x >> 9));
}

// e such that mx * 2^-e lies in [1, 2) (0 for zero / non-finite, which are left as they are)
__device__ __forceinline__ int scale_exponent(float mx) {
    int bits = __float_as_int(mx);
    int e = ((bits >> 23) & 0xff) - 127;
    if (e == -127) {
        if (mx == 0.0f) return 0;
        int ee;
        frexpf(mx, &ee);
        return ee - 1;
    }
    if (e == 128) return 0;
    return e;
}
__device__ __forceinline__ int scale_exponent64(double mx) {
    if (!(mx > 0.0) || isinf(mx)) return 0;
    int e;
    frexp(mx, &e);
    return e - 1;
}

// f in [0.5, 1) and e with x = f 2^e for a positive normal x, from the bit pattern (integer
// instructions only); frexp's result otherwise (zero, subnormal, infinite, NaN: x itself, e = 0,
// unless subnormal)
__device__ __forceinline__ double split_exponent(double x, int &e) {
    const long long b = __double_as_longlong(x);
    const int eb = (int)((b >> 52) & 0x7ff);
    if (b > 0 && eb != 0 && eb != 0x7ff) {
        e = eb - 1022;
        return __longlong_as_double((b & ~(0x7ffLL << 52)) | (1022LL << 52));
    }
    e = 0;
    if (b > 0 && eb == 0) return frexp(x, &e);
    return x;
}

__device__ __forceinline__ float pow2f(int e) {   // 2^e, e in [-126, 127]
    return __int_as_float((e + 127) << 23);
}
// x * 2^e in FP32 arithmetic: a multiplication by an exact power of two for e in [-126, 127]
// (exact for a normal result, one rounding for a subnormal one, as ldexpf), ldexpf beyond
__device__ __forceinline__ float ldexp2f(float x, int e) {
    if (e >= -126 && e <= 127) return x * pow2f(e);
    return ldexpf(x, e);
}
__device__ __forceinline__ float4 scale4(float4 v, int e) {   // v * 2^-e exactly
    if (e >= -126 && e <= 126) return scal(v, pow2f(-e));
    return f4(ldexpf(v.x, -e), ldexpf(v.y, -e), ldexpf(v.z, -e), ldexpf(v.w, -e));
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Adds v over the lanes of each node segment of this warp and hands (node, piece, sum) to
// emit on lane 0; also zero-fills the slots a node does not use (by its first chunk's warp).
template <class Emit>
__device__ __forceinline__ void segment_sums(int u, bool active, double v, int chunk, int cnt,
                                             int pieces, Emit &&emit) {
    const int lane = threadIdx.x & 31;
    const int u_lo = __shfl_sync(0xffffffffu, u, 0), u_hi = __shfl_sync(0xffffffffu, u, 31);
    for (int us = u_lo; us <= u_hi; ++us) {
        const double s = warp_sum((active && u == us) ? v : 0.0);
        const int first = (us * cnt) >> 5, last = ((us + 1) * cnt - 1) >> 5;
        if (lane == 0) {
            emit(us, chunk - first, s);
            if (chunk == first)
                for (int pc = last - first + 1; pc < pieces; ++pc) emit(us, pc, 0.0);
        }
    }
}

// segment_sums with an FP32 warp reduction (32 FP32 terms), handed on as FP64
template <class Emit>
__device__ __forceinline__ void segment_sums_f(int u, bool active, float v, int chunk, int cnt, int pieces,
                                               Emit &&emit) {
    const int lane = threadIdx.x & 31;
    const int u_lo = __shfl_sync(0xffffffffu, u, 0), u_hi = __shfl_sync(0xffffffffu, u, 31);
    for (int us = u_lo; us <= u_hi; ++us) {
        const float s = warp_sum_f((active && u == us) ? v : 0.f);
        const int first = (us * cnt) >> 5, last = ((us + 1) * cnt - 1) >> 5;
        if (lane == 0) {
            emit(us, chunk - first, (double)s);
            if (chunk == first)
                for (int pc = last - first + 1; pc < pieces; ++pc) emit(us, pc, 0.0);
        }
    }
}

// ---- programmatic dependent launch --------------------------------------------------------------
// Let the next kernel in the stream be scheduled now (its blocks still wait in pdl_wait), and wait
// until the previous kernel has completed with its memory visible.  Both are no-ops for a kernel
// launched without the programmatic-serialisation attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

// ---- shared-memory barriers and 1-D bulk (TMA) copies ------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
// one arrival that also announces `bytes` of transactions for the current phase
__device__ __forceinline__ void mbar_arrive_expect(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte aligned), completing
// on bar's transaction count
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// a plain arrival (no transactions)
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for phase `parity` of bar for at most ~limit_cycles SM clocks; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit_cycles) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit_cycles) return false;
    return true;
}

}  // namespace dev
}  // namespace pg
