// Tensor-core kernels of the general-state path (2..64 states): the products P x, G x, H x of the
// post-order (Section 2.3) and pre-order (Section 2.4) passes and P^T q of the pre-order, as
// Y[p][s] = sum_k X[p][k] W[s][k] on tcgen05 (kind::tf32, FP32 accumulation in tensor memory).
// With P = I + D only D x and D^T q go through the tensor core; the identity part (x, q) is added
// in FP32 by the threads.  The tensor core's accumulation truncates, and P x sums positive terms
// only, so keeping the O(1) identity out of it keeps that bias to the size of D x.
//
// One item is a tile of kTcTile = 128 patterns (the MMA's M) of one node.  Pattern row t is TMEM
// lane t of every accumulator.  A 128-thread block gives row t to thread t.  The 256-thread
// pre-order kernel gives it to two threads, one per half of the states; they combine their partial
// maxima and sums through shared memory.
//
// Operand tiles [128 x 64] FP32 and tables [64 x 64] arrive by TMA with 128-byte swizzling (the
// canonical K-major layout).  A tip child's rows are written by the threads as the tips' partial
// vectors (one-hot, all-ones, or a partially observed tip's row), so tips and internal children
// share the product.
//
// Each product runs three TF32 passes, hi x hi + hi x lo + lo x hi.  The tensor core truncates an
// FP32 operand to its TF32 part (hi); lo = x - trunc(x) is formed by the threads for the rows
// (in shared or tensor memory) and stored with the tables.  This gives about FP32 accuracy (error
// ~2^-21 relative per term).  Results leave through a swizzled staging tile and a TMA store;
// exponents go out with plain stores.
//
// Every wait is bounded (kWaitLimitCycles); a block that gives up records PG_ERR_TIMEOUT, lets its
// copies land, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pg_device.cuh"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

constexpr int kTcThreads = 128;
constexpr uint32_t kRowTile = kTcTile * kMP * 4;   // 32 KB: one [128 x 64] FP32 tile
constexpr uint32_t kRowKB = kTcTile * 128;         // 16 KB: its 32-state half (one K block)
constexpr uint32_t kTab = kMP * kMP * 4;           // 16 KB: one [64 x 64] table
constexpr uint32_t kTabKB = kMP * 128;             // 8 KB: its 32-state half

// ---- PTX wrappers ----------------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// instruction descriptor: kind::tf32, FP32 accumulator, both operands K-major, M x N
__device__ __forceinline__ uint32_t idesc_tf32(uint32_t M, uint32_t N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}
// acc (+)= A[128 x 64] * B[n x 64]^T in 8 steps of K = 8 (two 32-state K blocks of 4 steps)
__device__ __forceinline__ void mma_tile(uint32_t acc, uint32_t a, uint32_t b, uint32_t n, bool accumulate) {
    const uint32_t id = idesc_tf32(kTcTile, n);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
        mma_tf32(acc, umma_desc(a + kb * kRowKB + ko), umma_desc(b + kb * n * 128 + ko), id,
                 (accumulate || kk > 0) ? 1u : 0u);
    }
}
// the same with A[128 x 64] read from tensor memory (lane = row, one column per element)
__device__ __forceinline__ void mma_tile_ta(uint32_t acc, uint32_t a_tmem, uint32_t b, uint32_t n, bool accumulate) {
    const uint32_t id = idesc_tf32(kTcTile, n);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t kb = kk >> 2, ko = (kk & 3) * 32;
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n"
                     ::"r"(acc), "r"(a_tmem + (uint32_t)(kk * 8)), "l"(umma_desc(b + kb * n * 128 + ko)), "r"(id),
                       "r"((accumulate || kk > 0) ? 1u : 0u));
    }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float v[16]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                   "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                   "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                   "r"(__float_as_uint(v[15]))
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *m, int x, int y, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *m, int x, int y, int z, uint64_t *bar) {
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
                 ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *m, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n"
                 ::"l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }

// byte offset of 16-byte chunk cc (states 4 cc .. 4 cc + 3) of row r of a swizzled tile of `rows`
// rows: two 32-state K blocks, rows 128 bytes apart, chunk index XOR (row mod 8)
__device__ __forceinline__ uint32_t sw(int r, int cc, int rows) {
    return (uint32_t)((cc >> 3) * rows * 128 + r * 128 + (((cc & 7) ^ (r & 7)) << 4));
}
__device__ __forceinline__ float tf32_lo(float x) { return x - __uint_as_float(__float_as_uint(x) & 0xffffe000u); }
__device__ __forceinline__ float4 lo4(float4 v) { return f4(tf32_lo(v.x), tf32_lo(v.y), tf32_lo(v.z), tf32_lo(v.w)); }

__device__ __forceinline__ unsigned char *align1024(unsigned char *p) {
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// state s of the partial vector of tip code y (Section 2.1): the indicator of state y, the row of a
// partially observed tip, or all ones over the m states (missing data); 0 for y < 0 (no pattern)
__device__ __forceinline__ float tip_value(const MDesc &d, int y, int s) {
    if (y < 0) return 0.f;
    if (y < d.m) return s == y ? 1.f : 0.f;
    if (y < d.m + d.n_tv) return __ldg(d.tipv + (size_t)(y - d.m) * kMP + s);
    return s < d.m ? 1.f : 0.f;
}

// the partial vector of the tip code of row t of a tip child, zero past cnt.  Indicator and
// all-ones rows are exact in TF32; rows of partially observed tips (TV: the problem has tip
// vectors) need the remainder pass.
template <bool TV>
__device__ __forceinline__ void tip_row(unsigned char *X, const MDesc &d, int c, int p0, int cnt, int t) {
    const int y = t < cnt ? (int)__ldg(d.tips + (size_t)c * d.Ps + p0 + t) : -1;
    const bool amb = y >= d.m;
#pragma unroll
    for (int cc = 0; cc < kMP / 4; ++cc) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = 4 * cc + j;
            if constexpr (TV) v[j] = tip_value(d, y, s);
            else v[j] = (y >= 0 && (amb ? s < d.m : s == y)) ? 1.f : 0.f;
        }
        *reinterpret_cast<float4 *>(X + sw(t, cc, kTcTile)) = f4(v[0], v[1], v[2], v[3]);
    }
}
// the TF32 remainders of row t of a loaded tile
__device__ __forceinline__ void lo_row(const unsigned char *X, unsigned char *XL, int t) {
#pragma unroll
    for (int cc = 0; cc < kMP / 4; ++cc)
        *reinterpret_cast<float4 *>(XL + sw(t, cc, kTcTile)) = lo4(*reinterpret_cast<const float4 *>(X + sw(t, cc, kTcTile)));
}
// a table (tables consecutive kinds k0 .. k0 + nk - 1 of (c, l), each 64 rows) into a swizzled
// [64 nk x 64] operand at dst
__device__ __forceinline__ void load_tables(unsigned char *dst, const CUtensorMap *tm, const MDesc &d, int c, int l,
                                            int k0, int nk, uint64_t *bar) {
    const int row0 = ((c * d.C + l) * kTcKinds + k0) * kMP;
    for (int kb = 0; kb < 2; ++kb)
        for (int j = 0; j < nk; ++j)
            tma_load_2d(dst + kb * nk * kTabKB + j * kTabKB, tm, kb * 32, row0 + j * kMP, bar);
}

// every thread waits for the barrier's current phase; the phase advances only if all saw it
__device__ __forceinline__ bool wait_all(uint64_t *bar, uint32_t &phase) {
    const bool ok = __syncthreads_and(mbar_wait_bounded(bar, phase, kWaitLimitCycles)) != 0;
    if (ok) phase ^= 1u;
    return ok;
}
// After a wait gave up (called by the thread that issued every copy and product): let the products
// finish, tracked afresh by a new barrier and a commit of every tensor-core operation this thread
// issued (complete whatever phase the earlier barriers were in), and the copies behind the pending
// load barriers land; each wait bounded.  Returns false if something was still outstanding.  The
// block releases its tensor memory in either case: a block that left holding it would make every
// later allocation on that SM wait forever.  A false return is recorded as kStatusUnsettled.
__device__ __forceinline__ bool drain_block(uint64_t *fresh, uint64_t *loads, const uint32_t *ph, const bool *pend,
                                            int n_loads) {
    mbar_init(fresh, 1);
    mma_commit(fresh);
    bool ok = mbar_wait_bounded(fresh, 0u, kWaitLimitCycles);
    for (int i = 0; i < n_loads; ++i)
        if (pend[i]) ok = mbar_wait_bounded(&loads[i], ph[i], kWaitLimitCycles) && ok;
    return ok;
}

// row t of a tile (states 16 ch .. 16 ch + 15) from a swizzled [128 x 64] tile
__device__ __forceinline__ void row16(const unsigned char *X, int t, int ch, float v[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float4 x = *reinterpret_cast<const float4 *>(X + sw(t, ch * 4 + q, kTcTile));
        v[4 * q] = x.x;
        v[4 * q + 1] = x.y;
        v[4 * q + 2] = x.z;
        v[4 * q + 3] = x.w;
    }
}
__device__ __forceinline__ void put16(unsigned char *X, int t, int ch, const float v[16], int e) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4 *>(X + sw(t, ch * 4 + q, kTcTile)) =
            scale4(f4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]), e);
}

// q_c = qt + (D^T qt) for row t: the accumulator at ta plus the row of qt in X, scaled into
// [1, 2) by its largest state and written to the staging tile (which may be X itself)
__device__ __forceinline__ int store_sum_scaled(uint32_t ta, const unsigned char *X, unsigned char *stage, int t) {
    float mx = 0.f;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        float a[16], x[16];
        tmem_ld16(ta + ch * 16, a);
        row16(X, t, ch, x);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) mx = fmaxf(mx, a[j] + x[j]);
    }
    const int e = scale_exponent(mx);
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        float a[16], x[16];
        tmem_ld16(ta + ch * 16, a);
        row16(X, t, ch, x);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j) a[j] += x[j];
        put16(stage, t, ch, a, e);
    }
    return e;
}

// ---- post-order level: item = (node, category, 128-pattern tile), three blocks per SM ----------------------
// Per child: its D hi | D lo tables and rows (or tip rows) into shared memory, the rows'
// TF32 remainders into tensor memory (columns 64 .. 127), D x into columns 0 .. 63 by three passes;
// the first child's x + D x is kept in registers.  The result is scaled by its largest state,
// written over the rows and stored by TMA.  64 KB of shared memory and 128 TMEM columns per block.
template <bool TV>
__global__ void __launch_bounds__(kTcThreads, 3)
m_post_tc_kernel(const __grid_constant__ MDesc d, const __grid_constant__ CUtensorMap tm_post,
                 const __grid_constant__ CUtensorMap tm_tab, int o0, int n_pt) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *sm = align1024(tc_raw);
    unsigned char *XA = sm, *TB = sm + kRowTile;   // rows (then the result), D hi | D lo
    __shared__ __align__(8) uint64_t bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    const int C = d.C, N = d.n_tips, t = threadIdx.x, warp = t >> 5;
    const int per_node = C * n_pt;
    const int u = blockIdx.x / per_node, rem = blockIdx.x - u * per_node, l = rem / n_pt, pt = rem - l * n_pt;
    const int4 op = __ldg(d.ops + o0 + u);
    const int k = op.x, p0 = pt * kTcTile, cnt = min(kTcTile, d.P - p0);
    if (warp == 0) tmem_alloc(&tmem_slot, 128);
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot, lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t ph_load = 0, ph_mma = 0;
    bool ok = true, load_pending = false, mma_pending = false;
    int E = 0;
    float a0[kMP];   // x + D x of the first child
    for (int side = 0; side < 2 && ok; ++side) {
        const int c = side ? op.z : op.y;
        const bool tip = c < N;
        if (t == 0) {
            mbar_arrive_expect(&bar[0], 2 * kTab + (tip ? 0u : kRowTile));
            load_tables(TB, &tm_tab, d, c, l, kTcD, 1, &bar[0]);
            load_tables(TB + kTab, &tm_tab, d, c, l, kTcDlo, 1, &bar[0]);
        }
        // Launched with programmatic stream serialisation: the first child's tables (complete before
        // the first tensor-core post-order level, which follows the cherry level's completion) go out
        // before the wait; the rows and scales that earlier levels wrote after it.
        if (side == 0) {
            pdl_wait();
            // the next level may be scheduled only now, after this wait (at the kernel's start it
            // measured 3.071 against 3.055 ms per codon evaluation); its copies of rows wait for it
            pdl_launch_dependents();
        }
        if (t == 0 && !tip)
            for (int kb = 0; kb < 2; ++kb) tma_load_3d(XA + kb * kRowKB, &tm_post, kb * 32, p0, (c - N) * C + l, &bar[0]);
        // TF32 remainders: of internal rows, and of tip rows when some tip vectors are not exact
        const bool lo_pass = !tip || TV;
        if (tip) tip_row<TV>(XA, d, c, p0, cnt, t);
        else if (t < cnt) E += __ldcg(d.pe + ((size_t)(c - N) * C + l) * d.Ps + p0 + t);
        load_pending = true;
        ok = wait_all(&bar[0], ph_load);
        load_pending = !ok;
        if (!ok) break;
        if (lo_pass) {
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                float x[16];
                row16(XA, t, ch, x);
#pragma unroll
                for (int j = 0; j < 16; ++j) x[j] = tf32_lo(x[j]);
                tmem_st16(lane_base + 64 + ch * 16, x);
            }
            tmem_wait_st();
        }
        fence_async_smem();
        tc_before();
        __syncthreads();
        if (t == 0) {
            tc_after();
            mma_tile(tmem, smem_u32(XA), smem_u32(TB), kMP, false);
            mma_tile(tmem, smem_u32(XA), smem_u32(TB + kTab), kMP, true);
            if (lo_pass) mma_tile_ta(tmem, tmem + 64, smem_u32(TB), kMP, true);
            mma_commit(&bar[1]);
        }
        mma_pending = true;
        ok = wait_all(&bar[1], ph_mma);
        mma_pending = !ok;
        if (ok && side == 0) {   // keep x + D x of the first child before its rows are replaced
            tc_after();
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                float a[16], x[16];
                tmem_ld16(lane_base + ch * 16, a);
                row16(XA, t, ch, x);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) a0[16 * ch + j] = a[j] + x[j];
            }
            tc_before();
            __syncthreads();   // every row and accumulator read before the next child's copies and products
        }
    }
    if (ok) {
        tc_after();
        float mx = 0.f;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            float a[16], x[16];
            tmem_ld16(lane_base + ch * 16, a);
            row16(XA, t, ch, x);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                a0[16 * ch + j] *= a[j] + x[j];
                mx = fmaxf(mx, a0[16 * ch + j]);
            }
        }
        const int e = scale_exponent(mx);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) put16(XA, t, ch, a0 + 16 * ch, e);   // the row's own slots
        if (t < cnt) __stcg(d.pe + ((size_t)(k - N) * C + l) * d.Ps + p0 + t, E + e);
        fence_async_smem();
        __syncthreads();
        if (t == 0) {
            for (int kb = 0; kb < 2; ++kb) tma_store_3d(&tm_post, XA + kb * kRowKB, kb * 32, p0, (k - N) * C + l);
            bulk_commit();
            bulk_wait_read0();
        }
    } else if (t == 0) {
        atomicOr(d.status, kStatusTimeout);
        if (!drain_block(&drain_bar, &bar[0], &ph_load, &load_pending, 1)) atomicOr(d.status, kStatusUnsettled);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

// ---- pre-order level with the gradient: item = (node, 128-pattern tile), categories in turn -------------
// Per category: A_c = x_c [D_c; G_c]^T (TMEM columns 128 side .. +127: D_c x_c | u_c = G_c x_c),
// a_c = x_c + D_c x_c,
// optionally H_c x_c (columns 256 + 64 side); qt_c = q_k o a_other (q_root = pi), the branch terms
// qt_c . u_c (and qt_c . H_c x_c) 2^{E} / L_p; for an internal child q_c = P_c^T qt_c (columns
// 128 side .. +63 again: D_c^T qt_c, plus qt_c) scaled and stored.
template <bool HESS, bool TV>
__global__ void __launch_bounds__(kTcThreads, 1)
m_pre_tc_kernel(const __grid_constant__ MDesc d, const __grid_constant__ CUtensorMap tm_post,
                const __grid_constant__ CUtensorMap tm_pre, const __grid_constant__ CUtensorMap tm_tab, int o0, int n_pt) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char *sm = align1024(tc_raw);
    unsigned char *X[2] = {sm, sm + 2 * kRowTile};            // rows (hi) then remainders (lo) per child
    unsigned char *TB = sm + 4 * kRowTile;                     // tables: up to [128 x 64] hi | lo
    unsigned char *QK = sm + 4 * kRowTile + 2 * 2 * kTab;      // q_k rows
    __shared__ __align__(8) uint64_t bar[2], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ double red[2][2][kTcThreads / 32];
    constexpr uint32_t kCols = HESS ? 512 : 256;
    const int C = d.C, N = d.n_tips, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int u = blockIdx.x / n_pt, pt = blockIdx.x - u * n_pt;
    const int4 op = __ldg(d.ops + o0 + u);
    const int k = op.x, p0 = pt * kTcTile, cnt = min(kTcTile, d.P - p0);
    const bool root = k == d.root;
    const int cs[2] = {op.y, op.z};
    const bool tip[2] = {op.y < N, op.z < N};
    if (warp == 0) tmem_alloc(&tmem_slot, kCols);
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
    }
    tc_before();
    __syncthreads();
    tc_after();
    const uint32_t tmem = tmem_slot, lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    const bool on = t < cnt;
    const float inv = on ? __ldcg(d.site_invL + p0 + t) : 0.f;
    const int Er = on ? __ldcg(d.site_Er + p0 + t) : 0;
    float dsum[2] = {0.f, 0.f}, hsum[2] = {0.f, 0.f};
    uint32_t ph_load = 0, ph_mma = 0;
    bool ok = true, load_pending = false, mma_pending = false;
    for (int l = 0; l < C && ok; ++l) {
        const int Eq = (on && !root) ? __ldcg(d.qe + ((size_t)(k - N) * C + l) * d.Ps + p0 + t) : 0;
        int Ex[2];
        for (int side = 0; side < 2; ++side)
            Ex[side] = (on && !tip[side]) ? __ldcg(d.pe + ((size_t)(cs[side] - N) * C + l) * d.Ps + p0 + t) : 0;
        // rows of q_k and both children, [P; G] of child 0
        if (t == 0) {
            uint32_t bytes = 4 * kTab;
            if (!root) bytes += kRowTile;
            for (int side = 0; side < 2; ++side) bytes += tip[side] ? 0u : kRowTile;
            mbar_arrive_expect(&bar[0], bytes);
            if (!root)
                for (int kb = 0; kb < 2; ++kb) tma_load_3d(QK + kb * kRowKB, &tm_pre, kb * 32, p0, (k - N) * C + l, &bar[0]);
            for (int side = 0; side < 2; ++side)
                if (!tip[side])
                    for (int kb = 0; kb < 2; ++kb)
                        tma_load_3d(X[side] + kb * kRowKB, &tm_post, kb * 32, p0, (cs[side] - N) * C + l, &bar[0]);
            load_tables(TB, &tm_tab, d, cs[0], l, kTcD, 2, &bar[0]);
            load_tables(TB + 2 * kTab, &tm_tab, d, cs[0], l, kTcDlo, 2, &bar[0]);
        }
        for (int side = 0; side < 2; ++side)
            if (tip[side]) tip_row<TV>(X[side], d, cs[side], p0, cnt, t);
        load_pending = true;
        ok = wait_all(&bar[0], ph_load);
        load_pending = !ok;
        if (!ok) break;
        for (int side = 0; side < 2; ++side)
            if (!tip[side] || TV) lo_row(X[side], X[side] + kRowTile, t);
        fence_async_smem();
        // the products of both children: [P; G] (then H) tables of child `side`
        for (int side = 0; side < 2 && ok; ++side) {
            for (int pass = 0; pass < (HESS ? 2 : 1) && ok; ++pass) {
                if (side > 0 || pass > 0) {   // the next tables, once the previous products have read TB
                    if (t == 0) {
                        mbar_arrive_expect(&bar[0], pass ? 2 * kTab : 4 * kTab);
                        if (pass) {
                            load_tables(TB, &tm_tab, d, cs[side], l, kTcH, 1, &bar[0]);
                            load_tables(TB + kTab, &tm_tab, d, cs[side], l, kTcHlo, 1, &bar[0]);
                        } else {
                            load_tables(TB, &tm_tab, d, cs[side], l, kTcD, 2, &bar[0]);
                            load_tables(TB + 2 * kTab, &tm_tab, d, cs[side], l, kTcDlo, 2, &bar[0]);
                        }
                    }
                    load_pending = true;
        ok = wait_all(&bar[0], ph_load);
        load_pending = !ok;
                    if (!ok) break;
                }
                tc_before();
                __syncthreads();
                if (t == 0) {
                    tc_after();
                    const uint32_t n = pass ? kMP : 2 * kMP;
                    const uint32_t acc = tmem + (pass ? 256 + 64 * side : 128 * side);
                    const uint32_t xa = smem_u32(X[side]), xl = xa + kRowTile, tb = smem_u32(TB);
                    const uint32_t tl = tb + n * kMP * 4;
                    mma_tile(acc, xa, tb, n, false);
                    mma_tile(acc, xa, tl, n, true);
                    if (!tip[side] || TV) mma_tile(acc, xl, tb, n, true);
                    mma_commit(&bar[1]);
                }
                mma_pending = true;
        ok = wait_all(&bar[1], ph_mma);
        mma_pending = !ok;
            }
        }
        if (!ok) break;
        // qt_c = q_k o a_other, the branch terms, and qt of internal children as MMA operands
        tc_after();
        float dot[2] = {0.f, 0.f}, hdot[2] = {0.f, 0.f};
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {
            float a0[16], u0[16], a1[16], u1[16], x0[16], x1[16];
            tmem_ld16(lane_base + ch * 16, a0);
            tmem_ld16(lane_base + 64 + ch * 16, u0);
            tmem_ld16(lane_base + 128 + ch * 16, a1);
            tmem_ld16(lane_base + 192 + ch * 16, u1);
            row16(X[0], t, ch, x0);
            row16(X[1], t, ch, x1);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {   // P x = x + D x
                a0[j] += x0[j];
                a1[j] += x1[j];
            }
            float qk[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = root ? f4(d.pif[16 * ch + 4 * q], d.pif[16 * ch + 4 * q + 1], d.pif[16 * ch + 4 * q + 2],
                                           d.pif[16 * ch + 4 * q + 3])
                                      : *reinterpret_cast<const float4 *>(QK + sw(t, ch * 4 + q, kTcTile));
                qk[4 * q] = v.x;
                qk[4 * q + 1] = v.y;
                qk[4 * q + 2] = v.z;
                qk[4 * q + 3] = v.w;
            }
            float q0[16], q1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                q0[j] = qk[j] * a1[j];
                q1[j] = qk[j] * a0[j];
                dot[0] = fmaf(q0[j], u0[j], dot[0]);
                dot[1] = fmaf(q1[j], u1[j], dot[1]);
            }
            if (HESS) {
                float h0[16], h1[16];
                tmem_ld16(lane_base + 256 + ch * 16, h0);
                tmem_ld16(lane_base + 320 + ch * 16, h1);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    hdot[0] = fmaf(q0[j], h0[j], hdot[0]);
                    hdot[1] = fmaf(q1[j], h1[j], hdot[1]);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v0 = f4(q0[4 * q], q0[4 * q + 1], q0[4 * q + 2], q0[4 * q + 3]);
                const float4 v1 = f4(q1[4 * q], q1[4 * q + 1], q1[4 * q + 2], q1[4 * q + 3]);
                if (!tip[0]) {
                    *reinterpret_cast<float4 *>(X[0] + sw(t, ch * 4 + q, kTcTile)) = v0;
                    *reinterpret_cast<float4 *>(X[0] + kRowTile + sw(t, ch * 4 + q, kTcTile)) = lo4(v0);
                }
                if (!tip[1]) {
                    *reinterpret_cast<float4 *>(X[1] + sw(t, ch * 4 + q, kTcTile)) = v1;
                    *reinterpret_cast<float4 *>(X[1] + kRowTile + sw(t, ch * 4 + q, kTcTile)) = lo4(v1);
                }
            }
        }
        {
            const int dE = Eq + Ex[0] + Ex[1] - Er;   // the same for both child branches
            const float cw = (float)d.cw[l];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                dsum[side] += cw * ldexp2f(dot[side], dE) * inv;
                if (HESS) hsum[side] += cw * ldexp2f(hdot[side], dE) * inv;
            }
        }
        fence_async_smem();
        // q_c = P_c^T qt_c for the internal children, staged through QK (side 0) or X[0] (side 1)
        for (int side = 0; side < 2 && ok; ++side) {
            if (tip[side]) continue;
            const int c = cs[side];
            if (t == 0) {
                mbar_arrive_expect(&bar[0], 2 * kTab);
                load_tables(TB, &tm_tab, d, c, l, kTcDT, 1, &bar[0]);
                load_tables(TB + kTab, &tm_tab, d, c, l, kTcDTlo, 1, &bar[0]);
            }
            tc_before();
            load_pending = true;
        ok = wait_all(&bar[0], ph_load);
        load_pending = !ok;
            if (!ok) break;
            if (t == 0) {
                tc_after();
                const uint32_t acc = tmem + 128 * side;
                const uint32_t xa = smem_u32(X[side]), xl = xa + kRowTile, tb = smem_u32(TB);
                mma_tile(acc, xa, tb, kMP, false);
                mma_tile(acc, xa, tb + kTab, kMP, true);
                mma_tile(acc, xl, tb, kMP, true);
                mma_commit(&bar[1]);
            }
            mma_pending = true;
        ok = wait_all(&bar[1], ph_mma);
        mma_pending = !ok;
            if (!ok) break;
            tc_after();
            unsigned char *stage = side ? X[0] : QK;
            const int e = store_sum_scaled(lane_base + 128 * side, X[side], stage, t);
            if (on) __stcg(d.qe + ((size_t)(c - N) * C + l) * d.Ps + p0 + t, Eq + Ex[1 - side] + e);
            fence_async_smem();
            __syncthreads();
            if (t == 0) {
                for (int kb = 0; kb < 2; ++kb) tma_store_3d(&tm_pre, stage + kb * kRowKB, kb * 32, p0, (c - N) * C + l);
                bulk_commit();
                bulk_wait_read0();   // the staging tile is read before the next category's copies
            }
            __syncthreads();
        }
    }
    if (ok) {
        // per child branch: sum over the tile's patterns of w_p d_p and w_p (h_p - d_p^2)
        const double w = on ? d.weights[p0 + t] : 0.0;
        for (int side = 0; side < 2; ++side) {
            double g = w != 0.0 ? w * (double)dsum[side] : 0.0;
            double h = (HESS && w != 0.0) ? w * ((double)hsum[side] - (double)dsum[side] * (double)dsum[side]) : 0.0;
            g = warp_sum(g);
            h = warp_sum(h);
            if (lane == 0) {
                red[side][0][warp] = g;
                red[side][1][warp] = h;
            }
        }
        __syncthreads();
        if (t < 2) {
            double g = 0.0, h = 0.0;
            for (int j = 0; j < kTcThreads / 32; ++j) {
                g += red[t][0][j];
                h += red[t][1][j];
            }
            d.gpart[(size_t)cs[t] * d.n_gslots + pt] = g;
            if (HESS) d.hpart[(size_t)cs[t] * d.n_gslots + pt] = h;
            for (int j = 1; j < C; ++j) {   // one category group: the other slots stay zero
                d.gpart[(size_t)cs[t] * d.n_gslots + j * n_pt + pt] = 0.0;
                if (HESS) d.hpart[(size_t)cs[t] * d.n_gslots + j * n_pt + pt] = 0.0;
            }
        }
    } else if (t == 0) {
        atomicOr(d.status, kStatusTimeout);
        if (!drain_block(&drain_bar, &bar[0], &ph_load, &load_pending, 1)) atomicOr(d.status, kStatusUnsettled);
    }
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---- pre-order level without the Hessian: loads of the next category overlap this one ----------------
// Tensor memory holds, per category, A_c = x_c [D_c; G_c]^T (columns 128 c .. +127) and the
// children's rows as MMA A operands: x_c (256 + 128 c .. +63) and its TF32 remainder (+64 .. +127);
// the shared-memory row slots are only staging for TMA, so the next category's rows are copied
// into them while this category's products and epilogues run.  Per category: rows -> TMEM,
// products with both children's [D; G] tables, the epilogue forms qt_c = q_k o (x_other +
// D_other x_other) and the branch terms and writes qt_c (and remainder) over x_c in tensor memory,
// the D_c^T tables arrive meanwhile, the products D_c^T qt_c (columns 128 c .. +63 again) give
// q_c = qt_c + D_c^T qt_c, stored straight from registers.  Tip children's rows (their partial
// vectors) are written into tensor memory by the threads.
template <bool TV>
__global__ void __launch_bounds__(2 * kTcThreads, 1)
m_pre_tc2_kernel(const __grid_constant__ MDesc d, const __grid_constant__ CUtensorMap tm_post,
                 const __grid_constant__ CUtensorMap tm_pre, const __grid_constant__ CUtensorMap tm_tab, int o0, int n_pt,
                 int n_cg) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    if (smem_u32(tc_raw) & 1023u) {   // the layout needs a 1024-byte aligned base (see kPre2TcSmem)
        if (threadIdx.x == 0) atomicOr(d.status, kStatusTimeout);
        return;
    }
    unsigned char *sm = tc_raw;
    unsigned char *X[2] = {sm, sm + kRowTile};                 // children's rows (staging)
    unsigned char *QK = sm + 2 * kRowTile;                      // q_k rows
    // per child 64 KB: [D; G] hi in the lower half (then D^T hi | lo), [D; G] lo in the upper half
    // (then the staged result q_c)
    unsigned char *T[2] = {sm + 3 * kRowTile, sm + 3 * kRowTile + 4 * kTab};
    enum { BX = 0, BQ = 1, BTH = 2, BTL = 3, BD = 4, BM = 5, NB = 6 };   // rows, q_k, [D;G] hi, lo, D^T, products
    __shared__ __align__(8) uint64_t bar[NB], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ double red[2][kTcThreads / 32];
    __shared__ float half_part[2][2][kTcTile];   // per child, per half of the states, per row
    // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its quadrant) = rows t, and half w / 4
    // of the 64 states (chunks 2 hf, 2 hf + 1)
    const int C = d.C, N = d.n_tips, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int hf = warp >> 2, t = 32 * (warp & 3) + lane, ch0 = 2 * hf;
    // item = (node, category group, tile): group g takes categories l0 .. l1 - 1
    const int u = blockIdx.x / (n_cg * n_pt), rg = blockIdx.x - u * (n_cg * n_pt), g = rg / n_pt, pt = rg - g * n_pt;
    const int G = (C + n_cg - 1) / n_cg, l0 = g * G, l1 = min(C, l0 + G);
    const int4 op = __ldg(d.ops + o0 + u);
    const int k = op.x, p0 = pt * kTcTile, cnt = min(kTcTile, d.P - p0);
    const bool root = k == d.root;
    const int cs[2] = {op.y, op.z};
    const bool tip[2] = {op.y < N, op.z < N};
    const bool any_int = !tip[0] || !tip[1];
    if (warp == 0) tmem_alloc(&tmem_slot, 512);
    if (threadIdx.x == 0)
        for (int i = 0; i < NB; ++i) mbar_init(&bar[i], 1);
    tc_before();
    __syncthreads();
    tc_after();
    const bool leader = threadIdx.x == 0;   // issues every copy and product
    const uint32_t tmem = tmem_slot, lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const bool on = t < cnt;
    const float inv = on ? __ldcg(d.site_invL + p0 + t) : 0.f;
    const int Er = on ? __ldcg(d.site_Er + p0 + t) : 0;
    float dsum[2] = {0.f, 0.f};
    uint32_t ph[NB] = {0, 0, 0, 0, 0, 0};
    bool pend[NB] = {false, false, false, false, false, false};
    bool ok = true;
    bool store_pending = false;   // (leader) results of the previous category still being read from the upper halves
    // copies (thread 0): rows of the internal children, q_k, tables
    auto issue_rows = [&](int l) {
        uint32_t bytes = 0;
        for (int side = 0; side < 2; ++side) bytes += tip[side] ? 0u : kRowTile;
        if (!bytes) return;
        pend[BX] = true;
        mbar_arrive_expect(&bar[BX], bytes);
        for (int side = 0; side < 2; ++side)
            if (!tip[side])
                for (int kb = 0; kb < 2; ++kb)
                    tma_load_3d(X[side] + kb * kRowKB, &tm_post, kb * 32, p0, (cs[side] - N) * C + l, &bar[BX]);
    };
    auto issue_qk = [&](int l) {
        pend[BQ] = true;
        mbar_arrive_expect(&bar[BQ], kRowTile);
        for (int kb = 0; kb < 2; ++kb) tma_load_3d(QK + kb * kRowKB, &tm_pre, kb * 32, p0, (k - N) * C + l, &bar[BQ]);
    };
    auto issue_tables_hi = [&](int l) {   // [D; G] hi into the lower halves
        pend[BTH] = true;
        mbar_arrive_expect(&bar[BTH], 4 * kTab);
        for (int side = 0; side < 2; ++side) load_tables(T[side], &tm_tab, d, cs[side], l, kTcD, 2, &bar[BTH]);
    };
    auto issue_tables_lo = [&](int l) {   // [D; G] lo into the upper halves
        pend[BTL] = true;
        mbar_arrive_expect(&bar[BTL], 4 * kTab);
        for (int side = 0; side < 2; ++side)
            load_tables(T[side] + 2 * kTab, &tm_tab, d, cs[side], l, kTcDlo, 2, &bar[BTL]);
    };
    auto wait = [&](int i) {   // all threads, one phase of barrier i
        ok = wait_all(&bar[i], ph[i]);
        if (ok) pend[i] = false;
        return ok;
    };
    // Launched with programmatic stream serialisation: the copies that do not depend on the previous
    // pre-order level (the children's rows and tables, the per-site values of the root kernel: the
    // first pre-order level follows the root kernel's completion, and each later one starts after
    // its predecessor started) go out before the wait; q_k and its scales after it.
    if (leader) {
        issue_rows(l0);
        issue_tables_hi(l0);
        issue_tables_lo(l0);
    }
    pdl_wait();   // the previous level's q rows are complete and visible
    pdl_launch_dependents();   // the next level may be scheduled (after this wait: 3.071 -> 3.068 ms)
    if (leader && !root) issue_qk(l0);
    for (int l = l0; l < l1 && ok; ++l) {
        const int Eq = (on && !root) ? __ldcg(d.qe + ((size_t)(k - N) * C + l) * d.Ps + p0 + t) : 0;
        int Ex[2];
        for (int side = 0; side < 2; ++side)
            Ex[side] = (on && !tip[side]) ? __ldcg(d.pe + ((size_t)(cs[side] - N) * C + l) * d.Ps + p0 + t) : 0;
        // the children's rows (and remainders) into tensor memory
        if (any_int && !wait(BX)) break;
        for (int side = 0; side < 2; ++side) {
            const uint32_t xc = lane_base + 256 + 128 * side;
            if (tip[side]) {   // the tips' partial vectors
                const int y = on ? (int)__ldg(d.tips + (size_t)cs[side] * d.Ps + p0 + t) : -1;
                if constexpr (!TV) {   // one-hot or all-ones rows: exact in TF32, no remainders
#pragma unroll
                    for (int ch = ch0; ch < ch0 + 2; ++ch) {
                        float x[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int st = 16 * ch + j;
                            x[j] = (y >= 0 && (y >= d.m ? st < d.m : st == y)) ? 1.f : 0.f;
                        }
                        tmem_st16(xc + ch * 16, x);
                    }
                } else {   // rows of partially observed tips may not be: remainders too
#pragma unroll 1
                    for (int ch = ch0; ch < ch0 + 2; ++ch) {
                        float x[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) x[j] = tip_value(d, y, 16 * ch + j);
                        tmem_st16(xc + ch * 16, x);
#pragma unroll
                        for (int j = 0; j < 16; ++j) x[j] = tf32_lo(x[j]);
                        tmem_st16(xc + 64 + ch * 16, x);
                    }
                }
                continue;
            }
#pragma unroll
            for (int ch = ch0; ch < ch0 + 2; ++ch) {
                float x[16];
                row16(X[side], t, ch, x);
                tmem_st16(xc + ch * 16, x);
#pragma unroll
                for (int j = 0; j < 16; ++j) x[j] = tf32_lo(x[j]);
                tmem_st16(xc + 64 + ch * 16, x);
            }
        }
        tmem_wait_st();
        tc_before();
        __syncthreads();   // rows read: the slots may take the next category's rows
        if (leader && l + 1 < l1) issue_rows(l + 1);
        // the passes with the hi tables first (hi x hi, lo x hi); the lo tables may still be landing
        if (!wait(BTH)) break;
        if (leader) {
            tc_after();
            for (int side = 0; side < 2; ++side) {
                const uint32_t acc = tmem + 128 * side, xa = tmem + 256 + 128 * side, tb = smem_u32(T[side]);
                mma_tile_ta(acc, xa, tb, 2 * kMP, false);
                if (!tip[side] || TV) mma_tile_ta(acc, xa + 64, tb, 2 * kMP, true);
            }
            // while those run: the previous results leave the upper halves, this category's lo
            // tables take their place
            if (l > l0) {
                if (store_pending) bulk_wait_read0();
                store_pending = false;
                issue_tables_lo(l);
            }
        }
        if (!wait(BTL)) break;
        if (leader) {
            tc_after();
            for (int side = 0; side < 2; ++side) {
                const uint32_t acc = tmem + 128 * side, xa = tmem + 256 + 128 * side, tb = smem_u32(T[side]);
                mma_tile_ta(acc, xa, tb + 2 * kTab, 2 * kMP, true);
            }
            pend[BM] = true;
            mma_commit(&bar[BM]);
        }
        if (!wait(BM)) break;
        if (leader && !any_int && l + 1 < l1) issue_tables_hi(l + 1);   // no D^T products: the lower halves are free
        // the D^T tables of the internal children into their (now free) table slots
        if (leader && any_int) {
            pend[BD] = true;
            mbar_arrive_expect(&bar[BD], (tip[0] ? 0u : 2 * kTab) + (tip[1] ? 0u : 2 * kTab));
            for (int side = 0; side < 2; ++side) {
                if (tip[side]) continue;
                load_tables(T[side], &tm_tab, d, cs[side], l, kTcDT, 1, &bar[BD]);
                load_tables(T[side] + kTab, &tm_tab, d, cs[side], l, kTcDTlo, 1, &bar[BD]);
            }
        }
        if (!root && !wait(BQ)) break;
        // epilogue 1: qt, the branch terms; qt of internal children over their rows in TMEM
        tc_after();
        float dot[2] = {0.f, 0.f};
#pragma unroll 1
        for (int ch = ch0; ch < ch0 + 2; ++ch) {
            float a0[16], u0[16], a1[16], u1[16], x0[16], x1[16], qk[16];
            tmem_ld16(lane_base + ch * 16, a0);
            tmem_ld16(lane_base + 64 + ch * 16, u0);
            tmem_ld16(lane_base + 128 + ch * 16, a1);
            tmem_ld16(lane_base + 192 + ch * 16, u1);
            tmem_ld16(lane_base + 256 + ch * 16, x0);
            tmem_ld16(lane_base + 384 + ch * 16, x1);
            if (root) {
#pragma unroll
                for (int j = 0; j < 16; ++j) qk[j] = d.pif[16 * ch + j];
            } else {
                row16(QK, t, ch, qk);
            }
            tmem_wait_ld();
            float q0[16], q1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                q0[j] = qk[j] * (a1[j] + x1[j]);   // top of branch c0: q_k o P_1 x_1
                q1[j] = qk[j] * (a0[j] + x0[j]);
                dot[0] = fmaf(q0[j], u0[j], dot[0]);
                dot[1] = fmaf(q1[j], u1[j], dot[1]);
            }
            if (!tip[0]) {
                tmem_st16(lane_base + 256 + ch * 16, q0);
#pragma unroll
                for (int j = 0; j < 16; ++j) q0[j] = tf32_lo(q0[j]);
                tmem_st16(lane_base + 320 + ch * 16, q0);
            }
            if (!tip[1]) {
                tmem_st16(lane_base + 384 + ch * 16, q1);
#pragma unroll
                for (int j = 0; j < 16; ++j) q1[j] = tf32_lo(q1[j]);
                tmem_st16(lane_base + 448 + ch * 16, q1);
            }
        }
        tmem_wait_st();
        half_part[0][hf][t] = dot[0];
        half_part[1][hf][t] = dot[1];
        tc_before();
        __syncthreads();   // q_k read: its slot may take the next category's
        {
            const int dE = Eq + Ex[0] + Ex[1] - Er;
            const float cw = (float)d.cw[l];
            for (int side = 0; side < 2; ++side)
                dsum[side] += cw * ldexp2f(half_part[side][0][t] + half_part[side][1][t], dE) * inv;
        }
        if (leader && !root && l + 1 < l1) issue_qk(l + 1);
        if (any_int) {
            if (!wait(BD)) break;
            if (leader) {
                tc_after();
                for (int side = 0; side < 2; ++side) {
                    if (tip[side]) continue;
                    const uint32_t acc = tmem + 128 * side, qa = tmem + 256 + 128 * side;
                    const uint32_t tb = smem_u32(T[side]);
                    mma_tile_ta(acc, qa, tb, kMP, false);
                    mma_tile_ta(acc, qa, tb + kTab, kMP, true);
                    mma_tile_ta(acc, qa + 64, tb, kMP, true);
                }
                pend[BM] = true;
                mma_commit(&bar[BM]);
            }
            if (!wait(BM)) break;
            if (leader && l + 1 < l1) issue_tables_hi(l + 1);   // the D^T tables have been read
        }
        if (any_int) {
            // epilogue 2: q_c = qt_c + D_c^T qt_c, scaled, staged in the upper half of the child's
            // table slot and stored by TMA
            tc_after();
            for (int side = 0; side < 2; ++side) {
                if (tip[side]) continue;
                const uint32_t qa = lane_base + 256 + 128 * side, acc = lane_base + 128 * side;
                float v[2][16];   // this half's 32 states of q_c, kept in registers
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float q[16];
                    tmem_ld16(acc + (ch0 + i) * 16, v[i]);
                    tmem_ld16(qa + (ch0 + i) * 16, q);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[i][j] += q[j];
                }
                float mx = 0.f;
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 16; ++j) mx = fmaxf(mx, v[i][j]);
                half_part[side][hf][t] = mx;
            }
            __syncthreads();   // both halves' maxima
            for (int side = 0; side < 2; ++side) {
                if (tip[side]) continue;
                const uint32_t qa = lane_base + 256 + 128 * side, acc = lane_base + 128 * side;
                const int e = scale_exponent(fmaxf(half_part[side][0][t], half_part[side][1][t]));
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    float a[16], q[16];
                    tmem_ld16(acc + (ch0 + i) * 16, a);
                    tmem_ld16(qa + (ch0 + i) * 16, q);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) a[j] += q[j];
                    put16(T[side] + 2 * kTab, t, ch0 + i, a, e);
                }
                if (on && hf == 0) __stcg(d.qe + ((size_t)(cs[side] - N) * C + l) * d.Ps + p0 + t, Eq + Ex[1 - side] + e);
            }
            fence_async_smem();
            __syncthreads();
            if (leader) {
                for (int side = 0; side < 2; ++side) {
                    if (tip[side]) continue;
                    for (int kb = 0; kb < 2; ++kb)
                        tma_store_3d(&tm_pre, T[side] + 2 * kTab + kb * kRowKB, kb * 32, p0, (cs[side] - N) * C + l);
                }
                bulk_commit();
                store_pending = true;   // waited for before the next lo tables are copied over them
            }
        }
        tc_before();
        __syncthreads();   // tensor memory read before the next category's rows overwrite it
    }
    if (ok) {
        const double w = (on && hf == 0) ? d.weights[p0 + t] : 0.0;   // each row once
        for (int side = 0; side < 2; ++side) {
            double gs = w != 0.0 ? w * (double)dsum[side] : 0.0;
            gs = warp_sum(gs);
            if (lane == 0 && hf == 0) red[side][warp] = gs;
        }
        __syncthreads();
        if (threadIdx.x < 2) {
            double v = 0.0;
            for (int j = 0; j < kTcThreads / 32; ++j) v += red[threadIdx.x][j];
            double *slots = d.gpart + (size_t)cs[threadIdx.x] * d.n_gslots;
            slots[g * n_pt + pt] = v;
            if (g == n_cg - 1)   // the slots of groups this launch does not have stay zero
                for (int j = n_cg; j < C; ++j) slots[j * n_pt + pt] = 0.0;
        }
    } else if (leader) {
        atomicOr(d.status, kStatusTimeout);
        // let every copy (barriers BX .. BD) and product in flight finish
        if (!drain_block(&drain_bar, bar, ph, pend, BM)) atomicOr(d.status, kStatusUnsettled);
    }
    if (leader) bulk_wait_read0();   // the staging smem is read before the block exits
    tc_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

// no alignment slack: the static shared memory is padded so that the dynamic region starts on a
// 1024-byte boundary (checked in the kernel), and rows + tables + statics fill the 227 KB limit
constexpr size_t kPre2TcSmem = 3 * kRowTile + 8 * kTab;
constexpr size_t kPostTcSmem = 1024 + kRowTile + 2 * kTab;
constexpr size_t kPreTcSmem = 1024 + 4 * kRowTile + 4 * kTab + kRowTile;

}  // namespace

namespace {

// Each kernel has two instantiations: TV = true for problems with tip vectors (rows of partially
// observed tips, with their remainder passes), TV = false with the plain one-hot / all-ones rows.
template <bool TV>
cudaError_t launch_post_tc(const MDesc &d, const void *tm_post, const void *tm_tab, int o0, int nd, int n_pt,
                           cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_post_tc_kernel<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPostTcSmem); }); e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch (the kernel waits in pdl_wait)
    cfg.gridDim = dim3((unsigned)(nd * d.C * n_pt));
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = kPostTcSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, m_post_tc_kernel<TV>, d, *static_cast<const CUtensorMap *>(tm_post),
                              *static_cast<const CUtensorMap *>(tm_tab), o0, n_pt);
}

template <bool HESS, bool TV>
cudaError_t launch_pre_tc(const MDesc &d, const void *tm_post, const void *tm_pre, const void *tm_tab, int o0, int nd,
                          int n_pt, cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_pre_tc_kernel<HESS, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPreTcSmem); }); e != cudaSuccess)
        return e;
    m_pre_tc_kernel<HESS, TV><<<nd * n_pt, kTcThreads, kPreTcSmem, s>>>(
        d, *static_cast<const CUtensorMap *>(tm_post), *static_cast<const CUtensorMap *>(tm_pre),
        *static_cast<const CUtensorMap *>(tm_tab), o0, n_pt);
    return cudaGetLastError();
}

template <bool TV>
cudaError_t launch_pre_tc2(const MDesc &d, const void *tm_post, const void *tm_pre, const void *tm_tab, int o0,
                           int nd, int n_pt, int n_cg, cudaStream_t s) {
    static DeviceOnce once;   // the shared-memory attribute, once per device
    if (cudaError_t e = device_once(once, [](int &) { return cudaFuncSetAttribute(m_pre_tc2_kernel<TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPre2TcSmem); }); e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};   // programmatic dependent launch (the kernel waits in pdl_wait)
    cfg.gridDim = dim3((unsigned)(nd * n_cg * n_pt));
    cfg.blockDim = dim3(2 * kTcThreads);
    cfg.dynamicSmemBytes = kPre2TcSmem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, m_pre_tc2_kernel<TV>, d, *static_cast<const CUtensorMap *>(tm_post),
                              *static_cast<const CUtensorMap *>(tm_pre), *static_cast<const CUtensorMap *>(tm_tab), o0,
                              n_pt, n_cg);
}

}  // namespace

cudaError_t launch_m_post_level_tc(const MDesc &d, const void *tm_post, const void *tm_tab, int o0, int nd,
                                   cudaStream_t s) {
    const int n_pt = (d.P + kTcTile - 1) / kTcTile;
    if (nd <= 0 || n_pt <= 0) return cudaSuccess;
    return d.n_tv > 0 ? launch_post_tc<true>(d, tm_post, tm_tab, o0, nd, n_pt, s)
                      : launch_post_tc<false>(d, tm_post, tm_tab, o0, nd, n_pt, s);
}

// Categories per block: all of them (the next category's loads overlap this one's work) unless the
// level has too few (node, tile) items to fill the SMs; then the categories split into the most
// groups that still run in one wave, each group in its own block.  The gradient slots are per
// (group, tile), so the result depends only on the problem and the SM count.
int pre_category_groups(int C, int items, int n_sm) {
    int best = 1;
    for (int n_cg = 2; n_cg <= C; ++n_cg) {
        const int G = (C + n_cg - 1) / n_cg;
        if ((C + G - 1) / G == n_cg && (long)items * n_cg <= n_sm) best = n_cg;   // still one wave
    }
    return best;
}

cudaError_t launch_m_pre_level_tc(const MDesc &d, const void *tm_post, const void *tm_pre, const void *tm_tab,
                                  int o0, int nd, bool hess, int n_sm, cudaStream_t s) {
    const int n_pt = (d.P + kTcTile - 1) / kTcTile;
    if (nd <= 0 || n_pt <= 0) return cudaSuccess;
    const bool tv = d.n_tv > 0;
    if (hess)
        return tv ? launch_pre_tc<true, true>(d, tm_post, tm_pre, tm_tab, o0, nd, n_pt, s)
                  : launch_pre_tc<true, false>(d, tm_post, tm_pre, tm_tab, o0, nd, n_pt, s);
    const int n_cg = pre_category_groups(d.C, nd * n_pt, n_sm);
    return tv ? launch_pre_tc2<true>(d, tm_post, tm_pre, tm_tab, o0, nd, n_pt, n_cg, s)
              : launch_pre_tc2<false>(d, tm_post, tm_pre, tm_tab, o0, nd, n_pt, n_cg, s);
}

}  // namespace pg
