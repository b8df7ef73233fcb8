// Failure detection without a GPU fault.  Every kernel of the library waits on mbarriers with an
// iteration limit: a wait that gives up records a status bit, lets its own copies land, frees its
// tensor memory and returns, and the host reports PG_ERR_TIMEOUT.  pg_selftest_timeout runs that
// same bounded wait on an mbarrier that nothing arrives at, so the time-out path can be tested on a
// real GPU: the kernel returns after about limit_cycles and the context stays usable.
#include <cuda_runtime.h>

#include <cstdint>

#include "pg_device.cuh"
#include "pg_host.h"
#include "pg_internal.cuh"

namespace pg {
namespace {

using namespace dev;

__global__ void timeout_probe_kernel(int *status, long long limit_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);   // one arrival expected; none will come
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait_bounded(&bar, 0u, limit_cycles)) atomicOr(status, kStatusTimeout);
}

}  // namespace
}  // namespace pg

extern "C" pg_status pg_selftest_timeout(pg_ctx *ctx, uint64_t limit_cycles) {
    using pg::host::fail;
    if (!ctx) return fail(PG_ERR_INVALID, "NULL context");
    if (limit_cycles < 1000 || limit_cycles > (1ull << 32))
        return fail(PG_ERR_INVALID, "limit_cycles = %llu: must be in [1000, 2^32]", (unsigned long long)limit_cycles);
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(PG_ERR_CUDA, "cannot select device %d", ctx->device);
    int *d_status = nullptr;
    if (cudaMalloc(&d_status, sizeof(int)) != cudaSuccess) return fail(PG_ERR_OOM, "cudaMalloc of 4 bytes failed");
    int st = 0;
    cudaError_t e = cudaMemset(d_status, 0, sizeof(int));
    if (e == cudaSuccess) {
        pg::timeout_probe_kernel<<<1, 32>>>(d_status, (long long)limit_cycles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&st, d_status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d_status);
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, "selftest: %s", cudaGetErrorString(e));
    if (st & pg::kStatusTimeout) return fail(PG_ERR_TIMEOUT, "the bounded wait gave up after %llu cycles, as intended",
                                             (unsigned long long)limit_cycles);
    return PG_OK;
}
