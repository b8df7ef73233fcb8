// Random-effects clock parameterisation of the branch lengths and its chain rule.
//
// Section 2.1: the length of branch i is its rate times the time elapsed along it,
// b_i = r_i (t_i - t_parent(i)), with node times t in forward time.  Section 5.1 (random-effects
// relaxed clock): r_i = mu * eps_i, a tree-wise mean mu times a branch effect eps_i.  Given
// g_i = dlogL/db_i from the pre-order pass:
//   dlogL/d eps_i = mu dt_i g_i,   dlogL/d r_i = dt_i g_i,   dlogL/d mu = sum_i eps_i dt_i g_i,
//   dlogL/d t_k   = r_k g_k - sum over children c of k of r_c g_c   (the root has no own branch).
#include <cuda_runtime.h>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kClockThreads = 256;

template <int MAXB>
__global__ void __launch_bounds__(kClockThreads) clock_lengths_kernel(const __grid_constant__ ClockArgs<MAXB> a) {
    const ClockDesc &c = a.c[blockIdx.x];
    const double mu = *c.mu;
    for (int i = threadIdx.x; i < c.n_nodes; i += blockDim.x) {
        const int pa = c.parent[i];
        c.b[i] = pa < 0 ? 0.0 : mu * c.eps[i] * (c.t[i] - c.t[pa]);
    }
}

template <int MAXB>
__global__ void __launch_bounds__(kClockThreads) clock_grad_kernel(const __grid_constant__ ClockArgs<MAXB> a) {
    __shared__ double red[kClockThreads];
    const ClockDesc &c = a.c[blockIdx.x];
    const double mu = *c.mu;
    const int N = c.n_tips;
    double part = 0.0;   // this thread's share of dlogL/d mu, nodes i = threadIdx.x + j * blockDim.x
    for (int i = threadIdx.x; i < c.n_nodes; i += blockDim.x) {
        const int pa = c.parent[i];
        const double g = pa < 0 ? 0.0 : c.g[i];
        const double dt = pa < 0 ? 0.0 : c.t[i] - c.t[pa];
        if (c.g_eps) c.g_eps[i] = mu * dt * g;
        if (c.g_rate) c.g_rate[i] = dt * g;
        if (pa >= 0) part = fma(c.eps[i] * dt, g, part);   // the root's entries are ignored
        if (c.g_t && i < N) c.g_t[i] = mu * c.eps[i] * g;   // a tip has no children
    }
    if (c.g_t) {   // an internal node: its own branch minus its two children's
        for (int j = threadIdx.x; j < N - 1; j += blockDim.x) {
            const int4 op = c.ops[j];
            const int k = op.x;
            const double own = (k == c.root) ? 0.0 : mu * c.eps[k] * c.g[k];
            c.g_t[k] = own - mu * c.eps[op.y] * c.g[op.y] - mu * c.eps[op.z] * c.g[op.z];
        }
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int w = kClockThreads / 2; w > 0; w >>= 1) {   // fixed pairing: the same sum every call
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0 && c.g_mu) *c.g_mu = red[0];
}

}  // namespace

cudaError_t launch_clock(const ClockArgs<kMaxClock> &a, bool grad, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (grad) clock_grad_kernel<kMaxClock><<<a.n, kClockThreads, 0, s>>>(a);
    else clock_lengths_kernel<kMaxClock><<<a.n, kClockThreads, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pg
