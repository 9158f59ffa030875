// la_dual_certificate: exact integer LP duals (u, v) for an optimal
// assignment, in cost units.
//
// Given a perfect matching M (row x -> column M(x)), the duals of the
// assignment LP that are tight on M are the potentials v with
//   v(y) <= v(M(x)) + C[x][y] - C[x][M(x)]   for every row x and column y,
// u(x) = C[x][M(x)] - v(M(x)); they exist iff M is optimal (no negative
// cycle). This returns the largest such potential with v <= 0: the
// shortest-path distances from a virtual source joined to every column by a
// zero arc, computed by Bellman-Ford sweeps over the columns (each sweep is
// one coalesced pass over C). Values only decrease, so sweeps may read
// values written during the same sweep. With them, u(x) + v(y) <= C[x][y]
// everywhere, with equality on M, and sum u + sum v = cost(M): a certificate
// of optimality that needs no solver to check.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>

#include "la.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kColThreads = 256;
constexpr int kRowsPerBlock = 512;

// base(x) = v(M(x)) - C[x][M(x)]; also checks that M is a permutation.
__global__ void k_dual_base(const int32_t *__restrict__ C, int n, const int32_t *__restrict__ match,
                            const long long *__restrict__ v, long long *__restrict__ base, int *__restrict__ seen,
                            int *__restrict__ bad, int check) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int y = match[x];
    if (y < 0 || y >= n) {
        atomicExch(bad, 1);
        base[x] = 0;
        return;
    }
    if (check && atomicAdd(seen + y, 1) != 0) atomicExch(bad, 1);
    base[x] = v[y] - (long long)C[(size_t)x * n + y];
}

// v(y) <- min(v(y), min over a block of rows x of C[x][y] + base(x)).
__global__ void __launch_bounds__(kColThreads)
k_dual_sweep(const int32_t *__restrict__ C, int n, const long long *__restrict__ base, long long *__restrict__ v,
             int *__restrict__ changed) {
    __shared__ long long sb[kRowsPerBlock];
    const int y = blockIdx.x * kColThreads + threadIdx.x;
    const int x0 = blockIdx.y * kRowsPerBlock;
    const int x1 = min(n, x0 + kRowsPerBlock);
    for (int k = threadIdx.x; k < x1 - x0; k += kColThreads) sb[k] = base[x0 + k];
    __syncthreads();
    if (y >= n) return;
    long long best = LLONG_MAX;
    for (int x = x0; x < x1; ++x) {
        const long long c = (long long)C[(size_t)x * n + y] + sb[x - x0];
        best = c < best ? c : best;
    }
    const long long cur = v[y];
    if (best < cur) {
        atomicMin(v + y, best);
        *changed = 1;
    }
}

__global__ void k_dual_u(const int32_t *__restrict__ C, int n, const int32_t *__restrict__ match,
                         const long long *__restrict__ v, long long *__restrict__ u) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= n) return;
    const int y = match[x];
    u[x] = (long long)C[(size_t)x * n + y] - v[y];
}

struct DualWs {
    int cap = 0;
    long long *base = nullptr;
    int *seen = nullptr;
    int *flags = nullptr;     // [0] changed, [1] bad
    int *h_flags = nullptr;
};

std::mutex g_dmu;
DualWs g_dws[kMaxDevices];

}  // namespace

#define LA_DCK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) return LA_ERR_CUDA; \
    } while (0)

extern "C" la_status la_dual_certificate(const int32_t *cost, int32_t n, const int32_t *match, void *stream,
                                         int64_t *u_out, int64_t *v_out) {
    if (n < 0 || n > LA_MAX_N || (n > 0 && (!cost || !match || !v_out))) return LA_ERR_INVALID;
    if (n == 0) return LA_OK;
    std::lock_guard<std::mutex> lock(g_dmu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    LA_DCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LA_ERR_INVALID;
    DualWs &w = g_dws[dev];
    if (!w.h_flags) {
        LA_DCK(cudaMallocHost(&w.h_flags, 2 * sizeof(int)));
        LA_DCK(cudaMalloc(&w.flags, 2 * sizeof(int)));
    }
    if (w.cap < n) {
        cudaFree(w.base);
        cudaFree(w.seen);
        w.base = nullptr;
        w.seen = nullptr;
        w.cap = 0;
        if (cudaMalloc(&w.base, sizeof(long long) * n) != cudaSuccess) return LA_ERR_NOMEM;
        if (cudaMalloc(&w.seen, sizeof(int) * n) != cudaSuccess) return LA_ERR_NOMEM;
        w.cap = n;
    }
    long long *v = reinterpret_cast<long long *>(v_out);
    LA_DCK(cudaMemsetAsync(v, 0, sizeof(long long) * n, s));
    LA_DCK(cudaMemsetAsync(w.seen, 0, sizeof(int) * n, s));
    LA_DCK(cudaMemsetAsync(w.flags, 0, 2 * sizeof(int), s));
    const int tb = 256, gb = (n + tb - 1) / tb;
    const dim3 sweep_grid((n + kColThreads - 1) / kColThreads, (n + kRowsPerBlock - 1) / kRowsPerBlock);
    // shortest paths have at most n arcs: n + 1 quiet-or-not sweeps suffice
    for (int it = 0; it <= n + 1; ++it) {
        k_dual_base<<<gb, tb, 0, s>>>(cost, n, match, v, w.base, w.seen, w.flags + 1, it == 0);
        LA_DCK(cudaMemsetAsync(w.flags, 0, sizeof(int), s));
        k_dual_sweep<<<sweep_grid, kColThreads, 0, s>>>(cost, n, w.base, v, w.flags);
        LA_DCK(cudaGetLastError());
        LA_DCK(cudaMemcpyAsync(w.h_flags, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        LA_DCK(cudaStreamSynchronize(s));
        if (w.h_flags[1]) return LA_ERR_INVALID;         // not a permutation
        if (!w.h_flags[0]) {
            if (u_out) {
                k_dual_u<<<gb, tb, 0, s>>>(cost, n, match, v, reinterpret_cast<long long *>(u_out));
                LA_DCK(cudaGetLastError());
                LA_DCK(cudaStreamSynchronize(s));
            }
            return LA_OK;
        }
    }
    return LA_ERR_INTERNAL;   // still falling after n + 2 sweeps: M is not optimal
}
