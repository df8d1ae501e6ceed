// Latency probes behind the traversal's floor (test infrastructure): the
// time of one dependent L2 round trip (a single thread chasing a random cycle
// through an L2-resident buffer) and of one thread-block-cluster barrier
// (arrive + wait, every CTA of the cluster taking part).  Times are read from
// the GPU's global timer.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// every entry read once by many threads: the buffer is then in L2
__global__ void k_touch(const int32_t *next, int n, int *sink) {
    int acc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += next[i];
    if (acc == 0x7fffffff) *sink = acc;
}

// next[] is one cycle through n entries; `steps` dependent loads are timed
// (ld.cg: served by L2, not L1)
__global__ void k_chase(const int32_t *next, int steps, unsigned long long *out) {
    int j = 0;
    const unsigned long long t0 = gtime();
    for (int i = 0; i < steps; ++i) {
        int v;
        asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(next + j));
        j = v;
    }
    const unsigned long long t1 = gtime();
    out[0] = t1 - t0;
    out[1] = (unsigned long long)j;   // keeps the chain live
}

// every CTA of the cluster runs the same number of barriers
__global__ void k_cluster_barrier(int iters, unsigned long long *out) {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    const unsigned long long t0 = gtime();
    for (int i = 0; i < iters; ++i)
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    const unsigned long long t1 = gtime();
    if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = t1 - t0;
}

}  // namespace

extern "C" int probe_l2_round_trip_ns(int n, int steps, double *ns) {
    int32_t *next = nullptr;
    unsigned long long *out = nullptr;
    if (n < 2 || steps < 1) return 1;
    if (cudaMalloc(&next, sizeof(int32_t) * (size_t)n) != cudaSuccess) return 2;
    if (cudaMalloc(&out, 2 * sizeof(unsigned long long)) != cudaSuccess) { cudaFree(next); return 2; }
    // a single cycle: i -> (i + stride) mod n with stride coprime to n and large
    int32_t *h = new int32_t[n];
    long long stride = 1000003 % n;
    if (stride == 0) stride = 1;
    for (int i = 0; i < n; ++i) h[i] = (int32_t)((i + stride) % n);
    cudaMemcpy(next, h, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
    delete[] h;
    k_touch<<<256, 256>>>(next, n, reinterpret_cast<int *>(out));
    k_chase<<<1, 1>>>(next, steps, out);
    unsigned long long r[2] = {0, 0};
    cudaError_t e = cudaMemcpy(r, out, sizeof(r), cudaMemcpyDeviceToHost);
    cudaFree(next);
    cudaFree(out);
    if (e != cudaSuccess) return 3;
    *ns = (double)r[0] / steps;
    return 0;
}

extern "C" int probe_cluster_barrier_ns(int cluster, int threads, int iters, double *ns) {
    unsigned long long *out = nullptr;
    if (cudaMalloc(&out, sizeof(unsigned long long)) != cudaSuccess) return 2;
    if (cluster > 8) cudaFuncSetAttribute(k_cluster_barrier, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cluster);
    cfg.blockDim = dim3(threads);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_cluster_barrier, iters, out);
    unsigned long long r = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&r, out, sizeof(r), cudaMemcpyDeviceToHost);
    cudaFree(out);
    if (e != cudaSuccess) return 3;
    *ns = (double)r / iters;
    return 0;
}
