// Mean edge length without any device allocation.
//
// gh_mesh_load computes the mean edge length hbar (the length scale of the
// diffusion time t = m hbar^2) with a two-level deterministic reduction whose
// per-block partial sums live in memory it allocates.  This file holds a
// variant of that reduction for callers that must not allocate device memory
// themselves or through the library: code that runs while a CUDA stream is
// being captured into a graph (allocation calls are not allowed there),
// applications that hand every byte of the device to their own allocator and
// forbid others from calling cudaMalloc, and real-time paths where an
// allocation may block on a device-wide synchronisation.  The partial sums
// live in a fixed file-scope device array instead.
#include <mutex>

#include "internal.cuh"

namespace gh {

namespace {

constexpr int64_t kNaPerBlock = 65536;   // edges per partial sum (as in the mesh setup)
constexpr int kNaMaxParts = 8192;        // partial sums the fixed array holds
constexpr int kNaThreads = 256;
constexpr int kNaMaxDevices = 64;

// Scratch shared by every call on a device: kNaMaxParts partial sums
// (64 KiB).  Each GPU that loads the library holds it until the process exits.
static __device__ __align__(256) double g_na_partials[kNaMaxParts];

// per block: the sum of the lengths of edges [b * kNaPerBlock, (b+1) * kNaPerBlock)
// in a fixed order (strided per thread, then a tree)
__global__ void __launch_bounds__(kNaThreads) k_na_partial(const double *__restrict__ V, const int32_t *__restrict__ edges,
                                                           int64_t ne, double *part) {
    __shared__ double s[kNaThreads];
    const int64_t b0 = (int64_t)blockIdx.x * kNaPerBlock;
    const int64_t b1 = min(ne, b0 + kNaPerBlock);
    double acc = 0.0;
    for (int64_t e = b0 + threadIdx.x; e < b1; e += kNaThreads) {
        const double *a = V + 3 * (int64_t)edges[2 * e], *c = V + 3 * (int64_t)edges[2 * e + 1];
        const double d0 = c[0] - a[0], d1 = c[1] - a[1], d2 = c[2] - a[2];
        acc += sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kNaThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// sum of the partials in the same fixed order, divided by the edge count
__global__ void __launch_bounds__(kNaThreads) k_na_final(const double *__restrict__ part, int nb, int64_t ne,
                                                         double *out) {
    __shared__ double s[kNaThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kNaThreads) acc += part[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kNaThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = s[0] / (double)ne;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device address of the scratch array on the current device, looked up once
// per device.  In host code g_na_partials names a host-side stand-in, not
// device memory, so kernels get the address from cudaGetSymbolAddress.
gh_status na_scratch(double **out) {
    static std::mutex mu;
    static double *addr[kNaMaxDevices] = {};
    int dev = 0;
    GH_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("device ordinal out of range for the fixed scratch table");
        return GH_EINVAL;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev]) {
        double *p = nullptr;
        GH_CUDA(cudaGetSymbolAddress((void **)&p, g_na_partials));
        addr[dev] = p;
    }
    *out = addr[dev];
    return GH_OK;
}

}  // namespace

}  // namespace gh

using namespace gh;

extern "C" gh_status gh_mean_edge_length_noalloc(const double *V, const int32_t *edges, int64_t ne, double *out,
                                                 void *stream) {
    if (!V || !edges || !out) { set_error("NULL argument"); return GH_EINVAL; }
    if (ne < 1) { set_error("ne must be >= 1"); return GH_EINVAL; }
    const int64_t nb = (ne + kNaPerBlock - 1) / kNaPerBlock;
    if (nb > kNaMaxParts) {
        set_error("ne = " + std::to_string(ne) + " exceeds the fixed scratch limit of " +
                  std::to_string((int64_t)kNaMaxParts * kNaPerBlock) + " edges");
        return GH_EINVAL;
    }
    if (!on_device(V) || !on_device(edges) || !on_device(out)) {
        set_error("V, edges and out must be device memory of the current device");
        return GH_EINVAL;
    }
    double *part = nullptr;
    gh_status s = na_scratch(&part);
    if (s != GH_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_na_partial<<<(unsigned)nb, kNaThreads, 0, st>>>(V, edges, ne, part);
    k_na_final<<<1, kNaThreads, 0, st>>>(part, (int)nb, ne, out);
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}
