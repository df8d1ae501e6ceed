// Mean edge length without any device allocation.
//
// gh_mesh_load computes the mean edge length hbar (the length scale of the
// diffusion time t = m hbar^2) with a two-level deterministic reduction whose
// per-block partial sums live in memory it allocates.  This file holds a
// variant of that reduction for callers that cannot have the library
// allocate device memory: applications whose own allocator or memory pool
// owns the device memory and forbids other code from calling cudaMalloc (a
// renderer or a framework with its own caching allocator, a process that has
// reserved nearly all of the device), and latency-critical loops where a
// cudaMalloc or cudaFree may wait for the whole device to go idle.  The
// partial sums live in a fixed file-scope device array instead.
#include <mutex>
#include <string>

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

// true for device memory of the current device (or managed memory, which
// the current device can reach)
bool on_current_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Id of the current context (cuCtxGetId through the runtime's driver entry
// points, so the library needs no link to the driver library), 0 if the
// driver cannot tell.  A context made after a device reset has a new id.
unsigned long long current_context_id() {
    typedef int (*get_current_fn)(void **);
    typedef int (*get_id_fn)(void *, unsigned long long *);
    static get_current_fn get_current = nullptr;
    static get_id_fn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<get_current_fn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<get_id_fn>(f);
        (void)cudaGetLastError();
    });
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current && get_id && get_current(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

// Device address of the scratch array on the current device, looked up once
// per device and context.  In host code g_na_partials names a host-side
// stand-in, not device memory, so kernels get the address from
// cudaGetSymbolAddress, called while that device is current.
gh_status na_scratch(int dev, double **out) {
    static std::mutex mu;
    static double *addr[kNaMaxDevices] = {};
    static unsigned long long ctx_of[kNaMaxDevices] = {};
    if (dev < 0 || dev >= kNaMaxDevices) {
        set_error("device ordinal out of range for the fixed scratch table");
        return GH_EINVAL;
    }
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lk(mu);
    if (!addr[dev] || ctx_of[dev] != ctx) {
        double *p = nullptr;
        GH_CUDA(cudaGetSymbolAddress((void **)&p, g_na_partials));
        addr[dev] = p;
        ctx_of[dev] = ctx;
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
    int dev = 0;
    GH_CUDA(cudaGetDevice(&dev));
    if (!on_current_device(V, dev) || !on_current_device(edges, dev) || !on_current_device(out, dev)) {
        set_error("V, edges and out must be device memory of the current device (" + std::to_string(dev) + ")");
        return GH_EINVAL;
    }
    double *part = nullptr;
    gh_status s = na_scratch(dev, &part);
    if (s != GH_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_na_partial<<<(unsigned)nb, kNaThreads, 0, st>>>(V, edges, ne, part);
    k_na_final<<<1, kNaThreads, 0, st>>>(part, (int)nb, ne, out);
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}
