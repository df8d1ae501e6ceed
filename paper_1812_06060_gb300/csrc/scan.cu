// Device-wide exclusive prefix sum of int32 counts (row lengths, children per
// parent, tiles per level): per-block reduce, scan of the block sums (the same
// routine, recursively), per-block scan with the block's offset.
#include "internal.cuh"

namespace gh {

namespace {

constexpr int SB = 256;      // threads per block
constexpr int SI = 8;        // items per thread
constexpr int SCHUNK = SB * SI;

__device__ __forceinline__ int32_t warp_incl(int32_t v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += y;
    }
    return v;
}

// exclusive scan of one value per thread over the block; returns the block total
__device__ int32_t block_excl(int32_t v, int32_t &excl) {
    __shared__ int32_t wsum[SB / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = warp_incl(v);
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t s = (lane < SB / 32) ? wsum[lane] : 0;
        s = warp_incl(s);
        if (lane < SB / 32) wsum[lane] = s;
    }
    __syncthreads();
    int32_t before = (wid > 0) ? wsum[wid - 1] : 0;
    int32_t total = wsum[SB / 32 - 1];
    excl = before + incl - v;
    __syncthreads();
    return total;
}

__global__ void k_block_sums(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ sums) {
    int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i)
        if (base + i < n) s += in[base + i];
    int32_t ex;
    int32_t tot = block_excl(s, ex);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_block_scan(const int32_t *__restrict__ in, int64_t n, const int32_t *__restrict__ offs,
                             int32_t *__restrict__ out) {
    int64_t base = (int64_t)blockIdx.x * SCHUNK + (int64_t)threadIdx.x * SI;
    int32_t v[SI];
    int32_t s = 0;
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int32_t ex;
    int32_t tot = block_excl(s, ex);
    int32_t run = ex + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < SI; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    // the last block writes the grand total at out[n]
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (offs ? offs[blockIdx.x] : 0) + tot;
}

}  // namespace

// out[0..n) = exclusive prefix sums of in, out[n] = total (device memory).
gh_status exclusive_scan_u32_dev(Ctx *c, const int32_t *in, int32_t *out, int64_t n) {
    if (n <= 0) {
        GH_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), c->stream));
        return GH_OK;
    }
    int64_t nb = (n + SCHUNK - 1) / SCHUNK;
    if (nb == 1) {
        k_block_scan<<<1, SB, 0, c->stream>>>(in, n, nullptr, out); ++c->launches;
        GH_CUDA(cudaGetLastError());
        return GH_OK;
    }
    int32_t *sums = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&sums, sizeof(int32_t) * (size_t)(2 * nb + 1), c->stream));
    int32_t *soff = sums + nb;
    k_block_sums<<<(unsigned)nb, SB, 0, c->stream>>>(in, n, sums); ++c->launches;
    gh_status st = exclusive_scan_u32_dev(c, sums, soff, nb);
    if (st == GH_OK) {
        k_block_scan<<<(unsigned)nb, SB, 0, c->stream>>>(in, n, soff, out); ++c->launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "k_block_scan");
    }
    cudaFreeAsync(sums, c->stream);
    return st;
}

gh_status exclusive_scan_i32(Ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *total_host) {
    gh_status st = exclusive_scan_u32_dev(c, in, out, n);
    if (st != GH_OK) return st;
    if (total_host) {
        GH_CUDA(cudaMemcpyAsync(total_host, out + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        GH_CUDA(cudaStreamSynchronize(c->stream));
    }
    return GH_OK;
}

}  // namespace gh
