// Breadth-first Gauss-Seidel heat diffusion (eq. heat, eq. HeatDiffusionUpdate)
// as one persistent dataflow kernel.
//
// Sweep k updates the sets D_0, D_1, ... in order, each set all at once from
// the latest neighbour values: neighbours in D_{i-1} carry sweep k's value,
// neighbours in D_i and D_{i+1} sweep k-1's.  So (sweep k, set i) depends on
// (k, i-1), (k-1, i) and (k-1, i+1) only: every pair with 2k + i = s can run
// at once, and sweeps pipeline as a wavefront over s = 0 .. L-1 + 2(N-1).
// Two state buffers, selected by the parity of k, keep the within-set update
// simultaneous: (k, i) writes buffer k&1 while D_i's sweep k-1 values stay in
// buffer (k-1)&1; the last reader of the overwritten sweep k-2 values,
// (k-1, i-1), is a predecessor of (k, i-1).
//
// There is no grid-wide barrier.  Every set keeps a counter of finished
// tiles (it only grows, sweep after sweep).  A tile of (k, i) starts once the
// counters show that (k, i-1), (k-1, i) and (k-1, i+1) are complete, and
// bumps its own set's counter with a release add when done.  Tiles are
// numbered in step order s and dealt round-robin to the CTAs serving the
// query; every tile depends only on lower numbers, so the lowest unfinished
// tile can always run and the kernel cannot deadlock (all CTAs are resident:
// cooperative launch).  Each tile loads its rows (column positions, weights,
// diagonal) before it waits, so only the gather of the neighbour state sits
// on the dependency chain.  Several queries (right-hand sides) run in one
// launch, each on its own group of CTAs.
//
// Vertices sit in breadth-first queue order, so D_i is a contiguous range and
// the set of a neighbour follows from its position alone.  A tile is TILE
// consecutive positions inside one set.
//
// Each heat value is carried as (mantissa, binary exponent): the solution
// falls by about e^-1 per edge length and leaves the FP32 (and FP64) range a
// few hundred sets away from the sources.  The sum of one update is formed
// relative to the largest exponent among its terms; scaling by powers of two
// is exact, so this is the same arithmetic with an unbounded exponent.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace gh {

namespace {

constexpr unsigned long long kWaitTimeoutNs = 2000000000ull;  // 2 s for any single wait
constexpr int kMaxDeg = 8;                                    // row entries held in registers

template <class T> struct GsJob {
    int nlev;
    int nsteps;            // nlev + 2 (sweeps - 1)
    int n_even;            // number of even sets; ptile0[n_even] = first tile of the odd sets
    int ntickets;          // tiles over all steps
    int cta0, ncta;        // the CTAs serving this query
    const int32_t *lvl_off;
    const int32_t *grow;
    const int32_t *gcol;
    const T *gw;
    const T *diag;
    const int32_t *ptile0;
    const int32_t *ptile1;
    const int2 *tiles;
    const int32_t *stepoff;  // [nsteps + 1] first tile number of each step
    int32_t *done;           // [nlev] finished tiles per set
    XVal<T> *U[2];
};

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(int32_t *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *p >= target; bounded: on timeout (or when another CTA gave up)
// raise the abort flag and the status word and return false.
__device__ bool wait_ge(const int32_t *p, int target, int *abort_flag, int *status) {
    if (ld_acquire(p) >= target) return true;
    const unsigned long long t0 = gtime();
    for (unsigned n = 1;; ++n) {
        if (ld_acquire(p) >= target) return true;
        if ((n & 31) == 0) {
            if (*(volatile int *)abort_flag) return false;
            if (gtime() - t0 > kWaitTimeoutNs) {
                atomicExch(abort_flag, 1);
                atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                return false;
            }
        }
        if (n > 64) __nanosleep(32);
    }
}

template <class T> __device__ __forceinline__ T ldexp_t(T x, int n);
template <> __device__ __forceinline__ float ldexp_t<float>(float x, int n) { return ldexpf(x, n); }
template <> __device__ __forceinline__ double ldexp_t<double>(double x, int n) { return ldexp(x, n); }
template <class T> __device__ __forceinline__ T frexp_t(T x, int *e);
template <> __device__ __forceinline__ float frexp_t<float>(float x, int *e) { return frexpf(x, e); }
template <> __device__ __forceinline__ double frexp_t<double>(double x, int *e) { return frexp(x, e); }

__device__ __forceinline__ XVal<float> ld_state(const XVal<float> *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    XVal<float> x;
    x.m = v.x;
    x.e = __float_as_int(v.y);
    return x;
}
__device__ __forceinline__ XVal<double> ld_state(const XVal<double> *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    XVal<double> x;
    x.m = v.x;
    x.e = (int)__double_as_longlong(v.y);
    return x;
}

// tile range [first, first + count) of job j at step s
template <class T> __device__ __forceinline__ void step_range(const GsJob<T> &j, int s, int nsweeps, int &first,
                                                             int &count) {
    first = 0;
    count = 0;
    if (s >= j.nsteps) return;
    int p = s & 1;
    int ihi = min(j.nlev - 1, s);
    if ((ihi & 1) != p) --ihi;
    int ilo = max(p, s - 2 * (nsweeps - 1));
    if (ilo > ihi) return;
    int jlo = (ilo - p) >> 1, jhi = (ihi - p) >> 1;
    const int32_t *pt = p ? j.ptile1 : j.ptile0;
    int base = p ? j.ptile0[j.n_even] : 0;
    first = base + pt[jlo];
    count = pt[jhi + 1] - pt[jlo];
}

template <class T>
__global__ void k_step_counts(const GsJob<T> *__restrict__ jobs, int q, int nsweeps, int32_t *cnt) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    const GsJob<T> &j = jobs[q];
    if (s >= j.nsteps) return;
    int f, n;
    step_range(j, s, nsweeps, f, n);
    cnt[s] = n;
}

__device__ __forceinline__ int tiles_of(const int32_t *lvl_off, int i) {
    return (lvl_off[i + 1] - lvl_off[i] + TILE - 1) / TILE;
}

template <class T>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? 4 : 2) k_gs(const GsJob<T> *__restrict__ jobs, int njobs, int nsweeps, int *abort_flag,
                                             int *status) {
    __shared__ int s_ok;
    int q = 0;
    while (q + 1 < njobs && (int)blockIdx.x >= jobs[q + 1].cta0) ++q;
    const GsJob<T> &J = jobs[q];
    const int nlev = J.nlev;
    int scur = 0;
    for (int t = (int)blockIdx.x - J.cta0; t < J.ntickets; t += J.ncta) {
        // step of tile number t (tile numbers grow with the step)
        while (J.stepoff[scur + 1] <= t) ++scur;
        const int s = scur;
        int first, count;
        step_range(J, s, nsweeps, first, count);
        const int2 tl = J.tiles[first + (t - J.stepoff[s])];
        const int i = tl.x;
        const int k = (s - i) >> 1;
        const int lo_i = J.lvl_off[i];
        const int r = tl.y + (int)threadIdx.x;
        const bool act = r < J.lvl_off[i + 1];
        // static row data, loaded before the wait
        int b = 0, e = 0;
        T dg = T(1);
        int cols[kMaxDeg];
        T wts[kMaxDeg];
        if (act) {
            b = __ldg(&J.grow[r]);
            e = __ldg(&J.grow[r + 1]);
            dg = __ldg(&J.diag[r]);
#pragma unroll
            for (int a = 0; a < kMaxDeg; ++a) {
                if (b + a < e) {
                    cols[a] = __ldg(&J.gcol[b + a]);
                    wts[a] = __ldg(&J.gw[b + a]);
                }
            }
        }
        if (threadIdx.x == 0) {
            bool ok = true;
            if (i > 0) ok = wait_ge(&J.done[i - 1], (k + 1) * tiles_of(J.lvl_off, i - 1), abort_flag, status);
            if (ok && k > 0) {
                ok = wait_ge(&J.done[i], k * tiles_of(J.lvl_off, i), abort_flag, status);
                if (ok && i + 1 < nlev) ok = wait_ge(&J.done[i + 1], k * tiles_of(J.lvl_off, i + 1), abort_flag, status);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;
        if (act) {
            XVal<T> *Ucur = J.U[k & 1];
            const XVal<T> *Uprv = J.U[(k & 1) ^ 1];
            XVal<T> u[kMaxDeg];
#pragma unroll
            for (int a = 0; a < kMaxDeg; ++a)
                if (b + a < e) u[a] = ld_state((cols[a] < lo_i ? Ucur : Uprv) + cols[a]);
            T acc = (i == 0) ? T(1) : T(0);  // u_0 = 1 on the sources
            int eref = (i == 0) ? 0 : kZeroExp;
#pragma unroll
            for (int a = 0; a < kMaxDeg; ++a) {
                if (b + a < e && u[a].m != T(0)) {
                    if (u[a].e > eref) {
                        acc = ldexp_t<T>(acc, eref - u[a].e);
                        eref = u[a].e;
                    }
                    acc += wts[a] * ldexp_t<T>(u[a].m, u[a].e - eref);
                }
            }
            for (int a = b + kMaxDeg; a < e; ++a) {  // long rows
                const int c = __ldg(&J.gcol[a]);
                const XVal<T> x = ld_state((c < lo_i ? Ucur : Uprv) + c);
                if (x.m != T(0)) {
                    if (x.e > eref) {
                        acc = ldexp_t<T>(acc, eref - x.e);
                        eref = x.e;
                    }
                    acc += __ldg(&J.gw[a]) * ldexp_t<T>(x.m, x.e - eref);
                }
            }
            const T val = acc / dg;
            int ex = 0;
            const T mm = frexp_t<T>(val, &ex);
            XVal<T> out;
            out.m = mm;
            out.e = (mm == T(0)) ? kZeroExp : ex + eref;
            Ucur[r] = out;
        }
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(&J.done[i], 1);
    }
}

template <class T> __global__ void k_zero_state(XVal<T> *a, XVal<T> *b, int n) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        XVal<T> z;
        z.m = T(0);
        z.e = kZeroExp;
        a[r] = z;
        b[r] = z;
    }
}

template <class T> gh_status run_gs_t(Ctx *c, std::vector<QueryWs *> &ws, int sweeps, cudaEvent_t ev0,
                                     cudaEvent_t ev1) {
    cudaStream_t st = c->stream;
    const int K = (int)ws.size();
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs<T>, TILE, 0));
    if (per_sm < 1) { set_error("diffusion kernel does not fit on an SM"); return GH_EDEVICE; }
    const int grid = per_sm * c->num_sms;
    if (K > grid) { set_error("internal: more queries than resident CTAs in one diffusion launch"); return GH_EINVAL; }
    std::vector<GsJob<T>> jobs(K);
    size_t soff_total = 0;
    for (int q = 0; q < K; ++q) soff_total += (size_t)ws[q]->nlev + 2 * (size_t)sweeps + 2;
    int32_t *scratch = nullptr;   // per query: step counts and their prefix
    GH_CUDA(cudaMallocAsync((void **)&scratch, sizeof(int32_t) * 2 * soff_total, st));
    GsJob<T> *djobs = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&djobs, sizeof(GsJob<T>) * K, st));
    size_t at = 0;
    int cta = 0;
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        GsJob<T> j{};
        j.nlev = w.nlev;
        j.nsteps = w.nlev + 2 * (sweeps - 1);
        j.n_even = (w.nlev + 1) / 2;
        j.cta0 = cta;
        j.ncta = grid / K + (q < grid % K ? 1 : 0);
        cta += j.ncta;
        j.lvl_off = ptr<int32_t>(w.lvl_off);
        j.grow = ptr<int32_t>(w.grow);
        j.gcol = ptr<int32_t>(w.gent);
        j.gw = reinterpret_cast<const T *>(ptr<int32_t>(w.gent) + w.cap_nnz);
        j.diag = ptr<T>(w.diag);
        j.ptile0 = ptr<int32_t>(w.ptile);
        j.ptile1 = ptr<int32_t>(w.ptile) + j.n_even + 1;
        j.tiles = ptr<int2>(w.tiles);
        int32_t *cnt = scratch + at;
        int32_t *soff = scratch + soff_total + at;
        at += (size_t)j.nsteps + 2;
        j.stepoff = soff;
        j.done = ptr<int32_t>(w.n1);
        j.U[0] = ptr<XVal<T>>(w.U0);
        j.U[1] = ptr<XVal<T>>(w.U1);
        jobs[q] = j;
        w.final_buf = (sweeps - 1) & 1;
    }
    GH_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(GsJob<T>) * K, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> ntick(K);
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        k_zero_state<T><<<blocks_for(w.nreach, 256), 256, 0, st>>>(jobs[q].U[0], jobs[q].U[1], w.nreach); ++c->launches;
        GH_CUDA(cudaMemsetAsync(jobs[q].done, 0, sizeof(int32_t) * (w.nlev + 1), st));
        int32_t *cnt = const_cast<int32_t *>(jobs[q].stepoff) - soff_total;
        k_step_counts<T><<<blocks_for(jobs[q].nsteps, 256), 256, 0, st>>>(djobs, q, sweeps, cnt); ++c->launches;
        gh_status s = exclusive_scan_i32(c, cnt, const_cast<int32_t *>(jobs[q].stepoff), jobs[q].nsteps, &ntick[q]);
        if (s != GH_OK) { cudaFreeAsync(djobs, st); cudaFreeAsync(scratch, st); return s; }
        jobs[q].ntickets = ntick[q];
    }
    GH_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(GsJob<T>) * K, cudaMemcpyHostToDevice, st));
    GH_CUDA(cudaMemsetAsync(&c->bar_dev->abort, 0, sizeof(int), st));
    int njobs = K;
    int *status = c->status_dev;
    int *abort_flag = &c->bar_dev->abort;
    void *argv[] = {(void *)&djobs, (void *)&njobs, (void *)&sweeps, (void *)&abort_flag, (void *)&status};
    if (ev0) cudaEventRecord(ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_gs<T>, dim3(grid), dim3(TILE), argv, 0, st);
    ++c->launches;
    if (ev1) cudaEventRecord(ev1, st);
    cudaFreeAsync(djobs, st);
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the diffusion kernel");
    return GH_OK;
}

}  // namespace

gh_status run_gs(Ctx *c, const DevMesh &m, std::vector<QueryWs *> &ws, int sweeps, cudaEvent_t ev0, cudaEvent_t ev1) {
    (void)m;
    if (ws.empty()) return GH_OK;
    return ws[0]->fp64 ? run_gs_t<double>(c, ws, sweeps, ev0, ev1) : run_gs_t<float>(c, ws, sweeps, ev0, ev1);
}

}  // namespace gh
