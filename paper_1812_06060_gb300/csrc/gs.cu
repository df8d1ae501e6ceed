// Breadth-first Gauss-Seidel heat diffusion (eq. heat, eq. HeatDiffusionUpdate)
// as one persistent cooperative kernel.
//
// Sweep k updates the sets D_0, D_1, ... in order, each set all at once from
// the latest neighbour values: neighbours in D_{i-1} carry sweep k's value,
// neighbours in D_i and D_{i+1} sweep k-1's.  So (sweep k, set i) depends on
// (k, i-1), (k-1, i) and (k-1, i+1) only, and every pair (k, i) with
// 2k + i = s can run in the same grid step s.  The kernel runs the steps
// s = 0 .. L-1 + 2(N-1) with one grid barrier between steps: sweeps are
// pipelined as a wavefront instead of taking L barriers each.  Two state
// buffers, selected by the parity of k, keep the within-set updates
// simultaneous: a step writes buffer k&1 while the same set's previous values
// stay readable in buffer (k-1)&1 (the last reader of a value is two steps
// before its overwrite, see the schedule above).
//
// Vertices sit in breadth-first queue order, so D_i is a contiguous range and
// the set of a neighbour follows from its position alone.  Work is cut into
// tiles of TILE consecutive positions inside one set; the tiles of one step
// are a contiguous slice of a table sorted by (parity, set).  Several queries
// (right-hand sides) share the kernel: each step's tiles of all queries are
// concatenated.
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

constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s per barrier
constexpr int kMaxJobs = TILE;                                   // queries per launch

template <class T> struct GsJob {
    int nlev;
    int nsteps;            // nlev + 2 (sweeps - 1)
    int n_even;            // number of even sets; ptile0[n_even] = first tile of the odd sets
    int pad;
    const int32_t *lvl_off;
    const int32_t *grow;
    const int32_t *gcol;
    const T *gw;
    const T *diag;
    const int32_t *ptile0;
    const int32_t *ptile1;
    const int2 *tiles;
    XVal<T> *U[2];
};

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier with a bounded wait: on timeout it raises the abort flag
// and the status word and every CTA leaves the kernel.
__device__ bool grid_barrier(GridBarrier *b, unsigned nblocks, int *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *vgen = &b->gen;
        volatile int *vabort = &b->abort;
        unsigned g = *vgen;
        __threadfence();
        unsigned arrived = atomicAdd(&b->count, 1u) + 1u;
        if (arrived == nblocks) {
            b->count = 0;
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            unsigned long long t0 = gtime();
            while (*vgen == g) {
                if (*vabort) { ok = 0; break; }
                if (gtime() - t0 > kBarrierTimeoutNs) {
                    atomicExch(&b->abort, 1);
                    atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (*vabort) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class T> __device__ __forceinline__ T ldexp_t(T x, int n);
template <> __device__ __forceinline__ float ldexp_t<float>(float x, int n) { return ldexpf(x, n); }
template <> __device__ __forceinline__ double ldexp_t<double>(double x, int n) { return ldexp(x, n); }
template <class T> __device__ __forceinline__ T frexp_t(T x, int *e);
template <> __device__ __forceinline__ float frexp_t<float>(float x, int *e) { return frexpf(x, e); }
template <> __device__ __forceinline__ double frexp_t<double>(double x, int *e) { return frexp(x, e); }

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
__global__ void __launch_bounds__(TILE) k_gs(const GsJob<T> *__restrict__ jobs, int njobs, int nsweeps, int nsteps,
                                             GridBarrier *bar, int *status) {
    __shared__ int s_pref[kMaxJobs + 1];
    __shared__ int s_first[kMaxJobs];
    const unsigned nblocks = gridDim.x;
    for (int s = 0; s < nsteps; ++s) {
        // per-job tile ranges of this step and their prefix over jobs
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int q = 0; q < njobs; ++q) {
                int f, n;
                step_range(jobs[q], s, nsweeps, f, n);
                s_first[q] = f;
                s_pref[q] = acc;
                acc += n;
            }
            s_pref[njobs] = acc;
        }
        __syncthreads();
        const int total = s_pref[njobs];
        for (int t = blockIdx.x; t < total; t += nblocks) {
            int q = 0;
            while (q + 1 < njobs && s_pref[q + 1] <= t) ++q;
            const GsJob<T> &J = jobs[q];
            const int2 tl = J.tiles[s_first[q] + (t - s_pref[q])];
            const int i = tl.x;
            const int lo_i = J.lvl_off[i];
            const int end = J.lvl_off[i + 1];
            const int r = tl.y + threadIdx.x;
            if (r < end) {
                const int k = (s - i) >> 1;
                XVal<T> *Ucur = J.U[k & 1];
                const XVal<T> *Uprv = J.U[(k & 1) ^ 1];
                T acc = (i == 0) ? T(1) : T(0);     // u_0 = 1 on the sources
                int eref = (i == 0) ? 0 : kZeroExp;
                const int b = J.grow[r], e = J.grow[r + 1];
                for (int a = b; a < e; ++a) {
                    const int cpos = J.gcol[a];
                    const XVal<T> u = (cpos < lo_i) ? Ucur[cpos] : Uprv[cpos];
                    if (u.m != T(0)) {
                        if (u.e > eref) {
                            acc = ldexp_t<T>(acc, eref - u.e);
                            eref = u.e;
                        }
                        acc += J.gw[a] * ldexp_t<T>(u.m, u.e - eref);
                    }
                }
                const T val = acc / J.diag[r];
                int ex = 0;
                const T mm = frexp_t<T>(val, &ex);
                XVal<T> out;
                out.m = mm;
                out.e = (mm == T(0)) ? kZeroExp : ex + eref;
                Ucur[r] = out;
            }
        }
        if (s + 1 < nsteps && !grid_barrier(bar, nblocks, status)) return;
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
    int K = (int)ws.size();
    if (K > kMaxJobs) {
        set_error("internal: too many queries in one diffusion launch");
        return GH_EINVAL;
    }
    std::vector<GsJob<T>> jobs(K);
    int nsteps = 0;
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        GsJob<T> j{};
        j.nlev = w.nlev;
        j.nsteps = w.nlev + 2 * (sweeps - 1);
        int n_even = (w.nlev + 1) / 2;
        j.n_even = n_even;
        j.lvl_off = ptr<int32_t>(w.lvl_off);
        j.grow = ptr<int32_t>(w.grow);
        j.gcol = ptr<int32_t>(w.gent);
        j.gw = reinterpret_cast<const T *>(ptr<int32_t>(w.gent) + w.cap_nnz);
        j.diag = ptr<T>(w.diag);
        j.ptile0 = ptr<int32_t>(w.ptile);
        j.ptile1 = ptr<int32_t>(w.ptile) + n_even + 1;
        j.tiles = ptr<int2>(w.tiles);
        j.U[0] = ptr<XVal<T>>(w.U0);
        j.U[1] = ptr<XVal<T>>(w.U1);
        jobs[q] = j;
        nsteps = std::max(nsteps, j.nsteps);
        k_zero_state<T><<<blocks_for(w.nreach, 256), 256, 0, st>>>(j.U[0], j.U[1], w.nreach); ++c->launches;
        w.final_buf = (sweeps - 1) & 1;
    }
    if (sweeps <= 0) return GH_OK;
    GsJob<T> *djobs = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&djobs, sizeof(GsJob<T>) * K, st));
    GH_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(GsJob<T>) * K, cudaMemcpyHostToDevice, st));
    GH_CUDA(cudaMemsetAsync(c->bar_dev, 0, sizeof(GridBarrier), st));
    int per_sm = 0;
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gs<T>, TILE, 0));
    if (per_sm < 1) { cudaFreeAsync(djobs, st); set_error("diffusion kernel does not fit on an SM"); return GH_EDEVICE; }
    int grid = per_sm * c->num_sms;
    int njobs = K;
    int *status = c->status_dev;
    GridBarrier *bar = c->bar_dev;
    void *argv[] = {(void *)&djobs, (void *)&njobs, (void *)&sweeps, (void *)&nsteps, (void *)&bar, (void *)&status};
    if (ev0) cudaEventRecord(ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel((void *)k_gs<T>, dim3(grid), dim3(TILE), argv, 0, st);
    ++c->launches;
    if (ev1) cudaEventRecord(ev1, st);
    cudaFreeAsync(djobs, st);
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
