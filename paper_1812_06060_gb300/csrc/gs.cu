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
// numbered in step order s and dealt round-robin to the CTAs; every tile
// depends only on lower numbers of its own query.  Each tile loads its rows
// (column positions, weights, diagonal) before it waits, so only the gather
// of the neighbour state sits on the dependency chain.
//
// Several queries (right-hand sides) run in one launch and every CTA serves
// all of them: CTA c takes, for round r = 0, 1, ... and query q = 0..K-1 in
// turn, tile r * grid + c of query q (skipping queries with fewer tiles).
// While one query's next set waits for its predecessors, the CTA works on
// the other queries' tiles, so the dependency latency of one wavefront is
// filled with the work of the others.  In the order (r, q, c) every tile
// comes after the tiles it depends on and after the earlier tiles of its
// CTA, so the lowest unfinished tile can always run and the kernel cannot
// deadlock (all CTAs are resident: cooperative launch).
//
// Vertices sit in breadth-first set order (inside a set, the rows with few
// entries first), so D_i is a contiguous range and the set of a neighbour
// follows from its position alone.  A tile is TILE
// consecutive positions inside one set; its rows are one column-major block
// (entry a of position p at a * cp + p, padded with zero-weight entries to the
// tile's longest row), so the 32 lanes of a warp reading entry a of their
// rows read 32 consecutive entries of shared memory.
//
// Each heat value is carried as (mantissa, binary exponent): the solution
// falls by about e^-1 per edge length and leaves the FP32 (and FP64) range a
// few hundred sets away from the sources.  The sum of one update is formed
// relative to the largest exponent among its terms; scaling by powers of two
// is exact, so this is the same arithmetic with an unbounded exponent.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstddef>

#include "internal.cuh"

namespace gh {

namespace {

constexpr unsigned long long kWaitTimeoutNs = 2000000000ull;  // 2 s for a staging-barrier wait
constexpr int kMaxDeg = 8;                                    // row entries held in registers (wide stages)

template <class T> struct GsJob {
    int nlev;
    int nsteps;            // nbands * band_steps
    int nsweeps;           // this query's sweeps
    int band;              // sweeps per band
    int band_steps;        // steps per band: nlev + 2 (band - 1)
    int n_even;            // number of even sets; ptile0[n_even] = first tile of the odd sets
    int ntickets;          // tiles over all steps
    int zero_pos;          // a position that always holds the zero state (nreach)
    const int32_t *lvl_off;
    const Ent<T> *gent;
    const T *diag;
    const int32_t *ptile0;
    const int32_t *ptile1;
    const TileDesc *tiles;
    const int32_t *stepoff;  // [nsteps + 1] first tile number of each step
    int32_t *done;           // [nlev] tiles finished per set, over all sweeps
    XVal<T> *U[2];
};

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_relaxed(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// the acquire half of a relaxed poll: later loads see what the observed release published
__device__ __forceinline__ void fence_acquire() { asm volatile("fence.acquire.gpu;" ::: "memory"); }

__device__ __forceinline__ void red_release_add(int32_t *p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Exponent arithmetic on normalised mantissas (0.5 <= |m| < 1, or m = 0).
// xscale(m, d) = m * 2^d for d <= 0, made by adding d to the exponent field;
// a term more than 125 (FP64: 1021) binades below the largest term of a sum
// is below the precision of the sum and is dropped (returns 0).
__device__ __forceinline__ float xscale(float m, int d) {
    return (d >= -125) ? __int_as_float(__float_as_int(m) + (d << 23)) : 0.0f;
}
__device__ __forceinline__ double xscale(double m, int d) {
    return (d >= -1021) ? __longlong_as_double(__double_as_longlong(m) + ((long long)d << 52)) : 0.0;
}
// v * 2^eref -> (m, e) with m normalised (the role of frexp)
__device__ __forceinline__ void xnorm(float v, int eref, float &m, int &e) {
    int b = __float_as_int(v);
    int ex = (b >> 23) & 0xff;
    if (ex == 0) {
        if ((b & 0x7fffffff) == 0) { m = 0.0f; e = kZeroExp; return; }
        v *= 18446744073709551616.0f;  // subnormal: scale by 2^64 first
        b = __float_as_int(v);
        ex = ((b >> 23) & 0xff) - 64;
    }
    m = __int_as_float((b & 0x807fffff) | (126 << 23));
    e = eref + (ex - 126);
}
__device__ __forceinline__ void xnorm(double v, int eref, double &m, int &e) {
    long long b = __double_as_longlong(v);
    int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) {
        if ((b & 0x7fffffffffffffffll) == 0) { m = 0.0; e = kZeroExp; return; }
        v *= 18446744073709551616.0;
        b = __double_as_longlong(v);
        ex = (int)((b >> 52) & 0x7ff) - 64;
    }
    m = __longlong_as_double((b & (long long)0x800fffffffffffffull) | (1022ll << 52));
    e = eref + (ex - 1022);
}

// Neighbour state.  Plain (weak, L1-cached) loads: every value a tile reads
// was stored before a release add on a set counter that the tile's producer
// observed with an acquire load and passed on through the staging mbarrier
// (release/acquire within the CTA), so the PTX memory model makes these
// loads see it; L1 caching lets the 8 gathers of a warp share sectors.
__device__ __forceinline__ XVal<float> ld_state(const XVal<float> *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    XVal<float> x;
    x.m = v.x;
    x.e = __float_as_int(v.y);
    return x;
}
__device__ __forceinline__ XVal<double> ld_state(const XVal<double> *p) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    XVal<double> x;
    x.m = v.x;
    x.e = (int)__double_as_longlong(v.y);
    return x;
}

// Steps run band by band: band b holds sweeps [b * band, b * band + kb) and
// band_steps steps; its step s (global step b * band_steps + s) covers the
// pairs (k, i) with 2 (k - b * band) + i = s.  One band of all sweeps is the
// plain wavefront.
__device__ __forceinline__ void step_band(int g, int band_steps, int band, int &s, int &k0) {
    const int b = g / band_steps;
    s = g - b * band_steps;
    k0 = b * band;
}

// tile range [first, first + count) of job j at global step g
template <class T> __device__ __forceinline__ void step_range(const GsJob<T> &j, int g, int &first,
                                                             int &count) {
    first = 0;
    count = 0;
    if (g >= j.nsteps) return;
    int s, k0;
    step_band(g, j.band_steps, j.band, s, k0);
    const int kb = min(j.band, j.nsweeps - k0);
    int p = s & 1;
    int ihi = min(j.nlev - 1, s);
    if ((ihi & 1) != p) --ihi;
    int ilo = max(p, s - 2 * (kb - 1));
    if (ilo > ihi) return;
    int jlo = (ilo - p) >> 1, jhi = (ihi - p) >> 1;
    const int32_t *pt = p ? j.ptile1 : j.ptile0;
    int base = p ? j.ptile0[j.n_even] : 0;
    first = base + pt[jlo];
    count = pt[jhi + 1] - pt[jlo];
}

template <class T>
__global__ void k_step_counts(const GsJob<T> *__restrict__ jobs, int q, int32_t *cnt) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    const GsJob<T> &j = jobs[q];
    if (s >= j.nsteps) return;
    int f, n;
    step_range(j, s, f, n);
    cnt[s] = n;
}

// ---------------------------------------------------------------- bulk copies into shared memory

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// global -> shared bulk copy; both addresses and the size are multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx_only(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait until (k, i-1), (k-1, i) and (k-1, i+1) are complete: the set
// counters (tiles finished, over all sweeps so far) reach their targets
// (a target <= 0 means no wait).  The three counters are polled with relaxed
// loads that go out together; once all are met one acquire fence orders the
// tile's reads after the releases observed.  Bounded like every wait.
__device__ bool wait_sets(const int32_t *p0, int t0, const int32_t *p1, int t1, const int32_t *p2, int t2,
                          unsigned long long limit_ns, int *abort_flag, int *status) {
    const unsigned long long tstart = gtime();
    for (unsigned n = 0;; ++n) {
        const int v0 = (t0 > 0) ? ld_relaxed(p0) : 0;
        const int v1 = (t1 > 0) ? ld_relaxed(p1) : 0;
        const int v2 = (t2 > 0) ? ld_relaxed(p2) : 0;
        if (v0 >= t0 && v1 >= t1 && v2 >= t2) {
            fence_acquire();
            return true;
        }
        if ((n & 31) == 31) {
            if (*(volatile int *)abort_flag) return false;
            if (gtime() - tstart > limit_ns) {
                atomicExch(abort_flag, 1);
                atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                return false;
            }
        }
        if (n > 64) __nanosleep(32);
    }
}

constexpr int kCW = 8;                        // consumer warps per CTA
constexpr int kThreads = 32 * (kCW + 1);      // + one producer warp
constexpr int kVPT = TILE / (32 * kCW);       // positions per consumer thread
static_assert(kVPT * 32 * kCW == TILE, "tile must split evenly over the consumer threads");

// one staging buffer: the tile's diagonal and rows (up to MAXD entries per
// row; wider tiles read their rows from global memory), plus the tile's
// facts written by the producer
template <class T, int MAXD> struct alignas(128) Stage {
    Ent<T> ent[MAXD * TILE];
    T diag[TILE + 8];
    int start, count, lo, k, level, cp, w, d0, e0, fits, abort, finished, q, pad[3];
};
// every bulk-copy destination must start on a 16-byte boundary, in both stages
static_assert(sizeof(Stage<float, 8>) % 16 == 0 && sizeof(Stage<double, 8>) % 16 == 0, "stage size");
static_assert(sizeof(Stage<float, 6>) % 16 == 0, "stage size");
using StageF8 = Stage<float, 8>;
using StageD8 = Stage<double, 8>;
using StageF6 = Stage<float, 6>;
static_assert(offsetof(StageF8, diag) % 16 == 0 && offsetof(StageD8, diag) % 16 == 0 &&
              offsetof(StageF6, diag) % 16 == 0, "stage layout");

// resident CTAs per SM: FP32 with 8-entry stages 3 (shared memory and 72
// registers), with 6-entry stages 4 (56 registers); FP64 1
template <class T, int MAXD> constexpr int gs_ctas_per_sm() { return sizeof(T) == 4 ? (MAXD <= 6 ? 4 : 3) : 1; }

constexpr int kMaxJobs = 256;                 // queries per launch (larger batches take several launches)

// tile number t of job J -> descriptor and step (t < J.ntickets), walking
// forward from the step cursor scur
template <class T>
__device__ __forceinline__ void lookup_tile(const GsJob<T> &J, int t, int &scur, TileDesc &d, int &s,
                                            int &tile) {
    while (J.stepoff[scur + 1] <= t) ++scur;
    s = scur;
    int first, count;
    step_range(J, s, first, count);
    tile = first + (t - J.stepoff[s]);
    d = J.tiles[tile];
}

// bounded wait on an mbarrier phase
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int *abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    for (unsigned n = 1;; ++n) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((n & 63) == 0) {
            if (gtime() - t0 > kWaitTimeoutNs) return false;
        }
    }
}

// The rows of one tile (consumer warp cw's positions), the first D entries of
// each row held in registers; entries past D (tiles wider than kMaxDeg only)
// are read one at a time.  Ucur / Uprv: this and the previous sweep's state.
template <class T, int D, bool WIDE = true>
__device__ __forceinline__ void gs_tile_rows(XVal<T> *Ucur, const XVal<T> *Uprv, const Ent<T> *E, const T *sdiag,
                                             int zero_pos, int start, int count, int lo, int cp, int wt, int sd,
                                             int cw, int lane) {
    XVal<T> u[kVPT][D];
#pragma unroll
    for (int v = 0; v < kVPT; ++v) {
        const int p = v * 32 * kCW + cw * 32 + lane;
        // all gathers of the thread go out together; entries past the
        // block's width read the zero state kept at position nreach
#pragma unroll
        for (int a = 0; a < D; ++a) {
            int c = zero_pos;
            if (p < count && a < wt) c = E[a * cp + p].col;
            u[v][a] = ld_state((c < lo ? Ucur : Uprv) + c);
        }
    }
#pragma unroll
    for (int v = 0; v < kVPT; ++v) {
        const int p = v * 32 * kCW + cw * 32 + lane;
        if (p >= count) continue;
        const int r = start + p;
        // the sum is formed relative to its largest exponent (u_0 = 1 = 0.5 * 2^1 on the sources)
        int eref = (lo == 0) ? 1 : kZeroExp;   // zero states carry kZeroExp: no test needed
#pragma unroll
        for (int a = 0; a < D; ++a) eref = max(eref, u[v][a].e);
        for (int a = D; WIDE && a < wt; ++a) {  // rows longer than D (tiles wider than kMaxDeg)
            const Ent<T> x = E[a * cp + p];
            const XVal<T> w = ld_state((x.col < lo ? Ucur : Uprv) + x.col);
            if (w.m != T(0)) eref = max(eref, w.e);
        }
        T acc = (lo == 0) ? xscale(T(0.5), 1 - eref) : T(0);
#pragma unroll
        for (int a = 0; a < D; ++a) {
            const T w = (a < wt) ? E[a * cp + p].w : T(0);
            acc += w * xscale(u[v][a].m, u[v][a].e - eref);
        }
        for (int a = D; WIDE && a < wt; ++a) {
            const Ent<T> x = E[a * cp + p];
            const XVal<T> w = ld_state((x.col < lo ? Ucur : Uprv) + x.col);
            acc += x.w * xscale(w.m, w.e - eref);
        }
        XVal<T> out;
        xnorm(acc * sdiag[r - sd], eref, out.m, out.e);   // diag holds 1 / (A_v + t sum theta)
        Ucur[r] = out;
    }
}

// Producer warp (one lane): for each of this CTA's tiles, in order, wait until
// the staging buffer is free, stage the tile's row data with bulk copies,
// look up the next tile, wait for the tile's three predecessor sets, then
// release the buffer to the consumers.  Consumer warps: gather the neighbour
// state, update and store; the last warp of the tile to finish adds one to
// the set's counter with a release add, so a set of nt tiles is complete for
// sweep k once its counter reaches (k + 1) * nt.
template <class T, int MAXD>
__global__ void __launch_bounds__(kThreads, (gs_ctas_per_sm<T, MAXD>()))
    k_gs(const GsJob<T> *__restrict__ jobs, int njobs, int nrounds, unsigned long long wait_limit_ns,
         int *abort_flag, int *status) {
    constexpr int kEntStage = MAXD * TILE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Stage<T, MAXD> *stage = reinterpret_cast<Stage<T, MAXD> *>(smem_raw);
    __shared__ __align__(8) uint64_t full[2], empty[2];
    __shared__ int scur_job[kMaxJobs];   // producer: step cursor of each query
    for (int q = threadIdx.x; q < njobs; q += blockDim.x) scur_job[q] = 0;
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&full[b], 1);
            mbar_init(&empty[b], kCW);
            stage[b].finished = 0;
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grid = (int)gridDim.x, cta = (int)blockIdx.x;
    const int ncand = nrounds * njobs;   // candidates (r, q) in order; tile r * grid + cta of query q
    if (warp == 0) {
        // Producer warp.  Lane l looks up the l-th of the next 32 candidates
        // (one parallel lookup per 32); lane 0 then stages, waits and releases
        // the valid ones one by one.
        constexpr int DA = 16 / (int)sizeof(T);        // diagonal values per 16 bytes
        uint32_t eph[2] = {0u, 0u};
        int j = 0;
        for (int base = 0; base < ncand; base += 32) {
            const int cl = base + lane;
            const int ql = (cl < ncand) ? cl % njobs : 0;
            const int tl = (cl / njobs) * grid + cta;
            const bool vl = cl < ncand && tl < jobs[ql].ntickets;
            TileDesc dl{};
            int sl = 0, tidl = 0;
            if (vl) {
                int sc = scur_job[ql];
                lookup_tile(jobs[ql], tl, sc, dl, sl, tidl);
                atomicMax_block(&scur_job[ql], sc);   // the lane with the last tile of q sets it
            }
            __syncwarp();
            const unsigned vmask = __ballot_sync(0xffffffffu, vl);
            const int nwin = min(32, ncand - base);
            for (int w = 0; w < nwin; ++w) {
                if (!((vmask >> w) & 1u)) continue;
                TileDesc d;
                d.level = __shfl_sync(0xffffffffu, dl.level, w);
                d.start = __shfl_sync(0xffffffffu, dl.start, w);
                d.count = __shfl_sync(0xffffffffu, dl.count, w);
                d.lo = __shfl_sync(0xffffffffu, dl.lo, w);
                d.eb = __shfl_sync(0xffffffffu, dl.eb, w);
                d.ee = __shfl_sync(0xffffffffu, dl.ee, w);
                d.nt_prev = __shfl_sync(0xffffffffu, dl.nt_prev, w);
                d.nt_self = __shfl_sync(0xffffffffu, dl.nt_self, w);
                d.nt_next = __shfl_sync(0xffffffffu, dl.nt_next, w);
                const int s = __shfl_sync(0xffffffffu, sl, w);
                const int tile = __shfl_sync(0xffffffffu, tidl, w);
                const int q = __shfl_sync(0xffffffffu, ql, w);
                const GsJob<T> &J = jobs[q];
                (void)tile;
                int ok = 1;
                if (lane == 0) {
                    const int b = j & 1;
                    Stage<T, MAXD> &S = stage[b];
                    // predecessors: (k, i-1), (k-1, i), (k-1, i+1); their counters are
                    // read now, so the loads are in flight while the buffer frees up
                    int sb, k0;
                    step_band(s, J.band_steps, J.band, sb, k0);
                    const int i = d.level, k = k0 + ((sb - d.level) >> 1);
                    const int t0 = (i > 0) ? (k + 1) * d.nt_prev : 0;
                    const int t1 = (k > 0) ? k * d.nt_self : 0;
                    const int t2 = (k > 0) ? k * d.nt_next : 0;
                    const int32_t *c0 = J.done + (i > 0 ? i - 1 : 0), *c1 = J.done + i, *c2 = J.done + i + 1;
                    const int pv0 = (t0 > 0) ? ld_relaxed(c0) : 0;
                    const int pv1 = (t1 > 0) ? ld_relaxed(c1) : 0;
                    const int pv2 = (t2 > 0) ? ld_relaxed(c2) : 0;
                    if (j >= 2) {
                        if (!mbar_wait_bounded(&empty[b], eph[b], abort_flag)) {
                            atomicExch(abort_flag, 1);
                            atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
                            ok = 0;   // consumers time out on their own bounded waits
                        }
                        eph[b] ^= 1u;
                    }
                    if (ok) {
                        // the tile's row block (cp * W entries from a multiple of 32) and diagonal
                        const int cp = (d.count + 31) & ~31, nent = cp * d.ee;
                        const int d0 = d.start & ~(DA - 1), d1 = (d.start + d.count + DA - 1) & ~(DA - 1);
                        const int fits = nent <= kEntStage;
                        const uint32_t bd = (uint32_t)sizeof(T) * (d1 - d0);
                        const uint32_t be = fits ? (uint32_t)sizeof(Ent<T>) * nent : 0u;
                        fence_proxy_async();
                        mbar_expect_tx_only(&full[b], bd + be);
                        bulk_g2s(S.diag, J.diag + d0, bd, &full[b]);
                        if (be) bulk_g2s(S.ent, J.gent + d.eb, be, &full[b]);
                        S.start = d.start; S.count = d.count; S.lo = d.lo; S.k = k; S.level = i;
                        S.cp = cp; S.w = d.ee; S.d0 = d0; S.e0 = d.eb; S.fits = fits; S.q = q;
                        if (pv0 >= t0 && pv1 >= t1 && pv2 >= t2)
                            fence_acquire();
                        else
                            ok = wait_sets(c0, t0, c1, t1, c2, t2, wait_limit_ns, abort_flag, status) ? 1 : 0;
                        S.abort = ok ? 0 : 1;
                        mbar_arrive(&full[b]);
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) return;
                ++j;
            }
        }
        return;
    }
    // consumers
    const int cw = warp - 1;
    uint32_t fph[2] = {0u, 0u};
    int j = 0;
    for (int cand = 0; cand < ncand; ++cand) {
        if ((cand / njobs) * grid + cta >= jobs[cand % njobs].ntickets) continue;
        const int b = j & 1;
        ++j;
        Stage<T, MAXD> &S = stage[b];
        if (!mbar_wait_bounded(&full[b], fph[b], abort_flag)) {
            if (lane == 0) {
                atomicExch(abort_flag, 1);
                atomicCAS(status, DEV_OK, DEV_ETIMEOUT);
            }
            return;
        }
        fph[b] ^= 1u;
        if (S.abort) return;
        const int start = S.start, count = S.count, lo = S.lo, k = S.k, level = S.level;
        const int cp = S.cp, wt = S.w, sd = S.d0;
        const bool fits = S.fits != 0;
        const GsJob<T> &J = jobs[S.q];
        XVal<T> *Ucur = J.U[k & 1];
        const XVal<T> *Uprv = J.U[(k & 1) ^ 1];
        const Ent<T> *E = fits ? S.ent : J.gent + S.e0;   // the tile's row block
        // the tile's width picks how many entries of a row sit in registers,
        // so a tile of short rows does no arithmetic on padding (the skipped
        // terms are exact zeros: the result is the same)
        if (MAXD <= 6 && wt > MAXD) {
            // the host launches 6-entry stages only when no tile is wider
            if (lane == 0) {
                atomicExch(abort_flag, 1);
                atomicCAS(status, DEV_OK, DEV_EINTERNAL);
            }
            return;
        }
        if (wt <= 4)
            gs_tile_rows<T, 4, (MAXD > 6)>(Ucur, Uprv, E, S.diag, J.zero_pos, start, count, lo, cp, wt, sd, cw, lane);
        else if (MAXD <= 6 || wt <= 6)
            gs_tile_rows<T, 6, (MAXD > 6)>(Ucur, Uprv, E, S.diag, J.zero_pos, start, count, lo, cp, wt, sd, cw, lane);
        else
            gs_tile_rows<T, kMaxDeg>(Ucur, Uprv, E, S.diag, J.zero_pos, start, count, lo, cp, wt, sd, cw, lane);
        __syncwarp();
        if (lane == 0) {
            // the last warp of the tile publishes it with one release add
            __threadfence_block();
            const int before = atomicAdd(&S.finished, 1);
            if (before == kCW - 1) {
                S.finished = 0;
                __threadfence_block();
                red_release_add(&J.done[level], 1);
            }
            mbar_arrive(&empty[b]);
        }
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

// Sweeps per band.  A step of the plain wavefront holds a tile of up to
// half the sets (every set of its parity that some sweep is at), so on a
// mesh much larger than L2 a set's state and rows are evicted between one
// sweep's use and the next one's.  Bands of K sweeps hold K sets per step;
// K is chosen so that a step still has about kBandTiles tiles (its work then
// stays far above the latency of one dependent step), and bands are used
// only when there are four or more of them and the sets are large (at least
// kBandMinTiles tiles per set on average): measured on sinusoid icospheres,
// bands cut the launch by 5.5 % at 32 tiles per set (168M vertices) and by
// 3 % at 17 (42M), and lengthened it by 6.5 % at 9 (10.5M).
constexpr double kBandTiles = 6500.0;
constexpr double kBandMinTiles = 12.0;

// Bands of K sweeps take ceil(N / K) (L + 2 (K - 1)) steps; a band is widened
// (doubled) until that is at most kMaxSteps, which bounds the step table
// (8 bytes per step) whatever gs_band asks for.
constexpr long long kMaxSteps = 1ll << 26;

int gs_band(const QueryWs &w) {
    const int all = std::max(1, w.sweeps);
    int band;
    if (w.gs_band > 0) {
        band = std::min(w.gs_band, all);
    } else {
        const double tiles_per_set = ((double)w.nreach / TILE + w.nlev) / std::max(1, w.nlev);
        band = (int)std::ceil(kBandTiles / tiles_per_set);
        band = (tiles_per_set >= kBandMinTiles && 4.0 * band <= all) ? band : all;
    }
    while (band < all && (long long)((all + band - 1) / band) * (w.nlev + 2ll * (band - 1)) > kMaxSteps)
        band = (int)std::min<long long>(2ll * band, all);
    return band;
}

template <class T> gh_status run_gs_t(Ctx *c, std::vector<QueryWs *> &all_ws, cudaEvent_t ev0,
                                     cudaEvent_t ev1) {
    if ((int)all_ws.size() > kMaxJobs) {   // one launch per kMaxJobs queries
        for (size_t b = 0; b < all_ws.size(); b += kMaxJobs) {
            std::vector<QueryWs *> part(all_ws.begin() + b,
                                        all_ws.begin() + std::min(all_ws.size(), b + (size_t)kMaxJobs));
            gh_status s = run_gs_t<T>(c, part, b == 0 ? ev0 : nullptr,
                                      b + kMaxJobs >= all_ws.size() ? ev1 : nullptr);
            if (s != GH_OK) return s;
        }
        return GH_OK;
    }
    std::vector<QueryWs *> &ws = all_ws;
    cudaStream_t st = c->stream;
    const int K = (int)ws.size();
    int per_sm = 0;
    // 6-entry stages (4 resident CTAs per SM) when no tile of the launch is
    // wider than 6 entries (the icosphere meshes), else 8-entry stages (3)
    int maxw = 0;
    for (QueryWs *w : ws) maxw = std::max(maxw, w->max_w);
    const bool narrow = sizeof(T) == 4 && maxw <= 6;
    void *kfn = narrow ? (void *)k_gs<T, 6> : (void *)k_gs<T, kMaxDeg>;
    const size_t smem = narrow ? 2 * sizeof(Stage<T, 6>) : 2 * sizeof(Stage<T, kMaxDeg>);
    GH_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GH_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, smem));
    if (per_sm < 1) { set_error("diffusion kernel does not fit on an SM"); return GH_EDEVICE; }
    const int grid = std::max(1, per_sm * c->num_sms / std::max(1, c->gs_share));
    std::vector<GsJob<T>> jobs(K);
    std::vector<int> prev_buf(K);
    size_t soff_total = 0;
    for (int q = 0; q < K; ++q) {
        const int band = gs_band(*ws[q]);
        soff_total += (size_t)((ws[q]->sweeps + band - 1) / band) * (size_t)(ws[q]->nlev + 2 * (band - 1)) + 2;
    }
    int32_t *scratch = nullptr;   // per query: step counts and their prefix
    GH_CUDA(cudaMallocAsync((void **)&scratch, sizeof(int32_t) * 2 * soff_total, st));
    GsJob<T> *djobs = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&djobs, sizeof(GsJob<T>) * K, st));
    size_t at = 0;
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        GsJob<T> j{};
        j.nlev = w.nlev;
        j.nsweeps = w.sweeps;
        j.band = gs_band(w);
        j.band_steps = w.nlev + 2 * (j.band - 1);
        j.nsteps = ((w.sweeps + j.band - 1) / j.band) * j.band_steps;
        j.n_even = (w.nlev + 1) / 2;
        j.lvl_off = ptr<int32_t>(w.lvl_off);
        j.gent = ptr<Ent<T>>(w.gent);
        j.diag = ptr<T>(w.diag);
        j.ptile0 = ptr<int32_t>(w.ptile);
        j.ptile1 = ptr<int32_t>(w.ptile) + j.n_even + 1;
        j.tiles = ptr<TileDesc>(w.tiles);
        int32_t *soff = scratch + soff_total + at;
        at += (size_t)j.nsteps + 2;
        j.stepoff = soff;
        j.done = ptr<int32_t>(w.n1);
        j.U[0] = ptr<XVal<T>>(w.U0);
        j.U[1] = ptr<XVal<T>>(w.U1);
        j.zero_pos = w.nreach;
        jobs[q] = j;
        prev_buf[q] = w.final_buf;
        w.final_buf = (w.sweeps - 1) & 1;
    }
    GH_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(GsJob<T>) * K, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> ntick(K);
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        if (w.gs_continue) {
            // resume: both buffers hold the last state (the first sweep reads
            // its own and the next set's previous values from buffer 1, and
            // overwrites buffer 0 set by set before any later set reads it)
            GH_CUDA(cudaMemcpyAsync(jobs[q].U[prev_buf[q] ^ 1], jobs[q].U[prev_buf[q]], sizeof(XVal<T>) * (w.nreach + 1),
                                    cudaMemcpyDeviceToDevice, st));
        } else {
            k_zero_state<T><<<blocks_for(w.nreach + 1, 256), 256, 0, st>>>(jobs[q].U[0], jobs[q].U[1], w.nreach + 1);
            ++c->launches;
        }
        GH_CUDA(cudaMemsetAsync(jobs[q].done, 0, sizeof(int32_t) * (w.nlev + 1), st));
        int32_t *cnt = const_cast<int32_t *>(jobs[q].stepoff) - soff_total;
        k_step_counts<T><<<blocks_for(jobs[q].nsteps, 256), 256, 0, st>>>(djobs, q, cnt); ++c->launches;
        gh_status s = exclusive_scan_i32(c, cnt, const_cast<int32_t *>(jobs[q].stepoff), jobs[q].nsteps, &ntick[q]);
        if (s != GH_OK) { cudaFreeAsync(djobs, st); cudaFreeAsync(scratch, st); return s; }
        jobs[q].ntickets = ntick[q];
    }
    GH_CUDA(cudaMemcpyAsync(djobs, jobs.data(), sizeof(GsJob<T>) * K, cudaMemcpyHostToDevice, st));
    GH_CUDA(cudaMemsetAsync(&c->bar_dev->abort, 0, sizeof(int), st));
    int njobs = K;
    int maxtick = 0;
    for (int q = 0; q < K; ++q) maxtick = std::max(maxtick, ntick[q]);
    int nrounds = (maxtick + grid - 1) / grid;
    int *status = c->status_dev;
    int *abort_flag = &c->bar_dev->abort;
    unsigned long long wait_limit_ns = c->wait_limit_ns;
    void *argv[] = {(void *)&djobs,         (void *)&njobs,      (void *)&nrounds,
                    (void *)&wait_limit_ns, (void *)&abort_flag, (void *)&status};
    if (ev0) cudaEventRecord(ev0, st);
    cudaError_t e = cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads), argv, smem, st);
    ++c->launches;
    if (ev1) cudaEventRecord(ev1, st);
    cudaFreeAsync(djobs, st);
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the diffusion kernel");
    return GH_OK;
}

}  // namespace

gh_status run_gs(Ctx *c, std::vector<QueryWs *> &ws, cudaEvent_t ev0, cudaEvent_t ev1) {
    if (ws.empty()) return GH_OK;
    return ws[0]->fp64 ? run_gs_t<double>(c, ws, ev0, ev1) : run_gs_t<float>(c, ws, ev0, ev1);
}

}  // namespace gh
