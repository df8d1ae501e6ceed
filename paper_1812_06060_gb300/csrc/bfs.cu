// Breadth-first vertex sets and pairing (eq. VertexSets, Sec. 3.3, Sec. 5.2)
// and the per-query level-ordered layout the Gauss-Seidel kernel streams.
//
// The traversal reproduces a FIFO queue exactly: D_0 is the sorted source
// set; the rank of a vertex is its position in the queue; a vertex of D_{i+1}
// is discovered by its neighbour in D_i of lowest rank (the first one popped)
// and sits in the queue ordered by (rank of that parent, position in the
// parent's ascending one-ring).  Per set: every parent offers the key
// ((rank + 1) << 32 | slot) to each neighbour with a 64-bit atomicMin; a
// parent then counts the neighbours whose key is its own, an exclusive scan
// over the parents in rank order gives each parent's first child position.
// One thread-block cluster walks all sets of one query (one cluster per query
// of a batch).
#include <cooperative_groups.h>

#include <algorithm>

#include "internal.cuh"

namespace gh {

namespace {

constexpr int BT = 1024;

struct BfsArgs {
    const int32_t *rowptr;
    const int32_t *col;
    const int32_t *col_edge;
    int32_t *level;
    int32_t *parent;
    int32_t *pedge;
    int32_t *order;
    int32_t *rb, *re;       // row bounds of each queue entry, recorded when it is placed (scratch)
    unsigned long long *key;
    int32_t *lvl_off;
    int32_t *meta;
    int32_t n0;
    const int32_t *targets;  // optional: stop once all of these have a set (their paths are then complete)
    int32_t ntargets;
};

// the second level of this scan is one warp over the warps' totals: exactly
// 32 warps, one per lane (every lane reads and writes its entry of ws)
static_assert(BT == 1024, "bt_scan's second level assumes 32 warps per CTA");

__device__ int32_t bt_scan(int32_t v, int32_t &excl) {
    __shared__ int32_t ws[BT / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    excl = (wid ? ws[wid - 1] : 0) + x - v;
    int32_t total = ws[BT / 32 - 1];
    __syncthreads();
    return total;
}


// Keys: a vertex discovered by the parent of queue rank r through the
// parent's slot j holds ((r + 1) << 32 | j); sources hold 0 and undiscovered
// vertices the maximum, so no offer can equal a source's key.  A discovered
// vertex always holds a key below every key a later set offers, so the
// offers need no "already visited" test.
//
// One cluster of CL CTAs (8, or 16 where the device allows clusters that
// large) walks the sets of one query.  Each CTA owns a contiguous range of
// the current set's queue ranks (the ranges follow the CTA order).  Per set:
//   count:  every thread counts the children of its parents (the neighbours
//           whose key its parent holds), a block scan per chunk of BT ranks
//           gives the CTA's total, published in shared memory; cluster
//           barrier;
//   place:  each CTA reads the lower-ranked CTAs' totals through distributed
//           shared memory and writes its children in rank order (queue
//           entry, set, pairing vertex and edge); the children a
//           CTA placed are the parents it owns in the next set, so after a
//           CTA barrier it records their row bounds and offers their keys to
//           their neighbours (64-bit atomicMin) without waiting for the other
//           CTAs; cluster barrier.
// When the ownership grows lopsided (the busiest CTA would own more than 64
// parents above an even share, or need more chunks of BT parents: a single
// source starts in one CTA, and a set's time follows its busiest CTA), the
// set is split evenly instead, after one more cluster barrier.  Every prefix
// involved runs in rank order, so the queue is exactly the FIFO order.

__device__ __forceinline__ unsigned long long bfs_key(int r, int slot) {
    return ((unsigned long long)(unsigned)(r + 1) << 32) | (unsigned)slot;
}

// The slot loops below take a row kSlotBatch slots at a time, loading all of
// a batch's neighbours before the dependent key loads or atomics, so a row
// costs one round trip per level of the load chain rather than one per slot.
constexpr int kSlotBatch = 8;

// children of parent rank r (row [b, e)) among slots [from, e): their count;
// the first 32 slots are marked in mk
__device__ __forceinline__ int bfs_children(const BfsArgs &a, int r, int b, int from, int e, unsigned &mk) {
    int k = 0;
    for (int j0 = from; j0 < e; j0 += kSlotBatch) {
        int w[kSlotBatch];
        unsigned long long kv[kSlotBatch];
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) w[u] = j0 + u < e ? __ldg(&a.col[j0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) kv[u] = w[u] >= 0 ? __ldcg(&a.key[w[u]]) : 0ull;
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) {
            const int sl = j0 + u - b;
            if (w[u] >= 0 && kv[u] == bfs_key(r, sl)) {
                ++k;
                if (sl < 32) mk |= 1u << sl;
            }
        }
    }
    return k;
}

__device__ __forceinline__ void bfs_offer(const BfsArgs &a, int r, int b, int from, int e) {
    for (int j0 = from; j0 < e; j0 += kSlotBatch) {
        int w[kSlotBatch];
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) w[u] = j0 + u < e ? __ldg(&a.col[j0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u)
            if (w[u] >= 0) atomicMin(&a.key[w[u]], bfs_key(r, j0 + u - b));
    }
}

// A child placed at queue position at is, unless the next set is split
// evenly, a parent of the placing CTA in the next set, at rank at - nbase of
// the CTA's range; the first BT of them are also kept in shared memory, so
// the next set's held rows need no round trip to L2.
struct NextRow {
    int v, b, e;
};

// writes one child w (pairing vertex p, pairing edge ce) at queue position
// at, with its row bounds (loaded here, in the round trip of the edge id)
__device__ __forceinline__ void bfs_put(const BfsArgs &a, int nlev, int p, int w, int ce, int rb, int re, int at,
                                        NextRow *sn, int nbase) {
    a.order[at] = w;
    a.rb[at] = rb;
    a.re[at] = re;
    a.level[w] = nlev;
    a.parent[w] = p;
    a.pedge[w] = ce;
    if ((unsigned)(at - nbase) < (unsigned)BT) sn[at - nbase] = NextRow{w, rb, re};
}

// writes the children of parent p (rank r, row [b, e)) among slots [from, e)
// from queue position at on; returns the next position
__device__ __forceinline__ int bfs_place(const BfsArgs &a, int nlev, int p, int r, int b, int from, int e,
                                         unsigned mk, int at, NextRow *sn, int nbase) {
    for (int j0 = from; j0 < e; j0 += kSlotBatch) {
        int w[kSlotBatch];
        bool ch[kSlotBatch];
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) w[u] = j0 + u < e ? __ldg(&a.col[j0 + u]) : -1;
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) {
            const int sl = j0 + u - b;
            ch[u] = w[u] >= 0 && (sl < 32 ? ((mk >> sl) & 1u) != 0 : __ldcg(&a.key[w[u]]) == bfs_key(r, sl));
        }
        int ce[kSlotBatch], cb[kSlotBatch], cx[kSlotBatch];   // all loads first: one round trip
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) {
            ce[u] = ch[u] ? __ldg(&a.col_edge[j0 + u]) : 0;
            cb[u] = ch[u] ? __ldg(&a.rowptr[w[u]]) : 0;
            cx[u] = ch[u] ? __ldg(&a.rowptr[w[u] + 1]) : 0;
        }
#pragma unroll
        for (int u = 0; u < kSlotBatch; ++u) {
            if (ch[u]) {
                bfs_put(a, nlev, p, w[u], ce[u], cb[u], cx[u], at, sn, nbase);
                ++at;
            }
        }
    }
    return at;
}

// A thread's first parent of the current set (rank plo + threadIdx.x) stays
// in registers from its offers to its placement: the vertex, its row and the
// row's first kSlotBatch neighbours (after the count: the children among
// them, else -1).
struct Held {
    int v, b, e;
    int w[kSlotBatch];
};

// offers of rank r (its row bounds recorded at placement, or its entry of
// the placing CTA's shared copy sn when own); the first slots are kept in h
__device__ __forceinline__ void bfs_offer_held(const BfsArgs &a, int r, Held &h, const NextRow *sn, bool own) {
    if (own) {
        const NextRow x = sn[threadIdx.x];
        h.v = x.v;
        h.b = x.b;
        h.e = x.e;
    } else {
        h.v = __ldcg(&a.order[r]);
        h.b = __ldcg(&a.rb[r]);
        h.e = __ldcg(&a.re[r]);
    }
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) h.w[u] = h.b + u < h.e ? __ldg(&a.col[h.b + u]) : -1;
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u)
        if (h.w[u] >= 0) atomicMin(&a.key[h.w[u]], bfs_key(r, u));
    if (h.e > h.b + kSlotBatch) bfs_offer(a, r, h.b, h.b + kSlotBatch, h.e);
}

// the offers of the parents [plo, phi) of the next set (own: the CTA placed
// them, and sn holds its shared copy of their first BT rows)
__device__ __forceinline__ void bfs_offer_set(const BfsArgs &a, int plo, int phi, Held &h, const NextRow *sn,
                                              bool own) {
    h.v = -1;
    h.b = h.e = 0;
#pragma unroll
    for (int u = 0; u < kSlotBatch; ++u) h.w[u] = -1;
    if (plo + (int)threadIdx.x < phi) bfs_offer_held(a, plo + (int)threadIdx.x, h, sn, own);
    for (int r = plo + (int)threadIdx.x + BT; r < phi; r += BT) {
        const int b = __ldcg(&a.rb[r]), e = __ldcg(&a.re[r]);
        bfs_offer(a, r, b, b, e);
    }
}

template <int CL> __global__ void __launch_bounds__(BT, 1) k_bfs(const BfsArgs *__restrict__ all) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    // the arguments stay in shared memory: registers go to the held rows
    __shared__ BfsArgs s_args;
    __shared__ int s_tot[CL];   // this set's children per CTA of the cluster
    __shared__ NextRow s_next[BT];
    if (threadIdx.x == 0) s_args = all[blockIdx.x / CL];
    __syncthreads();
    const BfsArgs &a = s_args;
    int hi = a.n0, nlev = 1;
    if (crank == 0 && threadIdx.x == 0) a.lvl_off[0] = 0;
    Held h;
    // the sources, split evenly
    int plo, phi;
    {
        const int per = (a.n0 + CL - 1) / CL;
        plo = min(a.n0, crank * per);
        phi = min(a.n0, plo + per);
        for (int r = plo + (int)threadIdx.x; r < phi; r += BT) {
            const int v = a.order[r];
            a.rb[r] = a.rowptr[v];
            a.re[r] = a.rowptr[v + 1];
        }
        __syncthreads();
        bfs_offer_set(a, plo, phi, h, s_next, false);
    }
    cluster.sync();
    while (true) {
        // count: the children of this CTA's parents [plo, phi); chunk 0 from
        // the held rows, whose children and their edges stay held
        const int nchunk = (phi - plo + BT - 1) / BT;
        int k0 = 0, ex0 = 0, tot0 = 0;
        unsigned mk0 = 0;
        int mytotal = 0;
        for (int c = 0; c < nchunk; ++c) {
            const int r = plo + c * BT + (int)threadIdx.x;
            int k = 0;
            unsigned mk = 0;
            if (c == 0) {
                unsigned long long kv[kSlotBatch];
#pragma unroll
                for (int u = 0; u < kSlotBatch; ++u) kv[u] = h.w[u] >= 0 ? __ldcg(&a.key[h.w[u]]) : 0ull;
#pragma unroll
                for (int u = 0; u < kSlotBatch; ++u) {
                    if (h.w[u] >= 0 && kv[u] == bfs_key(r, u)) {
                        ++k;
                        mk |= 1u << u;
                    } else {
                        h.w[u] = -1;
                    }
                }
                if (h.e > h.b + kSlotBatch) k += bfs_children(a, r, h.b, h.b + kSlotBatch, h.e, mk);
            } else if (r < phi) {
                k = bfs_children(a, r, __ldcg(&a.rb[r]), __ldcg(&a.rb[r]), __ldcg(&a.re[r]), mk);
            }
            int excl;
            const int tot = bt_scan(k, excl);
            if (c == 0) { k0 = k; ex0 = excl; tot0 = tot; mk0 = mk; }
            mytotal += tot;
        }
        // every CTA's total goes to every CTA's shared memory before the
        // barrier (remote stores; the barrier publishes them), so after it the
        // totals are local: lane q of every warp reads CTA q's, shuffles sum them
        if ((int)threadIdx.x < CL) *cluster.map_shared_rank(&s_tot[crank], (int)threadIdx.x) = mytotal;
        cluster.sync();
        int before, total, most;
        {
            const int lane = (int)(threadIdx.x & 31);
            const int t = lane < CL ? s_tot[lane] : 0;
            before = lane < crank ? t : 0;
            total = t;
            most = t;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                before += __shfl_xor_sync(0xffffffffu, before, o);
                total += __shfl_xor_sync(0xffffffffu, total, o);
                most = max(most, __shfl_xor_sync(0xffffffffu, most, o));
            }
        }
        if (total == 0) {
            cluster.sync();   // no CTA leaves while another reads its shared memory
            break;
        }
        // place the children: queue position hi + before + (children of this
        // CTA's earlier chunks) + (earlier parents of the chunk)
        const int nbase = hi + before;
        if (k0) {
            int at = hi + before + ex0;
            int ce[kSlotBatch], cb[kSlotBatch], cx[kSlotBatch];   // all loads first: one round trip
#pragma unroll
            for (int u = 0; u < kSlotBatch; ++u) {
                const bool ch = h.w[u] >= 0;
                ce[u] = ch ? __ldg(&a.col_edge[h.b + u]) : 0;
                cb[u] = ch ? __ldg(&a.rowptr[h.w[u]]) : 0;
                cx[u] = ch ? __ldg(&a.rowptr[h.w[u] + 1]) : 0;
            }
#pragma unroll
            for (int u = 0; u < kSlotBatch; ++u) {
                if (h.w[u] >= 0) {
                    bfs_put(a, nlev, h.v, h.w[u], ce[u], cb[u], cx[u], at, s_next, nbase);
                    ++at;
                }
            }
            if (h.e > h.b + kSlotBatch)
                bfs_place(a, nlev, h.v, plo + (int)threadIdx.x, h.b, h.b + kSlotBatch, h.e, mk0, at, s_next, nbase);
        }
        int base_run = tot0;
        for (int c = 1; c < nchunk; ++c) {
            const int r = plo + c * BT + (int)threadIdx.x;
            int p = -1, b = 0, e = 0, k = 0, excl = 0;
            unsigned mk = 0;
            if (r < phi) {
                p = __ldcg(&a.order[r]);
                b = __ldcg(&a.rb[r]);
                e = __ldcg(&a.re[r]);
                k = bfs_children(a, r, b, b, e, mk);
            }
            const int tot = bt_scan(k, excl);
            if (k) bfs_place(a, nlev, p, r, b, b, e, mk, hi + before + base_run + excl, s_next, nbase);
            base_run += tot;
        }
        // the next set's parents of this CTA: its own children, or an even
        // split when the ownership is lopsided
        const int per = (total + CL - 1) / CL;
        bool own = false;
        if (most - per > 64 || (most + BT - 1) / BT > (per + BT - 1) / BT) {
            cluster.sync();   // every CTA's children are written
            plo = min(hi + total, hi + crank * per);
            phi = min(hi + total, plo + per);
        } else {
            __syncthreads();  // this CTA's children are written (and their shared copies)
            plo = nbase;
            phi = plo + mytotal;
            own = true;
        }
        bfs_offer_set(a, plo, phi, h, s_next, own);
        cluster.sync();
        if (crank == 0 && threadIdx.x == 0) a.lvl_off[nlev] = hi;
        ++nlev;
        hi += total;
        if (a.ntargets > 0) {   // every thread reads the same values after the barrier: a uniform decision
            bool all = true;
            for (int i = 0; i < a.ntargets; ++i) all = all && __ldcg(&a.level[a.targets[i]]) >= 0;
            if (all) break;
        }
    }
    if (crank == 0 && threadIdx.x == 0) {
        a.lvl_off[nlev] = hi;
        a.meta[0] = nlev;
        a.meta[1] = hi;
    }
}

// sources: set 0, key 0
__global__ void k_seed(int32_t *level, unsigned long long *key, const int32_t *order, int n0) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n0) {
        level[order[i]] = 0;
        key[order[i]] = 0ull;
    }
}

__global__ void k_pos(const int32_t *__restrict__ order, int n, int32_t *pos) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) pos[order[r]] = r;
}

__global__ void k_row_len(const int32_t *__restrict__ order, int n, const int32_t *__restrict__ rowptr, int32_t *len) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) {
        int v = order[r];
        len[r] = rowptr[v + 1] - rowptr[v];
    }
}

// Layout order.  The rows of one set are updated together from the previous
// sweep's values of their own set (eq. HeatDiffusionUpdate), so their positions
// may be permuted freely: each row keeps its entries in their order and every
// iterate stays the same.  The layout stable-partitions each set into the rows
// of at most `split` entries, then the longer ones, so a tile of short rows is
// not padded to the longest row of its set (on a grid whose vertices
// alternate between 4 and 8 neighbours, half the tiles drop from width 8 to 4).
constexpr int kLenBins = 32;   // row lengths >= kLenBins - 1 share the last bin

__global__ void k_len_hist(const int32_t *__restrict__ len, int n, int32_t *hist) {
    __shared__ int32_t h[kLenBins];
    if (threadIdx.x < kLenBins) h[threadIdx.x] = 0;
    __syncthreads();
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        atomicAdd(&h[min(len[r], kLenBins - 1)], 1);
    __syncthreads();
    if (threadIdx.x < kLenBins && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// the split that minimises the padded entries when the short part is padded
// to `split` and the long part to the longest row (one thread; kLenBins bins)
__global__ void k_pick_split(const int32_t *__restrict__ hist, int32_t *split) {
    if (threadIdx.x != 0) return;
    int lmax = 0;
    int64_t n = 0;
    for (int b = 0; b < kLenBins; ++b) {
        n += hist[b];
        if (hist[b]) lmax = b;
    }
    int best = lmax;
    int64_t best_cost = n * lmax, below = 0;
    for (int b = 0; b < lmax; ++b) {
        below += hist[b];
        if (!hist[b]) continue;
        const int64_t cost = below * b + (n - below) * lmax;
        if (cost < best_cost) {
            best_cost = cost;
            best = b;
        }
    }
    *split = best;
}

__global__ void k_split_flag(const int32_t *__restrict__ len, int n, const int32_t *__restrict__ split, int32_t *flag) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) flag[r] = len[r] > *split ? 1 : 0;
}

// lorder: the set's short rows in queue order, then its long rows in queue
// order; nlong_before is the exclusive scan of the long-row flags (n + 1 values)
__global__ void k_split_scatter(const int32_t *__restrict__ order, int n, const int32_t *__restrict__ level,
                                const int32_t *__restrict__ lvl_off, const int32_t *__restrict__ flag,
                                const int32_t *__restrict__ nlong_before, int32_t *lorder) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int v = order[r], s = level[v];
    const int b = lvl_off[s], e = lvl_off[s + 1];
    const int before = nlong_before[r] - nlong_before[b];
    const int nlong = nlong_before[e] - nlong_before[b];
    lorder[flag[r] ? e - nlong + before : r - before] = v;
}

// Level-ordered operator, one block per tile in column-major ("ELL") order:
// entry a of the row at tile position p (layout position start + p) sits at
// gent[eb + a * cp + p], cp = count rounded up to 32, for a < W (the tile's
// longest row); the entries of a row are its neighbours in ascending order,
// renumbered to layout positions, with weight t*theta, and (zero slot n, 0)
// past the row's end and in the padding columns.  A warp reading entry a of
// 32 consecutive rows touches 32 consecutive entries.  idiag = 1 / (A_v +
// t * sum theta) (FP64, then rounded).  A neighbour without a layout position
// would mean inconsistent breadth-first sets: it is pointed at the zero slot
// and the status word reports it.

// widest row of each tile (one warp per tile); wsize[t] = W * cp
__global__ void k_tile_width(const int32_t *__restrict__ ptile, int n_even, int n_odd, int tiles_cap,
                             const int32_t *__restrict__ len, TileDesc *tiles, int32_t *wsize, int32_t *maxw) {
    const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (t >= tiles_cap) return;
    const int ntiles = ptile[n_even] + ptile[n_even + 1 + n_odd];
    if (t >= ntiles) {
        if (lane == 0) wsize[t] = 0;
        return;
    }
    const int start = tiles[t].start, count = tiles[t].count;
    int w = 0;
    for (int p = lane; p < count; p += 32) w = max(w, len[start + p]);
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (lane == 0) {
        tiles[t].ee = w;
        wsize[t] = w * ((count + 31) & ~31);
        atomicMax(maxw, w);
    }
}

template <class T>
__global__ void __launch_bounds__(TILE) k_fill_ell(const int32_t *__restrict__ ptile, int n_even, int n_odd,
                                                  const int32_t *__restrict__ order, int n,
                                                  const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                  const int32_t *__restrict__ col_edge,
                                                  const double *__restrict__ theta, const double *__restrict__ Av,
                                                  const int32_t *__restrict__ pos, const int32_t *__restrict__ eoff,
                                                  double t, TileDesc *tiles, Ent<T> *gent, T *diag, int *status) {
    const int ti = blockIdx.x;
    const int ntiles = ptile[n_even] + ptile[n_even + 1 + n_odd];
    if (ti >= ntiles) return;
    const int start = tiles[ti].start, count = tiles[ti].count, W = tiles[ti].ee;
    const int cp = (count + 31) & ~31;
    const int64_t base = eoff[ti];
    const int p = threadIdx.x;
    if (p == 0) tiles[ti].eb = (int)base;
    if (p >= cp) return;
    int a = 0;
    if (p < count) {
        const int r = start + p;
        const int v = order[r];
        const int b = rowptr[v], e = rowptr[v + 1];
        double sum = 0.0;
        for (int j = b; j < e; ++j, ++a) {
            const double th = theta[col_edge[j]];
            sum += th;
            Ent<T> x;
            x.col = pos[col[j]];
            if (x.col < 0) {   // a neighbour of a reached vertex is always reached
                atomicCAS(status, DEV_OK, DEV_EINTERNAL);
                x.col = n;     // the zero slot
            }
            x.w = (T)(t * th);
            gent[base + (int64_t)a * cp + p] = x;
        }
        diag[r] = (T)(1.0 / (Av[v] + t * sum));
    }
    for (; a < W; ++a) {
        Ent<T> z;
        z.col = n;
        z.w = T(0);
        gent[base + (int64_t)a * cp + p] = z;
    }
}

// tiles of at most TILE layout positions inside one set, listed set by set,
// even sets first, then odd sets; ptile holds, per parity, the running tile
// count before each set of that parity
__device__ __forceinline__ int ntiles_of(const int32_t *lvl_off, int nlev, int i) {
    return (i < 0 || i >= nlev) ? 0 : (lvl_off[i + 1] - lvl_off[i] + TILE - 1) / TILE;
}

__global__ void __launch_bounds__(BT) k_tiles(const int32_t *__restrict__ lvl_off, int nlev, int32_t *ptile,
                                              TileDesc *tiles) {
    int n_even = (nlev + 1) / 2, n_odd = nlev / 2;
    int32_t *p0 = ptile, *p1 = ptile + n_even + 1;
    for (int par = 0; par < 2; ++par) {
        int nl = par ? n_odd : n_even;
        int32_t *pp = par ? p1 : p0;
        int carry = 0;
        for (int c0 = 0; c0 < nl; c0 += BT) {
            int j = c0 + threadIdx.x;
            int cnt = (j < nl) ? ntiles_of(lvl_off, nlev, par + 2 * j) : 0;
            int excl;
            int tot = bt_scan(cnt, excl);
            if (j < nl) pp[j] = carry + excl;
            carry += tot;
        }
        if (threadIdx.x == 0) pp[nl] = carry;
        __syncthreads();
    }
    int base1 = p0[n_even];
    for (int i = threadIdx.x; i < nlev; i += BT) {
        int par = i & 1, j = i >> 1;
        int first = (par ? base1 + p1[j] : p0[j]);
        int s = lvl_off[i], e = lvl_off[i + 1];
        int ntp = ntiles_of(lvl_off, nlev, i - 1), nts = ntiles_of(lvl_off, nlev, i), ntn = ntiles_of(lvl_off, nlev, i + 1);
        for (int k = 0; s + k * TILE < e; ++k) {
            TileDesc d;
            d.level = i;
            d.start = s + k * TILE;
            d.count = min(TILE, e - d.start);
            d.lo = s;
            d.eb = d.ee = 0;   // entry block and width: k_tile_width, k_fill_ell
            d.nt_prev = ntp;
            d.nt_self = nts;
            d.nt_next = ntn;
            d.pad0 = d.pad1 = d.pad2 = 0;
            tiles[first + k] = d;
        }
    }
}

}  // namespace

namespace {

template <int CL> cudaError_t launch_bfs(const BfsArgs *dargs, int K, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(K * CL);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_bfs<CL>, dargs);
}

// can clusters of CL CTAs of BT threads be placed on this device at all?
template <int CL> bool bfs_cluster_fits() {
    if (CL > 8 && cudaFuncSetAttribute(k_bfs<CL>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(BT);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_bfs<CL>, &cfg) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return n > 0;
}

}  // namespace

bool bfs_cluster_supported(int cl) {
    if (cl == 8) return bfs_cluster_fits<8>();
    if (cl == 16) return bfs_cluster_fits<16>();
    return false;
}

// One breadth-first launch for all queries (query q on mesh *mq[q]), with
// clusters of `cl` CTAs.
static gh_status run_bfs_once(Ctx *c, std::vector<DevMesh *> &mq, std::vector<QueryWs *> &ws,
                              const std::vector<std::vector<int32_t>> &src, int cl,
                              const std::vector<const int32_t *> *targets = nullptr,
                              const std::vector<int32_t> *ntargets = nullptr) {
    cudaStream_t st = c->stream;
    int K = (int)src.size();
    std::vector<BfsArgs> args(K);
    for (int q = 0; q < K; ++q) {
        QueryWs &w = *ws[q];
        const DevMesh &m = *mq[q];
        GH_CUDA(cudaMemsetAsync(w.level.p, 0xff, sizeof(int32_t) * m.nv, st));
        GH_CUDA(cudaMemsetAsync(w.parent.p, 0xff, sizeof(int32_t) * m.nv, st));
        GH_CUDA(cudaMemsetAsync(w.key.p, 0xff, sizeof(unsigned long long) * m.nv, st));
        GH_CUDA(cudaMemcpyAsync(w.order.p, src[q].data(), sizeof(int32_t) * src[q].size(), cudaMemcpyHostToDevice, st));
        k_seed<<<blocks_for((int64_t)src[q].size(), 256), 256, 0, st>>>(ptr<int32_t>(w.level), ptr<unsigned long long>(w.key), ptr<int32_t>(w.order),
                                                                       (int)src[q].size()); ++c->launches;
        // pos and n0 are free until the layout is built: they hold the row bounds
        args[q] = BfsArgs{ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col), ptr<int32_t>(m.col_edge), ptr<int32_t>(w.level),
                          ptr<int32_t>(w.parent), ptr<int32_t>(w.pedge), ptr<int32_t>(w.order),
                          ptr<int32_t>(w.pos), ptr<int32_t>(w.n0),
                          ptr<unsigned long long>(w.key), ptr<int32_t>(w.lvl_off), ptr<int32_t>(w.meta),
                          (int32_t)src[q].size(), targets ? (*targets)[q] : nullptr, ntargets ? (*ntargets)[q] : 0};
    }
    BfsArgs *dargs = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&dargs, sizeof(BfsArgs) * K, st));
    GH_CUDA(cudaMemcpyAsync(dargs, args.data(), sizeof(BfsArgs) * K, cudaMemcpyHostToDevice, st));
    cudaError_t le0 = (cl == 16) ? launch_bfs<16>(dargs, K, st) : launch_bfs<8>(dargs, K, st);
    ++c->launches;
    cudaError_t le = (le0 != cudaSuccess) ? le0 : cudaGetLastError();
    cudaFreeAsync(dargs, st);
    if (le != cudaSuccess) return cuda_fail(le, "cluster launch of k_bfs");
    std::vector<int32_t> meta(2 * K);
    for (int q = 0; q < K; ++q)
        GH_CUDA(cudaMemcpyAsync(&meta[2 * q], ws[q]->meta.p, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GH_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < K; ++q) {
        ws[q]->nlev = meta[2 * q];
        ws[q]->nreach = meta[2 * q + 1];
    }
    return GH_OK;
}

gh_status run_bfs_fixed(Ctx *c, std::vector<DevMesh *> &mq, std::vector<QueryWs *> &ws,
                        const std::vector<std::vector<int32_t>> &src, int cl,
                        const std::vector<const int32_t *> *targets, const std::vector<int32_t> *ntargets) {
    return run_bfs_once(c, mq, ws, src, cl, targets, ntargets);
}

// The breadth-first sets of every query.  The cluster size is tuned per mesh,
// separately for single queries and batches: the first solve of each kind
// runs every size the device supports, timed with events (a second,
// alternating round when the first is close), and keeps the fastest (all sizes give the same sets and order, so the last run's
// result is the solve's).  A batch over several meshes uses clusters of 8.
gh_status run_bfs(Ctx *c, std::vector<DevMesh *> &mq, std::vector<QueryWs *> &ws,
                  const std::vector<std::vector<int32_t>> &src) {
    for (DevMesh *x : mq)
        if (x != mq[0]) return run_bfs_once(c, mq, ws, src, 8);
    DevMesh &m = *mq[0];
    const int kind = src.size() > 1 ? 1 : 0;
    int cl;
    {
        std::lock_guard<std::mutex> lk(*m.rec_mu);
        cl = m.bfs_cluster[kind];
    }
    if (cl != 0) return run_bfs_once(c, mq, ws, src, cl);
    std::vector<int> cand = {8};
    if (bfs_cluster_supported(16)) cand.push_back(16);
    cudaEvent_t e0, e1;
    GH_CUDA(cudaEventCreate(&e0));
    GH_CUDA(cudaEventCreate(&e1));
    // up to two alternating rounds, each candidate's faster run counting: the
    // first launch of a solve runs on cold caches and can bias one round; the
    // second round runs only when the first is within 15 %
    std::vector<float> best_ms(cand.size(), 0.0f);
    gh_status s = GH_OK;
    for (int round = 0; round < 2 && s == GH_OK; ++round) {
        if (round == 1) {
            const float lo = *std::min_element(best_ms.begin(), best_ms.end());
            const float hi = *std::max_element(best_ms.begin(), best_ms.end());
            if (hi > 1.15f * lo) break;
        }
        for (size_t i = 0; i < cand.size(); ++i) {
            cudaEventRecord(e0, c->stream);
            if ((s = run_bfs_once(c, mq, ws, src, cand[i])) != GH_OK) break;   // synchronises the stream
            cudaEventRecord(e1, c->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (round == 0 || ms < best_ms[i]) best_ms[i] = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != GH_OK) return s;
    int best = cand[0];
    float best_t = best_ms[0];
    for (size_t i = 1; i < cand.size(); ++i)
        if (best_ms[i] < best_t) { best_t = best_ms[i]; best = cand[i]; }
    std::lock_guard<std::mutex> lk(*m.rec_mu);
    if (m.bfs_cluster[kind] == 0) m.bfs_cluster[kind] = best;
    return GH_OK;
}

gh_status build_layout(Ctx *c, const DevMesh &m, QueryWs &q, double t) {
    cudaStream_t st = c->stream;
    int n = q.nreach;
    const size_t tiles_cap = (size_t)n / TILE + (size_t)q.nlev + 2;
    gh_status s;
    if ((s = dalloc(c, q.tiles, sizeof(TileDesc) * tiles_cap)) != GH_OK) return s;
    if ((s = dalloc(c, q.twid, sizeof(int32_t) * std::max<size_t>(2 * tiles_cap + 2, kLenBins + 1))) != GH_OK) return s;
    int32_t *len = ptr<int32_t>(q.n0);
    k_row_len<<<blocks_for(n, 256), 256, 0, st>>>(ptr<int32_t>(q.order), n, ptr<int32_t>(m.rowptr), len); ++c->launches;
    {
        // the layout order: each set's short rows, then its long ones (histogram
        // and split in twid, the flags' scan (n + 1 values) in the traversal's
        // key buffer, free now)
        int32_t *hist = ptr<int32_t>(q.twid), *split = hist + kLenBins, *flag = ptr<int32_t>(q.n1);
        int32_t *nlong = reinterpret_cast<int32_t *>(ptr<unsigned long long>(q.key));
        GH_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * kLenBins, st));
        k_len_hist<<<std::min(blocks_for(n, 256), 4u * 152u), 256, 0, st>>>(len, n, hist); ++c->launches;
        k_pick_split<<<1, 32, 0, st>>>(hist, split); ++c->launches;
        k_split_flag<<<blocks_for(n, 256), 256, 0, st>>>(len, n, split, flag); ++c->launches;
        if ((s = exclusive_scan_u32_dev(c, flag, nlong, n)) != GH_OK) return s;
        k_split_scatter<<<blocks_for(n, 256), 256, 0, st>>>(ptr<int32_t>(q.order), n, ptr<int32_t>(q.level),
                                                           ptr<int32_t>(q.lvl_off), flag, nlong,
                                                           ptr<int32_t>(q.lorder)); ++c->launches;
    }
    GH_CUDA(cudaMemsetAsync(q.pos.p, 0xff, sizeof(int32_t) * m.nv, st));
    k_pos<<<blocks_for(n, 256), 256, 0, st>>>(ptr<int32_t>(q.lorder), n, ptr<int32_t>(q.pos)); ++c->launches;
    k_row_len<<<blocks_for(n, 256), 256, 0, st>>>(ptr<int32_t>(q.lorder), n, ptr<int32_t>(m.rowptr), len); ++c->launches;
    k_tiles<<<1, BT, 0, st>>>(ptr<int32_t>(q.lvl_off), q.nlev, ptr<int32_t>(q.ptile), ptr<TileDesc>(q.tiles)); ++c->launches;
    const int n_even = (q.nlev + 1) / 2, n_odd = q.nlev / 2;
    int32_t *wsize = ptr<int32_t>(q.twid), *eoff = wsize + tiles_cap + 1;
    int32_t *maxw_dev = ptr<int32_t>(q.meta) + 3;
    GH_CUDA(cudaMemsetAsync(maxw_dev, 0, sizeof(int32_t), st));
    k_tile_width<<<blocks_for((int64_t)tiles_cap * 32, 256), 256, 0, st>>>(ptr<int32_t>(q.ptile), n_even, n_odd,
                                                                       (int)tiles_cap, len, ptr<TileDesc>(q.tiles),
                                                                       wsize, maxw_dev); ++c->launches;
    GH_CUDA(cudaGetLastError());
    // read back with the scan's total (the scan waits for the stream)
    GH_CUDA(cudaMemcpyAsync(&q.max_w, maxw_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    int32_t total = 0;
    if ((s = exclusive_scan_i32(c, wsize, eoff, (int64_t)tiles_cap, &total)) != GH_OK) return s;
    const size_t es = q.fp64 ? sizeof(Ent<double>) : sizeof(Ent<float>);
    if ((s = dalloc(c, q.gent, es * ((size_t)total + 4))) != GH_OK) return s;
    if (q.fp64) {
        k_fill_ell<double><<<(unsigned)tiles_cap, TILE, 0, st>>>(
            ptr<int32_t>(q.ptile), n_even, n_odd, ptr<int32_t>(q.lorder), n, ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col),
            ptr<int32_t>(m.col_edge), ptr<double>(m.theta), ptr<double>(m.Av), ptr<int32_t>(q.pos), eoff, t,
            ptr<TileDesc>(q.tiles), ptr<Ent<double>>(q.gent), ptr<double>(q.diag), c->status_dev); ++c->launches;
    } else {
        k_fill_ell<float><<<(unsigned)tiles_cap, TILE, 0, st>>>(
            ptr<int32_t>(q.ptile), n_even, n_odd, ptr<int32_t>(q.lorder), n, ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col),
            ptr<int32_t>(m.col_edge), ptr<double>(m.theta), ptr<double>(m.Av), ptr<int32_t>(q.pos), eoff, t,
            ptr<TileDesc>(q.tiles), ptr<Ent<float>>(q.gent), ptr<float>(q.diag), c->status_dev); ++c->launches;
    }
    GH_CUDA(cudaGetLastError());
    q.t = t;
    return GH_OK;
}

}  // namespace gh
