// Internal declarations of the geoheat CUDA library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/geoheat.h"

namespace gh {

// ---------------------------------------------------------------- errors

// device-side error codes written to a status word by kernels
enum DevErr : int {
    DEV_OK = 0,
    DEV_EINVAL = 1,
    DEV_ENONMANIFOLD = 2,
    DEV_ETIMEOUT = 3,
    DEV_EINTERNAL = 4,   // an internal consistency check failed (the access was redirected, not made)
};

void set_error(const std::string &msg);
gh_status cuda_fail(cudaError_t e, const char *what);

#define GH_CUDA(call)                                                  \
    do {                                                               \
        cudaError_t _e = (call);                                       \
        if (_e != cudaSuccess) return ::gh::cuda_fail(_e, #call);      \
    } while (0)

// ---------------------------------------------------------------- memory

struct Ctx;

// device allocation charged to the context's budget
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

gh_status dalloc(Ctx *c, DBuf &b, size_t bytes);
void dfree(Ctx *c, DBuf &b);

template <class X>
inline X *ptr(const DBuf &b) { return static_cast<X *>(b.p); }

// ---------------------------------------------------------------- the extended value

// A heat value u = m * 2^e.  The heat solution falls by about e^-1 per edge
// length away from the sources; on large meshes it spans more binary
// exponents than any IEEE format holds, so the exponent travels separately.
// m == 0 encodes 0 and then e == kZeroExp.
constexpr int kZeroExp = -(1 << 28);

template <class T> struct alignas(sizeof(T) == 4 ? 8 : 16) XVal {
    T m;
    int e;
};

// One entry of a row of the level-ordered operator: neighbour position and
// weight t * theta.  8 bytes in FP32, 16 in FP64.
template <class T> struct alignas(sizeof(T) == 4 ? 8 : 16) Ent {
    int col;
    T w;
};

// Early termination of the ADMM (Sec. 3.2), on the device: once an
// iteration's residual norms meet the thresholds, `stop` is set and the
// remaining iteration kernels return at once; iters_done counts the
// iterations run.
struct AdmmCtl {
    int stop, iters_done, pad0, pad1;
    double th[2];   // |r_primal| and |r_dual| thresholds
};

// One Gauss-Seidel tile: up to TILE consecutive layout positions of one set.
struct alignas(16) TileDesc {
    int level, start, count, lo;      // set index, first position, positions, first position of the set
    int eb, ee, nt_prev, nt_self;     // first entry of its row block, width W; tiles in sets i-1 and i
    int nt_next, pad0, pad1, pad2;    // tiles in set i+1 (0 past the last set)
};

// ---------------------------------------------------------------- mesh

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
    int abort;
    int pad;
};

// Accounting shared by a context and its serving workers.
struct Shared {
    size_t budget = 0;                              // 0: unlimited
    std::atomic<size_t> in_use{0};                  // device bytes held
    std::atomic<unsigned long long> launches{0};    // kernels launched
};

struct LaunchCounter {
    std::atomic<unsigned long long> *p = nullptr;
    LaunchCounter &operator++() {
        p->fetch_add(1, std::memory_order_relaxed);
        return *this;
    }
};

// What a launcher needs: the device, a stream, a status word and abort flag
// of its own, and the shared accounting.  The context has one; every serving
// worker has another with its own stream.
struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    int gs_share = 1;                // a diffusion launch takes 1/gs_share of the resident CTAs
    unsigned long long wait_limit_ns = 2000000000ull;  // limit of any dependency wait inside a kernel
    int *status_dev = nullptr;       // device status word written by kernels
    GridBarrier *bar_dev = nullptr;  // abort flag of the persistent kernels
    Shared *shared = nullptr;
    LaunchCounter launches;
};

// Resident per-mesh operators (built once by gh_mesh_load).
struct DevMesh {
    int64_t nv = 0, nf = 0, ne = 0;
    double hbar = 0.0;
    DBuf P;          // double [nv*3]
    DBuf F;          // int32 [nf*3]
    DBuf rowptr;     // int32 [nv+1]
    DBuf col;        // int32 [2ne] neighbours ascending
    DBuf col_edge;   // int32 [2ne] edge id per entry
    DBuf edges;      // int32 [ne*2] (min, max)
    DBuf face_edge;  // int32 [nf*3] edge opposite corner k
    DBuf face_sign;  // int8 [nf*3]
    DBuf edge_face;  // int32 [ne*2] faces of the edge, ascending; -1 absent
    DBuf edge_slot;  // int32 [ne*2]
    DBuf twin;       // int32 [nf*3] (other face << 2 | its slot) or -1 on boundary
    DBuf Af;         // double [nf]
    DBuf Av;         // double [nv]
    DBuf theta;      // double [ne]
    DBuf ev;         // float [ne*3] edge vector max - min (orientation halfedge)
    DBuf gradop;     // float [nf*9] grad of corner k's hat function: (N x e_k)/(2A)
    DBuf Aff;        // float [nf] face area
    // face-form ADMM: per face, for slots k = 0..2 the unit edge vector and the
    // twin weight A'/(A + A'), then sqrt(A_f): 16 values (FP32 and FP64
    // copies), built on the first face-form solve
    DBuf face_rec32, face_rec64;
    DBuf elen;       // double [ne] edge lengths
    // an intrinsic triangulation (Sec. 5.3, gh_mesh_intrinsic_delaunay): the
    // triangulation is the face list plus the lengths; per face, in its own
    // frame, the hat-function gradients and the edge vectors of the three
    // slots (lower -> higher vertex), FP64 and FP32 (gradop holds the FP32
    // gradients); P keeps the input positions, which no longer define edges
    int intrinsic = 0;
    DBuf gradop64, evf64, evf32;
    // breadth-first cluster size per kind of solve ([0] one query, [1] a
    // batch): 0 until tuned on the first solve of that kind, or set by the user
    int bfs_cluster[2] = {0, 0};
    std::shared_ptr<std::mutex> rec_mu = std::make_shared<std::mutex>();   // guards the lazily built parts
    // cycle constraints of a connected closed surface (Sec. 5.1, cycles.cu),
    // per form ([0] face, [1] edge): -1 until built on the first solve that
    // asks for them; constraint j holds entries [cyc_off_h[j], cyc_off_h[j+1])
    int ncyc[2] = {-1, -1}, cyc_ent[2] = {0, 0};
    std::vector<int32_t> cyc_off_h[2];
    DBuf cyc_var[2], cyc_coef[2];
    std::shared_ptr<std::mutex> cyc_mu = std::make_shared<std::mutex>();
};

// Per-query workspace (BFS products, the level-ordered layout, solver state).
struct QueryWs {
    int64_t cap_nv = 0, cap_nf = 0, cap_ne = 0, cap_nnz = 0;
    int fp64 = 0;
    // breadth-first traversal
    DBuf level, parent, order, pos, key, lvl_off, meta;  // meta: [0] nlev [1] nreach [2] err
    DBuf pedge;     // int32 [nv] edge from each vertex to its pairing vertex
    DBuf lorder;    // int32 [nv] layout order: the queue with each set's short rows first; pos is its inverse
    // level-ordered Gauss-Seidel layout
    DBuf gent;      // Ent<T>: one column-major block per tile (see k_fill_ell)
    DBuf twid;      // int32 [2 tiles + 2]: block size and offset of each tile
    DBuf diag;      // T [nv] (+ padding): 1 / (A_v + t sum theta)
    DBuf tiles;     // TileDesc [nreach/TILE + nlev], sorted by (parity, level)
    DBuf ptile;     // int32 [nv + 8] per-parity tile prefix over levels
    DBuf U0, U1;    // XVal<T> [nv] ping-pong state
    // stages
    DBuf h;         // T [nf*3]
    DBuf g0, g1;    // T [nf*3] face form
    DBuf l0, l1;    // T [nf*9] face form: per slot q_k = g - lambda_k / (mu alpha)
    DBuf z, w, lam; // T [nf*3] edge form
    DBuf sz, x;     // T [ne] edge form
    DBuf inc;       // double [nv]
    DBuf d0, d1;    // double [nv]
    DBuf n0, n1;    // int32 [nv]
    DBuf resid;     // double [iters*2]
    DBuf actl;      // AdmmCtl: early termination of the ADMM
    DBuf e1;        // double [1]
    // multi-source path constraints (Sec. 5.2), built per solve when asked for
    // (see paths.cu): entries, distinct variables, Gram factor, per-iteration
    // values and corrections, and the block's variable -> distinct index map
    DBuf pc_src, pc_lv, pc_off, pc_var, pc_coef, pc_entu, pc_uvar, pc_ucoef, pc_dinv, pc_L, pc_drop, pc_meta;
    DBuf pc_val, pc_delta, pc_map;
    int pc_n = 0, pc_ent = 0, pc_dim = 1;   // constraints and entries of the last solve (0: none)
    // host-side facts of the last run
    int nlev = 0, nreach = 0, final_buf = 0, form = 1, admm_iters = 0, diagnostics = 0, sweeps = 0;
    int max_w = 8;         // widest row block of the layout (entries per row)
    int gs_continue = 0;   // 1: the next diffusion launch resumes from the state of the last one
    int gs_band = 0;       // sweeps per band of the next diffusion launch (0: from the layout)
    int sweeps_run = 0;    // sweeps of the last solve (all rounds)
    double t = 0.0;
};

struct MeshH {
    Ctx *ctx = nullptr;
    DevMesh m;
    std::vector<QueryWs *> ws;   // one per query slot of the last batch
    int last_k = 0;
    double stage_ms[5] = {0, 0, 0, 0, 0};
    double gs_kernel_ms = 0.0;   // the diffusion kernel alone, last solve
    std::atomic<int> inflight{0};  // serving requests not yet finished
};

// The whole path for a list of source sets on one mesh, with the launcher
// context `c` and the workspace pool `pool` (grown as needed).  d_out_dev:
// device, [K][nv] (may be null); d_out_host: host, [K][nv] (may be null),
// each query's distances copied there from its workspace, in stream order
// (the caller synchronises).  stage_ms6 (may be null) gets the stage times.
gh_status solve_core(Ctx *c, DevMesh &m, std::vector<QueryWs *> &pool, const std::vector<std::vector<int32_t>> &src,
                     const gh_params *p, double *d_out_dev, double *stage_ms6, int *last_k,
                     double *d_out_host = nullptr);

// One query of a heterogeneous batch.
struct Item {
    DevMesh *m;
    QueryWs *w;
    const std::vector<int32_t> *src;   // validated, sorted, de-duplicated
    const gh_params *p;
    double *d_out_dev;                 // device, [m->nv] (may be null)
};
gh_status solve_items(Ctx *c, std::vector<Item> &items, double *stage_ms6);
size_t ws_bytes(const DevMesh &m, int fp64, int form, int path_constraints);
void free_ws(Ctx *c, QueryWs *w);
gh_status validate_params(const gh_params *p);
gh_status prep_sources(const int32_t *src, int32_t nsrc, int64_t nv, std::vector<int32_t> &out);
constexpr int kMaxPc = 31;   // path constraints per query: sources - 1 (one warp per constraint)
gh_status check_pc_sources(const gh_params *p, const std::vector<int32_t> &set);
bool is_device_ptr(const void *p);

// ---------------------------------------------------------------- kernels (host launchers)

constexpr int TILE = 512;  // layout positions per Gauss-Seidel tile

// scan.cu
gh_status exclusive_scan_i32(Ctx *c, const int32_t *in, int32_t *out, int64_t n, int32_t *total_host);
gh_status exclusive_scan_u32_dev(Ctx *c, const int32_t *in, int32_t *out, int64_t n);

// setup.cu
gh_status build_mesh(Ctx *c, DevMesh &m, const double *V_dev, const int32_t *F_dev);
// the stages of build_mesh: connectivity of m.F; geometry from m.P; and the
// geometry of an intrinsic triangulation from the lengths L[3f+k] of the edge
// opposite corner k of every face (device, FP64)
gh_status build_connectivity(Ctx *c, DevMesh &m);
gh_status build_geometry_positions(Ctx *c, DevMesh &m);
gh_status build_geometry_lengths(Ctx *c, DevMesh &m, const double *L);

// idt.cu
// replaces m's triangulation by its intrinsic Delaunay triangulation
gh_status mesh_intrinsic_delaunay(Ctx *c, DevMesh &m, int64_t *flips);

// bfs.cu
// breadth-first sets of every query (each on its own mesh) in one launch
gh_status run_bfs(Ctx *c, std::vector<DevMesh *> &meshes, std::vector<QueryWs *> &ws,
                  const std::vector<std::vector<int32_t>> &src);
// the same with a given cluster size (8 is always supported), no tuning; any
// graph in CSR form works (rowptr, col ascending, col_edge, nv of `meshes`).
// targets (device, per query; may be null): the traversal may stop once all
// of them have a set, leaving the later sets undone
gh_status run_bfs_fixed(Ctx *c, std::vector<DevMesh *> &meshes, std::vector<QueryWs *> &ws,
                        const std::vector<std::vector<int32_t>> &src, int cl,
                        const std::vector<const int32_t *> *targets = nullptr,
                        const std::vector<int32_t> *ntargets = nullptr);
bool bfs_cluster_supported(int cl);
gh_status build_layout(Ctx *c, const DevMesh &m, QueryWs &q, double t);

// gs.cu
// ev0/ev1 (may be null) are recorded on the stream right around the kernel launch
// one persistent diffusion launch for all queries (each with its own sweeps,
// in QueryWs::sweeps; all of one precision)
gh_status run_gs(Ctx *c, std::vector<QueryWs *> &ws, cudaEvent_t ev0, cudaEvent_t ev1);

// paths.cu
// the multi-source path and cycle constraints of every item that asks for
// them; runs before the items' own traversal (it uses their traversal buffers)
gh_status build_path_constraints(Ctx *c, std::vector<Item> &items);

// cycles.cu
// the cycle constraints of mesh m for one form, built once (DevMesh::ncyc)
gh_status mesh_cycles(Ctx *c, DevMesh &m, int form);

// stages.cu
gh_status run_normalize(Ctx *c, const DevMesh &m, QueryWs &q);
gh_status run_face_admm(Ctx *c, DevMesh &m, QueryWs &q, const gh_params *p);
gh_status run_edge_admm(Ctx *c, const DevMesh &m, QueryWs &q, const gh_params *p);
gh_status run_integrate(Ctx *c, const DevMesh &m, QueryWs &q, double *d_out_dev);
gh_status run_heat_residual(Ctx *c, const DevMesh &m, QueryWs &q);

// device status word shared by launchers (one int in device memory per context)
int *dev_status(Ctx *c);
gh_status check_status(Ctx *c, const char *stage);

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// triangle area from its side lengths in Kahan's arrangement of Heron's
// formula (sides sorted a >= b >= c)
__device__ inline double heron_d(double a, double b, double c) {
    double t;
    if (a < b) { t = a; a = b; b = t; }
    if (b < c) { t = b; b = c; c = t; }
    if (a < b) { t = a; a = b; b = t; }
    const double q = (a + (b + c)) * (c - (a - b)) * (c + (a - b)) * (a + (b - c));
    return 0.25 * sqrt(q > 0.0 ? q : 0.0);
}

}  // namespace gh
