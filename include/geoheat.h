/*
 * geoheat: geodesic distance on triangle meshes by the parallel heat method
 * of Tao, Zhang, Deng, Fang, Peng and He, "Parallel and Scalable Heat
 * Methods for Geodesic Distance Computation" (arXiv 1812.06060), on one
 * NVIDIA GB300 (sm_103a).
 *
 * The problem (Sec. 3): given a manifold triangle mesh M = (V, E, F), a set
 * of source vertices and a diffusion time t, return the geodesic distance d
 * from the source set at every vertex.  Algorithm 1: heat diffusion by
 * breadth-first Gauss-Seidel (Sec. 3.1) -> face-wise normalised gradients
 * h = -grad u / |grad u| -> an integrable gradient field by ADMM, face form
 * (Sec. 3.2) or edge form (Sec. 4) -> breadth-first integration (Sec. 3.3).
 *
 * Conventions for every call:
 *  - Every call returns a gh_status; outputs are written only on GH_OK.
 *  - Inputs are copied; the caller keeps ownership of every buffer it
 *    passes.  Handles belong to the library until gh_mesh_free /
 *    gh_ctx_destroy.
 *  - Pointer arguments marked "host or device" may point to host memory or
 *    to device memory of the context's GPU; the library tells them apart
 *    with cudaPointerGetAttributes.  Other pointers are host pointers.
 *  - All device work of a context runs on the context's stream (the legacy
 *    default stream unless gh_ctx_set_stream set another one); blocking calls
 *    synchronise that stream before they return.
 *  - gh_last_error() returns a thread-local message for the last failing
 *    call of the calling thread.
 *  - Calls on one context must not run concurrently from several threads,
 *    except gh_submit / gh_poll / gh_wait, which are thread-safe.
 */
#ifndef GEOHEAT_H
#define GEOHEAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gh_ctx_s *gh_ctx;
typedef struct gh_mesh_s *gh_mesh;
typedef uint64_t gh_req;

typedef enum {
    GH_OK = 0,
    GH_EINVAL = 1,        /* bad argument: null pointer, index out of range, empty source set, bad params */
    GH_ENOMEM = 2,        /* device memory or the context's HBM budget is exhausted */
    GH_EDEVICE = 3,       /* a CUDA call failed; see gh_last_error() */
    GH_ETIMEOUT = 4,      /* a bounded wait ran out (a grid barrier inside a kernel, or gh_wait) */
    GH_EBUSY = 5,         /* the request is not finished yet */
    GH_ENOTFOUND = 6,     /* unknown request id */
    GH_ENONMANIFOLD = 7   /* an edge in more than two faces, or two faces that cross an edge in the same direction */
} gh_status;

typedef enum { GH_FORM_FACE = 0, GH_FORM_EDGE = 1 } gh_form;

/*
 * Solver parameters (Sec. 3.1, Sec. 3.2, Sec. 4.1, Sec. 6).
 *  m           diffusion-time factor: t = m * hbar^2, hbar = mean edge length
 *              (eq. DiffusionTime); used when t <= 0.  Default 1.
 *  t           explicit diffusion time when > 0.  Default 0.
 *  gs_sweeps   outer Gauss-Seidel iterations of the diffusion step (Sec. 3.1).
 *              Default 200.
 *  admm_iters  ADMM iterations, I_max (Sec. 6).  Default 10.
 *  mu          ADMM penalty parameter (Sec. 3.2, Sec. 4.1).  Default 100.
 *  form        GH_FORM_FACE (Sec. 3.2 + eq. IntegrationStep) or GH_FORM_EDGE
 *              (Sec. 4).  Default GH_FORM_EDGE.
 *  fp64        0: sweeps and ADMM in FP32 (the default); 1: in FP64.
 *              Geometry is always computed in FP64 and distances are always
 *              accumulated in FP64.
 *  diagnostics 1: also compute the heat residual E1 (eq. HeatSolutionError)
 *              and the ADMM primal / dual residual norms of every iteration,
 *              readable with gh_debug_dump.  Default 0.
 *  early_stop  1: end the ADMM once |r_primal| <= s * eps1 and
 *              |r_dual| <= s * eps2 (Sec. 3.2), s = |M|_F (the square root of
 *              the face area summed over interior-edge slots) in the face
 *              form and |Z|_F (the norm of the target edge differences) in
 *              the edge form, whose thresholds the paper does not print; at
 *              most admm_iters iterations either way.  The iterations run are
 *              readable with gh_debug_dump (GH_DUMP_ITERS).  Default 0.
 *  eps1, eps2  the thresholds of early_stop; >= 0.  Default 1e-5 (Sec. 3.2).
 *  path_constraints  1: with two or more sources, also make the line
 *              integral of the optimised field vanish along a path from the
 *              first (lowest-index) source to each other source (Sec. 5.2,
 *              eq. MultiSourceConstraint, eq. MultiSourceConstraintEdgeBased).
 *              The paths are the fewest-edge ones of a breadth-first
 *              traversal from the first source alone (its FIFO pairing);
 *              the constraints act inside the G (face form) or X (edge form)
 *              update, whose minimiser under them is a projection through a
 *              small Gram system.  At most 32 sources (GH_EINVAL otherwise).
 *              No effect with one source.  Default 0.
 *  cycle_constraints  1: on a connected closed mesh of genus g >= 1, also
 *              make the line integral vanish around each of the 2g cycles of
 *              a tree-cotree basis (Sec. 5.1, eq. TopologyConstraint,
 *              eq. EdgeTopologyConstraint): cycles of edges in the edge form,
 *              loops of faces through edge midpoints in the face form, built
 *              once per mesh and form from breadth-first trees rooted at
 *              vertex 0 and face 0.  A mesh with boundary edges or in several
 *              pieces gets none.  Path and cycle constraints together: at
 *              most 31 (GH_EINVAL otherwise).  Default 0.
 *  gs_tol      > 0: stop the diffusion on the heat residual E1 (eq.
 *              HeatSolutionError, the l2 norm of (A - t L_c) u - u_0 over
 *              the reached vertices, in FP64 from the state and the
 *              weights the sweeps use): E1 is evaluated after every
 *              gs_check sweeps and after the last, and the sweeps end at
 *              the first evaluation with E1 <= gs_tol, at most gs_sweeps in
 *              all.  The rounds continue one iteration: the state after n
 *              sweeps is the same, bit for bit, as that of an uninterrupted
 *              run of n sweeps.  Each round refills the pipelined sweeps
 *              (a round of c sweeps costs about L + 2c set steps instead of
 *              2c), so gs_check well above the number of breadth-first sets
 *              keeps the overhead small.  The sweeps run are readable with
 *              gh_debug_dump (GH_DUMP_GS_SWEEPS).  0 (the default): exactly
 *              gs_sweeps sweeps.  Must be finite and >= 0.
 *  gs_check    sweeps per E1 evaluation when gs_tol > 0; >= 1.  Default 100.
 *  gs_band     the order in which the pipelined sweeps run; the result is the
 *              same, bit for bit, for every value.  The sweeps run in bands
 *              of gs_band sweeps, one after the other, each band a wavefront
 *              over the breadth-first sets, so fewer sets are in flight at a
 *              time and more of a step's reads are found in L2.  0 (the
 *              default): chosen from the layout, one band (the plain
 *              wavefront) unless the sets hold many tiles (on a 168M-vertex
 *              mesh, about 200 sweeps).  Must be >= 0.
 */
typedef struct {
    double m;
    double t;
    int32_t gs_sweeps;
    int32_t admm_iters;
    double mu;
    int32_t form;
    int32_t fp64;
    int32_t diagnostics;
    int32_t early_stop;
    double eps1;
    double eps2;
    int32_t path_constraints;
    int32_t cycle_constraints;
    double gs_tol;
    int32_t gs_check;
    int32_t gs_band;
} gh_params;

/* Fills *p with the defaults listed above. */
void gh_params_default(gh_params *p);

/* Library version string. */
const char *gh_version(void);

/*
 * Context on CUDA device `device`.  hbm_budget_bytes caps the device memory
 * the context allocates (0: no cap beyond the device's).  The context owns
 * its meshes.  Errors: GH_EINVAL (bad device), GH_EDEVICE.
 */
gh_status gh_ctx_create(int device, size_t hbm_budget_bytes, gh_ctx *out);
gh_status gh_ctx_destroy(gh_ctx ctx);

/* Stream for all device work of the context (a cudaStream_t, passed as a
 * pointer; NULL = the legacy default stream).  The caller keeps the stream
 * alive while the context uses it. */
gh_status gh_ctx_set_stream(gh_ctx ctx, void *stream);

/* Limit of every dependency wait inside the persistent diffusion kernel
 * (microseconds; <= 0 restores the default of 2 s).  When a wait runs out,
 * the kernel raises its abort flag, every CTA leaves after its staged copies
 * have landed, and the solve returns GH_ETIMEOUT; the context stays usable.
 * Applies to the context's blocking solves. */
gh_status gh_ctx_set_wait_limit(gh_ctx ctx, int64_t microseconds);

/* Device bytes the context holds now. */
gh_status gh_ctx_memory(gh_ctx ctx, size_t *bytes_in_use);

/* Number of CUDA kernels the context has launched since it was created
 * (every launch of every geoheat kernel, setup included). */
gh_status gh_ctx_stats(gh_ctx ctx, uint64_t *kernel_launches);

/*
 * Mesh setup (the "initialization of data structures" of Sec. 6.4), done
 * once per mesh on the device and kept resident for every later solve.
 *  V  host or device, float64 [nv][3] vertex positions.
 *  F  host or device, int32 [nf][3] faces, vertex indices, each face's loop
 *     a->b->c->a consistently oriented over the mesh (an oriented 2-manifold,
 *     Sec. 4.1), boundaries allowed.
 * Builds the sorted one-ring of each vertex, edge ids (edges sorted by
 * (min, max) vertex index), per-face edge ids and integrability signs
 * s_k^f with orientation halfedges running from the smaller to the larger
 * vertex index (eq. Integrability), vertex areas A_v (one third of the
 * incident face area), cotangent weights theta_e = 1/2 sum cot(opposite
 * angle) (Sec. 3.1), face gradient operators and the mean edge length.
 * Errors: GH_EINVAL (nv < 3, nf < 1, an index outside [0, nv), a face with
 * a repeated vertex), GH_ENONMANIFOLD, GH_ENOMEM, GH_EDEVICE.
 */
gh_status gh_mesh_load(gh_ctx ctx, const double *V, int64_t nv, const int32_t *F, int64_t nf, gh_mesh *out);

/* Counts and mean edge length (hbar of eq. DiffusionTime).  Any output
 * pointer may be NULL. */
gh_status gh_mesh_info(gh_mesh mesh, int64_t *nv, int64_t *ne, int64_t *nf, double *mean_edge_len);

/* Launch shape of the breadth-first traversal (Sec. 3.3): one thread-block
 * cluster of `bfs_cluster` CTAs (8, or 16 where the device allows clusters
 * that large) walks the sets of each query.  By default the size is tuned
 * per mesh on the first solve of each kind ([0] a single query, [1] a
 * batch): every supported size runs once, timed, and the fastest is kept.
 * All sizes give the same sets, pairing and order.  The paper's traversal
 * is sequential and has no counterpart.
 * gh_mesh_tuning: writes the sizes in use (0: not tuned yet) to
 *   bfs_cluster[2].
 * gh_mesh_set_tuning: kind 0 or 1; size 0 (tune again), 8 or 16.
 *   GH_EINVAL for another kind or size, or a size the device cannot place. */
gh_status gh_mesh_tuning(gh_mesh mesh, int32_t *bfs_cluster);
gh_status gh_mesh_set_tuning(gh_mesh mesh, int32_t kind, int32_t bfs_cluster);

/*
 * Replaces the mesh's triangulation by its intrinsic Delaunay triangulation
 * (Sec. 5.3): edge flips by the opposite-angle criterion (an interior edge
 * whose opposite angles sum to more than pi, beyond a 1e-12 tolerance on
 * their cotangents, is flipped; the new edge's length comes from the two
 * triangles unfolded into the plane) until none is left.  A flip that would
 * join two vertices already joined is left out.  Afterwards the mesh is the
 * face list plus edge lengths: the diffusion uses cotangents and vertex areas
 * from the lengths, normalisation, the edge form's target differences and
 * the face form's gradients use each face's own frame (in the face form an
 * edge's compatibility compares each face's projection on its own unit
 * vector of the edge), and the constraints of Sec. 5 run in the edge form
 * only (GH_EINVAL otherwise).  The vertices and their indices are unchanged; faces and
 * edges are those of the new triangulation (GH_DUMP_FACES, GH_DUMP_EDGES,
 * GH_DUMP_ELEN).  flips (nullable) receives the number of flips.
 * GH_EINVAL if the mesh is already intrinsic, GH_EBUSY while serving
 * requests on it are in flight.
 */
gh_status gh_mesh_intrinsic_delaunay(gh_mesh mesh, int64_t *flips);

/* Frees the mesh; GH_EBUSY while serving requests on it are in flight. */
gh_status gh_mesh_free(gh_mesh mesh);

/*
 * One geodesic distance field from one source set (Algorithm 1; Sec. 5.2 for
 * several sources: all of them form D_0, u_0 = 1 on each, d = 0 on each).
 *  src    host or device, int32 [nsrc] vertex indices; duplicates allowed.
 *  d_out  host or device, float64 [nv]: distances; +infinity at vertices not
 *         connected to any source.
 * Errors: GH_EINVAL (nsrc < 1, a source outside [0, nv), bad params),
 * GH_ENOMEM, GH_ETIMEOUT, GH_EDEVICE.
 */
gh_status gh_solve(gh_mesh mesh, const int32_t *src, int32_t nsrc, const gh_params *params, double *d_out);

/*
 * K independent source sets solved together as K right-hand sides of the
 * same mesh, one persistent kernel per stage for all of them.
 *  src_off  host, int32 [K+1]: set q is src[src_off[q] .. src_off[q+1]).
 *  src      host, int32 [src_off[K]].
 *  d_out    host or device, float64 [K][nv].
 * Results are the same as K separate gh_solve calls.  Errors as gh_solve.
 */
gh_status gh_solve_batch(gh_mesh mesh, const int32_t *src_off, const int32_t *src, int32_t K,
                         const gh_params *params, double *d_out);

/*
 * Serving with continuous batching.  gh_submit queues one source set on a
 * loaded mesh and returns at once with a request id.  Worker threads of the
 * context (each with its own CUDA stream and workspaces) admit pending
 * requests as memory and batch slots free up, in arrival order: the oldest
 * pending request's precision and requests of similar work (vertices x
 * sweeps within 4x of it), on any mesh and with any other parameters, run
 * as one batch (one breadth-first launch and one diffusion launch for all of
 * it; with gs_tol, one launch per round for the requests still running);
 * requests that arrive while others run join the next batch, and the
 * workers' batches overlap on the device.  A request's distances equal those of gh_solve with
 * the same arguments.  gh_submit, gh_poll and gh_wait are thread-safe.
 *
 * gh_serve_config: number of workers (1..8, default 2) and the batch limit
 * (1..256, default 32); only before the first gh_submit on the context.
 * gh_submit: src is host or device int32 [nsrc] (copied); errors as gh_solve.
 * gh_poll: *done = 1 once the request has finished (successfully or not).
 * gh_wait: waits up to timeout_us microseconds (< 0: no limit), then copies
 *   the distances (float64 [nv], host or device) to d_out and forgets the
 *   request; GH_ETIMEOUT leaves it pending, GH_ENOTFOUND for unknown ids, and
 *   a failed request returns its error here.
 * A mesh cannot be freed while it has requests in flight (GH_EBUSY).
 */
gh_status gh_serve_config(gh_ctx ctx, int32_t workers, int32_t max_batch);
gh_status gh_submit(gh_ctx ctx, gh_mesh mesh, const int32_t *src, int32_t nsrc, const gh_params *params, gh_req *out);
gh_status gh_poll(gh_ctx ctx, gh_req req, int *done);
gh_status gh_wait(gh_ctx ctx, gh_req req, double *d_out, int64_t timeout_us);

/*
 * Intermediates of query `query` of the last gh_solve / gh_solve_batch on
 * this mesh, copied to the host buffer `out`, for parity tests and
 * diagnostics.  gh_debug_size gives the element count and element size in
 * bytes of each item.
 */
typedef enum {
    GH_DUMP_LEVEL = 0,      /* int32 [nv]  breadth-first set index i of each vertex (v in D_i), -1 unreachable */
    GH_DUMP_PARENT = 1,     /* int32 [nv]  pairing vertex in D_{i-1} (first discoverer), -1 for sources/unreachable */
    GH_DUMP_ORDER = 2,      /* int32 [nreach]  vertices in breadth-first (FIFO) order */
    GH_DUMP_LEVEL_OFF = 3,  /* int32 [L+1] D_i = order[off[i] .. off[i+1]) */
    GH_DUMP_U_MANT = 4,     /* float64 [nv] mantissa of u: u = mant * 2^exp */
    GH_DUMP_U_EXP = 5,      /* int32 [nv]  binary exponent of u */
    GH_DUMP_H = 6,          /* float64 [nf][3] normalised gradients h */
    GH_DUMP_G = 7,          /* float64 [nf][3] face form: optimised gradients g */
    GH_DUMP_X = 8,          /* float64 [ne]  edge form: optimised edge differences x */
    GH_DUMP_D = 9,          /* float64 [nv]  distances */
    GH_DUMP_EDGES = 10,     /* int32 [ne][2] (min, max) vertex pair of each edge */
    GH_DUMP_FACE_EDGE = 11, /* int32 [nf][3] edge id of the edge opposite corner k */
    GH_DUMP_FACE_SIGN = 12, /* int32 [nf][3] s_k^f in {-1, +1} */
    GH_DUMP_THETA = 13,     /* float64 [ne]  cotangent weight per edge */
    GH_DUMP_AV = 14,        /* float64 [nv]  vertex areas */
    GH_DUMP_AF = 15,        /* float64 [nf]  face areas */
    GH_DUMP_ROWPTR = 16,    /* int32 [nv+1]  one-ring CSR row pointers */
    GH_DUMP_COL = 17,       /* int32 [2ne]   one-ring neighbours, ascending per row */
    GH_DUMP_RESID = 18,     /* float64 [admm_iters][2] primal, dual residual norms (diagnostics = 1) */
    GH_DUMP_E1 = 19,        /* float64 [1]   heat residual E1 (diagnostics = 1) */
    GH_DUMP_T = 20,         /* float64 [1]   diffusion time used */
    GH_DUMP_ITERS = 21,     /* int32 [1]     ADMM iterations run (early_stop can end them before admm_iters) */
    GH_DUMP_PC_OFF = 22,    /* int32 [npc+1] path constraints: entries of constraint j are [off[j], off[j+1]) */
    GH_DUMP_PC_VAR = 23,    /* int32 [n]     constrained variable of each entry: edge id (edge form), face id (face form) */
    GH_DUMP_PC_COEF = 24,   /* float64 [n][dim] coefficient of each entry: sign (edge form), path edge vector (face form) */
    GH_DUMP_FACES = 25,     /* int32 [nf][3] the faces of the mesh's triangulation */
    GH_DUMP_ELEN = 26,      /* float64 [ne]  edge lengths */
    GH_DUMP_GS_SWEEPS = 27  /* int32 [1]     Gauss-Seidel sweeps run (gs_tol can end them before gs_sweeps) */
} gh_dump_item;

gh_status gh_debug_size(gh_mesh mesh, int32_t query, int32_t what, int64_t *count, int32_t *elem_bytes);
gh_status gh_debug_dump(gh_mesh mesh, int32_t query, int32_t what, void *out);

/* Per-stage device times of the last solve on this mesh, in milliseconds,
 * measured with CUDA events on the context's stream, summed over the passes
 * of a batch: ms6[0] breadth-first sets and layout, [1] Gauss-Seidel
 * diffusion stage, [2] normalisation (and E1 with diagnostics), [3] ADMM,
 * [4] integration, [5] the diffusion kernel launch alone. */
gh_status gh_stage_times(gh_mesh mesh, double *ms6);

/*
 * Mean edge length of a mesh whose data the caller already holds on the
 * device, with no device allocation at all.  The paper has no counterpart.
 * It serves callers that cannot have a library allocate device memory:
 * applications whose own allocator or memory pool owns the device memory
 * and forbids other code from calling cudaMalloc, and latency-critical loops
 * where a cudaMalloc or cudaFree may wait for the whole device to go idle.
 *  V       device memory of the current device (or managed memory), float64
 *          [nv][3] vertex positions.
 *  edges   the same, int32 [ne][2] vertex pairs, e.g. GH_DUMP_EDGES of a
 *          loaded mesh; every index must be inside V.
 *  ne      1 .. 536,870,912 edges (a fixed scratch of 8192 partial sums of
 *          65,536 edges each); larger counts return GH_EINVAL.
 *  out     the same, float64 [1]: the mean edge length, the same two-level
 *          fixed-order sum as gh_mesh_load uses (bit for bit).
 *  stream  cudaStream_t (NULL = legacy default stream); the call only
 *          enqueues two kernels and returns, out is ready when the stream
 *          reaches that point.
 * The partial sums live in one 64 KiB array in device memory that every GPU
 * loading the library holds until the process exits.  All calls on a device
 * share it, so calls whose kernels overlap on the GPU (different streams)
 * race; each call overwrites every partial it reads, so nothing needs
 * clearing.  The first call on a device (and the first after a device reset
 * made a new context) looks the array's address up with cudaGetSymbolAddress
 * while that device is current; make that first call before any stream
 * capture.  Errors: GH_EINVAL (NULL pointer, host memory or memory of
 * another device, ne out of range), GH_EDEVICE.
 */
gh_status gh_mean_edge_length_noalloc(const double *V, const int32_t *edges, int64_t ne, double *out, void *stream);

/* Message of the last failing call on this thread ("" if none). */
const char *gh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GEOHEAT_H */
