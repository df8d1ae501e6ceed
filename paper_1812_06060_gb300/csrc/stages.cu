// Stages after the diffusion: face-wise gradient normalisation (Algorithm 1,
// eq. HeatDiffusionNormalization), the face-based ADMM (Sec. 3.2), the
// edge-based ADMM (Sec. 4.1), breadth-first integration (eq. IntegrationStep,
// Sec. 4) and the heat residual E1 (eq. HeatSolutionError).
#include "admm.cuh"
#include "internal.cuh"

namespace gh {

namespace {

constexpr int NT = 256;

// The ADMM iterations and the integration are chains of short kernels on one
// stream (a few microseconds each on the smaller meshes).  They are launched
// as programmatic dependents: a block signals, once its writes are issued,
// that the next kernel may be scheduled, and the next kernel waits
// (griddepcontrol.wait: until the previous grid has completed and its writes
// are visible) before its first read, so its launch overlaps the previous
// kernel's tail instead of following it.  A kernel launched this way calls
// griddep_wait before it touches memory that earlier kernels wrote.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t st,
                             Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class T> __device__ __forceinline__ T ldexp_t(T x, int n);
template <> __device__ __forceinline__ float ldexp_t<float>(float x, int n) { return ldexpf(x, n); }
template <> __device__ __forceinline__ double ldexp_t<double>(double x, int n) { return ldexp(x, n); }
template <class T> __device__ __forceinline__ T sqrt_t(T x);
template <> __device__ __forceinline__ float sqrt_t<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sqrt_t<double>(double x) { return sqrt(x); }

// Geometry accessors: FP32 stages read the rounded per-face / per-edge
// operators; FP64 stages recompute them from the FP64 positions.  On an
// intrinsic triangulation (evf set) the gradients and the slot edge vectors
// are each face's own-frame ones, stored per face.
template <class T> struct Geo;
template <> struct Geo<float> {
    const float *gradop, *ev, *Af, *evf;
    __device__ void grad(int64_t f, int k, float *g) const {
        g[0] = gradop[9 * f + 3 * k]; g[1] = gradop[9 * f + 3 * k + 1]; g[2] = gradop[9 * f + 3 * k + 2];
    }
    __device__ void edge(int64_t e, float *v) const { v[0] = ev[3 * e]; v[1] = ev[3 * e + 1]; v[2] = ev[3 * e + 2]; }
    // the vector of face f's slot k (edge e), lower -> higher vertex
    __device__ void slot_edge(int64_t f, int k, int64_t e, float *v) const {
        if (evf) { v[0] = evf[9 * f + 3 * k]; v[1] = evf[9 * f + 3 * k + 1]; v[2] = evf[9 * f + 3 * k + 2]; }
        else edge(e, v);
    }
    __device__ float area(int64_t f) const { return Af[f]; }
};
template <> struct Geo<double> {
    const double *P, *Af;
    const int32_t *F, *edges;
    const double *gradop64, *evf;
    __device__ void grad(int64_t f, int k, double *g) const {
        if (gradop64) {
            g[0] = gradop64[9 * f + 3 * k]; g[1] = gradop64[9 * f + 3 * k + 1]; g[2] = gradop64[9 * f + 3 * k + 2];
            return;
        }
        const double *a = P + 3 * F[3 * f], *b = P + 3 * F[3 * f + 1], *c = P + 3 * F[3 * f + 2];
        double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        double twoA = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        double N[3] = {n[0] / twoA, n[1] / twoA, n[2] / twoA};
        const double *p1 = P + 3 * F[3 * f + (k + 1) % 3], *p2 = P + 3 * F[3 * f + (k + 2) % 3];
        double e[3] = {p2[0] - p1[0], p2[1] - p1[1], p2[2] - p1[2]};
        g[0] = (N[1] * e[2] - N[2] * e[1]) / twoA;
        g[1] = (N[2] * e[0] - N[0] * e[2]) / twoA;
        g[2] = (N[0] * e[1] - N[1] * e[0]) / twoA;
    }
    __device__ void edge(int64_t e, double *v) const {
        const double *a = P + 3 * edges[2 * e], *b = P + 3 * edges[2 * e + 1];
        v[0] = b[0] - a[0]; v[1] = b[1] - a[1]; v[2] = b[2] - a[2];
    }
    __device__ void slot_edge(int64_t f, int k, int64_t e, double *v) const {
        if (evf) { v[0] = evf[9 * f + 3 * k]; v[1] = evf[9 * f + 3 * k + 1]; v[2] = evf[9 * f + 3 * k + 2]; }
        else edge(e, v);
    }
    __device__ double area(int64_t f) const { return Af[f]; }
};

template <class T> Geo<T> make_geo(const DevMesh &m);
template <> Geo<float> make_geo<float>(const DevMesh &m) {
    return Geo<float>{ptr<float>(m.gradop), ptr<float>(m.ev), ptr<float>(m.Aff),
                      m.intrinsic ? ptr<float>(m.evf32) : nullptr};
}
template <> Geo<double> make_geo<double>(const DevMesh &m) {
    return Geo<double>{ptr<double>(m.P), ptr<double>(m.Af), ptr<int32_t>(m.F), ptr<int32_t>(m.edges),
                       m.intrinsic ? ptr<double>(m.gradop64) : nullptr, m.intrinsic ? ptr<double>(m.evf64) : nullptr};
}

// ------------------------------------------------------------------ normalise

// h = -grad u / |grad u|, grad u = sum_k u_k grad B_k; the three values are
// first brought to their largest exponent (exact); unreached faces get h = 0
template <class T>
__global__ void k_normalize(int64_t nf, const int32_t *__restrict__ F, const int32_t *__restrict__ pos,
                            const XVal<T> *__restrict__ U, Geo<T> geo, T *h) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    XVal<T> u[3];
    bool ok = true;
    for (int k = 0; k < 3; ++k) {
        int q = pos[F[3 * f + k]];
        if (q < 0) { ok = false; break; }
        u[k] = U[q];
    }
    T g[3] = {0, 0, 0};
    if (ok) {
        int eref = kZeroExp;
        for (int k = 0; k < 3; ++k)
            if (u[k].m != T(0) && u[k].e > eref) eref = u[k].e;
        for (int k = 0; k < 3; ++k) {
            T b[3];
            geo.grad(f, k, b);
            T uk = ldexp_t<T>(u[k].m, u[k].e - eref);
            g[0] += uk * b[0]; g[1] += uk * b[1]; g[2] += uk * b[2];
        }
    }
    T len = sqrt_t<T>(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int c = 0; c < 3; ++c) h[3 * f + c] = (len > T(0)) ? -g[c] / len : T(0);
}

// ------------------------------------------------------------------ early termination

__global__ void k_ctl_init(AdmmCtl *ctl, int iters) {
    ctl->stop = 0;
    ctl->iters_done = iters;
    ctl->th[0] = ctl->th[1] = 0.0;
}

// per-block partial sums of the squared scale: the face area over every
// interior-edge slot (|M|_F^2, Sec. 3.2) or the squared targets (|Z|_F^2)
__global__ void __launch_bounds__(NT) k_face_mnorm2(int64_t nf, const int32_t *__restrict__ twin,
                                                    const double *__restrict__ Af, double *part) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double a = 0.0;
    if (f < nf)
        for (int k = 0; k < 3; ++k) a += (twin[3 * f + k] >= 0) ? Af[f] : 0.0;
    __shared__ double sh[NT];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
template <class T>
__global__ void __launch_bounds__(NT) k_znorm2(int64_t n, const T *__restrict__ z, double *part) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double a = (i < n) ? (double)z[i] * (double)z[i] : 0.0;
    __shared__ double sh[NT];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
// thresholds = sqrt(sum of the partials) * (eps1, eps2), summed in a fixed order
__global__ void k_ctl_thresholds(const double *__restrict__ part, int nblocks, double eps1, double eps2,
                                 AdmmCtl *ctl) {
    __shared__ double sh[NT];
    double a = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += NT) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double s = sqrt(sh[0]);
        ctl->th[0] = s * eps1;
        ctl->th[1] = s * eps2;
    }
}
// after iteration it: stop once both residual norms are within the thresholds
__global__ void k_admm_check(const double *__restrict__ res2, AdmmCtl *ctl, int it) {
    if (!ctl->stop && res2[0] <= ctl->th[0] && res2[1] <= ctl->th[1]) {
        ctl->stop = 1;
        ctl->iters_done = it + 1;
    }
}
// the face form's result is in buffer (iterations run) & 1: keep it in g0
template <class T> __global__ void k_face_final(int64_t n, T *g0, const T *__restrict__ g1, const AdmmCtl *ctl) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (ctl->iters_done & 1)) g0[i] = g1[i];
}

// ------------------------------------------------------------------ face ADMM

// Static per-face data of the face form (FP64 arithmetic, stored as T):
// rec[12 f + 4 k + c] the unit vector of the edge opposite corner k (c < 3)
// and rec[12 f + 4 k + 3] the twin weight A'/(A + A') (0 on a boundary
// slot), 48 bytes per face in FP32; after all faces, rec[12 nf + f] =
// alpha = sqrt(A_f), read only for the residuals.
template <class T>
__global__ void k_face_rec(int64_t nf, const double *__restrict__ P, const int32_t *__restrict__ edges,
                           const int32_t *__restrict__ face_edge, const int32_t *__restrict__ twin,
                           const double *__restrict__ Af, const double *__restrict__ evf, T *rec) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const double A = Af[f];
    T *o = rec + 12 * f;
    for (int k = 0; k < 3; ++k) {
        double v[3];
        if (evf) {   // an intrinsic triangulation: the slot's vector in the face's own frame
            for (int c = 0; c < 3; ++c) v[c] = evf[9 * f + 3 * k + c];
        } else {
            const int e = face_edge[3 * f + k];
            const double *a = P + 3 * edges[2 * e], *b = P + 3 * edges[2 * e + 1];
            for (int c = 0; c < 3; ++c) v[c] = b[c] - a[c];
        }
        const double il = 1.0 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const int tw = twin[3 * f + k];
        const double A2 = (tw >= 0) ? Af[tw >> 2] : 0.0;
        o[4 * k] = (T)(v[0] * il);
        o[4 * k + 1] = (T)(v[1] * il);
        o[4 * k + 2] = (T)(v[2] * il);
        o[4 * k + 3] = (T)((tw >= 0) ? A2 / (A + A2) : 0.0);
    }
    rec[12 * nf + f] = (T)sqrt(A);
}

// One ADMM iteration per face, Y then G then lambda (Sec. 3.2), with the
// multiplier of slot k carried as q_k = g - lambda_k/(mu alpha) (the Y
// subproblem's input; lambda_k/(mu alpha) = g - q_k): face_update gives the
// Y- and G-updates, then
//   lambda_k += mu alpha (y_k - g')  <=>  q_k' = 2g' - g + q_k - y_k
// over the interior slots; the twins' q are the previous iteration's
// (buffers *_in), the new g and q go to *_out.  With multi-source path
// constraints, g' = gn - delta on the constrained faces (pcm[f] = the face's
// index in delta, else -1), the correction of the KKT projection.
// Optional residual partials per block: [0] |alpha (y - g')|^2,
// [1] |mu alpha (g' - g)|^2 summed over interior slots.  INTR: an intrinsic
// triangulation (face_update).
template <class T, bool INTR>
__global__ void __launch_bounds__(NT) k_face_admm(int64_t nf, const int32_t *__restrict__ twin,
                                                  const T *__restrict__ rec, const T *__restrict__ h,
                                                  const T *__restrict__ g_in, const T *__restrict__ q_in, T *g_out,
                                                  T *q_out, T mu, double *part, const AdmmCtl *ctl, int first,
                                                  const int32_t *__restrict__ pcm, const T *__restrict__ pcd) {
    griddep_wait();
    if (ctl && ctl->stop) return;   // the residuals met the thresholds (the same for every thread)
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rp = 0.0, rd = 0.0;
    if (f < nf) {
        FaceIter<T> s;
        face_update<T, INTR>(f, twin, rec, h, g_in, q_in, mu, first, s);
        if (pcm) {
            const int u = pcm[f];
            if (u >= 0)
                for (int c = 0; c < 3; ++c) s.gn[c] -= pcd[3 * u + c];
        }
        for (int c = 0; c < 3; ++c) g_out[3 * f + c] = s.gn[c];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) {
                T qn = s.gn[c];
                if (s.in[k]) {
                    qn = T(2) * s.gn[c] - s.g[c] + s.q[k][c] - s.y[k][c];
                    if (part) {   // residual norms only when asked for (FP64 arithmetic is slow here)
                        const T alpha = rec[12 * nf + f];
                        const T r = alpha * (s.y[k][c] - s.gn[c]);
                        rp += (double)r * (double)r;
                        const double dgv = (double)mu * (double)alpha * ((double)s.gn[c] - (double)s.g[c]);
                        rd += dgv * dgv;
                    }
                }
                q_out[9 * f + 3 * k + c] = qn;
            }
        }
    }
    if (part) {
        __shared__ double s0[NT], s1[NT];
        s0[threadIdx.x] = rp;
        s1[threadIdx.x] = rd;
        __syncthreads();
        for (int o = NT / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
            __syncthreads();
        }
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
    }
    griddep_launch_dependents();
}

// ------------------------------------------------------------------ edge ADMM

// z = h . e per face slot, e the orientation-halfedge vector (max - min)
// (eq. TargetDifference); w = z, lambda = 0
template <class T>
__global__ void k_edge_targets(int64_t nf, const int32_t *__restrict__ face_edge, Geo<T> geo, const T *__restrict__ h,
                               T *z, T *w, T *lam) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    for (int k = 0; k < 3; ++k) {
        T ev[3];
        geo.slot_edge(f, k, face_edge[3 * f + k], ev);
        T zz = h[3 * f] * ev[0] + h[3 * f + 1] * ev[1] + h[3 * f + 2] * ev[2];
        z[3 * f + k] = zz;
        w[3 * f + k] = zz;
        lam[3 * f + k] = T(0);
    }
}

// sum of targets per edge and x = their mean
template <class T>
__global__ void k_edge_init(int64_t ne, const int32_t *__restrict__ edge_face, const int32_t *__restrict__ edge_slot,
                            const T *__restrict__ z, T *sz, T *x) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    T s = 0;
    int n = 0;
    for (int j = 0; j < 2; ++j) {
        int f = edge_face[2 * e + j];
        if (f >= 0) { s += z[3 * f + edge_slot[2 * e + j]]; ++n; }
    }
    sz[e] = s;
    x[e] = s / T(n);
}

// face pass of iteration it: the lambda-update of iteration it-1
// (lambda += mu (w - x)) then the W-update w = (I - q q^T/3)(x_f - lambda/mu)
template <class T>
__global__ void k_edge_face_pass(int64_t nf, const int32_t *__restrict__ face_edge, const int8_t *__restrict__ sign,
                                 const T *__restrict__ x, T *w, T *lam, T mu, int do_lambda, const AdmmCtl *ctl) {
    griddep_wait();
    if (ctl && ctl->stop) return;
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    T v[3], q[3];
    T qv = 0;
    for (int k = 0; k < 3; ++k) {
        T xk = x[face_edge[3 * f + k]];
        T l = lam[3 * f + k];
        if (do_lambda) {
            l += mu * (w[3 * f + k] - xk);
            lam[3 * f + k] = l;
        }
        v[k] = xk - l / mu;
        q[k] = (T)sign[3 * f + k];
        qv += q[k] * v[k];
    }
    for (int k = 0; k < 3; ++k) w[3 * f + k] = v[k] - q[k] * qv / T(3);
    griddep_launch_dependents();
}

// X-update (eq. xeupdate, edge_update); with multi-source path constraints
// x = x_hat - delta on the constrained edges (pcm[e] = the edge's index in
// delta, else -1).  Optional residual partials per block: [0] sum (w - x)^2,
// [1] sum (mu dx)^2 over the edge's slots
template <class T>
__global__ void __launch_bounds__(NT) k_edge_edge_pass(int64_t ne, const int32_t *__restrict__ edge_face,
                                                       const int32_t *__restrict__ edge_slot, const T *__restrict__ sz,
                                                       const T *__restrict__ w, const T *__restrict__ lam, T *x, T mu,
                                                       double *part, const AdmmCtl *ctl,
                                                       const int32_t *__restrict__ pcm, const T *__restrict__ pcd) {
    griddep_wait();
    if (ctl && ctl->stop) return;
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rp = 0.0, rd = 0.0;
    if (e < ne) {
        int sl[2];
        // x[e] is read before the update on purpose: with the read issued
        // only for the residuals, the kernel wrote x without reading it and
        // ran 6x slower on GB300 (its L2 compression counters show every
        // written sector of x going through the compressor)
        const T xo = x[e];
        T xn = edge_update(e, edge_face, edge_slot, sz, w, lam, mu, sl);
        if (pcm) {
            const int u = pcm[e];
            if (u >= 0) xn -= pcd[u];
        }
        x[e] = xn;
        if (part) {
            for (int j = 0; j < 2; ++j) {
                if (sl[j] < 0) continue;
                double r = (double)w[sl[j]] - (double)xn;
                rp += r * r;
                double d = (double)mu * ((double)xn - (double)xo);
                rd += d * d;
            }
        }
    }
    if (part) {
        __shared__ double s0[NT], s1[NT];
        s0[threadIdx.x] = rp;
        s1[threadIdx.x] = rd;
        __syncthreads();
        for (int o = NT / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
            __syncthreads();
        }
        if (threadIdx.x == 0) { part[2 * blockIdx.x] = s0[0]; part[2 * blockIdx.x + 1] = s1[0]; }
    }
    griddep_launch_dependents();
}

// sum per-block residual partials in a fixed order: out = sqrt(sum); NaN for
// an iteration that an early stop skipped
__global__ void k_resid_final(const double *__restrict__ part, int nblocks, double *out, const AdmmCtl *ctl) {
    if (ctl && ctl->stop) {
        if (threadIdx.x == 0) out[0] = out[1] = __longlong_as_double(0x7ff8000000000000ll);
        return;
    }
    __shared__ double s0[NT], s1[NT];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += NT) { a += part[2 * i]; b += part[2 * i + 1]; }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) { s0[threadIdx.x] += s0[threadIdx.x + o]; s1[threadIdx.x] += s1[threadIdx.x + o]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { out[0] = sqrt(s0[0]); out[1] = sqrt(s1[0]); }
}

// ------------------------------------------------------------------ path constraints

// Per ADMM iteration, before the block update: the KKT projection of the
// multi-source path constraints (Sec. 5.2) on the constrained variables.
// One CTA: vhat of every constrained variable (face_update / edge_update,
// the update kernel's own code), r_j = sum over constraint j's entries of
// c . vhat (one warp per constraint, fixed order), nu from the Gram factor,
// then delta_u = (1/D_u) sum_j c_uj nu_j, which the update kernel subtracts.
constexpr int PJ = 1024;

template <class T>
__device__ void pc_finish(const PcDev &pc, const T *val, T *delta) {
    __shared__ double s_r[kMaxPc], s_nu[kMaxPc];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, dim = pc.dim, npc = pc.npc;
    if (warp < npc) {
        double acc = 0.0;
        for (int i = pc.off[warp] + lane; i < pc.off[warp + 1]; i += 32) {
            const int u = pc.entu[i];
            for (int c = 0; c < dim; ++c) acc += pc.coef[(size_t)i * dim + c] * (double)val[(size_t)u * dim + c];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s_r[warp] = acc;
    }
    __syncthreads();
    if (tid == 0) pc_solve(pc.L, pc.drop, npc, s_r, s_nu);
    __syncthreads();
    const int nu = pc.meta[0];
    for (int u = tid; u < nu; u += PJ)
        for (int c = 0; c < dim; ++c) {
            double sum = 0.0;
            for (int j = 0; j < npc; ++j) sum += pc.ucoef[((size_t)u * npc + j) * dim + c] * s_nu[j];
            delta[(size_t)u * dim + c] = (T)(pc.dinv[u] * sum);
        }
}

template <class T>
__global__ void __launch_bounds__(PJ, 1) k_pc_project_face(PcDev pc, const int32_t *__restrict__ twin,
                                                        const T *__restrict__ rec, const T *__restrict__ h,
                                                        const T *__restrict__ g_in, const T *__restrict__ q_in, T mu,
                                                        int first, T *val, T *delta, const AdmmCtl *ctl) {
    if (ctl && ctl->stop) return;
    const int nu = pc.meta[0];
    for (int u = threadIdx.x; u < nu; u += PJ) {
        FaceIter<T> s;
        face_update((int64_t)pc.uvar[u], twin, rec, h, g_in, q_in, mu, first, s);
        for (int c = 0; c < 3; ++c) val[3 * u + c] = s.gn[c];
    }
    __syncthreads();
    pc_finish(pc, val, delta);
}

template <class T>
__global__ void __launch_bounds__(PJ, 1) k_pc_project_edge(PcDev pc, const int32_t *__restrict__ edge_face,
                                                        const int32_t *__restrict__ edge_slot,
                                                        const T *__restrict__ sz, const T *__restrict__ w,
                                                        const T *__restrict__ lam, T mu, T *val, T *delta,
                                                        const AdmmCtl *ctl) {
    if (ctl && ctl->stop) return;
    const int nu = pc.meta[0];
    for (int u = threadIdx.x; u < nu; u += PJ) {
        int sl[2];
        val[u] = edge_update((int64_t)pc.uvar[u], edge_face, edge_slot, sz, w, lam, mu, sl);
    }
    __syncthreads();
    pc_finish(pc, val, delta);
}

PcDev pc_dev(const QueryWs &q) {
    return PcDev{q.pc_n, q.pc_dim, q.pc_ent, ptr<int32_t>(q.pc_off), ptr<int32_t>(q.pc_var),
                 ptr<int32_t>(q.pc_entu), ptr<int32_t>(q.pc_uvar), ptr<int32_t>(q.pc_meta), ptr<int32_t>(q.pc_drop),
                 ptr<double>(q.pc_coef), ptr<double>(q.pc_ucoef), ptr<double>(q.pc_dinv), ptr<double>(q.pc_L)};
}

// ------------------------------------------------------------------ integration


// increment of each vertex over its breadth-first pairing vertex k:
// face form  1/|T| sum_{f in T_jk} g_f . (p_j - p_k)   (eq. IntegrationStep)
// edge form  +x_e if v_j is the head of the orientation halfedge, else -x_e
// The increment of each reached vertex over its pairing vertex, in layout
// order: position r holds vertex v = lorder[r].  The chains of pairing
// vertices then run from a set to the previous one, whose positions lie
// close together, so the pointer-jumping rounds below gather nearly
// contiguous data.  nxt[r] is the position of the pairing vertex (-1 on the
// sources); d[r] starts as the increment.
template <class T>
__global__ void k_increments(int nr, const int32_t *__restrict__ lorder, const int32_t *__restrict__ pos,
                             const int32_t *__restrict__ level, const int32_t *__restrict__ parent,
                             const int32_t *__restrict__ pedge, const int32_t *__restrict__ edges,
                             const int32_t *__restrict__ edge_face, const double *__restrict__ P,
                             const T *__restrict__ g, const T *__restrict__ x, int form, int32_t *nxt, double *d,
                             const int32_t *__restrict__ edge_slot, const double *__restrict__ evf) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nr) return;
    const int v = lorder[r];
    if (level[v] == 0) {
        nxt[r] = -1;
        d[r] = 0.0;
        griddep_launch_dependents();
        return;
    }
    const int p = parent[v];
    const int e = pedge[v];   // the edge (v, p), recorded by the breadth-first traversal
    double dv;
    if (form == GH_FORM_EDGE) {
        double xe = (double)x[e];
        dv = (edges[2 * e + 1] == v) ? xe : -xe;
    } else {
        double dp[3] = {0.0, 0.0, 0.0};
        if (!evf) {
            dp[0] = P[3 * (int64_t)v] - P[3 * (int64_t)p];
            dp[1] = P[3 * (int64_t)v + 1] - P[3 * (int64_t)p + 1];
            dp[2] = P[3 * (int64_t)v + 2] - P[3 * (int64_t)p + 2];
        }
        double s = 0.0;
        int n = 0;
        for (int a = 0; a < 2; ++a) {
            int f = edge_face[2 * e + a];
            if (f < 0) continue;
            if (evf) {   // an intrinsic triangulation: p_v - p_p in face f's frame, its slot vector
                const double *sv = evf + 9 * (int64_t)f + 3 * edge_slot[2 * e + a];
                const double sg = (v > p) ? 1.0 : -1.0;
                dp[0] = sg * sv[0]; dp[1] = sg * sv[1]; dp[2] = sg * sv[2];
            }
            s += (double)g[3 * (int64_t)f] * dp[0] + (double)g[3 * (int64_t)f + 1] * dp[1] +
                 (double)g[3 * (int64_t)f + 2] * dp[2];
            ++n;
        }
        dv = s / n;
    }
    nxt[r] = pos[p];
    d[r] = dv;
    griddep_launch_dependents();
}

// the distances in vertex order, +infinity where no source reaches, with the
// last pointer-jumping round folded in: d_in / n_in are the chains before it
// (after it every chain has reached its source)
__global__ void k_gather_d(int64_t nv, const int32_t *__restrict__ pos, const double *__restrict__ d_in,
                           const int32_t *__restrict__ n_in, double *d) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const int r = pos[v];
    griddep_wait();   // d_in and n_in come from the previous kernel
    if (r < 0) {
        d[v] = __longlong_as_double(0x7ff0000000000000ll);
        return;
    }
    const int nx = n_in[r];
    d[v] = (nx >= 0) ? d_in[r] + d_in[nx] : d_in[r];
}

// Sum of the increments along each vertex's chain of pairing vertices by
// pointer jumping: after round r, d[v] holds the sum over the first 2^r
// links and nxt[v] the vertex 2^r links up.  All sets are integrated in
// ceil(log2 L) rounds instead of L dependent steps.
__global__ void k_jump(int64_t nv, const double *__restrict__ d_in, const int32_t *__restrict__ n_in, double *d_out,
                       int32_t *n_out) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    griddep_wait();   // the inputs come from the previous kernel
    int nx = n_in[v];
    if (nx >= 0) {
        d_out[v] = d_in[v] + d_in[nx];
        n_out[v] = n_in[nx];
    } else {
        d_out[v] = d_in[v];
        n_out[v] = -1;
    }
    griddep_launch_dependents();
}

// ------------------------------------------------------------------ heat residual

// per reached vertex r (layout order): (A - t L_c) u - u_0 in FP64
template <class T>
__global__ void __launch_bounds__(NT) k_heat_resid(int n, const int32_t *__restrict__ order,
                                                   const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                                   const int32_t *__restrict__ col_edge,
                                                   const double *__restrict__ theta, const int32_t *__restrict__ pos,
                                                   double t, const T *__restrict__ diag,
                                                   const int32_t *__restrict__ lvl_off, const XVal<T> *__restrict__ U,
                                                   double *part) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (r < n) {
        XVal<T> ur = U[r];
        double uv = ldexp((double)ur.m, max(ur.e, -2000));
        double res = uv / (double)diag[r];   // diag holds 1 / (A_v + t sum theta)
        const int v = order[r];
        for (int j = rowptr[v]; j < rowptr[v + 1]; ++j) {
            const int c = pos[col[j]];
            if (c < 0) continue;
            const T w = (T)(t * theta[col_edge[j]]);   // the weight the sweeps use
            XVal<T> uc = U[c];
            res -= (double)w * ldexp((double)uc.m, max(uc.e, -2000));
        }
        if (r < lvl_off[1]) res -= 1.0;
        acc = res * res;
    }
    __shared__ double s[NT];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = NT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s[0]; part[2 * blockIdx.x + 1] = 0.0; }
}

template <class T> gh_status normalize_t(Ctx *c, const DevMesh &m, QueryWs &q) {
    const XVal<T> *U = ptr<XVal<T>>(q.final_buf ? q.U1 : q.U0);
    k_normalize<T><<<blocks_for(m.nf, NT), NT, 0, c->stream>>>(m.nf, ptr<int32_t>(m.F), ptr<int32_t>(q.pos), U,
                                                              make_geo<T>(m), ptr<T>(q.h)); ++c->launches;
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

// the mesh's static face-form data, built once (under the mesh's lock, and
// finished before any solve may use it)
template <class T> gh_status face_rec(Ctx *c, DevMesh &m, const T *&out) {
    DBuf &buf = sizeof(T) == 4 ? m.face_rec32 : m.face_rec64;
    std::lock_guard<std::mutex> lk(*m.rec_mu);
    if (!buf.p) {
        gh_status s = dalloc(c, buf, sizeof(T) * 13 * (size_t)m.nf);
        if (s != GH_OK) return s;
        k_face_rec<T><<<blocks_for(m.nf, NT), NT, 0, c->stream>>>(m.nf, ptr<double>(m.P), ptr<int32_t>(m.edges),
                                                                 ptr<int32_t>(m.face_edge), ptr<int32_t>(m.twin),
                                                                 ptr<double>(m.Af),
                                                                 m.intrinsic ? ptr<double>(m.evf64) : nullptr,
                                                                 ptr<T>(buf)); ++c->launches;
        GH_CUDA(cudaGetLastError());
        GH_CUDA(cudaStreamSynchronize(c->stream));
    }
    out = ptr<T>(buf);
    return GH_OK;
}

template <class T> gh_status face_admm_t(Ctx *c, DevMesh &m, QueryWs &q, int iters, double mu, bool early,
                                        double eps1, double eps2) {
    cudaStream_t st = c->stream;
    unsigned nb = blocks_for(m.nf, NT);
    const T *rec = nullptr;
    gh_status s = face_rec<T>(c, m, rec);
    if (s != GH_OK) return s;
    T *g[2] = {ptr<T>(q.g0), ptr<T>(q.g1)};
    T *qq[2] = {ptr<T>(q.l0), ptr<T>(q.l1)};   // the q_k of each slot
    if (iters <= 0) {   // no iteration: g = h
        GH_CUDA(cudaMemcpyAsync(g[0], ptr<T>(q.h), sizeof(T) * 3 * m.nf, cudaMemcpyDeviceToDevice, st));
    }
    AdmmCtl *ctl = ptr<AdmmCtl>(q.actl);
    k_ctl_init<<<1, 1, 0, st>>>(ctl, iters); ++c->launches;
    double *part = nullptr;
    if (q.diagnostics || early)
        GH_CUDA(cudaMallocAsync((void **)&part, sizeof(double) * 2 * nb, st));
    if (early) {
        k_face_mnorm2<<<nb, NT, 0, st>>>(m.nf, ptr<int32_t>(m.twin), ptr<double>(m.Af), part); ++c->launches;
        k_ctl_thresholds<<<1, NT, 0, st>>>(part, (int)nb, eps1, eps2, ctl); ++c->launches;
    }
    const bool pc = q.pc_n > 0;
    for (int it = 0; it < iters; ++it) {
        int a = it & 1;
        if (pc) {
            k_pc_project_face<T><<<1, PJ, 0, st>>>(pc_dev(q), ptr<int32_t>(m.twin), rec, ptr<T>(q.h), g[a], qq[a],
                                                  (T)mu, it == 0, ptr<T>(q.pc_val), ptr<T>(q.pc_delta),
                                                  early ? ctl : nullptr); ++c->launches;
        }
        auto kern = m.intrinsic ? k_face_admm<T, true> : k_face_admm<T, false>;
        GH_CUDA(launch_dependent(kern, nb, NT, st, (int64_t)m.nf, ptr<int32_t>(m.twin), rec, ptr<T>(q.h), g[a], qq[a],
                                 g[a ^ 1], qq[a ^ 1], (T)mu, part, early ? ctl : nullptr, (int)(it == 0),
                                 pc ? ptr<int32_t>(q.pc_map) : nullptr, pc ? ptr<T>(q.pc_delta) : nullptr));
        ++c->launches;
        if (part) {
            k_resid_final<<<1, NT, 0, st>>>(part, (int)nb, ptr<double>(q.resid) + 2 * it, early ? ctl : nullptr); ++c->launches;
        }
        if (early) { k_admm_check<<<1, 1, 0, st>>>(ptr<double>(q.resid) + 2 * it, ctl, it); ++c->launches; }
    }
    k_face_final<T><<<blocks_for(3 * m.nf, NT), NT, 0, st>>>(3 * m.nf, g[0], g[1], ctl); ++c->launches;
    if (part) cudaFreeAsync(part, st);
    q.admm_iters = iters;
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

template <class T> gh_status edge_admm_t(Ctx *c, const DevMesh &m, QueryWs &q, int iters, double mu, bool early,
                                        double eps1, double eps2) {
    cudaStream_t st = c->stream;
    unsigned nbf = blocks_for(m.nf, NT), nbe = blocks_for(m.ne, NT);
    Geo<T> geo = make_geo<T>(m);
    k_edge_targets<T><<<nbf, NT, 0, st>>>(m.nf, ptr<int32_t>(m.face_edge), geo, ptr<T>(q.h), ptr<T>(q.z), ptr<T>(q.w),
                                          ptr<T>(q.lam)); ++c->launches;
    k_edge_init<T><<<nbe, NT, 0, st>>>(m.ne, ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot), ptr<T>(q.z),
                                       ptr<T>(q.sz), ptr<T>(q.x)); ++c->launches;
    AdmmCtl *ctl = ptr<AdmmCtl>(q.actl);
    k_ctl_init<<<1, 1, 0, st>>>(ctl, iters); ++c->launches;
    double *part = nullptr;
    const unsigned nbz = blocks_for(3 * m.nf, NT);
    if (q.diagnostics || early)
        GH_CUDA(cudaMallocAsync((void **)&part, sizeof(double) * 2 * std::max(nbe, nbz), st));
    if (early) {
        k_znorm2<T><<<nbz, NT, 0, st>>>(3 * m.nf, ptr<T>(q.z), part); ++c->launches;
        k_ctl_thresholds<<<1, NT, 0, st>>>(part, (int)nbz, eps1, eps2, ctl); ++c->launches;
    }
    const AdmmCtl *cx = early ? ctl : nullptr;
    const bool pc = q.pc_n > 0;
    for (int it = 0; it < iters; ++it) {
        GH_CUDA(launch_dependent(k_edge_face_pass<T>, nbf, NT, st, (int64_t)m.nf, ptr<int32_t>(m.face_edge),
                                 ptr<int8_t>(m.face_sign), ptr<T>(q.x), ptr<T>(q.w), ptr<T>(q.lam), (T)mu,
                                 (int)(it > 0), cx));
        ++c->launches;
        if (pc) {
            k_pc_project_edge<T><<<1, PJ, 0, st>>>(pc_dev(q), ptr<int32_t>(m.edge_face), ptr<int32_t>(m.edge_slot),
                                                  ptr<T>(q.sz), ptr<T>(q.w), ptr<T>(q.lam), (T)mu, ptr<T>(q.pc_val),
                                                  ptr<T>(q.pc_delta), cx); ++c->launches;
        }
        GH_CUDA(launch_dependent(k_edge_edge_pass<T>, nbe, NT, st, (int64_t)m.ne, ptr<int32_t>(m.edge_face),
                                 ptr<int32_t>(m.edge_slot), ptr<T>(q.sz), ptr<T>(q.w), ptr<T>(q.lam), ptr<T>(q.x),
                                 (T)mu, part, cx, pc ? ptr<int32_t>(q.pc_map) : nullptr,
                                 pc ? ptr<T>(q.pc_delta) : nullptr));
        ++c->launches;
        if (part) { k_resid_final<<<1, NT, 0, st>>>(part, (int)nbe, ptr<double>(q.resid) + 2 * it, cx); ++c->launches; }
        if (early) { k_admm_check<<<1, 1, 0, st>>>(ptr<double>(q.resid) + 2 * it, ctl, it); ++c->launches; }
    }
    if (part) cudaFreeAsync(part, st);
    q.admm_iters = iters;
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

template <class T> gh_status integrate_t(Ctx *c, const DevMesh &m, QueryWs &q, double *d_out) {
    cudaStream_t st = c->stream;
    const int nr = q.nreach;
    // position-ordered chains ping-pong between (inc, n0) and (d1, n1); the
    // result goes to d0 in vertex order (read by gh_debug_dump)
    double *d[2] = {ptr<double>(q.inc), ptr<double>(q.d1)};
    int32_t *n[2] = {ptr<int32_t>(q.n0), ptr<int32_t>(q.n1)};
    if (nr > 0) {
        k_increments<T><<<blocks_for(nr, NT), NT, 0, st>>>(
            nr, ptr<int32_t>(q.lorder), ptr<int32_t>(q.pos), ptr<int32_t>(q.level), ptr<int32_t>(q.parent),
            ptr<int32_t>(q.pedge), ptr<int32_t>(m.edges), ptr<int32_t>(m.edge_face), ptr<double>(m.P),
            ptr<T>(q.g0), ptr<T>(q.x), q.form, n[0], d[0], ptr<int32_t>(m.edge_slot),
            m.intrinsic ? ptr<double>(m.evf64) : nullptr); ++c->launches;
    }
    int rounds = 0;
    while ((1 << rounds) < q.nlev) ++rounds;
    int cur = 0;
    for (int r = 0; r + 1 < rounds && nr > 0; ++r) {   // the last round runs inside the gather
        GH_CUDA(launch_dependent(k_jump, blocks_for(nr, NT), NT, st, (int64_t)nr, (const double *)d[cur],
                                 (const int32_t *)n[cur], d[cur ^ 1], n[cur ^ 1]));
        ++c->launches;
        cur ^= 1;
    }
    GH_CUDA(launch_dependent(k_gather_d, blocks_for(m.nv, NT), NT, st, (int64_t)m.nv, (const int32_t *)ptr<int32_t>(q.pos),
                             (const double *)d[cur], (const int32_t *)n[cur], ptr<double>(q.d0)));
    ++c->launches;
    if (d_out) GH_CUDA(cudaMemcpyAsync(d_out, ptr<double>(q.d0), sizeof(double) * m.nv, cudaMemcpyDeviceToDevice, st));
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

template <class T> gh_status heat_resid_t(Ctx *c, const DevMesh &m, QueryWs &q) {
    cudaStream_t st = c->stream;
    int n = q.nreach;
    unsigned nb = blocks_for(n, NT);
    double *part = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&part, sizeof(double) * 2 * nb, st));
    k_heat_resid<T><<<nb, NT, 0, st>>>(n, ptr<int32_t>(q.lorder), ptr<int32_t>(m.rowptr), ptr<int32_t>(m.col),
                                       ptr<int32_t>(m.col_edge), ptr<double>(m.theta), ptr<int32_t>(q.pos), q.t,
                                       ptr<T>(q.diag), ptr<int32_t>(q.lvl_off), ptr<XVal<T>>(q.final_buf ? q.U1 : q.U0),
                                       part); ++c->launches;
    double *tmp = nullptr;
    GH_CUDA(cudaMallocAsync((void **)&tmp, sizeof(double) * 2, st));
    k_resid_final<<<1, NT, 0, st>>>(part, (int)nb, tmp, nullptr); ++c->launches;
    GH_CUDA(cudaMemcpyAsync(q.e1.p, tmp, sizeof(double), cudaMemcpyDeviceToDevice, st));
    cudaFreeAsync(part, st);
    cudaFreeAsync(tmp, st);
    GH_CUDA(cudaGetLastError());
    return GH_OK;
}

}  // namespace

gh_status run_normalize(Ctx *c, const DevMesh &m, QueryWs &q) {
    return q.fp64 ? normalize_t<double>(c, m, q) : normalize_t<float>(c, m, q);
}
gh_status run_face_admm(Ctx *c, DevMesh &m, QueryWs &q, const gh_params *p) {
    q.form = GH_FORM_FACE;
    const bool early = p->early_stop != 0;
    return q.fp64 ? face_admm_t<double>(c, m, q, p->admm_iters, p->mu, early, p->eps1, p->eps2)
                  : face_admm_t<float>(c, m, q, p->admm_iters, p->mu, early, p->eps1, p->eps2);
}
gh_status run_edge_admm(Ctx *c, const DevMesh &m, QueryWs &q, const gh_params *p) {
    q.form = GH_FORM_EDGE;
    const bool early = p->early_stop != 0;
    return q.fp64 ? edge_admm_t<double>(c, m, q, p->admm_iters, p->mu, early, p->eps1, p->eps2)
                  : edge_admm_t<float>(c, m, q, p->admm_iters, p->mu, early, p->eps1, p->eps2);
}
gh_status run_integrate(Ctx *c, const DevMesh &m, QueryWs &q, double *d_out_dev) {
    return q.fp64 ? integrate_t<double>(c, m, q, d_out_dev) : integrate_t<float>(c, m, q, d_out_dev);
}
gh_status run_heat_residual(Ctx *c, const DevMesh &m, QueryWs &q) {
    return q.fp64 ? heat_resid_t<double>(c, m, q) : heat_resid_t<float>(c, m, q);
}

}  // namespace gh
