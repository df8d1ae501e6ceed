// The unconstrained block updates of both ADMM forms, per face and per edge.
// The update kernels (stages.cu) and the path-constraint projections
// (paths.cu) compute them with the same code, so a projection sees exactly
// the values the update kernel subtracts its correction from.
#pragma once

#include "internal.cuh"

namespace gh {

// four values loaded as one vector (16 bytes in FP32, 32 in FP64)
template <class T> struct alignas(4 * sizeof(T)) Quad { T x, y, z, w; };

// One face of a face-form iteration (Sec. 3.2) up to the G-update:
//   q_k = g - lambda_k/(mu alpha) per slot (the first iteration starts from
//   g = h, lambda = 0, so q_k = h), then
//   y_k = q_k + A'/(A + A') ebar (ebar . (q'_k - q_k))   (q' of the twin slot)
//   gn  = (2h + mu sum_k (y_k + g - q_k)) / (2 + mu n)
// over the n interior slots.  rec holds 12 values per face (per slot the unit
// edge vector and the twin weight A'/(A + A'); 48 bytes in FP32), then
// sqrt(A_f) of every face at rec[12 nf + f].  INTR: an intrinsic
// triangulation (Sec. 5.3), where every face has its own frame and its own
// unit vector e of each edge; the condition e . y = e' . y' then gives
// y_k = q_k + A'/(A + A') e (e' . q'_k - e . q_k), the twin's e' read from
// the twin's record (the same update when e = e').
template <class T> struct FaceIter {
    T g[3], q[3][3], y[3][3], gn[3];
    bool in[3];
};

template <class T, bool INTR = false>
__device__ __forceinline__ void face_update(int64_t f, const int32_t *__restrict__ twin, const T *__restrict__ rec,
                                            const T *__restrict__ h, const T *__restrict__ g_in,
                                            const T *__restrict__ q_in, T mu, int first, FaceIter<T> &s) {
    const Quad<T> *r4 = reinterpret_cast<const Quad<T> *>(rec + 12 * f);
    const Quad<T> ek[3] = {r4[0], r4[1], r4[2]};
    const T *gsrc = first ? h : g_in;
    for (int c = 0; c < 3; ++c) s.g[c] = gsrc[3 * f + c];
    T acc[3] = {0, 0, 0};
    int n = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int c = 0; c < 3; ++c) s.q[k][c] = first ? s.g[c] : q_in[9 * f + 3 * k + c];
        const int tw = twin[3 * f + k];
        s.in[k] = tw >= 0;
        if (!s.in[k]) continue;
        const T *qt = first ? h + 3 * (int64_t)(tw >> 2) : q_in + 9 * (int64_t)(tw >> 2) + 3 * (tw & 3);
        const T eb[3] = {ek[k].x, ek[k].y, ek[k].z};
        T proj;
        if (INTR) {
            const T *et = rec + 12 * (int64_t)(tw >> 2) + 4 * (tw & 3);
            proj = (et[0] * qt[0] + et[1] * qt[1] + et[2] * qt[2]) -
                   (eb[0] * s.q[k][0] + eb[1] * s.q[k][1] + eb[2] * s.q[k][2]);
        } else {
            proj = eb[0] * (qt[0] - s.q[k][0]) + eb[1] * (qt[1] - s.q[k][1]) + eb[2] * (qt[2] - s.q[k][2]);
        }
        for (int c = 0; c < 3; ++c) {
            s.y[k][c] = s.q[k][c] + ek[k].w * eb[c] * proj;
            acc[c] += s.y[k][c] + (s.g[c] - s.q[k][c]);
        }
        ++n;
    }
    const T den = T(2) + mu * T(n);
    for (int c = 0; c < 3; ++c) s.gn[c] = (T(2) * h[3 * f + c] + mu * acc[c]) / den;
}

// The X-update of one edge (eq. xeupdate):
//   x_e = (sum z + sum (lambda + mu w)) / (n_e (1 + mu))
// over the edge's n_e slots; sl receives the slots (-1 where absent).
template <class T>
__device__ __forceinline__ T edge_update(int64_t e, const int32_t *__restrict__ edge_face,
                                         const int32_t *__restrict__ edge_slot, const T *__restrict__ sz,
                                         const T *__restrict__ w, const T *__restrict__ lam, T mu, int sl[2]) {
    T s = sz[e];
    int n = 0;
    for (int j = 0; j < 2; ++j) {
        const int f = edge_face[2 * e + j];
        sl[j] = -1;
        if (f >= 0) {
            sl[j] = 3 * f + edge_slot[2 * e + j];
            s += lam[sl[j]] + mu * w[sl[j]];
            ++n;
        }
    }
    return s / (T(n) * (T(1) + mu));
}

// Device view of one query's multi-source path constraints (built per solve
// by paths.cu).  Constraint j is sum_i coef_i . v_{var_i} = 0 over entries
// [off[j], off[j+1]); entu maps an entry to its distinct variable, uvar a
// distinct index to its variable (meta[0] of them), ucoef holds the
// coefficients summed per distinct variable and constraint ([u][j][dim]),
// dinv 1/D per distinct variable, L the lower Cholesky factor of the Gram
// matrix C D^-1 C^T ([npc][npc]) and drop its dropped constraints.
struct PcDev {
    int npc, dim, nent;
    const int32_t *off, *var, *entu, *uvar, *meta, *drop;
    const double *coef, *ucoef, *dinv, *L;
};

// nu from L L^T nu = r with the dropped constraints held at 0 (one thread)
__device__ inline void pc_solve(const double *L, const int32_t *drop, int n, const double *r, double *nu) {
    for (int j = 0; j < n; ++j) {
        if (drop[j]) { nu[j] = 0.0; continue; }
        double s = r[j];
        for (int m = 0; m < j; ++m) s -= L[j * n + m] * nu[m];
        nu[j] = s / L[j * n + j];
    }
    for (int j = n - 1; j >= 0; --j) {
        if (drop[j]) { nu[j] = 0.0; continue; }
        double s = nu[j];
        for (int m = j + 1; m < n; ++m) s -= L[m * n + j] * nu[m];
        nu[j] = s / L[j * n + j];
    }
}

}  // namespace gh
