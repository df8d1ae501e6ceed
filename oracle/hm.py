"""Direct-solve references for the oracle (TEST INFRASTRUCTURE ONLY).

The original heat method the paper starts from (Sec. 1, Sec. 3.1 eq. heat,
Sec. 3.2's Poisson system L d = b) solves two sparse linear systems directly.
Here scipy's sparse LU is the library routine for those solves.  They pin the
iterative stages of the oracle:

* ``heat_direct``: the solution of (A - t L_c) u = u_0 that the Gauss-Seidel
  sweeps converge to.
* ``poisson_face``: the scalar field whose face gradients are closest to h in
  the area-weighted least-squares sense.  On a genus-0 mesh the integrable
  fields are exactly the gradient fields, so this is the limit of the
  face-based ADMM of Sec. 3.2 integrated as in Sec. 3.3.
* ``lsq_edge``: the scalar field whose edge differences are closest to the
  targets z in the least-squares sense of Sec. 4.1; on a genus-0 mesh closed
  1-forms are exact, so this is the limit of the edge-based ADMM.

All three return plain doubles and only make sense on small meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as sla


def cotan_stiffness(md) -> sp.csr_matrix:
    """K = -L_c: K_vw = -theta_vw, K_vv = sum_w theta_vw."""
    rows = np.repeat(np.arange(md.nv), np.diff(md.rowptr))
    W = sp.csr_matrix((md.theta[md.col_edge], (rows, md.col)), shape=(md.nv, md.nv))
    return (sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W).tocsr()


def heat_direct(md, sources, t: float) -> np.ndarray:
    u0 = np.zeros(md.nv)
    u0[np.asarray(sources)] = 1.0
    A = sp.diags(md.Av) + t * cotan_stiffness(md)
    return sla.spsolve(A.tocsc(), u0)


def _solve_pinned(K: sp.csr_matrix, b: np.ndarray, pin: int) -> np.ndarray:
    """Solve K phi = b with phi[pin] = 0 (K singular with constant kernel)."""
    n = K.shape[0]
    keep = np.ones(n, bool)
    keep[pin] = False
    Kr = K[keep][:, keep].tocsc()
    phi = np.zeros(n)
    phi[keep] = sla.spsolve(Kr, b[keep])
    return phi


def face_gradient_basis(md):
    """grad of the hat function of corner k on face f: (N x e_k) / (2 A_f),
    e_k the edge opposite corner k, counter-clockwise.  Shape [nf, 3, 3]."""
    P = md.P[md.F]                                   # [nf, 3 corners, 3]
    n = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    twoA = np.linalg.norm(n, axis=1)
    N = n / twoA[:, None]
    out = np.empty((md.nf, 3, 3))
    for k in range(3):
        e = P[:, (k + 2) % 3] - P[:, (k + 1) % 3]
        out[:, k] = np.cross(N, e) / twoA[:, None]
    return out


def poisson_face(md, h: np.ndarray, pin: int) -> np.ndarray:
    """argmin_phi sum_f A_f |grad phi - h_f|^2 with phi[pin] = 0:
    K phi = b, b_v = sum_f A_f h_f . grad B_v."""
    G = face_gradient_basis(md)
    contrib = md.Af[:, None] * np.einsum("fkc,fc->fk", G, h)
    b = np.zeros(md.nv)
    np.add.at(b, md.F.ravel(), contrib.ravel())
    return _solve_pinned(cotan_stiffness(md), b, pin)


def lsq_edge(md, z: np.ndarray, pin: int) -> np.ndarray:
    """argmin_phi sum over (face, slot) of (phi(head) - phi(tail) - z)^2 with
    phi[pin] = 0; head/tail of each edge's orientation halfedge."""
    fe = md.face_edge.ravel()
    tail = md.edges[fe, 0].copy()
    head = md.edges[fe, 1].copy()
    if md.flip is not None:
        fl = md.flip[fe].astype(bool)
        tail[fl], head[fl] = head[fl], tail[fl].copy()
    m = fe.size
    B = sp.csr_matrix((np.concatenate([np.ones(m), -np.ones(m)]),
                       (np.concatenate([np.arange(m), np.arange(m)]), np.concatenate([head, tail]))),
                      shape=(m, md.nv))
    return _solve_pinned((B.T @ B).tocsr(), B.T @ z.ravel(), pin)
