"""FP64 oracle of the element residual / tangent with the MLP surrogate as the material law
(test infrastructure only).

At each Gauss point: F = I + grad u, E = 1/2 (F^T F - I); if every |E_ij| <= range, S and
D = dS/dE come from the FP64 network (oracle.mlp.surrogate_stress), otherwise from the
plain neo-Hookean law.  The fourth-order tangent is rebuilt from D (D differentiates with
respect to the tensor components of E, so a shear column carries both E_KL and E_LK):
CC_IJKL = D[a(IJ)][b(KL)] for K == L and D[a(IJ)][b(KL)] / 2 otherwise.  Then the plain
definitions R_e(a,i) = sum_q w detJ P_iJ G_aJ and
K_e(a,i)(b,k) = sum_q w detJ G_aJ (delta_ik S_JL + F_iI CC_IJKL F_kK) G_bL.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import fem, mlp

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def _geometry(X):
    dp = C.POINTER(C.c_double)
    out = []
    for q in range(8):
        xi = np.zeros(3)
        fem.lib().or_gauss_point(q, xi.ctypes.data_as(dp))
        N = np.zeros(8)
        dN = np.zeros((8, 3))
        fem.lib().or_shape(xi.ctypes.data_as(dp), N.ctypes.data_as(dp), dN.ctypes.data_as(dp))
        G = np.zeros((8, 3))
        d = C.c_double()
        Xc = np.ascontiguousarray(X)
        st = fem.lib().or_geometry(Xc.ctypes.data_as(dp), dN.ctypes.data_as(dp), G.ctypes.data_as(dp), C.byref(d))
        if st:
            raise fem.OracleError("inverted element")
        out.append((G, d.value))
    return out


def _voigt(T):
    return np.array([T[i, j] for i, j in VOIGT])


def _tensor(v):
    return np.array([[v[0], v[5], v[4]], [v[5], v[1], v[3]], [v[4], v[3], v[2]]])


def element(mesh: fem.Mesh, e: int, u, layers, in_scale, rng, out_scale, out_shift):
    """Element e: R_e [24], K_e [24, 24] (rows and columns (a, i)), the number of its Gauss
    points that fell back to the plain law, and the strains E [8, 6] (Voigt, tensor shear)."""
    en = mesh.conn[e].astype(np.int64)
    X = mesh.coords[en]
    ue = u[(3 * en[:, None] + np.arange(3))].reshape(8, 3)
    p = int(mesh.phase[e])
    pts = []
    for G, detJ in _geometry(X):
        F = np.eye(3) + ue.T @ G
        pts.append((G, detJ, F, _voigt(0.5 * (F.T @ F - np.eye(3)))))
    E6 = np.array([q[3] for q in pts])
    S_net, D_net = mlp.surrogate_stress(layers, E6, np.full(8, p), in_scale, out_scale, out_shift)
    Re = np.zeros(24)
    Ke = np.zeros((24, 24))
    fallback = 0
    for r, (G, detJ, F, _) in enumerate(pts):
        if np.all(np.abs(E6[r]) <= rng):
            S = _tensor(S_net[r])
            D = D_net[r]
            CC = np.zeros((3, 3, 3, 3))
            for a, (I, J) in enumerate(VOIGT):
                for b, (Kk, L) in enumerate(VOIGT):
                    v = D[a, b] if Kk == L else 0.5 * D[a, b]
                    for (i1, j1) in {(I, J), (J, I)}:
                        for (k1, l1) in {(Kk, L), (L, Kk)}:
                            CC[i1, j1, k1, l1] = v
        else:
            fallback += 1
            lam, mu = fem.lame(mesh.mat_E[p], mesh.mat_nu[p])
            S, CC = fem.neo_hookean(lam, mu, F)
        P = F @ S
        A = np.einsum("ik,JL->iJkL", np.eye(3), S) + np.einsum("iI,IJKL,kK->iJkL", F, CC, F)
        Re += detJ * (P @ G.T).T.ravel()  # [a, i]
        Ke += detJ * np.einsum("aJ,iJkL,bL->aibk", G, A, G).reshape(24, 24)
    return Re, Ke, fallback, E6


def assemble(mesh: fem.Mesh, u, layers, in_scale, rng, out_scale, out_shift):
    """Dense K (n_dof x n_dof), R (n_dof), the number of fallback Gauss points and the strains
    of every Gauss point (element by element)."""
    n_dof = mesh.n_dof
    K = np.zeros((n_dof, n_dof))
    R = np.zeros(n_dof)
    fallback = 0
    E6_all = []
    for e in range(mesh.n_elem):
        Re, Ke, fb, E6 = element(mesh, e, u, layers, in_scale, rng, out_scale, out_shift)
        en = mesh.conn[e].astype(np.int64)
        d = (3 * en[:, None] + np.arange(3)).ravel()
        R[d] += Re
        K[np.ix_(d, d)] += Ke
        fallback += fb
        E6_all.append(E6)
    return K, R, fallback, np.concatenate(E6_all) if E6_all else np.zeros((0, 6))


def sampled_rows(mesh: fem.Mesh, u, nodes, layers, in_scale, rng, out_scale, out_shift, adjacency=None):
    """Rows of R and K at a sample of nodes, summed element by element over the elements around
    each node (for meshes too big to assemble densely).  Returns dict node -> (R[3],
    {col: K[3]}), and the strains [m, 6] and phases [m] of the Gauss points of those elements."""
    ptr, eidx = adjacency if adjacency is not None else fem.node_elements(mesh.conn, mesh.n_nodes)
    out, E6s, phs, cache = {}, [], [], {}
    for n in nodes:
        n = int(n)
        R = np.zeros(3)
        krow = {}
        for e in eidx[ptr[n]:ptr[n + 1]]:
            e = int(e)
            if e not in cache:
                cache[e] = element(mesh, e, u, layers, in_scale, rng, out_scale, out_shift)
                E6s.append(cache[e][3])
                phs.append(np.full(8, int(mesh.phase[e])))
            Re, Ke = cache[e][0], cache[e][1]
            en = mesh.conn[e].astype(np.int64)
            a = int(np.where(en == n)[0][0])
            R += Re[3 * a:3 * a + 3]
            for b in range(8):
                for k in range(3):
                    c = 3 * int(en[b]) + k
                    krow[c] = krow.get(c, np.zeros(3)) + Ke[3 * a:3 * a + 3, 3 * b + k]
        out[n] = (R, krow)
    return out, np.concatenate(E6s), np.concatenate(phs)
