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


def assemble(mesh: fem.Mesh, u, layers, in_scale, rng, out_scale, out_shift):
    """Dense K (n_dof x n_dof), R (n_dof) and the number of fallback Gauss points."""
    n_dof = mesh.n_dof
    K = np.zeros((n_dof, n_dof))
    R = np.zeros(n_dof)
    recs = []
    E6_all, ph_all = [], []
    for e in range(mesh.n_elem):
        en = mesh.conn[e].astype(np.int64)
        X = mesh.coords[en]
        ue = u[(3 * en[:, None] + np.arange(3))].reshape(8, 3)
        for G, detJ in _geometry(X):
            F = np.eye(3) + ue.T @ G
            E6_all.append(_voigt(0.5 * (F.T @ F - np.eye(3))))
            ph_all.append(int(mesh.phase[e]))
            recs.append((e, en, G, detJ, F))
    E6_all = np.array(E6_all)
    ph_all = np.array(ph_all)
    S_net, D_net = mlp.surrogate_stress(layers, E6_all, ph_all, in_scale, out_scale, out_shift)
    fallback = 0
    for r, (e, en, G, detJ, F) in enumerate(recs):
        p = ph_all[r]
        if np.all(np.abs(E6_all[r]) <= rng):
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
        Re = detJ * (P @ G.T).T.ravel()  # [a, i]
        Ke = detJ * np.einsum("aJ,iJkL,bL->aibk", G, A, G).reshape(24, 24)
        d = (3 * en[:, None] + np.arange(3)).ravel()
        R[d] += Re
        K[np.ix_(d, d)] += Ke
    return K, R, fallback, E6_all
