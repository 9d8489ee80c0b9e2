"""ctypes wrapper over the C oracle plus the parts that are plain numpy.

Test infrastructure only (see the package docstring).  Functions follow the paper's
problem statement (Section II-A: R(u) = 0 assembled from element contributions, K = dR/du
sparse globally and dense per element; Section III-B: the sparse pattern is fixed before
the values, duplicates summed).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from .build import build

LAW_LINEAR_ELASTIC = 0
LAW_NEO_HOOKEAN = 1

_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lp = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.or_lame.argtypes = [C.c_double, C.c_double, _dp, _dp]
        L.or_element.argtypes = [C.c_int, C.c_double, C.c_double, _dp, _dp, _dp, _dp]
        L.or_element_of.argtypes = [C.c_int64, _ip, _dp, _dp, _ip, _dp, _dp, _ip, _dp, _dp, _dp]
        L.or_residual.argtypes = [C.c_int64, C.c_int64, _ip, _dp, _dp, _ip, _dp, _dp, _ip, _dp, _dp]
        L.or_tangent_csr.argtypes = [C.c_int64, C.c_int64, _ip, _dp, _dp, _ip, _dp, _dp, _ip, _dp,
                                     _lp, _ip, _dp, _dp]
        L.or_apply_tangent.argtypes = [C.c_int64, C.c_int64, _ip, _dp, _dp, _dp, _ip, _dp, _dp, _ip,
                                       _dp, _dp]
        L.or_spmv.argtypes = [C.c_int64, _lp, _ip, _dp, _dp, _dp]
        L.or_material_grad.argtypes = [C.c_int64, C.c_int64, _ip, _dp, _dp, _ip, _dp, _dp, _ip, _dp,
                                       _dp, _dp]
        L.or_energy.argtypes = [C.c_int64, _ip, _dp, _dp, _ip, _dp, _dp, _ip, _dp, _dp]
        L.or_neo_hookean.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_linear_elastic.argtypes = [C.c_double, C.c_double, _dp, _dp, _dp]
        L.or_geometry.argtypes = [_dp, _dp, _dp, _dp]
        L.or_shape.argtypes = [_dp, _dp, _dp]
        L.or_gauss_point.argtypes = [C.c_int, _dp]
        for f in ("or_element", "or_element_of", "or_residual", "or_tangent_csr", "or_apply_tangent",
                  "or_material_grad", "or_energy", "or_neo_hookean", "or_geometry"):
            getattr(L, f).restype = C.c_int
    return _lib


class OracleError(RuntimeError):
    pass


def _chk(st):
    if st != 0:
        raise OracleError({1: "bad argument", 2: "inverted element (detJ <= 0)",
                           3: "inadmissible state (det F <= 0)", 4: "entry missing from pattern"}
                          .get(st, f"status {st}"))


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def _l(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_lp)


def _opt_d(a):
    if a is None:
        return None, None
    return _d(a)


def lame(E, nu):
    lam, mu = C.c_double(), C.c_double()
    lib().or_lame(E, nu, C.byref(lam), C.byref(mu))
    return lam.value, mu.value


class Mesh:
    """Host arrays of one problem, kept contiguous for the C calls."""

    def __init__(self, coords, conn, phase, materials, E_elem=None):
        self.coords, self.p_coords = _d(coords)
        self.conn, self.p_conn = _i(conn)
        self.phase, self.p_phase = _i(phase)
        self.n_nodes = int(self.coords.shape[0])
        self.n_elem = int(self.conn.shape[0])
        self.mat_E, self.p_E = _d([m[0] for m in materials])
        self.mat_nu, self.p_nu = _d([m[1] for m in materials])
        self.mat_law, self.p_law = _i([m[2] for m in materials])
        self.E_elem, self.p_Eel = _opt_d(E_elem)

    @classmethod
    def of(cls, prob, E_elem="problem"):
        return cls(prob.coords, prob.conn, prob.phase, prob.materials,
                   prob.E_elem if isinstance(E_elem, str) else E_elem)

    @property
    def n_dof(self):
        return 3 * self.n_nodes

    def _mat(self):
        return (self.p_phase, self.p_E, self.p_nu, self.p_law, self.p_Eel)


def element(law, lam, mu, X, ue, tangent=True):
    """Element residual (24) and tangent (24x24) of one hex8 element."""
    X, pX = _d(np.reshape(X, (8, 3)))
    ue, pu = _d(np.reshape(ue, 24))
    Re = np.zeros(24)
    Ke = np.zeros((24, 24)) if tangent else None
    _chk(lib().or_element(law, lam, mu, pX, pu, Re.ctypes.data_as(_dp),
                          Ke.ctypes.data_as(_dp) if tangent else None))
    return (Re, Ke) if tangent else Re


def element_of(mesh: Mesh, e: int, u, tangent=True):
    u, pu = _d(u)
    Re = np.zeros(24)
    Ke = np.zeros((24, 24)) if tangent else None
    _chk(lib().or_element_of(e, mesh.p_conn, mesh.p_coords, pu, *mesh._mat(), Re.ctypes.data_as(_dp),
                             Ke.ctypes.data_as(_dp) if tangent else None))
    return (Re, Ke) if tangent else Re


def residual(mesh: Mesh, u):
    u, pu = _d(u)
    R = np.zeros(mesh.n_dof)
    _chk(lib().or_residual(mesh.n_elem, mesh.n_nodes, mesh.p_conn, mesh.p_coords, pu, *mesh._mat(),
                           R.ctypes.data_as(_dp)))
    return R


def csr_pattern(conn, n_nodes):
    """Sparsity pattern of K from the element connectivity: every (row, col) pair of every
    element's 24x24 block, sorted and de-duplicated.  Returns (rowptr int64, col int32)."""
    conn = np.asarray(conn, dtype=np.int64)
    n_dof = 3 * n_nodes
    if conn.shape[0] == 0:
        return np.zeros(n_dof + 1, dtype=np.int64), np.zeros(0, dtype=np.int32)
    dofs = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(len(conn), 24)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    key = np.unique(rows * n_dof + cols)
    r, c = key // n_dof, key % n_dof
    rowptr = np.zeros(n_dof + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    return np.cumsum(rowptr), c.astype(np.int32)


def tangent_csr(mesh: Mesh, u, rowptr, col, with_residual=True):
    u, pu = _d(u)
    rowptr, prp = _l(rowptr)
    col, pcol = _i(col)
    vals = np.zeros(len(col))
    R = np.zeros(mesh.n_dof) if with_residual else None
    _chk(lib().or_tangent_csr(mesh.n_elem, mesh.n_nodes, mesh.p_conn, mesh.p_coords, pu, *mesh._mat(),
                              prp, pcol, vals.ctypes.data_as(_dp),
                              R.ctypes.data_as(_dp) if with_residual else None))
    return (vals, R) if with_residual else vals


def apply_tangent(mesh: Mesh, u, v):
    u, pu = _d(u)
    v, pv = _d(v)
    y = np.zeros(mesh.n_dof)
    _chk(lib().or_apply_tangent(mesh.n_elem, mesh.n_nodes, mesh.p_conn, mesh.p_coords, pu, pv,
                                *mesh._mat(), y.ctypes.data_as(_dp)))
    return y


def spmv(rowptr, col, vals, v):
    rowptr, prp = _l(rowptr)
    col, pcol = _i(col)
    vals, pv = _d(vals)
    v, pvv = _d(v)
    y = np.zeros(len(rowptr) - 1)
    lib().or_spmv(len(rowptr) - 1, prp, pcol, pv, pvv, y.ctypes.data_as(_dp))
    return y


def material_grad(mesh: Mesh, u, R=None):
    """dL/dE per element for L = 1/2 ||R(u; E)||^2 (needs per-element E or phase moduli)."""
    if R is None:
        R = residual(mesh, u)
    u, pu = _d(u)
    R, pR = _d(R)
    g = np.zeros(mesh.n_elem)
    _chk(lib().or_material_grad(mesh.n_elem, mesh.n_nodes, mesh.p_conn, mesh.p_coords, pu, *mesh._mat(),
                                pR, g.ctypes.data_as(_dp)))
    return g


def energy(mesh: Mesh, u):
    u, pu = _d(u)
    out = C.c_double()
    _chk(lib().or_energy(mesh.n_elem, mesh.p_conn, mesh.p_coords, pu, *mesh._mat(), C.byref(out)))
    return out.value


def norm2(x):
    """Euclidean norm with a correctly rounded sum of squares (math.fsum)."""
    x = np.asarray(x, dtype=np.float64)
    return math.sqrt(math.fsum((x * x).tolist()))


def neo_hookean(lam, mu, F):
    F, pF = _d(np.reshape(F, (3, 3)))
    S = np.zeros((3, 3))
    CC = np.zeros((3, 3, 3, 3))
    _chk(lib().or_neo_hookean(lam, mu, pF, S.ctypes.data_as(_dp), CC.ctypes.data_as(_dp)))
    return S, CC


def linear_elastic(lam, mu, H):
    H, pH = _d(np.reshape(H, (3, 3)))
    sig = np.zeros((3, 3))
    D = np.zeros((3, 3, 3, 3))
    lib().or_linear_elastic(lam, mu, pH, sig.ctypes.data_as(_dp), D.ctypes.data_as(_dp))
    return sig, D


def node_elements(conn, n_nodes):
    """Node -> adjacent elements (CSR: ptr int64 [n_nodes+1], idx int64)."""
    conn = np.asarray(conn, dtype=np.int64)
    flat = conn.ravel()
    order = np.argsort(flat, kind="stable")
    ptr = np.zeros(n_nodes + 1, dtype=np.int64)
    np.add.at(ptr, flat + 1, 1)
    return np.cumsum(ptr), order // 8


def sampled_rows(mesh: Mesh, u, v, nodes, adjacency=None):
    """Oracle rows for a sample of nodes, computed element by element (for meshes too big
    to assemble on the CPU).  Returns dict node -> (R[3], Kv[3], {col: K[3]})."""
    ptr, eidx = adjacency if adjacency is not None else node_elements(mesh.conn, mesh.n_nodes)
    out = {}
    for n in nodes:
        n = int(n)
        R = np.zeros(3)
        Kv = np.zeros(3)
        krow = {}
        for e in eidx[ptr[n]:ptr[n + 1]]:
            e = int(e)
            Re, Ke = element_of(mesh, e, u)
            en = mesh.conn[e].astype(np.int64)
            a = int(np.where(en == n)[0][0])
            R += Re[3 * a:3 * a + 3]
            ve = v[(3 * en[:, None] + np.arange(3)).ravel()]
            Kv += Ke[3 * a:3 * a + 3] @ ve
            for b in range(8):
                for k in range(3):
                    c = 3 * int(en[b]) + k
                    krow[c] = krow.get(c, np.zeros(3)) + Ke[3 * a:3 * a + 3, 3 * b + k]
        out[n] = (R, Kv, krow)
    return out
