"""Pins of the FP64 oracle against facts fixed outside it (CPU only).

Each test ties the oracle to a closed form, an invariant of the mathematics, a brute-force
finite difference or a counting identity, so that a dropped term, a wrong sign, a
transposed index or a misplaced CSR entry in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2604_22087_b300 import inputs as I

LE, NH = I.LAW_LINEAR_ELASTIC, I.LAW_NEO_HOOKEAN
NODE_XI = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=float)


def rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300)


# ---------------------------------------------------------------- shape functions, geometry
def _shape(xi):
    import ctypes as C
    N = np.zeros(8)
    dN = np.zeros((8, 3))
    x = np.ascontiguousarray(xi, dtype=float)
    dp = C.POINTER(C.c_double)
    oracle.lib().or_shape(x.ctypes.data_as(dp), N.ctypes.data_as(dp), dN.ctypes.data_as(dp))
    return N, dN


def test_shape_functions_kronecker_and_partition_of_unity():
    for b in range(8):
        N, _ = _shape(NODE_XI[b])
        assert np.allclose(N, np.eye(8)[b], atol=1e-15)
    xi = np.array([0.3, -0.7, 0.1])
    N, dN = _shape(xi)
    assert abs(N.sum() - 1.0) < 1e-15
    assert np.allclose(dN.sum(axis=0), 0.0, atol=1e-15)
    # derivative by central differences of N itself
    h = 1e-6
    for d in range(3):
        e = np.zeros(3); e[d] = h
        fd = (_shape(xi + e)[0] - _shape(xi - e)[0]) / (2 * h)
        assert np.allclose(fd, dN[:, d], atol=1e-9)


def _geometry(X, q):
    import ctypes as C
    dp = C.POINTER(C.c_double)
    xi = np.zeros(3)
    oracle.lib().or_gauss_point(q, xi.ctypes.data_as(dp))
    _, dN = _shape(xi)
    X = np.ascontiguousarray(X, dtype=float)
    G = np.zeros((8, 3))
    detJ = C.c_double()
    st = oracle.lib().or_geometry(X.ctypes.data_as(dp), np.ascontiguousarray(dN).ctypes.data_as(dp),
                                  G.ctypes.data_as(dp), C.byref(detJ))
    return st, G, detJ.value, xi


def _distorted_element(seed=3):
    g = np.random.default_rng(seed)
    return 0.5 * (NODE_XI + 1.0) * np.array([0.7, 1.1, 0.9]) + g.uniform(-0.12, 0.12, (8, 3))


def test_gauss_points_and_gradient_invariants():
    g = 1.0 / math.sqrt(3.0)
    X = _distorted_element()
    vol = 0.0
    for q in range(8):
        st, G, detJ, xi = _geometry(X, q)
        assert st == 0
        assert np.allclose(np.abs(xi), g) and (xi[0] > 0) == bool(q & 1) and (xi[2] > 0) == bool(q & 4)
        # a linear field is reproduced exactly: sum_a X_a (x) G_a = I and sum_a G_a = 0
        assert np.allclose(X.T @ G, np.eye(3), atol=1e-13)
        assert np.allclose(G.sum(axis=0), 0.0, atol=1e-13)
        vol += detJ
    # affine element (parallelepiped): sum_q w detJ = |det A| exactly
    A = np.array([[0.9, 0.2, 0.1], [0.05, 1.2, -0.1], [0.0, 0.3, 0.8]])
    Xa = 0.5 * (NODE_XI + 1.0) @ A.T
    assert abs(sum(_geometry(Xa, q)[2] for q in range(8)) - np.linalg.det(A)) < 1e-14


def test_inverted_element_is_rejected():
    X = 0.5 * (NODE_XI + 1.0)
    X[[0, 1]] = X[[1, 0]]  # swap two nodes -> inverted
    with pytest.raises(oracle.OracleError):
        oracle.element(LE, 1.0, 1.0, X, np.zeros(24))


# ---------------------------------------------------------------- constitutive closed forms
def test_lame_constants():
    lam, mu = oracle.lame(3.5e9, 0.35)
    assert abs(lam - 3.0247e9) / 3.0247e9 < 1e-4 and abs(mu - 1.2963e9) / 1.2963e9 < 1e-4
    for E, nu in ((3.5e9, 0.35), (70e9, 0.22), (1e10, 0.3)):
        lam, mu = oracle.lame(E, nu)
        assert abs(mu * (3 * lam + 2 * mu) / (lam + mu) - E) / E < 1e-14
        assert abs(lam / (2 * (lam + mu)) - nu) < 1e-14


def test_uniaxial_strain_closed_forms():
    lam, mu = 2.0e9, 1.5e9
    e = 0.013
    H = np.zeros((3, 3)); H[0, 0] = e
    sig, D = oracle.linear_elastic(lam, mu, H)
    assert np.allclose(np.diag(sig), [(lam + 2 * mu) * e, lam * e, lam * e], rtol=1e-15)
    assert np.allclose(sig - np.diag(np.diag(sig)), 0.0)
    # neo-Hookean uniaxial stretch F = diag(1+e, 1, 1)
    F = np.diag([1.0 + e, 1.0, 1.0])
    S, CC = oracle.neo_hookean(lam, mu, F)
    S11 = mu * (1 - (1 + e) ** -2) + lam * math.log(1 + e) * (1 + e) ** -2
    S22 = lam * math.log(1 + e)
    assert np.allclose(np.diag(S), [S11, S22, S22], rtol=1e-13)
    assert np.allclose(S - np.diag(np.diag(S)), 0.0, atol=1e-6)
    # at F = I the neo-Hookean tangent equals the Hooke tensor
    S0, CC0 = oracle.neo_hookean(lam, mu, np.eye(3))
    assert np.allclose(S0, 0.0)
    assert np.allclose(CC0, D, rtol=1e-15)


def test_neo_hookean_tangent_is_stress_derivative():
    """CC_IJKL = 2 dS_IJ/dC_KL, checked by central differences in F along F dF."""
    lam, mu = 3.0e9, 1.3e9
    g = np.random.default_rng(7)
    F = np.eye(3) + g.uniform(-0.05, 0.05, (3, 3))
    S, CC = oracle.neo_hookean(lam, mu, F)
    dF = g.uniform(-1, 1, (3, 3))
    h = 1e-6
    Sp, _ = oracle.neo_hookean(lam, mu, F + h * dF)
    Sm, _ = oracle.neo_hookean(lam, mu, F - h * dF)
    dE = 0.5 * (dF.T @ F + F.T @ dF)
    pred = np.einsum("IJKL,KL->IJ", CC, dE)
    assert rel((Sp - Sm) / (2 * h), pred) < 1e-7
    # major and minor symmetries
    assert np.allclose(CC, CC.transpose(2, 3, 0, 1)) and np.allclose(CC, CC.transpose(1, 0, 2, 3))


# ---------------------------------------------------------------- element level
@pytest.mark.parametrize("law", [LE, NH])
def test_element_tangent_equals_fd_of_element_residual(law):
    X = _distorted_element(11)
    g = np.random.default_rng(5)
    ue = g.uniform(-0.02, 0.02, 24)
    lam, mu = 3.0e9, 1.3e9
    Re, Ke = oracle.element(law, lam, mu, X, ue)
    h = 1e-7
    fd = np.zeros((24, 24))
    for c in range(24):
        d = np.zeros(24); d[c] = h
        fd[:, c] = (oracle.element(law, lam, mu, X, ue + d, False)
                    - oracle.element(law, lam, mu, X, ue - d, False)) / (2 * h)
    assert rel(fd, Ke) < 1e-7
    assert rel(Ke, Ke.T) < 1e-14


def test_linear_elastic_unit_cube_element_is_linear():
    X = 0.5 * (NODE_XI + 1.0)
    g = np.random.default_rng(2)
    ue = g.uniform(-1e-3, 1e-3, 24)
    Re, Ke = oracle.element(LE, 2.0, 1.0, X, ue)
    assert rel(Ke @ ue, Re) < 1e-14


# ---------------------------------------------------------------- assembled problem pins
def _mesh(n=(3, 2, 4), law=NH, distort=0.2, seed=1, two_phase=True):
    coords, conn = I.box_mesh(*n, distort=distort, seed=seed)
    phase = (np.arange(len(conn)) % 3 == 0).astype(np.int32) if two_phase else np.zeros(len(conn), np.int32)
    mats = [(3.5e9, 0.35, law), (70e9, 0.22, law)]
    return oracle.Mesh(coords, conn, phase, mats), coords, conn


def _interior_nodes(coords):
    c = coords
    return np.where((c > 1e-12).all(1) & (c < 1 - 1e-12).all(1))[0]


@pytest.mark.parametrize("law", [LE, NH])
def test_patch_test_homogeneous_deformation(law):
    """u = A X + b on a distorted single-phase mesh: every interior nodal residual vanishes
    and the reaction on the face X1 = 1 equals the closed-form traction P e1 (unit area)."""
    M, coords, conn = _mesh(n=(3, 3, 3), law=law, distort=0.25, two_phase=False)
    A = np.array([[0.004, 0.001, -0.002], [0.0005, -0.003, 0.001], [0.002, 0.0, 0.0025]])
    u = (coords @ A.T + np.array([1e-3, -2e-3, 5e-4])).ravel()
    R = oracle.residual(M, u)
    lam, mu = oracle.lame(3.5e9, 0.35)
    if law == LE:
        P = oracle.linear_elastic(lam, mu, A)[0]
    else:
        F = np.eye(3) + A
        P = F @ oracle.neo_hookean(lam, mu, F)[0]
    inner = _interior_nodes(coords)
    Rn = R.reshape(-1, 3)
    assert np.max(np.abs(Rn[inner])) < 1e-12 * np.max(np.abs(Rn))
    face = np.where(np.abs(coords[:, 0] - 1.0) < 1e-12)[0]
    assert rel(Rn[face].sum(axis=0), P[:, 0]) < 1e-12


@pytest.mark.parametrize("law", [LE, NH])
def test_residual_is_energy_gradient(law):
    M, coords, _ = _mesh(law=law)
    g = np.random.default_rng(3)
    u = g.uniform(-2e-3, 2e-3, 3 * len(coords))
    R = oracle.residual(M, u)
    h = 1e-7
    for c in g.choice(len(u), 12, replace=False):
        d = np.zeros_like(u); d[c] = h
        fd = (oracle.energy(M, u + d) - oracle.energy(M, u - d)) / (2 * h)
        assert abs(fd - R[c]) < 2e-6 * np.max(np.abs(R))


@pytest.mark.parametrize("law", [LE, NH])
def test_tangent_symmetry_and_fd_of_residual(law):
    M, coords, conn = _mesh(law=law)
    g = np.random.default_rng(4)
    u = g.uniform(-2e-3, 2e-3, 3 * len(coords))
    v = g.uniform(-1, 1, 3 * len(coords))
    rp, col = oracle.csr_pattern(conn, len(coords))
    vals, R = oracle.tangent_csr(M, u, rp, col)
    K = np.zeros((M.n_dof, M.n_dof))
    for r in range(M.n_dof):
        K[r, col[rp[r]:rp[r + 1]]] = vals[rp[r]:rp[r + 1]]
    assert rel(K, K.T) < 1e-14
    assert rel(R, oracle.residual(M, u)) < 1e-15
    h = 1e-6 * np.max(np.abs(u)) / np.max(np.abs(v))
    fd = (oracle.residual(M, u + h * v) - oracle.residual(M, u - h * v)) / (2 * h)
    assert rel(fd, K @ v) < 1e-7
    assert rel(oracle.apply_tangent(M, u, v), K @ v) < 1e-14
    assert rel(oracle.spmv(rp, col, vals, v), K @ v) < 1e-14


def test_csr_pattern_counts_and_dense_assembly():
    nx, ny, nz = 3, 2, 4
    M, coords, conn = _mesh(n=(nx, ny, nz))
    rp, col = oracle.csr_pattern(conn, len(coords))
    assert rp[-1] == 9 * (3 * nx + 1) * (3 * ny + 1) * (3 * nz + 1)
    for r in range(0, M.n_dof, 7):
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)
    # values equal a dense assembly of the element matrices
    g = np.random.default_rng(9)
    u = g.uniform(-1e-3, 1e-3, M.n_dof)
    vals = oracle.tangent_csr(M, u, rp, col, with_residual=False)
    K = np.zeros((M.n_dof, M.n_dof))
    for e in range(M.n_elem):
        _, Ke = oracle.element_of(M, e, u)
        d = (3 * conn[e].astype(np.int64)[:, None] + np.arange(3)).ravel()
        K[np.ix_(d, d)] += Ke
    Kc = np.zeros_like(K)
    for r in range(M.n_dof):
        Kc[r, col[rp[r]:rp[r + 1]]] = vals[rp[r]:rp[r + 1]]
    assert rel(Kc, K) < 1e-15
    assert np.count_nonzero(K) <= rp[-1]


def _rigid_modes(coords):
    modes = []
    for i in range(3):
        t = np.zeros_like(coords); t[:, i] = 1.0
        modes.append(t.ravel())
    for W in (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0]]),
              np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0]])):
        modes.append((coords @ W.T).ravel())
    return modes, None


@pytest.mark.parametrize("law", [LE, NH])
def test_rigid_body_modes_at_rest(law):
    M, coords, _ = _mesh(law=law)
    u0 = np.zeros(M.n_dof)
    modes, _ = _rigid_modes(coords)
    scale = None
    for r in modes:
        y = oracle.apply_tangent(M, u0, r)
        if scale is None:
            scale = np.max(np.abs(oracle.apply_tangent(M, u0, np.random.default_rng(0).uniform(-1, 1, M.n_dof))))
        assert np.max(np.abs(y)) < 1e-13 * scale


def test_neo_hookean_objectivity_identity_at_stressed_state():
    """R(Q phi) = Q R(phi) for rotations Q; differentiating at Q = I along a skew W gives
    K (W phi) = W R for every node (phi = X + u), and translations are null vectors."""
    M, coords, _ = _mesh(law=NH)
    g = np.random.default_rng(12)
    u = g.uniform(-3e-3, 3e-3, M.n_dof)
    R = oracle.residual(M, u).reshape(-1, 3)
    phi = coords + u.reshape(-1, 3)
    scale = np.max(np.abs(oracle.apply_tangent(M, u, g.uniform(-1, 1, M.n_dof))))
    for W in (np.array([[0, -1, 0], [1, 0, 0], [0, 0, 0.]]), np.array([[0, 0, 1], [0, 0, 0], [-1, 0, 0.]]),
              np.array([[0, 0, 0], [0, 0, -1], [0, 1, 0.]])):
        y = oracle.apply_tangent(M, u, (phi @ W.T).ravel()).reshape(-1, 3)
        assert np.max(np.abs(y - R @ W.T)) < 1e-12 * scale
    for i in range(3):
        t = np.zeros_like(coords); t[:, i] = 1
        assert np.max(np.abs(oracle.apply_tangent(M, u, t.ravel()))) < 1e-13 * scale


def test_material_gradient_central_differences_exact():
    """L = 1/2 ||R||^2 is quadratic in each E_e (R is linear in E_e), so central differences
    are exact up to rounding."""
    coords, conn = I.box_mesh(4, distort=0.2, seed=2)
    g = np.random.default_rng(21)
    E = 1e10 * np.exp(0.5 * g.standard_normal(len(conn)))
    u = g.uniform(-1e-3, 1e-3, coords.size)
    phase = np.zeros(len(conn), np.int32)
    for law in (LE, NH):
        M = oracle.Mesh(coords, conn, phase, [(1e10, 0.3, law)], E)
        gr = oracle.material_grad(M, u)
        for e in g.choice(len(conn), 6, replace=False):
            h = 1e-6 * E[e]
            Ep, Em = E.copy(), E.copy()
            Ep[e] += h; Em[e] -= h
            Lp = 0.5 * np.sum(oracle.residual(oracle.Mesh(coords, conn, phase, [(1e10, 0.3, law)], Ep), u) ** 2)
            Lm = 0.5 * np.sum(oracle.residual(oracle.Mesh(coords, conn, phase, [(1e10, 0.3, law)], Em), u) ** 2)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - gr[e]) < 1e-6 * max(abs(gr[e]), 1e-3 * np.max(np.abs(gr)))


def test_sampled_rows_match_full_assembly():
    M, coords, conn = _mesh(n=(3, 3, 2))
    g = np.random.default_rng(8)
    u = g.uniform(-1e-3, 1e-3, M.n_dof)
    v = g.uniform(-1, 1, M.n_dof)
    rp, col = oracle.csr_pattern(conn, len(coords))
    vals, R = oracle.tangent_csr(M, u, rp, col)
    y = oracle.apply_tangent(M, u, v)
    nodes = [0, 5, 17, len(coords) - 1]
    rows = oracle.sampled_rows(M, u, v, nodes)
    for n in nodes:
        Rn, Kvn, krow = rows[n]
        assert rel(Rn, R[3 * n:3 * n + 3]) < 1e-14
        assert rel(Kvn, y[3 * n:3 * n + 3]) < 1e-13
        for i in range(3):
            r = 3 * n + i
            cs = col[rp[r]:rp[r + 1]]
            assert sorted(krow) == list(cs)
            assert rel([krow[c][i] for c in cs], vals[rp[r]:rp[r + 1]]) < 1e-14


# ---------------------------------------------------------------- MLP surrogate oracle
def _tiny_layers(seed=0):
    layers = I.mlp_init(seed)
    g = np.random.default_rng(seed)
    return [(W, g.uniform(-0.1, 0.1, b.shape)) for W, b in layers]


def test_silu_values():
    assert mlp.silu(np.array(0.0)) == 0.0 and mlp.silu_prime(np.array(0.0)) == 0.5
    z = np.array([-3.0, -0.4, 0.7, 2.5])
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)), rtol=1e-15)
    h = 1e-6
    assert np.allclose((mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), mlp.silu_prime(z), atol=1e-9)


def test_mlp_weight_gradients_fd():
    layers = _tiny_layers(1)
    g = np.random.default_rng(2)
    x = g.uniform(-1, 1, (16, 8))
    t = g.uniform(-1, 1, (16, 6))
    loss, grads = mlp.gradients(layers, x, t)
    h = 1e-6
    for li in range(4):
        W, b = layers[li]
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (2, 3)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h; Wm[i, j] -= h
            lp = mlp.mse(mlp.forward(layers[:li] + [(Wp, b)] + layers[li + 1:], x), t)
            lm = mlp.mse(mlp.forward(layers[:li] + [(Wm, b)] + layers[li + 1:], x), t)
            assert abs((lp - lm) / (2 * h) - grads[li][0][i, j]) < 1e-8
        bp, bm = b.copy(), b.copy()
        bp[1] += h; bm[1] -= h
        lp = mlp.mse(mlp.forward(layers[:li] + [(W, bp)] + layers[li + 1:], x), t)
        lm = mlp.mse(mlp.forward(layers[:li] + [(W, bm)] + layers[li + 1:], x), t)
        assert abs((lp - lm) / (2 * h) - grads[li][1][1]) < 1e-8


def test_mlp_input_jacobian_fd():
    layers = _tiny_layers(3)
    g = np.random.default_rng(4)
    x = g.uniform(-1, 1, (5, 8))
    Jm = mlp.input_jacobian(layers, x)
    h = 1e-6
    for c in range(6):
        d = np.zeros(8); d[c] = h
        fd = (mlp.forward(layers, x + d) - mlp.forward(layers, x - d)) / (2 * h)
        assert np.allclose(fd, Jm[:, :, c], atol=1e-8)


def test_adam_first_step_closed_form():
    """With zero moments, bias-corrected Adam's first step is lr * g / (|g| + eps)."""
    layers = _tiny_layers(5)
    g = np.random.default_rng(6)
    grads = [(g.standard_normal(W.shape), g.standard_normal(b.shape)) for W, b in layers]
    opt = mlp.Adam(layers)
    new = opt.step(layers, grads, 1e-3)
    for (W, b), (gW, gb), (W2, b2) in zip(layers, grads, new):
        assert np.allclose(W - W2, 1e-3 * gW / (np.abs(gW) + 1e-8), rtol=1e-12, atol=1e-18)
        assert np.allclose(b - b2, 1e-3 * gb / (np.abs(gb) + 1e-8), rtol=1e-12, atol=1e-18)


def test_surrogate_tangent_scaling():
    layers = _tiny_layers(7)
    g = np.random.default_rng(8)
    E6 = g.uniform(-0.05, 0.05, (4, 6))
    ph = np.array([0, 1, 1, 0])
    sc = np.array([[2.0] * 6, [30.0] * 6]); sh = np.zeros((2, 6))
    S, D = mlp.surrogate_stress(layers, E6, ph, 0.05, sc, sh)
    h = 1e-7
    for c in range(6):
        d = np.zeros(6); d[c] = h
        fd = (mlp.surrogate_stress(layers, E6 + d, ph, 0.05, sc, sh)[0]
              - mlp.surrogate_stress(layers, E6 - d, ph, 0.05, sc, sh)[0]) / (2 * h)
        assert np.allclose(fd, D[:, :, c], rtol=1e-6, atol=1e-6)


def test_surrogate_oracle_tangent_is_fd_of_its_residual():
    from oracle import surrogate_fem
    coords, conn = I.box_mesh(2, 2, 1, distort=0.2, seed=4)
    g = np.random.default_rng(4)
    phase = np.array([0, 1, 1, 0], np.int32)
    M = oracle.Mesh(coords, conn, phase, I.composite_materials(NH))
    layers = _tiny_layers(9)
    sc = np.array([[2e8] * 6, [3e9] * 6]); sh = np.zeros((2, 6))
    u = g.uniform(-3e-3, 3e-3, coords.size)
    K, R, fb, _ = surrogate_fem.assemble(M, u, layers, 0.05, 0.05, sc, sh)
    assert fb == 0
    v = g.uniform(-1, 1, coords.size)
    h = 1e-7
    Rp = surrogate_fem.assemble(M, u + h * v, layers, 0.05, 0.05, sc, sh)[1]
    Rm = surrogate_fem.assemble(M, u - h * v, layers, 0.05, 0.05, sc, sh)[1]
    assert rel((Rp - Rm) / (2 * h), K @ v) < 1e-6
    # all points out of range: the plain neo-Hookean oracle
    K0, R0, fb0, _ = surrogate_fem.assemble(M, u, layers, 0.05, 1e-12, sc, sh)
    assert fb0 == 8 * len(conn)
    rp, col = oracle.csr_pattern(conn, len(coords))
    vals, Rref = oracle.tangent_csr(M, u, rp, col)
    Kref = np.zeros_like(K0)
    for r in range(len(Kref)):
        Kref[r, col[rp[r]:rp[r + 1]]] = vals[rp[r]:rp[r + 1]]
    assert rel(R0, Rref) < 1e-13 and rel(K0, Kref) < 1e-13


def test_surrogate_oracle_sampled_rows_equal_its_dense_assembly():
    """The element-by-element rows at sampled nodes (used at sizes the dense assembly cannot
    reach) are the rows of the dense assembly exactly, on a distorted two-phase box; the
    strains and phases returned are those of the elements around the sampled nodes."""
    from oracle import surrogate_fem
    coords, conn = I.box_mesh(3, 2, 2, distort=0.2, seed=6)
    g = np.random.default_rng(6)
    phase = (g.uniform(size=len(conn)) < 0.5).astype(np.int32)
    M = oracle.Mesh(coords, conn, phase, I.composite_materials(NH))
    layers = _tiny_layers(11)
    sc = np.array([[2e8] * 6, [3e9] * 6]); sh = np.zeros((2, 6))
    u = g.uniform(-3e-3, 3e-3, coords.size)
    K, R, fb, E6 = surrogate_fem.assemble(M, u, layers, 0.05, 0.05, sc, sh)
    nodes = np.array([0, 5, len(coords) - 1])
    rows, E6s, phs = surrogate_fem.sampled_rows(M, u, nodes, layers, 0.05, 0.05, sc, sh)
    for n in nodes:
        Rn, krow = rows[int(n)]
        assert np.array_equal(Rn, R[3 * n:3 * n + 3])
        assert set(krow) == set(np.nonzero(np.any(K[3 * n:3 * n + 3] != 0, axis=0))[0])
        for c, col in krow.items():
            assert np.array_equal(col, K[3 * n:3 * n + 3, c])
    ptr, eidx = oracle.node_elements(conn, len(coords))
    around = sorted({int(e) for n in nodes for e in eidx[ptr[n]:ptr[n + 1]]})
    assert E6s.shape == (8 * len(around), 6) and phs.shape == (8 * len(around),)
    assert set(phs.tolist()) <= {0, 1}
