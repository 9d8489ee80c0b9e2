"""Residual and tangent with the MLP surrogate fused into the element kernel, against the
FP64 oracle (FP64 network and element arithmetic, same weights).

Tolerances: the network's BF16 error bound (first-order propagation of the u = 2^-9
roundings, computed from the oracle's forward pass as in test_gpu_surrogate.py) relative to
the largest stress / tangent entry, times 4 for the assembly sums, plus the FP32 element
arithmetic bound 2e-4 used for the FP32 path.  Gauss points whose strain lies within 1e-5
of the range boundary could be decided differently in FP32 and FP64; the test inputs keep
every point away from that band and the test asserts it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp, surrogate_fem
from paper_2604_22087_b300 import inputs as I

from test_gpu_surrogate import config, forward_bound, jacobian_bound

pytestmark = pytest.mark.gpu


def J():
    from paper_2604_22087_b300 import jetsci
    return jetsci


def _problem(seed=3):
    coords, conn = I.box_mesh(4, 3, 3, distort=0.2, seed=seed)
    g = np.random.default_rng(seed)
    phase = (g.uniform(size=len(conn)) < 0.5).astype(np.int32)
    u = g.uniform(-4e-3, 4e-3, coords.size) + np.repeat(coords[:, 0] * 0.01, 3) * np.tile([1, 0, 0], len(coords))
    return I.Problem("surrogate_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN), u,
                     g.uniform(-1, 1, coords.size))


def _csr_to_dense(rp, col, vals, n):
    K = np.zeros((n, n))
    for r in range(n):
        K[r, col[rp[r]:rp[r + 1]]] = vals[rp[r]:rp[r + 1]]
    return K


def _run(prob, layers_seed, rng):
    cfg = config()
    cfg["range_"] = rng
    g = np.random.default_rng(layers_seed)
    s = J().Surrogate([(W, g.uniform(-0.1, 0.1, b.shape)) for W, b in I.mlp_init(layers_seed)], **cfg)
    mesh = J().Mesh.of(prob)
    J().attach_surrogate(mesh, s)
    u = torch.as_tensor(prob.u).cuda()
    R = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R, precision=J().SURROGATE)
    R2 = mesh.residual(u, precision=J().SURROGATE)
    nfb = J().surrogate_fallbacks(mesh)
    assert mesh.check() == 0
    rp, col = mesh.pattern()
    Kg = _csr_to_dense(rp.cpu().numpy(), col.cpu().numpy(), vals.cpu().numpy().astype(np.float64), mesh.n_dof)
    layers = s.layers()
    om = oracle.Mesh.of(prob)
    K, Rref, fb, E6 = surrogate_fem.assemble(om, prob.u, layers, cfg["in_scale"], rng, cfg["out_scale"],
                                             cfg["out_shift"])
    return dict(Kg=Kg, Rg=R.cpu().numpy(), R2=R2.cpu().numpy(), nfb=nfb, K=K, R=Rref, fb=fb, E6=E6,
                layers=layers, cfg=cfg)


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_surrogate_tangent_and_residual_vs_oracle():
    prob = _problem()
    r = _run(prob, 4, 0.05)
    # every point inside the range and away from its boundary
    assert np.max(np.abs(r["E6"])) < 0.05 - 1e-5
    assert r["nfb"] == 0 and r["fb"] == 0
    cfg = r["cfg"]
    ph = np.repeat(prob.phase, 8)
    x = mlp.surrogate_inputs(r["E6"], ph, cfg["in_scale"])
    sc = cfg["out_scale"][ph]
    y = mlp.forward(r["layers"], x)
    tol_S = 4 * np.max(2 * forward_bound(r["layers"], x) * sc) / np.max(np.abs(y * sc)) + 2e-4
    Jm = mlp.input_jacobian(r["layers"], x)
    tol_D = 4 * np.max(2 * jacobian_bound(r["layers"], x) * sc[:, :, None]) / np.max(np.abs(Jm * sc[:, :, None])) + 2e-4
    assert rel(r["Rg"], r["R"]) <= tol_S, (rel(r["Rg"], r["R"]), tol_S)
    assert np.array_equal(r["Rg"], r["R2"])
    assert rel(r["Kg"], r["K"]) <= tol_D, (rel(r["Kg"], r["K"]), tol_D)
    # the surrogate tangent is not symmetric in general, and the kernel keeps that
    assert np.max(np.abs(r["Kg"] - r["Kg"].T)) > 0


def test_surrogate_fallback_equals_plain_law():
    """With a tiny range every Gauss point falls back to the plain neo-Hookean law."""
    prob = _problem(5)
    r = _run(prob, 7, 1e-9)
    n_q = 8 * prob.n_elem
    assert r["nfb"] == n_q and r["fb"] == n_q
    assert rel(r["Rg"], r["R"]) <= 2e-4
    assert rel(r["Kg"], r["K"]) <= 5e-5 * 4
    om = oracle.Mesh.of(prob)
    assert rel(r["R"], oracle.residual(om, prob.u)) <= 1e-13


def test_full_size_surrogate_sampled_rows():
    """The 128^3 fibre RVE through the fused surrogate tangent in the bench's launch
    configuration: rows of R and of the CSR values at sampled nodes against the oracle's
    surrogate element routine (summed element by element), within the small case's bounds
    computed from the Gauss points of the sampled elements."""
    prob = I.fibre_composite(128, seed=2)
    cfg = config()
    g = np.random.default_rng(4)
    s = J().Surrogate([(W, g.uniform(-0.1, 0.1, b.shape)) for W, b in I.mlp_init(4)], **cfg)
    mesh = J().Mesh.of(prob)
    J().attach_surrogate(mesh, s)
    u = torch.as_tensor(prob.u).cuda()
    R = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R, precision=J().SURROGATE)
    assert J().surrogate_fallbacks(mesh) == 0 and mesh.check() == 0
    rp, col = mesh.pattern(device="cpu")
    rp, col = rp.numpy(), col.numpy()
    Rg, vg = R.cpu().numpy(), vals.cpu().numpy().astype(np.float64)
    layers = s.layers()
    om = oracle.Mesh.of(prob)
    nodes = np.concatenate([[0, prob.n_nodes - 1], np.random.default_rng(0).choice(prob.n_nodes, 10, replace=False)])
    rows, E6, ph = surrogate_fem.sampled_rows(om, prob.u, nodes, layers, cfg["in_scale"], cfg["range_"],
                                              cfg["out_scale"], cfg["out_shift"])
    assert np.max(np.abs(E6)) < cfg["range_"] - 1e-5
    x = mlp.surrogate_inputs(E6, ph, cfg["in_scale"])
    sc = cfg["out_scale"][ph]
    y = mlp.forward(layers, x)
    tol_S = 4 * np.max(2 * forward_bound(layers, x) * sc) / np.max(np.abs(y * sc)) + 2e-4
    Jm = mlp.input_jacobian(layers, x)
    tol_D = 4 * np.max(2 * jacobian_bound(layers, x) * sc[:, :, None]) / np.max(np.abs(Jm * sc[:, :, None])) + 2e-4
    eR = sR = eK = sK = 0.0
    for n in nodes:
        n = int(n)
        Rn, krow = rows[n]
        eR, sR = max(eR, np.max(np.abs(Rg[3 * n:3 * n + 3] - Rn))), max(sR, np.max(np.abs(Rn)))
        for i in range(3):
            r = 3 * n + i
            cs = col[rp[r]:rp[r + 1]]
            kref = np.array([krow[c][i] for c in cs])
            eK, sK = max(eK, np.max(np.abs(vg[rp[r]:rp[r + 1]] - kref))), max(sK, np.max(np.abs(kref)))
    assert eR / sR <= tol_S, (eR / sR, tol_S)
    assert eK / sK <= tol_D, (eK / sK, tol_D)
    J().attach_surrogate(mesh, None)
    mesh.close()
    s.close()
