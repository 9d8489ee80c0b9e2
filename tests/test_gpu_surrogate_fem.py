"""Residual and tangent with the MLP surrogate fused into the element kernel, against the
FP64 oracle (FP64 network and element arithmetic, same weights).

Tolerances, entry by entry, derived from the arithmetic: at every Gauss point inside the
training range the network's stress and tangent carry the BF16 rounding bound of
test_gpu_surrogate.py (min(6 sigma, worst case) of the propagated roundings, per output and
direction); R and K are linear in S and in the elasticity tensor built from dS/dE, so the
point bounds propagate exactly through R_e(a,i) = sum_q w detJ (F S)_iJ G_aJ and
K_e = sum_q w detJ G (1 x S + F CC F) G with absolute values, and are summed over the points and
elements of each entry.  To that the FP32 element arithmetic adds its normwise bound 2e-4
(as for the FP32 path).  Gauss points whose strain lies within 1e-5 of the range boundary
could be decided differently in FP32 and FP64; the test inputs keep every point away from
that band and the tests assert it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp, surrogate_fem
from paper_2604_22087_b300 import inputs as I

from test_gpu_surrogate import config, output_bounds

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


def _element_bounds(om, e, u, layers, cfg, rng):
    """Absolute bounds (R_e [24], K_e [24, 24], rows and columns (a, i)) on the network part of
    the error of element e: the per-point bounds on S and dS/dE of its in-range Gauss points
    pushed through the residual and tangent definitions with absolute values."""
    en = om.conn[e].astype(np.int64)
    ue = u[(3 * en[:, None] + np.arange(3))].reshape(8, 3)
    geo = surrogate_fem._geometry(om.coords[en])
    Fs = [np.eye(3) + ue.T @ G for G, _ in geo]
    E6 = np.array([[(0.5 * (F.T @ F - np.eye(3)))[i, j] for i, j in surrogate_fem.VOIGT] for F in Fs])
    inside = np.all(np.abs(E6) <= rng, axis=1)
    bR, bK = np.zeros(24), np.zeros((24, 24))
    if not inside.any():
        return bR, bK
    ph = np.full(8, int(om.phase[e]))
    by, bJ = output_bounds(layers, mlp.surrogate_inputs(E6, ph, cfg["in_scale"]))
    sc = cfg["out_scale"][ph]
    dS, dD = by * sc, bJ * sc[:, :, None] / cfg["in_scale"]
    for q, ((G, detJ), F) in enumerate(zip(geo, Fs)):
        if not inside[q]:
            continue
        aS = np.abs(surrogate_fem._tensor(dS[q]))
        aC = np.zeros((3, 3, 3, 3))
        for a, (I_, J_) in enumerate(surrogate_fem.VOIGT):
            for b, (K_, L_) in enumerate(surrogate_fem.VOIGT):
                v = dD[q, a, b] if K_ == L_ else 0.5 * dD[q, a, b]
                for (i1, j1) in {(I_, J_), (J_, I_)}:
                    for (k1, l1) in {(K_, L_), (L_, K_)}:
                        aC[i1, j1, k1, l1] = v
        aF, aG = np.abs(F), np.abs(G)
        bR += detJ * ((aF @ aS) @ aG.T).T.ravel()
        A = np.einsum("ik,JL->iJkL", np.eye(3), aS) + np.einsum("iI,IJKL,kK->iJkL", aF, aC, aF)
        bK += detJ * np.einsum("aJ,iJkL,bL->aibk", aG, A, aG).reshape(24, 24)
    return bR, bK


def _assembled_bounds(om, u, layers, cfg, rng):
    """The element bounds summed into the global residual and the dense matrix."""
    bR, bK = np.zeros(om.n_dof), np.zeros((om.n_dof, om.n_dof))
    for e in range(om.n_elem):
        r, k = _element_bounds(om, e, u, layers, cfg, rng)
        d = (3 * om.conn[e].astype(np.int64)[:, None] + np.arange(3)).ravel()
        bR[d] += r
        bK[np.ix_(d, d)] += k
    return bR, bK


def _check_within(r, prob, rng):
    """Entry-wise: |GPU - oracle| <= network bound + FP32 bound; returns the bounds' largest
    share of the largest entry (to show they are informative)."""
    om = oracle.Mesh.of(prob)
    bR, bK = _assembled_bounds(om, prob.u, r["layers"], r["cfg"], rng)
    sR, sK = np.max(np.abs(r["R"])), np.max(np.abs(r["K"]))
    eR, eK = np.abs(r["Rg"] - r["R"]), np.abs(r["Kg"] - r["K"])
    assert np.all(eR <= bR + 2e-4 * sR), float(np.max(eR / (bR + 2e-4 * sR)))
    assert np.all(eK <= bK + 2e-4 * sK), float(np.max(eK / (bK + 2e-4 * sK)))
    return float(np.max(bR) / sR), float(np.max(bK) / sK)


# Regression guards, normwise, at about ten times the errors measured on B300 for these cases
# (all points in range: R 4.6e-3, K 2.3e-3; half the points falling back: R 8.3e-4, K 1.0e-4;
# all falling back: R 2.6e-6, K 1.6e-7).  The entry-wise bounds above hold with room; these catch
# a regression inside them.
GUARD = {"inrange": (5e-2, 2.5e-2), "mixed": (1e-2, 1e-3), "fallback": (3e-5, 2e-6)}


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def test_surrogate_tangent_and_residual_vs_oracle():
    prob = _problem()
    r = _run(prob, 4, 0.05)
    # every point inside the range and away from its boundary
    assert np.max(np.abs(r["E6"])) < 0.05 - 1e-5
    assert r["nfb"] == 0 and r["fb"] == 0
    share_R, share_K = _check_within(r, prob, 0.05)
    assert share_R <= 0.25 and share_K <= 0.25  # the bounds say something
    assert rel(r["Rg"], r["R"]) <= GUARD["inrange"][0] and rel(r["Kg"], r["K"]) <= GUARD["inrange"][1]
    assert np.array_equal(r["Rg"], r["R2"])
    # the surrogate tangent is not symmetric in general, and the kernel keeps that
    assert np.max(np.abs(r["Kg"] - r["Kg"].T)) > 0


def test_surrogate_fallback_equals_plain_law():
    """With a tiny range every Gauss point falls back to the plain neo-Hookean law."""
    prob = _problem(5)
    r = _run(prob, 7, 1e-9)
    n_q = 8 * prob.n_elem
    assert r["nfb"] == n_q and r["fb"] == n_q
    assert rel(r["Rg"], r["R"]) <= min(2e-4, GUARD["fallback"][0])
    assert rel(r["Kg"], r["K"]) <= min(5e-5 * 4, GUARD["fallback"][1])
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
    ptr, eidx = oracle.node_elements(prob.conn, prob.n_nodes)
    eb = {}
    sR = max(np.max(np.abs(rows[int(n)][0])) for n in nodes)
    sK = max(np.max(np.abs(list(rows[int(n)][1].values()))) for n in nodes)
    for n in nodes:
        n = int(n)
        Rn, krow = rows[n]
        bRn, bkrow = np.zeros(3), {}
        for e in eidx[ptr[n]:ptr[n + 1]]:
            e = int(e)
            if e not in eb:
                eb[e] = _element_bounds(om, e, prob.u, layers, cfg, cfg["range_"])
            en = prob.conn[e].astype(np.int64)
            a = int(np.where(en == n)[0][0])
            bRn += eb[e][0][3 * a:3 * a + 3]
            for b in range(8):
                for k in range(3):
                    c = 3 * int(en[b]) + k
                    bkrow[c] = bkrow.get(c, np.zeros(3)) + eb[e][1][3 * a:3 * a + 3, 3 * b + k]
        assert np.all(np.abs(Rg[3 * n:3 * n + 3] - Rn) <= bRn + 2e-4 * sR)
        for i in range(3):
            r = 3 * n + i
            cs = col[rp[r]:rp[r + 1]]
            kref = np.array([krow[c][i] for c in cs])
            kb = np.array([bkrow[c][i] for c in cs])
            assert np.all(np.abs(vg[rp[r]:rp[r + 1]] - kref) <= kb + 2e-4 * sK)
    J().attach_surrogate(mesh, None)
    mesh.close()
    s.close()


def _split_range(E6, band=1e-5):
    """A strain range that splits the Gauss points near the median of max_ij |E_ij|, at the
    midpoint of a gap of at least 2 * band between consecutive point maxima, so that no point
    lies within `band` of it (FP32 and FP64 then take the same in/out decision)."""
    m = np.sort(np.max(np.abs(E6), axis=1))
    n = len(m)
    for d in range(n // 2):
        for k in (n // 2 - d, n // 2 + d):
            if 0 < k < n and m[k] - m[k - 1] >= 2 * band:
                return 0.5 * (m[k] + m[k - 1])
    raise AssertionError("no gap in the strain maxima")


def test_surrogate_mixed_in_range_and_fallback_points():
    """Gauss points inside and outside the training range in the same elements and in the same
    128-point tensor-core tiles: the in-range points take S and dS/dE from the network, the
    others from the plain neo-Hookean law, point by point (the fallback of the surrogate
    model, Section III-B's remark on learned material laws).  The range is set at a gap in
    the points' strain maxima near their median, so about half the points fall back, none
    within 1e-5 of the boundary.  R and K against the oracle's surrogate element routine
    (the same per-point choice in FP64), and the fallback count equal to the oracle's."""
    prob = _problem(11)
    om = oracle.Mesh.of(prob)
    cfg0 = config()
    E6 = np.concatenate([surrogate_fem.element(om, e, prob.u, [(W, b) for W, b in I.mlp_init(4)], cfg0["in_scale"],
                                               1.0, cfg0["out_scale"], cfg0["out_shift"])[3]
                         for e in range(prob.n_elem)])
    rng = _split_range(E6)
    r = _run(prob, 4, rng)
    n_q = 8 * prob.n_elem
    inside = np.all(np.abs(r["E6"]) <= rng, axis=1)
    assert np.min(np.abs(np.max(np.abs(r["E6"]), axis=1) - rng)) >= 1e-5
    assert 0 < r["nfb"] < n_q and r["nfb"] == r["fb"] == int(np.sum(~inside))
    per_elem = inside.reshape(prob.n_elem, 8).sum(axis=1)
    assert np.sum((per_elem > 0) & (per_elem < 8)) >= prob.n_elem // 4  # mixed elements
    # the 128-point tiles (16 elements each) hold both kinds
    for t0 in range(0, n_q - 127, 128):
        assert 0 < np.sum(inside[t0:t0 + 128]) < 128
    share_R, share_K = _check_within(r, prob, rng)
    assert share_R <= 0.25 and share_K <= 0.25
    assert rel(r["Rg"], r["R"]) <= GUARD["mixed"][0] and rel(r["Kg"], r["K"]) <= GUARD["mixed"][1]
    assert np.array_equal(r["Rg"], r["R2"])
    # the plain law alone at the same state is far from the mixed result (both kinds matter)
    om_R = oracle.residual(om, prob.u)
    assert rel(r["R"], om_R) > 10 * (share_R + 2e-4)


def test_trained_surrogate_in_the_element_kernel():
    """The network trained on neo-Hookean labels by the library's own kernels (2^16 samples,
    20 epochs), fused into the element kernel on the 16^3 sphere RVE at a 1% stretch: R and K
    against the oracle's surrogate element routine with the trained weights (entry-wise
    bounds as above), and against the plain neo-Hookean oracle within the error the training
    left (its largest stress error on held-out strains, pushed through the residual definition
    with absolute values): the learned law stands in for the plain one in the assembled system,
    not only point by point."""
    n = 1 << 16
    E6s, phs = I.strain_samples(n, seed=5)
    E6d, phd = torch.as_tensor(E6s).cuda(), torch.as_tensor(phs).cuda()
    mats = I.composite_materials(I.LAW_NEO_HOOKEAN)
    Sd = J().Surrogate.label(mats, E6d, phd)
    cfg = config()
    s = J().Surrogate(I.mlp_init(5), **cfg)
    epochs, batch = 20, 2048
    order = torch.as_tensor(I.minibatch_order(n, epochs, seed=5)).cuda()
    s.train(E6d, phd, Sd, order, n_steps=epochs * (n // batch), batch=batch, lr_max=3e-3, lr_min=1e-5)
    prob = I.sphere_composite(16, seed=1, law=I.LAW_NEO_HOOKEAN)
    prob.u = I.uniform_field(prob.coords.size, 1e-3, 11) + np.repeat(prob.coords[:, :1] * 0.01, 3, 1).ravel() * \
        np.tile([1.0, 0.0, 0.0], prob.n_nodes)
    mesh = J().Mesh.of(prob)
    J().attach_surrogate(mesh, s)
    u = torch.as_tensor(prob.u).cuda()
    R = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R, precision=J().SURROGATE)
    assert J().surrogate_fallbacks(mesh) == 0 and mesh.check() == 0
    rp, col = mesh.pattern()
    Kg = _csr_to_dense(rp.cpu().numpy(), col.cpu().numpy(), vals.cpu().numpy().astype(np.float64), mesh.n_dof)
    layers = s.layers()
    om = oracle.Mesh.of(prob)
    K, Rref, fb, E6 = surrogate_fem.assemble(om, prob.u, layers, cfg["in_scale"], cfg["range_"], cfg["out_scale"],
                                             cfg["out_shift"])
    assert fb == 0 and np.max(np.abs(E6)) < cfg["range_"] - 1e-5
    r = dict(Kg=Kg, Rg=R.cpu().numpy(), K=K, R=Rref, layers=layers, cfg=cfg)
    share_R, share_K = _check_within(r, prob, cfg["range_"])
    assert share_R <= 0.25 and share_K <= 0.25
    # the trained network against the plain law: held-out stress error, then the assembled system
    Et, pt = I.strain_samples(4096, seed=99)
    S_true = J().Surrogate.label(mats, torch.as_tensor(Et).cuda(), torch.as_tensor(pt).cuda()).cpu().numpy()
    S_net = s.eval(torch.as_tensor(Et).cuda(), torch.as_tensor(pt).cuda(), tangent=False).cpu().numpy()
    # largest stress error of the trained network over held-out strains of the training box,
    # per phase (absolute, Pa); twice that bounds it at the RVE's strains, which lie in the box
    dS = [2.0 * float(np.max(np.abs(S_net - S_true)[pt == p])) for p in (0, 1)]
    # pushed through R_e(a,i) = sum_q w detJ (F S)_iJ G_aJ with absolute values: |dR_ai| <= dS
    # sum_q detJ sum_IJ |F_iI| |G_aJ|, summed over the elements of each DOF
    bR = np.zeros(om.n_dof)
    for e in range(om.n_elem):
        en = om.conn[e].astype(np.int64)
        ue = prob.u[(3 * en[:, None] + np.arange(3))].reshape(8, 3)
        w = np.zeros(24)
        for G, detJ in surrogate_fem._geometry(om.coords[en]):
            F = np.eye(3) + ue.T @ G
            w += detJ * (np.abs(F).sum(axis=1)[None, :] * np.abs(G).sum(axis=1)[:, None]).ravel()
        bR[(3 * en[:, None] + np.arange(3)).ravel()] += dS[int(om.phase[e])] * w
    R_nh = oracle.residual(om, prob.u)
    err = np.abs(r["Rg"] - R_nh)
    assert np.all(err <= bR + 2e-4 * np.max(np.abs(R_nh))), float(np.max(err / (bR + 1e-300)))
    # and it is the network's error, not the bound's looseness, that separates the two
    assert rel(r["Rg"], R_nh) > 10 * rel(r["Rg"], r["R"])
    s.close()
    J().attach_surrogate(mesh, None)
    mesh.close()
