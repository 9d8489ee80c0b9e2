"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Error metric: normwise max|x - x_ref| / max|x_ref| over the whole output (interior residual
entries cancel to near zero, so entry-wise relative error is meaningless there).
Tolerances: FP64 1e-12 (the target stated for the plain FP64 path).  FP32 element
arithmetic: unit roundoff 6e-8 times the depth of the per-Gauss-point computation
(~1e2 operations) times the cancellation between the 8 element contributions of a node
(~10) gives ~6e-5; the tests use 2e-4 for R and K.v and 5e-5 for CSR values (no
cross-element cancellation inside one entry beyond the 8-fold sum).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2604_22087_b300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12

# Regression guards at about ten times the errors measured on B300 (largest over the 16^3 sphere
# RVE linear and stretched, the ragged box and the high-valence mesh): FP32 CSR values 1.8e-7,
# R 4.4e-6, matrix-free K.v 1.4e-7, CSR K.v 1.9e-7; TF32 CSR values 6.0e-5, CSR K.v 1.0e-4
# (its R and matrix-free K.v are the FP32 ones: TF32 changes only the element stiffness, which
# the matrix-free product does not form).  The derived bounds are worst cases two orders above
# these; the guards catch a regression that would stay inside them.  At 128^3 the measured
# errors are lower still (FP32 R 1.7e-6, values 1.1e-7, K.v 9.9e-8; TF32 values 3.4e-5).
GUARD = {"FP32": dict(vals=2e-6, R=6e-5, ymf=1e-6, ycsr=2e-6),
         "TF32": dict(vals=1.2e-3, R=6e-5, ymf=1e-6, ycsr=1e-3)}


def jetsci():
    from paper_2604_22087_b300 import jetsci as J
    return J


def relerr(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def problems():
    """(id, Problem) cases: the 16^3 two-phase sphere RVE (linear elastic), the same
    geometry neo-Hookean, and a distorted ragged 5x7x3 neo-Hookean box."""
    out = []
    p = I.sphere_composite(16, seed=1, law=I.LAW_LINEAR_ELASTIC)
    out.append(("sphere16_linear", p))
    q = I.sphere_composite(16, seed=1, law=I.LAW_NEO_HOOKEAN)
    q.u = I.uniform_field(q.coords.size, 1e-3, 11) + np.repeat(q.coords[:, :1] * 0.01, 3, 1).ravel() * \
        np.tile([1.0, 0.0, 0.0], q.n_nodes)
    out.append(("sphere16_neohookean_stretch", q))
    coords, conn = I.box_mesh(5, 7, 3, distort=0.25, seed=3)
    g = np.random.default_rng(3)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    r = I.Problem("ragged_5x7x3_neohookean", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                  g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    out.append(("ragged_neohookean", r))
    return out


PROBLEMS = problems()


@pytest.fixture(scope="module", params=[p[0] for p in PROBLEMS])
def case(request):
    prob = dict(PROBLEMS)[request.param]
    J = jetsci()
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    ref = dict(R=R_ref, vals=vals_ref, rowptr=rp, col=col, y_mf=oracle.apply_tangent(om, prob.u, prob.v),
               y_csr=oracle.spmv(rp, col, vals_ref, prob.v))
    yield prob, mesh, om, ref
    mesh.close()


def test_pattern_matches_oracle_exactly(case):
    prob, mesh, _, ref = case
    rp, col = mesh.pattern()
    assert mesh.nnz == len(ref["col"])
    assert np.array_equal(rp.cpu().numpy(), ref["rowptr"])
    assert np.array_equal(col.cpu().numpy(), ref["col"])


def test_residual_fp64(case):
    prob, mesh, _, ref = case
    R = mesh.residual(cuda(prob.u))
    assert relerr(R.cpu().numpy(), ref["R"]) <= FP64_TOL
    assert mesh.check() == 0


def test_tangent_csr_fp64_with_residual(case):
    prob, mesh, _, ref = case
    R = mesh.new_vector()
    vals = mesh.tangent_csr(cuda(prob.u), R=R)
    assert relerr(vals.cpu().numpy(), ref["vals"]) <= FP64_TOL
    assert relerr(R.cpu().numpy(), ref["R"]) <= FP64_TOL


def test_apply_tangent_matrix_free_fp64(case):
    prob, mesh, _, ref = case
    y = mesh.apply_tangent(cuda(prob.u), cuda(prob.v))
    assert relerr(y.cpu().numpy(), ref["y_mf"]) <= FP64_TOL


def test_apply_tangent_csr_fp64(case):
    prob, mesh, _, ref = case
    vals = mesh.tangent_csr(cuda(prob.u))
    y = mesh.apply_tangent(None, cuda(prob.v), mode=jetsci().CSR, vals=vals)
    assert relerr(y.cpu().numpy(), ref["y_csr"]) <= FP64_TOL


def test_matrix_free_at_stored_linearisation(case):
    """An FP64 or two-float tangent (or residual) stores the neo-Hookean state at its u; a
    matrix-free product with u = NULL applies K at that state.  It must equal the product that
    forms the state from u (the same arithmetic on the same values) and the oracle."""
    prob, mesh, _, ref = case
    J = jetsci()
    u, v = cuda(prob.u), cuda(prob.v)
    y_direct = mesh.apply_tangent(u, v)
    mesh.tangent_csr(u)
    y_lin = mesh.apply_tangent(None, v)
    assert relerr(y_lin.cpu().numpy(), y_direct.cpu().numpy()) <= 1e-14
    assert relerr(y_lin.cpu().numpy(), ref["y_mf"]) <= FP64_TOL
    # a residual at another state replaces the linearisation
    u2 = u * 0.5
    mesh.residual(u2)
    y2 = mesh.apply_tangent(None, v)
    assert relerr(y2.cpu().numpy(), mesh.apply_tangent(u2, v).cpu().numpy()) <= 1e-14
    # FP32 calls do not touch it
    mesh.tangent_csr(u, precision=J.FP32)
    assert relerr(mesh.apply_tangent(None, v).cpu().numpy(), y2.cpu().numpy()) == 0.0
    # a two-float tangent stores its state too (rounded to double); the two-float product at it
    # matches the two-float product formed from u and the oracle
    mesh.tangent_csr(u, precision=J.DF64)
    y_df = mesh.apply_tangent(None, v, precision=J.DF64)
    assert relerr(y_df.cpu().numpy(), mesh.apply_tangent(u, v, precision=J.DF64).cpu().numpy()) <= 1e-13
    assert relerr(y_df.cpu().numpy(), ref["y_mf"]) <= FP64_TOL
    assert relerr(mesh.apply_tangent(None, v).cpu().numpy(), ref["y_mf"]) <= FP64_TOL


def test_matrix_free_linearisation_errors():
    J = jetsci()
    prob = dict(PROBLEMS)["ragged_neohookean"]
    mesh = J.Mesh.of(prob)
    u, v = cuda(prob.u), cuda(prob.v)
    with pytest.raises(J.JetsciError) as ei:  # nothing stored yet
        mesh.apply_tangent(None, v)
    assert ei.value.status == 1
    mesh.residual(u)
    with pytest.raises(J.JetsciError):  # stored for FP64 and two-float products only
        mesh.apply_tangent(None, v, precision=J.FP32)
    E = torch.full((mesh.n_elem,), 1e9, dtype=torch.float64, device="cuda")
    with pytest.raises(J.JetsciError):  # the state belongs to the phase moduli, not to E
        mesh.apply_tangent(None, v, E_elem=E)
    mesh.residual(u, E_elem=E)
    assert relerr(mesh.apply_tangent(None, v, E_elem=E).cpu().numpy(),
                  mesh.apply_tangent(u, v, E_elem=E).cpu().numpy()) <= 1e-14
    mesh.close()


def test_mesh_structure_validator(case):
    """The device validator of the creation-time assembly data (colouring, slot map, first-writer
    masks, node ids) finds nothing on the structured, distorted and ragged meshes."""
    _, mesh, _, _ = case
    assert mesh.validate() == dict(node_ids=0, colouring=0, slot_map=0, first_writers=0)


def test_mesh_structure_validator_detects_a_swapped_column():
    """Two column indices of node 0's first CSR row swapped in the mesh's own pattern (4-byte
    host-to-device copies into its device array, in bounds) must show as slot-map violations;
    with the entries restored the mesh validates clean again."""
    from cuda.bindings import runtime as cudart
    J = jetsci()
    prob = dict(PROBLEMS)["ragged_neohookean"]
    mesh = J.Mesh.of(prob)
    rp, col = mesh.pattern(device="cpu")
    a = int(rp[0])
    b = a + 3  # first column of node 0's second neighbour
    orig = col.numpy()[[a, b]].copy()

    def put(idx, val):
        buf = np.array([val], dtype=np.int32)
        (err,) = cudart.cudaMemcpy(mesh._col_ptr + 4 * idx, buf.ctypes.data, 4,
                                   cudart.cudaMemcpyKind.cudaMemcpyHostToDevice)
        assert err == cudart.cudaError_t.cudaSuccess

    put(a, orig[1])
    put(b, orig[0])
    with pytest.raises(J.JetsciError) as ei:
        mesh.validate()
    assert ei.value.status == 4
    bad = mesh.validate(raise_on_fail=False)
    assert bad["slot_map"] >= 2 and bad["node_ids"] == 0 and bad["colouring"] == 0
    put(a, orig[0])
    put(b, orig[1])
    assert mesh.validate() == dict(node_ids=0, colouring=0, slot_map=0, first_writers=0)
    mesh.close()


def test_norm2_fp64(case):
    prob, mesh, _, ref = case
    n = mesh.norm2(cuda(ref["R"])).item()
    assert abs(n - oracle.norm2(ref["R"])) <= 1e-14 * oracle.norm2(ref["R"])


def test_fp32_bounds(case):
    prob, mesh, _, ref = case
    J = jetsci()
    u = cuda(prob.u)
    g = GUARD["FP32"]
    R = mesh.residual(u, precision=J.FP32)
    assert relerr(R.cpu().numpy(), ref["R"]) <= min(2e-4, g["R"])
    R2 = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R2, precision=J.FP32)
    assert vals.dtype == torch.float32
    assert relerr(vals.cpu().numpy(), ref["vals"]) <= min(5e-5, g["vals"])
    assert relerr(R2.cpu().numpy(), ref["R"]) <= min(2e-4, g["R"])
    y = mesh.apply_tangent(u, cuda(prob.v), precision=J.FP32)
    assert relerr(y.cpu().numpy(), ref["y_mf"]) <= min(2e-4, g["ymf"])
    yc = mesh.apply_tangent(None, cuda(prob.v), mode=J.CSR, vals=vals, precision=J.FP32)
    assert relerr(yc.cpu().numpy(), ref["y_csr"]) <= min(2e-4, g["ycsr"])


def test_large_volume_change_fp64():
    """Neo-Hookean FP64 residual, tangent and matrix-free products (from u and at the stored
    linearisation) at a large smooth deformation, u_1 = 0.12 sin(pi X_1): the volume ratio J runs
    over about [0.62, 1.38], so Gauss points (often of one warp) take both ln J paths, the series
    in J - 1 for |J - 1| < 1/16 and the library log beyond.  Against the oracle (numpy log)."""
    J = jetsci()
    coords, conn = I.box_mesh(6, 5, 4, distort=0.2, seed=17)
    g = np.random.default_rng(17)
    phase = (g.uniform(size=len(conn)) < 0.5).astype(np.int32)
    u0 = np.zeros_like(coords)
    u0[:, 0] = 0.12 * np.sin(np.pi * coords[:, 0])
    u0 += g.uniform(-1e-3, 1e-3, coords.shape)
    prob = I.Problem("large_volume_change", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     u0.ravel(), g.uniform(-1, 1, coords.size))
    dux = 0.12 * np.pi * np.cos(np.pi * coords[:, 0])
    assert dux.min() < -0.1 and dux.max() > 0.1 and np.any(np.abs(dux) < 0.05)  # both paths
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    y_ref = oracle.apply_tangent(om, prob.u, prob.v)
    u, v = cuda(prob.u), cuda(prob.v)
    assert relerr(mesh.residual(u).cpu().numpy(), R_ref) <= FP64_TOL
    R = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R)
    assert relerr(vals.cpu().numpy(), vals_ref) <= FP64_TOL
    assert relerr(R.cpu().numpy(), R_ref) <= FP64_TOL
    assert relerr(mesh.apply_tangent(None, v).cpu().numpy(), y_ref) <= FP64_TOL  # stored linearisation
    assert relerr(mesh.apply_tangent(u, v).cpu().numpy(), y_ref) <= FP64_TOL
    assert mesh.check() == 0
    mesh.close()


def test_bitwise_determinism(case):
    prob, mesh, _, _ = case
    u, v = cuda(prob.u), cuda(prob.v)
    a = [mesh.tangent_csr(u), mesh.residual(u), mesh.apply_tangent(u, v)]
    b = [mesh.tangent_csr(u), mesh.residual(u), mesh.apply_tangent(u, v)]
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_material_gradient_fp64():
    prob = I.lognormal_problem(12, seed=4)
    J = jetsci()
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    u, E = cuda(prob.u), cuda(prob.E_elem)
    R = mesh.residual(u, E_elem=E)
    R_ref = oracle.residual(om, prob.u)
    assert relerr(R.cpu().numpy(), R_ref) <= FP64_TOL
    g = mesh.material_grad(u, R, E_elem=E)
    g_ref = oracle.material_grad(om, prob.u, R_ref)
    assert relerr(g.cpu().numpy(), g_ref) <= FP64_TOL
    # through torch.autograd
    Et = E.clone().requires_grad_(True)
    L = J.MaterialGrad.apply(Et, mesh, u)
    L.backward()
    assert relerr(Et.grad.cpu().numpy(), g_ref) <= FP64_TOL
    assert abs(L.item() - 0.5 * oracle.norm2(R_ref) ** 2) <= 1e-13 * L.item()


def test_material_gradient_from_kept_element_vectors():
    """A residual call given E_elem keeps its element vectors R_e; the gradient with u = NULL
    forms R[dofs_e] . R_e / E_e from them.  It must match the gradient pass that recomputes
    R_e(u; E = 1) (another formula on the same state) and the oracle in FP64, DF64 and FP32,
    and be refused with nothing kept, for another E_elem pointer or another precision.  Through
    torch.autograd a second forward in between makes the backward recompute instead."""
    prob = I.lognormal_problem(12, seed=4)
    J = jetsci()
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    u, E = cuda(prob.u), cuda(prob.E_elem)
    R_ref = oracle.residual(om, prob.u)
    g_ref = oracle.material_grad(om, prob.u, R_ref)
    Rd = cuda(R_ref)
    with pytest.raises(J.JetsciError) as ei:  # nothing kept yet
        mesh.material_grad(None, Rd, E_elem=E)
    assert ei.value.status == 1
    mesh.residual(u)  # the phase moduli: keeps nothing
    with pytest.raises(J.JetsciError):
        mesh.material_grad(None, Rd, E_elem=E)
    # (precision, kept vs recomputed, vs oracle): FP32 as the FP32 residual bound
    for p, tol_same, tol_ref in ((J.FP64, 1e-13, FP64_TOL), (J.DF64, 1e-13, FP64_TOL), (J.FP32, 1e-5, 2e-4)):
        R = mesh.residual(u, E_elem=E, precision=p)
        g_kept = mesh.material_grad(None, R, E_elem=E, precision=p).cpu().numpy()
        g_rec = mesh.material_grad(u, R, E_elem=E, precision=p).cpu().numpy()
        assert relerr(g_kept, g_rec) <= tol_same, p
        assert relerr(g_kept, g_ref) <= tol_ref, p
    with pytest.raises(J.JetsciError):  # kept by an FP32 call
        mesh.material_grad(None, Rd, E_elem=E, precision=J.FP64)
    with pytest.raises(J.JetsciError):  # another array with the same values
        mesh.material_grad(None, Rd, E_elem=E.clone(), precision=J.FP32)
    assert mesh.check() == 0
    Et = E.clone().requires_grad_(True)
    L1 = J.MaterialGrad.apply(Et, mesh, u)
    J.MaterialGrad.apply(Et, mesh, u * 0.5)  # replaces the element vectors L1's forward kept
    L1.backward()
    assert relerr(Et.grad.cpu().numpy(), g_ref) <= FP64_TOL
    mesh.close()


@pytest.mark.parametrize("name", ["FP64", "FP32", "DF64", "TF32"])
def test_tangent_overwrites_every_value(case, name):
    """The tangent does not clear the value array: in the coloured scatter (FP64) each CSR
    block's first writer (its lowest-colour element) stores and later colours add; in the
    row-gather assembly (FP32, TF32) each row is written once.  Whatever vals held before must
    not leak into the result, and every block must be written."""
    prob, mesh, _, _ = case
    J = jetsci()
    p = getattr(J, name)
    u = cuda(prob.u)
    a = mesh.new_values(p)
    a.zero_()
    mesh.tangent_csr(u, vals=a, precision=p)
    b = mesh.new_values(p)
    b.fill_(float("nan"))
    mesh.tangent_csr(u, vals=b, precision=p)
    assert torch.equal(a, b)


def test_shuffled_numbering_general_colouring():
    """Node ids and element order of a distorted 6x5x4 box shuffled: the greedy colouring is no
    longer the 8 parity classes, and the pattern, slot map and first-writer masks come from a
    general mesh.  FP64 residual, tangent (into NaN-filled values), matrix-free and CSR K.v
    against the oracle."""
    J = jetsci()
    coords, conn = I.box_mesh(6, 5, 4, distort=0.25, seed=9)
    g = np.random.default_rng(9)
    perm_n = g.permutation(len(coords))  # new id of old node k is inv[k]
    inv = np.empty_like(perm_n)
    inv[perm_n] = np.arange(len(coords))
    coords = coords[perm_n]
    conn = inv[conn][g.permutation(len(conn))].astype(np.int32)
    phase = (g.uniform(size=len(conn)) < 0.5).astype(np.int32)
    prob = I.Problem("shuffled_6x5x4", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    mesh = J.Mesh.of(prob)
    assert mesh.n_colours > 8
    assert mesh.validate() == dict(node_ids=0, colouring=0, slot_map=0, first_writers=0)  # general colouring, slot map and first writers
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    u, v = cuda(prob.u), cuda(prob.v)
    R = mesh.new_vector()
    vals = mesh.new_values(J.FP64)
    vals.fill_(float("nan"))
    mesh.tangent_csr(u, vals=vals, R=R)
    assert relerr(R.cpu().numpy(), R_ref) <= FP64_TOL
    assert relerr(vals.cpu().numpy(), vals_ref) <= FP64_TOL
    y_ref = oracle.apply_tangent(om, prob.u, prob.v)
    assert relerr(mesh.apply_tangent(u, v).cpu().numpy(), y_ref) <= FP64_TOL
    assert relerr(mesh.apply_tangent(None, v, mode=J.CSR, vals=vals).cpu().numpy(), y_ref) <= FP64_TOL
    # FP32 row-gather assembly on the same general numbering (NaN-filled outputs)
    R32 = torch.full_like(R, float("nan"))
    vals32 = mesh.new_values(J.FP32)
    vals32.fill_(float("nan"))
    mesh.tangent_csr(u, vals=vals32, R=R32, precision=J.FP32)
    assert relerr(vals32.cpu().numpy(), vals_ref) <= 5e-5
    assert relerr(R32.cpu().numpy(), R_ref) <= 2e-4
    assert mesh.check() == 0
    mesh.close()


def high_valence_problem():
    """Twelve hexahedra sharing node 0 (as local node k mod 8 of element k), each with seven
    nodes of its own, plus one node in no element: node 0 has 12 elements and 85 neighbours
    (more than the 8 elements and 32 neighbours one step of the row pass takes), the isolated
    node has empty rows and a zero residual."""
    g = np.random.default_rng(21)
    corner = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]], float)
    coords = [np.zeros(3)]
    conn = []
    for k in range(12):
        la, h = k % 8, 0.3 + 0.05 * k
        ids = []
        for b in range(8):
            if b == la:
                ids.append(0)
            else:
                coords.append(h * (corner[b] - corner[la]) + g.uniform(-0.03, 0.03, 3))
                ids.append(len(coords) - 1)
        conn.append(ids)
    coords.append(np.array([2.0, 2.0, 2.0]))
    coords = np.array(coords)
    conn = np.array(conn, dtype=np.int32)
    phase = (np.arange(12) % 2).astype(np.int32)
    return I.Problem("high_valence", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))


@pytest.mark.parametrize("name", ["FP64", "FP32", "TF32"])
def test_high_valence_node_and_isolated_node(name):
    J = jetsci()
    prob = high_valence_problem()
    mesh = J.Mesh.of(prob)
    assert mesh.validate() == dict(node_ids=0, colouring=0, slot_map=0, first_writers=0)  # slots up to 84, an empty node
    rp, col = mesh.pattern()
    rp = rp.cpu().numpy()
    assert (rp[1] - rp[0]) // 3 == 85 and rp[-1] == rp[-4]  # node 0: 85 neighbours; last node: none
    om = oracle.Mesh.of(prob)
    orp, ocol = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, orp, ocol)
    p = getattr(J, name)
    u = cuda(prob.u)
    R = torch.full((mesh.n_dof,), float("nan"), dtype=torch.float64, device="cuda")
    vals = mesh.new_values(p)
    vals.fill_(float("nan"))
    mesh.tangent_csr(u, vals=vals, R=R, precision=p)
    tol_v, tol_r = {"FP64": (FP64_TOL, FP64_TOL), "FP32": (GUARD["FP32"]["vals"], GUARD["FP32"]["R"]),
                    "TF32": (GUARD["TF32"]["vals"], GUARD["TF32"]["R"])}[name]
    assert relerr(vals.cpu().numpy(), vals_ref) <= tol_v
    assert relerr(R.cpu().numpy(), R_ref) <= tol_r
    assert torch.count_nonzero(R[-3:]).item() == 0
    assert mesh.check() == 0
    mesh.close()


def test_empty_mesh():
    J = jetsci()
    coords = np.zeros((4, 3))
    mesh = J.Mesh(coords, np.zeros((0, 8), np.int32), None, [(1e9, 0.3, 0)])
    assert mesh.nnz == 0 and mesh.n_dof == 12
    u = torch.ones(12, dtype=torch.float64, device="cuda")
    R = torch.full((12,), 7.0, dtype=torch.float64, device="cuda")
    mesh.residual(u, R=R)
    assert torch.count_nonzero(R).item() == 0
    y = mesh.apply_tangent(u, u.clone())
    assert torch.count_nonzero(y).item() == 0
    for p in (J.FP64, J.FP32):
        R.fill_(7.0)
        vals = mesh.tangent_csr(u, R=R, precision=p)
        assert vals.numel() == 0 and torch.count_nonzero(R).item() == 0
    assert mesh.norm2(u).item() == pytest.approx(np.sqrt(12.0), rel=1e-15)


def test_host_argument_errors():
    J = jetsci()
    coords, conn = I.box_mesh(2)
    with pytest.raises(J.JetsciError) as ei:
        J.Mesh(coords, conn + 100, None, [(1e9, 0.3, 0)])
    assert ei.value.status == 4
    with pytest.raises(J.JetsciError) as ei:
        J.Mesh(coords, conn, None, [(1e9, 0.7, 0)])
    assert ei.value.status == 1
    bad = conn.copy(); bad[0, 1] = bad[0, 0]
    with pytest.raises(J.JetsciError):
        J.Mesh(coords, bad, None, [(1e9, 0.3, 0)])
    mesh = J.Mesh(coords, conn, None, [(1e9, 0.3, 0)])
    u = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(J.JetsciError):
        J._check(J.lib.jetsci_residual(mesh.handle, J._ptr(u), J._ptr(u), 99, None, J._stream()))
    with pytest.raises(J.JetsciError):
        J._check(J.lib.jetsci_apply_tangent(mesh.handle, J._ptr(u), J._ptr(u), J._ptr(u), 0, None, 0, None,
                                            J._stream()))


def test_inverted_element_sets_flag_not_fault():
    """An inverted element is reported through the flag word; the kernel completes."""
    J = jetsci()
    coords, conn = I.box_mesh(2)
    conn = conn.copy()
    conn[0, [0, 1]] = conn[0, [1, 0]]
    mesh = J.Mesh(coords, conn, None, [(1e9, 0.3, 0)])
    u = torch.zeros(mesh.n_dof, dtype=torch.float64, device="cuda")
    mesh.residual(u)
    assert mesh.check() & J.FLAG_BAD_ELEMENT
    assert mesh.check() == 0  # cleared


def test_nonfinite_input_sets_flag_not_fault():
    """A NaN in u reaches the flag word through the residual, the FP64 and FP32 tangents and the
    matrix-free product (a non-finite force, or a state whose det F is not positive); every call
    completes, the check reads and clears the word (JETSCI_ERR_NONFINITE from the C call), and a
    clean input afterwards leaves it clear."""
    J = jetsci()
    prob = dict(PROBLEMS)["ragged_neohookean"]
    mesh = J.Mesh.of(prob)
    u, v = cuda(prob.u), cuda(prob.v)
    bad = u.clone()
    bad[7] = float("nan")
    for call in (lambda: mesh.residual(bad), lambda: mesh.tangent_csr(bad, R=mesh.new_vector()),
                 lambda: mesh.tangent_csr(bad, R=mesh.new_vector(), precision=J.FP32),
                 lambda: mesh.apply_tangent(bad, v)):
        call()
        flags = C.c_uint32()
        assert J.lib.jetsci_mesh_check(mesh.handle, C.byref(flags)) == 5
        assert flags.value & (J.FLAG_NONFINITE | J.FLAG_BAD_STATE)
        assert mesh.check() == 0  # read and cleared
    mesh.residual(u)
    mesh.tangent_csr(u)
    assert mesh.check() == 0
    mesh.close()


def test_newton_and_cg_iteration_caps_report_not_converged():
    """Forced caps: one Newton step, or three CG iterations per step, cannot reach 1e-10; the
    driver returns JETSCI_ERR_NOT_CONVERGED (6) with the iterations it ran and the capped CG solves
    counted, and leaves u finite."""
    J = jetsci()
    coords, conn = I.box_mesh(5, 4, 4, distort=0.15, seed=2)
    g = np.random.default_rng(2)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    prob = I.Problem("newton_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     np.zeros(coords.size), np.zeros(coords.size))
    dofs, vals = I.roller_bcs(coords, 0.01)
    mesh = J.Mesh.of(prob)
    u = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(J.JetsciError) as ei:
        J.newton_solve(mesh, u, dofs, vals, rtol=1e-10, max_newton=1, cg_rtol=1e-10)
    assert ei.value.status == 6
    u.zero_()
    info = J.newton_solve(mesh, u, dofs, vals, rtol=1e-10, max_newton=3, cg_rtol=1e-10, max_cg=3,
                          raise_on_fail=False)
    assert info.newton_iters == 3 and info.cg_capped == 3 and info.cg_iters_total == 9
    assert info.final_rel_residual > 1e-10
    assert torch.isfinite(u).all()
    mesh.close()


@pytest.fixture(scope="module")
def full_size():
    """128^3 fibre RVE, neo-Hookean, 1% stretch, with oracle rows of R, K and K.v at 42 sampled
    nodes computed element by element."""
    prob = I.fibre_composite(128, seed=2)
    om = oracle.Mesh.of(prob)
    g = np.random.default_rng(0)
    nodes = np.concatenate([[0, prob.n_nodes - 1], g.choice(prob.n_nodes, 40, replace=False)])
    rows = oracle.sampled_rows(om, prob.u, prob.v, nodes)
    mesh = jetsci().Mesh.of(prob)
    yield prob, mesh, nodes, rows
    mesh.close()


# (precision name, tolerance of R, of CSR values, of K.v), normwise over the sampled rows; FP32
# and TF32 at the regression guards of the small cases (tighter than their derived bounds).
FULL_SIZE_FORMS = [("FP64", FP64_TOL, FP64_TOL, FP64_TOL, FP64_TOL),
                   ("DF64", FP64_TOL, FP64_TOL, FP64_TOL, FP64_TOL),
                   ("FP32", GUARD["FP32"]["R"], GUARD["FP32"]["vals"], GUARD["FP32"]["ymf"], GUARD["FP32"]["ycsr"]),
                   ("TF32", GUARD["TF32"]["R"], GUARD["TF32"]["vals"], GUARD["TF32"]["ymf"], GUARD["TF32"]["ycsr"])]


def test_full_size_adjoint_sampled_elements():
    """The 64^3 lognormal adjoint workload at its full size, in the bench's launch configuration:
    dL/dE from the kept element vectors and from the recomputing pass, FP64, on 32 sampled
    elements against the oracle (R at each element's nodes summed element by element)."""
    J = jetsci()
    prob = I.lognormal_problem(64, seed=4)
    mesh = J.Mesh.of(prob)
    u, E = cuda(prob.u), cuda(prob.E_elem)
    R = mesh.residual(u, E_elem=E)
    g_kept = mesh.material_grad(None, R, E_elem=E).cpu().numpy()
    g_rec = mesh.material_grad(u, R, E_elem=E).cpu().numpy()
    om = oracle.Mesh.of(prob)
    ptr, eidx = oracle.node_elements(prob.conn, prob.n_nodes)
    sample = np.random.default_rng(7).choice(prob.n_elem, 32, replace=False)
    g_ref = []
    for e in sample:
        nodes = prob.conn[e].astype(np.int64)
        Rn = np.zeros(24)
        for a, n in enumerate(nodes):
            for e2 in eidx[ptr[n]:ptr[n + 1]]:
                Re2 = oracle.element_of(om, int(e2), prob.u, tangent=False)
                a2 = int(np.where(prob.conn[e2] == n)[0][0])
                Rn[3 * a:3 * a + 3] += Re2[3 * a2:3 * a2 + 3]
        Re = oracle.element_of(om, int(e), prob.u, tangent=False)
        g_ref.append(float(Rn @ Re) / float(prob.E_elem[e]))
    g_ref = np.array(g_ref)
    assert relerr(g_kept[sample], g_ref) <= FP64_TOL
    assert relerr(g_rec[sample], g_ref) <= FP64_TOL
    assert mesh.check() == 0
    mesh.close()


def test_full_size_mesh_validates(full_size):
    """The 128^3 mesh's colouring, slot map (513.6 M CSR entries) and first-writer masks."""
    _, mesh, _, _ = full_size
    assert mesh.validate() == dict(node_ids=0, colouring=0, slot_map=0, first_writers=0)


@pytest.mark.parametrize("form", FULL_SIZE_FORMS, ids=[f[0] for f in FULL_SIZE_FORMS])
def test_full_size_fibre_rve_sampled_rows(full_size, form):
    """All forms at the bench's size and launch configuration: sampled rows of R, the CSR
    values and K.v (matrix-free and CSR) against the oracle."""
    prob, mesh, nodes, rows = full_size
    J = jetsci()
    name, tol_R, tol_K, tol_ymf, tol_ycsr = form
    p = getattr(J, name)
    u, v = cuda(prob.u), cuda(prob.v)
    R = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R, precision=p)
    y = mesh.apply_tangent(u, v, precision=p)
    ycsr = mesh.apply_tangent(None, v, mode=J.CSR, vals=vals, precision=p)
    rp, col = mesh.pattern()
    rp, col, vals_h = rp.cpu().numpy(), col.cpu().numpy(), vals.double().cpu().numpy()
    R_h, y_h, yc_h = R.cpu().numpy(), y.cpu().numpy(), ycsr.cpu().numpy()
    scale_R = max(np.max(np.abs(rows[n][0])) for n in nodes)
    scale_y = max(np.max(np.abs(rows[n][1])) for n in nodes)
    scale_K = max(np.max(np.abs(list(rows[n][2].values()))) for n in nodes)
    for n in nodes:
        Rn, Kvn, krow = rows[n]
        assert np.max(np.abs(R_h[3 * n:3 * n + 3] - Rn)) <= tol_R * scale_R
        assert np.max(np.abs(y_h[3 * n:3 * n + 3] - Kvn)) <= tol_ymf * scale_y
        assert np.max(np.abs(yc_h[3 * n:3 * n + 3] - Kvn)) <= tol_ycsr * scale_y
        for i in range(3):
            r = 3 * n + i
            cs = col[rp[r]:rp[r + 1]]
            assert sorted(krow) == list(cs)
            kref = np.array([krow[c][i] for c in cs])
            assert np.max(np.abs(vals_h[rp[r]:rp[r + 1]] - kref)) <= tol_K * scale_K
    assert mesh.check() == 0
    del vals
    torch.cuda.empty_cache()


def test_tf32_tensor_core_bounds(case):
    """TF32 keeps 10 mantissa bits (u = 2^-11): both GEMM operands are rounded, so each
    product carries ~2u; the CSR entries sum 8 elements' contributions and K.v sums 81
    entries per row with cancellation, giving the 3e-3 (values) and 1e-2 (K.v) bounds."""
    prob, mesh, _, ref = case
    J = jetsci()
    u = cuda(prob.u)
    R = mesh.new_vector()
    g = GUARD["TF32"]
    vals = mesh.tangent_csr(u, R=R, precision=J.TF32)
    assert relerr(vals.cpu().numpy(), ref["vals"]) <= min(3e-3, g["vals"])
    assert relerr(R.cpu().numpy(), ref["R"]) <= min(2e-4, g["R"])
    y = mesh.apply_tangent(u, cuda(prob.v), precision=J.TF32)
    assert relerr(y.cpu().numpy(), ref["y_mf"]) <= min(1e-2, g["ymf"])
    yc = mesh.apply_tangent(None, cuda(prob.v), mode=J.CSR, vals=vals, precision=J.TF32)
    assert relerr(yc.cpu().numpy(), ref["y_csr"]) <= min(1e-2, g["ycsr"])
    assert mesh.check() == 0


def _oracle_newton(prob, dofs, vals, rtol=1e-12):
    """Oracle Newton: own assembly, direct sparse solve of the free block (library step)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    u = np.zeros(prob.n_dof)
    u[dofs] = vals
    free = np.ones(prob.n_dof, bool)
    free[dofs] = False
    r0 = None
    for _ in range(30):
        v, R = oracle.tangent_csr(om, u, rp, col)
        nr = np.linalg.norm(R[free])
        r0 = nr if r0 is None else r0
        if nr <= rtol * r0:
            break
        K = sp.csr_matrix((v, col, rp), shape=(prob.n_dof, prob.n_dof))[free][:, free]
        u[free] -= spla.spsolve(K.tocsc(), R[free])
    return u


@pytest.mark.parametrize("tp", ["fp64", "fp32", "tf32"])
def test_newton_cg_jacobi_converges_to_oracle_solution(tp):
    J = jetsci()
    coords, conn = I.box_mesh(5, 4, 4, distort=0.15, seed=2)
    g = np.random.default_rng(2)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    prob = I.Problem("newton_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     np.zeros(coords.size), np.zeros(coords.size))
    dofs, vals = I.roller_bcs(coords, 0.01)
    mesh = J.Mesh.of(prob)
    u = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    info = J.newton_solve(mesh, u, dofs, vals, tangent_precision={"fp64": J.FP64, "fp32": J.FP32, "tf32": J.TF32}[tp],
                          rtol=1e-10, cg_rtol=1e-10)
    assert info.final_rel_residual <= 1e-10
    assert info.newton_iters <= (6 if tp == "fp64" else 12)
    # the device-time split covers every phase that ran
    assert info.seconds_residual > 0 and info.seconds_tangent > 0 and info.seconds_solve > 0
    u_ref = _oracle_newton(prob, dofs, vals)
    assert relerr(u.cpu().numpy(), u_ref) <= 1e-8


def test_df64_two_float_path_meets_the_fp64_tolerance(case):
    """Two-float arithmetic (about 48 significant bits) on the FP32 pipes: the same 1e-12
    normwise bar as the FP64 path."""
    prob, mesh, om, ref = case
    J = jetsci()
    u, v = cuda(prob.u), cuda(prob.v)
    R = mesh.residual(u, precision=J.DF64)
    assert relerr(R.cpu().numpy(), ref["R"]) <= FP64_TOL
    R2 = mesh.new_vector()
    vals = mesh.tangent_csr(u, R=R2, precision=J.DF64)
    assert vals.dtype == torch.float64
    assert relerr(vals.cpu().numpy(), ref["vals"]) <= FP64_TOL
    assert relerr(R2.cpu().numpy(), ref["R"]) <= FP64_TOL
    y = mesh.apply_tangent(u, v, precision=J.DF64)
    assert relerr(y.cpu().numpy(), ref["y_mf"]) <= FP64_TOL
    assert mesh.check() == 0


def test_df64_material_gradient():
    prob = I.lognormal_problem(12, seed=4)
    J = jetsci()
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    u, E = cuda(prob.u), cuda(prob.E_elem)
    R = mesh.residual(u, E_elem=E, precision=J.DF64)
    R_ref = oracle.residual(om, prob.u)
    assert relerr(R.cpu().numpy(), R_ref) <= FP64_TOL
    g = mesh.material_grad(u, R, E_elem=E, precision=J.DF64)
    assert relerr(g.cpu().numpy(), oracle.material_grad(om, prob.u, R_ref)) <= FP64_TOL


def test_full_size_adjoint_central_differences():
    """dL/dE on the 64^3 lognormal workload against central differences of L = 1/2 ||R(u; E)||^2
    taken through the library's own residual and norm (the calibration gradient of the
    Introduction, checked as the adjoint-exactness pin states).  R is linear in each E_e, so L
    is exactly quadratic in E_e and the central difference has no truncation error for any
    step: h = 1e-2 E_e keeps the change of L (about 1e-7 of L) far above the rounding of the
    fixed-order norm (about 1e-15 of L), so the difference is accurate to about 1e-8.  FP64
    gradient (kept-vector and recomputing passes): 1e-6 relative to the largest sampled
    gradient, on 32 seeded elements.  The FP32 gradient against the same FP64 differences:
    the FP32 residual bound 2e-4 (its R and R_e carry that relative error)."""
    J = jetsci()
    prob = I.lognormal_problem(64, seed=4)
    mesh = J.Mesh.of(prob)
    u, E = cuda(prob.u), cuda(prob.E_elem)
    sample = np.random.default_rng(17).choice(prob.n_elem, 32, replace=False)
    R = mesh.residual(u, E_elem=E)
    g_kept = mesh.material_grad(None, R, E_elem=E).cpu().numpy()[sample]
    g_rec = mesh.material_grad(u, R, E_elem=E).cpu().numpy()[sample]
    R32 = mesh.residual(u, E_elem=E, precision=J.FP32)
    g32 = mesh.material_grad(None, R32, E_elem=E, precision=J.FP32).cpu().numpy()[sample]
    fd = []
    Ep = E.clone()
    for e in sample:
        h = 1e-2 * float(prob.E_elem[e])
        L = []
        for sgn in (1.0, -1.0):
            Ep[e] = float(prob.E_elem[e]) + sgn * h
            L.append(0.5 * mesh.norm2(mesh.residual(u, E_elem=Ep)).item() ** 2)
        Ep[e] = float(prob.E_elem[e])
        fd.append((L[0] - L[1]) / (2 * h))
    fd = np.array(fd)
    assert relerr(g_kept, fd) <= 1e-6, relerr(g_kept, fd)
    assert relerr(g_rec, fd) <= 1e-6, relerr(g_rec, fd)
    assert relerr(g32, fd) <= 2e-4, relerr(g32, fd)
    assert mesh.check() == 0
    mesh.close()


def test_medium_box_row_gather_fp32_tf32():
    """A distorted 40 x 40 x 24 box (38,400 elements, 2,400 element-pass blocks): the FP32 and TF32
    row-gather assembly against the oracle within their guards, every value written
    (NaN-prefilled outputs), and bitwise repeatable."""
    J = jetsci()
    coords, conn = I.box_mesh(40, 40, 24, distort=0.2, seed=12)
    g = np.random.default_rng(12)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    prob = I.Problem("medium_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    u = cuda(prob.u)
    for name in ("FP32", "TF32"):
        p = getattr(J, name)
        R = torch.full((mesh.n_dof,), float("nan"), dtype=torch.float64, device="cuda")
        vals = mesh.new_values(p)
        vals.fill_(float("nan"))
        mesh.tangent_csr(u, vals=vals, R=R, precision=p)
        assert relerr(vals.cpu().numpy(), vals_ref) <= GUARD[name]["vals"], name
        assert relerr(R.cpu().numpy(), R_ref) <= GUARD[name]["R"], name
        vals2 = mesh.tangent_csr(u, precision=p)
        assert torch.equal(vals, vals2)
    assert mesh.check() == 0
    mesh.close()


@pytest.mark.parametrize("n", [1, 7, 8, 23, 24, 25, 39, 40, 41, 81, 121])
def test_row_gather_batch_edges(n):
    """Element counts around the row-gather element passes' batch edges: partial octets, a batch
    of 40 tensor-core elements whose last staged chunk is partial or empty, several batches.  A
    chain of n distorted elements (box n x 1 x 1), FP32 and TF32 tangents from NaN-prefilled
    outputs against the oracle within their guards, and the FP64 tangent at 1e-12."""
    J = jetsci()
    coords, conn = I.box_mesh(n, 1, 1, distort=0.2, seed=40 + n)
    g = np.random.default_rng(40 + n)
    phase = (g.uniform(size=len(conn)) < 0.5).astype(np.int32)
    prob = I.Problem(f"chain_{n}", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    mesh = J.Mesh.of(prob)
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    u = cuda(prob.u)
    for name in ("FP64", "FP32", "TF32"):
        p = getattr(J, name)
        R = torch.full((mesh.n_dof,), float("nan"), dtype=torch.float64, device="cuda")
        vals = mesh.new_values(p)
        vals.fill_(float("nan"))
        mesh.tangent_csr(u, vals=vals, R=R, precision=p)
        tv = FP64_TOL if name == "FP64" else GUARD[name]["vals"]
        tr = FP64_TOL if name == "FP64" else GUARD[name]["R"]
        assert relerr(vals.cpu().numpy(), vals_ref) <= tv, name
        assert relerr(R.cpu().numpy(), R_ref) <= tr, name
    assert mesh.check() == 0
    mesh.close()


def test_bounded_wait_runs_out_and_reports():
    """The bounded mbarrier wait of the tensor-core kernels: on a barrier that nothing completes
    it gives up after its poll limit and reports it (no hang, no fault), on one that an arrival
    completes it returns at once; the device stays usable (a tangent afterwards matches the
    oracle)."""
    J = jetsci()
    assert J.selftest_bounded_wait(1000, arrive=False) is True
    assert J.selftest_bounded_wait(1000, arrive=True) is False
    assert J.selftest_bounded_wait(1, arrive=True) is False
    with pytest.raises(J.JetsciError):
        J.selftest_bounded_wait(0, arrive=True)
    prob = PROBLEMS[2][1]
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    mesh = J.Mesh.of(prob)
    R = mesh.new_vector()
    vals = mesh.tangent_csr(cuda(prob.u), R=R)
    assert relerr(vals.cpu().numpy(), vals_ref) <= FP64_TOL
    assert relerr(R.cpu().numpy(), R_ref) <= FP64_TOL
    assert mesh.check() == 0
    mesh.close()
