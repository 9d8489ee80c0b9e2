"""Insertion of caller-formed element blocks (jetsci_assemble_element_blocks) into the CSR
pattern, against the plain definition K = sum_e P_e^T K_e P_e written with scipy's COO -> CSR
conversion (which sums duplicate entries), and against the library's own tangent assembly when
the blocks are the oracle's element tangents.

Tolerances: the library sums the up to 8 contributions of an entry colour by colour, scipy in
its own order; the difference is rounding of at most 8 terms, so 1e-14 normwise for FP64
blocks and 2e-6 for FP32 (8 x 2^-24 with margin).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import oracle
from paper_2604_22087_b300 import inputs as I

pytestmark = pytest.mark.gpu


def jetsci():
    from paper_2604_22087_b300 import jetsci as J
    return J


def relerr(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)), 1e-300))


def coo_assemble(conn, n_nodes, Ke):
    """CSR (indptr, indices, data) of sum_e P_e^T K_e P_e, local DOF 3a + i."""
    conn = np.asarray(conn, dtype=np.int64)
    n = 3 * n_nodes
    dofs = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(len(conn), 24)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    K = sp.coo_matrix((np.asarray(Ke, dtype=np.float64).ravel(), (rows, cols)), shape=(n, n)).tocsr()
    K.sum_duplicates()
    K.sort_indices()
    return K.indptr, K.indices, K.data


def meshes():
    coords, conn = I.box_mesh(5, 7, 3, distort=0.25, seed=3)
    g = np.random.default_rng(3)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    ragged = I.Problem("ragged_5x7x3", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                       g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    sphere = I.sphere_composite(16, seed=1, law=I.LAW_NEO_HOOKEAN)
    return [("ragged_5x7x3", ragged), ("sphere16", sphere)]


MESHES = dict(meshes())


@pytest.fixture(scope="module", params=list(MESHES))
def case(request):
    prob = MESHES[request.param]
    mesh = jetsci().Mesh.of(prob)
    yield prob, mesh
    mesh.close()


def random_blocks(n_elem, seed):
    return np.random.default_rng(seed).normal(size=(n_elem, 24, 24))


def test_random_fp64_blocks_match_coo_sum(case):
    prob, mesh = case
    Ke = random_blocks(prob.n_elem, 41)
    vals = mesh.assemble_blocks(torch.as_tensor(Ke).cuda())
    indptr, indices, data = coo_assemble(prob.conn, prob.n_nodes, Ke)
    rp, col = mesh.pattern()
    assert np.array_equal(rp.cpu().numpy(), indptr)
    assert np.array_equal(col.cpu().numpy(), indices)
    assert relerr(vals.cpu().numpy(), data) <= 1e-14


def test_random_fp32_blocks_match_coo_sum(case):
    prob, mesh = case
    Ke = random_blocks(prob.n_elem, 43).astype(np.float32)
    vals = mesh.assemble_blocks(torch.as_tensor(Ke).cuda())
    assert vals.dtype == torch.float32
    _, _, data = coo_assemble(prob.conn, prob.n_nodes, Ke)
    assert relerr(vals.cpu().numpy(), data) <= 2e-6


def test_oracle_element_tangents_reproduce_the_assembled_tangent(case):
    """Blocks = the oracle's K_e at the case's state: the inserted matrix equals both the
    oracle's CSR tangent and the library's own FP64 tangent assembly."""
    prob, mesh = case
    om = oracle.Mesh.of(prob)
    Ke = np.stack([oracle.element_of(om, e, prob.u)[1] for e in range(prob.n_elem)])
    vals = mesh.assemble_blocks(torch.as_tensor(Ke).cuda()).cpu().numpy()
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    ref = oracle.tangent_csr(om, prob.u, rp, col, with_residual=False)
    assert relerr(vals, ref) <= 1e-14
    J = jetsci()
    own = mesh.tangent_csr(torch.as_tensor(prob.u).cuda(), precision=J.FP64).cpu().numpy()
    assert relerr(vals, own) <= 1e-12


def test_insertion_is_bitwise_reproducible(case):
    prob, mesh = case
    Ke = torch.as_tensor(random_blocks(prob.n_elem, 47)).cuda()
    a = mesh.assemble_blocks(Ke).cpu().numpy()
    b = mesh.assemble_blocks(Ke).cpu().numpy()
    assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_overwrites_previous_values(case):
    prob, mesh = case
    J = jetsci()
    vals = torch.full((mesh.nnz,), 5.0, dtype=torch.float64, device="cuda")
    Ke = torch.zeros(prob.n_elem, 24, 24, dtype=torch.float64, device="cuda")
    mesh.assemble_blocks(Ke, vals=vals)
    assert torch.count_nonzero(vals).item() == 0
    assert vals.dtype == torch.float64 and J.FP64 == 0


def test_argument_errors():
    J = jetsci()
    coords, conn = I.box_mesh(2)
    mesh = J.Mesh(coords, conn, None, [(1e9, 0.3, 0)])
    Ke = torch.zeros(mesh.n_elem, 24, 24, dtype=torch.float64, device="cuda")
    vals = mesh.new_values(J.FP64)
    with pytest.raises(J.JetsciError) as ei:
        J._check(J.lib.jetsci_assemble_element_blocks(mesh.handle, J._ptr(Ke), J._ptr(vals), J.TF32, J._stream()))
    assert ei.value.status == 1
    with pytest.raises(J.JetsciError) as ei:
        J._check(J.lib.jetsci_assemble_element_blocks(mesh.handle, None, J._ptr(vals), J.FP64, J._stream()))
    assert ei.value.status == 1
    with pytest.raises(ValueError):
        mesh.assemble_blocks(torch.zeros(mesh.n_elem, 24, 23, dtype=torch.float64, device="cuda"))
    # blocks are read in 16-byte pieces: a pointer off that boundary is refused before any launch
    flat = torch.zeros(mesh.n_elem * 576 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(J.JetsciError) as ei:
        J._check(J.lib.jetsci_assemble_element_blocks(mesh.handle, J._ptr(flat[1:]), J._ptr(vals), J.FP64,
                                                      J._stream()))
    assert ei.value.status == 1
    empty = J.Mesh(np.zeros((4, 3)), np.zeros((0, 8), np.int32), None, [(1e9, 0.3, 0)])
    out = empty.assemble_blocks(torch.zeros(0, 24, 24, dtype=torch.float64, device="cuda"))
    assert out.numel() == 0
    mesh.close()
    empty.close()
