"""Slab decomposition through the library's kernels: every part's sub-mesh on the one GPU of
this process (parts run one after another; the halo exchange copies between their local
vectors in the same process, since no rank here waits on another).  Owned rows of R, of the
CSR values, of matrix-free and CSR K v, and the norm from the parts' owned sums, against the
FP64 oracle of the whole mesh, at the FP64 tolerance 1e-12."""
import numpy as np
import pytest
import torch

import oracle
from paper_2604_22087_b300 import inputs as I
from paper_2604_22087_b300 import slab as S

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-12


def J():
    from paper_2604_22087_b300 import jetsci
    return jetsci


def _cases():
    coords, conn = I.box_mesh(5, 4, 9, distort=0.2, seed=6)
    g = np.random.default_rng(6)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    box = I.Problem("slab_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                    g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))
    sph = I.sphere_composite(16, seed=1, law=I.LAW_NEO_HOOKEAN)
    return [("box_2", box, 2), ("box_3", box, 3), ("sphere16_4", sph, 4)]


CASES = _cases()


@pytest.mark.parametrize("name,prob,n_parts", CASES, ids=[c[0] for c in CASES])
def test_owned_rows_match_oracle(name, prob, n_parts):
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    y_ref = oracle.apply_tangent(om, prob.u, prob.v)
    slabs = S.decompose(prob.coords, prob.conn, n_parts)
    parts = [S.SlabMesh(s, prob.coords, prob.phase, prob.materials) for s in slabs]
    us = [torch.as_tensor(s.scatter_owned(prob.u)).cuda() for s in slabs]
    vs = [torch.as_tensor(s.scatter_owned(prob.v)).cuda() for s in slabs]
    S.exchange_in_process(slabs, us)
    S.exchange_in_process(slabs, vs)
    sR, sK, sy = np.max(np.abs(R_ref)), np.max(np.abs(vals_ref)), np.max(np.abs(y_ref))
    partials = []
    for s, pm, u, v in zip(slabs, parts, us, vs):
        m = pm.mesh
        R = m.new_vector()
        vals = m.tangent_csr(u, R=R)
        y_mf = m.apply_tangent(None, v)  # at the linearisation the tangent stored
        y_csr = m.apply_tangent(None, v, mode=J().CSR, vals=vals)
        partials.append(pm.owned_norm(R).item() ** 2)
        assert m.check() == 0
        gd = s.dofs()
        n = s.n_owned_dof
        assert np.max(np.abs(pm.owned(R).cpu().numpy() - R_ref[gd[:n]])) <= FP64_TOL * sR
        assert np.max(np.abs(pm.owned(y_mf).cpu().numpy() - y_ref[gd[:n]])) <= FP64_TOL * sy
        assert np.max(np.abs(pm.owned(y_csr).cpu().numpy() - y_ref[gd[:n]])) <= FP64_TOL * sy
        lrp, lcol = m.pattern()
        lrp, lcol, lv = lrp.cpu().numpy(), lcol.cpu().numpy(), vals.cpu().numpy()
        for r in range(n):
            lc = gd[lcol[lrp[r]:lrp[r + 1]]]
            o = np.argsort(lc)
            g = gd[r]
            assert np.array_equal(lc[o], col[rp[g]:rp[g + 1]])
            assert np.max(np.abs(lv[lrp[r]:lrp[r + 1]][o] - vals_ref[rp[g]:rp[g + 1]])) <= FP64_TOL * sK
    nrm = S.norm2_from_partials(partials)
    ref = oracle.norm2(R_ref)
    assert abs(nrm - ref) <= 1e-14 * ref
    for pm in parts:
        pm.close()


def test_fp32_owned_rows():
    """The FP32 forms on the parts (row-gather assembly on each sub-mesh): owned rows within the
    FP32 bounds of the whole-mesh tests (2e-4 for R and K v, 5e-5 for CSR values)."""
    name, prob, n_parts = CASES[1]
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
    y_ref = oracle.apply_tangent(om, prob.u, prob.v)
    slabs = S.decompose(prob.coords, prob.conn, n_parts)
    parts = [S.SlabMesh(s, prob.coords, prob.phase, prob.materials) for s in slabs]
    us = S.exchange_in_process(slabs, [torch.as_tensor(s.scatter_owned(prob.u)).cuda() for s in slabs])
    vs = S.exchange_in_process(slabs, [torch.as_tensor(s.scatter_owned(prob.v)).cuda() for s in slabs])
    for s, pm, u, v in zip(slabs, parts, us, vs):
        m = pm.mesh
        R = m.new_vector()
        vals = m.tangent_csr(u, R=R, precision=J().FP32)
        y = m.apply_tangent(u, v, precision=J().FP32)
        gd = s.dofs()
        n = s.n_owned_dof
        assert np.max(np.abs(pm.owned(R).cpu().numpy() - R_ref[gd[:n]])) <= 2e-4 * np.max(np.abs(R_ref))
        assert np.max(np.abs(pm.owned(y).cpu().numpy() - y_ref[gd[:n]])) <= 2e-4 * np.max(np.abs(y_ref))
        lrp, lcol = m.pattern()
        lrp, lcol, lv = lrp.cpu().numpy(), lcol.cpu().numpy(), vals.double().cpu().numpy()
        for r in range(n):
            lc = gd[lcol[lrp[r]:lrp[r + 1]]]
            o = np.argsort(lc)
            g = gd[r]
            assert np.max(np.abs(lv[lrp[r]:lrp[r + 1]][o] - vals_ref[rp[g]:rp[g + 1]])) <= 5e-5 * np.max(np.abs(vals_ref))
        pm.close()


def _gpu_rank(rank, world, port, out_dir):
    """One rank of the two-process test: its part's sub-mesh on cuda:0, ghosts filled by the
    gloo halo exchange of host copies, the FP64 calls through the library, its owned rows
    against the oracle's rows of the whole mesh, the norm all-gathered over gloo."""
    import os
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        _, prob, _ = CASES[0]
        om = oracle.Mesh.of(prob)
        rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
        vals_ref, R_ref = oracle.tangent_csr(om, prob.u, rp, col)
        y_ref = oracle.apply_tangent(om, prob.u, prob.v)
        s = S.decompose(prob.coords, prob.conn, world)[rank]
        pm = S.SlabMesh(s, prob.coords, prob.phase, prob.materials)
        u_h = torch.as_tensor(s.scatter_owned(prob.u))
        v_h = torch.as_tensor(s.scatter_owned(prob.v))
        S.exchange(s, u_h)
        S.exchange(s, v_h)
        u, v = u_h.cuda(), v_h.cuda()
        m = pm.mesh
        R = m.new_vector()
        vals = m.tangent_csr(u, R=R)
        y_mf = m.apply_tangent(None, v)
        y_csr = m.apply_tangent(None, v, mode=J().CSR, vals=vals)
        assert m.check() == 0
        gd, n = s.dofs(), s.n_owned_dof
        sR, sK, sy = np.max(np.abs(R_ref)), np.max(np.abs(vals_ref)), np.max(np.abs(y_ref))
        assert np.max(np.abs(pm.owned(R).cpu().numpy() - R_ref[gd[:n]])) <= FP64_TOL * sR
        assert np.max(np.abs(pm.owned(y_mf).cpu().numpy() - y_ref[gd[:n]])) <= FP64_TOL * sy
        assert np.max(np.abs(pm.owned(y_csr).cpu().numpy() - y_ref[gd[:n]])) <= FP64_TOL * sy
        lrp, lcol = m.pattern()
        lrp, lcol, lv = lrp.cpu().numpy(), lcol.cpu().numpy(), vals.cpu().numpy()
        for r in range(n):
            lc = gd[lcol[lrp[r]:lrp[r + 1]]]
            o = np.argsort(lc)
            g = gd[r]
            assert np.array_equal(lc[o], col[rp[g]:rp[g + 1]])
            assert np.max(np.abs(lv[lrp[r]:lrp[r + 1]][o] - vals_ref[rp[g]:rp[g + 1]])) <= FP64_TOL * sK
        nrm = S.norm2(s, pm.owned_norm(R).item())
        ref = oracle.norm2(R_ref)
        assert abs(nrm - ref) <= 1e-14 * ref
        pm.close()
        with open(os.path.join(out_dir, f"rank{rank}.ok"), "w") as f:
            f.write(repr(nrm))
    finally:
        dist.destroy_process_group()


def test_two_processes_on_the_gpu(tmp_path):
    """Two processes (spawned, gloo over 127.0.0.1), each with its part on the one GPU: the
    kernels of the two ranks never wait on each other (they meet only in host-side gloo
    collectives between calls), so this runs the multi-rank path of the slab decomposition
    through the library as separate processes do."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.spawn(_gpu_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [open(tmp_path / f"rank{r}.ok").read() for r in range(2)]
    assert vals[0] == vals[1]
