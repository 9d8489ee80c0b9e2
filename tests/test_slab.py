"""Slab decomposition of one mesh over parts (host logic, CPU): partition structure, halo
exchange, and the owned rows of R, K and K v computed on each part's sub-mesh by the oracle
against the oracle's rows of the whole mesh; then the same with two gloo ranks exchanging
halos and reducing the norm through torch.distributed."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2604_22087_b300 import inputs as I
from paper_2604_22087_b300 import slab as S


def _problem(nx=4, ny=3, nz=7, seed=5):
    coords, conn = I.box_mesh(nx, ny, nz, distort=0.2, seed=seed)
    g = np.random.default_rng(seed)
    phase = (g.uniform(size=len(conn)) < 0.4).astype(np.int32)
    return I.Problem("slab_box", coords, conn, phase, I.composite_materials(I.LAW_NEO_HOOKEAN),
                     g.uniform(-3e-3, 3e-3, coords.size), g.uniform(-1, 1, coords.size))


def _global_rows(prob):
    om = oracle.Mesh.of(prob)
    rp, col = oracle.csr_pattern(prob.conn, prob.n_nodes)
    vals, R = oracle.tangent_csr(om, prob.u, rp, col)
    y = oracle.apply_tangent(om, prob.u, prob.v)
    return dict(R=R, rp=rp, col=col, vals=vals, y=y)


def _part_rows(prob, s, u_loc, v_loc):
    """The oracle on part s's sub-mesh (its elements, local numbering)."""
    om = oracle.Mesh(prob.coords[s.nodes], s.conn, prob.phase[s.elems], prob.materials)
    rp, col = oracle.csr_pattern(s.conn, len(s.nodes))
    vals, R = oracle.tangent_csr(om, u_loc, rp, col)
    y = oracle.apply_tangent(om, u_loc, v_loc)
    return dict(R=R, rp=rp, col=col, vals=vals, y=y)


def _check_owned(s, loc, glob):
    """Owned rows of a part equal the whole mesh's rows, bit for bit: every element around an
    owned node is in the part, in ascending global order, so each entry sums the same terms in
    the same order."""
    gd = s.dofs()
    n = s.n_owned_dof
    assert np.array_equal(loc["R"][:n], glob["R"][gd[:n]])
    assert np.array_equal(loc["y"][:n], glob["y"][gd[:n]])
    for r in range(n):
        lc = gd[loc["col"][loc["rp"][r]:loc["rp"][r + 1]]]
        lv = loc["vals"][loc["rp"][r]:loc["rp"][r + 1]]
        g = gd[r]
        gc = glob["col"][glob["rp"][g]:glob["rp"][g + 1]]
        gv = glob["vals"][glob["rp"][g]:glob["rp"][g + 1]]
        o = np.argsort(lc)
        assert np.array_equal(lc[o], gc)
        assert np.array_equal(lv[o], gv)


@pytest.mark.parametrize("n_parts", [1, 2, 3, 5])
def test_partition_structure(n_parts):
    prob = _problem()
    slabs = S.decompose(prob.coords, prob.conn, n_parts)
    owner = S.node_owner(prob.coords, n_parts)
    # owned nodes partition the mesh into slabs ordered along z
    owned = np.concatenate([s.nodes[:s.n_owned] for s in slabs])
    assert np.array_equal(np.sort(owned), np.arange(prob.n_nodes))
    zmax = [prob.coords[s.nodes[:s.n_owned], 2].max() for s in slabs]
    zmin = [prob.coords[s.nodes[:s.n_owned], 2].min() for s in slabs]
    assert all(zmax[p] <= zmin[p + 1] for p in range(n_parts - 1))
    counts = [s.n_owned for s in slabs]
    assert max(counts) - min(counts) <= 1
    for s in slabs:
        p = s.part
        # the part's elements are exactly those touching an owned node
        touch = np.nonzero(np.any(owner[prob.conn] == p, axis=1))[0]
        assert np.array_equal(s.elems, touch)
        # local numbering: owned then ghosts, each ascending; connectivity maps back
        assert np.all(np.diff(s.nodes[:s.n_owned]) > 0) and np.all(np.diff(s.nodes[s.n_owned:]) > 0)
        assert np.all(owner[s.nodes[s.n_owned:]] != p)
        assert np.array_equal(s.nodes[s.conn], prob.conn[s.elems])
        # every ghost is received once, from its owner
        got = np.concatenate([s.recv[q] for q in sorted(s.recv)]) if s.recv else np.zeros(0, int)
        assert np.array_equal(np.sort(got), np.arange(s.n_owned_dof, s.n_dof))
        for q, idx in s.recv.items():
            assert np.all(owner[s.nodes[idx[0::3] // 3]] == q)
            # the owner sends the same global DOFs in the same order
            assert np.array_equal(slabs[q].dofs()[slabs[q].send[p]], s.dofs()[idx])
            assert np.all(slabs[q].send[p] < slabs[q].n_owned_dof)
    if n_parts == 1:
        assert not slabs[0].recv and not slabs[0].send and len(slabs[0].elems) == prob.n_elem


@pytest.mark.parametrize("n_parts", [2, 3])
def test_owned_rows_equal_whole_mesh_rows(n_parts):
    """Halo exchange in one process (NaN ghosts before it), then the oracle on every part's
    sub-mesh: owned rows of R, CSR K and K v equal the whole mesh's, and the norm from the
    parts' owned sums matches the whole residual's."""
    prob = _problem()
    glob = _global_rows(prob)
    slabs = S.decompose(prob.coords, prob.conn, n_parts)
    us = [torch.as_tensor(s.scatter_owned(prob.u)) for s in slabs]
    vs = [torch.as_tensor(s.scatter_owned(prob.v)) for s in slabs]
    assert all(torch.isnan(x[s.n_owned_dof:]).all() for x, s in zip(us, slabs) if s.n_dof > s.n_owned_dof)
    S.exchange_in_process(slabs, us)
    S.exchange_in_process(slabs, vs)
    partials = []
    for s, u, v in zip(slabs, us, vs):
        assert np.array_equal(u.numpy(), prob.u[s.dofs()]) and np.array_equal(v.numpy(), prob.v[s.dofs()])
        loc = _part_rows(prob, s, u.numpy(), v.numpy())
        _check_owned(s, loc, glob)
        partials.append(oracle.norm2(loc["R"][:s.n_owned_dof]) ** 2)
    nrm = S.norm2_from_partials(partials)
    ref = oracle.norm2(glob["R"])
    assert abs(nrm - ref) <= 1e-14 * ref


def _gloo_rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob = _problem(3, 4, 9, seed=8)
        glob = _global_rows(prob)
        slabs = S.decompose(prob.coords, prob.conn, world)
        s = slabs[rank]
        u = torch.as_tensor(s.scatter_owned(prob.u))
        v = torch.as_tensor(s.scatter_owned(prob.v))
        S.exchange(s, u)
        S.exchange(s, v)
        assert np.array_equal(u.numpy(), prob.u[s.dofs()])
        assert np.array_equal(v.numpy(), prob.v[s.dofs()])
        loc = _part_rows(prob, s, u.numpy(), v.numpy())
        _check_owned(s, loc, glob)
        nrm = S.norm2(s, oracle.norm2(loc["R"][:s.n_owned_dof]))
        ref = oracle.norm2(glob["R"])
        assert abs(nrm - ref) <= 1e-14 * ref
        with open(os.path.join(out_dir, f"rank{rank}.ok"), "w") as f:
            f.write(repr(nrm))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_and_reduce(tmp_path):
    """Two processes over gloo (127.0.0.1): each builds its part, fills its ghosts by the
    point-to-point halo exchange, computes its sub-mesh with the oracle and checks its owned
    rows against the whole mesh; the all-gathered norm is the same on both ranks."""
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    mp.spawn(_gloo_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    vals = [open(tmp_path / f"rank{r}.ok").read() for r in range(2)]
    assert vals[0] == vals[1]
