"""Owner-computes slab decomposition of one hex8 mesh over ranks (the paper distributes its
assembled system over MPI ranks, Section III-D, and names multi-GPU runs as future work,
Section VI).

Each part owns the nodes of one slab along an axis (nodes ordered by coordinate, then id,
cut into equal counts) and holds every element that touches an owned node: the owned nodes'
rows of R, of the CSR matrix and of K v are then complete on that part, with no exchange of
element contributions.  The other nodes of those elements are its ghosts (a one-element
layer around the slab).  Local numbering puts the owned nodes first, in global order, then
the ghosts, in global order, so a part's owned DOFs are the prefix [0, n_owned_dof) of its
local vectors and its owned CSR rows are the first rows of its local pattern.

Before each residual, tangent or product the ghost entries of u (and v) are refreshed from
their owners (`exchange`, one halo of node values per neighbouring part); the norm of R is
the fixed-order sum of the parts' owned sums of squares (`norm2`).  This module holds only
the index bookkeeping and the exchanges; the element work and the norms run in the library's
kernels on each part's sub-mesh (`SlabMesh`), and the halo values are packed with plain
tensor indexing around the point-to-point calls.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def node_owner(coords: np.ndarray, n_parts: int, axis: int = 2) -> np.ndarray:
    """Part of every node: nodes ordered by (coordinate along `axis`, id) and cut into n_parts
    runs of equal length (the first n_nodes % n_parts runs one longer)."""
    n = coords.shape[0]
    if n_parts < 1 or n_parts > max(n, 1):
        raise ValueError("need 1 <= n_parts <= n_nodes")
    order = np.lexsort((np.arange(n), coords[:, axis]))
    counts = np.full(n_parts, n // n_parts)
    counts[: n % n_parts] += 1
    owner = np.empty(n, dtype=np.int32)
    owner[order] = np.repeat(np.arange(n_parts, dtype=np.int32), counts)
    return owner


@dataclass
class Slab:
    """One part of the decomposition (all arrays host numpy).

    elems        global ids of the part's elements (those touching an owned node), ascending
    nodes        local -> global node id: owned nodes first, then ghosts, each ascending
    n_owned      number of owned nodes (the first n_owned local nodes)
    conn         the elements' connectivity in local node ids [n_elem_local, 8]
    send[q]      local DOFs of owned nodes that part q holds as ghosts (q's receive order)
    recv[q]      local DOFs of this part's ghosts owned by q (ascending global id)
    """
    part: int
    n_parts: int
    elems: np.ndarray
    nodes: np.ndarray
    n_owned: int
    conn: np.ndarray
    send: dict
    recv: dict

    @property
    def n_owned_dof(self) -> int:
        return 3 * self.n_owned

    @property
    def n_dof(self) -> int:
        return 3 * len(self.nodes)

    def dofs(self) -> np.ndarray:
        """Global DOF of every local DOF."""
        return (3 * self.nodes[:, None].astype(np.int64) + np.arange(3)).ravel()

    def scatter_owned(self, x_global: np.ndarray) -> np.ndarray:
        """Local vector with the owned entries of a global vector and NaN at the ghosts (what a
        part holds before its first exchange)."""
        x = np.full(self.n_dof, np.nan)
        x[: self.n_owned_dof] = x_global[self.dofs()[: self.n_owned_dof]]
        return x


def _dofs_of(local_nodes: np.ndarray) -> np.ndarray:
    return (3 * local_nodes[:, None].astype(np.int64) + np.arange(3)).ravel()


def decompose(coords: np.ndarray, conn: np.ndarray, n_parts: int, axis: int = 2) -> list:
    """All parts of the decomposition (every rank computes the same list from the same mesh)."""
    coords = np.asarray(coords, dtype=np.float64)
    conn = np.asarray(conn, dtype=np.int64)
    n_nodes = coords.shape[0]
    owner = node_owner(coords, n_parts, axis)
    # element e belongs to every part that owns one of its nodes
    parts_of_elem = owner[conn]  # [n_elem, 8]
    elems, ghosts = [], []
    for p in range(n_parts):
        ep = np.nonzero(np.any(parts_of_elem == p, axis=1))[0]
        elems.append(ep)
        nodes = np.unique(conn[ep]) if len(ep) else np.zeros(0, dtype=np.int64)
        ghosts.append(nodes[owner[nodes] != p])
    owned = [np.nonzero(owner == p)[0] for p in range(n_parts)]
    out = []
    for p in range(n_parts):
        nodes = np.concatenate([owned[p], ghosts[p]]).astype(np.int64)
        local = -np.ones(n_nodes, dtype=np.int64)
        local[nodes] = np.arange(len(nodes))
        lconn = local[conn[elems[p]]].astype(np.int32)
        recv = {}
        for q in range(n_parts):
            if q == p:
                continue
            g = ghosts[p][owner[ghosts[p]] == q]
            if len(g):
                recv[q] = _dofs_of(local[g])
        out.append(Slab(p, n_parts, elems[p], nodes, len(owned[p]), lconn, {}, recv))
    # part p sends to q the owned nodes q holds as ghosts, in q's receive order (ascending id)
    for q in range(n_parts):
        for p, _ in out[q].recv.items():
            g = ghosts[q][owner[ghosts[q]] == p]
            local_p = -np.ones(n_nodes, dtype=np.int64)
            local_p[out[p].nodes] = np.arange(len(out[p].nodes))
            out[p].send[q] = _dofs_of(local_p[g])
    return out


# ------------------------------------------------------------------------------ exchanges
def _index(slab: Slab, kind: str, q: int, device):
    """The send or receive DOF list for peer q as an index tensor on `device` (made once)."""
    import torch
    cache = slab.__dict__.setdefault("_idx", {})
    key = (kind, q, str(device))
    if key not in cache:
        cache[key] = torch.as_tensor((slab.send if kind == "send" else slab.recv)[q], device=device)
    return cache[key]


def exchange(slab: Slab, x, group=None):
    """Refresh the ghost entries of the local vector x (a torch tensor on the part's device, or
    on the CPU for gloo) from their owners: one send and one receive per neighbouring part,
    posted together (torch.distributed batch_isend_irecv)."""
    import torch
    import torch.distributed as dist
    if not slab.send and not slab.recv:
        return x
    ops, bufs = [], {}
    for q in sorted(slab.send):
        ops.append(dist.P2POp(dist.isend, x.index_select(0, _index(slab, "send", q, x.device)), q, group))
    for q in sorted(slab.recv):
        bufs[q] = torch.empty(len(slab.recv[q]), dtype=x.dtype, device=x.device)
        ops.append(dist.P2POp(dist.irecv, bufs[q], q, group))
    for r in dist.batch_isend_irecv(ops):
        r.wait()
    for q, b in bufs.items():
        x.index_copy_(0, _index(slab, "recv", q, x.device), b)
    return x


def exchange_in_process(slabs: list, xs: list):
    """The same exchange among parts held by one process (xs[p] = part p's local vector): for
    a single device, or checks, where every part's vector is at hand."""
    import torch
    for p, s in enumerate(slabs):
        for q, idx in s.recv.items():
            src = slabs[q].send[p]
            dev = xs[p].device
            xs[p].index_copy_(0, torch.as_tensor(idx, device=dev),
                              xs[q].index_select(0, torch.as_tensor(src, device=xs[q].device)).to(dev))
    return xs


def norm2_from_partials(partials) -> float:
    """||x|| from the parts' owned sums of squares, added in part order (the same result on
    every rank and for every run)."""
    total = 0.0
    for s in partials:
        total += float(s)
    return float(np.sqrt(total))


def norm2(slab: Slab, owned_norm: float, group=None) -> float:
    """Global ||x||_2 from this part's ||x_owned||_2: all-gather of the squares, fixed-order sum."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([owned_norm * owned_norm], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    parts = [torch.empty_like(t) for _ in range(slab.n_parts)]
    dist.all_gather(parts, t, group=group)
    return norm2_from_partials([p.item() for p in parts])


def norm2_device(slab: Slab, owned_norm, group=None):
    """The same on the device, without a host synchronisation: owned_norm is a 1-entry CUDA
    tensor; the parts' squares are all-gathered and added in part order on the device."""
    import torch
    import torch.distributed as dist
    sq = owned_norm * owned_norm
    parts = torch.empty(slab.n_parts, dtype=sq.dtype, device=sq.device)
    dist.all_gather_into_tensor(parts, sq, group=group)
    total = parts[0:1].clone()
    for k in range(1, slab.n_parts):
        total += parts[k:k + 1]
    return total.sqrt_()


# ------------------------------------------------------------------------------ GPU part
class SlabMesh:
    """One part's sub-mesh on the current CUDA device (a jetsci Mesh of the part's elements and
    local nodes).  Results live in local vectors; their owned prefix holds the complete global
    rows.  The caller refreshes ghost entries (exchange / exchange_in_process) before a call
    that reads u or v."""

    def __init__(self, slab: Slab, coords, phase, materials, stream=None):
        from . import jetsci as J
        self.slab = slab
        ph = None if phase is None else np.asarray(phase)[slab.elems]
        self.mesh = J.Mesh(np.asarray(coords)[slab.nodes], slab.conn, ph, materials, stream)

    def owned(self, x):
        return x[: self.slab.n_owned_dof]

    def owned_norm(self, R, stream=None):
        """||R_owned||_2 by the library's fixed-shape reduction over the owned prefix."""
        return self.mesh.norm2(self.owned(R), stream=stream)

    def close(self):
        self.mesh.close()
