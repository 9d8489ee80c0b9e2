"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module draws random numbers and builds geometry only: structured hex8 meshes,
two-phase composite microstructures (spherical inclusions, unidirectional fibres),
a spatially correlated lognormal Young's-modulus field, displacement states, probe
vectors, strain samples and MLP initial weights.  It holds none of the finite-element
arithmetic (no shape functions, no constitutive law, no Lame constants): each side
computes those itself from the (E, nu, law) triples returned here.

The paper's benchmark is a two-phase composite micromechanics problem (Section V-A)
whose microstructure data and mesh sizes are not published; these generators stand in
for it.  All random draws use numpy's PCG64 with an explicit seed.

Conventions (the paper states none; fixed here once for every consumer):
  * unit box [0,1]^3 split into nx*ny*nz hexahedra; node (i,j,k) has id
    i + (nx+1)*(j + (ny+1)*k); element (i,j,k) has id i + nx*(j + ny*k);
  * hex8 local node order in reference coordinates (xi, eta, zeta):
    (-,-,-), (+,-,-), (+,+,-), (-,+,-), (-,-,+), (+,-,+), (+,+,+), (-,+,+);
  * DOF of node n, component c is 3*n + c (interleaved);
  * Voigt order [11, 22, 33, 23, 13, 12] with tensor (not engineering) shear components.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAW_LINEAR_ELASTIC = 0
LAW_NEO_HOOKEAN = 1

# Two-phase composite (matrix, inclusion/fibre): Young's modulus [Pa], Poisson ratio.
MATRIX_E, MATRIX_NU = 3.5e9, 0.35
INCLUSION_E, INCLUSION_NU = 70.0e9, 0.22

# Local node offsets (di, dj, dk) in the order listed in the module docstring.
HEX8_OFFSETS = np.array(
    [[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0], [0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1]],
    dtype=np.int64,
)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def box_mesh(nx: int, ny: int | None = None, nz: int | None = None, distort: float = 0.0,
             seed: int = 0):
    """Structured hex8 mesh of the unit box.

    Returns (coords [n_nodes,3] float64, conn [n_elem,8] int32).  With distort > 0 every
    interior node is moved by U[-distort, distort] times the local spacing along each
    axis (boundary nodes stay on the box faces), which keeps elements valid for
    distort < 0.5 and removes uniform-grid shortcuts from tests.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    if min(nx, ny, nz) < 0:
        raise ValueError("negative mesh size")
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    zs = np.linspace(0.0, 1.0, nz + 1)
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")  # node id = i + (nx+1)(j + (ny+1)k)
    coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)
    if distort > 0.0 and nx > 1 and ny > 1 and nz > 1:
        g = rng(seed)
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        interior = ((i > 0) & (i < nx) & (j > 0) & (j < ny) & (k > 0) & (k < nz)).ravel()
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        d = g.uniform(-distort, distort, size=coords.shape) * h
        coords[interior] += d[interior]
    ke, je, ie = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ie, je, ke = ie.ravel(), je.ravel(), ke.ravel()
    conn = np.empty((nx * ny * nz, 8), dtype=np.int64)
    for a, (di, dj, dk) in enumerate(HEX8_OFFSETS):
        conn[:, a] = (ie + di) + (nx + 1) * ((je + dj) + (ny + 1) * (ke + dk))
    return coords, conn.astype(np.int32)


def element_centroids(coords: np.ndarray, conn: np.ndarray) -> np.ndarray:
    return coords[conn.astype(np.int64)].mean(axis=1)


def sphere_phases(coords, conn, n_incl: int = 12, radius: float = 0.12, seed: int = 1):
    """Phase per element: 1 if the centroid lies within `radius` of any of `n_incl`
    sphere centres drawn U[0,1]^3 (Euclidean, non-periodic, overlaps allowed), else 0."""
    centres = rng(seed).uniform(0.0, 1.0, size=(n_incl, 3))
    c = element_centroids(coords, conn)
    phase = np.zeros(len(conn), dtype=np.int32)
    for p in centres:
        phase[np.sum((c - p) ** 2, axis=1) <= radius * radius] = 1
    return phase, centres


def fibre_centres(radius: float = 0.05, volume_fraction: float = 0.5, seed: int = 2,
                  sweeps: int = 2000, step: float = 0.02):
    """Random non-overlapping fibre centres in the periodic unit square.

    The fibre count is the smallest one whose area fraction reaches `volume_fraction`
    (64 for r = 0.05).  Starting from a jittered square lattice, `sweeps` rounds of
    hard-disk Metropolis moves (uniform step in [-step, step]^2, periodic wrap, minimum
    centre distance 2r) randomise the packing.
    """
    n = int(math.ceil(volume_fraction / (math.pi * radius * radius) - 1e-12))
    side = int(math.ceil(math.sqrt(n)))
    g = rng(seed)
    spacing = 1.0 / side
    jitter = max(0.0, 0.5 * (spacing - 2.0 * radius)) * 0.999
    pts = []
    for t in range(n):
        ix, iy = t % side, t // side
        pts.append([(ix + 0.5) * spacing, (iy + 0.5) * spacing])
    pts = np.array(pts) + g.uniform(-jitter, jitter, size=(n, 2))
    pts %= 1.0
    dmin2 = (2.0 * radius) ** 2
    for _ in range(sweeps):
        order = g.permutation(n)
        moves = g.uniform(-step, step, size=(n, 2))
        for t in order:
            trial = (pts[t] + moves[t]) % 1.0
            d = pts - trial
            d -= np.round(d)
            r2 = np.sum(d * d, axis=1)
            r2[t] = np.inf
            if np.all(r2 >= dmin2):
                pts[t] = trial
    return pts


def fibre_phases(coords, conn, centres, radius: float = 0.05):
    """Phase per element: 1 if the centroid's in-plane (x, y) periodic distance to any
    fibre axis (parallel to z) is at most `radius`, else 0."""
    c = element_centroids(coords, conn)[:, :2]
    phase = np.zeros(len(conn), dtype=np.int32)
    for p in centres:
        d = c - p
        d -= np.round(d)
        phase[np.sum(d * d, axis=1) <= radius * radius] = 1
    return phase


def lognormal_modulus(n: int, median: float = 1.0e10, sigma_log: float = 0.5,
                      blur_voxels: float = 3.0, seed: int = 4):
    """Per-element Young's modulus on an n^3 grid: seeded white N(0,1) noise, periodic
    Gaussian blur (sigma = blur_voxels, truncated at 4 sigma), re-standardised to zero
    mean / unit variance, then E = median * exp(sigma_log * z).  Element order matches
    box_mesh (i fastest)."""
    from scipy.ndimage import gaussian_filter

    z = rng(seed).standard_normal((n, n, n))  # indexed [k, j, i]
    z = gaussian_filter(z, sigma=blur_voxels, mode="wrap", truncate=4.0)
    z = (z - z.mean()) / z.std()
    return (median * np.exp(sigma_log * z)).ravel().astype(np.float64)


def uniform_field(n: int, amp: float, seed: int) -> np.ndarray:
    return rng(seed).uniform(-amp, amp, size=n).astype(np.float64)


def stretch_state(coords: np.ndarray, stretch: float = 0.01, noise: float = 1e-4, seed: int = 2):
    """u = stretch * X1 e1 + U[-noise, noise] per DOF (a uniaxial stretch plus noise)."""
    u = rng(seed + 1000).uniform(-noise, noise, size=coords.size)
    u[0::3] += stretch * coords[:, 0]
    return u.astype(np.float64)


def strain_samples(n: int, bound: float = 0.05, seed: int = 5):
    """Green-Lagrange strain samples: 6 Voigt tensor components U[-bound, bound] and a
    phase ~ Bernoulli(1/2).  Returns (E6 [n,6] float64, phase [n] int32)."""
    g = rng(seed)
    e6 = g.uniform(-bound, bound, size=(n, 6))
    phase = (g.uniform(size=n) < 0.5).astype(np.int32)
    return e6, phase


MLP_IN, MLP_HIDDEN, MLP_OUT = 8, 64, 6


def mlp_init(seed: int = 5):
    """Xavier-uniform initial weights of the 8 -> 64 -> 64 -> 64 -> 6 surrogate MLP,
    zero biases.  Returns a list [(W [out,in] float64, b [out] float64)] * 4."""
    g = rng(seed + 77)
    dims = [MLP_IN, MLP_HIDDEN, MLP_HIDDEN, MLP_HIDDEN, MLP_OUT]
    layers = []
    for fan_in, fan_out in zip(dims[:-1], dims[1:]):
        lim = math.sqrt(6.0 / (fan_in + fan_out))
        layers.append((g.uniform(-lim, lim, size=(fan_out, fan_in)), np.zeros(fan_out)))
    return layers


def minibatch_order(n: int, epochs: int, seed: int = 5) -> np.ndarray:
    """Concatenated per-epoch random permutations of range(n) (int32)."""
    g = rng(seed + 99)
    return np.concatenate([g.permutation(n) for _ in range(epochs)]).astype(np.int32)


@dataclass
class Problem:
    """One synthetic workload: mesh, per-element phase, materials and states."""
    name: str
    coords: np.ndarray
    conn: np.ndarray
    phase: np.ndarray
    materials: list  # [(E, nu, law)] indexed by phase
    u: np.ndarray
    v: np.ndarray
    E_elem: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes


def composite_materials(law: int):
    return [(MATRIX_E, MATRIX_NU, law), (INCLUSION_E, INCLUSION_NU, law)]


def sphere_composite(n: int = 16, seed: int = 1, law: int = LAW_LINEAR_ELASTIC,
                     distort: float = 0.0) -> Problem:
    """Two-phase RVE: 12 spherical inclusions of radius 0.12, u ~ U[-1e-3, 1e-3] per DOF,
    v ~ U[-1, 1] per DOF (linear elastic by default)."""
    coords, conn = box_mesh(n, distort=distort, seed=seed)
    phase, centres = sphere_phases(coords, conn, seed=seed)
    u = uniform_field(coords.size, 1e-3, seed + 10)
    v = uniform_field(coords.size, 1.0, seed + 20)
    return Problem(f"sphere_rve_{n}^3", coords, conn, phase, composite_materials(law), u, v,
                   meta={"inclusion_fraction": float(phase.mean()), "centres": centres})


def fibre_composite(n: int = 128, seed: int = 2, law: int = LAW_NEO_HOOKEAN) -> Problem:
    """Unidirectional fibre RVE (fibres along z, r = 0.05, 50% target fraction), at a 1%
    uniaxial stretch plus U[-1e-4, 1e-4] noise; v ~ U[-1, 1] per DOF."""
    coords, conn = box_mesh(n)
    centres = fibre_centres(seed=seed)
    phase = fibre_phases(coords, conn, centres)
    u = stretch_state(coords, seed=seed)
    v = uniform_field(coords.size, 1.0, seed + 20)
    return Problem(f"fibre_rve_{n}^3", coords, conn, phase, composite_materials(law), u, v,
                   meta={"fibre_fraction": float(phase.mean()), "n_fibres": len(centres)})


def lognormal_problem(n: int = 64, seed: int = 4) -> Problem:
    """Linear-elastic n^3 mesh with a lognormal per-element Young's modulus (median
    10 GPa, sigma_log 0.5, 3-voxel blur), nu = 0.3, u ~ U[-1e-3, 1e-3] per DOF."""
    coords, conn = box_mesh(n)
    E = lognormal_modulus(n, seed=seed)
    phase = np.zeros(len(conn), dtype=np.int32)
    u = uniform_field(coords.size, 1e-3, seed + 10)
    v = uniform_field(coords.size, 1.0, seed + 20)
    return Problem(f"lognormal_E_{n}^3", coords, conn, phase, [(1.0e10, 0.3, LAW_LINEAR_ELASTIC)],
                   u, v, E_elem=E)


def roller_bcs(coords: np.ndarray, stretch: float = 0.01, tol: float = 1e-12):
    """Uniaxial-stretch Dirichlet set: u1 = 0 on X1 = 0, u1 = stretch on X1 = 1, u2 = 0 on
    X2 = 0, u3 = 0 on X3 = 0 (rollers).  Returns (dofs int64, values float64)."""
    x = coords
    dofs, vals = [], []
    for n in np.where(np.abs(x[:, 0]) < tol)[0]:
        dofs.append(3 * n); vals.append(0.0)
    for n in np.where(np.abs(x[:, 0] - 1.0) < tol)[0]:
        dofs.append(3 * n); vals.append(stretch)
    for n in np.where(np.abs(x[:, 1]) < tol)[0]:
        dofs.append(3 * n + 1); vals.append(0.0)
    for n in np.where(np.abs(x[:, 2]) < tol)[0]:
        dofs.append(3 * n + 2); vals.append(0.0)
    return np.array(dofs, dtype=np.int64), np.array(vals, dtype=np.float64)


# Named, seed-pinned workloads.  Each entry gives the problem (mesh, phases, materials, u, v and,
# for the adjoint workload, E_elem), the precision(s) the workload is run in, and, for the
# surrogate workload, how its training set is drawn.  Calling a preset builds its inputs.
PRESETS = {
    "sphere16_linear": dict(
        build=lambda: sphere_composite(16, seed=1, law=LAW_LINEAR_ELASTIC),
        precisions=("fp64",),
        about="16^3 two-phase sphere RVE (12 inclusions, r = 0.12), linear elastic, u ~ U[+-1e-3]"),
    "fibre128_neohookean": dict(
        build=lambda: fibre_composite(128, seed=2, law=LAW_NEO_HOOKEAN),
        precisions=("fp64",),
        about="128^3 unidirectional fibre RVE (r = 0.05, 50%), neo-Hookean, 1% stretch + 1e-4 noise"),
    "fibre128_mixed_precision": dict(
        build=lambda: fibre_composite(128, seed=2, law=LAW_NEO_HOOKEAN),
        precisions=("fp32", "tf32"),
        about="the 128^3 fibre RVE with FP32 / TF32 element arithmetic, FP64 residual scatter and norm"),
    "lognormal64_adjoint": dict(
        build=lambda: lognormal_problem(64, seed=4),
        precisions=("fp64", "fp32"),
        about="64^3 linear elastic, lognormal E (median 10 GPa, sigma_log 0.5, 3-voxel blur), dL/dE"),
    "fibre128_surrogate": dict(
        build=lambda: fibre_composite(128, seed=2, law=LAW_NEO_HOOKEAN),
        precisions=("surrogate",),
        training=lambda: strain_samples(1 << 20, seed=5),
        about="the 128^3 fibre RVE with the MLP surrogate trained on 2^20 strains |E_ij| <= 0.05"),
}


def preset(name: str) -> Problem:
    """Builds the inputs of a named workload (PRESETS)."""
    if name not in PRESETS:
        raise KeyError(f"unknown preset {name!r}; known: {sorted(PRESETS)}")
    return PRESETS[name]["build"]()
