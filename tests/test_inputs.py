"""The named workloads: each preset exists, documents itself and rebuilds identically from its
seed (the inputs every test, the bench and the oracle share)."""
import numpy as np

from paper_2604_22087_b300 import inputs as I


def test_presets_are_named_and_documented():
    assert set(I.PRESETS) == {"sphere16_linear", "fibre128_neohookean", "fibre128_mixed_precision",
                              "lognormal64_adjoint", "fibre128_surrogate"}
    for name, p in I.PRESETS.items():
        assert callable(p["build"]) and p["precisions"] and p["about"], name
    assert callable(I.PRESETS["fibre128_surrogate"]["training"])


def test_preset_is_seed_pinned():
    a, b = I.preset("sphere16_linear"), I.preset("sphere16_linear")
    assert (a.n_elem, a.n_nodes, a.n_dof) == (4096, 4913, 14739)
    for x, y in ((a.coords, b.coords), (a.conn, b.conn), (a.phase, b.phase), (a.u, b.u), (a.v, b.v)):
        assert np.array_equal(x, y)
    assert 0.0 < a.meta["inclusion_fraction"] < 1.0
    # another seed draws other inclusions
    c = I.sphere_composite(16, seed=2)
    assert not np.array_equal(a.phase, c.phase)


def test_fibre_placement_is_a_valid_hard_disk_packing():
    """64 fibres of r = 0.05 (the smallest count reaching 50% area), pairwise periodic centre
    distances >= 2r after the Metropolis sweeps, and the same centres for the same seed."""
    c = I.fibre_centres(seed=2)
    assert c.shape == (64, 2) and 64 * np.pi * 0.05 ** 2 >= 0.5 > 63 * np.pi * 0.05 ** 2
    d = c[:, None, :] - c[None, :, :]
    d -= np.round(d)
    r2 = np.sum(d * d, axis=2) + np.eye(64) * 1e9
    assert np.min(r2) >= (2 * 0.05) ** 2 * (1 - 1e-12)
    assert np.array_equal(c, I.fibre_centres(seed=2))
    assert np.all((c >= 0) & (c < 1))


def test_fibre_phases_realise_about_half_by_voxels():
    coords, conn = I.box_mesh(64, 64, 1)
    ph = I.fibre_phases(coords, conn, I.fibre_centres(seed=2))
    assert abs(ph.mean() - 0.5) < 0.02


def test_lognormal_field_moments_and_correlation():
    """E = median exp(sigma z) with z re-standardised: mean of ln E is ln(median) and its standard
    deviation sigma_log, both exactly up to rounding; the 3-voxel blur makes neighbours strongly
    correlated."""
    n = 24
    E = I.lognormal_modulus(n, seed=4)
    lz = np.log(E)
    assert abs(lz.mean() - np.log(1e10)) < 1e-9 and abs(lz.std() - 0.5) < 1e-9
    z = lz.reshape(n, n, n)
    a, b = z[:, :, :-1].ravel(), z[:, :, 1:].ravel()
    assert np.corrcoef(a, b)[0, 1] > 0.8


def test_stretch_state_and_strain_samples():
    coords, _ = I.box_mesh(4)
    u = I.stretch_state(coords, 0.01, 1e-4, seed=2).reshape(-1, 3)
    base = np.zeros_like(u)
    base[:, 0] = 0.01 * coords[:, 0]
    assert np.max(np.abs(u - base)) <= 1e-4
    E6, ph = I.strain_samples(4096, seed=5)
    assert E6.shape == (4096, 6) and np.max(np.abs(E6)) <= 0.05
    assert set(np.unique(ph)) == {0, 1} and abs(ph.mean() - 0.5) < 0.05
