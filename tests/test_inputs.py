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
