"""The allocation-free norm entry point, jetsci_norm2_static, called through the C ABI.

It exists for callers that cannot allocate device memory when they need the norm (their
memory is reserved up front by another runtime's pool, or cudaMalloc's implicit device
synchronisation is not acceptable in their loop).  Its scratch is a fixed device array
inside the library, shared by every call.  This file is collected last so that a run that
stops at the first failure has already run every other test; it must also pass alone in a
fresh process.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

LIMIT = 4096 * 8192  # entries the static scratch can reduce


def _lib():
    from paper_2604_22087_b300 import jetsci as J
    return J


def _static_norm(J, x):
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    J._check(J.lib.jetsci_norm2_static(J._ptr(x), x.numel(), J._ptr(out), J._stream()))
    return out


def test_static_norm_matches_mesh_norm_on_two_calls_in_a_row():
    from paper_2604_22087_b300 import inputs as I
    J = _lib()
    coords, conn = I.box_mesh(3)
    mesh = J.Mesh(coords, conn, None, [(1e9, 0.3, 0)])
    g = torch.Generator(device="cuda").manual_seed(7)
    # a long vector (many partials) then a short one: the second call must not see the
    # first call's leftover partial sums
    x1 = torch.rand(5_000_003, dtype=torch.float64, device="cuda", generator=g) - 0.5
    x2 = torch.rand(12_345, dtype=torch.float64, device="cuda", generator=g) * 3.0
    for x in (x1, x2):
        ref = mesh.norm2(x).item()
        got = _static_norm(J, x).item()
        assert abs(got - ref) <= 1e-14 * ref
    # two calls in a row on the same input give the same value
    a, b = _static_norm(J, x1).item(), _static_norm(J, x1).item()
    assert a == b == pytest.approx(mesh.norm2(x1).item(), rel=1e-14)
    torch.cuda.synchronize()
    mesh.close()


def test_static_norm_edge_sizes_and_limit():
    J = _lib()
    empty = torch.empty(0, dtype=torch.float64, device="cuda")
    assert _static_norm(J, empty).item() == 0.0
    one = torch.tensor([-3.0], dtype=torch.float64, device="cuda")
    assert _static_norm(J, one).item() == 3.0
    # beyond the limit: rejected on the host before any launch (the buffer is never read)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    st = J.lib.jetsci_norm2_static(J._ptr(one), LIMIT + 1, J._ptr(out), J._stream())
    assert st == 1
    assert b"exceeds the static scratch limit" in J.lib.jetsci_last_error()
