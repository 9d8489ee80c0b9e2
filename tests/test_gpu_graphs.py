"""The library's calls inside CUDA graphs: every call is asynchronous on the caller's stream and
needs no host synchronisation, so a whole step (tangent with fused R, matrix-free and CSR
products, norm) can be captured once and replayed.  A replay must reproduce direct calls
bit for bit.  The row-gather assembly's workspace is allocated by the first call of a mesh;
that call cannot be captured, and inside a capture it is refused with JETSCI_ERR_ARG (on the
host, before any launch).
"""
import numpy as np
import pytest
import torch

from paper_2604_22087_b300 import inputs as I

pytestmark = pytest.mark.gpu


def jetsci():
    from paper_2604_22087_b300 import jetsci as J
    return J


@pytest.fixture(scope="module")
def problem():
    return I.sphere_composite(12, seed=1, law=I.LAW_NEO_HOOKEAN)


def _step(J, mesh, u, v, vals, R, y_mf, y_csr, nrm, precision):
    mesh.tangent_csr(u, vals=vals, R=R, precision=precision)
    mesh.apply_tangent(u, v, y=y_mf, precision=precision)
    mesh.apply_tangent(None, v, y=y_csr, mode=J.CSR, vals=vals, precision=precision)
    mesh.norm2(R, out=nrm)


@pytest.mark.parametrize("name", ["FP64", "FP32", "TF32", "DF64"])
def test_captured_step_replays_bitwise(problem, name):
    J = jetsci()
    p = getattr(J, name)
    mesh = J.Mesh.of(problem)
    u = torch.as_tensor(problem.u).cuda()
    v = torch.as_tensor(problem.v).cuda()

    def buffers():
        return (mesh.new_values(p), mesh.new_vector(), mesh.new_vector(), mesh.new_vector(),
                torch.empty(1, dtype=torch.float64, device="cuda"))

    ref = buffers()
    _step(J, mesh, u, v, *ref, p)  # direct calls (and the first call of the mesh for FP32)
    torch.cuda.synchronize()
    out = buffers()
    for t in out:
        t.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g):
            _step(J, mesh, u, v, *out, p)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    # a replay after the input changed follows the new input
    u.mul_(0.5)
    g.replay()
    direct = buffers()
    _step(J, mesh, u, v, *direct, p)
    torch.cuda.synchronize()
    for a, b in zip(direct, out):
        assert torch.equal(a, b)
    assert mesh.check() == 0
    mesh.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")  # nothing is launched before the refusal
def test_first_row_gather_call_inside_capture_is_refused(problem):
    J = jetsci()
    mesh = J.Mesh.of(problem)  # fresh mesh: no workspace yet
    u = torch.as_tensor(problem.u).cuda()
    vals = mesh.new_values(J.FP32)
    R = mesh.new_vector()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with pytest.raises(J.JetsciError) as ei:
            with torch.cuda.graph(g):
                mesh.tangent_csr(u, vals=vals, R=R, precision=J.FP32)
    assert ei.value.status == 1
    assert "capturing" in str(ei.value)
    torch.cuda.synchronize()
    # outside a capture the same call allocates the workspace and works
    mesh.tangent_csr(u, vals=vals, R=R, precision=J.FP32)
    torch.cuda.synchronize()
    assert np.isfinite(vals.cpu().numpy()).all()
    mesh.close()
