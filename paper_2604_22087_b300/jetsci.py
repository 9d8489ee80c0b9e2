"""Thin Python binding of libjetsci (ctypes): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts torch tensors
to raw pointers and the current CUDA stream, checks shapes/dtypes/devices, and turns
status codes into exceptions.  There is no CPU path: if the compiled library is missing
or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libjetsci.so")

FP64, FP32, TF32, SURROGATE, DF64 = 0, 1, 2, 3, 4
LINEAR_ELASTIC, NEO_HOOKEAN = 0, 1
MATRIX_FREE, CSR = 0, 1
FLAG_BAD_ELEMENT, FLAG_BAD_STATE, FLAG_NONFINITE = 0x1, 0x2, 0x4

_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_MESH", 5: "ERR_NONFINITE",
           6: "ERR_NOT_CONVERGED", 7: "ERR_UNSUPPORTED"}

# Names the C ABI exports (include/jetsci.h); checked by the CPU tests.
EXPORTS = [
    "jetsci_mesh_create", "jetsci_mesh_destroy", "jetsci_mesh_info", "jetsci_mesh_check",
    "jetsci_mesh_copy_pattern", "jetsci_mesh_validate", "jetsci_selftest_bounded_wait",
    "jetsci_residual", "jetsci_tangent_csr", "jetsci_apply_tangent", "jetsci_material_grad",
    "jetsci_assemble_element_blocks", "jetsci_norm2", "jetsci_norm2_static", "jetsci_last_error",
    "jetsci_version",
]


class JetsciError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Material(C.Structure):
    _fields_ = [("E", C.c_double), ("nu", C.c_double), ("law", C.c_int32), ("reserved", C.c_int32)]


_vp = C.c_void_p


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libjetsci.so not built ({LIB_PATH}); run paper_2604_22087_b300.build.build()")
    lib = C.CDLL(LIB_PATH)
    i64, i32 = C.c_int64, C.c_int32
    sig = {
        "jetsci_mesh_create": [_vp, i64, _vp, i64, _vp, C.POINTER(Material), i32, _vp, C.POINTER(_vp)],
        "jetsci_mesh_destroy": [_vp],
        "jetsci_mesh_info": [_vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(_vp), C.POINTER(_vp),
                             C.POINTER(i32)],
        "jetsci_mesh_check": [_vp, C.POINTER(C.c_uint32)],
        "jetsci_mesh_copy_pattern": [_vp, _vp, _vp, _vp],
        "jetsci_mesh_validate": [_vp, C.POINTER(C.c_uint64), _vp],
        "jetsci_residual": [_vp, _vp, _vp, i32, _vp, _vp],
        "jetsci_tangent_csr": [_vp, _vp, _vp, _vp, i32, _vp, _vp],
        "jetsci_apply_tangent": [_vp, _vp, _vp, _vp, i32, _vp, i32, _vp, _vp],
        "jetsci_material_grad": [_vp, _vp, _vp, _vp, _vp, i32, _vp],
        "jetsci_assemble_element_blocks": [_vp, _vp, _vp, i32, _vp],
        "jetsci_norm2": [_vp, _vp, i64, _vp, _vp],
        "jetsci_norm2_static": [_vp, i64, _vp, _vp],
        "jetsci_selftest_bounded_wait": [C.c_uint32, i32, C.POINTER(C.c_uint32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    lib.jetsci_last_error.restype = C.c_char_p
    lib.jetsci_version.restype = C.c_char_p
    return lib


lib = _load()


def _check(st):
    if st != 0:
        raise JetsciError(st, lib.jetsci_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_f64(t, n, name):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
            and t.numel() == n):
        raise ValueError(f"{name}: need a contiguous CUDA float64 tensor of {n} entries")
    return t


def vals_dtype(precision):
    return torch.float64 if precision in (FP64, DF64) else torch.float32


class Mesh:
    """A hex8 mesh on the current CUDA device (wraps jetsci_mesh)."""

    def __init__(self, coords, conn, phase, materials, stream=None):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        conn = np.ascontiguousarray(conn, dtype=np.int32)
        phase = None if phase is None else np.ascontiguousarray(phase, dtype=np.int32)
        mats = (Material * len(materials))(*[Material(float(E), float(nu), int(law), 0)
                                             for E, nu, law in materials])
        h = C.c_void_p()
        _check(lib.jetsci_mesh_create(coords.ctypes.data, coords.shape[0], conn.ctypes.data, conn.shape[0],
                                      None if phase is None else phase.ctypes.data, mats, len(materials),
                                      _stream(stream), C.byref(h)))
        self._h = h
        self.n_nodes, self.n_elem = int(coords.shape[0]), int(conn.shape[0])
        nd, nnz, rp, cp, nc = C.c_int64(), C.c_int64(), C.c_void_p(), C.c_void_p(), C.c_int32()
        _check(lib.jetsci_mesh_info(h, C.byref(nd), C.byref(nnz), C.byref(rp), C.byref(cp), C.byref(nc)))
        self.n_dof, self.nnz, self.n_colours = nd.value, nnz.value, nc.value
        self._rowptr_ptr, self._col_ptr = rp.value, cp.value
        self.device = torch.cuda.current_device()
        # counts the residual calls given E_elem: each replaces the element vectors the library
        # keeps for material_grad(None, ...), so MaterialGrad can tell whether its own are current
        self.residual_with_E_calls = 0

    @classmethod
    def of(cls, problem, stream=None):
        return cls(problem.coords, problem.conn, problem.phase, problem.materials, stream)

    def close(self):
        if getattr(self, "_h", None):
            lib.jetsci_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def pattern(self, device="cuda", stream=None):
        """Copies of the CSR pattern (rowptr int64 [n_dof+1], col int32 [nnz])."""
        pin = device == "cpu"
        rp = torch.empty(self.n_dof + 1, dtype=torch.int64, device=device, pin_memory=pin)
        col = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=device, pin_memory=pin)
        _check(lib.jetsci_mesh_copy_pattern(self._h, _ptr(rp), _ptr(col), _stream(stream)))
        return rp, col[:self.nnz]

    def check(self):
        """Reads and clears the device flag word; raises JetsciError if any bit was set."""
        f = C.c_uint32()
        st = lib.jetsci_mesh_check(self._h, C.byref(f))
        if st != 0 and st != 5:
            _check(st)
        return f.value

    def validate(self, stream=None, raise_on_fail=True):
        """Device check of the creation-time assembly data; returns the violation counts
        {node_ids, colouring, slot_map, first_writers} (all 0 for a valid mesh).  Any nonzero
        count raises JetsciError (JETSCI_ERR_MESH) unless raise_on_fail is False."""
        c = (C.c_uint64 * 4)()
        st = lib.jetsci_mesh_validate(self._h, c, _stream(stream))
        counts = dict(zip(("node_ids", "colouring", "slot_map", "first_writers"), [int(x) for x in c]))
        if st != 0 and (raise_on_fail or st != 4):
            _check(st)
        return counts

    # ------------------------------------------------------------------ compute calls
    def new_vector(self):
        return torch.empty(self.n_dof, dtype=torch.float64, device="cuda")

    def new_values(self, precision=FP64):
        return torch.empty(self.nnz, dtype=vals_dtype(precision), device="cuda")

    def residual(self, u, R=None, precision=FP64, E_elem=None, stream=None):
        _dev_f64(u, self.n_dof, "u")
        R = self.new_vector() if R is None else _dev_f64(R, self.n_dof, "R")
        _dev_f64(E_elem, self.n_elem, "E_elem")
        _check(lib.jetsci_residual(self._h, _ptr(u), _ptr(R), precision, _ptr(E_elem), _stream(stream)))
        if E_elem is not None:
            self.residual_with_E_calls += 1
        return R

    def tangent_csr(self, u, vals=None, R=None, precision=FP64, E_elem=None, stream=None):
        _dev_f64(u, self.n_dof, "u")
        vals = self.new_values(precision) if vals is None else vals
        if vals.dtype != vals_dtype(precision) or vals.numel() != self.nnz or not vals.is_cuda:
            raise ValueError("vals: wrong dtype/size/device for this precision")
        _dev_f64(R, self.n_dof, "R")
        _dev_f64(E_elem, self.n_elem, "E_elem")
        _check(lib.jetsci_tangent_csr(self._h, _ptr(u), _ptr(vals), _ptr(R), precision, _ptr(E_elem),
                                      _stream(stream)))
        return vals

    def assemble_blocks(self, Ke, vals=None, stream=None):
        """CSR values sum_e P_e^T K_e P_e from caller-formed element blocks Ke [n_elem][24][24]
        (float64 -> FP64 values, float32 -> FP32 values)."""
        if Ke.dtype not in (torch.float64, torch.float32) or not Ke.is_cuda or not Ke.is_contiguous() \
                or tuple(Ke.shape) != (self.n_elem, 24, 24):
            raise ValueError("Ke: contiguous CUDA float64/float32 tensor of shape [n_elem, 24, 24] expected")
        precision = FP64 if Ke.dtype == torch.float64 else FP32
        vals = self.new_values(precision) if vals is None else vals
        if vals.dtype != Ke.dtype or vals.numel() != self.nnz or not vals.is_cuda:
            raise ValueError("vals: wrong dtype/size/device")
        _check(lib.jetsci_assemble_element_blocks(self._h, _ptr(Ke), _ptr(vals), precision, _stream(stream)))
        return vals

    def apply_tangent(self, u, v, y=None, mode=MATRIX_FREE, vals=None, precision=FP64, E_elem=None,
                      stream=None):
        _dev_f64(v, self.n_dof, "v")
        if mode == MATRIX_FREE:
            _dev_f64(u, self.n_dof, "u")
        y = self.new_vector() if y is None else _dev_f64(y, self.n_dof, "y")
        if mode == CSR and (vals is None or vals.dtype != vals_dtype(precision) or vals.numel() != self.nnz):
            raise ValueError("vals: wrong dtype/size for CSR mode")
        _dev_f64(E_elem, self.n_elem, "E_elem")
        _check(lib.jetsci_apply_tangent(self._h, _ptr(u), _ptr(v), _ptr(y), mode, _ptr(vals), precision,
                                        _ptr(E_elem), _stream(stream)))
        return y

    def material_grad(self, u, R, E_elem=None, g=None, precision=FP64, stream=None):
        """dL/dE_e for L = 1/2 ||R||^2.  u=None: at the state of the last residual call given
        E_elem (the same tensor and precision), from the element vectors that call kept."""
        if u is not None:
            _dev_f64(u, self.n_dof, "u")
        _dev_f64(R, self.n_dof, "R")
        _dev_f64(E_elem, self.n_elem, "E_elem")
        g = torch.empty(self.n_elem, dtype=torch.float64, device="cuda") if g is None else g
        _check(lib.jetsci_material_grad(self._h, _ptr(u), _ptr(E_elem), _ptr(R), _ptr(g), precision,
                                        _stream(stream)))
        return g

    def norm2(self, x, out=None, stream=None):
        if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
            raise ValueError("x: need a contiguous CUDA float64 tensor")
        out = torch.empty(1, dtype=torch.float64, device="cuda") if out is None else out
        _check(lib.jetsci_norm2(self._h, _ptr(x), x.numel(), _ptr(out), _stream(stream)))
        return out


def selftest_bounded_wait(max_iter, arrive):
    """Runs the tensor-core kernels' bounded mbarrier wait on a barrier that one arrival
    completes (arrive=True) or that nothing completes; True if the wait ran out."""
    out = C.c_uint32(0)
    _check(lib.jetsci_selftest_bounded_wait(int(max_iter), 1 if arrive else 0, C.byref(out)))
    return bool(out.value)


def version():
    return lib.jetsci_version().decode()


class MaterialGrad(torch.autograd.Function):
    """L(E) = 1/2 ||R(u; E)||^2 with dL/dE from the library's adjoint kernel.

    forward(mesh, u, E, precision) -> L (0-dim float64 CUDA tensor).  The backward pass uses the
    element vectors its forward residual kept when no other residual call given E_elem went
    through Mesh.residual on the same mesh in between, and recomputes them from u otherwise.
    Residual calls made on the mesh's handle directly through the C ABI are not seen: mix them
    with this Function only when each backward follows its own forward."""

    @staticmethod
    def forward(ctx, E, mesh, u, precision=FP64):
        Ed = E.detach().contiguous()
        R = mesh.residual(u, precision=precision, E_elem=Ed)
        nrm = mesh.norm2(R)
        ctx.mesh, ctx.precision, ctx.calls = mesh, precision, mesh.residual_with_E_calls
        ctx.save_for_backward(E, u, R, Ed)
        return 0.5 * nrm[0] * nrm[0]

    @staticmethod
    def backward(ctx, gout):
        E, u, R, Ed = ctx.saved_tensors
        # the element vectors kept by this forward's residual call, unless another residual call
        # with E_elem has replaced them since; then the gradient pass recomputes them from u
        kept = ctx.mesh.residual_with_E_calls == ctx.calls
        g = ctx.mesh.material_grad(None if kept else u, R, E_elem=Ed, precision=ctx.precision)
        return g * gout, None, None, None


# ---------------------------------------------------------------------- MLP surrogate
MLP_PARAMS = 9286


class SurrogateConfig(C.Structure):
    _fields_ = [("in_scale", C.c_double), ("range", C.c_double), ("out_scale", C.c_double * 12),
                ("out_shift", C.c_double * 12)]


def _load_surrogate(lib):
    i64, i32 = C.c_int64, C.c_int32
    sig = {
        "jetsci_surrogate_create": [_vp, C.POINTER(SurrogateConfig), _vp, C.POINTER(_vp)],
        "jetsci_surrogate_destroy": [_vp],
        "jetsci_surrogate_get_params": [_vp, _vp],
        "jetsci_surrogate_label": [C.POINTER(Material), i32, _vp, _vp, i64, _vp, _vp, _vp],
        "jetsci_surrogate_train": [_vp, _vp, _vp, _vp, i64, _vp, i64, i64, i32, C.c_double, C.c_double, _vp, _vp],
        "jetsci_surrogate_gradient": [_vp, _vp, _vp, _vp, i64, _vp, i32, _vp, _vp, _vp],
        "jetsci_surrogate_eval": [_vp, _vp, _vp, i64, _vp, _vp, _vp],
        "jetsci_mesh_set_surrogate": [_vp, _vp],
        "jetsci_mesh_surrogate_fallbacks": [_vp, C.POINTER(C.c_uint32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int


_load_surrogate(lib)
EXPORTS += ["jetsci_surrogate_create", "jetsci_surrogate_destroy", "jetsci_surrogate_get_params",
            "jetsci_surrogate_label", "jetsci_surrogate_train", "jetsci_surrogate_gradient",
            "jetsci_surrogate_eval", "jetsci_mesh_set_surrogate", "jetsci_mesh_surrogate_fallbacks"]


def pack_layers(layers):
    """[(W [out,in], b [out])] * 4 -> flat FP64 parameter vector in the library's order."""
    parts = []
    for W, b in layers:
        parts += [np.asarray(W, dtype=np.float64).ravel(), np.asarray(b, dtype=np.float64).ravel()]
    p = np.concatenate(parts)
    if p.size != MLP_PARAMS:
        raise ValueError(f"expected {MLP_PARAMS} parameters, got {p.size}")
    return p


def unpack_layers(p):
    p = np.asarray(p, dtype=np.float64)
    shapes = [(64, 8), (64, 64), (64, 64), (6, 64)]
    out, o = [], 0
    for r, c in shapes:
        W = p[o:o + r * c].reshape(r, c)
        o += r * c
        b = p[o:o + r]
        o += r
        out.append((W.copy(), b.copy()))
    return out


def _dev(t, dtype, n, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == n):
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor of {n} entries")
    return t


class Surrogate:
    """The MLP surrogate on the current CUDA device (wraps jetsci_surrogate)."""

    def __init__(self, layers, in_scale, range_, out_scale, out_shift, stream=None):
        cfg = SurrogateConfig()
        cfg.in_scale, cfg.range = float(in_scale), float(range_)
        cfg.out_scale[:] = [float(v) for v in np.asarray(out_scale, dtype=np.float64).ravel()]
        cfg.out_shift[:] = [float(v) for v in np.asarray(out_shift, dtype=np.float64).ravel()]
        self.cfg = cfg
        p = np.ascontiguousarray(pack_layers(layers) if isinstance(layers, (list, tuple)) else layers,
                                 dtype=np.float64)
        h = C.c_void_p()
        _check(lib.jetsci_surrogate_create(p.ctypes.data, C.byref(cfg), _stream(stream), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib.jetsci_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def params(self):
        p = np.zeros(MLP_PARAMS)
        _check(lib.jetsci_surrogate_get_params(self._h, p.ctypes.data))
        return p

    def layers(self):
        return unpack_layers(self.params())

    def save(self, path, **meta):
        """Checkpoint as .npz: the parameters (FP64 copy of the library's weights), the input
        scale, the fallback range and the per-phase output scalings, plus any metadata given
        (for example the training seed and step count).  Surrogate.load restores it."""
        np.savez(path, params=self.params(), in_scale=self.cfg.in_scale, range=self.cfg.range,
                 out_scale=np.array(self.cfg.out_scale[:]), out_shift=np.array(self.cfg.out_shift[:]), **meta)

    @classmethod
    def load(cls, path, stream=None):
        """A surrogate on the current CUDA device from a checkpoint written by save()."""
        z = np.load(path)
        return cls(z["params"], float(z["in_scale"]), float(z["range"]), z["out_scale"], z["out_shift"],
                   stream=stream)

    @staticmethod
    def label(materials, E6, phase, stream=None):
        n = phase.numel()
        _dev(E6, torch.float64, 6 * n, "E6")
        _dev(phase, torch.int32, n, "phase")
        mats = (Material * len(materials))(*[Material(float(E), float(nu), int(law), 0) for E, nu, law in materials])
        S6 = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        _check(lib.jetsci_surrogate_label(mats, len(materials), _ptr(E6), _ptr(phase), n, _ptr(S6), _ptr(err),
                                          _stream(stream)))
        if int(err.item()) != 0:
            raise JetsciError(5, f"label error flags {int(err.item())}")
        return S6

    def train(self, E6, phase, S6, order, n_steps, batch=4096, lr_max=1e-3, lr_min=1e-5, stream=None):
        n = phase.numel()
        _dev(E6, torch.float64, 6 * n, "E6")
        _dev(S6, torch.float64, 6 * n, "S6")
        _dev(phase, torch.int32, n, "phase")
        _dev(order, torch.int32, order.numel(), "order")
        loss = torch.empty(max(n_steps, 1), dtype=torch.float32, device="cuda")
        _check(lib.jetsci_surrogate_train(self._h, _ptr(E6), _ptr(phase), _ptr(S6), n, _ptr(order), order.numel(),
                                          n_steps, batch, lr_max, lr_min, _ptr(loss), _stream(stream)))
        return loss[:n_steps]

    def gradient(self, E6, phase, S6, order, batch, stream=None):
        n = phase.numel()
        grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        _check(lib.jetsci_surrogate_gradient(self._h, _ptr(E6), _ptr(phase), _ptr(S6), n, _ptr(order), batch,
                                             _ptr(grad), _ptr(loss), _stream(stream)))
        return grad, loss

    def eval(self, E6, phase, tangent=True, stream=None):
        n = phase.numel()
        _dev(E6, torch.float64, 6 * n, "E6")
        _dev(phase, torch.int32, n, "phase")
        S6 = torch.empty(n, 6, dtype=torch.float64, device="cuda")
        D = torch.empty(n, 6, 6, dtype=torch.float64, device="cuda") if tangent else None
        _check(lib.jetsci_surrogate_eval(self._h, _ptr(E6), _ptr(phase), n, _ptr(S6), _ptr(D), _stream(stream)))
        return (S6, D) if tangent else S6


def surrogate_fallbacks(mesh):
    c = C.c_uint32()
    _check(lib.jetsci_mesh_surrogate_fallbacks(mesh.handle, C.byref(c)))
    return c.value


def attach_surrogate(mesh, surrogate):
    _check(lib.jetsci_mesh_set_surrogate(mesh.handle, None if surrogate is None else surrogate.handle))
    mesh._surrogate = surrogate  # keep it alive while attached


# ---------------------------------------------------------------------- Newton driver
class NewtonInfo(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("cg_iters_total", C.c_int32), ("cg_capped", C.c_int32),
                ("reserved", C.c_int32), ("final_rel_residual", C.c_double), ("residual_history", C.c_double * 32),
                ("seconds_residual", C.c_double), ("seconds_tangent", C.c_double), ("seconds_solve", C.c_double)]


lib.jetsci_newton_solve.argtypes = [_vp, _vp, C.c_int64, _vp, _vp, C.c_int32, C.c_double, C.c_int32, C.c_double,
                                    C.c_int32, _vp, C.POINTER(NewtonInfo)]
lib.jetsci_newton_solve.restype = C.c_int
EXPORTS += ["jetsci_newton_solve"]


def newton_solve(mesh, u, bc_dofs, bc_vals, tangent_precision=FP64, rtol=1e-10, max_newton=20, cg_rtol=1e-8,
                 max_cg=20000, stream=None, raise_on_fail=True):
    """Newton + Jacobi-CG on the device; u (CUDA float64) is updated in place.  Returns NewtonInfo."""
    _dev_f64(u, mesh.n_dof, "u")
    d = torch.as_tensor(np.ascontiguousarray(bc_dofs, dtype=np.int64)).cuda()
    v = torch.as_tensor(np.ascontiguousarray(bc_vals, dtype=np.float64)).cuda()
    info = NewtonInfo()
    st = lib.jetsci_newton_solve(mesh.handle, _ptr(u), d.numel(), _ptr(d), _ptr(v), tangent_precision, rtol,
                                 max_newton, cg_rtol, max_cg, _stream(stream), C.byref(info))
    if st != 0 and (raise_on_fail or st != 6):
        _check(st)
    return info
