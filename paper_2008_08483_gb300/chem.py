"""Thin Python binding of the C ABI in include/chem.h (argument marshalling only).

Every computation runs in the CUDA library libchemgb300.so; this module only
converts arguments.  It raises ChemError if the library has not been built: there
is no fallback path.  PyTorch provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libchemgb300.so")

FP64, FP32, SPLIT_BF16 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "split_bf16": SPLIT_BF16}

STATUS = {0: "CHEM_OK", 1: "CHEM_EINVAL", 2: "CHEM_ENOMEM", 3: "CHEM_ECUDA",
          4: "CHEM_EUNSUPPORTED", 5: "CHEM_EBUSY", 6: "CHEM_ETIMEOUT", 7: "CHEM_ENOTREADY",
          8: "CHEM_ENONCONV"}

_lock = threading.Lock()
_lib = None


class ChemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("n_reactions", C.c_int32), ("n_elements", C.c_int32),
                ("elem_comp", C.c_void_p), ("mol_weight", C.c_void_p), ("nu_f", C.c_void_p),
                ("nu_r", C.c_void_p), ("arrh", C.c_void_p), ("kind", C.c_void_p),
                ("reversible", C.c_void_p), ("eff", C.c_void_p), ("arrh_low", C.c_void_p),
                ("troe", C.c_void_p), ("nasa7", C.c_void_p), ("t_mid", C.c_double),
                ("p_ref", C.c_double)]


class _KcAnnDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("n_hidden", C.c_int32), ("activation", C.c_int32),
                ("x_mean", C.c_float), ("x_std", C.c_float), ("w_in", C.c_void_p),
                ("b_in", C.c_void_p), ("w_hid", C.c_void_p), ("b_hid", C.c_void_p),
                ("w_out", C.c_void_p), ("b_out", C.c_void_p), ("y_mean", C.c_void_p),
                ("y_std", C.c_void_p)]


class _IntegOpts(C.Structure):
    _fields_ = [("h_init", C.c_double), ("h_min", C.c_double), ("h_max", C.c_double),
                ("max_steps", C.c_int64), ("ign_dT", C.c_double), ("t_ign", C.c_void_p),
                ("n_accepted", C.c_void_p), ("n_rejected", C.c_void_p),
                ("fixed_steps", C.c_int32), ("jacobian_fp32", C.c_int32)]


CELL_OK, CELL_STEP_UNDERFLOW, CELL_MAX_STEPS, CELL_NONFINITE = 0, 1, 2, 3
REQ_SOURCE, REQ_INTEGRATE = 0, 1


class _Request(C.Structure):
    _fields_ = [("mech_index", C.c_int32), ("kind", C.c_int32), ("precision", C.c_int),
                ("fixed_steps", C.c_int32), ("n_cells", C.c_int64), ("T", C.c_void_p),
                ("P", C.c_void_p), ("Y", C.c_void_p), ("omega", C.c_void_p),
                ("T_out", C.c_void_p), ("Y_out", C.c_void_p), ("cell_status", C.c_void_p),
                ("dt", C.c_double), ("rtol", C.c_double), ("atol", C.c_double)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int), ("batch_requests", C.c_int32), ("n_cells", C.c_int64),
                ("batch_cells", C.c_int64), ("n_failed", C.c_int32), ("slot", C.c_int32),
                ("queue_us", C.c_double), ("latency_us", C.c_double),
                ("steps_accepted", C.c_int64), ("steps_rejected", C.c_int64)]


class _ServeInfo(C.Structure):
    _fields_ = [("n_slots", C.c_int32), ("slot_cells", C.c_int64), ("device_bytes", C.c_size_t),
                ("submitted", C.c_uint64), ("completed", C.c_uint64), ("batches", C.c_uint64),
                ("graphs_captured", C.c_uint64), ("graph_launches", C.c_uint64),
                ("max_batch_requests", C.c_int32), ("graph_updates", C.c_uint64),
                ("memory_waits", C.c_uint64), ("bytes_in_use", C.c_size_t),
                ("bytes_in_use_max", C.c_size_t), ("source_sms", C.c_int32),
                ("integrate_sms", C.c_int32), ("green_contexts", C.c_int32)]


def lib():
    """The loaded CUDA library (raises ChemError if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ChemError(3, f"CUDA library {LIB_PATH} is not built; run "
                                   "__graft_entry__.build() or paper_2008_08483_gb300/build.py")
            L = C.CDLL(LIB_PATH)
            P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
            L.chem_abi_version.restype = I32
            L.chem_last_error.restype = C.c_char_p
            L.chem_kernel_launch_count.restype = C.c_uint64
            L.chem_mechanism_load.argtypes = [C.POINTER(_Desc), C.POINTER(P)]
            L.chem_mechanism_free.argtypes = [P]
            L.chem_mechanism_info.argtypes = [P, C.POINTER(I32), C.POINTER(I32),
                                              C.POINTER(C.c_size_t)]
            L.chem_source_term.argtypes = [P, I64, P, P, P, I64, P, I64, C.c_int, P]
            L.chem_source_term_host_workspace.argtypes = [P, I64, I64, C.c_int]
            L.chem_source_term_host_workspace.restype = C.c_size_t
            L.chem_source_term_host.argtypes = [P, I64, P, P, P, I64, P, I64, C.c_int, I64, P,
                                                C.c_size_t, P]
            L.chem_device_status.argtypes = [P, C.POINTER(I32)]
            L.chem_source_term_jvp.argtypes = [P, I64, P, P, I64, P, P, P, P, I64, C.c_int, P]
            L.chem_source_term_vjp.argtypes = [P, I64, P, P, I64, P, I64, P, P, C.c_int, P]
            L.chem_source_term_jacobian.argtypes = [P, I64, P, P, I64, P, I64, C.c_int, P]
            for f in (L.chem_source_term_jvp, L.chem_source_term_vjp,
                      L.chem_source_term_jacobian):
                f.restype = C.c_int
            L.chem_ode_rhs.argtypes = [P, I64, P, P, P, I64, P, I64, P]
            L.chem_ode_jacobian.argtypes = [P, I64, P, P, P, I64, P, P]
            L.chem_integrate_cells.argtypes = [P, I64, P, P, P, I64, C.c_double, C.c_double,
                                               C.c_double, C.POINTER(_IntegOpts), P, P]
            L.chem_integrate_cells_noalloc.argtypes = L.chem_integrate_cells.argtypes
            L.chem_integrate_cells_noalloc.restype = C.c_int
            L.chem_rosenbrock_tableau.argtypes = [C.POINTER(I32), P, P, P, P, P]
            L.chem_log_kc.argtypes = [P, I64, P, P, I64, P]
            L.chem_kc_ann_load.argtypes = [P, C.POINTER(_KcAnnDesc), C.POINTER(P)]
            L.chem_kc_ann_free.argtypes = [P]
            L.chem_source_term_kc_ann.argtypes = [P, P, I64, P, P, P, I64, P, I64, P]
            for f in (L.chem_log_kc, L.chem_kc_ann_load, L.chem_kc_ann_free,
                      L.chem_source_term_kc_ann):
                f.restype = C.c_int
            L.chem_serve_create.argtypes = [C.POINTER(P), I32, C.c_size_t, C.POINTER(P)]
            L.chem_serve_submit.argtypes = [P, C.POINTER(_Request), C.POINTER(C.c_uint64)]
            L.chem_serve_poll.argtypes = [P, C.c_uint64, C.POINTER(_Result), I64]
            L.chem_serve_info_get.argtypes = [P, C.POINTER(_ServeInfo)]
            L.chem_serve_destroy.argtypes = [P]
            for f in (L.chem_ode_rhs, L.chem_ode_jacobian, L.chem_integrate_cells,
                      L.chem_rosenbrock_tableau, L.chem_serve_create, L.chem_serve_submit,
                      L.chem_serve_poll, L.chem_serve_info_get, L.chem_serve_destroy):
                f.restype = C.c_int
            for f in (L.chem_mechanism_load, L.chem_mechanism_free, L.chem_mechanism_info,
                      L.chem_source_term, L.chem_source_term_host, L.chem_device_status):
                f.restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise ChemError(rc, lib().chem_last_error().decode(errors="replace"))


def abi_version() -> int:
    return int(lib().chem_abi_version())


def kernel_launch_count() -> int:
    return int(lib().chem_kernel_launch_count())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Mechanism:
    """A mechanism loaded on the current CUDA device (chem_mechanism_load)."""

    def __init__(self, desc):
        keep = dict(
            elem_comp=np.ascontiguousarray(desc.elem_comp, np.int32),
            mol_weight=np.ascontiguousarray(desc.mol_weight, np.float64),
            nu_f=np.ascontiguousarray(desc.nu_f, np.int32),
            nu_r=np.ascontiguousarray(desc.nu_r, np.int32),
            arrh=np.ascontiguousarray(desc.arrh, np.float64),
            kind=np.ascontiguousarray(desc.kind, np.int32),
            reversible=np.ascontiguousarray(desc.reversible, np.int32),
            eff=np.ascontiguousarray(desc.eff, np.float64),
            arrh_low=np.ascontiguousarray(desc.arrh_low, np.float64),
            troe=np.ascontiguousarray(desc.troe, np.float64),
            nasa7=np.ascontiguousarray(desc.nasa7, np.float64),
        )
        ns, nr = keep["nu_f"].shape[1], keep["nu_f"].shape[0]
        ne = keep["elem_comp"].shape[1] if keep["elem_comp"].ndim == 2 else 0
        d = _Desc(ns, nr, ne, *(_ptr(keep[k]).value for k in (
            "elem_comp", "mol_weight", "nu_f", "nu_r", "arrh", "kind", "reversible", "eff",
            "arrh_low", "troe", "nasa7")), float(desc.t_mid), float(desc.p_ref))
        h = C.c_void_p()
        _check(lib().chem_mechanism_load(C.byref(d), C.byref(h)))
        self._h = h
        self.n_species, self.n_reactions = ns, nr

    @property
    def handle(self):
        if self._h is None:
            raise ChemError(1, "mechanism was freed")
        return self._h

    def info(self):
        ns, nr, nb = C.c_int32(), C.c_int32(), C.c_size_t()
        _check(lib().chem_mechanism_info(self.handle, C.byref(ns), C.byref(nr), C.byref(nb)))
        return {"n_species": ns.value, "n_reactions": nr.value, "device_bytes": nb.value}

    def device_status(self) -> int:
        """Nonzero if a tensor-core kernel gave up on a bounded wait (clears it)."""
        v = C.c_int32()
        _check(lib().chem_device_status(self.handle, C.byref(v)))
        return int(v.value)

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(lib().chem_mechanism_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype(precision):
    import torch
    return torch.float64 if precision == FP64 else torch.float32


def source_term(mech: Mechanism, T, P, Y, precision: int = SPLIT_BF16, out=None, stream=None):
    """omega [n, ns] from CUDA tensors T [n], P [n], Y [n, ldY] (chem_source_term)."""
    import torch
    dt = _dtype(precision)
    n = T.shape[0]
    for name, t in (("T", T), ("P", P), ("Y", Y)):
        if not t.is_cuda or t.dtype != dt:
            raise ChemError(1, f"{name} must be a CUDA {dt} tensor")
    if T.stride(0) != 1 or P.stride(0) != 1 or Y.dim() != 2 or Y.stride(1) != 1:
        raise ChemError(1, "T, P must be contiguous and Y row-major with unit column stride")
    if out is None:
        out = torch.empty((n, mech.n_species), dtype=dt, device=T.device)
    _check(lib().chem_source_term(mech.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(),
                                  Y.stride(0), out.data_ptr(), out.stride(0), int(precision),
                                  _stream_ptr(stream)))
    return out


def host_workspace_bytes(mech: Mechanism, chunk_cells: int, ldY: int, precision: int) -> int:
    return int(lib().chem_source_term_host_workspace(mech.handle, chunk_cells, ldY,
                                                     int(precision)))


def source_term_host(mech: Mechanism, T, P, Y, out, precision: int, workspace, chunk_cells: int,
                     stream=None):
    """chem_source_term_host: T, P, Y, out are host tensors (page-locked for overlap),
    workspace a CUDA byte tensor of at least host_workspace_bytes()."""
    n = T.shape[0]
    _check(lib().chem_source_term_host(mech.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(),
                                       Y.stride(0), out.data_ptr(), out.stride(0), int(precision),
                                       int(chunk_cells), workspace.data_ptr(),
                                       workspace.numel() * workspace.element_size(),
                                       _stream_ptr(stream)))
    return out


def _dptr(t):
    return None if t is None else t.data_ptr()


def _check_state(T, lnC, precision):
    dt = _dtype(precision)
    if precision not in (FP64, FP32):
        raise ChemError(4, "derivatives are built for FP64 and FP32")
    for name, t in (("T", T), ("lnC", lnC)):
        if not t.is_cuda or t.dtype != dt:
            raise ChemError(1, f"{name} must be a CUDA {dt} tensor")
    if T.stride(0) != 1 or lnC.dim() != 2 or lnC.stride(1) != 1:
        raise ChemError(1, "T contiguous and lnC row-major with unit column stride")


def source_term_jvp(mech: Mechanism, T, lnC, dT, dlnC, precision: int = FP64, with_omega=True,
                    stream=None):
    """(omega or None, d omega) for the tangent (dT, dlnC) at the state (T, ln C)."""
    import torch
    _check_state(T, lnC, precision)
    n = T.shape[0]
    dT = dT.contiguous()
    dlnC = dlnC if dlnC.stride(1) == 1 and dlnC.stride(0) == lnC.stride(0) else \
        _like_rows(dlnC, lnC)
    dom = torch.empty((n, mech.n_species), dtype=T.dtype, device=T.device)
    om = torch.empty_like(dom) if with_omega else None
    _check(lib().chem_source_term_jvp(mech.handle, n, T.data_ptr(), lnC.data_ptr(), lnC.stride(0),
                                      dT.data_ptr(), dlnC.data_ptr(), _dptr(om), dom.data_ptr(),
                                      dom.stride(0), int(precision), _stream_ptr(stream)))
    return om, dom


def _like_rows(x, ref):
    import torch
    out = torch.zeros((ref.shape[0], ref.stride(0)), dtype=ref.dtype, device=ref.device)
    out[:, :x.shape[1]] = x
    return out[:, :ref.shape[1]]


def source_term_vjp(mech: Mechanism, T, lnC, g_omega, precision: int = FP64, stream=None):
    """(g_T, g_lnC) = (d omega / d(T, ln C))^T g_omega."""
    import torch
    _check_state(T, lnC, precision)
    n = T.shape[0]
    g_omega = g_omega.contiguous()
    gT = torch.empty((n,), dtype=T.dtype, device=T.device)
    glnC = torch.empty((n, lnC.stride(0)), dtype=T.dtype, device=T.device)[:, :lnC.shape[1]]
    _check(lib().chem_source_term_vjp(mech.handle, n, T.data_ptr(), lnC.data_ptr(), lnC.stride(0),
                                      g_omega.data_ptr(), g_omega.stride(0), gT.data_ptr(),
                                      glnC.data_ptr(), int(precision), _stream_ptr(stream)))
    return gT, glnC


def source_term_jacobian(mech: Mechanism, T, lnC, precision: int = FP64, stream=None):
    """Dense Jacobian as a tensor [n, ns, ns + 1]: d omega_k / d ln C_m (m < ns), d / dT."""
    import torch
    _check_state(T, lnC, precision)
    n, ns = T.shape[0], mech.n_species
    J = torch.empty((ns, ns + 1, n), dtype=T.dtype, device=T.device)
    _check(lib().chem_source_term_jacobian(mech.handle, n, T.data_ptr(), lnC.data_ptr(),
                                           lnC.stride(0), J.data_ptr(), n, int(precision),
                                           _stream_ptr(stream)))
    return J.permute(2, 0, 1)


def _omega_fn():
    import torch

    class OmegaFn(torch.autograd.Function):
        """omega(T, ln C) with the hand-written vjp kernel as its backward pass."""

        @staticmethod
        def forward(ctx, mech, T, lnC, precision):
            Tc, lc = T.detach().contiguous(), lnC.detach().contiguous()
            om, _ = source_term_jvp(mech, Tc, lc, torch.zeros_like(Tc), torch.zeros_like(lc),
                                    precision)
            ctx.mech, ctx.precision = mech, precision
            ctx.save_for_backward(Tc, lc)
            return om

        @staticmethod
        def backward(ctx, g):
            Tc, lc = ctx.saved_tensors
            gT, glnC = source_term_vjp(ctx.mech, Tc, lc, g.contiguous(), ctx.precision)
            return None, gT, glnC, None

    return OmegaFn


def omega(mech: Mechanism, T, lnC, precision: int = FP64):
    """Differentiable omega(T, ln C) (torch.autograd), backward by chem_source_term_vjp."""
    return _omega_fn().apply(mech, T, lnC, precision)


# ---------------------------------------------------------------------------------------
# constant-pressure adiabatic reactor (chem_ode_rhs, chem_ode_jacobian, chem_integrate_cells)
# ---------------------------------------------------------------------------------------

def _check_reactor(T, P, Y):
    import torch
    for name, t in (("T", T), ("P", P), ("Y", Y)):
        if not t.is_cuda or t.dtype != torch.float64:
            raise ChemError(1, f"{name} must be a CUDA float64 tensor")
    if T.stride(0) != 1 or P.stride(0) != 1 or Y.dim() != 2 or Y.stride(1) != 1:
        raise ChemError(1, "T, P contiguous and Y row-major with unit column stride")


def ode_rhs(mech: Mechanism, T, P, Y, stream=None):
    """f [n, ns + 1] = (dT/dt, dY/dt) of the constant-pressure reactor at (T, P, Y)."""
    import torch
    _check_reactor(T, P, Y)
    n = T.shape[0]
    f = torch.empty((n, mech.n_species + 1), dtype=torch.float64, device=T.device)
    _check(lib().chem_ode_rhs(mech.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(),
                              Y.stride(0), f.data_ptr(), f.stride(0), _stream_ptr(stream)))
    return f


def ode_jacobian(mech: Mechanism, T, P, Y, stream=None):
    """J [n, ns + 1, ns + 1] = d f / d (T, Y) of the constant-pressure reactor."""
    import torch
    _check_reactor(T, P, Y)
    n, m = T.shape[0], mech.n_species + 1
    J = torch.empty((n, m, m), dtype=torch.float64, device=T.device)
    _check(lib().chem_ode_jacobian(mech.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(),
                                   Y.stride(0), J.data_ptr(), _stream_ptr(stream)))
    return J


def integrate(mech: Mechanism, T, P, Y, t_end: float, rtol: float = 1e-6, atol: float = 1e-12,
              h_init: float = 0.0, h_min: float = 0.0, h_max: float = 0.0, max_steps: int = 0,
              ign_dT: float = 0.0, stats: bool = True, raise_on_failure: bool = False,
              fixed_steps: int = 0, jacobian_fp32: bool = False, stream=None):
    """Integrate the reactors in place (T and Y are overwritten with the state at t_end).
    jacobian_fp32 evaluates the stage Jacobian in FP32 (everything else stays FP64).
    Returns a dict with per-cell 'status', 't_ign', 'n_accepted', 'n_rejected' (CUDA tensors)
    and 'failed' (bool).  CHEM_ENONCONV raises only when raise_on_failure is set."""
    import torch
    _check_reactor(T, P, Y)
    n = T.shape[0]
    dev = T.device
    status = torch.empty((n,), dtype=torch.int32, device=dev)
    out = {"status": status}
    opts = _IntegOpts(float(h_init), float(h_min), float(h_max), int(max_steps), float(ign_dT),
                      None, None, None, int(fixed_steps), int(bool(jacobian_fp32)))
    if stats:
        out["t_ign"] = torch.empty((n,), dtype=torch.float64, device=dev)
        out["n_accepted"] = torch.empty((n,), dtype=torch.int32, device=dev)
        out["n_rejected"] = torch.empty((n,), dtype=torch.int32, device=dev)
        opts.t_ign = out["t_ign"].data_ptr()
        opts.n_accepted = out["n_accepted"].data_ptr()
        opts.n_rejected = out["n_rejected"].data_ptr()
    rc = lib().chem_integrate_cells(mech.handle, n, T.data_ptr(), P.data_ptr(), Y.data_ptr(),
                                    Y.stride(0), float(t_end), float(rtol), float(atol),
                                    C.byref(opts), status.data_ptr(), _stream_ptr(stream))
    out["failed"] = rc == 8
    if rc != 0 and (rc != 8 or raise_on_failure):
        _check(rc)
    return out


def integrate_noalloc(mech: Mechanism, T, P, Y, t_end: float, rtol: float = 1e-6,
                      atol: float = 1e-12, stream=None):
    """chem_integrate_cells_noalloc: as integrate() (in place, defaults for every option) with
    the workspace taken from the library's static scratch; returns the per-cell status."""
    import torch
    _check_reactor(T, P, Y)
    status = torch.empty((T.shape[0],), dtype=torch.int32, device=T.device)
    rc = lib().chem_integrate_cells_noalloc(mech.handle, T.shape[0], T.data_ptr(), P.data_ptr(),
                                            Y.data_ptr(), Y.stride(0), float(t_end), float(rtol),
                                            float(atol), None, status.data_ptr(),
                                            _stream_ptr(stream))
    _check(rc)
    return status


def rosenbrock_tableau():
    """Classical coefficients of the integrator's Rosenbrock method (host call)."""
    s = C.c_int32()
    g = C.c_double()
    alpha, gamma = np.zeros((4, 4)), np.zeros((4, 4))
    b, bh = np.zeros(4), np.zeros(4)
    _check(lib().chem_rosenbrock_tableau(C.byref(s), C.byref(g), _ptr(alpha), _ptr(gamma),
                                         _ptr(b), _ptr(bh)))
    k = s.value
    return dict(stages=k, gamma_ii=g.value, alpha=alpha[:k, :k], gamma=gamma[:k, :k], b=b[:k],
                bhat=bh[:k])


# ---------------------------------------------------------------------------------------
# serving (chem_serve_*)
# ---------------------------------------------------------------------------------------

class Server:
    """A chem_serve server over loaded mechanisms; requests carry numpy host arrays."""

    def __init__(self, mechs, hbm_budget: int):
        self.mechs = list(mechs)
        arr = (C.c_void_p * len(self.mechs))(*[m.handle.value for m in self.mechs])
        h = C.c_void_p()
        _check(lib().chem_serve_create(arr, len(self.mechs), int(hbm_budget), C.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, mech_index: int, kind: int, T, P, Y, precision: int = FP64, out=None,
               dt: float = 0.0, rtol: float = 1e-6, atol: float = 1e-12, status=None,
               T_out=None, Y_out=None, fixed_steps: int = 0) -> int:
        """Queue a request.  SOURCE: `out` receives omega.  INTEGRATE: T_out / Y_out (default:
        T, Y in place) receive the state after dt; `status` the per-cell status."""
        req = _Request(int(mech_index), int(kind), int(precision), int(fixed_steps),
                       int(T.shape[0]),
                       _ptr(T), _ptr(P), _ptr(Y), _ptr(out),
                       _ptr(T if T_out is None else T_out), _ptr(Y if Y_out is None else Y_out),
                       _ptr(status), float(dt), float(rtol), float(atol))
        t = C.c_uint64()
        _check(lib().chem_serve_submit(self._h, C.byref(req), C.byref(t)))
        self._keep[t.value] = (T, P, Y, out, status, T_out, Y_out)
        return t.value

    def poll(self, ticket: int, timeout_us: int = -1):
        """dict of the request's chem_result; raises ChemError on ETIMEOUT / ENOTREADY."""
        r = _Result()
        _check(lib().chem_serve_poll(self._h, int(ticket), C.byref(r), int(timeout_us)))
        self._keep.pop(ticket, None)
        return {f: getattr(r, f) for f, _ in _Result._fields_}

    def info(self):
        i = _ServeInfo()
        _check(lib().chem_serve_info_get(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in _ServeInfo._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(lib().chem_serve_destroy(self._h))
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------
# equilibrium constants: exact table and the approximate network (chem_log_kc, chem_kc_ann_*)
# ---------------------------------------------------------------------------------------

def log_kc(mech: Mechanism, T, stream=None):
    """ln K_c [n, n_reactions] (FP64) at the temperatures T (CUDA float64 tensor)."""
    import torch
    if not T.is_cuda or T.dtype != torch.float64 or T.stride(0) != 1:
        raise ChemError(1, "T must be a contiguous CUDA float64 tensor")
    out = torch.empty((T.shape[0], mech.n_reactions), dtype=torch.float64, device=T.device)
    _check(lib().chem_log_kc(mech.handle, T.shape[0], T.data_ptr(), out.data_ptr(),
                             out.stride(0), _stream_ptr(stream)))
    return out


class KcAnn:
    """An approximate-ANN ln K_c network loaded for one mechanism (chem_kc_ann_load).
    `params`: dict with n_layers, n_hidden, activation ('relu' | 'elu'), x_mean, x_std and
    float32 arrays w_in, b_in, w_hid, b_hid, w_out, b_out, y_mean, y_std."""

    def __init__(self, mech: Mechanism, params):
        self.mech = mech
        f = lambda k: None if params.get(k) is None else np.ascontiguousarray(params[k], np.float32)
        self._keep = {k: f(k) for k in ("w_in", "b_in", "w_hid", "b_hid", "w_out", "b_out",
                                         "y_mean", "y_std")}
        act = {"relu": 0, "elu": 1}[params["activation"]]
        d = _KcAnnDesc(int(params["n_layers"]), int(params["n_hidden"]), act,
                       float(params["x_mean"]), float(params["x_std"]),
                       *(_ptr(self._keep[k]) for k in ("w_in", "b_in", "w_hid", "b_hid",
                                                       "w_out", "b_out", "y_mean", "y_std")))
        h = C.c_void_p()
        _check(lib().chem_kc_ann_load(mech.handle, C.byref(d), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise ChemError(1, "network was freed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            _check(lib().chem_kc_ann_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def source_term_kc_ann(mech: Mechanism, ann, T, P, Y, out=None, stream=None):
    """omega [n, ns] (float32) from the warp-per-cell FP32 kernel with ln K_c from the
    network; ann=None runs the same kernel with the exact Gibbs layer."""
    import torch
    for name, t in (("T", T), ("P", P), ("Y", Y)):
        if not t.is_cuda or t.dtype != torch.float32:
            raise ChemError(1, f"{name} must be a CUDA float32 tensor")
    n = T.shape[0]
    if out is None:
        out = torch.empty((n, mech.n_species), dtype=torch.float32, device=T.device)
    _check(lib().chem_source_term_kc_ann(mech.handle, ann.handle if ann is not None else None, n,
                                         T.data_ptr(), P.data_ptr(),
                                         Y.data_ptr(), Y.stride(0), out.data_ptr(), out.stride(0),
                                         _stream_ptr(stream)))
    return out
