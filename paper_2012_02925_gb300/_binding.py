"""ctypes binding of the C ABI in include/fvgb.h (argument marshalling only).

Every numerical step runs in the CUDA library; this module passes pointers,
sizes and the current torch CUDA stream.  It refuses to run without the
compiled library: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfvgb.so")

FV_OK, FV_ERR_INVALID_ARG, FV_ERR_CUDA, FV_ERR_OOM, FV_ERR_NONFINITE, FV_ERR_TIMEOUT, FV_ERR_UNSUPPORTED = range(7)
PREC_FP64, PREC_DF64, PREC_FP32FLUX = 0, 1, 2
PRECISIONS = {"fp64": PREC_FP64, "df64": PREC_DF64, "fp32flux": PREC_FP32FLUX}

EXPORTS = ("fv_config_default", "fv_create_blocks", "fv_destroy", "fv_last_error", "fv_state_size",
           "fv_field_size", "fv_cell_count", "fv_set_state", "fv_set_buffer", "fv_get_state", "fv_set_source",
           "fv_exchange_ghosts", "fv_residual", "fv_rk_stage", "fv_rk_step", "fv_residual_norms",
           "fv_adjoint_vjp", "fv_autotune", "fv_get_launch", "fv_set_boundaries", "fv_set_monitor",
           "fv_monitor_norms", "fv_stage_state", "fv_set_state_staged", "fv_graph_count",
           "fv_probe_alu_rates", "fv_set_halo", "fv_halo_size", "fv_halo_pack", "fv_halo_unpack",
           "fv_check_rcp64", "fv_check_sqrt64", "fv_set_adjoint_arith")


class FvError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("fvgb error %d: %s" % (code, msg))
        self.code = code


class fv_block_desc(ctypes.Structure):
    _fields_ = [("ni", ctypes.c_int), ("nj", ctypes.c_int), ("nk", ctypes.c_int),
                ("nodes", ctypes.POINTER(ctypes.c_double)),
                ("x0", ctypes.c_double * 3), ("h", ctypes.c_double * 3)]


class fv_connection(ctypes.Structure):
    _fields_ = [("dst_block", ctypes.c_int), ("dst_face", ctypes.c_int),
                ("dst_lo", ctypes.c_int * 2), ("dst_hi", ctypes.c_int * 2),
                ("src_block", ctypes.c_int), ("src_face", ctypes.c_int),
                ("src_lo", ctypes.c_int * 2), ("transform", ctypes.c_int * 2)]


class fv_bc_patch(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("face", ctypes.c_int),
                ("lo", ctypes.c_int * 2), ("hi", ctypes.c_int * 2),
                ("kind", ctypes.c_int), ("state", ctypes.c_double * 5)]


class fv_config(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("eps", ctypes.c_double), ("kappa", ctypes.c_double),
                ("harten", ctypes.c_double), ("va_delta2", ctypes.c_double),
                ("limiter", ctypes.c_int), ("fix_all", ctypes.c_int), ("dim", ctypes.c_int),
                ("n_stages", ctypes.c_int), ("alpha", ctypes.c_double * 8),
                ("precision", ctypes.c_int), ("tile", ctypes.c_int), ("kchunk", ctypes.c_int),
                ("flux", ctypes.c_int), ("visc", ctypes.c_int),
                ("mu", ctypes.c_double), ("prandtl", ctypes.c_double), ("r_gas", ctypes.c_double),
                ("sutherland", ctypes.c_int), ("t_ref", ctypes.c_double), ("s_suth", ctypes.c_double)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libfvgb.so (built by ``paper_2012_02925_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("CUDA library %s is missing: run `python -c \"import __graft_entry__ as g; g.build()\"` "
                           "(or python -m paper_2012_02925_gb300.build); there is no CPU fallback" % p)
    L = ctypes.CDLL(p)
    vp, i64, dbl, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.fv_config_default.argtypes = [ctypes.POINTER(fv_config)]
    L.fv_config_default.restype = None
    L.fv_create_blocks.argtypes = [ctypes.POINTER(fv_block_desc), i32, ctypes.POINTER(fv_connection), i32,
                                   ctypes.POINTER(fv_config), ctypes.POINTER(vp)]
    L.fv_destroy.argtypes = [vp]
    L.fv_last_error.argtypes = [vp]
    L.fv_last_error.restype = ctypes.c_char_p
    for f in ("fv_state_size", "fv_field_size", "fv_cell_count"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = i64
    L.fv_set_state.argtypes = [vp, vp, vp]
    L.fv_set_buffer.argtypes = [vp, i32, vp, vp]
    L.fv_get_state.argtypes = [vp, i32, vp, vp]
    L.fv_set_source.argtypes = [vp, vp, vp]
    L.fv_exchange_ghosts.argtypes = [vp, i32, vp]
    L.fv_residual.argtypes = [vp, i32, vp, vp]
    L.fv_rk_stage.argtypes = [vp, i32, dbl, vp]
    L.fv_rk_step.argtypes = [vp, dbl, i32, vp]
    L.fv_residual_norms.argtypes = [vp, i32, vp, vp]
    L.fv_adjoint_vjp.argtypes = [vp, i32, dbl, vp, vp, vp, vp, vp]
    L.fv_autotune.argtypes = [vp, dbl, i32, vp]
    L.fv_get_launch.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.fv_set_boundaries.argtypes = [vp, ctypes.POINTER(fv_bc_patch), i32]
    L.fv_set_monitor.argtypes = [vp, i32]
    L.fv_stage_state.argtypes = [vp, vp, vp]
    L.fv_set_state_staged.argtypes = [vp, vp]
    L.fv_monitor_norms.argtypes = [vp, vp, vp]
    L.fv_graph_count.argtypes = [vp]
    L.fv_graph_count.restype = i32
    L.fv_probe_alu_rates.argtypes = [vp, i32, vp]
    L.fv_probe_alu_rates.restype = i32
    L.fv_set_adjoint_arith.argtypes = [vp, i32]
    L.fv_set_adjoint_arith.restype = i32
    L.fv_check_rcp64.argtypes = [vp, i64, vp, vp]
    L.fv_check_rcp64.restype = i32
    L.fv_check_sqrt64.argtypes = [vp, i64, vp, vp]
    L.fv_check_sqrt64.restype = i32
    L.fv_set_halo.argtypes = [vp, ctypes.POINTER(fv_connection), i32, ctypes.POINTER(fv_connection), i32]
    L.fv_set_halo.restype = i32
    L.fv_halo_size.argtypes = [vp, i32]
    L.fv_halo_size.restype = i64
    L.fv_halo_pack.argtypes = [vp, i32, vp, vp]
    L.fv_halo_pack.restype = i32
    L.fv_halo_unpack.argtypes = [vp, i32, vp, vp]
    L.fv_halo_unpack.restype = i32
    for f in ("fv_create_blocks", "fv_destroy", "fv_set_state", "fv_set_buffer", "fv_get_state", "fv_set_source",
              "fv_exchange_ghosts", "fv_residual", "fv_rk_stage", "fv_rk_step", "fv_residual_norms",
              "fv_adjoint_vjp", "fv_autotune", "fv_get_launch", "fv_set_boundaries", "fv_set_monitor",
              "fv_monitor_norms", "fv_stage_state", "fv_set_state_staged"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def _ptr(x) -> int:
    """Raw address of a torch tensor or numpy array (contiguous float64)."""
    if isinstance(x, np.ndarray):
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"], "need a contiguous float64 array"
        return x.ctypes.data
    import torch
    assert isinstance(x, torch.Tensor) and x.dtype == torch.float64 and x.is_contiguous(), \
        "need a contiguous float64 tensor"
    return x.data_ptr()


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    import torch
    if torch.cuda.is_available():
        return torch.cuda.current_stream().cuda_stream
    return 0


PROBE_RATES = ("fp64_fma", "fp64_add", "fp64_mul", "fp64_rcp", "fp64_sqrt", "fp32_fma",
               "df64_add", "df64_mul", "df64_div", "df64_sqrt", "df64_abs", "fp64_rcp_refined",
               "fp64_sqrt_refined")


def probe_alu_rates(stream=None) -> dict:
    """Measured operations/s of the arithmetic the stage kernel's forms use
    (fv_probe_alu_rates) on the current device."""
    L = load_library()
    out = np.zeros(len(PROBE_RATES))
    rc = L.fv_probe_alu_rates(out.ctypes.data, len(PROBE_RATES), _stream(stream))
    if rc != FV_OK:
        raise FvError(rc, "fv_probe_alu_rates failed")
    return dict(zip(PROBE_RATES, out.tolist()))


def _conn_table(conns: Sequence):
    """ctypes array of fv_connection from objects with the fields of
    cases.Connection (at least one entry, so that the pointer is valid)."""
    cs = (fv_connection * max(1, len(conns)))()
    for n, c in enumerate(conns):
        e = cs[n]
        e.dst_block, e.dst_face = int(c.dst_block), int(c.dst_face)
        e.dst_lo[0], e.dst_lo[1] = map(int, c.dst_lo)
        e.dst_hi[0], e.dst_hi[1] = map(int, c.dst_hi)
        e.src_block, e.src_face = int(c.src_block), int(c.src_face)
        e.src_lo[0], e.src_lo[1] = map(int, c.src_lo)
        e.transform[0], e.transform[1] = map(int, c.transform)
    return cs


def _check_arith(name, x):
    import torch
    L = load_library()
    out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
    rc = getattr(L, name)(_ptr(x), x.numel(), out.data_ptr(), _stream(None))
    if rc != FV_OK:
        raise FvError(rc, name + " failed")
    return out


def check_rcp64(x):
    """(face-code reciprocal, IEEE 1.0 / x) of a float64 CUDA tensor x, as a
    (n, 2) tensor (fv_check_rcp64)."""
    return _check_arith("fv_check_rcp64", x)


def check_sqrt64(x):
    """(face-code square root, IEEE sqrt(x)) of a float64 CUDA tensor x, as a
    (n, 2) tensor (fv_check_sqrt64)."""
    return _check_arith("fv_check_sqrt64", x)


class Solver:
    """One fvgb handle: blocks, connections and method parameters on the
    current CUDA device.  Method names follow the C ABI."""

    def __init__(self, blocks: Sequence, conns: Sequence, dim: int, params: dict,
                 precision: str = "fp64", tile: int = 0, kchunk: int = 0):
        L = load_library()
        self._L = L
        self._h = ctypes.c_void_p()
        descs = (fv_block_desc * len(blocks))()
        keep = []
        for n, b in enumerate(blocks):
            d = descs[n]
            d.ni, d.nj, d.nk = int(b.ni), int(b.nj), int(b.nk)
            if b.nodes is not None:
                a = np.ascontiguousarray(b.nodes, dtype=np.float64)
                keep.append(a)
                d.nodes = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            else:
                d.nodes = None
            for x in range(3):
                d.x0[x] = float(b.x0[x])
                d.h[x] = float(b.h[x])
        cs = _conn_table(conns)
        cfg = fv_config()
        L.fv_config_default(ctypes.byref(cfg))
        cfg.gamma = params.get("gamma", 1.4)
        cfg.eps = params.get("eps", 1.0)
        cfg.kappa = params.get("kappa", -1.0)
        cfg.harten = params.get("harten", 0.1)
        cfg.va_delta2 = params.get("va_delta2", 1e-12)
        cfg.limiter = int(params.get("limiter", 1))
        cfg.fix_all = int(params.get("fix_all", 0))
        cfg.flux = int(params.get("flux", 0))
        cfg.visc = int(params.get("visc", 0))
        if cfg.visc:
            cfg.mu = float(params["mu"])
            cfg.prandtl = float(params.get("prandtl", 0.72))
            cfg.r_gas = float(params.get("r_gas", 287.0))
            cfg.sutherland = int(params.get("sutherland", 0))
            cfg.t_ref = float(params.get("t_ref", 273.15))
            cfg.s_suth = float(params.get("s_suth", 110.4))
        cfg.dim = int(dim)
        alpha = params.get("alpha", (0.25, 1.0 / 3.0, 0.5, 1.0))
        cfg.n_stages = len(alpha)
        for x, a in enumerate(alpha):
            cfg.alpha[x] = a
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.tile = int(tile)
        cfg.kchunk = int(kchunk)
        self.n_stages = cfg.n_stages
        self.precision = precision
        self.block_dims = [(int(b.ni), int(b.nj), int(b.nk)) for b in blocks]
        rc = L.fv_create_blocks(descs, len(blocks), cs, len(conns), ctypes.byref(cfg), ctypes.byref(self._h))
        if rc != FV_OK:
            raise FvError(rc, L.fv_last_error(None).decode())

    @classmethod
    def from_problem(cls, pb, precision: str = "fp64", **kw) -> "Solver":
        s = cls(pb.blocks, pb.conns, pb.dim, pb.params, precision, **kw)
        bcs = getattr(pb, "bcs", None)
        if bcs:
            s.set_boundaries(bcs)
        return s

    # -- plumbing ---------------------------------------------------------------
    def _check(self, rc: int):
        if rc != FV_OK:
            raise FvError(rc, self._L.fv_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._L.fv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def state_size(self) -> int:
        return int(self._L.fv_state_size(self._h))

    @property
    def field_size(self) -> int:
        return int(self._L.fv_field_size(self._h))

    @property
    def cell_count(self) -> int:
        return int(self._L.fv_cell_count(self._h))

    # -- C ABI calls ---------------------------------------------------------------
    def set_state(self, q, stream=None):
        self._check(self._L.fv_set_state(self._h, _ptr(q), _stream(stream)))

    def stage_state(self, q, stream=None):
        """Copy a packed state into the handle's staging buffer on `stream`
        (see fv_stage_state); set_state_staged() then makes it the state."""
        self._check(self._L.fv_stage_state(self._h, _ptr(q), _stream(stream)))

    def set_state_staged(self, stream=None):
        self._check(self._L.fv_set_state_staged(self._h, _stream(stream)))

    def set_buffer(self, buffer: int, q, stream=None):
        self._check(self._L.fv_set_buffer(self._h, int(buffer), _ptr(q), _stream(stream)))

    def stage_buffers(self, m: int):
        """(input buffer, output buffer) of RK stage m, as fv_rk_stage defines them."""
        M = self.n_stages
        src = 0 if m == 1 else (0 if m - 1 == M else (1 if (m - 1) % 2 == 1 else 2))
        dst = 0 if m == M else (1 if m % 2 == 1 else 2)
        return src, dst

    def get_state(self, buffer: int = 0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.state_size, dtype=torch.float64, device="cuda")
        self._check(self._L.fv_get_state(self._h, int(buffer), _ptr(out), _stream(stream)))
        return out

    def set_source(self, s, stream=None):
        self._check(self._L.fv_set_source(self._h, None if s is None else _ptr(s), _stream(stream)))

    def set_boundaries(self, patches: Sequence) -> None:
        """Physical boundary patches (objects with block, face, lo, hi, kind,
        state; see fv_bc_kind); an empty sequence clears them."""
        arr = (fv_bc_patch * max(1, len(patches)))()
        for n, p in enumerate(patches):
            a = arr[n]
            a.block, a.face, a.kind = int(p.block), int(p.face), int(p.kind)
            a.lo[0], a.lo[1] = int(p.lo[0]), int(p.lo[1])
            a.hi[0], a.hi[1] = int(p.hi[0]), int(p.hi[1])
            st = tuple(getattr(p, "state", (0.0,) * 5))
            for v in range(5):
                a.state[v] = float(st[v])
        self._check(self._L.fv_set_boundaries(self._h, arr, len(patches)))

    def exchange_ghosts(self, buffer: int = 0, stream=None):
        self._check(self._L.fv_exchange_ghosts(self._h, int(buffer), _stream(stream)))

    def residual(self, buffer: int = 0, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(self.field_size, dtype=torch.float64, device="cuda")
        self._check(self._L.fv_residual(self._h, int(buffer), _ptr(out), _stream(stream)))
        return out

    def rk_stage(self, stage: int, dt: float, stream=None):
        self._check(self._L.fv_rk_stage(self._h, int(stage), float(dt), _stream(stream)))

    def rk_step(self, dt: float, use_graph: bool = True, stream=None):
        self._check(self._L.fv_rk_step(self._h, float(dt), int(bool(use_graph)), _stream(stream)))

    # -- cross-device halo (fv_set_halo) ---------------------------------------
    def set_halo(self, send: Sequence, recv: Sequence) -> None:
        """Send and receive slab tables (connections with the local side's
        block index in this handle's numbering; see fv_set_halo)."""
        self._check(self._L.fv_set_halo(self._h, _conn_table(send), len(send), _conn_table(recv), len(recv)))

    def halo_size(self, recv: bool) -> int:
        return int(self._L.fv_halo_size(self._h, 1 if recv else 0))

    def halo_pack(self, buffer: int, send, stream=None):
        self._check(self._L.fv_halo_pack(self._h, int(buffer), _ptr(send) if send is not None else None,
                                         _stream(stream)))

    def halo_unpack(self, buffer: int, recv, stream=None):
        self._check(self._L.fv_halo_unpack(self._h, int(buffer), _ptr(recv) if recv is not None else None,
                                           _stream(stream)))

    def set_adjoint_arith(self, precision: str) -> None:
        """Arithmetic of the adjoint's face sweeps: "fp64" or "df64"."""
        self._check(self._L.fv_set_adjoint_arith(self._h, PRECISIONS[precision]))

    def graph_count(self) -> int:
        """RK-step graphs held (one per stream stepped on with use_graph)."""
        return int(self._L.fv_graph_count(self._h))

    def residual_norms(self, buffer: int = 0, stream=None):
        out = np.zeros(10)
        rc = self._L.fv_residual_norms(self._h, int(buffer), out.ctypes.data, _stream(stream))
        if rc == FV_ERR_NONFINITE:
            raise FvError(rc, self._L.fv_last_error(self._h).decode())
        self._check(rc)
        return out[:5].copy(), out[5:].copy()

    def set_monitor(self, on: bool = True):
        """Record the residual norms of every RK stage 1 from now on (the
        residual of the state each step starts from; see fv_set_monitor)."""
        self._check(self._L.fv_set_monitor(self._h, 1 if on else 0))

    def monitor_norms(self, stream=None):
        """(L2, Linf) per variable recorded by the latest monitored stage 1."""
        out = np.zeros(10)
        rc = self._L.fv_monitor_norms(self._h, out.ctypes.data, _stream(stream))
        if rc == FV_ERR_NONFINITE:
            raise FvError(rc, self._L.fv_last_error(self._h).decode())
        self._check(rc)
        return out[:5].copy(), out[5:].copy()

    def autotune(self, dt: float, reps: int = 3, stream=None):
        self._check(self._L.fv_autotune(self._h, float(dt), int(reps), _stream(stream)))
        return self.launch()

    def launch(self):
        out = (ctypes.c_int * 4)()
        self._check(self._L.fv_get_launch(self._h, out))
        return {"tile": out[0], "kchunk": out[1], "tiles": out[2], "ctas": out[3]}

    def adjoint_vjp(self, stage: int, dt: float, qin, lam_out, lam_in, lam_q0, stream=None):
        self._check(self._L.fv_adjoint_vjp(self._h, int(stage), float(dt), _ptr(qin), _ptr(lam_out),
                                           _ptr(lam_in), _ptr(lam_q0), _stream(stream)))
