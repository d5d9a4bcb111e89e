"""GB300-native equilibrium projection of voxelized stress fields.

Python face of libeq.so (include/eq.h): the closest L^2 divergence-free field to a measured
symmetric stress field on a periodic grid (Zhou et al., Sec. 3.2), computed in Fourier space with
the continuous (CDO, Sec. 4.1) or the central-difference modified wavevector (DDO, Sec. 4.2).
PyTorch provides device memory and streams; the work runs in the library's CUDA kernels.

Fields are tensors of shape (B, 6, nz, ny, nx) or (6, nz, ny, nx), x fastest, Voigt order
(xx, yy, zz, yz, xz, xy), float32 or float64, contiguous, on a CUDA device.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import EqError, EqNorms, EqPlanOpts

__all__ = ["Plan", "VarlenPlan", "Server", "project", "eq_plan_create_varlen", "eq_plan_create", "eq_project", "eq_project_host", "eq_norms",
           "eq_plan_workspace_bytes", "eq_plan_destroy", "eq_last_error", "eq_plan_set_timing",
           "eq_plan_pass_ms", "EqError"]

_OPS = {"ddo": _lib.EQ_OP_DDO, "cdo": _lib.EQ_OP_CDO}
_NYQ = {"keep": _lib.EQ_NYQ_KEEP, "zero": _lib.EQ_NYQ_ZERO}
_TARGET = {"equilibrium": _lib.EQ_TARGET_EQUILIBRIUM,
           "compatibility": _lib.EQ_TARGET_COMPATIBILITY}
_DT = {torch.float32: _lib.EQ_F32, torch.float64: _lib.EQ_F64}


def _opts(op="ddo", h=(1.0, 1.0, 1.0), nyq="keep", want_linf=True, graph=True,
          target="equilibrium") -> EqPlanOpts:
    o = EqPlanOpts()
    _lib.load().eq_plan_opts_default(ctypes.byref(o))
    o.op = _OPS[op]
    o.hx, o.hy, o.hz = (float(v) for v in h)
    o.nyq = _NYQ[nyq]
    o.want_linf = 1 if want_linf else 0
    o.graph = 1 if graph else 0
    o.target = _TARGET[target]
    return o


# ---- C-ABI names (thin marshalling) ------------------------------------------------------

def eq_plan_create(nx, ny, nz, dtype=torch.float32, batch=1, op="ddo", h=(1.0, 1.0, 1.0),
                   nyq="keep", want_linf=True, target="equilibrium") -> int:
    """Returns an opaque plan handle (int) on the current CUDA device."""
    handle = ctypes.c_void_p()
    opts = _opts(op, h, nyq, want_linf, target=target)
    st = _lib.load().eq_plan_create(int(nx), int(ny), int(nz), _DT[dtype], int(batch),
                                    ctypes.byref(opts), ctypes.byref(handle))
    _lib.check(st, "eq_plan_create")
    return handle.value


def eq_plan_create_varlen(dims, dtype=torch.float32, op="ddo", h=(1.0, 1.0, 1.0), nyq="keep",
                          want_linf=True, target="equilibrium") -> int:
    """dims: sequence of (nx, ny, nz) per field.  Returns an opaque plan handle."""
    flat = [int(v) for d in dims for v in d]
    arr = (ctypes.c_int * len(flat))(*flat)
    handle = ctypes.c_void_p()
    opts = _opts(op, h, nyq, want_linf, target=target)
    st = _lib.load().eq_plan_create_varlen(arr, len(dims), _DT[dtype], ctypes.byref(opts),
                                           ctypes.byref(handle))
    _lib.check(st, "eq_plan_create_varlen")
    return handle.value


def eq_project(plan: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _lib.check(_lib.load().eq_project(plan, d_in, d_out, stream or None), "eq_project")


def eq_project_host(plan: int, h_in: int, h_out: int, stream: int = 0) -> None:
    _lib.check(_lib.load().eq_project_host(plan, h_in, h_out, stream or None), "eq_project_host")


def eq_project_hodge(handle, d_in, d_out, d_y, stream) -> None:
    _lib.check(_lib.load().eq_project_hodge(ctypes.c_void_p(handle), ctypes.c_void_p(d_in),
                                            ctypes.c_void_p(d_out), ctypes.c_void_p(d_y),
                                            ctypes.c_void_p(stream)), "eq_project_hodge")


def eq_norms(plan: int, batch: int) -> list:
    arr = (EqNorms * batch)()
    _lib.check(_lib.load().eq_norms(plan, arr), "eq_norms")
    return [arr[i].to_dict() for i in range(batch)]


def eq_plan_workspace_bytes(plan: int) -> int:
    return int(_lib.load().eq_plan_workspace_bytes(plan))


def eq_plan_destroy(plan: int) -> None:
    _lib.load().eq_plan_destroy(plan)


def eq_plan_set_timing(plan: int, max_calls: int) -> None:
    _lib.check(_lib.load().eq_plan_set_timing(plan, int(max_calls)), "eq_plan_set_timing")


def eq_plan_pass_ms(plan: int):
    """(dict pass name -> summed ms, number of timed calls); timing is off afterwards."""
    ms = (ctypes.c_double * _lib.EQ_NUM_PASSES)()
    n = ctypes.c_int()
    _lib.check(_lib.load().eq_plan_pass_ms(plan, ms, ctypes.byref(n)), "eq_plan_pass_ms")
    return dict(zip(_lib.PASS_NAMES, list(ms))), n.value


def eq_last_error() -> str:
    return _lib.load().eq_last_error().decode()


# ---- convenience object ------------------------------------------------------------------

class Plan:
    """A plan for `batch` fields of one grid size and dtype on one device."""

    def __init__(self, nx, ny, nz, dtype=torch.float32, batch=1, op="ddo", h=(1.0, 1.0, 1.0),
                 nyq="keep", want_linf=True, device=None, target="equilibrium"):
        self.shape = (int(batch), 6, int(nz), int(ny), int(nx))
        self.numel = _numel(self.shape)
        self.dtype = dtype
        self.device = _cuda_device(device)
        with torch.cuda.device(self.device):
            self.handle = eq_plan_create(nx, ny, nz, dtype, batch, op, h, nyq, want_linf, target)

    def _check(self, t: torch.Tensor, name: str):
        if not t.is_cuda or t.device != self.device:
            raise ValueError(f"{name} must be on {self.device}")
        if t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.numel:
            raise ValueError(f"{name} must be a contiguous {self.dtype} tensor of shape {self.shape}")

    def project(self, x: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Enqueue the projection of x into out (allocated if None; may be x itself)."""
        self._check(x, "x")
        if out is None:
            out = torch.empty_like(x)
        self._check(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            eq_project(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
        return out

    def project_hodge(self, x: torch.Tensor, out: torch.Tensor | None = None,
                      y: torch.Tensor | None = None, stream=None):
        """Projection plus the Hodge potential: returns (out, y), y of shape (batch, 4, nz, ny, nx)
        with y_x, y_y, y_z in planes 0..2 (plane 3 is working space)."""
        self._check(x, "x")
        if out is None:
            out = torch.empty_like(x)
        if y is None:
            b, _, nz, ny, nx = self.shape
            y = torch.empty((b, 4, nz, ny, nx), dtype=self.dtype, device=self.device)
        self._check(out, "out")
        if not y.is_cuda or y.device != self.device or y.dtype != self.dtype \
                or not y.is_contiguous() or y.numel() != self.numel // 6 * 4:
            raise ValueError(f"y must be a contiguous {self.dtype} tensor of shape "
                             f"{(self.shape[0], 4) + self.shape[2:]} on {self.device}")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            eq_project_hodge(self.handle, x.data_ptr(), out.data_ptr(), y.data_ptr(), s.cuda_stream)
        return out, y

    def project_padded(self, x: torch.Tensor, out: torch.Tensor | None = None,
                       stream=None) -> torch.Tensor:
        """x: specimen fields (batch, 6, sz, sy, sx) on the plan's device, no larger than the
        plan's grid; projected inside a zero-stress buffer filling the grid, cut back out."""
        b, _, nz, ny, nx = self.shape
        if not x.is_cuda or x.device != self.device or x.dtype != self.dtype or x.dim() != 5 \
                or x.shape[0] != b or x.shape[1] != 6 or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous ({b}, 6, sz, sy, sx) {self.dtype} tensor")
        sz, sy, sx = x.shape[2:]
        if out is None:
            out = torch.empty_like(x)
        if out.shape != x.shape or out.dtype != x.dtype or not out.is_contiguous() \
                or out.device != x.device:
            raise ValueError("out must match x")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().eq_project_padded(ctypes.c_void_p(self.handle), sx, sy, sz,
                                                     ctypes.c_void_p(x.data_ptr()),
                                                     ctypes.c_void_p(out.data_ptr()),
                                                     ctypes.c_void_p(s.cuda_stream)),
                       "eq_project_padded")
        return out

    def project_host(self, x: torch.Tensor, out: torch.Tensor, stream=None,
                     wait: bool = True) -> torch.Tensor:
        """Host tensors in and out (pinned for full bandwidth).  wait=True blocks until done;
        wait=False only enqueues on the stream (eq_project_host_async): keep x and out untouched
        until the stream or norms() says the call has finished."""
        for t, n in ((x, "x"), (out, "out")):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() \
                    or t.numel() != self.numel:
                raise ValueError(f"{n} must be a contiguous host {self.dtype} tensor of shape {self.shape}")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            if wait:
                eq_project_host(self.handle, x.data_ptr(), out.data_ptr(), s.cuda_stream)
            else:
                _lib.check(_lib.load().eq_project_host_async(
                    ctypes.c_void_p(self.handle), ctypes.c_void_p(x.data_ptr()),
                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream)),
                    "eq_project_host_async")
        return out

    def norms(self) -> list:
        with torch.cuda.device(self.device):
            return eq_norms(self.handle, self.shape[0])

    def selftest_wait_timeout(self, polls: int = 1024, stream=None) -> None:
        """Enqueue the failure-detection self-test: a bounded wait that runs out after `polls`
        polls and raises the plan's error flag, so that the next norms() raises EqError with
        EQ_ERR_TIMEOUT (and clears the flag)."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().eq_selftest_wait_timeout(ctypes.c_void_p(self.handle),
                                                            int(polls), s.cuda_stream),
                       "eq_selftest_wait_timeout")

    def autotune(self, x: torch.Tensor, out: torch.Tensor, stream=None) -> None:
        """Pick the fastest pass shapes on these buffers (out is overwritten)."""
        self._check(x, "x")
        self._check(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().eq_plan_autotune(self.handle, x.data_ptr(), out.data_ptr(),
                                                    s.cuda_stream), "eq_plan_autotune")

    def set_timing(self, max_calls: int) -> None:
        eq_plan_set_timing(self.handle, max_calls)

    def pass_ms(self):
        with torch.cuda.device(self.device):
            return eq_plan_pass_ms(self.handle)

    @property
    def workspace_bytes(self) -> int:
        return eq_plan_workspace_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            eq_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VarlenPlan(Plan):
    """Fields of different sizes packed back to back in one flat tensor (see pack/unpack)."""

    def __init__(self, dims, dtype=torch.float32, op="ddo", h=(1.0, 1.0, 1.0), nyq="keep",
                 want_linf=True, device=None, target="equilibrium"):
        self.dims = [tuple(int(v) for v in d) for d in dims]
        self.dtype = dtype
        self.numel = sum(6 * nx * ny * nz for nx, ny, nz in self.dims)
        self.shape = (len(self.dims), self.numel)
        self.device = _cuda_device(device)
        with torch.cuda.device(self.device):
            self.handle = eq_plan_create_varlen(self.dims, dtype, op, h, nyq, want_linf, target)

    def _check(self, t, name):
        if not t.is_cuda or t.device != self.device or t.dtype != self.dtype \
                or not t.is_contiguous() or t.numel() != self.numel:
            raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor with "
                             f"{self.numel} elements on {self.device}")

    def pack(self, fields) -> torch.Tensor:
        return torch.cat([f.reshape(-1) for f in fields]).to(self.device, self.dtype).contiguous()

    def unpack(self, flat):
        out, off = [], 0
        for nx, ny, nz in self.dims:
            n = 6 * nx * ny * nz
            out.append(flat[off:off + n].view(6, nz, ny, nx))
            off += n
        return out


class Server:
    """Request loop (eq_server_*): single fields from host memory, admitted by HBM footprint."""

    def __init__(self, hbm_budget_bytes: int, max_inflight: int = 8, device=None):
        self.device = _cuda_device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(_lib.load().eq_server_create(int(hbm_budget_bytes), int(max_inflight),
                                                    ctypes.byref(h)), "eq_server_create")
        self.handle = h.value
        self._keep = {}

    def submit(self, x: torch.Tensor, out: torch.Tensor, op="ddo", h=(1.0, 1.0, 1.0),
               nyq="keep", want_linf=True, target="equilibrium") -> int:
        """x, out: host tensors (6, nz, ny, nx), float32/float64, contiguous (pinned is best)."""
        if x.is_cuda or out.is_cuda or x.shape != out.shape or x.dim() != 4 or x.shape[0] != 6 \
                or x.dtype != out.dtype or not (x.is_contiguous() and out.is_contiguous()):
            raise ValueError("x and out must be contiguous host tensors of shape (6, nz, ny, nx)")
        _, nz, ny, nx = x.shape
        opts = _opts(op, h, nyq, want_linf, target=target)
        t = ctypes.c_ulonglong()
        st = _lib.load().eq_serve_submit(self.handle, nx, ny, nz, _DT[x.dtype], ctypes.byref(opts),
                                         x.data_ptr(), out.data_ptr(), ctypes.byref(t))
        _lib.check(st, "eq_serve_submit")
        self._keep[t.value] = (x, out)
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """None while pending; else (norms dict, latency seconds).  Raises on a failed request."""
        n = EqNorms()
        lat = ctypes.c_double()
        st = _lib.load().eq_serve_poll(self.handle, int(ticket), int(timeout_us), ctypes.byref(n),
                                       ctypes.byref(lat))
        if st == _lib.EQ_PENDING:
            return None
        self._keep.pop(ticket, None)
        _lib.check(st, "eq_serve_poll")
        return n.to_dict(), lat.value

    def cancel(self, ticket: int) -> bool:
        """Withdraw a request that has not started: True if withdrawn, False if it already runs
        (EQ_ERR_BUSY: poll it instead).  Raises for an unknown ticket."""
        st = _lib.load().eq_serve_cancel(self.handle, int(ticket))
        if st == _lib.EQ_ERR_BUSY:
            return False
        _lib.check(st, "eq_serve_cancel")
        self._keep.pop(ticket, None)
        return True

    def stats(self) -> dict:
        """Counters since creation and the current state (eq_server_stats)."""
        st = _lib.EqServerStats()
        _lib.check(_lib.load().eq_server_stats(self.handle, ctypes.byref(st)), "eq_server_stats")
        return st.to_dict()

    def wait(self, ticket: int, timeout_s: float = 60.0):
        import time
        t0 = time.monotonic()
        while True:
            r = self.poll(ticket, 10000)
            if r is not None:
                return r
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"request {ticket} not done after {timeout_s} s")

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().eq_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _cuda_device(device) -> torch.device:
    d = torch.device("cuda") if device is None else torch.device(device)
    if d.type != "cuda":
        raise ValueError("plans live on a CUDA device")
    return torch.device("cuda", torch.cuda.current_device() if d.index is None else d.index)


def _numel(shape):
    n = 1
    for s in shape:
        n *= s
    return n


class Grains:
    """A fixed grain map for grain averaging (Sec. 5.1): ``gmap`` is a CPU int tensor or array of
    shape (nz, ny, nx) with ids in [0, ngrains)."""

    def __init__(self, gmap, ngrains: int, device=None):
        g = torch.as_tensor(gmap).to(torch.int32).contiguous()
        if g.dim() != 3 or g.is_cuda:
            raise ValueError("gmap must be a host (nz, ny, nx) integer map")
        self.shape = tuple(g.shape)
        self.ngrains = int(ngrains)
        self.device = _cuda_device(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            st = _lib.load().eq_grains_create(
                ctypes.cast(g.data_ptr(), ctypes.POINTER(ctypes.c_int)), self.shape[2],
                self.shape[1], self.shape[0], self.ngrains, ctypes.byref(h))
        _lib.check(st, "eq_grains_create")
        self.handle = h.value

    def average(self, x: torch.Tensor, means: torch.Tensor | None = None,
                out: torch.Tensor | None = None, want_field: bool = True, stream=None):
        """x: (B, 6, nz, ny, nx) CUDA float32/float64.  Returns (means, field): means (B, ngrains,
        6) float64 and, with want_field, the grain-averaged field (may be x itself via out=x)."""
        if not x.is_cuda or x.device != self.device or x.dim() != 5 or x.shape[1] != 6 \
                or tuple(x.shape[2:]) != self.shape or not x.is_contiguous() \
                or x.dtype not in _DT:
            raise ValueError(f"x must be a contiguous (B, 6) + {self.shape} CUDA tensor")
        b = x.shape[0]
        if means is None:
            means = torch.empty((b, self.ngrains, 6), dtype=torch.float64, device=self.device)
        if want_field and out is None:
            out = torch.empty_like(x)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            st = _lib.load().eq_grain_average(
                ctypes.c_void_p(self.handle), _DT[x.dtype], b, ctypes.c_void_p(x.data_ptr()),
                ctypes.c_void_p(means.data_ptr()),
                ctypes.c_void_p(out.data_ptr() if want_field else None),
                ctypes.c_void_p(s.cuda_stream))
        _lib.check(st, "eq_grain_average")
        return means, (out if want_field else None)

    def close(self):
        if getattr(self, "handle", None):
            _lib.load().eq_grains_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def project(x: torch.Tensor, op="ddo", h=(1.0, 1.0, 1.0), nyq="keep", out=None,
            target="equilibrium"):
    """Project a (6, nz, ny, nx) or (B, 6, nz, ny, nx) CUDA tensor; returns (out, norms).
    target="compatibility" returns the closest strain-compatible field instead."""
    single = x.dim() == 4
    xb = x.unsqueeze(0) if single else x
    b, six, nz, ny, nx = xb.shape
    if six != 6:
        raise ValueError("expected 6 Voigt components in dimension -4")
    plan = Plan(nx, ny, nz, x.dtype, b, op, h, nyq, device=x.device, target=target)
    o = plan.project(xb.contiguous(), None if out is None else out.view(xb.shape))
    nrm = plan.norms()
    plan.close()
    o = o.view(x.shape)
    return o, (nrm[0] if single else nrm)
