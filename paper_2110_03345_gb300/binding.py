"""ctypes binding of libfwi.so (include/fwi.h): argument marshalling only.

Every step of the solver runs in the CUDA library; this module converts torch
tensors and numpy arrays into the pointers and sizes of the C ABI and turns
status codes into exceptions.  There is no CPU fallback: if the library is
missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FWI_OK = 0
STATUS = {0: "FWI_OK", 1: "FWI_ERR_INVALID_ARG", 2: "FWI_ERR_UNSTABLE_CFL", 3: "FWI_ERR_BUDGET",
          4: "FWI_ERR_CUDA", 5: "FWI_ERR_NONFINITE", 6: "FWI_ERR_TIMEOUT",
          7: "FWI_ERR_UNSUPPORTED"}

# Every symbol include/fwi.h declares (checked by the tests).
EXPORTS = ("fwi_plan_create", "fwi_plan_set_options", "fwi_plan_stats", "fwi_plan_estimate",
           "fwi_plan_destroy", "fwi_forward", "fwi_gradient", "fwi_last_error", "fwi_cfl_limit",
           "fwi_forward_noalloc", "fwi_misfit_forward", "fwi_misfit_backward",
           "fwi_misfit_backward_ex",
           "fwi_batch_create", "fwi_batch_run", "fwi_batch_stats_get", "fwi_batch_destroy",
           "fwi_mem_available", "fwi_lowpass", "fwi_vp_update", "fwi_point_weights",
           "fwi_check_bounded_wait")


class FwiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class CGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("shape", ctypes.c_int64 * 3),
                ("spacing", ctypes.c_double * 3), ("order", ctypes.c_int),
                ("sponge", ctypes.c_int), ("c_ref", ctypes.c_double)]


PARAM_VP, PARAM_M = 0, 1


class CModel(ctypes.Structure):
    _fields_ = [("vp", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("param", ctypes.c_int),
                ("alpha0", ctypes.c_void_p), ("att_power", ctypes.c_int)]


class CGeometry(ctypes.Structure):
    _fields_ = [("nshots", ctypes.c_int), ("nsrc", ctypes.c_int), ("nrec", ctypes.c_int),
                ("src_xyz", ctypes.POINTER(ctypes.c_double)),
                ("rec_xyz", ctypes.POINTER(ctypes.c_double))]


class CProblem(ctypes.Structure):
    _fields_ = [("grid", CGrid), ("nt", ctypes.c_int), ("dt", ctypes.c_double),
                ("model", CModel), ("geom", CGeometry), ("wavelet", ctypes.c_void_p),
                ("traces", ctypes.c_void_p), ("observed", ctypes.c_void_p),
                ("grad_m", ctypes.c_void_p), ("misfit", ctypes.POINTER(ctypes.c_double))]


class CBatchStats(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int), ("units", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("updates", ctypes.c_int64),
                ("run_ms", ctypes.c_double), ("shots_per_cta", ctypes.c_int),
                ("checkpointed", ctypes.c_int)]


class COptions(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("tile", ctypes.c_int),
                ("profile", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("shots_per_cta", ctypes.c_int), ("time_order", ctypes.c_int),
                ("interp", ctypes.c_int), ("boundary", ctypes.c_int)]


class CStats(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("ckpt_every", ctypes.c_int), ("tile", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t), ("launches", ctypes.c_int64),
                ("updates", ctypes.c_int64), ("fwd_launches", ctypes.c_int64),
                ("adj_launches", ctypes.c_int64), ("fwd_ms", ctypes.c_double),
                ("adj_ms", ctypes.c_double), ("fwd_points", ctypes.c_int64),
                ("adj_points", ctypes.c_int64), ("fwd_timed", ctypes.c_int64),
                ("adj_timed", ctypes.c_int64)]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libfwi.so (building it first if it is missing and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise FwiError(4, f"{path} is missing; run the build first")
            _build.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        lib.fwi_plan_create.argtypes = [P(vp), P(CGrid), ctypes.c_int, ctypes.c_double,
                                        ctypes.c_size_t, vp]
        lib.fwi_plan_create.restype = ctypes.c_int
        lib.fwi_plan_set_options.argtypes = [vp, P(COptions)]
        lib.fwi_plan_set_options.restype = ctypes.c_int
        lib.fwi_plan_stats.argtypes = [vp, P(CStats)]
        lib.fwi_plan_stats.restype = ctypes.c_int
        lib.fwi_plan_estimate.argtypes = [vp, P(CGeometry), ctypes.c_int, P(ctypes.c_size_t)]
        lib.fwi_plan_estimate.restype = ctypes.c_int
        lib.fwi_plan_destroy.argtypes = [vp]
        lib.fwi_plan_destroy.restype = None
        lib.fwi_forward.argtypes = [vp, P(CModel), P(CGeometry), vp, ctypes.c_int, ctypes.c_double, vp]
        lib.fwi_forward.restype = ctypes.c_int
        lib.fwi_gradient.argtypes = [vp, P(CModel), P(CGeometry), vp, vp, P(ctypes.c_double), vp, vp]
        lib.fwi_gradient.restype = ctypes.c_int
        lib.fwi_last_error.argtypes = []
        lib.fwi_last_error.restype = ctypes.c_char_p
        lib.fwi_cfl_limit.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.fwi_cfl_limit.restype = ctypes.c_double
        lib.fwi_forward_noalloc.argtypes = [P(CGrid), ctypes.c_int, ctypes.c_double, P(CModel),
                                            P(CGeometry), vp, vp, vp]
        lib.fwi_forward_noalloc.restype = ctypes.c_int
        lib.fwi_misfit_forward.argtypes = [vp, P(CModel), P(CGeometry), vp, vp, P(ctypes.c_double), vp]
        lib.fwi_misfit_forward.restype = ctypes.c_int
        lib.fwi_misfit_backward.argtypes = [vp, vp]
        lib.fwi_misfit_backward.restype = ctypes.c_int
        lib.fwi_misfit_backward_ex.argtypes = [vp, vp, vp]
        lib.fwi_misfit_backward_ex.restype = ctypes.c_int
        lib.fwi_batch_create.argtypes = [P(vp), ctypes.c_int, P(CProblem), P(COptions),
                                         ctypes.c_size_t, vp, ctypes.c_int]
        lib.fwi_batch_create.restype = ctypes.c_int
        lib.fwi_mem_available.argtypes = [P(ctypes.c_size_t)]
        lib.fwi_mem_available.restype = ctypes.c_int
        lib.fwi_lowpass.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_int),
                                    ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    vp, vp]
        lib.fwi_lowpass.restype = ctypes.c_int
        lib.fwi_vp_update.argtypes = [vp, vp, vp, ctypes.c_longlong, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_float, vp, vp]
        lib.fwi_vp_update.restype = ctypes.c_int
        lib.fwi_point_weights.argtypes = [P(CGrid), P(ctypes.c_double), ctypes.c_int,
                                          P(ctypes.c_int64), P(ctypes.c_double), ctypes.c_int,
                                          P(ctypes.c_int)]
        lib.fwi_point_weights.restype = ctypes.c_int
        lib.fwi_batch_run.argtypes = [vp]
        lib.fwi_batch_run.restype = ctypes.c_int
        lib.fwi_batch_stats_get.argtypes = [vp, P(CBatchStats)]
        lib.fwi_batch_stats_get.restype = ctypes.c_int
        lib.fwi_batch_destroy.argtypes = [vp]
        lib.fwi_batch_destroy.restype = None
        lib.fwi_check_bounded_wait.argtypes = [ctypes.c_uint]
        lib.fwi_check_bounded_wait.restype = ctypes.c_int
        _lib = lib
        return lib


def _check(status: int):
    if status != FWI_OK:
        msg = load().fwi_last_error().decode(errors="replace")
        raise FwiError(status, msg)


def cfl_limit(ndim: int, order: int) -> float:
    return float(load().fwi_cfl_limit(ndim, order))


def mem_available() -> int:
    """fwi_mem_available: device bytes plan workspaces can still take (free
    memory plus the unused reserve of the stream-ordered pool)."""
    n = ctypes.c_size_t(0)
    _check(load().fwi_mem_available(ctypes.byref(n)))
    return int(n.value)


def check_bounded_wait(polls: int = 1000) -> int:
    """fwi_check_bounded_wait: one device thread waits, `polls` polls at most,
    on an mbarrier phase that nothing completes; returns the status
    (FWI_ERR_TIMEOUT when the wait gave up and flagged it, as expected)."""
    return int(load().fwi_check_bounded_wait(int(polls)))


def make_grid(shape, spacing, order=8, sponge=20, c_ref=0.0) -> CGrid:
    shape = tuple(int(v) for v in shape)
    if np.isscalar(spacing):
        spacing = (float(spacing),) * len(shape)
    g = CGrid()
    g.ndim = len(shape)
    for i in range(len(shape)):
        g.shape[i] = shape[i]
        g.spacing[i] = float(spacing[i])
    g.order, g.sponge, g.c_ref = int(order), int(sponge), float(c_ref)
    return g


def forward_noalloc(shape, spacing, nt, dt, vp, rho, geometry, wavelet, traces=None, order=8,
                    sponge=20, c_ref=0.0, stream=None):
    """fwi_forward_noalloc: forward modelling whose workspace is the library's
    fixed device scratch (no device allocation inside the call).  For callers
    that must not allocate device memory while they run; the caller still
    provides the inputs and the traces array."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(vp.device)
    # the C side runs on the current device: make it the stream's device, on
    # which every array must live (as for Plan)
    dev = _stream_device(stream)
    if traces is None:
        traces = torch.empty((geometry.nshots, geometry.nrec, int(nt)), device=dev,
                             dtype=torch.float32)
    n = int(np.prod(tuple(int(v) for v in shape)))
    check_array(vp, n, "vp", dev)
    check_array(rho, n, "rho", dev, optional=True)
    check_array(wavelet, geometry.nshots * geometry.nsrc * int(nt), "wavelet", dev)
    check_array(traces, geometry.nshots * geometry.nrec * int(nt), "traces", dev)
    g = make_grid(shape, spacing, order, sponge, c_ref)
    m = CModel(_ptr(vp), _ptr(rho))
    with torch.cuda.device(dev):
        _check(load().fwi_forward_noalloc(ctypes.byref(g), int(nt), float(dt), ctypes.byref(m),
                                          ctypes.byref(geometry.c), _ptr(wavelet), _ptr(traces),
                                          ctypes.c_void_p(stream.cuda_stream)))
    return traces


def _stream_device(stream):
    """torch.device of a CUDA stream (streams without a device attribute: the
    current device)."""
    import torch
    try:
        idx = stream.device.index
    except AttributeError:
        idx = None
    return torch.device("cuda", idx if idx is not None else torch.cuda.current_device())


LOWPASS_MAX_HALF_WIDTH = 2048
INTERP_LINEAR, INTERP_SINC = 0, 1
BOUNDARY_SPONGE, BOUNDARY_PML = 0, 1


def point_weights(shape, spacing, xyz, interp=INTERP_LINEAR, order=8, sponge=0):
    """fwi_point_weights (host only): (nodes [count][ndim], weights [count])
    of one off-grid point, bi-/tri-linear or Kaiser-windowed sinc."""
    g = make_grid(shape, spacing, order, sponge, 0.0)
    nd = len(tuple(shape))
    x = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(nd))
    cnt = ctypes.c_int(0)
    lib = load()
    dp = ctypes.POINTER(ctypes.c_double)
    st = lib.fwi_point_weights(ctypes.byref(g), x.ctypes.data_as(dp), int(interp), None, None, 0,
                               ctypes.byref(cnt))
    if cnt.value == 0:
        _check(st)
    nodes = np.zeros((cnt.value, nd), dtype=np.int64)
    w = np.zeros(cnt.value)
    _check(lib.fwi_point_weights(ctypes.byref(g), x.ctypes.data_as(dp), int(interp),
                                 nodes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 w.ctypes.data_as(dp), cnt.value, ctypes.byref(cnt)))
    return nodes, w


def lowpass(x, ids, dt, f_max, half_width, out=None, stream=None):
    """fwi_lowpass: out[i] = zero-phase low-pass (cut-off f_max, half-width
    `half_width` samples) of x[ids[i]] along the last axis.  x: CUDA float32
    [n][rows][nt]; ids: host integers; out: [len(ids)][rows][nt] or None."""
    import torch
    if x.dim() != 3:
        raise ValueError("x must be [n][rows][nt]")
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64).reshape(-1)).astype(np.int32)
    n, rows, nt = (int(v) for v in x.shape)
    if out is None:
        out = torch.empty((len(ids), rows, nt), device=x.device, dtype=torch.float32)
    if tuple(out.shape) != (len(ids), rows, nt):
        raise ValueError("out must be [len(ids)][rows][nt]")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().fwi_lowpass(_ptr(x), n, rows, nt,
                              ids.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), len(ids),
                              float(dt), float(f_max), int(half_width), _ptr(out),
                              ctypes.c_void_p(stream.cuda_stream)))
    return out


def vp_update(vp, grad_m, step, vp_min, vp_max, mask=None, work=None, stream=None):
    """fwi_vp_update: one normalised gradient-descent step on vp (in place):
    the largest change is `step`, restricted to `mask`, clipped to
    [vp_min, vp_max].  work: a CUDA float32 tensor of >= 1 element or None."""
    import torch
    if grad_m.numel() != vp.numel() or (mask is not None and mask.numel() != vp.numel()):
        raise ValueError("vp, grad_m and mask must have the same size")
    if work is None:
        work = torch.empty(1, device=vp.device, dtype=torch.float32)
    if work.numel() < 1:
        raise ValueError("work must hold at least one element")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().fwi_vp_update(_ptr(vp), _ptr(grad_m), _ptr(mask), int(vp.numel()),
                                float(step), float(vp_min), float(vp_max), _ptr(work),
                                ctypes.c_void_p(stream.cuda_stream)))
    return vp


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def check_array(t, count, name, device=None, optional=False):
    """Raise ValueError unless `t` holds exactly `count` elements (and lies on
    `device` when given).  The C ABI takes bare device pointers and cannot see
    a tensor's size: a short array would be read or written past its end."""
    if t is None:
        if optional:
            return
        raise ValueError(f"{name} is required")
    if int(t.numel()) != int(count):
        raise ValueError(f"{name} holds {int(t.numel())} elements, expected {int(count)}")
    if device is not None and getattr(t, "device", None) is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, the plan runs on {device}")


class Geometry:
    """Host-side acquisition geometry: src_xyz [nshots][nsrc][ndim], rec_xyz [nrec][ndim]."""

    def __init__(self, src_xyz, rec_xyz):
        self.src = np.ascontiguousarray(src_xyz, dtype=np.float64)
        self.rec = np.ascontiguousarray(rec_xyz, dtype=np.float64)
        if self.src.ndim == 2:
            self.src = self.src[None]
        if self.src.ndim != 3 or self.rec.ndim != 2 or self.src.shape[2] != self.rec.shape[1]:
            raise ValueError("src_xyz must be [nshots][nsrc][ndim] and rec_xyz [nrec][ndim]")
        dp = ctypes.POINTER(ctypes.c_double)
        self.c = CGeometry(self.src.shape[0], self.src.shape[1], self.rec.shape[0],
                           self.src.ctypes.data_as(dp), self.rec.ctypes.data_as(dp))

    @property
    def nshots(self):
        return self.src.shape[0]

    @property
    def nsrc(self):
        return self.src.shape[1]

    @property
    def nrec(self):
        return self.rec.shape[0]


class Plan:
    """A solver plan for one grid and time axis (fwi_plan_create)."""

    def __init__(self, shape, spacing, nt, dt, order=8, sponge=20, c_ref=0.0, budget=0,
                 stream=None):
        import torch
        lib = load()
        shape = tuple(int(s) for s in shape)
        nd = len(shape)
        if np.isscalar(spacing):
            spacing = (float(spacing),) * nd
        g = CGrid()
        g.ndim = nd
        for i in range(nd):
            g.shape[i] = shape[i]
            g.spacing[i] = float(spacing[i])
        g.order, g.sponge, g.c_ref = int(order), int(sponge), float(c_ref)
        self.shape, self.spacing, self.nt, self.dt = shape, tuple(spacing), int(nt), float(dt)
        self.order, self.sponge = order, sponge
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.device = _stream_device(stream)
        self.npoints = int(np.prod(shape))
        h = ctypes.c_void_p()
        _check(lib.fwi_plan_create(ctypes.byref(h), ctypes.byref(g), self.nt, self.dt,
                                   int(budget), ctypes.c_void_p(stream.cuda_stream)))
        self._h = h
        self._opts = COptions()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().fwi_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close

    def set_options(self, batch=0, ckpt_every=0, tile=0, profile=False, shots_per_cta=0,
                    time_order=0, interp=INTERP_LINEAR, boundary=BOUNDARY_SPONGE):
        """tile: 0 default; 2D 1-4 shared-memory staged (one shot per CTA), 5-8
        TMA-staged with shots looped inside a CTA; 3D 1-4 shared-memory staged,
        5-8 TMA plane ring, 9-12 TMA plane ring with two x points per thread.
        shots_per_cta: 2D TMA variants only.  time_order: 2 (leapfrog) or 4
        (fourth order in time).  interp: INTERP_LINEAR or INTERP_SINC points.
        boundary: BOUNDARY_SPONGE or BOUNDARY_PML."""
        # profile: True / 1 times every stencil launch, n > 1 every n-th
        self._opts = COptions(int(batch), int(ckpt_every), int(tile), int(profile),
                              0, int(shots_per_cta), int(time_order), int(interp), int(boundary))
        _check(load().fwi_plan_set_options(self._h, ctypes.byref(self._opts)))

    def stats(self) -> dict:
        s = CStats()
        _check(load().fwi_plan_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in CStats._fields_}

    def estimate(self, geometry: Geometry, gradient: bool) -> int:
        b = ctypes.c_size_t()
        _check(load().fwi_plan_estimate(self._h, ctypes.byref(geometry.c), int(gradient),
                                        ctypes.byref(b)))
        return int(b.value)

    def set_attenuation(self, alpha0=None, power=0):
        """Power-law attenuation of Eq. 10 for the following calls: alpha0 a
        CUDA float32 field of the grid's size (None: no attenuation), power
        y = 0 or 2.  The tensor must stay alive while it is set."""
        check_array(alpha0, self.npoints, "alpha0", self.device, optional=True)
        self._att = (alpha0, int(power))

    def _model(self, vp, rho, param=PARAM_VP):
        check_array(vp, self.npoints, "vp", self.device)
        check_array(rho, self.npoints, "rho", self.device, optional=True)
        alpha0, power = getattr(self, "_att", (None, 0))
        return CModel(_ptr(vp), _ptr(rho), int(param), _ptr(alpha0), int(power))

    def _check_shots(self, geometry, wavelet, traces=None, observed=None):
        ns, nrec = geometry.nshots, geometry.nrec
        check_array(wavelet, ns * geometry.nsrc * self.nt, "wavelet", self.device)
        check_array(observed, ns * nrec * self.nt, "observed", self.device, optional=True)
        check_array(traces, ns * nrec * self.nt, "traces", self.device, optional=True)

    def forward(self, vp, rho, geometry: Geometry, wavelet, traces=None):
        """Traces [nshots][nrec][nt] (CUDA float32) for the given wavelets."""
        import torch
        if traces is None:
            traces = torch.empty((geometry.nshots, geometry.nrec, self.nt), device=vp.device,
                                 dtype=torch.float32)
        m = self._model(vp, rho)
        self._check_shots(geometry, wavelet, traces=traces)
        _check(load().fwi_forward(self._h, ctypes.byref(m), ctypes.byref(geometry.c),
                                  _ptr(wavelet), self.nt, self.dt, _ptr(traces)))
        return traces

    def misfit_forward(self, vp, rho, geometry: Geometry, wavelet, observed, traces=False,
                       param=PARAM_VP):
        """J (and the traces if asked); keeps what misfit_backward needs in the plan.
        param=PARAM_M: `vp` holds the squared slowness m = 1/vp^2 instead."""
        import torch
        tr = None
        if traces is True:
            tr = torch.empty((geometry.nshots, geometry.nrec, self.nt), device=vp.device,
                             dtype=torch.float32)
        J = ctypes.c_double()
        m = self._model(vp, rho, param)
        self._check_shots(geometry, wavelet, traces=tr, observed=observed)
        check_array(observed, geometry.nshots * geometry.nrec * self.nt, "observed", self.device)
        self._kept = (vp, rho, geometry, wavelet, observed)   # must outlive the backward
        _check(load().fwi_misfit_forward(self._h, ctypes.byref(m), ctypes.byref(geometry.c),
                                         _ptr(wavelet), _ptr(observed), ctypes.byref(J), _ptr(tr)))
        return J.value, tr

    def misfit_backward(self, grad=None):
        """Gradient w.r.t. m = 1/vp^2 of the misfit of the last misfit_forward."""
        import torch
        if getattr(self, "_kept", None) is None:
            raise FwiError(1, "no pending misfit_forward on this plan")
        vp = self._kept[0]
        if grad is None:
            grad = torch.empty(vp.shape, device=vp.device, dtype=torch.float32)
        check_array(grad, self.npoints, "grad", self.device)
        try:
            _check(load().fwi_misfit_backward(self._h, _ptr(grad)))
        finally:
            self._kept = None
        return grad

    def misfit_backward_ex(self, grad=True, grad_wavelet=True):
        """(dJ/dm or None, dJ/dq or None) of the last misfit_forward: the
        gradient with respect to m = 1/vp^2 and with respect to the source
        wavelets ([nshots][nsrc][nt]); True allocates an output, None skips it,
        a tensor is written in place."""
        import torch
        if getattr(self, "_kept", None) is None:
            raise FwiError(1, "no pending misfit_forward on this plan")
        vp, _, geometry, wavelet, _ = self._kept
        if grad is True:
            grad = torch.empty(vp.shape, device=vp.device, dtype=torch.float32)
        if grad_wavelet is True:
            grad_wavelet = torch.empty(tuple(wavelet.shape), device=vp.device, dtype=torch.float32)
        check_array(grad, self.npoints, "grad", self.device, optional=True)
        check_array(grad_wavelet, geometry.nshots * geometry.nsrc * self.nt, "grad_wavelet",
                    self.device, optional=True)
        try:
            _check(load().fwi_misfit_backward_ex(self._h, _ptr(grad), _ptr(grad_wavelet)))
        finally:
            self._kept = None
        return grad, grad_wavelet

    def gradient(self, vp, rho, geometry: Geometry, wavelet, observed, grad=None, traces=False):
        """(J, grad_m, traces or None): L2 misfit and its gradient w.r.t. m = 1/vp^2."""
        import torch
        if grad is None:
            grad = torch.empty(vp.shape, device=vp.device, dtype=torch.float32)
        tr = None
        if traces is True:
            tr = torch.empty((geometry.nshots, geometry.nrec, self.nt), device=vp.device,
                             dtype=torch.float32)
        elif traces is not False and traces is not None:
            tr = traces
        J = ctypes.c_double()
        m = self._model(vp, rho)
        self._check_shots(geometry, wavelet, traces=tr, observed=observed)
        check_array(observed, geometry.nshots * geometry.nrec * self.nt, "observed", self.device)
        check_array(grad, self.npoints, "grad", self.device)
        _check(load().fwi_gradient(self._h, ctypes.byref(m), ctypes.byref(geometry.c),
                                   _ptr(wavelet), _ptr(observed), ctypes.byref(J), _ptr(grad),
                                   _ptr(tr)))
        return J.value, grad, tr


class Batch:
    """fwi_batch: many independent 2D problems advanced together, one
    multi-problem launch per time step, optionally one CUDA graph per run.

    problems: list of dicts with keys shape, spacing, nt, dt, order, sponge,
    c_ref, vp, rho (CUDA tensors or None), geometry (Geometry), wavelet (CUDA
    tensor [shots][src][nt]), and for a gradient batch observed (CUDA tensor
    [shots][rec][nt]).  Traces are allocated here (self.traces); a gradient
    batch also allocates self.grads (dJ/dm per problem) and fills
    self.misfits at each run."""

    def __init__(self, problems, budget=0, stream=None, use_graph=True, tile=0, shots_per_cta=0,
                 gradient=False):
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._keep = []
        self.traces = []
        self.grads = []
        self.gradient = bool(gradient)
        self._misfit = (ctypes.c_double * len(problems))()
        arr = (CProblem * len(problems))()
        for i, pr in enumerate(problems):
            geo = pr["geometry"]
            n = int(np.prod(tuple(int(v) for v in pr["shape"])))
            dev = pr["vp"].device
            check_array(pr["vp"], n, f"problem {i} vp", dev)
            check_array(pr.get("rho"), n, f"problem {i} rho", dev, optional=True)
            check_array(pr["wavelet"], geo.nshots * geo.nsrc * int(pr["nt"]),
                        f"problem {i} wavelet", dev)
            tr = torch.empty((geo.nshots, geo.nrec, int(pr["nt"])), device=pr["vp"].device,
                             dtype=torch.float32)
            self.traces.append(tr)
            self._keep.append((pr["vp"], pr.get("rho"), geo, pr["wavelet"], tr))
            arr[i].grid = make_grid(pr["shape"], pr["spacing"], pr.get("order", 8),
                                    pr.get("sponge", 20), pr.get("c_ref", 0.0))
            arr[i].nt = int(pr["nt"])
            arr[i].dt = float(pr["dt"])
            arr[i].model = CModel(_ptr(pr["vp"]), _ptr(pr.get("rho")), 0)
            arr[i].geom = geo.c
            arr[i].wavelet = _ptr(pr["wavelet"])
            arr[i].traces = _ptr(tr)
            if self.gradient:
                check_array(pr["observed"], geo.nshots * geo.nrec * int(pr["nt"]),
                            f"problem {i} observed", dev)
                g = torch.empty(tuple(int(v) for v in pr["shape"]), device=dev, dtype=torch.float32)
                self.grads.append(g)
                self._keep.append((pr["observed"], g))
                arr[i].observed = _ptr(pr["observed"])
                arr[i].grad_m = _ptr(g)
                arr[i].misfit = ctypes.cast(ctypes.byref(self._misfit, i * ctypes.sizeof(ctypes.c_double)),
                                            ctypes.POINTER(ctypes.c_double))
        self._arr = arr
        self._opts = COptions(0, 0, int(tile), 0, 0, int(shots_per_cta), 0, 0, 0)
        h = ctypes.c_void_p()
        _check(lib.fwi_batch_create(ctypes.byref(h), len(problems), arr, ctypes.byref(self._opts),
                                    int(budget), ctypes.c_void_p(stream.cuda_stream),
                                    int(bool(use_graph))))
        self._h = h

    def run(self):
        """Forward batch: the traces; gradient batch: (misfits, gradients)."""
        _check(load().fwi_batch_run(self._h))
        if self.gradient:
            return [float(v) for v in self._misfit], self.grads
        return self.traces

    def stats(self) -> dict:
        s = CBatchStats()
        _check(load().fwi_batch_stats_get(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in CBatchStats._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().fwi_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    __del__ = close
