"""ctypes binding of libashrt (argument marshalling only).

Every computation runs in the CUDA library; this module converts Python
arguments (torch CUDA tensors or raw device addresses, host float arrays) to
the C ABI of ``include/ashrt.h`` and raises ``AshrtError`` on a non-OK status.
There is no fallback: if the library is missing, ``load()`` raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libashrt.so")

c_int, c_float, c_double, c_void_p, c_size_t = (ctypes.c_int, ctypes.c_float, ctypes.c_double,
                                                 ctypes.c_void_p, ctypes.c_size_t)

STATUS = {0: "ASHRT_OK", 1: "ASHRT_EINVAL", 2: "ASHRT_ENOMEM", 3: "ASHRT_ECUDA",
          4: "ASHRT_ENAN", 5: "ASHRT_ENOTCONV", 6: "ASHRT_ETIMEOUT", 7: "ASHRT_EINTERNAL"}


class AshrtOpts(ctypes.Structure):
    _fields_ = [("pad_t", c_int), ("pad_x", c_int), ("fmax_hz", c_float),
                ("wavelet_peak_hz", c_float), ("max_batch", c_int), ("with_solver", c_int)]


class IrlsOpts(ctypes.Structure):
    _fields_ = [("p", c_double), ("q", c_double), ("n_outer", c_int), ("n_cg", c_int),
                ("tol", c_double), ("b_r", c_double), ("b_m", c_double), ("mu", c_double),
                ("warm_start_cg", c_int), ("eps_r_fixed", c_double), ("eps_m_fixed", c_double),
                ("trace_mask_dev", c_void_p), ("apex_mask_dev", c_void_p), ("use_graph", c_int),
                ("m0_dev", c_void_p), ("wr0_dev", c_void_p), ("wr_out_dev", c_void_p)]


class IrlsReport(ctypes.Structure):
    _fields_ = [("outer_done", c_int), ("applies_fwd", c_int), ("applies_adj", c_int),
                ("flags", c_int), ("misfit", c_double * 64)]


class FistaOpts(ctypes.Structure):
    _fields_ = [("mu", c_double), ("n_iter", c_int), ("n_power", c_int)]


class AshrtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load():
    """Load libashrt.so (built in-tree by ``build.py``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libashrt.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    try:  # the library links the shared CUDA runtime that torch has already loaded
        import torch  # noqa: F401
    except ImportError:
        pass
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.ashrt_default_opts.argtypes = [P(AshrtOpts)]
    lib.ashrt_default_opts.restype = None
    lib.irls_default_opts.argtypes = [P(IrlsOpts)]
    lib.irls_default_opts.restype = None
    lib.ashrt_plan_create.argtypes = [P(c_void_p), c_int, c_int, c_double, c_double,
                                      P(c_float), c_int, P(c_float), c_int, P(c_float), c_int,
                                      P(AshrtOpts)]
    lib.ashrt_plan_create.restype = c_int
    lib.ashrt_plan_create_irregular.argtypes = [P(c_void_p), c_int, c_int, c_double, c_double,
                                                P(c_float), c_int, P(c_float), c_int,
                                                P(c_double), c_int, P(AshrtOpts)]
    lib.ashrt_plan_create_irregular.restype = c_int
    lib.ashrt_plan_destroy.argtypes = [c_void_p]
    lib.ashrt_plan_destroy.restype = None
    lib.ashrt_plan_info.argtypes = [c_void_p, P(c_int), P(c_int), P(c_int), P(c_size_t)]
    lib.ashrt_plan_info.restype = c_int
    for name in ("ashrt_forward", "ashrt_adjoint"):
        f = getattr(lib, name)
        f.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p]
        f.restype = c_int
    lib.robust_irls_deblend.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                        P(IrlsOpts), P(IrlsReport), c_void_p]
    lib.robust_irls_deblend.restype = c_int
    lib.ashrt_forward_static.argtypes = [c_int, c_int, c_double, c_double, P(c_float), c_int,
                                         P(c_float), c_int, P(AshrtOpts), c_void_p, c_void_p,
                                         c_void_p, c_int, c_void_p]
    lib.ashrt_forward_static.restype = c_int
    lib.fista_default_opts.argtypes = [P(FistaOpts)]
    lib.fista_default_opts.restype = None
    lib.ashrt_fista.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                P(FistaOpts), P(c_double), c_void_p]
    lib.ashrt_fista.restype = c_int
    lib.ashrt_blend.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p, c_int,
                                c_void_p]
    lib.ashrt_pseudo_deblend.argtypes = [c_void_p, c_int, c_int, c_void_p, c_int, c_int,
                                         c_void_p, c_void_p]
    lib.ashrt_sort_gathers.argtypes = [c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]
    for f in (lib.ashrt_blend, lib.ashrt_pseudo_deblend, lib.ashrt_sort_gathers):
        f.restype = c_int
    for f in (lib.ashrt_td_forward, lib.ashrt_td_adjoint):
        f.argtypes = [c_int, c_int, c_double, c_double, P(c_float), c_int, P(c_float), c_int,
                      c_void_p, c_void_p, c_int, c_void_p]
        f.restype = c_int
    lib.ashrt_batch_create.argtypes = [P(c_void_p), c_int, P(c_int), c_int, c_double, c_double,
                                       P(c_float), c_int, P(c_float), c_int, P(AshrtOpts)]
    lib.ashrt_batch_create.restype = c_int
    lib.ashrt_batch_create_uneven.argtypes = [P(c_void_p), P(c_int), P(c_int), c_int, c_double,
                                              c_double, P(c_float), c_int, P(c_float), c_int,
                                              P(AshrtOpts)]
    lib.ashrt_batch_create_uneven.restype = c_int
    lib.ashrt_batch_destroy.argtypes = [c_void_p]
    lib.ashrt_batch_destroy.restype = None
    lib.ashrt_batch_autotune.argtypes = [c_void_p, ctypes.c_char_p]
    lib.ashrt_batch_autotune.restype = c_int
    lib.ashrt_batch_info.argtypes = [c_void_p, P(c_int), P(ctypes.c_longlong),
                                     P(ctypes.c_longlong), P(c_size_t)]
    lib.ashrt_batch_info.restype = c_int
    for name in ("ashrt_batch_forward", "ashrt_batch_adjoint"):
        f = getattr(lib, name)
        f.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
        f.restype = c_int
    lib.ashrt_batch_deblend.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, P(IrlsOpts),
                                        P(IrlsReport), c_void_p]
    lib.ashrt_batch_deblend.restype = c_int
    lib.ashrt_plan_autotune.argtypes = [c_void_p, c_int, ctypes.c_char_p, ctypes.POINTER(c_int),
                                        ctypes.POINTER(c_int)]
    lib.ashrt_plan_autotune.restype = c_int
    lib.ashrt_plan_set_variant.argtypes = [c_void_p, c_int, c_int]
    lib.ashrt_plan_set_variant.restype = c_int
    lib.ashrt_unet_create.argtypes = [P(c_void_p), c_int, c_int, c_int, c_int, P(c_float),
                                      ctypes.c_longlong]
    lib.ashrt_unet_create.restype = c_int
    lib.ashrt_unet_destroy.argtypes = [c_void_p]
    lib.ashrt_unet_destroy.restype = None
    lib.ashrt_unet_param_count.argtypes = [c_void_p]
    lib.ashrt_unet_param_count.restype = ctypes.c_longlong
    lib.ashrt_unet_get.argtypes = [c_void_p, P(c_float), P(c_float), ctypes.c_longlong]
    lib.ashrt_unet_get.restype = c_int
    lib.ashrt_unet_forward.argtypes = [c_void_p, c_void_p, c_void_p, c_int, c_int, c_float,
                                       c_void_p]
    lib.ashrt_unet_forward.restype = c_int
    lib.ashrt_unet_train_step.argtypes = [c_void_p, c_void_p, c_void_p, c_int, P(c_float),
                                          c_float, P(c_double), c_void_p]
    lib.ashrt_unet_train_step.restype = c_int
    lib.ashrt_unet_targets.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                       c_float, c_void_p]
    lib.ashrt_unet_targets.restype = c_int
    lib.ashrt_unet_predict.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_float,
                                       c_void_p]
    lib.ashrt_unet_predict.restype = c_int
    lib.ashrt_last_error.argtypes = []
    lib.ashrt_last_error.restype = ctypes.c_char_p
    lib.ashrt_profile_enable.argtypes = [c_int]
    lib.ashrt_profile_enable.restype = None
    lib.ashrt_profile_read.argtypes = [ctypes.POINTER(c_double), ctypes.POINTER(ctypes.c_longlong),
                                       c_int]
    lib.ashrt_profile_read.restype = c_int
    lib.ashrt_kernel_launches.argtypes = []
    lib.ashrt_kernel_launches.restype = ctypes.c_longlong
    lib.ashrt_fp32_peak.argtypes = [c_int, c_int, P(c_double), P(c_int), c_void_p]
    lib.ashrt_fp32_peak.restype = c_int
    lib.ashrt_quality_db.argtypes = [c_void_p, c_void_p, c_int, ctypes.c_longlong, c_void_p,
                                     P(c_double), c_void_p]
    lib.ashrt_quality_db.restype = c_int
    lib.ashrt_status_string.argtypes = [c_int]
    lib.ashrt_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise AshrtError(status, load().ashrt_last_error().decode())


def _ptr(x):
    """Device address of a torch tensor (checked contiguous float32) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda or x.dtype.itemsize != 4 or not x.is_contiguous():
        raise ValueError("expected a contiguous 4-byte CUDA tensor")
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _farr(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32).ravel())
    return a, a.ctypes.data_as(ctypes.POINTER(c_float))


PROFILE_CLASSES = ("xfft_r2c", "stolt_fwd_rows", "stolt_adj_rows", "xfft_c2r", "solver",
                   "xfft_r2c_data", "xfft_c2r_data")


def profile_enable(on=True):
    load().ashrt_profile_enable(1 if on else 0)


def profile_read():
    """{class: (total_ms, launches)} since the previous read (see ashrt_profile_read)."""
    n = len(PROFILE_CLASSES)
    ms = (c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    st = load().ashrt_profile_read(ms, cnt, n)
    if st != 0:
        raise AshrtError(7, "profile events could not be read")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(PROFILE_CLASSES)}


def kernel_launches():
    return int(load().ashrt_kernel_launches())


def fp32_peak(iters=20000, reps=5, stream=None):
    """ashrt_fp32_peak: measured FP32 FMA rate of the device, (TFLOP/s, SM count)."""
    t, n = c_double(), c_int()
    _check(load().ashrt_fp32_peak(int(iters), int(reps), ctypes.byref(t), ctypes.byref(n),
                                  _stream(stream)))
    return t.value, n.value


def quality_db(d_orig, d_test, sums, batch=None, n=None, sync=True, stream=None):
    """ashrt_quality_db: per-gather Q = 10 log10(||d_o||^2 / ||d_o - d_t||^2) in dB
    (FP64 sums in the device array ``sums`` [batch][2] of float64).  With
    sync=False the call stays asynchronous, returns None and leaves the sums."""
    b = int(batch if batch is not None else d_orig.shape[0])
    n = int(n if n is not None else d_orig.numel() // b)
    if sums.dtype.itemsize != 8 or not sums.is_cuda or not sums.is_contiguous() or \
            sums.numel() < 2 * b:
        raise ValueError("sums must be a contiguous CUDA float64 tensor of >= 2 * batch elements")
    q = (c_double * b)() if sync else None
    _check(load().ashrt_quality_db(_ptr(d_orig), _ptr(d_test), b, n, sums.data_ptr(), q,
                                   _stream(stream)))
    return list(q) if sync else None


def forward_static(nt, nx, dt, dx, velocities, m, d, t0s=None, mask=None, batch=1, pad_t=2,
                   pad_x=2, fmax_hz=0.0, wavelet_peak_hz=0.0, stream=None):
    """ashrt_forward_static: the forward operator with no plan and no device
    allocation (tables and workspace in the library's static scratch)."""
    lib = load()
    o = AshrtOpts()
    lib.ashrt_default_opts(ctypes.byref(o))
    o.pad_t, o.pad_x = int(pad_t), int(pad_x)
    o.fmax_hz, o.wavelet_peak_hz = float(fmax_hz), float(wavelet_peak_hz)
    va, vp = _farr(velocities)
    if t0s is None:
        tp, nt0 = None, 1
    else:
        ta, tp = _farr(t0s)
        nt0 = ta.size
    _check(lib.ashrt_forward_static(int(nt), int(nx), float(dt), float(dx), vp, va.size, tp,
                                    nt0, ctypes.byref(o), _ptr(m), _ptr(d), _ptr(mask),
                                    int(batch), _stream(stream)))


def blend(shots, fire, record, stream=None):
    """ashrt_blend: shots [ns][nr][nt] -> record [nr][nb]; fire int32 [ns]."""
    ns, nr, nt = shots.shape
    _check(load().ashrt_blend(_ptr(shots), ns, nr, nt, _ptr(fire), _ptr(record),
                              record.shape[-1], _stream(stream)))


def pseudo_deblend(record, fire, shots, stream=None):
    """ashrt_pseudo_deblend: record [nr][nb] -> shots [ns][nr][nt]."""
    nr, nb = record.shape
    _check(load().ashrt_pseudo_deblend(_ptr(record), nr, nb, _ptr(fire), shots.shape[0],
                                       shots.shape[2], _ptr(shots), _stream(stream)))


def sort_gathers(src, dst, stream=None):
    """ashrt_sort_gathers: src [n0][n1][nt] -> dst [n1][n0][nt]."""
    n0, n1, nt = src.shape
    _check(load().ashrt_sort_gathers(_ptr(src), n0, n1, nt, _ptr(dst), _stream(stream)))


def _td(fn, nt, nx, dt, dx, velocities, src, dst, t0s, batch, stream):
    va, vp = _farr(velocities)
    if t0s is None:
        tp, nt0 = None, 1
    else:
        ta, tp = _farr(t0s)
        nt0 = ta.size
    _check(fn(int(nt), int(nx), float(dt), float(dx), vp, va.size, tp, nt0, _ptr(src), _ptr(dst),
              int(batch), _stream(stream)))


def td_forward(nt, nx, dt, dx, velocities, m, d, t0s=None, batch=1, stream=None):
    """ashrt_td_forward: time-domain (hyperbolic summation) forward, m -> d."""
    _td(load().ashrt_td_forward, nt, nx, dt, dx, velocities, m, d, t0s, batch, stream)


def td_adjoint(nt, nx, dt, dx, velocities, d, m, t0s=None, batch=1, stream=None):
    """ashrt_td_adjoint: time-domain (hyperbolic summation) adjoint, d -> m."""
    _td(load().ashrt_td_adjoint, nt, nx, dt, dx, velocities, d, m, t0s, batch, stream)


class Plan:
    """A Stolt ASHRT/AASHRT plan (see ashrt_plan_create in include/ashrt.h)."""

    def __init__(self, nt, nx, dt, dx, velocities, t0s=None, apex_x=None, pad_t=2, pad_x=2,
                 fmax_hz=0.0, wavelet_peak_hz=0.0, max_batch=1, with_solver=False,
                 trace_x=None):
        """trace_x: positions [m] of the data traces (ashrt_plan_create_irregular);
        None for traces at the apex positions j dx."""
        lib = load()
        o = AshrtOpts()
        lib.ashrt_default_opts(ctypes.byref(o))
        o.pad_t, o.pad_x = int(pad_t), int(pad_x)
        o.fmax_hz, o.wavelet_peak_hz = float(fmax_hz), float(wavelet_peak_hz)
        o.max_batch, o.with_solver = int(max_batch), int(bool(with_solver))
        self._v, vp = _farr(velocities)
        if t0s is None:
            self._t0, tp, nt0 = None, None, 1
        else:
            self._t0, tp = _farr(t0s)
            nt0 = self._t0.size
        if apex_x is None:
            ap, na = None, 0
        else:
            self._ax, ap = _farr(apex_x)
            na = self._ax.size
        h = c_void_p()
        self._h = None
        if trace_x is None:
            _check(lib.ashrt_plan_create(ctypes.byref(h), int(nt), int(nx), float(dt), float(dx),
                                         vp, self._v.size, ap, na, tp, nt0, ctypes.byref(o)))
            self.nr = int(nx)
        else:
            if apex_x is not None:
                raise ValueError("apex_x and trace_x cannot both be given")
            self._tx = np.ascontiguousarray(np.asarray(trace_x, dtype=np.float64).ravel())
            _check(lib.ashrt_plan_create_irregular(
                ctypes.byref(h), int(nt), int(nx), float(dt), float(dx), vp, self._v.size, tp, nt0,
                self._tx.ctypes.data_as(ctypes.POINTER(c_double)), self._tx.size,
                ctypes.byref(o)))
            self.nr = self._tx.size
        self._h = h.value
        self.nt, self.nx, self.nv, self.nt0 = int(nt), int(nx), self._v.size, nt0
        self.max_batch = int(max_batch)
        Nt, Nx, P, ws = c_int(), c_int(), c_int(), c_size_t()
        _check(lib.ashrt_plan_info(self._h, ctypes.byref(Nt), ctypes.byref(Nx), ctypes.byref(P),
                                   ctypes.byref(ws)))
        self.Nt, self.Nx, self.P, self.workspace_bytes = Nt.value, Nx.value, P.value, ws.value

    @property
    def model_shape(self):
        return (self.nt0, self.nv, self.nx, self.nt)

    @property
    def data_shape(self):
        return (self.nr, self.nt)

    def forward(self, m, d, mask=None, batch=1, stream=None):
        _check(load().ashrt_forward(self._h, _ptr(m), _ptr(d), _ptr(mask), int(batch),
                                    _stream(stream)))

    def adjoint(self, d, m, mask=None, batch=1, stream=None):
        _check(load().ashrt_adjoint(self._h, _ptr(d), _ptr(m), _ptr(mask), int(batch),
                                    _stream(stream)))

    def autotune(self, batch=None, cache_path=None):
        """ashrt_plan_autotune: returns (rows_minb, xfft_cols) chosen for this plan."""
        mb, cols = c_int(), c_int()
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(load().ashrt_plan_autotune(self._h, int(batch or self.max_batch), path,
                                          ctypes.byref(mb), ctypes.byref(cols)))
        return mb.value, cols.value

    def set_variant(self, rows_minb, xfft_cols):
        _check(load().ashrt_plan_set_variant(self._h, int(rows_minb), int(xfft_cols)))

    def fista(self, d, m, v0, drec=None, mask=None, batch=1, stream=None, mu=0.0, n_iter=50,
              n_power=20):
        """ashrt_fista: l2-l1 sparse inversion (FISTA, power-method step).
        Returns the per-gather Lipschitz constants Lf."""
        lib = load()
        o = FistaOpts()
        lib.fista_default_opts(ctypes.byref(o))
        o.mu, o.n_iter, o.n_power = float(mu), int(n_iter), int(n_power)
        lf = (c_double * int(batch))()
        _check(lib.ashrt_fista(self._h, _ptr(d), _ptr(mask), _ptr(v0), _ptr(m), _ptr(drec),
                               int(batch), ctypes.byref(o), lf, _stream(stream)))
        return list(lf)

    def deblend(self, d, m, drec=None, batch=1, stream=None, mask=None, apex_mask=None, m0=None,
                wr0=None, wr_out=None, **kw):
        """robust_irls_deblend; keyword options are irls_opts fields. Returns reports."""
        lib = load()
        o = IrlsOpts()
        lib.irls_default_opts(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError("unknown irls option %r" % k)
            setattr(o, k, v)
        o.trace_mask_dev = _ptr(mask)
        o.apex_mask_dev = _ptr(apex_mask)
        o.m0_dev = _ptr(m0)
        o.wr0_dev = _ptr(wr0)
        o.wr_out_dev = _ptr(wr_out)
        reps = (IrlsReport * int(batch))()
        _check(lib.robust_irls_deblend(self._h, _ptr(d), _ptr(m), _ptr(drec), int(batch),
                                       ctypes.byref(o), reps, _stream(stream)))
        return [dict(outer_done=r.outer_done, applies_fwd=r.applies_fwd,
                     applies_adj=r.applies_adj, flags=r.flags,
                     misfit=list(r.misfit[:r.outer_done])) for r in reps]

    def close(self):
        if self._h:
            load().ashrt_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _reports(reps):
    return [dict(outer_done=r.outer_done, applies_fwd=r.applies_fwd, applies_adj=r.applies_adj,
                 flags=r.flags, misfit=list(r.misfit[:r.outer_done])) for r in reps]


class Batch:
    """Uneven batch of gathers (see ashrt_batch_create in include/ashrt.h).
    nt is one sample count for every gather or one per gather."""

    def __init__(self, nt, nx_per_gather, dt, dx, velocities, t0s=None, pad_t=2, pad_x=2,
                 fmax_hz=0.0, wavelet_peak_hz=0.0, max_resident=64, with_solver=False):
        lib = load()
        o = AshrtOpts()
        lib.ashrt_default_opts(ctypes.byref(o))
        o.pad_t, o.pad_x = int(pad_t), int(pad_x)
        o.fmax_hz, o.wavelet_peak_hz = float(fmax_hz), float(wavelet_peak_hz)
        o.max_batch, o.with_solver = int(max_resident), int(bool(with_solver))
        self.nx = np.ascontiguousarray(np.asarray(nx_per_gather, dtype=np.int32))
        self._v, vp = _farr(velocities)
        if t0s is None:
            tp, nt0 = None, 1
        else:
            self._t0, tp = _farr(t0s)
            nt0 = self._t0.size
        h = c_void_p()
        self._h = None
        ip = lambda a: a.ctypes.data_as(ctypes.POINTER(c_int))
        if np.ndim(nt) == 0:
            _check(lib.ashrt_batch_create(ctypes.byref(h), int(nt), ip(self.nx), self.nx.size,
                                          float(dt), float(dx), vp, self._v.size, tp, nt0,
                                          ctypes.byref(o)))
        else:
            self._nts = np.ascontiguousarray(np.asarray(nt, dtype=np.int32))
            _check(lib.ashrt_batch_create_uneven(ctypes.byref(h), ip(self._nts), ip(self.nx),
                                                 self.nx.size, float(dt), float(dx), vp,
                                                 self._v.size, tp, nt0, ctypes.byref(o)))
        self._h = h.value
        ncls, de, me, ws = c_int(), ctypes.c_longlong(), ctypes.c_longlong(), c_size_t()
        _check(lib.ashrt_batch_info(self._h, ctypes.byref(ncls), ctypes.byref(de),
                                    ctypes.byref(me), ctypes.byref(ws)))
        self.n_classes, self.data_elems, self.model_elems = ncls.value, de.value, me.value
        self.workspace_bytes = ws.value
        self.nt = int(nt) if np.ndim(nt) == 0 else [int(v) for v in nt]
        self.P = self._v.size * nt0

    def autotune(self, cache_path=None):
        """ashrt_batch_autotune: a kernel variant per (nt, Nx) class."""
        path = None if cache_path is None else os.fsencode(cache_path)
        _check(load().ashrt_batch_autotune(self._h, path))

    def forward(self, m, d, stream=None):
        _check(load().ashrt_batch_forward(self._h, _ptr(m), _ptr(d), _stream(stream)))

    def adjoint(self, d, m, stream=None):
        _check(load().ashrt_batch_adjoint(self._h, _ptr(d), _ptr(m), _stream(stream)))

    def deblend(self, d, m, drec=None, stream=None, **kw):
        lib = load()
        o = IrlsOpts()
        lib.irls_default_opts(ctypes.byref(o))
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError("unknown irls option %r" % k)
            setattr(o, k, v)
        reps = (IrlsReport * self.nx.size)()
        _check(lib.ashrt_batch_deblend(self._h, _ptr(d), _ptr(m), _ptr(drec), ctypes.byref(o),
                                       reps, _stream(stream)))
        return _reports(reps)

    def close(self):
        if self._h:
            load().ashrt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fp(a):
    """Pointer to a contiguous float32 numpy array (no copy)."""
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(c_float))


class UNet:
    """Warm-start U-Net (see ashrt_unet_create in include/ashrt.h).

    ``params`` (optional) is a flat float array in the C layout: per layer the
    weights [cout][cin][k][k] then the biases [cout].
    """

    def __init__(self, H, W, out_channels, max_batch=1, params=None):
        lib = load()
        h = c_void_p()
        init, n = None, 0
        if params is not None:
            self._init = np.ascontiguousarray(params, dtype=np.float32)
            init, n = _fp(self._init), self._init.size
        _check(lib.ashrt_unet_create(ctypes.byref(h), int(H), int(W), int(out_channels),
                                     int(max_batch), init, n))
        self._h = h.value
        self.H, self.W, self.out_channels, self.max_batch = H, W, out_channels, max_batch
        self.n_params = int(lib.ashrt_unet_param_count(self._h))

    def params(self):
        out = np.empty(self.n_params, np.float32)
        _check(load().ashrt_unet_get(self._h, _fp(out), None, self.n_params))
        return out

    def grads(self):
        out = np.empty(self.n_params, np.float32)
        _check(load().ashrt_unet_get(self._h, None, _fp(out), self.n_params))
        return out

    def forward(self, x, y, n=None, rescale=False, p=1.0, stream=None):
        n = int(n if n is not None else x.shape[0])
        _check(load().ashrt_unet_forward(self._h, _ptr(x), _ptr(y), n, int(bool(rescale)),
                                         float(p), _stream(stream)))

    def train_step(self, x, t, lr, n=None, channel_weight=None, stream=None):
        """One Adam step (lr = 0: gradients only); returns the loss before the step."""
        n = int(n if n is not None else x.shape[0])
        cw = None
        if channel_weight is not None:
            self._cw = np.ascontiguousarray(channel_weight, dtype=np.float32)
            cw = _fp(self._cw)
        loss = c_double()
        _check(load().ashrt_unet_train_step(self._h, _ptr(x), _ptr(t), n, cw, float(lr),
                                            ctypes.byref(loss), _stream(stream)))
        return loss.value

    def targets(self, x, m, wr, t, n=None, p=1.0, stream=None):
        n = int(n if n is not None else x.shape[0])
        _check(load().ashrt_unet_targets(self._h, _ptr(x), _ptr(m), _ptr(wr), _ptr(t), n,
                                         float(p), _stream(stream)))

    def predict(self, x, m0=None, wr0=None, n=None, p=1.0, stream=None):
        n = int(n if n is not None else x.shape[0])
        _check(load().ashrt_unet_predict(self._h, _ptr(x), _ptr(m0), _ptr(wr0), n, float(p),
                                         _stream(stream)))

    def close(self):
        if self._h:
            load().ashrt_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
