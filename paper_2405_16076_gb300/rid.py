"""ctypes binding of the C ABI in include/rid.h (argument marshalling only).

Every function of the header is exposed under the same name; ``OnlineRID``
is a small convenience wrapper that owns one handle.  Device memory and
streams come from PyTorch; every step of the method runs in librid.so.
There is no CPU fallback: importing this module fails if the library has
not been built, and ``rid_init`` fails with RID_ENOLIB without a GPU.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librid.so")

RID_OK, RID_EINVAL, RID_ENOMEM, RID_ECUDA, RID_ESTATE, RID_ENONFINITE, RID_ENOLIB, RID_ETIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
RID_LAMBDA_STREAMING, RID_LAMBDA_FIXED = 0, 1
RID_OMEGA_GAUSSIAN, RID_OMEGA_RADEMACHER = 0, 1
RID_F64, RID_F32 = 0, 1
RID_REFILL_FIRST, RID_REFILL_PROPORTIONAL = 0, 1
RID_SKETCH_NATIVE, RID_SKETCH_BF16, RID_SKETCH_BF16X2, RID_SKETCH_FP8, RID_SKETCH_FP8X2 = 0, 1, 2, 3, 4
(RID_STATE_SKETCH, RID_STATE_SKETCH_LEV, RID_STATE_SST, RID_STATE_FRO2, RID_STATE_JC,
 RID_STATE_TAU_OLD, RID_STATE_LAMBDA, RID_STATE_CAND, RID_STATE_BATCHES, RID_STATE_GRAM_SHIFT,
 RID_STATE_GRAD_SKETCH) = range(11)


class rid_config(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64), ("k", ctypes.c_int32), ("s", ctypes.c_int32), ("h", ctypes.c_int32),
        ("lambda_mode", ctypes.c_int32), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
        ("eps", ctypes.c_double), ("delta", ctypes.c_double), ("c_const", ctypes.c_double),
        ("lambda_fixed", ctypes.c_double), ("omega_kind", ctypes.c_int32), ("data_dtype", ctypes.c_int32),
        ("sketch_prec", ctypes.c_int32), ("grad_dims", ctypes.c_int32), ("nx", ctypes.c_int32),
        ("ny", ctypes.c_int32), ("nfields", ctypes.c_int32), ("n_max", ctypes.c_int64),
        ("seed", ctypes.c_uint64), ("group_max", ctypes.c_int32), ("defer_device_input", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p), ("right_l", ctypes.c_int32), ("grad_coeff", ctypes.c_int32),
        ("ingest_ctas", ctypes.c_int32), ("refill_mode", ctypes.c_int32), ("lookahead", ctypes.c_int32),
        ("row_offset", ctypes.c_int64), ("m_global", ctypes.c_int64), ("allreduce", ctypes.c_void_p),
        ("allreduce_user", ctypes.c_void_p), ("batch_sms", ctypes.c_int32),
    ]


# rid_allreduce_fn: int (*)(double* buf, int64_t count, void* cuda_stream, void* user)
RID_ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p)


class rid_log_record(ctypes.Structure):
    _fields_ = [
        ("batch", ctypes.c_int64), ("n_obs", ctypes.c_int64), ("lambda_", ctypes.c_double),
        ("fro2", ctypes.c_double), ("est_sq", ctypes.c_double * 4), ("est_unc", ctypes.c_double * 4),
        ("gram_shift", ctypes.c_double), ("q_star", ctypes.c_int32), ("n_active", ctypes.c_int32),
        ("n_kept", ctypes.c_int32), ("n_new", ctypes.c_int32),
    ]


class RIDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rid error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"librid.so is not built ({LIB_PATH}); run paper_2405_16076_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    H = ctypes.c_void_p
    P = ctypes.c_void_p
    sig = {
        "rid_config_default": (ctypes.c_int, [ctypes.POINTER(rid_config)]),
        "rid_init": (ctypes.c_int, [ctypes.POINTER(H), ctypes.POINTER(rid_config)]),
        "rid_ingest": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
        "rid_finalize": (ctypes.c_int, [H, P, P, ctypes.c_int64, ctypes.c_int32]),
        "rid_error_estimate": (ctypes.c_int, [H, P, P, P]),
        "rid_n_obs": (ctypes.c_int64, [H]),
        "rid_get_basis": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32]),
        "rid_get_right_sketch": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32]),
        "rid_gradient_coefficients": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32, P, P]),
        "rid_get_state": (ctypes.c_int, [H, ctypes.c_int32, P, ctypes.c_int64]),
        "rid_sync": (ctypes.c_int, [H]),
        "rid_profile": (ctypes.c_int, [H, ctypes.c_int32]),
        "rid_profile_read": (ctypes.c_int, [H, P, P, P]),
        "rid_profile_timeline": (ctypes.c_int, [H, P, ctypes.c_int32, P]),
        "rid_reset": (ctypes.c_int, [H]),
        "rid_last_error": (ctypes.c_char_p, [H]),
        "rid_destroy": (None, [H]),
        "rid_checkpoint_size": (ctypes.c_int, [H, P]),
        "rid_checkpoint": (ctypes.c_int, [H, P, ctypes.c_int64]),
        "rid_restore": (ctypes.c_int, [H, P, ctypes.c_int64]),
        "rid_batch_ingest": (ctypes.c_int, [P, ctypes.c_int32, P, P, P, ctypes.c_int32]),
        "rid_sketch_noalloc": (ctypes.c_int, [ctypes.POINTER(rid_config), P, ctypes.c_int64, ctypes.c_int32,
                                              P, ctypes.c_int64, P]),
        "rid_config_check": (ctypes.c_int, [ctypes.POINTER(rid_config)]),
        "rid_autotune": (ctypes.c_int, [ctypes.POINTER(rid_config), P, ctypes.c_int64, ctypes.c_int32, P]),
        "rid_log_enable": (ctypes.c_int, [H, ctypes.c_int32]),
        "rid_get_log": (ctypes.c_int, [H, P, ctypes.c_int32, P]),
        "rid_rcss_init": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int64, ctypes.c_int32, ctypes.c_double,
                                         ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P]),
        "rid_rcss_ingest": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]),
        "rid_rcss_selection": (ctypes.c_int, [H, P, ctypes.c_int32, P, P, P]),
        "rid_rcss_probabilities": (ctypes.c_int, [H, P, ctypes.c_int64, P]),
        "rid_rcss_basis": (ctypes.c_int, [H, P, ctypes.c_int64, ctypes.c_int32]),
        "rid_rcss_destroy": (ctypes.c_int, [H]),
        "rid_attach_rcss": (ctypes.c_int, [H, H]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()

rid_config_default = lib.rid_config_default
rid_init = lib.rid_init
rid_ingest = lib.rid_ingest
rid_finalize = lib.rid_finalize
rid_error_estimate = lib.rid_error_estimate
rid_n_obs = lib.rid_n_obs
rid_get_basis = lib.rid_get_basis
rid_get_right_sketch = lib.rid_get_right_sketch
rid_gradient_coefficients = lib.rid_gradient_coefficients
rid_get_state = lib.rid_get_state
rid_sync = lib.rid_sync
rid_profile = lib.rid_profile
rid_profile_read = lib.rid_profile_read
rid_profile_timeline = lib.rid_profile_timeline
rid_reset = lib.rid_reset
rid_last_error = lib.rid_last_error
rid_destroy = lib.rid_destroy
rid_sketch_noalloc = lib.rid_sketch_noalloc
rid_batch_ingest = lib.rid_batch_ingest
rid_checkpoint_size = lib.rid_checkpoint_size
rid_checkpoint = lib.rid_checkpoint
rid_restore = lib.rid_restore
rid_config_check = lib.rid_config_check
rid_autotune = lib.rid_autotune
rid_log_enable = lib.rid_log_enable
rid_get_log = lib.rid_get_log
rid_rcss_init = lib.rid_rcss_init
rid_rcss_ingest = lib.rid_rcss_ingest
rid_rcss_selection = lib.rid_rcss_selection
rid_rcss_probabilities = lib.rid_rcss_probabilities
rid_rcss_basis = lib.rid_rcss_basis
rid_rcss_destroy = lib.rid_rcss_destroy
rid_attach_rcss = lib.rid_attach_rcss


def batch_ingest(handles, blocks):
    """rid_batch_ingest: blocks[i] (b_i x m_i rows = columns, torch on the GPU or numpy on the
    host, all on the same side) into handles[i] (OnlineRID objects), in one call."""
    nh = len(handles)
    if nh == 0:
        return
    marsh = [_columns(b, hd.m, hd.esize) for hd, b in zip(handles, blocks)]
    on_dev = marsh[0][1]
    if any(x[1] != on_dev for x in marsh):
        raise ValueError("all blocks must be on the device, or all on the host")
    hs = (ctypes.c_void_p * nh)(*[hd.h.value for hd in handles])
    cols = (ctypes.c_void_p * nh)(*[x[0].value for x in marsh])
    ld = (ctypes.c_int64 * nh)(*[x[2] for x in marsh])
    nc = (ctypes.c_int32 * nh)(*[x[3] for x in marsh])
    rc = rid_batch_ingest(hs, nh, cols, ld, nc, 1 if on_dev else 0)
    if rc != RID_OK:
        msg = None
        for hd in handles:
            m = rid_last_error(hd.h)
            if m:
                msg = m
        raise RIDError(rc, (msg or rid_last_error(None) or b"").decode())


def _check(rc, h=None):
    if rc != RID_OK:
        msg = rid_last_error(h)
        raise RIDError(rc, msg.decode() if msg else "")


def _columns(cols, m, esize):
    """(pointer, on_device, ld, ncols, owner) of a block of m-long columns in the data dtype.

    Accepted: a torch tensor (device or host) of shape (m,), (m, b) with unit stride down each
    column, or (b, m) with unit stride along each row (row q = column q), of the data dtype; or
    anything numpy reads as such an array (converted to the data dtype, and copied to contiguous
    columns when needed).  Anything else raises TypeError or ValueError, so that the library never
    reads outside the caller's buffer.  ``owner`` must stay referenced until the call returns."""
    if hasattr(cols, "data_ptr"):
        want = "torch.float64" if esize == 8 else "torch.float32"
        if str(cols.dtype) != want:
            raise TypeError(f"columns must be {want}, not {cols.dtype}")
        shp, st = tuple(cols.shape), tuple(cols.stride())
        if len(shp) == 1 and st[0] == 1:
            ncols, ld = 1, shp[0]
        elif len(shp) == 2 and shp[0] == m and st[0] == 1:
            ncols, ld = shp[1], st[1]
        elif len(shp) == 2 and shp[1] == m and st[1] == 1:
            ncols, ld = shp[0], st[0]
        else:
            raise ValueError("tensor must hold contiguous m-long columns")
        if ncols == 1:
            ld = max(ld, m)                  # one column: its stride to a next one is irrelevant
        return ctypes.c_void_p(cols.data_ptr()), bool(cols.is_cuda), int(ld), int(ncols), cols
    want = np.float64 if esize == 8 else np.float32
    a = np.asarray(cols)
    if a.ndim == 1:
        a = np.ascontiguousarray(a, dtype=want)
        return ctypes.c_void_p(a.ctypes.data), False, int(a.shape[0]), 1, a
    if a.ndim != 2:
        raise ValueError("array must hold m-long columns")
    if a.shape[0] == m and a.flags.f_contiguous:
        a = np.asfortranarray(a, dtype=want)
        ncols = a.shape[1]
    elif a.shape[1] == m and a.flags.c_contiguous:
        a = np.ascontiguousarray(a, dtype=want)
        ncols = a.shape[0]
    elif a.shape[0] == m:
        a = np.asfortranarray(a, dtype=want)
        ncols = a.shape[1]
    elif a.shape[1] == m:
        a = np.ascontiguousarray(a, dtype=want)
        ncols = a.shape[0]
    else:
        raise ValueError("array must hold m-long columns")
    return ctypes.c_void_p(a.ctypes.data), False, int(m), int(ncols), a


def _device_out(x, dtype, numel, what):
    """Check a caller's output tensor before the library writes ``numel`` elements of ``dtype``
    (a torch dtype name) into it from the device: right dtype, contiguous, large enough, on a
    CUDA device.  Raises TypeError or ValueError otherwise."""
    if not hasattr(x, "data_ptr"):
        raise TypeError(f"{what} must be a torch tensor")
    if str(x.dtype) != dtype:
        raise TypeError(f"{what} must be {dtype}, not {x.dtype}")
    if not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if x.numel() < numel:
        raise ValueError(f"{what} holds {x.numel()} elements; {numel} are written")
    if not x.is_cuda:
        raise TypeError(f"{what} must be on a CUDA device")
    return ctypes.c_void_p(x.data_ptr())


def make_config(m, k, s, h=0, *, c1=1 / 6, c2=1 / 3, eps=0.5, delta=0.05, c_const=1.0,
                lambda_mode="streaming", lambda_fixed=0.0, omega="rademacher", dtype="f32",
                sketch="native", n_max=1024, seed=0, stream=None, group_max=0, defer=False,
                grad_dims=0, nx=0, ny=0, nfields=1, right_l=0, grad_coeff=False, ingest_ctas=0, refill="first",
                lookahead=0, row_offset=0, m_global=0, allreduce=None, batch_sms=0):
    """An rid_config from keyword arguments (the defaults of rid_config_default otherwise)."""
    cfg = rid_config()
    _check(rid_config_default(ctypes.byref(cfg)))
    cfg.m, cfg.k, cfg.s, cfg.h = int(m), int(k), int(s), int(h)
    cfg.c1, cfg.c2, cfg.eps, cfg.delta, cfg.c_const = c1, c2, eps, delta, c_const
    cfg.lambda_mode = RID_LAMBDA_FIXED if lambda_mode == "fixed" else RID_LAMBDA_STREAMING
    cfg.lambda_fixed = float(lambda_fixed)
    cfg.omega_kind = RID_OMEGA_GAUSSIAN if omega == "gaussian" else RID_OMEGA_RADEMACHER
    cfg.data_dtype = RID_F64 if dtype == "f64" else RID_F32
    cfg.sketch_prec = {"native": RID_SKETCH_NATIVE, "bf16": RID_SKETCH_BF16, "bf16x2": RID_SKETCH_BF16X2,
                       "fp8": RID_SKETCH_FP8, "fp8x2": RID_SKETCH_FP8X2}[sketch]
    cfg.n_max = int(n_max)
    cfg.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    cfg.group_max = int(group_max)
    cfg.defer_device_input = 1 if defer else 0
    cfg.grad_dims, cfg.nx, cfg.ny, cfg.nfields = int(grad_dims), int(nx), int(ny), int(nfields)
    cfg.right_l = int(right_l)
    cfg.grad_coeff = 1 if grad_coeff else 0
    cfg.ingest_ctas = int(ingest_ctas)
    cfg.refill_mode = {"first": RID_REFILL_FIRST, "proportional": RID_REFILL_PROPORTIONAL}[refill]
    cfg.lookahead = int(lookahead)
    cfg.batch_sms = int(batch_sms)
    cfg.row_offset = int(row_offset)
    cfg.m_global = int(m_global)
    if allreduce is not None:                 # a RID_ALLREDUCE_FN; the caller keeps it alive
        cfg.allreduce = ctypes.cast(allreduce, ctypes.c_void_p)
    cfg.cuda_stream = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    return cfg


def autotune_group(cols, m, k, s, h=0, **kw):
    """rid_autotune: the ingest's launch shape -- group size (columns per sketch launch) and
    CTAs per sketch launch -- measured for the configuration ``make_config(m, k, s, h, **kw)``
    on representative device columns ``cols`` (a torch tensor (b, m), row q = snapshot q).
    Returns (group_max, ingest_ctas, microseconds per column of a whole pass); pass both to
    OnlineRID.  RID_AUTOTUNE_CACHE in the environment names an optional cache file."""
    cfg = make_config(m, k, s, h, **kw)
    if not (hasattr(cols, "data_ptr") and cols.is_cuda) or cols.dim() != 2 or cols.shape[1] != int(m) \
            or cols.stride(1) != 1:
        raise ValueError("cols must be a device tensor (b, m) with contiguous rows")
    us = ctypes.c_double()
    _check(rid_autotune(ctypes.byref(cfg), ctypes.c_void_p(cols.data_ptr()), int(cols.stride(0)),
                        int(cols.shape[0]), ctypes.byref(us)))
    return int(cfg.group_max), int(cfg.ingest_ctas), float(us.value)


class OnlineRID:
    """One streaming decomposition handle (see include/rid.h)."""

    def __init__(self, m, k, s, h=0, **kw):
        """Keyword arguments as make_config: c1, c2, eps, delta, c_const, lambda_mode,
        lambda_fixed, omega, dtype, sketch, n_max, seed, stream, group_max, defer, grad_dims,
        nx, ny, nfields, right_l, grad_coeff, ingest_ctas, refill ("first" or "proportional"), lookahead,
        batch_sms (SMs of the batch steps' partition, 0 = no partition), and for a row shard
        row_offset, m_global and allreduce (a RID_ALLREDUCE_FN)."""
        cfg = make_config(m, k, s, h, **kw)
        self._allreduce = kw.get("allreduce")     # the callback must outlive the handle
        dtype = kw.get("dtype", "f32")
        self.cfg = cfg
        self.t = int(k)
        self.m = int(m)
        self.rows = int(s) + int(h)
        self.s = int(s)
        self.esize = 8 if dtype == "f64" else 4
        self.np_dtype = np.float64 if dtype == "f64" else np.float32
        hnd = ctypes.c_void_p()
        _check(rid_init(ctypes.byref(hnd), ctypes.byref(cfg)))
        self.h = hnd

    def close(self):
        if self.h:
            rid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ingest(self, cols):
        """cols: a block of m-long columns -- a torch tensor on the GPU (device input) or on the
        host, of shape (m, b) column-major or (b, m) with row q = snapshot q, in the data dtype;
        or a numpy array of either shape (converted to the data dtype)."""
        p, on_dev, ld, ncols, owner = _columns(cols, self.m, self.esize)
        _check(rid_ingest(self.h, p, ld, ncols, int(on_dev)), self.h)
        del owner

    def finalize(self):
        t = self.t
        n = int(rid_n_obs(self.h))
        J = np.empty(t, dtype=np.int64)
        P = np.empty((n, t), dtype=np.float64)     # row j = column j of the t x n matrix
        _check(rid_finalize(self.h, ctypes.c_void_p(J.ctypes.data), ctypes.c_void_p(P.ctypes.data), t, 0), self.h)
        return J, P.T.copy()

    def error_estimate(self):
        sq = np.empty(5)
        fro = np.empty(5)
        q = ctypes.c_int32()
        _check(rid_error_estimate(self.h, ctypes.c_void_p(sq.ctypes.data), ctypes.c_void_p(fro.ctypes.data),
                                  ctypes.byref(q)), self.h)
        return sq, fro, int(q.value)

    def n_obs(self):
        return int(rid_n_obs(self.h))

    def state(self, item):
        n = self.n_obs()
        t, s, rows = self.t, self.s, self.rows
        if item == RID_STATE_SKETCH:
            out = np.empty((n, rows))
        elif item == RID_STATE_SKETCH_LEV:
            out = np.empty((n, s))
        elif item == RID_STATE_SST:
            out = np.empty((s, s))
        elif item == RID_STATE_FRO2:
            out = np.empty(2)
        elif item == RID_STATE_JC:
            out = np.empty(t, dtype=np.int64)
        elif item == RID_STATE_TAU_OLD:
            out = np.empty(t)
        elif item in (RID_STATE_LAMBDA, RID_STATE_GRAM_SHIFT):
            out = np.empty(1)
        elif item == RID_STATE_GRAD_SKETCH:
            out = np.empty((n, 2, s))
            _check(rid_get_state(self.h, item, ctypes.c_void_p(out.ctypes.data), out.size), self.h)
            return out.transpose(1, 2, 0).copy()           # (2, s, n)
        elif item == RID_STATE_BATCHES:
            out = np.empty(1, dtype=np.int64)
        elif item == RID_STATE_CAND:
            raise ValueError("use candidates()")
        else:
            raise ValueError(item)
        _check(rid_get_state(self.h, item, ctypes.c_void_p(out.ctypes.data), out.size), self.h)
        if item in (RID_STATE_SKETCH, RID_STATE_SKETCH_LEV):
            return out.T.copy()
        if item == RID_STATE_SST:
            return out.T.copy()
        return out

    def candidates(self, n_prev):
        out = np.empty((4, n_prev, self.t))
        _check(rid_get_state(self.h, RID_STATE_CAND, ctypes.c_void_p(out.ctypes.data), out.size), self.h)
        return out.transpose(0, 2, 1).copy()    # (4, t, n_prev), rows = active positions

    def basis(self):
        out = np.zeros((self.t, self.m), dtype=self.np_dtype)
        _check(rid_get_basis(self.h, ctypes.c_void_p(out.ctypes.data), self.m, 0), self.h)
        return out.T.copy()

    def gradient_coefficients(self, out=None):
        """Sec. 3.4's gradient-augmented coefficients, lambda by the sketched GCV:
        (lambda*, P (t x n) on the host, GCV(lambda*)); with ``out`` (a device tensor (n, t),
        row j = column j) P is written there instead and None is returned in its place."""
        lam = ctypes.c_double()
        g = ctypes.c_double()
        if out is not None:
            po = _device_out(out, "torch.float64", self.n_obs() * self.t, "out")
            _check(rid_gradient_coefficients(self.h, po, self.t, 1, ctypes.byref(lam), ctypes.byref(g)), self.h)
            return lam.value, None, g.value
        n = self.n_obs()
        P = np.zeros((n, self.t))                      # row j = column j of the t x n matrix
        _check(rid_gradient_coefficients(self.h, ctypes.c_void_p(P.ctypes.data), self.t, 0, ctypes.byref(lam),
                                         ctypes.byref(g)), self.h)
        return lam.value, P.T.copy(), g.value

    def right_sketch(self):
        """The optional right sketch Y (m x right_l, data dtype) on the host."""
        l = int(self.cfg.right_l)
        out = np.zeros((l, self.m), dtype=self.np_dtype)      # row r = column r of Y
        _check(rid_get_right_sketch(self.h, ctypes.c_void_p(out.ctypes.data), self.m, 0), self.h)
        return out.T.copy()

    def right_sketch_device(self, out):
        """Copy Y into a contiguous device tensor of shape (right_l, m) (row r = column r of Y)."""
        l = int(self.cfg.right_l)
        want = "torch.float64" if self.esize == 8 else "torch.float32"
        if out.dim() != 2 or tuple(out.shape) != (l, self.m):
            raise ValueError(f"out must have shape ({l}, {self.m})")
        po = _device_out(out, want, l * self.m, "out")
        _check(rid_get_right_sketch(self.h, po, self.m, 1), self.h)

    def finalize_device(self, J, P, sync=True):
        """Finalize into device tensors: J (t,) int64 and P (n, t) float64 (row j = column j).

        sync=False queues the copies without a host synchronization (RID_OUT_DEVICE_ASYNC), so
        that reset / ingest / finalize can be captured into a CUDA graph."""
        pj = _device_out(J, "torch.int64", self.t, "J")
        pp = _device_out(P, "torch.float64", self.n_obs() * self.t, "P")
        _check(rid_finalize(self.h, pj, pp, self.t, 1 if sync else 2), self.h)

    def profile(self, enable=True):
        _check(rid_profile(self.h, 1 if enable else 0), self.h)

    def profile_read(self):
        ms = np.zeros(3)
        kern = np.zeros(3, dtype=np.int64)
        grp = np.zeros(3, dtype=np.int64)
        _check(rid_profile_read(self.h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(kern.ctypes.data),
                                ctypes.c_void_p(grp.ctypes.data)), self.h)
        return ms, kern, grp

    TIMELINE_PHASES = ("ingest", "lambda", "scores", "select", "gram", "qr", "coeff")

    def profile_timeline(self):
        """Per-batch phase records since profile(True): an (n, 4) array of (batch, phase, start
        ms, end ms); phase names in TIMELINE_PHASES."""
        n = ctypes.c_int32()
        _check(rid_profile_timeline(self.h, None, 0, ctypes.byref(n)), self.h)
        out = np.zeros((max(n.value, 1), 4))
        _check(rid_profile_timeline(self.h, ctypes.c_void_p(out.ctypes.data), n.value, ctypes.byref(n)), self.h)
        return out[:n.value]

    def checkpoint(self):
        """The stream state as bytes (rid_checkpoint)."""
        n = ctypes.c_int64()
        _check(rid_checkpoint_size(self.h, ctypes.byref(n)), self.h)
        buf = np.empty(n.value, dtype=np.uint8)
        _check(rid_checkpoint(self.h, ctypes.c_void_p(buf.ctypes.data), n.value), self.h)
        return buf.tobytes()

    def restore(self, state):
        """Continue the stream saved by checkpoint() (same configuration)."""
        buf = np.frombuffer(state, dtype=np.uint8)
        _check(rid_restore(self.h, ctypes.c_void_p(buf.ctypes.data), buf.size), self.h)

    def sync(self):
        _check(rid_sync(self.h), self.h)

    def log_enable(self, capacity=1024):
        """Keep the last ``capacity`` batch steps' decisions on the device (0: off)."""
        _check(rid_log_enable(self.h, int(capacity)), self.h)

    def log(self, max_records=None):
        """The logged batch steps (the newest ``max_records``, all by default), oldest first, as
        dicts (see rid_log_record in include/rid.h)."""
        n = ctypes.c_int32()
        _check(rid_get_log(self.h, None, 0, ctypes.byref(n)), self.h)         # records available
        cap = n.value if max_records is None else min(n.value, max(0, int(max_records)))
        if cap == 0:
            return []
        buf = (rid_log_record * cap)()
        _check(rid_get_log(self.h, ctypes.cast(buf, ctypes.c_void_p), cap, ctypes.byref(n)), self.h)
        out = []
        for r in buf[:n.value]:
            out.append({"batch": r.batch, "n_obs": r.n_obs, "lambda": r.lambda_, "fro2": r.fro2,
                        "est_sq": list(r.est_sq), "est_unc": list(r.est_unc), "gram_shift": r.gram_shift,
                        "q_star": r.q_star, "n_active": r.n_active, "n_kept": r.n_kept, "n_new": r.n_new})
        return out

    def reset(self):
        _check(rid_reset(self.h), self.h)

    def attach_rcss(self, g):
        """Algorithm 1 (a ``ResidualCSS`` on this handle's stream, cap <= t, stop_at_cap) as the
        selector; ``None`` detaches.  Keep ``g`` alive while the handle uses it."""
        _check(rid_attach_rcss(self.h, g.h if g is not None else None), self.h)
        self._rcss = g


class ResidualCSS:
    """Owns one rid_rcss handle: online column subset selection by residual-based sampling (the
    paper's Algorithm 1, Sec. 2.2.1), the selector the accuracy tables compare against."""

    def __init__(self, m, k, xi, *, seed=0, data_dtype=RID_F64, cap=1024, stop_at_cap=False, cuda_stream=None):
        self.m = int(m)
        self.esize = 8 if data_dtype == RID_F64 else 4
        self.data_dtype = data_dtype
        self.h = ctypes.c_void_p()
        _check(rid_rcss_init(ctypes.byref(self.h), self.m, int(k), float(xi), int(seed) & 0xFFFFFFFFFFFFFFFF,
                             int(data_dtype), int(cap), int(bool(stop_at_cap)), ctypes.c_void_p(cuda_stream)))

    def close(self):
        if self.h:
            rid_rcss_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ingest(self, cols):
        ptr, dev, ld, n, _own = _columns(cols, self.m, self.esize)
        _check(rid_rcss_ingest(self.h, ptr, ld, n, int(dev)))

    def selection(self):
        """(indices of C_pre then C_cur by arrival, sigma, basis size)."""
        n, sig, nb = ctypes.c_int32(), ctypes.c_double(), ctypes.c_int32()
        _check(rid_rcss_selection(self.h, None, 0, ctypes.byref(n), ctypes.byref(sig), ctypes.byref(nb)))
        idx = np.zeros(max(n.value, 1), dtype=np.int64)
        _check(rid_rcss_selection(self.h, ctypes.c_void_p(idx.ctypes.data), n.value, None, None, None))
        return idx[:n.value], sig.value, nb.value

    def probabilities(self):
        n = ctypes.c_int64()
        _check(rid_rcss_probabilities(self.h, None, 0, ctypes.byref(n)))
        p = np.zeros(max(n.value, 1))
        _check(rid_rcss_probabilities(self.h, ctypes.c_void_p(p.ctypes.data), n.value, None))
        return p[:n.value]

    def basis(self):
        nb = self.selection()[2]
        Q = np.zeros((nb, self.m), dtype=np.float64 if self.esize == 8 else np.float32)
        if nb:
            _check(rid_rcss_basis(self.h, ctypes.c_void_p(Q.ctypes.data), self.m, 0))
        return Q.T
