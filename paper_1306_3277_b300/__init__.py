"""B300 (sm_103a) bootstrap particle filter -- Python binding of the C ABI in
``include/pf.h``.

This module only marshals arguments: every step of the filter runs in the
CUDA kernels of ``libpf_b300.so``.  There is no CPU fallback; importing it
without the built library (and a CUDA device at call time) raises.

Names follow the C ABI: ``pf_create``, ``pf_run``, ``pf_wait``, ``pf_destroy``,
``pf_batch_run``, ``pf_server_*``; arrays may be numpy arrays (host memory) or
torch CUDA tensors (device memory, passed by pointer).
"""
import ctypes
import os

import numpy as np

from . import build as _build

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ECUDA, PF_EDEGENERATE, PF_ETIMEOUT, PF_EBUSY = range(7)
PF_WINDKESSEL, PF_LORENZ96, PF_WINDKESSEL_EXP, PF_LORENZ96_SDE = 0, 1, 2, 3
PF_FP64, PF_MIXED = 0, 1
PF_FLAG_ASYNC = 1
STATUS_NAMES = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_ENOMEM", 3: "PF_ECUDA", 4: "PF_EDEGENERATE",
                5: "PF_ETIMEOUT", 6: "PF_EBUSY"}
L96_SIZES = (4, 8, 12, 16, 20, 24, 32, 40)


class PFError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class pf_model(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("N", ctypes.c_int32), ("substeps", ctypes.c_int32),
                ("obs_stride", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("resampler", ctypes.c_int32), ("ess_threshold", ctypes.c_double),
                ("flow_peak", ctypes.c_double), ("flow_period", ctypes.c_double),
                ("obs_every", ctypes.c_int32), ("obs_count", ctypes.c_int32)]


class pf_batch_shape(ctypes.Structure):
    """Launch shape of a batch (include/pf.h): no field changes any result."""
    _fields_ = [("cta_max_particles", ctypes.c_int64), ("branches", ctypes.c_int32),
                ("resample_blocks_per_sm", ctypes.c_int32),
                ("persistent_blocks_per_sm", ctypes.c_int32), ("tiles_per_item", ctypes.c_int32)]

    def as_dict(self):
        return {"cta_max_particles": int(self.cta_max_particles), "branches": int(self.branches),
                "resample_blocks_per_sm": int(self.resample_blocks_per_sm),
                "persistent_blocks_per_sm": int(self.persistent_blocks_per_sm),
                "tiles_per_item": int(self.tiles_per_item)}


_lib = None
_vp = ctypes.c_void_p


def lib():
    """Load (building if stale) libpf_b300.so, or its checked build
    libpf_b300_checked.so when PF_B300_CHECKED=1 is in the environment."""
    global _lib
    if _lib is None:
        path = _build.build(checked=os.environ.get("PF_B300_CHECKED") == "1")
        L = ctypes.CDLL(path)
        L.pf_theta_size.argtypes = [ctypes.c_int32]
        L.pf_theta_size.restype = ctypes.c_int32
        L.pf_create.argtypes = [ctypes.POINTER(pf_model), ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_double, ctypes.POINTER(_vp)]
        L.pf_device_bytes.argtypes = [ctypes.POINTER(pf_model), ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32]
        L.pf_device_bytes.restype = ctypes.c_size_t
        L.pf_run.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp, ctypes.c_uint32, _vp]
        L.pf_wait.argtypes = [_vp]
        L.pf_destroy.argtypes = [_vp]
        L.pf_last_error.restype = ctypes.c_char_p
        L.pf_batch_run.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                   ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                   _vp]
        L.pf_profile_enable.argtypes = [_vp, ctypes.c_int32]
        L.pf_profile_read.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64)]
        L.pf_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double)]
        L.pf_weight_exp.argtypes = [_vp, _vp, ctypes.c_int64]
        L.pf_weight_prefix.argtypes = [_vp, _vp, _vp, ctypes.c_int64]
        L.pf_weight_sum_log.argtypes = [_vp, _vp, ctypes.c_int64]
        L.pf_debug_fail_allocation.argtypes = [ctypes.c_int32]
        L.pf_debug_fail_server_wait.argtypes = [ctypes.c_int32]
        L.pf_debug_persist_wait_limit.argtypes = [ctypes.c_double]
        L.pf_debug_persist_unfilled_slot.argtypes = [ctypes.c_int32]
        L.pf_debug_check_counts.argtypes = [ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_int32)]
        L.pf_pmmh_run.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp), _vp,
                                  ctypes.POINTER(pf_param), _vp, ctypes.c_int32,
                                  ctypes.c_uint64, _vp, _vp, _vp, _vp]
        L.pf_pmmh_run.restype = ctypes.c_int
        L.pf_smc2_run.argtypes = [ctypes.POINTER(pf_model), ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_double, _vp, ctypes.c_int32, ctypes.POINTER(pf_param),
                                  _vp, ctypes.c_uint64, _vp, _vp, _vp, _vp, _vp, _vp]
        L.pf_smc2_run.restype = ctypes.c_int
        L.pf_batch_configure.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp), ctypes.c_int64]
        L.pf_batch_configure.restype = ctypes.c_int
        L.pf_batch_set_shape.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp),
                                         ctypes.POINTER(pf_batch_shape)]
        L.pf_batch_set_shape.restype = ctypes.c_int
        L.pf_batch_get_shape.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp),
                                         ctypes.POINTER(pf_batch_shape)]
        L.pf_batch_get_shape.restype = ctypes.c_int
        L.pf_batch_autotune.argtypes = [ctypes.c_int32, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                        ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_uint64),
                                        ctypes.POINTER(ctypes.c_int64)]
        L.pf_batch_autotune.restype = ctypes.c_int
        L.pf_run_range.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                   _vp, _vp, _vp]
        L.pf_sample_path.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp, _vp]
        L.pf_debug_step.argtypes = [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_int32, _vp, _vp,
                                    _vp, _vp, _vp]
        for name in ("pf_run", "pf_wait", "pf_destroy", "pf_create", "pf_batch_run",
                     "pf_profile_enable", "pf_profile_read", "pf_measure_fma_peak",
                     "pf_run_range", "pf_sample_path", "pf_weight_exp", "pf_weight_prefix",
                     "pf_weight_sum_log",
                     "pf_debug_step",
                     "pf_debug_fail_allocation", "pf_debug_fail_server_wait",
                     "pf_debug_persist_wait_limit", "pf_debug_persist_unfilled_slot",
                     "pf_debug_check_counts"):
            getattr(L, name).restype = ctypes.c_int
        L.pf_run_noalloc.argtypes = [ctypes.POINTER(pf_model), ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_double, _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp,
                                     _vp]
        L.pf_run_noalloc.restype = ctypes.c_int
        if hasattr(L, "pf_server_create"):
            L.pf_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int32, ctypes.POINTER(_vp)]
            L.pf_server_submit.argtypes = [_vp, ctypes.POINTER(pf_model), ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_double, _vp, _vp,
                                           ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
            L.pf_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]
            L.pf_server_stats.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int64)] * 4
            L.pf_server_configure.argtypes = [_vp, ctypes.c_int32]
            L.pf_server_destroy.argtypes = [_vp]
            for name in ("pf_server_create", "pf_server_submit", "pf_server_poll",
                         "pf_server_stats", "pf_server_configure", "pf_server_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def library_path():
    return _build.LIB


def pf_last_error():
    return lib().pf_last_error().decode()


def _check(st, ok=(PF_OK,)):
    if st not in ok:
        raise PFError(st, pf_last_error())
    return st


PF_RESAMPLE_SYSTEMATIC, PF_RESAMPLE_STRATIFIED, PF_RESAMPLE_MULTINOMIAL = range(3)


def model(kind, N=1, substeps=1, obs_stride=1, prec=PF_FP64, ess_threshold=1.0, flow_peak=400.0,
          flow_period=1.0, resampler=PF_RESAMPLE_SYSTEMATIC, obs_every=0, obs_count=0):
    return pf_model(kind, N, substeps, obs_stride, prec, resampler, ess_threshold, flow_peak,
                    flow_period, obs_every, obs_count)


PF_PRIOR_FIXED, PF_PRIOR_UNIFORM, PF_PRIOR_GAUSSIAN, PF_PRIOR_GAMMA, PF_PRIOR_INV_GAMMA = range(5)
PF_PROPOSE_FIXED, PF_PROPOSE_TRUNC_GAUSSIAN, PF_PROPOSE_INV_GAMMA = range(3)


class pf_param(ctypes.Structure):
    """Prior and proposal of one component of theta (include/pf.h)."""
    _fields_ = [("prior", ctypes.c_int32), ("proposal", ctypes.c_int32),
                ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
                ("d", ctypes.c_double), ("e", ctypes.c_double)]


def params(spec):
    """List of (prior, proposal, a, b, c, d, e) tuples -> pf_param array."""
    arr = (pf_param * len(spec))()
    for k, t in enumerate(spec):
        t = tuple(t) + (0.0,) * (7 - len(t))
        arr[k] = pf_param(int(t[0]), int(t[1]), *[float(v) for v in t[2:7]])
    return arr


def pf_pmmh_run(filters, y, spec, theta0, niter, seed, stream=None):
    """Marginal Metropolis-Hastings chains, one per filter (Algorithm 3):
    returns samples [niter+1][nchains][nth], logliks [niter+1][nchains],
    accepted [nchains]."""
    nc = len(filters)
    th0 = np.ascontiguousarray(theta0, dtype=np.float64).reshape(nc, -1)
    y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
    sp = params(spec)
    hs = (_vp * nc)(*[f.h for f in filters])
    samples = np.zeros((niter + 1, nc, th0.shape[1]))
    lls = np.zeros((niter + 1, nc))
    acc = np.zeros(nc, dtype=np.int32)
    _check(lib().pf_pmmh_run(nc, hs, _ptr(y), sp, _ptr(th0), niter, ctypes.c_uint64(seed),
                             _ptr(samples), _ptr(lls), _ptr(acc), _stream_ptr(stream)))
    return samples, lls, acc


def pf_smc2_run(m, P, T, dt, y, ntheta, spec, theta_base, seed, stream=None):
    """SMC^2 (Algorithm 4): returns (status, theta [ntheta][nth], log-weights
    [ntheta], log evidence, per-step evidence increments [T], accepted moves [T])."""
    nth = len(theta_base)
    y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
    base = np.ascontiguousarray(theta_base, dtype=np.float64)
    sp = params(spec)
    th = np.zeros((ntheta, nth))
    logw = np.zeros(ntheta)
    lz = np.zeros(1)
    incr = np.zeros(T)
    acc = np.zeros(T, dtype=np.int32)
    st = lib().pf_smc2_run(ctypes.byref(m), P, T, dt, _ptr(y), ntheta, sp, _ptr(base),
                           ctypes.c_uint64(seed), _ptr(th), _ptr(logw), _ptr(lz), _ptr(incr),
                           _ptr(acc), _stream_ptr(stream))
    st = _check(st, ok=(PF_OK, PF_EDEGENERATE))
    return st, th, logw, float(lz[0]), incr, acc


def model_from_workload(w):
    return model(w.kind, w.N, w.substeps, w.obs_stride, w.prec, w.ess_threshold, w.flow_peak,
                 w.flow_period, getattr(w, "resampler", PF_RESAMPLE_SYSTEMATIC),
                 getattr(w, "obs_every", 0), getattr(w, "obs_count", 0))


def pf_theta_size(kind):
    return lib().pf_theta_size(kind)


def pf_device_bytes(m, P, T, history=False):
    return lib().pf_device_bytes(ctypes.byref(m), P, T, 1 if history else 0)


def _ptr(a):
    """Pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Filter:
    """A created filter (owns its device buffers until destroy())."""

    def __init__(self, m, P, T, dt):
        h = _vp()
        _check(lib().pf_create(ctypes.byref(m), P, T, dt, ctypes.byref(h)))
        self.h = h
        self.model = m
        self.P, self.T, self.dt = P, T, dt
        self.N = m.N
        wk = m.kind in (PF_WINDKESSEL, PF_WINDKESSEL_EXP)
        ny = 1 if wk else (m.N + m.obs_stride - 1) // m.obs_stride
        self.Ny = min(ny, m.obs_count) if (not wk and m.obs_count > 0) else ny
        self.state_dtype = np.float64 if m.prec == PF_FP64 else np.float32

    def run(self, theta, y, seed, want_particles=False, want_ancestors=False, stream=None):
        """Host-side convenience: returns (status, loglik, particles [N][P] or None,
        ancestors [T][P] or None).  PF_EDEGENERATE is returned, not raised."""
        theta = np.ascontiguousarray(theta, dtype=np.float64) if not hasattr(theta, "data_ptr") else theta
        y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
        ll = np.zeros(1, dtype=np.float64)
        x = np.zeros((self.N, self.P), dtype=self.state_dtype) if want_particles else None
        anc = np.zeros((self.T, self.P), dtype=np.int32) if want_ancestors else None
        st = pf_run(self, theta, y, seed, ll, x, anc, 0, stream)
        return st, float(ll[0]), x, anc

    def run_range(self, theta, y, seed, r, s, want_particles=False, stream=None):
        """Advance from t_r to t_s (y = the s - r observation rows y(t_{r+1..s})):
        returns (status, loglik of y(t_1..t_s), particles x(t_s) or None)."""
        theta = None if theta is None else (
            np.ascontiguousarray(theta, dtype=np.float64) if not hasattr(theta, "data_ptr") else theta)
        y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
        ll = np.zeros(1, dtype=np.float64)
        x = np.zeros((self.N, self.P), dtype=self.state_dtype) if want_particles else None
        st = pf_run_range(self, theta, y, seed, r, s, ll, x, stream)
        return st, float(ll[0]), x

    def sample_path(self, theta, y, seed, stream=None):
        """One path by ancestry: (status, loglik, path [T+1][N], indices [T+1])."""
        theta = np.ascontiguousarray(theta, dtype=np.float64) if not hasattr(theta, "data_ptr") else theta
        y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
        ll = np.zeros(1, dtype=np.float64)
        path = np.zeros((self.T + 1, self.N), dtype=np.float64)
        idx = np.zeros(self.T + 1, dtype=np.int32)
        st = pf_sample_path(self, theta, y, seed, ll, path, idx, stream)
        return st, float(ll[0]), path, idx

    def debug_step(self, theta, y, seed, i, x_prev, anc=None):
        """Teacher-forced step i from x(t_{i-1}) and a(t_i) (None: identity):
        returns (status, increment log Z_i, x(t_i) [N][P], a(t_{i+1}) [P] or
        None for i = T)."""
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        x_prev = np.ascontiguousarray(x_prev, dtype=self.state_dtype)
        anc = None if anc is None else np.ascontiguousarray(anc, dtype=np.int32)
        x = np.zeros((self.N, self.P), dtype=self.state_dtype)
        inc = np.zeros(1, dtype=np.float64)
        nxt = np.zeros(self.P, dtype=np.int32) if i < self.T else None
        st = lib().pf_debug_step(self.h, _ptr(theta), _ptr(y), ctypes.c_uint64(seed), i,
                                 _ptr(x_prev), _ptr(anc), _ptr(x), _ptr(inc), _ptr(nxt))
        st = _check(st, ok=(PF_OK, PF_EDEGENERATE))
        return st, float(inc[0]), x, nxt

    def destroy(self):
        if self.h:
            lib().pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pf_create(m, P, T, dt):
    return Filter(m, P, T, dt)


def pf_run(f, theta, y, seed, loglik, final_particles=None, ancestors=None, flags=0, stream=None):
    """Raw call: every array argument is passed by pointer (numpy or torch)."""
    st = lib().pf_run(f.h, _ptr(theta), _ptr(y), ctypes.c_uint64(seed), _ptr(loglik),
                      _ptr(final_particles), _ptr(ancestors), flags, _stream_ptr(stream))
    return _check(st, ok=(PF_OK, PF_EDEGENERATE))


def pf_run_range(f, theta, y, seed, r, s, loglik, particles=None, stream=None):
    """Raw call of pf_run_range (array arguments by pointer)."""
    st = lib().pf_run_range(f.h, _ptr(theta), _ptr(y), ctypes.c_uint64(seed), r, s, _ptr(loglik),
                            _ptr(particles), _stream_ptr(stream))
    return _check(st, ok=(PF_OK, PF_EDEGENERATE))


def pf_sample_path(f, theta, y, seed, loglik, path, path_index=None, stream=None):
    """Raw call of pf_sample_path (array arguments by pointer)."""
    st = lib().pf_sample_path(f.h, _ptr(theta), _ptr(y), ctypes.c_uint64(seed), _ptr(loglik),
                              _ptr(path), _ptr(path_index), _stream_ptr(stream))
    return _check(st, ok=(PF_OK, PF_EDEGENERATE))


PF_NOALLOC_SCRATCH_BYTES = 32 << 20


def pf_run_noalloc(m, P, T, dt, theta, y, seed, loglik, status=None, final_particles=None,
                   stream=None):
    """Allocation-free run: every array is a device pointer (torch CUDA tensor);
    only enqueues on `stream`.  Raises PFError (PF_EINVAL) if the filter does not
    fit in the library's fixed scratch array, and ValueError for an array that
    is not a CUDA tensor (the library also refuses host pointers)."""
    for name, a in (("theta", theta), ("y", y), ("loglik", loglik), ("status", status),
                    ("final_particles", final_particles)):
        if a is not None and not getattr(a, "is_cuda", False):
            raise ValueError("pf_run_noalloc: %s must be a CUDA tensor" % name)
    st = lib().pf_run_noalloc(ctypes.byref(m), P, T, dt, _ptr(theta), _ptr(y),
                              ctypes.c_uint64(seed), _ptr(loglik), _ptr(status),
                              _ptr(final_particles), _stream_ptr(stream))
    return _check(st)


def pf_wait(f):
    return _check(lib().pf_wait(f.h), ok=(PF_OK, PF_EDEGENERATE))


def pf_destroy(f):
    f.destroy()


def pf_profile_enable(f, on=True):
    _check(lib().pf_profile_enable(f.h, 1 if on else 0))


PROFILE_KINDS = ("init", "propagate", "resample", "results")


def pf_profile_read(f):
    """{kind: (total ms, launches)} for the runs since the last read."""
    ms = (ctypes.c_double * 4)()
    n = (ctypes.c_int64 * 4)()
    _check(lib().pf_profile_read(f.h, ms, n))
    return {k: (ms[i], n[i]) for i, k in enumerate(PROFILE_KINDS)}


def pf_measure_fma_peak(prec):
    """Measured FMA throughput (flop/s) of the current GPU for PF_FP64 or PF_MIXED (FP32)."""
    f = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib().pf_measure_fma_peak(prec, ctypes.byref(f), ctypes.byref(ms)))
    return f.value


def pf_debug_fail_allocation(k):
    """Fault injection: the k-th next device allocation of a filter or a served
    request fails as if the device were out of memory (once); 0 disarms."""
    _check(lib().pf_debug_fail_allocation(k))


def pf_debug_persist_wait_limit(seconds):
    """How long a CTA of a later persistent batch launch waits for a work item
    before the launch ends with PF_ETIMEOUT (current device; 4 s at load)."""
    _check(lib().pf_debug_persist_wait_limit(float(seconds)))


def pf_debug_persist_unfilled_slot(on):
    """Fault injection: persistent plans built afterwards count one slot that
    nothing fills (its wait runs out); False disarms."""
    _check(lib().pf_debug_persist_unfilled_slot(1 if on else 0))


def pf_debug_fail_server_wait(k):
    """Fault injection: the k-th next wait of a server's scheduler reports a
    CUDA error (once; 0 disarms); that server ends its requests with PF_ECUDA
    and refuses new ones."""
    _check(lib().pf_debug_fail_server_wait(k))


def pf_debug_check_counts():
    """(checked build?, {invariant: violations since the last call}) -- the
    counters of a PF_CHECKED=1 library (PF_B300_CHECKED=1); zeros otherwise."""
    c = (ctypes.c_uint64 * 4)()
    chk = ctypes.c_int32()
    _check(lib().pf_debug_check_counts(c, ctypes.byref(chk)))
    names = ("ancestor_out_of_range", "state_not_finite", "prefix_not_monotone",
             "offspring_range_invalid")
    return bool(chk.value), {n: int(v) for n, v in zip(names, c)}


def pf_weight_sum_log(s):
    """log s evaluated on the GPU by the step combine's weight-sum logarithm
    (diagnostic; s: float64 array, returns a new float64 array)."""
    s = np.ascontiguousarray(s, dtype=np.float64)
    y = np.empty_like(s)
    _check(lib().pf_weight_sum_log(s.ctypes.data, y.ctypes.data, s.size))
    return y


def pf_weight_exp(d):
    """e^d evaluated on the GPU by the propagate kernels' weight exponential
    (diagnostic; d: float64 array, returns a new float64 array)."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    w = np.empty_like(d)
    _check(lib().pf_weight_exp(d.ctypes.data, w.ctypes.data, d.size))
    return w


def pf_weight_prefix(w):
    """The propagate kernels' in-tile cumulative weights of the given weights
    in [0, 1], per tile of 256 (diagnostic): returns (prefix, totals)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    prefix = np.empty_like(w)
    totals = np.empty((w.size + 255) // 256, dtype=np.float64)
    _check(lib().pf_weight_prefix(w.ctypes.data, prefix.ctypes.data, totals.ctypes.data, w.size))
    return prefix, totals


def pf_batch_configure(filters, cta_max_particles):
    """Send the filters of this list with at most cta_max_particles particles
    to the thread-block cluster path (0: none); results do not change."""
    nf = len(filters)
    hs = (_vp * nf)(*[f.h for f in filters])
    _check(lib().pf_batch_configure(nf, hs, int(cta_max_particles)))


def pf_batch_set_shape(filters, cta_max_particles=0, branches=4, resample_blocks_per_sm=8,
                       persistent_blocks_per_sm=0, tiles_per_item=1):
    """Set the launch shape used for this filter list (results do not change)."""
    nf = len(filters)
    hs = (_vp * nf)(*[f.h for f in filters])
    sh = pf_batch_shape(int(cta_max_particles), int(branches), int(resample_blocks_per_sm),
                        int(persistent_blocks_per_sm), int(tiles_per_item))
    _check(lib().pf_batch_set_shape(nf, hs, ctypes.byref(sh)))


def pf_batch_get_shape(filters):
    """The launch shape used for this filter list, as a dict."""
    nf = len(filters)
    hs = (_vp * nf)(*[f.h for f in filters])
    sh = pf_batch_shape()
    _check(lib().pf_batch_get_shape(nf, hs, ctypes.byref(sh)))
    return sh.as_dict()


def pf_batch_autotune(filters, thetas, ys, seeds):
    """Time candidate launch shapes on these inputs (cluster bound, branches,
    resample grid, one field at a time, then the persistent launch's CTAs per
    SM with its tiles per item, jointly), keep the fastest for the list and
    return its cluster bound (pf_batch_get_shape gives the whole shape)."""
    nf = len(filters)
    hs = (_vp * nf)(*[f.h for f in filters])
    th = [np.ascontiguousarray(t, dtype=np.float64) if not hasattr(t, "data_ptr") else t
          for t in thetas]
    yy = [np.ascontiguousarray(v, dtype=np.float64) if not hasattr(v, "data_ptr") else v
          for v in ys]
    tp = (_vp * nf)(*[_ptr(t) for t in th])
    yp = (_vp * nf)(*[_ptr(v) for v in yy])
    sd = (ctypes.c_uint64 * nf)(*[int(x) for x in seeds])
    chosen = ctypes.c_int64()
    _check(lib().pf_batch_autotune(nf, hs, tp, yp, sd, ctypes.byref(chosen)))
    return chosen.value


def pf_batch_run(filters, thetas, ys, seeds, stream=None):
    """Run many filters in one launch plan; returns (logliks, statuses) numpy arrays."""
    n = len(filters)
    keep = []
    th = []
    yy = []
    for t, y in zip(thetas, ys):
        t = np.ascontiguousarray(t, dtype=np.float64) if not hasattr(t, "data_ptr") else t
        y = np.ascontiguousarray(y, dtype=np.float64) if not hasattr(y, "data_ptr") else y
        keep += [t, y]
        th.append(_ptr(t))
        yy.append(_ptr(y))
    fa = (_vp * n)(*[f.h for f in filters])
    ta = (_vp * n)(*th)
    ya = (_vp * n)(*yy)
    sa = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
    lls = np.zeros(n, dtype=np.float64)
    sts = np.zeros(n, dtype=np.int32)
    st = lib().pf_batch_run(n, fa, ta, ya, sa, lls.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                            sts.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _stream_ptr(stream))
    _check(st)
    return lls, sts


class Server:
    """Continuous-batching request server (pf_server_* of the C ABI)."""

    def __init__(self, device_mem_budget, max_slots=64):
        h = _vp()
        _check(lib().pf_server_create(device_mem_budget, max_slots, ctypes.byref(h)))
        self.h = h

    def submit(self, m, P, T, dt, theta, y, seed):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        t = ctypes.c_uint64()
        _check(lib().pf_server_submit(self.h, ctypes.byref(m), P, T, dt, _ptr(theta), _ptr(y),
                                      ctypes.c_uint64(seed), ctypes.byref(t)))
        return t.value

    def poll(self, ticket):
        """None while pending, else (status, loglik, latency_s)."""
        ll = ctypes.c_double()
        lat = ctypes.c_double()
        st = lib().pf_server_poll(self.h, ticket, ctypes.byref(ll), ctypes.byref(lat))
        if st == PF_EBUSY:
            return None
        _check(st, ok=(PF_OK, PF_EDEGENERATE))
        return st, ll.value, lat.value

    def configure(self, branches):
        """Launch groups per scheduler iteration (1..8); results do not depend on it."""
        _check(lib().pf_server_configure(self.h, int(branches)))

    def stats(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(lib().pf_server_stats(self.h, *[ctypes.byref(x) for x in v]))
        return dict(queued=v[0].value, running=v[1].value, completed=v[2].value,
                    iterations=v[3].value)

    def destroy(self):
        if self.h:
            lib().pf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def pf_server_create(device_mem_budget, max_slots=64, branches=None):
    s = Server(device_mem_budget, max_slots)
    if branches is not None:
        s.configure(branches)
    return s
