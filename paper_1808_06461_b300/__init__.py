"""Python binding of the B300 channel library (``libchan.so``, C ABI in include/chan.h).

Argument marshalling only: every step of the substep runs in the library's
CUDA kernels.  Importing this module does not need a GPU; creating a
channel does.  If the shared object is missing the import raises -- there
is no CPU fallback.

Host arrays are numpy complex128 of shape (Ny, Nz, Nx//2) for Fourier
fields (index [j, jz, kx], kz in FFT order, kz Nyquist row zero) and
float64 of shape (Ny,) for profiles.  Device arrays (the ``*_device``
calls) are torch tensors with the same shapes and dtypes.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libchan.so")

CHAN_OK, CHAN_EINVAL, CHAN_ENOMEM, CHAN_ECUDA, CHAN_ENAN, CHAN_ESTATE, CHAN_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
CHAN_BATCH_PERSISTENT = 1
CHAN_FILTER_SHARP, CHAN_FILTER_BOX = 0, 1
CHAN_PREC_FP64, CHAN_PREC_MIXED, CHAN_PREC_F64X, CHAN_PREC_MIXED_DF = 0, 1, 2, 3
CHAN_NSTAT = 20

# Exported symbols, exactly the declarations of include/chan.h.
SYMBOLS = ("chan_opts_default", "chan_init", "chan_init_ex", "chan_free", "chan_last_error",
           "chan_fourier_count", "chan_device_bytes", "chan_get_grid", "chan_set_state",
           "chan_set_state_device", "chan_get_state", "chan_get_state_device", "chan_step",
           "chan_filter_stresses", "chan_stats", "chan_nonlinear", "chan_sync", "chan_time",
           "chan_substeps", "chan_profile", "chan_profile_read", "chan_kernel_name",
           "chan_rhs_terms", "chan_rhs_terms_noalloc", "chan_footprint_bytes", "chan_set_graph",
           "chan_filtered_enstrophy", "chan_batch_create", "chan_batch_step", "chan_batch_last_error",
           "chan_batch_free", "chan_autotune", "chan_tuned_shape", "chan_database_record",
           "chan_spectra", "chan_optimize_mesh", "chan_filtered_pressure", "chan_checkpoint_bytes",
           "chan_checkpoint_save", "chan_checkpoint_load", "chan_batch_create_ex", "chan_batch_status",
           "chan_batch_set_wait", "chan_batch_persistent_grid", "chan_batch_step_each")
CHAN_NKERNELS = 18


class chan_opts(ctypes.Structure):
    _fields_ = [("re_tau", ctypes.c_double), ("Lx", ctypes.c_double), ("Lz", ctypes.c_double),
                ("Nx", ctypes.c_int), ("Ny", ctypes.c_int), ("Nz", ctypes.c_int),
                ("dt", ctypes.c_double), ("eta_w", ctypes.c_double), ("grid_re", ctypes.c_double),
                ("precision", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("mesh", ctypes.POINTER(ctypes.c_double)), ("slab_planes", ctypes.c_int),
                ("lean_tables", ctypes.c_int), ("y_tables", ctypes.c_int), ("keep_rhs", ctypes.c_int)]


class ChanError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("chan error %d: %s" % (code, msg))
        self.code = code


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("libchan.so not built (run paper_1808_06461_b300/build.py); "
                          "the channel substep has no fallback implementation")
    lib = ctypes.CDLL(path)
    P, D, I, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
    DP = ctypes.POINTER(ctypes.c_double)
    sig = {
        "chan_opts_default": (None, [ctypes.POINTER(chan_opts)]),
        "chan_init": (I, [ctypes.POINTER(P), D, D, D, I, I, I, D]),
        "chan_init_ex": (I, [ctypes.POINTER(P), ctypes.POINTER(chan_opts)]),
        "chan_free": (None, [P]),
        "chan_last_error": (ctypes.c_char_p, [P]),
        "chan_fourier_count": (S, [P]),
        "chan_device_bytes": (S, [P]),
        "chan_get_grid": (I, [P, DP]),
        "chan_set_state": (I, [P, P, P, P, P]),
        "chan_set_state_device": (I, [P, P, P, P, P]),
        "chan_get_state": (I, [P, P, P, P, P]),
        "chan_get_state_device": (I, [P, P, P, P, P]),
        "chan_checkpoint_bytes": (ctypes.c_size_t, [P]),
        "chan_checkpoint_save": (I, [P, P]),
        "chan_checkpoint_load": (I, [P, P]),
        "chan_step": (I, [P, I]),
        "chan_filter_stresses": (I, [P, I, D, D, P, P]),
        "chan_stats": (I, [P, P, DP, DP, DP]),
        "chan_nonlinear": (I, [P, P]),
        "chan_rhs_terms": (I, [P, P]),
        "chan_rhs_terms_noalloc": (I, [P, P, P]),
        "chan_footprint_bytes": (S, [I, I, I, I]),
        "chan_set_graph": (I, [P, I]),
        "chan_filtered_enstrophy": (I, [P, I, D, D, P]),
        "chan_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I, P]),
        "chan_batch_create_ex": (I, [ctypes.POINTER(P), ctypes.POINTER(P), I, P, I]),
        "chan_batch_status": (I, [P]),
        "chan_batch_step_each": (I, [P, P]),
        "chan_batch_set_wait": (I, [P, ctypes.c_longlong, I, I]),
        "chan_batch_persistent_grid": (I, [P]),
        "chan_batch_step": (I, [P, I]),
        "chan_batch_last_error": (ctypes.c_char_p, [P]),
        "chan_batch_free": (None, [P]),
        "chan_autotune": (I, [P]),
        "chan_database_record": (I, [P, D, D, P, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "chan_spectra": (I, [P, P]),
        "chan_filtered_pressure": (I, [P, I, D, D, P]),
        "chan_optimize_mesh": (I, [ctypes.POINTER(chan_opts), I, D, P, DP, DP]),
        "chan_tuned_shape": (I, [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]),
        "chan_sync": (I, [P]),
        "chan_time": (D, [P]),
        "chan_substeps": (ctypes.c_longlong, [P]),
        "chan_profile": (I, [P, I]),
        "chan_profile_read": (I, [P, P, P]),
        "chan_kernel_name": (ctypes.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = load_library()


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(a.data_ptr()))   # torch tensor on the device


def _need(a, shape, dtype):
    if not (isinstance(a, np.ndarray) and a.shape == tuple(shape) and a.dtype == dtype and a.flags.c_contiguous
            and a.flags.writeable):
        raise ValueError("output array must be a writeable C-contiguous %s array of shape %s" % (np.dtype(dtype), shape))


def _check(h, rc):
    if rc != CHAN_OK:
        raise ChanError(rc, _lib.chan_last_error(h).decode())


class Channel:
    """One channel box on the current CUDA device (owns its device memory).

    precision: CHAN_PREC_FP64; CHAN_PREC_MIXED (FP32 transforms and products, FP64
    wall-normal solves); CHAN_PREC_F64X (transforms, products and the substep's sweeps in
    FP32 pairs, about 2^-47); CHAN_PREC_MIXED_DF (FP32 transforms and products, pair sweeps).
    The mean flow and the statistics are FP64 in every mode.
    """

    def __init__(self, re_tau, Lx, Lz, Nx, Ny, Nz, dt, precision=CHAN_PREC_FP64, eta_w=1.0,
                 grid_re=0.0, stream=None, mesh=None, slab_planes=0, lean_tables=0, y_tables=0, keep_rhs=0):
        o = chan_opts()
        _lib.chan_opts_default(ctypes.byref(o))
        o.re_tau, o.Lx, o.Lz, o.Nx, o.Ny, o.Nz, o.dt = re_tau, Lx, Lz, Nx, Ny, Nz, dt
        o.eta_w, o.grid_re, o.precision = eta_w, grid_re, precision
        o.slab_planes = int(slab_planes)
        o.lean_tables = int(lean_tables)
        o.y_tables = int(y_tables)
        o.keep_rhs = int(keep_rhs)
        o.stream = stream
        if mesh is not None:
            self._mesh = np.ascontiguousarray(mesh, dtype=np.float64)
            o.mesh = self._mesh.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        rc = _lib.chan_init_ex(ctypes.byref(h), ctypes.byref(o))
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_last_error(None).decode())
        self.h = h
        self.Nx, self.Ny, self.Nz, self.nxh = Nx, Ny, Nz, Nx // 2
        self.shape = (Ny, Nz, Nx // 2)

    def close(self):
        if getattr(self, "h", None):
            _lib.chan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- queries
    def grid(self):
        y = np.empty(self.Ny)
        _check(self.h, _lib.chan_get_grid(self.h, y.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return y

    def device_bytes(self):
        return int(_lib.chan_device_bytes(self.h))

    def time(self):
        return float(_lib.chan_time(self.h))

    def substeps(self):
        return int(_lib.chan_substeps(self.h))

    def autotune(self):
        """Pick z-pass columns per CTA, x-pass threads and the y-table placement for this shape
        (results unchanged); returns (kb_z, xthreads, ytab_global)."""
        _check(self.h, _lib.chan_autotune(self.h))
        return self.tuned_shape()

    def tuned_shape(self):
        kb, nt, yt = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.h, _lib.chan_tuned_shape(self.h, ctypes.byref(kb), ctypes.byref(nt), ctypes.byref(yt)))
        return kb.value, nt.value, yt.value

    def set_graph(self, enable=True):
        _check(self.h, _lib.chan_set_graph(self.h, 1 if enable else 0))

    # ---- tracing
    def profile(self, enable=True):
        _check(self.h, _lib.chan_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kernel name: (total ms, launches)} since the last profile(True)."""
        ms = np.zeros(CHAN_NKERNELS)
        n = np.zeros(CHAN_NKERNELS, dtype=np.int64)
        _check(self.h, _lib.chan_profile_read(self.h, _ptr(ms), _ptr(n)))
        return {_lib.chan_kernel_name(k).decode(): (float(ms[k]), int(n[k])) for k in range(CHAN_NKERNELS)}

    # ---- state
    def set_state(self, v, omega2, U1, U3):
        v = np.ascontiguousarray(v, dtype=np.complex128)
        om = np.ascontiguousarray(omega2, dtype=np.complex128)
        U1 = np.ascontiguousarray(U1, dtype=np.float64)
        U3 = np.ascontiguousarray(U3, dtype=np.float64)
        if v.shape != self.shape or om.shape != self.shape or U1.shape != (self.Ny,) or U3.shape != (self.Ny,):
            raise ValueError("state shapes must be %s and (%d,)" % (self.shape, self.Ny))
        _check(self.h, _lib.chan_set_state(self.h, _ptr(v), _ptr(om), _ptr(U1), _ptr(U3)))

    def set_state_device(self, v, omega2, U1, U3):
        _check(self.h, _lib.chan_set_state_device(self.h, _ptr(v), _ptr(omega2), _ptr(U1), _ptr(U3)))

    def get_state(self, out=None):
        """The state (v, omega2, U1, U3) in host arrays; ``out`` (a dict of C-contiguous arrays
        of the right shapes and dtypes, e.g. in pinned memory) is filled instead of new arrays."""
        if out is None:
            out = dict(v=np.empty(self.shape, dtype=np.complex128), omega2=np.empty(self.shape, dtype=np.complex128),
                       U1=np.empty(self.Ny), U3=np.empty(self.Ny))
        _need(out["v"], self.shape, np.complex128)
        _need(out["omega2"], self.shape, np.complex128)
        _need(out["U1"], (self.Ny,), np.float64)
        _need(out["U3"], (self.Ny,), np.float64)
        _check(self.h, _lib.chan_get_state(self.h, _ptr(out["v"]), _ptr(out["omega2"]), _ptr(out["U1"]),
                                           _ptr(out["U3"])))
        return out

    def checkpoint(self, out=None):
        """Everything the next substep reads, as bytes (a uint8 array; ``out`` to fill one)."""
        n = int(_lib.chan_checkpoint_bytes(self.h))
        buf = np.empty(n, dtype=np.uint8) if out is None else out
        if buf.nbytes < n or buf.dtype != np.uint8 or not buf.flags.c_contiguous:
            raise ValueError("checkpoint buffer must be a C-contiguous uint8 array of at least %d bytes" % n)
        _check(self.h, _lib.chan_checkpoint_save(self.h, buf.ctypes.data_as(ctypes.c_void_p)))
        return buf

    def restore(self, buf):
        """Continue from a checkpoint of a handle with the same box, grid, dt and precision."""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(self.h, _lib.chan_checkpoint_load(self.h, buf.ctypes.data_as(ctypes.c_void_p)))

    def get_state_device(self, v, omega2, U1, U3):
        _check(self.h, _lib.chan_get_state_device(self.h, _ptr(v), _ptr(omega2), _ptr(U1), _ptr(U3)))

    # ---- the substep and its outputs
    def step(self, nsub=1):
        _check(self.h, _lib.chan_step(self.h, int(nsub)))

    def sync(self):
        _check(self.h, _lib.chan_sync(self.h))

    def nonlinear(self):
        H = np.empty((3,) + self.shape, dtype=np.complex128)
        _check(self.h, _lib.chan_nonlinear(self.h, _ptr(H)))
        return H

    def rhs_terms(self):
        """(N_chi, N_omega2) of the current state, shape (2, Ny, Nz, Nx/2)."""
        N = np.empty((2,) + self.shape, dtype=np.complex128)
        _check(self.h, _lib.chan_rhs_terms(self.h, _ptr(N)))
        return N

    def filter_stresses(self, kind, p1, p3, want=True, out=None):
        """(ubar, tau) of shapes (3,) + shape and (6,) + shape; ``out`` = (ubar, tau) arrays to fill."""
        if out is not None:
            ub, tau = out
            _need(ub, (3,) + self.shape, np.complex128)
            _need(tau, (6,) + self.shape, np.complex128)
        else:
            ub = np.empty((3,) + self.shape, dtype=np.complex128) if want else None
            tau = np.empty((6,) + self.shape, dtype=np.complex128) if want else None
        _check(self.h, _lib.chan_filter_stresses(self.h, int(kind), float(p1), float(p3), _ptr(ub), _ptr(tau)))
        return ub, tau

    def filtered_enstrophy(self, kind, p1, p3):
        """filt(omega_i omega_i), shape (Ny, Nz, Nx/2)."""
        ens = np.empty(self.shape, dtype=np.complex128)
        _check(self.h, _lib.chan_filtered_enstrophy(self.h, int(kind), float(p1), float(p3), _ptr(ens)))
        return ens

    def database_record(self, p1=120.0, p3=60.0):
        """The ten stored variables on the sharp filter's retained modes, shape (10, Ny, M3, M1)."""
        m1, m3 = ctypes.c_int(), ctypes.c_int()
        _check(self.h, _lib.chan_database_record(self.h, float(p1), float(p3), None, ctypes.byref(m1), ctypes.byref(m3)))
        rec = np.empty((10, self.Ny, m3.value, m1.value), dtype=np.complex128)
        _check(self.h, _lib.chan_database_record(self.h, float(p1), float(p3), _ptr(rec), ctypes.byref(m1),
                                                 ctypes.byref(m3)))
        return rec

    def filtered_pressure(self, kind, p1, p3):
        """pbar from the filtered stresses (Sec. 3.1, Eq. (2)), shape (Ny, Nz, Nx/2)."""
        pr = np.empty(self.shape, dtype=np.complex128)
        _check(self.h, _lib.chan_filtered_pressure(self.h, int(kind), float(p1), float(p3), _ptr(pr)))
        return pr

    def spectra(self):
        """E_i(k1, y, k3), shape (3, Ny, Nz, Nx/2)."""
        E = np.empty((3,) + self.shape)
        _check(self.h, _lib.chan_spectra(self.h, _ptr(E)))
        return E

    def stats(self):
        out = np.empty((CHAN_NSTAT, self.Ny))
        ut, ub, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(self.h, _lib.chan_stats(self.h, _ptr(out), ctypes.byref(ut), ctypes.byref(ub), ctypes.byref(f)))
        return out, ut.value, ub.value, f.value


class ChannelBatch:
    """Packed stepping of several Channels of one precision: one launch per kernel for all,
    or (persistent=True, at most 16 runs) persistent work-list launches of up to 48
    substeps of every run."""

    def __init__(self, channels, stream=None, persistent=False):
        self.channels = list(channels)
        arr = (ctypes.c_void_p * len(self.channels))(*[c.h.value for c in self.channels])
        b = ctypes.c_void_p()
        flags = CHAN_BATCH_PERSISTENT if persistent else 0
        rc = _lib.chan_batch_create_ex(ctypes.byref(b), arr, len(self.channels), stream, flags)
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_batch_last_error(None).decode())
        self.b = b
        self.persistent = bool(persistent)

    def step(self, nsub):
        rc = _lib.chan_batch_step(self.b, int(nsub))
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_batch_last_error(self.b).decode())

    def step_each(self, nsub):
        """Persistent batches: run r advances by nsub[r] substeps (counts may differ)."""
        arr = (ctypes.c_int * len(self.channels))(*[int(k) for k in nsub])
        rc = _lib.chan_batch_step_each(self.b, arr)
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_batch_last_error(self.b).decode())

    def status(self):
        """Wait for the batch; raises ChanError(CHAN_ETIMEOUT) if a persistent wait ran out."""
        rc = _lib.chan_batch_status(self.b)
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_batch_last_error(self.b).decode())

    def set_wait(self, polls, hold_run=-1, hold_stage=-1):
        """Wait limit of the persistent launches; (hold_run, hold_stage) for timeout tests."""
        rc = _lib.chan_batch_set_wait(self.b, int(polls), int(hold_run), int(hold_stage))
        if rc != CHAN_OK:
            raise ChanError(rc, _lib.chan_batch_last_error(self.b).decode())

    def persistent_grid(self):
        return int(_lib.chan_batch_persistent_grid(self.b))

    def close(self):
        if getattr(self, "b", None):
            _lib.chan_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# Module-level functions with the C names, for callers that prefer them.
def chan_init(re_tau, Lx, Lz, Nx, Ny, Nz, dt, **kw):
    return Channel(re_tau, Lx, Lz, Nx, Ny, Nz, dt, **kw)


def chan_set_state(ch, v, omega2, U1, U3):
    ch.set_state(v, omega2, U1, U3)


def chan_get_state(ch):
    return ch.get_state()


def chan_step(ch, nsub=1):
    ch.step(nsub)


def chan_filter_stresses(ch, kind, p1, p3):
    return ch.filter_stresses(kind, p1, p3)


def chan_stats(ch):
    return ch.stats()


def chan_nonlinear(ch):
    return ch.nonlinear()


def chan_free(ch):
    ch.close()


def chan_sync(ch):
    ch.sync()


def optimize_mesh(re_tau, Lx, Lz, Nx, Ny, Nz, dt, iters=60, C=1e-3, eta_w=1.0, grid_re=0.0):
    """Appendix B mesh: (y, |g - g_ana| before, after).  Host only."""
    o = chan_opts()
    _lib.chan_opts_default(ctypes.byref(o))
    o.re_tau, o.Lx, o.Lz, o.Nx, o.Ny, o.Nz, o.dt, o.eta_w, o.grid_re = re_tau, Lx, Lz, Nx, Ny, Nz, dt, eta_w, grid_re
    y = np.empty(Ny)
    eb, ea = ctypes.c_double(), ctypes.c_double()
    rc = _lib.chan_optimize_mesh(ctypes.byref(o), int(iters), float(C), _ptr(y), ctypes.byref(eb), ctypes.byref(ea))
    if rc != CHAN_OK:
        raise ChanError(rc, _lib.chan_last_error(None).decode())
    return y, eb.value, ea.value


def footprint_bytes(Nx, Ny, Nz, precision=CHAN_PREC_FP64):
    """Device bytes a channel of this size would allocate (no GPU needed)."""
    return int(_lib.chan_footprint_bytes(int(Nx), int(Ny), int(Nz), int(precision)))


def library():
    return _lib
