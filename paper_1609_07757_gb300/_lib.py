"""ctypes binding of libiscsi.so (include/iscsi.h): argument marshalling only.

Every function keeps the C name.  Device arguments accept torch CUDA tensors
(their data pointer is passed) or raw integer addresses; host arguments
accept numpy arrays.  A negative status raises ``IscsiError`` with the
library's last error message.  There is no fallback: if the CUDA library
cannot be built or loaded, importing this module's functions raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

ISCSI_OK = 0
ISCSI_E_ARG = -1
ISCSI_E_NOMEM = -2
ISCSI_E_CUDA = -3
ISCSI_E_NOCONV = -4
ISCSI_E_NOINIT = -5
ISCSI_E_NAN = -6
ISCSI_E_WAIT = -7

_lib = None


class IscsiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("iscsi status %d: %s" % (status, msg))
        self.status = status


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libiscsi.so (building it first if needed) and declare the ABI."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise OSError("libiscsi.so not built: %s" % path)
    lib = ctypes.CDLL(path)
    c_int, c_ll, c_d, vp = ctypes.c_int, ctypes.c_longlong, ctypes.c_double, ctypes.c_void_p
    sig = {
        "iscsi_init": (c_int, [c_int, c_int, c_int, c_int, vp, vp, c_d]),
        "iscsi_sigma": (c_int, [vp, vp, c_int]),
        "iscsi_sigma_host": (c_int, [vp, vp, c_int]),
        "iscsi_sigma_noalloc": (c_int, [vp, vp]),
        "iscsi_davidson": (c_int, [c_int, c_d, vp, vp]),
        "iscsi_check_bounded_wait": (c_int, [c_ll]),
        "iscsi_check_schedule": (c_int, [c_int, vp, vp, vp, vp, vp, c_int, vp, vp]),
        "iscsi_density": (c_int, [vp, vp, vp, vp]),
        "iscsi_propagate": (c_int, [vp, c_int, c_d, vp, c_int, c_int, c_int, vp]),
        "iscsi_density_host": (c_int, [vp, vp, vp, vp]),
        "iscsi_set_gas": (c_int, [c_int, vp, vp, vp, vp]),
        "iscsi_init_gas": (c_int, [c_int, c_int, c_int, c_int, vp, vp, vp, vp, vp, c_d]),
        "iscsi_gas_mask": (c_int, [vp]),
        "iscsi_ndet": (c_ll, []),
        "iscsi_nstrings": (c_ll, [c_int]),
        "iscsi_get_strings": (c_int, [c_int, vp, vp]),
        "iscsi_det_index": (c_ll, [vp, vp]),
        "iscsi_diagonal": (c_int, [vp]),
        "iscsi_set_stream": (c_int, [vp]),
        "iscsi_set_option": (c_int, [ctypes.c_char_p, c_d]),
        "iscsi_stats": (c_int, [ctypes.c_char_p, c_int]),
        "iscsi_updates_per_sigma": (c_d, []),
        "iscsi_last_error": (ctypes.c_char_p, []),
        "iscsi_finalize": (None, []),
        "iscsi_ctx_current": (c_int, []),
        "iscsi_ctx_use": (c_int, [c_int]),
        "iscsi_ctx_destroy": (c_int, [c_int]),
        "iscsi_batch_sigma": (c_int, [vp, vp, vp, c_int, c_int]),
        "iscsi_batch_check": (c_int, []),
        "iscsi_batch_davidson": (c_int, [vp, c_int, c_int, c_d, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status < 0:
        msg = load().iscsi_last_error()
        raise IscsiError(status, msg.decode() if msg else "")
    return status


def _dev(x):
    """Device address of a torch tensor (checked FP64 and contiguous) or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    import torch
    if not (x.is_cuda and x.dtype == torch.float64 and x.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return x.data_ptr()


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.c_void_p)


def iscsi_set_stream(stream=None):
    """Use a torch.cuda.Stream (or its raw handle); None = torch's current stream."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    handle = getattr(stream, "cuda_stream", stream)
    return _check(load().iscsi_set_stream(ctypes.c_void_p(handle)))


def iscsi_init(norb, nalpha, nbeta, max_excitation, h1, eri, tau):
    h, hp = _host_f64(h1)
    if eri is None:
        ep = None
    else:
        e, ep = _host_f64(eri)
    return _check(load().iscsi_init(norb, nalpha, nbeta, max_excitation, hp, ep, float(tau)))


def iscsi_sigma(c, sigma, nvec=1):
    return _check(load().iscsi_sigma(_dev(c), _dev(sigma), int(nvec)))


def iscsi_batch_sigma(handles, cs, sigmas, nvec=1):
    """sigma_i = H(context handles[i]) c_i for all i in one call (device tensors)."""
    n = len(handles)
    if len(cs) != n or len(sigmas) != n:
        raise ValueError("handles, cs and sigmas differ in length")
    h = (ctypes.c_int * n)(*[int(x) for x in handles])
    c = (ctypes.c_void_p * n)(*[_dev(x) for x in cs])
    s = (ctypes.c_void_p * n)(*[_dev(x) for x in sigmas])
    return _check(load().iscsi_batch_sigma(h, c, s, n, int(nvec)))


def iscsi_batch_check():
    return _check(load().iscsi_batch_check())


def iscsi_batch_davidson(handles, nroots, tol, vecs=None):
    """Lowest nroots eigenpairs of several contexts iterated together.
    Returns (status, energies [count][nroots], per-context statuses)."""
    n = len(handles)
    h = (ctypes.c_int * n)(*[int(x) for x in handles])
    e = np.zeros((n, nroots), dtype=np.float64)
    sts = (ctypes.c_int * n)()
    vp = None
    if vecs is not None:
        vp = (ctypes.c_void_p * n)(*[(_dev(v) if v is not None else None) for v in vecs])
    st = load().iscsi_batch_davidson(h, n, int(nroots), float(tol), e.ctypes.data_as(ctypes.c_void_p), vp, sts)
    if st < 0 and st not in (ISCSI_E_NOCONV,):
        _check(st)
    return st, e, list(sts)


def iscsi_sigma_noalloc(c, sigma):
    """FP64 single-vector sigma that allocates no device memory (static scratch)."""
    return _check(load().iscsi_sigma_noalloc(_dev(c), _dev(sigma)))


def iscsi_sigma_host(c, sigma, nvec=1):
    """c, sigma: host numpy float64 arrays of nvec * ndet elements (sigma is written)."""
    if not (isinstance(sigma, np.ndarray) and sigma.dtype == np.float64 and sigma.flags.c_contiguous):
        raise ValueError("sigma must be a C-contiguous float64 numpy array")
    cc, cp = _host_f64(c)
    return _check(load().iscsi_sigma_host(cp, sigma.ctypes.data_as(ctypes.c_void_p), int(nvec)))


def iscsi_density(bra, ket, d1, d2):
    """Spin-resolved density matrices of Eqs. d1, d2 on the device.
    bra, ket: device FP64 [ndet] (ket None: ket = bra); d1: device FP64
    [2, n, n] or None; d2: device FP64 [3, n, n, n, n] or None."""
    return _check(load().iscsi_density(_dev(bra), _dev(ket), _dev(d1), _dev(d2)))


def iscsi_density_host(bra, ket, d1, d2):
    """Host form: bra, ket numpy float64 [ndet] (ket may be None); d1 / d2
    C-contiguous float64 numpy outputs of 2 n^2 / 3 n^4 elements, or None."""
    for o in (d1, d2):
        if o is not None and not (isinstance(o, np.ndarray) and o.dtype == np.float64 and o.flags.c_contiguous):
            raise ValueError("outputs must be C-contiguous float64 numpy arrays")
    bb, bp = _host_f64(bra)
    kk, kp = _host_f64(ket) if ket is not None else (None, None)
    p1 = d1.ctypes.data_as(ctypes.c_void_p) if d1 is not None else None
    p2 = d2.ctypes.data_as(ctypes.c_void_p) if d2 is not None else None
    return _check(load().iscsi_density_host(bp, kp, p1, p2))


def iscsi_propagate(c, nsteps, dt, field=None, coupling=0, krylov=12, imaginary=False):
    """Propagate c (device FP64: [2, ndet] real time, [ndet] imaginary time) in
    place; returns the per-step diagnostics [nsteps, 2] (error indicator, energy)."""
    diag = np.zeros((nsteps, 2))
    fp = None
    if field is not None:
        fa = np.ascontiguousarray(field, dtype=np.float64)
        if fa.shape != (nsteps,):
            raise ValueError("field must have nsteps samples")
        fp = fa.ctypes.data_as(ctypes.c_void_p)
    _check(load().iscsi_propagate(_dev(c), int(nsteps), float(dt), fp, int(coupling), int(krylov),
                                  1 if imaginary else 0, diag.ctypes.data_as(ctypes.c_void_p)))
    return diag


def iscsi_set_gas(sizes=(), cmin=(), cmax=()):
    """GAS restriction of the current context (empty sizes: none); returns the
    number of kept determinants."""
    n = len(sizes)
    if len(cmin) != n or len(cmax) != n:
        raise ValueError("one (cmin, cmax) pair per subspace")
    arrs = [np.ascontiguousarray(x, dtype=np.int32) for x in (sizes, cmin, cmax)]
    ptrs = [a.ctypes.data_as(ctypes.c_void_p) if n else None for a in arrs]
    kept = ctypes.c_longlong(0)
    _check(load().iscsi_set_gas(n, ptrs[0], ptrs[1], ptrs[2], ctypes.byref(kept)))
    return int(kept.value)


def iscsi_init_gas(norb, nalpha, nbeta, sizes, cmin, cmax, h1, eri, tau):
    """A new current context on the GAS space of the accumulated limits (see iscsi_init_gas)."""
    n = len(sizes)
    if len(cmin) != n or len(cmax) != n or n == 0:
        raise ValueError("one (cmin, cmax) pair per subspace, at least one subspace")
    arrs = [np.ascontiguousarray(x, dtype=np.int32) for x in (sizes, cmin, cmax)]
    h, hp = _host_f64(h1)
    ep = None
    if eri is not None:
        e, ep = _host_f64(eri)
    return _check(load().iscsi_init_gas(norb, nalpha, nbeta, n, *[a.ctypes.data_as(ctypes.c_void_p) for a in arrs],
                                        hp, ep, float(tau)))


def iscsi_gas_mask(mask):
    """Copy the determinant mask into mask (a contiguous uint8 CUDA tensor of ndet elements)."""
    import torch
    if not (mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous() and mask.numel() == iscsi_ndet()):
        raise ValueError("expected a contiguous uint8 CUDA tensor of ndet elements")
    _check(load().iscsi_gas_mask(mask.data_ptr()))


def iscsi_check_bounded_wait(polls):
    """The bounded waits' failure path (ISCSI_E_WAIT is the expected status; raises IscsiError with it)."""
    return _check(load().iscsi_check_bounded_wait(int(polls)))


def iscsi_check_schedule(problems, nsm):
    """Plan synthetic contraction problems, each (M, N, [(K, nrows_b), ...]),
    for nsm SMs and check the plan (host only).  Returns (balance, counts) with
    counts = {"ctas", "items", "tiles", "split_tiles", "faults"}."""
    M = np.array([p[0] for p in problems], dtype=np.int32)
    N = np.array([p[1] for p in problems], dtype=np.int32)
    nseg = np.array([len(p[2]) for p in problems], dtype=np.int32)
    K = np.array([g[0] for p in problems for g in p[2]], dtype=np.int32)
    nrb = np.array([g[1] for p in problems for g in p[2]], dtype=np.int32)
    bal = np.zeros(1)
    cnt = np.zeros(5, dtype=np.int32)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(load().iscsi_check_schedule(len(problems), ptr(M), ptr(N), ptr(nseg), ptr(K), ptr(nrb), int(nsm),
                                       ptr(bal), ptr(cnt)))
    return float(bal[0]), dict(zip(("ctas", "items", "tiles", "split_tiles", "faults"), (int(x) for x in cnt)))


def iscsi_davidson(nroots, tol, vecs=None):
    """Returns (status, energies); status is 0 or ISCSI_E_NOCONV (other errors raise)."""
    en = np.zeros(nroots)
    st = load().iscsi_davidson(int(nroots), float(tol), en.ctypes.data_as(ctypes.c_void_p), _dev(vecs))
    if st != ISCSI_E_NOCONV:
        _check(st)
    return st, en


def iscsi_ndet():
    return int(load().iscsi_ndet())


def iscsi_nstrings(spin):
    return int(load().iscsi_nstrings(spin))


def iscsi_get_strings(spin, nel):
    cnt = iscsi_nstrings(spin)
    orbs = np.zeros((cnt, max(nel, 1)), dtype=np.int32)
    lev = np.zeros(cnt, dtype=np.int32)
    _check(load().iscsi_get_strings(spin, orbs.ctypes.data_as(ctypes.c_void_p),
                                    lev.ctypes.data_as(ctypes.c_void_p)))
    return orbs[:, :nel], lev


def iscsi_det_index(alpha_orbitals, beta_orbitals):
    a = np.ascontiguousarray(list(alpha_orbitals) or [0], dtype=np.int32)
    b = np.ascontiguousarray(list(beta_orbitals) or [0], dtype=np.int32)
    return int(load().iscsi_det_index(a.ctypes.data_as(ctypes.c_void_p), b.ctypes.data_as(ctypes.c_void_p)))


def iscsi_diagonal(diag):
    return _check(load().iscsi_diagonal(_dev(diag)))


def iscsi_set_option(key, value):
    return _check(load().iscsi_set_option(key.encode(), float(value)))


def iscsi_stats():
    import json
    buf = ctypes.create_string_buffer(65536)
    _check(load().iscsi_stats(buf, len(buf)))
    return json.loads(buf.value.decode())


def iscsi_updates_per_sigma():
    return float(load().iscsi_updates_per_sigma())


def iscsi_last_error():
    m = load().iscsi_last_error()
    return m.decode() if m else ""


def iscsi_finalize():
    load().iscsi_finalize()


def iscsi_ctx_current():
    return int(load().iscsi_ctx_current())


def iscsi_ctx_use(handle):
    return _check(load().iscsi_ctx_use(int(handle)))


def iscsi_ctx_destroy(handle):
    return _check(load().iscsi_ctx_destroy(int(handle)))
