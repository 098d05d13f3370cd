"""ctypes binding of libctm (include/ctm.h): the same names, argument
marshalling only.  Every computation runs in the CUDA library; if the
library is missing this module raises at import.

Host arrays are numpy float64 arrays; device arrays are torch CUDA tensors
(float64, contiguous), passed by pointer.  Streams are torch.cuda.Stream
objects or None.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libctm.so not found at {LIB_PATH}: run __graft_entry__.build() "
                      "(nvcc, sm_103a) first; there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)

c_int, c_double, c_size_t, c_void_p, c_char_p = (ctypes.c_int, ctypes.c_double, ctypes.c_size_t,
                                                 ctypes.c_void_p, ctypes.c_char_p)
c_dp = ctypes.POINTER(ctypes.c_double)
c_ip = ctypes.POINTER(ctypes.c_int)

CTM_OK, CTM_NOT_CONVERGED = 0, 1
CTM_ERR_ARG, CTM_ERR_OOM, CTM_ERR_CUDA, CTM_ERR_NONFINITE, CTM_ERR_TIMEOUT, CTM_ERR_STATE = -1, -2, -3, -4, -5, -6
CTM_FP64, CTM_SPLIT_BF16, CTM_3XTF32, CTM_OZAKI_INT8, CTM_OZAKI_BF16 = 0, 1, 2, 3, 4
ENV_INDEX = {"C1": 0, "T1": 1, "C2": 2, "T2": 3, "C3": 4, "T3": 5, "C4": 6, "T4": 7}


class ctm_options(ctypes.Structure):
    _fields_ = [("chi", c_int), ("max_sweeps", c_int), ("tol", c_double), ("precision", c_int),
                ("ozaki_slices", c_int), ("rsvd_oversample", c_int), ("rsvd_power_iters", c_int),
                ("sv_cutoff_rel", c_double), ("seed", ctypes.c_uint64), ("exact_svd_max_n", c_int),
                ("rsvd_warm_start", c_int), ("conv_measure", c_int), ("fp64_refine", c_int),
                ("batch_cuts", c_int)]


class ctm_profile_data(ctypes.Structure):
    _fields_ = [("ms", c_double * 8), ("flops", c_double * 8), ("bytes", c_double * 8),
                ("calls", ctypes.c_longlong * 8)]


PROFILE_CLASSES = ("gemm", "permute", "qr", "svd", "split")


def _sig(name, res, *args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_sig("ctm_default_options", c_int, ctypes.POINTER(ctm_options))
_sig("ctm_footprint_bytes", c_int, c_int, c_int, ctypes.POINTER(ctm_options), ctypes.POINTER(c_size_t))
_sig("ctm_create", c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(ctm_options), c_void_p,
     ctypes.POINTER(c_void_p))
_sig("ctm_destroy", c_int, c_void_p)
_sig("ctm_set_tensor", c_int, c_void_p, c_int, c_void_p, c_int)
_sig("ctm_set_env", c_int, c_void_p, c_int, c_int, c_void_p, c_int)
_sig("ctm_get_env", c_int, c_void_p, c_int, c_int, c_void_p, c_int)
_sig("ctm_sweep", c_int, c_void_p, c_int)
_sig("ctm_sweep_async", c_int, c_void_p, c_int)
_sig("ctm_sync", c_int, c_void_p)
_sig("ctm_batch_sweep", c_int, ctypes.POINTER(c_void_p), c_int, c_int)
_sig("ctm_spectrum_delta", c_int, c_void_p, c_dp)
_sig("ctm_loop_delta", c_int, c_void_p, c_dp)
_sig("ctm_set_precision", c_int, c_void_p, c_int)
_sig("ctm_run", c_int, c_void_p, c_ip, c_dp)
_sig("ctm_corner_spectra", c_int, c_void_p, c_dp)
_sig("ctm_rdm1", c_int, c_void_p, c_int, c_dp)
_sig("ctm_rdm2", c_int, c_void_p, c_int, c_int, c_int, c_dp)
_sig("ctm_measure1", c_int, c_void_p, c_int, c_dp, c_dp)
_sig("ctm_measure2", c_int, c_void_p, c_int, c_int, c_int, c_dp, c_dp)
_sig("ctm_op_from_elements", c_int, c_int, c_int, c_int, c_ip, c_dp, c_dp)
_sig("ctm_last_error", c_char_p, c_void_p)
_sig("ctm_status_string", c_char_p, c_int)
_sig("ctm_dgemm", c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_void_p, c_int,
     c_double, c_void_p, c_int, c_void_p)
_sig("ctm_permute", c_int, c_void_p, c_void_p, c_int, c_ip, c_ip, c_void_p)
_sig("ctm_qr_workspace_bytes", c_size_t, c_int, c_int)
_sig("ctm_qr", c_int, c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p)
_sig("ctm_svd_workspace_bytes", c_size_t, c_int)
_sig("ctm_svd", c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p)

_sig("ctm_gemm_ozaki_workspace_bytes", c_size_t, c_int, c_int, c_int, c_int)
_sig("ctm_gemm_ozaki", c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_void_p, c_int,
     c_double, c_void_p, c_int, c_int, c_void_p, c_void_p)
_sig("ctm_svd_noalloc", c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p)
_sig("ctm_create_in", c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(ctm_options), c_void_p, c_void_p, c_size_t,
     c_void_p)
_sig("ctm_pool_create", c_int, c_size_t, c_size_t, ctypes.POINTER(c_void_p))
_sig("ctm_pool_alloc", c_int, c_void_p, c_size_t, ctypes.POINTER(c_size_t))
_sig("ctm_pool_free", c_int, c_void_p, c_size_t, c_size_t)
_sig("ctm_pool_stats", c_int, c_void_p, ctypes.POINTER(c_size_t), ctypes.POINTER(c_size_t), ctypes.POINTER(c_size_t))
_sig("ctm_pool_destroy", c_int, c_void_p)
_sig("ctm_correlation", c_int, c_void_p, c_void_p, c_void_p, c_int, c_void_p)
_sig("ctm_transfer_spectrum", c_int, c_void_p, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p,
     ctypes.POINTER(c_int), ctypes.POINTER(c_double))
_sig("ctm_small_eig", c_int, c_void_p, c_int, c_int, c_double, c_void_p, c_void_p, c_void_p)
_sig("ctm_gemm_split_workspace_bytes", c_size_t, c_int, c_int, c_int, c_int)
_sig("ctm_gemm_split", c_int, c_int, c_int, c_int, c_int, c_int, c_int, c_double, c_void_p, c_int, c_void_p, c_int,
     c_double, c_void_p, c_int, c_void_p, c_void_p)
_sig("ctm_log_norm_per_site", c_int, c_void_p, c_dp)
_sig("ctm_init_env_random", c_int, c_void_p, ctypes.c_uint64)
_sig("ctm_wait_probe", c_int, ctypes.c_longlong, c_int, c_void_p, c_void_p)
_sig("ctm_fp64_peak", c_int, c_dp)
_sig("ctm_profile_enable", c_int, c_void_p, c_int)
_sig("ctm_profile_read", c_int, c_void_p, ctypes.POINTER(ctm_profile_data), c_int)
_sig("ctm_kernel_launches", ctypes.c_longlong)
_sig("ctm_profile_report", c_int, c_void_p, c_char_p, c_size_t, c_int)

EXPORTED = [n for n in dir(_lib) if n.startswith("ctm_")]


class CtmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.ctm_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def _check(st, h=None):
    if st < 0:
        msg = _lib.ctm_last_error(h).decode(errors="replace")
        raise CtmError(st, msg)
    return st


def _dp(a):
    return a.ctypes.data_as(c_dp)


def _host(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t):
    assert t.is_cuda and t.dtype.__str__() == "torch.float64" and t.is_contiguous(), "float64 CUDA contiguous"
    return ctypes.c_void_p(t.data_ptr())


# ---------------------------------------------------------------------------
# handle-level calls
# ---------------------------------------------------------------------------
def ctm_default_options(**kw) -> ctm_options:
    o = ctm_options()
    _check(_lib.ctm_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def ctm_footprint_bytes(d, D, opt: ctm_options) -> int:
    b = c_size_t()
    _check(_lib.ctm_footprint_bytes(d, D, ctypes.byref(opt), ctypes.byref(b)))
    return b.value


def ctm_create(d, D, opt: ctm_options, stream=None, Lx=2, Ly=2):
    h = c_void_p()
    _check(_lib.ctm_create(Lx, Ly, d, D, ctypes.byref(opt), _stream_ptr(stream), ctypes.byref(h)), None)
    return h


def ctm_create_in(d, D, opt: ctm_options, arena_ptr, arena_bytes, stream=None, Lx=2, Ly=2):
    """ctm_create with every buffer carved from [arena_ptr, arena_ptr + arena_bytes)."""
    h = c_void_p()
    _check(_lib.ctm_create_in(Lx, Ly, d, D, ctypes.byref(opt), _stream_ptr(stream), ctypes.c_void_p(arena_ptr),
                              c_size_t(arena_bytes), ctypes.byref(h)), None)
    return h


def ctm_destroy(h):
    _check(_lib.ctm_destroy(h))


def ctm_set_tensor(h, site, A):
    if hasattr(A, "is_cuda"):
        _check(_lib.ctm_set_tensor(h, site, _dev_ptr(A), 1), h)
    else:
        A = _host(A)
        _check(_lib.ctm_set_tensor(h, site, A.ctypes.data_as(c_void_p), 0), h)


def ctm_set_env(h, site, which, t):
    w = ENV_INDEX[which] if isinstance(which, str) else which
    if hasattr(t, "is_cuda"):
        _check(_lib.ctm_set_env(h, site, w, _dev_ptr(t), 1), h)
    else:
        t = _host(t)
        _check(_lib.ctm_set_env(h, site, w, t.ctypes.data_as(c_void_p), 0), h)


def ctm_get_env(h, site, which, shape):
    w = ENV_INDEX[which] if isinstance(which, str) else which
    out = np.empty(shape, dtype=np.float64)
    _check(_lib.ctm_get_env(h, site, w, out.ctypes.data_as(c_void_p), 0), h)
    return out


def ctm_sweep(h, n):
    _check(_lib.ctm_sweep(h, n), h)


def ctm_sweep_async(h, n):
    _check(_lib.ctm_sweep_async(h, n), h)


def ctm_sync(h):
    _check(_lib.ctm_sync(h), h)


def ctm_batch_sweep(hs, sweeps):
    arr = (c_void_p * len(hs))(*hs)
    st = _lib.ctm_batch_sweep(arr, len(hs), sweeps)
    if st < 0:
        raise CtmError(st, "batched sweep failed: " + "; ".join(
            _lib.ctm_last_error(h).decode(errors="replace") for h in hs))


def ctm_spectrum_delta(h):
    d = c_double()
    _check(_lib.ctm_spectrum_delta(h, ctypes.byref(d)), h)
    return d.value


def ctm_log_norm_per_site(h):
    v = c_double()
    _check(_lib.ctm_log_norm_per_site(h, ctypes.byref(v)), h)
    return v.value


def ctm_pool_create(nbytes, grain):
    p = c_void_p()
    _check(_lib.ctm_pool_create(nbytes, grain, ctypes.byref(p)))
    return p


def ctm_pool_alloc(pool, nbytes):
    """Offset of a block of at least nbytes, or None when no free block fits."""
    off = c_size_t()
    st = _lib.ctm_pool_alloc(pool, nbytes, ctypes.byref(off))
    if st == CTM_ERR_OOM:
        return None
    _check(st)
    return off.value


def ctm_pool_free(pool, offset, nbytes):
    _check(_lib.ctm_pool_free(pool, offset, nbytes))


def ctm_pool_stats(pool):
    """(bytes allocated, largest free block, number of free blocks)."""
    u, l, n = c_size_t(), c_size_t(), c_size_t()
    _check(_lib.ctm_pool_stats(pool, ctypes.byref(u), ctypes.byref(l), ctypes.byref(n)))
    return u.value, l.value, n.value


def ctm_pool_destroy(pool):
    _check(_lib.ctm_pool_destroy(pool))


def ctm_correlation(h, opA, opB, rmax):
    """C[dir, site, r] = <A(r0) B(r0 + r e_dir)>, dir 0: x, 1: y."""
    a, b = _host(opA), _host(opB)
    out = np.zeros((2, 4, rmax + 1))
    _check(_lib.ctm_correlation(h, _dp(a), _dp(b), rmax, _dp(out)), h)
    return out


def ctm_transfer_spectrum(h, direction, index, nev=4, block=None, max_iter=200, tol=1e-10):
    """(ratio lambda_i / lambda_0 [complex, nev], |lambda_i| [nev], e_i [nev],
    iterations, last change, status)."""
    block = block if block is not None else nev + 4
    out = np.zeros(4 * nev)
    it, ch = c_int(), c_double()
    st = _lib.ctm_transfer_spectrum(h, direction, index, nev, block, max_iter, tol, _dp(out), ctypes.byref(it),
                                    ctypes.byref(ch))
    if st not in (CTM_OK, CTM_NOT_CONVERGED):
        _check(st, h)
    ratio = out[:nev] + 1j * out[nev:2 * nev]
    return ratio, out[2 * nev:3 * nev], out[3 * nev:], it.value, ch.value, st


def ctm_small_eig(H, m, ldh, period, out, status, stream=None):
    _check(_lib.ctm_small_eig(_dev_ptr(H), m, ldh, period, _dev_ptr(out), ctypes.c_void_p(status.data_ptr()),
                              _stream_ptr(stream)))


def ctm_init_env_random(h, seed):
    _check(_lib.ctm_init_env_random(h, seed), h)


def ctm_wait_probe(limit_cycles, arrive, flag, stream=None):
    """Returns the status (CTM_OK or CTM_ERR_TIMEOUT); flag: a torch int32 CUDA tensor."""
    st = _lib.ctm_wait_probe(int(limit_cycles), int(arrive), ctypes.c_void_p(flag.data_ptr()), _stream_ptr(stream))
    if st not in (CTM_OK, CTM_ERR_TIMEOUT):
        _check(st)
    return st


def ctm_fp64_peak():
    v = c_double()
    _check(_lib.ctm_fp64_peak(ctypes.byref(v)))
    return v.value


def ctm_set_precision(h, precision):
    _check(_lib.ctm_set_precision(h, precision), h)


def ctm_loop_delta(h):
    d = c_double()
    _check(_lib.ctm_loop_delta(h, ctypes.byref(d)), h)
    return d.value


def ctm_run(h):
    n = c_int()
    dl = c_double()
    st = _check(_lib.ctm_run(h, ctypes.byref(n), ctypes.byref(dl)), h)
    return st, n.value, dl.value


def ctm_corner_spectra(h, chi):
    out = np.empty((4, 4, chi))
    _check(_lib.ctm_corner_spectra(h, _dp(out)), h)
    return out


def ctm_rdm1(h, site, d):
    out = np.empty((d, d))
    _check(_lib.ctm_rdm1(h, site, _dp(out)), h)
    return out


def ctm_rdm2(h, site, dx, dy, d):
    out = np.empty((d * d, d * d))
    _check(_lib.ctm_rdm2(h, site, dx, dy, _dp(out)), h)
    return out


def ctm_measure1(h, site, op):
    op = _host(op)
    v = c_double()
    _check(_lib.ctm_measure1(h, site, _dp(op), ctypes.byref(v)), h)
    return v.value


def ctm_measure2(h, site, dx, dy, op):
    op = _host(op)
    v = c_double()
    _check(_lib.ctm_measure2(h, site, dx, dy, _dp(op), ctypes.byref(v)), h)
    return v.value


def ctm_op_from_elements(d0, d1, lines):
    n = len(lines)
    idx = np.ascontiguousarray([[l[0], l[1], l[2], l[3]] for l in lines], dtype=np.int32).reshape(-1)
    re = np.ascontiguousarray([l[4] for l in lines], dtype=np.float64)
    for l in lines:
        if l[5] != 0.0:
            raise ValueError("real operators only")
    out = np.empty((d0 * d1, d0 * d1))
    _check(_lib.ctm_op_from_elements(d0, d1, n, idx.ctypes.data_as(c_ip), _dp(re), _dp(out)))
    return out


def ctm_profile_enable(h, on):
    _check(_lib.ctm_profile_enable(h, int(on)), h)


def ctm_profile_read(h, reset=False):
    p = ctm_profile_data()
    _check(_lib.ctm_profile_read(h, ctypes.byref(p), int(reset)), h)
    return {c: dict(ms=p.ms[i], flops=p.flops[i], bytes=p.bytes[i], calls=p.calls[i])
            for i, c in enumerate(PROFILE_CLASSES)}


def ctm_profile_report(h, reset=False):
    import json
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.ctm_profile_report(h, buf, len(buf), int(reset)), h)
    return json.loads(buf.value.decode())


def ctm_kernel_launches():
    return int(_lib.ctm_kernel_launches())


# ---------------------------------------------------------------------------
# kernel-level calls (torch CUDA tensors)
# ---------------------------------------------------------------------------
def ctm_dgemm(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, stream=None):
    _check(_lib.ctm_dgemm(int(transA), int(transB), M, N, K, alpha, _dev_ptr(A), lda, _dev_ptr(B), ldb,
                          beta, _dev_ptr(C), ldc, _stream_ptr(stream)))


def ctm_permute(src, dst, dims, perm, stream=None):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    p = np.ascontiguousarray(perm, dtype=np.int32)
    _check(_lib.ctm_permute(_dev_ptr(src), _dev_ptr(dst), len(dims), d.ctypes.data_as(c_ip),
                            p.ctypes.data_as(c_ip), _stream_ptr(stream)))


def ctm_qr_workspace_bytes(N, k):
    return _lib.ctm_qr_workspace_bytes(N, k)


def ctm_qr(Y, N, k, Q, R, ws, stream=None):
    _check(_lib.ctm_qr(_dev_ptr(Y), N, k, _dev_ptr(Q), _dev_ptr(R), ctypes.c_void_p(ws.data_ptr()),
                       _stream_ptr(stream)))


def ctm_svd_workspace_bytes(k):
    return _lib.ctm_svd_workspace_bytes(k)


def ctm_svd(G, k, U, S, V, ws, stream=None):
    _check(_lib.ctm_svd(_dev_ptr(G), k, _dev_ptr(U), _dev_ptr(S), _dev_ptr(V), ctypes.c_void_p(ws.data_ptr()),
                        _stream_ptr(stream)))


def ctm_gemm_ozaki_workspace_bytes(M, N, K, slices):
    return _lib.ctm_gemm_ozaki_workspace_bytes(M, N, K, slices)


def ctm_gemm_ozaki(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, slices, ws, stream=None):
    _check(_lib.ctm_gemm_ozaki(int(transA), int(transB), M, N, K, alpha, _dev_ptr(A), lda, _dev_ptr(B), ldb,
                               beta, _dev_ptr(C), ldc, slices, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)))


def ctm_gemm_split_workspace_bytes(precision, M, N, K):
    return _lib.ctm_gemm_split_workspace_bytes(precision, M, N, K)


def ctm_gemm_split(precision, transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, ws, stream=None):
    _check(_lib.ctm_gemm_split(precision, int(transA), int(transB), M, N, K, alpha, _dev_ptr(A), lda, _dev_ptr(B),
                               ldb, beta, _dev_ptr(C), ldc, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)))


def ctm_svd_noalloc(G, k, U, S, V, stream=None):
    """ctm_svd with the library's static scratch (k <= 256); allocates nothing."""
    _check(_lib.ctm_svd_noalloc(_dev_ptr(G), k, _dev_ptr(U), _dev_ptr(S), _dev_ptr(V), _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class CTMRG:
    """One 2x2-cell CTMRG instance on the current CUDA device."""

    def __init__(self, d, D, chi, stream=None, arena=None, **opts):
        """arena: optional (device pointer, bytes) the handle's buffers are
        carved from (ctm_create_in)."""
        self.d, self.D, self.chi = d, D, chi
        self.stream = stream
        self.opt = ctm_default_options(chi=chi, **opts)
        if arena is None:
            self.h = ctm_create(d, D, self.opt, stream)
        else:
            self.h = ctm_create_in(d, D, self.opt, arena[0], arena[1], stream)

    def close(self):
        if self.h:
            ctm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensors(self, As):
        for i, A in enumerate(As):
            ctm_set_tensor(self.h, i, A)

    def set_envs(self, envs):
        for i, e in enumerate(envs):
            for name, t in e.items():
                ctm_set_env(self.h, i, name, t)

    def get_envs(self):
        D, chi = self.D, self.chi
        out = []
        for i in range(4):
            e = {}
            for name, w in ENV_INDEX.items():
                e[name] = ctm_get_env(self.h, i, w, (chi, chi) if w % 2 == 0 else (chi, D, D, chi))
            out.append(e)
        return out

    def sweep(self, n):
        ctm_sweep(self.h, n)

    def sweep_async(self, n):
        ctm_sweep_async(self.h, n)

    def sync(self):
        ctm_sync(self.h)

    def spectrum_delta(self):
        return ctm_spectrum_delta(self.h)

    def loop_delta(self):
        return ctm_loop_delta(self.h)

    def run(self):
        return ctm_run(self.h)

    def rdm1(self, site):
        return ctm_rdm1(self.h, site, self.d)

    def rdm2(self, site, dx, dy):
        return ctm_rdm2(self.h, site, dx, dy, self.d)

    def measure1(self, site, op):
        return ctm_measure1(self.h, site, op)

    def measure2(self, site, dx, dy, op):
        return ctm_measure2(self.h, site, dx, dy, op)

    def corner_spectra(self):
        return ctm_corner_spectra(self.h, self.chi)

    def log_norm_per_site(self):
        return ctm_log_norm_per_site(self.h)

    def correlation(self, opA, opB, rmax):
        return ctm_correlation(self.h, opA, opB, rmax)

    def transfer_spectrum(self, direction, index, nev=4, block=None, max_iter=200, tol=1e-10):
        return ctm_transfer_spectrum(self.h, direction, index, nev, block, max_iter, tol)

    def init_env_random(self, seed):
        ctm_init_env_random(self.h, seed)
