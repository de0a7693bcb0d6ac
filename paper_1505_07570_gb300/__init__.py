"""Python binding of librmc (include/rmc.h): argument marshalling only.

Every function takes and returns torch tensors on the current CUDA device and calls the C entry point of the
same name; all arithmetic runs in the library's CUDA kernels.  There is no CPU path: importing this package
fails if the compiled library is missing (build it with ``python -m paper_1505_07570_gb300.build`` or
``__graft_entry__.build()``).

Calls are asynchronous on the current torch stream; ``rmc_sync()`` waits and raises ``RmcError`` for a
device-detected error (non-positive pivot, iteration cap).
"""
import ctypes
import os

from .build import LIB as _LIB_PATH

RMC_OK, RMC_EINVAL, RMC_EALIGN, RMC_ENOMEM, RMC_ENUMERIC, RMC_ETIMEOUT, RMC_ECUDA, RMC_PENDING = range(8)
RMC_GAUSSIAN, RMC_SRHT, RMC_COUNTSKETCH = 0, 1, 2
RMC_FP32, RMC_TF32, RMC_BF16, RMC_TF32X3 = 0, 1, 2, 3

KIND = {"gaussian": RMC_GAUSSIAN, "srht": RMC_SRHT, "countsketch": RMC_COUNTSKETCH}
PREC = {"fp32": RMC_FP32, "tf32": RMC_TF32, "bf16": RMC_BF16, "tf32x3": RMC_TF32X3}

if not os.path.exists(_LIB_PATH):
    raise ImportError("librmc.so is not built (expected at %s); run __graft_entry__.build()" % _LIB_PATH)

lib = ctypes.CDLL(_LIB_PATH)

_p, _i64, _u64, _u32, _int, _sz = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.c_size_t)
_SIGS = {
    "rmc_create": [ctypes.POINTER(_p), _p, _sz],
    "rmc_destroy": [_p],
    "rmc_set_stream": [_p, _p],
    "rmc_sync": [_p],
    "rmc_workspace_bytes": [_p, ctypes.POINTER(_sz)],
    "rmc_set_option": [_p, _int, _int],
    "rmc_get_option": [_p, _int, ctypes.POINTER(_int)],
    "rmc_sketch": [_p, _p, _i64, _i64, _i64, _i64, _int, _u64, _int, _p, _i64],
    "rmc_lsr_sketch": [_p, _p, _i64, _i64, _i64, _p, _i64, _int, _u64, _int, _p],
    "rmc_rsvd": [_p, _p, _i64, _i64, _i64, _int, _int, _int, _u64, _int, _p, _i64, _p, _p, _i64],
    "rmc_philox": [_p, _u64, _u32, _u32, _u64, _i64, _p],
    "rmc_gaussian_matrix": [_p, _u64, _u32, _i64, _i64, _p, _i64],
    "rmc_countsketch_hash": [_p, _u64, _u32, _i64, _i64, _p, _p],
    "rmc_srht_sample": [_p, _u64, _u32, _i64, _i64, _p],
    "rmc_cholqr2": [_p, _p, _i64, _i64, _i64, _p],
    "rmc_svd_wide": [_p, _p, _i64, _i64, _i64, _p, _p, _p, _i64],
    "rmc_matmul_an": [_p, _p, _i64, _i64, _i64, _p, _i64, _i64, _int, _p, _i64],
    "rmc_matmul_at": [_p, _p, _i64, _i64, _i64, _p, _i64, _i64, _int, _p, _i64],
}
_SIGS.update({
    "rmc_profile_begin": [_p],
    "rmc_profile_read": [_p, _int, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)],
    "rmc_profile_end": [_p],
    "rmc_profile_reference": [_p],
    "rmc_profile_spans": [_p, _int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), _int,
                          ctypes.POINTER(_int)],
    "rmc_launch_counter": [ctypes.POINTER(_u64)],
    "rmc_debug_wait_timeout": [_p, _u64],
    "rmc_gaussian_draw_floor": [_p, _i64, _i64, _u64, _p],
    "rmc_countsketch_noalloc": [_p, _p, _i64, _i64, _i64, _i64, _u64, _p, _i64],
    "rmc_lsr_precise": [_p, _p, _i64, _i64, _i64, _p, _i64, _int, _u64, _int, ctypes.c_double, _int,
                        ctypes.c_double, _p, _p],
    "rmc_rsvd_fast": [_p, _p, _i64, _i64, _i64, _int, _int, _int, _int, _u64, _int, _p, _i64, _p, _p, _i64],
    "rmc_countsketch_columns": [_p, _p, _i64, _i64, _i64, _i64, _u64, _u32, _p, _i64],
    "rmc_nystrom": [_p, _p, _i64, _i64, _i64, ctypes.c_double, _i64, _int, _u64, _p, _i64, _p, _p],
    "rmc_rbf": [_p, _p, _i64, _i64, _p, _i64, _i64, _i64, ctypes.c_double, _p, _i64],
    "rmc_block_lanczos": [_p, _p, _i64, _i64, _i64, _int, _int, _int, _u64, _int, _p, _i64, _p, _p, _i64],
})
RMC_ESCRATCH = 8
RMC_NOALLOC_SCRATCH_BYTES = 32 << 20
(K_COUNTSKETCH, K_SRHT, K_SRHT_REDUCE, K_GAUSSIAN, K_MATMUL_AN, K_MATMUL_AT, K_GRAM, K_SMALL, K_BATCH,
 K_LSR_PASS, K_RBF) = range(11)
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
lib.rmc_status_string.argtypes = [ctypes.c_int]
lib.rmc_status_string.restype = ctypes.c_char_p


class RmcError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, lib.rmc_status_string(status).decode(), status))


def _check(status, where):
    if status != RMC_OK:
        raise RmcError(status, where)


class Context:
    """An rmc_ctx bound to one device and one CUDA stream (each has its own workspace, so calls on different
    streams may run concurrently)."""

    def __init__(self, budget_bytes=0):
        import torch
        self.device = torch.cuda.current_device()
        self.handle = _p()
        stream = torch.cuda.current_stream().cuda_stream
        _check(lib.rmc_create(ctypes.byref(self.handle), _p(stream), _sz(budget_bytes)), "rmc_create")
        self.stream = stream

    def bind(self):
        return self.handle

    def close(self):
        if self.handle:
            lib.rmc_destroy(self.handle)
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_contexts = {}


def context():
    """The context of the current device and current torch stream (created on first use)."""
    import torch
    key = (torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    if key not in _contexts:
        _contexts[key] = Context()
    return _contexts[key]


def _device_contexts():
    import torch
    dev = torch.cuda.current_device()
    return [c for (d, _), c in _contexts.items() if d == dev]


def _ptr(t):
    return _p(t.data_ptr())


def _mat(t, name):
    """A CUDA float32 matrix with unit column stride on the current device (the library launches on the
    current device and the current torch stream)."""
    import torch
    if not (t.is_cuda and t.dtype == torch.float32 and t.dim() == 2 and t.stride(1) == 1):
        raise ValueError("%s must be a CUDA float32 matrix with unit column stride" % name)
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on %s but the current device is cuda:%d" % (name, t.device,
                                                                          torch.cuda.current_device()))
    if t.shape[0] > 1 and t.stride(0) < t.shape[1]:
        raise ValueError("%s rows overlap (row stride %d < %d columns)" % (name, t.stride(0), t.shape[1]))
    return t


def _out(t, shape, dtype, like, name):
    """A caller-supplied output: the exact shape and dtype, on ``like``'s device, unit column stride and
    row-major rows that do not overlap, so that the kernels never write past its allocation."""
    if not (t.is_cuda and t.dtype == dtype and tuple(t.shape) == tuple(shape) and t.device == like.device):
        raise ValueError("%s must be a %s CUDA tensor of shape %s on %s (got %s %s on %s)"
                         % (name, dtype, tuple(shape), like.device, t.dtype, tuple(t.shape), t.device))
    if len(shape) == 2:
        if t.stride(1) != 1 or (shape[0] > 1 and t.stride(0) < shape[1]):
            raise ValueError("%s must be row-major with unit column stride" % name)
    elif not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t


def _kind(kind):
    return KIND[kind] if isinstance(kind, str) else int(kind)


def _prec(prec):
    return PREC[prec] if isinstance(prec, str) else int(prec)


def rmc_sync():
    """Wait for the current stream's context; raise RmcError for a device-detected error."""
    _check(lib.rmc_sync(context().bind()), "rmc_sync")


def rmc_sync_all():
    """rmc_sync on every context of the current device."""
    for c in _device_contexts():
        _check(lib.rmc_sync(c.handle), "rmc_sync")


RMC_OPT_SMALL_FP64 = 1


def rmc_set_option(option, value):
    """Set a context option of the current stream's context (RMC_OPT_SMALL_FP64: 1 runs the small
    factorizations in FP64)."""
    _check(lib.rmc_set_option(context().bind(), option, value), "rmc_set_option")


def rmc_get_option(option):
    out = _int()
    _check(lib.rmc_get_option(context().bind(), option, ctypes.byref(out)), "rmc_get_option")
    return out.value


def rmc_workspace_bytes():
    out = _sz()
    _check(lib.rmc_workspace_bytes(context().bind(), ctypes.byref(out)), "rmc_workspace_bytes")
    return out.value


def rmc_sketch(A, s, kind, seed, prec="fp32", out=None):
    """C = S^T A (s x n)."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    C = (_out(out, (s, n), torch.float32, A, "out") if out is not None
         else torch.empty(s, n, device=A.device, dtype=torch.float32))
    _check(lib.rmc_sketch(context().bind(), _ptr(A), m, n, A.stride(0), s, _kind(kind), seed, _prec(prec),
                          _ptr(C), C.stride(0)), "rmc_sketch")
    return C


def rmc_lsr_sketch(A, b, s, kind, seed, prec="fp32", out=None):
    """x = argmin ||S^T A x - S^T b|| (FP64, n entries)."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    if not (b.is_cuda and b.dtype == torch.float32 and b.is_contiguous() and b.numel() == m):
        raise ValueError("b must be a contiguous CUDA float32 vector of length m")
    if b.device != A.device:
        raise ValueError("b must be on the device of A")
    x = (_out(out, (n,), torch.float64, A, "out") if out is not None
         else torch.empty(n, device=A.device, dtype=torch.float64))
    _check(lib.rmc_lsr_sketch(context().bind(), _ptr(A), m, n, A.stride(0), _ptr(b), s, _kind(kind), seed,
                              _prec(prec), _ptr(x)), "rmc_lsr_sketch")
    return x


def rmc_rsvd(A, k, p, q, seed, prec="fp32"):
    """U (m x k), sigma (k), V (n x k) of the randomized k-SVD with l = k + p and q power iterations."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    U = torch.empty(m, k, device=A.device, dtype=torch.float32)
    sigma = torch.empty(k, device=A.device, dtype=torch.float32)
    V = torch.empty(n, k, device=A.device, dtype=torch.float32)
    _check(lib.rmc_rsvd(context().bind(), _ptr(A), m, n, A.stride(0), k, p, q, seed, _prec(prec), _ptr(U),
                        U.stride(0), _ptr(sigma), _ptr(V), V.stride(0)), "rmc_rsvd")
    return U, sigma, V


def rmc_lsr_precise(A, b, s, kind, seed, prec="fp32", theta=0.0, max_iters=30, tol=1e-15, out=None,
                    want_iters=False):
    """Machine-precision least squares (Algorithm 4.1): x (FP64, n entries); with want_iters also the number
    of preconditioned steps taken (a device int tensor)."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    if not (b.is_cuda and b.dtype == torch.float32 and b.is_contiguous() and b.numel() == m
            and b.device == A.device):
        raise ValueError("b must be a contiguous CUDA float32 vector of length m on the device of A")
    x = (_out(out, (n,), torch.float64, A, "out") if out is not None
         else torch.empty(n, device=A.device, dtype=torch.float64))
    it = torch.zeros(1, device=A.device, dtype=torch.int32) if want_iters else None
    _check(lib.rmc_lsr_precise(context().bind(), _ptr(A), m, n, A.stride(0), _ptr(b), s, _kind(kind), seed,
                               _prec(prec), float(theta), int(max_iters), float(tol), _ptr(x),
                               _ptr(it) if want_iters else None), "rmc_lsr_precise")
    return (x, it) if want_iters else x


def rmc_block_lanczos(A, k, s, q, seed, prec="fp32"):
    """U (m x k), sigma (k), V (n x k) of the block Lanczos k-SVD (Algorithm 5.1), block size s, q blocks."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    U = torch.empty(m, k, device=A.device, dtype=torch.float32)
    sigma = torch.empty(k, device=A.device, dtype=torch.float32)
    V = torch.empty(n, k, device=A.device, dtype=torch.float32)
    _check(lib.rmc_block_lanczos(context().bind(), _ptr(A), m, n, A.stride(0), k, s, q, seed, _prec(prec),
                                 _ptr(U), U.stride(0), _ptr(sigma), _ptr(V), V.stride(0)), "rmc_block_lanczos")
    return U, sigma, V


def rmc_rsvd_fast(A, k, s, p_cs, p, seed, prec="fp32"):
    """U (m x k), sigma (k), V (n x k) of the faster randomized k-SVD (Algorithm 5.3)."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    U = torch.empty(m, k, device=A.device, dtype=torch.float32)
    sigma = torch.empty(k, device=A.device, dtype=torch.float32)
    V = torch.empty(n, k, device=A.device, dtype=torch.float32)
    _check(lib.rmc_rsvd_fast(context().bind(), _ptr(A), m, n, A.stride(0), k, s, p_cs, p, seed, _prec(prec),
                             _ptr(U), U.stride(0), _ptr(sigma), _ptr(V), V.stride(0)), "rmc_rsvd_fast")
    return U, sigma, V


def rmc_countsketch_columns(A, s, seed, instance=0):
    """C = A S with S an n x s count sketch over the columns (m x s)."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    C = torch.empty(m, s, device=A.device, dtype=torch.float32)
    _check(lib.rmc_countsketch_columns(context().bind(), _ptr(A), m, n, A.stride(0), s, seed, instance, _ptr(C),
                                       C.stride(0)), "rmc_countsketch_columns")
    return C


def rmc_nystrom(X, sigma, s, seed, k=0):
    """L (n x k), the eigenvalues lam (k) of the landmark block and the landmark indices (s) of the Nystrom
    method (Sec. 6.4) on the RBF kernel of width sigma; k = 0 takes ceil(0.8 s)."""
    import math
    import torch
    _mat(X, "X")
    n, d = X.shape
    kk = k if k else int(math.ceil(0.8 * s))
    L = torch.empty(n, kk, device=X.device, dtype=torch.float32)
    lam = torch.empty(kk, device=X.device, dtype=torch.float32)
    idx = torch.empty(s, device=X.device, dtype=torch.int64)
    _check(lib.rmc_nystrom(context().bind(), _ptr(X), n, d, X.stride(0), float(sigma), s, kk, seed, _ptr(L),
                           L.stride(0), _ptr(lam), _ptr(idx)), "rmc_nystrom")
    return L, lam, idx


def rmc_rbf(X, Y, sigma):
    """K_ij = exp(-||x_i - y_j||^2 / (2 sigma^2)) (n1 x n2)."""
    import torch
    _mat(X, "X")
    _mat(Y, "Y")
    K = torch.empty(X.shape[0], Y.shape[0], device=X.device, dtype=torch.float32)
    _check(lib.rmc_rbf(context().bind(), _ptr(X), X.shape[0], X.stride(0), _ptr(Y), Y.shape[0], Y.stride(0),
                       X.shape[1], float(sigma), _ptr(K), K.stride(0)), "rmc_rbf")
    return K


def rmc_philox(seed, stream, instance, first, count):
    """Philox4x32-10 words: int64 tensor (count, 4) holding the unsigned 32-bit words."""
    import torch
    out = torch.empty(count, 4, device="cuda", dtype=torch.int32)
    _check(lib.rmc_philox(context().bind(), seed, stream, instance, first, count, _ptr(out)), "rmc_philox")
    return out.to(torch.int64) & 0xFFFFFFFF


def rmc_gaussian_matrix(seed, instance, rows, cols):
    import torch
    out = torch.empty(rows, cols, device="cuda", dtype=torch.float32)
    _check(lib.rmc_gaussian_matrix(context().bind(), seed, instance, rows, cols, _ptr(out), cols),
           "rmc_gaussian_matrix")
    return out


def rmc_countsketch_hash(seed, instance, m, s):
    import torch
    bucket = torch.empty(m, device="cuda", dtype=torch.int32)
    sign = torch.empty(m, device="cuda", dtype=torch.float32)
    _check(lib.rmc_countsketch_hash(context().bind(), seed, instance, m, s, _ptr(bucket), _ptr(sign)),
           "rmc_countsketch_hash")
    return bucket, sign


def rmc_srht_sample(seed, instance, N, s):
    import torch
    idx = torch.empty(s, device="cuda", dtype=torch.int64)
    _check(lib.rmc_srht_sample(context().bind(), seed, instance, N, s, _ptr(idx)), "rmc_srht_sample")
    return idx


def rmc_cholqr2(Y, want_r=True):
    """In place: Y <- Q; returns R (l x l FP64) when want_r."""
    import torch
    _mat(Y, "Y")
    m, l = Y.shape
    R = torch.empty(l, l, device=Y.device, dtype=torch.float64) if want_r else None
    _check(lib.rmc_cholqr2(context().bind(), _ptr(Y), m, l, Y.stride(0), _ptr(R) if want_r else None),
           "rmc_cholqr2")
    return R


def rmc_svd_wide(B):
    """B (l x n, l <= n) = Ub diag(sigma) Vb^T."""
    import torch
    _mat(B, "B")
    l, n = B.shape
    Ub = torch.empty(l, l, device=B.device, dtype=torch.float32)
    sigma = torch.empty(l, device=B.device, dtype=torch.float32)
    Vb = torch.empty(n, l, device=B.device, dtype=torch.float32)
    _check(lib.rmc_svd_wide(context().bind(), _ptr(B), l, n, B.stride(0), _ptr(Ub), _ptr(sigma), _ptr(Vb),
                            Vb.stride(0)), "rmc_svd_wide")
    return Ub, sigma, Vb


def rmc_matmul_an(A, X, prec="fp32"):
    """Y = A X."""
    import torch
    _mat(A, "A")
    _mat(X, "X")
    m, n = A.shape
    l = X.shape[1]
    Y = torch.empty(m, l, device=A.device, dtype=torch.float32)
    _check(lib.rmc_matmul_an(context().bind(), _ptr(A), m, n, A.stride(0), _ptr(X), l, X.stride(0), _prec(prec),
                             _ptr(Y), Y.stride(0)), "rmc_matmul_an")
    return Y


def rmc_matmul_at(A, X, prec="fp32"):
    """W = X^T A."""
    import torch
    _mat(A, "A")
    _mat(X, "X")
    m, n = A.shape
    l = X.shape[1]
    W = torch.empty(l, n, device=A.device, dtype=torch.float32)
    _check(lib.rmc_matmul_at(context().bind(), _ptr(A), m, n, A.stride(0), _ptr(X), l, X.stride(0), _prec(prec),
                             _ptr(W), W.stride(0)), "rmc_matmul_at")
    return W


def rmc_profile_begin():
    """Start the event hooks on every context of the current device."""
    for c in _device_contexts():
        _check(lib.rmc_profile_begin(c.handle), "rmc_profile_begin")


def rmc_profile_read(tag):
    """(launches, total device milliseconds) of one kernel tag since rmc_profile_begin, summed over the
    contexts of the current device."""
    total_n, total_ms = 0, 0.0
    for c in _device_contexts():
        n, ms = _i64(), ctypes.c_double()
        _check(lib.rmc_profile_read(c.handle, tag, ctypes.byref(n), ctypes.byref(ms)), "rmc_profile_read")
        total_n += n.value
        total_ms += ms.value
    return total_n, total_ms


def rmc_profile_reference():
    """Record the process-wide reference event of rmc_profile_spans on the current stream's context."""
    _check(lib.rmc_profile_reference(context().bind()), "rmc_profile_reference")


def rmc_profile_spans(tag):
    """[(start_ms, stop_ms)] of every launch of one kernel tag since rmc_profile_begin that completed after the
    reference, relative to the reference, over the contexts of the current device."""
    out = []
    cap = 4096
    t0 = (ctypes.c_double * cap)()
    t1 = (ctypes.c_double * cap)()
    for c in _device_contexts():
        n = ctypes.c_int()
        _check(lib.rmc_profile_spans(c.handle, tag, t0, t1, cap, ctypes.byref(n)), "rmc_profile_spans")
        out.extend((t0[i], t1[i]) for i in range(n.value))
    return out


def rmc_profile_end():
    for c in _device_contexts():
        _check(lib.rmc_profile_end(c.handle), "rmc_profile_end")


def rmc_gaussian_draw_floor(m, s, seed):
    """Draw the m x s normals of the Gaussian sketch's operator without the product (the drawing bound of the
    tensor-core sketch), on the current torch stream; returns a 1-element FP64 CUDA tensor with their sum."""
    import torch
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    _check(lib.rmc_gaussian_draw_floor(context().bind(), int(m), int(s), int(seed), out.data_ptr()),
           "rmc_gaussian_draw_floor")
    return out


def rmc_launch_counter():
    out = _u64()
    _check(lib.rmc_launch_counter(ctypes.byref(out)), "rmc_launch_counter")
    return out.value


def rmc_countsketch_noalloc(A, s, seed, out=None):
    """Count sketch through the entry point that allocates no device memory (for callers that cannot
    allocate at call time); enqueued on the current torch stream.  ``out`` (s x n) must be supplied by the
    caller to keep the call allocation-free; a new tensor is made when it is None."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    C = (_out(out, (s, n), torch.float32, A, "out") if out is not None
         else torch.empty(s, n, device=A.device, dtype=torch.float32))
    _check(lib.rmc_countsketch_noalloc(_p(torch.cuda.current_stream().cuda_stream), _ptr(A), m, n, A.stride(0),
                                       s, seed, _ptr(C), C.stride(0)), "rmc_countsketch_noalloc")
    return C


RMC_REQ_LSR, RMC_REQ_RSVD = 0, 1


class rmc_request(ctypes.Structure):
    """Mirror of the C struct rmc_request (include/rmc.h)."""
    _fields_ = [("kind", _int), ("k", _int), ("p", _int), ("q", _int),
                ("m", _i64), ("n", _i64), ("lda", _i64), ("s", _i64),
                ("seed", _u64),
                ("A", _p), ("b", _p), ("x", _p), ("U", _p), ("sigma", _p), ("V", _p)]


lib.rmc_batch_run.argtypes = [_p, ctypes.POINTER(rmc_request), _int]
lib.rmc_batch_run.restype = ctypes.c_int


def lsr_request(A, b, s, seed):
    """A batch request for count-sketch least squares; returns (request, x) with x the FP64 output tensor."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    if not (b.is_cuda and b.dtype == torch.float32 and b.is_contiguous() and b.numel() == m):
        raise ValueError("b must be a contiguous CUDA float32 vector of length m")
    x = torch.empty(n, device=A.device, dtype=torch.float64)
    r = rmc_request(kind=RMC_REQ_LSR, k=0, p=0, q=0, m=m, n=n, lda=A.stride(0), s=s, seed=seed,
                    A=A.data_ptr(), b=b.data_ptr(), x=x.data_ptr())
    return r, x


def rsvd_request(A, k, p, q, seed):
    """A batch request for the randomized k-SVD; returns (request, (U, sigma, V)) with the output tensors."""
    import torch
    _mat(A, "A")
    m, n = A.shape
    U = torch.empty(m, k, device=A.device, dtype=torch.float32)
    sigma = torch.empty(k, device=A.device, dtype=torch.float32)
    V = torch.empty(n, k, device=A.device, dtype=torch.float32)
    r = rmc_request(kind=RMC_REQ_RSVD, k=k, p=p, q=q, m=m, n=n, lda=A.stride(0), s=0, seed=seed,
                    A=A.data_ptr(), U=U.data_ptr(), sigma=sigma.data_ptr(), V=V.data_ptr())
    return r, (U, sigma, V)


def rmc_batch_run(requests):
    """Run a list of rmc_request in one persistent launch on the current stream (outputs as given)."""
    arr = (rmc_request * len(requests))(*requests)
    _check(lib.rmc_batch_run(context().bind(), arr, len(requests)), "rmc_batch_run")


RMC_BATCH_TILE_CLASSES = 16
lib.rmc_batch_autotune.argtypes = [_p, ctypes.POINTER(rmc_request), _int, _int]
lib.rmc_batch_autotune.restype = ctypes.c_int
lib.rmc_batch_get_tiles.argtypes = [_p, ctypes.POINTER(_int), _int]
lib.rmc_batch_get_tiles.restype = ctypes.c_int
lib.rmc_batch_set_tiles.argtypes = [_p, ctypes.POINTER(_int), _int]
lib.rmc_batch_set_tiles.restype = ctypes.c_int


def rmc_batch_autotune(requests, reps=3):
    """Tune the batched kernel's row tiles on these problems (they are run); returns the 16-entry table."""
    arr = (rmc_request * len(requests))(*requests)
    _check(lib.rmc_batch_autotune(context().bind(), arr, len(requests), reps), "rmc_batch_autotune")
    return rmc_batch_get_tiles()


def rmc_batch_get_tiles():
    t = (_int * RMC_BATCH_TILE_CLASSES)()
    _check(lib.rmc_batch_get_tiles(context().bind(), t, RMC_BATCH_TILE_CLASSES), "rmc_batch_get_tiles")
    return list(t)


def rmc_batch_set_tiles(table):
    t = (_int * RMC_BATCH_TILE_CLASSES)(*table)
    _check(lib.rmc_batch_set_tiles(context().bind(), t, RMC_BATCH_TILE_CLASSES), "rmc_batch_set_tiles")


class rmc_serve_request(ctypes.Structure):
    """Mirror of the C struct rmc_serve_request."""
    _fields_ = [("req", rmc_request), ("sketch", _int), ("prec", _int)]


lib.rmc_server_create.argtypes = [ctypes.POINTER(_p), _sz, _int, _int]
lib.rmc_server_destroy.argtypes = [_p]
lib.rmc_server_submit.argtypes = [_p, ctypes.POINTER(rmc_serve_request), ctypes.POINTER(_u64)]
lib.rmc_server_progress.argtypes = [_p, ctypes.POINTER(_int), ctypes.POINTER(_int)]
lib.rmc_server_poll.argtypes = [_p, ctypes.POINTER(_u64), ctypes.POINTER(_int), ctypes.POINTER(ctypes.c_double),
                                _int, ctypes.POINTER(_int)]
lib.rmc_server_drain.argtypes = [_p]
lib.rmc_server_resident.argtypes = [_p, _sz]
lib.rmc_server_release.argtypes = [_p, _p]
for _f in ("rmc_server_create", "rmc_server_destroy", "rmc_server_submit", "rmc_server_progress",
           "rmc_server_poll", "rmc_server_drain", "rmc_server_resident", "rmc_server_release"):
    getattr(lib, _f).restype = ctypes.c_int


class Server:
    """Continuous-batching server (rmc_server_*) on the current device.  Requests are (rmc_request, sketch,
    prec); their tensors must stay alive until the request is polled as done."""

    def __init__(self, hbm_budget, nstreams=4, max_batch=256):
        self.handle = _p()
        _check(lib.rmc_server_create(ctypes.byref(self.handle), _sz(hbm_budget), nstreams, max_batch),
               "rmc_server_create")
        self._buf = 256
        self._t = (_u64 * self._buf)()
        self._s = (_int * self._buf)()
        self._l = (ctypes.c_double * self._buf)()

    def submit(self, request, sketch="countsketch", prec="fp32"):
        r = rmc_serve_request(req=request, sketch=_kind(sketch), prec=_prec(prec))
        t = _u64()
        _check(lib.rmc_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "rmc_server_submit")
        return t.value

    def progress(self):
        a, b = _int(), _int()
        _check(lib.rmc_server_progress(self.handle, ctypes.byref(a), ctypes.byref(b)), "rmc_server_progress")
        return a.value, b.value

    def poll(self):
        """[(ticket, status, latency_s)] of the requests completed since the last poll."""
        out = []
        while True:
            c = _int()
            _check(lib.rmc_server_poll(self.handle, self._t, self._s, self._l, self._buf, ctypes.byref(c)),
                   "rmc_server_poll")
            out.extend((self._t[i], self._s[i], self._l[i]) for i in range(c.value))
            if c.value < self._buf:
                return out

    def drain(self):
        _check(lib.rmc_server_drain(self.handle), "rmc_server_drain")

    def resident(self, nbytes):
        """Keep least-squares sketches and their factors resident, up to nbytes of device memory (0: off)."""
        _check(lib.rmc_server_resident(self.handle, _sz(nbytes)), "rmc_server_resident")

    def release(self, A):
        """Drop the resident state derived from A (before A is modified or freed)."""
        _check(lib.rmc_server_release(self.handle, _p(A.data_ptr())), "rmc_server_release")

    def close(self):
        if self.handle:
            lib.rmc_server_destroy(self.handle)
            self.handle = _p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
