"""GB300 single-pass randomized PCA (Yu et al., IJCAI 2017, Alg. 4) - Python binding.

A thin ctypes layer over the C ABI in include/spca.h: every function here has
the name of the C function it calls and only marshals arguments (torch tensors
or numpy arrays to pointers, sizes, dtype codes). All arithmetic of the method
runs in the CUDA library ``libspca.so``, built in-tree by ``build.build()``.
There is no fallback: if the library is missing or cannot load, every call
raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

SPCA_OK = 0
STATUS_NAMES = {0: "SPCA_OK", 1: "SPCA_E_INVALID", 2: "SPCA_E_NOMEM", 3: "SPCA_E_CUDA", 4: "SPCA_E_STATE",
                5: "SPCA_E_NUMERIC", 6: "SPCA_E_TIMEOUT", 7: "SPCA_E_UNSUPPORTED"}
SPCA_F32, SPCA_BF16, SPCA_F8E4M3, SPCA_F64 = 0, 1, 2, 3
SPCA_MATH_FP32, SPCA_MATH_BF16, SPCA_MATH_BF16X2, SPCA_MATH_FP8, SPCA_MATH_FP16 = 0, 1, 2, 3, 4
MATH_NAMES = {"fp32": SPCA_MATH_FP32, "bf16": SPCA_MATH_BF16, "bf16x2": SPCA_MATH_BF16X2, "fp8": SPCA_MATH_FP8,
              "fp16": SPCA_MATH_FP16}


class SpcaError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("math", ctypes.c_int32), ("center", ctypes.c_int32), ("max_block_rows", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_size_t), ("math", ctypes.c_int32), ("max_sessions", ctypes.c_int32),
                ("max_block_rows", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("updates_done", ctypes.c_int64), ("finalizes_done", ctypes.c_int64),
                ("sessions_admitted", ctypes.c_int64), ("sessions_waiting", ctypes.c_int64),
                ("update_p50_ms", ctypes.c_double), ("update_p99_ms", ctypes.c_double),
                ("finalize_p50_ms", ctypes.c_double), ("finalize_p99_ms", ctypes.c_double),
                ("rows_bytes", ctypes.c_double), ("active_seconds", ctypes.c_double),
                ("device_bytes_in_use", ctypes.c_size_t), ("device_bytes_budget", ctypes.c_size_t),
                ("sessions_pooled", ctypes.c_int64), ("admissions_from_pool", ctypes.c_int64),
                ("sessions_created", ctypes.c_int64), ("device_bytes_pooled", ctypes.c_size_t)]


SPCA_SERVER_AUTO_MATH = -1
_LIB = None


def lib_path():
    return _build.LIB


def lib():
    """The loaded libspca.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_1704_07669_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
        sig = {
            "spca_default_options": (None, [ctypes.POINTER(Options)]),
            "spca_create": (i32, [i64, i32, i32, u64, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
            "spca_update": (i32, [vp, vp, i64, i64, i32, vp, i32, vp]),
            "spca_finalize": (i32, [vp, vp, vp, i32]),
            "spca_left_vectors": (i32, [vp, vp, i64, vp, i32]),
            "spca_left_vectors_pass": (i32, [vp, vp, i64, i64, i32, vp, vp, i64]),
            "spca_power_step": (i32, [vp]),
            "spca_state_bytes": (i32, [vp, ctypes.POINTER(ctypes.c_size_t)]),
            "spca_save_state": (i32, [vp, vp, ctypes.c_size_t]),
            "spca_load_state": (i32, [vp, vp, ctypes.c_size_t]),
            "spca_get_state": (i32, [vp, vp, vp, vp, vp, vp]),
            "spca_merge": (i32, [vp, vp]),
            "spca_sync": (i32, [vp]),
            "spca_destroy": (i32, [vp]),
            "spca_last_error": (ctypes.c_char_p, [vp]),
            "spca_rows_seen": (i64, [vp]),
            "spca_reset": (i32, [vp, u64]),
            "spca_describe": (ctypes.c_char_p, [vp]),
            "spca_set_profiling": (i32, [vp, i32]),
            "spca_get_profile": (i32, [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]),
            "spca_clear_profile": (i32, [vp]),
            "spca_omega_words": (i32, [u64, i64, i32, vp]),
            "spca_omega": (i32, [u64, i64, i32, vp]),
            "spca_shift_static": (i32, [vp, i64, i64, i64, i32, vp, vp, vp]),
            "spca_wait_selftest": (i32, [i64, vp]),
            "spca_server_default_options": (None, [ctypes.POINTER(ServerOptions)]),
            "spca_server_create": (i32, [ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)]),
            "spca_server_open": (i32, [vp, i64, i32, i32, u64, ctypes.POINTER(i32)]),
            "spca_server_reserve": (i32, [vp, i64, i32, i32, i32, ctypes.POINTER(u64)]),
            "spca_server_update": (i32, [vp, i32, vp, i64, i64, ctypes.POINTER(u64)]),
            "spca_server_finalize": (i32, [vp, i32, vp, vp, ctypes.POINTER(u64)]),
            "spca_server_wait": (i32, [vp, u64, ctypes.c_double]),
            "spca_server_close": (i32, [vp, i32]),
            "spca_server_get_stats": (i32, [vp, ctypes.POINTER(ServerStats)]),
            "spca_server_destroy": (i32, [vp]),
            "spca_server_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(status, handle=None):
    if status != SPCA_OK:
        msg = lib().spca_last_error(handle)
        raise SpcaError(status, msg.decode() if msg else "")


def _ptr(x):
    """(address, on_device) of a torch tensor or numpy array, or (x, None) for an int."""
    if x is None:
        return None, None
    if isinstance(x, np.ndarray):
        return x.ctypes.data, False
    if hasattr(x, "data_ptr"):
        return x.data_ptr(), bool(x.is_cuda)
    return int(x), None


def _wait_for_torch(*tensors):
    """CUDA tensors handed to a library stream other than torch's may still be written by work
    queued on torch's current stream (their producer, or a fill of an output buffer): the host
    waits for that work before the library's stream reads or writes them."""
    for t in tensors:
        if t is not None and getattr(t, "is_cuda", False):
            import torch
            torch.cuda.current_stream(t.device).synchronize()
            return


def _unit_column_stride(x, what):
    """Rows are read row-major with leading dimension ld: a view whose columns are not adjacent
    would be read as if they were."""
    if hasattr(x, "stride") and callable(x.stride):
        ok = x.dim() == 2 and (x.stride(1) == 1 or x.shape[1] <= 1)
    elif isinstance(x, np.ndarray):
        ok = x.ndim == 2 and (x.strides[1] == x.itemsize or x.shape[1] <= 1)
    else:
        return
    if not ok:
        raise ValueError(f"{what} must be a 2-D row-major array with adjacent columns")


def _float64_buffer(x, what):
    """Result buffers are written as doubles; another dtype would be overrun."""
    if x is None or not (hasattr(x, "dtype")):
        return
    if not str(x.dtype).endswith("float64"):
        raise ValueError(f"{what} must hold float64 values, got {x.dtype}")
    contiguous = x.is_contiguous() if hasattr(x, "is_contiguous") else x.flags["C_CONTIGUOUS"]
    if not contiguous:
        raise ValueError(f"{what} must be contiguous")


def _dtype_code(x):
    name = str(getattr(x, "dtype", ""))
    if name.endswith("float32"):
        return SPCA_F32
    if name.endswith("float64"):
        return SPCA_F64
    if name.endswith("bfloat16"):
        return SPCA_BF16
    if name.endswith("float8_e4m3fn") or name.endswith("uint8"):
        return SPCA_F8E4M3
    raise ValueError(f"unsupported row dtype {name}")


# ---------------------------------------------------------------- C ABI, one function each

def spca_create(n, k, p, seed, math=SPCA_MATH_FP32, center=1, max_block_rows=0, stream=None):
    opt = Options()
    lib().spca_default_options(ctypes.byref(opt))
    opt.math = MATH_NAMES[math] if isinstance(math, str) else int(math)
    opt.center = int(center)
    opt.max_block_rows = int(max_block_rows)
    opt.cuda_stream = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    out = ctypes.c_void_p()
    _check(lib().spca_create(int(n), int(k), int(p), int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.byref(opt),
                             ctypes.byref(out)))
    return out.value


def spca_update(handle, rows, m_i=None, ld=None, dtype=None, block_scale=None, rows_on_device=None, G_out=None):
    if ld is None:
        _unit_column_stride(rows, "rows")
    addr, on_dev = _ptr(rows)
    if m_i is None:
        m_i = rows.shape[0]
    if ld is None:
        ld = (rows.stride(0) if hasattr(rows, "stride") and callable(rows.stride)
              else rows.strides[0] // rows.itemsize)
    if dtype is None:
        dtype = _dtype_code(rows)
    if rows_on_device is None:
        rows_on_device = bool(on_dev)
    scale = None
    if block_scale is not None:
        scale = ctypes.c_float(float(block_scale))
    g_addr, _ = _ptr(G_out)
    _check(lib().spca_update(handle, addr, int(m_i), int(ld), int(dtype),
                             ctypes.cast(ctypes.byref(scale), ctypes.c_void_p) if scale is not None else None,
                             int(rows_on_device), g_addr), handle)


def spca_finalize(handle, sigma, V, out_on_device=None):
    """Fill sigma (k doubles) and V (n x k doubles, column-major) - tensors or arrays."""
    _float64_buffer(sigma, "sigma")
    _float64_buffer(V, "V")
    sa, sdev = _ptr(sigma)
    va, vdev = _ptr(V)
    on = bool(sdev) if out_on_device is None else bool(out_on_device)
    _check(lib().spca_finalize(handle, sa, va, int(on)), handle)


def spca_left_vectors(handle, G, U, m=None, out_on_device=None):
    """Fill U (m x k doubles, column-major) from the kept sketch rows G (m x l FP32 CUDA tensor)."""
    _float64_buffer(U, "U")
    ga, _ = _ptr(G)
    ua, udev = _ptr(U)
    if m is None:
        m = G.shape[0]
    on = bool(udev) if out_on_device is None else bool(out_on_device)
    _check(lib().spca_left_vectors(handle, ga, int(m), ua, int(on)), handle)


def spca_left_vectors_pass(handle, rows, U, block_scale=None):
    """U rows of the device rows `rows` (m x n, any storage dtype) by a second pass, into U: a
    CUDA float64 tensor of shape (k, m) (column-major m x k; ldu = its row stride)."""
    _unit_column_stride(rows, "rows")
    if not str(getattr(U, "dtype", "")).endswith("float64") or U.dim() != 2 or U.stride(1) != 1:
        raise ValueError("spca_left_vectors_pass: U must be a 2-D float64 tensor with adjacent columns")
    addr, on_dev = _ptr(rows)
    ua, udev = _ptr(U)
    if not on_dev or not udev:
        raise ValueError("spca_left_vectors_pass: rows and U must be CUDA tensors")
    m = int(rows.shape[0])
    ld = rows.stride(0)
    scale = None if block_scale is None else ctypes.c_float(float(block_scale))
    _check(lib().spca_left_vectors_pass(handle, addr, m, int(ld), int(_dtype_code(rows)),
                                        ctypes.cast(ctypes.byref(scale), ctypes.c_void_p) if scale is not None else None,
                                        ua, int(U.stride(0))), handle)


def spca_wait_selftest(limit_ns, stream=None):
    """The bounded-wait self-test: raises SpcaError with status SPCA_E_TIMEOUT after about limit_ns."""
    st = None if stream is None else int(getattr(stream, "cuda_stream", stream))
    _check(lib().spca_wait_selftest(int(limit_ns), st))


def spca_power_step(handle):
    _check(lib().spca_power_step(handle), handle)


def spca_save_state(handle):
    """A checkpoint of the session's accumulators (bytes)."""
    nb = ctypes.c_size_t(0)
    _check(lib().spca_state_bytes(handle, ctypes.byref(nb)), handle)
    buf = ctypes.create_string_buffer(nb.value)
    _check(lib().spca_save_state(handle, ctypes.cast(buf, ctypes.c_void_p), nb), handle)
    return buf.raw


def spca_load_state(handle, data):
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(lib().spca_load_state(handle, ctypes.cast(buf, ctypes.c_void_p), len(data)), handle)


def spca_get_state(handle, H_bar=None, gram_bar=None, colsum=None, shift=None):
    m = ctypes.c_int64(0)
    _check(lib().spca_get_state(handle, _ptr(H_bar)[0], _ptr(gram_bar)[0], _ptr(colsum)[0], _ptr(shift)[0],
                                ctypes.byref(m)), handle)
    return m.value


def spca_merge(dst, src):
    _check(lib().spca_merge(dst, src), dst)


def spca_sync(handle):
    _check(lib().spca_sync(handle), handle)


def spca_destroy(handle):
    _check(lib().spca_destroy(handle))


def spca_last_error(handle=None):
    msg = lib().spca_last_error(handle)
    return msg.decode() if msg else ""


def spca_rows_seen(handle):
    return lib().spca_rows_seen(handle)


def spca_describe(handle):
    d = lib().spca_describe(handle)
    return d.decode() if d else ""


def spca_reset(handle, seed):
    _check(lib().spca_reset(handle, int(seed) & 0xFFFFFFFFFFFFFFFF), handle)


KERNEL_NAMES = ["omega", "shift", "g_partial", "g_finish", "gram_accum", "h_partial", "h_finish", "finalize",
                "tc_sketch"]


def spca_set_profiling(handle, on):
    _check(lib().spca_set_profiling(handle, int(bool(on))), handle)


def spca_get_profile(handle, kernel):
    """(total_ms, launches) for one kernel class (index or name)."""
    kid = KERNEL_NAMES.index(kernel) if isinstance(kernel, str) else int(kernel)
    ms = ctypes.c_double(0.0)
    n = ctypes.c_int64(0)
    _check(lib().spca_get_profile(handle, kid, ctypes.byref(ms), ctypes.byref(n)), handle)
    return ms.value, n.value


def spca_clear_profile(handle):
    _check(lib().spca_clear_profile(handle), handle)


def spca_omega_words(seed, n, l, out):
    _check(lib().spca_omega_words(int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), int(l), _ptr(out)[0]))


def spca_omega(seed, n, l, out):
    _check(lib().spca_omega(int(seed) & 0xFFFFFFFFFFFFFFFF, int(n), int(l), _ptr(out)[0]))


def spca_shift_static(rows, shift, block_scale=None, stream=None):
    """The allocation-free shift: shift[:n] = FP32 of the FP64 column means of the
    2-D device tensor ``rows`` (row stride = leading dimension), enqueued on
    ``stream`` (a torch.cuda.Stream or a raw handle; None: torch's current stream
    on the rows' device, so that the launch is ordered after the work that made
    ``rows``)."""
    if rows.dim() != 2 or not rows.is_cuda:
        raise ValueError("rows must be a 2-D CUDA tensor")
    m, n = rows.shape
    if rows.stride(1) != 1:
        raise ValueError("rows must be row-major with unit column stride")
    if not (getattr(shift, "is_cuda", False) and str(shift.dtype).endswith("float32")
            and shift.is_contiguous() and shift.numel() >= n and shift.device == rows.device):
        raise ValueError("shift must be a contiguous float32 CUDA tensor of at least n elements on the rows' device")
    scale = None if block_scale is None else ctypes.c_float(float(block_scale))
    bs = None if scale is None else ctypes.cast(ctypes.byref(scale), ctypes.c_void_p)
    if stream is None:
        import torch
        st = torch.cuda.current_stream(rows.device).cuda_stream
    else:
        st = int(getattr(stream, "cuda_stream", stream))
    _check(lib().spca_shift_static(_ptr(rows)[0], int(m), int(n), int(rows.stride(0)), _dtype_code(rows), bs,
                                   _ptr(shift)[0], st))


# ---------------------------------------------------------------- convenience wrapper

class Session:
    """RAII wrapper: Session(n, k, p, seed, math='fp32') with update/finalize/state."""

    def __init__(self, n, k, p, seed, math=SPCA_MATH_FP32, center=True, max_block_rows=0, stream=None):
        self.n, self.k, self.p = int(n), int(k), int(p)
        self.l = self.k + self.p
        self.seed, self.math, self.center, self.max_block_rows = int(seed), math, bool(center), int(max_block_rows)
        self.handle = spca_create(n, k, p, seed, math=math, center=int(center), max_block_rows=max_block_rows,
                                  stream=stream)
        self.own_stream = stream is None   # the library's own stream: not ordered after torch's

    def update(self, rows, G_out=None, block_scale=None):
        if self.own_stream:
            _wait_for_torch(rows, G_out)
        spca_update(self.handle, rows, G_out=G_out, block_scale=block_scale)

    def finalize(self):
        """(sigma, V) as float64 numpy arrays, V of shape (n, k)."""
        sigma = np.zeros(self.k)
        Vc = np.zeros((self.k, self.n))      # column-major n x k == row-major k x n
        spca_finalize(self.handle, sigma, Vc, out_on_device=False)
        return sigma, Vc.T.copy()

    def left_vectors(self, G):
        """U (m x k float64 numpy) of the last finalize, from the kept sketch rows G (the G_out
        rows, an m x l FP32 CUDA tensor)."""
        if self.own_stream:
            _wait_for_torch(G)
        m = int(G.shape[0])
        Uc = np.zeros((self.k, m))      # column-major m x k == row-major k x m
        spca_left_vectors(self.handle, G, Uc, m=m, out_on_device=False)
        return Uc.T.copy()

    def left_vectors_pass(self, rows, block_scale=None):
        """U (m x k float64 CUDA tensor) of the CUDA rows `rows` by a second pass over them (after
        a finalize): (rows - column means) V diag(sigma)^-1. Ordered on the session stream; the
        result is read after sync()."""
        import torch
        if self.own_stream:
            _wait_for_torch(rows)
        m = int(rows.shape[0])
        Uc = torch.empty((self.k, m), dtype=torch.float64, device=rows.device)
        spca_left_vectors_pass(self.handle, rows, Uc, block_scale=block_scale)
        return Uc.T

    def save_state(self):
        """A checkpoint (bytes) that load_state restores into a session of the same parameters."""
        return spca_save_state(self.handle)

    def load_state(self, data):
        spca_load_state(self.handle, data)

    def power_step(self):
        """Omega <- orth(H_bar) for one more pass over the same rows (power scheme, P = 1)."""
        spca_power_step(self.handle)

    def state(self):
        H = np.zeros((self.n, self.l))
        g = np.zeros((self.l, self.l))
        cs = np.zeros(self.n)
        sh = np.zeros(self.n, dtype=np.float32)
        m = spca_get_state(self.handle, H, g, cs, sh)
        return {"H_bar": H, "gram_bar": g, "colsum": cs, "shift": sh, "m": m}

    def reset(self, seed):
        spca_reset(self.handle, seed)

    def profile(self):
        """{kernel name: (total_ms, launches)} since the last clear."""
        return {name: spca_get_profile(self.handle, i) for i, name in enumerate(KERNEL_NAMES)}

    @property
    def rows_seen(self):
        return spca_rows_seen(self.handle)

    def sync(self):
        spca_sync(self.handle)

    def close(self):
        if self.handle:
            spca_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving loop (include/spca_server.h)

def _check_srv(status):
    if status != SPCA_OK:
        msg = lib().spca_server_last_error()
        raise SpcaError(status, msg.decode() if msg else "")


class Server:
    """Thin wrapper of the spca_server_* calls: sessions resident on the device, requests queued
    from any thread, completed by the library's worker thread."""

    def __init__(self, device_bytes=0, math=SPCA_SERVER_AUTO_MATH, max_sessions=1024, max_block_rows=4096):
        opt = ServerOptions()
        lib().spca_server_default_options(ctypes.byref(opt))
        opt.device_bytes = int(device_bytes)
        opt.math = MATH_NAMES[math] if isinstance(math, str) else int(math)
        opt.max_sessions = int(max_sessions)
        opt.max_block_rows = int(max_block_rows)
        h = ctypes.c_void_p()
        _check_srv(lib().spca_server_create(ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h.value
        self._shapes = {}   # session id -> (n, k), for the size of the result buffers

    def open(self, n, k, p, seed):
        sid = ctypes.c_int32(-1)
        _check_srv(lib().spca_server_open(self.handle, int(n), int(k), int(p), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                          ctypes.byref(sid)))
        self._shapes[sid.value] = (int(n), int(k))
        return sid.value

    def reserve(self, n, k, p, count):
        """Queue the creation of `count` pooled sessions of sizes (n, k, p); returns a ticket."""
        t = ctypes.c_uint64(0)
        _check_srv(lib().spca_server_reserve(self.handle, int(n), int(k), int(p), int(count), ctypes.byref(t)))
        return t.value

    def update(self, sid, rows):
        """Queue a block of device-resident FP32 rows (a 2-D CUDA tensor); returns a ticket. The
        worker reads them on its own streams, after the work queued on torch's current stream."""
        _unit_column_stride(rows, "rows")
        if not str(rows.dtype).endswith("float32"):
            raise ValueError(f"the serving loop takes FP32 rows, got {rows.dtype}")
        _wait_for_torch(rows)
        t = ctypes.c_uint64(0)
        _check_srv(lib().spca_server_update(self.handle, int(sid), _ptr(rows)[0], int(rows.shape[0]),
                                            int(rows.stride(0)), ctypes.byref(t)))
        return t.value

    def finalize(self, sid, sigma, V):
        """Queue a finalisation into host numpy buffers sigma (k) and V (k x n, i.e. n x k column-major)."""
        _float64_buffer(sigma, "sigma")
        _float64_buffer(V, "V")
        n, k = self._shapes.get(int(sid), (0, 0))
        if sigma.size < k or V.size < n * k:
            raise ValueError(f"sigma needs {k} and V {n * k} float64 values")
        t = ctypes.c_uint64(0)
        _check_srv(lib().spca_server_finalize(self.handle, int(sid), _ptr(sigma)[0], _ptr(V)[0], ctypes.byref(t)))
        return t.value

    def wait(self, ticket, timeout_s=-1.0):
        _check_srv(lib().spca_server_wait(self.handle, int(ticket), float(timeout_s)))

    def close_session(self, sid):
        _check_srv(lib().spca_server_close(self.handle, int(sid)))

    def stats(self):
        st = ServerStats()
        _check_srv(lib().spca_server_get_stats(self.handle, ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            lib().spca_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
