"""Thin ctypes binding of the C ABI in include/tdes.h (argument marshalling only).

Every function takes the same arguments as its C counterpart, with torch
tensors standing in for device pointers (uint8, contiguous, on the key
schedule's device) and the current torch stream standing in for the
cudaStream_t unless one is given.  All cipher work runs in the CUDA kernels
of libtdes_gb300.so; if that library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtdes_gb300.so")

TDES_OK = 0
TDES_EINVAL = -1
TDES_ENOMEM = -2
TDES_EBUSY = -3
TDES_ETIMEDOUT = -4
TDES_ECUDA = -5

# every symbol include/tdes.h declares
EXPORTED = (
    "tdes_key_schedule", "tdes_key_schedule_2key", "tdes_des_key_schedule",
    "tdes_key_schedule_stages", "tdes_key_free", "tdes_ecb_encrypt", "tdes_ecb_decrypt",
    "tdes_ctr_crypt", "tdes_cbc_decrypt", "tdes_cbc_encrypt", "tdes_cbc_decrypt_noalloc",
    "tdes_ecb_crypt_host", "tdes_keytable_create", "tdes_keytable_free", "tdes_batch_plan",
    "tdes_batch_configure", "tdes_batch_launch", "tdes_batch_launch_graph", "tdes_batch_info",
    "tdes_batch_free", "tdes_batch_set_shape", "tdes_batch_get_shape", "tdes_batch_autotune",
    "tdes_autotune_cache_path", "tdes_ctx_config_default", "tdes_ctx_create", "tdes_ctx_destroy",
    "tdes_batch_submit", "tdes_batch_submit_plan", "tdes_batch_poll", "tdes_batch_wait",
    "tdes_batch_release", "tdes_uniform_scratch_bytes", "tdes_uniform_crypt", "tdes_uniform_info",
    "tdes_server_config_default", "tdes_server_create", "tdes_server_submit",
    "tdes_server_poll", "tdes_server_wait", "tdes_server_submit_group",
    "tdes_server_poll_group", "tdes_server_wait_group", "tdes_server_destroy", "tdes_serve_loadtest",
    "tdes_server_stats", "tdes_server_autotune",
    "tdes_sbox_gate_count", "tdes_set_small_cutoff", "tdes_strerror", "tdes_last_error",
)

TUNE_FORCE = 1
TUNE_NO_STORE = 2
ROUNDS_PER_PASS = 0
ROUNDS_COMPACT = 1

MODE_ECB_ENCRYPT = 0
MODE_ECB_DECRYPT = 1
MODE_CTR = 2
MODE_CBC_DECRYPT = 3
MODE_CBC_ENCRYPT = 4


class Desc(ctypes.Structure):
    """tdes_desc_t"""
    _fields_ = [("mode", ctypes.c_uint32), ("key_index", ctypes.c_uint32),
                ("iv_or_ctr", ctypes.c_uint64), ("in_ptr", ctypes.c_void_p),
                ("out_ptr", ctypes.c_void_p), ("nbytes", ctypes.c_uint64)]


class ServerConfig(ctypes.Structure):
    """tdes_server_config_t"""
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_batch", ctypes.c_uint32), ("warps_per_cta", ctypes.c_int),
                ("reserve_ctas_per_sm", ctypes.c_int), ("ring_entries", ctypes.c_uint32),
                ("stage_bytes", ctypes.c_uint64), ("stage_min_bytes", ctypes.c_uint64),
                ("round_form", ctypes.c_int)]


class LoadtestConfig(ctypes.Structure):
    """tdes_loadtest_config_t"""
    _fields_ = [("n_requests", ctypes.c_uint64), ("offered_gbps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("small_frac", ctypes.c_double),
                ("small_min", ctypes.c_uint32), ("small_max", ctypes.c_uint32),
                ("large_min", ctypes.c_uint64), ("large_max", ctypes.c_uint64),
                ("mode_probs", ctypes.c_double * 3), ("n_keys", ctypes.c_uint32),
                ("in_pool", ctypes.c_void_p), ("in_pool_bytes", ctypes.c_uint64),
                ("out_pool", ctypes.c_void_p), ("out_pool_bytes", ctypes.c_uint64)]


class LoadtestResult(ctypes.Structure):
    """tdes_loadtest_result_t"""
    _fields_ = [(n, ctypes.c_double) for n in (
        "p50_ms", "p90_ms", "p99_ms", "p999_ms", "mean_ms", "max_ms", "small_p50_ms",
        "small_p99_ms", "large_p50_ms", "large_p99_ms", "gbps", "offered_gbps", "duration_s")] + [
        ("requests", ctypes.c_uint64), ("bytes", ctypes.c_uint64), ("batches", ctypes.c_uint64),
        ("max_slots_busy", ctypes.c_uint32), ("max_device_overlap", ctypes.c_uint32),
        ("device_overlap_frac", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    """tdes_server_stats_t"""
    _fields_ = [("batches", ctypes.c_uint64), ("max_slots_busy", ctypes.c_uint32),
                ("max_device_overlap", ctypes.c_uint32), ("device_busy_ms", ctypes.c_double),
                ("device_overlap_ms", ctypes.c_double), ("batch_ms_sum", ctypes.c_double),
                ("untimed_batches", ctypes.c_uint64)]


class ServerAutotuneResult(ctypes.Structure):
    """tdes_server_autotune_result_t"""
    _fields_ = [("key", ctypes.c_char * 64), ("best", ServerConfig), ("baseline", ServerConfig),
                ("best_gbps", ctypes.c_double), ("baseline_gbps", ctypes.c_double),
                ("candidates", ctypes.c_uint32), ("from_cache", ctypes.c_int),
                ("best_p99_ms", ctypes.c_double), ("baseline_p99_ms", ctypes.c_double),
                ("load_gbps", ctypes.c_double)]


class BatchInfo(ctypes.Structure):
    """tdes_batch_info_t"""
    _fields_ = [("n_cbc_enc_messages", ctypes.c_uint32), ("n_tiles", ctypes.c_uint64),
                ("n_small_items", ctypes.c_uint32), ("warps_per_cta", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("bytes_per_mode", ctypes.c_uint64 * 5),
                ("n_mixed_tiles", ctypes.c_uint64), ("n_direct_messages", ctypes.c_uint32),
                ("tiles_per_claim", ctypes.c_int), ("round_form", ctypes.c_int),
                ("tuned", ctypes.c_int)]


class LaunchShape(ctypes.Structure):
    """tdes_launch_shape_t"""
    _fields_ = [("warps_per_cta", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("tiles_per_claim", ctypes.c_int), ("round_form", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class AutotuneResult(ctypes.Structure):
    """tdes_autotune_result_t"""
    _fields_ = [("key", ctypes.c_char * 64), ("best", LaunchShape), ("baseline", LaunchShape),
                ("best_ms", ctypes.c_double), ("baseline_ms", ctypes.c_double),
                ("candidates", ctypes.c_uint32), ("from_cache", ctypes.c_int)]


class CtxConfig(ctypes.Structure):
    """tdes_ctx_config_t"""
    _fields_ = [("streams", ctypes.c_uint32)]

class UniformInfo(ctypes.Structure):
    """tdes_uniform_info_t"""
    _fields_ = [("skipped", ctypes.c_uint64), ("key_tiles", ctypes.c_uint32),
                ("mixed_slices", ctypes.c_uint32), ("chain_key_tiles", ctypes.c_uint32),
                ("chain_slices", ctypes.c_uint32)]


_lib = None


class TdesError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"tdes status {status}: {message}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load the CUDA library (built by paper_2007_10752_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run python -m paper_2007_10752_gb300.build")
    lib = ctypes.CDLL(path)
    vp, sz, u32, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint32, ctypes.c_uint64
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.tdes_key_schedule.argtypes = [u8p, u8p, u8p, ctypes.POINTER(vp)]
    lib.tdes_key_schedule_2key.argtypes = [u8p, u8p, ctypes.POINTER(vp)]
    lib.tdes_des_key_schedule.argtypes = [u8p, ctypes.POINTER(vp)]
    lib.tdes_key_schedule_stages.argtypes = [vp]
    lib.tdes_key_schedule_stages.restype = ctypes.c_int
    lib.tdes_key_free.argtypes = [vp]
    lib.tdes_key_free.restype = None
    for name in ("tdes_ecb_encrypt", "tdes_ecb_decrypt"):
        getattr(lib, name).argtypes = [vp, vp, vp, sz, vp]
    lib.tdes_ctr_crypt.argtypes = [vp, u32, u32, vp, vp, sz, vp]
    lib.tdes_cbc_decrypt.argtypes = [vp, u64, vp, vp, sz, vp]
    lib.tdes_cbc_encrypt.argtypes = [vp, u64, vp, vp, sz, vp]
    lib.tdes_cbc_decrypt_noalloc.argtypes = [vp, u64, vp, vp, sz, vp]
    lib.tdes_ecb_crypt_host.argtypes = [vp, ctypes.c_int, vp, vp, sz, vp, sz]
    lib.tdes_keytable_create.argtypes = [vp, u32, ctypes.POINTER(vp)]
    lib.tdes_keytable_free.argtypes = [vp]
    lib.tdes_keytable_free.restype = None
    lib.tdes_batch_plan.argtypes = [vp, vp, u32, vp, ctypes.POINTER(vp)]
    lib.tdes_batch_configure.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.tdes_batch_launch.argtypes = [vp, vp]
    lib.tdes_batch_launch_graph.argtypes = [vp, vp]
    lib.tdes_batch_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    lib.tdes_batch_free.argtypes = [vp]
    lib.tdes_batch_free.restype = None
    lib.tdes_batch_set_shape.argtypes = [vp, ctypes.POINTER(LaunchShape)]
    lib.tdes_batch_get_shape.argtypes = [vp, ctypes.POINTER(LaunchShape)]
    lib.tdes_batch_autotune.argtypes = [vp, ctypes.c_uint, ctypes.c_int, vp,
                                        ctypes.POINTER(AutotuneResult)]
    lib.tdes_autotune_cache_path.argtypes = []
    lib.tdes_autotune_cache_path.restype = ctypes.c_char_p
    lib.tdes_ctx_config_default.argtypes = [ctypes.POINTER(CtxConfig)]
    lib.tdes_ctx_config_default.restype = None
    lib.tdes_ctx_create.argtypes = [vp, ctypes.POINTER(CtxConfig), ctypes.POINTER(vp)]
    lib.tdes_ctx_destroy.argtypes = [vp]
    lib.tdes_ctx_destroy.restype = None
    lib.tdes_batch_submit.argtypes = [vp, vp, u32, ctypes.POINTER(u64)]
    lib.tdes_batch_submit_plan.argtypes = [vp, vp, ctypes.POINTER(u64)]
    lib.tdes_batch_poll.argtypes = [vp, u64, vp]
    lib.tdes_batch_wait.argtypes = [vp, u64, u64]
    lib.tdes_batch_release.argtypes = [vp, u64]
    lib.tdes_uniform_scratch_bytes.argtypes = [vp, u64, u64, ctypes.POINTER(sz)]
    lib.tdes_uniform_crypt.argtypes = [vp, vp, vp, vp, vp, vp, u64, u64, vp, sz, vp, vp]
    lib.tdes_uniform_info.argtypes = [vp, ctypes.POINTER(UniformInfo)]
    lib.tdes_server_config_default.argtypes = [ctypes.POINTER(ServerConfig)]
    lib.tdes_server_config_default.restype = None
    lib.tdes_server_create.argtypes = [vp, ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    lib.tdes_server_submit.argtypes = [vp, ctypes.POINTER(Desc), ctypes.POINTER(u64)]
    lib.tdes_server_poll.argtypes = [vp, u64]
    lib.tdes_server_wait.argtypes = [vp, u64, u64]
    lib.tdes_server_submit_group.argtypes = [vp, vp, u32, ctypes.POINTER(u64)]
    lib.tdes_server_poll_group.argtypes = [vp, u64, u32, vp]
    lib.tdes_server_wait_group.argtypes = [vp, u64, u32, u64]
    lib.tdes_server_destroy.argtypes = [vp]
    lib.tdes_server_destroy.restype = None
    lib.tdes_serve_loadtest.argtypes = [vp, ctypes.POINTER(LoadtestConfig),
                                        ctypes.POINTER(LoadtestResult)]
    lib.tdes_server_stats.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ServerStats)]
    lib.tdes_server_autotune.argtypes = [vp, ctypes.POINTER(LoadtestConfig), ctypes.c_uint,
                                         ctypes.POINTER(ServerAutotuneResult)]
    lib.tdes_sbox_gate_count.argtypes = []
    lib.tdes_set_small_cutoff.argtypes = [u64]
    lib.tdes_set_small_cutoff.restype = u64
    lib.tdes_strerror.argtypes = [ctypes.c_int]
    lib.tdes_strerror.restype = ctypes.c_char_p
    lib.tdes_last_error.argtypes = []
    lib.tdes_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != TDES_OK:
        msg = load().tdes_last_error().decode(errors="replace")
        raise TdesError(status, msg)


def _ptr(t) -> int:
    """Device (or host) address of a tensor / ndarray / int."""
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return t.data_ptr()


def _nbytes(t) -> int:
    if isinstance(t, np.ndarray):
        return t.nbytes
    return t.numel() * t.element_size()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _key_ptrs(*keys):
    if any(len(bytes(k)) != 8 for k in keys):
        raise ValueError("each key is 8 bytes")
    bufs = [(ctypes.c_uint8 * 8).from_buffer_copy(bytes(k)) for k in keys]
    return bufs, [ctypes.cast(b, ctypes.POINTER(ctypes.c_uint8)) for b in bufs]


class KeySchedule:
    """Owns a tdes_ks_t built on the current device: EDE3 under (k1, k2, k3)
    by tdes_key_schedule (a triple that reduces to one DES pass gets a
    single-DES schedule), or by the named constructors below."""

    def __init__(self, k1: bytes, k2: bytes, k3: bytes, *, _handle=None):
        if _handle is not None:
            self.handle = _handle
            return
        _bufs, ptrs = _key_ptrs(k1, k2, k3)
        h = ctypes.c_void_p()
        _check(load().tdes_key_schedule(*ptrs, ctypes.byref(h)))
        self.handle = h.value

    @classmethod
    def from_triple(cls, keys24) -> "KeySchedule":
        k = bytes(keys24)
        if len(k) != 24:
            raise ValueError("a key triple is 24 bytes")
        return cls(k[:8], k[8:16], k[16:])

    @classmethod
    def two_key(cls, k1: bytes, k2: bytes) -> "KeySchedule":
        """Two-key 3DES: EDE3 under (k1, k2, k1) (tdes_key_schedule_2key)."""
        _bufs, ptrs = _key_ptrs(k1, k2)
        h = ctypes.c_void_p()
        _check(load().tdes_key_schedule_2key(*ptrs, ctypes.byref(h)))
        return cls(b"", b"", b"", _handle=h.value)

    @classmethod
    def des(cls, key: bytes) -> "KeySchedule":
        """Single DES under `key` (tdes_des_key_schedule)."""
        _bufs, ptrs = _key_ptrs(key)
        h = ctypes.c_void_p()
        _check(load().tdes_des_key_schedule(*ptrs, ctypes.byref(h)))
        return cls(b"", b"", b"", _handle=h.value)

    @property
    def stages(self) -> int:
        """DES passes per block: 3 (EDE3) or 1 (single DES)."""
        rc = load().tdes_key_schedule_stages(self.handle)
        _check(rc if rc < 0 else 0)
        return rc

    def free(self):
        if self.handle:
            load().tdes_key_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _io(inp, out):
    n = _nbytes(inp)
    if out is None:
        out = inp.new_empty(inp.shape) if not isinstance(inp, np.ndarray) else np.empty_like(inp)
    if _nbytes(out) < n:
        raise ValueError("output smaller than input")
    return out, n


def tdes_ecb_encrypt(ks: KeySchedule, inp, out=None, stream=None, nbytes=None):
    out, n = _io(inp, out)
    _check(load().tdes_ecb_encrypt(ks.handle, _ptr(inp), _ptr(out),
                                   n if nbytes is None else nbytes, _stream(stream)))
    return out


def tdes_ecb_decrypt(ks: KeySchedule, inp, out=None, stream=None, nbytes=None):
    out, n = _io(inp, out)
    _check(load().tdes_ecb_decrypt(ks.handle, _ptr(inp), _ptr(out),
                                   n if nbytes is None else nbytes, _stream(stream)))
    return out


def tdes_ctr_crypt(ks: KeySchedule, nonce: int, ctr0: int, inp, out=None, stream=None,
                   nbytes=None):
    out, n = _io(inp, out)
    _check(load().tdes_ctr_crypt(ks.handle, nonce & 0xFFFFFFFF, ctr0 & 0xFFFFFFFF, _ptr(inp),
                                 _ptr(out), n if nbytes is None else nbytes, _stream(stream)))
    return out


def tdes_cbc_decrypt(ks: KeySchedule, iv: int, inp, out=None, stream=None, nbytes=None):
    out, n = _io(inp, out)
    _check(load().tdes_cbc_decrypt(ks.handle, iv & (2**64 - 1), _ptr(inp), _ptr(out),
                                   n if nbytes is None else nbytes, _stream(stream)))
    return out


def tdes_cbc_encrypt(ks: KeySchedule, iv: int, inp, out=None, stream=None, nbytes=None):
    out, n = _io(inp, out)
    _check(load().tdes_cbc_encrypt(ks.handle, iv & (2**64 - 1), _ptr(inp), _ptr(out),
                                   n if nbytes is None else nbytes, _stream(stream)))
    return out


def tdes_cbc_decrypt_noalloc(ks: KeySchedule, iv: int, inp, out=None, stream=None, nbytes=None):
    """CBC decryption that makes the library allocate nothing (see include/tdes.h).

    For callers that cannot let a library allocate device memory, e.g. a
    server whose memory pool owns the GPU.  In-place calls keep their scratch
    in a fixed 1 MiB array inside the library (limit TDES_NOALLOC_MAX_BYTES);
    in-place calls that overlap in time on the GPU race on that array.
    """
    out, n = _io(inp, out)
    _check(load().tdes_cbc_decrypt_noalloc(ks.handle, iv & (2**64 - 1), _ptr(inp), _ptr(out),
                                           n if nbytes is None else nbytes, _stream(stream)))
    return out


TDES_NOALLOC_MAX_BYTES = 131072 * 8192


def tdes_ecb_crypt_host(ks: KeySchedule, decrypt: bool, host_in, host_out, dev_buf,
                        nbytes=None):
    """Host buffers in and out (numpy arrays or CPU tensors, ideally pinned)."""
    n = _nbytes(host_in) if nbytes is None else nbytes
    _check(load().tdes_ecb_crypt_host(ks.handle, int(bool(decrypt)), _ptr(host_in),
                                      _ptr(host_out), n, _ptr(dev_buf), _nbytes(dev_buf)))
    return host_out


class KeyTable:
    """Owns a tdes_keytable_t: device-resident schedules of many key triples."""

    def __init__(self, keys):
        k = np.ascontiguousarray(np.asarray(keys, dtype=np.uint8).reshape(-1, 24))
        h = ctypes.c_void_p()
        _check(load().tdes_keytable_create(k.ctypes.data, k.shape[0], ctypes.byref(h)))
        self.handle = h.value
        self.count = k.shape[0]

    def free(self):
        if self.handle:
            load().tdes_keytable_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def make_descs(entries):
    """entries: iterable of (mode, key_index, iv_or_ctr, in_ptr, out_ptr, nbytes)."""
    entries = list(entries)
    arr = (Desc * max(1, len(entries)))()
    for i, (mode, key, iv, ip, op, n) in enumerate(entries):
        arr[i] = Desc(mode, key, iv & (2**64 - 1), _ptr(ip), _ptr(op), n)
    return arr, len(entries)


DESC_DTYPE = np.dtype([("mode", "<u4"), ("key_index", "<u4"), ("iv_or_ctr", "<u8"),
                       ("in_ptr", "<u8"), ("out_ptr", "<u8"), ("nbytes", "<u8")])


class Batch:
    """Owns a tdes_batch_t planned from descriptors (see include/tdes.h).

    ``entries`` is an iterable of (mode, key_index, iv_or_ctr, in, out, nbytes)
    or a numpy array of DESC_DTYPE (for very large batches).
    """

    def __init__(self, kt: KeyTable, entries):
        if isinstance(entries, np.ndarray):
            descs = np.ascontiguousarray(entries, dtype=DESC_DTYPE)
            n, addr = descs.shape[0], descs.ctypes.data
        else:
            descs, n = make_descs(entries)
            addr = ctypes.addressof(descs)
        self._descs = descs
        self.status = np.zeros(max(1, n), dtype=np.int32)
        h = ctypes.c_void_p()
        _check(load().tdes_batch_plan(kt.handle, addr, n, self.status.ctypes.data,
                                      ctypes.byref(h)))
        self.status = self.status[:n]
        self.handle = h.value
        self.kt = kt

    def configure(self, warps_per_cta: int, ctas_per_sm: int = 0):
        _check(load().tdes_batch_configure(self.handle, warps_per_cta, ctas_per_sm))

    def launch(self, stream=None):
        _check(load().tdes_batch_launch(self.handle, _stream(stream)))

    def launch_graph(self, stream=None):
        _check(load().tdes_batch_launch_graph(self.handle, _stream(stream)))

    def info(self) -> dict:
        bi = BatchInfo()
        _check(load().tdes_batch_info(self.handle, ctypes.byref(bi)))
        return {"n_cbc_enc_messages": bi.n_cbc_enc_messages, "n_tiles": bi.n_tiles,
                "n_small_items": bi.n_small_items, "warps_per_cta": bi.warps_per_cta,
                "ctas_per_sm": bi.ctas_per_sm, "bytes_per_mode": list(bi.bytes_per_mode),
                "n_mixed_tiles": bi.n_mixed_tiles, "n_direct_messages": bi.n_direct_messages,
                "tiles_per_claim": bi.tiles_per_claim, "round_form": bi.round_form,
                "tuned": bool(bi.tuned)}

    def set_shape(self, warps_per_cta: int, ctas_per_sm: int = 0, tiles_per_claim: int = 0,
                  round_form: int = ROUNDS_PER_PASS):
        sh = LaunchShape(warps_per_cta, ctas_per_sm, tiles_per_claim, round_form)
        _check(load().tdes_batch_set_shape(self.handle, ctypes.byref(sh)))

    def shape(self) -> dict:
        sh = LaunchShape()
        _check(load().tdes_batch_get_shape(self.handle, ctypes.byref(sh)))
        return sh.as_dict()

    def autotune(self, reps: int = 5, flags: int = 0, stream=None) -> dict:
        """tdes_batch_autotune: runs the batch's whole work repeatedly (its
        outputs are rewritten each time)."""
        r = AutotuneResult()
        _check(load().tdes_batch_autotune(self.handle, flags, reps, _stream(stream),
                                          ctypes.byref(r)))
        return {"key": r.key.decode(), "best": r.best.as_dict(), "baseline": r.baseline.as_dict(),
                "best_ms": r.best_ms, "baseline_ms": r.baseline_ms, "candidates": r.candidates,
                "from_cache": bool(r.from_cache)}

    def free(self):
        if self.handle:
            load().tdes_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tdes_autotune_cache_path() -> str:
    return load().tdes_autotune_cache_path().decode()


class Ctx:
    """Owns a tdes_ctx_t: batches submitted with a ticket, polled per
    descriptor and waited on with a time limit (tdes_batch_submit / poll /
    wait / release).

    The device reads a ticket's buffers and plan after submit returns, so
    the context keeps the tensors given as entries' in/out and the Batch of
    submit_plan referenced until the ticket is released or the context is
    closed.  Raw integer addresses are the caller's to keep valid."""

    def __init__(self, kt: KeyTable, streams: int = 2):
        lib = load()
        cfg = CtxConfig()
        lib.tdes_ctx_config_default(ctypes.byref(cfg))
        cfg.streams = streams
        h = ctypes.c_void_p()
        _check(lib.tdes_ctx_create(kt.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self.kt = kt
        self._counts = {}
        self._keep = {}  # ticket -> objects the device may still read

    def submit(self, entries) -> int:
        """entries: (mode, key_index, iv_or_ctr, in, out, nbytes) each, or a
        DESC_DTYPE array; returns the ticket."""
        keep = []
        if isinstance(entries, np.ndarray):
            descs = np.ascontiguousarray(entries, dtype=DESC_DTYPE)
            n, addr = descs.shape[0], descs.ctypes.data
        else:
            entries = list(entries)
            keep = [b for e in entries for b in (e[3], e[4]) if not isinstance(b, int)]
            descs, n = make_descs(entries)
            addr = ctypes.addressof(descs)
        t = ctypes.c_uint64()
        _check(load().tdes_batch_submit(self.handle, addr, n, ctypes.byref(t)))
        self._counts[t.value] = n
        if keep:
            self._keep[t.value] = keep
        return t.value

    def submit_plan(self, batch: "Batch") -> int:
        t = ctypes.c_uint64()
        _check(load().tdes_batch_submit_plan(self.handle, batch.handle, ctypes.byref(t)))
        self._counts[t.value] = len(batch.status)
        self._keep[t.value] = [batch]
        return t.value

    def poll(self, ticket: int, count: int | None = None) -> tuple:
        """(status, per-descriptor statuses) of a ticket."""
        n = self._counts.get(ticket, 0) if count is None else count
        st = np.zeros(max(1, n), dtype=np.int32)
        r = int(load().tdes_batch_poll(self.handle, ticket, st.ctypes.data if n else None))
        return r, st[:n]

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        return int(load().tdes_batch_wait(self.handle, ticket, int(timeout_s * 1e9)))

    def release(self, ticket: int) -> int:
        r = int(load().tdes_batch_release(self.handle, ticket))
        if r == TDES_OK:
            self._counts.pop(ticket, None)
            self._keep.pop(ticket, None)
        return r

    def close(self):
        if self.handle:
            load().tdes_ctx_destroy(self.handle)  # waits for the context's streams
            self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tdes_uniform_scratch_bytes(kt: KeyTable, n_msgs: int, msg_bytes: int) -> int:
    n = ctypes.c_size_t()
    _check(load().tdes_uniform_scratch_bytes(kt.handle, n_msgs, msg_bytes, ctypes.byref(n)))
    return n.value


def tdes_uniform_crypt(kt: KeyTable, key_index, mode, iv_or_ctr, inp, out, msg_bytes: int,
                       scratch=None, skipped=None, stream=None, n_msgs=None):
    """Messages of msg_bytes back to back in ``inp`` (device tensors; in place
    when ``out is inp``); key_index (int32/uint32), mode (uint8) and iv_or_ctr
    (int64/uint64) are device tensors of one entry per message.  ``scratch``
    (a uint8 CUDA tensor of tdes_uniform_scratch_bytes) is allocated when
    None; ``skipped`` (an int64 CUDA tensor of one element) receives the
    number of skipped messages.  Returns the scratch tensor (it holds the plan
    that tdes_uniform_info reads)."""
    if n_msgs is None:
        n_msgs = key_index.numel()
    if mode.numel() < n_msgs or iv_or_ctr.numel() < n_msgs:
        raise ValueError("mode and iv_or_ctr need one entry per message")
    if _nbytes(inp) < n_msgs * msg_bytes or _nbytes(out) < n_msgs * msg_bytes:
        raise ValueError("buffers shorter than n_msgs * msg_bytes")
    need = tdes_uniform_scratch_bytes(kt, n_msgs, msg_bytes)
    if scratch is None:
        import torch
        scratch = torch.empty(need + 256, dtype=torch.uint8, device=inp.device)
        off = (-scratch.data_ptr()) % 256
        scratch = scratch[off:off + need]
    _check(load().tdes_uniform_crypt(kt.handle, _ptr(key_index), _ptr(mode), _ptr(iv_or_ctr),
                                     _ptr(inp), _ptr(out), msg_bytes, n_msgs, _ptr(scratch),
                                     _nbytes(scratch), _ptr(skipped), _stream(stream)))
    return scratch


def tdes_uniform_info(scratch) -> dict:
    ui = UniformInfo()
    _check(load().tdes_uniform_info(_ptr(scratch), ctypes.byref(ui)))
    return {"skipped": ui.skipped, "key_tiles": ui.key_tiles, "mixed_slices": ui.mixed_slices,
            "chain_key_tiles": ui.chain_key_tiles, "chain_slices": ui.chain_slices}


def loadtest_config(kt, in_pool, out_pool, n_requests, offered_gbps, seed=1, small_frac=0.8,
                    small=(64, 4096), large=(64 << 10, 16 << 20), mode_probs=(1, 1, 1),
                    n_keys=None) -> LoadtestConfig:
    return LoadtestConfig(n_requests, offered_gbps, seed, small_frac, small[0], small[1],
                          large[0], large[1], (ctypes.c_double * 3)(*mode_probs),
                          kt.count if n_keys is None else n_keys, _ptr(in_pool),
                          _nbytes(in_pool), _ptr(out_pool), _nbytes(out_pool))


def tdes_server_autotune(kt, in_pool, out_pool, n_requests, flags=0, **mix) -> dict:
    """tdes_server_autotune over closed-loop load tests of the given request
    mix (the keyword arguments of Server.loadtest)."""
    c = loadtest_config(kt, in_pool, out_pool, n_requests, 0.0, **mix)
    r = ServerAutotuneResult()
    _check(load().tdes_server_autotune(kt.handle, ctypes.byref(c), flags, ctypes.byref(r)))
    cfg = lambda x: {f: getattr(x, f) for f, _ in ServerConfig._fields_}  # noqa: E731
    return {"key": r.key.decode(), "best": cfg(r.best), "baseline": cfg(r.baseline),
            "best_gbps": r.best_gbps, "baseline_gbps": r.baseline_gbps,
            "best_p99_ms": r.best_p99_ms, "baseline_p99_ms": r.baseline_p99_ms,
            "load_gbps": r.load_gbps, "candidates": r.candidates,
            "from_cache": bool(r.from_cache)}


class Server:
    """Owns a tdes_server_t (continuous-batching request server).

    Tensors given as a request's in/out stay referenced until a poll or wait
    reports the request finished (or the server is closed), so the torch
    allocator does not hand them out while the device still uses them."""

    def __init__(self, kt: KeyTable, **config):
        lib = load()
        cfg = ServerConfig()
        lib.tdes_server_config_default(ctypes.byref(cfg))
        for k, v in config.items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        _check(lib.tdes_server_create(kt.handle, ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self.kt = kt
        self.config = {f: getattr(cfg, f) for f, _ in ServerConfig._fields_}
        self._keep = {}  # first ticket -> (request count, tensors the device may still use)
        self._submits = 0

    def _hold(self, ticket: int, count: int, objs):
        objs = [o for o in objs if not isinstance(o, int)]
        if objs:
            self._keep[ticket] = (count, objs)
        self._submits += 1
        if self._submits % 1024 == 0:  # callers that never poll: drop finished requests
            for t, (c, _) in list(self._keep.items()):
                if int(load().tdes_server_poll_group(self.handle, t, c, None)) != 1:
                    del self._keep[t]

    def submit(self, mode, key_index, iv_or_ctr, inp, out, nbytes=None) -> int:
        n = _nbytes(inp) if nbytes is None else nbytes
        d = Desc(mode, key_index, iv_or_ctr & (2**64 - 1), _ptr(inp), _ptr(out), n)
        t = ctypes.c_uint64()
        _check(load().tdes_server_submit(self.handle, ctypes.byref(d), ctypes.byref(t)))
        self._hold(t.value, 1, (inp, out))
        return t.value

    def poll(self, ticket: int) -> int:
        r = int(load().tdes_server_poll(self.handle, ticket))
        if r != 1:
            self._keep.pop(ticket, None)
        return r

    def wait(self, ticket: int, timeout_s: float = 60.0) -> int:
        r = int(load().tdes_server_wait(self.handle, ticket, int(timeout_s * 1e9)))
        if r not in (1, TDES_ETIMEDOUT):
            self._keep.pop(ticket, None)
        return r

    def submit_group(self, entries) -> tuple:
        """entries: (mode, key_index, iv_or_ctr, in, out, nbytes) each; returns
        (ticket, count) of the group."""
        entries = list(entries)
        arr, n = make_descs(entries)
        t = ctypes.c_uint64()
        _check(load().tdes_server_submit_group(self.handle, ctypes.addressof(arr), n,
                                               ctypes.byref(t)))
        self._hold(t.value, n, [b for e in entries for b in (e[3], e[4])])
        return t.value, n

    def poll_group(self, group) -> tuple:
        """(group status, per-request statuses) of a (ticket, count) group."""
        ticket, n = group
        st = np.zeros(n, dtype=np.int32)
        r = int(load().tdes_server_poll_group(self.handle, ticket, n, st.ctypes.data))
        if r != 1:
            self._keep.pop(ticket, None)
        return r, st

    def wait_group(self, group, timeout_s: float = 60.0) -> int:
        ticket, n = group
        r = int(load().tdes_server_wait_group(self.handle, ticket, n, int(timeout_s * 1e9)))
        if r not in (1, TDES_ETIMEDOUT):
            self._keep.pop(ticket, None)
        return r

    def loadtest(self, in_pool, out_pool, n_requests, offered_gbps, seed=1, small_frac=0.8,
                 small=(64, 4096), large=(64 << 10, 16 << 20), mode_probs=(1, 1, 1),
                 n_keys=None) -> dict:
        c = loadtest_config(self.kt, in_pool, out_pool, n_requests, offered_gbps, seed,
                            small_frac, small, large, mode_probs, n_keys)
        r = LoadtestResult()
        _check(load().tdes_serve_loadtest(self.handle, ctypes.byref(c), ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in LoadtestResult._fields_}

    def stats(self, reset: bool = False) -> dict:
        st = ServerStats()
        _check(load().tdes_server_stats(self.handle, int(bool(reset)), ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self.handle:
            load().tdes_server_destroy(self.handle)  # drains the queue and the device work
            self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tdes_sbox_gate_count() -> int:
    return int(load().tdes_sbox_gate_count())


def tdes_set_small_cutoff(nblocks: int) -> int:
    """Calls of at most `nblocks` blocks run one block per thread
    (tdes_set_small_cutoff); returns the previous cutoff."""
    return int(load().tdes_set_small_cutoff(int(nblocks)))


class small_cutoff:
    """Context manager: run calls with the given small-call cutoff, then
    restore the previous one (0: always bitsliced)."""

    def __init__(self, nblocks: int):
        self.nblocks = nblocks

    def __enter__(self):
        self.prev = tdes_set_small_cutoff(self.nblocks)
        return self

    def __exit__(self, *exc):
        tdes_set_small_cutoff(self.prev)
        return False


def tdes_strerror(status: int) -> str:
    return load().tdes_strerror(status).decode()
