"""ctypes binding of libvfunc (include/vfunc.h): same entry-point names,
argument marshalling only. Accepts torch tensors (CUDA or CPU) and numpy
arrays; CUDA tensors are passed as device pointers, everything else as host
pointers (the library copies host data itself).

There is no CPU fallback: if libvfunc.so has not been built, every call
raises VFError.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

try:
    import torch
except ImportError:  # pragma: no cover - torch is part of the supported environment
    torch = None

HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(HERE, "libvfunc.so")

FUNC, FILTER = 0, 1
KEYS_U64, KEYS_BYTES = 0, 1
MODE_AUTO, MODE_FUSE, MODE_LGE, MODE_MWHC = 0, 1, 2, 3
REGIME_FUSE, REGIME_LGE, REGIME_MWHC = 1, 2, 3
SOLVER_FLOW, SOLVER_ROUNDS, SOLVER_WAVE = 0, 1, 2
STATUS = {0: "VF_OK", 1: "VF_EINVAL", 2: "VF_ENOMEM", 3: "VF_EBUILD", 4: "VF_EDUP", 5: "VF_ETIMEOUT",
          6: "VF_ECUDA", 7: "VF_ECAPACITY", 8: "VF_EAGAIN", 9: "VF_EIO"}
EAGAIN, EIO = 8, 9


class VFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class VfParams(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("b", C.c_int), ("key_kind", C.c_int), ("mode", C.c_int),
        ("max_retries", C.c_int), ("seed", C.c_uint64), ("eps", C.c_double), ("eta", C.c_double),
        ("lge_threshold", C.c_uint64), ("lge_target", C.c_uint64), ("lge_max_shard", C.c_uint64),
        ("fuse_solver", C.c_int), ("arity", C.c_int),
    ]


class VfInfo(C.Structure):
    _fields_ = [
        ("n", C.c_uint64), ("n_eff", C.c_uint64), ("kind", C.c_int), ("b", C.c_int),
        ("regime", C.c_int), ("h", C.c_int), ("h_bb", C.c_int), ("h_dup", C.c_int),
        ("shards", C.c_uint64), ("M", C.c_uint64), ("c", C.c_double), ("lg_seg", C.c_int),
        ("seg", C.c_uint64), ("l", C.c_uint64), ("T", C.c_uint64), ("cells", C.c_uint64),
        ("total_cells", C.c_uint64), ("data_bytes", C.c_uint64), ("seed", C.c_uint64),
        ("retries", C.c_int), ("peeled", C.c_uint64), ("core", C.c_uint64), ("rounds", C.c_uint64),
        ("k", C.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class VfBatchItem(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("values", C.c_void_p), ("n", C.c_uint64), ("kind", C.c_int),
                ("b", C.c_int), ("seed", C.c_uint64)]


class VfBatchOpts(C.Structure):
    _fields_ = [("lge_threshold", C.c_uint64), ("lge_target", C.c_uint64), ("lpt", C.c_int),
                ("use_graph", C.c_int), ("small_cta_keys", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class VfQueryReq(C.Structure):
    _fields_ = [("s", C.c_void_p), ("keys", C.c_void_p), ("m", C.c_uint64), ("out", C.c_void_p)]


EXPORTS = ["vf_params_default", "vf_build", "vf_query", "vf_get_info", "vf_plan", "vf_data", "vf_export",
           "vf_signatures", "vf_free", "vf_last_error"]

_lib = None


def lib():
    """Load libvfunc.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise VFError(6, f"{lib_path} is missing: build it with paper_2503_18397_gb300.build.build()")
        L = C.CDLL(lib_path)
        vp, u64, i32 = C.c_void_p, C.c_uint64, C.c_int
        L.vf_params_default.argtypes = [C.POINTER(VfParams)]
        L.vf_params_default.restype = None
        L.vf_build.argtypes = [vp, vp, vp, u64, C.POINTER(VfParams), vp, C.POINTER(vp)]
        L.vf_query.argtypes = [vp, vp, vp, u64, vp, vp]
        L.vf_get_info.argtypes = [vp, C.POINTER(VfInfo)]
        L.vf_plan.argtypes = [C.POINTER(VfParams), u64, u64, C.POINTER(VfInfo)]
        L.vf_data.argtypes = [vp, C.POINTER(vp), C.POINTER(u64)]
        L.vf_export.argtypes = [vp, vp]
        L.vf_signatures.argtypes = [i32, vp, vp, u64, u64, vp, vp]
        L.vf_free.argtypes = [vp]
        L.vf_build_static.argtypes = [vp, vp, u64, C.POINTER(VfParams), vp, u64, C.POINTER(VfInfo), vp]
        L.vf_build_static.restype = C.c_int
        L.vf_batch_opts_default.argtypes = [C.POINTER(VfBatchOpts)]
        L.vf_build_batch.argtypes = [C.POINTER(VfBatchItem), C.c_uint32, C.POINTER(VfParams),
                                     C.POINTER(VfBatchOpts), vp, C.POINTER(vp)]
        L.vf_tune_batch.argtypes = [C.POINTER(VfBatchItem), C.c_uint32, C.POINTER(VfParams), vp,
                                    C.POINTER(VfBatchOpts), C.POINTER(C.c_double)]
        for name in ("vf_batch_opts_default", "vf_build_batch", "vf_tune_batch"):
            getattr(L, name).restype = C.c_int
        L.vf_query_batch.argtypes = [C.POINTER(VfQueryReq), C.c_uint32, vp]
        L.vf_query_batch.restype = C.c_int
        L.vf_timing_enable.argtypes = [i32]
        L.vf_timing_read.argtypes = [C.POINTER(C.c_double), C.POINTER(u64)]
        L.vf_sector_rate.argtypes = [u64, vp, C.POINTER(C.c_double)]
        L.vf_build_resumable.argtypes = [vp, vp, vp, u64, C.POINTER(VfParams), C.c_char_p, u64, C.c_uint32, vp,
                                         C.POINTER(vp)]
        L.vf_serialize.argtypes = [vp, vp, u64, C.POINTER(u64)]
        L.vf_deserialize.argtypes = [vp, u64, vp, C.POINTER(vp)]
        L.vf_save.argtypes = [vp, C.c_char_p]
        L.vf_load.argtypes = [C.c_char_p, vp, C.POINTER(vp)]
        for name in ("vf_build_resumable", "vf_serialize", "vf_deserialize", "vf_save", "vf_load"):
            getattr(L, name).restype = C.c_int
        L.vf_last_error.argtypes = []
        L.vf_last_error.restype = C.c_char_p
        L.vf_debug_faults.argtypes = [i32, C.c_uint32, i32]
        for name in ("vf_build", "vf_query", "vf_get_info", "vf_plan", "vf_data", "vf_export", "vf_signatures",
                     "vf_free", "vf_timing_enable", "vf_timing_read", "vf_debug_faults"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(st: int):
    if st != 0:
        raise VFError(st, lib().vf_last_error().decode(errors="replace"))


def _is_tensor(x):
    return torch is not None and isinstance(x, torch.Tensor)


def _ptr(x):
    if x is None:
        return None
    if _is_tensor(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data_as(C.c_void_p)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream, *bufs):
    if stream is not None:
        return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    if torch is not None and any(_is_tensor(b) and b.is_cuda for b in bufs if b is not None):
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


def _len(keys, offsets):
    return (len(offsets) - 1) if offsets is not None else len(keys)


def vf_params_default(**overrides) -> VfParams:
    p = VfParams()
    lib().vf_params_default(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Structure:
    """Owning handle of a built vf_struct (released by vf_free / garbage collection)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        if not self._h:
            raise VFError(1, "structure already freed")
        return self._h

    @property
    def info(self) -> VfInfo:
        return vf_get_info(self)

    def query(self, keys, offsets=None, out=None, stream=None):
        return vf_query(self, keys, offsets=offsets, out=out, stream=stream)

    def free(self):
        if self._h:
            _check(lib().vf_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def vf_build(keys, values=None, *, offsets=None, params: VfParams | None = None, stream=None, **overrides):
    """Build a VFunc (values given) or a VFilter (values None, kind=FILTER)."""
    if params is None:
        params = vf_params_default()
        params.kind = FUNC if values is not None else FILTER
        params.key_kind = KEYS_BYTES if offsets is not None else KEYS_U64
    for k, v in overrides.items():
        setattr(params, k, v)
    n = _len(keys, offsets)
    out = C.c_void_p()
    _check(lib().vf_build(_ptr(keys), _ptr(offsets), _ptr(values), n, C.byref(params),
                          _stream(stream, keys, values, offsets), C.byref(out)))
    return Structure(out.value)


def vf_build_resumable(keys, values=None, *, checkpoint: str, offsets=None, params: VfParams | None = None,
                       group_keys: int = 0, max_groups: int = 0, stream=None, **overrides):
    """vf_build in shard groups checkpointed to `checkpoint`. Returns the Structure
    when complete, or None when max_groups groups were written and the build is
    to be resumed by calling again with the same arguments."""
    if params is None:
        params = vf_params_default()
        params.kind = FUNC if values is not None else FILTER
        params.key_kind = KEYS_BYTES if offsets is not None else KEYS_U64
    for k, v in overrides.items():
        setattr(params, k, v)
    n = _len(keys, offsets)
    out = C.c_void_p()
    st = lib().vf_build_resumable(_ptr(keys), _ptr(offsets), _ptr(values), n, C.byref(params),
                                  os.fsencode(checkpoint), group_keys, max_groups,
                                  _stream(stream, keys, values, offsets), C.byref(out))
    if st == EAGAIN:
        return None
    _check(st)
    return Structure(out.value)


def vf_serialize(s) -> bytes:
    """The serialized form (4096-byte header + data array) as bytes."""
    size = C.c_uint64()
    _check(lib().vf_serialize(s.handle, None, 0, C.byref(size)))
    buf = (C.c_uint8 * size.value)()
    _check(lib().vf_serialize(s.handle, buf, size.value, C.byref(size)))
    return bytes(buf)


def vf_deserialize(data: bytes, stream=None):
    out = C.c_void_p()
    buf = (C.c_uint8 * len(data)).from_buffer_copy(data)
    _check(lib().vf_deserialize(buf, len(data), _stream(stream), C.byref(out)))
    return Structure(out.value)


def vf_save(s, path: str):
    _check(lib().vf_save(s.handle, os.fsencode(path)))


def vf_load(path: str, stream=None):
    out = C.c_void_p()
    _check(lib().vf_load(os.fsencode(path), _stream(stream), C.byref(out)))
    return Structure(out.value)


def _out_dtype(info: VfInfo):
    """Output element type: u8 for filters, else the narrowest type holding b bits."""
    if info.kind == FILTER or info.b <= 8:
        return np.uint8
    return np.uint16 if info.b <= 16 else np.uint32 if info.b <= 32 else np.uint64


def _torch_dtype(dt):
    # 64-bit results come back as int64 tensors holding the bit patterns
    return {np.uint8: torch.uint8, np.uint16: torch.uint16, np.uint32: torch.uint32, np.uint64: torch.int64}[dt]


def vf_query(s: Structure, keys, offsets=None, out=None, stream=None):
    """Query keys; returns `out` (allocated like `keys`: CUDA tensor or numpy)."""
    m = _len(keys, offsets)
    if out is None:
        dt = _out_dtype(vf_get_info(s))
        if _is_tensor(keys):
            tdt = _torch_dtype(dt)
            out = torch.empty(m, dtype=tdt, device=keys.device)
        else:
            out = np.empty(m, dtype=dt)
    _check(lib().vf_query(s.handle, _ptr(keys), _ptr(offsets), m, _ptr(out), _stream(stream, keys, out)))
    return out


def vf_query_batch(requests, stream=None):
    """requests: sequence of (Structure, keys (CUDA u64 tensor), out (CUDA tensor or None)).
    Returns the outputs (allocated when None). One launch for all requests."""
    arr = (VfQueryReq * max(len(requests), 1))()
    outs = []
    for i, (s, keys, out) in enumerate(requests):
        if out is None:
            dt = _out_dtype(vf_get_info(s))
            tdt = _torch_dtype(dt)
            out = torch.empty(len(keys), dtype=tdt, device=keys.device)
        outs.append(out)
        arr[i].s = s.handle
        arr[i].keys = _ptr(keys)
        arr[i].m = len(keys)
        arr[i].out = _ptr(out)
    bufs = [r[1] for r in requests]
    _check(lib().vf_query_batch(arr, len(requests), _stream(stream, *bufs)))
    return outs


def vf_get_info(s: Structure) -> VfInfo:
    info = VfInfo()
    _check(lib().vf_get_info(s.handle, C.byref(info)))
    return info


def vf_plan(n: int, M: int, params: VfParams | None = None) -> VfInfo:
    params = params or vf_params_default()
    info = VfInfo()
    _check(lib().vf_plan(C.byref(params), n, M, C.byref(info)))
    return info


def vf_data(s: Structure):
    """(device address, bytes) of a structure's data array (owned by the structure)."""
    ptr, nb = C.c_void_p(), C.c_uint64()
    _check(lib().vf_data(s.handle, C.byref(ptr), C.byref(nb)))
    return ptr.value or 0, nb.value


def vf_export(s: Structure) -> np.ndarray:
    info = vf_get_info(s)
    buf = np.zeros(max(int(info.data_bytes), 1), dtype=np.uint8)
    _check(lib().vf_export(s.handle, _ptr(buf)))
    return buf[: info.data_bytes]


def vf_signatures(keys, seed: int, offsets=None, out=None, stream=None):
    """(n, 2) uint64 signatures (column 0 = high word)."""
    n = _len(keys, offsets)
    if out is None:
        if _is_tensor(keys):
            out = torch.empty((n, 2), dtype=torch.uint64, device=keys.device)
        else:
            out = np.empty((n, 2), dtype=np.uint64)
    kind = KEYS_BYTES if offsets is not None else KEYS_U64
    _check(lib().vf_signatures(kind, _ptr(keys), _ptr(offsets), n, seed, _ptr(out), _stream(stream, keys, out)))
    return out


def vf_build_static(keys, values, data, *, params: VfParams | None = None, stream=None) -> VfInfo:
    """Allocation-free build of <= 16384 u64 keys into the caller's device buffer `data`."""
    if params is None:
        params = vf_params_default()
        params.kind = FUNC if values is not None else FILTER
    info = VfInfo()
    nbytes = data.numel() * data.element_size() if _is_tensor(data) else data.nbytes
    _check(lib().vf_build_static(_ptr(keys), _ptr(values), len(keys), C.byref(params), _ptr(data), nbytes,
                                 C.byref(info), _stream(stream, keys, values, data)))
    return info


def vf_batch_opts_default(**overrides) -> VfBatchOpts:
    o = VfBatchOpts()
    _check(lib().vf_batch_opts_default(C.byref(o)))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def _batch_items(items):
    """items: sequence of (keys, values_or_None, kind, b, seed) with u64 keys."""
    arr = (VfBatchItem * max(len(items), 1))()
    for i, (keys, values, kind, b, seed) in enumerate(items):
        arr[i].keys = _ptr(keys)
        arr[i].values = _ptr(values)
        arr[i].n = len(keys)
        arr[i].kind = kind
        arr[i].b = b
        arr[i].seed = seed
    return arr


def vf_build_batch(items, *, params: VfParams | None = None, opts: VfBatchOpts | None = None, stream=None):
    """Build many structures at once; returns a list of Structure."""
    params = params or vf_params_default()
    arr = _batch_items(items)
    out = (C.c_void_p * max(len(items), 1))()
    bufs = [x for it in items for x in it[:2] if x is not None]
    _check(lib().vf_build_batch(arr, len(items), C.byref(params), None if opts is None else C.byref(opts),
                                _stream(stream, *bufs), out))
    return [Structure(out[i]) for i in range(len(items))]


def vf_tune_batch(items, *, params: VfParams | None = None, stream=None):
    """Autotuned batch options for this batch shape and the sample build time (ms, -1 if cached)."""
    params = params or vf_params_default()
    arr = _batch_items(items)
    best = VfBatchOpts()
    ms = C.c_double()
    bufs = [x for it in items for x in it[:2] if x is not None]
    _check(lib().vf_tune_batch(arr, len(items), C.byref(params), _stream(stream, *bufs), C.byref(best), C.byref(ms)))
    return best, ms.value


def vf_free(s: Structure):
    s.free()


PHASES = ["hash_hist", "scatter", "incidence", "peel", "assign", "lge", "query"]


def vf_timing_enable(on: bool = True):
    _check(lib().vf_timing_enable(1 if on else 0))


def vf_debug_faults(fail_attempts: int = 0, assign_poll_limit: int = 0, stall_assign: bool = False):
    """Fault injection for tests (process-wide; all zero = off)."""
    _check(lib().vf_debug_faults(int(fail_attempts), int(assign_poll_limit), 1 if stall_assign else 0))


def vf_sector_rate(table_bytes: int, stream=None) -> float:
    """Random 32-byte sector reads per second from a table of table_bytes bytes."""
    r = C.c_double()
    _check(lib().vf_sector_rate(table_bytes, _stream(stream), C.byref(r)))
    return r.value


def vf_timing_read() -> dict:
    """{phase: (milliseconds, launches)} accumulated since the last read."""
    ms = (C.c_double * 7)()
    n = (C.c_uint64 * 7)()
    _check(lib().vf_timing_read(ms, n))
    return {p: (ms[i], int(n[i])) for i, p in enumerate(PHASES)}
