"""ctypes front-end of the plain C oracle (vf_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg. The product package never imports it.

``build_oracle()`` compiles ``liboracle.so`` next to this file with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC = os.path.join(HERE, "vf_oracle.c")

FUNC, FILTER = 0, 1
KEYS_U64, KEYS_BYTES = 0, 1
MODE_AUTO, MODE_FUSE, MODE_LGE, MODE_MWHC = 0, 1, 2, 3
REGIME_FUSE, REGIME_LGE, REGIME_MWHC = 1, 2, 3
OK, EINVAL, ENOMEM, EBUILD, EDUP = 0, 1, 2, 3, 4


class Params(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("b", C.c_int), ("key_kind", C.c_int), ("mode", C.c_int),
        ("max_retries", C.c_int), ("seed", C.c_uint64), ("eps", C.c_double), ("eta", C.c_double),
        ("lge_threshold", C.c_uint64), ("lge_target", C.c_uint64), ("lge_max_shard", C.c_uint64),
        ("threads", C.c_int), ("arity", C.c_int),
    ]


class Info(C.Structure):
    _fields_ = [
        ("n", C.c_uint64), ("n_eff", C.c_uint64), ("kind", C.c_int), ("b", C.c_int),
        ("regime", C.c_int), ("h", C.c_int), ("h_bb", C.c_int), ("h_dup", C.c_int),
        ("shards", C.c_uint64), ("M", C.c_uint64), ("c", C.c_double), ("lg_seg", C.c_int),
        ("seg", C.c_uint64), ("l", C.c_uint64), ("T", C.c_uint64), ("cells", C.c_uint64),
        ("total_cells", C.c_uint64), ("data_bytes", C.c_uint64), ("seed", C.c_uint64),
        ("retries", C.c_int), ("peeled", C.c_uint64), ("core", C.c_uint64), ("k", C.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def build_oracle(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2) if missing or stale."""
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < os.path.getmtime(SRC):
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build_oracle()
        L = C.CDLL(LIB_PATH)
        u64, i32, dbl, vp = C.c_uint64, C.c_int, C.c_double, C.c_void_p
        L.orc_mix64.restype = u64
        L.orc_mix64.argtypes = [u64]
        L.orc_mulhi.restype = u64
        L.orc_mulhi.argtypes = [u64, u64]
        L.orc_lambert_w0.restype = dbl
        L.orc_lambert_w0.argtypes = [dbl]
        L.orc_h_ballsbins.argtypes = [u64, dbl]
        L.orc_h_dupfuse.argtypes = [u64, dbl, dbl]
        L.orc_h_dupmwhc.argtypes = [u64, dbl, dbl]
        L.orc_no_repeat_prob.restype = dbl
        L.orc_no_repeat_prob.argtypes = [dbl, u64]
        L.orc_plan_h.argtypes = [C.POINTER(Params), u64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.orc_geometry.argtypes = [C.POINTER(Info)]
        L.orc_edge.argtypes = [C.POINTER(Info), u64, C.POINTER(u64)]
        L.orc_fingerprint.restype = C.c_uint64
        L.orc_fingerprint.argtypes = [u64, i32]
        L.orc_build.argtypes = [C.POINTER(Params), vp, vp, vp, u64, C.POINTER(Info), C.POINTER(C.c_void_p)]
        L.orc_free.argtypes = [vp]
        L.orc_query.argtypes = [C.POINTER(Info), vp, i32, vp, vp, u64, vp]
        L.orc_query_mt.argtypes = [C.POINTER(Info), vp, i32, vp, vp, u64, vp, i32]
        L.orc_cell_get.restype = C.c_uint64
        L.orc_cell_get.argtypes = [vp, i32, u64]
        L.orc_peel.restype = u64
        L.orc_peel.argtypes = [u64, u64, vp, vp, vp]
        L.orc_gf2_solve.argtypes = [u64, u64, vp, vp, vp]
        L.orc_peel_k.restype = u64
        L.orc_peel_k.argtypes = [u64, u64, i32, vp, vp, vp]
        L.orc_gf2_solve_k.argtypes = [u64, u64, i32, vp, vp, vp]
        L.orc_sigs.argtypes = [i32, vp, vp, u64, u64, vp]
        L.orc_edges_of.argtypes = [C.POINTER(Info), vp, u64, vp]
        L.orc_params_default.argtypes = [C.POINTER(Params)]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def mix64(z: int) -> int:
    return lib().orc_mix64(z)


def sigs(keys, seed: int, offsets=None) -> np.ndarray:
    """(n, 2) uint64 signatures: column 0 = high word, column 1 = low word."""
    keys = np.ascontiguousarray(keys)
    kind = KEYS_U64 if offsets is None else KEYS_BYTES
    n = len(keys) if offsets is None else len(offsets) - 1
    out = np.zeros((n, 2), dtype=np.uint64)
    offs = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.uint64)
    lib().orc_sigs(kind, _ptr(keys), _ptr(offs), n, seed, _ptr(out))
    return out


def plan_h(params: Params, n: int):
    reg, hbb, hdup = C.c_int(), C.c_int(), C.c_int()
    h = lib().orc_plan_h(C.byref(params), n, C.byref(reg), C.byref(hbb), C.byref(hdup))
    return h, reg.value, hbb.value, hdup.value


def geometry(regime: int, h: int, M: int, b: int = 8, kind: int = FUNC, k: int = 3) -> Info:
    info = Info()
    info.regime, info.h, info.shards, info.M, info.b, info.kind, info.k = regime, h, 1 << h, M, b, kind, k
    lib().orc_geometry(C.byref(info))
    return info


def edges_of(info: Info, locals_: np.ndarray) -> np.ndarray:
    locals_ = np.ascontiguousarray(locals_, dtype=np.uint64)
    out = np.zeros((len(locals_), 4 if info.k == 4 else 3), dtype=np.uint64)
    lib().orc_edges_of(C.byref(info), _ptr(locals_), len(locals_), _ptr(out))
    return out


def shard_local(sig: np.ndarray, h: int):
    """Top-h shard index and local signature of (n,2) signatures (vectorised
    restatement used only to feed orc_edges_of in tests)."""
    hi, lo = sig[:, 0], sig[:, 1]
    if h == 0:
        return np.zeros(len(sig), dtype=np.uint64), hi.copy()
    sh = np.uint64(64 - h)
    return hi >> sh, (hi << np.uint64(h)) | (lo >> sh)


def fingerprint(local: int, b: int) -> int:
    return lib().orc_fingerprint(local, b)


def build(params: Params, keys, values=None, offsets=None):
    """Run the oracle build. Returns (status, Info, data bytes as np.uint8 array)."""
    keys = np.ascontiguousarray(keys)
    n = len(keys) if offsets is None else len(offsets) - 1
    offs = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.uint64)
    vals = None if values is None else np.ascontiguousarray(values)
    info = Info()
    dp = C.c_void_p()
    st = lib().orc_build(C.byref(params), _ptr(keys), _ptr(offs), _ptr(vals), n, C.byref(info), C.byref(dp))
    data = None
    if st == OK:
        data = np.ctypeslib.as_array(C.cast(dp, C.POINTER(C.c_uint8)), shape=(max(info.data_bytes, 1),)).copy()
        data = data[: info.data_bytes]
        lib().orc_free(dp)
    return st, info, data


def out_dtype(kind: int, b: int):
    if kind == FILTER:
        return np.uint8
    return np.uint8 if b <= 8 else np.uint16 if b <= 16 else np.uint32 if b <= 32 else np.uint64


def query(info: Info, data: np.ndarray, keys, offsets=None, threads: int = 1) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    m = len(keys) if offsets is None else len(offsets) - 1
    offs = None if offsets is None else np.ascontiguousarray(offsets, dtype=np.uint64)
    out = np.zeros(m, dtype=out_dtype(info.kind, info.b))
    data = np.ascontiguousarray(data, dtype=np.uint8)
    if data.size == 0:
        data = np.zeros(8, dtype=np.uint8)
    kk = KEYS_U64 if offsets is None else KEYS_BYTES
    if threads > 1:
        lib().orc_query_mt(C.byref(info), _ptr(data), kk, _ptr(keys), _ptr(offs), m, _ptr(out), threads)
    else:
        lib().orc_query(C.byref(info), _ptr(data), kk, _ptr(keys), _ptr(offs), m, _ptr(out))
    return out


def peel(V: int, edges: np.ndarray):
    """Stack peel of an (m, k) edge array (k = 3 or 4)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    m = len(edges)
    k = edges.shape[1] if edges.ndim == 2 else 3
    order = np.zeros(max(m, 1), dtype=np.uint32)
    side = np.zeros(max(m, 1), dtype=np.uint8)
    ne = lib().orc_peel_k(V, m, k, _ptr(edges), _ptr(order), _ptr(side))
    return ne, order[:ne], side[:ne]


def gf2_solve(V: int, edges: np.ndarray, rhs: np.ndarray):
    """Plain GF(2) elimination of an (m, k) edge system (k = 3 or 4)."""
    edges = np.ascontiguousarray(edges, dtype=np.uint32)
    rhs = np.ascontiguousarray(rhs, dtype=np.uint64)
    k = edges.shape[1] if edges.ndim == 2 else 3
    w = np.zeros(max(V, 1), dtype=np.uint64)
    ok = lib().orc_gf2_solve_k(V, len(edges), k, _ptr(edges), _ptr(rhs), _ptr(w))
    return bool(ok), w[:V]
