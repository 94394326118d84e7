"""Host-side checks of the C ABI: the library builds for sm_103a, loads,
exports every entry point include/vfunc.h declares, and its parameter
planning (pure host code) agrees with the oracle's."""
import math
import os
import re

import numpy as np
import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def vf():
    from paper_2503_18397_gb300 import build

    build.build()
    import paper_2503_18397_gb300 as vf

    vf.lib()
    return vf


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(vf_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(vf):
    names = declared_functions()
    assert "vf_build" in names and "vf_query" in names
    for name in names:
        assert hasattr(vf.lib(), name), name


def test_params_default_match_paper(vf, orc):
    p = vf.vf_params_default()
    o = orc.default_params()
    for f, _ in vf.VfParams._fields_:
        if f == "fuse_solver":  # a scheduling choice of the CUDA path, not a parameter of the method
            continue
        assert getattr(p, f) == getattr(o, f), f
    assert p.eps == 0.001 and p.lge_threshold == 800000
    assert p.fuse_solver == vf.SOLVER_FLOW


def test_batch_opts_default(vf):
    o = vf.vf_batch_opts_default()
    assert (o.lge_threshold, o.lge_target, o.lpt, o.use_graph, o.small_cta_keys) == (800000, 16384, 1, 1, 7168)


def _plan_pair(vf, orc, n, M, **kw):
    p = vf.vf_params_default(**kw)
    info = vf.vf_plan(n, M, p)
    op = orc.default_params(**kw)
    h, regime, h_bb, h_dup = orc.plan_h(op, n)
    k = 4 if kw.get("arity") == 4 and regime == orc.REGIME_FUSE else 3
    g = orc.geometry(regime, h, M, b=kw.get("b", 8), k=k)
    return info, (h, regime, h_bb, h_dup), g


FIELDS = ["shards", "c", "lg_seg", "seg", "l", "T", "cells", "total_cells", "data_bytes"]


def test_plan_matches_oracle_over_many_sizes(vf, orc):
    rng = np.random.default_rng(0)
    ns = sorted(set([0, 1, 2, 1000, 799_999, 800_000, 2**20, 10**7, 10**8, 5 * 10**9, 10**10, 10**11, 10**12]
                    + [int(10 ** x) for x in rng.uniform(0, 13, 400)]))
    for n in ns:
        for b in (1, 8, 13, 32, 33, 64):
            mean = n / (1 << max(0, 0))
            info, (h, regime, h_bb, h_dup), _ = _plan_pair(vf, orc, n, 1, b=b)
            assert (info.h, info.regime, info.h_bb, info.h_dup) == (h, regime, h_bb, h_dup), n
            M = int(n / (1 << h) + math.sqrt(max(n / (1 << h), 1)) * 3)
            info, _, g = _plan_pair(vf, orc, n, M, b=b)
            for f in FIELDS:
                assert getattr(info, f) == getattr(g, f), (n, b, f)


def test_plan_forced_regimes(vf, orc):
    for mode in (1, 2):
        for n in (10, 5000, 123_456, 10**7):
            info, (h, regime, _, _), g = _plan_pair(vf, orc, n, max(n // 3, 1), mode=mode)
            assert info.h == h and info.regime == regime
            for f in FIELDS:
                assert getattr(info, f) == getattr(g, f)


def test_plan_matches_oracle_mwhc(vf, orc):
    # MWHC mode (Sec. 4.1): shard bits from eq. (logballsbins) and eq. (dupmwhc),
    # 3-partite geometry with c = 1.23, for the paper's eps/eta and the defaults
    rng = np.random.default_rng(1)
    ns = sorted(set([0, 1, 2, 3, 47, 1000, 10**6, 10**8, 10**12] + [int(10 ** x) for x in rng.uniform(0, 13, 200)]))
    for eps, eta in ((0.01, 1e-3), (0.001, 0.1), (0.05, 0.5)):
        for n in ns:
            info, (h, regime, h_bb, h_dup), _ = _plan_pair(vf, orc, n, 1, mode=vf.MODE_MWHC, eps=eps, eta=eta)
            assert info.regime == regime == vf.REGIME_MWHC
            assert (info.h, info.h_bb, info.h_dup) == (h, h_bb, h_dup), (n, eps, eta)
            M = int(n / (1 << h) + math.sqrt(max(n / (1 << h), 1)) * 3)
            info, _, g = _plan_pair(vf, orc, n, M, mode=vf.MODE_MWHC, eps=eps, eta=eta)
            for f in FIELDS:
                assert getattr(info, f) == getattr(g, f), (n, f)
    p = vf.vf_params_default(mode=7)
    with pytest.raises(vf.VFError):
        vf.vf_plan(10, 10, p)


def test_plan_matches_oracle_arity4(vf, orc):
    # 4-uniform fuse graphs: shard bits from eq. (logballsbins) alone, l + 3
    # segments of the arity-4 size; the LGE regime stays 3-uniform
    rng = np.random.default_rng(2)
    ns = sorted(set([0, 1, 2, 1000, 800_000, 10**8, 10**12] + [int(10 ** x) for x in rng.uniform(0, 13, 200)]))
    for n in ns:
        info, (h, regime, h_bb, h_dup), _ = _plan_pair(vf, orc, n, 1, arity=4)
        assert (info.h, info.regime, info.h_bb, info.h_dup) == (h, regime, h_bb, h_dup), n
        M = int(n / (1 << h) + math.sqrt(max(n / (1 << h), 1)) * 3)
        info, _, g = _plan_pair(vf, orc, n, M, arity=4)
        assert info.k == (4 if regime == vf.REGIME_FUSE else 3)
        for f in FIELDS:
            assert getattr(info, f) == getattr(g, f), (n, f)
    with pytest.raises(vf.VFError):
        vf.vf_plan(10, 10, vf.vf_params_default(arity=5))


def test_serialized_form_rejects_foreign_bytes(vf, tmp_path):
    # header validation happens before any device work: garbage, a truncated
    # header and a missing file are VF_EIO, never a half-built structure
    for blob in (b"", b"VFSTORE1", b"\0" * 4096, b"VFSTORE1" + b"\xff" * 5000):
        with pytest.raises(vf.VFError) as e:
            vf.vf_deserialize(blob)
        assert e.value.status == vf.EIO
    with pytest.raises(vf.VFError) as e:
        vf.vf_load(str(tmp_path / "missing.vf"))
    assert e.value.status == vf.EIO
    bad = tmp_path / "bad.vf"
    bad.write_bytes(b"not a structure" * 400)
    with pytest.raises(vf.VFError) as e:
        vf.vf_load(str(bad))
    assert e.value.status == vf.EIO
