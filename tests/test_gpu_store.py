"""Serialized form and resumable (shard-group checkpointed) builds.

A structure survives serialize -> deserialize and save -> load with the same
info and the same answers; the file is the 4096-byte header followed by the
data array in its device layout. A build resumed from its checkpoint one
shard group at a time ends as vf_build does: same geometry, seed, retries and
n_eff as the oracle's build, every key decodes (the data array may differ
where the peel order does)."""
import numpy as np
import pytest

from paper_2503_18397_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18397_gb300 import build

    build.build()
    import paper_2503_18397_gb300 as vf

    vf.lib()
    return vf


def dev(a):
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32)
    return torch.from_numpy(a).cuda()


def host(t):
    m = {torch.uint16: (torch.int16, np.uint16), torch.uint32: (torch.int32, np.uint32)}
    if t.dtype in m:
        return t.view(m[t.dtype][0]).cpu().numpy().view(m[t.dtype][1])
    return t.cpu().numpy()


INFO = ("n", "n_eff", "kind", "b", "regime", "h", "h_bb", "h_dup", "shards", "M", "c", "lg_seg", "seg", "l", "T",
        "cells", "total_cells", "data_bytes", "seed", "retries", "peeled", "core", "rounds")


@pytest.mark.parametrize("case", ["fuse_func_b8", "lge_filter_b13", "mwhc_func_b32", "fuse_filter_b1"])
def test_round_trip(vf, tmp_path, case):
    n = {"fuse_func_b8": 1_200_000, "lge_filter_b13": 50_000, "mwhc_func_b32": 300_000,
         "fuse_filter_b1": 900_000}[case]
    b = int(case.split("_b")[1])
    kind = vf.FUNC if "func" in case else vf.FILTER
    keys = synth.u64_keys(0, n, 51)
    vals = synth.values(n, b, 51) if kind == vf.FUNC else None
    extra = {"mode": vf.MODE_MWHC, "eps": 0.01, "eta": 1e-3} if "mwhc" in case else {}
    p = vf.vf_params_default(kind=kind, b=b, seed=4, **extra)
    s = vf.vf_build(dev(keys), None if vals is None else dev(vals), params=p)
    blob = vf.vf_serialize(s)
    info = s.info
    assert blob[:8] == b"VFSTORE1" and len(blob) == 4096 + info.data_bytes
    assert np.array_equal(np.frombuffer(blob[4096:], np.uint8), vf.vf_export(s))
    other = synth.u64_keys(n, 100_000, 51)
    want = (host(s.query(dev(keys))), host(s.query(dev(other))))
    path = str(tmp_path / "s.vf")
    vf.vf_save(s, path)
    with open(path, "rb") as f:
        assert f.read() == blob
    for t in (vf.vf_deserialize(blob), vf.vf_load(path)):
        for f in INFO:
            assert getattr(t.info, f) == getattr(info, f), f
        got = (host(t.query(dev(keys))), host(t.query(dev(other))))
        assert all(np.array_equal(x, y) for x, y in zip(got, want))
        t.free()
    # a corrupt header (changed geometry) is rejected
    bad = bytearray(blob)
    bad[64 + 16 + 24] ^= 1  # shards
    with pytest.raises(vf.VFError) as e:
        vf.vf_deserialize(bytes(bad))
    assert e.value.status == vf.EIO


def _oracle_fields(orc, keys, vals, **kw):
    st, oi, _ = orc.build(orc.default_params(**kw), keys, vals)
    assert st == orc.OK
    return oi


@pytest.mark.parametrize("kind,mode", [(0, 1), (1, 3)], ids=["fuse_func", "mwhc_filter"])
def test_resumable_build_one_group_per_call(vf, orc, tmp_path, kind, mode):
    # 16 shards, groups of two shards -> 8 groups, one written per call. Fuse:
    # 16M keys (1M-key shards peel; eps/eta set for h = 4); MWHC: 3M keys with the
    # paper's eps/eta
    n = 16_000_000 if mode == 1 else 3_000_000
    keys = synth.u64_keys(0, n, 52)
    vals = synth.values(n, 8, 52) if kind == 0 else None
    kw = dict(kind=kind, b=8, eps=0.003 if mode == 1 else 0.01, eta=0.5 if mode == 1 else 1e-3, mode=mode, seed=7)
    p = vf.vf_params_default(**kw)
    path = str(tmp_path / "ck.vf")
    kd, vd = dev(keys), None if vals is None else dev(vals)
    calls, s = 0, None
    while s is None:
        s = vf.vf_build_resumable(kd, vd, checkpoint=path, params=p, group_keys=n // 7, max_groups=1)
        calls += 1
        assert calls < 100
    info = s.info
    assert info.shards == 16 and calls >= 8  # every call after the first resumed the file
    oi = _oracle_fields(orc, keys, vals, **kw)
    for f in ("regime", "h", "shards", "M", "c", "lg_seg", "seg", "l", "T", "cells", "total_cells", "data_bytes",
              "seed", "retries", "n_eff"):
        assert getattr(info, f) == getattr(oi, f), f
    out = host(s.query(kd))
    assert (out == vals).all() if kind == 0 else out.all()
    # the finished checkpoint is the serialized structure
    t = vf.vf_load(path)
    assert np.array_equal(vf.vf_export(t), vf.vf_export(s))
    assert np.array_equal(host(t.query(kd)), out)


def test_resume_restarts_on_other_parameters(vf, tmp_path):
    n = 2_000_000
    keys = synth.u64_keys(0, n, 53)
    kd = dev(keys)
    path = str(tmp_path / "ck.vf")
    pa = vf.vf_params_default(kind=vf.FILTER, b=8, eps=0.01, eta=1e-3, mode=vf.MODE_MWHC, seed=1)
    assert vf.vf_build_resumable(kd, None, checkpoint=path, params=pa, group_keys=300_000, max_groups=2) is None
    # other seed: the file belongs to another build and starts again
    pb = vf.vf_params_default(kind=vf.FILTER, b=8, eps=0.01, eta=1e-3, mode=vf.MODE_MWHC, seed=2)
    s = vf.vf_build_resumable(kd, None, checkpoint=path, params=pb, group_keys=300_000)
    assert s.info.shards == 16 and s.info.seed == 2 + s.info.retries and host(s.query(kd)).all()
    ref = vf.vf_build(kd, None, params=pb)
    for f in ("h", "shards", "M", "cells", "seed", "retries", "n_eff"):
        assert getattr(s.info, f) == getattr(ref.info, f), f
    # whole build in one call, and the LGE regime (a single group)
    small = synth.u64_keys(0, 60_000, 54)
    s2 = vf.vf_build_resumable(dev(small), None, checkpoint=str(tmp_path / "lge.vf"),
                               params=vf.vf_params_default(kind=vf.FILTER, b=8, seed=3))
    assert s2.info.regime == vf.REGIME_LGE and host(s2.query(dev(small))).all()
