"""vf_build_static: the allocation-free build entry point.

It serves callers that must not allocate device memory while building (code
whose device memory belongs to its own pool or arena, and latency-sensitive
paths where cudaMalloc/cudaFree could synchronise the device or fail under
memory pressure). Its scratch is one static device array shared by all calls,
so these checks also run several calls back to back: each must give the same
structure geometry as vf_build and decode every key exactly like the
structure vf_build returns.
"""
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


def _dev(a):
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32)
    return torch.from_numpy(a).cuda()


def _host(t):
    m = {torch.uint16: (torch.int16, np.uint16), torch.uint32: (torch.int32, np.uint32)}
    if t.dtype in m:
        return t.view(m[t.dtype][0]).cpu().numpy().view(m[t.dtype][1])
    return t.cpu().numpy()


FIELDS = ("regime", "h", "shards", "M", "c", "cells", "total_cells", "data_bytes", "seed", "retries")


def test_static_build_matches_vf_build_on_consecutive_calls(vf, orc):
    cases = [(12_000, 8, vf.FUNC), (16_384, 16, vf.FUNC), (5_000, 8, vf.FILTER), (777, 1, vf.FUNC),
             (16_384, 32, vf.FUNC)]
    for call, (n, b, kind) in enumerate(cases):
        keys = synth.u64_keys(0, n, 50 + call)
        vals = synth.values(n, b, 50 + call) if kind == vf.FUNC else None
        kd = _dev(keys)
        vd = None if vals is None else _dev(vals)
        params = vf.vf_params_default(kind=kind, b=b, seed=3 + call)
        plan = vf.vf_plan(n, n, params)
        data = torch.full((int(plan.data_bytes),), 0xAB, dtype=torch.uint8, device="cuda")  # stale contents
        info = vf.vf_build_static(kd, vd, data, params=params)
        ref = vf.vf_build(kd, vd, params=params)
        rinfo = ref.info
        for f in FIELDS:
            assert getattr(info, f) == getattr(rinfo, f), (call, f)
        oi = orc.Info()
        for f, _ in orc.Info._fields_:
            setattr(oi, f, getattr(info, f))
        got = orc.query(oi, data.cpu().numpy(), keys)
        want = _host(ref.query(kd))
        assert (got == want).all(), call
        if kind == vf.FUNC:
            assert (got == vals).all()
        else:
            assert got.all()
        ref.free()


def test_static_build_limits(vf):
    keys = _dev(synth.u64_keys(0, 16_385, 1))
    data = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(vf.VFError) as e:
        vf.vf_build_static(keys, None, data, params=vf.vf_params_default(kind=vf.FILTER))
    assert e.value.status == 7  # VF_ECAPACITY
    small = synth.u64_keys(0, 100, 1)
    with pytest.raises(vf.VFError) as e:
        vf.vf_build_static(small, None, data, params=vf.vf_params_default(kind=vf.FILTER))  # host keys
    assert e.value.status == 1
    with pytest.raises(vf.VFError) as e:
        vf.vf_build_static(_dev(small), None, torch.zeros(4, dtype=torch.uint8, device="cuda"),
                           params=vf.vf_params_default(kind=vf.FILTER))  # buffer too small
    assert e.value.status == 1


def _static_struct(vf, ref, data):
    """A structure holding the cells vf_build_static wrote: the serialized form
    of `ref` (same geometry and seed) with its data array replaced by them."""
    buf = vf.vf_serialize(ref)
    head = 4096
    assert len(buf) == head + data.numel()
    return vf.vf_deserialize(buf[:head] + data.cpu().numpy().tobytes())


def test_static_build_queried_by_the_gpu_kernel(vf, orc):
    # the GPU query kernel on cells written by vf_build_static: members and
    # disjoint keys, byte for byte against the oracle's query of the same cells
    for call, (n, b, kind) in enumerate([(9000, 8, vf.FUNC), (4000, 8, vf.FILTER), (16_384, 13, vf.FUNC)]):
        keys = synth.u64_keys(0, n, 70 + call)
        vals = synth.values(n, b, 70 + call) if kind == vf.FUNC else None
        kd = _dev(keys)
        vd = None if vals is None else _dev(vals)
        params = vf.vf_params_default(kind=kind, b=b, seed=11 + call)
        plan = vf.vf_plan(n, n, params)
        data = torch.full((int(plan.data_bytes),), 0x5A, dtype=torch.uint8, device="cuda")
        info = vf.vf_build_static(kd, vd, data, params=params)
        ref = vf.vf_build(kd, vd, params=params)
        assert (ref.info.seed, ref.info.cells) == (info.seed, info.cells)
        st = _static_struct(vf, ref, data)
        ref.free()
        oi = orc.Info()
        for f, _ in orc.Info._fields_:
            setattr(oi, f, getattr(info, f))
        host_data = data.cpu().numpy()
        other = synth.u64_keys(n + 5, 200_000, 70 + call)
        for q in (keys, other):
            got = _host(st.query(_dev(q)))
            want = orc.query(oi, host_data, q)
            assert got.dtype == want.dtype and (got == want).all(), call
        if kind == vf.FILTER:  # false-positive rate ~ 2^-b on disjoint keys (Sec. 3.1)
            fpr = _host(st.query(_dev(other))).mean()
            assert abs(fpr - 2.0 ** -b) < 6 * (2.0 ** -b / len(other)) ** 0.5
        else:
            assert (_host(st.query(kd)) == vals).all()
        st.free()


def test_static_build_retries_reuse_the_scratch(vf, orc):
    # (1) a real unsolvable first attempt: 40 keys, b = 2, seeds the oracle must
    # retry; (2) attempts failed by the vf_debug_faults hook. After either, a
    # normal call on the same scratch still decodes every key.
    n, b = 40, 2
    found = 0
    for seed in range(200):
        keys = synth.u64_keys(0, n, 1000 + seed)
        vals = synth.values(n, b, 1000 + seed)
        st, oi, _ = orc.build(orc.default_params(b=b, seed=seed, max_retries=30), keys, vals)
        if st != orc.OK or oi.retries == 0:
            continue
        data = torch.full((int(oi.data_bytes),), 0xFF, dtype=torch.uint8, device="cuda")
        info = vf.vf_build_static(_dev(keys), _dev(vals), data, params=vf.vf_params_default(b=b, seed=seed,
                                                                                               max_retries=30))
        assert (info.seed, info.retries, info.cells) == (oi.seed, oi.retries, oi.cells)
        oinfo = orc.Info()
        for f, _ in orc.Info._fields_:
            setattr(oinfo, f, getattr(info, f))
        assert (orc.query(oinfo, data.cpu().numpy(), keys) == vals).all()
        found += 1
        if found == 3:
            break
    assert found > 0
    keys = synth.u64_keys(0, 7000, 81)
    vals = synth.values(7000, 16, 81)
    kd, vd = _dev(keys), _dev(vals)
    params = vf.vf_params_default(b=16, seed=9, max_retries=4)
    plan = vf.vf_plan(7000, 7000, params)
    data = torch.zeros(int(plan.data_bytes), dtype=torch.uint8, device="cuda")
    vf.vf_debug_faults(3)
    try:
        info = vf.vf_build_static(kd, vd, data, params=params)
        ref = vf.vf_build(kd, vd, params=params)
        assert info.retries == ref.info.retries == 3 and info.seed == ref.info.seed == 12
        ref.free()
        with pytest.raises(vf.VFError) as e:
            vf.vf_build_static(kd, vd, data, params=vf.vf_params_default(b=16, seed=9, max_retries=2))
        assert e.value.status == 3  # VF_EBUILD: every attempt failed
    finally:
        vf.vf_debug_faults(0)
    info = vf.vf_build_static(kd, vd, data, params=params)
    assert info.retries == 0
    oinfo = orc.Info()
    for f, _ in orc.Info._fields_:
        setattr(oinfo, f, getattr(info, f))
    assert (orc.query(oinfo, data.cpu().numpy(), keys) == vals).all()


def test_static_build_duplicate_keys(vf, orc):
    # repeated (key, value) pairs are kept once; a key with two values is VF_EDUP
    keys = synth.u64_keys(0, 5000, 91)
    vals = synth.values(5000, 8, 91)
    dk = np.concatenate([keys, keys[:300]])
    dv = np.concatenate([vals, vals[:300]])
    params = vf.vf_params_default(b=8, seed=4)
    plan = vf.vf_plan(len(dk), len(dk), params)
    data = torch.zeros(int(plan.data_bytes), dtype=torch.uint8, device="cuda")
    info = vf.vf_build_static(_dev(dk), _dev(dv), data, params=params)
    st, oi, _ = orc.build(orc.default_params(b=8, seed=4), dk, dv)
    assert st == orc.OK and info.n_eff == oi.n_eff == 5000 and (info.seed, info.retries) == (oi.seed, oi.retries)
    oinfo = orc.Info()
    for f, _ in orc.Info._fields_:
        setattr(oinfo, f, getattr(info, f))
    assert (orc.query(oinfo, data.cpu().numpy(), dk) == dv).all()
    dv[-1] ^= 1
    with pytest.raises(vf.VFError) as e:
        vf.vf_build_static(_dev(dk), _dev(dv), data, params=params)
    assert e.value.status == 4
