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
