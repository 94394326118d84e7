"""Failure paths, exercised without faulting the GPU.

Injected attempt failures (a host-side flag) must retry with the next seeds
exactly as a failed peel or an unsolvable system does; and a wait of the
dataflow assignment that nothing can satisfy (no vertex starts final) must
give up after its poll limit, return VF_ETIMEOUT and leave the CUDA context
usable for the next build."""
import numpy as np
import pytest

from paper_2503_18397_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GEOM = ("regime", "h", "shards", "M", "c", "lg_seg", "seg", "l", "T", "cells", "total_cells", "data_bytes")


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18397_gb300 import build

    build.build()
    import paper_2503_18397_gb300 as vf

    vf.lib()
    yield vf
    vf.vf_debug_faults()


def _dev(a):
    return torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).cuda()


def test_injected_failures_retry_with_the_next_seeds(vf, orc):
    n = 1 << 20  # one fuse shard (regime chosen by size, as for the benchmark's 2^20-key VFunc)
    keys, vals = synth.u64_keys(0, n, 61), synth.values(n, 8, 61)
    p = vf.vf_params_default(kind=vf.FUNC, b=8, seed=11)
    try:
        vf.vf_debug_faults(fail_attempts=2)
        s = vf.vf_build(_dev(keys), _dev(vals), params=p)
    finally:
        vf.vf_debug_faults()
    info = s.info
    st, oi, _ = orc.build(orc.default_params(kind=orc.FUNC, b=8, seed=13), keys, vals)
    assert st == orc.OK and oi.retries == 0  # seed 13 succeeds on its own
    assert (info.seed, info.retries, info.regime) == (13, 2, vf.REGIME_FUSE)
    for f in GEOM:
        assert getattr(info, f) == getattr(oi, f), f
    assert (s.query(_dev(keys)).cpu().numpy() == vals).all()
    s.free()
    # more injected failures than retries: the build gives up like any other
    try:
        vf.vf_debug_faults(fail_attempts=3)
        with pytest.raises(vf.VFError) as ei:
            vf.vf_build(_dev(keys), _dev(vals), params=vf.vf_params_default(kind=vf.FUNC, b=8, seed=11,
                                                                            max_retries=2))
        assert ei.value.status == 3  # VF_EBUILD
    finally:
        vf.vf_debug_faults()


def test_assignment_wait_runs_out_and_the_context_stays_usable(vf):
    n = 1 << 20  # one fuse shard: the flow solver and its dataflow assignment
    keys, vals = synth.u64_keys(0, n, 62), synth.values(n, 8, 62)
    p = vf.vf_params_default(kind=vf.FUNC, b=8, seed=5, fuse_solver=vf.SOLVER_FLOW)
    try:
        vf.vf_debug_faults(assign_poll_limit=4096, stall_assign=True)
        with pytest.raises(vf.VFError) as ei:
            vf.vf_build(_dev(keys), _dev(vals), params=p)
        assert ei.value.status == 5  # VF_ETIMEOUT
    finally:
        vf.vf_debug_faults()
    # the same build right after, on the same context
    s = vf.vf_build(_dev(keys), _dev(vals), params=p)
    assert (s.query(_dev(keys)).cpu().numpy() == vals).all()
    s.free()
    torch.cuda.synchronize()
