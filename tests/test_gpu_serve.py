"""Serving loop: continuous batching of builds and queries under a device-memory
budget. Each result must be the same in the mix as alone: a query returns, byte
for byte, what vf_query returns for the same keys on the same resident
structure, and a structure built in the mix has the geometry, seed and retries
of the same build run alone and decodes every key to its value."""
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


def _np(t):
    m = {torch.uint16: (torch.int16, np.uint16), torch.uint32: (torch.int32, np.uint32)}
    if t.dtype in m:
        return t.view(m[t.dtype][0]).cpu().numpy().view(m[t.dtype][1])
    return t.cpu().numpy()


def _pinned(a):
    if a is None:
        return None
    view = {np.uint64: np.int64, np.uint16: np.int16, np.uint32: np.int32}.get(a.dtype.type)
    t = torch.from_numpy(a.view(view) if view else a)
    return t.pin_memory()


def _workload(nb, nq, seed, rate):
    from paper_2503_18397_gb300 import serve

    rng = np.random.default_rng(seed)
    sizes = synth.log_uniform_sizes(nb, 1e3, 3e5, seed)
    t = 0.0
    reqs, builds = [], {}
    rid = 0
    for i in range(nb):
        t += rng.exponential(1 / rate)
        n = int(sizes[i])
        kind = int(rng.integers(0, 2))
        b = int(rng.choice([8, 16]))
        keys = synth.u64_keys(i * 10**8, n, seed)
        vals = synth.values(n, b, seed + i) if kind == 0 else None
        builds[i] = (keys, vals, kind, b, 500 + i)
        reqs.append(serve.BuildRequest(rid, t, i, _pinned(keys), _pinned(vals), kind, b, 500 + i))
        rid += 1
        for _ in range(nq // nb):
            t += rng.exponential(1 / rate)
            sid = int(rng.integers(0, i + 1))
            m = int(10 ** rng.uniform(3, 5))
            k0 = builds[sid][0]
            members = k0[rng.integers(0, len(k0), size=m // 2)]
            others = synth.u64_keys(10**15 + rid * 10**6, m - m // 2, seed)
            q = np.concatenate([members, others])
            reqs.append(serve.QueryRequest(rid, t, sid, _pinned(q)))
            rid += 1
    return reqs, builds


def test_serving_mix_equals_alone(vf):
    from paper_2503_18397_gb300 import serve

    reqs, builds = _workload(10, 40, 3, rate=400.0)
    srv = serve.Server(budget=96 << 20)  # small budget: builds wait for memory
    try:
        recs = srv.run(reqs)
        assert all(r.done > 0 and r.done >= r.start >= 0 for r in recs.values())
        for r in reqs:
            rec = recs[r.rid]
            if isinstance(r, serve.BuildRequest):
                keys, vals, kind, b, seed = builds[r.sid]
                alone = vf.vf_build(keys, vals, params=vf.vf_params_default(kind=kind, b=b, seed=seed))
                for f in ("regime", "h", "shards", "M", "cells", "data_bytes", "seed", "retries"):
                    assert getattr(rec.result, f) == getattr(alone.info, f), f
                out = srv.resident[r.sid].query(keys)
                assert (out == vals).all() if kind == 0 else out.all()
                alone.free()
            else:
                alone = srv.resident[r.sid].query(r.keys.numpy().view(np.uint64))
                got = _np(rec.result)
                assert got.dtype.itemsize == alone.dtype.itemsize
                assert (got.view(alone.dtype) == alone).all()
        lat = serve.percentiles(recs, "query")
        assert lat["n"] == 40 and lat["p99_ms"] >= lat["p50_ms"] > 0
    finally:
        srv.close()


def test_query_batch_matches_single_queries(vf):
    structs, keysets = [], []
    for i, (n, kind, b) in enumerate([(5000, 0, 8), (70_000, 1, 8), (900_000, 0, 16), (1234, 0, 13)]):
        keys = synth.u64_keys(i * 10**7, n, 17)
        vals = synth.values(n, b, 17 + i) if kind == 0 else None
        structs.append(vf.vf_build(keys, vals, params=vf.vf_params_default(kind=kind, b=b, seed=i)))
        q = np.concatenate([keys[: n // 2], synth.u64_keys(10**12 + i * 10**6, 3000, 17)])
        keysets.append(torch.from_numpy(q.view(np.int64)).cuda())
    outs = vf.vf_query_batch([(s, k, None) for s, k in zip(structs, keysets)])
    torch.cuda.synchronize()
    for s, k, o in zip(structs, keysets, outs):
        single = s.query(k)
        assert o.dtype == single.dtype and (_np(o) == _np(single)).all()
        s.free()
