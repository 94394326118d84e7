"""Serving loop: continuous batching of builds and queries under a device-memory
budget. Each result must be the same in the mix as alone: a query returns, byte
for byte, what vf_query returns for the same keys on the same resident
structure, and a structure built in the mix has the geometry, seed and retries
of the same build run alone and decodes every key to its value. Both are also
checked against the CPU oracle: builds against the oracle's build of the same
keys, served and batched queries against the oracle's query on the exported
data array."""
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


def _oinfo(orc, info):
    oi = orc.Info()
    for f, _ in orc.Info._fields_:
        setattr(oi, f, getattr(info, f))
    return oi


def _host64(t):
    """Host copy of a query output; 64-bit results (int64 tensors) as uint64."""
    if t.dtype == torch.int64:
        return t.cpu().numpy().view(np.uint64)
    return _np(t)


def test_serving_results_equal_the_oracle(vf, orc):
    # every structure built in the mix equals the oracle's build of its keys
    # (geometry, seed, retries, n_eff), and every served query equals the
    # oracle's query on the resident structure's exported data array
    from paper_2503_18397_gb300 import serve

    reqs, builds = _workload(8, 32, 5, rate=300.0)
    srv = serve.Server(budget=96 << 20)
    try:
        recs = srv.run(reqs)
        exported = {}
        for r in reqs:
            rec = recs[r.rid]
            if isinstance(r, serve.BuildRequest):
                keys, vals, kind, b, seed = builds[r.sid]
                st, oi, _ = orc.build(orc.default_params(kind=kind, b=b, seed=seed), keys, vals)
                assert st == orc.OK
                for f in ("regime", "h", "shards", "M", "c", "cells", "total_cells", "data_bytes", "seed",
                          "retries", "n_eff"):
                    assert getattr(rec.result, f) == getattr(oi, f), f
            else:
                s = srv.resident[r.sid]
                if r.sid not in exported:
                    exported[r.sid] = vf.vf_export(s)
                q = r.keys.numpy().view(np.uint64)
                want = orc.query(_oinfo(orc, s.info), exported[r.sid], q)
                got = _np(rec.result)
                assert got.dtype.itemsize == want.dtype.itemsize
                assert (got.view(want.dtype) == want).all()
    finally:
        srv.close()


def test_query_batch_equals_the_oracle(vf, orc):
    # the cross-structure query kernel against the oracle's query on each
    # structure's exported array: functions and filters, native and bit-array
    # widths (1, 13), values wider than 32 bits (40, 64), the fuse, LGE and
    # MWHC regimes; half members, half disjoint keys
    specs = [(5000, 0, 8, {}), (70_000, 1, 8, {}), (900_000, 0, 16, {}), (1234, 0, 13, {}), (3000, 0, 1, {}),
             (20_000, 1, 1, {}), (40_000, 1, 13, {}), (50_000, 0, 40, {}), (8000, 0, 64, {}),
             (30_000, 1, 40, {}), (200_000, 0, 8, dict(mode=3, eps=0.01, eta=1e-3)),
             (1_000_000, 1, 8, dict(mode=1))]
    structs, keysets, hostkeys = [], [], []
    for i, (n, kind, b, kw) in enumerate(specs):
        keys = synth.u64_keys(i * 10**7, n, 27)
        vals = synth.values(n, b, 27 + i) if kind == 0 else None
        structs.append(vf.vf_build(keys, vals, params=vf.vf_params_default(kind=kind, b=b, seed=i, **kw)))
        q = np.concatenate([keys[: n // 2], synth.u64_keys(10**12 + i * 10**6, max(n // 2, 1000), 27)])
        hostkeys.append(q)
        keysets.append(torch.from_numpy(q.view(np.int64)).cuda())
    outs = vf.vf_query_batch([(s, k, None) for s, k in zip(structs, keysets)])
    torch.cuda.synchronize()
    for (n, kind, b, kw), s, q, o in zip(specs, structs, hostkeys, outs):
        want = orc.query(_oinfo(orc, s.info), vf.vf_export(s), q)
        got = _host64(o)
        assert got.dtype == want.dtype and (got == want).all(), (n, kind, b)
        if kind == 0:
            assert (got[: n // 2] == synth.values(n, b, 27 + specs.index((n, kind, b, kw)))[: n // 2]).all()
        else:
            assert got[: n // 2].all()
        s.free()
