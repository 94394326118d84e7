"""The serving loop's scheduler on CPU (no GPU, no library): the library calls
and CUDA streams are replaced by fakes that record what the scheduler asked
for, so its host logic is checked on its own: builds are admitted in arrival
order while their memory fits the budget (one that does not fit runs once
nothing else is in flight, resident arrays or not),
small builds are built together and large ones alone, a query starts only once
its structure is resident, and the memory it accounts for returns to the
resident data arrays at the end."""
import contextlib
import threading
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2503_18397_gb300 import serve as S  # noqa: E402

LGE_THRESHOLD = 800_000


class FakeStruct:
    def __init__(self, n, b):
        fuse = n >= LGE_THRESHOLD
        self.info = types.SimpleNamespace(n=n, b=b, regime=1 if fuse else 2, data_bytes=int(n * 1.13 * b / 8) + 64)
        self.freed = False

    def free(self):
        self.freed = True


class FakeLib:
    REGIME_FUSE = 1

    def __init__(self, server_ref):
        self.server_ref = server_ref
        self.calls = []  # ("build" | "batch" | "query", sizes, in_use at the call)
        self.mu = threading.Lock()

    def vf_params_default(self, **kw):
        p = types.SimpleNamespace(kind=0, b=8, seed=1, lge_threshold=LGE_THRESHOLD)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    def _log(self, what, sizes):
        with self.mu:
            self.calls.append((what, sizes, self.server_ref[0]._in_use))

    def vf_build(self, keys, values, params=None, stream=None):
        self._log("build", [len(keys)])
        return FakeStruct(len(keys), params.b)

    def vf_build_batch(self, items, params=None, stream=None):
        self._log("batch", [len(k) for k, _, _, _, _ in items])
        return [FakeStruct(len(k), b) for k, _, _, b, _ in items]

    def vf_query_batch(self, reqs, stream=None):
        self._log("query", [len(k) for _, k, _ in reqs])
        return [torch.zeros(len(k), dtype=torch.uint8) for _, k, _ in reqs]


class FakeStream:
    def __init__(self, device=None):
        pass

    def synchronize(self):
        pass


FAKE_TORCH = types.SimpleNamespace(cuda=types.SimpleNamespace(
    Stream=FakeStream, set_device=lambda d: None, stream=lambda s: contextlib.nullcontext()))


def _run(monkeypatch, requests, budget):
    ref = [None]
    lib = FakeLib(ref)
    monkeypatch.setattr(S, "B", lib)
    monkeypatch.setattr(S, "torch", FAKE_TORCH)
    srv = S.Server(device="cpu", budget=budget, batch_below=1 << 20, batch_keys=1 << 26)
    ref[0] = srv
    out = {}

    def go():
        try:
            out["recs"] = srv.run(requests, realtime=False)
        except Exception as e:  # noqa: BLE001
            out["err"] = e

    t = threading.Thread(target=go, daemon=True)
    t.start()
    t.join(60)
    if t.is_alive():  # a request that is never admitted: stop the loop, then fail
        srv._errors.append(TimeoutError("no progress"))
        t.join(10)
        pytest.fail("the scheduler left requests waiting for 60 s")
    if "err" in out:
        raise out["err"]
    return srv, lib, out["recs"]


def _keys(n):
    return torch.zeros(n, dtype=torch.int64)


def test_admission_batching_residency_and_accounting(monkeypatch):
    sizes = [1000, 50_000, 2_000_000, 3000, 1_500_000, 70_000]
    reqs, rid = [], 0
    for sid, n in enumerate(sizes):
        reqs.append(S.BuildRequest(rid, 0.0, sid, _keys(n), None, 1, 8, sid))
        rid += 1
    for sid, n in enumerate(sizes):
        for m in (10, 5000):
            reqs.append(S.QueryRequest(rid, 0.0, sid, _keys(m)))
            rid += 1
    budget = S.build_need(2_000_000, 8, True) + S.build_need(1_500_000, 8, True) // 2
    srv, lib, recs = _run(monkeypatch, reqs, budget)
    try:
        assert all(r.done > 0 and r.latency >= 0 for r in recs.values())
        # every build asked for while the accounted memory was within the budget
        # (the only exception: a build admitted alone, with nothing else in flight)
        for what, ns, in_use in lib.calls:
            if what in ("build", "batch"):
                assert in_use <= budget or len(ns) == 1
        # large builds alone with vf_build, small ones through the batched build
        built = {}
        for what, ns, _ in lib.calls:
            for n in ns:
                if what != "query":
                    built[n] = what
        assert built[2_000_000] == built[1_500_000] == "build"
        assert all(built[n] == "batch" for n in (1000, 50_000, 3000, 70_000))
        # a query starts after its structure's build is done
        bdone = {r.sid: recs[r.rid].done for r in reqs if isinstance(r, S.BuildRequest)}
        for r in reqs:
            if isinstance(r, S.QueryRequest):
                assert recs[r.rid].start >= bdone[r.sid]
        # what stays accounted is the resident data arrays
        assert srv._in_use == sum(s.info.data_bytes for s in srv.resident.values())
        assert sorted(srv.resident) == list(range(len(sizes)))
    finally:
        srv.close()


def test_oversized_build_runs_alone(monkeypatch):
    # a build larger than the whole budget is admitted once nothing else is in
    # flight, although a resident data array keeps memory accounted
    big = 3_000_000
    reqs = [S.BuildRequest(0, 0.0, 0, _keys(1000), None, 1, 8, 1),
            S.BuildRequest(1, 0.0, 1, _keys(big), None, 1, 8, 2),
            S.QueryRequest(2, 0.0, 1, _keys(100))]
    budget = S.build_need(big, 8, True) // 4
    srv, lib, recs = _run(monkeypatch, reqs, budget)
    try:
        assert all(r.done > 0 for r in recs.values())
        big_calls = [c for c in lib.calls if c[0] == "build" and c[1] == [big]]
        assert len(big_calls) == 1
        # when it ran, only its own need (and resident arrays) were accounted
        small_data = FakeStruct(1000, 8).info.data_bytes
        assert big_calls[0][2] <= S.build_need(big, 8, True) + small_data
    finally:
        srv.close()
