"""Batched construction (the batching pattern): many independent structures of
uneven sizes built together must each equal the structure vf_build makes from
the same keys, seed and parameters (same geometry, seed, retries; every key
decodes; the oracle's query on the batch-built array matches the GPU query)."""
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


FIELDS = ("regime", "h", "h_bb", "h_dup", "shards", "M", "c", "lg_seg", "seg", "l", "T", "cells", "total_cells",
          "data_bytes", "seed", "retries")


def _make(sizes, seed0):
    rng = np.random.default_rng(seed0)
    items, host = [], []
    for i, n in enumerate(sizes):
        kind = int(rng.integers(0, 2))
        b = int(rng.choice([1, 8, 16, 32]))
        keys = synth.u64_keys(i * 10_000_000, int(n), seed0)
        vals = synth.values(int(n), b, seed0 + i) if kind == 0 else None
        items.append((_dev(keys), None if vals is None else _dev(vals), kind, b, 100 + i))
        host.append((keys, vals, kind, b))
    return items, host


def _check_against_single(vf, orc, items, host, structs, opts_like_default=True):
    for (kd, vd, kind, b, seed), (keys, vals, _, _), s in zip(items, host, structs):
        info = s.info
        out = _host(s.query(kd))
        if kind == 0:
            assert (out == vals).all()
        else:
            assert out.all()
        oi = orc.Info()
        for f, _ in orc.Info._fields_:
            setattr(oi, f, getattr(info, f))
        ref_q = orc.query(oi, vf.vf_export(s), keys)
        assert (ref_q == out).all()
        if opts_like_default:
            single = vf.vf_build(kd, vd, params=vf.vf_params_default(kind=kind, b=b, seed=seed))
            si = single.info
            for f in FIELDS:
                assert getattr(info, f) == getattr(si, f), f
            single.free()


def test_batch_matches_single_builds(vf, orc):
    sizes = [0, 1, 3, 40, 999, 5000, 20_000, 70_000, 150_000, 12, 333, 31_000]
    items, host = _make(sizes, 7)
    structs = vf.vf_build_batch(items, params=vf.vf_params_default(), opts=vf.vf_batch_opts_default(use_graph=1))
    _check_against_single(vf, orc, items, host, structs)


def test_batch_without_graph_and_natural_order(vf, orc):
    items, host = _make([100, 2000, 17_000, 40_000], 9)
    structs = vf.vf_build_batch(items, opts=vf.vf_batch_opts_default(use_graph=0, lpt=0))
    _check_against_single(vf, orc, items, host, structs)


@pytest.mark.parametrize("small", [0, 1 << 20])
def test_batch_cta_configuration(vf, orc, small):
    # every LGE shard in the two-CTA configuration (0), or every shard offered
    # to the three-CTA one (those whose peel arrays do not fit its shared
    # memory pass through the spill list): same seeds, retries and geometry as
    # single builds, every member decoded, the oracle's query equal
    items, host = _make([700, 6000, 9000, 30_000, 150_000], 15)
    structs = vf.vf_build_batch(items, opts=vf.vf_batch_opts_default(small_cta_keys=small))
    _check_against_single(vf, orc, items, host, structs)


def test_batch_mixed_regimes(vf, orc):
    # one structure above the fuse threshold among small LGE ones
    items, host = _make([900_000, 3_000, 60_000], 11)
    structs = vf.vf_build_batch(items)
    assert structs[0].info.regime == vf.REGIME_FUSE and structs[1].info.regime == vf.REGIME_LGE
    _check_against_single(vf, orc, items, host, structs)


def test_batch_all_lge_threshold_and_tuner(vf, orc):
    sizes = synth.log_uniform_sizes(48, 1e3, 3e5, 5)
    items, host = _make(sizes, 13)
    best, ms = vf.vf_tune_batch(items)
    assert best.lge_target in (8192, 16384) and best.lpt in (0, 1) and best.small_cta_keys in (0, 7168)
    structs = vf.vf_build_batch(items, opts=best)
    _check_against_single(vf, orc, items, host, structs, opts_like_default=False)
    best2, ms2 = vf.vf_tune_batch(items)
    assert ms2 == -1.0 and best2.as_dict() == best.as_dict()  # cached per batch shape


def test_batch_large_shards(vf, orc):
    # single-shard structures of 20K-24.5K keys next to small ones: the largest
    # dense systems are solved outside shared memory, in the same launch as
    # shards solved inside it; every structure keeps the oracle's seed and retries
    sizes = [24_000, 500, 21_000, 23_500, 7_000, 60_000, 24_500, 20_000]
    items, host = _make(sizes, 17)
    structs = vf.vf_build_batch(items, opts=vf.vf_batch_opts_default(lge_target=24_576))
    for (kd, vd, kind, b, seed), (keys, vals, _, _), s in zip(items, host, structs):
        info = s.info
        out = _host(s.query(kd))
        assert (out == vals).all() if kind == 0 else out.all()
        op = orc.default_params(kind=kind, b=b, seed=seed, lge_target=24_576)
        st, oi, _ = orc.build(op, keys, vals)
        assert st == orc.OK
        for f in FIELDS:
            assert getattr(info, f) == getattr(oi, f), f
        s.free()


def test_batch_filter_duplicate_keys(vf, orc):
    # filters with repeated keys inside a batch: copies are dropped per shard in the
    # LGE solver (Sec. 4.5); n_eff and every query equal the oracle's build
    rng = np.random.default_rng(31)
    items, host = [], []
    for i, n in enumerate([3000, 40_000, 250_000]):
        keys = synth.u64_keys(i * 10_000_000, n, 31)
        rep = keys[rng.choice(n, size=n // 20, replace=False)]
        allk = np.concatenate([keys, rep, rep[: len(rep) // 3]])
        allk = allk[rng.permutation(len(allk))]
        items.append((_dev(allk), None, 1, 8, 500 + i))
        host.append((allk, n))
    structs = vf.vf_build_batch(items)
    for s, (allk, n) in zip(structs, host):
        info = s.info
        st, oi, _ = orc.build(orc.default_params(kind=orc.FILTER, b=8, seed=info.seed - info.retries), allk)
        assert st == orc.OK
        assert info.n_eff == oi.n_eff == n
        assert (info.seed, info.retries) == (oi.seed, oi.retries)
        assert _host(s.query(_dev(allk))).all()
        s.free()


def test_batch_function_duplicates(vf, orc):
    # functions with repeated (key, value) pairs inside a batch keep one copy
    # (LGE solver and, above the threshold, the fuse solver); a key given with
    # two values makes the whole batch call return VF_EDUP
    rng = np.random.default_rng(32)
    items, host = [], []
    for i, n in enumerate([2000, 30_000, 900_000]):
        keys = synth.u64_keys(i * 10_000_000, n, 32)
        vals = synth.values(n, 16, 32 + i)
        rep = rng.choice(n, size=n // 50, replace=False)
        idx = np.concatenate([np.arange(n), rep])
        idx = idx[rng.permutation(len(idx))]
        items.append((_dev(keys[idx]), _dev(vals[idx]), 0, 16, 600 + i))
        host.append((keys[idx], vals[idx], n))
    structs = vf.vf_build_batch(items)
    for s, (k, v, n) in zip(structs, host):
        info = s.info
        st, oi, _ = orc.build(orc.default_params(kind=orc.FUNC, b=16, seed=info.seed - info.retries), k, v)
        assert st == orc.OK
        assert info.n_eff == oi.n_eff == n
        assert (info.seed, info.retries) == (oi.seed, oi.retries)
        assert (_host(s.query(_dev(k))) == v).all()
        s.free()
    for j in (0, 2):  # a conflicting key in an LGE structure, then in a fuse one
        bad = list(items)
        k, v, n = host[j]
        v2 = v.copy()
        k2 = np.concatenate([k, k[:1]])
        v2 = np.concatenate([v2, (v2[:1] ^ 3).astype(v2.dtype)])
        bad[j] = (_dev(k2), _dev(v2), 0, 16, 600 + j)
        with pytest.raises(vf.VFError) as e:
            vf.vf_build_batch(bad)
        assert e.value.status == 4, str(e.value)
