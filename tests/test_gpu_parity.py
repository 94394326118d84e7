"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact: signatures; shard bits, largest shard, geometry, seed and retries of
every build; every member key decodes to its value (function) or is accepted
(filter); and for arbitrary keys the GPU query equals the oracle's query on the
same (GPU-built) data array byte for byte. The data array itself may differ
from the oracle's where the peel order differs.
"""
import math

import numpy as np
import pytest

from paper_2503_18397_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

_NP2T = {np.uint8: torch.uint8, np.int64: torch.int64}


@pytest.fixture(scope="module")
def vf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2503_18397_gb300 import build

    build.build()
    import paper_2503_18397_gb300 as vf

    vf.lib()
    return vf


def dev(a: np.ndarray):
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda()
    if a.dtype == np.uint16:
        return torch.from_numpy(a.view(np.int16)).cuda().view(torch.uint16)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32)
    return torch.from_numpy(a).cuda()


def host(t) -> np.ndarray:
    # int64 tensors are 64-bit results (values wider than 32 bits) or u64 keys
    m = {torch.uint16: (torch.int16, np.uint16), torch.uint32: (torch.int32, np.uint32),
         torch.uint64: (torch.int64, np.uint64), torch.int64: (torch.int64, np.uint64)}
    if t.dtype in m:
        sd, nd = m[t.dtype]
        return t.view(sd).cpu().numpy().view(nd)
    return t.cpu().numpy()


def oracle_info(orc, info):
    oi = orc.Info()
    for f, _ in orc.Info._fields_:
        setattr(oi, f, getattr(info, f))
    return oi


def check_build(vf, orc, keys, vals, offsets=None, n_other=20_000, **kw):
    """Build on GPU and with the oracle; compare geometry, decode and query parity."""
    kind = vf.FUNC if vals is not None else vf.FILTER
    key_kind = vf.KEYS_BYTES if offsets is not None else vf.KEYS_U64
    p = vf.vf_params_default(kind=kind, key_kind=key_kind, **kw)
    n = len(offsets) - 1 if offsets is not None else len(keys)
    s = vf.vf_build(dev(keys), None if vals is None else dev(vals), offsets=None if offsets is None else dev(offsets),
                    params=p)
    info = s.info
    op = orc.default_params(kind=kind, key_kind=key_kind, **{k: v for k, v in kw.items() if k != "fuse_solver"})
    st, oi, odata = orc.build(op, keys, vals, offsets=offsets)
    assert st == orc.OK
    for f in ("regime", "h", "h_bb", "h_dup", "shards", "M", "c", "lg_seg", "seg", "l", "T", "cells",
              "total_cells", "data_bytes", "seed", "retries", "n_eff", "k"):
        assert getattr(info, f) == getattr(oi, f), f
    if info.regime == vf.REGIME_FUSE:
        assert info.peeled == oi.peeled == info.n_eff
    out = host(s.query(dev(keys), offsets=None if offsets is None else dev(offsets)))
    if kind == vf.FUNC:
        assert (out == vals).all()
    else:
        assert out.all()
    data = vf.vf_export(s)
    assert len(data) == info.data_bytes
    # oracle query on the GPU-built array decodes members too
    ref = orc.query(oracle_info(orc, info), data, keys, offsets=offsets)
    assert (ref == out).all()
    if n_other:
        if offsets is None:
            other = synth.u64_keys(n + 7, n_other, 99)
            gq = host(s.query(dev(other)))
            oq = orc.query(oracle_info(orc, info), data, other)
        else:
            ob, oo = synth.byte_strings(n + 7, n_other, 99)
            gq = host(s.query(dev(ob), offsets=dev(oo)))
            oq = orc.query(oracle_info(orc, info), data, ob, offsets=oo)
        assert gq.dtype == oq.dtype and (gq == oq).all()
    return s, info, oi


# ---------------------------------------------------------------- signatures

@pytest.mark.parametrize("seed", [0, 1, 0xDEADBEEF, 2**64 - 1])
@pytest.mark.parametrize("n", [1, 31, 100_003])
def test_signatures_u64(vf, orc, seed, n):
    keys = synth.u64_keys(5, n, seed & 0xFFFF)
    g = host(vf.vf_signatures(dev(keys), seed))
    assert (g == orc.sigs(keys, seed)).all()


def test_signatures_bytes_unaligned(vf, orc):
    data, offs = synth.byte_strings(0, 50_001, 3, lmin=8, lmax=64)
    # shift the buffer so strings start at every alignment, include empty and short strings
    extra = [b"", b"x", b"abcdefg", b"abcdefgh", b"abcdefghi", bytes(range(200))]
    tail = np.frombuffer(b"".join(extra), dtype=np.uint8)
    buf = np.concatenate([np.zeros(3, np.uint8), data, tail])
    offs = np.concatenate([offs + np.uint64(3),
                           offs[-1] + np.uint64(3) + np.cumsum([len(x) for x in extra]).astype(np.uint64)])
    for seed in (0, 77):
        g = host(vf.vf_signatures(dev(buf), seed, offsets=dev(offs)))
        assert (g == orc.sigs(buf, seed, offsets=offs)).all()


def test_signatures_host_buffers(vf, orc):
    keys = synth.u64_keys(0, 4096, 1)
    g = vf.vf_signatures(keys, 5)  # numpy in, numpy out: staged through the device
    assert (g == orc.sigs(keys, 5)).all()


# -------------------------------------------------------------------- builds

@pytest.mark.parametrize("n", [0, 1, 2, 3, 97, 1000, 30_011])
@pytest.mark.parametrize("b", [1, 8, 13, 16, 32])
def test_function_lge_regime(vf, orc, n, b):
    keys = synth.u64_keys(0, n, 21 + n)
    vals = synth.values(n, b, 21 + n)
    check_build(vf, orc, keys, vals, b=b, seed=4, n_other=5000)


@pytest.mark.parametrize("b", [1, 8, 16, 32])
def test_filter_lge_regime(vf, orc, b):
    n = 50_000
    keys = synth.u64_keys(0, n, 2)
    s, info, _ = check_build(vf, orc, keys, None, b=b, seed=9)
    assert info.h >= 2 and info.core > 0


@pytest.mark.parametrize("kind", ["func", "filter"])
@pytest.mark.parametrize("n,s", [(22_000, 2), (24_000, 1)])
def test_lge_large_shard_dense_system_in_slab(vf, orc, kind, n, s):
    # One LGE shard of 22K-24K keys, near the largest shard the regime allows:
    # its dense system (~1000 rows over ~1450 active variables) outgrows shared
    # memory and is solved in the CTA's global slab. Seed and retries must stay
    # the oracle's (a capacity failure would retry where the oracle does not).
    keys = synth.u64_keys(s * 1_000_003, n, 77)
    vals = synth.values(n, 8, 77) if kind == "func" else None
    st, info, _ = check_build(vf, orc, keys, vals, b=8, mode=vf.MODE_LGE, lge_target=24_576, seed=5 + s,
                              n_other=5000)
    assert info.shards == 1 and info.retries == 0


def test_lge_peel_arrays_spill_to_large_configuration(vf, orc):
    # 8 shards of ~31K keys whose peel arrays (cells/4 + cells/2 + keys/32 words)
    # straddle the small solver configuration's 27648 words: 6 shards go through
    # the spill list to the large configuration, 2 stay in the small one
    n = 250_950
    keys = synth.u64_keys(0, n, 78)
    vals = synth.values(n, 16, 78)
    st, info, _ = check_build(vf, orc, keys, vals, b=16, mode=vf.MODE_LGE, lge_target=36_000, lge_max_shard=60_000,
                              seed=6, n_other=5000)
    assert info.shards == 8 and info.retries == 0
    sh, _ = orc.shard_local(orc.sigs(keys, info.seed), info.h)
    m = np.bincount(sh, minlength=8)
    words = -(-info.cells // 4) + -(-info.cells // 2) + -(-m // 32)
    assert 0 < int((words > 27 * 1024).sum()) < 8


def test_lge_sharded_byte_strings(vf, orc):
    n = 60_000
    data, offs = synth.byte_strings(0, n, 5)
    vals = synth.values(n, 16, 5)
    s, info, oi = check_build(vf, orc, data, vals, offsets=offs, b=16, mode=vf.MODE_LGE, lge_target=4096, seed=3)
    assert info.regime == vf.REGIME_LGE and info.shards >= 8 and info.core > 0


def test_lge_host_inputs(vf, orc):
    n = 20_000
    keys = synth.u64_keys(0, n, 8)
    vals = synth.values(n, 8, 8)
    s = vf.vf_build(keys, vals, params=vf.vf_params_default(seed=2))
    out = s.query(keys)  # numpy in, numpy out
    assert isinstance(out, np.ndarray) and (out == vals).all()


# both fuse-regime solvers (asynchronous worklist, round-synchronous) must give
# the oracle's outcome; SOLVER values are 0 (flow) and 1 (rounds)
SOLVERS = pytest.mark.parametrize("solver", [0, 1, 2], ids=["flow", "rounds", "wave"])


@SOLVERS
def test_function_fuse_unsharded_2pow20(vf, orc, solver):
    n = 1 << 20
    keys = synth.u64_keys(0, n, 1)
    vals = synth.values(n, 8, 1)
    s, info, _ = check_build(vf, orc, keys, vals, seed=1, n_other=1 << 18, fuse_solver=solver)
    if solver != 0:
        assert info.rounds > 0  # the round and wave solvers ran (no fallback to the worklist solver)
    assert info.regime == vf.REGIME_FUSE and info.h == 0 and info.lg_seg == 13
    assert (0 < info.rounds < n) if solver != 0 else info.rounds == 0


@SOLVERS
@pytest.mark.parametrize("b", [1, 7, 8, 16, 32])
def test_filter_fuse_regime(vf, orc, b, solver):
    n = 1_000_003
    keys = synth.u64_keys(0, n, 3)
    s, info, _ = check_build(vf, orc, keys, None, b=b, seed=5, n_other=200_000, fuse_solver=solver)
    other = synth.u64_keys(n, 400_000, 3)
    fpr = host(s.query(dev(other))).mean()
    p = 2.0 ** -b
    assert abs(fpr - p) < 5 * math.sqrt(p * (1 - p) / len(other)) + 1e-9


@SOLVERS
def test_fuse_sharded_byte_strings(vf, orc, solver):
    # epsilon forced up so that 2M keys shard (h > 0) in the fuse regime
    n = 2_000_000
    data, offs = synth.byte_strings(0, n, 6)
    vals = synth.values(n, 16, 6)
    s, info, _ = check_build(vf, orc, data, vals, offsets=offs, b=16, mode=vf.MODE_FUSE, eps=0.01, seed=2,
                             n_other=50_000, fuse_solver=solver)
    assert info.h >= 1


@SOLVERS
def test_retries_match_oracle(vf, orc, solver):
    # small forced fuse graphs often fail to peel: the GPU must fail exactly when
    # the oracle does (the 2-core is unique) and succeed with the same seed
    keys = synth.u64_keys(0, 600_000, 4)
    vals = synth.values(600_000, 8, 4)
    retried = 0
    for seed in range(8):
        s, info, oi = check_build(vf, orc, keys, vals, mode=vf.MODE_FUSE, seed=seed, max_retries=20, n_other=0,
                                  fuse_solver=solver)
        retried += info.retries > 0
    assert retried > 0


@SOLVERS
@pytest.mark.parametrize("n", [0, 1, 2, 3, 31, 1000, 20_000])
def test_fuse_forced_tiny_and_empty(vf, orc, n, solver):
    # fuse graphs of a few segments (eq. (ln) segments of 4 cells and up), far
    # below the sizes the fuse regime is meant for: whether every attempt fails
    # (ℓ of a few segments does not peel at c = 1.12) or one succeeds, and with
    # which seed, must be the oracle's; functions and filters, both arities
    keys = synth.u64_keys(0, n, 40 + n)
    vals = synth.values(n, 8, 40 + n)
    outcomes = set()
    for arity in (3, 4):
        for v in (vals, None):
            kind = orc.FUNC if v is not None else orc.FILTER
            st, oi, _ = orc.build(orc.default_params(kind=kind, b=8, mode=orc.MODE_FUSE, seed=n, max_retries=30,
                                                     arity=arity), keys, v)
            outcomes.add(st)
            if st == orc.OK:
                s, info, _ = check_build(vf, orc, keys, v, mode=vf.MODE_FUSE, seed=n, max_retries=30, n_other=500,
                                         fuse_solver=solver, arity=arity)
                if n:
                    assert info.regime == vf.REGIME_FUSE and info.k == arity
                s.free()
            else:
                assert st == orc.EBUILD
                with pytest.raises(vf.VFError) as e:
                    vf.vf_build(dev(keys), None if v is None else dev(v),
                                params=vf.vf_params_default(kind=kind, b=8, mode=vf.MODE_FUSE, seed=n, max_retries=30,
                                                            fuse_solver=solver, arity=arity))
                assert e.value.status == 3  # VF_EBUILD, like the oracle
    if n <= 3:
        assert outcomes == {orc.OK}


# ---------------------------------------------------------------- MWHC (Sec. 4.1)

@SOLVERS
@pytest.mark.parametrize("b", [1, 8, 13, 32])
def test_mwhc_function(vf, orc, b, solver):
    n = 300_000
    keys = synth.u64_keys(0, n, 41)
    vals = synth.values(n, b, 41)
    s, info, _ = check_build(vf, orc, keys, vals, b=b, mode=vf.MODE_MWHC, eps=0.01, eta=1e-3, seed=2,
                             n_other=50_000, fuse_solver=solver)
    assert info.regime == vf.REGIME_MWHC and info.c == 1.23 and info.cells % 3 == 0


@SOLVERS
def test_mwhc_filter_sharded(vf, orc, solver):
    n = 2_000_000
    keys = synth.u64_keys(0, n, 42)
    s, info, _ = check_build(vf, orc, keys, None, b=8, mode=vf.MODE_MWHC, eps=0.01, eta=1e-3, seed=9,
                             n_other=200_000, fuse_solver=solver)
    assert info.h == 4 and info.regime == vf.REGIME_MWHC
    other = synth.u64_keys(n, 400_000, 42)
    fpr = host(s.query(dev(other))).mean()
    assert abs(fpr - 2.0**-8) < 5 * math.sqrt(2.0**-8 / len(other))


def test_mwhc_byte_strings_and_duplicates(vf, orc):
    data, offs = synth.byte_strings(0, 400_000, 43)
    vals = synth.values(400_000, 16, 43)
    check_build(vf, orc, data, vals, offsets=offs, b=16, mode=vf.MODE_MWHC, eps=0.05, eta=1e-3, seed=1,
                n_other=30_000)
    keys = with_repeats(200_000, 0.02, 44)
    s, info, oi = check_build(vf, orc, keys, None, mode=vf.MODE_MWHC, eps=0.05, eta=1e-3, seed=5, n_other=0)
    assert info.n_eff == oi.n_eff == 200_000


@SOLVERS
def test_mwhc_retries_match_oracle(vf, orc, solver):
    # 256 shards of ~1560 keys: at this size c = 1.23 leaves a 2-core or a
    # duplicate edge in some shard most of the time, so attempts are retried; the
    # GPU fails exactly when the oracle does (every seed here needs 3..8 retries)
    keys = synth.u64_keys(0, 400_000, 45)
    vals = synth.values(400_000, 8, 45)
    retried = 0
    for seed in range(4):
        s, info, oi = check_build(vf, orc, keys, vals, mode=vf.MODE_MWHC, eps=0.5, eta=0.9, seed=seed,
                                  max_retries=30, n_other=0, fuse_solver=solver)
        assert info.h == 8
        retried += info.retries > 0
    assert retried > 0


# ------------------------------------------------------------ values wider than 32 bits

@pytest.mark.parametrize("b", [33, 40, 63, 64])
@pytest.mark.parametrize("regime", ["fuse", "lge", "mwhc"])
def test_wide_function(vf, orc, b, regime):
    # b > 32: two bit-plane slices on one hypergraph, packed into b-bit cells
    n = {"fuse": 1_200_000, "lge": 50_000, "mwhc": 300_000}[regime]
    keys = synth.u64_keys(0, n, 71)
    vals = synth.values(n, b, 71)
    extra = {"mode": vf.MODE_MWHC, "eps": 0.01, "eta": 1e-3} if regime == "mwhc" else {}
    s, info, _ = check_build(vf, orc, keys, vals, b=b, seed=3, n_other=30_000, **extra)
    assert info.b == b and info.regime == {"fuse": vf.REGIME_FUSE, "lge": vf.REGIME_LGE, "mwhc": vf.REGIME_MWHC}[regime]


@pytest.mark.parametrize("b", [33, 64])
def test_wide_filter(vf, orc, b):
    n = 1_000_003
    keys = with_repeats(n, 0.001, 72)
    s, info, oi = check_build(vf, orc, keys, None, b=b, seed=5, n_other=100_000)
    assert info.n_eff == oi.n_eff == n
    assert host(s.query(dev(synth.u64_keys(n, 400_000, 72)))).sum() == 0


def test_wide_byte_strings_and_host_buffers(vf, orc):
    data, offs = synth.byte_strings(0, 40_000, 73)
    vals = synth.values(40_000, 48, 73)
    check_build(vf, orc, data, vals, offsets=offs, b=48, seed=1, n_other=5_000)
    # host inputs and host output through the same entry points
    keys = synth.u64_keys(0, 20_000, 74)
    v = synth.values(20_000, 37, 74)
    s = vf.vf_build(keys, v, params=vf.vf_params_default(b=37, seed=2))
    out = s.query(keys)
    assert out.dtype == np.uint64 and (out == v).all()


def with_repeats(n, frac, seed, triples=False):
    """n distinct keys plus copies of a random subset (a few in triplicate), shuffled."""
    keys = synth.u64_keys(0, n, seed)
    rng = np.random.default_rng(seed)
    rep = keys[rng.choice(n, size=int(n * frac), replace=False)]
    parts = [keys, rep] + ([rep[: len(rep) // 4]] if triples else [])
    allk = np.concatenate(parts)
    return allk[rng.permutation(len(allk))]


@SOLVERS
def test_filter_duplicate_keys_fuse(vf, orc, solver):
    # repeated keys give identical edges, which never peel: the GPU drops the
    # copies found among the unpeeled edges and solves again (Sec. 4.5)
    keys = with_repeats(1_000_000, 0.02, 21, triples=True)
    s, info, oi = check_build(vf, orc, keys, None, seed=3, n_other=100_000, fuse_solver=solver)
    assert info.regime == vf.REGIME_FUSE
    assert info.n_eff == oi.n_eff == 1_000_000 < len(keys)


def test_filter_duplicate_keys_lge(vf, orc):
    keys = with_repeats(60_000, 0.05, 22, triples=True)
    s, info, oi = check_build(vf, orc, keys, None, b=16, seed=4, n_other=20_000)
    assert info.regime == vf.REGIME_LGE
    assert info.n_eff == oi.n_eff == 60_000


def test_filter_duplicate_keys_sharded_fuse(vf, orc):
    # sharded fuse regime (eps forced up): duplicates are per shard
    keys = with_repeats(2_000_000, 0.01, 23)
    s, info, oi = check_build(vf, orc, keys, None, mode=vf.MODE_FUSE, eps=0.01, seed=6, n_other=50_000)
    assert info.h >= 1 and info.n_eff == oi.n_eff == 2_000_000


def with_repeated_pairs(n, frac, seed, b):
    """n distinct keys with values, plus copies of a random subset (same values,
    a few in triplicate), shuffled; also returns the distinct keys and values."""
    keys = synth.u64_keys(0, n, seed)
    vals = synth.values(n, b, seed)
    rng = np.random.default_rng(seed)
    rep = rng.choice(n, size=int(n * frac), replace=False)
    idx = np.concatenate([np.arange(n), rep, rep[: len(rep) // 4]])
    idx = idx[rng.permutation(len(idx))]
    return keys[idx], vals[idx], keys, vals


DUP_REGIMES = {
    "fuse": (1_000_000, dict(seed=3)),
    "fuse_rounds": (1_000_000, dict(seed=3, fuse_solver=1)),
    "fuse_flow": (1_000_000, dict(seed=3, fuse_solver=0)),
    "sharded_fuse": (2_000_000, dict(mode=1, eps=0.01, seed=6)),
    "lge": (60_000, dict(seed=4)),
    "lge_unsharded": (10_000, dict(seed=5)),
    "mwhc": (300_000, dict(mode=3, eps=0.01, eta=1e-3, seed=7)),
}


@pytest.mark.parametrize("regime", sorted(DUP_REGIMES))
def test_function_repeated_pairs_are_dropped(vf, orc, regime):
    # Sec. 4.4: a (key, value) pair given several times is one equation: the
    # copies are dropped (fuse and MWHC regimes: found among the unpeeled edges
    # of the failed first peel; LGE: in the core), n_eff equals the oracle's
    n, kw = DUP_REGIMES[regime]
    dk, dv, keys, vals = with_repeated_pairs(n, 0.02, 31, 8)
    s, info, oi = check_build(vf, orc, dk, dv, n_other=20_000, **kw)
    assert info.n_eff == oi.n_eff == n < len(dk)
    assert (host(s.query(dev(keys))) == vals).all()


@pytest.mark.parametrize("regime", sorted(DUP_REGIMES))
def test_function_key_with_two_values_is_vf_edup(vf, orc, regime):
    # a key given with two different values has no solution at any seed: the
    # build stops at its first attempt with VF_EDUP, as the oracle does
    n, kw = DUP_REGIMES[regime]
    keys = synth.u64_keys(0, n, 32)
    vals = synth.values(n, 8, 32)
    dk = np.concatenate([keys, keys[n // 3: n // 3 + 1]])
    dv = np.concatenate([vals, (vals[n // 3: n // 3 + 1] ^ 5).astype(vals.dtype)])
    p = vf.vf_params_default(kind=vf.FUNC, **kw)
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(dev(dk), dev(dv), params=p)
    assert e.value.status == 4, str(e.value)  # VF_EDUP
    st, oi, _ = orc.build(orc.default_params(kind=orc.FUNC, **{k: v for k, v in kw.items() if k != "fuse_solver"}),
                          dk, dv)
    assert st == orc.EDUP and oi.retries == 0


def test_function_duplicates_byte_strings_and_wide_values(vf, orc):
    # byte strings in the LGE regime; 40-bit values (two 32-bit slices): a key
    # whose two values differ only in the high slice is still VF_EDUP
    data_, offs = synth.byte_strings(0, 30_000, 33)
    strs = [bytes(data_[offs[i]:offs[i + 1]]) for i in range(30_000)]
    vals = synth.values(30_000, 16, 33)
    s2 = strs + strs[:100]
    v2 = np.concatenate([vals, vals[:100]])
    o2 = np.zeros(len(s2) + 1, dtype=np.uint64)
    o2[1:] = np.cumsum([len(x) for x in s2])
    buf = np.frombuffer(b"".join(s2), dtype=np.uint8).copy()
    s, info, oi = check_build(vf, orc, buf, v2, offsets=o2, b=16, seed=2)
    assert info.n_eff == oi.n_eff == 30_000
    v2[-1] ^= 1
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(dev(buf), dev(v2), offsets=dev(o2), params=vf.vf_params_default(b=16, key_kind=vf.KEYS_BYTES))
    assert e.value.status == 4
    n = 50_000
    keys = synth.u64_keys(0, n, 34)
    vals = synth.values(n, 40, 34)
    dk = np.concatenate([keys, keys[:10]])
    dv = np.concatenate([vals, vals[:10]])
    s, info, oi = check_build(vf, orc, dk, dv, b=40, seed=3)
    assert info.n_eff == oi.n_eff == n
    dv[-1] ^= np.uint64(1 << 37)
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(dev(dk), dev(dv), params=vf.vf_params_default(b=40))
    assert e.value.status == 4


def test_query_stream_async_and_reuse(vf, orc):
    n = 100_000
    keys = synth.u64_keys(0, n, 12)
    vals = synth.values(n, 16, 12)
    s = vf.vf_build(dev(keys), dev(vals), params=vf.vf_params_default(b=16, seed=1))
    st = torch.cuda.Stream()
    kd = dev(keys)
    with torch.cuda.stream(st):
        outs = [s.query(kd, stream=st) for _ in range(3)]
    st.synchronize()
    for o in outs:
        assert (host(o) == vals).all()


def test_invalid_arguments(vf):
    keys = dev(synth.u64_keys(0, 10, 1))
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(keys, None, params=vf.vf_params_default(kind=vf.FILTER, b=0))
    assert e.value.status == 1
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(keys, None, params=vf.vf_params_default(kind=vf.FUNC))
    assert e.value.status == 1


@pytest.mark.parametrize("b,kind", [(8, "filter"), (16, "func"), (13, "func"), (40, "func")])
def test_query_host_buffers_pipelined(vf, orc, b, kind):
    # 64-bit keys or outputs in host memory go through the chunked two-stream
    # pipeline (chunks of 2^23 keys; here 2 full chunks and a ragged third):
    # every combination of host/device keys and outputs, pinned and pageable
    # host memory, equals the device-resident query and the oracle's query
    n = 200_000
    keys = synth.u64_keys(0, n, 51)
    vals = synth.values(n, b, 51) if kind == "func" else None
    s = vf.vf_build(dev(keys), None if vals is None else dev(vals),
                    params=vf.vf_params_default(kind=vf.FUNC if kind == "func" else vf.FILTER, b=b, seed=2))
    m = 2 * (1 << 23) + 12_345
    q = np.concatenate([keys, synth.u64_keys(n, m - n, 51)])
    qd = dev(q)
    want = host(s.query(qd))
    info = s.info
    ref = orc.query(oracle_info(orc, info), vf.vf_export(s), q[:300_000])
    assert (want[:300_000] == ref).all()
    pinned = torch.from_numpy(q.view(np.int64)).pin_memory()
    tdt = s.query(qd[:1]).dtype
    cases = [
        (q, None),                                          # pageable keys, host output
        (pinned, None),                                     # pinned keys, host output (CPU tensor)
        (q, torch.empty(m, dtype=tdt, device="cuda")),      # host keys, device output
        (qd, np.empty(m, dtype=want.dtype)),                # device keys, pageable host output
        (qd, torch.empty(m, dtype=tdt).pin_memory()),       # device keys, pinned host output
    ]
    for kin, out in cases:
        res = vf.vf_query(s, kin, out=out)
        got = res if isinstance(res, np.ndarray) else host(res)
        assert got.dtype == want.dtype and (got == want).all()
    s.free()


# ------------------------------------------------ 4-uniform fuse graphs (k = 4)

@SOLVERS
@pytest.mark.parametrize("b", [1, 8, 13, 16, 32])
def test_fuse4_function(vf, orc, b, solver):
    n = 1_000_000
    keys = synth.u64_keys(0, n, 71)
    vals = synth.values(n, b, 71)
    s, info, oi = check_build(vf, orc, keys, vals, b=b, mode=vf.MODE_FUSE, arity=4, seed=2, n_other=100_000,
                              fuse_solver=solver)
    assert info.k == oi.k == 4 and info.T == info.l + 3 and info.peeled == oi.peeled == n
    # the round solver counts its rounds; the worklist solver peels 4-uniform graphs
    # otherwise (the wave solver takes 3-uniform graphs only and hands them to it)
    assert info.rounds > 0 if solver == 1 else info.rounds == 0


def test_fuse4_filter_sharded_and_strings(vf, orc):
    n = 3_000_000
    keys = synth.u64_keys(0, n, 72)
    s, info, oi = check_build(vf, orc, keys, None, b=8, mode=vf.MODE_FUSE, arity=4, eps=0.01, seed=3,
                              n_other=200_000)
    assert info.k == 4 and info.h > 0 and info.h_dup == -1
    other = synth.u64_keys(n, 2_000_000, 72)
    fpr = host(s.query(dev(other))).mean()
    assert abs(fpr - 2.0**-8) < 5 * math.sqrt(2.0**-8 / len(other))
    data, offs = synth.byte_strings(0, 400_000, 73)
    vals = synth.values(400_000, 16, 73)
    check_build(vf, orc, data, vals, offsets=offs, b=16, mode=vf.MODE_FUSE, arity=4, eps=0.02, seed=1,
                n_other=20_000)


def test_fuse4_duplicates_retries_and_wide(vf, orc):
    # duplicates are dropped (filter) or kept once (function pairs); a key with two
    # values is VF_EDUP; retries equal the oracle's; 40-bit values in two slices
    keys = with_repeats(500_000, 0.02, 74, triples=True)
    s, info, oi = check_build(vf, orc, keys, None, mode=vf.MODE_FUSE, arity=4, seed=4, n_other=20_000)
    assert info.n_eff == oi.n_eff == 500_000
    dk, dv, _, _ = with_repeated_pairs(300_000, 0.01, 75, 8)
    s, info, oi = check_build(vf, orc, dk, dv, mode=vf.MODE_FUSE, arity=4, seed=5, n_other=0)
    assert info.n_eff == oi.n_eff == 300_000
    bad = dv.copy()
    first = {}
    for i, k in enumerate(dk.tolist()):
        if k in first:
            bad[i] ^= 1
            break
        first[k] = i
    with pytest.raises(vf.VFError) as e:
        vf.vf_build(dev(dk), dev(bad), params=vf.vf_params_default(mode=vf.MODE_FUSE, arity=4))
    assert e.value.status == 4
    seen = 0
    for seed in range(12):
        keys = synth.u64_keys(0, 3000, 80 + seed)
        vals = synth.values(3000, 8, 80 + seed)
        s, info, oi = check_build(vf, orc, keys, vals, mode=vf.MODE_FUSE, arity=4, seed=seed, max_retries=40,
                                  n_other=0)
        seen += info.retries > 0
    assert seen > 0  # small 4-uniform fuse graphs need retries, equal to the oracle's
    keys = synth.u64_keys(0, 200_000, 76)
    vals = synth.values(200_000, 40, 76)
    check_build(vf, orc, keys, vals, b=40, mode=vf.MODE_FUSE, arity=4, seed=6, n_other=20_000)


def test_fuse4_serialized_and_batched_queries(vf, orc):
    n = 400_000
    keys = synth.u64_keys(0, n, 77)
    vals = synth.values(n, 8, 77)
    s = vf.vf_build(dev(keys), dev(vals), params=vf.vf_params_default(mode=vf.MODE_FUSE, arity=4, seed=2))
    t = vf.vf_deserialize(vf.vf_serialize(s))
    assert t.info.k == 4 and (host(t.query(dev(keys))) == vals).all()
    other = synth.u64_keys(n, 50_000, 77)
    q = np.concatenate([keys[:50_000], other])
    outs = vf.vf_query_batch([(s, dev(q), None)])
    torch.cuda.synchronize()
    assert (host(outs[0]) == orc.query(oracle_info(orc, s.info), vf.vf_export(s), q)).all()
    assert (vf.vf_query(s, q) == host(outs[0])).all()  # host keys: the pipelined query
    s.free()
    t.free()
