"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Nothing here compares the oracle with itself: every expected value is a
number printed in the paper (tests/golden/), a closed form, a brute-force
enumeration, an invariant the method guarantees, or a statistical law.
"""
import itertools
import math

import numpy as np
import pytest

from conftest import golden
from paper_2503_18397_gb300 import synth

M64 = (1 << 64) - 1


# ---------------------------------------------------------------- hashing

def test_mix64_matches_published_splitmix64_vector(orc):
    expected = [int(r[0]) for r in golden("splitmix64_seed1234567.txt")]
    state = 1234567
    for want in expected:
        state = (state + 0x9E3779B97F4A7C15) & M64
        assert orc.mix64(state) == want


def test_mulhi_is_fixed_point_inversion(orc):
    rng = np.random.default_rng(1)
    for _ in range(200):
        a = int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2))
        b = int(rng.integers(1, 2**40))
        assert orc.lib().orc_mulhi(a, b) == (a * b) >> 64
        # monotone map of [0, 2^64) onto [0, b)
        assert orc.lib().orc_mulhi(a, b) < b


def test_signatures_distinct_and_uniform(orc):
    n = 400_000
    keys = synth.u64_keys(0, n, 7)
    s = orc.sigs(keys, seed=11)
    # 128-bit signatures of distinct keys are distinct
    both = s[:, 0].astype(object) * (1 << 64) + s[:, 1].astype(object)
    assert len(set(both.tolist())) == n
    # high word is a bijection of the key for integer keys
    assert len(np.unique(s[:, 0])) == n
    # top-8-bit histograms of both words are uniform (chi-square, 255 dof)
    for col in (0, 1):
        top = (s[:, col] >> np.uint64(56)).astype(np.int64)
        cnt = np.bincount(top, minlength=256)
        chi2 = ((cnt - n / 256) ** 2 / (n / 256)).sum()
        assert chi2 < 255 + 6 * math.sqrt(2 * 255)
    # the seed changes every signature
    s2 = orc.sigs(keys, seed=12)
    assert (s2[:, 0] != s[:, 0]).mean() > 0.999


def test_byte_signatures_fold_length_and_content(orc):
    strings = [b"", b"\x00", b"\x00\x00", b"\x00" * 8, b"\x00" * 9, b"a", b"b", b"ab", b"ba",
               b"abcdefgh", b"abcdefghi", bytes(range(64)), bytes(range(63))]
    data = np.frombuffer(b"".join(strings), dtype=np.uint8).copy()
    offs = np.zeros(len(strings) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum([len(x) for x in strings])
    s = orc.sigs(data, seed=3, offsets=offs)
    assert len({(int(a), int(b)) for a, b in s}) == len(strings)
    # a string's signature does not depend on where it sits in the buffer
    shifted = np.concatenate([np.zeros(5, np.uint8), data])
    s2 = orc.sigs(shifted, seed=3, offsets=offs + np.uint64(5))
    assert (s2 == s).all()


def test_random_strings_no_collision_and_uniform(orc):
    data, offs = synth.byte_strings(0, 200_000, 5)
    s = orc.sigs(data, seed=9, offsets=offs)
    assert len(np.unique(s[:, 0])) == len(s)
    top = (s[:, 1] >> np.uint64(58)).astype(np.int64)
    cnt = np.bincount(top, minlength=64)
    chi2 = ((cnt - len(s) / 64) ** 2 / (len(s) / 64)).sum()
    assert chi2 < 63 + 6 * math.sqrt(2 * 63)


# ------------------------------------------------------------- parameters

def test_lambert_w_closed_forms(orc):
    W = orc.lib().orc_lambert_w0
    assert W(0.0) == 0.0
    assert abs(W(1.0) - 0.5671432904097838) < 1e-15  # omega constant
    assert abs(W(math.e) - 1.0) < 1e-14
    assert abs(W(2 * math.e**2) - 2.0) < 1e-14
    for x in [1e-6, 0.3, 7.0, 38.24, 1e3, 1e9]:
        w = W(x)
        assert abs(w * math.exp(w) - x) <= 1e-12 * x


def test_table1_shard_counts(orc):
    # Table tab:offline; reading: eta = 0.1 in eq. (logdupfuse)
    p = orc.default_params()
    for keys, shards in golden("table1_offline_shards.txt"):
        h, regime, h_bb, h_dup = orc.plan_h(p, int(keys))
        assert regime == orc.REGIME_FUSE
        assert 1 << h == int(shards)
        assert h == min(h_bb, h_dup)


def test_logdupfuse_dominates_for_large_n(orc):
    # Sec. 4.2: in the long run eq. (logdupfuse) is the binding bound.
    p = orc.default_params()
    for n in [10**10, 10**11, 10**12, 10**13]:
        h, _, h_bb, h_dup = orc.plan_h(p, n)
        assert h_dup < h_bb and h == h_dup


def test_mwhc_shard_example(orc):
    for keys, c, eta, shards in golden("mwhc_shard_example.txt"):
        assert 1 << orc.lib().orc_h_dupmwhc(int(keys), float(eta), float(c)) == int(shards)


def test_ballsbins_bound_direct(orc):
    # eq. (ballsbins): s ln s <= n eps^2 / 2  <=>  ln s <= W(n eps^2 / 2)
    for n, eps in [(10**8, 0.001), (10**10, 0.001), (5 * 10**9, 0.001), (10**9, 0.01)]:
        h = orc.lib().orc_h_ballsbins(n, eps)
        x = n * eps * eps / 2
        assert h >= 1
        s = 2.0**h
        # the power-of-two approximation never exceeds the Lambert-W bound by more than a bit
        assert math.log(s) <= orc.lib().orc_lambert_w0(x) + math.log(2)
        # rough intuition of Sec. 4: shards of at least about 2/eps^2 keys
        assert n / s >= 0.5 * 2 / eps**2


def test_ballsbins_no_sharding_below_e(orc):
    eps = 0.001
    n_limit = int(2 * math.e / eps**2)
    assert orc.lib().orc_h_ballsbins(n_limit - 1000, eps) == 0
    assert orc.lib().orc_h_ballsbins(2**20, eps) == 0


def test_max_shard_within_eps(orc):
    # epsilon-cost sharding keeps max/mean shard size below 1 + eps (Sec. 4)
    n = 30_000_000
    p = orc.default_params(mode=orc.MODE_FUSE)
    h, _, _, _ = orc.plan_h(p, n)
    assert h >= 1
    s = orc.sigs(synth.u64_keys(0, n, 2), seed=5)
    sh = (s[:, 0] >> np.uint64(64 - h)).astype(np.int64)
    cnt = np.bincount(sh, minlength=1 << h)
    assert cnt.max() / (n / (1 << h)) <= 1 + p.eps


def test_no_repeat_product_and_bound(orc):
    # Sec. 4.1: F = prod_{i<t} (1 - i/n) (exact: n!/((n-t)! n^t)) <= exp(-t(t-1)/2n)
    for n, t in [(365, 23), (1000, 40), (10**6, 1000), (50, 50)]:
        p = orc.lib().orc_no_repeat_prob(float(n), t)
        exact = math.perm(n, t) / n**t
        assert abs(p - exact) <= 1e-12 + 1e-9 * exact
        assert p <= math.exp(-t * (t - 1) / (2 * n)) + 1e-15
    assert abs(orc.lib().orc_no_repeat_prob(365.0, 23) - 0.4927027656) < 1e-9  # birthday problem


def test_space_overhead_large_shards(orc):
    # Sec. 5: 10.5% overhead at epsilon = 0.001 for large key sets (fuse, c = 1.105)
    want = float(dict(golden("overhead.txt"))["large"])
    p = orc.default_params()
    for n in [10**8, 10**9, 10**10]:
        h, regime, _, _ = orc.plan_h(p, n)
        s = 1 << h
        M = int(n / s + math.sqrt(2 * (n / s) * math.log(s)))  # Raab-Steger max load, alpha = 1
        g = orc.geometry(regime, h, M)
        assert g.c == 1.105 and g.l == g.T - 2
        ovh = g.total_cells / n - 1
        assert want - 0.001 <= ovh <= want + 0.003, (n, ovh)


def test_segment_size_estimates(orc):
    # eq. (nln) for sharded large shards, eq. (ln) otherwise, floored powers of two
    g = orc.geometry(orc.REGIME_FUSE, 3, 12_500_000)
    assert g.lg_seg == math.floor(0.41 * math.log(12_500_000) * math.log(math.log(12_500_000)) - 3)
    assert g.lg_seg == 15
    g = orc.geometry(orc.REGIME_FUSE, 0, 2**20)
    assert g.lg_seg == 13 and g.c == 1.12
    assert g.cells == g.T * g.seg and g.T == math.ceil(1.12 * 2**20 / 8192)
    g = orc.geometry(orc.REGIME_LGE, 4, 10_000)
    assert g.cells == math.ceil(1.12 * 10_000)
    assert orc.geometry(orc.REGIME_LGE, 4, 3).cells == 32


# -------------------------------------------------------- edges, fingerprints

def _info(orc, regime, h, M):
    return orc.geometry(regime, h, M)


def test_fuse_edges_in_consecutive_segments_and_monotone(orc):
    info = _info(orc, orc.REGIME_FUSE, 0, 50_000)
    loc = np.sort(synth.u64_keys(0, 20_000, 4))
    e = orc.edges_of(info, loc)
    seg = np.uint64(info.seg)
    s = e[:, 0] // seg
    assert (s < info.l).all()
    assert ((e[:, 1] // seg) == s + np.uint64(1)).all()
    assert ((e[:, 2] // seg) == s + np.uint64(2)).all()
    assert (e < np.uint64(info.cells)).all()
    # fixed-point inversion: the first vertex (and segment) is monotone in the local signature
    assert (np.diff(e[:, 0].astype(np.int64)) >= 0).all()
    # start segment uniform over [0, l)
    cnt = np.bincount(s.astype(np.int64), minlength=info.l)
    exp_ = len(loc) / info.l
    assert ((cnt - exp_) ** 2 / exp_).sum() < info.l + 6 * math.sqrt(2 * info.l)


def test_lge_edges_distinct_uniform(orc):
    # sharded LGE-regime shards: three distinct uniform vertices
    info = _info(orc, orc.REGIME_LGE, 1, 1000)
    loc = synth.u64_keys(0, 50_000, 8)
    e = orc.edges_of(info, loc).astype(np.int64)
    assert (e < info.cells).all()
    assert ((e[:, 0] != e[:, 1]) & (e[:, 1] != e[:, 2]) & (e[:, 0] != e[:, 2])).all()
    for k in range(3):
        cnt = np.bincount(e[:, k], minlength=info.cells)
        exp_ = len(loc) / info.cells
        dof = info.cells - 1
        assert ((cnt - exp_) ** 2 / exp_).sum() < dof + 6 * math.sqrt(2 * dof)
    # small case, exhaustive: every ordered distinct triple is reachable
    tiny = _info(orc, orc.REGIME_LGE, 1, 3)
    tiny.cells = 5
    e = orc.edges_of(tiny, synth.u64_keys(0, 40_000, 9))
    assert len({tuple(r) for r in e.tolist()}) == 5 * 4 * 3


def test_duplicate_edge_rate_matches_paper_estimate(orc):
    # Sec. 4.2: no-duplicate probability ~ exp(-m / (2 c s^2)); expected number of
    # duplicate pairs m(m-1)/2 / (l s^3). Monte Carlo with small segments.
    m = 3000
    info = _info(orc, orc.REGIME_FUSE, 0, m)
    info.lg_seg, info.seg = 4, 16
    info.T = math.ceil(1.12 * m / 16)
    info.l = info.T - 2
    info.cells = info.T * 16
    trials, dups = 60, []
    for t in range(trials):
        e = orc.edges_of(info, synth.u64_keys(t * m, m, 10))
        _, c = np.unique(e, axis=0, return_counts=True)
        dups.append(int((c * (c - 1) // 2).sum()))
    lam = m * (m - 1) / 2 / (info.l * 16**3)
    mean = np.mean(dups)
    assert abs(mean - lam) < 5 * math.sqrt(lam / trials), (mean, lam)
    assert abs(lam - m / (2 * 1.12 * 16**2)) / lam < 0.05


def test_fingerprint_uniform_and_width(orc):
    loc = synth.u64_keys(0, 100_000, 12)
    for b in (1, 8, 16, 32):
        fp = np.array([orc.fingerprint(int(x), b) for x in loc[:20000]], dtype=np.uint64)
        assert (fp < np.uint64(1 << b)).all()
        if b <= 8:
            cnt = np.bincount(fp.astype(np.int64), minlength=1 << b)
            exp_ = len(fp) / (1 << b)
            dof = (1 << b) - 1
            assert ((cnt - exp_) ** 2 / exp_).sum() < dof + 6 * math.sqrt(2 * dof)


def test_shard_and_local_are_top_bits(orc):
    # Sorting by the 128-bit signature orders (shard, local signature)
    # lexicographically: shards are the top bits, the local signature the bits after.
    s = orc.sigs(synth.u64_keys(0, 50_000, 13), seed=2)
    order = np.lexsort((s[:, 1], s[:, 0]))
    s = s[order]
    for h in (1, 3, 7):
        sh, loc = orc.shard_local(s, h)
        assert (np.diff(sh.astype(np.int64)) >= 0).all()
        same = sh[1:] == sh[:-1]
        assert (loc[1:][same] >= loc[:-1][same]).all()


# -------------------------------------------------------- peeling and GF(2)

def _random_hypergraph(rng, V, m):
    edges = []
    for _ in range(m):
        edges.append(rng.choice(V, size=3, replace=False))
    return np.array(edges, dtype=np.uint32).reshape(m, 3)


def _brute_core(V, edges):
    """2-core as the union of all edge subsets where no vertex has degree 1."""
    m = len(edges)
    core = set()
    for mask in range(1, 1 << m):
        deg = [0] * V
        sub = [i for i in range(m) if mask >> i & 1]
        for i in sub:
            for v in edges[i]:
                deg[v] += 1
        if all(d != 1 for d in deg):
            core.update(sub)
    return core


def test_peel_matches_bruteforce_2core(orc):
    rng = np.random.default_rng(3)
    for trial in range(300):
        V = int(rng.integers(4, 9))
        m = int(rng.integers(1, 11))
        edges = _random_hypergraph(rng, V, m)
        ne, order, side = orc.peel(V, edges)
        core = _brute_core(V, edges.tolist())
        assert m - ne == len(core)
        peeled = [int(e) for e in order]
        assert set(peeled).isdisjoint(core)
        # definition of peelable (Sec. 2): in the peel order each edge has a vertex
        # (its side) that appears in no later edge and in no core edge.
        for i, e in enumerate(peeled):
            v = int(edges[e][side[i]])
            later = peeled[i + 1:] + sorted(core)
            assert all(v not in edges[f].tolist() for f in later)


def test_duplicate_edge_is_never_peelable(orc):
    # Sec. 4.1: a duplicate edge always leaves a non-empty 2-core
    edges = np.array([[0, 1, 2], [3, 4, 5], [0, 1, 2]], dtype=np.uint32)
    ne, _, _ = orc.peel(6, edges)
    assert ne == 1


def test_gf2_solve_matches_bruteforce(orc):
    rng = np.random.default_rng(5)
    for trial in range(300):
        V = int(rng.integers(3, 9))
        m = int(rng.integers(1, 12))
        edges = _random_hypergraph(rng, V, m)
        # value widths of 1..3 bits, and 64-bit values whose planes are checked
        # on a few bit positions (a high plane is solved like a low one)
        bits = int(rng.integers(1, 4))
        rhs = rng.integers(0, 1 << bits, size=m).astype(np.uint64)
        if trial % 3 == 0:
            rhs = rhs | (rng.integers(0, 1 << 62, size=m, dtype=np.uint64) << np.uint64(2) & np.uint64(~7 & (2**64 - 1)))
        ok, w = orc.gf2_solve(V, edges, rhs)
        # brute force: each bit plane independently
        solvable = True
        planes = list(range(bits)) + ([3, 31, 32, 63] if trial % 3 == 0 else [])
        for j in planes:
            plane = (rhs >> np.uint64(j)) & np.uint64(1)
            found = False
            for assign in itertools.product((0, 1), repeat=V):
                if all((assign[a] ^ assign[b] ^ assign[c]) == plane[i] for i, (a, b, c) in enumerate(edges)):
                    found = True
                    break
            solvable &= found
        assert ok == solvable
        if ok:
            for i, (a, b, c) in enumerate(edges):
                assert w[a] ^ w[b] ^ w[c] == rhs[i]


# ------------------------------------------------------------------ builds

@pytest.mark.parametrize("n", [0, 1, 2, 3, 97, 5000, 40_000])
@pytest.mark.parametrize("b", [1, 5, 8, 16, 32, 33, 64])
def test_build_function_decodes_every_key(orc, n, b):
    keys = synth.u64_keys(0, n, 21)
    vals = synth.values(n, b, 21)
    st, info, data = orc.build(orc.default_params(b=b, seed=4), keys, vals)
    assert st == orc.OK
    assert info.data_bytes == len(data)
    out = orc.query(info, data, keys)
    assert (out == vals).all()  # Problem 1


def test_build_fuse_regime_unsharded(orc):
    n = 2**20
    keys = synth.u64_keys(0, n, 1)
    vals = synth.values(n, 8, 1)
    st, info, data = orc.build(orc.default_params(seed=1), keys, vals)
    assert st == orc.OK and info.regime == orc.REGIME_FUSE and info.h == 0 and info.core == 0
    assert (orc.query(info, data, keys) == vals).all()


def test_build_lge_regime_sharded_strings(orc):
    data_, offs = synth.byte_strings(0, 30_000, 2)
    vals = synth.values(30_000, 16, 2)
    p = orc.default_params(b=16, key_kind=orc.KEYS_BYTES, mode=orc.MODE_LGE, lge_target=2048, seed=8)
    st, info, data = orc.build(p, data_, vals, offsets=offs)
    assert st == orc.OK and info.regime == orc.REGIME_LGE and info.h >= 3
    assert info.core > 0  # LGE really solved 2-cores
    assert (orc.query(info, data, data_, offsets=offs) == vals).all()


def test_filter_no_false_negatives_and_fpr(orc):
    n, b = 150_000, 8
    keys = synth.u64_keys(0, n, 31)
    st, info, data = orc.build(orc.default_params(kind=orc.FILTER, b=b, seed=2), keys)
    assert st == orc.OK
    assert orc.query(info, data, keys).all()  # no false negatives
    other = synth.u64_keys(n, 1_000_000, 31)
    fpr = orc.query(info, data, other).mean()
    p = 2.0**-b
    assert abs(fpr - p) < 5 * math.sqrt(p * (1 - p) / len(other))  # Sec. 3.1: FPR 2^-b


def test_filter_deduplicates_keys(orc):
    keys = synth.u64_keys(0, 20_000, 5)
    dup = np.concatenate([keys, keys[:5000]])
    st, info, data = orc.build(orc.default_params(kind=orc.FILTER, b=8, mode=orc.MODE_FUSE, seed=1), dup)
    assert st == orc.OK and info.n_eff == 20_000
    assert orc.query(info, data, dup).all()


def test_function_with_conflicting_duplicates_fails(orc):
    # a key given twice with two values makes two equations with the same left
    # side and different right sides (eq. MWHC): no seed solves it, so the build
    # stops at the first attempt with ORC_EDUP instead of retrying
    keys = synth.u64_keys(0, 1000, 5)
    dup = np.concatenate([keys, keys[:1]])
    vals = np.zeros(1001, dtype=np.uint8)
    vals[-1] = 1
    for mode in (orc.MODE_AUTO, orc.MODE_FUSE, orc.MODE_MWHC):
        for seed in (0, 1, 7):
            st, info, _ = orc.build(orc.default_params(max_retries=2, mode=mode, seed=seed), dup, vals)
            assert st == orc.EDUP and info.retries == 0 and info.seed == seed, (mode, seed)


def _lge_sharded(orc, **kw):
    return orc.default_params(mode=orc.MODE_LGE, lge_target=1024, **kw)


@pytest.mark.parametrize("regime", ["lge_unsharded", "lge_sharded", "fuse", "mwhc"])
def test_function_repeated_pairs_are_dropped(orc, regime):
    # Sec. 4.4: the local signature stands for the key inside its shard. A
    # function given the same (key, value) pair several times describes the
    # same function as one given it once: one copy of each equation is kept
    # (n_eff counts the distinct keys; the largest shard M, and with it the
    # geometry, counts every key given), and every key decodes to its value
    # (Problem 1).
    n = {"lge_unsharded": 6000, "lge_sharded": 20_000, "fuse": 3000, "mwhc": 30_000}[regime]
    keys = synth.u64_keys(0, n, 41)
    vals = synth.values(n, 8, 41)
    rng = np.random.default_rng(41)
    rep = rng.integers(0, n, size=n // 4)
    dk = np.concatenate([keys, keys[rep], keys[rep[:50]]])
    dv = np.concatenate([vals, vals[rep], vals[rep[:50]]])
    perm = rng.permutation(len(dk))
    dk, dv = dk[perm], dv[perm]
    kw = {"lge_unsharded": dict(), "lge_sharded": dict(mode=orc.MODE_LGE, lge_target=1024),
          "fuse": dict(mode=orc.MODE_FUSE, max_retries=60), "mwhc": dict(mode=orc.MODE_MWHC, eps=0.01, eta=1e-3,
                                                                       max_retries=60)}[regime]
    for seed in (3, 4):
        st, info, data = orc.build(orc.default_params(seed=seed, **kw), dk, dv)
        assert st == orc.OK
        assert info.n == len(dk) and info.n_eff == n and info.seed == seed + info.retries
        assert (orc.query(info, data, dk) == dv).all()
        # the same structure decodes the distinct keys: it is their function
        assert (orc.query(info, data, keys) == vals).all()


def test_byte_string_function_duplicates(orc):
    data_, offs = synth.byte_strings(0, 3000, 12)
    vals = synth.values(3000, 16, 12)
    # repeat string 7 with its value, and string 9 with another value
    strs = [bytes(data_[offs[i]:offs[i + 1]]) for i in range(3000)]
    for extra, ok in (([(7, vals[7])], True), ([(7, vals[7]), (9, vals[9] ^ 1)], False)):
        s2 = strs + [strs[i] for i, _ in extra]
        v2 = np.concatenate([vals, np.array([v for _, v in extra], dtype=vals.dtype)])
        o2 = np.zeros(len(s2) + 1, dtype=np.uint64)
        o2[1:] = np.cumsum([len(x) for x in s2])
        buf = np.frombuffer(b"".join(s2), dtype=np.uint8)
        st, info, data = orc.build(orc.default_params(b=16, key_kind=orc.KEYS_BYTES, seed=2), buf, v2, offsets=o2)
        if ok:
            assert st == orc.OK and info.n_eff == 3000
            assert (orc.query(info, data, buf, offsets=o2) == v2).all()
        else:
            assert st == orc.EDUP


def test_threads_give_the_same_structure(orc):
    # shards are independent systems (Sec. 4): solving them on a pool of threads
    # changes nothing in the result; bit-array cells (b = 13) share bytes across
    # shard boundaries
    cases = [(orc.FUNC, 8, dict(mode=orc.MODE_LGE, lge_target=2048), 40_000),
             (orc.FUNC, 13, dict(mode=orc.MODE_MWHC, eps=0.01, eta=1e-3), 100_000),
             (orc.FILTER, 8, dict(mode=orc.MODE_MWHC, eps=0.01, eta=1e-3), 100_000),
             (orc.FUNC, 5, dict(mode=orc.MODE_LGE, lge_target=1024), 20_000)]
    for kind, b, kw, n in cases:
        keys = synth.u64_keys(0, n, 17)
        vals = synth.values(n, b, 17) if kind == orc.FUNC else None
        st1, i1, d1 = orc.build(orc.default_params(kind=kind, b=b, seed=5, **kw), keys, vals)
        st4, i4, d4 = orc.build(orc.default_params(kind=kind, b=b, seed=5, threads=4, **kw), keys, vals)
        assert st1 == st4 == orc.OK and i1.h > 0
        assert i1.as_dict() == i4.as_dict()
        assert (d1 == d4).all()
        other = synth.u64_keys(n, n, 17)
        assert (orc.query(i1, d1, other) == orc.query(i1, d1, other, threads=5)).all()


# ------------------------------------------- LGE-regime hypergraphs (reading)

def _gf2_consistent(rows, rhs, nbits):
    """Rank test over GF(2), bit plane by bit plane: [A] and [A | v] have the
    same rank. rows: vertex sets as Python integer bit masks."""
    for j in range(nbits):
        piv = {}
        for r, v in zip(rows, rhs):
            x, y = r, (int(v) >> j) & 1
            while x:
                top = x.bit_length() - 1
                if top not in piv:
                    piv[top] = (x, y)
                    break
                px, py = piv[top]
                x, y = x ^ px, y ^ py
            if x == 0 and y == 1:
                return False
    return True


def _rows(e):
    return [(1 << int(a)) ^ (1 << int(c)) ^ (1 << int(d)) for a, c, d in e]


def test_lge_regime_uses_uniform_triples_not_small_fuse_graphs(orc):
    # Sec. 4.2 keeps c = 1.12 for small sizes with LGE. A fuse graph with l
    # start segments and c = 1.12 has (l + 2) / (l c) equations per vertex away
    # from its ends; with eq. (ln) segments at 1000 keys (l = 7) that is 1.15,
    # above the ~0.918 GF(2) solvability threshold of random 3-uniform systems,
    # so the system is inconsistent (rank test); three distinct uniform
    # vertices over the same ceil(1.12 n) cells are consistent.
    M = 1000
    lg = math.floor(math.log(M) / math.log(3.33) + 2.25)
    fuse = orc.geometry(orc.REGIME_FUSE, 0, M)
    assert fuse.lg_seg == lg == 7 and fuse.c == 1.12 and fuse.l == 7
    uni = orc.geometry(orc.REGIME_LGE, 0, M)
    assert uni.cells == math.ceil(1.12 * M)
    for r in range(4):
        loc = synth.u64_keys(0, M, 900 + r)
        rhs = synth.values(M, 1, 900 + r)
        assert not _gf2_consistent(_rows(orc.edges_of(fuse, loc)), rhs, 1)
        assert _gf2_consistent(_rows(orc.edges_of(uni, loc)), rhs, 1)


def test_lge_success_matches_gf2_rank(orc):
    # Sec. 3.3: a shard is solvable iff its system is consistent. Small builds
    # (40 keys in 45 cells, b = 2) fail often enough to see both outcomes; the
    # oracle's first attempt must succeed exactly when the rank test on its
    # edges says the system is consistent.
    n, b = 40, 2
    seen = {True: 0, False: 0}
    for seed in range(120):
        keys = synth.u64_keys(0, n, 1000 + seed)
        vals = synth.values(n, b, 1000 + seed)
        st, info, data = orc.build(orc.default_params(b=b, seed=seed, max_retries=0), keys, vals)
        geo = orc.geometry(orc.REGIME_LGE, 0, n)
        e = orc.edges_of(geo, orc.sigs(keys, seed)[:, 0])
        want = _gf2_consistent(_rows(e), vals, b)
        assert (st == orc.OK) == want, seed
        seen[want] += 1
        if st == orc.OK:
            assert info.regime == orc.REGIME_LGE and info.h == 0
            assert (orc.query(info, data, keys) == vals).all()
    assert seen[True] > 0 and seen[False] > 0, seen


def test_retry_restarts_with_next_seed(orc):
    # Sec. 4: a failure restarts the whole construction; find a seed whose
    # first attempt fails (tiny forced fuse graphs fail often) and check the
    # reported seed is the first one that succeeds.
    keys = synth.u64_keys(0, 400, 3)
    vals = synth.values(400, 8, 3)
    seen = 0
    for seed in range(40):
        st, info, data = orc.build(orc.default_params(mode=orc.MODE_FUSE, seed=seed, max_retries=50), keys, vals)
        assert st == orc.OK
        assert info.seed == seed + info.retries
        assert (orc.query(info, data, keys) == vals).all()
        seen += info.retries > 0
    assert seen > 0


def test_small_structure_overhead(orc):
    # Sec. 7: 11-12% overhead for small sizes: an unsharded LGE structure has c = 1.12
    g = dict(golden("overhead.txt"))
    lo, hi = float(g["small_low"]), float(g["small_high"])
    n = 5000
    keys = synth.u64_keys(0, n, 6)
    st, info, _ = orc.build(orc.default_params(seed=1), keys, synth.values(n, 8, 6))
    assert st == orc.OK and info.h == 0 and info.regime == orc.REGIME_LGE
    assert lo - 0.01 <= info.total_cells / n - 1 <= hi + 0.001
    for n in (50_000, 500_000):
        info = orc.geometry(orc.REGIME_LGE, 0, n)
        assert lo - 0.01 <= info.total_cells / n - 1 <= hi + 0.001


# ------------------------------------------------------------------ MWHC (Sec. 4.1)

def test_mwhc_planner_reproduces_paper_example(orc):
    # the planner in MWHC mode combines eq. (dupmwhc) with eq. (logballsbins): at
    # 10^12 keys, eps = 0.01, eta = 10^-3 the duplicate bound wins with 8192 shards
    for keys, c, eta, shards in golden("mwhc_shard_example.txt"):
        p = orc.default_params(mode=orc.MODE_MWHC, eps=0.01, eta=float(eta))
        h, regime, h_bb, h_dup = orc.plan_h(p, int(keys))
        assert regime == orc.REGIME_MWHC and 1 << h == int(shards) and h == h_dup < h_bb
        # eq. (logballsbins) directly: x = n eps^2 / 2, h_bb = floor(lg x - lg ln x)
        x = int(keys) * 0.01**2 / 2
        assert h_bb == math.floor(math.log2(x) - math.log2(math.log(x)))
    # small n: the balls-and-bins bound is the smaller one (no sharding below e)
    p = orc.default_params(mode=orc.MODE_MWHC, eps=0.01, eta=1e-3)
    h, regime, h_bb, h_dup = orc.plan_h(p, 20_000)
    assert regime == orc.REGIME_MWHC and h == h_bb == 0


def test_mwhc_geometry_three_parts_23_percent(orc):
    # Sec. 4.1: 3-partite hypergraph with c = 1.23 -> ~23% space overhead
    for M in (10_000, 1_000_003, 123_456_789):
        info = _info(orc, orc.REGIME_MWHC, 0, M)
        assert info.c == 1.23 and info.cells % 3 == 0
        assert info.cells == 3 * math.ceil(1.23 * M / 3)
        assert 0.23 - 1e-12 <= info.cells / M - 1 < 0.23 + 3.0 / M
    # tiny shards: at least 16 vertices per part
    assert _info(orc, orc.REGIME_MWHC, 0, 2).cells == 48


def test_mwhc_edges_one_per_part_uniform(orc):
    info = _info(orc, orc.REGIME_MWHC, 0, 3000)
    P = info.cells // 3
    loc = synth.u64_keys(0, 60_000, 12)
    e = orc.edges_of(info, loc).astype(np.int64)
    for k in range(3):
        assert ((e[:, k] >= k * P) & (e[:, k] < (k + 1) * P)).all()
        cnt = np.bincount(e[:, k] - k * P, minlength=P)
        exp_ = len(loc) / P
        dof = P - 1
        assert ((cnt - exp_) ** 2 / exp_).sum() < dof + 6 * math.sqrt(2 * dof)
    # the three coordinates are independent: the pair (v0, v1) is uniform over
    # B x B bins of (nearly) equal size; expected counts from the exact bin sizes
    B = 30
    b0 = e[:, 0] * B // P
    b1 = (e[:, 1] - P) * B // P
    cnt = np.bincount(b0 * B + b1, minlength=B * B).astype(float)
    size = np.bincount(np.arange(P) * B // P, minlength=B) / P
    exp_ = len(loc) * np.outer(size, size).ravel()
    dof = B * B - 1
    assert ((cnt - exp_) ** 2 / exp_).sum() < dof + 6 * math.sqrt(2 * dof)


def test_mwhc_duplicate_rate_matches_paper_estimate(orc):
    # Sec. 4.1: (cm/3)^3 possible edges; expected duplicate pairs m(m-1)/2 / P^3,
    # no-duplicate probability ~ exp(-1 / (2 (c/3)^3 m)). Monte Carlo, small parts.
    m = 200
    info = _info(orc, orc.REGIME_MWHC, 0, m)
    info.cells = 3 * 20  # P = 20 (forced) -> lambda ~ 2.5
    P = 20
    trials, dups = 200, []
    for t in range(trials):
        e = orc.edges_of(info, synth.u64_keys(t * m, m, 13))
        _, c = np.unique(e, axis=0, return_counts=True)
        dups.append(int((c * (c - 1) // 2).sum()))
    lam = m * (m - 1) / 2 / P**3
    mean = np.mean(dups)
    assert abs(mean - lam) < 5 * math.sqrt(lam / trials), (mean, lam)
    # the paper's closed form with c = 3P/m
    cc = 3 * P / m
    assert abs(lam - 1 / (2 * (cc / 3) ** 3 * m) * (m - 1) / m) / lam < 1e-9


@pytest.mark.parametrize("kind,b", [(0, 8), (0, 13), (1, 8), (1, 16)])
def test_mwhc_build_decodes_sharded(orc, kind, b):
    # eps forced up so that 200k keys shard; every key decodes (Problem 1) or is
    # accepted (Problem 2), and the structure is 3-partite with c = 1.23
    n = 200_000
    keys = synth.u64_keys(0, n, 14)
    vals = synth.values(n, b, 14) if kind == 0 else None
    p = orc.default_params(kind=kind, b=b, mode=orc.MODE_MWHC, eps=0.05, eta=1e-3, seed=3)
    st, info, data = orc.build(p, keys, vals)
    assert st == orc.OK and info.regime == orc.REGIME_MWHC and info.h >= 1
    assert info.peeled == info.n_eff == n and info.core == 0
    q = orc.query(info, data, keys)
    assert (q == vals).all() if kind == 0 else q.all()
    if kind == 1:
        other = orc.query(info, data, synth.u64_keys(n, 200_000, 14))
        pr = 2.0 ** -b
        assert abs(other.mean() - pr) < 5 * math.sqrt(pr * (1 - pr) / 200_000) + 1e-9



# ------------------------------------------------------------- wide values (b > 32)

@pytest.mark.parametrize("b", [33, 40, 63])
def test_bit_array_cells_wider_than_a_word(orc, b):
    # Sec. 5 bit array: cell i holds bits [i*b, (i+1)*b); b > 32 cells straddle
    # 32- and 64-bit words. Reading back a build's cells one bit at a time
    # (independently of orc_cell_get) gives the same values.
    n = 3000
    keys = synth.u64_keys(0, n, 61)
    vals = synth.values(n, b, 61)
    st, info, data = orc.build(orc.default_params(b=b, seed=2), keys, vals)
    assert st == orc.OK and info.data_bytes == ((info.total_cells * b + 63) // 64 + 1) * 8
    bits = np.unpackbits(data, bitorder="little")
    for i in range(0, info.total_cells, 97):
        want = 0
        for j in range(b):
            want |= int(bits[i * b + j]) << j
        assert orc.lib().orc_cell_get(data.ctypes.data, b, i) == want


def test_wide_filter_fingerprints_and_no_false_negatives(orc):
    # Problem 2 with b = 33 and 64: fingerprints are the top b bits of the remix;
    # members always pass, non-members almost never (FPR 2^-33 / 2^-64)
    n = 50_000
    keys = synth.u64_keys(0, n, 62)
    other = synth.u64_keys(n, 200_000, 62)
    for b in (33, 64):
        st, info, data = orc.build(orc.default_params(kind=orc.FILTER, b=b, seed=1), keys)
        assert st == orc.OK
        assert orc.query(info, data, keys).all() and orc.query(info, data, other).sum() == 0
        f = orc.fingerprint(int(keys[0]), b)
        assert f >> b == 0 and orc.fingerprint(int(keys[0]), 32) == f >> (b - 32)


# ------------------------------------------- 4-uniform fuse graphs (Sec. 4.2, k = 4)

def _random_hypergraph_k(rng, V, m, k):
    return np.array([rng.choice(V, size=k, replace=False) for _ in range(m)], dtype=np.uint32).reshape(m, k)


def test_peel4_matches_bruteforce_2core(orc):
    rng = np.random.default_rng(13)
    for trial in range(250):
        V = int(rng.integers(5, 10))
        m = int(rng.integers(1, 11))
        edges = _random_hypergraph_k(rng, V, m, 4)
        ne, order, side = orc.peel(V, edges)
        core = _brute_core(V, edges.tolist())
        assert m - ne == len(core)
        peeled = [int(e) for e in order]
        for i, e in enumerate(peeled):
            v = int(edges[e][side[i]])
            later = peeled[i + 1:] + sorted(core)
            assert all(v not in edges[f].tolist() for f in later)


def test_gf2_solve4_matches_bruteforce(orc):
    rng = np.random.default_rng(14)
    for trial in range(200):
        V = int(rng.integers(4, 9))
        m = int(rng.integers(1, 12))
        edges = _random_hypergraph_k(rng, V, m, 4)
        rhs = rng.integers(0, 2, size=m).astype(np.uint64)
        ok, w = orc.gf2_solve(V, edges, rhs)
        found = any(all((sum(assign[v] for v in edges[i]) & 1) == rhs[i] for i in range(m))
                    for assign in itertools.product((0, 1), repeat=V))
        assert ok == found
        if ok:
            for i in range(m):
                assert (int(w[edges[i][0]]) ^ int(w[edges[i][1]]) ^ int(w[edges[i][2]]) ^ int(w[edges[i][3]])) == rhs[i]


def test_fuse4_edges_in_four_consecutive_segments(orc):
    # Sec. 4.2's fuse graph of arity k = 4: a start segment s in [0, l) and
    # one vertex in each of segments s, s+1, s+2, s+3 (l + 3 segments)
    info = orc.geometry(orc.REGIME_FUSE, 0, 200_000, k=4)
    assert info.k == 4 and info.T == info.l + 3 and info.cells == info.T * info.seg
    loc = np.sort(synth.u64_keys(0, 60_000, 15))
    e = orc.edges_of(info, loc).astype(np.int64)
    assert e.shape == (60_000, 4)
    seg = int(info.seg)
    s = e[:, 0] // seg
    assert (s < info.l).all() and (e < info.cells).all()
    for k in range(1, 4):
        assert ((e[:, k] // seg) == s + k).all()
    assert (np.diff(e[:, 0]) >= 0).all()  # monotone in the local signature (Sec. 4.5)
    for cnt, n_bins in ((np.bincount(s, minlength=info.l), info.l), (np.bincount(e[:, 3] % seg, minlength=seg), seg)):
        exp_ = len(loc) / n_bins
        assert ((cnt - exp_) ** 2 / exp_).sum() < (n_bins - 1) + 6 * math.sqrt(2 * (n_bins - 1))


def test_fuse4_duplicate_edge_rate_matches_paper_estimate(orc):
    # Sec. 4.2's count of possible edges with k = 4: about l * s^4, so the
    # expected number of duplicate pairs is m (m - 1) / 2 / (l s^4); Monte Carlo
    # with tiny segments
    m = 2000
    info = orc.geometry(orc.REGIME_FUSE, 0, m, k=4)
    info.lg_seg, info.seg = 2, 4
    info.T = math.ceil(1.1 * m / 4)
    info.l = info.T - 3
    info.cells = info.T * 4
    trials, dups = 60, []
    for t in range(trials):
        e = orc.edges_of(info, synth.u64_keys(t * m, m, 16))
        _, c = np.unique(e, axis=0, return_counts=True)
        dups.append(int((c * (c - 1) // 2).sum()))
    lam = m * (m - 1) / 2 / (info.l * 4**4)
    assert abs(np.mean(dups) - lam) < 5 * math.sqrt(lam / trials), (np.mean(dups), lam)


def test_fuse4_shards_by_ballsbins_and_uses_less_space(orc):
    # k = 4: duplicate edges (exp(-m / (2 c s^3))) never bind, so the shard bits
    # are eq. (logballsbins)'s; the space overhead is below the 3-uniform one at
    # the same shard size (Sec. 7: one more probe for a smaller overhead)
    p3, p4 = orc.default_params(mode=orc.MODE_FUSE), orc.default_params(mode=orc.MODE_FUSE, arity=4)
    for n in (10**8, 10**10, 10**12):
        h3, _, hbb, _ = orc.plan_h(p3, n)
        h4, reg, hbb4, hdup4 = orc.plan_h(p4, n)
        assert reg == orc.REGIME_FUSE and h4 == hbb4 == hbb and hdup4 == -1 and h4 >= h3
    for M in (200_000, 12_500_000, 100_000_000):
        g3 = orc.geometry(orc.REGIME_FUSE, 3, M)
        g4 = orc.geometry(orc.REGIME_FUSE, 3, M, k=4)
        assert g4.total_cells < g3.total_cells, M
        info = orc.geometry(orc.REGIME_FUSE, 3, M, k=4)
        s = info.seg
        # the shard's cells are c M rounded up to whole segments
        assert info.c * M <= info.cells < info.c * M + s + 1


@pytest.mark.parametrize("kind,b,n,kw", [("func", 8, 300_000, {}), ("func", 13, 300_000, {}),
                                         ("filter", 8, 2_000_000, {}), ("func", 16, 3_000_000, {"eps": 0.01})])
def test_build_fuse4_decodes(orc, kind, b, n, kw):
    # Problem 1 / Problem 2 with 4-uniform fuse graphs: every key decodes, no
    # false negatives, FPR ~ 2^-b on disjoint keys; eps = 0.01 shards the keys
    keys = synth.u64_keys(0, n, 17)
    vals = synth.values(n, b, 17) if kind == "func" else None
    p = orc.default_params(kind=orc.FUNC if kind == "func" else orc.FILTER, b=b, mode=orc.MODE_FUSE, arity=4,
                           seed=3, threads=4, **kw)
    st, info, data = orc.build(p, keys, vals)
    assert st == orc.OK and info.k == 4 and info.regime == orc.REGIME_FUSE and info.core == 0
    if "eps" in kw:
        assert info.h > 0
    out = orc.query(info, data, keys)
    if kind == "func":
        assert (out == vals).all()
    else:
        assert out.all()
        other = synth.u64_keys(n, 1_000_000, 17)
        fpr = orc.query(info, data, other).mean()
        pb = 2.0**-b
        assert abs(fpr - pb) < 5 * math.sqrt(pb * (1 - pb) / len(other))
