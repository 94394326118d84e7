"""The roofline arithmetic of bench.py, on CPU: algorithmic bytes per unit (a
stream at its size, every random vertex or cell update one 32-byte sector read
and one written back, every random read one sector), units per phase (keys x
attempts for the per-attempt phases, keys x builds for assignment, 2n per step
for queries), achieved = bytes x units / time, frac = achieved / peak. The phase
times are those of one default bench line (VFilter, 10^8 keys, b = 8, 20 timed
steps, 29 attempts)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N = 10**8
STEPS = 20
HBM = 6785.2
# phase -> (ms over the timed steps, kernel launches)
PHASES = {"hash_hist": (5.952, 29), "scatter": (70.845, 116), "incidence": (41.529, 29),
          "peel": (969.249, 87), "assign": (211.241, 40), "query": (80.619, 40)}


def _gbs(bytes_per_unit, units, ms):
    return bytes_per_unit * units / (ms * 1e-3) / 1e9


def test_algorithmic_bytes_per_unit():
    # filter, b = 8: no value stream; 3-uniform edges
    assert bench._algo("hash_hist", 8, "filter", 3) == 8.0            # key read
    assert bench._algo("scatter", 8, "filter", 3) == 16.0             # local signature written and read
    assert bench._algo("incidence", 8, "filter", 3) == 8.0 + 3 * 64   # signature + 3 vertex RMW sectors
    assert bench._algo("peel", 8, "filter", 3) == 3 * 64.0            # 3 vertex RMW sectors
    assert bench._algo("assign", 8, "filter", 3) == pytest.approx(4 * 64 + 1.105)
    assert bench._algo("query", 8, "filter", 3) == 8 + 3 * 32 + 1     # 105 B: key, 3 sectors, 1 byte out
    # a function carries its value through the scatter and the assignment
    assert bench._algo("scatter", 16, "func", 3) == 8 + 2 + 8 + 2
    assert bench._algo("assign", 16, "func", 3) == pytest.approx(2 + 4 * 64 + 1.105 * 2)
    # 4-uniform: one more vertex update per edge, one more sector per query
    assert bench._algo("peel", 8, "filter", 4) == 4 * 64.0
    assert bench._algo("incidence", 8, "filter", 4) == 8.0 + 4 * 64
    assert bench._algo("query", 8, "filter", 4) == 8 + 4 * 32 + 1


def test_phase_table_against_a_recorded_line():
    per, dom, roof = bench.phase_table(PHASES, N, STEPS, 8, "filter", HBM, "measured", "c2", True, 3)
    attempts = 29
    assert dom == "peel"
    assert per["peel"]["passes"] == attempts and per["assign"]["passes"] == STEPS
    assert per["query"]["passes"] == 2 * STEPS
    assert per["peel"]["achieved_gbs"] == pytest.approx(_gbs(192, N * attempts, 969.249), abs=0.01)
    assert per["peel"]["achieved_gbs"] == pytest.approx(574.47, abs=0.01)  # the line's own figure
    assert per["assign"]["achieved_gbs"] == pytest.approx(_gbs(256 + 1.105, N * STEPS, 211.241), abs=0.01)
    assert per["query"]["achieved_gbs"] == pytest.approx(_gbs(105, 2 * N * STEPS, 80.619), abs=0.01)
    assert sum(p["share"] for p in per.values()) == pytest.approx(1.0, abs=1e-3)
    assert roof["kernel"] == "peel" and roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert roof["peak"] == HBM
    assert roof["frac"] == pytest.approx(574.47 / HBM, abs=1e-4)
    assert roof["algorithmic_bytes_per_unit"] == 192
    # the peel's DRAM traffic per launch: a 2e7-key capture scaled to 1e8 keys
    assert roof["traffic"] == round(1120.07e6 / 2e7 * 1e8)


def test_whole_build_models():
    # C2: key read twice (16) + local signature written and read (16) + data array
    # c b / 8 = 1.105 bytes: 33.1 B per key; plus 10 random sector RMWs: 673.1
    r = bench.build_roofline(65.467, N, 8, "filter", 1.105, HBM, "measured", True, 29 / 20)
    assert r["streaming"]["bytes_per_key"] == pytest.approx(33.1, abs=0.01)
    assert r["streaming_plus_random_sectors"]["bytes_per_key"] == pytest.approx(673.1, abs=0.01)
    assert r["streaming"]["bound_ns_per_key"] == pytest.approx(33.105 / HBM, abs=1e-5)
    assert r["streaming"]["achieved"] == pytest.approx(33.105 * N / 65.467e-3 / 1e9, abs=0.01)
    assert r["attempts_per_build"] == 1.45


def test_random_sector_query_model():
    q = bench.random_sector_roofline(15e9, 8, "filter", HBM, "measured")
    assert q["bytes_per_query"] == 105 and q["achieved"] == pytest.approx(105 * 15.0, abs=0.01)
    assert q["sectors_per_s"] == pytest.approx(45.0) and q["sector_peak_per_s"] == pytest.approx(HBM / 32, abs=1e-3)
    q4 = bench.random_sector_roofline(10e9, 8, "filter", HBM, "measured", k=4)
    assert q4["bytes_per_query"] == 137 and q4["sectors_per_s"] == pytest.approx(40.0)


def test_job_rates_aggregate_over_replicas():
    ns, gq = bench.job_rates(65.0, 4.0, N, 4)  # 4 replicas of 1e8 keys
    assert ns == pytest.approx(65.0e6 / (4 * N)) and gq == pytest.approx(8 * N / 4e-3 / 1e9)
