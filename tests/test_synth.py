"""The device key generator draws the same keys as the host one."""
import numpy as np

from paper_2503_18397_gb300 import synth


def test_torch_keys_equal_numpy_keys():
    for start, count, seed in [(0, 1000, 0), (12345, 777, 7), (2**40, 513, 99)]:
        a = synth.u64_keys(start, count, seed)
        b = synth.u64_keys_torch(start, count, seed, device="cpu").numpy().view(np.uint64)
        assert (a == b).all()


def test_keys_distinct_and_disjoint_ranges():
    a = synth.u64_keys(0, 100_000, 3)
    b = synth.u64_keys(100_000, 100_000, 3)
    assert len(np.unique(np.concatenate([a, b]))) == 200_000


def test_value_widths():
    for b in (1, 8, 13, 16, 32):
        v = synth.values(10_000, b, 5)
        assert int(v.max()) < (1 << b)
        t = synth.values_torch(10_000, b, 5, device="cpu")
        assert t.element_size() == v.dtype.itemsize
