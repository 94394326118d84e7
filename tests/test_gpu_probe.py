"""The random-sector probe behind the query's roofline: a positive rate,
higher for a table that fits in L2 than for one that does not, and invalid
arguments rejected."""
import pytest

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


def test_sector_rate_l2_above_hbm(vf):
    small = vf.vf_sector_rate(32 << 20)
    large = vf.vf_sector_rate(2 << 30)
    assert small > 0 and large > 0
    assert small > 1.5 * large, (small, large)
    with pytest.raises(vf.VFError) as e:
        vf.vf_sector_rate(100)
    assert e.value.status == 1
