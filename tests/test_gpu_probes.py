"""The measurement probes the bench's rooflines rest on: every instruction kind reports a positive
rate within what one GB300 can issue (152 SMs x 128 lanes x 2.07 GHz per kind of instruction), the
palette-evaluation mix at least as fast as its slowest single kind, and an unknown kind is refused
with nothing run."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2607_14513_gb300 import gsc
    c = gsc.Context(0)
    yield c
    c.close()


def test_op_rates(ctx):
    from paper_2607_14513_gb300 import gsc
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2.2e9
    rates = {k: gsc.op_rate(ctx, k) for k in gsc.PROBE_KINDS}
    for k, v in rates.items():
        assert 0 < v <= 3 * ceiling, (gsc.PROBE_KINDS[k], v)
    assert rates[5] >= 0.9 * min(rates[k] for k in (3, 4))
    for bad in (0, 6, -1):
        with pytest.raises(gsc.GscError):
            gsc.op_rate(ctx, bad)
