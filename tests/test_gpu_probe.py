"""The integer-issue probe (cdef_probe_int_mix), the measured ceiling the
bench reports the filter against: plausible rates and argument errors."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cdef():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1602_05975_gb300 import build, cdef as _c
    build.build()
    _c.load()
    return _c


def test_probe_rates_are_plausible(cdef):
    ctx = cdef.Context(0)
    try:
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        # one warp instruction per clock per scheduler, 4 schedulers of 32
        # lanes per SM, at most 2.2 GHz
        issue_limit = sms * 128 * 2.2e9
        mix = cdef.probe_int_mix(ctx, 0)
        alu = cdef.probe_int_mix(ctx, 1)
        assert 0.2 * issue_limit < mix <= 1.05 * issue_limit
        # the ALU pipe takes half the lanes of the issue rate
        assert 0.1 * issue_limit < alu <= 0.55 * issue_limit
        # the multiply-adds of the tap mix issue beside the ALU operations
        assert mix > alu
        # the single-pipe mixes: every rate within the issue limit; fp32 FMAs
        # (two pipes) faster than integer multiply-adds (one), and
        # multiplies-high slower than multiply-adds
        rates = [cdef.probe_int_mix(ctx, m) for m in range(2, 7)]
        assert all(0.05 * issue_limit < r <= 1.05 * issue_limit for r in rates)
        imad, hi, fma = rates[0], rates[1], rates[4]
        assert fma > imad > hi
    finally:
        ctx.close()


def test_probe_rejects_bad_arguments(cdef):
    ctx = cdef.Context(0)
    try:
        for mix, iters in ((7, 16), (-1, 16), (0, 0), (0, 1 << 21)):
            with pytest.raises(cdef.CdefError):
                cdef.probe_int_mix(ctx, mix, iters)
    finally:
        ctx.close()
