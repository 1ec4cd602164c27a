"""The pipe-rate probe on the device: rates in results per SM clock that a
Blackwell SM can issue (4 SMSPs x 32 FP32 lanes = 128 FP32 fma per clock at
most; the special-function unit far fewer), reproducible between calls."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_physical(gac):
    r = {op: gac.gac_pipe_rate(op) for op in gac.PIPE_OPS}
    print({k: round(v, 2) for k, v in r.items()})
    assert 100.0 <= r["ffma"] <= 130.0
    assert 100.0 <= r["ffma2"] <= 260.0
    for op in ("ex2", "sin", "lg2", "rsqrt", "rcp", "sqrt"):
        assert 4.0 <= r[op] <= 64.0, op
    assert 0.0 < r["dfma"] <= 64.0
    assert 8.0 <= r["imad_hi"] <= 130.0
    assert 32.0 <= r["lop3"] <= 130.0
    again = gac.gac_pipe_rate("sin")
    assert again == pytest.approx(r["sin"], rel=0.05)
