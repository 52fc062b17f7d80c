"""rd_probe_mma: the BF16 tcgen05 MMA rate with nothing else in the loop (the ceiling the split
GEMM is measured against) is positive and below the nominal dense peak; the INT8 kind, which does
not exist for sm_103a, is refused with RD_ERR_UNSUPPORTED."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2308_07403_gb300 import build
    from paper_2308_07403_gb300 import rd as _rd

    build.build()
    _rd.load()
    return _rd


def test_probe_bf16_rate_and_int8_refusal(rd):
    rate, seconds = rd.rd_probe_mma(0, 500)
    assert seconds > 0.0
    assert 100.0 < rate < 2600.0  # TFLOP/s: the nominal dense BF16 peak is 2250
    with pytest.raises(rd.RDError) as ei:
        rd.rd_probe_mma(1, 1)
    assert ei.value.status == rd.RD_ERR_UNSUPPORTED
    assert "kind::i8" in rd.rd_last_error()
