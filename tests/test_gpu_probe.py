"""The FP32 FMA throughput probe (the measured denominator beside the derived
FP32 peak of the trace kernel's roofline)."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2012_10357_b300 as pr  # noqa: E402


def test_fma_probe_is_near_the_derived_peak():
    tflops, ms = pr.fma_peak_probe(16384)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    derived = props.multi_processor_count * 128 * 2 * 2032e6 / 1e12   # at the maximum SM clock
    assert ms > 0.0
    assert 0.3 * derived < tflops < 1.1 * derived


def test_fma_probe_rejects_bad_arguments():
    with pytest.raises(pr.PrError):
        pr.fma_peak_probe(0)
