"""The bench-only throughput probes (bench_probes, not part of libsnn) behind the roofline denominators return rates in
the range the GB300's units allow (152 SMs at up to 2.07 GHz): the tcgen05
e4m3 MMA near twice the BF16 one, FP64 far below FP32."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probes():
    import bench_probes
    return bench_probes


def test_probe_rates_are_plausible(probes):
    r = {k: max(probes.measure_peak(k, it) for _ in range(3)) / 1e12
         for k, it in [("bf16_mma", 1 << 14), ("e4m3_mma", 1 << 14), ("fp32_fma", 1 << 15),
                       ("fp64_fma", 1 << 10)]}
    # nominal dense: BF16 2250, e4m3 4500, FP32 152 x 128 x 2 x 2.07 GHz = 80.5 TFLOP/s
    assert 300 < r["bf16_mma"] < 2600, r
    assert 1.5 < r["e4m3_mma"] / r["bf16_mma"] < 2.5, r
    assert 10 < r["fp32_fma"] < 90, r
    assert r["fp64_fma"] < r["fp32_fma"] / 4, r


def test_probe_rejects_bad_arguments(probes):
    from paper_2212_07679_gb300 import snn
    with pytest.raises(KeyError):
        probes.measure_peak("int8_mma", 1024)
    with pytest.raises(snn.SNNError):
        probes.measure_peak("bf16_mma", 8)
