"""The roofline calibration micro-benchmarks run and give rates of the right
order for a GB300-class GPU (FP32 FMA tens of TFLOP/s, FP64 around one
TFLOP/s, L2 reads several TB/s); bad kinds are rejected."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0801_1500_gb300 import gbrt
    return gbrt


def test_microbench_rates(G):
    with G.Renderer(0) as r:
        fp32 = G.gbrt_microbench(r.ctx, G.MB_FP32_FMA)
        fp64 = G.gbrt_microbench(r.ctx, G.MB_FP64_FMA)
        l2 = G.gbrt_microbench(r.ctx, G.MB_L2_READ)
        print("microbench", fp32, fp64, l2)
        assert 10.0 < fp32 < 200.0
        assert 0.05 < fp64 < 20.0
        assert fp32 > 8 * fp64
        assert 1000.0 < l2 < 100000.0
        with pytest.raises(G.GbrtError):
            G.gbrt_microbench(r.ctx, 7)
