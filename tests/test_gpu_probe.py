"""The pipe-rate probe (include/vx_probe.h), through the C ABI: it runs, and its per-SM-per-clock
rates fall in the ranges a Blackwell SM can deliver (FP32 FMA 128 lanes per clock nominal, FP64
a small fraction of it, MUFU ex2 and rcp a fraction of FP32, warp-level MMAs below the dense
tensor-core rate). These are sanity bounds on the measurement, wide enough for clock noise, not a
characterisation of the part."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1404_1719_gb300 import _build, capi
    _build.build()
    r = capi.vx_probe_pipes(torch.cuda.current_stream().cuda_stream)
    assert r["n_sm"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 200.0 < r["sm_mhz"] < 2300.0
    assert 64.0 < r["ffma"] <= 140.0 and 64.0 < r["ffma2"] <= 280.0
    assert 0.1 < r["dfma"] < r["ffma"] / 4
    assert 4.0 < r["ex2"] < r["ffma"] and 2.0 < r["rcp"] < r["ffma"]
    # dense BF16 on the tensor cores: 2.25 PFLOP/s nominal = ~3,600 multiply-adds per SM per clock
    assert 32.0 < r["mma_tf32"] < 4000.0 and 32.0 < r["mma_bf16"] < 8000.0
