"""The arithmetic-rate probes (invdft_peak_probe) run and give rates in the
range this part's units and clocks allow (needs a B300; marked gpu): FP64 FMA
well below FP32 (the FP64 pipe of this part is a small fraction of FP32),
packed FP32 pairs not slower than scalar FP32, and all below the nominal
2.25 PFLOP/s of the dense BF16 tensor rate."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_peak_probes_give_plausible_rates():
    import paper_2510_10529_b300 as P
    r = {k: P.invdft_peak_probe(k) for k in ("fp64", "fp32", "fp32x2", "tf32")}
    print("measured TFLOP/s:", {k: round(v, 2) for k, v in r.items()})
    assert 0.2 < r["fp64"] < 0.5 * r["fp32"]
    assert 20.0 < r["fp32"] < 200.0
    assert r["fp32x2"] > 0.8 * r["fp32"]
    assert 50.0 < r["tf32"] < 2250.0
