"""The CUDA-core FMA throughput probe (kss_peak_probe), the measured denominator of the FFT
passes' ALU rooflines: plausible rates on a GB300 (FP64 near its 1.26 TFLOP/s unit-count figure,
FP32 near 80 TFLOP/s, FP32 far above FP64) and refusal of an unknown pipe."""
import pytest

import paper_2507_08578_gb300.kss as K
from tests.kss_helpers import ensure_built, make_ctx

pytestmark = pytest.mark.gpu


def test_peak_probe_rates():
    import torch
    ensure_built()
    ctx = make_ctx()
    try:
        f64 = K.kss_peak_probe(ctx, 0)
        f32 = K.kss_peak_probe(ctx, 1)
        assert 0.5 < f64 < 1.5, f64
        assert 30.0 < f32 < 100.0, f32
        assert f32 > 20 * f64
        with pytest.raises(K.KssError):
            K.kss_peak_probe(ctx, 2)
    finally:
        torch.cuda.synchronize()
        K.kss_destroy(ctx)
