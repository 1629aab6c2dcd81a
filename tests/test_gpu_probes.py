"""The measurement probes behind the FP64 roofline's denominators.

seed_time_fma times FMA chains on the FP64 and FP32 pipes; seed_time_fp64_paths
times the FP64 matrix instructions (mma.sync f64) and whether they run beside
the FMA pipe or share it.  The tests check that the numbers are sane -- rates
bounded by the unit-count peaks, FP32 far above FP64, and the mix ratio between
full overlap (0.5) and full serialisation (1) -- not the part's exact rates.
"""
import pytest

pytestmark = pytest.mark.gpu

# unit-count bounds at the maximum clock, with margin: 152 SMs x 2.07 GHz
FP64_BOUND = 152 * 2.07e9 * 2 * 2 / 1e12 * 1.2      # 2 FP64 FMA per clock per SM
FP32_BOUND = 152 * 2.07e9 * 128 * 2 / 1e12 * 1.2    # 128 FP32 FMA per clock per SM


def test_fma_probe_rates(seedlib):
    f64 = seedlib.seed_time_fma(seedlib.SEED_F64)
    f32 = seedlib.seed_time_fma(seedlib.SEED_F32)
    assert 0.0 < f64["tflops"] <= FP64_BOUND and f64["ms"] > 0.0
    assert 0.0 < f32["tflops"] <= FP32_BOUND
    assert f32["tflops"] > 8 * f64["tflops"]


def test_fp64_matrix_probe(seedlib):
    r = seedlib.seed_time_fp64_paths()
    print(r)
    for k in ("fma_tflops", "dmma_m8n8k4_tflops", "dmma_m16n8k16_tflops"):
        assert 0.0 < r[k] <= 40.0, (k, r[k])
    assert 0.0 < r["fma_tflops"] <= FP64_BOUND
    assert 0.3 <= r["mix_over_sum"] <= 1.2, r
    assert min(r["ms_fma_half"], r["ms_dmma_half"]) > 0.0


def test_fma_probe_rejects_other_dtypes(seedlib):
    with pytest.raises(seedlib.SeedError) as e:
        seedlib.seed_time_fma(seedlib.SEED_C128)
    assert e.value.status == seedlib.SEED_EINVAL
