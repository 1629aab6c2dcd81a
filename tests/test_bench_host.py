"""Host arithmetic of bench.py's roofline and CG-branch bookkeeping (no GPU)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_and_flops_per_unit():
    # Wilson D per site: 4 links of 9 complex (144 B in FP64) read once, and a
    # 12-component spinor in and out per column (192 B each in FP64)
    assert bench.wilson_bytes(1, 1) == 4 * 9 * 16 + 2 * 12 * 16 == 960
    assert bench.wilson_bytes(4096, 11) == 4096 * (576 + 11 * 384)
    assert bench.wilson_bytes(131072, 11, fp32=True) == 314572800   # the 16^3 x 32 FP32 launch
    # CSR: 8 B value + 4 B index per nonzero, row pointers, x read and y written once
    assert bench.csr_bytes(4096, 20224) == 12 * 20224 + 4 * 4097 + 16 * 4096 == 324612
    # 1320 hopping flops (8 hops: projection, 3x3 complex matrix times two colour vectors,
    # reconstruction, accumulation); the 48 of psi - kappa * sum are reported separately
    assert bench.FLOPS_PER_SITE_D == 1320 and bench.FLOPS_PER_SITE_D_EPILOGUE == 48
    # the count: each of the 8 hops projects 4 -> 2 spin components (6 complex adds, 12 flops)
    # and multiplies the two colour vectors by a 3x3 complex matrix (2 x (9 complex multiplies
    # of 6 flops + 6 complex adds of 2) = 132 flops); 7 of the 8 hops add 24 reals into the
    # accumulated spinor (the first one stores); the reconstruction is sign changes only
    assert 8 * (12 + 2 * (9 * 6 + 6 * 2)) + 7 * 24 == bench.FLOPS_PER_SITE_D
    assert abs(bench.FP64_PEAK_GFLOPS - 1258.56) < 1e-9
    # the FP64 instructions the kernel issues per site: per direction the forward hop (12 adds of
    # the projection, 3 rows x 2 spins of one complex multiply (4 instructions) and two complex
    # FMAs (8) = 72) and the backward hop chained onto it (12 adds, 18 complex FMAs = 72, and the
    # lower half as 12 FMAs of 2 x forward - phase(upper)); 3 adds per real component to combine
    # the four direction partials (72) and 24 FMAs of psi - kappa * sum
    fwd = 12 + 3 * 2 * (4 + 2 * 4)
    bwd = 12 + 18 * 4 + 12
    assert 4 * (fwd + bwd) + 3 * 24 + 24 == bench.FP64_INSTR_PER_SITE_D == 816


def test_cg_branch_columns():
    for nc in range(1, 64):
        cols = bench.cg_branch_cols(nc)
        assert sum(cols) == nc and 1 <= len(cols) <= 3
        assert max(cols) - min(cols) <= 1
        if nc >= 2:
            assert min(cols) >= 2 or len(cols) == 1
    assert bench.cg_branch_cols(11) == [3, 4, 4]


def test_traffic_entries_only_for_captured_sources():
    # a traffic figure is reported only while the kernel source matches the capture
    assert bench.dslash_traffic() in (None, *bench.DSLASH_TRAFFIC.values())
    assert bench.dslash_traffic(fp32=True) in (None, *bench.DSLASH32_TRAFFIC.values())
    assert len(bench.dslash_source_hash()) == 16 and bench.dslash_source_hash() != bench.dslash_source_hash(fp32=True)


def test_workload_config_is_the_same_for_both_arms():
    a = bench.workload_config(bench.WL["dims"], "point", False)
    assert a["workload"] == bench.WORKLOAD_NAME and a["n"] == 49152 and a["nrhs"] == 12
    assert a == bench.workload_config((8, 8, 8, 8), "point", False, 1)
    assert "flushed" in a["l2"]
