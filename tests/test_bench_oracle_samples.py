"""Host checks of bench.py's oracle samples of the ring GEMM (no GPU)."""
import numpy as np

import bench


def test_oracle_gemm_rows_cover_the_product():
    # the row blocks the all-cores sample splits the GEMM into tile it exactly
    n, procs = 64, 5
    bounds = [(n, i * n // procs, (i + 1) * n // procs) for i in range(procs)]
    assert bounds[0][1] == 0 and bounds[-1][2] == n
    assert all(b[2] == c[1] for b, c in zip(bounds, bounds[1:]))


def test_oracle_gemm_measure_small():
    out = bench.oracle_gemm_measure(n=64, all_cores=False)
    assert out["kind"] == "oracle" and out["cores"] == 1
    assert out["value"] > 0 and np.isfinite(out["value"])
    assert out["extrapolated_s"]["8192"] == 8 * out["extrapolated_s"]["4096"]
