"""Host-side arithmetic of bench.py (no GPU): the tensor peak that the mixed
factorisation's roofline fraction is taken against."""
import numpy as np
import pytest

import bench


def _tile_products(T):
    """Count the 128 x 128 x 128 tile products of a right-looking blocked
    Cholesky with T tile columns by walking it: column k's panel solve has one
    product per tile below the diagonal; its trailing update one per lower
    tile (i, j) with k < j <= i (the super-panel grouping only reorders them)."""
    trsm = upd = 0
    for k in range(T):
        trsm += T - 1 - k
        for j in range(k + 1, T):
            upd += T - j
    return trsm, upd


@pytest.mark.parametrize("T", [1, 2, 3, 8, 24, 94])
def test_tile_counts_match_the_closed_forms(T):
    trsm, upd = _tile_products(T)
    assert trsm == T * (T - 1) // 2
    assert upd == (T - 1) * T * (T + 1) // 6


def test_factor_tensor_peak_is_the_flop_weighted_harmonic_mean():
    bf16 = 2000.0
    n = np.array([3000.0, 1500.0, 129.0])
    T = [int(np.ceil(x / 128)) for x in n]
    trsm = sum(_tile_products(t)[0] for t in T)
    upd = sum(_tile_products(t)[1] for t in T)
    # time per tile product at each rate, summed over the batch
    t_total = trsm / (0.5 * bf16) + upd / bf16
    peak, tf32, f = bench.factor_tensor_peak(n, bf16)
    assert tf32 == 0.5 * bf16
    assert f == pytest.approx(trsm / (trsm + upd), rel=1e-15)
    assert peak == pytest.approx((trsm + upd) / t_total, rel=1e-12)
    assert tf32 < peak < bf16


def test_factor_tensor_peak_single_tile_chains():
    # N <= 42 beads: one diagonal tile, no tensor-core products at all.
    peak, tf32, f = bench.factor_tensor_peak(np.array([126.0, 99.0]), 1800.0)
    assert (peak, tf32, f) == (900.0, 900.0, 1.0)


def test_default_workload_peak():
    # 64 chains of N = 1000 (order 3000, 24 tiles): TF32 share 276 / 2576.
    peak, tf32, f = bench.factor_tensor_peak(np.full(64, 3000.0), 1966.7)
    assert f == pytest.approx(276 / 2576, rel=1e-15)
    assert peak == pytest.approx(1776.374, rel=1e-6)


def test_hbm_roofline():
    # 64 chains of order 3000 in FP32: both triangles written by the assembly.
    b = 64 * 3000.0 ** 2 * 4
    r = bench.hbm_roofline(b, 0.372, 6694.5)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(b / 0.372e-3 / 1e9, rel=1e-15)
    assert r["frac"] == pytest.approx(r["achieved"] / 6694.5, rel=1e-15)
    assert r["algorithmic_bytes_per_launch"] == b and r["ms_per_launch"] == 0.372


def test_cpu_model_is_a_string():
    m = bench.cpu_model()
    assert isinstance(m, str) and m
