"""Host-side helpers of the benchmark (no GPU): FFT-friendly mesh sizes, the SPME mesh rule
of bench.spme_params, and the half-space mode count of the algorithmic work figure."""
import math

import bench


def test_fft_size_is_smallest_even_7_smooth_at_or_above():
    def smooth(k):
        for f in (2, 3, 5, 7):
            while k % f == 0:
                k //= f
        return k == 1
    for k in range(4, 700):
        K = bench.fft_size(k)
        assert K >= k and K % 2 == 0 and smooth(K)
        assert all(not (j % 2 == 0 and smooth(j)) for j in range(k, K))


def test_spme_params_auto_and_explicit():
    beta, L = 0.929, 32.0
    for p, bh in bench.SPME_BETA_H.items():
        K, order = bench.spme_params(f"auto:{p}", beta, L)
        assert order == p and beta * L / K <= bh + 1e-12
        assert K == bench.fft_size(beta * L / bh)
    assert bench.spme_params("auto", beta, L)[1] == 8
    assert bench.spme_params("64,10", beta, L) == (64, 10)


def test_half_space_mode_count_matches_the_oracle_k_set():
    import oracle
    for k in (1, 2, 5, 8, 10, 36):
        assert bench.len_kset_half(k) == len(oracle.kset_half(k))
