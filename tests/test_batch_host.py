"""Host logic of the batched solver: shape rules and autotuner candidates."""
from paper_2504_11167_gb300 import batch


def test_default_shape_targets_4096_row_partitions():
    assert batch.default_shape(262144, 64) == (64, 64)
    assert batch.default_shape(4096, 8) == (2, 8)          # at least two partitions
    assert batch.default_shape(100000, 17) == (24, 32)
    p, kb = batch.default_shape(128, 64)                    # n_i > k forces one partition
    assert p == 1 and kb == 64


def test_candidates_respect_partition_and_block_rules():
    for n, k in [(5000, 8), (70000, 33), (262144, 64), (4096, 16)]:
        cands = batch.candidate_shapes(n, k)
        assert len(cands) == len(set(cands)) and cands
        for p, kb in cands:
            assert p >= 1 and (p == 1 or n // p > k)
            assert kb >= k and kb in (8, 16, 32, 64)
    assert all(kb == 64 for _, kb in batch.candidate_shapes(262144, 64))
    assert {kb for _, kb in batch.candidate_shapes(5000, 8)} == {8, 16}


def test_size_classes_are_power_of_two_intervals():
    assert batch.size_class(4096) == batch.size_class(8191) == 12
    assert batch.size_class(8192) == 13


def test_device_band_generator_follows_the_recipe():
    import numpy as np
    import torch
    from paper_2504_11167_gb300 import inputs
    n, k, dom = 300, 7, 1.5
    ab = inputs.dominant_band_torch(n, k, dom, 3, device="cpu").numpy()
    for d in range(2 * k + 1):
        for j in (0, 1, n - 2, n - 1, 150):
            i = j + d - k
            if not 0 <= i < n:
                assert ab[d, j] == 0.0
            elif d != k:
                assert -1.0 <= ab[d, j] <= 1.0
    off = inputs.off_diagonal_row_sums(np.where(np.arange(2 * k + 1)[:, None] == k, 0.0, ab), k)
    assert np.allclose(ab[k], dom * off, rtol=1e-14, atol=0)
    b2 = inputs.dominant_band_torch(n, k, dom, 3, device="cpu").numpy()
    assert np.array_equal(ab, b2)
