"""Host logic of the autotuner's evaluation-path choice (no GPU): bucketing of node sizes and cache keys."""
import pytest

autotune = pytest.importorskip("paper_1409_2802_gb300.autotune")


def test_n_bucket_rounds_up_and_saturates():
    assert autotune.n_bucket(1) == 256 and autotune.n_bucket(256) == 256 and autotune.n_bucket(257) == 1024
    assert autotune.n_bucket(65536) == 65536 and autotune.n_bucket(10 ** 7) == 65536
    assert list(autotune.N_BUCKETS) == sorted(autotune.N_BUCKETS)


def test_candidates_are_the_tensor_core_paths():
    ffc = autotune.ffc
    assert autotune.EVAL_CANDIDATES[0] == ffc.EVAL_MMA_SYNC
    assert autotune.EVAL_CANDIDATES[1:] == tuple(range(ffc.EVAL_TCGEN05_TILE0,
                                                       ffc.EVAL_TCGEN05_TILE0 + ffc.EVAL_TCGEN05_TILES))


def test_cache_keys_separate_every_field():
    k = autotune._eval_key
    base = k(128, 1, 0, 4096, 2048, "torch.float64")
    for other in (k(64, 1, 0, 4096, 2048, "torch.float64"), k(128, 0, 0, 4096, 2048, "torch.float64"),
                  k(128, 1, 2, 4096, 2048, "torch.float64"), k(128, 1, 0, 1024, 2048, "torch.float64"),
                  k(128, 1, 0, 4096, 1024, "torch.float64"), k(128, 1, 0, 4096, 2048, "torch.float32")):
        assert other != base
