"""Seeded synthetic inputs: shapes, dtypes, ranges and determinism."""
import numpy as np

from paper_2104_00282_gb300 import workloads as W


def test_generators_are_deterministic_and_typed():
    for make in (lambda: W.config_plain_small(200, 4, seed=3),
                 lambda: W.config_hetero(5000, 8, seed=3),
                 lambda: W.config_large(3000, 32, seed=3),
                 lambda: W.paper_medium(4000, "target", seed=3),
                 lambda: W.random_small(300, 5, seed=3)):
        p, q = make(), make()
        for f in ("A", "kind", "w", "param", "R"):
            assert np.array_equal(getattr(p, f), getattr(q, f))
        assert p.A.dtype == np.float32 and p.A.flags.c_contiguous
        assert p.kind.dtype == np.uint8 and p.w.dtype == np.float32
        assert p.param.dtype == np.float32 and p.R.dtype == np.float64
        assert np.all(p.A > 0) and np.all(p.w > 0) and np.all(p.R > 0)


def test_large_recipe_mix_and_ranges():
    p = W.config_large(200_000, 32, seed=0)
    frac = np.bincount(p.kind, minlength=3) / p.n
    assert np.allclose(frac, [0.4, 0.4, 0.2], atol=0.01)
    assert np.all((p.param[p.kind == 1] >= 0.2) & (p.param[p.kind == 1] <= 0.8))
    assert np.all((p.param[p.kind == 2] >= 1) & (p.param[p.kind == 2] <= 10))
    assert np.all((p.R >= 0.05 * p.n) & (p.R <= 0.3 * p.n))
    # column scales s_j in [0.25, 8] times lognormal(0, 0.75): medians spread accordingly
    med = np.median(p.A, axis=0)
    assert med.min() >= 0.2 and med.max() <= 8.5


def test_batched_shapes():
    n, m = W.batched_shapes(4096, seed=0)
    assert n.min() >= 100 and n.max() <= 200_000
    assert set(np.unique(m)) == {4, 8, 16, 32}
