"""The seeded input generators: the same seed gives the same data on every call and machine
(the CUDA path's tests and the oracle read the same inputs), distinct seeds give distinct
frames, and every frame has the documented shape."""
import numpy as np
import pytest

import inputs


@pytest.mark.parametrize("family", sorted(inputs.FRAMES))
def test_frames_are_reproducible_and_well_formed(family):
    a, b, c = inputs.frame(family, 3), inputs.frame(family, 3), inputs.frame(family, 4)
    n = int(np.prod(a["dims"]))
    for key in ("rho", "b"):
        assert np.array_equal(a[key], b[key])
        assert a[key].shape == (n,) and a[key].dtype == np.float64
        assert not np.array_equal(a[key], c[key])
    assert (a["rho"] > 0).all()
    assert abs(a["b"].sum()) <= 1e-10 * np.abs(a["b"]).sum()      # zero-mean right-hand side
    assert n % a["leaf"] == 0 and (n // a["leaf"]) & (n // a["leaf"] - 1) == 0
    assert a["bc"] in ("dirichlet", "neumann") and a["face"] in ("inv_rho", "rho")


def test_network_blob_and_batch_shapes_are_reproducible():
    cfg = dict(d=64, n_layers=1, n_heads=2, d_mlp=64, leaf=64, rank=16)
    w1, w2, w3 = inputs.network_blob(5, **cfg), inputs.network_blob(5, **cfg), inputs.network_blob(6, **cfg)
    assert w1.dtype == np.float32 and np.array_equal(w1, w2) and not np.array_equal(w1, w3)
    assert w1.size == sum(int(np.prod(s)) for _, s in inputs.network_layout(**cfg))
    d1, d2 = inputs.batch_mixed_dims(7), inputs.batch_mixed_dims(7)
    assert d1 == d2 and len(d1) == 64
    assert {int(np.prod(d)) for d in d1} <= {1024, 2048, 4096, 8192, 16384}
    assert all(len(d) == (2 if i % 2 == 0 else 3) for i, d in enumerate(d1))
    assert np.array_equal(inputs.rhs(9, 100), inputs.rhs(9, 100))


def test_split_seeds_are_disjoint():
    for seed in (0, 1, 5):
        tr, te = inputs.split_seeds(seed, 100, 20)
        assert len(tr) == 100 and len(te) == 20 and not set(tr) & set(te)
    a = set(sum(inputs.split_seeds(0, 100, 20), []))
    b = set(sum(inputs.split_seeds(1, 100, 20), []))
    assert not a & b
