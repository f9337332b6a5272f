"""Pins for oracle.hmatrix: partition, layouts, SVD-H, dense M, structured apply."""
import os

import numpy as np
import pytest

from oracle import grid, hmatrix
import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append(line.split())
    return out


def test_table_s3_factor_sizes():
    # Supp. G, Table S3: L=128, L_s=32 -> K, M_H, K L^2, P and the float32 MB.
    def printed(value, text):
        # equal to the printed figure within half a unit of its last digit
        dec = len(text.split(".")[1]) if "." in text else 0
        return abs(value - float(text)) <= 0.5 * 10 ** (-dec) + 1e-12

    for n, k, mh, kl2, p, mb in _rows("table_s3.txt"):
        n, k, mh = int(n), int(k), int(mh)
        tiles = hmatrix.partition(n, 128)
        assert n // 128 == k and len(tiles) == mh == k - 1
        assert printed(k * 128 * 128 / 1e6, kl2)
        width = hmatrix.packed_width(n, 128, 32, "learned")
        assert printed(width / 1e6, p)
        assert printed(width * 4 / 1e6, mb)
    assert hmatrix.packed_width(1024, 128, 32) == 131072 + 7168 + 65536 + 1024


@pytest.mark.parametrize("n,leaf", [(64, 16), (256, 16), (1024, 64), (128, 8)])
def test_partition_covers_matrix_once(n, leaf):
    cover = np.zeros((n, n), dtype=int)
    for b in range(n // leaf):
        cover[b * leaf:(b + 1) * leaf, b * leaf:(b + 1) * leaf] += 1
    for (m, lev, (r0, r1), (c0, c1)) in hmatrix.partition(n, leaf):
        assert r1 - r0 == c1 - c0 == (n // leaf) >> lev
        assert r1 == c0  # siblings
        cover[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf] += 1
        cover[c0 * leaf:c1 * leaf, r0 * leaf:r1 * leaf] += 1
    assert (cover == 1).all()
    ms = [t[0] for t in hmatrix.partition(n, leaf)]
    assert ms == list(range(n // leaf - 1))


def _random_learned(n, leaf, rank, seed=0):
    rng = np.random.default_rng(seed)
    w = hmatrix.packed_width(n, leaf, rank, "learned")
    return hmatrix.unpack(rng.standard_normal(w), n, leaf, rank, "learned")


@pytest.mark.parametrize("n,leaf,rank", [(64, 16, 4), (256, 16, 4), (512, 64, 16)])
def test_structured_apply_equals_dense_learned(n, leaf, rank):
    f = _random_learned(n, leaf, rank)
    m = hmatrix.dense_m(f)
    assert np.array_equal(m, m.T)
    x = np.random.default_rng(1).standard_normal((n, 3))
    assert np.allclose(hmatrix.apply(f, x), m @ x, rtol=0, atol=1e-12 * np.abs(m).sum(1).max() * 10)
    assert np.allclose(hmatrix.apply(f, x[:, 0]), m @ x[:, 0], rtol=0, atol=1e-10)


def test_single_tile_touches_only_its_block():
    n, leaf, rank = 128, 16, 4
    f = _random_learned(n, leaf, rank)
    f["leafblk"][:] = 0
    f["g"][:] = 0
    keep = 3  # level-2 tile, t = 0
    for m in range(f["core"].shape[0]):
        if m != keep:
            f["core"][m] = 0
    m_, lev, (r0, r1), (c0, c1) = hmatrix.partition(n, leaf)[keep]
    dense = hmatrix.dense_m(f)
    mask = np.zeros_like(dense, dtype=bool)
    mask[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf] = True
    mask[c0 * leaf:c1 * leaf, r0 * leaf:r1 * leaf] = True
    assert (dense[~mask] == 0).all() and (np.abs(dense[mask]) > 0).any()
    # the apply on a basis vector reproduces that column
    e = np.zeros(n)
    e[c0 * leaf + 2] = 1.0
    assert np.allclose(hmatrix.apply(f, e), dense[:, c0 * leaf + 2], atol=1e-13)


def test_pack_roundtrip():
    f = _random_learned(256, 16, 4)
    p = hmatrix.pack(f)
    g = hmatrix.unpack(p, 256, 16, 4, "learned")
    for key in ("leafblk", "core", "U", "V", "g"):
        assert np.array_equal(f[key], g[key])


def _small_system(dims=(8, 8), seed=2):
    rho = inputs.density_discs(seed, dims, 1, (2.0, 2.0), 10.0)
    sys = grid.assemble(rho, dims)
    return sys, grid.dense_matrix(sys)


def test_svdh_full_rank_exact_leaves_is_inverse():
    sys, a = _small_system((8, 8))
    f = hmatrix.svdh_factors(a, 16, 32, leaves="inverse_block")
    m = hmatrix.dense_m(f)
    assert np.allclose(m, f["ainv"], rtol=0, atol=1e-12 * np.abs(f["ainv"]).max())
    x = np.random.default_rng(3).standard_normal(64)
    assert np.allclose(hmatrix.apply(f, x), f["ainv"] @ x, atol=1e-12)


def test_svdh_eckart_young_and_apply():
    sys, a = _small_system((16, 16), 4)
    rank = 4
    f = hmatrix.svdh_factors(a, 16, rank)
    m = hmatrix.dense_m(f)
    leaf = 16
    for (t, lev, (r0, r1), (c0, c1)) in hmatrix.partition(256, leaf):
        x = f["ainv"][r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf]
        xr = m[r0 * leaf:r1 * leaf, c0 * leaf:c1 * leaf]
        s = f["sigma"][t]
        err = np.sum((x - xr) ** 2)
        assert abs(err - np.sum(s[rank:] ** 2)) <= 1e-12 * np.sum(s ** 2)
    # leaves are the exact inverses of A's diagonal blocks
    for b in range(16):
        sl_ = slice(b * leaf, (b + 1) * leaf)
        assert np.allclose(m[sl_, sl_] @ a[sl_, sl_], np.eye(leaf), atol=1e-12)
    x = np.random.default_rng(5).standard_normal(256)
    assert np.allclose(hmatrix.apply(f, x), m @ x, atol=1e-12)
    assert np.array_equal(m, m.T)


def test_svdh_leaf_modes_definiteness_on_disc_frame():
    # With exact block inverses (A_kk)^-1 as leaves and rank-16 tiles the assembled M of the
    # 32x32 disc frame is indefinite; with (A^-1)_kk leaves it is SPD.  M-matrix theory gives
    # (A^-1)_kk >= (A_kk)^-1 entrywise, which is what the first mode drops.
    fr = inputs.frame("disc2d_1024", 0)
    ref = grid.assemble(fr["rho"], fr["dims"])
    ad = grid.dense_matrix(ref)
    f1 = hmatrix.svdh_factors(ad, 64, 16, leaves="block_inverse")
    f2 = hmatrix.svdh_factors(ad, 64, 16, leaves="inverse_block")
    assert np.linalg.eigvalsh(hmatrix.dense_m(f1)).min() < 0
    assert np.linalg.eigvalsh(hmatrix.dense_m(f2)).min() > 0
    for b in range(16):
        s = slice(b * 64, (b + 1) * 64)
        assert (f2["leafblk"][b] - f1["leafblk"][b] >= -1e-12).all()
