"""Pins for the oracle's highway buffers and off-diagonal token pooling (Sec. 4.2, Sec. 4.3;
Supp. B "Highways" and "Off-diagonal tokens").

Each pin reaches the expected values by a route of its own: explicit loops over
nodes and tokens with the tile list written out here from the partition's
definition (tile t of level l pairs row leaves [2tS, (2t+1)S) with column leaves
[(2t+1)S, (2t+2)S), S = K / 2^l, heap order), a constant-token case where every
mean equals the constant, and one-hot tokens that light exactly the rows and
columns their chunk covers.
"""
import numpy as np
import pytest
import torch

from oracle import network

TD = torch.float64


def _tiles(n, leaf, rank):
    """(row start node, column start node, chunk) per tile in heap order, from the definition."""
    k = n // leaf
    levels = k.bit_length() - 1
    out = []
    for lev in range(1, levels + 1):
        s = k >> lev
        for t in range(1 << (lev - 1)):
            out.append((2 * t * s * leaf, (2 * t + 1) * s * leaf, s * leaf // rank))
    return out


def _brute_highways(yd, yo, n, leaf, rank):
    """Highways by loops: each diagonal node lists the tokens covering its row / column."""
    d = yd.shape[1]
    tiles = _tiles(n, leaf, rank)
    rhw = np.zeros((n, d))
    chw = np.zeros((n, d))
    for i in range(n):
        rows = [yd[i]]
        cols = [yd[i]]
        for m, (r0, c0, ch) in enumerate(tiles):
            for a in range(rank):
                if r0 + a * ch <= i < r0 + (a + 1) * ch:
                    rows.append(yo[m * rank + a])
                if c0 + a * ch <= i < c0 + (a + 1) * ch:
                    cols.append(yo[m * rank + a])
        for c in range(d):
            rhw[i, c] = sum(v[c] for v in rows) / len(rows)
            chw[i, c] = sum(v[c] for v in cols) / len(cols)
    tot = yd.shape[0] + yo.shape[0]
    g = np.array([(sum(yd[:, c]) + sum(yo[:, c])) / tot for c in range(d)])
    ud = np.zeros((n, 4 * d))
    for i in range(n):
        ud[i] = np.concatenate([yd[i], rhw[i], chw[i], g])
    uo = np.zeros((len(tiles) * rank, 4 * d))
    for m, (r0, c0, ch) in enumerate(tiles):
        for a in range(rank):
            rr = np.zeros(d)
            cc = np.zeros(d)
            for q in range(ch):
                rr += rhw[r0 + a * ch + q]
                cc += chw[c0 + a * ch + q]
            uo[m * rank + a] = np.concatenate([yo[m * rank + a], rr / ch, cc / ch, g])
    return ud, uo


def _run(yd, yo, n, leaf, rank):
    ud, uo = network.highways(torch.as_tensor(yd, dtype=TD), torch.as_tensor(yo, dtype=TD), n, leaf, rank)
    return ud.numpy(), uo.numpy()


def test_tile_list_matches_the_oracle_geometry():
    for n, leaf, rank in [(8, 4, 2), (64, 8, 4), (256, 16, 4), (1024, 64, 16)]:
        geo = [(r0, c0, ch) for (_, _, r0, c0, ch) in network.tile_geometry(n, leaf, rank)]
        assert geo == _tiles(n, leaf, rank)


def test_highways_two_leaves_by_hand():
    # n = 8, leaf 4, rank 2: one tile (rows 0-3, columns 4-7), chunks of 2 nodes
    rng = np.random.default_rng(0)
    yd = rng.standard_normal((8, 3))
    yo = rng.standard_normal((2, 3))
    ud, uo = _run(yd, yo, 8, 4, 2)
    g = (yd.sum(0) + yo.sum(0)) / 10.0
    for i in range(8):
        r = (yd[i] + yo[i // 2]) / 2.0 if i < 4 else yd[i]
        c = (yd[i] + yo[(i - 4) // 2]) / 2.0 if i >= 4 else yd[i]
        assert np.allclose(ud[i], np.concatenate([yd[i], r, c, g]), rtol=0, atol=1e-15)
    for a in range(2):
        rmean = ((yd[2 * a] + yo[a]) / 2.0 + (yd[2 * a + 1] + yo[a]) / 2.0) / 2.0
        cmean = ((yd[4 + 2 * a] + yo[a]) / 2.0 + (yd[5 + 2 * a] + yo[a]) / 2.0) / 2.0
        assert np.allclose(uo[a], np.concatenate([yo[a], rmean, cmean, g]), rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,leaf,rank", [(16, 4, 2), (64, 8, 4), (128, 16, 4), (256, 16, 16)])
def test_highways_brute_force(n, leaf, rank):
    rng = np.random.default_rng(n + leaf + rank)
    mh = n // leaf - 1
    yd = rng.standard_normal((n, 5))
    yo = rng.standard_normal((mh * rank, 5))
    ud, uo = _run(yd, yo, n, leaf, rank)
    bd, bo = _brute_highways(yd, yo, n, leaf, rank)
    assert np.allclose(ud, bd, rtol=0, atol=1e-13)
    assert np.allclose(uo, bo, rtol=0, atol=1e-13)


def test_highways_constant_tokens_give_the_constant():
    # every buffer is a mean of copies of v: any wrong contributor count breaks this
    n, leaf, rank = 1024, 64, 16
    v = np.array([1.5, -2.0, 0.25, 7.0])
    yd = np.tile(v, (n, 1))
    yo = np.tile(v, ((n // leaf - 1) * rank, 1))
    ud, uo = _run(yd, yo, n, leaf, rank)
    assert np.allclose(ud, np.tile(v, 4)[None, :], rtol=0, atol=1e-13)
    assert np.allclose(uo, np.tile(v, 4)[None, :], rtol=0, atol=1e-13)


@pytest.mark.parametrize("m,a", [(0, 0), (0, 15), (1, 3), (2, 9), (6, 7), (14, 0)])
def test_highways_one_hot_token_lights_its_rows_and_columns(m, a):
    n, leaf, rank = 1024, 64, 16
    mh = n // leaf - 1
    tiles = _tiles(n, leaf, rank)
    yd = np.zeros((n, 1))
    yo = np.zeros((mh * rank, 1))
    yo[m * rank + a, 0] = 1.0
    ud, uo = _run(yd, yo, n, leaf, rank)
    r0, c0, ch = tiles[m]
    rows = set(range(r0 + a * ch, r0 + (a + 1) * ch))
    cols = set(range(c0 + a * ch, c0 + (a + 1) * ch))
    lit_r = {i for i in range(n) if ud[i, 1] != 0.0}
    lit_c = {i for i in range(n) if ud[i, 2] != 0.0}
    assert lit_r == rows and lit_c == cols
    # the value at a lit row is 1 / (1 + number of tiles whose row clusters cover that row)
    for i in rows:
        cover = 1 + sum(1 for (rr, _, cc) in tiles if rr <= i < rr + rank * cc)
        assert abs(ud[i, 1] - 1.0 / cover) < 1e-15
    assert np.allclose(ud[:, 3], 1.0 / (n + mh * rank), rtol=0, atol=1e-18)
    # the token's own row in the off-diagonal gather holds the mean over its own chunk
    assert abs(uo[m * rank + a, 1] - np.mean([ud[i, 1] for i in rows])) < 1e-15


def _brute_pool(h, n, leaf, rank):
    d = h.shape[1]
    tiles = _tiles(n, leaf, rank)
    out = np.zeros((len(tiles) * rank, 2 * d))
    for m, (r0, c0, ch) in enumerate(tiles):
        for a in range(rank):
            for c in range(d):
                out[m * rank + a, c] = sum(h[r0 + a * ch + q, c] for q in range(ch)) / ch
                out[m * rank + a, d + c] = sum(h[c0 + a * ch + q, c] for q in range(ch)) / ch
    return out


def test_pool_two_leaves_by_hand():
    h = np.arange(8 * 2, dtype=np.float64).reshape(8, 2)
    got = network.pool_tokens(torch.as_tensor(h), 8, 4, 2).numpy()
    want = np.array([np.concatenate([(h[0] + h[1]) / 2, (h[4] + h[5]) / 2]),
                     np.concatenate([(h[2] + h[3]) / 2, (h[6] + h[7]) / 2])])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,leaf,rank", [(16, 4, 2), (128, 16, 4), (512, 64, 16)])
def test_pool_brute_force(n, leaf, rank):
    h = np.random.default_rng(n).standard_normal((n, 3))
    got = network.pool_tokens(torch.as_tensor(h), n, leaf, rank).numpy()
    assert np.allclose(got, _brute_pool(h, n, leaf, rank), rtol=0, atol=1e-13)


def test_pool_constant_and_one_hot_nodes():
    n, leaf, rank = 1024, 64, 16
    tiles = _tiles(n, leaf, rank)
    got = network.pool_tokens(torch.full((n, 2), 3.0, dtype=TD), n, leaf, rank).numpy()
    assert np.allclose(got, 3.0, rtol=0, atol=1e-14)
    for i in (0, 63, 64, 511, 512, 1023):
        h = torch.zeros(n, 1, dtype=TD)
        h[i, 0] = 1.0
        got = network.pool_tokens(h, n, leaf, rank).numpy()
        for m, (r0, c0, ch) in enumerate(tiles):
            for a in range(rank):
                in_r = r0 + a * ch <= i < r0 + (a + 1) * ch
                in_c = c0 + a * ch <= i < c0 + (a + 1) * ch
                assert got[m * rank + a, 0] == (1.0 / ch if in_r else 0.0)
                assert got[m * rank + a, 1] == (1.0 / ch if in_c else 0.0)
