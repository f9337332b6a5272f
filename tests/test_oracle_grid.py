"""Pins for oracle.grid: Morton order and assembly (Supp. D; Sec. 7.1)."""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import grid
import inputs


def _interleave_by_strings(coords, dims):
    # Brute force by a different route: write each coordinate as a bit string,
    # then read the code off column by column from the least significant end.
    strs = [format(c, "b").zfill(int(np.log2(n))) [::-1] for c, n in zip(coords, dims)]
    bits = []
    level = 0
    while any(level < len(s) for s in strs):
        for s in strs:
            if level < len(s):
                bits.append(s[level])
        level += 1
    return int("".join(reversed(bits)), 2) if bits else 0


@pytest.mark.parametrize("dims", [(32, 32), (32, 16, 16), (16, 8, 8), (8, 8), (128, 64)])
def test_morton_bijection_and_string_key(dims):
    n = int(np.prod(dims))
    seen = set()
    rng = np.random.default_rng(1)
    for m in range(n):
        c = grid.morton_decode(m, dims)
        assert grid.morton_encode(c, dims) == m
        seen.add(c)
    assert len(seen) == n
    for m in rng.integers(0, n, size=200):
        c = grid.morton_decode(int(m), dims)
        assert _interleave_by_strings(c, dims) == m


def test_morton_leaves_are_blocks():
    # A leaf of 64 consecutive codes is an 8x8 block in 2D and 4x4x4 in 3D.
    for dims, ext in [((32, 32), (8, 8)), ((32, 16, 16), (4, 4, 4))]:
        for leaf in range(int(np.prod(dims)) // 64):
            cs = np.array([grid.morton_decode(leaf * 64 + i, dims) for i in range(64)])
            assert tuple(cs.max(0) - cs.min(0) + 1) == ext


def test_morton_sort_matches_argsort():
    dims = (16, 8, 8)
    perm = grid.morton_perm(dims)
    keys = [_interleave_by_strings(grid.morton_decode(0, dims), dims)]
    # argsort of the string-built key over lexicographic cells reproduces perm
    n = int(np.prod(dims))
    lex_coords = []
    for idx in range(n):
        x = idx % dims[0]
        y = (idx // dims[0]) % dims[1]
        z = idx // (dims[0] * dims[1])
        lex_coords.append((x, y, z))
    keys = np.array([_interleave_by_strings(c, dims) for c in lex_coords])
    assert np.array_equal(np.argsort(keys, kind="stable"), perm)


def _textbook_dirichlet(dims):
    # sum_d I x .. x T_n x .. x I with T = tridiag(-1, 2, -1), lexicographic, x fastest
    mats = [np.diag(2.0 * np.ones(n)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
            for n in dims]
    eyes = [np.eye(n) for n in dims]
    total = 0
    for d in range(len(dims)):
        term = np.ones((1, 1))
        for a in reversed(range(len(dims))):
            term = np.kron(term, mats[a] if a == d else eyes[a])
        total = total + term
    return total


@pytest.mark.parametrize("dims", [(8, 8), (4, 4, 4), (8, 4, 2)])
def test_uniform_density_is_textbook_laplacian(dims):
    n = int(np.prod(dims))
    sys = grid.assemble(np.ones(n), dims)
    a = grid.dense_matrix(sys)
    t = _textbook_dirichlet(dims)
    perm = sys["perm"]
    assert np.array_equal(a, t[np.ix_(perm, perm)])
    ev = np.sort(np.linalg.eigvalsh(a))
    closed = []
    import itertools
    for ks in itertools.product(*[range(1, nd + 1) for nd in dims]):
        closed.append(sum(4 * np.sin(np.pi * k / (2 * (nd + 1))) ** 2 for k, nd in zip(ks, dims)))
    assert np.allclose(ev, np.sort(closed), atol=1e-12, rtol=0)


def test_face_conductance_two_forms():
    # two cells 1 and 10: 2/(1+10) for the 1/rho harmonic mean, 2*10/11 for rho's
    rho = np.array([1.0, 10.0])
    s1 = grid.assemble(rho, (2,), bc="neumann")
    assert s1["wplus"][0][0] == 2.0 / 11.0
    s2 = grid.assemble(rho, (2,), bc="neumann", face="rho")
    assert s2["wplus"][0][0] == 20.0 / 11.0
    # Dirichlet ghost faces add 1/rho_i per boundary face
    s3 = grid.assemble(rho, (2,), bc="dirichlet")
    assert s3["diag"][0] == 1.0 + 2.0 / 11.0
    assert s3["diag"][1] == 2.0 / 11.0 + 0.1


@pytest.mark.parametrize("family,seed", [("disc2d_1024", 0), ("disc2d_1024", 3)])
def test_assembled_operator_is_spd_m_matrix(family, seed):
    fr = inputs.frame(family, seed)
    sys = grid.assemble(fr["rho"], fr["dims"])
    a = grid.dense_matrix(sys)
    assert np.array_equal(a, a.T)
    sl.cholesky(a, lower=True)
    off = a - np.diag(np.diag(a))
    assert (off <= 0).all()
    assert (np.diag(a) >= -off.sum(1) - 1e-15).all()


def test_m_matrix_inverse_positive():
    rho = inputs.density_discs(5, (8, 8), 1, (2.0, 2.0), 10.0)
    sys = grid.assemble(rho, (8, 8))
    ainv = np.linalg.inv(grid.dense_matrix(sys))
    assert (ainv > 0).all()


def test_spmv_matches_dense():
    fr = inputs.frame("disc2d_1024", 1)
    sys = grid.assemble(fr["rho"], fr["dims"])
    a = grid.dense_matrix(sys)
    x = np.random.default_rng(0).standard_normal(sys["n"])
    assert np.allclose(grid.spmv(sys, x), a @ x, rtol=0, atol=1e-12)
    assert np.allclose(grid.sparse_matrix(sys) @ x, a @ x, rtol=0, atol=1e-12)


def test_density_generator_membership_brute_force():
    # the 32x32 one-disc frame: count heavy cells by an explicit double loop
    rho = inputs.density_discs(7, (32, 32), 1, (8.0, 8.0), 10.0)
    rng = np.random.default_rng(7)
    px = rng.uniform(8.0, 24.0)
    py = rng.uniform(8.0, 24.0)
    cnt = 0
    for j in range(32):
        for i in range(32):
            if (i + 0.5 - px) ** 2 + (j + 0.5 - py) ** 2 <= 64.0:
                cnt += 1
                assert rho[i + 32 * j] == 10.0
    assert int((rho == 10.0).sum()) == cnt
