"""Pins for oracle.pcg, oracle.loss and oracle.rng."""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import grid, hmatrix, loss, pcg, rng
import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _sys(dims=(8, 8), seed=2, heavy=10.0):
    if len(dims) == 2:
        rho = inputs.density_discs(seed, dims, 1, (2.0, 2.0), heavy)
    else:
        rho = inputs.density_spheres(seed, dims, (1, 2), (1.0, 2.0), heavy)
    s = grid.assemble(rho, dims)
    return s, grid.dense_matrix(s)


# ---------------------------------------------------------------- rng
def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    assert rng.stream(0, 3) == want


def test_counter_form_equals_stream():
    key = 0x1234_5678_9ABC_DEF0
    s = rng.stream(key, 10)
    assert [rng.at(key, i) for i in range(10)] == s


def test_rademacher_probes_are_signs():
    z = loss.rademacher_probes(7, 3, 256, 16)
    assert set(np.unique(z)) == {-1.0, 1.0}
    assert abs(z.mean()) < 0.05
    assert np.array_equal(z, loss.rademacher_probes(7, 3, 256, 16))
    assert not np.array_equal(z, loss.rademacher_probes(7, 4, 256, 16))


# ---------------------------------------------------------------- pcg
def test_pcg_exact_inverse_one_iteration():
    s, a = _sys((8, 8))
    ainv = np.linalg.inv(a)
    b = inputs.rhs(0, 64)
    out = pcg.pcg(lambda v: a @ v, lambda v: ainv @ v, b, rtol=1e-10)
    assert out["iters"] == 1 and out["status"] == pcg.OK
    assert out["rel_res"] <= 1e-12


def test_cg_identity_converges_within_n():
    s, a = _sys((8, 8))
    b = inputs.rhs(1, 64)
    out = pcg.pcg(lambda v: a @ v, lambda v: v.copy(), b, rtol=1e-10, recompute_every=0)
    assert out["status"] == pcg.OK and out["iters"] <= 64
    assert out["rel_res"] <= 1e-9


def test_cg_energy_error_monotone_and_m_orthogonal_residuals():
    s, a = _sys((8, 8), 3)
    b = inputs.rhs(2, 64)
    xs = np.linalg.solve(a, b)
    d = s["diag"]
    out = pcg.pcg(lambda v: a @ v, lambda v: v / d, b, rtol=1e-12, recompute_every=0,
                  keep_history=True)
    e = [float((x - xs) @ a @ (x - xs)) for x in out["hist"]["x"]]
    assert all(e[i + 1] <= e[i] * (1 + 1e-12) for i in range(len(e) - 1))
    rs = out["hist"]["r"][:8]
    for i in range(len(rs)):
        for j in range(i):
            num = abs(rs[i] @ (rs[j] / d))
            assert num <= 1e-8 * np.linalg.norm(rs[i]) * np.linalg.norm(rs[j] / d)


def test_jacobi_pcg_equals_cg_on_scaled_system():
    s, a = _sys((8, 8), 4)
    b = inputs.rhs(3, 64)
    d = s["diag"]
    out = pcg.pcg(lambda v: a @ v, lambda v: v / d, b, rtol=1e-10, recompute_every=0,
                  keep_history=True)
    dh = 1.0 / np.sqrt(d)
    as_ = dh[:, None] * a * dh[None, :]
    out2 = pcg.pcg(lambda v: as_ @ v, lambda v: v.copy(), dh * b, rtol=1e-10,
                   recompute_every=0, keep_history=True)
    # x_k = D^-1/2 y_k for every iterate; the stop tests differ, so compare the common prefix
    k = min(len(out["hist"]["x"]), len(out2["hist"]["x"]))
    for i in range(k):
        assert np.allclose(out["hist"]["x"][i], dh * out2["hist"]["x"][i], atol=1e-9)


def test_pcg_matches_scipy_cg_solution():
    fr = inputs.frame("disc2d_1024", 0)
    s = grid.assemble(fr["rho"], fr["dims"])
    a = grid.sparse_matrix(s)
    out = pcg.pcg(lambda v: a @ v, lambda v: v / s["diag"], fr["b"], rtol=1e-10)
    x2, info = spla.cg(a, fr["b"], rtol=1e-12, maxiter=5000,
                       M=spla.LinearOperator(a.shape, matvec=lambda v: v / s["diag"]))
    assert info == 0
    assert np.linalg.norm(out["x"] - x2) <= 1e-8 * np.linalg.norm(x2)


def test_pcg_breakdown_on_indefinite_preconditioner():
    s, a = _sys((8, 8))
    b = inputs.rhs(4, 64)
    out = pcg.pcg(lambda v: a @ v, lambda v: -v, b)
    assert out["status"] == pcg.BREAKDOWN


# ---------------------------------------------------------------- loss
def test_cosine_loss_prop1():
    s, a = _sys((8, 8))
    rs = np.random.default_rng(0)
    z = rs.standard_normal((64, 16))
    m = rs.standard_normal((64, 64))
    m = m @ m.T + 0.1 * np.eye(64)
    y = m @ a @ z
    l1 = loss.cosine_loss(z, y)
    for alpha in (1e-3, 0.5, 7.0, 1e4):
        assert abs(loss.cosine_loss(z, (alpha * m) @ a @ z) - l1) <= 1e-14
    assert 0.0 <= l1 <= 2.0
    assert abs(loss.cosine_loss(z, -y) - (2.0 - l1)) <= 1e-14
    ainv = np.linalg.inv(a)
    assert abs(loss.cosine_loss(z, ainv @ a @ z)) <= 1e-14
    # projector identity: 1/2 ||Pi_u - Pi_v||^2 = 1 - cos^2
    u, v = z[:8, :2].ravel(), y[:8, :2].ravel()
    cos = 1.0 - loss.cosine_loss(u, v)
    assert abs(loss.projector_distance(u, v) - (1.0 - cos * cos)) <= 1e-13
    # the SAI loss is not scale invariant
    an = np.linalg.norm(a, 2)
    assert abs(loss.sai_loss(z, a @ m @ z, an) - loss.sai_loss(z, a @ (2 * m) @ z, an)) > 1e-3


@pytest.mark.parametrize("kz", [16, 64, 256, 1024])
def test_hutchinson_trace_within_closed_form_variance(kz):
    s, a = _sys((8, 8), 6)
    dvec = s["diag"]
    bmat = np.diag(1.0 / dvec) @ a      # B = M A with M = Jacobi (not symmetric)
    z = loss.rademacher_probes(11, kz, 64, kz)
    est = float(np.sum(z * (bmat @ z))) / kz
    tr = np.trace(bmat)
    var = np.sum(bmat ** 2) + np.trace(bmat @ bmat) - 2 * np.sum(np.diag(bmat) ** 2)
    assert abs(est - tr) <= 4 * np.sqrt(var / kz)
    # ||B Z||_F^2 / K_z estimates ||B||_F^2 (E[z z^T] = I)
    est2 = float(np.sum((bmat @ z) ** 2)) / kz
    assert abs(est2 - np.sum(bmat ** 2)) <= 0.5 * np.sum(bmat ** 2)


def test_gaussian_hutchinson_and_smoothing():
    s, a = _sys((8, 8), 6)
    d = s["diag"]
    rs = np.random.default_rng(9)
    g = rs.standard_normal((64, 4096))
    z = loss.jacobi_smooth(g, lambda v: a @ v, d)
    smat = np.eye(64) - 0.6 * (a / d[:, None])
    smat = smat @ smat
    assert np.allclose(z, smat @ g, atol=1e-12)
    bm = np.linalg.inv(a)
    est = float(np.sum(z * (bm @ z))) / 4096
    tr = np.trace(smat.T @ bm @ smat)
    c = smat.T @ bm @ smat
    var = np.sum(c ** 2) + np.trace(c @ c)
    assert abs(est - tr) <= 4 * np.sqrt(var / 4096)


def test_probe_count():
    assert loss.probe_count(1024) == 64 and loss.probe_count(16384) == 128
    assert loss.probe_count(8192) == 91


def test_gaussian_probes_are_standard_normal():
    # Box-Muller normals from the SplitMix64 stream: moments and the normal CDF (Kolmogorov-Smirnov)
    from scipy import stats
    z = np.array(rng.gaussian(5, 3, 4096, 8)).ravel()
    n = z.size
    assert abs(z.mean()) <= 4.0 / np.sqrt(n)
    assert abs(z.var() - 1.0) <= 4.0 * np.sqrt(2.0 / n)
    assert abs(stats.skew(z)) <= 4.0 * np.sqrt(6.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # different systems and steps draw different (uncorrelated) probes
    z2 = np.array(rng.gaussian(6, 3, 4096, 8)).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) <= 4.0 / np.sqrt(n)


def test_smoothed_gaussian_probes_follow_eq8():
    s, a = _sys((8, 8), 6)
    d = s["diag"]
    g = loss.gaussian_probes(2, 1, 64, 5)
    z = loss.smoothed_gaussian_probes(2, 1, 64, 5, lambda v: a @ v, d)
    smat = np.eye(64) - 0.6 * (a / d[:, None])
    assert np.allclose(z, smat @ (smat @ g), atol=1e-12)
