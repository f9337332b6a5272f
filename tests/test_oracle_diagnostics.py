"""Pins for the oracle's diagnostics (Fig. 1 spectra of M A, Fig. 3 rank audit), and what the
trained network gains over the same method untrained and over Jacobi.

The CG convergence theorem ties the spectrum to the oracle PCG: in the A-norm the error after
k iterations is at most 2 ((sqrt(kappa) - 1) / (sqrt(kappa) + 1))^k times the initial error,
kappa = lambda_max / lambda_min of M A.
"""
import math
import os

import numpy as np
import pytest
import torch

import inputs
from oracle import diagnostics as dg
from oracle import grid, hmatrix, network, pcg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TRAINED = os.path.join(ROOT, "paper_2605_13343_gb300", "weights", "hmpcg_d128_l4.f32")
CFG = dict(d=128, n_layers=4, n_heads=4, d_mlp=512, leaf=64, rank=16)


def _system(dims=(32, 32), seed=1):
    rho = inputs.density_for_dims(seed, dims)
    s = grid.assemble(rho, dims)
    return s, grid.dense_matrix(s)


# ---------------------------------------------------------------- spectrum of M A
def test_spectrum_special_cases():
    s, a = _system((16, 16))
    n = s["n"]
    assert np.allclose(dg.spectrum_ma(a, np.eye(n)), np.linalg.eigvalsh(a), rtol=1e-10, atol=0)
    assert np.abs(dg.spectrum_ma(a, np.linalg.inv(a)) - 1.0).max() <= 1e-10
    # Jacobi: M A is similar to D^-1/2 A D^-1/2
    d = s["diag"]
    want = np.linalg.eigvalsh(a / np.sqrt(np.outer(d, d)))
    assert np.allclose(dg.spectrum_ma(a, np.diag(1.0 / d)), want, rtol=1e-10, atol=0)
    # an SVD-H M against the general (nonsymmetric) eigensolver on M A itself
    m = hmatrix.dense_m(hmatrix.svdh_factors(a, 64, 16, leaves="inverse_block"))
    general = np.sort(np.linalg.eigvals(m @ a).real)
    assert np.allclose(dg.spectrum_ma(a, m), general, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("which", ["jacobi", "svdh"])
def test_pcg_error_obeys_the_cg_bound_for_the_measured_kappa(which):
    s, a = _system((32, 32), 4)
    b = inputs.rhs(4, s["n"])
    if which == "jacobi":
        m = np.diag(1.0 / s["diag"])
    else:
        m = hmatrix.dense_m(hmatrix.svdh_factors(a, 64, 16, leaves="inverse_block"))
    kappa = dg.condition_number(dg.spectrum_ma(a, m))
    out = pcg.pcg(lambda v: a @ v, lambda v: m @ v, b, rtol=1e-10, keep_history=True)
    x_star = np.linalg.solve(a, b)

    def a_norm(e):
        return math.sqrt(float(e @ (a @ e)))

    e0 = a_norm(x_star)                       # x0 = 0
    q = (math.sqrt(kappa) - 1.0) / (math.sqrt(kappa) + 1.0)
    checked = 0
    for k, xk in enumerate(out["hist"]["x"]):
        rel = a_norm(xk - x_star) / e0
        if rel < 1e-9:                        # below that, rounding, not the theorem, decides
            break
        assert rel <= 2.0 * q ** k * (1.0 + 1e-6), (k, rel, 2.0 * q ** k)
        checked += 1
    assert checked >= 5


def test_kappa_ordering_on_the_disc_frame():
    s, a = _system((32, 32), 0)
    kap = {name: dg.condition_number(dg.spectrum_ma(a, m)) for name, m in (
        ("none", np.eye(s["n"])), ("jacobi", np.diag(1.0 / s["diag"])),
        ("svdh", hmatrix.dense_m(hmatrix.svdh_factors(a, 64, 16, leaves="inverse_block"))))}
    assert kap["svdh"] < kap["jacobi"] < kap["none"]


# ---------------------------------------------------------------- rank audit
def test_eps_rank_against_explicit_truncation():
    rng = np.random.default_rng(0)
    u, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    v, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    sv = 10.0 ** (-0.4 * np.arange(30))
    x = u[:, :30] @ np.diag(sv) @ v.T
    norm = np.linalg.norm(x)
    got = np.linalg.svd(x, compute_uv=False)
    for eps in (1e-1, 1e-3, 1e-6, 1e-9, 1e-13):
        r = dg.eps_rank(got, eps)

        def err(k):
            xk = u[:, :k] @ np.diag(sv[:k]) @ v[:, :k].T
            return np.linalg.norm(x - xk) / norm
        assert err(r) <= eps * (1 + 1e-9)
        assert r == 0 or err(r - 1) > eps
    assert dg.eps_rank(np.zeros(5), 1e-3) == 0
    assert dg.eps_rank(np.ones(4), 0.0) == 4


@pytest.mark.parametrize("dims", [(32, 32), (16, 8, 8)])
def test_top_tile_rank_is_bounded_by_the_interface(dims):
    # (A^-1)_RC = -A_RR^-1 A_RC (A/A_RR)^-1, so its rank is at most rank(A_RC): the faces
    # between the two halves of the grid
    s, a = _system(dims)
    n = s["n"]
    h = n // 2
    coupling = np.linalg.matrix_rank(a[:h, h:])
    sv = np.linalg.svd(np.linalg.inv(a)[:h, h:], compute_uv=False)
    assert coupling == int(np.count_nonzero(a[:h, h:]))      # one face per coupled pair
    assert sv[coupling:].max() <= 1e-10 * sv[0]
    assert sv[coupling - 1] > 1e-6 * sv[0]


@pytest.mark.parametrize("dims", [(32, 32), (16, 8, 8)])
def test_required_rank_fraction_falls_with_distance_class(dims):
    # Fig. 3: far interactions are more compressible, per unit of tile width
    s, a = _system(dims)
    ainv = np.linalg.inv(a)
    au = dg.rank_audit(0.5 * (ainv + ainv.T), 64, 16)
    classes = sorted(au)
    assert classes == [1 << j for j in range(len(classes))]
    assert sum(au[c]["tiles"] for c in classes) == s["n"] // 64 - 1
    for e in range(3):
        means = [au[c]["mean"][e] for c in classes]
        assert all(x >= y for x, y in zip(means, means[1:])), means
    for c in classes:
        for r in au[c]["ranks"]:
            assert r[0] <= r[1] <= r[2]                          # tighter eps, higher rank
        assert au[c]["provided"] == 16 / (64 * c)


# ---------------------------------------------------------------- what training gains
@pytest.fixture(scope="module")
def weights():
    lay = inputs.network_layout(**CFG)
    trained = network.unflatten(np.fromfile(TRAINED, dtype=np.float32).astype(np.float64), lay)
    init = network.unflatten(inputs.network_blob(0, **CFG).astype(np.float64), lay)
    return trained, init


def _learned(p, s):
    with torch.no_grad():
        return network.to_numpy_factors(network.forward(p, s, CFG))


def test_trained_network_halves_pcg_iterations(weights):
    # a 32x16x16 frame outside every seed pool the training run drew from
    fr = inputs.frame("spheres3d_8192", 30000)
    s = grid.assemble(fr["rho"], fr["dims"])
    asp = grid.sparse_matrix(s)
    trained, init = weights
    runs = {}
    for name, prec in (("jacobi", lambda v: v / s["diag"]),
                       ("trained", (lambda f: lambda v: hmatrix.apply(f, v))(_learned(trained, s))),
                       ("init", (lambda f: lambda v: hmatrix.apply(f, v))(_learned(init, s)))):
        runs[name] = pcg.pcg(lambda v: asp @ v, prec, fr["b"], rtol=1e-6)
        assert runs[name]["status"] == pcg.OK and runs[name]["rel_res"] <= 1e-6, name
    it = {k: v["iters"] for k, v in runs.items()}
    assert it["trained"] <= 0.65 * it["jacobi"], it
    assert it["trained"] <= 0.65 * it["init"], it


def test_trained_network_lowers_kappa(weights):
    s, a = _system((16, 8, 8), 30000)
    trained, init = weights
    kap = {name: dg.condition_number(dg.spectrum_ma(a, m)) for name, m in (
        ("jacobi", np.diag(1.0 / s["diag"])), ("trained", hmatrix.dense_m(_learned(trained, s))),
        ("init", hmatrix.dense_m(_learned(init, s))))}
    assert kap["trained"] < 0.6 * kap["jacobi"], kap
    # the initialisation is Jacobi in disguise (gate 1, factor heads near zero)
    assert abs(kap["init"] / kap["jacobi"] - 1.0) < 0.05, kap
