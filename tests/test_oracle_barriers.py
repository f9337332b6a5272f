"""Pins for the paper's own benchmark distribution (Supp. D): the barrier density generator,
the zero-flux operator with its constant null space, the pseudo-inverse SVD-H builder, and PCG
to rtol 1e-8 on those frames (Supp. A)."""
import math
from collections import Counter

import numpy as np
import pytest

import inputs
from oracle import grid, hmatrix, pcg


def _components(mask, w, h):
    """4-connected components of the True cells of a lexicographic w x h mask (plain BFS)."""
    seen = np.zeros(w * h, dtype=bool)
    count = 0
    for start in range(w * h):
        if not mask[start] or seen[start]:
            continue
        count += 1
        stack = [start]
        seen[start] = True
        while stack:
            c = stack.pop()
            i, j = c % w, c // w
            for ii, jj in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                if 0 <= ii < w and 0 <= jj < h:
                    d = ii + w * jj
                    if mask[d] and not seen[d]:
                        seen[d] = True
                        stack.append(d)
    return count


# ---------------------------------------------------------------- generator
@pytest.mark.parametrize("seed", range(6))
def test_barrier_membership_brute_force(seed):
    w, h = 32, 32
    rho, p = inputs.density_barriers(seed, (w, h), return_params=True)
    heavy = np.zeros(w * h, dtype=bool)
    for j in range(h):
        for i in range(w):
            u, v = (i + 0.5) / w, (j + 0.5) / h
            for b in p["barriers"]:
                across, along = (u, v) if b["vertical"] else (v, u)
                if abs(across - b["centre"]) > 0.5 * b["thickness"]:
                    continue
                kind = b["gap_kind"]
                in_gap = ((kind == "top" and along > 0.8) or (kind == "bottom" and along < 0.2)
                          or (kind == "middle_hole" and abs(along - 0.5) < 0.1))
                if not in_gap:
                    heavy[i + w * j] = True
    assert np.array_equal(heavy, p["heavy"])
    # 5 % multiplicative jitter around the two phases
    eps = rho / np.where(heavy, p["rho_heavy"], 1.0) - 1.0
    assert abs(eps.std() - 0.05) < 0.01 and abs(eps.mean()) < 0.01
    assert 5.0 <= p["rho_heavy"] <= 100.0 and 1 <= len(p["barriers"]) <= 3
    for b in p["barriers"]:
        assert 0.2 <= b["centre"] <= 0.8 and 0.05 <= b["thickness"] <= 0.20


def test_barrier_parameters_follow_the_stated_distributions():
    # 300 frames: counts within ~5 sigma of the uniform laws, log-contrast mean of U[ln 5, ln 100]
    kinds, orient, nbs, logs = Counter(), Counter(), Counter(), []
    for seed in range(300):
        _, p = inputs.density_barriers(seed, (16, 16), return_params=True)
        nbs[len(p["barriers"])] += 1
        logs.append(math.log(p["rho_heavy"]))
        for b in p["barriers"]:
            kinds[b["gap_kind"]] += 1
            orient[b["vertical"]] += 1
    assert set(nbs) == {1, 2, 3} and all(abs(c - 100) <= 45 for c in nbs.values())
    total = sum(kinds.values())
    assert set(kinds) == set(inputs.BARRIER_GAPS)
    assert all(abs(c - total / 4) <= 5 * math.sqrt(total * 3 / 16) for c in kinds.values())
    assert abs(orient[True] - total / 2) <= 5 * math.sqrt(total / 4)
    lo, hi = math.log(5.0), math.log(100.0)
    assert abs(np.mean(logs) - 0.5 * (lo + hi)) <= 5 * (hi - lo) / math.sqrt(12 * 300)


@pytest.mark.parametrize("vertical", [True, False])
def test_gap_topologies_by_connectivity(vertical):
    # one barrier across the middle: closed splits the light phase in two, every gap kind
    # leaves it connected, through cells at the stated end of the barrier
    w = h = 32
    for kind, parts in (("closed", 2), ("top", 1), ("bottom", 1), ("middle_hole", 1)):
        m = inputs.barrier_mask((w, h), vertical, 0.5, 0.1, kind)
        assert m.any()
        assert _components(~m, w, h) == parts, kind
    cx, cy = inputs.grid_centres((w, h))
    along = (cy / h) if vertical else (cx / w)
    band = inputs.barrier_mask((w, h), vertical, 0.5, 0.1, "closed")
    for kind, where in (("top", along > 0.8), ("bottom", along < 0.2), ("middle_hole", np.abs(along - 0.5) < 0.1)):
        hole = band & ~inputs.barrier_mask((w, h), vertical, 0.5, 0.1, kind)
        assert hole.any() and np.array_equal(hole, band & where), kind


def test_barrier_frames_are_zero_flux_with_the_papers_face_rule():
    for n in (1024, 2048, 4096, 8192, 16384):
        fr = inputs.frame(f"barriers2d_{n}", 0)
        assert int(np.prod(fr["dims"])) == n and len(fr["dims"]) == 2
        assert fr["bc"] == "neumann" and fr["face"] == "rho" and fr["rtol"] == 1e-8
        assert abs(fr["b"].sum()) <= 1e-10 * np.abs(fr["b"]).sum()


# ---------------------------------------------------------------- zero-flux operator
def _barrier_system(seed=3, dims=(32, 32)):
    rho = inputs.density_barriers(seed, dims)
    s = grid.assemble(rho, dims, bc="neumann", face="rho")
    return s, grid.dense_matrix(s)


def test_zero_flux_operator_has_only_the_constant_null_space():
    s, a = _barrier_system()
    assert np.array_equal(a, a.T)
    assert np.abs(a @ np.ones(s["n"])).max() <= 1e-12 * np.abs(a).max()
    ev = np.linalg.eigvalsh(a)
    assert abs(ev[0]) <= 1e-10 * ev[-1], "A 1 = 0"
    assert ev[1] > 1e-6 * ev[-1], "the grid is connected: one null direction only"
    # the face rule is the paper's harmonic mean of rho: check one interior face by hand
    i = 5
    j = grid.neighbours(s["dims"])[i][1]
    ri, rj = s["rho"][i], s["rho"][j]
    assert a[i, j] == -(2.0 * ri * rj / (ri + rj))


def test_pseudo_inverse_moore_penrose_identities():
    s, a = _barrier_system(seed=1, dims=(16, 16))
    n = s["n"]
    p = hmatrix.pseudo_inverse(a)
    scale = np.abs(a).max()
    assert np.abs(a @ p @ a - a).max() <= 1e-10 * scale
    assert np.abs(p @ a @ p - p).max() <= 1e-10 * np.abs(p).max()
    # A A^+ is the orthogonal projector onto the complement of the constants
    assert np.abs(a @ p - (np.eye(n) - np.ones((n, n)) / n)).max() <= 1e-9
    assert np.abs(p @ np.ones(n)).max() <= 1e-9 * np.abs(p).max()
    # on a nonsingular (Dirichlet) operator it is the inverse
    sd = grid.assemble(inputs.density_barriers(1, (16, 16)), (16, 16))
    ad = grid.dense_matrix(sd)
    inv = np.linalg.inv(ad)
    assert np.abs(hmatrix.pseudo_inverse(ad) - inv).max() <= 1e-10 * np.abs(inv).max()


# ---------------------------------------------------------------- PCG to rtol 1e-8
@pytest.mark.parametrize("seed", [0, 1])
def test_pcg_reaches_rtol_1e8_on_barrier_frames(seed):
    fr = inputs.frame("barriers2d_1024", seed)
    s = grid.assemble(fr["rho"], fr["dims"], bc=fr["bc"], face=fr["face"])
    a = grid.dense_matrix(s)
    asp = grid.sparse_matrix(s)
    b = fr["b"]
    ev = np.linalg.eigvalsh(a)
    kappa = ev[-1] / ev[1]                       # condition number on the complement of 1
    f = hmatrix.svdh_factors(a, fr["leaf"], fr["rank"], leaves="inverse_block", inverse="pseudo")
    x_star = f["ainv"] @ b                      # A^+ b: the minimum-norm (zero-mean) solution
    runs = {
        "cg": pcg.pcg(lambda v: asp @ v, lambda v: v, b, rtol=fr["rtol"]),
        "jacobi": pcg.pcg(lambda v: asp @ v, lambda v: v / s["diag"], b, rtol=fr["rtol"]),
        "svdh": pcg.pcg(lambda v: asp @ v, lambda v: hmatrix.apply(f, v), b, rtol=fr["rtol"]),
    }
    for name, out in runs.items():
        assert out["status"] == pcg.OK and out["rel_res"] <= fr["rtol"], name
        x = out["x"] - out["x"].mean()          # solutions are unique up to a constant
        err = np.linalg.norm(x - x_star) / np.linalg.norm(x_star)
        assert err <= 1.01 * kappa * out["rel_res"] + 1e-12, (name, err, kappa)
    assert runs["svdh"]["iters"] < runs["jacobi"]["iters"] < runs["cg"]["iters"]


def test_papers_model_size_runs_on_a_barrier_frame():
    # the paper's default model (Sec. 7.3): d = 128, 3 layers, 8 heads, leaf 128, L_s = 32
    import torch
    from oracle import network
    cfg = dict(d=128, n_layers=3, n_heads=8, d_mlp=512, leaf=128, rank=32)
    fr = inputs.frame("barriers2d_1024", 5)
    s = grid.assemble(fr["rho"], fr["dims"], bc=fr["bc"], face=fr["face"])
    p = network.unflatten(inputs.network_blob(0, **cfg).astype(np.float64), inputs.network_layout(**cfg))
    with torch.no_grad():
        f = network.to_numpy_factors(network.forward(p, s, cfg))
    k = s["n"] // 128
    assert f["leafblk"].shape == (k, 128, 128) and f["core"].shape == (k - 1, 32, 32)
    assert all(np.isfinite(f[key]).all() for key in ("leafblk", "U", "V", "core", "g"))
    # at initialisation the learned M is Jacobi up to the small factor heads (their F F^T term
    # sums 128 products per entry at this leaf size, hence a few 1e-3)
    m = hmatrix.dense_m(f)
    assert np.allclose(np.diag(m) * s["diag"], 1.0, atol=1e-2)
    asp = grid.sparse_matrix(s)
    out = pcg.pcg(lambda v: asp @ v, lambda v: hmatrix.apply(f, v), fr["b"], rtol=fr["rtol"])
    assert out["status"] == pcg.OK and out["rel_res"] <= fr["rtol"]
