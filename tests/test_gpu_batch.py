"""Batched solves of ragged systems (hmpcg_solve_batch, hmpcg_autotune_batch).

Each system of a batch must come out as the FP64 oracle's PCG says: true relative
residual <= rtol evaluated by the oracle in FP64 and an iteration count within
max(2, 2 %) of the oracle's, whatever cluster size, work-list position or concurrent
group it ran in.  H-matrix factors are SPD learned-layout factors in BF16; the
oracle's PCG uses the same factors, dequantised.
"""
import numpy as np
import pytest
import torch

import inputs
from oracle import grid, hmatrix, pcg

pytestmark = pytest.mark.gpu

h = pytest.importorskip("paper_2605_13343_gb300")


def _batch(count, seed):
    dims = inputs.batch_mixed_dims(seed, count)
    out = []
    for i, d in enumerate(dims):
        rho = inputs.density_for_dims(seed * 1000 + i, d)
        n = int(np.prod(d))
        out.append(dict(dims=d, rho=rho, b=inputs.rhs(seed * 1000 + i, n), n=n))
    return out


def _upload(batch):
    systems, bs, xs = [], [], []
    for fr in batch:
        s = h.System(fr["dims"])
        h.assemble(torch.from_numpy(fr["rho"]).cuda(), s)
        systems.append(s)
        bs.append(torch.from_numpy(fr["b"]).cuda())
        xs.append(torch.zeros(fr["n"], dtype=torch.float64, device="cuda"))
    return systems, bs, xs


def _oracle(fr, precond_of):
    ref = grid.assemble(fr["rho"], fr["dims"])
    a = grid.sparse_matrix(ref)
    out = pcg.pcg(lambda v: a @ v, precond_of(ref), fr["b"], rtol=1e-6)
    return out, a


def _check(fr, info, x, out, a):
    assert info.status == h.OK
    assert abs(info.iters - out["iters"]) <= max(2, 0.02 * out["iters"])
    xg = x.cpu().numpy()
    rel = np.linalg.norm(fr["b"] - a @ xg) / np.linalg.norm(fr["b"])
    assert rel <= 1e-6
    assert abs(info.rel_res_true - rel) <= 1e-9


def test_batch_jacobi_ragged():
    """12 systems, N in {1024 ... 16384}, 2D and 3D: three cluster sizes run as concurrent
    persistent launches."""
    batch = _batch(12, 3)
    ctx = h.Context(max_n=16384, leaf=64, rank=16)
    systems, bs, xs = _upload(batch)
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    infos = h.solve_batch(ctx, systems, [jac] * len(systems), bs, xs, rtol=1e-6)
    for fr, info, x in zip(batch, infos, xs):
        out, a = _oracle(fr, lambda ref: (lambda v: v / ref["diag"]))
        _check(fr, info, x, out, a)
    ctx.close()


def _spd_learned(ref, seed):
    """Learned-layout factors that make M SPD and close to Jacobi: gate = 1/diag, small PSD
    leaf term F F^T, small far-field tiles."""
    n = ref["n"]
    rng = np.random.default_rng(seed)
    f = hmatrix.unpack(rng.standard_normal(hmatrix.packed_width(n, 64, 16, "learned")), n, 64, 16, "learned")
    dinv = 1.0 / ref["diag"]
    f["g"] = dinv
    for k in range(n // 64):
        f["leafblk"][k] *= 0.02 * np.sqrt(dinv[k * 64:(k + 1) * 64])[:, None]
    f["U"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["V"] *= 0.3 * np.sqrt(dinv / n)[:, None]
    f["core"] *= 0.3
    return f


def test_batch_learned_ragged_and_autotune():
    """BF16 learned-layout factors on a ragged batch; the autotuner's choice is a feasible
    cluster size and the tuned batch gives the same answers."""
    batch = _batch(10, 5)
    ctx = h.Context(max_n=16384, leaf=64, rank=16)
    systems, bs, xs = _upload(batch)
    facs, deqs, keep = [], [], []
    for i, fr in enumerate(batch):
        ref = grid.assemble(fr["rho"], fr["dims"])
        f = _spd_learned(ref, 40 + i)
        packed = torch.from_numpy(hmatrix.pack(f).astype(np.float32)).to(torch.bfloat16).cuda()
        keep.append(packed)
        facs.append(h.factors(h.PRE_LEARNED, packed, fr["n"], 64, 16))
        deqs.append(hmatrix.unpack(packed.double().cpu().numpy(), fr["n"], 64, 16, "learned"))
    infos = h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6)
    refs = []
    for fr, deq, info, x in zip(batch, deqs, infos, xs):
        out, a = _oracle(fr, lambda ref, deq=deq: (lambda v: hmatrix.apply(deq, v)))
        assert out["status"] == pcg.OK
        refs.append((out, a))
        _check(fr, info, x, out, a)
    cs = h.autotune_batch(ctx, systems, facs, bs, xs, rtol=1e-6)
    assert all(c in (4, 8, 16) for c in cs)
    for fr, c in zip(batch, cs):
        assert fr["n"] // c <= 2048 and (fr["n"] // (c * 64)) <= 16
    for x in xs:
        x.zero_()
    infos = h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6)
    for fr, info, x, (out, a) in zip(batch, infos, xs, refs):
        _check(fr, info, x, out, a)
    ctx.close()


def test_batch_fallback_to_jacobi():
    """A system whose H-matrix preconditioner is negative definite breaks down at once; with
    fallback on it is solved again with Jacobi on the same cluster (iteration count of the
    oracle's Jacobi PCG), the SPD neighbour in the same batch is untouched."""
    batch = _batch(2, 9)
    ctx = h.Context(max_n=16384, leaf=64, rank=16)
    systems, bs, xs = _upload(batch)
    facs, keep, deqs = [], [], []
    for i, fr in enumerate(batch):
        ref = grid.assemble(fr["rho"], fr["dims"])
        f = _spd_learned(ref, 70 + i)
        packed = torch.from_numpy(hmatrix.pack(f).astype(np.float32)).to(torch.bfloat16).cuda()
        if i == 0:
            packed = -packed
        keep.append(packed)
        facs.append(h.factors(h.PRE_LEARNED, packed, fr["n"], 64, 16))
        deqs.append(hmatrix.unpack(packed.double().cpu().numpy(), fr["n"], 64, 16, "learned"))
    infos = h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6, allow=(h.OK, h.E_BREAKDOWN))
    assert infos[0].status == h.E_BREAKDOWN and infos[0].fallback == 0
    for x in xs:
        x.zero_()
    infos = h.solve_batch(ctx, systems, facs, bs, xs, rtol=1e-6, fallback=True)
    out, a = _oracle(batch[0], lambda ref: (lambda v: v / ref["diag"]))
    assert infos[0].fallback == 1       # broke down before its first iteration: iters are Jacobi's
    _check(batch[0], infos[0], xs[0], out, a)
    out, a = _oracle(batch[1], lambda ref, deq=deqs[1]: (lambda v: hmatrix.apply(deq, v)))
    assert infos[1].fallback == 0
    _check(batch[1], infos[1], xs[1], out, a)
    ctx.close()


def test_batch_matches_single_solves_and_rejects_oversize():
    """A batch entry equals the single-system cluster solve of the same system (same kernel
    body, same cluster size 16 for N = 8192 when tuned so); an N the cluster shapes cannot
    hold is refused with E_SHAPE instead of falling back."""
    fr = inputs.frame("spheres3d_8192", 4)
    ctx = h.Context(max_n=1 << 16, leaf=64, rank=16)
    systems, bs, xs = _upload([dict(fr, n=8192)])
    jac = h.Factors()
    jac.kind = h.PRE_JACOBI
    x1 = torch.zeros_like(bs[0])
    one = h.solve(ctx, systems[0], jac, bs[0], x1, rtol=1e-6)
    (got,) = h.solve_batch(ctx, systems, [jac], bs, xs, rtol=1e-6)
    assert got.status == h.OK and abs(got.iters - one.iters) <= 1
    assert np.linalg.norm((xs[0] - x1).cpu().numpy()) <= 1e-6 * np.linalg.norm(x1.cpu().numpy())
    big = inputs.density_for_dims(1, (256, 256))
    s = h.System((256, 256))
    h.assemble(torch.from_numpy(big).cuda(), s)
    b = torch.from_numpy(inputs.rhs(1, 65536)).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(RuntimeError):
        h.solve_batch(ctx, [s], [jac], [b], [x], rtol=1e-6)
    ctx.close()
