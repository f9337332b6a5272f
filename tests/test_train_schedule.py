"""The training schedule of Supp. C on the CPU: the reduce-on-plateau scheduler against
PyTorch's ReduceLROnPlateau with the paper's settings, and the auto-stop rule."""
import numpy as np
import pytest
import torch

from paper_2605_13343_gb300.train import AutoStop, Plateau


def _torch_lrs(lr0, values, min_lr):
    p = torch.nn.Parameter(torch.zeros(1))
    opt = torch.optim.SGD([p], lr=lr0)
    sch = torch.optim.lr_scheduler.ReduceLROnPlateau(opt, mode="min", factor=0.5, patience=5,
                                                     threshold=5e-3, threshold_mode="rel", min_lr=min_lr)
    out = []
    for v in values:
        sch.step(v)
        out.append(opt.param_groups[0]["lr"])
    return out


@pytest.mark.parametrize("seed", range(4))
def test_plateau_matches_torch_reduce_on_plateau(seed):
    rng = np.random.default_rng(seed)
    # a loss curve that falls, stalls, jitters and falls again
    t = np.arange(300)
    values = (0.07 * np.exp(-t / 60.0) + 0.02 + 0.002 * rng.standard_normal(300)).tolist()
    values[150:220] = [values[150]] * 70
    lr0 = 2e-4
    ours = Plateau(lr0)
    assert ours.min_lr == max(lr0 * 1e-3, 1e-6)
    got = [ours.step(v) for v in values]
    want = _torch_lrs(lr0, values, ours.min_lr)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    assert min(got) < lr0                        # the curve does trigger reductions


def test_plateau_floor_follows_the_initial_rate():
    assert Plateau(3e-4).min_lr == 1e-6         # 3e-7 is below the absolute floor
    assert Plateau(1e-2).min_lr == pytest.approx(1e-5)
    s = Plateau(1e-2)
    for _ in range(200):
        s.step(1.0)                              # never improves after the first value
    assert s.lr == pytest.approx(1e-5)


def test_auto_stop_needs_the_floor_and_ten_stalled_log_steps():
    st = AutoStop()
    assert not st.step(1.0, 1e-6, 1e-6)         # first value sets the best
    for k in range(9):
        assert not st.step(1.0, 1e-6, 1e-6), k  # 1..9 stalled steps
    assert st.step(1.0, 1e-6, 1e-6)             # the 10th
    st = AutoStop()
    st.step(1.0, 1e-3, 1e-6)
    for _ in range(20):
        assert not st.step(1.0, 1e-3, 1e-6)     # stalled, but the rate is not at its floor
    st = AutoStop()
    st.step(1.0, 1e-6, 1e-6)
    for _ in range(9):
        st.step(0.999, 1e-6, 1e-6)              # 0.1 % better: below the 0.5 % threshold
    assert st.step(0.999, 1e-6, 1e-6)
    st = AutoStop()
    st.step(1.0, 1e-6, 1e-6)
    for _ in range(9):
        st.step(1.0, 1e-6, 1e-6)
    assert not st.step(0.99, 1e-6, 1e-6)        # a 1 % improvement resets the count
