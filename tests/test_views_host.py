"""Host logic of the view sampling layer, on the CPU: the scheduled trainer's
control flow (Alg. 1 steps 1-2 in front of the multi-view step) with the
GPU calls replaced by recorders, and the view sampler's scale-free default
distance weight."""
import numpy as np
import pytest
import torch

from paper_2606_15924_gb300 import scenes


class _Sampler:
    def __init__(self, means):
        self.means = list(means)
        self.calls = []

    def error_sums(self, maps):
        self.calls.append(("sums", tuple(maps.shape)))

    def mean_errors(self):
        return np.asarray(self.means.pop(0))

    def draw(self, k, it):
        self.calls.append(("draw", k, it))
        return torch.arange(k, dtype=torch.int32)


class _Trainer:
    def __init__(self, max_active):
        self.max_active = max_active
        self.sets, self.steps = [], 0

    def set_views(self, ids, n_pix):
        self.sets.append((list(ids), n_pix))

    def step(self):
        self.steps += 1


@pytest.fixture(scope="module")
def V():
    from paper_2606_15924_gb300 import build
    build.build()
    from paper_2606_15924_gb300 import views
    return views


def test_scheduled_step_control_flow(V):
    from paper_2606_15924_gb300.config import ScheduleConfig
    sched = ScheduleConfig(tau_until=10, K_max=8, K_min=2, alpha=3.0, lam=1.0)
    errs = [np.full(6, e) for e in (0.5, 0.45, 0.4, 0.3, 0.2, 0.2, 0.1, 0.1, 0.1, 0.1, 0.1, 0.1)]
    st = V.ScheduledTrainer.__new__(V.ScheduledTrainer)
    st.mv, st.sampler = _Trainer(max_active=5), _Sampler(errs)
    st.err_maps = torch.zeros(6, 4, 4, dtype=torch.int16)
    st.sched, st.E_init, st.t, st.history = sched, None, 0, []
    for t in range(12):
        rec = st.step()
        K, r = V.sampling_schedule(t, float(errs[t].mean()), 0.5, sched)
        assert st.E_init == 0.5                                    # fixed by the first step
        assert rec["K"] == max(1, min(K, 5)) and rec["n_pix"] == V.pixels_per_tile(r)
        assert st.mv.sets[-1] == (list(range(rec["K"])), rec["n_pix"])
        assert st.sampler.calls[-2] == ("sums", (6, 4, 4)) and st.sampler.calls[-1] == ("draw", rec["K"], t)
    assert st.mv.steps == 12 and st.t == 12
    ks = [h["K"] for h in st.history]
    assert ks[0] == 5 and ks[-1] == 2                              # capped at max_active, then K_min


def test_view_sampler_default_distance_weight(V):
    cams = scenes.orbit(12, 15.0, 64, 48)
    vs = V.ViewSampler(cams, device="cpu")
    c = np.stack([V.camera_pose(cm)[0] for cm in cams])
    d = [np.linalg.norm(c[i] - c[j]) for i in range(12) for j in range(i + 1, 12)]
    assert vs.lambda_d == pytest.approx(2.0 / np.median(d), rel=1e-12)
    assert vs.lambda_theta == 2.0
    # the weight is scale-free: the same cameras twice as far away halve lambda_d
    far = V.ViewSampler(scenes.orbit(12, 30.0, 64, 48), device="cpu")
    assert far.lambda_d == pytest.approx(vs.lambda_d / 2.0, rel=1e-3)
    assert vs.stack.dtype == torch.uint8 and int(vs.stack.sum()) == 12
    assert vs.cams.numel() == 12 * 92
    one = V.ViewSampler(cams[:1], device="cpu")
    assert one.lambda_d == 0.0
    with pytest.raises(ValueError):
        V.ViewSampler([], device="cpu")


def test_library_schedule_closed_forms():
    """The library's own host schedule (App. A, Eqs. 15-16), pinned to the
    closed forms directly rather than to the oracle's copy: at t = 0 with the
    initial error, rho = 1 and phi = 1 give K = K_max and r = lambda / K_max;
    from tau_until on (or with no error left) g = 1 gives
    K = round(K_min + (K_max - K_min) e^-alpha) and r = lambda / K_min;
    phi(1/4) = sin(pi/4); the error ratio is clipped to [0, 1]."""
    import math
    from paper_2606_15924_gb300.config import ScheduleConfig
    from paper_2606_15924_gb300.views import pixels_per_tile, sampling_schedule
    s = ScheduleConfig()
    assert (s.K_max, s.K_min, s.alpha, s.tau_until, s.lam) == (10, 3, 3.0, 3500, 1.0)   # Table 6
    K, r = sampling_schedule(0, 0.7, 0.7, s)
    assert K == 10 and r == pytest.approx(1.0 / 10, rel=1e-7)
    k_late = math.floor(3 + 7 * math.exp(-3.0) + 0.5)
    assert k_late == 3
    for t, e, e0 in ((3500, 0.7, 0.7), (9000, 0.1, 0.7), (0, 0.0, 0.7), (100, 0.0, 2.0)):
        K, r = sampling_schedule(t, e, e0, s)
        assert K == k_late and r == pytest.approx(1.0 / 3, rel=1e-7)
    # phi(1/4) = sin(pi/4) at t = 0: g = 1 - sqrt(2)/2
    K, r = sampling_schedule(0, 0.25, 1.0, s)
    g = 1.0 - math.sqrt(0.5)
    assert r == pytest.approx(0.1 + (1.0 / 3 - 0.1) * g, rel=1e-7)
    assert K == math.floor(3 + 7 * math.exp(-3.0 * g) + 0.5)
    # halfway to tau_until with the initial error: rho = 1/2, phi = 1, g = 1/2
    K, r = sampling_schedule(1750, 1.0, 1.0, s)
    assert r == pytest.approx(0.1 + (1.0 / 3 - 0.1) * 0.5, rel=1e-7)
    assert K == math.floor(3 + 7 * math.exp(-1.5) + 0.5)
    # lambda scales both rates
    K, r = sampling_schedule(0, 1.0, 1.0, ScheduleConfig(lam=0.5))
    assert r == pytest.approx(0.05, rel=1e-7)
    # more error than at the start counts as the start
    assert sampling_schedule(100, 5.0, 1.0, s) == sampling_schedule(100, 1.0, 1.0, s)
    # the pixel count per full tile
    assert pixels_per_tile(1.0 / 3) == 85 and pixels_per_tile(0.1) == 26
    assert pixels_per_tile(0.0) == 1 and pixels_per_tile(2.0) == 256
