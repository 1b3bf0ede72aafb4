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
