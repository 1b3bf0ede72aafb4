"""Host logic of the multi-view trainer, on the CPU: set_views' checks and
the per-view state it sets (loss weight 1/K, pixels per tile), with the pool
entries and the batch rebuild replaced by stand-ins; the persistent grid
candidates of the autotuner."""
import pytest


class _View:
    def __init__(self, n_select, n_pix):
        self.n_select, self.n_pix = n_select, n_pix
        self.P_max = n_select * n_pix
        self.loss_params = (1e-3, 1e-8, 0.4, 0.25)


@pytest.fixture(scope="module")
def MVT():
    from paper_2606_15924_gb300 import build
    build.build()
    from paper_2606_15924_gb300 import batched
    return batched


def _pool(batched, n=6, max_active=3):
    mv = batched.MultiViewTrainer.__new__(batched.MultiViewTrainer)
    mv.pool = [_View(10 + k, 85) for k in range(n)]
    mv.max_active = max_active
    mv.views, mv.K = mv.pool[:max_active], max_active
    mv.rebuilt = 0

    def rebuild():
        mv.rebuilt += 1
    mv._build_batches = rebuild
    mv.graph = object()
    return mv


def test_set_views(MVT):
    mv = _pool(MVT)
    mv.set_views([4, 1], n_pix=21)
    assert mv.K == 2 and mv.views == [mv.pool[4], mv.pool[1]]
    assert all(v.loss_params == (1e-3, 1e-8, 0.4, 0.5) and v.n_pix == 21 for v in mv.views)
    assert mv.pool[0].n_pix == 85 and mv.rebuilt == 1 and mv.graph is None
    mv.set_views([5, 0, 2])                                  # pixels per tile unchanged
    assert [v.n_pix for v in mv.views] == [85, 85, 85] and mv.views[0].loss_params[3] == pytest.approx(1 / 3)
    for ids, n_pix in (([], None), ([0, 1, 2, 3], None), ([1, 1], None), ([6], None), ([-1], None),
                       ([0], 0), ([0], 86)):
        with pytest.raises(ValueError):
            mv.set_views(ids, n_pix)
    assert mv.rebuilt == 2


def test_grid_candidates(MVT):
    assert MVT.grid_candidates(1216, 152) == [152, 304, 608, 1216]
    assert MVT.grid_candidates(1000, 152) == [152, 304, 608, 1000]
    assert MVT.grid_candidates(100, 152) == [100]
