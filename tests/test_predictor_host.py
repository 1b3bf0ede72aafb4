"""Host-side logic of the tile-error predictor (no GPU): the replay ring keeps
exactly the latest observations."""
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2606_15924_gb300.predictor import TileErrorPredictor  # noqa: E402


def _latest(pushes, cap):
    rows = [r for batch in pushes for r in batch]
    return sorted(rows[-cap:])


def test_replay_ring_keeps_the_latest_rows():
    cap = 7
    p = TileErrorPredictor(device="cpu", replay=cap)
    pushes, v = [], 0
    for size in (3, 5, 2, 9, 1, 4, 7, 6):   # wraps, and one push larger than the ring
        batch = list(range(v, v + size))
        v += size
        pushes.append(batch)
        x = torch.tensor(batch, dtype=torch.float32)[:, None].repeat(1, 16)
        t = torch.tensor(batch, dtype=torch.float32)
        p._push(x, t)
        n = min(sum(len(b) for b in pushes), cap)
        assert p.buf_n == n
        held = sorted(p.buf_t[:n].tolist())
        assert held == _latest(pushes, cap)[-n:]
        # features travel with their targets
        assert torch.equal(p.buf_x[:n, 3], p.buf_t[:n])
