"""Hyper-parameters of the sparse-sampled path.

Defaults follow TurboGS Table 6 (App. B) where the paper gives a value; the
rest are readings of passages the paper leaves open (each named below).
These mirror the ``tgs_config`` / ``tgs_opt_config`` structs of the C ABI.
"""
from __future__ import annotations

from dataclasses import dataclass, field

TILE = 16  # Sec. 3.5: S x S tiles, S = 16


@dataclass
class SamplingConfig:
    # Table 6: ratio of hard (error-drawn) and stable (oldest) pixels; the
    # remaining 0.3 is drawn uniformly ("mixed sampling").
    r_hard: float = 0.4
    r_stable: float = 0.3
    # tile level (extension of the pixel split to tiles; not in the paper)
    tile_r_hard: float = 0.4
    tile_r_stable: float = 0.3

    def permille(self):
        return (round(self.tile_r_hard * 1000), round(self.tile_r_stable * 1000),
                round(self.r_hard * 1000), round(self.r_stable * 1000))


@dataclass
class LossConfig:
    eps_charbonnier: float = 1e-3   # App. A, Charbonnier epsilon (value not given)
    eps_ncc: float = 1e-8           # App. A, NCC epsilon (value not given)
    beta_ema: float = 0.4           # Table 6, EMA blending ratio of pixel errors
    structure: str = "ncc"          # "ncc" (Sec. 3.7) or "ssim" (Table 4's S-SSIM variant)


@dataclass
class OptConfig:
    """Moment-damped LM / Adam hybrid (Sec. 3.9, App. A).  Learning rates per
    parameter group; the paper gives none, these are the usual 3DGS values."""
    lr_means: float = 1.6e-4
    lr_scales: float = 5e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 2.5e-2
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 1.25e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps_adam: float = 1e-15
    eps_lm: float = 1e-8
    mode: int = 1                   # 0 Adam, 1 LM with J^T J diagonal, 2 LM full (Cholesky)

    def as_list(self):
        return [self.lr_means, self.lr_scales, self.lr_quats, self.lr_opacity, self.lr_sh_dc,
                self.lr_sh_rest, self.beta1, self.beta2, self.eps_adam, self.eps_lm]


@dataclass
class ScheduleConfig:
    """Table 6 values of the adaptive view/pixel schedule (App. A)."""
    T: int = 5000
    tau_until: int = 3500
    tau_from: int = 200
    K_max: int = 10
    K_min: int = 3
    alpha: float = 3.0
    lambda_base: float = 0.8
    # tile pixel sampling scale lambda, in (0, 1] (Table 6 gives the range);
    # 1 makes the late rate lambda / K_min = 1/3, the rate of the sparse step
    lam: float = 1.0


@dataclass
class DensityConfig:
    """Error-driven density control (Sec. 3.8; Table 6 ranges, one value
    chosen in each)."""
    tau_from: int = 200            # first densification iteration
    tau_until: int = 3500          # last densification iteration
    interval: int = 250            # densification interval (100 to 350)
    prune_interval: int = 500      # final pruning interval
    topk: float = 0.8              # fraction for top-k densification (0.5 to 0.95)
    final_keep: float = 0.9        # fraction retained by final pruning (0.8 to 0.95)
    tau_grad: float = 2e-4         # gradient threshold for densification (1e-4 to 2e-4)
    percent_dense: float = 0.01    # clone/split size as a fraction of the scene extent (0.001 to 0.02)
    lambda_base: float = 0.8       # base weight of the distance term of Eq. 13
    prune_opacity: float = 0.005   # opacity below which a Gaussian is pruned (the 3DGS value; not in Table 6)
    eps: float = 1e-8              # Eq. 13's epsilon (not given)


@dataclass
class Config:
    sampling: SamplingConfig = field(default_factory=SamplingConfig)
    loss: LossConfig = field(default_factory=LossConfig)
    opt: OptConfig = field(default_factory=OptConfig)
    schedule: ScheduleConfig = field(default_factory=ScheduleConfig)
    density: DensityConfig = field(default_factory=DensityConfig)
