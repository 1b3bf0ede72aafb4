"""Seeded synthetic inputs shaped like the TurboGS workloads.

This module only draws random numbers and builds cameras; it contains none of
the method's arithmetic, so both the CUDA path (through the tests and the
benchmark) and the CPU oracle can be fed from it.  Everything is numpy on the
host with explicit seeds (PCG64), so a given seed gives the same arrays on
every machine.

Scene recipe (the paper's datasets are not available; these stand in for
them): means uniform in a cube, log-scales normal, unit quaternions from a
normalised 4D normal, opacity logits standard normal, SH degree-3 coefficients
normal.  Cameras are pinholes looking at the origin from an orbit.
"""
from __future__ import annotations

import math

import numpy as np

# common seeds: scene, target, masks, noise
SEED_SCENE = 0
SEED_TARGET = 1
SEED_MASK = 2
SEED_NOISE = 3


def gaussians(n: int, seed: int = SEED_SCENE, extent: float = 1.0, log_scale_mean: float = -3.5,
              log_scale_std: float = 0.5, sh_std: float = 0.2) -> dict:
    """n Gaussians as float32 structure-of-arrays (means [n,3], log_scales [n,3],
    quats [n,4] (w,x,y,z), opacity_logits [n], sh [n,16,3])."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, size=(n, 3)).astype(np.float32)
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    quats = q.astype(np.float32)
    opacity_logits = rng.normal(size=n).astype(np.float32)
    sh = rng.normal(0.0, sh_std, size=(n, 16, 3)).astype(np.float32)
    return dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)


def look_at(position, target=(0.0, 0.0, 0.0), width: int = 256, height: int = 256, fov_x_deg: float = 60.0,
            znear: float = 0.2) -> dict:
    """Pinhole camera at ``position`` looking at ``target``.

    Camera axes follow the usual computer-vision convention (x right, y down,
    z forward); the world's "down" is +y.  ``viewmat`` is the row-major 4x4
    world-to-camera transform.
    """
    c = np.asarray(position, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - c
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    r = np.cross(down, f)
    if np.linalg.norm(r) < 1e-8:
        r = np.cross(np.array([0.0, 0.0, 1.0]), f)
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], 0)
    t = -R @ c
    V = np.eye(4)
    V[:3, :3] = R
    V[:3, 3] = t
    fx = width / (2.0 * math.tan(math.radians(fov_x_deg) / 2.0))
    return dict(viewmat=V.astype(np.float32).astype(np.float64), fx=float(np.float32(fx)),
                fy=float(np.float32(fx)), cx=width / 2.0, cy=height / 2.0, width=int(width), height=int(height),
                znear=float(np.float32(znear)))


def orbit(n_views: int, distance: float, width: int, height: int, fov_x_deg: float = 60.0,
          elevation_deg: float = 20.0, seed: int = SEED_SCENE) -> list:
    """n_views cameras evenly spaced in azimuth on a circle at ``distance``,
    with a small seeded elevation jitter."""
    rng = np.random.default_rng(seed + 1000)
    cams = []
    for k in range(n_views):
        az = 2.0 * math.pi * k / n_views
        el = math.radians(elevation_deg + rng.uniform(-5.0, 5.0))
        pos = (distance * math.cos(el) * math.sin(az), -distance * math.sin(el),
               -distance * math.cos(el) * math.cos(az))
        cams.append(look_at(pos, width=width, height=height, fov_x_deg=fov_x_deg))
    return cams


def error_map(width: int, height: int, seed: int = SEED_MASK, scale: float = 0.1,
              hot_fraction: float = 0.1) -> np.ndarray:
    """fp16 error map [H,W] (as uint16 bit patterns): small half-normal
    background plus a few seeded hot blobs, the shape of a partly-fit view."""
    rng = np.random.default_rng(seed)
    e = np.abs(rng.normal(0.0, scale, size=(height, width)))
    n_blobs = max(1, int(hot_fraction * (width * height) / (32.0 * 32.0)))
    yy, xx = np.mgrid[0:height, 0:width]
    for _ in range(n_blobs):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        s = rng.uniform(8.0, 40.0)
        e += rng.uniform(0.2, 1.0) * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    return e.astype(np.float16).view(np.uint16)


def age_map(width: int, height: int, seed: int = SEED_MASK, max_age: int = 200) -> np.ndarray:
    """uint16 age map [H,W] of seeded ages in [0, max_age]."""
    rng = np.random.default_rng(seed + 7)
    return rng.integers(0, max_age + 1, size=(height, width)).astype(np.uint16)


def smooth_image(width: int, height: int, seed: int = SEED_TARGET) -> np.ndarray:
    """float32 image [H,W,3] in [0,1]: a seeded sum of smooth blobs."""
    rng = np.random.default_rng(seed)
    img = np.zeros((height, width, 3))
    yy, xx = np.mgrid[0:height, 0:width]
    for _ in range(24):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        s = rng.uniform(0.03, 0.25) * max(width, height)
        col = rng.uniform(0, 1, size=3)
        img += col * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))[..., None]
    img /= max(img.max(), 1e-6)
    img += rng.normal(0.0, 0.01, size=img.shape)
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def projected(n: int, width: int, height: int, seed: int = SEED_SCENE, radius_max: int = 24,
              depth_ties: bool = True) -> dict:
    """Seeded screen-space splats (the outputs of a projection) for tests of the
    steps after it: xy, conic (positive definite), opacity, rgb, depth, radius.

    A fraction of depths repeat exactly, so the tie order is exercised."""
    rng = np.random.default_rng(seed + 17)
    xy = np.stack([rng.uniform(-20, width + 20, n), rng.uniform(-20, height + 20, n)], 1).astype(np.float32)
    # covariance from random axis lengths and angle, conic = inverse
    s1 = rng.uniform(0.7, 6.0, n)
    s2 = rng.uniform(0.7, 6.0, n)
    th = rng.uniform(0, math.pi, n)
    c, s = np.cos(th), np.sin(th)
    A = c * c * s1 * s1 + s * s * s2 * s2
    B = c * s * (s1 * s1 - s2 * s2)
    Cc = s * s * s1 * s1 + c * c * s2 * s2
    det = A * Cc - B * B
    conic = np.stack([Cc / det, -B / det, A / det], 1).astype(np.float32)
    lam = np.maximum(s1, s2) ** 2
    radius = np.minimum(np.ceil(3.0 * np.sqrt(lam)), radius_max).astype(np.int32)
    radius[rng.uniform(size=n) < 0.05] = 0                      # some culled
    opac = rng.uniform(0.05, 0.99, n).astype(np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32)
    depth = rng.uniform(1.0, 10.0, n).astype(np.float32)
    if depth_ties and n > 4:
        k = n // 8
        idx = rng.choice(n, size=k, replace=False)
        depth[idx] = depth[rng.choice(n, size=k)]
    return dict(xy=xy, conic=conic, opac=opac, rgb=rgb, depth=depth, radius=radius)
