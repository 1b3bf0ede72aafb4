"""Closed-form pins of the oracle's projection conventions (Sec. 3.1, the 3DGS
model): the covariance R S S^T R^T of a rotated anisotropic Gaussian, with
the rotation matrices written out and quaternions composed by the Hamilton
product, so that a transposed rotation or a swapped quaternion component
fails; the EWA Jacobian's off-axis column through an off-centre isotropic
Gaussian; and the SH view direction (centre minus camera, not the reverse)
through degree-1 colour seen from opposite sides."""
import math

import numpy as np
import pytest

from paper_2606_15924_gb300 import scenes


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def _rx(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def _hamilton(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def _gauss(mean, scales, quat, dc=(0.2, 0.2, 0.2)):
    g = dict(means=np.array([mean], float), log_scales=np.log(np.array([scales], float)),
             quats=np.array([quat], float), opacity_logits=np.array([1.0]), sh=np.zeros((1, 16, 3)))
    g["sh"][0, 0, :] = dc
    return g


def _conic_of(S2):
    inv = np.linalg.inv(S2)
    return np.array([inv[0, 0], inv[0, 1], inv[1, 1]])


@pytest.mark.parametrize("theta,phi", [(0.6, 0.0), (-1.1, 0.0), (0.6, 0.9), (2.3, -0.4)])
def test_rotated_anisotropic_covariance(orc, theta, phi):
    """Camera at (0, 0, -d) looking at the origin has R = I, so at the image
    centre Sigma2 = (f / d)^2 Sigma[:2, :2] + 0.3 I with Sigma = R D R^T and
    R = Rz(theta) Rx(phi) for the quaternion qz(theta) * qx(phi)."""
    d, W, H = 4.0, 64, 48
    cam = scenes.look_at((0.0, 0.0, -d), width=W, height=H, fov_x_deg=50.0)
    assert np.allclose(np.asarray(cam["viewmat"])[:3, :3], np.eye(3))
    f = cam["fx"]
    sc = (0.09, 0.03, 0.05)
    qz = np.array([math.cos(theta / 2), 0.0, 0.0, math.sin(theta / 2)])
    qx = np.array([math.cos(phi / 2), math.sin(phi / 2), 0.0, 0.0])
    q = _hamilton(qz, qx)
    pr = orc.project(_gauss((0.0, 0.0, 0.0), sc, q), cam)
    R = _rz(theta) @ _rx(phi)
    Sigma = R @ np.diag(np.square(sc)) @ R.T
    S2 = (f / d) ** 2 * Sigma[:2, :2] + 0.3 * np.eye(2)
    np.testing.assert_allclose(pr["conic"][0], _conic_of(S2), rtol=1e-10)
    # an unnormalised quaternion gives the same Gaussian
    pr2 = orc.project(_gauss((0.0, 0.0, 0.0), sc, 3.7 * q), cam)
    np.testing.assert_allclose(pr2["conic"][0], pr["conic"][0], rtol=1e-12)


@pytest.mark.parametrize("x0,y0", [(0.3, 0.2), (-0.4, 0.25), (0.1, -0.35)])
def test_off_centre_jacobian(orc, x0, y0):
    """An isotropic Gaussian at (x0, y0, 0) seen from (0, 0, -d): depth z = d,
    centre (f x0 / z + cx, f y0 / z + cy), and Sigma2 = s^2 J J^T + 0.3 I with
    J = [[f/z, 0, -f x0/z^2], [0, f/z, -f y0/z^2]] (no clamp this close to
    the axis)."""
    d, W, H, s = 4.0, 64, 48, 0.05
    cam = scenes.look_at((0.0, 0.0, -d), width=W, height=H, fov_x_deg=50.0)
    f = cam["fx"]
    pr = orc.project(_gauss((x0, y0, 0.0), (s, s, s), (1.0, 0.0, 0.0, 0.0)), cam)
    z = d
    assert pr["depth"][0] == pytest.approx(z, rel=1e-12)
    np.testing.assert_allclose(pr["xy"][0], [f * x0 / z + W / 2, f * y0 / z + H / 2], rtol=1e-12)
    J = np.array([[f / z, 0.0, -f * x0 / z ** 2], [0.0, f / z, -f * y0 / z ** 2]])
    S2 = s * s * J @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(pr["conic"][0], _conic_of(S2), rtol=1e-10)
    assert pr["conic"][0][1] * x0 * y0 < 0.0      # the off-diagonal term is present, with its sign


def test_sh_direction_is_centre_minus_camera(orc):
    """Degree-1 colour of a Gaussian at the origin, seen from six cameras on
    the axes: rgb = max(0, sum_k c_k Y_k(dir) + 0.5) with dir = (mu - C) / |mu - C|
    and Y the SH basis (itself pinned to scipy)."""
    coef = np.zeros((16, 3))
    coef[0] = (0.1, 0.0, -0.1)
    coef[1] = (0.3, -0.2, 0.1)
    coef[2] = (-0.25, 0.15, 0.2)
    coef[3] = (0.2, 0.3, -0.3)
    seen = []
    for pos in ((0, 0, -4.0), (0, 0, 4.0), (4.0, 0, 0), (-4.0, 0, 0), (0, 4.0, 0.001), (0, -4.0, 0.001)):
        cam = scenes.look_at(pos, width=32, height=32)
        g = _gauss((0.0, 0.0, 0.0), (0.05, 0.05, 0.05), (1.0, 0.0, 0.0, 0.0))
        g["sh"][0] = coef
        pr = orc.project(g, cam, sh_degree=1)
        C = -np.asarray(cam["viewmat"])[:3, :3].T @ np.asarray(cam["viewmat"])[:3, 3]
        dvec = -C / np.linalg.norm(C)
        Y, _ = orc.sh_basis(dvec)
        want = np.maximum(0.0, Y[:4] @ coef[:4] + 0.5)
        np.testing.assert_allclose(pr["rgb"][0], want, rtol=1e-6, atol=1e-9)
        seen.append(pr["rgb"][0])
    # opposite cameras see different colours (the degree-1 terms change sign)
    assert np.abs(seen[0] - seen[1]).max() > 0.05 and np.abs(seen[2] - seen[3]).max() > 0.05
