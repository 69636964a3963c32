"""The sphere post-processing of bench.py (closed wake length L, separation
angle theta) on fields whose answers are known, CPU only."""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2304_09485_gb300 import inputs as I  # noqa: E402


def test_wake_length_and_separation_angle_of_a_synthetic_field():
    """u_x on the downstream axis changes sign at x = 0.5 + L0 (linear in x there),
    and the first layer's meridional velocity is proportional to (theta_s - theta):
    the post-processing returns L0 and theta_s to interpolation accuracy."""
    layers = 12
    st = I.sphere_stretch(layers, dr1=3e-2)
    m = I.hex_sphere_mesh(16, layers, stretch=st)
    radii = I.sphere_radii(layers, 0.5, 10.0, st)
    cen = m.xyz[m.hex8].mean(1)
    L0, theta_s = 0.9, 127.0
    r = np.linalg.norm(cen, axis=1)
    cn = cen / r[:, None]
    th = np.degrees(np.arccos(np.clip(-cn[:, 0], -1, 1)))
    e = np.array([1.0, 0.0, 0.0])[None, :] - cn * cn[:, :1]
    e_th = e / np.maximum(np.linalg.norm(e, axis=1), 1e-30)[:, None]
    u = e_th * (theta_s - th)[:, None] * 0.01                    # separation at theta_s
    axis = (cen[:, 0] > 0.5) & (np.linalg.norm(cen[:, 1:], axis=1) < 0.2)
    u[axis] = np.array([1.0, 0.0, 0.0]) * (cen[axis, 0] - (0.5 + L0))[:, None]
    Q = np.zeros((m.n_cells, 5))
    Q[:, 0] = 1.3
    Q[:, 1:4] = 1.3 * u
    Q[:, 4] = 2.0
    L, theta = bench.wake_and_separation(m, Q, radii)
    assert abs(L - L0) <= 1e-9
    assert abs(theta - theta_s) <= 0.5                             # 2-degree bins, azimuthal means: 0.14
