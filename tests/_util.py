"""Shared helpers for the tests (no method arithmetic)."""
import math

import numpy as np


def quat_angle(q1, q2) -> float:
    """Rotation angle between unit quaternions: 2 atan2(|vec(q1* q2)|, |w(q1* q2)|)."""
    w1, v1 = float(q1[0]), np.asarray(q1[1:], np.float64)
    w2, v2 = float(q2[0]), np.asarray(q2[1:], np.float64)
    w = w1 * w2 + v1 @ v2
    v = w1 * v2 - w2 * v1 - np.cross(v1, v2)
    return 2.0 * math.atan2(float(np.linalg.norm(v)), abs(w))


def f32(x: float) -> float:
    """The float32 value the library receives for delta, as a Python float."""
    return float(np.float32(x))
