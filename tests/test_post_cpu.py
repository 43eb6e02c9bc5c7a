"""Post-processing of the statistics: the forest friction velocity of Sec. 5
on synthetic profiles with known values."""
import numpy as np
import pytest

from paper_2206_15454_b300 import post


def test_at_height_interpolates_between_cell_centres():
    p = np.array([1.0, 3.0, 7.0])
    assert post.at_height(p, 0.5) == 1.0 and post.at_height(p, 1.5) == 3.0
    assert post.at_height(p, 1.0) == pytest.approx(2.0)
    assert post.at_height(p, 2.25) == pytest.approx(6.0)
    assert post.at_height(p, 0.0) == 1.0 and post.at_height(p, 9.0) == 7.0


def test_friction_velocity_of_known_stresses():
    ny, nb = 12, 3
    s = np.zeros((9, nb, ny))
    s[6] = -0.0009   # <u'v'>
    s[8] = 0.0012    # <v'w'>
    # (0.0009^2 + 0.0012^2)^(1/4) = 0.0015^(1/2)
    assert post.friction_velocity(s, 6.0) == pytest.approx(np.sqrt(0.0015), rel=1e-14)
    # a linear <u'v'> profile, <v'w'> = 0: |<u'v'>|^(1/2) at the height
    s[8] = 0.0
    s[6] = -(np.arange(ny) + 0.5)[None, :] * 1e-4 * np.array([1.0, 2.0, 3.0])[:, None]
    assert post.friction_velocity(s, 4.0) == pytest.approx(np.sqrt(4.0 * 2e-4), rel=1e-12)
    assert post.friction_velocity(s, 4.0, xbin=2) == pytest.approx(np.sqrt(4.0 * 3e-4), rel=1e-12)
