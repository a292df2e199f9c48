"""Host-side piece of the cavity study that needs no GPU: the centreline
profiles, on synthetic fields whose profiles are known."""
import numpy as np
import pytest

from paper_2506_09242_gb300 import workloads


@pytest.mark.parametrize("n", [9, 10])
def test_cavity_profiles_pick_the_centrelines(n):
    """u_x depending on z only and u_z on x only: the vertical and horizontal
    centreline profiles are those functions over the fluid nodes 1 .. n-2 (for
    even n the average of the four lines around the centre, equal here), at
    positions symmetric between the two halfway walls."""
    z = np.arange(n, dtype=float)
    u = np.zeros((3, n, n, n))
    u[0] = (np.sin(z) + 2.0)[:, None, None]          # u_x(z)
    u[2] = (np.cos(z) - 3.0)[None, None, :]          # u_z(x)
    u[1] = 7.0                                       # ignored
    xi, ux, uz = workloads._cavity_profiles(u, n, 0.5)
    k = np.arange(1, n - 1)
    assert np.allclose(ux, (np.sin(k) + 2.0) / 0.5, rtol=0, atol=1e-15)
    assert np.allclose(uz, (np.cos(k) - 3.0) / 0.5, rtol=0, atol=1e-15)
    assert xi[0] == pytest.approx(0.5 / (n - 2)) and xi[0] + xi[-1] == pytest.approx(1.0)
    assert np.all(np.diff(xi) > 0)
