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


def test_size_sweep_plan_counts_the_population_arrays():
    """Two arrays with A/B, one with AA; rows padded to 32 nodes and planes
    to 256 values; sizes past 80% of the free memory are left out."""
    gb = 10 ** 9
    plan = workloads.sweep_plan([64, 100, 512, 1024], 19, "f32", "ab", device_bytes=284 * gb, free_bytes=280 * gb)
    sizes = [n for n, _, _ in plan]
    assert sizes == [64, 100, 512, 1024]
    by_n = {n: b for n, b, _ in plan}
    assert by_n[512] == 2 * 19 * 512 ** 3 * 4          # 20.4 GB, as the bench reports
    px = 128                                             # 100 padded to a multiple of 32
    plane = (px * 100 * 100 + 255) // 256 * 256
    assert by_n[100] == 2 * 19 * plane * 4
    assert by_n[1024] == 2 * 19 * 1024 ** 3 * 4          # 163 GB: fits in 80% of 280 GB
    tight = workloads.sweep_plan([512, 1024], 19, "f32", "ab", device_bytes=284 * gb, free_bytes=150 * gb)
    assert [n for n, _, _ in tight] == [512]
    aa = workloads.sweep_plan([1024], 19, "f64", "aa", device_bytes=284 * gb, free_bytes=280 * gb)
    assert aa[0][1] == 19 * 1024 ** 3 * 8 and aa[0][2] == pytest.approx(19 * 8 * 1024 ** 3 / (284 * gb))
    # D3Q27 FP64 at 1024^3 needs 232 GB even with AA: more than 80% of 280 GB
    assert workloads.sweep_plan([1024], 27, "f64", "aa", device_bytes=284 * gb, free_bytes=280 * gb) == []
