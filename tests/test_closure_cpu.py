"""Host-side pieces of the closure workflow that need no GPU: the convective
scaling of the Taylor-Green relaxation time (coarse and fine grids at one
Reynolds number) and the dissipation-rate error that judges every coarse run."""
import math

import numpy as np
import pytest

from paper_2506_09242_gb300 import closure


def test_tgv_tau_convective_scaling():
    """tau - 1/2 = 3 nu with nu = u0 L / Re and L = n / (2 pi): at fixed Re
    and u0, nu grows linearly with the grid, so a 4x coarser grid has a 4x
    smaller tau - 1/2; one convective time is n / (2 pi u0) steps."""
    fine = closure.tgv_tau(512, 1600.0)
    coarse = closure.tgv_tau(128, 1600.0)
    assert fine == pytest.approx(0.5 + 3 * 0.04 * (512 / (2 * math.pi)) / 1600, rel=1e-15)
    assert (fine - 0.5) == pytest.approx(4 * (coarse - 0.5), rel=1e-14)
    assert round(fine, 6) == 0.506112
    assert closure.steps_per_tc(512) == pytest.approx(4 * closure.steps_per_tc(128), rel=1e-15)


def _runs(kf, kc, t):
    fine = closure.FineRun(re=1600.0, n=64, factor=4, times=t, k_filtered=kf, k_full=2 * kf)
    coarse = closure.CoarseRun(closure="bgk", times=t, k=kc, glups=1.0, diverged_at=None)
    return fine, coarse


def test_dissipation_error_closed_forms():
    t = np.linspace(0.0, 10.0, 101)
    kf = 0.125 * np.exp(-0.3 * t)
    fine, coarse = _runs(kf, kf.copy(), t)
    assert closure.dissipation_error(fine, coarse) == 0.0
    # twice the energy decays at twice the rate: a relative error of exactly 1
    fine, coarse = _runs(kf, 2 * kf, t)
    assert closure.dissipation_error(fine, coarse) == pytest.approx(1.0, rel=1e-12)
    # against the unfiltered run (k_full = 2 k_filtered here) the same run is exact
    assert closure.dissipation_error(fine, coarse, reference="fine") == pytest.approx(0.0, abs=1e-15)
    # a constant offset in k does not change the dissipation rate
    fine, coarse = _runs(kf, kf + 0.01, t)
    assert closure.dissipation_error(fine, coarse) == pytest.approx(0.0, abs=1e-12)


def test_dissipation_error_of_a_diverged_or_short_run_is_infinite():
    t = np.linspace(0.0, 10.0, 101)
    kf = np.exp(-t)
    fine, coarse = _runs(kf, kf.copy(), t)
    coarse.diverged_at = 8.1
    assert closure.dissipation_error(fine, coarse) == math.inf
    fine, coarse = _runs(kf, kf[:50].copy(), t)
    coarse.times = t[:50]
    assert closure.dissipation_error(fine, coarse) == math.inf
