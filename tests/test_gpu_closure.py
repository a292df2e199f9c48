"""What the learned closure gains over the method without it, and where.

A reduced version of the learned-closure workflow runs entirely on the GPU
through the library:
- fine 256^3 Taylor-Green runs at Re = 800, 1600 and 3200;
- box filtering by 4 into training samples for a 64^3 grid;
- about 1500 Adam steps;
- an a-posteriori scale of the network output chosen on coarse runs at the
  training Reynolds numbers;
- coarse 64^3 runs at Re = 1600 with plain BGK, Smagorinsky (Cs = 0.1), the
  raw learned closure and the calibrated one.

Each coarse run is judged by the relative L2 error of its dissipation rate
-dk/dt against the box-filtered fine run over 10 convective times.

The gain is specific to coarse grids past BGK's stability limit: at 64^3
(tau = 0.50076) plain BGK diverges before 10 convective times, and the
learned closure keeps the run stable with a bounded error.  On the 128^3
grid of the full workflow (512^3 filtered by 4) plain BGK is stable and its
dissipation error is smaller than that of any eddy-viscosity closure,
learned or Smagorinsky; test_closure_at_128_against_bgk records that case.
Smagorinsky is reported alongside; it is the fallback and the judge, not a
bar the network has to clear.
"""
import math

import pytest
import torch

from paper_2506_09242_gb300 import closure, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2506_09242_gb300 import _build
    _build.build()
    lbm.load()


def test_learned_closure_stabilises_the_underresolved_grid():
    res = closure.experiment(256, 4, (800.0, 1600.0, 3200.0), 1600.0, t_end=10.0, steps=1500,
                             samples_per_snapshot=200_000, seed=0)
    c = res["coarse"]
    print({k: (round(v["dissipation_rel_l2"], 4), v["diverged_at_tc"]) for k, v in c.items()})
    assert all(v is None for v in res["fine_diverged"].values())
    assert res["loss_first_last"][1] < res["loss_first_last"][0]
    mlp_err = c["mlp"]["dissipation_rel_l2"]
    assert c["mlp"]["diverged_at_tc"] is None
    assert math.isfinite(mlp_err) and mlp_err < 0.5
    assert mlp_err < c["bgk"]["dissipation_rel_l2"]
    cal = c["mlp_calibrated"]
    assert cal["diverged_at_tc"] is None
    assert cal["dissipation_rel_l2"] <= mlp_err
    assert cal["dissipation_rel_l2"] < c["bgk"]["dissipation_rel_l2"]


def test_closure_at_128_against_bgk():
    """The full workflow's grids (fine 512^3 at Re = 800, 1600, 3200, coarse
    128^3 at Re = 1600): every run stays stable and the learned closure keeps
    a bounded dissipation error.  The comparison is recorded, not required to
    favour the network: here plain BGK resolves the flow well enough that an
    added eddy viscosity, learned or Smagorinsky's, only adds dissipation, and
    the test pins that finding (BGK's error below Smagorinsky's)."""
    res = closure.experiment(512, 4, (800.0, 1600.0, 3200.0), 1600.0, t_end=10.0, steps=1500,
                             samples_per_snapshot=200_000, seed=0)
    c = res["coarse"]
    print({k: (round(v["dissipation_rel_l2"], 4), v["diverged_at_tc"]) for k, v in c.items()},
          "alpha", res["calibration"]["alpha"])
    assert all(v is None for v in res["fine_diverged"].values())
    for key in ("bgk", "smagorinsky", "mlp", "mlp_calibrated"):
        assert c[key]["diverged_at_tc"] is None, key
        assert math.isfinite(c[key]["dissipation_rel_l2"]) and c[key]["dissipation_rel_l2"] < 0.2, key
    assert c["bgk"]["dissipation_rel_l2"] < c["smagorinsky"]["dissipation_rel_l2"]
    assert c["mlp_calibrated"]["dissipation_rel_l2"] <= c["mlp"]["dissipation_rel_l2"] * 1.05
