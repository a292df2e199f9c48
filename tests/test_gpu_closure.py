"""What the learned closure gains over the method without it.

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
-dk/dt against the box-filtered fine run over 10 convective times. The
method without the network (plain BGK on the coarse grid) must do worse than
the learned closure, by diverging or by a larger error. The learned closure
must stay stable with a bounded error. Smagorinsky is reported alongside; it
is the fallback and the judge, not a bar the network has to clear.
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


def test_learned_closure_beats_plain_bgk_on_the_coarse_grid():
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
