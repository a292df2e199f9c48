"""Pins of the oracle's lattice tables, equilibrium and small closed forms.

Each check is a property the mathematics fixes independently of how the oracle
is written: lattice isotropy (the moment identities that make the discrete
velocity set reproduce Navier-Stokes), the closed-form moments of the
second-order equilibrium, the Smagorinsky defining equation, library rounding
routines, and the performance-model figures printed in Sec. 4.1.
"""
import itertools
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle

KD = np.eye(3)


@pytest.mark.parametrize("Q", [19, 27])
def test_lattice_isotropy(Q):
    c, w, opp = oracle.lattice(Q)
    assert len({tuple(v) for v in c}) == Q
    assert np.all(np.abs(c) <= 1)
    if Q == 19:
        assert np.all(np.sum(c * c, axis=1) <= 2)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), KD / 3.0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", KD, KD) + np.einsum("ac,bd->abcd", KD, KD)
           + np.einsum("ad,bc->abcd", KD, KD)) / 9.0
    assert np.allclose(m4, iso, atol=1e-16)
    # opposites: an involution pairing c with -c, stored as adjacent pairs
    assert np.all(opp[opp] == np.arange(Q))
    assert np.all(c[opp] == -c)
    assert opp[0] == 0
    for i in range(1, Q, 2):
        assert opp[i] == i + 1


def test_d3q27_is_full_cube():
    c, _, _ = oracle.lattice(27)
    assert {tuple(v) for v in c} == set(itertools.product((-1, 0, 1), repeat=3))


def test_bad_lattice_rejected():
    with pytest.raises(ValueError):
        oracle.lattice(15)


@pytest.mark.parametrize("Q", [19, 27])
def test_equilibrium_moments(Q):
    c, _, _ = oracle.lattice(Q)
    rng = np.random.default_rng(7)
    for _ in range(50):
        rho = rng.uniform(0.5, 1.5)
        u = rng.uniform(-0.2, 0.2, size=3)
        feq = oracle.equilibrium(Q, rho, u)
        assert abs(feq.sum() - rho) < 1e-14
        assert np.allclose(np.einsum("i,ia->a", feq, c), rho * u, atol=1e-15)
        pi = np.einsum("i,ia,ib->ab", feq, c, c)
        assert np.allclose(pi, rho * np.outer(u, u) + rho / 3.0 * KD, atol=1e-14)


def test_smagorinsky_defining_equation():
    """tau_eff = tau0 + 3 nu_t with nu_t = Cs^2 |S|, |S| = sqrt(2 S:S) and
    S = -Pi / (2 rho c_s^2 tau_eff): the closed form must satisfy it."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        tau0 = rng.uniform(0.501, 1.5)
        cs = rng.uniform(0.05, 0.3)
        rho = rng.uniform(0.8, 1.2)
        pi6 = rng.normal(scale=1e-3, size=6)
        te = oracle.tau_smagorinsky(tau0, cs, rho, pi6)
        P = np.array([[pi6[0], pi6[3], pi6[4]], [pi6[3], pi6[1], pi6[5]], [pi6[4], pi6[5], pi6[2]]])
        S = -P / (2.0 * rho * (1.0 / 3.0) * te)
        Smag = np.sqrt(2.0 * np.sum(S * S))
        assert te == pytest.approx(tau0 + 3.0 * cs * cs * Smag, rel=1e-13)
        assert te >= tau0
    assert oracle.tau_smagorinsky(0.6, 0.0, 1.0, np.ones(6)) == 0.6


def test_storage_rounding_matches_library_routines():
    rng = np.random.default_rng(11)
    h = np.concatenate([rng.normal(scale=s, size=2000) for s in (1e-1, 1e-3, 1e-5, 1e-7)])
    f16 = np.float16(np.float32(h)).astype(np.float64)
    bf = torch.tensor(np.float32(h)).to(torch.bfloat16).to(torch.float64).numpy()
    f32 = np.float32(h).astype(np.float64)
    for k in range(len(h)):
        assert oracle.round_scalar(h[k], oracle.F16) == f16[k]
        assert oracle.round_scalar(h[k], oracle.BF16) == bf[k]
        assert oracle.round_scalar(h[k], oracle.F32) == f32[k]
        assert oracle.round_scalar(h[k], oracle.F64) == h[k]


def test_scaled_fp16_rounding():
    """FP16 of h * 2^12: the library conversion of the scaled value, a
    relative error within half an FP16 ulp (2^-11) for every |h| from 2^-26
    (the scaled normal threshold) up to 16, where plain FP16 goes subnormal
    below 6.1e-5 and loses that bound, and overflow to infinity from 16 on."""
    rng = np.random.default_rng(12)
    h = np.concatenate([rng.normal(scale=s, size=2000) for s in (1e-1, 1e-3, 1e-5, 1e-7)])
    lib16 = np.float16(np.float32(h) * np.float32(4096.0)).astype(np.float64) / 4096.0
    mag = np.abs(h)
    for k in range(len(h)):
        r = oracle.round_scalar(h[k], oracle.F16_SCALED)
        assert r == lib16[k]
        if 2.0 ** -26 <= mag[k] < 16.0:
            assert abs(r - h[k]) <= 2.0 ** -11 * mag[k]
    tiny = h[(mag > 1e-7) & (mag < 2e-6)]
    plain = np.array([oracle.round_scalar(v, oracle.F16) for v in tiny])
    assert np.max(np.abs(plain - tiny) / np.abs(tiny)) > 1e-2  # subnormal FP16
    assert oracle.round_scalar(16.0, oracle.F16_SCALED) == np.inf
    assert oracle.round_scalar(-16.5, oracle.F16_SCALED) == -np.inf
    assert oracle.round_scalar(15.99, oracle.F16_SCALED) == pytest.approx(15.99, rel=2.0 ** -11)
    assert oracle.round_scalar(2.0 ** -30, oracle.F16_SCALED) == 2.0 ** -30  # scaled 2^-18: exact subnormal


def test_round_storage_keeps_offset():
    c, w, _ = oracle.lattice(19)
    f = w[:, None] * (1.0 + np.linspace(-0.1, 0.1, 7)[None, :])
    g = oracle.round_storage(f, oracle.BF16)
    for i in range(19):
        for n in range(7):
            assert g[i, n] == w[i] + oracle.round_scalar(f[i, n] - w[i], oracle.BF16)


def _golden(name):
    """key = value fixture of tests/golden (comments after #)."""
    vals = {}
    for line in (Path(__file__).parent / "golden" / name).read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("=", 1))
            vals[k] = float(v)
    return vals


def test_performance_model_reproduces_paper():
    """Sec. 4.1: the printed peaks (9.481 and 4.921 GLUPS) and memory-use
    figures (51% and 99% at L = 500) from the bandwidth over
    n_t = 2*19*n_store + 12 bytes (fixture tests/golden/performance_model.txt,
    with the readings of the two garbled formulas)."""
    g = _golden("performance_model.txt")
    for n_store, peak in ((g["n_store_sp"], g["peak_glups_sp"]), (g["n_store_dp"], g["peak_glups_dp"])):
        model = oracle.glups_peak(g["bandwidth_bytes_per_s"], int(g["populations"]), int(n_store),
                                  int(g["flag_bytes"]))
        assert abs(model - peak) < 1e-3
    for n_store, pct in ((g["n_store_sp"], g["memory_percent_sp"]), (g["n_store_dp"], g["memory_percent_dp"])):
        n_t = 2 * g["populations"] * n_store + g["flag_bytes"]
        mem = n_t * g["memory_L"] ** 3 / g["gpu_memory_bytes"]
        assert round(100 * mem) == pct