"""Parity of the library's Risky Gate (host arithmetic inside libolap.so, so
this runs without a GPU) with the gate oracle (Sec. II-B decision; Sec. V-D
fits and break-even N*): fitted coefficients within 1e-9 relative (fp64 with
a different summation order), the same CPU form, and the same decisions and
N* away from knife-edge ties."""
import math

import numpy as np
import pytest

from oracle import gate
from paper_2601_19911_gb300 import build, olap


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return olap.load()


def _noisy_samples(rng, op, form, count=24):
    n = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(1e8), count)))
    if op == gate.TOPK:
        km = np.floor(np.exp(rng.uniform(0, np.log(1e5), count)))
        km = np.minimum(km, n)
        x = n * np.log2(n) if form == gate.CPU_NLOGN else n * km
        out = km
        bpr = 8.0
    else:
        km = rng.uniform(1.0, 3.5, count)
        x = n * km
        out = n * (km - 1.0)
        bpr = 8.0
    noise = lambda: 1.0 + rng.normal(0.0, 0.03, count)
    t_cpu = (2e-6 * x + 0.05) * noise()
    tx = bpr * n
    t_tx = (1.0 / 2.0e8 * tx + 0.02) * noise()
    t_ker = (2e-8 * n + 0.01) * noise()
    t_post = (5e-7 * out + 0.005) * noise()
    return n, km, tx, out, t_cpu, t_tx, t_ker, t_post


@pytest.mark.parametrize("op,form,topk_cpu", [(gate.TOPK, gate.CPU_NLOGN, 0), (gate.TOPK, gate.CPU_NK, 0),
                                              (gate.PROBE, gate.CPU_NM, 0), (gate.TOPK, gate.CPU_NLOGN, gate.CPU_MAX),
                                              (gate.TOPK, gate.CPU_NK, gate.CPU_MAX)])
@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("weighting", [gate.ORDINARY, gate.RELATIVE])
def test_calibrate_and_decide_match_oracle(op, form, topk_cpu, seed, weighting):
    rng = np.random.default_rng(seed)
    smp = _noisy_samples(rng, op, form)
    for margin in (0.0, 5.0, 10.0):
        want = gate.calibrate(op, *smp, margin_ms=margin, weighting=weighting, topk_cpu=topk_cpu)
        got = olap.gate_calibrate(op, *smp, margin_ms=margin, weighting=weighting, topk_cpu=topk_cpu)
        assert got.cpu_form == want.cpu_form
        for nm in ("a", "b", "c", "d", "e", "f", "g", "h", "a2", "b2"):
            assert math.isclose(getattr(got, nm), getattr(want, nm), rel_tol=1e-9, abs_tol=1e-15), nm
        qn = np.floor(np.exp(rng.uniform(np.log(1e2), np.log(1e9), 50))).astype(np.int64)
        for nq in qn:
            km = 100.0 if op == gate.TOPK else 1.9
            out = min(km, nq) if op == gate.TOPK else nq * (km - 1.0)
            d = olap.gate_estimate(got, op, nq, km, 8.0 * nq, out, 8.0, km - 1.0)
            c = gate.costs(want, nq, km, 8.0 * nq, out)
            gain = c[0] - (c[1] + c[2] + c[3])
            if abs(gain - margin) > 1e-9 * max(1.0, abs(gain)):
                assert bool(d.offload) == (gain > margin)
            assert math.isclose(d.c_cpu, c[0], rel_tol=1e-9, abs_tol=1e-12)
            ns = gate.n_star(want, km, 8.0, km - 1.0, km if op == gate.TOPK else None)
            assert abs(int(d.n_star) - ns) <= max(1, ns * 1e-9)


@pytest.mark.parametrize("op,form,topk_cpu", [(gate.TOPK, gate.CPU_NLOGN, 0), (gate.TOPK, gate.CPU_NK, 0),
                                              (gate.PROBE, gate.CPU_NM, 0), (gate.TOPK, gate.CPU_NLOGN, gate.CPU_MAX)])
@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("weighting", [gate.ORDINARY, gate.RELATIVE])
def test_two_regime_fit_matches_oracle(op, form, topk_cpu, seed, weighting):
    """A CPU engine with two regimes (serial below 131072 rows, parallel
    above, as the host engine): the library's per-regime fits, decisions and
    N* against the oracle's."""
    rng = np.random.default_rng(100 + seed)
    n, km, tx, out, t_cpu, t_tx, t_ker, t_post = _noisy_samples(rng, op, form, count=30)
    split = 131072.0
    t_cpu = np.where(n < split, t_cpu, t_cpu * 0.15 + 0.2)     # the parallel regime: cheaper slope, a hand-off
    smp = (n, km, tx, out, t_cpu, t_tx, t_ker, t_post)
    for margin in (0.0, 5.0):
        want = gate.calibrate(op, *smp, margin_ms=margin, weighting=weighting, topk_cpu=topk_cpu,
                              cpu_split_n=split)
        got = olap.gate_calibrate(op, *smp, margin_ms=margin, weighting=weighting, topk_cpu=topk_cpu,
                                  cpu_split_n=split)
        assert got.cpu_form == want.cpu_form and got.split_n == split
        for nm in ("a", "b", "c", "d", "e", "f", "g", "h", "a2", "b2", "a_hi", "b_hi", "a2_hi", "b2_hi"):
            assert math.isclose(getattr(got, nm), getattr(want, nm), rel_tol=1e-9, abs_tol=1e-15), nm
        for nq in (1000, 50_000, 131_071, 131_072, 10**6, 10**8):
            kq = 100.0 if op == gate.TOPK else 1.9
            outq = min(kq, nq) if op == gate.TOPK else nq * (kq - 1.0)
            d = olap.gate_estimate(got, op, nq, kq, 8.0 * nq, outq, 8.0, kq - 1.0)
            c = gate.costs(want, nq, kq, 8.0 * nq, outq)
            assert math.isclose(d.c_cpu, c[0], rel_tol=1e-9, abs_tol=1e-12)
            ns = gate.n_star(want, kq, 8.0, kq - 1.0, kq if op == gate.TOPK else None)
            assert abs(int(d.n_star) - ns) <= max(1, ns * 1e-9)


def test_two_regime_needs_two_samples_per_side():
    n = [1e3, 2e3, 5e3, 1e6]
    z = [0.1] * 4
    with pytest.raises(olap.OlapError):
        olap.gate_calibrate(gate.TOPK, n, [10.0] * 4, n, [10.0] * 4, z, z, z, z, cpu_split_n=1e5)


def test_exact_knife_edge_is_not_offloaded():
    # dyadic constants: C_cpu - C_gpu equals the margin exactly (the paper's
    # "exceeds" is strict).  n=8, M=2: C_cpu = 0.5*16 + 1 = 9; C_tx = 0.25*8 +
    # 0.5 = 2.5; C_ker = 0.125*8 = 1; C_post = 0 -> gain 5.5.
    model = olap.olap_gate_model(gate.PROBE, gate.CPU_NM, 0.5, 1.0, 0.25, 0.5, 0.125, 0.0, 0.0, 0.0, 5.5, 0.0, 0.0,
                                 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0)
    d = olap.gate_estimate(model, gate.PROBE, 8, 2.0, 8.0, 0.0)
    assert d.gain_ms == 5.5 and d.offload == 0
    model.margin_ms = 5.25
    assert olap.gate_estimate(model, gate.PROBE, 8, 2.0, 8.0, 0.0).offload == 1
    o = gate.Model(gate.PROBE, gate.CPU_NM, 0.5, 1.0, 0.25, 0.5, 0.125, 0.0, 0.0, 0.0, 5.5)
    assert not gate.decide(o, 8, 2.0, 8.0, 0.0)


def test_rejects_bad_input():
    with pytest.raises(olap.OlapError):
        olap.gate_calibrate(gate.TOPK, [1.0], [1.0], [1.0], [1.0], [1.0], [1.0], [1.0], [1.0])


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("weighting", [gate.ORDINARY, gate.RELATIVE])
def test_signed_component_samples_match_oracle(seed, weighting):
    """Transfer and post-processing measured as differences of calls can come
    out zero or slightly negative near the break-even; both sides then weigh
    such a sample, under 1/y^2 weights, like the smallest positive one."""
    rng = np.random.default_rng(100 + seed)
    n, km, tx, out, t_cpu, t_tx, t_ker, t_post = _noisy_samples(rng, gate.TOPK, gate.CPU_NLOGN)
    t_post = t_post - 0.006                      # about half the samples at or below zero
    t_tx = t_tx.copy()
    t_tx[::7] = -0.001
    t_post[3] = 0.0
    assert (t_post <= 0).any() and (t_post > 0).any()
    for margin in (0.0, 5.0):
        want = gate.calibrate(gate.TOPK, n, km, tx, out, t_cpu, t_tx, t_ker, t_post, margin_ms=margin,
                              weighting=weighting, cpu_split_n=131072.0)
        got = olap.gate_calibrate(gate.TOPK, n, km, tx, out, t_cpu, t_tx, t_ker, t_post, margin_ms=margin,
                                  weighting=weighting, cpu_split_n=131072.0)
        for nm in ("a", "b", "c", "d", "e", "f", "g", "h", "a_hi", "b_hi"):
            assert math.isclose(getattr(got, nm), getattr(want, nm), rel_tol=1e-9, abs_tol=1e-15), nm
        d = olap.gate_estimate(got, gate.TOPK, 1 << 20, 100.0, 8.0 * (1 << 20), 100.0, 8.0)
        assert abs(int(d.n_star) - gate.n_star(want, 100.0, 8.0, 0.0, 100.0)) <= 1


def test_relative_weights_of_non_positive_samples():
    """The weighting rule itself: 1 / y^2, with a sample at or below zero
    weighted like the smallest positive one (and all ones when none is)."""
    w = gate.weights([2.0, -1.0, 0.0, 4.0], gate.RELATIVE)
    np.testing.assert_allclose(w, [0.25, 0.25, 0.25, 1.0 / 16.0])
    np.testing.assert_allclose(gate.weights([-1.0, 0.0], gate.RELATIVE), [1.0, 1.0])
    np.testing.assert_allclose(gate.weights([-1.0, 5.0], gate.ORDINARY), [1.0, 1.0])
