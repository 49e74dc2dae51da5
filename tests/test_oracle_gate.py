"""Pins for the gate oracle (Sec. II-B cost models and decision; Sec. V-D
least-squares fits and break-even N*): exact recovery of known coefficients,
a closed-form N* for the linear CPU model, the defining sign change at N*,
and the strictness of "exceeds"."""
import math

import numpy as np
import pytest

from oracle import gate


def _samples(a, b, c, d, e, f, g, h, form, bytes_per_row=8):
    n = np.unique(np.floor(np.logspace(3, 8, 20)).astype(np.int64))
    kk = np.array([10, 100, 1000, 37] * 5, dtype=np.int64)[: n.shape[0]]
    if form == gate.CPU_NLOGN:
        t_cpu = a * n * np.log2(n) + b
    else:
        t_cpu = a * n * kk + b
    tx = bytes_per_row * n
    out = np.minimum(kk, n)
    return n, kk, tx, out, t_cpu, c * tx + d, e * n + f, g * out + h


@pytest.mark.parametrize("form", [gate.CPU_NLOGN, gate.CPU_NK])
def test_recovers_known_coefficients(form):
    co = dict(a=3.1e-6, b=0.25, c=2.5e-9, d=0.04, e=1.5e-7, f=0.01, g=3e-6, h=0.002)
    n, kk, tx, out, t_cpu, t_tx, t_ker, t_post = _samples(**co, form=form)
    m = gate.calibrate(gate.TOPK, n, kk, tx, out, t_cpu, t_tx, t_ker, t_post)
    assert m.cpu_form == form
    for name, want in co.items():
        assert math.isclose(getattr(m, name), want, rel_tol=1e-9, abs_tol=1e-12), name


def test_linear_model_closed_form_n_star():
    # T_cpu = a*N*K + b, C_gpu = (c*w + e)*N + (d + f + g*K + h): the root is
    # N = (d + f + g*K + h + margin - b) / (a*K - c*w - e).
    m = gate.Model(gate.TOPK, gate.CPU_NK, a=1e-6, b=0.0, c=1e-8, d=2.0, e=1e-7, f=0.5,
                   g=0.0, h=0.25, margin_ms=5.0)
    k, w = 100, 8
    root = (2.0 + 0.5 + 0.25 + 5.0 - 0.0) / (1e-6 * k - 1e-8 * w - 1e-7)
    ns = gate.n_star(m, k, w, out_fixed=k)
    assert ns == math.floor(root) + 1
    assert gate.gain(m, ns, k, w, 0.0, k) > 0.0 >= gate.gain(m, ns - 1, k, w, 0.0, k)


def test_nlogn_bisection_defining_property():
    m = gate.Model(gate.TOPK, gate.CPU_NLOGN, a=2e-6, b=0.01, c=2e-9, d=0.05, e=1e-7,
                   f=0.02, g=1e-6, h=0.01, margin_ms=0.0)
    for margin in (0.0, 5.0, 10.0):
        m.margin_ms = margin
        ns = gate.n_star(m, 100, 8, out_fixed=100)
        assert 1 < ns < gate.N_STAR_HI
        assert gate.gain(m, ns, 100, 8, 0.0, 100) > 0.0 >= gate.gain(m, ns - 1, 100, 8, 0.0, 100)
    # a larger margin moves the switching point up (Sec. IV, gate margin)
    ns0 = gate.n_star(gate.Model(**{**m.__dict__, "margin_ms": 0.0}), 100, 8, out_fixed=100)
    ns10 = gate.n_star(gate.Model(**{**m.__dict__, "margin_ms": 10.0}), 100, 8, out_fixed=100)
    assert ns10 > ns0


def test_n_star_edges():
    never = gate.Model(gate.TOPK, gate.CPU_NK, a=0.0, b=0.0, c=1.0, d=1.0, e=0.0, f=0.0,
                       g=0.0, h=0.0, margin_ms=0.0)
    assert gate.n_star(never, 10, 8, out_fixed=10) == 0
    always = gate.Model(gate.TOPK, gate.CPU_NK, a=1.0, b=100.0, c=0.0, d=0.0, e=0.0, f=0.0,
                        g=0.0, h=0.0, margin_ms=0.0)
    assert gate.n_star(always, 10, 8, out_fixed=10) == 1


def test_decision_is_strict():
    # dyadic values so the sums are exact: C_cpu - C_gpu == margin exactly
    m = gate.Model(gate.PROBE, gate.CPU_NM, a=0.5, b=1.0, c=0.25, d=0.5, e=0.125, f=0.0,
                   g=0.0, h=0.0, margin_ms=2.0)
    # n=8, M=2: c_cpu = 0.5*16+1 = 9; c_tx = 0.25*8+0.5 = 2.5; c_ker = 1; gpu = 3.5 -> gain 5.5
    assert gate.decide(m, 8, 2, 8, 0)
    m.margin_ms = 5.5
    assert not gate.decide(m, 8, 2, 8, 0)
    m.margin_ms = 5.25
    assert gate.decide(m, 8, 2, 8, 0)


def test_probe_fit():
    n = np.array([1e3, 1e4, 1e5, 1e6, 1e7])
    mm = np.array([1.1, 1.9, 2.5, 1.5, 3.0])
    t_cpu = 4e-6 * n * mm + 0.3
    m = gate.calibrate(gate.PROBE, n, mm, 8 * n, n, t_cpu, 1e-9 * 8 * n + 0.01, 1e-8 * n, 1e-9 * n)
    assert m.cpu_form == gate.CPU_NM
    assert math.isclose(m.a, 4e-6, rel_tol=1e-9) and math.isclose(m.b, 0.3, rel_tol=1e-9)


def test_relative_weighting_recovers_exact_data_and_favours_small_points():
    # exact data: both weightings recover the coefficients
    co = dict(a=3.1e-6, b=0.25, c=2.5e-9, d=0.04, e=1.5e-7, f=0.01, g=3e-6, h=0.002)
    smp = _samples(**co, form=gate.CPU_NLOGN)
    m = gate.calibrate(gate.TOPK, *smp, weighting=gate.RELATIVE)
    for name, want in co.items():
        assert math.isclose(getattr(m, name), want, rel_tol=1e-9, abs_tol=1e-12), name
    # a fixed cost at small x and a different slope at large x: the relative
    # fit keeps the small-x intercept, the ordinary fit does not
    x = np.array([1e3, 1e4, 1e5, 1e6, 1e7, 1e8])
    y = np.array([0.05, 0.05, 0.06, 0.15, 1.0, 10.0])
    s_o, i_o = gate.ols(x, y, gate.ORDINARY)
    s_r, i_r = gate.ols(x, y, gate.RELATIVE)
    assert abs(i_r - 0.05) < abs(i_o - 0.05)
    # weights 1/y^2 by hand on two points reduce to the line through them
    s2, i2 = gate.ols([1.0, 3.0], [2.0, 4.0], gate.RELATIVE)
    assert math.isclose(s2, 1.0) and math.isclose(i2, 1.0)


def test_max_form_keeps_both_fits_and_takes_the_larger():
    """CPU_MAX: each form's coefficients are that form's own least-squares
    fit (checked against numpy.polyfit, a different routine), and the CPU
    estimate is the larger of the two, at every (N, K)."""
    rng = np.random.default_rng(11)
    n = np.floor(np.exp(rng.uniform(np.log(1e3), np.log(1e8), 30)))
    k = np.minimum(np.floor(np.exp(rng.uniform(0, np.log(1e5), 30))), n)
    t_cpu = (3e-9 * n * np.log2(n) + 1e-9 * n * k + 0.02) * (1.0 + rng.normal(0, 0.02, 30))
    z = np.zeros(30)
    m = gate.calibrate(gate.TOPK, n, k, 8 * n, k, t_cpu, z + 0.1, z + 0.1, z + 0.1, topk_cpu=gate.CPU_MAX)
    assert m.cpu_form == gate.CPU_MAX
    a1, b1 = np.polyfit(n * np.log2(n), t_cpu, 1)
    a2, b2 = np.polyfit(n * k, t_cpu, 1)
    for got, want in ((m.a, a1), (m.b, b1), (m.a2, a2), (m.b2, b2)):
        assert math.isclose(got, want, rel_tol=1e-7, abs_tol=1e-12)
    for ni, ki in ((1e3, 1.0), (1e6, 1e5), (1e8, 10.0), (5e4, 5e4)):
        c_cpu = gate.costs(m, ni, ki, 8 * ni, ki)[0]
        assert math.isclose(c_cpu, max(m.a * ni * math.log2(ni) + m.b, m.a2 * ni * ki + m.b2), rel_tol=1e-14)


# ---------------------------------------------------------------------------
# Two CPU regimes (a host engine that goes parallel above a size)
# ---------------------------------------------------------------------------

def _two_regime_samples(split, lo, hi, form=gate.CPU_NLOGN):
    n = np.unique(np.floor(np.logspace(3, 8, 24)).astype(np.int64))
    kk = np.array([10, 100, 1000, 37] * 6, dtype=np.int64)[: n.shape[0]]
    x = n * np.log2(n) if form == gate.CPU_NLOGN else n * kk
    t_cpu = np.where(n < split, lo[0] * x + lo[1], hi[0] * x + hi[1])
    tx = 8 * n
    out = np.minimum(kk, n)
    return n, kk, tx, out, t_cpu, 2e-9 * tx + 0.03, 1e-7 * n + 0.01, 1e-6 * out + 0.002


@pytest.mark.parametrize("form", [gate.CPU_NLOGN, gate.CPU_NK])
def test_two_regimes_recover_each_regime(form):
    """Exact timings that follow one line below the split and another above
    it: each regime's coefficients come back exactly, in the right form."""
    lo, hi = (6e-6, 0.002), (4e-7, 0.2)
    smp = _two_regime_samples(131072, lo, hi, form)
    for wt in (gate.ORDINARY, gate.RELATIVE):
        m = gate.calibrate(gate.TOPK, *smp, weighting=wt, cpu_split_n=131072)
        assert m.cpu_form == form and m.split_n == 131072
        for got, want in ((m.a, lo[0]), (m.b, lo[1]), (m.a_hi, hi[0]), (m.b_hi, hi[1])):
            assert math.isclose(got, want, rel_tol=1e-9, abs_tol=1e-12)
        # below and above the split the estimate follows its own regime
        assert math.isclose(gate.costs(m, 1e4, 10, 8e4, 10)[0],
                            lo[0] * (1e4 * math.log2(1e4) if form == gate.CPU_NLOGN else 1e5) + lo[1],
                            rel_tol=1e-9)
        assert math.isclose(gate.costs(m, 1e7, 10, 8e7, 10)[0],
                            hi[0] * (1e7 * math.log2(1e7) if form == gate.CPU_NLOGN else 1e8) + hi[1],
                            rel_tol=1e-9)


def test_two_regimes_one_line_is_no_split():
    # timings on one line: the split changes nothing but where the fit is made
    co = dict(a=3.1e-6, b=0.25, c=2.5e-9, d=0.04, e=1.5e-7, f=0.01, g=3e-6, h=0.002)
    smp = _samples(**co, form=gate.CPU_NLOGN)
    m0 = gate.calibrate(gate.TOPK, *smp)
    m1 = gate.calibrate(gate.TOPK, *smp, cpu_split_n=1e5)
    for nm in ("a", "b"):
        assert math.isclose(getattr(m1, nm), getattr(m0, nm), rel_tol=1e-9)
        assert math.isclose(getattr(m1, nm + "_hi"), getattr(m0, nm), rel_tol=1e-9)


def _linear_two(split, lo, hi, margin=0.0):
    # CPU a*N*K + b per regime; GPU C = 1e-8*8*N + 0.5 (transfer) + 0 + 0
    return gate.Model(gate.TOPK, gate.CPU_NK, a=lo[0], b=lo[1], c=1e-8, d=0.5, e=0.0, f=0.0, g=0.0, h=0.0,
                      margin_ms=margin, split_n=split, a_hi=hi[0], b_hi=hi[1])


def test_two_regimes_n_star_in_the_lower_regime():
    # root of a*K*N + b = 8e-8*N + 0.5 in the lower regime: N = (0.5 - b) / (a*K - 8e-8)
    m = _linear_two(1e6, (1e-6, 0.0), (1e-9, 0.3))
    k = 100
    root = 0.5 / (1e-6 * k - 8e-8)
    ns = gate.n_star(m, k, 8, out_fixed=k)
    assert ns == math.floor(root) + 1 and ns < 1e6
    assert gate.gain(m, ns, k, 8, 0.0, k) > 0.0 >= gate.gain(m, ns - 1, k, 8, 0.0, k)


def test_two_regimes_n_star_at_the_step():
    # the lower regime never pays; the upper one pays from its first size on
    m = _linear_two(1e6, (0.0, 0.0), (1e-6, 10.0))
    assert gate.n_star(m, 100, 8, out_fixed=100) == 1_000_000


def test_two_regimes_n_star_in_the_upper_regime():
    # neither the lower regime nor the step pays; the upper line crosses at
    # N = (0.5 - b_hi) / (a_hi*K - 8e-8)
    m = _linear_two(1000.5, (0.0, 0.0), (1e-9, -2.0))
    k = 1000
    root = (0.5 + 2.0) / (1e-9 * k - 8e-8)
    ns = gate.n_star(m, k, 8, out_fixed=k)
    assert ns == math.floor(root) + 1
    assert gate.gain(m, ns, k, 8, 0.0, k) > 0.0 >= gate.gain(m, ns - 1, k, 8, 0.0, k)
    assert gate.gain(m, 1000, k, 8, 0.0, k) <= 0.0 and gate.gain(m, 1001, k, 8, 0.0, k) <= 0.0
