"""Three-level envelope interpolation (Sec. III-A: field coefficients as
second-order Lagrange polynomials in time over [t_{n-1}, t_{n+1}]; Sec.
III-D: the simpler particle scheme samples them at the fine step).

CPU pins of the oracle's weights against what interpolation theory fixes,
and the library's host-side weight function against the oracle's."""
import numpy as np
import pytest

from oracle.oracle import envelope3, lagrange3_weights

TAU = (-3.0e-9, 7.0e-9, 17.0e-9)      # t_{n-1}, t_n, t_{n+1}: a field step of 10 ns


def test_weights_are_the_identity_at_the_level_times():
    for k, tk in enumerate(TAU):
        w = lagrange3_weights(TAU, tk)
        assert w == [1.0 if j == k else 0.0 for j in range(3)]


def test_weights_sum_to_one_and_reproduce_quadratics_exactly():
    rng = np.random.default_rng(3)
    for t in rng.uniform(TAU[0], TAU[2], 50):
        w = lagrange3_weights(TAU, t)
        assert abs(sum(w) - 1.0) <= 1e-15
        a, b, c = rng.standard_normal(3)
        f = lambda s: a + b * (s / 1e-8) + c * (s / 1e-8) ** 2
        interp = sum(wk * f(tk) for wk, tk in zip(w, TAU))
        assert abs(interp - f(t)) <= 1e-13 * (abs(a) + abs(b) + abs(c))


def test_weights_are_second_order_not_higher():
    # a cubic is not reproduced: the interpolation error is the classical
    # f'''/6 (t - t0)(t - t1)(t - t2) for f = s^3
    t = 1.0e-9
    w = lagrange3_weights(TAU, t)
    f = lambda s: (s / 1e-8) ** 3
    err = sum(wk * f(tk) for wk, tk in zip(w, TAU)) - f(t)
    expect = -np.prod([(t - tk) / 1e-8 for tk in TAU])
    assert abs(err - expect) <= 1e-12 * abs(expect) and abs(expect) > 0.1


def test_envelope3_is_the_weighted_sum_of_levels():
    rng = np.random.default_rng(4)
    lv = [rng.standard_normal(7) + 1j * rng.standard_normal(7) for _ in range(3)]
    w = lagrange3_weights(TAU, 2.0e-9)
    out = envelope3(lv, w)
    for i in range(7):
        assert out[i] == w[0] * lv[0][i] + w[1] * lv[1][i] + w[2] * lv[2][i]


def test_library_weights_match_the_oracle_on_the_host():
    from paper_2208_12795_gb300 import build, capi
    build.build()
    rng = np.random.default_rng(5)
    for t in np.r_[TAU, rng.uniform(TAU[0], TAU[2], 20)]:
        lw = capi.fempic_lagrange3(TAU, t)
        ow = lagrange3_weights(TAU, t)
        assert np.allclose(lw, ow, rtol=1e-15, atol=1e-16)
    with pytest.raises(capi.FempicError):
        capi.fempic_lagrange3((0.0, 1.0, 1.0), 0.5)


# ------------------------------------------- printed per-level carrier phase
def _fields(omega0, dtau, env, t):
    """The field Re{e^{j omega0 t} sum_k N_k(t) env(tau_k)} of the reading
    taken, the printed formula's Re{sum_k N_k(t) env(tau_k) e^{j omega0 tau_k}},
    and the field Re{env(t) e^{j omega0 t}} the levels sample."""
    from oracle.oracle import envelope3_literal
    tau = (-dtau, 0.0, dtau)
    lv = [np.array([env(tk)]) for tk in tau]
    w = lagrange3_weights(tau, t)
    carrier = np.exp(1j * omega0 * t)
    taken = (carrier * envelope3(lv, w))[0].real
    literal = (carrier * envelope3_literal(lv, w, tau, omega0, t))[0].real
    return taken, literal, (env(t) * carrier).real


def test_literal_phase_agrees_when_the_field_step_resolves_the_carrier():
    """With a field step much shorter than a carrier period the per-level
    carrier is itself interpolated to third order: the printed formula and
    the reading taken differ by O((omega0 dtau)^3), falling 8x per halving,
    and agree exactly at the level times."""
    omega0 = 2 * np.pi * 1e9
    env = lambda s: (1.0 + 0.3j) + (0.2 - 0.1j) * s / 1e-6     # a slow envelope (quadratic is exact)
    diffs = []
    for dtau in (2e-12, 1e-12, 5e-13):
        ts = np.linspace(-dtau, dtau, 41)
        d = max(abs(_fields(omega0, dtau, env, t)[0] - _fields(omega0, dtau, env, t)[1]) for t in ts)
        diffs.append(d)
        assert d <= 2 * (omega0 * dtau) ** 3
        for tk in (-dtau, 0.0, dtau):
            a, b, _ = _fields(omega0, dtau, env, tk)
            assert abs(a - b) <= 1e-15
    assert 6.0 < diffs[0] / diffs[1] < 10.0 and 6.0 < diffs[1] / diffs[2] < 10.0


def test_literal_phase_aliases_when_a_field_step_spans_the_carrier():
    """With a field step of half a carrier period (the regime the method is
    for: many fine steps, and carrier periods, per field step) the samples
    e^{j omega0 tau_k} alternate in sign and their quadratic interpolant is
    not the carrier: the printed formula's field misses the sampled field by
    O(1), while the reading taken reproduces it exactly (the envelope is
    linear in t)."""
    omega0 = 2 * np.pi * 1e9
    dtau = np.pi / omega0
    env = lambda s: (1.0 + 0.3j) + (0.2 - 0.1j) * s / 1e-6
    worst_taken, worst_literal = 0.0, 0.0
    for t in np.linspace(-dtau, dtau, 81):
        taken, literal, true = _fields(omega0, dtau, env, t)
        worst_taken = max(worst_taken, abs(taken - true))
        worst_literal = max(worst_literal, abs(literal - true))
    assert worst_taken <= 1e-12 and worst_literal > 0.5
