"""Pins of the downshifted integrator's oracle (Sec. III-D: velocity rule with
the carrier integrated analytically through the M and L weights, AB4
positions) against what the mathematics fixes, independent of its formulas:
symbolic integrals, Adams-Bashforth coefficients, closed-form trajectories,
the closed-form gyration, a high-accuracy ODE solution, the mesh-free form of
the same rule, and the deposit's charge identity.  Also the library's host
weight function against the oracle's."""
import math

import numpy as np
import pytest

from oracle.downshift import (AB4, History, boris_uniform, integrate_uniform, ml_weights, push_step_downshift,
                              uniform_step)
from oracle.oracle import OracleMesh, OracleState
from paper_2208_12795_gb300 import inputs as I


def _ab3(lag):
    # int_0^1 of the Lagrange basis on the nodes -lag, -lag-1, -lag-2
    return np.array([23.0, -16.0, 5.0]) / 12.0 if lag == 0 else np.array([53.0, -64.0, 23.0]) / 12.0


@pytest.mark.parametrize("lag", [0, 1])
def test_weights_reduce_to_adams_bashforth_without_carrier(lag):
    dt = 0.5e-9
    Mr, Mi, Lr, Li = ml_weights(3.0e-9, dt, 0.0, lag)
    np.testing.assert_allclose(Mr, dt * _ab3(lag), rtol=1e-14)
    assert np.all(Mi == 0) and np.all(Li == 0)
    np.testing.assert_allclose(Lr, Lr.T, rtol=1e-14)
    np.testing.assert_allclose(Lr.sum(1), Mr, rtol=1e-13)


@pytest.mark.parametrize("theta,phi,lag", [(0.3, 0.4, 0), (2.0, -1.1, 0), (7.0, 2.5, 0), (1.5, 0.9, 1)])
def test_weights_match_symbolic_integrals(theta, phi, lag):
    sp = pytest.importorskip("sympy")
    x = sp.Symbol("x")
    nodes = [-(k + lag) for k in range(3)]
    N = []
    for k in range(3):
        e = sp.Integer(1)
        for j in range(3):
            if j != k:
                e *= (x - nodes[j]) / sp.Integer(nodes[k] - nodes[j])
        N.append(sp.expand(e))
    th, ph = sp.Rational(theta).limit_denominator(1000), sp.Rational(phi).limit_denominator(1000)
    dt = 1.0
    Mr, Mi, Lr, Li = ml_weights(float(ph / th), dt, float(th), lag)
    for k in range(3):
        mr = sp.integrate(N[k] * sp.cos(th * x + ph), (x, 0, 1))
        mi = -sp.integrate(N[k] * sp.sin(th * x + ph), (x, 0, 1))
        assert abs(Mr[k] - float(sp.N(mr, 30))) < 3e-14 and abs(Mi[k] - float(sp.N(mi, 30))) < 3e-14
        for j in range(3):
            lr = sp.integrate(N[j] * N[k] * sp.cos(th * x + ph), (x, 0, 1))
            li = -sp.integrate(N[j] * N[k] * sp.sin(th * x + ph), (x, 0, 1))
            # the basis products reach 9 on [0, 1]: quadrature rounding ~1e-14
            assert abs(Lr[j, k] - float(sp.N(lr, 30))) < 1e-13 and abs(Li[j, k] - float(sp.N(li, 30))) < 1e-13


def test_weights_sum_to_the_carrier_integral():
    rng = np.random.default_rng(11)
    for _ in range(20):
        dt = 0.5e-9
        om = rng.uniform(-3.0, 3.0) / dt
        t = rng.uniform(0.0, 50e-9)
        Mr, Mi, Lr, Li = ml_weights(t, dt, om)
        a, b = om * t, om * (t + dt)
        assert abs(Mr.sum() - (math.sin(b) - math.sin(a)) / om) < 1e-12 * dt
        assert abs(Mi.sum() - (math.cos(b) - math.cos(a)) / om) < 1e-12 * dt
        np.testing.assert_allclose(Lr.sum(1), Mr, atol=1e-13 * dt)
        np.testing.assert_allclose(Li.sum(0), Mi, atol=1e-13 * dt)


def test_library_weights_match_the_oracle_on_the_host():
    from paper_2208_12795_gb300 import build, capi
    build.build()
    rng = np.random.default_rng(12)
    dt = 0.5e-9
    for theta in [0.0, 1e-7, 0.3, 1.0, 1.0000001, 2.5, 6.0, -0.8]:
        t = rng.uniform(0.0, 1e-7)
        got = capi.fempic_downshift_weights(t, dt, theta / dt)
        want = ml_weights(t, dt, theta / dt)
        for g, w in zip(got, want):
            np.testing.assert_allclose(np.array(g), np.asarray(w), rtol=0, atol=1e-13 * dt)
    with pytest.raises(capi.FempicError):
        capi.fempic_downshift_weights(0.0, 0.0, 1.0)


@pytest.mark.parametrize("lag", [0, 1])
def test_exact_for_a_cubic_velocity(lag):
    """omega0 = 0, B = 0, E quadratic in time: the quadratic interpolation of
    the samples is exact, so v is exact (cubic) and AB4 is exact for cubic v;
    with the exact history the whole trajectory is the closed form."""
    qm = -1.7e11
    a0, a1, a2 = np.array([3.0, -1.0, 2.0]), np.array([1e9, 2e8, -5e8]), np.array([4e17, -1e17, 3e17])
    r0, v0 = np.array([0.1, 0.2, 0.3]), np.array([1e5, -2e5, 3e4])
    E = lambda t: a0 + a1 * t + a2 * t * t
    v = lambda t: v0 + qm * (a0 * t + a1 * t ** 2 / 2 + a2 * t ** 3 / 3)
    r = lambda t: r0 + v0 * t + qm * (a0 * t ** 2 / 2 + a1 * t ** 3 / 6 + a2 * t ** 4 / 12)
    dt = 0.5e-9
    zero = np.zeros(3, complex)
    hv = [v(-k * dt) for k in (1, 2, 3)]
    he = [E(-k * dt).astype(complex) for k in range(1, 3 + lag)]
    hb = [zero for _ in range(2 + lag)]
    rr, vv = r(0.0), v(0.0)
    for n in range(12):
        t = n * dt
        rr, vv, hv, he, hb = uniform_step(qm, rr, vv, hv, he, hb, E(t).astype(complex), zero, t, dt, 0.0, lag)
        np.testing.assert_allclose(vv, v(t + dt), rtol=1e-13, atol=1e-13 * np.abs(v(t + dt)).max())
        np.testing.assert_allclose(rr, r(t + dt), rtol=1e-13, atol=1e-13)


def test_velocity_rule_integrates_the_carrier_exactly():
    """omega0 != 0, B = 0, complex envelope quadratic in time: one step's
    velocity increment is qm int Re{E~(t) e^{j w0 t}} dt exactly (the sign of
    the M^i term included)."""
    from scipy.integrate import quad
    qm = 2.3e7
    dt = 0.5e-9
    om = 2 * math.pi * 0.9e9
    c0 = np.array([1 + 2j, -0.5 + 1j, 3 - 1j])
    c1 = np.array([0.2 - 0.1j, 1j, -0.4]) / dt
    c2 = np.array([0.05j, -0.02, 0.03 + 0.01j]) / dt ** 2
    env = lambda t: c0 + c1 * t + c2 * t * t
    t_n = 7 * dt
    zero = np.zeros(3, complex)
    v_n = np.zeros(3)                # B = 0: the velocity does not enter, and the increment is exact
    hv = [v_n, v_n, v_n]
    _, v1, *_ = uniform_step(qm, np.zeros(3), v_n, hv, [env(t_n - dt), env(t_n - 2 * dt)], [zero, zero],
                             env(t_n), zero, t_n, dt, om)
    for a in range(3):
        f = lambda t: (env(t)[a] * complex(math.cos(om * t), math.sin(om * t))).real
        want = qm * quad(f, t_n, t_n + dt, epsabs=0, epsrel=1e-13)[0]
        assert abs((v1[a] - v_n[a]) - want) <= 1e-11 * abs(want)


def test_gyration_is_third_order_and_turns_the_right_way():
    """omega0 = 0, E = 0, static B along z: the rule is three-step Adams-Bashforth
    on dv/dt = qm v x B; against the closed-form gyration the velocity error
    is the AB3 truncation error and drops by 2^3 per halving of dt.  A wrong
    sign of the cross product fails by O(1)."""
    qm, B0 = -1.758820e11, 1e-3
    wc = qm * B0                                 # signed: v rotates by -wc t about +z
    v0 = np.array([1e6, 0.0, 2e3])
    vex = lambda t: np.array([v0[0] * math.cos(wc * t) + v0[1] * math.sin(wc * t),
                              -v0[0] * math.sin(wc * t) + v0[1] * math.cos(wc * t), v0[2]])
    T = 2 * math.pi / abs(wc)
    errs = []
    for nstep in (64, 128, 256):
        dt = T / nstep
        zero = np.zeros(3, complex)
        bz = np.array([0, 0, B0], complex)
        hv = [vex(-k * dt) for k in (1, 2, 3)]
        he, hb = [zero, zero], [bz, bz]
        rr, vv = np.zeros(3), vex(0.0)
        for n in range(nstep):
            rr, vv, hv, he, hb = uniform_step(qm, rr, vv, hv, he, hb, zero, bz, n * dt, dt, 0.0)
        errs.append(np.linalg.norm(vv - vex(T)) / np.linalg.norm(v0))
    # leading error of AB3 (error constant 3/8) over one turn: (3/8) (2 pi / N)^3 2 pi
    est = 3.0 / 8.0 * (2 * math.pi / 64) ** 3 * 2 * math.pi
    assert abs(errs[0] / est - 1.0) < 0.05
    for a, b in zip(errs, errs[1:]):
        assert 6.5 < a / b < 9.5


def test_trend_of_table_I_fewer_steps_than_the_fine_step_scheme():
    """Sec. IV-B (Table I trend): one particle in E = x v(t), B = z v(t),
    v(t) = cos(w0 t) exp(-(t - 6s)^2 / 2s^2), s = 2 / w_bw, f0 = 2 GHz,
    f_bw = 20 MHz, q/m = 1 (reading: the example gives no particle).  Against
    a high-accuracy ODE solution, the downshifted scheme's position error
    falls at fourth order (AB4 positions), the fine-step Boris scheme's at
    second, and the downshifted scheme at half the steps is already the more
    accurate one."""
    from scipy.integrate import solve_ivp
    f0, fbw, qm = 2e9, 20e6, 1.0
    om = 2 * math.pi * f0
    sig = 2.0 / (2 * math.pi * fbw)
    g = lambda t: math.exp(-(t - 6 * sig) ** 2 / (2 * sig ** 2))
    env = lambda t: (np.array([g(t), 0, 0], complex), np.array([0, 0, g(t)], complex))
    ef = lambda t: np.array([math.cos(om * t) * g(t), 0.0, 0.0])
    bf = lambda t: np.array([0.0, 0.0, math.cos(om * t) * g(t)])

    def rhs(t, y):
        v = y[3:]
        return np.r_[v, qm * (ef(t) + np.cross(v, bf(t)))]

    n64 = 2 * int(round(12 * sig * f0 * 32))
    tg = np.arange(n64 + 1) / (f0 * 64)
    ref64 = solve_ivp(rhs, (0, tg[-1]), np.zeros(6), method="DOP853", rtol=1e-12, atol=1e-30, t_eval=tg).y[:3].T
    errs = {}
    for per in (32, 64):
        dt = 1.0 / (f0 * per)
        n = n64 * per // 64
        ref = ref64[::64 // per]
        l2 = lambda rs: math.sqrt(np.sum((rs - ref) ** 2) / np.sum(ref ** 2))
        errs[per] = (l2(integrate_uniform(qm, np.zeros(3), np.zeros(3), env, dt, n, om)[0]),
                     l2(boris_uniform(qm, np.zeros(3), np.zeros(3), ef, bf, dt, n)))
    ds32, bo32 = errs[32]
    ds64, bo64 = errs[64]
    assert 12.0 < ds32 / ds64 < 20.0          # fourth order
    assert 3.5 < bo32 / bo64 < 4.5            # second order
    assert ds32 < bo64                        # half the steps, smaller error


def _uniform_dofs(m, om, E, B):
    tb = om.tables()
    en, fn = tb["edge_nodes"], tb["face_nodes"]
    e = ((m.nodes[en[:, 1]] - m.nodes[en[:, 0]]) @ np.asarray(E)).astype(complex)
    nA = 0.5 * np.cross(m.nodes[fn[:, 1]] - m.nodes[fn[:, 0]], m.nodes[fn[:, 2]] - m.nodes[fn[:, 0]])
    b = (nA @ np.asarray(B)).astype(complex)
    return e, b


def _single(x, v, q=-I.E_CHARGE, mass=I.M_ELECTRON, w=1e3):
    return I.Particles(np.array([x[0]]), np.array([x[1]]), np.array([x[2]]),
                       np.array([v[0]]), np.array([v[1]]), np.array([v[2]]),
                       np.array([0, 1], np.int64), np.array([q]), np.array([mass]), np.array([w]))


@pytest.fixture(scope="module")
def cube4j():
    m = I.kuhn_cube_mesh(4, jitter=0.2, rng=np.random.default_rng(7))
    return m, OracleMesh(m.nodes, m.tets)


def test_mesh_step_equals_the_mesh_free_rule_in_uniform_fields(cube4j):
    """Whitney DoFs of uniform complex fields reproduce them exactly, so a
    particle inside the box follows the mesh-free rule with the same samples,
    whatever tets it crosses; the slow amplitude a(t) scales every sample."""
    m, om = cube4j
    E = np.array([2e3, -1e3, 5e2]); B = np.array([1e-4, 3e-4, -2e-4])
    e_re, b_re = _uniform_dofs(m, om, E, B)
    e_dof, b_dof = e_re * (1 - 0.5j), b_re * (0.3 + 1j)
    env_c = (E * (1 - 0.5j), B * (0.3 + 1j))
    P = _single([0.41, 0.52, 0.47], [3e7, -2e7, 1.5e7])
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    hist = History(1)
    dt, omega0 = 0.5e-9, 2 * math.pi * 1.3e9
    amp = lambda t: 0.5 + 1e7 * t
    G = np.zeros(om.n_edges)
    qm = P.q[0] / P.m[0]
    rs, v = integrate_uniform(qm, [0.41, 0.52, 0.47], [3e7, -2e7, 1.5e7],
                              lambda t: (amp(t) * env_c[0], amp(t) * env_c[1]), dt, 30, omega0)
    for n in range(30):
        push_step_downshift(om, st, hist, e_dof, b_dof, amp(n * dt), omega0, n * dt, dt, G)
        np.testing.assert_allclose([st.x[0], st.y[0], st.z[0]], rs[n + 1], rtol=1e-12, atol=1e-14)
    assert st.n_cross[0] > 3 and st.tet[0] >= 0
    np.testing.assert_allclose([st.vx[0], st.vy[0], st.vz[0]], v, rtol=1e-11)


def test_mesh_step_conserves_charge_and_mirrors_the_history(cube4j):
    """Many particles, random fields, reflecting walls: D^T G = rho^K - rho^0 to
    rounding; a field-free particle heading into the wall at x = 1 comes back
    on the mirror image of its free path, which needs the velocity history
    mirrored too (without it the AB4 velocity after the bounce is -86/24 v)."""
    m, om = cube4j
    rng = np.random.default_rng(13)
    tb = om.tables()
    e_dof, b_dof = I.random_windowed_dofs(m.nodes, tb["edge_nodes"], tb["face_nodes"], rng, e_scale=1e3,
                                          b_scale=1e-4)
    P = I.uniform_maxwellian(300, 50.0, rng)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    hist = History(st.n)
    rho0 = om.nodal_charge(st.x, st.y, st.z, st.tet, P.species_begin, P.q, P.w)
    G = np.zeros(om.n_edges)
    dt, omega0 = 2e-9, 2 * math.pi * 0.4e9
    for n in range(25):
        push_step_downshift(om, st, hist, e_dof, b_dof, 1.0, omega0, n * dt, dt, G)
    assert st.n_cross.sum() > 50
    rho1 = om.nodal_charge(st.x, st.y, st.z, st.tet, P.species_begin, P.q, P.w)
    scale = abs(P.q[0] * P.w[0])
    np.testing.assert_allclose(om.edge_divergence(G), rho1 - rho0, atol=1e-12 * scale)
    # the mirror: field-free, constant velocity toward x = 1
    zero_e, zero_b = np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex)
    x0, v0 = np.array([0.93, 0.4, 0.6]), np.array([2e7, 1e6, -3e6])
    Q = _single(x0, v0)
    tq, _ = om.locate(Q.x, Q.y, Q.z)
    sq = OracleState(Q, tq)
    hq = History(1)
    for n in range(8):
        push_step_downshift(om, sq, hq, zero_e, zero_b, 1.0, 0.0, n * dt, dt, np.zeros(om.n_edges))
        free = x0 + (n + 1) * dt * v0
        want = free.copy()
        if free[0] > 1.0:
            want[0] = 2.0 - free[0]
        np.testing.assert_allclose([sq.x[0], sq.y[0], sq.z[0]], want, rtol=1e-13, atol=1e-15)
    assert sq.vx[0] == -v0[0] and np.all(hq.v[:, 0, 0] == -v0[0])
    assert AB4.sum() == pytest.approx(1.0, abs=1e-15)


def test_walk_records_its_wall_mirrors():
    """The oracle's walk records, where it reflects, which velocity
    components it mirrored an odd number of times (the downshifted rule
    mirrors its history with that record, D6): a corner hit mirrors two
    axes, a step long enough to bounce off both x walls mirrors none, and
    on a hot load the record equals what the velocity signs show."""
    from oracle.oracle import OracleMesh, OracleState, push_step
    from paper_2208_12795_gb300 import inputs as I
    m = I.kuhn_cube_mesh(4)
    om = OracleMesh(m.nodes, m.tets)
    dt = 1e-9
    x = np.array([0.9, 0.9, 0.5, 0.3])
    y = np.array([0.9, 0.5, 0.5, 0.3])
    z = np.array([0.5, 0.5, 0.5, 0.3])
    vx = np.array([0.3, 1.5, 0.0, 0.2]) / dt      # corner; two x walls; at rest in x; no wall
    vy = np.array([0.3, 0.0, 0.0, 0.1]) / dt
    vz = np.zeros(4)
    P = I.Particles(x, y, z, vx, vy, vz, np.array([0, 4], np.int64), np.array([-I.E_CHARGE]),
                    np.array([I.M_ELECTRON]), np.array([1.0]))
    tet, _ = om.locate(x, y, z)
    st = OracleState(P, tet)
    mirror = np.full(4, 255, np.uint8)
    e0 = np.zeros(om.n_edges, np.complex128)
    b0 = np.zeros(om.n_faces, np.complex128)
    push_step(om, st, e0, b0, 0.0, 1.0, 0.0, dt, np.zeros(om.n_edges), mirror=mirror)
    assert list(mirror) == [0b011, 0b000, 0b000, 0b000]
    assert st.vx[0] < 0 and st.vy[0] < 0 and st.vx[1] == vx[1]             # two x mirrors cancel
    assert abs(st.x[1] - 0.4) < 1e-12 and abs(st.x[0] - 0.8) < 1e-12 and abs(st.y[0] - 0.8) < 1e-12
    wl = I.workload_hot_small(jitter=0.2)
    om2 = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    st = OracleState(wl.particles, om2.locate(wl.particles.x, wl.particles.y, wl.particles.z)[0])
    v0 = np.stack([st.vx, st.vy, st.vz], 1).copy()
    mirror = np.zeros(st.n, np.uint8)
    push_step(om2, st, np.zeros(om2.n_edges, np.complex128), np.zeros(om2.n_faces, np.complex128), 0.0, 1.0,
              0.0, wl.dt, np.zeros(om2.n_edges), mirror=mirror)
    v1 = np.stack([st.vx, st.vy, st.vz], 1)
    bits = ((mirror[:, None] >> np.arange(3)[None, :]) & 1).astype(bool)
    assert bits.any() and np.array_equal(bits, (v0 != 0) & (v1 == -v0))
