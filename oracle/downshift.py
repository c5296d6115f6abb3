"""Downshifted particle integrator of Sec. III-D (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline): the product
path never imports this module.

Sec. III-D integrates the Lorentz force with the fast carrier treated
analytically: over one particle step [t_n, t_{n+1}] the slowly varying
envelope samples are interpolated in time by the quadratic Lagrange basis
N_{n,k}, and the carrier enters only through the exact integrals

    M^r_{n,k}   =  int N_k cos(w0 t) dt      M^i_{n,k}   = -int N_k sin(w0 t) dt
    L^r_{n,j,k} =  int N_j N_k cos(w0 t) dt  L^i_{n,j,k} = -int N_j N_k sin(w0 t) dt

Positions advance with the fourth-order Adams-Bashforth stencil
(55, -59, 37, -9) / 24 on the velocities of the last four steps.

Readings taken where the printed rule is garbled (the velocity equation's
level indices, and a two-index L used with one index):

* D1  The three samples are the newest ones, levels n, n-1, n-2 (nodes
      tau_k = t_{n-k}).  The printed indices n-1-k would skip the sample at
      the newest known position; ``lag=1`` selects that literal variant.
* D2  "E (M^r + M^i)" is Re(E~) M^r + Im(E~) M^i: that is exactly
      int N Re{E~ e^{j w0 t}} dt.
* D3  The magnetic term interpolates the velocity (basis N_j) and the
      envelope B~ (basis N_k) separately, which is what a two-index L_{j,k}
      integrates: sum_j sum_k v_j x (Re(B~_k) L^r_jk + Im(B~_k) L^i_jk).
* D4  Field samples are the envelope at the particle's own position at each
      level, times the slow amplitude a(t) of that level.
* D5  Start-up: the history is filled with the first step's own values
      (constant extrapolation backwards).
* D6  Tracking, walls and the deposit act on the straight AB4 segment
      r^n -> r^n + dt u, u = (55 v^n - 59 v^{n-1} + 37 v^{n-2} - 9 v^{n-3}) / 24.
      A specular wall mirrors, in that axis, the new velocity and every
      stored velocity of the history; field samples are not mirrored.

Parity status: the weights are pinned to symbolic integrals and to
Adams-Bashforth coefficients (w0 = 0); the step to closed-form polynomial
trajectories (exact for cubic velocities), to the closed-form gyration
(third order in dt) and to a high-accuracy ODE solution (fourth order in
the positions).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss

from .oracle import OracleMesh, OracleState, lagrange3_weights, push_step

_XG, _WG = leggauss(40)


def nodes(dt, lag=0):
    """Node times of the basis relative to t_n: tau_k = -(k + lag) dt (D1)."""
    return [-(k + lag) * dt for k in range(3)]


def ml_weights(t_n, dt, omega0, lag=0):
    """M^r, M^i (3,) and L^r, L^i (3, 3) over [t_n, t_n + dt] (Sec. III-D).

    Gauss-Legendre quadrature in s = t - t_n; 40 nodes integrate the quartic
    basis products times the carrier to rounding for |w0 dt| up to ~10.
    """
    tau = nodes(dt, lag)
    s = 0.5 * dt * (_XG + 1.0)
    w = 0.5 * dt * _WG
    N = np.array([lagrange3_weights(tau, si) for si in s])          # [q, 3]
    c = np.cos(omega0 * (t_n + s))
    sn = np.sin(omega0 * (t_n + s))
    Mr = (w * c) @ N
    Mi = -((w * sn) @ N)
    Lr = np.einsum("q,qj,qk->jk", w * c, N, N)
    Li = -np.einsum("q,qj,qk->jk", w * sn, N, N)
    return Mr, Mi, Lr, Li


AB4 = np.array([55.0, -59.0, 37.0, -9.0]) / 24.0


def _cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def velocity_increment(qm, vs, es, bs, W):
    """dv of the downshifted rule (D2, D3).

    vs: velocities at the three sample levels [3][3]; es, bs: complex
    envelope samples [3][3]; W = ml_weights(...)."""
    Mr, Mi, Lr, Li = W
    dv = np.zeros(3)
    for k in range(3):
        dv += qm * (es[k].real * Mr[k] + es[k].imag * Mi[k])
        for j in range(3):
            dv += qm * _cross(vs[j], bs[k].real * Lr[j, k] + bs[k].imag * Li[j, k])
    return dv


def ab4_velocity(vh4):
    """u = sum_i AB4_i v^{n-i} (the displacement is dt u)."""
    return AB4[0] * vh4[0] + AB4[1] * vh4[1] + AB4[2] * vh4[2] + AB4[3] * vh4[3]


class History:
    """Per-particle history: velocities v^{n-1..n-3} and the complex envelope
    samples of the levels before n (two for lag 0, three for lag 1)."""

    def __init__(self, n, lag=0):
        self.lag = lag
        self.v = np.zeros((3, n, 3))                        # v^{n-1}, v^{n-2}, v^{n-3}
        self.e = np.zeros((2 + lag, n, 3), np.complex128)   # E~ at levels n-1, n-2 (, n-3)
        self.b = np.zeros((2 + lag, n, 3), np.complex128)
        self.started = False


def uniform_step(qm, r, v, hist_v, hist_e, hist_b, e_n, b_n, t_n, dt, omega0, lag=0):
    """One step of a particle in spatially uniform fields (no mesh, no walls).

    Returns (r^{n+1}, v^{n+1}, new histories)."""
    es = [e_n] + list(hist_e)
    bs = [b_n] + list(hist_b)
    vv = [v] + list(hist_v)
    W = ml_weights(t_n, dt, omega0, lag)
    dv = velocity_increment(qm, vv[lag:lag + 3], es[lag:lag + 3], bs[lag:lag + 3], W)
    u = ab4_velocity(vv)
    r1 = r + dt * u
    return r1, v + dv, vv[:3], es[:len(hist_e)], bs[:len(hist_b)]


def integrate_uniform(qm, r0, v0, env, dt, nsteps, omega0, lag=0):
    """Positions r^0..r^nsteps of one particle in E = Re{E~(t) e^{j w0 t}},
    B = Re{B~(t) e^{j w0 t}} with env(t) = (E~(t), B~(t)) uniform in space."""
    r = np.asarray(r0, float).copy()
    v = np.asarray(v0, float).copy()
    e0, b0 = env(0.0)
    hv = [v.copy() for _ in range(3)]
    he = [np.asarray(e0, complex) for _ in range(2 + lag)]
    hb = [np.asarray(b0, complex) for _ in range(2 + lag)]
    out = [r.copy()]
    for n in range(nsteps):
        t_n = n * dt
        e_n, b_n = env(t_n)
        r, v, hv, he, hb = uniform_step(qm, r, v, hv, he, hb, np.asarray(e_n, complex),
                                        np.asarray(b_n, complex), t_n, dt, omega0, lag)
        out.append(r.copy())
    return np.array(out), v


def boris_uniform(qm, r0, v0, efield, bfield, dt, nsteps):
    """The fine-step scheme the paper compares against: fields sampled at t_n,
    Boris leapfrog (v0 taken as v^{-1/2}).  Positions r^0..r^nsteps."""
    r = np.asarray(r0, float).copy()
    v = np.asarray(v0, float).copy()
    k = 0.5 * qm * dt
    out = [r.copy()]
    for n in range(nsteps):
        t = n * dt
        E = np.asarray(efield(t), float)
        B = np.asarray(bfield(t), float)
        vm = v + k * E
        tt = k * B
        s = 2.0 * tt / (1.0 + tt @ tt)
        vp = vm + _cross(vm, tt)
        v = vm + _cross(vp, s) + k * E
        r = r + dt * v
        out.append(r.copy())
    return np.array(out)


def push_step_downshift(mesh: OracleMesh, st: OracleState, hist: History, e_dof, b_dof, amp, omega0, t, dt,
                        dG, max_crossings=4096, wall_mode=0):
    """One downshifted step of every particle on the mesh (D1-D6).

    The envelope samples are the Whitney sums of the DoFs at each particle's
    position times amp = a(t_n); the AB4 segment is then tracked, reflected
    or absorbed and deposited by the oracle's own step with a zero field
    (its Boris update then leaves the velocity unchanged)."""
    n = st.n
    lag = hist.lag
    qm_p = np.zeros(n)
    for s in range(len(st.q)):
        qm_p[st.species_begin[s]:st.species_begin[s + 1]] = st.q[s] / st.m[s]
    active = st.tet >= 0
    v_n = np.stack([st.vx, st.vy, st.vz], 1)
    e_n = np.zeros((n, 3), np.complex128)
    b_n = np.zeros((n, 3), np.complex128)
    for p in np.nonzero(active)[0]:
        E, B = mesh.gather(int(st.tet[p]), np.array([st.x[p], st.y[p], st.z[p]]), e_dof, b_dof)
        e_n[p] = amp * E
        b_n[p] = amp * B
    if not hist.started:                      # D5 (particles already frozen keep no history)
        hist.v[:, active] = v_n[active]
        hist.e[:, active] = e_n[active]
        hist.b[:, active] = b_n[active]
        hist.started = True
    W = ml_weights(t, dt, omega0, lag)
    v_next = v_n.copy()
    u = v_n.copy()
    for p in np.nonzero(active)[0]:
        vv = [v_n[p], hist.v[0, p], hist.v[1, p], hist.v[2, p]]
        es = [e_n[p]] + [hist.e[i, p] for i in range(hist.e.shape[0])]
        bs = [b_n[p]] + [hist.b[i, p] for i in range(hist.b.shape[0])]
        v_next[p] = v_n[p] + velocity_increment(qm_p[p], vv[lag:lag + 3], es[lag:lag + 3], bs[lag:lag + 3], W)
        u[p] = ab4_velocity(vv)
    # track the AB4 segment with the oracle's own step under a zero field
    st.vx[:] = u[:, 0]
    st.vy[:] = u[:, 1]
    st.vz[:] = u[:, 2]
    zero_e = np.zeros(mesh.n_edges, np.complex128)
    zero_b = np.zeros(mesh.n_faces, np.complex128)
    mirror = np.zeros(n, np.uint8)
    push_step(mesh, st, zero_e, zero_b, 0.0, omega0, t, dt, dG, max_crossings=max_crossings,
              wall_mode=wall_mode, mirror=mirror)
    # D6: the axes the walk mirrored an odd number of times, as recorded by
    # the walk itself where it reflects
    flip = ((mirror[:, None] >> np.arange(3)[None, :]) & 1).astype(bool)
    sign = np.where(flip, -1.0, 1.0)
    # history shift (active particles only), then the mirror of every velocity
    new_hv = hist.v.copy()
    new_hv[2, active] = hist.v[1, active]
    new_hv[1, active] = hist.v[0, active]
    new_hv[0, active] = v_n[active]
    hist.v[:] = new_hv * sign[None]
    for arr, cur in ((hist.e, e_n), (hist.b, b_n)):
        for i in range(arr.shape[0] - 1, 0, -1):
            arr[i, active] = arr[i - 1, active]
        arr[0, active] = cur[active]
    vf = v_next * sign
    st.vx[:] = vf[:, 0]
    st.vy[:] = vf[:, 1]
    st.vz[:] = vf[:, 2]
