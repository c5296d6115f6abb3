"""Pin of the oracle's forward-mode tangent (JVP) against central finite
differences of the oracle itself, for the total kinetic energy after K steps
as a function of the envelope DoFs and the initial phase space.  The tet
sequence is the same for the +h and -h runs (checked), so the loss is smooth
there and central differences are accurate to O(h^2)."""
import numpy as np
import pytest

from oracle.oracle import (OracleMesh, OracleState, kinetic_energy, kinetic_energy_jvp, push_step,
                           push_step_jvp)
from paper_2208_12795_gb300 import inputs as I


def _run(om, wl, P, tet, e, b, K, jvp=None):
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    if jvp is not None:
        tr, tv, de, db = (x.copy() for x in jvp)
    for n in range(K):
        t = n * wl.dt
        if jvp is None:
            push_step(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, wall_mode=wl.wall_mode)
        else:
            push_step_jvp(om, st, e, b, wl.amp(t), wl.omega0, t, wl.dt, G, tr, tv, de, db,
                          wall_mode=wl.wall_mode)
    return st, (kinetic_energy_jvp(st, tv) if jvp is not None else None)


@pytest.mark.parametrize("maker,K", [(I.workload_small, 20), (lambda: I.workload_hot_small(n_particles=60), 6)])
def test_jvp_matches_central_differences(maker, K):
    wl = maker()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles.subset(min(wl.particles.n, 300))
    tet, _ = om.locate(P.x, P.y, P.z)
    rng = np.random.default_rng(31)
    n = P.n
    sv = np.std(np.r_[P.vx, P.vy, P.vz])
    for trial in range(3):
        de = (rng.standard_normal(om.n_edges) + 1j * rng.standard_normal(om.n_edges)) * np.abs(wl.e_tilde).max()
        db = (rng.standard_normal(om.n_faces) + 1j * rng.standard_normal(om.n_faces)) * np.abs(wl.b_tilde).max()
        tv = rng.standard_normal((n, 3)) * sv
        tr = rng.standard_normal((n, 3)) * 1e-3 * wl.mesh.h
        base, jv = _run(om, wl, P, tet, wl.e_tilde, wl.b_tilde, K, jvp=(tr, tv, de, db))
        h = 1e-6
        outs = []
        for sgn in (1, -1):
            Pp = I.Particles(P.x + sgn * h * tr[:, 0], P.y + sgn * h * tr[:, 1], P.z + sgn * h * tr[:, 2],
                             P.vx + sgn * h * tv[:, 0], P.vy + sgn * h * tv[:, 1], P.vz + sgn * h * tv[:, 2],
                             P.species_begin, P.q, P.m, P.w)
            st, _ = _run(om, wl, Pp, tet, wl.e_tilde + sgn * h * de, wl.b_tilde + sgn * h * db, K)
            assert np.array_equal(st.tet, base.tet) and np.array_equal(st.n_cross, base.n_cross)
            outs.append(kinetic_energy(st))
        fd = (outs[0] - outs[1]) / (2 * h)
        assert abs(fd - jv) <= 1e-6 * abs(jv), (fd, jv)
