"""Invariants of the face walk (all three forms) that hold whatever the
rounding: a particle frozen by the crossing cap stops on a face of the tet
it was in, an absorbed particle stops on the boundary of the domain, the
particles that keep moving end inside their tet, and charge is conserved
through all of it (to 1e-13).  Checked through the C ABI on the device, with
the barycentrics recomputed in FP64 on the host.  Tolerances in barycentric
units, per form: the FP64 form and the contract mixed form place crossing
points from FP64-accurate exit parameters; the 24-bit form from 24-bit
integer barycentrics and an FP32 path parameter (about 1e-7 of a step), and
decides "inside" on those integers."""
import numpy as np
import pytest

from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED, Q24 = 0, 1, 2
CAP, ABSORBED = 1, 2
LAM_TOL = {FP64: 1e-12, MIXED: 1e-11, Q24: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _bary(nodes, tet_nodes, T, r):
    X = nodes[tet_nodes[T]]                       # [n, 4, 3]
    A = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)
    l123 = np.linalg.solve(A, (r - X[:, 0])[..., None])[..., 0]
    return np.concatenate([1.0 - l123.sum(1, keepdims=True), l123], axis=1)


def _run(wl, steps, prec, **kw):
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    env = FempicEnv.from_mesh(wl.mesh, precision=prec, wall_mode=wl.wall_mode, **kw)
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    rho0 = env.nodal_charge(st).cpu().numpy()
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    for n in range(steps):
        t = n * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
    rho1 = env.nodal_charge(st).cpu().numpy()
    torch.cuda.synchronize()
    q = env.query()
    div = np.zeros(env.n_nodes)
    np.add.at(div, q["edge_nodes"][:, 1], G.cpu().numpy())
    np.subtract.at(div, q["edge_nodes"][:, 0], G.cpu().numpy())
    res = np.abs(div - (rho1 - rho0)).max() / np.abs(rho1).max()
    return st.to_numpy(), q["tet_nodes"], res


def _positions(g, idx):
    return np.stack([g["x"][idx], g["y"][idx], g["z"][idx]], 1)


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_cap_freezes_on_a_face_of_the_tet(prec):
    wl = I.workload_hot_small(jitter=0.2)
    g, tn, res = _run(wl, 5, prec, max_crossings=2)
    capped = g["status"] == CAP
    assert capped.sum() > 50 and set(np.unique(g["status"])) <= {0, CAP}
    T = -2 - g["tet"][capped]
    assert (T >= 0).all()
    lam = _bary(wl.mesh.nodes, tn, T, _positions(g, capped))
    tol = LAM_TOL[prec]
    assert lam.min() >= -tol                       # inside (or on) the tet it froze in
    assert np.abs(lam).min(1).max() <= tol         # and on one of its faces
    moving = ~capped
    lam_m = _bary(wl.mesh.nodes, tn, g["tet"][moving], _positions(g, moving))
    assert lam_m.min() >= -tol
    assert res <= 1e-13


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_absorbing_walls_stop_particles_on_the_boundary(prec):
    wl = I.workload_hot_small(jitter=0.2, wall_mode=1)
    g, tn, res = _run(wl, 10, prec)
    absorbed = g["status"] == ABSORBED
    assert absorbed.sum() > wl.particles.n // 4
    r = _positions(g, absorbed)
    dist = np.minimum(r - wl.mesh.lo, wl.mesh.hi - r).min(1)   # distance to the nearest wall plane
    tol = LAM_TOL[prec]
    assert np.abs(dist).max() <= tol * wl.mesh.h
    T = -2 - g["tet"][absorbed]
    lam = _bary(wl.mesh.nodes, tn, T, r)
    assert lam.min() >= -tol and np.abs(lam).min(1).max() <= tol
    assert res <= 1e-13


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_reflecting_walls_keep_every_particle_inside(prec):
    wl = I.workload_hot_small(jitter=0.2, wall_mode=0)
    g, tn, res = _run(wl, 20, prec)
    assert (g["status"] == 0).all() and g["n_cross"].sum() > 10 * wl.particles.n
    r = _positions(g, slice(None))
    assert (r >= wl.mesh.lo - 1e-9).all() and (r <= wl.mesh.hi + 1e-9).all()
    lam = _bary(wl.mesh.nodes, tn, g["tet"], r)
    assert lam.min() >= -LAM_TOL[prec]
    assert res <= 1e-13


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_deposit_off_leaves_trajectories_unchanged_and_adds_nothing(prec):
    """fempic_set_deposit(0): the same particle states, bit for bit, and no
    deposit; switching back on deposits again."""
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.workload_hot_small(jitter=0.2, n_particles=2000)
    res = []
    for on in (True, False):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(wl.particles, prec)
        env.locate(st)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        env.set_deposit(on)
        G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
        for n in range(6):
            t = n * wl.dt
            env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
            env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
        torch.cuda.synchronize()
        res.append((st.to_numpy(), G.cpu().numpy()))
        if not on:
            env.set_deposit(True)
            env.push_step(st, e, b, wl.amp(0.0), wl.omega0, 6 * wl.dt, wl.dt)
            env.deposit(wl.omega0, 7 * wl.dt, G_cum_out=G)
            torch.cuda.synchronize()
            assert np.abs(G.cpu().numpy()).max() > 0
    (a, Ga), (b_, Gb) = res
    for k in a:
        if a[k] is not None:
            assert np.array_equal(a[k], b_[k]), k
    assert np.abs(Ga).max() > 0 and not Gb.any()


def test_bounded_wait_runs_out_and_the_step_reports_incomplete():
    """A CTA of the staged mixed push is made to wait (test support, 1 ms
    limit) on a barrier that no copy completes, after its first tile's copies
    have landed.  Its wait runs out, it drains its copies in flight and
    stops: the particles of its tiles are not advanced, fempic_stats counts
    the timeout and fempic_error_count returns FEMPIC_EINCOMPLETE.  The
    context stays usable: the next step runs normally and reports OK."""
    from paper_2208_12795_gb300 import capi
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.te101_cavity(8, 400_000, 5.0, 1e4, 3, 11)
    env = FempicEnv.from_mesh(wl.mesh, precision=1)
    st = ParticleState.from_host(wl.particles, 1)
    env.locate(st)
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    ok, _ = env.error_count()
    assert ok
    x0 = st.x.clone()
    capi.fempic_debug_stall(env.h, 0, 1_000_000)
    env.push_step(st, e, b, wl.amp(0.0), wl.omega0, 0.0, wl.dt)
    env.deposit(wl.omega0, wl.dt)
    ok, frozen = env.error_count()
    stats = env.stats()
    assert not ok and stats["wait_timeouts"] == 1
    assert "gave up" in capi.fempic_last_error()
    moved = (st.x != x0).cpu().numpy()
    assert moved[:256].sum() == 0            # CTA 0's first tile was never advanced
    assert moved.mean() > 0.9                # every other CTA ran
    env.push_step(st, e, b, wl.amp(wl.dt), wl.omega0, wl.dt, wl.dt)
    env.deposit(wl.omega0, 2 * wl.dt)
    ok, frozen = env.error_count()
    assert ok and frozen == 0 and env.stats()["wait_timeouts"] == 1
