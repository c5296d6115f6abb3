"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs.

FP64 form: tet ids, crossing counts and statuses bit-exact; positions and
velocities within 1e-12 relative; G_cum within 1e-12 of its max (atomic
summation order differs).  Mixed form: per-quantity error against the FP64
oracle is measured and bounded.  Both forms: charge conservation
D^T G_cum = rho^n - rho^0 within 1e-13 of max |rho|.
"""
import math

import numpy as np
import pytest

from oracle.oracle import (OracleMesh, OracleState, envelope_frame, push_step as oracle_push,
                           run as oracle_run)
from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED, Q24 = 0, 1, 2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _env_mod():
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    return FempicEnv, ParticleState


def gpu_run(wl, precision, steps, parts=None, max_crossings=4096, wall_mode=None, tet=None):
    FempicEnv, ParticleState = _env_mod()
    env = FempicEnv.from_mesh(wl.mesh, precision=precision, max_crossings=max_crossings,
                              wall_mode=wl.wall_mode if wall_mode is None else wall_mode)
    st = ParticleState.from_host(parts if parts is not None else wl.particles, precision)
    if tet is None:
        env.locate(st)
    else:
        st.tet.copy_(torch.from_numpy(tet).cuda())
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    tet0 = st.tet.cpu().numpy().copy()
    rho0 = env.nodal_charge(st)
    G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    for n in range(steps):
        t = n * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
    rho1 = env.nodal_charge(st)
    torch.cuda.synchronize()
    return env, st, G.cpu().numpy(), rho0.cpu().numpy(), rho1.cpu().numpy(), tet0


def oracle_run_wl(wl, steps, parts=None, max_crossings=4096, wall_mode=None):
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi)
    P = parts if parts is not None else wl.particles
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    for n in range(steps):
        t = n * wl.dt
        oracle_push(om, st, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G,
                    max_crossings=max_crossings, wall_mode=wl.wall_mode if wall_mode is None else wall_mode)
    return om, st, G, tet


def divergence(env, G):
    en = env.query()["edge_nodes"]
    out = np.zeros(env.n_nodes)
    np.add.at(out, en[:, 1], G)
    np.subtract.at(out, en[:, 0], G)
    return out


def conservation_residual(env, G, rho0, rho1):
    return np.abs(divergence(env, G) - (rho1 - rho0)).max() / np.abs(rho1).max()


def rel_vec_err(a, b, floor):
    d = np.sqrt(sum((a[k] - b[k]) ** 2 for k in range(3)))
    nrm = np.maximum(np.sqrt(sum(b[k] ** 2 for k in range(3))), floor)
    return d / nrm


# ----------------------------------------------------------------- tables
def test_tables_match_generator_and_oracle():
    FempicEnv, _ = _env_mod()
    for m in (I.kuhn_cube_mesh(4), I.kuhn_cube_mesh(5, jitter=0.2, rng=np.random.default_rng(3))):
        env = FempicEnv.from_mesh(m)
        q = env.query()
        ts, e, f, te, tf = I.mesh_topology(m.tets)
        om = OracleMesh(m.nodes, m.tets)
        ot = om.tables()
        assert np.array_equal(q["edge_nodes"], e) and np.array_equal(q["face_nodes"], f)
        assert np.array_equal(q["tet_edges"], te) and np.array_equal(q["tet_faces"], tf)
        for k in q:
            assert np.array_equal(q[k], ot[k]), k


# ----------------------------------------------------------------- locate
def test_locate_bit_exact():
    FempicEnv, ParticleState = _env_mod()
    rng = np.random.default_rng(5)
    for m in (I.kuhn_cube_mesh(4), I.kuhn_cube_mesh(6, jitter=0.2, rng=np.random.default_rng(9))):
        n = 20000
        pts = rng.random((n, 3))
        pts[:200] = rng.integers(0, 5, size=(200, 3)) * 0.25          # lattice points: ties
        pts[200:210] = [[1.5, 0.5, 0.5]] * 10                           # outside -> LOST
        pts[210, 0] = np.nan
        P = I.Particles(pts[:, 0], pts[:, 1], pts[:, 2], np.zeros(n), np.zeros(n), np.zeros(n),
                        np.array([0, n], np.int64), np.array([-I.E_CHARGE]), np.array([I.M_ELECTRON]),
                        np.array([1.0]))
        env = FempicEnv.from_mesh(m)
        st = ParticleState.from_host(P, FP64)
        env.locate(st)
        om = OracleMesh(m.nodes, m.tets)
        ot, os_ = om.locate(P.x, P.y, P.z)
        assert np.array_equal(st.tet.cpu().numpy(), ot)
        assert np.array_equal(st.status.cpu().numpy(), os_)
        assert (ot[200:211] == -1).all()


# ----------------------------------------------------------- FP64 parity
def _compare_fp64(wl, steps, **kw):
    env, st, G, rho0, rho1, tet0 = gpu_run(wl, FP64, steps, **kw)
    om, ost, oG, otet0 = oracle_run_wl(wl, steps, **kw)
    g = st.to_numpy()
    assert np.array_equal(tet0, otet0)
    assert np.array_equal(g["tet"], ost.tet)
    assert np.array_equal(g["status"], ost.status)
    assert np.array_equal(g["n_cross"], ost.n_cross)
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    assert er.max() <= 1e-12, er.max()
    assert ev.max() <= 1e-12, ev.max()
    assert np.abs(G - oG).max() <= 1e-12 * np.abs(oG).max()
    return env, st, G, rho0, rho1, ost


def test_fp64_small_cavity_200_steps():
    wl = I.workload_small()
    env, st, G, rho0, rho1, ost = _compare_fp64(wl, wl.steps)
    assert ost.n_cross.sum() > 1000
    assert conservation_residual(env, G, rho0, rho1) <= 1e-13


@pytest.mark.parametrize("jitter,wall", [(0.0, 0), (0.2, 0), (0.2, 1)])
def test_fp64_hot_tracking_walls(jitter, wall):
    wl = I.workload_hot_small(jitter=jitter, wall_mode=wall)
    env, st, G, rho0, rho1, ost = _compare_fp64(wl, wl.steps)
    if wall == 0:
        assert ost.n_cross.sum() > 10 * wl.particles.n
        assert (ost.status == 0).all()
        assert conservation_residual(env, G, rho0, rho1) <= 1e-13
    else:                                   # absorbed particles stop crossing early
        assert ost.n_cross.sum() > 2 * wl.particles.n
        assert (ost.status == 2).sum() > wl.particles.n // 4


def test_fp64_crossing_cap_matches_oracle():
    wl = I.workload_hot_small(jitter=0.2)
    _, st, _, _, _, ost = _compare_fp64(wl, 5, max_crossings=2)
    assert (ost.status == 1).sum() > 50


def test_edge_cases_empty_skipped_bad_tet_nonfinite():
    FempicEnv, ParticleState = _env_mod()
    wl = I.workload_small()
    for prec in (FP64, MIXED):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        empty = ParticleState.from_host(wl.particles.subset(0), prec)
        env.push_step(empty, e, b, 1.0, wl.omega0, 0.0, wl.dt)          # n = 0 is valid
        P = wl.particles.subset(8)
        P.vx[3] = np.nan
        st = ParticleState.from_host(P, prec)
        env.locate(st)
        tet = st.tet.cpu().numpy()
        tet[0] = -1                       # no tet: skipped
        tet[1] = env.n_tets + 3           # out of range: LOST
        tet[2] = -2 - tet[2]              # frozen: skipped
        st.tet.copy_(torch.from_numpy(tet).cuda())
        x0 = st.x.clone()
        env.push_step(st, e, b, 1.0, wl.omega0, 0.0, wl.dt)
        env.deposit(wl.omega0, wl.dt)
        s = st.status.cpu().numpy()
        t2 = st.tet.cpu().numpy()
        assert s[1] == 4 and t2[1] == -1
        assert s[3] == 3 and t2[3] == -2 - tet[3] and st.x[3].item() == x0[3].item()
        assert t2[0] == -1 and t2[2] == tet[2] and st.x[0].item() == x0[0].item()
        assert (s[4:] == 0).all() and (t2[4:] >= 0).all()
        stats = env.stats()
        assert stats["frozen"] == 2 and stats["steps"] == 2


def test_bad_dof_dtype_rejected():
    FempicEnv, ParticleState = _env_mod()
    from paper_2208_12795_gb300.capi import FempicError
    wl = I.workload_small()
    env = FempicEnv.from_mesh(wl.mesh, precision=MIXED)
    st = ParticleState.from_host(wl.particles.subset(4), MIXED)
    e = torch.from_numpy(wl.e_tilde).cuda()      # complex128 for a mixed env
    b = torch.from_numpy(wl.b_tilde).cuda()
    with pytest.raises(FempicError):
        env.push_step(st, e, b, 1.0, wl.omega0, 0.0, wl.dt)


# ------------------------------------------------- envelope-frame deposit
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 1e-5), (Q24, 1e-4)])
def test_envelope_frame_deposit_matches_oracle(prec, tol):
    """fempic_deposit's outputs after every step: dG_out, G_cum_out and the
    envelope-frame current G~ = e^{-j omega0 t_next} G_cum that the field
    solve consumes (Sec. III-A forcing term, Sec. III-D G_integral).  G~ is
    the oracle's envelope-frame map of the GPU's own G_cum to rounding (so
    its phase is taken at t_next, not t), and the oracle's G~ within the
    form's tolerance of its maximum."""
    FempicEnv, ParticleState = _env_mod()
    wl = I.workload_small()
    steps = 12
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    tet, _ = om.locate(wl.particles.x, wl.particles.y, wl.particles.z)
    ost = OracleState(wl.particles, tet)
    oG = np.zeros(om.n_edges)
    dG = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    Gc = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    Ge = torch.zeros(env.n_edges, dtype=torch.complex128, device="cuda")
    G_sum = np.zeros(env.n_edges)
    for n in range(steps):
        t, t1 = n * wl.dt, (n + 1) * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t1, dG_out=dG, G_cum_out=Gc, G_env_out=Ge)
        oracle_push(om, ost, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, oG)
        g_cum, g_env, d = Gc.cpu().numpy(), Ge.cpu().numpy(), dG.cpu().numpy()
        G_sum += d
        scale = np.abs(g_cum).max()
        assert np.abs(G_sum - g_cum).max() <= 1e-14 * scale
        own = envelope_frame(g_cum, wl.omega0, t1)
        assert np.abs(g_env - own).max() <= 1e-15 * scale
        ref = envelope_frame(oG, wl.omega0, t1)
        err = np.abs(g_env - ref).max() / np.abs(ref).max()
        assert err <= tol, (n, err)
        # the phase of the step's own start time would not match
        assert np.abs(g_env - envelope_frame(g_cum, wl.omega0, t)).max() > 1e-3 * scale
    print(f"\n[envelope frame prec={prec}] after {steps} steps: rel err {err:.2e}")


# ---------------------------------------------------------- mixed form
# Stated error of the mixed forms against the FP64 oracle (per workload):
# median / max relative error of positions and velocities, max |dG| / max |G|.
# The FP32 push sets the position and velocity errors of both forms; the
# deposit error of the contract form follows the trajectories' (the path
# integral itself is FP64-accurate), the 24-bit form adds its 2^-24 of a tet.
MIXED_TOL = {
    (MIXED, "cube4_2k_te101"): dict(r_med=1e-7, r_max=1e-6, v_med=2e-6, v_max=1e-5, G=1e-5, tet=0.99),
    (MIXED, "cube4j_hot"): dict(r_med=1e-5, r_max=1e-4, v_med=1e-5, v_max=1e-4, G=1e-4, tet=0.99),
    (Q24, "cube4_2k_te101"): dict(r_med=1e-7, r_max=1e-6, v_med=2e-6, v_max=1e-5, G=1e-4, tet=0.99),
    (Q24, "cube4j_hot"): dict(r_med=1e-5, r_max=1e-4, v_med=1e-5, v_max=1e-4, G=1e-4, tet=0.99),
}


@pytest.mark.parametrize("prec", [MIXED, Q24])
@pytest.mark.parametrize("maker", [I.workload_small, I.workload_hot_small])
def test_mixed_error_vs_oracle_and_conservation(maker, prec):
    wl = maker()
    steps = min(wl.steps, 100)
    env, st, G, rho0, rho1, _ = gpu_run(wl, prec, steps)
    om, ost, oG, _ = oracle_run_wl(wl, steps)
    g = st.to_numpy()
    same_tet = (g["tet"] == ost.tet).mean()
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    eG = np.abs(G - oG).max() / np.abs(oG).max()
    res = conservation_residual(env, G, rho0, rho1)
    print(f"\n[prec={prec} {wl.name}] tet agree {same_tet:.5f}  r err max {er.max():.2e} med {np.median(er):.2e}  "
          f"v err max {ev.max():.2e} med {np.median(ev):.2e}  G err {eG:.2e}  conservation {res:.2e}")
    tol = MIXED_TOL[(prec, wl.name)]
    assert (g["status"] == 0).all()
    assert res <= 1e-13
    assert same_tet >= tol["tet"]
    assert np.median(er) <= tol["r_med"] and er.max() <= tol["r_max"]
    assert np.median(ev) <= tol["v_med"] and ev.max() <= tol["v_max"]
    assert eG <= tol["G"]


@pytest.mark.parametrize("prec,tol", [(MIXED, 2.0 ** -24), (Q24, 64 * 2.0 ** -24)])
def test_mixed_one_step_deposit_close_to_oracle(prec, tol):
    """One step from identical FP64 inputs: each mixed form's deposit is the
    exact path integral of its own (FP32-pushed) trajectory; the difference
    from the oracle's is the trajectory's FP32 error (contract form) plus the
    24-bit barycentrics' resolution (24-bit form), in units of q w."""
    wl = I.workload_small()
    env, st, G, _, _, _ = gpu_run(wl, prec, 1)
    om, ost, oG, _ = oracle_run_wl(wl, 1)
    scale = abs(wl.particles.q[0] * wl.particles.w[0])
    err = np.abs(G - oG).max() / scale
    print(f"\n[one-step deposit prec={prec}] max |dG - dG_oracle| = {err:.2e} q w")
    assert err <= tol


# ------------------------------------------------ full-size sampled parity
@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_full_size_cavity48_sampled(prec):
    """10M electrons on the 48^3 x 6 cube, one step in the benchmark's launch
    configuration; 20k sampled particles checked against the oracle one by
    one, conservation checked over all particles."""
    wl = I.workload_cavity48()
    env, st, G, rho0, rho1, tet0 = gpu_run(wl, prec, 1)
    assert (tet0 >= 0).all()
    rng = np.random.default_rng(123)
    idx = np.sort(rng.choice(wl.particles.n, 20000, replace=False))
    P = wl.particles
    sub = I.Particles(P.x[idx], P.y[idx], P.z[idx], P.vx[idx], P.vy[idx], P.vz[idx],
                      np.array([0, len(idx)], np.int64), P.q, P.m, P.w)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    ost = OracleState(sub, tet0[idx])
    oG = np.zeros(om.n_edges)
    oracle_push(om, ost, wl.e_tilde, wl.b_tilde, wl.amp(0.0), wl.omega0, 0.0, wl.dt, oG)
    g = {k: v[idx] for k, v in st.to_numpy().items() if v is not None}
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    same = (g["tet"] == ost.tet).mean()
    print(f"\n[cavity48 prec={prec}] tet agree {same:.6f} r err {er.max():.2e} v err {ev.max():.2e}")
    if prec == FP64:
        assert same == 1.0 and er.max() <= 1e-12 and ev.max() <= 1e-12
        assert np.array_equal(g["n_cross"], ost.n_cross)
    else:
        assert same >= 0.999 and er.max() <= 1e-6 and ev.max() <= 1e-4
    assert conservation_residual(env, G, rho0, rho1) <= 1e-13


# ------------------------------------------------------------------ sort
@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_sort_by_species_and_tet(prec):
    FempicEnv, ParticleState = _env_mod()
    m = I.kuhn_cube_mesh(6)
    rng = np.random.default_rng(77)
    a = I.uniform_maxwellian(30000, 1.0, rng)
    b = I.uniform_maxwellian(17001, 1.0, rng, q=I.E_CHARGE, m=1836 * I.M_ELECTRON)
    P = I.concat_species([a, b])
    env = FempicEnv.from_mesh(m, precision=prec)
    st = ParticleState.from_host(P, prec)
    env.locate(st)
    tet = st.tet.cpu().numpy()
    tet[::97] = -1                           # unlocated: sorted last in its species range
    st.tet.copy_(torch.from_numpy(tet).cuda())
    st.n_cross.copy_(torch.arange(P.n, dtype=torch.int32, device="cuda"))
    before = st.to_numpy()
    scratch = st.empty_like()
    env.sort(st, scratch)
    after = st.to_numpy()
    perm = after["n_cross"]                  # the original index travels with each particle
    assert np.array_equal(np.sort(perm), np.arange(P.n))
    for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status"):
        assert np.array_equal(after[k], before[k][perm]), k
    sb = P.species_begin
    for s in range(2):
        seg = slice(sb[s], sb[s + 1])
        assert np.all((perm[seg] >= sb[s]) & (perm[seg] < sb[s + 1]))   # species ranges stay put
        key = np.where(after["tet"][seg] >= 0, after["tet"][seg], env.n_tets)
        assert np.all(np.diff(key) >= 0)


# -------------------------------------------------- staged vs plain path
def _unaligned_copy(t):
    """Same values in a buffer offset by one element: not 16-byte aligned."""
    buf = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
    v = buf[1:]
    v.copy_(t)
    return v


@pytest.mark.parametrize("prec", [MIXED, Q24])
def test_mixed_staged_path_equals_plain_path(prec):
    """The bulk-copy staged common-path kernel (16-byte aligned particle
    arrays) and the plain kernel (unaligned arrays) give bit-identical
    particles; dG is bit-identical in the 24-bit form (integer sums) and
    equal to FP64 rounding in the contract form (FP64 atomics)."""
    FempicEnv, ParticleState = _env_mod()
    wl = I.te101_cavity(12, 2_000_000, 5.0, 1e4, 5, 7, dt=2e-9)   # ~13 tiles per staged CTA
    res = []
    for aligned in (True, False):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(wl.particles, prec)
        if not aligned:
            for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status", "n_cross"):
                setattr(st, k, _unaligned_copy(getattr(st, k)))
        env.locate(st)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
        for n in range(wl.steps):
            env.push_step(st, e, b, wl.amp(n * wl.dt), wl.omega0, n * wl.dt, wl.dt)
            env.deposit(wl.omega0, (n + 1) * wl.dt, G_cum_out=G)
        torch.cuda.synchronize()
        res.append((st.to_numpy(), G.cpu().numpy(), env.stats()))
        env.close()
    (a, Ga, sa), (b_, Gb, sb) = res
    for k in a:
        assert np.array_equal(a[k], b_[k]), k
    if prec == Q24:
        assert np.array_equal(Ga, Gb)
    else:
        assert np.abs(Ga - Gb).max() <= 1e-13 * np.abs(Ga).max()
    assert sa["crossings"] == sb["crossings"] > 0 and sa["wait_timeouts"] == sb["wait_timeouts"] == 0


# ------------------------------------------- other workload shapes, sampled
def _sampled_parity(wl, prec, n_sample, seed):
    """One step of every particle on the GPU; n_sample particles checked one
    by one against the oracle; conservation checked over all particles."""
    env, st, G, rho0, rho1, tet0 = gpu_run(wl, prec, 1)
    assert (tet0 >= 0).all()
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(wl.particles.n, n_sample, replace=False))
    P = wl.particles
    # keep each sampled particle's species: rebuild species ranges over the sample
    sp = np.searchsorted(P.species_begin[1:], idx, side="right")
    order = np.argsort(sp, kind="stable")
    idx = idx[order]
    sp = sp[order]
    begins = np.searchsorted(sp, np.arange(len(P.q) + 1))
    sub = I.Particles(P.x[idx], P.y[idx], P.z[idx], P.vx[idx], P.vy[idx], P.vz[idx],
                      begins.astype(np.int64), P.q, P.m, P.w)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi)
    ost = OracleState(sub, tet0[idx])
    oG = np.zeros(om.n_edges)
    oracle_push(om, ost, wl.e_tilde, wl.b_tilde, wl.amp(0.0), wl.omega0, 0.0, wl.dt, oG)
    g = {k: v[idx] for k, v in st.to_numpy().items() if v is not None}
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    same = (g["tet"] == ost.tet).mean()
    res = conservation_residual(env, G, rho0, rho1)
    return same, er, ev, res, g, ost


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_full_size_jittered64_beam_plasma_sampled(prec):
    """64^3 x 6 jittered cube, 5M 10 keV beam electrons (several face crossings
    per step) + 45M cosine-profile plasma electrons, random windowed DoFs."""
    wl = I.workload_jittered64()
    same, er, ev, res, g, ost = _sampled_parity(wl, prec, 20000, 321)
    print(f"\n[jittered64 prec={prec}] tet agree {same:.6f} r err {er.max():.2e} v err {ev.max():.2e} "
          f"conservation {res:.2e} crossings/particle {ost.n_cross.mean():.3f}")
    assert ost.n_cross.mean() > 0.1
    if prec == FP64:
        assert same == 1.0 and er.max() <= 1e-12 and ev.max() <= 1e-12
        assert np.array_equal(g["n_cross"], ost.n_cross)
    else:
        assert same >= 0.999 and np.median(er) <= 1e-7 and np.median(ev) <= 1e-5
        assert er.max() <= 1e-6 and ev.max() <= 1e-4
    assert res <= 1e-13


@pytest.mark.parametrize("prec", [FP64, MIXED, Q24])
def test_large96_two_species_slice_sampled(prec):
    """96^3 x 6 cube (5.3M tets) with the two-species load (electrons and
    1836 m_e ions at 2 eV) and random windowed DoFs, on a 4M-particle slice."""
    base = I.workload_large96(n_particles=2)
    sb, q, m, w, temp = I.large96_species(4_000_000)
    cols = []
    for s in range(2):
        n = int(sb[s + 1] - sb[s])
        cols.append(I.maxwellian_chunk(I.SEED_BASE + 5 + 1000 * s, 0, n, temp, m[s]))
    arr = [np.concatenate([c[k] for c in cols]) for k in range(6)]
    parts = I.Particles(*arr, sb, q, m, w)
    wl = I.Workload("large96_slice", base.mesh, parts, base.e_tilde, base.b_tilde, base.omega0, base.dt, 1, 0.0)
    same, er, ev, res, g, ost = _sampled_parity(wl, prec, 20000, 654)
    print(f"\n[large96 slice prec={prec}] tet agree {same:.6f} r err {er.max():.2e} v err {ev.max():.2e} "
          f"conservation {res:.2e}")
    if prec == FP64:
        assert same == 1.0 and er.max() <= 1e-12 and ev.max() <= 1e-12
    else:
        assert same >= 0.999 and np.median(er) <= 1e-7 and np.median(ev) <= 1e-5
        assert er.max() <= 1e-6 and ev.max() <= 1e-4
    assert res <= 1e-13
