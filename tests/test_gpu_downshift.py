"""GPU parity of the downshifted integrator (Sec. III-D: M/L velocity rule,
AB4 positions) through the C ABI against the FP64 oracle of the same rule.

Tet ids, crossing counts and statuses bit-exact; positions, velocities and
the history planes within 1e-12 relative; G_cum within 1e-12 of its max
(atomic summation order differs); charge conservation D^T G_cum = rho^n -
rho^0 within 1e-13 of max |rho|.
"""
import math

import numpy as np
import pytest

from oracle.downshift import History, push_step_downshift
from oracle.oracle import OracleMesh, OracleState
from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64 = 0


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def rel_vec_err(a, b, floor):
    d = np.sqrt(sum((a[k] - b[k]) ** 2 for k in range(3)))
    nrm = np.maximum(np.sqrt(sum(b[k] ** 2 for k in range(3))), floor)
    return d / nrm


def divergence(env, G):
    en = env.query()["edge_nodes"]
    out = np.zeros(env.n_nodes)
    np.add.at(out, en[:, 1], G)
    np.subtract.at(out, en[:, 0], G)
    return out


def gpu_run(wl, steps, parts, wall_mode, tet=None, prec=FP64):
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState
    env = FempicEnv.from_mesh(wl.mesh, precision=prec, wall_mode=wall_mode)
    st = ParticleState.from_host(parts, prec)
    if tet is None:
        env.locate(st)
    else:
        st.tet.copy_(torch.from_numpy(tet).cuda())
    ds = Downshift(env, st.n)
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    tet0 = st.tet.cpu().numpy().copy()
    rho0 = env.nodal_charge(st)
    G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    for n in range(steps):
        t = n * wl.dt
        ds.step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
    rho1 = env.nodal_charge(st)
    torch.cuda.synchronize()
    return env, st, ds, G.cpu().numpy(), rho0.cpu().numpy(), rho1.cpu().numpy(), tet0


def oracle_run(wl, steps, parts, wall_mode, tet):
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi)
    st = OracleState(parts, tet)
    hist = History(st.n)
    G = np.zeros(om.n_edges)
    for n in range(steps):
        t = n * wl.dt
        push_step_downshift(om, st, hist, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G,
                            wall_mode=wall_mode)
    return om, st, hist, G


def _compare(wl, steps, wall_mode, parts=None):
    parts = parts if parts is not None else wl.particles
    env, st, ds, G, rho0, rho1, tet0 = gpu_run(wl, steps, parts, wall_mode)
    om, ost, oh, oG = oracle_run(wl, steps, parts, wall_mode, tet0)
    g = st.to_numpy()
    assert np.array_equal(g["tet"], ost.tet)
    assert np.array_equal(g["status"], ost.status)
    assert np.array_equal(g["n_cross"], ost.n_cross)
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    assert er.max() <= 1e-12, er.max()
    assert ev.max() <= 1e-12, ev.max()
    assert np.abs(G - oG).max() <= 1e-12 * np.abs(oG).max()
    # history planes: velocities v^{n-1..n-3} and the envelope samples of levels n-1, n-2
    from paper_2208_12795_gb300 import capi
    H = ds.planes.cpu().numpy()
    vsc = np.abs(np.stack([ost.vx, ost.vy, ost.vz])).max()
    for i in range(3):
        np.testing.assert_allclose(H[capi.FEMPIC_DS_VH + 3 * i:capi.FEMPIC_DS_VH + 3 * i + 3].T, oh.v[i],
                                   rtol=1e-12, atol=1e-13 * vsc)
    for lvl in range(2):
        base = capi.FEMPIC_DS_F + 12 * lvl
        for arr, off in ((oh.e, 0), (oh.b, 6)):
            want = np.concatenate([arr[lvl].real, arr[lvl].imag], axis=1)
            got = H[base + off:base + off + 6].T
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * max(np.abs(want).max(), 1e-300))
    res = np.abs(divergence(env, G) - (rho1 - rho0)).max() / np.abs(rho1).max()
    return env, st, ost, res


def test_downshift_small_cavity_matches_oracle():
    wl = I.workload_small()
    steps = 40
    env, st, ost, res = _compare(wl, steps, wl.wall_mode)
    assert ost.n_cross.sum() > 100
    assert res <= 1e-13


@pytest.mark.parametrize("wall", [0, 1])
def test_downshift_hot_tracking_walls(wall):
    """Fast particles on a jittered mesh: many crossings per step, wall hits
    (mirrored velocity histories, or absorption)."""
    wl = I.workload_hot_small(jitter=0.2, wall_mode=wall, n_particles=300)
    env, st, ost, res = _compare(wl, 12, wall)
    assert ost.n_cross.sum() > 2 * wl.particles.n
    if wall == 0:
        assert (ost.status == 0).all() and res <= 1e-13
    else:
        assert (ost.status == 2).sum() > 10


def test_downshift_full_size_sampled():
    """10M electrons on the 48^3 x 6 cube (the benchmark's workload and launch
    configuration), two steps (the first fills the history); 2000 sampled
    particles checked against the oracle one by one, conservation over all."""
    wl = I.workload_cavity48()
    env, st, ds, G, rho0, rho1, tet0 = gpu_run(wl, 2, wl.particles, wl.wall_mode)
    assert (tet0 >= 0).all()
    rng = np.random.default_rng(77)
    idx = np.sort(rng.choice(wl.particles.n, 2000, replace=False))
    P = wl.particles
    sub = I.Particles(P.x[idx], P.y[idx], P.z[idx], P.vx[idx], P.vy[idx], P.vz[idx],
                      np.array([0, len(idx)], np.int64), P.q, P.m, P.w)
    om, ost, oh, oG = oracle_run(wl, 2, sub, wl.wall_mode, tet0[idx])
    g = {k: v[idx] for k, v in st.to_numpy().items() if v is not None}
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    assert np.array_equal(g["tet"], ost.tet) and np.array_equal(g["n_cross"], ost.n_cross)
    assert er.max() <= 1e-12 and ev.max() <= 1e-12
    res = np.abs(divergence(env, G) - (rho1 - rho0)).max() / np.abs(rho1).max()
    assert res <= 1e-13


def test_downshift_rejects_bad_arguments():
    from paper_2208_12795_gb300 import capi
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState
    wl = I.workload_small()
    mixed = FempicEnv.from_mesh(wl.mesh, precision=1)
    mst = ParticleState.from_host(wl.particles, 1)
    mixed.locate(mst)
    mds = Downshift(mixed, mst.n)   # the mixed form takes complex64 DoFs and f32 velocities
    with pytest.raises(capi.FempicError):
        mds.step(mst, torch.from_numpy(wl.e_tilde).cuda(), torch.from_numpy(wl.b_tilde).cuda(), 1.0,
                 wl.omega0, 0.0, wl.dt)
    env = FempicEnv.from_mesh(wl.mesh, precision=FP64)
    st = ParticleState.from_host(wl.particles, FP64)
    env.locate(st)
    ds = Downshift(env, st.n)
    e = torch.from_numpy(wl.e_tilde).to(torch.complex128).cuda()
    b = torch.from_numpy(wl.b_tilde).to(torch.complex128).cuda()
    with pytest.raises(capi.FempicError):
        ds.step(st, e.to(torch.complex64), b.to(torch.complex64), 1.0, wl.omega0, 0.0, wl.dt)
    with pytest.raises(capi.FempicError):
        ds.step(st, e, b, 1.0, wl.omega0, 0.0, -wl.dt)
    with pytest.raises(capi.FempicError):
        ds.step(st, e, b, math.nan, wl.omega0, 0.0, wl.dt)
    other = FempicEnv.from_mesh(I.kuhn_cube_mesh(3), precision=FP64)
    with pytest.raises(capi.FempicError):
        Downshift(other, st.n).step(st, e, b, 1.0, wl.omega0, 0.0, wl.dt)
    short = Downshift(env, st.n - 1)
    with pytest.raises(capi.FempicError):
        short.step(st, e, b, 1.0, wl.omega0, 0.0, wl.dt)
    # nothing ran: the state is unchanged and a valid step still works
    ds.step(st, e, b, 1.0, wl.omega0, 0.0, wl.dt)
    torch.cuda.synchronize()
    assert (st.status.cpu().numpy() == 0).all()


def test_downshift_c_entry_checks_everything_before_any_launch():
    """Through the C entry point itself (no Python-side checks): an f64
    history on a mixed-form env is rejected (the form's f32 velocities and
    history would be read with the wrong width), and a bad species table
    (NULL weights) is rejected before the first launch, so the particles and
    history are untouched."""
    import ctypes as C

    from paper_2208_12795_gb300 import capi
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState, _ptr
    wl = I.workload_small()
    lib = capi.load()
    stream = torch.cuda.current_stream().cuda_stream
    env = FempicEnv.from_mesh(wl.mesh, precision=FP64)
    st = ParticleState.from_host(wl.particles.subset(500), FP64)
    env.locate(st)
    ds = Downshift(env, st.n)
    ds.planes.fill_(0.25)
    e = torch.from_numpy(wl.e_tilde).to(torch.complex128).cuda()
    b = torch.from_numpy(wl.b_tilde).to(torch.complex128).cuda()
    envl = capi.fempic_envelope(_ptr(e), _ptr(b), 1.0)
    hist = capi.fempic_downshift_history(st.n, _ptr(ds.planes), 0)
    before = st.to_numpy()
    mixed = FempicEnv.from_mesh(wl.mesh, precision=1)
    rc = lib.fempic_push_step_downshift(mixed.h, ds.h, C.byref(st.cstruct()), C.byref(hist), C.byref(envl),
                                        wl.omega0, 0.0, wl.dt, 1, stream)
    assert rc == capi.FEMPIC_EINVAL and "f32" in capi.fempic_downshift_last_error()
    p = st.cstruct()
    p.w = None
    rc = lib.fempic_push_step_downshift(env.h, ds.h, C.byref(p), C.byref(hist), C.byref(envl), wl.omega0, 0.0,
                                        wl.dt, 1, stream)
    assert rc == capi.FEMPIC_EINVAL
    torch.cuda.synchronize()
    after = st.to_numpy()
    for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status"):
        assert np.array_equal(before[k], after[k]), k
    assert bool((ds.planes == 0.25).all())


def test_sorted_run_carries_history_and_equals_unsorted():
    """Downshift.sort re-sorts the particle set by tet and carries the history
    planes through the same permutation (fempic_downshift_permute): a run
    sorted every 3 steps gives every particle the state and history of the
    unsorted run bit for bit, and G_cum to 1e-13 of its maximum."""
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState
    wl = I.workload_hot_small(n_particles=3000)
    steps = 12
    e = torch.from_numpy(wl.e_tilde).to(torch.complex128).cuda()
    b = torch.from_numpy(wl.b_tilde).to(torch.complex128).cuda()
    res = []
    for sort_every in (0, 3):
        env = FempicEnv.from_mesh(wl.mesh, precision=FP64)
        st = ParticleState.from_host(wl.particles, FP64)
        env.locate(st)
        ds = Downshift(env, st.n)
        scratch = st.empty_like()
        orig = torch.arange(st.n, device="cuda")
        G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
        for n in range(steps):
            t = n * wl.dt
            ds.step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
            env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
            if sort_every and (n + 1) % sort_every == 0:
                perm = ds.sort(st, scratch)
                orig = orig[perm.long()]
        torch.cuda.synchronize()
        inv = torch.empty_like(orig)
        inv[orig] = torch.arange(st.n, device="cuda")   # position of each original particle
        cols = {k: getattr(st, k)[inv].cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status")}
        cols["hist"] = ds.planes[:33, inv].cpu().numpy()
        res.append((cols, G.cpu().numpy()))
    (a, Ga), (c, Gc) = res
    for k in a:
        assert np.array_equal(a[k], c[k]), k
    assert np.abs(Ga).max() > 0
    assert np.abs(Ga - Gc).max() <= 1e-13 * np.abs(Ga).max()


# Stated error of the mixed downshifted step against the FP64 oracle: the
# rule, the samples and the history run in FP32 and positions in FP64, so r
# and v carry FP32 rounding (median and max relative error), and a particle
# whose FP32 path passes within rounding of a face may take the other tet.
DS_MIXED_TOL = {"cube4_2k_te101": dict(r_med=1e-8, r_max=1e-7, v_med=1e-6, v_max=1e-5, tet=0.99),
                "cube4j_hot": dict(r_med=2e-6, r_max=1e-5, v_med=1e-6, v_max=1e-5, tet=0.99)}


@pytest.mark.parametrize("maker,steps", [(I.workload_small, 40),
                                         (lambda: I.workload_hot_small(jitter=0.2, wall_mode=0, n_particles=300),
                                          12)])
def test_downshift_mixed_form_error_vs_oracle(maker, steps):
    """The mixed form (contract env: f32 velocities, samples and history) on
    the cavity and the hot jittered load with reflecting walls, against the
    FP64 oracle of the rule: stated bounds on r and v, tet agreement, and
    charge conservation D^T G = rho^n - rho^0 to 1e-13 (the env's mixed step
    deposits the AB4 segments)."""
    wl = maker()
    parts = wl.particles
    env, st, ds, G, rho0, rho1, tet0 = gpu_run(wl, steps, parts, wl.wall_mode, prec=1)
    om, ost, oh, oG = oracle_run(wl, steps, parts, wl.wall_mode, tet0)
    g = st.to_numpy()
    same = (g["tet"] == ost.tet).mean()
    er = rel_vec_err((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = rel_vec_err((g["vx"].astype(np.float64), g["vy"].astype(np.float64), g["vz"].astype(np.float64)),
                     (ost.vx, ost.vy, ost.vz), 1e-30)
    res = np.abs(divergence(env, G) - (rho1 - rho0)).max() / np.abs(rho1).max()
    tol = DS_MIXED_TOL[wl.name]
    print(f"\n[downshift mixed {wl.name}] tet agree {same:.4f}  r med {np.median(er):.2e} max {er.max():.2e}  "
          f"v med {np.median(ev):.2e} max {ev.max():.2e}  conservation {res:.2e}")
    assert ost.n_cross.sum() > 100
    assert same >= tol["tet"]
    assert np.median(er) <= tol["r_med"] and er.max() <= tol["r_max"]
    assert np.median(ev) <= tol["v_med"] and ev.max() <= tol["v_max"]
    assert res <= 1e-13


def test_downshift_mixed_sorted_run_equals_unsorted():
    """The mixed form's f32 history follows the sort too: bit for bit."""
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState
    wl = I.workload_hot_small(n_particles=3000)
    steps = 9
    res = []
    for sort_every in (0, 3):
        env = FempicEnv.from_mesh(wl.mesh, precision=1)
        e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
        b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
        st = ParticleState.from_host(wl.particles, 1)
        env.locate(st)
        ds = Downshift(env, st.n)
        assert ds.planes.dtype == torch.float32
        scratch = st.empty_like()
        orig = torch.arange(st.n, device="cuda")
        for n in range(steps):
            t = n * wl.dt
            ds.step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
            env.deposit(wl.omega0, t + wl.dt)
            if sort_every and (n + 1) % sort_every == 0:
                orig = orig[ds.sort(st, scratch).long()]
        torch.cuda.synchronize()
        inv = torch.empty_like(orig)
        inv[orig] = torch.arange(st.n, device="cuda")
        cols = {k: getattr(st, k)[inv].cpu().numpy() for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status")}
        cols["hist"] = ds.planes[:33, inv].cpu().numpy()
        res.append(cols)
    for k in res[0]:
        assert np.array_equal(res[0][k], res[1][k]), k
