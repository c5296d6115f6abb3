"""The library's debug build (libfempic_env_debug.so, compiled with
FEMPIC_BOUNDS_CHECK): every index read from a mesh table is checked against
its range before it addresses memory.  A test writes out-of-range entries
into the device edge-id and neighbour tables of one populated tet
(fempic_debug_set_table, which only the debug build accepts) and runs steps
of every form: the checks skip the bad accesses (the DoF reads as zero, the
deposit term is dropped, a walking particle freezes with status LOST),
fempic_error_count reports FEMPIC_EBOUNDS, and the context stays usable.
The downshifted step's own edge- and face-id tables are corrupted the same
way (fempic_downshift_debug_set_table) in the FP64 and contract forms.  With
intact tables the debug build reports nothing and advances particles
exactly as the release build does.  The debug library runs in a spawned
process (the library is chosen when the binding is first loaded)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _steps(env, st, wl, k0, k1):
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    for k in range(k0, k1):
        t = k * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt)


def _run(prec):
    """Clean steps, then steps with corrupted tables; returns the error codes,
    the clean state and the number of LOST particles."""
    from paper_2208_12795_gb300 import capi, inputs as I
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.workload_hot_small(n_particles=3000)
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    _steps(env, st, wl, 0, 2)
    rc_clean, _ = capi.fempic_error_count(env.h)
    clean = {k: getattr(st, k).cpu().numpy().copy() for k in ("x", "vx", "tet")}
    tet = st.tet.cpu().numpy()
    T = int(np.bincount(tet[tet >= 0]).argmax())
    rc_set = [capi.fempic_debug_set_table(env.h, capi.FEMPIC_TABLE_EDGE, 6 * T + 2, env.n_edges + 1000)]
    for k in range(4):
        rc_set.append(capi.fempic_debug_set_table(env.h, capi.FEMPIC_TABLE_NEIGHBOUR, 4 * T + k, env.n_tets + 77))
    _steps(env, st, wl, 2, 5)
    rc_bad, n_frozen = capi.fempic_error_count(env.h)
    torch.cuda.synchronize()
    status = st.status.cpu().numpy()
    ok_after = bool(torch.isfinite(st.x).all().item())
    return rc_clean, clean, rc_set, rc_bad, int((status == capi.FEMPIC_P_LOST).sum()), n_frozen, ok_after


def _ds_steps(env, ds, st, wl, k0, k1):
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    for k in range(k0, k1):
        t = k * wl.dt
        ds.step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt)


def _ds_setup(prec):
    from paper_2208_12795_gb300 import inputs as I
    from paper_2208_12795_gb300.env import Downshift, FempicEnv, ParticleState
    wl = I.workload_hot_small(n_particles=300)
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    return wl, env, st, Downshift(env, st.n)


def _run_ds(prec):
    """The downshifted step's own edge- and face-id tables: clean steps, then
    steps with one out-of-range entry in each."""
    from paper_2208_12795_gb300 import capi
    wl, env, st, ds = _ds_setup(prec)
    tet0 = st.tet.cpu().numpy().copy()
    _ds_steps(env, ds, st, wl, 0, 2)
    rc_clean, _ = capi.fempic_error_count(env.h)
    clean = {k: getattr(st, k).cpu().numpy().copy() for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status")}
    clean["tet0"] = tet0
    tet = st.tet.cpu().numpy()
    T = int(np.bincount(tet[tet >= 0]).argmax())
    rc_set = [capi.fempic_downshift_debug_set_table(ds.h, capi.FEMPIC_TABLE_EDGE, 6 * T + 1, env.n_edges + 1000),
              capi.fempic_downshift_debug_set_table(ds.h, capi.FEMPIC_TABLE_FACE, 4 * T + 2, -5)]
    _ds_steps(env, ds, st, wl, 2, 4)
    rc_bad, _ = capi.fempic_error_count(env.h)
    torch.cuda.synchronize()
    ok_after = bool(torch.isfinite(st.x).all().item()) and bool(torch.isfinite(st.vx).all().item())
    return rc_clean, clean, rc_set, rc_bad, ok_after


def _rel(a, b, floor):
    d = np.sqrt(sum((a[k] - b[k]) ** 2 for k in range(3)))
    return d / np.maximum(np.sqrt(sum(b[k] ** 2 for k in range(3))), floor)


def _ds_against_oracle(prec, g):
    """Two downshifted steps of the FP64 oracle from the same located start:
    FP64 form tets and statuses exact, r and v within 1e-12 relative; mixed
    form within the hot load's stated bounds of the downshift parity tests."""
    from oracle.downshift import History, push_step_downshift
    from oracle.oracle import OracleMesh, OracleState
    from paper_2208_12795_gb300 import inputs as I
    wl = I.workload_hot_small(n_particles=300)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi)
    ost = OracleState(wl.particles, g["tet0"])
    hist = History(ost.n)
    G = np.zeros(om.n_edges)
    for n in range(2):
        t = n * wl.dt
        push_step_downshift(om, ost, hist, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G,
                            wall_mode=wl.wall_mode)
    er = _rel((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = _rel(tuple(g[k].astype(np.float64) for k in ("vx", "vy", "vz")), (ost.vx, ost.vy, ost.vz), 1e-30)
    if prec == 0:
        assert np.array_equal(g["tet"], ost.tet) and np.array_equal(g["status"], ost.status)
        assert er.max() <= 1e-12 and ev.max() <= 1e-12, (er.max(), ev.max())
    else:
        assert (g["tet"] == ost.tet).mean() >= 0.99
        assert np.median(er) <= 2e-6 and er.max() <= 1e-5, (np.median(er), er.max())
        assert np.median(ev) <= 1e-6 and ev.max() <= 1e-5, (np.median(ev), ev.max())


def _child(q, lib):
    os.environ["FEMPIC_LIBRARY"] = lib
    try:
        q.put(("ok", ({prec: _run(prec) for prec in (0, 1, 2)}, {prec: _run_ds(prec) for prec in (0, 1)})))
    except Exception as exc:   # report, do not hang the parent
        q.put(("error", repr(exc)))


def test_release_build_refuses_table_writes():
    from paper_2208_12795_gb300 import capi, inputs as I
    from paper_2208_12795_gb300.env import FempicEnv
    env = FempicEnv.from_mesh(I.workload_small().mesh, precision=0)
    assert capi.fempic_debug_set_table(env.h, capi.FEMPIC_TABLE_EDGE, 0, 10 ** 8) == capi.FEMPIC_EINVAL
    from paper_2208_12795_gb300.env import Downshift
    ds = Downshift(env, 1)
    assert capi.fempic_downshift_debug_set_table(ds.h, capi.FEMPIC_TABLE_FACE, 0, 10 ** 8) == capi.FEMPIC_EINVAL


def test_debug_build_skips_and_reports_bad_table_indices():
    import multiprocessing as mp
    from paper_2208_12795_gb300 import build, capi
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_child, args=(q, build.DEBUG_LIB))
    p.start()
    kind, res = q.get(timeout=600)
    p.join(timeout=120)
    assert kind == "ok", res
    assert p.exitcode == 0
    res, res_ds = res
    for prec, (rc_clean, clean, rc_set, rc_bad, ok_after) in res_ds.items():
        print(f"\n[debug build downshift prec={prec}] clean rc {rc_clean}, corrupted rc {rc_bad}")
        assert rc_clean == capi.FEMPIC_OK
        assert rc_set == [capi.FEMPIC_OK] * 2
        assert rc_bad == capi.FEMPIC_EBOUNDS
        assert ok_after
        # with intact tables the debug build's downshifted step meets the
        # downshift parity bounds against the FP64 oracle (its field pass is
        # compiled with the checks, so it need not match the release build's
        # rounding bit for bit)
        _ds_against_oracle(prec, clean)
    for prec, (rc_clean, clean, rc_set, rc_bad, n_lost, n_frozen, ok_after) in res.items():
        print(f"\n[debug build prec={prec}] clean rc {rc_clean}, corrupted rc {rc_bad}, LOST {n_lost}, "
              f"frozen {n_frozen}")
        assert rc_clean == capi.FEMPIC_OK
        assert rc_set == [capi.FEMPIC_OK] * 5
        assert rc_bad == capi.FEMPIC_EBOUNDS
        assert n_lost > 0 and n_frozen >= n_lost
        assert ok_after
        # with intact tables the debug build advances particles exactly as the release build
        from paper_2208_12795_gb300 import inputs as I
        from paper_2208_12795_gb300.env import FempicEnv, ParticleState
        wl = I.workload_hot_small(n_particles=3000)
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(wl.particles, prec)
        env.locate(st)
        _steps(env, st, wl, 0, 2)
        torch.cuda.synchronize()
        for k in ("x", "vx", "tet"):
            assert np.array_equal(getattr(st, k).cpu().numpy(), clean[k]), (prec, k)
