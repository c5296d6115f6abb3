"""GPU parity of the three-level envelope step (fempic_push_step3) against
the oracle stepping with the interpolated envelope (Sec. III-A Lagrange
representation in time, sampled at each fine step as in Sec. III-D)."""
import numpy as np
import pytest

from oracle.oracle import OracleMesh, OracleState, lagrange3_weights, push_step3 as oracle_push3
from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _levels(wl, seed):
    """Envelope levels at t_{n-1}, t_n, t_{n+1}: the workload's DoFs scaled
    and perturbed by a windowed complex field of 5 % of their size."""
    rng = np.random.default_rng(seed)
    es, bs = np.abs(wl.e_tilde).max(), np.abs(wl.b_tilde).max()
    e_lv, b_lv = [], []
    for s in (0.9, 1.0, 1.15):
        e_lv.append(s * wl.e_tilde + 0.05 * es * (rng.standard_normal(wl.e_tilde.shape)
                                                 + 1j * rng.standard_normal(wl.e_tilde.shape)))
        b_lv.append(s * wl.b_tilde + 0.05 * bs * (rng.standard_normal(wl.b_tilde.shape)
                                                 + 1j * rng.standard_normal(wl.b_tilde.shape)))
    return e_lv, b_lv


def _run(wl, prec, steps, tau):
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    tet0 = st.tet.cpu().numpy().copy()
    e_lv, b_lv = _levels(wl, 11)
    e_d = [torch.from_numpy(x).to(env.dof_dtype).cuda() for x in e_lv]
    b_d = [torch.from_numpy(x).to(env.dof_dtype).cuda() for x in b_lv]
    G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    for n in range(steps):
        t = n * wl.dt
        env.push_step3(st, e_d, b_d, lagrange3_weights(tau, t), wl.amp(t), wl.omega0, t, wl.dt)
        env.deposit(wl.omega0, t + wl.dt, G_cum_out=G)
    torch.cuda.synchronize()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets, wl.mesh.lo, wl.mesh.hi)
    ost = OracleState(wl.particles, tet0)
    oG = np.zeros(om.n_edges)
    for n in range(steps):
        t = n * wl.dt
        oracle_push3(om, ost, e_lv, b_lv, lagrange3_weights(tau, t), wl.amp(t), wl.omega0, t, wl.dt, oG,
                     wall_mode=wl.wall_mode)
    return env, st, G.cpu().numpy(), ost, oG


def _rel(a, b, floor):
    d = np.sqrt(sum((a[k] - b[k]) ** 2 for k in range(3)))
    return d / np.maximum(np.sqrt(sum(b[k] ** 2 for k in range(3))), floor)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_push_step3_matches_oracle(prec):
    wl = I.workload_small()
    steps = 40
    tau = (-5 * wl.dt, 16 * wl.dt, 37 * wl.dt)      # a field step of 21 fine steps
    env, st, G, ost, oG = _run(wl, prec, steps, tau)
    g = st.to_numpy()
    er = _rel((g["x"], g["y"], g["z"]), (ost.x, ost.y, ost.z), 1.0)
    ev = _rel((g["vx"], g["vy"], g["vz"]), (ost.vx, ost.vy, ost.vz), 1e-30)
    same = (g["tet"] == ost.tet).mean()
    eG = np.abs(G - oG).max() / np.abs(oG).max()
    print(f"\n[push_step3 prec={prec}] tet agree {same:.5f} r {er.max():.2e} v {ev.max():.2e} G {eG:.2e}")
    if prec == FP64:
        assert same == 1.0 and er.max() <= 1e-12 and ev.max() <= 1e-12 and eG <= 1e-12
        assert np.array_equal(g["n_cross"], ost.n_cross)
    else:
        assert same >= 0.99 and np.median(er) <= 1e-7 and np.median(ev) <= 2e-6 and eG <= 1e-5
        assert er.max() <= 1e-6 and ev.max() <= 1e-5


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_push_step3_with_unit_weight_equals_single_level_step(prec):
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    wl = I.workload_small()
    e_lv, b_lv = _levels(wl, 12)
    out = []
    for three in (False, True):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(wl.particles, prec)
        env.locate(st)
        e_d = [torch.from_numpy(x).to(env.dof_dtype).cuda() for x in e_lv]
        b_d = [torch.from_numpy(x).to(env.dof_dtype).cuda() for x in b_lv]
        for n in range(20):
            t = n * wl.dt
            if three:
                env.push_step3(st, e_d, b_d, (0.0, 1.0, 0.0), wl.amp(t), wl.omega0, t, wl.dt)
            else:
                env.push_step(st, e_d[1], b_d[1], wl.amp(t), wl.omega0, t, wl.dt)
        torch.cuda.synchronize()
        out.append(st.to_numpy())
    a, b = out
    assert np.array_equal(a["tet"], b["tet"]) and np.array_equal(a["status"], b["status"])
    tol = 1e-15 if prec == FP64 else 1e-7
    for k in ("x", "y", "z"):
        assert np.abs(a[k] - b[k]).max() <= tol
    for k in ("vx", "vy", "vz"):
        assert np.abs(a[k] - b[k]).max() <= tol * np.abs(b[k]).max() * 10


def test_push_step3_rejects_missing_level():
    from paper_2208_12795_gb300 import capi
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState, _ptr
    wl = I.workload_small()
    env = FempicEnv.from_mesh(wl.mesh, precision=FP64)
    st = ParticleState.from_host(wl.particles.subset(16), FP64)
    env.locate(st)
    e = torch.from_numpy(wl.e_tilde).cuda()
    b = torch.from_numpy(wl.b_tilde).cuda()
    envl = capi.fempic_envelope3()
    for k in range(3):
        envl.e_tilde[k] = _ptr(e)
        envl.b_tilde[k] = _ptr(b)
        envl.weight[k] = 1.0 / 3.0
    envl.amp = 1.0
    envl.e_tilde[2] = None
    with pytest.raises(capi.FempicError):
        capi.fempic_push_step3(env.h, st.cstruct(), envl, wl.omega0, 0.0, wl.dt)
    envl.e_tilde[2] = _ptr(e)
    envl.weight[1] = float("nan")
    with pytest.raises(capi.FempicError):
        capi.fempic_push_step3(env.h, st.cstruct(), envl, wl.omega0, 0.0, wl.dt)
