"""Checkpoint/resume of a run (paper_2208_12795_gb300.resume): K steps, save,
a fresh env loads the file, K more steps; the particle state equals the
uninterrupted 2K-step run bit for bit and G_cum to 1e-13 of its maximum
(the device sums the deposit with atomics).  A file from another mesh or
precision form is refused."""
import numpy as np
import pytest

from paper_2208_12795_gb300 import inputs as I

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


def _G(env):
    G = torch.empty(env.n_edges, dtype=torch.float64, device="cuda")
    env.accumulate(0.0, 0.0, torch.zeros_like(G), G_cum_out=G)
    return G.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_continues_the_run(prec, tmp_path):
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    from paper_2208_12795_gb300.resume import load_run, save_run
    wl = I.workload_hot_small(n_particles=3000)
    K = 6
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    ref = ParticleState.from_host(wl.particles, prec)
    env.locate(ref)
    _steps(env, ref, wl, 0, 2 * K)
    G_ref = _G(env)

    env1 = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st = ParticleState.from_host(wl.particles, prec)
    env1.locate(st)
    _steps(env1, st, wl, 0, K)
    path = str(tmp_path / "run.pt")
    save_run(path, env1, st, K, K * wl.dt, extra={"seed": 7})
    env1.close()

    env2 = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st2, step, t, extra = load_run(path, env2)
    assert step == K and t == K * wl.dt and extra == {"seed": 7}
    _steps(env2, st2, wl, step, 2 * K)
    torch.cuda.synchronize()
    for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status", "n_cross"):
        assert torch.equal(getattr(st2, k), getattr(ref, k)), k
    G2 = _G(env2)
    assert np.abs(G_ref).max() > 0
    assert np.abs(G2 - G_ref).max() <= 1e-13 * np.abs(G_ref).max()

    other = FempicEnv.from_mesh(wl.mesh, precision=1 - prec)
    with pytest.raises(ValueError, match="precision"):
        load_run(path, other)
    env3 = FempicEnv.from_mesh(I.te101_cavity(6, 100, 5.0, 1e3, 1, 3).mesh, precision=prec)
    assert env3.n_tets != env2.n_tets
    with pytest.raises(ValueError, match="mesh"):
        load_run(path, env3)
