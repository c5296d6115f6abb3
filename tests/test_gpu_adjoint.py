"""GPU adjoint of the particle step (kinetic energy after K steps) against the
oracle's forward-mode tangent and against central finite differences of the
GPU forward run.

The derivative is that of the piecewise smooth map for a fixed tet sequence;
the finite-difference runs check that the sequence (tets, crossing counts)
is unchanged.
"""
import numpy as np
import pytest

from oracle.oracle import OracleMesh, OracleState, kinetic_energy_jvp, push_step_jvp
from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP64, MIXED = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _mods():
    from paper_2208_12795_gb300 import adjoint as A
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    return A, FempicEnv, ParticleState


def _directions(rng, wl, n, om_ne, om_nf):
    de = (rng.standard_normal(om_ne) + 1j * rng.standard_normal(om_ne)) * np.abs(wl.e_tilde).max()
    db = (rng.standard_normal(om_nf) + 1j * rng.standard_normal(om_nf)) * np.abs(wl.b_tilde).max()
    sv = np.std(np.r_[wl.particles.vx, wl.particles.vy, wl.particles.vz])
    tv = rng.standard_normal((n, 3)) * sv
    tr = rng.standard_normal((n, 3)) * 1e-3 * wl.mesh.h
    return de, db, tr, tv


def _oracle_jvp(wl, P, tet, K, de, db, tr, tv):
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    st = OracleState(P, tet)
    G = np.zeros(om.n_edges)
    tr, tv = tr.copy(), tv.copy()
    for k in range(K):
        t = k * wl.dt
        push_step_jvp(om, st, wl.e_tilde, wl.b_tilde, wl.amp(t), wl.omega0, t, wl.dt, G, tr, tv, de, db,
                      wall_mode=wl.wall_mode)
    return kinetic_energy_jvp(st, tv), st


def _gpu_grad(wl, P, prec, K, every):
    A, FempicEnv, ParticleState = _mods()
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st0 = ParticleState.from_host(P, prec)
    env.locate(st0)
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    sch = A.Schedule(wl.amp, wl.omega0, wl.dt, K, every)
    L, eg, bg, adj = A.kinetic_energy_and_grad(env, st0, e, b, sch)
    torch.cuda.synchronize()
    return env, st0, e, b, sch, float(L.item()), eg.cpu().numpy(), bg.cpu().numpy(), adj


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 1e-5)])
@pytest.mark.parametrize("maker,K,every", [(I.workload_small, 20, 6),
                                           (lambda: I.workload_hot_small(n_particles=80), 8, 3)])
def test_adjoint_matches_oracle_jvp(prec, tol, maker, K, every):
    A, _, _ = _mods()
    wl = maker()
    P = wl.particles.subset(min(wl.particles.n, 400))
    env, st0, e, b, sch, L, eg, bg, adj = _gpu_grad(wl, P, prec, K, every)
    tet0 = st0.tet.cpu().numpy()
    rng = np.random.default_rng(77)
    for trial in range(3):
        de, db, tr, tv = _directions(rng, wl, P.n, env.n_edges, env.n_faces)
        jv, ost = _oracle_jvp(wl, P, tet0, K, de, db, tr, tv)
        g = A.grad_dot(eg, bg, adj, de, db, tr, tv)
        print(f"\n[adjoint prec={prec} {wl.name}] <g,d> {g:.12e} jvp {jv:.12e} rel {abs(g - jv) / abs(jv):.2e}")
        assert abs(g - jv) <= tol * abs(jv)


def test_adjoint_matches_central_differences_fp64():
    """GPU FP64 gradient vs central differences of the GPU FP64 forward run."""
    A, FempicEnv, ParticleState = _mods()
    wl = I.workload_small()
    P = wl.particles.subset(500)
    K, every = 30, 7
    env, st0, e, b, sch, L, eg, bg, adj = _gpu_grad(wl, P, FP64, K, every)
    rng = np.random.default_rng(5)
    h = 1e-6
    for trial in range(4):
        de, db, tr, tv = _directions(rng, wl, P.n, env.n_edges, env.n_faces)
        g = A.grad_dot(eg, bg, adj, de, db, tr, tv)
        vals, seqs = [], []
        for sgn in (1, -1):
            Pp = I.Particles(P.x + sgn * h * tr[:, 0], P.y + sgn * h * tr[:, 1], P.z + sgn * h * tr[:, 2],
                             P.vx + sgn * h * tv[:, 0], P.vy + sgn * h * tv[:, 1], P.vz + sgn * h * tv[:, 2],
                             P.species_begin, P.q, P.m, P.w)
            st = ParticleState.from_host(Pp, FP64)
            st.tet.copy_(st0.tet)
            ep = torch.from_numpy(wl.e_tilde + sgn * h * de).cuda()
            bp = torch.from_numpy(wl.b_tilde + sgn * h * db).cuda()
            final, _ = A.forward_checkpointed(env, st, ep, bp, sch)
            vals.append(float(A.kinetic_energy(env, final).item()))
            seqs.append((final.tet.cpu().numpy(), final.n_cross.cpu().numpy()))
        assert np.array_equal(seqs[0][0], seqs[1][0]) and np.array_equal(seqs[0][1], seqs[1][1])
        fd = (vals[0] - vals[1]) / (2 * h)
        print(f"\n[adjoint vs FD] <g,d> {g:.10e} fd {fd:.10e} rel {abs(g - fd) / abs(fd):.2e}")
        assert abs(g - fd) <= 1e-5 * abs(fd)


def test_autograd_function_matches_driver():
    A, FempicEnv, ParticleState = _mods()
    wl = I.workload_small()
    P = wl.particles.subset(300)
    for prec in (FP64, MIXED):
        env, st0, e, b, sch, L, eg, bg, adj = _gpu_grad(wl, P, prec, 12, 5)
        ei = e.clone().requires_grad_(True)
        bi = b.clone().requires_grad_(True)
        ins = [t.clone().requires_grad_(True) for t in (st0.x, st0.y, st0.z, st0.vx, st0.vy, st0.vz)]
        Lt = A.KineticEnergyAfterSteps.apply(ei, bi, *ins, env, st0, sch)
        assert abs(float(Lt.item()) - L) <= 1e-12 * abs(L)
        (2.0 * Lt).backward()
        np.testing.assert_allclose(ei.grad.cpu().numpy(), 2.0 * eg.astype(ei.grad.cpu().numpy().dtype),
                                   rtol=1e-6, atol=1e-6 * np.abs(eg).max())
        np.testing.assert_allclose(ins[3].grad.cpu().numpy(), 2.0 * adj.vx.cpu().numpy(), rtol=1e-6,
                                   atol=1e-6 * float(adj.vx.abs().max()))


def test_adjoint_cavity48_subset_vs_oracle():
    """The 48^3 x 6 cube workload shape (5 eV, TE101 10 kV/m), K = 50 steps with
    checkpoints every 10, on a 20k-particle subset: GPU gradient (both forms)
    against the oracle's tangent on the same particles."""
    A, _, _ = _mods()
    wl = I.workload_adjoint48(n_particles=20_000)
    P = wl.particles
    K = wl.steps
    rng = np.random.default_rng(9)
    for prec, tol in ((FP64, 1e-12), (MIXED, 1e-5)):
        env, st0, e, b, sch, L, eg, bg, adj = _gpu_grad(wl, P, prec, K, 10)
        de, db, tr, tv = _directions(rng, wl, P.n, env.n_edges, env.n_faces)
        jv, _ = _oracle_jvp(wl, P, st0.tet.cpu().numpy(), K, de, db, tr, tv)
        g = A.grad_dot(eg, bg, adj, de, db, tr, tv)
        print(f"\n[adjoint cavity48 20k prec={prec}] rel {abs(g - jv) / abs(jv):.2e}")
        assert abs(g - jv) <= tol * abs(jv)
