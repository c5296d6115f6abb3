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
    for trial in range(8):
        de, db, tr, tv = _directions(rng, wl, P.n, env.n_edges, env.n_faces)
        jv, ost = _oracle_jvp(wl, P, tet0, K, de, db, tr, tv)
        g = A.grad_dot(eg, bg, adj, de, db, tr, tv)
        print(f"\n[adjoint prec={prec} {wl.name}] <g,d> {g:.12e} jvp {jv:.12e} rel {abs(g - jv) / abs(jv):.2e}")
        assert abs(g - jv) <= tol * abs(jv)


def test_adjoint_matches_central_differences_fp64():
    """GPU FP64 gradient vs central differences of the GPU FP64 forward run on
    64 random directions of (e~, b~, r0, v0).  The derivative is that of the
    map for a fixed tet sequence: a direction whose +h and -h runs take
    different sequences is retried with h/10 and, if they still differ,
    left out and counted (at most 2 of 64 allowed)."""
    A, FempicEnv, ParticleState = _mods()
    wl = I.workload_small()
    P = wl.particles.subset(500)
    K, every = 30, 7
    env, st0, e, b, sch, L, eg, bg, adj = _gpu_grad(wl, P, FP64, K, every)
    rng = np.random.default_rng(5)

    def run(h, de, db, tr, tv):
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
            # the checkpoint sorts may order particles of one tet differently:
            # compare the sorted (tet, crossings) pairs
            seqs.append(np.sort(final.tet.cpu().numpy().astype(np.int64) * 2 ** 32 + final.n_cross.cpu().numpy()))
        return (vals[0] - vals[1]) / (2 * h), np.array_equal(seqs[0], seqs[1])

    excluded, worst = 0, 0.0
    for trial in range(64):
        de, db, tr, tv = _directions(rng, wl, P.n, env.n_edges, env.n_faces)
        g = A.grad_dot(eg, bg, adj, de, db, tr, tv)
        fd, same = run(1e-6, de, db, tr, tv)
        if not same:
            fd, same = run(1e-7, de, db, tr, tv)
        if not same:
            excluded += 1
            continue
        rel = abs(g - fd) / abs(fd)
        worst = max(worst, rel)
        assert rel <= 1e-5, (trial, g, fd)
    print(f"\n[adjoint vs FD, 64 directions] worst rel {worst:.2e}, excluded {excluded}")
    assert excluded <= 2


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


def test_sort_perm_and_adjoint_unpermute_are_inverse():
    from paper_2208_12795_gb300 import capi
    A, FempicEnv, ParticleState = _mods()
    wl = I.workload_hot_small(n_particles=3000)
    for prec in (FP64, MIXED):
        env = FempicEnv.from_mesh(wl.mesh, precision=prec)
        st = ParticleState.from_host(wl.particles, prec)
        env.locate(st)
        out = st.empty_like()
        perm = torch.empty(st.n, dtype=torch.int32, device="cuda")
        env.sort_perm(st, out, perm)
        pi = perm.long()
        assert torch.equal(torch.sort(pi).values, torch.arange(st.n, device="cuda"))
        for k in ("x", "y", "z", "vx", "vy", "vz", "tet", "status"):
            assert torch.equal(getattr(out, k), getattr(st, k)[pi]), k
        t = out.tet.cpu().numpy()
        assert np.all(np.diff(t) >= 0)
        vdt = torch.float64 if prec == FP64 else torch.float32
        a, b = A.AdjointState(st.n, vdt), A.AdjointState(st.n, vdt)
        for k in ("rx", "ry", "rz", "vx", "vy", "vz"):
            getattr(a, k).copy_(torch.randn(st.n, device="cuda", dtype=getattr(a, k).dtype))
        capi.fempic_adjoint_unpermute(env.h, a.cstruct(), b.cstruct(), perm.data_ptr())
        torch.cuda.synchronize()
        for k in ("rx", "ry", "rz", "vx", "vy", "vz"):
            assert torch.equal(getattr(b, k)[pi], getattr(a, k)), k


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 2e-6)])
def test_gradient_with_checkpoint_sorts_equals_unsorted(prec, tol):
    """Sorting at every checkpoint reorders the work, not the map: L and the
    gradient (returned in the initial order) agree with the unsorted run."""
    A, FempicEnv, ParticleState = _mods()
    wl = I.workload_hot_small(n_particles=400)
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st0 = ParticleState.from_host(wl.particles, prec)
    env.locate(st0)
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    sch = A.Schedule(wl.amp, wl.omega0, wl.dt, 9, 3)
    vdt = torch.float64 if prec == FP64 else torch.float32
    res = []
    for sort in (False, True):
        final, ck = A.forward_checkpointed(env, st0, e, b, sch, sort=sort)
        adj = A.AdjointState(st0.n, vdt)
        L = float(A.kinetic_energy(env, final, seed=adj).item())
        eg, bg = A.reverse_sweep(env, ck, e, b, sch, adj)
        torch.cuda.synchronize()
        res.append((L, eg.cpu().numpy(), bg.cpu().numpy(), adj.vx.cpu().numpy().astype(np.float64),
                    adj.rz.cpu().numpy()))
    (L0, e0, b0, v0, r0), (L1, e1, b1, v1, r1) = res
    assert abs(L1 - L0) <= 1e-12 * abs(L0)
    np.testing.assert_allclose(e1, e0, rtol=0, atol=tol * np.abs(e0).max())
    np.testing.assert_allclose(b1, b0, rtol=0, atol=tol * np.abs(b0).max())
    np.testing.assert_allclose(v1, v0, rtol=0, atol=tol * np.abs(v0).max())
    np.testing.assert_allclose(r1, r0, rtol=0, atol=tol * np.abs(r0).max())
