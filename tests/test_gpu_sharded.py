"""The sharded particle path (paper_2208_12795_gb300.shard) on the GPU: two
processes on one GPU, each advancing a contiguous tet range of one tet-sorted
load, all-reducing the step's edge deposit over gloo (host copies) and
adding it to G_cum with fempic_accumulate; the gradient windows (kinetic
energy, deposited current) with the loss and the DoF gradients summed over
the ranks.  G_cum, the envelope-frame G~ and the
gradients equal those of one process holding the whole load, to 1e-13 of
their maxima (summation order differs).  The processes' kernels never wait on
each other: the only exchange is the host-side all-reduce between steps."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 8


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _load():
    from paper_2208_12795_gb300 import inputs as I
    return I.te101_cavity(8, 20000, 50.0, 1e4, K, 21, dt=1e-9)


def _global_sorted(env, wl, prec):
    """The load sorted by tet, and each sorted particle's index in the load
    (carried through the sort in n_cross; the order inside a tet is
    unspecified)."""
    from paper_2208_12795_gb300.env import ParticleState
    st = ParticleState.from_host(wl.particles, prec)
    env.locate(st)
    st.n_cross.copy_(torch.arange(st.n, dtype=torch.int32, device="cuda"))
    scratch = st.empty_like()
    env.sort(st, scratch)
    ids = st.n_cross.cpu().numpy().copy()
    st.n_cross.zero_()
    return st, ids


def _run(env, st, wl, deposit):
    """K steps; deposit(omega0, t_next, G_cum_out, G_env_out) finalizes each."""
    Gc = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    Ge = torch.zeros(env.n_edges, dtype=torch.complex128, device="cuda")
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    for n in range(K):
        t = n * wl.dt
        env.push_step(st, e, b, wl.amp(t), wl.omega0, t, wl.dt)
        deposit(wl.omega0, t + wl.dt, Gc, Ge)
    return Gc.cpu().numpy(), Ge.cpu().numpy()


def _grad(env, st, wl, group=None, current=False):
    """Kinetic-energy loss, or (current) the deposited-current loss with
    seeded edge weights."""
    from paper_2208_12795_gb300 import adjoint as A
    e = torch.from_numpy(wl.e_tilde).to(env.dof_dtype).cuda()
    b = torch.from_numpy(wl.b_tilde).to(env.dof_dtype).cuda()
    sch = A.Schedule(wl.amp, wl.omega0, wl.dt, K, 3)
    if current:
        u = torch.from_numpy(np.random.default_rng(8).standard_normal(env.n_edges)).cuda()
        L, eg, bg, adj = A.current_loss_and_grad(env, A.clone_state(st), e, b, sch, u, group=group)
    else:
        L, eg, bg, adj = A.kinetic_energy_and_grad(env, st, e, b, sch, group=group)
    return float(L.item()), eg.cpu().numpy(), bg.cpu().numpy(), adj.vx.cpu().numpy().astype(np.float64)


def _worker(rank, world, port, prec, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2208_12795_gb300 import build, shard
    from paper_2208_12795_gb300.env import FempicEnv
    build.build()
    wl = _load()
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    mine = shard.tet_range(_global_sorted(env, wl, prec)[0], rank, world)
    sd = shard.ShardedDeposit(env)
    Gc, Ge = _run(env, mine, wl, lambda om, t1, gc, ge: sd(om, t1, G_cum_out=gc, G_env_out=ge))
    st2, ids = _global_sorted(env, wl, prec)
    n = st2.n
    a, b = rank * n // world, (rank + 1) * n // world
    mine2 = shard.tet_range(st2, rank, world)
    cur = _grad(env, mine2, wl, group=dist.group.WORLD, current=True)
    L, eg, bg, av = _grad(env, mine2, wl, group=dist.group.WORLD)
    torch.cuda.synchronize()
    q.put((rank, Gc, Ge, L, eg, bg, (ids[a:b], av), cur[:3]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("prec", [0, 1])
def test_two_processes_equal_one(prec):
    import torch.multiprocessing as mp
    from paper_2208_12795_gb300 import build
    from paper_2208_12795_gb300.env import FempicEnv
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, prec, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict()
    for _ in range(2):
        r = q.get(timeout=600)
        got[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # one process, the whole load
    wl = _load()
    env = FempicEnv.from_mesh(wl.mesh, precision=prec)
    st, _ = _global_sorted(env, wl, prec)
    Gc, Ge = _run(env, st, wl, lambda om, t1, gc, ge: env.deposit(om, t1, G_cum_out=gc, G_env_out=ge))
    st2, ids = _global_sorted(env, wl, prec)
    cur = _grad(env, st2, wl, current=True)
    L, eg, bg, av = _grad(env, st2, wl)
    (Gc0, Ge0, L0, eg0, bg0, av0, cur0), (Gc1, Ge1, L1, eg1, bg1, av1, cur1) = got[0], got[1]
    tol = 1e-13
    for a in (Gc0, Gc1):
        assert np.abs(a - Gc).max() <= tol * np.abs(Gc).max()
    for a in (Ge0, Ge1):
        assert np.abs(a - Ge).max() <= tol * np.abs(Ge).max()
    gtol = 1e-12 if prec == 0 else 1e-6
    assert abs(L0 - L) <= 1e-13 * abs(L) and L0 == L1
    for a, ref in ((eg0, eg), (eg1, eg), (bg0, bg), (bg1, bg)):
        assert np.abs(a - ref).max() <= gtol * np.abs(ref).max()
    n = wl.particles.n
    ref = np.zeros(n)
    ref[ids] = av                                   # the whole run's vbar_x, in load order
    got_v = np.full(n, np.nan)
    for sid, sv in (av0, av1):
        got_v[sid] = sv
    assert not np.isnan(got_v).any() and len(av0[0]) == n // 2 and len(av1[0]) == n - n // 2
    assert np.abs(got_v - ref).max() <= gtol * np.abs(ref).max()
    # the deposited-current loss: L and the DoF gradients summed over the ranks
    for c in (cur0, cur1):
        assert abs(c[0] - cur[0]) <= 1e-12 * abs(cur[0])
        for a, ref in ((c[1], cur[1]), (c[2], cur[2])):
            assert np.abs(a - ref).max() <= gtol * np.abs(ref).max()
    print(f"\n[sharded x2 prec={prec}] G_cum {np.abs(Gc0 - Gc).max() / np.abs(Gc).max():.2e}  "
          f"G~ {np.abs(Ge0 - Ge).max() / np.abs(Ge).max():.2e}  e-grad {np.abs(eg0 - eg).max() / np.abs(eg).max():.2e}")
