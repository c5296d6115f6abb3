"""Multi-rank path on CPU: particles sharded over 2 gloo ranks, each rank runs
its shard, the per-step edge deposit dG is summed with all_reduce (the one
exchange step of the particle path), and the result equals the unsharded
run up to summation order.  The oracle stands in for each rank's device work
so the test runs without a GPU; the collective logic is the benchmark's.
Both the Boris step and the downshifted step (Sec. III-D, whose per-particle
history stays with the rank that owns the particle) are covered."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q, mode="boris"):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.oracle import OracleMesh, OracleState, push_step
    from paper_2208_12795_gb300 import inputs as I
    wl = I.workload_hot_small(n_particles=400, steps=6)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles
    n = P.n
    lo, hi = rank * n // world, (rank + 1) * n // world
    sub = I.Particles(P.x[lo:hi], P.y[lo:hi], P.z[lo:hi], P.vx[lo:hi], P.vy[lo:hi], P.vz[lo:hi],
                      np.array([0, hi - lo], np.int64), P.q, P.m, P.w)
    tet, _ = om.locate(sub.x, sub.y, sub.z)
    st = OracleState(sub, tet)
    G = torch.zeros(om.n_edges, dtype=torch.float64)
    if mode == "downshift":
        from oracle.downshift import History, push_step_downshift
        hist = History(st.n)
    for k in range(wl.steps):
        dG = np.zeros(om.n_edges)
        if mode == "downshift":
            push_step_downshift(om, st, hist, wl.e_tilde, wl.b_tilde, wl.amp(k * wl.dt), wl.omega0, k * wl.dt,
                                wl.dt, dG)
        else:
            push_step(om, st, wl.e_tilde, wl.b_tilde, wl.amp(k * wl.dt), wl.omega0, k * wl.dt, wl.dt, dG)
        t = torch.from_numpy(dG)
        dist.all_reduce(t)
        G += t
    if rank == 0:
        q.put(G.numpy().copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("mode", ["boris", "downshift"])
def test_two_rank_dG_allreduce_equals_unsharded(mode):
    from oracle.downshift import History, push_step_downshift
    from oracle.oracle import OracleMesh, OracleState, run
    from paper_2208_12795_gb300 import inputs as I
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    G_sharded = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = I.workload_hot_small(n_particles=400, steps=6)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    tet, _ = om.locate(wl.particles.x, wl.particles.y, wl.particles.z)
    if mode == "downshift":
        st = OracleState(wl.particles, tet)
        hist = History(st.n)
        G = np.zeros(om.n_edges)
        for k in range(wl.steps):
            push_step_downshift(om, st, hist, wl.e_tilde, wl.b_tilde, wl.amp(k * wl.dt), wl.omega0, k * wl.dt,
                                wl.dt, G)
    else:
        _, G = run(om, wl, OracleState(wl.particles, tet), wl.steps)
    assert np.abs(G).max() > 0
    assert np.abs(G_sharded - G).max() <= 1e-13 * np.abs(G).max()
