"""Multi-rank path on CPU: particles sharded over 2 gloo ranks, each rank runs
its shard, the per-step edge deposit dG is summed with the package's
all-reduce (paper_2208_12795_gb300.shard.allreduce_, the one exchange step of
the particle path), and the result equals the unsharded run up to summation
order.  The oracle stands in for each rank's device work so the test runs
without a GPU.  Shards: contiguous ranges of the tet-sorted load, and the
benchmark's z-slab shares of a uniform load (shard.slab_load).  Both the
Boris step and the downshifted step (Sec. III-D, whose per-particle history
stays with the rank that owns the particle) are covered."""
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
    from paper_2208_12795_gb300 import shard
    wl = I.workload_hot_small(n_particles=400, steps=6)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles
    tet_all, _ = om.locate(P.x, P.y, P.z)
    order = np.argsort(tet_all, kind="stable")      # the tet-sorted load
    n = P.n
    lo, hi = rank * n // world, (rank + 1) * n // world
    idx = order[lo:hi]                               # this rank's contiguous tet range
    sub = I.Particles(P.x[idx], P.y[idx], P.z[idx], P.vx[idx], P.vy[idx], P.vz[idx],
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
        shard.allreduce_(t)
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


def test_slab_shares_form_a_uniform_global_load():
    """shard.slab_load: the ranks' shares of a uniform load are disjoint
    z-slabs whose union is uniform over the cube (world x the particles), and
    on a Kuhn cube with a multiple of `world` cells along z each slab's
    particles lie in one contiguous range of tet ids."""
    from oracle.oracle import OracleMesh
    from paper_2208_12795_gb300 import inputs as I, shard
    wl = I.te101_cavity(8, 4000, 5.0, 1e3, 1, 9)
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    world = 4
    ranges = []
    zs = []
    for r in range(world):
        p = shard.slab_load(wl.particles, r, world)
        assert np.array_equal(p.x, wl.particles.x) and np.array_equal(p.vz, wl.particles.vz)
        assert (p.z >= r / world).all() and (p.z < (r + 1) / world).all()
        tet, _ = om.locate(p.x, p.y, p.z)
        assert (tet >= 0).all()
        ranges.append((tet.min(), tet.max()))
        zs.append(p.z)
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 < b0                                 # disjoint, increasing tet ranges
    counts, _ = np.histogram(np.concatenate(zs), bins=16, range=(0.0, 1.0))
    assert counts.min() > 0.8 * counts.mean()          # uniform along z overall
    assert shard.slab_load(wl.particles, 0, 1) is wl.particles
