"""The FP32-mixed forms against the FP64 oracle on identical segment
endpoints.

With a zero field the FP32 Boris step returns the velocity unchanged, and
with a step dt = 2^-31 s (a power of two) the mixed position update
b = a + f64(fl32(dt v)) equals the oracle's FP64 b = a + dt v bit for bit.
Both sides then track and deposit exactly the same straight segments, so
what is compared is the tracking (Sec. III-D's per-tet path split) and the
deposit (Sec. II eq. g_def, Sec. III-D eq. G_integral) alone:

* contract form (FEMPIC_MIXED): tet ids, crossing counts, statuses and
  positions bit-exact, except the crossing points where particles froze:
  those are a0 + S (b - a0) with the path fraction S accumulated in
  double-float over the walk's exit parameters, within 1e-13 m of the
  oracle's FP64 point; the accumulated G within 1e-12 of its maximum;
* 24-bit form (FEMPIC_MIXED_Q24): the same walk on 24-bit barycentrics, G
  within its resolution (2^-24 of a tet per segment).

Both conserve charge, D^T G = rho^n - rho^0, to <= 1e-13 of max |rho|.
"""
import numpy as np
import pytest

from oracle.oracle import OracleMesh, OracleState, push_step as oracle_push
from paper_2208_12795_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MIXED, Q24 = 1, 2
DT = 2.0 ** -31


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2208_12795_gb300 import build
    build.build()


def _fast_particles(n, speed, seed, mesh_lo=0.0, mesh_hi=1.0):
    """Uniform positions, isotropic directions, FP32-exact velocities of
    about `speed` (several face crossings per step at DT)."""
    rng = np.random.default_rng(seed)
    pos = rng.uniform(mesh_lo, mesh_hi, size=(n, 3))
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    v = (d * speed * rng.uniform(0.2, 1.0, size=(n, 1))).astype(np.float32).astype(np.float64)
    return I.Particles(pos[:, 0], pos[:, 1], pos[:, 2], v[:, 0], v[:, 1], v[:, 2], np.array([0, n], np.int64),
                       np.array([-I.E_CHARGE]), np.array([I.M_ELECTRON]), np.array([1e3]))


def _divergence(edges, nn, G):
    out = np.zeros(nn)
    np.add.at(out, edges[:, 1], G)
    np.subtract.at(out, edges[:, 0], G)
    return out


def _run_both(mesh, parts, prec, steps, wall_mode=0, max_crossings=4096):
    from paper_2208_12795_gb300.env import FempicEnv, ParticleState
    _, edges, faces, _, _ = I.mesh_topology(mesh.tets)
    rng = np.random.default_rng(4)
    e_t = rng.standard_normal(len(edges)) + 1j * rng.standard_normal(len(edges))   # zero amplitude below
    b_t = rng.standard_normal(len(faces)) + 1j * rng.standard_normal(len(faces))
    env = FempicEnv.from_mesh(mesh, precision=prec, wall_mode=wall_mode, max_crossings=max_crossings)
    st = ParticleState.from_host(parts, prec)
    env.locate(st)
    e = torch.from_numpy(e_t).to(env.dof_dtype).cuda()
    b = torch.from_numpy(b_t).to(env.dof_dtype).cuda()
    om = OracleMesh(mesh.nodes, mesh.tets, mesh.lo, mesh.hi)
    tet0, _ = om.locate(parts.x, parts.y, parts.z)
    ost = OracleState(parts, tet0)
    rho0 = om.nodal_charge(ost.x, ost.y, ost.z, ost.tet, ost.species_begin, ost.q, ost.w)
    grho0 = env.nodal_charge(st).cpu().numpy()
    oG = np.zeros(om.n_edges)
    G = torch.zeros(env.n_edges, dtype=torch.float64, device="cuda")
    omega0 = 1.3e9
    for n in range(steps):
        env.push_step(st, e, b, 0.0, omega0, n * DT, DT)
        env.deposit(omega0, (n + 1) * DT, G_cum_out=G)
        oracle_push(om, ost, e_t, b_t, 0.0, omega0, n * DT, DT, oG, max_crossings=max_crossings,
                    wall_mode=wall_mode)
    grho1 = env.nodal_charge(st).cpu().numpy()
    torch.cuda.synchronize()
    g = st.to_numpy()
    Gg = G.cpu().numpy()
    res = np.abs(_divergence(edges, env.n_nodes, Gg) - (grho1 - grho0)).max() / np.abs(grho1).max()
    return g, ost, Gg, oG, res


CASES = [
    # (name, mesh, speed, wall_mode, max_crossings, steps)
    ("jittered6_reflect", lambda: I.kuhn_cube_mesh(6, jitter=0.2, rng=np.random.default_rng(31)), 6e8, 0, 4096, 12),
    ("cube8_reflect", lambda: I.kuhn_cube_mesh(8), 2e8, 0, 4096, 12),
    ("jittered6_absorb", lambda: I.kuhn_cube_mesh(6, jitter=0.2, rng=np.random.default_rng(32)), 6e8, 1, 4096, 4),
    ("jittered6_cap", lambda: I.kuhn_cube_mesh(6, jitter=0.2, rng=np.random.default_rng(33)), 9e8, 0, 2, 3),
]


@pytest.mark.parametrize("name,mk,speed,wall,cap,steps", CASES, ids=[c[0] for c in CASES])
def test_contract_form_identical_endpoints(name, mk, speed, wall, cap, steps):
    mesh = mk()
    parts = _fast_particles(20000, speed, 7)
    g, ost, G, oG, res = _run_both(mesh, parts, MIXED, steps, wall_mode=wall, max_crossings=cap)
    frozen = ost.status != 0
    print(f"\n[contract {name}] crossings/particle-step {ost.n_cross.mean() / steps:.2f}  frozen {frozen.sum()}  "
          f"tets differ {(g['tet'] != ost.tet).sum()}  G err {np.abs(G - oG).max() / np.abs(oG).max():.2e}  "
          f"conservation {res:.2e}")
    assert ost.n_cross.mean() > 0.5 * steps
    assert np.array_equal(g["tet"], ost.tet)
    assert np.array_equal(g["n_cross"], ost.n_cross)
    assert np.array_equal(g["status"], ost.status)
    for k in ("x", "y", "z"):
        assert np.array_equal(g[k][~frozen], getattr(ost, k)[~frozen]), k
        assert np.abs(g[k][frozen] - getattr(ost, k)[frozen]).max(initial=0.0) <= 1e-13, k
    for k in ("vx", "vy", "vz"):
        assert np.array_equal(g[k].astype(np.float64), getattr(ost, k)), k
    assert np.abs(G - oG).max() <= 1e-12 * np.abs(oG).max()
    assert res <= 1e-13
    if wall == 1:
        assert (ost.status == 2).sum() > 1000
    if cap < 10:
        assert (ost.status == 1).sum() > 1000


def test_q24_form_identical_endpoints():
    mesh = I.kuhn_cube_mesh(6, jitter=0.2, rng=np.random.default_rng(31))
    parts = _fast_particles(20000, 6e8, 7)
    steps = 6
    g, ost, G, oG, res = _run_both(mesh, parts, Q24, steps)
    same = (g["tet"] == ost.tet).mean()
    err = np.abs(G - oG).max() / np.abs(oG).max()
    print(f"\n[q24 identical endpoints] tet agree {same:.6f}  G err {err:.2e}  conservation {res:.2e}")
    assert same >= 0.999
    # per crossing piece the 24-bit barycentrics place the end within ~2^-24
    # of a tet: relative to max |G| after 6 steps of ~4 pieces, below 1e-5
    assert err <= 1e-5
    assert res <= 1e-13
