"""Pins of the seeded input generators (mesh, numbering, prescribed envelopes)."""
import math

import numpy as np
import pytest

from paper_2208_12795_gb300 import inputs as I


@pytest.mark.parametrize("n", [1, 2, 4, 7])
def test_kuhn_counts_and_volumes(n):
    m = I.kuhn_cube_mesh(n)
    _, e, f, te, tf = I.mesh_topology(m.tets)
    c = I.kuhn_counts(n)
    assert (m.n_nodes, len(e), len(f), m.n_tets) == (c["n_nodes"], c["n_edges"], c["n_faces"], c["n_tets"])
    X = m.nodes[m.tets]
    vol = np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0])) / 6
    assert np.allclose(np.abs(vol), m.h ** 3 / 6) and abs(np.abs(vol).sum() - 1.0) < 1e-12
    # every face is in 1 (boundary) or 2 tets; boundary count 12 n^2
    cnt = np.bincount(tf.ravel(), minlength=len(f))
    assert set(np.unique(cnt)) <= {1, 2} and (cnt == 1).sum() == c["n_boundary_faces"]


def test_jittered_mesh_valid():
    m = I.kuhn_cube_mesh(8, jitter=0.2, rng=np.random.default_rng(0))
    X = m.nodes[m.tets]
    vol = np.einsum("ij,ij->i", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0])) / 6
    assert np.abs(vol).min() > 0.05 * m.h ** 3 / 6
    assert abs(np.abs(vol).sum() - 1.0) < 1e-12          # still tiles the unit cube
    b = np.any((m.nodes == 0.0) | (m.nodes == 1.0), axis=1)
    assert np.all(m.nodes[b] * 8 == np.round(m.nodes[b] * 8))  # boundary nodes unmoved


def test_te101_edge_dofs_vs_gauss_legendre():
    m = I.kuhn_cube_mesh(5, jitter=0.2, rng=np.random.default_rng(1))
    _, e, f, _, _ = I.mesh_topology(m.tets)
    p0, p1 = m.nodes[e[:, 0]], m.nodes[e[:, 1]]
    analytic = I.te101_edge_circulation(p0, p1, 1e3)
    gx, gw = np.polynomial.legendre.leggauss(16)
    s = 0.5 * (gx + 1); w = 0.5 * gw
    quad = np.zeros(len(e))
    for sk, wk in zip(s, w):
        p = p0 + sk * (p1 - p0)
        Ey = 1e3 * np.sin(math.pi * p[:, 0]) * np.sin(math.pi * p[:, 2])
        quad += wk * Ey * (p1 - p0)[:, 1]
    assert np.abs(analytic - quad).max() <= 1e-14 * np.abs(analytic).max()


def test_te101_face_dofs_divergence_free_and_flux():
    m = I.kuhn_cube_mesh(4)
    ts, e, f, te, tf = I.mesh_topology(m.tets)
    om0 = I.te101_omega0()
    et, bt = I.te101_dofs(m.nodes, e, f, 1e3, om0)
    assert np.all(et.imag == 0) and np.all(bt.real == 0)
    # outward-signed face fluxes sum to zero in every tet (div B = 0)
    X = m.nodes
    fn = f[tf]                                   # [Nt,4,3]
    P = X[fn]
    nrm = np.cross(P[:, :, 1] - P[:, :, 0], P[:, :, 2] - P[:, :, 0])
    opp = X[ts]                                  # face k opposite sorted node k
    sgn = np.sign(np.einsum("tkc,tkc->tk", nrm, P.mean(2) - opp))
    div = np.abs((sgn * bt[tf].imag).sum(1)).max()
    assert div <= 1e-15 * np.abs(bt).max() * 4
    # flux of the analytic B = (j/omega0) curl E through a face vs the DoF (midpoint-rich quadrature)
    rng = np.random.default_rng(2)
    for fi in rng.choice(len(f), 20, replace=False):
        Pf = X[f[fi]]
        nA = 0.5 * np.cross(Pf[1] - Pf[0], Pf[2] - Pf[0])
        ws = rng.dirichlet(np.ones(3), size=20000)
        q = ws @ Pf
        curl = 1e3 * math.pi * np.c_[-np.sin(math.pi * q[:, 0]) * np.cos(math.pi * q[:, 2]),
                                     np.zeros(len(q)),
                                     np.cos(math.pi * q[:, 0]) * np.sin(math.pi * q[:, 2])]
        flux = (curl @ nA).mean() / om0
        assert abs(flux - bt[fi].imag) <= 2e-2 * np.abs(bt).max()


def test_omega0_te101():
    assert abs(I.te101_omega0() / (2 * math.pi) - 211.985e6) < 1e3


def test_envelope_ramp():
    s = 20e-9
    assert I.envelope_ramp(3 * s, s) == 1.0 and I.envelope_ramp(10 * s, s) == 1.0
    assert abs(I.envelope_ramp(0.0, s) - math.exp(-4.5)) < 1e-15
    assert abs(I.envelope_ramp(6 * s, s, centered=True) - 1.0) < 1e-15


def test_seeded_loads_reproducible():
    a = I.workload_small().particles
    b = I.workload_small().particles
    assert np.array_equal(a.x, b.x) and np.array_equal(a.vz, b.vz)
    sig = I.thermal_sigma(1.0, I.M_ELECTRON)
    assert abs(np.std(np.r_[a.vx, a.vy, a.vz]) / sig - 1) < 0.05


def test_complex_gradient_convention_matches_torch():
    """For real L of complex z, torch's gradient is dL/dRe + j dL/dIm: for
    L = |z|^2 that is 2z, the convention the adjoint returns."""
    torch = pytest.importorskip("torch")
    z = torch.tensor([1.5 - 2.0j, -0.25 + 0.5j], dtype=torch.complex128, requires_grad=True)
    (z.abs() ** 2).sum().backward()
    assert torch.allclose(z.grad, 2 * z.detach())
