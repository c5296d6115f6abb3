"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own formulas: hand-computed
values, closed forms (Boris rotation, Dirichlet sums, Gauss-Legendre path
integrals), exact integer incidence identities, brute-force point location
and brute-force segment/face intersection.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle.oracle import OracleMesh, OracleState, kinetic_energy, push_step, run, envelope_frame
from paper_2208_12795_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LE = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LF = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


@pytest.fixture(scope="module")
def cube4():
    m = I.kuhn_cube_mesh(4)
    return m, OracleMesh(m.nodes, m.tets)


@pytest.fixture(scope="module")
def cube4j():
    m = I.kuhn_cube_mesh(4, jitter=0.2, rng=np.random.default_rng(7))
    return m, OracleMesh(m.nodes, m.tets)


def _rand_point_in_tet(rng, X):
    w = rng.dirichlet(np.ones(4))
    return w @ X, w


# ------------------------------------------------------------------ golden
def test_reference_tet_golden():
    g = json.load(open(os.path.join(GOLDEN, "reference_tet_whitney.json")))
    nodes = np.array(g["nodes"], float)
    om = OracleMesh(nodes, np.array([[0, 1, 2, 3]], np.int32))
    r = np.array(g["point"])
    np.testing.assert_allclose(om.bary(0, r), g["lambda"], atol=1e-15)
    np.testing.assert_allclose(om.grad_bary(0), g["grad_lambda"], atol=0)
    np.testing.assert_allclose(om.whitney1(0, r), g["W1"], atol=1e-15)
    np.testing.assert_allclose(om.whitney2(0, r), g["W2"], atol=1e-15)


# -------------------------------------------------------------- barycentric
def test_bary_nodes_and_partition_of_unity(cube4j):
    m, om = cube4j
    tb = om.tables()
    rng = np.random.default_rng(1)
    for t in rng.choice(om.n_tets, 40, replace=False):
        X = m.nodes[tb["tet_nodes"][t]]
        for j in range(4):
            lam = om.bary(t, X[j])
            e = np.zeros(4); e[j] = 1
            np.testing.assert_allclose(lam, e, atol=1e-14)
        r, w = _rand_point_in_tet(rng, X)
        lam = om.bary(t, r)
        assert abs(lam.sum() - 1.0) < 1e-15
        np.testing.assert_allclose(lam, w, atol=1e-14)


def test_locate_grid_equals_brute(cube4, cube4j):
    rng = np.random.default_rng(3)
    for jittered, (m, om) in ((False, cube4), (True, cube4j)):
        pts = rng.random((3000, 3))
        # exact lattice points (shared by many tets: smallest id wins); on the
        # unjittered mesh every barycentric at a lattice point is exact in FP64
        if not jittered:
            pts[:50] = rng.integers(0, 5, size=(50, 3)) * 0.25
        tg, sg = om.locate(pts[:, 0], pts[:, 1], pts[:, 2])
        tb, sb = om.locate(pts[:, 0], pts[:, 1], pts[:, 2], brute=True)
        assert (tg == tb).all() and (tg >= 0).all()
        # smallest id among all containing tets, by an independent numpy scan
        X = m.nodes[np.sort(m.tets, axis=1)]
        A = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 2)
        Ainv = np.linalg.inv(A)
        for i in range(80):
            p = pts[i]
            l = np.einsum("tij,tj->ti", Ainv, p - X[:, 0])
            lam = np.c_[1 - l.sum(1), l]
            if not jittered:
                cont = np.nonzero(lam.min(1) >= -1e-12)[0]
                assert tg[i] == cont.min()
            else:
                assert lam[tg[i]].min() >= -1e-12
                assert not np.any(lam[:tg[i]].min(1) > 1e-12)
    # outside the mesh -> LOST
    m, om = cube4
    t, s = om.locate(np.array([1.5]), np.array([0.5]), np.array([0.5]))
    assert t[0] == -1 and s[0] == 4


# ------------------------------------------------------------------ Whitney
def test_whitney1_edge_circulations_are_kronecker(cube4j):
    m, om = cube4j
    tb = om.tables()
    gx, gw = np.polynomial.legendre.leggauss(20)
    s = 0.5 * (gx + 1); w = 0.5 * gw
    for t in (0, 17, 200, 383):
        X = m.nodes[tb["tet_nodes"][t]]
        for e2, (i, j) in enumerate(LE):
            d = X[j] - X[i]
            circ = sum(wk * om.whitney1(t, X[i] + sk * d) @ d for sk, wk in zip(s, w))
            e = np.zeros(6); e[e2] = 1
            np.testing.assert_allclose(circ, e, atol=1e-13)


def test_whitney2_face_fluxes_are_kronecker(cube4j):
    m, om = cube4j
    tb = om.tables()
    rng = np.random.default_rng(5)
    # W2 is affine, so its flux equals the mean over many random face points times the area vector
    for t in (0, 17, 200, 383):
        X = m.nodes[tb["tet_nodes"][t]]
        for f2, (i, j, l) in enumerate(LF):
            nA = 0.5 * np.cross(X[j] - X[i], X[l] - X[i])
            ws = rng.dirichlet(np.ones(3), size=64)
            pts = ws @ X[[i, j, l]]
            flux = np.mean([om.whitney2(t, p) @ nA for p in pts], axis=0)
            e = np.zeros(4); e[f2] = 1
            np.testing.assert_allclose(flux, e, atol=1e-13)


def test_constant_fields_reproduced(cube4j):
    m, om = cube4j
    tb = om.tables()
    rng = np.random.default_rng(9)
    Ec = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    Bc = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    en, fn = tb["edge_nodes"], tb["face_nodes"]
    e_dof = (m.nodes[en[:, 1]] - m.nodes[en[:, 0]]) @ Ec
    nA = 0.5 * np.cross(m.nodes[fn[:, 1]] - m.nodes[fn[:, 0]], m.nodes[fn[:, 2]] - m.nodes[fn[:, 0]])
    b_dof = nA @ Bc
    for t in rng.choice(om.n_tets, 30, replace=False):
        r, _ = _rand_point_in_tet(rng, m.nodes[tb["tet_nodes"][t]])
        Et, Bt = om.gather(t, r, e_dof, b_dof)
        np.testing.assert_allclose(Et, Ec, rtol=0, atol=1e-12 * np.abs(Ec).max())
        np.testing.assert_allclose(Bt, Bc, rtol=0, atol=1e-12 * np.abs(Bc).max())


def _shared_faces(om):
    tb = om.tables()
    nb = tb["tet_nbr"]
    out = []
    for t in range(om.n_tets):
        for k in range(4):
            if nb[t, k] > t:
                out.append((t, k, nb[t, k]))
    return tb, out


def test_tangential_and_normal_continuity(cube4j):
    m, om = cube4j
    tb, shared = _shared_faces(om)
    rng = np.random.default_rng(11)
    e_dof = rng.standard_normal(om.n_edges) + 1j * rng.standard_normal(om.n_edges)
    b_dof = rng.standard_normal(om.n_faces) + 1j * rng.standard_normal(om.n_faces)
    jumps_n = []
    for idx in rng.choice(len(shared), 60, replace=False):
        t1, k, t2 = shared[idx]
        fnodes = [tb["tet_nodes"][t1][i] for i in LF[k]]
        P = m.nodes[fnodes]
        n = np.cross(P[1] - P[0], P[2] - P[0]); n /= np.linalg.norm(n)
        p = rng.dirichlet(np.ones(3)) @ P
        E1, B1 = om.gather(t1, p, e_dof, b_dof)
        E2, B2 = om.gather(t2, p, e_dof, b_dof)
        sc = max(np.abs(E1).max(), 1.0)
        assert np.abs(np.cross(E1 - E2, n)).max() < 1e-12 * sc          # W1: tangential continuous
        assert abs(np.dot(B1 - B2, n)) < 1e-12 * max(np.abs(B1).max(), 1.0)  # W2: normal continuous
        jumps_n.append(abs(np.dot(E1 - E2, n)) / sc)
    assert max(jumps_n) > 1e-3   # the normal part of W1 does jump: the test is not vacuous


def test_de_rham_commuting_curl(cube4j):
    """curl(sum e W1) = sum (C e) W2 inside each tet (C = face circulation)."""
    m, om = cube4j
    tb = om.tables()
    rng = np.random.default_rng(13)
    e_dof = rng.standard_normal(om.n_edges)
    b_dof = om.face_circulation(e_dof)
    zero_b = np.zeros(om.n_faces)
    for t in rng.choice(om.n_tets, 20, replace=False):
        r, _ = _rand_point_in_tet(rng, m.nodes[tb["tet_nodes"][t]])
        dl = 1e-4
        J = np.zeros((3, 3))
        for a in range(3):
            dr = np.zeros(3); dr[a] = dl
            Ep, _ = om.gather(t, r + dr, e_dof, zero_b)
            Em, _ = om.gather(t, r - dr, e_dof, zero_b)
            J[:, a] = (Ep.real - Em.real) / (2 * dl)      # exact for affine fields up to rounding
        curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        _, Bt = om.gather(t, r, np.zeros(om.n_edges), b_dof)
        np.testing.assert_allclose(Bt.real, curl, atol=1e-8 * np.abs(curl).max())


def test_incidence_identities(cube4j):
    m, om = cube4j
    tb = om.tables()
    rng = np.random.default_rng(17)
    assert om.n_nodes - om.n_edges + om.n_faces - om.n_tets == 1
    # C D1 = 0: circulation of a discrete gradient vanishes exactly (integers)
    phi = rng.integers(-1000, 1000, om.n_nodes).astype(float)
    grad = phi[tb["edge_nodes"][:, 1]] - phi[tb["edge_nodes"][:, 0]]
    assert np.all(om.face_circulation(grad) == 0.0)
    # D2 C = 0: outward-signed sum of face circulations over each tet vanishes
    v = rng.integers(-1000, 1000, om.n_edges).astype(float)
    circ = om.face_circulation(v)
    X = m.nodes
    for t in range(om.n_tets):
        tn = tb["tet_nodes"][t]
        tot = 0.0
        for k in range(4):
            f = tb["tet_faces"][t, k]
            P = X[tb["face_nodes"][f]]
            nrm = np.cross(P[1] - P[0], P[2] - P[0])
            out = np.sign(nrm @ (P.mean(0) - X[tn[k]]))
            tot += out * circ[f]
        assert tot == 0.0
    # edge divergence: D^T of a unit edge value is -1 at its tail, +1 at its head
    G = np.zeros(om.n_edges); G[5] = 1.0
    d = om.edge_divergence(G)
    en = tb["edge_nodes"][5]
    assert d[en[1]] == 1.0 and d[en[0]] == -1.0 and np.abs(d).sum() == 2.0
    # wall codes: every boundary face lies in the bbox plane its code names
    for t in range(om.n_tets):
        for k in range(4):
            c = tb["tet_nbr"][t, k]
            if c < 0:
                ax, side = divmod(-1 - c, 2)
                P = X[tb["face_nodes"][tb["tet_faces"][t, k]]]
                assert np.all(P[:, ax] == (1.0 if side else 0.0))


# ----------------------------------------------------------------- deposit
def _single(x, v, q=-I.E_CHARGE, mass=I.M_ELECTRON, w=1e3):
    return I.Particles(np.array([x[0]]), np.array([x[1]]), np.array([x[2]]),
                       np.array([v[0]]), np.array([v[1]]), np.array([v[2]]),
                       np.array([0, 1], np.int64), np.array([q]), np.array([mass]), np.array([w]))


def _brute_pieces(m, om, a, b):
    """Brute-force segment a->b against every face: sorted crossing params and
    the tet containing each piece (by brute-force location of its midpoint)."""
    tb = om.tables()
    X = m.nodes
    ss = [0.0, 1.0]
    d = b - a
    for f in range(om.n_faces):
        P = X[tb["face_nodes"][f]]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        den = n @ d
        if abs(den) < 1e-300:
            continue
        s = n @ (P[0] - a) / den
        if not (1e-12 < s < 1 - 1e-12):
            continue
        p = a + s * d
        # inside-triangle test by barycentric areas
        A = np.stack([P[1] - P[0], P[2] - P[0]], 1)
        uv, *_ = np.linalg.lstsq(A, p - P[0], rcond=None)
        if uv.min() > 1e-9 and uv.sum() < 1 - 1e-9:
            ss.append(s)
    ss = sorted(ss)
    pieces = []
    for s0, s1 in zip(ss[:-1], ss[1:]):
        mid = a + 0.5 * (s0 + s1) * d
        pieces.append((s0, s1, om.locate_brute_one(mid)))
    return pieces


def test_tracking_and_deposit_vs_brute_force(cube4j):
    """Straight field-free segments through the jittered mesh: crossing count
    and final tet equal a brute-force segment/face intersection, and dG equals
    the 20-point Gauss-Legendre integral of q w W1 . dr over the pieces."""
    m, om = cube4j
    rng = np.random.default_rng(19)
    gx, gw = np.polynomial.legendre.leggauss(20)
    zero_e = np.zeros(om.n_edges, complex); zero_b = np.zeros(om.n_faces, complex)
    tb = om.tables()
    n_multi = 0
    for trial in range(25):
        a = 0.1 + 0.8 * rng.random(3)
        b = 0.1 + 0.8 * rng.random(3)
        dt = 1e-9
        v = (b - a) / dt
        P = _single(a, v)
        tet, _ = om.locate(P.x, P.y, P.z)
        st = OracleState(P, tet)
        dG = np.zeros(om.n_edges)
        push_step(om, st, zero_e, zero_b, 1.0, 0.0, 0.0, dt, dG)
        bb = a + dt * v               # the oracle's own rounding of b
        pieces = _brute_pieces(m, om, a, bb)
        assert st.status[0] == 0
        assert st.n_cross[0] == len(pieces) - 1
        assert st.tet[0] == pieces[-1][2]
        n_multi += len(pieces) > 2
        ref = np.zeros(om.n_edges)
        qw = P.q[0] * P.w[0]
        for s0, s1, t in pieces:
            pa, pb = a + s0 * (bb - a), a + s1 * (bb - a)
            seg = pb - pa
            for sk, wk in zip(0.5 * (gx + 1), 0.5 * gw):
                W = om.whitney1(t, pa + sk * seg)
                ref[tb["tet_edges"][t]] += qw * wk * (W @ seg)
        np.testing.assert_allclose(dG, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert n_multi > 10


def test_reflection_off_a_wall(cube4):
    m, om = cube4
    a = np.array([0.9, 0.37, 0.61]); v = np.array([2e8, 1e7, -3e7]); dt = 1e-9
    P = _single(a, v)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG)
    b = a + dt * v
    expect = b.copy(); expect[0] = 2.0 - b[0]
    got = np.array([st.x[0], st.y[0], st.z[0]])
    np.testing.assert_allclose(got, expect, atol=1e-15)
    np.testing.assert_allclose([st.vx[0], st.vy[0], st.vz[0]], [-v[0], v[1], v[2]], rtol=1e-15)
    assert st.tet[0] == om.locate(got[:1], got[1:2], got[2:])[0][0]
    # charge: D^T dG = q w (lambda(end) - lambda(start)) at the nodes
    rho0 = om.nodal_charge(P.x, P.y, P.z, tet, P.species_begin, P.q, P.w)
    rho1 = om.nodal_charge(st.x, st.y, st.z, st.tet, P.species_begin, P.q, P.w)
    np.testing.assert_allclose(om.edge_divergence(dG), rho1 - rho0, atol=1e-15 * abs(P.q[0] * P.w[0]))


def test_segments_ending_on_a_face_do_not_ping_pong(cube4j):
    """Segments from inside a tet to a point of one of its interior faces
    (on the face up to rounding), field free.  Either end of the rounding is
    correct, so each particle ends in that tet or in the neighbour across the
    face after at most one crossing, at the segment's end.  The entry face of
    the new tet is not a candidate exit (the tie rule): without it, a point
    that both tets' barycentrics put outside bounces between them up to the
    crossing cap."""
    m, om = cube4j
    tb = om.tables()
    nb, tn = tb["tet_nbr"], tb["tet_nodes"]
    rng = np.random.default_rng(5)
    dt = 1e-9
    xs, vs, home, other = [], [], [], []
    for t in range(om.n_tets):
        for k in range(4):
            if nb[t, k] < 0:
                continue
            X = m.nodes[[tn[t, i] for i in range(4) if i != k]]
            inner = m.nodes[tn[t]].mean(0)
            for _ in range(4):
                b = rng.dirichlet(np.ones(3)) @ X
                a = b + (inner - b) * rng.uniform(0.05, 0.5)
                xs.append(a); vs.append((b - a) / dt); home.append(t); other.append(nb[t, k])
    xs, vs = np.array(xs), np.array(vs)
    n = len(xs)
    P = I.Particles(*(np.ascontiguousarray(c) for c in (xs[:, 0], xs[:, 1], xs[:, 2], vs[:, 0], vs[:, 1], vs[:, 2])),
                    np.array([0, n], np.int64), np.array([-I.E_CHARGE]), np.array([I.M_ELECTRON]), np.array([1.0]))
    tet, _ = om.locate(P.x, P.y, P.z)
    assert np.array_equal(tet, home)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG,
              max_crossings=16)
    assert (st.status == 0).all() and st.n_cross.max() <= 1
    assert np.all((st.tet == home) | (st.tet == other))
    assert (st.n_cross == 1).sum() > n // 10 and (st.n_cross == 0).sum() > n // 10
    b = xs + dt * vs
    np.testing.assert_allclose(np.stack([st.x, st.y, st.z], 1), b, rtol=0, atol=1e-15)


@pytest.mark.parametrize("nodes,tets,code", [
    ([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], [[0, 1, 2, 3]], 2),                       # zero volume
    ([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0.2, 0.2, 1], [0.2, 0.2, -1], [0.3, 0.3, 0.5]],
     [[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], 3),                                          # face in 3 tets
])
def test_degenerate_and_nonconforming_meshes_rejected(nodes, tets, code):
    with pytest.raises(ValueError, match=f"code {code}"):
        OracleMesh(np.array(nodes, float), np.array(tets, np.int32))


def test_boundary_face_inside_the_box_absorbs_in_reflect_mode():
    """A mesh with a hole (one interior tet removed): the hole's faces are
    boundary faces off the bounding-box planes, so a particle reaching one
    is absorbed on it even with reflecting walls."""
    m = I.kuhn_cube_mesh(4)
    c_all = m.nodes[m.tets].mean(1)
    hole = int(np.argmin(np.linalg.norm(c_all - 0.5 + 0.01, axis=1)))
    tets = np.delete(m.tets, hole, axis=0)
    om = OracleMesh(m.nodes, tets)
    tb = om.tables()
    assert (tb["tet_nbr"] == -7).sum() == 4
    t_nb, k_nb = np.argwhere(tb["tet_nbr"] == -7)[0]
    a = m.nodes[tb["tet_nodes"][t_nb]].mean(0)
    face = m.nodes[[tb["tet_nodes"][t_nb][i] for i in range(4) if i != k_nb]].mean(0)
    dt = 1e-9
    v = 3.0 * (face - a) / dt                                        # well past the face, into the hole
    P = I.Particles(np.array([a[0]]), np.array([a[1]]), np.array([a[2]]), np.array([v[0]]), np.array([v[1]]),
                    np.array([v[2]]), np.array([0, 1], np.int64), np.array([-I.E_CHARGE]),
                    np.array([I.M_ELECTRON]), np.array([1.0]))
    tet, _ = om.locate(P.x, P.y, P.z)
    assert tet[0] == t_nb
    st = OracleState(P, tet)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt,
              np.zeros(om.n_edges), wall_mode=0)
    assert st.status[0] == 2 and st.tet[0] == -2 - t_nb
    lam = om.bary(t_nb, np.array([st.x[0], st.y[0], st.z[0]]))
    assert abs(lam[k_nb]) < 1e-14 and (lam > -1e-14).all()


def test_absorbing_wall_and_crossing_cap(cube4):
    m, om = cube4
    a = np.array([0.9, 0.37, 0.61]); v = np.array([2e8, 1e7, -3e7]); dt = 1e-9
    P = _single(a, v)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG,
              wall_mode=1)
    assert st.status[0] == 2 and st.tet[0] <= -2 and abs(st.x[0] - 1.0) < 1e-15
    # crossing cap: a long field-free segment with max_crossings = 1
    P = _single(np.array([0.1, 0.1, 0.1]), np.array([7e8, 6e8, 5e8]))
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG,
              max_crossings=1)
    assert st.status[0] == 1 and st.n_cross[0] == 2 and st.tet[0] <= -2
    # out-of-range tet id and non-finite velocity
    P = _single(np.array([0.5, 0.5, 0.5]), np.array([np.nan, 0.0, 0.0]))
    st = OracleState(P, np.array([om.n_tets + 5], np.int32))
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG)
    assert st.status[0] == 4 and st.tet[0] == -1
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    push_step(om, st, np.zeros(om.n_edges, complex), np.zeros(om.n_faces, complex), 1.0, 0.0, 0.0, dt, dG)
    assert st.status[0] == 3 and st.x[0] == 0.5


# ------------------------------------------------------------------- Boris
def _uniform_b_dofs(m, om, B):
    tb = om.tables()
    fn = tb["face_nodes"]
    nA = 0.5 * np.cross(m.nodes[fn[:, 1]] - m.nodes[fn[:, 0]], m.nodes[fn[:, 2]] - m.nodes[fn[:, 0]])
    return (nA @ np.asarray(B)).astype(complex)


def _uniform_e_dofs(m, om, E):
    tb = om.tables()
    en = tb["edge_nodes"]
    return ((m.nodes[en[:, 1]] - m.nodes[en[:, 0]]) @ np.asarray(E)).astype(complex)


def test_boris_gyration_closed_form(cube4):
    """Uniform B, E = 0, omega0 = 0: |v| invariant, v_perp turns by
    theta = 2 atan(|q B dt / 2m|) per step (counter-clockwise about +z for an
    electron), positions lie on the circle of radius dt|v_perp| / (2 sin(theta/2))."""
    m, om = cube4
    B0 = 1e-3
    b_dof = _uniform_b_dofs(m, om, [0, 0, B0])
    e_dof = np.zeros(om.n_edges, complex)
    dt = 0.5e-9
    v0 = np.array([1e6, 0.0, 2e3])
    P = _single(np.array([0.5, 0.5, 0.5]), v0)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    k = abs(P.q[0] / P.m[0]) * dt * 0.5
    theta = 2 * math.atan(k * B0)
    R = dt * np.hypot(*v0[:2]) / (2 * math.sin(theta / 2))
    vs, rs = [v0.copy()], [np.array([0.5, 0.5, 0.5])]
    for n in range(60):
        push_step(om, st, e_dof, b_dof, 1.0, 0.0, n * dt, dt, dG)
        vs.append(np.array([st.vx[0], st.vy[0], st.vz[0]]))
        rs.append(np.array([st.x[0], st.y[0], st.z[0]]))
    assert st.n_cross.sum() > 0          # the orbit crosses faces around the centre node
    vs = np.array(vs); rs = np.array(rs)
    np.testing.assert_allclose(np.linalg.norm(vs, axis=1), np.linalg.norm(v0), rtol=1e-14)
    np.testing.assert_allclose(vs[:, 2], v0[2], rtol=1e-14)
    ang = np.arctan2(vs[:-1, 0] * vs[1:, 1] - vs[:-1, 1] * vs[1:, 0],
                     vs[:-1, 0] * vs[1:, 0] + vs[:-1, 1] * vs[1:, 1])
    np.testing.assert_allclose(ang, theta, rtol=1e-12)
    # discrete circle: centre from the closed-form geometry of the first step
    # positions r_{n+1} = r_n + dt v_{n+1/2}; the chord r_n -> r_{n+1} subtends theta
    xy = rs[:, :2]
    c = np.mean(xy, axis=0)
    for _ in range(3):   # refine centre: least squares circle fit
        d = np.linalg.norm(xy - c, axis=1)
        A = np.c_[2 * xy, np.ones(len(xy))]
        sol, *_ = np.linalg.lstsq(A, (xy ** 2).sum(1), rcond=None)
        c = sol[:2]
    rad = np.linalg.norm(xy - c, axis=1)
    np.testing.assert_allclose(rad, R, rtol=1e-10)


def test_boris_uniform_e_with_carrier_dirichlet_sum(cube4):
    """Uniform E0 x_hat carried by cos(omega0 t): v_n = v_0 + (q dt/m) E0 sum_k cos(omega0 k dt)."""
    m, om = cube4
    E0 = 1e3
    e_dof = _uniform_e_dofs(m, om, [E0, 0, 0])
    b_dof = np.zeros(om.n_faces, complex)
    dt = 0.5e-9
    om0 = I.te101_omega0()
    P = _single(np.array([0.5, 0.5, 0.5]), np.zeros(3))
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    qm = P.q[0] / P.m[0]
    x = om0 * dt
    for n in range(1, 101):
        push_step(om, st, e_dof, b_dof, 1.0, om0, (n - 1) * dt, dt, dG)
        s = math.sin(n * x / 2) * math.cos((n - 1) * x / 2) / math.sin(x / 2)
        expect = qm * dt * E0 * s
        assert abs(st.vx[0] - expect) <= 1e-12 * abs(qm * dt * E0)
        assert st.vy[0] == 0.0 and st.vz[0] == 0.0


def test_boris_b_carrier_total_angle(cube4):
    """B = B0 z_hat cos(omega0 t): total turn angle = sum_n 2 atan(k B0 cos(omega0 t_n))."""
    m, om = cube4
    B0 = 5e-3
    b_dof = _uniform_b_dofs(m, om, [0, 0, B0])
    dt = 0.5e-9
    om0 = 2 * math.pi * 150e6
    v0 = np.array([3e5, 0.0, 0.0])
    P = _single(np.array([0.5, 0.5, 0.5]), v0)
    tet, _ = om.locate(P.x, P.y, P.z)
    st = OracleState(P, tet)
    dG = np.zeros(om.n_edges)
    k = abs(P.q[0] / P.m[0]) * dt * 0.5
    total = 0.0
    for n in range(40):
        push_step(om, st, np.zeros(om.n_edges, complex), b_dof, 1.0, om0, n * dt, dt, dG)
        total += 2 * math.atan(k * B0 * math.cos(om0 * n * dt))
    ang = math.atan2(st.vy[0], st.vx[0])
    assert abs(math.remainder(ang - total, 2 * math.pi)) < 1e-12
    assert abs(math.hypot(st.vx[0], st.vy[0]) - 3e5) < 1e-9


# ---------------------------------------------------------- conservation
@pytest.mark.parametrize("maker", [I.workload_small, I.workload_hot_small])
def test_charge_conservation_global(maker):
    """D^T G_cum = rho^n - rho^0 (Whitney-0 nodal charge) to machine precision."""
    wl = maker()
    om = OracleMesh(wl.mesh.nodes, wl.mesh.tets)
    P = wl.particles
    tet, st0 = om.locate(P.x, P.y, P.z)
    assert (st0 == 0).all()
    st = OracleState(P, tet)
    rho0 = om.nodal_charge(st.x, st.y, st.z, st.tet, st.species_begin, st.q, st.w)
    steps = min(wl.steps, 60)
    st, G = run(om, wl, st, steps)
    rho1 = om.nodal_charge(st.x, st.y, st.z, st.tet, st.species_begin, st.q, st.w)
    res = np.abs(om.edge_divergence(G) - (rho1 - rho0)).max() / np.abs(rho1).max()
    assert res < 1e-13
    assert (st.status == 0).all()


def test_envelope_frame_map():
    G = np.array([1.0, -2.0, 0.5])
    om0, t = 1.3e9, 7e-9
    out = envelope_frame(G, om0, t)
    np.testing.assert_allclose(out, G * np.exp(-1j * om0 * t), rtol=1e-15)


def test_kinetic_energy_closed_form():
    P = _single(np.array([0.5, 0.5, 0.5]), np.array([3.0, 4.0, 12.0]), mass=2.0, w=5.0)
    st = OracleState(P, np.array([0], np.int32))
    assert kinetic_energy(st) == 0.5 * 2.0 * 5.0 * 169.0


def test_te101_gather_converges_at_first_order():
    """Whitney-1/2 interpolation of the TE101 mode (de Rham DoFs) reproduces
    E = E0 sin(pi x) sin(pi z) y^ and B = (j/omega0) curl E with an error
    that halves with h (first order): RMS error over random points on Kuhn
    meshes of 8^3, 16^3 and 32^3 hexes."""
    E0 = 1e3
    om0 = I.te101_omega0()
    errs_e, errs_b = [], []
    for n in (8, 16, 32):
        m = I.kuhn_cube_mesh(n)
        om = OracleMesh(m.nodes, m.tets)
        tb = om.tables()
        e_dof, b_dof = I.te101_dofs(m.nodes, tb["edge_nodes"], tb["face_nodes"], E0, om0)
        rng = np.random.default_rng(100 + n)
        se, sb = [], []
        for t in rng.choice(om.n_tets, 400, replace=False):
            r, _ = _rand_point_in_tet(rng, m.nodes[tb["tet_nodes"][t]])
            Et, Bt = om.gather(t, r, e_dof, b_dof)
            x, _, z = r
            E = np.array([0.0, E0 * math.sin(math.pi * x) * math.sin(math.pi * z), 0.0])
            B = (1j / om0) * E0 * math.pi * np.array([-math.sin(math.pi * x) * math.cos(math.pi * z), 0.0,
                                                      math.cos(math.pi * x) * math.sin(math.pi * z)])
            se.append(np.sum(np.abs(Et - E) ** 2) / E0 ** 2)
            sb.append(np.sum(np.abs(Bt - B) ** 2) / (E0 * math.pi / om0) ** 2)
        errs_e.append(math.sqrt(np.mean(se)))
        errs_b.append(math.sqrt(np.mean(sb)))
    for errs in (errs_e, errs_b):
        assert 1.7 <= errs[0] / errs[1] <= 2.5 and 1.7 <= errs[1] / errs[2] <= 2.5, errs
