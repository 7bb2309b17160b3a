"""Pins of the oracle's discretisation (Sec. II.A) against facts fixed by the
mathematics, not by the oracle itself: exact incidence identities, Euler
characteristic, reproduction of uniform fields by Whitney forms, the
commuting diagram curl W1 -> W2, brute-force quadrature of the Hodge
matrices with an independent formula for W2, the direct curl-curl stiffness,
and the textbook P1 Laplacian.
"""
import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.fixture(scope="module")
def cube6(oracle_lib):
    wl = W.kuhn_box((6, 6, 6), (1.0, 1.0, 1.0))
    return wl, oracle_lib.OracleMesh(wl.xyz, wl.tets)


@pytest.fixture(scope="module")
def jittered4(oracle_lib):
    wl = W.kuhn_box((4, 3, 5), (0.4, 0.3, 0.5), jitter=0.2, seed=7)
    return wl, oracle_lib.OracleMesh(wl.xyz, wl.tets)


# ---- the test's own geometry (independent of the oracle's formulas) ----
def bary_matrix(xyz, tet):
    """4x4 matrix T with T @ [1, x, y, z] = lambda (inverse of the vertex matrix)."""
    V = np.ones((4, 4))
    V[1:, :] = xyz[tet].T
    return np.linalg.inv(V)


def lam_at(T, r):
    return T @ np.concatenate([[1.0], r])


def grads(T):
    return T[:, 1:]                       # row k = grad lambda_k


def rt0(xyz, tet, local_face, r, face_nodes):
    """Whitney-2 / RT0 function of the face opposite local vertex k in its
    global orientation: (r - x_k)/(3V) times +-1 (outward normal vs face order)."""
    x = xyz[tet]
    vol6 = np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]]))
    V = abs(vol6) / 6.0
    xa, xb, xc = xyz[face_nodes]
    n = np.cross(xb - xa, xc - xa)
    out = np.dot(n, xa - x[local_face]) > 0
    return (1.0 if out else -1.0) * (r - x[local_face]) / (3.0 * V)


# Degree-2 exact 4-point rule on a tet (Keast/Stroud): barycentric (a,b,b,b).
_A, _B = 0.5854101966249685, 0.1381966011250105
QP2 = np.array([[_A, _B, _B, _B], [_B, _A, _B, _B], [_B, _B, _A, _B], [_B, _B, _B, _A]])


def test_counts_match_kuhn_box(cube6):
    _, m = cube6
    assert (m.n_nodes, m.n_edges, m.n_faces, m.n_tets) == (343, 1854, 2808, 1296)
    assert m.n_int_edges == 1206 and m.n_int_nodes == 125
    # Euler characteristic of a ball: N_s - N_e + N_f - N_t = 1
    assert m.n_nodes - m.n_edges + m.n_faces - m.n_tets == 1


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_incidence_identities(meshname, request):
    _, m = request.getfixturevalue(meshname)
    G, Cm, D = (m.incidence_dense(w) for w in "GCD")
    assert np.all(Cm @ G == 0)                   # curl grad = 0
    assert np.all(D @ Cm == 0)                   # div curl = 0
    assert set(np.unique(G)) <= {-1, 0, 1} and np.all(np.abs(G).sum(1) == 2)
    assert np.all(np.abs(Cm).sum(1) == 3) and np.all(np.abs(D).sum(1) == 4)
    # every interior face is shared by two tets with opposite D signs
    colsum = D.sum(0)
    eb, nb, fb = m.flags()
    assert np.all(colsum[fb == 0] == 0)


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_G_is_the_gradient(meshname, request):
    mesh, m = request.getfixturevalue(meshname)
    G = m.incidence_dense("G")
    edges = m.edges()
    for a in range(3):
        phi = mesh.xyz[:, a]
        assert np.allclose(G @ phi, mesh.xyz[edges[:, 1], a] - mesh.xyz[edges[:, 0], a], atol=1e-15)


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_whitney_reproduces_uniform_fields(meshname, request):
    mesh, m = request.getfixturevalue(meshname)
    rng = np.random.default_rng(3)
    E0 = np.array([1.5, -0.7, 2.25])
    B0 = np.array([-0.3, 0.8, 1.1])
    edges, faces = m.edges(), m.faces()
    x = mesh.xyz
    e = (x[edges[:, 1]] - x[edges[:, 0]]) @ E0
    area = 0.5 * np.cross(x[faces[:, 1]] - x[faces[:, 0]], x[faces[:, 2]] - x[faces[:, 0]])
    b = area @ B0
    for t in rng.choice(m.n_tets, 40, replace=False):
        lam = rng.dirichlet(np.ones(4))
        r = lam @ x[mesh.tets[t]]
        E, B = m.gather(t, r, e, b)
        assert np.allclose(E, E0, rtol=1e-12, atol=1e-12)
        assert np.allclose(B, B0, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_commuting_diagram_and_divergence(meshname, request):
    """curl(sum e_i W1_i) = sum (C e)_f W2_f, and (D b)_t = V_t div B."""
    mesh, m = request.getfixturevalue(meshname)
    rng = np.random.default_rng(5)
    Cm, D = m.incidence_dense("C"), m.incidence_dense("D")
    e = rng.standard_normal(m.n_edges)
    b = rng.standard_normal(m.n_faces)
    zero_e = np.zeros(m.n_edges)
    _, vol = m.geom()
    for t in rng.choice(m.n_tets, 15, replace=False):
        T = bary_matrix(mesh.xyz, mesh.tets[t])
        r0 = np.array([0.25, 0.25, 0.25, 0.25]) @ mesh.xyz[mesh.tets[t]]
        h = 1e-3 * np.cbrt(vol[t])
        # the fields are affine in a tet, so central differences are exact up to rounding
        J = np.zeros((3, 3))
        JB = np.zeros((3, 3))
        for a in range(3):
            d = np.zeros(3)
            d[a] = h
            Ep, _ = m.gather(t, r0 + d, e, b)
            Em, _ = m.gather(t, r0 - d, e, b)
            _, Bp = m.gather(t, r0 + d, zero_e, b)
            _, Bm = m.gather(t, r0 - d, zero_e, b)
            J[:, a] = (Ep - Em) / (2 * h)
            JB[:, a] = (Bp - Bm) / (2 * h)
        curlE = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        _, Bc = m.gather(t, r0, zero_e, Cm @ e)
        assert np.allclose(curlE, Bc, rtol=1e-7, atol=1e-7 * np.abs(Bc).max())
        divB = np.trace(JB)
        assert np.isclose((D @ b)[t], vol[t] * divB, rtol=1e-7, atol=1e-9 * np.abs(b).max())
        del T


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_hodge_matrices_by_quadrature(meshname, request):
    """[*eps] and [*mu^-1] against a degree-2 exact quadrature, with W1 built
    from the test's own barycentrics and W2 from the RT0 formula (r-x_k)/(3V)."""
    mesh, m = request.getfixturevalue(meshname)
    eps0, mu0 = W.EPS0, W.MU0
    Md, Hd = m.matrix_dense("M"), m.matrix_dense("H")
    te, tf, _ = m.tet_data()
    edges, faces = m.edges(), m.faces()
    Mq = np.zeros_like(Md)
    Hq = np.zeros_like(Hd)
    for t in range(m.n_tets):
        tet = mesh.tets[t]
        T = bary_matrix(mesh.xyz, tet)
        g = grads(T)
        x = mesh.xyz[tet]
        V = abs(np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]]))) / 6.0
        loc = {int(n): i for i, n in enumerate(tet)}
        for q in QP2:
            r = q @ x
            lam = lam_at(T, r)
            w1 = []
            for k in range(6):
                a, bnode = edges[te[t, k]]
                ia, ib = loc[int(a)], loc[int(bnode)]
                w1.append(lam[ia] * g[ib] - lam[ib] * g[ia])
            w1 = np.array(w1)
            w2 = np.array([rt0(mesh.xyz, tet, k, r, faces[tf[t, k]]) for k in range(4)])
            Mq[np.ix_(te[t], te[t])] += eps0 * (V / 4) * (w1 @ w1.T)
            Hq[np.ix_(tf[t], tf[t])] += (V / 4) * (w2 @ w2.T) / mu0
    assert np.allclose(Md, Mq, rtol=1e-10, atol=1e-12 * np.abs(Md).max())
    assert np.allclose(Hd, Hq, rtol=1e-10, atol=1e-12 * np.abs(Hd).max())


@pytest.mark.parametrize("meshname", ["cube6", "jittered4"])
def test_curl_curl_and_laplacian_closed_forms(meshname, request):
    """K = C^T [*mu^-1] C equals the curl-curl stiffness with curl W1_ab =
    2 grad lam_a x grad lam_b; G^T M G equals the P1 stiffness eps0 int grad lam_i . grad lam_j."""
    mesh, m = request.getfixturevalue(meshname)
    Kd, Ld = m.matrix_dense("K"), m.matrix_dense("L")
    te, _, _ = m.tet_data()
    edges = m.edges()
    Kc = np.zeros_like(Kd)
    Lc = np.zeros_like(Ld)
    for t in range(m.n_tets):
        tet = mesh.tets[t]
        T = bary_matrix(mesh.xyz, tet)
        g = grads(T)
        x = mesh.xyz[tet]
        V = abs(np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]]))) / 6.0
        loc = {int(n): i for i, n in enumerate(tet)}
        curls = []
        for k in range(6):
            a, b = edges[te[t, k]]
            curls.append(2.0 * np.cross(g[loc[int(a)]], g[loc[int(b)]]))
        curls = np.array(curls)
        Kc[np.ix_(te[t], te[t])] += V * (curls @ curls.T) / W.MU0
        Lc[np.ix_(tet, tet)] += W.EPS0 * V * (g @ g.T)
    assert np.allclose(Kd, Kc, rtol=1e-9, atol=1e-11 * np.abs(Kd).max())
    assert np.allclose(Ld, Lc, rtol=1e-9, atol=1e-11 * np.abs(Ld).max())
    # gradients are in the kernel of the curl-curl operator
    G = m.incidence_dense("G").astype(float)
    assert np.abs(Kd @ G).max() <= 1e-12 * np.abs(Kd).max()
