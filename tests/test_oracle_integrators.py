"""Pins of the oracle's second integrator, absorbing walls and negative control.

* First-order absorbing walls (Sec. II.A, Eq. impedanceBC; the c [*I] term of
  Eq. maxwell_semi / Eq. wave_cont): the surface impedance matrix against a
  brute-force quadrature of the tangential traces of the tets' own Whitney-1
  functions; G_int^T [*I] = 0; and the exact discrete energy balances of both
  Newmark forms, in which the walls remove energy at the rate the damping term
  predicts and nowhere else.
* Backward-difference Maxwell-solver form (BD-MFEM, Sec. IV.B): one curl
  eigenmode decays and turns by the closed-form factor 1 / (1 + i w dt) per
  step; its discrete energy balance; and, driven by Gbar, continuity and
  Gauss's law at round-off (the integrator-agnostic claim of Sec. III.A).
* Negative control (Sec. II.B, Eqs. badNmB / badwave): driving the update by
  point currents instead of Gbar breaks Gauss's law far above round-off on
  the same run that keeps it at round-off with Gbar; for a path inside one
  tet the point current equals the path integral.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2102_06248_gb300 import workloads as W

DT_CFL_6 = 1.3017565848335032e-10   # tests/golden/dt_cfl.json, thermal_plasma_cube_6^3


def absorbing_mesh(oracle_lib, cells=3, jitter=0.15, seed=5, walls=W.BOX_WALLS):
    box = W.kuhn_box((cells,) * 3, (1.0,) * 3, jitter=jitter, seed=seed)
    m = oracle_lib.OracleMesh(box.xyz, box.tets)
    m.set_absorbing(W.box_wall_bc(box, walls))
    return box, m


def test_impedance_matrix_by_quadrature(oracle_lib):
    """[*I]_ij = int_{absorbing faces} (n x W1_i).(n x W1_j) / mu0 against a
    degree-2 triangle rule applied to the tets' 3D Whitney-1 functions
    (W1 = lam_tail grad lam_head - lam_head grad lam_tail, barycentrics and
    gradients from the tet), projected on the face plane."""
    box, m = absorbing_mesh(oracle_lib, walls=("x0", "y1", "z0"))
    grad, vol = m.geom()
    edges = m.edges()
    eidx = {tuple(e): i for i, e in enumerate(edges)}
    bc = W.box_wall_bc(box, ("x0", "y1", "z0"))
    Iq = np.zeros((m.n_edges, m.n_edges))
    # 3-point rule exact for quadratics: barycentric points (2/3,1/6,1/6) and perms, weights S/3
    pts = [(2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3)]
    for t in range(box.n_tets):
        vt = box.tets[t]
        for k in range(4):
            if not bc[t, k]:
                continue
            fv = [j for j in range(4) if j != k]
            xs = box.xyz[vt[fv]]
            nrm = np.cross(xs[1] - xs[0], xs[2] - xs[0])
            S = 0.5 * np.linalg.norm(nrm)
            n = nrm / (2 * S)
            loc = [(a, b) for a in range(4) for b in range(a + 1, 4)]
            for wq in pts:
                lam = np.zeros(4)
                lam[fv] = wq
                tr = {}
                for (a, b) in loc:
                    tail, head = (a, b) if vt[a] < vt[b] else (b, a)
                    w = lam[tail] * grad[t, head] - lam[head] * grad[t, tail]
                    tr[eidx[(vt[tail], vt[head])]] = w - n * (n @ w)
                for i, wi in tr.items():
                    for j, wj in tr.items():
                        Iq[i, j] += (S / 3) * (wi @ wj) / W.MU0
    I = m.matrix_dense("I")
    assert np.abs(I - Iq).max() <= 1e-12 * np.abs(Iq).max()
    assert np.abs(I).max() > 0
    assert np.allclose(I, I.T, atol=1e-15 * np.abs(I).max())
    assert sl.eigvalsh(I).min() >= -1e-12 * np.abs(I).max()


def test_impedance_structure_and_dofs(oracle_lib):
    """Edges on conducting faces are held at zero, the rest are unknowns;
    interior-node gradients never touch an absorbing-face edge (G_int^T I = 0)."""
    box, m_all = absorbing_mesh(oracle_lib)
    assert m_all.n_int_edges == m_all.n_edges
    box, m = absorbing_mesh(oracle_lib, walls=("z0", "z1"))
    eb, nb, fb = m.flags()
    e = m.edges()
    z = box.xyz[:, 2]
    on_side = lambda ax, v: np.abs(box.xyz[:, ax] - v) < 1e-12
    side = np.zeros(m.n_nodes, bool)
    for ax in (0, 1):
        side |= on_side(ax, 0.0) | on_side(ax, 1.0)
    # an edge is held at zero exactly when both ends lie on one conducting side wall
    held = np.zeros(m.n_edges, bool)
    for ax in (0, 1):
        for v in (0.0, 1.0):
            held |= on_side(ax, v)[e[:, 0]] & on_side(ax, v)[e[:, 1]]
    assert np.array_equal(eb.astype(bool), held)
    G = m.incidence_dense("G").astype(float)
    I = m.matrix_dense("I")
    interior = np.where(nb == 0)[0]
    assert np.abs(G[:, interior].T @ I).max() == 0.0
    rows = np.where(np.abs(I).sum(axis=1) > 0)[0]
    on_z = (np.abs(z - 0.0) < 1e-12) | (np.abs(z - 1.0) < 1e-12)
    assert np.all(on_z[e[rows, 0]] & on_z[e[rows, 1]])


def vacuum_sim(oracle_lib, m, dt, form, seed=1):
    cfg = oracle_lib.OracleConfig(dt=dt, form=form, cg_tol=1e-14)
    sim = oracle_lib.OracleSim(m, cfg)
    sim.init()
    rng = np.random.default_rng(seed)
    eb, _, _ = m.flags()
    e0 = rng.normal(size=m.n_edges)
    e1 = rng.normal(size=m.n_edges)
    e0[eb == 1] = 0
    e1[eb == 1] = 0
    sim.set_field("E", e0)
    sim.set_field("E_PREV", e1)
    b0 = rng.normal(size=m.n_faces) * 1e-9
    sim.set_field("B", b0)
    sim.set_field("B_PREV", b0 * 0.5)
    return sim


@pytest.mark.parametrize("walls", [(), W.BOX_WALLS])
def test_we_energy_balance(oracle_lib, walls):
    """Newmark wave equation in vacuum: with E^{n+1/2} = (e'-e)^T M (e'-e)
    + dt^2/4 (e'+e)^T K (e'+e), multiplying the recurrence by e^{n+1} - e^{n-1}
    gives E^{n+1/2} - E^{n-1/2} = -dt/(2c) (e^{n+1}-e^{n-1})^T I (e^{n+1}-e^{n-1})
    exactly: conserved with conducting walls, decaying at exactly that rate
    with absorbing ones."""
    box, m = absorbing_mesh(oracle_lib, walls=walls)
    M, K, I = m.matrix_dense("M"), m.matrix_dense("K"), m.matrix_dense("I")
    dt = 3.0 * 0.2342 * (1.0 / 3) / W.C0
    sim = vacuum_sim(oracle_lib, m, dt, "we")
    hist = [sim.field("E_PREV"), sim.field("E")]
    for _ in range(12):
        sim.step()
        hist.append(sim.field("E"))

    def energy(a, b):
        d, s_ = a - b, a + b
        return d @ M @ d + 0.25 * dt * dt * (s_ @ K @ s_)

    scale = energy(hist[1], hist[0])
    for n in range(1, len(hist) - 1):
        lhs = energy(hist[n + 1], hist[n]) - energy(hist[n], hist[n - 1])
        dd = hist[n + 1] - hist[n - 1]
        rhs = -0.5 * dt / W.C0 * (dd @ I @ dd)
        assert abs(lhs - rhs) <= 1e-10 * scale, (n, lhs, rhs)
        if walls:
            assert rhs < -1e-6 * scale


@pytest.mark.parametrize("form", ["mfem", "bd"])
def test_maxwell_forms_energy_balance(oracle_lib, form):
    """Maxwell-solver forms in vacuum with absorbing walls.
    Newmark: with ebar = e'/4 + e/2 + e''/4, multiplying the Ampere row by
    ebar and the Faraday row by H bbar gives F^{n+1/2} - F^{n-1/2} =
    -dt/c ebar^T I ebar, F = 1/8 (e'+e)^T M (e'+e) + 1/8 (b'+b)^T H (b'+b).
    Backward difference: with W = 1/2 e^T M e + 1/2 b^T H b,
    W' - W + 1/2 |e'-e|_M^2 + 1/2 |b'-b|_H^2 = -dt/c e'^T I e'."""
    box, m = absorbing_mesh(oracle_lib)
    M, H, I = m.matrix_dense("M"), m.matrix_dense("H"), m.matrix_dense("I")
    dt = 2.0 * 0.2342 * (1.0 / 3) / W.C0
    sim = vacuum_sim(oracle_lib, m, dt, form, seed=7)
    es = [sim.field("E_PREV"), sim.field("E")]
    bs = [sim.field("B_PREV"), sim.field("B")]
    for _ in range(10):
        sim.step()
        es.append(sim.field("E"))
        bs.append(sim.field("B"))
    if form == "mfem":
        def F(n):
            u, v = es[n + 1] + es[n], bs[n + 1] + bs[n]
            return (u @ M @ u + v @ H @ v) / 8.0
        scale = F(1)
        for n in range(1, len(es) - 1):
            eb_ = 0.25 * es[n + 1] + 0.5 * es[n] + 0.25 * es[n - 1]
            lhs = F(n) - F(n - 1)
            rhs = -dt / W.C0 * (eb_ @ I @ eb_)
            assert abs(lhs - rhs) <= 1e-10 * scale, (n, lhs, rhs)
    else:
        def Wn(n):
            return 0.5 * (es[n] @ M @ es[n] + bs[n] @ H @ bs[n])
        scale = Wn(1)
        for n in range(1, len(es) - 1):
            de, db = es[n + 1] - es[n], bs[n + 1] - bs[n]
            lhs = Wn(n + 1) - Wn(n) + 0.5 * (de @ M @ de + db @ H @ db)
            rhs = -dt / W.C0 * (es[n + 1] @ I @ es[n + 1])
            assert abs(lhs - rhs) <= 1e-10 * scale, (n, lhs, rhs)
            assert Wn(n + 1) < Wn(n)


def test_backward_difference_single_mode(oracle_lib):
    """BD-MFEM on one curl eigenmode K u = w^2 M u with conducting walls:
    e^n = a_n u, b^n = beta_n C u, and z_n = a_n + i w beta_n obeys
    z_{n+1} = z_n / (1 + i w dt) (backward Euler on a' = w^2 beta,
    beta' = -a), so the mode decays by (1 + w^2 dt^2)^(-1/2) and turns by
    -atan(w dt) per step."""
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.1, seed=3)
    m = oracle_lib.OracleMesh(box.xyz, box.tets)
    eb, _, _ = m.flags()
    ii = np.where(eb == 0)[0]
    M, K = m.matrix_dense("M"), m.matrix_dense("K")
    w2, U = sl.eigh(K[np.ix_(ii, ii)], M[np.ix_(ii, ii)])
    k = int(np.argmax(w2 > 1e-6 * w2.max())) + 40
    omega = math.sqrt(w2[k])
    dt = 0.5 / omega
    u = np.zeros(m.n_edges)
    u[ii] = U[:, k] / np.abs(U[:, k]).max()
    cu = m.incidence_dense("C").astype(float) @ u
    cfg = oracle_lib.OracleConfig(dt=dt, form="bd", cg_tol=1e-14)
    sim = oracle_lib.OracleSim(m, cfg)
    sim.init()
    sim.set_field("E", u)
    sim.set_field("E_PREV", u)
    sim.set_field("B", np.zeros(m.n_faces))
    z = 1.0 + 0.0j
    for n in range(1, 16):
        sim.step()
        z = z / (1.0 + 1j * omega * dt)
        assert np.allclose(sim.field("E"), z.real * u, atol=1e-9), n
        assert np.allclose(sim.field("B"), (z.imag / omega) * cu, atol=1e-9 * np.abs(cu).max() / omega), n
    assert abs(abs(z) - (1 + (omega * dt) ** 2) ** (-7.5)) < 1e-12


@pytest.mark.parametrize("form,walls", [("bd", ()), ("bd", W.BOX_WALLS), ("we", W.BOX_WALLS),
                                        ("mfem", W.BOX_WALLS)])
def test_conservation_other_integrator_and_walls(oracle_lib, form, walls):
    """Sec. III.A for the backward-difference integrator and for absorbing
    walls: driven by Gbar, continuity at every node and Gauss's law at the
    interior nodes stay at round-off (thermal cube, 60 steps)."""
    wl = W.thermal_plasma_cube(n_cells=5, n_particles=4000, seed=11)
    wl.form = form
    if walls:
        wl.wall_bc = W.box_wall_bc(wl.mesh, walls)
    from oracle.oracle import from_workload
    dt = DT_CFL_6 * 6 / 5 * (1.0 if form == "bd" else 2.0)
    sim = from_workload(wl, dt)
    worst_c = worst_g = 0.0
    for _ in range(60):
        sim.step()
        d = sim.diag()
        worst_c = max(worst_c, d["continuity_abs"] / d["rho_max"])
        worst_g = max(worst_g, d["gauss_abs"] / d["rho_max"])
        assert d["cg_relres"] <= 2e-10
    assert worst_c <= 1e-12 and worst_g <= 1e-12, (worst_c, worst_g)
    assert d["n_alive"] < 4000


@pytest.mark.parametrize("form", ["we", "mfem"])
def test_negative_control_point_current(oracle_lib, form):
    """The same run driven by point currents (the direct treatment of
    Eqs. badNmB / badwave) loses Gauss's law by many orders of magnitude,
    while the Gbar run keeps it at round-off."""
    wl = W.thermal_plasma_cube(n_cells=5, n_particles=4000, seed=12)
    wl.form = form
    from oracle.oracle import from_workload
    res = {}
    for cur in ("gbar", "point"):
        sim = from_workload(wl, 2 * DT_CFL_6 * 6 / 5, current=cur)
        worst = 0.0
        for _ in range(20):
            sim.step()
            d = sim.diag()
            worst = max(worst, d["gauss_abs"] / d["rho_max"])
        res[cur] = worst
    assert res["gbar"] <= 1e-12, res
    assert res["point"] >= 1e-6, res


def test_point_current_equals_path_integral_inside_one_tet(oracle_lib):
    """For a path that stays in its tet, W1 is linear along it and the
    midpoint sample of the negative control equals the path integral."""
    box = W.kuhn_box((2, 2, 2), (1.0, 1.0, 1.0), jitter=0.1, seed=2)
    m = oracle_lib.OracleMesh(box.xyz, box.tets)
    x, tet = W.place_in_box(box, np.array([[0.31, 0.22, 0.13]]))
    dt = 1e-9
    v = np.array([[1e5, -2e5, 5e4]])       # 1e-4 m per step: stays in the tet
    out = {}
    for cur in ("gbar", "point"):
        cfg = oracle_lib.OracleConfig(dt=dt, current=cur)
        sim = oracle_lib.OracleSim(m, cfg)
        sim.add_species(W.Q_E, W.M_E, 1.0, x, v, tet)
        sim.init()
        sim.set_field("E", np.zeros(m.n_edges))
        sim.particle_phase()
        assert sim.particles()[2][0] == tet[0]
        out[cur] = sim.field("DG")
    assert np.abs(out["gbar"]).max() > 0
    assert np.abs(out["point"] - out["gbar"]).max() <= 1e-13 * np.abs(out["gbar"]).max()
