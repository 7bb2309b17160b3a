"""Pins of the oracle's field update (Sec. II.B with the Gbar substitution of
Sec. III.A): single discrete eigenmodes evolve with the closed-form Newmark
phase 2 atan(w dt / 2) and no dissipation in both the wave-equation and the
Maxwell-solver forms; one Newmark solve agrees with a dense LAPACK solve; and
the thermal-plasma run keeps discrete continuity and Gauss's law at round-off.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sl

from paper_2102_06248_gb300 import workloads as W


@pytest.fixture(scope="module")
def small(oracle_lib):
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.1, seed=3)
    m = oracle_lib.OracleMesh(box.xyz, box.tets)
    eb, nb, fb = m.flags()
    ii = np.where(eb == 0)[0]
    M, K = m.matrix_dense("M"), m.matrix_dense("K")
    w2, U = sl.eigh(K[np.ix_(ii, ii)], M[np.ix_(ii, ii)])
    return box, m, ii, w2, U


def empty_sim(oracle_lib, m, dt, form):
    cfg = oracle_lib.OracleConfig(dt=dt, form=form, cg_tol=1e-13)
    sim = oracle_lib.OracleSim(m, cfg)
    sim.init()
    return sim


@pytest.mark.parametrize("form", ["we", "mfem"])
def test_newmark_single_mode(oracle_lib, small, form):
    """Vacuum, e^n = a_n u for a mode K u = w^2 M u: both forms advance the phase
    by 2 atan(w dt/2) per step with unit amplitude (gamma = 1/2, beta = 1/4)."""
    box, m, ii, w2, U = small
    k = int(np.argmax(w2 > 1e-6 * w2.max())) + 40         # a curl mode, not a gradient
    omega = math.sqrt(w2[k])
    dt = 3.0 * 2.0 / math.sqrt(w2.max())                  # three times the explicit limit
    phi = 2.0 * math.atan(omega * dt / 2.0)
    u = np.zeros(m.n_edges)
    u[ii] = U[:, k] / np.abs(U[:, k]).max()
    sim = empty_sim(oracle_lib, m, dt, form)
    sim.set_field("E", u)
    sim.set_field("E_PREV", math.cos(phi) * u)
    # b^n = -sin(n phi)/w C u in both forms.  Maxwell-solver form: the
    # Faraday/Ampere pair of the recurrence keeps it.  Wave-equation form: the
    # trapezoid update b^{n+1} = b^n - dt/2 C (e^{n+1} + e^n) sums to it
    # because tan(phi/2) = w dt/2 (the Newmark phase), so this pins the
    # wave-equation Faraday step against a closed form as well.
    Cm = m.incidence_dense("C").astype(float)
    cu = Cm @ u
    sim.set_field("B", np.zeros(m.n_faces))
    sim.set_field("B_PREV", (math.sin(phi) / omega) * cu)
    n = 25
    for k in range(1, n + 1):
        sim.step()
        if k in (1, 2, 7, n):
            b = sim.field("B")
            assert np.allclose(b, -(math.sin(k * phi) / omega) * cu, atol=1e-9 * np.abs(cu).max() / omega), k
    e = sim.field("E")
    assert np.allclose(e, math.cos(n * phi) * u, atol=1e-9)


def test_newmark_solve_matches_dense(oracle_lib):
    """One wave-equation Newmark solve against LAPACK on the recurrence's
    linear system (M + dt^2/4 K) e^{n+1} = rhs on interior edges."""
    wl = W.thermal_plasma_cube(n_cells=4, n_particles=3000, seed=5)
    m = oracle_lib.OracleMesh(wl.mesh.xyz, wl.mesh.tets)
    from oracle.oracle import from_workload
    dt = 3.0e-10
    sim = from_workload(wl, dt, cg_tol=1e-13, mesh=m)
    sim.step(3)
    e_n, e_p, g_n, g_p = (sim.field(x) for x in ("E", "E_PREV", "G", "G_PREV"))
    sim.step(1)
    g_n1, e_n1 = sim.field("G"), sim.field("E")
    M, K = m.matrix_dense("M"), m.matrix_dense("K")
    A = M + 0.25 * dt * dt * K
    rhs = (2 * M - 0.5 * dt * dt * K) @ e_n - A @ e_p - (g_n1 - 2 * g_n + g_p)
    eb, _, _ = m.flags()
    ii = np.where(eb == 0)[0]
    x = sl.solve(A[np.ix_(ii, ii)], rhs[ii], assume_a="pos")
    assert np.allclose(e_n1[ii], x, rtol=1e-9, atol=1e-10 * np.abs(x).max())
    assert np.all(e_n1[eb == 1] == 0)


def test_initial_state(oracle_lib):
    """rho^0 sums to the total charge (sum of barycentrics is 1), the initial
    electrostatic field satisfies Gauss's law, and b^0 reproduces B0."""
    wl = W.thermal_plasma_cube(n_cells=4, n_particles=2000, seed=9)
    from oracle.oracle import from_workload
    sim = from_workload(wl, 3.0e-10)
    rho = sim.field("RHO")
    sp = wl.species[0]
    assert np.isclose(rho.sum(), sp.q * sp.w * sp.x.shape[0], rtol=1e-13)
    bg = sim.field("RHO_BG")
    assert np.isclose(bg.sum(), wl.rho_background * 1.0, rtol=1e-13)
    d = sim.diag()
    assert d["gauss_abs"] <= 1e-13 * d["rho_max"]


@pytest.mark.parametrize("form", ["we", "mfem"])
def test_conservation_thermal_cube(oracle_lib, form):
    """Sec. III.A: with Gbar driving the Newmark update, discrete continuity
    holds at every node every step and the Gauss residual stays at round-off
    (full 6^3 workload, 100 steps at twice the explicit limit)."""
    wl = W.thermal_plasma_cube()
    wl.form = form
    m = oracle_lib.OracleMesh(wl.mesh.xyz, wl.mesh.tets)
    from oracle.oracle import from_workload
    sim = from_workload(wl, 2 * 1.3017565848335032e-10, mesh=m)
    worst_c = worst_g = 0.0
    for _ in range(100):
        sim.step()
        d = sim.diag()
        worst_c = max(worst_c, d["continuity_abs"] / d["rho_max"])
        worst_g = max(worst_g, d["gauss_abs"] / d["rho_max"])
        assert d["cg_relres"] <= 2e-10      # true residual after the gradient completion
    assert worst_c <= 1e-12 and worst_g <= 1e-12, (worst_c, worst_g)
    assert d["n_alive"] < 10_000       # some electrons reached the walls
    assert d["divb_abs"] <= 1e-12 * np.abs(sim.field("B")).max()


def test_background_charge_neutralises(oracle_lib):
    """A static node background equal to minus the particles' initial node
    charge leaves nothing for the initial electrostatic solve: phi = 0 and
    e^0 = 0 exactly; a smooth non-uniform background then keeps Gauss's law
    (G^T M e + rho + wall + rho_bg = 0) at round-off while the plasma moves."""
    wl = W.thermal_plasma_cube(n_cells=4, n_particles=3000, seed=19)
    wl.rho_background = 0.0
    from oracle.oracle import from_workload
    probe = from_workload(wl, 3e-10)
    rho0 = probe.field("RHO")
    m = probe.mesh
    sp = wl.species[0]
    cfg = oracle_lib.OracleConfig(dt=3e-10, b0=wl.b0)
    sim = oracle_lib.OracleSim(m, cfg)
    sim.add_species(sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    sim.set_background_charge(-rho0)
    sim.init()
    assert np.abs(sim.field("PHI")).max() == 0.0
    assert np.abs(sim.field("E")).max() == 0.0
    assert np.allclose(sim.field("RHO_BG"), -rho0, rtol=0, atol=0)
    xyz = wl.mesh.xyz
    bump = np.exp(-np.sum((xyz - 0.4) ** 2, axis=1) / 0.05)
    bg = -rho0.sum() * bump / bump.sum()
    sim2 = oracle_lib.OracleSim(m, cfg)
    sim2.add_species(sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    sim2.set_background_charge(bg)
    sim2.init()
    for _ in range(20):
        sim2.step()
        d = sim2.diag()
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"], d
