"""Pins of the oracle's curved particle path (Sec. III.B, Eq. path; Sec. III.C,
Algorithms 1 and 2, per-cell Gauss-Legendre quadrature).

* For uniform straight motion the Lagrange path through equally spaced
  collinear positions is the straight segment, so the curved walk (bisection
  exits, quadrature) must reproduce the straight walk (exact linear crossings,
  exact bilinear integral) to the bisection tolerance, crossings and wall
  absorptions included.
* On the Table I cyclotron orbit (Sec. IV.A) with an exact start-up history,
  the Whitney-1 integral along the curved path agrees with the integral along
  the true circular arc far better than the straight chord does.
* Driven by Gbar, the curved path keeps continuity and Gauss's law at
  round-off (continuity holds for any path, Sec. III.A).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DT_CFL_6 = 1.3017565848335032e-10   # tests/golden/dt_cfl.json, thermal_plasma_cube_6^3


def uniform_motion_sims(oracle_lib, curved, n=600, seed=11):
    box = W.kuhn_box((3, 3, 3), (1.0, 1.0, 1.0), jitter=0.15, seed=seed)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    rng = np.random.default_rng(seed)
    x, tet = W.place_in_box(box, rng.uniform(0.05, 0.95, (n, 3)))
    dt = 1e-9
    v = rng.normal(size=(n, 3)) * 0.4 / dt          # ~0.4 m per step: several cells, some walls
    cfg = oracle_lib.OracleConfig(dt=dt, pusher="ab4", curved_path=curved)
    sim = oracle_lib.OracleSim(om, cfg)
    sim.add_species(W.Q_E, W.M_E, 1.0, x, v, tet)
    sim.init()
    sim.set_field("E", np.zeros(om.n_edges))
    sim.set_field("B", np.zeros(om.n_faces))
    return sim


def test_curved_path_reduces_to_the_straight_walk_for_uniform_motion(oracle_lib):
    a = uniform_motion_sims(oracle_lib, True)
    b = uniform_motion_sims(oracle_lib, False)
    crossed = 0
    for step in range(5):             # path degree ramps 1, 2, 3, 4, 4
        a.particle_phase()
        b.particle_phase()
        for f in ("DG", "RHO", "WALL"):
            fa, fb = a.field(f), b.field(f)
            assert np.abs(fa - fb).max() <= 1e-12 * np.abs(fb).max(), (step, f)
        xa, va, ta, aa = a.particles()
        xb, vb, tb, ab = b.particles()
        assert np.array_equal(aa, ab) and np.array_equal(ta[aa], tb[ab])
        assert np.abs(xa - xb).max() <= 1e-12
        crossed += int((~ab).sum())
    assert crossed > 0                # some paths ended on a wall


def test_curved_path_follows_the_true_arc(oracle_lib):
    """One step of the Table I electron (uniform B, E = 0) with AB4 and the
    exact start-up history of accelerations, velocities and positions: the
    deposited Gbar increment is compared with the Whitney-1 integral along the
    exact circular arc (pieces split where the arc crosses faces, each
    integrated with a 20-point Gauss-Legendre rule)."""
    with open(os.path.join(GOLDEN, "table1_cyclotron.json")) as f:
        tab = json.load(f)
    q, mass, Bz = tab["q_C"], tab["m_kg"], tab["B_z_T"]
    v0 = np.array(tab["v0_m_per_s"])
    r0 = np.array(tab["r0_m"])
    wc = abs(q) * Bz / mass
    dt = 2 * math.pi / wc / 64.0
    r_l = np.linalg.norm(v0) / wc
    cx, cy = r0[0] - r_l, r0[1]

    def exact(t):
        ph = wc * t
        return (np.array([cx + r_l * math.cos(ph), cy + r_l * math.sin(ph), 0.0]),
                np.array([-r_l * wc * math.sin(ph), r_l * wc * math.cos(ph), 0.0]))

    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.1, seed=2)
    xyz = box.xyz.copy()
    xyz[:, 2] -= 0.5 - 0.0137            # orbit plane z = 0 inside the box, clear of faces
    om = oracle_lib.OracleMesh(xyz, box.tets)
    grad, _ = om.geom()
    edges = om.edges()
    eidx = {tuple(e): i for i, e in enumerate(edges)}

    def locate(r, exclude=-1):
        for t in range(box.n_tets):
            lam = om.lam(t, r)
            if t != exclude and lam.min() >= -1e-12:
                return t, lam
        raise AssertionError("outside")

    dg = {}
    for curved in (True, False):
        cfg = oracle_lib.OracleConfig(dt=dt, pusher="ab4", b0=(0, 0, Bz), curved_path=curved)
        sim = oracle_lib.OracleSim(om, cfg)
        t0, _ = locate(r0)
        sim.add_species(q, mass, 1.0, r0[None, :], v0[None, :], np.array([t0], dtype=np.int32))
        sim.init()
        sim.set_field("E", np.zeros(om.n_edges))
        ah, vh, rh = [], [], []
        for j in range(1, 4):
            rj, vj = exact(-j * dt)
            ah.append((q / mass) * np.cross(vj, [0, 0, Bz])[None, :])
            vh.append(vj[None, :])
            rh.append(rj[None, :])
        sim.set_ab_history(np.array(ah), np.array(vh))
        sim.set_position_history(np.array(rh))
        sim.particle_phase()
        dg[curved] = sim.field("DG") / q
    # the exact arc from r(0) to r(dt), split where it crosses faces (located
    # by sampling and bisection on the arc itself), each in-tet piece
    # integrated by 20-point Gauss-Legendre (numpy's rule)
    tets = box.tets
    gx, gw = np.polynomial.legendre.leggauss(20)
    arc = np.zeros(om.n_edges)

    def inside(t_tet, tt):
        return om.lam(t_tet, exact(tt)[0]).min() >= 0.0

    t_start = 0.0
    cur, _ = locate(exact(0.0)[0])
    for _ in range(20):
        samples = np.linspace(t_start, dt, 401)[1:]
        out = [tt for tt in samples if not inside(cur, tt)]
        t_end = dt if not out else out[0]
        if out:
            lo = t_start
            hi = t_end
            for _ in range(80):
                mid = 0.5 * (lo + hi)
                if inside(cur, mid):
                    lo = mid
                else:
                    hi = mid
            t_end = lo
        vt = tets[cur]
        for xq, wq in zip(gx, gw):
            tt = 0.5 * (t_start + t_end) + 0.5 * (t_end - t_start) * xq
            r, v = exact(tt)
            lam = om.lam(cur, r)
            for a_ in range(4):
                for b_ in range(a_ + 1, 4):
                    tail, head = (a_, b_) if vt[a_] < vt[b_] else (b_, a_)
                    w = lam[tail] * grad[cur, head] - lam[head] * grad[cur, tail]
                    arc[eidx[(vt[tail], vt[head])]] += 0.5 * (t_end - t_start) * wq * (w @ v)
        if not out:
            break
        t_start = t_end
        cur, _ = locate(exact(hi)[0], exclude=cur)
    err_c = np.abs(dg[True] - arc).max()
    err_s = np.abs(dg[False] - arc).max()
    assert err_s > 0
    assert err_c < 0.05 * err_s, (err_c, err_s)


@pytest.mark.parametrize("form", ["we", "mfem"])
def test_curved_path_conservation(oracle_lib, form):
    wl = W.thermal_plasma_cube(n_cells=5, n_particles=3000, seed=14, b0z=0.0)
    wl.form = form
    wl.pusher = "ab4"
    from oracle.oracle import OracleConfig, OracleMesh, OracleSim
    om = OracleMesh(wl.mesh.xyz, wl.mesh.tets)
    cfg = OracleConfig(dt=2 * DT_CFL_6 * 6 / 5, form=form, pusher="ab4", rho_background=wl.rho_background,
                       curved_path=True)
    sim = OracleSim(om, cfg)
    sp = wl.species[0]
    sim.add_species(sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    sim.init()
    worst_c = worst_g = 0.0
    for _ in range(40):
        sim.step()
        d = sim.diag()
        worst_c = max(worst_c, d["continuity_abs"] / d["rho_max"])
        worst_g = max(worst_g, d["gauss_abs"] / d["rho_max"])
    assert worst_c <= 1e-12 and worst_g <= 1e-12, (worst_c, worst_g)
