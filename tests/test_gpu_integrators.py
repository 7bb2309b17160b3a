"""GPU path vs the FP64 oracle for the second integrator and absorbing walls.

* BD-MFEM (the backward-difference Maxwell-solver integrator of Sec. IV.B)
  driven by the same Gbar deposit: fields and particles within 1e-10 of the
  oracle for 10 steps, continuity and Gauss at round-off for 60 steps (the
  integrator-agnostic claim of Sec. III.A on the GPU), and MIXED precision
  within the FP32-state tolerance.
* First-order absorbing walls (Sec. II.A, Eq. impedanceBC; the c [*I] term of
  Eqs. maxwell_semi / wave_cont) in all three forms, on every wall and on two
  walls only: fields and particles within 1e-10 for 10 steps, conservation at
  the interior nodes at round-off.
"""
import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DT_CFL_6 = 1.3017565848335032e-10   # tests/golden/dt_cfl.json, thermal_plasma_cube_6^3


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic
    fempic.load()
    return fempic


def rel_err(a, b, scale=None):
    scale = max(np.abs(b).max() if scale is None else max(scale, np.abs(b).max()), 1e-300)
    return np.abs(a - b).max() / scale


def compare_particles(gpu, orc, tol=1e-10):
    gx, gv, gt, gid = gpu
    ox, ov, ot, alive = orc
    ids = np.where(alive)[0]
    assert np.array_equal(gid, ids)
    assert np.array_equal(gt, ot[ids])
    assert np.abs(gx - ox[ids]).max() <= tol
    assert np.abs(gv - ov[ids]).max() <= tol * np.abs(ov).max()


def case(form, walls, n_cells=6, n=10000, seed=1001):
    wl = W.thermal_plasma_cube(n_cells=n_cells, n_particles=n, seed=seed)
    wl.form = form
    if walls:
        wl.wall_bc = W.box_wall_bc(wl.mesh, walls)
    dt = (1.0 if form == "bd" else 2.0) * DT_CFL_6 * 6 / n_cells
    return wl, dt


@pytest.mark.parametrize("form,walls", [("bd", ()), ("bd", W.BOX_WALLS), ("we", W.BOX_WALLS),
                                        ("mfem", W.BOX_WALLS), ("we", ("z0", "z1")), ("mfem", ("x0",))])
def test_parity_10_steps(F, oracle_lib, form, walls):
    wl, dt = case(form, walls)
    osim = oracle_lib.from_workload(wl, dt, cg_tol=1e-13)
    gsim = F.sim_from_workload(wl, dt, cg_tol=1e-13)
    if walls:
        assert gsim.mesh.n_int_edges == osim.mesh.n_int_edges
    for step in range(10):
        osim.step()
        gsim.step()
        for name in ("E", "E_PREV", "G", "DG", "RHO", "WALL"):
            assert rel_err(gsim.field(name), osim.field(name)) <= 1e-10, (step, name)
        sc = np.abs(osim.field("E")).max() * wl.mesh.h / W.C0
        assert rel_err(gsim.field("B"), osim.field("B"), sc) <= 1e-10, step
        compare_particles(gsim.particles(), osim.particles())
        gd, od = gsim.diag(), osim.diag()
        assert gd["n_alive"] == od["n_alive"]
        assert abs(gd["cg_iters"] - od["cg_iters"]) <= 1
        assert gd["continuity_abs"] <= 1e-12 * gd["rho_max"], gd
        assert gd["gauss_abs"] <= 1e-12 * gd["rho_max"], gd
        assert gd["cg_relres"] <= 1e-12, gd


@pytest.mark.parametrize("form,walls,precision", [("bd", (), "plain"), ("bd", W.BOX_WALLS, "mixed"),
                                                  ("we", W.BOX_WALLS, "mixed"), ("mfem", W.BOX_WALLS, "plain")])
def test_conservation_60_steps(F, form, walls, precision):
    wl, dt = case(form, walls)
    gsim = F.sim_from_workload(wl, dt, precision=precision)
    worst_c = worst_g = 0.0
    for _ in range(60):
        gsim.step()
        d = gsim.diag()
        worst_c = max(worst_c, d["continuity_abs"] / d["rho_max"])
        worst_g = max(worst_g, d["gauss_abs"] / d["rho_max"])
        assert d["cg_relres"] <= 2e-10
    assert worst_c <= 1e-12 and worst_g <= 1e-12, (worst_c, worst_g)


def test_bd_mixed_against_oracle(F, oracle_lib):
    """MIXED precision with the backward difference: the FP32-state tolerance
    2 eps32 L / (v_th dt) of the thermal cube (L = 1 m, v_th = 0.01 c)."""
    wl, dt = case("bd", W.BOX_WALLS)
    osim = oracle_lib.from_workload(wl, dt, cg_tol=1e-13)
    gsim = F.sim_from_workload(wl, dt, precision="mixed", cg_tol=1e-13)
    tol = 2.0 * np.finfo(np.float32).eps / (0.01 * W.C0 * dt)
    for step in range(10):
        osim.step()
        gsim.step()
        for name in ("E", "G", "RHO"):
            assert rel_err(gsim.field(name), osim.field(name)) <= tol, (step, name, tol)
        d = gsim.diag()
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"] and d["gauss_abs"] <= 1e-12 * d["rho_max"], d


def test_absorbing_walls_drain_a_vacuum_field(F, oracle_lib):
    """A divergence-free vacuum field (e = M^-1 C^T r: G^T M e = 0) between
    absorbing walls loses a large part of its energy within 60 steps, while
    between conducting walls it keeps it (wave form, on the GPU).  A
    first-order condition does not absorb grid-scale or grazing waves, so
    only part of the energy leaves (the oracle shows the same plateau)."""
    import scipy.linalg as sl
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.1, seed=4)
    rng = np.random.default_rng(3)
    ratio = {}
    for name, bc in (("pec", None), ("abc", W.box_wall_bc(box))):
        om = oracle_lib.OracleMesh(box.xyz, box.tets)
        if bc is not None:
            om.set_absorbing(bc)
        eb, _, _ = om.flags()
        ii = np.where(eb == 0)[0]
        M = om.matrix_dense("M")
        Cm = om.incidence_dense("C").astype(float)
        e = np.zeros(om.n_edges)
        e[ii] = sl.solve(M[np.ix_(ii, ii)], (Cm.T @ rng.normal(size=om.n_faces))[ii])
        pm = F.Mesh(box.xyz, box.tets, wall_bc=bc)
        s = F.Sim(pm, 2.0 * DT_CFL_6 * 6 / 4, cg_tol=1e-13)
        s.init()
        s.set_field("E", e)
        s.set_field("E_PREV", e)
        out = []
        for _ in range(60):
            s.step()
            d = s.diag()
            out.append(d["energy_e"] + d["energy_b"])
        out = np.array(out)
        ratio[name] = out[-10:].mean() / out[:10].mean()
    assert ratio["pec"] > 0.9, ratio
    assert ratio["abc"] < 0.75, ratio
