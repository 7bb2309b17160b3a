"""GPU curved particle path (Sec. III.B, Eq. path; Sec. III.C, Algorithms 1-2)
against the FP64 oracle.

The library keeps the path in Newton form and integrates with closed-form
Gauss-Legendre rules; the oracle uses the Lagrange product form and rules
found by Newton iteration.  Both walk with the same algorithm (samples at the
quadrature points, bisection to 1e-15 of the step, exit across the most
negative barycentric), so exits agree to rounding:

* frozen random fields and fast particles (several crossings, wall hits),
  Adams-Bashforth 4 with the path degree ramping 1..4: particles and the
  deposited Gbar increment, node and wall charges within 1e-12;
* full steps of the thermal cube: fields and particles within 1e-10 for 10
  steps, continuity and Gauss's law at round-off for 40 steps;
* the configuration is refused with the Boris pusher or MIXED precision.
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


def rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def compare_particles(gpu, orc, box_scale, tol):
    gx, gv, gt, gid = gpu
    ox, ov, ot, alive = orc
    ids = np.where(alive)[0]
    assert np.array_equal(gid, ids), (len(gid), len(ids))
    assert np.array_equal(gt, ot[ids])
    assert np.abs(gx - ox[ids]).max() <= tol * box_scale
    assert np.abs(gv - ov[ids]).max() <= tol * max(np.abs(ov).max(), 1e-300)


def test_curved_particle_phase_frozen_fields(F, oracle_lib):
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.15, seed=9)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    rng = np.random.default_rng(9)
    n = 1500
    x, tet = W.place_in_box(box, rng.uniform(0.0, 1.0, (n, 3)))
    dt = 1e-9
    v = rng.normal(size=(n, 3)) * 0.3 * 0.25 / dt
    e = rng.normal(size=om.n_edges) * 1e-3
    eb, _, _ = om.flags()
    e[eb == 1] = 0.0
    b = rng.normal(size=om.n_faces) * 1e-12
    osim = oracle_lib.OracleSim(om, oracle_lib.OracleConfig(dt=dt, pusher="ab4", curved_path=True))
    osim.add_species(W.Q_E, W.M_E, 1e3, x, v, tet)
    osim.init()
    osim.set_field("E", e)
    osim.set_field("B", b)
    pm = F.Mesh(box.xyz, box.tets)
    gsim = F.Sim(pm, dt, pusher="ab4", curved_path=True)
    gsim.particles_load(0, W.Q_E, W.M_E, 1e3, x, v, tet)
    gsim.init()
    gsim.set_field("E", e)
    gsim.set_field("B", b)
    for step in range(6):
        osim.particle_phase()
        gsim.particle_phase()
        compare_particles(gsim.particles(), osim.particles(), 1.0, 1e-12)
        for name in ("DG", "RHO", "WALL"):
            assert rel_err(gsim.field(name), osim.field(name)) <= 1e-12, (step, name)
    assert osim.particles()[3].sum() < n           # some particles reached the walls


@pytest.mark.parametrize("form", ["we", "mfem"])
def test_curved_full_steps(F, oracle_lib, form):
    wl = W.thermal_plasma_cube(n_cells=5, n_particles=6000, seed=15, b0z=0.0)
    wl.form = form
    dt = 2 * DT_CFL_6 * 6 / 5
    from oracle.oracle import OracleConfig, OracleMesh, OracleSim
    om = OracleMesh(wl.mesh.xyz, wl.mesh.tets)
    osim = OracleSim(om, OracleConfig(dt=dt, form=form, pusher="ab4", rho_background=wl.rho_background,
                                      cg_tol=1e-13, curved_path=True))
    sp = wl.species[0]
    osim.add_species(sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    osim.init()
    pm = F.Mesh(wl.mesh.xyz, wl.mesh.tets)
    gsim = F.Sim(pm, dt, form=form, pusher="ab4", rho_background=wl.rho_background, cg_tol=1e-13,
                 curved_path=True)
    gsim.particles_load(0, sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    gsim.init()
    for step in range(40):
        osim.step()
        gsim.step()
        if step < 10:
            for name in ("E", "G", "RHO", "WALL"):
                assert rel_err(gsim.field(name), osim.field(name)) <= 1e-10, (step, name)
            compare_particles(gsim.particles(), osim.particles(), 1.0, 1e-10)
        d = gsim.diag()
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"], (step, d)
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"], (step, d)


def test_curved_path_configuration_is_checked(F):
    box = W.kuhn_box((2, 2, 2), (1.0, 1.0, 1.0))
    pm = F.Mesh(box.xyz, box.tets)
    for kw in ({"pusher": "boris"}, {"pusher": "ab4", "precision": "mixed"}):
        with pytest.raises(F.PicError) as ei:
            F.Sim(pm, 1e-9, curved_path=True, **kw)
        assert ei.value.code == 1
