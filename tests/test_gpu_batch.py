"""Batched stepping: several independent runs of uneven size stepped together
(one stream per run, one persistent launch per solve over all runs, six-step
CUDA graphs, tuned solver launch shapes) give exactly what stepping each run
alone gives, each run still conserves charge, and each member agrees with the
FP64 oracle.
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


def runs(F, precision):
    out = []
    for k, (cells, n) in enumerate([(4, 3000), (6, 8000), (8, 20000)]):
        wl = W.thermal_plasma_cube(n_cells=cells, n_particles=n, seed=40 + k)
        dt = 2 * DT_CFL_6 * 6 / cells
        out.append((wl, dt))
    return out


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_batch_equals_individual_steps(F, precision):
    cases = runs(F, precision)
    solo = [F.sim_from_workload(wl, dt, precision=precision) for wl, dt in cases]
    memb = [F.sim_from_workload(wl, dt, precision=precision) for wl, dt in cases]
    batch = F.Batch(memb)
    steps = 13            # one eager step, then two six-step graph launches
    batch.step(steps)
    for s in solo:
        s.step(steps)
    info = batch.info()
    assert info["graph"] == 1 and info["graph_launches"] == 2, info
    # the tuner timed every candidate of both solves (or took an earlier
    # batch's choice for this shape) and kept one of each
    times = info["tune_newmark_ms"] + info["tune_completion_ms"]
    assert all(t > 0 for t in times) or all(t == -1 for t in times), info
    cands = {(b, F.BATCH_BUILDS[k]) for b, k in F.BATCH_TUNE_CANDIDATES}
    assert (info["solver_blocks_per_sm"], info["solver_build"]) in cands, info
    assert (info["completion_blocks_per_sm"], info["completion_build"]) in cands, info
    for a, b in zip(solo, memb):
        for f in ("E", "B", "RHO", "G"):
            np.testing.assert_array_equal(a.field(f), b.field(f))
        xa, va, ta, ia = a.particles()
        xb, vb, tb, ib = b.particles()
        np.testing.assert_array_equal(ia, ib)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(va, vb)
        d = b.diag()
        assert d["step"] == steps
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"]
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"]
    # a member stepped on its own afterwards continues from the batched state
    memb[1].step(1)
    solo[1].step(1)
    np.testing.assert_array_equal(solo[1].field("E"), memb[1].field("E"))
    batch.step(7)         # graph dropped (a member moved), recaptured
    assert batch.info()["graph"] == 1


def test_batch_members_match_oracle(F, oracle_lib):
    """Each member of a batch (eager first step, then a six-step graph
    launch) against the FP64 oracle stepped alone: fields and particles
    within 1e-10 relative, as for a single simulation (solves at 1e-13)."""
    cases = runs(F, "plain")
    memb = [F.sim_from_workload(wl, dt, cg_tol=1e-13) for wl, dt in cases]
    orcs = [oracle_lib.from_workload(wl, dt, cg_tol=1e-13) for wl, dt in cases]
    batch = F.Batch(memb)
    steps = 7
    batch.step(steps)
    assert batch.info()["graph_launches"] == 1
    for o in orcs:
        o.step(steps)
    for (wl, _), g, o in zip(cases, memb, orcs):
        for f in ("E", "E_PREV", "G", "RHO", "WALL"):
            a, b = g.field(f), o.field(f)
            assert np.abs(a - b).max() <= 1e-10 * max(np.abs(b).max(), 1e-300), (wl.name, f)
        b_ref = o.field("B")
        sc = max(np.abs(b_ref).max(), np.abs(o.field("E")).max() * wl.mesh.h / W.C0)
        assert np.abs(g.field("B") - b_ref).max() <= 1e-10 * sc, wl.name
        gx, gv, gt, gid = g.particles()
        ox, ov, ot, alive = o.particles()
        ids = np.where(alive)[0]
        assert np.array_equal(gid, ids) and np.array_equal(gt, ot[ids]), wl.name
        assert np.abs(gx - ox[ids]).max() <= 1e-10
        assert np.abs(gv - ov[ids]).max() <= 1e-10 * np.abs(ov).max()
        assert g.diag()["n_alive"] == o.diag()["n_alive"]


def test_batch_rejects_bad_members(F):
    wl = W.thermal_plasma_cube(n_cells=4, n_particles=100, seed=3)
    s = F.sim_from_workload(wl, 2 * DT_CFL_6 * 1.5)
    with pytest.raises(F.PicError) as ei:
        F.Batch([s, s])
    assert ei.value.code == 1
    g = F.sim_from_workload(wl, 2 * DT_CFL_6 * 1.5, preconditioner="gnn")
    with pytest.raises(F.PicError):
        F.Batch([g])


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_batch_with_multigrid_member(F, precision):
    """A member with 8,192 or more interior nodes completes with the
    multigrid-preconditioned solve in the batch too (the batch's completions
    run as one launch: that member's multigrid PCG beside the others'
    Jacobi-PCG), and the batch follows stepping each run alone to the solve
    tolerance (the batch gives the multigrid member fewer blocks, so the
    reduction order differs)."""
    cases = [(22, 20000, 50), (6, 8000, 51), (8, 20000, 52)]
    wls = []
    for cells, n, seed in cases:
        wl = W.thermal_plasma_cube(n_cells=cells, n_particles=n, seed=seed)
        wls.append((wl, 2 * DT_CFL_6 * 6 / cells))
    solo = [F.sim_from_workload(wl, dt, precision=precision, cg_tol=1e-13) for wl, dt in wls]
    memb = [F.sim_from_workload(wl, dt, precision=precision, cg_tol=1e-13) for wl, dt in wls]
    assert solo[0].mesh.n_int_nodes >= 8192
    batch = F.Batch(memb)
    steps = 13
    batch.step(steps)
    for s in solo:
        s.step(steps)
    info = batch.info()
    assert info["graph"] == 1 and info["graph_launches"] == 2, info
    assert info["completion_blocks_per_sm"] in (2, 3, 4) and info["completion_build"] == "64-register", info
    tol = 1e-9 if precision == "plain" else 1e-6
    for a, b in zip(solo, memb):
        for f in ("E", "RHO", "G"):
            ref = a.field(f)
            assert np.abs(b.field(f) - ref).max() <= tol * np.abs(ref).max(), f
        d = b.diag()
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"]
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"]
    # the multigrid member's completion takes the iterations it takes alone (a
    # Jacobi-PCG completion of that mesh would take several times more)
    it_b, it_s = memb[0].diag()["completion_iters"], solo[0].diag()["completion_iters"]
    assert it_b <= 30 and abs(it_b - it_s) <= 3, (it_b, it_s)
