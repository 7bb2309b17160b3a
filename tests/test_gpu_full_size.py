"""The benchmark's own configuration at full size against the oracle: the
64^3 jittered plasma ball (1,572,864 tets) with 16M electrons + 16M protons,
MIXED precision, in the launch configuration `bench.py` times.

The oracle cannot step 33.5M particles in test time, so the checks are the
two kinds that hold at any size:

* properties: after two full steps, continuity and Gauss's law at round-off,
  no latched error, a million random particles inside their tets (to the
  FP32 rounding of their positions);
* sampled outputs the oracle computes one by one: 4,000 particles (2,000 of
  each species) are copied, with the GPU's current E and B, into an oracle
  simulation on the same mesh, and one particle phase of both is compared for
  those particles (position, velocity, tet, absorption), at the tolerance of
  the other MIXED particle-phase tests.
"""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SAMPLE = 2000   # per species


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic
    fempic.load()
    return fempic


def barycentrics(box, tet, x):
    P = box.xyz[box.tets[tet]]
    Mx = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    lam = np.linalg.solve(Mx, (x - P[:, 0])[..., None])[..., 0]
    return np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], axis=1)


def test_full_size_benchmark_configuration(F, oracle_lib):
    sys.path.insert(0, ROOT)
    import bench
    wl, dt, _ = bench.make_workload("plasma_ball", 64, 16 * 1024 * 1024)
    n_sp = [sp.x.shape[0] for sp in wl.species]
    sim = F.sim_from_workload(wl, dt, precision="mixed")
    sim.step(2)
    d = sim.diag()
    assert d["status"] == 0
    assert d["continuity_abs"] <= 1e-12 * d["rho_max"], d
    assert d["gauss_abs"] <= 1e-12 * d["rho_max"], d

    x, v, tet, ids = sim.particles()
    box = wl.mesh
    rng = np.random.default_rng(64)
    some = rng.choice(len(ids), size=1_000_000, replace=False)
    assert barycentrics(box, tet[some], x[some]).min() >= -1e-5   # FP32 positions: inside up to their rounding

    # the sample, by species (ids are assigned in load order); the oracle takes
    # a particle only if its FP64 barycentrics in its tet are not negative, so
    # the sample is drawn from particles not within FP32 rounding of a face
    e, b = sim.field("E"), sim.field("B")
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    osim = oracle_lib.OracleSim(om, oracle_lib.OracleConfig(dt=dt, pusher="boris", form=wl.form))
    picks = []
    lo = 0
    for k, sp in enumerate(wl.species):
        members = np.where((ids >= lo) & (ids < lo + n_sp[k]))[0]
        cand = rng.choice(members, size=4 * SAMPLE, replace=False)
        cand = cand[barycentrics(box, tet[cand], x[cand]).min(axis=1) > 1e-9]
        sel = np.sort(cand[:SAMPLE])
        assert len(sel) == SAMPLE
        picks.append(sel)
        osim.add_species(sp.q, sp.m, sp.w, x[sel].astype(np.float64), v[sel].astype(np.float64), tet[sel])
        lo += n_sp[k]
    osim.init()
    osim.set_field("E", e)
    osim.set_field("B", b)
    sample_ids = ids[np.concatenate(picks)]      # GPU ids of the oracle's particles 0, 1, ...

    sim.particle_phase()
    osim.particle_phase()
    gx, gv, gt, gid = sim.particles()
    ox, ov, ot, alive = osim.particles()
    pos = np.searchsorted(gid, sample_ids)
    found = (pos < len(gid)) & (gid[np.minimum(pos, len(gid) - 1)] == sample_ids)
    # the same particles are absorbed (at most a handful may differ, at FP32
    # distance from a wall)
    assert np.mean(found == alive) >= 0.999
    both = found & alive
    gi = pos[both]
    side = box.xyz.max() - box.xyz.min()
    assert np.abs(gx[gi] - ox[both]).max() <= 1e-5 * side
    assert np.abs(gv[gi] - ov[both]).max() <= 1e-5 * np.abs(ov).max()
    assert np.mean(gt[gi] == ot[both]) >= 0.999
    assert sim.diag()["status"] == 0
