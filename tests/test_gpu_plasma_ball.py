"""GPU path vs the FP64 oracle on a reduced copy of the plasma-ball workload.

The benchmark steps a neutral electron + proton ball (mass ratio 1836) in a
jittered Kuhn box (Sec. IV.C analogue).  This file runs the same recipe at
16^3 cells (24,576 tets, so particle keys tet << 2 | species exceed 2^16 and
the radix sort takes three passes) with 2 x 65,536 particles, 20% vertex
jitter and dt = 4 x CFL, through the C ABI, against the oracle:

* PLAIN (FP64 throughout): fields and particles within 1e-10 relative for 10
  steps (Newmark solves at 1e-13 so that the two CG recurrences are not what
  is measured), conservation <= 1e-12 relative every step.
* MIXED (FP32 state, gather and push, 24-bit fixed-point barycentrics,
  integer deposit, FP64-judged solve): within the tolerance that FP32
  positions allow (derived below), conservation <= 1e-12 every step.

Both legs exercise two species in the per-tet accumulators, per-species node
charges, the three-pass sort and the walk on a jittered mesh.
"""
import math

import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KAPPA_JITTER = 0.19447878340721006   # dt_CFL c / h of the 20%-jittered Kuhn lattice (tests/golden/dt_cfl.json)
CELLS = 16
NPS = 65536


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic
    fempic.load()
    return fempic


@pytest.fixture(scope="module")
def ball():
    wl = W.plasma_ball(n_cells=CELLS, n_per_species=NPS, seed=41)
    dt = 4.0 * KAPPA_JITTER * wl.mesh.h / W.C0
    return wl, dt


def rel_err(a, b, scale=None):
    scale = max(np.abs(b).max() if scale is None else max(scale, np.abs(b).max()), 1e-300)
    return np.abs(a - b).max() / scale


def b_scale(e, h):
    return np.abs(e).max() * h / W.C0


def test_ball_keys_need_three_sort_passes(ball):
    wl, _ = ball
    n_tets = wl.mesh.tets.shape[0]
    assert n_tets == 6 * CELLS ** 3
    assert ((n_tets << 2) | 3).bit_length() > 16      # the dead-particle key n_tets << 2 included


def test_plasma_ball_plain_parity_10_steps(F, oracle_lib, ball):
    wl, dt = ball
    osim = oracle_lib.from_workload(wl, dt, cg_tol=1e-13)
    gsim = F.sim_from_workload(wl, dt, cg_tol=1e-13)
    side = wl.mesh.size[0]
    for name in ("E", "RHO", "PHI"):
        assert rel_err(gsim.field(name), osim.field(name)) <= 1e-12, name
    for step in range(10):
        osim.step()
        gsim.step()
        for name in ("E", "E_PREV", "G", "DG", "RHO", "WALL"):
            assert rel_err(gsim.field(name), osim.field(name)) <= 1e-10, (step, name)
        assert rel_err(gsim.field("B"), osim.field("B"), b_scale(osim.field("E"), wl.mesh.h)) <= 1e-10, step
        gx, gv, gt, gid = gsim.particles()
        ox, ov, ot, alive = osim.particles()
        ids = np.where(alive)[0]
        assert np.array_equal(gid, ids)
        assert np.array_equal(gt, ot[ids])
        assert np.abs(gx - ox[ids]).max() <= 1e-10 * side
        # electrons and protons separately: each against its own speed scale
        for sl in (slice(0, NPS), slice(NPS, 2 * NPS)):
            sel = (ids >= sl.start) & (ids < sl.stop)
            vs = np.abs(ov[ids[sel]]).max()
            assert np.abs(gv[sel] - ov[ids[sel]]).max() <= 1e-10 * vs
        gd, od = gsim.diag(), osim.diag()
        assert gd["n_alive"] == od["n_alive"]
        assert gd["continuity_abs"] <= 1e-12 * gd["rho_max"], gd
        assert gd["gauss_abs"] <= 1e-12 * gd["rho_max"], gd
        assert abs(gd["cg_iters"] - od["cg_iters"]) <= 1


def test_plasma_ball_mixed_against_oracle(F, oracle_lib, ball):
    """MIXED precision on the two-species jittered ball.  An FP32 position
    carries an ulp of ~eps32 * L (L the box side), while a thermal electron
    moves v_th,e * dt per step, so the current of one step, and the fields it
    drives, are known to about 2 eps32 L / (v_th,e dt) relative (1.1e-3 here;
    the protons move less but carry 1/43 of the current).  Positions agree to
    a few FP32 ulps of the box."""
    wl, dt = ball
    osim = oracle_lib.from_workload(wl, dt, cg_tol=1e-13)
    gsim = F.sim_from_workload(wl, dt, precision="mixed", cg_tol=1e-13)
    side = wl.mesh.size[0]
    vth_e = math.sqrt(10.0 * W.EV / W.M_E)
    tol = 2.0 * np.finfo(np.float32).eps * side / (vth_e * dt)
    worst = {}
    for step in range(10):
        osim.step()
        gsim.step()
        for name in ("E", "G", "RHO"):
            err = rel_err(gsim.field(name), osim.field(name))
            worst[name] = max(worst.get(name, 0.0), err)
            assert err <= tol, (step, name, err, tol)
        d = gsim.diag()
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"], d
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"], d
    gx, gv, gt, gid = gsim.particles()
    ox, ov, ot, alive = osim.particles()
    ids = np.where(alive)[0]
    common = np.intersect1d(gid, ids)
    assert len(common) >= 0.999 * len(ids)
    gi = np.searchsorted(gid, common)
    assert np.abs(gx[gi] - ox[common]).max() <= 64 * np.finfo(np.float32).eps * side
    assert np.mean(gt[gi] == ot[common]) >= 0.999
    print("MIXED vs oracle, max relative error over 10 steps:", worst, "tolerance", tol)
