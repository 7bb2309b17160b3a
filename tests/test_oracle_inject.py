"""Particles injected between steps (the beam source of Sec. IV.B) in the oracle.

Injection moves charge q w lambda(x) from the node wall reservoir into rho, so
rho + wall -- and with it the weak Gauss residual G^T M e + rho + wall -- is
unchanged by the injection itself, and the next step's discrete continuity
(rho + wall)^{n+1} - (rho + wall)^n = G^T dGbar holds as for any particle.
The checks below compare against these laws, not against the oracle.
"""
import numpy as np

from paper_2102_06248_gb300 import workloads as W

H = 1.0e-3
KAPPA = 0.2305    # tests/golden/dt_cfl.json, kuhn_lattice_16^3


def test_injection_keeps_gauss_and_continuity(oracle_lib):
    wl = W.electron_beam(cells=(4, 4, 8), h=H, n_inflight=400, seed=11)
    dt = 4.0 * KAPPA * H / W.C0
    sim = oracle_lib.from_workload(wl, dt, cg_tol=1e-12)
    sp = wl.species[0]
    n0 = sim.particles()[0].shape[0]
    for step in range(5):
        sim.step()
        d = sim.diag()
        scale = max(d["rho_max"], 1e-300)
        assert d["continuity_abs"] <= 1e-12 * scale
        assert d["gauss_abs"] <= 1e-12 * scale
        rho, wall = sim.field("RHO"), sim.field("WALL")
        n = W.inject_per_step(wl, dt) + 3
        x, v, tet = W.beam_injection(wl, step, n, dt, seed=11)
        sim.inject(sp.q, sp.m, sp.w, x, v, tet)
        rho2, wall2 = sim.field("RHO"), sim.field("WALL")
        # the total node charge is unchanged, and the injected charge sits at the
        # nodes of the particles' tets
        assert np.abs((rho2 + wall2) - (rho + wall)).max() <= 1e-15 * np.abs(rho + wall).max()
        lam_total = np.abs(rho2 - rho).sum()
        assert abs(lam_total - abs(sp.q * sp.w) * n) <= 1e-12 * abs(sp.q * sp.w) * n
        n0 += n
    assert sim.particles()[0].shape[0] == n0
