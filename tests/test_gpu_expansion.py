"""Adiabatic expansion of a neutral Gaussian plasma ball (Sec. IV.C) against
the self-similar solution of Kovalev and Bychenkov that the paper compares
with: a quasi-neutral Gaussian cloud of ions and hot electrons stays Gaussian
and its ion variance per axis grows as

    sigma^2(t) = sigma_0^2 + k_B (T_e + T_i) t^2 / m_i,

the electrons' thermal energy going into the ions' radial motion.  The
solution is the limit sigma / lambda_D -> infinity; at a finite ratio the
hottest electrons leave the ball before the ambipolar field holds them, so
the ions are driven a little less hard.  The check is statistical: MIXED
precision, Maxwell-solver Newmark form, first-order absorbing walls, one
e-/ion ball with sigma = 13.7 lambda_D (lambda_D resolved to h / 2.9) and a
reduced ion mass of 100 m_e, so that one expansion time sigma_0 / c_s takes
682 steps at omega_pe dt = 0.2.  Measured on a GB300: the growth of sigma^2
is 0.85-0.89 of the closed form from 0.4 to 1.0 expansion times, 5% of the
electrons and no ions reach the walls, and continuity and Gauss's law stay
at round-off; the assertions leave room around those numbers.
"""
import math

import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CELLS, PER, TE_EV, TI_EV, DEBYE_OVER_H, SIGMA_FRAC, MASS_RATIO, H = 48, 200_000, 1000.0, 10.0, 0.35, 0.1, 100.0, 1.0e-4
WPE_DT = 0.2


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic
    fempic.load()
    return fempic


def test_ion_variance_follows_kovalev_bychenkov(F):
    wl = W.plasma_ball(n_cells=CELLS, n_per_species=PER, h=H, jitter=0.2, te_ev=TE_EV, ti_ev=TI_EV,
                       sigma_frac=SIGMA_FRAC, debye_over_h=DEBYE_OVER_H, mass_ratio=MASS_RATIO)
    wl.form = "mfem"
    wl.wall_bc = W.box_wall_bc(wl.mesh, W.BOX_WALLS)
    # omega_pe at the peak density = v_te / lambda_D
    wpe = math.sqrt(TE_EV * W.EV / W.M_E) / (DEBYE_OVER_H * H)
    dt = WPE_DT / wpe
    cs2 = (TE_EV + TI_EV) * W.EV / (MASS_RATIO * W.M_E)
    t_exp = SIGMA_FRAC * CELLS * H / math.sqrt(cs2)
    n_steps = int(round(t_exp / dt))
    sim = F.sim_from_workload(wl, dt, precision="mixed")
    centre = 0.5 * CELLS * H

    def ions():
        x, _, _, ids = sim.particles()
        return x[ids >= PER] - centre, int((ids < PER).sum())

    d0, ne0 = ions()
    s20 = (d0 ** 2).mean()          # per-axis variance, all three axes pooled
    assert ne0 == PER and d0.shape[0] == PER
    checks = {int(round(f * n_steps)): f for f in (0.4, 0.6, 0.8, 1.0)}
    ratios = []
    for step in range(1, n_steps + 1):
        sim.step()
        if step in checks:
            d = sim.diag()
            assert d["continuity_abs"] <= 1e-12 * d["rho_max"], (step, d)
            assert d["gauss_abs"] <= 1e-12 * d["rho_max"], (step, d)
            di, ne = ions()
            t = step * dt
            grow = (di ** 2).mean() - s20
            ratios.append(grow / (cs2 * t * t))
            assert di.shape[0] == PER, "an ion reached a wall"
            assert ne >= 0.9 * PER, ("too many electrons escaped", ne)
    assert len(ratios) == 4
    assert all(0.78 <= r <= 1.05 for r in ratios), ratios
