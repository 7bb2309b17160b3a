"""The multigrid-preconditioned completion against the FP64 oracle.

Meshes with at least 8,192 interior nodes get a smoothed-aggregation
hierarchy of the node Laplacian and complete every field solve with a
multigrid-preconditioned flexible PCG instead of Jacobi-PCG.  Both stop at the
same absolute defect (completion_tol * max|rho + wall|), so the result is the
oracle's to that defect: fields and particles within 1e-10 for 8 steps of a
24^3 thermal cube (12,167 interior nodes), conservation at round-off for 40
steps, with an order of magnitude fewer completion iterations than the
Jacobi-PCG that the oracle and smaller meshes use.
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


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_multigrid_completion(F, oracle_lib, precision):
    wl = W.thermal_plasma_cube(n_cells=24, n_particles=40000, seed=33)
    dt = 2 * DT_CFL_6 * 6 / 24
    assert (24 - 1) ** 3 >= 8192
    gsim = F.sim_from_workload(wl, dt, precision=precision, cg_tol=1e-13)
    osim = oracle_lib.from_workload(wl, dt, cg_tol=1e-13) if precision == "plain" else None
    iters = []
    for step in range(40):
        gsim.step()
        d = gsim.diag()
        iters.append(d["completion_iters"])
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"], (step, d)
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"], (step, d)
        if osim is not None and step < 8:
            osim.step()
            for name in ("E", "G", "RHO"):
                assert rel_err(gsim.field(name), osim.field(name)) <= 1e-10, (step, name)
    assert max(iters) <= 40, iters       # Jacobi-PCG needs ~100 here
