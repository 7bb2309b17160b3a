"""Particle loads through the device staging arrays: the same particles given as
host arrays or as CUDA tensors, in one load or in several (the staging grows by
a device copy), with a rejected load in between, give the same simulation bit
for bit.
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


@pytest.mark.parametrize("precision", ["mixed", "plain"])
def test_host_device_and_split_loads_agree(F, precision):
    import torch
    wl = W.thermal_plasma_cube(n_cells=6, n_particles=3000, seed=11)
    mesh = F.Mesh(wl.mesh.xyz, wl.mesh.tets)

    def make(device, pieces, bad_in_between=False):
        s = F.Sim(mesh, 2 * DT_CFL_6, form=wl.form, pusher=wl.pusher, precision=precision, b0=wl.b0,
                  rho_background=wl.rho_background)
        for k, sp in enumerate(wl.species):
            cuts = np.linspace(0, sp.x.shape[0], pieces + 1).astype(int)
            for lo, hi in zip(cuts[:-1], cuts[1:]):
                x, v, t = sp.x[lo:hi], sp.v[lo:hi], sp.tet[lo:hi].astype(np.int32)
                if device:
                    x, v, t = (torch.tensor(a, device="cuda") for a in (x, v, t))
                s.particles_load(k, sp.q, sp.m, sp.w, x, v, t)
                if bad_in_between:
                    with pytest.raises(F.PicError):
                        s.particles_load(k, sp.q, sp.m, sp.w, np.array([[np.inf, 0.0, 0.0]]), np.zeros((1, 3)))
        s.init()
        return s

    sims = [make(False, 1), make(True, 1), make(False, 3, bad_in_between=True), make(True, 4)]
    for s in sims:
        s.step(4)
    ref = sims[0]
    xr, vr, tr, ir = ref.particles()
    for s in sims[1:]:
        for f in ("E", "B", "RHO", "G"):
            np.testing.assert_array_equal(ref.field(f), s.field(f))
        x, v, t, i = s.particles()
        np.testing.assert_array_equal(ir, i)
        np.testing.assert_array_equal(xr, x)
        np.testing.assert_array_equal(vr, v)
        np.testing.assert_array_equal(tr, t)
