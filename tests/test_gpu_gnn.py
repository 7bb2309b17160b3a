"""Learned edge preconditioner on the GPU against its FP64 oracle.

Forward output and the training gradient of the GPU kernels are compared
with oracle/gnn_oracle.py at the same bfloat16 weights (the GPU computes the
network in FP32: 1e-4 relative on the learned correction, 1e-3 relative on
gradients).  The training test shows what the trained network changes in the
Newmark solve: iterations against Jacobi-PCG on the same system, the same
solution to the solve tolerance, and conservation untouched.
"""
import numpy as np
import pytest

from oracle import gnn_oracle as GO
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


@pytest.fixture(scope="module")
def case(F, oracle_lib):
    box = W.kuhn_box((4, 4, 4), (1.0, 1.0, 1.0), jitter=0.15, seed=21)
    dt = 2 * DT_CFL_6
    pm = F.Mesh(box.xyz, box.tets)
    sim = F.Sim(pm, dt)
    sim.init()
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    A, ids = GO.interior_system(om, dt)
    return sim, pm, A, ids


def random_weights(seed, scale=0.25):
    return np.random.default_rng(seed).normal(0.0, scale, GO.N_PARAMS).astype(np.float32)


def test_forward_matches_oracle(case):
    sim, pm, A, ids = case
    w = random_weights(1)
    sim.gnn_set_weights(w)
    rng = np.random.default_rng(2)
    r = np.zeros(pm.n_edges)
    r[ids] = rng.normal(size=ids.size)
    z = sim.gnn_apply(r)
    zo, _ = GO.EdgeNet(A).forward(r[ids], GO.bf16(w))
    jac = r[ids] / A.diagonal()
    corr_g, corr_o = z[ids] - jac, zo - jac
    assert np.abs(corr_o).max() > 0.1 * np.abs(jac).max()       # the network part is not negligible
    assert np.abs(corr_g - corr_o).max() <= 1e-4 * np.abs(corr_o).max()
    assert np.abs(z[ids] - zo).max() <= 1e-5 * np.abs(zo).max()
    wall = np.setdiff1d(np.arange(pm.n_edges), ids)
    assert np.all(z[wall] == 0.0)


def test_gradient_matches_oracle(case):
    sim, pm, A, ids = case
    w = random_weights(3)
    sim.gnn_set_weights(w)
    rng = np.random.default_rng(4)
    r = np.zeros(pm.n_edges)
    r[ids] = rng.normal(size=ids.size)
    L, g = sim.gnn_loss_grad(r)
    Lo, go, _ = GO.EdgeNet(A).loss_and_grad(r[ids], GO.bf16(w))
    assert L == pytest.approx(Lo, rel=1e-5, abs=1e-6)
    for name, (o, s) in GO.OFFSETS.items():
        if name == "_size":
            continue
        sl = slice(o, o + int(np.prod(s)))
        scale = max(np.abs(go[sl]).max(), 1e-3 * np.abs(go).max())
        assert np.abs(g[sl] - go[sl]).max() <= 1e-3 * scale, name


def test_zero_output_layer_is_jacobi(case):
    sim, pm, A, ids = case
    w = random_weights(5)
    w[GO.OFFSETS["o"][0]:GO.OFFSETS["o"][0] + 32] = 0.0
    w[GO.OFFSETS["d0"][0]] = 0.0
    sim.gnn_set_weights(w)
    r = np.zeros(pm.n_edges)
    r[ids] = np.random.default_rng(6).normal(size=ids.size)
    z = sim.gnn_apply(r)
    np.testing.assert_allclose(z[ids], r[ids] / A.diagonal(), rtol=1e-15, atol=0)


def test_training_gain_and_conservation(F):
    """Two identical runs; after 3 Jacobi steps one of them trains the network
    on residuals of its last Newmark system and steps on with the flexible
    PCG.  The next system is solved in fewer iterations to the same
    tolerance, and continuity and Gauss stay at round-off."""
    wl = W.thermal_plasma_cube(n_cells=10, n_particles=20000, seed=7)
    dt = 2 * DT_CFL_6 * 6 / 10
    mesh = F.Mesh(wl.mesh.xyz, wl.mesh.tets)
    ja = F.sim_from_workload(wl, dt, mesh=mesh)
    gn = F.sim_from_workload(wl, dt, mesh=mesh, preconditioner="gnn")
    for _ in range(3):
        ja.step()
        gn.step()
    np.testing.assert_array_equal(ja.field("E"), gn.field("E"))
    loss = gn.gnn_train(steps=400, lr=3e-3, samples=8)
    it_j, it_g = [], []
    for _ in range(3):
        ja.step()
        gn.step()
        it_j.append(ja.diag()["cg_iters"])
        it_g.append(gn.diag()["cg_iters"])
        e_j, e_g = ja.field("E"), gn.field("E")
        assert np.abs(e_g - e_j).max() <= 1e-7 * np.abs(e_j).max()
        d = gn.diag()
        assert d["continuity_abs"] <= 1e-12 * d["rho_max"]
        assert d["gauss_abs"] <= 1e-12 * d["rho_max"]
    print(f"GNN training loss {loss:.6f}; Newmark PCG iterations Jacobi {it_j} vs learned {it_g}")
    assert sum(it_g) < sum(it_j)
