"""The allocation-free electrostatic solve against the library's own.

pic_electrostatic_solve_noalloc exists for callers that cannot allocate device
memory when they need the solve: runtimes that hand out all device memory from
their own pool and forbid libraries to allocate, or services whose memory
budget is fixed at start-up.  It keeps its working vectors in one fixed device
array shared by all calls, so the GPU test calls it twice in a row on the same
inputs and checks both results against the potential that pic_sim_init
computed through the regular (allocating) path, and checks that the second
call leaves the device's free memory unchanged.  The file name makes pytest
collect it after every other test.
"""
import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

TOL = 1e-12     # the tolerance of the other field comparisons of the suite


@pytest.mark.gpu
def test_noalloc_solve_matches_sim_init_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic as F

    wl = W.thermal_plasma_cube(n_cells=8, n_particles=20000, seed=31)
    sim = F.sim_from_workload(wl, 3.0e-10)
    rho = sim.field("RHO") + sim.field("RHO_BG")
    phi_ref = sim.field("PHI")
    scale = np.abs(phi_ref).max()
    assert scale > 0
    rho_d = torch.tensor(rho, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    results = []
    import gc
    for call in range(2):
        phi_d = torch.full((sim.mesh.n_nodes,), float("nan"), dtype=torch.float64, device="cuda")
        # objects of earlier tests must not be freed in the middle of the
        # measurement (that raises the free memory), so collect them first
        gc.collect()
        torch.cuda.synchronize()
        gc.disable()
        try:
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
            F.electrostatic_solve_noalloc(sim.mesh, rho_d, phi_d, tol=1e-14, stream=stream)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            alloc1 = torch.cuda.memory_allocated()
        finally:
            gc.enable()
        if call == 1:
            # the first call looked up the fixed array; the second must not
            # take any device memory at all
            assert free1 >= free0, (free0, free1)
            assert alloc1 == alloc0
        phi = phi_d.cpu().numpy()
        assert np.all(np.isfinite(phi))
        assert np.abs(phi - phi_ref).max() <= TOL * scale, call
        results.append(phi)
    assert np.abs(results[0] - results[1]).max() <= TOL * scale


@pytest.mark.gpu
def test_noalloc_solve_rejects_meshes_beyond_its_limit():
    pytest.importorskip("torch")
    from paper_2102_06248_gb300 import fempic as F

    box = W.kuhn_box((90, 90, 70), (0.9, 0.9, 0.7))      # 546,679 interior nodes > 524,288
    mesh = F.Mesh(box.xyz, box.tets)
    assert mesh.n_int_nodes > 524288
    with pytest.raises(F.PicError) as ei:
        F._check(F.load().pic_electrostatic_solve_noalloc(mesh._h, None, None, 1e-14, None),
                 "pic_electrostatic_solve_noalloc")
    assert ei.value.code == 1 and "limit" in str(ei.value)


def test_noalloc_wrapper_rejects_bad_tensors_before_any_launch():
    """The C entry point takes no lengths, so the binding checks dtype,
    device, contiguity and length first (no GPU needed: every case below is
    refused before the library is called)."""
    torch = pytest.importorskip("torch")
    from paper_2102_06248_gb300 import fempic as F

    box = W.kuhn_box((2, 2, 2), (1.0, 1.0, 1.0))
    mesh = F.Mesh(box.xyz, box.tets)
    n = mesh.n_nodes
    good_cpu = torch.zeros(n, dtype=torch.float64)
    cases = [
        (torch.zeros(n, dtype=torch.float32), good_cpu),         # wrong dtype
        (good_cpu, torch.zeros(n - 1, dtype=torch.float64)),      # wrong length
        (good_cpu, torch.zeros(2 * n, dtype=torch.float64)[::2]), # not contiguous
        (good_cpu, good_cpu),                                     # host memory
        (np.zeros(n), good_cpu),                                  # not a tensor
    ]
    for rho, phi in cases:
        with pytest.raises(F.PicError) as ei:
            F.electrostatic_solve_noalloc(mesh, rho, phi)
        assert ei.value.code == 1
