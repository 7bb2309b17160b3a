"""Degenerate particle paths (Sec. III.C, Algorithm 1) on the GPU against the
FP64 oracle: an unjittered Kuhn box with E = B = 0, so every path is a
straight line, started exactly at mesh nodes, edge midpoints and face
centroids and moving along the lattice axes, the face diagonals and the body
diagonals (the Kuhn tets share the body diagonal, so those paths run along
tet edges), by half, one and one and a half cells per step (landing exactly
on nodes, edges and faces), plus particles at rest.

Where a path passes exactly through a shared face, edge or vertex, several
tets contain the point and either choice is correct; what must not depend
on the choice is compared exactly: positions, which particles are absorbed,
and the deposits -- Gbar (W1 has a continuous tangential trace, and along a
shared face the opposite barycentric stays 0), node charges (the point's
barycentrics on the shared nodes) and wall charges.  Every particle's tet
must contain its position, and continuity must hold to round-off.
"""
import numpy as np
import pytest

from paper_2102_06248_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CELLS, DT = 4, 2.0 ** -20      # h = 1/4 and dt exact: dt * v and the landing points are exact in FP64 and FP32


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_06248_gb300 import fempic
    fempic.load()
    return fempic


def start_points(box, om):
    xyz = box.xyz
    inner = lambda p: np.all((p > 1e-12) & (p < 1.0 - 1e-12), axis=-1)
    nodes = xyz[inner(xyz)]
    ed = om.edges()
    mids = 0.5 * (xyz[ed[:, 0]] + xyz[ed[:, 1]])
    mids = mids[inner(mids)]
    fa = om.faces()
    cents = (xyz[fa[:, 0]] + xyz[fa[:, 1]] + xyz[fa[:, 2]]) / 3.0
    cents = cents[inner(cents)]
    rng = np.random.default_rng(5)
    mids = mids[rng.choice(len(mids), size=min(60, len(mids)), replace=False)]
    cents = cents[rng.choice(len(cents), size=min(60, len(cents)), replace=False)]
    return np.concatenate([nodes, mids, cents])


def workload(box, om):
    pts = start_points(box, om)
    dirs = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)], dtype=float)
    h = 1.0 / CELLS
    x, v = [], []
    for d in (0.5, 1.0, 1.5):
        for u in dirs:
            x.append(pts)
            v.append(np.broadcast_to(u * d * h / DT, pts.shape))
    x = np.concatenate(x)
    v = np.concatenate(v)
    x, tet = W.place_in_box(box, x)          # unjittered box: the same point, with a tet that contains it
    return x, v, tet


def tet_contains(box, tet, x, tol=1e-12):
    T = box.tets[tet]
    P = box.xyz[T]                            # [n, 4, 3]
    Mx = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]], axis=2)
    l = np.linalg.solve(Mx, (x - P[:, 0])[..., None])[..., 0]
    lam = np.concatenate([1.0 - l.sum(1, keepdims=True), l], axis=1)
    return lam.min(axis=1) >= -tol


def continuity_defect(om, rho0, wall0, rho1, wall1, dg):
    """max |(rho + wall)^{n+1} - (rho + wall)^n - G^T dGbar|, relative."""
    r, c, v = om.incidence("G")
    gtd = np.zeros(om.n_nodes)
    np.add.at(gtd, c, v * dg[r])
    d1 = (rho1 + wall1) - (rho0 + wall0)
    scale = max(np.abs(rho1).max(), np.abs(wall1).max(), 1e-300)
    return np.abs(d1 - gtd).max() / scale


@pytest.mark.parametrize("precision", ["plain", "mixed"])
def test_degenerate_paths(F, oracle_lib, precision):
    box = W.kuhn_box((CELLS,) * 3, (1.0,) * 3, jitter=0.0)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    x, v, tet = workload(box, om)
    q, m, w = W.Q_E, W.M_E, 1.0e3
    osim = oracle_lib.OracleSim(om, oracle_lib.OracleConfig(dt=DT, pusher="boris"))
    osim.add_species(q, m, w, x, v, tet)
    osim.init()
    pm = F.Mesh(box.xyz, box.tets)
    gsim = F.Sim(pm, DT, pusher="boris", precision=precision)
    gsim.particles_load(0, q, m, w, x, v, tet)
    gsim.init()
    for s in (osim, gsim):
        s.set_field("E", np.zeros(om.n_edges))
        s.set_field("B", np.zeros(om.n_faces))
    # MIXED keeps FP32 state and 2^-24 fixed-point barycentrics: positions agree
    # to FP32 rounding of the box, deposits to the tolerance of the other
    # MIXED particle-phase test
    tol = 1e-12 if precision == "plain" else 4e-7
    dtol = 1e-12 if precision == "plain" else 2e-5
    for it in range(3):
        prev = {s: (s.field("RHO"), s.field("WALL")) for s in (osim, gsim)}
        osim.particle_phase()
        gsim.particle_phase()
        for s in (osim, gsim):
            assert continuity_defect(om, *prev[s], s.field("RHO"), s.field("WALL"), s.field("DG")) <= 1e-12, it
        gx, gv, gt, gid = gsim.particles()
        ox, ov, ot, alive = osim.particles()
        ids = np.where(alive)[0]
        assert np.array_equal(gid, ids), (it, len(gid), len(ids))
        assert np.all(np.isfinite(gx)) and np.all(np.isfinite(gv))
        assert np.abs(gx - ox[ids]).max() <= tol, it
        assert np.abs(gv - ov[ids]).max() <= tol * np.abs(ov).max(), it
        assert np.all(tet_contains(box, gt, gx, 1e-12 if precision == "plain" else 1e-6)), it
        for name in ("DG", "RHO", "WALL"):
            a, b = gsim.field(name), osim.field(name)
            assert np.abs(a - b).max() <= dtol * max(np.abs(b).max(), 1e-300), (it, name)
    assert 0 < alive.sum() < alive.size          # some paths reached the walls, some did not
    assert gsim.diag()["status"] == 0
