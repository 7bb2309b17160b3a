"""C-ABI checks that need no GPU: the library loads and exports every entry
point include/fempic.h declares, and pic_mesh_create (host-side build)
produces exactly the oracle's edges, faces and G/C/D incidence (integer work,
bit-exact), and rejects malformed meshes with PIC_ERR_MESH / INVALID_ARG."""
import os
import re

import numpy as np
import pytest

from paper_2102_06248_gb300 import fempic as F
from paper_2102_06248_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    hdr = open(os.path.join(ROOT, "include", "fempic.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(pic_\w+)\s*\(", hdr, re.M)))


def test_library_exports_every_declared_symbol():
    lib = F.load()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("cells,jit", [((6, 6, 6), 0.0), ((4, 3, 5), 0.2), ((2, 2, 2), 0.0)])
def test_mesh_entities_and_incidence_match_oracle(oracle_lib, cells, jit):
    box = W.kuhn_box(cells, tuple(0.1 * c for c in cells), jitter=jit, seed=5)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    pm = F.Mesh(box.xyz, box.tets)
    assert (pm.n_nodes, pm.n_edges, pm.n_faces, pm.n_tets, pm.n_int_edges, pm.n_int_nodes) == \
        (om.n_nodes, om.n_edges, om.n_faces, om.n_tets, om.n_int_edges, om.n_int_nodes)
    e, f = pm.entities()
    assert np.array_equal(e, om.edges()) and np.array_equal(f, om.faces())
    for which in "GCD":
        pr, pc, pv = pm.incidence(which)
        orr, oc, ov = om.incidence(which)
        # same sparse matrix (entries may be listed in another order)
        a = sorted(zip(pr.tolist(), pc.tolist(), pv.tolist()))
        b = sorted(zip(orr.tolist(), oc.tolist(), ov.tolist()))
        assert a == b, which


def test_supplied_incidence_is_validated(oracle_lib):
    box = W.kuhn_box((3, 3, 3), (0.3, 0.3, 0.3))
    pm = F.Mesh(box.xyz, box.tets)
    e, f = pm.entities()
    inc = {w: np.concatenate(pm.incidence(w)) for w in "GCD"}
    F.Mesh(box.xyz, box.tets, edges=e, faces=f, incidence=inc)     # accepted as is
    bad = dict(inc)
    C = inc["C"].copy()
    n = C.size // 3
    C[2 * n] = -C[2 * n]                                            # flip one curl sign
    bad["C"] = C
    with pytest.raises(F.PicError) as ei:
        F.Mesh(box.xyz, box.tets, incidence=bad)
    assert ei.value.code == 2
    e2 = e.copy()
    e2[[0, 1]] = e2[[1, 0]]
    with pytest.raises(F.PicError):
        F.Mesh(box.xyz, box.tets, edges=e2)


def test_malformed_meshes_are_rejected():
    box = W.kuhn_box((2, 2, 2), (1.0, 1.0, 1.0))
    t = box.tets.copy()
    t[3, 1] = t[3, 0]                                   # repeated node
    with pytest.raises(F.PicError) as ei:
        F.Mesh(box.xyz, t)
    assert ei.value.code == 2
    t = box.tets.copy()
    t[0, 0] = box.xyz.shape[0] + 5                      # node id out of range
    with pytest.raises(F.PicError):
        F.Mesh(box.xyz, t)
    xyz = box.xyz.copy()
    flat = box.tets[0]
    xyz[flat[3]] = xyz[flat[0]] + 0.5 * (xyz[flat[1]] - xyz[flat[0]]) + 0.5 * (xyz[flat[2]] - xyz[flat[0]])
    with pytest.raises(F.PicError):                      # a flat (zero-volume) tet
        F.Mesh(xyz, box.tets)
    with pytest.raises(F.PicError) as ei:
        F.Mesh(np.zeros((0, 3)), np.zeros((0, 4), dtype=np.int32))
    assert ei.value.code == 1
    # three tets on one face: non-manifold
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 1.0]])
    tets = np.array([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 5]], dtype=np.int32)
    with pytest.raises(F.PicError):
        F.Mesh(xyz, tets)


@pytest.mark.parametrize("walls", [W.BOX_WALLS, ("z0", "z1"), ("x1",)])
def test_absorbing_walls_unknowns_match_oracle(oracle_lib, walls):
    """With absorbing wall faces (Sec. II.A, Eq. impedanceBC) the edges held at
    zero are exactly those on conducting faces: the host-side mesh build and
    the oracle agree on how many unknowns the field update has."""
    box = W.kuhn_box((3, 4, 3), (0.3, 0.4, 0.3), jitter=0.1, seed=8)
    bc = W.box_wall_bc(box, walls)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    om.set_absorbing(bc)
    pm = F.Mesh(box.xyz, box.tets, wall_bc=bc)
    plain = F.Mesh(box.xyz, box.tets)
    assert pm.n_int_edges == om.n_int_edges > plain.n_int_edges
    assert pm.n_int_nodes == om.n_int_nodes == plain.n_int_nodes
    with pytest.raises(F.PicError):
        F.Mesh(box.xyz, box.tets, wall_bc=bc[:-1])
