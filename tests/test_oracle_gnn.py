"""Pins of the FP64 oracle of the learned edge preconditioner.

The network is a project addition (the paper has none), so its pins are
mathematical: the backward pass against central finite differences of the
loss, the Jacobi special case, positive scale invariance, permutation
equivariance of the graph operations, the closed form of the loss at the exact
solve, and the bfloat16 rounding rule on hand-made bit patterns.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import gnn_oracle as G
from paper_2102_06248_gb300 import workloads as W

DT = 1.3017565848335032e-10   # tests/golden/dt_cfl.json, thermal_plasma_cube_6^3


@pytest.fixture(scope="module")
def system(oracle_lib):
    box = W.kuhn_box((3, 3, 3), (1.0, 1.0, 1.0), jitter=0.15, seed=4)
    om = oracle_lib.OracleMesh(box.xyz, box.tets)
    A, ids = G.interior_system(om, 2 * DT)
    return A, ids


def random_theta(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    th = rng.normal(0.0, scale, G.N_PARAMS).astype(np.float32)
    return th


def test_layout_size():
    assert G.N_PARAMS == 3 * 32 + 3 * (2 * 32 * 32 + 32) + 32 + 1


def test_bf16_rounding_rule():
    # 1 + 2^-8 is halfway between two bfloat16 values: ties go to the even one (1.0)
    # 1 + 3*2^-8 is halfway too: the even neighbour is 1 + 2^-6... rounding up
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5, 3.0e-39],
                    dtype=np.float32)
    out = G.bf16(vals)
    assert out[0] == 1.0
    assert out[1] == 1.0
    assert out[2] == 1.0 + 2.0 ** -6
    assert out[3] == 1.0 + 2.0 ** -7
    assert out[4] == -2.5
    # every result is a float32 whose low 16 bits are zero
    assert np.all((out.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_zero_output_layer_is_jacobi(system):
    A, _ = system
    net = G.EdgeNet(A)
    th = random_theta(1).astype(np.float64)
    p = G.OFFSETS
    th[p["o"][0]:p["o"][0] + 32] = 0.0
    th[p["d0"][0]] = 0.0
    r = np.random.default_rng(2).normal(size=A.shape[0])
    z, _ = net.forward(r, th)
    np.testing.assert_allclose(z, r / A.diagonal(), rtol=1e-14, atol=0)


def test_positive_scale_invariance(system):
    A, _ = system
    net = G.EdgeNet(A)
    th = G.bf16(random_theta(3))
    r = np.random.default_rng(4).normal(size=A.shape[0])
    z1, _ = net.forward(r, th)
    z2, _ = net.forward(7.25 * r, th)
    np.testing.assert_allclose(z2, 7.25 * z1, rtol=1e-12, atol=1e-14 * np.abs(z2).max())


def test_permutation_equivariance(system):
    A, _ = system
    n = A.shape[0]
    perm = np.random.default_rng(5).permutation(n)
    P = sp.csr_matrix((np.ones(n), (np.arange(n), perm)), shape=(n, n))
    Ap = P @ A @ P.T
    th = G.bf16(random_theta(6))
    r = np.random.default_rng(7).normal(size=n)
    z, _ = G.EdgeNet(A).forward(r, th)
    zp, _ = G.EdgeNet(Ap).forward(P @ r, th)
    np.testing.assert_allclose(zp, P @ z, rtol=1e-11, atol=1e-14 * np.abs(z).max())


def test_loss_closed_form_at_exact_solve(system):
    A, _ = system
    net = G.EdgeNet(A)
    r = np.random.default_rng(8).normal(size=A.shape[0])
    e = spla.spsolve(sp.csc_matrix(A), r)
    nrm = np.sum(r * r / A.diagonal())
    # at z = A^-1 r the loss is -r^T A^-1 r / (r^T D^-1 r), and any other z is higher
    assert net.loss(r, e) == pytest.approx(-(r @ e) / nrm, rel=1e-10)
    dz = np.random.default_rng(9).normal(size=A.shape[0]) * 1e-3 * np.abs(e).max()
    assert net.loss(r, e + dz) > net.loss(r, e)


def test_backward_matches_central_differences(system):
    A, _ = system
    net = G.EdgeNet(A)
    th = G.bf16(random_theta(10, scale=0.4))
    r = np.random.default_rng(11).normal(size=A.shape[0])
    L, grad, _ = net.loss_and_grad(r, th)
    rng = np.random.default_rng(12)
    # every parameter group, a few entries each
    picks = []
    for k, (o, s) in G.OFFSETS.items():
        if k == "_size":
            continue
        size = int(np.prod(s))
        picks += list(o + rng.choice(size, size=min(size, 4), replace=False))
    for i in picks:
        h = 1e-6 * max(1.0, abs(th[i]))
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        zp, _ = net.forward(r, tp)
        zm, _ = net.forward(r, tm)
        fd = (net.loss(r, zp) - net.loss(r, zm)) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(grad[i])) + 1e-7, (i, fd, grad[i])
