"""FP64 oracle of the learned edge preconditioner (test infrastructure only).

The paper has no learned component.  This project adds one to the Newmark
solve of Sec. III (the CG step the paper leaves open): a small message-passing
network on the graph of the interior-edge system A = M + dt^2/4 K whose output
is used as the preconditioner of a flexible CG.  Its definition, restated here
in plain numpy/scipy at FP64 so that the GPU kernels can be checked against it:

  d_i = A_ii,  Ahat = D^-1/2 A D^-1/2 (unit diagonal),  a_i = log d_i - mean(log d)
  rho = sqrt(mean_i r_i^2 / d_i),   x_i = r_i / (sqrt(d_i) rho)
  h0_i = relu(U x_i + V a_i + c)                               (R^32)
  for l = 1, 2, 3:
      g_l = Ahat h_{l-1}                                        (aggregation)
      h_l,i = relu(W_l h_{l-1,i} + Q_l g_l,i + b_l)
  y_i = o . h_3,i + d0
  z_i = rho (x_i + y_i) / sqrt(d_i)          (= the Jacobi step when y = 0)

Training loss for one residual r (the A-norm error of z as an approximation
of A^-1 r, up to the constant r^T A^-1 r, so it needs no solve):

  L(z) = (z^T A z - 2 z^T r) / (r^T D^-1 r)

Parameters are one float32 vector theta (layout in ``OFFSETS``); the network
computes with their bfloat16 roundings (``bf16``).  relu'(0) = 0.

Only the tests may import this module.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np
import scipy.sparse as sp

H = 32
LAYERS = 3


def _layout() -> Dict[str, Tuple[int, Tuple[int, ...]]]:
    out, off = {}, 0

    def add(name, shape):
        nonlocal off
        size = int(np.prod(shape))
        out[name] = (off, shape)
        off += size

    add("U", (H,))
    add("V", (H,))
    add("c", (H,))
    for l in range(1, LAYERS + 1):
        add(f"W{l}", (H, H))     # W[f, k]: output feature f, input feature k
        add(f"Q{l}", (H, H))
        add(f"b{l}", (H,))
    add("o", (H,))
    add("d0", (1,))
    out["_size"] = (off, ())
    return out


OFFSETS = _layout()
N_PARAMS = OFFSETS["_size"][0]


def unpack(theta: np.ndarray) -> Dict[str, np.ndarray]:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS
    return {k: theta[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFFSETS.items() if k != "_size"}


def bf16(theta32: np.ndarray) -> np.ndarray:
    """bfloat16 rounding (to nearest, ties to even) of float32 values, as float64.

    A bfloat16 is the upper 16 bits of a float32; rounding adds half an ulp
    of the kept part plus the kept part's lowest bit, then truncates."""
    bits = np.asarray(theta32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    keep_lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + keep_lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def relu(v):
    return np.maximum(v, 0.0)


class EdgeNet:
    """The network on one SPD matrix A (scipy sparse, the interior-edge system)."""

    def __init__(self, A):
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.d = self.A.diagonal().copy()
        assert np.all(self.d > 0)
        s = 1.0 / np.sqrt(self.d)
        self.Ahat = sp.diags(s) @ self.A @ sp.diags(s)
        logd = np.log(self.d)
        self.a = logd - logd.mean()
        self.n = self.A.shape[0]

    def forward(self, r: np.ndarray, theta: np.ndarray):
        """z and the activations the backward pass needs (theta: float64 values
        the network computes with, i.e. already rounded to bfloat16)."""
        p = unpack(theta)
        r = np.asarray(r, dtype=np.float64)
        rho = np.sqrt(np.mean(r * r / self.d))
        if rho == 0.0:
            return np.zeros(self.n), None
        x = r / (np.sqrt(self.d) * rho)
        pre = [np.outer(x, p["U"]) + np.outer(self.a, p["V"]) + p["c"]]
        h = [relu(pre[0])]
        g = [None]
        for l in range(1, LAYERS + 1):
            g.append(self.Ahat @ h[l - 1])
            pre.append(h[l - 1] @ p[f"W{l}"].T + g[l] @ p[f"Q{l}"].T + p[f"b{l}"])
            h.append(relu(pre[l]))
        y = h[LAYERS] @ p["o"] + p["d0"][0]
        z = rho * (x + y) / np.sqrt(self.d)
        return z, {"rho": rho, "x": x, "pre": pre, "h": h, "g": g, "y": y}

    def loss(self, r: np.ndarray, z: np.ndarray) -> float:
        nrm = float(np.sum(r * r / self.d))
        return float(z @ (self.A @ z) - 2.0 * z @ r) / nrm

    def backward(self, r: np.ndarray, theta: np.ndarray, z: np.ndarray, cache) -> np.ndarray:
        """dL/dtheta (float64, layout of theta)."""
        p = unpack(theta)
        grad = {k: np.zeros(s) for k, (o, s) in OFFSETS.items() if k != "_size"}
        nrm = float(np.sum(r * r / self.d))
        gz = 2.0 * (self.A @ z - r) / nrm
        gy = gz * cache["rho"] / np.sqrt(self.d)
        h, g, pre = cache["h"], cache["g"], cache["pre"]
        grad["o"] = h[LAYERS].T @ gy
        grad["d0"] = np.array([gy.sum()])
        dh = np.outer(gy, p["o"])
        for l in range(LAYERS, 0, -1):
            dpre = dh * (pre[l] > 0)
            grad[f"W{l}"] = dpre.T @ h[l - 1]
            grad[f"Q{l}"] = dpre.T @ g[l]
            grad[f"b{l}"] = dpre.sum(axis=0)
            dh = dpre @ p[f"W{l}"] + self.Ahat @ (dpre @ p[f"Q{l}"])
        dpre0 = dh * (pre[0] > 0)
        grad["U"] = dpre0.T @ cache["x"]
        grad["V"] = dpre0.T @ self.a
        grad["c"] = dpre0.sum(axis=0)
        out = np.zeros(N_PARAMS)
        for k, (o, s) in OFFSETS.items():
            if k != "_size":
                out[o:o + int(np.prod(s))] = grad[k].ravel()
        return out

    def loss_and_grad(self, r: np.ndarray, theta: np.ndarray):
        z, cache = self.forward(r, theta)
        if cache is None:
            return 0.0, np.zeros(N_PARAMS), z
        return self.loss(r, z), self.backward(r, theta, z, cache), z


def interior_system(mesh, dt: float):
    """A = M + dt^2/4 K restricted to the interior edges (global edge order),
    from the oracle's own matrices, and the interior edge ids."""
    n = mesh.n_edges
    rp, col, val = mesh.matrix("M")
    M = sp.csr_matrix((val, col, rp), shape=(n, n))
    rp, col, val = mesh.matrix("K")
    K = sp.csr_matrix((val, col, rp), shape=(n, n))
    eb, _, _ = mesh.flags()
    ids = np.where(eb == 0)[0]
    A = (M + 0.25 * dt * dt * K).tocsr()[ids][:, ids]
    return sp.csr_matrix(A), ids
