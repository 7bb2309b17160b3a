"""Writes dt_cfl.json: the explicit (leap-frog) stability limit of the meshes
the workloads use, dt_CFL = 2 / sqrt(lambda_max(M^-1 K)) on interior edges,
with M and K assembled by the oracle only.  Sec. IV.B defines the time steps
of the beam runs as multiples of this limit ("the largest stable step size in
a leap frog time marching method for the given mesh").

Small meshes use a dense generalized eigensolver; larger ones LOBPCG on the
same pencil scaled to unit diagonal.  kappa = dt_CFL * c / h.

Run:  python tests/golden/make_dt_cfl.py
"""
import json
import os
import sys
import warnings

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as sla

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle.oracle import OracleMesh  # noqa: E402
from paper_2102_06248_gb300 import workloads as W  # noqa: E402


def lambda_max(box, dense):
    m = OracleMesh(box.xyz, box.tets)
    eb, _, _ = m.flags()
    ii = np.where(eb == 0)[0]
    mats = []
    for w in ("M", "K"):
        rp, c, v = m.matrix(w)
        mats.append(sp.csr_matrix((v, c, rp), shape=(m.n_edges, m.n_edges))[ii][:, ii])
    M, K = mats
    if dense:
        return float(sl.eigh(K.toarray(), M.toarray(), eigvals_only=True).max())
    d = 1.0 / np.sqrt(M.diagonal())
    S = sp.diags(d)
    Ms, Ks = S @ M @ S, S @ K @ S
    scale = Ks.diagonal().max()
    X = np.random.default_rng(0).standard_normal((len(ii), 8))
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        lam, _ = sla.lobpcg(Ks / scale, X, B=Ms, largest=True, tol=1e-10, maxiter=3000)
    return float(lam.max() * scale)


def entry(box, dense):
    lmax = lambda_max(box, dense)
    dt = 2.0 / np.sqrt(lmax)
    return {"cells": list(box.cells), "size_m": list(box.size), "h_m": box.h, "dt_cfl_s": dt,
            "kappa": dt * W.C0 / box.h}


def main():
    out = {"definition": "dt_CFL = 2/sqrt(lambda_max(M^-1 K)) on interior edges (Sec. IV.B); kappa = dt_CFL c / h"}
    out["thermal_plasma_cube_6^3"] = entry(W.kuhn_box((6, 6, 6), (1.0, 1.0, 1.0)), dense=True)
    # kappa of the unjittered Kuhn lattice (converged to ~1e-3 by 16^3) and of
    # the 20%-jittered lattice; larger meshes use dt = kappa h / c
    out["kuhn_lattice_16^3"] = entry(W.kuhn_box((16, 16, 16), (1.0, 1.0, 1.0)), dense=False)
    out["kuhn_lattice_16^3_jitter0.2"] = entry(
        W.kuhn_box((16, 16, 16), (1.0, 1.0, 1.0), jitter=0.2, seed=1004), dense=False)
    with open(os.path.join(HERE, "dt_cfl.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
