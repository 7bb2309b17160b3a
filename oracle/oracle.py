"""ctypes binding of the C oracle (fempic_oracle.c); test infrastructure only.

``build()`` compiles the oracle with gcc (-ffp-contract=off, so that x86 and
Arm hosts produce the same bits) into ``oracle/_build/libfempic_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
from typing import Dict, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fempic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfempic_oracle.so")


def lib_path() -> str:
    return _LIB


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(_BUILD, exist_ok=True)
    hdr = os.path.join(_HERE, "fempic_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(hdr))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "step", "continuity_abs", "gauss_abs", "rho_max", "divb_abs", "cg_iters", "cg_relres",
        "n_alive", "energy_e", "energy_b", "energy_k", "status")]


class _Config(C.Structure):
    _fields_ = [("form", C.c_int), ("pusher", C.c_int), ("dt", C.c_double), ("b0", C.c_double * 3),
                ("cg_tol", C.c_double), ("cg_max_iters", C.c_int), ("init_tol", C.c_double),
                ("rho_background", C.c_double), ("walk_cap", C.c_int),
                ("gradient_completion", C.c_int), ("completion_tol", C.c_double),
                ("current_form", C.c_int), ("curved_path", C.c_int)]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    lib.orc_mesh_new.restype = P
    lib.orc_mesh_new.argtypes = [C.c_int, dp, C.c_int, ip, C.c_char_p, C.c_int]
    lib.orc_mesh_free.argtypes = [P]
    for name in ("orc_mesh_counts", "orc_mesh_edges", "orc_mesh_faces"):
        getattr(lib, name).argtypes = [P, ip]
    for name in ("orc_mesh_G", "orc_mesh_C", "orc_mesh_D"):
        getattr(lib, name).argtypes = [P, ip, ip, ip]
    lib.orc_mesh_tet_data.argtypes = [P, ip, ip, ip]
    lib.orc_mesh_flags.argtypes = [P, ip, ip, ip]
    lib.orc_mesh_geom.argtypes = [P, dp, dp]
    lib.orc_mesh_set_absorbing.argtypes = [P, ip]
    lib.orc_mesh_set_absorbing.restype = C.c_int
    lib.orc_matrix_nnz.argtypes = [P, C.c_int]
    lib.orc_matrix_nnz.restype = C.c_int
    lib.orc_matrix_csr.argtypes = [P, C.c_int, ip, ip, dp]
    lib.orc_lambda.argtypes = [P, C.c_int, dp, dp]
    lib.orc_gather.argtypes = [P, C.c_int, dp, dp, dp, dp, dp]
    lib.orc_segment_w1.argtypes = [P, C.c_int, dp, dp, dp]
    lib.orc_walk.argtypes = [P, C.c_int, dp, dp, C.c_int, ip, dp, ip, ip]
    lib.orc_walk.restype = C.c_int
    lib.orc_boris.argtypes = [C.c_double, C.c_double, dp, dp, dp]
    lib.orc_sim_new.restype = P
    lib.orc_sim_new.argtypes = [P, C.POINTER(_Config)]
    lib.orc_sim_free.argtypes = [P]
    lib.orc_add_species.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, ip]
    lib.orc_inject.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, ip]
    lib.orc_inject.restype = C.c_int
    for name in ("orc_init", "orc_step", "orc_particle_phase", "orc_add_species"):
        getattr(lib, name).restype = C.c_int
    lib.orc_init.argtypes = [P]
    lib.orc_set_background_charge.argtypes = [P, dp]
    lib.orc_set_background_charge.restype = C.c_int
    lib.orc_set_ab_history.argtypes = [P, C.c_int, dp, dp]
    lib.orc_set_ab_history.restype = C.c_int
    lib.orc_set_position_history.argtypes = [P, C.c_int, dp]
    lib.orc_set_position_history.restype = C.c_int
    lib.orc_step.argtypes = [P]
    lib.orc_particle_phase.argtypes = [P]
    lib.orc_n_particles.argtypes = [P]
    lib.orc_n_particles.restype = C.c_int
    lib.orc_get_particles.argtypes = [P, dp, dp, ip, ip]
    lib.orc_get_field.argtypes = [P, C.c_int, dp]
    lib.orc_set_field.argtypes = [P, C.c_int, dp]
    lib.orc_get_diag.argtypes = [P, C.POINTER(_Diag)]
    lib.orc_sim_error.argtypes = [P]
    lib.orc_sim_error.restype = C.c_char_p
    _lib = lib
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


FIELDS = {"E": 0, "E_PREV": 1, "B": 2, "G": 3, "RHO": 4, "WALL": 5, "PHI": 6, "DG": 7, "RHO_BG": 8,
          "B_PREV": 9, "G_PREV": 10}
MATS = {"M": 0, "K": 1, "H": 2, "L": 3, "I": 4}


class OracleMesh:
    """Mesh entities, incidence, geometry and Hodge matrices built by the oracle."""

    def __init__(self, xyz: np.ndarray, tets: np.ndarray):
        lib = _load()
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        err = C.create_string_buffer(256)
        h = lib.orc_mesh_new(self.xyz.shape[0], _dp(self.xyz), self.tets.shape[0], _ip(self.tets), err, 256)
        if not h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self._h = h
        c = np.zeros(6, dtype=np.int32)
        lib.orc_mesh_counts(h, _ip(c))
        (self.n_nodes, self.n_edges, self.n_faces, self.n_tets,
         self.n_int_edges, self.n_int_nodes) = (int(x) for x in c)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_mesh_free(self._h)
            self._h = None

    def edges(self) -> np.ndarray:
        out = np.zeros((self.n_edges, 2), dtype=np.int32)
        _lib.orc_mesh_edges(self._h, _ip(out))
        return out

    def faces(self) -> np.ndarray:
        out = np.zeros((self.n_faces, 3), dtype=np.int32)
        _lib.orc_mesh_faces(self._h, _ip(out))
        return out

    def incidence(self, which: str):
        """(rows, cols, vals) of G, C or D."""
        n = {"G": 2 * self.n_edges, "C": 3 * self.n_faces, "D": 4 * self.n_tets}[which]
        r = np.zeros(n, dtype=np.int32)
        c = np.zeros(n, dtype=np.int32)
        v = np.zeros(n, dtype=np.int32)
        getattr(_lib, "orc_mesh_" + which)(self._h, _ip(r), _ip(c), _ip(v))
        return r, c, v

    def incidence_dense(self, which: str) -> np.ndarray:
        shape = {"G": (self.n_edges, self.n_nodes), "C": (self.n_faces, self.n_edges),
                 "D": (self.n_tets, self.n_faces)}[which]
        r, c, v = self.incidence(which)
        out = np.zeros(shape, dtype=np.int64)
        np.add.at(out, (r, c), v)
        return out

    def tet_data(self):
        te = np.zeros((self.n_tets, 6), dtype=np.int32)
        tf = np.zeros((self.n_tets, 4), dtype=np.int32)
        tn = np.zeros((self.n_tets, 4), dtype=np.int32)
        _lib.orc_mesh_tet_data(self._h, _ip(te), _ip(tf), _ip(tn))
        return te, tf, tn

    def flags(self):
        eb = np.zeros(self.n_edges, dtype=np.int32)
        nb = np.zeros(self.n_nodes, dtype=np.int32)
        fb = np.zeros(self.n_faces, dtype=np.int32)
        _lib.orc_mesh_flags(self._h, _ip(eb), _ip(nb), _ip(fb))
        return eb, nb, fb

    def geom(self):
        g = np.zeros((self.n_tets, 4, 3))
        v = np.zeros(self.n_tets)
        _lib.orc_mesh_geom(self._h, _dp(g), _dp(v))
        return g, v

    def matrix(self, which: str):
        """(rowptr, col, val) CSR of M, K, H or L (= G^T M G)."""
        w = MATS[which]
        nnz = _lib.orc_matrix_nnz(self._h, w)
        n = {"M": self.n_edges, "K": self.n_edges, "I": self.n_edges, "H": self.n_faces, "L": self.n_nodes}[which]
        rp = np.zeros(n + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        _lib.orc_matrix_csr(self._h, w, _ip(rp), _ip(col), _dp(val))
        return rp, col, val

    def matrix_dense(self, which: str) -> np.ndarray:
        rp, col, val = self.matrix(which)
        n = rp.size - 1
        out = np.zeros((n, n))
        for r in range(n):
            out[r, col[rp[r]:rp[r + 1]]] += val[rp[r]:rp[r + 1]]
        return out

    def set_absorbing(self, tet_face_bc: np.ndarray):
        """Wall conditions per tet face (1 absorbing, 0 conducting), [n_tets, 4]
        with entry k the face opposite the tet's k-th vertex; call before
        creating simulations."""
        bc = np.ascontiguousarray(tet_face_bc, dtype=np.int32).reshape(-1)
        if bc.size != 4 * self.n_tets:
            raise ValueError("tet_face_bc needs 4 entries per tet")
        _lib.orc_mesh_set_absorbing(self._h, _ip(bc))
        c = np.zeros(6, dtype=np.int32)
        _lib.orc_mesh_counts(self._h, _ip(c))
        self.n_int_edges = int(c[4])

    def lam(self, tet: int, r: Sequence[float]) -> np.ndarray:
        out = np.zeros(4)
        rr = np.ascontiguousarray(r, dtype=np.float64)
        _lib.orc_lambda(self._h, int(tet), _dp(rr), _dp(out))
        return out

    def gather(self, tet: int, r, e: np.ndarray, b: np.ndarray):
        E = np.zeros(3)
        B = np.zeros(3)
        rr = np.ascontiguousarray(r, dtype=np.float64)
        e = np.ascontiguousarray(e, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        _lib.orc_gather(self._h, int(tet), _dp(rr), _dp(e), _dp(b), _dp(E), _dp(B))
        return E, B

    def segment_w1(self, tet: int, S, X) -> np.ndarray:
        out = np.zeros(6)
        s = np.ascontiguousarray(S, dtype=np.float64)
        x = np.ascontiguousarray(X, dtype=np.float64)
        _lib.orc_segment_w1(self._h, int(tet), _dp(s), _dp(x), _dp(out))
        return out

    def walk(self, tet: int, P, Q, cap: int = 64):
        tl = np.zeros(cap, dtype=np.int32)
        pts = np.zeros((cap, 3))
        nseg = np.zeros(1, dtype=np.int32)
        ab = np.zeros(1, dtype=np.int32)
        p = np.ascontiguousarray(P, dtype=np.float64)
        q = np.ascontiguousarray(Q, dtype=np.float64)
        rc = _lib.orc_walk(self._h, int(tet), _dp(p), _dp(q), cap, _ip(tl), _dp(pts), _ip(nseg), _ip(ab))
        n = int(nseg[0])
        return rc, tl[:n].copy(), pts[:n].copy(), bool(ab[0])


def boris(qm: float, dt: float, E, B, v) -> np.ndarray:
    lib = _load()
    vv = np.array(v, dtype=np.float64)
    e = np.ascontiguousarray(E, dtype=np.float64)
    b = np.ascontiguousarray(B, dtype=np.float64)
    lib.orc_boris(qm, dt, _dp(e), _dp(b), _dp(vv))
    return vv


@dataclasses.dataclass
class OracleConfig:
    dt: float
    form: str = "we"             # "we" | "mfem" | "bd"
    pusher: str = "boris"        # "boris" | "ab1".."ab5"
    b0: Sequence[float] = (0.0, 0.0, 0.0)
    cg_tol: float = 1e-10
    cg_max_iters: int = 10000
    init_tol: float = 1e-14
    rho_background: float = 0.0
    walk_cap: int = 64
    gradient_completion: bool = True
    completion_tol: float = 1e-16
    current: str = "gbar"        # "gbar" (the paper's method) | "point" (negative control)
    curved_path: bool = False    # Lagrange path through the newest positions (Adams-Bashforth only)

    def to_c(self) -> _Config:
        c = _Config()
        c.form = {"we": 0, "mfem": 1, "bd": 2}[self.form]
        c.current_form = {"gbar": 0, "point": 1}[self.current]
        c.curved_path = int(self.curved_path)
        c.pusher = 0 if self.pusher == "boris" else int(self.pusher[2:])
        c.dt = self.dt
        for i in range(3):
            c.b0[i] = self.b0[i]
        c.cg_tol = self.cg_tol
        c.cg_max_iters = self.cg_max_iters
        c.init_tol = self.init_tol
        c.rho_background = self.rho_background
        c.walk_cap = self.walk_cap
        c.gradient_completion = int(self.gradient_completion)
        c.completion_tol = self.completion_tol
        return c


class OracleSim:
    def __init__(self, mesh: OracleMesh, cfg: OracleConfig):
        self.mesh = mesh
        self.cfg = cfg
        self._c = cfg.to_c()
        self._h = _lib.orc_sim_new(mesh._h, C.byref(self._c))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_sim_free(self._h)
            self._h = None

    def _check(self, rc: int, what: str):
        if rc:
            raise RuntimeError(f"oracle {what} failed ({rc}): {_lib.orc_sim_error(self._h).decode()}")

    def add_species(self, q: float, m: float, w: float, x: np.ndarray, v: np.ndarray, tet: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        tet = np.ascontiguousarray(tet, dtype=np.int32)
        self._check(_lib.orc_add_species(self._h, q, m, w, x.shape[0], _dp(x), _dp(v), _ip(tet)), "add_species")

    def inject(self, q: float, m: float, w: float, x: np.ndarray, v: np.ndarray, tet: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        v = np.ascontiguousarray(v, dtype=np.float64)
        tet = np.ascontiguousarray(tet, dtype=np.int32)
        self._check(_lib.orc_inject(self._h, q, m, w, x.shape[0], _dp(x), _dp(v), _ip(tet)), "inject")

    def set_background_charge(self, rho_nodes: np.ndarray):
        a = np.ascontiguousarray(rho_nodes, dtype=np.float64)
        self._check(_lib.orc_set_background_charge(self._h, _dp(a)), "set_background_charge")

    def init(self):
        self._check(_lib.orc_init(self._h), "init")

    def set_ab_history(self, a_hist: np.ndarray, v_hist: np.ndarray):
        a = np.ascontiguousarray(a_hist, dtype=np.float64)
        v = np.ascontiguousarray(v_hist, dtype=np.float64)
        self._check(_lib.orc_set_ab_history(self._h, a.shape[0], _dp(a), _dp(v)), "set_ab_history")

    def set_position_history(self, r_hist: np.ndarray):
        r = np.ascontiguousarray(r_hist, dtype=np.float64)
        self._check(_lib.orc_set_position_history(self._h, r.shape[0], _dp(r)), "set_position_history")

    def step(self, n: int = 1):
        for _ in range(n):
            self._check(_lib.orc_step(self._h), "step")

    def particle_phase(self):
        self._check(_lib.orc_particle_phase(self._h), "particle_phase")

    def particles(self):
        n = _lib.orc_n_particles(self._h)
        x = np.zeros((n, 3))
        v = np.zeros((n, 3))
        t = np.zeros(n, dtype=np.int32)
        a = np.zeros(n, dtype=np.int32)
        _lib.orc_get_particles(self._h, _dp(x), _dp(v), _ip(t), _ip(a))
        return x, v, t, a.astype(bool)

    def field(self, which: str) -> np.ndarray:
        n = {"E": self.mesh.n_edges, "E_PREV": self.mesh.n_edges, "G": self.mesh.n_edges,
             "G_PREV": self.mesh.n_edges, "DG": self.mesh.n_edges, "B": self.mesh.n_faces,
             "B_PREV": self.mesh.n_faces}.get(which, self.mesh.n_nodes)
        out = np.zeros(n)
        _lib.orc_get_field(self._h, FIELDS[which], _dp(out))
        return out

    def set_field(self, which: str, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=np.float64)
        _lib.orc_set_field(self._h, FIELDS[which], _dp(a))

    def diag(self) -> Dict[str, float]:
        d = _Diag()
        _lib.orc_get_diag(self._h, C.byref(d))
        return {n: getattr(d, n) for n, _ in _Diag._fields_}


def from_workload(wl, dt: float, cg_tol: float = 1e-10, init_tol: float = 1e-14,
                  mesh: Optional[OracleMesh] = None, gradient_completion: bool = True,
                  completion_tol: float = 1e-16, current: str = "gbar") -> OracleSim:
    """Oracle simulation of a ``workloads.Workload`` with the given dt (its
    walls absorbing where ``wl.wall_bc`` says so)."""
    if mesh is None:
        mesh = OracleMesh(wl.mesh.xyz, wl.mesh.tets)
        if getattr(wl, "wall_bc", None) is not None:
            mesh.set_absorbing(wl.wall_bc)
    cfg = OracleConfig(dt=dt, form=wl.form, pusher=wl.pusher, b0=wl.b0, cg_tol=cg_tol,
                       init_tol=init_tol, rho_background=wl.rho_background,
                       gradient_completion=gradient_completion, completion_tol=completion_tol,
                       current=current)
    sim = OracleSim(mesh, cfg)
    for sp in wl.species:
        sim.add_species(sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    sim.init()
    return sim
