"""Python binding of the GB300 FEM-PIC C ABI (include/fempic.h).

Argument marshalling only: every step of the method runs in the CUDA library
``_build/libfempic_gb300.so``.  The functions below carry the C names; the
``Mesh`` and ``Sim`` classes wrap the handles.  PyTorch is used only for device
buffers (``on_device`` transfers) and streams.  There is no CPU fallback: if
the library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build

PIC_OK = 0
ERRORS = {1: "INVALID_ARG", 2: "MESH", 3: "OOM", 4: "PARTICLE_OUTSIDE", 5: "WALK_CAP",
          6: "CG_NO_CONVERGENCE", 7: "NAN", 8: "CUDA", 9: "OVERFLOW", 10: "STATE"}
FORMS = {"we": 0, "mfem": 1, "bd": 2}
PRECISIONS = {"plain": 0, "mixed": 1}
FIELDS = {"E": 0, "E_PREV": 1, "B": 2, "B_PREV": 3, "G": 4, "G_PREV": 5, "DG": 6, "RHO": 7,
          "WALL": 8, "RHO_BG": 9, "PHI": 10}


class PicError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: PIC_ERR_{ERRORS.get(code, code)}: {msg}")
        self.code = code


class pic_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("xyz", C.POINTER(C.c_double)), ("n_tets", C.c_int32),
                ("tets", C.POINTER(C.c_int32)), ("n_edges", C.c_int32), ("edges", C.POINTER(C.c_int32)),
                ("n_faces", C.c_int32), ("faces", C.POINTER(C.c_int32)), ("G_coo", C.POINTER(C.c_int32)),
                ("C_coo", C.POINTER(C.c_int32)), ("D_coo", C.POINTER(C.c_int32)),
                ("wall_bc", C.POINTER(C.c_int32))]


class pic_config(C.Structure):
    _fields_ = [("form", C.c_int32), ("pusher", C.c_int32), ("precision", C.c_int32),
                ("preconditioner", C.c_int32), ("dt", C.c_double), ("b0", C.c_double * 3),
                ("rho_background", C.c_double), ("cg_tol", C.c_double), ("cg_max_iters", C.c_int32),
                ("init_tol", C.c_double), ("completion_tol", C.c_double), ("walk_cap", C.c_int32),
                ("solver_blocks_per_sm", C.c_int32),
                ("max_species", C.c_int32), ("profile", C.c_int32), ("stream", C.c_void_p),
                ("barrier_spin_limit", C.c_int32), ("curved_path", C.c_int32)]


class pic_gnn_train_cfg(C.Structure):
    _fields_ = [("steps", C.c_int32), ("lr", C.c_double), ("samples", C.c_int32)]


GNN_PARAMS = 6369
PRECONDITIONERS = {"jacobi": 0, "gnn": 1}


class pic_batch_info_t(C.Structure):
    _fields_ = [("n_sims", C.c_int32), ("graph", C.c_int32), ("graph_steps", C.c_int32),
                ("solver_blocks_per_sm", C.c_int32), ("graph_launches", C.c_int64), ("eager_steps", C.c_int64),
                ("tune_ms", C.c_double * 3), ("solver_build", C.c_int32), ("completion_blocks_per_sm", C.c_int32),
                ("completion_build", C.c_int32), ("pad_", C.c_int32), ("tune_newmark_ms", C.c_double * 9),
                ("tune_completion_ms", C.c_double * 9)]

BATCH_BUILDS = ("64-register", "80-register", "40-register", "32-register")
BATCH_TUNE_CANDIDATES = ((2, 0), (3, 0), (4, 0), (2, 1), (3, 1), (5, 2), (6, 2), (7, 3), (8, 3))   # (blocks/SM, build)


class pic_diag(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "step", "continuity_abs", "gauss_abs", "rho_max", "divb_abs", "cg_iters", "cg_relres", "n_alive",
        "energy_e", "energy_b", "energy_k", "status", "completion_iters", "cg_iters_sum",
        "completion_iters_sum", "cg_outer")]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads the CUDA library (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise ImportError(f"GB300 library not built: {_build.LIB}")
        _build.build()
    lib = C.CDLL(_build.LIB)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    dp, ip, lp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig = {
        "pic_mesh_create": ([C.POINTER(pic_mesh_desc), C.POINTER(P)], I32),
        "pic_mesh_destroy": ([P], None),
        "pic_mesh_info": ([P, lp], I32),
        "pic_mesh_entities": ([P, ip, ip], I32),
        "pic_mesh_incidence": ([P, I32, ip, ip, ip], I32),
        "pic_config_default": ([C.POINTER(pic_config)], None),
        "pic_sim_create": ([P, C.POINTER(pic_config), C.POINTER(P)], I32),
        "pic_sim_destroy": ([P], None),
        "pic_particles_load": ([P, I32, D, D, D, I64, C.c_void_p, C.c_void_p, C.c_void_p, I32], I32),
        "pic_sim_init": ([P], I32),
        "pic_set_ab_history": ([P, I32, dp, dp], I32),
        "pic_step": ([P, I32], I32),
        "pic_particle_phase": ([P], I32),
        "pic_field_get": ([P, I32, C.c_void_p, I64, I32], I32),
        "pic_field_set": ([P, I32, C.c_void_p, I64, I32], I32),
        "pic_particles_count": ([P, lp], I32),
        "pic_particles_get": ([P, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, I64, lp, I32], I32),
        "pic_diagnostics_get": ([P, C.POINTER(pic_diag)], I32),
        "pic_sim_synchronize": ([P], I32),
        "pic_profile_get": ([P, dp, lp], I32),
        "pic_profile_reset": ([P], I32),
        "pic_launch_count": ([], I64),
        "pic_electrostatic_solve_noalloc": ([P, C.c_void_p, C.c_void_p, D, C.c_void_p], I32),
        "pic_gnn_train": ([P, C.POINTER(pic_gnn_train_cfg), dp], I32),
        "pic_particles_inject": ([P, I32, I64, dp, dp, ip], I32),
        "pic_batch_create": ([C.POINTER(P), I32, C.POINTER(P)], I32),
        "pic_batch_step": ([P, I32], I32),
        "pic_batch_info": ([P, C.POINTER(pic_batch_info_t)], I32),
        "pic_batch_destroy": ([P], None),
        "pic_gnn_get_weights": ([P, C.POINTER(C.c_float), I64], I32),
        "pic_gnn_set_weights": ([P, C.POINTER(C.c_float), I64], I32),
        "pic_gnn_apply": ([P, dp, dp], I32),
        "pic_gnn_loss_grad": ([P, dp, dp, dp], I32),
        "pic_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != PIC_OK:
        raise PicError(rc, where, (_lib.pic_last_error() or b"").decode())


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


class Mesh:
    """pic_mesh_create on node coordinates and tets (host arrays)."""

    def __init__(self, xyz: np.ndarray, tets: np.ndarray, edges: Optional[np.ndarray] = None,
                 faces: Optional[np.ndarray] = None, incidence: Optional[Dict[str, np.ndarray]] = None,
                 wall_bc: Optional[np.ndarray] = None):
        """wall_bc: optional [n_tets, 4] per tet face (entry k: the face opposite
        the tet's k-th vertex), 1 = first-order absorbing wall, 0 = conducting."""
        lib = load()
        self._xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        self._tets = np.ascontiguousarray(tets, dtype=np.int32)
        d = pic_mesh_desc()
        d.n_nodes = self._xyz.shape[0]
        d.xyz = _ptr(self._xyz, C.c_double)
        d.n_tets = self._tets.shape[0]
        d.tets = _ptr(self._tets, C.c_int32)
        keep = []
        if edges is not None:
            e = np.ascontiguousarray(edges, dtype=np.int32)
            keep.append(e)
            d.n_edges = e.shape[0]
            d.edges = _ptr(e, C.c_int32)
        if faces is not None:
            f = np.ascontiguousarray(faces, dtype=np.int32)
            keep.append(f)
            d.n_faces = f.shape[0]
            d.faces = _ptr(f, C.c_int32)
        if wall_bc is not None:
            wb = np.ascontiguousarray(wall_bc, dtype=np.int32).reshape(-1)
            if wb.size != 4 * d.n_tets:
                raise PicError(1, "pic_mesh_create", "wall_bc needs 4 entries per tet")
            keep.append(wb)
            d.wall_bc = _ptr(wb, C.c_int32)
        for key, field in (("G", "G_coo"), ("C", "C_coo"), ("D", "D_coo")):
            if incidence and key in incidence:
                a = np.ascontiguousarray(incidence[key], dtype=np.int32)
                keep.append(a)
                setattr(d, field, _ptr(a, C.c_int32))
        h = C.c_void_p()
        _check(lib.pic_mesh_create(C.byref(d), C.byref(h)), "pic_mesh_create")
        self._h = h
        c = np.zeros(8, dtype=np.int64)
        _check(lib.pic_mesh_info(h, _ptr(c, C.c_int64)), "pic_mesh_info")
        (self.n_nodes, self.n_edges, self.n_faces, self.n_tets,
         self.n_int_edges, self.n_int_nodes, self.nnz_A, self.nnz_L) = (int(x) for x in c)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.pic_mesh_destroy(self._h)
            self._h = None

    def entities(self):
        e = np.zeros((self.n_edges, 2), dtype=np.int32)
        f = np.zeros((self.n_faces, 3), dtype=np.int32)
        _check(_lib.pic_mesh_entities(self._h, _ptr(e, C.c_int32), _ptr(f, C.c_int32)), "pic_mesh_entities")
        return e, f

    def incidence(self, which: str):
        n = {"G": 2 * self.n_edges, "C": 3 * self.n_faces, "D": 4 * self.n_tets}[which]
        r, c, v = (np.zeros(n, dtype=np.int32) for _ in range(3))
        _check(_lib.pic_mesh_incidence(self._h, "GCD".index(which), _ptr(r, C.c_int32), _ptr(c, C.c_int32),
                                       _ptr(v, C.c_int32)), "pic_mesh_incidence")
        return r, c, v


def default_config() -> pic_config:
    load()
    c = pic_config()
    _lib.pic_config_default(C.byref(c))
    return c


class Sim:
    """pic_sim_create / pic_particles_load / pic_sim_init / pic_step ... on one mesh."""

    def __init__(self, mesh: Mesh, dt: float, form: str = "we", pusher: str = "boris",
                 precision: str = "plain", b0: Sequence[float] = (0.0, 0.0, 0.0), rho_background: float = 0.0,
                 cg_tol: float = 1e-10, init_tol: float = 1e-14, cg_max_iters: int = 10000,
                 walk_cap: int = 63, stream=None, profile: bool = False, solver_blocks_per_sm: int = 0,
                 preconditioner: str = "jacobi", barrier_spin_limit: int = 0, curved_path: bool = False):
        lib = load()
        self.mesh = mesh
        c = default_config()
        c.form = FORMS[form]
        c.pusher = 0 if pusher == "boris" else int(pusher[2:])
        c.precision = PRECISIONS[precision]
        c.dt = dt
        for i in range(3):
            c.b0[i] = b0[i]
        c.rho_background = rho_background
        c.cg_tol = cg_tol
        c.init_tol = init_tol
        c.cg_max_iters = cg_max_iters
        c.walk_cap = walk_cap
        c.solver_blocks_per_sm = solver_blocks_per_sm
        c.preconditioner = PRECONDITIONERS[preconditioner]
        c.profile = int(profile)
        c.barrier_spin_limit = int(barrier_spin_limit)
        c.curved_path = int(curved_path)
        if stream is not None:
            c.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.config = c
        h = C.c_void_p()
        _check(lib.pic_sim_create(mesh._h, C.byref(c), C.byref(h)), "pic_sim_create")
        self._h = h
        self.n_loaded = 0

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.pic_sim_destroy(self._h)
            self._h = None

    def particles_load(self, species: int, q: float, m: float, w: float, x, v, tet=None):
        """Host numpy arrays, or CUDA torch tensors (x, v float64 [n,3]; tet int32 [n])."""
        on_dev = hasattr(x, "is_cuda") and x.is_cuda
        if on_dev:
            n = x.shape[0]
            xp, vp = C.c_void_p(x.data_ptr()), C.c_void_p(v.data_ptr())
            tp = C.c_void_p(tet.data_ptr()) if tet is not None else None
        else:
            x = np.ascontiguousarray(x, dtype=np.float64)
            v = np.ascontiguousarray(v, dtype=np.float64)
            n = x.shape[0]
            xp, vp = C.c_void_p(x.ctypes.data), C.c_void_p(v.ctypes.data)
            if tet is not None:
                tet = np.ascontiguousarray(tet, dtype=np.int32)
                tp = C.c_void_p(tet.ctypes.data)
            else:
                tp = None
        _check(_lib.pic_particles_load(self._h, species, q, m, w, n, xp, vp, tp, int(on_dev)),
               "pic_particles_load")
        self.n_loaded += n

    def set_background_charge(self, rho_nodes: np.ndarray):
        """pic_set_background_charge: static node charges [n_nodes] (before init)."""
        a = np.ascontiguousarray(rho_nodes, dtype=np.float64).reshape(-1)
        if a.size != self.mesh.n_nodes:
            raise PicError(1, "pic_set_background_charge", f"needs {self.mesh.n_nodes} node charges")
        _check(_lib.pic_set_background_charge(self._h, _ptr(a, C.c_double)), "pic_set_background_charge")

    def init(self):
        _check(_lib.pic_sim_init(self._h), "pic_sim_init")

    def set_ab_history(self, a_hist: np.ndarray, v_hist: np.ndarray):
        a = np.ascontiguousarray(a_hist, dtype=np.float64)
        v = np.ascontiguousarray(v_hist, dtype=np.float64)
        _check(_lib.pic_set_ab_history(self._h, a.shape[0], _ptr(a, C.c_double), _ptr(v, C.c_double)),
               "pic_set_ab_history")

    def step(self, n: int = 1):
        _check(_lib.pic_step(self._h, n), "pic_step")

    def particle_phase(self):
        _check(_lib.pic_particle_phase(self._h), "pic_particle_phase")

    def field_len(self, which: str) -> int:
        m = self.mesh
        if which in ("E", "E_PREV", "G", "G_PREV", "DG"):
            return m.n_edges
        if which in ("B", "B_PREV"):
            return m.n_faces
        return m.n_nodes

    def field(self, which: str, out=None):
        n = self.field_len(which)
        if out is not None and hasattr(out, "is_cuda") and out.is_cuda:
            _check(_lib.pic_field_get(self._h, FIELDS[which], C.c_void_p(out.data_ptr()), n, 1), "pic_field_get")
            return out
        a = np.zeros(n)
        _check(_lib.pic_field_get(self._h, FIELDS[which], C.c_void_p(a.ctypes.data), n, 0), "pic_field_get")
        return a

    def set_field(self, which: str, values):
        n = self.field_len(which)
        if hasattr(values, "is_cuda") and values.is_cuda:
            _check(_lib.pic_field_set(self._h, FIELDS[which], C.c_void_p(values.data_ptr()), n, 1), "pic_field_set")
            return
        a = np.ascontiguousarray(values, dtype=np.float64)
        _check(_lib.pic_field_set(self._h, FIELDS[which], C.c_void_p(a.ctypes.data), n, 0), "pic_field_set")

    def count(self) -> int:
        n = C.c_int64()
        _check(_lib.pic_particles_count(self._h, C.byref(n)), "pic_particles_count")
        return n.value

    def particles_inject(self, species: int, x, v, tet=None):
        """pic_particles_inject with host numpy arrays x, v [n,3] (float64), tet [n] (int32) or None."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        tp = None
        if tet is not None:
            tet = np.ascontiguousarray(tet, dtype=np.int32)
            tp = _ptr(tet, C.c_int32)
        _check(_lib.pic_particles_inject(self._h, int(species), x.shape[0], _ptr(x, C.c_double), _ptr(v, C.c_double),
                                         tp), "pic_particles_inject")
        self.n_loaded += x.shape[0]

    def particles(self):
        """(x [n,3], v [n,3], tet [n], id [n]) of the live particles, sorted by id."""
        cap = max(self.n_loaded, 1)
        x = np.zeros((cap, 3))
        v = np.zeros((cap, 3))
        t = np.zeros(cap, dtype=np.int32)
        i = np.zeros(cap, dtype=np.int32)
        n = C.c_int64()
        _check(_lib.pic_particles_get(self._h, C.c_void_p(x.ctypes.data), C.c_void_p(v.ctypes.data),
                                      C.c_void_p(t.ctypes.data), C.c_void_p(i.ctypes.data), cap, C.byref(n), 0),
               "pic_particles_get")
        k = n.value
        order = np.argsort(i[:k], kind="stable")
        return x[:k][order], v[:k][order], t[:k][order], i[:k][order]

    def diag(self) -> Dict[str, float]:
        d = pic_diag()
        _check(_lib.pic_diagnostics_get(self._h, C.byref(d)), "pic_diagnostics_get")
        return {n: getattr(d, n) for n, _ in pic_diag._fields_}

    PHASES = ("sort", "coef", "push", "deposit", "rhs", "cg", "completion", "field_other")

    def profile(self) -> Dict[str, tuple]:
        ms = np.zeros(len(self.PHASES))
        cnt = np.zeros(len(self.PHASES), dtype=np.int64)
        _check(_lib.pic_profile_get(self._h, _ptr(ms, C.c_double), _ptr(cnt, C.c_int64)), "pic_profile_get")
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(self.PHASES)}

    def profile_reset(self):
        _check(_lib.pic_profile_reset(self._h), "pic_profile_reset")

    def synchronize(self):
        _check(_lib.pic_sim_synchronize(self._h), "pic_sim_synchronize")

    # ---- learned preconditioner ----
    def gnn_train(self, steps: int = 300, lr: float = 1e-3, samples: int = 8) -> float:
        cfg = pic_gnn_train_cfg(int(steps), float(lr), int(samples))
        loss = C.c_double(0.0)
        _check(_lib.pic_gnn_train(self._h, C.byref(cfg), C.byref(loss)), "pic_gnn_train")
        return float(loss.value)

    def gnn_weights(self) -> np.ndarray:
        w = np.zeros(GNN_PARAMS, dtype=np.float32)
        _check(_lib.pic_gnn_get_weights(self._h, _ptr(w, C.c_float), GNN_PARAMS), "pic_gnn_get_weights")
        return w

    def gnn_set_weights(self, w: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float32)
        _check(_lib.pic_gnn_set_weights(self._h, _ptr(w, C.c_float), w.size), "pic_gnn_set_weights")

    def gnn_apply(self, r_edges: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r_edges, dtype=np.float64)
        z = np.zeros_like(r)
        _check(_lib.pic_gnn_apply(self._h, _ptr(r, C.c_double), _ptr(z, C.c_double)), "pic_gnn_apply")
        return z

    def gnn_loss_grad(self, r_edges: np.ndarray):
        r = np.ascontiguousarray(r_edges, dtype=np.float64)
        loss = C.c_double(0.0)
        g = np.zeros(GNN_PARAMS)
        _check(_lib.pic_gnn_loss_grad(self._h, _ptr(r, C.c_double), C.byref(loss), _ptr(g, C.c_double)),
               "pic_gnn_loss_grad")
        return float(loss.value), g


class Batch:
    """pic_batch_create / pic_batch_step over simulations on one device."""

    def __init__(self, sims: Sequence["Sim"]):
        lib = load()
        self.sims = list(sims)              # keep the members alive
        arr = (C.c_void_p * len(self.sims))(*[s._h for s in self.sims])
        h = C.c_void_p()
        _check(lib.pic_batch_create(arr, len(self.sims), C.byref(h)), "pic_batch_create")
        self._h = h

    def step(self, n: int = 1):
        _check(_lib.pic_batch_step(self._h, int(n)), "pic_batch_step")

    def info(self) -> Dict[str, object]:
        d = pic_batch_info_t()
        _check(_lib.pic_batch_info(self._h, C.byref(d)), "pic_batch_info")
        return {"n_sims": d.n_sims, "graph": d.graph, "graph_steps": d.graph_steps,
                "solver_blocks_per_sm": d.solver_blocks_per_sm, "graph_launches": d.graph_launches,
                "eager_steps": d.eager_steps, "tune_ms": list(d.tune_ms),
                "solver_build": BATCH_BUILDS[d.solver_build],
                "completion_blocks_per_sm": d.completion_blocks_per_sm,
                "completion_build": BATCH_BUILDS[d.completion_build],
                "tune_newmark_ms": list(d.tune_newmark_ms), "tune_completion_ms": list(d.tune_completion_ms)}

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.pic_batch_destroy(self._h)
            self._h = None


def electrostatic_solve_noalloc(mesh: Mesh, rho, phi, tol: float = 1e-14, stream=None):
    """pic_electrostatic_solve_noalloc on CUDA tensors rho, phi [n_nodes] (float64).

    The library allocates nothing during this call.  The C entry point takes
    no lengths, so both tensors are checked here before any launch: float64,
    contiguous, n_nodes elements, on the current CUDA device."""
    load()
    import torch
    for name, t in (("rho", rho), ("phi", phi)):
        if not isinstance(t, torch.Tensor):
            raise PicError(1, "electrostatic_solve_noalloc", f"{name} must be a torch tensor")
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or t.numel() != mesh.n_nodes:
            raise PicError(1, "electrostatic_solve_noalloc",
                           f"{name} must be a contiguous float64 CUDA tensor of {mesh.n_nodes} elements "
                           f"(got {t.dtype}, {t.device}, {t.numel()} elements)")
        if t.device.index != torch.cuda.current_device():
            raise PicError(1, "electrostatic_solve_noalloc", f"{name} is not on the current CUDA device")
    st = None if stream is None else C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(_lib.pic_electrostatic_solve_noalloc(mesh._h, C.c_void_p(rho.data_ptr()), C.c_void_p(phi.data_ptr()),
                                                tol, st), "pic_electrostatic_solve_noalloc")
    return phi


def launch_count() -> int:
    return int(load().pic_launch_count())


def sim_from_workload(wl, dt: float, precision: str = "plain", cg_tol: float = 1e-10,
                      init_tol: float = 1e-14, mesh: Optional[Mesh] = None, stream=None,
                      profile: bool = False, cg_max_iters: int = 10000, solver_blocks_per_sm: int = 0,
                      preconditioner: str = "jacobi") -> Sim:
    """Builds and initialises a simulation of a ``workloads.Workload`` (its
    walls absorbing where ``wl.wall_bc`` says so)."""
    mesh = mesh or Mesh(wl.mesh.xyz, wl.mesh.tets, wall_bc=getattr(wl, "wall_bc", None))
    sim = Sim(mesh, dt, form=wl.form, pusher=wl.pusher, precision=precision, b0=wl.b0,
              rho_background=wl.rho_background, cg_tol=cg_tol, init_tol=init_tol, stream=stream,
              profile=profile, cg_max_iters=cg_max_iters, solver_blocks_per_sm=solver_blocks_per_sm,
              preconditioner=preconditioner)
    for k, sp in enumerate(wl.species):
        sim.particles_load(k, sp.q, sp.m, sp.w, sp.x, sp.v, sp.tet)
    sim.init()
    return sim
