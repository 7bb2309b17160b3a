"""Seeded synthetic inputs shared by the GPU path, the oracle and the benchmark.

This module only *generates inputs*: node coordinates and tet connectivity of
Kuhn-split boxes, vertex jitter, and particle positions / velocities / start
tets drawn from a counter-based generator.  It holds none of the method's
arithmetic (no Whitney forms, no matrices, no push, no deposit), so both sides
of every parity test consume identical arrays without sharing any method code.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated at a counter, mapped to
doubles in [0, 1) with the top 53 bits, and to normals by Box-Muller.

The paper's meshes and particle data are not published (Sec. V, data statement),
so each workload below is a synthetic stand-in with the shape of the paper's
experiments: Sec. IV.A (single particle gyration, Table I), Sec. IV.B (electron
beam with space charge, Table II) and Sec. IV.C (neutral plasma expansion with
the real mass ratio, Table III).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# Physical constants (SI).  q and m of the electron are the values printed in
# Table I of the paper (Sec. IV.A); c and eps0 are CODATA.
Q_E = -1.60217646e-19
M_E = 9.10938370e-31
C0 = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C0 * C0)
KB = 1.380649e-23
EV = 1.602176634e-19
MASS_RATIO_P = 1836.0

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counter: np.ndarray) -> np.ndarray:
    """SplitMix64 output for ``counter`` (uint64 array) under ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from counters stream*2^40 + [0, n)."""
    ctr = np.arange(n, dtype=np.uint64) + np.uint64(stream) * np.uint64(1 << 40)
    return (splitmix64(seed, ctr) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller from two uniform streams."""
    u1 = 1.0 - uniform(seed, 2 * stream, n)          # (0, 1]
    u2 = uniform(seed, 2 * stream + 1, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ---------------------------------------------------------------------------
# Kuhn-split box meshes
# ---------------------------------------------------------------------------
# The six tets of a unit cube that share its main diagonal: for a permutation
# (a0, a1, a2) of the axes, v0 = corner, v1 = v0 + e_a0, v2 = v1 + e_a1,
# v3 = v2 + e_a2.  A point with fractional coordinates f lies in the tet whose
# permutation sorts f in decreasing order, which lets the generator place
# particles in known tets without any search.
KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


@dataclasses.dataclass
class BoxMesh:
    cells: Tuple[int, int, int]
    size: Tuple[float, float, float]
    xyz: np.ndarray          # float64 [n_nodes, 3]
    tets: np.ndarray         # int32 [n_tets, 4]
    ref_xyz: np.ndarray      # unjittered coordinates (used only to place particles)

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]

    @property
    def h(self) -> float:
        return min(s / c for s, c in zip(self.size, self.cells))


def kuhn_box(cells: Tuple[int, int, int], size: Tuple[float, float, float],
             jitter: float = 0.0, seed: int = 0) -> BoxMesh:
    """Box of nx*ny*nz cubes, each split into 6 Kuhn tets (conforming).

    Node (i, j, k) has index i + (nx+1)*(j + (ny+1)*k).  Tet index is
    6*cell + perm, cell = ci + nx*(cj + ny*ck).  ``jitter`` moves every
    interior vertex by a uniform offset in [-jitter*h, jitter*h] per component
    (boundary vertices stay on the walls).
    """
    nx, ny, nz = cells
    lx, ly, lz = size
    hx, hy, hz = lx / nx, ly / ny, lz / nz
    i = np.arange(nx + 1)
    j = np.arange(ny + 1)
    k = np.arange(nz + 1)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    ref = np.stack([I.ravel() * hx, J.ravel() * hy, K.ravel() * hz], axis=1).astype(np.float64)
    xyz = ref.copy()
    if jitter > 0.0:
        n = xyz.shape[0]
        interior = ((I.ravel() > 0) & (I.ravel() < nx) & (J.ravel() > 0) & (J.ravel() < ny)
                    & (K.ravel() > 0) & (K.ravel() < nz))
        h = np.array([hx, hy, hz])
        for a in range(3):
            d = (2.0 * uniform(seed, 100 + a, n) - 1.0) * jitter * h[a]
            xyz[:, a] += np.where(interior, d, 0.0)

    def nid(ci, cj, ck):
        return ci + (nx + 1) * (cj + (ny + 1) * ck)

    cK, cJ, cI = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    cI, cJ, cK = cI.ravel(), cJ.ravel(), cK.ravel()
    tets = np.empty((cI.size, 6, 4), dtype=np.int64)
    for p, perm in enumerate(KUHN_PERMS):
        off = np.zeros((cI.size, 3), dtype=np.int64)
        tets[:, p, 0] = nid(cI, cJ, cK)
        for v in range(1, 4):
            off[:, perm[v - 1]] += 1
            tets[:, p, v] = nid(cI + off[:, 0], cJ + off[:, 1], cK + off[:, 2])
    return BoxMesh(cells=(nx, ny, nz), size=(lx, ly, lz), xyz=xyz,
                   tets=tets.reshape(-1, 4).astype(np.int32), ref_xyz=ref)


BOX_WALLS = ("x0", "x1", "y0", "y1", "z0", "z1")


def box_wall_bc(mesh: "BoxMesh", absorbing=BOX_WALLS) -> np.ndarray:
    """Per tet face (entry [t, k]: the face opposite the tet's k-th vertex) a
    1 when the face lies on one of the named box walls ("x0" is x = 0, "x1"
    is x = size_x, ...), else 0.  Boundary vertices are never jittered, so a
    wall face is one whose three vertices share the wall coordinate."""
    tets = mesh.tets
    out = np.zeros((tets.shape[0], 4), dtype=np.int32)
    tol = 1e-9 * max(mesh.size)
    for name in absorbing:
        ax = "xyz".index(name[0])
        val = 0.0 if name[1] == "0" else mesh.size[ax]
        on = np.abs(mesh.xyz[:, ax] - val) <= tol            # nodes on that wall
        on_t = on[tets]                                       # [n_tets, 4]
        for k in range(4):
            others = [j for j in range(4) if j != k]
            out[:, k] |= np.all(on_t[:, others], axis=1).astype(np.int32)
    return out


def place_in_box(mesh: BoxMesh, pos_ref: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Map points given in unjittered box coordinates to (physical point, tet).

    The point's Kuhn tet and barycentric weights are found in the unjittered
    cell from its fractional coordinates; the physical point is the same
    barycentric combination of the (possibly jittered) tet vertices, so the
    returned tet contains it by construction.  Points are first clamped into
    the open box.
    """
    nx, ny, nz = mesh.cells
    lx, ly, lz = mesh.size
    hvec = np.array([lx / nx, ly / ny, lz / nz])
    ncell = np.array([nx, ny, nz])
    s = np.clip(pos_ref / hvec, 1e-9, ncell - 1e-9)
    cidx = np.minimum(np.floor(s).astype(np.int64), ncell - 1)
    f = s - cidx
    # Kuhn permutation = axes in decreasing order of f; ties broken by axis index.
    order = np.argsort(-f, axis=1, kind="stable")
    perm_id = np.zeros(f.shape[0], dtype=np.int64)
    for p, perm in enumerate(KUHN_PERMS):
        perm_id[np.all(order == np.array(perm), axis=1)] = p
    fs = np.take_along_axis(f, order, axis=1)
    lam = np.stack([1.0 - fs[:, 0], fs[:, 0] - fs[:, 1], fs[:, 1] - fs[:, 2], fs[:, 2]], axis=1)
    cell = cidx[:, 0] + nx * (cidx[:, 1] + ny * cidx[:, 2])
    tet = (6 * cell + perm_id).astype(np.int32)
    verts = mesh.xyz[mesh.tets[tet]]                      # [n, 4, 3]
    pos = np.einsum("nk,nkd->nd", lam, verts)
    return pos, tet


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Species:
    q: float
    m: float
    w: float                 # macro-particle weight
    x: np.ndarray            # [n, 3] float64
    v: np.ndarray            # [n, 3] float64
    tet: np.ndarray          # [n] int32


@dataclasses.dataclass
class Workload:
    name: str
    mesh: BoxMesh
    species: List[Species]
    b0: Tuple[float, float, float]
    form: str                # "we" or "mfem"
    pusher: str              # "boris" or "ab1".."ab5"
    dt_cfl_multiple: Optional[float]
    dt: Optional[float]
    steps: int
    rho_background: float    # uniform static background charge density (C/m^3)
    notes: str = ""
    wall_bc: Optional[np.ndarray] = None   # [n_tets, 4] 1 = absorbing wall face, 0 = conducting (None: all conducting)

    @property
    def n_particles(self) -> int:
        return sum(s.x.shape[0] for s in self.species)


def maxwellian(seed: int, stream: int, n: int, vth: float) -> np.ndarray:
    return np.stack([vth * normal(seed, stream + a, n) for a in range(3)], axis=1)


def thermal_plasma_cube(n_cells: int = 6, n_particles: int = 10_000, seed: int = 1001,
                        steps: int = 100, side: float = 1.0, vth_over_c: float = 0.01,
                        weight: float = 1.0e7, b0z: float = 0.1) -> Workload:
    """Thermal electrons in a PEC cube with a neutralising ion background.

    Defaults: 1 m cube, 6^3 cells (1,296 tets), 10,000 electrons uniform in
    space, Maxwellian with v_th = 0.01c per component, B0 = 0.1 T along z,
    wave-equation Newmark, dt = 2 x the explicit CFL limit, 100 steps.  The
    weight 1e7 gives n = 1e11 m^-3 and a Debye length of about h.
    """
    mesh = kuhn_box((n_cells,) * 3, (side,) * 3)
    ref = np.stack([side * uniform(seed, a, n_particles) for a in range(3)], axis=1)
    x, tet = place_in_box(mesh, ref)
    v = maxwellian(seed, 10, n_particles, vth_over_c * C0)
    sp = Species(q=Q_E, m=M_E, w=weight, x=x, v=v, tet=tet)
    rho_bg = -(Q_E * weight * n_particles) / side ** 3
    return Workload(name=f"thermal_plasma_cube_{n_cells}^3", mesh=mesh, species=[sp],
                    b0=(0.0, 0.0, b0z), form="we", pusher="boris", dt_cfl_multiple=2.0,
                    dt=None, steps=steps, rho_background=rho_bg)


def batched_runs(n_runs: int = 64, seed: int = 1005, cells: Tuple[int, int] = (8, 32),
                 particles: Tuple[float, float] = (1.0e4, 1.0e6), vth_over_c: float = 0.01,
                 b0z: float = 0.1) -> List[Workload]:
    """Independent thermal-electron runs of uneven size for batched stepping.

    Run k: a unit PEC cube of c_k^3 Kuhn cells with N_k Maxwellian electrons
    (v_th = 0.01c), c_k and N_k log-uniform in the given ranges (counter-based
    draws from `seed`).  The density scales as (c_k/6)^2 x 1e11 m^-3, so the
    Debye length stays about one cell and the plasma period resolves the same
    way at dt = 2 x CFL on every mesh; weight = density / N_k.
    """
    lo_c, hi_c = math.log(cells[0]), math.log(cells[1] + 0.999)
    lo_n, hi_n = math.log(particles[0]), math.log(particles[1])
    uc = uniform(seed, 0, n_runs)
    un = uniform(seed, 1, n_runs)
    out = []
    for k in range(n_runs):
        c = int(math.exp(lo_c + (hi_c - lo_c) * uc[k]))
        n = int(round(math.exp(lo_n + (hi_n - lo_n) * un[k])))
        density = 1.0e11 * (c / 6.0) ** 2
        wl = thermal_plasma_cube(n_cells=c, n_particles=n, seed=seed * 1000 + k, vth_over_c=vth_over_c,
                                 weight=density / n, b0z=b0z)
        wl.name = f"batched_run_{k}_{c}^3_{n}"
        out.append(wl)
    return out


def _beam_particles(seed: int, stream: int, n: int, side_xy: float, z0: float, z1: float, sigma: float,
                    vz: float, vth: float) -> Tuple[np.ndarray, np.ndarray]:
    """n beam electrons: radial Gaussian (sigma) about the box axis, cut at
    0.45 of the width, z uniform in (z0, z1); v = (0, 0, vz) + vth N(0, 1)."""
    c = 0.5 * side_xy
    r = np.stack([normal(seed, stream, n), normal(seed, stream + 1, n)], axis=1) * sigma
    lim = 0.45 * side_xy
    r = np.clip(r, -lim, lim)
    z = z0 + (z1 - z0) * uniform(seed, stream + 2, n)
    x = np.stack([c + r[:, 0], c + r[:, 1], z], axis=1)
    v = np.stack([vth * normal(seed, stream + 3 + a, n) for a in range(3)], axis=1)
    v[:, 2] += vz
    return x, v


def electron_beam(cells: Tuple[int, int, int] = (32, 32, 128), h: float = 1.25e-3, n_inflight: int = 2_000_000,
                  seed: int = 1003, sigma_frac: float = 0.1, vz_over_c: float = 0.1, spread: float = 0.01,
                  current: float = 0.25, steps: int = 2000, dt_cfl_multiple: float = 4.0) -> Workload:
    """Non-neutral electron beam with space charge (Sec. IV.B analogue).

    A PEC box of cells[0] x cells[1] x cells[2] Kuhn cells of side h; electrons
    enter at z = 0 with a radial Gaussian profile (sigma = sigma_frac * width),
    axial speed vz_over_c * c and a thermal spread of `spread` of it per
    component.  The beam starts in its steady state: n_inflight electrons
    spread uniformly along the box (the in-flight population the injection
    keeps), with the macro weight that carries `current` amperes.  Each step
    then injects `inject_per_step(dt)` electrons (see beam_injection); they
    leave through the far wall.
    """
    size = (cells[0] * h, cells[1] * h, cells[2] * h)
    mesh = kuhn_box(cells, size)
    vz = vz_over_c * C0
    x, v = _beam_particles(seed, 0, n_inflight, size[0], 0.0, size[2], sigma_frac * size[0], vz, spread * vz)
    x, tet = place_in_box(mesh, x)
    w = current * size[2] / (vz * abs(Q_E) * n_inflight)
    sp = Species(q=Q_E, m=M_E, w=w, x=x, v=v, tet=tet)
    return Workload(name=f"electron_beam_{cells[0]}x{cells[1]}x{cells[2]}", mesh=mesh, species=[sp],
                    b0=(0.0, 0.0, 0.0), form="we", pusher="boris", dt_cfl_multiple=dt_cfl_multiple, dt=None,
                    steps=steps, rho_background=0.0,
                    notes=f"h={h} m, sigma={sigma_frac * size[0]:.4e} m, vz={vz:.4e} m/s, weight={w:.6e}, "
                          f"I={current} A, seed={seed}")


def inject_per_step(wl: Workload, dt: float) -> int:
    """Electrons entering per step so that the in-flight population stays
    constant: N * vz * dt / Lz."""
    sp = wl.species[0]
    lz = float(wl.mesh.xyz[:, 2].max())
    vz = float(np.mean(sp.v[:, 2]))
    return max(1, int(round(sp.x.shape[0] * vz * dt / lz)))


def beam_injection(wl: Workload, step: int, n: int, dt: float, seed: int = 1003,
                   sigma_frac: float = 0.1, vz_over_c: float = 0.1, spread: float = 0.01):
    """The electrons injected before step `step`: the beam profile at
    z in (0, vz dt) (the slab that entered during one step); (x [n,3], v [n,3], tet [n])."""
    side = float(wl.mesh.xyz[:, 0].max())
    vz = vz_over_c * C0
    zmax = min(vz * dt, 0.5 * float(wl.mesh.xyz[:, 2].max()))
    x, v = _beam_particles(seed, 100 + 8 * step, n, side, 0.0, zmax, sigma_frac * side, vz, spread * vz)
    x[:, 2] = np.maximum(x[:, 2], 1e-9 * zmax)
    x, tet = place_in_box(wl.mesh, x)
    return x, v, tet


def larmor_orbit_box(n_cells: int = 20, b0z: float = 0.05, vperp_over_c: float = 0.05,
                     steps: int = 10_000, form: str = "mfem", pusher: str = "boris") -> Workload:
    """One electron gyrating in uniform B0 inside a PEC box (Sec. IV.A analogue).

    Box side 10 Larmor radii centred on the guiding centre, n_cells^3 cells,
    dt = T_c / 64, Maxwell-solver (MFEM) Newmark form.
    """
    wc = abs(Q_E) * b0z / M_E
    vperp = vperp_over_c * C0
    r_l = vperp / wc
    side = 10.0 * r_l
    mesh = kuhn_box((n_cells,) * 3, (side,) * 3)
    centre = np.array([0.5 * side, 0.5 * side, 0.5 * side])
    # Electron (q < 0) in B0 z gyrates counter-clockwise seen from +z; starting
    # at centre + r_L x with velocity +vperp y keeps the guiding centre near the
    # centre.  The start is shifted by (0, 0.137, 0.291) h so that the orbit
    # plane and the start point stay clear of mesh faces and edges.
    h = side / n_cells
    ref = (centre + np.array([r_l, 0.137 * h, 0.291 * h]))[None, :]
    x, tet = place_in_box(mesh, ref)
    v = np.array([[0.0, vperp, 0.0]])
    sp = Species(q=Q_E, m=M_E, w=1.0, x=x, v=v, tet=tet)
    t_c = 2.0 * math.pi / wc
    return Workload(name=f"larmor_orbit_{n_cells}^3", mesh=mesh, species=[sp],
                    b0=(0.0, 0.0, b0z), form=form, pusher=pusher, dt_cfl_multiple=None,
                    dt=t_c / 64.0, steps=steps, rho_background=0.0,
                    notes=f"r_L={r_l:.6e} m, T_c={t_c:.6e} s")


def plasma_ball(n_cells: int = 64, n_per_species: int = 16 * 1024 * 1024, seed: int = 1004,
                steps: int = 1000, h: float = 1.0e-4, jitter: float = 0.2,
                te_ev: float = 10.0, ti_ev: float = 0.1, sigma_frac: float = 0.15,
                debye_over_h: float = 2.0, mass_ratio: float = MASS_RATIO_P) -> Workload:
    """Neutral e-/p+ Gaussian plasma ball in a jittered PEC box (Sec. IV.C analogue).

    Defaults: 64^3 cells (1,572,864 tets) of side h = 0.1 mm with interior
    vertices jittered up to 20% of h; 16M electrons + 16M protons (mass ratio
    1836) in a Gaussian sphere of sigma = 0.15 L; Te = 10 eV, Ti = 0.1 eV;
    the weight puts the peak-density Debye length at 2h; dt = 4 x CFL.
    `mass_ratio` sets the ion mass in electron masses.
    """
    side = n_cells * h
    mesh = kuhn_box((n_cells,) * 3, (side,) * 3, jitter=jitter, seed=seed)
    sigma = sigma_frac * side
    te = te_ev * EV
    n_peak = EPS0 * te / ((debye_over_h * h) ** 2 * Q_E ** 2)
    weight = n_peak * (2.0 * math.pi) ** 1.5 * sigma ** 3 / n_per_species
    out = []
    for s_idx, (q, m, temp) in enumerate(((Q_E, M_E, te), (-Q_E, mass_ratio * M_E, ti_ev * EV))):
        base = 1000 * (s_idx + 1)
        ref = 0.5 * side + sigma * np.stack([normal(seed, base + a, n_per_species) for a in range(3)], axis=1)
        ref = np.clip(ref, 0.01 * side, 0.99 * side)
        x, tet = place_in_box(mesh, ref)
        v = maxwellian(seed, base + 10, n_per_species, math.sqrt(temp / m))
        out.append(Species(q=q, m=m, w=weight, x=x, v=v, tet=tet))
    return Workload(name=f"plasma_ball_{n_cells}^3", mesh=mesh, species=out,
                    b0=(0.0, 0.0, 0.0), form="we", pusher="boris", dt_cfl_multiple=4.0,
                    dt=None, steps=steps, rho_background=0.0,
                    notes=f"weight={weight:.6e}, sigma={sigma:.6e} m")
