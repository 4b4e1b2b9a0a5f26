"""Seeded synthetic inputs for the UGKWP-LTS step: meshes, boundary tags, gas and flow states.

This module defines *workloads* only. It holds none of the method's arithmetic (no time steps, relaxation
times, fluxes, sampling or transport): it produces the vertex coordinates, boundary-condition tags and
reference states that both the CUDA library and the CPU oracle take as inputs, so that both sides see the
identical mesh.

Non-dimensionalisation (a reading; the paper does not state one): rho_inf = 1, T_inf = 1, R = 1/2, so that
2 R T_inf = 1, and U_inf = Ma * sqrt(gamma R T_inf) with gamma = 5/3 (monatomic gas, three translational
degrees of freedom, no internal ones; Sec. II "Gas-kinetic theory", eq. (1) with D = 0).

Structured meshes (`Mesh`) are ni x nj quadrilaterals with vertex (i, j) stored at index i + (ni + 1) * j; for
a 1-D line mesh nj = 1 and only the x coordinates matter. Unstructured meshes (`UMesh`) list triangles and
convex quadrilaterals by counter-clockwise vertex indices, with a tag for every boundary edge.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

R_GAS = 0.5
GAMMA = 5.0 / 3.0

# boundary-condition tags shared by the C ABI of the library and of the oracle (plain integers)
BC_WALL = 1        # diffuse isothermal wall at T_w
BC_FARFIELD = 2    # freestream ghost on inflow, zero-gradient ghost on outflow; particles leaving are deleted
BC_FIXED = 3       # ghost fixed at the second reference state (1-D downstream state); particles deleted
BC_SYMMETRY = 4    # specular mirror
BC_PERIODIC = 5    # 1-D only: the two ends of the line are joined

MESH_LINE = 0
MESH_OMESH = 1
MESH_PLATE = 2
MESH_UNSTRUCTURED = 3


@dataclass
class Mesh:
    kind: int
    ni: int
    nj: int
    dim: int
    periodic_j: int
    xv: np.ndarray
    yv: np.ndarray
    bc_imin: np.ndarray
    bc_imax: np.ndarray
    bc_jmin: np.ndarray
    bc_jmax: np.ndarray
    info: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return self.ni * self.nj


@dataclass
class UMesh:
    """Triangles and convex quadrilaterals: `cells` (C, 4) counter-clockwise vertex indices with -1 in the last
    column for a triangle; `boundary` (n, 3) rows (vertex, vertex, tag), one per edge of a single cell."""
    xv: np.ndarray
    yv: np.ndarray
    cells: np.ndarray
    boundary: np.ndarray
    info: dict = field(default_factory=dict)
    kind: int = MESH_UNSTRUCTURED
    dim: int = 2

    @property
    def ncells(self) -> int:
        return int(self.cells.shape[0])


def freestream_speed(Ma: float) -> float:
    return Ma * math.sqrt(GAMMA * R_GAS * 1.0)


def geometric_sizes(n: int, h1: float, ratio: float) -> np.ndarray:
    return h1 * ratio ** np.arange(n, dtype=np.float64)


def solve_ratio(n: int, h1: float, span: float) -> float:
    """Geometric ratio r with sum_{k<n} h1 r^k == span (bisection; workload geometry, not the method)."""
    lo, hi = 1.0 + 1e-12, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if h1 * (mid ** n - 1.0) / (mid - 1.0) > span:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def line_mesh(ni: int, x0: float, x1: float, end_ratio: float = 1.0, bc_left: int = BC_FARFIELD,
              bc_right: int = BC_FIXED) -> Mesh:
    """1-D line [x0, x1] with ni cells whose sizes grow geometrically from left to right by end_ratio."""
    if end_ratio == 1.0:
        xs = np.linspace(x0, x1, ni + 1)
    else:
        r = end_ratio ** (1.0 / (ni - 1))
        h = geometric_sizes(ni, 1.0, r)
        h *= (x1 - x0) / h.sum()
        xs = np.concatenate([[x0], x0 + np.cumsum(h)])
        xs[-1] = x1
    xv = np.zeros((2, ni + 1))
    xv[0] = xs
    xv[1] = xs
    yv = np.zeros((2, ni + 1))
    yv[1] = 1.0
    return Mesh(MESH_LINE, ni, 1, 1, 0, xv.reshape(-1).copy(), yv.reshape(-1).copy(),
                np.array([bc_left], np.int32), np.array([bc_right], np.int32),
                np.zeros(ni, np.int32), np.zeros(ni, np.int32), info={"x0": x0, "x1": x1})


def omesh(ni: int, nj: int, h1: float, r_out: float, r_cyl: float = 0.5) -> Mesh:
    """Body-fitted O-mesh around a cylinder of radius r_cyl: i radial (wall at i = 0), j circumferential.

    The radial stretching ratio is solved so that ni cells of first height h1 reach r_out exactly.
    Vertex angle theta_j = 2 pi j / nj (counter-clockwise), so theta = pi (the stagnation point of a
    +x freestream) is a vertex whenever nj is even.
    """
    ratio = solve_ratio(ni, h1, r_out - r_cyl)
    h = geometric_sizes(ni, h1, ratio)
    r = np.concatenate([[r_cyl], r_cyl + np.cumsum(h)])
    r[-1] = r_out
    th = 2.0 * np.pi * np.arange(nj + 1) / nj
    th[-1] = 0.0
    xv = (r[None, :] * np.cos(th)[:, None]).reshape(-1)
    yv = (r[None, :] * np.sin(th)[:, None]).reshape(-1)
    return Mesh(MESH_OMESH, ni, nj, 2, 1, xv.copy(), yv.copy(),
                np.full(nj, BC_WALL, np.int32), np.full(nj, BC_FARFIELD, np.int32),
                np.zeros(ni, np.int32), np.zeros(ni, np.int32),
                info={"ratio": ratio, "r_cyl": r_cyl, "r_out": r_out, "h1": h1})


def plate_mesh(ni: int = 240, nj: int = 120, h1: float = 1e-4, ratio: float = 1.06, L: float = 1.0,
               x_lead: float = -0.1, x_trail: float = 1.1) -> Mesh:
    """Cartesian mesh over a sharp flat plate of length L on y = 0 (wall for 0 <= x <= L, mirror elsewhere)."""
    xs = np.linspace(x_lead * L, x_trail * L, ni + 1)
    hy = geometric_sizes(nj, h1 * L, ratio)
    ys = np.concatenate([[0.0], np.cumsum(hy)])
    xv = np.tile(xs, nj + 1)
    yv = np.repeat(ys, ni + 1)
    xc = 0.5 * (xs[:-1] + xs[1:])
    bc_jmin = np.where((xc >= 0.0) & (xc <= L), BC_WALL, BC_SYMMETRY).astype(np.int32)
    return Mesh(MESH_PLATE, ni, nj, 2, 0, xv, yv,
                np.full(nj, BC_FARFIELD, np.int32), np.full(nj, BC_FARFIELD, np.int32),
                bc_jmin, np.full(ni, BC_FARFIELD, np.int32), info={"L": L, "ratio": ratio})


def tri_plate(ni: int = 107, n_quad: int = 15, nj: int = 35, h1: float = 1e-5, height: float = 1.0, L: float = 1.0,
              x_lead: float = -0.1, x_trail: float = 1.1) -> UMesh:
    """Hybrid flat-plate mesh: the Cartesian plate mesh (wall for 0 <= x <= L on y = 0, mirror elsewhere) with
    rows stretched from h1 to `height`, its first n_quad rows kept as quadrilaterals and the rest cut into
    triangles; n_quad ni + 2 (nj - n_quad) ni cells."""
    m = plate_mesh(ni, nj, h1, solve_ratio(nj, h1 * L, height * L), L, x_lead, x_trail)
    u = split_quads(m, n_quad, "j")
    u.info.update({"L": L, "h1": h1, "ni": ni, "nj": nj, "n_quad": n_quad})
    return u


def _vid(m: Mesh, i: int, j: int) -> int:
    return i + (m.ni + 1) * (0 if (m.periodic_j and j == m.nj) else j)


def as_unstructured(m: Mesh) -> UMesh:
    """A 2-D structured mesh restated as an unstructured one: the same vertices, cell c = i + ni j with corners
    (i, j), (i+1, j), (i+1, j+1), (i, j+1) and the same boundary tags."""
    assert m.dim == 2
    cells = np.array([[_vid(m, i, j), _vid(m, i + 1, j), _vid(m, i + 1, j + 1), _vid(m, i, j + 1)]
                      for j in range(m.nj) for i in range(m.ni)], np.int32)
    bnd = [(_vid(m, 0, j), _vid(m, 0, j + 1), m.bc_imin[j]) for j in range(m.nj)]
    bnd += [(_vid(m, m.ni, j), _vid(m, m.ni, j + 1), m.bc_imax[j]) for j in range(m.nj)]
    if not m.periodic_j:
        bnd += [(_vid(m, i, 0), _vid(m, i + 1, 0), m.bc_jmin[i]) for i in range(m.ni)]
        bnd += [(_vid(m, i, m.nj), _vid(m, i + 1, m.nj), m.bc_jmax[i]) for i in range(m.ni)]
    return UMesh(m.xv.copy(), m.yv.copy(), cells, np.array(bnd, np.int32).reshape(-1, 3), info=dict(m.info))


def split_quads(m: Mesh, first_tri_row: int = 0, axis: str = "i") -> UMesh:
    """A 2-D structured mesh with every quadrilateral from row `first_tri_row` on (rows counted along `axis`)
    cut into two triangles, the diagonal alternating like a chequerboard; the quadrilaterals before that row
    stay (a hybrid mesh: quadrilateral layers at the wall, triangles outside)."""
    u = as_unstructured(m)
    cells = []
    for c, q in enumerate(u.cells):
        i, j = c % m.ni, c // m.ni
        if (i if axis == "i" else j) < first_tri_row:
            cells.append(q)
        elif (i + j) % 2 == 0:
            cells += [[q[0], q[1], q[2], -1], [q[0], q[2], q[3], -1]]
        else:
            cells += [[q[0], q[1], q[3], -1], [q[1], q[2], q[3], -1]]
    u.cells = np.array(cells, np.int32)
    u.info["first_tri_row"] = first_tri_row
    return u


def jitter_interior(u: UMesh, seed: int, amount: float) -> UMesh:
    """Moves every vertex that lies on no boundary edge by a seeded uniform offset of up to `amount` times the
    shortest edge at that vertex in each coordinate (the cells must stay counter-clockwise and convex)."""
    rng = np.random.default_rng(seed)
    on_b = np.zeros(len(u.xv), bool)
    on_b[u.boundary[:, 0]] = True
    on_b[u.boundary[:, 1]] = True
    hmin = np.full(len(u.xv), np.inf)
    for q in u.cells:
        vs = [v for v in q if v >= 0]
        for a, b in zip(vs, vs[1:] + vs[:1]):
            h = math.hypot(u.xv[b] - u.xv[a], u.yv[b] - u.yv[a])
            hmin[a] = min(hmin[a], h)
            hmin[b] = min(hmin[b], h)
    move = ~on_b & np.isfinite(hmin)
    dx = rng.uniform(-1.0, 1.0, len(u.xv)) * amount * np.where(move, hmin, 0.0)
    dy = rng.uniform(-1.0, 1.0, len(u.xv)) * amount * np.where(move, hmin, 0.0)
    return UMesh(u.xv + dx, u.yv + dy, u.cells.copy(), u.boundary.copy(), info=dict(u.info, jitter=amount))


def box_mesh(nx: int, ny: int, x0: float = 0.0, x1: float = 1.0, y0: float = 0.0, y1: float = 1.0,
             tags=(BC_FARFIELD, BC_FARFIELD, BC_FARFIELD, BC_FARFIELD)) -> Mesh:
    """Uniform Cartesian nx x ny mesh of [x0, x1] x [y0, y1]; tags of the sides x0, x1, y0, y1."""
    xs = np.linspace(x0, x1, nx + 1)
    ys = np.linspace(y0, y1, ny + 1)
    return Mesh(MESH_PLATE, nx, ny, 2, 0, np.tile(xs, ny + 1), np.repeat(ys, nx + 1),
                np.full(ny, tags[0], np.int32), np.full(ny, tags[1], np.int32),
                np.full(nx, tags[2], np.int32), np.full(nx, tags[3], np.int32), info={"box": (x0, x1, y0, y1)})


def tri_omesh(n_quad: int, ni: int, nj: int, h1: float, r_out: float, r_cyl: float = 0.5) -> UMesh:
    """Hybrid cylinder mesh: the O-mesh of `omesh` with its first n_quad radial layers kept as quadrilaterals
    and the ni - n_quad outer layers cut into triangles; n_quad nj + 2 (ni - n_quad) nj cells."""
    u = split_quads(omesh(ni, nj, h1, r_out, r_cyl), n_quad, "i")
    u.info.update({"r_cyl": r_cyl, "r_out": r_out, "h1": h1, "ni": ni, "nj": nj, "n_quad": n_quad})
    return u


def rankine_hugoniot(Ma: float, gamma: float = GAMMA):
    """Downstream (rho, u, T) of a normal shock for upstream (1, U_inf(Ma), 1): textbook jump relations."""
    rho2 = (gamma + 1.0) * Ma ** 2 / ((gamma - 1.0) * Ma ** 2 + 2.0)
    p2 = (2.0 * gamma * Ma ** 2 - (gamma - 1.0)) / (gamma + 1.0)
    u1 = freestream_speed(Ma)
    u2 = u1 / rho2
    T2 = p2 / rho2
    return rho2, u2, T2


def shock_initial_field(mesh: Mesh, Ma: float) -> np.ndarray:
    """Per-cell primitive (rho, U, V, T): the Rankine-Hugoniot step at x = 0."""
    xs = mesh.xv[: mesh.ni + 1]
    xc = 0.5 * (xs[:-1] + xs[1:])
    rho2, u2, T2 = rankine_hugoniot(Ma)
    prim = np.zeros((mesh.ni, 4))
    up = xc < 0.0
    prim[up] = [1.0, freestream_speed(Ma), 0.0, 1.0]
    prim[~up] = [rho2, u2, 0.0, T2]
    return prim


@dataclass
class Case:
    name: str
    mesh: Mesh | UMesh
    Kn: float
    Ma: float
    Tw: float
    cfl: float
    omega: float = 0.81
    Pr: float = 1.0
    n_ref: int = 100
    wall_specular: float = 0.0                  # Maxwell wall: specular fraction 1 - alpha (0: fully diffuse)
    seed: int = 0
    ghost_state: tuple = (1.0, 0.0, 0.0, 1.0)   # (rho, U, V, T) used by BC_FIXED faces
    init_prim: np.ndarray | None = None


def case_shock1d(ni: int = 200, n_ref: int = 100, Ma: float = 3.0, Pr: float = 2.0 / 3.0) -> Case:
    """1-D normal shock, Ma 3, 200 cells stretched 50x, x in [-30, 30] mean free paths (Kn = 1 on lambda)."""
    m = line_mesh(ni, -30.0, 30.0, end_ratio=50.0, bc_left=BC_FARFIELD, bc_right=BC_FIXED)
    rho2, u2, T2 = rankine_hugoniot(Ma)
    c = Case("shock1d", m, Kn=1.0, Ma=Ma, Tw=1.0, cfl=0.5, omega=0.81, Pr=Pr, n_ref=n_ref,
             ghost_state=(rho2, u2, 0.0, T2))
    c.init_prim = shock_initial_field(m, Ma)
    return c


def case_cylinder(ni: int = 120, nj: int = 160, h1: float = 1e-3, r_out: float = 15.0, Kn: float = 0.1,
                  Ma: float = 5.0, Tw: float = 1.0, n_ref: int = 100, cfl: float = 0.8) -> Case:
    """Hypersonic cylinder (diameter 1) on a body-fitted O-mesh; Kn on the diameter."""
    return Case(f"cylinder_{ni}x{nj}_Kn{Kn}_Ma{Ma}", omesh(ni, nj, h1, r_out), Kn=Kn, Ma=Ma, Tw=Tw, cfl=cfl,
                n_ref=n_ref)


def case_cylinder_kn01() -> Case:
    return case_cylinder(120, 160, 1e-3, 15.0, Kn=0.1, Ma=5.0, n_ref=100)


def case_cylinder_kn001() -> Case:
    return case_cylinder(240, 320, 1e-4, 20.0, Kn=0.01, Ma=15.0, n_ref=150)


def case_cylinder_tri(n_quad: int = 13, ni: int = 33, nj: int = 140, h1: float = 0.005, r_out: float = 15.0,
                      Kn: float = 0.05, Ma: float = 5.0, Tw: float = 1.0, n_ref: int = 100, cfl: float = 0.8) -> Case:
    """Hypersonic cylinder on a hybrid unstructured mesh standing in for the paper's Kn = 0.1 case (Sec. V A:
    Kn on the radius, 7,420 cells, first wall cell 0.01 R; here Kn is on the diameter, so 0.05):
    13 quadrilateral layers at the wall and 20 triangulated layers."""
    m = tri_omesh(n_quad, ni, nj, h1, r_out)
    return Case(f"cylinder_tri_{m.ncells}_Kn{Kn}_Ma{Ma}", m, Kn=Kn, Ma=Ma, Tw=Tw, cfl=cfl, n_ref=n_ref)


def case_cylinder_tri_kn001() -> Case:
    """The paper's dense-regime cylinder (Sec. V A: Ma 5, Kn 0.01 on the radius, 16,100 cells, first wall cell
    0.0005 R, N_ref 100) on a hybrid stand-in: 15 quadrilateral layers and 50 triangulated ones, 140 around."""
    return case_cylinder_tri(15, 65, 140, 0.00025, 15.0, Kn=0.005, Ma=5.0, n_ref=100)


def case_plate_tri() -> Case:
    """The paper's hypersonic plate (Sec. V B: Ma 20.2, Kn 0.0169 on L, T_w / T_inf = 290 / 13.32, Maxwell wall
    with accommodation 0.85, 5,885 cells, first cell 1e-5 L, N_ref 200) on a hybrid stand-in of 107 columns,
    15 quadrilateral rows and 20 triangulated ones; a monatomic gas (omega 0.81) stands in for nitrogen."""
    m = tri_plate()
    return Case(f"plate_tri_{m.ncells}_Kn0.0169_Ma20.2", m, Kn=0.0169, Ma=20.2, Tw=290.0 / 13.32, cfl=0.8,
                n_ref=200, wall_specular=0.15)


def case_periodic_box(ni: int = 16, end_ratio: float = 50.0, n_ref: int = 50, Kn: float = 0.05,
                      seed: int = 0) -> Case:
    """Closed periodic 1-D box with cell sizes varying end_ratio times: a smooth density/temperature wave."""
    m = line_mesh(ni, 0.0, 1.0, end_ratio=end_ratio, bc_left=BC_PERIODIC, bc_right=BC_PERIODIC)
    xs = m.xv[: ni + 1]
    xc = 0.5 * (xs[:-1] + xs[1:])
    prim = np.zeros((ni, 4))
    prim[:, 0] = 1.0 + 0.2 * np.sin(2 * np.pi * xc)
    prim[:, 1] = 0.3 * np.cos(2 * np.pi * xc)
    prim[:, 3] = 1.0 + 0.1 * np.cos(2 * np.pi * xc)
    c = Case("periodic_box", m, Kn=Kn, Ma=0.0, Tw=1.0, cfl=0.5, n_ref=n_ref, seed=seed)
    c.init_prim = prim
    return c


def case_plate(Kn: float = 0.0169, Ma: float = 5.0, Tw: float = 1.0, n_ref: int = 50, ni: int = 240, nj: int = 120,
               h1: float = 1e-4, ratio: float = 1.06, cfl: float = 0.8) -> Case:
    """Sharp flat plate of length L = 1 on a 240 x 120 Cartesian mesh, Kn on L, wall at T_w for 0 <= x <= 1."""
    return Case(f"plate_{ni}x{nj}_Kn{Kn:.4g}_Ma{Ma:.3g}", plate_mesh(ni, nj, h1, ratio), Kn=Kn, Ma=Ma, Tw=Tw,
                cfl=cfl, n_ref=n_ref)


def batch_sweep(seed: int = 0, n_cases: int = 16, n_plates: int = 4, scale: float = 1.0):
    """Seeded sweep of uneven 2-D cases: cylinders (the 120 x 160 or the 240 x 320 O-mesh, chosen by a
    uniform draw) and flat plates in a fixed split; log10 Kn ~ U[log10 0.005, log10 0.2], Ma ~ U[5, 15],
    T_w / T_inf ~ U[1, 5]; N_ref per case so that it holds about 2-12 million particles (times `scale`)."""
    rng = np.random.default_rng(seed)
    cases = []
    for k in range(n_cases):
        kn = 10.0 ** rng.uniform(math.log10(0.005), math.log10(0.2))
        ma = rng.uniform(5.0, 15.0)
        tw = rng.uniform(1.0, 5.0)
        target = rng.uniform(2e6, 12e6) * scale
        if k < n_cases - n_plates:
            big = rng.uniform() < 0.5
            ni, nj, h1, ro = (240, 320, 1e-4, 20.0) if big else (120, 160, 1e-3, 15.0)
            n_ref = max(4, int(round(target / (ni * nj))))
            c = case_cylinder(ni, nj, h1, ro, Kn=kn, Ma=ma, Tw=tw, n_ref=n_ref)
        else:
            n_ref = max(4, int(round(target / (240 * 120))))
            c = case_plate(Kn=kn, Ma=ma, Tw=tw, n_ref=n_ref)
        c.seed = seed * 1000 + k
        cases.append(c)
    return cases


def mlp_init(seed: int, n_features: int = 64, width: int = 256, depth: int = 4, n_out: int = 4) -> np.ndarray:
    """Seeded initial parameters of the warm-start network (float32): weights uniform in (-a, a) with
    a = sqrt(6 / fan_in), zero biases. Layout: every layer's weight matrix [out][in] row-major in layer order,
    then every layer's bias in layer order."""
    rng = np.random.default_rng(seed)
    ins = [n_features] + [width] * depth
    outs = [width] * depth + [n_out]
    parts = [rng.uniform(-math.sqrt(6.0 / i), math.sqrt(6.0 / i), size=i * o) for i, o in zip(ins, outs)]
    parts += [np.zeros(o) for o in outs]
    return np.concatenate(parts).astype(np.float32)


def held_out_conditions(seed: int = 1000, n_cyl: int = 4, n_plate: int = 4):
    """Seeded (geometry, Kn, Ma, T_w) conditions for evaluation cases, drawn from the same ranges as
    `batch_sweep` but from a different seed."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_cyl + n_plate):
        kn = 10.0 ** rng.uniform(math.log10(0.005), math.log10(0.2))
        ma = rng.uniform(5.0, 15.0)
        tw = rng.uniform(1.0, 5.0)
        out.append(("cylinder" if k < n_cyl else "plate", kn, ma, tw))
    return out
