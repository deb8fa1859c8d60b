"""Seeded synthetic quad/hex meshes shaped like the paper's workloads.

Input generators only: vertex coordinates, corner connectivity, optional
high-order geometry nodes and boundary tags.  Nothing here evaluates any part
of the Flux Reconstruction method (no quadrature points, metrics, fluxes or
face-point matching); both the FP64 oracle and the CUDA library derive all of
that themselves from a ``Mesh``.

Conventions shared by every consumer of a ``Mesh``:

* corners of an element are listed in tensor order of the reference
  coordinates, xi fastest: quad (-1,-1), (1,-1), (-1,1), (1,1); hex the same
  square at zeta=-1 followed by the square at zeta=+1;
* faces are numbered -xi, +xi, -eta, +eta (, -zeta, +zeta);
* optional geometry nodes are the element map sampled at the equispaced
  tensor lattice of degree ``geo_order`` (xi fastest), corners included;
* face tags: 0 interior (matched through shared corner vertices), 1 periodic
  (matched to a face whose corners coincide after adding or subtracting one
  of ``periodic_shift``), 2 no-slip adiabatic wall, 3 characteristic far
  field, 4 inflow (far field with a boundary-layer profile), 5 outflow
  (characteristic, same construction as far field).

Workload shapes follow the paper: cavity (Sec. 3.1.1: inlet 5D upstream,
outlet 60D downstream with a 50D buffer, domain height 15D with a 5D buffer,
stretching 1.05 / 1.075), NACA 4-digit O-meshes (Sec. 5), periodic boxes for
the isentropic vortex and Taylor-Green cases.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

TAG_INTERIOR = 0
TAG_PERIODIC = 1
TAG_WALL = 2
TAG_FARFIELD = 3
TAG_INFLOW = 4
TAG_OUTFLOW = 5


@dataclass
class Mesh:
    dim: int
    xyz: np.ndarray                 # (n_vert, dim) float64
    elem_vert: np.ndarray           # (n_elem, 2**dim) int64
    face_tag: np.ndarray            # (n_elem, 2*dim) int32
    periodic_shift: np.ndarray      # (n_shift, dim) float64
    geo_order: int = 1
    geo_nodes: np.ndarray | None = None   # (n_elem, (q+1)**dim, dim) float64
    info: dict = field(default_factory=dict)

    @property
    def n_elem(self) -> int:
        return int(self.elem_vert.shape[0])

    def node_coords(self) -> np.ndarray:
        """Geometry nodes of every element, (n_elem, (q+1)**dim, dim)."""
        if self.geo_nodes is not None:
            return self.geo_nodes
        return self.xyz[self.elem_vert]


# ---------------------------------------------------------------------------
# boundary classification helper (pure bookkeeping on corner vertex ids)
# ---------------------------------------------------------------------------

_QUAD_FACES = [(0, 2), (1, 3), (0, 1), (2, 3)]
_HEX_FACES = [(0, 2, 4, 6), (1, 3, 5, 7), (0, 1, 4, 5), (2, 3, 6, 7),
              (0, 1, 2, 3), (4, 5, 6, 7)]


def face_corners(dim: int):
    return _QUAD_FACES if dim == 2 else _HEX_FACES


def _tag_unmatched(elem_vert, xyz, dim, classify):
    """Tag every face without a vertex-sharing partner via ``classify``."""
    faces = face_corners(dim)
    n_elem = elem_vert.shape[0]
    tags = np.zeros((n_elem, 2 * dim), dtype=np.int32)
    keys = {}
    for e in range(n_elem):
        for f, loc in enumerate(faces):
            k = tuple(sorted(int(elem_vert[e, c]) for c in loc))
            keys.setdefault(k, []).append((e, f))
    for k, lst in keys.items():
        if len(lst) == 1:
            e, f = lst[0]
            centre = xyz[list(k)].mean(axis=0)
            tags[e, f] = classify(centre, f)
        elif len(lst) > 2:
            raise ValueError("non-manifold face in generated mesh")
    return tags


# ---------------------------------------------------------------------------
# G1 / G3: periodic Cartesian boxes
# ---------------------------------------------------------------------------

def periodic_box(dim: int, n, lo, hi, jitter: float = 0.0, seed: int = 2312) -> Mesh:
    """Periodic box of n[0] x n[1] (x n[2]) straight-sided elements.

    ``jitter`` moves every vertex that is not on the box boundary by a seeded
    uniform offset of at most ``jitter`` times the local spacing, giving
    non-affine elements for free-stream tests.
    """
    n = [int(v) for v in n]
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    axes = [np.linspace(lo[a], hi[a], n[a] + 1) for a in range(dim)]
    grids = np.meshgrid(*axes, indexing="ij")
    xyz = np.stack([g.ravel(order="F") for g in grids], axis=1)  # x fastest
    nv = [v + 1 for v in n]

    def vid(idx):
        out = 0
        stride = 1
        for a in range(dim):
            out += idx[a] * stride
            stride *= nv[a]
        return out

    elems = []
    if dim == 2:
        for j in range(n[1]):
            for i in range(n[0]):
                elems.append([vid((i, j)), vid((i + 1, j)),
                              vid((i, j + 1)), vid((i + 1, j + 1))])
    else:
        for k in range(n[2]):
            for j in range(n[1]):
                for i in range(n[0]):
                    elems.append([vid((i + a, j + b, k + c))
                                  for c in (0, 1) for b in (0, 1) for a in (0, 1)])
    elem_vert = np.asarray(elems, dtype=np.int64)

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        h = (hi - lo) / np.asarray(n, float)
        inner = np.ones(xyz.shape[0], bool)
        for a in range(dim):
            inner &= (xyz[:, a] > lo[a] + 1e-12) & (xyz[:, a] < hi[a] - 1e-12)
        off = rng.uniform(-1.0, 1.0, size=xyz.shape) * h * jitter
        xyz = xyz + off * inner[:, None]

    shift = np.diag(hi - lo)
    tags = _tag_unmatched(elem_vert, xyz, dim, lambda c, f: TAG_PERIODIC)
    return Mesh(dim=dim, xyz=xyz, elem_vert=elem_vert, face_tag=tags,
                periodic_shift=shift, info={"kind": "periodic_box", "n": n})


def vortex_mesh(n: int = 16, jitter: float = 0.0, seed: int = 2312) -> Mesh:
    """Isentropic-vortex box [-5,5]^2 with n x n quads."""
    return periodic_box(2, (n, n), (-5.0, -5.0), (5.0, 5.0), jitter, seed)


def curved_periodic_box(n: int, q: int, amp: float = 0.15) -> Mesh:
    """Periodic (2 pi)^3 box of n^3 hexes, every element curved in all three
    directions: the map X -> X + amp (sin Y sin Z, sin Z sin X, sin X sin Y)
    (periodic, so periodic faces still match) sampled at the degree-q node
    lattice of each element."""
    b = periodic_box(3, (n, n, n), (0, 0, 0), (2 * np.pi,) * 3)

    def warp(X):
        s = np.sin(X)
        return X + amp * np.stack([s[..., 1] * s[..., 2], s[..., 2] * s[..., 0],
                                   s[..., 0] * s[..., 1]], -1)

    h = 2 * np.pi / n
    x0 = b.xyz[b.elem_vert].min(axis=1)
    t = np.linspace(0.0, 1.0, q + 1)
    lat = np.array([[i, j, k] for k in t for j in t for i in t])      # xi fastest
    nodes = warp(x0[:, None, :] + h * lat[None])
    return Mesh(dim=3, xyz=warp(b.xyz), elem_vert=b.elem_vert, face_tag=b.face_tag,
                periodic_shift=b.periodic_shift, geo_order=q, geo_nodes=nodes,
                info={"kind": "curved_box"})


def tgv_mesh(n: int = 16) -> Mesh:
    """Taylor-Green box [0, 2 pi]^3 with n^3 hexes."""
    two_pi = 2.0 * np.pi
    return periodic_box(3, (n, n, n), (0.0, 0.0, 0.0), (two_pi, two_pi, two_pi))


# ---------------------------------------------------------------------------
# 1-D graded distributions
# ---------------------------------------------------------------------------

def graded_line(x0: float, x1: float, h0: float, ratio: float, at_start=True):
    """Nodes from x0 to x1 whose spacing starts at about h0 at one end and
    grows geometrically by ``ratio``; the last cell is absorbed so that the
    end point is hit exactly."""
    length = abs(x1 - x0)
    sizes = []
    h = h0
    tot = 0.0
    while tot + h < length - 1e-12:
        sizes.append(h)
        tot += h
        h *= ratio
    if not sizes:
        sizes = [length]
    else:
        rem = length - tot
        if rem < 0.5 * sizes[-1]:
            sizes[-1] += rem
        else:
            sizes.append(rem)
    sizes = np.asarray(sizes)
    if not at_start:
        sizes = sizes[::-1]
    s = np.concatenate([[0.0], np.cumsum(sizes)])
    s *= length / s[-1]
    return x0 + np.sign(x1 - x0) * s


def _two_zone(x0, x1, xb, h0, r1, r2):
    """Spacing h0 at x0 grows by r1 up to xb, then by r2 to x1 (a buffer)."""
    a = graded_line(x0, xb, h0, r1)
    if abs(x1 - xb) < 1e-12:
        return a
    hb = abs(a[-1] - a[-2])
    b = graded_line(xb, x1, hb * r2, r2)
    return np.concatenate([a, b[1:]])


# ---------------------------------------------------------------------------
# G2: 2-D deep-cavity proxy
# ---------------------------------------------------------------------------

def _cavity_count(h0, LD):
    xs = _cavity_x(h0, LD)
    ys, yc = _cavity_y(h0)
    return (len(xs) - 1) * (len(ys) - 1) + (len(_cavity_xc(xs, LD)) - 1) * (len(yc) - 1)


def _cavity_x(h0, LD):
    ncav = max(2, int(round(LD / h0)))
    xc = np.linspace(0.0, LD, ncav + 1)
    up = _two_zone(0.0, -5.0, -5.0, xc[1] - xc[0], 1.05, 1.05)[::-1]
    down = _two_zone(LD, LD + 60.0, LD + 10.0, xc[1] - xc[0], 1.05, 1.075)
    return np.concatenate([up[:-1], xc, down[1:]])


def _cavity_xc(xs, LD):
    return xs[(xs >= -1e-12) & (xs <= LD + 1e-12)]


def _cavity_y(h0):
    ys = _two_zone(0.0, 15.0, 10.0, h0, 1.05, 1.075)
    nc = max(2, int(round(1.0 / h0)))
    yc = np.linspace(-1.0, 0.0, nc + 1)
    return ys, yc


def cavity_mesh(target_elems: int = 32000, LD: float = 0.5, seed: int = 2312) -> Mesh:
    """2-D channel over a flat plate with a rectangular cavity of depth D=1.

    Cavity occupies 0<x<LD, -1<y<0.  Plate wall at y=0 elsewhere; inflow at
    x=-5 (5D upstream), outflow at x=LD+60 with the last 50D stretched by 1.075
    as a buffer; top boundary at y=15 with the last 5D stretched by 1.075.
    The minimum spacing is found by bisection so that the element count is
    close to ``target_elems``.  ``seed`` is accepted for interface symmetry;
    the cavity proxy has no random component.
    """
    lo, hi = 1e-3, 0.5
    for _ in range(60):
        mid = np.sqrt(lo * hi)
        if _cavity_count(mid, LD) > target_elems:
            lo = mid
        else:
            hi = mid
    h0 = hi
    xs = _cavity_x(h0, LD)
    ys, yc = _cavity_y(h0)
    xc = _cavity_xc(xs, LD)
    nx, ny = len(xs), len(ys)
    # channel block vertices
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    pts = [np.stack([X.ravel(order="F"), Y.ravel(order="F")], 1)]

    def vA(i, j):
        return i + nx * j

    # cavity block shares its top row (y=0) with the channel block
    i0 = int(np.where(np.abs(xs) < 1e-12)[0][0])
    ncx, ncy = len(xc), len(yc)
    base = nx * ny
    Xc, Yc = np.meshgrid(xc, yc[:-1], indexing="ij")
    pts.append(np.stack([Xc.ravel(order="F"), Yc.ravel(order="F")], 1))

    def vC(i, j):
        if j == ncy - 1:
            return vA(i0 + i, 0)
        return base + i + ncx * j

    elems = []
    for j in range(ny - 1):
        for i in range(nx - 1):
            elems.append([vA(i, j), vA(i + 1, j), vA(i, j + 1), vA(i + 1, j + 1)])
    for j in range(ncy - 1):
        for i in range(ncx - 1):
            elems.append([vC(i, j), vC(i + 1, j), vC(i, j + 1), vC(i + 1, j + 1)])
    xyz = np.concatenate(pts, 0)
    elem_vert = np.asarray(elems, np.int64)
    x_in, x_out, y_top = xs[0], xs[-1], ys[-1]

    def classify(c, f):
        if abs(c[0] - x_in) < 1e-9:
            return TAG_INFLOW
        if abs(c[0] - x_out) < 1e-9:
            return TAG_OUTFLOW
        if abs(c[1] - y_top) < 1e-9:
            return TAG_FARFIELD
        return TAG_WALL

    tags = _tag_unmatched(elem_vert, xyz, 2, classify)
    probe = np.array([0.5 * LD, 7.16])
    # dense sampling of the walls: plate, cavity sides and floor
    hs = 0.25 * h0
    seg = lambda a, b: np.linspace(a, b, max(2, int(np.linalg.norm(np.subtract(b, a)) / hs)))
    wall = np.concatenate([
        np.stack([seg(x_in, 0.0), np.zeros(len(seg(x_in, 0.0)))], 1),
        np.stack([np.zeros(len(seg(0.0, -1.0))), seg(0.0, -1.0)], 1),
        np.stack([seg(0.0, LD), np.full(len(seg(0.0, LD)), -1.0)], 1),
        np.stack([np.full(len(seg(-1.0, 0.0)), LD), seg(-1.0, 0.0)], 1),
        np.stack([seg(LD, x_out), np.zeros(len(seg(LD, x_out)))], 1)])
    return Mesh(dim=2, xyz=xyz, elem_vert=elem_vert, face_tag=tags,
                periodic_shift=np.zeros((0, 2)),
                info={"kind": "cavity", "LD": LD, "h0": h0, "probe": probe,
                      "wall_y": 0.0, "x_inflow": x_in, "wall_points": wall})


# ---------------------------------------------------------------------------
# G4: NACA 4-digit O-meshes
# ---------------------------------------------------------------------------

def naca4(m: float, pc: float, t: float, xc: np.ndarray):
    """Upper and lower surface points of a NACA 4-digit profile at chord
    stations xc (standard open trailing edge: a blunt base of height about
    0.021 t)."""
    yt = 5.0 * t * (0.2969 * np.sqrt(xc) - 0.1260 * xc - 0.3516 * xc ** 2
                    + 0.2843 * xc ** 3 - 0.1015 * xc ** 4)
    if m > 0.0:
        yc = np.where(xc < pc, m / pc ** 2 * (2 * pc * xc - xc ** 2),
                      m / (1 - pc) ** 2 * ((1 - 2 * pc) + 2 * pc * xc - xc ** 2))
        dy = np.where(xc < pc, 2 * m / pc ** 2 * (pc - xc),
                      2 * m / (1 - pc) ** 2 * (pc - xc))
    else:
        yc = np.zeros_like(xc)
        dy = np.zeros_like(xc)
    th = np.arctan(dy)
    xu, yu = xc - yt * np.sin(th), yc + yt * np.cos(th)
    xl, yl = xc + yt * np.sin(th), yc - yt * np.cos(th)
    return xu, yu, xl, yl


def _naca_surface(m, pc, t, s, s_base=0.0):
    """Surface point at O-mesh parameter s in [0,1), clockwise: s in
    [0, s_base/2) runs down the lower half of the blunt trailing-edge base
    from its midpoint, [s_base/2, 0.5) along the lower surface from the
    trailing edge to the leading edge, [0.5, 1 - s_base/2) back over the upper
    surface and [1 - s_base/2, 1) down the upper half of the base."""
    s = np.asarray(s, float) % 1.0
    hb = 0.5 * s_base
    xu1, yu1, xl1, yl1 = naca4(m, pc, t, np.array([1.0]))
    xm, ym = 0.5 * (xu1[0] + xl1[0]), 0.5 * (yu1[0] + yl1[0])
    lower = s < 0.5
    if hb > 0:
        u = np.where(lower, 1.0 - (s - hb) / (0.5 - hb), (s - 0.5) / (0.5 - hb))
    else:
        u = np.where(lower, 1.0 - 2.0 * s, 2.0 * s - 1.0)   # 1 at TE, 0 at LE
    u = np.clip(u, 0.0, 1.0)
    # clustered at the leading edge only; spacing at the trailing edge stays
    # comparable to the wall-normal cells so that no cell there is a sliver
    xc = 1.0 - np.cos(0.5 * np.pi * u)
    xu, yu, xl, yl = naca4(m, pc, t, xc)
    x = np.where(lower, xl, xu)
    y = np.where(lower, yl, yu)
    if hb > 0:
        b_lo = s < hb
        b_up = s >= 1.0 - hb
        f_lo = s / hb
        f_up = (s - (1.0 - hb)) / hb
        x = np.where(b_lo, xm + f_lo * (xl1[0] - xm), x)
        y = np.where(b_lo, ym + f_lo * (yl1[0] - ym), y)
        x = np.where(b_up, xu1[0] + f_up * (xm - xu1[0]), x)
        y = np.where(b_up, yu1[0] + f_up * (ym - yu1[0]), y)
    return x, y


def naca_omesh(m: float, pc: float, t: float, aoa_deg: float, n_elem: int,
               p_geo: int = 3, radius: float = 20.0) -> Mesh:
    """Curved O-mesh around a NACA 4-digit profile of unit chord.

    N_theta x N_r quads, geometric stretching in the radial direction out to
    ``radius`` chords, geometry nodes of degree ``p_geo`` sampled from the
    continuous map, profile rotated about the quarter chord so that a free
    stream along +x meets it at ``aoa_deg``.  Wall tag on the profile, far
    field on the outer circle; the O-cut is an ordinary interior connection.
    """
    nr = max(4, int(round(np.sqrt(n_elem / 2.0))))
    nth = max(8, 2 * int(round(n_elem / nr / 2.0)))
    q = int(p_geo)
    # radial distance: geometric cells from h_wall at the profile to ``radius``
    h_wall = 1e-3
    lo_r, hi_r = 1.0 + 1e-9, 2.0
    for _ in range(200):
        mid = 0.5 * (lo_r + hi_r)
        if h_wall * (mid ** nr - 1.0) / (mid - 1.0) > radius:
            hi_r = mid
        else:
            lo_r = mid
    ratio = 0.5 * (lo_r + hi_r)

    def dist(sr):
        return h_wall * (ratio ** (sr * nr) - 1.0) / (ratio - 1.0)

    s_base = 2.0 / nth                    # one theta cell per half of the base

    def surf(sth):
        return _naca_surface(m, pc, t, sth, s_base)

    def raw_normal(sth):
        # outward normal of the clockwise surface curve: tangent rotated +90 deg
        ds = 1e-7
        xp, yp = surf(sth + ds)
        xm_, ym_ = surf(sth - ds)
        tx, ty = xp - xm_, yp - ym_
        nrm = np.hypot(tx, ty)
        return -ty / nrm, tx / nrm

    sigma = 1.5 / nth

    def normal(sth):
        """Surface normal averaged with Gaussian weights over about three
        cells along the wall, so the departure direction turns smoothly
        around the corners of the trailing-edge base."""
        sth = np.asarray(sth, float)
        ax, ay = np.zeros_like(sth), np.zeros_like(sth)
        for k in range(-64, 65):
            w = np.exp(-0.5 * (k / 16.0) ** 2)
            nx0, ny0 = raw_normal(sth + k * sigma / 16.0)
            ax += w * nx0
            ay += w * ny0
        nrm = np.hypot(ax, ay)
        return ax / nrm, ay / nrm

    # Lines leave the wall along the smoothed normal (blend weight
    # g = rho (1 - rho)^2 on a unit chord) and end on the far-field circle
    # (weight h = rho^2), rho in [0, 1] from the radial distance.
    # fine lattice of geometry nodes, shared by neighbouring elements; the map
    # is separable, so evaluate the wall quantities once per theta station
    fth = np.arange(nth * q) / (nth * q)
    fr = np.arange(nr * q + 1) / (nr * q)
    xs, ys = surf(fth)
    nx_, ny_ = normal(fth)
    ang = 2.0 * np.pi * fth
    xf = 0.5 + radius * np.cos(ang)
    yf = -radius * np.sin(ang)
    d = dist(fr)
    rho = (-1.0 + np.sqrt(1.0 + 4.0 * radius * d)) / (2.0 * radius)
    h = (rho * rho)[None, :]
    g = (rho * (1.0 - rho) ** 2)[None, :]
    FX = (1 - h) * xs[:, None] + h * xf[:, None] + g * nx_[:, None]
    FY = (1 - h) * ys[:, None] + h * yf[:, None] + g * ny_[:, None]
    # rotate by -aoa about quarter chord
    a = np.deg2rad(aoa_deg)
    ca, sa = np.cos(a), np.sin(a)
    FX0, FY0 = FX - 0.25, FY
    FX, FY = 0.25 + ca * FX0 + sa * FY0, -sa * FX0 + ca * FY0
    # corner vertices
    xyz = np.stack([FX[::q, ::q].ravel(order="F"), FY[::q, ::q].ravel(order="F")], 1)

    def vid(i, j):
        return (i % nth) + nth * j

    jj_e, ii_e = np.meshgrid(np.arange(nr), np.arange(nth), indexing="ij")
    ii_e, jj_e = ii_e.ravel(), jj_e.ravel()          # element (i, j), theta fastest
    elems = np.stack([vid(ii_e, jj_e), vid(ii_e + 1, jj_e), vid(ii_e, jj_e + 1),
                      vid(ii_e + 1, jj_e + 1)], 1)
    a_loc = np.arange(q + 1)
    # node (a, b) of element (i, j): lattice index (i q + a, j q + b), a fastest
    la = ((ii_e[:, None, None] * q + a_loc[None, None, :]) % (nth * q))
    lb = (jj_e[:, None, None] * q + a_loc[None, :, None])
    la, lb = np.broadcast_arrays(la, lb)
    nodes = np.stack([FX[la, lb].reshape(len(ii_e), -1), FY[la, lb].reshape(len(ii_e), -1)], -1)
    elem_vert = np.asarray(elems, np.int64)
    geo_nodes = np.ascontiguousarray(nodes)
    # the profile wall is eta=-1 of the first ring, the far field eta=+1 of the last
    tags = np.zeros((elem_vert.shape[0], 4), np.int32)
    tags[:nth, 2] = TAG_WALL
    tags[(nr - 1) * nth:, 3] = TAG_FARFIELD
    te = np.array([0.25 + ca * 0.75, -sa * 0.75])
    # dense sampling of the wall (for wall-distance based initial states)
    ws = np.linspace(0.0, 1.0, 8 * nth * q, endpoint=False)
    wx, wy = surf(ws)
    wx0 = wx - 0.25
    wall = np.stack([0.25 + ca * wx0 + sa * wy, -sa * wx0 + ca * wy], 1)
    return Mesh(dim=2, xyz=xyz, elem_vert=elem_vert, face_tag=tags,
                periodic_shift=np.zeros((0, 2)), geo_order=q, geo_nodes=geo_nodes,
                info={"kind": "naca", "m": m, "pc": pc, "t": t, "aoa": aoa_deg,
                      "nth": nth, "nr": nr, "probe": te + np.array([0.0, -2.0]),
                      "wall_points": wall})


def airfoil_batch(n_inst: int = 32, seed: int = 2312, e_lo: int = 8000,
                  e_hi: int = 40000, p_geo: int = 3):
    """One MADS poll's worth of NACA 4-digit candidates, drawn from ``seed``:
    max camber U[0,0.06], camber position U[0.2,0.6], thickness U[0.08,0.16],
    angle of attack U[0,6] deg, element count U[e_lo, e_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        m = rng.uniform(0.0, 0.06)
        pc = rng.uniform(0.2, 0.6)
        t = rng.uniform(0.08, 0.16)
        aoa = rng.uniform(0.0, 6.0)
        ne = int(rng.uniform(e_lo, e_hi))
        out.append(naca_omesh(m, pc, t, aoa, ne, p_geo))
    return out


def concat_info(meshes):
    return [mm.info for mm in meshes]


# ---------------------------------------------------------------------------
# G5: spanwise-extruded tandem cylinders (3-D hexes)
# ---------------------------------------------------------------------------

def _graded_from(x0, x1, h, r_res, dist_res, r_buf):
    """Nodes from x0 towards x1 (either direction): spacing h growing by
    r_res for dist_res, then by r_buf (buffer) to x1."""
    sgn = 1.0 if x1 > x0 else -1.0
    L = abs(x1 - x0)
    nodes = [0.0]
    hh = h
    while nodes[-1] + hh < L - 1e-12:
        nodes.append(nodes[-1] + hh)
        hh *= r_res if nodes[-1] < dist_res else r_buf
    if L - nodes[-1] < 0.5 * hh and len(nodes) > 1:
        nodes[-1] = L
    else:
        nodes.append(L)
    return x0 + sgn * np.asarray(nodes)


def tandem_cylinders_2d(s_gap: float, r_ratio: float, target_quads: int, q: int = 2):
    """2-D section: cylinders of diameters D1 = 1 (centre at the origin) and
    D2 = r_ratio, surface gap s_gap (rear of the upstream to the front of the
    downstream cylinder), each inside an O-ring that ends on a square hole of
    a Cartesian background; inlet 5 D1 upstream, outlet 55 D1 downstream of
    the second cylinder, +-10 D1 laterally; stretching 1.05 (resolved) and
    1.075 (buffer).  Returns (xyz, elem_vert, geo_nodes (q), wall/outflow
    edge tags, info)."""
    R1, R2 = 0.5, 0.5 * r_ratio
    x1, x2 = 0.0, R1 + s_gap + R2
    x_in, x_out, y_max = x1 - 5.0, x2 + 55.0, 10.0

    def count(h):
        m1 = max(4, 2 * int(round(1.5 * R1 * 2 / h / 2)))
        m2 = max(4, 2 * int(round(1.5 * R2 * 2 / h / 2)))
        H1, H2 = 0.5 * m1 * h, 0.5 * m2 * h
        gap = (x2 - H2) - (x1 + H1)
        ng = max(1, int(round(gap / h)))
        nr = max(3, int(round(0.6 * m1)))
        Ymax = max(H1, H2)
        xs_core = (x2 + H2) - (x1 - H1)
        ny_core = 2 * int(round(Ymax / h))
        xs = len(_graded_from(0, 5 - H1, h, 1.05, 3.0, 1.075)) + \
            len(_graded_from(0, 55 - H2, h, 1.05, 12.0, 1.075)) + int(round(xs_core / h))
        ys = ny_core + 2 * len(_graded_from(0, y_max - Ymax, h, 1.05, 3.0, 1.075))
        return xs * ys - m1 * m1 - m2 * m2 + 4 * m1 * nr + 4 * m2 * nr

    lo, hi = 0.01, 1.0
    for _ in range(50):
        mid = np.sqrt(lo * hi)
        if count(mid) > target_quads:
            lo = mid
        else:
            hi = mid
    h0 = hi
    m1 = max(4, 2 * int(round(1.5 * R1 * 2 / h0 / 2)))
    m2 = max(4, 2 * int(round(1.5 * R2 * 2 / h0 / 2)))
    # one spacing for both holes: the gap between them a whole number of cells
    H1g, H2g = 0.5 * m1 * h0, 0.5 * m2 * h0
    ng = max(1, int(round(((x2 - H2g) - (x1 + H1g)) / h0)))
    h = ((x2 - x1)) / (0.5 * m1 + ng + 0.5 * m2)
    H1, H2 = 0.5 * m1 * h, 0.5 * m2 * h
    Ymax = max(H1, H2)
    ny2 = int(round(Ymax / h))
    # x and y nodes: uniform core, graded outside
    core_x = x1 - H1 + h * np.arange(m1 + ng + m2 + 1)
    up = _graded_from(core_x[0], x_in, h * 1.05, 1.05, 3.0, 1.075)[::-1]
    down = _graded_from(core_x[-1], x_out, h * 1.05, 1.05, 12.0, 1.075)
    xs = np.concatenate([up[:-1], core_x, down[1:]])
    core_y = h * np.arange(-ny2, ny2 + 1)
    top = _graded_from(core_y[-1], y_max, h * 1.05, 1.05, 3.0, 1.075)
    ys = np.concatenate([-top[::-1][:-1], core_y, top[1:]])
    nx, ny = len(xs), len(ys)
    i0 = len(up) - 1            # index of core_x[0] in xs
    j0 = len(top) - 1           # index of core_y[0] in ys
    vid_bg = lambda i, j: i + nx * j
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    pts = [np.stack([X.ravel(order="F"), Y.ravel(order="F")], 1)]
    nvert = nx * ny
    # holes in background index space: cells [a, b) x [c, d)
    holes = []
    for (xc, m) in ((x1, m1), (x2, m2)):
        ia = i0 + int(round((xc - 0.5 * m * h - core_x[0]) / h))
        ja = j0 + ny2 - m // 2
        holes.append((ia, ia + m, ja, ja + m))
    elems, nodes = [], []
    a = np.linspace(0.0, 1.0, q + 1)
    # background quads (straight): nodes by bilinear interpolation
    for j in range(ny - 1):
        for i in range(nx - 1):
            if any(hx0 <= i < hx1 and hy0 <= j < hy1 for hx0, hx1, hy0, hy1 in holes):
                continue
            c = [vid_bg(i, j), vid_bg(i + 1, j), vid_bg(i, j + 1), vid_bg(i + 1, j + 1)]
            elems.append(c)
            B, T_ = np.meshgrid(a, a, indexing="ij")   # [xi, eta]
            xx = xs[i] + (xs[i + 1] - xs[i]) * B
            yy = ys[j] + (ys[j + 1] - ys[j]) * T_
            nodes.append(np.stack([xx.T.ravel(), yy.T.ravel()], 1))
    # O-rings
    for (xc, R, m, (hx0, hx1, hy0, hy1)) in ((x1, R1, m1, holes[0]), (x2, R2, m2, holes[1])):
        H = 0.5 * m * h
        nr = max(3, int(round(0.6 * m)))
        ratio = 1.15

        def frac(r):      # radial fraction, geometric from the wall
            return (ratio ** (r * nr) - 1.0) / (ratio ** nr - 1.0)

        def square(t):    # perimeter parameter t in [0, 4m) -> point, counter-clockwise
            t = np.asarray(t, float) % (4 * m)
            side = np.floor(t / m).astype(int)
            u = t / m - side
            px = np.select([side == 0, side == 1, side == 2, side == 3],
                           [H + 0 * u, H - 2 * H * u, -H + 0 * u, -H + 2 * H * u])
            py = np.select([side == 0, side == 1, side == 2, side == 3],
                           [-H + 2 * H * u, H + 0 * u, H - 2 * H * u, -H + 0 * u])
            return px, py

        def ring_map(t, r):
            sx, sy = square(t)
            ang = np.arctan2(sy, sx)
            cx, cy = R * np.cos(ang), R * np.sin(ang)
            f = frac(r)
            return xc + cx + f * (sx - cx), cy + f * (sy - cy)

        # vertices: perimeter index k (0..4m-1), ring index l (0..nr); l = nr on the hole
        def hole_vid(k):
            sx, sy = square(k)
            i = hx0 + int(round((sx + H) / h))
            jj = hy0 + int(round((sy + H) / h))
            return vid_bg(i, jj)
        base = nvert
        inner = np.zeros((4 * m, nr), np.int64)
        newp = []
        for l in range(nr):
            for k in range(4 * m):
                px, py = ring_map(k, l / nr)
                newp.append((px, py))
                inner[k, l] = base + l * 4 * m + k
        pts.append(np.asarray(newp))
        nvert += nr * 4 * m

        def rv(k, l):
            k = k % (4 * m)
            return hole_vid(k) if l == nr else inner[k, l]
        for l in range(nr):
            for k in range(4 * m):
                # xi clockwise along the perimeter, eta outward (positive J)
                elems.append([rv(k + 1, l), rv(k, l), rv(k + 1, l + 1), rv(k, l + 1)])
                T_, Rr = np.meshgrid(k + 1 - a, (l + a) / nr, indexing="ij")
                gx, gy = ring_map(T_, Rr)
                nodes.append(np.stack([gx.T.ravel(), gy.T.ravel()], 1))
    xyz = np.concatenate(pts, 0)
    elem_vert = np.asarray(elems, np.int64)
    info = {"h": h, "m1": m1, "m2": m2, "x2": x2, "R1": R1, "R2": R2, "x_in": x_in,
            "x_out": x_out, "y_max": y_max}
    return xyz, elem_vert, np.asarray(nodes), info


def tandem_cylinders(s_gap: float, r_ratio: float, n_hex: int, n_span: int = 16,
                     q: int = 2) -> Mesh:
    """Spanwise extrusion of ``tandem_cylinders_2d`` over pi D1 with n_span
    periodic layers (about n_hex hexes in total); walls on the cylinders,
    characteristic far field at the inlet and the lateral boundaries,
    outflow at the outlet; observers 2 D1 above the upstream cylinder."""
    xyz2, ev2, nodes2, info = tandem_cylinders_2d(s_gap, r_ratio, max(16, n_hex // n_span), q)
    span = np.pi
    z = np.linspace(0.0, span, n_span + 1)
    nv2 = xyz2.shape[0]
    xyz = np.concatenate([np.concatenate([xyz2, np.full((nv2, 1), zz)], 1) for zz in z], 0)
    ne2 = ev2.shape[0]
    ev = np.concatenate([np.concatenate([ev2 + k * nv2, ev2 + (k + 1) * nv2], 1)
                         for k in range(n_span)], 0)
    a = np.linspace(0.0, 1.0, q + 1)
    nodes = []
    for k in range(n_span):
        zz = z[k] + (z[k + 1] - z[k]) * a                      # (q+1,)
        nz = np.repeat(zz, (q + 1) ** 2)                        # zeta slowest
        n3 = np.concatenate([np.tile(nodes2, (1, q + 1, 1)),
                             np.broadcast_to(nz[None, :, None], (ne2, (q + 1) ** 3, 1))], 2)
        nodes.append(n3)
    geo = np.concatenate(nodes, 0)

    x_in, x_out, y_max = info["x_in"], info["x_out"], info["y_max"]

    def classify(c, f):
        if f in (4, 5):
            return TAG_PERIODIC
        if abs(c[0] - x_out) < 1e-9:
            return TAG_OUTFLOW
        if abs(c[0] - x_in) < 1e-9 or abs(abs(c[1]) - y_max) < 1e-9:
            return TAG_FARFIELD
        return TAG_WALL

    tags = _tag_unmatched(ev, xyz, 3, classify)
    probes = np.array([[0.0, 2.0, (kk + 0.5) * span / n_span] for kk in range(n_span)])
    # wall sampling for wall-damped starts
    th = np.linspace(0, 2 * np.pi, 400, endpoint=False)
    ring = lambda xc, R: np.stack([xc + R * np.cos(th), R * np.sin(th)], 1)
    w2 = np.concatenate([ring(0.0, info["R1"]), ring(info["x2"], info["R2"])], 0)
    wall = np.concatenate([np.concatenate([w2, np.full((len(w2), 1), zz)], 1)
                           for zz in np.linspace(0, span, 33)], 0)
    info.update({"kind": "tandem", "s": s_gap, "r": r_ratio, "probes": probes,
                 "wall_points": wall})
    return Mesh(dim=3, xyz=xyz, elem_vert=ev, face_tag=tags,
                periodic_shift=np.array([[0.0, 0.0, span]]), geo_order=q, geo_nodes=geo,
                info=info)


def tandem_batch(n_inst: int = 16, seed: int = 2312, h_lo: int = 60000, h_hi: int = 150000,
                 n_span: int = 16, q: int = 2):
    """One poll of tandem-cylinder candidates: gap s/D1 ~ U[2, 5], diameter
    ratio D2/D1 ~ U[0.5, 1.5], hex count ~ U[h_lo, h_hi]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_inst):
        s = rng.uniform(2.0, 5.0)
        r = rng.uniform(0.5, 1.5)
        nh = int(rng.uniform(h_lo, h_hi))
        out.append(tandem_cylinders(s, r, nh, n_span, q))
    return out


# ---------------------------------------------------------------------------
# element relabelling and per-element degree (input bookkeeping only)
# ---------------------------------------------------------------------------

def _rotations(dim):
    """Signed permutation matrices with determinant +1 (the rotations of the
    reference square / cube): 4 in 2-D, 24 in 3-D."""
    import itertools
    out = []
    for perm in itertools.permutations(range(dim)):
        for signs in itertools.product((1, -1), repeat=dim):
            R = np.zeros((dim, dim), dtype=np.int64)
            for r, (c, sg) in enumerate(zip(perm, signs)):
                R[r, c] = sg
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return out


def reorient(mesh: Mesh, seed: int = 2312) -> Mesh:
    """The same mesh with every element's local frame replaced by a seeded
    random rotation of its reference element: the corner list and the face
    tags are relabelled, the physical element is unchanged, so neighbouring
    faces meet in every relative orientation.  Straight-sided (q = 1) meshes
    only."""
    if mesh.geo_nodes is not None:
        raise ValueError("reorient: straight-sided meshes only")
    dim = mesh.dim
    rots = _rotations(dim)
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(rots), size=mesh.n_elem)
    corner_pos = np.array([[2 * ((c >> a) & 1) - 1 for a in range(dim)] for c in range(1 << dim)])

    def corner_index(y):
        return int(sum(((int(y[a]) + 1) // 2) << a for a in range(dim)))

    def face_index(normal):
        k = int(np.nonzero(normal)[0][0])
        return 2 * k + (1 if normal[k] > 0 else 0)

    ev = np.empty_like(mesh.elem_vert)
    ft = np.empty_like(mesh.face_tag)
    for e in range(mesh.n_elem):
        R = rots[pick[e]]
        for c in range(1 << dim):
            ev[e, c] = mesh.elem_vert[e, corner_index(R.T @ corner_pos[c])]
        for f in range(2 * dim):
            nrm = np.zeros(dim, dtype=np.int64)
            nrm[f // 2] = 1 if f % 2 else -1
            ft[e, f] = mesh.face_tag[e, face_index(R.T @ nrm)]
    return Mesh(mesh.dim, mesh.xyz, ev, ft, mesh.periodic_shift, 1, None, dict(mesh.info))


def element_centroids(mesh: Mesh) -> np.ndarray:
    return mesh.node_coords().mean(axis=1)


def checker_degrees(mesh: Mesh, degrees=(2, 3), seed: int | None = None) -> np.ndarray:
    """Per-element degree: a seeded random choice among ``degrees`` (or, with
    seed None, alternating along the element numbering), so that most faces
    join elements of different degree."""
    if seed is None:
        return np.asarray(degrees, dtype=np.int32)[np.arange(mesh.n_elem) % len(degrees)]
    rng = np.random.default_rng(seed)
    return np.asarray(degrees, dtype=np.int32)[rng.integers(0, len(degrees), size=mesh.n_elem)]


def sponge_degrees(mesh: Mesh, centre, radii, degrees) -> np.ndarray:
    """Per-element degree by distance of the element centroid from
    ``centre``: degrees[0] inside radii[0], degrees[i] between radii[i-1]
    and radii[i], the last degree beyond (the lower-degree far-field
    sponge layers of the paper's airfoil grids, Sec. 5.1)."""
    r = np.linalg.norm(element_centroids(mesh)[:, :len(centre)] - np.asarray(centre, float), axis=1)
    out = np.full(mesh.n_elem, degrees[-1], dtype=np.int32)
    for rad, deg in reversed(list(zip(radii, degrees))):
        out[r < rad] = deg
    return out
