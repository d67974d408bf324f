"""Seeded synthetic multipatch problems (input generation only).

This module builds the *inputs* of the method: patch layouts, glued control nets,
per-patch reluctivities, subdomain partitions of the patch dual graph and source
parameters. It holds none of the method's arithmetic (no basis functions, no
quadrature, no gauge, no solver) and is the only module shared by the CUDA path
and by the oracle.

Problem shape (Sec. 2, patches / patch-facets / subdomains):
  * a structured block grid of P0 x P1 x P2 patches, each the image of (0,1)^3
    under a B-spline/NURBS map of degree p with an open uniform knot vector;
    patch slab ``a`` in direction d has ``nspan[d][a]`` knot spans, so
    neighbouring patches share full facets (conforming patch interfaces);
  * consecutive patches share the control points of their common facet, so the
    whole domain has one glued control net with N_d = sum_a (n_a + p - 1) + 1
    points in direction d (N_0 = sum_a (n_a + p - 1) when direction 0 is periodic);
  * the control net is stored as ``ctrl[k, j, i, :] = (x, y, z, w)``;
  * patch (a, b, c) has flat index a + P0 * (b + P1 * c);
  * ``sub_of_patch`` groups patches into connected subdomains (Sec. 2).

Source kinds (right-hand side j of Eq. (3), one column per load case):
  * SOURCE_SINE: J = s * 2 pi^2 (sin(pi y) sin(pi z), sin(pi x) sin(pi z),
    sin(pi x) sin(pi y)), params = the amplitudes s, one per load case. With
    nu = 1 this is curl curl A for A = J / (2 pi^2), which has n x A = 0 on the
    unit cube's boundary.
  * SOURCE_FOURIER: J = sum_m Re(c_m exp(2 pi i k_m . x)); params per load case:
    nmodes, then for each mode k (3 values) and Re c (3), Im c (3).
  * SOURCE_PATCHWISE: J constant on each patch; params = nrhs x npatch x 3.
  * SOURCE_TRIG: J = s * 3 A_ana with A_ana = (cos y cos z sin x,
    -2 cos x cos z sin y, cos x cos y sin z), params = the amplitudes s. With
    nu = 1, s A_ana solves the strong problem with the tangential boundary data
    n x (s A_ana), which is not zero: this kind goes with the non-homogeneous
    Dirichlet data of the same field.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

SOURCE_SINE = 0
SOURCE_FOURIER = 1
SOURCE_PATCHWISE = 2
SOURCE_TRIG = 3


@dataclasses.dataclass
class Problem:
    name: str
    p: int
    npatch: Tuple[int, int, int]
    nspan: List[List[int]]
    periodic0: bool
    ctrl: np.ndarray            # (N2, N1, N0, 4) float64
    nu: np.ndarray              # (npatch_total,) float64
    sub_of_patch: np.ndarray    # (npatch_total,) int32
    source_kind: int
    source_params: np.ndarray   # float64, layout per kind (module docstring)
    nrhs: int
    affine: bool = False        # every patch map is an axis-aligned affine map (a box)

    @property
    def npatch_total(self) -> int:
        return int(self.npatch[0] * self.npatch[1] * self.npatch[2])

    @property
    def nsub(self) -> int:
        return int(self.sub_of_patch.max()) + 1

    def grid_shape(self) -> Tuple[int, int, int]:
        """Control points per direction of the glued net (N0, N1, N2)."""
        out = []
        for d in range(3):
            n = sum(s + self.p - 1 for s in self.nspan[d])
            if not (d == 0 and self.periodic0):
                n += 1
            out.append(n)
        return tuple(out)

    def with_params(self, nu=None, source_params=None, nrhs=None) -> "Problem":
        return dataclasses.replace(
            self,
            nu=self.nu if nu is None else np.asarray(nu, np.float64),
            source_params=self.source_params if source_params is None
            else np.asarray(source_params, np.float64),
            nrhs=self.nrhs if nrhs is None else int(nrhs))


# ----------------------------------------------------------------------------
# geometry helpers (control nets)
# ----------------------------------------------------------------------------

def _greville_1d(p: int, nspan: int) -> np.ndarray:
    """Greville abscissae of the open uniform knot vector of degree p with
    ``nspan`` spans on [0, 1]; control points placed there give the identity map."""
    inner = [i / nspan for i in range(1, nspan)]
    t = [0.0] * (p + 1) + inner + [1.0] * (p + 1)
    n = nspan + p
    return np.array([sum(t[i + 1:i + p + 1]) / p for i in range(n)])


def _glued_coords_1d(p: int, spans: Sequence[int], breaks: Sequence[float]) -> np.ndarray:
    pts = []
    for a, s in enumerate(spans):
        g = breaks[a] + (breaks[a + 1] - breaks[a]) * _greville_1d(p, s)
        pts.extend(g if a == 0 else g[1:])
    return np.array(pts)


def box_control_net(p: int, nspan: List[List[int]], breaks: List[Sequence[float]]) -> np.ndarray:
    """Affine box patches: tensor product of 1D Greville coordinates, weights 1."""
    xs = [_glued_coords_1d(p, nspan[d], breaks[d]) for d in range(3)]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return np.stack([x, y, z, np.ones_like(x)], axis=-1)


def exact_arc_1d(p: int, nspan: int, th0: float, dth: float):
    """Control points (m x 2) and weights (m) of the circular arc of angle ``dth``
    starting at angle ``th0`` on the unit circle, in the degree-p spline space
    with ``nspan`` uniform spans (m = nspan + p).

    The arc is the rational quadratic Bezier curve with end points on the circle
    and middle weight cos(dth / 2); its homogeneous coordinates (w x, w y, w)
    are quadratic polynomials of the parameter, so for p >= 2 they lie in the
    spline space and interpolation at the Greville abscissae reproduces them
    exactly (degree elevation and knot insertion without changing the curve)."""
    from scipy.interpolate import BSpline

    if p < 2:
        raise ValueError("an exact circular arc needs degree p >= 2")
    h = 0.5 * dth
    P = np.array([[math.cos(th0), math.sin(th0)],
                  [math.cos(th0 + h) / math.cos(h), math.sin(th0 + h) / math.cos(h)],
                  [math.cos(th0 + dth), math.sin(th0 + dth)]])
    w = np.array([1.0, math.cos(h), 1.0])
    g = _greville_1d(p, nspan)
    bern = np.stack([(1 - g) ** 2, 2 * g * (1 - g), g * g], axis=1)        # (m, 3)
    H = np.concatenate([bern @ (w[:, None] * P), (bern @ w)[:, None]], 1)  # homogeneous
    t = np.array([0.0] * (p + 1) + [i / nspan for i in range(1, nspan)] + [1.0] * (p + 1))
    A = BSpline.design_matrix(np.clip(g, 0.0, 1.0 - 1e-15), t, p).toarray()
    A[-1] = 0.0
    A[-1, -1] = 1.0                                                         # x = 1 is the last coefficient
    C = np.linalg.solve(A, H)
    C[0] = H[0]
    C[-1] = H[-1]
    return C[:, :2] / C[:, 2:3], C[:, 2].copy()


def annulus_control_net(p: int, nspan: List[List[int]], r_breaks: Sequence[float], z_breaks: Sequence[float],
                        arc: float, th0: float = 0.0, closed: bool = False) -> np.ndarray:
    """Control net of a thick cylindrical shell (or a sector of it): direction 0 is
    the angle (each angular patch an exact arc of ``arc / P0``, glued C^0; with
    ``closed`` the ring wraps around and direction 0 is periodic), direction 1 the
    radius (linear between the ``r_breaks``), direction 2 the axis (linear between
    the ``z_breaks``). Control point (i, j, k) is r_j (q_i, 0) + z_k e_z with
    weight w_i, where (q_i, w_i) are the angular control points: the map is
    x = r(xi_1) c(xi_0) + z(xi_2) e_z with c the exact circular arc."""
    P0 = len(nspan[0])
    dth = arc / P0
    qs, ws = [], []
    for a, s in enumerate(nspan[0]):
        q, w = exact_arc_1d(p, s, th0 + a * dth, dth)
        last = a == P0 - 1
        keep = slice(0 if a == 0 else 1, -1 if (closed and last) else None)
        qs.append(q[keep])
        ws.append(w[keep])
    q = np.concatenate(qs)
    w = np.concatenate(ws)
    r = _glued_coords_1d(p, nspan[1], r_breaks)
    z = _glued_coords_1d(p, nspan[2], z_breaks)
    ctrl = np.zeros((len(z), len(r), len(q), 4))
    ctrl[..., 0] = r[None, :, None] * q[None, None, :, 0]
    ctrl[..., 1] = r[None, :, None] * q[None, None, :, 1]
    ctrl[..., 2] = z[:, None, None]
    ctrl[..., 3] = w[None, None, :]
    return ctrl


# ----------------------------------------------------------------------------
# partitions of the patch dual graph
# ----------------------------------------------------------------------------

def block_partition(npatch: Tuple[int, int, int], block: Tuple[int, int, int]) -> np.ndarray:
    """Subdomains = aligned blocks of patches (recursive coordinate bisection of a
    power-of-two patch grid gives exactly these blocks)."""
    P0, P1, P2 = npatch
    B0, B1, B2 = block
    n0, n1 = P0 // B0, P1 // B1
    sub = np.empty(P0 * P1 * P2, np.int32)
    for c in range(P2):
        for b in range(P1):
            for a in range(P0):
                sub[a + P0 * (b + P1 * c)] = (a // B0) + n0 * ((b // B1) + n1 * (c // B2))
    return sub


def _patch_neighbours(npatch, q):
    P0, P1, P2 = npatch
    a, r = q % P0, q // P0
    b, c = r % P1, r // P1
    out = []
    for d, (x, lim) in enumerate(((a, P0), (b, P1), (c, P2))):
        for s in (-1, 1):
            y = x + s
            if 0 <= y < lim:
                abc = [a, b, c]
                abc[d] = y
                out.append(abc[0] + P0 * (abc[1] + P1 * abc[2]))
    return out


def _euler_char_of_patch_union(npatch, members) -> int:
    """Euler characteristic V - E + F - C of the union of closed unit cubes
    (patches) in the patch block grid; 1 for a contractible union."""
    P0, P1, P2 = npatch
    cubes = set()
    for q in members:
        a, r = q % P0, q // P0
        cubes.add((a, r % P1, r // P1))
    verts, edges, faces = set(), set(), set()
    for (a, b, c) in cubes:
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    verts.add((a + dx, b + dy, c + dz))
        for d in range(3):
            for o1 in (0, 1):
                for o2 in (0, 1):
                    base = [a, b, c]
                    others = [e for e in range(3) if e != d]
                    base[others[0]] += o1
                    base[others[1]] += o2
                    edges.add((d, tuple(base)))
            for o in (0, 1):
                base = [a, b, c]
                base[d] += o
                faces.add((d, tuple(base)))
    return len(verts) - len(edges) + len(faces) - len(cubes)


def _complement_connected(npatch, members) -> bool:
    """True if the patches NOT in ``members`` plus the outside form a connected
    set (no enclosed cavity)."""
    P0, P1, P2 = npatch
    mem = set(members)
    # pad the grid by one layer representing the outside
    seen = set()
    start = (-1, -1, -1)
    stack = [start]
    seen.add(start)
    while stack:
        a, b, c = stack.pop()
        for d in range(3):
            for s in (-1, 1):
                n = [a, b, c]
                n[d] += s
                if not (-1 <= n[0] <= P0 and -1 <= n[1] <= P1 and -1 <= n[2] <= P2):
                    continue
                t = tuple(n)
                if t in seen:
                    continue
                inside = 0 <= t[0] < P0 and 0 <= t[1] < P1 and 0 <= t[2] < P2
                if inside and (t[0] + P0 * (t[1] + P1 * t[2])) in mem:
                    continue
                seen.add(t)
                stack.append(t)
    n_out = sum(1 for t in seen if 0 <= t[0] < P0 and 0 <= t[1] < P1 and 0 <= t[2] < P2)
    return n_out == P0 * P1 * P2 - len(mem)


def is_simply_connected_union(npatch, members) -> bool:
    """Connected, Euler characteristic 1 and connected complement (no cavity):
    for unions of grid cubes this characterises a contractible set."""
    members = list(members)
    if not members:
        return False
    mem = set(members)
    seen = {members[0]}
    stack = [members[0]]
    while stack:
        q = stack.pop()
        for n in _patch_neighbours(npatch, q):
            if n in mem and n not in seen:
                seen.add(n)
                stack.append(n)
    if len(seen) != len(mem):
        return False
    return _euler_char_of_patch_union(npatch, members) == 1 and _complement_connected(npatch, members)


def greedy_partition(npatch, sizes_lo: int, sizes_hi: int, nsub: int, seed: int,
                     moves: int = 600) -> np.ndarray:
    """Uneven partition of the patch grid into ``nsub`` simply connected
    subdomains with sizes in [sizes_lo, sizes_hi]: start from the aligned block
    partition into nsub equal blocks and apply seeded boundary moves (a patch
    joins the subdomain of a face neighbour); a move is kept only if both
    subdomains stay within the size bounds and simply connected."""
    total = int(np.prod(npatch))
    per = total // nsub
    side = round(per ** (1.0 / 3.0))
    if side ** 3 * nsub != total or any(n % side for n in npatch):
        raise ValueError("the start partition needs nsub equal cubic blocks")
    sub = block_partition(tuple(npatch), (side, side, side))
    size = np.bincount(sub, minlength=nsub)
    rng = np.random.default_rng(seed)
    done, attempts = 0, 0
    while done < moves and attempts < 50 * moves:
        attempts += 1
        q = int(rng.integers(total))
        nbrs = [n for n in _patch_neighbours(npatch, q) if sub[n] != sub[q]]
        if not nbrs:
            continue
        src, dst = int(sub[q]), int(sub[nbrs[int(rng.integers(len(nbrs)))]])
        if size[src] - 1 < sizes_lo or size[dst] + 1 > sizes_hi:
            continue
        sub[q] = dst
        if (is_simply_connected_union(npatch, np.flatnonzero(sub == src))
                and is_simply_connected_union(npatch, np.flatnonzero(sub == dst))):
            size[src] -= 1
            size[dst] += 1
            done += 1
        else:
            sub[q] = src
    return sub


# ----------------------------------------------------------------------------
# sources
# ----------------------------------------------------------------------------

def fourier_source_params(nrhs: int, kmax: int, seed: int, nmodes: int | None = None) -> np.ndarray:
    """Random divergence-free Fourier sources: modes 0 < |k|_inf <= kmax (half of
    the +-k pairs, since the real part is taken), complex N(0,1) coefficients with
    the Leray projection c <- c - (k.c) k / |k|^2 applied."""
    rng = np.random.default_rng(seed)
    ks = []
    for kz in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kx in range(-kmax, kmax + 1):
                k = (kx, ky, kz)
                if k == (0, 0, 0):
                    continue
                # keep one of each +-k pair
                if k > tuple(-v for v in k):
                    ks.append(k)
    ks = np.array(ks, np.float64)
    out = []
    for _ in range(nrhs):
        sel = ks if nmodes is None else ks[rng.choice(len(ks), nmodes, replace=False)]
        col = [float(len(sel))]
        for k in sel:
            c = rng.standard_normal(3) + 1j * rng.standard_normal(3)
            c = c - (k @ c) * k / (k @ k)
            col.extend(list(k) + list(c.real) + list(c.imag))
        out.append(np.array(col))
    return np.concatenate(out)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def unit_cube(p: int, patches: Tuple[int, int, int], spans, sub_of_patch=None, nu=None,
              name="cube", source_kind=SOURCE_SINE, source_params=None, nrhs=1) -> Problem:
    """Unit cube split into a block grid of affine patches."""
    if isinstance(spans, int):
        spans = [[spans] * patches[d] for d in range(3)]
    breaks = [np.linspace(0.0, 1.0, patches[d] + 1) for d in range(3)]
    ctrl = box_control_net(p, spans, breaks)
    npt = int(np.prod(patches))
    if sub_of_patch is None:
        sub_of_patch = np.arange(npt, dtype=np.int32)
    if nu is None:
        nu = np.ones(npt)
    if source_params is None:
        source_params = np.arange(1, nrhs + 1, dtype=np.float64)
    return Problem(name=name, p=p, npatch=tuple(patches), nspan=[list(s) for s in spans],
                   periodic0=False, ctrl=ctrl, nu=np.asarray(nu, np.float64),
                   sub_of_patch=np.asarray(sub_of_patch, np.int32), source_kind=source_kind,
                   source_params=np.asarray(source_params, np.float64), nrhs=nrhs, affine=True)


def cube8_p2n4(spans: int = 4, p: int = 2) -> Problem:
    """Unit cube, 2x2x2 patches, one patch per subdomain, p=2, 4 spans per
    direction per patch, nu=1, manufactured sine source."""
    return unit_cube(p, (2, 2, 2), spans, name=f"cube8_p{p}n{spans}")


def cube64_p3n8_sub16(seed: int = 2, spans: int = 8, p: int = 3, nrhs: int = 1) -> Problem:
    """Unit cube, 4x4x4 patches in 16 subdomains of 2x2x1 patches, p=3, 8 spans,
    per-patch nu log-uniform in [1, 1e3] (seeded), sine source."""
    rng = np.random.default_rng(seed)
    nu = 10.0 ** rng.uniform(0.0, 3.0, size=64)
    sub = block_partition((4, 4, 4), (2, 2, 1))
    return unit_cube(p, (4, 4, 4), spans, sub_of_patch=sub, nu=nu,
                     name=f"cube64_p{p}n{spans}_sub16", nrhs=nrhs,
                     source_params=np.arange(1, nrhs + 1, dtype=np.float64))


def cube512_p3_uneven64(seed: int = 3, nrhs: int = 32, span_lo: int = 4, span_hi: int = 12) -> Problem:
    """Unit cube, 8x8x8 patches, spans per patch slab drawn from {4..12}, p=3,
    64 uneven simply connected subdomains of 4-12 patches, divergence-free random
    Fourier sources (|k|_inf <= 4), nu = 1."""
    rng = np.random.default_rng(seed)
    spans = [list(rng.integers(span_lo, span_hi + 1, size=8)) for _ in range(3)]
    sub = greedy_partition((8, 8, 8), 4, 12, 64, seed)
    sp = fourier_source_params(nrhs, 4, seed)
    return unit_cube(3, (8, 8, 8), spans, sub_of_patch=sub, nu=np.ones(512),
                     name="cube512_p3_uneven64", source_kind=SOURCE_FOURIER,
                     source_params=sp, nrhs=nrhs)


def cube64_uneven8(seed: int = 3, nrhs: int = 32, span_lo: int = 2, span_hi: int = 4) -> Problem:
    """The reduced uneven case of cube512_p3_uneven64: 4x4x4 patches, spans per
    patch slab drawn from {2..4}, p=3, 8 uneven simply connected subdomains of
    4-12 patches, 32 divergence-free random Fourier sources (6 modes each of
    |k|_inf <= 2), nu = 1; small enough for the oracle."""
    rng = np.random.default_rng(seed)
    spans = [list(rng.integers(span_lo, span_hi + 1, size=4)) for _ in range(3)]
    sub = greedy_partition((4, 4, 4), 4, 12, 8, seed)
    sp = fourier_source_params(nrhs, 2, seed, nmodes=6)
    return unit_cube(3, (4, 4, 4), spans, sub_of_patch=sub, nu=np.ones(64),
                     name="cube64_uneven8", source_kind=SOURCE_FOURIER, source_params=sp, nrhs=nrhs)


def annulus(p: int, patches: Tuple[int, int, int], spans, r_in: float, r_out: float, length: float,
            arc: float = 2 * math.pi, sub_of_patch=None, nu=None, name="annulus",
            source_kind=SOURCE_PATCHWISE, source_params=None, nrhs=1) -> Problem:
    """Thick cylindrical shell r_in < r < r_out, 0 < z < length, split into
    P0 angular x P1 radial x P2 axial NURBS patches with exact circular arcs.
    ``arc`` = 2 pi closes the ring (direction 0 periodic, P0 >= 3); a smaller
    ``arc`` gives the sector 0 < theta < arc."""
    if isinstance(spans, int):
        spans = [[spans] * patches[d] for d in range(3)]
    closed = abs(arc - 2 * math.pi) < 1e-12
    ctrl = annulus_control_net(p, spans, np.linspace(r_in, r_out, patches[1] + 1),
                               np.linspace(0.0, length, patches[2] + 1), arc, closed=closed)
    npt = int(np.prod(patches))
    if sub_of_patch is None:
        sub_of_patch = np.arange(npt, dtype=np.int32)
    if nu is None:
        nu = np.ones(npt)
    if source_params is None:
        source_params = np.zeros(nrhs * npt * 3)
    return Problem(name=name, p=p, npatch=tuple(patches), nspan=[list(s) for s in spans],
                   periodic0=closed, ctrl=ctrl, nu=np.asarray(nu, np.float64),
                   sub_of_patch=np.asarray(sub_of_patch, np.int32), source_kind=source_kind,
                   source_params=np.asarray(source_params, np.float64), nrhs=nrhs)


NU0 = 1.0 / (4e-7 * math.pi)


def machine_annulus(n_ang: int = 36, n_ax: int = 4, spans: int = 6, p: int = 3, nrhs: int = 16, seed: int = 5,
                    per_sub: int = 3, r_in: float = 0.05, r_out: float = 0.10, length: float = 0.10) -> Problem:
    """Machine-like ring: n_ang angular x 2 radial x n_ax axial NURBS patches
    (exact arcs of 360/n_ang degrees), inner ring air nu0 = 1/(4 pi 1e-7), outer
    ring iron nu0/1000; axial current density in every third angular sector of
    the inner ring over the whole length (slot s = a // 3 of sector a), load
    case c: J_z = 1e6 (-1)^s cos(theta_c - 2 pi (s mod 3) / 3) with theta_c
    drawn uniformly in [0, 2 pi) (seeded). Subdomains: runs of ``per_sub``
    angular patches of one radial and one axial slab."""
    P = (n_ang, 2, n_ax)
    npt = int(np.prod(P))
    nu = np.empty(npt)
    sub = np.empty(npt, np.int32)
    nga = n_ang // per_sub
    for c in range(n_ax):
        for b in range(2):
            for a in range(n_ang):
                q = a + n_ang * (b + 2 * c)
                nu[q] = NU0 if b == 0 else NU0 / 1000.0
                sub[q] = a // per_sub + nga * (b + 2 * c)
    rng = np.random.default_rng(seed)
    theta = rng.uniform(0.0, 2 * math.pi, size=nrhs)
    J = np.zeros((nrhs, npt, 3))
    for r in range(nrhs):
        for c in range(n_ax):
            for a in range(0, n_ang, 3):
                s = a // 3
                J[r, a + n_ang * (0 + 2 * c), 2] = 1e6 * (-1) ** s * math.cos(theta[r] - 2 * math.pi * (s % 3) / 3)
    return annulus(p, P, spans, r_in, r_out, length, sub_of_patch=sub, nu=nu,
                   name=f"annulus{npt}_p{p}n{spans}_sub{int(sub.max()) + 1}",
                   source_kind=SOURCE_PATCHWISE, source_params=J.ravel(), nrhs=nrhs)


def snake_order(npatch) -> List[int]:
    """Patches of the grid in boustrophedon order: direction 0 fastest, its
    sense reversed on every other row, the rows' sense reversed on every other
    layer, so that consecutive patches always share a facet."""
    P0, P1, P2 = npatch
    out = []
    for c in range(P2):
        rows = range(P1) if c % 2 == 0 else range(P1 - 1, -1, -1)
        for n, b in enumerate(rows):
            fwd = (n + c * P1) % 2 == 0
            cols = range(P0) if fwd else range(P0 - 1, -1, -1)
            out.extend(a + P0 * (b + P1 * c) for a in cols)
    return out


def snake_partition(npatch, nsub: int) -> np.ndarray:
    """nsub subdomains of consecutive patches in snake order with sizes that
    differ by at most one; every subdomain is checked to be simply connected
    (ValueError otherwise)."""
    order = snake_order(npatch)
    total = len(order)
    if not 1 <= nsub <= total:
        raise ValueError("nsub out of range")
    sub = np.empty(total, np.int32)
    bounds = [round(i * total / nsub) for i in range(nsub + 1)]
    for k in range(nsub):
        for q in order[bounds[k]:bounds[k + 1]]:
            sub[q] = k
    for k in range(nsub):
        if not is_simply_connected_union(npatch, np.flatnonzero(sub == k)):
            raise ValueError(f"snake subdomain {k} of {nsub} is not simply connected")
    return sub


def three_columns_partition() -> np.ndarray:
    """Three subdomains of nine patches on the 3 x 3 x 3 grid: the slab a = 0
    and two L-shaped columns, {(1,0), (2,0), (2,1)} and {(1,1), (1,2), (2,2)} in
    (a, b) over all c. The three meet along one interior line of patch edges
    (x = 1, y = 1), whose edges are the cross-edges of the layout."""
    sub = np.empty(27, np.int32)
    col1 = {(1, 0), (2, 0), (2, 1)}
    for c in range(3):
        for b in range(3):
            for a in range(3):
                sub[a + 3 * (b + 3 * c)] = 0 if a == 0 else (1 if (a, b) in col1 else 2)
    return sub


def paper_cube(p: int, spans: int, nsub: int = 3, nrhs: int = 1, amps=None, layout: str = "columns") -> Problem:
    """The cube (0,3)^3 of 3 x 3 x 3 unit patches of Sec. 3 (Fig. of the
    decomposition) with the manufactured field A_ana (SOURCE_TRIG, nu = 1):
    ``spans`` knot spans per patch and direction (mesh size h = 1 / spans).
    Subdomains: with layout "columns" and nsub = 3 the three columns of
    three_columns_partition; otherwise (layout "snake") ``nsub`` subdomains of
    consecutive patches in snake order (nsub = 3 gives three slabs)."""
    breaks = [np.linspace(0.0, 3.0, 4)] * 3
    sp_ = [[spans] * 3 for _ in range(3)]
    ctrl = box_control_net(p, sp_, breaks)
    if amps is None:
        amps = np.ones(nrhs)
    if layout not in ("columns", "snake"):
        raise ValueError("layout is 'columns' or 'snake'")
    cols = layout == "columns" and nsub == 3
    sub = three_columns_partition() if cols else snake_partition((3, 3, 3), nsub)
    return Problem(name=f"paper_cube_p{p}n{spans}_{'columns' if cols else 'snake'}{nsub}", p=p, npatch=(3, 3, 3),
                   nspan=sp_, periodic0=False, ctrl=ctrl, nu=np.ones(27),
                   sub_of_patch=sub, source_kind=SOURCE_TRIG,
                   source_params=np.asarray(amps, np.float64), nrhs=nrhs, affine=True)


def small_cases():
    """Tiny problems for the parity tests (several tiles, ragged sizes)."""
    out = []
    out.append(cube8_p2n4(spans=2))
    out.append(unit_cube(1, (2, 2, 2), 2, name="cube8_p1n2"))
    out.append(unit_cube(3, (2, 2, 1), 2, name="cube4_p3n2"))
    rng = np.random.default_rng(7)
    out.append(unit_cube(2, (3, 2, 2), [[2, 3, 2], [2, 2], [3, 2]],
                         sub_of_patch=np.array([0, 0, 1, 2, 2, 1, 3, 3, 4, 5, 5, 4], np.int32),
                         nu=10.0 ** rng.uniform(0, 3, 12), name="cube12_p2_mixed"))
    return out


# ----------------------------------------------------------------------------
# parameter family for the learned warm start
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class WarmstartFamily:
    """Instances of one mesh that differ in the per-patch reluctivity and in 16
    source coefficients: nu_q = 10^(3 u_q), u_q ~ U(0, 1) per patch, and
    J = sum_m (a_{2m} cos(2 pi k_m.x) - a_{2m+1} sin(2 pi k_m.x)) e_m with 8
    fixed modes k_m, fixed unit directions e_m orthogonal to k_m (so J is
    divergence free) and a ~ N(0, 1)^16. The network input of an instance is
    x = [log10 nu (npatch values), a (16 values)]."""
    base: Problem
    modes: np.ndarray        # (8, 3) integer wave vectors
    dirs: np.ndarray         # (8, 3) unit vectors, dirs[m] . modes[m] = 0
    log_nu: np.ndarray       # (n, npatch)
    coef: np.ndarray         # (n, 16)

    @property
    def n(self) -> int:
        return int(self.log_nu.shape[0])

    def inputs(self) -> np.ndarray:
        return np.concatenate([self.log_nu, self.coef], axis=1).astype(np.float32)

    def nu(self, i: int) -> np.ndarray:
        return 10.0 ** self.log_nu[i]

    def source_params(self, i: int) -> np.ndarray:
        """SOURCE_FOURIER parameters of instance i (one load case)."""
        return self.source_params_for(self.coef[i])

    def source_params_for(self, coef) -> np.ndarray:
        """SOURCE_FOURIER parameters of one load case with coefficients `coef` (16)."""
        col = [float(len(self.modes))]
        for m, (k, e) in enumerate(zip(self.modes, self.dirs)):
            col.extend(list(k) + list(coef[2 * m] * e) + list(coef[2 * m + 1] * e))
        return np.array(col)

    def basis_source_params(self) -> np.ndarray:
        """16 load cases, load case c with coefficient vector e_c: the solution of
        an instance with coefficients a is sum_c a_c times the solution of load
        case c (the source enters Eq. (3) linearly)."""
        return np.concatenate([self.source_params_for(np.eye(16)[c]) for c in range(16)])


def warmstart_family(n: int, seed: int, patches=(4, 4, 4), block=(2, 2, 2), spans: int = 2,
                     p: int = 2, kmax: int = 2) -> WarmstartFamily:
    """n seeded instances on the unit cube split into `patches` affine patches,
    grouped into equal subdomains of `block` patches."""
    rng = np.random.default_rng(seed)
    # modes and directions are fixed by a generator of their own so that every
    # seed shares them
    frng = np.random.default_rng(12345)
    modes, dirs = [], []
    while len(modes) < 8:
        k = frng.integers(-kmax, kmax + 1, size=3)
        if not k.any() or any((k == q).all() or (k == -q).all() for q in modes):
            continue
        e = frng.standard_normal(3)
        e = e - (e @ k) * k / (k @ k)
        modes.append(k)
        dirs.append(e / np.linalg.norm(e))
    npt = int(np.prod(patches))
    sub = block_partition(tuple(patches), tuple(block))
    fam = WarmstartFamily(base=None, modes=np.array(modes, np.float64), dirs=np.array(dirs),
                          log_nu=rng.uniform(0.0, 3.0, size=(n, npt)),
                          coef=rng.standard_normal((n, 16)))
    fam.base = unit_cube(p, tuple(patches), spans, sub_of_patch=sub, nu=fam.nu(0),
                         name=f"warmstart_{patches[0]}x{patches[1]}x{patches[2]}_p{p}n{spans}",
                         source_kind=SOURCE_FOURIER, source_params=fam.source_params(0), nrhs=1)
    return fam
