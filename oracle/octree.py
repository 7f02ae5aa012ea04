"""Octree (brick) grid and its operator: the FP64 oracle.

TEST INFRASTRUCTURE ONLY: called by the test suite (and nothing in the CUDA
library).  Plain numpy / scipy.sparse in FP64, written for small cases; the
per-node primitives (inside test, edge inside-fraction, Coulomb sums, units)
come from the uniform oracle ``pb_oracle.c``.

The paper's octree (Sec. 3, refined near the molecular surface, Sec. 3.4)
defers the treatment of hanging nodes to prior work, so this oracle takes the
following reading, which the GPU library implements independently:

* Domain: a cube of n0 coarse bricks per axis, brick side 8 h_bulk, centred
  on the bounding box of the atom spheres (side n0 * 8 * h_bulk with
  n0 = ceil(fill * extent / (8 h_bulk))), or an explicit origin and n0.
* Levels l = 0..Lmax, cell size h_l = h_bulk / 2^l, h_Lmax = h_fine.  All
  positions are integers in units of h_fine ("node units"); the world
  coordinate of node-unit position P is origin + P * h_fine.
* A brick is an 8^3-cell cube at one level; a level-l brick (l < Lmax) is
  split into 8 children when its closed box lies within refine_dist of some
  atom's sphere surface: dmin <= R + d and dmax >= R - d, with dmin / dmax
  the smallest / largest distance from the centre to the box (compared as
  squares, sums of squares as (x^2 + y^2) + z^2).
* 2:1 balance: leaves that share a face, an edge or a corner differ by at
  most one level; violating leaves are split until none is left.
* Leaves are ordered by the Morton code of their low corner (x bit lowest).
  Brick b owns its 8^3 low-corner nodes; slot = 512 b + (8 k + j) 8 + i.
* Node kinds: boundary (a coordinate is 0 or the domain side), hanging (a
  touching leaf does not have the node on its lattice: then its value is the
  mean of the 2 ends of the coarse edge, or of the 4 corners of the coarse
  face, it lies on), regular otherwise.
* Operator, element form on each leaf cell of size h: every one of the 12
  cell edges adds (eps_e h / 4) (d_a - d_b)(d_a - d_b)^T, with eps_e the
  interface-averaged coefficient of Eq. WHA of that edge; every corner v
  adds eps_s k_D^2 h^3 / 8 if v is in the solvent.  K is assembled over all
  corner positions (edge weight = (eps_e h) * (cells / 4), mass =
  sum_l kappa(h_l) * (cells_l / 8)), and A = P^T K P over the regular
  interior nodes, P the hanging-node interpolation.  On a single-level tree
  this is exactly the uniform operator (G^T W G + C).
* refine_dist must be at least the largest radius, h_fine and 1.5 h_bulk, so
  that every solute node, every edge meeting the surface and every charge
  cell lies in the all-finest region (where everything matches the uniform
  grid at h_fine), and every row next to a level change sees solvent only.
* De-refined domain (Sec. 3.4, "Exploiting de-refinement for more efficient
  BCs"): with h_tight set, h_bulk is the spacing of the coarse far field and
  a level-l brick is also split while its cells are coarser than h_tight and
  its closed box meets the tight box: a cube of side tight_fill * extent
  centred on the same bounding box (tight_fill about 1.1, a perfil near
  90 %).  The domain itself (fill) can then be several times the extent (a
  perfil of 15-20 %), where null Dirichlet values are accurate.  The
  refine_dist condition uses h_tight in place of h_bulk: cells coarser than
  h_tight lie outside the tight box, away from the molecule.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import oracle as U


def morton3(x, y, z) -> np.ndarray:
    x = np.asarray(x, dtype=np.int64)
    y = np.asarray(y, dtype=np.int64)
    z = np.asarray(z, dtype=np.int64)
    code = np.zeros(np.broadcast(x, y, z).shape, dtype=np.int64)
    for b in range(20):
        code |= ((x >> b) & 1) << (3 * b)
        code |= ((y >> b) & 1) << (3 * b + 1)
        code |= ((z >> b) & 1) << (3 * b + 2)
    return code


@dataclass
class Octree:
    origin: np.ndarray   # (3,)
    h_fine: float
    h_bulk: float
    Lmax: int
    n0: int              # coarse bricks per axis
    level_field: np.ndarray  # [x, y, z] over finest-brick cells, leaf level
    blevel: np.ndarray   # (nb,)
    blow: np.ndarray     # (nb, 3) low corner, node units

    @property
    def NL(self) -> int:
        """Domain side in node units."""
        return self.n0 * 8 * (1 << self.Lmax)

    @property
    def nb(self) -> int:
        return len(self.blevel)

    def spacing(self, level):
        return 1 << (self.Lmax - np.asarray(level))

    def slot_positions(self) -> np.ndarray:
        """(512 nb, 3) node-unit positions of every owned slot."""
        loc = np.arange(512)
        ijk = np.stack([loc % 8, (loc // 8) % 8, loc // 64], axis=1)
        s = self.spacing(self.blevel)[:, None, None]
        P = self.blow[:, None, :] + s * ijk[None, :, :]
        return P.reshape(-1, 3)

    def world(self, P) -> np.ndarray:
        return self.origin[None, :] + np.asarray(P, dtype=np.float64) * self.h_fine


# ----------------------------------------------------------------- build ---
def place(atoms: np.ndarray, h_bulk: float, fill: float):
    """Origin and coarse brick count of the automatically placed domain."""
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(axis=0)
    hi = (atoms[:, :3] + atoms[:, 3:4]).max(axis=0)
    extent = float((hi - lo).max())
    n0 = max(1, math.ceil(fill * extent / (8.0 * h_bulk)))
    side = n0 * 8.0 * h_bulk
    origin = 0.5 * (lo + hi) - 0.5 * side
    return origin, n0


def near_boxes(atoms: np.ndarray, origin, h_fine, low: np.ndarray, side: int,
               dist: float, chunk: int = 1 << 22) -> np.ndarray:
    """True for each box [low, low + side] (node units) that lies within
    `dist` of some atom's sphere surface."""
    a = origin[None, :] + low.astype(np.float64) * h_fine
    b = origin[None, :] + (low + side).astype(np.float64) * h_fine
    out = np.zeros(len(low), dtype=bool)
    per = max(1, chunk // max(1, len(atoms)))
    c = atoms[:, :3]
    R = atoms[:, 3]
    rin = (R + dist) * (R + dist)
    rout_ok = (R - dist) <= 0.0
    rout = (R - dist) * (R - dist)
    for s in range(0, len(low), per):
        A = a[s:s + per, None, :]
        B = b[s:s + per, None, :]
        t = np.maximum(np.maximum(A - c[None], 0.0), c[None] - B)
        dmin2 = (t[..., 0] * t[..., 0] + t[..., 1] * t[..., 1]) + t[..., 2] * t[..., 2]
        u = np.maximum(np.abs(c[None] - A), np.abs(c[None] - B))
        dmax2 = (u[..., 0] * u[..., 0] + u[..., 1] * u[..., 1]) + u[..., 2] * u[..., 2]
        ok = (dmin2 <= rin[None]) & (rout_ok[None] | (dmax2 >= rout[None]))
        out[s:s + per] = ok.any(axis=1)
    return out


def _box_max(field: np.ndarray, f: int) -> np.ndarray:
    """Max over f^3 blocks of a cubic field."""
    n = field.shape[0] // f
    return field.reshape(n, f, n, f, n, f).max(axis=(1, 3, 5))


def tight_box(atoms: np.ndarray, tight_fill: float):
    """Low and high corners of the tight box: a cube of side tight_fill *
    extent centred on the bounding box of the atom spheres."""
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(axis=0)
    hi = (atoms[:, :3] + atoms[:, 3:4]).max(axis=0)
    half = 0.5 * tight_fill * float((hi - lo).max())
    c = 0.5 * (lo + hi)
    return c - half, c + half


def build(atoms, h_fine: float, h_bulk: float, refine_dist: float, fill: float = 1.5,
          origin=None, n0: int | None = None, h_tight: float | None = None,
          tight_fill: float = 1.1) -> Octree:
    atoms = np.ascontiguousarray(atoms, dtype=np.float64)
    ratio = h_bulk / h_fine
    Lmax = int(round(math.log2(ratio)))
    if Lmax < 0 or h_fine * (1 << Lmax) != h_bulk:
        raise ValueError("h_bulk must be h_fine times a power of two")
    h_near = h_bulk
    if h_tight is not None:
        Lt = int(round(math.log2(h_bulk / h_tight)))
        if Lt < 0 or Lt > Lmax or h_tight * (1 << Lt) != h_bulk:
            raise ValueError("h_tight must be h_bulk over a power of two, at least h_fine")
        h_near = h_tight
    if refine_dist < max(float(atoms[:, 3].max()), h_fine, 1.5 * h_near):
        raise ValueError("refine_dist must be at least the largest radius, h_fine and 1.5 h_bulk "
                         "(h_tight on a de-refined domain)")
    if origin is None:
        origin, n0 = place(atoms, h_bulk, fill)
    origin = np.asarray(origin, dtype=np.float64)
    nf = n0 << Lmax                      # finest bricks per axis
    # leaf level of every finest-brick cell from the refinement test
    level = np.zeros((nf, nf, nf), dtype=np.int64)
    for l in range(Lmax):
        f = 1 << (Lmax - l)              # finest bricks per level-l brick
        nl = n0 << l
        g = np.stack(np.meshgrid(np.arange(nl), np.arange(nl), np.arange(nl), indexing="ij"), -1)
        low = g.reshape(-1, 3) * (8 * f)
        near = near_boxes(atoms, origin, h_fine, low, 8 * f, refine_dist)
        if h_tight is not None and l < Lt:
            # the brick's closed box meets the tight box
            tlo, thi = tight_box(atoms, tight_fill)
            a = origin[None, :] + low.astype(np.float64) * h_fine
            b = origin[None, :] + (low + 8 * f).astype(np.float64) * h_fine
            near = near | ((a <= thi[None, :]) & (b >= tlo[None, :])).all(axis=1)
        near = near.reshape(nl, nl, nl)
        up = np.repeat(np.repeat(np.repeat(near, f, 0), f, 1), f, 2)
        level[(level == l) & up] = l + 1
    # 2:1 balance over faces, edges and corners
    while True:
        pad = np.pad(level, 1, constant_values=-1)
        nbmax = np.full_like(level, -1)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    nbmax = np.maximum(nbmax, pad[1 + dx:1 + dx + nf, 1 + dy:1 + dy + nf,
                                                  1 + dz:1 + dz + nf])
        req = np.maximum(level, nbmax - 1)
        new = np.full_like(level, Lmax)
        for l in range(Lmax - 1, -1, -1):
            f = 1 << (Lmax - l)
            split = _box_max(req, f) > l
            keep = ~np.repeat(np.repeat(np.repeat(split, f, 0), f, 1), f, 2)
            new[keep] = l
        if np.array_equal(new, level):
            break
        level = new
    # leaves (one per low-corner cell), Morton order
    cx, cy, cz = np.meshgrid(np.arange(nf), np.arange(nf), np.arange(nf), indexing="ij")
    s = 1 << (Lmax - level)
    is_low = (cx % s == 0) & (cy % s == 0) & (cz % s == 0)
    lx, ly, lz = cx[is_low], cy[is_low], cz[is_low]
    order = np.argsort(morton3(lx, ly, lz), kind="stable")
    blow = np.stack([lx[order], ly[order], lz[order]], axis=1) * 8
    blevel = level[is_low][order]
    return Octree(origin, float(h_fine), float(h_bulk), Lmax, int(n0), level, blevel, blow)


# ------------------------------------------------------------- node kinds ---
def touching_spacings(tree: Octree, P: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """For node-unit positions P: (largest, smallest) lattice spacing among the
    leaves whose closed box contains P."""
    nf = tree.level_field.shape[0]
    smax = np.zeros(len(P), dtype=np.int64)
    smin = np.full(len(P), 1 << 40, dtype=np.int64)
    for off in np.ndindex(2, 2, 2):
        c = P // 8 - np.array(off)[None, :] * (P % 8 == 0)
        ok = np.all((c >= 0) & (c < nf), axis=1) & np.all((P // 8 - c <= 1) & (P // 8 - c >= 0), axis=1)
        cc = np.clip(c, 0, nf - 1)
        lv = tree.level_field[cc[:, 0], cc[:, 1], cc[:, 2]]
        sp_ = 1 << (tree.Lmax - lv)
        smax = np.where(ok, np.maximum(smax, sp_), smax)
        smin = np.where(ok, np.minimum(smin, sp_), smin)
    return smax, smin


def node_kind(tree: Octree, P: np.ndarray) -> np.ndarray:
    """0 regular interior, 1 boundary, 2 hanging."""
    NL = tree.NL
    bnd = np.any((P == 0) | (P == NL), axis=1)
    smax, _ = touching_spacings(tree, P)
    hang = np.any(P % smax[:, None] != 0, axis=1)
    return np.where(bnd, 1, np.where(hang, 2, 0)).astype(np.int8)


def hanging_parents(tree: Octree, P: np.ndarray):
    """Parents (k, 4, 3) and weights (k, 4) of hanging positions (2 or 4
    parents; unused entries have weight 0 and repeat the first parent)."""
    smax, _ = touching_spacings(tree, P)
    half = smax // 2
    odd = (P % smax[:, None]) != 0
    par = np.repeat(P[:, None, :], 4, axis=1).copy()
    w = np.zeros((len(P), 4))
    for r in range(len(P)):
        dims = np.nonzero(odd[r])[0]
        combos = list(np.ndindex(*([2] * len(dims))))
        for q, cmb in enumerate(combos):
            for d, sgn in zip(dims, cmb):
                par[r, q, d] = P[r, d] + (half[r] if sgn else -half[r])
            w[r, q] = 1.0 / len(combos)
    return par, w


# ---------------------------------------------------------- all positions ---
def corner_positions(tree: Octree):
    """Unique corner positions of all leaf cells (node units) and, per brick
    cell corner, the index into that list: (pos (m, 3), idx (nb, 9, 9, 9))."""
    g = np.arange(9)
    ijk = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)  # [i, j, k]
    s = tree.spacing(tree.blevel)[:, None, None]
    P = (tree.blow[:, None, :] + s * ijk[None]).reshape(-1, 3)
    NL1 = tree.NL + 1
    key = (P[:, 2] * NL1 + P[:, 1]) * NL1 + P[:, 0]
    ukey, inv = np.unique(key, return_inverse=True)
    pos = np.stack([ukey % NL1, (ukey // NL1) % NL1, ukey // (NL1 * NL1)], axis=1)
    return pos, inv.reshape(tree.nb, 9, 9, 9)


def _virtual_grid(tree: Octree, level: int) -> U.Grid:
    s = 1 << (tree.Lmax - level)
    n = tree.NL // s + 1
    return U.Grid((n, n, n), tree.origin, tree.h_fine * s)


def _inside(tree: Octree, atoms, pos) -> np.ndarray:
    g = _virtual_grid(tree, tree.Lmax)
    NL1 = tree.NL + 1
    ids = (pos[:, 2] * NL1 + pos[:, 1]) * NL1 + pos[:, 0]
    return U.classify_nodes(g, atoms, ids)


def operator(tree: Octree, atoms, eps_in: float, eps_out: float, kD: float) -> dict:
    """K over all corner positions, and the hanging-node interpolation."""
    atoms = np.ascontiguousarray(atoms, dtype=np.float64)
    pos, cidx = corner_positions(tree)
    m = len(pos)
    inside = _inside(tree, atoms, pos)
    NL1 = tree.NL + 1
    pkey = (pos[:, 2] * NL1 + pos[:, 1]) * NL1 + pos[:, 0]
    # edges of every leaf cell: (a, b, level, d), counted per distinct edge
    ea, eb, el, ed = [], [], [], []
    for d in range(3):
        sl_lo = [slice(0, 8)] * 3
        sl_lo[d] = slice(0, 8)
        for t1 in range(2):
            for t2 in range(2):
                # the 4 edges of a cell along d, indexed by the other two offsets
                o = [None, None, None]
                others = [x for x in range(3) if x != d]
                lo = [slice(0, 8)] * 3
                hi = [slice(0, 8)] * 3
                lo[others[0]] = slice(t1, t1 + 8)
                hi[others[0]] = slice(t1, t1 + 8)
                lo[others[1]] = slice(t2, t2 + 8)
                hi[others[1]] = slice(t2, t2 + 8)
                lo[d] = slice(0, 8)
                hi[d] = slice(1, 9)
                a = cidx[(slice(None),) + tuple(lo)].reshape(tree.nb, -1)
                b = cidx[(slice(None),) + tuple(hi)].reshape(tree.nb, -1)
                ea.append(a.reshape(-1))
                eb.append(b.reshape(-1))
                el.append(np.repeat(tree.blevel, 512))
                ed.append(np.full(a.size, d))
                del o
    ea, eb, el, ed = (np.concatenate(x) for x in (ea, eb, el, ed))
    # an edge is its low end, direction and level (a coarse and a fine edge
    # can start at the same node in the same direction)
    ekey = (ea.astype(np.int64) * 3 + ed) * (tree.Lmax + 1) + el
    uk, first, cnt = np.unique(ekey, return_index=True, return_counts=True)
    a, b, lev, d = ea[first], eb[first], el[first], ed[first]
    # eps_e h_l for each distinct edge: pure medium or Eq. WHA (listed edges)
    h = tree.h_fine * (1 << (tree.Lmax - lev)).astype(np.float64)
    epsh = np.where(inside[a] == 1, eps_in, eps_out) * h
    alpha = np.zeros(len(a))
    for lv in np.unique(lev):
        sel = np.nonzero(lev == lv)[0]
        g = _virtual_grid(tree, int(lv))
        s = 1 << (tree.Lmax - int(lv))
        Pa = pos[a[sel]] // s
        n = int(g.n[0])
        ids = d[sel].astype(np.int64) * (n ** 3) + (Pa[:, 2] * n + Pa[:, 1]) * n + Pa[:, 0]
        alpha[sel] = U.edge_alpha(g, atoms, ids)
    listed = ((alpha > 0.0) & (alpha < 1.0)) | (inside[a] != inside[b])
    wha = 1.0 / (alpha / eps_in + (1.0 - alpha) / eps_out)
    epsh = np.where(listed, wha * h, epsh)
    W = epsh * (cnt.astype(np.float64) / 4.0)
    # vertex masses: per level, number of level-l cells having the vertex
    mass = np.zeros(m)
    kap_s = {}
    for lv in np.unique(tree.blevel):
        hl = tree.h_fine * (1 << (tree.Lmax - int(lv)))
        kap_s[int(lv)] = eps_out * kD * kD * hl * hl * hl
    corners = []
    for ci in np.ndindex(2, 2, 2):
        sl = tuple(slice(c, c + 8) for c in ci)
        corners.append(cidx[(slice(None),) + sl].reshape(tree.nb, -1))
    corners = np.stack(corners, axis=-1)  # (nb, 512 cells, 8)
    for lv in np.unique(tree.blevel):
        bsel = tree.blevel == lv
        ncell = np.bincount(corners[bsel].reshape(-1), minlength=m).astype(np.float64)
        mass = mass + np.where(ncell > 0, kap_s[int(lv)] * (ncell / 8.0), 0.0)
    mass = np.where(inside == 1, 0.0, mass)
    K = sp.coo_matrix((np.concatenate([-W, -W, W, W, mass]),
                       (np.concatenate([a, b, a, b, np.arange(m)]),
                        np.concatenate([b, a, a, b, np.arange(m)]))), shape=(m, m)).tocsr()
    kind = node_kind(tree, pos)
    return {"pos": pos, "key": pkey, "inside": inside, "kind": kind, "K": K,
            "edges": {"a": a, "b": b, "level": lev, "d": d, "W": W, "alpha": alpha,
                      "count": cnt, "listed": listed, "key": uk},
            "mass": mass}


def crossing_edges(tree: Octree, op: dict, atoms) -> dict:
    """Listed edges (0 < alpha < 1, or ends in different media): they all lie
    in the all-finest region, so they are the listed edges of the uniform
    grid at h_fine spanning the domain, with the same alpha, r_p and sign.
    Adds the octree position indices of their ends and their slot-based id
    d * (512 nb) + slot(a).  The re-triangulated surface of Sec. 3.3.2 is
    that of the same uniform grid: its vertex weights ("mc_w") and analytic
    normals ("mc_n") come along with each edge."""
    g = _virtual_grid(tree, tree.Lmax)
    inside_g = U.classify(g, atoms)
    cr = U.crossing_edges(g, atoms, inside_g)
    cr["mc_w"] = U.mc_weights(g, inside_g, cr)
    cr["mc_n"] = U.mc_normals(cr, atoms)
    n = int(g.n[0])
    N = n ** 3
    d = (cr["ids"] // N).astype(np.int64)
    av = cr["ids"] % N
    Pa = np.stack([av % n, (av // n) % n, av // (n * n)], axis=1)
    Pb = Pa.copy()
    Pb[np.arange(len(d)), d] += 1
    NL1 = tree.NL + 1
    ka = (Pa[:, 2] * NL1 + Pa[:, 1]) * NL1 + Pa[:, 0]
    kb = (Pb[:, 2] * NL1 + Pb[:, 1]) * NL1 + Pb[:, 0]
    ia = np.searchsorted(op["key"], ka)
    ib = np.searchsorted(op["key"], kb)
    if np.any(op["key"][ia] != ka) or np.any(op["key"][ib] != kb):
        raise AssertionError("a listed edge end is not an octree node")
    # the owning slot of the low end
    slots = tree.slot_positions()
    skey = (slots[:, 2] * NL1 + slots[:, 1]) * NL1 + slots[:, 0]
    order = np.argsort(skey)
    js = np.searchsorted(skey[order], ka)
    if np.any(skey[order][js] != ka):
        raise AssertionError("a listed edge's low end has no slot")
    slot_a = order[js]
    oct_id = d * (512 * tree.nb) + slot_a
    srt = np.argsort(oct_id, kind="stable")
    out = {k: v[srt] for k, v in cr.items()}
    out.update(d=d[srt], a=ia[srt], b=ib[srt], slot_a=slot_a[srt], ids_octree=oct_id[srt])
    return out


def interpolation(tree: Octree, op: dict):
    """P (positions x unknowns) and the list of unknown positions (the
    regular interior nodes, in slot order)."""
    pos, kind, key = op["pos"], op["kind"], op["key"]
    slots = tree.slot_positions()
    NL1 = tree.NL + 1
    skey = (slots[:, 2] * NL1 + slots[:, 1]) * NL1 + slots[:, 0]
    sidx = np.searchsorted(key, skey)
    sreg = kind[sidx] == 0
    unk_slot = np.nonzero(sreg)[0]               # slot ids of the unknowns
    col_of_pos = np.full(len(pos), -1, dtype=np.int64)
    col_of_pos[sidx[unk_slot]] = np.arange(len(unk_slot))
    rows, cols, vals = [], [], []
    reg = np.nonzero(kind == 0)[0]
    if np.any(col_of_pos[reg] < 0):
        raise AssertionError("a regular interior position has no owning slot")
    rows.append(reg)
    cols.append(col_of_pos[reg])
    vals.append(np.ones(len(reg)))
    hang = np.nonzero(kind == 2)[0]
    par, w = hanging_parents(tree, pos[hang])
    pk = (par[..., 2] * NL1 + par[..., 1]) * NL1 + par[..., 0]
    pidx = np.searchsorted(key, pk)
    if np.any(key[np.clip(pidx, 0, len(key) - 1)] != pk):
        raise AssertionError("a hanging parent is not a corner position")
    if np.any(kind[pidx][w > 0] == 2):
        raise AssertionError("a hanging parent is itself hanging")
    for q in range(4):
        use = (w[:, q] > 0) & (kind[pidx[:, q]] == 0)
        rows.append(hang[use])
        cols.append(col_of_pos[pidx[use, q]])
        vals.append(w[use, q])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(len(pos), len(unk_slot))).tocsr()
    return P, unk_slot, (hang, pidx, w)


def boundary_field(tree: Octree, op: dict, hang_info, phib_of_pos: np.ndarray) -> np.ndarray:
    """x_b over all positions: boundary values at boundary positions, their
    interpolated share at hanging positions, zero elsewhere."""
    kind = op["kind"]
    xb = np.where(kind == 1, phib_of_pos, 0.0)
    hang, pidx, w = hang_info
    add = np.zeros(len(hang))
    for q in range(4):
        use = (w[:, q] > 0) & (kind[pidx[:, q]] == 1)
        add[use] += w[use, q] * phib_of_pos[pidx[use, q]]
    xb[hang] = add
    return xb


def bc_values(tree: Octree, op: dict, atoms, lB, eps_out, bc: int, kD: float) -> np.ndarray:
    """Dirichlet values (Sec. 2.3) at every boundary position."""
    pos = op["pos"]
    out = np.zeros(len(pos))
    if bc == U.BC_ZERO:
        return out
    sel = np.nonzero(op["kind"] == 1)[0]
    k = kD if bc == U.BC_DH else 0.0
    out[sel] = (lB / eps_out) * U.coulomb_phi(tree.world(pos[sel]), atoms, k)
    return out


def deposit(tree: Octree, op: dict, atoms, lB) -> np.ndarray:
    """4 pi l_B q_i times the trilinear weights of the charge's finest cell
    (Eq. RVop), over all positions."""
    pos, key = op["pos"], op["key"]
    NL1 = tree.NL + 1
    f = np.zeros(len(pos))
    for p in atoms:
        u = (p[:3] - tree.origin) / tree.h_fine
        c = np.clip(np.floor(u).astype(np.int64), 0, tree.NL - 1)
        t = u - c
        for off in np.ndindex(2, 2, 2):
            P = c + np.array(off)
            wgt = 1.0
            for dd in range(3):
                wgt *= t[dd] if off[dd] else 1.0 - t[dd]
            k = (P[2] * NL1 + P[1]) * NL1 + P[0]
            i = np.searchsorted(key, k)
            if i >= len(key) or key[i] != k or op["kind"][i] != 0:
                raise ValueError("a charge's cell corner is not a regular finest node")
            f[i] += 4.0 * math.pi * lB * p[4] * wgt
    return f


def jacobi_pcg(A, b, rtol: float, max_iter: int = 200000):
    """Jacobi-preconditioned CG from a zero guess; stops on the true relative
    residual (recomputed whenever the recursive one says converged)."""
    dg = A.diagonal()
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0, True
    r = b.copy()
    z = r / dg
    p = z.copy()
    rz = r @ z
    for it in range(1, max_iter + 1):
        q = A @ p
        al = rz / (p @ q)
        x += al * p
        r -= al * q
        if np.linalg.norm(r) <= rtol * bn:
            r = b - A @ x
            if np.linalg.norm(r) <= rtol * bn:
                return x, it, np.linalg.norm(r) / bn, True
        z = r / dg
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, max_iter, np.linalg.norm(b - A @ x) / bn, False


def energy(tree: Octree, op: dict, cross: dict, phi_pos: np.ndarray, atoms, lB, eps_in,
           eps_out) -> dict:
    """Energy terms of Sec. 3.3 from phi at all positions, over the flux
    edges (ends in different media) of the crossing list: Eq. polen, Eq.
    energy_ion (first integral on staircase faces with Eq. phi0, and on the
    re-triangulated surface of Sec. 3.3.2 as "e_ion_mc")."""
    e = op["edges"]
    flux = np.nonzero(cross["sign"] != 0)[0]
    a, b, d = cross["a"][flux], cross["b"][flux], cross["d"][flux]
    sign = cross["sign"][flux]
    # edge weight of the finest edge (a, d)
    ek = (a.astype(np.int64) * 3 + d) * (tree.Lmax + 1) + tree.Lmax
    ei = np.searchsorted(e["key"], ek)
    if np.any(e["key"][ei] != ek):
        raise AssertionError("a flux edge is not a finest-level edge")
    pin = np.where(sign > 0, phi_pos[a], phi_pos[b])
    pout = np.where(sign > 0, phi_pos[b], phi_pos[a])
    F = e["W"][ei] * (pin - pout)
    rp = cross["rp"][flux]
    al = cross["alpha"][flux]
    Phi = U.coulomb_phi(rp, atoms)
    Psi = U.coulomb_psi(rp, d.astype(np.int8), sign, atoms)
    phip = pin + (al / eps_in) * (pout - pin) / (al / eps_in + (1.0 - al) / eps_out)
    h = tree.h_fine
    S = float(np.sum(F * Phi))
    I = float(np.sum(phip * (h * h) * Psi))
    W = cross["mc_w"][flux]
    psin = U.coulomb_psi_n(rp, cross["mc_n"][flux], atoms)
    Imc = float(np.sum(W * phip * psin))
    e_coul = U.ecoul(atoms, lB, eps_in)
    e_pol = 0.5 * (1.0 / eps_out - 1.0 / eps_in) * S / (4.0 * math.pi)
    e_ion_flux = -0.5 * (1.0 / eps_out) * S / (4.0 * math.pi)
    e_ion_surf = 0.5 * I / (4.0 * math.pi)
    return {"e_coul": e_coul, "e_pol": e_pol, "e_ion_surf": e_ion_surf,
            "e_ion_flux": e_ion_flux, "e_total": e_coul + e_pol + e_ion_surf + e_ion_flux,
            "flux_charge": float(np.sum(F)) / (4.0 * math.pi * lB),
            "e_ion_mc": 0.5 * Imc / (4.0 * math.pi)}


def solve_problem(atoms, tree: Octree, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                  temperature_K=298.15, bc=U.BC_ZERO, rtol=1e-10, with_energy=True) -> dict:
    """Whole octree pipeline in the paper's order; returns every intermediate."""
    atoms = np.ascontiguousarray(atoms, dtype=np.float64)
    lB, kD = U.units(temperature_K, ionic_strength_M, eps_out)
    op = operator(tree, atoms, eps_in, eps_out, kD)
    P, unk_slot, hang_info = interpolation(tree, op)
    phib = bc_values(tree, op, atoms, lB, eps_out, bc, kD)
    xb = boundary_field(tree, op, hang_info, phib)
    K = op["K"]
    A = (P.T @ K @ P).tocsr()
    fpos = deposit(tree, op, atoms, lB)
    f = P.T @ (fpos - K @ xb)
    x, iters, rel, conv = jacobi_pcg(A, f, rtol)
    phi_pos = P @ x + xb
    res = {"tree": tree, "op": op, "P": P, "A": A, "f": f, "x": x, "xb": xb,
           "unk_slot": unk_slot, "phi_pos": phi_pos, "iters": iters, "relres": rel,
           "converged": conv, "lB": lB, "kD": kD}
    if with_energy:
        cross = crossing_edges(tree, op, atoms)
        res["cross"] = cross
        res["energy"] = energy(tree, op, cross, phi_pos, atoms, lB, eps_in, eps_out)
    return res
