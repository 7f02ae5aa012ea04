"""The reasoning the crossing-edge build rests on, checked against the
oracle's own interval union (``orc.edge_alpha``) on inputs full of exact ties.

The build evaluates the union of the balls' intervals only where it can
matter.  It marks, per ball and lattice line, the edges where that ball's
interval is partial (t0 > 0 or t1 < 1), found by scanning the line from both
ends, and the edges where it is all of [0, 1].  It then lists:
* every edge whose end nodes differ in the inside flag;
* a candidate that no ball covers when its union lies strictly inside (0, 1).

Pinned here:
* along a line the interval ends a0, a1 only fall as the edge moves up (what
  lets the scan stop at the first t0 = 0 from below and the first t1 = 1
  from above);
* an edge where no ball's interval is partial has alpha exactly 0 (no ball
  meets it) or exactly 1 (some ball covers it);
* an edge some ball covers has alpha exactly 1;
* the listing rule reproduces the oracle's crossing list.

The per-ball interval is the formula of Sec. 3.2's inside fraction, written
out here with each step rounded as in the oracle and the CUDA path."""
import numpy as np
import pytest

import pb_inputs

N, O, H = (33, 33, 33), (-8.0, -8.0, -8.0), 0.5


def _line_intervals(atom, d):
    """(edge ids, unclamped a0, a1, valid, t0, t1) for the ball's lattice lines
    along direction d, each row one line, each column one edge of it."""
    c, r = atom[:3], atom[3]
    e, f = (1, 2) if d == 0 else ((0, 2) if d == 1 else (0, 1))
    lo = [int(np.clip(np.floor((c[q] - r - O[q]) / H) - 1, 0, N[q] - 1)) for q in range(3)]
    hi = [int(np.clip(np.ceil((c[q] + r - O[q]) / H) + 1, 0, N[q] - 1)) for q in range(3)]
    ie = np.arange(lo[e], hi[e] + 1)
    jf = np.arange(lo[f], hi[f] + 1)
    idd = np.arange(lo[d], min(hi[d], N[d] - 2) + 1)
    E, F, I = np.meshgrid(ie, jf, idd, indexing="ij")
    E, F, I = E.reshape(len(ie) * len(jf), -1), F.reshape(len(ie) * len(jf), -1), I.reshape(
        len(ie) * len(jf), -1)
    xd = O[d] + I.astype(np.float64) * H
    xe = O[e] + E.astype(np.float64) * H
    xf = O[f] + F.astype(np.float64) * H
    ud, ue, uf = xd - c[d], xe - c[e], xf - c[f]
    s = r * r - (ue * ue + uf * uf)
    w = np.sqrt(np.where(s > 0.0, s, 0.0))
    a0 = ((-ud) - w) / H
    a1 = ((-ud) + w) / H
    t0 = np.where(a0 < 0.0, 0.0, a0)
    t1 = np.where(a1 > 1.0, 1.0, a1)
    valid = (s > 0.0) & (t1 > t0)
    ijk = [None, None, None]
    ijk[d], ijk[e], ijk[f] = I, E, F
    node = (ijk[2] * N[1] + ijk[1]) * N[0] + ijk[0]
    ids = d * (N[0] * N[1] * N[2]) + node
    return ids, a0, a1, s > 0.0, valid, t0, t1


def _marks(atoms):
    cand, cov, met = set(), set(), set()
    mono = True
    for atom in atoms:
        for d in range(3):
            ids, a0, a1, cut, valid, t0, t1 = _line_intervals(atom, d)
            # a0, a1 fall along every line that the ball cuts
            rows = cut[:, 0]
            if rows.any():
                mono &= bool(np.all(np.diff(a0[rows], axis=1) <= 0.0))
                mono &= bool(np.all(np.diff(a1[rows], axis=1) <= 0.0))
            partial = valid & ((t0 > 0.0) | (t1 < 1.0))
            whole = valid & ~(t0 > 0.0) & ~(t1 < 1.0)
            cand.update(ids[partial].tolist())
            cov.update(ids[whole].tolist())
            met.update(ids[valid].tolist())
    return cand, cov, met, mono


@pytest.mark.parametrize("kind", ["placed", "snapped"])
def test_candidate_and_cover_reasoning(orc, kind):
    atoms = pb_inputs.lattice_balls() if kind == "placed" else pb_inputs.snapped_molecule()
    g = orc.Grid(N, O, H)
    cand, cov, met, mono = _marks(atoms)
    assert mono
    assert cand and cov
    # every existing edge of the grid
    nn = np.array(N)
    ids = []
    for d in range(3):
        k, j, i = np.meshgrid(np.arange(N[2]), np.arange(N[1]), np.arange(N[0]), indexing="ij")
        ok = (np.stack([i, j, k])[d] < nn[d] - 1).reshape(-1)
        ids.append(d * int(np.prod(nn)) + np.nonzero(ok)[0])
    ids = np.concatenate(ids)
    alpha = orc.edge_alpha(g, atoms, ids)
    in_cand = np.isin(ids, np.fromiter(cand, dtype=np.int64))
    in_cov = np.isin(ids, np.fromiter(cov, dtype=np.int64))
    in_met = np.isin(ids, np.fromiter(met, dtype=np.int64))
    # no partial interval: alpha is exactly 0 or 1, and which one is decided
    assert np.all(alpha[~in_cand & in_cov] == 1.0)
    assert np.all(alpha[~in_cand & ~in_met] == 0.0)
    assert np.array_equal(in_met[~in_cand], in_cov[~in_cand])
    # a covering ball decides alpha = 1 whatever the others add
    assert np.all(alpha[in_cov] == 1.0)
    # the listing rule gives the oracle's crossing list
    inside = orc.classify(g, atoms)
    d = ids // int(np.prod(nn))
    a = ids - d * int(np.prod(nn))
    step = np.array([1, N[0], N[0] * N[1]])[d]
    differ = inside[a] != inside[a + step]
    listed = differ | (in_cand & ~in_cov & (alpha > 0.0) & (alpha < 1.0))
    cr = orc.crossing_edges(g, atoms, inside)
    assert np.array_equal(np.sort(ids[listed]), cr["ids"])
