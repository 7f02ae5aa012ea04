"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms printed in the paper, discrete identities that hold exactly, special
cases that reduce to a library routine (dense LU/Cholesky, the DST-I Poisson
solver), or brute force on tiny inputs.  None of these needs a GPU.
"""
import math
import os

import numpy as np
import pytest
import scipy.fft
import scipy.linalg

import pb_inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return rows


def _centered_sphere(orc, n, h, R=2.0, q=1.0):
    c = (n - 1) * h / 2.0
    atoms = np.array([[c, c, c, R, q]])
    return atoms, orc.Grid((n, n, n), (0.0, 0.0, 0.0), h)


def _dense_operator(orc, g, coef):
    """Columns of A obtained by applying the oracle to unit vectors."""
    n = g.n
    interior = [a for a in range(g.N)
                if 0 < a % n[0] < n[0] - 1 and 0 < (a // n[0]) % n[1] < n[1] - 1
                and 0 < a // (n[0] * n[1]) < n[2] - 1]
    M = np.empty((len(interior), len(interior)))
    e = np.zeros(g.N)
    for c, a in enumerate(interior):
        e[:] = 0.0
        e[a] = 1.0
        M[:, c] = orc.apply(g, coef, e)[interior]
    return M, np.array(interior)


# --------------------------------------------------------------------------
# grid placement (perfil, Sec. 2.3 and Sec. 3.4)
# --------------------------------------------------------------------------

# Three balls chosen by hand.  Their union spans x in [-1, 6], y in [-1, 5.5]
# and z in [-4, 3.5]: the largest span (7.5) is along z, the low and high
# ends of each axis come from different balls, and the centres alone span
# only 4, 5 and 5.  Every number below is exact in binary, so placement is
# checked for equality.
_PLACE_ATOMS = np.array([[0.0, 0.0, 0.0, 1.0, 0.5],
                         [4.0, 1.0, -2.0, 2.0, -0.3],
                         [1.0, 5.0, 3.0, 0.5, 0.1]])


def test_uniform_placement_by_hand(orc):
    """Cube of side fill * extent (extent = largest axis span of the union of
    the balls) centred on the balls' bounding box, with h = L / (n - 1): here
    L = 1.5 * 7.5 = 11.25, h = 11.25 / 9 = 1.25 and the box centre is
    (2.5, 2.25, -0.25).  Taking the extent over the centres (L = 7.5), the
    spacing as L / n (1.125), or the centroid of the atoms as the centre
    would each change the result."""
    g = orc.place_grid(_PLACE_ATOMS, 10, 1.5)
    assert tuple(int(v) for v in g.n) == (10, 10, 10)
    assert g.h == 1.25
    assert tuple(g.origin) == (-3.125, -3.375, -5.875)
    # the far corner is the box centre plus L/2 on every axis
    far = np.asarray(g.origin) + 9 * g.h
    assert tuple(far) == (8.125, 7.875, 5.375)


def test_octree_placement_by_hand(orc):
    """The octree domain is n0 coarse bricks of side 8 h_bulk per axis, with
    n0 = ceil(fill * extent / (8 h_bulk)), centred on the same bounding box:
    1.5 * 7.5 / 8 = 1.40625 gives n0 = 2 (side 16 at h_bulk = 1) and
    0.5 * 7.5 / 8 gives n0 = 1 (side 8); at h_bulk = 0.25 it is
    ceil(11.25 / 2) = 6 (side 12)."""
    from oracle import octree
    for h_bulk, fill, n0, side in ((1.0, 1.5, 2, 16.0), (1.0, 0.5, 1, 8.0),
                                   (0.25, 1.5, 6, 12.0)):
        origin, got = octree.place(_PLACE_ATOMS, h_bulk, fill)
        assert got == n0
        centre = np.array([2.5, 2.25, -0.25])
        assert np.array_equal(origin, centre - side / 2)


# --------------------------------------------------------------------------
# units and closed forms
# --------------------------------------------------------------------------

def test_units_reproduce_printed_kirkwood_values(orc):
    """The paper's analytic Kirkwood energies (Table tab:energies_1sf) follow
    from the closed forms of Sec. 6.1.1 only with the right l_B and k_D."""
    (pol, ion, tot), = _golden("kirkwood_table.txt")
    lB, kD = orc.units(298.15, 0.145, 80.0)
    R, q = 2.0, 1.0
    e_pol = 0.5 * (1 / 80.0 - 1 / 2.0) * q * q * lB / R
    e_ion = -0.5 * q * q * lB / 80.0 * kD / (1.0 + kD * R)
    assert abs(e_pol - pol) <= 0.005
    assert abs(e_ion - ion) <= 0.005
    assert abs(e_pol + e_ion - tot) <= 0.005
    assert abs(kD - 0.124) < 5e-4  # "k ~ 0.125 1/A" for 0.145 M


def test_born_ion_polarization_energy_exact(orc):
    """Born ion (eps 1/80, R = 2 A, 65^3, h = 0.3125, Coulomb BC): by the
    discrete Gauss identity the flux-based E_pol of Sec. 3.3.1 equals the
    closed form up to the solver tolerance (the paper reports 7.38e-10)."""
    (born,), = _golden("born_ion.txt")
    g = orc.Grid((65, 65, 65), (0.0, 0.0, 0.0), 0.3125)
    r = orc.solve_problem(pb_inputs.born_ion(), g, eps_in=1.0, eps_out=80.0,
                          ionic_strength_M=0.0, bc=orc.BC_COULOMB, rtol=1e-10)
    assert r["converged"] and r["relres"] <= 1e-10
    e = r["energy"]
    closed = 0.5 * (1 / 80.0 - 1.0) * r["lB"] / 2.0
    assert abs(closed - born) < 5e-4
    assert abs(e["e_pol"] - closed) / abs(closed) < 1e-8
    assert abs(e["flux_charge"] - 1.0) < 1e-8
    # no salt: the two ionic integrals cancel in the continuum limit
    assert abs(e["e_ion_surf"] + e["e_ion_flux"]) < 0.01 * abs(closed)


def test_kirkwood_epol_exact_and_eion_converges(orc):
    """Kirkwood sphere in 0.145 M salt with Debye-Hueckel BC: E_pol exact,
    ionic energy converging to its closed form (Sec. 6.1.1) as h shrinks."""
    lB, kD = orc.units(298.15, 0.145, 80.0)
    e_pol = 0.5 * (1 / 80.0 - 1 / 2.0) * lB / 2.0
    e_ion = -0.5 * lB / 80.0 * kD / (1.0 + kD * 2.0)
    errs = []
    for n, h in ((33, 0.5), (65, 0.25)):
        atoms, g = _centered_sphere(orc, n, h)
        r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                              bc=orc.BC_DH, rtol=1e-11)
        e = r["energy"]
        assert abs(e["e_pol"] - e_pol) / abs(e_pol) < 1e-9
        errs.append(abs(e["e_ion_surf"] + e["e_ion_flux"] - e_ion) / abs(e_ion))
    assert errs[1] < 0.6 * errs[0]
    assert errs[1] < 0.06


def test_debye_hueckel_potential_outside_sphere(orc):
    """Nodal phi outside a charged sphere in salt vs the exact outside
    potential of Sec. 2.3, converging under refinement."""
    lB, kD = orc.units(298.15, 0.145, 80.0)
    errs = []
    for n, h in ((33, 0.5), (65, 0.25)):
        atoms, g = _centered_sphere(orc, n, h)
        r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                              bc=orc.BC_DH, rtol=1e-11, with_energy=False)
        nx = n
        idx = np.arange(g.N)
        pos = np.stack([idx % nx, (idx // nx) % nx, idx // (nx * nx)], 1) * h
        dist = np.linalg.norm(pos - atoms[0, :3], axis=1)
        interior = (pos > 0.0).all(1) & (pos < (n - 1) * h).all(1)
        sel = interior & (dist >= 2.0 + 2 * h) & (dist <= 6.0)
        exact = lB / 80.0 * np.exp(-kD * (dist[sel] - 2.0)) / (dist[sel] * (1 + kD * 2.0))
        errs.append(np.max(np.abs(r["phi"][sel] - exact) / exact))
    assert errs[1] < errs[0]
    assert errs[1] < 0.05


# --------------------------------------------------------------------------
# operator structure
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_system(orc):
    atoms = pb_inputs.globular_molecule(6, seed=11, radius=2.0)
    g = orc.place_grid(atoms, 9, 1.2)
    lB, kD = orc.units(298.15, 0.145, 80.0)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    coef = orc.assemble(g, inside, cross, 2.0, 80.0, kD)
    return atoms, g, inside, cross, coef, lB, kD


def test_operator_symmetric_spd_mmatrix(orc, small_system):
    atoms, g, inside, cross, coef, lB, kD = small_system
    assert inside.sum() > 0 and len(cross["ids"]) > 0
    M, _ = _dense_operator(orc, g, coef)
    assert np.array_equal(M, M.T)  # bitwise symmetric
    scipy.linalg.cholesky(M)  # SPD
    off = M - np.diag(np.diag(M))
    assert (off <= 0).all()
    assert (np.diag(M) + off.sum(1) >= -1e-12).all()  # weak diagonal dominance


def test_dense_direct_solve_matches_pcg(orc, small_system):
    atoms, g, inside, cross, coef, lB, kD = small_system
    phib = orc.bc_values(g, atoms, lB, 80.0, orc.BC_DH, kD)
    f = orc.rhs(g, atoms, lB, coef, phib)
    M, interior = _dense_operator(orc, g, coef)
    xd = scipy.linalg.solve(M, f[interior], assume_a="pos")
    x, it, rel, ok = orc.pcg(g, coef, f, 1e-13)
    assert ok
    assert np.max(np.abs(x[interior] - xd)) <= 1e-10 * np.max(np.abs(xd))


def test_uniform_eps_reduces_to_dst_poisson(orc):
    """eps_in = eps_out, no salt: A = eps h (7-point Laplacian), which the
    type-I discrete sine transform diagonalises exactly."""
    n, eps = 17, 3.0
    atoms = pb_inputs.globular_molecule(5, seed=3, radius=2.5)
    g = orc.place_grid(atoms, n, 1.6)
    lB, kD = orc.units(298.15, 0.0, eps)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    coef = orc.assemble(g, inside, cross, eps, eps, kD)
    f = orc.rhs(g, atoms, lB, coef, np.zeros(g.N))
    x, it, rel, ok = orc.pcg(g, coef, f, 1e-13)
    assert ok
    m = n - 2
    F = f.reshape(n, n, n)[1:-1, 1:-1, 1:-1] / (eps * g.h)
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(1, m + 1) / (m + 1))
    L = lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    U = scipy.fft.idstn(scipy.fft.dstn(F, type=1, norm="ortho") / L, type=1, norm="ortho")
    X = x.reshape(n, n, n)[1:-1, 1:-1, 1:-1]
    assert np.max(np.abs(X - U)) <= 1e-10 * np.max(np.abs(U))


def test_dirichlet_lift_reproduces_linear_field(orc):
    """A linear potential is discretely harmonic: with uniform eps, no charge
    and boundary values from a linear function, the solve returns it."""
    n = 13
    atoms = np.array([[3.0, 3.0, 3.0, 1.5, 0.0]])
    g = orc.Grid((n, n, n), (0.0, 0.0, 0.0), 0.5)
    lB, kD = orc.units(298.15, 0.0, 5.0)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    coef = orc.assemble(g, inside, cross, 5.0, 5.0, kD)
    idx = np.arange(g.N)
    pos = np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) * g.h
    lin = 0.3 * pos[:, 0] - 1.1 * pos[:, 1] + 0.7 * pos[:, 2] + 2.0
    bnd = ((pos == 0.0) | (pos == (n - 1) * g.h)).any(1)
    phib = np.where(bnd, lin, 0.0)
    f = orc.rhs(g, atoms, lB, coef, phib)
    x, it, rel, ok = orc.pcg(g, coef, f, 1e-14)
    assert np.max(np.abs(x[~bnd] - lin[~bnd])) < 1e-10


def test_deposit_moments(orc):
    """Trilinear charge assignment (Eq. RVop): weights sum to one and keep
    the first moment, so sum_k f_k = 4 pi l_B Q and sum_k f_k x_k = 4 pi
    l_B sum_i q_i x_i (zero BC, so f holds the deposit only)."""
    atoms = pb_inputs.globular_molecule(40, seed=5)
    g = orc.place_grid(atoms, 33, 1.5)
    lB, kD = orc.units()
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    coef = orc.assemble(g, inside, cross, 2.0, 80.0, kD)
    f = orc.rhs(g, atoms, lB, coef, np.zeros(g.N)) / (4 * np.pi * lB)
    n = g.n[0]
    idx = np.arange(g.N)
    pos = g.origin + np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1) * g.h
    q = atoms[:, 4]
    assert abs(f.sum() - q.sum()) < 1e-12 * np.abs(q).sum()
    m1 = (f[:, None] * pos).sum(0)
    assert np.allclose(m1, (q[:, None] * atoms[:, :3]).sum(0), rtol=0, atol=1e-10 * np.abs(q).sum() * 50)


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def test_classification_matches_brute_force(orc):
    atoms = pb_inputs.globular_molecule(30, seed=8)
    g = orc.place_grid(atoms, 25, 1.4)
    inside = orc.classify(g, atoms)
    n = g.n[0]
    idx = np.arange(g.N)
    pos = g.origin + np.stack([idx % n, (idx // n) % n, idx // (n * n)], 1).astype(float) * g.h
    d2 = ((pos[:, None, :] - atoms[None, :, :3]) ** 2).sum(-1)
    brute = (d2 < atoms[None, :, 3] ** 2).any(1)
    # numpy's summation order may differ in the last bit only at |d|=R ties
    assert (inside.astype(bool) != brute).sum() == 0
    assert np.array_equal(orc.classify_nodes(g, atoms, idx), inside)


def test_inside_fraction_against_dense_sampling(orc):
    """alpha of an edge (the WHA weight of Sec. 3.2) equals the measure of
    the edge inside the union of balls, here measured by midpoint sampling;
    includes edges crossing one ball, two overlapping balls and a cap."""
    atoms = np.array([[0.0, 0.0, 0.0, 1.3, 0.5], [1.6, 0.1, 0.0, 1.1, -0.5],
                      [0.4, 2.2, 0.3, 1.2, 0.1]])
    g = orc.Grid((24, 24, 24), (-2.9, -2.7, -2.6), 0.29)
    rng = np.random.Generator(np.random.PCG64(1))
    n = 24
    N = g.N
    ids = []
    while len(ids) < 150:
        d = int(rng.integers(3))
        i, j, k = (int(v) for v in rng.integers(0, n - 1, 3))
        ids.append(d * N + (k * n + j) * n + i)
    # plus edges near the surface (chosen from the list; checked by sampling)
    listed = orc.crossing_edges(g, atoms, orc.classify(g, atoms))["ids"]
    ids += list(rng.choice(listed, 150, replace=False))
    alpha = orc.edge_alpha(g, atoms, ids)
    M = 100000
    t = (np.arange(M) + 0.5) / M
    nontrivial = 0
    for e, a in zip(ids, alpha):
        d, node = divmod(e, N)
        p0 = g.origin + np.array([node % n, (node // n) % n, node // (n * n)], float) * g.h
        pts = np.repeat(p0[None], M, 0)
        pts[:, d] += t * g.h
        d2 = ((pts[:, None, :] - atoms[None, :, :3]) ** 2).sum(-1)
        frac = (d2 < atoms[None, :, 3] ** 2).any(1).mean()
        assert abs(frac - a) <= 2.0 / M + 1e-12
        nontrivial += 0.0 < a < 1.0
    assert nontrivial > 100


def test_crossing_list_matches_brute_force(orc):
    atoms = pb_inputs.globular_molecule(25, seed=9)
    g = orc.place_grid(atoms, 21, 1.4)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    n = 21
    N = g.N
    ids = []
    for d in range(3):
        for a in range(N):
            c = (a % n, (a // n) % n, a // (n * n))[d]
            if c < n - 1:
                ids.append(d * N + a)
    ids = np.array(ids)
    alpha = orc.edge_alpha(g, atoms, ids)
    stride = np.array([1, n, n * n])
    d = ids // N
    a = ids % N
    differ = inside[a] != inside[a + stride[d]]
    keep = ((alpha > 0) & (alpha < 1)) | differ
    assert np.array_equal(cross["ids"], ids[keep])
    assert np.array_equal(cross["alpha"], alpha[keep])  # bit-exact
    # the polarisation point sits on a sphere surface for single crossings
    sg = cross["sign"]
    assert set(np.unique(sg)) <= {-1, 0, 1}
    flux = sg != 0
    r = np.min(np.abs(np.linalg.norm(cross["rp"][flux][:, None, :] - atoms[None, :, :3], axis=2)
                      - atoms[None, :, 3]), axis=1)
    assert np.median(r) < 1e-9


def test_node_coeffs_match_assembly(orc, small_system):
    atoms, g, inside, cross, coef, lB, kD = small_system
    n = g.n[0]
    nodes = np.array([(k * n + j) * n + i for k in range(1, n - 1)
                      for j in range(1, n - 1) for i in range(1, n - 1)])
    nc = orc.node_coeffs(g, atoms, 2.0, 80.0, kD, nodes)
    s = np.array([1, n, n * n])
    W = [coef["Wx"], coef["Wy"], coef["Wz"]]
    for dd in range(3):
        assert np.array_equal(nc[:, 2 * dd], W[dd][nodes - s[dd]])
        assert np.array_equal(nc[:, 2 * dd + 1], W[dd][nodes])
    assert np.array_equal(nc[:, 6], coef["kap"][nodes])
    assert np.array_equal(nc[:, 7], coef["diag"][nodes])


def test_wha_special_cases(orc):
    """WHA (Eq. WHA): equal media give eps whatever alpha; otherwise the
    edge permittivity lies between the two media."""
    atoms = pb_inputs.globular_molecule(12, seed=4)
    g = orc.place_grid(atoms, 21, 1.3)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    lB, kD = orc.units(298.15, 0.0, 7.0)
    c_eq = orc.assemble(g, inside, cross, 7.0, 7.0, kD)
    ids = cross["ids"]
    N = g.N
    W = np.stack([c_eq["Wx"], c_eq["Wy"], c_eq["Wz"]])
    assert np.allclose(W[ids // N, ids % N] / g.h, 7.0, rtol=1e-15, atol=0)
    c = orc.assemble(g, inside, cross, 2.0, 80.0, kD)
    W = np.stack([c["Wx"], c["Wy"], c["Wz"]])[ids // N, ids % N] / g.h
    assert (W >= 2.0 - 1e-12).all() and (W <= 80.0 + 1e-12).all()
    a = cross["alpha"]
    order = np.argsort(a)
    assert (np.diff(W[order]) <= 1e-12).all()  # more solute -> smaller eps


# --------------------------------------------------------------------------
# N-body terms
# --------------------------------------------------------------------------

def test_coulomb_closed_forms(orc):
    lB = 560.0
    s = 2.5
    tri = np.array([[0, 0, 0, 1, 1.0], [s, 0, 0, 1, -0.5],
                    [s / 2, s * math.sqrt(3) / 2, 0, 1, 0.25]])
    q = tri[:, 4]
    expect = (lB / 2.0) * (q[0] * q[1] + q[0] * q[2] + q[1] * q[2]) / s
    assert abs(orc.ecoul(tri, lB, 2.0) - expect) < 1e-12 * abs(expect)
    one = np.array([[1.0, -2.0, 0.5, 1.5, 0.7]])
    rng = np.random.Generator(np.random.PCG64(2))
    v = rng.normal(size=(50, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    pts = one[0, :3] + 3.0 * v
    assert np.allclose(orc.coulomb_phi(pts, one), 0.7 / 3.0, rtol=1e-14)
    k = 0.3
    assert np.allclose(orc.coulomb_phi(pts, one, k), 0.7 * math.exp(-0.9) / 3.0, rtol=1e-14)
    tgt = one[0, :3] + np.array([[2.0, 0, 0], [0, -4.0, 0]])
    psi = orc.coulomb_psi(tgt, [0, 1], [1, 1], one)
    assert np.allclose(psi, [0.7 / 4.0, -0.7 / 16.0], rtol=1e-14)


def test_staircase_solid_angle(orc):
    """The staircase faces of the flux edges close around the solute, so
    sum_e h^2 (r_p - r_c).n_e / (4 pi |r_p - r_c|^3) approximates the full
    solid angle 1 seen from an enclosed charge (quadrature of the first
    integral of Eq. energy_ion)."""
    atoms, g = _centered_sphere(orc, 65, 0.25)
    inside = orc.classify(g, atoms)
    cross = orc.crossing_edges(g, atoms, inside)
    flux = cross["sign"] != 0
    dirs = (cross["ids"][flux] // g.N).astype(np.int8)
    psi = orc.coulomb_psi(cross["rp"][flux], dirs, cross["sign"][flux], atoms[:, :5] * [1, 1, 1, 1, 0] + [0, 0, 0, 0, 1])
    omega = (g.h ** 2) * psi.sum() / (4 * np.pi)
    assert abs(omega - 1.0) < 0.02


def test_gauss_identity_molecule(orc):
    """Discrete Gauss law: the outward flux through the flux edges equals
    4 pi l_B times the enclosed charge (Sec. 3.3.1), for a random molecule."""
    atoms = pb_inputs.globular_molecule(60, seed=21)
    g = orc.place_grid(atoms, 41, 1.5)
    r = orc.solve_problem(atoms, g, rtol=1e-12)
    Q = atoms[:, 4].sum()
    assert abs(r["energy"]["flux_charge"] - Q) < 1e-8 * max(1.0, np.abs(atoms[:, 4]).sum())


# --------------------------------------------------------------------------
# first integral of Eq. energy_ion on the re-triangulated surface (Sec. 3.3.2)
# --------------------------------------------------------------------------

def _sphere_mc(orc, n, L, c, R):
    h = L / (n - 1)
    atoms = np.array([[*c, R, 1.0]])
    g = orc.Grid((n, n, n), (0.0, 0.0, 0.0), h)
    ins = orc.classify(g, atoms)
    cr = orc.crossing_edges(g, atoms, ins)
    return atoms, g, cr, orc.mc_weights(g, ins, cr), orc.mc_normals(cr, atoms)


def test_mc_surface_area_converges_second_order(orc):
    """The marching-cubes triangles through the exact intersection points
    approximate a sphere: their total area tends to 4 pi R^2 with an error
    that falls fourfold when h halves (the staircase faces never converge)."""
    R, L = 2.0, 8.0
    c = (L / 2 + 0.0123, L / 2 - 0.0311, L / 2 + 0.0207)
    errs = []
    for n in (17, 33, 65):
        _, _, cr, W, _ = _sphere_mc(orc, n, L, c, R)
        assert np.all(W[cr["sign"] == 0] == 0.0) and np.all(W[cr["sign"] != 0] > 0.0)
        errs.append(abs(W.sum() / (4 * math.pi * R * R) - 1.0))
    assert errs[0] < 2e-2 and errs[2] < 1.2e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


def test_mc_surface_of_a_plane_is_exact(orc):
    """A ball of radius 1e6 is a plane on the scale of the grid: inside every
    cell the marching-cubes polygon is the plane's cross-section, so the
    total area is that of the plane inside the box, L^2 |n| / |n_z| for the
    tilted normal n = (0.2, 0.1, 1)."""
    n, L, R = 21, 4.0, 1e6
    nv = np.array([0.2, 0.1, 1.0])
    nv /= np.linalg.norm(nv)
    p0 = np.array([L / 2 + 0.013, L / 2 - 0.021, L / 2 + 0.007])
    atoms, g, cr, W, nrm = _sphere_mc(orc, n, L, p0 - R * nv, R)
    expect = L * L / nv[2]
    assert abs(W.sum() / expect - 1.0) < 1e-9
    flux = cr["sign"] != 0
    assert np.allclose(nrm[flux], nv, atol=1e-5)


def test_mc_normals_belong_to_the_exposed_sphere(orc):
    """Each vertex normal is the unit vector from the centre of a ball whose
    sphere passes through the vertex, and the vertex lies in no other ball."""
    atoms = np.array([[4.0, 4.0, 4.0, 1.8, 1.0], [5.9, 4.3, 4.1, 1.5, -0.5],
                      [4.2, 5.7, 3.6, 1.3, 0.25]])
    g = orc.Grid((33, 33, 33), (0.0, 0.0, 0.0), 0.3)
    ins = orc.classify(g, atoms)
    cr = orc.crossing_edges(g, atoms, ins)
    nrm = orc.mc_normals(cr, atoms)
    flux = np.flatnonzero(cr["sign"] != 0)
    assert np.allclose(np.linalg.norm(nrm[flux], axis=1), 1.0, atol=1e-14)
    for s in flux:
        p = cr["rp"][s]
        d = np.linalg.norm(p - atoms[:, :3], axis=1)
        owner = [a for a in range(3) if np.allclose(p - atoms[a, :3], nrm[s] * d[a], atol=1e-12)]
        assert owner and abs(d[owner[0]] - atoms[owner[0], 3]) < 1e-9
        assert np.all(d >= atoms[:, 3] - 1e-9)


def test_mc_solid_angle_of_a_union_of_balls(orc):
    """Gauss: the solid angle of a closed surface seen from a point inside is
    4 pi.  The vertex rule on the re-triangulated union of three balls gives
    it to within about 1e-2, closing in under refinement (the creases where
    spheres meet keep the rate near first order)."""
    atoms = np.array([[4.0, 4.0, 4.0, 1.8, 1.0], [5.9, 4.3, 4.1, 1.5, -0.5],
                      [4.2, 5.7, 3.6, 1.3, 0.25]])
    x = np.array([4.6, 4.4, 4.0])
    errs = []
    for n, h in ((33, 0.3), (65, 0.15)):
        g = orc.Grid((n, n, n), (0.0, 0.0, 0.0), h)
        ins = orc.classify(g, atoms)
        cr = orc.crossing_edges(g, atoms, ins)
        W = orc.mc_weights(g, ins, cr)
        nrm = orc.mc_normals(cr, atoms)
        d = cr["rp"] - x
        r = np.linalg.norm(d, axis=1)
        errs.append(abs((W * np.einsum("ij,ij->i", d, nrm) / r ** 3).sum() / (4 * math.pi) - 1))
    assert errs[0] < 3e-2 and errs[1] < 0.5 * errs[0] and errs[1] < 1e-2


def test_kirkwood_eion_with_mc_surface_converges(orc):
    """Kirkwood sphere in 0.145 M salt (Sec. 6.1.1): the paper's E_ion, the
    first integral on the re-triangulated surface plus the flux term,
    converges to the closed form, and beats the staircase quadrature at
    every spacing."""
    lB, kD = orc.units(298.15, 0.145, 80.0)
    e_ion = -0.5 * lB / 80.0 * kD / (1.0 + kD * 2.0)
    errs = []
    for n, h in ((33, 0.5), (65, 0.25)):
        atoms, g = _centered_sphere(orc, n, h)
        r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                              bc=orc.BC_DH, rtol=1e-11)
        e = r["energy"]
        mc = abs(e["e_ion_mc"] + e["e_ion_flux"] - e_ion) / abs(e_ion)
        stair = abs(e["e_ion_surf"] + e["e_ion_flux"] - e_ion) / abs(e_ion)
        assert mc < stair
        errs.append(mc)
    assert errs[0] < 0.06 and errs[1] < 0.6 * errs[0]
