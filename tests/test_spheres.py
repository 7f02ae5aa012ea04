"""The paper's analytical benchmark: non-overlapping dielectric spheres with
central charges, solved by multipole expansion (oracle/spheres.py).

First the expansion is pinned against what fixes it independently: the
Born and Debye-Hueckel closed forms for one sphere, the plain Coulomb energy
when the two media are the same, the far-apart limit, and convergence in the
expansion order.  Then it pins the discretisation: the energies of the
box-method scheme (the oracle, which the GPU path matches to 1e-6) agree with
the analytic ones to a few 1e-4 on grids of 0.5 and 0.4 A, without salt
(E_coul + E_pol) and in 0.145 M salt (E_total, staircase ionic surface term
included)."""
import numpy as np
import pytest

# three spheres with small gaps (0.6 to 1.5 A), charges of both signs
C3 = np.array([[0.0, 0.0, 0.0], [4.6, 0.4, -0.3], [1.9, 3.9, 1.1]])
R3 = np.array([2.0, 1.6, 1.4])
Q3 = np.array([1.0, -1.0, 0.6])


@pytest.fixture(scope="module")
def S():
    from oracle import spheres
    return spheres


def test_one_sphere_closed_forms(S, orc):
    lB, kD = orc.units(298.15, 0.145, 80.0)
    for k in (0.0, kD):
        for R, q, ein in ((2.0, 1.0, 1.0), (1.3, -0.7, 4.0)):
            e = S.SphereSystem([[0.3, -0.2, 0.1]], [R], [q], ein, 80.0, k, lB, L=4).solve()["energy"]
            exact = 0.5 * q * q * lB / R * (1.0 / (80.0 * (1.0 + k * R)) - 1.0 / ein)
            assert abs(e / exact - 1.0) < 1e-12


def test_equal_media_give_the_coulomb_energy(S, orc):
    lB, _ = orc.units(298.15, 0.0, 80.0)
    e = S.SphereSystem(C3, R3, Q3, 5.0, 5.0, 0.0, lB, L=12).solve()["energy"]
    assert abs(e / S.coulomb_energy(C3, Q3, 5.0, lB) - 1.0) < 1e-12


def test_expansion_converges_and_ignores_order(S, orc):
    for I in (0.0, 0.145):
        lB, kD = orc.units(298.15, I, 80.0)
        e = [S.SphereSystem(C3, R3, Q3, 2.0, 80.0, kD, lB, L=L).solve()["energy"] for L in (12, 18, 24)]
        assert abs(e[1] - e[2]) < 1e-9 * abs(e[2]) and abs(e[0] - e[2]) < 1e-6 * abs(e[2])
        p = [2, 0, 1]
        ep = S.SphereSystem(C3[p], R3[p], Q3[p], 2.0, 80.0, kD, lB, L=18).solve()["energy"]
        assert abs(ep - e[1]) < 1e-11 * abs(e[1])


def test_far_apart_limit(S, orc):
    """Two spheres 60 A apart: the two Born energies plus the charges'
    interaction in the solvent (screened), up to the induced terms."""
    lB, kD = orc.units(298.15, 0.145, 80.0)
    c = [[0.0, 0.0, 0.0], [60.0, 0.0, 0.0]]
    for k in (0.0, kD):
        e = S.SphereSystem(c, [2.0, 1.5], [1.0, -0.7], 2.0, 80.0, k, lB, L=8).solve()["energy"]
        born = sum(0.5 * q * q * lB / R * (1.0 / (80.0 * (1.0 + k * R)) - 1.0 / 2.0)
                   for R, q in ((2.0, 1.0), (1.5, -0.7)))
        # Debye-Hueckel interaction of two ions of radii R1, R2 at distance d
        d = 60.0
        inter = (1.0 * -0.7 * lB / (80.0 * d) * np.exp(-k * (d - 3.5)) /
                 ((1.0 + k * 2.0) * (1.0 + k * 1.5)))
        assert abs(e - (born + inter)) < 2e-5 * abs(born)


@pytest.mark.parametrize("I,bc,tol", [(0.0, "coulomb", 3e-4), (0.145, "dh", 1e-3)])
def test_box_method_energies_match_the_analytic_ones(S, orc, I, bc, tol):
    lB, kD = orc.units(298.15, I, 80.0)
    exact = S.SphereSystem(C3, R3, Q3, 2.0, 80.0, kD, lB, L=20).solve()["energy"]
    atoms = np.column_stack([C3, R3, Q3])
    cen = 0.5 * ((C3 - R3[:, None]).min(0) + (C3 + R3[:, None]).max(0))
    for h in (0.5, 0.4):
        n = int(round(28.0 / h)) + 1
        g = orc.Grid((n, n, n), cen - 0.5 * (n - 1) * h, h)
        r = orc.solve_problem(atoms, g, eps_in=2.0, eps_out=80.0, ionic_strength_M=I,
                              bc=orc.BC_COULOMB if bc == "coulomb" else orc.BC_DH, rtol=1e-10)
        e = r["energy"]
        got = e["e_coul"] + e["e_pol"] if I == 0.0 else e["e_total"]
        assert abs(got - exact) <= tol * abs(exact), (h, got, exact)
