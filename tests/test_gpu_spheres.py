"""The CUDA path against the paper's analytical benchmark: three close
dielectric spheres with central charges (oracle/spheres.py, multipole
expansion).  Mixed-precision solves to a true residual of 1e-10 on a 0.4 A
grid give the analytic energies within the discretisation bars the oracle
meets: 3e-4 without salt (E_coul + E_pol), 1e-3 in 0.145 M salt (E_total,
staircase ionic surface term included)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C3 = np.array([[0.0, 0.0, 0.0], [4.6, 0.4, -0.3], [1.9, 3.9, 1.1]])
R3 = np.array([2.0, 1.6, 1.4])
Q3 = np.array([1.0, -1.0, 0.6])


@pytest.fixture(scope="module")
def pb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_09323_gb300 import build
    build.build()
    import paper_2502_09323_gb300 as pb
    return pb


@pytest.mark.parametrize("I,tol", [(0.0, 3e-4), (0.145, 1e-3)])
def test_energies_match_the_analytic_spheres(pb, orc, I, tol):
    from oracle import spheres
    lB, kD = orc.units(298.15, I, 80.0)
    exact = spheres.SphereSystem(C3, R3, Q3, 2.0, 80.0, kD, lB, L=20).solve()["energy"]
    atoms = np.column_stack([C3, R3, Q3])
    cen = 0.5 * ((C3 - R3[:, None]).min(0) + (C3 + R3[:, None]).max(0))
    h, n = 0.4, 71
    spec = pb.GridSpec(n=(n, n, n), origin=tuple(float(v) for v in cen - 0.5 * (n - 1) * h), h=h)
    params = pb.Params(eps_in=2.0, eps_out=80.0, ionic_strength_M=I,
                       bc=pb.BC_COULOMB if I == 0.0 else pb.BC_DH)
    out = pb.solve_molecule(atoms, spec=spec, params=params,
                            opts=pb.SolveOpts(precision=pb.MIXED, rtol=1e-10))
    assert out["stats"]["status"] == 0
    e = out["energy"]
    got = e["e_coul"] + e["e_pol"] if I == 0.0 else e["e_total"]
    assert abs(got - exact) <= tol * abs(exact), (got, exact)
    out["system"].free()
