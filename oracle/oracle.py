"""ctypes shim around the FP64 CPU oracle (``pb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  Nothing here imports the CUDA library;
all arithmetic of the method lives in ``pb_oracle.c`` and this file only
marshals numpy arrays and chains the C functions in the order of the paper:
placement -> classification -> crossing edges -> coefficients (Sec. 3.1-3.2)
-> boundary values (Sec. 2.3) -> right-hand side (Eq. RVop) -> Jacobi-PCG ->
energy terms (Sec. 3.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_ZERO, BC_COULOMB, BC_DH = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no FMA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared",
                               "-ffp-contract=off", "-fno-fast-math",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            P = C.c_void_p
            L.orc_units.argtypes = [C.c_double, C.c_double, C.c_double, P, P]
            L.orc_place_grid.argtypes = [P, C.c_long, C.c_int, C.c_double, P, P]
            L.orc_classify.argtypes = [P, P, C.c_double, P, C.c_long, P]
            L.orc_classify_nodes.argtypes = [P, P, C.c_double, P, C.c_long, P, C.c_long, P]
            L.orc_edge_alpha.argtypes = [P, P, C.c_double, P, C.c_long, P, C.c_long, P]
            L.orc_crossing_edges.argtypes = [P, P, C.c_double, P, C.c_long, P, C.c_long, P, P, P, P]
            L.orc_crossing_edges.restype = C.c_long
            L.orc_assemble.argtypes = [P, C.c_double, P, C.c_long, P, P, C.c_double,
                                       C.c_double, C.c_double, P, P, P, P, P]
            L.orc_bc_values.argtypes = [P, P, C.c_double, P, C.c_long, C.c_double,
                                        C.c_double, C.c_double, P]
            L.orc_rhs.argtypes = [P, P, C.c_double, P, C.c_long, C.c_double, P, P, P, P, P]
            L.orc_rhs.restype = C.c_int
            L.orc_apply.argtypes = [P, P, P, P, P, P, P]
            L.orc_pcg.argtypes = [P, P, P, P, P, P, C.c_double, C.c_long, P, P, P]
            L.orc_pcg.restype = C.c_int
            L.orc_coulomb_phi.argtypes = [P, C.c_long, P, C.c_long, C.c_double, P]
            L.orc_coulomb_psi.argtypes = [P, P, P, C.c_long, P, C.c_long, P]
            L.orc_ecoul.argtypes = [P, C.c_long, C.c_double, C.c_double]
            L.orc_ecoul.restype = C.c_double
            L.orc_energy.argtypes = [P, P, C.c_double, P, C.c_long, P, P, P, P, P, P, P,
                                     P, P, C.c_long, C.c_double, C.c_double, C.c_double, P]
            L.orc_node_coeffs.argtypes = [P, P, C.c_double, P, C.c_long, C.c_double,
                                          C.c_double, C.c_double, P, C.c_long, P]
            L.orc_mc_weights.argtypes = [P, P, C.c_long, P, P, P]
            L.orc_mc_normals.argtypes = [C.c_long, P, P, P, C.c_long, P]
            L.orc_coulomb_psi_n.argtypes = [P, P, C.c_long, P, C.c_long, P]
            L.orc_energy_ion_mc.argtypes = [P, C.c_long, P, P, P, P, P, P, P, P, C.c_long,
                                            C.c_double, C.c_double]
            L.orc_energy_ion_mc.restype = C.c_double
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def units(temperature_K: float = 298.15, ionic_strength_M: float = 0.145,
          eps_out: float = 80.0) -> tuple[float, float]:
    """(l_B in A, k_D in 1/A)."""
    lb = C.c_double()
    kd = C.c_double()
    lib().orc_units(temperature_K, ionic_strength_M, eps_out, C.byref(lb), C.byref(kd))
    return lb.value, kd.value


class Grid:
    """Uniform grid: ``n`` = (nx, ny, nz), ``origin`` (3,), spacing ``h``."""

    def __init__(self, n, origin, h):
        self.n = np.ascontiguousarray(n, dtype=np.int32).reshape(3)
        self.origin = _f64(origin).reshape(3)
        self.h = float(h)

    @property
    def N(self) -> int:
        return int(np.prod(self.n.astype(np.int64)))

    def shape_zyx(self):
        return (int(self.n[2]), int(self.n[1]), int(self.n[0]))


def place_grid(atoms: np.ndarray, n: int, fill: float) -> Grid:
    atoms = _f64(atoms)
    o = np.zeros(3)
    h = C.c_double()
    lib().orc_place_grid(_p(atoms), len(atoms), int(n), float(fill), _p(o), C.byref(h))
    return Grid((n, n, n), o, h.value)


def classify(g: Grid, atoms: np.ndarray) -> np.ndarray:
    atoms = _f64(atoms)
    out = np.empty(g.N, dtype=np.uint8)
    lib().orc_classify(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms), _p(out))
    return out


def classify_nodes(g: Grid, atoms: np.ndarray, nodes) -> np.ndarray:
    atoms = _f64(atoms)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty(len(nodes), dtype=np.uint8)
    lib().orc_classify_nodes(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms),
                             _p(nodes), len(nodes), _p(out))
    return out


def edge_alpha(g: Grid, atoms: np.ndarray, ids) -> np.ndarray:
    atoms = _f64(atoms)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty(len(ids))
    lib().orc_edge_alpha(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms),
                         _p(ids), len(ids), _p(out))
    return out


def crossing_edges(g: Grid, atoms: np.ndarray, inside: np.ndarray) -> dict:
    atoms = _f64(atoms)
    inside = np.ascontiguousarray(inside, dtype=np.uint8)
    L = lib()
    args = (_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms), _p(inside))
    cap = 0
    dummy = np.zeros(1, dtype=np.int64)
    cnt = L.orc_crossing_edges(*args, cap, _p(dummy), _p(dummy), _p(dummy), _p(dummy))
    ids = np.empty(cnt, dtype=np.int64)
    alpha = np.empty(cnt)
    rp = np.empty((cnt, 3))
    sign = np.empty(cnt, dtype=np.int8)
    L.orc_crossing_edges(*args, cnt, _p(ids), _p(alpha), _p(rp), _p(sign))
    return {"ids": ids, "alpha": alpha, "rp": rp, "sign": sign}


def assemble(g: Grid, inside, cross, eps_in, eps_out, kD) -> dict:
    N = g.N
    W = [np.empty(N) for _ in range(3)]
    kap = np.empty(N)
    diag = np.empty(N)
    lib().orc_assemble(_p(g.n), g.h, _p(np.ascontiguousarray(inside, dtype=np.uint8)),
                       len(cross["ids"]), _p(cross["ids"]), _p(cross["alpha"]),
                       float(eps_in), float(eps_out), float(kD),
                       _p(W[0]), _p(W[1]), _p(W[2]), _p(kap), _p(diag))
    return {"Wx": W[0], "Wy": W[1], "Wz": W[2], "kap": kap, "diag": diag}


def bc_values(g: Grid, atoms, lB, eps_out, bc: int, kD: float) -> np.ndarray:
    out = np.zeros(g.N)
    if bc == BC_ZERO:
        return out
    k = 0.0 if bc == BC_COULOMB else float(kD)
    atoms = _f64(atoms)
    lib().orc_bc_values(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms),
                        float(lB), float(eps_out), k, _p(out))
    return out


def rhs(g: Grid, atoms, lB, coef: dict, phib) -> np.ndarray:
    atoms = _f64(atoms)
    f = np.empty(g.N)
    st = lib().orc_rhs(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms), float(lB),
                       _p(coef["Wx"]), _p(coef["Wy"]), _p(coef["Wz"]), _p(_f64(phib)), _p(f))
    if st != 0:
        raise ValueError("a charge lies in a cell that touches the box boundary")
    return f


def apply(g: Grid, coef: dict, x) -> np.ndarray:
    x = _f64(x).reshape(-1)
    y = np.empty(g.N)
    lib().orc_apply(_p(g.n), _p(coef["Wx"]), _p(coef["Wy"]), _p(coef["Wz"]),
                    _p(coef["diag"]), _p(x), _p(y))
    return y


def pcg(g: Grid, coef: dict, f, rtol: float, max_iter: int = 100000):
    """Returns (x, iters, true relative residual, converged)."""
    f = _f64(f)
    x = np.empty(g.N)
    it = C.c_long()
    rel = C.c_double()
    st = lib().orc_pcg(_p(g.n), _p(coef["Wx"]), _p(coef["Wy"]), _p(coef["Wz"]),
                       _p(coef["diag"]), _p(f), float(rtol), int(max_iter), _p(x),
                       C.byref(it), C.byref(rel))
    return x, it.value, rel.value, st == 0


def coulomb_phi(targets, atoms, k: float = 0.0) -> np.ndarray:
    t = _f64(targets).reshape(-1, 3)
    atoms = _f64(atoms)
    out = np.empty(len(t))
    lib().orc_coulomb_phi(_p(t), len(t), _p(atoms), len(atoms), float(k), _p(out))
    return out


def coulomb_psi(targets, dirs, signs, atoms) -> np.ndarray:
    t = _f64(targets).reshape(-1, 3)
    atoms = _f64(atoms)
    d = np.ascontiguousarray(dirs, dtype=np.int8)
    s = np.ascontiguousarray(signs, dtype=np.int8)
    out = np.empty(len(t))
    lib().orc_coulomb_psi(_p(t), _p(d), _p(s), len(t), _p(atoms), len(atoms), _p(out))
    return out


def ecoul(atoms, lB, eps_in) -> float:
    atoms = _f64(atoms)
    return lib().orc_ecoul(_p(atoms), len(atoms), float(lB), float(eps_in))


ENERGY_KEYS = ("e_coul", "e_pol", "e_ion_surf", "e_ion_flux", "e_total", "flux_charge")


def energy(g: Grid, inside, cross, coef, phi, atoms, lB, eps_in, eps_out) -> dict:
    atoms = _f64(atoms)
    out = np.empty(6)
    lib().orc_energy(_p(g.n), _p(g.origin), g.h, _p(np.ascontiguousarray(inside, dtype=np.uint8)),
                     len(cross["ids"]), _p(cross["ids"]), _p(cross["alpha"]),
                     _p(np.ascontiguousarray(cross["rp"])), _p(cross["sign"]),
                     _p(coef["Wx"]), _p(coef["Wy"]), _p(coef["Wz"]), _p(_f64(phi)),
                     _p(atoms), len(atoms), float(lB), float(eps_in), float(eps_out), _p(out))
    return dict(zip(ENERGY_KEYS, out.tolist()))


def mc_weights(g: Grid, inside, cross) -> np.ndarray:
    """Vertex weights (sum of T_j/3 over the marching-cubes triangles at each
    crossing point) of the re-triangulated surface (Sec. 3.3.2)."""
    out = np.empty(len(cross["ids"]))
    lib().orc_mc_weights(_p(g.n), _p(np.ascontiguousarray(inside, dtype=np.uint8)),
                         len(cross["ids"]), _p(cross["ids"]),
                         _p(np.ascontiguousarray(cross["rp"])), _p(out))
    return out


def mc_normals(cross, atoms) -> np.ndarray:
    """Analytic outward unit normal of the ball surface at each crossing
    point (zero where the edge's ends lie in the same medium)."""
    atoms = _f64(atoms)
    out = np.empty((len(cross["ids"]), 3))
    lib().orc_mc_normals(len(cross["ids"]), _p(np.ascontiguousarray(cross["rp"])),
                         _p(cross["sign"]), _p(atoms), len(atoms), _p(out))
    return out


def coulomb_psi_n(targets, normals, atoms) -> np.ndarray:
    t = _f64(targets).reshape(-1, 3)
    nv = _f64(normals).reshape(-1, 3)
    atoms = _f64(atoms)
    out = np.empty(len(t))
    lib().orc_coulomb_psi_n(_p(t), _p(nv), len(t), _p(atoms), len(atoms), _p(out))
    return out


def energy_ion_mc(g: Grid, cross, W, normals, phi, atoms, eps_in, eps_out) -> float:
    """First integral of Eq. energy_ion on the re-triangulated surface (kT)."""
    atoms = _f64(atoms)
    return lib().orc_energy_ion_mc(_p(g.n), len(cross["ids"]), _p(cross["ids"]),
                                   _p(cross["alpha"]), _p(np.ascontiguousarray(cross["rp"])),
                                   _p(cross["sign"]), _p(_f64(W)), _p(_f64(normals)),
                                   _p(_f64(phi)), _p(atoms), len(atoms), float(eps_in),
                                   float(eps_out))


def node_coeffs(g: Grid, atoms, eps_in, eps_out, kD, nodes) -> np.ndarray:
    """(count, 8): W(-x), W(+x), W(-y), W(+y), W(-z), W(+z), kappa h^3, diag."""
    atoms = _f64(atoms)
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    out = np.empty((len(nodes), 8))
    lib().orc_node_coeffs(_p(g.n), _p(g.origin), g.h, _p(atoms), len(atoms), float(eps_in),
                          float(eps_out), float(kD), _p(nodes), len(nodes), _p(out))
    return out


def solve_problem(atoms, grid: Grid, eps_in=2.0, eps_out=80.0, ionic_strength_M=0.145,
                  temperature_K=298.15, bc=BC_ZERO, rtol=1e-10, max_iter=200000,
                  with_energy=True) -> dict:
    """Whole pipeline in the paper's order; returns every intermediate."""
    atoms = _f64(atoms)
    lB, kD = units(temperature_K, ionic_strength_M, eps_out)
    inside = classify(grid, atoms)
    cross = crossing_edges(grid, atoms, inside)
    coef = assemble(grid, inside, cross, eps_in, eps_out, kD)
    phib = bc_values(grid, atoms, lB, eps_out, bc, kD)
    f = rhs(grid, atoms, lB, coef, phib)
    x, iters, rel, conv = pcg(grid, coef, f, rtol, max_iter)
    phi = x + phib
    res = {"grid": grid, "lB": lB, "kD": kD, "inside": inside, "cross": cross,
           "coef": coef, "phib": phib, "f": f, "x": x, "phi": phi, "iters": iters,
           "relres": rel, "converged": conv}
    if with_energy:
        res["energy"] = energy(grid, inside, cross, coef, phi, atoms, lB, eps_in, eps_out)
        W = mc_weights(grid, inside, cross)
        nrm = mc_normals(cross, atoms)
        res["mc"] = {"W": W, "normals": nrm}
        res["energy"]["e_ion_mc"] = energy_ion_mc(grid, cross, W, nrm, phi, atoms, eps_in,
                                                  eps_out)
    return res
