"""Analytic electrostatics of non-overlapping dielectric spheres (the paper's
analytical benchmark, Sec. An analytical benchmark).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests import it.
It pins the discretisation itself (finite differences on the box-method
grid), where the other pins reach the discrete system.

N_s spheres of radius R_i, permittivity eps_in, a point charge q_i at each
centre, in a solvent of permittivity eps_out with inverse Debye length k_D
(k_D = 0: pure dielectric).  In reduced units (potential in kT/e, lengths in
A, l_B the vacuum Bjerrum length) the potential is, per Eq.
potential_total_selfconsist_ and Eq. Lin_pbe_phi_in_out:

* inside sphere i:  l_B q_i / (eps_in r_i) + sum_{n,m} A_{i,nm} r_i^n Y_nm
* in the solvent:   sum_j sum_{n,m} B_{j,nm} k_n(k_D r_j) / k_n(k_D R_j) Y_nm   (k_D > 0)
                    sum_j sum_{n,m} B_{j,nm} (R_j / r_j)^(n+1) Y_nm             (k_D = 0)

with r_j, Y_nm taken about centre j (real orthonormal spherical harmonics,
n <= L).  On each sphere the potential and eps times its normal derivative
are continuous.  The field of the other spheres is re-expanded about centre
i by projecting its values on sphere i onto Y_nm (Gauss-Legendre in cos
theta, uniform in phi): it is regular inside the ball that reaches the
nearest other sphere, so the projection converges like (R_i / gap
distance)^n.  The radial factors it carries inside that ball are r^n (k_D =
0) or i_n(k_D r) (k_D > 0).  The interface conditions then give B_i in terms
of that external part, one linear system for all B.

The total electrostatic energy is E = 1/2 sum_i q_i (phi_i(c_i) - own
Coulomb term), as in the paper: 1/2 sum_i q_i A_{i,00} Y_00.  It equals
E_coul + E_pol + E_ion of the energy partition (Sec. 3.3).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special as sp


def _real_ylm(L: int, theta: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonics, rows (n, m) for n <= L in the
    order (0,0), (1,-1), (1,0), (1,1), ...; columns the points.  Built from
    the associated Legendre functions: sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!)
    P_n^|m|(cos theta), times sqrt(2) cos(m phi) for m > 0 and sqrt(2)
    sin(|m| phi) for m < 0."""
    x = np.cos(theta)
    out = np.empty(((L + 1) ** 2, theta.size))
    row = 0
    for n in range(L + 1):
        for m in range(-n, n + 1):
            am = abs(m)
            norm = math.sqrt((2 * n + 1) / (4.0 * math.pi) *
                             math.exp(math.lgamma(n - am + 1) - math.lgamma(n + am + 1)))
            p = sp.lpmv(am, n, x)
            if m > 0:
                out[row] = math.sqrt(2.0) * norm * p * np.cos(am * phi)
            elif m < 0:
                out[row] = math.sqrt(2.0) * norm * p * np.sin(am * phi)
            else:
                out[row] = norm * p
            row += 1
    return out


def _degrees(L: int) -> np.ndarray:
    return np.concatenate([np.full(2 * n + 1, n) for n in range(L + 1)])


class SphereSystem:
    def __init__(self, centers, radii, charges, eps_in: float, eps_out: float, kD: float,
                 lB: float, L: int = 20, quad: int | None = None):
        self.c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        self.R = np.asarray(radii, dtype=np.float64).reshape(-1)
        self.q = np.asarray(charges, dtype=np.float64).reshape(-1)
        self.ns = len(self.R)
        for i in range(self.ns):
            for j in range(i + 1, self.ns):
                if np.linalg.norm(self.c[i] - self.c[j]) <= self.R[i] + self.R[j]:
                    raise ValueError("spheres overlap")
        self.ei, self.eo, self.kD, self.lB, self.L = eps_in, eps_out, kD, lB, L
        nq = quad or (L + 24)
        x, w = np.polynomial.legendre.leggauss(nq)
        ph = 2.0 * math.pi * np.arange(2 * nq) / (2 * nq)
        T, P = np.meshgrid(np.arccos(x), ph, indexing="ij")
        W = np.outer(w, np.full(2 * nq, 2.0 * math.pi / (2 * nq)))
        self.dirs = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
        self.w = W.reshape(-1)
        self.Yq = _real_ylm(L, T.reshape(-1), P.reshape(-1))
        self.deg = _degrees(L)

    # radial factors of the solvent field of sphere j: outgoing g_n, scaled
    # to 1 on that sphere's surface (k_n(k_D r) spans many decades in n, so
    # unscaled modes lose every digit past n ~ 16)
    def _g(self, n, r, Rj):
        if self.kD == 0.0:
            return (Rj / r) ** (n + 1.0)
        return sp.spherical_kn(n, self.kD * r) / sp.spherical_kn(n, self.kD * Rj)

    def _g_log_derivative(self, n, R):
        """g_n'(R) / g_n(R) on the sphere's own surface."""
        if self.kD == 0.0:
            return -(n + 1.0) / R
        return self.kD * sp.spherical_kn(n, self.kD * R, derivative=True) / sp.spherical_kn(
            n, self.kD * R)

    def _h_log_derivative(self, n, R):
        """h_n'(R) / h_n(R) for the regular factor (r^n or i_n(k_D r))."""
        if self.kD == 0.0:
            return n / R
        return self.kD * sp.spherical_in(n, self.kD * R, derivative=True) / sp.spherical_in(
            n, self.kD * R)

    def _field_at(self, j: int, pts: np.ndarray) -> np.ndarray:
        """Values at pts of the unit solvent modes of sphere j: rows (n, m)."""
        d = pts - self.c[j]
        r = np.linalg.norm(d, axis=1)
        th = np.arccos(np.clip(d[:, 2] / r, -1.0, 1.0))
        ph = np.arctan2(d[:, 1], d[:, 0])
        Y = _real_ylm(self.L, th, ph)
        rad = np.stack([self._g(n, r, self.R[j]) for n in range(self.L + 1)])
        return Y * rad[self.deg]

    def solve(self) -> dict:
        ns, K = self.ns, (self.L + 1) ** 2
        n = self.deg.astype(np.float64)
        # external part on sphere i, per unit B_j: M[i][j] (K x K)
        M = np.zeros((ns * K, ns * K))
        for i in range(ns):
            pts = self.c[i] + self.R[i] * self.dirs
            proj = self.Yq * self.w  # (K, Q)
            for j in range(ns):
                if j == i:
                    continue
                F = self._field_at(j, pts)  # (K_j, Q)
                M[i * K:(i + 1) * K, j * K:(j + 1) * K] = proj @ F.T
        # interface conditions: B_i = a_i * C_i + b_i, C_i = sum_j M_ij B_j
        a = np.empty(ns * K)
        b = np.zeros(ns * K)
        Q = [self.lB * qi * math.sqrt(4.0 * math.pi) / self.ei for qi in self.q]
        for i in range(ns):
            R = self.R[i]
            # g_n(R) = 1 on the sphere's own surface
            dg = np.array([self._g_log_derivative(k, R) for k in range(self.L + 1)])[self.deg]
            eta = np.array([self._h_log_derivative(k, R) for k in range(self.L + 1)])[self.deg]
            den = self.ei * (n / R) - self.eo * dg
            a[i * K:(i + 1) * K] = (self.eo * eta - self.ei * n / R) / den
            b[i * K] = self.ei * Q[i] / R ** 2 / den[0]
        A_sys = np.eye(ns * K) - a[:, None] * M
        B = np.linalg.solve(A_sys, b)
        C = M @ B
        # inside coefficients from continuity (g_n(R) = 1): A R^n = B + C - delta_n0 Q / R
        energy = 0.0
        coef_in = np.empty(ns * K)
        for i in range(ns):
            R = self.R[i]
            sl = slice(i * K, (i + 1) * K)
            val = B[sl] + C[sl]
            val[0] -= Q[i] / R
            coef_in[sl] = val / R ** n
            energy += 0.5 * self.q[i] * coef_in[i * K] / math.sqrt(4.0 * math.pi)
        return {"energy": energy, "B": B, "A": coef_in}


def coulomb_energy(centers, charges, eps_in: float, lB: float) -> float:
    """(l_B / eps_in) sum_{i<j} q_i q_j / r_ij."""
    c = np.asarray(centers, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(charges, dtype=np.float64)
    e = 0.0
    for i in range(len(q)):
        for j in range(i + 1, len(q)):
            e += q[i] * q[j] / np.linalg.norm(c[i] - c[j])
    return lB / eps_in * e
