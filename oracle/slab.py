"""Slab decomposition of the oracle's Jacobi-PCG over several processes.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the tests import it.
It checks the exchange and reduction steps that a solve sharded across
devices needs, against the single-process oracle.

The paper assembles and solves its linear systems in distributed memory
(Sec. Software Architecture).  Here P ranks each own a contiguous range of
interior z-planes of the uniform grid and run the oracle's Jacobi-PCG with
true-residual restarts (``oracle.pcg``, the operator of Sec. 3.1) on them:

* the operator on a rank's planes reads one plane of its operand from each
  neighbouring rank, exchanged before every application (``exchange``);
* an inner product is formed in one of two orders:
  - ``"chain"``: the oracle's own order, one sequential sum over the interior
    nodes in (k, j, i) order; rank r continues the running sum it receives
    from rank r - 1 and hands it on, and the last rank broadcasts the total.
    Every rank's part of the iterate then equals the single-process
    oracle's, bit for bit.
  - ``"rank"``: each rank sums its own nodes in that order and the partials
    are added in rank order, as a sharded GPU solve would do; every rank
    gets the same bits, and the result agrees with the single-process one
    up to rounding.

Arrays are numpy float64 in (z, y, x) order; the communicator is a
``torch.distributed`` process group (gloo on the host).
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.distributed as dist


def slab_ranges(nz: int, world: int) -> list[tuple[int, int]]:
    """Interior planes 1 .. nz-2 split into ``world`` contiguous ranges
    [k0, k1) whose lengths differ by at most one (the first ranks take the
    extra planes)."""
    m = nz - 2
    if world < 1 or world > m:
        raise ValueError("need 1 <= world <= number of interior planes")
    base, extra = divmod(m, world)
    out, k = [], 1
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((k, k + n))
        k += n
    return out


class Slab:
    """One rank's share: planes [k0, k1) of the coefficient arrays, with one
    plane of the neighbours' below and above where the operator needs it."""

    def __init__(self, n, coef: dict, rank: int, world: int, order: str = "chain"):
        self.nx, self.ny, self.nz = (int(v) for v in n)
        self.rank, self.world = rank, world
        if order not in ("chain", "rank"):
            raise ValueError("order must be 'chain' or 'rank'")
        self.order = order
        self.k0, self.k1 = slab_ranges(self.nz, world)[rank]
        shp = (self.nz, self.ny, self.nx)
        sl = slice(self.k0, self.k1)
        below = slice(self.k0 - 1, self.k1)  # the -z faces of plane k0 sit on plane k0 - 1
        self.Wx = coef["Wx"].reshape(shp)[sl]
        self.Wy = coef["Wy"].reshape(shp)[sl]
        self.Wz = coef["Wz"].reshape(shp)[below]
        self.diag = coef["diag"].reshape(shp)[sl]
        m = self.k1 - self.k0
        self.inside = np.zeros((m, self.ny, self.nx), dtype=bool)
        self.inside[:, 1:-1, 1:-1] = True

    # ----------------------------------------------------------- exchange
    def exchange(self, v: np.ndarray) -> np.ndarray:
        """v on the own planes -> v on planes k0-1 .. k1 (the global boundary
        planes are zero: the unknowns vanish there)."""
        m = v.shape[0]
        ext = np.zeros((m + 2, self.ny, self.nx))
        ext[1:-1] = v
        ops, keep = [], []
        lo = torch.zeros(self.ny * self.nx, dtype=torch.float64)
        hi = torch.zeros(self.ny * self.nx, dtype=torch.float64)
        if self.rank > 0:
            keep.append(torch.from_numpy(np.ascontiguousarray(v[0]).reshape(-1)))
            ops.append(dist.isend(keep[-1], self.rank - 1))
            ops.append(dist.irecv(lo, self.rank - 1))
        if self.rank < self.world - 1:
            keep.append(torch.from_numpy(np.ascontiguousarray(v[-1]).reshape(-1)))
            ops.append(dist.isend(keep[-1], self.rank + 1))
            ops.append(dist.irecv(hi, self.rank + 1))
        for op in ops:
            op.wait()
        if self.rank > 0:
            ext[0] = lo.numpy().reshape(self.ny, self.nx)
        if self.rank < self.world - 1:
            ext[-1] = hi.numpy().reshape(self.ny, self.nx)
        return ext

    # -------------------------------------------------------------- apply
    def apply(self, v: np.ndarray) -> np.ndarray:
        """(A v) on the own planes, term by term in the oracle's order:
        s = 0, then the -x, +x, -y, +y, -z, +z couplings (each skipped next
        to the box boundary), y = diag v - s; zero on boundary nodes."""
        e = self.exchange(v)
        c = e[1:-1]
        nx, ny, nz = self.nx, self.ny, self.nz
        k = np.arange(self.k0, self.k1)[:, None, None]
        j = np.arange(ny)[None, :, None]
        i = np.arange(nx)[None, None, :]
        s = np.zeros_like(c)
        xm = np.zeros_like(c)
        xm[:, :, 1:] = self.Wx[:, :, :-1] * c[:, :, :-1]
        s = np.where(i > 1, s + xm, s)
        xp = np.zeros_like(c)
        xp[:, :, :-1] = self.Wx[:, :, :-1] * c[:, :, 1:]
        s = np.where(i < nx - 2, s + xp, s)
        ym = np.zeros_like(c)
        ym[:, 1:, :] = self.Wy[:, :-1, :] * c[:, :-1, :]
        s = np.where(j > 1, s + ym, s)
        yp = np.zeros_like(c)
        yp[:, :-1, :] = self.Wy[:, :-1, :] * c[:, 1:, :]
        s = np.where(j < ny - 2, s + yp, s)
        zm = self.Wz[:-1] * e[:-2]
        s = np.where(k > 1, s + zm, s)
        zp = self.Wz[1:] * e[2:]
        s = np.where(k < nz - 2, s + zp, s)
        y = self.diag * c - s
        return np.where(self.inside, y, 0.0)

    # ---------------------------------------------------------------- dot
    def _seq(self, start: float, u: np.ndarray, v: np.ndarray) -> float:
        """start + u0 v0 + u1 v1 + ... over the interior nodes, left to right."""
        prod = (u * v)[self.inside]
        acc = np.add.accumulate(np.concatenate(([start], prod)))
        return float(acc[-1])

    def dot(self, u: np.ndarray, v: np.ndarray) -> float:
        buf = torch.zeros(1, dtype=torch.float64)
        if self.order == "chain":
            start = 0.0
            if self.rank > 0:
                dist.recv(buf, self.rank - 1)
                start = float(buf[0])
            total = self._seq(start, u, v)
            buf[0] = total
            if self.rank < self.world - 1:
                dist.send(buf, self.rank + 1)
            dist.broadcast(buf, self.world - 1)
            return float(buf[0])
        parts = [torch.zeros(1, dtype=torch.float64) for _ in range(self.world)]
        dist.all_gather(parts, torch.tensor([self._seq(0.0, u, v)], dtype=torch.float64))
        total = 0.0
        for p in parts:
            total += float(p[0])
        return total

    # ---------------------------------------------------------------- pcg
    def pcg(self, f: np.ndarray, rtol: float, max_iter: int = 100000):
        """The oracle's Jacobi-PCG on this rank's planes of f (zero initial
        guess, restart from the true residual whenever the recursive one
        passes the test).  Returns (x on the own planes, iterations, true
        relative residual, converged)."""
        shp = (self.nz, self.ny, self.nx)
        fl = np.where(self.inside, f.reshape(shp)[self.k0:self.k1], 0.0)
        x = np.zeros_like(fl)
        fnorm = math.sqrt(self.dot(fl, fl))
        it, rel = 0, 0.0
        if fnorm == 0.0:
            return x, 0, 0.0, True
        r = fl.copy()
        while True:
            z = np.where(self.inside, r / self.diag, 0.0)
            p = z.copy()
            rho = self.dot(r, z)
            restart = False
            while it < max_iter:
                q = self.apply(p)
                sigma = self.dot(p, q)
                al = rho / sigma
                x = np.where(self.inside, x + al * p, x)
                r = np.where(self.inside, r - al * q, r)
                it += 1
                rn = math.sqrt(self.dot(r, r))
                if rn <= rtol * fnorm:
                    q = self.apply(x)
                    r = np.where(self.inside, fl - q, 0.0)
                    rel = math.sqrt(self.dot(r, r)) / fnorm
                    if rel <= rtol:
                        return x, it, rel, True
                    restart = True
                    break
                z = np.where(self.inside, r / self.diag, 0.0)
                rho1 = self.dot(r, z)
                be = rho1 / rho
                rho = rho1
                p = z + be * p
            if not restart:
                break
        q = self.apply(x)
        r = np.where(self.inside, fl - q, 0.0)
        rel = math.sqrt(self.dot(r, r)) / fnorm
        return x, it, rel, False
