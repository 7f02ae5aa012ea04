"""A single solve split into z-slabs over gloo ranks (CPU, no GPU), against
the single-process oracle.

Each rank owns a range of interior planes, exchanges one boundary plane with
each neighbour before every operator application and joins every inner
product.  With the chained reduction order the split run must reproduce the
oracle's iterate, iteration count and residual bit for bit (a missing or
misplaced halo plane, or a sum taken in another order, breaks that); with
rank-order partials every rank must agree to the bit and the solution must
agree with the oracle's to rounding."""
import os
import socket

import numpy as np
import pytest

import pb_inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, n, coef, f, order, rtol, q):
    import sys

    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import slab
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = slab.Slab(n, coef, rank, world, order)
    x, it, rel, conv = s.pcg(f, rtol)
    # the same scalar on every rank: gather every rank's view of one sum
    mine = torch.tensor([s.dot(x, x)], dtype=torch.float64)
    views = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(views, mine)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, s.k0, s.k1, x, it, rel, conv, [float(v[0]) for v in views]))


def _run(world, n, coef, f, order, rtol):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, n, coef, f, order, rtol, q))
             for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


@pytest.fixture(scope="module")
def problem(orc):
    """A small molecule on a non-cubic grid with Debye-Hueckel boundary values
    (every coefficient kind present: solute, solvent, listed edges, lift)."""
    atoms = pb_inputs.globular_molecule(24, seed=31)
    h = 0.45
    lo = (atoms[:, :3] - atoms[:, 3:4]).min(0) - 2.0
    ext = (atoms[:, :3] + atoms[:, 3:4]).max(0) + 2.0 - lo
    n = tuple(int(np.ceil(e / h)) + 2 for e in ext)
    n = (n[0], n[1] + 1, n[2] + 3)
    g = orc.Grid(n, lo, h)
    ref = orc.solve_problem(atoms, g, bc=orc.BC_DH, rtol=1e-11, with_energy=False)
    assert ref["converged"]
    return g, ref


def test_slab_ranges():
    from oracle import slab
    for nz, world in ((5, 1), (5, 3), (23, 2), (23, 3), (24, 4), (40, 7)):
        rs = slab.slab_ranges(nz, world)
        assert rs[0][0] == 1 and rs[-1][1] == nz - 1
        assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
        sizes = [k1 - k0 for k0, k1 in rs]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        slab.slab_ranges(5, 4)


def _assemble(g, parts):
    nx, ny, nz = (int(v) for v in g.n)
    x = np.zeros((nz, ny, nx))
    for _, k0, k1, xl, *_ in parts:
        x[k0:k1] = xl
    return x.reshape(-1)


@pytest.mark.parametrize("world", [2, 3])
def test_chain_order_is_the_oracle_bit_for_bit(problem, world):
    g, ref = problem
    parts = _run(world, tuple(int(v) for v in g.n), ref["coef"], ref["f"], "chain", 1e-11)
    x = _assemble(g, parts)
    assert np.array_equal(x, ref["x"])
    for _, _, _, _, it, rel, conv, views in parts:
        assert conv and it == ref["iters"] and rel == ref["relres"]
        assert len(set(views)) == 1


def test_rank_order_partials(problem):
    g, ref = problem
    world = 3
    parts = _run(world, tuple(int(v) for v in g.n), ref["coef"], ref["f"], "rank", 1e-11)
    x = _assemble(g, parts)
    its = {p[4] for p in parts}
    assert len(its) == 1  # every rank took the same decisions
    for p in parts:
        assert p[6] and p[5] <= 1e-11 and len(set(p[7])) == 1
    assert np.max(np.abs(x - ref["x"])) <= 1e-9 * np.max(np.abs(ref["x"]))
