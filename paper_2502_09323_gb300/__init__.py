"""Python binding of libpbgpu, the GB300 linear Poisson-Boltzmann hot path.

The functions ``pb_build_grid``, ``pb_assemble_coeffs``, ``pb_coulomb_terms``,
``pb_solve``, ``pb_energy``, ``pb_get_array``, ``pb_apply`` and
``pb_solve_batch`` have the names and meaning of the C ABI in
``include/pb.h``; this module only marshals arguments (numpy / torch tensors,
the current torch CUDA stream) and owns the returned handles.  Every step of
the computation runs in the CUDA library; if the library is missing this
module raises instead of computing anything itself.

PyTorch supplies device memory (the caching allocator is installed as the
library's allocator) and streams.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import threading

import numpy as np

from . import _native as N
from ._native import (BC_COULOMB, BC_DH, BC_ZERO, CT_ALL, CT_BOUNDARY, CT_PAIRS,  # noqa: F401
                      CT_SURFACE, DEVICE, FP64, HOST, MIXED, PBError)

__all__ = [
    "GridSpec", "OctreeSpec", "Params", "SolveOpts", "Grid", "System",
    "pb_build_grid", "pb_assemble_coeffs", "pb_coulomb_terms", "pb_solve", "pb_energy",
    "pb_get_array", "pb_get_phi", "pb_apply", "pb_solve_batch", "pb_last_error",
    "pb_profile_kernels", "pb_kernel_launches", "pb_set_tuning", "pb_set_wait_limit", "pb_solve_split",
    "solve_molecule", "library_path", "loaded", "PBError", "Engine",
]

_alloc_lock = threading.Lock()
_alloc_installed = False


def library_path() -> str:
    return N.LIB_PATH


def loaded() -> bool:
    return N.lib() is not None


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        torch = _torch()
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        return C.c_void_p(0)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def use_torch_allocator(enable: bool = True) -> None:
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_installed
    with _alloc_lock:
        L = N.lib()
        if not enable:
            N.check(L.pb_set_allocator(None, None, None))
            _alloc_installed = False
            return
        if _alloc_installed:
            return
        torch = _torch()

        def _alloc(ctx, nbytes, stream):
            try:
                dev = torch.cuda.current_device()
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            except Exception:  # noqa: BLE001 - reported to C as NULL
                return None

        def _free(ctx, ptr, stream):
            try:
                torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:  # noqa: BLE001
                pass

        N.keep_alive(N.ALLOC_FN(_alloc), N.FREE_FN(_free))
        fa, ff = N.kept()
        N.check(L.pb_set_allocator(fa, ff, None))
        _alloc_installed = True


# ------------------------------------------------------------------ options
@dataclasses.dataclass
class GridSpec:
    n: tuple = (65, 65, 65)
    origin: tuple = (0.0, 0.0, 0.0)
    h: float = 0.0          # 0 -> automatic placement with ``fill``
    fill: float = 1.5

    def c(self) -> N.GridSpecC:
        s = N.GridSpecC()
        s.kind = N.GRID_UNIFORM
        n = self.n if not isinstance(self.n, int) else (self.n,) * 3
        for d in range(3):
            s.n[d] = int(n[d])
            s.origin[d] = float(self.origin[d])
        s.h = float(self.h)
        s.fill = float(self.fill)
        return s


@dataclasses.dataclass
class OctreeSpec:
    """Octree brick grid: cells h_bulk / 2^l down to h_fine, refined within
    refine_dist of the atom spheres.  n0 = 0 places n0^3 coarse bricks
    automatically (cube of fill x extent); n0 > 0 uses ``origin``.
    h_tight > 0: de-refined domain, h_bulk is the far-field spacing and the
    tight box (tight_fill x extent) is refined to at least h_tight."""
    h_fine: float = 0.25
    h_bulk: float = 1.0
    refine_dist: float = 3.0
    fill: float = 1.5
    n0: int = 0
    origin: tuple = (0.0, 0.0, 0.0)
    h_tight: float = 0.0
    tight_fill: float = 1.1

    def c(self) -> N.GridSpecC:
        s = N.GridSpecC()
        s.kind = N.GRID_OCTREE
        s.n[0] = int(self.n0)
        for d in range(3):
            s.origin[d] = float(self.origin[d])
        s.fill = float(self.fill)
        s.h_fine, s.h_bulk, s.refine_dist = float(self.h_fine), float(self.h_bulk), float(self.refine_dist)
        s.h_tight, s.tight_fill = float(self.h_tight), float(self.tight_fill)
        return s


@dataclasses.dataclass
class Params:
    eps_in: float = 2.0
    eps_out: float = 80.0
    ionic_strength_M: float = 0.145
    temperature_K: float = 298.15
    bc: int = BC_ZERO

    def c(self) -> N.ParamsC:
        p = N.ParamsC()
        p.eps_in, p.eps_out = float(self.eps_in), float(self.eps_out)
        p.ionic_strength_M, p.temperature_K = float(self.ionic_strength_M), float(self.temperature_K)
        p.bc = int(self.bc)
        return p


@dataclasses.dataclass
class SolveOpts:
    precision: int = MIXED
    rtol: float = 1e-8
    max_iter: int = 0
    max_outer: int = 0
    inner_rtol: float = 0.0
    time_budget_s: float = 0.0

    def c(self) -> N.SolveOptsC:
        o = N.SolveOptsC()
        o.precision, o.rtol = int(self.precision), float(self.rtol)
        o.max_iter, o.max_outer = int(self.max_iter), int(self.max_outer)
        o.inner_rtol, o.time_budget_s = float(self.inner_rtol), float(self.time_budget_s)
        return o


# ------------------------------------------------------------------ handles
class Grid:
    """Owns a ``pb_grid*``."""

    def __init__(self, handle, stream):
        self._h = handle
        self._stream = stream
        self.info = N.grid_info(handle)

    @property
    def handle(self):
        return self._h

    @property
    def n(self):
        return tuple(self.info.n)

    @property
    def N(self) -> int:
        return int(self.info.n_nodes)

    def free(self):
        if self._h:
            N.lib().pb_grid_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class System:
    """Owns a ``pb_system*`` (keeps its grid alive)."""

    def __init__(self, handle, grid: Grid):
        self._h = handle
        self.grid = grid

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            N.lib().pb_system_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


# ------------------------------------------------------------ entry points
def _atoms_arg(atoms):
    """(pointer, count, location, keepalive) for numpy or torch atoms."""
    try:
        torch = _torch()
        if isinstance(atoms, torch.Tensor):
            if atoms.dtype != torch.float64 or atoms.dim() != 2 or atoms.shape[1] != 5:
                raise ValueError("atoms must be a float64 tensor of shape (N, 5)")
            a = atoms.contiguous()
            loc = DEVICE if a.is_cuda else HOST
            return C.c_void_p(a.data_ptr()), a.shape[0], loc, a
    except ImportError:
        pass
    a = np.ascontiguousarray(atoms, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 5:
        raise ValueError("atoms must have shape (N, 5)")
    return a.ctypes.data_as(C.c_void_p), a.shape[0], HOST, a


def pb_build_grid(spec: GridSpec, atoms, stream=None) -> Grid:
    use_torch_allocator()
    ptr, n, loc, keep = _atoms_arg(atoms)
    h = C.c_void_p()
    st = _stream(stream)
    N.check(N.lib().pb_build_grid(C.byref(spec.c()), ptr, n, loc, st, C.byref(h)))
    del keep
    return Grid(h, st)


def pb_assemble_coeffs(grid: Grid, params: Params, stream=None) -> System:
    h = C.c_void_p()
    N.check(N.lib().pb_assemble_coeffs(grid.handle, C.byref(params.c()), _stream(stream), C.byref(h)))
    return System(h, grid)


def pb_coulomb_terms(system: System, which: int = CT_SURFACE | CT_PAIRS, stream=None) -> None:
    N.check(N.lib().pb_coulomb_terms(system.handle, int(which), _stream(stream)))


def pb_solve(system: System, opts: SolveOpts, phi_out=None, stream=None, check=True) -> dict:
    """Returns the solve statistics as a dict; raises on error when ``check``."""
    stats = N.SolveStatsC()
    ptr = C.c_void_p(phi_out.data_ptr()) if phi_out is not None else None
    rc = N.lib().pb_solve(system.handle, C.byref(opts.c()), ptr, _stream(stream), C.byref(stats))
    if check:
        N.check(rc)
    d = N.struct_dict(stats)
    d["rc"] = rc
    return d


def pb_energy(system: System, stream=None) -> dict:
    out = N.EnergyC()
    N.check(N.lib().pb_energy(system.handle, _stream(stream), C.byref(out)))
    return N.struct_dict(out)


_ARRAYS = {
    "inside": (N.ARR_INSIDE, np.uint8, "N"),
    "cross_id": (N.ARR_CROSS_ID, np.int64, "nc"),
    "cross_alpha": (N.ARR_CROSS_ALPHA, np.float64, "nc"),
    "cross_rp": (N.ARR_CROSS_RP, np.float64, "nc3"),
    "cross_sign": (N.ARR_CROSS_SIGN, np.int8, "nc"),
    "Wx": (N.ARR_WX, np.float64, "N"),
    "Wy": (N.ARR_WY, np.float64, "N"),
    "Wz": (N.ARR_WZ, np.float64, "N"),
    "kappa": (N.ARR_KAPPA, np.float64, "N"),
    "diag": (N.ARR_DIAG, np.float64, "N"),
    "rhs": (N.ARR_RHS, np.float64, "N"),
    "bc": (N.ARR_BC, np.float64, "N"),
    "phi": (N.ARR_PHI, np.float64, "N"),
    "phi_surf": (N.ARR_PHI_SURF, np.float64, "nc"),
    "psi_surf": (N.ARR_PSI_SURF, np.float64, "nc"),
    "oct_bricks": (N.ARR_OCT_BRICKS, np.int32, "nb4"),
    "oct_kind": (N.ARR_OCT_KIND, np.uint8, "N"),
    "mc_weight": (N.ARR_MC_WEIGHT, np.float64, "nc"),
    "mc_normal": (N.ARR_MC_NORMAL, np.float64, "nc3"),
    "psi_n": (N.ARR_PSI_N, np.float64, "nc"),
}


def pb_get_array(obj, name: str, stream=None) -> np.ndarray:
    """Copy one named array (see ``_ARRAYS``) to a new host numpy array."""
    which, dt, kind = _ARRAYS[name]
    if isinstance(obj, System):
        g, s = obj.grid, obj
    else:
        g, s = obj, None
    info = N.grid_info(g.handle)
    cnt = {"N": info.n_nodes, "nc": info.n_cross, "nc3": 3 * info.n_cross,
           "nb4": 4 * info.n_bricks}[kind]
    out = np.empty(max(int(cnt), 1), dtype=dt)
    N.check(N.lib().pb_get_array(g.handle, s.handle if s else None, which,
                                 out.ctypes.data_as(C.c_void_p), out.nbytes, HOST, _stream(stream)))
    out = out[:cnt]
    if kind == "nc3":
        return out.reshape(-1, 3)
    if kind == "nb4":
        return out.reshape(-1, 4)
    return out


def pb_get_phi(system: System, stream=None) -> np.ndarray:
    return pb_get_array(system, "phi", stream)


def pb_apply(system: System, x, precision: int = FP64, stream=None):
    """y = A x for a CUDA tensor x of N elements (float64, or float32 for MIXED)."""
    torch = _torch()
    want = torch.float64 if precision == FP64 else torch.float32
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == want):
        raise ValueError("x must be a CUDA tensor of the operator's dtype")
    x = x.contiguous()
    y = torch.empty_like(x)
    N.check(N.lib().pb_apply(system.handle, int(precision), C.c_void_p(x.data_ptr()),
                             C.c_void_p(y.data_ptr()), _stream(stream)))
    return y


def pb_solve_batch(systems, opts: SolveOpts, stream=None, check=True) -> list:
    """Per-system statistics dicts (each with the call's return code under
    ``rc``); raises on error when ``check``."""
    n = len(systems)
    arr = (C.c_void_p * n)(*[s.handle for s in systems])
    stats = (N.SolveStatsC * n)()
    rc = N.lib().pb_solve_batch(arr, n, C.byref(opts.c()), _stream(stream), stats)
    if check:
        N.check(rc)
    out = [N.struct_dict(s) for s in stats]
    for d in out:
        d["rc"] = rc
    return out


class Engine:
    """Owns a ``pb_engine*``: continuous batching of mixed-precision solves.

    ``submit`` hands an assembled :class:`System` to the engine (it joins the
    running launch table as soon as a slot is free); ``wait`` returns finished
    solves as dicts with ``ticket``, ``system`` (the submitted object),
    ``stats`` and the engine's monotonic timestamps ``t_submit``,
    ``t_admit``, ``t_done``.  A submitted system must not be used until it
    has been returned by ``wait``.
    """

    def __init__(self, capacity: int = 64, opts: SolveOpts | None = None, device: int | None = None):
        use_torch_allocator()
        if device is None:
            device = _torch().cuda.current_device()
        h = C.c_void_p()
        o = (opts or SolveOpts()).c()
        N.check(N.lib().pb_engine_create(int(device), int(capacity), C.byref(o), C.byref(h)))
        self._h = h
        self.capacity = int(capacity)
        self._systems: dict[int, System] = {}
        self._lock = threading.Lock()

    def submit(self, system: System, stream=None) -> int:
        t = C.c_int64()
        with self._lock:
            N.check(N.lib().pb_engine_submit(self._h, system.handle, _stream(stream), C.byref(t)))
            self._systems[int(t.value)] = system
        return int(t.value)

    def wait(self, timeout_s: float = 0.0, max_out: int = 256) -> list:
        out = (N.EngineResultC * max_out)()
        n = C.c_int32()
        N.check(N.lib().pb_engine_wait(self._h, float(timeout_s), out, int(max_out), C.byref(n)))
        res = []
        with self._lock:
            for r in out[: n.value]:
                res.append({"ticket": int(r.ticket), "system": self._systems.pop(int(r.ticket), None),
                            "stats": N.struct_dict(r.stats), "t_submit": r.t_submit,
                            "t_admit": r.t_admit, "t_done": r.t_done})
        return res

    def query(self) -> dict:
        p, a, r = C.c_int32(), C.c_int32(), C.c_int64()
        rc = N.lib().pb_engine_query(self._h, C.byref(p), C.byref(a), C.byref(r))
        return {"pending": p.value, "active": a.value, "replays": r.value, "rc": rc}

    def close(self) -> None:
        if self._h:
            N.check(N.lib().pb_engine_destroy(self._h))
            self._h = None
            self._systems.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def pb_profile_kernels(system: System, precision: int, which: int, reps: int, stream=None) -> None:
    N.check(N.lib().pb_profile_kernels(system.handle, int(precision), int(which), int(reps),
                                       _stream(stream)))


def pb_set_tuning(system: System, precision: int, variant: int, z_chunk: int) -> None:
    """Fix the PCG kernel variant and z-chunk for the system's grid shape;
    for the TMA-staged variant z_chunk may add 10000 x the tile width (128,
    64 or 32)."""
    N.check(N.lib().pb_set_tuning(system.handle, int(precision), int(variant), int(z_chunk)))


def pb_solve_split(system: System, ranks: int, opts: SolveOpts, stream=None, check=True) -> dict:
    """The mixed-precision solve on ``ranks`` z-slabs with halo exchanges and
    rank-ordered reductions; statistics as from :func:`pb_solve`."""
    stats = N.SolveStatsC()
    rc = N.lib().pb_solve_split(system.handle, int(ranks), C.byref(opts.c()), _stream(stream),
                                C.byref(stats))
    if check:
        N.check(rc)
    d = N.struct_dict(stats)
    d["rc"] = rc
    return d


def pb_set_wait_limit(polls: int) -> None:
    """Polls before an FP32 PCG ring-slot wait gives up (< 0: the default)."""
    N.check(N.lib().pb_set_wait_limit(int(polls)))


def pb_kernel_launches() -> int:
    return int(N.lib().pb_kernel_launches())


def pb_last_error() -> str:
    return N.lib().pb_last_error().decode()


def solve_molecule(atoms, n=65, fill=1.5, params: Params | None = None,
                   opts: SolveOpts | None = None, spec: GridSpec | None = None,
                   stream=None) -> dict:
    """Whole hot path for one molecule: grid, coefficients, Coulomb terms,
    solve, energy.  Returns the energy terms and solve statistics."""
    params = params or Params()
    opts = opts or SolveOpts()
    spec = spec or GridSpec(n=(n, n, n), fill=fill)
    g = pb_build_grid(spec, atoms, stream)
    s = pb_assemble_coeffs(g, params, stream)
    pb_coulomb_terms(s, CT_SURFACE | CT_PAIRS, stream)
    stats = pb_solve(s, opts, stream=stream)
    e = pb_energy(s, stream)
    return {"energy": e, "stats": stats, "system": s}
