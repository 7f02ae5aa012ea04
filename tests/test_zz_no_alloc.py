"""pb_apply_dot_noalloc: the allocation-free FP64 apply + dot.

It exists for callers that cannot allocate device memory while they work; it
must give the same y = A x as pb_apply (which allocates padded temporaries)
and the same x.(A x), within the FP64 apply tolerance of the parity tests
(1e-12 relative), on consecutive calls that share its static scratch.  This
file is collected last so that a run stopping at its first failure has run
every other test already; it builds its own system and also passes alone.
"""
import ctypes

import numpy as np
import pytest

import pb_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_09323_gb300 import build
    build.build()
    import paper_2502_09323_gb300 as pb
    return pb


def _noalloc(pb, s, x, y, d):
    import torch
    lib = pb._native.lib()
    rc = lib.pb_apply_dot_noalloc(s.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                  ctypes.c_void_p(d.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


def test_noalloc_apply_dot_matches_pb_apply(pb):
    import torch
    atoms = pb_inputs.globular_molecule(80, seed=31)
    g = pb.pb_build_grid(pb.GridSpec(n=(97, 97, 97), fill=1.5), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params(bc=pb.BC_DH))
    N = g.N
    y = torch.empty(N, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    for seed in (5, 6):  # two calls in a row on the shared static scratch
        x = torch.tensor(pb_inputs.random_field(N, seed=seed), device="cuda")
        assert _noalloc(pb, s, x, y, d) == 0, pb.pb_last_error()
        torch.cuda.synchronize()
        y_ref = pb.pb_apply(s, x, precision=pb.FP64)
        dot_ref = float((x * y_ref).sum())
        scale = float(y_ref.abs().max())
        assert float((y - y_ref).abs().max()) <= 1e-12 * scale
        assert abs(float(d[0]) - dot_ref) <= 1e-12 * abs(dot_ref)


def test_noalloc_rejects_grids_beyond_its_scratch(pb):
    import torch
    atoms = np.array([[0.0, 0.0, 0.0, 1.5, 1.0]])
    n = 325  # 325^3 = 34,328,125 nodes > 33,554,432
    g = pb.pb_build_grid(pb.GridSpec(n=(n, n, n), origin=(-40.0,) * 3, h=0.25), atoms)
    s = pb.pb_assemble_coeffs(g, pb.Params())
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(pb, s, x, x, d) == -1
    assert "scratch" in pb.pb_last_error()
