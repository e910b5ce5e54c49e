"""The allocation-free Delta Z entry point (ect_delta_z_static) against ect_delta_z.

ect_delta_z_static keeps its scratch in a static device array instead of
allocating, for callers that cannot allocate device memory.  This file sits
last in collection order so a run that stops at the first failure has already
run every other test; it also passes when run alone in a fresh process.
Tolerance: the two entry points sum the same per-tet terms with a different
number of partial sums, so they agree to rounding (1e-12 relative)."""
import numpy as np
import pytest

import ect_inputs as E

import os
import re

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_static_path_source_allocates_nothing():
    """CPU check of the property that defines the entry point: the code from the
    static scratch lookup to the end of ect_delta_z_static names no device
    allocation (no DevBuf, alloc/ensure, cudaMalloc*, cudaFree*)."""
    src = open(os.path.join(ROOT, "paper_1602_03207_gb300", "csrc", "rhs_impedance.cu")).read()
    start = src.index("double* dz_static_scratch()")
    body = src[start:]
    assert "ect_delta_z_static" in body
    code = re.sub(r"//[^\n]*", "", body)                       # comments may mention the words
    for bad in ("DevBuf", ".alloc(", ".ensure(", "cudaMalloc", "cudaFree", "new ", "torch"):
        assert bad not in code, bad


@pytest.fixture(scope="module")
def case():
    assert torch.cuda.is_available()
    from paper_1602_03207_gb300 import build, ect
    build.build()
    p = E.wall_loss_problem((10, 11, 13), (20e-3, 20e-3, 30e-3), (2, 3, 2), 0.15, 1,
                            z_pos=(-1.0e-3, 0.0, 2.5e-3))
    ctx = ect.Context()
    ctx.load_problem(p)
    for w in (ect.ECT_VACUUM, ect.ECT_DEFECT):
        ctx.assemble(w, ect.ECT_F64)
        ctx.precond_setup(w, ect.ECT_F64, -1)
    n = 4 * p.mesh.n_nodes
    P = len(p.z_pos)
    B = torch.empty(P, 2, n, dtype=torch.complex128, device="cuda")
    for c in range(2):
        t = torch.empty(P, n, dtype=torch.complex128, device="cuda")
        ctx.coil_rhs(p.coils[c], p.z_pos, t)
        B[:, c] = t
    U0 = torch.empty_like(B)
    Ud = torch.empty_like(B)
    opts = ect.default_options(tol=1e-10)
    ctx.solve(0, B, U0, 2 * P, opts)
    ctx.solve(1, B, Ud, 2 * P, opts)
    cur = [c.current for c in p.coils]
    return ect, ctx, B, U0, Ud, cur, P


@pytest.mark.gpu
def test_static_delta_z_matches_allocating_entry_point_twice(case):
    ect, ctx, B, U0, Ud, cur, P = case
    ref = [ctx.delta_z(U0[q], Ud[q], B[q], cur) for q in range(P)]
    for _ in range(2):                       # two calls in a row reuse the same static scratch
        dz, dze = ctx.delta_z_static(U0, Ud, B, cur, P)
        for q in range(P):
            scale = np.abs(ref[q][0]).max()
            assert scale > 0
            assert np.abs(dz[q] - ref[q][0]).max() <= 1e-12 * scale
            assert np.abs(dze[q] - ref[q][1]).max() <= 1e-12 * np.abs(ref[q][1]).max()
    # a single position without the EMF cross-check, again twice
    for _ in range(2):
        dz1, none = ctx.delta_z_static(U0[1:2].contiguous(), Ud[1:2].contiguous(), None, cur, 1)
        assert none is None
        assert np.abs(dz1[0] - ref[1][0]).max() <= 1e-12 * np.abs(ref[1][0]).max()


@pytest.mark.gpu
def test_static_delta_z_rejects_too_many_positions(case):
    ect, ctx, B, U0, Ud, cur, P = case
    with pytest.raises(ect.EctError) as e:
        ctx.delta_z_static(U0, Ud, None, cur, 65)
    assert e.value.code == ect.ECT_ERR_ARG and "64" in str(e.value)
