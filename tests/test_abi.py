"""The C-ABI library loads and exports every entry point include/pff.h declares;
host-only calls (argument checks, basis tables) work without a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpff():
    from paper_2607_21150_gb300 import build, pff
    build.build()
    return pff.lib()


def header_functions():
    src = open(os.path.join(ROOT, "include", "pff.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pff_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(libpff):
    from paper_2607_21150_gb300 import build, pff
    names = header_functions()
    assert len(names) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pff_[a-z0-9_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(pff.declared_symbols()) == names  # the binding covers the header exactly


def test_argument_errors_without_gpu(libpff):
    from paper_2607_21150_gb300 import inputs, pff
    with pytest.raises(pff.PffError, match="nphase"):
        pff.pff_create_context(np.zeros((0, 12)), 2, 1e-3, 1e-2, 0.01, 1.0)
    with pytest.raises(pff.PffError, match="at must be"):
        pff.pff_create_context(inputs.phase_vector(inputs.EX3_MATRIX)[None], 3, 1e-3, 1e-2, 0.01, 1.0)
    ctx = pff.pff_create_context(inputs.phase_vector(inputs.EX3_MATRIX)[None], 2, 1e-3, 1e-2, 0.01, 1.0)
    with pytest.raises(pff.PffError, match="p \\+ 1 <= q"):
        pff.pff_create_basis(ctx, 4, 4)
    with pytest.raises(pff.PffError, match="nnodes"):
        pff.pff_create_restriction(ctx, (2, 2, 2, 0.1, 0.1, 0.1), 2, None, 7)
    pff.pff_destroy_context(ctx)
    # the pipe-rate probe checks its arguments before any launch (the sink
    # address is never dereferenced on the host)
    sink = ctypes.c_void_p(16)
    with pytest.raises(pff.PffError, match="multiple of 4"):
        pff.pff_probe_pipe(pff.PFF_PROBE_CVT, 3, 1, 32, sink, 0)
    with pytest.raises(pff.PffError, match="unknown probe kind"):
        pff.pff_probe_pipe(7, 4, 1, 32, sink, 0)


def test_degenerate_arguments_rejected_without_gpu(libpff):
    """Empty and degenerate inputs are refused on the host with PFF_ERR_INVALID
    before any device work: an empty element grid, non-positive element sizes,
    orders outside 1..4, moduli outside E > 0, -1 < nu < 0.5, a non-positive
    time step, and hardening laws that would lower the yield stress."""
    from paper_2607_21150_gb300 import inputs, pff

    def invalid(fn, *args, match):
        with pytest.raises(pff.PffError, match=match) as e:
            fn(*args)
        assert e.value.code == pff.ERR_INVALID

    row = inputs.phase_vector(inputs.EX3_MATRIX)
    bad_nu = row.copy()
    bad_nu[3] = 0.5
    invalid(pff.pff_create_context, bad_nu[None], 2, 1e-3, 1e-2, 0.01, 1.0, match="moduli")
    invalid(pff.pff_create_context, row[None], 2, 1e-3, 1e-2, 0.0, 1.0, match="dt")
    ctx = pff.pff_create_context(row[None], 2, 1e-3, 1e-2, 0.01, 1.0)
    for nx, ny, nz in ((0, 2, 2), (2, 0, 2), (2, 2, 0)):
        invalid(pff.pff_create_restriction, ctx, (nx, ny, nz, 0.1, 0.1, 0.1), 2, None, 1, match="empty element grid")
    invalid(pff.pff_create_restriction, ctx, (2, 2, 2, 0.1, -0.1, 0.1), 2, None, 125, match="element sizes")
    invalid(pff.pff_create_restriction, ctx, (2, 2, 2, 0.1, 0.1, 0.1), 5, None, 1331, match="p <= 4")
    invalid(pff.pff_create_basis, ctx, 0, 2, match="p \\+ 1 <= q")
    invalid(pff.pff_create_basis, ctx, 4, 6, match="p \\+ 1 <= q")
    invalid(pff.pff_context_set_time_step, ctx, -1.0, match="dt")
    invalid(pff.pff_context_set_hardening, ctx, 0, 100.0, 0.5 * row[11], 10.0, match="sigma_inf >= sigma0")
    invalid(pff.pff_context_set_hardening, ctx, 1, 100.0, 2.0 * row[11], 10.0, match="phase out of range")
    r = pff.pff_create_restriction(ctx, (1, 1, 1, 0.1, 0.1, 0.1), 1, None, 8)   # one element is valid
    pff.pff_destroy_restriction(r)
    pff.pff_destroy_context(ctx)


@pytest.mark.parametrize("p,q", [(1, 2), (2, 3), (3, 4), (4, 5), (2, 5), (1, 5)])
def test_library_basis_tables_match_oracle(libpff, orc, p, q):
    from paper_2607_21150_gb300 import inputs, pff
    ctx = pff.pff_create_context(inputs.phase_vector(inputs.EX3_MATRIX)[None], 2, 1e-3, 1e-2, 0.01, 1.0)
    b = pff.pff_create_basis(ctx, p, q)
    xg, xq, wq, B, Dc = pff.pff_basis_get(b, p, q)
    oxg, oxq, owq, oB, oD = orc.basis(p, q)
    assert np.abs(xg - oxg).max() < 1e-15
    assert np.abs(xq - oxq).max() < 1e-15 and np.abs(wq - owq).max() < 1e-15
    assert np.abs(B - oB).max() < 1e-14
    assert np.abs(Dc @ B - oD).max() < 1e-12
    pff.pff_destroy_basis(b)
    pff.pff_destroy_context(ctx)


def test_hardening_rows_through_the_binding(libpff):
    """15-column phase rows carry the hardening law to pff_context_set_hardening
    (host only): valid rows are accepted, a law that would lower the yield
    stress is refused, and perfect-plasticity rows make no call."""
    from paper_2607_21150_gb300 import inputs, pff
    ph = np.stack([inputs.phase_vector(inputs.EX3_MATRIX), inputs.phase_vector(inputs.EX3_PARTICLE)])
    ctx = pff.pff_create_context(inputs.harden(ph, 2000.0, 800.0, 40.0), 1, 1e-3, 1e-2, 0.01, 1.0)
    pff.pff_destroy_context(ctx)
    perfect = inputs.harden(ph, 0.0, 0.0, 0.0)
    perfect[:, 13] = perfect[:, 11]                                 # (0, sigma0, 0): perfect plasticity
    ctx = pff.pff_create_context(perfect, 1, 1e-3, 1e-2, 0.01, 1.0)
    pff.pff_destroy_context(ctx)
    bad = inputs.harden(ph, 2000.0, 0.5 * ph[0, 11], 40.0)
    with pytest.raises(pff.PffError, match="sigma_inf >= sigma0") as e:
        pff.pff_create_context(bad, 1, 1e-3, 1e-2, 0.01, 1.0)
    assert e.value.code == pff.ERR_INVALID
