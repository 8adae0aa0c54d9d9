"""The allocation-free symbolic pass, mcl_symbolic_noalloc, for callers that
cannot allocate device memory where they need output sizes (a service that
reserves its GPU memory in a pool at start-up and forbids allocation
afterwards).  It must return exactly what the context-based mcl_symbolic
returns, on consecutive calls sharing its one scratch array, and must
reject inputs beyond its fixed scratch size with a clear error.

Collected last on purpose (file name) so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2002_10083_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import mcl
    c = mcl.Context(0)
    yield c
    c.close()


def _run_noalloc(D):
    from paper_2002_10083_gb300 import mcl
    fl = torch.full((max(D.n, 1),), -1, dtype=torch.int64, device="cuda")
    nz = torch.full((max(D.n, 1),), -1, dtype=torch.int64, device="cuda")
    mcl.symbolic_noalloc(D, fl, nz)
    torch.cuda.synchronize()
    return fl[:D.n], nz[:D.n]


def test_noalloc_matches_symbolic_on_consecutive_calls(ctx):
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=200000, mean=30.0, d_max=3000, seed=3).with_val32()
    B = synth.random_sparse(3000, 0.01, seed=4).with_val32()
    DA = mcl.DeviceCSC.from_host(A)
    DB = mcl.DeviceCSC.from_host(B)
    ref_a = ctx.symbolic(DA)
    ref_b = ctx.symbolic(DB)
    # two calls in a row on the same input, then a different input: the
    # shared scratch keeps the previous call's contents in between
    for D, (rf, rn) in ((DA, ref_a), (DA, ref_a), (DB, ref_b), (DA, ref_a)):
        fl, nz = _run_noalloc(D)
        assert torch.equal(fl, rf)
        assert torch.equal(nz, rn)


def test_noalloc_rejects_inputs_beyond_its_scratch():
    from paper_2002_10083_gb300 import mcl
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    # n above the fixed maximum is rejected before any device access
    small = torch.zeros(2, dtype=torch.int64, device="cuda")
    big = mcl.DeviceCSC(10_000_000, small, torch.zeros(0, dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.float32, device="cuda"))
    big_c = big.c()
    big_c.n = 10_000_000
    lib = mcl.load()
    err = ctypes.create_string_buffer(512)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.mcl_symbolic_noalloc(ctypes.byref(big_c), ctypes.c_void_p(out.data_ptr()), None, err,
                                  len(err), None)
    assert st == 1
    assert b"maximum" in err.value
