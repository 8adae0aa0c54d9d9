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

import oracle
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


def _run_noalloc(D, want_flops=True, want_nnz=True):
    from paper_2002_10083_gb300 import mcl
    fl = torch.full((max(D.n, 1),), -1, dtype=torch.int64, device="cuda")
    nz = torch.full((max(D.n, 1),), -1, dtype=torch.int64, device="cuda")
    mcl.symbolic_noalloc(D, fl if want_flops else None, nz if want_nnz else None)
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


def test_noalloc_matches_oracle_on_sampled_columns():
    """Against the FP64 oracle's symbolic counts (the definition: flops_j =
    sum over the sources of their lengths, nnz_j = distinct rows reached)."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=200000, mean=30.0, d_max=3000, seed=3).with_val32()
    fl, nz = _run_noalloc(mcl.DeviceCSC.from_host(A))
    deg = np.diff(A.colptr)
    cols = np.concatenate([np.random.default_rng(7).choice(A.n, 2000, replace=False),
                           np.argsort(-deg)[:20]]).astype(np.int32)
    of, on = oracle.symbolic_cols(A, cols=cols)
    assert np.array_equal(fl.cpu().numpy()[cols], of)
    assert np.array_equal(nz.cpu().numpy()[cols], on)


def test_noalloc_row_windows_of_a_large_span(ctx):
    """Spans above one bitmap window (524,288 rows) walk their sources in
    several windows through the cursor region of the static array."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=700000, mean=8.0, d_max=500, seed=1).with_val32()
    D = mcl.DeviceCSC.from_host(A)
    fl, nz = _run_noalloc(D)
    rf, rn = ctx.symbolic(D)
    assert torch.equal(fl, rf) and torch.equal(nz, rn)
    cols = np.random.default_rng(1).choice(A.n, 1500, replace=False).astype(np.int32)
    of, on = oracle.symbolic_cols(A, cols=cols)
    assert np.array_equal(nz.cpu().numpy()[cols], on)
    assert np.array_equal(fl.cpu().numpy()[cols], of)


def test_noalloc_one_output_and_empty_input():
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(3000, 0.01, seed=4).with_val32()
    D = mcl.DeviceCSC.from_host(A)
    fl, nz = _run_noalloc(D)
    fl_only, untouched = _run_noalloc(D, want_nnz=False)
    assert torch.equal(fl_only, fl) and bool((untouched == -1).all())
    untouched, nz_only = _run_noalloc(D, want_flops=False)
    assert torch.equal(nz_only, nz) and bool((untouched == -1).all())
    E = mcl.DeviceCSC(0, torch.zeros(1, dtype=torch.int64, device="cuda"),
                      torch.zeros(0, dtype=torch.int32, device="cuda"),
                      torch.zeros(0, dtype=torch.float32, device="cuda"))
    fl0, nz0 = _run_noalloc(E)
    assert fl0.numel() == 0 and nz0.numel() == 0


def test_noalloc_allocates_nothing():
    """After one warm-up call (which loads the module that holds the static
    array), further calls leave torch's allocator and the device's free
    memory unchanged."""
    from paper_2002_10083_gb300 import mcl
    A = synth.chung_lu(n=100000, mean=20.0, d_max=2000, seed=9).with_val32()
    D = mcl.DeviceCSC.from_host(A)
    fl = torch.empty(A.n, dtype=torch.int64, device="cuda")
    nz = torch.empty(A.n, dtype=torch.int64, device="cuda")
    mcl.symbolic_noalloc(D, fl, nz)
    torch.cuda.synchronize()
    before = (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
    for _ in range(3):
        mcl.symbolic_noalloc(D, fl, nz)
    torch.cuda.synchronize()
    assert (torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]) == before


def test_noalloc_on_a_second_device():
    """Each device gets its own copy of the static array and its own kernel
    attributes."""
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(3000, 0.01, seed=4).with_val32()
    with torch.cuda.device(1):
        D = mcl.DeviceCSC.from_host(A, device="cuda:1")
        c1 = mcl.Context(1)
        try:
            rf, rn = c1.symbolic(D)
            fl = torch.empty(A.n, dtype=torch.int64, device="cuda:1")
            nz = torch.empty(A.n, dtype=torch.int64, device="cuda:1")
            mcl.symbolic_noalloc(D, fl, nz, stream=torch.cuda.current_stream(1))
            torch.cuda.synchronize(1)
            assert torch.equal(fl, rf) and torch.equal(nz, rn)
        finally:
            c1.close()
