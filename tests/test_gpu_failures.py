"""Failure handling through the C ABI, made on the host: the device
allocator (the context's callback) refuses one allocation.  The call
returns MCL_ERR_OOM, nothing is thrown across the ABI, and the same
context then computes the iteration normally."""
import numpy as np
import pytest

from paper_2002_10083_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _failing_context_class():
    from paper_2002_10083_gb300 import mcl

    class FailingContext(mcl.Context):
        """Refuses the fail_at-th device allocation (1-based), then works."""

        def __init__(self, fail_at):
            self.fail_at = fail_at
            self.calls = 0
            super().__init__(0)

        def _alloc(self, nbytes, user, stream):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            return super()._alloc(nbytes, user, stream)

    return FailingContext


def test_every_allocation_failure_of_an_iteration_is_reported_and_recovered():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2002_10083_gb300 import mcl
    A = synth.random_sparse(1500, 0.01, seed=7, w="lognormal").with_val32()
    D = mcl.DeviceCSC.from_host(A)
    prm = mcl.Params(threshold=1e-4, select_k=64, recover_pct=0.9, inflation=2.0)
    ref_ctx = mcl.Context(0)
    ref, _ = ref_ctx.expand(D, prm)
    ref_ctx.close()
    FailingContext = _failing_context_class()
    failures = 0
    for fail_at in range(1, 60):
        ctx = FailingContext(fail_at)
        try:
            try:
                out, _ = ctx.expand(D, prm)
                ok_first = True
            except mcl.MclError as e:
                assert e.status == 2, (fail_at, str(e))
                ok_first = False
                failures += 1
            if ok_first and ctx.calls < fail_at:
                break  # the iteration needs fewer allocations: every one was refused once
            out, _ = ctx.expand(D, prm)  # the same context, allocator working again
            assert torch.equal(out.colptr, ref.colptr) and torch.equal(out.rowidx, ref.rowidx)
            assert torch.equal(out.val.view(torch.int32), ref.val.view(torch.int32))
        finally:
            ctx.close()
    assert failures >= 5
