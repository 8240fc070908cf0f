"""Device-side failures surface as status codes, tested without a failing kernel.

  * The bounded mbarrier wait of the tensor-core kernels, run by a one-CTA
    self-test on a barrier phase that nothing completes, runs out, records
    the timeout in a status word and returns; the context stays usable.
  * The solver's status path: a status word with bit 0 set (what a Gram or
    update kernel leaves when one of its waits ran out, here set by the
    solver itself on request) ends the solve with LOBPCG_ERR_TIMEOUT and a
    message, and the next solve on the same device is unaffected.
"""
import numpy as np
import pytest

import synth
import paper_1704_07458_gb300 as gb
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_reports():
    torch_cuda()
    assert gb.lobpcg_wait_selftest(1000) == gb.LOBPCG_ERR_TIMEOUT
    assert gb.lobpcg_wait_selftest(1) == gb.LOBPCG_ERR_TIMEOUT
    p = synth.make_problem("lap2d_32")
    with gb.Solver(gemm_mode="ozaki_tc") as s:
        s.set_operator(p.A.rowptr, p.A.col, p.A.val)
        lam, X, it, be, rc = s.solve(p.k, p.tol, raise_on_error=False)
    assert rc == gb.LOBPCG_OK
    np.testing.assert_allclose(lam, p.closed_form[:p.k], rtol=1e-10)


@pytest.mark.parametrize("mode", ["f64", "ozaki_tc"])
def test_status_word_ends_the_solve_with_timeout(mode):
    torch_cuda()
    p = synth.make_problem("lap2d_32")
    with gb.Solver(gemm_mode=mode, inject_wait_timeout_at=3) as s:
        s.set_operator(p.A.rowptr, p.A.col, p.A.val)
        lam, X, it, be, rc = s.solve(p.k, p.tol, raise_on_error=False)
        assert rc == gb.LOBPCG_ERR_TIMEOUT
        assert it == 3
        assert "bounded wait" in gb.lobpcg_last_error(s.h)
    with gb.Solver(gemm_mode=mode) as s:
        s.set_operator(p.A.rowptr, p.A.col, p.A.val)
        lam, X, it, be, rc = s.solve(p.k, p.tol, raise_on_error=False)
    assert rc == gb.LOBPCG_OK
    np.testing.assert_allclose(lam, p.closed_form[:p.k], rtol=1e-10)
