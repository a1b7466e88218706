"""Failure paths across the C ABI: every documented status is returned (no
exception crosses the boundary) with a message in h2_last_error().  The
failures are made on the host side or by inputs whose arithmetic is exact
(coincident points make the kernel matrix exactly rank one); nothing here
faults or stalls the GPU."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402


def last_error():
    return H.lib().h2_last_error().decode()


def small_handle(N=2048, **kw):
    X = synth.sphere_ball(N, 31)
    opt = dict(leaf=128, tol=1e-8, max_rank=96)
    opt.update(kw)
    return H.h2_construct(torch.from_numpy(X).cuda(), N, H.make_kernel("laplace"), H.make_options(**opt)), N


def test_budget_exceeded_at_construct():
    X = synth.sphere_ball(4096, 32)
    with pytest.raises(H.H2Error) as e:
        H.h2_construct(torch.from_numpy(X).cuda(), len(X), H.make_kernel("laplace"),
                       H.make_options(leaf=128, hbm_budget_bytes=1 << 20))
    assert e.value.status == H.H2_ERR_BUDGET
    assert "bytes" in last_error()


def test_calls_before_factor_are_out_of_order():
    h, N = small_handle()
    try:
        b = torch.ones(N, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        st = H.lib().h2_solve(h, H._ptr(b), H._ptr(x), 1, N, 1e-10, 5, None, None)
        assert st == H.H2_ERR_STATE and "before h2_factor" in last_error()
        for f in (H.h2_logdet, H.h2_logdet_noalloc):
            with pytest.raises(H.H2Error) as e:
                f(h)
            assert e.value.status == H.H2_ERR_STATE
    finally:
        H.h2_destroy(h)


def test_refinement_stops_at_max_iter():
    h, N = small_handle()
    try:
        H.h2_factor(h, H.H2_MIXED)
        b = torch.from_numpy(synth.rhs(N, 1, 5)[:, 0].copy()).cuda()
        x = torch.zeros_like(b)
        st, ach, it = H.h2_solve(h, b, x, 1, N, 1e-16, 1)
        assert st == H.H2_ERR_NOT_CONVERGED and it == 1 and ach[0] > 1e-16
        assert "did not reach" in last_error()
        assert torch.isfinite(x).all() and float(x.abs().max()) > 0   # x holds the last iterate
    finally:
        H.h2_destroy(h)


def test_invalid_solve_arguments_and_nonfinite_rhs():
    h, N = small_handle()
    try:
        H.h2_factor(h, H.H2_FP64)
        b = torch.ones(N, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        assert H.lib().h2_solve(h, H._ptr(b), H._ptr(x), 1, N - 1, 1e-10, 5, None, None) == H.H2_ERR_ARG
        assert H.lib().h2_solve(h, H._ptr(b), H._ptr(x), 0, N, 1e-10, 5, None, None) == H.H2_ERR_ARG
        b[7] = float("nan")
        st, _, _ = H.h2_solve(h, b, x, 1, N, 1e-10, 5, check=False)
        assert st == H.H2_ERR_NONFINITE and "right-hand side" in last_error()
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("spd,status", [(0, H.H2_ERR_SINGULAR), (1, H.H2_ERR_NOT_SPD)])
def test_coincident_points_give_an_exactly_singular_matrix(spd, status):
    """100 copies of one point: every entry is K(0) = 1 / delta = 1000
    exactly, so the first elimination step leaves exact zeros and the next
    pivot is 0: LU reports a singular matrix, Cholesky a non-positive
    pivot.  The handle stays usable afterwards."""
    X = np.tile(np.array([[0.25, 0.5, 0.75]]), (100, 1))
    h = H.h2_construct(torch.from_numpy(X).cuda(), 100, H.make_kernel("laplace"), H.make_options(leaf=256))
    try:
        with pytest.raises(H.H2Error) as e:
            H.h2_factor(h, H.H2_FP64, spd)
        assert e.value.status == status
        assert ("zero pivot" in last_error()) if spd == 0 else ("non-positive pivot" in last_error())
        # a state error, not a broken handle: solving is refused cleanly
        b = torch.ones(100, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        assert H.lib().h2_solve(h, H._ptr(b), H._ptr(x), 1, 100, 1e-10, 5, None, None) == H.H2_ERR_STATE
    finally:
        H.h2_destroy(h)
