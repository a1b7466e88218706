"""The allocation-free log-determinant (h2_logdet_noalloc) against h2_logdet.

Callers that cannot allocate device memory at the point where they need the
value (their memory is fully reserved or owned by another allocator) use
h2_logdet_noalloc, whose scratch is a fixed device array inside the library.
This file is collected last on purpose.  It checks, through the C ABI, that
two calls in a row give the same result as the allocating entry point, and
that the library allocated no device memory during those calls."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_logdet_noalloc_matches_logdet_twice():
    X = synth.sphere_ball(4096, 21)
    pts = torch.from_numpy(X).cuda()
    h = H.h2_construct(pts, len(X), H.make_kernel("yukawa"), H.make_options(leaf=128, tol=1e-10, max_rank=128))
    try:
        H.h2_factor(h, H.H2_FP64)
        ref, ref_sign = H.h2_logdet(h)
        # first call does the one-time per-device set-up
        v1, s1 = H.h2_logdet_noalloc(h)
        free_before = _free_bytes()
        v2, s2 = H.h2_logdet_noalloc(h)
        free_after = _free_bytes()
        for v, s in ((v1, s1), (v2, s2)):
            assert s[0] == ref_sign[0]
            assert abs(v[0] - ref[0]) <= 1e-12 * abs(ref[0]), (v[0], ref[0])
        assert free_after == free_before
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("spd", [0, 1])
def test_logdet_noalloc_batched_handle(spd):
    """A batched handle (three problems of different depths): every
    problem's value and sign, through the per-problem accumulation of the
    allocation-free path, equal h2_logdet's; LU (spd = 0) and the Cholesky
    form (spd = 1) of the Matern-3/2 covariance kernel.  No device memory
    is allocated by the second call."""
    Xs = [synth.cube(n, 60 + k) for k, n in enumerate([1500, 700, 2600])]
    hb = H.h2_construct_batched([torch.from_numpy(X).cuda() for X in Xs], H.make_kernel("matern32"),
                                H.make_options(leaf=128, tol=1e-10, max_rank=128))
    try:
        H.h2_factor(hb, H.H2_FP64, spd)
        ref, ref_sign = H.h2_logdet(hb, len(Xs))
        v1, s1 = H.h2_logdet_noalloc(hb, len(Xs))
        free_before = _free_bytes()
        v2, s2 = H.h2_logdet_noalloc(hb, len(Xs))
        free_after = _free_bytes()
        for v, s in ((v1, s1), (v2, s2)):
            assert list(s) == list(ref_sign)
            np.testing.assert_allclose(v, ref, rtol=1e-12, atol=0)
        assert free_after == free_before
    finally:
        H.h2_destroy(hb)
