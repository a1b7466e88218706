"""Batched handle (several independent problems of different sizes and
depths factored and solved height by height in shared launches): every
problem's refined solution and log-determinant against the oracle and
against its own single-problem handle."""
import numpy as np
import pytest

import synth
from oracle import h2ulv_oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402


def problems():
    rng = np.random.default_rng(100)
    out = []
    for k, n in enumerate([3000, 700, 5200, 130, 2049]):
        r = np.random.default_rng(100 + k)
        geo = k % 3
        if geo == 0:
            X = synth.cube_surface(n, r)
        elif geo == 1:
            X = synth.sphere_surface(n, r)
        else:
            X = synth.ellipsoid_surface(n, r, tuple(0.5 + 1.5 * r.random(3)))
        out.append(X)
    return out


@pytest.mark.parametrize("precision", [H.H2_FP64, H.H2_MIXED])
def test_batched_matches_oracle_and_single(precision):
    Xs = problems()
    opt = H.make_options(leaf=128, tol=1e-8, max_rank=100)
    kern = H.make_kernel("laplace")
    hb = H.h2_construct_batched([torch.from_numpy(X).cuda() for X in Xs], kern, opt)
    try:
        H.h2_factor(hb, precision)
        Ns = [len(X) for X in Xs]
        off = np.concatenate([[0], np.cumsum(Ns)])
        nrhs = 3
        B = np.zeros((off[-1], nrhs))
        for p, N in enumerate(Ns):
            B[off[p]:off[p + 1]] = synth.rhs(N, nrhs, 50 + p)
        Bc = np.ascontiguousarray(B.T)                       # column-major stacked
        Xc = np.zeros_like(Bc)
        st, ach, it = H.h2_solve(hb, Bc, Xc, nrhs, off[-1], 1e-10, 40)
        assert st == H.H2_OK and np.all(ach <= 1e-10), (st, ach)
        ldb, sgb = H.h2_logdet(hb, len(Xs))
        for p, X in enumerate(Xs):
            pb = O.Problem(X, "laplace", 128, 1.0, 1e-8, 100)
            fac = O.ULVFactor(pb)
            xo, _, _ = O.refine(O.H2Operator(pb), fac, B[off[p]:off[p + 1]], 1e-10, 40)
            xg = Xc.T[off[p]:off[p + 1]]
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
            # log-det against the oracle: FP64 the same route (1e-9); mixed
            # the oracle's Gram route at the effective tolerance, N 2^-17
            # (each of the N pivots within 2^7 FP32 unit roundoffs)
            if precision == H.H2_FP64:
                lo, so = fac.logdet()
                assert sgb[p] == so and abs(ldb[p] - lo) <= 1e-9 * abs(lo), (p, ldb[p], lo)
            else:
                lo, so = O.ULVFactor(pb, route="gram", tol_basis=2.0 ** -10).logdet()
                assert sgb[p] == so and abs(ldb[p] - lo) <= len(X) * 2.0 ** -17, (p, ldb[p], lo)
            # the same problem alone
            h1 = H.h2_construct(torch.from_numpy(X).cuda(), len(X), kern, opt)
            try:
                H.h2_factor(h1, precision)
                l1, s1 = H.h2_logdet(h1)
                assert s1[0] == sgb[p]
                # FP64: same arithmetic per box; mixed: FP32-accurate factors
                rel = 1e-9 if precision == H.H2_FP64 else 1e-6
                assert abs(l1[0] - ldb[p]) <= rel * abs(l1[0])
            finally:
                H.h2_destroy(h1)
    finally:
        H.h2_destroy(hb)


@pytest.mark.parametrize("precision", [H.H2_FP64, H.H2_MIXED])
def test_batched_workload_per_problem_right_hand_sides(precision):
    """The batched workload's own problems: the 8 smallest of the 64 seeded
    problems (N log-uniform in [2 048, 65 536], cube / sphere / ellipsoid
    surfaces, Laplace, leaf 256 so leaves hold 128-256 points, tol 1e-8),
    each with its own number of right-hand sides (1-256), solved in one
    batched call; every problem's every column reaches the target on its own
    norm and matches the oracle's refined solution."""
    probs = synth.batched_problems(64)
    sel = sorted(range(64), key=lambda p: len(probs[p]["points"]))[:8]
    Xs = [probs[p]["points"] for p in sel]
    nr = [probs[p]["nrhs"] for p in sel]
    assert len(set(nr)) > 1
    opt = H.make_options(leaf=256, tol=1e-8, max_rank=128)
    hb = H.h2_construct_batched([torch.from_numpy(X).cuda() for X in Xs], H.make_kernel("laplace"), opt)
    try:
        H.h2_factor(hb, precision)
        Bs = [synth.rhs(len(X), k, 300 + q) for q, (X, k) in enumerate(zip(Xs, nr))]
        bt = [torch.from_numpy(np.ascontiguousarray(B.T)).cuda() for B in Bs]   # column-major N x k
        xt = [torch.zeros_like(b) for b in bt]
        st, ach, it = H.h2_solve_batched(hb, bt, xt, nr, [len(X) for X in Xs], 1e-10, 40)
        assert st == H.H2_OK and np.all(ach <= 1e-10), (st, ach, it)
        for q, X in enumerate(Xs):
            pb = O.Problem(X, "laplace", 256, 1.0, 1e-8, 128)
            xo, rel, _ = O.refine(O.H2Operator(pb), O.ULVFactor(pb), Bs[q], 1e-10, 40)
            xg = xt[q].cpu().numpy().T
            assert xg.shape == xo.shape
            err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
            assert err <= 1e-8, (q, err)
    finally:
        H.h2_destroy(hb)
