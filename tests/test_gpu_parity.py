"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same seeded inputs.  Solutions after refinement are compared (pivot choices
may differ, so factors are not); the H^2 matvec and the log-determinant are
compared directly."""
import numpy as np
import pytest

import synth
from oracle import h2ulv_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402

CASES = {
    # name: (points, kernel, leaf, tol, max_rank)
    "sphereball4k_yukawa": (lambda: synth.sphere_ball(4096, 21), "yukawa", 128, 1e-10, 128),
    "surfaces8k_laplace": (lambda: synth.surface_union(8192, 4), "laplace", 128, 1e-6, 128),
    "ragged3000": (lambda: synth.sphere_ball(3000, 5), "laplace", 100, 1e-8, 64),
    "cube4k_dense": (lambda: synth.cube(4096, 0), "laplace", 256, 1e-8, 128),
    "tiny100": (lambda: synth.cube(100, 9), "laplace", 256, 1e-8, 128),
    "cube4k_matern": (lambda: synth.cube(4096, 5), "matern32", 256, 1e-8, 128),
}

_cache = {}


def oracle_case(name):
    if name not in _cache:
        mk, kern, leaf, tol, mr = CASES[name]
        X = mk()
        pb = O.Problem(X, kern, leaf, 1.0, tol, mr)
        _cache[name] = (X, pb, O.H2Operator(pb), O.ULVFactor(pb))
    return _cache[name]


def gpu_handle(X, kern, leaf, tol, mr):
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    return H.h2_construct(pts, len(X), H.make_kernel(kern), H.make_options(leaf=leaf, tol=tol, max_rank=mr))


@pytest.mark.parametrize("name", list(CASES))
def test_matvec_matches_oracle_operator(name):
    X, pb, op, _ = oracle_case(name)
    _, kern, leaf, tol, mr = CASES[name]
    h = gpu_handle(X, kern, leaf, tol, mr)
    try:
        N = len(X)
        xs = synth.rhs(N, 3, 11)
        x = torch.from_numpy(np.ascontiguousarray(xs.T)).cuda()
        y = torch.zeros_like(x)
        H.h2_matvec(h, x, y, 3, N)
        yg = y.cpu().numpy().T
        yo = op.matvec(xs)
        err = np.linalg.norm(yg - yo) / np.linalg.norm(yo)
        assert err < 1e-11, err
        # one right-hand side takes the double-float near-field pass
        x1 = torch.from_numpy(np.ascontiguousarray(xs[:, 0])).cuda()
        y1 = torch.zeros_like(x1)
        H.h2_matvec(h, x1, y1, 1, N)
        err1 = np.linalg.norm(y1.cpu().numpy() - yo[:, 0]) / np.linalg.norm(yo[:, 0])
        assert err1 < 1e-11, err1
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", [H.H2_FP64, H.H2_MIXED])
def test_refined_solution_matches_oracle(name, precision):
    X, pb, op, fac = oracle_case(name)
    _, kern, leaf, tol, mr = CASES[name]
    N = len(X)
    b = synth.rhs(N, 1, 3)[:, 0].copy()
    xo, relo, ito = O.refine(op, fac, b, 1e-10, 30)
    h = gpu_handle(X, kern, leaf, tol, mr)
    try:
        H.h2_factor(h, precision)
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e-10, 30)
        assert st == H.H2_OK, (st, ach, it)
        assert ach[0] <= 1e-10
        err = np.linalg.norm(xt.cpu().numpy() - xo) / np.linalg.norm(xo)
        bound = 1e-8 if precision == H.H2_FP64 else 10 * tol
        assert err <= max(bound, 1e-8), err
        if precision == H.H2_FP64:
            assert it <= ito + 1
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("name", ["sphereball4k_yukawa", "cube4k_dense", "tiny100"])
def test_logdet_matches_oracle(name):
    X, pb, op, fac = oracle_case(name)
    _, kern, leaf, tol, mr = CASES[name]
    h = gpu_handle(X, kern, leaf, tol, mr)
    try:
        H.h2_factor(h, H.H2_FP64)
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == so
        assert abs(ld[0] - lo) <= 1e-9 * abs(lo), (ld[0], lo)
    finally:
        H.h2_destroy(h)


def test_host_buffers_multiple_rhs():
    X, pb, op, fac = oracle_case("ragged3000")
    _, kern, leaf, tol, mr = CASES["ragged3000"]
    N = len(X)
    B = synth.rhs(N, 4, 8)
    Bc = np.ascontiguousarray(B.T)          # column-major N x 4, host
    Xc = np.zeros_like(Bc)
    h = H.h2_construct(np.ascontiguousarray(X), N, H.make_kernel(kern), H.make_options(leaf=leaf, tol=tol, max_rank=mr))
    try:
        H.h2_factor(h, H.H2_FP64)
        st, ach, it = H.h2_solve(h, Bc, Xc, 4, N, 1e-10, 30)
        assert st == H.H2_OK and np.all(ach <= 1e-10)
        xo, _, _ = O.refine(op, fac, B, 1e-10, 30)
        err = np.linalg.norm(Xc.T - xo) / np.linalg.norm(xo)
        assert err <= 1e-8, err
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("name", ["sphereball4k_yukawa", "cube4k_matern"])
def test_spd_path_matches_oracle_cholesky(name):
    """spd = 1: redundant blocks and the root are factored without pivoting
    with positive pivots (the LDL^T form of the Cholesky-ULV); the log-det
    equals the oracle's Cholesky factorization's.  The Matern-3/2 case (plus
    the nugget on the diagonal) is the covariance workload's kernel."""
    X, pb, op, fac = oracle_case(name)
    _, kern, leaf, tol, mr = CASES[name]
    facs = O.ULVFactor(pb, spd=True)
    N = len(X)
    b = synth.rhs(N, 1, 3)[:, 0].copy()
    xo, _, _ = O.refine(op, facs, b, 1e-10, 30)
    h = gpu_handle(X, kern, leaf, tol, mr)
    try:
        H.h2_factor(h, H.H2_FP64, 1)
        ld, sg = H.h2_logdet(h)
        lo, so = facs.logdet()
        assert sg[0] == 1 and abs(ld[0] - lo) <= 1e-9 * abs(lo)
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e-10, 30)
        assert st == H.H2_OK
        assert np.linalg.norm(xt.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("precision", [H.H2_FP64, H.H2_MIXED])
def test_64_right_hand_sides(precision):
    """64 right-hand sides (the Yukawa workload's block solve): more than 8
    columns take the stationary refinement x <- x + ULV^-1 (b - A_H2 x)
    column block at once; every column reaches the target and matches the
    oracle's refined solution."""
    X, pb, op, fac = oracle_case("sphereball4k_yukawa")
    _, kern, leaf, tol, mr = CASES["sphereball4k_yukawa"]
    N = len(X)
    B = synth.rhs(N, 64, 12)
    h = gpu_handle(X, kern, leaf, tol, mr)
    try:
        H.h2_factor(h, precision)
        bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
        xt = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, xt, 64, N, 1e-10, 40)
        assert st == H.H2_OK and np.all(ach <= 1e-10), (st, ach.max(), it)
        xo, _, _ = O.refine(op, fac, B, 1e-10, 30)
        err = np.linalg.norm(xt.cpu().numpy().T - xo) / np.linalg.norm(xo)
        assert err <= 1e-8, err
    finally:
        H.h2_destroy(h)


def test_hss_special_case_weak_admissibility():
    """eta -> infinity on a line: distinct boxes are far from the first level
    below the root on (weak admissibility), there are no fill-ins, and the
    method reduces to the paper's HSS-ULV (Sec. II-C).  Exact far-field block
    rows (far_s0 = 0), tol 1e-10.  The FP64 factorization's log-det and its
    unrefined solution match the oracle's (and dense LU, which the oracle
    matches to rounding here); the refined solution matches too."""
    X = synth.line(1024, 5)
    N = len(X)
    pb = O.Problem(X, "laplace", 64, 1e12, 1e-10, 128, s0=0)
    assert all(pb.near[pb.L][i] == [i] for i in range(2 ** pb.L))
    op, fac = O.H2Operator(pb), O.ULVFactor(pb)
    b = synth.rhs(N, 1, 9)[:, 0].copy()
    xo, _, _ = O.refine(op, fac, b, 1e-10, 30)
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h = H.h2_construct(pts, N, H.make_kernel("laplace"),
                       H.make_options(eta=1e12, leaf=64, tol=1e-10, max_rank=128, far_s0=0, far_smin=1))
    try:
        H.h2_factor(h, H.H2_FP64)
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e300, 0)      # unrefined ULV solve
        assert st == H.H2_OK and it == 0
        x0 = fac.solve(b)
        assert np.linalg.norm(xt.cpu().numpy() - x0) / np.linalg.norm(x0) <= 1e-8
        st, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e-10, 30)
        assert st == H.H2_OK and ach[0] <= 1e-10, (st, ach, it)
        assert np.linalg.norm(xt.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-8
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= 1e-9 * abs(lo), (ld[0], lo)
        sd, ldd = np.linalg.slogdet(O.kernel_matrix("laplace", X, X))
        assert sd == sg[0] and abs(ld[0] - ldd) <= 1e-9 * abs(ldd), (ld[0], ldd)
    finally:
        H.h2_destroy(h)


def test_blr2_special_case_one_level():
    """One level (L = 1): the two halves of a line are far from each other,
    so the method is the paper's BLR^2-ULV (Sec. II-B, eq. lu ... eq.
    BLR2final): one basis, one partial LU per box (n = 256), and the dense
    LU of the merged skeletons.  Log-det and unrefined solution against the
    oracle (which matches dense LU here)."""
    X = synth.line(512, 13)
    N = len(X)
    pb = O.Problem(X, "yukawa", 256, 1e12, 1e-10, 128, s0=0)
    assert pb.L == 1 and pb.ltop == 0
    fac = O.ULVFactor(pb)
    b = synth.rhs(N, 1, 10)[:, 0].copy()
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h = H.h2_construct(pts, N, H.make_kernel("yukawa"),
                       H.make_options(eta=1e12, leaf=256, tol=1e-10, max_rank=128, far_s0=0, far_smin=1))
    try:
        H.h2_factor(h, H.H2_FP64)
        F, R = H.h2_box_features(h, 0, with_ranks=True)
        assert R.tolist() == fac.rank_log[0][1]
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= 1e-9 * abs(lo), (ld[0], lo)
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e300, 0)
        x0 = fac.solve(b)
        assert st == H.H2_OK and np.linalg.norm(xt.cpu().numpy() - x0) / np.linalg.norm(x0) <= 1e-8
    finally:
        H.h2_destroy(h)
