"""GPU parity of the factorization itself (not only of refined solutions):
the unrefined ULV solve x = ULV^-1 b (h2_solve with max_iter = 0), the
log-determinant and the ranks, against the oracle on the same seeded inputs.

FP64: against the oracle's default route (Householder fold of the
fill-in and far-field block row, pivoted QR of the triangle, eq. fillu).
Below tol = 2^-20 the GPU takes that route too: ranks agree box for box,
the unrefined solution to 1e-8 and the log-det to 1e-9 (relative).  At and
above 2^-20 the GPU takes the Gram route (pivoted Cholesky of B B^T, its
rank threshold then at least 2^12 roundoffs above the Gram's noise):
ranks and log-det match the paper's route the same way, and the unrefined
solution within the Gram route's own resolution: rounding in B B^T
perturbs R_kk^2 by about eps R_11^2, so at the rank threshold
R_kk >= tol R_11 the basis moves by about eps / tol relative; through the
factorization (condition about 1e2 on these cases) the unrefined solution
moves by at most 1e3 eps / tol.

Mixed precision: the GPU takes the Gram route in FP32 with the basis
tolerance floored at 2^-10 (h2_stats reports it); the reference is the
oracle's FP64 Gram route at that same effective tolerance.  Bounds:
  * log-det: every one of the N pivots of the factorization (each row is
    eliminated exactly once, in a redundant block or in the root) is
    allowed a relative error of 2^7 u_32 (u_32 = 2^-24) in its absolute
    value, so |ld_mixed - ld_oracle| <= N 2^-17;
  * unrefined solve: its H^2 residual is at most twice the oracle's at the
    effective tolerance plus the floor, and its distance to the oracle's
    unrefined solution at most 10 times the effective tolerance;
  * the refined solve reaches 1e-10 in at most 5 corrections.
"""
import json

import numpy as np
import pytest

import synth
from oracle import h2ulv_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402

FLOOR = 2.0 ** -10

CASES = {
    # name: (points, kernel, leaf, tol, max_rank)
    "sphereball4k_yukawa": (lambda: synth.sphere_ball(4096, 21), "yukawa", 128, 1e-10, 128),
    "surfaces8k_laplace": (lambda: synth.surface_union(8192, 4), "laplace", 128, 1e-6, 128),
    "ragged3000": (lambda: synth.sphere_ball(3000, 5), "laplace", 100, 1e-8, 64),
    "surfaces2k_two_levels": (lambda: synth.surface_union(2048, 4), "laplace", 64, 1e-6, 64),
    # leaf 256: n reaches 256 and every rank reaches the cap of 128
    "sphereball16k_leaf256": (lambda: synth.sphere_ball(16384, 21), "yukawa", 256, 1e-10, 128),
    # rank cap 256: parent boxes reach n = r_a + r_b > 256 (up to 512)
    "sphereball16k_rank256": (lambda: synth.sphere_ball(16384, 21), "yukawa", 256, 1e-10, 256),
}

_cache = {}


def oracle(name, route="qr", tol_basis=None):
    key = (name, route, tol_basis)
    if key not in _cache:
        mk, kern, leaf, tol, mr = CASES[name]
        if name not in _cache:
            X = mk()
            _cache[name] = (X, O.Problem(X, kern, leaf, 1.0, tol, mr))
        X, pb = _cache[name]
        _cache[key] = O.ULVFactor(pb, route=route, tol_basis=tol_basis)
    return _cache[name][0], _cache[name][1], _cache[key]


def gpu_factor(name, precision):
    X, pb, _ = oracle(name)
    _, kern, leaf, tol, mr = CASES[name]
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h = H.h2_construct(pts, len(X), H.make_kernel(kern), H.make_options(leaf=leaf, tol=tol, max_rank=mr))
    H.h2_factor(h, precision)
    return h


def unrefined(h, b):
    bt = torch.from_numpy(b).cuda()
    xt = torch.zeros_like(bt)
    st, ach, it = H.h2_solve(h, bt, xt, 1, len(b), 1e300, 0)
    assert st == H.H2_OK and it == 0
    return xt.cpu().numpy()


def gpu_ranks(h):
    st = json.loads(H.h2_stats(h))
    return [H.h2_box_features(h, k, with_ranks=True)[1].tolist() for k in range(st["heights"])], st


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


EPS = np.finfo(np.float64).eps


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_factorization_matches_oracle(name):
    X, pb, fac = oracle(name)
    tol = CASES[name][3]
    gram = tol >= 2.0 ** -20
    N = len(X)
    b = synth.rhs(N, 1, 3)[:, 0].copy()
    h = gpu_factor(name, H.H2_FP64)
    try:
        ranks, st = gpu_ranks(h)
        assert st["basis_route"] == ("gram" if gram else "qr")
        assert st["tol_basis"] == tol
        assert ranks == [r for _, r in fac.rank_log]
        if name == "sphereball16k_leaf256":
            assert max(max(r) for r in ranks) == 128 and pb.L - pb.ltop >= 2
        if name == "sphereball16k_rank256":
            # boxes wider than 256 at the second ULV level, and ranks above 128
            assert max(max(r) for r in ranks) > 128
            assert max(a + b for a, b in zip(ranks[0][0::2], ranks[0][1::2])) > 256
            # the H^2 operator (its bases up to 256 wide) against the oracle's
            op = O.H2Operator(pb)
            xs = synth.rhs(N, 2, 11)
            xt = torch.from_numpy(np.ascontiguousarray(xs.T)).cuda()
            yt = torch.zeros_like(xt)
            H.h2_matvec(h, xt, yt, 2, N)
            assert rel(yt.cpu().numpy().T, op.matvec(xs)) < 1e-11
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= 1e-9 * abs(lo), (ld[0], lo)
        x = unrefined(h, b)
        assert rel(x, fac.solve(b)) <= (1e3 * EPS / tol if gram else 1e-8)
    finally:
        H.h2_destroy(h)


def test_fp64_matches_literal_fill_in_route():
    """Against the oracle's literal route (every fill-in T_{I,K,J} formed
    explicitly, Sec. III-B), at tol 1e-6 on a case with fill-ins at two ULV
    levels (the GPU's Gram route there, within its resolution bound)."""
    name = "surfaces2k_two_levels"
    X, pb, lit = oracle(name, route="literal")
    b = synth.rhs(len(X), 1, 4)[:, 0].copy()
    h = gpu_factor(name, H.H2_FP64)
    try:
        ranks, _ = gpu_ranks(h)
        assert ranks == [r for _, r in lit.rank_log]
        assert any(r < 64 for r in ranks[0])
        ld, sg = H.h2_logdet(h)
        lo, so = lit.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= 1e-9 * abs(lo)
        assert rel(unrefined(h, b), lit.solve(b)) <= 1e3 * EPS / CASES[name][3]
    finally:
        H.h2_destroy(h)


@pytest.mark.parametrize("name", ["sphereball4k_yukawa", "surfaces8k_laplace", "ragged3000",
                                  "surfaces2k_two_levels"])
def test_mixed_factorization_against_oracle_at_effective_tolerance(name):
    X, pb, _ = oracle(name)
    N = len(X)
    teff = max(CASES[name][3], FLOOR)
    _, _, fg = oracle(name, route="gram", tol_basis=teff)
    op = O.H2Operator(pb)
    b = synth.rhs(N, 1, 3)[:, 0].copy()
    h = gpu_factor(name, H.H2_MIXED)
    try:
        _, st = gpu_ranks(h)
        assert st["basis_route"] == "gram" and st["tol_basis"] == pytest.approx(teff)
        ld, sg = H.h2_logdet(h)
        lo, so = fg.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= N * 2.0 ** -17, (ld[0], lo)
        x = unrefined(h, b)
        xo = fg.solve(b)
        r_gpu = np.linalg.norm(b - op.matvec(x)) / np.linalg.norm(b)
        r_orc = np.linalg.norm(b - op.matvec(xo)) / np.linalg.norm(b)
        assert r_gpu <= 2 * r_orc + FLOOR, (r_gpu, r_orc)
        assert rel(x, xo) <= 10 * teff
        bt = torch.from_numpy(b).cuda()
        xt = torch.zeros_like(bt)
        st_, ach, it = H.h2_solve(h, bt, xt, 1, N, 1e-10, 30)
        assert st_ == H.H2_OK and ach[0] <= 1e-10 and it <= 5, (st_, ach, it)
    finally:
        H.h2_destroy(h)


def test_spd_matern_covariance_at_the_rank_cap():
    """The covariance workload's kernel and factorization, down-scaled:
    Matern-3/2 (length 0.1, nugget 1e-4) on 16 384 points in the unit cube,
    leaf 256, tol 1e-8, Cholesky-ULV (spd = 1), rank cap 256.  At this
    length scale the tolerance needs more than 256 skeletons per box above
    the leaves, so the bases are truncated at the cap (parent boxes 512
    wide); the GPU must still reproduce the oracle's factorization of the
    same truncated operator: ranks box for box, a positive log-det to 1e-9
    and the unrefined solve to 1e-8."""
    X = synth.cube(16384, 5)
    N = len(X)
    pb = O.Problem(X, "matern32", 256, 1.0, 1e-8, 256)
    fac = O.ULVFactor(pb, spd=True)
    b = synth.rhs(N, 1, 3)[:, 0].copy()
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h = H.h2_construct(pts, N, H.make_kernel("matern32"), H.make_options(leaf=256, tol=1e-8, max_rank=256))
    try:
        H.h2_factor(h, H.H2_FP64, 1)
        ranks, st = gpu_ranks(h)
        assert st["basis_route"] == "qr"
        assert ranks == [r for _, r in fac.rank_log]
        assert max(ranks[-1]) == 256 and max(a + b for a, b in zip(ranks[0][0::2], ranks[0][1::2])) > 256
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == 1 and so == 1 and abs(ld[0] - lo) <= 1e-9 * abs(lo), (ld[0], lo)
        assert rel(unrefined(h, b), fac.solve(b)) <= 1e-8
    finally:
        H.h2_destroy(h)


def test_kmeans_partition_through_the_library():
    """The k-means partition (Sec. V; balanced 2-means splits, partition =
    1) through the library on a surface cloud: the H^2 operator, the ranks,
    the FP64 log-det and the refined solution match the oracle built on the
    same k-means tree."""
    X = synth.surface_union(8192, 4)
    N = len(X)
    pb = O.Problem(X, "laplace", 128, 1.0, 1e-8, 128, partition="kmeans")
    fac = O.ULVFactor(pb)
    op = O.H2Operator(pb)
    pts = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    h = H.h2_construct(pts, N, H.make_kernel("laplace"),
                       H.make_options(leaf=128, tol=1e-8, max_rank=128, partition="kmeans"))
    try:
        xs = synth.rhs(N, 2, 13)
        xt = torch.from_numpy(np.ascontiguousarray(xs.T)).cuda()
        yt = torch.zeros_like(xt)
        H.h2_matvec(h, xt, yt, 2, N)
        assert rel(yt.cpu().numpy().T, op.matvec(xs)) < 1e-11
        H.h2_factor(h, H.H2_FP64)
        ranks, _ = gpu_ranks(h)
        assert ranks == [r for _, r in fac.rank_log]
        ld, sg = H.h2_logdet(h)
        lo, so = fac.logdet()
        assert sg[0] == so and abs(ld[0] - lo) <= 1e-9 * abs(lo)
        b = synth.rhs(N, 1, 3)[:, 0].copy()
        xo, _, _ = O.refine(op, fac, b, 1e-10, 30)
        bt = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bt)
        st, ach, it = H.h2_solve(h, bt, x, 1, N, 1e-10, 30)
        assert st == H.H2_OK and rel(x.cpu().numpy(), xo) <= 1e-8
    finally:
        H.h2_destroy(h)
