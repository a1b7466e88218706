"""Pins of the CPU oracle against facts fixed by the paper and by
mathematics: closed forms, textbook routines, invariants, special cases that
reduce to dense LU or to HSS-ULV, and brute force on small inputs."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import h2ulv_oracle as O


def line_points(n, seed):
    x = np.sort(np.random.default_rng(seed).random(n))
    return np.stack([x, np.zeros(n), np.zeros(n)], 1)


# ---------------------------------------------------------------- kernels --
def test_kernel_closed_forms():
    X = np.array([[0.0, 0, 0], [3.0, 4.0, 0.0]])
    K = O.kernel_matrix("laplace", X, X)
    assert K[0, 0] == pytest.approx(1e3)
    assert K[0, 1] == pytest.approx(1.0 / 5.001)
    Y = O.kernel_matrix("yukawa", X, X)
    assert Y[0, 1] == pytest.approx(np.exp(-5.0) / 5.001)
    M = O.kernel_matrix("matern32", X, X)
    assert M[0, 0] == pytest.approx(1.0 + 1e-4)
    s = np.sqrt(3.0) * 5.0 / 0.1
    assert M[0, 1] == pytest.approx((1 + s) * np.exp(-s), rel=1e-12, abs=1e-300)


# ------------------------------------------------------------------- tree --
def test_tree_partition_and_bisection():
    X = synth.cube(3000, 7)
    L, perm, boxes = O.cluster_tree(X, 100)
    assert L == 5 and sorted(perm) == list(range(3000))
    sizes = [e - s for s, e in boxes[L]]
    assert min(sizes) > 50 and max(sizes) <= 100
    Xt = X[perm]
    for l in range(L):
        for p, (s, e) in enumerate(boxes[l]):
            (s1, e1), (s2, e2) = boxes[l + 1][2 * p], boxes[l + 1][2 * p + 1]
            assert s1 == s and e2 == e and e1 == s2 and (e1 - s1) == (e - s) // 2
            ext = Xt[s:e].max(0) - Xt[s:e].min(0)
            ax = int(np.argmax(ext))
            assert Xt[s1:e1, ax].max() <= Xt[s2:e2, ax].min()


def test_block_partition_covers_matrix_once():
    """Strong admissibility partition: every leaf pair (i, j) lies in exactly
    one block (a leaf near pair or one far pair at some level)."""
    X = synth.sphere_ball(2048, 3)
    L, perm, boxes = O.cluster_tree(X, 32)
    Xt = X[perm]
    near, far = O.interaction_lists(Xt, boxes, L, 1.0)
    cover = np.zeros((2 ** L, 2 ** L), dtype=int)
    for l in range(1, L + 1):
        span = 2 ** (L - l)
        for i in range(2 ** l):
            for j in far[l][i]:
                assert O.admissible(O.box_bounds(Xt, [boxes[l]])[0][i],
                                    O.box_bounds(Xt, [boxes[l]])[0][j], 1.0)
                cover[i * span:(i + 1) * span, j * span:(j + 1) * span] += 1
    for i in range(2 ** L):
        for j in near[L][i]:
            cover[i, j] += 1
    assert np.all(cover == 1)
    # symmetry of the lists
    for l in range(L + 1):
        for i in range(2 ** l):
            for j in near[l][i]:
                assert i in near[l][j]
            for j in far[l][i]:
                assert i in far[l][j]


def test_far_samples_rule():
    X = synth.sphere_ball(4096, 2)
    pb = O.Problem(X, "laplace", 64, 1.0, 1e-8, 64)
    l, i = pb.L, 5
    fs = pb.samples(l, i)
    near_pts = set()
    for j in pb.near[l][i]:
        s, e = pb.boxes[l][j]
        near_pts.update(range(s, e))
    assert not (set(fs.tolist()) & near_pts)
    assert len(set(fs.tolist())) == len(fs)
    exact = O.far_samples(pb.boxes, pb.far, l, i, s0=0)
    assert len(exact) + sum(e - s for j in pb.near[l][i] for (s, e) in [pb.boxes[l][j]]) == 4096


def _golden(name):
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", name)))


def test_far_samples_positions_hand_computed():
    """Positions of the deterministic far-field sample of one leaf, its far
    lists at every level and l_top, against values worked out by hand
    (fixture tests/golden/far_samples_line64.json, with its derivation)."""
    fx = _golden("far_samples_line64.json")
    X = np.stack([np.arange(64.0), np.zeros(64), np.zeros(64)], 1)
    pb = O.Problem(X, "laplace", 4, 1.0, 1e-8, 4, s0=fx["s0"], s_min=fx["s_min"])
    assert pb.L == 4 and list(pb.perm) == list(range(64))
    i = fx["box"]
    for lev, lst in fx["far"].items():
        a = i >> (pb.L - int(lev))
        assert pb.far[int(lev)][a] == lst, (lev, pb.far[int(lev)][a])
    got = O.far_samples(pb.boxes, pb.far, fx["level"], i, fx["s0"], fx["s_min"])
    assert got.tolist() == fx["samples"]
    assert pb.ltop == fx["l_top"]


def test_admissibility_closed_forms():
    """O-2 on unit boxes: max(diam) = sqrt(3); a face gap of 2 is far for
    eta = 1 and near for eta = 0.8 (0.8 * 2 < sqrt(3)); a corner gap of
    sqrt(3) sits exactly on the boundary (far for eta = 1, near just below)."""
    u = (np.zeros(3), np.ones(3))
    face = (np.array([3.0, 0, 0]), np.array([4.0, 1, 1]))
    corner = (np.full(3, 2.0), np.full(3, 3.0))
    overlap = (np.full(3, 0.5), np.full(3, 1.5))
    assert O.admissible(u, face, 1.0) and not O.admissible(u, face, 0.8)
    assert O.admissible(u, corner, 1.0) and not O.admissible(u, corner, 0.999)
    assert not O.admissible(u, overlap, 1e12)


# ------------------------------------------------------ pivoted QR and ID --
def _lowrank(m, n, r, seed):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((m, r)))[0]
    V = np.linalg.qr(rng.standard_normal((n, r)))[0]
    s = np.logspace(0, -12, r)
    return (U * s) @ V.T


def test_pivoted_qr_matches_lapack_geqp3():
    B = np.random.default_rng(4).standard_normal((60, 40)) * np.logspace(0, -3, 40)
    piv, R, rk = O.pivoted_qr(B, 0.0, 1000)
    Q2, R2, P2 = sla.qr(B, pivoting=True)
    assert rk == 40
    np.testing.assert_array_equal(piv, P2)
    np.testing.assert_allclose(np.abs(np.diag(R)), np.abs(np.diag(R2)), rtol=1e-10)


def test_pivoted_cholesky_equals_pivoted_qr_of_transpose():
    B = _lowrank(50, 300, 35, 9)        # block row, n = 50 rows
    p1, R1, r1 = O.pivoted_qr(B.T, 1e-6, 100)
    p2, R2, r2 = O.pivoted_cholesky(B @ B.T, 1e-6, 100)
    assert r1 == r2
    np.testing.assert_array_equal(p1[:r1], p2[:r2])
    np.testing.assert_allclose(np.abs(R1), np.abs(R2), rtol=1e-6, atol=1e-9 * abs(R1[0, 0]))


def test_fold_rows_keeps_pivoted_qr():
    B = _lowrank(40, 500, 30, 3)
    p1, R1, r1 = O.pivoted_qr(B.T, 1e-8, 100)
    p2, R2, r2 = O.pivoted_qr(O.fold_rows(B.T), 1e-8, 100)
    assert r1 == r2
    np.testing.assert_array_equal(p1[:r1], p2[:r2])
    np.testing.assert_allclose(np.abs(R1), np.abs(R2), rtol=1e-8, atol=1e-12)


def test_interpolative_decomposition_error_bound():
    B = _lowrank(64, 400, 40, 5)
    tol = 1e-7
    piv, R, rk = O.pivoted_qr(B.T, tol, 1000)
    P = O.interpolation_matrix(piv, R, rk, 64)
    np.testing.assert_allclose(P[piv[:rk]], np.eye(rk), atol=0)
    err = np.linalg.norm(B - P @ B[piv[:rk]], 2)
    assert err <= 64 * tol * abs(R[0, 0])
    # rank rule: the next pivot is below tol
    full_piv, full_R, _ = O.pivoted_qr(B.T, 0.0, 1000)
    assert abs(full_R[rk, rk]) <= tol * abs(full_R[0, 0]) < abs(full_R[rk - 1, rk - 1])


# ---------------------------------------------------- special-case solves --
def test_dense_special_case_n_le_leaf():
    X = synth.cube(200, 1)
    pb = O.Problem(X, "laplace", 256, 1.0, 1e-8, 128)
    assert pb.L == 0
    F = O.ULVFactor(pb)
    A = O.kernel_matrix("laplace", X, X)
    b = np.random.default_rng(2).standard_normal(200)
    np.testing.assert_allclose(F.solve(b), np.linalg.solve(A, b), rtol=1e-10)
    sg, ld = np.linalg.slogdet(A)
    assert F.logdet()[0] == pytest.approx(ld, rel=1e-12) and F.logdet()[1] == sg


def test_all_near_degenerates_to_dense_lu():
    """At N = 4096 in the unit cube with leaf 256 and eta = 1 every leaf pair
    is near, so l_top = L and the whole matrix is one dense LU."""
    X = synth.cube(4096, 0)
    pb = O.Problem(X, "laplace", 256, 1.0, 1e-8, 128)
    assert pb.L == 4 and pb.ltop == 4


def test_hss_special_case_matches_dense():
    """Points on a line with eta -> infinity: every off-diagonal pair is far
    at level 1 (weak admissibility), there are no fill-ins and the method is
    the paper's HSS-ULV (Sec. II-C).  Its solve and log-det must agree with
    dense LU to about tol."""
    X = line_points(1024, 5)
    tol = 1e-10
    pb = O.Problem(X, "laplace", 64, 1e12, tol, 1 << 30, s0=0)
    assert all(pb.near[pb.L][i] == [i] for i in range(2 ** pb.L))
    assert pb.ltop == 0 and pb.L == 4
    op = O.H2Operator(pb)
    A = O.kernel_matrix("laplace", X, X)
    b = np.random.default_rng(6).standard_normal(1024)
    xd = np.linalg.solve(A, b)
    ld_dense = np.linalg.slogdet(A)[1]
    # the paper's route (Householder QR of the block row, default) and the
    # literal one: exact to about tol, unrefined
    for route in ("qr", "literal"):
        F1 = O.ULVFactor(pb, route=route)
        assert all(0 < r < 64 for r in F1.rank_log[0][1])
        x0 = F1.solve(b)
        assert np.linalg.norm(x0 - xd) / np.linalg.norm(xd) < 1e3 * tol
        assert F1.logdet()[0] == pytest.approx(ld_dense, rel=1e-12)
    # Gram route (limited to ~sqrt(eps) in the basis): refinement restores it.
    F = O.ULVFactor(pb, route="gram")
    x, rel, it = O.refine(op, F, b, 1e-12, 10)
    assert rel[0] <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e3 * tol
    assert F.logdet()[0] == pytest.approx(ld_dense, rel=1e-8)


def test_blr2_special_case_one_level():
    """One level (L = 1) with the two halves far from each other: the
    paper's BLR^2-ULV (Sec. II-B, eq. lu ... eq. BLR2final) with shared
    bases, one partial LU per box and the dense LU of the merged skeleton
    matrix.  No fill-ins; exact to about tol against dense LU."""
    X = line_points(512, 13)
    tol = 1e-10
    pb = O.Problem(X, "yukawa", 256, 1e12, tol, 256, s0=0)
    assert pb.L == 1 and pb.ltop == 0 and pb.far[1] == [[1], [0]]
    F = O.ULVFactor(pb)
    (l, r), = F.rank_log
    assert l == 1 and all(0 < q < 256 for q in r)
    assert F.root_dense.shape == (sum(r), sum(r))
    A = O.kernel_matrix("yukawa", X, X)
    b = np.random.default_rng(14).standard_normal(512)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(F.solve(b) - xd) / np.linalg.norm(xd) < 1e3 * tol
    sg, ld = np.linalg.slogdet(A)
    assert F.logdet()[0] == pytest.approx(ld, rel=1e-12) and F.logdet()[1] == sg


def test_orthonormal_bases():
    X = synth.sphere_ball(2048, 4)
    pb = O.Problem(X, "laplace", 64, 1.0, 1e-8, 48)
    F = O.ULVFactor(pb)
    for lev in F.levels:
        for Q in lev["Q"]:
            assert np.linalg.norm(Q.T @ Q - np.eye(len(Q))) < 1e-13


# --------------------------------------------------------- H2 operator ----
@pytest.mark.parametrize("s0", [0, 32])
def test_h2_operator_accuracy(s0):
    X = synth.sphere_ball(2048, 8)
    tol = 1e-8
    pb = O.Problem(X, "laplace", 64, 1.0, tol, 1 << 30, s0=s0)
    op = O.H2Operator(pb)
    A = O.kernel_matrix("laplace", X, X)[np.ix_(pb.perm, pb.perm)]
    H = op.dense()
    assert np.linalg.norm(H - A) / np.linalg.norm(A) < 10 * tol
    x = np.random.default_rng(0).standard_normal(2048)
    assert np.linalg.norm(op.matvec(x) - O.kernel_matrix("laplace", X, X) @ x) \
        <= 10 * tol * np.linalg.norm(A) * np.linalg.norm(x)


# ---------------------------------------------------------- fill-in forms --
def test_fill_in_routes_agree_on_a_multilevel_case():
    """The three forms of the fill-in block row (eq. fillu) on a surface
    cloud with two ULV levels and fill-ins at both (N = 2048, leaf 64,
    tol 1e-6): the default route (per-K QR compression of the fill-in rows)
    and the literal one (every T_{I,K,J} formed) choose the same ranks and
    give the same factorization to rounding; the Gram route agrees at this
    tolerance (above its sqrt(eps) resolution)."""
    X = synth.surface_union(2048, 4)
    pb = O.Problem(X, "laplace", 64, 1.0, 1e-6, 64)
    assert pb.L - pb.ltop == 2
    F1 = O.ULVFactor(pb, route="literal")
    F2 = O.ULVFactor(pb, route="qr")
    F3 = O.ULVFactor(pb, route="gram")
    assert any(r < 64 for r in F1.rank_log[0][1])        # something is eliminated
    for (l1, r1), (l2, r2), (l3, r3) in zip(F1.rank_log, F2.rank_log, F3.rank_log):
        assert r1 == r2 == r3
    assert F2.logdet()[0] == pytest.approx(F1.logdet()[0], rel=1e-13)
    assert F3.logdet()[0] == pytest.approx(F1.logdet()[0], rel=1e-10)
    b = np.random.default_rng(1).standard_normal(2048)
    x1, x2, x3 = F1.solve(b), F2.solve(b), F3.solve(b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-11
    assert np.linalg.norm(x1 - x3) / np.linalg.norm(x1) < 1e-6


# ------------------------------------------------ brute force, small N ----
@pytest.mark.parametrize("kind,tol", [("laplace", 1e-8), ("yukawa", 1e-10)])
def test_refined_solution_matches_dense(kind, tol):
    X = synth.sphere_ball(4096, 21)
    pb = O.Problem(X, kind, 128, 1.0, tol, 128)
    assert pb.L > pb.ltop
    op = O.H2Operator(pb)
    F = O.ULVFactor(pb)
    A = O.kernel_matrix(kind, X, X)
    b = np.random.default_rng(22).standard_normal(4096)
    xd = np.linalg.solve(A, b)
    x, rel, it = O.refine(op, F, b, 1e-10, 20)
    assert rel[0] <= 1e-10 and it <= 6
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 100 * tol
    ld = F.logdet()[0]
    assert ld == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-6)


def test_spd_cholesky_path():
    X = synth.cube(1024, 30)
    pb = O.Problem(X, "matern32", 64, 1.0, 1e-10, 1 << 30, s0=0)
    F = O.ULVFactor(pb, spd=True)
    A = O.kernel_matrix("matern32", X, X)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    b = np.random.default_rng(3).standard_normal(1024)
    op = O.H2Operator(pb)
    x, rel, it = O.refine(op, F, b, 1e-10, 30)
    xd = np.linalg.solve(A, b)
    assert rel[0] <= 1e-10
    assert F.logdet()[0] == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-6)


def test_fill_in_set_matches_paper_example():
    """The paper's worked example of the fill-in pre-computation (fixture
    tests/golden/fill_in_example.json, with its citation): eliminating the
    other boxes of the first block row/column fills exactly A_{0,2}, A_{2,0}
    and A_{0,0}.  Dropping the J = i terms (reading B) would miss A_{0,0};
    counting K = i would add the dense blocks themselves."""
    import json
    import os
    fx = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fill_in_example.json")))
    got = O.fill_in_blocks(fx["near"], fx["row"])
    assert [list(p) for p in got] == fx["fill_in"]


# ------------------------------------------------------- k-means tree -----
def test_balanced_two_means_separates_two_blobs():
    """Two equal, well separated blobs: the balanced 2-means split puts each
    blob in one child, whichever blob the seeds start from."""
    rng = np.random.default_rng(40)
    A = rng.normal(0.0, 0.1, (50, 3))
    B = rng.normal(0.0, 0.1, (50, 3)) + np.array([5.0, 0.0, 0.0])
    X = np.vstack([A, B])[rng.permutation(100)]
    order, it = O.balanced_two_means(X, np.arange(100))
    left, right = set(order[:50].tolist()), set(order[50:].tolist())
    blob_a = set(np.flatnonzero(X[:, 0] < 2.5).tolist())
    assert left == blob_a or right == blob_a
    assert it < 20


def test_balanced_two_means_line_closed_form():
    """Points 0, 1, 2 and 10, 11, 12 on a line: the split is {0,1,2} | {10,11,12}
    in one Lloyd step, and the order within a child follows the key."""
    X = np.zeros((6, 3))
    X[:, 0] = [10.0, 0.0, 11.0, 2.0, 12.0, 1.0]
    order, it = O.balanced_two_means(X, np.arange(6))
    assert set(order[:3].tolist()) in ({1, 3, 5}, {0, 2, 4})
    assert set(order[3:].tolist()) == {0, 1, 2, 3, 4, 5} - set(order[:3].tolist())


def test_kmeans_tree_is_balanced_and_a_lloyd_fixed_point():
    """Every split is balanced (floor(n/2) left) and, where the iteration
    stopped before its cap, is a fixed point of the Lloyd step: recomputing
    both centroids from the children and reassigning gives the same children."""
    X = synth.surface_union(3000, 11)
    L, perm, boxes = O.cluster_tree_kmeans(X, 100)
    assert sorted(perm) == list(range(3000))
    for l in range(L):
        for p, (s, e) in enumerate(boxes[l]):
            (s1, e1), (s2, e2) = boxes[l + 1][2 * p], boxes[l + 1][2 * p + 1]
            assert s1 == s and e2 == e and e1 - s1 == (e - s) // 2
            order, it = O.balanced_two_means(X, perm[s:e])
            # the tree's children are that split (their order is refined further down)
            assert set(order[:e1 - s1].tolist()) == set(perm[s1:e1].tolist())
            if it < 20:
                Pl, Pr = X[perm[s1:e1]], X[perm[s2:e2]]
                c0, c1 = Pl.mean(0), Pr.mean(0)
                idx = np.sort(perm[s:e])
                P = X[idx]
                key = ((P - c0) ** 2).sum(1) - ((P - c1) ** 2).sum(1)
                left = set(idx[np.lexsort((idx, key))[:e1 - s1]].tolist())
                assert left == set(perm[s1:e1].tolist())
