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
    the paper's HSS-ULV.  Its solve must agree with dense LU to ~tol."""
    X = line_points(1024, 5)
    tol = 1e-10
    pb = O.Problem(X, "laplace", 64, 1e12, tol, 1 << 30, s0=0)
    assert all(pb.near[pb.L][i] == [i] for i in range(2 ** pb.L))
    op = O.H2Operator(pb)
    A = O.kernel_matrix("laplace", X, X)
    b = np.random.default_rng(6).standard_normal(1024)
    xd = np.linalg.solve(A, b)
    # Householder route (block row formed explicitly): exact to ~tol.
    F1 = O.ULVFactor(pb, literal_fill=True)
    x0 = F1.solve(b)
    assert np.linalg.norm(x0 - xd) / np.linalg.norm(xd) < 1e3 * tol
    assert F1.logdet()[0] == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-10)
    # Gram route (limited to ~sqrt(eps) in the basis): refinement restores it.
    F = O.ULVFactor(pb)
    x, rel, it = O.refine(op, F, b, 1e-12, 10)
    assert rel[0] <= 1e-12
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e3 * tol
    assert F.logdet()[0] == pytest.approx(np.linalg.slogdet(A)[1], rel=1e-8)


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
def test_literal_fill_in_block_row_equals_gram_route():
    X = synth.sphere_ball(1024, 12)
    pb = O.Problem(X, "laplace", 64, 1.0, 1e-6, 40)
    F1 = O.ULVFactor(pb, literal_fill=True)
    F2 = O.ULVFactor(pb, literal_fill=False)
    for (l1, r1), (l2, r2) in zip(F1.rank_log, F2.rank_log):
        assert r1 == r2
    b = np.random.default_rng(1).standard_normal(1024)
    x1, x2 = F1.solve(b), F2.solve(b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-6


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
