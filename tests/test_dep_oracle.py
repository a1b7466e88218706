"""Pins of the H^2-ULV reference WITH trailing dependencies (Sec. II-D,
eq. u2 / eq. v2; oracle/h2ulv_dep_oracle.py), against the dense solution and
log-determinant, and its ranks beside the dependency-free factorization's.

The far field is exact here (s0 = 0), so the only approximation is the rank
truncation at tol: near-exact at tol 1e-12, within tol at 1e-6 and 1e-8."""
import numpy as np
import pytest

import synth
from oracle import h2ulv_oracle as O
from oracle.h2ulv_dep_oracle import DependentULV


def _case(kind, tol):
    if kind == "line":
        X, kern, leaf = synth.line(1024, 3), "laplace", 32
    else:
        X, kern, leaf = synth.surface_union(2048, 7), "laplace", 64
    pb = O.Problem(X, kern, leaf, 1.0, tol, 4096, s0=0, s_min=0)
    A = O.kernel_matrix(kern, X, X, same=True)
    b = np.random.default_rng(1).standard_normal(len(X))
    return pb, A, b


def _errors(f, A, b):
    xd = np.linalg.solve(A, b)
    e = np.linalg.norm(f.solve(b) - xd) / np.linalg.norm(xd)
    sd, ldd = np.linalg.slogdet(A)
    ld, sg = f.logdet()
    return e, abs(ld - ldd) / abs(ldd), sg == sd


@pytest.mark.parametrize("kind", ["line", "union"])
def test_dependent_ulv_is_near_exact_at_tiny_tol(kind):
    pb, A, b = _case(kind, 1e-12)
    f = DependentULV(pb)
    assert pb.L > pb.ltop
    # every level compresses: some box eliminates a redundant part
    for (_, r), (_, n) in zip(f.rank_log, f.size_log):
        assert any(ri < ni for ri, ni in zip(r, n))
    e, lde, same_sign = _errors(f, A, b)
    assert e <= 1e-11 and lde <= 1e-12 and same_sign, (e, lde)


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_dependent_ulv_error_within_tol(tol):
    pb, A, b = _case("line", tol)
    f = DependentULV(pb)
    assert len(f.rank_log) == pb.L - pb.ltop >= 3
    e, lde, same_sign = _errors(f, A, b)
    assert e <= tol and lde <= tol and same_sign, (e, lde)
    assert f.dropped <= 10 * tol


def test_dependent_ulv_spd_cholesky():
    X = synth.line(1024, 3)
    pb = O.Problem(X, "matern32", 32, 1.0, 1e-8, 4096, s0=0, s_min=0)
    A = O.kernel_matrix("matern32", X, X, same=True)
    b = np.random.default_rng(2).standard_normal(len(X))
    f = DependentULV(pb, spd=True)
    e, lde, same_sign = _errors(f, A, b)
    assert e <= 1e-8 and lde <= 1e-12 and same_sign, (e, lde)


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_dependency_free_bases_carry_more_rank(tol):
    """Sec. III-C builds one shared basis per box that has to hold, from the
    start, every fill-in block the factorization could create as well as the
    low-rank blocks; the method with dependencies only absorbs the fill-ins
    that its eliminations actually create (Sec. II-D).  Sec. IV notes that
    shared, nested bases raise the ranks.  With the same tree, tolerance and
    exact far field, the dependency-free ranks are larger at every level."""
    pb, A, b = _case("line", tol)
    dep = DependentULV(pb)
    free = O.ULVFactor(pb)
    rd = {l: np.mean(r) for l, r in dep.rank_log}
    rf = {l: np.mean(r) for l, r in free.rank_log}
    assert rd.keys() == rf.keys()
    assert all(rf[l] > rd[l] for l in rd), (rd, rf)
