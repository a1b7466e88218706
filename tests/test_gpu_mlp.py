"""Rank-predictor MLP on the GPU: gradients of the library's own backward
kernel against the CPU oracle, training on the GPU, and the trained
predictor inside the factorization: the solution is unchanged (pivoted QR
still decides every rank) and its storage estimate is tighter than the
rank-cap bound.  The factorization without a predictor sizes its storage
exactly after the rank readback, so the predictor has no time or memory
advantage over that path."""
import json

import numpy as np
import pytest

import synth
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2208_10907_gb300 import h2ulv as H  # noqa: E402


def init_params(seed):
    # the caller draws the initial parameters (scaled Gaussians)
    rng = np.random.default_rng(seed)
    P = M.param_count(8)
    p = np.zeros(P)
    W1, b1, W2, b2, w3, b3, _ = M.unpack(np.arange(P, dtype=float), 8)
    p[:512] = rng.standard_normal(512) / np.sqrt(8)
    p[576:576 + 4096] = rng.standard_normal(4096) / np.sqrt(64)
    p[4736:4800] = rng.standard_normal(64) / np.sqrt(64)
    return p.astype(np.float32)


def test_gpu_gradient_matches_oracle():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((700, 8)).astype(np.float32)
    T = rng.standard_normal(700).astype(np.float32)
    p = init_params(1)
    m = H.h2_mlp_create(p)
    try:
        g, loss = H.h2_mlp_gradient(m, X, T)
        lo, go = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
        assert abs(loss - lo) <= 1e-5 * abs(lo)
        assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
        np.testing.assert_array_equal(H.h2_mlp_params(m), p)   # the gradient call does not step
    finally:
        H.h2_mlp_destroy(m)


def test_gpu_training_reduces_loss():
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (1500, 8)).astype(np.float32)
    T = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    m = H.h2_mlp_create(init_params(2))
    try:
        l0 = H.h2_mlp_train(m, X, T, 0)
        l1 = H.h2_mlp_train(m, X, T, 400, 3e-3)
        assert l1 < 0.1 * l0, (l0, l1)
        y = H.h2_mlp_forward(m, X)
        yo, _, _ = M.forward(H.h2_mlp_params(m).astype(np.float64), X.astype(np.float64))
        np.testing.assert_allclose(y, yo, atol=2e-5, rtol=1e-4)
    finally:
        H.h2_mlp_destroy(m)


def _problem(seed, n=16384):
    X = synth.surface_union(n, seed)
    pts = torch.from_numpy(X).cuda()
    h = H.h2_construct(pts, n, H.make_kernel("laplace"), H.make_options(leaf=128, tol=1e-6, far_s0=16, far_smin=2))
    return X, h


def _heights(h):
    return json.loads(H.h2_stats(h))["heights"]


def test_rank_predictor_trained_on_pivoted_qr_ranks():
    feats, ranks = [], []
    for seed in range(1000, 1010):
        X, h = _problem(seed)
        try:
            H.h2_factor(h, H.H2_MIXED)
            for ht in range(_heights(h)):
                F, R = H.h2_box_features(h, ht, with_ranks=True)
                feats.append(F)
                ranks.append(R)
        finally:
            H.h2_destroy(h)
    F = np.concatenate(feats)
    R = np.concatenate(ranks).astype(np.float32) / 128.0
    assert len(F) >= 1000
    m = H.h2_mlp_create(init_params(5))
    try:
        H.h2_mlp_train(m, F, R, 1500, 3e-3)
        # held-out problem
        X, h = _problem(2000)
        try:
            H.h2_factor(h, H.H2_MIXED)
            b = torch.from_numpy(synth.rhs(len(X), 1, 7)[:, 0].copy()).cuda()
            x0 = torch.zeros_like(b)
            H.h2_solve(h, b, x0, 1, len(X), 1e-10, 30)
            Fh = np.concatenate([H.h2_box_features(h, t) for t in range(_heights(h))])
            Rh = np.concatenate([H.h2_box_features(h, t, True)[1] for t in range(_heights(h))])
            pred = H.h2_mlp_forward(m, Fh) * 128.0
            mae = np.mean(np.abs(pred - Rh))
            base = np.mean(np.abs(Rh - np.mean(R) * 128.0))
            assert mae < 0.5 * base, (mae, base)      # better than predicting the mean rank
            # the factorization with the predictor attached
            H.h2_set_rank_predictor(h, m, 0.15)
            H.h2_factor(h, H.H2_MIXED)
            st = json.loads(H.h2_stats(h))["predictor"]
            x1 = torch.zeros_like(b)
            H.h2_solve(h, b, x1, 1, len(X), 1e-10, 30)
            assert torch.equal(x0, x1)                 # pivoted QR still decides every rank
            assert st["hits"] >= 1
            assert st["presized_bytes"] < 0.5 * st["worstcase_bytes"], st   # tighter than the cap bound
        finally:
            H.h2_destroy(h)
    finally:
        H.h2_mlp_destroy(m)
