"""Plain FP64 CPU reference of the H^2-ULV factorization WITH trailing
dependencies (Sec. II-D, eq. u2 / eq. v2).

TEST INFRASTRUCTURE ONLY, like ``h2ulv_oracle``: only ``tests/`` may import
it.  It is the serial method that the paper's dependency-free factorization
replaces, kept here as a rank and accuracy reference for the readings of the
dependency-free method (O-5: which fill-ins enter the basis; O-7: which
blocks are eliminated).  It shares the cluster tree, admissibility and
kernels of ``h2ulv_oracle.Problem`` and nothing of the CUDA library.

The method, per level l = L .. l_top+1, box after box in index order:
  1. shared basis of box i from its low-rank block row: the interaction of
     i's active coordinates with every active coordinate outside N_l(i)
     (Sec. II-D: the concatenation of the low-rank blocks; dense blocks are
     not used).  Fill-ins created in those blocks by the eliminations of
     earlier boxes are part of that block row, so the basis absorbs them;
     this is what the recompression of eq. u2 / eq. v2 achieves, folding
     each fill-in into the row and column bases so that the skeleton matrix
     keeps its sparsity.  Column-pivoted Householder QR of the block row
     (eq. u), rank #{k : |R_kk| > tol |R_00|} capped at max_rank;
     Q_i = [U^R_i U^S_i];
  2. the block row and column of i are rotated into Q_i (eq. rs / eq. ss);
     the low-rank part, the redundant rows against the far coordinates, is
     dropped (it is below tol);
  3. the redundant block S^RR_ii is factored (LU, or Cholesky for SPD) and
     eliminated against every coordinate it still couples to (its own
     skeleton part and the near boxes' active coordinates): a Schur update
     of the trailing matrix, which is the dependency the paper's method
     removes, and which creates fill-in where two near boxes of i are far
     from each other;
  4. after the last box of the level, the children's skeleton coordinates
     form the parent boxes (Sec. II-C, the merge), and at l_top the rest is
     factored densely (eq. BLR2final).

Reading O-16 (the paper describes the method on one example): bases are
formed just before each box's elimination from the current trailing matrix,
which contains every fill-in created so far, instead of being formed first
and recompressed when a fill-in arrives; the two span the same far block row
up to tol.  The matrix is tracked densely (N x N), so this reference is for
small N only.  A box with an empty or zero far block row keeps all of its
coordinates as skeletons, as in the dependency-free oracle.

Parity status: pinned in tests/test_dep_oracle.py against the dense solve
and log-det (near-exact at tol 1e-14, within a tol-proportional bound at
tol 1e-6 and 1e-8) and against the paper's statement that the
dependency-free bases, which carry the pre-computed fill-ins, have larger
ranks.
"""
import numpy as np
import scipy.linalg as sla


class DependentULV:
    """H^2-ULV with trailing dependencies on ``pb`` (an ``h2ulv_oracle.Problem``).

    ``tol`` overrides the problem's rank tolerance.  Attributes after
    construction: ``rank_log`` = [(l, [r_i for the boxes of level l])],
    ``size_log`` = [(l, [n_i ...])] alike, ``dropped`` = the largest relative
    norm of a dropped low-rank part."""

    def __init__(self, pb, spd=False, tol=None):
        self.pb = pb
        self.spd = spd
        tol = pb.tol if tol is None else tol
        N, L = pb.N, pb.L
        M = pb.K(np.arange(N), np.arange(N))
        active = np.ones(N, dtype=bool)
        D = [np.arange(s, e) for (s, e) in pb.boxes[L]]     # active coordinates per box
        self.ops = []          # ("rot", idx, Q) and ("elim", R, C, factor, M_CR, M_RC) in order
        self.rank_log = []
        self.size_log = []
        self.dropped = 0.0
        self.logabsdet, self.sign = 0.0, 1.0
        for l in range(L, pb.ltop, -1):
            nb = len(pb.boxes[l])
            ranks = []
            S = [None] * nb
            for i in range(nb):
                Di = D[i]
                ni = len(Di)
                near = set(pb.near[l][i])
                in_near = np.zeros(N, dtype=bool)
                for j in near:
                    in_near[D[j]] = True
                far = np.flatnonzero(active & ~in_near)
                # --- 1. basis from the current low-rank block row (eq. u, u2)
                B = M[np.ix_(Di, far)]
                if B.shape[1] == 0 or not np.any(B):
                    r = ni
                    Q = np.eye(ni)
                else:
                    Qf, Rf, _ = sla.qr(B, pivoting=True)
                    d = np.abs(np.diag(Rf))
                    r = int(np.sum(d > tol * d[0])) if d[0] > 0 else 0
                    r = min(r, pb.max_rank, ni)
                    Q = np.hstack([Qf[:, r:], Qf[:, :r]])           # [U^R U^S] (Qf is ni x ni)
                ranks.append(r)
                m = ni - r
                # --- 2. rotate the block row and column of i into Q_i
                M[Di, :] = Q.T @ M[Di, :]
                M[:, Di] = M[:, Di] @ Q
                self.ops.append(("rot", Di.copy(), Q))
                R, Si = Di[:m], Di[m:]
                S[i] = Si
                if m == 0:
                    continue
                # drop the low-rank part of the redundant rows / columns
                if len(far):
                    bn = np.linalg.norm(B) if B.size else 0.0
                    if bn > 0:
                        self.dropped = max(self.dropped, np.linalg.norm(M[np.ix_(R, far)]) / bn)
                    M[np.ix_(R, far)] = 0.0
                    M[np.ix_(far, R)] = 0.0
                # --- 3. eliminate S^RR_ii against everything it couples to
                C = np.flatnonzero(active & in_near)
                C = C[~np.isin(C, R)]
                X = M[np.ix_(R, R)]
                MCR = M[np.ix_(C, R)].copy()
                MRC = M[np.ix_(R, C)].copy()
                if spd:
                    c = sla.cholesky(X, lower=True)
                    fac = ("chol", c)
                    Y = sla.cho_solve((c, True), MRC)
                    self.logabsdet += 2.0 * float(np.sum(np.log(np.diag(c))))
                else:
                    lu, pv = sla.lu_factor(X)
                    fac = ("lu", lu, pv)
                    Y = sla.lu_solve((lu, pv), MRC)
                    dg = np.diag(lu)
                    self.logabsdet += float(np.sum(np.log(np.abs(dg))))
                    self.sign *= float(np.prod(np.sign(dg))) * (-1.0) ** int(np.sum(pv != np.arange(len(pv))))
                M[np.ix_(C, C)] -= MCR @ Y
                M[R, :] = 0.0
                M[:, R] = 0.0
                active[R] = False
                self.ops.append(("elim", R, C, fac, MCR, MRC))
            self.rank_log.append((l, ranks))
            self.size_log.append((l, [len(d) for d in D]))
            # --- 4. merge: the children's skeletons form the parent boxes
            D = [np.concatenate([S[2 * p], S[2 * p + 1]]) for p in range(nb // 2)]
        # root (eq. BLR2final)
        self.root_idx = np.flatnonzero(active)
        Dm = M[np.ix_(self.root_idx, self.root_idx)]
        if spd:
            c = sla.cholesky(Dm, lower=True)
            self.root = ("chol", c)
            self.logabsdet += 2.0 * float(np.sum(np.log(np.diag(c))))
        else:
            lu, pv = sla.lu_factor(Dm)
            self.root = ("lu", lu, pv)
            dg = np.diag(lu)
            self.logabsdet += float(np.sum(np.log(np.abs(dg))))
            self.sign *= float(np.prod(np.sign(dg))) * (-1.0) ** int(np.sum(pv != np.arange(len(pv))))

    def _xsolve(self, fac, B):
        if fac[0] == "chol":
            return sla.cho_solve((fac[1], True), B)
        return sla.lu_solve((fac[1], fac[2]), B)

    def solve_tree(self, bt):
        """Forward: the rotations and eliminations in factorization order;
        the root solve; backward in reverse order (Sec. II-B)."""
        y = np.array(bt, dtype=np.float64, copy=True)
        stash = []
        for op in self.ops:
            if op[0] == "rot":
                _, idx, Q = op
                y[idx] = Q.T @ y[idx]
            else:
                _, R, C, fac, MCR, _ = op
                z = self._xsolve(fac, y[R])
                y[C] -= MCR @ z
                stash.append(y[R].copy())
        x = np.zeros_like(y)
        x[self.root_idx] = self._xsolve(self.root, y[self.root_idx])
        k = len(stash)
        for op in reversed(self.ops):
            if op[0] == "rot":
                _, idx, Q = op
                x[idx] = Q @ x[idx]
            else:
                k -= 1
                _, R, C, fac, _, MRC = op
                x[R] = self._xsolve(fac, stash[k] - MRC @ x[C])
        return x

    def solve(self, b):
        pb = self.pb
        xt = self.solve_tree(np.asarray(b, dtype=np.float64)[pb.perm])
        x = np.empty_like(xt)
        x[pb.perm] = xt
        return x

    def logdet(self):
        """log|det| and sign: the eliminated S^RR blocks and the root
        (the rotations are orthogonal and applied on both sides)."""
        return self.logabsdet, self.sign
