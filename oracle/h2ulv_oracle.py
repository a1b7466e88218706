"""Plain FP64 CPU oracle of the dependency-free H^2-ULV solver.

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
it.  It shares no code with the CUDA library; the only module both sides
use is ``synth`` (seeded inputs, no solver arithmetic).

Every function follows a passage of the paper (Ma, Deshmukh, Yokota,
"Scalable Linear Time Dense Direct Solver for 3-D Problems Without Trailing
Sub-Matrix Dependencies", arXiv 2208.10907).  Where the paper is silent the
reading taken is named (O-1 ... O-15) at the code that applies it.

Notation (Sec. II-A, Fig. "notation"): a box I at level l owns n_I
"level coordinates"; Q_I = [U^R_I U^S_I] is its orthogonal basis, r_I its
rank (skeleton size) and m_I = n_I - r_I its redundant size.  N_l(I) and
F_l(I) are its near (dense) and far (low-rank) lists.

Parity status of each function is stated in its docstring; the pins that
check them live in tests/test_oracle_pins.py.
"""
import numpy as np
import scipy.linalg as sla

# ----------------------------------------------------------------------------
# Kernels (Sec. IV eq. for the Laplace Green's function; Sec. V for Yukawa).
# Reading O-11: the singular 1/(4 pi r) and exp(-r)/r are regularised as
# 1/(r + delta) and exp(-kappa r)/(r + delta); Matern-3/2 is
# (1 + sqrt3 r/ell) exp(-sqrt3 r/ell) plus nugget on the diagonal.
# ----------------------------------------------------------------------------
KERNELS = ("laplace", "yukawa", "matern32")


def kernel_matrix(kind, X, Y, delta=1e-3, kappa=1.0, ell=0.1, nugget=1e-4, same=False):
    """K(X_i, Y_j) in FP64.  ``same`` adds the nugget where X_i == Y_j for the
    Matern kernel (identical point, r == 0)."""
    d = np.sqrt(((X[:, None, :] - Y[None, :, :]) ** 2).sum(-1))
    if kind == "laplace":
        return 1.0 / (d + delta)
    if kind == "yukawa":
        return np.exp(-kappa * d) / (d + delta)
    if kind == "matern32":
        s = np.sqrt(3.0) * d / ell
        K = (1.0 + s) * np.exp(-s)
        return K + nugget * (d == 0.0)
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# O-1  Cluster tree: full binary tree of 2^L leaves (Sec. III-E: the row /
# column tree is a full binary tree), built by coordinate bisection.
# ----------------------------------------------------------------------------
def cluster_tree(X, leaf):
    """Return (L, perm, boxes).  ``perm`` maps tree order to user order;
    ``boxes[l]`` lists the (start, end) tree-order ranges of the 2^l boxes of
    level l.  L = ceil(log2(N / leaf)) (0 when N <= leaf).  Each box is split
    along the longest side of its points' bounding box (ties -> lowest axis);
    points are ordered by (coordinate, original index) and the left child
    takes floor(n/2) of them."""
    N = len(X)
    L = int(np.ceil(np.log2(N / leaf))) if N > leaf else 0
    perm = np.arange(N)
    boxes = [[(0, N)]]
    for _ in range(L):
        nxt = []
        for (s, e) in boxes[-1]:
            idx = perm[s:e]
            P = X[idx]
            ext = P.max(0) - P.min(0)
            ax = int(np.argmax(ext))
            order = np.lexsort((idx, P[:, ax]))
            perm[s:e] = idx[order]
            mid = s + (e - s) // 2
            nxt += [(s, mid), (mid, e)]
        boxes.append(nxt)
    return L, perm, boxes


# ----------------------------------------------------------------------------
# O-15  k-means partition (Sec. V: a 3-D k-means clustering forms the leaf
# boxes, with the number of clusters a power of two).  Reading: every box is
# split by a balanced 2-means (Lloyd iterations whose assignment step gives
# the floor(n/2) points closest to centroid 0 relative to centroid 1 to the
# left child), which keeps the full binary tree of 2^L leaves.  Seeds: the
# point farthest from the box's mean, then the point farthest from that one.
# Sums run over the box's points in increasing caller index, distances are
# ((dx^2 + dy^2) + dz^2), ties go to the lowest caller index, at most 20
# Lloyd steps.
# ----------------------------------------------------------------------------
def _seq_mean(P):
    return np.array([np.cumsum(P[:, a])[-1] for a in range(3)]) / len(P)


def _sqdist(P, c):
    return ((P[:, 0] - c[0]) ** 2 + (P[:, 1] - c[1]) ** 2) + (P[:, 2] - c[2]) ** 2


def balanced_two_means(X, idx, iters=20):
    """Order the caller indices idx of one box as [left child, right child]
    (left = the first floor(n/2)); returns (order, Lloyd steps taken)."""
    idx = np.sort(np.asarray(idx))
    n = len(idx)
    P = X[idx]
    if n < 2:
        return idx, 0
    a = int(np.argmax(_sqdist(P, _seq_mean(P))))
    c0 = P[a].copy()
    b = int(np.argmax(_sqdist(P, c0)))
    c1 = P[b].copy()
    left = None
    h = n // 2
    for it in range(iters):
        key = _sqdist(P, c0) - _sqdist(P, c1)
        order = np.lexsort((idx, key))
        new_left = np.sort(order[:h])
        if left is not None and np.array_equal(new_left, left):
            return idx[order], it
        left = new_left
        right = np.sort(order[h:])
        c0 = _seq_mean(P[left])
        c1 = _seq_mean(P[right])
    key = _sqdist(P, c0) - _sqdist(P, c1)
    return idx[np.lexsort((idx, key))], iters


def cluster_tree_kmeans(X, leaf):
    """Same outputs as cluster_tree, with every split a balanced 2-means."""
    N = len(X)
    L = int(np.ceil(np.log2(N / leaf))) if N > leaf else 0
    perm = np.arange(N)
    boxes = [[(0, N)]]
    for _ in range(L):
        nxt = []
        for (s, e) in boxes[-1]:
            perm[s:e] = balanced_two_means(X, perm[s:e])[0]
            mid = s + (e - s) // 2
            nxt += [(s, mid), (mid, e)]
        boxes.append(nxt)
    return L, perm, boxes


# ----------------------------------------------------------------------------
# O-2  Strong admissibility (Sec. I: blocks in close proximity are subdivided
# down to the leaf, where they stay dense).  (I, J) at level l is far when
# its parent pair is near and max(diam I, diam J) <= eta * dist(I, J), with
# diam the bounding-box diagonal and dist the gap between bounding boxes.
# ----------------------------------------------------------------------------
def box_bounds(Xt, boxes):
    return [[(Xt[s:e].min(0), Xt[s:e].max(0)) for (s, e) in lev] for lev in boxes]


def admissible(b1, b2, eta):
    lo1, hi1 = b1
    lo2, hi2 = b2
    d1 = np.sqrt(((hi1 - lo1) ** 2).sum())
    d2 = np.sqrt(((hi2 - lo2) ** 2).sum())
    gap = np.maximum(0.0, np.maximum(lo1 - hi2, lo2 - hi1))
    dist = np.sqrt((gap ** 2).sum())
    return max(d1, d2) <= eta * dist


def interaction_lists(Xt, boxes, L, eta):
    """near[l][i], far[l][i]: sorted box indices at level l."""
    bb = box_bounds(Xt, boxes)
    near = [[[] for _ in lev] for lev in boxes]
    far = [[[] for _ in lev] for lev in boxes]
    near[0][0] = [0]
    for l in range(1, L + 1):
        for P in range(len(boxes[l - 1])):
            for Qb in near[l - 1][P]:
                for a in (2 * P, 2 * P + 1):
                    for c in (2 * Qb, 2 * Qb + 1):
                        if admissible(bb[l][a], bb[l][c], eta):
                            far[l][a].append(c)
                        else:
                            near[l][a].append(c)
    for l in range(L + 1):
        for i in range(len(boxes[l])):
            near[l][i].sort()
            far[l][i].sort()
    return near, far


def top_level(far, L):
    """O-8: l_top = the largest l such that no level <= l has a far pair.
    The ULV runs on levels L .. l_top+1; the level-l_top matrix is dense."""
    lt = 0
    for l in range(L + 1):
        if any(len(f) for f in far[l]):
            break
        lt = l
    return lt


# ----------------------------------------------------------------------------
# O-4  Far-field block row.  The shared basis is built from the concatenation
# of the low-rank blocks of the block row (eq. u, Sec. II-D: "the
# concatenation of all low-rank blocks").  Its columns are the points of the
# far boxes of I and of I's ancestors.  Deterministic sample: the far boxes
# of level l' contribute s(l') = max(s_min, s0 >> (l - l')) points each, at
# tree-order positions start + floor((2k+1) |J| / (2 s)); a box with at most
# s points is taken whole.  s0 = 0 takes every far point (exact variant).
# ----------------------------------------------------------------------------
def far_samples(boxes, far, l, i, s0=32, s_min=4):
    out = []
    a = i
    for ll in range(l, 0, -1):
        s = max(s_min, s0 >> (l - ll)) if s0 > 0 else 0
        for J in far[ll][a]:
            st, e = boxes[ll][J]
            nJ = e - st
            if s0 == 0 or nJ <= s:
                out.append(np.arange(st, e))
            else:
                k = np.arange(s)
                out.append(st + ((2 * k + 1) * nJ) // (2 * s))
        a //= 2
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


# ----------------------------------------------------------------------------
# O-3  Rank-revealing column-pivoted QR (eq. u: "[U^S U^R], R = QR(A_{i,+})",
# Sec. II-A: column pivoted or rank revealing QR).  Pivot = the remaining
# column of largest 2-norm (recomputed, ties -> lowest index); the rank is
# #{k : |R_kk| > tol |R_11|}, capped at max_rank.
# ----------------------------------------------------------------------------
def pivoted_qr(Bt, tol, max_rank):
    """Householder QR with column pivoting of Bt (m x n), the transpose of the
    block row, so the pivots select rows of the block row (skeleton rows).
    Returns (piv, R[:rank], rank)."""
    A = np.array(Bt, dtype=np.float64, copy=True)
    m, n = A.shape
    piv = np.arange(n)
    R = np.zeros((n, n))
    r11 = None
    rank = min(m, n, max_rank)
    for k in range(min(m, n)):
        norms = np.sqrt((A[k:, k:] ** 2).sum(0))
        j = k + int(np.argmax(norms))
        A[:, [k, j]] = A[:, [j, k]]
        R[:, [k, j]] = R[:, [j, k]]
        piv[[k, j]] = piv[[j, k]]
        x = A[k:, k].copy()
        alpha = np.sqrt((x ** 2).sum())
        if r11 is None:
            r11 = alpha
        if k >= max_rank or alpha <= tol * r11 or alpha == 0.0:
            rank = k
            break
        beta = -alpha if x[0] >= 0 else alpha
        v = x
        v[0] -= beta
        vn = np.sqrt((v ** 2).sum())
        v /= vn
        A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        R[k, k:] = A[k, k:]
    else:
        rank = min(m, n, max_rank)
    return piv, R[:rank], rank


def fold_rows(Bt):
    """Replace a tall Bt (m x n, m > n) by the R factor of its unpivoted
    Householder QR (LAPACK geqrf through numpy).  Bt = Q0 R0 with Q0
    orthonormal, so pivoted QR of R0 has the same pivots and R as pivoted QR
    of Bt (up to row signs)."""
    Bt = np.asarray(Bt, dtype=np.float64)
    if Bt.shape[0] <= Bt.shape[1]:
        return Bt
    return np.linalg.qr(Bt, mode="r")


def pivoted_cholesky(G, tol, max_rank):
    """The same pivoted QR computed from the Gram matrix G = B B^T.

    Householder QR of B^T with column pivoting has R^T R = P^T (B B^T) P and
    pivots on the largest remaining column norm, i.e. on the largest diagonal
    entry of the Schur complement of the Gram matrix.  So diagonal-pivoted
    Cholesky of B B^T reproduces the pivots and R of eq. (u) without forming
    the (very wide) block row.  Rank rule: R_kk^2 > tol^2 R_11^2."""
    G = np.array(G, dtype=np.float64, copy=True)
    n = len(G)
    piv = np.arange(n)
    R = np.zeros((n, n))
    d1 = None
    rank = min(n, max_rank)
    for k in range(n):
        j = k + int(np.argmax(np.diag(G)[k:]))
        G[[k, j]] = G[[j, k]]
        G[:, [k, j]] = G[:, [j, k]]
        R[:, [k, j]] = R[:, [j, k]]
        piv[[k, j]] = piv[[j, k]]
        if d1 is None:
            d1 = G[k, k]
        if k >= max_rank or G[k, k] <= tol * tol * d1 or G[k, k] <= 0.0:
            rank = k
            break
        R[k, k] = np.sqrt(G[k, k])
        R[k, k + 1:] = G[k, k + 1:] / R[k, k]
        G[k + 1:, k + 1:] -= np.outer(R[k, k + 1:], R[k, k + 1:])
    else:
        rank = min(n, max_rank)
    return piv, R[:rank], rank


def interpolation_matrix(piv, R, rank, n):
    """Interpolative decomposition from the pivoted QR of B^T (Sec. II-A: the
    QR may be replaced by an ID).  B ~= P B[piv[:rank]] with
    P[piv[:rank]] = I and P[piv[rank:]] = (R11^-1 R12)^T."""
    P = np.zeros((n, rank))
    P[piv[:rank], np.arange(rank)] = 1.0
    if rank < n:
        T = sla.solve_triangular(R[:rank, :rank], R[:rank, rank:])
        P[piv[rank:], :] = T.T
    return P


# ----------------------------------------------------------------------------
# The H^2 matrix used as the refinement residual (reading O-12): shared,
# nested interpolative bases built from the far-field (low-rank) blocks only
# (eq. u; Sec. II-D "Dense blocks are never used for the construction of the
# shared basis"), nested through transfer matrices (eq. transfer).
# ----------------------------------------------------------------------------
class Problem:
    def __init__(self, X, kernel, leaf, eta, tol, max_rank, s0=32, s_min=4, kparams=None, partition="bisection"):
        self.X = np.asarray(X, dtype=np.float64)
        self.N = len(self.X)
        self.kernel = kernel
        self.kp = dict(kparams or {})
        self.leaf, self.eta, self.tol, self.max_rank = leaf, eta, tol, max_rank
        self.s0, self.s_min = s0, s_min
        if partition == "kmeans":
            self.L, self.perm, self.boxes = cluster_tree_kmeans(self.X, leaf)
        else:
            self.L, self.perm, self.boxes = cluster_tree(self.X, leaf)
        self.Xt = self.X[self.perm]
        self.near, self.far = interaction_lists(self.Xt, self.boxes, self.L, eta)
        self.ltop = top_level(self.far, self.L)

    def K(self, I, J):
        """Kernel block between tree-order index sets I and J."""
        same = True
        return kernel_matrix(self.kernel, self.Xt[I], self.Xt[J], same=same, **self.kp)

    def samples(self, l, i):
        return far_samples(self.boxes, self.far, l, i, self.s0, self.s_min)


class H2Operator:
    """A_H2 with near blocks exact and far blocks K(sk_I, sk_J) through nested
    interpolation matrices.  Parity: pinned against the dense matrix
    (tests check ||A_H2 - A|| / ||A|| against tol)."""

    def __init__(self, pb):
        self.pb = pb
        L, boxes = pb.L, pb.boxes
        self.P = {}
        self.sk = {}
        cand = [np.arange(s, e) for (s, e) in boxes[L]]
        for l in range(L, pb.ltop, -1):
            sk_l = []
            for i, c in enumerate(cand):
                fs = pb.samples(l, i)
                n = len(c)
                if len(fs) == 0:
                    rank, Pm, sk = n, np.eye(n), c
                else:
                    B = pb.K(c, fs)
                    piv, R, rank = pivoted_qr(fold_rows(B.T), pb.tol, pb.max_rank)
                    if rank == 0:
                        rank, Pm, sk = n, np.eye(n), c
                    else:
                        Pm = interpolation_matrix(piv, R, rank, n)
                        sk = c[piv[:rank]]
                self.P[(l, i)] = Pm
                self.sk[(l, i)] = sk
                sk_l.append(sk)
            cand = [np.concatenate([sk_l[2 * p], sk_l[2 * p + 1]]) for p in range(len(sk_l) // 2)]

    def ranks(self, l):
        return [self.sk[(l, i)].size for i in range(len(self.pb.boxes[l]))]

    def matvec_tree(self, xt):
        """y = A_H2 x for x in tree order (N x k)."""
        pb = self.pb
        L, boxes = pb.L, pb.boxes
        xt = np.asarray(xt, dtype=np.float64)
        squeeze = xt.ndim == 1
        if squeeze:
            xt = xt[:, None]
        y = np.zeros_like(xt)
        for i, (s, e) in enumerate(boxes[L]):
            for j in pb.near[L][i]:
                s2, e2 = boxes[L][j]
                y[s:e] += pb.K(np.arange(s, e), np.arange(s2, e2)) @ xt[s2:e2]
        if L > pb.ltop:
            xh = {}
            for i, (s, e) in enumerate(boxes[L]):
                xh[(L, i)] = self.P[(L, i)].T @ xt[s:e]
            for l in range(L - 1, pb.ltop, -1):
                for i in range(len(boxes[l])):
                    xh[(l, i)] = self.P[(l, i)].T @ np.vstack([xh[(l + 1, 2 * i)], xh[(l + 1, 2 * i + 1)]])
            yh = {}
            for l in range(pb.ltop + 1, L + 1):
                for i in range(len(boxes[l])):
                    acc = np.zeros_like(xh[(l, i)])
                    for j in pb.far[l][i]:
                        acc += pb.K(self.sk[(l, i)], self.sk[(l, j)]) @ xh[(l, j)]
                    if l > pb.ltop + 1:
                        par = self.P[(l - 1, i // 2)] @ yh[(l - 1, i // 2)]
                        ra = self.sk[(l, i - (i % 2))].size
                        acc += par[:ra] if i % 2 == 0 else par[ra:]
                    yh[(l, i)] = acc
            for i, (s, e) in enumerate(boxes[L]):
                y[s:e] += self.P[(L, i)] @ yh[(L, i)]
        return y[:, 0] if squeeze else y

    def matvec(self, x):
        """y = A_H2 x in user order."""
        pb = self.pb
        x = np.asarray(x, dtype=np.float64)
        yt = self.matvec_tree(x[pb.perm])
        y = np.empty_like(yt)
        y[pb.perm] = yt
        return y

    def dense(self):
        """A_H2 as a dense matrix in tree order (small N only)."""
        return self.matvec_tree(np.eye(self.pb.N))


# ----------------------------------------------------------------------------
# Dependency-free H^2-ULV factorization (Sec. III-B .. III-D, with the
# per-level elimination of Sec. II-B/C applied to every box at once).
# ----------------------------------------------------------------------------
def lu_nopiv_parts(A):
    """LU with partial pivoting (reading O-9): returns (lu, piv) as LAPACK
    getrf does (scipy.linalg.lu_factor)."""
    return sla.lu_factor(A, check_finite=True)


def lu_apply_Linv(lu, piv, B):
    """L^-1 P^T B for the getrf factors."""
    Y = np.array(B, dtype=np.float64, copy=True)
    for t, p in enumerate(piv):
        if p != t:
            Y[[t, p]] = Y[[p, t]]
    return sla.solve_triangular(lu, Y, lower=True, unit_diagonal=True)


def lu_logdet(lu, piv):
    d = np.diag(lu)
    sign = np.prod(np.sign(d)) * (-1.0) ** int(np.sum(piv != np.arange(len(piv))))
    return float(np.sum(np.log(np.abs(d)))), float(sign)


def fill_in_terms(near_l, i):
    """Sec. III-B (Fig. fill-in): the fill-ins of block row i are
    A_{i,K} A_{K,K}^-1 A_{K,J} for every box K != i with a dense block to i
    and every J != K with a dense block to K (reading O-5 A: J = i included).
    Returns the (K, J) pairs, K in the order of i's near list, J in K's."""
    return [(K, J) for K in near_l[i] if K != i for J in near_l[K] if J != K]


def fill_in_blocks(near_l, i):
    """Block positions that fill in in block row i and block column i: (i, J)
    from the row terms and, by the symmetry of the near relation, (J, i) from
    the column terms A_{J,K} A_{K,K}^-1 A_{K,i}."""
    pos = set()
    for K, J in fill_in_terms(near_l, i):
        pos.add((i, J))
        pos.add((J, i))
    return sorted(pos)


class ULVFactor:
    """The dependency-free H^2-ULV factorization.

    Per level l = L .. l_top+1 and for every box independently:
      1. fill-in pre-computation (Sec. III-B, Fig. fill-in): for each box K,
         LU of the dense diagonal block A_KK and the fill-ins
         T_{I,K,J} = A_IK A_KK^-1 A_KJ for I, J in N_l(K) \\ {K}
         (reading O-5 A: every near J, the diagonal J = I included), kept
         separate (never accumulated);
      2. shared basis with fill-ins (eq. fillu): column-pivoted QR of the
         concatenation [F_{I,+}  A_{I,+}], taken as an interpolative
         decomposition in point form and orthogonalised, Q_I = [U^R U^S];
      3. projection (eq. rs for dense blocks, eq. ss for low-rank blocks);
      4. partial LU of S^RR_II (eq. lu), the eliminations of S^RS and S^SR
         and the Schur update of S^SS_II (reading O-7 lit: only the box's own
         diagonal block is eliminated);
      5. merge of the children's S^SS blocks into the parent level
         (Sec. II-C, the merge equation), then the dense LU of the level
         l_top matrix (eq. BLR2final).

    ``route`` selects how step 2 forms the block row (all three give the
    same pivoted QR in exact arithmetic; pinned against each other):
      "literal": every T_{I,K,J} is formed and the pivoted QR runs on the
                 explicit block row (the paper's statement; small cases),
                 after the row fold that keeps its pivots and R (fold_rows);
      "qr"     : (default) the fill-ins that share K share the row factor
                 A_KK^-1 [A_KJ]_J, whose QR R-factor R_K is taken once, so
                 row I holds the n x n blocks A_IK A_KK^-1 R_K^T instead of
                 one block per J (same column space: [A_KJ]_J = R_K^T Q^T
                 with Q orthonormal); the block row is folded by Householder
                 QR and pivoted QR decides, all in FP64 without squaring;
      "gram"   : the Gram matrix sum_K A_IK M_K A_IK^T + G G^T, M_K =
                 A_KK^-1 (sum_J A_KJ A_KJ^T) A_KK^-T, and pivoted Cholesky
                 (the mixed-precision GPU route; it resolves the block row
                 only to about sqrt(eps) of its norm).
    ``tol_basis`` overrides the rank tolerance of step 2 (the problem's tol
    by default).
    """

    def __init__(self, pb, route="qr", spd=False, tol_basis=None):
        if route not in ("qr", "literal", "gram"):
            raise ValueError(route)
        self.pb = pb
        self.spd = spd
        self.route = route
        L, boxes, near, far = pb.L, pb.boxes, pb.near, pb.far
        tol = pb.tol if tol_basis is None else tol_basis
        max_rank = pb.max_rank
        cand = [np.arange(s, e) for (s, e) in boxes[L]]
        T = [None] * len(cand)           # level coords = T @ point form (None = identity)
        A = {}
        for i in range(len(boxes[L])):
            for j in near[L][i]:
                A[(i, j)] = pb.K(cand[i], cand[j])
        self.levels = []
        self.rank_log = []
        for l in range(L, pb.ltop, -1):
            nb = len(boxes[l])
            n = [len(c) for c in cand]
            # --- 1. fill-ins (Sec. III-B) --------------------------------
            lus = {}
            Z = {}       # "qr": A_KK^-1 R_K^T
            Minv = {}    # "gram": A_KK^-1 (sum_J A_KJ A_KJ^T) A_KK^-T
            Wlit = {}    # "literal": A_KK^-1 A_KJ
            for K in range(nb):
                others = [J for J in near[l][K] if J != K]
                if not others:
                    continue
                lus[K] = sla.lu_factor(A[(K, K)])
                if route == "literal":
                    # the triangular solves are shared by every row I (Sec. III-B)
                    for J in others:
                        Wlit[(K, J)] = sla.lu_solve(lus[K], A[(K, J)])
                elif route == "qr":
                    RK = fold_rows(np.hstack([A[(K, J)] for J in others]).T)
                    Z[K] = sla.lu_solve(lus[K], RK.T)
                elif route == "gram":
                    NG = np.zeros((n[K], n[K]))
                    for J in others:
                        NG += A[(K, J)] @ A[(K, J)].T
                    Zg = sla.lu_solve(lus[K], NG)
                    Minv[K] = sla.lu_solve(lus[K], Zg.T).T
            # --- 2. bases (eq. fillu) -------------------------------------
            Q, W, sk, r = [], [], [], []
            for I in range(nb):
                fs = pb.samples(l, I)
                G = kernel_matrix(pb.kernel, pb.Xt[cand[I]], pb.Xt[fs], same=True, **pb.kp) \
                    if len(fs) else np.zeros((n[I], 0))
                Kn = [K for K in near[l][I] if K != I and K in lus]
                if route in ("literal", "qr"):
                    if route == "literal":
                        Fblocks = [A[(I, K)] @ Wlit[(K, J)]
                                   for K, J in fill_in_terms(near[l], I) if K in lus]
                    else:
                        Fblocks = [A[(I, K)] @ Z[K] for K in Kn]
                    F = np.hstack(Fblocks) if Fblocks else np.zeros((n[I], 0))
                    if T[I] is not None:
                        F = sla.solve(T[I], F)
                    B = np.hstack([F, G])
                    if B.shape[1] == 0 or not np.any(B):
                        piv, R, rk = np.arange(n[I]), None, 0
                    else:
                        piv, R, rk = pivoted_qr(fold_rows(B.T), tol, max_rank)
                else:
                    Gr = G @ G.T
                    if Kn:
                        GF = np.zeros((n[I], n[I]))
                        for K in Kn:
                            GF += A[(I, K)] @ Minv[K] @ A[(I, K)].T
                        if T[I] is not None:
                            GF = sla.solve(T[I], sla.solve(T[I], GF).T).T
                        Gr = Gr + GF
                    if not np.any(Gr):
                        piv, R, rk = np.arange(n[I]), None, 0
                    else:
                        piv, R, rk = pivoted_cholesky(Gr, tol, max_rank)
                if rk == 0:
                    rk, Pm = n[I], np.eye(n[I])
                    piv = np.arange(n[I])
                else:
                    Pm = interpolation_matrix(piv, R, rk, n[I])
                Mb = Pm if T[I] is None else T[I] @ Pm
                Qf, Rf = np.linalg.qr(Mb, mode="complete")
                Q.append(np.hstack([Qf[:, rk:], Qf[:, :rk]]))   # [U^R U^S]
                W.append(Rf[:rk, :rk])
                sk.append(cand[I][piv[:rk]])
                r.append(rk)
            m = [n[i] - r[i] for i in range(nb)]
            self.rank_log.append((l, r))
            # --- 3. projection (eq. rs, eq. ss) ---------------------------
            SS = {}
            diagS = {}
            for (i, j), a in A.items():
                if i == j:
                    diagS[i] = Q[i].T @ a @ Q[i]
                else:
                    SS[(i, j)] = Q[i][:, m[i]:].T @ a @ Q[j][:, m[j]:]
            for i in range(nb):
                for j in far[l][i]:
                    SS[(i, j)] = W[i] @ pb.K(sk[i], sk[j]) @ W[j].T
            # --- 4. partial factorization (eq. lu and the two TRSMs) ------
            fac = []
            for i in range(nb):
                S = diagS[i]
                mi = m[i]
                if mi == 0:
                    fac.append(None)
                    SS[(i, i)] = S.copy()
                    continue
                if spd:
                    c = sla.cholesky(S[:mi, :mi], lower=True)
                    Urs = sla.solve_triangular(c, S[:mi, mi:], lower=True)
                    Lsr = Urs.T
                    fac.append(("chol", c, Urs, Lsr))
                else:
                    lu, pv = sla.lu_factor(S[:mi, :mi])
                    Urs = lu_apply_Linv(lu, pv, S[:mi, mi:])
                    Lsr = sla.solve_triangular(lu, S[mi:, :mi].T, trans="T", lower=False).T
                    fac.append(("lu", lu, pv, Urs, Lsr))
                SS[(i, i)] = S[mi:, mi:] - Lsr @ Urs
            self.levels.append(dict(l=l, Q=Q, m=m, r=r, fac=fac))
            # --- 5. merge into level l-1 ----------------------------------
            nbp = nb // 2
            A = {}
            for P in range(nbp):
                for Qb in near[l - 1][P]:
                    A[(P, Qb)] = np.block([[SS[(a, c)] for c in (2 * Qb, 2 * Qb + 1)]
                                           for a in (2 * P, 2 * P + 1)])
            cand = [np.concatenate([sk[2 * p], sk[2 * p + 1]]) for p in range(nbp)]
            T = [sla.block_diag(W[2 * p], W[2 * p + 1]) for p in range(nbp)]
        # --- root (eq. BLR2final) -----------------------------------------
        nb = len(boxes[pb.ltop])
        sizes = [A[(i, i)].shape[0] for i in range(nb)]
        self.root_off = np.concatenate([[0], np.cumsum(sizes)]).astype(int)
        D = np.zeros((self.root_off[-1], self.root_off[-1]))
        for (i, j), a in A.items():
            D[self.root_off[i]:self.root_off[i + 1], self.root_off[j]:self.root_off[j + 1]] = a
        self.root_dense = D
        if spd:
            self.root = ("chol", sla.cholesky(D, lower=True))
        else:
            self.root = ("lu",) + tuple(sla.lu_factor(D))

    # ---- solve (Sec. II-B: L z = U^T b, U y = z, x = V^T y) ----------------
    def solve_tree(self, bt):
        pb = self.pb
        bt = np.asarray(bt, dtype=np.float64)
        squeeze = bt.ndim == 1
        if squeeze:
            bt = bt[:, None]
        cur = [bt[s:e] for (s, e) in pb.boxes[pb.L]]
        stash = []
        for lev in self.levels:
            Q, m, fac = lev["Q"], lev["m"], lev["fac"]
            yR, nxt = [], []
            cS = []
            for i, b in enumerate(cur):
                c = Q[i].T @ b
                mi = m[i]
                if mi == 0:
                    yR.append(np.zeros((0, b.shape[1])))
                    cS.append(c)
                    continue
                f = fac[i]
                if f[0] == "chol":
                    y = sla.solve_triangular(f[1], c[:mi], lower=True)
                    cS.append(c[mi:] - f[3] @ y)
                else:
                    y = lu_apply_Linv(f[1], f[2], c[:mi])
                    cS.append(c[mi:] - f[4] @ y)
                yR.append(y)
            stash.append(yR)
            cur = [np.vstack([cS[2 * p], cS[2 * p + 1]]) for p in range(len(cS) // 2)]
        rb = np.vstack(cur)
        if self.root[0] == "chol":
            z = sla.cho_solve((self.root[1], True), rb)
        else:
            z = sla.lu_solve((self.root[1], self.root[2]), rb)
        xs = [z[self.root_off[i]:self.root_off[i + 1]] for i in range(len(cur))]
        for lev, yR in zip(reversed(self.levels), reversed(stash)):
            Q, m, r, fac = lev["Q"], lev["m"], lev["r"], lev["fac"]
            xS = []
            for p, xp in enumerate(xs):
                ra = r[2 * p]
                xS += [xp[:ra], xp[ra:]]
            xn = []
            for i in range(len(Q)):
                mi = m[i]
                if mi == 0:
                    xn.append(Q[i] @ xS[i])
                    continue
                f = fac[i]
                if f[0] == "chol":
                    xR = sla.solve_triangular(f[1], yR[i] - f[2] @ xS[i], lower=True, trans="T")
                else:
                    xR = sla.solve_triangular(f[1], yR[i] - f[3] @ xS[i], lower=False)
                xn.append(Q[i] @ np.vstack([xR, xS[i]]))
            xs = xn
        x = np.vstack(xs)
        return x[:, 0] if squeeze else x

    def solve(self, b):
        pb = self.pb
        b = np.asarray(b, dtype=np.float64)
        xt = self.solve_tree(b[pb.perm])
        x = np.empty_like(xt)
        x[pb.perm] = xt
        return x

    # ---- log-determinant (reading O-10) ------------------------------------
    def logdet(self):
        """log|det| and sign of the factored matrix: the product of the
        eliminated S^RR_II determinants and the root's (|det Q_I| = 1, and
        det(Q_I)^2 = 1 because the row and column bases coincide)."""
        tot, sign = 0.0, 1.0
        for lev in self.levels:
            for f in lev["fac"]:
                if f is None:
                    continue
                if f[0] == "chol":
                    tot += 2.0 * float(np.sum(np.log(np.diag(f[1]))))
                else:
                    ld, sg = lu_logdet(f[1], f[2])
                    tot += ld
                    sign *= sg
        if self.root[0] == "chol":
            tot += 2.0 * float(np.sum(np.log(np.diag(self.root[1]))))
        else:
            ld, sg = lu_logdet(self.root[1], self.root[2])
            tot += ld
            sign *= sg
        return tot, sign


def refine(op, fac, b, target=1e-10, max_iter=50):
    """FP64 iterative refinement with the H^2 matvec as residual (reading
    O-12): x <- x + ULV^-1 (b - A_H2 x) until ||r|| / ||b|| <= target per
    right-hand side.  Returns (x, achieved relative residual, iterations)."""
    b = np.asarray(b, dtype=np.float64)
    squeeze = b.ndim == 1
    if squeeze:
        b = b[:, None]
    bn = np.linalg.norm(b, axis=0)
    bn[bn == 0] = 1.0
    x = fac.solve(b)
    it = 0
    while True:
        res = b - op.matvec(x)
        rel = np.linalg.norm(res, axis=0) / bn
        if np.all(rel <= target) or it >= max_iter:
            break
        x = x + fac.solve(res)
        it += 1
    if squeeze:
        return x[:, 0], rel, it
    return x, rel, it
