"""Seeded generators for the five synthetic workloads.

The paper evaluates on Slashdot, Flickr, Epinions and MovieLens25M (Section 4,
"Datasets").  None of them is available here, so every workload is a seeded
synthetic stand-in with the same structure: power-law graphs whose nodes arrive
in batches (link prediction, Section 4.1), a Zipf-popularity rating matrix whose
users arrive in batches (collaborative filtering), and Gaussian sparse matrices
with sparse low-rank weight updates (the third update kind of Section 2).

Conventions
-----------
A batch of ``s`` update vectors of length ``d`` is a CSR matrix with ``s`` rows
and ``d`` columns: row ``j`` of the CSR is update vector ``j``.  For new columns
``E_c`` (m x s) the CSR therefore holds ``E_c^T``; for new rows ``E_r`` (s x n)
it holds ``E_r`` itself; for a weight update ``D E_m^T`` it holds ``D^T`` and
``E_m^T``.  Indices are int32, values float64 (cast by the consumer).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class CSR:
    """A batch in CSR form: ``rows`` update vectors of length ``cols``."""
    indptr: np.ndarray   # int32, rows+1
    indices: np.ndarray  # int32, nnz
    values: np.ndarray   # float64, nnz
    rows: int
    cols: int

    @property
    def nnz(self) -> int:
        return int(self.indices.shape[0])

    def dense(self) -> np.ndarray:
        out = np.zeros((self.rows, self.cols))
        for j in range(self.rows):
            a, b = self.indptr[j], self.indptr[j + 1]
            out[j, self.indices[a:b]] = self.values[a:b]
        return out


def csr_from_coo(r: np.ndarray, c: np.ndarray, v: np.ndarray, rows: int, cols: int,
                 shuffle_within_rows: np.random.Generator | None = None) -> CSR:
    """Group COO triplets by row.  Within a row the column order is sorted, or a
    seeded shuffle of it when ``shuffle_within_rows`` is given (CSR batches need
    not have sorted column indices)."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], v[order]
    counts = np.bincount(r, minlength=rows)
    indptr = np.zeros(rows + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    if shuffle_within_rows is not None:
        for j in range(rows):
            a, b = indptr[j], indptr[j + 1]
            if b - a > 1:
                p = shuffle_within_rows.permutation(b - a) + a
                c[a:b] = c[p]
                v[a:b] = v[p]
    return CSR(indptr.astype(np.int32), c.astype(np.int32), v, rows, cols)


def csr_to_scipy(b: CSR) -> sp.csr_matrix:
    return sp.csr_matrix((b.values, b.indices, b.indptr), shape=(b.rows, b.cols))


def init_factors(A: sp.spmatrix | np.ndarray, k: int, seed: int, power_iters: int = 4,
                 oversample: int = 16) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Starting rank-k factors (U, sigma, V) of A, FP64, orthonormal U and V.

    Small dense inputs use a full SVD; large sparse ones a seeded randomized
    range finder with power iterations.  Any orthonormal start is a valid input
    of the update step (the maintained matrix is U diag(sigma) V^T by
    definition), so the start only needs to be a good rank-k approximation.
    """
    m, n = A.shape
    if not sp.issparse(A) or min(m, n) <= 2000:
        Ad = A.toarray() if sp.issparse(A) else np.asarray(A, dtype=np.float64)
        U, s, Vt = np.linalg.svd(Ad, full_matrices=False)
        return U[:, :k].copy(), s[:k].copy(), Vt[:k].T.copy()
    A = sp.csr_matrix(A, dtype=np.float64)
    At = A.T.tocsr()
    g = rng(seed)
    l = k + oversample
    Y = A @ g.standard_normal((n, l))
    Q, _ = np.linalg.qr(Y)
    for _ in range(power_iters):
        Z, _ = np.linalg.qr(At @ Q)
        Q, _ = np.linalg.qr(A @ Z)
    Bt = At @ Q                       # n x l  = (Q^T A)^T
    Vb, s, Uh_t = np.linalg.svd(Bt, full_matrices=False)   # Bt = Vb s Uh_t
    U = Q @ Uh_t.T
    return U[:, :k].copy(), s[:k].copy(), Vb[:, :k].copy()


# --------------------------------------------------------------------------
# C1: plain method, FP64
# --------------------------------------------------------------------------
def c1_problem(seed: int = 1001, m: int = 2000, n: int = 1000, nnz_a: int = 10000,
               k: int = 16, n_batches: int = 10, s: int = 10, lam: float = 5.0) -> dict:
    """Binary 2000x1000 matrix with 10,000 distinct uniform positions, rank-16
    start from the full SVD, then 10 batches of 10 new columns, each column
    with Poisson(5) ones at distinct uniform rows (empty columns allowed)."""
    g = rng(seed)
    flat = g.choice(m * n, size=nnz_a, replace=False)
    A = sp.csr_matrix((np.ones(nnz_a), (flat // n, flat % n)), shape=(m, n))
    U, sig, V = init_factors(A, k, seed)
    batches = []
    for _ in range(n_batches):
        r, c = [], []
        for j in range(s):
            cnt = min(int(g.poisson(lam)), m)
            rows = g.choice(m, size=cnt, replace=False)
            r.extend([j] * cnt)
            c.extend(rows.tolist())
        batches.append(("cols", csr_from_coo(np.array(r, dtype=np.int64), np.array(c, dtype=np.int64),
                                              np.ones(len(r)), s, m, shuffle_within_rows=g)))
    return dict(name="C1", A=A, U=U, sigma=sig, V=V, k=k, batches=batches)


# --------------------------------------------------------------------------
# C2: graph node insertion (Chung-Lu power-law graph)
# --------------------------------------------------------------------------
def chung_lu_edges(N: int, gamma: float, mean_deg: float, g: np.random.Generator) -> np.ndarray:
    """Undirected simple edge list (u < v) of an approximate Chung-Lu graph:
    weights w_i ~ (i+1)^(-1/(gamma-1)) scaled to mean ``mean_deg`` and capped at
    sqrt(sum w); Poisson(sum w / 2) endpoint pairs drawn i.i.d. proportional
    to w; self-loops dropped, duplicates merged."""
    w = (np.arange(N) + 1.0) ** (-1.0 / (gamma - 1.0))
    w *= mean_deg / w.mean()
    w = np.minimum(w, np.sqrt(w.sum()))
    p = w / w.sum()
    n_pairs = int(g.poisson(w.sum() / 2.0))
    a = g.choice(N, size=n_pairs, p=p)
    b = g.choice(N, size=n_pairs, p=p)
    keep = a != b
    u = np.minimum(a[keep], b[keep]).astype(np.int64)
    v = np.maximum(a[keep], b[keep]).astype(np.int64)
    key = np.unique(u * N + v)
    return np.stack([key // N, key % N], axis=1)


def c2_problem(seed: int = 1002, N: int = 100_000, gamma: float = 2.1, mean_deg: float = 10.0,
               k: int = 64, s: int = 256, init_frac: float = 0.5, n_batches: int | None = None,
               power_iters: int = 4) -> dict:
    """Node insertion on a symmetric binary Chung-Lu adjacency matrix.

    Nodes are put in a seeded random order; the start is a rank-k SVD of the
    adjacency among the first ``init_frac`` of them.  The rest arrive in
    batches of ``s``: first ``add_rows`` with their edges to existing nodes,
    then ``add_cols`` with their edges to existing and new nodes, so that every
    new-new edge enters exactly once (in the column step).
    """
    g = rng(seed)
    edges = chung_lu_edges(N, gamma, mean_deg, g)
    perm = g.permutation(N)               # perm[old id] = position
    u = perm[edges[:, 0]]
    v = perm[edges[:, 1]]
    rr = np.concatenate([u, v])
    cc = np.concatenate([v, u])
    n0 = int(round(N * init_frac))
    m0 = n0
    mask = (rr < n0) & (cc < n0)
    A0 = sp.csr_matrix((np.ones(int(mask.sum())), (rr[mask], cc[mask])), shape=(n0, n0))
    U, sig, V = init_factors(A0, k, seed, power_iters=power_iters)
    Afull = sp.csr_matrix((np.ones(rr.shape[0]), (rr, cc)), shape=(N, N))
    batches = []
    cur = n0
    bidx = 0
    while cur < N and (n_batches is None or bidx < n_batches):
        ss = min(s, N - cur)
        blk = Afull[cur:cur + ss]                           # new nodes' rows
        # add_rows: edges of the new nodes to existing nodes (columns < cur)
        er = blk[:, :cur].tocoo()
        Er = csr_from_coo(er.row, er.col, er.data, ss, cur, shuffle_within_rows=g)
        # add_cols: edges of the new nodes to existing and new nodes (rows < cur+ss)
        ec = blk[:, :cur + ss].tocoo()
        Ec = csr_from_coo(ec.row, ec.col, ec.data, ss, cur + ss, shuffle_within_rows=g)
        batches.append(("rows", Er))
        batches.append(("cols", Ec))
        cur += ss
        bidx += 1
    deg = np.asarray(Afull.sum(axis=1)).ravel()
    return dict(name="C2", A0=A0, U=U, sigma=sig, V=V, k=k, batches=batches,
                N=N, n0=n0, mean_degree=float(deg.mean()), max_degree=int(deg.max()))


# --------------------------------------------------------------------------
# C5: one differentiated column step of C2
# --------------------------------------------------------------------------
def distinct_nonempty_rows(b: CSR) -> CSR:
    """The batch without its empty update vectors and without repeats of an
    earlier vector (same indices and values).  Such vectors are dependent, and
    the differentiated step needs independent ones."""
    seen, keep = set(), []
    for j in range(b.rows):
        a, e = int(b.indptr[j]), int(b.indptr[j + 1])
        if e == a:
            continue
        key = tuple(sorted(zip(b.indices[a:e].tolist(), b.values[a:e].tolist())))
        if key in seen:
            continue
        seen.add(key)
        keep.append(j)
    r, c, v = [], [], []
    for jj, j in enumerate(keep):
        a, e = int(b.indptr[j]), int(b.indptr[j + 1])
        r.extend([jj] * (e - a))
        c.extend(b.indices[a:e].tolist())
        v.extend(b.values[a:e].tolist())
    return csr_from_coo(np.asarray(r, dtype=np.int64), np.asarray(c, dtype=np.int64), np.asarray(v, dtype=np.float64),
                        len(keep), b.cols)


def c5_problem(seed: int = 1002, N: int = 100_000, k: int = 64, s: int = 256, n_loss: int = 4096,
               loss_seed: int = 1005, power_iters: int = 4) -> dict:
    """C2's start, its first node batch, and the loss rows of the
    differentiation workload: the row step runs first (the caller applies
    it), then the column step ``cols`` (the first column batch, restricted to
    its distinct non-empty update vectors) is differentiated for the loss over
    ``n_loss`` seeded random existing rows ``S_rows`` (sorted)."""
    p = c2_problem(seed=seed, N=N, k=k, s=s, n_batches=1, power_iters=power_iters)
    (kr, rows), (kc, cols) = p["batches"][0], p["batches"][1]
    assert kr == "rows" and kc == "cols"
    g = rng(loss_seed)
    S_rows = np.sort(g.choice(p["n0"], size=min(n_loss, p["n0"]), replace=False)).astype(np.int64)
    return dict(name="C5", U=p["U"], sigma=p["sigma"], V=p["V"], k=k, rows=rows,
                cols=distinct_nonempty_rows(cols), cols_raw=cols, S_rows=S_rows, N=N)


# --------------------------------------------------------------------------
# C3: rating matrix, users appended as rows
# --------------------------------------------------------------------------
def zipf_ratings(n_users: int, n_items: int, mean_per_user: float, zipf_a: float,
                 g: np.random.Generator) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """COO (user, item, rating): item popularity ~ (j+1)^-zipf_a over a seeded
    item permutation, n_u = max(1, Poisson(mean)) distinct items per user
    (duplicates redrawn), ratings uniform integers 1..5."""
    p = (np.arange(n_items) + 1.0) ** (-zipf_a)
    p /= p.sum()
    item_perm = g.permutation(n_items)
    n_u = np.maximum(1, g.poisson(mean_per_user, size=n_users)).astype(np.int64)
    n_u = np.minimum(n_u, n_items)
    users = np.repeat(np.arange(n_users, dtype=np.int64), n_u)
    items = item_perm[g.choice(n_items, size=users.shape[0], p=p)]
    for _ in range(200):
        key = users * n_items + items
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup = np.zeros(ks.shape[0], dtype=bool)
        dup[1:] = ks[1:] == ks[:-1]
        if not dup.any():
            break
        redo = order[dup]
        items[redo] = item_perm[g.choice(n_items, size=redo.shape[0], p=p)]
    ratings = g.integers(1, 6, size=users.shape[0]).astype(np.float64)
    return users, items, ratings


def c3_problem(seed: int = 1003, n_users: int = 1_000_000, n_items: int = 50_000,
               mean_per_user: float = 20.0, zipf_a: float = 1.1, k: int = 128, s: int = 1024,
               init_frac: float = 0.5, n_batches: int | None = None, power_iters: int = 4) -> dict:
    """Users x items rating matrix; start on the first half of the users, then
    users are appended as row batches of ``s`` (``add_rows``)."""
    g = rng(seed)
    users, items, ratings = zipf_ratings(n_users, n_items, mean_per_user, zipf_a, g)
    m0 = int(round(n_users * init_frac))
    A = sp.csr_matrix((ratings, (users, items)), shape=(n_users, n_items))
    A0 = A[:m0]
    U, sig, V = init_factors(A0, k, seed, power_iters=power_iters)
    batches = []
    cur = m0
    while cur < n_users and (n_batches is None or len(batches) < n_batches):
        ss = min(s, n_users - cur)
        blk = A[cur:cur + ss].tocoo()
        batches.append(("rows", csr_from_coo(blk.row, blk.col, blk.data, ss, n_items,
                                             shuffle_within_rows=g)))
        cur += ss
    return dict(name="C3", A0=A0, U=U, sigma=sig, V=V, k=k, batches=batches)


# --------------------------------------------------------------------------
# C4: many independent matrices, sparse rank-s weight updates A + D E^T
# --------------------------------------------------------------------------
def random_csr_batch(s: int, d: int, per_vec: int, g: np.random.Generator) -> CSR:
    """``s`` update vectors of length ``d``, each with ``per_vec`` distinct
    uniform positions holding N(0,1) values (duplicates within a vector are
    redrawn)."""
    p = min(per_vec, d)
    pos = g.integers(0, d, size=(s, p))
    for _ in range(1000):
        srt = np.sort(pos, axis=1)
        dup = np.zeros_like(pos, dtype=bool)
        if p > 1:
            dup_rows = np.any(srt[:, 1:] == srt[:, :-1], axis=1)
        else:
            dup_rows = np.zeros(s, dtype=bool)
        if not dup_rows.any():
            break
        pos[dup_rows] = g.integers(0, d, size=(int(dup_rows.sum()), p))
    r = np.repeat(np.arange(s, dtype=np.int64), p)
    return csr_from_coo(r, pos.reshape(-1).astype(np.int64), g.standard_normal(s * p), s, d,
                        shuffle_within_rows=g)


def random_start(m: int, n: int, k: int, g: np.random.Generator, decay: float = 0.97):
    """A seeded orthonormal rank-k start (Gaussian QR) with geometrically
    decaying singular values: a valid start of the update step that does not
    need the matrix it came from."""
    U, _ = np.linalg.qr(g.standard_normal((m, k), dtype=np.float32).astype(np.float64))
    V, _ = np.linalg.qr(g.standard_normal((n, k), dtype=np.float32).astype(np.float64))
    sig = 10.0 * decay ** np.arange(k)
    return U, sig, V


def c4_problem(seed: int = 1004, n_mats: int = 64, m_lo: int = 5_000, m_hi: int = 200_000,
               density: float = 1e-4, ks=(16, 32, 64, 128), n_batches: int = 10,
               s_lo: int = 8, s_hi: int = 128, per_vec: int = 4, power_iters: int = 2,
               start: str = "rsvd") -> dict:
    """Independent Gaussian sparse matrices (m ~ U[m_lo, m_hi], n = m // 2,
    density 1e-4), each with ``n_batches`` weight updates D E^T of a random
    width s ~ U[s_lo, s_hi] and ``per_vec`` nonzeros per column of D and E.

    start="rsvd": the start is a randomized SVD of the drawn matrix A.
    start="random": A is not drawn; the start is ``random_start`` (the update
    step only ever sees the start factors and the batches, so its work is the
    same; used for benchmark-size runs where drawing A dominates).
    start="none": A and the start are left to the caller (U, sigma, V None)."""
    g = rng(seed)
    mats = []
    for _ in range(n_mats):
        m = int(g.integers(m_lo, m_hi + 1))
        n = m // 2
        k = int(g.choice(np.array(ks)))
        if start == "none":
            A, U, sig, V = None, None, None, None
        elif start == "random":
            A = None
            U, sig, V = random_start(m, n, k, g)
        else:
            nnz = max(1, int(round(density * m * n)))
            flat = np.unique(g.integers(0, m * n, size=nnz))
            A = sp.csr_matrix((g.standard_normal(flat.shape[0]), (flat // n, flat % n)), shape=(m, n))
            U, sig, V = init_factors(A, k, int(g.integers(1 << 30)), power_iters=power_iters)
        batches = []
        for _ in range(n_batches):
            s = int(g.integers(s_lo, s_hi + 1))
            D = random_csr_batch(s, m, per_vec, g)
            E = random_csr_batch(s, n, per_vec, g)
            batches.append(("weights", (D, E)))
        mats.append(dict(A=A, U=U, sigma=sig, V=V, k=k, m=m, n=n, batches=batches))
    return dict(name="C4", mats=mats)


# ---------------------------------------------------------------------------
def lookahead_batches(seed: int = 1006, n_users: int = 1_000_000, n_vectors: int = 65_536,
                      mean_nnz: float = 20.0) -> CSR:
    """Pending update vectors for the look-ahead projection: n_vectors new
    item columns over n_users rows (the rating matrix of the C3 shape), each
    with max(1, Poisson(mean_nnz)) distinct users drawn uniformly and
    ratings 1..5, as one CSR of n_vectors rows (64 pending batches of 1024)."""
    g = rng(seed)
    cnt = np.maximum(1, g.poisson(mean_nnz, size=n_vectors))
    r = np.repeat(np.arange(n_vectors, dtype=np.int64), cnt)
    c = g.integers(0, n_users, size=r.size)
    key = np.unique(r * n_users + c)                      # distinct users per vector
    r, c = key // n_users, key % n_users
    v = g.integers(1, 6, size=r.size).astype(np.float64)
    return csr_from_coo(r, c, v, n_vectors, n_users)
