"""Oracle: the sparse sign embedding of Sec. 2 as the sketch of Algorithm 1.

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 2 describes Omega = c (omega_1 ... omega_m): column omega_j has zeta entries in
rows chosen at random and uniformly, each +1 or -1 with probability 1/2, the rest
zero; Omega A then samples and adds or subtracts rows of A.

Readings where the paper is silent or garbled:
* Scale: the printed factor sqrt(m / zeta) does not make Omega an embedding
  (||Omega e_j||^2 = m); the isometry in expectation, E ||Omega x||^2 = ||x||^2,
  needs c = zeta^-1/2, taken here.  A scalar factor of Omega leaves A R^-1 unchanged.
* The random choice, made a pure function of (seed, j): Philox4x32-10 with
  counter (j lo, j hi, call, 1) and key (seed lo, seed hi) (word 3 = 1 keeps it
  apart from the Gaussian stream, whose word 3 is 0); calls 0 and 1 give eight
  32-bit words w_0..w_7 (zeta <= 8).  The rows are drawn without replacement by
  Floyd's algorithm: for k = 0..zeta-1 with t = s - zeta + k, r = floor(w_k (t + 1)
  / 2^32); row r if it is not yet chosen, else row t.  The sign of the k-th chosen
  row is - if w_k is odd.
* The sum: A's column c is put on the fixed-point grid 2^-q_c, q_c chosen from
  the column's largest magnitude and the largest number of data rows any sketch
  row receives (so no partial sum leaves 62 bits), each entry rounded to the
  nearest grid point (ties to even), and the signed sums formed exactly in
  integers; Y = 2^-q_c zeta^-1/2 (the integer sum), rounded once to FP64.  The
  grid step is about 2^-47 of the column's largest entry at the configurations'
  sizes: the sketch is exact up to that quantisation, whatever the order of the
  additions.
"""
import numpy as np

from .rng import philox4x32_10

MAX_ZETA = 8


def sparse_rows(m, s, zeta, seed):
    """(rows, signs): (m, zeta) int64 sketch rows of each data row and +-1 signs."""
    if not (1 <= zeta <= min(MAX_ZETA, s)):
        raise ValueError("1 <= zeta <= min(8, s)")
    j = np.arange(m, dtype=np.uint64)
    lo = (j & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    hi = (j >> np.uint64(32)).astype(np.uint32)
    k0 = np.uint32(seed & 0xFFFFFFFF)
    k1 = np.uint32((seed >> 32) & 0xFFFFFFFF)
    words = []
    for call in (0, 1):
        c2 = np.full(m, call, dtype=np.uint32)
        c3 = np.ones(m, dtype=np.uint32)
        x = philox4x32_10(lo, hi, c2, c3, k0, k1)
        words.extend(x)
    W = np.stack(words[:MAX_ZETA], axis=1).astype(np.uint64)        # (m, 8)
    rows = np.zeros((m, zeta), dtype=np.int64)
    for k in range(zeta):
        t = s - zeta + k
        r = ((W[:, k] * np.uint64(t + 1)) >> np.uint64(32)).astype(np.int64)
        taken = np.zeros(m, dtype=bool)
        for q in range(k):
            taken |= rows[:, q] == r
        rows[:, k] = np.where(taken, t, r)
    signs = np.where((W[:, :zeta] & np.uint64(1)) == 1, -1, 1).astype(np.int64)
    return rows, signs


def row_counts(rows, s):
    """How many data rows each sketch row receives."""
    return np.bincount(rows.ravel(), minlength=s)


def grid_exponents(M, max_count):
    """q_c with max_i |M_ic| 2^q_c <= 2^(61 - h), h = bit length of max_count (0 for a
    zero column): no partial sum of at most max_count such entries leaves 62 bits."""
    h = int(max_count).bit_length()
    cmax = np.abs(np.asarray(M, dtype=np.float64)).max(axis=0)
    _, e = np.frexp(cmax)                    # cmax = f 2^e, f in [0.5, 1)
    q = (61 - h) - e.astype(np.int64)
    return np.where(cmax == 0, 0, q)


def to_grid(x, q):
    """round(x 2^q) to the nearest integer, ties to even, as int64 (exact: from the
    FP64 significand and exponent)."""
    x = np.asarray(x, dtype=np.float64)
    u = x.view(np.uint64)
    E = ((u >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    M = (u & np.uint64((1 << 52) - 1)).astype(np.int64)
    M = np.where(E > 0, M | (1 << 52), M)
    sh = np.where(E > 0, E, 1) - 1075 + q
    out = np.zeros(x.shape, dtype=np.int64)
    up = sh >= 0
    out[up] = M[up] << sh[up]
    dn = (sh < 0) & (sh > -64)
    r = -sh[dn]
    Md = M[dn]
    qv = Md >> r
    rem = Md - (qv << r)
    half = np.int64(1) << (r - 1)
    qv = qv + ((rem > half) | ((rem == half) & ((qv & 1) == 1))).astype(np.int64)
    out[dn] = qv
    return np.where(x < 0, -out, out)


def sparse_sketch(A, b, s, zeta, seed):
    """Y = Omega [A | b] (s x (n+1), FP64) for the sparse sign embedding (see the module
    docstring): exact integer sums on the per-column grids, then one rounding."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Ab = np.concatenate([A, np.asarray(b, dtype=np.float64).reshape(-1, 1)], axis=1)
    rows, signs = sparse_rows(m, s, zeta, seed)
    counts = row_counts(rows, s)
    q = grid_exponents(Ab, counts.max())
    # Exact integer sums: each grid value is hi 2^31 + lo with |hi|, lo < 2^31, and a sketch
    # row receives at most max(counts) <= 2^22 of them, so the sums of the halves stay below
    # 2^53 and are exact in FP64 (bincount); acc = hi_sum 2^31 + lo_sum in int64.
    assert counts.max() <= 1 << 22
    idx = rows.ravel()
    sg = signs.ravel()
    acc = np.zeros((s, n + 1), dtype=np.int64)
    for c in range(n + 1):
        Qc = to_grid(Ab[:, c], q[c])
        hi, lo = Qc >> 31, Qc & ((1 << 31) - 1)
        hs = np.bincount(idx, weights=(sg * np.repeat(hi, zeta)).astype(np.float64), minlength=s)
        ls = np.bincount(idx, weights=(sg * np.repeat(lo, zeta)).astype(np.float64), minlength=s)
        acc[:, c] = hs.astype(np.int64) * (1 << 31) + ls.astype(np.int64)
    Y = np.ldexp(acc.astype(np.float64), -q[None, :])
    return Y * (1.0 / np.sqrt(float(zeta)))


def dense_omega(m, s, zeta, seed):
    """The explicit s x m matrix Omega (tiny cases only)."""
    rows, signs = sparse_rows(m, s, zeta, seed)
    Om = np.zeros((s, m))
    for k in range(zeta):
        Om[rows[:, k], np.arange(m)] = signs[:, k]
    return Om / np.sqrt(float(zeta))
