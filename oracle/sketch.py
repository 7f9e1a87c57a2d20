"""Oracle: Algorithm 1 (the sketch) -- the sketch Y = Omega [A | b] in precision u_s.

Test infrastructure only (see ``oracle/__init__.py``).

* Sec. 3.2 (one-sided diagonal scaling): each column is scaled before the
  cast to the low precision, so the largest entry sits near the top of the
  format's range; the preconditioner becomes R S^-1.  The reading taken here
  uses a power of two d_j per column (exact, so S^-1 is exact), chosen so
  that max_i |a_ij| d_j lies in [T, 2T) with T = 2^14 for f16/bf16 and
  T = 2^7 for e4m3 (T = 1, no scaling, for f32/f64).
* Alg. 1 input: "A stored in precision u_s" -- A_s = fl_s(A D), and the
  right-hand side is appended as an extra column (its own d_b) so that the
  same pass also yields Omega b, needed by the sketch-and-solve start
  x_s = R^-1 Q^T Omega b (Sec. 4).
* The sketch operand is fl_s(G) from ``oracle.rng``; Omega = s^-1/2 fl_s(G).
* The product of the rounded operands is accumulated in FP64 here (a library
  matmul is one step); the scale s^-1/2 and D^-1 are applied afterwards.
  ``accumulate="us"`` is instead the model of Sec. 3.2's error bound, the
  product formed in u_s: every product and every partial sum is rounded to
  the sketch format, summing over the rows of A in order.  Its columns are
  scaled to a largest entry in [1, 2) so that partial sums stay in range.
  It loops over the m rows (paper-sized problems only).
"""
import numpy as np

from . import rng

#: power-of-two target T for the largest entry of each scaled column
SCALE_TARGET_LOG2 = {"f64": None, "f32": None, "f16": 14, "bf16": 14, "e4m3": 7, "bf16x3": 14}


def column_scale_exponents(M, fmt):
    """Integer exponents k_j with max_i |M_ij| 2^k_j in [2^t, 2^(t+1)).

    Columns that are entirely zero get k_j = 0.  Formats without scaling
    return zeros.
    """
    M = np.asarray(M, dtype=np.float64)
    t = SCALE_TARGET_LOG2[fmt]
    if t is None:
        return np.zeros(M.shape[1], dtype=np.int64)
    cmax = np.abs(M).max(axis=0)
    _, ex = np.frexp(cmax)                 # cmax = f 2^ex, f in [0.5, 1)
    k = t - (ex.astype(np.int64) - 1)
    return np.where(cmax == 0, 0, k)


def cast_scaled(A, b, fmt):
    """Return (A_s, b_s, kA, kb): fl_s(A 2^kA), fl_s(b 2^kb) as FP64 arrays.

    For ``bf16x3`` (u_s = single on BF16 tensor cores) the operand is
    y = fl_single(A 2^k), Sec. 3.2's A_s for single precision, carried as the
    three BF16 terms hi + lo + lo2 of ``rng.split3(y)``.  A_s is their exact
    sum: y itself, except where y - hi - lo falls below BF16's normal range
    (|y| below about 2^-110), where lo2 is rounded on BF16's subnormal grid.
    """
    Ab = np.concatenate([np.asarray(A, dtype=np.float64),
                         np.asarray(b, dtype=np.float64).reshape(-1, 1)], axis=1)
    k = column_scale_exponents(Ab, fmt)
    if fmt == "bf16x3":
        y = rng.round_to_format(np.ldexp(Ab, k[None, :]), "f32")
        hi, lo, lo2 = rng.split3(y, "bf16")
        As = hi + lo + lo2
    else:
        As = rng.round_to_format(np.ldexp(Ab, k[None, :]), fmt)
    return As[:, :-1], As[:, -1], k[:-1], int(k[-1])


def sketch(A, b, s, seed, fmt, accumulate="f64"):
    """Y = Omega [A | b] with Omega = s^-1/2 fl_s(G), A and b cast to ``fmt``.

    Returns Y (s x (n+1), FP64) already unscaled: column j is divided by the
    power of two 2^k_j used for the cast, so Y approximates Omega [A | b].
    ``accumulate``: "f64" (default) or "us" (see the module docstring).
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if accumulate == "us":
        return _sketch_accumulated_in_us(A, b, s, seed, fmt)
    As, bs, kA, kb = cast_scaled(A, b, fmt)
    Ab = np.concatenate([As, bs.reshape(-1, 1)], axis=1)
    Y = np.zeros((s, n + 1))
    step = 1 << 14
    for j0 in range(0, m, step):           # blocks of A's rows; FP64 accumulation
        j1 = min(m, j0 + step)
        Gs = rng.sketch_operand(s, j0, j1, seed, fmt)
        Y += Gs @ Ab[j0:j1]
    Y *= 1.0 / np.sqrt(float(s))
    k = np.concatenate([kA, [kb]])
    return np.ldexp(Y, -k[None, :])


def _sketch_accumulated_in_us(A, b, s, seed, fmt):
    """Sec. 3.2's model: fl_s of every product and of every partial sum, rows in order."""
    m, n = A.shape
    Ab = np.concatenate([A, np.asarray(b, dtype=np.float64).reshape(-1, 1)], axis=1)
    cmax = np.abs(Ab).max(axis=0)
    _, ex = np.frexp(cmax)
    k = np.where(cmax == 0, 0, -(ex.astype(np.int64) - 1))      # largest entry in [1, 2)
    opf = rng.OPERAND_FORMAT[fmt]
    As = rng.round_to_format(np.ldexp(Ab, k[None, :]), opf)
    Gs = rng.sketch_operand(s, 0, m, seed, fmt)
    # numpy's float16 / float32 conversions are the same round-to-nearest-even as
    # rng.round_to_format (checked against each other in the tests) and much faster
    native = {"f16": np.float16, "f32": np.float32}.get(opf)
    if native is not None:
        def fl(v):
            with np.errstate(over="ignore"):
                return v.astype(native).astype(np.float64)
    else:
        def fl(v):
            return rng.round_to_format(v, opf)
    acc = np.zeros((s, n + 1))
    for j in range(m):
        acc = fl(acc + fl(np.outer(Gs[:, j], As[j])))
    return np.ldexp(acc / np.sqrt(float(s)), -k[None, :])
