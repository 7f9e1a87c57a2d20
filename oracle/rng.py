"""Oracle: the sketch matrix G (Omega = s^-1/2 G) from a counter-based stream.

Test infrastructure only (see ``oracle/__init__.py``).

The paper draws Omega with i.i.d. N(0, 1/s) entries (Sec. 2, Gaussian
embedding; Sec. 5 uses Omega = (4n)^-1/2 G with G standard normal).  It does
not say how G is drawn.  The reading taken here: G is never stored; entry
G[i, j] (i = sketch row in [0, s), j = row of A in [0, m)) is a pure function
of (i, j, seed), defined as follows.

1. Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
   easy as 1, 2, 3", SC'11): 10 rounds, multipliers 0xD2511F53 / 0xCD9E8D57,
   Weyl increments 0x9E3779B9 / 0xBB67AE85.
   counter = (j >> 2 low 32 bits, i, j >> 34, 0), key = (seed low, seed high).
2. The four output words give two (a, b) pairs: words (0, 1) serve columns
   4q+0 and 4q+1, words (2, 3) serve 4q+2 and 4q+3 (q = j >> 2).
3. U1 = (a + 1) 2^-32 in (0, 1], U2 = b 2^-32 in [0, 1).
4. Box-Muller in FP64: R = sqrt(-2 ln U1); even column -> R cos(2 pi U2),
   odd column -> R sin(2 pi U2).  If a = 2^32 - 1 (U1 = 1) the entry is +0.
   ln and (cos, sin)(2 pi U2) are the fixed IEEE-754 double operation
   sequences in ``ln_u1`` and ``cos_sin_2pi``: correctly rounded +, -, *, /
   and sqrt only, no fused multiply-add, so that any IEEE machine gives the
   same bits.
5. The entry used by a sketch in precision u_s is fl_s(G) (round to nearest,
   ties to even), see ``round_to_format``.
"""
import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (SC'11), vectorised over numpy arrays.

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (64-bit products);
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is
    bumped by the Weyl increments.  Returns four uint64 arrays holding 32-bit
    words.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        c = [(p1 >> _S32) ^ c[1] ^ k0, p1 & _MASK, (p0 >> _S32) ^ c[3] ^ k1, p0 & _MASK]
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c


# Polynomial coefficients: each is one correctly rounded IEEE division.
_ATANH_C = [1.0 / (2 * k + 1) for k in range(1, 12)]            # 1/3 .. 1/23
_SIN_C = [(-1.0) ** k / float(math.factorial(2 * k + 1)) for k in range(1, 11)]
_COS_C = [(-1.0) ** k / float(math.factorial(2 * k)) for k in range(1, 11)]
_LN2 = 0.6931471805599453          # ln 2 rounded to double
_HALF_PI = 1.5707963267948966      # pi / 2 rounded to double
_SQRT2 = 1.4142135623730951        # sqrt 2 rounded to double


def ln_u1(a):
    """FP64 ln(U1), U1 = (a + 1) 2^-32, as a fixed IEEE operation sequence.

    U1 = 2^e f with f in [sqrt(1/2), sqrt(2)); ln f = 2 atanh(z),
    z = (f - 1)/(f + 1), |z| <= 0.1716; the series 2z (1 + w/3 + w^2/5 + ...)
    with w = z^2 is truncated after w^11/23 and evaluated by Horner's rule
    with separate multiply and add; ln U1 = e ln2 + ln f.
    """
    a = np.asarray(a, dtype=np.uint64)
    u1 = (a + np.uint64(1)).astype(np.float64) * 2.0 ** -32        # exact
    fr, ex = np.frexp(u1)                                          # u1 = fr 2^ex, fr in [0.5, 1)
    f = fr * 2.0                                                   # [1, 2), exact
    e = (ex - 1).astype(np.float64)
    big = f > _SQRT2
    f = np.where(big, f * 0.5, f)
    e = np.where(big, e + 1.0, e)
    z = (f - 1.0) / (f + 1.0)
    w = z * z
    p = np.full_like(w, _ATANH_C[-1])
    for ck in reversed(_ATANH_C[:-1]):
        p = ck + w * p
    z2 = z * 2.0
    lnf = z2 + z2 * (w * p)
    return e * _LN2 + lnf


def cos_sin_2pi(b):
    """FP64 (cos, sin)(2 pi U2), U2 = b 2^-32, as a fixed IEEE operation sequence.

    4 U2 = q + r with the quadrant q = b >> 30 and r in [0, 1) exact; r is
    moved to [-1/2, 1/2) (q += 1 when r >= 1/2); phi = r * (pi/2)_double;
    sin and cos of phi by their Taylor series to phi^21 / phi^20 (Horner,
    separate multiply and add); the quadrant then rotates (cos, sin).
    """
    b = np.asarray(b, dtype=np.uint64)
    q = (b >> np.uint64(30)).astype(np.int64)
    rb = (b & np.uint64(0x3FFFFFFF)).astype(np.int64)
    wrap = rb >= (1 << 29)
    rb = np.where(wrap, rb - (1 << 30), rb)
    q = np.where(wrap, q + 1, q) & 3
    r = rb.astype(np.float64) * 2.0 ** -30                          # exact
    phi = r * _HALF_PI
    w = phi * phi
    ps = np.full_like(w, _SIN_C[-1])
    for ck in reversed(_SIN_C[:-1]):
        ps = ck + w * ps
    sphi = phi + phi * (w * ps)
    pc = np.full_like(w, _COS_C[-1])
    for ck in reversed(_COS_C[:-1]):
        pc = ck + w * pc
    cphi = 1.0 + w * pc
    cos_t = np.select([q == 0, q == 1, q == 2], [cphi, -sphi, -cphi], sphi)
    sin_t = np.select([q == 0, q == 1, q == 2], [sphi, cphi, -sphi], -cphi)
    return cos_t, sin_t


def gaussian_pair(a, b):
    """FP64 Box-Muller of one (a, b) word pair -> (G_even, G_odd)."""
    a = np.asarray(a, dtype=np.uint64)
    lnu = ln_u1(a)
    rad = np.sqrt(-2.0 * lnu)
    ct, st = cos_sin_2pi(b)
    ge = rad * ct
    go = rad * st
    one = a == np.uint64(0xFFFFFFFF)
    return np.where(one, 0.0, ge), np.where(one, 0.0, go)


def gaussian_block(i0, i1, j0, j1, seed):
    """G[i0:i1, j0:j1] in FP64 (rows = sketch rows, columns = rows of A)."""
    ii = np.arange(i0, i1, dtype=np.uint64)[:, None]
    jj = np.arange(j0, j1, dtype=np.uint64)[None, :]
    q = jj >> np.uint64(2)
    t = (jj & np.uint64(3)).astype(np.int64)
    ii, q = np.broadcast_arrays(ii, q)
    seed = int(seed)
    x0, x1, x2, x3 = philox4x32_10(q & _MASK, ii, q >> _S32, np.zeros_like(q),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    a = np.where(t < 2, x0, x2)
    b = np.where(t < 2, x1, x3)
    ge, go = gaussian_pair(a, b)
    return np.where((t & 1) == 0, ge, go)


# ---------------------------------------------------------------------------
# Rounding to the sketch precision u_s (round to nearest, ties to even).
# ---------------------------------------------------------------------------
#: name -> (mantissa bits, minimum normal exponent, largest finite value, saturate)
FORMATS = {
    "f64": None,
    "f32": (23, -126, float(np.finfo(np.float32).max), False),
    "f16": (10, -14, 65504.0, False),
    "bf16": (7, -126, float.fromhex("0x1.fep127"), False),
    "e4m3": (3, -6, 448.0, True),
}

#: unit roundoff of each format (2^-(mantissa bits + 1)); "bf16x3" is the
#: single-precision cast of A carried as its three-term BF16 split, with FP32
#: accumulation, i.e. single precision.
UNIT_ROUNDOFF = {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "f16": 2.0 ** -11,
                 "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4, "bf16x3": 2.0 ** -24}

#: format of the sketch operand fl_s(G) for each sketch precision
OPERAND_FORMAT = {"f64": "f64", "f32": "f32", "f16": "f16", "bf16": "bf16", "e4m3": "e4m3",
                  "bf16x3": "bf16"}


def round_to_format(x, fmt):
    """Round FP64 values to the format ``fmt`` (result returned as FP64).

    Direct single rounding of the FP64 value: scale by a power of two so that
    the format's unit in the last place becomes 1 (normal or subnormal
    range), round to the nearest integer with ties to even, scale back.
    Out-of-range values saturate to the largest finite value for e4m3
    (the 'satfinite' conversion) and become +-inf otherwise.
    """
    x = np.asarray(x, dtype=np.float64)
    spec = FORMATS[fmt]
    if spec is None:
        return x.copy()
    mbits, emin, xmax, sat = spec
    _, ex = np.frexp(x)                      # |x| = f 2^ex, f in [0.5, 1)
    lead = ex.astype(np.int64) - 1            # exponent of the leading bit
    q = np.maximum(lead, emin) - mbits        # exponent of one ulp
    y = np.rint(np.ldexp(x, -q))              # rint: ties to even
    out = np.ldexp(y, q)
    out = np.where(x == 0, x, out)
    over = np.abs(out) > xmax
    if sat:
        out = np.where(over, np.copysign(xmax, x), out)
    else:
        out = np.where(over, np.copysign(np.inf, x), out)
    return out


def sketch_operand(s, j0, j1, seed, fmt):
    """fl_s(G)[0:s, j0:j1] -- the sketch operand as used in precision ``fmt``."""
    return round_to_format(gaussian_block(0, s, j0, j1, seed), OPERAND_FORMAT[fmt])


def split3(x, fmt="bf16"):
    """Three-term split x ~ hi + lo + lo2 with each term in ``fmt``.

    hi = fl(x), lo = fl(x - hi), lo2 = fl(x - hi - lo); the differences are exact
    in FP64 for BF16 terms, so the sum carries 3 x 8 significant bits of x.
    """
    x = np.asarray(x, dtype=np.float64)
    hi = round_to_format(x, fmt)
    r1 = x - hi
    lo = round_to_format(r1, fmt)
    lo2 = round_to_format(r1 - lo, fmt)
    return hi, lo, lo2
