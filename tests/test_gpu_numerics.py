"""The library's own device arithmetic helpers (grmhd_numerics_eval) held to their
definitions: exact values from Python's decimal arithmetic (60 digits, each double
converted exactly), numpy's IEEE binary32 rounding, and CUDA's own FP64 reciprocal and
reciprocal square root (torch on the device) beside them.

- rsqrt_ge1 and rcp_pos (an FP32 estimate and one correction of order three): within
  one ulp of the exact value, and of CUDA's results.
- d2f / f2d (binary64 <-> binary32 on the integer pipe): numpy's round-to-nearest-even
  except at exact ties (rounded away from zero), signed zero below the normal binary32
  range, infinity above it, NaN kept; f2d exact for normal values.
- double-word split, sum, product, reciprocal and square root: within 2^-44 of the
  exact result (the split to 2^-48).
- exponent moves x/4, 2x: exact in the normal range, the stated flushes outside it.
- minmod3 (binary64 and binary32), the sign of a product, the PPM limits: the
  definitions in exact arithmetic, decided on the same inputs.
- the integer-pipe tests finite / positive / |x| < 1e10."""
import math
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

getcontext().prec = 60


@pytest.fixture(scope="module")
def G():
    from paper_2110_03732_gb300 import build, grmhd
    build.build()
    return grmhd


def run(G, name, x):
    t = torch.as_tensor(np.asarray(x, dtype=np.float64), device="cuda")
    out = G.numerics_eval(name, t)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def ulps(got, exact):
    """|got - exact| in units of the last place of the double nearest exact."""
    ref = float(exact)
    return float(abs(Decimal(float(got)) - exact) / Decimal(float(np.spacing(abs(ref)))))


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.uint64)


def test_rsqrt_ge1_within_an_ulp(G):
    rng = np.random.default_rng(11)
    x = np.concatenate([10.0 ** rng.uniform(0, 30, 3000), 1.0 + rng.uniform(0, 1e-3, 500),
                        [1.0, np.nextafter(1.0, 2.0), 2.0, 3.0, 4.0, 2.0 ** 100, 1e30, 2.0 ** 126]])
    y = run(G, "rsqrt_ge1", x)
    cu = torch.rsqrt(torch.as_tensor(x, device="cuda")).cpu().numpy()
    worst = max(ulps(y[i], 1 / Decimal(float(x[i])).sqrt()) for i in range(len(x)))
    print(f"rsqrt_ge1: worst {worst:.3f} ulp")
    assert worst <= 1.0
    assert np.all(np.abs(y - cu) <= np.spacing(np.abs(cu)))


def test_rcp_pos_within_an_ulp(G):
    rng = np.random.default_rng(12)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 3000), [1.0, 2.0, 3.0, 0.1, 1e-30, 1e30, 2.0 ** -100]])
    y = run(G, "rcp_pos", x)
    cu = torch.reciprocal(torch.as_tensor(x, device="cuda")).cpu().numpy()
    worst = max(ulps(y[i], 1 / Decimal(float(x[i]))) for i in range(len(x)))
    print(f"rcp_pos: worst {worst:.3f} ulp")
    assert worst <= 1.0
    assert np.all(np.abs(y - cu) <= np.spacing(np.abs(cu)))


def _f32_ties(rng, n):
    """Doubles exactly halfway between two adjacent binary32 values."""
    f = rng.uniform(1, 2, n).astype(np.float32) * np.float32(2.0) ** rng.integers(-100, 100, n).astype(np.float32)
    f = f * np.where(rng.random(n) < 0.5, -1, 1).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf) * np.sign(f))
    return (f.astype(np.float64) + up.astype(np.float64)) / 2, f, up


def test_d2f_rounding_and_range(G):
    rng = np.random.default_rng(13)
    n = 6000
    x = np.ldexp(rng.uniform(1, 2, n), rng.integers(-130, 129, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    y = run(G, "d2f", x)
    small = np.abs(x) < 2.0 ** -126
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    # round to nearest away from ties: equal to numpy's RNE (ties have probability 0 here)
    assert np.array_equal(y[~small], ref[~small])
    # below the normal binary32 range: a signed zero
    assert np.all(y[small] == 0) and np.array_equal(np.signbit(y[small]), np.signbit(x[small]))
    # exact ties round away from zero
    t, f, up = _f32_ties(rng, 500)
    yt = run(G, "d2f", t)
    assert np.array_equal(yt, up.astype(np.float64))
    # special values
    s = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.5e38, -3.5e38, float(np.finfo(np.float32).max)])
    ys = run(G, "d2f", s)
    assert ys[0] == 0 and not np.signbit(ys[0]) and ys[1] == 0 and np.signbit(ys[1])
    assert ys[2] == np.inf and ys[3] == -np.inf and np.isnan(ys[4])
    assert ys[5] == np.inf and ys[6] == -np.inf and ys[7] == float(np.finfo(np.float32).max)


def test_f2d_exact(G):
    rng = np.random.default_rng(14)
    f = rng.integers(0, 2 ** 32, 20000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38],
                                    dtype=np.float32)])
    with np.errstate(invalid="ignore"):
        x = f.astype(np.float64)
    y = run(G, "f2d", x)
    sub = (np.abs(f) < np.finfo(np.float32).tiny) & (f != 0)
    nan = np.isnan(f)
    ok = ~sub & ~nan
    assert np.array_equal(bits(y[ok]), bits(x[ok]))   # exact, signed zeros and infinities included
    assert np.all(y[sub] == 0) and np.array_equal(np.signbit(y[sub]), np.signbit(x[sub]))
    assert np.all(np.isnan(y[nan]))


def test_double_word_split(G):
    rng = np.random.default_rng(15)
    n = 4000
    x = np.ldexp(rng.uniform(1, 2, n), rng.integers(-70, 120, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    hl = run(G, "dw_split", x)
    for i in range(n):
        hi, lo = hl[i]
        assert np.float32(hi) == hi and np.float32(lo) == lo
        assert abs(Decimal(float(x[i])) - Decimal(float(hi))) <= abs(Decimal(float(np.spacing(np.float32(hi))))) / 2
        err = abs(Decimal(float(x[i])) - Decimal(float(hi)) - Decimal(float(lo)))
        assert err <= Decimal(2.0 ** -48) * abs(Decimal(float(x[i])))


def _dw(v):
    return Decimal(float(v[0])) + Decimal(float(v[1]))


def test_double_word_operations(G):
    rng = np.random.default_rng(16)
    n = 2000
    a = np.ldexp(rng.uniform(1, 2, n), rng.integers(-40, 40, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    b = a * np.ldexp(rng.uniform(0.5, 2, n), rng.integers(-20, 20, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    s = run(G, "dw_add", np.stack([a, b], 1))
    p = run(G, "dw_mul", np.stack([a, b], 1))
    pos = np.abs(a)
    r = run(G, "dw_rcp", pos)
    q = run(G, "dw_sqrt", pos)
    e44 = Decimal(2.0 ** -44)
    for i in range(n):
        A, B = Decimal(float(a[i])), Decimal(float(b[i]))
        assert abs(_dw(s[i]) - (A + B)) <= e44 * (abs(A) + abs(B))
        assert abs(_dw(p[i]) - A * B) <= e44 * abs(A * B)
        P = abs(A)
        assert abs(_dw(r[i]) - 1 / P) <= e44 / P
        assert abs(_dw(q[i]) - P.sqrt()) <= e44 * P.sqrt()


def test_exponent_moves(G):
    rng = np.random.default_rng(17)
    n = 4000
    x = np.ldexp(rng.uniform(1, 2, n), rng.integers(-1024, 1024, n)) * np.where(rng.random(n) < 0.5, -1, 1)
    x = np.concatenate([x, [0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 2.0 ** -1021, 2.0 ** 1023, -2.0 ** 1023]])
    q = run(G, "quarter", x)
    t = run(G, "twice", x)
    fin = np.isfinite(x)
    with np.errstate(over="ignore", under="ignore"):
        qe, te = x / 4, x * 2
    qn = fin & (np.abs(qe) >= 2.0 ** -1022)          # normal results: exact
    assert np.array_equal(q[qn], qe[qn])
    qz = fin & ~qn                                   # below the normal range: a signed zero
    assert np.all(q[qz] == 0) and np.array_equal(np.signbit(q[qz]), np.signbit(x[qz]))
    tn = fin & (x != 0) & (np.abs(x) >= 2.0 ** -1022)
    assert np.array_equal(t[tn], te[tn])             # overflow gives the signed infinity too
    tz = fin & ~tn
    assert np.all(t[tz] == 0) and np.array_equal(np.signbit(t[tz]), np.signbit(x[tz]))
    assert np.array_equal(q[~fin][:2], x[~fin][:2]) and np.isnan(q[~fin][2])
    assert np.array_equal(t[~fin][:2], x[~fin][:2]) and np.isnan(t[~fin][2])


def _minmod_ref(a, b, c):
    sb = [math.copysign(1.0, v) < 0 for v in (a, b, c)]
    if sb[0] != sb[1] or sb[0] != sb[2]:
        return 0.0
    best = a
    for v in (b, c):
        if abs(v) < abs(best):
            best = v
    return best


@pytest.mark.parametrize("name,dt", [("minmod3", np.float64), ("minmod3_f32", np.float32)])
def test_minmod3_is_the_definition(G, name, dt):
    rng = np.random.default_rng(18)
    pool = np.array([0.0, -0.0, 1.0, -1.0, 0.5, -0.5, 2.0, 1e-300, -1e-300, 3.0], dtype=np.float64)
    n = 6000
    x = np.where(rng.random((n, 3)) < 0.5, rng.choice(pool, (n, 3)), rng.normal(0, 1, (n, 3))).astype(dt)
    x = x.astype(np.float64)
    y = run(G, name, x)
    for i in range(n):
        ref = _minmod_ref(*x[i])
        assert bits(y[i]) == bits(np.float64(ref)) or (ref == 0 and y[i] == 0 and not np.signbit(y[i])), (x[i], y[i])


def test_product_sign(G):
    rng = np.random.default_rng(19)
    pool = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, -5e-324, 1e300, -1e300])
    n = 4000
    x = np.where(rng.random((n, 2)) < 0.5, rng.choice(pool, (n, 2)), rng.normal(0, 1, (n, 2)))
    y = run(G, "prod_sign", x)
    ref = np.where((x[:, 0] == 0) | (x[:, 1] == 0), 0.0,
                   np.where(np.signbit(x[:, 0]) == np.signbit(x[:, 1]), 1.0, -1.0))
    assert np.array_equal(y, ref)


def _ppm_ref(a0, aL, aR):
    """Colella & Woodward's limits in exact rational arithmetic; returns the edges and
    whether the second decision is clear of rounding (its product not near zero)."""
    A0, L, R = Fraction(a0), Fraction(aL), Fraction(aR)
    if (R - A0) * (A0 - L) <= 0:
        return A0, A0, True
    dd = R - L
    m6 = 6 * (A0 - (L + R) / 2)
    t1 = dd * (m6 - dd)          # dd m6 > dd^2  <=>  dd (3 a0 - aL - 2 aR) > 0
    t2 = dd * (m6 + dd)          # -dd^2 > dd m6 <=>  dd (3 a0 - 2 aL - aR) < 0
    scale = (abs(A0) + abs(L) + abs(R)) ** 2
    clear = abs(t1) > scale * Fraction(1, 10 ** 12) and abs(t2) > scale * Fraction(1, 10 ** 12)
    if t1 > 0:
        return 3 * A0 - 2 * R, R, clear
    if t2 < 0:
        return L, 3 * A0 - 2 * L, clear
    return L, R, clear


def test_ppm_limit_is_the_definition(G):
    rng = np.random.default_rng(20)
    n = 4000
    x = rng.normal(0, 1, (n, 3))
    x[: n // 8, 2] = x[: n // 8, 0]             # aR = a0: a flat edge (extremum test at equality)
    x[n // 8: n // 4, 1] = x[n // 8: n // 4, 0]  # aL = a0
    y = run(G, "ppm_limit", x)
    checked = 0
    for i in range(n):
        L, R, clear = _ppm_ref(*x[i])
        if not clear:
            continue
        checked += 1
        tol = 8 * np.spacing(3 * np.max(np.abs(x[i])))
        assert abs(float(L) - y[i, 0]) <= tol and abs(float(R) - y[i, 1]) <= tol, (x[i], y[i], float(L), float(R))
    assert checked > 0.95 * n


def test_integer_pipe_tests(G):
    x = np.array([0.0, -0.0, 1.0, -1.0, 5e-324, np.inf, -np.inf, np.nan, 9.9e9, 1e10, -9.9e9, -1e10, 1e300, 9.999e9])
    y = run(G, "tests", x).astype(int)
    fin = np.isfinite(x)
    pos = fin & (x > 0)
    below = fin & (np.abs(x) < 0.99999e10)
    above = ~fin | (np.abs(x) >= 1e10)
    assert np.array_equal(y & 1, fin.astype(int))
    assert np.array_equal((y >> 1) & 1, pos.astype(int))
    assert np.all(((y >> 2) & 1)[below] == 1) and np.all(((y >> 2) & 1)[above] == 0)


def test_numerics_eval_rejects_bad_arguments(G):
    L = G.lib()
    assert L.grmhd_numerics_eval(-1, None, None, 0, None) == G.GRMHD_ERR_ARG
    assert L.grmhd_numerics_eval(99, None, None, 0, None) == G.GRMHD_ERR_ARG
    assert L.grmhd_numerics_eval(0, None, None, -1, None) == G.GRMHD_ERR_ARG
    assert L.grmhd_numerics_eval(0, None, None, 4, None) == G.GRMHD_ERR_ARG
    assert L.grmhd_numerics_eval(0, None, None, 0, None) == 0
