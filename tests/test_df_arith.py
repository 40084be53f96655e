"""Host emulation of the FP64 form's divisor arithmetic on the FP32 pipe
(phi_kernels.cuh: df_cut, df_widen, df_dot, df_add, df_divide), step for
step in numpy float32, against exact rational arithmetic.

It pins the derived bound the FP64 parity claim rests on: v = x / max(s, eps)
with s = <B[i_n], pi> over up to 4 lanes of 8 ranks is within 7.5e-13
relative (first-order analysis in phi_kernels.cuh), with operands spread
over 30 decades, entries below the float range, zeros, and a reciprocal
estimate one ulp off at random (the hardware estimate's stated error)."""
import struct
from fractions import Fraction

import numpy as np

f32 = np.float32


def _u2f(u):
    return f32(struct.unpack("<f", struct.pack("<I", u & 0xFFFFFFFF))[0])


def _f2u(f):
    return struct.unpack("<I", struct.pack("<f", f))[0]


def _d2u(d):
    return struct.unpack("<Q", struct.pack("<d", d))[0]


def _u2d(u):
    return struct.unpack("<d", struct.pack("<Q", u & 0xFFFFFFFFFFFFFFFF))[0]


def fmaf(a, b, c):
    # a*b of two floats is exact in double; the sum is then rounded once to
    # double and once to float, which is close enough for an error check
    return f32(float(a) * float(b) + float(c))


def cut(x):
    """x >= 0 as hi + lo floats (48 leading bits); big for x >= 2^31."""
    bits = _d2u(x)
    H, L = bits >> 32, bits & 0xFFFFFFFF
    e = H >> 20
    big = e >= 1023 + 31
    if e < 1023 - 126:
        return f32(0), f32(0), big
    hi = _u2f((((H << 3) | (L >> 29)) & 0xFFFFFFFF) - (896 << 23))
    v = L & 0x1FFFFFFF
    nb = v.bit_length()
    if nb > 24:  # integer-to-float conversion rounding toward zero
        v = (v >> (nb - 24)) << (nb - 24)
    lo = f32(f32(f32(v) * _u2f((e - 1075 + 64 + 127) << 23)) * f32(2.0 ** -64))
    return hi, lo, big


def widen(f):
    b = _f2u(f)
    if (b & 0x7F800000) == 0:
        return 0.0
    return _u2d((((b & 0x7FFFFFFF) << 29) + (896 << 52)) | ((b & 0x80000000) << 32))


def dot_pair(a, b):
    S = C = D = f32(0)
    big = False
    for ar, br in zip(a, b):
        ah, al, g1 = cut(ar)
        bh, bl, g2 = cut(br)
        big = big or g1 or g2
        p = f32(ah * bh)
        D = f32(fmaf(ah, bh, -p) + D)
        D = fmaf(ah, bl, D)
        D = fmaf(al, bh, D)
        t = f32(S + p)
        z = f32(t - S)
        C = f32(C + f32(f32(S - f32(t - z)) + f32(p - z)))
        S = t
    E = f32(C + D)
    h = f32(S + E)
    return (h, f32(E - f32(h - S))), big


def add_pair(a, b):
    s = f32(a[0] + b[0])
    z = f32(s - a[0])
    e = f32(f32(f32(a[0] - f32(s - z)) + f32(b[0] - z)) + f32(a[1] + b[1]))
    h = f32(s + e)
    return h, f32(e - f32(h - s))


def divide(x, s, eh, el, rcp):
    xh, xl, _ = cut(x)
    use_s = f32(f32(s[0] - eh) + f32(s[1] - el)) >= 0
    mh, ml = (s[0], s[1]) if use_s else (eh, el)
    r = rcp(mh)
    q0 = f32(xh * r)
    p = f32(q0 * mh)
    pe = fmaf(q0, mh, -p)
    res = f32(f32(f32(xh - p) - pe) + fmaf(-q0, ml, xl))
    return widen(q0) + widen(f32(res * r))


def test_divisor_on_fp32_pipe_within_derived_bound():
    rng = np.random.default_rng(2024)

    def rcp(m):
        r = f32(1.0 / float(m))
        d = rng.integers(-1, 2)
        return np.nextafter(r, f32(np.inf)) if d > 0 else (np.nextafter(r, f32(0)) if d < 0 else r)

    eps = 1e-10
    eh, el, _ = cut(eps)
    worst = 0.0
    for trial in range(600):
        lanes = int(rng.choice([1, 2, 4]))
        sa, sb = 10.0 ** rng.uniform(-12, 6), 10.0 ** rng.uniform(-25, 0)
        exact = Fraction(0)
        tot = None
        for _ in range(lanes):
            a = rng.random(8) * sa
            b = rng.random(8) * sb
            if trial % 7 == 0:
                b[rng.integers(8)] = 1e-40  # below the float range: dropped
            if trial % 11 == 0:
                a[rng.integers(8)] = 0.0
            exact += sum(Fraction(float(p)) * Fraction(float(q)) for p, q in zip(a, b))
            part, big = dot_pair(list(a), list(b))
            assert not big
            tot = part if tot is None else add_pair(tot, part)
        x = float(rng.choice([1.0, 2.0, 7.0, 123.0, 1e5, 2.0 ** 30, 0.37, 2.0 ** -19]))
        if trial % 13 == 0:
            x = 0.0
        got = divide(x, tot, eh, el, rcp)
        want = Fraction(x) / max(exact, Fraction(eps))
        err = abs(Fraction(got) - want) / want if want else abs(Fraction(got))
        worst = max(worst, float(err))
    assert worst < 7.5e-13
    assert worst < 2e-13  # far inside the first-order bound in practice (3.9e-14 here)


def test_cut_and_widen_special_values():
    for x in [1.0, 3.14159, 1e-20, 2.0 ** -120, 2.0 ** -126, 1e8, 2.0 ** 30]:
        h, l, big = cut(x)
        assert not big
        assert abs(float(h) + float(l) - x) <= 2.0 ** -47 * x
    assert cut(2.0 ** 31)[2]
    assert cut(2.0 ** -127)[:2] == (0.0, 0.0)
    assert cut(0.0)[:2] == (0.0, 0.0)
    assert widen(f32(1.5)) == 1.5
    assert widen(f32(-2.5e-30)) == float(f32(-2.5e-30))
    assert widen(f32(1e-40)) == 0.0  # subnormal floats widen to zero


def _to_f32_bits(d):
    """The integer rounding of internal.cuh's to_f32 for doubles whose float
    is normal (None where the kernel takes the conversion instruction)."""
    u = _d2u(d)
    e = (u >> 52) & 0x7FF
    if e < 1023 - 126 or e > 1023 + 127:
        return None
    rem = u & 0x1FFFFFFF
    r = ((e - 896) << 23) | ((u >> 29) & 0x7FFFFF)
    r += 1 if (rem > 0x10000000 or (rem == 0x10000000 and (r & 1))) else 0
    return r | ((u >> 32) & 0x80000000)


def test_float_double_conversions_by_integer_operations_are_exact():
    """to_f32 (round to nearest even) and to_f64 equal the conversions, bit for
    bit, over random doubles, exact ties, carries into the exponent and the
    edges of the float range."""
    rng = np.random.default_rng(7)
    xs = list(rng.random(20000) * 10.0 ** rng.uniform(-37, 38, 20000))
    xs += [float(np.float32(x)) for x in xs[:2000]]  # exact floats
    for x in xs[:3000]:  # ties: half an ulp of the float above its value
        f = np.float32(x)
        xs.append(float(f) + (float(np.nextafter(f, np.float32(np.inf))) - float(f)) / 2)
    xs += [1.0, 2.0 ** -126, 2.0 ** 127 * (2 - 2.0 ** -23), 2.0 ** 127 * (2 - 2.0 ** -24), 3.4028235677973366e38,
           1.0 - 2.0 ** -25, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24]
    checked = 0
    for x in xs:
        for v in (x, -x):
            r = _to_f32_bits(v)
            if r is None:
                continue
            with np.errstate(over="ignore"):
                want = _f2u(np.float32(v))
            assert r == want, (v, hex(r), hex(want))
            checked += 1
            f = _u2f(r)
            if np.isfinite(f) and f != 0:
                assert widen(f) == float(f)  # to_f64 of a normal float: the df_widen bits
    assert checked > 40000


def _hi_of(x):
    """internal phi_kernels.cuh hi_of: the leading 24 bits of x >= 0 as a float
    (None outside the float range)."""
    if x == 0.0:
        return f32(0)
    bits = _d2u(x)
    e = bits >> 52
    if not (1023 - 126 <= e < 1023 + 127):
        return None
    H, L = bits >> 32, bits & 0xFFFFFFFF
    return _u2f((((H << 3) | (L >> 29)) & 0xFFFFFFFF) - (896 << 23))


def test_kkt_estimate_margin_covers_the_exact_term():
    """The FP64 kernel takes a KKT term |min(b, 1 - phi)| in FP64 only where
    its FP32 estimate from the leading 24 bits of b and phi, plus the margin
    2^-21 (1 + phi_hi + b_hi), reaches the running maximum.  The estimate must
    be within half that margin of the exact term, so that no term above the
    maximum is skipped: checked against exact rationals over values near 1
    (where 1 - phi cancels), tiny (b below the float range), large and zero."""
    rng = np.random.default_rng(11)
    cases = []
    for _ in range(20000):
        kind = rng.integers(5)
        if kind == 0:
            phi = 1.0 + rng.normal() * 10.0 ** rng.uniform(-12, -1)
        elif kind == 1:
            phi = 10.0 ** rng.uniform(-40, 6)
        elif kind == 2:
            phi = 0.0
        else:
            phi = rng.random() * 3
        b = 0.0 if rng.integers(7) == 0 else 10.0 ** rng.uniform(-45, 3)
        cases.append((abs(phi), b))
    for phi, b in cases:
        ph = _hi_of(phi)
        bh, _, big = cut(b)  # the B row's hi floats of the kernel (0 below 2^-126)
        if ph is None or big:
            continue  # the kernel takes the exact term there
        est = abs(min(float(bh), float(f32(f32(1.0) - ph))))
        exact = abs(min(Fraction(b), 1 - Fraction(phi)))
        margin = 2.0 ** -21 * (1.0 + float(ph) + float(bh))
        assert abs(Fraction(est) - exact) <= Fraction(margin) / 2, (phi, b)
