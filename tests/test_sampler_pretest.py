"""The FP32 pre-test of the sampler's acceptance test (calF of Eq. 62, one Yukawa term).

The acceptance test u (A t + Q2a) < A t, A t = A (k^2 + lambda^-2), is evaluated in FP64
(IEEE operations in a fixed order, the oracle's test).  The GPU first forms, in FP32,
D32 = fma(-u32, den, At32) with den = At32 + Q2a32 and u32 the leading 24 bits of u, and
takes the FP64 test only when |D32| <= 1e-5 den.  Its comment states that D32 is within
2e-6 (A t + Q2a) of D = At64 - u (At64 + Q2a) in real arithmetic, so that a decided draw
agrees with the FP64 test.  This test emulates the FP32 steps with numpy float32 (a fused
multiply-add as one FP64 evaluation rounded to FP32) and checks, with exact rationals:
  * |D32 - D| <= 2e-6 (At64 + Q2a) on draws over wide parameter ranges;
  * every draw the pre-test decides is decided as the FP64 test decides it;
  * the pre-test leaves open only a small fraction of the draws.
"""
from fractions import Fraction

import numpy as np
import pytest

F32 = np.float32


def fma32(a, b, c):
    return F32(float(a) * float(b) + float(c))


def pretest(tpl, n, A, il2, Q2a, wx, wy):
    """(D32, den) as the GPU forms them, or None when its range checks send the draw to FP64."""
    u32 = F32(float(((wx >> 11) << 3) | (wy >> 29)) * 5.9604644775390625e-8)
    tplf = [F32(t) for t in tpl]
    kx, ky, kz = (F32(tplf[d] * F32(n[d])) for d in range(3))
    k2 = fma32(kz, kz, fma32(ky, ky, F32(kx * kx)))
    At = F32(F32(A) * F32(k2 + F32(il2)))
    den = F32(At + F32(Q2a))
    if not (At >= F32(1e-25) and den <= F32(1e30)):
        return None
    return fma32(F32(-u32), den, At), den


def fp64_test(tpl, n, A, il2, Q2a, wx, wy):
    """The oracle's test and its FP64 operands: (accept, At64, u)."""
    u = float(((wx >> 11) << 32) | wy) * 1.1102230246251565404e-16
    kx, ky, kz = (tpl[d] * float(n[d]) for d in range(3))
    k2 = (kx * kx + ky * ky) + kz * kz
    At = A * (k2 + il2)
    return u * (At + Q2a) < At, At, u


def draws(seed, count):
    rng = np.random.default_rng(seed)
    for _ in range(count):
        tpl = [float(10 ** rng.uniform(-3, 1))] * 3
        n = [int(v) for v in rng.integers(-40, 41, 3)]
        if n == [0, 0, 0]:
            n[0] = 1
        A = float(10 ** rng.uniform(-3, 6))
        il2 = float(10 ** rng.uniform(-3, 2)) if rng.random() < 0.9 else 0.0
        Q2a = float(10 ** rng.uniform(0, 7))
        wx, wy = int(rng.integers(0, 2**32)), int(rng.integers(0, 2**32))
        yield tpl, n, A, il2, Q2a, wx, wy


def near_threshold(seed, count):
    """Draws whose u sits within a few 1e-5 of the acceptance probability: the pre-test's
    margin is exercised from both sides."""
    rng = np.random.default_rng(seed)
    for tpl, n, A, il2, Q2a, _, _ in draws(seed + 1, count):
        _, At, _ = fp64_test(tpl, n, A, il2, Q2a, 0, 0)
        p = At / (At + Q2a)
        u = min(max(p * (1.0 + rng.uniform(-4e-5, 4e-5)), 0.0), 1.0 - 2**-53)
        U = int(u * 2**53)
        yield tpl, n, A, il2, Q2a, ((U >> 32) << 11) | int(rng.integers(0, 2**11)), U & 0xffffffff


@pytest.mark.parametrize("source", ["wide", "threshold"])
def test_pretest_bound_and_decisions(source):
    gen = draws(11, 6000) if source == "wide" else near_threshold(23, 6000)
    decided = opened = 0
    for tpl, n, A, il2, Q2a, wx, wy in gen:
        acc64, At64, u = fp64_test(tpl, n, A, il2, Q2a, wx, wy)
        pt = pretest(tpl, n, A, il2, Q2a, wx, wy)
        if pt is None:
            opened += 1
            continue
        D32, den = pt
        D = Fraction(At64) - Fraction(u) * (Fraction(At64) + Fraction(Q2a))
        err = abs(Fraction(float(D32)) - D)
        assert err <= Fraction(2, 10**6) * (Fraction(At64) + Fraction(Q2a)), (tpl, n, A, il2, Q2a, float(err))
        m = F32(F32(1e-5) * den)
        if D32 > m:
            decided += 1
            assert acc64, "pre-test accepts what the FP64 test rejects"
        elif D32 < -m:
            decided += 1
            assert not acc64, "pre-test rejects what the FP64 test accepts"
        else:
            opened += 1
    total = decided + opened
    if source == "wide":
        assert opened <= 0.001 * total, (opened, total)
    else:
        # the draws sit within 4e-5 of the threshold, so many are left to FP64, and all the
        # rest must still agree (checked above)
        assert decided > 0 and opened > 0, (decided, opened)
