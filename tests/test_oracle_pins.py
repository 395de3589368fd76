"""Pins of the CPU oracle against facts that do not come from the oracle itself.

* STREAM's closed form (Section 5, Listing 4 with q=3 from a=1, b=2, c=0): exact in binary64
  for k<=13 passes and in binary32 for k<=6; within a proven error bound beyond.
* Hand-derived IEEE-754 cases (``tests/golden/rounding_cases.txt``): ties to even, two
  roundings in Triad (no fused multiply-add), signed zeros, subnormals, overflow, NaN bits.
* numpy's elementwise ufuncs, which compute add and multiply with one IEEE rounding each:
  Add and Scale are exactly ``np.add``/``np.multiply``; Triad is ``np.add(b, np.multiply(c, q))``.
* The pass invariant ``c == 4*a_prev`` (proof in ``test_invariant_c_is_four_a``).
* Seeded inputs: SplitMix64's published first outputs from state 0.

``test_planted_mistakes_are_caught`` compiles deliberately broken copies of the oracle and
checks that these pins reject each one.
"""
import math
import os
import struct
from fractions import Fraction

import numpy as np
import pytest

import oracle
import stream_inputs as si

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = Fraction(1, 2 ** 53)
U32 = Fraction(1, 2 ** 24)


# ----------------------------------------------------------------------------------------
# golden parsing
# ----------------------------------------------------------------------------------------

def _parse_value(tok, dtype):
    if tok == "-":
        return None
    if tok.startswith("bits:"):
        bits = int(tok[5:], 16)
        if dtype == np.float64:
            return np.frombuffer(struct.pack("<Q", bits), np.float64)[0]
        return np.frombuffer(struct.pack("<I", bits), np.float32)[0]
    if tok in ("inf", "-inf"):
        return dtype(float(tok))
    return dtype(float.fromhex(tok))


def rounding_cases():
    cases = []
    with open(os.path.join(GOLDEN, "rounding_cases.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split(None, 6)
            dt = np.float64 if parts[0] == "f64" else np.float32
            op = parts[1]
            x, y = _parse_value(parts[2], dt), _parse_value(parts[3], dt)
            q = 0.0 if parts[4] == "-" else float.fromhex(parts[4])
            exp = _parse_value(parts[5], dt)
            cases.append((dt, op, x, y, q, exp, parts[6] if len(parts) > 6 else ""))
    return cases


def bits(a):
    a = np.asarray(a)
    return a.view(np.uint64 if a.dtype == np.float64 else np.uint32)


def check_rounding_cases(orc):
    for dt, op, x, y, q, exp, note in rounding_cases():
        # replicate the case across a ragged array so position does not matter
        n = 37
        xa = np.full(n, x, dt)
        ya = np.full(n, y if y is not None else 0, dt)
        out = orc.apply(op, xa, ya, q)
        want = np.full(n, exp, dt)
        assert np.array_equal(bits(out), bits(want)), (op, dt, note, out[0], exp)


def check_closed_form(orc):
    # fixture: k=10 in binary64
    with open(os.path.join(GOLDEN, "stream_closed_form_fp64_k10.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    k, a_k, b_k, c_k = (int(v) for v in rows[0])
    a, b, c = si.closed_form_arrays(1000, np.float64)
    orc.stream(a, b, c, 3.0, k)
    assert (a == a_k).all() and (b == b_k).all() and (c == c_k).all()
    # every k where the closed form is exact
    for dt, kmax in ((np.float64, 13), (np.float32, 6)):
        a, b, c = si.closed_form_arrays(257, dt)
        for k in range(1, kmax + 1):
            orc.stream(a, b, c, 3.0, 1)
            assert (a == 15 ** k).all(), (dt, k)
            assert (b == 3 * 15 ** (k - 1)).all(), (dt, k)
            assert (c == 4 * 15 ** (k - 1)).all(), (dt, k)


def _rel_bound(u, k):
    # after k passes each of a, b, c carries at most 3k roundings of relative size <= u on a
    # positive-only computation: |x - X| <= ((1+u)^(3k) - 1) |X|
    return (1 + u) ** (3 * k) - 1


def check_error_bound(orc):
    for dt, u, ks in ((np.float64, U64, (14, 20, 50, 100)), (np.float32, U32, (7, 12, 20, 30))):
        for k in ks:
            a, b, c = si.closed_form_arrays(3, dt)
            orc.stream(a, b, c, 3.0, k)
            bound = _rel_bound(u, k)
            for got, exact in ((a[0], 15 ** k), (b[0], 3 * 15 ** (k - 1)), (c[0], 4 * 15 ** (k - 1))):
                assert math.isfinite(got)
                err = abs(Fraction(float(got)) - exact) / exact
                assert err <= bound, (dt, k, float(err), float(bound))


def check_numpy_ufuncs(orc):
    for dt in (np.float64, np.float32):
        for n in (1, 7, 1000, 4099):
            x = si.uniform(si.array_seed(7, 0, n), n, dt)
            y = si.uniform(si.array_seed(7, 1, n), n, dt)
            for q in (3.0, 0.1, -2.5):
                qd = dt(q)
                assert np.array_equal(bits(orc.copy(x)), bits(x))
                assert np.array_equal(bits(orc.scale(x, q)), bits(np.multiply(x, qd)))
                assert np.array_equal(bits(orc.add(x, y)), bits(np.add(x, y)))
                want = np.add(x, np.multiply(y, qd))
                assert np.array_equal(bits(orc.triad(x, y, q)), bits(want)), (dt, n, q)


def check_invariant(orc):
    for dt in (np.float64, np.float32):
        a, b, c = si.stream_arrays(5000, dt, base_seed=11)
        a0 = a.copy()
        orc.stream(a, b, c, 3.0, 1)
        assert np.array_equal(c, a0 * dt(4))
        assert np.array_equal(bits(b), bits(np.multiply(a0, dt(3))))
        # and the next pass sees the previous a
        a1 = a.copy()
        orc.stream(a, b, c, 3.0, 1)
        assert np.array_equal(c, a1 * dt(4))


# ----------------------------------------------------------------------------------------
# the pins as tests on the committed oracle
# ----------------------------------------------------------------------------------------

def test_rounding_cases_golden():
    check_rounding_cases(oracle.default())


def test_closed_form_exact():
    check_closed_form(oracle.default())


def test_closed_form_error_bound():
    check_error_bound(oracle.default())


def test_matches_numpy_ufuncs():
    check_numpy_ufuncs(oracle.default())


def test_invariant_c_is_four_a():
    """After one pass, c == 4*a_prev exactly for finite inputs that do not overflow.

    c = RN(a + RN(3a)).  Write RN(3a) = 3a - r.  4a is representable and ulp(4a) = 4 ulp(a);
    |r| <= ulp(3a)/2 <= 2 ulp(a) = ulp(4a)/2, so 4a is a nearest value of a + RN(3a) = 4a - r.
    Equality |r| = 2 ulp(a) needs a/ulp(a) = 2 (mod 4), where 4a has an even significand and
    wins the tie.  Hence c == 4a bit for bit.
    """
    check_invariant(oracle.default())


def test_stream_passes_compose():
    for dt in (np.float64, np.float32):
        a, b, c = si.stream_arrays(999, dt, base_seed=3)
        a2, b2, c2 = a.copy(), b.copy(), c.copy()
        oracle.stream(a, b, c, 3.0, 5)
        for _ in range(5):
            oracle.stream(a2, b2, c2, 3.0, 1)
        assert np.array_equal(bits(a), bits(a2)) and np.array_equal(bits(b), bits(b2))
        assert np.array_equal(bits(c), bits(c2))


def test_fp32_hundred_passes_overflow_to_signed_inf():
    """Reading of the 100-pass binary32 workload: |a| grows as 15^k and passes FLT_MAX near
    k=33, after which inf*3 and inf+inf keep the sign; no NaN can arise."""
    a, b, c = si.stream_arrays(4096, np.float32, base_seed=5)
    a0 = a.copy()
    oracle.stream(a, b, c, 3.0, 100)
    nz = a0 != 0
    assert np.all(np.isinf(a[nz])) and np.all(np.sign(a[nz]) == np.sign(a0[nz]))
    assert np.all(np.isinf(b[nz])) and np.all(np.isinf(c[nz]))
    assert not np.isnan(a).any()


def test_fp64_hundred_passes_uniform_within_bound():
    a, b, c = si.stream_arrays(64, np.float64, base_seed=9)
    a0 = a.copy()
    oracle.stream(a, b, c, 3.0, 100)
    bound = _rel_bound(U64, 100)
    for i in range(64):
        if a0[i] == 0:
            continue
        exact = Fraction(float(a0[i])) * 15 ** 100
        assert abs(Fraction(float(a[i])) - exact) <= bound * abs(exact)


def test_aliasing_out_equals_input():
    x = si.uniform(1, 1001, np.float64)
    y = si.uniform(2, 1001, np.float64)
    want = oracle.triad(x, y, 3.0)
    xx = x.copy()
    oracle.triad(xx, y, 3.0, out=xx)
    assert np.array_equal(bits(xx), bits(want))


def test_to_upper_listing3_example():
    s = np.frombuffer(b"helloworld", np.uint8).copy()
    assert oracle.to_upper(s).tobytes() == b"HELLOWORLD"
    r = np.frombuffer(bytes(range(256)) * 3, np.uint8).copy()
    assert oracle.to_upper(r).tobytes() == r.tobytes().upper()  # bytes.upper is ASCII-only


def test_splitmix64_published_outputs():
    # First outputs of SplitMix64 from state 0, as published with the generator.
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
            0xF88BB8A8724C81EC, 0x1B39896A51A8749B]
    assert [si.word_scalar(0, i) for i in range(5)] == want
    assert [int(v) for v in si.words(0, 5)] == want


def test_uniform_inputs_are_exact_grid_values():
    x = si.uniform(12345, 100000, np.float64)
    assert x.min() >= -1.0 and x.max() < 1.0
    assert np.all(np.ldexp(x, 52) == np.rint(np.ldexp(x, 52)))
    w = si.words(12345, 100000)
    assert np.array_equal(x, (w >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0)
    x32 = si.uniform(12345, 100000, np.float32)
    assert np.array_equal(x32.astype(np.float64),
                          (w >> np.uint64(40)).astype(np.float64) * 2.0 ** -23 - 1.0)
    idx = np.array([0, 5, 99999, 77], np.uint64)
    assert np.array_equal(si.uniform_at(12345, idx, np.float64), x[idx.astype(np.int64)])


# ----------------------------------------------------------------------------------------
# planted mistakes: each broken oracle must fail at least one pin
# ----------------------------------------------------------------------------------------

_MUTANTS = {
    # fused multiply-add in Triad (what contraction would do)
    "fma_triad": (None, ["-O2", "-std=c11", "-ffp-contract=fast", "-mfma", "-fPIC", "-shared"]),
    # operands of Triad transposed: c + b*q
    "triad_transposed": (("a[i] = b[i] + t;", "a[i] = c[i] + b[i] * q;"), None),
    # sign error in Add
    "add_sign": (("c[i] = a[i] + b[i];\n}", "c[i] = a[i] - b[i];\n}"), None),
    # Scale and Add swapped in the pass
    "pass_order": (("oracle_scale_f64(c, b, n, q);\n        oracle_add_f64(a, b, c, n);",
                    "oracle_add_f64(a, b, c, n);\n        oracle_scale_f64(c, b, n, q);"), None),
    # binary32 Scale computed in binary64 and rounded once (a precision slip)
    "f32_wide_scale": (("b[i] = c[i] * qf;", "b[i] = (float)((double)c[i] * q);"), None),
    # dropped product term in binary32 Triad
    "f32_triad_dropped": (("float t = c[i] * qf;", "float t = c[i];"), None),
}

_CHECKS = [check_rounding_cases, check_closed_form, check_error_bound, check_numpy_ufuncs,
           check_invariant]


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_mistakes_are_caught(name, tmp_path):
    subst, cflags = _MUTANTS[name]
    src = open(oracle.SOURCE).read()
    if subst is not None:
        assert subst[0] in src, f"mutation anchor for {name} not found"
        src = src.replace(subst[0], subst[1], 1)
    p = tmp_path / "mutant.c"
    p.write_text(src)
    lib = oracle.compile_library(str(p), str(tmp_path / f"libmutant_{name}.so"), cflags)
    orc = oracle.Oracle(lib)
    failed = 0
    for check in _CHECKS:
        try:
            check(orc)
        except AssertionError:
            failed += 1
    assert failed > 0, f"planted mistake {name} passed every pin"
