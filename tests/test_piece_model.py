"""The constants of the dense chain's FP16 operand pieces, pinned on the CPU with a model.

The FP16-piece chain (NN_MIXED_F16) cuts each value, times an exact power-of-two scale, into
FP16 pieces (round to nearest even; each remainder exact in FP32) and uses, for a level's
rounding floor, the BF16 constants times 2^-3 per piece: one piece leaves an rms relative error
of about 2^-11.8, as one BF16 piece leaves about 2^-8.8 (a rounding error uniform over half an
ulp has rms u / sqrt(3), and the ulp of a normal FP16 number is 2^-3 of BF16's). The scales put
a row's largest entry in [2^13, 2^14), so every piece the chain can use stays finite and the
pieces of entries within 2^18 of the row's largest are normal numbers. One-piece R and T are
written at 8 significant bits, which must be exactly the BF16 value. These are properties of
the formats and of the piece arithmetic; the model below is test code, not the oracle.
"""
import numpy as np

import synth


def _bf16(x):
    """Round float32 values to BF16 (nearest, ties to even), returned as float32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def _f16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def _row_scales(a):
    """2^e per row with the row's largest |entry| times 2^e in [2^13, 2^14)."""
    m = np.max(np.abs(a), axis=1)
    _, ex = np.frexp(m)
    return np.ldexp(1.0, 14 - ex)


def _pieces_f16(x, p):
    out, rem = [], np.asarray(x, dtype=np.float32)
    for _ in range(p):
        h = _f16(rem)
        out.append(h)
        rem = (rem - h).astype(np.float32)
    return out


def test_row_scale_puts_row_maxima_in_range():
    r = synth.rng(3)
    a = r.standard_normal((64, 200)) * np.exp(r.uniform(-30, 30, size=(64, 1)))
    s = _row_scales(a)
    top = np.max(np.abs(a), axis=1) * s
    assert np.all(top >= 2.0 ** 13) and np.all(top < 2.0 ** 14)
    assert np.all(s == np.exp2(np.round(np.log2(s))))  # powers of two: exact scaling


def test_one_fp16_piece_rms_error_matches_the_floor_constant():
    # A level-1 residual rounds both operands once: R's error dA X + A dX is the sum of two
    # independent terms, each the per-element relative rounding of one operand carried through
    # the product, so its floor is sqrt(2) times that rms in units of c. Pinned: sqrt(2) times
    # the modelled rms of one FP16 rounding is the constant 0x1.27p-12 (2^-11.8; measured on the
    # GPU: 2.77-2.84e-4 c), and BF16's 0x1.27p-9 by the same measure, 2^3 apart.
    r = synth.rng(5)
    x = (r.uniform(1.0, 2.0, size=400000) * np.exp2(r.integers(-8, 8, size=400000))).astype(np.float32)
    rel16 = np.sqrt(2.0 * np.mean(((x - _f16(x)) / x) ** 2))
    rel_bf = np.sqrt(2.0 * np.mean(((x - _bf16(x)) / x) ** 2))
    assert abs(np.log2(rel16) - np.log2(float.fromhex("0x1.27p-12"))) < 0.05, np.log2(rel16)
    assert abs(np.log2(rel_bf) - np.log2(float.fromhex("0x1.27p-9"))) < 0.05, np.log2(rel_bf)
    assert abs(np.log2(rel_bf / rel16) - 3.0) < 0.05


def test_two_piece_floor_constants():
    # Two pieces per operand, products A0 X0 + A0 X1 + A1 X0: the error is A1 X1 (the product of
    # the two one-piece roundings) plus each operand's two-piece remainder carried through the
    # product, three independent terms: sqrt(2 r2^2 + r1^4) in units of c, with r1, r2 the rms
    # relative remainders after one and two pieces. Pinned against the constants the schedule
    # uses: 0x1.15p-18 for BF16 (2^-17.9, measured on the GPU) and 0x1.15p-24 for FP16.
    # (values in [1, 2^14): the range the scales give the operands, where the second FP16 piece
    # is a normal number)
    r = synth.rng(13)
    x = (r.uniform(1.0, 2.0, size=400000) * np.exp2(r.integers(0, 14, size=400000))).astype(np.float32)
    for rnd, const in ((_bf16, "0x1.15p-18"), (_f16, "0x1.15p-24")):
        p0 = rnd(x)
        rem1 = (x - p0).astype(np.float32)
        p1 = rnd(rem1)
        rem2 = (rem1 - p1).astype(np.float32)
        r1 = np.sqrt(np.mean((rem1 / x) ** 2))
        r2 = np.sqrt(np.mean((rem2 / x) ** 2))
        model = np.sqrt(2.0 * r2 ** 2 + r1 ** 4)
        # within 0.2 in log2: an FP32 value's two FP16 pieces leave only its last two bits, so
        # the model's FP16 remainder sits a little above the BF16 constant times 2^-6 (2^-23.7
        # against 2^-23.9); at level 2 the accumulation floor dominates that term anyway
        assert abs(np.log2(model) - np.log2(float.fromhex(const))) < 0.2, (const, np.log2(model))


def test_scaled_pieces_are_finite_and_exact_to_their_width():
    # a matrix with rows over 2^80 of range: after the row scales no piece overflows, two
    # pieces hold each FP32 value to 2^-22 of its row's largest entry, three to 2^-33
    r = synth.rng(7)
    a = (r.standard_normal((48, 256)) * np.exp(r.uniform(-28, 28, size=(48, 1)))).astype(np.float32)
    xs = (a * _row_scales(a)[:, None]).astype(np.float32)
    rowmax = np.max(np.abs(xs), axis=1, keepdims=True)
    for p, bound in ((1, 2.0 ** -11), (2, 2.0 ** -22), (3, 2.0 ** -33)):
        ps = _pieces_f16(xs, p)
        assert all(np.all(np.isfinite(q)) for q in ps)
        err = np.abs(xs.astype(np.float64) - sum(q.astype(np.float64) for q in ps))
        assert np.all(err <= bound * rowmax * 1.0001), (p, float(np.max(err / rowmax)))


def test_eight_bit_fp16_piece_is_the_bf16_value():
    # R and T pieces at 8 significant bits: FP16 after BF16 rounding keeps the BF16 value exactly
    # over FP16's normal range up to the largest scaled entry (2^12 times an entry of R or T);
    # BF16 rounds 65408 and above to 2^16, past FP16's largest finite 65504, so the 8-bit pieces
    # overflow from |entry| = 65408 / 2^12 = 15.97
    r = synth.rng(11)
    x = (r.choice([-1.0, 1.0], size=200000) * r.uniform(1.0, 2.0, size=200000)
         * np.exp2(r.integers(-14, 15, size=200000))).astype(np.float32)
    x = np.concatenate([x, np.float32([65407.0, -65407.0, 65280.0])])
    b = _bf16(x)
    h = _f16(b)
    assert np.array_equal(h, b)
    with np.errstate(over="ignore"):
        assert np.all(np.isinf(_f16(_bf16(np.float32([65408.0, 65500.0])))))
