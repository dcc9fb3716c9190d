"""Oracle pins: section arithmetic, project tanh, chain gradient (CPU only).

Expected values are worked out by hand from the definitions (stated beside each
case), chosen so that a dropped term, a swapped operand, a wrong shift, a fused
multiply-add or another summation order changes the answer.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from synth.workloads import Section, F32, F64, I32, BF16

fs = frozenset


def run(sec, dtypes, cols, perm=None):
    arrs = [np.ascontiguousarray(np.asarray(c, dtype=oracle.core.NP[d])) for c, d in zip(cols, dtypes)]
    oracle.section(sec, dtypes, arrs, perm)
    return arrs


def f32(x):
    return np.float32(x)


def test_madd3_is_not_fused():
    e = 2.0 ** -12
    x = f32(1 + e)
    # x*x = 1 + 2^-11 + 2^-24 rounds (tie to even) to 1 + 2^-11; adding -(1 + 2^-11) gives 0.
    # A fused multiply-add would give 2^-24.
    out = run(Section("madd3", (0, 1, 2), fs([0, 1, 2]), fs([2])), [F32] * 3, [[x, 0.5], [x, 0.25], [-(1 + 2 * e), 1.0]])
    assert out[2][0] == 0.0 and out[2][1] == 1.125
    assert out[0][0] == x and out[1][1] == f32(0.25)          # operands untouched


def test_xorshift_logical():
    out = run(Section("xorshift", (0, 1), fs([0]), fs([1])), [I32, I32], [[8, 2 ** 20 - 1, -8], [0, 0, 0]])
    # 8 ^ 1 = 9; 0xFFFFF ^ 0x1FFFF = 0xE0000; -8 = 0xFFFFFFF8, >>3 logical = 0x1FFFFFFF -> 0xE0000007
    assert out[1].tolist() == [9, 0xE0000, np.int32(np.uint32(0xE0000007).view(np.int32))]


def test_add_operand_order():
    out = run(Section("add", (0, 3, 0), fs(range(4)), fs([0])), [F32] * 4, [[1.5], [7.0], [9.0], [0.25]])
    assert out[0][0] == 1.75 and out[1][0] == 7.0 and out[2][0] == 9.0


def test_mix_sum_is_ascending_field_order():
    # s = ((0 + 1) + 1e8) + (-1e8) = 0 in fp32 (1e8 + 1 rounds to 1e8); descending order would give 1.
    sec = Section("mix", (), fs([0, 1, 2]), fs([0]))
    out = run(sec, [F32] * 3, [[1.0], [1e8], [-1e8]])
    assert out[0][0] == 0.5                                   # w*0.5 + t with t = 0


def test_mix_fp32_only():
    sec = Section("mix", (), fs([0]), fs([0]))
    out = run(sec, [F32], [[0.5, -3.0]])
    assert out[0].tolist() == [0.75, -4.5]                    # 0.5*w + w


def test_mix_int_only():
    # h = 8, t = 8/256 = 2^-5 whose bits are 0x3D000000; (h ^ bits) >> 3 = 0x07A00001; 8 ^ that = 0x07A00009
    sec = Section("mix", (), fs([0]), fs([0]))
    out = run(sec, [I32], [[8, 0]])
    assert out[0].tolist() == [0x07A00009, 0]


def test_mix_fp64_and_cross_terms():
    # fp64 d = 1.0 (bits 0x3FF0000000000000): h = 0x3FF00000 ^ 0 -> h & 255 = 0, t = s = 0.25 (one fp32 0.25)
    # d' = 1.0*0.5 + 0.25 = 0.75; fp32 w = 0.25*0.5 + 0.25 = 0.375;
    # int32 i = 5: h = 0x3FF00000 ^ 5 = 0x3FF00005, h & 255 = 5 -> t = 0.25 + 5/256 = 0.26953125
    sec = Section("mix", (), fs([0, 1, 2]), fs([0, 1]))
    out = run(sec, [F64, F32, I32], [[1.0], [0.25], [5]])
    t = 0.25 + 5 / 256
    assert out[1][0] == f32(0.25 * 0.5 + t)                  # exact: 0.39453125
    assert out[0][0] == 1.0 * 0.5 + t
    assert out[2][0] == 5                                     # not written


def test_mix_bf16_raw_bits():
    # bf16 bits 0x0100: h = 0x100, h & 255 = 0, t = 0 (bits 0); k = 0x100 >> 3 = 0x20; w = 0x100 ^ 0x20
    sec = Section("mix", (), fs([0]), fs([0]))
    out = run(sec, [BF16], [[0x100]])
    assert out[0][0] == 0x120


def test_drift_wraps_into_unit_box():
    sec = Section("drift", (0, 1, 2, 3, 4, 5), fs(range(6)), fs([0, 1, 2]), params=(2.0 ** -7,))
    # dt*v = 0.5, -0.25, 0: 0.75 -> 1.25 -> 0.25; 0.125 -> -0.125 -> 0.875; 0.5 stays
    out = run(sec, [F32] * 6, [[0.75], [0.125], [0.5], [64.0], [-32.0], [0.0]])
    assert [o[0] for o in out[:3]] == [0.25, 0.875, 0.5]
    assert [o[0] for o in out[3:]] == [64.0, -32.0, 0.0]


def test_bin_cells_and_clamp():
    sec = Section("bin", (0, 1, 2, 3), fs([0, 1, 2]), fs([3]), params=(128.0,))
    below_one = float(np.nextafter(f32(1.0), f32(0.0)))
    out = run(sec, [F32, F32, F32, I32], [[0.0, 1.0], [0.5, 0.0], [below_one, 0.0], [-1, -1]])
    assert out[3].tolist() == [0 + 128 * (64 + 128 * 127), 127]


def test_kinetic_energy():
    sec = Section("ke", (0, 1, 2, 3, 4), fs([0, 1, 2, 3]), fs([4]))
    out = run(sec, [F32, F32, F32, F32, F64], [[1.0, 3.0], [2.0, 0.0], [2.0, 0.0], [2.0, 0.5], [0.0, 0.0]])
    assert out[4].tolist() == [9.0, 2.25]                    # 0.5*2*(1+4+4); 0.5*0.5*9


def test_flags():
    sec = Section("flags", (0, 1), fs([0, 1]), fs([0]), params=(1.5,))
    out = run(sec, [I32, F64], [[0b1010101, 200, 3], [2.0, 1.0, 1.5]])
    assert out[0].tolist() == [0b10101011, 144, 6]            # 1.5 is not > 1.5


def test_gather_reads_the_permuted_record():
    sec = Section("gather", (0, 1, 2, 3, 4, 5, 6), fs([0, 1, 2]), fs([0, 1, 2]), fs([3, 4, 5, 6]), params=(2.0 ** -7,))
    perm = np.array([1, 0], dtype=np.int32)
    # record 0 reads record 1: charge -1, p = (0.75, 0.25, 0.5) -> dv = -2^-7*(0.25, -0.25, 0)
    cols = [[1.0, 2.0], [1.0, 2.0], [1.0, 2.0], [0.5, 0.75], [0.5, 0.25], [0.5, 0.5], [1.0, -1.0]]
    out = run(sec, [F32] * 7, cols, perm)
    d = 2.0 ** -7
    assert [out[a][0] for a in range(3)] == [1 - 0.25 * d, 1 + 0.25 * d, 1.0]
    assert [out[a][1] for a in range(3)] == [2.0, 2.0, 2.0]   # record 1 reads record 0: p - 0.5 = 0


def test_kick():
    sec = Section("kick", (0, 1, 2, 3), fs(range(4)), fs([0, 1, 2]), params=(2.0 ** -7, 0.125, -0.0625, 0.03125))
    out = run(sec, [F32] * 4, [[0.0], [1.0], [-1.0], [-1.0]])
    d = 2.0 ** -7
    assert [out[a][0] for a in range(3)] == [-d * 0.125, 1 + d * 0.0625, -1 - d * 0.03125]


def test_axpb_mul_tanh():
    ax = Section("axpb", (0, 1), fs([0]), fs([1]), params=(0.5, -2.0))
    out = run(ax, [F32, F32], [[3.0], [99.0]])
    assert out[1][0] == -0.5 and out[0][0] == 3.0
    ip = Section("axpb", (0, 0), fs([0]), fs([0]), params=(2.0, 1.0))
    assert run(ip, [F32], [[3.0]])[0][0] == 7.0
    mu = Section("mul", (0, 1, 2), fs([0, 1]), fs([2]))
    assert run(mu, [F32] * 3, [[3.0], [-0.5], [1.0]])[2][0] == -1.5
    th = Section("tanh", (0, 1), fs([0]), fs([1]))
    assert run(th, [F32] * 2, [[0.0, 20.0], [5.0, 5.0]])[1].tolist() == [0.0, 1.0]


# ------------------------------------------------------------------ tanh

def _ulps(a, b):
    a = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    b = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    a = np.where(a < 0, -(a & 0x7FFFFFFF), a)
    b = np.where(b < 0, -(b & 0x7FFFFFFF), b)
    return np.abs(a - b)


def test_tanh_accuracy_bound():
    xs = np.concatenate([np.linspace(-10, 10, 200001, dtype=np.float32),
                         np.float32(np.logspace(-38, 1, 5000)), -np.float32(np.logspace(-38, 1, 5000))])
    ref = np.tanh(xs.astype(np.float64)).astype(np.float32)
    assert _ulps(oracle.tanhf(xs), ref).max() <= 8


def test_tanh_shape():
    xs = np.linspace(-12, 12, 20001, dtype=np.float32)
    y = oracle.tanhf(xs)
    assert np.array_equal(oracle.tanhf(-xs), -y)             # odd
    assert np.all(np.diff(y) >= -5e-7)                        # monotone up to the 8-ulp error bound
    coarse = oracle.tanhf(np.arange(-4, 4, 0.05, dtype=np.float32))
    assert np.all(np.diff(coarse) > 0)                        # strictly increasing at a coarser step
    assert oracle.tanhf([0.0])[0] == 0 and np.signbit(oracle.tanhf([-0.0])[0])
    assert np.all(np.abs(oracle.tanhf(np.array([9.0, 10.0, 1e30], np.float32))) == 1.0)
    tiny = np.float32(1e-20)
    assert oracle.tanhf([tiny])[0] == tiny                    # tanh x ~ x near 0


def test_tanh_polynomials_are_the_continued_fraction():
    # P_K(a)/Q_K(a) must equal 1 + a/(3 + a/(5 + ... + a/(2K+1))) evaluated exactly, bottom up
    K, p, q = oracle.tanh_coeffs()
    for a in [Fraction(1, 3), Fraction(2), Fraction(81, 4)]:
        d = Fraction(2 * K + 1)
        for k in range(K - 1, -1, -1):
            d = (2 * k + 1) + a / d
        num = sum(Fraction(int(np.float64(c))) * a ** j for j, c in enumerate(p))
        den = sum(Fraction(int(np.float64(c))) * a ** j for j, c in enumerate(q))
        assert abs(float(num / den / d) - 1.0) < 1e-6        # coefficients rounded to fp32 once
    # constant terms: P_K(0) = Q_K(0) = 3*5*...*(2K+1)
    df = 1
    for k in range(1, K + 1):
        df *= 2 * k + 1
    assert p[0] == np.float32(df) and q[0] == np.float32(df)


# ------------------------------------------------------------ chain gradient

def _fwd64(sections, fields64):
    v = [a.copy() for a in fields64]
    for s in sections:
        if s.op == "axpb":
            v[s.args[1]] = s.params[0] * v[s.args[0]] + s.params[1]
        elif s.op == "mul":
            v[s.args[2]] = v[s.args[0]] * v[s.args[1]]
        else:
            v[s.args[1]] = np.tanh(v[s.args[0]])
    return v


def test_chain_grad_single_sections():
    c = [0.5, -2.0, 0.25]
    secs = [Section("axpb", (0, 2), fs([0]), fs([2]), params=(3.0, 1.0))]
    st = [np.array([1.0], np.float32), np.array([2.0], np.float32), np.array([4.0], np.float32)]
    g = oracle.chain_grad(secs, st, c)
    assert [x[0] for x in g] == [0.5 + 3.0 * 0.25, -2.0, 0.0] and st[2][0] == 4.0 * 0 + 4.0
    secs = [Section("mul", (0, 1, 2), fs([0, 1]), fs([2]))]
    st = [np.array([3.0], np.float32), np.array([-2.0], np.float32), np.array([9.0], np.float32)]
    g = oracle.chain_grad(secs, st, c)
    assert [x[0] for x in g] == [0.5 + 0.25 * -2.0, -2.0 + 0.25 * 3.0, 0.0] and st[2][0] == -6.0
    secs = [Section("mul", (0, 0, 0), fs([0]), fs([0]))]         # x <- x*x: dL/dx = 2*x*c
    st = [np.array([3.0], np.float32), np.array([0.0], np.float32), np.array([0.0], np.float32)]
    g = oracle.chain_grad(secs, st, c)
    assert g[0][0] == 3.0 and st[0][0] == 9.0


def test_chain_grad_matches_central_differences():
    import synth
    wl = synth.config5(n=1 << 12, n_sections=64)
    x0 = [wl.values(f) for f in range(wl.F)]
    st = [a.copy() for a in x0]
    g = oracle.chain_grad(wl.sections, st, wl.loss_weights)
    c = np.array(wl.loss_weights, np.float64)
    base = [a.astype(np.float64) for a in x0]
    h = 1e-4
    checked = 0
    for f in range(wl.F):
        up = [a.copy() for a in base]
        dn = [a.copy() for a in base]
        up[f] += h
        dn[f] -= h
        Lu = sum(c[k] * v for k, v in enumerate(_fwd64(wl.sections, up)))
        Ld = sum(c[k] * v for k, v in enumerate(_fwd64(wl.sections, dn)))
        fd = (Lu - Ld) / (2 * h)
        an = g[f].astype(np.float64)
        scale = np.maximum(1.0, np.abs(fd))
        err = np.abs(fd - an) / scale
        # every record, no quantile: the ops are smooth (no kinks), the fp32 gradient's rounding over
        # at most 64 sections is a few 1e-6 relative at worst, the central difference's truncation
        # (h^2 |f'''| / 6 with h = 1e-4) far below that; a dropped term or a wrong sign is O(1)
        assert err.max() < 1e-5, (f, float(err.max()))
        checked += 1
    assert checked == wl.F
    # the fp32 forward state also agrees with the fp64 forward to fp32 accuracy
    fwd = _fwd64(wl.sections, base)
    for f in range(wl.F):
        assert np.allclose(st[f], fwd[f], rtol=1e-3, atol=1e-4)
