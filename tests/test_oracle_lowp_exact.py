"""Exact-arithmetic pins of the oracle's low-precision semantics.

The low-precision stencil oracle (fp32 / bf16 storage) and the fp32-inner
refinement CG (FP32-IR) are extensions of the paper's stencil (Eq.
iterativeStencil, Sec. 2.2.1) and CG (Sec. 2.2.2) with a precision rule the
paper does not print; the rule they follow is the library's stated reading:

  * stencil, fp32 / bf16 storage: each output cell is an fp32 fused
    multiply-add chain acc = fma(w_o, x(c+o), acc) over the offset table in
    table order from acc = 0, with w_o the fp32 value of the weight; the
    result is rounded (nearest, ties to even) to the storage type after every
    step;
  * FP32-IR: the correction d of every outer step comes out of an fp32 CG
    (fp32 vectors and axpys), and x += d is done in fp64.

The expected values here come from exact rational arithmetic
(``fractions.Fraction``) rounded by that rule, written out in this file, not
from the oracle; each case is chosen so that the plausible alternatives -- an
fp64 (or exact) accumulation, the reversed order, separate multiply and add,
truncation instead of round-to-nearest-even, no rounding between steps, an
fp64 inner solve -- give a different answer, and the test asserts that too, so
a mistake of any of those kinds in the oracle fails here.
"""
from __future__ import annotations

from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs


@pytest.fixture(scope="module")
def oracle():
    from oracle import oracle as o
    return o


# ----------------------------------------------------------- exact rounding

def round_bits(v: Fr, bits: int) -> Fr:
    """v rounded to the nearest binary floating-point number with a `bits`-bit
    significand (24: fp32, 53: fp64, 8: bf16), ties to even; normal range
    only (the cases below stay far from underflow and overflow)."""
    if v == 0:
        return Fr(0)
    sign = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    if Fr(2) ** (e + 1) <= a:
        e += 1
    scale = Fr(2) ** (bits - 1 - e)
    return sign * Fr(round(a * scale)) / scale   # round() on a Fraction: half to even


def truncate_bits(v: Fr, bits: int) -> Fr:
    """Round toward zero to a `bits`-bit significand (an alternative rule)."""
    if v == 0:
        return Fr(0)
    sign = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fr(2) ** e > a:
        e -= 1
    if Fr(2) ** (e + 1) <= a:
        e += 1
    scale = Fr(2) ** (bits - 1 - e)
    return sign * Fr(int(a * scale)) / scale


def f32(v: Fr) -> Fr:
    return round_bits(v, 24)


# ------------------------------------------------------ rule and its rivals

def fma_chain(ws, xs):
    acc = Fr(0)
    for w, x in zip(ws, xs):
        acc = f32(w * x + acc)
    return acc


def exact_sum_then_f32(ws, xs):
    return f32(sum(w * x for w, x in zip(ws, xs)))


def exact_sum(ws, xs):
    return sum(w * x for w, x in zip(ws, xs))


def reversed_chain(ws, xs):
    return fma_chain(ws[::-1], xs[::-1])


def unfused_chain(ws, xs):
    acc = Fr(0)
    for w, x in zip(ws, xs):
        acc = f32(acc + f32(w * x))
    return acc


def run_rule(field, offs, w, steps, cell_sum, store):
    """Jacobi steps on a 2-D (ny, nx) interior with Dirichlet 0, every cell's
    terms in table order, in exact arithmetic with the given rounding of the
    sum (`cell_sum`) and of the stored value (`store`)."""
    ny, nx = field.shape
    wf = [f32(Fr(float(v))) for v in w]
    cur = [[Fr(float(field[j, i])) for i in range(nx)] for j in range(ny)]
    for _ in range(steps):
        nxt = [[Fr(0)] * nx for _ in range(ny)]
        for j in range(ny):
            for i in range(nx):
                xs = []
                for dx, dy, _dz in offs:
                    jj, ii = j + dy, i + dx
                    xs.append(cur[jj][ii] if 0 <= jj < ny and 0 <= ii < nx else Fr(0))
                nxt[j][i] = store(cell_sum(wf, xs))
        cur = nxt
    return np.array([[float(v) for v in row] for row in cur], dtype=np.float64)


def _ident(v):
    return v


def _bf16(v):
    return round_bits(v, 8)


# -------------------------------------------------------------- fp32 storage

def test_lowp_fp32_is_fma_chain_in_table_order(oracle):
    """fp32 storage: a seeded 6 x 7 field, a 2d5pt table with seeded weights,
    two steps.  The oracle must equal the fp32 FMA chain in table order bit
    for bit; the exact sum rounded once, the reversed order and the unfused
    chain each differ from it in at least one cell."""
    ny, nx = 6, 7
    f = inputs.uniform(inputs.substream(91, 1), ny * nx).reshape(ny, nx).astype(np.float32)
    offs = inputs.shape_offsets("2d5pt")
    w = 0.05 + 0.35 * inputs.uniform(inputs.substream(91, 2), len(offs))
    got = oracle.stencil_run_lowp(f, offs, w, 2, "f32").astype(np.float64)
    want = run_rule(f, offs, w, 2, fma_chain, _ident)
    assert np.array_equal(got, want)
    for rival in (exact_sum_then_f32, reversed_chain, unfused_chain):
        other = run_rule(f, offs, w, 2, rival, _ident)
        assert not np.array_equal(other, want), f"{rival.__name__} does not discriminate"


# -------------------------------------------------------------- bf16 storage

# One-dimensional three-point cases (centre, -x, +x) on a 3 x 1 grid whose
# middle cell sees all three terms; each was found by a search for a sum close
# to a bf16 rounding midpoint, so that one rival rounds to the other side.
# (weights as doubles, field [x(-1), x(0), x(+1)] of bf16 values, rival)
_BF16_CASES = [
    ([0.16508769750620705, 0.26564267230832367, 0.15132764136439425],
     [0.76171875, 0.107421875, 0.6171875], exact_sum),
    ([0.21207992865004976, 0.12826438238856977, 0.18209049653276327],
     [0.76171875, 0.9453125, 0.73828125], reversed_chain),
    ([0.48726845849355926, 0.346530619036001, 0.313188036766178],
     [0.451171875, 0.78125, 0.125], unfused_chain),
]


@pytest.mark.parametrize("case", range(len(_BF16_CASES)))
def test_lowp_bf16_fp32_chain_then_round(oracle, case):
    w, field, rival = _BF16_CASES[case]
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0)]
    f = np.array([field], dtype=np.float32)
    assert np.array_equal(oracle.bf16_round(f), f)       # the inputs are bf16 values
    got = oracle.stencil_run_lowp(f, offs, w, 1, "bf16").astype(np.float64)
    want = run_rule(f, offs, w, 1, fma_chain, _bf16)
    assert np.array_equal(got, want)
    other = run_rule(f, offs, w, 1, rival, _bf16)
    assert other[0, 1] != want[0, 1], f"{rival.__name__} does not discriminate"


def test_lowp_bf16_rounds_every_step_to_nearest_even(oracle):
    """bf16 storage, a seeded 6 x 6 field, 2d5pt, three steps: equal to the
    rule bit for bit; truncation instead of round-to-nearest-even, and
    carrying fp32 values between steps (rounding only the final field), both
    differ from it."""
    ny, nx = 6, 6
    f = oracle.bf16_round(inputs.uniform(inputs.substream(92, 1), ny * nx).reshape(ny, nx).astype(np.float32))
    offs = inputs.shape_offsets("2d5pt")
    w = 0.05 + 0.35 * inputs.uniform(inputs.substream(92, 2), len(offs))
    got = oracle.stencil_run_lowp(f, offs, w, 3, "bf16").astype(np.float64)
    want = run_rule(f, offs, w, 3, fma_chain, _bf16)
    assert np.array_equal(got, want)
    trunc = run_rule(f, offs, w, 3, fma_chain, lambda v: truncate_bits(v, 8))
    assert not np.array_equal(trunc, want)
    carried = run_rule(f, offs, w, 3, fma_chain, _ident)
    carried = np.vectorize(lambda v: float(round_bits(Fr(v), 8)))(carried)
    assert not np.array_equal(carried, want)


# ------------------------------------------------------------------- FP32-IR

def _diag_csr(d):
    n = len(d)
    return (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32),
            np.asarray(d, dtype=np.float64))


def test_fp32_ir_first_correction_is_the_fp32_solution(oracle):
    """A = [3], b = [1]: the inner fp32 CG takes one step, alpha = fl32(1/3),
    so after one outer step x is the fp32 number nearest 1/3 (an fp64 inner
    solve would give the fp64 one).  The residual 1 - 3 fl32(1/3) = -2^-25 is
    above 1e-12, and the second correction, fl32(1/3) * (-2^-25), leaves a
    residual of exactly 2^-50: the solve to 1e-12 takes exactly two outer
    steps."""
    rp, c, v = _diag_csr([3.0])
    b = np.array([1.0])
    one = oracle.cg_fp32_ir(rp, c, v, b, rtol=1e-14, inner_rtol=1e-6, max_outer=1)
    third32 = float(np.float32(1.0) / np.float32(3.0))    # IEEE division: nearest fp32 to 1/3
    assert one["x"][0] == third32
    assert one["x"][0] != 1.0 / 3.0
    assert one["true_rel"] == 2.0 ** -25
    two = oracle.cg_fp32_ir(rp, c, v, b, rtol=1e-12, inner_rtol=1e-6)
    assert two["status"] == 0 and two["outer_iters"] == 2
    assert two["x"][0] == third32 * (1.0 - 2.0 ** -25)
    assert two["true_rel"] == 2.0 ** -50


def test_fp32_ir_corrections_are_fp32_vectors(oracle):
    """A diagonal system with three distinct eigenvalues: whatever the inner
    CG's stopping point, one outer step from x0 = 0 leaves x equal to the fp32
    correction vector (every component an fp32 number), and the fp64 solution
    1/a_i is not reached to fp64 accuracy."""
    rp, c, v = _diag_csr([1.0, 3.0, 7.0])
    b = np.array([1.0, 1.0, 1.0])
    res = oracle.cg_fp32_ir(rp, c, v, b, rtol=1e-15, inner_rtol=1e-12, max_inner=50, max_outer=1)
    assert res["outer_iters"] == 1
    x = res["x"]
    assert np.array_equal(x.astype(np.float32).astype(np.float64), x)
    assert np.max(np.abs(x * v - b)) > 1e-12
    assert np.max(np.abs(x * v - b)) < 1e-5
