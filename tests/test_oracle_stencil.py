"""Pins of the stencil oracle (Eq. iterativeStencil, Sec. 2.2.1) against
closed forms, invariants and independent formulations -- never against itself.

* sine eigenmodes of the Dirichlet problem decay by their closed-form factor;
* a constant field with a matching Dirichlet value is preserved (weights sum to 1);
* a Dirac delta spreads into the coefficients of the N-th power of the
  stencil's generating polynomial (computed by FFT, asymmetric weights, so a
  flipped offset or swapped axis fails);
* on 8x8 and 4x4x4 grids the result equals M^N x0 with M assembled from
  Kronecker products of shift matrices (a linear-algebra formulation);
* linearity and run(a) then run(b) == run(a+b).
"""
import numpy as np
import pytest

from paper_2204_02064_gb300 import inputs


def _field(shape, seed=11):
    return inputs.stencil_field(shape, seed)


# ---------------------------------------------------------------- eigenmodes

@pytest.mark.parametrize("L,p,q,steps", [(16, 1, 1, 37), (24, 3, 5, 20), (9, 8, 2, 11)])
def test_2d5pt_sine_mode_decay(oracle, L, p, q, steps):
    C, w = 0.2, 0.2
    i = np.arange(1, L + 1)
    a, b = p * np.pi / (L + 1), q * np.pi / (L + 1)
    u = np.outer(np.sin(b * i), np.sin(a * i))        # [y, x]
    lam = C + 2 * w * (np.cos(a) + np.cos(b))
    offs = inputs.shape_offsets("2d5pt")
    out = oracle.stencil_run(u, offs, [C] + [w] * 4, steps)
    ref = lam ** steps * u
    # relative to the decayed amplitude, floored at 1 % of the initial one:
    # rounding noise lives in other modes and does not decay with this one
    assert np.max(np.abs(out - ref)) <= 1e-13 * max(np.max(np.abs(ref)), 1e-2 * np.max(np.abs(u)))


def test_3d7pt_sine_mode_decay(oracle):
    L, steps = 10, 25
    C, w = 0.4, 0.1
    i = np.arange(1, L + 1)
    ks = (1, 2, 3)
    ang = [k * np.pi / (L + 1) for k in ks]
    u = (np.sin(ang[2] * i)[:, None, None] * np.sin(ang[1] * i)[None, :, None]
         * np.sin(ang[0] * i)[None, None, :])
    lam = C + 2 * w * sum(np.cos(t) for t in ang)
    out = oracle.stencil_run(u, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"),
                             steps)
    ref = lam ** steps * u
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_2d9pt_box_sine_mode_decay(oracle):
    L, steps, p, q = 12, 15, 2, 3
    i = np.arange(1, L + 1)
    a, b = p * np.pi / (L + 1), q * np.pi / (L + 1)
    u = np.outer(np.sin(b * i), np.sin(a * i))
    lam = (1 + 2 * np.cos(a)) * (1 + 2 * np.cos(b)) / 9.0
    out = oracle.stencil_run(u, inputs.shape_offsets("2d9pt"), inputs.workload_weights("2d9pt"),
                             steps)
    ref = lam ** steps * u
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_3d27pt_box_sine_mode_decay(oracle):
    L, steps = 7, 6
    i = np.arange(1, L + 1)
    ang = [k * np.pi / (L + 1) for k in (1, 2, 1)]
    u = (np.sin(ang[2] * i)[:, None, None] * np.sin(ang[1] * i)[None, :, None]
         * np.sin(ang[0] * i)[None, None, :])
    lam = np.prod([1 + 2 * np.cos(t) for t in ang]) / 27.0
    out = oracle.stencil_run(u, inputs.shape_offsets("3d27pt"),
                             inputs.workload_weights("3d27pt"), steps)
    ref = lam ** steps * u
    assert np.max(np.abs(out - ref)) <= 1e-13 * np.max(np.abs(ref))


# ---------------------------------------------------------- constant field

@pytest.mark.parametrize("name", list(inputs.SHAPES))
def test_constant_field_preserved(oracle, name):
    kind, ndim, r = inputs.SHAPES[name]
    shape = (7, 6, 5)[3 - ndim:] if ndim == 3 else (9, 11)
    c, steps = 0.7310585786300049, 30
    f = np.full(shape, c)
    w = inputs.workload_weights(name, seed=5)
    out = oracle.stencil_run(f, inputs.shape_offsets(name), w, steps, boundary=c)
    assert np.max(np.abs(out - c)) <= 4 * steps * len(w) * np.finfo(float).eps * c


def test_constant_field_with_wrong_boundary_is_not_preserved(oracle):
    # The invariant needs the Dirichlet value to equal the constant: the
    # cells next to the wall must feel a zero boundary.
    f = np.ones((8, 8))
    out = oracle.stencil_run(f, inputs.shape_offsets("2d5pt"), [0.2] * 5, 1, boundary=0.0)
    assert out[0, 0] == pytest.approx(0.6) and out[4, 4] == pytest.approx(1.0)


# ------------------------------------------------------- Dirac delta by FFT

def _fft_power(offs, w, ndim, n_steps, size):
    """Response to a centred delta after n_steps, as coefficients of
    (sum_o w_o X^{-o})^n_steps on a periodic box large enough to avoid wrap."""
    k = np.zeros((size,) * ndim)
    for (dx, dy, dz), wo in zip(offs, w):
        idx = (-dx, -dy, -dz)[:ndim][::-1]     # array axes are (z, y, x)
        k[tuple(i % size for i in idx)] += wo
    spec = np.fft.fftn(k) ** n_steps
    resp = np.real(np.fft.ifftn(spec))
    return np.fft.fftshift(resp)


@pytest.mark.parametrize("name,L,steps", [("2d5pt", 41, 12), ("2d25pt", 45, 9),
                                           ("2ds9pt", 45, 9), ("3d7pt", 21, 6),
                                           ("2d9pt", 31, 10)])
def test_delta_spreads_as_polynomial_power(oracle, name, L, steps):
    kind, ndim, r = inputs.SHAPES[name]
    offs = inputs.shape_offsets(name)
    # asymmetric positive weights: every offset distinguishable
    w = 0.5 + inputs.uniform(99, len(offs))
    w /= w.sum()
    shape = (L,) * ndim
    f = np.zeros(shape)
    f[(L // 2,) * ndim] = 1.0
    assert steps * r < L // 2          # the spread never touches the wall
    out = oracle.stencil_run(f, offs, w, steps)
    ref = _fft_power(offs, w, ndim, steps, L)
    assert np.max(np.abs(out - ref)) <= 1e-14


# ------------------------------------------------- Kronecker brute force

def _shift(L, k):
    return np.eye(L, k=k)


def test_2d_brute_force_8x8_kronecker(oracle):
    L, steps = 8, 9
    offs = inputs.shape_offsets("2d5pt")       # C, -x, +x, -y, +y
    w = np.array([0.31, 0.07, 0.23, 0.11, 0.28])
    I = np.eye(L)
    # state vector index = y*L + x; kron(A_y, A_x)
    M = (w[0] * np.kron(I, I) + w[1] * np.kron(I, _shift(L, -1)) + w[2] * np.kron(I, _shift(L, 1))
         + w[3] * np.kron(_shift(L, -1), I) + w[4] * np.kron(_shift(L, 1), I))
    x0 = _field((L, L))
    ref = (np.linalg.matrix_power(M, steps) @ x0.reshape(-1)).reshape(L, L)
    out = oracle.stencil_run(x0, offs, w, steps)
    assert np.max(np.abs(out - ref)) <= 1e-14


def test_3d_brute_force_4x4x4_kronecker_nonzero_boundary(oracle):
    L, steps, bval = 4, 5, 0.37
    offs = inputs.shape_offsets("3d7pt")       # C, -x, +x, -y, +y, -z, +z
    w = np.array([0.2, 0.05, 0.15, 0.09, 0.16, 0.13, 0.22])
    I = np.eye(L)
    K = lambda az, ay, ax: np.kron(az, np.kron(ay, ax))
    M = (w[0] * K(I, I, I) + w[1] * K(I, I, _shift(L, -1)) + w[2] * K(I, I, _shift(L, 1))
         + w[3] * K(I, _shift(L, -1), I) + w[4] * K(I, _shift(L, 1), I)
         + w[5] * K(_shift(L, -1), I, I) + w[6] * K(_shift(L, 1), I, I))
    # boundary source: every missing neighbour contributes w * bval
    ones = np.ones(L ** 3)
    src = bval * (w.sum() * ones - M @ ones)
    x = _field((L, L, L)).reshape(-1)
    for _ in range(steps):
        x = M @ x + src
    out = oracle.stencil_run(_field((L, L, L)), offs, w, steps, boundary=bval)
    assert np.max(np.abs(out.reshape(-1) - x)) <= 1e-14


# --------------------------------------------------------- linear structure

def test_linearity_and_composition(oracle):
    offs = inputs.shape_offsets("2d25pt")
    w = inputs.workload_weights("2d25pt", seed=3)
    f, g = _field((20, 17), 1), _field((20, 17), 2)
    a = 2.5
    lhs = oracle.stencil_run(a * f + g, offs, w, 13)
    rhs = a * oracle.stencil_run(f, offs, w, 13) + oracle.stencil_run(g, offs, w, 13)
    assert np.max(np.abs(lhs - rhs)) <= 1e-13
    two = oracle.stencil_run(oracle.stencil_run(f, offs, w, 5), offs, w, 8)
    one = oracle.stencil_run(f, offs, w, 13)
    assert np.array_equal(one, two)


def test_zero_steps_is_identity(oracle):
    f = _field((5, 6, 7))
    out = oracle.stencil_run(f, inputs.shape_offsets("3d7pt"), inputs.workload_weights("3d7pt"), 0)
    assert np.array_equal(out, f)


def test_rejects_offset_beyond_radius(oracle):
    with pytest.raises(ValueError):
        oracle.stencil_run(np.zeros((4, 4)), [(0, 0, 0), (2, 0, 0)], [0.5, 0.5], 1, radius=1)


# --------------------------------------------- low-precision storage oracle

def test_bf16_rounding_matches_torch(oracle):
    torch = pytest.importorskip("torch")
    x = (inputs.uniform(5, 4000) - 0.5) * np.float64(2.0) ** np.floor(inputs.uniform(6, 4000) * 40 - 20)
    x = x.astype(np.float32)
    # ties: values exactly halfway between two bf16 numbers
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8)], dtype=np.float32)
    x = np.concatenate([x, ties])
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle.bf16_round(x), ref)


def test_lowp_fp32_close_to_fp64(oracle):
    f = _field((17, 19, 23))
    offs = inputs.shape_offsets("3d7pt")
    w = inputs.workload_weights("3d7pt")
    lo = oracle.stencil_run_lowp(f.astype(np.float32), offs, w, 30, "f32")
    hi = oracle.stencil_run(f.astype(np.float32).astype(np.float64), offs, w, 30)
    assert np.max(np.abs(lo - hi)) <= 30 * 8 * np.finfo(np.float32).eps


def test_lowp_bf16_values_are_bf16_and_constant_preserved(oracle):
    c = 0.75                                    # exact in bf16; weights 1/9 sum to 1
    f = np.full((12, 13), c, dtype=np.float32)
    out = oracle.stencil_run_lowp(f, inputs.shape_offsets("2d9pt"), inputs.workload_weights("2d9pt"),
                                  20, "bf16", boundary=c)
    assert np.array_equal(oracle.bf16_round(out), out)
    assert np.max(np.abs(out - c)) <= 2.0 ** -8
    g = oracle.bf16_round(_field((12, 13)).astype(np.float32))
    o2 = oracle.stencil_run_lowp(g, inputs.shape_offsets("2d5pt"), [0.2] * 5, 7, "bf16")
    assert np.array_equal(oracle.bf16_round(o2), o2)
    # bf16 results track the fp64 oracle to a few bf16 ulps per step
    ref = oracle.stencil_run(g.astype(np.float64), inputs.shape_offsets("2d5pt"), [0.2] * 5, 7)
    assert np.max(np.abs(o2 - ref)) <= 7 * 2.0 ** -8


def test_poisson19_sine_mode_eigenvalue(oracle):
    """Table 3's 19-point stencil (centre, faces, edges) with weights that
    depend only on the offset's class: a product of sines vanishing on the
    Dirichlet-0 ghost layer is an eigenvector, with eigenvalue
    w_c + 2 w_f sum_d cos k_d + 4 w_e sum_{d<e} cos k_d cos k_e
    (the +-o pairs of each class combine into cosines)."""
    L = (6, 7, 9)  # z, y, x extents
    kx, ky, kz = (np.pi * 2 / (L[2] + 1), np.pi * 3 / (L[1] + 1), np.pi * 1 / (L[0] + 1))
    ix, iy, iz = (np.arange(1, n + 1) for n in (L[2], L[1], L[0]))
    u = np.sin(kz * iz)[:, None, None] * np.sin(ky * iy)[None, :, None] * np.sin(kx * ix)[None, None, :]
    offs = inputs.shape_offsets("poisson")
    wc, wf, we = 0.28, 0.07, 0.025
    w = [wc if sum(map(abs, o)) == 0 else (wf if sum(map(abs, o)) == 1 else we) for o in offs]
    cx, cy, cz = np.cos(kx), np.cos(ky), np.cos(kz)
    lam = wc + 2 * wf * (cx + cy + cz) + 4 * we * (cx * cy + cx * cz + cy * cz)
    steps = 7
    out = oracle.stencil_run(u, offs, w, steps)
    assert np.max(np.abs(out - lam ** steps * u)) <= 1e-13 * np.max(np.abs(u))


@pytest.mark.parametrize("name,shape,steps", [("3d7pt", (17, 12, 9), 6), ("2d25pt", (31, 26), 5),
                                              ("3d27pt", (9, 10, 11), 3)])
def test_all_cores_build_is_bitwise_the_serial_oracle(oracle, name, shape, steps):
    """The OpenMP build of the oracle (the all-cores CPU baseline) splits a
    step's planes over threads but computes every cell as the serial build
    does, so the two agree bit for bit."""
    from paper_2204_02064_gb300 import inputs
    f = inputs.stencil_field(shape, 47)
    offs, w = inputs.shape_offsets(name), inputs.workload_weights(name, seed=5)
    serial = oracle.stencil_run(f, offs, w, steps)
    parallel, threads = oracle.stencil_run_all_cores(f, offs, w, steps)
    assert threads >= 1
    assert np.array_equal(serial, parallel)
