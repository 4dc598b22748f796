"""Pins of the FP64 oracle to facts other than its own code.

Each test fixes the oracle against the mathematics of Section 2 (the
correlation formula and the loop nest of Fig. 2): a library routine for the
same Hermitian product, closed-form signals, invariants the paper states
(conjugate symmetry of baselines, autocorrelations included, all four
polarisation pairs), exact integers, and finite differences for the
gradients. A dropped term, a wrong sign, a conjugate on the wrong station or
a wrong baseline index fails at least one of them (``test_planted_mistakes``
checks that on mutated copies of the oracle's loop).
"""
import numpy as np
import pytest

import oracle
import synth


def full_matrix(V, S, P):
    """Complete the (B, P, P) triangle to the (S*P, S*P) Hermitian matrix."""
    N = S * P
    F = np.zeros((N, N), dtype=complex)
    for s2 in range(S):
        for s1 in range(s2 + 1):
            b = s2 * (s2 + 1) // 2 + s1
            for p1 in range(P):
                for p2 in range(P):
                    F[s1 * P + p1, s2 * P + p2] = V[b, p1, p2]
                    F[s2 * P + p2, s1 * P + p1] = np.conj(V[b, p1, p2])
    return F


def rows(x):
    """(S, T, P) samples -> (S*P, T) matrix whose row index is s*P + p."""
    S, T, P = x.shape
    return np.transpose(x, (0, 2, 1)).reshape(S * P, T)


# ---------------------------------------------------------------- library pin
@pytest.mark.parametrize("S,T,C", [(1, 1, 1), (2, 3, 2), (3, 7, 1), (5, 16, 3), (8, 33, 2)])
def test_matches_numpy_hermitian_product(S, T, C):
    """Every stored entry equals the (s1,p1),(s2,p2) entry of X X^H computed by
    numpy's matmul, X having rows (station, pol) and columns time."""
    g = synth.rng(99, S * 100 + T)
    x = synth.complex_normal(g, (C, S, T, 2)).astype(np.complex128)
    V = oracle.correlate(x)
    for c in range(C):
        X = rows(x[c])
        ref = X @ X.conj().T
        F = full_matrix(V[c], S, 2)
        np.testing.assert_allclose(F, ref, rtol=1e-12, atol=1e-12)


def test_exact_integers_match_python_ints():
    """Integer samples: the FP64 result is exactly the Python-integer product."""
    g = synth.rng(98)
    x8 = synth.int8_normal(g, (2, 4, 9, 2), sigma=60.0)
    V = oracle.correlate(x8, "ci8")
    for c in range(2):
        re = x8[c, ..., 0].astype(object)
        im = x8[c, ..., 1].astype(object)
        for s2 in range(4):
            for s1 in range(s2 + 1):
                b = s2 * (s2 + 1) // 2 + s1
                for p1 in range(2):
                    for p2 in range(2):
                        ar, ai = re[s1, :, p1], im[s1, :, p1]
                        br, bi = re[s2, :, p2], im[s2, :, p2]
                        sr = int(sum(ar * br + ai * bi))
                        si = int(sum(ai * br - ar * bi))
                        assert V[c, b, p1, p2].real == sr
                        assert V[c, b, p1, p2].imag == si


def test_adversarial_int8_extremes_exact():
    """All-(+-127) samples: results are exact integers up to 2*T*127^2."""
    T = 512
    x8 = np.full((1, 3, T, 2, 2), 127, dtype=np.int8)
    x8[0, 1, :, :, 1] = -127
    V = oracle.correlate(x8, "ci8")
    # station 0 autocorrelation XX: sum_t (127^2 + 127^2)
    assert V[0, 0, 0, 0] == 2 * T * 127 * 127
    # baseline (s1=0, s2=1): a=(127+127i), b=(127-127i): a*conj(b) = (127+127i)^2 = 2*127^2 i
    b01 = 1 * 2 // 2 + 0
    assert V[0, b01, 0, 0] == 2j * T * 127 * 127


# --------------------------------------------------------------- closed forms
def test_constant_signal():
    """x = c everywhere -> V = T |c|^2 on every baseline and pol pair."""
    c0 = 0.3 - 1.7j
    x = np.full((2, 5, 11, 2), c0, dtype=np.complex128)
    V = oracle.correlate(x)
    np.testing.assert_allclose(V, 11 * abs(c0) ** 2, rtol=1e-13)


def test_plane_wave_phases():
    """x_{s,p}(t) = exp(i(phi_{s,p} + w t)) -> V_ab = T exp(i(phi_a - phi_b)).

    The sign of the phase difference fixes which station is conjugated."""
    S, T, P = 6, 40, 2
    g = synth.rng(97)
    phi = g.uniform(-np.pi, np.pi, size=(S, P))
    t = np.arange(T)
    x = np.exp(1j * (phi[:, None, :] + 0.37 * t[None, :, None]))[None]
    V = oracle.correlate(x)[0]
    for s2 in range(S):
        for s1 in range(s2 + 1):
            b = s2 * (s2 + 1) // 2 + s1
            for p1 in range(P):
                for p2 in range(P):
                    want = T * np.exp(1j * (phi[s1, p1] - phi[s2, p2]))
                    assert abs(V[b, p1, p2] - want) < 1e-11


def test_orthogonal_tones():
    """Distinct DFT tones per (station, pol) -> V_ab = T delta_ab."""
    S, P, T = 4, 2, 16
    k = np.arange(S * P).reshape(S, P)
    t = np.arange(T)
    x = np.exp(2j * np.pi * k[:, None, :] * t[None, :, None] / T)[None]
    V = oracle.correlate(x)[0]
    F = full_matrix(V, S, P)
    np.testing.assert_allclose(F, T * np.eye(S * P), atol=1e-11)


def test_single_active_station():
    """Only station j non-zero -> only baseline (j, j) is non-zero."""
    S, T = 5, 9
    g = synth.rng(96)
    x = np.zeros((1, S, T, 2), dtype=np.complex128)
    j = 3
    x[0, j] = synth.complex_normal(g, (T, 2))
    V = oracle.correlate(x)[0]
    bj = j * (j + 1) // 2 + j
    for b in range(V.shape[0]):
        if b == bj:
            assert np.abs(V[b]).max() > 0
        else:
            assert np.abs(V[b]).max() == 0


# ---------------------------------------------------------------- invariants
def test_autocorrelations_real_nonnegative_and_hermitian_pol_block():
    d = synth.tiny()
    V = oracle.correlate(d["x"])
    S = d["S"]
    for s in range(S):
        b = s * (s + 1) // 2 + s
        for p in range(2):
            assert V[:, b, p, p].imag.max() == 0.0
            assert V[:, b, p, p].real.min() >= 0.0
        np.testing.assert_allclose(V[:, b, 0, 1], np.conj(V[:, b, 1, 0]), rtol=1e-13)


def test_identical_stations_identical_rows():
    """Stations 1 and 4 carry the same signal -> their baselines with any third
    station are identical."""
    g = synth.rng(95)
    x = synth.complex_normal(g, (2, 6, 21, 2)).astype(np.complex128)
    x[:, 4] = x[:, 1]
    V = oracle.correlate(x)
    for s in (5,):
        b1 = s * (s + 1) // 2 + 1
        b4 = s * (s + 1) // 2 + 4
        np.testing.assert_array_equal(V[:, b1], V[:, b4])
    np.testing.assert_array_equal(V[:, 1 * 2 // 2 + 1], V[:, 4 * 5 // 2 + 4])


def test_station_permutation():
    """Permuting stations permutes (or conjugates) baselines: V(B,A) = conj V(A,B)."""
    g = synth.rng(94)
    S = 5
    x = synth.complex_normal(g, (1, S, 13, 2)).astype(np.complex128)
    perm = np.array([3, 0, 4, 1, 2])
    F = full_matrix(oracle.correlate(x)[0], S, 2)
    Fp = full_matrix(oracle.correlate(x[:, perm])[0], S, 2)
    idx = (perm[:, None] * 2 + np.arange(2)[None, :]).reshape(-1)
    np.testing.assert_allclose(Fp, F[np.ix_(idx, idx)], rtol=1e-12, atol=1e-12)


def test_channel_independence_and_linearity_in_time():
    g = synth.rng(93)
    x = synth.complex_normal(g, (4, 3, 30, 2)).astype(np.complex128)
    V = oracle.correlate(x)
    order = np.array([2, 0, 3, 1])
    np.testing.assert_array_equal(oracle.correlate(x[order]), V[order])
    Va = oracle.correlate(x[:, :, :11])
    Vb = oracle.correlate(x[:, :, 11:])
    np.testing.assert_allclose(Va + Vb, V, rtol=1e-12, atol=1e-12)


def test_empty_time_axis():
    x = np.zeros((2, 3, 0, 2), dtype=np.complex128)
    V = oracle.correlate(x)
    assert V.shape == (2, 6, 2, 2) and not V.any()


# ----------------------------------------------------------- gain loss/grads
def _gain_case(S=3, T=6, C=2, seed=92):
    g = synth.rng(seed)
    x = synth.complex_normal(g, (C, S, T, 2)).astype(np.complex128)
    gains = (1 + synth.complex_normal(g, (C, S, 2), sigma=0.3)).astype(np.complex128)
    B = S * (S + 1) // 2
    M = synth.complex_normal(g, (C, B, 2, 2), sigma=3.0).astype(np.complex128)
    return x, gains, M


def test_gain_loss_special_cases():
    x, gains, M = _gain_case()
    R = oracle.correlate(x)
    L0, V0 = oracle.gain_loss(R, np.ones_like(gains), np.zeros_like(M))
    np.testing.assert_allclose(V0, R, rtol=1e-14)
    assert abs(L0 - (np.abs(R) ** 2).sum()) < 1e-9 * L0
    # a common phase on every gain cancels in g_a conj(g_b)
    ph = np.exp(0.7j) * np.ones_like(gains)
    _, Vp = oracle.gain_loss(R, ph, M)
    np.testing.assert_allclose(Vp, R, rtol=1e-12, atol=1e-12)
    # V(g*x) computed by correlating gain-scaled samples
    y = x * gains[:, :, None, :]
    L1, V1 = oracle.gain_loss(R, gains, M)
    np.testing.assert_allclose(V1, oracle.correlate(y), rtol=1e-12, atol=1e-12)
    assert abs(L1 - (np.abs(oracle.correlate(y) - M) ** 2).sum()) < 1e-9 * L1


def _fd_complex(f, z, h=1e-6):
    """Central differences of a real function of a complex array:
    returns dL/dRe + i dL/dIm (the PyTorch convention)."""
    out = np.zeros_like(z)
    flat = z.reshape(-1)
    o = out.reshape(-1)
    for k in range(flat.size):
        for unit in (1.0, 1j):
            zp = flat.copy(); zm = flat.copy()
            zp[k] += h * unit
            zm[k] -= h * unit
            d = (f(zp.reshape(z.shape)) - f(zm.reshape(z.shape))) / (2 * h)
            o[k] += d * (1.0 if unit == 1.0 else 1j)
    return out


def test_gain_grad_finite_differences():
    x, gains, M = _gain_case()
    R = oracle.correlate(x)
    ana = oracle.gain_grad(R, gains, M)
    fd = _fd_complex(lambda gg: oracle.gain_loss(R, gg, M)[0], gains)
    assert np.abs(ana - fd).max() < 1e-6 * np.abs(fd).max()


def test_input_grad_finite_differences():
    x, gains, M = _gain_case(S=3, T=4, C=1, seed=91)
    R = oracle.correlate(x)
    ana = oracle.input_grad(x, R, gains, M)

    def loss_of_x(xx):
        return oracle.gain_loss(oracle.correlate(xx), gains, M)[0]

    fd = _fd_complex(loss_of_x, x)
    assert np.abs(ana - fd).max() < 1e-6 * np.abs(fd).max()


# ----------------------------------------------------- pins catch mistakes
def _mutant_correlate(x, mutation):
    """A plain-Python copy of the loop nest with one planted mistake."""
    C, S, T, P = x.shape
    B = S * (S + 1) // 2
    out = np.zeros((C, B, P, P), dtype=complex)
    for c in range(C):
        for s2 in range(S):
            for s1 in range(s2 + 1):
                for p1 in range(P):
                    for p2 in range(P):
                        a = x[c, s1, :, p1]
                        b = x[c, s2, :, p2]
                        if mutation == "conj_wrong_side":
                            v = (np.conj(a) * b).sum()
                        elif mutation == "im_sign":
                            v = (a * np.conj(b)).sum().conjugate()
                        elif mutation == "dropped_term":
                            v = (a.real * b.real + 1j * (a.imag * b.real - a.real * b.imag)).sum()
                        elif mutation == "pol_swap":
                            v = (x[c, s1, :, p2] * np.conj(x[c, s2, :, p1])).sum()
                        else:
                            v = (a * np.conj(b)).sum()
                        if mutation == "baseline_index":
                            bb = s1 * (s1 + 1) // 2 + s2 if s1 * (s1 + 1) // 2 + s2 < B else 0
                        else:
                            bb = s2 * (s2 + 1) // 2 + s1
                        out[c, bb, p1, p2] = v
    return out


@pytest.mark.parametrize("mutation", ["conj_wrong_side", "im_sign", "dropped_term",
                                      "pol_swap", "baseline_index"])
def test_planted_mistakes_are_caught(mutation):
    """Each planted mistake breaks the numpy-matmul pin or the plane-wave pin."""
    g = synth.rng(90)
    S, T = 4, 10
    x = synth.complex_normal(g, (1, S, T, 2)).astype(np.complex128)
    assert np.allclose(_mutant_correlate(x, "none"), oracle.correlate(x))
    bad = _mutant_correlate(x, mutation)
    X = rows(x[0])
    ref = X @ X.conj().T
    F = full_matrix(bad[0], S, 2)
    assert not np.allclose(F, ref, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------- sample layouts
def _place_by_loops(x_cst, layout):
    """Builds a layout from its definition with plain loops: element
    (i, c, s, t) of the correlator layout goes to the layout's index tuple."""
    I, C, S, T = x_cst.shape[:4]
    shape = {"cst": (C, S, T), "cts": (C, T, S), "sct": (S, C, T)}[layout]
    out = np.zeros((I,) + shape + x_cst.shape[4:], dtype=x_cst.dtype)
    for i in range(I):
        for c in range(C):
            for s in range(S):
                for t in range(T):
                    idx = {"cst": (c, s, t), "cts": (c, t, s), "sct": (s, c, t)}[layout]
                    out[(i,) + idx] = x_cst[i, c, s, t]
    return out


def test_reorder_matches_placement_by_definition():
    rng = np.random.default_rng(7)
    x = rng.integers(-128, 128, size=(2, 3, 5, 4, 2, 2)).astype(np.int8)  # [I][C][S][T][pol][re,im]
    layouts = ("cst", "cts", "sct")
    built = {L: _place_by_loops(x, L) for L in layouts}
    for a in layouts:
        for b in layouts:
            np.testing.assert_array_equal(oracle.reorder(built[a], a, b), built[b])


def test_reorder_round_trip_and_composition():
    rng = np.random.default_rng(8)
    x = (rng.standard_normal((1, 4, 6, 7, 2)) + 1j * rng.standard_normal((1, 4, 6, 7, 2))).astype(np.complex64)
    for a in ("cts", "sct"):
        np.testing.assert_array_equal(oracle.reorder(oracle.reorder(x, "cst", a), a, "cst"), x)
    np.testing.assert_array_equal(oracle.reorder(oracle.reorder(x, "cst", "sct"), "sct", "cts"),
                                  oracle.reorder(x, "cst", "cts"))


# ------------------------------------------------------ single polarisation
def test_single_pol_is_the_xx_block_of_two_pols():
    """With P = 1 the loop nest of Fig. 2 runs over one pol: its visibilities
    equal the XX entries of a P = 2 correlation whose X pol carries the same
    samples (whatever Y holds), and a brute-force sum of exact integers."""
    rng = np.random.default_rng(21)
    C, S, T = 3, 7, 19
    x1 = rng.integers(-128, 128, size=(C, S, T, 1, 2)).astype(np.int8)
    y = rng.integers(-128, 128, size=(C, S, T, 1, 2)).astype(np.int8)
    x2 = np.concatenate([x1, y], axis=3)                       # pols (X = x1, Y = other)
    v1 = oracle.correlate(x1, "ci8")
    v2 = oracle.correlate(x2, "ci8")
    assert v1.shape == (C, S * (S + 1) // 2, 1, 1)
    np.testing.assert_array_equal(v1[..., 0, 0], v2[..., 0, 0])
    z = x1[..., 0, 0].astype(np.int64) + 1j * x1[..., 0, 1].astype(np.int64)
    for c in range(C):
        for s2 in range(S):
            for s1 in range(s2 + 1):
                want = sum(complex(z[c, s1, t]) * complex(z[c, s2, t]).conjugate() for t in range(T))
                assert v1[c, s2 * (s2 + 1) // 2 + s1, 0, 0] == want
