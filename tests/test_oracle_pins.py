"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
constants printed in Appendix A, closed forms derived from the transfer
function, dense triangular-solve matrices, invariants and exact identities.
"""
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly
from scipy.linalg import solve_triangular

from oracle import oracle as orc

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def paper_constants():
    out = {}
    with open(GOLD) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


C = paper_constants()


# ---------------------------------------------------------------- Appendix A
def test_abramowitz_stegun_approximation_bound():
    """The rational approximation of the Gaussian (Appendix A) is within the
    printed bound of exp(-t^2/2)/sqrt(2 pi)."""
    t = np.linspace(-8, 8, 20001)
    approx = 1.0 / (C["as_b0"] + C["as_b2"] * t**2 + C["as_b4"] * t**4
                    + C["as_b6"] * t**6)
    exact = np.exp(-t**2 / 2) / np.sqrt(2 * np.pi)
    assert np.max(np.abs(approx - exact)) < C["as_err_bound"]


def test_newton_root_and_factorisation():
    """s = 1.16680481/sigma is a root of b0 - b2 u^2 + b4 u^4 - b6 u^6 and the
    printed causal/anticausal factors multiply back to that polynomial."""
    b0, b2, b4, b6 = C["as_b0"], C["as_b2"], C["as_b4"], C["as_b6"]
    poly = np.array([b0, 0, -b2, 0, b4, 0, -b6])          # ascending in u
    x = C["newton_root"]
    assert abs(npoly.polyval(x, poly)) < 1e-6 * b0
    fr, q0, q1 = C["factor_real"], C["factor_quad_c0"], C["factor_quad_c1"]
    causal = npoly.polymul([fr, 1.0], [q0, q1, 1.0])
    anticausal = npoly.polymul([fr, -1.0], [q0, -q1, 1.0])
    prod = npoly.polymul(causal, anticausal)
    np.testing.assert_allclose(prod, poly / b6, rtol=0, atol=2e-5 * abs(b0 / b6))
    # the causal factor is the Theorem's cubic: P0 + P1 u + P2 u^2 + u^3
    np.testing.assert_allclose(
        causal, [C["theorem_P0"], C["theorem_P1"], C["theorem_P2"], 1.0],
        rtol=5e-7)
    assert C["theorem_a1_quad"] == pytest.approx(2 * C["theorem_P2"], abs=1e-6)


@pytest.mark.parametrize("sigma", [0.3, 1.0, 2.0, 7.5, 10.0, 40.0, 123.0])
def test_theorem_coefficients_from_z_transform(sigma):
    """a_{i,0..3} are the coefficients of D(sigma (1 - z^-1)), D being the
    product of the printed causal factors (backward difference s = 1 - z^-1)."""
    fr, q0, q1 = C["factor_real"], C["factor_quad_c0"], C["factor_quad_c1"]
    D = npoly.polymul([fr, 1.0], [q0, q1, 1.0])
    u = np.array([sigma, -sigma])                       # u(w) = sigma - sigma w
    acc = np.zeros(1)
    upow = np.array([1.0])
    for c in D:
        acc = npoly.polyadd(acc, c * upow)
        upow = npoly.polymul(upow, u)
    expect = np.array([acc[0], -acc[1], -acc[2], -acc[3]])
    a, alpha, beta = orc.rf3_coeffs(sigma)
    np.testing.assert_allclose(a, expect, rtol=2e-6, atol=2e-6 * abs(expect[0]))
    np.testing.assert_allclose(alpha, a[1:] / a[0], rtol=1e-15)
    # normalisation: beta = (2 pi sigma^2)^(1/4) (a0 - a1 - a2 - a3)/a0
    g = (2 * np.pi * sigma**2) ** 0.25
    assert beta == pytest.approx(g * C["theorem_P0"] / a[0], rel=1e-9)


# ------------------------------------------------------------- closed forms
def impulse_line(sigma, **kw):
    n = int(60 * sigma) + 64
    x = np.zeros(2 * n + 1)
    x[n] = 1.0
    return np.arange(2 * n + 1) - n, orc.line(x, sigma, img_factor=0.0, **kw)


@pytest.mark.parametrize("sigma", [2.0, 10.0, 40.0])
def test_rf3_dc_gain_is_sqrt_2pi_sigma(sigma):
    """Each pass has DC gain (2 pi sigma^2)^(1/4) (Appendix A normalisation),
    so forward + backward sum to sqrt(2 pi) sigma: the sum of exp(-x^2/2s^2)."""
    _, h = impulse_line(sigma)
    assert h.sum() == pytest.approx(np.sqrt(2 * np.pi) * sigma, rel=1e-12)


@pytest.mark.parametrize("sigma", [2.0, 10.0, 40.0])
def test_rf3_impulse_variance_closed_form(sigma):
    """Cumulant expansion of 1/D(sigma(1-e^t)) times its mirror gives
    Var = 2[(P1/P0) sigma + ((P1/P0)^2 - 2 P2/P0) sigma^2], mean 0."""
    n, h = impulse_line(sigma)
    P0, P1, P2 = C["theorem_P0"], C["theorem_P1"], C["theorem_P2"]
    m0 = h.sum()
    mean = (n * h).sum() / m0
    var = ((n - mean) ** 2 * h).sum() / m0
    r = P1 / P0
    assert abs(mean) < 1e-9 * sigma
    assert var == pytest.approx(2 * (r * sigma + (r * r - 2 * P2 / P0) * sigma**2),
                                rel=1e-9)


@pytest.mark.parametrize("sigma,K", [(2.0, 1), (4.0, 5), (10.0, 5), (10.0, 10)])
def test_rf1_hayden_variance_and_gain(sigma, K):
    """Hayden's relation R^2 = 2K alpha/(1-alpha)^2 dx^2 makes the K-times
    iterated forward+backward impulse response have variance sigma^2; the
    unit-sum form has gain 1, the Gaussian-peak form sqrt(2 pi) sigma."""
    n, h = impulse_line(sigma, order=1, iters=K, norm=orc.NORM_UNIT_SUM)
    assert h.sum() == pytest.approx(1.0, rel=1e-11)
    assert ((n * n) * h).sum() == pytest.approx(sigma**2, rel=1e-9)
    _, hg = impulse_line(sigma, order=1, iters=K)
    assert hg.sum() == pytest.approx(np.sqrt(2 * np.pi) * sigma, rel=1e-11)


@pytest.mark.parametrize("sigma", [0.7, 2.0, 5.0, 10.0, 40.0])
def test_q_corrected_rf3_has_variance_sigma_squared(sigma):
    """The q-corrected 3rd-RF (an option, not the paper's filter)
    takes the Theorem 3.1 coefficients at q(sigma) so that the measured
    variance of the line filter's impulse response is sigma^2, while the
    normalisation of sigma keeps the response sum at sqrt(2 pi) sigma."""
    n = int(40 * sigma) + 40
    x = np.zeros(2 * n + 1)
    x[n] = 1.0
    h = orc.line(x, sigma, img_factor=0.0, qcorr=True)
    k = np.arange(-n, n + 1)
    m0 = h.sum()
    assert m0 == pytest.approx(np.sqrt(2 * np.pi) * sigma, rel=1e-11)
    assert abs((k * h).sum() / m0) < 1e-9 * sigma
    assert (k * k * h).sum() / m0 == pytest.approx(sigma**2, rel=1e-9)
    q = orc.q_of_sigma(sigma)
    assert 0.0 < q < sigma   # the plain filter is wider than sigma
    _, _, beta = orc.rf3_coeffs(sigma, qcorr=True)
    _, _, beta_q = orc.rf3_coeffs(q)
    # beta: the recursion of q with the normalisation of sigma
    assert beta == pytest.approx(beta_q * np.sqrt(sigma / q), rel=1e-12)


def test_q_corrected_rf3_fits_the_gaussian_better_at_small_sigma():
    """Relative L2 distance of the impulse response to exp(-x^2/2 sigma^2):
    the variance match helps where the plain filter is much too wide (small
    sigma) and costs at large sigma, where the responses' heavier tails carry
    the extra variance."""
    def l2(sigma, qcorr):
        n = int(40 * sigma) + 40
        x = np.zeros(2 * n + 1)
        x[n] = 1.0
        h = orc.line(x, sigma, img_factor=0.0, qcorr=qcorr)
        k = np.arange(-n, n + 1)
        g = np.exp(-k * k / (2 * sigma * sigma))
        return np.sqrt(((h - g) ** 2).sum() / (g * g).sum())
    assert l2(2.0, True) < 0.5 * l2(2.0, False)
    assert l2(5.0, True) < l2(5.0, False)
    assert l2(40.0, True) > l2(40.0, False)


def test_rf1_coefficients_satisfy_hayden():
    for sigma, K in [(1.5, 1), (5.0, 5), (40.0, 10)]:
        alpha, beta = orc.rf1_coeffs(sigma, K, orc.NORM_UNIT_SUM)
        assert 0 < alpha < 1
        assert beta == pytest.approx(1 - alpha, rel=1e-13)
        assert 2 * K * alpha / (1 - alpha) ** 2 == pytest.approx(sigma**2, rel=1e-11)


# ------------------------------------------------------------- dense matrices
def dense_pair_matrix(sig, order, K, norm):
    """One forward+backward pair U^-1 D L^-1 D on an all-sea extended
    segment, from triangular solves (L unit lower with L[i,i-j] = -alpha_{i,j},
    U unit upper with U[i,i+j] = -alpha_{i,j}, D = diag(beta)); the 1st-RF
    coefficients are those for K iterations."""
    m = len(sig)
    Lm = np.eye(m)
    Um = np.eye(m)
    beta = np.zeros(m)
    for i, s in enumerate(sig):
        if order == 3:
            _, al, beta[i] = orc.rf3_coeffs(s, norm)
        else:
            a1, beta[i] = orc.rf1_coeffs(s, K, norm)
            al = [a1]
        for j, a in enumerate(al, start=1):
            if i - j >= 0:
                Lm[i, i - j] = -a
            if i + j < m:
                Um[i, i + j] = -a
    D = np.diag(beta)
    return solve_triangular(Um, D @ solve_triangular(Lm, D, lower=True), lower=False)


def dense_line_matrix(mask, sig, order=3, K=1, img=3.0, norm=0):
    """The whole line operator as a dense matrix, segment by segment: extend
    each sea run by ceil(img*sigma_coast) points with the coastal sigma,
    apply the pair, restrict back; K iterations give (R G E)^K."""
    n = len(mask)
    G = np.zeros((n, n))
    i = 0
    while i < n:
        if not mask[i]:
            i += 1
            continue
        b = i
        while i < n and mask[i]:
            i += 1
        seg = list(range(b, i))
        nl = int(np.ceil(img * sig[b])) if img > 0 else 0
        nr = int(np.ceil(img * sig[i - 1])) if img > 0 else 0
        ext = [sig[b]] * nl + [sig[t] for t in seg] + [sig[i - 1]] * nr
        L = len(seg)
        R = np.zeros((L, len(ext)))
        R[np.arange(L), nl + np.arange(L)] = 1.0
        blk = R @ dense_pair_matrix(ext, order, K, norm) @ R.T
        G[np.ix_(seg, seg)] = np.linalg.matrix_power(blk, K)
    return G


def oracle_line_matrix(mask, sig, adjoint=False, **kw):
    n = len(mask)
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(orc.line(e, sig, mask, adjoint=adjoint, **kw))
    return np.array(cols).T


@pytest.mark.parametrize("img", [0.0, 1.0, 2.5])
@pytest.mark.parametrize("order,K", [(3, 1), (1, 1), (1, 5)])
def test_line_matches_dense_triangular_solves(order, K, img):
    rng = np.random.default_rng(7)
    n = 23
    mask = np.ones(n, np.uint8)
    mask[[0, 6, 7, 15]] = 0
    sig = rng.uniform(0.6, 3.0, n)
    G = dense_line_matrix(mask, sig, order, K, img)
    O = oracle_line_matrix(mask, sig, order=order, iters=K, img_factor=img)
    np.testing.assert_allclose(O, G, rtol=0, atol=1e-12 * np.abs(G).max())
    OT = oracle_line_matrix(mask, sig, adjoint=True, order=order, iters=K,
                            img_factor=img)
    np.testing.assert_allclose(OT, G.T, rtol=0, atol=1e-12 * np.abs(G).max())


def test_heuristic_initial_conditions_printed_form():
    """With no imaginary points, the first three forward outputs and the last
    three backward outputs follow the printed initial conditions (Sec. 3.1)."""
    rng = np.random.default_rng(3)
    n = 9
    sig = rng.uniform(1.0, 4.0, n)
    x = rng.standard_normal(n)
    al = np.zeros((n, 3))
    be = np.zeros(n)
    for i in range(n):
        _, al[i], be[i] = orc.rf3_coeffs(sig[i])
    p = np.zeros(n)
    p[0] = be[0] * x[0]
    p[1] = be[1] * x[1] + al[1, 0] * p[0]
    p[2] = be[2] * x[2] + al[2, 0] * p[1] + al[2, 1] * p[0]
    for i in range(3, n):
        p[i] = be[i] * x[i] + al[i, 0] * p[i - 1] + al[i, 1] * p[i - 2] + al[i, 2] * p[i - 3]
    s = np.zeros(n)
    s[n - 1] = be[n - 1] * p[n - 1]
    s[n - 2] = be[n - 2] * p[n - 2] + al[n - 2, 0] * s[n - 1]
    s[n - 3] = be[n - 3] * p[n - 3] + al[n - 3, 0] * s[n - 2] + al[n - 3, 1] * s[n - 1]
    for i in range(n - 4, -1, -1):
        s[i] = be[i] * p[i] + al[i, 0] * s[i + 1] + al[i, 1] * s[i + 2] + al[i, 2] * s[i + 3]
    np.testing.assert_allclose(orc.line(x, sig, img_factor=0.0), s, rtol=1e-13,
                               atol=1e-14)


# ---------------------------------------------------------------- coasts
def test_single_point_segment_gives_beta_squared():
    mask = np.array([0, 1, 0], np.uint8)
    x = np.array([5.0, 2.0, 7.0])
    _, _, beta = orc.rf3_coeffs(3.0)
    y = orc.line(x, 3.0, mask, img_factor=0.0)
    assert y[0] == 0.0 and y[2] == 0.0
    assert y[1] == pytest.approx(beta * beta * 2.0, rel=1e-14)


def test_imaginary_points_equal_zero_padded_sea():
    """A segment extended by imaginary points behaves exactly as the same
    segment inside a longer all-sea line padded with zero input and the
    coastal length scale, restricted back to the segment."""
    rng = np.random.default_rng(11)
    L = 40
    sig = rng.uniform(2.0, 6.0, L)
    x = rng.standard_normal(L)
    f = 2.0
    nl = int(np.ceil(f * sig[0]))
    nr = int(np.ceil(f * sig[-1]))
    pad_sig = np.concatenate([[sig[0]] * nl, sig, [sig[-1]] * nr])
    # 3rd-RF: one pass pair over the padded line, read back on the segment
    y = orc.line(x, sig, img_factor=f)
    pad_x = np.concatenate([np.zeros(nl), x, np.zeros(nr)])
    ref = orc.line(pad_x, pad_sig, img_factor=0.0)[nl:nl + L]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-13)
    # 1st-RF x5: every iteration re-pads with zeros (no carried imaginary values)
    G = dense_line_matrix(np.ones(L, np.uint8), sig, 1, 5, f)
    y1 = orc.line(x, sig, img_factor=f, order=1, iters=5)
    np.testing.assert_allclose(y1, G @ x, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
@pytest.mark.parametrize("adjoint", [False, True])
def test_infinite_imaginary_sea_equals_long_zero_padding(order, K, adjoint):
    """img_factor = inf (the infinite imaginary sea) on a segment equals the
    same segment in the middle of an all-sea line padded on each side with
    zero input and the coastal length scale, filtered with no imaginary
    points and read back on the segment.  The padding (2000 points for the
    3rd-RF, 500 for the 1st-RF: 50 and 12 length scales at sigma <= 40) is
    long enough for the response to die out.  For K > 1 every iteration
    re-pads with zeros: K applications of the pair matrix of the K-filter
    (dense triangular solves) on the padded line."""
    rng = np.random.default_rng(12)
    L = 60
    pad = 2000 if order == 3 else 500
    sig = rng.uniform(2.0, 40.0, L)
    x = rng.standard_normal(L)
    y = orc.line(x, sig, img_factor=np.inf, order=order, iters=K, adjoint=adjoint)
    pad_sig = np.concatenate([[sig[0]] * pad, sig, [sig[-1]] * pad])
    if order == 3:
        pad_x = np.concatenate([np.zeros(pad), x, np.zeros(pad)])
        ref = orc.line(pad_x, pad_sig, img_factor=0.0, adjoint=adjoint)[pad:pad + L]
    else:
        G = dense_pair_matrix(pad_sig, 1, K, 0)
        if adjoint:
            G = G.T
        blk = G[pad:pad + L, pad:pad + L]   # zero padding in, restriction out
        ref = np.linalg.matrix_power(blk, K) @ x
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("order,K", [(3, 1), (1, 1), (1, 5)])
def test_infinite_imaginary_sea_cut_is_below_fp64(order, K):
    """The oracle cuts the infinite imaginary sea at n points; the part it
    drops decays like rho^n with rho the spectral radius of the one-step
    companion matrix of the recursion (from the oracle's own coefficients).
    rho^n must be below 1e-30 over the length scales in use."""
    for sigma in [0.3, 0.7, 1.5, 3.0, 10.0, 40.0, 200.0]:
        if order == 3:
            _, al, _ = orc.rf3_coeffs(sigma)
            comp = np.array([al, [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
            rho = np.max(np.abs(np.linalg.eigvals(comp)))
        else:
            rho, _ = orc.rf1_coeffs(sigma, K)
        n = orc.n_imaginary(np.inf, sigma)
        assert rho < 1.0
        assert n * np.log(rho) < np.log(1e-30), (sigma, rho, n)


def test_infinite_imaginary_sea_adjoint_dot_product():
    rng = np.random.default_rng(13)
    n = 90
    mask = (rng.random(n) > 0.25).astype(np.uint8)
    sig = rng.uniform(1.5, 30.0, n)
    for order, K in [(3, 1), (1, 5)]:
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        a = orc.line(x, sig, mask, order=order, iters=K, img_factor=np.inf)
        b = orc.line(y, sig, mask, order=order, iters=K, img_factor=np.inf, adjoint=True)
        assert abs(a @ y - x @ b) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(y)


def test_land_isolates_signal():
    """An impulse on one side of a one-cell land strip gives exactly zero on
    the other side, in 1-D and behind a full land wall in 2-D."""
    n = 60
    mask = np.ones(n, np.uint8)
    mask[30] = 0
    x = np.zeros(n)
    x[25] = 1.0
    for order, K in [(3, 1), (1, 5)]:
        y = orc.line(x, 8.0, mask, order=order, iters=K)
        assert np.all(y[30:] == 0.0)
        assert np.all(y[:30] != 0.0)
    ny, nx = 24, 32
    m2 = np.ones((ny, nx), np.uint8)
    m2[:, 16] = 0
    f = np.zeros((ny, nx))
    f[12, 8] = 1.0
    L = np.full((ny, nx), 5.0)
    for order, K in [(3, 1), (1, 5)]:
        for adj in (False, True):
            out = orc.vh(f, m2, L, L, order=order, iters=K, adjoint=adj)
            assert np.all(out[:, 16:] == 0.0)


# ---------------------------------------------------------------- 2-D
@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_constant_field_is_scaled_by_2pi_sx_sy(order, K):
    """Away from the boundaries a constant c maps to c * 2 pi sigma_x sigma_y
    (Gaussian-peak normalisation), and to c with the unit-sum form."""
    ny, nx = 200, 220
    sx, sy = 4.0, 3.0
    m = np.ones((ny, nx), np.uint8)
    f = np.full((ny, nx), 1.7)
    out = orc.vh(f, m, np.full((ny, nx), sx), np.full((ny, nx), sy),
                 order=order, iters=K, img_factor=0.0)
    interior = out[90:110, 100:120]
    np.testing.assert_allclose(interior, 1.7 * 2 * np.pi * sx * sy, rtol=1e-10)
    out1 = orc.vh(f, m, np.full((ny, nx), sx), np.full((ny, nx), sy),
                  order=order, iters=K, img_factor=0.0, norm=orc.NORM_UNIT_SUM)
    np.testing.assert_allclose(out1[90:110, 100:120], 1.7, rtol=1e-10)


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_vh_equals_kronecker_of_line_matrices(order, K):
    """V_H = G_y G_x on a tiny grid with land and varying sigma equals the
    product of the block-diagonal row operator and column operator."""
    rng = np.random.default_rng(5)
    ny, nx = 9, 11
    mask = (rng.uniform(size=(ny, nx)) > 0.25).astype(np.uint8)
    Lx = rng.uniform(0.8, 3.0, (ny, nx))
    Ly = rng.uniform(0.8, 3.0, (ny, nx))
    N = nx * ny
    Gx = np.zeros((N, N))
    for j in range(ny):
        idx = j * nx + np.arange(nx)
        Gx[np.ix_(idx, idx)] = dense_line_matrix(mask[j], Lx[j], order, K, 1.5)
    Gy = np.zeros((N, N))
    for i in range(nx):
        idx = np.arange(ny) * nx + i
        Gy[np.ix_(idx, idx)] = dense_line_matrix(mask[:, i], Ly[:, i], order, K, 1.5)
    V = Gy @ Gx
    x = rng.standard_normal((ny, nx))
    y = orc.vh(x, mask, Lx, Ly, order=order, iters=K, img_factor=1.5)
    np.testing.assert_allclose(y.ravel(), V @ x.ravel(), rtol=0,
                               atol=1e-12 * np.abs(V @ x.ravel()).max())
    yt = orc.vh(x, mask, Lx, Ly, order=order, iters=K, img_factor=1.5, adjoint=True)
    np.testing.assert_allclose(yt.ravel(), V.T @ x.ravel(), rtol=0,
                               atol=1e-12 * np.abs(V.T @ x.ravel()).max())


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_adjoint_dot_product(order, K):
    """<V x, y> = <x, V^T y> to 1e-12 on a multi-level field with land."""
    rng = np.random.default_rng(9)
    nz, ny, nx = 3, 40, 56
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.2).astype(np.uint8)
    Lx = rng.uniform(2.0, 12.0, (ny, nx))
    Ly = rng.uniform(2.0, 12.0, (ny, nx))
    x = rng.standard_normal((2, nz, ny, nx))
    y = rng.standard_normal((2, nz, ny, nx))
    Vx = orc.vh(x, mask, Lx, Ly, order=order, iters=K)
    VTy = orc.vh(y, mask, Lx, Ly, order=order, iters=K, adjoint=True)
    lhs = np.vdot(Vx, y)
    rhs = np.vdot(x, VTy)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Vx) * np.linalg.norm(y)


def test_uniform_sigma_all_sea_is_self_adjoint():
    rng = np.random.default_rng(1)
    ny, nx = 30, 34
    m = np.ones((ny, nx), np.uint8)
    L = np.full((ny, nx), 4.0)
    x = rng.standard_normal((ny, nx))
    a = orc.vh(x, m, L, L)
    b = orc.vh(x, m, L, L, adjoint=True)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- Remark 1
@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_remark1_valid_bounds(order, K):
    """Remark 1 in the two forms that hold for a discrete convolution:
    pointwise |s - s*| <= ||eps_h||_2 ||s0||_2 (the Cauchy-Schwarz step of its
    proof) and ||eps_s||_2 <= ||eps_h||_1 ||s0||_2 (Young)."""
    sigma = 4.0
    n = 1200
    rng = np.random.default_rng(2)
    s0 = np.zeros(n)
    s0[400:800] = rng.standard_normal(400)
    s = orc.line(s0, sigma, img_factor=0.0, order=order, iters=K)
    k = np.arange(-300, 301)
    g = np.exp(-k**2 / (2 * sigma**2))
    s_star = np.convolve(s0, g, mode="same")
    imp = np.zeros(n)
    imp[600] = 1.0
    h = orc.line(imp, sigma, img_factor=0.0, order=order, iters=K)[300:901]
    eps_h = g - h
    bound_pt = np.linalg.norm(eps_h) * np.linalg.norm(s0)
    err = s - s_star
    assert np.max(np.abs(err)) <= bound_pt
    assert np.linalg.norm(err) <= np.abs(eps_h).sum() * np.linalg.norm(s0)


def dense_gaussian(mask, sigma):
    """Brute force: G_ij = exp(-|r_i - r_j|^2 / (2 sigma^2)) between the grid
    points of a [ny][nx] grid (row-major), zero rows and columns at land."""
    ny, nx = mask.shape
    jj, ii = np.divmod(np.arange(ny * nx), nx)
    r2 = (jj[:, None] - jj[None, :]) ** 2 + (ii[:, None] - ii[None, :]) ** 2
    G = np.exp(-r2 / (2.0 * sigma * sigma))
    sea = mask.ravel().astype(bool)
    G[~sea, :] = 0.0
    G[:, ~sea] = 0.0
    return G


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_dense_gaussian_brute_force_2d(order, K):
    """V_H against the dense 2-D Gaussian matrix-vector product G x on a
    24 x 32 grid at sigma = 3.  All sea with the infinite imaginary sea,
    V_H is the restriction of the 2-D convolution with h_x (x) h_y (h the
    1-D impulse response), so the two valid forms of Remark 1 hold in 2-D
    with eps_h = g - h_x (x) h_y: pointwise |V x - G x| <= ||eps_h||_2 ||x||_2
    and ||V x - G x||_2 <= ||eps_h||_1 ||x||_2.  With land (25 % scattered
    land points) the Gaussian reaches across land and the filters do not;
    land rows stay exactly zero.  The relative distances ||V x - G x|| /
    ||G x|| are the reported comparison (about 0.37 for the 3rd-RF and 0.15
    for the 1st-RF x5 all sea, about 0.66 for both with land)."""
    rng = np.random.default_rng(15)
    ny, nx, sigma = 24, 32, 3.0
    L = np.full((ny, nx), sigma)
    # all sea, infinite imaginary sea: the bounds
    mask = np.ones((ny, nx), np.uint8)
    x = rng.standard_normal((ny, nx))
    v = orc.vh(x, mask, L, L, order=order, iters=K, img_factor=np.inf)
    gx = (dense_gaussian(mask, sigma) @ x.ravel()).reshape(ny, nx)
    n = 401
    imp = np.zeros(n)
    imp[n // 2] = 1.0
    h = orc.line(imp, sigma, order=order, iters=K, img_factor=np.inf)
    d = np.arange(n) - n // 2
    eps = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * sigma * sigma)) - np.outer(h, h)
    err = v - gx
    xn = np.linalg.norm(x)
    assert np.abs(err).max() <= np.linalg.norm(eps) * xn
    assert np.linalg.norm(err) <= np.abs(eps).sum() * xn
    rel_sea = np.linalg.norm(err) / np.linalg.norm(gx)
    assert (0.25 < rel_sea < 0.5) if order == 3 else (0.08 < rel_sea < 0.25)
    # with land: the brute-force comparison, land exactly zero
    mask = (rng.random((ny, nx)) > 0.25).astype(np.uint8)
    x = rng.standard_normal((ny, nx)) * mask
    v = orc.vh(x, mask, L, L, order=order, iters=K, img_factor=3.0)
    gx = (dense_gaussian(mask, sigma) @ x.ravel()).reshape(ny, nx)
    assert np.all(v[mask == 0] == 0.0)
    rel_land = np.linalg.norm(v - gx) / np.linalg.norm(gx)
    assert rel_sea < rel_land < 1.0


# ------------------------------------------- constant-extension coasts
def dense_const_line_matrix(mask, sig, order=3, K=1, img=3.0, norm=0):
    """The line operator with constant-extension coasts as a dense matrix:
    per sea run, E_c copies the first sea value into the ceil(img*sigma)
    imaginary points on the left and the last one into those on the right,
    the pair matrix filters the extended run and R reads the sea points
    back; K iterations give (R G E_c)^K."""
    n = len(mask)
    G = np.zeros((n, n))
    i = 0
    while i < n:
        if not mask[i]:
            i += 1
            continue
        b = i
        while i < n and mask[i]:
            i += 1
        seg = list(range(b, i))
        L = len(seg)
        nl = int(np.ceil(img * sig[b])) if img > 0 else 0
        nr = int(np.ceil(img * sig[i - 1])) if img > 0 else 0
        ext = [sig[b]] * nl + [sig[t] for t in seg] + [sig[i - 1]] * nr
        E = np.zeros((len(ext), L))
        E[:nl, 0] = 1.0
        E[nl + np.arange(L), np.arange(L)] = 1.0
        E[nl + L:, L - 1] = 1.0
        R = np.zeros((L, len(ext)))
        R[np.arange(L), nl + np.arange(L)] = 1.0
        blk = R @ dense_pair_matrix(ext, order, K, norm) @ E
        G[np.ix_(seg, seg)] = np.linalg.matrix_power(blk, K)
    return G


@pytest.mark.parametrize("img", [1.0, 2.5])
@pytest.mark.parametrize("order,K", [(3, 1), (1, 1), (1, 5)])
def test_constant_coast_matches_dense_extension_matrix(order, K, img):
    """Constant extension against its definition as matrices, forward and
    adjoint (the adjoint is the transpose: E_c^T sums the imaginary values
    into the edge point).  The runs include one of a single point."""
    rng = np.random.default_rng(17)
    n = 24
    mask = np.ones(n, np.uint8)
    mask[[0, 6, 7, 9, 16]] = 0           # point 8 is a one-point segment
    sig = rng.uniform(0.6, 3.0, n)
    G = dense_const_line_matrix(mask, sig, order, K, img)
    kw = dict(order=order, iters=K, img_factor=img, coast=orc.COAST_CONSTANT)
    O = oracle_line_matrix(mask, sig, **kw)
    np.testing.assert_allclose(O, G, rtol=0, atol=1e-12 * np.abs(G).max())
    OT = oracle_line_matrix(mask, sig, adjoint=True, **kw)
    np.testing.assert_allclose(OT, G.T, rtol=0, atol=1e-12 * np.abs(G).max())
    # the zero-input coasts give a different operator
    assert np.abs(dense_line_matrix(mask, sig, order, K, img) - G).max() > 1e-3


def test_constant_coast_equals_padded_line_with_edge_values():
    """A segment with constant-extension coasts behaves as the same segment
    inside a longer sea line whose padding holds the edge values (and the
    coastal length scales), filtered without any imaginary points."""
    rng = np.random.default_rng(19)
    L = 37
    sig = rng.uniform(2.0, 6.0, L)
    x = rng.standard_normal(L)
    f = 2.0
    nl = int(np.ceil(f * sig[0]))
    nr = int(np.ceil(f * sig[-1]))
    pad_sig = np.concatenate([[sig[0]] * nl, sig, [sig[-1]] * nr])
    pad_x = np.concatenate([[x[0]] * nl, x, [x[-1]] * nr])
    y = orc.line(x, sig, img_factor=f, coast=orc.COAST_CONSTANT)
    ref = orc.line(pad_x, pad_sig, img_factor=0.0)[nl:nl + L]
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_constant_coast_keeps_a_constant_up_to_the_coast(order, K):
    """A constant field keeps its interior gain sqrt(2 pi) sigma (both
    filters, Gaussian-peak normalisation) right up to the coast when the
    imaginary points carry the edge value: with 20 sigma of them the edge
    transient (decaying like |pole|^distance) is below 1e-6.  With zero
    input at the imaginary points the coastal value loses about half."""
    sigma, n = 3.0, 160
    mask = np.ones(n, np.uint8)
    mask[70:74] = 0
    gain = np.sqrt(2 * np.pi) * sigma
    kw = dict(order=order, iters=K, img_factor=20.0)
    y = orc.line(np.ones(n), sigma, mask, coast=orc.COAST_CONSTANT, **kw)
    sea = mask == 1
    np.testing.assert_allclose(y[sea], gain, rtol=1e-6)
    assert np.all(y[~sea] == 0.0)
    y0 = orc.line(np.ones(n), sigma, mask, **kw)
    assert y0[69] < 0.75 * gain and y0[0] < 0.75 * gain


def test_constant_coast_isolated_point_gets_the_line_gain():
    """One sea point between land: with constant extension the extended run
    is constant, so the point is multiplied by the 1-D gain sqrt(2 pi) sigma
    (to the edge transient, below 1e-6 with 20 sigma of imaginary points);
    without imaginary points it is multiplied by beta^2."""
    sigma = 2.5
    mask = np.array([0, 1, 0], np.uint8)
    x = np.array([4.0, -3.0, 9.0])
    y = orc.line(x, sigma, mask, img_factor=20.0, coast=orc.COAST_CONSTANT)
    assert y[1] == pytest.approx(-3.0 * np.sqrt(2 * np.pi) * sigma, rel=1e-6)
    _, _, beta = orc.rf3_coeffs(sigma)
    y0 = orc.line(x, sigma, mask, img_factor=0.0, coast=orc.COAST_CONSTANT)
    assert y0[1] == pytest.approx(-3.0 * beta * beta, rel=1e-14)


@pytest.mark.parametrize("order,K", [(3, 1), (1, 5)])
def test_constant_coast_adjoint_dot_product(order, K):
    rng = np.random.default_rng(23)
    nz, ny, nx = 2, 30, 44
    mask = (rng.uniform(size=(nz, ny, nx)) > 0.25).astype(np.uint8)
    Lx = rng.uniform(1.0, 9.0, (ny, nx))
    Ly = rng.uniform(1.0, 9.0, (ny, nx))
    x = rng.standard_normal((2, nz, ny, nx))
    y = rng.standard_normal((2, nz, ny, nx))
    kw = dict(order=order, iters=K, coast=orc.COAST_CONSTANT)
    Vx = orc.vh(x, mask, Lx, Ly, **kw)
    VTy = orc.vh(y, mask, Lx, Ly, adjoint=True, **kw)
    lhs, rhs = np.vdot(Vx, y), np.vdot(x, VTy)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Vx) * np.linalg.norm(y)
    # with no imaginary points the two coast treatments coincide exactly
    a = orc.vh(x, mask, Lx, Ly, img_factor=0.0, **kw)
    b = orc.vh(x, mask, Lx, Ly, img_factor=0.0, order=order, iters=K)
    assert np.array_equal(a, b)


# ------------------------------------- comparison with the exact Gaussian
# ------------------------------------------------- carried coasts
def dense_carried_line_matrix(mask, sig, K, img, norm=0):
    """The 1st-RF x K line operator with carried coasts as a dense matrix: per
    sea run, zero-extend once by ceil(img*sigma) imaginary points with the
    coastal sigma, apply the pair matrix K times on the extended run, read the
    sea points back: R G_ext^K R^T."""
    n = len(mask)
    G = np.zeros((n, n))
    i = 0
    while i < n:
        if not mask[i]:
            i += 1
            continue
        b = i
        while i < n and mask[i]:
            i += 1
        seg = list(range(b, i))
        L = len(seg)
        nl = int(np.ceil(img * sig[b])) if img > 0 else 0
        nr = int(np.ceil(img * sig[i - 1])) if img > 0 else 0
        ext = [sig[b]] * nl + [sig[t] for t in seg] + [sig[i - 1]] * nr
        R = np.zeros((L, len(ext)))
        R[np.arange(L), nl + np.arange(L)] = 1.0
        G[np.ix_(seg, seg)] = R @ np.linalg.matrix_power(dense_pair_matrix(ext, 1, K, norm), K) @ R.T
    return G


@pytest.mark.parametrize("K,img", [(2, 1.0), (5, 1.0), (5, 2.5), (3, 0.6)])
def test_carried_coast_matches_dense_extension_power(K, img):
    """Carried coasts against their definition as matrices, forward and
    adjoint (the transpose), on runs that include a one-point segment."""
    rng = np.random.default_rng(23)
    n = 26
    mask = np.ones(n, np.uint8)
    mask[[0, 5, 6, 8, 17]] = 0           # point 7 is a one-point segment
    sig = rng.uniform(0.6, 3.0, n)
    G = dense_carried_line_matrix(mask, sig, K, img)
    kw = dict(order=1, iters=K, img_factor=img, coast=orc.COAST_CARRIED)
    O = oracle_line_matrix(mask, sig, **kw)
    np.testing.assert_allclose(O, G, rtol=0, atol=1e-12 * np.abs(G).max())
    OT = oracle_line_matrix(mask, sig, adjoint=True, **kw)
    np.testing.assert_allclose(OT, G.T, rtol=0, atol=1e-12 * np.abs(G).max())
    # it is a different operator from re-extending with zeros every iteration
    assert np.abs(dense_line_matrix(mask, sig, 1, K, img) - G).max() > 1e-4


def test_carried_coast_equals_iterating_on_the_zero_padded_line():
    """On one sea run the carried coast is the filter iterated K times on the
    run padded with explicit sea points carrying the coastal sigma and zero
    input (no imaginary points: img_factor 0), read back on the run."""
    rng = np.random.default_rng(31)
    L, K, img = 40, 5, 2.0
    sig = rng.uniform(1.0, 4.0, L)
    x = rng.standard_normal(L)
    nl, nr = int(np.ceil(img * sig[0])), int(np.ceil(img * sig[-1]))
    pad_sig = np.concatenate([np.full(nl, sig[0]), sig, np.full(nr, sig[-1])])
    pad_x = np.concatenate([np.zeros(nl), x, np.zeros(nr)])
    for adjoint in (False, True):
        ref = orc.line(pad_x, pad_sig, order=1, iters=K, img_factor=0.0, adjoint=adjoint)[nl:nl + L]
        got = orc.line(x, sig, order=1, iters=K, img_factor=img, adjoint=adjoint,
                       coast=orc.COAST_CARRIED)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_carried_coast_reduces_to_zero_coast_for_one_iteration():
    rng = np.random.default_rng(37)
    ny, nx = 14, 19
    mask = (rng.random((ny, nx)) > 0.3).astype(np.uint8)
    L = rng.uniform(0.8, 3.0, (ny, nx))
    x = rng.standard_normal((1, 1, ny, nx))
    for order in (1, 3):
        for adjoint in (False, True):
            a = orc.vh(x, mask, L, L, order=order, iters=1, img_factor=2.0, adjoint=adjoint)
            b = orc.vh(x, mask, L, L, order=order, iters=1, img_factor=2.0, adjoint=adjoint,
                       coast=orc.COAST_CARRIED)
            assert np.array_equal(a, b)


def test_carried_coast_adjoint_dot_product_2d():
    rng = np.random.default_rng(41)
    ny, nx = 17, 23
    mask = (rng.random((ny, nx)) > 0.25).astype(np.uint8)
    Lx = rng.uniform(0.8, 3.5, (ny, nx))
    Ly = rng.uniform(0.8, 3.5, (ny, nx))
    x = rng.standard_normal((2, 2, ny, nx))
    y = rng.standard_normal((2, 2, ny, nx))
    kw = dict(order=1, iters=5, img_factor=2.5, coast=orc.COAST_CARRIED)
    vx = orc.vh(x, mask, Lx, Ly, **kw)
    vty = orc.vh(y, mask, Lx, Ly, adjoint=True, **kw)
    lhs, rhs = float((vx * y).sum()), float((x * vty).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gaussian_comparison_trends():
    """The filters approximate exp(-r^2 / 2 sigma^2) (reported, not a parity
    bar).  What the mathematics fixes: iterating the first-order pair K times
    approaches the Gaussian as K grows (central limit), the third-order
    filter approaches it as sigma grows (its variance is 3.10 sigma +
    1.18 sigma^2, so the linear term fades), and the 2-D impulse response of
    the 256 x 128 grid at L = 10 sums to at most 2 pi L^2 (the infinite-grid
    gain), minus what the grid's edges cut off."""
    def err(order, K, sigma, m):
        x = np.zeros(m)
        c = m // 2
        x[c] = 1.0
        h = orc.line(x, sigma, order=order, iters=K, img_factor=0.0)
        g = np.exp(-((np.arange(m) - c) ** 2) / (2 * sigma ** 2))
        return np.abs(h - g).max()
    for sigma in (2.0, 10.0):
        e = [err(1, K, sigma, 301) for K in (1, 5, 10)]
        assert e[0] > e[1] > e[2]
    e3 = [err(3, 1, s, m) for s, m in ((2.0, 301), (10.0, 301), (40.0, 801))]
    assert e3[0] > e3[1] > e3[2]
    ny, nx = 128, 256
    x = np.zeros((ny, nx))
    x[64, 128] = 1.0
    mask = np.ones((ny, nx), np.uint8)
    L = np.full((ny, nx), 10.0)
    for order, K in ((3, 1), (1, 5)):
        total = orc.vh(x, mask, L, L, order=order, iters=K, img_factor=0.0).sum()
        assert 0.99 * 2 * np.pi * 100.0 <= total <= 2 * np.pi * 100.0 * (1 + 1e-12)


# ------------------------------------------------------------- validation
def test_threads_do_not_change_the_result():
    """vh() on several threads (OpenMP over the (variable, level) slices)
    equals the single-thread result bit for bit: every slice is computed
    sequentially and independently."""
    rng = np.random.default_rng(14)
    nx, ny, nz = 37, 23, 5
    mask = (rng.random((ny, nx)) > 0.3).astype(np.uint8)
    L = rng.uniform(1.0, 9.0, (ny, nx))
    x = rng.standard_normal((2, nz, ny, nx))
    a = orc.vh(x, mask, L, L * 0.7, order=3)
    try:
        orc.set_threads(4)
        b = orc.vh(x, mask, L, L * 0.7, order=3)
        c = orc.vh(x, mask, L, L * 0.7, order=1, iters=5, adjoint=True)
    finally:
        orc.set_threads(1)
    assert np.array_equal(a, b)
    assert np.array_equal(c, orc.vh(x, mask, L, L * 0.7, order=1, iters=5, adjoint=True))


def test_invalid_inputs_rejected():
    with pytest.raises(ValueError):
        orc.line(np.ones(5), -1.0)
    with pytest.raises(ValueError):
        orc.line(np.ones(5), np.nan)
    with pytest.raises(ValueError):
        orc.line(np.ones(5), 2.0, order=3, iters=2)
    with pytest.raises(ValueError):
        orc.line(np.ones(5), 2.0, order=1, iters=5, qcorr=True)
    with pytest.raises(ValueError):
        orc.line(np.ones(5), 2.0, coast=3)
    # land points may carry any length scale
    mask = np.array([1, 0, 1, 1, 0], np.uint8)
    sig = np.array([2.0, -5.0, 2.0, 3.0, np.nan])
    orc.line(np.ones(5), sig, mask)
