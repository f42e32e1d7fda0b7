"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle routine to something other than itself: a direct
sum written here with NumPy, a closed form, a hand-computed value, an
invariant between two different routes (EPIC vs correlator + XFFT), or
brute force on tiny inputs.  None needs a GPU.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2411_17804_gb300 import inputs as I


def dft_matrix(n):
    k = np.arange(n)
    return np.exp(2j * np.pi * np.outer(k, k) / n)


def dft2_direct(g):
    """F = W g W^T with W[l][j] = exp(+2 pi i l j / N): the definition."""
    w = dft_matrix(g.shape[0])
    return w @ g @ w.T


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def placed_conj_taps(n, anchors, taps):
    """Aperture illumination g[j] = sum_a conj(w_a[j - anchor_a])."""
    g = np.zeros((n, n), complex)
    k = taps.shape[1]
    for a in range(len(anchors)):
        x0, y0 = anchors[a]
        g[y0:y0 + k, x0:x0 + k] += taps[a, :, :, 0] - 1j * taps[a, :, :, 1]
    return g


def checker(n):
    j = np.arange(n)
    return (-1.0) ** (j[:, None] + j[None, :])


# ---------------------------------------------------------------- FFT pins
@pytest.mark.parametrize("n", [2, 4, 8, 16])
def test_fft2d_matches_direct_and_brute_dft(n):
    rng = np.random.default_rng(n)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    f = O.fft2d(g)
    assert rel(f, dft2_direct(g)) < 1e-12
    assert rel(f, O.dft2d_brute(g)) < 1e-12


@pytest.mark.parametrize("n", [8, 64])
def test_fft1d_closed_forms(n):
    k = np.arange(n)
    for n0 in (0, 1, 3, n - 1):
        x = np.zeros(n, complex)
        x[n0] = 1.0
        assert np.abs(O.fft1d(x) - np.exp(2j * np.pi * n0 * k / n)).max() < 1e-12
    X = O.fft1d(np.ones(n, complex))
    assert abs(X[0] - n) < 1e-12 and np.abs(X[1:]).max() < 1e-12
    # a pure +frequency tone lands in its own bin (sign of the exponent)
    X = O.fft1d(np.exp(-2j * np.pi * 3 * k / n))
    assert abs(X[3] - n) < 1e-10 and np.abs(np.delete(X, 3)).max() < 1e-10


def test_fft2d_parseval_and_axes():
    n = 32
    rng = np.random.default_rng(7)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    f = O.fft2d(g)
    assert abs(np.sum(np.abs(f) ** 2) - n * n * np.sum(np.abs(g) ** 2)) < 1e-9 * np.sum(np.abs(f) ** 2)
    # a tone along x only lands on row ly = 0 (row-major [y][x])
    x = np.arange(n)
    g = np.tile(np.exp(-2j * np.pi * 5 * x / n), (n, 1))
    f = O.fft2d(g)
    assert abs(f[0, 5] - n * n) < 1e-8 and np.abs(f).sum() - abs(f[0, 5]) < 1e-7


# ------------------------------------------------------------- gridding pin
def test_grid_hand_computed():
    n, k = 16, 3
    anchors = np.array([[2, 5]], np.int32)          # window x 2..4, y 5..7
    taps = np.zeros((1, k, k, 2), np.float32)
    taps[0, 0, 1] = (0.5, 0.25)                      # (v=0, u=1) -> cell (y=5, x=3)
    taps[0, 2, 0] = (-1.0, 2.0)                      # (v=2, u=0) -> cell (y=7, x=2)
    e = np.array([3, -4], np.int8)                   # E = 3 - 4i
    g = O.grid(n, anchors, taps, e)
    # conj(0.5 + 0.25i)(3 - 4i) = 0.5 - 2.75i ; conj(-1 + 2i)(3 - 4i) = -11 - 2i
    assert g[5, 3] == pytest.approx(0.5 - 2.75j)
    assert g[7, 2] == pytest.approx(-11 - 2j)
    mask = np.ones((n, n), bool)
    mask[5, 3] = mask[7, 2] = False
    assert np.all(g[mask] == 0)


def test_off_grid_is_rejected():
    anchors = np.array([[14, 3]], np.int32)
    taps = np.ones((1, 3, 3, 2), np.float32)
    volt = np.zeros((1, 1, 1, 1, 2), np.int8)
    with pytest.raises(ValueError):
        O.epic_image(16, anchors, taps, volt)


# --------------------------------------------------------- EPIC chain pins
def _small_station(n_elem=24, diameter=6.0, n=16, k=3, seed=5):
    rng = np.random.default_rng(seed)
    pos = I.disk_layout(n_elem, diameter, 0.6, rng)
    anchors, taps = I.gaussian_kernel(pos, 2.0, 0.5, n, k)
    return pos, anchors, taps


def test_point_source_at_phase_centre_gives_aperture_power_pattern():
    n, T = 16, 5
    pos, anchors, taps = _small_station()
    ne = len(anchors)
    A = np.array([5, -3])
    volt = np.zeros((1, T, 1, ne, 2), np.int8)
    volt[..., 0], volt[..., 1] = A
    img = O.epic_image(n, anchors, taps, volt)[0, 0]
    g = placed_conj_taps(n, anchors, taps)
    pattern = T * (A @ A) * np.abs(dft2_direct(checker(n) * g)) ** 2
    assert rel(img, pattern) < 1e-12
    peak = T * (A @ A) * abs(g.sum()) ** 2                     # closed form
    assert np.unravel_index(np.argmax(img), img.shape) == (n // 2, n // 2)
    assert img[n // 2, n // 2] == pytest.approx(peak, rel=1e-12)


def _on_cell_station(n):
    """Elements exactly on distinct cells with 1 x 1 unit taps."""
    cells = np.array([[x, y] for y in range(n // 4, 3 * n // 4, 2)
                      for x in range(n // 4, 3 * n // 4, 3)], np.int32)
    taps = np.zeros((len(cells), 1, 1, 2), np.float32)
    taps[..., 0] = 1.0
    return cells, taps


@pytest.mark.parametrize("n", [16, 32])
def test_quarter_turn_source_matches_beamformer_everywhere(n):
    """A source on pixel (ly, lx) = (N/2, 3N/4): element phases are quarter
    turns, so the int8 voltages are exact.  EPIC equals the Eq. (BF) power
    at every pixel direction and peaks on that pixel with T (100 N_e)^2."""
    cells, taps = _on_cell_station(n)
    ne, T = len(cells), 3
    jx = cells[:, 0] - n // 2
    e = 100 * (-1j) ** jx                                    # exp(-2 pi i s.r / lambda)
    volt = np.zeros((1, T, 2, ne, 2), np.int8)
    volt[:, :, 0, :, 0], volt[:, :, 0, :, 1] = e.real, e.imag
    ey = 1j * e                                              # Y = i X exactly
    volt[:, :, 1, :, 0], volt[:, :, 1, :, 1] = ey.real, ey.imag
    img = O.epic_image(n, cells, taps, volt)[0]
    # Eq. (intra-station BF) with unit weights at every pixel direction:
    # s.r/lambda = (l - N/2)(j - N/2)/N for r/lambda = (j - N/2) cells of 1/2
    l = np.arange(n) - n // 2
    rel_cells = cells - n // 2
    phase = 2 * np.pi * (np.einsum("x,a->xa", l, rel_cells[:, 0])[None, :, :]
                         + np.einsum("y,a->ya", l, rel_cells[:, 1])[:, None, :]) / n
    bf = np.einsum("yxa,a->yx", np.exp(1j * phase), e)
    assert rel(img[0], T * np.abs(bf) ** 2) < 1e-12
    # (the 2-cell row spacing makes a grating lobe at ly = 0 of equal height)
    assert img[0, n // 2, 3 * n // 4] == pytest.approx(img[0].max(), rel=1e-12)
    assert img[0, n // 2, 3 * n // 4] == pytest.approx(T * (100 * ne) ** 2, rel=1e-12)
    assert img[0, n // 2 + 1, 3 * n // 4] < 0.9 * img[0].max()
    # Y = iX:  YY = XX, X conj(Y) = -i |X|^2
    assert rel(img[1], img[0]) < 1e-12
    assert np.abs(img[2]).max() < 1e-9 * img[0].max()
    assert rel(img[3], -img[0]) < 1e-12


def test_parseval_per_pixel_sum():
    """sum_l XX[l] = N^2 sum_t sum_j |G_X[j]|^2."""
    n = 16
    pos, anchors, taps = _small_station()
    volt = I.random_voltages((1, 4, 1, len(anchors), 2), seed=3).numpy()
    img = O.epic_image(n, anchors, taps, volt)[0, 0]
    tot = sum(np.sum(np.abs(O.grid(n, anchors, taps, volt[0, t, 0])) ** 2) for t in range(4))
    assert img.sum() == pytest.approx(n * n * tot, rel=1e-12)


def test_epic_sums_samples_and_channels_independently():
    n = 16
    pos, anchors, taps = _small_station()
    volt = I.random_voltages((2, 6, 2, len(anchors), 2), seed=9).numpy()
    full = O.epic_image(n, anchors, taps, volt)
    parts = O.epic_image(n, anchors, taps, volt[:, :2]) + O.epic_image(n, anchors, taps, volt[:, 2:])
    assert rel(full, parts) < 1e-13
    assert rel(full[1], O.epic_image(n, anchors, taps, volt[1:])[0]) < 1e-14


# ---------------------------------------------------------- integer paths
def _cplx(v):
    return v[..., 0].astype(np.int64) + 1j * v[..., 1].astype(np.int64)


def test_correlator_brute_force_and_symmetries():
    rng = np.random.default_rng(11)
    volt = rng.integers(-128, 128, (2, 7, 2, 9, 2)).astype(np.int8)
    vis = O.correlate(volt)
    e = volt[..., 0].astype(np.int64), volt[..., 1].astype(np.int64)
    C, T, P, ne, _ = volt.shape
    for c in range(C):
        for a in range(ne):
            for b in range(a + 1):
                for p in range(P):
                    for q in range(P):
                        ar, ai = e[0][c, :, p, a], e[1][c, :, p, a]
                        br, bi = e[0][c, :, q, b], e[1][c, :, q, b]
                        want = (int(np.sum(ar * br + ai * bi)), int(np.sum(ai * br - ar * bi)))
                        assert tuple(vis[c, a * (a + 1) // 2 + b, p, q]) == want
    autos = vis[:, [a * (a + 1) // 2 + a for a in range(ne)]]
    assert np.all(autos[:, :, 0, 0, 1] == 0) and np.all(autos[:, :, 0, 0, 0] >= 0)
    # V^{pq}_{aa} = conj(V^{qp}_{aa})
    assert np.all(autos[:, :, 0, 1, 0] == autos[:, :, 1, 0, 0])
    assert np.all(autos[:, :, 0, 1, 1] == -autos[:, :, 1, 0, 1])


def test_correlator_adversarial_extremes():
    T, ne = 5, 4
    volt = np.full((1, T, 1, ne, 2), -128, np.int8)
    vis = O.correlate(volt)
    assert np.all(vis[..., 0] == T * 2 * 128 * 128) and np.all(vis[..., 1] == 0)
    volt[..., 1] = 127                                        # E = -128 + 127 i
    vis = O.correlate(volt)
    assert np.all(vis[..., 0] == T * (128 * 128 + 127 * 127)) and np.all(vis[..., 1] == 0)


def test_beamformer_brute_force():
    rng = np.random.default_rng(12)
    volt = rng.integers(-128, 128, (2, 2, 3, 2, 5, 2)).astype(np.int8)
    w = rng.integers(-127, 128, (2, 3, 2, 5, 2)).astype(np.int8)
    out = O.beamform(volt, w)
    want = np.einsum("skpa,sctpa->sctkp", np.conj(_cplx(w)), _cplx(volt))
    assert np.array_equal(out[..., 0], want.real.astype(np.int64))
    assert np.array_equal(out[..., 1], want.imag.astype(np.int64))


def test_beamformer_steers_onto_its_direction():
    """Weights built for direction s_k and a plane wave from s_k: every
    element adds in phase, so |B| = sum_a |w_a||E_a| up to rounding."""
    rng = np.random.default_rng(2)
    pos = I.disk_layout(32, 10.0, 0.8, rng)
    dirs = I.beam_directions(4, 2.0, 10.0)
    w = I.bf_weights(pos, 2.0, dirs, 1)
    ph = -2 * np.pi * (dirs[2] @ pos.T) / 2.0
    e = np.stack([np.round(100 * np.cos(ph)), np.round(100 * np.sin(ph))], -1)
    volt = e.astype(np.int8)[None, None, None, None]
    b = O.beamform(volt, w[None])[0, 0, 0, :, 0]
    mag = np.hypot(b[:, 0], b[:, 1])
    assert np.argmax(mag) == 2
    assert mag[2] > 0.99 * 127 * 100 * 32


@pytest.mark.parametrize("x,shift,want,sat", [
    (3, 1, 2, 0), (-3, 1, -2, 0), (2, 1, 1, 0), (1, 1, 1, 0), (-1, 1, -1, 0),
    (5, 2, 1, 0), (6, 2, 2, 0), (-6, 2, -2, 0), (7, 2, 2, 0), (0, 3, 0, 0),
    (1000, 2, 127, 1), (-1000, 2, -127, 1), (127, 0, 127, 0), (128, 0, 127, 1),
    (-128, 0, -127, 1), (508, 2, 127, 0), (510, 2, 127, 1)])
def test_requant_rounds_half_away_and_saturates(x, shift, want, sat):
    out, n = O.requant(np.array([x]), shift)
    assert int(out[0]) == want and n == sat


# ------------------------------------------------------------ XFFT pins
def test_vis_kernel_sum_and_hermitian():
    pos, anchors, taps = _small_station()
    taps = taps.copy()
    taps[..., 1] = 0.1 * np.random.default_rng(4).standard_normal(taps.shape[:-1])
    for a, b in [(0, 0), (3, 1), (1, 3), (5, 2)]:
        kab, base = O.vis_kernel(anchors, taps, a, b)
        t64 = taps.astype(np.float64)
        ga = t64[a, :, :, 0] - 1j * t64[a, :, :, 1]
        gb = t64[b, :, :, 0] - 1j * t64[b, :, :, 1]
        assert kab.sum() == pytest.approx(ga.sum() * np.conj(gb.sum()), rel=1e-12)
        kba, base2 = O.vis_kernel(anchors, taps, b, a)
        assert base2 == (-base[0], -base[1])
        assert np.allclose(kba, np.conj(kab[::-1, ::-1]), atol=1e-15)
    kaa, _ = O.vis_kernel(anchors, taps, 2, 2)
    k = taps.shape[1]
    assert kaa[k - 1, k - 1] == pytest.approx(np.sum(taps[2].astype(np.float64) ** 2), rel=1e-12)


@pytest.mark.parametrize("P,cplx_taps", [(1, False), (2, False), (2, True)])
def test_epic_equals_xfft_of_full_correlation_set(P, cplx_taps):
    """The invariant: the direct-imaged power equals the FFT image of all
    correlations (autos included) gridded with the illumination
    autocorrelation kernel, for every polarisation product."""
    n = 16
    pos, anchors, taps = _small_station()
    if cplx_taps:
        taps = taps.copy()
        taps[..., 1] = 0.2 * np.random.default_rng(8).standard_normal(taps.shape[:-1])
    volt = I.random_voltages((2, 6, P, len(anchors), 2), seed=21).numpy()
    epic = O.epic_image(n, anchors, taps, volt)
    ximg = O.xfft_image(n, anchors, taps, O.correlate(volt))
    assert rel(O.xfft_as_epic_planes(ximg), epic) < 1e-11
    scale = np.abs(ximg).max()
    for p in range(P):
        assert np.abs(ximg[:, p, p].imag).max() < 1e-11 * scale      # autos real
    if P == 2:
        assert np.abs(ximg[:, 1, 0] - np.conj(ximg[:, 0, 1])).max() < 1e-11 * scale


def test_epic_equals_xfft_with_wrapped_lags():
    """Apertures wider than N/2 alias the lag grid; the circular wrap keeps
    the invariant exact."""
    n = 8
    anchors = np.array([[0, 0], [5, 1], [2, 5], [4, 4]], np.int32)
    taps = np.random.default_rng(1).standard_normal((4, 3, 3, 2)).astype(np.float32)
    volt = I.random_voltages((1, 5, 2, 4, 2), seed=2).numpy()
    epic = O.epic_image(n, anchors, taps, volt)
    ximg = O.xfft_image(n, anchors, taps, O.correlate(volt))
    assert rel(O.xfft_as_epic_planes(ximg), epic) < 1e-11


# ---------------------------------------------------------------- inter-station XFFT
def _vis_const(K, C, S, P, value):
    vis = np.zeros((K, C, S * (S + 1) // 2, P, P, 2), np.int64)
    vis[..., 0] = value
    return vis


def test_station_xfft_source_at_phase_centre_closed_form():
    """Visibilities of a source at the phase centre (V = A for every pair):
    all S^2 ordered pairs add at pixel (N/2, N/2), whatever the layout, and
    XX is real and peaks there."""
    rng = np.random.default_rng(4)
    S, n, A = 7, 32, 3
    pos = rng.uniform(-20.0, 20.0, (S, 2))
    img, dropped = O.station_xfft(n, pos, 3.0, 4.0, np.zeros((1, 2)), _vis_const(1, 1, S, 1, A))
    xx = img[0, 0, 0, 0]
    assert dropped == 0
    assert xx[n // 2, n // 2].real == pytest.approx(A * S * S, rel=1e-12)
    assert np.abs(xx.imag).max() < 1e-10 * A * S * S
    assert xx.real.max() == pytest.approx(A * S * S, rel=1e-12)


@pytest.mark.parametrize("shift", [(3, 0), (-2, 5)])
def test_station_xfft_steering_moves_the_source_by_closed_form(shift):
    """Stations on whole cells, V = A (a source at zenith): steering towards
    s_k puts the source at s_src - s_k, i.e. pixel (N/2, N/2) - N cell s_k /
    lambda, with the full peak A S^2 (fixes the sign of the steering phase)."""
    S, n, A, lam, cell = 6, 32, 2, 3.0, 5.0
    rng = np.random.default_rng(9)
    pos = rng.integers(-4, 5, (S, 2)).astype(np.float64) * cell
    px, py = shift
    d = np.array([[px * lam / (n * cell), py * lam / (n * cell)]])
    img, _ = O.station_xfft(n, pos, lam, cell, d, _vis_const(1, 1, S, 1, A))
    xx = img[0, 0, 0, 0].real
    assert xx[n // 2 - py, n // 2 - px] == pytest.approx(A * S * S, rel=1e-12)
    assert np.unravel_index(np.argmax(xx), xx.shape) == (n // 2 - py, n // 2 - px)


def test_station_xfft_bilinear_half_cell_closed_form():
    """Two stations half a cell apart in x: the grid holds 3A at u = 0 and
    A/2 at u = +-1, so every image row is A (3 + cos(2 pi (l - N/2) / N))."""
    n, A = 16, 4
    pos = np.array([[0.0, 0.0], [0.5, 0.0]])
    img, dropped = O.station_xfft(n, pos, 1.0, 1.0, np.zeros((1, 2)), _vis_const(1, 1, 2, 1, A))
    xx = img[0, 0, 0, 0]
    l = np.arange(n)
    want = A * (3 + np.cos(2 * np.pi * (l - n // 2) / n))
    assert dropped == 0
    for row in range(n):
        assert np.allclose(xx[row].real, want, atol=1e-12)
    assert np.abs(xx.imag).max() < 1e-12


def test_station_xfft_offgrid_pairs_brute_force():
    """A pair is dropped when its 2x2 footprint or its mirror's leaves
    [-N/2, N/2 - 1]^2; count by brute force and check the dropped pairs no
    longer contribute (image = image of the kept stations only)."""
    rng = np.random.default_rng(12)
    n, cell = 16, 1.0
    core = rng.uniform(-3.0, 3.0, (5, 2))
    tail = np.array([[40.0, 1.0], [-2.0, 30.0]])
    pos = np.vstack([core, tail])
    S = len(pos)
    want = 0
    for m in range(S):
        for q in range(m):
            ok = True
            for sgn in (1, -1):
                u0 = np.floor(sgn * (pos[m, 0] - pos[q, 0]) / cell)
                v0 = np.floor(sgn * (pos[m, 1] - pos[q, 1]) / cell)
                ok &= (-n // 2 <= u0) and (u0 + 1 <= n // 2 - 1) and (-n // 2 <= v0) and (v0 + 1 <= n // 2 - 1)
            want += not ok
    img, dropped = O.station_xfft(n, pos, 2.0, cell, np.zeros((1, 2)), _vis_const(1, 1, S, 1, 1))
    assert dropped == want
    # every pair with a tail station is off the grid: of the tail only its two
    # autos (value 1 at uv = 0, a constant 1 in the image each) remain
    core_img, _ = O.station_xfft(n, core, 2.0, cell, np.zeros((1, 2)), _vis_const(1, 1, len(core), 1, 1))
    assert dropped == 2 * len(core) + 1
    assert np.allclose(img[0, 0, 0, 0].real, core_img[0, 0, 0, 0].real + 2.0, atol=1e-10)


def test_station_xfft_equals_intra_xfft_with_unit_taps():
    """Stations on whole cells, no steering: the bilinear kernel reduces to a
    single tap, so the inter-station XFFT equals the intra-station XFFT of
    the same visibilities with 1x1 unit taps at the same cells, for every
    polarisation pair (two independently written oracle routines)."""
    rng = np.random.default_rng(5)
    n, S, P, C, cell = 16, 6, 2, 2, 2.0
    cells = np.stack([rng.permutation(6)[:S], rng.permutation(6)[:S]], axis=1) + 4
    pos = cells.astype(np.float64) * cell
    vis = rng.integers(-500, 500, (C, S * (S + 1) // 2, P, P, 2)).astype(np.int64)
    # autos of the auto-pol products are real
    for m in range(S):
        bl = m * (m + 1) // 2 + m
        vis[:, bl, 0, 0, 1] = 0
        vis[:, bl, 1, 1, 1] = 0
        vis[:, bl, 1, 0] = vis[:, bl, 0, 1] * np.array([1, -1])
    st, dropped = O.station_xfft(n, pos, 3.0, cell, np.zeros((1, 2)), vis[None])
    taps = np.zeros((S, 1, 1, 2), np.float32)
    taps[..., 0] = 1.0
    intra = O.xfft_image(n, cells.astype(np.int32), taps, vis)
    assert dropped == 0
    assert np.abs(st[0] - intra).max() < 1e-9 * np.abs(intra).max()


# ---------------------------------------------------------------- FFT correlator
@pytest.mark.parametrize("P,cplx_taps", [(1, False), (2, False), (2, True)])
def test_fft_correlator_recovers_the_gridded_visibilities(P, cplx_taps):
    """The inverse DFT of the accumulated EPIC image is the full correlation
    set gridded with the illumination autocorrelation kernel (the bracket of
    Eq. intra-station XFFT), computed here by the other route: the int64
    correlator and the explicit lag sums."""
    n = 16
    pos, anchors, taps = _small_station()
    if cplx_taps:
        taps = taps.copy()
        taps[..., 1] = 0.3 * np.random.default_rng(9).standard_normal(taps.shape[:-1])
    volt = I.random_voltages((2, 5, P, len(anchors), 2), seed=31).numpy()
    got = O.fft_correlate(O.epic_image(n, anchors, taps, volt))
    want = O.xfft_grid(n, anchors, taps, O.correlate(volt))
    assert rel(got, want) < 1e-11
    # Hermitian: R_ab[-d] = conj(R_ba[d])
    flip = np.roll(np.flip(want, axis=(-2, -1)), 1, axis=(-2, -1))
    assert rel(np.conj(flip), np.swapaxes(want, 1, 2)) < 1e-12


def test_fft_correlator_on_a_lattice_sums_redundant_baselines():
    """Elements on distinct cells with 1 x 1 unit taps: every lag holds the
    plain sum of the visibilities of the pairs separated by it (the FFT
    correlator of redundant arrays), brute-forced pair by pair."""
    n = 16
    cells, taps = _on_cell_station(n)
    ne = len(cells)
    P = 2
    volt = I.random_voltages((1, 4, P, ne, 2), seed=4).numpy()
    e = volt[..., 0].astype(np.int64) + 1j * volt[..., 1].astype(np.int64)   # [C][T][P][ne]
    want = np.zeros((1, P, P, n, n), complex)
    for a in range(ne):
        for b in range(ne):
            d = (cells[a] - cells[b]) % n
            for al in range(P):
                for be in range(P):
                    want[0, al, be, d[1], d[0]] += np.sum(e[0, :, al, a] * np.conj(e[0, :, be, b]))
    got = O.fft_correlate(O.epic_image(n, cells, taps, volt))
    assert rel(got, want) < 1e-12
    assert rel(O.xfft_grid(n, cells, taps, O.correlate(volt)), want) == 0.0


def test_fft_correlate_closed_forms():
    """Normalisation and sign of the inverse transform: a constant XX plane
    is a zero-lag delta of that value; an XY plane exp(+2 pi i o.d0 / n) is a
    delta (-1)^(d0x+d0y) at lag d0 for XY and at -d0 for YX (the
    checkerboard that puts the phase centre at pixel n/2)."""
    n = 8
    planes = np.zeros((1, 4, n, n))
    planes[0, 0] = 3.0
    oy, ox = np.mgrid[0:n, 0:n]
    d0 = (3, 1)
    ph = 2 * np.pi * (ox * d0[0] + oy * d0[1]) / n
    planes[0, 2], planes[0, 3] = np.cos(ph), np.sin(ph)
    g = O.fft_correlate(planes)
    want_xx = np.zeros((n, n), complex)
    want_xx[0, 0] = 3.0
    assert np.abs(g[0, 0, 0] - want_xx).max() < 1e-14
    assert np.abs(g[0, 1, 1]).max() < 1e-14
    want_xy = np.zeros((n, n), complex)
    sgn = (-1.0) ** (d0[0] + d0[1])
    want_xy[d0[1], d0[0]] = sgn
    assert np.abs(g[0, 0, 1] - want_xy).max() < 1e-14
    want_yx = np.zeros((n, n), complex)
    want_yx[(-d0[1]) % n, (-d0[0]) % n] = sgn
    assert np.abs(g[0, 1, 0] - want_yx).max() < 1e-14


# ---------------------------------------------------------------- inter-station EPIC
def _stations_on_cells(n, S, cell, seed, far=0):
    """S stations on distinct whole cells of the central (n/2 - 1)^2 box of
    the grid (every pair's 2 x 2 bilinear footprint stays on the grid), plus
    `far` stations on cells well outside it."""
    rng = np.random.default_rng(seed)
    w = n // 2 - 1
    idx = rng.choice(w * w, S, replace=False)
    cells = np.stack([idx % w, idx // w], axis=1) - n // 4
    pos = cells.astype(np.float64) * cell
    if far:
        pos = np.concatenate([pos, rng.integers(3 * n, 5 * n, (far, 2)) * cell])
    return pos


def _quarter_turn_beams(pos, lam, cell, src, A, T):
    """Station beams of a point source at direction `src` whose phases
    exp(-2 pi i src.r_m / lambda) are whole quarter turns (exact in int8)."""
    turns = (pos @ np.asarray(src, np.float64)) / lam
    q = np.rint(4 * turns).astype(np.int64)
    assert np.allclose(4 * turns, q)
    rot = (-1j) ** (q % 4)                                   # exp(-2 pi i q / 4)
    S, P = len(pos), len(A)
    b = np.zeros((1, 1, T, P, S, 2), np.int8)
    for p in range(P):
        v = A[p] * rot
        b[0, 0, :, p, :, 0] = np.rint(v.real).astype(np.int8)
        b[0, 0, :, p, :, 1] = np.rint(v.imag).astype(np.int8)
    return b


@pytest.mark.parametrize("offset", [(0, 0), (4, 0), (-4, 4)])
def test_station_epic_steered_point_source_closed_form(offset):
    """Beams of a source at s_k + (l - n/2) lambda / (n cell) from stations on
    cells: after the FP64 steering weights every on-grid station adds
    coherently at pixel l, with power T |S_on A|^2 (XX, YY) and
    T S_on^2 A_X conj(A_Y) (XY); far stations are dropped and counted."""
    n, lam, cell, T = 16, 2.0, 2.0, 3
    pos = _stations_on_cells(n, 10, cell, seed=3, far=3)
    s_k = np.array([0.25, 0.5])                      # quarter turns per cell (cell = lambda)
    src = s_k + np.array(offset) * lam / (n * cell)
    A = np.array([3 - 2j, -1 + 4j])
    beams = _quarter_turn_beams(pos, lam, cell, src, A, T)
    img, dropped = O.station_epic(n, pos, lam, cell, s_k[None], beams)
    assert dropped == 3
    S_on = 10
    ly, lx = n // 2 + offset[1], n // 2 + offset[0]
    xx = img[0, 0, 0]
    assert np.unravel_index(np.argmax(xx), xx.shape) == (ly, lx)
    assert xx[ly, lx] == pytest.approx(T * abs(S_on * A[0]) ** 2, rel=1e-6)
    assert img[0, 0, 1, ly, lx] == pytest.approx(T * abs(S_on * A[1]) ** 2, rel=1e-6)
    xy = T * S_on ** 2 * A[0] * np.conj(A[1])
    assert img[0, 0, 2, ly, lx] == pytest.approx(xy.real, rel=1e-6)
    assert img[0, 0, 3, ly, lx] == pytest.approx(xy.imag, rel=1e-6)


def test_station_epic_equals_station_xfft_for_stations_on_cells():
    """The array-level invariant: for stations on whole cells the bilinear
    kernel of the inter-station XFFT is the autocorrelation of the 1-cell
    EPIC kernel, so the two independently written routines give the same
    image, steering included (EPIC weights in FP32, XFFT phases in FP64)."""
    n, lam, cell, T, S = 16, 3.0, 5.0, 4, 9
    pos = _stations_on_cells(n, S, cell, seed=11)
    dirs = np.array([[0.0, 0.0], [0.137, -0.291]])
    rng = np.random.default_rng(12)
    beams = rng.integers(-60, 60, (2, 2, T, 2, S, 2)).astype(np.int8)
    epic, dropped = O.station_epic(n, pos, lam, cell, dirs, beams)
    assert dropped == 0
    vis = np.stack([O.correlate(beams[k]) for k in range(2)])
    ximg, off = O.station_xfft(n, pos, lam, cell, dirs, vis)
    assert off == 0
    for k in range(2):
        assert rel(O.xfft_as_epic_planes(ximg[k]), epic[k]) < 1e-6


# ---------------------------------------------------------------- inter-station XBF
def _hermitian_vis(rng, K, C, S, P, lo=-500, hi=500):
    """Random int64 station visibilities whose autos are what a correlator
    gives: XX, YY real and YX = conj(XY)."""
    vis = rng.integers(lo, hi, (K, C, S * (S + 1) // 2, P, P, 2)).astype(np.int64)
    for m in range(S):
        bl = m * (m + 1) // 2 + m
        for p in range(P):
            vis[..., bl, p, p, 1] = 0
        if P == 2:
            vis[..., bl, 1, 0, 0] = vis[..., bl, 0, 1, 0]
            vis[..., bl, 1, 0, 1] = -vis[..., bl, 0, 1, 1]
    return vis


def test_station_xbf_array_factor_closed_form():
    """Unit visibilities for every pair: the image is |sum_m exp(2 pi i
    sigma . r_m / lambda)|^2, the squared array factor, at every pixel."""
    n, lam, cell, S = 16, 3.0, 7.3, 11
    rng = np.random.default_rng(21)
    pos = rng.uniform(-40.0, 40.0, (S, 2))
    vis = np.zeros((1, 1, S * (S + 1) // 2, 1, 1, 2), np.int64)
    vis[..., 0] = 1
    s_k = np.array([0.021, -0.034])
    img = O.station_xbf(n, pos, lam, cell, s_k[None], vis)[0, 0, 0, 0]
    ly, lx = np.mgrid[0:n, 0:n]
    sx = s_k[0] + (lx - n // 2) * lam / (n * cell)
    sy = s_k[1] + (ly - n // 2) * lam / (n * cell)
    af = np.zeros((n, n), complex)
    for m in range(S):
        af += np.exp(2j * np.pi * (sx * pos[m, 0] + sy * pos[m, 1]) / lam)
    assert np.abs(img - np.abs(af) ** 2).max() < 1e-10 * S * S


def test_station_xbf_equals_station_xfft_on_whole_cells():
    """Stations on whole cells with every pair on the grid: gridding is exact
    and the FFT evaluates the same sum, so XBF (direct DFT) = XFFT, steering
    included, for every polarisation pair."""
    n, lam, cell, S = 16, 3.0, 5.0, 8
    pos = _stations_on_cells(n, S, cell, seed=31)
    dirs = np.array([[0.0, 0.0], [0.11, -0.07]])
    vis = _hermitian_vis(np.random.default_rng(32), 2, 2, S, 2)
    xfft, off = O.station_xfft(n, pos, lam, cell, dirs, vis)
    assert off == 0
    xbf = O.station_xbf(n, pos, lam, cell, dirs, vis)
    assert rel(xbf, xfft) < 1e-10


def test_station_xbf_images_exactly_the_pairs_the_grid_drops():
    """A core and a far tail, all on whole cells: the XFFT image of the kept
    pairs plus the XBF image of the dropped pairs is the XBF image of all
    pairs."""
    n, lam, cell, S = 16, 3.0, 5.0, 9
    pos = _stations_on_cells(n, S - 3, cell, seed=41, far=3)
    dirs = np.array([[0.05, 0.02]])
    vis = _hermitian_vis(np.random.default_rng(42), 1, 2, S, 2)
    xfft, off = O.station_xfft(n, pos, lam, cell, dirs, vis)
    assert off >= 3 * (S - 3)
    part = O.station_xbf(n, pos, lam, cell, dirs, vis, offgrid_only=True)
    full = O.station_xbf(n, pos, lam, cell, dirs, vis)
    assert rel(xfft + part, full) < 1e-10
    assert np.abs(part).max() > 0.1 * np.abs(full).max()
