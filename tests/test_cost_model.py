"""The Table 2 cost model: formulas checked against operation counts of the
algorithms they describe, against the filling factors Table 1 prints, and
against the architecture choices of Table 3 and Section 6."""
import math
import os

import numpy as np
import pytest

from paper_2411_17804_gb300 import cost as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
COLS = {"0.1ms": 1e-4, "1ms": 1e-3, "100ms": 1e-1, "10s": 10.0}


def rows(name):
    out = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].split()
        if line:
            out.append(line)
    return out


# ---------------------------------------------------------------- Table 1
def test_filling_factors_as_printed():
    for name, fa, fs in rows("table1_filling_factors.txt"):
        a = K.ARRAYS[name]
        if name == "CASPA":
            # recorded inconsistency of Table 1: with the printed D_e / lambda =
            # 0.5 the formula gives a quarter of the printed f_s; the printed
            # value is the formula with D_e = lambda
            assert a.f_s == pytest.approx(float(fs) / 4, rel=0.01)
            assert float(f"{K.CASPA_DE1.f_s:.3g}") == pytest.approx(float(fs), rel=1e-9)
        else:
            assert float(f"{a.f_s:.3g}") == pytest.approx(float(fs), rel=1e-9), name
        if name == "LAMBDA-I":
            # the printed f_A is twice N_s (D_s / D_A)^2 with the printed N_s = 4
            assert a.f_A == pytest.approx(float(fa) / 2, rel=0.01)
        else:
            assert a.f_A == pytest.approx(float(fa), rel=0.01), name


# ---------------------------------------------------------------- operation counts
def counted_fft(x, radix, counter):
    """Decimation-in-time FFT (exponent +) whose stages compute every output
    as an r-term sum of twiddled inputs; counts the complex multiply-adds."""
    n = len(x)
    if n == 1:
        return x.copy()
    subs = [counted_fft(x[j::radix], radix, counter) for j in range(radix)]
    m = n // radix
    out = np.zeros(n, complex)
    for k in range(n):
        acc = 0j
        for j in range(radix):
            acc += subs[j][k % m] * np.exp(2j * np.pi * j * k / n)
            counter[0] += 1
        out[k] = acc
    return out


@pytest.mark.parametrize("radix,ratio,gamma", [(2, 4, 2), (4, 8, 2), (2, 8, 1)])
def test_epic_fft_term_counts_a_radix_r_fft(radix, ratio, gamma):
    """8 n_p (r / log2 r) gamma^2 log2(gamma D_s/D_e)^2 per voxel = 8 FLOP per
    CMAC of a 2D radix-r FFT of the (gamma ratio)^2 grid per polarisation,
    over ratio^2 voxels."""
    M = gamma * ratio
    rng = np.random.default_rng(M)
    g = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    cnt = [0]
    rows_ = np.array([counted_fft(r, radix, cnt) for r in g])
    full = np.array([counted_fft(c, radix, cnt) for c in rows_.T]).T
    assert np.allclose(full, np.conj(np.fft.fft2(np.conj(g))))      # it is the DFT (+)
    n_p = 2
    fft = [t for t in K.components("EPIC", 10, ratio, n_p=n_p, gamma=gamma, radix=radix) if t.component == "fft"][0]
    assert fft.flop == pytest.approx(8 * cnt[0] * n_p / ratio ** 2, rel=1e-12)


def test_correlator_and_beamformer_terms_count_their_loops():
    """Correlator: one complex multiply (6) and one add (2) per cross pair
    and polarisation pair per sample, over ratio^2 voxels; beamformer: one
    CMAC per element and input polarisation per output polarisation per
    voxel; XBF DFT: one CMAC per cross pair and polarisation pair per voxel."""
    n, n_p, ratio = 7, 2, 3.0
    mults = sum(1 for a in range(n) for b in range(a) for p in range(n_p) for q in range(n_p))
    terms = {t.component: t.flop for t in K.components("XBF", n, ratio, n_p=n_p)}
    assert terms["correlator"] == pytest.approx(6 * mults / ratio ** 2)
    assert terms["accumulation"] == pytest.approx(2 * mults / ratio ** 2)
    assert terms["dft"] == pytest.approx(8 * mults)
    cmacs = sum(1 for alpha in range(n_p) for a in range(n) for p in range(n_p))
    bf = {t.component: t.flop for t in K.components("BF", n, ratio, n_p=n_p)}
    assert bf["beamforming"] == pytest.approx(8 * cmacs)
    # squaring: every (alpha, beta) product is a complex multiply
    assert bf["squaring"] == 6 * n_p * n_p and bf["accumulation"] == 2 * n_p * n_p


# ---------------------------------------------------------------- Table 3 and Section 6
def test_intra_station_choice_matches_table3_in_every_cell():
    for name, stage, *cells in rows("table3_cadence.txt"):
        if stage != "intra":
            continue
        for col, want in zip(COLS.values(), cells):
            if name == "CASPA":
                # the printed row follows D_e = lambda (see the filling factor)
                assert K.ranking(K.CASPA_DE1, "intra", col)[0][0] == want, (name, col)
                continue
            assert K.ranking(name, "intra", col)[0][0] == want, (name, col)


def test_caspa_as_printed_is_a_recorded_inconsistency():
    """With the printed D_e / lambda = 0.5 the Table 2 formulas move CASPA's
    station-level EPIC / XFFT crossover to about 0.1 ms, so Table 3's EPIC at
    1 ms does not follow from them; with D_e = lambda it does."""
    rank = K.ranking("CASPA", "intra", 1e-3)
    assert rank[0][0] == "XFFT"
    assert K.ranking(K.CASPA_DE1, "intra", 1e-3)[0][0] == "EPIC"
    for arr, lo, hi in ((K.ARRAYS["CASPA"], 3e-5, 3e-4), (K.CASPA_DE1, 1e-3, 10e-3)):
        n, ratio = K.level_args(arr, "intra")
        ts = np.geomspace(1e-5, 1.0, 800)
        diff = [K.density("EPIC", n, ratio, t) - K.density("XFFT", n, ratio, t) for t in ts]
        cross = ts[np.argmax(np.array(diff) > 0)]
        assert lo < cross < hi, (arr.name, cross)


def test_inter_station_choice_is_among_table3_entries():
    for name, stage, *cells in rows("table3_cadence.txt"):
        if stage != "inter":
            continue
        for col, want in zip(COLS.values(), cells):
            rank = K.ranking(name, "inter", col)
            best, cost = rank[0]
            if (name, col) == ("SKA-low-core", 1e-3):
                # Table 3 names EPIC; the printed formulas tie EPIC and XFFT
                d = dict(rank)
                assert abs(d["EPIC"] / d["XFFT"] - 1) < 0.01
                continue
            assert best in want.split("/"), (name, col, rank)


def test_section6_statements():
    # EPIC beats BF inside every station at every cadence
    for name in K.ARRAYS:
        for t in K.CADENCES:
            d = dict(K.ranking(name, "intra", t))
            assert d["EPIC"] < d["BF"]
    # CASPA stations: EPIC below and XFFT above a crossover of a few ms (with
    # D_e = lambda; the printed D_e puts it near 0.1 ms, tested above)
    n, ratio = K.level_args(K.CASPA_DE1, "intra")
    ts = np.geomspace(1e-4, 1.0, 400)
    diff = [K.density("EPIC", n, ratio, t) - K.density("XFFT", n, ratio, t) for t in ts]
    cross = ts[np.argmax(np.array(diff) > 0)]
    assert 1e-3 < cross < 10e-3
    # LAMBDA-I and CASPA between stations: XBF by a large factor at >= 1 ms
    for name in ("LAMBDA-I", "CASPA"):
        rank = K.ranking(name, "inter", 1e-3)
        assert rank[0][0] == "XBF" and rank[1][1] / rank[0][1] > 5


def test_flop_per_cadence_scales():
    """Per-sample terms scale with the samples, per-cadence terms do not."""
    n, ratio = 256, 17.5
    a = K.flop_per_cadence("XFFT", n, ratio, 1, 1000)
    b = K.flop_per_cadence("XFFT", n, ratio, 2, 2000)
    terms = K.components("XFFT", n, ratio)
    per_s = sum(t.flop for t in terms if t.per == "sample") * ratio ** 2
    per_c = sum(t.flop for t in terms if t.per == "cadence") * ratio ** 2
    assert a == pytest.approx(1000 * per_s + per_c)
    assert b == pytest.approx(2 * (2000 * per_s + per_c))
    assert math.isclose(K.flop_per_cadence("EPIC", n, ratio, 3, 10), 30 * K.flop_per_cadence("EPIC", n, ratio, 1, 1))
