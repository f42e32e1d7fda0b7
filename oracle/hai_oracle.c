/*
 * hai_oracle.c -- plain FP64 CPU oracle of the hybrid-imaging hot path of
 * "Comparison of Fast, Hybrid Imaging Architectures for Multi-scale,
 * Hierarchical Aperture Arrays" (Thyagarajan, PASA).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU baseline call these routines; the product library never links, loads
 * or calls them, and they share no code, header or table with it.
 *
 * Every routine writes out the paper's definition as nested loops in IEEE
 * FP64 (built without fast-math).  Integer paths (beamformer, correlator)
 * accumulate in int64.  Readings of the paper that the code fixes:
 *   - DFT of the aperture grid: unnormalised, exponent +2 pi i l.j / N
 *     (Eq. intra-station EPIC, with delta^2 r_j = 1), computed by a textbook
 *     iterative radix-2 Cooley-Tukey FFT (the FFT the cost model of Table 2
 *     counts, radix r = 2).
 *   - phase centre at pixel (N/2, N/2): the grid is multiplied by
 *     (-1)^(jx+jy) before the DFT; images are row-major [l_y][l_x].
 *   - gridding: G[j] = sum_a sum_taps conj(w_a[tap]) E_a with the tap (u, v)
 *     of element a at cell (x0_a + u, y0_a + v)  (Eq. intra-station EPIC).
 *   - squaring and temporal averaging (Eq. intra-station squaring): the sum
 *     over the T samples of F_alpha conj(F_beta) (the mean is that sum / T).
 *   - correlator (Eq. intra-station visibilities): V^{pq}_{ab} =
 *     sum_t E^p_a conj(E^q_b), lower triangle a >= b, packed a(a+1)/2 + b.
 *   - voltage beamformer (Eq. intra-station BF) with diagonal polarisation
 *     weights: B^p_k = sum_a conj(w^p_{k,a}) E^p_a.
 *   - XFFT (Eq. intra-station XFFT): visibilities of all ordered pairs
 *     (autos included) gridded with the autocorrelation of the element
 *     kernels, K_ab[d] = sum_j g_a[j + d] conj(g_b[j]), g_a = placed conj taps,
 *     on the circular N grid, then the same (-1)^d and DFT as EPIC.
 *   - FFT correlator (Section 4.1.2, Section 5.2.2): the inverse DFT of the
 *     accumulated EPIC image planes, normalised by 1/N^2 and multiplied by
 *     (-1)^d, read as gridded visibilities at the lags d (zero lag at cell
 *     (0, 0)).
 *   - inter-station XBF (Eq. inter-station XBF): the direct DFT of the
 *     station visibilities at every pixel, FP64 phase, all pairs or only the
 *     pairs the inter-station XFFT grid drops.
 *   - inter-station XFFT (Eq. inter-station XFFT): station visibilities
 *     phased towards the beam direction with exp(+2 pi i s_k.dr / lambda) in
 *     FP64, gridded with a 2x2 bilinear kernel at uv = dr / cell; pairs whose
 *     footprint leaves the grid are dropped and counted.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OFF_GRID (-2)
#define ORC_ERR_NOMEM (-3)

static const double ORC_TWO_PI = 6.283185307179586476925286766559;

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (timing on one core); n <= 0
 * leaves the count unchanged.  Returns the count in force. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* FFT: textbook iterative radix-2 Cooley-Tukey, X[k] = sum_n x[n] e^{+2 pi i nk/n} */
/* ------------------------------------------------------------------------- */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

int orc_fft1d(int n, double *re, double *im, long stride) {
    if (!is_pow2(n)) return ORC_ERR_ARG;
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = re[i * stride], ti = im[i * stride];
            re[i * stride] = re[j * stride];
            im[i * stride] = im[j * stride];
            re[j * stride] = tr;
            im[j * stride] = ti;
        }
    }
    /* butterflies: stage of length len combines two halves of len/2 */
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; k++) {
            double ang = ORC_TWO_PI * (double)k / (double)len;  /* + sign */
            double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < n; s += len) {
                long p = (long)(s + k) * stride, q = (long)(s + k + half) * stride;
                double xr = re[q] * wr - im[q] * wi;
                double xi = re[q] * wi + im[q] * wr;
                re[q] = re[p] - xr;
                im[q] = im[p] - xi;
                re[p] += xr;
                im[p] += xi;
            }
        }
    }
    return ORC_OK;
}

/* 2D transform of a row-major [n][n] grid: along x (rows), then along y. */
int orc_fft2d(int n, double *re, double *im) {
    if (!is_pow2(n)) return ORC_ERR_ARG;
    for (int y = 0; y < n; y++) orc_fft1d(n, re + (long)y * n, im + (long)y * n, 1);
    for (int x = 0; x < n; x++) orc_fft1d(n, re + x, im + x, n);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Gridding of one (channel, sample, pol) field (Eq. intra-station EPIC).      */
/* e points at [ne][2] int8 (re, im); anchors [ne][2] (x0, y0); taps            */
/* [ne][k][k][2] float indexed [v][u][re,im].                                   */
/* ------------------------------------------------------------------------- */
int orc_check_layout(int n, int ne, int k, const int32_t *anchors) {
    for (int a = 0; a < ne; a++) {
        int x0 = anchors[2 * a], y0 = anchors[2 * a + 1];
        if (x0 < 0 || y0 < 0 || x0 + k > n || y0 + k > n) return ORC_ERR_OFF_GRID;
    }
    return ORC_OK;
}

void orc_grid(int n, int ne, int k, const int32_t *anchors, const float *taps,
              const int8_t *e, double *gre, double *gim) {
    memset(gre, 0, sizeof(double) * n * n);
    memset(gim, 0, sizeof(double) * n * n);
    for (int a = 0; a < ne; a++) {
        double er = e[2 * a], ei = e[2 * a + 1];
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) {
                const float *w = taps + (((long)a * k + v) * k + u) * 2;
                double wr = w[0], wi = w[1];
                long cell = (long)(anchors[2 * a + 1] + v) * n + (anchors[2 * a] + u);
                /* conj(w) * E */
                gre[cell] += wr * er + wi * ei;
                gim[cell] += wr * ei - wi * er;
            }
    }
}

/* multiply by (-1)^(x+y): puts the phase centre at pixel (n/2, n/2) */
static void checkerboard(int n, double *re, double *im) {
    for (int y = 0; y < n; y++)
        for (int x = 0; x < n; x++)
            if ((x + y) & 1) {
                re[(long)y * n + x] = -re[(long)y * n + x];
                im[(long)y * n + x] = -im[(long)y * n + x];
            }
}

/* Electric field image of one field: grid, checkerboard, 2D DFT (+). */
int orc_efield_image(int n, int ne, int k, const int32_t *anchors, const float *taps,
                     const int8_t *e, double *fre, double *fim) {
    if (!is_pow2(n) || n < 4) return ORC_ERR_ARG;
    if (orc_check_layout(n, ne, k, anchors)) return ORC_ERR_OFF_GRID;
    orc_grid(n, ne, k, anchors, taps, e, fre, fim);
    checkerboard(n, fre, fim);
    return orc_fft2d(n, fre, fim);
}

/* ------------------------------------------------------------------------- */
/* EPIC image (Eq. intra-station EPIC + Eq. intra-station squaring).           */
/* volt [C][T][P][ne][2] int8; img [C][Q][n][n] double with Q = 1 (P = 1: XX)   */
/* or Q = 4 (P = 2: XX, YY, Re XY, Im XY), summed over the T samples.          */
/* ------------------------------------------------------------------------- */
int orc_epic_image(int n, int ne, int k, const int32_t *anchors, const float *taps,
                   const int8_t *volt, int C, int T, int P, double *img) {
    if (!is_pow2(n) || n < 4 || ne <= 0 || k <= 0 || C < 0 || T < 0 || (P != 1 && P != 2))
        return ORC_ERR_ARG;
    if (orc_check_layout(n, ne, k, anchors)) return ORC_ERR_OFF_GRID;
    const int Q = (P == 2) ? 4 : 1;
    const long nn = (long)n * n;
    memset(img, 0, sizeof(double) * (size_t)C * Q * nn);
    if (C == 0 || T == 0) return ORC_OK;
    /* work items: (channel, block of samples); partial sums reduced in order */
    int nthr = orc_num_threads();
    int nblk = (C >= 2 * nthr) ? 1 : (2 * nthr + C - 1) / C;
    if (nblk > T) nblk = T;
    int tb = (T + nblk - 1) / nblk;
    double *part = (double *)calloc((size_t)C * nblk * Q * nn, sizeof(double));
    if (!part) return ORC_ERR_NOMEM;
    int nwork = C * nblk;
#pragma omp parallel
    {
        double *fre = (double *)malloc(sizeof(double) * P * nn);
        double *fim = (double *)malloc(sizeof(double) * P * nn);
#pragma omp for schedule(dynamic, 1)
        for (int w = 0; w < nwork; w++) {
            int c = w / nblk, b = w % nblk;
            double *acc = part + (size_t)w * Q * nn;
            for (int t = b * tb; t < T && t < (b + 1) * tb; t++) {
                for (int p = 0; p < P; p++) {
                    const int8_t *e = volt + ((((size_t)c * T + t) * P + p) * ne) * 2;
                    orc_efield_image(n, ne, k, anchors, taps, e, fre + p * nn, fim + p * nn);
                }
                for (long l = 0; l < nn; l++) {
                    double xr = fre[l], xi = fim[l];
                    acc[l] += xr * xr + xi * xi;                 /* XX */
                    if (P == 2) {
                        double yr = fre[nn + l], yi = fim[nn + l];
                        acc[nn + l] += yr * yr + yi * yi;         /* YY */
                        acc[2 * nn + l] += xr * yr + xi * yi;     /* Re X conj(Y) */
                        acc[3 * nn + l] += xi * yr - xr * yi;     /* Im X conj(Y) */
                    }
                }
            }
        }
        free(fre);
        free(fim);
    }
    for (int c = 0; c < C; c++)
        for (int b = 0; b < nblk; b++) {
            const double *src = part + ((size_t)c * nblk + b) * Q * nn;
            double *dst = img + (size_t)c * Q * nn;
            for (long i = 0; i < Q * nn; i++) dst[i] += src[i];
        }
    free(part);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Correlator (Eq. intra-station visibilities): int64 sums over T.             */
/* volt [C][T][P][ne][2]; vis [C][ne(ne+1)/2][P][P][2], bl = a(a+1)/2 + b.     */
/* ------------------------------------------------------------------------- */
int orc_correlate(const int8_t *volt, int C, int T, int ne, int P, int64_t *vis) {
    if (C < 0 || T < 0 || ne <= 0 || P < 1 || P > 2) return ORC_ERR_ARG;
    const long nbl = (long)ne * (ne + 1) / 2;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int c = 0; c < C; c++)
        for (int a = 0; a < ne; a++)
            for (int b = 0; b <= a; b++)
                for (int p = 0; p < P; p++)
                    for (int q = 0; q < P; q++) {
                        int64_t sr = 0, si = 0;
                        for (int t = 0; t < T; t++) {
                            const int8_t *ea = volt + ((((size_t)c * T + t) * P + p) * ne + a) * 2;
                            const int8_t *eb = volt + ((((size_t)c * T + t) * P + q) * ne + b) * 2;
                            int64_t ar = ea[0], ai = ea[1], br = eb[0], bi = eb[1];
                            sr += ar * br + ai * bi;      /* Re E_a conj(E_b) */
                            si += ai * br - ar * bi;      /* Im E_a conj(E_b) */
                        }
                        long bl = (long)a * (a + 1) / 2 + b;
                        int64_t *o = vis + ((((size_t)c * nbl + bl) * P + p) * P + q) * 2;
                        o[0] = sr;
                        o[1] = si;
                    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Voltage beamformer (Eq. intra-station BF), diagonal polarisation weights.   */
/* volt [S][C][T][P][ne][2], w [S][K][P][ne][2], out int64 [S][C][T][K][P][2]. */
/* ------------------------------------------------------------------------- */
int orc_beamform(const int8_t *volt, const int8_t *w, int S, int C, int T, int K,
                 int ne, int P, int64_t *out) {
    if (S < 0 || C < 0 || T < 0 || K <= 0 || ne <= 0 || P < 1 || P > 2) return ORC_ERR_ARG;
#pragma omp parallel for collapse(3) schedule(static)
    for (int s = 0; s < S; s++)
        for (int c = 0; c < C; c++)
            for (int t = 0; t < T; t++)
                for (int kk = 0; kk < K; kk++)
                    for (int p = 0; p < P; p++) {
                        int64_t sr = 0, si = 0;
                        for (int a = 0; a < ne; a++) {
                            const int8_t *e = volt + (((((size_t)s * C + c) * T + t) * P + p) * ne + a) * 2;
                            const int8_t *g = w + ((((size_t)s * K + kk) * P + p) * ne + a) * 2;
                            int64_t er = e[0], ei = e[1], wr = g[0], wi = g[1];
                            sr += wr * er + wi * ei;      /* Re conj(w) E */
                            si += wr * ei - wi * er;      /* Im conj(w) E */
                        }
                        int64_t *o = out + (((((size_t)s * C + c) * T + t) * K + kk) * P + p) * 2;
                        o[0] = sr;
                        o[1] = si;
                    }
    return ORC_OK;
}

/* Requantise one integer to int8: divide by 2^shift rounding half away from
 * zero, then clamp to [-127, 127]; *sat is incremented when clamping bites. */
int8_t orc_requant(int64_t x, int shift, int64_t *sat) {
    int64_t m = x < 0 ? -x : x;
    if (shift > 0) m = (m + ((int64_t)1 << (shift - 1))) >> shift;
    if (m > 127) {
        m = 127;
        if (sat) (*sat)++;
    }
    return (int8_t)(x < 0 ? -m : m);
}

void orc_requant_array(const int64_t *x, long count, int shift, int8_t *out, int64_t *sat) {
    for (long i = 0; i < count; i++) out[i] = orc_requant(x[i], shift, sat);
}

/* ------------------------------------------------------------------------- */
/* XFFT (Eq. intra-station XFFT) from int64 visibilities.                      */
/* img [C][P][P][n][n][2]: full complex image I^{alpha beta} for every pair.   */
/* ------------------------------------------------------------------------- */

/* placed conj taps of element a at absolute cell (x, y), 0 outside the window */
static void placed_conj_tap(int k, const int32_t *anchors, const float *taps, int a,
                            int x, int y, double *gr, double *gi) {
    int u = x - anchors[2 * a], v = y - anchors[2 * a + 1];
    if (u < 0 || v < 0 || u >= k || v >= k) {
        *gr = 0.0;
        *gi = 0.0;
        return;
    }
    const float *w = taps + (((long)a * k + v) * k + u) * 2;
    *gr = w[0];
    *gi = -(double)w[1];
}

/* K_ab[d] = sum_j g_a[j + d] conj(g_b[j]) for the lags d where the two
 * windows overlap: d = (x0_a - x0_b, y0_a - y0_b) + (ex, ey) with ex, ey in
 * [-(k-1), k-1].  kab [(2k-1)][(2k-1)][2] is indexed [ey+k-1][ex+k-1]. */
void orc_vis_kernel(int k, const int32_t *anchors, const float *taps, int a, int b,
                    double *kab) {
    int w2 = 2 * k - 1;
    memset(kab, 0, sizeof(double) * 2 * w2 * w2);
    for (int vb = 0; vb < k; vb++)
        for (int ub = 0; ub < k; ub++) {
            int xb = anchors[2 * b] + ub, yb = anchors[2 * b + 1] + vb;   /* j */
            double br, bi;
            placed_conj_tap(k, anchors, taps, b, xb, yb, &br, &bi);
            for (int va = 0; va < k; va++)
                for (int ua = 0; ua < k; ua++) {
                    int xa = anchors[2 * a] + ua, ya = anchors[2 * a + 1] + va;  /* j + d */
                    double ar, ai;
                    placed_conj_tap(k, anchors, taps, a, xa, ya, &ar, &ai);
                    int ex = ua - ub, ey = va - vb;
                    double *o = kab + ((long)(ey + k - 1) * w2 + (ex + k - 1)) * 2;
                    o[0] += ar * br + ai * bi;    /* g_a conj(g_b) */
                    o[1] += ai * br - ar * bi;
                }
        }
}

/* Gridded visibilities of Eq. intra-station XFFT (the bracket): for every
 * (channel, alpha, beta) the grid sum over all ordered pairs (a, b), autos
 * included, of V^{alpha beta}_{ab} K_ab[d] at the lags d on the circular n
 * grid (cell (d_x mod n, d_y mod n) of a row-major [n][n] grid).
 * grid [C][P][P][n][n][2]. */
int orc_xfft_grid(int n, int ne, int k, const int32_t *anchors, const float *taps,
                  const int64_t *vis, int C, int P, double *grid) {
    if (!is_pow2(n) || n < 4 || ne <= 0 || k <= 0 || C < 0 || P < 1 || P > 2) return ORC_ERR_ARG;
    if (orc_check_layout(n, ne, k, anchors)) return ORC_ERR_OFF_GRID;
    const long nn = (long)n * n, nbl = (long)ne * (ne + 1) / 2;
    const int w2 = 2 * k - 1;
    memset(grid, 0, sizeof(double) * (size_t)C * P * P * nn * 2);
#pragma omp parallel
    {
        double *kab = (double *)malloc(sizeof(double) * 2 * w2 * w2);
#pragma omp for collapse(3) schedule(dynamic, 1)
        for (int c = 0; c < C; c++)
            for (int al = 0; al < P; al++)
                for (int be = 0; be < P; be++) {
                    double *g = grid + ((((size_t)c * P + al) * P + be) * nn) * 2;
                    /* every ordered pair (a, b), autos included */
                    for (int a = 0; a < ne; a++)
                        for (int b = 0; b < ne; b++) {
                            double vr, vi;
                            if (a >= b) {   /* stored: V^{al be}_{ab} */
                                const int64_t *v = vis + ((((size_t)c * nbl + (long)a * (a + 1) / 2 + b) * P + al) * P + be) * 2;
                                vr = (double)v[0];
                                vi = (double)v[1];
                            } else {        /* V^{al be}_{ab} = conj(V^{be al}_{ba}) */
                                const int64_t *v = vis + ((((size_t)c * nbl + (long)b * (b + 1) / 2 + a) * P + be) * P + al) * 2;
                                vr = (double)v[0];
                                vi = -(double)v[1];
                            }
                            orc_vis_kernel(k, anchors, taps, a, b, kab);
                            int dx0 = anchors[2 * a] - anchors[2 * b];
                            int dy0 = anchors[2 * a + 1] - anchors[2 * b + 1];
                            for (int ey = -(k - 1); ey <= k - 1; ey++)
                                for (int ex = -(k - 1); ex <= k - 1; ex++) {
                                    const double *kk = kab + ((long)(ey + k - 1) * w2 + (ex + k - 1)) * 2;
                                    /* lag wrapped onto the circular n grid */
                                    int cx = ((dx0 + ex) % n + n) % n, cy = ((dy0 + ey) % n + n) % n;
                                    long cell = (long)cy * n + cx;
                                    g[2 * cell] += vr * kk[0] - vi * kk[1];
                                    g[2 * cell + 1] += vr * kk[1] + vi * kk[0];
                                }
                        }
                }
        free(kab);
    }
    return ORC_OK;
}

/* Dirty image of Eq. intra-station XFFT: the gridded visibilities, then the
 * same (-1)^d and DFT (+) as EPIC.  img [C][P][P][n][n][2]. */
int orc_xfft_image(int n, int ne, int k, const int32_t *anchors, const float *taps,
                   const int64_t *vis, int C, int P, double *img) {
    int rc = orc_xfft_grid(n, ne, k, anchors, taps, vis, C, P, img);
    if (rc != ORC_OK) return rc;
    const long nn = (long)n * n;
#pragma omp parallel
    {
        double *gr = (double *)malloc(sizeof(double) * nn);
        double *gi = (double *)malloc(sizeof(double) * nn);
#pragma omp for schedule(dynamic, 1)
        for (long pl = 0; pl < (long)C * P * P; pl++) {
            double *o = img + (size_t)pl * nn * 2;
            for (long l = 0; l < nn; l++) {
                gr[l] = o[2 * l];
                gi[l] = o[2 * l + 1];
            }
            checkerboard(n, gr, gi);
            orc_fft2d(n, gr, gi);
            for (long l = 0; l < nn; l++) {
                o[2 * l] = gr[l];
                o[2 * l + 1] = gi[l];
            }
        }
        free(gr);
        free(gi);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* FFT correlator (Section 4.1.2 and Section 5.2.2: visibilities obtained from */
/* accumulated EPIC images by an inverse FFT).  The accumulated image          */
/* I_{alpha beta}[l] = sum_t F_alpha[l] conj(F_beta[l]) is the DFT (+) of the  */
/* circular autocorrelation of the checkerboarded grids (-1)^j G[j], so        */
/* R[d] = (-1)^(dx+dy) (1/n^2) sum_l I[l] exp(-2 pi i l.d / n)                 */
/* returns the gridded visibilities sum_j G_alpha[j+d] conj(G_beta[j]) at lag  */
/* d.  planes [C][Q][n][n] as the EPIC image stores them (Q = 1: XX; Q = 4:    */
/* XX, YY, Re XY, Im XY); I_YX is conj(I_XY) pixel by pixel.                   */
/* grid [C][P][P][n][n][2].                                                    */
/* ------------------------------------------------------------------------- */
int orc_fft_correlate(int n, int C, int P, const double *planes, double *grid) {
    if (!is_pow2(n) || n < 4 || C < 0 || P < 1 || P > 2) return ORC_ERR_ARG;
    const long nn = (long)n * n;
    const int Q = (P == 2) ? 4 : 1;
#pragma omp parallel
    {
        double *gr = (double *)malloc(sizeof(double) * nn);
        double *gi = (double *)malloc(sizeof(double) * nn);
#pragma omp for collapse(3) schedule(dynamic, 1)
        for (int c = 0; c < C; c++)
            for (int al = 0; al < P; al++)
                for (int be = 0; be < P; be++) {
                    const double *pl = planes + (size_t)c * Q * nn;
                    for (long o = 0; o < nn; o++) {
                        double ir, ii;
                        if (al == be) {            /* XX or YY: real */
                            ir = pl[(size_t)al * nn + o];
                            ii = 0.0;
                        } else {                   /* XY, or YX = conj(XY) */
                            ir = pl[2 * nn + o];
                            ii = (al == 0) ? pl[3 * nn + o] : -pl[3 * nn + o];
                        }
                        /* inverse DFT as conj(DFT+(conj(x))) / n^2 */
                        gr[o] = ir;
                        gi[o] = -ii;
                    }
                    orc_fft2d(n, gr, gi);
                    for (long d = 0; d < nn; d++) gi[d] = -gi[d];
                    checkerboard(n, gr, gi);
                    double *g = grid + ((((size_t)c * P + al) * P + be) * nn) * 2;
                    for (long d = 0; d < nn; d++) {
                        g[2 * d] = gr[d] / (double)nn;
                        g[2 * d + 1] = gi[d] / (double)nn;
                    }
                }
        free(gr);
        free(gi);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Inter-station XFFT (Eq. inter-station XFFT) of station visibilities phased  */
/* towards beam directions s_k: every ordered station pair (m, n), autos        */
/* included, contributes V~_mn = V_mn exp(+2 pi i s_k.(r_m - r_n) / lambda)     */
/* (phase in FP64) through the 2x2 bilinear kernel at uv = (r_m - r_n) / cell   */
/* (in cells): weights (1-fu)(1-fv), fu(1-fv), (1-fu)fv, fu fv on the cells     */
/* (u0, v0) .. (u0+1, v0+1), u0 = floor(u), fu = u - u0.  A pair whose 2x2      */
/* footprint, or its mirror's, leaves [-n/2, n/2 - 1]^2 is dropped (counted     */
/* once per unordered pair in *n_offgrid).  Cell (u, v) sits at (u mod n,       */
/* v mod n) of the row-major grid; then (-1)^(u+v) and the DFT (+) as EPIC.     */
/* pos [S][2] m; dir [K][2]; vis int64 [K][C][S(S+1)/2][P][P][2];               */
/* img [K][C][P][P][n][n][2] complex for every polarisation pair.               */
/* ------------------------------------------------------------------------- */
static void bilinear(double u, long *u0, double *fu) {
    double f = floor(u);
    *u0 = (long)f;
    *fu = u - f;
}

static int footprint_on_grid(int n, long u0, long v0) {
    return u0 >= -n / 2 && u0 + 1 <= n / 2 - 1 && v0 >= -n / 2 && v0 + 1 <= n / 2 - 1;
}

int orc_station_xfft(int n, int S, const double *pos, double lambda, double cell, int K, const double *dir,
                     const int64_t *vis, int C, int P, double *img, int64_t *n_offgrid) {
    if (!is_pow2(n) || n < 4 || S <= 0 || K <= 0 || C < 0 || P < 1 || P > 2 || !(lambda > 0) || !(cell > 0))
        return ORC_ERR_ARG;
    const long nn = (long)n * n, nbl = (long)S * (S + 1) / 2;
    /* pairs dropped: the test is geometric, the same for every image */
    int64_t dropped = 0;
    for (int m = 0; m < S; m++)
        for (int q = 0; q < m; q++) {
            long a0, b0, c0, d0;
            double fa, fb, fc, fd;
            bilinear((pos[2 * m] - pos[2 * q]) / cell, &a0, &fa);
            bilinear((pos[2 * m + 1] - pos[2 * q + 1]) / cell, &b0, &fb);
            bilinear((pos[2 * q] - pos[2 * m]) / cell, &c0, &fc);
            bilinear((pos[2 * q + 1] - pos[2 * m + 1]) / cell, &d0, &fd);
            if (!footprint_on_grid(n, a0, b0) || !footprint_on_grid(n, c0, d0)) dropped++;
        }
    if (n_offgrid) *n_offgrid = dropped;
    memset(img, 0, sizeof(double) * (size_t)K * C * P * P * nn * 2);
#pragma omp parallel
    {
        double *gr = (double *)malloc(sizeof(double) * nn);
        double *gi = (double *)malloc(sizeof(double) * nn);
#pragma omp for collapse(4) schedule(dynamic, 1)
        for (int kk = 0; kk < K; kk++)
            for (int c = 0; c < C; c++)
                for (int al = 0; al < P; al++)
                    for (int be = 0; be < P; be++) {
                        memset(gr, 0, sizeof(double) * nn);
                        memset(gi, 0, sizeof(double) * nn);
                        for (int m = 0; m < S; m++)
                            for (int q = 0; q < S; q++) {
                                const double dx = pos[2 * m] - pos[2 * q], dy = pos[2 * m + 1] - pos[2 * q + 1];
                                long u0, v0, mu0, mv0;
                                double fu, fv, mfu, mfv;
                                bilinear(dx / cell, &u0, &fu);
                                bilinear(dy / cell, &v0, &fv);
                                bilinear(-dx / cell, &mu0, &mfu);
                                bilinear(-dy / cell, &mv0, &mfv);
                                if (!footprint_on_grid(n, u0, v0) || !footprint_on_grid(n, mu0, mv0)) continue;
                                double vr, vi;
                                if (m >= q) {      /* stored: V^{al be}_{mq} */
                                    const int64_t *v = vis + (((((size_t)kk * C + c) * nbl + (long)m * (m + 1) / 2 + q) * P + al) * P + be) * 2;
                                    vr = (double)v[0];
                                    vi = (double)v[1];
                                } else {           /* V^{al be}_{mq} = conj(V^{be al}_{qm}) */
                                    const int64_t *v = vis + (((((size_t)kk * C + c) * nbl + (long)q * (q + 1) / 2 + m) * P + be) * P + al) * 2;
                                    vr = (double)v[0];
                                    vi = -(double)v[1];
                                }
                                /* steering towards s_k, FP64 phase */
                                const double ph = ORC_TWO_PI * (dir[2 * kk] * dx + dir[2 * kk + 1] * dy) / lambda;
                                const double cr = cos(ph), ci = sin(ph);
                                const double sr = vr * cr - vi * ci, si = vr * ci + vi * cr;
                                const double w[4] = {(1 - fu) * (1 - fv), fu * (1 - fv), (1 - fu) * fv, fu * fv};
                                for (int t = 0; t < 4; t++) {
                                    const long uu = u0 + (t & 1), vv = v0 + (t >> 1);
                                    const long cx = ((uu % n) + n) % n, cy = ((vv % n) + n) % n;
                                    gr[cy * n + cx] += w[t] * sr;
                                    gi[cy * n + cx] += w[t] * si;
                                }
                            }
                        checkerboard(n, gr, gi);
                        orc_fft2d(n, gr, gi);
                        double *o = img + (((((size_t)kk * C + c) * P + al) * P + be) * nn) * 2;
                        for (long l = 0; l < nn; l++) {
                            o[2 * l] = gr[l];
                            o[2 * l + 1] = gi[l];
                        }
                    }
        free(gr);
        free(gi);
    }
    return ORC_OK;
}

/* Brute-force 2D DFT (O(n^4)), exponent +2 pi i l.j / n, for tiny grids. */
/* ------------------------------------------------------------------------- */
/* Inter-station XBF (Eq. inter-station XBF) with diagonal, unit polarisation  */
/* weights: for every beam k, channel c and polarisation pair (al, be) the     */
/* direct sum over ordered station pairs (m, q), autos once,                   */
/*   I[ly][lx] = sum V^{al be}_{mq} exp(+2 pi i sigma . (r_m - r_q) / lambda), */
/*   sigma = s_k + ((lx - n/2), (ly - n/2)) lambda / (n cell),                 */
/* phase in FP64.  pair_set 0: every pair; 1: only the pairs the              */
/* inter-station XFFT drops (2x2 footprint or its mirror's off the n grid;    */
/* autos are never dropped).  Layouts as orc_station_xfft; img                 */
/* [K][C][P][P][n][n][2].                                                      */
/* ------------------------------------------------------------------------- */
static int pair_dropped(int n, const double *pos, double cell, int m, int q) {
    long a0, b0, c0, d0;
    double fa, fb, fc, fd;
    bilinear((pos[2 * m] - pos[2 * q]) / cell, &a0, &fa);
    bilinear((pos[2 * m + 1] - pos[2 * q + 1]) / cell, &b0, &fb);
    bilinear((pos[2 * q] - pos[2 * m]) / cell, &c0, &fc);
    bilinear((pos[2 * q + 1] - pos[2 * m + 1]) / cell, &d0, &fd);
    return !footprint_on_grid(n, a0, b0) || !footprint_on_grid(n, c0, d0);
}

int orc_station_xbf(int n, int S, const double *pos, double lambda, double cell, int K, const double *dir,
                    const int64_t *vis, int C, int P, int pair_set, double *img) {
    if (!is_pow2(n) || n < 4 || S <= 0 || K <= 0 || C < 0 || P < 1 || P > 2 || !(lambda > 0) || !(cell > 0) ||
        (pair_set != 0 && pair_set != 1))
        return ORC_ERR_ARG;
    const long nn = (long)n * n, nbl = (long)S * (S + 1) / 2;
    memset(img, 0, sizeof(double) * (size_t)K * C * P * P * nn * 2);
#pragma omp parallel for collapse(4) schedule(dynamic, 1)
    for (int kk = 0; kk < K; kk++)
        for (int c = 0; c < C; c++)
            for (int al = 0; al < P; al++)
                for (int be = 0; be < P; be++) {
                    double *o = img + (((((size_t)kk * C + c) * P + al) * P + be) * nn) * 2;
                    for (int m = 0; m < S; m++)
                        for (int q = 0; q < S; q++) {
                            if (m != q && pair_set == 1 && !pair_dropped(n, pos, cell, m, q)) continue;
                            if (m == q && pair_set == 1) continue;
                            double vr, vi;
                            if (m >= q) {      /* stored: V^{al be}_{mq} */
                                const int64_t *v = vis + (((((size_t)kk * C + c) * nbl + (long)m * (m + 1) / 2 + q) * P + al) * P + be) * 2;
                                vr = (double)v[0];
                                vi = (double)v[1];
                            } else {           /* V^{al be}_{mq} = conj(V^{be al}_{qm}) */
                                const int64_t *v = vis + (((((size_t)kk * C + c) * nbl + (long)q * (q + 1) / 2 + m) * P + be) * P + al) * 2;
                                vr = (double)v[0];
                                vi = -(double)v[1];
                            }
                            const double dx = pos[2 * m] - pos[2 * q], dy = pos[2 * m + 1] - pos[2 * q + 1];
                            for (int ly = 0; ly < n; ly++)
                                for (int lx = 0; lx < n; lx++) {
                                    const double sx = dir[2 * kk] + (lx - n / 2) * lambda / (n * cell);
                                    const double sy = dir[2 * kk + 1] + (ly - n / 2) * lambda / (n * cell);
                                    const double ph = ORC_TWO_PI * (sx * dx + sy * dy) / lambda;
                                    const double cr = cos(ph), ci = sin(ph);
                                    o[2 * (ly * n + lx)] += vr * cr - vi * ci;
                                    o[2 * (ly * n + lx) + 1] += vr * ci + vi * cr;
                                }
                        }
                }
    return ORC_OK;
}

void orc_dft2d_brute(int n, const double *re, const double *im, double *ore, double *oim) {
    for (int ly = 0; ly < n; ly++)
        for (int lx = 0; lx < n; lx++) {
            double sr = 0, si = 0;
            for (int jy = 0; jy < n; jy++)
                for (int jx = 0; jx < n; jx++) {
                    double ang = ORC_TWO_PI * (double)((lx * jx + ly * jy) % n) / n;
                    double c = cos(ang), s = sin(ang);
                    double xr = re[jy * n + jx], xi = im[jy * n + jx];
                    sr += xr * c - xi * s;
                    si += xr * s + xi * c;
                }
            ore[ly * n + lx] = sr;
            oim[ly * n + lx] = si;
        }
}
