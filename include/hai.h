/*
 * hai.h -- C ABI of the GB300 hybrid aperture-array imaging library (libhai.so).
 *
 * The library implements the data-parallel hot path of the hybrid imaging
 * architectures of Thyagarajan, "Comparison of Fast, Hybrid Imaging
 * Architectures for Multi-scale, Hierarchical Aperture Arrays" (PASA):
 *   - the generic FFT direct imager (EPIC): gridding of element voltages with
 *     an illumination kernel, a 2D spatial DFT per (channel, sample, pol),
 *     squaring (polarisation outer product) and accumulation over the cadence
 *     (Section 5.2, Eq. intra-station EPIC + Eq. intra-station squaring);
 *   - the comparison paths: the int8 correlator (Eq. intra-station
 *     visibilities), the correlator + FFT imager (Eq. intra-station XFFT) and
 *     the pre-correlation voltage beamformer (Eq. intra-station BF);
 *   - the inter-station stage of a hierarchical array: station beams to the
 *     correlator layout, the FP64-steered XFFT (Eq. inter-station XFFT) and
 *     the coherent EPIC over stations (Eq. inter-station EPIC);
 *   - the FFT correlator: visibilities from accumulated EPIC images.
 *
 * Conventions shared by every entry point
 *   - Every function returns hai_status; HAI_OK is 0.  On failure nothing is
 *     launched and hai_last_error() returns a message (thread-local).
 *   - Data buffers are owned by the caller and are DEVICE pointers (for
 *     example torch tensors' data_ptr()) on the context's device, unless a
 *     parameter says "host".  Voltage buffers are at least 2-byte aligned
 *     (one complex int8 value), float buffers 4-byte aligned; an entry point
 *     that needs more says so (HAI_ERR_INVALID_ARG otherwise).  Opaque objects (context, layout) are owned by
 *     the library and released with their destroy function.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is asynchronous on that stream; errors of the kernels
 *     themselves surface at hai_sync() or at the next CUDA call.
 *   - The compute entry points allocate no memory: scratch space is reserved
 *     when the context or layout is created.
 *   - Complex values are interleaved (re, im).  int8 voltages hold any value
 *     in [-128, 127].
 *   - Image planes: for P = 1 input polarisation one plane (XX); for P = 2
 *     four planes XX, YY, Re XY, Im XY with XY = sum_t F_X conj(F_Y) (YX is
 *     conj(XY) and not stored).  Images are row-major [l_y][l_x] with the
 *     phase centre at pixel (N/2, N/2); pixel l looks along direction cosines
 *     s = (l - N/2) / (N * cell), cell in wavelengths.  The temporal
 *     "average" of the paper is returned as the SUM over the T samples.
 */
#ifndef HAI_H
#define HAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HAI_OK = 0,
    HAI_ERR_INVALID_ARG = 1,   /* a size, pointer or enum is out of range  */
    HAI_ERR_OFF_GRID = 2,      /* a gridding kernel tap falls off the grid */
    HAI_ERR_OVERFLOW_RISK = 3, /* int32 accumulation could overflow        */
    HAI_ERR_UNSUPPORTED = 4,   /* valid request this build does not cover  */
    HAI_ERR_CUDA = 5,          /* a CUDA runtime call failed               */
    HAI_ERR_TIMEOUT = 6,       /* a bounded device wait gave up            */
    HAI_ERR_NO_MEMORY = 7      /* allocation at create time failed         */
} hai_status;

typedef enum {
    HAI_PREC_FP32 = 0,       /* FP32 FFT on CUDA cores                              */
    HAI_PREC_FP16 = 1,       /* FP16 DFT-as-GEMM on tcgen05 tensor cores, FP32 acc.  */
    HAI_PREC_FP16_SPLIT = 2, /* as FP16 with every operand split into hi + lo fp16
                                parts and the products hi*hi + hi*lo + lo*hi:
                                ~FP32 accuracy at 3x the tensor work              */
    HAI_PREC_BF16 = 3,       /* BF16 DFT-as-GEMM (8-bit mantissa: ~8x the FP16
                                error), FP32 accumulation                         */
    HAI_PREC_BF16_SPLIT = 4  /* as BF16 with hi + lo bf16 parts (three products)  */
} hai_precision;

typedef struct hai_ctx hai_ctx;
typedef struct hai_layout hai_layout;

/* Library version as major * 10000 + minor * 100 + patch. */
int hai_version(void);

/* Message of the last failed call on this thread ("" if none). */
const char *hai_last_error(void);

/* Name of a status code. */
const char *hai_status_string(hai_status s);

/* Create a context on CUDA device `device` (makes it current on this thread).
 * Reserves the device status word used by bounded device-side waits. */
hai_status hai_create(int device, hai_ctx **out);
void hai_destroy(hai_ctx *ctx);

/* Wait for `stream`, then report kernel faults: HAI_ERR_CUDA for a CUDA
 * error, HAI_ERR_TIMEOUT if a bounded device wait gave up since the last
 * call (the status word is cleared). */
hai_status hai_sync(hai_ctx *ctx, void *stream);

/* Self-check of the bounded device waits (no counterpart in the paper: it
 * tests the library's failure detection).  Every pipelined kernel waits on
 * mbarrier phases through one bounded wait that, when a phase never
 * completes, gives up, sets HAI_DEV_TIMEOUT in the context's status word and
 * lets the kernel end instead of hanging.  This call launches one CTA on
 * `stream` that waits on a phase nothing will complete (no copy or MMA is in
 * flight), with a limit of `limit_cycles` SM cycles in [1024, 2^24] (else
 * HAI_ERR_INVALID_ARG): the wait gives up within microseconds, the next
 * hai_sync returns HAI_ERR_TIMEOUT and clears the word, and the context stays
 * usable.  hai_check_device_wait_result (after a sync) returns 1 in *gave_up
 * if the wait gave up, 0 if it saw the phase complete. */
hai_status hai_check_device_wait(hai_ctx *ctx, long long limit_cycles, void *stream);
hai_status hai_check_device_wait_result(hai_ctx *ctx, int *gave_up);

/* Peak-rate probe (no counterpart in the paper: a measurement aid for the
 * roofline fractions).  Launches on `stream` one kernel of 4 CTAs x 256
 * threads per SM, every thread running independent dependency chains of
 * `iters` (1 .. 2^24) steps of:
 *   kind 0  scalar FP32 fused multiply-add (2 FLOP each),
 *   kind 1  packed FP32 fused multiply-add on pairs, FFMA2 (4 FLOP each),
 *   kind 2  warp-level int8 MMA, mma.sync m16n8k32 s8 x s8 + s32 (8,192
 *           integer operations each).
 * *ops (host) receives the operation count of the launch; time it with
 * events on `stream`.  HAI_ERR_INVALID_ARG for another kind or iters. */
hai_status hai_probe_peak(hai_ctx *ctx, int kind, long long iters, double *ops, void *stream);

/* Profiling.  While enabled, every compute call records a pair of CUDA events
 * on the caller's stream around its dominant kernel (the first kernels it
 * launches are the one named in the call's description) and counts every
 * kernel it launches.  Enabling creates an event pool of `max_records`
 * pairs; further calls are counted but not timed. */
hai_status hai_profile_enable(hai_ctx *ctx, int enable, int max_records);

/* Synchronise the recorded events and return the summed duration (ms) of the
 * timed dominant-kernel launches, their count, and the count of all kernels
 * launched since the last read; then reset. */
hai_status hai_profile_read(hai_ctx *ctx, double *dominant_ms, long long *dominant_launches,
                            long long *total_launches);

/* ---------------------------------------------------------------------------
 * Station layout and gridding kernel (Eq. intra-station EPIC, the bracket:
 * G[j] = sum_a conj(W~_a(r_j - r_a)) E_a).
 * The illumination kernel W~ is an input: every element a carries an anchor
 * cell (x0, y0) and ksize x ksize complex taps; tap (u, v) weights cell
 * (x0 + u, y0 + v) of the N x N grid whose cell (N/2, N/2) holds the station
 * origin.  The taps are used conjugated, as the equation states.
 * ------------------------------------------------------------------------- */
typedef struct {
    int n_elem;              /* N_e > 0                                       */
    int grid_n;              /* N: power of two, 16..512                       */
    int ksize;               /* K >= 1                                        */
    int n_pol;               /* P: 1 or 2                                     */
    const int32_t *anchors;  /* host [n_elem][2] (x0, y0), copied             */
    const float *taps;       /* host [n_elem][K][K][2] indexed [v][u][re,im]   */
} hai_layout_desc;

/* Copy the layout in and reserve its scratch.  HAI_ERR_OFF_GRID if any tap
 * cell lies outside [0, N)^2; HAI_ERR_UNSUPPORTED for a grid size this build
 * has no kernel for. */
hai_status hai_layout_create(hai_ctx *ctx, const hai_layout_desc *desc, hai_layout **out);
void hai_layout_destroy(hai_layout *layout);

/* A layout from element positions with the library's default illumination
 * kernel (the paper leaves W~ to the user; Section 5.2): element a at
 * g = pos_m[a] / (lambda_m cell_lambda) + N/2 cells (FP64) gets the K x K cells
 * around its nearest cell floor(g + 1/2) (anchor = that cell - (K - 1) / 2 per
 * axis) with real taps exp(-|cell - g|^2 / (2 sigma_cells^2)) normalised to
 * unit sum.  Then as hai_layout_create (HAI_ERR_OFF_GRID if a tap leaves the
 * grid).  hai_layout_anchors returns the anchors and taps a layout uses. */
typedef struct {
    int n_elem;              /* N_e > 0                                       */
    const double *pos_m;     /* host [n_elem][2] (x, y) metres, station frame  */
    double lambda_m;         /* wavelength                                    */
    double cell_lambda;      /* grid cell in wavelengths                      */
    int grid_n;              /* N                                             */
    int ksize;               /* K, 1 .. 15                                    */
    double sigma_cells;      /* Gaussian width in cells (> 0)                 */
    int n_pol;               /* P: 1 or 2                                     */
} hai_position_desc;
hai_status hai_layout_create_from_positions(hai_ctx *ctx, const hai_position_desc *desc, hai_layout **out);

/* The layout's anchors (host int32 [n_elem][2]) and taps (host float
 * [n_elem][K][K][2], as given, not conjugated); either may be NULL. */
hai_status hai_layout_anchors(const hai_layout *layout, int32_t *anchors, float *taps);

/* Device memory held by a layout (gather tables, partial images, the scratch
 * of its tensor-core and large-grid paths, the XFFT lists once built; an
 * N = 512 layout holds two 1 GB row scratches of the FP32 path) or by a
 * context (status words, DFT operands, and the correlator workspace and host
 * staging once first used); bytes on the host. */
hai_status hai_layout_workspace_size(const hai_layout *layout, size_t *bytes);
hai_status hai_ctx_workspace_size(const hai_ctx *ctx, size_t *bytes);

/* Bounding box of the cells the kernel touches, host int[4] = (x0, y0, x1, y1)
 * half-open. */
hai_status hai_layout_box(const hai_layout *layout, int *box);

/* ---------------------------------------------------------------------------
 * EPIC image: for every channel c the sum over samples t of the polarisation
 * outer product of the synthesised fields F_{c,t,p}[l] =
 * sum_j (-1)^(jx+jy) G_{c,t,p}[j] exp(+2 pi i l.j / N)
 * (Eq. intra-station EPIC, then Eq. intra-station squaring with the temporal
 * average taken as a sum).
 *   volt  device int8 [C][T][P][N_e][2]
 *   img   device float [C][Q][N][N], Q = 1 (P = 1) or 4 (P = 2); overwritten
 *         (accumulate = 0) or added to (accumulate = 1)
 *   prec  HAI_PREC_FP32 (CUDA-core FFT; N = 16 .. 512), or a tensor-core
 *         precision (HAI_PREC_FP16, _BF16, _FP16_SPLIT, _BF16_SPLIT; N = 32,
 *         64, 128, 256 or 512, P = 2 and a kernel box of at most N/2 x N/2
 *         cells, for N >= 256 at most 128 cells high, else
 *         HAI_ERR_UNSUPPORTED).  At N = 128 the split precisions run on the
 *         large-grid kernels (the layout then holds their 64 MB scratch).
 * C >= 0, T >= 0 (C = 0 or T = 0: nothing to image; with accumulate = 0 the
 * image is zeroed).  A layout's scratch (partial images, the large-grid batch
 * and row scratches, and at N = 512 the FP32 path's second stream, joined to
 * `stream` by events) serves one call at a time: calls with the same layout
 * must be ordered on the device (one stream, or events between streams);
 * calls with different layouts may overlap. */
hai_status hai_epic_image(hai_ctx *ctx, const hai_layout *layout, const int8_t *volt,
                          int C, int T, hai_precision prec, float *img, int accumulate,
                          void *stream);

/* Autotuner of hai_epic_image's large-grid tensor-core path (N = 256, 512,
 * and the hi/lo split at N = 128): the
 * channels imaged per internal chunk, which sets how many samples of each
 * channel one pass of the stage scratch holds (longer sample blocks mean
 * fewer image read-modify-writes, fewer stage-2 items shared between CTAs,
 * but fewer items per pass).  Candidates 1, 2, 4, ... up to min(C, 16)
 * channels are timed on a synthetic cadence of min(C, 16) channels x
 * min(T, 1024) samples of the layout (random voltages, device memory
 * allocated for the trial and freed), and the fastest is kept in the layout
 * for later calls; *chosen (may be NULL) receives it, or 0 when there is
 * nothing to tune (FP32, a grid side below 128, or plain operands at 128).
 * cache_path (may be NULL): a text file of "<key> | chunk <c> | <time>"
 * lines, key = device, N, K, P, N_e bucket (floor log2) and precision; a
 * matching line is applied without timing, a new choice is appended.  Not
 * for use while other work runs on the device (it times kernels). */
hai_status hai_autotune(hai_ctx *ctx, hai_layout *layout, int C, int T, hai_precision prec, const char *cache_path,
                        int *chosen);

/* hai_epic_image on HOST buffers, the channels streamed through the GPU in
 * chunks so that the copies overlap the imaging: chunk k is imaged on
 * `stream` while the context's copy stream moves chunk k+1's voltages in and
 * chunk k-1's images out (two device staging buffers of each, owned by the
 * context, grown on first use).
 *   volt   host int8 [C][T][P][N_e][2]; img host float [C][Q][N][N]
 *          (overwritten, or added to with accumulate = 1: then the host
 *          image is copied in as well).  Page-locked (pinned) host memory is
 *          needed for the copies to overlap; pageable memory works but the
 *          copies then serialise.
 *   chunk  channels per chunk, 1..C (0: C/4 rounded up); the first two
 *          chunks take a quarter and a half of it, to start imaging early
 * Same precisions, limits and errors as hai_epic_image.  Asynchronous like
 * it: synchronise `stream` before reading img.  The staging buffers belong to
 * the context: calls issued one after another (from one host thread) are
 * ordered through the context's copy stream, even on different caller
 * streams, but calls on one context from two host threads at once race. */
hai_status hai_epic_image_host(hai_ctx *ctx, const hai_layout *layout, const int8_t *volt, int C, int T,
                               hai_precision prec, float *img, int accumulate, int chunk, void *stream);

/* ---------------------------------------------------------------------------
 * Batched EPIC over an array of stations of uneven size (the heterogeneous
 * stations the paper's hierarchical arrays allow, Section 2): the EPIC image
 * of every station (as hai_epic_image with HAI_PREC_FP16) for one cadence of
 * C channels x T samples, run as ONE CUDA-graph launch per cadence.  The
 * plan groups the stations by grid side, gives every group a share of the
 * SMs (a persistent tensor-core kernel per group, all groups concurrent) and
 * cuts each group's (station, channel) blocks into per-CTA ranges of equal
 * modelled cost; hai_plan_autotune refits the shares from measured times.
 *
 * hai_plan_create: `stations` = S layouts (host array of pointers) of this
 * context, each with P = 2, grid side 32, 64 or 128 and a kernel box of at
 * most N/2 x N/2 (else HAI_ERR_UNSUPPORTED); prec must be HAI_PREC_FP16.
 * The plan copies what it needs: the layouts may be destroyed afterwards.
 * Device memory for tables and schedules is reserved here, none at run time.
 */
typedef struct hai_plan hai_plan;
hai_status hai_plan_create(hai_ctx *ctx, const hai_layout *const *stations, int S, int C, int T,
                           hai_precision prec, hai_plan **out);
void hai_plan_destroy(hai_plan *plan);

/* Buffer layout of the plan (host outputs; pass NULL for any not wanted):
 *   volt_off[S]  byte offset of station s's voltages [C][T][2][N_e,s][2]
 *                int8 inside the one voltage buffer; every block starts on
 *                16 bytes and has at least 16 unused bytes before and after
 *                it (the kernels read 16-byte aligned spans that may cover
 *                them; their content is ignored)
 *   img_off[S]   float offset of station s's images [C][4][N_s][N_s]
 *   volt_bytes   size of the voltage buffer;  img_floats  size of the image buffer */
hai_status hai_plan_layout(const hai_plan *plan, int64_t *volt_off, int64_t *img_off, int64_t *volt_bytes,
                           int64_t *img_floats);

/* Image one cadence: volt (device, volt_bytes, 16-byte aligned) -> img
 * (device, img_floats, 16-byte aligned, overwritten).  The first call with a
 * given (volt, img) pair captures the graph (allocating host-side graph
 * objects); later calls with the same pair only launch it on `stream`. */
hai_status hai_plan_run(hai_plan *plan, const int8_t *volt, float *img, void *stream);

/* Autotuner: `rounds` times, run every grid group alone on its current SM
 * share (twice, timing the second run with events on `stream`), then
 * re-divide the SMs so that the groups' measured SM-time is balanced.  Runs
 * the kernels on (volt, img), overwriting img.  Synchronises the stream. */
hai_status hai_plan_autotune(hai_plan *plan, const int8_t *volt, float *img, int rounds, void *stream);

/* hai_plan_autotune with a cache: cache_path is a text file of
 * "<key> | units <u_0> ... | <time>" lines, key = device, C, T and per grid
 * class its side, station count and modelled cost.  A matching line (the
 * last one) sets the classes' shares (CTAs, clusters at N = 128) without
 * timing and *from_cache (may be NULL) is set to 1; otherwise the plan is
 * autotuned as hai_plan_autotune does and a line is appended. */
hai_status hai_plan_autotune_cached(hai_plan *plan, const int8_t *volt, float *img, int rounds, const char *cache_path,
                                    int *from_cache, void *stream);

/* Device memory the plan holds (its copies of the gather tables, station
 * records and per-CTA ranges), bytes on the host.  The run itself allocates
 * nothing. */
hai_status hai_workspace_size(const hai_plan *plan, size_t *bytes);

/* Schedule of the plan (host outputs, arrays of length *n_class <= 3):
 * grid side, CTAs and last measured time alone (ms, 0 before autotuning) of
 * every grid group. */
hai_status hai_plan_schedule(const hai_plan *plan, int *n_class, int *grid_n, int *ctas, double *measured_ms);

/* Second level of the hierarchy in the same graph launch (Section 6, the
 * two-stage architectures: station-synthesised fields imaged between
 * stations).  Set once per plan; hai_plan_run_hier then runs, as ONE graph
 * launch per cadence, the station EPIC images of hai_plan_run and after them
 *   1. K voltage beams of every station (Eq. intra-station BF, diagonal pol:
 *      B^p_{s,k} = sum_a conj(w^p_{s,k,a}) E^p_{s,a}; exact int32 sums, then
 *      |x| / 2^shift rounded half away from zero and clamped to 127, as
 *      hai_beamform's requantised output),
 *   2. their inter-station order (hai_beams_to_corr),
 *   3. the inter-station correlator + XFFT dirty image of every beam (Eq.
 *      inter-station visibilities and XFFT; hai_correlate with the K*C
 *      (beam, channel) pairs as channels, then hai_xfft_station_image) when
 *      `xfft` is set, and/or
 *   4. the inter-station EPIC image of every beam (Eq. inter-station EPIC:
 *      hai_epic_image of beam k's block with epic[k], a layout from
 *      hai_station_epic_layout_create) when `epic` is set. */
typedef struct hai_vis_layout hai_vis_layout;   /* declared with its functions below */
typedef struct {
    int n_beam;                     /* K, 1..64 */
    const int8_t *weights;          /* device int8: station s's weights [K][2][N_e,s][2]
                                       start at byte weight_off[s] (even) */
    const int64_t *weight_off;      /* host [S] */
    int requant_shift;              /* 0..30 */
    const hai_vis_layout *xfft;     /* S stations, K directions; or NULL */
    const hai_layout *const *epic;  /* host array of K layouts (S elements, 2 pols); or NULL */
    hai_precision epic_prec;        /* precision of the inter-station EPIC */
} hai_plan_hier_desc;
/* The plan re-packs the weights into its own device memory (the caller's
 * buffer may be freed after the call, which synchronises the device) and
 * keeps the layouts (not copies): they must outlive the plan or the next
 * hai_plan_set_hierarchy.  At least one of xfft and epic;
 * HAI_ERR_UNSUPPORTED if 4 K (S + 1) bytes exceed 48 KB. */
hai_status hai_plan_set_hierarchy(hai_plan *plan, const hai_plan_hier_desc *desc);

/* Sizes of the second level's buffers (host outputs, NULL for any not
 * wanted): beams and their reorder, bytes each; visibilities, int32 count;
 * the XFFT and EPIC images, float counts (0 when that stage is not set). */
hai_status hai_plan_hier_sizes(const hai_plan *plan, int64_t *beam_bytes, int64_t *vis_ints, int64_t *xfft_floats,
                               int64_t *epic_floats);

/* Device buffers of the second level, owned by the caller, 16-byte aligned:
 *   beams     int8 [S][C][T][K][2][2] (station beams, hai_beamform's layout)
 *   corr      int8 [K][C][T][2][S][2] (their inter-station order)
 *   vis       int32 [K][C][S(S+1)/2][2][2][2] (with xfft; else may be NULL)
 *   xfft_img  float [K][C][4][N_A][N_A] (with xfft; else may be NULL)
 *   epic_img  float: beam k's images [C][4][N_k][N_k] one after another
 *             (with epic; else may be NULL)
 *   n_saturated  device int64 count of clamped beam components (or NULL) */
typedef struct {
    int8_t *beams;
    int8_t *corr;
    int32_t *vis;
    float *xfft_img;
    float *epic_img;
    long long *n_saturated;
} hai_plan_hier_buffers;
/* As hai_plan_run, plus the second level into `buffers`; the graph is
 * captured again when any pointer changes. */
hai_status hai_plan_run_hier(hai_plan *plan, const int8_t *volt, float *img, const hai_plan_hier_buffers *buffers,
                             void *stream);

/* ---------------------------------------------------------------------------
 * Correlator (Eq. intra-station visibilities): for every element pair a >= b
 * (autos included) and polarisation pair (p, q),
 *   V^{pq}_{ab} = sum_t E^p_a(t) conj(E^q_b(t)).
 *   volt  device int8 [C][T][P][N][2] (the EPIC input layout), N elements
 *   vis   device int32 [C][N(N+1)/2][P][P][2], baseline index a(a+1)/2 + b;
 *         overwritten (accumulate = 0) or added to (accumulate = 1)
 * Results are exact: tensor-core products of the int8 values are summed in
 * FP32 over blocks of at most 512 samples (every partial sum is an integer
 * below 2^24) and the blocks in int32.  V^{qp}_{ba} = conj(V^{pq}_{ab}) gives
 * the upper triangle.  HAI_ERR_OVERFLOW_RISK if T > 65535 (|V| could exceed
 * 2^31 - 1); HAI_ERR_UNSUPPORTED if N > 65535.  vis must be 8-byte aligned and volt
 * 2-byte aligned (one complex int8 value).
 * The fp16 operands are staged in the context's 512 MB workspace (allocated
 * by the first call), so calls on one context must not run concurrently on
 * different streams. */
hai_status hai_correlate(hai_ctx *ctx, const int8_t *volt, int C, int T, int N, int P,
                         int32_t *vis, int accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * Correlator + FFT image (Eq. intra-station XFFT): the visibilities of every
 * ordered element pair (a, b), autos included, gridded with the
 * autocorrelation of the two elements' illumination kernels,
 *   K_ab[d] = sum_j g_a[j + d] conj(g_b[j]),  g = the layout's placed conj taps,
 * on the circular N x N grid, multiplied by (-1)^(dx+dy) and transformed with
 * exp(+2 pi i l.d / N).  With this kernel the result equals the EPIC image
 * of the same voltages (same planes and pixel convention as hai_epic_image).
 *   vis   device int32 [C][N_e(N_e+1)/2][P][P][2] as written by hai_correlate
 *   img   device float [C][Q][N][N]; overwritten or added to (accumulate)
 * The pair (b, a) is the Hermitian mirror of the stored (a, b).  FP32 grid and
 * FFT; each grid cell sums its contributions in a fixed order, so results are
 * deterministic.  The first call for a layout builds on the host, and copies
 * to the device (synchronously), the per-cell list of K_ab contributions
 * (layout-only data, freed with the layout; HAI_ERR_UNSUPPORTED beyond 2e8
 * entries, i.e. N_e(N_e+1)(2K-1)^2 > 2e8); the channels are staged through
 * the context's operand workspace, so calls on one context must not run
 * concurrently on different streams.  N = 16, 32 or 64. */
hai_status hai_xfft_image(hai_ctx *ctx, const hai_layout *layout, const int32_t *vis, int C,
                          float *img, int accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * FFT correlator (Section 4.1.2 and Section 5.2.2: visibilities from the
 * accumulated EPIC images by an inverse FFT).  For every channel and
 * polarisation pair (alpha, beta)
 *   R_ab[d] = (-1)^(dx+dy) / N^2  sum_l I_ab[l] exp(-2 pi i l.d / N),
 * which for an image written by hai_epic_image is the gridded visibility set
 * sum_t sum_j G_alpha[j + d] conj(G_beta[j]) = sum over ordered element pairs
 * of V^{alpha beta}_{ab} K_ab[d] (the bracket of Eq. intra-station XFFT); on
 * a lattice with one unit tap per element each lag is the sum of the
 * visibilities of the baselines separated by it.
 *   img   device float [C][Q][N][N] as hai_epic_image writes it (Q = 1: XX;
 *         Q = 4: XX, YY, Re XY, Im XY), 4-byte aligned; read only
 *   grid  device float complex [C][P][P][N][N][2], 8-byte aligned; lag d at
 *         cell (dx mod N, dy mod N) of the row-major plane (zero lag at
 *         (0, 0)); overwritten.  YX is conj(XY) mirrored.
 * N a power of two in [16, 512] (else HAI_ERR_UNSUPPORTED).  FP32 radix-2
 * transforms; no scratch memory. */
hai_status hai_fft_correlate(hai_ctx *ctx, const float *img, int C, int N, int P, float *grid, void *stream);

/* ---------------------------------------------------------------------------
 * Voltage beamformer (Eq. intra-station BF) with diagonal polarisation
 * weights: for every station s, channel c, sample t, beam k and pol p,
 *   B^p_k = sum_a conj(w^p_{s,k,a}) E^p_{s,a}(c, t).
 *   volt   device int8 [S][C][T][P][N][2], 16-byte aligned
 *   w      device int8 [S][K][P][N][2]
 *   beams  16-byte aligned; requant_shift < 0: device int32
 *          [S][C][T][K][P][2], exact; requant_shift >= 0: device int8, same
 *          layout, each component
 *          divided by 2^shift rounding half away from zero and clamped to
 *          [-127, 127]
 *   n_saturated  device int64 counter (or NULL), incremented by the number of
 *          clamped components
 * Exact for N <= 512 (products summed in FP32 stay integers below 2^24).
 * HAI_ERR_UNSUPPORTED unless N is a multiple of 8 and <= 512 and K a multiple
 * of 8 and <= 64, or if one station's weights do not fit in shared memory. */
hai_status hai_beamform(hai_ctx *ctx, const int8_t *volt, const int8_t *w, int S, int C, int T, int K,
                        int N, int P, int requant_shift, void *beams, long long *n_saturated,
                        void *stream);

/* ---------------------------------------------------------------------------
 * Inter-station stage of a hierarchical array (Section 6).
 *
 * hai_beams_to_corr: station beams -> correlator input, so that hai_correlate
 * with the K*C (beam, channel) pairs as channels and the S stations as
 * elements gives the inter-station visibilities of Eq. inter-station
 * visibilities, V^{pq}_{mn}(s_k) = sum_t E^p_m(s_k) conj(E^q_n(s_k)).
 *   beams  device int8 [S][C][T][K][P][2] (hai_beamform's requantised output)
 *   out    device int8 [K][C][T][P][S][2]
 * HAI_ERR_UNSUPPORTED if 2 K P (S + 1) bytes exceed 48 KB. */
hai_status hai_beams_to_corr(hai_ctx *ctx, const int8_t *beams, int S, int C, int T, int K, int P, int8_t *out,
                             void *stream);

/* Station array for the inter-station XFFT (copied in; FP64 geometry). */
typedef struct {
    int n_station;       /* S */
    const double *pos_m; /* host [S][2] station centres, metres */
    double lambda_m;     /* wavelength */
    double cell_m;       /* uv cell of the array grid, metres */
    int grid_n;          /* N: power of two, 16..256 */
    int n_pol;           /* must be 2 */
    int n_dir;           /* K beam directions */
    const double *dir;   /* host [K][2] direction cosines s_k, or NULL (all zenith) */
} hai_vis_layout_desc;
typedef struct hai_vis_layout hai_vis_layout;

/* Build the gridding records (FP64 on the host: the 2x2 bilinear footprint of
 * every station pair at uv = (r_m - r_n) / cell and of its mirror) and the
 * steering phasors exp(+2 pi i s_k.(r_m - r_n) / lambda), computed in FP64 on
 * the GPU and stored in FP32.  Pairs whose footprint, or its mirror's, leaves
 * [-N/2, N/2 - 1]^2 are dropped (hai_vis_layout_offgrid counts them).
 * HAI_ERR_UNSUPPORTED if the uv window of the kept pairs does not fit in
 * shared memory or n_pol != 2. */
hai_status hai_vis_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *desc, hai_vis_layout **out);
void hai_vis_layout_destroy(hai_vis_layout *layout);
/* Station pairs (unordered, autos never) dropped off the grid, per image. */
hai_status hai_vis_layout_offgrid(const hai_vis_layout *layout, long long *n_offgrid);

/* Dirty images of Eq. inter-station XFFT: for every beam k and channel c,
 * all ordered station pairs (autos included) of the visibilities, phased
 * towards s_k, gridded bilinearly, (-1)^(u+v) and a 2D DFT (exponent +).
 *   vis  device int32 [K][C][S(S+1)/2][2][2][2] (hai_correlate's output for
 *        the K*C channels of hai_beams_to_corr).  As from a correlator, the
 *        autos must have real XX and YY and YX = conj(XY): the XX and YY
 *        images are real and are computed together as one complex FFT.
 *   img  device float [K][C][4][N][N]: XX, YY, Re XY, Im XY (overwritten; the
 *        planes also serve as the gridding scratch)
 * Phase centre at pixel (N/2, N/2); pixel l looks along s_k + (l - N/2) *
 * lambda / (N cell). */
hai_status hai_xfft_station_image(hai_ctx *ctx, const hai_vis_layout *layout, const int32_t *vis, int C, float *img,
                                  void *stream);

/* ---------------------------------------------------------------------------
 * Inter-station EPIC (Eq. inter-station EPIC, then the squaring and temporal
 * sum of Eq. inter-station squaring) runs on hai_epic_image with a layout in
 * which the stations are the elements: for beam direction s_k = dir[k],
 * station m sits on its nearest cell of the array grid,
 *   j_m = floor(r_m / cell + N/2 + 1/2)  (per axis),
 * with one tap (N_ks = 1 cell) W~_m such that conj(W~_m) = exp(+2 pi i
 * s_k . r_m / lambda): the phase is taken in FP64 on the host, reduced to a
 * fraction of a turn, and stored in FP32.  The padding factor 2 per
 * dimension (Section 5.2.2) gives the array the central half of the grid: a
 * station whose cell falls outside [N/4, 3N/4)^2 is dropped (weight 0,
 * counted in *n_dropped when non-NULL); the kept stations' box then fits
 * N/2, so the tensor-core kernels take N = 32, 64, 128.  The
 * voltages are the station beams of direction k in the layout [C][T][P][S][2],
 * i.e. block k of hai_beams_to_corr's output.  Phase centre at pixel
 * (N/2, N/2); pixel l looks along s_k + (l - N/2) lambda / (N cell).
 *   desc  as for hai_vis_layout_create (grid_n: any size hai_layout_create
 *         takes; n_pol 1 or 2); k in [0, max(1, n_dir))
 * Release with hai_layout_destroy. */
hai_status hai_station_epic_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *desc, int k, hai_layout **out,
                                          long long *n_dropped);

/* ---------------------------------------------------------------------------
 * Inter-station correlator beamforming (Eq. inter-station XBF) with diagonal,
 * unit polarisation weights: for beam k, channel c and polarisation pair
 * (a, b), at the same pixels as hai_xfft_station_image (pixel l looks along
 * s_k + (l - N/2) lambda / (N cell)),
 *   I[l] = sum over ordered station pairs (m, n) of the set, autos once, of
 *          V^{ab}_{mn} exp(+2 pi i sigma_l . (r_m - r_n) / lambda),
 * evaluated directly (no gridding).  Pair sets:
 *   HAI_XBF_ALL_PAIRS      every pair and every auto;
 *   HAI_XBF_OFFGRID_PAIRS  only the pairs the inter-station XFFT drops (its
 *                          2x2 footprint or its mirror's off the N grid), so
 *                          that hai_xfft_station_image followed by this call
 *                          with accumulate = 1 images every pair.
 * The layout holds the geometry phases exp(+2 pi i (l - N/2).(r_m - r_n) /
 * (N cell)) of every pair and pixel (FP64 phase on the GPU, fp16 storage:
 * 4 N^2 bytes per pair, 1.45 GB for 5,515 pairs at N = 256) and a coefficient
 * buffer for up to n_dir * max_channels images; hai_xbf_layout_info reports
 * the pair count and these bytes.  HAI_ERR_NO_MEMORY if they do not fit.
 * desc as for hai_vis_layout_create (n_pol 2; grid_n a power of two in
 * 16..512).  prec: HAI_PREC_FP16 (fp16 operands) or HAI_PREC_FP16_SPLIT (every
 * operand as fp16 hi + lo parts, products hi*hi + hi*lo + lo*hi: FP32-level
 * accuracy, three times the work and phase memory). */
enum { HAI_XBF_ALL_PAIRS = 0, HAI_XBF_OFFGRID_PAIRS = 1 };
typedef struct hai_xbf_layout hai_xbf_layout;
hai_status hai_xbf_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *desc, int pair_set, int max_channels,
                                 hai_precision prec, hai_xbf_layout **out);
void hai_xbf_layout_destroy(hai_xbf_layout *layout);
hai_status hai_xbf_layout_info(const hai_xbf_layout *layout, long long *n_pairs, long long *device_bytes);

/* Images of the layout's pair set.
 *   vis  device int32 [K][C][S(S+1)/2][2][2][2] (hai_correlate's output for
 *        the K*C channels of hai_beams_to_corr); C <= max_channels
 *   img  device float [K][C][4][N][N]: XX, YY, Re XY, Im XY, 16-byte aligned;
 *        overwritten (accumulate = 0) or added to (accumulate = 1)
 * One tcgen05 GEMM, img[rows][pixels] = A x Phi^T, fp16 operands and FP32
 * accumulation: the per-image coefficients A (from V and the FP64 steering
 * phasor exp(+2 pi i s_k . (r_m - r_n) / lambda)) are scaled by a power of two
 * per image to keep them in fp16 range, which the epilogue undoes. */
hai_status hai_xbf_station_image(hai_ctx *ctx, const hai_xbf_layout *layout, const int32_t *vis, int C, float *img,
                                 int accumulate, void *stream);

/* ---------------------------------------------------------------------------
 * EPIC image, FP32 path, without any device allocation.  (The paper has no
 * counterpart: this is an interface for callers, not a step of the method.)
 *
 * Some callers cannot call cudaMalloc: a plug-in whose host application owns
 * and hands out all device memory, a real-time loop whose device budget is
 * fixed before it starts, or a thread that must not make allocating CUDA
 * calls while another thread captures a CUDA graph in global mode.  They
 * cannot create a hai_layout (hai_layout_create allocates its gather table
 * and scratch), so this entry point takes the layout description on the
 * host and keeps the gather table and the time-split partial images in one
 * file-scope static device array of 9.2 MiB (2,408,452 floats) that every
 * GPU loading the library holds until the process exits.  It computes the
 * same image as hai_epic_image with HAI_PREC_FP32 (up to FP32 rounding of a
 * different time split).
 *   device  CUDA device index; made current
 *   desc    host layout description as for hai_layout_create (read only)
 *   volt    device int8 [C][T][P][N_e][2];  img  device float [C][Q][N][N]
 * Limits: grid_n 16, 32 or 64 and n_elem * ksize^2 <= 102400, else
 * HAI_ERR_UNSUPPORTED; taps off the grid give HAI_ERR_OFF_GRID.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Every call shares the array and a static host
 * staging buffer: calls that overlap on the GPU, or run from two host
 * threads at once, race.  The table is copied in on `stream` from pageable
 * host memory, so the call returns only once the runtime has staged that
 * copy (the host blocks for it).  No context is needed. */
hai_status hai_epic_image_fp32_static(int device, const hai_layout_desc *desc, const int8_t *volt,
                                      int C, int T, float *img, int accumulate, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HAI_H */
