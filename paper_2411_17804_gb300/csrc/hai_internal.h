// Internal declarations shared by the host API and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/hai.h"

// Device status word bits, set by kernels whose bounded waits give up.
enum : unsigned { HAI_DEV_TIMEOUT = 1u, HAI_DEV_BOUNDS = 2u };

struct hai_ctx {
    int device = 0;
    int num_sms = 0;
    int smem_optin = 0;
    unsigned *d_status = nullptr;   // device status word
    // profiling (hai_profile_enable)
    int prof_on = 0;
    std::vector<cudaEvent_t> prof_ev;   // pairs: [2i] before, [2i+1] after
    size_t prof_used = 0;               // pairs recorded
    long long prof_launches = 0;        // all kernels launched
    void *d_dft[6] = {};                // tensor-core DFT operands: FP16 N = 32, 64, 128; BF16 N = 32, 64, 128
    int capturing = 0;                  // a plan is capturing a graph: no profiling events
    void *d_corr_ws = nullptr;          // correlator: fp16 operand images of a batch of channels,
    size_t corr_ws_bytes = 0;           // allocated on the first hai_correlate call
    // hai_epic_image_host: copy stream and device staging (two voltage and two
    // image chunks), created / grown on first use
    cudaStream_t copy_stream = nullptr;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    size_t dev_bytes = 0;               // other device memory the context holds (status, DFT operands)
};

// Operand workspace of the correlator and the XFFT (allocated on first use by
// hai_workspace; calls that use it on one context run on one stream).
constexpr size_t kCorrWorkspaceBytes = (size_t)512 << 20;
hai_status hai_workspace(hai_ctx *ctx);

// Profiling helpers: prof_begin returns the pair index or -1.
int prof_begin(hai_ctx *ctx, cudaStream_t st);
void prof_end(hai_ctx *ctx, int idx, cudaStream_t st);
inline void prof_count(hai_ctx *ctx, int n) { if (ctx->prof_on) ctx->prof_launches += n; }

// Gather table of the gridding step: for every cell of the kernel's bounding
// box (row-major inside the box) the list of (element, conj tap) pairs.
struct hai_layout {
    hai_ctx *ctx = nullptr;
    int n_elem = 0, grid_n = 0, ksize = 0, n_pol = 0;
    int box[4] = {0, 0, 0, 0};          // x0, y0, x1, y1 (half-open)
    int box_w = 0, box_h = 0;
    int nnz = 0;
    std::vector<int32_t> h_anchors;     // host copy [n_elem][2]
    std::vector<float> h_taps;          // host copy [n_elem][K][K][2]
    int32_t *d_anchors = nullptr;       // [n_elem][2]
    float2 *d_taps = nullptr;           // [n_elem][K][K] as given (not conjugated)
    int32_t *d_cell_start = nullptr;    // [box_w * box_h + 1]
    int32_t *d_entry_elem = nullptr;    // [nnz]
    float2 *d_entry_w = nullptr;        // [nnz] conj(tap)
    float *d_partials = nullptr;        // EPIC time-split partial images
    size_t partial_slots = 0;           // capacity in images of [Q][N][N]
    // tensor-core path: gather table (or, for N = 128, the per-rank blob),
    // its size in shared memory, and the one-station record the kernels read
    void *d_tc_tables = nullptr;
    size_t tc_tables_bytes = 0;         // kept in shared memory by one CTA
    size_t tc_blob_bytes = 0;           // whole device table
    long long tc_entries = 0;           // gather entries one CTA runs per sample step
    int tc_groups = 0;                  // CTAs (N = 128: 4-CTA clusters) resident at once
    // FP32 path of large grids (N >= 128): L2-resident row-transform scratch
    void *d_large_scratch = nullptr;
    size_t large_scratch_bytes = 0;
    void *d_large_cell = nullptr;       // N = 512, at most one entry per cell: int4 {element, conj(W~)} per box cell
    cudaStream_t large_stream = nullptr;   // N = 512: the row pass's stream
    cudaEvent_t large_ev[5] = {};          // rows done (2), columns done (2), fork / join
    void *d_tc_station = nullptr;
    // tensor-core path of large grids (N = 256, 512): DFT operands and the
    // stage scratch of one batch of (channel, sample) pairs
    void *d_big = nullptr;
    void *big_b1[4][2] = {}, *big_b2[4][2] = {};   // [fp16, bf16, fp16 split, bf16 split][hi, lo]
    void *big_a1 = nullptr, *big_a2 = nullptr, *big_slots = nullptr;
    int big_chunk = 0;                  // channels per internal chunk (hai_autotune; 0 = as many as fit)
    void *big_cell = nullptr;           // dense per-cell gather table (at most one entry per cell), or NULL
    size_t big_cell_w_off = 0;          // byte offset of its weights
    long long big_batch = 0;
    cudaStream_t big_stream = nullptr;  // the fixup of batch i beside batch i + 1's gridding and stage 1
    cudaEvent_t big_ev[2] = {};         // stage 2 done, fixup done
    // XFFT: per grid cell the (pair, K_ab value, mirror) entries landing there,
    // built on the first hai_xfft_image call (layout-only data)
    mutable int32_t *d_xcell = nullptr, *d_xent = nullptr;
    mutable float2 *d_xk = nullptr;
    mutable std::mutex xfft_mu;
    mutable size_t dev_bytes = 0;       // device memory the layout holds (guarded by xfft_mu after creation)
};

// ---------------------------------------------------------------- errors
void hai_set_error(const std::string &msg);
hai_status hai_fail(hai_status s, const std::string &msg);
hai_status hai_cuda_fail(cudaError_t e, const char *what);
bool hai_fault_injected(const char *site);   // host-side fault injection

// Let `kern` use the device's whole opt-in dynamic shared memory (less its
// static shared memory).  The value is the same for every call, so callers on
// other host threads launching with other sizes never lower each other's
// limit between their set and their launch; each launch's own size still
// decides its occupancy.
template <typename K>
inline cudaError_t hai_allow_dyn_smem(K kern, int smem_optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin - (int)a.sharedSizeBytes);
}

#define HAI_CUDA_TRY(call)                                         \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return hai_cuda_fail(_e, #call);    \
    } while (0)

// ---------------------------------------------------------------- EPIC split
// The (channel, sample) space is cut into n_cta contiguous ranges of the
// flattened index c * T + t; each CTA sums its range per channel segment into
// a partial image, and epic_reduce adds the partials of each channel in CTA
// order (deterministic).
struct EpicSplit {
    int n_cta = 0;        // CTAs launched
    long long len = 0;    // samples per CTA (last may be shorter)
    int direct = 0;       // 1: one CTA per channel writes img directly
};
EpicSplit epic_make_split(int C, int T, int target_ctas);
size_t epic_partial_slots(int target_ctas);

hai_status epic_fp32_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img,
                            int accumulate, cudaStream_t st);
int epic_fp32_target_ctas(const hai_ctx *ctx, int grid_n);
hai_status epic_tc_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img,
                          int accumulate, cudaStream_t st, int split, int bf16);
bool epic_tc_supported(const hai_layout *L);
// Gather table of a layout for the tensor-core kernel of its grid side;
// shared_bytes = what the kernel keeps in shared memory.
void epic_tc_station_table(int grid_n, int box_w, int box_h, const std::vector<int32_t> &cstart,
                           const std::vector<int32_t> &elem, const std::vector<float2> &w,
                           std::vector<uint8_t> &out, int &ntile, int &nent, uint32_t &shared_bytes,
                           long long &entries);
hai_status epic_reduce_launch(const hai_layout *L, const EpicSplit &sp, int C, int T, float *img,
                              int accumulate, cudaStream_t st);
// FP32 EPIC for N = 128, 256, 512 (row FFTs to a scratch, then column FFTs,
// squaring and accumulation).
bool epic_large_supported(int grid_n);
size_t epic_large_scratch_bytes(int grid_n, int box_h);
hai_status epic_large_prepare(hai_layout *L);   // constant tables in the scratch's tail
hai_status epic_large_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                             cudaStream_t st);
// Tensor-core EPIC for N = 256, 512 (box <= N/2, box height <= 128), FP16 or
// BF16 operands, plain or split: gridding, stage-1 GEMM and stage-2 GEMM +
// squaring through an HBM scratch.
bool epic_big_supported(const hai_layout *L);
void vis_layout_dims(const hai_vis_layout *L, int *S, int *N, int *K);   // stations, grid side, directions
bool epic_big_used(const hai_layout *L, hai_precision prec);   // this precision runs on the large-grid kernels
hai_status epic_big_prepare(hai_layout *L);
hai_status epic_big_launch(const hai_layout *L, const int8_t *volt, int C, int T, float *img, int accumulate,
                           hai_precision prec, cudaStream_t st);

// ---------------------------------------------------------------- station pairs
// The inter-station XFFT keeps a pair when the 2x2 bilinear footprint of its
// uv = (r_m - r_n) / cell and of its mirror -uv both lie in [-N/2, N/2 - 1]^2
// (du, dv in cells, FP64); the XBF images the pairs it drops.
inline bool station_pair_kept(int N, double du, double dv) {
    auto on_grid = [&](double u, double v) {
        const double a = floor(u), b = floor(v);
        return a >= -N / 2 && a + 1 <= N / 2 - 1 && b >= -N / 2 && b + 1 <= N / 2 - 1;
    };
    return on_grid(du, dv) && on_grid(-du, -dv);
}

