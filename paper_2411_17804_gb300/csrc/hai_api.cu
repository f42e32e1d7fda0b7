// Host side of the C ABI: contexts, layouts, argument checks, dispatch.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "epic_tc.cuh"
#include "hai_internal.h"
#include "tc.cuh"

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void hai_set_error(const std::string &msg) { g_last_error = msg; }

hai_status hai_fail(hai_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

hai_status hai_cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return HAI_ERR_CUDA;
}

// HAI_FAULT is a comma-separated list of sites ("alloc", "launch", "timeout")
// at which the host wrapper reports a failure without touching the GPU.
bool hai_fault_injected(const char *site) {
    const char *env = getenv("HAI_FAULT");
    if (!env || !*env) return false;
    std::string s(env);
    size_t pos = 0;
    while (pos <= s.size()) {
        size_t e = s.find(',', pos);
        if (e == std::string::npos) e = s.size();
        if (s.compare(pos, e - pos, site) == 0) return true;
        pos = e + 1;
    }
    return false;
}

extern "C" int hai_version(void) { return 100; }

extern "C" const char *hai_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *hai_status_string(hai_status s) {
    switch (s) {
        case HAI_OK: return "HAI_OK";
        case HAI_ERR_INVALID_ARG: return "HAI_ERR_INVALID_ARG";
        case HAI_ERR_OFF_GRID: return "HAI_ERR_OFF_GRID";
        case HAI_ERR_OVERFLOW_RISK: return "HAI_ERR_OVERFLOW_RISK";
        case HAI_ERR_UNSUPPORTED: return "HAI_ERR_UNSUPPORTED";
        case HAI_ERR_CUDA: return "HAI_ERR_CUDA";
        case HAI_ERR_TIMEOUT: return "HAI_ERR_TIMEOUT";
        case HAI_ERR_NO_MEMORY: return "HAI_ERR_NO_MEMORY";
    }
    return "HAI_ERR_UNKNOWN";
}

// ------------------------------------------------------------------ context
hai_status epic_fp32_init_tables(void);

extern "C" hai_status hai_create(int device, hai_ctx **out) {
    if (!out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_create: out is NULL");
    *out = nullptr;
    if (hai_fault_injected("alloc")) return hai_fail(HAI_ERR_NO_MEMORY, "hai_create: injected allocation failure");
    int ndev = 0;
    HAI_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return hai_fail(HAI_ERR_INVALID_ARG, "hai_create: no such device");
    HAI_CUDA_TRY(cudaSetDevice(device));
    hai_ctx *c = new hai_ctx();
    c->device = device;
    cudaError_t e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    // word 0: the status word; word 1: outcome of the wait self-check; word 2:
    // sink of the peak-rate probes
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, 4 * sizeof(unsigned));
    if (e == cudaSuccess) c->dev_bytes += 4 * sizeof(unsigned);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 4 * sizeof(unsigned));
    if (e != cudaSuccess) {
        if (c->d_status) cudaFree(c->d_status);
        delete c;
        return hai_cuda_fail(e, "hai_create");
    }
    hai_status s = epic_fp32_init_tables();
    if (s != HAI_OK) {
        cudaFree(c->d_status);
        delete c;
        return s;
    }
    *out = c;
    return HAI_OK;
}

hai_status hai_workspace(hai_ctx *ctx) {
    if (ctx->d_corr_ws) return HAI_OK;
    HAI_CUDA_TRY(cudaMalloc(&ctx->d_corr_ws, kCorrWorkspaceBytes));
    ctx->corr_ws_bytes = kCorrWorkspaceBytes;
    return HAI_OK;
}

static void prof_release(hai_ctx *ctx) {
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    ctx->prof_used = 0;
}

extern "C" void hai_destroy(hai_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    prof_release(ctx);
    cudaFree(ctx->d_status);
    cudaFree(ctx->d_corr_ws);
    for (void *d : ctx->d_dft) cudaFree(d);
    cudaFree(ctx->d_stage);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    delete ctx;
}

extern "C" hai_status hai_profile_enable(hai_ctx *ctx, int enable, int max_records) {
    if (!ctx || max_records < 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_profile_enable: bad argument");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    prof_release(ctx);
    ctx->prof_on = enable ? 1 : 0;
    ctx->prof_launches = 0;
    if (enable) {
        ctx->prof_ev.resize(2 * (size_t)max_records);
        for (size_t i = 0; i < ctx->prof_ev.size(); i++) {
            cudaError_t e = cudaEventCreate(&ctx->prof_ev[i]);
            if (e != cudaSuccess) {
                ctx->prof_ev.resize(i);
                prof_release(ctx);
                ctx->prof_on = 0;
                return hai_cuda_fail(e, "hai_profile_enable");
            }
        }
    }
    return HAI_OK;
}

int prof_begin(hai_ctx *ctx, cudaStream_t st) {
    if (!ctx->prof_on || ctx->capturing || 2 * (ctx->prof_used + 1) > ctx->prof_ev.size()) return -1;
    int idx = (int)ctx->prof_used++;
    cudaEventRecord(ctx->prof_ev[2 * idx], st);
    return idx;
}

void prof_end(hai_ctx *ctx, int idx, cudaStream_t st) {
    if (idx >= 0) cudaEventRecord(ctx->prof_ev[2 * idx + 1], st);
}

extern "C" hai_status hai_profile_read(hai_ctx *ctx, double *ms, long long *n_dom, long long *n_all) {
    if (!ctx || !ms || !n_dom || !n_all) return hai_fail(HAI_ERR_INVALID_ARG, "hai_profile_read: NULL argument");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    double tot = 0.0;
    for (size_t i = 0; i < ctx->prof_used; i++) {
        HAI_CUDA_TRY(cudaEventSynchronize(ctx->prof_ev[2 * i + 1]));
        float e = 0.f;
        HAI_CUDA_TRY(cudaEventElapsedTime(&e, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
        tot += e;
    }
    *ms = tot;
    *n_dom = (long long)ctx->prof_used;
    *n_all = ctx->prof_launches;
    ctx->prof_used = 0;
    ctx->prof_launches = 0;
    return HAI_OK;
}

extern "C" hai_status hai_sync(hai_ctx *ctx, void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_sync: ctx is NULL");
    if (hai_fault_injected("timeout")) return hai_fail(HAI_ERR_TIMEOUT, "hai_sync: injected device timeout");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    HAI_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned st = 0;
    HAI_CUDA_TRY(cudaMemcpy(&st, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st) {
        HAI_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(unsigned)));
        if (st & HAI_DEV_TIMEOUT) return hai_fail(HAI_ERR_TIMEOUT, "a bounded device wait gave up");
        return hai_fail(HAI_ERR_CUDA, "a device-side bounds check fired");
    }
    return HAI_OK;
}

// ------------------------------------------------------------------ wait self-check
// One CTA: thread 0 sets up an mbarrier expecting one arrival that never
// comes (no copy or MMA is issued) and waits on its first phase through the
// same bounded wait every pipelined kernel uses, with a short limit.  The wait
// gives up, flags HAI_DEV_TIMEOUT in the status word and the kernel returns.
__global__ void wait_selfcheck_kernel(unsigned *status, long long limit, int *gave_up) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) *gave_up = tc::mbar_wait(&bar, 0u, status, limit) ? 0 : 1;
    __syncthreads();
}

extern "C" hai_status hai_check_device_wait(hai_ctx *ctx, long long limit_cycles, void *stream) {
    if (!ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_check_device_wait: ctx is NULL");
    if (limit_cycles < 1024 || limit_cycles > (1ll << 24))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_check_device_wait: limit must be in [1024, 2^24] cycles");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    // the wait's outcome goes to the word after the status word
    wait_selfcheck_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(ctx->d_status, limit_cycles,
                                                              reinterpret_cast<int *>(ctx->d_status + 1));
    prof_count(ctx, 1);
    HAI_CUDA_TRY(cudaGetLastError());
    return HAI_OK;
}

extern "C" hai_status hai_check_device_wait_result(hai_ctx *ctx, int *gave_up) {
    if (!ctx || !gave_up) return hai_fail(HAI_ERR_INVALID_ARG, "hai_check_device_wait_result: NULL argument");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    HAI_CUDA_TRY(cudaMemcpy(gave_up, ctx->d_status + 1, sizeof(int), cudaMemcpyDeviceToHost));
    return HAI_OK;
}

// ------------------------------------------------------------------ layout
static bool grid_supported(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || n == 256 || n == 512; }

static void layout_free(hai_layout *L) {
    if (!L) return;
    cudaFree(L->d_anchors);
    cudaFree(L->d_taps);
    cudaFree(L->d_cell_start);
    cudaFree(L->d_entry_elem);
    cudaFree(L->d_entry_w);
    cudaFree(L->d_partials);
    cudaFree(L->d_tc_tables);
    cudaFree(L->d_tc_station);
    cudaFree(L->d_large_scratch);
    cudaFree(L->d_large_cell);
    if (L->large_stream) cudaStreamDestroy(L->large_stream);
    for (cudaEvent_t ev : L->large_ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(L->d_big);
    if (L->big_stream) cudaStreamDestroy(L->big_stream);
    for (cudaEvent_t ev : L->big_ev)
        if (ev) cudaEventDestroy(ev);
    cudaFree(L->d_xcell);
    cudaFree(L->d_xent);
    cudaFree(L->d_xk);
    delete L;
}

extern "C" hai_status hai_layout_create(hai_ctx *ctx, const hai_layout_desc *d, hai_layout **out) {
    if (!ctx || !d || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_create: NULL argument");
    *out = nullptr;
    if (d->n_elem <= 0 || d->ksize <= 0 || d->grid_n <= 0 || (d->n_pol != 1 && d->n_pol != 2) ||
        !d->anchors || !d->taps)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_create: bad descriptor");
    if ((d->grid_n & (d->grid_n - 1)) != 0)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_create: grid_n must be a power of two");
    if (!grid_supported(d->grid_n))
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_layout_create: grid_n not supported by this build");
    const int n = d->grid_n, k = d->ksize, ne = d->n_elem;
    int bx0 = n, by0 = n, bx1 = 0, by1 = 0;
    for (int a = 0; a < ne; a++) {
        int x0 = d->anchors[2 * a], y0 = d->anchors[2 * a + 1];
        if (x0 < 0 || y0 < 0 || (long)x0 + k > n || (long)y0 + k > n)
            return hai_fail(HAI_ERR_OFF_GRID, "hai_layout_create: element " + std::to_string(a) +
                                                  " has taps outside the grid");
        bx0 = std::min(bx0, x0);
        by0 = std::min(by0, y0);
        bx1 = std::max(bx1, x0 + k);
        by1 = std::max(by1, y0 + k);
    }
    if (hai_fault_injected("alloc")) return hai_fail(HAI_ERR_NO_MEMORY, "hai_layout_create: injected allocation failure");

    hai_layout *L = new hai_layout();
    L->ctx = ctx;
    L->n_elem = ne;
    L->grid_n = n;
    L->ksize = k;
    L->n_pol = d->n_pol;
    L->box[0] = bx0; L->box[1] = by0; L->box[2] = bx1; L->box[3] = by1;
    L->box_w = bx1 - bx0;
    L->box_h = by1 - by0;
    L->h_anchors.assign(d->anchors, d->anchors + 2 * (size_t)ne);
    L->h_taps.assign(d->taps, d->taps + 2 * (size_t)ne * k * k);

    // gather table: cells of the box in row-major order, entries by element
    const int ncell = L->box_w * L->box_h;
    std::vector<int32_t> count(ncell + 1, 0);
    for (int a = 0; a < ne; a++)
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) {
                int cell = (d->anchors[2 * a + 1] + v - by0) * L->box_w + (d->anchors[2 * a] + u - bx0);
                count[cell + 1]++;
            }
    for (int i = 0; i < ncell; i++) count[i + 1] += count[i];
    L->nnz = count[ncell];
    std::vector<int32_t> fill(count.begin(), count.end() - 1);
    std::vector<int32_t> elem(L->nnz);
    std::vector<float2> w(L->nnz);
    for (int a = 0; a < ne; a++)
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) {
                int cell = (d->anchors[2 * a + 1] + v - by0) * L->box_w + (d->anchors[2 * a] + u - bx0);
                const float *t = d->taps + (((size_t)a * k + v) * k + u) * 2;
                int slot = fill[cell]++;
                elem[slot] = a;
                w[slot] = make_float2(t[0], -t[1]);   // conj(W~)
            }

    cudaError_t e = cudaSetDevice(ctx->device);
    auto dmalloc = [&](void **p, size_t bytes) {
        const cudaError_t r = cudaMalloc(p, bytes);
        if (r == cudaSuccess) L->dev_bytes += bytes;
        return r;
    };
    if (e == cudaSuccess) e = dmalloc((void **)&L->d_anchors, sizeof(int32_t) * 2 * ne);
    if (e == cudaSuccess) e = dmalloc((void **)&L->d_taps, sizeof(float2) * (size_t)ne * k * k);
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_anchors, d->anchors, sizeof(int32_t) * 2 * ne, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_taps, d->taps, sizeof(float2) * (size_t)ne * k * k, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dmalloc((void **)&L->d_cell_start, sizeof(int32_t) * (ncell + 1));
    if (e == cudaSuccess) e = dmalloc((void **)&L->d_entry_elem, sizeof(int32_t) * std::max(1, L->nnz));
    if (e == cudaSuccess) e = dmalloc((void **)&L->d_entry_w, sizeof(float2) * std::max(1, L->nnz));
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_cell_start, count.data(), sizeof(int32_t) * (ncell + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_entry_elem, elem.data(), sizeof(int32_t) * L->nnz, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(L->d_entry_w, w.data(), sizeof(float2) * L->nnz, cudaMemcpyHostToDevice);
    // partial images of the time split (two channel segments per CTA)
    const int Q = (L->n_pol == 2) ? 4 : 1;
    // time-split partial images (grids up to 128); row scratch of the large-grid FP32 path
    if (n <= 128) {
        L->partial_slots = epic_partial_slots(std::max(epic_fp32_target_ctas(ctx, n), ctx->num_sms));
        if (e == cudaSuccess)
            e = dmalloc((void **)&L->d_partials, sizeof(float) * L->partial_slots * Q * (size_t)n * n);
    }
    if (n >= 128 && e == cudaSuccess) {
        L->large_scratch_bytes = epic_large_scratch_bytes(n, L->box_h);
        e = dmalloc(&L->d_large_scratch, L->large_scratch_bytes);
        if (e == cudaSuccess && epic_large_prepare(L) != HAI_OK) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess && epic_tc_supported(L)) {   // tensor-core path: gather table, station record
        std::vector<uint8_t> tab;
        TcStation rec = {};
        uint32_t shared_bytes = 0;
        epic_tc_station_table(n, L->box_w, L->box_h, count, elem, w, tab, rec.ntile, rec.nent, shared_bytes,
                              L->tc_entries);
        L->tc_tables_bytes = shared_bytes;
        L->tc_blob_bytes = tab.size();
        e = dmalloc(&L->d_tc_tables, tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(L->d_tc_tables, tab.data(), tab.size(), cudaMemcpyHostToDevice);
        rec.table = static_cast<const uint8_t *>(L->d_tc_tables);
        rec.ne = ne;
        rec.table_bytes = shared_bytes;
        if (e == cudaSuccess) e = dmalloc(&L->d_tc_station, sizeof(TcStation));
        if (e == cudaSuccess) e = cudaMemcpy(L->d_tc_station, &rec, sizeof(TcStation), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && epic_tc_dft_prepare(ctx, n) != HAI_OK) e = cudaErrorMemoryAllocation;
        L->tc_groups = n == 128 ? std::min(ctx->num_sms / 4, epic_tc128_max_groups(ctx, ne, shared_bytes))
                                : ctx->num_sms;
        if (L->tc_groups <= 0) L->tc_groups = 1;
    }
    if (e == cudaSuccess && epic_big_supported(L)) {
        const hai_status bs = epic_big_prepare(L);
        if (bs != HAI_OK) {
            layout_free(L);
            return bs;
        }
    }
    if (e != cudaSuccess) {
        layout_free(L);
        if (e == cudaErrorMemoryAllocation) return hai_cuda_fail(e, "hai_layout_create: allocation");
        return hai_cuda_fail(e, "hai_layout_create");
    }
    *out = L;
    return HAI_OK;
}

// Inter-station EPIC (Eq. inter-station EPIC, N_ks = 1 cell): station m at
// its nearest cell floor(r_m / cell + N/2 + 1/2), weight conj(W~_m) =
// exp(+2 pi i s_k . r_m / lambda) from an FP64 phase reduced to a fraction of
// a turn.  With the padding factor 2 per dimension (Section 5.2.2) the array
// keeps to the central half of the grid: stations outside [N/4, 3N/4)^2 are
// parked on the centre cell with weight 0 (the box then fits N/2, which the
// tensor-core kernels need, and no lag of the squared image wraps).
extern "C" hai_status hai_station_epic_layout_create(hai_ctx *ctx, const hai_vis_layout_desc *d, int k,
                                                     hai_layout **out, long long *n_dropped) {
    if (!ctx || !d || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_station_epic_layout_create: NULL argument");
    *out = nullptr;
    const int S = d->n_station, n = d->grid_n;
    if (S <= 0 || !d->pos_m || !(d->lambda_m > 0.0) || !(d->cell_m > 0.0) || n <= 0 ||
        (d->n_pol != 1 && d->n_pol != 2) || k < 0 || k >= std::max(1, d->n_dir))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_station_epic_layout_create: bad descriptor or direction index");
    const double sx = d->dir ? d->dir[2 * k] : 0.0, sy = d->dir ? d->dir[2 * k + 1] : 0.0;
    if (!std::isfinite(sx) || !std::isfinite(sy))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_station_epic_layout_create: direction not finite");
    std::vector<int32_t> anchors(2 * (size_t)S);
    std::vector<float> taps(2 * (size_t)S, 0.0f);
    long long dropped = 0;
    for (int m = 0; m < S; m++) {
        const double x = d->pos_m[2 * m], y = d->pos_m[2 * m + 1];
        const double gx = std::floor(x / d->cell_m + n / 2.0 + 0.5), gy = std::floor(y / d->cell_m + n / 2.0 + 0.5);
        const double lo = n / 4, hi = n - n / 4;
        if (!(gx >= lo && gx < hi && gy >= lo && gy < hi)) {
            anchors[2 * m] = anchors[2 * m + 1] = n / 2;
            dropped++;
            continue;
        }
        anchors[2 * m] = (int32_t)gx;
        anchors[2 * m + 1] = (int32_t)gy;
        const double turns = (sx * x + sy * y) / d->lambda_m;
        const double ang = 6.283185307179586476925286766559 * (turns - std::nearbyint(turns));
        taps[2 * m] = (float)std::cos(ang);              // W~_m = exp(-i ang)
        taps[2 * m + 1] = (float)-std::sin(ang);
    }
    hai_layout_desc ld;
    ld.n_elem = S;
    ld.grid_n = n;
    ld.ksize = 1;
    ld.n_pol = d->n_pol;
    ld.anchors = anchors.data();
    ld.taps = taps.data();
    const hai_status rc = hai_layout_create(ctx, &ld, out);
    if (rc == HAI_OK && n_dropped) *n_dropped = dropped;
    return rc;
}

extern "C" void hai_layout_destroy(hai_layout *L) {
    if (!L) return;
    cudaSetDevice(L->ctx->device);
    layout_free(L);
}

// Default illumination kernel (the paper leaves W~ to the user): a real
// Gaussian of sigma_cells evaluated at the K x K cells around the element's
// nearest cell floor(g + 1/2), g = pos / (lambda cell) + N/2 in FP64,
// normalised to unit sum; tap (u, v) on cell (x0 + u, y0 + v).
extern "C" hai_status hai_layout_create_from_positions(hai_ctx *ctx, const hai_position_desc *d, hai_layout **out) {
    if (!ctx || !d || !out || !d->pos_m) return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_create_from_positions: NULL argument");
    *out = nullptr;
    if (d->n_elem <= 0 || d->ksize <= 0 || d->ksize > 15 || !(d->lambda_m > 0) || !(d->cell_lambda > 0) ||
        !(d->sigma_cells > 0))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_create_from_positions: bad descriptor");
    const int ne = d->n_elem, k = d->ksize;
    std::vector<int32_t> anchors(2 * (size_t)ne);
    std::vector<float> taps(2 * (size_t)ne * k * k, 0.f);
    std::vector<double> w((size_t)k * k);
    for (int a = 0; a < ne; a++) {
        double gc[2];
        for (int ax = 0; ax < 2; ax++) {
            gc[ax] = d->pos_m[2 * a + ax] / (d->lambda_m * d->cell_lambda) + d->grid_n / 2.0;
            if (!std::isfinite(gc[ax]) || std::fabs(gc[ax]) > 1e9)
                return hai_fail(HAI_ERR_OFF_GRID, "hai_layout_create_from_positions: element position off the grid");
            anchors[2 * a + ax] = (int32_t)std::floor(gc[ax] + 0.5) - (k - 1) / 2;
        }
        double sum = 0;
        for (int v = 0; v < k; v++)
            for (int u = 0; u < k; u++) {
                const double dx = anchors[2 * a] + u - gc[0], dy = anchors[2 * a + 1] + v - gc[1];
                w[(size_t)v * k + u] = std::exp(-(dx * dx + dy * dy) / (2 * d->sigma_cells * d->sigma_cells));
                sum += w[(size_t)v * k + u];
            }
        for (int i = 0; i < k * k; i++) taps[((size_t)a * k * k + i) * 2] = (float)(w[i] / sum);
    }
    hai_layout_desc ld;
    ld.n_elem = ne;
    ld.grid_n = d->grid_n;
    ld.ksize = k;
    ld.n_pol = d->n_pol;
    ld.anchors = anchors.data();
    ld.taps = taps.data();
    return hai_layout_create(ctx, &ld, out);
}

extern "C" hai_status hai_layout_anchors(const hai_layout *L, int32_t *anchors, float *taps) {
    if (!L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_anchors: NULL layout");
    if (anchors) memcpy(anchors, L->h_anchors.data(), sizeof(int32_t) * L->h_anchors.size());
    if (taps) memcpy(taps, L->h_taps.data(), sizeof(float) * L->h_taps.size());
    return HAI_OK;
}

extern "C" hai_status hai_layout_workspace_size(const hai_layout *L, size_t *bytes) {
    if (!L || !bytes) return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_workspace_size: NULL argument");
    std::lock_guard<std::mutex> g(L->xfft_mu);
    *bytes = L->dev_bytes;
    return HAI_OK;
}

extern "C" hai_status hai_ctx_workspace_size(const hai_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return hai_fail(HAI_ERR_INVALID_ARG, "hai_ctx_workspace_size: NULL argument");
    *bytes = ctx->dev_bytes + ctx->corr_ws_bytes + ctx->stage_bytes;
    return HAI_OK;
}

extern "C" hai_status hai_layout_box(const hai_layout *L, int *box) {
    if (!L || !box) return hai_fail(HAI_ERR_INVALID_ARG, "hai_layout_box: NULL argument");
    memcpy(box, L->box, sizeof(L->box));
    return HAI_OK;
}

// ------------------------------------------------------------------ EPIC
EpicSplit epic_make_split(int C, int T, int target_ctas) {
    EpicSplit sp;
    // one CTA per channel once the channels fill the CTAs; below that a time
    // split whose ranges (len <= T) touch at most two channels each, which
    // is what the two partial slots per CTA hold
    if (C >= target_ctas) {
        sp.direct = 1;
        sp.n_cta = C;
        sp.len = T;
        return sp;
    }
    long long total = (long long)C * T;
    sp.len = (total + target_ctas - 1) / target_ctas;   // <= T since C < target
    sp.n_cta = (int)((total + sp.len - 1) / sp.len);
    return sp;
}

size_t epic_partial_slots(int target_ctas) { return 2 * (size_t)target_ctas; }

extern "C" hai_status hai_epic_image(hai_ctx *ctx, const hai_layout *L, const int8_t *volt, int C,
                                     int T, hai_precision prec, float *img, int accumulate,
                                     void *stream) {
    if (!ctx || !L) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: NULL ctx or layout");
    if (L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: layout of another context");
    if (C < 0 || T < 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: negative C or T");
    if (accumulate != 0 && accumulate != 1)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: accumulate must be 0 or 1");
    if (prec != HAI_PREC_FP32 && prec != HAI_PREC_FP16 && prec != HAI_PREC_FP16_SPLIT && prec != HAI_PREC_BF16 &&
        prec != HAI_PREC_BF16_SPLIT)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: unknown precision");
    if (C == 0) return HAI_OK;
    if (!img || (T > 0 && !volt)) return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: NULL buffer");
    if ((((uintptr_t)volt) & 1) || (((uintptr_t)img) & 3))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_epic_image: volt must be 2-byte and img 4-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_epic_image: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int Q = (L->n_pol == 2) ? 4 : 1;
    if (T == 0) {
        if (!accumulate)
            HAI_CUDA_TRY(cudaMemsetAsync(img, 0, sizeof(float) * (size_t)C * Q * L->grid_n * L->grid_n, st));
        return HAI_OK;
    }
    if (prec == HAI_PREC_FP32) return epic_fp32_launch(L, volt, C, T, img, accumulate, st);
    if (L->grid_n >= 256 || epic_big_used(L, prec)) return epic_big_launch(L, volt, C, T, img, accumulate, prec, st);
    const int split = (prec == HAI_PREC_FP16_SPLIT || prec == HAI_PREC_BF16_SPLIT) ? 1 : 0;
    const int bf16 = (prec == HAI_PREC_BF16 || prec == HAI_PREC_BF16_SPLIT) ? 1 : 0;
    return epic_tc_launch(L, volt, C, T, img, accumulate, st, split, bf16);
}
