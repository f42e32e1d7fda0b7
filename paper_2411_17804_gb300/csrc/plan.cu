// Batched EPIC over many stations of uneven size (hai_plan_*): one CUDA-graph
// launch per cadence images every (station, channel) of the array.
//
// Stations are grouped by grid side into classes (N = 32, 64, 128); each
// class runs its tensor-core kernel persistently over a share of the SMs,
// and the class kernels run concurrently as parallel branches of one graph.
// Inside a class, the blocks (station, channel) are laid out station-major
// and cut into contiguous per-CTA (per-cluster for N = 128) ranges of equal
// modelled cost, whole blocks only, so every image is written by exactly one
// CTA (no partial images, no reduction).  The SM shares start from the cost
// model and hai_plan_autotune refits them from measured class times.
//
// Cost model of one sample of a station, in SM cycles: a fixed part for the
// two DFT stages and the epilogue plus a part per gather entry of the
// gridding step (entries of the largest rank for N = 128).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "epic_tc.cuh"
#include "hai_internal.h"

namespace {

struct PlanClass {
    int N = 0;
    std::vector<int> stations;            // plan station indices
    std::vector<double> cost;             // modelled cycles per sample, per class station
    std::vector<TcStation> host_st;
    TcStation *d_st = nullptr;
    long long *d_begin = nullptr;         // per CTA (group) first flat sample, n_cta + 1
    size_t begin_bytes = 0;
    int n_cta = 0;                        // CTAs, or clusters for N = 128
    int ne_max = 0;
    uint32_t table_max = 0;
    size_t smem = 0;
    int max_units = 0;                    // CTAs (clusters) resident at once
    double measured_ms = 0.0;             // last autotune time of the class alone
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
};

double model_fixed(int N) { return N == 32 ? 350.0 : N == 64 ? 700.0 : 1100.0; }
double model_entry(int N) { return N == 32 ? 0.5 : N == 64 ? 0.75 : 1.0; }

}  // namespace

struct hai_plan {
    hai_ctx *ctx = nullptr;
    int S = 0, C = 0, T = 0;
    std::vector<int> grid_n, ne;
    std::vector<long long> volt_off, img_off;
    long long volt_bytes = 0, img_floats = 0;
    std::vector<void *> tables;            // plan-owned copies of the gather tables
    size_t table_bytes = 0;                // their total size
    std::vector<PlanClass> cls;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_volt = nullptr, *g_img = nullptr;
};

namespace {

void plan_free(hai_plan *p) {
    if (!p) return;
    cudaSetDevice(p->ctx->device);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto &c : p->cls) {
        cudaFree(c.d_st);
        cudaFree(c.d_begin);
        if (c.stream) cudaStreamDestroy(c.stream);
        if (c.done) cudaEventDestroy(c.done);
    }
    for (void *t : p->tables) cudaFree(t);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->fork) cudaEventDestroy(p->fork);
    delete p;
}

int group_of(int N) { return epic_tc_group(N); }

// Contiguous ranges of whole blocks, n ranges of about equal cost; returns
// the number of non-empty ranges and fills begin (flat samples, n + 1).
int split_blocks(const PlanClass &c, int C, int T, int n, std::vector<long long> &begin) {
    const long long nblk = (long long)c.stations.size() * C;
    n = (int)std::max(1ll, std::min<long long>(n, nblk));
    double total = 0.0;
    for (double v : c.cost) total += v * C;
    begin.assign(1, 0);
    double acc = 0.0;
    int made = 0;
    for (long long b = 0; b < nblk; b++) {
        acc += c.cost[b / C];
        const double goal = total * (made + 1) / n;
        // close the range once it reaches its share (keep one block per remaining range)
        if (made + 1 < n && acc >= goal && nblk - (b + 1) >= n - (made + 1)) {
            begin.push_back((b + 1) * T);
            made++;
        }
    }
    begin.push_back(nblk * T);
    return (int)begin.size() - 1;
}

hai_status class_upload_ranges(hai_plan *p, PlanClass &c, int want) {
    std::vector<long long> begin;
    c.n_cta = split_blocks(c, p->C, p->T, want, begin);
    cudaFree(c.d_begin);
    c.d_begin = nullptr;
    HAI_CUDA_TRY(cudaMalloc(&c.d_begin, sizeof(long long) * begin.size()));
    c.begin_bytes = sizeof(long long) * begin.size();
    HAI_CUDA_TRY(cudaMemcpy(c.d_begin, begin.data(), sizeof(long long) * begin.size(), cudaMemcpyHostToDevice));
    return HAI_OK;
}

// SM shares proportional to the classes' modelled (or measured) times;
// N = 128 shares are whole clusters of 4.
void shares_from_work(const hai_plan *p, const std::vector<double> &work, std::vector<int> &units) {
    const int sms = p->ctx->num_sms;
    const double tot = std::accumulate(work.begin(), work.end(), 0.0);
    units.assign(p->cls.size(), 0);
    int used = 0;
    for (size_t k = 0; k < p->cls.size(); k++) {
        const int g = group_of(p->cls[k].N);
        const double want = tot > 0 ? sms * work[k] / tot : 0.0;
        units[k] = std::min(p->cls[k].max_units, std::max(1, (int)floor(want / g)));
        used += units[k] * g;
    }
    // give back or take SMs, largest share first
    while (used > sms) {
        size_t k = 0;
        for (size_t j = 1; j < units.size(); j++)
            if (units[j] * group_of(p->cls[j].N) > units[k] * group_of(p->cls[k].N)) k = j;
        if (units[k] <= 1) break;
        units[k]--;
        used -= group_of(p->cls[k].N);
    }
    bool grew = true;
    while (grew) {
        grew = false;
        // the class with the largest work per SM gets the next unit that fits
        size_t best = units.size();
        double best_load = -1.0;
        for (size_t k = 0; k < units.size(); k++) {
            const int g = group_of(p->cls[k].N);
            if (used + g > sms || units[k] >= p->cls[k].max_units) continue;
            const double load = work[k] / (units[k] * g);
            if (load > best_load) {
                best_load = load;
                best = k;
            }
        }
        if (best < units.size()) {
            units[best]++;
            used += group_of(p->cls[best].N);
            grew = true;
        }
    }
}

TcLaunch class_launch(const hai_plan *p, const PlanClass &c, const int8_t *volt, float *img) {
    TcLaunch l;
    l.volt = volt;
    l.img = img;
    l.stations = c.d_st;
    l.n_station = (int)c.stations.size();
    l.ne_max = c.ne_max;
    l.table_max = c.table_max;
    l.cta_begin = c.d_begin;
    l.len = 0;
    l.n_cta = c.n_cta;
    l.C = p->C;
    l.T = p->T;
    l.direct = 1;
    l.accumulate = 0;
    l.guard = 1;
    l.partials = nullptr;
    l.no_attr = 1;
    l.split = 0;
    l.bf16 = 0;
    return l;
}

void drop_graph(hai_plan *p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->g_volt = p->g_img = nullptr;
}

hai_status capture(hai_plan *p, const int8_t *volt, float *img) {
    drop_graph(p);
    hai_ctx *ctx = p->ctx;
    HAI_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    ctx->capturing = 1;
    hai_status s = HAI_OK;
    cudaError_t e = cudaEventRecord(p->fork, p->cap);
    for (auto &c : p->cls) {
        if (e != cudaSuccess || s != HAI_OK) break;
        e = cudaStreamWaitEvent(c.stream, p->fork, 0);
        if (e == cudaSuccess) s = epic_tc_run(ctx, c.N, class_launch(p, c, volt, img), c.stream);
        if (e == cudaSuccess && s == HAI_OK) e = cudaEventRecord(c.done, c.stream);
        if (e == cudaSuccess && s == HAI_OK) e = cudaStreamWaitEvent(p->cap, c.done, 0);
    }
    ctx->capturing = 0;
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(p->cap, &g);
    if (s != HAI_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return hai_cuda_fail(e, "hai_plan_run: capture");
    }
    if (e2 != cudaSuccess) return hai_cuda_fail(e2, "hai_plan_run: end capture");
    p->graph = g;
    HAI_CUDA_TRY(cudaGraphInstantiate(&p->exec, g, 0));
    p->g_volt = volt;
    p->g_img = img;
    return HAI_OK;
}

}  // namespace

extern "C" hai_status hai_plan_create(hai_ctx *ctx, const hai_layout *const *stations, int S, int C, int T,
                                      hai_precision prec, hai_plan **out) {
    if (!ctx || !stations || !out) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_create: NULL argument");
    *out = nullptr;
    if (S <= 0 || C <= 0 || T <= 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_create: S, C and T must be > 0");
    if (prec != HAI_PREC_FP16)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_plan_create: the batched plan runs the FP16 tensor-core path");
    for (int s = 0; s < S; s++) {
        const hai_layout *L = stations[s];
        if (!L || L->ctx != ctx) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_create: bad layout " + std::to_string(s));
        if (!epic_tc_supported(L) || !L->d_tc_tables)
            return hai_fail(HAI_ERR_UNSUPPORTED, "hai_plan_create: station " + std::to_string(s) +
                                                     " needs N in {32, 64, 128}, 2 pols and a box <= N/2");
    }
    if (hai_fault_injected("alloc")) return hai_fail(HAI_ERR_NO_MEMORY, "hai_plan_create: injected allocation failure");
    HAI_CUDA_TRY(cudaSetDevice(ctx->device));
    hai_plan *p = new hai_plan();
    p->ctx = ctx;
    p->S = S;
    p->C = C;
    p->T = T;
    // buffer layouts: 16 guard bytes before and after every voltage block
    long long vo = 16, io = 0;
    for (int s = 0; s < S; s++) {
        const hai_layout *L = stations[s];
        p->grid_n.push_back(L->grid_n);
        p->ne.push_back(L->n_elem);
        p->volt_off.push_back(vo);
        vo = ((vo + (long long)C * T * 4 * L->n_elem + 15) & ~15ll) + 16;
        p->img_off.push_back(io);
        io += (long long)C * 4 * L->grid_n * L->grid_n;
    }
    p->volt_bytes = vo;
    p->img_floats = io;

    hai_status st = HAI_OK;
    cudaError_t e = cudaSuccess;
    for (int N : {128, 64, 32}) {
        PlanClass c;
        c.N = N;
        for (int s = 0; s < S; s++)
            if (stations[s]->grid_n == N) c.stations.push_back(s);
        if (c.stations.empty()) continue;
        for (int s : c.stations) {
            const hai_layout *L = stations[s];
            void *tab = nullptr;
            if (e == cudaSuccess) e = cudaMalloc(&tab, L->tc_blob_bytes);
            if (e == cudaSuccess) p->table_bytes += L->tc_blob_bytes;
            if (e == cudaSuccess)
                e = cudaMemcpy(tab, L->d_tc_tables, L->tc_blob_bytes, cudaMemcpyDeviceToDevice);
            if (tab) p->tables.push_back(tab);
            TcStation rec;
            if (e == cudaSuccess) e = cudaMemcpy(&rec, L->d_tc_station, sizeof(rec), cudaMemcpyDeviceToHost);
            rec.table = static_cast<const uint8_t *>(tab);
            rec.volt_off = p->volt_off[s];
            rec.img_off = p->img_off[s];
            c.host_st.push_back(rec);
            c.ne_max = std::max(c.ne_max, L->n_elem);
            c.table_max = std::max(c.table_max, (uint32_t)L->tc_tables_bytes);
            c.cost.push_back(model_fixed(N) + model_entry(N) * (double)L->tc_entries);
        }
        if (e == cudaSuccess) e = cudaMalloc(&c.d_st, sizeof(TcStation) * c.host_st.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(c.d_st, c.host_st.data(), sizeof(TcStation) * c.host_st.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming);
        c.smem = epic_tc_smem(ctx, N, c.ne_max, c.table_max);
        c.max_units = N == 128 ? std::max(1, epic_tc128_max_groups(ctx, c.ne_max, c.table_max)) : ctx->num_sms;
        p->cls.push_back(c);
        if (c.smem + kStaticSmem > (size_t)ctx->smem_optin) {
            st = hai_fail(HAI_ERR_UNSUPPORTED, "hai_plan_create: a grid class needs more shared memory than the device has");
            break;
        }
        if (e == cudaSuccess && st == HAI_OK) st = epic_tc_set_attr(ctx, N);
        if (st != HAI_OK) break;
    }
    if (e == cudaSuccess && st == HAI_OK) e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && st == HAI_OK) e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming);
    if (e == cudaSuccess && st == HAI_OK) {
        std::vector<double> work;
        for (auto &c : p->cls) work.push_back(std::accumulate(c.cost.begin(), c.cost.end(), 0.0));
        std::vector<int> units;
        shares_from_work(p, work, units);
        for (size_t k = 0; k < p->cls.size() && st == HAI_OK; k++) st = class_upload_ranges(p, p->cls[k], units[k]);
    }
    if (e != cudaSuccess || st != HAI_OK) {
        plan_free(p);
        if (st != HAI_OK) return st;
        return hai_cuda_fail(e, "hai_plan_create");
    }
    *out = p;
    return HAI_OK;
}

extern "C" void hai_plan_destroy(hai_plan *p) { plan_free(p); }

extern "C" hai_status hai_plan_layout(const hai_plan *p, int64_t *volt_off, int64_t *img_off, int64_t *volt_bytes,
                                      int64_t *img_floats) {
    if (!p) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_layout: NULL plan");
    for (int s = 0; s < p->S; s++) {
        if (volt_off) volt_off[s] = p->volt_off[s];
        if (img_off) img_off[s] = p->img_off[s];
    }
    if (volt_bytes) *volt_bytes = p->volt_bytes;
    if (img_floats) *img_floats = p->img_floats;
    return HAI_OK;
}

extern "C" hai_status hai_workspace_size(const hai_plan *p, size_t *bytes) {
    if (!p || !bytes) return hai_fail(HAI_ERR_INVALID_ARG, "hai_workspace_size: NULL argument");
    size_t b = p->table_bytes;
    for (const auto &c : p->cls) b += sizeof(TcStation) * c.host_st.size() + c.begin_bytes;
    *bytes = b;
    return HAI_OK;
}

extern "C" hai_status hai_plan_schedule(const hai_plan *p, int *n_class, int *grid_n, int *ctas, double *measured_ms) {
    if (!p || !n_class) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_schedule: NULL argument");
    *n_class = (int)p->cls.size();
    for (size_t k = 0; k < p->cls.size(); k++) {
        if (grid_n) grid_n[k] = p->cls[k].N;
        if (ctas) ctas[k] = p->cls[k].n_cta * group_of(p->cls[k].N);
        if (measured_ms) measured_ms[k] = p->cls[k].measured_ms;
    }
    return HAI_OK;
}

extern "C" hai_status hai_plan_run(hai_plan *p, const int8_t *volt, float *img, void *stream) {
    if (!p || !volt || !img) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run: NULL argument");
    if ((((uintptr_t)volt) & 15) != 0 || (((uintptr_t)img) & 15) != 0)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run: buffers must be 16-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_plan_run: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(p->ctx->device));
    if (!p->exec || p->g_volt != volt || p->g_img != img) {
        const hai_status s = capture(p, volt, img);
        if (s != HAI_OK) return s;
    }
    const int pidx = prof_begin(p->ctx, (cudaStream_t)stream);
    HAI_CUDA_TRY(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    prof_end(p->ctx, pidx, (cudaStream_t)stream);
    prof_count(p->ctx, (int)p->cls.size());
    return HAI_OK;
}

extern "C" hai_status hai_plan_autotune(hai_plan *p, const int8_t *volt, float *img, int rounds, void *stream) {
    if (!p || !volt || !img || rounds < 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_autotune: bad argument");
    HAI_CUDA_TRY(cudaSetDevice(p->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a, b;
    HAI_CUDA_TRY(cudaEventCreate(&a));
    HAI_CUDA_TRY(cudaEventCreate(&b));
    hai_status s = HAI_OK;
    for (int r = 0; r < rounds && s == HAI_OK; r++) {
        // time every class alone on its current share (second of two runs)
        std::vector<double> work;
        for (auto &c : p->cls) {
            const TcLaunch l = class_launch(p, c, volt, img);
            for (int rep = 0; rep < 2 && s == HAI_OK; rep++) {
                if (cudaEventRecord(a, st) != cudaSuccess) s = hai_fail(HAI_ERR_CUDA, "hai_plan_autotune: event");
                if (s == HAI_OK) s = epic_tc_run(p->ctx, c.N, l, st);
                if (s == HAI_OK && cudaEventRecord(b, st) != cudaSuccess) s = hai_fail(HAI_ERR_CUDA, "hai_plan_autotune: event");
            }
            float ms = 0.f;
            if (s == HAI_OK && (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess))
                s = hai_fail(HAI_ERR_CUDA, "hai_plan_autotune: timing");
            c.measured_ms = ms;
            // SM-milliseconds of the class at its share: what it needs at any share
            work.push_back((double)ms * c.n_cta * group_of(c.N));
        }
        if (s != HAI_OK) break;
        std::vector<int> units;
        shares_from_work(p, work, units);
        for (size_t k = 0; k < p->cls.size() && s == HAI_OK; k++) s = class_upload_ranges(p, p->cls[k], units[k]);
        drop_graph(p);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return s;
}
