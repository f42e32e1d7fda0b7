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
//
// Second level (hai_plan_set_hierarchy, Section 6): after the station images
// the same graph beamforms every station (int8 weights, exact int32 sums,
// requantised to int8), reorders the beams for the inter-station stage and
// images them with the inter-station correlator + XFFT and/or the
// inter-station EPIC of every beam.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
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
    // second level
    int hK = 0, hshift = 0;
    void *d_hst = nullptr;                       // per station: voltage and weight offsets, elements
    void *d_pw = nullptr;                        // the weights re-packed for the integer dot products
    // the persistent beam kernel (when its shared memory fits): weights per
    // (beam, pair) in 32 bytes, item starts per station, CTA item ranges
    void *d_pw2 = nullptr, *d_hitem = nullptr, *d_order = nullptr, *d_next = nullptr;
    int bf2_grid = 0;                            // 0: the per-block kernel instead
    size_t bf2_w = 0, bf2_raw = 0, bf2_smem = 0;
    const hai_vis_layout *hx = nullptr;          // inter-station XFFT (or NULL)
    std::vector<const hai_layout *> he;          // inter-station EPIC layouts, one per beam (or none)
    hai_precision hprec = HAI_PREC_FP16;
    bool g_hier = false;                         // the captured graph holds the second level
    hai_plan_hier_buffers gb = {};               // with these buffers
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
    cudaFree(p->d_hst);
    cudaFree(p->d_pw);
    cudaFree(p->d_pw2);
    cudaFree(p->d_hitem);
    cudaFree(p->d_order);
    cudaFree(p->d_next);
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
    p->g_hier = false;
}

// ------------------------------------------------------------------ station beams
// Eq. intra-station BF with diagonal polarisation weights, for stations of
// any element count, in exact integer dot products:
//   Re conj(w) E = w.re E.re + w.im E.im  -> __dp4a over two elements' (re, im)
//   Im conj(w) E = w.re E.im - w.im E.re  -> __dp2a of (w.re, -w.im) as int16
//                                            with (E.im, E.re)
// The weights are re-packed once (hai_plan_set_hierarchy) into both forms:
// per station WP[k][p][pair] (4 int8: two elements' re, im) then
// WQ[k][p][element] (2 int16: re, -im), odd element counts padded with a zero
// element.  Block (station s, channel c, 64 samples, or 32 with more than 16
// beam pairs), thread (sample t, beam pair kp): the two beams' sums of both
// pols in int32 (exact: |sum| <= 2^15 N_e), the voltages staged through
// shared memory 128 elements at a time;
// the sums are requantised as hai_beamform does (|x| / 2^shift rounded half
// away from zero, clamped to 127) into beams [S][C][T][K][2][2].
struct HierStation {
    long long volt_off, w_off;   // bytes into the plan's voltage buffer / the caller's weights
    long long pw_off;            // 32-bit words into the packed weights
    long long pw2_off;           // 16-byte units into the persistent kernel's weights
    int ne, ne2;                 // elements, element pairs
    int tb, nblk;                // persistent kernel: (channel, sample) rows per item, items of the station
};
constexpr int kBfTMax = 64;              // samples per block: 64, or 32 for more than 16 beam pairs
__host__ __device__ __forceinline__ int bf_samples(int K) { return (K + 1) / 2 > 16 ? 32 : kBfTMax; }
constexpr int kBfPairs = 64;             // element pairs per shared-memory pass
constexpr int kBfERow = kBfPairs + 1;    // words per staged (sample, pol) row: rows t fall in distinct banks
constexpr int kBfWRow = kBfPairs + 1;    // words per staged WP row
constexpr int kBfQRow = 2 * kBfPairs + 2;   // words per staged WQ row (8-byte aligned, rows 4 banks apart)

__global__ void plan_bf_pack_kernel(const int8_t *__restrict__ w, const HierStation *__restrict__ hst, int K,
                                    uint32_t *__restrict__ pw, uint4 *__restrict__ pw2) {
    const HierStation h = hst[blockIdx.x];
    const char2 *W = reinterpret_cast<const char2 *>(w + h.w_off);      // [K][2][ne]
    if (pw2) {
        // per (beam k, pair j): {WP_0, WQ_0[2j], WQ_0[2j+1], WP_1} {WQ_1[2j], WQ_1[2j+1], 0, 0}
        auto pk = [&](int k, int p, int a) {
            return a < h.ne ? W[(size_t)(k * 2 + p) * h.ne + a] : make_char2(0, 0);
        };
        auto wpw = [](char2 g0, char2 g1) {
            return (uint32_t)(uint8_t)g0.x | ((uint32_t)(uint8_t)g0.y << 8) | ((uint32_t)(uint8_t)g1.x << 16) |
                   ((uint32_t)(uint8_t)g1.y << 24);
        };
        auto wqw = [](char2 g) { return (uint32_t)(uint16_t)(int16_t)g.x | ((uint32_t)(uint16_t)(int16_t)(-(int)g.y) << 16); };
        uint4 *o = pw2 + h.pw2_off;
        for (int i = threadIdx.x; i < K * h.ne2; i += blockDim.x) {
            const int k = i / h.ne2, j = i % h.ne2;
            const char2 a0 = pk(k, 0, 2 * j), a1 = pk(k, 0, 2 * j + 1), b0 = pk(k, 1, 2 * j), b1 = pk(k, 1, 2 * j + 1);
            o[2 * i] = make_uint4(wpw(a0, a1), wqw(a0), wqw(a1), wpw(b0, b1));
            o[2 * i + 1] = make_uint4(wqw(b0), wqw(b1), 0u, 0u);
        }
    }
    uint32_t *wp = pw + h.pw_off, *wq = wp + (size_t)K * 2 * h.ne2;
    for (int i = threadIdx.x; i < K * 2 * h.ne2; i += blockDim.x) {
        const int row = i / h.ne2, j = i % h.ne2, a = 2 * j;
        const char2 g0 = W[(size_t)row * h.ne + a];
        const char2 g1 = a + 1 < h.ne ? W[(size_t)row * h.ne + a + 1] : make_char2(0, 0);
        wp[i] = (uint32_t)(uint8_t)g0.x | ((uint32_t)(uint8_t)g0.y << 8) | ((uint32_t)(uint8_t)g1.x << 16) |
                ((uint32_t)(uint8_t)g1.y << 24);
    }
    for (int i = threadIdx.x; i < K * 2 * 2 * h.ne2; i += blockDim.x) {
        const int row = i / (2 * h.ne2), a = i % (2 * h.ne2);
        const char2 g = a < h.ne ? W[(size_t)row * h.ne + a] : make_char2(0, 0);
        wq[i] = (uint32_t)(uint16_t)(int16_t)g.x | ((uint32_t)(uint16_t)(int16_t)(-(int)g.y) << 16);
    }
}

__device__ __forceinline__ int bf_requant(int x, int shift, int &sat) {
    int m = x < 0 ? -x : x;
    if (shift > 0) m = (m + (1 << (shift - 1))) >> shift;
    if (m > 127) {
        m = 127;
        sat++;
    }
    return x < 0 ? -m : m;
}

__global__ void __launch_bounds__(1024) plan_bf_kernel(const int8_t *__restrict__ volt,
                                                       const uint32_t *__restrict__ pw,
                                                       const HierStation *__restrict__ hst, int C, int T, int K,
                                                       int shift, int8_t *__restrict__ beams,
                                                       unsigned long long *__restrict__ n_sat) {
    extern __shared__ uint32_t sbw[];
    const int KP = (K + 1) / 2;
    const int TB = bf_samples(K);
    uint32_t *sE = sbw;                                   // [TB][2][kBfERow]
    uint32_t *sP = sE + TB * 2 * kBfERow;                 // [2 KP][2][kBfWRow] (a padded odd beam reads zeros)
    uint32_t *sQ = sP + 2 * KP * 2 * kBfWRow;             // [2 KP][2][kBfQRow]
    const int s = blockIdx.x, c = blockIdx.y, t0 = blockIdx.z * TB;
    const HierStation h = hst[s];
    const int ne = h.ne, ne2 = h.ne2, nt = min(TB, T - t0);
    const int t = threadIdx.x / KP, kp = threadIdx.x % KP;
    const char2 *E = reinterpret_cast<const char2 *>(volt + h.volt_off) + ((size_t)c * T + t0) * 2 * ne;
    const uint32_t *WP = pw + h.pw_off, *WQ = WP + (size_t)K * 2 * ne2;
    for (int i = threadIdx.x; i < 2 * KP * 2 * (kBfWRow + kBfQRow); i += blockDim.x) sP[i] = 0u;   // beam K (odd K)
    int acc[2][2][2] = {};                                // [beam of the pair][pol][re, im]
    for (int j0 = 0; j0 < ne2; j0 += kBfPairs) {
        const int np = min(kBfPairs, ne2 - j0);
        __syncthreads();
#pragma unroll 4
        for (int i = threadIdx.x; i < nt * 2 * np; i += blockDim.x) {
            const int j = i % np, row = i / np;            // row = (sample, pol)
            const int a = 2 * (j0 + j);
            const char2 e0 = E[(size_t)row * ne + a];
            const char2 e1 = a + 1 < ne ? E[(size_t)row * ne + a + 1] : make_char2(0, 0);
            sE[row * kBfERow + j] = (uint32_t)(uint8_t)e0.x | ((uint32_t)(uint8_t)e0.y << 8) |
                                    ((uint32_t)(uint8_t)e1.x << 16) | ((uint32_t)(uint8_t)e1.y << 24);
        }
        for (int i = threadIdx.x; i < K * 2 * np; i += blockDim.x) {
            const int j = i % np, row = i / np;            // row = (beam, pol)
            sP[row * kBfWRow + j] = WP[(size_t)row * ne2 + j0 + j];
        }
        for (int i = threadIdx.x; i < K * 2 * 2 * np; i += blockDim.x) {
            const int a = i % (2 * np), row = i / (2 * np);
            sQ[row * kBfQRow + a] = WQ[(size_t)row * 2 * ne2 + 2 * j0 + a];
        }
        __syncthreads();
        if (t < nt) {
#pragma unroll 2
            for (int j = 0; j < np; j++) {
#pragma unroll
                for (int pol = 0; pol < 2; pol++) {
                    const int e = (int)sE[(2 * t + pol) * kBfERow + j];
                    const int es = (int)__byte_perm((uint32_t)e, 0u, 0x2301);   // (im, re) of both elements
#pragma unroll
                    for (int b = 0; b < 2; b++) {
                        const int row = (2 * kp + b) * 2 + pol;
                        const int wp = (int)sP[row * kBfWRow + j];
                        const uint2 wq = *reinterpret_cast<const uint2 *>(sQ + row * kBfQRow + 2 * j);
                        acc[b][pol][0] = __dp4a(wp, e, acc[b][pol][0]);
                        acc[b][pol][1] = __dp2a_lo((int)wq.x, es, acc[b][pol][1]);
                        acc[b][pol][1] = __dp2a_hi((int)wq.y, es, acc[b][pol][1]);
                    }
                }
            }
        }
    }
    int sat = 0;
    if (t < nt) {
#pragma unroll
        for (int b = 0; b < 2; b++) {
            const int k = 2 * kp + b;
            if (k >= K) break;
            const int b0 = bf_requant(acc[b][0][0], shift, sat), b1 = bf_requant(acc[b][0][1], shift, sat);
            const int b2 = bf_requant(acc[b][1][0], shift, sat), b3 = bf_requant(acc[b][1][1], shift, sat);
            const char4 v = make_char4((signed char)b0, (signed char)b1, (signed char)b2, (signed char)b3);
            reinterpret_cast<char4 *>(beams)[(((size_t)s * C + c) * T + t0 + t) * K + k] = v;
        }
    }
    if (n_sat) {
        for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xffffffffu, sat, o);
        if ((threadIdx.x & 31) == 0 && sat) atomicAdd(n_sat, (unsigned long long)sat);
    }
}

size_t bf_smem(int K) {
    const int KP = (K + 1) / 2;
    return sizeof(uint32_t) * ((size_t)bf_samples(K) * 2 * kBfERow + (size_t)2 * KP * 2 * (kBfWRow + kBfQRow));
}

// The same beams from a persistent kernel, one CTA per SM taking items
// (station, block of tb consecutive (channel, sample) rows of its flat C T
// rows; a block may cross channels) from an atomic counter, the largest
// stations' items first so that the small ones even out the end:
//   - the item's voltages are one contiguous run of tb x 2 pols x N_e
//     complex int8 ([C][T][2][N_e][2] per station): copied by 16-byte
//     cp.async from the enclosing 16-byte-aligned span (the plan leaves 16
//     spare bytes around each station) while the previous item is summed;
//   - the run is re-laid into rows of element pairs (one 32-bit word per two
//     elements, odd element counts completed with a zero element) with an odd
//     row stride, pols in separate planes, so that 32 consecutive samples read
//     32 distinct banks;
//   - the station's weights stay in shared memory while its items last, per
//     (beam, pair) two 16-byte words that every lane of a warp reads at once;
//   - a group of spl lanes per (beam, 4 rows) (one row where an item has too
//     few rows to fill the CTA; spl = 1, 2, 4 or 8, the largest that keeps the
//     item's groups within the CTA): each lane sums its share of the element
//     pairs for both pols' Re and Im in int32, reading a pair's weights once
//     for its rows; shuffles join the shares, and the sums are requantised on
//     the way out exactly as by the per-block kernel.
constexpr int kBf2Threads = 512;

__device__ __forceinline__ void bf2_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

// The sums of one item: task (beam k, rows t + r S1, r < R; S1 = ceil(nt / R))
// by a group of spl lanes, each over its share of the element pairs; the
// weights of (k, pair) are read once for the R rows.  Returns the saturations.
template <int R>
__device__ __forceinline__ int bf2_sum(const uint32_t *__restrict__ sE, const uint4 *__restrict__ sW,
                                       int8_t *__restrict__ beams, int tid, int RS, int m, int tb, int nt, int K,
                                       int shift, size_t row0) {
    const int S1 = (nt + R - 1) / R, tasks = S1 * K;
    int spl = 1;
    while (spl < 8 && tasks * spl * 2 <= kBf2Threads) spl *= 2;
    const int part = tid & (spl - 1), mp = (m + spl - 1) / spl;
    const int jb = min(m, part * mp), je = min(m, jb + mp);
    int sat = 0;
    for (int q0 = 0; q0 < tasks; q0 += kBf2Threads / spl) {                // CTA-uniform trip count
        const int q = q0 + tid / spl;
        const bool live = q < tasks;
        const int k = live ? q / S1 : 0, t = live ? q - k * S1 : 0;
        const uint4 *wk = sW + (size_t)k * m * 2;
        int acc[R][4];
#pragma unroll
        for (int r = 0; r < R; r++) acc[r][0] = acc[r][1] = acc[r][2] = acc[r][3] = 0;
#pragma unroll 2
        for (int j = jb; j < (live ? je : jb); j++) {
            const uint4 wa = wk[2 * j], wb = wk[2 * j + 1];
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int tr = min(t + r * S1, nt - 1);                    // rows past nt: read, not written
                const int e0 = (int)sE[(size_t)tr * RS + j], e1 = (int)sE[((size_t)tb + tr) * RS + j];
                const int es0 = (int)__byte_perm((uint32_t)e0, 0u, 0x2301);
                const int es1 = (int)__byte_perm((uint32_t)e1, 0u, 0x2301);
                acc[r][0] = __dp4a((int)wa.x, e0, acc[r][0]);
                acc[r][1] = __dp2a_lo((int)wa.y, es0, acc[r][1]);
                acc[r][1] = __dp2a_hi((int)wa.z, es0, acc[r][1]);
                acc[r][2] = __dp4a((int)wa.w, e1, acc[r][2]);
                acc[r][3] = __dp2a_lo((int)wb.x, es1, acc[r][3]);
                acc[r][3] = __dp2a_hi((int)wb.y, es1, acc[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            for (int o = 1; o < spl; o <<= 1)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[r][v] += __shfl_xor_sync(0xffffffffu, acc[r][v], o);
            const int tr = t + r * S1;
            if (live && part == 0 && tr < nt) {
                const int b0 = bf_requant(acc[r][0], shift, sat), b1 = bf_requant(acc[r][1], shift, sat);
                const int b2 = bf_requant(acc[r][2], shift, sat), b3 = bf_requant(acc[r][3], shift, sat);
                reinterpret_cast<char4 *>(beams)[(row0 + tr) * K + k] =
                    make_char4((signed char)b0, (signed char)b1, (signed char)b2, (signed char)b3);
            }
        }
    }
    return sat;
}

__global__ void __launch_bounds__(kBf2Threads, 1) plan_bf2_kernel(
    const int8_t *__restrict__ volt, const uint4 *__restrict__ pw2, const HierStation *__restrict__ hst,
    const long long *__restrict__ hitem, const int *__restrict__ order, unsigned long long *__restrict__ next_item,
    int S, int C, int T, int K, int shift, int w_bytes, int raw_bytes, int8_t *__restrict__ beams,
    unsigned long long *__restrict__ n_sat) {
    extern __shared__ __align__(16) uint8_t sm2[];
    __shared__ long long s_item;
    uint4 *sW = reinterpret_cast<uint4 *>(sm2);                          // [K][ne2][2]
    uint8_t *raw = sm2 + w_bytes;                                         // the item's voltage run
    uint32_t *sE = reinterpret_cast<uint32_t *>(raw + raw_bytes);        // [2][tb][RS]
    const int tid = threadIdx.x, lane = tid & 31;
    const int CT = C * T;                                                 // rows (channel, sample) of a station
    const long long n_items = hitem[S];
    // item -> (station, block): items run over the stations in the order
    // given (largest first, so that the small ones fill the end)
    auto locate = [&](long long item, int &st, int &blk) {
        int lo = 0, hi = S - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (hitem[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        st = order[lo];
        blk = (int)(item - hitem[lo]);
    };
    auto issue = [&](const HierStation &hh, int bb) {                     // returns the run's word offset
        const int t0 = bb * hh.tb, nt = min(hh.tb, CT - t0);
        const long long start = hh.volt_off + (long long)t0 * 4ll * hh.ne;
        const long long a0 = start & ~15ll, a1 = (start + (long long)nt * 4 * hh.ne + 15) & ~15ll;
        const int n16 = (int)((a1 - a0) >> 4);
        for (int i = tid; i < n16; i += kBf2Threads) bf2_cp16(raw + 16 * i, volt + a0 + 16 * i);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        return (int)((start - a0) >> 2);
    };
    if (tid == 0) s_item = (long long)atomicAdd(next_item, 1ull);
    __syncthreads();
    long long cur = s_item;
    if (cur >= n_items) return;
    int s, blk;
    locate(cur, s, blk);
    HierStation h = hst[s];
    int off = issue(h, blk);
    int cur_w = -1, sat = 0;
    for (;;) {
        if (tid == 0) s_item = (long long)atomicAdd(next_item, 1ull);
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();                                   // the run has landed; the previous item is summed
        const long long nxt = s_item;
        if (s != cur_w) {                                  // this station's weights
            const int n16 = K * h.ne2 * 2;
            for (int i = tid; i < n16; i += kBf2Threads) bf2_cp16(sW + i, pw2 + h.pw2_off + i);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            cur_w = s;
        }
        const int m = h.ne2, ne = h.ne, tb = h.tb, t0 = blk * tb, nt = min(tb, CT - t0);
        const int RS = m | 1;                              // odd row stride (words)
        {
            // word w = r m + j of the item (row r = (sample r >> 1, pol r & 1)),
            // lanes over consecutive words, (r, j) carried along
            const int nw = 2 * nt * m;
            int r = tid / m, j = tid - r * m;
            const int dr = kBf2Threads / m, dj = kBf2Threads - dr * m;
            for (int w = tid; w < nw; w += kBf2Threads) {
                uint32_t v;
                if (!(ne & 1)) {
                    v = reinterpret_cast<const uint32_t *>(raw)[off + w];
                } else {
                    const uint16_t *src = reinterpret_cast<const uint16_t *>(raw) + 2 * off + (size_t)r * ne;
                    const uint32_t lo = src[2 * j], hi = (2 * j + 1 < ne) ? src[2 * j + 1] : 0u;
                    v = lo | (hi << 16);
                }
                sE[((size_t)(r & 1) * tb + (r >> 1)) * RS + j] = v;
                r += dr;
                j += dj;
                if (j >= m) {
                    j -= m;
                    r++;
                }
            }
        }
        __syncthreads();                                   // rows ready, the run buffer free
        // the next item's run, in flight while this one is summed
        const int cs = s;
        if (nxt < n_items) {
            locate(nxt, s, blk);
            if (s != cs) h = hst[s];
            off = issue(h, blk);
        }
        if (nt >= 16)
            sat += bf2_sum<4>(sE, sW, beams, tid, RS, m, tb, nt, K, shift, (size_t)cs * CT + t0);
        else
            sat += bf2_sum<1>(sE, sW, beams, tid, RS, m, tb, nt, K, shift, (size_t)cs * CT + t0);
        if (nxt >= n_items) break;
    }
    if (n_sat) {
        for (int o = 16; o > 0; o >>= 1) sat += __shfl_xor_sync(0xffffffffu, sat, o);
        if (lane == 0 && sat) atomicAdd(n_sat, (unsigned long long)sat);
    }
}

// The second level on stream st (inside the capture): beams, their
// inter-station order, then the correlator + XFFT and/or the EPIC of every beam.
hai_status run_second_level(hai_plan *p, const int8_t *volt, const hai_plan_hier_buffers *b, cudaStream_t st) {
    hai_ctx *ctx = p->ctx;
    const int S = p->S, C = p->C, T = p->T, K = p->hK;
    if (b->n_saturated) HAI_CUDA_TRY(cudaMemsetAsync(b->n_saturated, 0, sizeof(long long), st));
    if (p->bf2_grid > 0) {
        HAI_CUDA_TRY(cudaMemsetAsync(p->d_next, 0, sizeof(unsigned long long), st));
        plan_bf2_kernel<<<(unsigned)p->bf2_grid, kBf2Threads, p->bf2_smem, st>>>(
            volt, static_cast<const uint4 *>(p->d_pw2), static_cast<const HierStation *>(p->d_hst),
            static_cast<const long long *>(p->d_hitem), static_cast<const int *>(p->d_order),
            static_cast<unsigned long long *>(p->d_next), S, C, T, K, p->hshift, (int)p->bf2_w, (int)p->bf2_raw,
            b->beams, reinterpret_cast<unsigned long long *>(b->n_saturated));
    } else {
        const int TB = bf_samples(K);
        plan_bf_kernel<<<dim3((unsigned)S, (unsigned)C, (unsigned)((T + TB - 1) / TB)), TB * ((K + 1) / 2), bf_smem(K),
                         st>>>(volt, static_cast<const uint32_t *>(p->d_pw), static_cast<const HierStation *>(p->d_hst),
                               C, T, K, p->hshift, b->beams, reinterpret_cast<unsigned long long *>(b->n_saturated));
    }
    HAI_CUDA_TRY(cudaGetLastError());
    hai_status s = hai_beams_to_corr(ctx, b->beams, S, C, T, K, 2, b->corr, st);
    if (s != HAI_OK) return s;
    if (p->hx) {
        s = hai_correlate(ctx, b->corr, K * C, T, S, 2, b->vis, 0, st);
        if (s == HAI_OK) s = hai_xfft_station_image(ctx, p->hx, b->vis, C, b->xfft_img, st);
        if (s != HAI_OK) return s;
    }
    const size_t beam_block = (size_t)C * T * 2 * S * 2;
    for (int k = 0; k < (int)p->he.size(); k++) {
        const hai_layout *L = p->he[k];
        s = hai_epic_image(ctx, L, b->corr + (size_t)k * beam_block, C, T, p->hprec,
                           b->epic_img + (size_t)k * C * 4 * L->grid_n * L->grid_n, 0, st);
        if (s != HAI_OK) return s;
    }
    return HAI_OK;
}

hai_status capture(hai_plan *p, const int8_t *volt, float *img, const hai_plan_hier_buffers *hb) {
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
    if (hb && e == cudaSuccess && s == HAI_OK) s = run_second_level(p, volt, hb, p->cap);
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
    p->g_hier = hb != nullptr;
    if (hb) p->gb = *hb;
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
    if (!p->exec || p->g_volt != volt || p->g_img != img || p->g_hier) {
        const hai_status s = capture(p, volt, img, nullptr);
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

extern "C" hai_status hai_plan_set_hierarchy(hai_plan *p, const hai_plan_hier_desc *d) {
    if (!p || !d) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: NULL argument");
    const int K = d->n_beam, S = p->S;
    if (K < 1 || K > 64 || !d->weights || !d->weight_off || d->requant_shift < 0 || d->requant_shift > 30)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: n_beam in 1..64, weights, offsets and a "
                                             "shift in 0..30 are needed");
    if (!d->xfft && !d->epic)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: no inter-station stage (xfft or epic)");
    if (d->xfft) {
        int vs = 0, vn = 0, vk = 0;
        vis_layout_dims(d->xfft, &vs, &vn, &vk);
        if (vs != S || vk != K) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: the XFFT layout needs "
                                                                     "the plan's S stations and n_beam directions");
    }
    if (d->epic) {
        for (int k = 0; k < K; k++) {
            const hai_layout *L = d->epic[k];
            if (!L || L->ctx != p->ctx || L->n_elem != S || L->n_pol != 2)
                return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: EPIC layout " + std::to_string(k) +
                                                         " must have the plan's S stations as elements and 2 pols");
        }
        if (d->epic_prec < HAI_PREC_FP32 || d->epic_prec > HAI_PREC_BF16_SPLIT)
            return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: EPIC precision");
    }
    if (2 * K * 2 * (S + 1) > 48 * 1024)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_plan_set_hierarchy: S x n_beam too large for the beam reorder");
    std::vector<HierStation> hs(S);
    long long pw_words = 0;
    for (int s = 0; s < S; s++) {
        if (d->weight_off[s] < 0 || (d->weight_off[s] & 1))
            return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_set_hierarchy: weight offsets must be even and >= 0");
        hs[s].volt_off = p->volt_off[s];
        hs[s].w_off = d->weight_off[s];
        hs[s].ne = p->ne[s];
        hs[s].ne2 = (p->ne[s] + 1) / 2;
        hs[s].pw_off = pw_words;
        pw_words += 3ll * K * 2 * hs[s].ne2;             // WP (K 2 ne2 words) then WQ (K 2 2 ne2)
    }
    HAI_CUDA_TRY(cudaSetDevice(p->ctx->device));
    if (d->xfft) {
        const hai_status ws = hai_workspace(p->ctx);         // the correlator's operand workspace, before any capture
        if (ws != HAI_OK) return ws;
    }
    HAI_CUDA_TRY(hai_allow_dyn_smem(plan_bf_kernel, p->ctx->smem_optin));
    if (bf_smem(K) > (size_t)p->ctx->smem_optin)
        return hai_fail(HAI_ERR_UNSUPPORTED, "hai_plan_set_hierarchy: n_beam too large for shared memory");
    // the persistent beam kernel: each station's weights (K ne2 x 32 bytes),
    // one voltage run and its re-laid rows share the SM; rows per item so
    // that the run and the rows take at most half of the rest each
    const int C = p->C, T = p->T;
    int m_max = 1;
    for (int st = 0; st < S; st++) m_max = std::max(m_max, hs[st].ne2);
    const size_t w_bytes = (size_t)K * m_max * 32;
    const long long budget = (long long)p->ctx->smem_optin - (long long)w_bytes - 1024;
    int bf2_grid = 0;
    size_t raw_bytes = 0, se_bytes = 0;
    std::vector<long long> hitem(S + 1, 0);                // item starts, in the order below
    std::vector<int> order(S);                             // stations, most elements first
    long long pw2_units = 0;
    if (budget > 0) {
        const long long cap = budget / 2;
        bool ok = true;
        for (int st = 0; st < S && ok; st++) {
            const long long rs = hs[st].ne2 | 1;
            const long long tb = std::min<long long>({(long long)C * T, (cap - 48) / (4ll * hs[st].ne), cap / (8 * rs)});
            if (tb < 1) ok = false;
            hs[st].tb = (int)std::max<long long>(tb, 1);
            hs[st].nblk = (int)(((long long)C * T + hs[st].tb - 1) / hs[st].tb);
            hs[st].pw2_off = pw2_units;
            pw2_units += 2ll * K * hs[st].ne2;
            raw_bytes = std::max(raw_bytes, (size_t)hs[st].tb * 4 * (size_t)hs[st].ne + 32);
            se_bytes = std::max(se_bytes, (size_t)(2ll * hs[st].tb * rs * 4));
        }
        raw_bytes = (raw_bytes + 15) / 16 * 16;
        for (int st = 0; st < S; st++) order[st] = st;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return hs[x].ne > hs[y].ne; });
        for (int i = 0; i < S; i++) hitem[i + 1] = hitem[i] + hs[order[i]].nblk;
        if (ok && w_bytes + raw_bytes + se_bytes <= (size_t)p->ctx->smem_optin && hitem[S] > 0)
            bf2_grid = (int)std::min<long long>(p->ctx->num_sms, hitem[S]);
    }
    void *d_hst = nullptr, *d_pw = nullptr, *d_pw2 = nullptr, *d_hitem = nullptr, *d_order = nullptr,
         *d_next = nullptr;
    cudaError_t e = cudaMalloc(&d_hst, sizeof(HierStation) * S);
    if (e == cudaSuccess) e = cudaMalloc(&d_pw, sizeof(uint32_t) * (size_t)pw_words);
    if (e == cudaSuccess && bf2_grid > 0) {
        e = cudaMalloc(&d_pw2, sizeof(uint4) * (size_t)pw2_units);
        if (e == cudaSuccess) e = cudaMalloc(&d_hitem, sizeof(long long) * (S + 1));
        if (e == cudaSuccess) e = cudaMalloc(&d_order, sizeof(int) * S);
        if (e == cudaSuccess) e = cudaMalloc(&d_next, sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaMemcpy(d_hitem, hitem.data(), sizeof(long long) * (S + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_order, order.data(), sizeof(int) * S, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = hai_allow_dyn_smem(plan_bf2_kernel, p->ctx->smem_optin);
    }
    if (e == cudaSuccess) e = cudaMemcpy(d_hst, hs.data(), sizeof(HierStation) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        plan_bf_pack_kernel<<<(unsigned)S, 256>>>(d->weights, static_cast<const HierStation *>(d_hst), K,
                                                 static_cast<uint32_t *>(d_pw), static_cast<uint4 *>(d_pw2));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d_hst);
        cudaFree(d_pw);
        cudaFree(d_pw2);
        cudaFree(d_hitem);
        cudaFree(d_order);
        cudaFree(d_next);
        return hai_cuda_fail(e, "hai_plan_set_hierarchy: station records and packed weights");
    }
    cudaFree(p->d_hst);
    cudaFree(p->d_pw);
    cudaFree(p->d_pw2);
    cudaFree(p->d_hitem);
    cudaFree(p->d_order);
    cudaFree(p->d_next);
    p->d_hst = d_hst;
    p->d_pw = d_pw;
    p->d_pw2 = d_pw2;
    p->d_hitem = d_hitem;
    p->d_order = d_order;
    p->d_next = d_next;
    p->bf2_grid = bf2_grid;
    p->bf2_w = w_bytes;
    p->bf2_raw = raw_bytes;
    p->bf2_smem = w_bytes + raw_bytes + se_bytes;
    p->hK = K;
    p->hshift = d->requant_shift;
    p->hx = d->xfft;
    p->he.clear();
    if (d->epic) p->he.assign(d->epic, d->epic + K);
    p->hprec = d->epic_prec;
    drop_graph(p);
    return HAI_OK;
}

extern "C" hai_status hai_plan_hier_sizes(const hai_plan *p, int64_t *beam_bytes, int64_t *vis_ints,
                                          int64_t *xfft_floats, int64_t *epic_floats) {
    if (!p) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_hier_sizes: NULL plan");
    if (p->hK == 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_hier_sizes: no hierarchy set");
    const long long S = p->S, K = p->hK;
    if (beam_bytes) *beam_bytes = S * p->C * p->T * K * 4;
    if (vis_ints) *vis_ints = p->hx ? K * p->C * (S * (S + 1) / 2) * 8 : 0;
    if (xfft_floats) {
        int vs = 0, vn = 0, vk = 0;
        if (p->hx) vis_layout_dims(p->hx, &vs, &vn, &vk);
        *xfft_floats = p->hx ? K * p->C * 4ll * vn * vn : 0;
    }
    if (epic_floats) {
        long long f = 0;
        for (const hai_layout *L : p->he) f += (long long)p->C * 4 * L->grid_n * L->grid_n;
        *epic_floats = p->he.empty() ? 0 : f;
    }
    return HAI_OK;
}

extern "C" hai_status hai_plan_run_hier(hai_plan *p, const int8_t *volt, float *img, const hai_plan_hier_buffers *b,
                                        void *stream) {
    if (!p || !volt || !img || !b) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run_hier: NULL argument");
    if (p->hK == 0) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run_hier: no hierarchy set");
    if (!b->beams || !b->corr || (p->hx && (!b->vis || !b->xfft_img)) || (!p->he.empty() && !b->epic_img))
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run_hier: a buffer of the second level is NULL");
    const uintptr_t al = (uintptr_t)volt | (uintptr_t)img | (uintptr_t)b->beams | (uintptr_t)b->corr |
                         (uintptr_t)b->vis | (uintptr_t)b->xfft_img | (uintptr_t)b->epic_img;
    if (al & 15) return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_run_hier: buffers must be 16-byte aligned");
    if (hai_fault_injected("launch")) return hai_fail(HAI_ERR_CUDA, "hai_plan_run_hier: injected launch failure");
    HAI_CUDA_TRY(cudaSetDevice(p->ctx->device));
    if (!p->exec || p->g_volt != volt || p->g_img != img || !p->g_hier ||
        memcmp(&p->gb, b, sizeof(hai_plan_hier_buffers)) != 0) {
        const hai_status s = capture(p, volt, img, b);
        if (s != HAI_OK) return s;
    }
    const int pidx = prof_begin(p->ctx, (cudaStream_t)stream);
    HAI_CUDA_TRY(cudaGraphLaunch(p->exec, (cudaStream_t)stream));
    prof_end(p->ctx, pidx, (cudaStream_t)stream);
    return HAI_OK;
}

// Key of a plan in the autotune cache: the device and, per grid class, its
// side, stations, modelled cost (rounded) and the cadence shape.
static std::string plan_cache_key(const hai_plan *p) {
    cudaDeviceProp prop;
    std::string key = "unknown";
    if (cudaGetDeviceProperties(&prop, p->ctx->device) == cudaSuccess)
        key = "sm" + std::to_string(prop.major) + std::to_string(prop.minor) + "x" + std::to_string(prop.multiProcessorCount);
    key += " plan C" + std::to_string(p->C) + " T" + std::to_string(p->T);
    for (const auto &c : p->cls) {
        const double cost = std::accumulate(c.cost.begin(), c.cost.end(), 0.0);
        key += " N" + std::to_string(c.N) + ":" + std::to_string(c.stations.size()) + ":" +
               std::to_string((long long)llround(cost));
    }
    return key;
}

extern "C" hai_status hai_plan_autotune_cached(hai_plan *p, const int8_t *volt, float *img, int rounds,
                                               const char *cache_path, int *from_cache, void *stream) {
    if (!p || !volt || !img || rounds < 0 || !cache_path)
        return hai_fail(HAI_ERR_INVALID_ARG, "hai_plan_autotune_cached: bad argument");
    if (from_cache) *from_cache = 0;
    const std::string key = plan_cache_key(p);
    // "<key> | units <u_0> <u_1> ... | <ms>": the last matching line wins
    std::vector<int> units;
    if (FILE *f = fopen(cache_path, "r")) {
        char line[1024];
        while (fgets(line, sizeof(line), f)) {
            const char *bar = strstr(line, " | units ");
            if (!bar || std::string(line, bar - line) != key) continue;
            std::vector<int> u;
            const char *q = bar + 9;
            for (size_t k = 0; k < p->cls.size(); k++) {
                int v = 0, n = 0;
                if (sscanf(q, "%d%n", &v, &n) != 1 || v <= 0) {
                    u.clear();
                    break;
                }
                u.push_back(v);
                q += n;
            }
            if (u.size() == p->cls.size()) units = u;
        }
        fclose(f);
    }
    HAI_CUDA_TRY(cudaSetDevice(p->ctx->device));
    if (!units.empty()) {
        for (size_t k = 0; k < p->cls.size(); k++) {
            const hai_status st = class_upload_ranges(p, p->cls[k], std::min(units[k], p->cls[k].max_units));
            if (st != HAI_OK) return st;
        }
        drop_graph(p);
        if (from_cache) *from_cache = 1;
        return HAI_OK;
    }
    const hai_status st = hai_plan_autotune(p, volt, img, rounds, stream);
    if (st != HAI_OK) return st;
    if (FILE *f = fopen(cache_path, "a")) {
        fprintf(f, "%s | units", key.c_str());
        double worst = 0.0;
        for (const auto &c : p->cls) {
            fprintf(f, " %d", c.n_cta);
            worst = std::max(worst, c.measured_ms);
        }
        fprintf(f, " | %.3f ms slowest class alone\n", worst);
        fclose(f);
    }
    return HAI_OK;
}
