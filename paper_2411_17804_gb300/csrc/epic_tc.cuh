// Pieces shared by the tensor-core EPIC kernels (epic_tc.cu for N = 32 and
// 64, epic_tc128.cu for N = 128) and the batched plan (plan.cu).
//
// A launch images one or more stations ("a class": same grid side) over one
// cadence of C channels x T samples.  The flattened sample index runs over
// blocks (station, channel) of T samples each, block = station * C + channel,
// and every CTA (or CTA group) takes a contiguous range of it.
#pragma once

#include <stdint.h>

#include <vector>

#include "hai_internal.h"

// Static shared memory of the tensor-core EPIC kernels (mbarriers, TMEM
// address), which the device's per-block opt-in limit also has to hold.
constexpr size_t kStaticSmem = 1024;

// One station of a launch, in device memory.
struct TcStation {
    const uint8_t *table;   // gather table (GatherLayout) in global memory
    long long volt_off;     // byte offset of the station's voltages [C][T][2][ne][2] int8
    long long img_off;      // float offset of the station's images [C][4][N][N]
    int ne;                 // elements
    int ntile, nent;        // gather tiles and entries
    uint32_t table_bytes;   // multiple of 16
};

// One step of a CTA's range: samples [t, t + nv) of channel chan of station
// stn (a step never straddles a block); src = its first voltage byte.
struct TcStep {
    int stn, chan, t, nv, ne;
    const int8_t *src;
    __device__ long long blk(int C) const { return (long long)stn * C + chan; }
};

// Walks a CTA's range [f, end) of the flattened index step by step, keeping
// the current station's element count and voltage offset in registers: one
// division at the start, none per step, a station-record load only when the
// station changes.
struct TcWalker {
    const int8_t *volt;
    const TcStation *stations;
    int C, T;
    long long f, end;
    int stn, chan, t, ne;
    long long volt_off;
    __device__ void init(const int8_t *v, const TcStation *st, int C_, int T_, long long s0, long long s1) {
        volt = v;
        stations = st;
        C = C_;
        T = T_;
        f = s0;
        end = s1;
        const long long blk = s0 / T;
        t = (int)(s0 - blk * T);
        stn = (int)(blk / C);
        chan = (int)(blk - (long long)stn * C);
        ne = 0;
        volt_off = 0;
        if (f < end) load();
    }
    __device__ void load() {
        ne = stations[stn].ne;
        volt_off = stations[stn].volt_off;
    }
    __device__ TcStep next(int sps) {
        TcStep s;
        s.stn = stn;
        s.chan = chan;
        s.t = t;
        s.nv = (int)min((long long)min(sps, T - t), end - f);
        s.ne = ne;
        s.src = volt + volt_off + ((long long)chan * T + t) * 4ll * ne;
        f += s.nv;
        t += s.nv;
        if (t == T) {
            t = 0;
            if (++chan == C) {
                chan = 0;
                ++stn;
                if (f < end) load();
            }
        }
        return s;
    }
};

// Start of a step's voltages rounded down to 16 bytes when the layout has
// guard bytes (delta = bytes skipped).
__device__ __forceinline__ const int8_t *tc_aligned_src(const int8_t *src, int guard, uint32_t &delta) {
    delta = guard ? (uint32_t)((uintptr_t)src & 15u) : 0u;
    return src - delta;
}

// Steps of size `sps` in the range [s0, s1): whole blocks of T samples.
__device__ __forceinline__ int tc_count_steps(long long s0, long long s1, int T, int sps) {
    int n = 0;
    for (long long f = s0; f < s1;) {
        const long long lim = min((f / T + 1) * (long long)T, s1);
        n += (int)((lim - f + sps - 1) / sps);
        f = lim;
    }
    return n;
}

// Gather table of the gridding step.  The non-empty cells of the kernel's
// bounding box are dealt into tiles of 32 (one per warp lane), sorted by
// entry count so a tile's lanes run the same number of slots; a tile's
// entries are stored slot-major, entry (slot k, lane l) at tile_base + 32 k
// + l, with zero-weight padding.
//   cell offsets   uint32 [ntile * 32]  byte offset of the lane's cell in the
//                                       stage-1 operand (field 0), or
//                                       0xffffffff for an unused lane
//   tile bases     int32 [ntile + 1]    first entry of each tile
//   warp ranges    int32 [kGatherWarps + 1]  warp w grids tiles [r[w], r[w+1]);
//                                       tiles are dealt to the warps by
//                                       longest-first (slots + 1 per tile)
//   (pad to 16)
//   weights        float2 [nent]        a + ib = conj(W~)
//   elements       uint16 [nent]
constexpr int kGatherWarps = 7;
struct GatherLayout {
    uint32_t off_cell, off_base, off_warp, off_w, off_e, bytes;
};
__host__ __device__ inline GatherLayout gather_layout(int ntile, int nent) {
    GatherLayout t;
    t.off_cell = 0;
    t.off_base = 4u * 32u * ntile;
    t.off_warp = t.off_base + 4u * (ntile + 1);
    t.off_w = (t.off_warp + 4u * (kGatherWarps + 1) + 15u) & ~15u;
    t.off_e = t.off_w + 8u * nent;
    t.bytes = (t.off_e + 2u * nent + 15u) & ~15u;
    return t;
}

// Builds the gather table of one station from its CSR cell lists (cells of
// the box row-major, cstart[box_w * box_h + 1]).  Cell (x, y) of the box
// lands at byte tc::off_kmajor(y, 2 x, k_stride, mn_stride) of the stage-1
// operand.
// n_warps (<= kGatherWarps) of the front warps get tiles; the others none.
void epic_tc_build_gather(int box_w, int box_h, const std::vector<int32_t> &cstart,
                          const std::vector<int32_t> &elem, const std::vector<float2> &w, uint32_t k_stride,
                          uint32_t mn_stride, std::vector<uint8_t> &out, int &ntile, int &nent,
                          int n_warps = kGatherWarps);

// fp16 W'[j][l] = (-1)^j exp(+2 pi i l j / N) as a real matrix entry: row
// (c_out, l), column (j, c_in) of the complex product y = W'^T x written for
// (re, im) pairs.
double epic_tc_dft_entry(int N, int c_out, int l, int j, int c_in);

// DFT operands of the tensor-core kernels for grid side N (built once per
// context, device memory owned by the context).
const void *epic_tc_dft(hai_ctx *ctx, int N, bool bf16 = false);
hai_status epic_tc_dft_prepare(hai_ctx *ctx, int N);

// Launchers over a list of stations of one grid side.  cta_begin (device,
// n_cta + 1 flat sample indices) gives each CTA's range; when it is null the
// ranges are b * len.  direct = 1: every block lies inside one CTA's range
// and is written straight into the station's image (with accumulate);
// direct = 0: blocks go to two partial slots per CTA for epic_reduce.
// guard = 1: every station's voltage block has 16 spare bytes before and
// after it, so voltage copies may round their start down and their end up
// to 16 bytes.
struct TcLaunch {
    const int8_t *volt;
    float *img;
    const TcStation *stations;
    int n_station;
    int ne_max;
    uint32_t table_max;
    const long long *cta_begin;
    long long len;
    int n_cta;
    int C, T;
    int direct, accumulate, guard;
    float *partials;
    int no_attr;            // 1: the kernel's shared-memory attribute is already set
    int split;              // 1: hi/lo split products (N = 32, 64)
    int bf16;               // 1: BF16 operands (N = 32, 64)
};
// Raises the kernel's dynamic shared-memory limit to the device's.
hai_status epic_tc_set_attr(hai_ctx *ctx, int N);
hai_status epic_tc_run(hai_ctx *ctx, int N, const TcLaunch &l, cudaStream_t st);
size_t epic_tc_smem(hai_ctx *ctx, int N, int ne_max, uint32_t table_max);
// Stage-1 operand strides of the gather table for grid side N.
void epic_tc_a1_strides(int N, uint32_t &k_stride, uint32_t &mn_stride);
// CTAs that image one channel together (1, or 4 for N = 128).
int epic_tc_group(int N);
hai_status epic_tc128_run(hai_ctx *ctx, const TcLaunch &l, cudaStream_t st);
hai_status epic_tc128_set_attr(hai_ctx *ctx);
size_t epic_tc128_smem(int ne_max, uint32_t table_max);
// Per-rank gather blob of one station for the N = 128 kernel;
// max_rank_bytes = the largest rank table (what a CTA keeps in shared memory).
void epic_tc128_build_blob(int box_w, int box_h, const std::vector<int32_t> &cstart,
                           const std::vector<int32_t> &elem, const std::vector<float2> &w,
                           std::vector<uint8_t> &out, uint32_t &max_rank_bytes, long long &max_rank_entries);
// Clusters of the N = 128 kernel resident at once (0 if it cannot run).
int epic_tc128_max_groups(hai_ctx *ctx, int ne_max, uint32_t table_max);
