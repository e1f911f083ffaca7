// Factored numerator of the matched filter (Section 3.2, Eq. 5) for
// separable footprints, sm_103a.
//
// N_k(p) = sum_t sum_{a,b} u_x(a) u_y(b) y_t(p + s_{k,t} + (a, b)) is computed
// per frame as a row pass H(i, c) = sum_a u_x(a) R(i, c + a) over the staged
// window R, then a column pass N += sum_b u_y(b) H(i + b, c).  The row pass
// depends on the trajectory only through s_x and u_x, which every trajectory
// of a CTA shares (they have one v_x), so it is made once per frame for the
// whole CTA; the column pass is per trajectory.  Per (trajectory, pixel,
// frame) this costs 5 FMAs plus the row pass's share, against 25 FMAs for the
// general 5 x 5 stencil; the arithmetic is the same sum regrouped.
//
// Per pair of frames (t, t + 1): every thread waits for both windows (TMA
// boxes, mbarriers with bounded waits); the CTA's threads split both row
// passes into items of 16 outputs (the column phase is applied as an item
// reads the window, so the row-pass buffer holds exactly the tile's columns;
// items go to the last warps first, so the row-pass-only warps that round a
// CTA up to a multiple of 4 warps and the warps of empty slots take them);
// one CTA barrier; thread 0 refills both
// stages with frames t + stages and t + 1 + stages; each warp runs the
// column passes of its (trajectory slot, 32 x 32 sub-tile) for both frames:
// a lane owns 2 adjacent columns x 16 rows, reading 20 row-pass pairs with
// 64-bit loads (a half-warp reads one row's 32 columns, conflict-free).  Four
// row-pass buffers rotate, so one barrier per two frames orders both their
// writes and their reuse.  FP32 throughout, with the blocked accumulation of
// the general kernel (partials over 16 frames).  A CTA has at most
// kFacMaxWarps = 20 warps (96 registers a thread), enough for a whole v_x
// class of ten trajectories on two 32-row sub-tiles.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <type_traits>

#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {
namespace {

using namespace dev;

// The work of one CTA on one (output tile, trajectory group) of one search;
// false if it gave up (a bounded wait ran out; the device status word says
// why).  The CTA may have more warps than the search's layout uses (batched
// searches share one launch): the extra warps take part in the row pass and
// the barriers only.  `smem` is the CTA's 1024-aligned dynamic shared memory.
// Values of a staged window: FP32, or the 16-bit types of a bf16 / fp16
// weighted stack, converted exactly to FP32 as they are read.
template <typename E>
struct Win;
template <>
struct Win<float> {
    static constexpr int kPer = 4;  // values per 128-bit load
    static __device__ __forceinline__ void load(const void *p, float *v) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        v[0] = x.x;
        v[1] = x.y;
        v[2] = x.z;
        v[3] = x.w;
    }
    static __device__ __forceinline__ float one(const float *p) { return *p; }
};
template <>
struct Win<__nv_bfloat16> {
    static constexpr int kPer = 8;
    static __device__ __forceinline__ void load(const void *p, float *v) {
        const uint4 x = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {  // a bf16 is the high half of the FP32 with the same value
            v[2 * i] = __uint_as_float(w[i] << 16);
            v[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
        }
    }
    static __device__ __forceinline__ float one(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
};
template <>
struct Win<__half> {
    static constexpr int kPer = 8;
    static __device__ __forceinline__ void load(const void *p, float *v) {
        const uint4 x = *reinterpret_cast<const uint4 *>(p);
        const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            v[2 * i] = f.x;
            v[2 * i + 1] = f.y;
        }
    }
    static __device__ __forceinline__ float one(const __half *p) { return __half2float(*p); }
};

// One row-pass item: H(row, c0 .. c0 + 15) = sum_a u_x(a) R(row, c0 + M + c + a)
// for a column phase M known at compile time; src = R(row, c0), 16-byte
// aligned, dst = H(row, c0).  TAPS = 1 (single-tap footprints: the
// shift-stack filter) keeps the centre tap only.
template <int M, int TAPS, typename E>
__device__ __forceinline__ void row_item(const E *__restrict__ src, float *__restrict__ dst, float ux0,
                                         float ux1, float ux2, float ux3, float ux4) {
    constexpr int PER = Win<E>::kPer;
    constexpr int NL = (kFacItem + (TAPS == 1 ? 3 : 4) + M + PER - 1) / PER;  // 128-bit loads covering the inputs
    float v[PER * NL];
#pragma unroll
    for (int q = 0; q < NL; q++) Win<E>::load(src + PER * q, v + PER * q);
    float o[kFacItem];
#pragma unroll
    for (int c = 0; c < kFacItem; c++) {
        if (TAPS == 1) {
            o[c] = ux2 * v[M + c + 2];
        } else {
            float h = ux0 * v[M + c];
            h = fmaf(ux1, v[M + c + 1], h);
            h = fmaf(ux2, v[M + c + 2], h);
            h = fmaf(ux3, v[M + c + 3], h);
            o[c] = fmaf(ux4, v[M + c + 4], h);
        }
    }
#pragma unroll
    for (int q = 0; q < kFacItem / 4; q++)
        reinterpret_cast<float4 *>(dst)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
}

// The (group, tile) of CTA `cta` of the launch that computes segment p.seg,
// in the order tile row, tile column, group: the CTAs running at the same
// time then read the same frames of neighbouring tiles for every group,
// which keeps those frames in L2.  Tile rows are in reference coordinates (a
// trajectory's start pixel is the tile pixel minus its s_y at the segment's
// first frame) and start at the group's smallest such s_y; every group gets
// as many tile rows as the segment's widest spread needs,
// ceil((H + spread) / tile_h).  False if cta is past the last tile.
__device__ __forceinline__ bool fac_locate(const FacParams &p, int tw, long long cta, int &g, int &y0, int &x0,
                                           int &t0, int &t1) {
    const int4 *segs = reinterpret_cast<const int4 *>(p.segs);
    int spread = 0;
    for (int e = 0; e < p.G; e++) spread = max(spread, segs[(size_t)e * p.S + p.seg].w);
    const long long rows = (p.H + spread + p.th - 1) / p.th;
    if (cta >= rows * p.tiles_x * p.G) return false;
    g = (int)(cta % p.G);
    const long long rest = cta / p.G;
    const int4 sg = segs[(size_t)g * p.S + p.seg];
    y0 = sg.z + (int)(rest / p.tiles_x) * p.th;
    x0 = (int)(rest % p.tiles_x) * tw;
    t0 = sg.x;
    t1 = sg.y;
    return true;
}

// QG: the phase-plane form (phase-quantised banks, five taps, FP32 stacks):
// per frame the row pass, then one column pass per rounded y-phase present
// (a plane over the whole window), then one add per (trajectory, pixel)
// gathered from its phase's plane.
template <int TW, int TAPS, typename E, bool QG = false>
__device__ __forceinline__ bool fac_tile(const CUtensorMap &ymap, const FacParams &p, long long cta,
                                         unsigned char *smem) {
    static_assert(!QG || (TAPS == 5 && sizeof(E) == 4), "phase planes: five taps, FP32 stacks");
    constexpr bool k16 = sizeof(E) == 2;
    // window pitch (values) and row-pass layout
    constexpr int RP = k16 ? fac_rpitch16(TW) : fac_rpitch(TW), HP = fac_hpitch(TW), NI = fac_hcols(TW) / kFacItem;
    constexpr int R = kFacRecordChunk;
    constexpr int NSUBX = TW / 32;

    const int NS = p.ns, BH = p.bh, KT = p.kt;
    const int seg = p.seg;
    int g = 0, tile_y0 = 0, tile_x0 = 0, t0 = 0, t1 = 0;
    if (!fac_locate(p, TW, cta, g, tile_y0, tile_x0, t0, t1)) return true;  // uniform: nothing to do
    {
        // a tile row past every member's start pixels (groups with a smaller
        // spread than the segment's widest) has nothing to compute
        bool any = false;
        for (int w = 0; w < KT; w++) {
            if (p.members[(size_t)g * KT + w] < 0) continue;
            const int r = tile_y0 - p.refs[((size_t)g * p.S + seg) * KT + w];
            any |= r + p.th > 0 && r < p.H;
        }
        if (!any) return true;  // same for every thread of the CTA
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nsub = (p.th / 32) * NSUBX;
    // a slot's warps are consecutive, so they spread over the SM's four
    // schedulers and an empty slot leaves every scheduler the same work
    const int slot = warp / nsub, sub = warp % nsub;
    const int sub_y = sub / NSUBX, sub_x = sub % NSUBX;
    const uint32_t kBB = (uint32_t)fac_block_bytes(KT, QG ? p.npl : 0);

    const int SF = fac_stage_floats(TW, BH);                              // stage stride in floats (128-byte multiple)
    constexpr int EPF = 4 / (int)sizeof(E);                              // window values per float of a stage
    E *rwin = reinterpret_cast<E *>(smem);                               // [NS] windows of BH x RP values
    float *hbuf = reinterpret_cast<float *>(smem) + (size_t)NS * SF;     // [kFacHBufs][BH][HP] (QG: [1])
    float *pbuf = hbuf + (size_t)(QG ? 2 : kFacHBufs) * BH * HP;         // QG: [2][npl][BH][HP] phase planes
    unsigned char *fb = reinterpret_cast<unsigned char *>(pbuf + (size_t)(QG ? 2 * p.npl : 0) * BH * HP);  // [2][R]
    uint64_t *bars = reinterpret_cast<uint64_t *>(fb + 2 * R * kBB);
    int *last_issued = reinterpret_cast<int *>(bars + NS);
    int *bad_flag = last_issued + NS;

    const unsigned char *gblocks = p.blocks + (size_t)g * p.T * kBB;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(smem_u32(&bars[s]), 1);
            last_issued[s] = -1;
        }
        *bad_flag = status_now(p.status);  // an earlier CTA gave up: do not start
        fence_barrier_init();
    }
    __syncthreads();
    if (*bad_flag != 0) return false;  // same value for every thread of the CTA

    const uint32_t box_bytes = (uint32_t)BH * RP * sizeof(E);
    auto issue = [&](int f, int s, int roy, int rox) {
        const uint32_t bar = smem_u32(&bars[s]);
        const int nrec = (f % R == 0) ? min(R, p.T - f) : 0;  // the chunk's records ride on its first frame
        mbar_expect_tx(bar, box_bytes + (uint32_t)nrec * kBB);
        // a 16-bit window starts at a multiple of 8 columns (16 bytes; the tile
        // origin is a multiple of 32): one 4-column step left of rox when rox is
        // an odd multiple of 4, which the row pass's column phase cofs8 absorbs
        const int x = tile_x0 + (k16 ? (rox & ~7) : rox);
        tma_load_3d(smem_u32(rwin + (size_t)s * SF * EPF), &ymap, x, tile_y0 + roy, f, bar);
        if (nrec)
            bulk_load(smem_u32(fb + ((f / R) & 1) * R * kBB), gblocks + (size_t)f * kBB, (uint32_t)nrec * kBB, bar);
        last_issued[s] = f;
    };
    if (threadIdx.x == 0) {
        fence_proxy_async();
        for (int s = 0; s < NS && t0 + s < t1; s++) {
            const FrameHdr h = p.hdr[(size_t)g * p.T + t0 + s];
            issue(t0 + s, s, h.roy, h.rox);
        }
    }

    const int kk = warp < p.warps ? p.members[(size_t)g * KT + slot] : -1;
    // the slot's s_y at the segment's first frame; its start pixels are the
    // tile pixels minus that: a warp whose rows hold none is idle
    const int ref = kk >= 0 ? p.refs[((size_t)g * p.S + seg) * KT + slot] : 0;
    const int qrow = tile_y0 + 32 * sub_y - ref;
    const bool active = kk >= 0 && qrow + 32 > 0 && qrow < p.H && tile_x0 + 32 * sub_x < p.W;
    // five taps: lane = column pair cp (2 adjacent columns) x row half rh
    // (16 rows), acc / blk[r * 2 + j] at row 16 rh + r, column 2 cp + j;
    // single tap: lane = column, acc / blk[r] at row r
    const int cp = lane & 15, rh = lane >> 4;
    float acc[32], blk[32];
#pragma unroll
    for (int r = 0; r < 32; r++) {
        acc[r] = 0.f;
        blk[r] = 0.f;
    }
    auto record = [&](int f) { return fb + (((f / R) & 1) * R + f % R) * kBB; };
    auto column = [&](int f) {
        if (!active) return;
        const unsigned char *fblk = record(f);
        const FacSlot *fs = reinterpret_cast<const FacSlot *>(fblk + sizeof(FacHdr)) + slot;
        const float4 u4 = *reinterpret_cast<const float4 *>(fs->uy);
        const float2 u5 = *reinterpret_cast<const float2 *>(fs->uy + 4);  // u_y(2) and the row offset
        const float u[5] = {u4.x, u4.y, u4.z, u4.w, u5.x};
        const float *col = hbuf + (size_t)(f % kFacHBufs) * BH * HP + (32 * sub_y + 16 * rh + __float_as_int(u5.y)) * HP + 32 * sub_x + 2 * cp;
        // taps b = B0 .. B1 of the footprint (all five, or the centre one)
        constexpr int B0 = 2 - TAPS / 2, B1 = 2 + TAPS / 2;
#pragma unroll
        for (int i = B0; i < 16 + B1; i++) {
            const float2 h = *reinterpret_cast<const float2 *>(col + i * HP);
#pragma unroll
            for (int b = B0; b <= B1; b++) {
                const int r = i - b;
                if (r >= 0 && r < 16) {
                    blk[2 * r] = fmaf(u[b], h.x, blk[2 * r]);
                    blk[2 * r + 1] = fmaf(u[b], h.y, blk[2 * r + 1]);
                }
            }
        }
    };
    // single tap (both factors one-hot at the centre, exactly 1): the column
    // pass adds the window's values at the base pixel straight from the
    // stage, blk += R(row + oy + 2, column + 2 + cofs) -- the same sums in the
    // same order as the five-tap passes on such a table (zero taps add exact
    // zeros), so the results are bit-identical
    auto column_direct = [&](int f, int st) {
        if (!active) return;
        const unsigned char *fblk = record(f);
        const FacHdr *fh = reinterpret_cast<const FacHdr *>(fblk);
        const FacSlot *fs = reinterpret_cast<const FacSlot *>(fblk + sizeof(FacHdr)) + slot;
        const E *col = rwin + (size_t)st * SF * EPF + (32 * sub_y + fs->oy + 2) * RP + 32 * sub_x + lane + 2 +
                       (k16 ? fh->cofs8 : fh->cofs);
        if constexpr (k16) {
            const float bt = p.beta ? p.beta[f] : 1.f;  // a power of two: the products are exact
#pragma unroll
            for (int r = 0; r < 32; r++) blk[r] += bt * Win<E>::one(col + r * RP);
        } else {
#pragma unroll
            for (int r = 0; r < 32; r++) blk[r] += Win<E>::one(col + r * RP);
        }
    };
    // the row passes of frames f0 (stage s0) and f0 + 1 (stage s1, if it
    // exists) as one list of items: item it < n0 is (row, m) of frame f0
    auto row_pair = [&](int f0, int s0, int s1, bool two) {
        const FacHdr *h0 = reinterpret_cast<const FacHdr *>(record(f0));
        const FacHdr *h1 = reinterpret_cast<const FacHdr *>(record(two ? f0 + 1 : f0));
        const int n0 = h0->nrows * NI, n1 = two ? h1->nrows * NI : 0;
        for (int it = (int)blockDim.x - 1 - (int)threadIdx.x; it < n0 + n1; it += blockDim.x) {
            const bool second = it >= n0;
            const FacHdr *fh = second ? h1 : h0;
            const int f = second ? f0 + 1 : f0, st = second ? s1 : s0, j = second ? it - n0 : it;
            const int nrows = fh->nrows;
            const int m = (int)(((float)j + 0.5f) * fh->inv_nrows), row = j - m * nrows;
            const E *src = rwin + (size_t)st * SF * EPF + row * RP + kFacItem * m;
            float *dst = hbuf + (size_t)(QG ? (f & 1) : f % kFacHBufs) * BH * HP + row * HP + kFacItem * m;
            if constexpr (k16) {
                // the taps carry the frame's scale of a 16-bit weighted stack
                // (a power of two: u_x * beta is exact)
                const float bt = p.beta ? p.beta[f] : 1.f;
                const float ux0 = fh->ux[0] * bt, ux1 = fh->ux[1] * bt, ux2 = fh->ux[2] * bt,
                            ux3 = fh->ux[3] * bt, ux4 = fh->ux[4] * bt;
                switch (fh->cofs8) {
                    case 0: row_item<0, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 1: row_item<1, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 2: row_item<2, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 3: row_item<3, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 4: row_item<4, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 5: row_item<5, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 6: row_item<6, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    default: row_item<7, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                }
            } else {
                const float ux0 = fh->ux[0], ux1 = fh->ux[1], ux2 = fh->ux[2], ux3 = fh->ux[3], ux4 = fh->ux[4];
                switch (fh->cofs) {
                    case 0: row_item<0, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 1: row_item<1, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    case 2: row_item<2, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                    default: row_item<3, TAPS>(src, dst, ux0, ux1, ux2, ux3, ux4); break;
                }
            }
        }
    };

    // phase planes of frames f0 and f0 + 1 (if `two`): plane j row i =
    // sum_b u_j(b) H(i + b), rows 0 .. nrows - 5, items of 8 rows x 2
    // columns dealt over all threads (consecutive threads on consecutive
    // column pairs: conflict-free); frame f's planes go to set f & 1
    auto plane_pair = [&](int f0, bool two) {
        constexpr int PR = 8;  // rows per item
        constexpr int NCP = TW / 2;
        int n[2], nrc[2];
        for (int e = 0; e < 2; e++) {
            const FacHdr *fh = reinterpret_cast<const FacHdr *>(record(f0 + (two ? e : 0)));
            nrc[e] = (fh->nrows - 4 + PR - 1) / PR;
            n[e] = (e == 0 || two) ? fh->pad * nrc[e] * NCP : 0;
        }
        for (int it = threadIdx.x; it < n[0] + n[1]; it += blockDim.x) {
            const int e = it >= n[0], k = e ? it - n[0] : it, f = f0 + e;
            const unsigned char *fblk = record(f);
            const FacHdr *fh = reinterpret_cast<const FacHdr *>(fblk);
            const FacPlane *pl =
                reinterpret_cast<const FacPlane *>(fblk + sizeof(FacHdr) + (size_t)KT * sizeof(FacSlot));
            const int nrows = fh->nrows, prow = nrows - 4;
            const int cp = k % NCP, rest = k / NCP, rc = rest % nrc[e], j = rest / nrc[e];
            const float4 u4 = *reinterpret_cast<const float4 *>(pl[j].uy);
            const float u[5] = {u4.x, u4.y, u4.z, u4.w, pl[j].uy[4]};
            const float *src = hbuf + (size_t)(f & 1) * BH * HP + (size_t)(PR * rc) * HP + 2 * cp;
            float *dst = pbuf + ((size_t)(f & 1) * p.npl + j) * BH * HP + (size_t)(PR * rc) * HP + 2 * cp;
            float2 o[PR];
#pragma unroll
            for (int r = 0; r < PR; r++) o[r] = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < PR + 4; i++) {
                // rows past the frame's window hold nothing the stored rows use
                const float2 h = PR * rc + i < nrows ? *reinterpret_cast<const float2 *>(src + i * HP)
                                                     : make_float2(0.f, 0.f);
#pragma unroll
                for (int b = 0; b < 5; b++) {
                    const int r = i - b;
                    if (r >= 0 && r < PR) {
                        o[r].x = fmaf(u[b], h.x, o[r].x);
                        o[r].y = fmaf(u[b], h.y, o[r].y);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < PR; r++)
                if (PR * rc + r < prow) *reinterpret_cast<float2 *>(dst + (size_t)r * HP) = o[r];
        }
    };
    // the gather of frame f: each output adds its trajectory's plane value at
    // the row the column pass would have started from
    auto gather = [&](int f) {
        if (!active) return;
        const unsigned char *fblk = record(f);
        const FacSlot *fs = reinterpret_cast<const FacSlot *>(fblk + sizeof(FacHdr)) + slot;
        const float *col = pbuf + ((size_t)(f & 1) * p.npl + fs->plane) * BH * HP +
                           (32 * sub_y + 16 * rh + fs->oy) * HP + 32 * sub_x + 2 * cp;
#pragma unroll
        for (int r = 0; r < 16; r++) {
            const float2 v = *reinterpret_cast<const float2 *>(col + r * HP);
            blk[2 * r] += v.x;
            blk[2 * r + 1] += v.y;
        }
    };

    bool bad = false;
    int s = 0;  // stage of frame t and its phase
    uint32_t par = 0;
    if constexpr (QG) {
        // two frames at a time: row passes -> barrier -> planes -> barrier ->
        // gathers.  The next pair's row passes overwrite the row-pass
        // buffers only after the barrier that ends every thread's plane
        // work, and its planes the plane sets only after the barrier every
        // thread reaches past its gathers (frame f uses row-pass buffer and
        // plane set f & 1, which differ for the two frames of a pair)
        for (int t = t0; t < t1; t += 2) {
            const bool two = t + 1 < t1;
            const int s1 = (s + 1 == NS) ? 0 : s + 1;
            const uint32_t par1 = (s + 1 == NS) ? (par ^ 1u) : par;
            bool ready = mbar_wait(smem_u32(&bars[s]), par, 1, p.status);
            if (ready && two) ready = mbar_wait(smem_u32(&bars[s1]), par1, 1, p.status);
            if (ready) row_pair(t, s, s1, two);
            if (__syncthreads_or(!ready)) {
                bad = true;
                break;
            }
            if (threadIdx.x == 0) {
                fence_proxy_async();
                if (t + NS < t1) {
                    const FacHdr *fh = reinterpret_cast<const FacHdr *>(record(t));
                    issue(t + NS, s, fh->next_roy, fh->next_rox);
                }
                if (two && t + 1 + NS < t1) {
                    const FacHdr *fh = reinterpret_cast<const FacHdr *>(record(t + 1));
                    issue(t + 1 + NS, s1, fh->next_roy, fh->next_rox);
                }
            }
            plane_pair(t, two);
            __syncthreads();
            gather(t);
            if (two) gather(t + 1);
            if ((t - t0 + 2) % kFrameBlock == 0) {
#pragma unroll
                for (int r = 0; r < 32; r++) {
                    acc[r] += blk[r];
                    blk[r] = 0.f;
                }
            }
            s = (s1 + 1 == NS) ? 0 : s1 + 1;
            par = (s1 + 1 == NS) ? (par1 ^ 1u) : par1;
        }
    }
    for (int t = t0; t < t1 && !QG; t += 2) {  // column passes (the loop is empty for QG)
        const bool two = t + 1 < t1;
        const int s1 = (s + 1 == NS) ? 0 : s + 1;
        const uint32_t par1 = (s + 1 == NS) ? (par ^ 1u) : par;
        bool ready = mbar_wait(smem_u32(&bars[s]), par, 1, p.status);
        if (ready && two) ready = mbar_wait(smem_u32(&bars[s1]), par1, 1, p.status);
        if (TAPS == 1) {
            // the column passes read the stages themselves: they run before
            // the barrier that frees the stages for refilling
            if (ready) {
                column_direct(t, s);
                if (two) column_direct(t + 1, s1);
            }
        } else if (ready) {
            row_pair(t, s, s1, two);
        }
        if (__syncthreads_or(!ready)) {
            bad = true;
            break;
        }
        // every thread is done with stages s (and s1): refill them with frames t + NS (and t + 1 + NS)
        if (threadIdx.x == 0) {
            fence_proxy_async();
            if (t + NS < t1) {
                const FacHdr *fh = reinterpret_cast<const FacHdr *>(record(t));
                issue(t + NS, s, fh->next_roy, fh->next_rox);
            }
            if (two && t + 1 + NS < t1) {
                const FacHdr *fh = reinterpret_cast<const FacHdr *>(record(t + 1));
                issue(t + 1 + NS, s1, fh->next_roy, fh->next_rox);
            }
        }
        if (TAPS != 1) {
            column(t);
            if (two) column(t + 1);
        }
        if ((t - t0 + 2) % kFrameBlock == 0) {
#pragma unroll
            for (int r = 0; r < 32; r++) {
                acc[r] += blk[r];
                blk[r] = 0.f;
            }
        }
        // advance two stages
        s = (s1 + 1 == NS) ? 0 : s1 + 1;
        par = (s1 + 1 == NS) ? (par1 ^ 1u) : par1;
    }
    if (bad) {
        // let any copy still in flight land before the CTA's shared memory goes away
        if (threadIdx.x == 0) {
            for (int q = 0; q < NS; q++) {
                const int f = last_issued[q];
                if (f >= 0) mbar_wait(smem_u32(&bars[q]), (uint32_t)(((f - t0) / NS) & 1), 2, p.status);
            }
        }
        return false;
    }

    // Epilogue: this segment's numerator of each (trajectory, start pixel)
    // into the plane, stored by segment 0 and added by the later segments
    // (launched in order, so the sum follows the segment order); the start
    // pixel is the tile pixel minus the trajectory's s_y at the segment's
    // first frame, and each is reached by one CTA of the launch
    const int64_t P = p.H * p.W;
    if (kk >= 0) {
        float *plane = p.plane + (size_t)kk * P;
#pragma unroll
        for (int r = 0; r < 32; r++) {
            const int64_t px = tile_x0 + 32 * sub_x + (TAPS == 1 ? lane : 2 * cp + (r & 1));
            const int64_t py = (int64_t)tile_y0 + 32 * sub_y + (TAPS == 1 ? r : 16 * rh + (r >> 1)) - ref;
            if (py >= 0 && py < p.H && px < p.W) {
                const int64_t q = py * p.W + px;
                plane[q] = seg == 0 ? acc[r] + blk[r] : plane[q] + (acc[r] + blk[r]);
            }
        }
    }
    // the barriers may be initialised again for this CTA's next tile
    if (threadIdx.x == 0)
        for (int q = 0; q < NS; q++) mbar_inval(smem_u32(&bars[q]));
    return true;
}

template <int TW, int TAPS, typename E>
__global__ void __launch_bounds__(32 * kFacMaxWarps, 1)
    k_numerator_fac(const __grid_constant__ CUtensorMap ymap, const FacParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    fac_tile<TW, TAPS, E>(ymap, p, (long long)blockIdx.x, smem);
}

// The factored numerator with phase planes (phase-quantised banks).
template <int TW>
__global__ void __launch_bounds__(32 * kFacMaxWarps, 1)
    k_numerator_fac_planes(const __grid_constant__ CUtensorMap ymap, const FacParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    fac_tile<TW, 5, float, true>(ymap, p, (long long)blockIdx.x, smem);
}

// Persistent factored numerator over a batch of searches: one CTA per SM
// takes (search, tile, group) work entries from a global counter until the
// list is exhausted, running the same per-tile code as k_numerator_fac.
template <int TW, typename E>
__global__ void __launch_bounds__(32 * kFacMaxWarps, 1)
    k_numerator_fac_batch(const CUtensorMap *__restrict__ maps, const __grid_constant__ FacBatchArgs a,
                          unsigned long long *counter) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ long long work;
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long w = (long long)atomicAdd(counter, 1ull);
            int lo = 0, hi = a.n_items - 1;  // last item whose cta_begin <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.items[mid].cta_begin <= w) lo = mid;
                else hi = mid - 1;
            }
            work = w;
            item = lo;
        }
        __syncthreads();
        const long long w = work;
        const int i = item;
        __syncthreads();
        if (w >= a.total) break;
        const FacParams &p = a.items[i].p;
        // the five-tap code: single-tap footprints give the same sums (zero
        // taps add exact zeros), so a batch of mixed tables needs one kernel
        if (!fac_tile<TW, 5, E>(maps[i], p, w - a.items[i].cta_begin, smem)) break;
        __syncthreads();
    }
}

// Per pixel: SNR_k = N_k / sqrt(D_k) over the filters with D_k > 0, the
// maximum and the smallest k attaining it (-1 and 0 where no filter has
// D > 0), and optionally the SNR cube (0 where D = 0).  V consecutive pixels
// per thread (V = 4 when P is a multiple of 4: 128-bit loads).
template <int V>
__global__ void k_finalize_planes(const float *__restrict__ plane, const float *__restrict__ isd, int K, int64_t P,
                                  float *__restrict__ snr_max, int32_t *__restrict__ argmax,
                                  float *__restrict__ snr_all, const int *slot, int *global_status) {
    using VecT = typename std::conditional<V == 4, float4, float>::type;
    // a failure of this search also goes into the device-wide word
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int s = *(const volatile int *)slot;
        if (s != 0) atomicCAS(global_status, 0, s);
    }
    const int64_t n = P / V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float best[V];
        int arg[V];
#pragma unroll
        for (int v = 0; v < V; v++) {
            best[v] = 0.f;
            arg[v] = -1;
        }
        for (int k = 0; k < K; k++) {
            const VecT xv = reinterpret_cast<const VecT *>(plane + (int64_t)k * P)[i];
            const VecT dv = reinterpret_cast<const VecT *>(isd + (int64_t)k * P)[i];
            const float *x = reinterpret_cast<const float *>(&xv);
            const float *d = reinterpret_cast<const float *>(&dv);
            float snr[V];
#pragma unroll
            for (int v = 0; v < V; v++) {
                snr[v] = x[v] * d[v];
                if (d[v] > 0.f && (arg[v] < 0 || snr[v] > best[v])) {
                    best[v] = snr[v];
                    arg[v] = k;
                }
                if (d[v] <= 0.f) snr[v] = 0.f;
            }
            if (snr_all) reinterpret_cast<VecT *>(snr_all + (int64_t)k * P)[i] = *reinterpret_cast<const VecT *>(snr);
        }
#pragma unroll
        for (int v = 0; v < V; v++) {
            snr_max[i * V + v] = arg[v] < 0 ? 0.f : best[v];
            argmax[i * V + v] = arg[v];
        }
    }
}

}  // namespace

int fac_finalize_enqueue(const float *plane, const float *isd, int K, int64_t P, float *snr_max, int32_t *argmax,
                         float *snr_all, const int *slot, int *global_status, void *stream, char *err,
                         size_t errlen) {
    if (P <= 0) return 0;
    const bool vec = P % 4 == 0 && (uintptr_t)snr_all % 16 == 0;
    const int64_t items = vec ? P / 4 : P;
    int64_t blocks = (items + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (vec)
        k_finalize_planes<4><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(plane, isd, K, P, snr_max, argmax,
                                                                                 snr_all, slot, global_status);
    else
        k_finalize_planes<1><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(plane, isd, K, P, snr_max, argmax,
                                                                                 snr_all, slot, global_status);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "k_finalize_planes: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

namespace {

typedef void (*FacBatchKernel)(const CUtensorMap *, const FacBatchArgs, unsigned long long *);
typedef void (*FacKernel)(const CUtensorMap, const FacParams);

FacBatchKernel pick_fac_batch(int tw, int etype) {
    if (etype == MF_BF16) return tw == 64 ? k_numerator_fac_batch<64, __nv_bfloat16> : k_numerator_fac_batch<32, __nv_bfloat16>;
    if (etype == MF_F16) return tw == 64 ? k_numerator_fac_batch<64, __half> : k_numerator_fac_batch<32, __half>;
    return tw == 64 ? k_numerator_fac_batch<64, float> : k_numerator_fac_batch<32, float>;
}

template <typename E>
FacKernel pick_fac_e(int tw, int taps) {
    return tw == 64 ? (taps == 1 ? k_numerator_fac<64, 1, E> : k_numerator_fac<64, 5, E>)
                    : (taps == 1 ? k_numerator_fac<32, 1, E> : k_numerator_fac<32, 5, E>);
}

FacKernel pick_fac(int tw, int taps, int etype, bool planes) {
    if (planes) return tw == 64 ? k_numerator_fac_planes<64> : k_numerator_fac_planes<32>;
    if (etype == MF_BF16) return pick_fac_e<__nv_bfloat16>(tw, taps);
    if (etype == MF_F16) return pick_fac_e<__half>(tw, taps);
    return pick_fac_e<float>(tw, taps);
}

}  // namespace

int fac_batch_attr(int tw, int etype, size_t smem, char *err, size_t errlen) {
    cudaError_t e = cudaFuncSetAttribute(pick_fac_batch(tw, etype), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaFuncSetAttribute(smem=%zu): %s", smem, cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

int fac_batch_enqueue(const void *maps, const FacBatchItem *items, int n_items, long long total,
                      unsigned long long *counter, int tw, int etype, int warps, size_t smem, int grid, void *stream,
                      char *err, size_t errlen) {
    FacBatchKernel kern = pick_fac_batch(tw, etype);
    cudaError_t e;
    if (total <= 0 || grid <= 0) return 0;
    if (n_items < 1 || n_items > kFacBatchArgItems) {
        snprintf(err, errlen, "k_numerator_fac_batch: %d searches in one launch (1 .. %d)", n_items,
                 kFacBatchArgItems);
        return (int)cudaErrorInvalidValue;
    }
    static thread_local FacBatchArgs args;  // 28 KB: off the stack
    std::memcpy(args.items, items, (size_t)n_items * sizeof(FacBatchItem));
    args.total = total;
    args.n_items = n_items;
    kern<<<grid, warps * 32, smem, (cudaStream_t)stream>>>(reinterpret_cast<const CUtensorMap *>(maps), args,
                                                           counter);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "k_numerator_fac_batch: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

int fac_enqueue(const void *tensor_map, const FacParams &p, int tw, int taps, int etype, int warps, size_t smem,
                long long nblocks, void *stream, char *err, size_t errlen) {
    const CUtensorMap &map = *reinterpret_cast<const CUtensorMap *>(tensor_map);
    FacKernel kern = pick_fac(tw, taps, etype, p.npl > 0);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaFuncSetAttribute(smem=%zu): %s", smem, cudaGetErrorString(e));
        return (int)e;
    }
    if (nblocks <= 0) return 0;
    kern<<<(unsigned)nblocks, warps * 32, smem, (cudaStream_t)stream>>>(map, p);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "k_numerator_fac: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

}  // namespace mf
