// Device side of libmf: the matched-filter search of Ganapathi (2022),
// Section 3.2 (Eq. 5 and the maximum over the filter bank), for sm_103a.
//
// Kernels, in launch order:
//   k_lambda       inverse variance lambda = (1 - m) / sigma^2 into a zero-
//                  padded image (Section 3.2 noise model; clipped pixels and
//                  pixels outside the frame weigh 0);
//   k_weight       y_t = lambda * r_t, the inverse-variance weighted stack;
//   k_denominator  D_k(p) = sum_t sum_ab W^2 lambda, from runs of frames with
//                  a constant base shift, FP32 products accumulated in FP64;
//                  stores 1 / sqrt(D);
//   k_numerator    N_k(p) = sum_t sum_ab W y_t, the gather stencil: frame
//                  windows staged in shared memory by TMA and reused by the
//                  eight trajectories of a CTA, 25 FP32 FMAs per
//                  (trajectory, pixel, frame); epilogue forms SNR, reduces the
//                  max / argmax over the CTA's trajectories and merges it into
//                  a per-pixel 64-bit key with atomicMax;
//   k_finalize     key -> (snr_max, argmax).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "mf_internal.h"

namespace mf {

// Device status word: 0, or the code of a bounded wait that gave up.
__device__ int g_status;

namespace {

constexpr long long kWaitCycles = 1ll << 31;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ int status_now() { return *(volatile int *)&g_status; }

// Wait for a phase of an mbarrier, giving up after kWaitCycles or as soon as
// another CTA has recorded a failure; on giving up the device status word
// records `code` (if nothing was recorded before).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (unsigned it = 1;; it++) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && status_now() != 0) return false;
        if (clock64() - t0 > kWaitCycles) {
            atomicCAS(&g_status, 0, code);
            return false;
        }
    }
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Order-preserving 64-bit key: larger SNR first, then smaller k.  Any valid
// key is nonzero, so 0 means "no filter with D > 0".
__device__ __forceinline__ unsigned long long pack_key(float snr, int k) {
    uint32_t b = __float_as_uint(snr);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    return ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)k);
}

template <typename T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }

// ------------------------------------------------------------- lambda ---

__global__ void k_lambda(const float *__restrict__ sigma, const uint8_t *__restrict__ mask, int64_t H,
                         int64_t W, int64_t pad, int64_t lw, int64_t lh, float *__restrict__ lam) {
    const int64_t n = lw * lh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t yy = i / lw - pad, xx = i % lw - pad;
        float v = 0.f;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
            const int64_t q = yy * W + xx;
            const float s = sigma[q];
            const bool m = mask ? (mask[q] != 0) : false;
            if (!m && s > 0.f && isfinite(s)) v = (float)(1.0 / ((double)s * (double)s));
        }
        lam[i] = v;
    }
}

// ------------------------------------------------------------- weight ---

template <typename TIn>
__global__ void k_weight(const TIn *__restrict__ r, int64_t fstride, int64_t rstride,
                         const float *__restrict__ scale, const float *__restrict__ lam, int64_t pad, int64_t lw,
                         float *__restrict__ y, int64_t T, int64_t H, int64_t W, int64_t yp) {
    const int64_t wq = (W + 3) / 4;
    const int64_t n = T * H * wq;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xq = i % wq;
        const int64_t rest = i / wq;
        const int64_t yy = rest % H;
        const int64_t t = rest / H;
        const float sc = scale ? scale[t] : 1.f;
        const float *lrow = lam + (yy + pad) * lw + pad;
        const TIn *rrow = r + t * fstride + yy * rstride;
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t x = xq * 4 + j;
            o[j] = (x < W) ? lrow[x] * (sc * to_f32(rrow[x])) : 0.f;
        }
        *reinterpret_cast<float4 *>(y + (t * H + yy) * yp + xq * 4) = make_float4(o[0], o[1], o[2], o[3]);
    }
}

// -------------------------------------------------------- denominator ---

// One warp per (32 x 32 tile, trajectory); lane (tx, ty) owns a 4 x 8 block.
__global__ void __launch_bounds__(128) k_denominator(const float *__restrict__ lam, int64_t lw, int64_t pad,
                                                     const SegRec *__restrict__ segs,
                                                     const int32_t *__restrict__ seg_off, int64_t H, int64_t W,
                                                     int tiles_x, int tiles, float *__restrict__ isd) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x * 4 + warp;
    if (tile >= tiles) return;
    const int k = blockIdx.y;
    const int tx = lane & 3, ty = lane >> 2;
    const int64_t y0 = (int64_t)(tile / tiles_x) * kTile + kMicroRows * ty;
    const int64_t x0 = (int64_t)(tile % tiles_x) * kTile + kMicroCols * tx;
    double d[kMicroRows][kMicroCols];
    float blk[kMicroRows][kMicroCols];
#pragma unroll
    for (int r = 0; r < kMicroRows; r++)
#pragma unroll
        for (int c = 0; c < kMicroCols; c++) {
            d[r][c] = 0.0;
            blk[r][c] = 0.f;
        }
    const int j0 = seg_off[k], j1 = seg_off[k + 1];
    int cnt = 0;
    for (int j = j0; j < j1; j++) {
        const SegRec *sr = segs + j;
        float w[28];
        const float4 *w4 = reinterpret_cast<const float4 *>(sr->w2);
#pragma unroll
        for (int i = 0; i < 7; i++) {
            const float4 v = __ldg(w4 + i);
            w[4 * i + 0] = v.x;
            w[4 * i + 1] = v.y;
            w[4 * i + 2] = v.z;
            w[4 * i + 3] = v.w;
        }
        const int sx = __float_as_int(w[25]);
        const int sy = __float_as_int(w[26]);
        const float *base = lam + (y0 + sy - 2 + pad) * lw + (x0 + sx - 2 + pad);
#pragma unroll
        for (int i = 0; i < kMicroRows + 4; i++) {
            float v[kMicroCols + 4];
#pragma unroll
            for (int c = 0; c < kMicroCols + 4; c++) v[c] = __ldg(base + i * lw + c);
#pragma unroll
            for (int r = 0; r < kMicroRows; r++) {
                const int a = i - r;
                if (a < 0 || a > 4) continue;
#pragma unroll
                for (int c = 0; c < kMicroCols; c++)
#pragma unroll
                    for (int b = 0; b < 5; b++) blk[r][c] = fmaf(w[a * 5 + b], v[c + b], blk[r][c]);
            }
        }
        if (++cnt == kSegBlock) {
            cnt = 0;
#pragma unroll
            for (int r = 0; r < kMicroRows; r++)
#pragma unroll
                for (int c = 0; c < kMicroCols; c++) {
                    d[r][c] += (double)blk[r][c];
                    blk[r][c] = 0.f;
                }
        }
    }
    const int64_t P = H * W;
#pragma unroll
    for (int r = 0; r < kMicroRows; r++)
#pragma unroll
        for (int c = 0; c < kMicroCols; c++) {
            const double dd = d[r][c] + (double)blk[r][c];
            const int64_t py = y0 + r, px = x0 + c;
            if (py < H && px < W) isd[(int64_t)k * P + py * W + px] = dd > 0.0 ? rsqrtf((float)dd) : 0.f;
        }
}

// ---------------------------------------------------------- numerator ---

struct NumParams {
    const FrameBlock *blocks;  // [G][T]
    const FrameHdr *hdr;       // [G][T]
    const float *isd;          // [K][H][W]
    unsigned long long *keys;  // [H][W]
    float *snr_all;            // [K][H][W] or null
    int T, G;
    int64_t H, W;
    int tiles_x;
    int S, BH;
};

// The 4 x 8 block of one lane for one (trajectory, frame): 8 window rows of
// 12 values each, 25 FMAs per output.
__device__ __forceinline__ void stencil_4x8(const float *__restrict__ base, int S, const float (&w)[28],
                                            float (&blk)[kMicroRows][kMicroCols]) {
#pragma unroll
    for (int i = 0; i < kMicroRows + 4; i++) {
        float v[kMicroCols + 4];
#pragma unroll
        for (int c = 0; c < kMicroCols + 4; c++) v[c] = base[i * S + c];
#pragma unroll
        for (int r = 0; r < kMicroRows; r++) {
            const int a = i - r;
            if (a < 0 || a > 4) continue;
#pragma unroll
            for (int c = 0; c < kMicroCols; c++)
#pragma unroll
                for (int b = 0; b < 5; b++) blk[r][c] = fmaf(w[a * 5 + b], v[c + b], blk[r][c]);
        }
    }
}

template <int KG, int NS>
__global__ void __launch_bounds__(KG * 32, 2) k_numerator(const __grid_constant__ CUtensorMap ymap,
                                                          const NumParams p) {
    extern __shared__ unsigned char smem_raw[];
    const uintptr_t base_addr = ((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023;
    float *win = reinterpret_cast<float *>(base_addr);
    const int win_floats = p.BH * p.S;
    FrameBlock *fb = reinterpret_cast<FrameBlock *>(win + NS * win_floats);
    unsigned long long *red = reinterpret_cast<unsigned long long *>(fb + NS);
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + kTile * kTile);
    int *cnt = reinterpret_cast<int *>(bars + NS);
    int *last_issued = cnt + NS;
    int *bad_flag = last_issued + NS;

    const int g = (int)(blockIdx.x % (unsigned)p.G);
    const int tile = (int)(blockIdx.x / (unsigned)p.G);
    const int tile_y0 = (tile / p.tiles_x) * kTile;
    const int tile_x0 = (tile % p.tiles_x) * kTile + kTileOriginX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = lane & 3, ty = lane >> 2;
    const FrameBlock *gblocks = p.blocks + (size_t)g * p.T;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(smem_u32(&bars[s]), 1);
            cnt[s] = 0;
            last_issued[s] = -1;
        }
        *bad_flag = status_now();  // an earlier CTA gave up: do not start
        fence_barrier_init();
    }
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) red[i] = 0ull;
    __syncthreads();
    if (*bad_flag != 0) return;  // same value for every thread of the CTA

    // Load frame f into stage s: the rows the group's window needs at frame f
    // (TMA, zero fill outside the frame) and the frame's slot records.
    auto issue = [&](int f, int s, FrameHdr h) {
        const uint32_t bar = smem_u32(&bars[s]);
        const int nl = h.nrows / kLoadRows;
        const uint32_t row_bytes = (uint32_t)kLoadRows * p.S * 4;
        mbar_expect_tx(bar, nl * row_bytes + (uint32_t)sizeof(FrameBlock));
        const uint32_t dst = smem_u32(win + (size_t)s * win_floats);
        for (int l = 0; l < nl; l++)
            tma_load_3d(dst + l * row_bytes, &ymap, tile_x0 + h.rox, tile_y0 + h.roy + l * kLoadRows, f, bar);
        bulk_load(smem_u32(&fb[s]), gblocks + f, (uint32_t)sizeof(FrameBlock), bar);
        last_issued[s] = f;
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS && s < p.T; s++) issue(s, s, p.hdr[(size_t)g * p.T + s]);
    }

    float acc[kMicroRows][kMicroCols], blk[kMicroRows][kMicroCols];
#pragma unroll
    for (int r = 0; r < kMicroRows; r++)
#pragma unroll
        for (int c = 0; c < kMicroCols; c++) {
            acc[r][c] = 0.f;
            blk[r][c] = 0.f;
        }
    int kk = -1;
    bool bad = false;
    for (int t = 0; t < p.T; t++) {
        const int s = t % NS;
        if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)((t / NS) & 1), 1)) {
            bad = true;
            break;
        }
        const SlotRec &rec = fb[s].slot[warp];
        kk = rec.k;
        if (kk >= 0) {
            float w[28];
            const float4 *w4 = reinterpret_cast<const float4 *>(rec.taps);
#pragma unroll
            for (int i = 0; i < 7; i++) {
                const float4 v = w4[i];
                w[4 * i + 0] = v.x;
                w[4 * i + 1] = v.y;
                w[4 * i + 2] = v.z;
                w[4 * i + 3] = v.w;
            }
            const int offy = __float_as_int(w[25]);
            const int offx = __float_as_int(w[26]);
            const float *base =
                win + (size_t)s * win_floats + (offy + kMicroRows * ty) * p.S + offx + kMicroCols * tx + ty;
            stencil_4x8(base, p.S, w, blk);
        }
        if ((t + 1) % kFrameBlock == 0) {
#pragma unroll
            for (int r = 0; r < kMicroRows; r++)
#pragma unroll
                for (int c = 0; c < kMicroCols; c++) {
                    acc[r][c] += blk[r][c];
                    blk[r][c] = 0.f;
                }
        }
        // Release stage s; the last warp to release it loads frame t + NS.
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int prev = atomicAdd(&cnt[s], 1);
            if (prev == KG - 1) {
                cnt[s] = 0;
                if (t + NS < p.T) {
                    const FrameHdr h = fb[s].next;
                    fence_proxy_async();
                    issue(t + NS, s, h);
                }
            }
        }
    }
    if (bad) atomicExch(bad_flag, 1);
    __syncthreads();
    if (*bad_flag) {
        // Let any copy still in flight land before the CTA's shared memory goes away.
        if (threadIdx.x == 0) {
            for (int s = 0; s < NS; s++) {
                const int f = last_issued[s];
                if (f >= 0) mbar_wait(smem_u32(&bars[s]), (uint32_t)((f / NS) & 1), 2);
            }
        }
        return;
    }

    const int64_t P = p.H * p.W;
#pragma unroll
    for (int r = 0; r < kMicroRows; r++)
#pragma unroll
        for (int c = 0; c < kMicroCols; c++) {
            const float n = acc[r][c] + blk[r][c];
            const int64_t py = tile_y0 + kMicroRows * ty + r;
            const int64_t px = tile_x0 + kMicroCols * tx + ty + c;
            if (kk >= 0 && py < p.H && px >= 0 && px < p.W) {
                const int64_t q = py * p.W + px;
                const float isd = p.isd[(int64_t)kk * P + q];
                const float snr = n * isd;
                if (p.snr_all) p.snr_all[(int64_t)kk * P + q] = isd > 0.f ? snr : 0.f;
                if (isd > 0.f)
                    atomicMax(&red[(kMicroRows * ty + r) * kTile + kMicroCols * tx + c], pack_key(snr, kk));
            }
        }
    __syncthreads();
    for (int i = threadIdx.x; i < kTile * kTile; i += blockDim.x) {
        const unsigned long long key = red[i];
        if (key == 0ull) continue;
        const int ly = i / kTile, lx = i % kTile;
        const int64_t py = tile_y0 + ly;
        const int64_t px = tile_x0 + lx + ly / kMicroRows;
        atomicMax(&p.keys[py * p.W + px], key);
    }
}

// ----------------------------------------------------------- finalize ---

__global__ void k_finalize(const unsigned long long *__restrict__ keys, int64_t P, float *__restrict__ snr_max,
                           int32_t *__restrict__ argmax) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if (key == 0ull) {
            snr_max[i] = 0.f;
            argmax[i] = -1;
        } else {
            uint32_t b = (uint32_t)(key >> 32);
            b = (b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b;
            snr_max[i] = __uint_as_float(b);
            argmax[i] = (int32_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
        }
    }
}

// --------------------------------------------------------------- host ---

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encode(char *err, size_t errlen) {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled is not available from the driver");
        return (int)cudaErrorNotSupported;
    }
    return 0;
}

int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    if (b < 1) b = 1;
    return (int)b;
}

size_t numerator_smem(const Plan &pl) {
    size_t s = 1024;  // alignment slack
    s += (size_t)kStages * pl.BH * pl.S * sizeof(float);
    s += (size_t)kStages * sizeof(FrameBlock);
    s += (size_t)kTile * kTile * sizeof(unsigned long long);
    s += (size_t)kStages * sizeof(uint64_t) + 3 * kStages * sizeof(int) + sizeof(int) + 64;
    return s;
}

#define MF_CHECK_LAUNCH(what)                                                             \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e_));                \
            return (int)e_;                                                               \
        }                                                                                 \
    } while (0)

}  // namespace

int launch_search(const SearchArgs &a, char *err, size_t errlen) {
    const mf_stack &st = *a.stack;
    const mf_prf_table &tab = *a.tab;
    const Plan &pl = tab.plan;
    const WorkspaceLayout &L = a.L;
    cudaStream_t stream = (cudaStream_t)a.stream;
    const int64_t T = st.T, H = st.H, W = st.W, P = H * W;
    float *lam = reinterpret_cast<float *>(a.ws + L.lam_off);
    float *y = reinterpret_cast<float *>(a.ws + L.y_off);
    float *isd = reinterpret_cast<float *>(a.ws + L.isd_off);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.ws + L.keys_off);

    int rc = get_encode(err, errlen);
    if (rc) return rc;

    k_lambda<<<grid_for(L.lam_w * L.lam_h, 256), 256, 0, stream>>>(a.sigma, a.mask, H, W, L.pad, L.lam_w, L.lam_h,
                                                                    lam);
    MF_CHECK_LAUNCH("k_lambda");

    const int64_t nw = T * H * ((W + 3) / 4);
    const int64_t fs = st.frame_stride, rs = st.row_stride;
    switch (st.dtype) {
        case MF_F32:
            k_weight<float><<<grid_for(nw, 256), 256, 0, stream>>>((const float *)st.data, fs, rs, st.frame_scale,
                                                                   lam, L.pad, L.lam_w, y, T, H, W, L.y_pitch);
            break;
        case MF_BF16:
            k_weight<__nv_bfloat16><<<grid_for(nw, 256), 256, 0, stream>>>(
                (const __nv_bfloat16 *)st.data, fs, rs, st.frame_scale, lam, L.pad, L.lam_w, y, T, H, W, L.y_pitch);
            break;
        default:
            k_weight<__half><<<grid_for(nw, 256), 256, 0, stream>>>((const __half *)st.data, fs, rs, st.frame_scale,
                                                                    lam, L.pad, L.lam_w, y, T, H, W, L.y_pitch);
            break;
    }
    MF_CHECK_LAUNCH("k_weight");

    {
        const int tiles_x = (int)((W + kTile - 1) / kTile);
        const int tiles = tiles_x * (int)((H + kTile - 1) / kTile);
        dim3 grid((tiles + 3) / 4, tab.K);
        k_denominator<<<grid, 128, 0, stream>>>(lam, L.lam_w, L.pad, tab.d_segs, tab.d_seg_off, H, W, tiles_x,
                                                tiles, isd);
        MF_CHECK_LAUNCH("k_denominator");
    }

    cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)P * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return (int)e;
    }

    CUtensorMap map;
    {
        cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
        cuuint64_t strides[2] = {(cuuint64_t)L.y_pitch * 4, (cuuint64_t)(H * L.y_pitch * 4)};
        cuuint32_t box[3] = {(cuuint32_t)pl.S, (cuuint32_t)kLoadRows, 1};
        cuuint32_t estr[3] = {1, 1, 1};
        CUresult cr = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, y, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
            return (int)cudaErrorInvalidValue;
        }
    }
    {
        NumParams np;
        np.blocks = tab.d_blocks;
        np.hdr = tab.d_hdr;
        np.isd = isd;
        np.keys = keys;
        np.snr_all = a.snr_all;
        np.T = (int)T;
        np.G = pl.G;
        np.H = H;
        np.W = W;
        np.tiles_x = (int)((W - kTileOriginX + kTile - 1) / kTile);
        const int tiles_y = (int)((H + kTile - 1) / kTile);
        np.S = pl.S;
        np.BH = pl.BH;
        const size_t smem = numerator_smem(pl);
        auto kern = k_numerator<kWarpsPerCta, kStages>;
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "cudaFuncSetAttribute(smem=%zu): %s", smem, cudaGetErrorString(e));
            return (int)e;
        }
        const long long nblocks = (long long)pl.G * np.tiles_x * tiles_y;
        kern<<<(unsigned)nblocks, kWarpsPerCta * 32, smem, stream>>>(map, np);
        MF_CHECK_LAUNCH("k_numerator");
    }
    k_finalize<<<grid_for(P, 256), 256, 0, stream>>>(keys, P, a.snr_max, a.argmax);
    MF_CHECK_LAUNCH("k_finalize");
    return 0;
}

size_t rescore_workspace(int64_t H, int64_t W, int32_t k_top) {
    (void)H;
    (void)W;
    return (size_t)k_top * 64 + 256;
}

int launch_rescore(const RescoreArgs &a, char *err, size_t errlen) {
    (void)a;
    snprintf(err, errlen, "mf_rescore_topk is not built yet");
    return (int)cudaErrorNotSupported;
}

int read_device_status(int *status) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return (int)e;
    int v = 0, zero = 0;
    e = cudaMemcpyFromSymbol(&v, g_status, sizeof(int));
    if (e != cudaSuccess) return (int)e;
    e = cudaMemcpyToSymbol(g_status, &zero, sizeof(int));
    if (e != cudaSuccess) return (int)e;
    *status = v;
    return 0;
}

}  // namespace mf
