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
#include <type_traits>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "mf_device.cuh"
#include "mf_internal.h"

namespace mf {

// Device status word: 0, or the code of a bounded wait that gave up.
__device__ int g_status;

namespace {

using namespace dev;

// A bounded wait that records a failure in the device-wide word (the search
// kernels record theirs in their own search's status slot instead).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int code) {
    return dev::mbar_wait(bar, parity, code, &g_status);
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

// Also the largest lambda, into *lmax_bits (cleared before; lambda >= 0, so
// the float bits order as unsigned integers).
__global__ void k_lambda(const float *__restrict__ sigma, const uint8_t *__restrict__ mask, int64_t H,
                         int64_t W, int64_t pad, int64_t lw, int64_t lh, float *__restrict__ lam,
                         unsigned int *lmax_bits) {
    const int64_t n = lw * lh;
    float vmax = 0.f;
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
        vmax = fmaxf(vmax, v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(lmax_bits, __float_as_uint(vmax));
}

// ------------------------------------------------------------- weight ---

// y_t = lambda * (scale_t * r_t) in FP32; stored as FP32 (TOut = float) or
// in the stack's own 16-bit type (TOut = TIn): bf16 as is (beta_t = 1), fp16
// times 1 / beta_t, beta_t the power of two at or above lambda_max * scale_t,
// (of |scale_t|), so that no value overflows (|stored r| <= 65504) and the
// scaling is exact.
// The thread of (frame t, row 0, first column quad) writes beta[t].
__device__ __forceinline__ float fp16_frame_beta(float lmax, float sc, float *inv) {
    const float x = lmax * sc;
    if (!(x > 0.f)) {
        *inv = 1.f;
        return 1.f;
    }
    // x = 1.m * 2^(e - 127) <= 2^(e - 126): beta = 2^(e - 126), from the bits
    const int e = min((int)((__float_as_uint(x) >> 23) & 0xFFu), 253);
    *inv = __uint_as_float((uint32_t)(253 - e) << 23);  // 2^(126 - e)
    return __uint_as_float((uint32_t)(e + 1) << 23);    // 2^(e - 126)
}

template <typename T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }

// Four consecutive stack values as FP32, from one 128-bit (FP32) or 64-bit
// (16-bit types) read: p is aligned to four elements.
template <typename T>
__device__ __forceinline__ void load4_f32(const T *p, float v[4]) {
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
        const uint2 q = *reinterpret_cast<const uint2 *>(p);
        const T *e = reinterpret_cast<const T *>(&q);
#pragma unroll
        for (int j = 0; j < 4; j++) v[j] = to_f32(e[j]);
    }
}

// y_t = lambda * (scale_t * r_t) (16-bit outputs of an fp16 stack also times
// 2^-e_t, exact).  A warp takes one (frame, row) at a time, so the row's
// index split is made once per row; lanes walk the row four values each,
// reading lambda and writing y with aligned vector accesses and the stack
// with them too when its rows allow (VR: aligned base, strides multiples of
// four elements).
template <typename TIn, typename TOut, bool VR>
__global__ void k_weight(const TIn *__restrict__ r, int64_t fstride, int64_t rstride,
                         const float *__restrict__ scale, const float *__restrict__ lam, int64_t pad, int64_t lw,
                         TOut *__restrict__ y, int64_t T, int64_t H, int64_t W, int64_t yp,
                         const unsigned int *lmax_bits, float *__restrict__ beta) {
    constexpr bool kHalfScaled = std::is_same<TOut, __half>::value;
    const float lmax = kHalfScaled ? __uint_as_float(*lmax_bits) : 0.f;
    const int64_t wq = (W + 3) / 4, rows = T * H;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t ri = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ri < rows; ri += nwarps) {
        const int64_t t = ri / H, yy = ri - t * H;
        const float sc = scale ? scale[t] : 1.f;
        float inv = 1.f, bt = 1.f;
        if (kHalfScaled) bt = fp16_frame_beta(lmax, fabsf(sc), &inv);
        if (beta && yy == 0 && lane == 0) beta[t] = bt;
        const float *lrow = lam + (yy + pad) * lw + pad;  // padded: columns W .. W + 3 exist
        const TIn *rrow = r + t * fstride + yy * rstride;
        TOut *yrow = y + ri * yp;
        for (int64_t xq = lane; xq < wq; xq += 32) {
            const int64_t x0 = xq * 4;
            const float4 l4 = *reinterpret_cast<const float4 *>(lrow + x0);
            const float l[4] = {l4.x, l4.y, l4.z, l4.w};
            float v[4];
            if (VR && x0 + 4 <= W) {
                load4_f32(rrow + x0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) v[j] = x0 + j < W ? to_f32(rrow[x0 + j]) : 0.f;
            }
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                o[j] = (x0 + j < W) ? l[j] * (sc * v[j]) : 0.f;
                if (kHalfScaled) o[j] *= inv;  // a power of two: exact
            }
            TOut *dst = yrow + x0;
            if (std::is_same<TOut, float>::value) {
                *reinterpret_cast<float4 *>(dst) = make_float4(o[0], o[1], o[2], o[3]);
            } else {
                TOut q[4] = {from_f32<TOut>(o[0]), from_f32<TOut>(o[1]), from_f32<TOut>(o[2]), from_f32<TOut>(o[3])};
                *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(q);
            }
        }
    }
}

// -------------------------------------------------------- denominator ---

// D_k(p) = sum_u G_k(u) lambda(p + u) over the rows (runs) of the collapsed
// kernel G_k.  A thread owns 8 consecutive start pixels of one row, a warp 256
// of them, a CTA 8 rows; blockIdx.y walks the trajectories.  For each run the
// thread slides an 8-wide register window along the lambda row (one aligned
// float4 per 4 taps), so every loaded value feeds 8 FMAs.  Products and
// partial sums are FP32 over at most kDenTaps taps; the partials are added in
// FP64.  The result is stored as 1 / sqrt(D) (0 where D = 0).
__global__ void __launch_bounds__(256) k_denominator(const float *__restrict__ lam, int64_t lw, int64_t pad,
                                                     const RunRec *__restrict__ runs,
                                                     const int32_t *__restrict__ run_off,
                                                     const float *__restrict__ wts, int K, int64_t H, int64_t W,
                                                     int nbx, float *__restrict__ isd) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t py = (int64_t)(blockIdx.x / nbx) * 8 + warp;
    const int64_t px0 = (int64_t)(blockIdx.x % nbx) * kDenCols + 8 * lane;
    const int64_t P = H * W;
    for (int k = blockIdx.y; k < K; k += gridDim.y) {
        double d[8];
        float a[8];
#pragma unroll
        for (int c = 0; c < 8; c++) {
            d[c] = 0.0;
            a[c] = 0.f;
        }
        int taps = 0;
        const int r0 = run_off[k], r1 = run_off[k + 1];
        for (int r = r0; r < r1; r++) {
            const RunRec rr = runs[r];
            const float4 *row = reinterpret_cast<const float4 *>(lam + (py + rr.dy + pad) * lw + px0 + rr.x0 + pad);
            const float4 *wp = reinterpret_cast<const float4 *>(wts + rr.woff);
            // 12-value window of lambda in three float4 slots that rotate:
            // chunk ch (4 taps) uses slot ch mod 3 onwards and, before its
            // FMAs, loads the slot two ahead; unrolled by 3 so that every
            // register index is static
            float v[12];
            {
                const float4 p0 = __ldg(row), p1 = __ldg(row + 1);
                v[0] = p0.x; v[1] = p0.y; v[2] = p0.z; v[3] = p0.w;
                v[4] = p1.x; v[5] = p1.y; v[6] = p1.z; v[7] = p1.w;
            }
            for (int ch = 0; ch < rr.nch; ch += 3) {
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    if (ch + u < rr.nch) {
                        const float4 pn = __ldg(row + ch + u + 2);
                        const int ns = ((u + 2) % 3) * 4;  // slot receiving columns 4 (ch + u + 2) ..
                        v[ns] = pn.x; v[ns + 1] = pn.y; v[ns + 2] = pn.z; v[ns + 3] = pn.w;
                        const float4 w4 = __ldg(wp + ch + u);
                        const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int c = 0; c < 8; c++) a[c] = fmaf(w[i], v[(4 * u + i + c) % 12], a[c]);
                    }
                }
            }
            taps += rr.nch * 4;
            if (taps >= kDenTaps) {
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    d[c] += (double)a[c];
                    a[c] = 0.f;
                }
                taps = 0;
            }
        }
        if (py < H) {
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const double dd = d[c] + (double)a[c];
                const int64_t px = px0 + c;
                if (px < W) isd[(int64_t)k * P + py * W + px] = dd > 0.0 ? rsqrtf((float)dd) : 0.f;
            }
        }
    }
}

// The same sums from a staged box.  A CTA owns `th` rows x kDenBoxCols start
// pixels of one trajectory k: it copies the lambda box its start pixels
// reach through G_k (rows dy0 .., columns x0 .. of the box, plus the tile),
// G_k's weights and its runs into shared memory.  A thread then owns NO
// consecutive start pixels of one tile row and slides an NO-wide register
// window along each run, so that every 128-bit read of lambda feeds 4 NO
// FMAs.  A warp covers 8 rows x 4 NO columns: the 8 threads of a quarter
// warp hold the same columns of 8 consecutive rows, which an odd row pitch
// (in 16-byte chunks) puts in 8 distinct bank groups, so the reads are
// conflict-free at plain row-major addresses (base + chunk, no per-read
// index arithmetic).  Same FP32 products, same FP64 accumulation as
// k_denominator.
template <int NO>
__global__ void __launch_bounds__(32 * kDenBoxCols / NO) k_den_box(
    const float *__restrict__ lam, int64_t lw, int64_t lh, int64_t pad, const RunRec *__restrict__ runs,
    const int32_t *__restrict__ run_off, const float *__restrict__ wts, const DenBox *__restrict__ boxes, int K,
    int64_t H, int64_t W, int nbx, int th, float *__restrict__ isd) {
    static_assert(NO % 4 == 0 && kDenBoxCols % (4 * NO) == 0, "whole chunks, whole warps per 8 rows");
    constexpr int WR = kDenBoxCols / (4 * NO);  // warps per 8 tile rows
    constexpr int S = NO / 4 + 1;                // window slots of 4 values
    extern __shared__ __align__(16) float4 dsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // tile row y and first column xs of this thread's NO start pixels
    const int y = 8 * (warp / WR) + (lane & 7), xs = 4 * NO * (warp % WR) + NO * (lane >> 3);
    const int64_t py = (int64_t)(blockIdx.x / nbx) * th + y;
    const int64_t px0 = (int64_t)(blockIdx.x % nbx) * kDenBoxCols;
    const int64_t P = H * W;
    const bool vec = (W & 3) == 0;  // rows (and planes) start on 16-byte boundaries
    for (int k = blockIdx.y; k < K; k += gridDim.y) {
        const DenBox bx = boxes[k];
        const int R = th + bx.rows - 1, NC = (kDenBoxCols + bx.cols) / 4, PC = den_pitch(bx.cols);
        const int r0 = run_off[k], nr = run_off[k + 1] - r0;
        float4 *wsm = dsm + (size_t)R * PC;                           // weights after the box
        RunRec *rsm = reinterpret_cast<RunRec *>(wsm + bx.nw / 4);    // then the runs
        __syncthreads();                                               // the previous trajectory's reads are done
        // lambda rows py0 + dy0 .. of the padded image (zero beyond its last row)
        const int64_t gy0 = py - y + bx.dy0 + pad, gx0 = px0 + bx.x0 + pad;
        for (int i = threadIdx.x; i < R * NC; i += blockDim.x) {
            const int r = i / NC, j = i % NC;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (gy0 + r < lh) v = __ldg(reinterpret_cast<const float4 *>(lam + (gy0 + r) * lw + gx0) + j);
            dsm[(size_t)r * PC + j] = v;
        }
        for (int i = threadIdx.x; i < bx.nw / 4; i += blockDim.x)
            wsm[i] = __ldg(reinterpret_cast<const float4 *>(wts + bx.w0) + i);
        for (int i = threadIdx.x; i < nr; i += blockDim.x) rsm[i] = runs[r0 + i];
        __syncthreads();
        if (py >= H) continue;
        double d[NO];
        float a[NO];
#pragma unroll
        for (int c = 0; c < NO; c++) {
            d[c] = 0.0;
            a[c] = 0.f;
        }
        int taps = 0;
        for (int r = 0; r < nr; r++) {
            const RunRec rr = rsm[r];
            // the thread's first chunk of the run
            const float4 *row = dsm + (size_t)(y + rr.dy - bx.dy0) * PC + (rr.x0 - bx.x0 + xs) / 4;
            const float4 *wp = wsm + (rr.woff - bx.w0) / 4;
            // window of NO + 4 lambda values in S float4 slots that rotate:
            // chunk ch (4 taps) uses slot ch mod S onwards and, before its
            // FMAs, loads the slot S - 1 ahead; unrolled by S so that every
            // register index is static
            float v[4 * S];
#pragma unroll
            for (int q = 0; q < S - 1; q++) {
                const float4 pq = row[q];
                v[4 * q] = pq.x; v[4 * q + 1] = pq.y; v[4 * q + 2] = pq.z; v[4 * q + 3] = pq.w;
            }
            for (int ch = 0; ch < rr.nch; ch += S) {
#pragma unroll
                for (int u = 0; u < S; u++) {
                    if (ch + u < rr.nch) {
                        const float4 pn = row[ch + u + S - 1];
                        const int ns = ((u + S - 1) % S) * 4;  // slot receiving columns 4 (ch + u + S - 1) ..
                        v[ns] = pn.x; v[ns + 1] = pn.y; v[ns + 2] = pn.z; v[ns + 3] = pn.w;
                        const float4 w4 = wp[ch + u];
                        const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int c = 0; c < NO; c++) a[c] = fmaf(w[i], v[(4 * u + i + c) % (4 * S)], a[c]);
                    }
                }
            }
            taps += rr.nch * 4;
            if (taps >= kDenTaps) {
#pragma unroll
                for (int c = 0; c < NO; c++) {
                    d[c] += (double)a[c];
                    a[c] = 0.f;
                }
                taps = 0;
            }
        }
        float o[NO];
#pragma unroll
        for (int c = 0; c < NO; c++) {
            const double dd = d[c] + (double)a[c];
            o[c] = dd > 0.0 ? rsqrtf((float)dd) : 0.f;
        }
        const int64_t px = px0 + xs;
        float *dst = isd + (int64_t)k * P + py * W + px;
        if (vec && px + NO <= W) {
#pragma unroll
            for (int q = 0; q < NO / 4; q++)
                reinterpret_cast<float4 *>(dst)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        } else {
#pragma unroll
            for (int c = 0; c < NO; c++)
                if (px + c < W) dst[c] = o[c];
        }
    }
}

// ---------------------------------------------------------- numerator ---

struct NumParams {
    const unsigned char *blocks;  // [G][T] frame blocks
    const FrameHdr *hdr;          // [G][T]
    const float *isd;             // [K][H][W]
    unsigned long long *keys;     // [H][W]
    float *snr_all;               // [K][H][W] or null
    int *status;                  // the search's status slot
    int T, G;
    int64_t H, W;
    int tiles_x;
    int S, BH;
    int lockstep;  // 1: CTA barrier after every frame; 0: the last warp out refills the stage
};

// Column skew of lane row-group ty for window loads of VEC floats: it keeps
// the lanes of every shared-memory wavefront on distinct banks (pitch a
// multiple of 32 words) and is a multiple of VEC, so a lane's row segment
// starts VEC-aligned whenever the warp's window offset is.
template <int VEC>
__device__ __forceinline__ int lane_skew(int ty) {
    return VEC == 1 ? ty : (VEC == 2 ? 2 * (ty & 3) : 4 * (ty & 1));
}

// The 4 x 8 block of one lane for one (trajectory, frame): 8 window rows of
// 12 values each, 25 FMAs per output.  `base` is the lane's first window value
// minus M (so VEC-aligned); M = window offset mod VEC is a compile-time
// constant of the variant, so the row segment is read with aligned VEC-wide
// loads and the register selection costs nothing.
template <int VEC, int M>
__device__ __forceinline__ void stencil_4x8(const float *__restrict__ base, int S, const float (&w)[28],
                                            float (&blk)[kMicroRows][kMicroCols]) {
    constexpr int NV = (kMicroCols + 4 + M + VEC - 1) / VEC;  // vector loads per row
#pragma unroll
    for (int i = 0; i < kMicroRows + 4; i++) {
        float f[NV * VEC];
        const float *rp = base + i * S;
#pragma unroll
        for (int q = 0; q < NV; q++) {
            if (VEC == 4) {
                const float4 x = reinterpret_cast<const float4 *>(rp)[q];
                f[4 * q] = x.x;
                f[4 * q + 1] = x.y;
                f[4 * q + 2] = x.z;
                f[4 * q + 3] = x.w;
            } else if (VEC == 2) {
                const float2 x = reinterpret_cast<const float2 *>(rp)[q];
                f[2 * q] = x.x;
                f[2 * q + 1] = x.y;
            } else {
                f[q] = rp[q];
            }
        }
#pragma unroll
        for (int r = 0; r < kMicroRows; r++) {
            const int a = i - r;
            if (a < 0 || a > 4) continue;
#pragma unroll
            for (int c = 0; c < kMicroCols; c++)
#pragma unroll
                for (int b = 0; b < 5; b++) blk[r][c] = fmaf(w[a * 5 + b], f[M + c + b], blk[r][c]);
        }
    }
}

template <int VEC>
__device__ __forceinline__ void stencil_dispatch(const float *__restrict__ base, int m, int S, const float (&w)[28],
                                                 float (&blk)[kMicroRows][kMicroCols]) {
    if (VEC == 1) {
        stencil_4x8<1, 0>(base, S, w, blk);
    } else if (VEC == 2) {
        if (m == 0) stencil_4x8<2, 0>(base, S, w, blk);
        else stencil_4x8<2, 1>(base - 1, S, w, blk);
    } else {
        switch (m) {
            case 0: stencil_4x8<4, 0>(base, S, w, blk); break;
            case 1: stencil_4x8<4, 1>(base - 1, S, w, blk); break;
            case 2: stencil_4x8<4, 2>(base - 2, S, w, blk); break;
            default: stencil_4x8<4, 3>(base - 3, S, w, blk); break;
        }
    }
}

// One CTA: an output tile of (32 TYS) x (32 TXS) start pixels for KT
// trajectories, kWarps warps, one (trajectory, sub-tile) pair per warp.
// The work of one CTA on one (output tile, trajectory group): returns false
// if it gave up (a bounded wait ran out; the device status word says why).
// `smem` is the CTA's 1024-aligned dynamic shared memory, derived from the
// extern array so that its loads stay shared-memory loads.
template <int KT, int TXS, int TYS, int VEC>
__device__ __forceinline__ bool numerator_tile(const CUtensorMap *ymap, const NumParams &p, int g, int tile,
                                               unsigned char *smem) {
    static_assert(KT * TXS * TYS == kWarps, "one warp per (trajectory, sub-tile)");
    constexpr int NS = kStages;
    constexpr int TH = kTile * TYS, TW = kTile * TXS;
    constexpr uint32_t kBlockBytes = (uint32_t)(sizeof(FrameHdr) + KT * sizeof(SlotRec));
    constexpr int R = kRecordChunk;  // frames per record chunk
    static_assert(R >= NS, "a record chunk must outlive the frames in flight");
    const int win_floats = p.BH * p.S;
    float *win = reinterpret_cast<float *>(smem);
    unsigned char *fb = smem + (size_t)NS * win_floats * sizeof(float);  // NS frame blocks
    uint64_t *bars = reinterpret_cast<uint64_t *>(fb + 2 * R * kBlockBytes);  // fb: 2 chunks of R blocks
    int *cnt = reinterpret_cast<int *>(bars + NS);
    int *last_issued = cnt + NS;
    int *bad_flag = last_issued + NS;
    unsigned long long *red = reinterpret_cast<unsigned long long *>(smem);  // epilogue reuses the windows

    const int tile_y0 = (tile / p.tiles_x) * TH;
    const int tile_x0 = (tile % p.tiles_x) * TW + kTileOriginX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = warp % KT, sub = warp / KT;
    const int stx = sub % TXS, sty = sub / TXS;
    const int tx = lane & 3, ty = lane >> 2;
    const int skew = lane_skew<VEC>(ty);
    const unsigned char *gblocks = p.blocks + (size_t)g * p.T * kBlockBytes;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; s++) {
            mbar_init(smem_u32(&bars[s]), 1);
            cnt[s] = 0;
            last_issued[s] = -1;
        }
        *bad_flag = dev::status_now(p.status);  // an earlier CTA of this search gave up: do not start
        fence_barrier_init();
    }
    __syncthreads();
    if (*bad_flag != 0) return false;  // same value for every thread of the CTA

    // Load frame f into stage s: the rows the group's window needs at frame f
    // (TMA, zero fill outside the frame) and the frame's slot records.
    auto issue = [&](int f, int s, FrameHdr h) {
        // one box of the whole window (BH x S): every TMA operation costs the
        // CTA's shared-memory pipeline more than the rows it would save
        const uint32_t bar = smem_u32(&bars[s]);
        // the first frame of a chunk also brings the records of the chunk's
        // frames (its buffer last held chunk f / R - 2, long released)
        const int nrec = (f % R == 0) ? min(R, p.T - f) : 0;
        mbar_expect_tx(bar, (uint32_t)win_floats * 4 + (uint32_t)nrec * kBlockBytes);
        tma_load_3d(smem_u32(win + (size_t)s * win_floats), ymap, tile_x0 + h.rox, tile_y0 + h.roy, f, bar);
        if (nrec)
            bulk_load(smem_u32(fb + ((f / R) & 1) * R * kBlockBytes), gblocks + (size_t)f * kBlockBytes,
                      (uint32_t)nrec * kBlockBytes, bar);
        last_issued[s] = f;
    };
    if (threadIdx.x == 0) {
        fence_proxy_async();  // earlier generic writes to these buffers precede the copies
        for (int s = 0; s < NS && s < p.T; s++) issue(s, s, p.hdr[(size_t)g * p.T + s]);
    }

    // A warp whose sub-tile lies entirely outside the image only keeps pace.
    const int sub_y0 = tile_y0 + kTile * sty, sub_x0 = tile_x0 + kTile * stx;
    const bool inside = sub_y0 < p.H && sub_x0 + kTile + 7 > 0 && sub_x0 < p.W;

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
    bool next_ready = false;  // frame t's data already seen complete during frame t - 1
    // lane's offset in a window; stage and barrier phase advance incrementally
    const int lane_off = (kTile * sty + kMicroRows * ty) * p.S + kTile * stx + kMicroCols * tx + skew;
    int s = 0;
    uint32_t par = 0;
    for (int t = 0; t < p.T; t++) {
        const int s1 = (s + 1 == NS) ? 0 : s + 1;            // stage and phase of frame t + 1
        const uint32_t par1 = (s + 1 == NS) ? (par ^ 1u) : par;
        const bool ready = next_ready || dev::mbar_wait(smem_u32(&bars[s]), par, 1, p.status);
        if (!ready && !p.lockstep) {
            bad = true;
            break;
        }
        const unsigned char *fblk = fb + (((t / R) & 1) * R + t % R) * kBlockBytes;  // frame t's block
        const SlotRec *rec = reinterpret_cast<const SlotRec *>(fblk + sizeof(FrameHdr)) + slot;
        kk = rec->k;
        // Look at the next frame's barrier now: the check's latency then hides
        // behind this frame's arithmetic instead of stalling the next frame.
        next_ready = !p.lockstep && t + 1 < p.T && mbar_test_wait(smem_u32(&bars[s1]), par1);
        if (ready && kk >= 0 && inside) {
            float w[28];
            const float4 *w4 = reinterpret_cast<const float4 *>(rec->taps);
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
            const float *base = win + (size_t)s * win_floats + offy * p.S + offx + lane_off;
            stencil_dispatch<VEC>(base, offx & (VEC - 1), p.S, w, blk);
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
        if (p.lockstep) {
            // every warp is done with stage s: refill it with frame t + NS
            if (__syncthreads_or(!ready)) {
                bad = true;
                break;
            }
            if (threadIdx.x == 0 && t + NS < p.T) {
                const FrameHdr h = *reinterpret_cast<const FrameHdr *>(fblk);
                fence_proxy_async();
                issue(t + NS, s, h);
            }
            s = s1;
            par = par1;
            continue;
        }
        // Release stage s; the last warp to release it loads frame t + NS.
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();
            const int prev = atomicAdd(&cnt[s], 1);
            if (prev == kWarps - 1) {
                cnt[s] = 0;
                if (t + NS < p.T) {
                    const FrameHdr h = *reinterpret_cast<const FrameHdr *>(fblk);
                    fence_proxy_async();
                    issue(t + NS, s, h);
                }
            }
        }
        s = s1;
        par = par1;
    }
    if (bad) atomicExch(bad_flag, 1);
    __syncthreads();
    if (*bad_flag) {
        // Let any copy still in flight land before the CTA's shared memory goes away.
        if (threadIdx.x == 0) {
            for (int s = 0; s < NS; s++) {
                const int f = last_issued[s];
                if (f >= 0) dev::mbar_wait(smem_u32(&bars[s]), (uint32_t)((f / NS) & 1), 2, p.status);
            }
        }
        return false;
    }

    // Epilogue: every issued frame has been consumed, so the windows are free
    // for the tile of packed (SNR, k) keys.
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) red[i] = 0ull;
    __syncthreads();
    const int64_t P = p.H * p.W;
#pragma unroll
    for (int r = 0; r < kMicroRows; r++)
#pragma unroll
        for (int c = 0; c < kMicroCols; c++) {
            const float n = acc[r][c] + blk[r][c];
            const int64_t py = sub_y0 + kMicroRows * ty + r;
            const int64_t px = sub_x0 + kMicroCols * tx + skew + c;
            if (kk >= 0 && py < p.H && px >= 0 && px < p.W) {
                const int64_t q = py * p.W + px;
                const float isd = p.isd[(int64_t)kk * P + q];
                const float snr = n * isd;
                if (p.snr_all) p.snr_all[(int64_t)kk * P + q] = isd > 0.f ? snr : 0.f;
                if (isd > 0.f)
                    atomicMax(&red[(kTile * sty + kMicroRows * ty + r) * TW + kTile * stx + kMicroCols * tx + c],
                              pack_key(snr, kk));
            }
        }
    __syncthreads();
    for (int i = threadIdx.x; i < TH * TW; i += blockDim.x) {
        const unsigned long long key = red[i];
        if (key == 0ull) continue;
        const int ly = i / TW, lx = i % TW;
        const int64_t py = tile_y0 + ly;
        const int64_t px = tile_x0 + lx + lane_skew<VEC>((ly / kMicroRows) % 8);
        atomicMax(&p.keys[py * p.W + px], key);
    }
    // the barriers may be initialised again for this CTA's next tile
    if (threadIdx.x == 0)
        for (int s = 0; s < NS; s++) mbar_inval(smem_u32(&bars[s]));
    return true;
}

template <int KT, int TXS, int TYS, int VEC>
__global__ void __launch_bounds__(kWarps * 32, 1) k_numerator(const __grid_constant__ CUtensorMap ymap,
                                                              const NumParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    numerator_tile<KT, TXS, TYS, VEC>(&ymap, p, (int)(blockIdx.x % (unsigned)p.G),
                                      (int)(blockIdx.x / (unsigned)p.G), smem);
}

// One item of a batched search: its numerator parameters, tile count and the
// first entry of its CTA work in the batch-wide work list.
struct BatchItem {
    NumParams p;
    int tiles_y;
    int pad;
    long long cta_begin;
};

// Persistent numerator over a batch of searches: one CTA per SM takes
// (item, tile, group) work entries from a global counter until the list is
// exhausted, running the same per-tile code as k_numerator.
template <int KT, int TXS, int TYS, int VEC>
__global__ void __launch_bounds__(kWarps * 32, 1) k_numerator_batch(const CUtensorMap *__restrict__ maps,
                                                                    const BatchItem *__restrict__ items, int n_items,
                                                                    long long total,
                                                                    unsigned long long *counter) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    __shared__ long long work;
    __shared__ int item;
    for (;;) {
        if (threadIdx.x == 0) {
            const long long w = (long long)atomicAdd(counter, 1ull);
            int lo = 0, hi = n_items - 1;  // last item whose cta_begin <= w
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].cta_begin <= w) lo = mid;
                else hi = mid - 1;
            }
            work = w;
            item = lo;
        }
        __syncthreads();
        const long long w = work;
        const int i = item;
        __syncthreads();
        if (w >= total) break;
        const NumParams &p = items[i].p;
        const long long local = w - items[i].cta_begin;
        if (!numerator_tile<KT, TXS, TYS, VEC>(maps + i, p, (int)(local % p.G), (int)(local / p.G), smem)) break;
        __syncthreads();
    }
}

// ----------------------------------------------------------- finalize ---

__global__ void k_finalize(const unsigned long long *__restrict__ keys, int64_t P, float *__restrict__ snr_max,
                           int32_t *__restrict__ argmax, const int *slot, int *global_status) {
    // a failure of this search also goes into the device-wide word
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int s = *(const volatile int *)slot;
        if (s != 0) atomicCAS(global_status, 0, s);
    }
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


#define MF_CHECK_LAUNCH(what)                                                             \
    do {                                                                                  \
        cudaError_t e_ = cudaGetLastError();                                              \
        if (e_ != cudaSuccess) {                                                          \
            snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e_));                \
            return (int)e_;                                                               \
        }                                                                                 \
    } while (0)

// ---------------------------------------------------------- profiling ---

const char *kKernelNames[kKernelCount] = {"k_lambda",    "k_weight",      "k_denominator", "k_numerator",
                                          "k_finalize",  "k_select",      "k_rescore",     "k_compact",
                                          "k_sort",      "k_det_stats",   "k_det_cc",      "k_det_emit",
                                          "k_refit"};

struct ProfPending {
    int kid;
    cudaEvent_t a, b;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfPending> g_pending;
double g_prof_ms[kKernelCount];
long long g_prof_count[kKernelCount];

// Bracket one launch: call with stage 0 before and stage 1 after it.
struct LaunchScope {
    int kid;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchScope(int k, cudaStream_t s) : kid(k), st(s) {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        g_prof_count[kid]++;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
        if (g_prof_on && cs == cudaStreamCaptureStatusNone && cudaEventCreate(&a) == cudaSuccess &&
            cudaEventCreate(&b) == cudaSuccess)
            cudaEventRecord(a, st);
    }
    ~LaunchScope() {
        if (a && b) {
            cudaEventRecord(b, st);
            std::lock_guard<std::mutex> lk(g_prof_mu);
            g_pending.push_back({kid, a, b});
        }
    }
};

}  // namespace

ProfToken prof_begin(int kid, void *stream) {
    LaunchScope *ls = new LaunchScope(kid, (cudaStream_t)stream);
    return ProfToken{ls};
}

void prof_end(const ProfToken &t) { delete static_cast<LaunchScope *>(t.scope); }

int profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return 0;
}

int profile_read(mf_profile *out, int reset) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
            g_prof_ms[p.kid] += ms;
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_pending.clear();
    std::memset(out, 0, sizeof *out);
    for (int i = 0; i < kKernelCount && i < 16; i++) {
        std::snprintf(out->k[i].name, sizeof out->k[i].name, "%s", kKernelNames[i]);
        out->k[i].launches = g_prof_count[i];
        out->k[i].ms = g_prof_ms[i];
        out->launches += g_prof_count[i];
    }
    out->n = kKernelCount;
    if (reset) {
        for (int i = 0; i < kKernelCount; i++) {
            g_prof_ms[i] = 0.0;
            g_prof_count[i] = 0;
        }
    }
    return 0;
}

namespace {

// Inverse variance, weighted stack, denominator and a cleared key buffer.
int enqueue_pre(const SearchArgs &a, cudaStream_t stream, char *err, size_t errlen) {
    const mf_stack &st = *a.stack;
    const mf_prf_table &tab = *a.tab;
    const WorkspaceLayout &L = a.L;
    const int64_t T = st.T, H = st.H, W = st.W, P = H * W;
    float *lam = reinterpret_cast<float *>(a.ws + L.lam_off);
    void *y = a.ws + L.y_off;
    float *beta = reinterpret_cast<float *>(a.ws + L.beta_off);
    float *isd = reinterpret_cast<float *>(a.ws + L.isd_off);
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.ws + L.keys_off);
    unsigned int *lmax = reinterpret_cast<unsigned int *>(a.ws + L.status_off + 8);
    // the search's status slot and the lambda maximum start clear (the
    // kernels after this in stream order write the slot only on a failure)
    cudaError_t e0 = cudaMemsetAsync(a.ws + L.status_off, 0, 16, stream);
    if (e0 != cudaSuccess) {
        snprintf(err, errlen, "cudaMemsetAsync: %s", cudaGetErrorString(e0));
        return (int)e0;
    }
    {
        LaunchScope ls(kKLambda, stream);
        k_lambda<<<grid_for(L.lam_w * L.lam_h, 256), 256, 0, stream>>>(a.sigma, a.mask, H, W, L.pad, L.lam_w,
                                                                        L.lam_h, lam, lmax);
    }
    MF_CHECK_LAUNCH("k_lambda");

    const int64_t fs = st.frame_stride, rs = st.row_stride;
    {
        LaunchScope ls(kKWeight, stream);
        const int gw = grid_for(T * H * 32, 256);  // a warp per (frame, row)
        const bool y16 = L.ybytes == 2;
        const size_t esz = st.dtype == MF_F32 ? 4 : 2;
        // vector reads of the stack: aligned base, rows and frames on multiples of four elements
        const bool vr = ((uintptr_t)st.data % (4 * esz)) == 0 && fs % 4 == 0 && rs % 4 == 0;
        auto go = [&](auto tin, auto tout, auto vrc) {
            using TI = decltype(tin);
            using TO = decltype(tout);
            k_weight<TI, TO, decltype(vrc)::value><<<gw, 256, 0, stream>>>(
                (const TI *)st.data, fs, rs, st.frame_scale, lam, L.pad, L.lam_w, (TO *)y, T, H, W, L.y_pitch, lmax,
                beta);
        };
        auto go2 = [&](auto tin, auto tout) {
            if (vr) go(tin, tout, std::true_type{});
            else go(tin, tout, std::false_type{});
        };
        if (st.dtype == MF_F32) go2(float{}, float{});
        else if (st.dtype == MF_BF16 && y16) go2(__nv_bfloat16{}, __nv_bfloat16{});
        else if (st.dtype == MF_BF16) go2(__nv_bfloat16{}, float{});
        else if (y16) go2(__half{}, __half{});
        else go2(__half{}, float{});
    }
    MF_CHECK_LAUNCH("k_weight");
    if (tab.den_th > 0) {
        // staged: one CTA per (tile of den_th x 256 start pixels, trajectory)
        const int th = tab.den_th;
        const int nbx = (int)((W + kDenBoxCols - 1) / kDenBoxCols);
        const int nby = (int)((H + th - 1) / th);
        dim3 grid((unsigned)(nbx * nby), (unsigned)std::min(tab.K, 65535));
        cudaError_t ea = cudaFuncSetAttribute(k_den_box<kDenOut>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)tab.den_smem);
        if (ea != cudaSuccess) {
            snprintf(err, errlen, "cudaFuncSetAttribute(k_den_box): %s", cudaGetErrorString(ea));
            return (int)ea;
        }
        LaunchScope ls(kKDenominator, stream);
        k_den_box<kDenOut><<<grid, th * kDenBoxCols / kDenOut, tab.den_smem, stream>>>(
            lam, L.lam_w, L.lam_h, L.pad, tab.d_runs, tab.d_run_off, tab.d_wts, tab.d_boxes, tab.K, H, W, nbx, th,
            isd);
        MF_CHECK_LAUNCH("k_den_box");
    } else {
        const int nbx = (int)((W + kDenCols - 1) / kDenCols);
        const int nby = (int)((H + 7) / 8);
        dim3 grid((unsigned)(nbx * nby), (unsigned)std::min(tab.K, 65535));
        LaunchScope ls(kKDenominator, stream);
        k_denominator<<<grid, 256, 0, stream>>>(lam, L.lam_w, L.pad, tab.d_runs, tab.d_run_off, tab.d_wts, tab.K, H,
                                                W, nbx, isd);
        MF_CHECK_LAUNCH("k_denominator");
    }
    cudaError_t e = cudaMemsetAsync(keys, 0, (size_t)P * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

// Tensor map over the weighted stack and the numerator's parameters.
int numerator_params(const SearchArgs &a, CUtensorMap *map, NumParams *np, int *tiles_y, char *err,
                     size_t errlen) {
    const mf_stack &st = *a.stack;
    const mf_prf_table &tab = *a.tab;
    const Plan &pl = tab.plan;
    const WorkspaceLayout &L = a.L;
    const int64_t T = st.T, H = st.H, W = st.W;
    int rc = get_encode(err, errlen);
    if (rc) return rc;
    float *y = reinterpret_cast<float *>(a.ws + L.y_off);
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)L.y_pitch * 4, (cuuint64_t)(H * L.y_pitch * 4)};
    cuuint32_t box[3] = {(cuuint32_t)pl.S, (cuuint32_t)pl.BH, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult cr = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, y, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
        return (int)cudaErrorInvalidValue;
    }
    np->blocks = tab.d_blocks;
    np->hdr = tab.d_hdr;
    np->isd = reinterpret_cast<float *>(a.ws + L.isd_off);
    np->keys = reinterpret_cast<unsigned long long *>(a.ws + L.keys_off);
    np->snr_all = a.snr_all;
    np->status = reinterpret_cast<int *>(a.ws + L.status_off);
    np->T = (int)T;
    np->G = pl.G;
    np->H = H;
    np->W = W;
    np->tiles_x = (int)((W - kTileOriginX + pl.tile_w() - 1) / pl.tile_w());
    np->S = pl.S;
    np->BH = pl.BH;
    np->lockstep = pl.lockstep;
    *tiles_y = (int)((H + pl.tile_h() - 1) / pl.tile_h());
    return 0;
}

// Tensor map and parameters of the factored numerator; *nblocks = CTAs.
int fac_params(const SearchArgs &a, CUtensorMap *map, FacParams *fp, long long *nblocks, char *err,
               size_t errlen) {
    const mf_stack &st = *a.stack;
    const mf_prf_table &tab = *a.tab;
    const Plan &pl = tab.plan;
    const WorkspaceLayout &L = a.L;
    const int64_t T = st.T, H = st.H, W = st.W;
    int rc = get_encode(err, errlen);
    if (rc) return rc;
    int *status = reinterpret_cast<int *>(a.ws + L.status_off);
    void *y = a.ws + L.y_off;
    const bool y16 = L.ybytes == 2;
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)L.y_pitch * L.ybytes, (cuuint64_t)(H * L.y_pitch * L.ybytes)};
    cuuint32_t box[3] = {(cuuint32_t)(y16 ? fac_rpitch16(pl.f_tw) : fac_rpitch(pl.f_tw)), (cuuint32_t)pl.f_bh, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType ty = !y16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                        : (st.dtype == MF_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    CUresult cr = g_encode(map, ty, 3, y, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
        return (int)cudaErrorInvalidValue;
    }
    fp->blocks = tab.d_blocks;
    fp->hdr = tab.d_hdr;
    fp->members = tab.d_members;
    fp->segs = tab.d_segs;
    fp->refs = tab.d_refs;
    fp->plane = reinterpret_cast<float *>(a.ws + L.planes_off);
    fp->status = status;
    // fp16 weighted stacks carry a power-of-two scale per frame; bf16 ones none
    fp->beta = (y16 && st.dtype == MF_F16) ? reinterpret_cast<const float *>(a.ws + L.beta_off) : nullptr;
    fp->T = (int)T;
    fp->G = pl.G;
    fp->kt = pl.f_kt;
    fp->npl = pl.f_planes;
    fp->th = pl.f_th;
    fp->bh = pl.f_bh;
    fp->ns = pl.f_ns;
    fp->S = pl.f_seg;
    fp->seg = 0;
    fp->K = tab.K;
    fp->warps = pl.warps();
    fp->H = H;
    fp->W = W;
    fp->tiles_x = (int)((W + pl.f_tw - 1) / pl.f_tw);
    *nblocks = fac_ctas(tab, H, W, 0);
    return 0;
}

typedef void (*NumKernel)(const CUtensorMap, const NumParams);
typedef void (*NumBatchKernel)(const CUtensorMap *, const BatchItem *, int, long long, unsigned long long *);

NumKernel pick_numerator(int shape, int vec) {
#define MF_PICK(V)                                       \
    switch (shape) {                                     \
        case 0: return k_numerator<16, 1, 1, V>;         \
        case 1: return k_numerator<8, 2, 1, V>;          \
        case 2: return k_numerator<4, 2, 2, V>;          \
        default: return k_numerator<2, 4, 2, V>;         \
    }
    if (vec == 4) {
        MF_PICK(4)
    } else if (vec == 2) {
        MF_PICK(2)
    } else {
        MF_PICK(1)
    }
#undef MF_PICK
}

NumBatchKernel pick_numerator_batch(int shape) {
    switch (shape) {
        case 0: return k_numerator_batch<16, 1, 1, 2>;
        case 1: return k_numerator_batch<8, 2, 1, 2>;
        case 2: return k_numerator_batch<4, 2, 2, 2>;
        default: return k_numerator_batch<2, 4, 2, 2>;
    }
}

int enqueue_finalize(const SearchArgs &a, cudaStream_t stream, char *err, size_t errlen) {
    const int64_t P = a.stack->H * a.stack->W;
    const int *slot = reinterpret_cast<const int *>(a.ws + a.L.status_off);
    int *gstatus = status_word(err, errlen);
    if (!gstatus) return (int)cudaErrorInvalidSymbol;
    if (a.tab->plan.kernel == 2) {
        LaunchScope ls(kKFinalize, stream);
        return fac_finalize_enqueue(reinterpret_cast<const float *>(a.ws + a.L.planes_off),
                                    reinterpret_cast<const float *>(a.ws + a.L.isd_off), a.tab->K, P, a.snr_max,
                                    a.argmax, a.snr_all, slot, gstatus, stream, err, errlen);
    }
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(a.ws + a.L.keys_off);
    {
        LaunchScope ls(kKFinalize, stream);
        k_finalize<<<grid_for(P, 256), 256, 0, stream>>>(keys, P, a.snr_max, a.argmax, slot, gstatus);
    }
    MF_CHECK_LAUNCH("k_finalize");
    return 0;
}

}  // namespace

int launch_search(const SearchArgs &a, char *err, size_t errlen) {
    cudaStream_t stream = (cudaStream_t)a.stream;
    const Plan &pl = a.tab->plan;
    int rc = enqueue_pre(a, stream, err, errlen);
    if (rc) return rc;
    CUtensorMap map;
    if (pl.kernel == 2) {
        FacParams fp;
        long long nblocks = 0;
        rc = fac_params(a, &map, &fp, &nblocks, err, errlen);
        if (rc) return rc;
        // one launch per time segment, in order: segment 0 stores the
        // numerator plane, the later ones add to it
        for (int j = 0; j < pl.f_seg; j++) {
            fp.seg = j;
            LaunchScope ls(kKNumerator, stream);
            rc = fac_enqueue(&map, fp, pl.f_tw, pl.f_taps, a.L.ybytes == 2 ? a.stack->dtype : MF_F32,
                             pl.launch_warps(), pl.smem(), fac_ctas(*a.tab, a.stack->H, a.stack->W, j), stream, err,
                             errlen);
            if (rc) return rc;
        }
        return enqueue_finalize(a, stream, err, errlen);
    }
    NumParams np;
    int tiles_y = 0;
    rc = numerator_params(a, &map, &np, &tiles_y, err, errlen);
    if (rc) return rc;
    {
        const size_t smem = numerator_smem_bytes(pl.S, pl.BH, pl.kt());
        NumKernel kern = pick_numerator(pl.shape, pl.vec);
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "cudaFuncSetAttribute(smem=%zu): %s", smem, cudaGetErrorString(e));
            return (int)e;
        }
        const long long nblocks = (long long)pl.G * np.tiles_x * tiles_y;
        LaunchScope ls(kKNumerator, stream);
        kern<<<(unsigned)nblocks, kWarps * 32, smem, stream>>>(map, np);
        MF_CHECK_LAUNCH("k_numerator");
    }
    return enqueue_finalize(a, stream, err, errlen);
}

// ------------------------------------------------------------ batching ---
//
// A batch of searches (uneven cutouts, each with its own filter bank) runs as
// per-item preparation kernels spread over side streams, one persistent
// numerator launch per CTA shape in the batch (usually one), and per-item
// finalisation.  The descriptors the persistent kernel reads (tensor maps,
// parameters, work-list offsets) live in device memory owned by the batch.

struct BatchDevice {
    struct Group {
        int shape = 0;
        int first = 0, count = 0;  // range in the device arrays
        long long total = 0;       // CTA work entries
        size_t smem = 0;
    };
    std::vector<Group> groups;
    std::vector<int> order;  // device-array position -> item
    // searches with a factored numerator: one persistent launch per tile
    // width, with as many warps and as much shared memory as its largest
    // layout needs
    struct FacGroup {
        int tw = 32;
        int etype = MF_F32;        // element type of the weighted stacks
        int seg = 0;               // time segment (groups run in segment order)
        int first = 0, count = 0;  // range in d_fmaps / d_fitems
        long long total = 0;       // CTA work entries
        size_t smem = 0;
        int warps = 0;
    };
    std::vector<FacGroup> fac;
    CUtensorMap *d_fmaps = nullptr;
    FacBatchItem *d_fitems = nullptr;
    std::vector<FacBatchItem> h_fitems;  // the same, passed by value to each launch
    unsigned long long *d_fcounters = nullptr;  // one per group
    CUtensorMap *d_maps = nullptr;
    BatchItem *d_items = nullptr;
    unsigned long long *d_counters = nullptr;
    static constexpr int kSide = 4;
    cudaStream_t side[kSide] = {};
    cudaEvent_t fork = nullptr, join[kSide] = {};
    int sms = 0;
};

void batch_free(BatchDevice *b) {
    if (!b) return;
    cudaFree(b->d_maps);
    cudaFree(b->d_items);
    cudaFree(b->d_counters);
    cudaFree(b->d_fmaps);
    cudaFree(b->d_fitems);
    cudaFree(b->d_fcounters);
    for (int i = 0; i < BatchDevice::kSide; i++) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
}

int batch_build(const SearchArgs *items, int n, BatchDevice **out, char *err, size_t errlen) {
    auto *b = new BatchDevice;
    std::vector<CUtensorMap> maps;
    std::vector<BatchItem> bitems;
    for (int shape = 0; shape < kNumShapes; shape++) {
        BatchDevice::Group grp;
        grp.shape = shape;
        grp.first = (int)bitems.size();
        for (int i = 0; i < n; i++) {
            const Plan &pl = items[i].tab->plan;
            if (pl.kernel != 1 || pl.shape != shape) continue;
            CUtensorMap m;
            BatchItem bi;
            std::memset(&bi, 0, sizeof bi);
            int rc = numerator_params(items[i], &m, &bi.p, &bi.tiles_y, err, errlen);
            if (rc) {
                batch_free(b);
                return rc;
            }
            bi.cta_begin = grp.total;
            grp.total += (long long)pl.G * bi.p.tiles_x * bi.tiles_y;
            grp.smem = std::max(grp.smem, numerator_smem_bytes(pl.S, pl.BH, pl.kt()));
            maps.push_back(m);
            bitems.push_back(bi);
            b->order.push_back(i);
        }
        grp.count = (int)bitems.size() - grp.first;
        if (grp.count > 0) b->groups.push_back(grp);
    }
    std::vector<CUtensorMap> fmaps;
    std::vector<FacBatchItem> fitems;
    int max_seg = 0;
    for (int i = 0; i < n; i++)
        if (items[i].tab->plan.kernel == 2) max_seg = std::max(max_seg, items[i].tab->plan.f_seg);
    // one persistent launch per (segment, tile width, element type of the
    // weighted stack)
    for (int j = 0; j < max_seg; j++) {
        for (int tw : {32, 64})
        for (int et : {(int)MF_F32, (int)MF_BF16, (int)MF_F16}) {
            BatchDevice::FacGroup grp;
            grp.tw = tw;
            grp.etype = et;
            grp.seg = j;
            grp.first = (int)fitems.size();
            for (int i = 0; i < n; i++) {
                const Plan &pl = items[i].tab->plan;
                const int item_et = items[i].L.ybytes == 2 ? items[i].stack->dtype : MF_F32;
                if (pl.kernel != 2 || pl.f_tw != tw || item_et != et || j >= pl.f_seg) continue;
                CUtensorMap m;
                FacBatchItem fi;
                std::memset(&fi, 0, sizeof fi);
                long long nblocks = 0;
                int rc = fac_params(items[i], &m, &fi.p, &nblocks, err, errlen);
                if (rc) {
                    batch_free(b);
                    return rc;
                }
                fi.p.seg = j;
                fi.cta_begin = grp.total;
                grp.total += fac_ctas(*items[i].tab, items[i].stack->H, items[i].stack->W, j);
                grp.smem = std::max(grp.smem, pl.smem());
                grp.warps = std::max(grp.warps, pl.launch_warps());
                fmaps.push_back(m);
                fitems.push_back(fi);
                if ((int)fitems.size() - grp.first == kFacBatchArgItems) {
                    // a launch takes at most kFacBatchArgItems searches: the
                    // rest of this segment goes to the next launch
                    grp.count = kFacBatchArgItems;
                    b->fac.push_back(grp);
                    grp.first = (int)fitems.size();
                    grp.total = 0;
                    grp.smem = 0;
                    grp.warps = 0;
                }
            }
            grp.count = (int)fitems.size() - grp.first;
            if (grp.count > 0) b->fac.push_back(grp);
        }
    }
    cudaError_t e = cudaSuccess;
    if (!fitems.empty()) e = cudaMalloc((void **)&b->d_fmaps, fmaps.size() * sizeof(CUtensorMap));
    if (e == cudaSuccess && !fitems.empty()) e = cudaMalloc((void **)&b->d_fitems, fitems.size() * sizeof(FacBatchItem));
    if (e == cudaSuccess && !fitems.empty())
        e = cudaMalloc((void **)&b->d_fcounters, b->fac.size() * sizeof(unsigned long long));
    if (e == cudaSuccess && !fitems.empty())
        e = cudaMemcpy(b->d_fmaps, fmaps.data(), fmaps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !fitems.empty())
        e = cudaMemcpy(b->d_fitems, fitems.data(), fitems.size() * sizeof(FacBatchItem), cudaMemcpyHostToDevice);
    b->h_fitems = fitems;
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && !maps.empty()) e = cudaMalloc((void **)&b->d_maps, maps.size() * sizeof(CUtensorMap));
    if (e == cudaSuccess && !bitems.empty()) e = cudaMalloc((void **)&b->d_items, bitems.size() * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_counters, kNumShapes * sizeof(unsigned long long));
    if (e == cudaSuccess && !maps.empty())
        e = cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !bitems.empty())
        e = cudaMemcpy(b->d_items, bitems.data(), bitems.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    for (int i = 0; i < BatchDevice::kSide && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (const auto &grp : b->groups) {
        if (e != cudaSuccess) break;
        e = cudaFuncSetAttribute(pick_numerator_batch(grp.shape), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)grp.smem);
    }
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batch set-up: %s", cudaGetErrorString(e));
        batch_free(b);
        return (int)e;
    }
    for (int tw : {32, 64})  // one attribute per kernel: the largest layout of that tile width and type
        for (int et : {(int)MF_F32, (int)MF_BF16, (int)MF_F16}) {
            size_t smem = 0;
            for (const auto &grp : b->fac)
                if (grp.tw == tw && grp.etype == et) smem = std::max(smem, grp.smem);
            if (smem == 0) continue;
            const int rc = fac_batch_attr(tw, et, smem, err, errlen);
            if (rc) {
                batch_free(b);
                return rc;
            }
        }
    *out = b;
    return 0;
}

int batch_enqueue(BatchDevice *b, const SearchArgs *items, int n, void *stream_v, char *err, size_t errlen) {
    cudaStream_t stream = (cudaStream_t)stream_v;
    cudaError_t e = cudaEventRecord(b->fork, stream);
    for (int s = 0; s < BatchDevice::kSide && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->side[s], b->fork, 0);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batch fork: %s", cudaGetErrorString(e));
        return (int)e;
    }
    for (int i = 0; i < n; i++) {
        int rc = enqueue_pre(items[i], b->side[i % BatchDevice::kSide], err, errlen);
        if (rc) return rc;
    }
    for (int s = 0; s < BatchDevice::kSide && e == cudaSuccess; s++) {
        e = cudaEventRecord(b->join[s], b->side[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, b->join[s], 0);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, kNumShapes * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "batch join: %s", cudaGetErrorString(e));
        return (int)e;
    }
    for (const auto &grp : b->groups) {
        const int grid = (int)std::min<long long>(grp.total, (long long)b->sms);
        LaunchScope ls(kKNumerator, stream);
        pick_numerator_batch(grp.shape)<<<grid, kWarps * 32, grp.smem, stream>>>(
            b->d_maps + grp.first, b->d_items + grp.first, grp.count, grp.total, b->d_counters + grp.shape);
        MF_CHECK_LAUNCH("k_numerator_batch");
    }
    if (!b->fac.empty()) {
        e = cudaMemsetAsync(b->d_fcounters, 0, b->fac.size() * sizeof(unsigned long long), stream);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "batch counters: %s", cudaGetErrorString(e));
            return (int)e;
        }
    }
    for (size_t gi = 0; gi < b->fac.size(); gi++) {
        const auto &grp = b->fac[gi];
        const int grid = (int)std::min<long long>(grp.total, (long long)b->sms);
        LaunchScope ls(kKNumerator, stream);
        int rc = fac_batch_enqueue(b->d_fmaps + grp.first, b->h_fitems.data() + grp.first, grp.count, grp.total,
                                   b->d_fcounters + gi, grp.tw, grp.etype, grp.warps, grp.smem, grid, stream, err,
                                   errlen);
        if (rc) return rc;
    }
    for (int i = 0; i < n; i++) {
        int rc = enqueue_finalize(items[i], stream, err, errlen);
        if (rc) return rc;
    }
    return 0;
}

// ------------------------------------------------------------ rescore ---
//
// Candidate list (Section 3.3: scores above a threshold are candidates) and
// FP64 re-score.  Candidates are ranked by a unique 64-bit key, (order-
// preserving SNR bits << 32) | (0xFFFFFFFF - flat index): descending key =
// SNR descending, then flat index ascending.  A 4-pass radix select over 16
// bits at a time finds the k_top-th largest key, a compaction keeps the keys
// at or above it, one CTA sorts them, and one warp per candidate recomputes
// N and D in FP64 from the master stack.

namespace {

__global__ void k_sel_keys(const float *__restrict__ snr_max, const int32_t *__restrict__ argmax, int64_t P,
                           unsigned long long *__restrict__ keys, unsigned int *__restrict__ hist,
                           SelState *st) {
    // the block's bins in a shared-memory table (open addressing, bin ->
    // count), flushed into the global histogram with one add per distinct
    // bin: a score map's keys fall in few bins, which global atomics from
    // every pixel would serialise on; a bin that finds the table full is
    // added globally at once
    constexpr int kSlots = 1024;
    constexpr unsigned int kEmpty = 0xFFFFFFFFu;
    __shared__ unsigned int slot_bin[kSlots], slot_cnt[kSlots];
    for (int j = threadIdx.x; j < kSlots; j += blockDim.x) {
        slot_bin[j] = kEmpty;
        slot_cnt[j] = 0u;
    }
    __syncthreads();
    unsigned int valid = 0;  // keys this thread made; summed per warp into st->total
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = 0ull;
        if (argmax[i] >= 0) {
            uint32_t b = __float_as_uint(snr_max[i]);
            b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
            key = ((unsigned long long)b << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)i);
            valid++;
            const unsigned int bin = (unsigned int)(key >> 48);
            unsigned int h = (bin * 2654435761u) >> 22;  // 10 bits
            bool added = false;
            for (int probe = 0; probe < kSlots; probe++, h = (h + 1) & (kSlots - 1)) {
                const unsigned int old = atomicCAS(&slot_bin[h], kEmpty, bin);
                if (old == kEmpty || old == bin) {
                    atomicAdd(&slot_cnt[h], 1u);
                    added = true;
                    break;
                }
            }
            if (!added) atomicAdd(&hist[bin], 1u);
        }
        keys[i] = key;
    }
    valid = __reduce_add_sync(0xffffffffu, valid);  // blocks are whole warps
    if ((threadIdx.x & 31) == 0 && valid) atomicAdd(&st->total, valid);
    __syncthreads();
    for (int j = threadIdx.x; j < kSlots; j += blockDim.x)
        if (slot_cnt[j]) atomicAdd(&hist[slot_bin[j]], slot_cnt[j]);
}

// Histogram of the next 16 bits among keys that match the selected prefix.
__global__ void k_sel_hist(const unsigned long long *__restrict__ keys, int64_t P, int pass,
                           unsigned int *__restrict__ hist, const SelState *st) {
    const int hi_shift = 64 - 16 * pass;  // bits above this are fixed
    const unsigned long long prefix = st->prefix;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if (key != 0ull && (key >> hi_shift) == (prefix >> hi_shift))
            atomicAdd(&hist[(key >> (hi_shift - 16)) & 0xFFFFull], 1u);
    }
}

// One CTA: find, from the top, the bin holding the `need`-th largest key,
// extend the prefix, and clear the histogram.  Thread t sums the 64 bins
// 65535 - 64 t .. 65472 - 64 t; a block scan of those sums gives each thread
// the count above its bins, and the one thread whose range holds the
// need-th key walks its 64 bins.
__global__ void __launch_bounds__(1024) k_sel_pick(unsigned int *__restrict__ hist, int pass, SelState *st,
                                                   unsigned int k_top) {
    __shared__ unsigned int warp_sum[32];
    __shared__ unsigned int chosen_bin, above;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (pass == 0) {
        if (tid == 0) {
            st->need = st->total < k_top ? st->total : k_top;
            st->prefix = 0ull;
        }
        __syncthreads();
    }
    const unsigned int need = st->need;
    unsigned int sum = 0;
    for (int j = 0; j < 64; j++) sum += hist[65535 - (tid * 64 + j)];
    // inclusive scan over the block, thread order = bins from the top
    unsigned int inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_sum[warp] = inc;
    if (tid == 0) {
        chosen_bin = 0;
        above = 0;
    }
    __syncthreads();
    if (warp == 0) {
        const unsigned int w = warp_sum[lane];
        unsigned int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned int o = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += o;
        }
        warp_sum[lane] = wi - w;  // keys in the bins of earlier warps
    }
    __syncthreads();
    const unsigned int before = warp_sum[warp] + inc - sum;  // keys in bins above this thread's
    if (need > 0 && before < need && before + sum >= need) {
        unsigned int acc = before;
        for (int j = 0; j < 64; j++) {
            const unsigned int b = 65535 - (tid * 64 + j);
            if (acc + hist[b] >= need) {
                chosen_bin = b;
                above = acc;
                break;
            }
            acc += hist[b];
        }
    }
    __syncthreads();
    for (int j = tid; j < 65536; j += blockDim.x) hist[j] = 0u;
    if (tid == 0) {
        const int shift = 48 - 16 * pass;
        st->prefix |= (unsigned long long)chosen_bin << shift;
        st->need = need - above;
        if (pass == 3) st->thresh = need == 0 ? ~0ull : st->prefix;
    }
}

__global__ void k_sel_compact(const unsigned long long *__restrict__ keys, int64_t P,
                              unsigned long long *__restrict__ out, SelState *st, unsigned int cap) {
    const unsigned long long th = st->thresh;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = keys[i];
        if (key != 0ull && key >= th) {
            const unsigned int slot = atomicAdd(&st->count, 1u);
            if (slot < cap) out[slot] = key;
        }
    }
}

// One CTA bitonic sort (descending) of up to kMaxTop keys in shared memory.
__global__ void __launch_bounds__(1024) k_sel_sort(unsigned long long *__restrict__ keys, const SelState *st,
                                                   unsigned int cap) {
    extern __shared__ unsigned long long sk[];
    unsigned int n = st->count < cap ? st->count : cap;
    unsigned int m = 1;
    while (m < n) m <<= 1;
    for (unsigned int i = threadIdx.x; i < m; i += blockDim.x) sk[i] = i < n ? keys[i] : 0ull;
    __syncthreads();
    for (unsigned int size = 2; size <= m; size <<= 1) {
        for (unsigned int stride = size >> 1; stride > 0; stride >>= 1) {
            for (unsigned int i = threadIdx.x; i < m; i += blockDim.x) {
                const unsigned int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = sk[i], b = sk[j];
                    if (desc ? (a < b) : (a > b)) {
                        sk[i] = b;
                        sk[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (unsigned int i = threadIdx.x; i < n; i += blockDim.x) keys[i] = sk[i];
}

template <typename TIn>
__device__ __forceinline__ double to_f64(TIn v) { return (double)to_f32(v); }

// One warp per candidate: N and D in FP64 from the master stack, the FP64
// footprints and the FP64 inverse variance.
// FP64 inverse variance of every pixel for the re-score: 1 / (s * s) from
// the FP32 noise value s in FP64, 0 where the pixel is masked or s is not a
// usable noise value (s <= 0 or not finite; a finite FP32 s never makes the
// FP64 quotient 0).  Computed once per re-score instead of per tap.
__global__ void k_lambda64(const float *__restrict__ sigma, const uint8_t *__restrict__ mask, int64_t P,
                           double *__restrict__ lam64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = (double)sigma[i];
        lam64[i] = ((mask && mask[i]) || !(s > 0.0) || !isfinite(s)) ? 0.0 : 1.0 / (s * s);
    }
}

template <typename TIn>
__global__ void k_rescore(const TIn *__restrict__ r, int64_t fstride, int64_t rstride,
                          const float *__restrict__ scale, const double *__restrict__ lam64,
                          const double *__restrict__ taps64,
                          const int32_t *__restrict__ shifts, const float *__restrict__ snr_max,
                          const int32_t *__restrict__ argmax, const unsigned long long *__restrict__ keys,
                          const SelState *st, unsigned int cap, int T, int64_t H, int64_t W,
                          mf_candidate *__restrict__ out, int32_t *__restrict__ n_out) {
    const unsigned int n = st->count < cap ? st->count : cap;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp == 0 && lane == 0) *n_out = (int32_t)n;
    if ((unsigned)warp >= n) return;
    const unsigned long long key = keys[warp];
    const int64_t idx = (int64_t)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFull));
    const int64_t py = idx / W, px = idx % W;
    const int k = argmax[idx];
    double num = 0.0, den = 0.0;
    for (int t = lane; t < T; t += 32) {
        const size_t kt = (size_t)k * T + t;
        const int sx = shifts[kt * 2 + 0], sy = shifts[kt * 2 + 1];
        const double sc = scale ? (double)scale[t] : 1.0;
        const double *w = taps64 + kt * 25;
        for (int b = 0; b < 5; b++) {
            const int64_t qy = py + sy + b - 2;
            if (qy < 0 || qy >= H) continue;
            for (int a = 0; a < 5; a++) {
                const int64_t qx = px + sx + a - 2;
                if (qx < 0 || qx >= W) continue;
                const int64_t q = qy * W + qx;
                const double lam = lam64[q];
                if (lam == 0.0) continue;  // masked, or no usable noise value
                const double wl = w[b * 5 + a] * lam;  // w lambda, shared by both sums
                num = fma(wl, sc * to_f64(r[t * fstride + qy * rstride + qx]), num);
                den = fma(w[b * 5 + a], wl, den);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        num += __shfl_xor_sync(0xffffffffu, num, o);
        den += __shfl_xor_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        mf_candidate c;
        c.y = (int32_t)py;
        c.x = (int32_t)px;
        c.k = k;
        c.reserved = 0;
        c.snr = den > 0.0 ? num / sqrt(den) : 0.0;
        c.flux = den > 0.0 ? num / den : 0.0;
        c.snr_search = snr_max[idx];
        c.reserved2 = 0.f;
        out[warp] = c;
    }
}

}  // namespace

SelectLayout select_layout(int64_t P, int32_t k_top) {
    SelectLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    };
    L.keys_off = take((size_t)P * sizeof(unsigned long long));
    L.hist_off = take(65536 * sizeof(unsigned int));
    L.st_off = take(sizeof(SelState));
    L.top_off = take((size_t)k_top * sizeof(unsigned long long));
    L.total = off;
    return L;
}

int launch_select(const float *score, const int32_t *valid, int64_t P, int32_t k_top, char *ws,
                  const SelectLayout &L, void *stream_, char *err, size_t errlen) {
    cudaStream_t stream = (cudaStream_t)stream_;
    if (k_top > kMaxTop) {
        snprintf(err, errlen, "k_top above %d", kMaxTop);
        return (int)cudaErrorInvalidValue;
    }
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(ws + L.keys_off);
    unsigned int *hist = reinterpret_cast<unsigned int *>(ws + L.hist_off);
    SelState *sst = reinterpret_cast<SelState *>(ws + L.st_off);
    unsigned long long *top = reinterpret_cast<unsigned long long *>(ws + L.top_off);
    cudaError_t e = cudaMemsetAsync(ws + L.hist_off, 0, L.top_off - L.hist_off, stream);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return (int)e;
    }
    {
        LaunchScope ls(kKSelect, stream);
        k_sel_keys<<<grid_for(P, 256), 256, 0, stream>>>(score, valid, P, keys, hist, sst);
    }
    MF_CHECK_LAUNCH("k_sel_keys");
    for (int pass = 0; pass < 4; pass++) {
        if (pass > 0) {
            LaunchScope ls(kKSelect, stream);
            k_sel_hist<<<grid_for(P, 256), 256, 0, stream>>>(keys, P, pass, hist, sst);
            MF_CHECK_LAUNCH("k_sel_hist");
        }
        LaunchScope ls(kKSelect, stream);
        k_sel_pick<<<1, 1024, 0, stream>>>(hist, pass, sst, (unsigned)k_top);
        MF_CHECK_LAUNCH("k_sel_pick");
    }
    {
        LaunchScope ls(kKCompact, stream);
        k_sel_compact<<<grid_for(P, 256), 256, 0, stream>>>(keys, P, top, sst, (unsigned)k_top);
    }
    MF_CHECK_LAUNCH("k_sel_compact");
    {
        unsigned int m = 1;
        while (m < (unsigned)k_top) m <<= 1;
        const size_t smem = (size_t)m * sizeof(unsigned long long);
        e = cudaFuncSetAttribute(k_sel_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "cudaFuncSetAttribute(sort): %s", cudaGetErrorString(e));
            return (int)e;
        }
        LaunchScope ls(kKSort, stream);
        k_sel_sort<<<1, 1024, smem, stream>>>(top, sst, (unsigned)k_top);
    }
    MF_CHECK_LAUNCH("k_sel_sort");
    return 0;
}

size_t rescore_workspace(int64_t H, int64_t W, int32_t k_top) { return select_layout(H * W, k_top).total; }

int launch_rescore(const RescoreArgs &a, char *err, size_t errlen) {
    const mf_stack &st = *a.stack;
    const mf_prf_table &tab = *a.tab;
    cudaStream_t stream = (cudaStream_t)a.stream;
    const int64_t H = st.H, W = st.W, P = H * W;
    const SelectLayout L = select_layout(P, a.k_top);
    SelState *sst = reinterpret_cast<SelState *>(a.ws + L.st_off);
    unsigned long long *top = reinterpret_cast<unsigned long long *>(a.ws + L.top_off);
    int rc = launch_select(a.snr_max, a.argmax, P, a.k_top, a.ws, L, stream, err, errlen);
    if (rc) return rc;
    // the selection is done with the per-pixel keys: their space holds the
    // FP64 inverse variance (P doubles) the re-score reads (both launches
    // count as the re-score)
    static_assert(sizeof(double) == sizeof(unsigned long long), "one double per key");
    double *lam64 = reinterpret_cast<double *>(a.ws + L.keys_off);
    {
        LaunchScope ls(kKRescore, stream);
        k_lambda64<<<grid_for(P, 256), 256, 0, stream>>>(a.sigma, a.mask, P, lam64);
    }
    MF_CHECK_LAUNCH("k_lambda64");
    {
        const int threads = 256;
        const int blocks = (int)(((int64_t)a.k_top * 32 + threads - 1) / threads);
        LaunchScope ls(kKRescore, stream);
        const int64_t fs = st.frame_stride, rs = st.row_stride;
        switch (st.dtype) {
            case MF_F32:
                k_rescore<float><<<blocks, threads, 0, stream>>>(
                    (const float *)st.data, fs, rs, st.frame_scale, lam64, tab.d_taps64, tab.d_shifts,
                    a.snr_max, a.argmax, top, sst, (unsigned)a.k_top, tab.T, H, W, a.out, a.n_out);
                break;
            case MF_BF16:
                k_rescore<__nv_bfloat16><<<blocks, threads, 0, stream>>>(
                    (const __nv_bfloat16 *)st.data, fs, rs, st.frame_scale, lam64, tab.d_taps64,
                    tab.d_shifts, a.snr_max, a.argmax, top, sst, (unsigned)a.k_top, tab.T, H, W, a.out, a.n_out);
                break;
            default:
                k_rescore<__half><<<blocks, threads, 0, stream>>>(
                    (const __half *)st.data, fs, rs, st.frame_scale, lam64, tab.d_taps64, tab.d_shifts,
                    a.snr_max, a.argmax, top, sst, (unsigned)a.k_top, tab.T, H, W, a.out, a.n_out);
                break;
        }
    }
    MF_CHECK_LAUNCH("k_rescore");
    return 0;
}

namespace {

// One CTA whose thread 0 waits on an mbarrier that nothing arrives at, with
// the same bounded wait as every kernel of the library: the wait gives up,
// records `code` in the status word (and in a search's status slot, if one is
// given) and returns, and the CTA exits.  It exercises the failure path of
// the search kernels on purpose; nothing faults, traps or hangs.
__global__ void k_wait_probe(int code, int *slot) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(smem_u32(&bar), 0u, code) && slot) atomicCAS(slot, 0, code);
    __syncthreads();
    if (threadIdx.x == 0) mbar_inval(smem_u32(&bar));
}

}  // namespace

int launch_wait_probe(void *stream, int *slot, char *err, size_t errlen) {
    k_wait_probe<<<1, 32, 0, (cudaStream_t)stream>>>(kWaitProbeCode, slot);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "k_wait_probe: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

int *status_word(char *err, size_t errlen) {
    static std::mutex mu;
    static std::vector<int *> addr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaGetDevice: %s", cudaGetErrorString(e));
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(mu);
    if ((int)addr.size() <= dev) addr.resize(dev + 1, nullptr);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_status);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "cudaGetSymbolAddress(status word): %s", cudaGetErrorString(e));
            return nullptr;
        }
        addr[dev] = static_cast<int *>(p);
    }
    return addr[dev];
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
