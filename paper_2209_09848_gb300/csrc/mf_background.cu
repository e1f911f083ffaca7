// Per-pixel background re-fit (Section 3.1 of Ganapathi 2022): with the
// low-resolution scattered light fixed, every pixel's time series is
// regressed on the same six jitter basis values under the Huber loss,
// reached by least-squares steps on clipped residuals.
//
// The host turns the basis Phi [T][6] into an orthonormal one, Q = Phi R^-1
// (G = Phi^T Phi = R^T R, FP64 Cholesky), so the shared Gram inverse becomes
// the identity and each step is beta_Q <- beta_Q + Q^T psi(y - Q beta_Q):
// the same iterates as beta <- beta + G^-1 Phi^T psi(y - Phi beta) with
// beta = R^-1 beta_Q, but with well-scaled FP32 arithmetic.
//
// k_refit: one thread per pixel, 256 consecutive pixels per CTA, every
// thread walking the frames in the same order so the CTA stages Q 256 frames
// at a time in shared memory; a thread loads eight frames before using them,
// so eight loads per thread are in flight.  Pass 0 reads D_t, subtracts the bilinear
// scattered light, writes y_t to the residual buffer and sums Q^T (y - y_0)
// (the first frame's value taken out, so FP32 sums see noise-sized values);
// each of the `iterations` passes reads y_t back and sums Q^T psi(e); the
// last pass writes r_t = y_t - Q beta_Q.  FP32 partial sums over 32 frames
// are added into FP32 totals.  Memory-bound: (iterations + 4) x 4 bytes per
// pixel and frame.

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "mf_internal.h"

namespace mf {
namespace {

constexpr int kRefitThreads = 256;
constexpr int kRefitChunk = 256;  // frames of Q staged in shared memory
constexpr int kRefitBlock = 32;   // frames per FP32 partial sum
constexpr int kRefitUnroll = 8;   // frames whose loads are in flight together

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

__global__ void __launch_bounds__(kRefitThreads) k_refit(const float *data, int T, int H, int W,
                                                         const float *__restrict__ scatter, int n,
                                                         const float4 *__restrict__ Q,
                                                         const double *__restrict__ Rinv,
                                                         const double *__restrict__ q1, int iterations, float delta,
                                                         float *resid, float *__restrict__ coef) {
    __shared__ float4 qs[kRefitChunk * 2];
    const int64_t P = (int64_t)H * W;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = p < P;
    // bilinear weights of this pixel on the scattered-light grid
    int o00 = 0, o01 = 0, o10 = 0, o11 = 0;
    float fy = 0.f, fx = 0.f;
    if (scatter && live) {
        const int i = (int)(p / W), j = (int)(p % W);
        const float u = fminf(fmaxf(((float)i + 0.5f) * (float)n / (float)H - 0.5f, 0.f), (float)(n - 1));
        const float v = fminf(fmaxf(((float)j + 0.5f) * (float)n / (float)W - 0.5f, 0.f), (float)(n - 1));
        const int i0 = (int)floorf(u), j0 = (int)floorf(v);
        const int i1 = min(i0 + 1, n - 1), j1 = min(j0 + 1, n - 1);
        fy = u - (float)i0;
        fx = v - (float)j0;
        o00 = i0 * n + j0;
        o01 = i0 * n + j1;
        o10 = i1 * n + j0;
        o11 = i1 * n + j1;
    }
    float beta[6], acc[6], part[6];
#pragma unroll
    for (int k = 0; k < 6; k++) beta[k] = 0.f;
    float y0 = 0.f;
    // pass 0: least-squares start; passes 1 .. iterations: clipped steps;
    // pass iterations + 1: residuals
    for (int pass = 0; pass <= iterations + 1; pass++) {
        const bool last = pass == iterations + 1;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            acc[k] = 0.f;
            part[k] = 0.f;
        }
        for (int c0 = 0; c0 < T; c0 += kRefitChunk) {
            const int cn = min(kRefitChunk, T - c0);
            __syncthreads();
            for (int q = threadIdx.x; q < 2 * cn; q += blockDim.x) qs[q] = Q[(size_t)c0 * 2 + q];
            __syncthreads();
            if (!live) continue;
            // eight frames at a time: their loads are issued before any use
            for (int tt0 = 0; tt0 < cn; tt0 += kRefitUnroll) {
                float v[kRefitUnroll];
                const float *src = pass == 0 ? data : resid;
#pragma unroll
                for (int u = 0; u < kRefitUnroll; u++)
                    v[u] = tt0 + u < cn ? src[(size_t)(c0 + tt0 + u) * P + p] : 0.f;
#pragma unroll
                for (int u = 0; u < kRefitUnroll; u++) {
                    const int tt = tt0 + u;
                    if (tt >= cn) break;
                    const int t = c0 + tt;
                    const size_t idx = (size_t)t * P + p;
                    const float4 qa = qs[2 * tt], qb = qs[2 * tt + 1];
                    const float qv[6] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y};
                    float val;
                    if (pass == 0) {
                        float y = v[u];
                        if (scatter) {
                            const float *S = scatter + (size_t)t * n * n;
                            const float top = S[o00] * (1.f - fx) + S[o01] * fx;
                            const float bot = S[o10] * (1.f - fx) + S[o11] * fx;
                            y -= top * (1.f - fy) + bot * fy;
                        }
                        resid[idx] = y;
                        if (t == 0) y0 = y;
                        val = y - y0;
                    } else {
                        float fit = 0.f;
#pragma unroll
                        for (int k = 0; k < 6; k++) fit = fmaf(qv[k], beta[k], fit);
                        const float e = v[u] - fit;
                        if (last) {
                            resid[idx] = e;
                            continue;
                        }
                        val = fminf(fmaxf(e, -delta), delta);
                    }
#pragma unroll
                    for (int k = 0; k < 6; k++) part[k] = fmaf(qv[k], val, part[k]);
                    if ((t + 1) % kRefitBlock == 0) {
#pragma unroll
                        for (int k = 0; k < 6; k++) {
                            acc[k] += part[k];
                            part[k] = 0.f;
                        }
                    }
                }
            }
        }
        if (last) break;
#pragma unroll
        for (int k = 0; k < 6; k++) {
            const float s = acc[k] + part[k];
            beta[k] = pass == 0 ? s + y0 * (float)q1[k] : beta[k] + s;
        }
    }
    if (coef && live) {
        // coefficients in the basis (1, x, y, x^2, y^2, x y): beta = R^-1 beta_Q
#pragma unroll
        for (int i = 0; i < 6; i++) {
            double c = 0.0;
#pragma unroll
            for (int k = 0; k < 6; k++) c += Rinv[i * 6 + k] * (double)beta[k];
            coef[(size_t)p * 6 + i] = (float)c;
        }
    }
}

}  // namespace

size_t refit_q_off() { return 0; }
size_t refit_rinv_off(int64_t T) { return align256((size_t)T * kRefitBasisPitch * sizeof(float)); }
size_t refit_q1_off(int64_t T) { return refit_rinv_off(T) + align256(36 * sizeof(double)); }
size_t refit_workspace(int64_t T) { return refit_q1_off(T) + align256(6 * sizeof(double)); }

int launch_refit(const RefitArgs &a, char *err, size_t errlen) {
    cudaStream_t stream = (cudaStream_t)a.stream;
    const int64_t P = a.H * a.W;
    const float4 *Q = reinterpret_cast<const float4 *>(a.ws + refit_q_off());
    const double *Rinv = reinterpret_cast<const double *>(a.ws + refit_rinv_off(a.T));
    const double *q1 = reinterpret_cast<const double *>(a.ws + refit_q1_off(a.T));
    const ProfToken tok = prof_begin(kKRefit, stream);
    k_refit<<<(unsigned)((P + kRefitThreads - 1) / kRefitThreads), kRefitThreads, 0, stream>>>(
        a.data, (int)a.T, (int)a.H, (int)a.W, a.scatter, a.n, Q, Rinv, q1, a.iterations, a.delta, a.resid, a.coef);
    prof_end(tok);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(err, errlen, "k_refit: %s", cudaGetErrorString(e));
        return (int)e;
    }
    return 0;
}

}  // namespace mf
