// Score normalisation and candidate extraction (Section 3.3 of Ganapathi
// 2022): each pixel's best score in units of the standard deviation of the
// scores in the square centred on it, candidates above a threshold, and one
// detection per group of touching candidates.
//
// Data path, all on the caller's stream, P = H x W pixels:
//   k_det_cols     thread per (column, chunk of 64 rows): sliding sums over
//                  the window's rows of the valid scores, their squares and
//                  the valid count (FP64, FP64, int32 per pixel);
//   k_det_rows     block per (row, 1024-column tile), row-major: the tile's column sums
//                  plus halo in shared memory, prefix sums along the row,
//                  window sums as prefix differences, then mean, sigma, z,
//                  the candidate flag and the union-find parent (itself for a
//                  candidate, -1 otherwise);
//   k_det_union    thread per candidate: union with the candidate neighbours
//                  above it and to its left (lock-free union-find in which a
//                  root only ever hangs below a smaller index, so every
//                  component ends rooted at its smallest flat index);
//   k_det_flatten  every candidate points at its root;
//   k_det_peak     per component the largest z (atomicMax on order-
//                  preserving FP64 bits) and the pixel count; then the
//                  smallest index attaining that z;
//   k_det_mark     per root: the peak's FP32 z and root id into a sparse map;
//   top-k select   the shared radix select and sort (z desc, index asc);
//   k_det_emit     one record per selected detection and the counts.
// Every reduction is an integer atomic or a fixed-order sum, so reruns are
// bit-identical.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>

#include "mf_internal.h"

namespace mf {
namespace {

constexpr int kRowTile = 1024;    // output columns per k_det_rows block
constexpr int kRowThreads = 256;
constexpr int kUnionBudget = 1 << 20;  // iterations of one find or merge loop

struct DetectLayout {
    size_t c1, c2, cn, zd, mean, sd, parent, vsel, ncomp, sel_base, total;
    // aliases once the window sums are consumed
    size_t zmax() const { return c1; }                            // P x uint64
    size_t peak() const { return c2; }                            // P x uint32
    size_t npix(int64_t P) const { return c2 + (size_t)P * 4; }   // P x int32
    size_t zsel() const { return cn; }                            // P x float
    SelectLayout sel;
};

DetectLayout detect_layout(int64_t P, int32_t max_out) {
    DetectLayout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) / 256 * 256;
        return o;
    };
    L.c1 = take((size_t)P * 8);
    L.c2 = take((size_t)P * 8);
    L.cn = take((size_t)P * 4);
    L.zd = take((size_t)P * 8);
    L.mean = take((size_t)P * 8);
    L.sd = take((size_t)P * 8);
    L.parent = take((size_t)P * 4);
    L.vsel = take((size_t)P * 4);
    L.ncomp = take(16);
    L.sel_base = off;
    L.sel = select_layout(P, max_out > 0 ? max_out : 1);
    L.total = L.sel_base + L.sel.total;
    return L;
}

__device__ __forceinline__ unsigned long long ord_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

// Vertical window sums: for output row y the rows y - R .. y + R clipped to
// the image.  A thread owns one column of a chunk of kColChunk output rows:
// it sums its first row's window directly, then each step adds the row
// entering the window and drops the row leaving it.
constexpr int kColChunk = 64;
__global__ void k_det_cols(const float *__restrict__ s, const int32_t *__restrict__ am, int H, int W, int R,
                           double *__restrict__ c1, double *__restrict__ c2, int *__restrict__ cn) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= W) return;
    for (int y0 = blockIdx.y * kColChunk; y0 < H; y0 += gridDim.y * kColChunk) {
        double a1 = 0.0, a2 = 0.0;
        int an = 0;
        auto take = [&](int y, bool add) {
            if (y < 0 || y >= H) return;
            const size_t i = (size_t)y * W + x;
            if (am[i] < 0) return;
            const double v = (double)s[i];
            if (add) {
                a1 += v;
                a2 += v * v;
                an += 1;
            } else {
                a1 -= v;
                a2 -= v * v;
                an -= 1;
            }
        };
        for (int y = max(0, y0 - R - 1); y < y0 + R && y < H; y++) take(y, true);
        const int y1 = min(H, y0 + kColChunk);
        for (int y = y0; y < y1; y++) {
            take(y + R, true);
            take(y - R - 1, false);
            const size_t i = (size_t)y * W + x;
            c1[i] = a1;
            c2[i] = a2;
            cn[i] = an;
        }
    }
}

// Exclusive scan of one value over the block (fixed order: the warp's
// shuffles, then the warps' totals in order).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T o = __shfl_up_sync(0xffffffffu, ti, d);
            if (lane >= d) ti += o;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = ti - t;  // exclusive offsets of the warps
    }
    __syncthreads();
    const T r = warp_tot[warp] + inc - v;
    __syncthreads();  // warp_tot may be reused
    return r;
}

// Horizontal window sums, statistics, z and the candidate flag for the
// columns x0 .. x0 + kRowTile - 1 of row y.  Shared entry j holds column
// lo + j, lo = x0 - R - 1 (0 outside the image); after the prefix scan the
// window [x - R, x + R] of column x = x0 + t is entries t + 1 .. t + 2R + 1.
__global__ void __launch_bounds__(kRowThreads) k_det_rows(
    const float *__restrict__ s, const int32_t *__restrict__ am, const double *__restrict__ c1,
    const double *__restrict__ c2, const int *__restrict__ cn, int H, int W, int R, double thr, int submean,
    float *__restrict__ z_out, double *__restrict__ zd, double *__restrict__ mean_o, double *__restrict__ sd_o,
    int *__restrict__ parent) {
    extern __shared__ double sm[];
    __shared__ double wt1[kRowThreads / 32], wt2[kRowThreads / 32];
    __shared__ int wtn[kRowThreads / 32];
    const int tiles = (W + kRowTile - 1) / kRowTile;
    const int y = (int)(blockIdx.x / tiles);
    const int x0 = (int)(blockIdx.x % tiles) * kRowTile;
    const int lo = x0 - R - 1;
    const int L = kRowTile + 2 * R + 1;
    double *p1 = sm;
    double *p2 = sm + L;
    int *pn = reinterpret_cast<int *>(sm + 2 * L);
    const size_t row = (size_t)y * W;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        const int x = lo + j;
        const bool in = x >= 0 && x < W;
        p1[j] = in ? c1[row + x] : 0.0;
        p2[j] = in ? c2[row + x] : 0.0;
        pn[j] = in ? cn[row + x] : 0;
    }
    __syncthreads();
    const int per = (L + blockDim.x - 1) / blockDim.x;
    const int j0 = min(L, (int)threadIdx.x * per), j1 = min(L, j0 + per);
    double r1 = 0.0, r2 = 0.0;
    int rn = 0;
    for (int j = j0; j < j1; j++) {
        r1 += p1[j];
        p1[j] = r1;
        r2 += p2[j];
        p2[j] = r2;
        rn += pn[j];
        pn[j] = rn;
    }
    const double o1 = block_exclusive_scan(r1, wt1);
    const double o2 = block_exclusive_scan(r2, wt2);
    const int on = block_exclusive_scan(rn, wtn);
    for (int j = j0; j < j1; j++) {
        p1[j] += o1;
        p2[j] += o2;
        pn[j] += on;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kRowTile; t += blockDim.x) {
        const int x = x0 + t;
        if (x >= W) break;
        const int n = pn[t + 2 * R + 1] - pn[t];
        const double s1 = p1[t + 2 * R + 1] - p1[t];
        const double s2 = p2[t + 2 * R + 1] - p2[t];
        const size_t i = row + x;
        double mean = 0.0, var = 0.0, z = 0.0;
        if (n > 0) {
            const double inv_n = 1.0 / n;
            mean = s1 * inv_n;
            var = fmax(s2 * inv_n - mean * mean, 0.0);
        }
        const double sd = sqrt(var);
        bool flag = false;
        if (am[i] >= 0 && n >= 2 && var > 1e-12 * (mean * mean + var)) {
            z = ((double)s[i] - (submean ? mean : 0.0)) * rsqrt(var);
            flag = z > thr;
        }
        zd[i] = z;
        mean_o[i] = mean;
        sd_o[i] = sd;
        if (z_out) z_out[i] = (float)z;
        parent[i] = flag ? (int)i : -1;
    }
}

__device__ __forceinline__ int uf_find(const int *parent, int x, int *status) {
    for (int it = 0; it < kUnionBudget; it++) {
        const int p = *(const volatile int *)(parent + x);
        if (p == x) return x;
        x = p;
    }
    atomicCAS(status, 0, 3);
    return x;
}

// Join the components of candidates a and b: the larger root is hung below
// the smaller one; if it stopped being a root meanwhile, retry from its new
// parent (the pixel keeps a parent in the same component either way).
__device__ __forceinline__ void uf_merge(int *parent, int a, int b, int *status) {
    for (int it = 0; it < kUnionBudget; it++) {
        a = uf_find(parent, a, status);
        b = uf_find(parent, b, status);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicMin(parent + a, b);
        if (old == a) return;
        a = old;
    }
    atomicCAS(status, 0, 3);
}

__global__ void k_det_union(int *__restrict__ parent, int H, int W, int *status) {
    const int64_t P = (int64_t)H * W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (parent[i] < 0) continue;
        const int y = (int)(i / W), x = (int)(i % W);
        const int me = (int)i;
        if (x > 0 && parent[i - 1] >= 0) uf_merge(parent, me, me - 1, status);
        if (y > 0) {
            const int64_t up = i - W;
            if (x > 0 && parent[up - 1] >= 0) uf_merge(parent, me, (int)(up - 1), status);
            if (parent[up] >= 0) uf_merge(parent, me, (int)up, status);
            if (x + 1 < W && parent[up + 1] >= 0) uf_merge(parent, me, (int)(up + 1), status);
        }
    }
}

__global__ void k_det_flatten(int *__restrict__ parent, int64_t P, int *status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x)
        if (parent[i] >= 0) parent[i] = uf_find(parent, (int)i, status);
}

__global__ void k_det_peak_z(const int *__restrict__ parent, const double *__restrict__ zd, int64_t P,
                             unsigned long long *__restrict__ zmax, int *__restrict__ npix) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = parent[i];
        if (r < 0) continue;
        atomicMax(zmax + r, ord_bits(zd[i]));
        atomicAdd(npix + r, 1);
    }
}

__global__ void k_det_peak_at(const int *__restrict__ parent, const double *__restrict__ zd, int64_t P,
                              const unsigned long long *__restrict__ zmax, unsigned int *__restrict__ peak) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = parent[i];
        if (r < 0) continue;
        if (ord_bits(zd[i]) == zmax[r]) atomicMin(peak + r, (unsigned int)i);
    }
}

__global__ void k_det_mark(const int *__restrict__ parent, const double *__restrict__ zd, int64_t P,
                           const unsigned int *__restrict__ peak, float *__restrict__ zsel, int *__restrict__ vsel,
                           int *ncomp) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        if (parent[i] != (int)i) continue;
        const unsigned int pk = peak[i];
        zsel[pk] = (float)zd[pk];
        vsel[pk] = (int)i;
        atomicAdd(ncomp, 1);
    }
}

__global__ void k_det_emit(const unsigned long long *__restrict__ top, const SelState *st, int max_out,
                           const int *__restrict__ vsel, const float *__restrict__ s, const int32_t *__restrict__ am,
                           const double *__restrict__ zd, const double *__restrict__ mean_o,
                           const double *__restrict__ sd_o, const int *__restrict__ npix, int W, const int *ncomp,
                           mf_detection *__restrict__ out, int32_t *__restrict__ n_out) {
    const int n = st ? (int)min(st->count, (unsigned int)max_out) : 0;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        n_out[0] = *ncomp;
        n_out[1] = n;
    }
    if (i >= n) return;
    const unsigned long long key = top[i];
    const int p = (int)(0xFFFFFFFFu - (unsigned int)(key & 0xFFFFFFFFull));
    mf_detection d;
    d.y = p / W;
    d.x = p % W;
    d.k = am[p];
    d.npix = npix[vsel[p]];
    d.z = zd[p];
    d.mean = mean_o[p];
    d.sigma = sd_o[p];
    d.snr = s[p];
    d.reserved = 0;
    out[i] = d;
}

int grid_for(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

struct Scope {
    ProfToken t;
    Scope(int kid, cudaStream_t s) : t(prof_begin(kid, s)) {}
    ~Scope() { prof_end(t); }
};

}  // namespace

size_t detect_workspace(int64_t H, int64_t W, int32_t max_out) { return detect_layout(H * W, max_out).total; }

int launch_detect(const DetectArgs &a, char *err, size_t errlen) {
    cudaStream_t stream = (cudaStream_t)a.stream;
    const int H = (int)a.H, W = (int)a.W;
    const int64_t P = a.H * a.W;
    const int R = a.window / 2;
    const DetectLayout L = detect_layout(P, a.max_out);
    char *ws = a.ws;
    double *c1 = reinterpret_cast<double *>(ws + L.c1);
    double *c2 = reinterpret_cast<double *>(ws + L.c2);
    int *cn = reinterpret_cast<int *>(ws + L.cn);
    double *zd = reinterpret_cast<double *>(ws + L.zd);
    double *mean = reinterpret_cast<double *>(ws + L.mean);
    double *sd = reinterpret_cast<double *>(ws + L.sd);
    int *parent = reinterpret_cast<int *>(ws + L.parent);
    int *vsel = reinterpret_cast<int *>(ws + L.vsel);
    int *ncomp = reinterpret_cast<int *>(ws + L.ncomp);
    unsigned long long *zmax = reinterpret_cast<unsigned long long *>(ws + L.zmax());
    unsigned int *peak = reinterpret_cast<unsigned int *>(ws + L.peak());
    int *npix = reinterpret_cast<int *>(ws + L.npix(P));
    float *zsel = reinterpret_cast<float *>(ws + L.zsel());
    int *status = status_word(err, errlen);
    if (!status) return (int)cudaErrorUnknown;
    cudaError_t e;
#define DET_CHECK(what)                                                          \
    do {                                                                         \
        e = cudaGetLastError();                                                  \
        if (e != cudaSuccess) {                                                  \
            snprintf(err, errlen, "%s: %s", what, cudaGetErrorString(e));        \
            return (int)e;                                                       \
        }                                                                        \
    } while (0)
    {
        Scope sc(kKDetStats, stream);
        const dim3 grid((unsigned)((W + 127) / 128), (unsigned)std::min(65535, (H + kColChunk - 1) / kColChunk));
        k_det_cols<<<grid, 128, 0, stream>>>(a.snr_max, a.argmax, H, W, R, c1, c2, cn);
    }
    DET_CHECK("k_det_cols");
    {
        const size_t smem = (size_t)(kRowTile + 2 * R + 1) * (8 + 8 + 4);
        e = cudaFuncSetAttribute(k_det_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            snprintf(err, errlen, "cudaFuncSetAttribute(k_det_rows): %s", cudaGetErrorString(e));
            return (int)e;
        }
        Scope sc(kKDetStats, stream);
        const unsigned grid = (unsigned)(((W + kRowTile - 1) / kRowTile) * (int64_t)H);
        k_det_rows<<<grid, kRowThreads, smem, stream>>>(a.snr_max, a.argmax, c1, c2, cn, H, W, R, a.threshold,
                                                        a.subtract_mean, a.z_out, zd, mean, sd, parent);
    }
    DET_CHECK("k_det_rows");
    // the window sums are consumed: their space holds the per-root maxima,
    // peaks and counts from here on
    e = cudaMemsetAsync(zmax, 0, (size_t)P * 8, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(peak, 0xFF, (size_t)P * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(npix, 0, (size_t)P * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(vsel, 0xFF, (size_t)P * 4, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ncomp, 0, 16, stream);
    if (e != cudaSuccess) {
        snprintf(err, errlen, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return (int)e;
    }
    {
        Scope sc(kKDetComponents, stream);
        const int g = grid_for(P, 256);
        k_det_union<<<g, 256, 0, stream>>>(parent, H, W, status);
        k_det_flatten<<<g, 256, 0, stream>>>(parent, P, status);
        k_det_peak_z<<<g, 256, 0, stream>>>(parent, zd, P, zmax, npix);
        k_det_peak_at<<<g, 256, 0, stream>>>(parent, zd, P, zmax, peak);
        k_det_mark<<<g, 256, 0, stream>>>(parent, zd, P, peak, zsel, vsel, ncomp);
    }
    DET_CHECK("k_det components");
    const SelState *sst = nullptr;
    const unsigned long long *top = nullptr;
    if (a.max_out > 0) {
        char *sws = ws + L.sel_base;
        const int rc = launch_select(zsel, vsel, P, a.max_out, sws, L.sel, stream, err, errlen);
        if (rc) return rc;
        sst = reinterpret_cast<const SelState *>(sws + L.sel.st_off);
        top = reinterpret_cast<const unsigned long long *>(sws + L.sel.top_off);
    }
    {
        Scope sc(kKDetEmit, stream);
        const int n = a.max_out > 0 ? a.max_out : 1;
        k_det_emit<<<(n + 255) / 256, 256, 0, stream>>>(top, sst, a.max_out, vsel, a.snr_max, a.argmax, zd, mean,
                                                        sd, npix, W, ncomp, a.out, a.n_out);
    }
    DET_CHECK("k_det_emit");
#undef DET_CHECK
    return 0;
}

}  // namespace mf
