// Host side of libmf: filter-bank construction, trajectory grouping, argument
// validation and the C entry points declared in include/mf.h.
//
// The filter bank follows Section 3.2 of Ganapathi (2022): one filter per
// trajectory, the trajectory line convolved with the PRF.  It is stored in
// sparse form, a base shift and a 5x5 footprint per (trajectory, frame).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <numeric>
#include <string>

#include "mf_internal.h"

namespace {

thread_local std::string g_err;

mf_status fail(mf_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

mf_status ok() {
    g_err.clear();
    return MF_OK;
}

int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// One axis of the PRF's 5 x 5 footprint for a source at sub-pixel offset ph
// from the base pixel, before normalisation (Section 2: the PRF shares a
// point source's flux between neighbouring pixels).  kind 0 integrates a
// Gaussian over each pixel, kind 1 samples it at the pixel centre, kind 2 is
// the shift-stack filter of Section 3.2 (all the weight in the base pixel).
void axis_profile(int kind, double sigma, double ph, double *g) {
    if (kind == 2) {
        for (int i = 0; i < 5; i++) g[i] = i == 2 ? 1.0 : 0.0;
    } else if (kind == 0) {
        // pixel d spans [d - 1/2, d + 1/2]: six shared boundaries
        const double s = sigma * std::sqrt(2.0);
        double e[6];
        for (int i = 0; i < 6; i++) e[i] = std::erf((i - 2.5 - ph) / s);
        for (int i = 0; i < 5; i++) g[i] = 0.5 * (e[i + 1] - e[i]);
    } else {
        for (int i = 0; i < 5; i++) {
            const int d = i - 2;
            g[i] = std::exp(-(d - ph) * (d - ph) / (2.0 * sigma * sigma));
        }
    }
}

// The footprint from its two axis profiles, renormalised to unit sum, and
// the normalised 1-D factors: w[b * 5 + a] = fy[b] * fx[a] up to rounding
// (the 5 x 5 sum is the product of the two 1-D sums).
void footprint_from_axes(const double *gx, const double *gy, double *w, double *fx, double *fy) {
    double total = 0.0;
    for (int b = 0; b < 5; b++)
        for (int a = 0; a < 5; a++) {
            w[b * 5 + a] = gy[b] * gx[a];
            total += w[b * 5 + a];
        }
    for (int i = 0; i < 25; i++) w[i] /= total;
    double sx = 0.0, sy = 0.0;
    for (int i = 0; i < 5; i++) {
        sx += gx[i];
        sy += gy[i];
    }
    for (int i = 0; i < 5; i++) {
        fx[i] = gx[i] / sx;
        fy[i] = gy[i] / sy;
    }
}

// Balanced k-d split of the velocity set into `groups` parts of at most `cap`
// members, so that trajectories sharing a CTA (and its frame window) have
// similar shifts at every frame.
void kd_split(std::vector<int> &idx, int lo, int hi, int groups, int cap, const std::vector<double> &ex,
              const std::vector<double> &ey, std::vector<std::vector<int>> &out) {
    const int n = hi - lo;
    if (groups <= 1 || n <= 1) {
        out.emplace_back(idx.begin() + lo, idx.begin() + hi);
        for (int g = 1; g < groups; g++) out.emplace_back();
        return;
    }
    double x0 = 1e300, x1 = -1e300, y0 = 1e300, y1 = -1e300;
    for (int i = lo; i < hi; i++) {
        x0 = std::min(x0, ex[idx[i]]);
        x1 = std::max(x1, ex[idx[i]]);
        y0 = std::min(y0, ey[idx[i]]);
        y1 = std::max(y1, ey[idx[i]]);
    }
    // a column of spread costs less than a row (rows are padded to a 32-word
    // pitch anyway), so split along y unless x is clearly wider
    const bool by_x = (x1 - x0) > 1.5 * (y1 - y0);
    auto key = [&](int a, int b) {
        const double pa = by_x ? ex[a] : ey[a], pb = by_x ? ex[b] : ey[b];
        if (pa != pb) return pa < pb;
        const double qa = by_x ? ey[a] : ex[a], qb = by_x ? ey[b] : ex[b];
        if (qa != qb) return qa < qb;
        return a < b;
    };
    std::sort(idx.begin() + lo, idx.begin() + hi, key);
    const int g1 = groups / 2, g2 = groups - g1;
    int n1 = (int)std::llround((double)n * g1 / groups);
    n1 = std::max(n1, n - g2 * cap);
    n1 = std::min(n1, g1 * cap);
    n1 = std::max(0, std::min(n, n1));
    kd_split(idx, lo, lo + n1, g1, cap, ex, ey, out);
    kd_split(idx, lo + n1, hi, g2, cap, ex, ey, out);
}

size_t smem_bytes(const mf::Plan &p) { return mf::numerator_smem_bytes(p.S, p.BH, p.kt()); }

// Window geometry and estimated cost of a grouping; false if it does not fit.
// Cost model per CTA and frame, in SM cycles: the numerator is latency-bound
// with one 16-warp CTA per SM, so a CTA-frame costs about the issue time of
// all its warps (idle slots included: they leave the SM with fewer warps to
// switch between), unless the shared-memory traffic of the loads plus the
// staged window takes longer.  Summed over groups and frames and divided by
// the tile area.
bool measure(mf::Plan &p, const mf_prf_table &t) {
    const int kt = p.kt();
    const mf::Shape sh = mf::kShapes[p.shape];
    int max_offx = 0, max_spread_y = 0;
    std::vector<int> rows((size_t)p.G * t.T, 0);
    for (int g = 0; g < p.G; g++) {
        for (int f = 0; f < t.T; f++) {
            int64_t mnx = INT64_MAX, mxx = INT64_MIN, mny = INT64_MAX, mxy = INT64_MIN;
            bool any = false;
            for (int w = 0; w < kt; w++) {
                const int k = p.members[(size_t)g * kt + w];
                if (k < 0) continue;
                any = true;
                const int64_t sx = t.shifts[((size_t)k * t.T + f) * 2 + 0];
                const int64_t sy = t.shifts[((size_t)k * t.T + f) * 2 + 1];
                mnx = std::min(mnx, sx);
                mxx = std::max(mxx, sx);
                mny = std::min(mny, sy);
                mxy = std::max(mxy, sy);
            }
            if (!any) continue;
            const int64_t rox = 4 * floor_div(mnx - 2, 4);
            max_offx = (int)std::max<int64_t>(max_offx, mxx - 2 - rox);
            max_spread_y = (int)std::max<int64_t>(max_spread_y, mxy - mny);
            rows[(size_t)g * t.T + f] = (int)round_up(mxy - mny + p.tile_h() + 4, mf::kLoadRows);
        }
    }
    // widest read: offx + tile_w - 32 + 24 (lanes) + 7 (skew) + 3 (alignment) + 12
    p.S = (int)round_up(max_offx + p.tile_w() + 14, 32);
    p.BH = (int)round_up(max_spread_y + p.tile_h() + 4, mf::kLoadRows);
    if (!(p.S <= 256 && p.BH <= 256 && smem_bytes(p) <= (size_t)mf::kSmemBudget)) return false;
    double cyc = 0.0;
    for (int g = 0; g < p.G; g++) {
        int active = 0;
        for (int w = 0; w < kt; w++) active += p.members[(size_t)g * kt + w] >= 0;
        const int aw = active * sh.txs * sh.tys;
        const double issue = mf::kWarps * 950.0 / 4.0;
        for (int f = 0; f < t.T; f++) {
            // the kernel stages the whole BH x S window every frame
            const double smem = aw * 105.0 + p.BH * (double)p.S / 32.0;
            cyc += std::max(issue, smem);
        }
    }
    p.cost = cyc / ((double)p.tile_h() * p.tile_w());
    return true;
}

mf_status plan_groups(mf_prf_table &t) {
    const int K = t.K;
    std::vector<double> ex(K), ey(K);
    for (int k = 0; k < K; k++) {
        // displacement over the stack, in pixels: what sets the window spread
        const size_t last = ((size_t)k * t.T + (t.T - 1)) * 2;
        const size_t first = (size_t)k * t.T * 2;
        ex[k] = (double)t.shifts[last + 0] - t.shifts[first + 0];
        ey[k] = (double)t.shifts[last + 1] - t.shifts[first + 1];
        // trajectories with equal endpoints but different start shifts (custom
        // tables) still differ at frame 0: fold that in
        ex[k] += 1e-3 * t.shifts[first + 0];
        ey[k] += 1e-3 * t.shifts[first + 1];
    }
    int mx = 0;
    for (size_t i = 0; i < t.shifts.size(); i++) mx = std::max(mx, std::abs(t.shifts[i]));
    bool have = false;
    mf::Plan best;
    for (int si = 0; si < mf::kNumShapes; si++) {
        if (t.forced_shape >= 0 && si != t.forced_shape) continue;
        const int kt = mf::kShapes[si].kt;
        int G = (K + kt - 1) / kt;
        for (;;) {
            std::vector<int> idx(K);
            std::iota(idx.begin(), idx.end(), 0);
            std::vector<std::vector<int>> parts;
            kd_split(idx, 0, K, G, kt, ex, ey, parts);
            mf::Plan p;
            p.shape = si;
            p.vec = t.forced_vec > 0 ? t.forced_vec : 2;
            p.lockstep = t.forced_lockstep >= 0 ? t.forced_lockstep : 0;
            p.G = 0;
            for (auto &part : parts)
                if (!part.empty()) p.G++;
            p.members.assign((size_t)p.G * kt, -1);
            int g = 0;
            for (auto &part : parts) {
                if (part.empty()) continue;
                std::sort(part.begin(), part.end());
                for (size_t i = 0; i < part.size(); i++) p.members[(size_t)g * kt + i] = part[i];
                g++;
            }
            if (measure(p, t)) {
                p.max_abs_shift = mx;
                if (!have || p.cost < best.cost) {
                    best = std::move(p);
                    have = true;
                }
                break;
            }
            if (G >= K) break;
            G = std::min(K, std::max(G + 1, G * 5 / 4));
        }
    }
    if (!have) return fail(MF_EUNSUPPORTED, "trajectory shifts too far apart for the frame window");
    t.plan = std::move(best);
    return MF_OK;
}

// Factored numerator: trajectories with the same v_x form a class (they
// share s_x and u_x at every frame); each class, sorted by v_y, is split into
// groups of consecutive members, one group per CTA.  The frames are split
// into segments; within a segment a CTA follows each member from its s_y at
// the segment's first frame, so the rows a group's window spans at frame t
// grow with t - (segment start) only.  For each candidate CTA geometry
// (trajectories per CTA, tile) and segment count, the window rows BH follow
// from the largest such spread, the stages from the shared-memory budget,
// and the cost from a per-frame model of one CTA in SM cycles: FP32 FMAs of
// both passes at 128 per cycle, or the shared-memory bytes they move at 128
// per cycle, whichever is larger, a fixed cost for the frame barrier, and a
// penalty when a pair of frames has more row-pass items than the CTA has
// threads; plus, per segment, writing and reading a K x P plane.  Returns
// false if the table is not separable or no geometry fits.
bool plan_factored(const mf_prf_table &t, mf::Plan &out) {
    if (t.fx.empty() || t.vx.size() != (size_t)t.K) return false;
    const int K = t.K, T = t.T;
    std::map<double, std::vector<int>> cls;
    for (int k = 0; k < K; k++) cls[t.vx[k]].push_back(k);
    std::vector<std::vector<int>> classes;
    for (auto &c : cls) {
        std::vector<int> v = c.second;
        std::sort(v.begin(), v.end(), [&](int a, int b) { return t.vy[a] != t.vy[b] ? t.vy[a] < t.vy[b] : a < b; });
        classes.push_back(std::move(v));
    }
    struct Geo {
        int th, tw;
    };
    // segment counts: starts at multiples of the record chunk, at least one
    // chunk per segment
    std::vector<int> seg_counts;
    if (t.forced_segments) {
        seg_counts.push_back(t.forced_segments);
    } else {
        for (int S : {1, 2, 3, 4, 6, 8}) seg_counts.push_back(S);
    }
    auto seg_starts = [&](int S, std::vector<int32_t> &t0) {
        t0.clear();
        for (int j = 0; j < S; j++) {
            const int f = (int)((int64_t)j * T / S) / mf::kFacRecordChunk * mf::kFacRecordChunk;
            if (t0.empty() || f > t0.back()) t0.push_back(f);
        }
        t0.push_back(T);
        return (int)t0.size() - 1;
    };
    // rows past the tile a window can hold at all (256 rows, 32-row tile,
    // 4 footprint rows)
    constexpr int kMaxSpread = 256 - 32 - 4;
    bool have = false;
    std::vector<int32_t> t0;
    std::vector<int32_t> rel((size_t)K * T);  // s_y at a frame minus s_y at its segment's first frame
    std::vector<int32_t> mn(T), mx(T);
    std::vector<int> count(kMaxSpread + 2);
    for (int S_req : seg_counts) {
        const int S = seg_starts(S_req, t0);
        if (t.forced_segments && S != S_req) continue;  // fewer frames than the segments asked for
        for (int k = 0; k < K; k++)
            for (int j = 0; j < S; j++) {
                const int32_t *sy = &t.shifts[(size_t)k * T * 2 + 1];
                const int32_t ref = sy[(size_t)t0[j] * 2];
                for (int f = t0[j]; f < t0[j + 1]; f++) rel[(size_t)k * T + f] = sy[(size_t)f * 2] - ref;
            }
        // the groups of each v_x class for the previous kt; several kt give
        // the same split, and then the same spreads
        std::vector<int> prev_split;
        std::vector<std::vector<int>> groups;
        std::vector<int32_t> seg_qy, seg_ref;
        std::vector<std::vector<std::pair<int, int>>> hist;
        int spread_max = 0, G = 0;
        for (int kt = 1; kt <= mf::kFacMaxWarps; kt++) {
            if (t.forced_group && kt != t.forced_group) continue;
            // phase planes: at most one per rounded y-phase (Q + 1 of them) or
            // per trajectory of the CTA, whichever is fewer
            const int npl = t.forced_kernel == 3 ? std::min(kt, t.phase_steps + 1) : 0;
            std::vector<Geo> geos;
            for (int tw : {32, 64}) {
                if (t.forced_tw && tw != t.forced_tw) continue;
                const int per = kt * (tw / 32);  // warps per 32 rows of tile
                if (per > mf::kFacMaxWarps) continue;
                if (t.forced_th) {
                    if (t.forced_th / 32 * per <= mf::kFacMaxWarps) geos.push_back({t.forced_th, tw});
                } else {
                    for (int th = std::min(224, 32 * (mf::kFacMaxWarps / per)); th >= 32; th -= 32)
                        geos.push_back({th, tw});
                }
            }
            if (geos.empty()) continue;
            // each v_x class splits into groups of at most kt consecutive
            // members, as even as possible
            std::vector<int> split;
            for (const auto &c : classes) split.push_back(((int)c.size() + kt - 1) / kt);
            if (split != prev_split) {
                prev_split = split;
                groups.clear();
                for (size_t ci = 0; ci < classes.size(); ci++) {
                    const auto &c = classes[ci];
                    const int n = (int)c.size(), ng = split[ci];
                    for (int g = 0, i = 0; g < ng; g++) {
                        const int sz = n / ng + (g < n % ng ? 1 : 0);
                        groups.emplace_back(c.begin() + i, c.begin() + i + sz);
                        i += sz;
                    }
                }
                G = (int)groups.size();
                size_t gmax = 0;
                for (const auto &m : groups) gmax = std::max(gmax, m.size());
                // per (group, segment): the members' smallest s_y at the
                // segment's first frame and their spread there, each member's
                // s_y there, and how many frames have each row spread (largest
                // minus smallest member shift relative to the segment start)
                // as (spread, count) pairs
                seg_qy.assign((size_t)G * S * 2, 0);
                seg_ref.assign((size_t)G * S * gmax, INT32_MIN);
                hist.assign((size_t)G * S, {});
                spread_max = 0;
                for (int g = 0; g < G && spread_max <= kMaxSpread; g++) {
                    const auto &m = groups[g];
                    for (int j = 0; j < S; j++) {
                        int rmn = INT32_MAX, rmx = INT32_MIN;
                        for (size_t i = 0; i < m.size(); i++) {
                            const int sy0 = t.shifts[((size_t)m[i] * T + t0[j]) * 2 + 1];
                            seg_ref[((size_t)g * S + j) * gmax + i] = sy0;
                            rmn = std::min(rmn, sy0);
                            rmx = std::max(rmx, sy0);
                        }
                        seg_qy[((size_t)g * S + j) * 2 + 0] = rmn;
                        seg_qy[((size_t)g * S + j) * 2 + 1] = rmx - rmn;
                    }
                    const int32_t *r0 = &rel[(size_t)m[0] * T];
                    std::copy(r0, r0 + T, mn.begin());
                    std::copy(r0, r0 + T, mx.begin());
                    for (size_t i = 1; i < m.size(); i++) {
                        const int32_t *r = &rel[(size_t)m[i] * T];
                        for (int f = 0; f < T; f++) {
                            mn[f] = std::min(mn[f], r[f]);
                            mx[f] = std::max(mx[f], r[f]);
                        }
                    }
                    for (int j = 0; j < S; j++) {
                        std::fill(count.begin(), count.end(), 0);
                        for (int f = t0[j]; f < t0[j + 1]; f++) count[std::min(mx[f] - mn[f], kMaxSpread + 1)]++;
                        auto &h = hist[(size_t)g * S + j];
                        for (int d = 0; d <= kMaxSpread + 1; d++)
                            if (count[d]) {
                                h.emplace_back(d, count[d]);
                                spread_max = std::max(spread_max, d);
                            }
                    }
                }
            }
            if (spread_max > kMaxSpread) continue;  // no tile height fits
            for (const Geo &geo : geos) {
                // window height: the tile, the footprint and the largest spread
                const int bh = geo.th + 4 + spread_max;
                if (bh > 256) continue;
                int ns = 0;
                for (int c = t.forced_stages ? t.forced_stages : mf::kFacMaxStages; c >= 2; c--) {
                    if (mf::fac_smem_bytes(geo.tw, bh, c, kt, npl) <= (size_t)mf::kSmemBudget &&
                        (size_t)c * mf::fac_stage_floats(geo.tw, bh) * 4 >= (size_t)geo.th * geo.tw * 8) {
                        ns = c;
                        break;
                    }
                    if (t.forced_stages) break;
                }
                if (ns == 0) continue;
                const int warps = kt * (geo.th / 32) * (geo.tw / 32);
                const int threads = 32 * ((warps + 3) / 4 * 4);
                const double hc = mf::fac_hcols(geo.tw), rp = mf::fac_rpitch(geo.tw);
                const double ni = hc / mf::kFacItem;
                const double sub = (geo.th / 32) * (geo.tw / 32);
                // the column-pass warps are dealt to the SM's four schedulers; the
                // busiest sets the pace
                const double skew = (double)((warps + 3) / 4 * 4) / warps;
                double cyc = 0.0;
                for (int g = 0; g < G; g++) {
                    const double n = (double)groups[g].size();
                    for (int j = 0; j < S; j++) {
                        // tile rows cover the members' spread at the segment start
                        // too (nominal 1024-row image)
                        const double extra = 1.0 + seg_qy[((size_t)g * S + j) * 2 + 1] / 1024.0;
                        double seg = 0.0;
                        for (const auto &dc : hist[(size_t)g * S + j]) {
                            const double nr = geo.th + 4 + dc.first;
                            // the row pass overlaps the column passes of other warps:
                            // weighted by what measurements of the two fitted
                            const double fma = (n * geo.th * geo.tw * 5.0 * skew + 0.5 * nr * hc * 5.0) / 128.0;
                            const double sm = (n * sub * 40.0 * 128.0 + 0.5 * nr * ni * 160.0 + bh * rp * 4.0) / 128.0;
                            const double rounds = std::ceil(2.0 * nr * ni / threads);
                            seg += dc.second * (std::max(fma, sm) / 0.8 + 200.0 + 300.0 * (rounds - 1.0));
                        }
                        // prologue (first windows in flight) and epilogue of each CTA
                        cyc += (seg + 20000.0) * extra;
                    }
                }
                // plane: K x 4 bytes written per segment and read by the next (at
                // ~6.7 TB/s, 152 SMs at 2.07 GHz: 0.38 K cycles per pixel each),
                // the extra CTA prologues and epilogues and the launch tail per
                // segment (measured: about three times the traffic term)
                const double cost = cyc / ((double)geo.th * geo.tw) + 1.2 * S * K;
                if (have && cost >= out.cost) continue;
                mf::Plan p;
                p.kernel = 2;
                p.f_kt = kt;
                p.f_th = geo.th;
                p.f_tw = geo.tw;
                p.f_seg = S;
                p.seg_t0 = t0;
                p.seg_qy = seg_qy;
                const size_t gmax = seg_ref.size() / ((size_t)G * S);
                p.seg_ref.assign((size_t)G * S * kt, INT32_MIN);
                for (size_t gj = 0; gj < (size_t)G * S; gj++)
                    for (size_t i = 0; i < gmax; i++) p.seg_ref[gj * kt + i] = seg_ref[gj * gmax + i];
                p.f_ns = ns;
                p.f_bh = bh;
                p.f_planes = npl;
                p.cost = cost;
                p.G = G;
                p.members.assign((size_t)G * kt, -1);
                for (int g = 0; g < G; g++)
                    for (size_t i = 0; i < groups[g].size(); i++) p.members[(size_t)g * kt + i] = groups[g][i];
                out = std::move(p);
                have = true;
            }
        }
    }
    if (!have) return false;
    int mxs = 0;
    for (size_t i = 0; i < t.shifts.size(); i++) mxs = std::max(mxs, std::abs(t.shifts[i]));
    out.max_abs_shift = mxs;
    // single centre tap on both axes for every (trajectory, frame): the
    // passes need only the centre tap
    bool single = true;
    for (size_t i = 0; i < t.fx.size() && single; i += 5)
        for (int a = 0; a < 5; a++)
            if (t.fx[i + a] != (a == 2 ? 1.0 : 0.0) || t.fy[i + a] != (a == 2 ? 1.0 : 0.0)) single = false;
    out.f_taps = single ? 1 : 5;
    return true;
}

// A table's device arrays share one block, allocated and freed in stream
// order (on a private non-blocking stream) where the device has memory
// pools: unlike cudaFree, freeing it does not wait for the whole device, so
// a finished search's table can be dropped while other streams still run.
struct DeviceBlock {
    struct Part {
        void **dst;
        const void *src;
        size_t bytes, off;
    };
    std::vector<Part> parts;
    size_t total = 0;
    template <class T>
    void add(T **dst, const T *src, size_t n) {
        *dst = nullptr;
        if (n == 0) return;
        total = (total + 255) / 256 * 256;
        parts.push_back({(void **)dst, src, n * sizeof(T), total});
        total += n * sizeof(T);
    }
    mf_status upload(void **block, bool *pooled) {
        *block = nullptr;
        *pooled = false;
        if (total == 0) return MF_OK;
        int dev = 0, pools = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, dev);
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return fail(MF_ECUDA, "cudaStreamCreateWithFlags: %s", cudaGetErrorString(e));
        e = pools ? cudaMallocAsync(block, total, st) : cudaMalloc(block, total);
        if (e != cudaSuccess) {
            *block = nullptr;
            cudaStreamDestroy(st);
            return fail(MF_ENOMEM, "device allocation of %zu bytes: %s", total, cudaGetErrorString(e));
        }
        *pooled = pools != 0;
        for (const Part &q : parts) {
            *q.dst = (unsigned char *)*block + q.off;
            if (e == cudaSuccess) e = cudaMemcpyAsync(*q.dst, q.src, q.bytes, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
        if (e != cudaSuccess) return fail(MF_ECUDA, "table upload: %s", cudaGetErrorString(e));
        return MF_OK;
    }
};

struct HostLayouts {
    std::vector<mf::FrameHdr> hdr;
    std::vector<unsigned char> blocks;
    std::vector<int32_t> segs;  // factored: [G][S][4]
    std::vector<mf::RunRec> runs;
    std::vector<mf::DenBox> boxes;
    std::vector<int32_t> run_off;
    std::vector<float> wts;
};

size_t layout_bytes(const mf_prf_table *t, const HostLayouts &h) {
    return h.blocks.size() + h.hdr.size() * sizeof(mf::FrameHdr) + t->plan.members.size() * sizeof(int32_t) +
           h.segs.size() * sizeof(int32_t) + t->plan.seg_ref.size() * sizeof(int32_t) +
           h.runs.size() * sizeof(mf::RunRec) + h.boxes.size() * sizeof(mf::DenBox) +
           h.run_off.size() * sizeof(int32_t) + h.wts.size() * sizeof(float) + t->taps.size() * sizeof(double) +
           t->shifts.size() * sizeof(int32_t);
}

void general_layouts(mf_prf_table *t, HostLayouts &out);
bool fac_layouts(mf_prf_table *t, HostLayouts &out);
void denominator_layouts(mf_prf_table *t, HostLayouts &out);

// Plan the groups and build the layouts the kernels read: frame headers and
// blocks (numerator), constant-shift runs (denominator).  The factored
// numerator is used whenever the table is separable and a layout fits,
// unless the options ask for the general one.
mf_status host_layouts(mf_prf_table *t, HostLayouts &out) {
    bool factored = false;
    if (t->forced_kernel != 1) {
        mf::Plan fp;
        factored = plan_factored(*t, fp);
        if (factored) t->plan = std::move(fp);
        else if (t->forced_kernel >= 2)
            return fail(t->fx.empty() ? MF_EINVAL : MF_EUNSUPPORTED,
                        t->fx.empty() ? "the factored numerator needs a separable (Gaussian PRF) table"
                                      : "no factored layout holds these trajectories' frame windows");
    }
    if (factored) {
        if (!fac_layouts(t, out))
            return fail(MF_EUNSUPPORTED, "a frame needs more phase planes than the layout holds");
    } else {
        mf_status s = plan_groups(*t);
        if (s != MF_OK) return s;
        general_layouts(t, out);
    }
    denominator_layouts(t, out);
    return MF_OK;
}

// Frame headers and blocks of the general numerator.
void general_layouts(mf_prf_table *t, HostLayouts &out) {
    const int T = t->T;
    const mf::Plan &p = t->plan;
    const int kt = p.kt();
    std::vector<mf::FrameHdr> hdr((size_t)p.G * T);
    for (int g = 0; g < p.G; g++) {
        for (int f = 0; f < T; f++) {
            int64_t mnx = INT64_MAX, mny = INT64_MAX, mxy = INT64_MIN;
            for (int w = 0; w < kt; w++) {
                const int k = p.members[(size_t)g * kt + w];
                if (k < 0) continue;
                mnx = std::min<int64_t>(mnx, t->shifts[((size_t)k * T + f) * 2 + 0]);
                mny = std::min<int64_t>(mny, t->shifts[((size_t)k * T + f) * 2 + 1]);
                mxy = std::max<int64_t>(mxy, t->shifts[((size_t)k * T + f) * 2 + 1]);
            }
            mf::FrameHdr &h = hdr[(size_t)g * T + f];
            h.roy = (int32_t)(mny - 2);
            h.rox = (int32_t)(4 * floor_div(mnx - 2, 4));
            h.nrows = (int32_t)round_up(mxy - mny + p.tile_h() + 4, mf::kLoadRows);
            h.pad = 0;
        }
    }
    const size_t bb = mf::frame_block_bytes(kt);
    std::vector<unsigned char> blocks((size_t)p.G * T * bb, 0);
    for (int g = 0; g < p.G; g++) {
        for (int f = 0; f < T; f++) {
            unsigned char *b = blocks.data() + ((size_t)g * T + f) * bb;
            mf::FrameHdr next{0, 0, 0, 0};
            if (f + mf::kStages < T) next = hdr[(size_t)g * T + f + mf::kStages];
            std::memcpy(b, &next, sizeof next);
            const mf::FrameHdr &h = hdr[(size_t)g * T + f];
            for (int w = 0; w < kt; w++) {
                const int k = p.members[(size_t)g * kt + w];
                mf::SlotRec r;
                std::memset(&r, 0, sizeof r);
                r.k = k;
                if (k >= 0) {
                    const size_t ktf = (size_t)k * T + f;
                    for (int i = 0; i < 25; i++) r.taps[i] = (float)t->taps[ktf * 25 + i];
                    r.offy = t->shifts[ktf * 2 + 1] - 2 - h.roy;
                    r.offx = t->shifts[ktf * 2 + 0] - 2 - h.rox;
                }
                std::memcpy(b + sizeof(mf::FrameHdr) + (size_t)w * sizeof(mf::SlotRec), &r, sizeof r);
            }
        }
    }
    out.hdr = std::move(hdr);
    out.blocks = std::move(blocks);
}

// Frame headers and blocks of the factored numerator: per (group, frame) the
// window origin (rows from min s_y - 2, columns from s_x - 2 rounded down to
// a multiple of 4 for the TMA box), the row-pass rows, u_x, and per slot u_y
// and the slot's row offset in the row-pass buffer.
bool fac_layouts(mf_prf_table *t, HostLayouts &out) {
    const int T = t->T;
    const mf::Plan &p = t->plan;
    const int kt = p.f_kt, S = p.f_seg;
    std::vector<int> seg_of(T);
    for (int j = 0; j < S; j++)
        for (int f = p.seg_t0[j]; f < p.seg_t0[j + 1]; f++) seg_of[f] = j;
    // s_y of slot w at frame f relative to its s_y at the segment's first frame
    auto rel = [&](int g, int w, int f) {
        const int k = p.members[(size_t)g * kt + w];
        return t->shifts[((size_t)k * T + f) * 2 + 1] - p.seg_ref[((size_t)g * S + seg_of[f]) * kt + w];
    };
    std::vector<mf::FrameHdr> hdr((size_t)p.G * T);
    for (int g = 0; g < p.G; g++) {
        const int k0 = p.members[(size_t)g * kt];
        for (int f = 0; f < T; f++) {
            int mny = INT32_MAX, mxy = INT32_MIN;
            for (int w = 0; w < kt; w++) {
                if (p.members[(size_t)g * kt + w] < 0) continue;
                mny = std::min(mny, rel(g, w, f));
                mxy = std::max(mxy, rel(g, w, f));
            }
            const int64_t sx = t->shifts[((size_t)k0 * T + f) * 2 + 0];
            mf::FrameHdr &h = hdr[(size_t)g * T + f];
            h.roy = mny - 2;
            h.rox = (int32_t)(4 * floor_div(sx - 2, 4));
            h.nrows = p.f_th + 4 + (mxy - mny);
            h.pad = (int32_t)(sx - 2 - h.rox);  // column phase
        }
    }
    const int npl = p.f_planes;
    const size_t bb = mf::fac_block_bytes(kt, npl);
    std::vector<unsigned char> blocks((size_t)p.G * T * bb, 0);
    for (int g = 0; g < p.G; g++) {
        const int k0 = p.members[(size_t)g * kt];
        for (int f = 0; f < T; f++) {
            unsigned char *b = blocks.data() + ((size_t)g * T + f) * bb;
            const mf::FrameHdr &h = hdr[(size_t)g * T + f];
            mf::FacHdr fh;
            std::memset(&fh, 0, sizeof fh);
            const int fn = f + p.f_ns;  // frame loaded next into this stage, if in the same segment
            if (fn < p.seg_t0[seg_of[f] + 1]) {
                fh.next_roy = hdr[(size_t)g * T + fn].roy;
                fh.next_rox = hdr[(size_t)g * T + fn].rox;
            }
            fh.cofs = h.pad;
            fh.cofs8 = (int32_t)(t->shifts[((size_t)k0 * T + f) * 2 + 0] - 2 - 8 * floor_div(
                                     t->shifts[((size_t)k0 * T + f) * 2 + 0] - 2, 8));
            fh.nrows = h.nrows;
            fh.inv_nrows = 1.0f / (float)h.nrows;
            for (int a = 0; a < 5; a++) fh.ux[a] = (float)t->fx[((size_t)k0 * T + f) * 5 + a];
            // phase planes: the distinct column-pass taps among the slots
            // (one per rounded y-phase present), in order of first use
            std::vector<mf::FacPlane> planes;
            for (int w = 0; w < kt; w++) {
                const int k = p.members[(size_t)g * kt + w];
                mf::FacSlot fs;
                std::memset(&fs, 0, sizeof fs);
                if (k >= 0) {
                    const size_t ktf = (size_t)k * T + f;
                    for (int c = 0; c < 5; c++) fs.uy[c] = (float)t->fy[ktf * 5 + c];
                    fs.oy = rel(g, w, f) - 2 - h.roy;
                    if (npl > 0) {
                        size_t j = 0;
                        while (j < planes.size() && std::memcmp(planes[j].uy, fs.uy, sizeof fs.uy) != 0) j++;
                        if (j == planes.size()) {
                            mf::FacPlane pl;
                            std::memset(&pl, 0, sizeof pl);
                            std::memcpy(pl.uy, fs.uy, sizeof pl.uy);
                            planes.push_back(pl);
                        }
                        fs.plane = (int32_t)j;
                    }
                }
                std::memcpy(b + sizeof fh + (size_t)w * sizeof fs, &fs, sizeof fs);
            }
            if (npl > 0) {
                // the bank rounds every phase to one of Q + 1 values, so a
                // frame never needs more than the planner allowed
                if ((int)planes.size() > npl) return false;
                fh.pad = (int32_t)planes.size();
                std::memcpy(b + sizeof fh + (size_t)kt * sizeof(mf::FacSlot), planes.data(),
                            planes.size() * sizeof(mf::FacPlane));
            }
            std::memcpy(b, &fh, sizeof fh);
        }
    }
    // per (group, segment): first frame, end frame, min s_y, spread
    std::vector<int32_t> segs((size_t)p.G * S * 4);
    for (int g = 0; g < p.G; g++)
        for (int j = 0; j < S; j++) {
            int32_t *q = &segs[((size_t)g * S + j) * 4];
            q[0] = p.seg_t0[j];
            q[1] = p.seg_t0[j + 1];
            q[2] = p.seg_qy[((size_t)g * S + j) * 2 + 0];
            q[3] = p.seg_qy[((size_t)g * S + j) * 2 + 1];
        }
    out.hdr = std::move(hdr);
    out.blocks = std::move(blocks);
    out.segs = std::move(segs);
    return true;
}

// Denominator layout: constant-shift runs of the collapsed kernels.
void denominator_layouts(mf_prf_table *t, HostLayouts &out) {
    const int K = t->K, T = t->T;
    // Denominator: lambda does not depend on t, so D_k(p) = sum_u G_k(u)
    // lambda(p + u) with the collapsed kernel G_k(u) = sum over (t, a, b)
    // with s_{k,t} + (a, b) = u of W_{k,t}(a, b)^2, summed here in FP64.
    // Each row of G_k's support becomes one run of weights starting at a
    // column that is a multiple of 4 and padded to whole chunks of 4.
    std::vector<mf::RunRec> runs;
    std::vector<int32_t> run_off(K + 1, 0);
    std::vector<float> wts;
    int64_t nnz_total = 0;
    std::vector<double> dense;
    std::vector<char> hit;
    for (int k = 0; k < K; k++) {
        run_off[k] = (int32_t)runs.size();
        // bounding box of G_k's support
        int32_t x_lo = INT32_MAX, x_hi = INT32_MIN, y_lo = INT32_MAX, y_hi = INT32_MIN;
        for (int f = 0; f < T; f++) {
            const size_t kt_ = (size_t)k * T + f;
            x_lo = std::min(x_lo, t->shifts[kt_ * 2 + 0] - 2);
            x_hi = std::max(x_hi, t->shifts[kt_ * 2 + 0] + 2);
            y_lo = std::min(y_lo, t->shifts[kt_ * 2 + 1] - 2);
            y_hi = std::max(y_hi, t->shifts[kt_ * 2 + 1] + 2);
        }
        const int64_t bw = (int64_t)x_hi - x_lo + 1, bh = (int64_t)y_hi - y_lo + 1;
        // one run per row of the support: from the first column some frame's
        // footprint reached to the last, starting at a multiple of 4
        auto emit = [&](int32_t row, int32_t xfirst, int32_t xlast, const double *val, const int32_t *col,
                        size_t n) {
            const int32_t x0 = (int32_t)(4 * floor_div(xfirst, 4));
            const int32_t nch = (int32_t)((xlast - x0 + 1 + 3) / 4);
            while (wts.size() % 4) wts.push_back(0.f);
            mf::RunRec r;
            r.dy = row;
            r.x0 = x0;
            r.nch = nch;
            r.woff = (int32_t)wts.size();
            const size_t base = wts.size();
            wts.resize(base + (size_t)nch * 4, 0.f);
            for (size_t q = 0; q < n; q++) wts[base + (col ? col[q] : xfirst + (int32_t)q) - x0] = (float)val[q];
            runs.push_back(r);
        };
        if (bw * bh <= (int64_t)100 * T + 4096) {
            dense.assign((size_t)(bw * bh), 0.0);
            hit.assign((size_t)(bw * bh), 0);
            for (int f = 0; f < T; f++) {
                const size_t kt_ = (size_t)k * T + f;
                const int32_t sx = t->shifts[kt_ * 2 + 0], sy = t->shifts[kt_ * 2 + 1];
                for (int b = 0; b < 5; b++)
                    for (int a = 0; a < 5; a++) {
                        const double w = t->taps[kt_ * 25 + b * 5 + a];
                        const size_t i = (size_t)((sy + b - 2 - y_lo) * bw + (sx + a - 2 - x_lo));
                        dense[i] += w * w;
                        hit[i] = 1;
                    }
            }
            for (int64_t r = 0; r < bh; r++) {
                int64_t c0 = -1, c1 = -1;
                for (int64_t c = 0; c < bw; c++)
                    if (hit[(size_t)(r * bw + c)]) {
                        if (c0 < 0) c0 = c;
                        c1 = c;
                    }
                if (c0 < 0) continue;
                nnz_total += c1 - c0 + 1;
                emit((int32_t)(r + y_lo), (int32_t)(c0 + x_lo), (int32_t)(c1 + x_lo), &dense[(size_t)(r * bw + c0)],
                     nullptr, (size_t)(c1 - c0 + 1));
            }
        } else {
            std::map<std::pair<int32_t, int32_t>, double> sparse;  // (row, column) -> weight
            for (int f = 0; f < T; f++) {
                const size_t kt_ = (size_t)k * T + f;
                const int32_t sx = t->shifts[kt_ * 2 + 0], sy = t->shifts[kt_ * 2 + 1];
                for (int b = 0; b < 5; b++)
                    for (int a = 0; a < 5; a++) {
                        const double w = t->taps[kt_ * 25 + b * 5 + a];
                        sparse[{sy + b - 2, sx + a - 2}] += w * w;
                    }
            }
            nnz_total += (int64_t)sparse.size();
            std::vector<double> val;
            std::vector<int32_t> col;
            auto it = sparse.begin();
            while (it != sparse.end()) {
                const int32_t row = it->first.first;
                val.clear();
                col.clear();
                auto jt = it;
                for (; jt != sparse.end() && jt->first.first == row; ++jt) {
                    val.push_back(jt->second);
                    col.push_back(jt->first.second);
                }
                emit(row, col.front(), col.back(), val.data(), col.data(), val.size());
                it = jt;
            }
        }
    }
    run_off[K] = (int32_t)runs.size();
    t->n_seg = (int)runs.size();
    t->g_nnz = nnz_total;
    // bounding boxes for the staged denominator, and its tile height: the
    // tallest of 32, 16, 8 rows whose largest lambda box fits shared memory
    std::vector<mf::DenBox> boxes(K);
    int rows_max = 1, cols_max = 4, nw_max = 4, nr_max = 1;
    for (int k = 0; k < K; k++) {
        mf::DenBox b{};
        const int r0 = run_off[k], r1 = run_off[k + 1];
        if (r1 > r0) {
            int dy0 = INT32_MAX, dy1 = INT32_MIN, x0 = INT32_MAX, x1 = INT32_MIN;
            for (int r = r0; r < r1; r++) {
                dy0 = std::min(dy0, runs[r].dy);
                dy1 = std::max(dy1, runs[r].dy);
                x0 = std::min(x0, runs[r].x0);
                x1 = std::max(x1, runs[r].x0 + 4 * runs[r].nch);
            }
            b.dy0 = dy0;
            b.rows = dy1 - dy0 + 1;
            b.x0 = x0;
            b.cols = x1 - x0;
            b.w0 = runs[r0].woff;
            b.nw = runs[r1 - 1].woff + 4 * runs[r1 - 1].nch - b.w0;
        } else {
            b.rows = 1;
            b.cols = 4;
        }
        rows_max = std::max(rows_max, b.rows);
        cols_max = std::max(cols_max, b.cols);
        nw_max = std::max(nw_max, b.nw);
        nr_max = std::max(nr_max, run_off[k + 1] - run_off[k]);
        boxes[k] = b;
    }
    t->den_th = 0;
    t->den_smem = 0;
    for (int th : {32, 16, 8}) {
        const size_t sm = mf::den_box_smem(th, rows_max, cols_max, nw_max, nr_max);
        if (sm <= (size_t)mf::kSmemBudget) {
            t->den_th = th;
            t->den_smem = sm;
            break;
        }
    }
    out.boxes = std::move(boxes);
    out.runs = std::move(runs);
    out.run_off = std::move(run_off);
    out.wts = std::move(wts);
}

mf_status finish_table(mf_prf_table *t) {
    HostLayouts h;
    mf_status s = host_layouts(t, h);
    if (s != MF_OK) return s;
    DeviceBlock blk;
    blk.add(&t->d_blocks, h.blocks.data(), h.blocks.size());
    blk.add(&t->d_hdr, h.hdr.data(), h.hdr.size());
    blk.add(&t->d_members, t->plan.members.data(), t->plan.members.size());
    if (t->plan.kernel == 2) {
        blk.add(&t->d_segs, h.segs.data(), h.segs.size());
        blk.add(&t->d_refs, t->plan.seg_ref.data(), t->plan.seg_ref.size());
    }
    blk.add(&t->d_runs, h.runs.data(), h.runs.size());
    blk.add(&t->d_boxes, h.boxes.data(), h.boxes.size());
    blk.add(&t->d_run_off, h.run_off.data(), h.run_off.size());
    blk.add(&t->d_wts, h.wts.data(), h.wts.size());
    blk.add(&t->d_taps64, t->taps.data(), t->taps.size());
    blk.add(&t->d_shifts, t->shifts.data(), t->shifts.size());
    if ((s = blk.upload(&t->d_mem, &t->d_mem_pooled)) != MF_OK) return s;
    t->device_bytes = layout_bytes(t, h);
    return MF_OK;
}

void fill_info(const mf_prf_table *t, mf_table_info *info) {
    std::memset(info, 0, sizeof *info);
    info->K = t->K;
    info->T = t->T;
    info->groups = t->plan.G;
    info->warps_per_group = t->plan.kt();
    info->tile_h = t->plan.tile_h();
    info->tile_w = t->plan.tile_w();
    const bool fac = t->plan.kernel == 2;
    info->window_pitch = fac ? mf::fac_rpitch(t->plan.f_tw) : t->plan.S;
    info->window_rows = fac ? t->plan.f_bh : t->plan.BH;
    info->segments = t->n_seg;
    info->g_nnz = t->g_nnz;
    info->max_abs_shift = t->plan.max_abs_shift;
    info->smem_bytes = (int64_t)t->plan.smem();
    info->cost = t->plan.cost;
    info->vec = fac ? 1 : t->plan.vec;
    info->lockstep = fac ? 1 : t->plan.lockstep;
    info->kernel = t->plan.kernel;
    info->stages = fac ? t->plan.f_ns : mf::kStages;
    info->time_segments = fac ? t->plan.f_seg : 1;
    info->taps = fac ? t->plan.f_taps : 5;
    info->den_tile_h = t->den_th;
    info->phase_planes = fac ? t->plan.f_planes : 0;
    info->device_bytes = (int64_t)t->device_bytes;
}

void free_device(mf_prf_table *t) {
    if (t->d_mem) {
        cudaStream_t st = nullptr;
        if (t->d_mem_pooled && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) {
            cudaFreeAsync(t->d_mem, st);
            cudaStreamDestroy(st);
        } else {
            cudaFree(t->d_mem);
        }
    }
    t->d_mem = nullptr;
    t->d_blocks = nullptr;
    t->d_hdr = nullptr;
    t->d_members = nullptr;
    t->d_segs = nullptr;
    t->d_refs = nullptr;
    t->d_runs = nullptr;
    t->d_boxes = nullptr;
    t->d_run_off = nullptr;
    t->d_wts = nullptr;
    t->d_taps64 = nullptr;
    t->d_shifts = nullptr;
}

mf_status create_common(mf_prf_table *t, mf_prf_table **out) {
    if (cudaGetDevice(&t->device) != cudaSuccess) {
        delete t;
        return fail(MF_ECUDA, "no current CUDA device");
    }
    mf_status s = finish_table(t);
    if (s != MF_OK) {
        const std::string msg = g_err;
        free_device(t);
        delete t;
        g_err = msg;
        return s;
    }
    *out = t;
    return ok();
}

size_t elem_size(int dtype) { return dtype == MF_F32 ? 4 : 2; }

mf_status check_stack(const mf_stack *st) {
    if (!st) return fail(MF_EINVAL, "stack is NULL");
    if (st->dtype != MF_F32 && st->dtype != MF_BF16 && st->dtype != MF_F16)
        return fail(MF_EINVAL, "unknown dtype %d", st->dtype);
    if (st->T < 1 || st->H < 0 || st->W < 0) return fail(MF_EINVAL, "bad stack shape T=%lld H=%lld W=%lld",
                                                         (long long)st->T, (long long)st->H, (long long)st->W);
    if (st->H > (1 << 20) || st->W > (1 << 20) || st->T > (1 << 20))
        return fail(MF_EINVAL, "stack dimension above 2^20");
    if (st->H * st->W == 0) return MF_OK;
    if (!st->data) return fail(MF_EINVAL, "stack data is NULL");
    if (st->row_stride < st->W) return fail(MF_EINVAL, "row_stride %lld < W %lld", (long long)st->row_stride,
                                            (long long)st->W);
    if (st->T > 1 && st->frame_stride < st->H * st->row_stride)
        return fail(MF_EINVAL, "frame_stride %lld < H * row_stride", (long long)st->frame_stride);
    if ((uintptr_t)st->data % elem_size(st->dtype) != 0) return fail(MF_EINVAL, "stack data misaligned");
    return MF_OK;
}

}  // namespace

namespace mf {

mf_status set_error(mf_status s, const char *msg) { return fail(s, "%s", msg); }

long long fac_ctas(const mf_prf_table &tab, int64_t H, int64_t W, int seg) {
    const Plan &p = tab.plan;
    if (seg < 0 || seg >= p.f_seg) return 0;
    const long long tiles_x = (W + p.f_tw - 1) / p.f_tw;
    int spread = 0;
    for (int g = 0; g < p.G; g++) spread = std::max(spread, p.seg_qy[((size_t)g * p.f_seg + seg) * 2 + 1]);
    return (H + spread + p.f_th - 1) / p.f_th * tiles_x * p.G;
}

WorkspaceLayout search_layout(int64_t T, int64_t H, int64_t W, int32_t dtype, const mf_prf_table *tab) {
    WorkspaceLayout L;
    // zero border wide enough for every denominator read: shifts up to
    // max_abs_shift, footprint 2, run padding and the last partial row block
    L.pad = round_up((int64_t)tab->plan.max_abs_shift + 2 + 16, 4);
    L.lam_w = round_up(round_up(W, kDenCols) + 2 * L.pad + 32, 4);
    L.lam_h = round_up(H, 8) + 2 * L.pad;
    // a bf16 / fp16 stack searched by the factored numerator keeps its
    // weighted stack in its own 16-bit type (rows a multiple of 16 bytes)
    L.ybytes = (dtype != MF_F32 && tab->plan.kernel == 2 && tab->plan.f_planes == 0) ? 2 : 4;
    L.y_pitch = round_up(W, L.ybytes == 2 ? 8 : 4);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (size_t)round_up((int64_t)(off + bytes), 256);
        return o;
    };
    L.status_off = take(16);  // offset 0 (mf_search_status reads it there); bytes 8..11: largest lambda
    L.lam_off = take((size_t)L.lam_w * L.lam_h * sizeof(float));
    L.y_off = take((size_t)T * H * L.y_pitch * L.ybytes);
    L.beta_off = take((size_t)T * sizeof(float));
    L.isd_off = take((size_t)tab->K * H * W * sizeof(float));
    L.keys_off = take((size_t)H * W * sizeof(unsigned long long));
    L.planes_off = take(tab->plan.kernel == 2 ? (size_t)tab->K * H * W * sizeof(float) : 0);
    L.total = off;
    return L;
}

}  // namespace mf

extern "C" {

static mf_status build_gauss_host(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                                  int32_t T, mf_prf_table **out_t, const mf_frames *frames = nullptr) {
    if (!prf || !vx || !vy) return fail(MF_EINVAL, "NULL argument");
    if (K < 1 || T < 1) return fail(MF_EINVAL, "K=%d and T=%d must be >= 1", K, T);
    if (T > (1 << 20) || K > (1 << 22)) return fail(MF_EINVAL, "K or T too large");
    if (prf->kind < 0 || prf->kind > 2) return fail(MF_EINVAL, "unknown PRF kind %d", prf->kind);
    if (!(prf->sigma_px > 0.0) || !std::isfinite(prf->sigma_px))
        return fail(MF_EINVAL, "sigma_px must be finite and > 0");
    if (prf->phase_steps < 0 || prf->phase_steps > 4096)
        return fail(MF_EINVAL, "phase_steps=%d out of range 0..4096", prf->phase_steps);
    const double Q = (double)prf->phase_steps;
    const double *times = frames ? frames->times : nullptr;
    const double *jitter = frames ? frames->jitter : nullptr;
    // the frame model: time and (x, y) pointing offset of frame f
    auto tau = [&](int f) { return times ? times[f] : (double)f; };
    auto jit = [&](int f, int axis) { return jitter ? jitter[(size_t)f * 2 + axis] : 0.0; };
    double tmax = 0.0, jmax = 0.0;
    for (int f = 0; f < T; f++) {
        if (!std::isfinite(tau(f)) || !std::isfinite(jit(f, 0)) || !std::isfinite(jit(f, 1)))
            return fail(MF_EINVAL, "frame %d: time or jitter not finite", f);
        tmax = std::max(tmax, std::fabs(tau(f)));
        jmax = std::max({jmax, std::fabs(jit(f, 0)), std::fabs(jit(f, 1))});
    }
    for (int k = 0; k < K; k++) {
        if (!std::isfinite(vx[k]) || !std::isfinite(vy[k])) return fail(MF_EINVAL, "velocity %d not finite", k);
        if (std::fabs(vx[k]) * std::max(tmax, (double)T) + jmax > (1 << 20) ||
            std::fabs(vy[k]) * std::max(tmax, (double)T) + jmax > (1 << 20))
            return fail(MF_EINVAL, "velocity %d moves more than 2^20 pixels", k);
    }
    auto *t = new mf_prf_table;
    t->K = K;
    t->T = T;
    t->phase_steps = prf->phase_steps;
    t->shifts.resize((size_t)K * T * 2);
    t->taps.resize((size_t)K * T * 25);
    t->fx.resize((size_t)K * T * 5);
    t->fy.resize((size_t)K * T * 5);
    t->vx.assign(vx, vx + K);
    t->vy.assign(vy, vy + K);
    // the x profile depends on (v_x, frame) only and the y profile on (v_y,
    // frame) -- the jitter is common to all trajectories: evaluate each once
    // per distinct velocity component
    auto profiles = [&](const double *v, int axis, std::vector<int> &idx, std::vector<double> &prof) {
        std::map<double, int> distinct;
        idx.resize(K);
        for (int k = 0; k < K; k++) idx[k] = distinct.emplace(v[k], (int)distinct.size()).first->second;
        prof.resize(distinct.size() * (size_t)T * 5);
        for (const auto &d : distinct)
            for (int f = 0; f < T; f++) {
                const double c = d.first * tau(f) + jit(f, axis);
                double ph = c - std::floor(c + 0.5);
                if (Q > 0.0) ph = std::floor(ph * Q + 0.5) / Q;  // the phase-quantised bank
                axis_profile(prf->kind, prf->sigma_px, ph, &prof[((size_t)d.second * T + f) * 5]);
            }
    };
    std::vector<int> ix, iy;
    std::vector<double> px, py;
    profiles(vx, 0, ix, px);
    profiles(vy, 1, iy, py);
    for (int k = 0; k < K; k++) {
        for (int f = 0; f < T; f++) {
            // position in frame f, base pixel floor(c + 1/2), phase c - s
            const double cx = vx[k] * tau(f) + jit(f, 0);
            const double cy = vy[k] * tau(f) + jit(f, 1);
            const size_t kt = (size_t)k * T + f;
            t->shifts[kt * 2 + 0] = (int32_t)std::floor(cx + 0.5);
            t->shifts[kt * 2 + 1] = (int32_t)std::floor(cy + 0.5);
            footprint_from_axes(&px[((size_t)ix[k] * T + f) * 5], &py[((size_t)iy[k] * T + f) * 5], &t->taps[kt * 25],
                                &t->fx[kt * 5], &t->fy[kt * 5]);
        }
    }
    *out_t = t;
    return MF_OK;
}

static mf_status apply_opts(mf_prf_table *t, const mf_plan_opts *opts) {
    if (!opts) return MF_OK;
    if (opts->shape < -1 || opts->shape >= mf::kNumShapes) {
        delete t;
        return fail(MF_EINVAL, "shape %d out of range", opts->shape);
    }
    if (opts->vec != 0 && opts->vec != 1 && opts->vec != 2 && opts->vec != 4) {
        delete t;
        return fail(MF_EINVAL, "vec %d must be 0, 1, 2 or 4", opts->vec);
    }
    if (opts->kernel < 0 || opts->kernel > 3) {
        delete t;
        return fail(MF_EINVAL, "kernel %d must be 0, 1, 2 or 3", opts->kernel);
    }
    if (opts->kernel == 3 && t->phase_steps == 0) {
        delete t;
        return fail(MF_EINVAL, "kernel 3 (phase planes) needs a phase-quantised bank (phase_steps > 0)");
    }
    if (opts->group < 0 || opts->group > mf::kFacMaxWarps || opts->tile_h < 0 || opts->tile_h % 32 != 0 ||
        (opts->tile_w != 0 && opts->tile_w != 32 && opts->tile_w != 64) || opts->stages < 0 ||
        opts->stages == 1 || opts->stages > mf::kFacMaxStages) {
        delete t;
        return fail(MF_EINVAL, "factored layout group=%d tile_h=%d tile_w=%d stages=%d out of range", opts->group,
                    opts->tile_h, opts->tile_w, opts->stages);
    }
    t->forced_shape = opts->shape;
    t->forced_vec = opts->vec;
    t->forced_lockstep = opts->lockstep;
    t->forced_kernel = opts->kernel;
    if (opts->kernel == 0 && opts->shape >= 0) t->forced_kernel = 1;
    t->forced_group = opts->group;
    t->forced_th = opts->tile_h;
    t->forced_tw = opts->tile_w;
    t->forced_stages = opts->stages;
    if (opts->segments < 0 || opts->segments > mf::kFacMaxSegments) {
        delete t;
        return fail(MF_EINVAL, "segments=%d out of range 0..%d", opts->segments, mf::kFacMaxSegments);
    }
    t->forced_segments = opts->segments;
    return MF_OK;
}

mf_status mf_prf_table_create_ex(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                                 int32_t T, const mf_plan_opts *opts, mf_prf_table **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    mf_prf_table *t = nullptr;
    mf_status s = build_gauss_host(prf, vx, vy, K, T, &t);
    if (s != MF_OK) return s;
    if ((s = apply_opts(t, opts)) != MF_OK) return s;
    return create_common(t, out);
}

mf_status mf_prf_table_create_frames(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                                     int32_t T, const mf_frames *frames, const mf_plan_opts *opts,
                                     mf_prf_table **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    mf_prf_table *t = nullptr;
    mf_status s = build_gauss_host(prf, vx, vy, K, T, &t, frames);
    if (s != MF_OK) return s;
    if ((s = apply_opts(t, opts)) != MF_OK) return s;
    return create_common(t, out);
}

mf_status mf_prf_table_create(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                              int32_t T, mf_prf_table **out) {
    return mf_prf_table_create_ex(prf, vx, vy, K, T, nullptr, out);
}

mf_status mf_prf_plan(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K, int32_t T,
                      const mf_plan_opts *opts, mf_table_info *info) {
    return mf_prf_plan_frames(prf, vx, vy, K, T, nullptr, opts, info);
}

mf_status mf_prf_plan_frames(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K, int32_t T,
                             const mf_frames *frames, const mf_plan_opts *opts, mf_table_info *info) {
    if (!info) return fail(MF_EINVAL, "info is NULL");
    mf_prf_table *t = nullptr;
    mf_status s = build_gauss_host(prf, vx, vy, K, T, &t, frames);
    if (s != MF_OK) return s;
    if ((s = apply_opts(t, opts)) != MF_OK) return s;
    HostLayouts h;
    s = host_layouts(t, h);
    if (s == MF_OK) {
        t->device_bytes = layout_bytes(t, h);
        fill_info(t, info);
    }
    delete t;
    return s == MF_OK ? ok() : s;
}

mf_status mf_prf_bank(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K, int32_t T,
                      const mf_frames *frames, int32_t *shifts, double *taps) {
    mf_prf_table *t = nullptr;
    const mf_status s = build_gauss_host(prf, vx, vy, K, T, &t, frames);
    if (s != MF_OK) return s;
    if (shifts) std::memcpy(shifts, t->shifts.data(), t->shifts.size() * sizeof(int32_t));
    if (taps) std::memcpy(taps, t->taps.data(), t->taps.size() * sizeof(double));
    delete t;
    return ok();
}

mf_status mf_prf_table_info(const mf_prf_table *table, mf_table_info *info) {
    if (!table || !info) return fail(MF_EINVAL, "NULL argument");
    fill_info(table, info);
    return ok();
}

mf_status mf_prf_table_create_custom(const int32_t *shifts, const double *taps, int32_t K, int32_t T,
                                     mf_prf_table **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!shifts || !taps) return fail(MF_EINVAL, "NULL argument");
    if (K < 1 || T < 1) return fail(MF_EINVAL, "K=%d and T=%d must be >= 1", K, T);
    if (T > (1 << 20) || K > (1 << 22)) return fail(MF_EINVAL, "K or T too large");
    const size_t n = (size_t)K * T;
    for (size_t i = 0; i < n * 2; i++)
        if (std::abs((int64_t)shifts[i]) > (1 << 20)) return fail(MF_EINVAL, "shift beyond 2^20 pixels");
    for (size_t i = 0; i < n * 25; i++)
        if (!std::isfinite(taps[i])) return fail(MF_EINVAL, "tap %zu not finite", i);
    auto *t = new mf_prf_table;
    t->K = K;
    t->T = T;
    t->shifts.assign(shifts, shifts + n * 2);
    t->taps.assign(taps, taps + n * 25);
    return create_common(t, out);
}

void mf_prf_table_destroy(mf_prf_table *table) {
    if (!table) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != table->device) cudaSetDevice(table->device);
    free_device(table);
    if (cur != table->device) cudaSetDevice(cur);
    delete table;
}

mf_status mf_prf_table_dims(const mf_prf_table *table, int32_t *K, int32_t *T) {
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (K) *K = table->K;
    if (T) *T = table->T;
    return ok();
}

mf_status mf_prf_table_export(const mf_prf_table *table, int32_t *shifts, double *taps) {
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (shifts) std::memcpy(shifts, table->shifts.data(), table->shifts.size() * sizeof(int32_t));
    if (taps) std::memcpy(taps, table->taps.data(), table->taps.size() * sizeof(double));
    return ok();
}

mf_status mf_search_workspace_size(const mf_stack *stack, const mf_prf_table *table, size_t *bytes) {
    if (!bytes) return fail(MF_EINVAL, "bytes is NULL");
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (!stack) return fail(MF_EINVAL, "stack is NULL");
    if (stack->T < 1 || stack->H < 0 || stack->W < 0) return fail(MF_EINVAL, "bad stack shape");
    *bytes = mf::search_layout(stack->T, stack->H, stack->W, stack->dtype, table).total;
    return ok();
}

mf_status mf_search(const mf_stack *stack, const float *sigma, const uint8_t *mask, const mf_prf_table *table,
                    float *snr_max, int32_t *argmax, float *snr_all, void *workspace, size_t workspace_bytes,
                    mf_stream stream) {
    mf_status s = check_stack(stack);
    if (s != MF_OK) return s;
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (stack->T != table->T) return fail(MF_EINVAL, "stack has T=%lld, table has T=%d", (long long)stack->T,
                                          table->T);
    if (stack->H * stack->W == 0) return ok();  // nothing to search
    if (!sigma || !snr_max || !argmax) return fail(MF_EINVAL, "sigma, snr_max and argmax are required");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != table->device)
        return fail(MF_EINVAL, "table lives on device %d, current device is %d", table->device, dev);
    const mf::WorkspaceLayout L = mf::search_layout(stack->T, stack->H, stack->W, stack->dtype, table);
    if (!workspace || workspace_bytes < L.total)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", L.total, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    mf::SearchArgs a{stack, sigma, mask, table, snr_max, argmax, snr_all, (char *)workspace, L, stream};
    char err[256] = {0};
    const int rc = mf::launch_search(a, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

}  // extern "C"

// ----------------------------------------------------------- batching ---

struct mf_batch {
    struct Item {
        mf_stack stack;
        const float *sigma;
        const uint8_t *mask;
        const mf_prf_table *table;
        float *snr_max;
        int32_t *argmax;
        float *snr_all;
    };
    int device = 0;
    std::vector<Item> items;
    std::vector<mf::SearchArgs> args;
    std::vector<mf::WorkspaceLayout> layouts;
    char *ws = nullptr;
    mf::BatchDevice *dev = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture = nullptr;  // private stream the graph is captured on
    cudaEvent_t done = nullptr;      // recorded after every run, for mf_batch_poll
    bool ran = false;
    bool prepared = false;
};

namespace {

size_t batch_item_offsets(const mf_batch *b, std::vector<size_t> *offs) {
    size_t off = 0;
    for (const auto &it : b->items) {
        if (offs) offs->push_back(off);
        off += (size_t)round_up(
            (int64_t)mf::search_layout(it.stack.T, it.stack.H, it.stack.W, it.stack.dtype, it.table).total, 256);
    }
    return off;
}

void batch_release(mf_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->done) cudaEventDestroy(b->done);
    b->done = nullptr;
    b->ran = false;
    b->exec = nullptr;
    b->graph = nullptr;
    b->capture = nullptr;
    mf::batch_free(b->dev);
    b->dev = nullptr;
    b->prepared = false;
}

}  // namespace

extern "C" {

mf_status mf_batch_create(mf_batch **out) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    auto *b = new mf_batch;
    if (cudaGetDevice(&b->device) != cudaSuccess) {
        delete b;
        return fail(MF_ECUDA, "no current CUDA device");
    }
    *out = b;
    return ok();
}

mf_status mf_batch_add(mf_batch *b, const mf_stack *stack, const float *sigma, const uint8_t *mask,
                       const mf_prf_table *table, float *snr_max, int32_t *argmax, float *snr_all,
                       int32_t *index) {
    if (!b) return fail(MF_EINVAL, "batch is NULL");
    if (b->prepared) return fail(MF_EINVAL, "batch already prepared; create a new one to change it");
    mf_status s = check_stack(stack);
    if (s != MF_OK) return s;
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (stack->T != table->T) return fail(MF_EINVAL, "stack has T=%lld, table has T=%d", (long long)stack->T,
                                          table->T);
    if (stack->H * stack->W == 0) return fail(MF_EINVAL, "empty stack in a batch");
    if (!sigma || !snr_max || !argmax) return fail(MF_EINVAL, "sigma, snr_max and argmax are required");
    if (table->device != b->device) return fail(MF_EINVAL, "table and batch live on different devices");
    if (table->plan.kernel == 2 && table->plan.f_planes > 0)
        return fail(MF_EUNSUPPORTED, "the phase-plane numerator (kernel 3) is not batched; use mf_search");
    b->items.push_back({*stack, sigma, mask, table, snr_max, argmax, snr_all});
    if (index) *index = (int32_t)b->items.size() - 1;
    return ok();
}

mf_status mf_batch_workspace_size(const mf_batch *b, size_t *bytes) {
    if (!b || !bytes) return fail(MF_EINVAL, "NULL argument");
    *bytes = batch_item_offsets(b, nullptr);
    return ok();
}

mf_status mf_batch_prepare(mf_batch *b, void *workspace, size_t workspace_bytes) {
    if (!b) return fail(MF_EINVAL, "batch is NULL");
    if (b->items.empty()) return fail(MF_EINVAL, "batch has no items");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device)
        return fail(MF_EINVAL, "batch lives on device %d, current device is %d", b->device, dev);
    std::vector<size_t> offs;
    const size_t need = batch_item_offsets(b, &offs);
    if (!workspace || workspace_bytes < need)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", need, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    batch_release(b);
    b->ws = (char *)workspace;
    b->layouts.clear();
    b->args.clear();
    for (const auto &it : b->items)
        b->layouts.push_back(mf::search_layout(it.stack.T, it.stack.H, it.stack.W, it.stack.dtype, it.table));
    for (size_t i = 0; i < b->items.size(); i++) {
        const auto &it = b->items[i];
        b->args.push_back(mf::SearchArgs{&it.stack, it.sigma, it.mask, it.table, it.snr_max, it.argmax, it.snr_all,
                                         b->ws + offs[i], b->layouts[i], nullptr});
    }
    char err[256] = {0};
    const int rc = mf::batch_build(b->args.data(), (int)b->args.size(), &b->dev, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e != cudaSuccess) return fail(MF_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    b->prepared = true;
    return ok();
}

mf_status mf_batch_run(mf_batch *b, mf_stream stream) {
    if (!b) return fail(MF_EINVAL, "batch is NULL");
    if (!b->prepared) return fail(MF_EINVAL, "call mf_batch_prepare first");
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->exec) {
        // capture on the batch's own stream (the legacy default stream cannot
        // be captured); the graph is then launched on the caller's stream
        char err[256] = {0};
        cudaStream_t cs = b->capture;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail(MF_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
        const int rc = mf::batch_enqueue(b->dev, b->args.data(), (int)b->args.size(), cs, err, sizeof err);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (rc != 0 || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(MF_ECUDA, "batch capture: %s", rc ? err : cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return fail(MF_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        b->graph = g;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return fail(MF_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    if (!b->done && (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess)
        return fail(MF_ECUDA, "cudaEventCreateWithFlags: %s", cudaGetErrorString(e));
    if ((e = cudaEventRecord(b->done, st)) != cudaSuccess)
        return fail(MF_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(e));
    b->ran = true;
    return ok();
}

mf_status mf_batch_poll(const mf_batch *b, int32_t *done) {
    if (!b || !done) return fail(MF_EINVAL, "NULL argument");
    if (!b->ran) {
        *done = 1;  // nothing launched
        return ok();
    }
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) {
        *done = 1;
        return ok();
    }
    if (e == cudaErrorNotReady) {
        *done = 0;
        return ok();
    }
    return fail(MF_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
}

mf_status mf_batch_info(const mf_batch *b, int32_t *items, int32_t *shape_groups, int32_t *graph_ready) {
    if (!b) return fail(MF_EINVAL, "batch is NULL");
    if (items) *items = (int32_t)b->items.size();
    if (shape_groups) {
        int mask = 0;  // bits 0..3: general shapes, 4..5: factored tile widths 32 and 64
        for (const auto &it : b->items) {
            const mf::Plan &pl = it.table->plan;
            mask |= pl.kernel == 2 ? 1 << (3 + pl.f_tw / 32) : 1 << pl.shape;
        }
        int n = 0;
        for (int i = 0; i < 6; i++) n += (mask >> i) & 1;
        *shape_groups = n;
    }
    if (graph_ready) *graph_ready = b->exec != nullptr;
    return ok();
}

void mf_batch_destroy(mf_batch *b) {
    if (!b) return;
    batch_release(b);
    delete b;
}

mf_status mf_rescore_workspace_size(int64_t H, int64_t W, int32_t k_top, size_t *bytes) {
    if (!bytes) return fail(MF_EINVAL, "bytes is NULL");
    if (H < 1 || W < 1 || k_top < 1) return fail(MF_EINVAL, "bad sizes");
    *bytes = mf::rescore_workspace(H, W, k_top);
    return ok();
}

mf_status mf_rescore_topk(const mf_stack *master, const float *sigma, const uint8_t *mask,
                          const mf_prf_table *table, const float *snr_max, const int32_t *argmax, int32_t k_top,
                          mf_candidate *out, int32_t *n_out, void *workspace, size_t workspace_bytes,
                          mf_stream stream) {
    mf_status s = check_stack(master);
    if (s != MF_OK) return s;
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (master->T != table->T) return fail(MF_EINVAL, "stack T differs from table T");
    if (master->H * master->W == 0) return fail(MF_EINVAL, "empty stack");
    if (!sigma || !snr_max || !argmax || !out || !n_out) return fail(MF_EINVAL, "NULL argument");
    if (k_top < 1 || (int64_t)k_top > master->H * master->W) return fail(MF_EINVAL, "k_top=%d out of range", k_top);
    if (k_top > 16384) return fail(MF_EUNSUPPORTED, "k_top above 16384");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != table->device)
        return fail(MF_EINVAL, "table lives on device %d, current device is %d", table->device, dev);
    const size_t need = mf::rescore_workspace(master->H, master->W, k_top);
    if (!workspace || workspace_bytes < need)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", need, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    mf::RescoreArgs a{master, sigma, mask, table, snr_max, argmax, k_top, out, n_out, (char *)workspace,
                      workspace_bytes, stream};
    char err[256] = {0};
    const int rc = mf::launch_rescore(a, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

mf_status mf_detect_workspace_size(int64_t H, int64_t W, int32_t max_out, size_t *bytes) {
    if (!bytes) return fail(MF_EINVAL, "bytes is NULL");
    if (H < 1 || W < 1 || H * W >= ((int64_t)1 << 31)) return fail(MF_EINVAL, "H=%lld W=%lld out of range",
                                                                  (long long)H, (long long)W);
    if (max_out < 0) return fail(MF_EINVAL, "max_out=%d < 0", max_out);
    *bytes = mf::detect_workspace(H, W, max_out);
    return ok();
}

mf_status mf_detect(const float *snr_max, const int32_t *argmax, int64_t H, int64_t W, const mf_detect_opts *opts,
                    float *z_out, mf_detection *out, int32_t max_out, int32_t *n_out, void *workspace,
                    size_t workspace_bytes, mf_stream stream) {
    if (!snr_max || !argmax || !opts || !n_out || (max_out > 0 && !out)) return fail(MF_EINVAL, "NULL argument");
    if (H < 1 || W < 1 || H * W >= ((int64_t)1 << 31))
        return fail(MF_EINVAL, "H=%lld W=%lld out of range", (long long)H, (long long)W);
    if (opts->window < 1 || opts->window > 2047 || opts->window % 2 == 0)
        return fail(MF_EINVAL, "window=%d must be odd and in 1..2047", opts->window);
    if (!std::isfinite(opts->threshold)) return fail(MF_EINVAL, "threshold not finite");
    if (max_out < 0) return fail(MF_EINVAL, "max_out=%d < 0", max_out);
    if (max_out > 16384) return fail(MF_EUNSUPPORTED, "max_out above 16384");
    const size_t need = mf::detect_workspace(H, W, max_out);
    if (!workspace || workspace_bytes < need)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", need, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    mf::DetectArgs a{snr_max, argmax, H, W, opts->window, opts->subtract_mean ? 1 : 0, opts->threshold,
                     z_out, out, max_out, n_out, (char *)workspace, workspace_bytes, stream};
    char err[256] = {0};
    const int rc = mf::launch_detect(a, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

mf_status mf_refit_workspace_size(int64_t T, size_t *bytes) {
    if (!bytes) return fail(MF_EINVAL, "bytes is NULL");
    if (T < 6 || T > (1 << 20)) return fail(MF_EINVAL, "T=%lld out of range 6..2^20", (long long)T);
    *bytes = mf::refit_workspace(T);
    return ok();
}

mf_status mf_background_refit(const float *data, int64_t T, int64_t H, int64_t W, const float *scatter, int32_t n,
                              const double *jitter, const mf_refit_opts *opts, float *resid, float *coef,
                              void *workspace, size_t workspace_bytes, mf_stream stream) {
    if (!data || !jitter || !opts || !resid) return fail(MF_EINVAL, "NULL argument");
    if (T < 6 || T > (1 << 20)) return fail(MF_EINVAL, "T=%lld: the fit needs at least 6 frames", (long long)T);
    if (H < 1 || W < 1 || H > (1 << 20) || W > (1 << 20) || H * W >= ((int64_t)1 << 31))
        return fail(MF_EINVAL, "H=%lld W=%lld out of range", (long long)H, (long long)W);
    if (scatter && (n < 1 || n > 4096)) return fail(MF_EINVAL, "scattered-light grid n=%d out of range", n);
    if (opts->iterations < 0 || opts->iterations > 1000)
        return fail(MF_EINVAL, "iterations=%d out of range 0..1000", opts->iterations);
    if (!(opts->delta > 0.0)) return fail(MF_EINVAL, "delta must be > 0");
    const size_t need = mf::refit_workspace(T);
    if (!workspace || workspace_bytes < need)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", need, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    // basis phi_t = (1, x, y, x^2, y^2, x y) and its Gram matrix, FP64
    std::vector<double> phi((size_t)T * 6);
    double G[36] = {0};
    for (int64_t t = 0; t < T; t++) {
        const double x = jitter[t * 2], y = jitter[t * 2 + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return fail(MF_EINVAL, "jitter of frame %lld not finite", (long long)t);
        double *f = &phi[(size_t)t * 6];
        f[0] = 1.0;
        f[1] = x;
        f[2] = y;
        f[3] = x * x;
        f[4] = y * y;
        f[5] = x * y;
        for (int i = 0; i < 6; i++)
            for (int j = 0; j < 6; j++) G[i * 6 + j] += f[i] * f[j];
    }
    // Cholesky G = R^T R (R upper triangular); a pivot that vanishes against
    // its diagonal means the jitter does not determine the six coefficients
    double R[36] = {0};
    for (int i = 0; i < 6; i++) {
        for (int j = i; j < 6; j++) {
            double v = G[i * 6 + j];
            for (int k = 0; k < i; k++) v -= R[k * 6 + i] * R[k * 6 + j];
            if (j == i) {
                if (!(v > 1e-12 * G[i * 6 + i]))
                    return fail(MF_EINVAL, "the jitter does not determine the background model (basis term %d)", i);
                R[i * 6 + i] = std::sqrt(v);
            } else {
                R[i * 6 + j] = v / R[i * 6 + i];
            }
        }
    }
    // R^-1 (upper triangular), Q = Phi R^-1 and Q^T 1
    double Rinv[36] = {0};
    for (int j = 0; j < 6; j++) {
        Rinv[j * 6 + j] = 1.0 / R[j * 6 + j];
        for (int i = j - 1; i >= 0; i--) {
            double v = 0.0;
            for (int k = i + 1; k <= j; k++) v += R[i * 6 + k] * Rinv[k * 6 + j];
            Rinv[i * 6 + j] = -v / R[i * 6 + i];
        }
    }
    std::vector<float> Q((size_t)T * mf::kRefitBasisPitch, 0.f);
    double q1[6] = {0};
    for (int64_t t = 0; t < T; t++) {
        const double *f = &phi[(size_t)t * 6];
        for (int j = 0; j < 6; j++) {
            double v = 0.0;
            for (int k = 0; k <= j; k++) v += f[k] * Rinv[k * 6 + j];
            Q[(size_t)t * mf::kRefitBasisPitch + j] = (float)v;
            q1[j] += v;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    cudaError_t e = cudaMemcpyAsync(ws + mf::refit_q_off(), Q.data(), Q.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws + mf::refit_rinv_off(T), Rinv, sizeof Rinv, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws + mf::refit_q1_off(T), q1, sizeof q1, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(MF_ECUDA, "basis upload: %s", cudaGetErrorString(e));
    mf::RefitArgs a{data, T, H, W, scatter, scatter ? n : 0, opts->iterations, (float)opts->delta, resid, coef,
                    ws, stream};
    char err[256] = {0};
    const int rc = mf::launch_refit(a, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

// ------------------------------------------------- host-buffer search ---

namespace {

struct HostSearchLayout {
    size_t stack_off, smax_off, amax_off, cand_off, n_off, search_off, rescore_off, total;
    size_t search_bytes, rescore_bytes;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

HostSearchLayout host_search_layout(const mf_stack *st, const mf_prf_table *table, int32_t k_top) {
    HostSearchLayout L{};
    const int64_t T = st->T, H = st->H, W = st->W;
    size_t off = 0;
    // the search's own workspace first: its status slot is then at offset 0
    // of this workspace too (mf_search_status)
    L.search_bytes = mf::search_layout(T, H, W, st->dtype, table).total;
    L.search_off = off;
    off = align256(off + L.search_bytes);
    L.stack_off = off;
    off = align256(off + (size_t)T * H * W * elem_size(st->dtype));
    L.smax_off = off;
    off = align256(off + (size_t)H * W * sizeof(float));
    L.amax_off = off;
    off = align256(off + (size_t)H * W * sizeof(int32_t));
    L.cand_off = off;
    off = align256(off + (size_t)(k_top > 0 ? k_top : 0) * sizeof(mf_candidate));
    L.n_off = off;
    off = align256(off + sizeof(int32_t));
    L.rescore_bytes = k_top > 0 ? mf::rescore_workspace(H, W, k_top) : 0;
    L.rescore_off = off;
    off = align256(off + L.rescore_bytes);
    L.total = off;
    return L;
}

}  // namespace

extern "C" {

mf_status mf_search_host_workspace_size(const mf_stack *stack, const mf_prf_table *table, int32_t k_top,
                                        size_t *bytes) {
    if (!bytes || !table || !stack) return fail(MF_EINVAL, "NULL argument");
    if (stack->T < 1 || stack->H < 0 || stack->W < 0) return fail(MF_EINVAL, "bad stack shape");
    if (stack->dtype != MF_F32 && stack->dtype != MF_BF16 && stack->dtype != MF_F16)
        return fail(MF_EINVAL, "unknown dtype %d", stack->dtype);
    if (k_top < 0) return fail(MF_EINVAL, "k_top=%d is negative", k_top);
    *bytes = host_search_layout(stack, table, k_top).total;
    return ok();
}

mf_status mf_search_host(const mf_stack *host_stack, const float *sigma, const uint8_t *mask,
                         const mf_prf_table *table, float *snr_max_host, int32_t *argmax_host, int32_t k_top,
                         mf_candidate *cand_host, int32_t *n_cand_host, void *workspace, size_t workspace_bytes,
                         mf_stream stream, mf_stream copy_stream, void *ws_free) {
    mf_status s = check_stack(host_stack);
    if (s != MF_OK) return s;
    if (!table) return fail(MF_EINVAL, "table is NULL");
    if (host_stack->T != table->T)
        return fail(MF_EINVAL, "stack has T=%lld, table has T=%d", (long long)host_stack->T, table->T);
    const int64_t T = host_stack->T, H = host_stack->H, W = host_stack->W;
    if (H * W == 0) return ok();
    if (!sigma || !snr_max_host || !argmax_host) return fail(MF_EINVAL, "sigma, snr_max and argmax are required");
    if (k_top < 0 || (int64_t)k_top > H * W) return fail(MF_EINVAL, "k_top=%d out of range", k_top);
    if (k_top > 16384) return fail(MF_EUNSUPPORTED, "k_top above 16384");
    if (k_top > 0 && (!cand_host || !n_cand_host)) return fail(MF_EINVAL, "k_top > 0 needs cand and n_cand");
    const HostSearchLayout L = host_search_layout(host_stack, table, k_top);
    if (!workspace || workspace_bytes < L.total)
        return fail(MF_EINVAL, "workspace of %zu bytes needed, %zu given", L.total, workspace_bytes);
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != table->device)
        return fail(MF_EINVAL, "table lives on device %d, current device is %d", table->device, dev);
    char *ws = (char *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStream_t up = copy_stream ? (cudaStream_t)copy_stream : st;
    cudaEvent_t freed = (cudaEvent_t)ws_free;
    const size_t es = elem_size(host_stack->dtype);
    cudaError_t e = cudaSuccess;
    if (freed) e = cudaStreamWaitEvent(up, freed, 0);  // the previous call on this workspace is done with it
    // upload: one 2-D copy when rows are contiguous, else one per frame
    if (e == cudaSuccess && host_stack->row_stride == W) {
        e = cudaMemcpy2DAsync(ws + L.stack_off, (size_t)H * W * es, host_stack->data,
                              (size_t)(T > 1 ? host_stack->frame_stride : H * W) * es, (size_t)H * W * es, (size_t)T,
                              cudaMemcpyHostToDevice, up);
    } else {
        for (int64_t t = 0; t < T && e == cudaSuccess; t++)
            e = cudaMemcpy2DAsync(ws + L.stack_off + (size_t)t * H * W * es, (size_t)W * es,
                                  (const char *)host_stack->data + (size_t)t * host_stack->frame_stride * es,
                                  (size_t)host_stack->row_stride * es, (size_t)W * es, (size_t)H,
                                  cudaMemcpyHostToDevice, up);
    }
    if (e == cudaSuccess && up != st) {
        // the kernels wait for the upload (the event object may go once the wait is enqueued)
        cudaEvent_t landed = nullptr;
        e = cudaEventCreateWithFlags(&landed, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(landed, up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, landed, 0);
        if (landed) cudaEventDestroy(landed);
    }
    if (e != cudaSuccess) return fail(MF_ECUDA, "stack upload: %s", cudaGetErrorString(e));
    mf_stack dstack = *host_stack;
    dstack.data = ws + L.stack_off;
    dstack.row_stride = W;
    dstack.frame_stride = H * W;
    float *smax = (float *)(ws + L.smax_off);
    int32_t *amax = (int32_t *)(ws + L.amax_off);
    s = mf_search(&dstack, sigma, mask, table, smax, amax, nullptr, ws + L.search_off, L.search_bytes, stream);
    if (s != MF_OK) return s;
    if (k_top > 0) {
        s = mf_rescore_topk(&dstack, sigma, mask, table, smax, amax, k_top, (mf_candidate *)(ws + L.cand_off),
                            (int32_t *)(ws + L.n_off), ws + L.rescore_off, L.rescore_bytes, stream);
        if (s != MF_OK) return s;
    }
    e = cudaMemcpyAsync(snr_max_host, smax, (size_t)H * W * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(argmax_host, amax, (size_t)H * W * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && k_top > 0)
        e = cudaMemcpyAsync(cand_host, ws + L.cand_off, (size_t)k_top * sizeof(mf_candidate), cudaMemcpyDeviceToHost,
                            st);
    if (e == cudaSuccess && k_top > 0)
        e = cudaMemcpyAsync(n_cand_host, ws + L.n_off, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && freed) e = cudaEventRecord(freed, st);
    if (e != cudaSuccess) return fail(MF_ECUDA, "result download: %s", cudaGetErrorString(e));
    return ok();
}

}  // extern "C"

mf_status mf_profile_enable(int32_t on) {
    mf::profile_enable(on);
    return ok();
}

mf_status mf_profile_read(mf_profile *out, int32_t reset) {
    if (!out) return fail(MF_EINVAL, "out is NULL");
    mf::profile_read(out, reset);
    return ok();
}

const char *mf_last_error(void) { return g_err.c_str(); }

mf_status mf_device_status(void) {
    int st = 0;
    const int rc = mf::read_device_status(&st);
    if (rc != 0) return fail(MF_ECUDA, "%s", cudaGetErrorString((cudaError_t)rc));
    if (st != 0) return fail(MF_ETIMEOUT, "a device wait ran out of its budget (code %d)", st);
    return ok();
}

mf_status mf_wait_probe(mf_stream stream) {
    char err[256] = {0};
    const int rc = mf::launch_wait_probe(stream, nullptr, err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

mf_status mf_wait_probe_search(void *workspace, mf_stream stream) {
    if (!workspace) return fail(MF_EINVAL, "workspace is NULL");
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    char err[256] = {0};
    const int rc = mf::launch_wait_probe(stream, static_cast<int *>(workspace), err, sizeof err);
    if (rc != 0) return fail(MF_ECUDA, "%s", err);
    return ok();
}

mf_status mf_search_status(const void *workspace, int32_t *out, mf_stream stream) {
    if (!workspace || !out) return fail(MF_EINVAL, "NULL argument");
    if ((uintptr_t)workspace % 256 != 0) return fail(MF_EINVAL, "workspace must be 256-byte aligned");
    const cudaError_t e = cudaMemcpyAsync(out, workspace, sizeof(int32_t), cudaMemcpyDefault, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(MF_ECUDA, "status copy: %s", cudaGetErrorString(e));
    return ok();
}

const char *mf_version(void) { return "libmf 0.1 (sm_103a)"; }

}  // extern "C"
