/*
 * FP64 CPU oracle for the trajectory matched filter of Ganapathi (2022),
 * "Maximum Likelihood Systematic Effect Modeling and Matched Filtering to
 * Detect Trans-Neptunian Objects with TESS", Section 3.2 (Matched Filter).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA library and includes nothing but the C standard library.
 *
 * What it computes (plain definitions, FP64, no blocking or fusion):
 *   - a pixel response function (PRF) footprint of 5x5 pixels around the
 *     pixel nearest to the sub-pixel source position (Section 2: the PRF
 *     spreads a point source over a few pixels);
 *   - linear trajectories in pixel space, p + v*t (Section 2 and 4.2: each
 *     trajectory is a straight line characterised by its displacement);
 *   - the matched filter of one trajectory: the trajectory line convolved
 *     with the PRF, one 5x5 footprint per frame (Section 3.2);
 *   - the score: the dot product of that filter with the inverse-variance
 *     weighted residual stack at every start pixel (Section 3.2, Eq. 5),
 *     normalised by the filter energy to a signal-to-noise ratio, and the
 *     maximum over the filter bank (Section 3.2, last paragraph before
 *     the shift-stack discussion).
 *
 * Readings of the paper taken here (the paper is silent on them):
 *   - the PRF is a circular Gaussian integrated over each pixel,
 *     truncated to the 5x5 footprint and renormalised to unit sum;
 *   - base pixel s = floor(c + 1/2) per axis for the position c = v*t;
 *     the sub-pixel phase is c - s in [-1/2, 1/2);
 *   - "S = D * F" is a cross-correlation (a dot product at each location);
 *   - pixels outside the frame and masked pixels have zero inverse variance
 *     (they drop out of both the dot product and the normalisation);
 *   - the score is SNR = N / sqrt(D), N = sum W*lambda*r, D = sum W^2*lambda.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>

/* One pixel of a 1-D Gaussian of width sigma centred at phase, integrated
 * over the pixel [a - 1/2, a + 1/2] (Section 2: the PRF sets how a point
 * source's flux is shared between neighbouring pixels). */
double orc_pixel_integrated_gauss(int a, double phase, double sigma)
{
    const double s = sigma * sqrt(2.0);
    return 0.5 * (erf((a + 0.5 - phase) / s) - erf((a - 0.5 - phase) / s));
}

/* 5x5 PRF footprint for a source at sub-pixel offset (phx, phy) from the
 * centre of the base pixel.  taps[(dy + 2) * 5 + (dx + 2)] is the fraction
 * of the flux that lands in the pixel (dx, dy) away from the base pixel.
 * kind 0: pixel-integrated Gaussian; kind 1: Gaussian sampled at pixel
 * centres; kind 2: the shift-stack filter (Section 3.2, after Rice et al.
 * 2020): a single value of 1 in the pixel that holds the source's centre
 * (the base pixel), 0 elsewhere.  The footprint is divided by its own sum. */
void orc_prf_taps(double phx, double phy, double sigma, int kind, double *taps)
{
    double total = 0.0;
    for (int dy = -2; dy <= 2; dy++) {
        for (int dx = -2; dx <= 2; dx++) {
            double w;
            if (kind == 0) {
                w = orc_pixel_integrated_gauss(dx, phx, sigma) *
                    orc_pixel_integrated_gauss(dy, phy, sigma);
            } else if (kind == 2) {
                w = (dx == 0 && dy == 0) ? 1.0 : 0.0;
            } else {
                double ex = dx - phx, ey = dy - phy;
                w = exp(-(ex * ex + ey * ey) / (2.0 * sigma * sigma));
            }
            taps[(dy + 2) * 5 + (dx + 2)] = w;
            total += w;
        }
    }
    for (int i = 0; i < 25; i++) taps[i] /= total;
}

/* Filter bank of K linear trajectories over T frames (Section 3.2: one
 * filter per trajectory, the trajectory line convolved with the PRF).
 * For trajectory k and frame t the source sits at c = v_k * t from its
 * start pixel.  shifts[(k*T + t)*2 + 0] = s_x, [.. + 1] = s_y (base pixel),
 * taps[(k*T + t)*25 + ...] = the 5x5 PRF at the phase c - s. */
void orc_trajectory_table(int K, int T, const double *vx, const double *vy,
                          double sigma, int kind, int32_t *shifts, double *taps)
{
    for (int k = 0; k < K; k++) {
        for (int t = 0; t < T; t++) {
            double cx = vx[k] * (double)t;
            double cy = vy[k] * (double)t;
            double sx = floor(cx + 0.5);
            double sy = floor(cy + 0.5);
            shifts[((size_t)k * T + t) * 2 + 0] = (int32_t)sx;
            shifts[((size_t)k * T + t) * 2 + 1] = (int32_t)sy;
            orc_prf_taps(cx - sx, cy - sy, sigma, kind,
                         taps + ((size_t)k * T + t) * 25);
        }
    }
}

/* The filter bank of a phase-quantised search (the precompute-then-gather
 * form of a sparse matched filter: each frame is correlated once with the
 * footprints of Q x Q sub-pixel phases, and every trajectory then gathers the
 * image of its phase).  Its value is the plain matched filter with the
 * footprint of frame t evaluated at the phase rounded to a multiple of 1/Q
 * pixel, phi_q = floor(phi Q + 1/2) / Q per axis (halves round up, as for the
 * base pixel); the base pixel is unchanged. */
void orc_trajectory_table_quantised(int K, int T, const double *vx, const double *vy, double sigma, int kind,
                                    int Q, int32_t *shifts, double *taps)
{
    for (int k = 0; k < K; k++) {
        for (int t = 0; t < T; t++) {
            double cx = vx[k] * (double)t;
            double cy = vy[k] * (double)t;
            double sx = floor(cx + 0.5);
            double sy = floor(cy + 0.5);
            double qx = floor((cx - sx) * Q + 0.5) / Q;
            double qy = floor((cy - sy) * Q + 0.5) / Q;
            shifts[((size_t)k * T + t) * 2 + 0] = (int32_t)sx;
            shifts[((size_t)k * T + t) * 2 + 1] = (int32_t)sy;
            orc_prf_taps(qx, qy, sigma, kind, taps + ((size_t)k * T + t) * 25);
        }
    }
}

/* The same table with the frames' times and the pointing jitter (Section
 * 2.1: the spacecraft's pointing jitters by a fraction of a pixel, and the
 * filter follows the trajectory line including that jitter; Fig. 3: frames
 * are missing while TESS downlinks, so time jumps).  Frame t is taken at
 * time times[t] (in frame cadences; NULL: t) and every source appears
 * displaced by (jx[t], jy[t]) pixels (NULL: 0), so the position is
 * c = v * times[t] + j[t].  Q > 0 rounds the phases to multiples of 1/Q as
 * orc_trajectory_table_quantised does (Q = 0: exact phases). */
void orc_trajectory_table_frames(int K, int T, const double *vx, const double *vy, const double *times,
                                 const double *jx, const double *jy, double sigma, int kind, int Q,
                                 int32_t *shifts, double *taps)
{
    for (int k = 0; k < K; k++) {
        for (int t = 0; t < T; t++) {
            double tau = times ? times[t] : (double)t;
            double cx = vx[k] * tau + (jx ? jx[t] : 0.0);
            double cy = vy[k] * tau + (jy ? jy[t] : 0.0);
            double sx = floor(cx + 0.5);
            double sy = floor(cy + 0.5);
            double px = cx - sx, py = cy - sy;
            if (Q > 0) {
                px = floor(px * Q + 0.5) / Q;
                py = floor(py * Q + 0.5) / Q;
            }
            shifts[((size_t)k * T + t) * 2 + 0] = (int32_t)sx;
            shifts[((size_t)k * T + t) * 2 + 1] = (int32_t)sy;
            orc_prf_taps(px, py, sigma, kind, taps + ((size_t)k * T + t) * 25);
        }
    }
}

/* Inverse variance per pixel (Section 3.2: Gaussian noise of known width;
 * bright pixels are clipped).  Masked pixels get weight 0.  A pixel whose
 * noise is not a finite positive number carries no usable measurement
 * (Section 3.2 weighs each pixel by its known noise), so it is excluded the
 * same way: sigma <= 0, NaN or infinite gives weight 0. */
void orc_inverse_variance(int H, int W, const float *sigma, const uint8_t *mask,
                          double *lam)
{
    for (size_t i = 0; i < (size_t)H * W; i++) {
        double s = (double)sigma[i];
        int masked = mask ? (mask[i] != 0) : 0;
        int usable = s > 0.0 && isfinite(s);
        lam[i] = (masked || !usable) ? 0.0 : 1.0 / (s * s);
    }
}

/* N and D for one start pixel (py, px) and one filter k, straight from the
 * definition: loop over frames, then over the 25 footprint pixels.
 * r_t(q) = frame_scale[t] * residual[t][q] (frame_scale NULL means 1). */
static void orc_one(int T, int H, int W, const float *res, const double *frame_scale,
                    const double *lam, const int32_t *shifts, const double *taps,
                    int k, int py, int px, double *n_out, double *d_out)
{
    double n = 0.0, d = 0.0;
    for (int t = 0; t < T; t++) {
        const int32_t *s = shifts + ((size_t)k * T + t) * 2;
        const double *w = taps + ((size_t)k * T + t) * 25;
        double scale = frame_scale ? frame_scale[t] : 1.0;
        for (int dy = -2; dy <= 2; dy++) {
            for (int dx = -2; dx <= 2; dx++) {
                long qy = (long)py + s[1] + dy;
                long qx = (long)px + s[0] + dx;
                if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue; /* outside: weight 0 */
                size_t q = (size_t)qy * W + (size_t)qx;
                double wt = w[(dy + 2) * 5 + (dx + 2)];
                double r = scale * (double)res[(size_t)t * H * W + q];
                n += wt * lam[q] * r;
                d += wt * wt * lam[q];
            }
        }
    }
    *n_out = n;
    *d_out = d;
}

/* Every filter at every start pixel: N[k][y][x] and D[k][y][x]
 * (Section 3.2, Eq. 5: the dot product at all pixel locations). */
void orc_search_full(int T, int H, int W, const float *res, const double *frame_scale,
                     const double *lam, int K, const int32_t *shifts, const double *taps,
                     double *N, double *D)
{
    long P = (long)H * W;
#pragma omp parallel for schedule(dynamic, 16)
    for (long p = 0; p < P; p++) {
        int py = (int)(p / W), px = (int)(p % W);
        for (int k = 0; k < K; k++) {
            orc_one(T, H, W, res, frame_scale, lam, shifts, taps, k, py, px,
                    &N[(size_t)k * P + p], &D[(size_t)k * P + p]);
        }
    }
}

/* The same for a list of (y, x, k) triples; used for sampled checks at
 * sizes where the full map is out of reach. */
void orc_search_points(int T, int H, int W, const float *res, const double *frame_scale,
                       const double *lam, const int32_t *shifts, const double *taps,
                       long n, const int32_t *py, const int32_t *px, const int32_t *pk,
                       double *N, double *D)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (long i = 0; i < n; i++) {
        orc_one(T, H, W, res, frame_scale, lam, shifts, taps, pk[i], py[i], px[i],
                &N[i], &D[i]);
    }
}
