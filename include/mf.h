/*
 * mf.h -- C ABI of libmf, a GB300 (sm_103a) trajectory matched filter.
 *
 * The operation is the matched filter of Ganapathi (2022), "Maximum
 * Likelihood Systematic Effect Modeling and Matched Filtering to Detect
 * Trans-Neptunian Objects with TESS", Section 3.2 (Matched Filter), Eq. 5:
 * one filter per candidate trajectory (the trajectory line convolved with the
 * pixel response function, PRF), its dot product with the residual stack at
 * every start pixel, and the maximum over the filter bank.
 *
 * Notation used in the comments below.  T frames of H x W pixels; K
 * trajectories.  r_t(q) is the residual at pixel q of frame t, sigma(q) the
 * per-pixel noise, m(q) the mask.  lambda(q) = (1 - m(q)) / sigma(q)^2 is the
 * inverse variance, taken as 0 outside the frame.  For trajectory k and frame
 * t the library stores a base shift s_{k,t} (integer pixels) and a 5x5
 * footprint W_{k,t}(a, b), a, b in -2..2.  Then, for start pixel p,
 *     N_k(p) = sum_t sum_{a,b} W_{k,t}(a,b) lambda(q) r_t(q),
 *     D_k(p) = sum_t sum_{a,b} W_{k,t}(a,b)^2 lambda(q),
 *     q = p + s_{k,t} + (a, b),   SNR_k(p) = N_k(p) / sqrt(D_k(p)),
 * and the flux estimate is N_k(p) / D_k(p).  N is the dot product of Eq. 5
 * weighted by the Gaussian noise model of Section 3.2; D is its variance.
 *
 * Conventions for every entry point:
 *   - Device pointers are CUDA device memory on the current device, owned by
 *     the caller.  The library owns only the table and batch handles it
 *     creates.  The host-only calls (mf_prf_plan, mf_prf_plan_frames,
 *     mf_prf_bank) touch no device and need no GPU.
 *   - Work is enqueued on the given stream and is asynchronous; results are
 *     valid once the caller synchronises that stream.  NULL stream means the
 *     legacy default stream.
 *   - Arguments are validated before anything is enqueued.  On a bad argument
 *     the call returns MF_EINVAL, enqueues nothing and leaves outputs as they
 *     were; mf_last_error() then describes the problem.
 *   - mf_search and mf_rescore_topk allocate nothing: scratch memory is the
 *     caller's workspace, sized by the matching *_workspace_size call.
 *   - A device-side wait that runs out of its iteration budget gives up
 *     instead of hanging or trapping.  A search records the failure in its
 *     own status slot (the first bytes of its workspace, read with
 *     mf_search_status without synchronising anything); the search's
 *     finalisation copies it into a device-wide status word, which
 *     mf_device_status() reads.  A failure in one search does not stop
 *     others, on the same or other streams.
 *   - The library looks up the device addresses of its own device-side
 *     variables (the status word, mf_search_noalloc's scratch) once per
 *     device and keeps them for the process: they do not survive
 *     cudaDeviceReset, after which the library must not be used again in
 *     that process.
 */
#ifndef MF_H
#define MF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque CUDA stream (a cudaStream_t). */
typedef void *mf_stream;

typedef enum {
    MF_OK = 0,
    MF_EINVAL = 1,        /* bad argument; nothing was enqueued */
    MF_ENOMEM = 2,        /* table creation could not allocate device memory */
    MF_ECUDA = 3,         /* a CUDA runtime call failed (text in mf_last_error) */
    MF_ETIMEOUT = 4,      /* a bounded device wait gave up (see mf_device_status) */
    MF_EUNSUPPORTED = 5   /* valid request the library does not handle */
} mf_status;

typedef enum {
    MF_F32 = 0,   /* float32 residuals */
    MF_BF16 = 1,  /* bfloat16 residuals, r_t = frame_scale[t] * value */
    MF_F16 = 2    /* float16 residuals, r_t = frame_scale[t] * value */
} mf_dtype;

/* PRF used to build the filter bank (Section 2: a point source spreads over
 * neighbouring pixels; the paper's TESS PRF has no closed form, so a Gaussian
 * of width sigma_px stands in).  The footprint is always 5 x 5 pixels around
 * the base pixel and is renormalised to unit sum at each sub-pixel phase.
 *   kind 0: Gaussian integrated over each pixel (erf differences);
 *   kind 1: Gaussian sampled at pixel centres;
 *   kind 2: the shift-stack filter (Section 3.2, after Rice et al. 2020): a
 *           single 1 in the base pixel, the pixel holding the source's
 *           centre; sigma_px must still be a finite value > 0 (unused).
 * phase_steps: 0 evaluates the footprint at the exact sub-pixel phase;
 * Q in 1 .. 4096 rounds each axis's phase to the nearest multiple of 1/Q
 * (halves up, as for the base pixel; the base pixel is unchanged).  Not in
 * the paper: the filter bank of a phase-quantised search, in which every
 * frame would be correlated once per rounded phase and each trajectory
 * would gather the result of its own (one route to the faster sparse
 * evaluation Section 3.2 anticipates); the search runs it exactly. */
typedef struct {
    int32_t kind;
    int32_t phase_steps;
    double sigma_px;
} mf_prf_params;

/* A residual stack in device memory, frame-major: element (t, y, x) lives at
 * data + t * frame_stride + y * row_stride + x (strides in elements).
 * frame_scale is a device array of T floats (NULL means all 1); the residual
 * used by the filter is frame_scale[t] * element.  Scaled bf16/fp16 storage
 * is not in the paper; it halves the bytes of the stack, and of the weighted
 * stack the search keeps (see mf_search). */
typedef struct {
    const void *data;
    int32_t dtype;            /* mf_dtype */
    int32_t reserved;
    int64_t T, H, W;
    int64_t frame_stride;     /* >= H * row_stride */
    int64_t row_stride;       /* >= W */
    const float *frame_scale; /* device, [T], or NULL */
} mf_stack;

/* One re-scored candidate (mf_rescore_topk). */
typedef struct {
    int32_t y, x;        /* start pixel */
    int32_t k;           /* trajectory index (as given at table creation) */
    int32_t reserved;
    double snr;          /* FP64 N / sqrt(D) recomputed from the FP32 master stack */
    double flux;         /* FP64 flux estimate N / D (Section 3.2: the score estimates the flux) */
    float snr_search;    /* the value mf_search reported for this pixel */
    float reserved2;
} mf_candidate;

/* Filter bank handle: per (k, t) base shift and 5x5 footprint, kept on the
 * host in FP64 and on the device in the layouts the kernels read. */
typedef struct mf_prf_table mf_prf_table;

/* Build the filter bank for K linear trajectories over T frames (Section 2:
 * trajectories are straight lines in pixel space; Section 3.2: a filter is
 * the trajectory line convolved with the PRF).  vx[k], vy[k] are host arrays
 * of velocities in pixels per frame (x = column, y = row).  For frame t the
 * position is c = v * t (FP64); base shift s = floor(c + 1/2) per axis; phase
 * c - s; footprint = the PRF at that phase.  Allocates device memory for the
 * table (the only allocation the library makes) on the current device.
 * Errors: MF_EINVAL (K < 1, T < 1, NULL pointers, non-finite velocity,
 * sigma_px <= 0, unknown kind, phase_steps outside 0 .. 4096, |v| * T beyond
 * 2^20 pixels), MF_ENOMEM. */
mf_status mf_prf_table_create(const mf_prf_params *prf, const double *vx, const double *vy,
                              int32_t K, int32_t T, mf_prf_table **out);

/* Kernel-layout choices for a table (not in the paper).
 *
 * kernel selects the numerator: 1 = the general kernel, 25 FMAs per
 * (trajectory, pixel, frame), for any footprint; 2 = the factored kernel for
 * separable footprints W(a, b) = u_x(a) u_y(b) (every table built by
 * mf_prf_table_create is separable): a 5-tap pass along rows, shared by the
 * trajectories of a CTA that have the same v_x, then a 5-tap pass down
 * columns per trajectory; 3 = the factored kernel with phase planes, for
 * phase-quantised banks (phase_steps > 0; the precompute-then-gather form
 * of a sparse matched filter): per frame, one 5-tap column pass per rounded
 * y-phase present among the CTA's trajectories over the whole window, then
 * one add per (trajectory, pixel) gathered from its phase's plane (FP32
 * stacks; bf16 / fp16 ones are weighted in FP32; not in batches);
 * 0 = automatic (factored whenever the table is separable and the frame
 * windows fit).  All give the same sums up to FP32 rounding.
 *
 * General kernel: shape selects how a CTA's 16 warps split between
 * trajectories and 32 x 32 sub-tiles: 0: 16 trajectories x 1 sub-tile,
 * 1: 8 x (1 x 2), 2: 4 x (2 x 2), 3: 2 x (2 x 4) (rows x columns of
 * sub-tiles); -1 lets the planner's cost model choose.  A shape >= 0 with
 * kernel = 0 selects the general kernel.
 *
 * Factored kernel: group = trajectories per CTA (all with one v_x), tile_h a
 * multiple of 32, tile_w 32 or 64, with group * tile_h / 32 * tile_w / 32 <= 20
 * warps; stages = frame windows in flight (2..6); segments = number of
 * consecutive frame ranges the frames are split into (1..16): within a
 * segment a CTA follows each trajectory from where it stands at the
 * segment's first frame, so the rows a group's window spans grow with the
 * segment's length instead of the stack's; segments run as consecutive
 * launches, the first storing the numerators and the others adding to them
 * (a fixed summation order); 0 = planner's choice.
 * An autotuner times several layouts and keeps the fastest. */
typedef struct {
    int32_t shape;
    int32_t vec;         /* floats per shared-memory load in the general numerator: 1, 2, 4;
                            0 = default */
    int32_t lockstep;    /* general numerator frame hand-off: 1 = CTA barrier per frame, 0 = last
                            warp out refills the stage, -1 = default */
    int32_t kernel;      /* 0 automatic, 1 general, 2 factored */
    int32_t group;       /* factored: trajectories per CTA, 0 = automatic */
    int32_t tile_h;      /* factored: output rows per CTA, 0 = automatic */
    int32_t tile_w;      /* factored: output columns per CTA, 0 = automatic */
    int32_t stages;      /* factored: frame windows in flight, 0 = automatic */
    int32_t segments;    /* factored: time segments, 0 = automatic (see below) */
} mf_plan_opts;

/* mf_prf_table_create with layout options (opts NULL = automatic).
 * MF_EUNSUPPORTED if the requested shape cannot hold the trajectories'
 * frame windows in shared memory. */
mf_status mf_prf_table_create_ex(const mf_prf_params *prf, const double *vx, const double *vy,
                                 int32_t K, int32_t T, const mf_plan_opts *opts,
                                 mf_prf_table **out);

/* Frame times and pointing jitter (Section 2.1: the pointing jitters by a
 * fraction of a pixel and the filter follows the trajectory including it;
 * Fig. 3: time jumps where frames are missing while TESS downlinks).  A
 * source at start pixel p appears at c = p + v * times[t] + jitter[t] in
 * frame t; base pixel and phase follow from c as for the linear table.
 *   times   host double[T], frame times in frame cadences (any finite
 *           values: gaps, fractional mid-exposure times); NULL: 0..T-1;
 *   jitter  host double[T][2], (x, y) pointing offset in pixels; NULL: 0. */
typedef struct {
    const double *times;
    const double *jitter;
} mf_frames;

/* mf_prf_table_create_ex with a frame model (frames NULL = the linear
 * table).  The arrays are read during the call only.  Trajectories that
 * share v_x still share the row pass of the factored numerator (the jitter
 * is common to all of them).
 * Errors as mf_prf_table_create_ex, plus MF_EINVAL for a non-finite time or
 * jitter or a position beyond 2^20 pixels. */
mf_status mf_prf_table_create_frames(const mf_prf_params *prf, const double *vx, const double *vy,
                                     int32_t K, int32_t T, const mf_frames *frames,
                                     const mf_plan_opts *opts, mf_prf_table **out);

/* Build a filter bank from explicit per-(k, t) shifts and footprints (host
 * arrays): shifts[(k*T + t)*2 + 0] = s_x, [.. + 1] = s_y;
 * taps[(k*T + t)*25 + (b + 2)*5 + (a + 2)] = W_{k,t}(a, b), a = column offset,
 * b = row offset.  Any footprint is accepted (not necessarily separable or
 * normalised), e.g. the single unit tap that turns the search into
 * shift-and-add (Section 3.2, the shift-stack comparison).
 * Errors as mf_prf_table_create, plus non-finite taps. */
mf_status mf_prf_table_create_custom(const int32_t *shifts, const double *taps,
                                     int32_t K, int32_t T, mf_prf_table **out);

/* Free the table's host and device memory.  NULL is a no-op.  The caller must
 * make sure no enqueued work still uses it. */
void mf_prf_table_destroy(mf_prf_table *table);

/* K and T of a table. */
mf_status mf_prf_table_dims(const mf_prf_table *table, int32_t *K, int32_t *T);

/* Copy the FP64 filter bank back to host arrays laid out as in
 * mf_prf_table_create_custom (either pointer may be NULL). */
mf_status mf_prf_table_export(const mf_prf_table *table, int32_t *shifts, double *taps);

/* How the library laid out a filter bank for the kernels (not in the paper):
 * trajectories are grouped so that a CTA's warps share one staged frame
 * window; these numbers describe that grouping and its memory. */
typedef struct {
    int32_t K, T;
    int32_t groups;           /* trajectory groups = CTAs per output tile */
    int32_t warps_per_group;  /* trajectories per CTA */
    int32_t tile_h, tile_w;   /* output tile of one CTA, start pixels */
    int32_t window_pitch;     /* floats per staged window row */
    int32_t window_rows;      /* rows of the largest staged window */
    int32_t segments;         /* rows of the collapsed denominator kernels */
    int32_t max_abs_shift;    /* largest |s| over all (k, t), pixels */
    int64_t g_nnz;            /* nonzero weights of the collapsed denominator kernels */
    int64_t smem_bytes;       /* dynamic shared memory of the numerator kernel */
    int64_t device_bytes;     /* device memory the table holds */
    double cost;              /* planner's estimate, SM cycles per start pixel */
    int32_t vec;              /* floats per shared-memory load in the numerator */
    int32_t lockstep;         /* numerator frame hand-off (see mf_plan_opts) */
    int32_t kernel;           /* numerator: 1 general, 2 factored (see mf_plan_opts) */
    int32_t stages;           /* frame windows in flight per CTA */
    int32_t time_segments;    /* time segments of the factored numerator (1 otherwise) */
    int32_t taps;             /* footprint taps per axis the factored passes run: 5, or 1
                                 when every footprint is a single centre tap (kind 2) */
    int32_t den_tile_h;       /* denominator: rows of start pixels per CTA when each CTA
                                 stages the lambda box its trajectory reaches in shared
                                 memory; 0 when the largest box does not fit (the
                                 denominator then reads lambda through the L1 cache) */
    int32_t phase_planes;     /* factored numerator with phase planes (kernel 3): planes a
                                 CTA holds per frame; 0: a column pass per trajectory */
} mf_table_info;

/* Layout of an existing table. */
mf_status mf_prf_table_info(const mf_prf_table *table, mf_table_info *info);

/* Plan a Gaussian-PRF filter bank on the host only (same arguments and errors
 * as mf_prf_table_create) and report its layout; allocates no device memory
 * and needs no GPU.  device_bytes is what mf_prf_table_create would allocate. */
mf_status mf_prf_plan(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                      int32_t T, const mf_plan_opts *opts, mf_table_info *info);
/* mf_prf_plan for a filter bank with a frame model (mf_prf_table_create_frames):
 * the same layout, host only, no device needed.  frames may be NULL. */
mf_status mf_prf_plan_frames(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K,
                             int32_t T, const mf_frames *frames, const mf_plan_opts *opts,
                             mf_table_info *info);

/* The filter bank itself, built on the host only (no device needed): the
 * base shifts and FP64 footprints that mf_prf_table_create_frames would
 * build, in mf_prf_table_export's layout (Section 3.2: the trajectory line
 * convolved with the PRF).  frames may be NULL (the linear table).  shifts:
 * host int32[K][T][2] or NULL; taps: host double[K][T][25] or NULL.  Errors
 * as mf_prf_table_create_frames. */
mf_status mf_prf_bank(const mf_prf_params *prf, const double *vx, const double *vy, int32_t K, int32_t T,
                      const mf_frames *frames, int32_t *shifts, double *taps);

/* Bytes of workspace mf_search needs for this stack shape and table. */
mf_status mf_search_workspace_size(const mf_stack *stack, const mf_prf_table *table,
                                   size_t *bytes);

/* The matched-filter search (Section 3.2, Eq. 5 and the maximum over the
 * filter bank).  Inputs, all device memory:
 *   stack      residuals r (see mf_stack); T must equal the table's T;
 *   sigma      float[H*W] row-major per-pixel noise;
 *   mask       uint8[H*W] row-major, nonzero = pixel excluded (the paper
 *              clips bright pixels), or NULL for none.  Unmasked pixels need
 *              a finite sigma > 0; others are treated as masked;
 *   table      filter bank (K trajectories);
 * Outputs, device memory:
 *   snr_max    float[H*W]: max_k SNR_k(p) over filters with D_k(p) > 0;
 *   argmax     int32[H*W]: the smallest k attaining it; a pixel where no
 *              filter has D > 0 gets snr_max 0 and argmax -1;
 *   snr_all    float[K*H*W] (k-major) with every SNR_k(p), 0 where D = 0,
 *              or NULL to skip it.
 * workspace: device memory of at least mf_search_workspace_size bytes,
 * 256-byte aligned; its contents on entry do not matter.
 * Arithmetic: numerator in FP32 with blocked accumulation over frames;
 * denominator from FP32 products accumulated in FP64.  Precision form (a
 * bf16 / fp16 stack searched by the factored numerator, i.e. any table built
 * from velocities unless the general kernel is forced): the weighted
 * residual lambda * frame_scale[t] * value is formed in FP32 and stored in
 * the stack's own 16-bit type -- bf16 as it is, fp16 divided by the power of
 * two at or above max(lambda) * frame_scale[t] -- which the numerator reads
 * (half the bytes of an FP32 weighted stack); that adds one rounding to
 * each weighted value (relative 2^-8 for bf16, 2^-11 for fp16).  The general
 * numerator weighs bf16 / fp16 stacks in FP32.
 * Errors: MF_EINVAL on shape/stride/pointer problems (nothing enqueued),
 * MF_ECUDA if a launch fails. */
mf_status mf_search(const mf_stack *stack, const float *sigma, const uint8_t *mask,
                    const mf_prf_table *table, float *snr_max, int32_t *argmax,
                    float *snr_all, void *workspace, size_t workspace_bytes,
                    mf_stream stream);

/* mf_search for callers that cannot allocate device memory.  The paper has
 * no counterpart; this exists for callers such as plug-ins whose host
 * application owns every device allocation, or real-time loops that may not
 * call cudaMalloc (it can synchronise the device and stall other streams).
 * Arguments, outputs, arithmetic and errors are those of mf_search minus the
 * workspace: the scratch is a static device array of 64 MiB inside libmf,
 * which a GPU holds from the first use of the array there (with CUDA's
 * default lazy module loading: this entry point's first call on that device;
 * with eager loading: when the library loads) until the process exits.
 * A search needing more scratch than that (mf_search_workspace_size) is
 * rejected with MF_EINVAL and nothing is enqueued.  The first call on a
 * device looks the array's device address up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * address is kept for the process and does not survive cudaDeviceReset: do
 * not call this entry point after resetting the device.  All
 * calls share the one array and it keeps the previous call's contents (the
 * search clears what it needs cleared), so calls whose work overlaps on the
 * GPU (different streams, no ordering between them) race on it: serialise
 * them.  This entry point itself allocates nothing. */
mf_status mf_search_noalloc(const mf_stack *stack, const float *sigma, const uint8_t *mask,
                            const mf_prf_table *table, float *snr_max, int32_t *argmax,
                            float *snr_all, mf_stream stream);

/* Bytes of workspace mf_rescore_topk needs. */
mf_status mf_rescore_workspace_size(int64_t H, int64_t W, int32_t k_top, size_t *bytes);

/* Candidate list (Section 3.3: scores above a threshold are candidates) with
 * an FP64 re-score.  Picks the k_top pixels with the largest snr_max (ties:
 * smaller flat index y*W + x first; pixels with argmax -1 never qualify),
 * then recomputes N and D for (pixel, argmax) in FP64 from `master`, which
 * should be the FP32 residuals (bf16/fp16 are accepted and read as stored).
 * out: device mf_candidate[k_top], sorted by snr_search descending then flat
 * index; n_out: device int32, the number written (<= k_top).
 * Errors: MF_EINVAL (k_top < 1 or > H*W, shape mismatch, NULL pointers),
 * MF_EUNSUPPORTED (k_top above 16384). */
mf_status mf_rescore_topk(const mf_stack *master, const float *sigma, const uint8_t *mask,
                          const mf_prf_table *table, const float *snr_max,
                          const int32_t *argmax, int32_t k_top, mf_candidate *out,
                          int32_t *n_out, void *workspace, size_t workspace_bytes,
                          mf_stream stream);

/* The search with the residual stack in HOST memory (not in the paper):
 * the whole path a user with frames on the host runs, enqueued on `stream`
 * in order -- upload of the stack into the workspace (one 2-D copy when the
 * rows are contiguous, one per frame otherwise), mf_search, optionally
 * mf_rescore_topk (k_top > 0) from the uploaded stack, and download of the
 * results into host memory.
 *   host_stack  residuals as in mf_search, but `data` is HOST memory (pinned
 *               for asynchronous copies; pageable memory works but the copy
 *               then synchronises); frame_scale, if given, is DEVICE memory;
 *   sigma, mask DEVICE memory as in mf_search (static per field);
 *   snr_max_host float[H*W], argmax_host int32[H*W]: HOST memory;
 *   k_top       0 for no candidates, else 1..16384: cand_host
 *               mf_candidate[k_top] and n_cand_host int32, HOST memory;
 *   workspace   DEVICE memory of mf_search_host_workspace_size bytes,
 *               256-byte aligned (holds the stack copy, the maps and the
 *               search / rescore workspaces).
 *   copy_stream NULL: everything runs on `stream`.  Otherwise the upload
 *               runs on copy_stream and `stream` waits for it before the
 *               kernels, so a caller that alternates two workspaces keeps
 *               uploading the next stack while the kernels of the previous
 *               one run on `stream`;
 *   ws_free     NULL, or a CUDA event (cudaEvent_t) tied to this workspace:
 *               the upload waits for it and the call records it on `stream`
 *               once it no longer needs the workspace (after the download);
 *               pass the same event with the same workspace every time.
 * Results are valid once `stream` has reached them (synchronise it).
 * Errors: those of mf_search and mf_rescore_topk, plus MF_EINVAL for a
 * missing output or a small workspace; nothing is enqueued on MF_EINVAL. */
mf_status mf_search_host_workspace_size(const mf_stack *stack, const mf_prf_table *table,
                                        int32_t k_top, size_t *bytes);
mf_status mf_search_host(const mf_stack *host_stack, const float *sigma, const uint8_t *mask,
                         const mf_prf_table *table, float *snr_max_host, int32_t *argmax_host,
                         int32_t k_top, mf_candidate *cand_host, int32_t *n_cand_host,
                         void *workspace, size_t workspace_bytes, mf_stream stream,
                         mf_stream copy_stream, void *ws_free);

/* Score normalisation and candidate extraction (Section 3.3: each pixel's
 * score is expressed in units of the standard deviation of the scores in the
 * 255 x 255 square centred on it, and scores above 3 sigma are candidates).
 *
 * Per pixel p with a score (argmax[p] >= 0), over the window x window square
 * centred on p, clipped to the image, counting only pixels with a score: n,
 * mean and the population standard deviation sigma (FP64 sums of the scores
 * and their squares; variance = mean square - mean^2).  The normalised score
 * is z = (snr_max - mean) / sigma (subtract_mean = 1) or snr_max / sigma
 * (subtract_mean = 0, the literal reading); it is 0 where p has no score,
 * n < 2 or the window is constant (sigma^2 <= 1e-12 (mean^2 + sigma^2)).
 * Candidates are pixels with z > threshold, decided in FP64; candidates that
 * touch (8 neighbours) form one detection, reported at its largest z
 * (smallest flat index y*W + x among equal z). */
typedef struct {
    int32_t window;        /* side of the square, odd, 1..2047 (255 in the paper) */
    int32_t subtract_mean; /* 1: z = (s - mean) / sigma; 0: z = s / sigma */
    double threshold;      /* candidates: z > threshold (3 in the paper) */
} mf_detect_opts;

/* One detection (mf_detect). */
typedef struct {
    int32_t y, x;     /* peak pixel */
    int32_t k;        /* argmax trajectory at the peak */
    int32_t npix;     /* candidate pixels in the detection */
    double z;         /* normalised score at the peak (FP64) */
    double mean;      /* local mean at the peak */
    double sigma;     /* local standard deviation at the peak */
    float snr;        /* snr_max at the peak */
    int32_t reserved;
} mf_detection;

/* Bytes of workspace mf_detect needs (H * W < 2^31). */
mf_status mf_detect_workspace_size(int64_t H, int64_t W, int32_t max_out, size_t *bytes);

/* Normalise snr_max / argmax (device, H x W, as mf_search writes them) and
 * extract the detections.
 *   z_out    device float[H*W] for the normalised score, or NULL;
 *   out      device mf_detection[max_out]: the max_out detections with the
 *            largest z, ordered by z rounded to FP32 descending, then flat
 *            index ascending (max_out 0..16384; 0 only counts);
 *   n_out    device int32[2]: detections found, detections written.
 * Asynchronous on `stream`; allocates nothing.  A union-find step that runs
 * past its iteration budget records code 3 in the status word read by
 * mf_device_status and leaves that pixel's detection incomplete.
 * Errors: MF_EINVAL (NULL pointers, H or W < 1, H * W >= 2^31, window even or
 * out of range, threshold not finite, small workspace), MF_EUNSUPPORTED
 * (max_out above 16384); nothing is enqueued on an error. */
mf_status mf_detect(const float *snr_max, const int32_t *argmax, int64_t H, int64_t W,
                    const mf_detect_opts *opts, float *z_out, mf_detection *out, int32_t max_out,
                    int32_t *n_out, void *workspace, size_t workspace_bytes, mf_stream stream);

/* Per-pixel background re-fit (Section 3.1: with the low-resolution
 * scattered light S_t fixed, the model D_t = U(S_t) + B + B_theta theta_t^k
 * (Eq. 1) separates into one regression per pixel on the same six basis
 * values phi_t = (1, x_t, y_t, x_t^2, y_t^2, x_t y_t) of the jitter theta_t =
 * (x_t, y_t), under the Huber loss (Eqs. 2-4); the fit is reached by
 * least-squares solves with clipped residuals sharing one Gram inverse).
 *
 * Per pixel: y_t = D_t - U(S_t) with U bilinear from the n x n grid (pixel
 * centres aligned: row i sits at grid coordinate (i + 1/2) n / H - 1/2,
 * clamped to the grid); beta starts at the least-squares fit and takes
 * `iterations` steps beta <- beta + G^-1 sum_t phi_t psi(y_t - phi_t . beta),
 * psi(a) = min(max(a, -delta), delta), G = sum_t phi_t phi_t^T; the output
 * residual is r_t = y_t - phi_t . beta (the matched filter's input).  The
 * library applies G^-1 through an orthonormal basis Q = Phi R^-1 (G = R^T R,
 * built on the host in FP64); FP32 sums in blocks of 32 frames. */
typedef struct {
    int32_t iterations;    /* clipped steps after the least-squares start, 0..1000 */
    int32_t reserved;
    double delta;          /* Huber threshold, > 0 (data units); +inf: least squares */
} mf_refit_opts;

/* Bytes of workspace mf_background_refit needs for T frames. */
mf_status mf_refit_workspace_size(int64_t T, size_t *bytes);

/* data     device float[T][H][W], raw frames (contiguous);
 * scatter  device float[T][n][n], low-resolution scattered light, or NULL
 *          (U = 0; n ignored);
 * jitter   HOST double[T][2], (x_t, y_t) in pixels, read during the call;
 * resid    device float[T][H][W] for r, may be `data` itself (in place);
 * coef     device float[H][W][6] for (B, B_x, B_y, B_xx, B_yy, B_xy), or NULL.
 * Asynchronous on `stream` (the basis is copied from pageable host memory
 * into the workspace first); allocates nothing.
 * Errors: MF_EINVAL (NULL pointers, T < 6, H or W < 1, n < 1 with scatter,
 * non-finite jitter, delta <= 0 or NaN, iterations out of range, jitter that
 * does not determine the six coefficients (a singular Gram matrix), small
 * workspace); nothing is enqueued on an error. */
mf_status mf_background_refit(const float *data, int64_t T, int64_t H, int64_t W,
                              const float *scatter, int32_t n, const double *jitter,
                              const mf_refit_opts *opts, float *resid, float *coef,
                              void *workspace, size_t workspace_bytes, mf_stream stream);

/* Per-kernel accounting of the library's own launches (for benchmarks and
 * roofline reports; not in the paper).  Launch counts are always kept; device
 * times are recorded with CUDA events on the launching stream only while
 * profiling is enabled. */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;          /* summed device time while profiling was on */
} mf_kernel_stat;

typedef struct {
    int32_t n;          /* entries filled in k[] */
    int32_t reserved;
    int64_t launches;   /* all kernel launches counted */
    mf_kernel_stat k[16];
} mf_profile;

/* Turn event timing on (1) or off (0) for subsequent launches. */
mf_status mf_profile_enable(int32_t on);

/* Copy the counters out (waits for the recorded events); reset != 0 clears
 * them afterwards. */
mf_status mf_profile_read(mf_profile *out, int32_t reset);

/* Batched searches (not in the paper).  Many searches -- uneven cutouts,
 * each with its own stack, noise map, mask, filter bank and outputs -- run as
 * one CUDA graph: preparation kernels spread over side streams, persistent
 * numerator launches (one CTA per SM taking (search, tile, trajectory
 * group) work from a global counter: one launch per general CTA shape
 * present, and for the factored kernel one per time segment, tile width and
 * stack element type present, in segment order, each carrying at most 192
 * searches in its parameters), then per-search finalisation.  Each search's results equal those
 * of mf_search on the same inputs (same per-tile code and summation order).
 *
 * Usage: mf_batch_create; mf_batch_add per search (pointers are the caller's
 * and must stay valid while the batch is used); mf_batch_workspace_size;
 * mf_batch_prepare with a workspace of that size (builds the device
 * descriptors and a private stream: the only allocations besides the
 * handle); mf_batch_run on any stream (the first run captures the graph on
 * the batch's private stream, every run launches it on the given stream:
 * change inputs in place, not their addresses); mf_batch_destroy.
 * Errors as mf_search, plus MF_EINVAL for running an unprepared batch or
 * adding to a prepared one. */
typedef struct mf_batch mf_batch;
mf_status mf_batch_create(mf_batch **out);
mf_status mf_batch_add(mf_batch *batch, const mf_stack *stack, const float *sigma, const uint8_t *mask,
                       const mf_prf_table *table, float *snr_max, int32_t *argmax, float *snr_all,
                       int32_t *index);
mf_status mf_batch_workspace_size(const mf_batch *batch, size_t *bytes);
mf_status mf_batch_prepare(mf_batch *batch, void *workspace, size_t workspace_bytes);
mf_status mf_batch_run(mf_batch *batch, mf_stream stream);
/* Whether the work of the latest mf_batch_run has finished on the device,
 * without waiting: *done = 1 (finished, or never run) or 0 (in flight).
 * Errors: MF_EINVAL (NULL pointers), MF_ECUDA (a failed launch surfaced). */
mf_status mf_batch_poll(const mf_batch *batch, int32_t *done);
/* Number of searches, of CTA shapes present (one per general CTA shape and
 * one per factored tile width; the persistent launches of a factored shape
 * follow its time segments, element types and the 192 searches a launch
 * carries) and whether the graph has been captured. */
mf_status mf_batch_info(const mf_batch *batch, int32_t *items, int32_t *shape_groups, int32_t *graph_ready);
void mf_batch_destroy(mf_batch *batch);

/* Text of the last error on this host thread ("" if none). */
const char *mf_last_error(void);

/* Read and clear the device status word of the current device (synchronises
 * the device).  MF_OK, or MF_ETIMEOUT if a kernel's bounded wait gave up. */
mf_status mf_device_status(void);

/* The status of one search (not in the paper): enqueue on `stream` a copy
 * of the 4-byte status slot at the start of `workspace` -- the workspace
 * given to mf_search, or the one given to mf_search_host (whose search
 * workspace starts at the same address) -- into `out` (host memory, pinned
 * for an asynchronous copy, or device memory).  Once `stream` has reached
 * the copy, *out is 0 if every bounded wait of that search completed, or the
 * code of the wait that gave up (1-3 from the search kernels, 4 from
 * mf_wait_probe_search); a nonzero code means the search's maps are not
 * valid (MF_ETIMEOUT).  Enqueue it after the search on the same stream: the
 * search clears the slot when it starts.  Synchronises nothing, so a server
 * can attribute a failure to the request that met it.
 * Errors: MF_EINVAL (NULL pointers, workspace not 256-byte aligned),
 * MF_ECUDA (the copy could not be enqueued). */
mf_status mf_search_status(const void *workspace, int32_t *out, mf_stream stream);

/* Exercise the failure path of the bounded device waits (no counterpart in
 * the paper): enqueue on `stream` one CTA that waits on an mbarrier nothing
 * completes, with the same bound as every wait in the kernels (about one
 * second).  The wait gives up and records code 4 in the device status word,
 * so the next mf_device_status() returns MF_ETIMEOUT and clears it.  Nothing
 * faults, traps or hangs, and the context stays usable.  For tests of the
 * error path; searches read their own status slots, so they are unaffected. */
mf_status mf_wait_probe(mf_stream stream);

/* mf_wait_probe aimed at one search (not in the paper): the wait's code (4)
 * goes into the status slot of `workspace` (a search workspace, as for
 * mf_search_status) as well as the device status word.  Enqueued after that
 * search on the same stream, it makes the search report MF_ETIMEOUT through
 * mf_search_status, as if one of its own waits had run out; for tests of how
 * a caller handles a failed search.  Errors: MF_EINVAL (NULL or unaligned
 * workspace), MF_ECUDA. */
mf_status mf_wait_probe_search(void *workspace, mf_stream stream);

/* Library version string. */
const char *mf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MF_H */
