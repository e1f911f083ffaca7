// Internal layouts shared by the host planner (mf_host.cpp) and the kernels
// (mf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/mf.h"

namespace mf {

// Numerator CTA: kWarps warps sharing one staged frame window.  A CTA covers
// an output tile of (32 * tys) x (32 * txs) start pixels for kt trajectories;
// each warp owns one (trajectory, 32 x 32 sub-tile) pair.  In a sub-tile,
// lane (tx, ty), tx in 0..3, ty in 0..7, owns rows 4*ty .. 4*ty+3 and
// columns 8*tx + ty .. 8*tx + ty + 7: the column skew ty keeps the 32 lanes on
// 32 distinct shared-memory banks when the window pitch is a multiple of 32
// words.  The skew is the same in every tile, so tiles cover the plane.
constexpr int kTile = 32;
constexpr int kMicroRows = 4;
constexpr int kMicroCols = 8;
constexpr int kTileOriginX = -8;     // first tile column (covers the skewed rows at x = 0)
constexpr int kWarps = 16;           // warps per numerator CTA
constexpr int kStages = 3;           // frame windows in flight per CTA
constexpr int kLoadRows = 8;         // window rows are a multiple of this
constexpr int kFrameBlock = 16;      // frames per FP32 partial sum in the numerator
constexpr int kDenTaps = 256;        // denominator taps per FP32 partial before the FP64 add
constexpr int kDenCols = 256;        // denominator: start pixels per warp (one row)
// Warps of a factored-numerator CTA at most (its trajectories x sub-tiles,
// rounded up to a multiple of 4): 20 warps fit the register file at 96
// registers a thread, which holds the blocked sums of a lane's 32 outputs.
constexpr int kFacMaxWarps = 20;
constexpr int kSmemBudget = 220 * 1024;  // dynamic shared memory of one CTA per SM

// CTA shapes: trajectories per CTA x sub-tiles across x sub-tiles down = kWarps.
struct Shape {
    int kt, txs, tys;
};
constexpr Shape kShapes[] = {{16, 1, 1}, {8, 2, 1}, {4, 2, 2}, {2, 4, 2}};
constexpr int kNumShapes = 4;

// Record of one trajectory slot for one frame, 128 bytes.
struct alignas(16) SlotRec {
    float taps[25];   // W(a, b) at [(b + 2) * 5 + (a + 2)], FP32
    int32_t offy;     // window row of (row of tile origin + s_y - 2)
    int32_t offx;     // window column of (column of tile origin + s_x - 2)
    int32_t k;        // trajectory index, -1 for an unused slot
    int32_t pad[4];
};
static_assert(sizeof(SlotRec) == 128, "SlotRec is 128 bytes");

// Per (group, frame): where the shared window starts relative to the tile
// origin, and how many rows it needs.
struct alignas(16) FrameHdr {
    int32_t roy;    // min_k s_y - 2
    int32_t rox;    // floor4(min_k s_x - 2)
    int32_t nrows;  // rows the group's window needs at this frame (the kernel loads all BH)
    int32_t pad;
};

// Block read by one bulk copy per (group, frame): the header of frame
// t + kStages (the frame the issuing warp loads next into this stage) followed
// by kt slot records of frame t.
inline size_t frame_block_bytes(int kt) { return sizeof(FrameHdr) + (size_t)kt * sizeof(SlotRec); }

// Frame blocks arrive in chunks of kRecordChunk consecutive frames (one bulk
// copy per chunk, double-buffered); at least kStages frames per chunk.
constexpr int kRecordChunk = 4;

// One row of the collapsed denominator kernel G_k: weights for columns
// x0 .. x0 + 4 * nch - 1 (x0 a multiple of 4) of row offset dy.
struct alignas(16) RunRec {
    int32_t dy, x0, nch, woff;  // woff: index of the first weight (multiple of 4)
};

// Bounding box of G_k's runs: row offsets dy0 .. dy0 + rows - 1, columns x0 ..
// x0 + cols - 1 (x0 and cols multiples of 4), weights w0 .. w0 + nw - 1.  The
// staged denominator copies, per (trajectory, tile of th x kDenBoxCols start
// pixels), the lambda box those start pixels reach into shared memory.
struct alignas(16) DenBox {
    int32_t dy0, rows, x0, cols, w0, nw, pad[2];
};
constexpr int kDenBoxCols = 256;  // start pixels per row of a staged-denominator tile
constexpr int kDenOut = 8;        // start pixels per thread of the staged denominator
// Row pitch in 16-byte chunks of a staged lambda box for `cols` box columns:
// odd, so that the same chunk of 8 consecutive rows falls in 8 distinct bank
// groups.
__host__ __device__ constexpr int den_pitch(int cols) { return (kDenBoxCols + cols) / 4 | 1; }
// Box, weights and the trajectory's runs (nruns RunRec) in shared memory.
inline size_t den_box_smem(int th, int rows, int cols, int nw, int nruns) {
    return (size_t)(th + rows - 1) * den_pitch(cols) * 16 + (size_t)(nw + 4) * 4 + (size_t)nruns * 16 + 64;
}

// ------------------------------------------------ factored numerator ---
// When every footprint factors as W(a, b) = u_x(a) u_y(b) (the Gaussian PRF
// tables do: the pixel-integrated Gaussian is a product of two erf
// differences, and so is its 5 x 5 renormalisation), the numerator runs as a
// 5-tap pass along rows with u_x into a row-pass buffer H, then a 5-tap pass
// down columns of H with u_y.  Trajectories with the same v_x have the same
// s_x and u_x at every frame, so a CTA holding several of them (different
// v_y) makes the row pass once per frame for all of them.
//
// CTA: (slots per CTA) x (tile_h / 32) x (tile_w / 32) warps, each warp one
// (trajectory slot, 32 x 32 sub-tile); a lane owns 2 columns x 16 rows (five
// taps) or 1 column x 32 rows (single-tap footprints).  The staged window R of a frame is a TMA box of fac_rpitch(tile_w)
// columns (the box is as wide as the row pitch) and BH rows.
struct alignas(16) FacHdr {
    int32_t next_roy, next_rox;  // window origin of frame t + stages, relative to the tile origin
    int32_t cofs;                // row-pass column of output column 0 (0..3)
    int32_t nrows;               // row-pass rows this frame needs
    float ux[5];                 // u_x(a), a = -2..2
    float inv_nrows;             // 1 / nrows, rounded to FP32 (splits row-pass items)
    int32_t cofs8;               // the same for a window starting at a multiple of 8 columns (0..7):
                                 // 16-bit stacks, whose TMA boxes start at 16-byte boundaries
    int32_t pad;
};
static_assert(sizeof(FacHdr) == 48, "FacHdr is 48 bytes");
struct alignas(16) FacSlot {
    float uy[5];    // u_y(b), b = -2..2
    int32_t oy;     // row-pass row of (tile row 0 + s_y - 2)
    int32_t plane;  // phase planes: the plane of this slot's rounded y-phase at this frame
    int32_t pad;
};
static_assert(sizeof(FacSlot) == 32, "FacSlot is 32 bytes");
// Phase planes (the precompute-then-gather numerator of a phase-quantised
// bank): the column-pass taps of one rounded y-phase present among a CTA's
// trajectories at a frame.  A frame block then ends with `npl` of these and
// its FacHdr.pad holds how many are in use.
struct alignas(16) FacPlane {
    float uy[5];
    int32_t pad[3];
};
static_assert(sizeof(FacPlane) == 32, "FacPlane is 32 bytes");
__host__ __device__ inline size_t fac_block_bytes(int kt, int npl = 0) {
    return sizeof(FacHdr) + (size_t)kt * sizeof(FacSlot) + (size_t)npl * sizeof(FacPlane);
}
// Row-pass outputs per row: tile_w, in items of 16 (the column phase 0..3
// is applied when the row pass reads the window, so the column pass reads
// aligned columns); an item reads 24 window values from a 16-aligned start.
// Both pitches are odd multiples of 4 floats, so 8 lanes on 8 consecutive
// rows hit 8 distinct 16-byte bank groups with 128-bit accesses.
constexpr int kFacItem = 16;
__host__ __device__ constexpr int fac_hcols(int tw) { return tw; }
__host__ __device__ constexpr int fac_odd4(int n) { return (n / 4) % 2 ? n : n + 4; }
__host__ __device__ constexpr int fac_hpitch(int tw) { return fac_odd4(fac_hcols(tw)); }
__host__ __device__ constexpr int fac_rpitch(int tw) { return fac_odd4(fac_hcols(tw) + 8); }
// 16-bit weighted stacks: the window starts at a multiple of 8 columns (16
// bytes), an item reads 32 values (4 x 128 bits) from a 16-aligned start, and
// the row pitch is an odd multiple of 8 values (16 bytes) for the same
// conflict-free 128-bit accesses.
__host__ __device__ constexpr int fac_odd8(int n) { return (n / 8) % 2 ? n : n + 8; }
__host__ __device__ constexpr int fac_rpitch16(int tw) { return fac_odd8(fac_hcols(tw) + 16); }
constexpr int kFacMaxStages = 6;
// Frame records arrive in chunks of kFacRecordChunk frames (one bulk copy per
// chunk, two chunk buffers); a chunk buffer is refilled while frame t + stages
// is issued, so kFacRecordChunk >= kFacMaxStages keeps frame t's chunk intact.
constexpr int kFacRecordChunk = 8;
static_assert(kFacRecordChunk >= kFacMaxStages, "record chunks must outlive the frames in flight");
// Floats of one window stage, rounded to 128 bytes (TMA destination alignment);
// a stage of a 16-bit stack (bh x fac_rpitch16 values) is never larger.
__host__ __device__ constexpr int fac_stage_floats(int tw, int bh) { return (bh * fac_rpitch(tw) + 31) / 32 * 32; }
static_assert(2 * fac_rpitch16(32) <= 4 * fac_rpitch(32) && 2 * fac_rpitch16(64) <= 4 * fac_rpitch(64),
              "a 16-bit window fits the stage of a 32-bit one");
// Row-pass buffers: the CTA makes the row passes of two frames, meets at one
// barrier, then runs both column passes; the next pair writes the other two
// buffers, so one barrier per two frames orders writes and reuse.
constexpr int kFacHBufs = 4;
// With phase planes (npl > 0) a CTA makes two frames at a time: two
// row-pass buffers, then npl planes per frame over the window, then the
// gathers.
inline size_t fac_smem_bytes(int tw, int bh, int ns, int kt, int npl = 0) {
    return 1024 + (size_t)ns * fac_stage_floats(tw, bh) * sizeof(float) +
           (size_t)(npl > 0 ? 2 + 2 * npl : kFacHBufs) * bh * fac_hpitch(tw) * sizeof(float) +
           2 * (size_t)kFacRecordChunk * fac_block_bytes(kt, npl) +
           (size_t)ns * (sizeof(uint64_t) + sizeof(int)) + sizeof(int) + 64;
}

constexpr int kFacMaxSegments = 16;

struct Plan {
    int kernel = 1;       // 1: general 5 x 5 numerator, 2: factored numerator
    int f_kt = 0, f_th = 0, f_tw = 0, f_ns = 0, f_bh = 0;  // factored numerator geometry
    // factored numerator time segments: frames seg_t0[j] .. seg_t0[j + 1] - 1
    // (starts are multiples of kFacRecordChunk); per (group, segment) the
    // smallest s_y of the members at the segment's first frame and the
    // members' spread there; per (group, segment, slot) that member's s_y
    int f_seg = 1;
    int f_taps = 5;      // factored footprint taps per axis: 5, or 1 (single centre tap)
    int f_planes = 0;    // phase planes per frame (precompute-then-gather numerator), 0: column passes
    std::vector<int32_t> seg_t0;      // f_seg + 1
    std::vector<int32_t> seg_qy;      // G * f_seg * 2: (min s_y, spread)
    std::vector<int32_t> seg_ref;     // G * f_seg * kt, INT32_MIN for an empty slot
    int shape = 0;        // index into kShapes
    int vec = 2;          // width of the numerator's shared-memory loads (1, 2 or 4 floats)
    int lockstep = 0;     // numerator frame hand-off: 1 = CTA barrier per frame
    int G = 0;            // groups (CTAs per tile)
    int S = 0;            // window pitch in floats (multiple of 32, <= 256)
    int BH = 0;           // window rows (multiple of kLoadRows)
    int max_abs_shift = 0;
    double cost = 0.0;    // planner estimate, cycles per output pixel
    std::vector<int32_t> members;  // G * kt original k, or -1
    int kt() const { return kernel == 2 ? f_kt : kShapes[shape].kt; }
    int tile_h() const { return kernel == 2 ? f_th : kTile * kShapes[shape].tys; }
    int tile_w() const { return kernel == 2 ? f_tw : kTile * kShapes[shape].txs; }
    int warps() const { return kernel == 2 ? f_kt * (f_th / 32) * (f_tw / 32) : kWarps; }
    // warps launched: the factored kernel rounds up to a multiple of 4 so
    // that each SM scheduler has as many warps; the extra warps make row-pass
    // items only
    int launch_warps() const { return kernel == 2 ? (warps() + 3) / 4 * 4 : kWarps; }
    size_t smem() const;
};

// Dynamic shared memory of the numerator kernel: windows (the key tile of the
// epilogue reuses them), frame blocks, barriers and counters, alignment slack.
inline size_t numerator_smem_bytes(int S, int BH, int kt) {
    return 1024 + (size_t)kStages * BH * S * sizeof(float) + 2 * (size_t)kRecordChunk * frame_block_bytes(kt) +
           (size_t)kStages * sizeof(uint64_t) + 3 * kStages * sizeof(int) + sizeof(int) + 64;
}

inline size_t Plan::smem() const {
    return kernel == 2 ? fac_smem_bytes(f_tw, f_bh, f_ns, f_kt, f_planes) : numerator_smem_bytes(S, BH, kt());
}

}  // namespace mf

struct mf_prf_table {
    int K = 0, T = 0;
    int device = 0;
    std::vector<int32_t> shifts;  // K*T*2, (s_x, s_y)
    std::vector<double> taps;     // K*T*25
    // factors of separable footprints, W(a, b) = fx(a) fy(b) (empty when the
    // table was given as explicit footprints), and the velocities that group
    // trajectories sharing the row pass
    std::vector<double> fx, fy;   // K*T*5
    std::vector<double> vx, vy;   // K
    mf::Plan plan;
    int forced_segments = 0;  // factored time segments, 0: automatic
    int forced_kernel = 0;  // 0: automatic, 1: general, 2: factored, 3: factored with phase planes
    int phase_steps = 0;    // Q of a phase-quantised bank (0: exact phases)
    int forced_group = 0, forced_th = 0, forced_tw = 0, forced_stages = 0;  // factored geometry, 0: automatic
    int forced_shape = -1;  // -1: cost model
    int forced_vec = 0;     // 0: default
    int forced_lockstep = -1;
    int n_seg = 0;          // runs of the collapsed denominator kernels
    int64_t g_nnz = 0;      // nonzero weights of the collapsed kernels
    size_t device_bytes = 0;
    // device copies
    void *d_mem = nullptr;               // one device block holding every array below
    bool d_mem_pooled = false;           // allocated with cudaMallocAsync
    unsigned char *d_blocks = nullptr;   // [G][T] frame blocks (frame_block_bytes or fac_block_bytes)
    int32_t *d_members = nullptr;        // [G][kt] trajectory of each slot, -1 for none
    int32_t *d_segs = nullptr;           // factored: [G][S] (first frame, last frame + 1, min s_y, spread)
    int32_t *d_refs = nullptr;           // factored: [G][S][kt] s_y of each slot at the segment's first frame
    mf::FrameHdr *d_hdr = nullptr;       // [G][T]
    mf::RunRec *d_runs = nullptr;        // [n_seg]
    mf::DenBox *d_boxes = nullptr;       // [K] staged denominator: G_k's bounding box
    int den_th = 0;                      // staged denominator tile rows (0: the unstaged kernel)
    size_t den_smem = 0;                 // its dynamic shared memory
    int32_t *d_run_off = nullptr;        // [K + 1]
    float *d_wts = nullptr;              // run weights
    double *d_taps64 = nullptr;          // [K][T][25]
    int32_t *d_shifts = nullptr;         // [K][T][2]
};

namespace mf {

// The first 256 bytes of a search workspace hold the search's status slot:
// 0, or the code of a bounded wait of that search that gave up (its kernels
// write and read this slot only, so a failure stays with its own search).
// The weighted stack y is FP32, or 16-bit (the stack's own type) when the
// stack is bf16 / fp16 and the factored numerator reads it; y_t = beta_t *
// stored value, beta [T] FP32 (bf16: 1; fp16: a power of two per frame).
// Bytes 8..11 of the status area hold the largest lambda (fp16 scales).
struct WorkspaceLayout {
    size_t status_off, lam_off, y_off, beta_off, isd_off, keys_off, planes_off, total;
    int ybytes;        // 4 or 2
    int64_t pad;       // zero border of the padded lambda image
    int64_t lam_w;     // padded lambda row pitch
    int64_t lam_h;
    int64_t y_pitch;   // weighted-stack row pitch (floats, multiple of 4)
};

WorkspaceLayout search_layout(int64_t T, int64_t H, int64_t W, int32_t dtype, const mf_prf_table *tab);

struct SearchArgs {
    const mf_stack *stack;
    const float *sigma;
    const uint8_t *mask;
    const mf_prf_table *tab;
    float *snr_max;
    int32_t *argmax;
    float *snr_all;
    char *ws;
    WorkspaceLayout L;
    void *stream;
};

// Launch the whole search; returns a CUDA error code (0 on success) and
// writes a message into err on failure.
int launch_search(const SearchArgs &a, char *err, size_t errlen);

// Batched searches: device descriptors for a fixed list of searches (built
// once), and the enqueue of all of them on a stream (side streams fork and
// join inside; capturable into a CUDA graph).
struct BatchDevice;
int batch_build(const SearchArgs *items, int n, BatchDevice **out, char *err, size_t errlen);
int batch_enqueue(BatchDevice *b, const SearchArgs *items, int n, void *stream, char *err, size_t errlen);
void batch_free(BatchDevice *b);

struct RescoreArgs {
    const mf_stack *stack;
    const float *sigma;
    const uint8_t *mask;
    const mf_prf_table *tab;
    const float *snr_max;
    const int32_t *argmax;
    int32_t k_top;
    mf_candidate *out;
    int32_t *n_out;
    char *ws;
    size_t ws_bytes;
    void *stream;
};
size_t rescore_workspace(int64_t H, int64_t W, int32_t k_top);

// Top-k selection by a float score (mf_kernels.cu): among pixels with
// valid[i] >= 0, the k_top largest keys (order-preserving score bits << 32 |
// (0xFFFFFFFF - i)), i.e. score descending then index ascending, sorted
// descending into the `top` slice of the workspace.  P < 2^32, k_top <=
// kMaxTop.
constexpr int kMaxTop = 16384;
struct SelState {
    unsigned long long prefix;  // selected high bits so far
    unsigned long long thresh;  // final k_top-th largest key (0: take every valid key)
    unsigned int need;          // keys still to take at and below the current prefix
    unsigned int total;         // valid keys
    unsigned int count;         // compacted keys
    unsigned int pad;
};
struct SelectLayout {
    size_t keys_off, hist_off, st_off, top_off, total;
};
SelectLayout select_layout(int64_t P, int32_t k_top);
int launch_select(const float *score, const int32_t *valid, int64_t P, int32_t k_top, char *ws,
                  const SelectLayout &L, void *stream, char *err, size_t errlen);
int launch_rescore(const RescoreArgs &a, char *err, size_t errlen);

// Score normalisation and candidate extraction (mf_detect.cu).
struct DetectArgs {
    const float *snr_max;
    const int32_t *argmax;
    int64_t H, W;
    int32_t window, subtract_mean;
    double threshold;
    float *z_out;
    mf_detection *out;
    int32_t max_out;
    int32_t *n_out;
    char *ws;
    size_t ws_bytes;
    void *stream;
};
size_t detect_workspace(int64_t H, int64_t W, int32_t max_out);
int launch_detect(const DetectArgs &a, char *err, size_t errlen);

// Per-pixel background re-fit (mf_background.cu).  The workspace holds the
// orthonormal basis Q [T][8] (six values, two pad), R^-1 (6 x 6, row-major,
// FP64) and Q^T 1 (6 doubles), uploaded by the host.
struct RefitArgs {
    const float *data;
    int64_t T, H, W;
    const float *scatter;
    int32_t n, iterations;
    float delta;
    float *resid, *coef;
    char *ws;
    void *stream;
};
constexpr int kRefitBasisPitch = 8;
size_t refit_workspace(int64_t T);
// Offsets of the basis pieces in the workspace.
size_t refit_q_off();
size_t refit_rinv_off(int64_t T);
size_t refit_q1_off(int64_t T);
int launch_refit(const RefitArgs &a, char *err, size_t errlen);

int read_device_status(int *status);
// Status code a wait probe records (the kernels' waits use 1 to 3).
constexpr int kWaitProbeCode = 4;
// slot: a search's status slot to record the probe's code in as well, or null.
int launch_wait_probe(void *stream, int *slot, char *err, size_t errlen);

// Device address of the status word that bounded waits write on giving up.
int *status_word(char *err, size_t errlen);

// Factored numerator (mf_factored.cu).  The tensor map covers the weighted
// stack y [T][H][y_pitch] with a box of fac_rpitch(tile_w) x f_bh x 1.
struct FacParams {
    const unsigned char *blocks;  // [G][T] blocks of fac_block_bytes(kt)
    const FrameHdr *hdr;          // [G][T] window origins (pad = column phase)
    const int32_t *members;       // [G][kt] trajectory of each slot, -1 for none
    const int32_t *segs;          // [G][S][4] first frame, end frame, min s_y, spread
    const int32_t *refs;          // [G][S][kt] s_y of each slot at the segment's first frame
    float *plane;                 // [K][H][W] numerator: segment 0 stores, later segments add
    int *status;                  // the search's status slot
    const float *beta;            // [T] scale of a 16-bit weighted stack, or null (1)
    int T, G, kt, th, bh, ns, S, K;
    int npl;                      // phase planes per frame block (0: column passes)
    int seg;                      // the segment this launch computes
    int warps;                    // warps of the layout (a batched launch may have more)
    int64_t H, W;
    int tiles_x;
};
// SNR with 1 / sqrt(D) from the numerator plane, per-pixel max over k
// (smallest k on ties) and the optional SNR cube.
// The search's status slot is copied into the device-wide status word (first
// failure wins) by the finalisation.
int fac_finalize_enqueue(const float *plane, const float *isd, int K, int64_t P, float *snr_max, int32_t *argmax,
                         float *snr_all, const int *slot, int *global_status, void *stream, char *err,
                         size_t errlen);
// CTAs of segment `seg` of a factored search: groups x tile columns x tile
// rows ceil((H + spread) / tile_h), spread the widest of the segment's groups.
long long fac_ctas(const mf_prf_table &tab, int64_t H, int64_t W, int seg);
struct FacBatchItem {
    FacParams p;
    long long cta_begin;  // first entry of this search in the batch's work list
};
// A persistent launch's searches, passed by value in the launch's parameter
// space (where the one-launch kernel finds its FacParams), at most
// kFacBatchArgItems per launch.
constexpr int kFacBatchArgItems = 192;
struct FacBatchArgs {
    FacBatchItem items[kFacBatchArgItems];
    long long total;  // work entries of the launch
    int n_items;
};
static_assert(sizeof(FacBatchArgs) <= 32000, "within the 32 KB of kernel parameters");
// Shared-memory limit of the persistent kernel (set once, outside capture).
// etype: element type of the weighted stack, an mf_dtype (MF_F32, MF_BF16, MF_F16).
int fac_batch_attr(int tw, int etype, size_t smem, char *err, size_t errlen);
// items: host array of n_items (1 .. kFacBatchArgItems) searches, copied
// into the launch's parameters.
int fac_batch_enqueue(const void *maps, const FacBatchItem *items, int n_items, long long total,
                      unsigned long long *counter, int tw, int etype, int warps, size_t smem, int grid, void *stream,
                      char *err, size_t errlen);
// taps: 5, or 1 when every footprint is a single centre tap (the shift-stack
// filter), which runs the row and column passes on the centre tap only.
int fac_enqueue(const void *tensor_map, const FacParams &p, int tw, int taps, int etype, int warps, size_t smem,
                long long nblocks, void *stream, char *err, size_t errlen);

// Record an error message for mf_last_error() and return the status.
mf_status set_error(mf_status s, const char *msg);

// Launch accounting (mf_profile_*).  Kernel ids index kKernelNames.
enum KernelId { kKLambda = 0, kKWeight, kKDenominator, kKNumerator, kKFinalize, kKSelect, kKRescore,
                kKCompact, kKSort, kKDetStats, kKDetComponents, kKDetEmit, kKRefit, kKernelCount };
int profile_enable(int on);
// Bracket a launch made in another translation unit: prof_begin before it,
// prof_end after it.
struct ProfToken {
    void *scope;
};
ProfToken prof_begin(int kid, void *stream);
void prof_end(const ProfToken &t);
int profile_read(mf_profile *out, int reset);

}  // namespace mf
