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
// x0 .. x0 + 8 * nch - 1 (x0 a multiple of 4) of row offset dy.
struct alignas(16) RunRec {
    int32_t dy, x0, nch, woff;  // woff: index of the first weight (multiple of 4)
};

struct Plan {
    int shape = 0;        // index into kShapes
    int vec = 2;          // width of the numerator's shared-memory loads (1, 2 or 4 floats)
    int lockstep = 0;     // numerator frame hand-off: 1 = CTA barrier per frame
    int G = 0;            // groups (CTAs per tile)
    int S = 0;            // window pitch in floats (multiple of 32, <= 256)
    int BH = 0;           // window rows (multiple of kLoadRows)
    int max_abs_shift = 0;
    double cost = 0.0;    // planner estimate, cycles per output pixel
    std::vector<int32_t> members;  // G * kt original k, or -1
    int kt() const { return kShapes[shape].kt; }
    int tile_h() const { return kTile * kShapes[shape].tys; }
    int tile_w() const { return kTile * kShapes[shape].txs; }
};

// Dynamic shared memory of the numerator kernel: windows (the key tile of the
// epilogue reuses them), frame blocks, barriers and counters, alignment slack.
inline size_t numerator_smem_bytes(int S, int BH, int kt) {
    return 1024 + (size_t)kStages * BH * S * sizeof(float) + 2 * (size_t)kRecordChunk * frame_block_bytes(kt) +
           (size_t)kStages * sizeof(uint64_t) + 3 * kStages * sizeof(int) + sizeof(int) + 64;
}

}  // namespace mf

struct mf_prf_table {
    int K = 0, T = 0;
    int device = 0;
    std::vector<int32_t> shifts;  // K*T*2, (s_x, s_y)
    std::vector<double> taps;     // K*T*25
    mf::Plan plan;
    int forced_shape = -1;  // -1: cost model
    int forced_vec = 0;     // 0: default
    int forced_lockstep = -1;
    int n_seg = 0;          // runs of the collapsed denominator kernels
    int64_t g_nnz = 0;      // nonzero weights of the collapsed kernels
    size_t device_bytes = 0;
    // device copies
    unsigned char *d_blocks = nullptr;   // [G][T] frame blocks of frame_block_bytes(kt)
    mf::FrameHdr *d_hdr = nullptr;       // [G][T]
    mf::RunRec *d_runs = nullptr;        // [n_seg]
    int32_t *d_run_off = nullptr;        // [K + 1]
    float *d_wts = nullptr;              // run weights
    double *d_taps64 = nullptr;          // [K][T][25]
    int32_t *d_shifts = nullptr;         // [K][T][2]
};

namespace mf {

struct WorkspaceLayout {
    size_t lam_off, y_off, isd_off, keys_off, total;
    int64_t pad;       // zero border of the padded lambda image
    int64_t lam_w;     // padded lambda row pitch
    int64_t lam_h;
    int64_t y_pitch;   // weighted-stack row pitch (floats, multiple of 4)
};

WorkspaceLayout search_layout(int64_t T, int64_t H, int64_t W, const mf_prf_table *tab);

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
int launch_rescore(const RescoreArgs &a, char *err, size_t errlen);

int read_device_status(int *status);

// Record an error message for mf_last_error() and return the status.
mf_status set_error(mf_status s, const char *msg);

// Launch accounting (mf_profile_*).  Kernel ids index kKernelNames.
enum KernelId { kKLambda = 0, kKWeight, kKDenominator, kKNumerator, kKFinalize, kKSelect, kKRescore,
                kKCompact, kKSort, kKernelCount };
int profile_enable(int on);
int profile_read(mf_profile *out, int reset);

}  // namespace mf
