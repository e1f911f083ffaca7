// Internal layouts shared by the host planner (mf_host.cpp) and the kernels
// (mf_kernels.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/mf.h"

namespace mf {

// Output tile of the numerator kernel: 32 x 32 start pixels per trajectory.
// Lane (tx, ty), tx in 0..3, ty in 0..7, owns rows 4*ty .. 4*ty+3 and columns
// 8*tx + ty .. 8*tx + ty + 7 of the tile: the column skew ty keeps the 32
// lanes on 32 distinct shared-memory banks when the window pitch is a
// multiple of 32 words.
constexpr int kTile = 32;
constexpr int kMicroRows = 4;
constexpr int kMicroCols = 8;
constexpr int kSkew = 7;             // largest column skew of a lane
constexpr int kTileOriginX = -8;     // first tile column (covers the skewed rows at x = 0)
constexpr int kWarpsPerCta = 8;      // trajectories per CTA (one warp each)
constexpr int kStages = 3;           // frame windows in flight per CTA
constexpr int kLoadRows = 8;         // rows per TMA box
constexpr int kRecFloats = 32;       // per-(trajectory, frame) record: 25 taps + offsets
constexpr int kFrameBlock = 16;      // frames per FP32 partial sum in the numerator
constexpr int kSegBlock = 4;         // segments per FP32 partial in the denominator
constexpr int kSmemBudget = 110 * 1024;  // per CTA, so that two CTAs share an SM

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
    int32_t nrows;  // rows to load, a multiple of kLoadRows
    int32_t pad;
};

// Block read by one TMA bulk copy per (group, frame): header of frame
// t + kStages (the frame the issuing warp loads next into this slot) and the
// kWarpsPerCta slot records of frame t.
struct alignas(16) FrameBlock {
    FrameHdr next;
    SlotRec slot[kWarpsPerCta];
};

// One run of frames with a constant base shift (denominator kernel).
struct alignas(16) SegRec {
    float w2[25];     // sum over the run of W^2, FP64 sum rounded to FP32
    int32_t sx, sy;
    int32_t pad[5];
};
static_assert(sizeof(SegRec) == 128, "SegRec is 128 bytes");

struct Plan {
    int G = 0;            // groups (CTAs per tile)
    int S = 0;            // window pitch in floats (multiple of 32, <= 256)
    int BH = 0;           // window rows (multiple of kLoadRows)
    int max_abs_shift = 0;
    std::vector<int32_t> members;  // G * kWarpsPerCta original k, or -1
};

}  // namespace mf

struct mf_prf_table {
    int K = 0, T = 0;
    int device = 0;
    std::vector<int32_t> shifts;  // K*T*2, (s_x, s_y)
    std::vector<double> taps;     // K*T*25
    mf::Plan plan;
    int n_seg = 0;
    // device copies
    mf::FrameBlock *d_blocks = nullptr;  // [G][T]
    mf::FrameHdr *d_hdr = nullptr;       // [G][T]
    mf::SegRec *d_segs = nullptr;        // [n_seg]
    int32_t *d_seg_off = nullptr;        // [K + 1]
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

}  // namespace mf
