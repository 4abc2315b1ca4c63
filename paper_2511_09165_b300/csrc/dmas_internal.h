// Private declarations shared by the host plan builder (dmas_plan.cpp) and the
// CUDA side of the library (dmas_api.cu).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "dmas.h"

namespace dmas {

// Directions per CTA row ("group"): one warp of the beamform kernel per direction.
constexpr int kGroup = 8;
// Output samples per CTA along t for the scalar beamform kernel (8 per lane,
// lanes strided by one sample); the pair kernel uses 64 * pairs.
constexpr int kTimeTile = 256;
// Sample alignment of every staged window start and length (8 elements = 32 B
// of FP32, 16 B of FP16/BF16: every bulk copy starts and ends 16-byte aligned).
constexpr int kAlign = 8;
// Largest envelope FIR.
constexpr int kMaxTaps = 1023;
constexpr int kMfMaxLen = 8192;  // longest emitted signal for the matched filter
// Shared memory a beamform CTA may use for its staged windows: the scalar and
// interpolated-delay pair kernels (one buffer), and the persistent pair
// kernel's two staging buffers together (three or more CTAs per SM).
constexpr size_t kWindowSmemBudget = 96 * 1024;
constexpr size_t kPairSmemBudget = 72 * 1024;

// Host-side result of planning: everything the device needs, before upload.
struct HostPlan {
    // desc, normalised
    int N = 0, M = 0, T = 0, order = 0, delay_mode = 0, flags = 0;
    int chan_prec = 0, ng_prec = 0;
    double fs = 0.0, c = 0.0, cf_eps = 1e-30, env_fc = 5000.0;
    int L = 0;  // envelope taps (0 without DMAS_F_ENVELOPE)

    // delay table in desc order: shift[M*N], frac[M*N]
    std::vector<int32_t> shift;
    std::vector<float> frac;

    // grouping
    int n_groups = 0;
    std::vector<int32_t> gdir;  // [n_groups * kGroup], -1 = empty slot
    std::vector<int32_t> gws;   // [n_groups * N] window start relative to t0
    std::vector<int32_t> rel;   // [n_groups][N][kGroup] shift - window start
    std::vector<float> gfrac;   // [n_groups][N][kGroup] interpolation weight f
    // interpolated-delay pair kernel: byte offset, from the staged windows'
    // base, of the direction's staged sample for pixel t0 (its microphone's
    // block + 4 x rel), and the weight f twice (one packed operand)
    std::vector<int32_t> gsel;  // [n_groups][N][kGroup]
    std::vector<float> gwf2;    // [n_groups][N][kGroup][2] {f, f}

    int window = 0;      // staged samples per microphone row (multiple of kAlign)
    int mic_chunk = 0;   // microphones staged per pass
    int tile = 0;        // output samples per CTA along t
    int pairs = 0;       // pair kernel: pixel pairs per lane (tile = 64 * pairs); 0 = scalar kernel
    int n_tiles = 0;     // time tiles of `tile` samples
    int padl = 0;        // zero samples before t = 0 in the root channel rows
    int row = 0;         // root channel row length (multiple of kAlign)
    int spread = 0;      // largest (last sample read - window start) over groups, mics

    // every-order pass (dmas_beamform_orders; FP32 channels, order <= 5):
    // its time tile, staged window, microphones per stage and time tiles;
    // mo_chunk == 0 when the pass is not available for this plan
    int mo_tile = 0, mo_window = 0, mo_chunk = 0, mo_tiles = 0;
    // interpolated delays: the CTA's tile is summed in mo_halves pieces of 64
    // samples from one staged window (2 or 3 when every microphone fits one
    // stage)
    int mo_halves = 1;

    std::vector<float> taps;  // [L]
    std::vector<float> mf;    // matched filter: the emitted signal (empty: off)
};

// Validate the desc and build the host tables.  Returns DMAS_OK or DMAS_EINVAL
// with a reason in *why.
dmas_status build_host_plan(const dmas_plan_desc &d, HostPlan &hp, std::string *why);

// The pipelined pair kernel runs FP32 channels up to this order; higher orders
// (too many running sums for its registers) and FP16/BF16 channels run the
// scalar beamform kernel.
constexpr int kPairMaxOrder = 5;
// Pixel pairs per lane of the nearest-sample pair kernel: six up to order 3
// (a 384-sample tile, 80 registers, three CTAs per SM) and four above (a
// 256-sample tile, 80 registers, three CTAs per SM), for fewer staged bytes
// and table loads per output than two (128 samples, four CTAs per SM).
// Measured on B300, passive 256-microphone frame: n = 3 19.99 / 16.12 /
// 14.79 ms with two / four / six pairs; n = 5 23.35 / 21.98 / 22.15 ms;
// hemisphere frame, n = 5 460 / 454 / 458 us.  A frame with fewer than
// kWideMinItems wide work items (two per CTA at four CTAs on each of the 148
// SMs: the device not filled twice) keeps two pairs, more items, so its CTAs
// end sooner.
constexpr int round_pairs(int order) { return order <= 3 ? 6 : 4; }
// Pixel pairs per lane of the interpolated-delay pair kernel: three, a
// 192-sample tile (orders up to 3 at three CTAs per SM, 72-80 registers;
// orders 4 and 5, six running sums split plain and f-weighted, at two CTAs per
// SM, 118 registers).  Measured on B300 against two pairs (128 samples, three
// CTAs per SM at n = 5) and four (two CTAs per SM): hemisphere frame, n = 5
// 749 / 745 against 728 us; n = 1, 2, 3 0.305 / 0.535 / 0.520 against
// 0.274 / 0.496 / 0.493 ms with three.
constexpr int kLinPairs = 3;
constexpr size_t kWideMinItems = 148 * 4 * 2;

inline bool uses_pair_kernel(int chan_prec, int order) {
    return chan_prec == DMAS_CH_F32 && order <= kPairMaxOrder;
}

// Bytes of one element of the root channel for a dmas_chan_prec.
inline size_t chan_elem_bytes(int chan_prec) { return chan_prec == DMAS_CH_F32 ? 4 : 2; }

// Persistent pair kernel (nearest-sample delays): one of its two staging
// buffers holds mic_chunk FP32 window rows (padded to 128 bytes), then the
// chunk's shift table.
inline size_t pair_window_bytes(int mic_chunk, int window) {
    return ((size_t)mic_chunk * window * 4 + 127) & ~(size_t)127;
}
inline size_t pair_stage_bytes(int mic_chunk, int window) {
    return (pair_window_bytes(mic_chunk, window) + (size_t)mic_chunk * kGroup * 4 + 127) &
           ~(size_t)127;
}
// Pair kernel with interpolated delays: beside the root rows the roots kernel
// writes the raw samples as a second plane; its CTA stages, per microphone,
// one 128-byte aligned block holding the root window and then the raw-sample
// window (lin_mic_bytes), and per microphone and direction the byte offset of
// its first staged sample (int) and the weight f twice (2 floats).
inline bool uses_raw_rows(int chan_prec, int order, int delay_mode) {
    return uses_pair_kernel(chan_prec, order) && delay_mode == DMAS_DELAY_LINEAR;
}
inline size_t lin_mic_bytes(int window) { return ((size_t)2 * window * 4 + 127) & ~(size_t)127; }
// The CTA also keeps per-lane partial sums of the sample past its tile
// (8 warps x up to 6 sums x 32 lanes).
inline size_t lin_pair_smem_bytes(int mic_chunk, int window) {
    return 128 + (size_t)mic_chunk * lin_mic_bytes(window) + (size_t)mic_chunk * kGroup * 12 +
           8 * 6 * 32 * 4;
}
// Largest window one tensor copy (box dimension <= 256) stages.
constexpr int kTmaMaxBox = 256;

// Every-order pass (dmas_beamform_orders): one microphone's staged block
// (its plane rows), padded to 128 bytes; one staging buffer (mic_chunk blocks,
// the chunk's shift table and, interpolated, its {f, f} weight table); the
// CTA's dynamic shared memory: barrier slot, two staging buffers and, for
// interpolated delays, the per-lane sums of the sample past the tile.
constexpr int kOrdersMaxOrder = 5;  // highest order of the every-order pass
inline int orders_tile(bool lin) { return lin ? 64 : 128; }
inline int orders_num_sums(int nmax) { return 2 + (nmax >= 2 ? 1 : 0) + nmax * (nmax - 1) / 2; }
// staged root planes: orders floor(nmax/2)+1..nmax (the lower roots follow
// from them)
inline int orders_planes(int nmax) { return nmax >= 2 ? nmax - nmax / 2 : 1; }
inline size_t orders_mic_bytes(int nmax, int window) {
    return ((size_t)orders_planes(nmax) * window * 4 + 127) & ~(size_t)127;
}
inline size_t orders_stage_bytes(int nmax, bool lin, int mic_chunk, int window) {
    return ((size_t)mic_chunk * orders_mic_bytes(nmax, window) + (size_t)mic_chunk * kGroup * 4 +
            (lin ? (size_t)mic_chunk * kGroup * 8 : 0) + 127) & ~(size_t)127;
}
// (halves > 1: pieces of the tile from one microphone chunk, one staging
// buffer)
inline size_t orders_smem_bytes(int nmax, bool lin, int mic_chunk, int window, int halves = 1) {
    return 128 + (halves > 1 ? 1 : 2) * orders_stage_bytes(nmax, lin, mic_chunk, window) +
           (lin ? (size_t)8 * orders_num_sums(nmax) * 32 * 4 : 0);
}
// Shared memory of one every-order CTA: two per SM with interpolated delays,
// three with nearest-sample ones (the register limits).
constexpr size_t kOrdersSmemBudget = 110 * 1024;
constexpr size_t kOrdersRoundSmemBudget = 72 * 1024;

}  // namespace dmas
