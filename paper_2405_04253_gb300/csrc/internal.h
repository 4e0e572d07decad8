// internal.h -- device-side work descriptors shared by the kernels and the host
// side of libfnt (not part of the public C ABI).
#pragma once

#include <cstdint>

namespace fnt {

constexpr int kCdcN = 64;          // CDC transform length
constexpr int kMaxCdTaps = 31;     // |Re z|, |Im z| <= 31 * 2 * 16 * 32 < 2^15 (eq. (5), int16 out)
constexpr int kAeqK = 16;          // taps per real AEQ filter
constexpr int kBlocksPerItem = 32; // CDC blocks per warp work item (one per lane)
// CDC work item: int4 (frame, first block, blocks, polarisation); a group of 32
// blocks of an n_pol = 2 frame is two consecutive items (pol 0, pol 1).

// One frame as the kernels see it (16-byte aligned).
struct alignas(16) DevFrame {
    const int8_t *in;      // CDC / chain: int8 [n][n_pol][2]; AEQ alone: int8 [n][4]
    void *out;             // CDC: int16 [n][n_pol][2]; chain / AEQ: int16 [n_sym][4]
    int8_t *aeq_in;        // AEQ input int8 [n_sym][4] (chain: intermediate buffer)
    int32_t *state;        // AEQ master taps [4][4][K] or nullptr
    int64_t n;             // samples (CDC, chain) or symbols (AEQ alone)
    int64_t n_sym;         // AEQ symbols
    int32_t n_pol;
    int32_t L;             // CD taps
    int32_t S;             // CDC overlap-save step
    int32_t shift;         // CDC -> AEQ requantisation shift s_c
    int32_t phase;         // decimation phase
    int32_t flags;         // kFrameInjectTmaTimeout: test hook (the CDC's bulk-copy waits run out)
    int32_t *hspec;        // CDC tap spectra H_u [64], H_v [64] (cdc_spectra_kernel writes them)
    int8_t taps[64];       // [L][2] (re, im), zero beyond L
};
static_assert(sizeof(DevFrame) % 16 == 0 && sizeof(DevFrame) <= 256, "DevFrame layout");
constexpr size_t kSpecBytes = 2 * kCdcN * sizeof(int32_t);   // per frame

// One AEQ run: a whole frame, or one segment of a long frame.
struct alignas(16) AeqChain {
    int32_t frame;
    int32_t write_state;   // 1: write the final taps to the frame's state
    int64_t begin;         // first symbol the run processes
    int64_t lo;            // first symbol its windows may read as input history (zero before it)
    int64_t keep;          // first symbol whose output is stored
    int64_t end;           // one past the last symbol
    const int32_t *init;   // initial taps (frame state, a copy of it, or the plan's initial taps)
    int32_t init_copy;     // host side only: index of the state copy `init` must point to, or -1
    int32_t need_item;     // host side only: last CDC work item whose output this chain reads
};
static_assert(sizeof(AeqChain) == 64, "AeqChain layout");

struct AeqParams {
    int32_t mu_shift;
    int32_t rde_a;
    int32_t period;       // blocks per tap update, >= 1
    int32_t tensor_gradient;  // 1: gradient on the tensor cores (same results)
    int32_t freq_sum;     // 0 per pair, 1 inputs summed in Z_F, 2 summed where the bound guard holds
};

constexpr int kMaxUpdatePeriod = 64;   // keeps the summed int64 gradient exact

// DevFrame::flags
constexpr int32_t kFrameInjectTmaTimeout = 1;   // arm the CDC's window barrier without issuing its copy

// Device fault word (fnt_device_faults): bits set by kernels whose bounded waits ran out.
constexpr unsigned kFaultCdcWindowWait = 1u;

}  // namespace fnt
