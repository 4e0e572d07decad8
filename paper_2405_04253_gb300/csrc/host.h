// host.h -- host-side declarations shared by the translation units of libfnt.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <vector>

#include "fnt.h"
#include "internal.h"

struct fnt_plan {
    fnt_plan_desc d;
    int32_t h_init[16 * fnt::kAeqK];
    int32_t *d_init = nullptr;   // device copy of the initial taps
    int device = 0;
    int n_sm = 1;
    int cdc_warps = 4;
    int aeq_warps = 2;
    int chunks = 1;              // pipelined chunks of prepared chain batches (1 = off)
    int tensor_gradient = 0;     // AEQ gradient on the tensor cores (opt-in, same results)
    int cdc_pols_per_item = 0;   // CDC items: 0 auto, 1 one polarisation, 2 both
    int aeq_occupancy = 0;       // AEQ warps per SM cap (0: as many as resources allow)
    int aeq_kernel = 0;          // AEQ kernel: 0 auto, 1 a warp per chain, 2 a CTA per chain
    int cdc_kernel = 0;          // CDC kernel: 0 auto, 1 a block per lane, 2 a block per 8 threads
    int test_inject = 0;         // DevFrame::flags of the one-shot calls and batches (test hook)
    int smem_per_sm = 0;         // the device's shared memory per SM and per-CTA reserve
    int smem_reserved = 0;
    cudaMemPool_t pool = nullptr;  // per-call work memory, kept mapped between calls
};

namespace fnt {

// An NVTX range over a host-side scope (visible in Nsight Systems timelines;
// without a tool attached the calls do next to nothing).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

fnt_status fail(fnt_status st, const char *fmt, ...);
fnt_status check_device(const fnt_plan *p);   // FNT_ERR_INVALID unless the plan's device is current
fnt_status cuda_fail(cudaError_t e, const char *what);

int cdc_shift_of(const int8_t *taps, int L);
int decim_phase_of(int L);
int64_t chain_nsym(int64_t n, int phase);

// Work lists of one call or prepared batch.
struct Work {
    int op = 0;
    bool cdc_both = false;            // CDC items may cover both polarisations (item.w = 2)
    bool spectra_ready = false;       // the frames' CDC tap spectra are computed (prepared batches)
    std::vector<DevFrame> frames;
    std::vector<int4> items;          // CDC: (frame, first block, blocks)
    std::vector<AeqChain> chains;     // AEQ runs, longest first
    std::vector<int64_t> scratch_off; // chain: per-frame offset of the intermediate buffer
    std::vector<int> init_src;        // segmented frames with a state: frame whose state is copied
    std::vector<int> item_cut;        // pipelined chunks: CDC items [item_cut[k], item_cut[k+1])
    std::vector<int> chain_cut;       //                   AEQ chains [chain_cut[k], chain_cut[k+1])
    int64_t scratch_bytes = 0;
    size_t off_frames = 0, off_items = 0, off_chains = 0, off_init = 0, off_spec = 0, off_scratch = 0, total = 0;
};

constexpr size_t kStateBytes = 16 * kAeqK * sizeof(int32_t);
constexpr uint64_t kPoolKeepBytes = 1ull << 30;   // work memory a plan keeps mapped between calls

// Device-accessible address of a buffer (page-locked host memory through its
// device mapping); nullptr for pageable host memory.
void *device_view(const void *p);

// Blocks per AEQ tap update: 0 in the descriptor means every block.
inline int update_period(const fnt_plan_desc &d) { return d.aeq_update_period > 1 ? d.aeq_update_period : 1; }

fnt_status build_work(const fnt_plan *p, const fnt_frame_batch *b, int op, Work &w);
void layout(Work &w);
// Points every CDC frame's tap-spectrum slot into the allocation at dev.
void point_spectra(Work &w, char *dev);
fnt_status upload_work(Work &w, char *dev, cudaStream_t stream);
// stages: bit 0 = CDC kernel, bit 1 = AEQ kernel
fnt_status launch_work(const fnt_plan *p, const Work &w, const char *dev, cudaStream_t stream, int stages = 3);
// Chunked CDC -> AEQ with the AEQ chunks on side streams (w.item_cut / w.chain_cut).
fnt_status launch_pipelined(const fnt_plan *p, const Work &w, const char *dev, cudaStream_t stream,
                            const std::vector<cudaStream_t> &side, const std::vector<cudaEvent_t> &ev);
int work_kernel_count(const Work &w);

// kernels
constexpr int kCdcCtasPerSm = 3;     // cdc_kernel's __launch_bounds__ minimum
constexpr int kSerialCtasPerSm = 1;  // aeq_serial_kernel CTAs resident per SM (registers)
constexpr int kSerialMinBlocks = 256;  // shortest longest-chain (blocks) for which the automatic choice takes it
size_t cdc_smem_bytes(int warps);
int cdc_mults_per_block();
int cdc_butterflies_per_block();
int aeq_mults_per_block(int na);
cudaError_t cdc_configure();
cudaError_t cdc_read_faults(unsigned *faults, bool clear);   // the current device's fault word
cudaError_t cdc_spectra_launch(const DevFrame *frames, int n_frames, cudaStream_t stream);
cudaError_t cdc_launch(const DevFrame *frames, const int4 *items, int n_items, bool chain, bool both, int warps, int grid,
                       cudaStream_t stream, bool split = false);
// Whether a CDC launch of n_items 32-block items takes the split-block kernel.
bool cdc_use_split(const fnt_plan *p, int64_t n_items);
size_t aeq_smem_bytes(int na, int warps, int period);
cudaError_t aeq_configure();
cudaError_t aeq_launch(int na, const DevFrame *frames, const AeqChain *chains, int n_chains, AeqParams prm,
                       int warps, int grid, cudaStream_t stream, size_t min_smem = 0);
size_t aeq_min_smem(const fnt_plan *p);   // shared memory per AEQ CTA that enforces the occupancy cap
// The CTA-per-chain AEQ kernel (aeq_serial.cu): few long chains, latency per block.
size_t aeq_serial_smem_bytes(int na);
int aeq_serial_mults_per_block(int na);
cudaError_t aeq_serial_configure();
cudaError_t aeq_serial_launch(int na, const DevFrame *frames, const AeqChain *chains, int n_chains, AeqParams prm,
                              int grid, cudaStream_t stream);
// Whether a launch of n_chains chains, the longest of longest_symbols symbols,
// takes the CTA-per-chain kernel.
bool aeq_use_serial(const fnt_plan *p, int64_t n_chains, int64_t longest_symbols);
// Launches the AEQ kernel the plan picks for those chains.
cudaError_t aeq_launch_for(const fnt_plan *p, const DevFrame *frames, const AeqChain *chains, int n_chains,
                           int64_t longest_symbols, cudaStream_t stream);

}  // namespace fnt
