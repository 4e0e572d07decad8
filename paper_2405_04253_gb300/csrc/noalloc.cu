// noalloc.cu -- a variant of the chain entry point that allocates nothing.
//
// Why it exists.  fnt_cdc_aeq_run allocates device memory for its work tables
// and for the CDC -> AEQ intermediate symbols on every call (stream-ordered
// cudaMallocAsync).  Some callers cannot do that where they process a frame: a
// latency-critical receive loop in which an allocation's possible device
// synchronisation and unbounded latency are not acceptable, or an application
// that has handed all device memory to its own allocator and does not let
// libraries allocate more.  fnt_cdc_aeq_run_noalloc does the same work for one
// frame with its scratch in a fixed array in device global memory that is part
// of the library image: every GPU that loads libfnt holds it until the process
// exits, and no call allocates.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address (cudaGetSymbolAddress), creates the events that guard
// the host copies of the work tables, and (once per process) page-locks those
// host copies (cudaHostRegister); later calls on that device reuse all of it.
// Make that first call outside any stream capture.  The call cannot itself be
// captured in a CUDA graph: it refuses a capturing stream with FNT_ERR_INVALID,
// because a captured table upload would read host memory that later calls
// reuse.  All calls on a device share the array, so calls whose work overlaps
// on the GPU race on it: issue them on one stream, or wait for one to finish
// before the next starts.  Nothing in the array needs to start at zero: each
// call rewrites the tables and the CDC stage writes every intermediate symbol
// the AEQ stage reads.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "fnt.h"
#include "host.h"
#include "internal.h"

namespace fnt {
namespace {

constexpr int64_t kMaxSamples = FNT_NOALLOC_MAX_SAMPLES;
constexpr int64_t kMaxSym = kMaxSamples / 2;
constexpr int kMaxItems = 2 * (int)((kMaxSamples / 32 + kBlocksPerItem - 1) / kBlocksPerItem);   // S >= 32, 2 pols
constexpr int kMaxChains = FNT_NOALLOC_MAX_SEGMENTS;

constexpr size_t kOffFrame = 0;
constexpr size_t kOffItems = 256;
constexpr size_t kOffChains = kOffItems + ((size_t)kMaxItems * sizeof(int4) + 255) / 256 * 256;
constexpr size_t kOffInit = kOffChains + ((size_t)kMaxChains * sizeof(AeqChain) + 255) / 256 * 256;
constexpr size_t kOffSpec = kOffInit + (kStateBytes + 255) / 256 * 256;
constexpr size_t kOffSym = kOffSpec + (kSpecBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kOffSym + (size_t)kMaxSym * 4;

constexpr int kMaxDevices = 64;

}  // namespace
}  // namespace fnt

// The scratch: frame descriptor, CDC work items, AEQ chains, a copy of the
// initial taps, the CDC tap spectra, intermediate symbols.
static __device__ __align__(256) unsigned char g_noalloc_scratch[fnt::kScratchBytes];

namespace fnt {
namespace {

std::mutex g_mu;                               // guards the host tables, the events and the address cache
char *g_dev_addr[kMaxDevices] = {nullptr};     // device address of the array, per device

// Host copies of the work tables, laid out as the array's first kOffInit bytes
// are for a call (frame at 0, CDC items at 256, AEQ chains after them), in a
// ring so that a call does not wait for the previous call's upload.  They are
// page-locked once, so each call uploads its tables with one asynchronous copy
// that never waits for the stream; before a host copy is rewritten, the event
// recorded after its last upload is waited for (four calls earlier).
constexpr int kMirrors = 4;
struct alignas(4096) Mirror {   // whole pages, for cudaHostRegister
    unsigned char bytes[kOffInit];
};
Mirror g_mirror[kMirrors];
bool g_mirror_locked = false;
cudaEvent_t g_mirror_done[kMirrors][kMaxDevices] = {};
int g_mirror_dev[kMirrors] = {-1, -1, -1, -1};   // device of the mirror's last upload
unsigned g_next = 0;

}  // namespace
}  // namespace fnt

using namespace fnt;

extern "C" fnt_status fnt_cdc_aeq_run_noalloc(const fnt_plan *p, const fnt_frame *f, void *stream_) {
    if (!p || !f) return fail(FNT_ERR_INVALID, "noalloc: null argument");
    Range trace("fnt_cdc_aeq_run_noalloc");
    fnt_status dst = check_device(p);
    if (dst != FNT_OK) return dst;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (f->n < 0) return fail(FNT_ERR_INVALID, "noalloc: n < 0");
    if (f->n > kMaxSamples)
        return fail(FNT_ERR_BOUND, "noalloc: frame of %lld samples exceeds the fixed scratch (at most %lld samples)",
                    (long long)f->n, (long long)kMaxSamples);
    if (f->n_pol != 2) return fail(FNT_ERR_INVALID, "noalloc: the chain needs n_pol = 2");
    if (f->cd_len < 1 || !f->cd_taps) return fail(FNT_ERR_INVALID, "noalloc: no CD taps");
    if (f->cd_len > kMaxCdTaps) return fail(FNT_ERR_BOUND, "noalloc: cd_len %d > %d", f->cd_len, kMaxCdTaps);
    for (int k = 0; k < 2 * f->cd_len; ++k)
        if (f->cd_taps[k] < -32 || f->cd_taps[k] > 31) return fail(FNT_ERR_INVALID, "noalloc: tap outside 6 bits");
    const int S = p->d.cdc_step ? p->d.cdc_step : kCdcN - f->cd_len + 1;
    if (S < 32 || S > kCdcN - f->cd_len + 1) return fail(FNT_ERR_BOUND, "noalloc: step %d with %d taps", S, f->cd_len);
    if (f->n > 0 && (!f->in || !f->out)) return fail(FNT_ERR_INVALID, "noalloc: null buffer");
    if (((uintptr_t)f->in % 4) || ((uintptr_t)f->out % 4) || ((uintptr_t)f->aeq_state % 4))
        return fail(FNT_ERR_INVALID, "noalloc: buffers must be 4-byte aligned");

    const int phase = decim_phase_of(f->cd_len);
    const int64_t nsym = chain_nsym(f->n, phase);
    const int64_t seg = p->d.aeq_segment;
    const int64_t n_chains = nsym == 0 ? 0 : ((seg <= 0 || seg >= nsym) ? 1 : (nsym + seg - 1) / seg);
    if (n_chains > kMaxChains)
        return fail(FNT_ERR_BOUND, "noalloc: %lld AEQ segments exceed the fixed scratch (at most %d)",
                    (long long)n_chains, kMaxChains);

    // a captured upload would read a host table that later calls rewrite
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(FNT_ERR_INVALID, "noalloc: the stream is capturing; this call cannot be captured in a graph");

    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FNT_ERR_INVALID, "noalloc: device %d not supported", dev);

    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_addr[dev]) {
        // set-up, once per device (and the page-locking once per process)
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
        for (int m = 0; m < kMirrors && e == cudaSuccess; ++m)
            if (!g_mirror_done[m][dev]) e = cudaEventCreateWithFlags(&g_mirror_done[m][dev], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaEventCreate");
        if (!g_mirror_locked) {
            e = cudaHostRegister(g_mirror, sizeof g_mirror, cudaHostRegisterPortable);
            if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaHostRegister");
            g_mirror_locked = true;
        }
        g_dev_addr[dev] = (char *)addr;
    }
    char *base = g_dev_addr[dev];
    if (f->n == 0) return FNT_OK;

    const int mi = (int)(g_next++ % kMirrors);
    if (g_mirror_dev[mi] >= 0) {
        e = cudaEventSynchronize(g_mirror_done[mi][g_mirror_dev[mi]]);   // its last upload has run
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: table buffer wait");
    }
    unsigned char *mir = g_mirror[mi].bytes;
    DevFrame &df = *(DevFrame *)(mir + kOffFrame);
    memset(&df, 0, sizeof df);
    df.in = (const int8_t *)f->in;
    df.out = f->out;
    df.aeq_in = (int8_t *)(base + kOffSym);
    df.hspec = (int32_t *)(base + kOffSpec);
    df.state = f->aeq_state;
    df.n = f->n;
    df.n_sym = nsym;
    df.n_pol = 2;
    df.L = f->cd_len;
    df.S = S;
    df.shift = cdc_shift_of(f->cd_taps, f->cd_len);
    df.phase = phase;
    memcpy(df.taps, f->cd_taps, 2 * (size_t)f->cd_len);

    int4 *items = (int4 *)(mir + kOffItems);
    const int64_t nblk = (f->n + S - 1) / S;
    int n_items = 0;
    for (int64_t b = 0; b < nblk; b += kBlocksPerItem)
        for (int pol = 0; pol < 2; ++pol)
            items[n_items++] = make_int4(0, (int)b, (int)std::min<int64_t>(kBlocksPerItem, nblk - b), pol);

    // the chains follow the items (kOffChains bounds them for the largest frame)
    const size_t off_chains = (kOffItems + (size_t)n_items * sizeof(int4) + 255) / 256 * 256;
    AeqChain *chains = (AeqChain *)(mir + off_chains);
    int nc = 0;
    if (n_chains == 1) {
        AeqChain &c = chains[nc++];
        c = AeqChain{};
        c.write_state = f->aeq_state != nullptr;
        c.end = nsym;
        c.init = f->aeq_state ? f->aeq_state : p->d_init;
        c.init_copy = -1;
    } else {
        for (int64_t k = 0; k < nsym; k += seg) {
            AeqChain &c = chains[nc++];
            c = AeqChain{};
            c.keep = k;
            c.end = std::min(nsym, k + seg);
            c.begin = std::max<int64_t>(0, k - p->d.aeq_warmup);
            c.lo = std::max<int64_t>(0, c.begin - kAeqK);   // the stream's preceding symbols
            c.write_state = (f->aeq_state != nullptr) && c.end == nsym;
            // segments start from the state as it was at the call (copied below)
            c.init = f->aeq_state ? (const int32_t *)(base + kOffInit) : p->d_init;
            c.init_copy = -1;
        }
        // segments are all equal but the last, so they need no longest-first sort
    }

    e = cudaMemcpyAsync(base, mir, off_chains + (size_t)nc * sizeof(AeqChain), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(g_mirror_done[mi][dev], stream);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: table upload");
    g_mirror_dev[mi] = dev;

    const DevFrame *frames = (const DevFrame *)(base + kOffFrame);
    const int nw = p->cdc_warps;
    e = cdc_spectra_launch(frames, 1, stream);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: tap spectra launch");
    e = cdc_launch(frames, (const int4 *)(base + kOffItems), n_items, true, false, nw,
                   std::min((n_items + nw - 1) / nw, p->n_sm * 64), stream, cdc_use_split(p, n_items));
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cdc kernel launch");
    if (nc > 0) {
        if (n_chains > 1 && f->aeq_state) {
            e = cudaMemcpyAsync(base + kOffInit, f->aeq_state, kStateBytes, cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "noalloc: copy initial taps");
        }
        int64_t longest = 0;
        for (int c = 0; c < nc; ++c) longest = std::max(longest, chains[c].end - chains[c].begin);
        e = aeq_launch_for(p, frames, (const AeqChain *)(base + off_chains), nc, longest, stream);
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: aeq kernel launch");
    }
    return FNT_OK;
}
