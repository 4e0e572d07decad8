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
// array's device address (cudaGetSymbolAddress) and keeps it for later calls on
// that device; make that first call before any stream capture.  All calls on a
// device share the array, so calls whose work overlaps on the GPU race on it:
// issue them on one stream, or wait for one to finish before the next starts.
// Nothing in the array needs to start at zero: each call rewrites the tables and
// the CDC stage writes every intermediate symbol the AEQ stage reads.
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

std::mutex g_mu;                               // guards the host staging and the address cache
char *g_dev_addr[kMaxDevices] = {nullptr};     // device address of the array, per device
DevFrame g_frame;                              // host staging of the tables (no heap use)
int4 g_items[kMaxItems];
AeqChain g_chains[kMaxChains];

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

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(FNT_ERR_INVALID, "noalloc: device %d not supported", dev);

    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_addr[dev]) {
        void *addr = nullptr;
        e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: cudaGetSymbolAddress");
        g_dev_addr[dev] = (char *)addr;
    }
    char *base = g_dev_addr[dev];
    if (f->n == 0) return FNT_OK;

    DevFrame &df = g_frame;
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

    const int64_t nblk = (f->n + S - 1) / S;
    int n_items = 0;
    for (int64_t b = 0; b < nblk; b += kBlocksPerItem)
        for (int pol = 0; pol < 2; ++pol)
            g_items[n_items++] = make_int4(0, (int)b, (int)std::min<int64_t>(kBlocksPerItem, nblk - b), pol);

    int nc = 0;
    if (n_chains == 1) {
        AeqChain &c = g_chains[nc++];
        c = AeqChain{};
        c.write_state = f->aeq_state != nullptr;
        c.end = nsym;
        c.init = f->aeq_state ? f->aeq_state : p->d_init;
        c.init_copy = -1;
    } else {
        for (int64_t k = 0; k < nsym; k += seg) {
            AeqChain &c = g_chains[nc++];
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

    e = cudaMemcpyAsync(base + kOffFrame, &df, sizeof df, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + kOffItems, g_items, (size_t)n_items * sizeof(int4), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess && nc > 0)
        e = cudaMemcpyAsync(base + kOffChains, g_chains, (size_t)nc * sizeof(AeqChain), cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: table upload");

    const DevFrame *frames = (const DevFrame *)(base + kOffFrame);
    const int nw = p->cdc_warps;
    e = cdc_spectra_launch(frames, 1, stream);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: tap spectra launch");
    e = cdc_launch(frames, (const int4 *)(base + kOffItems), n_items, true, false, nw,
                   std::min((n_items + nw - 1) / nw, p->n_sm * 64), stream);
    if (e != cudaSuccess) return cuda_fail(e, "noalloc: cdc kernel launch");
    if (nc > 0) {
        if (n_chains > 1 && f->aeq_state) {
            e = cudaMemcpyAsync(base + kOffInit, f->aeq_state, kStateBytes, cudaMemcpyDeviceToDevice, stream);
            if (e != cudaSuccess) return cuda_fail(e, "noalloc: copy initial taps");
        }
        e = aeq_launch_for(p, frames, (const AeqChain *)(base + kOffChains), nc, stream);
        if (e != cudaSuccess) return cuda_fail(e, "noalloc: aeq kernel launch");
    }
    return FNT_OK;
}
