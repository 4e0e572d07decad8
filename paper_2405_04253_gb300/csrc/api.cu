// api.cu -- host side of libfnt: plans, frame validation, work lists, batch
// execution and the C ABI entry points declared in include/fnt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "fnt.h"
#include "host.h"
#include "internal.h"

namespace fnt {

// ------------------------------------------------------------------ errors ---

static thread_local std::string t_err;

fnt_status fail(fnt_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

fnt_status cuda_fail(cudaError_t e, const char *what) {
    return fail(FNT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ------------------------------------------------------------ field checks ---

static constexpr int64_t kF = 65537;   // F_4 = 2^16 + 1

static int64_t hmod(int64_t v) { return ((v % kF) + kF) % kF; }

static int64_t hpow(int64_t a, int64_t e) {
    int64_t r = 1, b = hmod(a);
    while (e > 0) {
        if (e & 1) r = r * b % kF;
        b = b * b % kF;
        e >>= 1;
    }
    return r;
}

// eq. (4) for the prime F = 65537, plus order exactly N and N invertible.
static bool valid_transform(int64_t N, int64_t alpha) {
    if (N < 2 || hmod(alpha) == 0) return false;
    if (hpow(alpha, N) != 1) return false;
    for (int64_t d = 1; d < N; ++d)
        if (N % d == 0 && hpow(alpha, d) == 1) return false;
    return hmod(N) != 0;
}

// CDC -> AEQ requantisation shift: the smallest s with 2^(2s) >= 2 E, E the
// taps' energy.  CD taps have an in-band gain near sqrt(2 E) on a signal that
// fills about half of the sampled band, so the 5-bit AEQ input keeps at most
// the 5-bit CDC input's loading and does not saturate.
int cdc_shift_of(const int8_t *taps, int L) {
    int64_t E = 0;
    for (int k = 0; k < L; ++k) E += (int64_t)taps[2 * k] * taps[2 * k] + (int64_t)taps[2 * k + 1] * taps[2 * k + 1];
    int s = 0;
    while (E > 0 && (int64_t{1} << (2 * s)) < 2 * E) ++s;
    return s;
}

int decim_phase_of(int L) { return ((L - 1) / 2) & 1; }

int64_t chain_nsym(int64_t n, int phase) { return n > phase ? (n - phase + 1) / 2 : 0; }

}  // namespace fnt

using namespace fnt;

// --------------------------------------------------------------------- ABI ---

extern "C" size_t fnt_last_error(char *buf, size_t len) {
    if (buf && len) {
        size_t m = std::min(len - 1, t_err.size());
        memcpy(buf, t_err.data(), m);
        buf[m] = 0;
    }
    return t_err.size();
}

extern "C" const char *fnt_version(void) { return "fnt 1.0 sm_103a"; }

extern "C" void fnt_plan_desc_default(fnt_plan_desc *d) {
    if (!d) return;
    memset(d, 0, sizeof *d);
    d->n_cdc = 64;
    d->alpha_cdc = 4080;
    d->cdc_step = 0;
    d->n_aeq = 32;
    d->alpha_aeq = 2;
    d->aeq_taps = 16;
    d->mu_shift = 10;
    d->rde_a = 64;
    d->tap_init = 2048;
    d->aeq_segment = 0;
    d->aeq_warmup = 0;
    d->aeq_update_period = 0;
    d->aeq_freq_sum = 0;
}

// Kernel attributes (the dynamic shared memory limits) are per device: set them
// once on every device a plan is created on.
static std::mutex g_config_mu;
static std::set<int> g_configured;

static fnt_status configure_kernels(int device) {
    std::lock_guard<std::mutex> lk(g_config_mu);
    if (g_configured.count(device)) return FNT_OK;
    cudaError_t e = cdc_configure();
    if (e != cudaSuccess) return cuda_fail(e, "cdc_configure");
    e = aeq_configure();
    if (e != cudaSuccess) return cuda_fail(e, "aeq_configure");
    e = aeq_serial_configure();
    if (e != cudaSuccess) return cuda_fail(e, "aeq_serial_configure");
    g_configured.insert(device);
    return FNT_OK;
}

// The calls of a plan run on the plan's device, which must be current.
fnt_status fnt::check_device(const fnt_plan *p) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) return fail(FNT_ERR_INVALID, "the plan was created on device %d, device %d is current",
                                      p->device, dev);
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_create(const fnt_plan_desc *d, fnt_plan **out) {
    if (!d || !out) return fail(FNT_ERR_INVALID, "plan_create: null argument");
    *out = nullptr;
    if (!valid_transform(d->n_cdc, d->alpha_cdc))
        return fail(FNT_ERR_BOUND, "CDC: alpha=%d is not of order N=%d mod 65537 (eq. (4))", d->alpha_cdc, d->n_cdc);
    if (!valid_transform(d->n_aeq, d->alpha_aeq))
        return fail(FNT_ERR_BOUND, "AEQ: alpha=%d is not of order N=%d mod 65537 (eq. (4))", d->alpha_aeq, d->n_aeq);
    if (d->n_cdc != 64 || d->alpha_cdc != 4080)
        return fail(FNT_ERR_INVALID, "CDC: only N=64 with alpha=4080 is compiled");
    if (!((d->n_aeq == 32 && d->alpha_aeq == 2) || (d->n_aeq == 64 && d->alpha_aeq == 4080)))
        return fail(FNT_ERR_INVALID, "AEQ: only (N=32, alpha=2) and (N=64, alpha=4080) are compiled");
    if (d->aeq_taps != kAeqK) return fail(FNT_ERR_INVALID, "AEQ: aeq_taps must be %d", kAeqK);
    if (d->cdc_step != 0 && (d->cdc_step < 32 || d->cdc_step > 64))
        return fail(FNT_ERR_INVALID, "CDC: cdc_step must be 0 or in [32, 64]");
    if (d->mu_shift < 0 || d->mu_shift > 63) return fail(FNT_ERR_INVALID, "mu_shift must be in [0, 63]");
    if (d->rde_a < 1 || d->rde_a > 4096) return fail(FNT_ERR_INVALID, "rde_a must be in [1, 4096]");
    if (d->tap_init < -8192 || d->tap_init > 8191) return fail(FNT_ERR_INVALID, "tap_init must be a 14-bit tap");
    if (d->aeq_segment < 0 || d->aeq_warmup < 0) return fail(FNT_ERR_INVALID, "negative AEQ segment/warmup");
    if (d->aeq_update_period < 0 || d->aeq_update_period > kMaxUpdatePeriod)
        return fail(FNT_ERR_INVALID, "aeq_update_period must be in [0, %d]", kMaxUpdatePeriod);
    if (d->aeq_freq_sum < 0 || d->aeq_freq_sum > 2) return fail(FNT_ERR_INVALID, "aeq_freq_sum must be 0, 1 or 2");
    int device = 0;
    cudaError_t e = cudaGetDevice(&device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    fnt_status st = configure_kernels(device);
    if (st != FNT_OK) return st;

    fnt_plan *p = new (std::nothrow) fnt_plan();
    if (!p) return fail(FNT_ERR_NOMEM, "plan_create: out of host memory");
    p->d = *d;
    p->device = device;
    cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device);
    cudaDeviceGetAttribute(&p->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
    cudaDeviceGetAttribute(&p->smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, p->device);
    int32_t init[16 * kAeqK] = {0};
    for (int s = 0; s < 4; ++s) init[(s * 4 + s) * kAeqK + kAeqK / 2] = (int32_t)((int64_t)d->tap_init * 65536);
    memcpy(p->h_init, init, sizeof init);
    e = cudaMalloc(&p->d_init, sizeof init);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaMalloc(init taps)");
    }
    e = cudaMemcpy(p->d_init, init, sizeof init, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->d_init);
        delete p;
        return cuda_fail(e, "cudaMemcpy(init taps)");
    }
    // the per-call work memory comes from a pool of the plan's own that keeps
    // up to kPoolKeepBytes mapped between calls (the device's default pool
    // returns freed memory to the system at every synchronisation)
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = p->device;
    e = cudaMemPoolCreate(&p->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = kPoolKeepBytes;
        e = cudaMemPoolSetAttribute(p->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e != cudaSuccess) {
        if (p->pool) cudaMemPoolDestroy(p->pool);
        cudaFree(p->d_init);
        delete p;
        return cuda_fail(e, "cudaMemPoolCreate");
    }
    *out = p;
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_destroy(fnt_plan *p) {
    if (!p) return FNT_OK;
    cudaDeviceSynchronize();             // calls still in flight hold pool memory
    cudaMemPoolDestroy(p->pool);
    cudaFree(p->d_init);
    delete p;
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_launch(fnt_plan *p, int32_t cdc_warps, int32_t aeq_warps) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (cdc_warps < 0 || cdc_warps > 4 || aeq_warps < 0 || aeq_warps > 4)
        return fail(FNT_ERR_INVALID, "warps per CTA must be in [1, 4]");
    if (cdc_warps) p->cdc_warps = cdc_warps;
    if (aeq_warps) p->aeq_warps = aeq_warps;
    return FNT_OK;
}

extern "C" fnt_status fnt_op_counts_for(const fnt_plan_desc *d, int32_t cd_len, fnt_op_counts *out) {
    if (!d || !out) return fail(FNT_ERR_INVALID, "null argument");
    if (cd_len < 1 || cd_len > kMaxCdTaps) return fail(FNT_ERR_BOUND, "cd_len %d outside 1..%d", cd_len, kMaxCdTaps);
    if (d->n_cdc != kCdcN || (d->n_aeq != 32 && d->n_aeq != 64) || d->aeq_taps != kAeqK)
        return fail(FNT_ERR_INVALID, "unsupported transform lengths");
    const int S = d->cdc_step ? d->cdc_step : kCdcN - cd_len + 1;
    if (S < 32 || S > kCdcN - cd_len + 1) return fail(FNT_ERR_BOUND, "step %d with %d taps", S, cd_len);
    const double sym_per_block = S / 2.0;                  // 2 samples per symbol
    out->cdc_mults_per_symbol = cdc_mults_per_block() / sym_per_block;
    out->cdc_butterflies_per_symbol = cdc_butterflies_per_block() / sym_per_block;
    out->aeq_mults_per_symbol = (double)aeq_mults_per_block(d->n_aeq) / (d->n_aeq - kAeqK);
    out->aeq_cta_mults_per_symbol = (double)aeq_serial_mults_per_block(d->n_aeq) / (d->n_aeq - kAeqK);
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_pipeline(fnt_plan *p, int32_t chunks) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (chunks < 1 || chunks > 16) return fail(FNT_ERR_INVALID, "chunks must be in [1, 16]");
    p->chunks = chunks;
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_aeq_occupancy(fnt_plan *p, int32_t max_warps_per_sm) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (max_warps_per_sm < 0 || max_warps_per_sm > 64)
        return fail(FNT_ERR_INVALID, "AEQ warps per SM must be in [0, 64]");
    p->aeq_occupancy = max_warps_per_sm;
    return FNT_OK;
}

size_t fnt::aeq_min_smem(const fnt_plan *p) {
    if (p->aeq_occupancy <= 0 || p->smem_per_sm <= 0) return 0;
    const int ctas = std::max(1, p->aeq_occupancy / p->aeq_warps);
    const int per_cta = p->smem_per_sm / ctas - p->smem_reserved;
    return per_cta > 0 ? (size_t)per_cta : 0;
}

extern "C" fnt_status fnt_plan_set_aeq_kernel(fnt_plan *p, int32_t kind) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (kind < 0 || kind > 2) return fail(FNT_ERR_INVALID, "AEQ kernel must be 0 (auto), 1 or 2");
    p->aeq_kernel = kind;
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_cdc_kernel(fnt_plan *p, int32_t kind) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (kind < 0 || kind > 2) return fail(FNT_ERR_INVALID, "CDC kernel must be 0 (auto), 1 or 2");
    p->cdc_kernel = kind;
    return FNT_OK;
}

// One block per lane needs many blocks to fill the GPU; with fewer work items
// than two per SM, a block per 8 threads (8 warps per item) is taken instead.
bool fnt::cdc_use_split(const fnt_plan *p, int64_t n_items) {
    if (p->cdc_kernel != 0) return p->cdc_kernel == 2;
    return n_items < 2 * (int64_t)p->n_sm;
}

extern "C" fnt_status fnt_plan_set_test_inject(fnt_plan *p, int32_t mode) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (mode != 0 && mode != 1) return fail(FNT_ERR_INVALID, "test inject mode must be 0 or 1");
    p->test_inject = mode;
    return FNT_OK;
}

extern "C" fnt_status fnt_device_faults(int32_t clear, uint32_t *faults) {
    if (!faults) return fail(FNT_ERR_INVALID, "null argument");
    unsigned v = 0;
    cudaError_t e = cdc_read_faults(&v, clear != 0);
    if (e != cudaSuccess) return cuda_fail(e, "fnt_device_faults");
    *faults = v;
    return FNT_OK;
}

extern "C" int32_t fnt_plan_cdc_kernel_for(const fnt_plan *p, int64_t n_items) {
    if (!p) return 0;
    return cdc_use_split(p, n_items) ? 2 : 1;
}

extern "C" int32_t fnt_plan_aeq_kernel_for(const fnt_plan *p, int64_t n_chains, int64_t longest_symbols) {
    if (!p) return 0;
    return aeq_use_serial(p, n_chains, longest_symbols) ? 2 : 1;
}

// The CTA-per-chain kernel holds one (chain, polarisation) per SM.  It is taken
// when that many fit in one wave and the longest chain is long enough for its
// shorter block time to matter (short chains, such as the segments of a
// served frame, finish sooner in the warp kernel once several launches share
// the GPU, since each CTA holds a whole SM), and only for per-pair inverse
// transforms.
bool fnt::aeq_use_serial(const fnt_plan *p, int64_t n_chains, int64_t longest_symbols) {
    if (p->d.aeq_freq_sum != 0 || p->aeq_kernel == 1) return false;
    if (p->aeq_kernel == 2) return true;
    const int64_t blocks = (longest_symbols + (p->d.n_aeq - kAeqK) - 1) / (p->d.n_aeq - kAeqK);
    return 2 * n_chains <= (int64_t)p->n_sm * kSerialCtasPerSm && blocks >= kSerialMinBlocks;
}

cudaError_t fnt::aeq_launch_for(const fnt_plan *p, const DevFrame *frames, const AeqChain *chains, int n_chains,
                                int64_t longest_symbols, cudaStream_t stream) {
    AeqParams prm{p->d.mu_shift, p->d.rde_a, update_period(p->d), p->tensor_gradient, p->d.aeq_freq_sum};
    if (aeq_use_serial(p, n_chains, longest_symbols))
        return aeq_serial_launch(p->d.n_aeq, frames, chains, n_chains, prm, 0, stream);
    return aeq_launch(p->d.n_aeq, frames, chains, n_chains, prm, p->aeq_warps, 0, stream, aeq_min_smem(p));
}

extern "C" fnt_status fnt_plan_initial_taps(const fnt_plan *p, int32_t *state) {
    if (!p || !state) return fail(FNT_ERR_INVALID, "null argument");
    memcpy(state, p->h_init, sizeof p->h_init);
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_cdc_items(fnt_plan *p, int32_t pols) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (pols < 0 || pols > 2) return fail(FNT_ERR_INVALID, "pols per CDC item must be 0, 1 or 2");
    p->cdc_pols_per_item = pols;
    return FNT_OK;
}

extern "C" fnt_status fnt_plan_set_tensor_gradient(fnt_plan *p, int32_t on) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    if (on != 0 && on != 1) return fail(FNT_ERR_INVALID, "tensor_gradient must be 0 or 1");
    p->tensor_gradient = on;
    return FNT_OK;
}

// ---------------------------------------------------------- work building ---

namespace fnt {

static bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

// Device-accessible address of a buffer: device (or managed) memory as it is,
// page-locked host memory through its device mapping (on GB300 the GPU reads
// and writes Grace memory coherently over NVLink-C2C); nullptr for pageable
// host memory.
void *device_view(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return const_cast<void *>(p);
    if (a.type == cudaMemoryTypeHost) return a.devicePointer;
    return nullptr;
}

// Validates one frame for `op` and fills its DevFrame (pointers as given).
static fnt_status make_frame(const fnt_plan *p, const fnt_frame &f, int op, int idx, DevFrame &df) {
    memset(&df, 0, sizeof df);
    if (f.n < 0) return fail(FNT_ERR_INVALID, "frame %d: n < 0", idx);
    df.in = (const int8_t *)f.in;
    df.out = f.out;
    df.state = f.aeq_state;
    df.n = f.n;
    df.flags = p->test_inject;
    if (op == FNT_OP_AEQ) {
        df.n_pol = 2;
        df.n_sym = f.n;
        df.aeq_in = (int8_t *)f.in;
        if (f.n > 0 && (!f.in || !f.out)) return fail(FNT_ERR_INVALID, "frame %d: null buffer", idx);
        if (!aligned(f.in, 4) || !aligned(f.out, 4) || !aligned(f.aeq_state, 4))
            return fail(FNT_ERR_INVALID, "frame %d: buffers must be 4-byte aligned", idx);
        return FNT_OK;
    }
    if (f.n_pol != 1 && f.n_pol != 2) return fail(FNT_ERR_INVALID, "frame %d: n_pol must be 1 or 2", idx);
    if (op == FNT_OP_CHAIN && f.n_pol != 2) return fail(FNT_ERR_INVALID, "frame %d: the chain needs n_pol = 2", idx);
    if (f.cd_len < 1) return fail(FNT_ERR_INVALID, "frame %d: cd_len < 1", idx);
    if (f.cd_len > kMaxCdTaps)
        return fail(FNT_ERR_BOUND, "frame %d: cd_len %d > %d breaks constraint (5) for 5-bit x 6-bit with int16 output",
                    idx, f.cd_len, kMaxCdTaps);
    if (!f.cd_taps) return fail(FNT_ERR_INVALID, "frame %d: null cd_taps", idx);
    for (int k = 0; k < 2 * f.cd_len; ++k) {
        if (f.cd_taps[k] < -32 || f.cd_taps[k] > 31)
            return fail(FNT_ERR_INVALID, "frame %d: tap value %d outside 6 bits", idx, f.cd_taps[k]);
        df.taps[k] = f.cd_taps[k];
    }
    const int S = p->d.cdc_step ? p->d.cdc_step : kCdcN - f.cd_len + 1;
    if (S > kCdcN - f.cd_len + 1 || S < 32)
        return fail(FNT_ERR_BOUND, "frame %d: step %d with %d taps: need 32 <= S <= N - L + 1", idx, S, f.cd_len);
    df.n_pol = f.n_pol;
    df.L = f.cd_len;
    df.S = S;
    df.shift = cdc_shift_of(f.cd_taps, f.cd_len);
    df.phase = decim_phase_of(f.cd_len);
    if (f.n > 0 && (!f.in || !f.out)) return fail(FNT_ERR_INVALID, "frame %d: null buffer", idx);
    if (!aligned(f.in, 2 * f.n_pol)) return fail(FNT_ERR_INVALID, "frame %d: input must be %d-byte aligned", idx, 2 * f.n_pol);
    if (op == FNT_OP_CDC) {
        if (!aligned(f.out, 4 * f.n_pol))
            return fail(FNT_ERR_INVALID, "frame %d: output must be %d-byte aligned", idx, 4 * f.n_pol);
    } else {
        df.n_sym = chain_nsym(f.n, df.phase);
        if (!aligned(f.out, 4) || !aligned(f.aeq_state, 4))
            return fail(FNT_ERR_INVALID, "frame %d: output and state must be 4-byte aligned", idx);
    }
    return FNT_OK;
}

// CDC items of one frame: 32 blocks of one polarisation each (w = pol), or, with
// `both`, of both polarisations of a PDM frame (w = 2: one window fill and one
// tap-spectrum set serve the two).
static void add_cdc_items(const DevFrame &df, int fi, bool both, std::vector<int4> &items) {
    const int64_t nblk = (df.n + df.S - 1) / df.S;
    for (int64_t b = 0; b < nblk; b += kBlocksPerItem) {
        const int nb = (int)std::min<int64_t>(kBlocksPerItem, nblk - b);
        if (both && df.n_pol == 2) {
            items.push_back(make_int4(fi, (int)b, nb, 2));
        } else {
            for (int p = 0; p < df.n_pol; ++p) items.push_back(make_int4(fi, (int)b, nb, p));
        }
    }
}

// Whether the CDC items of this work take both polarisations at once.  Per-
// polarisation items double the warps (better for work that does not fill the
// GPU twice over); two-polarisation items halve the window fills and the tap
// spectra per block (better once there is work for several waves).
static bool cdc_items_both(const fnt_plan *p, const Work &w) {
    if (p->cdc_pols_per_item != 0) return p->cdc_pols_per_item == 2;
    int64_t items = 0;
    for (const DevFrame &df : w.frames)
        if (df.n_pol == 2) items += ((df.n + df.S - 1) / df.S + kBlocksPerItem - 1) / kBlocksPerItem;
    const int64_t resident = (int64_t)p->n_sm * kCdcCtasPerSm * p->cdc_warps;
    return items >= 2 * resident;
}

// AEQ runs of one frame.  Unsegmented: one chain that reads and writes the
// frame's state (or starts from the plan's taps).  Segmented: every segment
// starts from the frame's state as it was when the call began (a copy taken on
// the stream first, since the last segment overwrites the state) or from the
// plan's taps; only the last segment writes the state.
static void add_aeq_chains(const fnt_plan *p, const DevFrame &df, int fi, const int32_t *init_dev, Work &w) {
    const int64_t n = df.n_sym;
    if (n == 0) return;
    const int64_t seg = p->d.aeq_segment;
    if (seg <= 0 || seg >= n) {
        AeqChain c{};
        c.frame = fi;
        c.write_state = df.state != nullptr;
        c.begin = 0;
        c.keep = 0;
        c.end = n;
        c.init = df.state ? df.state : init_dev;
        c.init_copy = -1;
        w.chains.push_back(c);
        return;
    }
    int copy = -1;
    if (df.state) {
        copy = (int)w.init_src.size();
        w.init_src.push_back(fi);
    }
    for (int64_t k = 0; k < n; k += seg) {
        AeqChain c{};
        c.frame = fi;
        c.keep = k;
        c.end = std::min(n, k + seg);
        c.begin = std::max<int64_t>(0, k - p->d.aeq_warmup);
        c.lo = std::max<int64_t>(0, c.begin - kAeqK);   // the stream's preceding symbols
        c.write_state = (df.state != nullptr) && c.end == n;
        c.init = init_dev;
        c.init_copy = copy;
        w.chains.push_back(c);
    }
}

fnt_status build_work(const fnt_plan *p, const fnt_frame_batch *b, int op, Work &w) {
    if (!b || b->n_frames < 0 || (b->n_frames > 0 && !b->frames))
        return fail(FNT_ERR_INVALID, "bad frame batch");
    w = Work();
    w.op = op;
    w.frames.resize(b->n_frames);
    int64_t scratch = 0;
    for (int i = 0; i < b->n_frames; ++i) {
        fnt_status st = make_frame(p, b->frames[i], op, i, w.frames[i]);
        if (st != FNT_OK) return st;
        if (op == FNT_OP_CHAIN) {
            w.scratch_off.push_back(scratch);
            scratch += (w.frames[i].n_sym * 4 + 255) / 256 * 256;
        }
    }
    w.scratch_bytes = scratch;
    // Longest frames first, both for their CDC items and their AEQ chains: the
    // serial AEQ recurrences of long frames bound the makespan, and with
    // pipelined chunks they then start in the first chunk.
    std::vector<int> order(b->n_frames);
    for (int i = 0; i < b->n_frames; ++i) order[i] = i;
    if (op == FNT_OP_CHAIN)
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int c) { return w.frames[a].n_sym > w.frames[c].n_sym; });
    const bool both = op != FNT_OP_AEQ && cdc_items_both(p, w);
    w.cdc_both = both;
    {
        size_t n_items = 0, n_chains = 0;
        for (const DevFrame &df : w.frames) {
            if (op != FNT_OP_AEQ) n_items += (size_t)(((df.n + df.S - 1) / df.S + kBlocksPerItem - 1) / kBlocksPerItem) * 2;
            if (op != FNT_OP_CDC)
                n_chains += p->d.aeq_segment > 0 ? (size_t)((df.n_sym + p->d.aeq_segment - 1) / p->d.aeq_segment) : 1;
        }
        w.items.reserve(n_items);
        w.chains.reserve(n_chains);
    }
    for (int i : order) {
        const int first_item = (int)w.items.size();
        if (op != FNT_OP_AEQ) add_cdc_items(w.frames[i], i, both, w.items);
        if (op != FNT_OP_CDC) {
            const size_t c0 = w.chains.size();
            add_aeq_chains(p, w.frames[i], i, p->d_init, w);
            for (size_t c = c0; c < w.chains.size(); ++c) {
                const DevFrame &df = w.frames[i];
                // last 2-sps sample the chain reads, and the CDC item that produces it
                const int64_t t_last = 2 * (w.chains[c].end - 1) + df.phase;
                const int per = both && df.n_pol == 2 ? 1 : df.n_pol;     // items per 32 blocks
                w.chains[c].need_item =
                    op == FNT_OP_CHAIN ? first_item + (int)(t_last / df.S / kBlocksPerItem) * per + per - 1 : 0;
            }
        }
    }
    if (w.items.size() > (size_t)INT32_MAX || w.chains.size() > (size_t)INT32_MAX)
        return fail(FNT_ERR_INVALID, "batch too large");
    // pipelined chunks (chain op only): cut the item list evenly; a chain joins
    // the first chunk whose CDC items cover everything it reads
    int C = 1;
    if (op == FNT_OP_CHAIN && p->chunks > 1 && (int)w.items.size() >= 8 * p->chunks) C = p->chunks;
    w.item_cut.assign(C + 1, 0);
    for (int k = 0; k <= C; ++k) w.item_cut[k] = (int)((int64_t)w.items.size() * k / C);
    auto chunk_of = [&](const AeqChain &c) {
        int k = 0;
        while (k + 1 < C && c.need_item >= w.item_cut[k + 1]) ++k;
        return k;
    };
    // within a chunk, longest chains first (often already so: skip the sort then)
    auto before = [&](const AeqChain &a, const AeqChain &c) {
        const int ka = chunk_of(a), kc = chunk_of(c);
        if (ka != kc) return ka < kc;
        return (a.end - a.begin) > (c.end - c.begin);
    };
    if (!std::is_sorted(w.chains.begin(), w.chains.end(), before))
        std::stable_sort(w.chains.begin(), w.chains.end(), before);
    w.chain_cut.assign(C + 1, (int)w.chains.size());
    w.chain_cut[0] = 0;
    for (int k = 1; k < C; ++k) {
        int c = w.chain_cut[k - 1];
        while (c < (int)w.chains.size() && chunk_of(w.chains[c]) < k) ++c;
        w.chain_cut[k] = c;
    }
    return FNT_OK;
}

// Layout of one device allocation holding the tables and the intermediate buffer.
void layout(Work &w) {
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    w.off_frames = 0;
    w.off_items = up(w.off_frames + w.frames.size() * sizeof(DevFrame));
    w.off_chains = up(w.off_items + w.items.size() * sizeof(int4));
    w.off_init = up(w.off_chains + w.chains.size() * sizeof(AeqChain));
    w.off_spec = up(w.off_init + w.init_src.size() * kStateBytes);
    w.off_scratch = up(w.off_spec + (w.op != FNT_OP_AEQ ? w.frames.size() * kSpecBytes : 0));
    w.total = up(w.off_scratch + (size_t)w.scratch_bytes);
    if (w.total == 0) w.total = 256;
}

// A page-locked host buffer per thread for table uploads, with an event that
// marks when the last copy out of it has run (on the device it was recorded on).
struct Staging {
    char *buf = nullptr;
    size_t cap = 0;
    cudaEvent_t done = nullptr;
    int device = -1;
    cudaError_t reserve(size_t bytes) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (done) {
            e = cudaEventSynchronize(done);       // the previous copy has read the buffer
            if (e != cudaSuccess) return e;
        }
        if (dev != device && done) {
            cudaEventDestroy(done);
            done = nullptr;
        }
        if (!done) {
            e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
            device = dev;
        }
        if (cap < bytes) {                        // geometric: reallocation stays rare
            const size_t want = std::max({bytes, 2 * cap, (size_t)64 << 10});
            if (buf) cudaFreeHost(buf);
            buf = nullptr;
            cap = 0;
            e = cudaMallocHost((void **)&buf, want);
            if (e != cudaSuccess) return e;
            cap = want;
        }
        return cudaSuccess;
    }
};

// Four per thread in rotation, so that a thread can queue a few calls ahead of
// the device before it waits for a staging buffer.
static Staging &thread_staging() {
    static thread_local Staging sg[4];     // kept for the thread's life
    static thread_local unsigned next = 0;
    return sg[next++ & 3];
}

void point_spectra(Work &w, char *dev) {
    if (w.op == FNT_OP_AEQ) return;
    for (size_t i = 0; i < w.frames.size(); ++i)
        w.frames[i].hspec = (int32_t *)(dev + w.off_spec + i * kSpecBytes);
}

// Points the chain frames' intermediate buffers and tap-spectrum slots into the
// allocation and copies the three tables (host -> device, on `stream`).
fnt_status upload_work(Work &w, char *dev, cudaStream_t stream) {
    point_spectra(w, dev);
    if (w.op == FNT_OP_CHAIN)
        for (size_t i = 0; i < w.frames.size(); ++i)
            w.frames[i].aeq_in = (int8_t *)(dev + w.off_scratch + w.scratch_off[i]);
    for (AeqChain &c : w.chains)
        if (c.init_copy >= 0) c.init = (const int32_t *)(dev + w.off_init + (size_t)c.init_copy * kStateBytes);
    // the three tables are contiguous in [0, off_init): one copy from a page-
    // locked staging buffer of this thread, reused once its previous copy is done
    const size_t bytes = w.off_init;
    if (bytes == 0) return FNT_OK;
    Staging &sg = thread_staging();
    cudaError_t e = sg.reserve(bytes);
    if (e != cudaSuccess) return cuda_fail(e, "table staging");
    if (!w.frames.empty()) memcpy(sg.buf + w.off_frames, w.frames.data(), w.frames.size() * sizeof(DevFrame));
    if (!w.items.empty()) memcpy(sg.buf + w.off_items, w.items.data(), w.items.size() * sizeof(int4));
    if (!w.chains.empty()) memcpy(sg.buf + w.off_chains, w.chains.data(), w.chains.size() * sizeof(AeqChain));
    e = cudaMemcpyAsync(dev, sg.buf, bytes, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaEventRecord(sg.done, stream);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "upload tables");
}

static fnt_status launch_cdc_range(const fnt_plan *p, const Work &w, const char *dev, int i0, int i1,
                                   cudaStream_t stream) {
    if (i1 <= i0) return FNT_OK;
    const DevFrame *frames = (const DevFrame *)(dev + w.off_frames);
    const int nw = p->cdc_warps;
    const int n = i1 - i0;
    const int grid = std::min((n + nw - 1) / nw, p->n_sm * 64);
    cudaError_t e = cdc_launch(frames, (const int4 *)(dev + w.off_items) + i0, n, w.op == FNT_OP_CHAIN, w.cdc_both,
                               nw, grid, stream, cdc_use_split(p, (int64_t)w.items.size()));
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "cdc kernel launch");
}

static fnt_status copy_initial_taps(const Work &w, const char *dev, cudaStream_t stream) {
    for (size_t k = 0; k < w.init_src.size(); ++k) {
        cudaError_t e = cudaMemcpyAsync((void *)(dev + w.off_init + k * kStateBytes), w.frames[w.init_src[k]].state,
                                        kStateBytes, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy initial taps");
    }
    return FNT_OK;
}

static fnt_status launch_aeq_range(const fnt_plan *p, const Work &w, const char *dev, int c0, int c1,
                                   cudaStream_t stream) {
    if (c1 <= c0) return FNT_OK;
    const DevFrame *frames = (const DevFrame *)(dev + w.off_frames);
    int64_t longest = 0;                  // chains are sorted longest first within a chunk; take the max anyway
    for (int c = c0; c < c1; ++c) longest = std::max(longest, w.chains[c].end - w.chains[c].begin);
    cudaError_t e = aeq_launch_for(p, frames, (const AeqChain *)(dev + w.off_chains) + c0, c1 - c0, longest, stream);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "aeq kernel launch");
}

static fnt_status launch_spectra(const Work &w, const char *dev, cudaStream_t stream) {
    if (w.op == FNT_OP_AEQ || w.spectra_ready || w.frames.empty()) return FNT_OK;
    cudaError_t e = cdc_spectra_launch((const DevFrame *)(dev + w.off_frames), (int)w.frames.size(), stream);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "tap spectra launch");
}

fnt_status launch_work(const fnt_plan *p, const Work &w, const char *dev, cudaStream_t stream, int stages) {
    fnt_status st = FNT_OK;
    if ((stages & 1) && w.op != FNT_OP_AEQ) {
        st = launch_spectra(w, dev, stream);
        if (st == FNT_OK) st = launch_cdc_range(p, w, dev, 0, (int)w.items.size(), stream);
    }
    if (st == FNT_OK && (stages & 2) && w.op != FNT_OP_CDC && !w.chains.empty()) {
        st = copy_initial_taps(w, dev, stream);
        if (st == FNT_OK) st = launch_aeq_range(p, w, dev, 0, (int)w.chains.size(), stream);
    }
    return st;
}

fnt_status launch_pipelined(const fnt_plan *p, const Work &w, const char *dev, cudaStream_t stream,
                            const std::vector<cudaStream_t> &side, const std::vector<cudaEvent_t> &ev) {
    const int C = (int)w.item_cut.size() - 1;
    fnt_status st = copy_initial_taps(w, dev, stream);
    if (st == FNT_OK) st = launch_spectra(w, dev, stream);
    for (int k = 0; k < C && st == FNT_OK; ++k) {
        st = launch_cdc_range(p, w, dev, w.item_cut[k], w.item_cut[k + 1], stream);
        if (st != FNT_OK) break;
        cudaError_t e = cudaEventRecord(ev[k], stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side[k], ev[k], 0);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline fork");
        st = launch_aeq_range(p, w, dev, w.chain_cut[k], w.chain_cut[k + 1], side[k]);
        if (st != FNT_OK) break;
        e = cudaEventRecord(ev[C + k], side[k]);
        if (e != cudaSuccess) return cuda_fail(e, "pipeline record");
    }
    // join every side stream back (also after an error, so a capture can end)
    for (int k = 0; k < C; ++k) {
        cudaError_t e = cudaStreamWaitEvent(stream, ev[C + k], 0);
        if (e != cudaSuccess && st == FNT_OK) st = cuda_fail(e, "pipeline join");
    }
    return st;
}

int work_kernel_count(const Work &w) {
    const int C = (int)w.item_cut.size() - 1;
    int k = 0;
    if (w.op != FNT_OP_AEQ && !w.spectra_ready && !w.frames.empty()) k += 1;   // tap spectra
    if (w.op != FNT_OP_AEQ) k += C > 1 ? C : (w.items.empty() ? 0 : 1);
    if (w.op != FNT_OP_CDC) {
        if (C > 1) {
            for (int c = 0; c < C; ++c) k += w.chain_cut[c + 1] > w.chain_cut[c];
        } else {
            k += w.chains.empty() ? 0 : 1;
        }
    }
    return k;
}

// Per-frame host<->device sizes for host_buffers = 1.
static size_t in_bytes(const fnt_frame &f, int op) { return op == FNT_OP_AEQ ? f.n * 4 : f.n * 2 * f.n_pol; }

static size_t out_bytes(const fnt_frame &f, int op, const DevFrame &df) {
    if (op == FNT_OP_CDC) return f.n * 4 * f.n_pol;
    if (op == FNT_OP_AEQ) return f.n * 8;
    return df.n_sym * 8;
}

static fnt_status run(const fnt_plan *p, const fnt_frame_batch *b, int op, void *stream_) {
    if (!p) return fail(FNT_ERR_INVALID, "null plan");
    fnt_status dst = check_device(p);
    if (dst != FNT_OK) return dst;
    cudaStream_t stream = (cudaStream_t)stream_;
    Work w;
    fnt_status st = build_work(p, b, op, w);
    if (st != FNT_OK) return st;
    layout(w);
    // host buffers: page-locked ones are read and written in place through
    // their device mapping; pageable ones get device copies after the tables
    std::vector<size_t> io_in, io_out;
    std::vector<char> stage_in, stage_out;
    size_t total = w.total;
    if (b->host_buffers) {
        for (int i = 0; i < b->n_frames; ++i) {
            const fnt_frame &f = b->frames[i];
            DevFrame &df = w.frames[i];
            const bool has_in = in_bytes(f, op) > 0, has_out = out_bytes(f, op, df) > 0;
            void *vin = has_in ? device_view(f.in) : nullptr;
            void *vout = has_out ? device_view(f.out) : nullptr;
            stage_in.push_back(has_in && !vin);
            stage_out.push_back(has_out && !vout);
            if (vin) {
                df.in = (const int8_t *)vin;
                if (op == FNT_OP_AEQ) df.aeq_in = (int8_t *)vin;
            }
            if (vout) df.out = vout;
            io_in.push_back(total);
            if (stage_in.back()) total += (in_bytes(f, op) + 255) / 256 * 256;
            io_out.push_back(total);
            if (stage_out.back()) total += (out_bytes(f, op, df) + 255) / 256 * 256;
        }
    }
    char *dev = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&dev, total, p->pool, stream);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(FNT_ERR_NOMEM, "device memory") : cuda_fail(e, "cudaMallocFromPoolAsync");
    if (b->host_buffers) {
        for (int i = 0; i < b->n_frames; ++i) {
            const fnt_frame &f = b->frames[i];
            DevFrame &df = w.frames[i];
            if (stage_out[i]) df.out = dev + io_out[i];
            if (!stage_in[i]) continue;
            df.in = (const int8_t *)(dev + io_in[i]);
            if (op == FNT_OP_AEQ) df.aeq_in = (int8_t *)df.in;
            const size_t nb = in_bytes(f, op);
            e = cudaMemcpyAsync(dev + io_in[i], f.in, nb, cudaMemcpyHostToDevice, stream);
            if (e != cudaSuccess) { cudaFreeAsync(dev, stream); return cuda_fail(e, "copy input"); }
        }
    }
    st = upload_work(w, dev, stream);
    if (st == FNT_OK) st = launch_work(p, w, dev, stream);
    if (st == FNT_OK && b->host_buffers) {
        for (int i = 0; i < b->n_frames; ++i) {
            const size_t nb = out_bytes(b->frames[i], op, w.frames[i]);
            if (!nb || !stage_out[i]) continue;
            e = cudaMemcpyAsync(b->frames[i].out, dev + io_out[i], nb, cudaMemcpyDeviceToHost, stream);
            if (e != cudaSuccess) { st = cuda_fail(e, "copy output"); break; }
        }
    }
    cudaFreeAsync(dev, stream);
    if (st == FNT_OK && b->host_buffers) {
        e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaStreamSynchronize");
    }
    return st;
}

}  // namespace fnt

extern "C" fnt_status fnt_cdc_run(const fnt_plan *p, const fnt_frame_batch *b, void *stream) {
    Range trace("fnt_cdc_run");
    return run(p, b, FNT_OP_CDC, stream);
}

extern "C" fnt_status fnt_aeq_run(const fnt_plan *p, const fnt_frame_batch *b, void *stream) {
    Range trace("fnt_aeq_run");
    return run(p, b, FNT_OP_AEQ, stream);
}

extern "C" fnt_status fnt_cdc_aeq_run(const fnt_plan *p, const fnt_frame_batch *b, void *stream) {
    Range trace("fnt_cdc_aeq_run");
    return run(p, b, FNT_OP_CHAIN, stream);
}

// -------------------------------------------------------- prepared batches ---

struct fnt_batch {
    const fnt_plan *plan = nullptr;
    Work work;
    char *dev = nullptr;
    int use_graph = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaStream_t> side;   // one per pipelined chunk
    std::vector<cudaEvent_t> ev;      // fork (k) and join (C + k) events
    // Page-locked host inputs (host-buffer batches) and, with the input copy
    // on, their device copies: frame, host pointer, its device mapping, offset
    // in dev_in and size.
    struct Input {
        int frame;
        const void *src;
        const void *view;
        size_t off, bytes;
    };
    std::vector<Input> inputs;
    bool in_copy = false;
    char *dev_in = nullptr;
    cudaStream_t copy = nullptr;      // the batch's own copy stream
    cudaEvent_t copy_done = nullptr;  // this launch's inputs are on the device
    cudaEvent_t in_free = nullptr;    // the previous launch has consumed them
};

static fnt_status batch_enqueue(fnt_batch *bt, cudaStream_t stream) {
    if (bt->side.empty()) return launch_work(bt->plan, bt->work, bt->dev, stream);
    return launch_pipelined(bt->plan, bt->work, bt->dev, stream, bt->side, bt->ev);
}

// Input copy: the frames' inputs go to the device on the batch's copy stream,
// which waits only for the batch's previous launch to have consumed them, not
// for `stream`; `stream` then waits for the copies.
static fnt_status start_input_copy(fnt_batch *bt, cudaStream_t stream) {
    cudaError_t e = cudaStreamWaitEvent(bt->copy, bt->in_free, 0);
    for (size_t k = 0; k < bt->inputs.size() && e == cudaSuccess; ++k) {
        const fnt_batch::Input &in = bt->inputs[k];
        e = cudaMemcpyAsync(bt->dev_in + in.off, in.src, in.bytes, cudaMemcpyHostToDevice, bt->copy);
    }
    if (e == cudaSuccess) e = cudaEventRecord(bt->copy_done, bt->copy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, bt->copy_done, 0);
    return e == cudaSuccess ? FNT_OK : cuda_fail(e, "batch input copy");
}

extern "C" fnt_status fnt_batch_create(const fnt_plan *p, const fnt_frame_batch *b, int32_t op, int32_t use_graph,
                                       fnt_batch **out) {
    if (!p || !out) return fail(FNT_ERR_INVALID, "null argument");
    *out = nullptr;
    if (op < FNT_OP_CDC || op > FNT_OP_CHAIN) return fail(FNT_ERR_INVALID, "unknown op %d", op);
    fnt_status dst = check_device(p);
    if (dst != FNT_OK) return dst;
    fnt_batch *bt = new (std::nothrow) fnt_batch();
    if (!bt) return fail(FNT_ERR_NOMEM, "host memory");
    bt->plan = p;
    bt->use_graph = use_graph;
    fnt_status st = build_work(p, b, op, bt->work);
    if (st != FNT_OK) {
        delete bt;
        return st;
    }
    if (b && b->host_buffers) {
        // page-locked host buffers are used in place through their device
        // mapping; the prepared work cannot stage pageable ones
        for (int i = 0; i < b->n_frames; ++i) {
            DevFrame &df = bt->work.frames[i];
            if (df.n == 0) continue;
            void *vin = device_view(b->frames[i].in), *vout = device_view(b->frames[i].out);
            if (!vin || !vout) {
                delete bt;
                return fail(FNT_ERR_INVALID, "fnt_batch: frame %d host buffers must be page-locked", i);
            }
            df.in = (const int8_t *)vin;
            if (op == FNT_OP_AEQ) df.aeq_in = (int8_t *)vin;
            df.out = vout;
            bt->inputs.push_back({i, b->frames[i].in, vin, 0, in_bytes(b->frames[i], op)});
        }
    }
    layout(bt->work);
    const int C = (int)bt->work.item_cut.size() - 1;
    if (C > 1) {
        bt->side.resize(C);
        bt->ev.resize(2 * C);
        for (auto &sd : bt->side) cudaStreamCreateWithFlags(&sd, cudaStreamNonBlocking);
        for (auto &e : bt->ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    }
    cudaError_t e = cudaMalloc((void **)&bt->dev, bt->work.total);
    if (e != cudaSuccess) {
        delete bt;
        return e == cudaErrorMemoryAllocation ? fail(FNT_ERR_NOMEM, "device memory") : cuda_fail(e, "cudaMalloc");
    }
    st = upload_work(bt->work, bt->dev, 0);
    // the taps of a prepared batch never change: its tap spectra are computed
    // once here, and its launches (and graph) hold only the CDC and AEQ kernels
    if (st == FNT_OK) st = launch_spectra(bt->work, bt->dev, 0);
    if (st == FNT_OK) {
        bt->work.spectra_ready = true;
        e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) st = cuda_fail(e, "upload sync");
    }
    if (st != FNT_OK) {
        cudaFree(bt->dev);
        delete bt;
        return st;
    }
    *out = bt;
    return FNT_OK;
}

extern "C" fnt_status fnt_batch_set_input_copy(fnt_batch *bt, int32_t on) {
    if (!bt) return fail(FNT_ERR_INVALID, "null batch");
    if (on && bt->inputs.empty()) return fail(FNT_ERR_INVALID, "input copy: not a host-buffer batch with input");
    if ((on != 0) == bt->in_copy) return FNT_OK;
    cudaError_t e = cudaDeviceSynchronize();          // no launch of the batch is in flight
    if (e == cudaSuccess && on && !bt->dev_in) {
        size_t total = 0;
        for (fnt_batch::Input &in : bt->inputs) {
            in.off = total;
            total += (in.bytes + 255) / 256 * 256;
        }
        e = cudaMalloc((void **)&bt->dev_in, total);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->copy, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->copy_done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->in_free, cudaEventDisableTiming);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? fail(FNT_ERR_NOMEM, "input copy: device memory")
                                                                    : cuda_fail(e, "input copy setup");
    }
    if (e != cudaSuccess) return cuda_fail(e, "input copy");
    // the kernels read the frame table from device memory: repoint the inputs
    // there (a captured graph stays valid)
    for (const fnt_batch::Input &in : bt->inputs) {
        DevFrame &df = bt->work.frames[in.frame];
        const int8_t *p = on ? (const int8_t *)(bt->dev_in + in.off) : (const int8_t *)in.view;
        df.in = p;
        if (bt->work.op == FNT_OP_AEQ) df.aeq_in = (int8_t *)p;
    }
    e = cudaMemcpy(bt->dev + bt->work.off_frames, bt->work.frames.data(), bt->work.frames.size() * sizeof(DevFrame),
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "input copy: frame table");
    bt->in_copy = on != 0;
    return FNT_OK;
}

static fnt_status batch_launch_all(fnt_batch *bt, cudaStream_t stream);

extern "C" fnt_status fnt_batch_launch(fnt_batch *bt, void *stream_) {
    if (!bt) return fail(FNT_ERR_INVALID, "null batch");
    Range trace("fnt_batch_launch");
    cudaStream_t stream = (cudaStream_t)stream_;
    if (!bt->in_copy) return batch_launch_all(bt, stream);
    fnt_status st = start_input_copy(bt, stream);
    if (st == FNT_OK) st = batch_launch_all(bt, stream);
    if (st == FNT_OK) {
        cudaError_t e = cudaEventRecord(bt->in_free, stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch input release");
    }
    return st;
}

static fnt_status batch_launch_all(fnt_batch *bt, cudaStream_t stream) {
    if (!bt->use_graph) return batch_enqueue(bt, stream);
    if (!bt->exec) {
        cudaStream_t cap;
        cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaStreamDestroy(cap);
            return cuda_fail(e, "cudaStreamBeginCapture");
        }
        fnt_status st = batch_enqueue(bt, cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(cap, &graph);
        cudaStreamDestroy(cap);
        if (st != FNT_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&bt->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    }
    cudaError_t e = cudaGraphLaunch(bt->exec, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return FNT_OK;
}

extern "C" fnt_status fnt_batch_launch_stage(fnt_batch *bt, int32_t stage, void *stream_) {
    if (!bt) return fail(FNT_ERR_INVALID, "null batch");
    Range trace(stage == 0 ? "fnt_batch_launch_stage cdc" : "fnt_batch_launch_stage aeq");
    if (stage != 0 && stage != 1) return fail(FNT_ERR_INVALID, "stage must be 0 (CDC) or 1 (AEQ)");
    cudaStream_t stream = (cudaStream_t)stream_;
    // with the input copy on, the stage that reads the inputs copies them first
    const bool reads_input = bt->in_copy && stage == (bt->work.op == FNT_OP_AEQ ? 1 : 0);
    fnt_status st = reads_input ? start_input_copy(bt, stream) : FNT_OK;
    if (st == FNT_OK) st = launch_work(bt->plan, bt->work, bt->dev, stream, 1 << stage);
    if (st == FNT_OK && reads_input) {
        cudaError_t e = cudaEventRecord(bt->in_free, stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch input release");
    }
    return st;
}

extern "C" int32_t fnt_batch_kernel_count(const fnt_batch *bt) { return bt ? work_kernel_count(bt->work) : 0; }

extern "C" fnt_status fnt_batch_destroy(fnt_batch *bt) {
    if (!bt) return FNT_OK;
    cudaDeviceSynchronize();
    if (bt->exec) cudaGraphExecDestroy(bt->exec);
    for (auto &sd : bt->side) cudaStreamDestroy(sd);
    for (auto &e : bt->ev) cudaEventDestroy(e);
    if (bt->copy) cudaStreamDestroy(bt->copy);
    if (bt->copy_done) cudaEventDestroy(bt->copy_done);
    if (bt->in_free) cudaEventDestroy(bt->in_free);
    cudaFree(bt->dev_in);
    cudaFree(bt->dev);
    delete bt;
    return FNT_OK;
}
