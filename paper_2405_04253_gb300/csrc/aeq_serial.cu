// aeq_serial.cu -- FNT-AEQ for few, long serial chains: the same method and the
// same results as aeq_kernel (4x4 real-valued MIMO with two 7-bit tap groups,
// one inverse transform per (input, output, group), RDE update of eq. (6);
// section "Proposed FNT-CDC&AEQ structure"), laid out for the latency of one
// block instead of throughput.
//
// The update of eq. (6) makes block b + 1 depend on the outputs of block b, so
// a chain's blocks run one after another.  aeq_kernel gives a (chain,
// polarisation) one warp; when a launch has only a few chains (a single stream
// under the paper's update rule, a serving wave) most of the GPU idles and the
// time per block of one warp sets the run time.  Here one CTA owns a (chain,
// polarisation), and each block is spread over it:
//
//   phase 1 (128 threads = 16 tasks x R = 8).  Task (o, s1, g) is the
//     length-N transform pair of filter S1 -> S2 = 2p + o and tap group g.
//     Thread r of the task handles the frequencies k = R k' + r:
//       X[R k' + r] = FNT_{N/R, alpha^R}( u ),  u_j = sum_m w_{j + mN/R} alpha^{(j + mN/R) r}
//     (the 16 zero-padded taps folded onto N/R points), multiplies by the input
//     spectrum (computed ahead, N^-1 folded in) and inverts its piece:
//       E_r = IFNT_{N/R, alpha^R}(Y[R . + r]),  v_r[n'] = alpha^{-n' r} E_r[n'].
//     The outputs then follow from an R-point transform across the R threads,
//       c[n' + (N/R) m] = sum_r (alpha^{-N/R})^{m r} v_r[n'],
//     done in registers after a transpose through shared memory.  Kept outputs
//     (n >= K) are decoded (exact by constraint (5)), weighted 128 / 1 and
//     summed over the warp's tasks by shuffles.
//   phase 2 (SA threads): y summed over the task partials, z = sat16(y >> 7),
//     the RDE error e of the polarisation; outputs are stored.
//   phase 3 (256 threads): the gradient of eq. (6), G[f][k] = sum_i e_i z_o,i
//     x_s1[t0 + i - k], as (filter, 4 taps, 1/8 of the symbols) per thread with
//     a shuffle reduction, then the tap update in shared memory.
//
// A ninth warp produces the input spectra: it stages the input words of the
// next PRE blocks with cp.async (zero outside the chain's window) and runs one
// N-point transform per (block, input) per lane, one batch ahead of the
// consumers.  The phases meet at named barriers (bar.sync 1, consumers only;
// bar.sync 2, all warps, once per batch): nothing waits on a flag.
#include <cuda_runtime.h>

#include "internal.h"
#include "zf.cuh"

namespace fnt {

namespace {

template <int NA_, int64_t ALPHA_>
struct SerCfg {
    static constexpr int NA = NA_;
    static constexpr int64_t ALPHA = ALPHA_;
    static constexpr int K = kAeqK;
    static constexpr int SA = NA - K;                       // symbols per block
    static constexpr int R = 8;                             // threads per tap transform
    static constexpr int NP = NA / R;                       // points per thread
    static constexpr int MKEEP = K / NP;                    // first kept output group m
    static constexpr int64_t BETA = zpow(ALPHA, R);         // radix of the N/R-point pieces
    static constexpr int64_t AINV = zinv(ALPHA);
    static constexpr int64_t GAMMA = zpow(AINV, NP);        // radix of the R-point stage
    static constexpr int32_t NINV = zcent(zinv(NA));
    static constexpr int PRE = 8;                           // blocks per producer batch
    static constexpr int XS = PRE * SA + K;                 // staged input words per batch
    // input spectra of one block: [s1][r][XROW]; XROW = 4 (mod 8) words makes
    // the 8 r-rows of a quarter warp's 16-byte loads hit distinct banks
    static constexpr int XROW = NP % 8 == 4 ? NP : NP + 4;
    static constexpr int S1STR = R * XROW + 4;
    static constexpr int XBLK = 4 * S1STR;
    static constexpr int TP = R + 4;                        // transpose row (one n')
    static constexpr int TT = NP * TP + 8;                  // transpose rows of one task
    static constexpr int TROW = K + 4;                      // master-tap row
    static constexpr int PROW = SA + 4;                     // partial-output row
    static constexpr int NPW = 16 * R / 32;                 // warps of phase 1
    static constexpr int NCONS = 256;                       // consumer threads
    static constexpr int NTHR = NCONS + 32;                 // + the producer warp
    static constexpr int GSYM = SA / 8;                     // gradient symbols per thread
    // shared memory (words); every region a multiple of 4 words
    static constexpr int O_TAPS = 0;
    static constexpr int O_XF = O_TAPS + 8 * TROW;
    static constexpr int O_TB = O_XF + 2 * PRE * XBLK;
    static constexpr int O_XS = O_TB + 16 * TT;
    static constexpr int O_PART = O_XS + (2 * XS + 3) / 4 * 4;
    static constexpr int O_ZE = O_PART + NPW * PROW;
    static constexpr int WORDS = O_ZE + 3 * SA;
    static_assert(NA % R == 0 && K % NP == 0 && SA % 8 == 0 && R == 8, "shapes");
    static_assert(O_XF % 4 == 0 && O_TB % 4 == 0 && O_XS % 4 == 0 && O_PART % 4 == 0 && XROW % 4 == 0 &&
                      S1STR % 4 == 0 && TT % 4 == 0 && TP % 4 == 0,
                  "16-byte aligned rows");
};

__device__ __forceinline__ int32_t sx8s(uint32_t w, int sh) { return (int32_t)(w << (24 - sh)) >> 24; }

__device__ __forceinline__ void cp_async4s(uint32_t *smem, const uint32_t *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_alls() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ int64_t mad_wides(int32_t a, int32_t b, int64_t c) {
    int64_t d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// Named barriers: 1 = the consumer warps, 2 = every warp of the CTA.
__device__ __forceinline__ void bar_consumers(int n) { asm volatile("bar.sync 1, %0;\n" ::"r"(n) : "memory"); }
__device__ __forceinline__ void bar_all(int n) { asm volatile("bar.sync 2, %0;\n" ::"r"(n) : "memory"); }

__device__ __forceinline__ int32_t centred(int64_t v) {
    v %= kF;
    if (v < 0) v += kF;
    return v > 32768 ? (int32_t)(v - kF) : (int32_t)v;
}

// Spectrum register J of a length-N DIF transform holds X[k], k = bitrev(J);
// it goes to row (s1, r = k mod R), position bitrev_{N/R}(k / R), which is the
// register of the consumer's N/R-point piece that holds that frequency.
template <class C, int J>
struct StoreSpectrum {
    static __device__ __forceinline__ void run(const int32_t (&v)[C::NA], int32_t *dst) {
        constexpr int k = bitrev(J, ilog2(C::NA));
        constexpr int r = k % C::R;
        constexpr int i = bitrev(k / C::R, ilog2(C::NP));
        dst[r * C::XROW + i] = rhoc(rho(rhoc(v[J]) * C::NINV));
        if constexpr (J + 1 < C::NA) StoreSpectrum<C, J + 1>::run(v, dst);
    }
};

// The producer warp: input words of blocks [batch PRE, batch PRE + PRE) (plus
// the K before them), zero outside [lo, end), and their N-point spectra with
// N^-1 folded in; lane = 4 block + input.
template <class C>
__device__ __forceinline__ void produce(const AeqChain &ch, const uint32_t *xin, int64_t batch, uint32_t *xs,
                                        int32_t *xf, int lane) {
    const int64_t t_first = ch.begin + batch * C::PRE * C::SA - C::K;
    for (int q = lane; q < C::XS; q += 32) {
        const int64_t t = t_first + q;
        const bool ok = t >= ch.lo && t < ch.end;
        cp_async4s(xs + q, ok ? xin + t : xin, ok);
    }
    cp_async_wait_alls();
    __syncwarp();
    const int b = lane >> 2, s1 = lane & 3;
    const uint32_t *xw = xs + b * C::SA;
    int32_t v[C::NA];
#pragma unroll
    for (int j = 0; j < C::NA; ++j) v[j] = sx8s(xw[j], 8 * s1);
    fnt_fwd<C::NA, C::ALPHA, 5>(v);                                   // |x| <= 16
    StoreSpectrum<C, 0>::run(v, xf + b * C::XBLK + s1 * C::S1STR);
}

// Decoded, weighted outputs of the kept groups m >= MKEEP (register i of the
// R-point stage holds group m = bitrev_R(i)) of output column n' = q, summed
// over the warp's tasks and stored by the first task's threads at block
// position n' + NP m - K.
template <class C, int I>
struct KeepOutputs {
    static __device__ __forceinline__ void run(const int32_t (&a)[C::R], int32_t wgt, int32_t *prow, int q,
                                               int lane) {
        constexpr int m = bitrev(I, ilog2(C::R));
        if constexpr (m >= C::MKEEP) {
            int32_t v = decode(a[I]) * wgt;
#pragma unroll
            for (int s = C::R; s < 32; s <<= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
            if (lane < C::NP) prow[q + C::NP * m - C::K] = v;   // the warp's first task, one thread per n'
        }
        if constexpr (I + 1 < C::R) KeepOutputs<C, I + 1>::run(a, wgt, prow, q, lane);
    }
};

template <int NA, int64_t ALPHA>
__global__ void __launch_bounds__(SerCfg<NA, ALPHA>::NTHR, 1)
    aeq_serial_kernel(const DevFrame *__restrict__ frames, const AeqChain *__restrict__ chains, int n_items,
                      AeqParams prm) {
    using C = SerCfg<NA, ALPHA>;
    constexpr int K = C::K, SA = C::SA, R = C::R, NP = C::NP;
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t *ttab = (int32_t *)smem + C::O_TAPS;
    int32_t *xf2 = (int32_t *)smem + C::O_XF;
    int32_t *tb = (int32_t *)smem + C::O_TB;
    uint32_t *xs2 = smem + C::O_XS;
    int32_t *part = (int32_t *)smem + C::O_PART;
    int32_t *zs = (int32_t *)smem + C::O_ZE;     // z of both outputs [2][SA], then e [SA]
    int32_t *es = zs + 2 * SA;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int warp = tid >> 5;
    const bool producer = tid >= C::NCONS;
    const int64_t A2 = (int64_t)prm.rde_a * prm.rde_a;
    const int mu = prm.mu_shift;
    const int period = prm.period > 1 ? prm.period : 1;

    // phase-1 role: task (o, s1, g), r; twiddles alpha^{j r} and alpha^{-n' r}
    const int task = tid / R, r = tid % R;
    const int po = task >> 3, ps1 = (task >> 1) & 3, pg = task & 1;
    int32_t twf[K], twi[NP];
    {
        int64_t ar = 1, ai = 1;
        for (int i = 0; i < r; ++i) {
            ar = ar * C::ALPHA % kF;
            ai = ai * C::AINV % kF;
        }
        int64_t pw = 1;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            twf[j] = centred(pw);
            pw = pw * ar % kF;
        }
        pw = 1;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            twi[j] = centred(pw);
            pw = pw * ai % kF;
        }
    }
    // phase-3 role: filter f = warp (o = f >> 2, s1 = f & 3), taps k0 .. k0 + 3,
    // symbols i0 .. i0 + GSYM - 1
    const int gf = warp & 7, go = gf >> 2, gs1 = gf & 3;
    const int gsp = lane & 7, k0 = 4 * ((lane >> 3) & 3), i0 = gsp * C::GSYM;
    const int gb1 = (gsp >> 1) & 1, gb2 = (gsp >> 2) & 1;
    const int gk = k0 + 2 * gb2 + gb1;             // the tap this lane holds after the reduction

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const AeqChain ch = chains[item >> 1];
        const int p = item & 1;
        const DevFrame &fr = frames[ch.frame];
        const uint32_t *xin = (const uint32_t *)fr.aeq_in;
        int16_t *out = (int16_t *)fr.out;
        const int64_t nblk = (ch.end - ch.begin + SA - 1) / SA;
        const int64_t nbatch = (nblk + C::PRE - 1) / C::PRE;

        if (tid < 8 * K) {
            const int f = tid >> 4, k = tid & 15;
            ttab[f * C::TROW + k] = ch.init[((2 * p + (f >> 2)) * 4 + (f & 3)) * K + k];
        }
        if (producer && nbatch > 0) produce<C>(ch, xin, 0, xs2, xf2, lane);
        bar_all(C::NTHR);

        int64_t gsum = 0;                          // gradient of tap gk over the period
        int in_period = 0;
        for (int64_t j = 0; j < nbatch; ++j) {
            const int buf = (int)(j & 1);
            if (producer) {
                if (j + 1 < nbatch)
                    produce<C>(ch, xin, j + 1, xs2 + (buf ^ 1) * C::XS, xf2 + (buf ^ 1) * C::PRE * C::XBLK, lane);
            } else {
                const uint32_t *xs = xs2 + buf * C::XS;
                const int32_t *xf = xf2 + buf * C::PRE * C::XBLK;
                for (int bb = 0; bb < C::PRE; ++bb) {
                    const int64_t blk = j * C::PRE + bb;
                    if (blk >= nblk) break;                       // uniform over the consumers
                    const int64_t t0 = ch.begin + blk * SA;

                    // ---- phase 1: tap transforms, products, inverses, outputs
                    if (tid < 16 * R) {
                        const int32_t *trow = ttab + (4 * po + ps1) * C::TROW;
                        const int tsh = pg ? 16 : 23;             // hi = T >> 23, lo = (T >> 16) & 127
                        const int32_t tmask = pg ? 127 : -1;
                        int32_t w[K];
#pragma unroll
                        for (int q = 0; q < K / 4; ++q) {
                            const int4 t4 = *(const int4 *)(trow + 4 * q);
                            w[4 * q] = (t4.x >> tsh) & tmask;
                            w[4 * q + 1] = (t4.y >> tsh) & tmask;
                            w[4 * q + 2] = (t4.z >> tsh) & tmask;
                            w[4 * q + 3] = (t4.w >> tsh) & tmask;
                        }
                        int32_t u[NP];
#pragma unroll
                        for (int jj = 0; jj < NP; ++jj) {
                            int32_t s = jj == 0 ? w[0] : w[jj] * twf[jj];   // |w alpha^..| < 2^22
#pragma unroll
                            for (int m = 1; m < K / NP; ++m) s += w[jj + NP * m] * twf[jj + NP * m];
                            u[jj] = rho(s);
                        }
                        fnt_fwd<NP, C::BETA, 17>(u);
                        const int32_t *xrow = xf + bb * C::XBLK + ps1 * C::S1STR + r * C::XROW;
#pragma unroll
                        for (int i = 0; i < NP; i += 4) {
                            const int4 x4 = *(const int4 *)(xrow + i);
                            u[i] = rho(rhoc(u[i]) * x4.x);
                            u[i + 1] = rho(rhoc(u[i + 1]) * x4.y);
                            u[i + 2] = rho(rhoc(u[i + 2]) * x4.z);
                            u[i + 3] = rho(rhoc(u[i + 3]) * x4.w);
                        }
                        fnt_inv<NP, C::BETA, 17>(u);
                        int32_t *trows = tb + task * C::TT;
                        trows[r] = rho(u[0]);
#pragma unroll
                        for (int n = 1; n < NP; ++n) trows[n * C::TP + r] = rho(rhoc(u[n]) * twi[n]);
                        __syncwarp();
                        // after the transpose thread r takes output column n' = r mod NP
                        // (when NP < R, threads r and r + NP compute the same column)
                        const int nq = r % NP;
                        int32_t a[R];
#pragma unroll
                        for (int q = 0; q < R; q += 4) {
                            const int4 v4 = *(const int4 *)(trows + nq * C::TP + q);
                            a[q] = v4.x;
                            a[q + 1] = v4.y;
                            a[q + 2] = v4.z;
                            a[q + 3] = v4.w;
                        }
                        fnt_fwd<R, C::GAMMA, 17>(a);
                        KeepOutputs<C, 0>::run(a, pg ? 1 : 128, part + warp * C::PROW, nq, lane);
                    }
                    bar_consumers(C::NCONS);

                    // ---- phase 2: outputs and RDE error of the polarisation
                    if (tid < SA) {
                        const int i = tid;
                        int32_t y0 = 0, y1 = 0;
#pragma unroll
                        for (int w = 0; w < C::NPW / 2; ++w) {
                            y0 += part[w * C::PROW + i];
                            y1 += part[(C::NPW / 2 + w) * C::PROW + i];
                        }
                        const int32_t z0 = min(max(y0 >> 7, -32768), 32767);
                        const int32_t z1 = min(max(y1 >> 7, -32768), 32767);
                        const int64_t t = t0 + i;
                        const bool valid = t < ch.end;
                        const int64_t r2 = (int64_t)z0 * z0 + (int64_t)z1 * z1;
                        const int64_t Rr = r2 < 6 * A2 ? 2 * A2 : (r2 < 14 * A2 ? 10 * A2 : 18 * A2);
                        if (valid && t >= ch.keep)
                            *(uint32_t *)(out + t * 4 + 2 * p) = ((uint32_t)z0 & 0xFFFFu) | ((uint32_t)z1 << 16);
                        zs[i] = valid ? z0 : 0;
                        zs[SA + i] = valid ? z1 : 0;
                        es[i] = valid ? (int32_t)(Rr - r2) : 0;
                    }
                    bar_consumers(C::NCONS);

                    // ---- phase 3: gradient of eq. (6) and the tap update
                    if (mu < 63) {
                        const int8_t *xb = (const int8_t *)(xs + bb * SA + K - k0) + gs1;   // x_s1[t0 + i - k0] at xb[4 i]
                        int32_t w1 = xb[4 * (i0 - 1)], w2 = xb[4 * (i0 - 2)], w3 = xb[4 * (i0 - 3)];
                        const int32_t *zrow = zs + go * SA;
                        int64_t acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
#pragma unroll
                        for (int ii = 0; ii < C::GSYM; ++ii) {
                            const int i = i0 + ii;
                            const int32_t w0 = xb[4 * i];
                            const int32_t e = es[i], z = zrow[i];
                            acc0 = mad_wides(e, z * w0, acc0);          // |z x| <= 2^19
                            acc1 = mad_wides(e, z * w1, acc1);
                            acc2 = mad_wides(e, z * w2, acc2);
                            acc3 = mad_wides(e, z * w3, acc3);
                            w3 = w2;
                            w2 = w1;
                            w1 = w0;
                        }
                        // sum over the 8 symbol ranges (lane bits 0..2); the lane
                        // keeps tap k0 + 2 b2 + b1
                        int64_t k01 = gb2 ? acc2 : acc0, k11 = gb2 ? acc3 : acc1;
                        const int64_t s01 = gb2 ? acc0 : acc2, s11 = gb2 ? acc1 : acc3;
                        k01 += __shfl_xor_sync(0xffffffffu, s01, 4);
                        k11 += __shfl_xor_sync(0xffffffffu, s11, 4);
                        int64_t kv = gb1 ? k11 : k01;
                        kv += __shfl_xor_sync(0xffffffffu, gb1 ? k01 : k11, 2);
                        kv += __shfl_xor_sync(0xffffffffu, kv, 1);
                        gsum += kv;
                        if (++in_period == period || blk + 1 == nblk) {
                            in_period = 0;
                            if ((lane & 1) == 0) {
                                int32_t *tp = ttab + gf * C::TROW + gk;
                                int64_t v = (int64_t)*tp + (gsum >> mu);
                                v = v < -(1ll << 29) ? -(1ll << 29) : (v > (1ll << 29) - 1 ? (1ll << 29) - 1 : v);
                                *tp = (int32_t)v;
                            }
                            gsum = 0;
                        }
                    }
                    bar_consumers(C::NCONS);
                }
            }
            bar_all(C::NTHR);
        }
        if (ch.write_state && tid < 8 * K) {
            const int f = tid >> 4, k = tid & 15;
            fr.state[((2 * p + (f >> 2)) * 4 + (f & 3)) * K + k] = ttab[f * C::TROW + k];
        }
        bar_all(C::NTHR);
    }
}

template <int NA, int64_t ALPHA>
size_t serial_smem() {
    return (size_t)SerCfg<NA, ALPHA>::WORDS * sizeof(uint32_t);
}

}  // namespace

size_t aeq_serial_smem_bytes(int na) { return na == 64 ? serial_smem<64, 4080>() : serial_smem<32, 2>(); }

cudaError_t aeq_serial_configure() {
    cudaError_t e = cudaFuncSetAttribute(aeq_serial_kernel<64, 4080>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)serial_smem<64, 4080>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(aeq_serial_kernel<32, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)serial_smem<32, 2>());
    return e;
}

cudaError_t aeq_serial_launch(int na, const DevFrame *frames, const AeqChain *chains, int n_chains, AeqParams prm,
                              int grid, cudaStream_t stream) {
    if (n_chains <= 0) return cudaSuccess;
    const int n_items = 2 * n_chains;
    if (grid <= 0 || grid > n_items) grid = n_items;
    if (na == 64)
        aeq_serial_kernel<64, 4080><<<grid, SerCfg<64, 4080>::NTHR, serial_smem<64, 4080>(), stream>>>(
            frames, chains, n_items, prm);
    else
        aeq_serial_kernel<32, 2><<<grid, SerCfg<32, 2>::NTHR, serial_smem<32, 2>(), stream>>>(frames, chains,
                                                                                               n_items, prm);
    return cudaGetLastError();
}

}  // namespace fnt
