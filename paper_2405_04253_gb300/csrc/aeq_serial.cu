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
//     (n >= K) are decoded (exact by constraint (5)) and stored per task.
//   phase 2 (2 SA threads): y summed over the task rows (weights 128 and 1 for
//     the two tap groups), z = sat16(y >> 7),
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
    static constexpr int WROW = K + 4;                      // split-tap row [filter][group]
    // decoded outputs [task][PROW]; the tasks of output 1 sit 16 words further,
    // so that the two outputs of a symbol are read from opposite bank halves
    static constexpr int PROW = SA + 8;
    static constexpr int NCONS = 256;                       // consumer threads
    static constexpr int NTHR = NCONS + 32;                 // + the producer warp
    // gradient layout: at N = 64 a thread takes one tap of the four filters of
    // an output over 1/8 of the block's symbols (three shuffle stages); at N = 32
    // one tap of one filter over half of them (one shuffle stage)
    static constexpr bool G4 = NA == 64;
    static constexpr int GSYM = G4 ? SA / 8 : SA / 2;       // gradient symbols per thread
    // shared memory (words); every region a multiple of 4 words
    static constexpr int O_WSPL = 0;
    static constexpr int O_XF = O_WSPL + 16 * WROW;
    static constexpr int O_TB = O_XF + 2 * PRE * XBLK;
    static constexpr int O_XS = O_TB + 16 * TT;
    static constexpr int O_PART = O_XS + (2 * XS + 3) / 4 * 4;
    static constexpr int O_EZ = O_PART + 16 * PROW + 16;    // e z_o limb pairs [2][SA]
    static constexpr int WORDS = O_EZ + 4 * SA;
    static_assert(NA % R == 0 && K % NP == 0 && SA % 16 == 0 && R == 8 && GSYM % 2 == 0, "shapes");
    static_assert(O_WSPL % 4 == 0 && O_XF % 4 == 0 && O_TB % 4 == 0 && O_XS % 4 == 0 && O_PART % 4 == 0 &&
                      O_EZ % 4 == 0 && XROW % 4 == 0 && S1STR % 4 == 0 && TT % 4 == 0 && TP % 4 == 0 &&
                      WROW % 4 == 0,
                  "16-byte aligned rows");
    static constexpr int part_row(int task) { return task * PROW + (task >= 8 ? 16 : 0); }
};

__device__ __forceinline__ int32_t sx8s(uint32_t w, int sh) { return (int32_t)(w << (24 - sh)) >> 24; }

__device__ __forceinline__ void cp_async4s(uint32_t *smem, const uint32_t *gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_alls() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One thread's piece of a pointwise product: u[i] <- u[i] X_in[i], the input
// spectrum row read 16 bytes at a time (RedArith in the kernel).
template <class A, int NP>
FNT_HD void piece_products(const A &ar, int32_t (&u)[NP], const int32_t *xrow) {
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
        const int4 x4 = *(const int4 *)(xrow + i);
        u[i] = ar.mulmod(u[i], x4.x);
        u[i + 1] = ar.mulmod(u[i + 1], x4.y);
        u[i + 2] = ar.mulmod(u[i + 2], x4.z);
        u[i + 3] = ar.mulmod(u[i + 3], x4.w);
    }
}

// Byte J of w (J runtime), sign-extended.
__device__ __forceinline__ int32_t sbyte_rt(uint32_t w, uint32_t sel) {
    int32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(w), "r"(sel));
    return r;
}

// Byte j of w, sign-extended (prmt with the sign-replicating selector nibbles).
template <int J>
__device__ __forceinline__ int32_t sbyte(uint32_t w) {
    constexpr uint32_t sel = J | ((8 | J) << 4) | ((8 | J) << 8) | ((8 | J) << 12);
    int32_t r;
    asm("prmt.b32 %0, %1, 0, %2;" : "=r"(r) : "r"(w), "r"(sel));
    return r;
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

// Kept outputs m >= MKEEP (register i of the R-point stage holds group
// m = bitrev_R(i)) of output column n' = q, stored at block position
// n' + NP m - K of the task's row (threads r < NP of the task, one per column).
// A per-pair convolution value c has |c| <= 32512 (constraint (5)) and the
// register holds c + jF with |c + jF| < 2^18; the centred reduction rhoc then
// returns c itself (its result lies within 2^15 + 5 of zero, and c is the only
// representative there), so no further fix-up is needed.
template <class C, int I>
struct StoreOutputs {
    static __device__ __forceinline__ void run(const int32_t (&a)[C::R], int32_t *prow, int q) {
        constexpr int m = bitrev(I, ilog2(C::R));
        if constexpr (m >= C::MKEEP) prow[q + C::NP * m - C::K] = rhoc(a[I]);
        if constexpr (I + 1 < C::R) StoreOutputs<C, I + 1>::run(a, prow, q);
    }
};

template <int NA, int64_t ALPHA>
__global__ void __launch_bounds__(SerCfg<NA, ALPHA>::NTHR, 1)
    aeq_serial_kernel(const DevFrame *__restrict__ frames, const AeqChain *__restrict__ chains, int n_items,
                      AeqParams prm) {
    using C = SerCfg<NA, ALPHA>;
    constexpr int K = C::K, SA = C::SA, R = C::R, NP = C::NP;
    extern __shared__ __align__(16) uint32_t smem[];
    int32_t *wspl = (int32_t *)smem + C::O_WSPL;     // tap groups [filter][g][WROW]: T >> 23, (T >> 16) & 127
    int32_t *xf2 = (int32_t *)smem + C::O_XF;
    int32_t *tb = (int32_t *)smem + C::O_TB;
    uint32_t *xs2 = smem + C::O_XS;
    int32_t *part = (int32_t *)smem + C::O_PART;
    int2 *ez2 = (int2 *)(smem + C::O_EZ);             // e z_o as limbs (c0, c1) [o][SA]

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
    // phase-3 role (C::G4 layout or the N = 32 one).  The lane that ends up
    // with the sum of filter (go, gs1), tap gk owns that master tap: it keeps T
    // in a register, updates it and publishes its two 7-bit groups.
    int go, gk, gsp, gs1;
    bool owner;
    if constexpr (C::G4) {
        go = (warp >> 2) & 1;
        gk = 4 * (warp & 3) + ((lane >> 3) & 3);
        gsp = lane & 7;
        gs1 = 2 * ((gsp >> 2) & 1) + ((gsp >> 1) & 1);
        owner = !producer && (lane & 1) == 0;
    } else {
        gsp = tid & 1;
        gs1 = (tid >> 1) & 3;
        gk = (tid >> 3) & 15;
        go = (tid >> 7) & 1;
        owner = !producer && gsp == 0;
    }
    const int i0 = gsp * C::GSYM;
    const int gb1 = (gsp >> 1) & 1, gb2 = (gsp >> 2) & 1;
    const int gf = 4 * go + gs1;
    const uint32_t gsel = 0x8880u + 0x1111u * (uint32_t)gs1;   // prmt: byte gs1, sign-extended
    int32_t treg = 0;

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const AeqChain ch = chains[item >> 1];
        const int p = item & 1;
        const DevFrame &fr = frames[ch.frame];
        const uint32_t *xin = (const uint32_t *)fr.aeq_in;
        int16_t *out = (int16_t *)fr.out;
        const int64_t nblk = (ch.end - ch.begin + SA - 1) / SA;
        const int64_t nbatch = (nblk + C::PRE - 1) / C::PRE;

        if (owner) {
            treg = ch.init[((2 * p + go) * 4 + gs1) * K + gk];
            wspl[(2 * gf) * C::WROW + gk] = treg >> 23;
            wspl[(2 * gf + 1) * C::WROW + gk] = (treg >> 16) & 127;
        }
        if (producer && nbatch > 0) produce<C>(ch, xin, 0, xs2, xf2, lane);
        bar_all(C::NTHR);

        int64_t gsum = 0;                          // gradient of (go, gs1, gk) over the period
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
                        const int32_t *wrow = wspl + (2 * (4 * po + ps1) + pg) * C::WROW;
                        int32_t w[K];
#pragma unroll
                        for (int q = 0; q < K / 4; ++q) {
                            const int4 t4 = *(const int4 *)(wrow + 4 * q);
                            w[4 * q] = t4.x;
                            w[4 * q + 1] = t4.y;
                            w[4 * q + 2] = t4.z;
                            w[4 * q + 3] = t4.w;
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
                        piece_products(RedArith{}, u, xrow);
                        fnt_inv<NP, C::BETA, 17>(u);
                        int32_t *trows = tb + task * C::TT;
                        trows[r] = rho(u[0]);
#pragma unroll
                        for (int n = 1; n < NP; ++n) trows[n * C::TP + r] = mulred(u[n], twi[n]);
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
                        if (r < NP) StoreOutputs<C, 0>::run(a, part + C::part_row(task), nq);
                    }
                    bar_consumers(C::NCONS);

                    // ---- phase 2: outputs and RDE error; thread (symbol i, output o)
                    if (tid < 2 * SA) {
                        const int i = tid >> 1, o = tid & 1;
                        const int32_t *pc = part + C::part_row(8 * o) + i;
                        int32_t y = 0;              // sum over s1 of 128 c_hi + c_lo (tasks 2 s1 + g)
#pragma unroll
                        for (int t = 0; t < 8; t += 2) y += 128 * pc[t * C::PROW] + pc[(t + 1) * C::PROW];
                        const int32_t z = min(max(y >> 7, -32768), 32767);
                        const int32_t zp = __shfl_xor_sync(0xffffffffu, z, 1);
                        const int32_t z0 = o ? zp : z, z1 = o ? z : zp;
                        const int64_t t = t0 + i;
                        const bool valid = t < ch.end;
                        const int64_t r2 = (int64_t)z0 * z0 + (int64_t)z1 * z1;
                        const int64_t Rr = r2 < 6 * A2 ? 2 * A2 : (r2 < 14 * A2 ? 10 * A2 : 18 * A2);
                        if (o == 0 && valid && t >= ch.keep)
                            *(uint32_t *)(out + t * 4 + 2 * p) = ((uint32_t)z0 & 0xFFFFu) | ((uint32_t)z1 << 16);
                        // e z_o (|e z| <= 2^31 2^15 = 2^46) as a 23-bit low limb and the
                        // signed rest: e z = c1 2^23 + c0, 0 <= c0 < 2^23, |c1| <= 2^23
                        const int64_t ez = valid ? (int64_t)(int32_t)(Rr - r2) * z : 0;
                        ez2[o * SA + i] = make_int2((int32_t)(ez & 0x7FFFFF), (int32_t)(ez >> 23));
                    }
                    bar_consumers(C::NCONS);

                    // ---- phase 3: gradient of eq. (6) and the tap update
                    if (mu < 63) {
                        // word of symbol t0 + i - k (all four inputs) at xw[i]
                        const uint32_t *xw = xs + bb * SA + K - gk;
                        const int2 *ez = ez2 + go * SA + i0;
                        int64_t kv;
                        // G = sum_i (c1_i 2^23 + c0_i) x_i: each limb sum over a thread's
                        // GSYM <= 8 symbols stays below 8 2^23 16 = 2^30, exact in int32
                        if constexpr (C::G4) {
                            int32_t l0[4] = {0, 0, 0, 0}, l1[4] = {0, 0, 0, 0};
#pragma unroll
                            for (int ii = 0; ii < C::GSYM; ii += 2) {
                                const int4 q = *(const int4 *)(ez + ii);     // limbs of symbols i, i + 1
                                const uint32_t wa = xw[i0 + ii], wb = xw[i0 + ii + 1];
                                const int32_t xa[4] = {sbyte<0>(wa), sbyte<1>(wa), sbyte<2>(wa), sbyte<3>(wa)};
                                const int32_t xb[4] = {sbyte<0>(wb), sbyte<1>(wb), sbyte<2>(wb), sbyte<3>(wb)};
#pragma unroll
                                for (int s = 0; s < 4; ++s) {
                                    l0[s] += q.x * xa[s] + q.z * xb[s];
                                    l1[s] += q.y * xa[s] + q.w * xb[s];
                                }
                            }
                            int64_t acc[4];
#pragma unroll
                            for (int s = 0; s < 4; ++s) acc[s] = ((int64_t)l1[s] << 23) + l0[s];
                            // sum over the 8 symbol ranges (lane bits 0..2); the lane
                            // keeps input s1 = 2 b2 + b1
                            int64_t k01 = gb2 ? acc[2] : acc[0], k11 = gb2 ? acc[3] : acc[1];
                            const int64_t s01 = gb2 ? acc[0] : acc[2], s11 = gb2 ? acc[1] : acc[3];
                            k01 += __shfl_xor_sync(0xffffffffu, s01, 4);
                            k11 += __shfl_xor_sync(0xffffffffu, s11, 4);
                            kv = gb1 ? k11 : k01;
                            kv += __shfl_xor_sync(0xffffffffu, gb1 ? k01 : k11, 2);
                            kv += __shfl_xor_sync(0xffffffffu, kv, 1);
                        } else {
                            int32_t l0 = 0, l1 = 0;
#pragma unroll
                            for (int ii = 0; ii < C::GSYM; ii += 2) {
                                const int4 q = *(const int4 *)(ez + ii);
                                const int32_t xa = sbyte_rt(xw[i0 + ii], gsel), xb = sbyte_rt(xw[i0 + ii + 1], gsel);
                                l0 += q.x * xa + q.z * xb;
                                l1 += q.y * xa + q.w * xb;
                            }
                            kv = ((int64_t)l1 << 23) + l0;
                            kv += __shfl_xor_sync(0xffffffffu, kv, 1);    // the two symbol halves
                        }
                        gsum += kv;
                        if (++in_period == period || blk + 1 == nblk) {
                            in_period = 0;
                            if (owner) {
                                int64_t v = (int64_t)treg + (gsum >> mu);
                                v = v < -(1ll << 29) ? -(1ll << 29) : (v > (1ll << 29) - 1 ? (1ll << 29) - 1 : v);
                                treg = (int32_t)v;
                                wspl[(2 * gf) * C::WROW + gk] = treg >> 23;
                                wspl[(2 * gf + 1) * C::WROW + gk] = (treg >> 16) & 127;
                            }
                            gsum = 0;
                        }
                    }
                    bar_consumers(C::NCONS);
                }
            }
            bar_all(C::NTHR);
        }
        if (ch.write_state && owner) fr.state[((2 * p + go) * 4 + gs1) * K + gk] = treg;
        bar_all(C::NTHR);
    }
}

template <int NA, int64_t ALPHA>
size_t serial_smem() {
    return (size_t)SerCfg<NA, ALPHA>::WORDS * sizeof(uint32_t);
}

}  // namespace

// Pointwise products per AEQ block of both polarisations on this kernel: the
// 16 R threads of a polarisation's phase 1 each run the product stage of their
// N/R-point piece once per block (the stage counted on the host).
template <int NA, int64_t ALPHA>
static int serial_mults_per_block() {
    using C = SerCfg<NA, ALPHA>;
    int mults = 0, shifts = 0;
    int32_t u[C::NP] = {}, x[C::NP] = {};
    piece_products(CountArith{&mults, &shifts}, u, x);
    return 2 * 16 * C::R * mults;
}

int aeq_serial_mults_per_block(int na) {
    return na == 64 ? serial_mults_per_block<64, 4080>() : serial_mults_per_block<32, 2>();
}

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
