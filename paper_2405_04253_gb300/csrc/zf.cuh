// zf.cuh -- arithmetic in Z_F, F = 2^16 + 1 = 65537, and per-thread length-N
// Fermat number transforms (eq. (1) / eq. (2) of the paper, section "Fermat
// number transform") for sm_103a.
//
// Representation.  Values are int32 "lazy residues": any x with x = v (mod F)
// and |x| < 2^17 stands for the residue v.  Reduction by a Fermat modulus is
// split-and-subtract: t = h * 2^16 + l  ==>  t = l - h (mod F), because
// 2^16 = -1 (mod F).  On the GPU that is one shift and one multiply-add:
//     rho(t)  = t - (t >> 16) * F                      -> [-32767, 98303]
//     rhoc(t) = t - ((t + 2^15) >> 16) * F             -> |r| <= 2^15 + |t| / 2^16
// (the multiply runs on the FMA pipe, the shift on the integer pipe).
//
// Transforms.  One thread owns a whole length-N transform in N registers; every
// index and twiddle is a compile-time constant after unrolling, so "bit-reversed
// order" costs nothing.  The radix-2 decimation-in-frequency network
// (a, b) -> (a + b, (a - b) w) takes natural order and leaves X[k] in register
// bitrev(k).  The inverse runs the same network with alpha^-1 through a
// bit-reversed view of the registers, which consumes bit-reversed spectra and
// leaves natural-order samples.  Twiddles are stored as centred residues
// (|w| <= 2^15); the powers of the radix sqrt(2) = 4080 or 2 make most of them
// small powers of two, which keeps most products inside 32 bits without a
// pre-reduction.
#pragma once

#include <cstdint>

#ifndef FNT_HD
#define FNT_HD __host__ __device__ __forceinline__
#endif

namespace fnt {

constexpr int32_t kF = 65537;

constexpr int64_t zmod(int64_t v) { return ((v % kF) + kF) % kF; }

constexpr int64_t zpow(int64_t a, int64_t e) {
    int64_t r = 1, b = zmod(a);
    while (e > 0) {
        if (e & 1) r = r * b % kF;
        b = b * b % kF;
        e >>= 1;
    }
    return r;
}

constexpr int64_t zinv(int64_t a) { return zpow(a, kF - 2); }   // F is prime

// Centred representative in [-32768, 32768].
constexpr int32_t zcent(int64_t v) {
    int64_t r = zmod(v);
    return r > 32768 ? (int32_t)(r - kF) : (int32_t)r;
}

constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }

constexpr int bitrev(int i, int bits) {
    int r = 0;
    for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
    return r;
}

// Centred powers alpha^e, e in [0, N).
template <int N, int64_t ALPHA>
struct Twiddles {
    int32_t w[N];
    constexpr Twiddles() : w() {
        for (int e = 0; e < N; ++e) w[e] = zcent(zpow(ALPHA, e));
    }
};

template <int N, int64_t ALPHA>
struct TwTab {
    static constexpr Twiddles<N, ALPHA> tab{};
};

// ------------------------------------------------------------- reductions ----

FNT_HD int32_t rho(int32_t t) {
    // l - h with t = h * 2^16 + l; exact in wrapping 32-bit arithmetic because the
    // result fits in int32.
    return (int32_t)((uint32_t)t - (uint32_t)(t >> 16) * (uint32_t)kF);
}

FNT_HD int32_t rhoc(int32_t t) {
    // requires |t| < 2^31 - 2^15
    return (int32_t)((uint32_t)t - (uint32_t)((t + 32768) >> 16) * (uint32_t)kF);
}

// Exact signed value of a residue whose true integer value v satisfies
// |v| <= 32768 (constraint (5)), from any lazy x = v (mod F) with |x| < 2^24.
FNT_HD int32_t decode(int32_t x) {
    int32_t r = rhoc(x);                 // |r| <= 32768 + 256
    r = r > 32768 ? r - kF : r;
    r = r < -32768 ? r + kF : r;
    return r;
}

// Multiply a lazy residue (|x| < 2^18) by a centred compile-time constant.
template <int32_t W>
FNT_HD int32_t mulc(int32_t x) {
    if constexpr (W == 1) {
        return rho(x);
    } else if constexpr (W == -1) {
        return rho(-x);
    } else if constexpr (W <= 4096 && W >= -4096) {
        return rho(x * W);               // |x W| < 2^30
    } else {
        return rho(rhoc(x) * W);         // |rhoc(x)| <= 2^15 + 4, |W| <= 2^15
    }
}

// Runtime variant for a centred constant w (|w| <= 2^15) and |x| < 2^30.
FNT_HD int32_t mulw(int32_t x, int32_t w) { return rho(rhoc(x) * w); }

// -------------------------------------------------------------- transforms ----

// One DIF butterfly with twiddle index e of a length-N network of radix ALPHA.
template <int N, int64_t ALPHA, int E>
FNT_HD void bfly(int32_t &a, int32_t &b) {
    constexpr int32_t W = TwTab<N, ALPHA>::tab.w[E];
    const int32_t s = a + b;
    const int32_t d = a - b;
    a = rho(s);
    b = mulc<W>(d);
}

template <int N, int64_t ALPHA, bool BR, int S, int J>
struct DifStage {
    static FNT_HD void run(int32_t (&x)[N]) {
        constexpr int LOGN = ilog2(N);
        constexpr int HALF = N >> (S + 1);
        constexpr int BLK = J / HALF;
        constexpr int JJ = J % HALF;
        constexpr int I0 = BLK * 2 * HALF + JJ;
        constexpr int I1 = I0 + HALF;
        constexpr int R0 = BR ? bitrev(I0, LOGN) : I0;
        constexpr int R1 = BR ? bitrev(I1, LOGN) : I1;
        bfly<N, ALPHA, (JJ << S)>(x[R0], x[R1]);
        if constexpr (J + 1 < N / 2) DifStage<N, ALPHA, BR, S, J + 1>::run(x);
    }
};

template <int N, int64_t ALPHA, bool BR, int S>
struct Dif {
    static FNT_HD void run(int32_t (&x)[N]) {
        DifStage<N, ALPHA, BR, S, 0>::run(x);
        if constexpr (S + 1 < ilog2(N)) Dif<N, ALPHA, BR, S + 1>::run(x);
    }
};

// Forward transform, eq. (1) without the final reduction: natural order in
// (|x| < 2^17), X[k] in register bitrev(k) out (|X| < 2^17).
template <int N, int64_t ALPHA>
FNT_HD void fnt_fwd(int32_t (&x)[N]) {
    Dif<N, ALPHA, false, 0>::run(x);
}

// Inverse transform, eq. (2) without the factor N^-1: P[k] in register
// bitrev(k) in, p[n] in register n out.
template <int N, int64_t ALPHA>
FNT_HD void fnt_inv(int32_t (&x)[N]) {
    Dif<N, zinv(ALPHA), true, 0>::run(x);
}

// Forward transform of a sequence whose entries NZ..N-1 are zero (NZ <= N/2):
// the first stage reduces to (a, a * w).
template <int N, int64_t ALPHA, int J>
struct DifFirstZeroPad {
    static FNT_HD void run(int32_t (&x)[N]) {
        constexpr int32_t W = TwTab<N, ALPHA>::tab.w[J];
        x[J + N / 2] = mulc<W>(x[J]);
        if constexpr (J + 1 < N / 2) DifFirstZeroPad<N, ALPHA, J + 1>::run(x);
    }
};

template <int N, int64_t ALPHA>
FNT_HD void fnt_fwd_halfzero(int32_t (&x)[N]) {
    DifFirstZeroPad<N, ALPHA, 0>::run(x);
    if constexpr (N > 2) Dif<N, ALPHA, false, 1>::run(x);
}

}  // namespace fnt
