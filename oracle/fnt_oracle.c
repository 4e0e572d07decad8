/*
 * fnt_oracle.c -- plain, slow, CPU reference for the FNT-CDC / FNT-AEQ path of
 * "Fermat Number Transform Based Chromatic Dispersion Compensation and Adaptive
 * Equalization Algorithm" (arXiv 2405.04253).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check of the package
 * entry module and the CPU-baseline leg of the benchmark may build, load or call
 * this file.  It shares no code, header, table or constant with the CUDA library;
 * every value it needs it derives here from the equations.
 *
 * Everything is int64 and every transform is the literal O(N^2) sum of eq. (1) /
 * eq. (2).  No blocking, fusion or reordering beyond what the equations state.
 *
 * Parity status (see the pins in the test suite):
 *   orc_fnt / orc_ifnt / field helpers  pinned (closed forms, 8-point mod-17
 *                                       worked case of Fig. 1, brute-force cyclic
 *                                       convolution, round trip)
 *   orc_cdc                             pinned (equals exact integer linear
 *                                       convolution, computed by numpy)
 *   orc_requant_decimate                pinned (hand-worked cases)
 *   orc_cdc_shift                       pinned (hand-worked cases; on the
 *                                       synthetic 75 km link the AEQ input
 *                                       stays within the ADC's loading)
 *   orc_aeq, mu = 0                     pinned (equals exact 4x4 integer MIMO
 *                                       convolution, computed by numpy)
 *   orc_aeq, adaptive                   pinned: the one-block gradient against a
 *                                       float64 finite-difference derivative of
 *                                       the RDE cost; the gradient summed over
 *                                       many blocks (x[t-k] across block
 *                                       boundaries and into the input history,
 *                                       whole runs and segments) against a numpy
 *                                       closed form of eq. (6); the update
 *                                       period rebuilt period by period
 */
#include "fnt_oracle.h"

#include <stdlib.h>
#include <string.h>

typedef long long i64;

/* ---------------------------------------------------------------- field ---- */

/* a mod F in [0, F). */
static i64 md(i64 a, i64 F) {
    i64 r = a % F;
    return r < 0 ? r + F : r;
}

i64 orc_powmod(i64 a, i64 e, i64 F) {
    i64 r = 1 % F, b = md(a, F);
    while (e > 0) {
        if (e & 1) r = (r * b) % F;
        b = (b * b) % F;
        e >>= 1;
    }
    return r;
}

/* Inverse by the extended Euclidean algorithm; returns -1 when gcd(a, F) != 1. */
i64 orc_invmod(i64 a, i64 F) {
    i64 r0 = F, r1 = md(a, F), t0 = 0, t1 = 1;
    while (r1 != 0) {
        i64 q = r0 / r1, tmp;
        tmp = r0 - q * r1; r0 = r1; r1 = tmp;
        tmp = t0 - q * t1; t0 = t1; t1 = tmp;
    }
    if (r0 != 1) return -1;
    return md(t0, F);
}

/* Multiplicative order of alpha mod F (0 if alpha is not a unit). */
i64 orc_order(i64 alpha, i64 F) {
    i64 a = md(alpha, F), x = a;
    if (orc_invmod(a, F) < 0) return 0;
    for (i64 k = 1; k <= F; ++k) {
        if (x == 1) return k;
        x = (x * a) % F;
    }
    return 0;
}

/* Eqs. (3)-(4) for a prime modulus, plus the two conditions the transform pair
 * (1)-(2) needs to be mutually inverse: alpha of order exactly N and N invertible.
 * Returns 0 when (N, alpha, F) defines a valid length-N transform. */
int orc_check_transform(int N, i64 alpha, i64 F) {
    if (N <= 0 || F < 3) return 1;
    if (orc_powmod(alpha, N, F) != 1) return 2;          /* eq. (4) */
    if (orc_order(alpha, F) != N) return 3;
    if (orc_invmod(N, F) < 0) return 4;
    return 0;
}

/* Signed representative: the residue r in [0, F) stands for r when r <= (F-1)/2
 * and for r - F otherwise.  Constraint (5) is what makes this the true value. */
i64 orc_decode(i64 r, i64 F) {
    r = md(r, F);
    return r <= (F - 1) / 2 ? r : r - F;
}

/* ------------------------------------------------------------ transforms ---- */

/* Eq. (1): X(k) = sum_n x(n) alpha^(nk) mod F. */
void orc_fnt(const i64 *x, i64 *X, int N, i64 alpha, i64 F) {
    for (int k = 0; k < N; ++k) {
        i64 acc = 0;
        for (int n = 0; n < N; ++n) {
            i64 w = orc_powmod(alpha, (i64)n * k % N, F);
            acc = (acc + md(x[n], F) * w) % F;
        }
        X[k] = acc;
    }
}

/* Eq. (2): x(n) = N^-1 sum_k X(k) alpha^(-nk) mod F. */
void orc_ifnt(const i64 *X, i64 *x, int N, i64 alpha, i64 F) {
    i64 ainv = orc_invmod(alpha, F);
    i64 ninv = orc_invmod(N, F);
    for (int n = 0; n < N; ++n) {
        i64 acc = 0;
        for (int k = 0; k < N; ++k) {
            i64 w = orc_powmod(ainv, (i64)n * k % N, F);
            acc = (acc + md(X[k], F) * w) % F;
        }
        x[n] = (acc * ninv) % F;
    }
}

/* The same two sums with a precomputed power table, for the long loops below.
 * tab[e] = alpha^e mod F for e in [0, N); itab[e] = alpha^-e mod F. */
typedef struct {
    int N;
    i64 F;
    i64 ninv;
    i64 *tab;
    i64 *itab;
} xform;

static int xform_init(xform *t, int N, i64 alpha, i64 F) {
    if (orc_check_transform(N, alpha, F) != 0) return 1;
    t->N = N;
    t->F = F;
    t->ninv = orc_invmod(N, F);
    t->tab = (i64 *)malloc(sizeof(i64) * N);
    t->itab = (i64 *)malloc(sizeof(i64) * N);
    i64 ainv = orc_invmod(alpha, F);
    for (int e = 0; e < N; ++e) {
        t->tab[e] = orc_powmod(alpha, e, F);
        t->itab[e] = orc_powmod(ainv, e, F);
    }
    return 0;
}

static void xform_free(xform *t) {
    free(t->tab);
    free(t->itab);
}

static void xfnt(const xform *t, const i64 *x, i64 *X) {
    const int N = t->N;
    for (int k = 0; k < N; ++k) {
        i64 acc = 0;
        for (int n = 0; n < N; ++n) acc = (acc + x[n] * t->tab[(n * k) % N]) % t->F;
        X[k] = acc;
    }
}

static void xifnt(const xform *t, const i64 *X, i64 *x) {
    const int N = t->N;
    for (int n = 0; n < N; ++n) {
        i64 acc = 0;
        for (int k = 0; k < N; ++k) acc = (acc + X[k] * t->itab[(n * k) % N]) % t->F;
        x[n] = (acc * t->ninv) % t->F;
    }
}

/* ------------------------------------------------------------------- CDC ---- */

/*
 * FNT-CDC (section "Proposed FNT-CDC&AEQ structure", eqs. (5), (7), (8)).
 *
 * in   : int8 [n][n_pol][2]  (I, Q) 5-bit signed samples
 * taps : int8 [L][2]         (re, im) 6-bit signed CD taps, same for every pol
 * out  : int32 [n][n_pol][2] z[t] = sum_k h[k] x[t-k] (x = 0 outside [0, n))
 *
 * Overlap-save: block b takes the N samples starting at b*S - (N - S) (zeros
 * outside the frame), its circular convolution with the zero-padded taps is exact
 * linear convolution at positions j >= L-1, and the last S positions are kept.
 * Per block and polarization, following the paper's notation (q = 16):
 *   X = FNT(Re x), Xh = FNT(Im x), Y = FNT(Re h), Yh = FNT(Im h)
 *   P = (X + 2^(q/2) Xh)(Y + 2^(q/2) Yh),  M = (X - 2^(q/2) Xh)(Y - 2^(q/2) Yh)
 *   Re z = -2^(q-1)   IFNT{P + M}          eq. (7)
 *   Im z = -2^(q/2-1) IFNT{P - M}          eq. (8)
 * then the signed decode.  Returns 0 on success.
 */
int orc_cdc(const int8_t *in, i64 n, int n_pol, const int8_t *taps, int L,
            int N, i64 alpha, int S, int32_t *out) {
    const i64 F = 65537;
    const i64 q = 16;
    if (n < 0 || (n_pol != 1 && n_pol != 2) || L < 1 || S < 1 || S > N - L + 1) return 1;
    xform t;
    if (xform_init(&t, N, alpha, F) != 0) return 2;
    const i64 j = orc_powmod(2, q / 2, F);                 /* 2^(q/2); j^2 = -1 */
    const i64 c_re = md(-orc_powmod(2, q - 1, F), F);      /* -2^(q-1)   */
    const i64 c_im = md(-orc_powmod(2, q / 2 - 1, F), F);  /* -2^(q/2-1) */

    i64 *hr = calloc(N, sizeof(i64)), *hi = calloc(N, sizeof(i64));
    i64 *Y = malloc(N * sizeof(i64)), *Yh = malloc(N * sizeof(i64));
    i64 *xr = malloc(N * sizeof(i64)), *xi = malloc(N * sizeof(i64));
    i64 *X = malloc(N * sizeof(i64)), *Xh = malloc(N * sizeof(i64));
    i64 *A = malloc(N * sizeof(i64)), *B = malloc(N * sizeof(i64));
    i64 *a = malloc(N * sizeof(i64)), *b = malloc(N * sizeof(i64));
    for (int k = 0; k < L; ++k) {
        hr[k] = md(taps[2 * k], F);
        hi[k] = md(taps[2 * k + 1], F);
    }
    xfnt(&t, hr, Y);
    xfnt(&t, hi, Yh);

    const i64 nblk = (n + S - 1) / S;
    for (int p = 0; p < n_pol; ++p) {
        for (i64 blk = 0; blk < nblk; ++blk) {
            const i64 start = blk * S - (N - S);
            for (int m = 0; m < N; ++m) {
                const i64 s = start + m;
                if (s >= 0 && s < n) {
                    xr[m] = md(in[(s * n_pol + p) * 2], F);
                    xi[m] = md(in[(s * n_pol + p) * 2 + 1], F);
                } else {
                    xr[m] = xi[m] = 0;
                }
            }
            xfnt(&t, xr, X);
            xfnt(&t, xi, Xh);
            for (int k = 0; k < N; ++k) {
                i64 ux = (X[k] + j * Xh[k]) % F, uy = (Y[k] + j * Yh[k]) % F;
                i64 vx = md(X[k] - j * Xh[k], F), vy = md(Y[k] - j * Yh[k], F);
                i64 P = ux * uy % F, M = vx * vy % F;
                A[k] = (P + M) % F;
                B[k] = md(P - M, F);
            }
            xifnt(&t, A, a);
            xifnt(&t, B, b);
            for (int m = N - S; m < N; ++m) {
                const i64 s = start + m;
                if (s < 0 || s >= n) continue;
                out[(s * n_pol + p) * 2] = (int32_t)orc_decode(c_re * a[m] % F, F);
                out[(s * n_pol + p) * 2 + 1] = (int32_t)orc_decode(c_im * b[m] % F, F);
            }
        }
    }
    free(hr); free(hi); free(Y); free(Yh); free(xr); free(xi); free(X); free(Xh);
    free(A); free(B); free(a); free(b);
    xform_free(&t);
    return 0;
}

/* --------------------------------------------------- requant + resample ---- */

static i64 clampll(i64 v, i64 lo, i64 hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor(v / 2^s) for any sign. */
static i64 floor_shift(i64 v, int s) {
    if (s <= 0) return v;
    if (s >= 63) return v < 0 ? -1 : 0;
    i64 d = (i64)1 << s;
    i64 q = v / d;
    if ((v % d) != 0 && v < 0) q -= 1;
    return q;
}


/* CDC -> AEQ requantisation shift s_c (the paper fixes only the 5-bit signal
 * width): with E = sum_k (h_re[k]^2 + h_im[k]^2), s_c is the smallest s >= 0
 * with 4^s >= 2 E, i.e. 2^s >= sqrt(2 E).  CD taps designed for a signal that
 * fills about half of the sampled band have an in-band gain near sqrt(2 E)
 * (sqrt(E) is their gain on white input), so the 5-bit AEQ input keeps at
 * most the 5-bit CDC input's loading and does not saturate.  E = 0 gives 0. */
int orc_cdc_shift(const int8_t *taps, int L) {
    i64 E = 0;
    for (int k = 0; k < L; ++k) E += (i64)taps[2 * k] * taps[2 * k] + (i64)taps[2 * k + 1] * taps[2 * k + 1];
    int s = 0;
    while (E > 0 && ((i64)1 << (2 * s)) < 2 * E) ++s;
    return s;
}

/* Decimation phase (2 sps -> 1 sps keeps times t = phase mod 2): the parity of
 * the CD filter's centre delay (L-1)/2. */
int orc_decim_phase(int L) { return ((L - 1) / 2) & 1; }

static int32_t sat5(i64 v) { return v < -16 ? -16 : (v > 15 ? 15 : (int32_t)v); }

/*
 * z    : int32 [n][2][2] CDC output (PDM)
 * x    : int8  [n_sym][4] AEQ input (XI, XQ, YI, YQ), n_sym = count of t in
 *        [0, n) with t = phase mod 2.
 * x = sat[-16, 15]( floor((z + 2^(s-1)) / 2^s) )   (s = 0: no rounding term)
 */
i64 orc_requant_decimate(const int32_t *z, i64 n, int shift, int phase, int8_t *x) {
    i64 m = 0;
    const i64 rnd = shift > 0 ? ((i64)1 << (shift - 1)) : 0;
    for (i64 t = phase; t < n; t += 2, ++m) {
        for (int c = 0; c < 4; ++c) {
            x[m * 4 + c] = (int8_t)sat5(floor_shift((i64)z[t * 4 + c] + rnd, shift));
        }
    }
    return m;
}

/* ------------------------------------------------------------------- AEQ ---- */

void orc_aeq_init_taps(int K, int w0, int32_t *T) {
    memset(T, 0, sizeof(int32_t) * 16 * K);
    for (int s = 0; s < 4; ++s) T[(s * 4 + s) * K + K / 2] = (int32_t)((i64)w0 << 16);
}

/*
 * FNT-AEQ with RDE tap update (eq. (6)); 4x4 real-valued MIMO over the streams
 * S in {XI, XQ, YI, YQ} = {0, 1, 2, 3}.
 *
 * x   : int8  [n_sym][4] 5-bit input at 1 sample/symbol
 * T   : int32 [4 (S2)][4 (S1)][K] master taps (16 fractional bits above the
 *       14-bit tap), read at entry and holding the adapted taps at exit
 * out : int16 [n_sym][4]
 * use_fnt = 1: every convolution through eqs. (1)-(2) (the method);
 * use_fnt = 0: the same convolutions as direct integer sums (the cross-check).
 *
 * Block b (step S = N - K) outputs times [bS, bS + S).  With W = T >> 16 (14-bit),
 * the two 7-bit groups are W_hi = W >> 7 (signed) and W_lo = W & 127 (unsigned),
 * so W = 128 W_hi + W_lo.  Per pair S1 -> S2 and group g the circular convolution
 * of the window [bS - (N - S), bS + S) with the zero-padded group taps is taken
 * through FNT, product and IFNT, decoded to a signed value and weighted:
 *   y_S2[t] = sum_S1 (128 c_hi[t] + c_lo[t]),   z_S2[t] = sat16(floor(y / 2^7)).
 * RDE error for pol p with r^2 = z_pI^2 + z_pQ^2: R = 2A^2 if r^2 < 6A^2, 10A^2 if
 * r^2 < 14A^2, else 18A^2 (the 16QAM rings); e_p = R - r^2.  After the block,
 *   G[S2][S1][k] = sum_t e_p(S2)[t] z_S2[t] x_S1[t - k]   (valid t of the block)
 *   T <- clamp(T + floor(G / 2^m), -2^29, 2^29 - 1).
 * m >= 63 stands for mu = 0 (taps held fixed).  With an update period P > 1
 * (the paper updates every step, P = 1) G is summed over P blocks and the
 * update is applied after every P-th block and after the last block; the taps
 * stay fixed in between.
 * freq_sum (FNT path only): 0 = one IFNT per (input, output, group), as in
 * the default reading; 1 = the products of the four inputs are summed in Z_F
 * before one IFNT per (output, group), which wraps when constraint (5) fails
 * for the sum; 2 = as 1 for a block and polarisation only where 16 times the
 * sum of |tap group values| over the four inputs is at most 32767 (every
 * output decodes exactly), otherwise as 0.
 * hist: symbols x[-hist .. -1] precede the run and are read as its input
 * history (windows and gradient); before them the history is zero.  No output
 * is produced for them and they take no part in the updates.  Returns 0 on
 * success.
 */
int orc_aeq(const int8_t *x, i64 n_sym, int N, i64 alpha, int K, int mu_shift, int rde_a,
            int32_t *T, int16_t *out, int use_fnt, int period, int freq_sum, int hist) {
    const i64 F = 65537;
    const int S = N - K;
    if (n_sym < 0 || K < 1 || S < 1 || N > 256 || mu_shift < 0 || rde_a < 1 || period < 1) return 1;
    if (freq_sum < 0 || freq_sum > 2 || (freq_sum == 1 && !use_fnt)) return 3;
    if (hist < 0) return 1;
    xform t;
    if (use_fnt && xform_init(&t, N, alpha, F) != 0) return 2;
    const i64 A2 = (i64)rde_a * rde_a;

    i64 *win = malloc(sizeof(i64) * N * 4);      /* [S1][N] windows (residues)    */
    i64 *Xf = malloc(sizeof(i64) * N * 4);       /* [S1][N] FNT of the windows    */
    i64 *wv = malloc(sizeof(i64) * N);
    i64 *Wf = malloc(sizeof(i64) * N);
    i64 *P = malloc(sizeof(i64) * N);
    i64 *Psum = malloc(sizeof(i64) * N);
    i64 *c = malloc(sizeof(i64) * N);
    i64 *y = malloc(sizeof(i64) * S * 4);
    i64 *z = malloc(sizeof(i64) * S * 4);
    i64 *e = malloc(sizeof(i64) * S * 2);
    int *W = malloc(sizeof(int) * 16 * K);
    i64 *Gacc = calloc(16 * K, sizeof(i64));     /* gradient summed over the update period */

    const i64 nblk = (n_sym + S - 1) / S;
    for (i64 blk = 0; blk < nblk; ++blk) {
        const i64 t0 = blk * S;
        const i64 start = t0 - (N - S);
        const int nvalid = (int)((n_sym - t0) < S ? (n_sym - t0) : S);

        for (int f = 0; f < 16 * K; ++f) W[f] = (int)floor_shift(T[f], 16);

        for (int s1 = 0; s1 < 4; ++s1)
            for (int m = 0; m < N; ++m) {
                const i64 tt = start + m;
                win[s1 * N + m] = (tt >= -hist && tt < n_sym) ? x[tt * 4 + s1] : 0;
            }
        if (use_fnt) {
            for (int s1 = 0; s1 < 4; ++s1) {
                i64 tmp[256];
                for (int m = 0; m < N; ++m) tmp[m] = md(win[s1 * N + m], F);
                xfnt(&t, tmp, Xf + s1 * N);
            }
        }

        /* frequency-domain summation over the inputs (freq_sum 1, or 2 when the
           block's guard holds for the polarisation): 16 * sum |taps of a group|
           over the four inputs bounds the summed convolution (|x| <= 16) */
        int sum_pol[2] = {freq_sum == 1, freq_sum == 1};
        if (freq_sum == 2) {
            for (int p = 0; p < 2; ++p) {
                int ok = 1;
                for (int s2 = 2 * p; s2 < 2 * p + 2; ++s2)
                    for (int g = 0; g < 2; ++g) {
                        i64 l1 = 0;
                        for (int s1 = 0; s1 < 4; ++s1)
                            for (int k = 0; k < K; ++k) {
                                const int wk = W[(s2 * 4 + s1) * K + k];
                                const i64 v = g == 0 ? floor_shift(wk, 7) : (i64)(wk & 127);
                                l1 += v < 0 ? -v : v;
                            }
                        if (16 * l1 > 32767) ok = 0;
                    }
                sum_pol[p] = ok;
            }
        }

        memset(y, 0, sizeof(i64) * S * 4);
        for (int s2 = 0; s2 < 4; ++s2)
            for (int g = 0; g < 2; ++g) {
                const i64 weight = g == 0 ? 128 : 1;
                const int summed = use_fnt && sum_pol[s2 / 2];
                if (summed)
                    for (int k = 0; k < N; ++k) Psum[k] = 0;
                for (int s1 = 0; s1 < 4; ++s1) {
                    const int *w = W + (s2 * 4 + s1) * K;
                    for (int m = 0; m < N; ++m) {
                        i64 v = 0;
                        if (m < K) v = g == 0 ? floor_shift(w[m], 7) : (i64)(w[m] & 127);
                        wv[m] = v;
                    }
                    if (summed) {
                        for (int m = 0; m < N; ++m) wv[m] = md(wv[m], F);
                        xfnt(&t, wv, Wf);
                        for (int k = 0; k < N; ++k) Psum[k] = (Psum[k] + Xf[s1 * N + k] * Wf[k]) % F;
                    } else if (use_fnt) {
                        for (int m = 0; m < N; ++m) wv[m] = md(wv[m], F);
                        xfnt(&t, wv, Wf);
                        for (int k = 0; k < N; ++k) P[k] = Xf[s1 * N + k] * Wf[k] % F;
                        xifnt(&t, P, c);
                        for (int i = 0; i < S; ++i) y[s2 * S + i] += weight * orc_decode(c[N - S + i], F);
                    } else {
                        for (int i = 0; i < S; ++i) {
                            const int m = N - S + i;
                            i64 acc = 0;
                            for (int k = 0; k < K; ++k)
                                if (m - k >= 0) acc += wv[k] * win[s1 * N + m - k];
                            y[s2 * S + i] += weight * acc;
                        }
                    }
                }
                if (summed) {
                    xifnt(&t, Psum, c);
                    for (int i = 0; i < S; ++i) y[s2 * S + i] += weight * orc_decode(c[N - S + i], F);
                }
            }

        for (int i = 0; i < nvalid; ++i) {
            for (int s2 = 0; s2 < 4; ++s2) {
                z[s2 * S + i] = clampll(floor_shift(y[s2 * S + i], 7), -32768, 32767);
                out[(t0 + i) * 4 + s2] = (int16_t)z[s2 * S + i];
            }
            for (int p = 0; p < 2; ++p) {
                const i64 zi = z[(2 * p) * S + i], zq = z[(2 * p + 1) * S + i];
                const i64 r2 = zi * zi + zq * zq;
                const i64 R = r2 < 6 * A2 ? 2 * A2 : (r2 < 14 * A2 ? 10 * A2 : 18 * A2);
                e[p * S + i] = R - r2;
            }
        }

        /* the update is applied after every period-th block and after the last one */
        const int apply = ((blk + 1) % period == 0) || (blk == nblk - 1);
        for (int s2 = 0; s2 < 4; ++s2)
            for (int s1 = 0; s1 < 4; ++s1)
                for (int k = 0; k < K; ++k) {
                    i64 G = 0;
                    for (int i = 0; i < nvalid; ++i) {
                        const i64 tt = t0 + i - k;
                        const i64 xv = tt >= -hist ? x[tt * 4 + s1] : 0;
                        G += e[(s2 / 2) * S + i] * z[s2 * S + i] * xv;
                    }
                    const int f = (s2 * 4 + s1) * K + k;
                    Gacc[f] += G;
                    if (!apply) continue;
                    const i64 Gp = Gacc[f];
                    Gacc[f] = 0;
                    if (mu_shift >= 63) continue;               /* mu = 0: fixed taps */
                    T[f] = (int32_t)clampll((i64)T[f] + floor_shift(Gp, mu_shift), -((i64)1 << 29),
                                            ((i64)1 << 29) - 1);
                }
    }
    free(Gacc);
    free(win); free(Xf); free(wv); free(Wf); free(P); free(Psum); free(c); free(y); free(z); free(e); free(W);
    if (use_fnt) xform_free(&t);
    return 0;
}

/*
 * Segmented AEQ for long streams (the paper is silent on streams longer than
 * its offline captures): output segment s covers times [s*L, min((s+1)*L, n));
 * its AEQ run starts `warmup` symbols earlier (at most at 0) from the taps T0,
 * reads the K stream symbols before its start as input history (zero before
 * the stream), and only the segment's own times are kept.  With fixed taps a
 * segment therefore reproduces the unsegmented outputs exactly.  seg_len <= 0
 * means one unsegmented run.  T_out (may be NULL) receives the last segment's
 * final taps.
 */
int orc_aeq_segmented(const int8_t *x, i64 n_sym, int N, i64 alpha, int K, int mu_shift,
                      int rde_a, const int32_t *T0, i64 seg_len, i64 warmup, int32_t *T_out,
                      int16_t *out, int use_fnt, int period, int freq_sum) {
    int32_t *T = malloc(sizeof(int32_t) * 16 * K);
    int rc = 0;
    if (seg_len <= 0) seg_len = n_sym > 0 ? n_sym : 1;
    const i64 nseg = (n_sym + seg_len - 1) / seg_len;
    for (i64 s = 0; s < nseg && rc == 0; ++s) {
        const i64 keep = s * seg_len;
        const i64 end = keep + seg_len < n_sym ? keep + seg_len : n_sym;
        const i64 begin = keep - warmup > 0 ? keep - warmup : 0;
        const int hist = begin < K ? (int)begin : K;            /* the stream's preceding symbols */
        int16_t *tmp = malloc(sizeof(int16_t) * 4 * (end - begin));
        memcpy(T, T0, sizeof(int32_t) * 16 * K);
        rc = orc_aeq(x + begin * 4, end - begin, N, alpha, K, mu_shift, rde_a, T, tmp, use_fnt, period,
                     freq_sum, hist);
        memcpy(out + keep * 4, tmp + (keep - begin) * 4, sizeof(int16_t) * 4 * (end - keep));
        free(tmp);
    }
    if (T_out) memcpy(T_out, nseg > 0 ? T : T0, sizeof(int32_t) * 16 * K);
    free(T);
    return rc;
}
