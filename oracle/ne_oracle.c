/*
 * ne_oracle.c -- plain, slow, obviously-correct CPU oracle for numerical
 * entanglement (Anam & Andreopoulos, "Reliable Linear, Sesquilinear and
 * Bijective Operations on Integer Data Streams via Numerical Entanglement").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; it exists so that the GPU path can be compared against an
 * independent statement of the method.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Conventions
 *  - Every intermediate is computed in __int128 with an explicit overflow
 *    check (checked_* below).  A failed check sets *err = OR_EOVERFLOW and the
 *    function returns that code; nothing aborts the process.
 *  - "x >> s" in the paper (Sec. II footnote: arithmetic shift with truncation
 *    at the least-significant side) is floor(x / 2^s); we write it as an
 *    explicit floor division so the rounding does not depend on the C
 *    compiler's treatment of signed shifts.
 *  - "x << s" is x * 2^s with an overflow check.
 *  - a mod b is the floor modulo a - floor(a/b) * b (Sec. II footnote).
 *  - Outputs that the method defines on w = 64-bit words are stored as the
 *    low 64 bits (two's complement) of the exact value.
 *
 * Parity pins for every function live in tests/test_oracle_*.py; no function
 * here is "parity unpinned".
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

enum { OR_OK = 0, OR_EOVERFLOW = 1, OR_EINVAL = 2, OR_EINFEASIBLE = 3 };

static const i128 I64_MAX_ = (i128)INT64_MAX;
static const i128 I64_MIN_ = (i128)INT64_MIN;

/* ---- checked 128-bit arithmetic ---------------------------------------- */

static void set_err(int *err, int code) {
    /* several OpenMP threads may report; any non-zero code is kept */
    __atomic_store_n(err, code, __ATOMIC_RELAXED);
}

static i128 checked_add(i128 a, i128 b, int *err) {
    i128 r;
    if (__builtin_add_overflow(a, b, &r)) { set_err(err, OR_EOVERFLOW); return 0; }
    return r;
}

static i128 checked_sub(i128 a, i128 b, int *err) {
    i128 r;
    if (__builtin_sub_overflow(a, b, &r)) { set_err(err, OR_EOVERFLOW); return 0; }
    return r;
}

static i128 checked_mul(i128 a, i128 b, int *err) {
    i128 r;
    if (__builtin_mul_overflow(a, b, &r)) { set_err(err, OR_EOVERFLOW); return 0; }
    return r;
}

/* 2^s as a 128-bit integer, 0 <= s <= 125 */
static i128 pow2(int s) { return ((i128)1) << s; }

/* S_s{x} for s >= 0: x * 2^s (Eq. 9, left shift) */
static i128 shift_left(i128 x, int s, int *err) { return checked_mul(x, pow2(s), err); }

/* S_{-s}{x} for s >= 0: floor(x / 2^s) (Eq. 9, arithmetic right shift) */
static i128 shift_right_floor(i128 x, int s) {
    i128 p = pow2(s);
    i128 q = x / p;                 /* C division truncates toward zero */
    if ((x % p) != 0 && x < 0) q -= 1;
    return q;
}

/* floor modulo (Sec. II footnote): a - floor(a/b) b, for b > 0 */
static i128 floor_mod(i128 a, i128 b) {
    i128 m = a % b;
    if (m < 0) m += b;
    return m;
}

/* sign extension of the low b bits: ((x mod 2^b) + 2^(b-1)) mod 2^b - 2^(b-1).
 * This is what Eq. 18 does by shifting a 2w-bit word left by 2w - b and back
 * arithmetically. */
static i128 sext(i128 x, int b) {
    i128 P = pow2(b), H = pow2(b - 1);
    return floor_mod(floor_mod(x, P) + H, P) - H;
}

static int64_t low64(i128 x) { return (int64_t)(uint64_t)(unsigned __int128)x; }

static int fits_i64(i128 x) { return x >= I64_MIN_ && x <= I64_MAX_; }

int or_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads for the following calls (timing only; the results do not depend on it). */
void or_set_threads(int n) {
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- parameter choice (Eq. 13, Eq. 14, Table II) ------------------------- */

/* Eq. 14: the output range supported is |d| <= 2^((M-3)l+k) (2^(l-1) - 1).
 * Returns that bound, or -1 if it does not fit 127 bits. */
i128 or_range_eq14_i128(int M, int l, int k) {
    int e = (M - 3) * l + k;
    if (e < 0 || e + l > 120) return -1;
    return pow2(e) * (pow2(l - 1) - 1);
}

/* int64 view for the Python wrapper; returns -1 when the bound is >= 2^63 */
int64_t or_range_eq14(int M, int l, int k) {
    i128 D = or_range_eq14_i128(M, l, k);
    if (D < 0 || D > I64_MAX_) return -1;
    return (int64_t)D;
}

/*
 * Choose (l, k).
 *  policy 0 ("paper rule", Sec. III-C after Eq. 14, reproduced by Table II):
 *     maximise (M-2)l + k subject to (M-1)l + k <= w and 1 <= k <= l;
 *     ties go to the larger (M-1)l + k.  out_bound is ignored.
 *  policy 1 ("smallest l"): the smallest l >= 1 for which some k with
 *     1 <= k <= l satisfies Eq. 13 and makes the Eq. 14 range cover
 *     out_bound; k is the smallest such k.
 *  policy 2 ("smallest byte-aligned l"): as policy 1 but l must be a multiple
 *     of 8.
 * Returns OR_OK or OR_EINFEASIBLE.
 */
int or_choose_l(int M, int w, int64_t out_bound, int policy, int *l_out, int *k_out) {
    if (M < 3 || w < 4 || w > 64 || !l_out || !k_out) return OR_EINVAL;
    if (policy == 0) {
        int best_l = -1, best_k = -1, best_v = -1, best_t = -1;
        for (int l = 1; l < w; l++) {
            for (int k = 1; k <= l; k++) {
                int t = (M - 1) * l + k;
                if (t > w) continue;
                int v = (M - 2) * l + k;
                if (v > best_v || (v == best_v && t > best_t)) {
                    best_v = v; best_t = t; best_l = l; best_k = k;
                }
            }
        }
        if (best_l < 0) return OR_EINFEASIBLE;
        *l_out = best_l; *k_out = best_k;
        return OR_OK;
    }
    if (policy == 1 || policy == 2) {
        for (int l = 1; l < w; l++) {
            if (policy == 2 && (l % 8) != 0) continue;
            for (int k = 1; k <= l; k++) {
                if ((M - 1) * l + k > w) break;
                i128 D = or_range_eq14_i128(M, l, k);
                if (D >= 0 && D >= (i128)out_bound) {
                    *l_out = l; *k_out = k;
                    return OR_OK;
                }
            }
        }
        return OR_EINFEASIBLE;
    }
    return OR_EINVAL;
}

/* ---- entanglement (Eq. 7 for M = 3, Eq. 15-16 in general) -------------- */

/*
 * eps[m][i] = c[m][i] + S_l{ c[(m-1) mod M][i] }   for 0 <= m < M.
 * Row m of the circulant operator E (Eq. 15) has a 1 on the diagonal and
 * S_l one column to the left (cyclically), so each entangled word is a
 * stream plus its cyclic predecessor shifted by l.  Layout: c and eps are
 * M planes of n values ([M][n], row-major).
 */
int or_entangle(int M, int l, const int32_t *c, int64_t *eps, int64_t n) {
    if (M < 3 || l < 1 || l > 62 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int m = 0; m < M; m++) {
        int prev = (m - 1 + M) % M;
        for (int64_t i = 0; i < n; i++) {
            i128 v = checked_add((i128)c[(int64_t)m * n + i],
                                 shift_left((i128)c[(int64_t)prev * n + i], l, &err), &err);
            if (!fits_i64(v)) err = OR_EOVERFLOW;
            eps[(int64_t)m * n + i] = low64(v);
        }
    }
    return err;
}

/* ---- the LSB operations (Eq. 2, Eq. 10) --------------------------------- */

/*
 * Matrix product D = A G on one stream (the inner-product case of Eq. 2 used
 * by the GEMM experiment of Sec. V): A is [m][k] int64, G is [k][n] int8,
 * D is [m][n] int64.  D[i][j] = sum_t A[i][t] G[t][j], summed in order of t;
 * every partial sum must fit int64 (the method's w = 64 word).
 */
int or_gemm(const int64_t *A, const int8_t *G, int64_t *D, int m, int n, int k) {
    if (m < 0 || n < 0 || k < 0) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int i = 0; i < m; i++) {
        for (int j = 0; j < n; j++) {
            int lerr = OR_OK;
            i128 acc = 0;
            for (int t = 0; t < k; t++) {
                acc = checked_add(acc, checked_mul((i128)A[(int64_t)i * k + t],
                                                   (i128)G[(int64_t)t * n + j], &lerr), &lerr);
                if (!fits_i64(acc)) lerr = OR_EOVERFLOW;
            }
            if (lerr) set_err(&err, lerr);
            D[(int64_t)i * n + j] = low64(acc);
        }
    }
    return err;
}

/*
 * Circular convolution of one length-N signal with a length-N kernel
 * (the "circular convolution" member of Eq. 2):
 *   y[n] = sum_{j=0}^{N-1} x[j] g[(n - j) mod N]
 * Every partial sum must fit int64.
 */
static int cconv_one(const int64_t *x, const int8_t *g, int64_t *y, int64_t N) {
    int err = OR_OK;
    for (int64_t n = 0; n < N; n++) {
        i128 acc = 0;
        for (int64_t j = 0; j < N; j++) {
            int64_t idx = (int64_t)floor_mod((i128)(n - j), (i128)N);
            acc = checked_add(acc, checked_mul((i128)x[j], (i128)g[idx], &err), &err);
            if (!fits_i64(acc)) err = OR_EOVERFLOW;
        }
        y[n] = low64(acc);
    }
    return err;
}

/*
 * Selected outputs of the same circular convolution, one by one: for each of
 * the count requests (signal index bs of the batched [B][S][N] layout,
 * position n), y_at[t] = sum_j x[bs][j] g[bs / S][(n - j) mod N].  For
 * lengths whose full convolution is too long to check output by output.
 */
int or_cconv_at(const int64_t *x, const int8_t *g, int64_t S, int64_t N, const int64_t *bs, const int64_t *pos,
                int64_t count, int64_t *y_at) {
    if (S < 1 || N < 1 || count < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t t = 0; t < count; t++) {
        const int64_t *xs = x + bs[t] * N;
        const int8_t *gb = g + (bs[t] / S) * N;
        i128 acc = 0;
        for (int64_t j = 0; j < N; j++) {
            int64_t idx = (int64_t)floor_mod((i128)(pos[t] - j), (i128)N);
            acc = checked_add(acc, checked_mul((i128)xs[j], (i128)gb[idx], &err), &err);
            if (!fits_i64(acc)) err = OR_EOVERFLOW;
        }
        y_at[t] = low64(acc);
    }
    return err;
}

/*
 * Batched form: x is [B][S][N] (B groups of S signals), g is [B][N] (one
 * kernel per group), y is [B][S][N].  Signal s of group b is convolved with
 * kernel b.
 */
int or_cconv(const int64_t *x, const int8_t *g, int64_t *y, int64_t B, int64_t S, int64_t N) {
    if (B < 0 || S < 0 || N < 1) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t bs = 0; bs < B * S; bs++) {
        int64_t b = bs / S;
        int e = cconv_one(x + bs * N, g + b * N, y + bs * N, N);
        if (e) set_err(&err, e);
    }
    return err;
}

/*
 * Linear (aperiodic) convolution of a long stream with a short kernel in its
 * full form, the convolution of the paper's second experiment (Sec. V):
 *     y[i] = sum_{t=0}^{K-1} g[t] x[i - t],   0 <= i < n + K - 1,
 * with x taken as 0 outside [0, n).  Sec. IV-A processes such streams as
 * overlapping blocks (overlap-save); the blocks reproduce exactly these
 * outputs, so the oracle is the definition itself.
 */
static int lconv_one(const int64_t *x, const int8_t *g, int64_t *y, int64_t n, int64_t K) {
    int err = OR_OK;
    for (int64_t i = 0; i < n + K - 1; i++) {
        const int64_t t0 = i - (n - 1) > 0 ? i - (n - 1) : 0;
        const int64_t t1 = i < K - 1 ? i : K - 1;
        i128 acc = 0;
        for (int64_t t = t0; t <= t1; t++) {
            acc = checked_add(acc, checked_mul((i128)x[i - t], (i128)g[t], &err), &err);
            if (!fits_i64(acc)) err = OR_EOVERFLOW;
        }
        y[i] = low64(acc);
    }
    return err;
}

/* Batched: x [B][S][n] (B groups of S signals), g [B][K] (one kernel per
 * group), y [B][S][n + K - 1]. */
int or_lconv(const int64_t *x, const int8_t *g, int64_t *y, int64_t B, int64_t S, int64_t n, int64_t K) {
    if (B < 0 || S < 0 || n < 1 || K < 1) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t bs = 0; bs < B * S; bs++) {
        int64_t b = bs / S;
        int e = lconv_one(x + bs * n, g + b * K, y + bs * (n + K - 1), n, K);
        if (e) set_err(&err, e);
    }
    return err;
}

/* Selected outputs y[bs[t]][pos[t]] of or_lconv, one by one (bs = b * S + s). */
int or_lconv_at(const int64_t *x, const int8_t *g, int64_t S, int64_t n, int64_t K, const int64_t *bs,
                const int64_t *pos, int64_t count, int64_t *y_at) {
    if (S < 1 || n < 1 || K < 1 || count < 0) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t q = 0; q < count; q++) {
        const int64_t *xs = x + bs[q] * n;
        const int8_t *gb = g + (bs[q] / S) * K;
        const int64_t i = pos[q];
        int e = OR_OK;
        i128 acc = 0;
        if (i < 0 || i >= n + K - 1) e = OR_EINVAL;
        for (int64_t t = 0; e == OR_OK && t < K; t++) {
            if (i - t < 0 || i - t >= n) continue;
            acc = checked_add(acc, checked_mul((i128)xs[i - t], (i128)gb[t], &e), &e);
            if (!fits_i64(acc)) e = OR_EOVERFLOW;
        }
        y_at[q] = low64(acc);
        if (e) set_err(&err, e);
    }
    return err;
}

/*
 * Element-wise LSB operations of Eq. 2 on one stream, y[i] = x[i] op g[i]:
 *   op 0: addition, op 1: subtraction, op 2: multiplication.
 * (For op in {+,-} the entangled pipeline must first entangle g with itself,
 * g <- S_l{g} + g; see or_entangle_kernel_self below.)
 */
int or_elementwise(int op, const int64_t *x, const int64_t *g, int64_t *y, int64_t n) {
    if (op < 0 || op > 2 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        i128 v;
        if (op == 0) v = checked_add((i128)x[i], (i128)g[i], &err);
        else if (op == 1) v = checked_sub((i128)x[i], (i128)g[i], &err);
        else v = checked_mul((i128)x[i], (i128)g[i], &err);
        if (!fits_i64(v)) err = OR_EOVERFLOW;
        y[i] = low64(v);
    }
    return err;
}

/* The footnote to Eq. 10: for op in {+,-} the kernel is replaced by
 * S_l{g} + g so that the entangled sum stays a codeword. */
int or_entangle_kernel_self(int l, const int64_t *g, int64_t *ge, int64_t n) {
    int err = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        i128 v = checked_add(shift_left((i128)g[i], l, &err), (i128)g[i], &err);
        if (!fits_i64(v)) err = OR_EOVERFLOW;
        ge[i] = low64(v);
    }
    return err;
}

/*
 * The remaining LSB operators of Eq. 2, batched like or_cconv: B groups of S
 * signals of length n, one kernel g per group.
 *
 * Inner product, op = <.,.>:  y[b][s] = sum_i x[b][s][i] g[b][i]
 *   (x [B][S][n], g [B][n], y [B][S]); every partial sum must fit int64.
 */
int or_inner(const int64_t *x, const int64_t *g, int64_t *y, int64_t B, int64_t S, int64_t n) {
    if (B < 0 || S < 0 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t b = 0; b < B; b++) {
        for (int64_t s = 0; s < S; s++) {
            i128 acc = 0;
            for (int64_t i = 0; i < n; i++) {
                acc = checked_add(acc, checked_mul((i128)x[(b * S + s) * n + i], (i128)g[b * n + i], &err), &err);
                if (!fits_i64(acc)) err = OR_EOVERFLOW;
            }
            y[b * S + s] = low64(acc);
        }
    }
    return err;
}

/*
 * Outer product, op = (x):  y[b][s][i][j] = x[b][s][i] g[b][j]
 *   (x [B][S][n], g [B][k], y [B][S][n][k]).
 */
int or_outer(const int64_t *x, const int64_t *g, int64_t *y, int64_t B, int64_t S, int64_t n, int64_t k) {
    if (B < 0 || S < 0 || n < 0 || k < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t b = 0; b < B; b++)
        for (int64_t s = 0; s < S; s++)
            for (int64_t i = 0; i < n; i++)
                for (int64_t j = 0; j < k; j++) {
                    i128 v = checked_mul((i128)x[(b * S + s) * n + i], (i128)g[b * k + j], &err);
                    if (!fits_i64(v)) err = OR_EOVERFLOW;
                    y[((b * S + s) * n + i) * k + j] = low64(v);
                }
    return err;
}

/*
 * Permutation, op = (I over G), a bijection from the sequential index set to
 * the index set given by g: output position i holds the input element at
 * index g[i], y[b][s][i] = x[b][s][g[i]].  One index set serves every signal
 * (the method covers data-independent permutations only).  g must be a
 * permutation of 0..n-1; anything else is OR_EINVAL.
 */
int or_permute(const int64_t *x, const int64_t *g, int64_t *y, int64_t B, int64_t S, int64_t n) {
    if (B < 0 || S < 0 || n < 0) return OR_EINVAL;
    for (int64_t i = 0; i < n; i++)
        if (g[i] < 0 || g[i] >= n) return OR_EINVAL;
    for (int64_t i = 0; i < n; i++)           /* bijective: no index repeats */
        for (int64_t j = i + 1; j < n; j++)
            if (g[i] == g[j]) return OR_EINVAL;
    for (int64_t bs = 0; bs < B * S; bs++)
        for (int64_t i = 0; i < n; i++) y[bs * n + i] = x[bs * n + g[i]];
    return OR_OK;
}

/*
 * Circular cross-correlation, the correlation form of the star operator of
 * Eq. 2:  y[b][s][i] = sum_{j=0}^{N-1} x[b][s][(i + j) mod N] g[b][j].
 */
int or_cxcorr(const int64_t *x, const int8_t *g, int64_t *y, int64_t B, int64_t S, int64_t N) {
    if (B < 0 || S < 0 || N < 1) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t bs = 0; bs < B * S; bs++) {
        int lerr = OR_OK;
        const int64_t *xs = x + bs * N;
        const int8_t *gb = g + (bs / S) * N;
        for (int64_t i = 0; i < N; i++) {
            i128 acc = 0;
            for (int64_t j = 0; j < N; j++) {
                int64_t idx = (int64_t)floor_mod((i128)(i + j), (i128)N);
                acc = checked_add(acc, checked_mul((i128)xs[idx], (i128)gb[j], &lerr), &lerr);
                if (!fits_i64(acc)) lerr = OR_EOVERFLOW;
            }
            y[bs * N + i] = low64(acc);
        }
        if (lerr) set_err(&err, lerr);
    }
    return err;
}

/* ---- disentanglement, check and recovery (Eq. 17-20, Eq. 24) ------------ */

/*
 * For one position, from the M entangled outputs delta[0..M-1] (delta[r] is
 * never read), compute all M outputs and the reliability check.
 *
 *  Eq. 17: dtemp = sum_{m=0}^{M-2} (-1)^m S_{(M-2-m)l}{ delta_{(r+1+m) mod M} },
 *          multiplied by (-1)^M.  (Read literally, Eq. 17 yields the negated
 *          outputs for odd M; the factor (-1)^M makes it coincide with the
 *          M = 3 form of Eq. 11, dtemp = delta_2 - S_l{delta_1} at r = 0.)
 *  Eq. 18: d_{(r-1) mod M} = sign extension of the low (M-1)l bits of dtemp.
 *  Eq. 19: d_r = S_{-(M-1)l}{ (-1)^M (dtemp - d_{(r-1) mod M}) }
 *          (the printed index "M-1" is the r = 0 case of (r-1) mod M).
 *  Eq. 20: d_{(r+m) mod M} = delta_{(r+m) mod M} - S_l{ d_{(r+m-1) mod M} }
 *          for 1 <= m <= M-2 (the printed "m < M-2" would leave stream
 *          r+M-2 unrecovered; Eq. 11 at M = 3 computes it this way).
 *  Eq. 24: flag = delta_r - [ d_r + S_l{ d_{(r-1) mod M} } ] != 0,
 *          evaluated on the exact (untruncated) values.
 * The outputs d are written as their low 64 bits.
 */
static int extract_one(int M, int l, const int64_t *delta, int r, int64_t *d_out, int *flag) {
    int err = OR_OK;
    i128 d[64];
    i128 dtemp = 0;
    for (int m = 0; m <= M - 2; m++) {
        i128 term = shift_left((i128)delta[(r + 1 + m) % M], (M - 2 - m) * l, &err);
        if (m % 2 == 0) dtemp = checked_add(dtemp, term, &err);
        else dtemp = checked_sub(dtemp, term, &err);
    }
    if (M % 2 != 0) dtemp = checked_sub(0, dtemp, &err);

    int L = (M - 1) * l;
    int rm1 = (r - 1 + M) % M;
    d[rm1] = sext(dtemp, L);
    i128 diff = checked_sub(dtemp, d[rm1], &err);
    if (M % 2 != 0) diff = checked_sub(0, diff, &err);
    d[r] = shift_right_floor(diff, L);
    for (int m = 1; m <= M - 2; m++) {
        int cur = (r + m) % M, prv = (r + m - 1) % M;
        d[cur] = checked_sub((i128)delta[cur], shift_left(d[prv], l, &err), &err);
    }
    i128 recreated = checked_add(d[r], shift_left(d[rm1], l, &err), &err);
    *flag = (checked_sub((i128)delta[r], recreated, &err) != 0);
    for (int m = 0; m < M; m++) d_out[m] = low64(d[m]);
    return err;
}

/*
 * delta, dhat: [M][n] planes.  flags: n bytes (1 = check failed) or NULL.
 * r: the stream not used for extraction (the one checked, or the lost one).
 */
int or_extract(int M, int l, const int64_t *delta, int64_t n, int r, int64_t *dhat, uint8_t *flags) {
    if (M < 3 || M > 64 || l < 1 || (M - 1) * l > 63 || r < 0 || r >= M || n < 0) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; i++) {
        int64_t dl[64], dout[64];
        for (int m = 0; m < M; m++) dl[m] = (m == r) ? 0 : delta[(int64_t)m * n + i];
        if (flags) dl[r] = delta[(int64_t)r * n + i];
        int f = 0;
        int e = extract_one(M, l, dl, r, dout, &f);
        if (e) set_err(&err, e);
        for (int m = 0; m < M; m++) dhat[(int64_t)m * n + i] = dout[m];
        if (flags) flags[i] = (uint8_t)f;
    }
    return err;
}

/* ---- checksum ABFT comparator (Eq. 3-6) --------------------------------- */

/* Eq. 4: r_i = sum_m c[m][i]; c is [M][n] int32, rsum is [n] int64 */
int or_abft_encode(int M, const int32_t *c, int64_t n, int64_t *rsum) {
    if (M < 1 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        i128 s = 0;
        for (int m = 0; m < M; m++) s = checked_add(s, (i128)c[(int64_t)m * n + i], &err);
        rsum[i] = low64(s);
    }
    return err;
}

/* Eq. 6: flag_i = (sum_{m<M} d[m][i] != e_i); d is [M+1][n], plane M is e */
int or_abft_check(int M, const int64_t *d, int64_t n, uint8_t *flags) {
    if (M < 1 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        i128 s = 0;
        for (int m = 0; m < M; m++) s = checked_add(s, (i128)d[(int64_t)m * n + i], &err);
        flags[i] = (uint8_t)(s != (i128)d[(int64_t)M * n + i]);
    }
    return err;
}

/* Sec. II-A: a lost stream j is rebuilt as e - sum_{m != j} d_m, in place */
int or_abft_recover(int M, int64_t *d, int64_t n, int j) {
    if (M < 1 || n < 0 || j < 0 || j >= M) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t i = 0; i < n; i++) {
        i128 v = (i128)d[(int64_t)M * n + i];
        for (int m = 0; m < M; m++)
            if (m != j) v = checked_sub(v, (i128)d[(int64_t)m * n + i], &err);
        if (!fits_i64(v)) err = OR_EOVERFLOW;
        d[(int64_t)j * n + i] = low64(v);
    }
    return err;
}

/* ---- row/column checksum ABFT of a product (the "ABFT RC-check" comparator
 *      of Sec. V, after Huang and Abraham) -------------------------------- */

/*
 * Encoding: the column-checksum matrix of A (m x k) is A with the row e^T A
 * appended, ac [m+1][k]; the row-checksum matrix of B (k x n) is B with the
 * column B e appended, br [k][n+1].  Their product is the full-checksum
 * matrix of C = A B: C bordered by the row e^T C and the column C e.
 */
int or_rc_encode(const int64_t *A, const int8_t *B, int64_t m, int64_t k, int64_t n, int64_t *ac, int64_t *br) {
    if (m < 0 || k < 0 || n < 0) return OR_EINVAL;
    int err = OR_OK;
    for (int64_t t = 0; t < k; t++) {
        i128 s = 0;
        for (int64_t i = 0; i < m; i++) {
            ac[i * k + t] = A[i * k + t];
            s = checked_add(s, (i128)A[i * k + t], &err);
        }
        if (!fits_i64(s)) err = OR_EOVERFLOW;
        ac[m * k + t] = low64(s);
    }
    for (int64_t t = 0; t < k; t++) {
        i128 s = 0;
        for (int64_t j = 0; j < n; j++) {
            br[t * (n + 1) + j] = B[t * n + j];
            s += (i128)B[t * n + j];
        }
        br[t * (n + 1) + n] = low64(s);
    }
    return err;
}

/* The product of two int64 matrices, Z = X Y (X [m][k], Y [k][n]); every
 * partial sum must fit int64. */
int or_gemm64(const int64_t *X, const int64_t *Y, int64_t *Z, int64_t m, int64_t k, int64_t n) {
    if (m < 0 || k < 0 || n < 0) return OR_EINVAL;
    int err = OR_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < m; i++) {
        int lerr = OR_OK;
        for (int64_t j = 0; j < n; j++) {
            i128 acc = 0;
            for (int64_t t = 0; t < k; t++) {
                acc = checked_add(acc, checked_mul((i128)X[i * k + t], (i128)Y[t * n + j], &lerr), &lerr);
                if (!fits_i64(acc)) lerr = OR_EOVERFLOW;
            }
            Z[i * n + j] = low64(acc);
        }
        if (lerr) set_err(&err, lerr);
    }
    return err;
}

/*
 * The check of a full-checksum matrix Cf [m+1][n+1]: row i (i <= m) is
 * inconsistent when the sum of its first n entries differs from Cf[i][n];
 * column j (j <= n) when the sum of its first m entries differs from Cf[m][j].
 * rowbad [m+1], colbad [n+1].
 */
int or_rc_check(const int64_t *Cf, int64_t m, int64_t n, uint8_t *rowbad, uint8_t *colbad) {
    if (m < 0 || n < 0) return OR_EINVAL;
    const int64_t w = n + 1;
    for (int64_t i = 0; i <= m; i++) {
        i128 s = 0;
        for (int64_t j = 0; j < n; j++) s += (i128)Cf[i * w + j];
        rowbad[i] = (uint8_t)(s != (i128)Cf[i * w + n]);
    }
    for (int64_t j = 0; j <= n; j++) {
        i128 s = 0;
        for (int64_t i = 0; i < m; i++) s += (i128)Cf[i * w + j];
        colbad[j] = (uint8_t)(s != (i128)Cf[m * w + j]);
    }
    return OR_OK;
}

/*
 * Single-error correction: when exactly one row i and one column j are
 * inconsistent, the entry Cf[i][j] is the faulty one.  For j < n it is
 * replaced by Cf[i][n] minus the other entries of row i; for j = n (a row
 * checksum, or the corner when i = m) by the sum of the first n entries of
 * row i.  *corrected = 1 when an entry was replaced.
 */
int or_rc_correct(int64_t *Cf, int64_t m, int64_t n, int *corrected) {
    if (m < 0 || n < 0) return OR_EINVAL;
    const int64_t w = n + 1;
    int64_t bi = -1, bj = -1, nbi = 0, nbj = 0;
    for (int64_t i = 0; i <= m; i++) {
        i128 s = 0;
        for (int64_t j = 0; j < n; j++) s += (i128)Cf[i * w + j];
        if (s != (i128)Cf[i * w + n]) { bi = i; nbi++; }
    }
    for (int64_t j = 0; j <= n; j++) {
        i128 s = 0;
        for (int64_t i = 0; i < m; i++) s += (i128)Cf[i * w + j];
        if (s != (i128)Cf[m * w + j]) { bj = j; nbj++; }
    }
    *corrected = 0;
    if (nbi != 1 || nbj != 1) return OR_OK;
    int err = OR_OK;
    i128 v;
    if (bj < n) {
        v = (i128)Cf[bi * w + n];
        for (int64_t j = 0; j < n; j++)
            if (j != bj) v = checked_sub(v, (i128)Cf[bi * w + j], &err);
    } else {
        v = 0;
        for (int64_t j = 0; j < n; j++) v = checked_add(v, (i128)Cf[bi * w + j], &err);
    }
    if (!fits_i64(v)) err = OR_EOVERFLOW;
    Cf[bi * w + bj] = low64(v);
    *corrected = 1;
    return err;
}
