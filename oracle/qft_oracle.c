/*
 * qft_oracle.c -- plain, slow CPU reference for the QFT->FFT method
 * (Markidis et al., "Not Your Usual FFT: QFT->FFT via Classical Quantum-Circuit
 * Simulation").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The GPU library never
 * links, includes or calls it, and it shares no code, header or table with the
 * GPU path.
 *
 * Everything is complex double (FP64), stored interleaved (re, im), index
 * i = sum_j b_j 2^j with qubit q_j = bit j of the index (Sec. 2, "From Linear
 * Algebra to Quantum Circuit Operators": a 1-wire gate on q_j is
 * I_{2^{n-1-j}} (x) U (x) I_{2^j}; Fig. 1 caption: LSB q_0).
 *
 * Sign convention: sign = -1 is the paper's forward transform
 * (omega_N = e^{-2 pi i / N}, Sec. 2; R_k = diag(1, e^{-2 pi i / 2^k})),
 * sign = +1 the inverse.
 *
 * Functions:
 *   oracle_encode        Sec. 3 step 1 (scale_in = ||x||_2, psi = x / scale_in)
 *   oracle_circuit       Sec. 3 steps 2-3, Fig. 1, Sec. 2 "Approximate QFT":
 *                        gate by gate, H then the kept controlled phases,
 *                        then the qubit-reversal swaps
 *   oracle_decode        Sec. 3 step 4 (rescaling to FFT units)
 *   oracle_dft           Sec. 2: the plain DFT definition, O(N^2)
 *   oracle_aqft_direct   the AQFT matrix element written out in closed form
 *                        (a sum of per-gate phases, derived from Fig. 1 /
 *                        Eq. 5), O(N^2); also used for a few output bins at
 *                        large n (O(N) per bin)
 *   oracle_gate_counts   gate counts of the (A)QFT circuit (Table 2)
 *   oracle_gate_list     the gate sequence itself (Fig. 1)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_TWO_PI 6.283185307179586476925286766559

/* Number of threads OpenMP will use for the gate loops (1 without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* Effective cutoff: the range-k AQFT keeps controlled rotations whose
 * control-target distance d satisfies d <= k; k >= n-1 (or k < 0) is the
 * exact QFT (Sec. 2, "Approximate QFT"). */
static int effective_k(int n, int k)
{
    if (k < 0 || k > n - 1) return n - 1 > 0 ? n - 1 : 0;
    return k;
}

/* ---------------------------------------------------------------- encode */

/* Sec. 3 step 1: scale_in = ||x||_2 (FP64), psi = x / scale_in.
 * A zero vector has no normalised form; it is encoded as zeros with
 * scale_in = 0.  Returns scale_in. */
double oracle_encode(int n, const double *x, double *psi)
{
    const int64_t N = (int64_t)1 << n;
    double s = 0.0;
    for (int64_t i = 0; i < N; i++) s += x[2 * i] * x[2 * i] + x[2 * i + 1] * x[2 * i + 1];
    const double scale_in = sqrt(s);
    for (int64_t i = 0; i < 2 * N; i++) psi[i] = scale_in > 0.0 ? x[i] / scale_in : 0.0;
    return scale_in;
}

/* ------------------------------------------------------------------ gates */

/* Hadamard on q_t, normalised as (1/sqrt 2)[[1,1],[1,-1]] so that the whole
 * circuit is the unitary U = DFT_N / sqrt(N) (Eq. 1 with Sec. 3 step 3).
 * Updates the 2^{n-1} pairs (i, i + 2^t) with bit t of i clear (Sec. 2). */
static void apply_h(double *psi, int n, int t)
{
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t low = ((int64_t)1 << t) - 1;
    const double r = 1.0 / sqrt(2.0);
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < half; p++) {
        /* p enumerates the pairs: insert a zero at bit t */
        const int64_t i0 = ((p & ~low) << 1) | (p & low);
        const int64_t i1 = i0 | ((int64_t)1 << t);
        const double ar = psi[2 * i0], ai = psi[2 * i0 + 1];
        const double br = psi[2 * i1], bi = psi[2 * i1 + 1];
        psi[2 * i0] = (ar + br) * r;
        psi[2 * i0 + 1] = (ai + bi) * r;
        psi[2 * i1] = (ar - br) * r;
        psi[2 * i1 + 1] = (ai - bi) * r;
    }
}

/* Controlled-R_m between control q_c and target q_t: R_m = diag(1, e^{s 2 pi i / 2^m}),
 * controlled-R_m = E1 (x) I + E2 (x) R_m (Sec. 2).  It multiplies by
 * e^{s 2 pi i / 2^m} every amplitude whose bits c and t are both 1 and leaves
 * the others unchanged: a diagonal update on a quarter of the entries. */
static void apply_cp(double *psi, int n, int c, int t, int m, int sign)
{
    const int64_t N = (int64_t)1 << n;
    const int64_t mask = ((int64_t)1 << c) | ((int64_t)1 << t);
    const double theta = sign * ORACLE_TWO_PI / ldexp(1.0, m);
    const double cr = cos(theta), ci = sin(theta);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; i++) {
        if ((i & mask) != mask) continue;
        const double ar = psi[2 * i], ai = psi[2 * i + 1];
        psi[2 * i] = ar * cr - ai * ci;
        psi[2 * i + 1] = ar * ci + ai * cr;
    }
}

static int64_t bit_reverse(int64_t i, int n)
{
    int64_t r = 0;
    for (int b = 0; b < n; b++)
        if (i & ((int64_t)1 << b)) r |= (int64_t)1 << (n - 1 - b);
    return r;
}

/* SWAP(q_j, q_{n-1-j}) for j < floor(n/2): together the output bit reversal
 * psi'[i] = psi[bitrev_n(i)] (Fig. 1 caption; Sec. 3 step 2). */
static void apply_swaps(double *psi, int n)
{
    const int64_t N = (int64_t)1 << n;
    for (int j = 0; j < n / 2; j++) {
        const int64_t bj = (int64_t)1 << j, bk = (int64_t)1 << (n - 1 - j);
        /* each exchanged pair is visited once, from its bit-j-set member */
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; i++) {
            /* exchange the amplitudes of |..1..0..> and |..0..1..> once */
            if ((i & bj) && !(i & bk)) {
                const int64_t o = (i & ~bj) | bk;
                double tr = psi[2 * i], ti = psi[2 * i + 1];
                psi[2 * i] = psi[2 * o];
                psi[2 * i + 1] = psi[2 * o + 1];
                psi[2 * o] = tr;
                psi[2 * o + 1] = ti;
            }
        }
    }
}

/* Sec. 3 steps 2-3 and Fig. 1: the n-qubit (A)QFT circuit applied gate by
 * gate to psi (in place).  For t = n-1 down to 0: H on q_t, then the
 * controlled-R_{d+1} with control q_{t-d} and target q_t for d = 1..min(k, t)
 * (range-k AQFT: distance d <= k kept, Sec. 2).  natural_order != 0 applies the
 * final swaps; natural_order == 0 leaves them to the caller (the paper's
 * deferred output permutation, Sec. 3 step 2). */
void oracle_circuit(int n, int k, int sign, int natural_order, double *psi)
{
    const int kk = effective_k(n, k);
    for (int t = n - 1; t >= 0; t--) {
        apply_h(psi, n, t);
        for (int d = 1; d <= kk && d <= t; d++) apply_cp(psi, n, t - d, t, d + 1, sign);
    }
    if (natural_order) apply_swaps(psi, n);
}

/* Single gates, exposed so that a benchmark can time a bounded sample of a
 * large circuit (one sweep per gate) without running all of it.
 * kind 0: H on q_a; 1: controlled-R_m, control q_a, target q_b; 2: the swaps. */
void oracle_apply_gate(int n, int kind, int a, int b, int m, int sign, double *psi)
{
    if (kind == 0) apply_h(psi, n, a);
    else if (kind == 1) apply_cp(psi, n, a, b, m, sign);
    else apply_swaps(psi, n);
}

/* ----------------------------------------------------------------- decode */

/* Sec. 3 step 4.  psi' = DFT_N x / (scale_in sqrt N).  mode 0: the state psi'
 * itself; 1: unitary FFT = scale_in psi'; 2: unnormalised FFT
 * = scale_in sqrt(N) psi'; 3: the 1/N-scaled FFT = scale_in psi' / sqrt(N). */
void oracle_decode(int n, const double *psi, double scale_in, int mode, double *out)
{
    const int64_t N = (int64_t)1 << n;
    const double rootN = sqrt(ldexp(1.0, n));
    double f = 1.0;
    if (mode == 1) f = scale_in;
    else if (mode == 2) f = scale_in * rootN;
    else if (mode == 3) f = scale_in / rootN;
    for (int64_t i = 0; i < 2 * N; i++) out[i] = psi[i] * f;
}

/* ------------------------------------------------------- plain definitions */

/* Sec. 2: DFT_N = [omega^{k l}], omega = e^{s 2 pi i / N} (s = -1 forward).
 * X[y] = sum_x x[x] e^{s 2 pi i (x y mod N) / N}; the exponent is reduced
 * exactly in integers before the angle is formed.  Unnormalised, O(N^2). */
void oracle_dft(int n, int sign, const double *x, double *X)
{
    const int64_t N = (int64_t)1 << n;
    const uint64_t mask = (uint64_t)N - 1;
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < N; y++) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < N; j++) {
            const uint64_t p = ((uint64_t)j * (uint64_t)y) & mask;
            const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);
            const double c = cos(th), s = sin(th);
            sr += x[2 * j] * c - x[2 * j + 1] * s;
            si += x[2 * j] * s + x[2 * j + 1] * c;
        }
        X[2 * y] = sr;
        X[2 * y + 1] = si;
    }
}

/* Integer phase (in units of 2^-n turns, reduced mod 2^n) that the range-k
 * circuit with swaps assigns to the matrix element <y|U_k|x>.  Wire t
 * (after its H and kept controlled phases) carries the factor
 * exp(s 2 pi i y_{n-1-t} sum_{d=0}^{min(k,t)} x_{t-d} 2^{-(d+1)}), and the swaps
 * put wire t at output bit n-1-t; with i = t-d and j = n-1-t this is the sum of
 * x_i y_j 2^{i+j-n} over n-1-k <= i+j <= n-1.  k >= n-1 gives x*y mod 2^n. */
static uint64_t aqft_phase(int n, int kk, uint64_t x, uint64_t y)
{
    const uint64_t mask = (n == 64) ? ~(uint64_t)0 : (((uint64_t)1 << n) - 1);
    uint64_t p = 0;
    for (int i = 0; i < n; i++) {
        if (!((x >> i) & 1)) continue;
        /* output bits j with n-1-kk-i <= j <= n-1-i */
        const int jhi = n - 1 - i;
        int jlo = n - 1 - kk - i;
        if (jlo < 0) jlo = 0;
        const uint64_t win = (((uint64_t)1 << (jhi - jlo + 1)) - 1) << jlo;
        p += (y & win) << i;
    }
    return p & mask;
}

/* <y|U_k|x> = N^{-1/2} exp(s 2 pi i phase(x, y) / N) summed over x, i.e. the
 * range-k AQFT with swaps applied to x (no normalisation of x), O(N^2). */
void oracle_aqft_direct(int n, int k, int sign, const double *x, double *out)
{
    const int64_t N = (int64_t)1 << n;
    const int kk = effective_k(n, k);
    const double inv_root = 1.0 / sqrt(ldexp(1.0, n));
#pragma omp parallel for schedule(static)
    for (int64_t y = 0; y < N; y++) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < N; j++) {
            const uint64_t p = aqft_phase(n, kk, (uint64_t)j, (uint64_t)y);
            const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);
            const double c = cos(th), s = sin(th);
            sr += x[2 * j] * c - x[2 * j + 1] * s;
            si += x[2 * j] * s + x[2 * j + 1] * c;
        }
        out[2 * y] = sr * inv_root;
        out[2 * y + 1] = si * inv_root;
    }
}

/* A few output bins of the range-k AQFT with swaps, each by direct O(N)
 * summation (for sizes where the full circuit is too slow to run here).
 * out[b] = <ys[b]| U_k |x>, natural output order, no normalisation of x. */
void oracle_aqft_bins(int n, int k, int sign, const double *x, const int64_t *ys,
                      int nbins, double *out)
{
    const int64_t N = (int64_t)1 << n;
    const int kk = effective_k(n, k);
    const double inv_root = 1.0 / sqrt(ldexp(1.0, n));
    for (int b = 0; b < nbins; b++) {
        const uint64_t y = (uint64_t)ys[b];
        double sr = 0.0, si = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sr, si)
        for (int64_t j = 0; j < N; j++) {
            const uint64_t p = aqft_phase(n, kk, (uint64_t)j, y);
            const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);
            const double c = cos(th), s = sin(th);
            sr += x[2 * j] * c - x[2 * j + 1] * s;
            si += x[2 * j] * s + x[2 * j + 1] * c;
        }
        out[2 * b] = sr * inv_root;
        out[2 * b + 1] = si * inv_root;
    }
}

/* ---------------------------------------------------------- circuit shape */

/* Gate counts of the range-k circuit (Table 2; Sec. 2 "Approximate QFT"):
 * n Hadamards, sum over t of min(k, t) controlled phases, floor(n/2) swaps. */
void oracle_gate_counts(int n, int k, int64_t *n_h, int64_t *n_cp, int64_t *n_swap)
{
    const int kk = effective_k(n, k);
    int64_t cp = 0;
    for (int t = n - 1; t >= 0; t--)
        for (int d = 1; d <= kk && d <= t; d++) cp++;
    *n_h = n;
    *n_cp = cp;
    *n_swap = n / 2;
}

/* The gate sequence of Fig. 1 generalised to n wires.  Each gate is four
 * ints: (kind, a, b, m) with kind 0 = H on q_a, 1 = controlled-R_m with
 * control q_a and target q_b, 2 = SWAP(q_a, q_b).  Returns the number of gates
 * written (at most cap). */
int oracle_gate_list(int n, int k, int natural_order, int *gates, int cap)
{
    const int kk = effective_k(n, k);
    int g = 0;
    for (int t = n - 1; t >= 0; t--) {
        if (g < cap) { gates[4 * g] = 0; gates[4 * g + 1] = t; gates[4 * g + 2] = t; gates[4 * g + 3] = 0; }
        g++;
        for (int d = 1; d <= kk && d <= t; d++) {
            if (g < cap) { gates[4 * g] = 1; gates[4 * g + 1] = t - d; gates[4 * g + 2] = t; gates[4 * g + 3] = d + 1; }
            g++;
        }
    }
    if (natural_order)
        for (int j = 0; j < n / 2; j++) {
            if (g < cap) { gates[4 * g] = 2; gates[4 * g + 1] = j; gates[4 * g + 2] = n - 1 - j; gates[4 * g + 3] = 0; }
            g++;
        }
    return g;
}

/* Bit reversal of an n-bit index (exposed for the tests' index-map checks). */
int64_t oracle_bit_reverse(int64_t i, int n) { return bit_reverse(i, n); }

/* ------------------------------------ Monte Carlo sum over histories (Sec. 6)
 *
 * Sec. 6 proposes a Monte Carlo backend "in the sum-over-histories style": the
 * amplitude <y|U_k|x> is a sum over input indices j of x_j times the phase the
 * kept controlled rotations give the path j -> y, and sampling input indices
 * with importance weights gives unbiased estimates of single output bins and
 * of the power spectrum.  Readings (the passage gives no formulas):
 *   - the proposal follows the magnitude of term j: p_j proportional to
 *     m_j = max(|Re x_j|, |Im x_j|) (within a factor sqrt(2) of |x_j|, and
 *     formed without rounding), made exact in integers from the binary
 *     representation of m_j: with its significand s_j (53 bits, the implicit
 *     bit included for normal numbers) and biased exponent e_j (at least 1),
 *     e_max the largest e_j and S = min(62 - n, 52),
 *         q_j = (s_j >> (e_max - e_j + 53 - S)) + 1  (0 if x_j = 0),
 *     i.e. floor(m_j 2^S / 2^(E+1)) + 1 with 2^E <= max m < 2^(E+1): an
 *     integer within one of m_j's share of 2^S, at least 1 whenever x_j != 0
 *     (so no nonzero term is left out and the estimator stays unbiased);
 *     T = sum_j q_j <= 2^n (2^S + 1), p_j = q_j / T;
 *   - a uniform u in [0, 1), a multiple of 2^-53, selects the target
 *     t = floor(u 2^53 T / 2^53) in [0, T) and the index j with
 *     C_{j-1} <= t < C_j, C the inclusive prefix sums of q;
 *   - the sample's weight is w = x_j T / q_j (= x_j / p_j), so that
 *     z = w exp(s 2 pi i phase(j, y) / N) / sqrt(N) has mean <y|U_k|x>;
 *   - per bin: the mean of z over the M samples, the unbiased estimate
 *     (|sum z|^2 - sum |z|^2) / (M (M - 1)) of |<y|U_k|x>|^2, and the
 *     standard error sqrt((sum |z|^2 / M - |mean|^2) / (M - 1)) of the mean. */

/* The bits of m_j = max(|Re x_j|, |Im x_j|) (sign cleared). */
static uint64_t mc_mag_bits(const double *x, int64_t j)
{
    uint64_t a, b;
    memcpy(&a, &x[2 * j], 8);
    memcpy(&b, &x[2 * j + 1], 8);
    a &= 0x7FFFFFFFFFFFFFFFull;
    b &= 0x7FFFFFFFFFFFFFFFull;
    return a > b ? a : b;
}

/* q_j of the proposal from the bits of m_j (see above). */
static uint64_t mc_weight(uint64_t bits, int emax, int S)
{
    if (bits == 0) return 0;
    const int eb = (int)(bits >> 52);
    const int e = eb > 0 ? eb : 1;
    const uint64_t sig = (bits & 0xFFFFFFFFFFFFFull) | (eb > 0 ? (uint64_t)1 << 52 : 0);
    const int sh = emax - e + 53 - S;
    return (sh < 64 ? sig >> sh : 0) + 1;
}

/* Importance sampling of M entries of a list of K amplitudes x (entry j at
 * list position j): idx[m] = the drawn position and the complex weight w[2m],
 * w[2m+1] for the uniform u[m]; S = min(62 - lg, 52) with K <= 2^lg.  Returns
 * T (0 for an all-zero list: then every position is 0 and every weight 0). */
static uint64_t mc_sample_list(int64_t N, int lg, const double *x, const double *u, int64_t m, int64_t *idx,
                               double *w)
{
    uint64_t mb = 0;
    for (int64_t j = 0; j < N; j++) {
        const uint64_t b = mc_mag_bits(x, j);
        if (b > mb) mb = b;
    }
    if (mb == 0) {
        for (int64_t i = 0; i < m; i++) { idx[i] = 0; w[2 * i] = 0.0; w[2 * i + 1] = 0.0; }
        return 0;
    }
    const int emax = (int)(mb >> 52) > 0 ? (int)(mb >> 52) : 1;
    const int S = 62 - lg < 52 ? 62 - lg : 52;
    uint64_t *C = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)N);
    if (!C) return 0;
    uint64_t acc = 0;
    for (int64_t j = 0; j < N; j++) {
        acc += mc_weight(mc_mag_bits(x, j), emax, S);
        C[j] = acc;
    }
    const uint64_t T = acc;
    for (int64_t i = 0; i < m; i++) {
        const uint64_t u53 = (uint64_t)(u[i] * 9007199254740992.0); /* u * 2^53, exact */
        const uint64_t t = (uint64_t)(((unsigned __int128)u53 * T) >> 53);
        int64_t lo = 0, hi = N - 1; /* smallest j with C[j] > t */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (C[mid] > t) hi = mid; else lo = mid + 1;
        }
        const uint64_t q = C[lo] - (lo ? C[lo - 1] : 0);
        const double f = (double)T / (double)q;
        idx[i] = lo;
        w[2 * i] = x[2 * lo] * f;
        w[2 * i + 1] = x[2 * lo + 1] * f;
    }
    free(C);
    return T;
}

/* The dense input x of 2^n amplitudes: positions are the input indices. */
uint64_t oracle_mc_sample(int n, const double *x, const double *u, int64_t m, int64_t *idx, double *w)
{
    return mc_sample_list((int64_t)1 << n, n, x, u, m, idx, w);
}

/* A sparse input of K >= 1 nonzeros: amplitude vals[j] at input index pos[j]
 * of an n-wire register (n <= 62, far beyond a state vector): the proposal
 * runs over the list (S from lg = ceil(log2 K)), and idx[m] receives the
 * drawn entry's input index pos[j]. */
uint64_t oracle_mc_sample_sparse(int64_t K, const int64_t *pos, const double *vals, const double *u, int64_t m,
                                 int64_t *idx, double *w)
{
    int lg = 0;
    while (((int64_t)1 << lg) < K) lg++;
    const uint64_t T = mc_sample_list(K, lg, vals, u, m, idx, w);
    for (int64_t i = 0; i < m; i++) idx[i] = pos[idx[i]];
    return T;
}

/* Per output bin ys[b] of the range-k transform with swaps (natural order):
 * out[4b..4b+3] = (Re mean, Im mean, power estimate, standard error) of the
 * M samples (idx, w) drawn by oracle_mc_sample. */
void oracle_mc_bins(int n, int k, int sign, const int64_t *idx, const double *w, int64_t m, const int64_t *ys,
                    int nbins, double *out)
{
    /* n <= 62: phases mod 2^n in 64-bit integers */
    const int kk = effective_k(n, k);
    const double inv_root = 1.0 / sqrt(ldexp(1.0, n));
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < nbins; b++) {
        double sr = 0.0, si = 0.0, sq = 0.0;
        for (int64_t i = 0; i < m; i++) {
            const uint64_t p = aqft_phase(n, kk, (uint64_t)idx[i], (uint64_t)ys[b]);
            const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);
            const double c = cos(th), s = sin(th);
            const double zr = (w[2 * i] * c - w[2 * i + 1] * s) * inv_root;
            const double zi = (w[2 * i] * s + w[2 * i + 1] * c) * inv_root;
            sr += zr;
            si += zi;
            sq += zr * zr + zi * zi;
        }
        const double M = (double)m;
        const double mr = sr / M, mi = si / M;
        out[4 * b] = mr;
        out[4 * b + 1] = mi;
        out[4 * b + 2] = m > 1 ? (sr * sr + si * si - sq) / (M * (M - 1.0)) : 0.0;
        const double v = m > 1 ? (sq / M - (mr * mr + mi * mi)) / (M - 1.0) : 0.0;
        out[4 * b + 3] = v > 0.0 ? sqrt(v) : 0.0;
    }
}

/* A few output bins of the range-k AQFT with swaps of an input with K
 * nonzero amplitudes vals[j] at indices pos[j] of an n-wire register
 * (n <= 62): the closed-form matrix elements summed over the nonzeros only
 * (no normalisation of x).  out[b] = <ys[b]| U_k |x>. */
void oracle_aqft_bins_sparse(int n, int k, int sign, int64_t K, const int64_t *pos, const double *vals,
                             const int64_t *ys, int nbins, double *out)
{
    const int kk = effective_k(n, k);
    const double inv_root = 1.0 / sqrt(ldexp(1.0, n));
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < nbins; b++) {
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < K; j++) {
            const uint64_t p = aqft_phase(n, kk, (uint64_t)pos[j], (uint64_t)ys[b]);
            const double th = sign * ORACLE_TWO_PI * ldexp((double)p, -n);
            const double c = cos(th), s = sin(th);
            sr += vals[2 * j] * c - vals[2 * j + 1] * s;
            si += vals[2 * j] * s + vals[2 * j + 1] * c;
        }
        out[2 * b] = sr * inv_root;
        out[2 * b + 1] = si * inv_root;
    }
}
