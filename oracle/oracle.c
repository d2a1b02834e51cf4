/*
 * FP64 CPU oracle for perfect sampling from a right-canonical complex MPS.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the sampler computes.  It is used by the tests, the
 * smoke check and the benchmark's CPU-baseline leg; the product library never
 * links, loads or calls it, and it shares no code with the CUDA path.
 *
 * Method (Sec. 2.2, Fig. 1; Algorithm 2 "Measurement"; Sec. 3.3.1 per-sample
 * scaling), written out exactly in complex double precision:
 *
 *   v_0 = [1]                                   (left boundary, b_0 = 1)
 *   for k = 0 .. M-1:
 *     y_s[b] = sum_a v_k[a] A_k[a, s, b]         contraction, s < d, b < chi_r
 *     w_s    = sum_b |y_s[b]|^2                   unnormalised probabilities
 *     C_s    = w_0 + ... + w_s   (in s order)     cumulative sum, Z = C_{d-1}
 *     u      = U(seed, n, k, job) in (0,1)        Philox4x32-10 uniform
 *     s*     = #{ s < d-1 : C_s < u Z }           "sum(threshold > cdf)"
 *     logp  += log(w_{s*}) - log(Z)
 *     v_{k+1} = y_{s*} / sqrt(w_{s*})             exact per-sample rescaling
 *
 * Readings of the paper taken here (the paper's Vidal-form line
 * "probs = dot(temp, Lambda)" is read as the squared norm; the garbled slice
 * "temp[range(N2), :, :samples]" as selecting block s*; the random threshold
 * as a (0,1) uniform from a counter-based generator keyed by (seed, n, k)).
 *
 * Site tensors are passed as interleaved complex doubles, A_k[a][s][b]
 * row-major with shape (chi_l = bond[k], d, chi_r = bond[k+1]).
 *
 * Two extensions of the same loop (both optional per call):
 *  - Vidal form (Sec. 2.2: the workflow contracts Gamma_i into the left
 *    environment; Algorithm 2 takes the coefficient vector Lambda): the site
 *    tensors are Gamma_k and lam[k] holds Lambda_k, the Schmidt coefficients
 *    on the bond to the right of site k.  Then temp_s = v Gamma_k[:, s, :],
 *    w_s = sum_b |temp_s[b]|^2 Lambda_k[b]^2, and the carried left vector is
 *    v_{k+1}[b] = temp_{s*}[b] Lambda_k[b] / sqrt(w_{s*}).
 *  - GBS random displacement (Sec. 3.4.1): sample n at site k carries a complex
 *    amplitude mu[n, k]; the physical index of the contracted tensor is mixed
 *    by the displacement matrix D(mu) of Eq. (zass),
 *    temp_s <- sum_t D[s, t] temp_t, before the probabilities are formed.
 *
 * Parity pins for every function are in tests/test_oracle_pins.py: brute
 * force over all d^M configurations, closed forms, special cases (product
 * state, GHZ chain), Philox known-answer vectors and marginal statistics.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as  */
/* easy as 1, 2, 3", SC'11).  Ten rounds of the 4x32 bijection with the      */
/* published multipliers and Weyl key increments.                            */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The uniform of sample n at site k: key = (seed lo, seed hi), counter =
 * (n lo, n hi, k, job); u = (53 bits of (x0, x1) + 1/2) * 2^-53, in (0, 1). */
double orc_uniform(uint64_t seed, uint64_t n, uint32_t k, uint32_t job)
{
    uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), k, job};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint64_t bits = ((uint64_t)x[0] << 21) | (uint64_t)(x[1] >> 11);
    return ((double)bits + 0.5) * 0x1p-53;
}

/* ------------------------------------------------------------------------ */
/* One site of a batch of samples, complex double.                           */
/* ------------------------------------------------------------------------ */

/* For every sample r of a batch (Algorithm 2 contracts the left environments
 * of a whole batch of samples with the site tensor at once):
 * y_r[s*chi_r + b] (interleaved re, im) = sum_a v_r[a] A[a, s, b], the sum
 * taken over a in increasing order.  Plain loops; the output columns are
 * taken ORC_CBLOCK at a time, the real and imaginary parts of a block are
 * accumulated in separate arrays, and within a block the sample loop sits
 * inside the loop over a -- only so that a block's partial sums of the whole
 * batch stay in the L1 cache, each entry of A is read once per batch and the
 * compiler can use plain vector arithmetic.  Every output entry receives the
 * same operations in the same order as in a row-at-a-time, column-at-a-time
 * loop: starting from 0, y += (v_r * a_r - v_i * a_i) for the real part and
 * y += (v_r * a_i + v_i * a_r) for the imaginary part, for a = 0, 1, ...
 * A holds interleaved complex doubles (a_is_f32 = 0) or floats
 * (a_is_f32 = 1); float entries are widened exactly to double. */
#define ORC_BATCH 8 /* samples contracted together per site (Algorithm 2's batch) */
#define ORC_CBLOCK 128 /* output columns per block */

static inline double orc_elem(const void *A, int a_is_f32, size_t i)
{
    return a_is_f32 ? (double)((const float *)A)[i] : ((const double *)A)[i];
}

static void orc_contract(int nrows, double *const *vs, int chi_l, int d, int chi_r, const void *A, int a_is_f32,
                         double *const *ys)
{
    const int cols = d * chi_r;
    double ar[ORC_CBLOCK], ai[ORC_CBLOCK];
    double yre[ORC_BATCH][ORC_CBLOCK], yim[ORC_BATCH][ORC_CBLOCK];
    for (int c0 = 0; c0 < cols; c0 += ORC_CBLOCK) {
        const int nc = cols - c0 < ORC_CBLOCK ? cols - c0 : ORC_CBLOCK;
        for (int r = 0; r < nrows; ++r)
            for (int c = 0; c < nc; ++c) {
                yre[r][c] = 0.0;
                yim[r][c] = 0.0;
            }
        for (int a = 0; a < chi_l; ++a) {
            /* entries c0 .. c0+nc-1 of row a of A as doubles, read once for the batch */
            const size_t row = (size_t)2 * ((size_t)a * cols + c0);
            for (int c = 0; c < nc; ++c) {
                ar[c] = orc_elem(A, a_is_f32, row + 2 * c);
                ai[c] = orc_elem(A, a_is_f32, row + 2 * c + 1);
            }
            for (int r = 0; r < nrows; ++r) {
                const double vr = vs[r][2 * a], vi = vs[r][2 * a + 1];
                double *yr = yre[r], *yi = yim[r];
                for (int c = 0; c < nc; ++c) {
                    yr[c] += vr * ar[c] - vi * ai[c];
                    yi[c] += vr * ai[c] + vi * ar[c];
                }
            }
        }
        for (int r = 0; r < nrows; ++r)
            for (int c = 0; c < nc; ++c) {
                ys[r][2 * (c0 + c)] = yre[r][c];
                ys[r][2 * (c0 + c) + 1] = yim[r][c];
            }
    }
}

/* w_s = sum_b |y_s[b]|^2 */
static void orc_block_norms(const double *y, int d, int chi_r, double *w)
{
    for (int s = 0; s < d; ++s) {
        double acc = 0.0;
        for (int b = 0; b < chi_r; ++b) {
            const double re = y[2 * (s * chi_r + b)], im = y[2 * (s * chi_r + b) + 1];
            acc += re * re + im * im;
        }
        w[s] = acc;
    }
}

/* s* = #{ s < d-1 : C_s < u Z } with C the cumulative sum of w in s order. */
static int orc_draw(const double *w, int d, double u, double *Z_out, double *margin_out)
{
    double C[256];
    double acc = 0.0;
    for (int s = 0; s < d; ++s) {
        acc += w[s];
        C[s] = acc;
    }
    const double Z = C[d - 1];
    const double t = u * Z;
    int cnt = 0;
    double margin = INFINITY;
    for (int s = 0; s < d - 1; ++s) {
        if (C[s] < t) cnt++;
        double dist = fabs(t - C[s]) / Z;
        if (dist < margin) margin = dist;
    }
    if (Z_out) *Z_out = Z;
    if (margin_out) *margin_out = margin;
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* GBS displacement (Sec. 3.4.1, Eq. (zass))                                 */
/* ------------------------------------------------------------------------ */

/* Z = X Y for n x n complex matrices (row-major). */
static void orc_cmatmul(int n, const double complex *X, const double complex *Y, double complex *Z)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double complex acc = 0.0;
            for (int q = 0; q < n; ++q) acc += X[i * n + q] * Y[q * n + j];
            Z[i * n + j] = acc;
        }
}

/* E = exp(X) for a nilpotent X (X^n = 0): the power series ends after n terms,
 * E = sum_{m=0}^{n-1} X^m / m!. */
static void orc_exp_nilpotent(int n, const double complex *X, double complex *E, double complex *term,
                              double complex *tmp)
{
    for (int i = 0; i < n * n; ++i) {
        E[i] = (i / n == i % n) ? 1.0 : 0.0;
        term[i] = E[i];
    }
    for (int m = 1; m < n; ++m) {
        orc_cmatmul(n, term, X, tmp);
        for (int i = 0; i < n * n; ++i) {
            term[i] = tmp[i] / (double)m;
            E[i] += term[i];
        }
    }
}

/*
 * D = exp(-|mu|^2 / 2) exp(mu a^dag) exp(-mu^* a), the paper's Zassenhaus
 * approximation of the displacement operator exp(mu a^dag - mu^* a), in the
 * n-level truncation: a|j> = sqrt(j)|j-1>, so a[j-1][j] = sqrt(j) and
 * a^dag = a^T.  Both exponents are nilpotent there (strictly triangular), so
 * the two exponentials are finite sums: exp(mu a^dag) is lower and
 * exp(-mu^* a) upper triangular.  D is written row-major as n*n interleaved
 * complex doubles (D[2*(s*n+t)], D[2*(s*n+t)+1]).
 */
void orc_displacement(double mu_re, double mu_im, int n, double *D)
{
    const double complex mu = mu_re + I * mu_im;
    const size_t nn = (size_t)n * n;
    double complex *buf = (double complex *)calloc(7 * nn, sizeof(double complex));
    if (!buf) {
        for (size_t i = 0; i < 2 * nn; ++i) D[i] = NAN;
        return;
    }
    double complex *X = buf, *Y = buf + nn, *EX = buf + 2 * nn, *EY = buf + 3 * nn, *term = buf + 4 * nn,
                   *tmp = buf + 5 * nn, *P = buf + 6 * nn;
    for (int j = 1; j < n; ++j) {
        const double r = sqrt((double)j);
        X[j * n + (j - 1)] = mu * r;          /* mu a^dag:  (a^dag)[j][j-1] = sqrt(j) */
        Y[(j - 1) * n + j] = -conj(mu) * r;   /* -mu^* a:   a[j-1][j] = sqrt(j)       */
    }
    orc_exp_nilpotent(n, X, EX, term, tmp);
    orc_exp_nilpotent(n, Y, EY, term, tmp);
    orc_cmatmul(n, EX, EY, P);
    const double g = exp(-0.5 * (mu_re * mu_re + mu_im * mu_im));
    for (size_t i = 0; i < nn; ++i) {
        D[2 * i] = g * creal(P[i]);
        D[2 * i + 1] = g * cimag(P[i]);
    }
    free(buf);
}

/* y_s <- sum_t D[s][t] y_t for every column b (D: d x d interleaved complex). */
static void orc_displace(double *y, int d, int chi_r, const double *D, double *tmp)
{
    for (int s = 0; s < d; ++s)
        for (int b = 0; b < chi_r; ++b) {
            double re = 0.0, im = 0.0;
            for (int t = 0; t < d; ++t) {
                const double dr = D[2 * (s * d + t)], di = D[2 * (s * d + t) + 1];
                const double yr = y[2 * (t * chi_r + b)], yi = y[2 * (t * chi_r + b) + 1];
                re += dr * yr - di * yi;
                im += dr * yi + di * yr;
            }
            tmp[2 * (s * chi_r + b)] = re;
            tmp[2 * (s * chi_r + b) + 1] = im;
        }
    memcpy(y, tmp, sizeof(double) * 2 * (size_t)d * chi_r);
}

/* Vidal form: w_s = sum_b |temp_s[b]|^2 Lambda[b]^2 */
static void orc_block_norms_lambda(const double *y, int d, int chi_r, const double *lam, double *w)
{
    for (int s = 0; s < d; ++s) {
        double acc = 0.0;
        for (int b = 0; b < chi_r; ++b) {
            const double re = y[2 * (s * chi_r + b)], im = y[2 * (s * chi_r + b) + 1];
            acc += (re * re + im * im) * lam[b] * lam[b];
        }
        w[s] = acc;
    }
}

/* ------------------------------------------------------------------------ */
/* Sampling                                                                  */
/* ------------------------------------------------------------------------ */

static int max_bond(int M, const int *bond)
{
    int m = 1;
    for (int k = 0; k <= M; ++k)
        if (bond[k] > m) m = bond[k];
    return m;
}

/*
 * Sample rows n = n0 .. n0+N-1 over the sites k0 .. k1-1 of an M-site chain.
 *
 * Row i starts from the left vector vstate[i] (2*ldv doubles: re, im of
 * bond[k0] entries) or, when vstate is NULL, from v_0 = [1] (then k0 must be
 * 0); with vstate non-NULL the row's final left vector (bond[k1] entries) is
 * written back there, so a chain can be sampled in segments.
 * samples[i*M + k] = outcome of row n0+i at site k (columns k0..k1-1 written);
 * logprob[i] += sum_k log p(s_k | s_<k) over the segment (set to 0 first by
 * the caller or by orc_sample).  probs (nullable, [N][M][d]) receives the
 * normalised conditionals p(s | prefix) = w_s / Z.  forced (nullable,
 * [N][M]): teacher-forced replay; the row follows the given outcomes instead
 * of its own draws, while own_draw (nullable, [N][M]) records the outcome its
 * own uniform would have picked and margin (nullable, [N][M]) the distance
 * min_s |u - C_s/Z| of that uniform to the nearest interior CDF boundary.
 * A holds one pointer per site, interleaved complex doubles or, with
 * a_is_f32, complex floats.  lam (nullable): Vidal form, lam[k] = Lambda_k
 * (bond[k+1] doubles) and A[k] = Gamma_k.  mu (nullable): GBS displacement,
 * interleaved complex doubles, amplitude of row i at site k at
 * mu[2*(k*ldmu + i)] (re) and +1 (im).  nlist (nullable): row i is sample
 * nlist[i] (its uniform is keyed by that index) instead of n0+i.  Returns 0,
 * -1 on bad arguments, -2 on allocation failure.
 */
int orc_sample_segment(int M, int d, const int *bond, const void *const *A, int a_is_f32, uint64_t seed,
                       uint32_t job, int64_t n0, int64_t N, int k0, int k1, double *vstate, int ldv,
                       uint8_t *samples, double *logprob, double *probs, const uint8_t *forced,
                       uint8_t *own_draw, double *margin, int nthreads, const double *const *lam,
                       const double *mu, int64_t ldmu, const int64_t *nlist)
{
    if (M < 1 || d < 2 || d > 255 || N < 0 || !bond || !A) return -1;
    if (mu && ldmu < N) return -1;
    if (k0 < 0 || k1 > M || k0 > k1) return -1;
    if (!vstate && k0 != 0) return -1;
    if (bond[0] != 1 || bond[M] != 1) return -1;
    const int chi = max_bond(M, bond);
    if (vstate && ldv < chi) return -1;
    int bad = 0;
    enum { B = ORC_BATCH };
    /* rows per batch: ORC_BATCH, or fewer when the rows would not keep every thread busy (a batch's
     * sums are those of its samples taken one by one, so the batch size changes no result) */
    int64_t bsz = B;
#ifdef _OPENMP
    /* threads of this call only (a num_threads clause leaves the process default unchanged) */
    const int nth = nthreads > 0 ? nthreads : omp_get_max_threads();
    {
        const int64_t per = nth > 0 ? (N + nth - 1) / nth : (int64_t)B;
        if (per < bsz) bsz = per < 1 ? 1 : per;
    }
#pragma omp parallel num_threads(nth) reduction(| : bad)
#endif
    {
        double *vbuf = (double *)malloc(sizeof(double) * 2 * (size_t)chi * B);
        double *ybuf = (double *)malloc(sizeof(double) * 2 * (size_t)d * chi * B);
        double *w = (double *)malloc(sizeof(double) * (size_t)d);
        double *Dm = (double *)malloc(sizeof(double) * 2 * (size_t)d * d);
        double *ytmp = (double *)malloc(sizeof(double) * 2 * (size_t)d * chi);
        if (!vbuf || !ybuf || !w || !Dm || !ytmp) bad = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t i0 = 0; i0 < N; i0 += bsz) {
            if (bad) continue;
            const int nb = (int)(N - i0 < bsz ? N - i0 : bsz);
            double lps[B];
            int deads[B];
            double *vr_[B], *yr_[B];
            for (int j = 0; j < nb; ++j) {
                const int64_t i = i0 + j;
                double *v = vbuf + (size_t)j * 2 * chi;
                if (vstate) {
                    for (int b = 0; b < 2 * bond[k0]; ++b) v[b] = vstate[(size_t)i * 2 * ldv + b];
                } else {
                    v[0] = 1.0;
                    v[1] = 0.0;
                }
                lps[j] = 0.0;
                deads[j] = 0;
            }
            for (int k = k0; k < k1; ++k) {
                const int cl = bond[k], cr = bond[k + 1];
                /* the contraction of every live sample of the batch at site k */
                int nl = 0;
                for (int j = 0; j < nb; ++j)
                    if (!deads[j]) {
                        vr_[nl] = vbuf + (size_t)j * 2 * chi;
                        yr_[nl] = ybuf + (size_t)j * 2 * d * chi;
                        ++nl;
                    }
                orc_contract(nl, vr_, cl, d, cr, A[k], a_is_f32, yr_);
                for (int j = 0; j < nb; ++j) {
                    const int64_t i = i0 + j;
                    const uint64_t n = nlist ? (uint64_t)nlist[i] : (uint64_t)(n0 + i);
                    double *v = vbuf + (size_t)j * 2 * chi;
                    double *y = ybuf + (size_t)j * 2 * d * chi;
                    if (deads[j]) {
                        if (samples) samples[i * M + k] = 0;
                        if (own_draw) own_draw[i * M + k] = 0;
                        if (margin) margin[i * M + k] = INFINITY;
                        if (probs)
                            for (int t = 0; t < d; ++t) probs[((size_t)i * M + k) * d + t] = NAN;
                        continue;
                    }
                    if (mu) {
                        const double *m = mu + 2 * ((size_t)k * ldmu + (size_t)i);
                        orc_displacement(m[0], m[1], d, Dm);
                        orc_displace(y, d, cr, Dm, ytmp);
                    }
                    if (lam)
                        orc_block_norms_lambda(y, d, cr, lam[k], w);
                    else
                        orc_block_norms(y, d, cr, w);
                    const double u = orc_uniform(seed, n, (uint32_t)k, job);
                    double Z, mg;
                    const int mine = orc_draw(w, d, u, &Z, &mg);
                    const int s = forced ? (int)forced[i * M + k] : mine;
                    if (own_draw) own_draw[i * M + k] = (uint8_t)mine;
                    if (margin) margin[i * M + k] = mg;
                    if (probs)
                        for (int t = 0; t < d; ++t) probs[((size_t)i * M + k) * d + t] = w[t] / Z;
                    if (samples) samples[i * M + k] = (uint8_t)s;
                    if (s < 0 || s >= d || !(w[s] > 0.0)) {
                        /* a forced outcome of zero probability: the replay of this row stops */
                        lps[j] = -INFINITY;
                        deads[j] = 1;
                        continue;
                    }
                    lps[j] += log(w[s]) - log(Z);
                    const double inv = 1.0 / sqrt(w[s]);
                    for (int b = 0; b < cr; ++b) {
                        v[2 * b] = y[2 * (s * cr + b)] * inv;
                        v[2 * b + 1] = y[2 * (s * cr + b) + 1] * inv;
                    }
                    if (lam)
                        for (int b = 0; b < cr; ++b) {
                            v[2 * b] *= lam[k][b];
                            v[2 * b + 1] *= lam[k][b];
                        }
                }
            }
            for (int j = 0; j < nb; ++j) {
                const int64_t i = i0 + j;
                const double *v = vbuf + (size_t)j * 2 * chi;
                if (logprob) logprob[i] += lps[j];
                if (vstate)
                    for (int b = 0; b < 2 * bond[k1]; ++b) vstate[(size_t)i * 2 * ldv + b] = deads[j] ? NAN : v[b];
            }
        }
        free(vbuf);
        free(ybuf);
        free(w);
        free(Dm);
        free(ytmp);
    }
    return bad ? -2 : 0;
}

/* Whole chain from v_0 = [1]; logprob[i] is overwritten.  See orc_sample_segment. */
int orc_sample(int M, int d, const int *bond, const double *const *A, uint64_t seed, uint32_t job,
               int64_t n0, int64_t N, uint8_t *samples, double *logprob, double *probs,
               const uint8_t *forced, uint8_t *own_draw, double *margin, int nthreads)
{
    if (logprob)
        for (int64_t i = 0; i < N; ++i) logprob[i] = 0.0;
    return orc_sample_segment(M, d, bond, (const void *const *)A, 0, seed, job, n0, N, 0, M, NULL, 0, samples,
                              logprob, probs, forced, own_draw, margin, nthreads, NULL, NULL, 0, NULL);
}

/* ------------------------------------------------------------------------ */
/* Closed forms used as pins                                                 */
/* ------------------------------------------------------------------------ */

/*
 * log |psi(s)|^2 = log |A_0[s_0] A_1[s_1] ... A_{M-1}[s_{M-1}]|^2 for one
 * configuration: the Born probability of the plain definition, by a left to
 * right chain of vector-matrix products with the running norm factored out
 * (log-norm tracking) so that long chains do not underflow.
 */
double orc_born_logprob(int M, int d, const int *bond, const double *const *A, const uint8_t *config)
{
    const int chi = max_bond(M, bond);
    double *r = (double *)calloc(2 * (size_t)chi, sizeof(double));
    double *t = (double *)calloc(2 * (size_t)chi, sizeof(double));
    if (!r || !t) {
        free(r);
        free(t);
        return NAN;
    }
    r[0] = 1.0;
    double lognorm = 0.0;
    for (int k = 0; k < M; ++k) {
        const int cl = bond[k], cr = bond[k + 1], s = config[k];
        for (int b = 0; b < cr; ++b) {
            double re = 0.0, im = 0.0;
            for (int a = 0; a < cl; ++a) {
                const double *e = A[k] + 2 * (((size_t)a * d + s) * cr + b);
                re += r[2 * a] * e[0] - r[2 * a + 1] * e[1];
                im += r[2 * a] * e[1] + r[2 * a + 1] * e[0];
            }
            t[2 * b] = re;
            t[2 * b + 1] = im;
        }
        double nrm2 = 0.0;
        for (int b = 0; b < cr; ++b) nrm2 += t[2 * b] * t[2 * b] + t[2 * b + 1] * t[2 * b + 1];
        if (!(nrm2 > 0.0)) {
            free(r);
            free(t);
            return -INFINITY;
        }
        lognorm += log(nrm2);
        const double inv = 1.0 / sqrt(nrm2);
        for (int b = 0; b < cr; ++b) {
            r[2 * b] = t[2 * b] * inv;
            r[2 * b + 1] = t[2 * b + 1] * inv;
        }
    }
    free(r);
    free(t);
    return lognorm;
}

/*
 * Brute force: |psi(s)|^2 for every configuration, index = sum_k s_k d^(M-1-k)
 * (s_0 most significant).  Depth-first over prefixes so that each prefix
 * vector A_0[s_0]...A_k[s_k] is formed once; no normalisation, no sampling.
 * out has d^M entries.
 */
static void orc_bf_rec(int M, int d, const int *bond, const double *const *A, int k, const double *pref,
                       size_t index, double *out, double *scratch)
{
    const int cl = bond[k], cr = bond[k + 1];
    double *next = scratch; /* 2*cr doubles for this depth */
    for (int s = 0; s < d; ++s) {
        for (int b = 0; b < cr; ++b) {
            double re = 0.0, im = 0.0;
            for (int a = 0; a < cl; ++a) {
                const double *e = A[k] + 2 * (((size_t)a * d + s) * cr + b);
                re += pref[2 * a] * e[0] - pref[2 * a + 1] * e[1];
                im += pref[2 * a] * e[1] + pref[2 * a + 1] * e[0];
            }
            next[2 * b] = re;
            next[2 * b + 1] = im;
        }
        const size_t idx = index * (size_t)d + (size_t)s;
        if (k == M - 1) {
            out[idx] = next[0] * next[0] + next[1] * next[1];
        } else {
            orc_bf_rec(M, d, bond, A, k + 1, next, idx, out, scratch + 2 * (size_t)cr);
        }
    }
}

int orc_brute_force(int M, int d, const int *bond, const double *const *A, double *out)
{
    if (M < 1 || M > 24 || d < 2) return -1;
    int total_scratch = 0;
    for (int k = 0; k <= M; ++k) total_scratch += 2 * bond[k];
    double *scratch = (double *)calloc((size_t)total_scratch + 2, sizeof(double));
    if (!scratch) return -2;
    double one[2] = {1.0, 0.0};
    orc_bf_rec(M, d, bond, A, 0, one, 0, out, scratch);
    free(scratch);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
