/*
 * mc_oracle.c -- plain, slow CPU oracle for hash- and stride-seeded LCG
 * streams and the Monte Carlo transport built on them, after
 * B. S. Cuneo and I. Variansyah, "An Alternative to Stride-Based RNG for
 * Monte Carlo Transport" (arXiv 2403.06362).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The CUDA library is
 * the product; it shares no code, header or table with this file and never
 * calls it.
 *
 * Written to be checked against the paper by eye, not to be fast:
 *   - fp64 throughout, built with -O2 -ffp-contract=off (every a*b+c rounds
 *     twice), default round-to-nearest;
 *   - integer arithmetic in uint64_t, where C's unsigned wrap-around is the
 *     "mod 2^64" of the paper, followed by a mask for "mod 2^m";
 *   - the skip-ahead count Q*k is carried in 128 bits, so no periodicity
 *     argument is needed to reduce it.
 *
 * Readings of points the paper leaves open are marked READING; every one is
 * listed in the design notes of the repository.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mc_oracle.h"

/* ---------------------------------------------------------------------------
 * Section 2, Eq. (1): the LCG.  X_{n+1} = (g X_n + c) mod 2^m; the new state
 * is also the output.
 * ------------------------------------------------------------------------- */

uint64_t or_mask(uint32_t m) { return m >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << m) - 1); }

uint64_t or_lcg_next(uint64_t x, uint32_t m, uint64_t g, uint64_t c) {
    /* (g*x + c) wraps mod 2^64; 2^m divides 2^64, so masking gives mod 2^m. */
    return (g * x + c) & or_mask(m);
}

/* READING (uniform): the top 53 of the m state bits, scaled by 2^-53, i.e.
 * u = floor(X / 2^(m-53)) * 2^-53 in [0,1).  States narrower than 53 bits
 * are scaled by 2^-m.  Both are exact in fp64. */
double or_u01(uint64_t x, uint32_t m) {
    if (m >= 53) return (double)(x >> (m - 53)) * 0x1p-53;
    return ldexp((double)x, -(int)m);
}

/* ---------------------------------------------------------------------------
 * Section 3, Eq. (2): Brown's skip-ahead.
 * READING: the printed first term lacks the X_0 factor; the skip is
 *   X_k = g^k X_0 + c (1 + g + ... + g^(k-1))   (mod 2^m),
 * evaluated with Brown's binary method: (h, f) is the affine map of 2^j
 * steps, x -> h x + f, and the maps for the set bits of k are composed.
 * The maps are all powers of one map, so they commute.
 * ------------------------------------------------------------------------- */

static uint64_t skip128(uint64_t x0, unsigned __int128 k, uint32_t m, uint64_t g, uint64_t c) {
    uint64_t G = 1, C = 0;     /* accumulated map x -> G x + C */
    uint64_t h = g, f = c;     /* map of 2^j steps             */
    while (k != 0) {
        if (k & 1) {
            G = G * h;
            C = C * h + f;
        }
        f = f * (h + 1);       /* 2^(j+1) steps: h(hx+f)+f = h^2 x + f(h+1) */
        h = h * h;
        k >>= 1;
    }
    return (G * x0 + C) & or_mask(m);
}

uint64_t or_lcg_skip(uint64_t x0, uint64_t k, uint32_t m, uint64_t g, uint64_t c) {
    return skip128(x0, (unsigned __int128)k, m, g, c);
}

/* Section 3: unit u_k is assigned X_{Qk}, counted from X_0 (unit 0 gets X_0). */
uint64_t or_stride_seed(uint64_t x0, uint64_t q, uint64_t k, uint32_t m, uint64_t g, uint64_t c) {
    return skip128(x0, (unsigned __int128)q * (unsigned __int128)k, m, g, c);
}

/* ---------------------------------------------------------------------------
 * Section 4, Listing 1; Eq. (3): the hash of a key k under a parent seed s.
 * It is built from one mixing map on 64-bit words,
 *   mix(v) = p XOR floor(p / 2^47),   p = v * M mod 2^64,
 * with M the multiplier the listing prints.  The seed enters as
 * a = mix(s XOR (8 M mod 2^64)), the key as b = mix(k) * M mod 2^64, and the
 * hash is mix(a XOR b).  READING: every value is an unsigned 64-bit word and
 * every product is taken mod 2^64; here each product is formed exactly in
 * 128 bits and reduced by keeping its low word, and the shift is logical.
 * ------------------------------------------------------------------------- */

#define OR_MURMUR_M 0xC6A4A7935BD1E995ULL

static uint64_t or_mulmod64(uint64_t a, uint64_t b) {
    const unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    return (uint64_t)(p & (unsigned __int128)UINT64_MAX);
}

/* mix(v); exported under the listing's name for the tests. */
uint64_t or_subhash(uint64_t v) {
    const uint64_t p = or_mulmod64(v, OR_MURMUR_M);
    return p ^ (p >> 47);
}

uint64_t or_hash(uint64_t k, uint64_t s) {
    const uint64_t a = or_subhash(s ^ or_mulmod64(8, OR_MURMUR_M));
    const uint64_t b = or_mulmod64(or_subhash(k), OR_MURMUR_M);
    return or_subhash(a ^ b);
}

/* Eq. (3) S_k = hash(k, s), and Eq. (4) S_{i,j} = hash(j, hash(i, s)).
 * READING: the 64-bit hash becomes an m-bit LCG state by keeping its low
 * m bits ("mod 2^m"); keys are 0-based history ids. */
uint64_t or_hash_seed(uint64_t k, uint64_t s, uint32_t m) { return or_hash(k, s) & or_mask(m); }

void or_seed_hash(uint32_t m, uint64_t parent, uint64_t key_begin, uint64_t count, uint64_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = or_hash_seed(key_begin + i, parent, m);
}

void or_seed_stride(uint32_t m, uint64_t g, uint64_t c, uint64_t x0, uint64_t q, uint64_t id_begin,
                    uint64_t count, uint64_t* out) {
    for (uint64_t i = 0; i < count; ++i) out[i] = or_stride_seed(x0, q, id_begin + i, m, g, c);
}

/* Draws: each stream advances `draws` times; draw j of stream i is the
 * uniform of its (j+1)-th state (the seed itself is never an output).
 * u (nullable) is draw-major: u[j*n + i].  digest (nullable) is the
 * wrapping 64-bit sum of the IEEE-754 bit patterns of the stream's draws. */
void or_lcg_draw(uint32_t m, uint64_t g, uint64_t c, uint64_t* states, uint64_t n, uint32_t draws,
                 double* u, uint64_t* digest) {
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t x = states[i], sum = 0;
        for (uint32_t j = 0; j < draws; ++j) {
            x = or_lcg_next(x, m, g, c);
            double v = or_u01(x, m);
            uint64_t bits;
            memcpy(&bits, &v, sizeof bits);
            sum += bits;
            if (u) u[(uint64_t)j * n + i] = v;
        }
        states[i] = x;
        if (digest) digest[i] = sum;
    }
}

/* ---------------------------------------------------------------------------
 * One-speed slab transport, history-based (Section 1 and Section 5 describe
 * the setting; the paper gives no transport code, so every step below is a
 * READING, fixed once so that any implementation can reproduce it draw for
 * draw):
 *   source   isotropic:  x = L*u, mu = 2u - 1       (two draws)
 *            beam:       x = 0,   mu = 1            (no draw)
 *   flight   d = -ln(1 - u) * (1/Sigma_t); x' = x + d*mu
 *            mu > 0 and x' >= L: leak at L;  mu < 0 and x' <= 0: leak at 0
 *   collide  absorb iff u < 1 - c; else mu = 2u - 1
 *   tally    track length in bin j = |[a,b] & [e_j, e_{j+1}]| * (1/|mu|),
 *            e_j = j*(L/nb) for j < nb, e_nb = L; fixed point
 *            llrint(length * 2^32) into int64 bins per batch.
 * 1/|mu| is rounded once per direction; mu == 0 adds d to the bin holding x.
 * ------------------------------------------------------------------------- */

typedef struct {
    uint64_t x;
    uint64_t draws;
    uint32_t m;
    uint64_t g, c;
} or_rng;

static double or_next(or_rng* r) {
    r->x = or_lcg_next(r->x, r->m, r->g, r->c);
    r->draws++;
    return or_u01(r->x, r->m);
}

uint64_t or_slab_seed(const or_lcg* l, const or_slab_problem* p, uint64_t id) {
    switch (p->seeding) {
    case OR_SEED_HASH:
        return or_hash_seed(id, p->seed, l->m);                       /* Eq. (3) */
    case OR_SEED_HASH_HIER:
        return or_hash_seed(id, or_hash(p->key, p->seed), l->m);      /* Eq. (4) */
    default:
        return or_stride_seed(p->seed, p->stride_q, p->id_offset + id, l->m, l->g, l->c);
    }
}

static double edge(const or_slab_problem* p, double h, uint32_t j) {
    return j >= p->n_bins ? p->L : (double)j * h;
}

static void tally_segment(const or_slab_problem* p, double h, double a, double b, double w_mu,
                          int64_t* t, double* tf) {
    for (uint32_t j = 0; j < p->n_bins; ++j) {
        double lo_e = edge(p, h, j), hi_e = edge(p, h, j + 1);
        double lo = a > lo_e ? a : lo_e;
        double hi = b < hi_e ? b : hi_e;
        if (hi > lo) {
            double ell = (hi - lo) * w_mu;
            t[j] += llrint(ell * 4294967296.0);
            if (tf) tf[j] += ell;
        }
    }
}

static void tally_point(const or_slab_problem* p, double h, double x, double d, int64_t* t, double* tf) {
    uint32_t j = 0;
    while (j + 1 < p->n_bins && x >= edge(p, h, j + 1)) ++j;
    t[j] += llrint(d * 4294967296.0);
    if (tf) tf[j] += d;
}

uint64_t or_batch_of(uint64_t id, uint64_t n_histories, uint32_t n_batches) {
    return (uint64_t)(((unsigned __int128)id * n_batches) / n_histories);
}

static void finish_history(const or_slab_problem* p, const or_rng* r, uint64_t* cnt) {
    cnt[OR_C_DRAWS] += r->draws;
    if (r->draws > cnt[OR_C_MAX_DRAWS]) cnt[OR_C_MAX_DRAWS] = r->draws;
    if (p->stride_q != 0 && r->draws > p->stride_q) {
        cnt[OR_C_EXCEED_HIST] += 1;
        cnt[OR_C_EXCEED_DRAWS] += r->draws - p->stride_q;
    }
}

int or_slab_run(const or_lcg* l, const or_slab_problem* p, uint64_t id_begin, uint64_t id_end,
                uint64_t event_cap, int64_t* tally, double* tally_fp, uint64_t* counts,
                uint64_t* hist_state, uint64_t* hist_draws) {
    const double h = p->L / (double)p->n_bins;
    const double inv_st = 1.0 / p->sigma_t;
    const double p_abs = 1.0 - p->c;
    int status = 0;
    for (uint64_t id = id_begin; id < id_end; ++id) {
        uint64_t batch = or_batch_of(id, p->n_histories, p->n_batches);
        int64_t* t = tally + p->tally_offset + batch * p->n_bins;
        double* tf = tally_fp ? tally_fp + p->tally_offset + batch * p->n_bins : NULL;
        or_rng r = {or_slab_seed(l, p, id), 0, l->m, l->g, l->c};
        double x, mu;
        if (p->source == OR_SRC_BEAM) {
            x = 0.0;
            mu = 1.0;
        } else {
            x = p->L * or_next(&r);
            mu = 2.0 * or_next(&r) - 1.0;
        }
        double w_mu = mu != 0.0 ? 1.0 / fabs(mu) : 0.0;
        counts[OR_C_SOURCE]++;
        for (uint64_t events = 0;; ++events) {
            if (events == event_cap) {
                counts[OR_C_CAPPED]++;
                status = 1;
                break;
            }
            counts[OR_C_FLIGHTS]++;
            double u = or_next(&r);
            double d = -log(1.0 - u) * inv_st;
            double xn = x + d * mu;
            if (mu > 0.0 && xn >= p->L) {
                tally_segment(p, h, x, p->L, w_mu, t, tf);
                counts[OR_C_LEAK_HI]++;
                break;
            }
            if (mu < 0.0 && xn <= 0.0) {
                tally_segment(p, h, 0.0, x, w_mu, t, tf);
                counts[OR_C_LEAK_LO]++;
                break;
            }
            if (mu == 0.0)
                tally_point(p, h, x, d, t, tf);
            else if (mu > 0.0)
                tally_segment(p, h, x, xn, w_mu, t, tf);
            else
                tally_segment(p, h, xn, x, w_mu, t, tf);
            x = xn;
            counts[OR_C_COLLISIONS]++;
            if (or_next(&r) < p_abs) {
                counts[OR_C_ABSORPTIONS]++;
                break;
            }
            counts[OR_C_SCATTERS]++;
            mu = 2.0 * or_next(&r) - 1.0;
            w_mu = mu != 0.0 ? 1.0 / fabs(mu) : 0.0;
        }
        finish_history(p, &r, counts);
        if (hist_state) hist_state[id - id_begin] = r.x;
        if (hist_draws) hist_draws[id - id_begin] = r.draws;
    }
    return status;
}

/* ---------------------------------------------------------------------------
 * Section 5 statistics: normalised deviations of batch means and the
 * Shapiro-Wilk test.  READING: the W statistic and its p-value follow
 * Royston's approximation (Royston 1992, "Approximating the Shapiro-Wilk
 * W-test for non-normality", Stat. Comput. 2:117-119; Algorithm AS R94,
 * Appl. Statist. 44:547-551, 1995), valid for 3 <= n <= 5000.
 * ------------------------------------------------------------------------- */

double or_norm_cdf(double z) { return 0.5 * erfc(-z / sqrt(2.0)); }

/* Inverse of the standard normal CDF by plain bisection on or_norm_cdf:
 * slow and obviously monotone; stops when the bracket no longer shrinks. */
double or_norm_ppf(double p) {
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (or_norm_cdf(mid) < p)
            lo = mid;
        else
            hi = mid;
    }
    return 0.5 * (lo + hi);
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double poly(const double* c, int nc, double x) {
    double r = 0.0, xp = 1.0;
    for (int i = 0; i < nc; ++i) {
        r += c[i] * xp;
        xp *= x;
    }
    return r;
}

/* Returns 0 on success, -1 for n < 3 or n > 5000 or zero spread. */
int or_shapiro_wilk(const double* x_in, int n, double* w_out, double* p_out) {
    if (n < 3 || n > 5000) return -1;
    double* x = (double*)malloc(sizeof(double) * (size_t)n);
    double* a = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(x, x_in, sizeof(double) * (size_t)n);
    qsort(x, (size_t)n, sizeof(double), cmp_double);

    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += x[i];
    mean /= n;
    double ss = 0.0;
    for (int i = 0; i < n; ++i) ss += (x[i] - mean) * (x[i] - mean);
    if (!(ss > 0.0)) {
        free(x);
        free(a);
        return -1;
    }

    double W, pval;
    if (n == 3) {
        /* Exact weights (-sqrt(1/2), 0, sqrt(1/2)) and exact p-value. */
        double s = sqrt(0.5);
        double num = s * (x[2] - x[0]);
        W = num * num / ss;
        if (W < 0.75) W = 0.75;
        pval = (6.0 / M_PI) * (asin(sqrt(W)) - asin(sqrt(0.75)));
    } else {
        /* Expected normal order statistics (Blom-type scores). */
        double mm = 0.0;
        for (int i = 0; i < n; ++i) {
            a[i] = or_norm_ppf(((double)(i + 1) - 0.375) / ((double)n + 0.25));
            mm += a[i] * a[i];
        }
        /* Royston's polynomial corrections for the two outermost weights. */
        static const double c1[6] = {0.0, 0.221157, -0.147981, -2.071190, 4.434685, -2.706056};
        static const double c2[6] = {0.0, 0.042981, -0.293762, -1.752461, 5.682633, -3.582633};
        double u = 1.0 / sqrt((double)n);
        double m_n = a[n - 1], m_n1 = a[n - 2];
        double an = m_n / sqrt(mm) + poly(c1, 6, u);
        double phi;
        double* coef = (double*)malloc(sizeof(double) * (size_t)n);
        if (n > 5) {
            double an1 = m_n1 / sqrt(mm) + poly(c2, 6, u);
            phi = (mm - 2.0 * m_n * m_n - 2.0 * m_n1 * m_n1) / (1.0 - 2.0 * an * an - 2.0 * an1 * an1);
            for (int i = 0; i < n; ++i) coef[i] = a[i] / sqrt(phi);
            coef[n - 1] = an;
            coef[0] = -an;
            coef[n - 2] = an1;
            coef[1] = -an1;
        } else {
            phi = (mm - 2.0 * m_n * m_n) / (1.0 - 2.0 * an * an);
            for (int i = 0; i < n; ++i) coef[i] = a[i] / sqrt(phi);
            coef[n - 1] = an;
            coef[0] = -an;
        }
        double num = 0.0;
        for (int i = 0; i < n; ++i) num += coef[i] * x[i];
        free(coef);
        W = num * num / ss;
        if (W > 1.0) W = 1.0;

        /* Royston's normalising transformation of 1 - W. */
        double z;
        if (n <= 11) {
            double gam = -2.273 + 0.459 * n;
            static const double cm[4] = {0.5440, -0.39978, 0.025054, -0.0006714};
            static const double cs[4] = {1.3822, -0.77857, 0.062767, -0.0020322};
            double mu = poly(cm, 4, (double)n);
            double sg = exp(poly(cs, 4, (double)n));
            double y = log(1.0 - W);
            if (y >= gam) {
                z = 1e10;
            } else {
                z = (-log(gam - y) - mu) / sg;
            }
        } else {
            double ln = log((double)n);
            static const double cm[4] = {-1.5861, -0.31082, -0.083751, 0.0038915};
            static const double cs[3] = {-0.4803, -0.082676, 0.0030302};
            double mu = poly(cm, 4, ln);
            double sg = exp(poly(cs, 3, ln));
            z = (log(1.0 - W) - mu) / sg;
        }
        pval = or_norm_cdf(-z); /* upper tail, without cancellation */
    }
    free(x);
    free(a);
    *w_out = W;
    *p_out = pval;
    return 0;
}

/* Section 5: for each data point (column) of x[n_batches][n_points], the
 * normalised deviations z = (x - mean)/sd over the batches (sd with n-1;
 * READING) and the Shapiro-Wilk W and p of that column. */
int or_batch_stats(const double* x, uint32_t n_batches, uint32_t n_points, double* z, double* w,
                   double* p) {
    int status = 0;
    double* col = (double*)malloc(sizeof(double) * n_batches);
    for (uint32_t j = 0; j < n_points; ++j) {
        double mean = 0.0;
        for (uint32_t b = 0; b < n_batches; ++b) mean += x[(uint64_t)b * n_points + j];
        mean /= n_batches;
        double var = 0.0;
        for (uint32_t b = 0; b < n_batches; ++b) {
            double dv = x[(uint64_t)b * n_points + j] - mean;
            var += dv * dv;
        }
        double sd = n_batches > 1 ? sqrt(var / (n_batches - 1)) : 0.0;
        for (uint32_t b = 0; b < n_batches; ++b) {
            col[b] = x[(uint64_t)b * n_points + j];
            if (z) z[(uint64_t)b * n_points + j] = sd > 0.0 ? (col[b] - mean) / sd : 0.0;
        }
        double wj = 0.0, pj = 0.0;
        if (or_shapiro_wilk(col, (int)n_batches, &wj, &pj) != 0) {
            status = -1;
            wj = pj = NAN;
        }
        if (w) w[j] = wj;
        if (p) p[j] = pj;
    }
    free(col);
    return status;
}
