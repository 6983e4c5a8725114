/*
 * mc_oracle_census.c -- CPU oracle of the pulse problem (Section 5) run in
 * census phases with population control by one-off hashed values
 * (Section 4: seed hashing gives deterministic one-off pseudo-random values,
 * e.g. for population control between batches, as long as every one-off
 * value drawn from one parent seed uses its own key; on-demand seeds of new
 * particles by Eq. 5).
 *
 * TEST INFRASTRUCTURE ONLY (see mc_oracle.c).  Plain fp64, -ffp-contract=off.
 *
 * READINGS (the paper names the use, not a scheme):
 *   phases    C = n_census phases [T_{p-1}, T_p): T_0 = 0, T_p = t_end p / C
 *             for 0 < p < C, T_C = t_end
 *   census    a flight with t + d >= T_p, p < C, stops at T_p:
 *             x <- x + (T_p - t) mu, and the particle is banked with its
 *             stream (state and draw count), direction and weight.  At T_C
 *             the particle ends (census count), as without phases
 *   groups    population control works per (repetition, batch) group, the
 *             unit of the batch statistics; groups never exchange particles
 *   control   at the end of phase p < C, for the group's banked particles:
 *               W   = sum_i llrint(w_i 2^32)         (exact integer sum)
 *               Wd  = W 2^-32,  N = target population
 *               xi_i = (hash(2^63 + p, S_i) >> 11) 2^-53
 *                     (one-off value; parent seed: the particle's state S_i;
 *                      key: 2^63 + p, disjoint from the child ordinals)
 *               n_i = floor(w_i (N / Wd) + xi_i) copies of weight Wd / N
 *             E[n_i] = w_i N / Wd, so the expected population is N and the
 *             expected weight is conserved (the tallies stay unbiased).
 *             Copy 0 continues the particle's stream; copy c >= 1 gets the
 *             stream hash(c - 1, S_i) mod 2^m (Eq. 5).  Copies keep x and mu
 *             and start at T_p.  W = 0 gives no copies.
 *   weights   secondaries inherit their parent's weight; a collision in
 *             [-h, h] adds llrint((w / Sigma_t) 2^32) to its time bin
 *   seeding   hash modes only: a stride-seeded stream cannot be given to a
 *             copy without numbering the copies across the whole population
 * Counters: BANKED (particles banked at a census T_p, p < C), SPLITS (copies
 * beyond the first), ROULETTE_KILLS (banked particles given no copy); a
 * stream's draws are counted where it ends (absorption, census at t_end, no
 * copy at a control, event cap).  Per-history outputs and the stride
 * exceedance are not defined in this mode.
 *
 * The result does not depend on the order in which particles are followed
 * or banked: `reverse` != 0 follows every list backwards (a test of that
 * property).  `pop` (nullable) receives, per group and phase, the number of
 * particles that start the phase: pop[(group - first group) * C + p - 1];
 * `wphase` (nullable) the weight every one of them carries (1 in phase 1,
 * Wd / N after each control), in the same layout.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mc_oracle.h"

#define CZ_ONEOFF_KEY 0x8000000000000000ull

typedef struct {
    double x, mu, w;
    uint64_t s, draws;
    int need_dir; /* a source particle draws its direction when it starts */
} cz_part;

typedef struct {
    double x, t;
    uint64_t seed;
} cz_sec;

typedef struct {
    cz_part* v;
    size_t n, cap;
} cz_list;

typedef struct {
    uint64_t x, draws;
    uint32_t m;
    uint64_t g, c;
} cz_rng;

static double cz_next(cz_rng* r) {
    r->x = or_lcg_next(r->x, r->m, r->g, r->c);
    r->draws++;
    return or_u01(r->x, r->m);
}

static void cz_push(cz_list* L, cz_part p) {
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->v = (cz_part*)realloc(L->v, L->cap * sizeof(cz_part));
    }
    L->v[L->n++] = p;
}

static double cz_census_time(const or_azurv1_problem* a, uint32_t p) {
    if (p == 0) return 0.0;
    if (p >= a->n_census) return a->t_end;
    return a->t_end * (double)p / (double)a->n_census;
}

static void cz_stream_end(uint64_t draws, uint64_t* counts) {
    counts[OR_C_DRAWS] += draws;
    if (draws > counts[OR_C_MAX_DRAWS]) counts[OR_C_MAX_DRAWS] = draws;
}

/* Follows particle `e` (starting at time t0) and the secondaries it creates
 * until each is absorbed or reaches T_p; banked particles go to `bank`. */
static int cz_follow(const or_lcg* l, const or_azurv1_problem* a, cz_part e, double t0, uint32_t p,
                     uint64_t event_cap, int64_t* row, uint64_t* counts, cz_list* bank, cz_sec** stk,
                     size_t* stk_cap) {
    const int last = p >= a->n_census;
    const double tp = cz_census_time(a, p);
    const double inv_st = 1.0 / a->sigma_t;
    const double w = e.w;
    const int64_t unit = llrint(w * inv_st * 4294967296.0);
    int status = 0;
    size_t sp = 0;
    cz_rng r = {e.s, e.draws, l->m, l->g, l->c};
    double x = e.x, t = t0, mu = e.mu;
    if (e.need_dir) mu = 2.0 * cz_next(&r) - 1.0;
    for (;;) {
        int banked = 0;
        for (uint64_t ev = 0;; ++ev) {
            if (ev == event_cap) {
                counts[OR_C_CAPPED]++;
                status = 1;
                break;
            }
            counts[OR_C_FLIGHTS]++;
            const double d = -log(1.0 - cz_next(&r)) * inv_st;
            const double tn = t + d;
            if (tn >= tp) {
                if (last) {
                    counts[OR_C_LEAK_HI]++;
                } else {
                    cz_part b = {x + (tp - t) * mu, mu, w, r.x, r.draws, 0};
                    cz_push(bank, b);
                    counts[OR_C_BANKED]++;
                    banked = 1;
                }
                break;
            }
            const double xn = x + d * mu;
            counts[OR_C_COLLISIONS]++;
            if (xn >= -a->x_half && xn <= a->x_half) {
                uint64_t j = (uint64_t)floor(tn);
                if (j >= a->n_time_bins) j = a->n_time_bins - 1;
                row[j] += unit;
            }
            x = xn;
            t = tn;
            if (cz_next(&r) < a->c) {
                counts[OR_C_SCATTERS]++;
                const uint32_t n = (uint32_t)floor(a->nu + cz_next(&r));
                for (uint32_t k = 0; k + 1 < n; ++k) {
                    if (sp == *stk_cap) {
                        *stk_cap *= 2;
                        *stk = (cz_sec*)realloc(*stk, *stk_cap * sizeof(cz_sec));
                    }
                    (*stk)[sp].x = x;
                    (*stk)[sp].t = t;
                    (*stk)[sp].seed = or_hash(k, r.x) & or_mask(l->m);
                    ++sp;
                    counts[OR_C_CHILDREN]++;
                }
                mu = 2.0 * cz_next(&r) - 1.0;
            } else {
                counts[OR_C_ABSORPTIONS]++;
                break;
            }
        }
        if (!banked) cz_stream_end(r.draws, counts);
        if (sp == 0) break;
        --sp;
        x = (*stk)[sp].x;
        t = (*stk)[sp].t;
        r.x = (*stk)[sp].seed;
        r.draws = 0;
        mu = 2.0 * cz_next(&r) - 1.0;
    }
    return status;
}

/* Population control of one group's bank at the end of phase p (Section 4,
 * one-off values; Eq. 5 for the copies' streams). */
static double cz_control(const or_lcg* l, const or_azurv1_problem* a, uint32_t p, const cz_list* bank,
                         cz_list* next, uint64_t* counts, int reverse) {
    const uint32_t target = a->pc_target ? a->pc_target : a->per_batch;
    int64_t W = 0;
    for (size_t i = 0; i < bank->n; ++i) W += llrint(bank->v[i].w * 4294967296.0);
    const double wd = (double)W * 0x1p-32;
    const double ratio = (double)target / wd;
    const double w_new = wd / (double)target;
    for (size_t q = 0; q < bank->n; ++q) {
        const cz_part* b = &bank->v[reverse ? bank->n - 1 - q : q];
        uint64_t n = 0;
        if (W > 0) {
            const double xi = (double)(or_hash(CZ_ONEOFF_KEY + p, b->s) >> 11) * 0x1p-53;
            n = (uint64_t)floor(b->w * ratio + xi);
        }
        if (n == 0) {
            counts[OR_C_ROULETTE_KILLS]++;
            cz_stream_end(b->draws, counts);
            continue;
        }
        counts[OR_C_SPLITS] += n - 1;
        for (uint64_t c = 0; c < n; ++c) {
            cz_part cp = {b->x, b->mu, w_new, c == 0 ? b->s : (or_hash(c - 1, b->s) & or_mask(l->m)),
                          c == 0 ? b->draws : 0, 0};
            cz_push(next, cp);
        }
    }
    return w_new;
}

int or_azurv1_census_run(const or_lcg* l, const or_azurv1_problem* a, uint64_t g_begin, uint64_t g_end,
                         uint64_t event_cap, int64_t* tally, uint64_t* counts, int reverse, uint64_t* pop,
                         double* wphase) {
    const uint64_t P = a->per_batch;
    if (a->seeding == OR_SEED_STRIDE || a->n_census < 2 || g_begin % P != 0 || g_end % P != 0) return -1;
    const uint32_t C = a->n_census;
    int status = 0;
    size_t stk_cap = 64;
    cz_sec* stk = (cz_sec*)malloc(stk_cap * sizeof(cz_sec));
    cz_list cur = {0}, bank = {0};
    for (uint64_t grp = g_begin / P; grp < g_end / P; ++grp) {
        int64_t* row = tally + a->tally_offset + grp * a->n_time_bins;
        cur.n = 0;
        for (uint64_t j = 0; j < P; ++j) {
            cz_part s = {0.0, 0.0, 1.0, or_azurv1_seed(l, a, grp * P + j), 0, 1};
            cz_push(&cur, s);
            counts[OR_C_SOURCE]++;
        }
        double w_phase = 1.0;
        for (uint32_t p = 1; p <= C; ++p) {
            if (pop) pop[(grp - g_begin / P) * C + (p - 1)] = cur.n;
            if (wphase) wphase[(grp - g_begin / P) * C + (p - 1)] = w_phase;
            const double t0 = cz_census_time(a, p - 1);
            bank.n = 0;
            for (size_t q = 0; q < cur.n; ++q) {
                const cz_part e = cur.v[reverse ? cur.n - 1 - q : q];
                status |= cz_follow(l, a, e, t0, p, event_cap, row, counts, &bank, &stk, &stk_cap);
            }
            cur.n = 0;
            if (p < C) w_phase = cz_control(l, a, p, &bank, &cur, counts, reverse);
        }
    }
    free(stk);
    free(cur.v);
    free(bank.v);
    return status;
}
