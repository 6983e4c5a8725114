/*
 * mc_oracle_azurv1.c -- CPU oracle for the paper's own test problem
 * (Section 5): a supercritical, time-dependent, mono-energetic problem in an
 * infinite homogeneous medium driven by a pulse at t = x = 0, with the
 * collision-estimator flux averaged over x in [-h, h] in unit time bins.
 *
 * TEST INFRASTRUCTURE ONLY (see mc_oracle.c).  Plain fp64, -ffp-contract=off.
 *
 * READINGS (the paper names the problem and its parameters, not the
 * algorithm):
 *   units      Sigma_t = 1, speed 1, so a flight of length d takes time d
 *   source     x = 0, t = 0, mu = 2u - 1 (one draw)
 *   flight     d = -ln(1-u) / Sigma_t; t' = t + d; t' >= T ends the particle
 *              at census; else x' = x + d mu and the particle collides
 *   tally      collision estimator: a collision with -h <= x' <= h and
 *              t' < T adds llrint(2^32 / Sigma_t) to time bin floor(t')
 *   collision  u < c (= Sigma_s/Sigma_t): scattering with multiplicity
 *              n = floor(nu + u) outgoing particles; otherwise absorption.
 *              On scattering, n - 1 secondaries are created at (x', t');
 *              then the incident particle continues with mu = 2u - 1
 *   secondaries  hash mode (Eq. 5): secondary k = 0..n-2 gets its own
 *              stream, seeded hash(k, S_p) mod 2^m with S_p the parent's
 *              state after the multiplicity draw; stride mode: secondaries
 *              draw from the history's one stream.  Either way they wait on
 *              a last-in first-out stack and are followed depth-first once
 *              the current particle ends; each starts with mu = 2u - 1
 *   seeds      global history index g = (rep * B + batch) * P + particle;
 *              hash: hash(g, s); hierarchical: hash(particle, hash(batch,
 *              hash(rep, s))) (Eq. 4 twice); stride: X_{Q (id_offset + g)}
 * Per history the oracle reports the final state and draw count of the
 * source particle's stream (hash) or of the history's stream (stride).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mc_oracle.h"

typedef struct {
    double x, t;
    uint64_t seed;
} az_entry;

typedef struct {
    uint64_t x, draws;
    uint32_t m;
    uint64_t g, c;
} az_rng;

static double az_next(az_rng* r) {
    r->x = or_lcg_next(r->x, r->m, r->g, r->c);
    r->draws++;
    return or_u01(r->x, r->m);
}

uint64_t or_azurv1_seed(const or_lcg* l, const or_azurv1_problem* a, uint64_t g) {
    const uint64_t P = a->per_batch, B = a->n_batches;
    switch (a->seeding) {
    case OR_SEED_HASH:
        return or_hash_seed(g, a->seed, l->m);
    case OR_SEED_HASH_HIER: {
        uint64_t rep = g / (P * B), batch = (g / P) % B, part = g % P;
        return or_hash_seed(part, or_hash(batch, or_hash(rep, a->seed)), l->m);
    }
    default:
        return or_stride_seed(a->seed, a->stride_q, a->id_offset + g, l->m, l->g, l->c);
    }
}

int or_azurv1_run(const or_lcg* l, const or_azurv1_problem* a, uint64_t g_begin, uint64_t g_end,
                  uint64_t event_cap, int64_t* tally, uint64_t* counts, uint64_t* hist_state,
                  uint64_t* hist_draws) {
    if (a->n_census >= 2) return or_azurv1_census_run(l, a, g_begin, g_end, event_cap, tally, counts, 0, NULL, NULL);
    const int hash_mode = a->seeding != OR_SEED_STRIDE;
    const double inv_st = 1.0 / a->sigma_t;
    const int64_t unit = llrint(inv_st * 4294967296.0);
    size_t cap = 64, sp = 0;
    az_entry* st = (az_entry*)malloc(cap * sizeof(az_entry));
    int status = 0;
    for (uint64_t g = g_begin; g < g_end; ++g) {
        const uint64_t rb = g / a->per_batch; /* rep * B + batch */
        int64_t* row = tally + a->tally_offset + rb * a->n_time_bins;
        az_rng r = {or_azurv1_seed(l, a, g), 0, l->m, l->g, l->c};
        uint64_t fam_draws = 0;
        int primary = 1;
        double x = 0.0, t = 0.0, mu = 2.0 * az_next(&r) - 1.0;
        counts[OR_C_SOURCE]++;
        for (;;) {
            /* follow the current particle to its end */
            int ended = 0;
            for (uint64_t ev = 0; !ended; ++ev) {
                if (ev == event_cap) {
                    counts[OR_C_CAPPED]++;
                    status = 1;
                    break;
                }
                counts[OR_C_FLIGHTS]++;
                double d = -log(1.0 - az_next(&r)) * inv_st;
                double tn = t + d;
                if (tn >= a->t_end) {
                    counts[OR_C_LEAK_HI]++; /* census */
                    break;
                }
                double xn = x + d * mu;
                counts[OR_C_COLLISIONS]++;
                if (xn >= -a->x_half && xn <= a->x_half) {
                    uint64_t j = (uint64_t)floor(tn);
                    if (j >= a->n_time_bins) j = a->n_time_bins - 1;
                    row[j] += unit;
                }
                x = xn;
                t = tn;
                if (az_next(&r) < a->c) {
                    counts[OR_C_SCATTERS]++;
                    uint32_t n = (uint32_t)floor(a->nu + az_next(&r));
                    for (uint32_t k = 0; k + 1 < n; ++k) {
                        if (sp == cap) {
                            cap *= 2;
                            st = (az_entry*)realloc(st, cap * sizeof(az_entry));
                        }
                        st[sp].x = x;
                        st[sp].t = t;
                        st[sp].seed = hash_mode ? (or_hash(k, r.x) & or_mask(l->m)) : 0;
                        ++sp;
                        counts[OR_C_CHILDREN]++;
                    }
                    mu = 2.0 * az_next(&r) - 1.0;
                } else {
                    counts[OR_C_ABSORPTIONS]++;
                    ended = 1;
                }
            }
            if (hash_mode) {
                fam_draws += r.draws;
                if (r.draws > counts[OR_C_MAX_DRAWS]) counts[OR_C_MAX_DRAWS] = r.draws;
                if (primary) {
                    if (hist_state) hist_state[g - g_begin] = r.x;
                    if (hist_draws) hist_draws[g - g_begin] = r.draws;
                    if (a->stride_q != 0 && r.draws > a->stride_q) {
                        counts[OR_C_EXCEED_HIST]++;
                        counts[OR_C_EXCEED_DRAWS] += r.draws - a->stride_q;
                    }
                }
            }
            primary = 0;
            if (sp == 0) break;
            --sp;
            x = st[sp].x;
            t = st[sp].t;
            if (hash_mode) {
                r.x = st[sp].seed;
                r.draws = 0;
            }
            mu = 2.0 * az_next(&r) - 1.0;
        }
        if (!hash_mode) {
            fam_draws = r.draws;
            if (r.draws > counts[OR_C_MAX_DRAWS]) counts[OR_C_MAX_DRAWS] = r.draws;
            if (hist_state) hist_state[g - g_begin] = r.x;
            if (hist_draws) hist_draws[g - g_begin] = r.draws;
            if (a->stride_q != 0 && r.draws > a->stride_q) {
                counts[OR_C_EXCEED_HIST]++;
                counts[OR_C_EXCEED_DRAWS] += r.draws - a->stride_q;
            }
        }
        counts[OR_C_DRAWS] += fam_draws;
    }
    free(st);
    return status;
}
