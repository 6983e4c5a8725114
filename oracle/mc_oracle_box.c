/*
 * mc_oracle_box.c -- CPU oracle for multigroup transport in a two-region
 * box with weight windows, where the children of a split are seeded on
 * demand by S_c = hash(k, S_p) (Section 4, Eq. 5).
 *
 * TEST INFRASTRUCTURE ONLY (see mc_oracle.c).  Plain fp64, -ffp-contract=off.
 *
 * The paper gives no transport code; every step below is a READING, fixed so
 * that any implementation can reproduce it draw for draw:
 *   geometry   box [0,S]^3, inner cube [lo,hi]^3 = region 1, the rest region 0;
 *              vacuum outside the box
 *   source     x = S*u, y = S*u, z = S*u, direction by Marsaglia's method,
 *              group 0, weight 1
 *   direction  Marsaglia (1972): repeat v1 = 2u-1, v2 = 2u-1, s = v1^2+v2^2
 *              until s < 1; then (2 v1 sqrt(1-s), 2 v2 sqrt(1-s), 1 - 2s)
 *   flight     d = -ln(1-u) * (1/Sigma_t[region]); the distance to the region
 *              surface along the ray is ds; d < ds collides, otherwise the
 *              particle moves to the surface and either leaks (box face) or
 *              changes region and samples a new flight
 *   collision  implicit capture w *= c[region]; group g' = first with
 *              u < CDF[region][g][g']; new direction; weight window of the
 *              region: w < w_low -> roulette (survive iff u < w/w_survive,
 *              then w = w_survive); w > w_high -> split into
 *              n = min(ceil(w/w_high), max_split) particles of weight w/n;
 *              the parent keeps one, child k = 0..n-2 starts with state
 *              hash(k, S_p) mod 2^m, S_p the parent's current state, and
 *              the parent's position, direction, group and region
 *   tally      track length of every segment clipped at every mesh plane;
 *              each piece adds llrint(w * length * 2^32) to the voxel holding
 *              its midpoint (group-summed [batch][mesh^3] int64 slots)
 * A particle is followed until it leaks or is killed by roulette (or reaches
 * the per-particle event cap); children are followed the same way.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "mc_oracle.h"

typedef struct {
    uint64_t x, draws;
    uint32_t m;
    uint64_t g, c;
} rng_t;

static double next_u(rng_t* r) {
    r->x = or_lcg_next(r->x, r->m, r->g, r->c);
    r->draws++;
    return or_u01(r->x, r->m);
}

typedef struct {
    double p[3], u[3], w;
    uint32_t g, region;
    uint64_t rng, draws;
    int primary;
} part_t;

static void iso_dir(rng_t* r, double u[3]) {
    double v1, v2, s;
    do {
        v1 = 2.0 * next_u(r) - 1.0;
        v2 = 2.0 * next_u(r) - 1.0;
        s = v1 * v1 + v2 * v2;
    } while (s >= 1.0);
    double t = sqrt(1.0 - s);
    u[0] = 2.0 * v1 * t;
    u[1] = 2.0 * v2 * t;
    u[2] = 1.0 - 2.0 * s;
}

/* Region of a point moving along u: inside the inner cube, with a point on
 * a face counted on the side it moves into. */
static uint32_t region_of(const or_box_problem* b, const double p[3], const double u[3]) {
    for (int a = 0; a < 3; ++a) {
        int above_lo = p[a] > b->inner_lo || (p[a] == b->inner_lo && u[a] > 0.0);
        int below_hi = p[a] < b->inner_hi || (p[a] == b->inner_hi && u[a] < 0.0);
        if (!above_lo || !below_hi) return 0;
    }
    return 1;
}

/* Distance to leave the cube [lo,hi]^3 from inside, along u (inv = 1/u). */
static double exit_dist(const double p[3], const double u[3], const double inv[3], double lo, double hi) {
    double t = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double ta;
        if (u[a] > 0.0)
            ta = (hi - p[a]) * inv[a];
        else if (u[a] < 0.0)
            ta = (lo - p[a]) * inv[a];
        else
            continue;
        if (ta < t) t = ta;
    }
    return t < 0.0 ? 0.0 : t;
}

/* Distance to enter the cube [lo,hi]^3 from outside; INFINITY on a miss. */
static double entry_dist(const double p[3], const double u[3], const double inv[3], double lo, double hi) {
    double tn = -INFINITY, tf = INFINITY;
    for (int a = 0; a < 3; ++a) {
        if (u[a] != 0.0) {
            double t1 = (lo - p[a]) * inv[a], t2 = (hi - p[a]) * inv[a];
            double tmin = t1 < t2 ? t1 : t2, tmax = t1 < t2 ? t2 : t1;
            if (tmin > tn) tn = tmin;
            if (tmax < tf) tf = tmax;
        } else if (p[a] <= lo || p[a] >= hi) {
            return INFINITY;
        }
    }
    if (tn >= 0.0 && tn < tf) return tn;
    return INFINITY;
}

static int cmp_d(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double plane_of(const or_box_problem* b, double h, uint32_t j) {
    return j >= b->mesh ? b->side : (double)j * h;
}

/* Track-length tally of the segment p + t u, 0 <= t <= L, weight w. */
static void trace(const or_box_problem* b, const double p[3], const double u[3], const double inv[3], double L,
                  double w, int64_t* t64, double* tfp) {
    const double h = b->side / (double)b->mesh;
    const uint32_t nm = b->mesh;
    double* ts = (double*)malloc(sizeof(double) * (3 * (nm + 1) + 2));
    int n = 0;
    ts[n++] = 0.0;
    for (int a = 0; a < 3; ++a) {
        if (u[a] == 0.0) continue;
        for (uint32_t j = 0; j <= nm; ++j) {
            double t = (plane_of(b, h, j) - p[a]) * inv[a];
            if (t > 0.0 && t < L) ts[n++] = t;
        }
    }
    ts[n++] = L;
    qsort(ts + 1, (size_t)(n - 2), sizeof(double), cmp_d);
    for (int k = 0; k + 1 < n; ++k) {
        double t0 = ts[k], t1 = ts[k + 1];
        if (!(t1 > t0)) continue;
        double mid = 0.5 * (t0 + t1);
        uint32_t idx[3];
        for (int a = 0; a < 3; ++a) {
            double c = p[a] + mid * u[a];
            double f = floor(c / h);
            int i = f < 0.0 ? 0 : (f >= (double)nm ? (int)nm - 1 : (int)f);
            idx[a] = (uint32_t)i;
        }
        uint64_t v = ((uint64_t)idx[2] * nm + idx[1]) * nm + idx[0];
        double len = t1 - t0;
        t64[v] += llrint(w * len * 4294967296.0);
        if (tfp) tfp[v] += w * len;
    }
    free(ts);
}

static void set_inv(const double u[3], double inv[3]) {
    for (int a = 0; a < 3; ++a) inv[a] = u[a] != 0.0 ? 1.0 / u[a] : 0.0;
}

typedef struct {
    part_t* a;
    size_t n, cap;
} stack_t_;

static void push(stack_t_* s, const part_t* p) {
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 64;
        s->a = (part_t*)realloc(s->a, s->cap * sizeof(part_t));
    }
    s->a[s->n++] = *p;
}

/* Follows one particle to its end; pushes the children of its splits. */
/* Downscatter: the first group g' >= g with u < CDF[region][g][g'] (R18). */
static uint32_t next_group(const or_box_problem* b, uint32_t rg, uint32_t g, double u) {
    for (uint32_t k = g; k < b->n_groups; ++k)
        if (u < b->cdf[rg][g][k]) return k;
    return g;
}

static int follow(const or_lcg* l, const or_box_problem* b, part_t* q, uint64_t event_cap, int64_t* t64,
                  double* tfp, uint64_t* cnt, stack_t_* st) {
    rng_t r = {q->rng, q->draws, l->m, l->g, l->c};
    double inv[3];
    set_inv(q->u, inv);
    int status = 0;
    for (uint64_t events = 0;; ++events) {
        if (events == event_cap) {
            cnt[OR_C_CAPPED]++;
            status = 1;
            break;
        }
        cnt[OR_C_FLIGHTS]++;
        double d = -log(1.0 - next_u(&r)) * (1.0 / b->sigma_t[q->region]);
        double ds;
        int kind; /* 1: into the other region, 2: leak */
        if (q->region == 1) {
            ds = exit_dist(q->p, q->u, inv, b->inner_lo, b->inner_hi);
            kind = 1;
        } else {
            double de = entry_dist(q->p, q->u, inv, b->inner_lo, b->inner_hi);
            double dx = exit_dist(q->p, q->u, inv, 0.0, b->side);
            if (de < dx) {
                ds = de;
                kind = 1;
            } else {
                ds = dx;
                kind = 2;
            }
        }
        if (d < ds) {
            trace(b, q->p, q->u, inv, d, q->w, t64, tfp);
            for (int a = 0; a < 3; ++a) q->p[a] = q->p[a] + d * q->u[a];
        } else {
            trace(b, q->p, q->u, inv, ds, q->w, t64, tfp);
            for (int a = 0; a < 3; ++a) q->p[a] = q->p[a] + ds * q->u[a];
            if (kind == 2) {
                cnt[OR_C_LEAK_HI]++;
                break;
            }
            q->region ^= 1u;
            continue;
        }
        /* collision */
        cnt[OR_C_COLLISIONS]++;
        const uint32_t rg = q->region;
        q->w = q->w * b->c[rg];
        q->g = next_group(b, rg, q->g, next_u(&r));
        iso_dir(&r, q->u);
        set_inv(q->u, inv);
        cnt[OR_C_SCATTERS]++;
        if (q->w < b->ww_low[rg]) {
            if (next_u(&r) < q->w / b->ww_survive[rg]) {
                q->w = b->ww_survive[rg];
            } else {
                cnt[OR_C_ROULETTE_KILLS]++;
                break;
            }
        } else if (q->w > b->ww_high[rg]) {
            double nd = ceil(q->w / b->ww_high[rg]);
            uint32_t ns = nd > (double)b->max_split ? b->max_split : (uint32_t)nd;
            if (ns > 1) {
                q->w = q->w / (double)ns;
                cnt[OR_C_SPLITS]++;
                for (uint32_t k = 0; k + 1 < ns; ++k) {
                    part_t c = *q;
                    c.rng = or_hash(k, r.x) & or_mask(l->m); /* Eq. (5) */
                    c.draws = 0;
                    c.primary = 0;
                    push(st, &c);
                    cnt[OR_C_CHILDREN]++;
                }
            }
        }
    }
    q->rng = r.x;
    q->draws = r.draws;
    return status;
}

uint64_t or_box_seed(const or_lcg* l, const or_box_problem* b, uint64_t id) {
    switch (b->seeding) {
    case OR_SEED_HASH:
        return or_hash_seed(id, b->seed, l->m);
    case OR_SEED_HASH_HIER:
        return or_hash_seed(id, or_hash(b->key, b->seed), l->m);
    default:
        return or_stride_seed(b->seed, b->stride_q, b->id_offset + id, l->m, l->g, l->c);
    }
}

int or_box_run(const or_lcg* l, const or_box_problem* b, uint64_t id_begin, uint64_t id_end, uint64_t event_cap,
               int64_t* tally, double* tally_fp, uint64_t* counts, uint64_t* hist_state, uint64_t* hist_draws) {
    int status = 0;
    const uint64_t nvox = (uint64_t)b->mesh * b->mesh * b->mesh;
    stack_t_ st = {NULL, 0, 0};
    for (uint64_t id = id_begin; id < id_end; ++id) {
        uint64_t batch = or_batch_of(id, b->n_histories, b->n_batches);
        int64_t* t64 = tally + b->tally_offset + batch * nvox;
        double* tfp = tally_fp ? tally_fp + b->tally_offset + batch * nvox : NULL;
        rng_t r = {or_box_seed(l, b, id), 0, l->m, l->g, l->c};
        part_t q;
        memset(&q, 0, sizeof q);
        for (int a = 0; a < 3; ++a) q.p[a] = b->side * next_u(&r);
        iso_dir(&r, q.u);
        q.w = 1.0;
        q.g = 0;
        q.region = region_of(b, q.p, q.u);
        q.rng = r.x;
        q.draws = r.draws;
        q.primary = 1;
        counts[OR_C_SOURCE]++;
        status |= follow(l, b, &q, event_cap, t64, tfp, counts, &st);
        counts[OR_C_DRAWS] += q.draws;
        if (q.draws > counts[OR_C_MAX_DRAWS]) counts[OR_C_MAX_DRAWS] = q.draws;
        if (b->stride_q != 0 && q.draws > b->stride_q) {
            counts[OR_C_EXCEED_HIST]++;
            counts[OR_C_EXCEED_DRAWS] += q.draws - b->stride_q;
        }
        if (hist_state) hist_state[id - id_begin] = q.rng;
        if (hist_draws) hist_draws[id - id_begin] = q.draws;
        while (st.n > 0) {
            part_t c = st.a[--st.n];
            status |= follow(l, b, &c, event_cap, t64, tfp, counts, &st);
            counts[OR_C_DRAWS] += c.draws;
            if (c.draws > counts[OR_C_MAX_DRAWS]) counts[OR_C_MAX_DRAWS] = c.draws;
        }
    }
    free(st.a);
    return status;
}

/* Test hooks: one isotropic direction from a state; the segment tally; the
 * downscatter group choice. */
uint32_t or_box_next_group(const or_box_problem* b, uint32_t region, uint32_t g, double u) {
    return next_group(b, region, g, u);
}

uint64_t or_box_iso_dir(const or_lcg* l, uint64_t x, double* u_out) {
    rng_t r = {x, 0, l->m, l->g, l->c};
    iso_dir(&r, u_out);
    return r.draws;
}

void or_box_trace(const or_box_problem* b, const double* p, const double* u, double L, double w, int64_t* t64,
                  double* tfp) {
    double inv[3];
    set_inv(u, inv);
    trace(b, p, u, inv, L, w, t64, tfp);
}

double or_box_surface_dist(const or_box_problem* b, const double* p, const double* u, uint32_t region,
                           int* kind_out) {
    double inv[3];
    set_inv(u, inv);
    if (region == 1) {
        *kind_out = 1;
        return exit_dist(p, u, inv, b->inner_lo, b->inner_hi);
    }
    double de = entry_dist(p, u, inv, b->inner_lo, b->inner_hi);
    double dx = exit_dist(p, u, inv, 0.0, b->side);
    *kind_out = de < dx ? 1 : 2;
    return de < dx ? de : dx;
}
