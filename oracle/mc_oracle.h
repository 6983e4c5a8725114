/*
 * mc_oracle.h -- declarations of the CPU oracle (test infrastructure only;
 * see mc_oracle.c).  Nothing in the CUDA library includes this header.
 */
#ifndef MC_ORACLE_H
#define MC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* LCG parameters of Eq. (1): X_{n+1} = (g X_n + c) mod 2^m. */
typedef struct {
    uint32_t m;
    uint32_t pad;
    uint64_t g;
    uint64_t c;
} or_lcg;

enum { OR_SEED_HASH = 0, OR_SEED_STRIDE = 1, OR_SEED_HASH_HIER = 2 };
enum { OR_SRC_ISOTROPIC = 0, OR_SRC_BEAM = 1 };

/* One slab problem.  seed: hash mode = global seed s; stride mode = X_0. */
typedef struct {
    double L, sigma_t, c;
    uint64_t n_histories;
    uint64_t seed;
    uint64_t stride_q;     /* stride Q; also the nominal stride for exceedance counts */
    uint64_t id_offset;    /* stride mode: unit index of local history 0 */
    uint64_t key;          /* hierarchical hash: key i of hash(j, hash(i, s)) */
    uint64_t tally_offset; /* first int64 slot of this problem's [batch][bin] tally */
    uint32_t n_bins, n_batches;
    uint32_t source, seeding;
} or_slab_problem;

/* Indices into a per-problem uint64 counter block of OR_NCOUNT entries. */
enum {
    OR_C_SOURCE = 0,
    OR_C_FLIGHTS,
    OR_C_COLLISIONS,
    OR_C_ABSORPTIONS,
    OR_C_SCATTERS,
    OR_C_LEAK_LO,
    OR_C_LEAK_HI,
    OR_C_DRAWS,
    OR_C_EXCEED_HIST,
    OR_C_EXCEED_DRAWS,
    OR_C_SPLITS,
    OR_C_ROULETTE_KILLS,
    OR_C_CAPPED,
    OR_C_MAX_DRAWS,
    OR_C_CHILDREN,
    OR_C_RESERVED,
    OR_C_BANKED, /* census phases: particles banked at an intermediate census */
    OR_NCOUNT
};

uint64_t or_mask(uint32_t m);
uint64_t or_lcg_next(uint64_t x, uint32_t m, uint64_t g, uint64_t c);
double or_u01(uint64_t x, uint32_t m);
uint64_t or_lcg_skip(uint64_t x0, uint64_t k, uint32_t m, uint64_t g, uint64_t c);
uint64_t or_stride_seed(uint64_t x0, uint64_t q, uint64_t k, uint32_t m, uint64_t g, uint64_t c);
uint64_t or_subhash(uint64_t x);
uint64_t or_hash(uint64_t k, uint64_t s);
uint64_t or_hash_seed(uint64_t k, uint64_t s, uint32_t m);
void or_seed_hash(uint32_t m, uint64_t parent, uint64_t key_begin, uint64_t count, uint64_t* out);
void or_seed_stride(uint32_t m, uint64_t g, uint64_t c, uint64_t x0, uint64_t q, uint64_t id_begin,
                    uint64_t count, uint64_t* out);
void or_lcg_draw(uint32_t m, uint64_t g, uint64_t c, uint64_t* states, uint64_t n, uint32_t draws,
                 double* u, uint64_t* digest);

uint64_t or_slab_seed(const or_lcg* l, const or_slab_problem* p, uint64_t id);
uint64_t or_batch_of(uint64_t id, uint64_t n_histories, uint32_t n_batches);
int or_slab_run(const or_lcg* l, const or_slab_problem* p, uint64_t id_begin, uint64_t id_end,
                uint64_t event_cap, int64_t* tally, double* tally_fp, uint64_t* counts,
                uint64_t* hist_state, uint64_t* hist_draws);

/* Two-region multigroup box with weight windows (mc_oracle_box.c). */
#define OR_BOX_MAX_GROUPS 8
typedef struct {
    double side, inner_lo, inner_hi;
    double sigma_t[2], c[2];                 /* region 0 = outer, 1 = inner */
    double ww_low[2], ww_high[2], ww_survive[2];
    double cdf[2][OR_BOX_MAX_GROUPS][OR_BOX_MAX_GROUPS]; /* [region][g][g'] */
    uint64_t n_histories, seed, stride_q, id_offset, key, tally_offset;
    uint32_t n_groups, mesh, max_split, n_batches;
    uint32_t seeding, source;
} or_box_problem;

uint64_t or_box_seed(const or_lcg* l, const or_box_problem* b, uint64_t id);
int or_box_run(const or_lcg* l, const or_box_problem* b, uint64_t id_begin, uint64_t id_end, uint64_t event_cap,
               int64_t* tally, double* tally_fp, uint64_t* counts, uint64_t* hist_state, uint64_t* hist_draws);
uint64_t or_box_iso_dir(const or_lcg* l, uint64_t x, double* u_out);
void or_box_trace(const or_box_problem* b, const double* p, const double* u, double L, double w, int64_t* t64,
                  double* tfp);
double or_box_surface_dist(const or_box_problem* b, const double* p, const double* u, uint32_t region,
                           int* kind_out);
uint32_t or_box_next_group(const or_box_problem* b, uint32_t region, uint32_t g, double u);

/* The paper's supercritical time-dependent problem (mc_oracle_azurv1.c). */
typedef struct {
    double c, nu, t_end, x_half, sigma_t;
    uint64_t seed, stride_q, id_offset, tally_offset;
    uint32_t n_reps, n_batches, per_batch, n_time_bins;
    uint32_t seeding;
    uint32_t n_census;  /* >= 2: census phases with population control (mc_oracle_census.c) */
    uint32_t pc_target; /* population per group after a control; 0 = per_batch */
    uint32_t pad;
} or_azurv1_problem;

uint64_t or_azurv1_seed(const or_lcg* l, const or_azurv1_problem* a, uint64_t g);
int or_azurv1_run(const or_lcg* l, const or_azurv1_problem* a, uint64_t g_begin, uint64_t g_end,
                  uint64_t event_cap, int64_t* tally, uint64_t* counts, uint64_t* hist_state,
                  uint64_t* hist_draws);

/* Census phases with population control by one-off hashed values
 * (mc_oracle_census.c); g_begin, g_end multiples of per_batch, hash seeding. */
int or_azurv1_census_run(const or_lcg* l, const or_azurv1_problem* a, uint64_t g_begin, uint64_t g_end,
                         uint64_t event_cap, int64_t* tally, uint64_t* counts, int reverse, uint64_t* pop,
                         double* wphase);

double or_norm_cdf(double z);
double or_norm_ppf(double p);
int or_shapiro_wilk(const double* x, int n, double* w, double* p);
int or_batch_stats(const double* x, uint32_t n_batches, uint32_t n_points, double* z, double* w,
                   double* p);

#ifdef __cplusplus
}
#endif
#endif
