/*
 * CPU oracle for the VibeLSD decoding path (arXiv 2508.15743) -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded-per-shot C that follows the paper step by step: serial-V min-sum
 * BP (Appendix A, Algorithm 1), the ensemble of K permuted serial schedules with the correction
 * limit M and likelihood ranking (Sec. III.D.2, steps 3-4), the normalised LLR average (Sec. III.D.2,
 * step 5, displayed equation) and LSD post-processing (Sec. III.C; LSD-0 per Sec. III.D.1 step 5,
 * higher order as an OSD-E search inside each cluster).
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load this library. It
 * shares no code with the CUDA path. Readings where the paper is silent are stated at each function.
 */
#ifndef VIBE_ORACLE_H
#define VIBE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic modes of the oracle. */
enum { OR_FP32 = 0,      /* FP32 messages and arithmetic, fixed operation order */
       OR_FP16MSG = 1,   /* messages stored as IEEE binary16 (round to nearest even), FP32 arithmetic */
       OR_FP64 = 2 };    /* everything in double */

/* Per-shot statistics; same field meaning as the library's per-shot record. */
typedef struct {
  uint8_t status;          /* 0 ok, 1 unsolvable (syndrome outside the column span of H) */
  uint8_t lsd_invoked;     /* 1 if no member converged and LSD produced the correction */
  uint8_t n_converged;     /* size of the candidate set, min(M, members converged when BP stopped) */
  uint8_t chosen_member;   /* index of the member whose correction was chosen, 255 if LSD */
  uint16_t iters;          /* iteration at which the ensemble stopped (T if fewer than M converged) */
  uint16_t largest_cluster;/* error nodes (columns) in the largest LSD cluster, 0 if no LSD */
  uint32_t n_clusters;     /* number of final LSD clusters, 0 if no LSD */
} or_shot_stats;

typedef struct {
  int32_t m, n, k;                 /* detectors, mechanisms, logicals */
  const int32_t* rowptr;           /* H in CSR: rowptr[m+1], colidx[nnz], ascending per row */
  const int32_t* colidx;
  const int32_t* lrowptr;          /* L in CSR: lrowptr[k+1], lcolidx[...] */
  const int32_t* lcolidx;
  const double* priors;            /* p_j in (0, 0.5) */
} or_problem;

typedef struct {
  int32_t T;          /* max BP iterations per member */
  float alpha;        /* min-sum scaling factor */
  int32_t M;          /* correction limit */
  int32_t lsd_order;  /* 0 = LSD-0; > 0 = OSD-E search over that many free columns per cluster */
  int32_t mode;       /* OR_FP32, OR_FP16MSG or OR_FP64 */
  int32_t n_flood;    /* members 0 .. n_flood-1 use the parallel (flooding) schedule (R8), the rest
                         the serial one; their permutations are not used */
  const float* member_alpha;  /* NULL, or K factors: member i scales its check messages by
                                 member_alpha[i] instead of alpha (R9) */
  int32_t n_layered;  /* members n_flood .. n_flood+n_layered-1 use the layered schedule (R10);
                         n_flood + n_layered <= K */
} or_params;

/* Prior LLRs lambda_j = log((1 - p_j)/p_j) evaluated in double; lam32 gets the float rounding. */
void or_prior_llr(int32_t n, const double* priors, float* lam32, double* lam64);

/* One serial min-sum BP member (Algorithm 1, serial branch) on one syndrome.
 * syndrome: uint8[m] (0/1). perm: processing order, a permutation of 0..n-1.
 * Runs until H e = s (if early_stop) or T iterations. Outputs: posterior[n] (final L_v, as double),
 * ebits uint8[n]; returns the first iteration (1..T) whose decision satisfied H e = s, 0 if none. */
int32_t or_bp_member(const or_problem* P, const uint8_t* syndrome, const uint32_t* perm,
                     int32_t T, float alpha, int32_t mode, int32_t early_stop, double* posterior,
                     uint8_t* ebits);

/* One parallel (flooding) min-sum BP member (Algorithm 1, parallel branch; reading R8): same
 * inputs and outputs as or_bp_member without a permutation. */
int32_t or_bp_member_flood(const or_problem* P, const uint8_t* syndrome, int32_t T, float alpha, int32_t mode,
                           int32_t early_stop, double* posterior, uint8_t* ebits);

/* One layered min-sum BP member (R10): same inputs and outputs as or_bp_member_flood; *nlayer (if
 * not NULL) receives the number of check layers. */
int32_t or_bp_member_layered(const or_problem* P, const uint8_t* syndrome, int32_t T, float alpha, int32_t mode,
                             int32_t early_stop, double* posterior, uint8_t* ebits, int32_t* nlayer);

/* The check layers of R10: layer_of_check[m] receives each check's layer; returns the layer count. */
int32_t or_check_layers(const or_problem* P, int32_t* layer_of_check);

/* Full VibeLSD on B shots. syndromes: uint32[B][ceil(m/32)] bit-packed; perms uint32[K][n].
 * Outputs (any may be NULL except corrections): corrections uint32[B][ceil(n/32)],
 * logical uint32[B][ceil(k/32)], stats[B], soft double[B][n] (posterior of the chosen member, or the
 * averaged vector passed to LSD). nthreads >= 1 worker threads split the shots. Returns 0 or -1. */
int32_t or_decode(const or_problem* P, int32_t K, const uint32_t* perms, const or_params* prm,
                  int64_t B, const uint32_t* syndromes, uint32_t* corrections, uint32_t* logical,
                  or_shot_stats* stats, double* soft, int32_t nthreads);

/* LSD on one shot: soft[n] reliabilities (lower = more likely flipped), syndrome uint8[m].
 * lam: weights for the order-lambda search (float, or double in FP64 mode via lam64 != NULL).
 * Outputs ebits uint8[n], cluster_of_col int32[n] (final cluster root per column, -1 if none),
 * and the cluster statistics. Returns 0 ok, 1 unsolvable. */
int32_t or_lsd(const or_problem* P, const double* soft, const uint8_t* syndrome, int32_t order,
               const float* lam32, const double* lam64, uint8_t* ebits, int32_t* cluster_of_col,
               int32_t* n_clusters, int32_t* largest_cluster);

/* Seeded schedules: member i uses SplitMix64 started at seed + (i+1)*0xD1B54A32D192ED03 and a
 * Durstenfeld shuffle drawing j = high 64 bits of (next() * (k+1)) for k = n-1 down to 1. */
void or_seeded_schedules(int32_t n, int32_t K, uint64_t seed, uint32_t* perms);

#ifdef __cplusplus
}
#endif
#endif
