/*
 * CPU oracle for the VibeLSD decoding path (arXiv 2508.15743) -- TEST INFRASTRUCTURE ONLY.
 *
 * Loaded by the tests, the smoke check and the benchmark's CPU-baseline leg; never by the library.
 * Shares no code with the CUDA path. Compile with -ffp-contract=off and without fast-math: every
 * float operation below is one IEEE operation in the order written.
 *
 * Readings of the paper used here (the paper is silent or ambiguous on each):
 *  R1 lambda_j = log((1-p_j)/p_j) in double, rounded once to float (FP32 modes).
 *  R2 The check update carries the syndrome: m_{c->v} = (-1)^{s_c} alpha prod sgn(.) min |.| over
 *     N(c)\v (Algorithm 1 prints it without s_c and without alpha; "syndrome-based decoding" needs
 *     the sign, and alpha is the min-sum scaling factor). sgn(x) = -1 iff x < 0.
 *  R3 Serial-V: for v in pi order, compute m_{c->v} for c in N(v) from the current m_{v'->c}, then
 *     L_v = lambda_v + sum_c m_{c->v} and m_{v->c} = lambda_v + sum_{c' != c} m_{c'->v}, both sums
 *     left folds in ascending check index (the literal formula of Algorithm 1).
 *  R4 e_v = 1 iff L_v <= 0; a member converges at the first iteration t whose e satisfies H e = s.
 *  R5 Members run in lock step; after iteration t, once M members have converged the rest stop.
 *     (Members 0 .. n_flood-1 may run the parallel schedule of R8; the rule is the same.)
 *     The candidates are the first min(M, #converged) members in (t, member) order; the chosen one
 *     minimises W(e) = sum_{e_j = 1} lambda_j (float left fold, ascending j), ties to the earlier.
 *  R2b A check of degree 1 has an empty N(c)\v: its minimum is +inf and its sign product +1, so it
 *     sends (-1)^{s_c} inf -- the exact hard constraint e_v = s_c. Posteriors may then be +-inf.
 *  R6 With no converged member the LSD input is (1/K) sum_i LLR^i / ||LLR^i||_2 (Sec. III.D.2
 *     step 5), the norm's sum of squares taken as 32 strided partial sums (entry j into partial
 *     j mod 32, ascending) combined pairwise at distances 16, 8, 4, 2, 1. Only finite entries enter
 *     the norm and get divided; an infinite entry (a hard constraint, R2b) is added as it is; a zero
 *     norm makes the finite entries' terms 0.
 *  R8 Parallel (flooding) schedule, the other branch of Algorithm 1: iteration t computes every
 *     m_{c->v} from the m_{v->c} of iteration t-1 (the priors at t = 1), with R2's rule, then every
 *     posterior L_v and every m_{v->c} from those m_{c->v}, with R3's sums in the same order. With
 *     FP16 storage the m_{v->c} are rounded to binary16 when stored; the m_{c->v} of an iteration
 *     are float temporaries.
 *  R10 Layered schedule (Sec. V names layered schedules, between serial and parallel, without
 *     defining one; this is row-layered min-sum). The checks are split into layers by greedy
 *     colouring in ascending check order: check c joins the smallest layer holding no earlier check
 *     that shares a variable with it, so no two checks of a layer share a variable. Each member keeps
 *     its m_{c->v} (zero before its first iteration) and its m_{v->c} (the priors). An iteration
 *     takes the layers in ascending order: every check of the layer computes its m_{c->v} from the
 *     current m_{v->c} with R2's rule, then every variable of those checks recomputes all its
 *     m_{v->c} from its current m_{c->v} with R3's exclusion sums, so later layers see the update.
 *     After the last layer L_v = lambda_v + sum_c m_{c->v} (R3's order). FP16 storage rounds the
 *     stored m_{v->c}; the m_{c->v} stay float.
 *  R9 Ensembles mixing heuristics (Sec. V names combining heuristics across the ensemble): a member
 *     may carry its own scaling factor alpha_i; the rest of Algorithm 1 and R5 are unchanged.
 *  R7 LSD (Sec. III.C): columns ranked by soft value ascending, ties by index; one cluster per flipped
 *     check; in each round every cluster whose syndrome is outside the span of its columns adds its
 *     best-ranked adjacent free column together with all that column's checks; clusters sharing a
 *     check merge. When all clusters are valid each is solved by OSD-0 on its submatrix with columns
 *     in rank order (free columns zero). Order > 0: search 2^q settings of the first q free columns
 *     (q = min(order, #free)) for the smallest W, ties to the lower setting index.
 */
#include "vibe_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------ */
/* Tanner graph: CSR edges (row-major) and, per column, its checks ascending with edge ids.     */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int m, n, E, maxcol;
  const int32_t* rowptr;
  const int32_t* colidx;
  int32_t* colptr;   /* n+1 */
  int32_t* col_chk;  /* E: check of the k-th edge of column v */
  int32_t* col_edge; /* E: CSR edge id of that edge */
  int32_t* edge_col; /* E: column of CSR edge e */
  int nlayer;        /* layers of the layered schedule (R10) */
  int32_t* layer_ptr; /* nlayer+1 */
  int32_t* layer_chk; /* m: checks of each layer, ascending */
} graph;

static void graph_build(graph* g, const or_problem* P) {
  g->m = P->m; g->n = P->n; g->rowptr = P->rowptr; g->colidx = P->colidx;
  g->E = P->rowptr[P->m];
  g->colptr = (int32_t*)calloc((size_t)g->n + 1, sizeof(int32_t));
  g->col_chk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->E + 1));
  g->col_edge = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->E + 1));
  g->edge_col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->E + 1));
  for (int e = 0; e < g->E; ++e) g->colptr[g->colidx[e] + 1]++;
  for (int v = 0; v < g->n; ++v) g->colptr[v + 1] += g->colptr[v];
  int32_t* fill = (int32_t*)calloc((size_t)g->n, sizeof(int32_t));
  for (int c = 0; c < g->m; ++c)
    for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
      int v = g->colidx[e];
      int pos = g->colptr[v] + fill[v]++;
      g->col_chk[pos] = c;      /* rows are scanned ascending, so checks land ascending */
      g->col_edge[pos] = e;
      g->edge_col[e] = v;
    }
  free(fill);
  g->maxcol = 0;
  for (int v = 0; v < g->n; ++v)
    if (g->colptr[v + 1] - g->colptr[v] > g->maxcol) g->maxcol = g->colptr[v + 1] - g->colptr[v];
  /* layers (R10): smallest layer not taken by an earlier check sharing a variable with c */
  int32_t* layer_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
  uint8_t* taken = (uint8_t*)calloc((size_t)g->m + 1, 1);
  g->nlayer = 0;
  for (int c = 0; c < g->m; ++c) {
    for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
      int v = g->colidx[e];
      for (int k = g->colptr[v]; k < g->colptr[v + 1] && g->col_chk[k] < c; ++k) taken[layer_of[g->col_chk[k]]] = 1;
    }
    int l = 0;
    while (taken[l]) ++l;
    layer_of[c] = l;
    if (l + 1 > g->nlayer) g->nlayer = l + 1;
    for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
      int v = g->colidx[e];
      for (int k = g->colptr[v]; k < g->colptr[v + 1] && g->col_chk[k] < c; ++k) taken[layer_of[g->col_chk[k]]] = 0;
    }
  }
  g->layer_ptr = (int32_t*)calloc((size_t)g->nlayer + 2, sizeof(int32_t));
  g->layer_chk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->m + 1));
  for (int c = 0; c < g->m; ++c) g->layer_ptr[layer_of[c] + 1]++;
  for (int l = 0; l < g->nlayer; ++l) g->layer_ptr[l + 1] += g->layer_ptr[l];
  int32_t* at = (int32_t*)calloc((size_t)g->nlayer + 1, sizeof(int32_t));
  for (int c = 0; c < g->m; ++c) g->layer_chk[g->layer_ptr[layer_of[c]] + at[layer_of[c]]++] = c;
  free(at); free(taken); free(layer_of);
}

static void graph_free(graph* g) {
  free(g->colptr); free(g->col_chk); free(g->col_edge); free(g->edge_col); free(g->layer_ptr); free(g->layer_chk);
}

void or_prior_llr(int32_t n, const double* priors, float* lam32, double* lam64) {
  for (int j = 0; j < n; ++j) {
    double l = log((1.0 - priors[j]) / priors[j]);
    if (lam64) lam64[j] = l;
    if (lam32) lam32[j] = (float)l;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* One serial sweep of Algorithm 1 (R2, R3), float arithmetic. fp16 != 0 rounds every stored   */
/* variable-to-check message to binary16.                                                       */
/* ------------------------------------------------------------------------------------------ */
static float store_msg(float a, int fp16) { return fp16 ? (float)(_Float16)a : a; }

static void sweep_f32(const graph* g, const uint32_t* perm, const uint8_t* s, const float* lam,
                      float alpha, int fp16, float* msg, float* post, float* mcv) {
  for (int idx = 0; idx < g->n; ++idx) {
    int v = (int)perm[idx];
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    for (int k = 0; k < deg; ++k) {         /* check-to-variable messages for c in N(v) */
      int c = g->col_chk[b + k], own = g->col_edge[b + k];
      int neg = s[c];
      float mn = INFINITY;
      for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
        if (e == own) continue;
        float x = msg[e];
        if (x < 0.0f) neg ^= 1;
        float ax = fabsf(x);
        if (ax < mn) mn = ax;
      }
      float mag = alpha * mn;
      mcv[k] = neg ? -mag : mag;
    }
    float L = lam[v];                       /* posterior */
    for (int k = 0; k < deg; ++k) L = L + mcv[k];
    for (int k = 0; k < deg; ++k) {         /* variable-to-check messages, literal exclusion sums */
      float a = lam[v];
      for (int k2 = 0; k2 < deg; ++k2)
        if (k2 != k) a = a + mcv[k2];
      msg[g->col_edge[b + k]] = store_msg(a, fp16);
    }
    post[v] = L;
  }
}

static void sweep_f64(const graph* g, const uint32_t* perm, const uint8_t* s, const double* lam,
                      double alpha, double* msg, double* post, double* mcv) {
  for (int idx = 0; idx < g->n; ++idx) {
    int v = (int)perm[idx];
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    for (int k = 0; k < deg; ++k) {
      int c = g->col_chk[b + k], own = g->col_edge[b + k];
      int neg = s[c];
      double mn = INFINITY;
      for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
        if (e == own) continue;
        double x = msg[e];
        if (x < 0.0) neg ^= 1;
        double ax = fabs(x);
        if (ax < mn) mn = ax;
      }
      double mag = alpha * mn;
      mcv[k] = neg ? -mag : mag;
    }
    double L = lam[v];
    for (int k = 0; k < deg; ++k) L = L + mcv[k];
    for (int k = 0; k < deg; ++k) {
      double a = lam[v];
      for (int k2 = 0; k2 < deg; ++k2)
        if (k2 != k) a = a + mcv[k2];
      msg[g->col_edge[b + k]] = a;
    }
    post[v] = L;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* One parallel (flooding) iteration of Algorithm 1 (R2, R8). c2v: E temporaries (CSR order).  */
/* ------------------------------------------------------------------------------------------ */
static void flood_f32(const graph* g, const uint8_t* s, const float* lam, float alpha, int fp16, float* msg,
                      float* c2v, float* post) {
  for (int c = 0; c < g->m; ++c)            /* every check-to-variable message, old messages only */
    for (int own = g->rowptr[c]; own < g->rowptr[c + 1]; ++own) {
      int neg = s[c];
      float mn = INFINITY;
      for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
        if (e == own) continue;
        float x = msg[e];
        if (x < 0.0f) neg ^= 1;
        float ax = fabsf(x);
        if (ax < mn) mn = ax;
      }
      float mag = alpha * mn;
      c2v[own] = neg ? -mag : mag;
    }
  for (int v = 0; v < g->n; ++v) {          /* every posterior and variable-to-check message */
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    float L = lam[v];
    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];
    for (int k = 0; k < deg; ++k) {
      float a = lam[v];
      for (int k2 = 0; k2 < deg; ++k2)
        if (k2 != k) a = a + c2v[g->col_edge[b + k2]];
      msg[g->col_edge[b + k]] = store_msg(a, fp16);
    }
    post[v] = L;
  }
}

static void flood_f64(const graph* g, const uint8_t* s, const double* lam, double alpha, double* msg,
                      double* c2v, double* post) {
  for (int c = 0; c < g->m; ++c)
    for (int own = g->rowptr[c]; own < g->rowptr[c + 1]; ++own) {
      int neg = s[c];
      double mn = INFINITY;
      for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
        if (e == own) continue;
        double x = msg[e];
        if (x < 0.0) neg ^= 1;
        double ax = fabs(x);
        if (ax < mn) mn = ax;
      }
      double mag = alpha * mn;
      c2v[own] = neg ? -mag : mag;
    }
  for (int v = 0; v < g->n; ++v) {
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    double L = lam[v];
    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];
    for (int k = 0; k < deg; ++k) {
      double a = lam[v];
      for (int k2 = 0; k2 < deg; ++k2)
        if (k2 != k) a = a + c2v[g->col_edge[b + k2]];
      msg[g->col_edge[b + k]] = a;
    }
    post[v] = L;
  }
}

/* ------------------------------------------------------------------------------------------ */
/* One layered iteration (R2, R3, R10). c2v: the member's E check-to-variable messages (CSR     */
/* order), kept between iterations.                                                             */
/* ------------------------------------------------------------------------------------------ */
static void layered_f32(const graph* g, const uint8_t* s, const float* lam, float alpha, int fp16, float* msg,
                        float* c2v, float* post) {
  for (int l = 0; l < g->nlayer; ++l) {
    for (int q = g->layer_ptr[l]; q < g->layer_ptr[l + 1]; ++q) {   /* the layer's checks */
      int c = g->layer_chk[q];
      for (int own = g->rowptr[c]; own < g->rowptr[c + 1]; ++own) {
        int neg = s[c];
        float mn = INFINITY;
        for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
          if (e == own) continue;
          float x = msg[e];
          if (x < 0.0f) neg ^= 1;
          float ax = fabsf(x);
          if (ax < mn) mn = ax;
        }
        float mag = alpha * mn;
        c2v[own] = neg ? -mag : mag;
      }
    }
    for (int q = g->layer_ptr[l]; q < g->layer_ptr[l + 1]; ++q) {   /* their variables */
      int c = g->layer_chk[q];
      for (int ce = g->rowptr[c]; ce < g->rowptr[c + 1]; ++ce) {
        int v = g->edge_col[ce];
        int b = g->colptr[v], deg = g->colptr[v + 1] - b;
        for (int k = 0; k < deg; ++k) {
          float a = lam[v];
          for (int k2 = 0; k2 < deg; ++k2)
            if (k2 != k) a = a + c2v[g->col_edge[b + k2]];
          msg[g->col_edge[b + k]] = store_msg(a, fp16);
        }
      }
    }
  }
  for (int v = 0; v < g->n; ++v) {
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    float L = lam[v];
    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];
    post[v] = L;
  }
}

static void layered_f64(const graph* g, const uint8_t* s, const double* lam, double alpha, double* msg,
                        double* c2v, double* post) {
  for (int l = 0; l < g->nlayer; ++l) {
    for (int q = g->layer_ptr[l]; q < g->layer_ptr[l + 1]; ++q) {
      int c = g->layer_chk[q];
      for (int own = g->rowptr[c]; own < g->rowptr[c + 1]; ++own) {
        int neg = s[c];
        double mn = INFINITY;
        for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
          if (e == own) continue;
          double x = msg[e];
          if (x < 0.0) neg ^= 1;
          double ax = fabs(x);
          if (ax < mn) mn = ax;
        }
        double mag = alpha * mn;
        c2v[own] = neg ? -mag : mag;
      }
    }
    for (int q = g->layer_ptr[l]; q < g->layer_ptr[l + 1]; ++q) {
      int c = g->layer_chk[q];
      for (int ce = g->rowptr[c]; ce < g->rowptr[c + 1]; ++ce) {
        int v = g->edge_col[ce];
        int b = g->colptr[v], deg = g->colptr[v + 1] - b;
        for (int k = 0; k < deg; ++k) {
          double a = lam[v];
          for (int k2 = 0; k2 < deg; ++k2)
            if (k2 != k) a = a + c2v[g->col_edge[b + k2]];
          msg[g->col_edge[b + k]] = a;
        }
      }
    }
  }
  for (int v = 0; v < g->n; ++v) {
    int b = g->colptr[v], deg = g->colptr[v + 1] - b;
    double L = lam[v];
    for (int k = 0; k < deg; ++k) L = L + c2v[g->col_edge[b + k]];
    post[v] = L;
  }
}

/* H e = s with e_v = [L_v <= 0] (R4). */
static int satisfies_f32(const graph* g, const uint8_t* s, const float* post) {
  for (int c = 0; c < g->m; ++c) {
    int par = s[c];
    for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) par ^= (post[g->colidx[e]] <= 0.0f);
    if (par) return 0;
  }
  return 1;
}

static int satisfies_f64(const graph* g, const uint8_t* s, const double* post) {
  for (int c = 0; c < g->m; ++c) {
    int par = s[c];
    for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) par ^= (post[g->colidx[e]] <= 0.0);
    if (par) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Per-thread workspace                                                                         */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const or_problem* P;
  graph g;
  int K, mode;
  float* lam32; double* lam64;
  float* msg32; double* msg64;     /* K * E */
  float* post32; double* post64;   /* K * n */
  float* mcv32; double* mcv64;     /* maxcol */
  float* c2v32; double* c2v64;     /* E: check-to-variable temporaries of a flooding iteration */
  float* lc2v32; double* lc2v64;   /* K * E: layered members' check-to-variable messages (R10), on demand */
  int32_t* conv_t;                 /* K */
  uint8_t* s;                      /* m */
  uint8_t* ebits;                  /* n */
  double* soft;                    /* n */
  /* LSD scratch */
  int32_t* ck_par;                 /* m: union-find parent, -1 = not in a cluster */
  int32_t* col_root;               /* n */
  int32_t* roots; int32_t* picks;  /* m, 2m */
  int32_t* cl_checks; int32_t* cl_cols; int32_t* tmp; /* m, n, n */
  uint8_t* mat;                    /* dense submatrix, grown on demand */
  size_t mat_cap;
  int32_t* pivrow;                 /* n */
  uint8_t* x; uint8_t* xbest;      /* n */
  int32_t* asc;                    /* n: cluster columns by ascending index */
} workspace;

static void ws_init(workspace* w, const or_problem* P, int K, int mode) {
  memset(w, 0, sizeof(*w));
  w->P = P; w->K = K; w->mode = mode;
  graph_build(&w->g, P);
  int n = P->n, m = P->m, E = w->g.E;
  w->lam32 = (float*)malloc(sizeof(float) * (size_t)n);
  w->lam64 = (double*)malloc(sizeof(double) * (size_t)n);
  or_prior_llr(n, P->priors, w->lam32, w->lam64);
  size_t ke = (size_t)K * (size_t)(E > 0 ? E : 1), kn = (size_t)K * (size_t)n;
  if (mode == OR_FP64) {
    w->msg64 = (double*)malloc(sizeof(double) * ke);
    w->post64 = (double*)malloc(sizeof(double) * kn);
  } else {
    w->msg32 = (float*)malloc(sizeof(float) * ke);
    w->post32 = (float*)malloc(sizeof(float) * kn);
  }
  w->mcv32 = (float*)malloc(sizeof(float) * (size_t)(w->g.maxcol + 1));
  w->mcv64 = (double*)malloc(sizeof(double) * (size_t)(w->g.maxcol + 1));
  w->c2v32 = (float*)malloc(sizeof(float) * (size_t)(w->g.E + 1));
  w->c2v64 = (double*)malloc(sizeof(double) * (size_t)(w->g.E + 1));
  w->conv_t = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  w->s = (uint8_t*)malloc((size_t)m + 1);
  w->ebits = (uint8_t*)malloc((size_t)n + 1);
  w->soft = (double*)malloc(sizeof(double) * (size_t)(n + 1));
  w->ck_par = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  w->col_root = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  w->roots = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  w->picks = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * m + 2));
  w->cl_checks = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
  w->cl_cols = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  w->tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  w->pivrow = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
  w->x = (uint8_t*)malloc((size_t)n + 1);
  w->xbest = (uint8_t*)malloc((size_t)n + 1);
  w->asc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n + 1));
}

static void ws_free(workspace* w) {
  graph_free(&w->g);
  free(w->lam32); free(w->lam64); free(w->msg32); free(w->msg64); free(w->post32); free(w->post64);
  free(w->mcv32); free(w->mcv64); free(w->c2v32); free(w->c2v64); free(w->lc2v32); free(w->lc2v64); free(w->conv_t); free(w->s); free(w->ebits); free(w->soft);
  free(w->ck_par); free(w->col_root); free(w->roots); free(w->picks); free(w->cl_checks);
  free(w->cl_cols); free(w->tmp); free(w->mat); free(w->pivrow); free(w->x); free(w->xbest); free(w->asc);
}

/* ------------------------------------------------------------------------------------------ */
/* Dense GF(2) elimination (used for cluster validity and the OSD solve inside each cluster)    */
/* ------------------------------------------------------------------------------------------ */
/* A is rows x (cols+1), row-major, last column the right-hand side. Columns are eliminated in the
 * given order to reduced row echelon form; pivrow[c] = pivot row of column c or -1 (free).
 * Returns 1 if the system is consistent. */
static int gf2_rref(uint8_t* A, int rows, int cols, int32_t* pivrow) {
  int w = cols + 1, r = 0;
  for (int c = 0; c < cols; ++c) {
    pivrow[c] = -1;
    if (r == rows) continue;
    int p = -1;
    for (int i = r; i < rows; ++i)
      if (A[i * w + c]) { p = i; break; }
    if (p < 0) continue;
    if (p != r)
      for (int t = 0; t < w; ++t) { uint8_t tt = A[p * w + t]; A[p * w + t] = A[r * w + t]; A[r * w + t] = tt; }
    for (int i = 0; i < rows; ++i)
      if (i != r && A[i * w + c])
        for (int t = 0; t < w; ++t) A[i * w + t] ^= A[r * w + t];
    pivrow[c] = r++;
  }
  for (int i = r; i < rows; ++i)
    if (A[i * w + cols]) return 0;
  return 1;
}

static int uf_find(int32_t* par, int x) {
  while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
  return x;
}

static void uf_union(int32_t* par, int a, int b) {
  a = uf_find(par, a); b = uf_find(par, b);
  if (a == b) return;
  if (a < b) par[b] = a; else par[a] = b;
}

/* soft-value rank order: a before b iff soft[a] < soft[b], or equal and a < b (R7) */
static int ranks_before(const double* soft, int a, int b) {
  return soft[a] < soft[b] || (soft[a] == soft[b] && a < b);
}

/* Collect the checks (ascending) and the columns (in rank order) of the cluster rooted at r. */
static void cluster_members(workspace* w, const double* soft, int r, int* nck, int* ncol) {
  const graph* g = &w->g;
  int a = 0, b = 0;
  for (int c = 0; c < g->m; ++c)
    if (w->ck_par[c] >= 0 && uf_find(w->ck_par, c) == r) w->cl_checks[a++] = c;
  for (int j = 0; j < g->n; ++j)
    if (w->col_root[j] >= 0 && uf_find(w->ck_par, w->col_root[j]) == r) w->cl_cols[b++] = j;
  /* insertion sort of the columns by rank */
  for (int i = 1; i < b; ++i) {
    int v = w->cl_cols[i], t = i - 1;
    while (t >= 0 && ranks_before(soft, v, w->cl_cols[t])) { w->cl_cols[t + 1] = w->cl_cols[t]; --t; }
    w->cl_cols[t + 1] = v;
  }
  *nck = a; *ncol = b;
}

/* Dense [H_C | s_C] for the current cluster lists; returns its row width. */
static int cluster_matrix(workspace* w, const uint8_t* s, int nck, int ncol) {
  const graph* g = &w->g;
  int wd = ncol + 1;
  size_t need = (size_t)(nck > 0 ? nck : 1) * (size_t)wd;
  if (need > w->mat_cap) { free(w->mat); w->mat = (uint8_t*)malloc(need); w->mat_cap = need; }
  memset(w->mat, 0, need);
  for (int i = 0; i < nck; ++i) {
    int c = w->cl_checks[i];
    for (int t = 0; t < ncol; ++t) {
      int j = w->cl_cols[t];
      for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e)
        if (g->colidx[e] == j) { w->mat[i * wd + t] = 1; break; }
    }
    w->mat[i * wd + ncol] = s[c];
  }
  return wd;
}

static int lsd_core(workspace* w, const double* soft, const uint8_t* s, int order, uint8_t* ebits,
                    int32_t* cluster_of_col, int32_t* n_clusters, int32_t* largest) {
  const graph* g = &w->g;
  int m = g->m, n = g->n;
  for (int c = 0; c < m; ++c) w->ck_par[c] = s[c] ? c : -1;   /* one cluster per flipped check */
  for (int j = 0; j < n; ++j) { w->col_root[j] = -1; ebits[j] = 0; }
  int status = 0;
  for (int round = 0; round <= n + 1; ++round) {
    int nroots = 0;
    for (int c = 0; c < m; ++c)
      if (w->ck_par[c] >= 0 && uf_find(w->ck_par, c) == c) w->roots[nroots++] = c;
    int npick = 0;
    for (int q = 0; q < nroots; ++q) {
      int r = w->roots[q], nck, ncol;
      cluster_members(w, soft, r, &nck, &ncol);
      cluster_matrix(w, s, nck, ncol);
      if (gf2_rref(w->mat, nck, ncol, w->pivrow)) continue;       /* valid */
      int best = -1;                                             /* best free adjacent column */
      for (int i = 0; i < nck; ++i) {
        int c = w->cl_checks[i];
        for (int e = g->rowptr[c]; e < g->rowptr[c + 1]; ++e) {
          int j = g->colidx[e];
          if (w->col_root[j] < 0 && (best < 0 || ranks_before(soft, j, best))) best = j;
        }
      }
      if (best < 0) { status = 1; break; }                        /* whole component, still invalid */
      w->picks[2 * npick] = r; w->picks[2 * npick + 1] = best; ++npick;
    }
    if (status) break;
    if (npick == 0) break;                                        /* every cluster valid */
    for (int q = 0; q < npick; ++q) {
      int r = w->picks[2 * q], j = w->picks[2 * q + 1];
      int rr = uf_find(w->ck_par, r);
      for (int t = g->colptr[j]; t < g->colptr[j + 1]; ++t) {
        int c = g->col_chk[t];
        if (w->ck_par[c] < 0) w->ck_par[c] = rr;
        else uf_union(w->ck_par, rr, c);
        rr = uf_find(w->ck_par, rr);
      }
      w->col_root[j] = rr;
    }
  }
  /* final clusters: solve each (OSD-0, then the optional search) */
  int nroots = 0, big = 0;
  for (int c = 0; c < m; ++c)
    if (w->ck_par[c] >= 0 && uf_find(w->ck_par, c) == c) w->roots[nroots++] = c;
  if (status == 0) {
    for (int q = 0; q < nroots; ++q) {
      int r = w->roots[q], nck, ncol;
      cluster_members(w, soft, r, &nck, &ncol);
      if (ncol > big) big = ncol;
      int wd = cluster_matrix(w, s, nck, ncol);
      gf2_rref(w->mat, nck, ncol, w->pivrow);
      /* free columns in rank order */
      int nfree = 0;
      for (int t = 0; t < ncol; ++t)
        if (w->pivrow[t] < 0) w->tmp[nfree++] = t;
      int qn = order < nfree ? order : nfree;
      /* columns of the cluster in ascending index, for the weight sum */
      int32_t* asc = w->asc;
      for (int t = 0; t < ncol; ++t) asc[t] = t;
      for (int i = 1; i < ncol; ++i) {
        int v = asc[i], t = i - 1;
        while (t >= 0 && w->cl_cols[asc[t]] > w->cl_cols[v]) { asc[t + 1] = asc[t]; --t; }
        asc[t + 1] = v;
      }
      double bestW = INFINITY;
      for (long a = 0; a < (1L << qn); ++a) {
        memset(w->x, 0, (size_t)ncol);
        for (int b = 0; b < qn; ++b) w->x[w->tmp[b]] = (uint8_t)((a >> b) & 1);
        for (int t = 0; t < ncol; ++t) {
          int pr = w->pivrow[t];
          if (pr < 0) continue;
          int val = w->mat[pr * wd + ncol];
          for (int b = 0; b < qn; ++b) val ^= w->mat[pr * wd + w->tmp[b]] & w->x[w->tmp[b]];
          w->x[t] = (uint8_t)val;
        }
        double W;
        if (w->mode == OR_FP64) {
          double acc = 0.0;
          for (int i = 0; i < ncol; ++i) if (w->x[asc[i]]) acc = acc + w->lam64[w->cl_cols[asc[i]]];
          W = acc;
        } else {
          float acc = 0.0f;
          for (int i = 0; i < ncol; ++i) if (w->x[asc[i]]) acc = acc + w->lam32[w->cl_cols[asc[i]]];
          W = (double)acc;
        }
        if (a == 0 || W < bestW) { bestW = W; memcpy(w->xbest, w->x, (size_t)ncol); }
      }
      for (int t = 0; t < ncol; ++t) ebits[w->cl_cols[t]] = w->xbest[t];
    }
  } else {
    for (int q = 0; q < nroots; ++q) {
      int nck, ncol;
      cluster_members(w, soft, w->roots[q], &nck, &ncol);
      if (ncol > big) big = ncol;
    }
  }
  if (cluster_of_col)
    for (int j = 0; j < n; ++j) cluster_of_col[j] = w->col_root[j] < 0 ? -1 : uf_find(w->ck_par, w->col_root[j]);
  *n_clusters = nroots;
  *largest = big;
  return status;
}

/* ------------------------------------------------------------------------------------------ */
/* Full decoder, one shot                                                                       */
/* ------------------------------------------------------------------------------------------ */
static void init_member(workspace* w, int i) {
  const graph* g = &w->g;
  if (w->mode == OR_FP64) {
    double* msg = w->msg64 + (size_t)i * g->E;
    for (int e = 0; e < g->E; ++e) msg[e] = w->lam64[g->edge_col[e]];
    if (w->lc2v64) memset(w->lc2v64 + (size_t)i * g->E, 0, sizeof(double) * (size_t)g->E);
  } else {
    float* msg = w->msg32 + (size_t)i * g->E;
    for (int e = 0; e < g->E; ++e) msg[e] = store_msg(w->lam32[g->edge_col[e]], w->mode == OR_FP16MSG);
    if (w->lc2v32) memset(w->lc2v32 + (size_t)i * g->E, 0, sizeof(float) * (size_t)g->E);
  }
}

/* Storage for the layered members' check-to-variable messages (all K, zeroed by init_member). */
static void ws_layered(workspace* w) {
  size_t ke = (size_t)w->K * (size_t)(w->g.E > 0 ? w->g.E : 1);
  if (w->mode == OR_FP64) w->lc2v64 = (double*)calloc(ke, sizeof(double));
  else w->lc2v32 = (float*)calloc(ke, sizeof(float));
}

static void decode_one(workspace* w, const uint32_t* perms, const or_params* prm, const uint32_t* syn,
                       uint32_t* corr, uint32_t* logi, or_shot_stats* st, double* soft_out) {
  const graph* g = &w->g;
  const or_problem* P = w->P;
  int m = g->m, n = g->n, K = w->K, T = prm->T, M = prm->M;
  int fp64 = w->mode == OR_FP64, fp16 = w->mode == OR_FP16MSG;
  for (int c = 0; c < m; ++c) w->s[c] = (uint8_t)((syn[c >> 5] >> (c & 31)) & 1u);
  for (int i = 0; i < K; ++i) { init_member(w, i); w->conv_t[i] = 0; }
  int nconv = 0, t_stop = T;
  for (int t = 1; t <= T; ++t) {
    for (int i = 0; i < K; ++i) {
      if (w->conv_t[i]) continue;
      const uint32_t* perm = perms + (size_t)i * n;
      const float alpha = prm->member_alpha ? prm->member_alpha[i] : prm->alpha;
      int ok;
      const int layered = i >= prm->n_flood && i < prm->n_flood + prm->n_layered;
      if (fp64) {
        if (i < prm->n_flood)
          flood_f64(g, w->s, w->lam64, (double)alpha, w->msg64 + (size_t)i * g->E, w->c2v64,
                    w->post64 + (size_t)i * n);
        else if (layered)
          layered_f64(g, w->s, w->lam64, (double)alpha, w->msg64 + (size_t)i * g->E, w->lc2v64 + (size_t)i * g->E,
                      w->post64 + (size_t)i * n);
        else
          sweep_f64(g, perm, w->s, w->lam64, (double)alpha, w->msg64 + (size_t)i * g->E,
                    w->post64 + (size_t)i * n, w->mcv64);
        ok = satisfies_f64(g, w->s, w->post64 + (size_t)i * n);
      } else {
        if (i < prm->n_flood)
          flood_f32(g, w->s, w->lam32, alpha, fp16, w->msg32 + (size_t)i * g->E, w->c2v32,
                    w->post32 + (size_t)i * n);
        else if (layered)
          layered_f32(g, w->s, w->lam32, alpha, fp16, w->msg32 + (size_t)i * g->E, w->lc2v32 + (size_t)i * g->E,
                      w->post32 + (size_t)i * n);
        else
          sweep_f32(g, perm, w->s, w->lam32, alpha, fp16, w->msg32 + (size_t)i * g->E,
                    w->post32 + (size_t)i * n, w->mcv32);
        ok = satisfies_f32(g, w->s, w->post32 + (size_t)i * n);
      }
      if (ok) { w->conv_t[i] = t; ++nconv; }
    }
    if (nconv >= M) { t_stop = t; break; }
  }
  memset(st, 0, sizeof(*st));
  st->iters = (uint16_t)t_stop;
  /* candidate set: first min(M, nconv) converged members in (t, member) order (R5) */
  int ncand = nconv < M ? nconv : M, chosen = -1;
  double bestW = INFINITY;
  for (int t = 1, taken = 0; t <= t_stop && taken < ncand; ++t)
    for (int i = 0; i < K && taken < ncand; ++i) {
      if (w->conv_t[i] != t) continue;
      ++taken;
      double W;
      if (fp64) {
        const double* post = w->post64 + (size_t)i * n;
        double acc = 0.0;
        for (int j = 0; j < n; ++j) if (post[j] <= 0.0) acc = acc + w->lam64[j];
        W = acc;
      } else {
        const float* post = w->post32 + (size_t)i * n;
        float acc = 0.0f;
        for (int j = 0; j < n; ++j) if (post[j] <= 0.0f) acc = acc + w->lam32[j];
        W = (double)acc;
      }
      if (chosen < 0 || W < bestW) { bestW = W; chosen = i; }
    }
  st->n_converged = (uint8_t)ncand;
  if (chosen >= 0) {
    st->chosen_member = (uint8_t)chosen;
    for (int j = 0; j < n; ++j) {
      double L = fp64 ? w->post64[(size_t)chosen * n + j] : (double)w->post32[(size_t)chosen * n + j];
      w->ebits[j] = (uint8_t)(L <= 0.0);
      w->soft[j] = L;
    }
  } else {
    /* normalised LLR average over all K members (R6) */
    st->chosen_member = 255;
    st->lsd_invoked = 1;
    if (fp64) {
      for (int j = 0; j < n; ++j) w->soft[j] = 0.0;
      for (int i = 0; i < K; ++i) {
        const double* post = w->post64 + (size_t)i * n;
        double part[32];
        for (int l = 0; l < 32; ++l) {
          part[l] = 0.0;
          for (int j = l; j < n; j += 32) part[l] = part[l] + (isfinite(post[j]) ? post[j] * post[j] : 0.0);
        }
        for (int off = 16; off >= 1; off >>= 1) {
          double nxt[32];
          for (int l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
          memcpy(part, nxt, sizeof(part));
        }
        double nrm = sqrt(part[0]);
        for (int j = 0; j < n; ++j)
          w->soft[j] = w->soft[j] + (!isfinite(post[j]) ? post[j] : (nrm == 0.0 ? 0.0 : post[j] / nrm));
      }
      for (int j = 0; j < n; ++j) w->soft[j] = w->soft[j] / (double)K;
    } else {
      float* acc = (float*)w->tmp;   /* n floats of scratch */
      for (int j = 0; j < n; ++j) acc[j] = 0.0f;
      for (int i = 0; i < K; ++i) {
        const float* post = w->post32 + (size_t)i * n;
        float part[32];
        for (int l = 0; l < 32; ++l) {
          part[l] = 0.0f;
          for (int j = l; j < n; j += 32) {
            float sq = isfinite(post[j]) ? post[j] * post[j] : 0.0f;
            part[l] = part[l] + sq;
          }
        }
        for (int off = 16; off >= 1; off >>= 1) {
          float nxt[32];
          for (int l = 0; l < 32; ++l) nxt[l] = part[l] + part[l ^ off];
          memcpy(part, nxt, sizeof(part));
        }
        float nrm = sqrtf(part[0]);
        for (int j = 0; j < n; ++j)
          acc[j] = acc[j] + (!isfinite(post[j]) ? post[j] : (nrm == 0.0f ? 0.0f : post[j] / nrm));
      }
      for (int j = 0; j < n; ++j) w->soft[j] = (double)(acc[j] / (float)K);
    }
    int32_t ncl = 0, big = 0;
    int status = lsd_core(w, w->soft, w->s, prm->lsd_order, w->ebits, NULL, &ncl, &big);
    st->status = (uint8_t)status;
    st->n_clusters = (uint32_t)ncl;
    st->largest_cluster = (uint16_t)big;
    if (status) memset(w->ebits, 0, (size_t)n);
  }
  int nw = (n + 31) / 32;
  for (int t = 0; t < nw; ++t) corr[t] = 0;
  for (int j = 0; j < n; ++j)
    if (w->ebits[j]) corr[j >> 5] |= 1u << (j & 31);
  if (logi) {
    int kw = (P->k + 31) / 32;
    for (int t = 0; t < kw; ++t) logi[t] = 0;
    for (int r = 0; r < P->k; ++r) {
      int par = 0;
      for (int e = P->lrowptr[r]; e < P->lrowptr[r + 1]; ++e) par ^= w->ebits[P->lcolidx[e]];
      if (par) logi[r >> 5] |= 1u << (r & 31);
    }
  }
  if (soft_out) memcpy(soft_out, w->soft, sizeof(double) * (size_t)n);
}

/* ------------------------------------------------------------------------------------------ */
/* Public entry points                                                                          */
/* ------------------------------------------------------------------------------------------ */
int32_t or_bp_member(const or_problem* P, const uint8_t* syndrome, const uint32_t* perm, int32_t T,
                     float alpha, int32_t mode, int32_t early_stop, double* posterior, uint8_t* ebits) {
  workspace w;
  ws_init(&w, P, 1, mode);
  memcpy(w.s, syndrome, (size_t)P->m);
  init_member(&w, 0);
  int conv = 0;
  for (int t = 1; t <= T; ++t) {
    int ok;
    if (mode == OR_FP64) {
      sweep_f64(&w.g, perm, w.s, w.lam64, (double)alpha, w.msg64, w.post64, w.mcv64);
      ok = satisfies_f64(&w.g, w.s, w.post64);
    } else {
      sweep_f32(&w.g, perm, w.s, w.lam32, alpha, mode == OR_FP16MSG, w.msg32, w.post32, w.mcv32);
      ok = satisfies_f32(&w.g, w.s, w.post32);
    }
    if (ok && !conv) conv = t;
    if (ok && early_stop) break;
  }
  for (int j = 0; j < P->n; ++j) {
    double L = mode == OR_FP64 ? w.post64[j] : (double)w.post32[j];
    if (posterior) posterior[j] = L;
    if (ebits) ebits[j] = (uint8_t)(L <= 0.0);
  }
  ws_free(&w);
  return conv;
}

int32_t or_bp_member_flood(const or_problem* P, const uint8_t* syndrome, int32_t T, float alpha, int32_t mode,
                           int32_t early_stop, double* posterior, uint8_t* ebits) {
  workspace w;
  ws_init(&w, P, 1, mode);
  memcpy(w.s, syndrome, (size_t)P->m);
  init_member(&w, 0);
  float* c2v32 = w.c2v32;
  double* c2v64 = w.c2v64;
  int conv = 0;
  for (int t = 1; t <= T; ++t) {
    int ok;
    if (mode == OR_FP64) {
      flood_f64(&w.g, w.s, w.lam64, (double)alpha, w.msg64, c2v64, w.post64);
      ok = satisfies_f64(&w.g, w.s, w.post64);
    } else {
      flood_f32(&w.g, w.s, w.lam32, alpha, mode == OR_FP16MSG, w.msg32, c2v32, w.post32);
      ok = satisfies_f32(&w.g, w.s, w.post32);
    }
    if (ok && !conv) conv = t;
    if (ok && early_stop) break;
  }
  for (int j = 0; j < P->n; ++j) {
    double L = mode == OR_FP64 ? w.post64[j] : (double)w.post32[j];
    if (posterior) posterior[j] = L;
    if (ebits) ebits[j] = (uint8_t)(L <= 0.0);
  }
  ws_free(&w);
  return conv;
}

int32_t or_bp_member_layered(const or_problem* P, const uint8_t* syndrome, int32_t T, float alpha, int32_t mode,
                             int32_t early_stop, double* posterior, uint8_t* ebits, int32_t* nlayer) {
  workspace w;
  ws_init(&w, P, 1, mode);
  ws_layered(&w);
  memcpy(w.s, syndrome, (size_t)P->m);
  init_member(&w, 0);
  int conv = 0;
  for (int t = 1; t <= T; ++t) {
    int ok;
    if (mode == OR_FP64) {
      layered_f64(&w.g, w.s, w.lam64, (double)alpha, w.msg64, w.lc2v64, w.post64);
      ok = satisfies_f64(&w.g, w.s, w.post64);
    } else {
      layered_f32(&w.g, w.s, w.lam32, alpha, mode == OR_FP16MSG, w.msg32, w.lc2v32, w.post32);
      ok = satisfies_f32(&w.g, w.s, w.post32);
    }
    if (ok && !conv) conv = t;
    if (ok && early_stop) break;
  }
  for (int j = 0; j < P->n; ++j) {
    double L = mode == OR_FP64 ? w.post64[j] : (double)w.post32[j];
    if (posterior) posterior[j] = L;
    if (ebits) ebits[j] = (uint8_t)(L <= 0.0);
  }
  if (nlayer) *nlayer = w.g.nlayer;
  ws_free(&w);
  return conv;
}

int32_t or_check_layers(const or_problem* P, int32_t* layer_of_check) {
  graph g;
  graph_build(&g, P);
  for (int l = 0; l < g.nlayer; ++l)
    for (int q = g.layer_ptr[l]; q < g.layer_ptr[l + 1]; ++q) layer_of_check[g.layer_chk[q]] = l;
  int nl = g.nlayer;
  graph_free(&g);
  return nl;
}

int32_t or_lsd(const or_problem* P, const double* soft, const uint8_t* syndrome, int32_t order,
               const float* lam32, const double* lam64, uint8_t* ebits, int32_t* cluster_of_col,
               int32_t* n_clusters, int32_t* largest_cluster) {
  workspace w;
  ws_init(&w, P, 1, lam64 ? OR_FP64 : OR_FP32);
  if (lam32) memcpy(w.lam32, lam32, sizeof(float) * (size_t)P->n);
  if (lam64) memcpy(w.lam64, lam64, sizeof(double) * (size_t)P->n);
  int st = lsd_core(&w, soft, syndrome, order, ebits, cluster_of_col, n_clusters, largest_cluster);
  ws_free(&w);
  return st;
}

typedef struct {
  const or_problem* P; int K; const uint32_t* perms; const or_params* prm;
  int64_t b0, b1; const uint32_t* syn; uint32_t* corr; uint32_t* logi; or_shot_stats* stats; double* soft;
} job;

static void* run_job(void* arg) {
  job* j = (job*)arg;
  const or_problem* P = j->P;
  int mw = (P->m + 31) / 32, nw = (P->n + 31) / 32, kw = (P->k + 31) / 32;
  workspace w;
  ws_init(&w, P, j->K, j->prm->mode);
  if (j->prm->n_layered > 0) ws_layered(&w);
  for (int64_t b = j->b0; b < j->b1; ++b) {
    or_shot_stats st;
    decode_one(&w, j->perms, j->prm, j->syn + (size_t)b * mw, j->corr + (size_t)b * nw,
               j->logi ? j->logi + (size_t)b * kw : NULL, &st, j->soft ? j->soft + (size_t)b * P->n : NULL);
    if (j->stats) j->stats[b] = st;
  }
  ws_free(&w);
  return NULL;
}

int32_t or_decode(const or_problem* P, int32_t K, const uint32_t* perms, const or_params* prm, int64_t B,
                  const uint32_t* syndromes, uint32_t* corrections, uint32_t* logical,
                  or_shot_stats* stats, double* soft, int32_t nthreads) {
  if (!P || !perms || !prm || !syndromes || !corrections || K < 1 || prm->M < 1 || prm->M > K ||
      prm->T < 1 || B < 0 || prm->n_flood < 0 || prm->n_layered < 0 || prm->n_flood + prm->n_layered > K)
    return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > B) nthreads = B > 0 ? (int32_t)B : 1;
  job* jobs = (job*)calloc((size_t)nthreads, sizeof(job));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    job j = {P, K, perms, prm, B * t / nthreads, B * (t + 1) / nthreads, syndromes, corrections, logical, stats, soft};
    jobs[t] = j;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
  run_job(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  free(jobs); free(th);
  return 0;
}

static uint64_t splitmix64_next(uint64_t* st) {
  uint64_t z = (*st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

void or_seeded_schedules(int32_t n, int32_t K, uint64_t seed, uint32_t* perms) {
  for (int i = 0; i < K; ++i) {
    uint32_t* p = perms + (size_t)i * n;
    uint64_t st = seed + (uint64_t)(i + 1) * 0xD1B54A32D192ED03ull;
    for (int j = 0; j < n; ++j) p[j] = (uint32_t)j;
    for (int k = n - 1; k >= 1; --k) {
      uint64_t r = splitmix64_next(&st);
      uint64_t j = (uint64_t)(((unsigned __int128)r * (unsigned __int128)(uint64_t)(k + 1)) >> 64);
      uint32_t t = p[k]; p[k] = p[j]; p[j] = t;
    }
  }
}
