// Host side of the C ABI declared in include/vibe.h: input validation, the resident device tables
// of a decoding problem, the batch workspace, and the launch sequence of one decode
// (persistent BP ensemble -> LSD on the unresolved shots), chunked when a batch outgrows the workspace.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vibe_internal.cuh"

namespace vibe {
long long lsd_scratch_words(const Tables& t);
}

using vibe::Tables;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(VIBE_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(VIBE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define VIBE_CUDA(call, what)                 \
  do {                                        \
    cudaError_t e_ = (call);                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t kWorkspaceBytes = size_t(4) << 30;   // LSD hand-off buffer budget per handle

int check_csr(const vibe_csr* A, const char* name, bool rows_nonempty) {
  if (!A || !A->rowptr || (!A->colidx && A->nrows > 0)) return fail(VIBE_ERR_INVALID, "%s: NULL matrix", name);
  if (A->nrows < 0 || A->ncols < 1) return fail(VIBE_ERR_INVALID, "%s: bad shape %d x %d", name, A->nrows, A->ncols);
  if (A->rowptr[0] != 0) return fail(VIBE_ERR_INVALID, "%s: rowptr[0] != 0", name);
  for (int r = 0; r < A->nrows; ++r) {
    const int b = A->rowptr[r], e = A->rowptr[r + 1];
    if (e < b) return fail(VIBE_ERR_INVALID, "%s: rowptr decreases at row %d", name, r);
    if (rows_nonempty && e == b) return fail(VIBE_ERR_INVALID, "%s: row %d has no entry", name, r);
    for (int q = b; q < e; ++q) {
      const int c = A->colidx[q];
      if (c < 0 || c >= A->ncols) return fail(VIBE_ERR_INVALID, "%s: column %d out of range in row %d", name, c, r);
      if (q > b && c <= A->colidx[q - 1])
        return fail(VIBE_ERR_INVALID, "%s: columns not strictly ascending in row %d", name, r);
    }
  }
  return VIBE_OK;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

}  // namespace

struct vibe_handle {
  int device = 0;
  int num_sms = 0;
  Tables t{};
  int T = 0, M = 0, lsd_order = 0, msg_fp16 = 0;
  float alpha = 0.f;
  // resident tables
  int32_t *rowptr = nullptr, *colidx = nullptr, *colptr = nullptr, *rowidx = nullptr;
  int32_t *lrowptr = nullptr, *lcolidx = nullptr, *nlev = nullptr;
  uint32_t *csc_ent = nullptr, *sched = nullptr, *lvl_off = nullptr, *perm = nullptr;
  float* lam = nullptr;
  void* msg_init = nullptr;
  // launch configuration
  vibe::BpLayout L{};
  int bp_blocks_per_sm = 0, lsd_blocks_per_sm = 0;
  // workspace (grown on demand)
  long long ws_chunk = 0;
  long long chunk_max = 0;
  unsigned int* ctrl = nullptr;           // [0] next shot, [1] LSD count, [2] next LSD shot
  uint32_t* lsd_shots = nullptr;
  float* lsd_soft = nullptr;
  float* bp_scratch = nullptr;
  uint32_t* lsd_scratch = nullptr;
  unsigned long long* tmp_counters = nullptr;
  // host-buffer staging
  long long stage_cap = 0;
  uint32_t *st_syn = nullptr, *st_corr = nullptr, *st_log = nullptr, *st_obs = nullptr;
  vibe_shot_stats* st_stats = nullptr;
  // kernel timing
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  long long bp_launches = 0, lsd_launches = 0;

  void release_workspace() {
    cudaFree(ctrl); cudaFree(lsd_shots); cudaFree(lsd_soft); cudaFree(bp_scratch); cudaFree(lsd_scratch);
    ctrl = nullptr; lsd_shots = nullptr; lsd_soft = nullptr; bp_scratch = nullptr; lsd_scratch = nullptr;
    ws_chunk = 0;
  }
  void release_stage() {
    cudaFree(st_syn); cudaFree(st_corr); cudaFree(st_log); cudaFree(st_obs); cudaFree(st_stats);
    st_syn = st_corr = st_log = st_obs = nullptr; st_stats = nullptr; stage_cap = 0;
  }
  ~vibe_handle() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    release_workspace();
    release_stage();
    cudaFree(tmp_counters);
    cudaFree(rowptr); cudaFree(colidx); cudaFree(colptr); cudaFree(rowidx); cudaFree(lrowptr); cudaFree(lcolidx);
    cudaFree(nlev); cudaFree(csc_ent); cudaFree(sched); cudaFree(lvl_off); cudaFree(perm); cudaFree(lam);
    cudaFree(msg_init);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    cudaSetDevice(prev);
  }
  int bp_grid() const { return std::max(1, bp_blocks_per_sm * num_sms); }
  int lsd_grid() const { return std::max(1, lsd_blocks_per_sm * num_sms); }
};

namespace {

int ensure_workspace(vibe_handle* h, long long need) {
  const long long chunk = std::min(need, h->chunk_max);
  if (h->ctrl && chunk <= h->ws_chunk) return VIBE_OK;
  h->release_workspace();
  const Tables& t = h->t;
  const long long bp_warps = (long long)h->bp_grid() * vibe::kBpWarpsPerCta;
  VIBE_CUDA(dalloc(&h->ctrl, 4), "workspace");
  VIBE_CUDA(dalloc(&h->lsd_shots, (size_t)chunk), "workspace");
  VIBE_CUDA(dalloc(&h->lsd_soft, (size_t)chunk * t.n), "workspace");
  VIBE_CUDA(dalloc(&h->bp_scratch, (size_t)bp_warps * (size_t)(2 + h->M) * t.n), "workspace");
  VIBE_CUDA(dalloc(&h->lsd_scratch, (size_t)h->lsd_grid() * (size_t)vibe::lsd_scratch_words(t)), "workspace");
  h->ws_chunk = chunk;
  return VIBE_OK;
}

cudaEvent_t next_event(vibe_handle* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

int decode_device(vibe_handle* h, const uint32_t* syn, long long B, uint32_t* corr, uint32_t* logical,
                  vibe_shot_stats* stats, float* soft, const uint32_t* obs, unsigned long long* counters,
                  cudaStream_t s) {
  int rc = ensure_workspace(h, B);
  if (rc != VIBE_OK) return rc;
  const Tables& t = h->t;
  for (long long b0 = 0; b0 < B; b0 += h->ws_chunk) {
    const long long nb = std::min(h->ws_chunk, B - b0);
    VIBE_CUDA(cudaMemsetAsync(h->ctrl, 0, 4 * sizeof(unsigned int), s), "decode");
    vibe::BpArgs a{};
    a.t = t;
    a.T = h->T; a.M = h->M; a.alpha = h->alpha; a.want_soft = soft != nullptr;
    a.warp_smem = h->L.warp_smem; a.off_msg = h->L.off_msg; a.off_dec = h->L.off_dec;
    a.off_s = h->L.off_s; a.off_par = h->L.off_par; a.off_cand = h->L.off_cand;
    a.syn = syn + (size_t)b0 * t.mw;
    a.nshots = (uint32_t)nb;
    a.corr = corr + (size_t)b0 * t.nw;
    a.logical = logical ? logical + (size_t)b0 * t.kw : nullptr;
    a.stats = stats ? stats + b0 : nullptr;
    a.soft = soft ? soft + (size_t)b0 * t.n : nullptr;
    a.obs = obs ? obs + (size_t)b0 * t.kw : nullptr;
    a.counters = counters;
    a.next_shot = h->ctrl;
    a.lsd_count = h->ctrl + 1;
    a.lsd_shots = h->lsd_shots;
    a.lsd_soft = h->lsd_soft;
    a.scratch = h->bp_scratch;
    a.scratch_pitch = (long long)(2 + h->M) * t.n;
    const int bp_grid = (int)std::min<long long>(h->bp_grid(), (nb + vibe::kBpWarpsPerCta - 1) / vibe::kBpWarpsPerCta);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (h->profiling) { e0 = next_event(h); e1 = next_event(h); e2 = next_event(h); }
    if (e0) cudaEventRecord(e0, s);
    VIBE_CUDA(vibe::launch_bp(a, h->msg_fp16, bp_grid, s), "BP kernel launch");
    if (e1) cudaEventRecord(e1, s);
    vibe::LsdArgs l{};
    l.t = t;
    l.T = h->T; l.order = h->lsd_order; l.want_soft = soft != nullptr;
    l.CW = (t.n + 31) / 32;
    l.syn = a.syn; l.corr = a.corr; l.logical = a.logical; l.stats = a.stats; l.soft = a.soft; l.obs = a.obs;
    l.counters = counters;
    l.lsd_count = h->ctrl + 1; l.lsd_shots = h->lsd_shots; l.lsd_soft = h->lsd_soft; l.lsd_next = h->ctrl + 2;
    l.scratch = h->lsd_scratch;
    l.scratch_pitch = vibe::lsd_scratch_words(t);
    VIBE_CUDA(vibe::launch_lsd(l, h->lsd_grid(), s), "LSD kernel launch");
    if (e2) cudaEventRecord(e2, s);
    h->bp_launches++;
    h->lsd_launches++;
  }
  return VIBE_OK;
}

}  // namespace

extern "C" {

const char* vibe_last_error(void) { return g_err.c_str(); }

int vibe_create(const vibe_csr* H, const vibe_csr* L, const double* priors, int32_t K, const uint32_t* schedules,
                const vibe_params* p, vibe_handle** out) {
  if (!out) return fail(VIBE_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!p || !priors) return fail(VIBE_ERR_INVALID, "NULL params or priors");
  int rc;
  if ((rc = check_csr(H, "H", true)) != VIBE_OK) return rc;
  if ((rc = check_csr(L, "L", false)) != VIBE_OK) return rc;
  const int m = H->nrows, n = H->ncols, k = L->nrows;
  if (m < 1) return fail(VIBE_ERR_INVALID, "H has no rows");
  if (L->ncols != n) return fail(VIBE_ERR_INVALID, "L has %d columns, H has %d", L->ncols, n);
  if (k < 1 || k > 1024) return fail(VIBE_ERR_INVALID, "L must have 1..1024 rows, got %d", k);
  if (K < 1 || K > 255) return fail(VIBE_ERR_INVALID, "K must be in 1..255, got %d", K);
  if (p->max_iter < 1 || p->max_iter > 65535) return fail(VIBE_ERR_INVALID, "max_iter must be in 1..65535");
  if (!(p->alpha > 0.f && p->alpha <= 1.f)) return fail(VIBE_ERR_INVALID, "alpha must be in (0, 1]");
  if (p->M < 1 || p->M > K || p->M > 32) return fail(VIBE_ERR_INVALID, "M must be in 1..min(K, 32)");
  if (p->lsd_order < 0 || p->lsd_order > 10) return fail(VIBE_ERR_INVALID, "lsd_order must be in 0..10");
  if (p->msg_fp16 != 0 && p->msg_fp16 != 1) return fail(VIBE_ERR_INVALID, "msg_fp16 must be 0 or 1");
  for (int j = 0; j < n; ++j)
    if (!(priors[j] > 0.0 && priors[j] < 0.5)) return fail(VIBE_ERR_INVALID, "prior %d = %g outside (0, 0.5)", j, priors[j]);
  if (n >= (1 << 24) || m >= (1 << 24)) return fail(VIBE_ERR_UNSUPPORTED, "n and m must be below 2^24");
  const int E = H->rowptr[m];
  int maxrow = 0;
  for (int r = 0; r < m; ++r) maxrow = std::max(maxrow, H->rowptr[r + 1] - H->rowptr[r]);
  std::vector<int> coldeg(n, 0);
  for (int e = 0; e < E; ++e) coldeg[H->colidx[e]]++;
  const int maxcol = *std::max_element(coldeg.begin(), coldeg.end());
  if (maxrow > vibe::kMaxRowDeg) return fail(VIBE_ERR_UNSUPPORTED, "a row of H has %d > 255 entries", maxrow);
  if (maxcol > vibe::kMaxColDeg) return fail(VIBE_ERR_UNSUPPORTED, "a column of H has %d > 32 entries", maxcol);
  if (schedules) {
    std::vector<unsigned char> seen(n);
    for (int i = 0; i < K; ++i) {
      std::fill(seen.begin(), seen.end(), 0);
      for (int j = 0; j < n; ++j) {
        const uint32_t v = schedules[(size_t)i * n + j];
        if (v >= (uint32_t)n || seen[v]) return fail(VIBE_ERR_INVALID, "schedule %d is not a permutation", i);
        seen[v] = 1;
      }
    }
  }
  std::vector<float> lam(n);
  for (int j = 0; j < n; ++j) lam[j] = (float)std::log((1.0 - priors[j]) / priors[j]);

  vibe_handle* h = new (std::nothrow) vibe_handle();
  if (!h) return fail(VIBE_ERR_NOMEM, "host allocation failed");
  auto bail = [&](int code) { delete h; return code; };
  cudaError_t e;
  if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(cuda_fail(e, "cudaGetDevice"));
  if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
    return bail(cuda_fail(e, "device query"));
  h->T = p->max_iter; h->M = p->M; h->alpha = p->alpha; h->lsd_order = p->lsd_order; h->msg_fp16 = p->msg_fp16;
  Tables& t = h->t;
  t.m = m; t.n = n; t.k = k; t.E = E; t.K = K;
  t.RP = std::max(8, (maxrow + 7) / 8 * 8);
  t.DP = maxcol <= 4 ? 4 : maxcol <= 8 ? 8 : maxcol <= 16 ? 16 : 32;
  t.mw = (m + 31) / 32; t.nw = (n + 31) / 32; t.kw = (k + 31) / 32; t.W = t.mw;
  const int Lnnz = L->rowptr[k];
  const size_t msg_bytes = (size_t)m * t.RP * (p->msg_fp16 ? 2 : 4);
  const size_t lev_scratch = std::max<size_t>(2 * (size_t)n + E, (size_t)K * ((size_t)m + 3 * (size_t)n + 1));
  int32_t* scratch = nullptr;
  cudaStream_t s = nullptr;
#define VIBE_TRY(call, what) \
  if ((e = (call)) != cudaSuccess) { cudaFree(scratch); if (s) cudaStreamDestroy(s); return bail(cuda_fail(e, what)); }
  VIBE_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream");
  VIBE_TRY(dalloc(&h->rowptr, m + 1), "tables");
  VIBE_TRY(dalloc(&h->colidx, E), "tables");
  VIBE_TRY(dalloc(&h->colptr, n + 1), "tables");
  VIBE_TRY(dalloc(&h->rowidx, E), "tables");
  VIBE_TRY(dalloc(&h->lrowptr, k + 1), "tables");
  VIBE_TRY(dalloc(&h->lcolidx, Lnnz), "tables");
  VIBE_TRY(dalloc(&h->nlev, K), "tables");
  VIBE_TRY(dalloc(&h->csc_ent, (size_t)n * t.DP), "tables");
  VIBE_TRY(dalloc(&h->sched, (size_t)K * n), "tables");
  VIBE_TRY(dalloc(&h->lvl_off, (size_t)K * (n + 1)), "tables");
  VIBE_TRY(dalloc(&h->perm, (size_t)K * n), "tables");
  VIBE_TRY(dalloc(&h->lam, n), "tables");
  VIBE_TRY(cudaMalloc(&h->msg_init, std::max<size_t>(msg_bytes, 16)), "tables");
  VIBE_TRY(dalloc(&scratch, lev_scratch), "tables");
  VIBE_TRY(dalloc(&h->tmp_counters, VIBE_NUM_COUNTERS), "tables");
  VIBE_TRY(cudaMemcpyAsync(h->rowptr, H->rowptr, sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->colidx, H->colidx, sizeof(int32_t) * std::max(E, 0), cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->lrowptr, L->rowptr, sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, s), "upload");
  if (Lnnz > 0)
    VIBE_TRY(cudaMemcpyAsync(h->lcolidx, L->colidx, sizeof(int32_t) * Lnnz, cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->lam, lam.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s), "upload");
  if (schedules) {
    VIBE_TRY(cudaMemcpyAsync(h->perm, schedules, sizeof(uint32_t) * (size_t)K * n, cudaMemcpyHostToDevice, s), "upload");
  } else {
    VIBE_TRY(vibe::seeded_schedules(h->perm, n, K, p->seed, s), "schedule kernel");
  }
  VIBE_TRY(vibe::build_tables(h->rowptr, h->colidx, m, n, K, h->perm, t.RP, t.DP, p->msg_fp16, h->lam, h->colptr,
                              h->rowidx, h->csc_ent, h->msg_init, h->sched, h->lvl_off, h->nlev, scratch, s),
           "graph builder");
  VIBE_TRY(cudaStreamSynchronize(s), "graph builder");
  cudaFree(scratch);
  scratch = nullptr;
  cudaStreamDestroy(s);
  s = nullptr;
#undef VIBE_TRY
  t.rowptr = h->rowptr; t.colidx = h->colidx; t.colptr = h->colptr; t.rowidx = h->rowidx;
  t.csc_ent = h->csc_ent; t.lam = h->lam; t.msg_init = h->msg_init; t.sched = h->sched; t.lvl_off = h->lvl_off;
  t.nlev = h->nlev; t.lrowptr = h->lrowptr; t.lcolidx = h->lcolidx;

  const size_t wsm = vibe::bp_warp_smem_bytes(t, h->M, h->msg_fp16, &h->L);
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (wsm * vibe::kBpWarpsPerCta > (size_t)optin)
    return bail(fail(VIBE_ERR_UNSUPPORTED, "BP state of one shot (%zu bytes) does not fit in shared memory", wsm));
  if (vibe::lsd_smem_bytes(t) > (size_t)optin)
    return bail(fail(VIBE_ERR_UNSUPPORTED, "LSD state does not fit in shared memory"));
  if ((e = vibe::bp_occupancy(t, h->msg_fp16, wsm * vibe::kBpWarpsPerCta, &h->bp_blocks_per_sm)) != cudaSuccess)
    return bail(cuda_fail(e, "BP occupancy"));
  if ((e = vibe::lsd_occupancy(t, &h->lsd_blocks_per_sm)) != cudaSuccess) return bail(cuda_fail(e, "LSD occupancy"));
  if (h->bp_blocks_per_sm < 1 || h->lsd_blocks_per_sm < 1)
    return bail(fail(VIBE_ERR_UNSUPPORTED, "kernels cannot be resident with this problem size"));
  h->chunk_max = std::max<long long>(1, (long long)(kWorkspaceBytes / ((size_t)n * 4 + 8)));
  *out = h;
  return VIBE_OK;
}

int vibe_decode(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, uint32_t* d_corrections, uint32_t* d_logical,
                vibe_shot_stats* d_stats, float* d_soft, const uint32_t* d_observables, uint64_t* d_counters,
                void* stream) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  if (B < 0) return fail(VIBE_ERR_INVALID, "negative batch");
  if (B == 0) return VIBE_OK;
  if (!d_syndromes || !d_corrections) return fail(VIBE_ERR_INVALID, "NULL syndromes or corrections");
  if (B > 0x7fffffffLL) return fail(VIBE_ERR_INVALID, "batch too large");
  return decode_device(h, d_syndromes, B, d_corrections, d_logical, d_stats, d_soft, d_observables,
                       reinterpret_cast<unsigned long long*>(d_counters), static_cast<cudaStream_t>(stream));
}

int vibe_decode_host(vibe_handle* h, const uint32_t* h_syndromes, int64_t B, uint32_t* h_corrections,
                     uint32_t* h_logical, vibe_shot_stats* h_stats, const uint32_t* h_observables,
                     uint64_t* h_counters, void* stream) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  if (B < 0) return fail(VIBE_ERR_INVALID, "negative batch");
  if (!h_syndromes || !h_corrections) return fail(VIBE_ERR_INVALID, "NULL syndromes or corrections");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Tables& t = h->t;
  if (h_counters) VIBE_CUDA(cudaMemsetAsync(h->tmp_counters, 0, sizeof(uint64_t) * VIBE_NUM_COUNTERS, s), "counters");
  if (B > 0) {
    const long long chunk = std::min<long long>(B, h->chunk_max);
    if (chunk > h->stage_cap) {
      h->release_stage();
      VIBE_CUDA(dalloc(&h->st_syn, (size_t)chunk * t.mw), "staging");
      VIBE_CUDA(dalloc(&h->st_corr, (size_t)chunk * t.nw), "staging");
      VIBE_CUDA(dalloc(&h->st_log, (size_t)chunk * t.kw), "staging");
      VIBE_CUDA(dalloc(&h->st_obs, (size_t)chunk * t.kw), "staging");
      VIBE_CUDA(dalloc(&h->st_stats, (size_t)chunk), "staging");
      h->stage_cap = chunk;
    }
    for (long long b0 = 0; b0 < B; b0 += h->stage_cap) {
      const long long nb = std::min(h->stage_cap, B - b0);
      VIBE_CUDA(cudaMemcpyAsync(h->st_syn, h_syndromes + (size_t)b0 * t.mw, sizeof(uint32_t) * nb * t.mw,
                                cudaMemcpyHostToDevice, s), "H2D");
      if (h_observables)
        VIBE_CUDA(cudaMemcpyAsync(h->st_obs, h_observables + (size_t)b0 * t.kw, sizeof(uint32_t) * nb * t.kw,
                                  cudaMemcpyHostToDevice, s), "H2D");
      int rc = decode_device(h, h->st_syn, nb, h->st_corr, h->st_log, h->st_stats, nullptr,
                             h_observables ? h->st_obs : nullptr, h_counters ? h->tmp_counters : nullptr, s);
      if (rc != VIBE_OK) return rc;
      VIBE_CUDA(cudaMemcpyAsync(h_corrections + (size_t)b0 * t.nw, h->st_corr, sizeof(uint32_t) * nb * t.nw,
                                cudaMemcpyDeviceToHost, s), "D2H");
      if (h_logical)
        VIBE_CUDA(cudaMemcpyAsync(h_logical + (size_t)b0 * t.kw, h->st_log, sizeof(uint32_t) * nb * t.kw,
                                  cudaMemcpyDeviceToHost, s), "D2H");
      if (h_stats)
        VIBE_CUDA(cudaMemcpyAsync(h_stats + b0, h->st_stats, sizeof(vibe_shot_stats) * nb, cudaMemcpyDeviceToHost, s),
                  "D2H");
    }
  }
  if (h_counters)
    VIBE_CUDA(cudaMemcpyAsync(h_counters, h->tmp_counters, sizeof(uint64_t) * VIBE_NUM_COUNTERS,
                              cudaMemcpyDeviceToHost, s), "D2H");
  VIBE_CUDA(cudaStreamSynchronize(s), "decode");
  return VIBE_OK;
}

int vibe_get_wavefronts(vibe_handle* h, int32_t member, uint32_t* order_out, uint32_t* level_offsets_out,
                        int32_t* nlevels_out) {
  if (!h || !order_out || !level_offsets_out || !nlevels_out) return fail(VIBE_ERR_INVALID, "NULL argument");
  if (member < 0 || member >= h->t.K) return fail(VIBE_ERR_INVALID, "member out of range");
  const int n = h->t.n;
  VIBE_CUDA(cudaMemcpy(order_out, h->sched + (size_t)member * n, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost), "copy");
  VIBE_CUDA(cudaMemcpy(level_offsets_out, h->lvl_off + (size_t)member * (n + 1), sizeof(uint32_t) * (n + 1),
                       cudaMemcpyDeviceToHost), "copy");
  VIBE_CUDA(cudaMemcpy(nlevels_out, h->nlev + member, sizeof(int32_t), cudaMemcpyDeviceToHost), "copy");
  for (int j = 0; j < n; ++j) order_out[j] &= 0xffffffu;
  return VIBE_OK;
}

int vibe_profile(vibe_handle* h, int32_t enable) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  h->profiling = enable != 0;
  h->ev_used = 0;
  h->bp_launches = 0;
  h->lsd_launches = 0;
  return VIBE_OK;
}

int vibe_profile_read(vibe_handle* h, double* bp_ms, double* lsd_ms, int64_t* bp_launches, int64_t* lsd_launches) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  double bp = 0.0, lsd = 0.0;
  for (size_t i = 0; i + 3 <= h->ev_used; i += 3) {
    float a = 0.f, b = 0.f;
    VIBE_CUDA(cudaEventSynchronize(h->ev_pool[i + 2]), "profile");
    VIBE_CUDA(cudaEventElapsedTime(&a, h->ev_pool[i], h->ev_pool[i + 1]), "profile");
    VIBE_CUDA(cudaEventElapsedTime(&b, h->ev_pool[i + 1], h->ev_pool[i + 2]), "profile");
    bp += a;
    lsd += b;
  }
  if (bp_ms) *bp_ms = bp;
  if (lsd_ms) *lsd_ms = lsd;
  if (bp_launches) *bp_launches = h->bp_launches;
  if (lsd_launches) *lsd_launches = h->lsd_launches;
  return VIBE_OK;
}

int vibe_destroy(vibe_handle* h) {
  delete h;
  return VIBE_OK;
}

}  // extern "C"

// Read-only access to a handle's resident problem for the library's other host translation units.
namespace vibe {

int handle_view(const vibe_handle* h, HandleView* v) {
  if (!h || !v) return fail(VIBE_ERR_INVALID, "NULL handle");
  v->t = h->t;
  v->device = h->device;
  v->T = h->T; v->M = h->M; v->lsd_order = h->lsd_order; v->msg_fp16 = h->msg_fp16; v->alpha = h->alpha;
  v->L = h->L;
  v->bp_grid = h->bp_grid();
  v->lsd_grid = h->lsd_grid();
  v->num_sms = h->num_sms;
  return VIBE_OK;
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace vibe
