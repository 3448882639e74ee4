// Host side of the C ABI declared in include/vibe.h: input validation, the resident device tables
// of a decoding problem, batch workspaces, the launch sequence of one decode (persistent BP ensemble
// -> LSD on the unresolved shots, chunked when a batch outgrows the workspace), mixed batches over
// several problems, kernel timing and the launch-size tuner.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vibe_internal.cuh"

using vibe::Bounds;
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

#define VIBE_CUDA(call, what)                          \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t kWorkspaceBytes = size_t(4) << 30;   // LSD hand-off buffer budget per workspace

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

// What one decode launch needs besides the batch buffers.
struct Launch {
  Tables one{};                     // host descriptor of a single-problem launch
  bool mixed = false;               // shots name their problems (vibe_batch)
  const Tables* d_desc = nullptr;   // ndem problem descriptors on the device
  int ndem = 0;
  Bounds bnd{};
  int msg_fp16 = 0;
  int device = 0, num_sms = 0;
  int bp_blocks_per_sm = 0, bpx_blocks_per_sm = 0, lsd_blocks_per_sm = 0;
  int pair_mode = 0;                // one warp per (shot, member) pair (vibe_params.pair_mode)
  int lsd_threads = vibe::kLsdThreads;   // threads per LSD CTA (tuned: 64, 128 or 256)
  bool warp_engine() const { return (bnd.engines & 1) != 0; }
  bool cta_engine() const { return (bnd.engines & 2) != 0; }
  int bp_grid() const { return warp_engine() ? std::max(1, bp_blocks_per_sm * num_sms) : 0; }
  int bpx_grid() const { return cta_engine() ? std::max(1, bpx_blocks_per_sm * num_sms) : 0; }
  int lsd_grid() const { return std::max(1, lsd_blocks_per_sm * num_sms); }
  // per-warp global scratch of the summary engine, bytes; the candidate posteriors only with soft output
  long long bpx_pitch(bool soft) const {
    return (bnd.x_warp_scratch + (soft ? 4LL * bnd.M * bnd.n : 0LL) + 15) & ~15LL;
  }
  // pair mode: bytes of one shot's member records (iteration, weight, correction, LLR term, posterior)
  long long pair_shot_bytes(bool soft) const {
    return (long long)bnd.K * (8LL + 4LL * bnd.nw + 4LL * bnd.n * (soft ? 2 : 1)) + 4;
  }
  // pair mode: shots per launch -- as many as kPairBytes of member records hold, so that a large batch
  // keeps every warp busy across shots (a launch ends with its slowest pair) and a small one runs whole
  long long pair_chunk(bool soft) const { return std::max(1LL, kPairBytes / pair_shot_bytes(soft)); }
  static constexpr long long kPairBytes = 8LL << 30;
};

// Device memory a decode uses besides its inputs and outputs; grown on demand, reused afterwards.
struct Workspace {
  long long chunk = 0, chunk_max = 0;
  long long pk_nw = 0, pk_n = 0;   // pair records' sizes per shot the buffers were made for
  long long lsd_words = 0;         // LSD scratch words per CTA the buffer was made for
  int bp_warps = 0, lsd_ctas = 0;
  long long bpx_bytes = 0;
  unsigned int* ctrl = nullptr;   // [0] next shot (image engine), [1] LSD count, [2] next LSD shot,
                                  // [3] next shot (summary engine), [4] / [5] next pair (image / summary)
  uint32_t* lsd_shots = nullptr;
  float* lsd_soft = nullptr;
  float* bp_scratch = nullptr;
  unsigned char* bpx_scratch = nullptr;
  uint32_t* lsd_scratch = nullptr;
  // pair mode: member records of `pair_shots` shots (see BpArgs)
  long long pair_shots = 0;
  bool pair_soft = false;
  int* pconv = nullptr;
  float* pW = nullptr;
  uint32_t* pbits = nullptr;
  float* pterms = nullptr;
  float* ppost = nullptr;
  unsigned int* pdone = nullptr;

  void release() {
    cudaFree(ctrl); cudaFree(lsd_shots); cudaFree(lsd_soft); cudaFree(bp_scratch); cudaFree(bpx_scratch);
    cudaFree(lsd_scratch);
    cudaFree(pconv); cudaFree(pW); cudaFree(pbits); cudaFree(pterms); cudaFree(ppost); cudaFree(pdone);
    ctrl = nullptr; lsd_shots = nullptr; lsd_soft = nullptr; bp_scratch = nullptr; bpx_scratch = nullptr;
    lsd_scratch = nullptr;
    pconv = nullptr; pW = nullptr; pbits = nullptr; pterms = nullptr; ppost = nullptr; pdone = nullptr;
    chunk = 0; bp_warps = 0; lsd_ctas = 0; bpx_bytes = 0; pair_shots = 0; pair_soft = false; lsd_words = 0;
  }
  int ensure(const Launch& L, long long need, bool soft) {
    const long long ps = L.pair_mode ? std::min(need, L.pair_chunk(soft)) : 0;
    const long long want = std::min(need, chunk_max);
    const int warps = L.bp_grid() * vibe::kBpWarpsPerCta;
    const long long xb = (long long)L.bpx_grid() * vibe::kBpxWarpsPerCta * L.bpx_pitch(soft);
    const bool pair_ok = !L.pair_mode || (ps <= pair_shots && (!soft || pair_soft) && L.bnd.K * L.bnd.nw <= pk_nw &&
                                          L.bnd.K * L.bnd.n <= pk_n);
    const bool lsd_ok = (long long)L.lsd_grid() * vibe::lsd_scratch_words(L.bnd, L.lsd_threads) <=
                        (long long)lsd_ctas * lsd_words;
    if (ctrl && want <= chunk && warps <= bp_warps && lsd_ok && xb <= bpx_bytes && pair_ok)
      return VIBE_OK;
    const long long c = std::max(want, chunk);
    const long long xkeep = std::max(xb, bpx_bytes);
    release();
    const Bounds& b = L.bnd;
    VIBE_CUDA(dalloc(&ctrl, 8), "workspace");
    VIBE_CUDA(dalloc(&lsd_shots, (size_t)c), "workspace");
    VIBE_CUDA(dalloc(&lsd_soft, (size_t)c * b.n), "workspace");
    VIBE_CUDA(dalloc(&bp_scratch, (size_t)warps * (size_t)(2 + b.M) * b.n), "workspace");
    VIBE_CUDA(dalloc(&bpx_scratch, (size_t)xkeep), "workspace");
    VIBE_CUDA(dalloc(&lsd_scratch, (size_t)L.lsd_grid() * (size_t)vibe::lsd_scratch_words(b, L.lsd_threads)),
              "workspace");
    lsd_words = vibe::lsd_scratch_words(b, L.lsd_threads);
    if (L.pair_mode) {
      const size_t S = (size_t)ps;
      VIBE_CUDA(dalloc(&pconv, S * b.K), "workspace");
      VIBE_CUDA(dalloc(&pW, S * b.K), "workspace");
      VIBE_CUDA(dalloc(&pbits, S * b.K * (size_t)b.nw), "workspace");
      VIBE_CUDA(dalloc(&pterms, S * b.K * (size_t)b.n), "workspace");
      if (soft) VIBE_CUDA(dalloc(&ppost, S * b.K * (size_t)b.n), "workspace");
      VIBE_CUDA(dalloc(&pdone, S), "workspace");
      pair_shots = ps;
      pair_soft = soft;
      pk_nw = (long long)b.K * b.nw;
      pk_n = (long long)b.K * b.n;
    }
    chunk = c;
    bp_warps = warps;
    lsd_ctas = L.lsd_grid();
    bpx_bytes = xkeep;
    return VIBE_OK;
  }
  ~Workspace() { release(); }
};

// CUDA events around every kernel launch while enabled.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  long long bp_launches = 0, lsd_launches = 0;
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  ~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

struct Batch {
  const int32_t* dem_of_shot;
  const uint32_t* syn;
  int syn_stride;
  long long B;
  uint32_t* corr;
  int corr_stride;
  uint32_t* logical;
  int log_stride;
  vibe_shot_stats* stats;
  float* soft;
  int soft_stride;
  const uint32_t* obs;
  unsigned long long* counters;
};

// Decodes q in chunks of up to ws.chunk shots (the LSD hand-off space): the BP kernels over the chunk,
// then one LSD launch over the shots they queued. In pair mode the BP part of a chunk runs in
// sub-chunks of up to ws.pair_shots shots (the member records), all queueing into the chunk's LSD
// launch, so a chunk's slowest LSD shots are waited for once, not once per sub-chunk.
int run_decode(const Launch& L, Workspace& ws, Profiler& prof, const Batch& q, cudaStream_t s) {
  int rc = ws.ensure(L, q.B, q.soft != nullptr);
  if (rc != VIBE_OK) return rc;
  const long long step = ws.chunk;
  for (long long b0 = 0; b0 < q.B; b0 += step) {
    const long long nb = std::min(step, q.B - b0);
    VIBE_CUDA(cudaMemsetAsync(ws.ctrl, 0, 8 * sizeof(unsigned int), s), "decode");
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
    if (prof.on) { e0 = prof.next(); e1 = prof.next(); e2 = prof.next(); }
    if (e0) cudaEventRecord(e0, s);
    const long long sub = L.pair_mode ? std::min(nb, ws.pair_shots) : nb;
    for (long long s0 = 0; s0 < nb; s0 += sub) {
      const long long ns = std::min(sub, nb - s0);
      const long long o = b0 + s0;
      if (s0 > 0) {   // the BP work counters start again; the LSD queue keeps filling
        VIBE_CUDA(cudaMemsetAsync(ws.ctrl, 0, sizeof(unsigned int), s), "decode");
        VIBE_CUDA(cudaMemsetAsync(ws.ctrl + 3, 0, 3 * sizeof(unsigned int), s), "decode");
      }
      if (L.pair_mode) {
        VIBE_CUDA(cudaMemsetAsync(ws.pconv, 0, sizeof(int) * (size_t)ns * L.bnd.K, s), "decode");
        VIBE_CUDA(cudaMemsetAsync(ws.pdone, 0, sizeof(unsigned int) * (size_t)ns, s), "decode");
      }
      vibe::BpArgs a{};
      a.one = L.one;
      a.dems = L.d_desc; a.ndem = L.ndem; a.dem_of_shot = q.dem_of_shot ? q.dem_of_shot + o : nullptr;
      a.bnd = L.bnd;
      a.want_soft = q.soft != nullptr;
      a.syn = q.syn + (size_t)o * q.syn_stride; a.syn_stride = q.syn_stride;
      a.nshots = (uint32_t)ns;
      a.corr = q.corr + (size_t)o * q.corr_stride; a.corr_stride = q.corr_stride;
      a.logical = q.logical ? q.logical + (size_t)o * q.log_stride : nullptr; a.log_stride = q.log_stride;
      a.stats = q.stats ? q.stats + o : nullptr;
      a.soft = q.soft ? q.soft + (size_t)o * q.soft_stride : nullptr; a.soft_stride = q.soft_stride;
      a.obs = q.obs ? q.obs + (size_t)o * q.log_stride : nullptr;
      a.counters = q.counters;
      a.next_shot = ws.ctrl; a.lsd_count = ws.ctrl + 1; a.lsd_shots = ws.lsd_shots; a.lsd_soft = ws.lsd_soft;
      a.lsd_shot_base = (uint32_t)s0;
      a.scratch = ws.bp_scratch;
      a.scratch_pitch = (long long)(2 + L.bnd.M) * L.bnd.n;
      a.xscratch = ws.bpx_scratch;
      a.xscratch_pitch = L.bpx_pitch(a.want_soft != 0);
      a.next_shot_x = ws.ctrl + 3;
      a.pair_mode = L.pair_mode;
      a.pair_K = L.bnd.K;
      a.pconv = ws.pconv; a.pW = ws.pW; a.pbits = ws.pbits; a.pterms = ws.pterms; a.ppost = ws.ppost;
      a.pdone = ws.pdone;
      a.next_pair = ws.ctrl + 4;
      a.next_pair_x = ws.ctrl + 5;
      const long long units = L.pair_mode ? ns * L.bnd.K : ns;   // shots, or (shot, member) pairs
      if (L.warp_engine()) {
        const int grid =
            (int)std::min<long long>(L.bp_grid(), (units + vibe::kBpWarpsPerCta - 1) / vibe::kBpWarpsPerCta);
        a.flag_bad = 1;
        VIBE_CUDA(vibe::launch_bp(a, L.msg_fp16, grid, s), "BP kernel launch");
      }
      if (L.cta_engine()) {
        const int grid =
            (int)std::min<long long>(L.bpx_grid(), (units + vibe::kBpxWarpsPerCta - 1) / vibe::kBpxWarpsPerCta);
        a.flag_bad = L.warp_engine() ? 0 : 1;
        VIBE_CUDA(vibe::launch_bpx(a, L.msg_fp16, grid, s), "BP kernel launch");
      }
      prof.bp_launches++;
    }
    if (e1) cudaEventRecord(e1, s);
    vibe::LsdArgs l{};
    l.dems = L.d_desc; l.ndem = L.ndem; l.dem_of_shot = q.dem_of_shot ? q.dem_of_shot + b0 : nullptr;
    l.bnd = L.bnd;
    l.want_soft = q.soft != nullptr;
    l.syn = q.syn + (size_t)b0 * q.syn_stride; l.syn_stride = q.syn_stride;
    l.corr = q.corr + (size_t)b0 * q.corr_stride; l.corr_stride = q.corr_stride;
    l.logical = q.logical ? q.logical + (size_t)b0 * q.log_stride : nullptr; l.log_stride = q.log_stride;
    l.stats = q.stats ? q.stats + b0 : nullptr;
    l.soft = q.soft ? q.soft + (size_t)b0 * q.soft_stride : nullptr; l.soft_stride = q.soft_stride;
    l.obs = q.obs ? q.obs + (size_t)b0 * q.log_stride : nullptr;
    l.counters = q.counters;
    l.lsd_count = ws.ctrl + 1; l.lsd_shots = ws.lsd_shots; l.lsd_soft = ws.lsd_soft; l.lsd_next = ws.ctrl + 2;
    l.scratch = ws.lsd_scratch;
    l.scratch_pitch = vibe::lsd_scratch_words(L.bnd, L.lsd_threads);
    VIBE_CUDA(vibe::launch_lsd(l, L.lsd_grid(), L.lsd_threads, s), "LSD kernel launch");
    if (e2) cudaEventRecord(e2, s);
    prof.lsd_launches++;
  }
  return VIBE_OK;
}

// Occupancy-limited launch sizes for a launch configuration; fails if a kernel cannot be resident.
int size_launch(Launch& L) {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, L.device);
  const int nd = L.mixed ? L.ndem : 0;
  if (L.warp_engine()) {
    if (vibe::bp_cta_smem_bytes(L.bnd, nd) > (size_t)optin)
      return fail(VIBE_ERR_UNSUPPORTED, "BP state of one shot (%d bytes per warp) does not fit in shared memory",
                  L.bnd.warp_smem);
    VIBE_CUDA(vibe::bp_occupancy(L.bnd, nd, L.msg_fp16, &L.bp_blocks_per_sm), "BP occupancy");
    if (L.bp_blocks_per_sm < 1) return fail(VIBE_ERR_UNSUPPORTED, "the BP kernel cannot be resident");
  }
  if (L.cta_engine()) {
    if (vibe::bpx_cta_smem_bytes(L.bnd, nd) > (size_t)optin)
      return fail(VIBE_ERR_UNSUPPORTED, "check summaries of one shot (%d bytes per warp) do not fit in shared memory",
                  L.bnd.x_warp_smem);
    VIBE_CUDA(vibe::bpx_occupancy(L.bnd, nd, L.msg_fp16, &L.bpx_blocks_per_sm), "BP occupancy");
    if (L.bpx_blocks_per_sm < 1) return fail(VIBE_ERR_UNSUPPORTED, "the BP kernel cannot be resident");
  }
  if (vibe::lsd_smem_bytes(L.bnd, L.ndem) > (size_t)optin)
    return fail(VIBE_ERR_UNSUPPORTED, "LSD state of one shot does not fit in shared memory");
  VIBE_CUDA(vibe::lsd_occupancy(L.bnd, L.ndem, L.lsd_threads, &L.lsd_blocks_per_sm), "LSD occupancy");
  if (L.lsd_blocks_per_sm < 1) return fail(VIBE_ERR_UNSUPPORTED, "the LSD kernel cannot be resident");
  return VIBE_OK;
}

// Sizes bounding every problem of a launch; the engine-specific ones over that engine's problems only.
Bounds bounds_over(const Tables* ts, int count) {
  Bounds b{};
  bool first_warp = true;
  for (int i = 0; i < count; ++i) {
    const Tables& t = ts[i];
    b.m = std::max(b.m, t.m); b.n = std::max(b.n, t.n); b.W = std::max(b.W, t.W); b.nw = std::max(b.nw, t.nw);
    b.kw = std::max(b.kw, t.kw); b.M = std::max(b.M, t.M); b.DP = std::max(b.DP, t.DP); b.K = std::max(b.K, t.K);
    b.lsd_order = std::max(b.lsd_order, t.lsd_order);
    if (t.engine == VIBE_ENGINE_IMAGE) {
      b.engines |= 1;
      b.RP = first_warp ? t.RP : (b.RP == t.RP ? b.RP : 0);
      first_warp = false;
      b.warp_smem = std::max(b.warp_smem, t.warp_smem);
    } else {
      b.engines |= 2;
      b.XD = std::max(b.XD, t.XD);
      b.x_warp_smem = std::max(b.x_warp_smem, t.x_warp_smem);
      b.x_warp_scratch = std::max(b.x_warp_scratch, t.x_warp_scratch);
    }
  }
  if (b.engines & 2) b.x_warp_smem += vibe::bpx_ring_bytes(b.XD);
  return b;
}

// Searches the launch knobs that leave every result unchanged (shots, and within a shot the members'
// arithmetic, are fixed; only their placement on the GPU moves) for the fastest decode of the sample q:
// pair or shot mode (one warp per (shot, member) pair, or one per shot), then each present BP engine's
// persistent grid (occupancy maximum, 3/4, 1/2 CTAs per SM), then the LSD CTA size (64, 128, 256
// threads) with its grid (maximum, half). A candidate is timed on a first decode (the workspace grown
// beforehand) and, unless that took more than twice the best time so far, on a second one, which
// counts; a mode whose first candidate is rejected that way is dropped. L keeps the fastest; best_ms
// its time.
int tune_launch(Launch& L, Workspace& ws, Profiler& prof, const Batch& q, cudaStream_t s, float& best_ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  VIBE_CUDA(cudaEventCreate(&e0), "autotune");
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return cuda_fail(cudaGetLastError(), "autotune"); }
  const Launch base = L;
  Launch keep = base;
  float best = 1e30f;
  int rc = VIBE_OK;
  auto timed = [&](float& ms) -> int {
    cudaEventRecord(e0, s);
    const int r = run_decode(L, ws, prof, q, s);
    if (r != VIBE_OK) return r;
    cudaEventRecord(e1, s);
    VIBE_CUDA(cudaEventSynchronize(e1), "autotune");
    cudaEventElapsedTime(&ms, e0, e1);
    return VIBE_OK;
  };
  // times the current L; ms = 0 marks a rejected candidate
  auto time_once = [&](float& ms) -> int {
    int r = ws.ensure(L, q.B, q.soft != nullptr);
    if (r != VIBE_OK) return r;
    float first = 0.f;
    if ((r = timed(first)) != VIBE_OK) return r;
    if (first > 2.f * best) { ms = 0.f; return VIBE_OK; }
    if ((r = timed(ms)) != VIBE_OK) return r;
    if (ms < best) { best = ms; keep = L; }
    return VIBE_OK;
  };
  // one BP grid knob: the occupancy maximum and two fractions of it; leaves the fastest in cfg.
  // dropped: the first candidate was rejected
  auto grid_search = [&](int& cfg, bool& dropped) -> int {
    const int mx = cfg;
    const int cand[] = {mx, (mx * 3 + 3) / 4, (mx + 1) / 2};
    int pick = mx;
    float pick_ms = 1e30f;
    dropped = false;
    for (int i = 0; i < 3; ++i) {
      if (i > 0 && std::max(1, cand[i]) == std::max(1, cand[i - 1])) continue;
      cfg = std::max(1, cand[i]);
      float ms = 0.f;
      const int r = time_once(ms);
      if (r != VIBE_OK) return r;
      if (ms == 0.f && i == 0) { dropped = true; break; }
      if (ms > 0.f && ms < pick_ms) { pick_ms = ms; pick = cfg; }
    }
    cfg = pick;
    return VIBE_OK;
  };
  for (int pm = 1; pm >= 0 && rc == VIBE_OK; --pm) {
    L = base;
    L.pair_mode = pm;
    bool dropped = false;
    if (L.warp_engine()) rc = grid_search(L.bp_blocks_per_sm, dropped);
    if (rc == VIBE_OK && !dropped && L.cta_engine()) rc = grid_search(L.bpx_blocks_per_sm, dropped);
  }
  const int nts[] = {64, 128, 256};
  for (int ni = 0; ni < 3 && rc == VIBE_OK; ++ni) {
    L = keep;
    L.lsd_threads = nts[ni];
    int mx = 0;
    if (vibe::lsd_occupancy(L.bnd, L.ndem, nts[ni], &mx) != cudaSuccess || mx < 1) {
      cudaGetLastError();
      continue;
    }
    const int cand[] = {mx, std::max(1, mx / 2)};
    for (int i = 0; i < 2 && rc == VIBE_OK; ++i) {
      if (i > 0 && cand[1] == cand[0]) continue;
      L.lsd_blocks_per_sm = cand[i];
      float ms = 0.f;
      rc = time_once(ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L = rc == VIBE_OK ? keep : base;
  best_ms = best;
  return rc;
}

}  // namespace

struct vibe_handle {
  int device = 0;
  Tables t{};                 // host copy of the problem descriptor
  Tables* d_desc = nullptr;   // device copy
  Launch L;
  Workspace ws;
  Profiler prof;
  // resident tables
  int32_t *rowptr = nullptr, *colidx = nullptr, *colptr = nullptr, *rowidx = nullptr;
  int32_t *lrowptr = nullptr, *lcolidx = nullptr, *nlev = nullptr;
  uint32_t *csc_ent = nullptr, *sched = nullptr, *lvl_off = nullptr, *perm = nullptr;
  float* lam = nullptr;
  float* alpha_m = nullptr;
  void* msg_init = nullptr;
  uint32_t *xcol = nullptr, *xrmap = nullptr;
  uint2* xrec = nullptr;
  int32_t *layer_ptr = nullptr, *layer_chk = nullptr, *layer_vptr = nullptr, *layer_var = nullptr,
          *nlayer_d = nullptr;
  float4* xsum = nullptr;
  unsigned long long* tmp_counters = nullptr;
  // host-buffer staging
  long long stage_cap = 0;
  uint32_t *st_syn = nullptr, *st_corr = nullptr, *st_log = nullptr, *st_obs = nullptr;
  vibe_shot_stats* st_stats = nullptr;

  void release_stage() {
    cudaFree(st_syn); cudaFree(st_corr); cudaFree(st_log); cudaFree(st_obs); cudaFree(st_stats);
    st_syn = st_corr = st_log = st_obs = nullptr; st_stats = nullptr; stage_cap = 0;
  }
  ~vibe_handle() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    ws.release();
    release_stage();
    cudaFree(tmp_counters);
    cudaFree(rowptr); cudaFree(colidx); cudaFree(colptr); cudaFree(rowidx); cudaFree(lrowptr); cudaFree(lcolidx);
    cudaFree(nlev); cudaFree(csc_ent); cudaFree(sched); cudaFree(lvl_off); cudaFree(perm); cudaFree(lam); cudaFree(alpha_m);
    cudaFree(msg_init); cudaFree(xcol); cudaFree(xrec); cudaFree(xrmap); cudaFree(xsum); cudaFree(d_desc);
    cudaFree(layer_ptr); cudaFree(layer_chk); cudaFree(layer_vptr); cudaFree(layer_var); cudaFree(nlayer_d);
    cudaSetDevice(prev);
  }
};

struct vibe_batch {
  int device = 0;
  std::vector<vibe_handle*> hs;
  Tables* d_desc = nullptr;
  Launch L;
  Workspace ws;
  Profiler prof;
  ~vibe_batch() {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    ws.release();
    cudaFree(d_desc);
    cudaSetDevice(prev);
  }
};

namespace vibe {

int handle_view(const vibe_handle* h, HandleView* v) {
  if (!h || !v) return fail(VIBE_ERR_INVALID, "NULL handle");
  v->t = h->t;
  v->d_desc = h->d_desc;
  v->bnd = h->L.bnd;
  v->device = h->device;
  v->num_sms = h->L.num_sms;
  v->msg_fp16 = h->L.msg_fp16;
  v->bp_grid = h->L.bp_grid();
  v->lsd_grid = h->L.lsd_grid();
  return VIBE_OK;
}

int set_error(int code, const char* msg) { return fail(code, "%s", msg); }

}  // namespace vibe

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
  if (p->bp_engine < VIBE_ENGINE_AUTO || p->bp_engine > VIBE_ENGINE_SUMMARY)
    return fail(VIBE_ERR_INVALID, "bp_engine must be VIBE_ENGINE_AUTO, _IMAGE or _SUMMARY");
  if (p->n_flood < 0 || p->n_flood > K) return fail(VIBE_ERR_INVALID, "n_flood must be in 0..K");
  if (p->pair_mode != 0 && p->pair_mode != 1) return fail(VIBE_ERR_INVALID, "pair_mode must be 0 or 1");
  if (p->n_layered < 0 || p->n_layered > K - p->n_flood)
    return fail(VIBE_ERR_INVALID, "n_layered must be in 0..K - n_flood");
  const bool other_schedules = p->n_flood > 0 || p->n_layered > 0;
  if (other_schedules && p->bp_engine == VIBE_ENGINE_SUMMARY)
    return fail(VIBE_ERR_UNSUPPORTED, "flooding and layered members run on the image engine only");
  if (p->member_alpha)
    for (int i = 0; i < K; ++i)
      if (!(p->member_alpha[i] > 0.f && p->member_alpha[i] <= 1.f))
        return fail(VIBE_ERR_INVALID, "member_alpha[%d] must be in (0, 1]", i);
  for (int j = 0; j < n; ++j)
    if (!(priors[j] > 0.0 && priors[j] < 0.5)) return fail(VIBE_ERR_INVALID, "prior %d = %g outside (0, 0.5)", j, priors[j]);
  if (n >= (1 << 23)) return fail(VIBE_ERR_UNSUPPORTED, "n must be below 2^23");
  if (m > 16384) return fail(VIBE_ERR_UNSUPPORTED, "m must be at most 16384");
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
  h->L.device = h->device;
  if ((e = cudaDeviceGetAttribute(&h->L.num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
    return bail(cuda_fail(e, "device query"));
  h->L.msg_fp16 = p->msg_fp16;
  h->L.pair_mode = p->pair_mode;
  Tables& t = h->t;
  t.m = m; t.n = n; t.k = k; t.E = E; t.K = K;
  t.RP = std::max(8, (maxrow + 7) / 8 * 8);
  t.DP = maxcol <= 4 ? 4 : maxcol <= 8 ? 8 : maxcol <= 16 ? 16 : 32;
  t.mw = (m + 31) / 32; t.nw = (n + 31) / 32; t.kw = (k + 31) / 32; t.W = t.mw;
  t.T = p->max_iter; t.M = p->M; t.lsd_order = p->lsd_order; t.alpha = p->alpha; t.n_flood = p->n_flood;
  t.n_layered = p->n_layered;
  vibe::bp_warp_smem_bytes(&t, p->msg_fp16);
  t.XD = vibe::bpx_degree_bucket(maxcol);
  t.XP = (t.XD + 3) / 4 * 4;
  vibe::bpx_layout(&t, p->msg_fp16);
  t.engine = p->bp_engine;
  if (t.engine == VIBE_ENGINE_SUMMARY && t.XD == 0)
    return bail(fail(VIBE_ERR_UNSUPPORTED, "the summary engine takes columns of at most 16 checks"));
  if (t.engine == VIBE_ENGINE_AUTO) {
    // the image engine when its per-warp image leaves at least 8 warps per SM, else the summary engine
    int optin = 0, blocks = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    t.engine = VIBE_ENGINE_IMAGE;
    const Bounds bw = bounds_over(&t, 1);
    t.engine = VIBE_ENGINE_SUMMARY;
    if (vibe::bp_cta_smem_bytes(bw, 0) <= (size_t)optin &&
        vibe::bp_occupancy(bw, 0, p->msg_fp16, &blocks) == cudaSuccess &&
        (blocks * vibe::kBpWarpsPerCta >= 8 || (other_schedules && blocks >= 1) || (t.XD == 0 && blocks >= 1)))
      t.engine = VIBE_ENGINE_IMAGE;
    if (other_schedules && t.engine != VIBE_ENGINE_IMAGE)
      return bail(fail(VIBE_ERR_UNSUPPORTED,
                       "flooding and layered members need the image engine; the message image does not fit"));
  }
  const int Lnnz = L->rowptr[k];
  const size_t msg_bytes = (size_t)m * t.RP * (p->msg_fp16 ? 2 : 4);
  const size_t lev_scratch = std::max<size_t>(std::max<size_t>(2 * (size_t)n + E, 2 * (size_t)m + 2),
                                              (size_t)K * ((size_t)m + 3 * (size_t)n + 1));
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
  VIBE_TRY(dalloc(&h->alpha_m, K), "tables");
  VIBE_TRY(cudaMalloc(&h->msg_init, std::max<size_t>(msg_bytes, 16)), "tables");
  VIBE_TRY(dalloc(&h->xcol, (size_t)n * t.XP), "tables");
  VIBE_TRY(dalloc(&h->xrec, t.XP ? (size_t)K * n : 0), "tables");
  VIBE_TRY(dalloc(&h->xrmap, t.XP ? (size_t)K * E : 0), "tables");
  VIBE_TRY(dalloc(&h->xsum, m), "tables");
  VIBE_TRY(dalloc(&h->d_desc, 1), "tables");
  if (p->n_layered > 0) {
    VIBE_TRY(dalloc(&h->layer_ptr, (size_t)m + 1), "tables");
    VIBE_TRY(dalloc(&h->layer_chk, (size_t)m), "tables");
    VIBE_TRY(dalloc(&h->layer_vptr, (size_t)m + 1), "tables");
    VIBE_TRY(dalloc(&h->layer_var, (size_t)E), "tables");
    VIBE_TRY(dalloc(&h->nlayer_d, 1), "tables");
  }
  VIBE_TRY(dalloc(&scratch, lev_scratch), "tables");
  VIBE_TRY(dalloc(&h->tmp_counters, VIBE_NUM_COUNTERS), "tables");
  VIBE_TRY(cudaMemcpyAsync(h->rowptr, H->rowptr, sizeof(int32_t) * (m + 1), cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->colidx, H->colidx, sizeof(int32_t) * std::max(E, 0), cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->lrowptr, L->rowptr, sizeof(int32_t) * (k + 1), cudaMemcpyHostToDevice, s), "upload");
  if (Lnnz > 0)
    VIBE_TRY(cudaMemcpyAsync(h->lcolidx, L->colidx, sizeof(int32_t) * Lnnz, cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaMemcpyAsync(h->lam, lam.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s), "upload");
  std::vector<float> alpha_m(K, p->alpha);
  if (p->member_alpha) std::copy(p->member_alpha, p->member_alpha + K, alpha_m.begin());
  VIBE_TRY(cudaMemcpyAsync(h->alpha_m, alpha_m.data(), sizeof(float) * K, cudaMemcpyHostToDevice, s), "upload");
  if (schedules) {
    VIBE_TRY(cudaMemcpyAsync(h->perm, schedules, sizeof(uint32_t) * (size_t)K * n, cudaMemcpyHostToDevice, s), "upload");
  } else {
    VIBE_TRY(vibe::seeded_schedules(h->perm, n, K, p->seed, s), "schedule kernel");
  }
  VIBE_TRY(vibe::build_tables(h->rowptr, h->colidx, m, n, K, h->perm, t.RP, t.DP, t.XP, p->msg_fp16, h->lam,
                              h->colptr, h->rowidx, h->csc_ent, h->msg_init, h->sched, h->lvl_off, h->nlev, h->xcol,
                              h->xrec, h->xrmap, h->xsum, scratch, s),
           "graph builder");
  if (p->n_layered > 0) {
    VIBE_TRY(vibe::build_layers(h->rowptr, h->colidx, h->colptr, h->rowidx, m, h->layer_ptr, h->layer_chk,
                                h->layer_vptr, h->layer_var, h->nlayer_d, scratch, s),
             "layer builder");
    VIBE_TRY(cudaMemcpyAsync(&t.nlayer, h->nlayer_d, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "layer builder");
    VIBE_TRY(cudaStreamSynchronize(s), "layer builder");
    t.layer_ptr = h->layer_ptr; t.layer_chk = h->layer_chk; t.layer_vptr = h->layer_vptr; t.layer_var = h->layer_var;
  }
  t.rowptr = h->rowptr; t.colidx = h->colidx; t.colptr = h->colptr; t.rowidx = h->rowidx;
  t.csc_ent = h->csc_ent; t.lam = h->lam; t.alpha_m = h->alpha_m; t.msg_init = h->msg_init; t.sched = h->sched; t.lvl_off = h->lvl_off;
  t.nlev = h->nlev; t.lrowptr = h->lrowptr; t.lcolidx = h->lcolidx;
  t.xcol = h->xcol; t.xrec = h->xrec; t.xrmap = h->xrmap; t.xsum = h->xsum;
  VIBE_TRY(cudaMemcpyAsync(h->d_desc, &t, sizeof(Tables), cudaMemcpyHostToDevice, s), "upload");
  VIBE_TRY(cudaStreamSynchronize(s), "graph builder");
  cudaFree(scratch);
  scratch = nullptr;
  cudaStreamDestroy(s);
  s = nullptr;
#undef VIBE_TRY
  h->L.one = t;
  h->L.d_desc = h->d_desc;
  h->L.ndem = 1;
  h->L.bnd = bounds_over(&t, 1);
  if ((rc = size_launch(h->L)) != VIBE_OK) return bail(rc);
  h->ws.chunk_max = std::max<long long>(1, (long long)(kWorkspaceBytes / ((size_t)n * 4 + 8)));
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
  const Tables& t = h->t;
  Batch q{nullptr, d_syndromes, t.mw, B, d_corrections, t.nw, d_logical, t.kw, d_stats, d_soft, t.n,
          d_observables, reinterpret_cast<unsigned long long*>(d_counters)};
  return run_decode(h->L, h->ws, h->prof, q, static_cast<cudaStream_t>(stream));
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
    const long long chunk = std::min<long long>(B, h->ws.chunk_max);
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
      Batch q{nullptr, h->st_syn, t.mw, nb, h->st_corr, t.nw, h->st_log, t.kw, h->st_stats, nullptr, t.n,
              h_observables ? h->st_obs : nullptr, h_counters ? h->tmp_counters : nullptr};
      int rc = run_decode(h->L, h->ws, h->prof, q, s);
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

int vibe_get_layers(vibe_handle* h, int32_t* layer_of_check_out, int32_t* nlayer_out) {
  if (!h || h->t.n_layered < 1) return fail(VIBE_ERR_INVALID, "NULL handle or no layered members");
  const Tables& t = h->t;
  if (nlayer_out) *nlayer_out = t.nlayer;
  if (!layer_of_check_out) return VIBE_OK;
  std::vector<int32_t> ptr(t.nlayer + 1), chk(t.m);
  VIBE_CUDA(cudaMemcpy(ptr.data(), h->layer_ptr, sizeof(int32_t) * (t.nlayer + 1), cudaMemcpyDeviceToHost), "layers");
  VIBE_CUDA(cudaMemcpy(chk.data(), h->layer_chk, sizeof(int32_t) * t.m, cudaMemcpyDeviceToHost), "layers");
  for (int l = 0; l < t.nlayer; ++l)
    for (int q = ptr[l]; q < ptr[l + 1]; ++q) layer_of_check_out[chk[q]] = l;
  return VIBE_OK;
}

int vibe_profile(vibe_handle* h, int32_t enable) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  h->prof.on = enable != 0;
  h->prof.used = 0;
  h->prof.bp_launches = 0;
  h->prof.lsd_launches = 0;
  return VIBE_OK;
}

static int profile_read(Profiler& P, double* bp_ms, double* lsd_ms, int64_t* nb, int64_t* nl) {
  double bp = 0.0, lsd = 0.0;
  for (size_t i = 0; i + 3 <= P.used; i += 3) {
    float a = 0.f, b = 0.f;
    VIBE_CUDA(cudaEventSynchronize(P.pool[i + 2]), "profile");
    VIBE_CUDA(cudaEventElapsedTime(&a, P.pool[i], P.pool[i + 1]), "profile");
    VIBE_CUDA(cudaEventElapsedTime(&b, P.pool[i + 1], P.pool[i + 2]), "profile");
    bp += a;
    lsd += b;
  }
  if (bp_ms) *bp_ms = bp;
  if (lsd_ms) *lsd_ms = lsd;
  if (nb) *nb = P.bp_launches;
  if (nl) *nl = P.lsd_launches;
  return VIBE_OK;
}

int vibe_profile_read(vibe_handle* h, double* bp_ms, double* lsd_ms, int64_t* bp_launches, int64_t* lsd_launches) {
  if (!h) return fail(VIBE_ERR_INVALID, "NULL handle");
  return profile_read(h->prof, bp_ms, lsd_ms, bp_launches, lsd_launches);
}

// Moves handle h to BP engine `engine` (descriptor on the device, bounds, launch sizes); the handle is
// unchanged if the engine cannot run this problem.
static int set_engine(vibe_handle* h, int engine) {
  if (engine == VIBE_ENGINE_SUMMARY && (h->t.n_flood > 0 || h->t.n_layered > 0))
    return fail(VIBE_ERR_UNSUPPORTED, "flooding and layered members run on the image engine only");
  if (engine == VIBE_ENGINE_SUMMARY && h->t.XD == 0)
    return fail(VIBE_ERR_UNSUPPORTED, "the summary engine takes columns of at most 16 checks");
  Tables t = h->t;
  t.engine = engine;
  Launch L = h->L;
  L.one = t;
  L.bnd = bounds_over(&t, 1);
  int rc = size_launch(L);
  if (rc != VIBE_OK) return rc;
  VIBE_CUDA(cudaMemcpy(h->d_desc, &t, sizeof(Tables), cudaMemcpyHostToDevice), "engine switch");
  h->t = t;
  h->L = L;
  return VIBE_OK;
}

int vibe_autotune(vibe_handle* h, const uint32_t* d_syndromes, int64_t B, void* stream, int32_t* engine_out,
                  int32_t* bp_blocks_per_sm, int32_t* lsd_blocks_per_sm, int32_t* lsd_threads_out) {
  if (!h || !d_syndromes || B < 1) return fail(VIBE_ERR_INVALID, "NULL handle/syndromes or empty sample");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int start_engine = h->t.engine;
  const Launch start = h->L;
  uint32_t* corr = nullptr;
  VIBE_CUDA(dalloc(&corr, (size_t)B * h->t.nw), "autotune");
  int rc = VIBE_OK;
  float best = 1e30f;
  int best_engine = start_engine;
  Launch best_L = start;
  const int cand_engine[] = {VIBE_ENGINE_IMAGE, VIBE_ENGINE_SUMMARY};
  for (int ci = 0; ci < 2 && rc == VIBE_OK; ++ci) {
    h->L = start;
    if (set_engine(h, cand_engine[ci]) != VIBE_OK) continue;   // the problem does not fit this engine
    const Tables& t = h->t;
    Batch q{nullptr, d_syndromes, t.mw, B, corr, t.nw, nullptr, t.kw, nullptr, nullptr, t.n, nullptr, nullptr};
    float ms = 0.f;
    if ((rc = tune_launch(h->L, h->ws, h->prof, q, s, ms)) != VIBE_OK) break;
    if (ms < best) { best = ms; best_engine = cand_engine[ci]; best_L = h->L; }
  }
  cudaFree(corr);
  h->L = start;
  if (rc != VIBE_OK) {
    set_engine(h, start_engine);
    return rc;
  }
  if ((rc = set_engine(h, best_engine)) != VIBE_OK) return rc;
  h->L = best_L;   // same engine, so the same problem descriptor and bounds
  if (engine_out) *engine_out = best_engine;
  if (bp_blocks_per_sm) *bp_blocks_per_sm = h->L.warp_engine() ? h->L.bp_blocks_per_sm : h->L.bpx_blocks_per_sm;
  if (lsd_blocks_per_sm) *lsd_blocks_per_sm = h->L.lsd_blocks_per_sm;
  if (lsd_threads_out) *lsd_threads_out = h->L.lsd_threads;
  return VIBE_OK;
}

int vibe_get_launch(const vibe_handle* h, const vibe_batch* b, vibe_launch* out) {
  if ((!h) == (!b) || !out) return fail(VIBE_ERR_INVALID, "give exactly one of handle and batch, and an output");
  const Launch& L = h ? h->L : b->L;
  out->engines = L.bnd.engines;
  out->pair_mode = L.pair_mode;
  out->bp_blocks_per_sm = L.warp_engine() ? L.bp_blocks_per_sm : 0;
  out->bpx_blocks_per_sm = L.cta_engine() ? L.bpx_blocks_per_sm : 0;
  out->lsd_blocks_per_sm = L.lsd_blocks_per_sm;
  out->lsd_threads = L.lsd_threads;
  out->num_sms = L.num_sms;
  return VIBE_OK;
}

int vibe_destroy(vibe_handle* h) {
  delete h;
  return VIBE_OK;
}

int vibe_batch_create(vibe_handle* const* handles, int32_t count, vibe_batch** out) {
  if (!out) return fail(VIBE_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!handles || count < 1 || count > vibe::kMaxDems)
    return fail(VIBE_ERR_INVALID, "need 1..%d handles", vibe::kMaxDems);
  for (int i = 0; i < count; ++i)
    if (!handles[i]) return fail(VIBE_ERR_INVALID, "handle %d is NULL", i);
  const vibe_handle* h0 = handles[0];
  std::vector<Tables> desc(count);
  for (int i = 0; i < count; ++i) {
    const vibe_handle* h = handles[i];
    if (h->device != h0->device) return fail(VIBE_ERR_INVALID, "handles live on different devices");
    if (h->L.msg_fp16 != h0->L.msg_fp16) return fail(VIBE_ERR_INVALID, "handles mix FP16 and FP32 messages");
    desc[i] = h->t;
  }
  const Bounds b = bounds_over(desc.data(), count);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != h0->device)
    return fail(VIBE_ERR_INVALID, "the handles' device must be current");
  vibe_batch* bt = new (std::nothrow) vibe_batch();
  if (!bt) return fail(VIBE_ERR_NOMEM, "host allocation failed");
  bt->device = h0->device;
  bt->hs.assign(handles, handles + count);
  cudaError_t e;
  if ((e = dalloc(&bt->d_desc, count)) != cudaSuccess) { delete bt; return cuda_fail(e, "batch"); }
  if ((e = cudaMemcpy(bt->d_desc, desc.data(), sizeof(Tables) * count, cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete bt;
    return cuda_fail(e, "batch");
  }
  bt->L.mixed = true;
  bt->L.d_desc = bt->d_desc;
  bt->L.ndem = count;
  bt->L.bnd = b;
  bt->L.msg_fp16 = h0->L.msg_fp16;
  bt->L.pair_mode = h0->L.pair_mode;
  bt->L.device = h0->device;
  bt->L.num_sms = h0->L.num_sms;
  int rc = size_launch(bt->L);
  if (rc != VIBE_OK) { delete bt; return rc; }
  bt->ws.chunk_max = std::max<long long>(1, (long long)(kWorkspaceBytes / ((size_t)b.n * 4 + 8)));
  *out = bt;
  return VIBE_OK;
}

int vibe_batch_decode(vibe_batch* b, const int32_t* d_problem, const uint32_t* d_syndromes, int32_t syn_stride,
                      int64_t B, uint32_t* d_corrections, int32_t corr_stride, uint32_t* d_logical, int32_t log_stride,
                      vibe_shot_stats* d_stats, const uint32_t* d_observables, uint64_t* d_counters, void* stream) {
  if (!b) return fail(VIBE_ERR_INVALID, "NULL batch");
  if (B < 0) return fail(VIBE_ERR_INVALID, "negative batch");
  if (B == 0) return VIBE_OK;
  if (!d_problem || !d_syndromes || !d_corrections) return fail(VIBE_ERR_INVALID, "NULL problem ids, syndromes or corrections");
  if (B > 0x7fffffffLL) return fail(VIBE_ERR_INVALID, "batch too large");
  if (syn_stride < b->L.bnd.W || corr_stride < b->L.bnd.nw || ((d_logical || d_observables) && log_stride < b->L.bnd.kw))
    return fail(VIBE_ERR_INVALID, "strides smaller than the largest problem's words");
  Batch q{d_problem, d_syndromes, syn_stride, B, d_corrections, corr_stride, d_logical, log_stride, d_stats, nullptr,
          b->L.bnd.n, d_observables, reinterpret_cast<unsigned long long*>(d_counters)};
  return run_decode(b->L, b->ws, b->prof, q, static_cast<cudaStream_t>(stream));
}

int vibe_batch_autotune(vibe_batch* b, const int32_t* d_problem, const uint32_t* d_syndromes, int32_t syn_stride,
                        int64_t B, void* stream) {
  if (!b || !d_problem || !d_syndromes || B < 1) return fail(VIBE_ERR_INVALID, "NULL batch/inputs or empty sample");
  if (B > 0x7fffffffLL) return fail(VIBE_ERR_INVALID, "sample too large");
  if (syn_stride < b->L.bnd.W) return fail(VIBE_ERR_INVALID, "syndrome stride smaller than the largest problem's words");
  uint32_t* corr = nullptr;
  VIBE_CUDA(dalloc(&corr, (size_t)B * b->L.bnd.nw), "autotune");
  Batch q{d_problem, d_syndromes, syn_stride, B, corr, b->L.bnd.nw, nullptr, b->L.bnd.kw, nullptr, nullptr,
          b->L.bnd.n, nullptr, nullptr};
  float ms = 0.f;
  const int rc = tune_launch(b->L, b->ws, b->prof, q, static_cast<cudaStream_t>(stream), ms);
  cudaFree(corr);
  return rc;
}

int vibe_batch_destroy(vibe_batch* b) {
  delete b;
  return VIBE_OK;
}

}  // extern "C"
