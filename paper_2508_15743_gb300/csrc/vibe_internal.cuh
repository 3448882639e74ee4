// Internal declarations shared by the CUDA translation units of libvibe.so.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "vibe.h"

namespace vibe {

constexpr int kBpWarpsPerCta = 2;   // image engine: warps per CTA, one shot per warp
constexpr int kBpxWarpsPerCta = 1;  // summary engine: warps per CTA, one shot per warp
constexpr int kLsdThreads = 128;    // LSD kernel: default threads per CTA (64, 128 or 256), one shot per CTA
constexpr int kMaxRowDeg = 255;     // position of an edge inside its check row fits in 8 bits
constexpr int kMaxColDeg = 32;
constexpr int kMaxDems = 64;        // decoding problems in one mixed launch
constexpr int kMaxDevices = 64;
constexpr uint32_t kFull = 0xffffffffu;

// Position of slot `slot` of check row c inside the message image. A row is RP slots stored as
// 16-byte chunks of `spc` slots (4 for float, 8 for half). When the row has 2, 4 or 8 chunks their
// order is XOR-swizzled by the row index so that the same chunk of consecutive rows falls on all
// eight 16-byte bank groups of shared memory (rows are read by lanes at random, one 16-byte load per
// chunk). Used by the builder only; the BP kernel reads positions from csc_ent.
__host__ __device__ inline uint32_t row_position(uint32_t c, uint32_t slot, int RP, int spc) {
  const int nchunk = RP / spc;
  const uint32_t sw = (nchunk == 2 || nchunk == 4 || nchunk == 8) ? (c * (uint32_t)nchunk / 8u) % (uint32_t)nchunk : 0u;
  return slot ^ (sw * (uint32_t)spc);
}

// Packed csc_ent entry: check << 9 | position of the edge in the check's row of the message image.
__host__ __device__ inline uint32_t csc_entry(uint32_t c, uint32_t slot, int RP, int spc) {
  return (c << 9) | row_position(c, slot, RP, spc);
}

// One decoding problem as the kernels see it: sizes, decoder parameters, the BP shared-memory layout
// of one warp, and the device-resident tables (owned by the handle). Plain data, copied to the device.
struct Tables {
  int m, n, k, E, K;
  int RP;        // row pitch of the padded message image: max row degree rounded up to 8
  int DP;        // column pitch of csc_ent: max column degree rounded up to 4 (4, 8, 16 or 32)
  int mw, nw, kw;
  int W;         // words of a bit vector over the checks: ceil(m/32)
  int T, M, lsd_order;
  int n_flood;   // members 0 .. n_flood-1 run the parallel (flooding) schedule
  int n_layered; // members n_flood .. n_flood+n_layered-1 run the layered schedule
  int nlayer;    // check layers of the layered schedule (0 unless n_layered > 0)
  float alpha;   // the shared factor (alpha_m holds the one each member uses)
  int off_msg, off_dec, off_s, off_par, off_cand, warp_smem;   // image engine: per-warp shared memory, bytes
  int off_cv;    // image engine: float image of check-to-variable messages (layered members, flooding
                 // members with FP16 storage), laid out like the message image; -1 when unused
  int engine;    // VIBE_ENGINE_IMAGE or VIBE_ENGINE_SUMMARY
  // summary engine: column-degree bound XD (4, 6, 8 or 16; 0 when a column has more than 16 checks and
  // the engine cannot run the problem), xcol pitch XP, shared memory of one warp (the m check
  // summaries, bytes) and the parts of one warp's global scratch (bytes, 16-aligned)
  int XD, XP, x_warp_smem;   // x_warp_smem: the m check summaries only
  // xg_cpost = x_warp_scratch: the M*n candidate posteriors (soft output only) follow the fixed part
  long long xg_msg, xg_st, xg_dec, xg_lpost, xg_acc, xg_cand, xg_cpost, x_warp_scratch;
  const int32_t* rowptr;   // H CSR
  const int32_t* colidx;
  const int32_t* colptr;   // H CSC, checks ascending in each column
  const int32_t* rowidx;
  const uint32_t* csc_ent; // n*DP: csc_entry() of each edge, ascending check, zero padded
  const float* lam;        // n prior LLRs
  const float* alpha_m;    // K scaling factors, member i's in alpha_m[i]
  const void* msg_init;    // m*RP messages (float or half): lambda of the edge's column, +inf padding
  const uint32_t* sched;   // K*n: column | (degree << 24), grouped by wavefront level
  const uint32_t* lvl_off; // K*(n+1): level offsets into sched
  const int32_t* nlev;     // K level counts
  const int32_t* lrowptr;  // L CSR
  const int32_t* lcolidx;
  // layered schedule (only when n_layered > 0)
  const int32_t* layer_ptr;   // nlayer+1 offsets into layer_chk
  const int32_t* layer_chk;   // m checks grouped by layer, ascending within a layer
  const int32_t* layer_vptr;  // nlayer+1 offsets into layer_var
  const int32_t* layer_var;   // E: per layer, the columns of its checks in layer_chk order (each at most once)
  // summary engine
  const uint32_t* xcol;    // n*XP: (check << 8) | position of the edge in the check's CSR row, ascending check
  const uint2* xrec;       // K*n: (sched entry, offset of the column's first message in the member's
                           // schedule-ordered message array), same order as sched
  const uint32_t* xrmap;   // K*E: per member, the message slot of each CSR entry of H
  const float4* xsum;      // m: summaries of the prior messages (see vibe_bpx.cu)
};

// Sizes that bound every problem of a launch (shared-memory layouts, strides, scratch pitches).
struct Bounds {
  int m, n, W, nw, kw, M, DP;
  int RP;          // common row pitch if all problems share it, else 0
  int warp_smem;   // largest BP per-warp layout
  int lsd_order;   // largest LSD order
  int x_warp_smem;    // summary-engine shared memory per warp: the prefetch ring for XD and the largest
                      // problem's check summaries (0 if no problem uses that engine)
  long long x_warp_scratch;   // largest summary-engine global scratch per warp, bytes
  int engines;     // bit 0: some problem uses the image engine, bit 1: the summary engine
  int XD;          // largest summary-engine column-degree bound
  int K;           // largest ensemble size
};

struct BpArgs {
  Tables one;                  // the problem of every shot when dem_of_shot is NULL
  const Tables* dems;          // device array of ndem problems (mixed launches)
  int ndem;
  const int32_t* dem_of_shot;  // problem of each shot (mixed launch), or NULL
  Bounds bnd;
  int want_soft;
  int flag_bad;                // this kernel reports shots whose problem index is out of range
  // batch (one chunk); strides in 32-bit words, soft stride in floats
  const uint32_t* syn;
  int syn_stride;
  uint32_t nshots;
  uint32_t* corr;
  int corr_stride;
  uint32_t* logical;
  int log_stride;
  vibe_shot_stats* stats;
  float* soft;
  int soft_stride;
  const uint32_t* obs;
  unsigned long long* counters;
  // work distribution and hand-off to LSD
  unsigned int* next_shot;
  unsigned int* lsd_count;
  uint32_t* lsd_shots;         // queued shots, as lsd_shot_base + the shot's index in this launch
  float* lsd_soft;             // pitch bnd.n floats per queued shot
  uint32_t lsd_shot_base;      // this launch's first shot within the LSD launch that follows
  // image engine, per-warp global scratch: n floats (LLR accumulator), n floats (posterior), M*n floats
  // (candidate posteriors, only with want_soft); pitch in floats
  float* scratch;
  long long scratch_pitch;
  // summary engine, per-warp global scratch (Tables::xg_* offsets); pitch in bytes
  unsigned char* xscratch;
  long long xscratch_pitch;
  unsigned int* next_shot_x;   // the summary engine's own shot counter
  // pair mode (one warp per (shot, member) pair; see pair_epilogue): when pair_mode is set, pairs
  // q = shot * pair_K + member are taken from next_pair (image engine) or next_pair_x (summary
  // engine) and each shot of the chunk has a slot, its index in the chunk
  int pair_mode;
  int pair_K;                  // members per shot slot: the largest K of the launch
  int* pconv;                  // [slot][pair_K] iteration at which the member converged, 0 if not
  float* pW;                   // [slot][pair_K] weight of a converged member's correction
  uint32_t* pbits;             // [slot][pair_K][bnd.nw] a converged member's correction
  float* pterms;               // [slot][pair_K][bnd.n] LLR^i / ||LLR^i|| of a member that ran T sweeps
  float* ppost;                // [slot][pair_K][bnd.n] a converged member's posterior (soft output), or NULL
  unsigned int* pdone;         // [slot] members finished
  unsigned int* next_pair;
  unsigned int* next_pair_x;
};

struct LsdArgs {
  const Tables* dems;
  int ndem;
  const int32_t* dem_of_shot;
  Bounds bnd;
  int want_soft;
  const uint32_t* syn;
  int syn_stride;
  uint32_t* corr;
  int corr_stride;
  uint32_t* logical;
  int log_stride;
  vibe_shot_stats* stats;
  float* soft;
  int soft_stride;
  const uint32_t* obs;
  unsigned long long* counters;
  const unsigned int* lsd_count;
  const uint32_t* lsd_shots;
  const float* lsd_soft;
  unsigned int* lsd_next;
  // per-CTA global scratch (see lsd_scratch_words)
  uint32_t* scratch;
  long long scratch_pitch; // 32-bit words per CTA
};

// ---- pair mode: one warp per (shot, member) -------------------------------------------------------
//
// The members of a shot run at the same time on different warps. Member i stops before iteration t
// once M members have converged with a smaller (iteration, member) key than (t, i): it can no longer
// be among the first M candidates of the correction limit (Sec. III.D.2 step 3), the only ones that
// count. A member that converges records its correction, its weight W and its iteration; a member
// that runs all T sweeps records LLR^i / ||LLR^i|| (Sec. III.D.2 step 5). The last member of a shot
// to finish applies the same rule as the one-warp-per-shot driver to the records: the candidates are
// the first M converged members in (iteration, member) order, the chosen one the first of them with
// the smallest W; with no candidate, (1/K) times the sum of the recorded terms in member order goes
// to LSD. The outputs are therefore identical to the other driver's.

// Whether member i must stop before iteration t: at least M members converged with a smaller key.
__device__ __forceinline__ bool pair_should_stop(const int* conv, int K, int M, int i, int t, int lane) {
  int cnt = 0;
  for (int j0 = 0; j0 < K; j0 += 32) {
    const int j = j0 + lane;
    const int c = j < K ? *reinterpret_cast<const volatile int*>(conv + j) : 0;
    cnt += __popc(__ballot_sync(kFull, c > 0 && (c < t || (c == t && j < i))));
  }
  return cnt >= M;
}

// Done-count of a pair's shot; the caller that finishes last (returns true) runs the epilogue. All
// of the pair's records must be written before the call.
__device__ __forceinline__ bool pair_finish(unsigned int* done, int K, int lane) {
  __threadfence();
  unsigned int old = 0;
  if (lane == 0) old = atomicAdd(done, 1u);
  old = __shfl_sync(kFull, old, 0);
  __threadfence();
  return old == (unsigned int)(K - 1);
}

// LLR^i / ||LLR^i||_2 of a posterior (Sec. III.D.2 step 5; finite entries only, the norm's sum of
// squares in the canonical order: 32 strided partial sums combined at distances 16 .. 1), added to
// acc[v], which starts from +0 when `first`.
__device__ inline void llr_term_add(const float* post, float* acc, int n, bool first, int lane) {
  float part = 0.0f;
  for (int v = lane; v < n; v += 32) {
    const float x = post[v];
    part = __fadd_rn(part, ((__float_as_uint(x) & 0x7f800000u) != 0x7f800000u) ? __fmul_rn(x, x) : 0.0f);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) part = __fadd_rn(part, __shfl_xor_sync(kFull, part, off));
  const float nrm = __fsqrt_rn(part);
  for (int v = lane; v < n; v += 32) {
    const float x = post[v];
    const bool fin = (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
    const float term = fin ? (nrm == 0.0f ? 0.0f : __fdiv_rn(x, nrm)) : x;
    acc[v] = __fadd_rn(first ? 0.0f : acc[v], term);
  }
}

// The shot's outcome from its members' records (see above). Returns whether the shot's logical flips
// differ from the given observables (warp-uniform).
__device__ inline bool pair_epilogue(const BpArgs& a, const Tables& t, uint32_t shot, int slot, int lane) {
  const int K = t.K, M = t.M, T = t.T, n = t.n, nw = t.nw, kw = t.kw;
  const int* conv = a.pconv + (size_t)slot * a.pair_K;
  const float* Wr = a.pW + (size_t)slot * a.pair_K;
  // rank of each converged member among the converged ones by (iteration, member); candidates have
  // rank < M. Lane l examines members l, l + 32, ...
  int nconv = 0, best = -1, tM = T;
  float bestW = 0.0f;
  int best_rank = 1 << 30;
  for (int j0 = 0; j0 < K; j0 += 32) {
    const int j = j0 + lane;
    const int cj = j < K ? __ldcg(conv + j) : 0;
    int rank = 0;
    for (int q = 0; q < K; ++q) {
      const int cq = __ldcg(conv + q);
      rank += (cq > 0 && (cq < cj || (cq == cj && q < j))) ? 1 : 0;
    }
    const bool cand = cj > 0 && rank < M;
    nconv += __popc(__ballot_sync(kFull, cj > 0));
    if (cand && rank == M - 1) tM = cj;
    if (cand) {
      const float w = __ldcg(Wr + j);
      if (best < 0 || w < bestW || (w == bestW && rank < best_rank)) { best = j; bestW = w; best_rank = rank; }
    }
  }
  // warp reductions: the first minimum of W over the candidates (by rank), and the M-th iteration
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const int ob = __shfl_xor_sync(kFull, best, off), orank = __shfl_xor_sync(kFull, best_rank, off);
    const float ow = __shfl_xor_sync(kFull, bestW, off);
    const int otm = __shfl_xor_sync(kFull, tM, off);
    if (ob >= 0 && (best < 0 || ow < bestW || (ow == bestW && orank < best_rank))) { best = ob; bestW = ow; best_rank = orank; }
    tM = min(tM, otm);
  }
  const int ncand = min(nconv, M);
  uint32_t* out_corr = a.corr + (size_t)shot * a.corr_stride;
  if (ncand > 0) {
    const uint32_t* bits = a.pbits + ((size_t)slot * a.pair_K + best) * a.bnd.nw;
    for (int w = lane; w < nw; w += 32) out_corr[w] = __ldcg(bits + w);
    if (a.want_soft) {
      const float* src = a.ppost + ((size_t)slot * a.pair_K + best) * a.bnd.n;
      float* dst = a.soft + (size_t)shot * a.soft_stride;
      for (int v = lane; v < n; v += 32) dst[v] = __ldcg(src + v);
    }
    uint32_t fail = 0;
    for (int rb = 0; rb < kw; ++rb) {
      const int r = 32 * rb + lane;
      uint32_t par = 0;
      if (r < t.k)
        for (int e = __ldg(t.lrowptr + r); e < __ldg(t.lrowptr + r + 1); ++e) {
          const int j = __ldg(t.lcolidx + e);
          par ^= (__ldcg(bits + (j >> 5)) >> (j & 31)) & 1u;
        }
      const uint32_t word = __ballot_sync(kFull, par != 0);
      if (a.logical && lane == 0) a.logical[(size_t)shot * a.log_stride + rb] = word;
      if (a.obs) fail |= word ^ a.obs[(size_t)shot * a.log_stride + rb];
    }
    if (a.stats && lane == 0) {
      vibe_shot_stats st;
      st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)ncand;
      st.chosen_member = (uint8_t)best; st.iters = (uint16_t)(ncand == M ? tM : T);
      st.largest_cluster = 0; st.n_clusters = 0;
      a.stats[shot] = st;
    }
    return fail != 0u;
  } else {
    // (1/K) sum over the members, in index order from +0, of their recorded terms -> LSD
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(a.lsd_count, 1u);
    q = __shfl_sync(kFull, q, 0);
    if (lane == 0) a.lsd_shots[q] = a.lsd_shot_base + shot;
    float* dst = a.lsd_soft + (size_t)q * a.bnd.n;
    const float kf = (float)K;
    const float* terms = a.pterms + (size_t)slot * a.pair_K * a.bnd.n;
    for (int v = lane; v < n; v += 32) {
      float acc = 0.0f;
      for (int i = 0; i < K; ++i) acc = __fadd_rn(acc, __ldcg(terms + (size_t)i * a.bnd.n + v));
      dst[v] = __fdiv_rn(acc, kf);
    }
    return false;   // LSD decides, and counts, this shot
  }
}

// A handle's resident problem and launch configuration, as other host files see it (vibe_api.cu).
struct HandleView {
  Tables t;                  // host copy of the descriptor
  const Tables* d_desc;      // the same descriptor on the device
  Bounds bnd;
  int device, num_sms, msg_fp16;
  int bp_grid, lsd_grid;
};
int handle_view(const vibe_handle* h, HandleView* v);

// Raises kernel Kern's dynamic shared-memory limit on the current device to at least `smem`. The
// attribute call is made only when the limit must grow, so repeated launches (and launches recorded
// into a CUDA graph after a first decode) make none.
template <auto Kern>
cudaError_t ensure_dyn_smem(size_t smem) {
  static std::mutex mu;
  static int limit[kMaxDevices] = {};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 0 || dev >= kMaxDevices) return cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  std::lock_guard<std::mutex> g(mu);
  if (limit[dev] >= (int)smem) return cudaSuccess;
  err = cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err == cudaSuccess) limit[dev] = (int)smem;
  return err;
}
int set_error(int code, const char* msg);

// K0: graph builder (vibe_graph.cu)
cudaError_t build_tables(const int32_t* d_rowptr, const int32_t* d_colidx, int m, int n, int K, const uint32_t* d_perm,
                         int RP, int DP, int XP, int msg_fp16, const float* d_lam, int32_t* d_colptr, int32_t* d_rowidx,
                         uint32_t* d_csc_ent, void* d_msg_init, uint32_t* d_sched, uint32_t* d_lvl_off, int32_t* d_nlev,
                         uint32_t* d_xcol, uint2* d_xrec, uint32_t* d_xrmap, float4* d_xsum, int32_t* d_scratch,
                         cudaStream_t s);
cudaError_t seeded_schedules(uint32_t* d_perm, int n, int K, uint64_t seed, cudaStream_t s);
// Check layers of the layered schedule (greedy colouring in ascending check order) from the CSR and
// CSC of H: layer_ptr (m+1 entries), layer_chk (m), layer_vptr (m+1), layer_var (E), the layer count in
// *d_nlayer; scratch: 2*m + 2 ints.
cudaError_t build_layers(const int32_t* d_rowptr, const int32_t* d_colidx, const int32_t* d_colptr,
                         const int32_t* d_rowidx, int m, int32_t* d_layer_ptr, int32_t* d_layer_chk,
                         int32_t* d_layer_vptr, int32_t* d_layer_var, int32_t* d_nlayer, int32_t* d_scratch,
                         cudaStream_t s);

// K1: persistent BP + ensemble selection (vibe_bp.cu)
size_t bp_warp_smem_bytes(Tables* t, int msg_fp16);   // fills t's layout fields, returns its size
// ndem: descriptors a mixed launch keeps in shared memory; 0 for a single-problem launch.
size_t bp_cta_smem_bytes(const Bounds& b, int ndem);
cudaError_t launch_bp(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s);
cudaError_t bp_occupancy(const Bounds& b, int ndem, int msg_fp16, int* blocks_per_sm);

// K1': summary-engine BP + ensemble selection (vibe_bpx.cu)
int bpx_degree_bucket(int maxcol);          // XD for a largest column degree (0: above 16)
int bpx_ring_bytes(int XD);                  // per-warp shared-memory prefetch ring of a launch with bound XD
void bpx_layout(Tables* t, int msg_fp16);   // fills t's x_warp_smem and xg_* fields
size_t bpx_cta_smem_bytes(const Bounds& b, int ndem);
cudaError_t launch_bpx(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s);
cudaError_t bpx_occupancy(const Bounds& b, int ndem, int msg_fp16, int* blocks_per_sm);

// K3: LSD (vibe_lsd.cu). The per-column arrays (4 words per column) stay in shared memory up to 6144
// columns and move to the CTA's global scratch above that.
__host__ __device__ inline bool lsd_cols_in_smem(const Bounds& b) { return b.n <= 6144; }
size_t lsd_smem_bytes(const Bounds& b, int ndem);
long long lsd_scratch_words(const Bounds& b, int threads);   // per CTA of `threads` threads
cudaError_t launch_lsd(const LsdArgs& a, int grid, int threads, cudaStream_t s);
cudaError_t lsd_occupancy(const Bounds& b, int ndem, int threads, int* blocks_per_sm);

}  // namespace vibe
