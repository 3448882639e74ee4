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
constexpr int kLsdThreads = 128;    // LSD kernel: threads per CTA, one LSD shot per CTA at a time
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
  float alpha;   // the shared factor (alpha_m holds the one each member uses)
  int off_msg, off_dec, off_s, off_par, off_cand, warp_smem;   // image engine: per-warp shared memory, bytes
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
  uint32_t* lsd_shots;
  float* lsd_soft;             // pitch bnd.n floats per queued shot
  // image engine, per-warp global scratch: n floats (LLR accumulator), n floats (posterior), M*n floats
  // (candidate posteriors, only with want_soft); pitch in floats
  float* scratch;
  long long scratch_pitch;
  // summary engine, per-warp global scratch (Tables::xg_* offsets); pitch in bytes
  unsigned char* xscratch;
  long long xscratch_pitch;
  unsigned int* next_shot_x;   // the summary engine's own shot counter
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
long long lsd_scratch_words(const Bounds& b);
cudaError_t launch_lsd(const LsdArgs& a, int grid, cudaStream_t s);
cudaError_t lsd_occupancy(const Bounds& b, int ndem, int* blocks_per_sm);

}  // namespace vibe
