// K1' -- the BP ensemble for problems whose message image does not fit in shared memory (circuit-level
// detector error models: rows of 100-200 entries, E up to ~4e5): the summary engine. Same method, same
// results as the image engine (vibe_bp.cu), which keeps a member's whole message image in shared
// memory; a different layout.
//
// Why a warp per (shot, member). The wavefront levels of a random serial order on these graphs are
// short: a column conflicts with every column of its ~4 checks (~600 others), so a sweep of the d=11
// problem has ~1000 levels of ~32 columns. One warp matches that width and synchronises with
// __syncwarp. In shot mode each warp decodes one shot at a time (persistent, shots from a global
// counter), running the members one after another with the iteration budget of the correction limit
// (Sec. III.D.2); in pair mode each warp takes one (shot, member) pair at a time, and the last member
// of a shot to finish runs the shot's selection and epilogue.
//
// Check-node state: a 16-byte summary per check in shared memory.
//   x, y   the values m1 <= m2 held by up to two "holder" edges of the row (their positions p1, p2
//          inside the check's CSR row, bits 0-7 and 8-15 of w; nh = number of valid holders, bits
//          16-17; a row of fewer than two entries holds a phantom second holder, position 255, +inf)
//   z      a floor F: every entry of the row that is not a holder has magnitude >= F, and the
//          holders' magnitudes are <= F (after a rescan, F is the third smallest magnitude, or +inf)
//   w      also carries the parity of the sign bits of the row's messages (bit 18), the syndrome bit
//          (bit 19) and the check's parity (H e)_c XOR s_c (bit 20).
// The minimum over the row without the edge at position p is then m2 if p == p1 and nh == 2, m1 if
// p != p1 and nh >= 1, and +inf if F is +inf; otherwise (the only remaining holder asks, or no holder
// is left) the row is rescanned first -- lazily, only when a column actually needs the answer. The
// sign product without p is the sign parity XOR the sign of p's own message. Together these are
// exactly the minimum and sign product that Algorithm 1's check update takes over N(c) \ v.
//
// Keeping the summary exact after the edge at position p gets the new magnitude x:
//   p holds m1:   x <= m2: m1 = x;  m2 < x <= F: the holders swap;  x > F: p leaves (nh - 1)
//   p holds m2:   x < m1: the holders swap;  x <= F: m2 = x;  x > F: p leaves
//   otherwise:    x < F: p becomes a holder (an empty slot, or the larger holder is evicted and its
//                 value becomes the floor, or x itself becomes the floor if x >= m2)
// With the floor most holders that grow stay answerable; on circuit-level colour codes this needs
// ~2.5x fewer row rescans per sweep than two holders without a floor (117 vs 296 at d=11).
//
// Messages. A member's variable-to-check messages live in the warp's global scratch in the member's
// schedule order: the columns of one level (and of one 32-column chunk) are consecutive, so a chunk's
// messages form one contiguous block and its stores coalesce. The column update never reads its old
// messages: it needs only their signs, kept with its previous decision in a 32-bit state word per
// schedule position (bit k: sign of the message to its k-th check; bit 31: decision). Messages are
// read only by rescans, through a per-member map from each CSR entry of H to its message slot.
//
// Pipeline: each lane copies the column data (checks with row positions, prior, state word) into a
// shared-memory ring one chunk ahead of its update, and the schedule records that locate it two
// chunks ahead; none of it is written by the chunks in between.
//
// Arithmetic equals the oracle's bit for bit: same per-node operation order (__fadd_rn/__fmul_rn), min
// and sign exact, FP16 storage with -0 stored as +0.
#include <type_traits>

#include "vibe_internal.cuh"

namespace vibe {
namespace {

template <typename MT>
struct XMsg;

template <>
struct XMsg<float> {
  __device__ __forceinline__ static float load(const float* p) { return __ldcg(p); }
  __device__ __forceinline__ static float value(float x) { return x; }
  __device__ __forceinline__ static float round(float x) { return x; }
  __device__ __forceinline__ static float from(float x) { return x; }
};

template <>
struct XMsg<__half> {
  __device__ __forceinline__ static __half load(const __half* p) {
    return __ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p)));
  }
  __device__ __forceinline__ static float value(__half x) { return __half2float(x); }
  // rounds to half, -0 as +0, and returns the stored value as a float
  __device__ __forceinline__ static float round(float x) {
    unsigned short h = __half_as_ushort(__float2half_rn(x));
    if (h == 0x8000u) h = 0;
    return __half2float(__ushort_as_half(h));
  }
  __device__ __forceinline__ static __half from(float x) { return __float2half_rn(x); }   // x already rounded
};

template <typename MT>
__device__ __forceinline__ void store_msg(MT* p, float x) {
  if constexpr (std::is_same<MT, float>::value) __stcs(p, x);
  else __stcs(reinterpret_cast<unsigned short*>(p), __half_as_ushort(__float2half_rn(x)));
}

constexpr uint32_t kInfBits = 0x7f800000u;
constexpr uint32_t kDecBit = 1u << 31;   // decision bit of a column state word

__device__ __forceinline__ uint32_t sign_bit(float x) { return __float_as_uint(x) >> 31; }

__device__ __forceinline__ bool is_finite_bits(float x) { return (__float_as_uint(x) & kInfBits) != kInfBits; }

// Check summaries in registers: float4 {m1, m2, F, w}, w = p1 | p2 << 8 | nh << 16 | sign parity << 18 |
// syndrome << 19 | parity << 20 (see the header comment).
constexpr uint32_t kNhShift = 16, kSgnBit = 1u << 18, kSynBit = 1u << 19, kParBit = 1u << 20;

// Minimum magnitude over the row without the edge at position p; false if the summary cannot answer.
__device__ __forceinline__ bool xquery(const float4 s, uint32_t p, float& out) {
  const uint32_t w = __float_as_uint(s.w);
  const uint32_t nh = (w >> kNhShift) & 3u, p1 = w & 0xffu;
  const bool mine = p == p1;
  out = nh == 2u ? (mine ? s.y : s.x) : (nh == 1u && !mine ? s.x : s.z);
  return nh == 2u || (nh == 1u && !mine) || __float_as_uint(s.z) == kInfBits;   // +inf floor: all others +inf
}

// Whether the edge at position p taking magnitude x can change more than the flags: it holds m1 or
// m2, or it drops below the floor.
__device__ __forceinline__ bool xslow(const float4 s, uint32_t p, float x) {
  const uint32_t w = __float_as_uint(s.w);
  const uint32_t nh = (w >> kNhShift) & 3u;
  return (nh >= 1u && p == (w & 0xffu)) || (nh == 2u && p == ((w >> 8) & 0xffu)) || x < s.z;
}

// The summary after the edge at position p takes magnitude x (the case analysis in the header),
// written as: take p out of the holder list, then put (x, p) back if it stays within the floor --
// a former holder when x <= F, any other edge when x < F -- evicting the larger holder into the
// floor when the list is full.
__device__ __forceinline__ float4 xupdate(const float4 s, uint32_t p, float x) {
  const uint32_t w = __float_as_uint(s.w);
  const uint32_t nh0 = (w >> kNhShift) & 3u, q10 = w & 0xffu, q2 = (w >> 8) & 0xffu;
  const bool is1 = nh0 >= 1u && p == q10, is2 = nh0 == 2u && p == q2;
  const bool was = is1 || is2;
  const float a1 = is1 ? s.y : s.x, a2 = s.y, F = s.z;
  const uint32_t q1 = is1 ? q2 : q10;
  const uint32_t k = nh0 - (was ? 1u : 0u);
  const bool ins = was ? x <= F : x < F;
  const bool lt1 = k == 0u || x < a1;
  const bool lt2 = k <= 1u || x < a2;
  const float n1 = ins && lt1 ? x : a1;
  const uint32_t r1 = ins && lt1 ? p : q1;
  const float n2 = ins ? (lt1 ? a1 : (lt2 ? x : a2)) : a2;
  const uint32_t r2 = ins ? (lt1 ? q1 : (lt2 ? p : q2)) : q2;
  const float nF = ins && k == 2u ? (lt2 ? a2 : x) : F;
  const uint32_t nk = ins ? min(k + 1u, 2u) : k;
  return make_float4(n1, n2, nF, __uint_as_float((w & ~0x3ffffu) | r1 | (r2 << 8) | (nk << kNhShift)));
}

// Shared-memory storage of the summaries. FP32 messages: the float4 itself (16 bytes per check).
// FP16 messages: 8 bytes, {m1 | sign parity << 15 | m2 << 16 | syndrome << 31, F | parity << 15 |
// p1 << 16 | p2 << 24} with every magnitude a binary16 (exact: the magnitudes are those of stored
// binary16 messages) and position 255 for an empty holder slot, from which the holder count follows.
template <typename MT>
struct SumIO;

template <>
struct SumIO<float> {
  float4* v;
  __device__ __forceinline__ float4 load(int c) const { return v[c]; }
  __device__ __forceinline__ void store(int c, float4 s) const { v[c] = s; }
  __device__ __forceinline__ void flip(int c, uint32_t bits) const { reinterpret_cast<uint32_t*>(v + c)[3] ^= bits; }
};

template <>
struct SumIO<__half> {
  uint2* v;
  __device__ __forceinline__ static float hf(uint32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }
  __device__ __forceinline__ static uint32_t hb(float x) { return (uint32_t)__half_as_ushort(__float2half_rn(x)); }
  __device__ __forceinline__ float4 load(int c) const {
    const uint2 a = v[c];
    const uint32_t p1 = (a.y >> 16) & 0xffu, p2 = a.y >> 24;
    const uint32_t nh = (p1 != 255u ? 1u : 0u) + (p2 != 255u ? 1u : 0u);
    const uint32_t w = p1 | (p2 << 8) | (nh << kNhShift) | (((a.x >> 15) & 1u) << 18) | ((a.x >> 31) << 19) |
                       (((a.y >> 15) & 1u) << 20);
    return make_float4(hf(a.x & 0x7fffu), hf((a.x >> 16) & 0x7fffu), hf(a.y & 0x7fffu), __uint_as_float(w));
  }
  __device__ __forceinline__ void store(int c, float4 s) const {
    const uint32_t w = __float_as_uint(s.w);
    const uint32_t nh = (w >> kNhShift) & 3u;
    const uint32_t p1 = nh >= 1u ? (w & 0xffu) : 255u, p2 = nh == 2u ? ((w >> 8) & 0xffu) : 255u;
    v[c] = make_uint2(hb(s.x) | (((w >> 18) & 1u) << 15) | (hb(s.y) << 16) | (((w >> 19) & 1u) << 31),
                      hb(s.z) | (((w >> 20) & 1u) << 15) | (p1 << 16) | (p2 << 24));
  }
  __device__ __forceinline__ void flip(int c, uint32_t bits) const {
    if (bits & kSgnBit) v[c].x ^= 1u << 15;
    if (bits & kParBit) v[c].y ^= 1u << 15;
  }
};

// (value, position) pairs ordered by value, then position
__device__ __forceinline__ bool before(float a, uint32_t ia, float b, uint32_t ib) {
  return a < b || (a == b && ia < ib);
}

struct Top3 {
  float a1, a2, a3;
  uint32_t q1, q2;
  __device__ __forceinline__ void init() {
    a1 = a2 = a3 = __uint_as_float(kInfBits);
    q1 = q2 = 255u;
  }
  __device__ __forceinline__ void insert(float x, uint32_t q) {
    const bool b1 = before(x, q, a1, q1), b2 = before(x, q, a2, q2);
    a3 = b2 ? a2 : fminf(a3, x);
    a2 = b1 ? a1 : (b2 ? x : a2);
    q2 = b1 ? q1 : (b2 ? q : q2);
    a1 = b1 ? x : a1;
    q1 = b1 ? q : q1;
  }
};

// Chunks of column data in flight ahead of the update (1 or 2); schedule records go one chunk further.
constexpr int kAhead = 1;

template <typename MT>
__device__ __forceinline__ SumIO<MT> sum_io(unsigned char* p);
template <>
__device__ __forceinline__ SumIO<float> sum_io<float>(unsigned char* p) { return SumIO<float>{reinterpret_cast<float4*>(p)}; }
template <>
__device__ __forceinline__ SumIO<__half> sum_io<__half>(unsigned char* p) { return SumIO<__half>{reinterpret_cast<uint2*>(p)}; }

// Warp-cooperative rescan of check c, whose CSR row is b .. b + d: the two smallest magnitudes with
// their positions and the third smallest as the floor; the flags are kept.
template <typename MT>
__device__ __forceinline__ void rescan_row(int c, int b, int d, const uint32_t* rmap, const MT* msg,
                                           const SumIO<MT>& S, int lane) {
  uint32_t loc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = lane + 32 * u;
    loc[u] = q < d ? __ldg(rmap + b + q) : 0u;
  }
  Top3 T;
  T.init();
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int q = lane + 32 * u;
    if (q < d) T.insert(fabsf(XMsg<MT>::value(XMsg<MT>::load(msg + loc[u]))), (uint32_t)q);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float b1 = __shfl_xor_sync(kFull, T.a1, off), b2 = __shfl_xor_sync(kFull, T.a2, off);
    const float b3 = __shfl_xor_sync(kFull, T.a3, off);
    const uint32_t r1 = __shfl_xor_sync(kFull, T.q1, off), r2 = __shfl_xor_sync(kFull, T.q2, off);
    T.insert(b1, r1);
    T.insert(b2, r2);
    T.insert(b3, 255u);
  }
  if (lane == 0) {
    const uint32_t w = __float_as_uint(S.load(c).w);
    S.store(c, make_float4(T.a1, T.a2, T.a3, __uint_as_float((w & ~0x3ffffu) | T.q1 | (T.q2 << 8) | (2u << kNhShift))));
  }
}

// What a column update reads besides the check summaries: its schedule record (column, degree, first
// message slot), its checks with their row positions, its prior and its state word. None of it is
// written by the chunks in between, so it is copied into a shared-memory ring with cp.async ahead of
// use: the records of chunk c+2 and the rest of chunk c+1 while chunk c is updated. The copies hold
// no registers, so the warp waits for nothing it does not yet need.
template <int DP>
struct XRing {
  static constexpr int XP = (DP + 3) / 4 * 4;   // words of a column record
  static constexpr int kStwWords = 48;          // the 16-byte blocks covering 32 state words
  static constexpr int kRecSlots = kAhead + 2;   // chunk q's records stay until its update
  static constexpr int kStages = kAhead + 1;
  static constexpr int kRecBytes = kRecSlots * 32 * 8;
  static constexpr int kStageBytes = 32 * XP * 4 + 32 * 4 + kStwWords * 4;
  static constexpr int kBytes = kRecBytes + kStages * kStageBytes;
  unsigned char* base;
  __device__ __forceinline__ uint2* rec(uint32_t q) { return reinterpret_cast<uint2*>(base) + (q % kRecSlots) * 32; }
  __device__ __forceinline__ unsigned char* stage(uint32_t q) { return base + kRecBytes + (q % kStages) * kStageBytes; }
  __device__ __forceinline__ uint32_t* xc(uint32_t q) { return reinterpret_cast<uint32_t*>(stage(q)); }
  __device__ __forceinline__ float* lam(uint32_t q) { return reinterpret_cast<float*>(stage(q) + 32 * XP * 4); }
  __device__ __forceinline__ uint32_t* stw(uint32_t q) {
    return reinterpret_cast<uint32_t*>(stage(q) + 32 * XP * 4 + 32 * 4);
  }
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// cp.async in its plain form with the source size stated (equal to the copy size). Read-only tables
// may be cached in L1 (.ca); the per-warp state words, written through L2 by earlier sweeps, are
// copied with .cg so that no L1 line can be stale.
__device__ __forceinline__ void cp_async_ca4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_ca8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_cg16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A chunk of a sweep: up to 32 consecutive schedule entries [cs, min(cs + 32, e)) of level l, whose
// entries end at e. l == nl marks the end of the sweep.
struct Chunk {
  int l;
  uint32_t cs, e;
};

// The member's level offsets lo[0 .. nl] as the chunk walker needs them, one level at a time: lane l
// holds lo[32k + l] of the current window k and lo[32k + 32 + l] of the next one, loaded 32 levels
// before it is needed, so that starting a level costs a shuffle instead of a dependent global load.
struct LevelWin {
  const uint32_t* lo;
  int nl, k;
  uint32_t cur, nxt;
  __device__ __forceinline__ uint32_t load(int x, int lane) const {
    return x + lane <= nl ? __ldg(lo + x + lane) : 0u;
  }
  __device__ __forceinline__ void start(const uint32_t* lo_, int nl_, int lane) {
    lo = lo_;
    nl = nl_;
    k = 0;
    cur = load(0, lane);
    nxt = load(32, lane);
  }
  // lo[x]; x never decreases and grows by at most one per call (warp-uniform)
  __device__ __forceinline__ uint32_t get(int x, int lane) {
    if (x >= 32 * (k + 1)) {
      ++k;
      cur = nxt;
      nxt = load(32 * (k + 1), lane);
    }
    return __shfl_sync(kFull, cur, x - 32 * k);
  }
};

__device__ __forceinline__ Chunk first_chunk(LevelWin& W, int lane) {
  const uint32_t a = W.get(0, lane);
  return Chunk{0, a, W.get(1, lane)};
}

__device__ __forceinline__ Chunk next_chunk(const Chunk& c, LevelWin& W, int lane) {
  if (c.l >= W.nl) return c;
  if (c.cs + 32 < c.e) return Chunk{c.l, c.cs + 32, c.e};
  return Chunk{c.l + 1, c.e, c.l + 1 < W.nl ? W.get(c.l + 2, lane) : c.e};
}

__device__ __forceinline__ bool in_chunk(const Chunk& c, int nl, int lane) {
  return c.l < nl && c.cs + (uint32_t)lane < c.e;
}

// Per-warp views of the current pair's state.
template <typename MT>
struct XState {
  SumIO<MT> S;       // shared: m check summaries
  MT* msg;           // global: E messages in the member's schedule order
  uint32_t* stw;     // global: n column state words in schedule order
  uint32_t* dec;     // global: nw decision bits in column order
  const uint2* rec;  // the member's schedule records
  const uint32_t* rmap;   // the member's CSR-entry -> message-slot map
};

// Serial-V update of one chunk (lane's column d when active). Returns the lane's change of the number
// of unsatisfied checks.
// The lane's column as the update sees it (read from the ring).
template <int DP>
struct XCol {
  uint32_t v, deg, spos, st;
  float lam;
  uint32_t ent[DP];   // (check << 8) | position in the check's row
};

template <typename MT, int DP>
__device__ __forceinline__ int update_chunk(bool active, const XCol<DP>& d, uint32_t j, const Tables& t, float alpha,
                                            const XState<MT>& X, float* lpost, int lane, uint32_t& my_rescans) {
  // check-to-variable messages from the summaries (Algorithm 1's check update over N(c) \ v)
  float mcv[DP];
  uint32_t need = 0u;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    mcv[k] = 0.0f;
    if (active && (uint32_t)k < d.deg) {
      const float4 s = X.S.load((int)(d.ent[k] >> 8));
      float mn;
      if (!xquery(s, d.ent[k] & 0xffu, mn)) need |= 1u << k;
      const uint32_t w = __float_as_uint(s.w);
      const float mag = __fmul_rn(alpha, mn);
      mcv[k] = (((w >> 18) ^ (w >> 19) ^ (d.st >> k)) & 1u) ? -mag : mag;   // sign parity, syndrome, own sign
    }
  }
  if (__any_sync(kFull, need != 0u)) {
    // rescan every check whose summary could not answer (checks of one level are touched by one
    // column each, so the rows are distinct), then ask again. Row bounds of all of them first.
    int rb[DP], rd[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      rb[k] = 0;
      rd[k] = 0;
      if ((need >> k) & 1u) {
        const int c = (int)(d.ent[k] >> 8);
        rb[k] = __ldg(t.rowptr + c);
        rd[k] = __ldg(t.rowptr + c + 1);
      }
    }
    uint32_t pend = need;
    while (__any_sync(kFull, pend != 0u)) {
      const int k0 = __ffs(pend) - 1;
      uint32_t csel = 0u;
      int bsel = 0, esel = 0;
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        csel = k == k0 ? d.ent[k] >> 8 : csel;
        bsel = k == k0 ? rb[k] : bsel;
        esel = k == k0 ? rd[k] : esel;
      }
      uint32_t bal = __ballot_sync(kFull, pend != 0u);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1u;
        const int b = __shfl_sync(kFull, bsel, src);
        rescan_row<MT>((int)__shfl_sync(kFull, csel, src), b, __shfl_sync(kFull, esel, src) - b, X.rmap, X.msg,
                       X.S, lane);
        ++my_rescans;
      }
      pend &= pend - 1u;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if ((need >> k) & 1u) {
        const float4 s = X.S.load((int)(d.ent[k] >> 8));
        float mn;
        xquery(s, d.ent[k] & 0xffu, mn);
        const uint32_t w = __float_as_uint(s.w);
        const float mag = __fmul_rn(alpha, mn);
        mcv[k] = (((w >> 18) ^ (w >> 19) ^ (d.st >> k)) & 1u) ? -mag : mag;
      }
  }
  if (!active) return 0;
  const uint32_t deg = d.deg;
  float L = d.lam;
#pragma unroll
  for (int k = 0; k < DP; ++k)
    if ((uint32_t)k < deg) L = __fadd_rn(L, mcv[k]);
  const uint32_t e_new = L <= 0.0f ? 1u : 0u;
  const bool flip = e_new != ((d.st & kDecBit) ? 1u : 0u);
  uint32_t st = e_new << 31;
  int dpar = 0;
  float pre = d.lam;   // lambda + m_0 + ... + m_{k-1}, the shared head of every exclusion sum
  MT* out = X.msg + d.spos;
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    if ((uint32_t)k < deg) {
      float a = pre;
#pragma unroll
      for (int k2 = k + 1; k2 < DP; ++k2)
        if ((uint32_t)k2 < deg) a = __fadd_rn(a, mcv[k2]);
      const float x = XMsg<MT>::round(a);
      store_msg<MT>(out + k, x);   // streamed: read again only by rescans
      pre = __fadd_rn(pre, mcv[k]);
      const uint32_t sx = sign_bit(x);
      st |= sx << k;
      // this level's only reader and writer of the check: the full summary update for holders and
      // for edges that drop below the floor, a flag update for the rest
      const int c = (int)(d.ent[k] >> 8);
      const uint32_t p = d.ent[k] & 0xffu;
      const float4 s = X.S.load(c);
      const float ax = fabsf(x);
      const uint32_t fl = ((((d.st >> k) ^ sx) & 1u) ? kSgnBit : 0u) | (flip ? kParBit : 0u);
      if (flip) dpar += (__float_as_uint(s.w) & kParBit) ? -1 : 1;
      if (xslow(s, p, ax)) {
        float4 u = xupdate(s, p, ax);
        u.w = __uint_as_float(__float_as_uint(u.w) ^ fl);
        X.S.store(c, u);
      } else if (fl) {
        X.S.flip(c, fl);
      }
    }
  }
  __stcs(X.stw + j, st);
  if (flip) atomicXor(X.dec + (d.v >> 5), 1u << (d.v & 31));
  if (lpost) lpost[d.v] = L;
  return dpar;
}

// Ring copies for chunk number q. Records: each active lane copies its own 8-byte schedule record.
template <int DP>
__device__ __forceinline__ void issue_rec(XRing<DP>& R, uint32_t q, const Chunk& c, int nl, int lane, const uint2* rec) {
  if (in_chunk(c, nl, lane)) cp_async_ca8(R.rec(q) + lane, rec + c.cs + lane);
}

// Column data: each active lane copies its column's record and prior (its schedule record is in the
// ring already); lanes 0..8 copy the 16-byte blocks that cover the chunk's state words.
template <int DP>
__device__ __forceinline__ void issue_data(XRing<DP>& R, uint32_t q, const Chunk& c, int nl, int lane, const Tables& t,
                                           const uint32_t* stw) {
  if (c.l >= nl) return;
  if (in_chunk(c, nl, lane)) {
    const uint32_t v = R.rec(q)[lane].x & 0xffffffu;
    const uint32_t* src = t.xcol + (size_t)v * t.XP;
    uint32_t* dst = R.xc(q) + lane * XRing<DP>::XP;
#pragma unroll
    for (int b = 0; b < XRing<DP>::XP / 4; ++b)
      if (4 * b < t.XP) cp_async_cg16(dst + 4 * b, src + 4 * b);
    cp_async_ca4(R.lam(q) + lane, t.lam + v);
  }
  const uint32_t first = c.cs & ~3u, end = min(c.cs + 32u, c.e);
  if ((uint32_t)lane < (end - first + 3u) / 4u) cp_async_cg16(R.stw(q) + 4 * lane, stw + first + 4 * lane);
}

template <int DP>
__device__ __forceinline__ void read_col(XRing<DP>& R, uint32_t q, const Chunk& c, int lane, bool act, XCol<DP>& d) {
  if (!act) {
    d.deg = 0u;
    return;
  }
  const uint2 r = R.rec(q)[lane];
  d.v = r.x & 0xffffffu;
  d.deg = r.x >> 24;
  d.spos = r.y;
  d.lam = R.lam(q)[lane];
  d.st = R.stw(q)[(c.cs & 3u) + lane];
  const uint4* src = reinterpret_cast<const uint4*>(R.xc(q) + lane * XRing<DP>::XP);
#pragma unroll
  for (int b = 0; b < XRing<DP>::XP / 4; ++b) {
    const uint4 x = src[b];
    if (4 * b + 0 < DP) d.ent[4 * b + 0] = x.x;
    if (4 * b + 1 < DP) d.ent[4 * b + 1] = x.y;
    if (4 * b + 2 < DP) d.ent[4 * b + 2] = x.z;
    if (4 * b + 3 < DP) d.ent[4 * b + 3] = x.w;
  }
}

// One member (index i) on one shot: initialises the member's state and runs up to `budget` sweeps,
// stopping at the first that leaves H e = s, or before sweep `it` when stop(it) holds. Returns the
// converging sweep (0 if none) and in `ran` the sweeps run; leaves the decisions in X.dec and the
// posterior of the last sweep in lpost when soft output is on or `keep_last` is set and the member
// reached sweep T.
template <typename MT, int DP, typename Stop>
__device__ __forceinline__ int run_member_x(const BpArgs& a, const Tables& t, int i, const uint32_t* syn, int nsyn,
                                            int budget, bool keep_last, XState<MT>& X, unsigned char* base,
                                            float* lpost, int lane, uint32_t& my_iters, uint32_t& my_rescans,
                                            int& ran, Stop stop) {
  const int n = t.n, m = t.m, T = t.T, nw = t.nw;
  X.rec = t.xrec + (size_t)i * n;
  X.rmap = t.xrmap + (size_t)i * t.E;
  // member init: prior summaries with this shot's syndrome (parity = s), prior messages in the
  // member's schedule order, state words and decisions 0
  for (int c = lane; c < m; c += 32) {
    float4 s = __ldg(t.xsum + c);
    const uint32_t sb = (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u;
    s.w = __uint_as_float(__float_as_uint(s.w) | (sb ? (kSynBit | kParBit) : 0u));
    X.S.store(c, s);
  }
  for (int j = lane; j < n; j += 32) {
    const uint2 r = __ldg(X.rec + j);
    const float x = XMsg<MT>::round(__ldg(t.lam + (r.x & 0xffffffu)));
    for (uint32_t k = 0; k < (r.x >> 24); ++k) store_msg<MT>(X.msg + r.y + k, x);
    __stcg(X.stw + j, 0u);
  }
  for (int w = lane; w < nw; w += 32) __stcg(X.dec + w, 0u);
  __syncwarp();
  const uint32_t* lo = t.lvl_off + (size_t)i * (n + 1);
  const int nl = __ldg(t.nlev + i);
  XRing<DP> R{base};
  const float alpha = __ldg(t.alpha_m + i);   // member i's scaling factor
  int unsat = nsyn;
  int conv = 0;
  ran = 0;
  for (int it = 1; it <= budget; ++it) {
    if (stop(it)) break;
    // the posterior is needed after the last possible sweep of a member that may end without
    // converging (LLR average) and, for soft output, after every sweep
    float* lp = (a.want_soft || (it == T && keep_last)) ? lpost : nullptr;
    // the sweep in chunks of up to 32 columns of one level, one column per lane, through the ring:
    // q counts chunks; the records of chunk q+2 and the column data of chunk q+1 are in flight while
    // chunk q is updated
    LevelWin W;
    W.start(lo, nl, lane);
    Chunk c0 = first_chunk(W, lane);
    Chunk c1 = next_chunk(c0, W, lane);
    Chunk c2 = next_chunk(c1, W, lane);
    issue_rec(R, 0u, c0, nl, lane, X.rec);
    issue_rec(R, 1u, c1, nl, lane, X.rec);
    cp_async_commit();
    cp_async_wait<0>();
    issue_data<DP>(R, 0u, c0, nl, lane, t, X.stw);
    cp_async_commit();
    int dpar = 0;
    for (uint32_t q = 0; c0.l < nl; ++q) {
      cp_async_wait<0>();   // chunk q's data and chunk q+1's records
      __syncwarp();
      issue_rec(R, q + 2u, c2, nl, lane, X.rec);
      issue_data<DP>(R, q + 1u, c1, nl, lane, t, X.stw);
      cp_async_commit();
      const bool act = in_chunk(c0, nl, lane);
      XCol<DP> d;
      read_col<DP>(R, q, c0, lane, act, d);
      dpar += update_chunk<MT, DP>(act, d, c0.cs + lane, t, alpha, X, lp, lane, my_rescans);
      __syncwarp();
      c0 = c1;
      c1 = c2;
      c2 = next_chunk(c2, W, lane);
    }
    cp_async_wait<0>();
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) dpar += __shfl_xor_sync(kFull, dpar, off);
    unsat += dpar;
    ++my_iters;
    ran = it;
    if (unsat == 0) { conv = it; break; }
  }
  return conv;
}

// W(e) = sum of lambda_j over e_j = 1, ascending j, of the decisions in dec (every lane folds the same
// sequence); with bits != NULL the decision words are copied there.
__device__ __forceinline__ float decision_weight(const Tables& t, const uint32_t* dec, uint32_t* bits, int lane) {
  const int nw = t.nw;
  if (bits)
    for (int w = lane; w < nw; w += 32) bits[w] = __ldcg(dec + w);
  float W = 0.0f;
  for (int w = 0; w < nw; ++w) {
    uint32_t x = __ldcg(dec + w);
    while (x) {
      const int bpos = __ffs(x) - 1;
      W = __fadd_rn(W, __ldg(t.lam + 32 * w + bpos));
      x &= x - 1;
    }
  }
  return W;
}

// Decodes shot `shot` of problem t with one warp. base: the warp's shared memory; gs: its global
// scratch (messages, state words, decisions, posterior, LLR accumulator, candidate records).
template <typename MT, int DP>
__device__ __forceinline__ void decode_shot_x(const BpArgs& a, const Tables& t, uint32_t shot, unsigned char* base,
                                              unsigned char* gs, int lane, uint32_t& my_iters,
                                              uint32_t& my_shots, uint32_t& my_fail, uint32_t& my_rescans) {
  const int n = t.n, m = t.m, K = t.K, M = t.M, T = t.T, nw = t.nw, kw = t.kw, mw = t.mw;
  XState<MT> X;
  X.S = sum_io<MT>(base + XRing<DP>::kBytes);
  X.msg = reinterpret_cast<MT*>(gs + t.xg_msg);
  X.stw = reinterpret_cast<uint32_t*>(gs + t.xg_st);
  X.dec = reinterpret_cast<uint32_t*>(gs + t.xg_dec);
  float* lpost = reinterpret_cast<float*>(gs + t.xg_lpost);
  float* acc = reinterpret_cast<float*>(gs + t.xg_acc);
  uint32_t* cand = reinterpret_cast<uint32_t*>(gs + t.xg_cand);
  float* cpost = reinterpret_cast<float*>(gs + t.xg_cpost);

  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  int nsyn = 0;
  for (int w = lane; w < mw; w += 32) {
    const int rem = m - 32 * w;
    nsyn += __popc(__ldg(syn + w) & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u)));
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) nsyn += __shfl_xor_sync(kFull, nsyn, off);
  ++my_shots;
  uint32_t* out_corr = a.corr + (size_t)shot * a.corr_stride;

  if (nsyn == 0 && !a.want_soft) {
    // s = 0: every member converges in iteration 1 to e = 0; member 0 is chosen
    for (int w = lane; w < nw; w += 32) out_corr[w] = 0u;
    if (a.logical)
      for (int w = lane; w < kw; w += 32) a.logical[(size_t)shot * a.log_stride + w] = 0u;
    if (a.obs) {
      uint32_t f = 0;
      for (int w = lane; w < kw; w += 32) f |= a.obs[(size_t)shot * a.log_stride + w];
      if (__any_sync(kFull, f) && lane == 0) ++my_fail;
    }
    if (a.stats && lane == 0) {
      vibe_shot_stats st;
      st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)M; st.chosen_member = 0;
      st.iters = 1; st.largest_cluster = 0; st.n_clusters = 0;
      a.stats[shot] = st;
    }
    return;
  }

  // candidate list, lane j holds entry j (sorted by iteration, then member)
  int ncand = 0;
  int c_t = 0, c_i = 0, c_slot = 0;
  float c_W = 0.0f;

  for (int i = 0; i < K; ++i) {
    const int budget = ncand < M ? T : __shfl_sync(kFull, c_t, M - 1) - 1;
    if (budget <= 0) break;
    int ran = 0;
    const int conv = run_member_x<MT, DP>(a, t, i, syn, nsyn, budget, ncand == 0, X, base, lpost, lane, my_iters,
                                          my_rescans, ran, [](int) { return false; });
    if (conv) {
      // insert (conv, i); i exceeds every member already listed, so it goes after equal iterations
      const int p = __popc(__ballot_sync(kFull, lane < ncand && c_t <= conv));
      const int slot = ncand < M ? ncand : __shfl_sync(kFull, c_slot, M - 1);
      const float W = decision_weight(t, X.dec, cand + (size_t)slot * nw, lane);
      if (a.want_soft) {
        float* dst = cpost + (size_t)slot * n;
        for (int v = lane; v < n; v += 32) dst[v] = lpost[v];
      }
      const float uW = __shfl_up_sync(kFull, c_W, 1);
      const int ut = __shfl_up_sync(kFull, c_t, 1), ui = __shfl_up_sync(kFull, c_i, 1);
      const int us = __shfl_up_sync(kFull, c_slot, 1);
      const int last = min(ncand, M - 1);
      if (lane > p && lane <= last) { c_W = uW; c_t = ut; c_i = ui; c_slot = us; }
      if (lane == p) { c_W = W; c_t = conv; c_i = i; c_slot = slot; }
      ncand = min(ncand + 1, M);
    } else if (ncand == 0) {
      // not converged after T sweeps and no candidate yet: add LLR^i / ||LLR^i|| (finite entries)
      llr_term_add(lpost, acc, n, i == 0, lane);
    }
    __syncwarp();
  }

  if (ncand > 0) {
    // first minimum of W over the candidate list
    float bw = lane < ncand ? c_W : __int_as_float(0x7f800000);
    int bi = lane;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      const float ow = __shfl_xor_sync(kFull, bw, off);
      const int oi = __shfl_xor_sync(kFull, bi, off);
      if (ow < bw || (ow == bw && oi < bi)) { bw = ow; bi = oi; }
    }
    const int slot = __shfl_sync(kFull, c_slot, bi);
    const int member = __shfl_sync(kFull, c_i, bi);
    const int iters = ncand == M ? __shfl_sync(kFull, c_t, M - 1) : T;
    const uint32_t* bits = cand + (size_t)slot * nw;
    for (int w = lane; w < nw; w += 32) out_corr[w] = bits[w];
    if (a.want_soft) {
      const float* src = cpost + (size_t)slot * n;
      float* dst = a.soft + (size_t)shot * a.soft_stride;
      for (int v = lane; v < n; v += 32) dst[v] = src[v];
    }
    uint32_t fail = 0;
    for (int rb = 0; rb < kw; ++rb) {
      const int r = 32 * rb + lane;
      uint32_t par = 0;
      if (r < t.k)
        for (int e = __ldg(t.lrowptr + r); e < __ldg(t.lrowptr + r + 1); ++e) {
          const int j = __ldg(t.lcolidx + e);
          par ^= (bits[j >> 5] >> (j & 31)) & 1u;
        }
      const uint32_t word = __ballot_sync(kFull, par != 0);
      if (a.logical && lane == 0) a.logical[(size_t)shot * a.log_stride + rb] = word;
      if (a.obs) fail |= word ^ a.obs[(size_t)shot * a.log_stride + rb];
    }
    if (fail && lane == 0) ++my_fail;
    if (a.stats && lane == 0) {
      vibe_shot_stats st;
      st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)ncand;
      st.chosen_member = (uint8_t)member; st.iters = (uint16_t)iters; st.largest_cluster = 0; st.n_clusters = 0;
      a.stats[shot] = st;
    }
  } else {
    // hand the averaged soft vector to the LSD kernel
    uint32_t q = 0;
    if (lane == 0) q = atomicAdd(a.lsd_count, 1u);
    q = __shfl_sync(kFull, q, 0);
    if (lane == 0) a.lsd_shots[q] = a.lsd_shot_base + shot;
    float* dst = a.lsd_soft + (size_t)q * a.bnd.n;
    const float kf = (float)K;
    for (int v = lane; v < n; v += 32) dst[v] = __fdiv_rn(acc[v], kf);
  }
  __syncwarp();
}

// Pair mode: member i of shot `shot` (slot `slot` of the chunk) with one warp; the last member of the
// shot to finish writes the shot's outcome (pair_epilogue, vibe_internal.cuh).
template <typename MT, int DP>
__device__ __forceinline__ void decode_pair_x(const BpArgs& a, const Tables& t, uint32_t shot, int slot, int i,
                                              unsigned char* base, unsigned char* gs, int lane, uint32_t& my_iters,
                                              uint32_t& my_shots, uint32_t& my_fail, uint32_t& my_rescans) {
  const int K = t.K, M = t.M, T = t.T, n = t.n, m = t.m, mw = t.mw, nw = t.nw, kw = t.kw;
  if (i >= K) return;
  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  int nsyn = 0;
  for (int w = lane; w < mw; w += 32) {
    const int rem = m - 32 * w;
    nsyn += __popc(__ldg(syn + w) & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u)));
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) nsyn += __shfl_xor_sync(kFull, nsyn, off);
  if (nsyn == 0 && !a.want_soft) {
    // s = 0: every member converges in iteration 1 to e = 0; member 0 is chosen -- written by member 0
    if (i != 0) return;
    ++my_shots;
    for (int w = lane; w < nw; w += 32) a.corr[(size_t)shot * a.corr_stride + w] = 0u;
    if (a.logical)
      for (int w = lane; w < kw; w += 32) a.logical[(size_t)shot * a.log_stride + w] = 0u;
    if (a.obs) {
      uint32_t f = 0;
      for (int w = lane; w < kw; w += 32) f |= a.obs[(size_t)shot * a.log_stride + w];
      if (__any_sync(kFull, f) && lane == 0) ++my_fail;
    }
    if (a.stats && lane == 0) {
      vibe_shot_stats st;
      st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)M; st.chosen_member = 0;
      st.iters = 1; st.largest_cluster = 0; st.n_clusters = 0;
      a.stats[shot] = st;
    }
    return;
  }
  if (i == 0) ++my_shots;
  XState<MT> X;
  X.S = sum_io<MT>(base + XRing<DP>::kBytes);
  X.msg = reinterpret_cast<MT*>(gs + t.xg_msg);
  X.stw = reinterpret_cast<uint32_t*>(gs + t.xg_st);
  X.dec = reinterpret_cast<uint32_t*>(gs + t.xg_dec);
  float* lpost = reinterpret_cast<float*>(gs + t.xg_lpost);
  int* conv = a.pconv + (size_t)slot * a.pair_K;
  int ran = 0;
  const int cv = run_member_x<MT, DP>(a, t, i, syn, nsyn, T, true, X, base, lpost, lane, my_iters, my_rescans, ran,
                                      [&](int it) { return pair_should_stop(conv, K, M, i, it, lane); });
  const size_t rec = (size_t)slot * a.pair_K + i;
  if (cv) {
    const float W = decision_weight(t, X.dec, a.pbits + rec * a.bnd.nw, lane);
    if (lane == 0) a.pW[rec] = W;
    if (a.want_soft)
      for (int v = lane; v < n; v += 32) a.ppost[rec * a.bnd.n + v] = lpost[v];
    __threadfence();
    __syncwarp();
    if (lane == 0) *reinterpret_cast<volatile int*>(conv + i) = cv;
  } else if (ran == T) {
    llr_term_add(lpost, a.pterms + rec * a.bnd.n, n, true, lane);
  }
  __syncwarp();
  if (pair_finish(a.pdone + slot, K, lane) && pair_epilogue(a, t, shot, slot, lane) && lane == 0) ++my_fail;
  __syncwarp();
}

// Blocks (one warp each) per SM the register budget targets.
constexpr int kMinBlocksX = 16 / kBpxWarpsPerCta;

// MIXED: shots name their problems (dem_of_shot); the descriptors are copied to shared memory after
// the warps' regions and shots of image-engine problems are left to that kernel. Otherwise every shot
// decodes a.one from the parameter space.
template <typename MT, int DP, bool MIXED>
__global__ void __launch_bounds__(kBpxWarpsPerCta * 32, kMinBlocksX) k_bpx(const BpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wcta = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBpxWarpsPerCta + wcta;
  Tables* sdem = reinterpret_cast<Tables*>(smem + (size_t)kBpxWarpsPerCta * a.bnd.x_warp_smem);
  if (MIXED) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.dems);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sdem);
    const int words = a.ndem * (int)(sizeof(Tables) / 4);
    for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = __ldg(src + q);
    __syncthreads();
  }
  unsigned char* base = smem + (size_t)wcta * a.bnd.x_warp_smem;
  unsigned char* gs = a.xscratch + gw * a.xscratch_pitch;
  uint32_t my_iters = 0, my_shots = 0, my_fail = 0, my_rescans = 0;   // flushed before they could wrap

  if (a.pair_mode) {
    const unsigned long long npairs = (unsigned long long)a.nshots * (unsigned long long)a.pair_K;
    for (;;) {
      unsigned long long q = 0;
      if (lane == 0) q = atomicAdd(a.next_pair_x, 1u);
      q = __shfl_sync(kFull, q, 0);
      if (q >= npairs) break;
      const uint32_t shot = (uint32_t)(q / a.pair_K);
      const int i = (int)(q % a.pair_K);
      if (MIXED) {
        const int di = __ldg(a.dem_of_shot + shot);
        if ((unsigned)di >= (unsigned)a.ndem) {
          if (i != 0 || !a.flag_bad) continue;
          for (int w = lane; w < a.corr_stride; w += 32) a.corr[(size_t)shot * a.corr_stride + w] = 0u;
          if (a.logical)
            for (int w = lane; w < a.log_stride; w += 32) a.logical[(size_t)shot * a.log_stride + w] = 0u;
          if (lane == 0) {
            if (a.stats) {
              vibe_shot_stats st;
              st.status = VIBE_STATUS_BAD_PROBLEM; st.lsd_invoked = 0; st.n_converged = 0; st.chosen_member = 0;
              st.iters = 0; st.largest_cluster = 0; st.n_clusters = 0;
              a.stats[shot] = st;
            }
            if (a.counters) atomicAdd(a.counters + VIBE_CNT_BAD_PROBLEM, 1ull);
          }
          continue;
        }
        if (sdem[di].engine != VIBE_ENGINE_SUMMARY) continue;   // left to the image engine
        decode_pair_x<MT, DP>(a, sdem[di], shot, (int)shot, i, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
      } else {
        decode_pair_x<MT, DP>(a, a.one, shot, (int)shot, i, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
      }
    }
  }
  for (;;) {
    if (a.pair_mode) break;
    if (my_iters > 0x70000000u || my_rescans > 0x70000000u) {
      if (lane == 0 && a.counters) {
        atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, (unsigned long long)my_iters);
        atomicAdd(a.counters + VIBE_CNT_RESCANS, (unsigned long long)my_rescans);
      }
      my_iters = 0;
      my_rescans = 0;
    }
    uint32_t shot = 0;
    if (lane == 0) shot = atomicAdd(a.next_shot_x, 1u);
    shot = __shfl_sync(kFull, shot, 0);
    if (shot >= a.nshots) break;
    if (MIXED) {
      const int di = __ldg(a.dem_of_shot + shot);
      if ((unsigned)di >= (unsigned)a.ndem) {
        if (!a.flag_bad) continue;
        for (int w = lane; w < a.corr_stride; w += 32) a.corr[(size_t)shot * a.corr_stride + w] = 0u;
        if (a.logical)
          for (int w = lane; w < a.log_stride; w += 32) a.logical[(size_t)shot * a.log_stride + w] = 0u;
        if (a.soft)
          for (int j = lane; j < a.soft_stride; j += 32) a.soft[(size_t)shot * a.soft_stride + j] = 0.0f;
        if (lane == 0) {
          if (a.stats) {
            vibe_shot_stats st;
            st.status = VIBE_STATUS_BAD_PROBLEM; st.lsd_invoked = 0; st.n_converged = 0; st.chosen_member = 0;
            st.iters = 0; st.largest_cluster = 0; st.n_clusters = 0;
            a.stats[shot] = st;
          }
          if (a.counters) atomicAdd(a.counters + VIBE_CNT_BAD_PROBLEM, 1ull);
        }
        continue;
      }
      if (sdem[di].engine != VIBE_ENGINE_SUMMARY) continue;   // left to the image engine
      decode_shot_x<MT, DP>(a, sdem[di], shot, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
    } else {
      decode_shot_x<MT, DP>(a, a.one, shot, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
    }
  }
  if (lane == 0 && a.counters) {
    atomicAdd(a.counters + VIBE_CNT_SHOTS, (unsigned long long)my_shots);
    atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, (unsigned long long)my_iters);
    if (my_fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, (unsigned long long)my_fail);
    if (my_rescans) atomicAdd(a.counters + VIBE_CNT_RESCANS, (unsigned long long)my_rescans);
  }
}

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename MT, int DP, bool MIXED>
cudaError_t prefer_shared() {
  // the summaries and the ring are the working set; L1 caches little here
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return cudaSuccess;
  if (done[dev]) return cudaSuccess;
  cudaError_t err = cudaFuncSetAttribute(k_bpx<MT, DP, MIXED>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (err == cudaSuccess) done[dev] = true;
  return err;
}

template <typename MT, int DP, bool MIXED>
cudaError_t launch_x(const BpArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = prefer_shared<MT, DP, MIXED>();
  if (err != cudaSuccess) return err;
  err = ensure_dyn_smem<k_bpx<MT, DP, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  k_bpx<MT, DP, MIXED><<<grid, kBpxWarpsPerCta * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename MT, int DP, bool MIXED>
cudaError_t occupancy_x(size_t smem, int* out) {
  cudaError_t err = prefer_shared<MT, DP, MIXED>();
  if (err != cudaSuccess) return err;
  err = ensure_dyn_smem<k_bpx<MT, DP, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bpx<MT, DP, MIXED>, kBpxWarpsPerCta * 32, smem);
}

template <typename Fn>
cudaError_t by_xd(int XD, Fn&& f) {
  switch (XD) {
    case 4: return f(std::integral_constant<int, 4>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
  }
}

template <typename MT>
cudaError_t launch_x_mt(const BpArgs& a, int grid, cudaStream_t s) {
  const bool mixed = a.dem_of_shot != nullptr;
  const size_t smem = bpx_cta_smem_bytes(a.bnd, mixed ? a.ndem : 0);
  return by_xd(a.bnd.XD, [&](auto dp) {
    if (mixed) return launch_x<MT, decltype(dp)::value, true>(a, grid, smem, s);
    return launch_x<MT, decltype(dp)::value, false>(a, grid, smem, s);
  });
}

template <typename MT>
cudaError_t occupancy_x_mt(const Bounds& b, int ndem, int* out) {
  const size_t smem = bpx_cta_smem_bytes(b, ndem);
  return by_xd(b.XD, [&](auto dp) {
    if (ndem > 0) return occupancy_x<MT, decltype(dp)::value, true>(smem, out);
    return occupancy_x<MT, decltype(dp)::value, false>(smem, out);
  });
}

}  // namespace

int bpx_degree_bucket(int maxcol) {
  return maxcol <= 4 ? 4 : maxcol <= 6 ? 6 : maxcol <= 8 ? 8 : maxcol <= 16 ? 16 : 0;
}

int bpx_ring_bytes(int XD) {
  switch (XD) {
    case 4: return XRing<4>::kBytes;
    case 6: return XRing<6>::kBytes;
    case 8: return XRing<8>::kBytes;
    case 16: return XRing<16>::kBytes;
    default: return 0;
  }
}

void bpx_layout(Tables* t, int msg_fp16) {
  // the check summaries (16 or 8 bytes per check); the prefetch ring comes on top (bounds)
  t->x_warp_smem = (int)a16((msg_fp16 ? 8 : 16) * (size_t)t->m);
  long long g = 0;
  t->xg_msg = g;   g += (long long)a16((size_t)t->E * (msg_fp16 ? 2 : 4));
  t->xg_st = g;    g += (long long)a16(4 * (size_t)t->n);
  t->xg_dec = g;   g += (long long)a16(4 * (size_t)t->nw);
  t->xg_lpost = g; g += (long long)a16(4 * (size_t)t->n);
  t->xg_acc = g;   g += (long long)a16(4 * (size_t)t->n);
  t->xg_cand = g;  g += (long long)a16(4 * (size_t)t->M * t->nw);
  t->xg_cpost = g;
  t->x_warp_scratch = g;
}

size_t bpx_cta_smem_bytes(const Bounds& b, int ndem) {
  return (size_t)kBpxWarpsPerCta * b.x_warp_smem + a16((size_t)ndem * sizeof(Tables));
}

cudaError_t launch_bpx(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s) {
  return msg_fp16 ? launch_x_mt<__half>(a, grid, s) : launch_x_mt<float>(a, grid, s);
}

cudaError_t bpx_occupancy(const Bounds& b, int ndem, int msg_fp16, int* blocks_per_sm) {
  return msg_fp16 ? occupancy_x_mt<__half>(b, ndem, blocks_per_sm) : occupancy_x_mt<float>(b, ndem, blocks_per_sm);
}

}  // namespace vibe
