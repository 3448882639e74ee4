// K1 -- persistent serial-schedule min-sum BP ensemble with the ensemble selection fused in.
//
// One warp decodes one shot at a time and pulls shots from a global counter until the batch is
// done. For its shot the warp runs the K members one after another (Sec. III.D.2): member i keeps its
// variable-to-check messages in the warp's slice of shared memory, sweeps its dependency wavefronts
// (lanes = columns of one level, which share no check) and stops as soon as H e = s (Algorithm 1).
//
// Correction limit (Sec. III.D.2 step 3). The candidates are the first M converged members in
// (iteration, member) order. Running members in index order, member i can only enter that set by
// converging before the M-th candidate's iteration, so it gets the budget t_M - 1 once M candidates
// exist (T before). Members whose budget is 0 are skipped. This is the lock-step rule of the paper
// without the waiting: every member's trajectory is independent of the others, so the candidate set
// and the chosen correction are identical, and no sweep that cannot change the result is run.
//
// Ranking (step 4): the chosen candidate minimises W(e) = sum over e_j = 1 of lambda_j (float, ascending
// j), ties to the earlier candidate. With no converged member (step 5) the warp accumulates
// LLR^i / ||LLR^i||_2 over all members in index order and hands (1/K) * sum to the LSD kernel.
//
// Arithmetic is the oracle's to the bit: fixed per-node operation order, __fadd_rn/__fmul_rn (no
// contraction), min and sign exact. Stored messages are never -0 (a sum that starts at lambda_v > 0
// cannot round to -0 in FP32; FP16 stores map -0 to +0), so the sign bit of a message equals x < 0.
#include <type_traits>

#include "vibe_internal.cuh"

namespace vibe {
namespace {

template <typename MT>
struct Msg;

template <>
struct Msg<float> {
  // Minimum magnitude (as a float) and XOR of the raw words over 8 slots starting at row8.
  __device__ __forceinline__ static void scan8(const float* row8, float& mn, uint32_t& sg) {
    const float4 a = reinterpret_cast<const float4*>(row8)[0];
    const float4 b = reinterpret_cast<const float4*>(row8)[1];
    const float m01 = fminf(fabsf(a.x), fabsf(a.y)), m23 = fminf(fabsf(a.z), fabsf(a.w));
    const float m45 = fminf(fabsf(b.x), fabsf(b.y)), m67 = fminf(fabsf(b.z), fabsf(b.w));
    mn = fminf(mn, fminf(fminf(m01, m23), fminf(m45, m67)));
    sg ^= __float_as_uint(a.x) ^ __float_as_uint(a.y) ^ __float_as_uint(a.z) ^ __float_as_uint(a.w) ^
          __float_as_uint(b.x) ^ __float_as_uint(b.y) ^ __float_as_uint(b.z) ^ __float_as_uint(b.w);
  }
  __device__ __forceinline__ static uint32_t sign(uint32_t sg) { return sg >> 31; }
  __device__ __forceinline__ static void set_inf(float* p) { *p = __int_as_float(0x7f800000); }
  __device__ __forceinline__ static void store(float* p, float x) { *p = x; }
  __device__ __forceinline__ static float value(float x) { return x; }
  static constexpr int kSpc = 4;   // slots per 16-byte chunk of a row
};

template <>
struct Msg<__half> {
  __device__ __forceinline__ static void scan8(const __half* row8, float& mn, uint32_t& sg) {
    const uint4 q = *reinterpret_cast<const uint4*>(row8);
    const __half2 h0 = __habs2(*reinterpret_cast<const __half2*>(&q.x));
    const __half2 h1 = __habs2(*reinterpret_cast<const __half2*>(&q.y));
    const __half2 h2 = __habs2(*reinterpret_cast<const __half2*>(&q.z));
    const __half2 h3 = __habs2(*reinterpret_cast<const __half2*>(&q.w));
    const __half2 hm = __hmin2(__hmin2(h0, h1), __hmin2(h2, h3));
    mn = fminf(mn, __half2float(__hmin(__low2half(hm), __high2half(hm))));
    const uint32_t x = q.x ^ q.y ^ q.z ^ q.w;
    sg ^= x ^ (x >> 16);
  }
  __device__ __forceinline__ static uint32_t sign(uint32_t sg) { return (sg >> 15) & 1u; }
  __device__ __forceinline__ static void set_inf(__half* p) { *reinterpret_cast<unsigned short*>(p) = 0x7c00u; }
  __device__ __forceinline__ static void store(__half* p, float x) {
    unsigned short h = __half_as_ushort(__float2half_rn(x));
    if (h == 0x8000u) h = 0;
    *reinterpret_cast<unsigned short*>(p) = h;
  }
  __device__ __forceinline__ static float value(__half x) { return __half2float(x); }
  static constexpr int kSpc = 8;
};

__device__ __forceinline__ bool is_finite_bits(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

// One serial-V column update (readings R2, R3 of the oracle): check-to-variable messages from the
// current variable-to-check messages of the other columns, posterior, literal exclusion sums, decision.
// RPC = row pitch in 8-slot chunks (0: read it from the tables).
//
// Exclusion of the column's own message from its check rows: a check is touched by exactly one
// column per wavefront level, so the updating lane owns the row until the level ends. It overwrites
// its own slot with +inf (magnitude that never wins a minimum, sign bit 0), takes the minimum
// magnitude and the XOR of the sign bits over the whole row, and later stores its new message in
// the same slot. Minimum and parity equal those over the other slots exactly.
// DP is the launch's largest column pitch; dp the problem's own (dp <= DP).
template <typename MT, int DP, int RPC>
__device__ __forceinline__ void update_column(uint32_t v, int deg, const uint32_t* csc, int dp, const float* lam,
                                              uint32_t rp, float alpha, MT* msgs, uint8_t* dec8, const uint8_t* s8,
                                              uint8_t* par8, float* lpost) {
  uint32_t ent[DP];
  const uint4* ce = reinterpret_cast<const uint4*>(csc + (size_t)v * dp);
#pragma unroll
  for (int q = 0; q < DP / 4; ++q) {
    uint4 x = make_uint4(0u, 0u, 0u, 0u);
    if (4 * q < dp) x = __ldg(ce + q);
    ent[4 * q + 0] = x.x; ent[4 * q + 1] = x.y; ent[4 * q + 2] = x.z; ent[4 * q + 3] = x.w;
  }
  const float lamv = __ldg(lam + v);
  const uint32_t RP = RPC ? (uint32_t)RPC * 8u : rp;
  float mcv[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    mcv[k] = 0.0f;
    if (k < deg) {
      const uint32_t c = ent[k] >> 9;
      MT* row = msgs + c * RP;
      Msg<MT>::set_inf(row + (ent[k] & 0xffu));
      float mn = __int_as_float(0x7f800000);
      uint32_t sg = 0;
      if (RPC) {
#pragma unroll
        for (int ch = 0; ch < RPC; ++ch) Msg<MT>::scan8(row + 8 * ch, mn, sg);
      } else {
        for (uint32_t ch = 0; ch < RP; ch += 8) Msg<MT>::scan8(row + ch, mn, sg);
      }
      const uint32_t neg = Msg<MT>::sign(sg) ^ (uint32_t)s8[c];
      const float mag = __fmul_rn(alpha, mn);
      mcv[k] = neg ? -mag : mag;
    }
  }
  float L = lamv;
#pragma unroll
  for (int k = 0; k < DP; ++k)
    if (k < deg) L = __fadd_rn(L, mcv[k]);
  float pre = lamv;  // lambda + m_0 + ... + m_{k-1}, the shared head of every exclusion sum
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    if (k < deg) {
      float a = pre;
#pragma unroll
      for (int k2 = k + 1; k2 < DP; ++k2)
        if (k2 < deg) a = __fadd_rn(a, mcv[k2]);
      Msg<MT>::store(msgs + (ent[k] >> 9) * RP + (ent[k] & 0xffu), a);
      pre = __fadd_rn(pre, mcv[k]);
    }
  }
  const uint8_t e_new = L <= 0.0f;
  if (e_new != dec8[v]) {
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k < deg) par8[ent[k] >> 9] ^= 1u;
    dec8[v] = e_new;
  }
  if (lpost) lpost[v] = L;
}

// One parallel (flooding) iteration of Algorithm 1 on the warp's FP32 message image.
// Check pass: a lane takes whole rows; from the smallest magnitude, the second smallest, the slot
// holding the smallest and the sign parity of the row's variable-to-check messages it overwrites each
// real slot with that edge's check-to-variable message (minimum and sign product over the other
// slots: exactly the exclusion over N(c) \ v). Column pass: a lane takes whole columns and turns its
// own slots into the new variable-to-check messages with the sums of the serial update. Every column
// reads only its own slots, so the passes need no second image. Parity pass: (H e)_c XOR s_c from
// the decisions (many columns touch a check in the column pass).
template <int DP>
__device__ __forceinline__ void flood_sweep(const Tables& t, float alpha, float* msgs, uint8_t* dec8,
                                            const uint8_t* s8, uint8_t* par8, float* lpost, int lane) {
  const int m = t.m, n = t.n;
  const uint32_t RP = (uint32_t)t.RP;
  for (int c = lane; c < m; c += 32) {
    const int deg = __ldg(t.rowptr + c + 1) - __ldg(t.rowptr + c);
    float* row = msgs + (size_t)c * RP;
    float m1 = __int_as_float(0x7f800000), m2 = m1;
    int a1 = -1;
    uint32_t sx = 0;
    for (int j = 0; j < deg; ++j) {
      const float x = row[row_position((uint32_t)c, (uint32_t)j, (int)RP, 4)];
      const float ax = fabsf(x);
      sx ^= __float_as_uint(x) >> 31;
      if (ax < m1) { m2 = m1; m1 = ax; a1 = j; }
      else if (ax < m2) m2 = ax;
    }
    for (int j = 0; j < deg; ++j) {
      const uint32_t pos = row_position((uint32_t)c, (uint32_t)j, (int)RP, 4);
      const float x = row[pos];
      const float mn = j == a1 ? m2 : m1;
      const uint32_t neg = (sx ^ (__float_as_uint(x) >> 31) ^ (uint32_t)s8[c]) & 1u;
      const float mag = __fmul_rn(alpha, mn);
      row[pos] = neg ? -mag : mag;
    }
  }
  __syncwarp();
  for (int v = lane; v < n; v += 32) {
    const int deg = __ldg(t.colptr + v + 1) - __ldg(t.colptr + v);
    float* slot[DP];
    float cv[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      slot[k] = msgs;
      cv[k] = 0.0f;
      if (k < deg) {
        const uint32_t ent = __ldg(t.csc_ent + (size_t)v * t.DP + k);
        slot[k] = msgs + (size_t)(ent >> 9) * RP + (ent & 0xffu);
        cv[k] = *slot[k];
      }
    }
    const float lamv = __ldg(t.lam + v);
    float L = lamv;
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k < deg) L = __fadd_rn(L, cv[k]);
    float pre = lamv;   // lambda + m_0 + ... + m_{k-1}, the shared head of every exclusion sum
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      if (k < deg) {
        float a = pre;
#pragma unroll
        for (int k2 = k + 1; k2 < DP; ++k2)
          if (k2 < deg) a = __fadd_rn(a, cv[k2]);
        *slot[k] = a;
        pre = __fadd_rn(pre, cv[k]);
      }
    }
    dec8[v] = L <= 0.0f ? 1u : 0u;
    if (lpost) lpost[v] = L;
  }
  __syncwarp();
  for (int c = lane; c < m; c += 32) {
    uint32_t p = s8[c];
    for (int e = __ldg(t.rowptr + c); e < __ldg(t.rowptr + c + 1); ++e) p ^= dec8[__ldg(t.colidx + e)];
    par8[c] = (uint8_t)p;
  }
  __syncwarp();
}

// One iteration of a schedule over check layers, with the check-to-variable messages in their own
// float image cv (same slot layout as the message image msgs): the layered schedule (the oracle's
// reading R10; layers from the graph builder) or, with flood set, the parallel schedule as a single
// layer of all checks (Algorithm 1's other branch, reading R8), which FP16 message storage needs:
// there the check-to-variable messages of an iteration are float temporaries and only the stored
// variable-to-check messages are rounded.
// Per layer, a check pass (lane per check of the layer: smallest and second-smallest magnitude, the
// slot of the smallest and the sign parity of the row's variable-to-check messages give each edge's
// minimum and sign product over the other edges, scaled by alpha and signed by the syndrome bit) and a
// column pass (lane per column of the layer's checks, which share no column: the serial update's
// exclusion sums over the column's current cv entries, stored as its new variable-to-check messages).
// Then every posterior (lambda plus the column's cv entries in ascending check order), decision and
// check parity. cv holds zeros when a layered member starts (init in run_member).
template <typename MT, int DP>
__device__ __forceinline__ void layer_sweep(const Tables& t, float alpha, bool flood, MT* msgs, float* cv,
                                            uint8_t* dec8, const uint8_t* s8, uint8_t* par8, float* lpost,
                                            int lane) {
  const int m = t.m, n = t.n;
  const uint32_t RP = (uint32_t)t.RP;
  const int nl = flood ? 1 : t.nlayer;
  for (int l = 0; l < nl; ++l) {
    const int c0 = flood ? 0 : __ldg(t.layer_ptr + l), c1 = flood ? m : __ldg(t.layer_ptr + l + 1);
    for (int q = c0 + lane; q < c1; q += 32) {
      const int c = flood ? q : __ldg(t.layer_chk + q);
      const int deg = __ldg(t.rowptr + c + 1) - __ldg(t.rowptr + c);
      const MT* row = msgs + (size_t)c * RP;
      float* crow = cv + (size_t)c * RP;
      float m1 = __int_as_float(0x7f800000), m2 = m1;
      int a1 = -1;
      uint32_t sx = 0;
      for (int j = 0; j < deg; ++j) {
        const float x = Msg<MT>::value(row[row_position((uint32_t)c, (uint32_t)j, (int)RP, Msg<MT>::kSpc)]);
        const float ax = fabsf(x);
        sx ^= __float_as_uint(x) >> 31;
        if (ax < m1) { m2 = m1; m1 = ax; a1 = j; }
        else if (ax < m2) m2 = ax;
      }
      for (int j = 0; j < deg; ++j) {
        const uint32_t pos = row_position((uint32_t)c, (uint32_t)j, (int)RP, Msg<MT>::kSpc);
        const float x = Msg<MT>::value(row[pos]);
        const uint32_t neg = (sx ^ (__float_as_uint(x) >> 31) ^ (uint32_t)s8[c]) & 1u;
        const float mag = __fmul_rn(alpha, j == a1 ? m2 : m1);
        crow[pos] = neg ? -mag : mag;
      }
    }
    __syncwarp();
    const int v0 = flood ? 0 : __ldg(t.layer_vptr + l), v1 = flood ? n : __ldg(t.layer_vptr + l + 1);
    for (int q = v0 + lane; q < v1; q += 32) {
      const int v = flood ? q : __ldg(t.layer_var + q);
      const int deg = __ldg(t.colptr + v + 1) - __ldg(t.colptr + v);
      uint32_t slot[DP];
      float c2v[DP];
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        slot[k] = 0u;
        c2v[k] = 0.0f;
        if (k < deg) {
          const uint32_t ent = __ldg(t.csc_ent + (size_t)v * t.DP + k);
          slot[k] = (ent >> 9) * RP + (ent & 0xffu);
          c2v[k] = cv[slot[k]];
        }
      }
      float pre = __ldg(t.lam + v);   // lambda + m_0 + ... + m_{k-1}, the shared head of every exclusion sum
#pragma unroll
      for (int k = 0; k < DP; ++k) {
        if (k < deg) {
          float a = pre;
#pragma unroll
          for (int k2 = k + 1; k2 < DP; ++k2)
            if (k2 < deg) a = __fadd_rn(a, c2v[k2]);
          Msg<MT>::store(msgs + slot[k], a);
          pre = __fadd_rn(pre, c2v[k]);
        }
      }
    }
    __syncwarp();
  }
  for (int v = lane; v < n; v += 32) {
    const int deg = __ldg(t.colptr + v + 1) - __ldg(t.colptr + v);
    float L = __ldg(t.lam + v);
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k < deg) {
        const uint32_t ent = __ldg(t.csc_ent + (size_t)v * t.DP + k);
        L = __fadd_rn(L, cv[(ent >> 9) * RP + (ent & 0xffu)]);
      }
    dec8[v] = L <= 0.0f ? 1u : 0u;
    if (lpost) lpost[v] = L;
  }
  __syncwarp();
  for (int c = lane; c < m; c += 32) {
    uint32_t p = s8[c];
    for (int e = __ldg(t.rowptr + c); e < __ldg(t.rowptr + c + 1); ++e) p ^= dec8[__ldg(t.colidx + e)];
    par8[c] = (uint8_t)p;
  }
  __syncwarp();
}

// Blocks per SM the register budget targets: FP16 states are small enough for 24 warps per SM,
// FP32 states (twice the message bytes) fill shared memory at about 16-18.
template <typename MT>
struct MinBlocks { static constexpr int value = 16 / kBpWarpsPerCta; };
template <>
struct MinBlocks<__half> { static constexpr int value = 24 / kBpWarpsPerCta; };

// Decodes one shot of problem t with the warp (the body of the persistent loop below).
// One member (index i) of the shot whose syndrome bytes are in the warp's shared memory: initialises
// the member's message image and runs up to `budget` sweeps, stopping at the first that leaves
// H e = s, or before sweep `it` when stop(it) holds. Returns the converging sweep (0 if none) and in
// `ran` the sweeps run; leaves the decisions in the warp's decision bytes and the posterior of the
// last sweep in lpost when soft output is on or `keep_last` is set and the member reached sweep T.
template <typename MT, int DP, int RPC, bool MIXED, typename Stop>
__device__ __forceinline__ int run_member(const Tables& t, int i, int budget, bool want_soft, bool keep_last,
                                          unsigned char* base, float* lpost, int lane, unsigned long long& my_iters,
                                          int& ran, Stop stop) {
  const int n = t.n, m = t.m, T = t.T;
  const int m4 = (m + 3) >> 2;
  const int n4 = (n + 3) >> 2;
  const int msg_vec = (int)(((size_t)m * t.RP * sizeof(MT)) / 16);
  const uint32_t* csc = t.csc_ent;
  const float* lam = t.lam;
  const int dp = MIXED ? t.DP : DP;   // one problem: the pitch is the launch's
  const uint32_t rp = (uint32_t)t.RP;
  MT* msgs = reinterpret_cast<MT*>(base + t.off_msg);
  uint8_t* dec8 = base + t.off_dec;
  uint8_t* s8 = base + t.off_s;
  uint8_t* par8 = base + t.off_par;
  // member init: messages from the prior image, decisions 0, parity = s
  {
    const uint4* src = reinterpret_cast<const uint4*>(t.msg_init);
    uint4* dst = reinterpret_cast<uint4*>(msgs);
    for (int q = lane; q < msg_vec; q += 32) dst[q] = __ldg(src + q);
    uint32_t* d32 = reinterpret_cast<uint32_t*>(dec8);
    for (int q = lane; q < n4; q += 32) d32[q] = 0u;
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(s8);
    uint32_t* p32 = reinterpret_cast<uint32_t*>(par8);
    for (int q = lane; q < m4; q += 32) p32[q] = s32[q];
  }
  const bool layered = i >= t.n_flood && i < t.n_flood + t.n_layered;
  float* cv = t.off_cv >= 0 ? reinterpret_cast<float*>(base + t.off_cv) : nullptr;
  if (layered) {   // the layered member's check-to-variable messages start at zero
    uint4* c4 = reinterpret_cast<uint4*>(cv);
    const int cv_vec = (int)(((size_t)m * t.RP * 4) / 16);
    for (int q = lane; q < cv_vec; q += 32) c4[q] = make_uint4(0u, 0u, 0u, 0u);
  }
  __syncwarp();

  const uint32_t* sch = t.sched + (size_t)i * n;
  const uint32_t* lo = t.lvl_off + (size_t)i * (n + 1);
  const int nl = __ldg(t.nlev + i);
  const float alpha = __ldg(t.alpha_m + i);   // member i's scaling factor
  int conv = 0;
  ran = 0;
  for (int it = 1; it <= budget; ++it) {
    if (stop(it)) break;
    // the posterior is needed after the last possible sweep of a member that may end without
    // converging (LLR average) and, for soft output, after every sweep
    float* lp = (want_soft || (it == T && keep_last)) ? lpost : nullptr;
    bool swept = false;   // by a schedule other than the member's serial one
    if (i < t.n_flood) {   // parallel schedule
      if constexpr (std::is_same<MT, float>::value) flood_sweep<DP>(t, alpha, msgs, dec8, s8, par8, lp, lane);
      else layer_sweep<MT, DP>(t, alpha, true, msgs, cv, dec8, s8, par8, lp, lane);
      swept = true;
    } else if (layered) {
      layer_sweep<MT, DP>(t, alpha, false, msgs, cv, dec8, s8, par8, lp, lane);
      swept = true;
    }
    for (int l = 0; l < nl && !swept; ++l) {
      const uint32_t b = __ldg(lo + l), e = __ldg(lo + l + 1);
      for (uint32_t idx = b + lane; idx < e; idx += 32) {
        const uint32_t ent = __ldg(sch + idx);
        update_column<MT, DP, RPC>(ent & 0xffffffu, (int)(ent >> 24), csc, dp, lam, rp, alpha, msgs, dec8, s8,
                                   par8, lp);
      }
      __syncwarp();
    }
    ++my_iters;
    ran = it;
    uint32_t bad = 0;
    const uint32_t* p32 = reinterpret_cast<const uint32_t*>(par8);
    for (int q = lane; q < m4; q += 32) bad |= p32[q];
    if (!__any_sync(kFull, bad)) { conv = it; break; }
  }
  return conv;
}

template <typename MT, int DP, int RPC, bool MIXED>
__device__ __forceinline__ void decode_shot(const BpArgs& a, const Tables& t, uint32_t shot, unsigned char* base,
                                            float* acc, float* lpost, float* cand_post, int lane,
                                            unsigned long long& my_iters, unsigned long long& my_shots,
                                            unsigned long long& my_fail) {
  const int n = t.n, m = t.m, K = t.K, M = t.M, T = t.T, nw = t.nw, kw = t.kw;
  const int m4 = (m + 3) >> 2;
  const int n4 = (n + 3) >> 2;
  const int msg_vec = (int)(((size_t)m * t.RP * sizeof(MT)) / 16);
  const uint32_t* csc = t.csc_ent;
  const float* lam = t.lam;
  const int dp = MIXED ? t.DP : DP;   // one problem: the pitch is the launch's
  const uint32_t rp = (uint32_t)t.RP;
  MT* msgs = reinterpret_cast<MT*>(base + t.off_msg);
  uint8_t* dec8 = base + t.off_dec;
  uint8_t* s8 = base + t.off_s;
  uint8_t* par8 = base + t.off_par;
  uint32_t* cand = reinterpret_cast<uint32_t*>(base + t.off_cand);
  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  uint32_t any = 0;
  for (int c = lane; c < 4 * m4; c += 32) {
    uint32_t b = c < m ? (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u : 0u;
    s8[c] = (uint8_t)b;
    any |= b;
  }
  any = __any_sync(kFull, any);
  __syncwarp();
  ++my_shots;
  uint32_t* out_corr = a.corr + (size_t)shot * a.corr_stride;

  if (!any && !a.want_soft) {
    // s = 0: every member converges in iteration 1 to e = 0; the first M are the candidates, all of
    // weight 0, so member 0 is chosen.
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
    const int conv = run_member<MT, DP, RPC, MIXED>(t, i, budget, a.want_soft != 0, ncand == 0, base, lpost, lane,
                                                    my_iters, ran, [](int) { return false; });
    if (conv) {
      // insert (conv, i); i exceeds every member already listed, so it goes after equal iterations
      const int p = __popc(__ballot_sync(kFull, lane < ncand && c_t <= conv));
      const int slot = ncand < M ? ncand : __shfl_sync(kFull, c_slot, M - 1);
      uint32_t* bits = cand + (size_t)slot * nw;
      float W = 0.0f;
      for (int w = 0; w < nw; ++w) {
        const int v = 32 * w + lane;
        const uint32_t word = __ballot_sync(kFull, v < n && dec8[v] != 0);
        if (lane == 0) bits[w] = word;
        uint32_t x = word;
        while (x) {
          const int bpos = __ffs(x) - 1;
          W = __fadd_rn(W, __ldg(lam + 32 * w + bpos));
          x &= x - 1;
        }
      }
      if (a.want_soft) {
        float* dst = cand_post + (size_t)slot * n;
        for (int v = lane; v < n; v += 32) dst[v] = lpost[v];
      }
      const float uW = __shfl_up_sync(kFull, c_W, 1);
      const int ut = __shfl_up_sync(kFull, c_t, 1), ui = __shfl_up_sync(kFull, c_i, 1);
      const int us = __shfl_up_sync(kFull, c_slot, 1);
      const int last = min(ncand, M - 1);
      if (lane > p && lane <= last) { c_W = uW; c_t = ut; c_i = ui; c_slot = us; }
      if (lane == p) { c_W = W; c_t = conv; c_i = i; c_slot = slot; }
      ncand = min(ncand + 1, M);
      __syncwarp();
    } else if (ncand == 0) {
      // not converged after T sweeps and no candidate yet: add LLR^i / ||LLR^i|| (finite entries)
      float part = 0.0f;
      for (int v = lane; v < n; v += 32) {
        const float x = lpost[v];
        part = __fadd_rn(part, is_finite_bits(x) ? __fmul_rn(x, x) : 0.0f);
      }
#pragma unroll
      for (int off = 16; off >= 1; off >>= 1) part = __fadd_rn(part, __shfl_xor_sync(kFull, part, off));
      const float nrm = __fsqrt_rn(part);
      for (int v = lane; v < n; v += 32) {
        const float x = lpost[v];
        const float term = is_finite_bits(x) ? (nrm == 0.0f ? 0.0f : __fdiv_rn(x, nrm)) : x;
        acc[v] = __fadd_rn(i == 0 ? 0.0f : acc[v], term);
      }
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
      const float* src = cand_post + (size_t)slot * n;
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
template <typename MT, int DP, int RPC, bool MIXED>
__device__ __forceinline__ void decode_pair(const BpArgs& a, const Tables& t, uint32_t shot, int slot, int i,
                                            unsigned char* base, float* lpost, int lane, unsigned long long& my_iters,
                                            unsigned long long& my_shots, unsigned long long& my_fail) {
  const int K = t.K, M = t.M, T = t.T, n = t.n, m = t.m, nw = t.nw, kw = t.kw;
  if (i >= K) return;
  const int m4 = (m + 3) >> 2;
  uint8_t* s8 = base + t.off_s;
  const uint8_t* dec8 = base + t.off_dec;
  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  uint32_t any = 0;
  for (int c = lane; c < 4 * m4; c += 32) {
    const uint32_t b = c < m ? (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u : 0u;
    s8[c] = (uint8_t)b;
    any |= b;
  }
  any = __any_sync(kFull, any);
  __syncwarp();
  if (!any && !a.want_soft) {
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
  int* conv = a.pconv + (size_t)slot * a.pair_K;
  int ran = 0;
  const int cv = run_member<MT, DP, RPC, MIXED>(t, i, T, a.want_soft != 0, true, base, lpost, lane, my_iters, ran,
                                                [&](int it) { return pair_should_stop(conv, K, M, i, it, lane); });
  const size_t rec = (size_t)slot * a.pair_K + i;
  if (cv) {
    // the correction's bits and W(e) = sum of lambda_j over e_j = 1, ascending j
    uint32_t* bits = a.pbits + rec * a.bnd.nw;
    float W = 0.0f;
    for (int w = 0; w < nw; ++w) {
      const int v = 32 * w + lane;
      const uint32_t word = __ballot_sync(kFull, v < n && dec8[v] != 0);
      if (lane == 0) bits[w] = word;
      uint32_t x = word;
      while (x) {
        const int bpos = __ffs(x) - 1;
        W = __fadd_rn(W, __ldg(t.lam + 32 * w + bpos));
        x &= x - 1;
      }
    }
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

// MIXED: the shots of the launch name their problems (dem_of_shot); the problems' descriptors are
// copied to shared memory after the warps' regions. Otherwise every shot decodes a.one, which the
// kernel reads from its parameter space.
template <typename MT, int DP, int RPC, bool MIXED>
__global__ void __launch_bounds__(kBpWarpsPerCta * 32, MinBlocks<MT>::value) k_bp(const BpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wcta = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBpWarpsPerCta + wcta;
  Tables* sdem = reinterpret_cast<Tables*>(smem + (size_t)kBpWarpsPerCta * a.bnd.warp_smem);
  if (MIXED) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.dems);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sdem);
    const int words = a.ndem * (int)(sizeof(Tables) / 4);
    for (int q = threadIdx.x; q < words; q += blockDim.x) dst[q] = __ldg(src + q);
    __syncthreads();
  }
  unsigned char* base = smem + (size_t)wcta * a.bnd.warp_smem;
  float* acc = a.scratch + gw * a.scratch_pitch;  // n floats: LLR average accumulator
  float* lpost = acc + a.bnd.n;                    // n floats: the member's posterior when needed
  float* cand_post = lpost + a.bnd.n;              // M * n floats (only with want_soft)
  unsigned long long my_iters = 0, my_shots = 0, my_fail = 0;

  if (a.pair_mode) {
    const unsigned long long npairs = (unsigned long long)a.nshots * (unsigned long long)a.pair_K;
    for (;;) {
      unsigned long long q = 0;
      if (lane == 0) q = atomicAdd(a.next_pair, 1u);
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
          if (a.stats && lane == 0) {
            vibe_shot_stats st;
            st.status = VIBE_STATUS_BAD_PROBLEM; st.lsd_invoked = 0; st.n_converged = 0; st.chosen_member = 0;
            st.iters = 0; st.largest_cluster = 0; st.n_clusters = 0;
            a.stats[shot] = st;
          }
          if (a.counters && lane == 0) atomicAdd(a.counters + VIBE_CNT_BAD_PROBLEM, 1ull);
          continue;
        }
        if (sdem[di].engine != VIBE_ENGINE_IMAGE) continue;   // left to the summary engine
        decode_pair<MT, DP, RPC, true>(a, sdem[di], shot, (int)shot, i, base, lpost, lane, my_iters, my_shots, my_fail);
      } else {
        decode_pair<MT, DP, RPC, false>(a, a.one, shot, (int)shot, i, base, lpost, lane, my_iters, my_shots, my_fail);
      }
    }
  }
  for (;;) {
    if (a.pair_mode) break;
    uint32_t shot = 0;
    if (lane == 0) shot = atomicAdd(a.next_shot, 1u);
    shot = __shfl_sync(kFull, shot, 0);
    if (shot >= a.nshots) break;
    if (MIXED) {
      const int di = __ldg(a.dem_of_shot + shot);
      if ((unsigned)di >= (unsigned)a.ndem) {
        if (!a.flag_bad) continue;
        // problem index outside the launch's table: zero outputs, status BAD_PROBLEM, no decoding
        for (int w = lane; w < a.corr_stride; w += 32) a.corr[(size_t)shot * a.corr_stride + w] = 0u;
        if (a.logical)
          for (int w = lane; w < a.log_stride; w += 32) a.logical[(size_t)shot * a.log_stride + w] = 0u;
        if (a.soft)
          for (int j = lane; j < a.soft_stride; j += 32) a.soft[(size_t)shot * a.soft_stride + j] = 0.0f;
        if (a.stats && lane == 0) {
          vibe_shot_stats st;
          st.status = VIBE_STATUS_BAD_PROBLEM; st.lsd_invoked = 0; st.n_converged = 0; st.chosen_member = 0;
          st.iters = 0; st.largest_cluster = 0; st.n_clusters = 0;
          a.stats[shot] = st;
        }
        if (a.counters && lane == 0) atomicAdd(a.counters + VIBE_CNT_BAD_PROBLEM, 1ull);
        continue;
      }
      if (sdem[di].engine != VIBE_ENGINE_IMAGE) continue;   // left to the summary engine
      decode_shot<MT, DP, RPC, true>(a, sdem[di], shot, base, acc, lpost, cand_post, lane, my_iters, my_shots,
                                     my_fail);
    } else {
      decode_shot<MT, DP, RPC, false>(a, a.one, shot, base, acc, lpost, cand_post, lane, my_iters, my_shots,
                                      my_fail);
    }
  }
  if (lane == 0 && a.counters) {
    atomicAdd(a.counters + VIBE_CNT_SHOTS, my_shots);
    atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, my_iters);
    if (my_fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, my_fail);
  }
}

// RPC: row pitch in 8-slot chunks when every problem of the launch has RP 8, 16 or 32, else 0.
inline int rpc_of(const Bounds& b) { return (b.RP == 8 || b.RP == 16 || b.RP == 32) ? b.RP / 8 : 0; }

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename MT, int DP, int RPC, bool MIXED>
cudaError_t launch_one(const BpArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = ensure_dyn_smem<k_bp<MT, DP, RPC, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  k_bp<MT, DP, RPC, MIXED><<<grid, kBpWarpsPerCta * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename MT, int DP, int RPC, bool MIXED>
cudaError_t occupancy_one(size_t smem, int* out) {
  cudaError_t err = ensure_dyn_smem<k_bp<MT, DP, RPC, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bp<MT, DP, RPC, MIXED>, kBpWarpsPerCta * 32, smem);
}

template <typename Fn>
cudaError_t by_rpc(int rpc, Fn&& f) {
  switch (rpc) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 4: return f(std::integral_constant<int, 4>{});
    default: return f(std::integral_constant<int, 0>{});
  }
}

template <typename Fn>
cudaError_t by_dp(int DP, Fn&& f) {
  switch (DP) {
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    default: return cudaErrorInvalidValue;
  }
}

// Mixed launches use the generic row scan (RPC 0) only, which keeps the number of instantiations down.
template <typename MT>
cudaError_t launch_mt(const BpArgs& a, int grid, cudaStream_t s) {
  const bool mixed = a.dem_of_shot != nullptr;
  const size_t smem = bp_cta_smem_bytes(a.bnd, mixed ? a.ndem : 0);
  return by_dp(a.bnd.DP, [&](auto dp) {
    if (mixed) return launch_one<MT, decltype(dp)::value, 0, true>(a, grid, smem, s);
    return by_rpc(rpc_of(a.bnd), [&](auto rpc) {
      return launch_one<MT, decltype(dp)::value, decltype(rpc)::value, false>(a, grid, smem, s);
    });
  });
}

template <typename MT>
cudaError_t occupancy_mt(const Bounds& b, int ndem, int* out) {
  const size_t smem = bp_cta_smem_bytes(b, ndem);
  return by_dp(b.DP, [&](auto dp) {
    if (ndem > 0) return occupancy_one<MT, decltype(dp)::value, 0, true>(smem, out);
    return by_rpc(rpc_of(b), [&](auto rpc) {
      return occupancy_one<MT, decltype(dp)::value, decltype(rpc)::value, false>(smem, out);
    });
  });
}

}  // namespace

size_t bp_warp_smem_bytes(Tables* t, int msg_fp16) {
  size_t o = 0;
  t->off_msg = (int)o;
  o = align16(o + (size_t)t->m * t->RP * (msg_fp16 ? 2 : 4));
  t->off_dec = (int)o;
  o = align16(o + ((size_t)t->n + 3) / 4 * 4);
  const size_t m4 = ((size_t)t->m + 3) / 4 * 4;
  t->off_s = (int)o;
  o = align16(o + m4);
  t->off_par = (int)o;
  o = align16(o + m4);
  t->off_cand = (int)o;
  o = align16(o + (size_t)t->M * t->nw * 4);
  t->off_cv = -1;
  if (t->n_layered > 0 || (t->n_flood > 0 && msg_fp16)) {
    t->off_cv = (int)o;
    o = align16(o + (size_t)t->m * t->RP * 4);
  }
  t->warp_smem = (int)o;
  return o;
}

size_t bp_cta_smem_bytes(const Bounds& b, int ndem) {
  return (size_t)kBpWarpsPerCta * b.warp_smem + align16((size_t)ndem * sizeof(Tables));
}

cudaError_t launch_bp(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s) {
  return msg_fp16 ? launch_mt<__half>(a, grid, s) : launch_mt<float>(a, grid, s);
}

cudaError_t bp_occupancy(const Bounds& b, int ndem, int msg_fp16, int* blocks_per_sm) {
  return msg_fp16 ? occupancy_mt<__half>(b, ndem, blocks_per_sm) : occupancy_mt<float>(b, ndem, blocks_per_sm);
}

}  // namespace vibe
