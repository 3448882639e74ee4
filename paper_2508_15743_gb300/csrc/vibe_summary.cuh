// Check-node summaries of the summary engine (vibe_bpx.cu), host- and device-callable.
//
// For a check c the summary describes the magnitudes of the variable-to-check messages of its row:
// up to two "holder" edges with their exact magnitudes m1 <= m2 and their positions inside the CSR
// row (255 marks an empty slot; a single holder sits in slot 1), and a floor F, a lower bound on every
// magnitude of the row outside the holders. Every non-holder is also >= every holder, so the
// effective floor Fe = max(F, largest holder) bounds the non-holders too. Then
//   min over the row without position p = m2 if p holds m1 (two holders), m1 if p is not the first
//   holder (at least one holder), +inf if Fe is +inf (every other entry is +inf), and unknown
//   otherwise -- the row must be rescanned first.
// When the edge at position p takes the magnitude x: p leaves the holder list if it was in it; it
// re-enters if x <= Fe (a former holder) or x < Fe (any other edge); a full list evicts its larger
// entry, whose value (or x itself, when x is the larger) becomes the floor. These keep both
// invariants exactly, whatever lower bound F is stored, so F may be rounded down.
//
// Beside it the summary carries three flags: the parity of the sign bits of the row's messages, the
// syndrome bit s_c and the check's parity (H e)_c XOR s_c.
//
// Storage (16-byte aligned arrays in shared memory, one element per check):
//   FP32 messages, 12 bytes: float2 {m1 | sign-parity flag in bit 31, m2 | syndrome flag in bit 31}
//     and a word {p1 | p2 << 8 | F << 16 | parity flag << 31}, F as binary16 without its sign bit,
//     rounded down from the float floor.
//   FP16 messages, 8 bytes: uint2 {m1 | sign-parity << 15 | m2 << 16 | syndrome << 31,
//     F | parity << 15 | p1 << 16 | p2 << 24}, every magnitude a binary16 (message magnitudes are
//     exact in binary16 when messages are stored in binary16).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace vibe {

constexpr uint32_t kEmptyPos = 255u;

// A summary in registers.
struct SumV {
  float m1, m2, F;
  uint32_t p1, p2;
  uint32_t sgn, syn, par;   // flags, 0 or 1
};

__host__ __device__ inline uint32_t holders(const SumV& s) {
  return s.p1 == kEmptyPos ? 0u : (s.p2 == kEmptyPos ? 1u : 2u);
}

__host__ __device__ inline float fmax_nan0(float a, float b) { return a > b ? a : b; }

// Effective floor: a lower bound on every non-holder magnitude.
__host__ __device__ inline float eff_floor(const SumV& s) {
  const uint32_t nh = holders(s);
  return nh == 2u ? fmax_nan0(s.F, s.m2) : (nh == 1u ? fmax_nan0(s.F, s.m1) : s.F);
}

__host__ __device__ inline bool is_inf_pos(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x) == 0x7f800000u;
#else
  return x == __builtin_inff();
#endif
}

// Minimum magnitude over the row without the edge at position p; false when the summary cannot tell.
__host__ __device__ inline bool sum_query(const SumV& s, uint32_t p, float& out) {
  const uint32_t nh = holders(s);
  const bool mine = p == s.p1;
  const float fe = eff_floor(s);
  out = nh == 2u ? (mine ? s.m2 : s.m1) : (nh == 1u && !mine ? s.m1 : fe);
  return nh == 2u || (nh == 1u && !mine) || is_inf_pos(fe);
}

// Lower bound of x representable in the stored floor (identity for the FP16 summary).
template <bool HALF>
__host__ __device__ inline float floor_round(float x);

// The summary after the edge at position p takes magnitude x. Also says whether anything but the
// flags could change (`slow`); when it is false the summary is returned unchanged.
template <bool HALF>
__host__ __device__ inline SumV sum_update(const SumV& s, uint32_t p, float x) {
  const uint32_t nh0 = holders(s);
  const bool is1 = nh0 >= 1u && p == s.p1, is2 = nh0 == 2u && p == s.p2;
  const bool was = is1 || is2;
  const float fe = eff_floor(s);
  // the list without p
  const float a1 = is1 ? s.m2 : s.m1, a2 = s.m2;
  const uint32_t q1 = is1 ? s.p2 : s.p1;
  const uint32_t k = nh0 - (was ? 1u : 0u);
  const bool ins = was ? x <= fe : x < fe;
  const bool lt1 = k == 0u || x < a1;
  const bool lt2 = k <= 1u || x < a2;
  SumV r = s;
  r.m1 = ins && lt1 ? x : a1;
  r.p1 = ins && lt1 ? p : (k >= 1u ? q1 : kEmptyPos);
  r.m2 = ins ? (lt1 ? a1 : (lt2 ? x : a2)) : a2;
  const uint32_t nk = ins ? (k + 1u < 2u ? k + 1u : 2u) : k;
  const uint32_t q2 = ins ? (lt1 ? q1 : (lt2 ? p : s.p2)) : s.p2;
  r.p2 = nk == 2u ? q2 : kEmptyPos;
  if (nk == 0u) r.p1 = kEmptyPos;
  r.F = ins && k == 2u ? floor_round<HALF>(lt2 ? a2 : x) : s.F;
  return r;
}

// Whether the update of position p to x can change more than the flags.
__host__ __device__ inline bool sum_slow(const SumV& s, uint32_t p, float x) {
  const uint32_t nh = holders(s);
  return (nh >= 1u && p == s.p1) || (nh == 2u && p == s.p2) || x < eff_floor(s);
}

// ---- storage ----

template <>
__host__ __device__ inline float floor_round<false>(float x) {
  return __half2float(__float2half_rd(x));
}
template <>
__host__ __device__ inline float floor_round<true>(float x) {
  return x;
}

__host__ __device__ inline uint32_t f2u(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  __builtin_memcpy(&u, &x, 4);
  return u;
#endif
}
__host__ __device__ inline float u2f(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  __builtin_memcpy(&x, &u, 4);
  return x;
#endif
}
__host__ __device__ inline uint32_t h_bits(float x) { return (uint32_t)__half_as_ushort(__float2half_rn(x)); }
__host__ __device__ inline float h_val(uint32_t b) { return __half2float(__ushort_as_half((unsigned short)b)); }

// FP32-message summaries: 12 bytes per check in two arrays.
struct SumStore32 {
  float2* m;       // m1, m2 with the sign-parity and syndrome flags in their sign bits
  uint32_t* meta;  // p1, p2, floor, parity flag
  static constexpr int kBytesPerCheck = 12;
  __host__ __device__ SumV load(int c) const {
    const float2 a = m[c];
    const uint32_t w = meta[c];
    SumV s;
    s.m1 = u2f(f2u(a.x) & 0x7fffffffu);
    s.m2 = u2f(f2u(a.y) & 0x7fffffffu);
    s.sgn = f2u(a.x) >> 31;
    s.syn = f2u(a.y) >> 31;
    s.p1 = w & 0xffu;
    s.p2 = (w >> 8) & 0xffu;
    s.F = h_val((w >> 16) & 0x7fffu);
    s.par = w >> 31;
    return s;
  }
  __host__ __device__ void store(int c, const SumV& s) const {
    m[c] = make_float2(u2f(f2u(s.m1) | (s.sgn << 31)), u2f(f2u(s.m2) | (s.syn << 31)));
    meta[c] = s.p1 | (s.p2 << 8) | ((uint32_t)__half_as_ushort(__float2half_rd(s.F)) & 0x7fffu) << 16 | (s.par << 31);
  }
  // flags only: the word holding the parity flag and the float holding the sign-parity flag
  __host__ __device__ void flip_flags(int c, bool sgn, bool par) const {
    if (sgn) reinterpret_cast<uint32_t*>(m + c)[0] ^= 0x80000000u;
    if (par) meta[c] ^= 0x80000000u;
  }
};

// FP16-message summaries: 8 bytes per check.
struct SumStore16 {
  uint2* v;
  static constexpr int kBytesPerCheck = 8;
  __host__ __device__ SumV load(int c) const {
    const uint2 a = v[c];
    SumV s;
    s.m1 = h_val(a.x & 0x7fffu);
    s.sgn = (a.x >> 15) & 1u;
    s.m2 = h_val((a.x >> 16) & 0x7fffu);
    s.syn = a.x >> 31;
    s.F = h_val(a.y & 0x7fffu);
    s.par = (a.y >> 15) & 1u;
    s.p1 = (a.y >> 16) & 0xffu;
    s.p2 = a.y >> 24;
    return s;
  }
  __host__ __device__ void store(int c, const SumV& s) const {
    v[c] = make_uint2(h_bits(s.m1) | (s.sgn << 15) | (h_bits(s.m2) << 16) | (s.syn << 31),
                      h_bits(s.F) | (s.par << 15) | (s.p1 << 16) | (s.p2 << 24));
  }
  __host__ __device__ void flip_flags(int c, bool sgn, bool par) const {
    uint32_t x = 0u, y = 0u;
    if (sgn) x = 1u << 15;
    if (par) y = 1u << 15;
    if (x) v[c].x ^= x;
    if (y) v[c].y ^= y;
  }
};

}  // namespace vibe
