// K1' -- the BP ensemble for problems whose message image does not fit in shared memory (circuit-level
// detector error models: rows of 100-200 entries, E up to ~4e5): the summary engine. Same method, same
// results as the image engine (vibe_bp.cu), which keeps a member's whole message image in shared
// memory; a different layout.
//
// Why a warp per shot. The wavefront levels of a random serial order on these graphs are short: a
// column conflicts with every column of its ~4 checks (~600 others), so a sweep of the d=11 problem
// has ~1000 levels of ~32 columns. One warp matches that width and synchronises with __syncwarp.
//
// Each warp decodes one shot at a time (persistent, shots from a global counter), running the members
// one after another with the iteration budget of the correction limit (Sec. III.D.2).
//
// Check-node state. For every check c the warp keeps in shared memory a 16-byte summary of the current
// variable-to-check messages of its row: the smallest magnitude, the second smallest (with
// multiplicity, +inf for a one-entry row), the edges holding them, and the parity of the sign bits
// (bit 31 of the second holder word). The magnitude minimum over the row without edge e is then
// (e == first holder ? second : smallest), and the sign parity without e is parity XOR sign(m_e):
// exactly the minimum and sign product that Algorithm 1's check update takes over N(c) \ v, with no
// row scan. The messages themselves (E floats or halves per warp, in CSC edge order so that a column's
// are contiguous) stay in global memory, where the column update reads its old values and writes the
// new ones. Two layouts of the rest of a warp's state (same results): "bytes" keeps the decision
// bits in shared memory and one byte per check for the syndrome and the check parity; "packed" moves
// the decision bits to global memory (each lane fetches its column's bit with the column's data, and
// only that column changes it) and packs syndrome and parity 32 bits to a word, for ~16 bytes of
// shared memory per check and more resident warps. Measured on circuit-level colour codes, packed is
// faster at d=5..9 and bytes at d=11 (the host picks by the number of checks; the tuner times both).
//
// Keeping the summary exact after column v replaces its message on c with magnitude x:
//   v holds the smallest:  x <= second -> smallest = x;  else the row is rescanned;
//   v holds the second:    x > second -> rescan; x < smallest -> v and the first holder swap places;
//                          else second = x;
//   otherwise:             x < smallest -> v holds the smallest, the old one the second;
//                          x < second -> v holds the second.
// Holding both holders keeps rescans rare even when many messages tie (equal priors at the start).
// Every check is touched by one column per level, so the updates of a level never collide. Rescans
// are queued and done after the level by the whole warp (a minimum/second-minimum reduction over the
// row's messages), before any later level reads the summary. A column's global reads (checks, old
// messages, prior) do not depend on the level before it, so each lane fetches its next column while
// the current level finishes.
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
  __device__ __forceinline__ static float store(float* p, float x) {
    __stcg(p, x);
    return x;
  }
};

template <>
struct XMsg<__half> {
  __device__ __forceinline__ static __half load(const __half* p) {
    return __ushort_as_half(__ldcg(reinterpret_cast<const unsigned short*>(p)));
  }
  __device__ __forceinline__ static float value(__half x) { return __half2float(x); }
  // rounds to half, stores -0 as +0, returns the stored value as a float
  __device__ __forceinline__ static float store(__half* p, float x) {
    unsigned short h = __half_as_ushort(__float2half_rn(x));
    if (h == 0x8000u) h = 0;
    __stcg(reinterpret_cast<unsigned short*>(p), h);
    return __half2float(__ushort_as_half(h));
  }
};

__device__ __forceinline__ uint32_t sign_bit(float x) { return __float_as_uint(x) >> 31; }

__device__ __forceinline__ bool is_finite_bits(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

// Shared state of one warp for its current shot.
struct XShared {
  float4* summ;     // m check summaries (smallest, second, holder edges, sign parity)
  uint32_t* s32;    // packed: ceil(m/32) syndrome words
  uint32_t* par32;  // packed: ceil(m/32) words, (H e) XOR s
  uint8_t* s8;      // bytes: m syndrome bytes
  uint8_t* par8;    // bytes: m bytes, (H e)_c XOR s_c
  uint32_t* dec;    // nw: the member's decisions, bit-packed (packed: in the warp's global scratch)
  int32_t* rlist;   // 32 * DP: checks to rescan after the current chunk of 32 columns
};

// Blocks per SM the register budget targets (16 warps per SM).
template <typename MT>
struct MinBlocksX { static constexpr int value = 16 / kBpxWarpsPerCta; };

// What a column update reads from global memory: its checks, its current messages and its prior.
// None of it changes before the column's own update (a column's messages are written only by that
// column), so it can be fetched a level early.
template <int DP>
struct ColData {
  uint32_t v, e0;
  uint32_t e_old;   // the column's current decision
  int deg;
  float lam;
  int c[DP];
  float o[DP];
};

template <typename MT, int DP, bool PK>
__device__ __forceinline__ void fetch_column(uint2 rec, const Tables& t, const MT* msg, const uint32_t* dec,
                                             ColData<DP>& d) {
  d.v = rec.x & 0xffffffu;
  d.deg = (int)(rec.x >> 24);
  d.e0 = rec.y;
  d.lam = __ldg(t.lam + d.v);
  d.e_old = PK ? (__ldcg(dec + (d.v >> 5)) >> (d.v & 31)) & 1u : 0u;   // only column v writes its bit
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    d.c[k] = 0;
    d.o[k] = 0.0f;
    if (k < d.deg) {
      d.c[k] = __ldg(t.rowidx + d.e0 + k);
      d.o[k] = XMsg<MT>::value(XMsg<MT>::load(msg + d.e0 + k));
    }
  }
}

// Serial-V update of column v (deg checks, edges e0 .. e0 + deg - 1 in ascending check order).
template <typename MT, int DP, bool PK>
__device__ __forceinline__ void update_column_x(const ColData<DP>& d, const Tables& t, float alpha, MT* msg,
                                                const XShared& X, int* rcount, float* lpost) {
  const uint32_t v = d.v, e0 = d.e0;
  const int deg = d.deg;
  const int* c = d.c;
  const float* o = d.o;
  const float lamv = d.lam;
  float mcv[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    mcv[k] = 0.0f;
    if (k < deg) {
      const float4 sm = X.summ[c[k]];
      const bool holder = __float_as_uint(sm.z) == e0 + k;
      const float mn = holder ? sm.y : sm.x;
      const uint32_t sk = PK ? X.s32[c[k] >> 5] >> (c[k] & 31) : (uint32_t)X.s8[c[k]];
      const uint32_t neg = ((__float_as_uint(sm.w) >> 31) ^ sign_bit(o[k]) ^ sk) & 1u;
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
      const float x = XMsg<MT>::store(msg + e0 + k, a);
      pre = __fadd_rn(pre, mcv[k]);
      // summary maintenance
      const float nm = fabsf(x);
      const uint32_t e = e0 + k;
      float4 s = X.summ[c[k]];   // this level's only reader and writer of check c
      uint32_t i1 = __float_as_uint(s.z), i2 = __float_as_uint(s.w) & 0x7fffffffu;
      const uint32_t sg = (__float_as_uint(s.w) >> 31) ^ sign_bit(o[k]) ^ sign_bit(x);
      bool rescan = false;
      if (e == i1) {
        if (nm <= s.y) s.x = nm;
        else rescan = true;
      } else if (e == i2) {
        if (nm > s.y) rescan = true;
        else if (nm < s.x) { s.y = s.x; i2 = i1; s.x = nm; i1 = e; }
        else s.y = nm;
      } else if (nm < s.x) {
        s.y = s.x; i2 = i1; s.x = nm; i1 = e;
      } else if (nm < s.y) {
        s.y = nm; i2 = e;
      }
      s.z = __uint_as_float(i1);
      s.w = __uint_as_float(i2 | (sg << 31));
      X.summ[c[k]] = s;
      if (rescan) X.rlist[atomicAdd(rcount, 1)] = c[k];
    }
  }
  const uint32_t e_new = L <= 0.0f ? 1u : 0u;
  const uint32_t bit = 1u << (v & 31);
  const uint32_t e_old = PK ? d.e_old : (X.dec[v >> 5] & bit) ? 1u : 0u;
  if (e_new != e_old) {
    atomicXor(&X.dec[v >> 5], bit);
#pragma unroll
    for (int k = 0; k < DP; ++k) {
      if (k < deg) {
        if (PK) atomicXor(&X.par32[c[k] >> 5], 1u << (c[k] & 31));
        else X.par8[c[k]] ^= 1u;   // this level's only writer of check c's byte
      }
    }
  }
  if (lpost) lpost[v] = L;
}

// (value, edge) pairs ordered by value, then edge
__device__ __forceinline__ bool before(float a, uint32_t ia, float b, uint32_t ib) {
  return a < b || (a == b && ia < ib);
}

// Warp-cooperative rescan of check c: smallest and second smallest magnitude (with multiplicity) and
// their edges over the row's current messages; the sign parity is kept as it is.
template <typename MT>
__device__ __forceinline__ void rescan_row(int c, const Tables& t, const MT* msg, float4* summ, int lane) {
  float m1 = __int_as_float(0x7f800000), m2 = m1;
  uint32_t i1 = 0x7fffffffu, i2 = 0x7fffffffu;
  const int b = __ldg(t.rowptr + c), e = __ldg(t.rowptr + c + 1);
  for (int q = b + lane; q < e; q += 32) {
    const uint32_t ed = __ldg(t.row_edge + q);
    const float a = fabsf(XMsg<MT>::value(XMsg<MT>::load(msg + ed)));
    if (before(a, ed, m1, i1)) { m2 = m1; i2 = i1; m1 = a; i1 = ed; }
    else if (before(a, ed, m2, i2)) { m2 = a; i2 = ed; }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float n1 = __shfl_xor_sync(kFull, m1, off), n2 = __shfl_xor_sync(kFull, m2, off);
    const uint32_t j1 = __shfl_xor_sync(kFull, i1, off), j2 = __shfl_xor_sync(kFull, i2, off);
    if (before(n1, j1, m1, i1)) {   // the other's first wins; second = better of my first, its second
      if (before(m1, i1, n2, j2)) { m2 = m1; i2 = i1; } else { m2 = n2; i2 = j2; }
      m1 = n1; i1 = j1;
    } else if (before(n1, j1, m2, i2)) {
      m2 = n1; i2 = j1;
    }
  }
  if (lane == 0) {
    float4 s = summ[c];
    s.x = m1; s.y = m2; s.z = __uint_as_float(i1);
    s.w = __uint_as_float((__float_as_uint(s.w) & 0x80000000u) | i2);
    summ[c] = s;
  }
}


// A chunk of a sweep: up to 32 consecutive schedule entries [cs, min(cs + 32, e)) of level l, whose
// entries end at e. l == nl marks the end of the sweep.
struct Chunk {
  int l;
  uint32_t cs, e;
};

__device__ __forceinline__ Chunk first_chunk(const uint32_t* lo) { return Chunk{0, __ldg(lo), __ldg(lo + 1)}; }

__device__ __forceinline__ Chunk next_chunk(const Chunk& c, const uint32_t* lo, int nl) {
  if (c.l >= nl) return c;
  if (c.cs + 32 < c.e) return Chunk{c.l, c.cs + 32, c.e};
  return Chunk{c.l + 1, c.e, c.l + 1 < nl ? __ldg(lo + c.l + 2) : c.e};
}

__device__ __forceinline__ bool in_chunk(const Chunk& c, int nl, int lane) {
  return c.l < nl && c.cs + (uint32_t)lane < c.e;
}

// Decodes shot `shot` of problem t with one warp. base: the warp's shared memory; gs: its global
// scratch (messages, posterior, LLR accumulator, candidate records).
template <typename MT, int DP, bool PK>
__device__ __forceinline__ void decode_shot_x(const BpArgs& a, const Tables& t, uint32_t shot, unsigned char* base,
                                              unsigned char* gs, int lane, unsigned long long& my_iters,
                                              unsigned long long& my_shots, unsigned long long& my_fail,
                                              unsigned long long& my_rescans) {
  const int n = t.n, m = t.m, K = t.K, M = t.M, T = t.T, nw = t.nw, kw = t.kw;
  const int mw = t.mw;
  const int m4 = (m + 3) >> 2;
  XShared X;
  X.summ = reinterpret_cast<float4*>(base + t.xo_summ);
  X.s32 = reinterpret_cast<uint32_t*>(base + t.xo_s);
  X.par32 = reinterpret_cast<uint32_t*>(base + t.xo_par);
  X.s8 = base + t.xo_s;
  X.par8 = base + t.xo_par;
  X.dec = PK ? reinterpret_cast<uint32_t*>(gs + t.xg_dec) : reinterpret_cast<uint32_t*>(base + t.xo_dec);
  X.rlist = reinterpret_cast<int32_t*>(base + t.xo_rl);
  volatile int* rcount = reinterpret_cast<volatile int*>(base + t.xo_rc);
  MT* msg = reinterpret_cast<MT*>(gs + t.xg_msg);
  float* lpost = reinterpret_cast<float*>(gs + t.xg_lpost);
  float* acc = reinterpret_cast<float*>(gs + t.xg_acc);
  uint32_t* cand = reinterpret_cast<uint32_t*>(gs + t.xg_cand);
  float* cpost = reinterpret_cast<float*>(gs + t.xg_cpost);

  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  uint32_t any = 0;
  if (PK) {
    for (int w = lane; w < mw; w += 32) {
      const int rem = m - 32 * w;
      const uint32_t x = __ldg(syn + w) & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
      X.s32[w] = x;
      any |= x;
    }
  } else {
    for (int c = lane; c < 4 * m4; c += 32) {
      const uint32_t b = c < m ? (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u : 0u;
      X.s8[c] = (uint8_t)b;
      any |= b;
    }
  }
  any = __any_sync(kFull, any);
  __syncwarp();
  ++my_shots;
  uint32_t* out_corr = a.corr + (size_t)shot * a.corr_stride;

  if (!any && !a.want_soft) {
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
    // member init: prior messages and summaries, decisions 0, parity = s
    {
      for (int c = lane; c < m; c += 32) X.summ[c] = __ldg(t.sum_init + c);
      const uint4* src = reinterpret_cast<const uint4*>(t.msg_csc);
      uint4* dst = reinterpret_cast<uint4*>(msg);
      const int nv = (int)(((size_t)t.E * sizeof(MT) + 15) / 16);
      for (int q = lane; q < nv; q += 32) __stcg(dst + q, __ldg(src + q));
      if (PK) {
        for (int w = lane; w < nw; w += 32) __stcg(X.dec + w, 0u);
        for (int w = lane; w < mw; w += 32) X.par32[w] = X.s32[w];
      } else {
        for (int w = lane; w < nw; w += 32) X.dec[w] = 0u;
        const uint32_t* s32 = reinterpret_cast<const uint32_t*>(X.s8);
        uint32_t* p32 = reinterpret_cast<uint32_t*>(X.par8);
        for (int q = lane; q < m4; q += 32) p32[q] = s32[q];
      }
      if (lane == 0) *rcount = 0;
    }
    __syncwarp();
    const uint2* rec = t.sched_rec + (size_t)i * n;
    const uint32_t* lo = t.lvl_off + (size_t)i * (n + 1);
    const int nl = __ldg(t.nlev + i);
    const float alpha = __ldg(t.alpha_m + i);   // member i's scaling factor
    int conv = 0;
    ColData<DP> cd;
    for (int it = 1; it <= budget; ++it) {
      // the posterior is needed after the last possible sweep of a member that may end without
      // converging (LLR average) and, for soft output, after every sweep
      float* lp = (a.want_soft || (it == T && ncand == 0)) ? lpost : nullptr;
      // the sweep in chunks of up to 32 columns of one level, one column per lane; rescans after each
      // chunk (later chunks of the same level touch other checks). Software pipeline: chunk j+1's
      // column data (checks, old messages, prior) is fetched before chunk j is updated -- a column's
      // messages are written only by that column, so the early read sees the same values -- and the
      // schedule records two chunks ahead.
      Chunk c = first_chunk(lo);
      Chunk c1 = next_chunk(c, lo, nl);
      Chunk c2 = next_chunk(c1, lo, nl);
      if (in_chunk(c, nl, lane)) fetch_column<MT, DP, PK>(__ldg(rec + c.cs + lane), t, msg, X.dec, cd);
      uint2 r1 = in_chunk(c1, nl, lane) ? __ldg(rec + c1.cs + lane) : make_uint2(0u, 0u);
      while (c.l < nl) {
        ColData<DP> cdn;
        if (in_chunk(c1, nl, lane)) fetch_column<MT, DP, PK>(r1, t, msg, X.dec, cdn);
        const uint2 r2 = in_chunk(c2, nl, lane) ? __ldg(rec + c2.cs + lane) : make_uint2(0u, 0u);
        if (in_chunk(c, nl, lane)) update_column_x<MT, DP, PK>(cd, t, alpha, msg, X, const_cast<int*>(rcount), lp);
        __syncwarp();
        const int nres = *rcount;
        if (nres > 0) {
          for (int q = 0; q < nres; ++q) rescan_row<MT>(X.rlist[q], t, msg, X.summ, lane);
          my_rescans += (unsigned long long)nres;
          __syncwarp();
          if (lane == 0) *rcount = 0;
          __syncwarp();
        }
        cd = cdn;
        r1 = r2;
        c = c1;
        c1 = c2;
        c2 = next_chunk(c2, lo, nl);
      }
      ++my_iters;
      uint32_t bad = 0;
      if (PK) {
        for (int w = lane; w < mw; w += 32) bad |= X.par32[w];
      } else {
        const uint32_t* p32 = reinterpret_cast<const uint32_t*>(X.par8);
        for (int q = lane; q < m4; q += 32) bad |= p32[q];
      }
      if (!__any_sync(kFull, bad)) { conv = it; break; }
    }
    if (conv) {
      // insert (conv, i); i exceeds every member already listed, so it goes after equal iterations
      const int p = __popc(__ballot_sync(kFull, lane < ncand && c_t <= conv));
      const int slot = ncand < M ? ncand : __shfl_sync(kFull, c_slot, M - 1);
      uint32_t* bits = cand + (size_t)slot * nw;
      for (int w = lane; w < nw; w += 32) bits[w] = PK ? __ldcg(X.dec + w) : X.dec[w];
      // W(e) = sum of lambda_j over e_j = 1, ascending j (every lane folds the same sequence)
      float W = 0.0f;
      for (int w = 0; w < nw; ++w) {
        uint32_t x = PK ? __ldcg(X.dec + w) : X.dec[w];
        while (x) {
          const int bpos = __ffs(x) - 1;
          W = __fadd_rn(W, __ldg(t.lam + 32 * w + bpos));
          x &= x - 1;
        }
      }
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
    if (lane == 0) a.lsd_shots[q] = shot;
    float* dst = a.lsd_soft + (size_t)q * a.bnd.n;
    const float kf = (float)K;
    for (int v = lane; v < n; v += 32) dst[v] = __fdiv_rn(acc[v], kf);
  }
  __syncwarp();
}

// MIXED: shots name their problems (dem_of_shot); the descriptors are copied to shared memory after
// the warps' regions and shots of image-engine problems are left to that kernel (mixed batches give
// every summary-engine problem the packed layout, PK). Otherwise every shot decodes a.one from the
// parameter space in layout PK.
template <typename MT, int DP, bool MIXED, bool PK>
__global__ void __launch_bounds__(kBpxWarpsPerCta * 32, MinBlocksX<MT>::value) k_bpx(const BpArgs a) {
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
  unsigned long long my_iters = 0, my_shots = 0, my_fail = 0, my_rescans = 0;

  for (;;) {
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
      decode_shot_x<MT, DP, PK>(a, sdem[di], shot, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
    } else {
      decode_shot_x<MT, DP, PK>(a, a.one, shot, base, gs, lane, my_iters, my_shots, my_fail, my_rescans);
    }
  }
  if (lane == 0 && a.counters) {
    atomicAdd(a.counters + VIBE_CNT_SHOTS, my_shots);
    atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, my_iters);
    if (my_fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, my_fail);
    if (my_rescans) atomicAdd(a.counters + VIBE_CNT_RESCANS, my_rescans);
  }
}

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename MT, int DP, bool MIXED, bool PK>
cudaError_t launch_x(const BpArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = ensure_dyn_smem<k_bpx<MT, DP, MIXED, PK>>(smem);
  if (err != cudaSuccess) return err;
  k_bpx<MT, DP, MIXED, PK><<<grid, kBpxWarpsPerCta * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename MT, int DP, bool MIXED, bool PK>
cudaError_t occupancy_x(size_t smem, int* out) {
  cudaError_t err = ensure_dyn_smem<k_bpx<MT, DP, MIXED, PK>>(smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bpx<MT, DP, MIXED, PK>, kBpxWarpsPerCta * 32, smem);
}

template <typename Fn>
cudaError_t by_dp_x(int DP, Fn&& f) {
  switch (DP) {
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    default: return cudaErrorInvalidValue;
  }
}

template <typename MT>
cudaError_t launch_x_mt(const BpArgs& a, int grid, cudaStream_t s) {
  const bool mixed = a.dem_of_shot != nullptr;
  const size_t smem = bpx_cta_smem_bytes(a.bnd, mixed ? a.ndem : 0);
  return by_dp_x(a.bnd.DP, [&](auto dp) {
    if (mixed) return launch_x<MT, decltype(dp)::value, true, true>(a, grid, smem, s);
    return a.one.x_packed ? launch_x<MT, decltype(dp)::value, false, true>(a, grid, smem, s)
                          : launch_x<MT, decltype(dp)::value, false, false>(a, grid, smem, s);
  });
}

template <typename MT>
cudaError_t occupancy_x_mt(const Bounds& b, int ndem, int* out) {
  const size_t smem = bpx_cta_smem_bytes(b, ndem);
  return by_dp_x(b.DP, [&](auto dp) {
    if (ndem > 0) return occupancy_x<MT, decltype(dp)::value, true, true>(smem, out);
    return b.x_packed ? occupancy_x<MT, decltype(dp)::value, false, true>(smem, out)
                      : occupancy_x<MT, decltype(dp)::value, false, false>(smem, out);
  });
}

}  // namespace

void bpx_layout(Tables* t, int msg_fp16) {
  const bool pk = t->x_packed != 0;
  const size_t flag_bytes = pk ? 4 * (size_t)t->mw : ((size_t)t->m + 3) / 4 * 4;   // syndrome / parity
  size_t o = 0;
  t->xo_summ = (int)o;  o = a16(o + 16 * (size_t)t->m);
  t->xo_s = (int)o;     o = a16(o + flag_bytes);
  t->xo_par = (int)o;   o = a16(o + flag_bytes);
  t->xo_dec = (int)o;   o = a16(o + (pk ? 0 : 4 * (size_t)t->nw));
  t->xo_rl = (int)o;    o = a16(o + 4 * 32 * (size_t)t->DP);
  t->xo_rc = (int)o;    o = a16(o + 4);
  t->x_warp_smem = (int)o;
  long long g = 0;
  t->xg_msg = g;   g += (long long)a16((size_t)t->E * (msg_fp16 ? 2 : 4));
  t->xg_dec = g;   g += (long long)a16(pk ? 4 * (size_t)t->nw : 0);
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
