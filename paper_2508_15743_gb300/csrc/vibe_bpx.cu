// K1' -- the BP ensemble for problems whose message image does not fit in shared memory (circuit-level
// detector error models: rows of 100-200 entries, E up to ~4e5). Same method, same results as the warp
// engine (vibe_bp.cu); a different layout.
//
// One CTA decodes one shot at a time (persistent, shots from a global counter), running the members
// one after another with the iteration budget of the correction limit (Sec. III.D.2). A member sweeps
// the dependency wavefronts of its schedule; the threads of the CTA take the columns of one level, then
// the CTA synchronises.
//
// Check-node state. For every check c the CTA keeps in shared memory a 16-byte summary of the current
// variable-to-check messages of its row: the smallest magnitude, the second smallest (with
// multiplicity, +inf for a one-entry row), the edge holding the smallest, and the parity of the sign
// bits. The magnitude minimum over the row without edge e is then (e == holder ? second : smallest),
// and the sign parity without e is parity XOR sign(m_e): exactly the minimum and sign product that
// Algorithm 1's check update takes over N(c) \ v, with no row scan. The messages themselves (E floats or
// halves per CTA, in CSC edge order so that a column's are contiguous) stay in global memory, where the
// column update reads its old values and writes the new ones.
//
// Keeping the summary exact after column v replaces its message on c (old magnitude o, new x):
//   v holds the smallest:  x <= second -> smallest = x;  else the row is rescanned;
//   o == second (v may hold it): x > second -> rescan; x < smallest -> v becomes the holder and the old
//                          smallest the second; else second = x;
//   otherwise:             x < smallest -> shift; x < second -> second = x.
// Every check is touched by one column per level, so the updates of a level never collide. Rescans
// are queued and done after the level by one warp per check (a minimum/second-minimum reduction over
// the row's messages), before any later level reads the summary.
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

// Shared state of the CTA for its current shot.
struct XShared {
  float4* summ;     // m check summaries (smallest, second, holder edge bits, sign parity bits)
  uint8_t* s8;      // m syndrome bits
  uint8_t* par8;    // m: (H e)_c XOR s_c
  uint32_t* dec;    // nw: the member's decisions e, bit-packed
  int32_t* rlist;   // m: checks to rescan after the current level
  int* ctl;         // control words (see k_bpx)
};

// Serial-V update of column v (deg checks, edges e0 .. e0 + deg - 1 in ascending check order).
template <typename MT, int DP>
__device__ __forceinline__ void update_column_x(uint32_t v, int deg, const Tables& t, MT* msg, const XShared& X,
                                                int* rcount, float* lpost) {
  const uint32_t e0 = (uint32_t)__ldg(t.colptr + v);
  int c[DP];
  float o[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    c[k] = 0;
    o[k] = 0.0f;
    if (k < deg) {
      c[k] = __ldg(t.rowidx + e0 + k);
      o[k] = XMsg<MT>::value(XMsg<MT>::load(msg + e0 + k));
    }
  }
  const float lamv = __ldg(t.lam + v);
  const float alpha = t.alpha;
  float mcv[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    mcv[k] = 0.0f;
    if (k < deg) {
      const float4 sm = X.summ[c[k]];
      const bool holder = __float_as_uint(sm.z) == e0 + k;
      const float mn = holder ? sm.y : sm.x;
      const uint32_t neg = (__float_as_uint(sm.w) ^ sign_bit(o[k]) ^ (uint32_t)X.s8[c[k]]) & 1u;
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
      const float om = fabsf(o[k]), nm = fabsf(x);
      float4 s = X.summ[c[k]];   // this level's only reader and writer of check c
      s.w = __uint_as_float(__float_as_uint(s.w) ^ sign_bit(o[k]) ^ sign_bit(x));
      bool rescan = false;
      if (__float_as_uint(s.z) == e0 + k) {
        if (nm <= s.y) s.x = nm;
        else rescan = true;
      } else if (om == s.y && nm > s.y) {
        rescan = true;
      } else if (nm < s.x) {
        s.y = s.x; s.x = nm; s.z = __uint_as_float(e0 + k);
      } else if (nm < s.y) {
        s.y = nm;
      }
      X.summ[c[k]] = s;
      if (rescan) X.rlist[atomicAdd(rcount, 1)] = c[k];
    }
  }
  const uint32_t e_new = L <= 0.0f ? 1u : 0u;
  const uint32_t bit = 1u << (v & 31);
  const uint32_t e_old = (X.dec[v >> 5] & bit) ? 1u : 0u;
  if (e_new != e_old) {
    atomicXor(&X.dec[v >> 5], bit);
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k < deg) X.par8[c[k]] ^= 1u;
  }
  if (lpost) lpost[v] = L;
}

// Warp-cooperative rescan of check c: smallest and second smallest magnitude (with multiplicity) and
// the edge of the smallest over the row's current messages; the sign parity is kept as it is.
template <typename MT>
__device__ __forceinline__ void rescan_row(int c, const Tables& t, const MT* msg, float4* summ, int lane) {
  float m1 = __int_as_float(0x7f800000), m2 = m1;
  uint32_t i1 = 0xffffffffu;
  const int b = __ldg(t.rowptr + c), e = __ldg(t.rowptr + c + 1);
  for (int q = b + lane; q < e; q += 32) {
    const uint32_t ed = __ldg(t.row_edge + q);
    const float a = fabsf(XMsg<MT>::value(XMsg<MT>::load(msg + ed)));
    if (a < m1 || (a == m1 && ed < i1)) { m2 = m1; m1 = a; i1 = ed; }
    else if (a < m2) m2 = a;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const float n1 = __shfl_xor_sync(kFull, m1, off), n2 = __shfl_xor_sync(kFull, m2, off);
    const uint32_t j1 = __shfl_xor_sync(kFull, i1, off);
    if (n1 < m1 || (n1 == m1 && j1 < i1)) {
      m2 = fminf(n2, m1);
      m1 = n1;
      i1 = j1;
    } else {
      m2 = fminf(m2, n1);
    }
  }
  if (lane == 0) {
    float4 s = summ[c];
    s.x = m1; s.y = m2; s.z = __uint_as_float(i1);
    summ[c] = s;
  }
}

// control words in static shared memory
enum : int { C_SHOT = 0, C_RC = 1 /* 3 rescan counters */, C_SLOT = 4, C_Q = 5, C_BEST = 6, C_ITERS = 7, C_NCTL = 8 };

struct XCand {
  int t[32], i[32], slot[32];
  float W[32];
  float nrm;
};

// Decodes shot `shot` of problem t with the whole CTA.
template <typename MT, int DP>
__device__ __forceinline__ void decode_shot_x(const BpArgs& a, const Tables& t, uint32_t shot, unsigned char* smem,
                                              unsigned char* gs, int* ctl, XCand& cl, uint32_t& gl,
                                              unsigned long long& my_iters, unsigned long long& my_shots,
                                              unsigned long long& my_fail) {
  constexpr int NT = kBpxThreads, NWARP = kBpxThreads / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = t.n, m = t.m, K = t.K, M = t.M, T = t.T, nw = t.nw, kw = t.kw;
  const int m4 = (m + 3) >> 2;
  XShared X;
  X.summ = reinterpret_cast<float4*>(smem + t.xo_summ);
  X.s8 = smem + t.xo_s;
  X.par8 = smem + t.xo_par;
  X.dec = reinterpret_cast<uint32_t*>(smem + t.xo_dec);
  X.rlist = reinterpret_cast<int32_t*>(smem + t.xo_rl);
  X.ctl = ctl;
  MT* msg = reinterpret_cast<MT*>(gs + t.xg_msg);
  float* lpost = reinterpret_cast<float*>(gs + t.xg_lpost);
  float* acc = reinterpret_cast<float*>(gs + t.xg_acc);
  uint32_t* cand = reinterpret_cast<uint32_t*>(gs + t.xg_cand);
  float* cpost = reinterpret_cast<float*>(gs + t.xg_cpost);

  const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;
  uint32_t any = 0;
  for (int c = tid; c < 4 * m4; c += NT) {
    const uint32_t b = c < m ? (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u : 0u;
    X.s8[c] = (uint8_t)b;
    any |= b;
  }
  const int anyS = __syncthreads_or(any != 0);
  if (tid == 0) ++my_shots;
  uint32_t* out_corr = a.corr + (size_t)shot * a.corr_stride;

  if (!anyS && !a.want_soft) {
    // s = 0: every member converges in iteration 1 to e = 0; member 0 is chosen
    for (int w = tid; w < nw; w += NT) out_corr[w] = 0u;
    if (a.logical)
      for (int w = tid; w < kw; w += NT) a.logical[(size_t)shot * a.log_stride + w] = 0u;
    if (warp == 0 && a.obs) {
      uint32_t f = 0;
      for (int w = lane; w < kw; w += 32) f |= a.obs[(size_t)shot * a.log_stride + w];
      if (__any_sync(kFull, f) && lane == 0) ++my_fail;
    }
    if (a.stats && tid == 0) {
      vibe_shot_stats st;
      st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)M; st.chosen_member = 0;
      st.iters = 1; st.largest_cluster = 0; st.n_clusters = 0;
      a.stats[shot] = st;
    }
    __syncthreads();
    return;
  }

  int ncand = 0;   // the same in every thread
  for (int i = 0; i < K; ++i) {
    const int budget = ncand < M ? T : cl.t[M - 1] - 1;
    if (budget <= 0) break;
    // member init: prior messages and summaries, decisions 0, parity = s
    {
      for (int c = tid; c < m; c += NT) X.summ[c] = __ldg(t.sum_init + c);
      const uint4* src = reinterpret_cast<const uint4*>(t.msg_csc);
      uint4* dst = reinterpret_cast<uint4*>(msg);
      const int nv = (int)(((size_t)t.E * sizeof(MT) + 15) / 16);
      for (int q = tid; q < nv; q += NT) __stcg(dst + q, __ldg(src + q));
      for (int w = tid; w < nw; w += NT) X.dec[w] = 0u;
      const uint32_t* s32 = reinterpret_cast<const uint32_t*>(X.s8);
      uint32_t* p32 = reinterpret_cast<uint32_t*>(X.par8);
      for (int q = tid; q < m4; q += NT) p32[q] = s32[q];
    }
    __syncthreads();
    const uint32_t* sch = t.sched + (size_t)i * n;
    const uint32_t* lo = t.lvl_off + (size_t)i * (n + 1);
    const int nl = __ldg(t.nlev + i);
    int conv = 0;
    for (int it = 1; it <= budget; ++it) {
      float* lp = (a.want_soft || (it == T && ncand == 0)) ? lpost : nullptr;
      for (int l = 0; l < nl; ++l, ++gl) {
        // rescan counters rotate over three words: the one zeroed here was last read two levels ago
        if (tid == 0) ctl[C_RC + (gl + 1) % 3] = 0;
        int* rc = ctl + C_RC + gl % 3;
        const uint32_t b = __ldg(lo + l), e = __ldg(lo + l + 1);
        for (uint32_t idx = b + tid; idx < e; idx += NT) {
          const uint32_t ent = __ldg(sch + idx);
          update_column_x<MT, DP>(ent & 0xffffffu, (int)(ent >> 24), t, msg, X, rc, lp);
        }
        __syncthreads();
        const int nres = *rc;
        if (nres > 0) {
          for (int q = warp; q < nres; q += NWARP) rescan_row<MT>(X.rlist[q], t, msg, X.summ, lane);
          __syncthreads();
        }
      }
      if (tid == 0) ++my_iters;
      uint32_t bad = 0;
      const uint32_t* p32 = reinterpret_cast<const uint32_t*>(X.par8);
      for (int q = tid; q < m4; q += NT) bad |= p32[q];
      if (!__syncthreads_or(bad != 0)) { conv = it; break; }
    }
    if (conv) {
      if (tid == 0) {
        // W(e) = sum of lambda_j over e_j = 1, ascending j
        float W = 0.0f;
        for (int w = 0; w < nw; ++w) {
          uint32_t x = X.dec[w];
          while (x) {
            const int bpos = __ffs(x) - 1;
            W = __fadd_rn(W, __ldg(t.lam + 32 * w + bpos));
            x &= x - 1;
          }
        }
        // insert (conv, i) after the entries with t <= conv; a full list drops its last entry
        int p = 0;
        while (p < ncand && cl.t[p] <= conv) ++p;
        const int slot = ncand < M ? ncand : cl.slot[M - 1];
        const int last = min(ncand, M - 1);
        for (int j = last; j > p; --j) {
          cl.t[j] = cl.t[j - 1]; cl.i[j] = cl.i[j - 1]; cl.slot[j] = cl.slot[j - 1]; cl.W[j] = cl.W[j - 1];
        }
        if (p <= last) { cl.t[p] = conv; cl.i[p] = i; cl.slot[p] = slot; cl.W[p] = W; }
        ctl[C_SLOT] = slot;
      }
      __syncthreads();
      const int slot = ctl[C_SLOT];
      for (int w = tid; w < nw; w += NT) cand[(size_t)slot * nw + w] = X.dec[w];
      if (a.want_soft)
        for (int v = tid; v < n; v += NT) cpost[(size_t)slot * n + v] = lpost[v];
      ncand = min(ncand + 1, M);
    } else if (ncand == 0) {
      // not converged after T sweeps and no candidate yet: add LLR^i / ||LLR^i|| (finite entries);
      // the norm is the canonical 32-partial sum with an XOR-butterfly combine
      if (warp == 0) {
        float part = 0.0f;
        for (int v = lane; v < n; v += 32) {
          const float x = lpost[v];
          part = __fadd_rn(part, is_finite_bits(x) ? __fmul_rn(x, x) : 0.0f);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) part = __fadd_rn(part, __shfl_xor_sync(kFull, part, off));
        if (lane == 0) cl.nrm = __fsqrt_rn(part);
      }
      __syncthreads();
      const float nrm = cl.nrm;
      for (int v = tid; v < n; v += NT) {
        const float x = lpost[v];
        const float term = is_finite_bits(x) ? (nrm == 0.0f ? 0.0f : __fdiv_rn(x, nrm)) : x;
        acc[v] = __fadd_rn(i == 0 ? 0.0f : acc[v], term);
      }
    }
    __syncthreads();
  }

  if (ncand > 0) {
    if (tid == 0) {
      int best = 0;   // first minimum of W over the list
      for (int j = 1; j < ncand; ++j)
        if (cl.W[j] < cl.W[best]) best = j;
      ctl[C_BEST] = best;
      ctl[C_ITERS] = ncand == M ? cl.t[M - 1] : T;
    }
    __syncthreads();
    const int best = ctl[C_BEST];
    const int slot = cl.slot[best];
    const uint32_t* bits = cand + (size_t)slot * nw;
    for (int w = tid; w < nw; w += NT) out_corr[w] = bits[w];
    if (a.want_soft) {
      const float* src = cpost + (size_t)slot * n;
      float* dst = a.soft + (size_t)shot * a.soft_stride;
      for (int v = tid; v < n; v += NT) dst[v] = src[v];
    }
    if (warp == 0) {
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
        st.chosen_member = (uint8_t)cl.i[best]; st.iters = (uint16_t)ctl[C_ITERS];
        st.largest_cluster = 0; st.n_clusters = 0;
        a.stats[shot] = st;
      }
    }
  } else {
    // hand the averaged soft vector to the LSD kernel
    if (tid == 0) {
      const unsigned int q = atomicAdd(a.lsd_count, 1u);
      a.lsd_shots[q] = shot;
      ctl[C_Q] = (int)q;
    }
    __syncthreads();
    float* dst = a.lsd_soft + (size_t)(unsigned)ctl[C_Q] * a.bnd.n;
    const float kf = (float)K;
    for (int v = tid; v < n; v += NT) dst[v] = __fdiv_rn(acc[v], kf);
  }
  __syncthreads();
}

// MIXED: shots name their problems (dem_of_shot); the descriptors are copied to shared memory after
// the CTA's layout and shots of warp-engine problems are left to that kernel. Otherwise every shot
// decodes a.one from the parameter space.
template <typename MT, int DP, bool MIXED>
__global__ void __launch_bounds__(kBpxThreads, 2) k_bpx(const BpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int ctl[C_NCTL];
  __shared__ XCand cl;
  const int tid = threadIdx.x;
  Tables* sdem = reinterpret_cast<Tables*>(smem + a.bnd.cta_smem);
  if (MIXED) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.dems);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sdem);
    const int words = a.ndem * (int)(sizeof(Tables) / 4);
    for (int q = tid; q < words; q += kBpxThreads) dst[q] = __ldg(src + q);
  }
  if (tid < C_NCTL) ctl[tid] = 0;
  unsigned char* gs = a.xscratch + (long long)blockIdx.x * a.xscratch_pitch;
  unsigned long long my_iters = 0, my_shots = 0, my_fail = 0;
  uint32_t gl = 0;   // levels swept by this CTA (rotates the rescan counters)

  for (;;) {
    __syncthreads();
    if (tid == 0) ctl[C_SHOT] = (int)atomicAdd(a.next_shot_x, 1u);
    __syncthreads();
    const uint32_t shot = (uint32_t)ctl[C_SHOT];
    if (shot >= a.nshots) break;
    if (MIXED) {
      const int di = __ldg(a.dem_of_shot + shot);
      if ((unsigned)di >= (unsigned)a.ndem) {
        if (!a.flag_bad) continue;
        for (int w = tid; w < a.corr_stride; w += kBpxThreads) a.corr[(size_t)shot * a.corr_stride + w] = 0u;
        if (a.logical)
          for (int w = tid; w < a.log_stride; w += kBpxThreads) a.logical[(size_t)shot * a.log_stride + w] = 0u;
        if (a.soft)
          for (int j = tid; j < a.soft_stride; j += kBpxThreads) a.soft[(size_t)shot * a.soft_stride + j] = 0.0f;
        if (tid == 0) {
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
      if (sdem[di].engine != VIBE_ENGINE_CTA) continue;
      decode_shot_x<MT, DP>(a, sdem[di], shot, smem, gs, ctl, cl, gl, my_iters, my_shots, my_fail);
    } else {
      decode_shot_x<MT, DP>(a, a.one, shot, smem, gs, ctl, cl, gl, my_iters, my_shots, my_fail);
    }
  }
  if (tid == 0 && a.counters) {
    atomicAdd(a.counters + VIBE_CNT_SHOTS, my_shots);
    atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, my_iters);
  }
  if ((tid & 31) == 0 && a.counters && my_fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, my_fail);
}

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

template <typename MT, int DP, bool MIXED>
cudaError_t launch_x(const BpArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = ensure_dyn_smem<k_bpx<MT, DP, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  k_bpx<MT, DP, MIXED><<<grid, kBpxThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename MT, int DP, bool MIXED>
cudaError_t occupancy_x(size_t smem, int* out) {
  cudaError_t err = ensure_dyn_smem<k_bpx<MT, DP, MIXED>>(smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bpx<MT, DP, MIXED>, kBpxThreads, smem);
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
    return mixed ? launch_x<MT, decltype(dp)::value, true>(a, grid, smem, s)
                 : launch_x<MT, decltype(dp)::value, false>(a, grid, smem, s);
  });
}

template <typename MT>
cudaError_t occupancy_x_mt(const Bounds& b, int ndem, int* out) {
  const size_t smem = bpx_cta_smem_bytes(b, ndem);
  return by_dp_x(b.DP, [&](auto dp) {
    return ndem > 0 ? occupancy_x<MT, decltype(dp)::value, true>(smem, out)
                    : occupancy_x<MT, decltype(dp)::value, false>(smem, out);
  });
}

}  // namespace

void bpx_layout(Tables* t, int msg_fp16) {
  const size_t m4 = ((size_t)t->m + 3) / 4 * 4;
  size_t o = 0;
  t->xo_summ = (int)o;  o = a16(o + 16 * (size_t)t->m);
  t->xo_s = (int)o;     o = a16(o + m4);
  t->xo_par = (int)o;   o = a16(o + m4);
  t->xo_dec = (int)o;   o = a16(o + 4 * (size_t)t->nw);
  t->xo_rl = (int)o;    o = a16(o + 4 * (size_t)t->m);
  t->cta_smem = (int)o;
  long long g = 0;
  t->xg_msg = g;   g += (long long)a16((size_t)t->E * (msg_fp16 ? 2 : 4));
  t->xg_lpost = g; g += (long long)a16(4 * (size_t)t->n);
  t->xg_acc = g;   g += (long long)a16(4 * (size_t)t->n);
  t->xg_cand = g;  g += (long long)a16(4 * (size_t)t->M * t->nw);
  t->xg_cpost = g;
  t->cta_scratch = g;
}

size_t bpx_cta_smem_bytes(const Bounds& b, int ndem) {
  return (size_t)b.cta_smem + a16((size_t)ndem * sizeof(Tables));
}

cudaError_t launch_bpx(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s) {
  return msg_fp16 ? launch_x_mt<__half>(a, grid, s) : launch_x_mt<float>(a, grid, s);
}

cudaError_t bpx_occupancy(const Bounds& b, int ndem, int msg_fp16, int* blocks_per_sm) {
  return msg_fp16 ? occupancy_x_mt<__half>(b, ndem, blocks_per_sm) : occupancy_x_mt<float>(b, ndem, blocks_per_sm);
}

}  // namespace vibe
