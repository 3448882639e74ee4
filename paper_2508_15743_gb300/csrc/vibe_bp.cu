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
#include "vibe_internal.cuh"

namespace vibe {
namespace {

template <typename MT>
struct Msg;

template <>
struct Msg<float> {
  static constexpr uint32_t kInf = 0x7f800000u;
  // min |x| (as ordered bit patterns) and XOR of the raw words over 8 slots, skipping slot `skip`
  __device__ __forceinline__ static void scan8(const float* row8, int skip, uint32_t& mn, uint32_t& sg) {
    const float4 a = reinterpret_cast<const float4*>(row8)[0];
    const float4 b = reinterpret_cast<const float4*>(row8)[1];
    uint32_t u[8] = {__float_as_uint(a.x), __float_as_uint(a.y), __float_as_uint(a.z), __float_as_uint(a.w),
                     __float_as_uint(b.x), __float_as_uint(b.y), __float_as_uint(b.z), __float_as_uint(b.w)};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t keep = (j != skip) ? 0xffffffffu : 0u;
      mn = min(mn, (u[j] & 0x7fffffffu) | ~keep);
      sg ^= u[j] & keep;
    }
  }
  __device__ __forceinline__ static float min_value(uint32_t mn) { return __uint_as_float(mn); }
  __device__ __forceinline__ static uint32_t sign(uint32_t sg) { return sg >> 31; }
  __device__ __forceinline__ static void store(float* p, float x) { *p = x; }
};

template <>
struct Msg<__half> {
  static constexpr uint32_t kInf = 0x7c00u;
  __device__ __forceinline__ static void scan8(const __half* row8, int skip, uint32_t& mn, uint32_t& sg) {
    const uint4 q = *reinterpret_cast<const uint4*>(row8);
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t h = (w[j >> 1] >> ((j & 1) * 16)) & 0xffffu;
      uint32_t keep = (j != skip) ? 0xffffffffu : 0u;
      mn = min(mn, (h & 0x7fffu) | ~keep);
      sg ^= h & keep;
    }
  }
  __device__ __forceinline__ static float min_value(uint32_t mn) {
    return __half2float(__ushort_as_half((unsigned short)mn));
  }
  __device__ __forceinline__ static uint32_t sign(uint32_t sg) { return (sg >> 15) & 1u; }
  __device__ __forceinline__ static void store(__half* p, float x) {
    unsigned short h = __half_as_ushort(__float2half_rn(x));
    if (h == 0x8000u) h = 0;
    *reinterpret_cast<unsigned short*>(p) = h;
  }
};

__device__ __forceinline__ bool is_finite_bits(float x) {
  return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}

// One serial-V column update (R2, R3 of the oracle): check-to-variable messages from the current
// variable-to-check messages of the other columns, posterior, literal exclusion sums, decision.
template <typename MT, int DP>
__device__ __forceinline__ void update_column(uint32_t v, int deg, const Tables& t, float alpha, MT* msgs,
                                              float* post, const uint8_t* s8, uint8_t* par8) {
  uint32_t ent[DP];
  const uint4* ce = reinterpret_cast<const uint4*>(t.csc_ent + (size_t)v * DP);
#pragma unroll
  for (int q = 0; q < DP / 4; ++q) {
    uint4 x = __ldg(ce + q);
    ent[4 * q + 0] = x.x; ent[4 * q + 1] = x.y; ent[4 * q + 2] = x.z; ent[4 * q + 3] = x.w;
  }
  const float lamv = __ldg(t.lam + v);
  const int RP = t.RP;
  float mcv[DP];
#pragma unroll
  for (int k = 0; k < DP; ++k) {
    mcv[k] = 0.0f;
    if (k < deg) {
      const uint32_t c = ent[k] >> 8;
      const int slot = (int)(ent[k] & 0xffu);
      const MT* row = msgs + (size_t)c * RP;
      uint32_t mn = Msg<MT>::kInf, sg = 0;
      for (int ch = 0; ch < RP; ch += 8) Msg<MT>::scan8(row + ch, slot - ch, mn, sg);
      const uint32_t neg = Msg<MT>::sign(sg) ^ (uint32_t)s8[c];
      const float mag = __fmul_rn(alpha, Msg<MT>::min_value(mn));
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
      Msg<MT>::store(msgs + (size_t)(ent[k] >> 8) * RP + (ent[k] & 0xffu), a);
      pre = __fadd_rn(pre, mcv[k]);
    }
  }
  const bool e_new = L <= 0.0f;
  const bool e_old = post[v] <= 0.0f;
  if (e_new != e_old) {
#pragma unroll
    for (int k = 0; k < DP; ++k)
      if (k < deg) par8[ent[k] >> 8] ^= 1u;
  }
  post[v] = L;
}

template <typename MT, int DP>
__global__ void __launch_bounds__(kBpWarpsPerCta * 32) k_bp(const BpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tables& t = a.t;
  const int lane = threadIdx.x & 31;
  const int wcta = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * kBpWarpsPerCta + wcta;
  unsigned char* base = smem + (size_t)wcta * a.warp_smem;
  MT* msgs = reinterpret_cast<MT*>(base + a.off_msg);
  float* post = reinterpret_cast<float*>(base + a.off_post);
  uint8_t* s8 = base + a.off_s;
  uint8_t* par8 = base + a.off_par;
  uint32_t* cand = reinterpret_cast<uint32_t*>(base + a.off_cand);
  float* acc = a.scratch + gw * a.scratch_pitch;  // n floats
  float* cand_post = acc + t.n;                    // M * n floats (only with want_soft)

  const int n = t.n, m = t.m, K = t.K, M = a.M, T = a.T, nw = t.nw, mw = t.mw;
  const int m4 = (m + 3) >> 2;
  const int msg_vec = (int)(((size_t)m * t.RP * sizeof(MT)) / 16);
  unsigned long long my_iters = 0, my_shots = 0, my_fail = 0;

  for (;;) {
    uint32_t shot = 0;
    if (lane == 0) shot = atomicAdd(a.next_shot, 1u);
    shot = __shfl_sync(kFull, shot, 0);
    if (shot >= a.nshots) break;
    const uint32_t* syn = a.syn + (size_t)shot * mw;
    uint32_t any = 0;
    for (int c = lane; c < 4 * m4; c += 32) {
      uint32_t b = c < m ? (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u : 0u;
      s8[c] = (uint8_t)b;
      any |= b;
    }
    any = __any_sync(kFull, any);
    __syncwarp();
    ++my_shots;
    uint32_t* out_corr = a.corr + (size_t)shot * nw;

    if (!any && !a.want_soft) {
      // s = 0: every member converges in iteration 1 to e = 0; the first M are the candidates, all of
      // weight 0, so member 0 is chosen.
      for (int w = lane; w < nw; w += 32) out_corr[w] = 0u;
      if (a.logical)
        for (int w = lane; w < t.kw; w += 32) a.logical[(size_t)shot * t.kw + w] = 0u;
      if (a.obs) {
        uint32_t f = 0;
        for (int w = lane; w < t.kw; w += 32) f |= a.obs[(size_t)shot * t.kw + w];
        if (__any_sync(kFull, f) && lane == 0) ++my_fail;
      }
      if (a.stats && lane == 0) {
        vibe_shot_stats st;
        st.status = VIBE_STATUS_OK; st.lsd_invoked = 0; st.n_converged = (uint8_t)M; st.chosen_member = 0;
        st.iters = 1; st.largest_cluster = 0; st.n_clusters = 0;
        a.stats[shot] = st;
      }
      continue;
    }

    // candidate list, lane j holds entry j (sorted by iteration, then member)
    int ncand = 0;
    int c_t = 0, c_i = 0, c_slot = 0;
    float c_W = 0.0f;

    for (int i = 0; i < K; ++i) {
      const int budget = ncand < M ? T : __shfl_sync(kFull, c_t, M - 1) - 1;
      if (budget <= 0) break;
      // member init: messages = prior LLR image, posterior = lambda (decision 0), parity = s
      {
        const uint4* src = reinterpret_cast<const uint4*>(t.msg_init);
        uint4* dst = reinterpret_cast<uint4*>(msgs);
        for (int q = lane; q < msg_vec; q += 32) dst[q] = __ldg(src + q);
        for (int v = lane; v < n; v += 32) post[v] = __ldg(t.lam + v);
        const uint32_t* s32 = reinterpret_cast<const uint32_t*>(s8);
        uint32_t* p32 = reinterpret_cast<uint32_t*>(par8);
        for (int q = lane; q < m4; q += 32) p32[q] = s32[q];
      }
      __syncwarp();
      const uint32_t* sch = t.sched + (size_t)i * n;
      const uint32_t* lo = t.lvl_off + (size_t)i * (n + 1);
      const int nl = __ldg(t.nlev + i);
      int conv = 0;
      for (int it = 1; it <= budget; ++it) {
        for (int l = 0; l < nl; ++l) {
          const uint32_t b = __ldg(lo + l), e = __ldg(lo + l + 1);
          for (uint32_t idx = b + lane; idx < e; idx += 32) {
            const uint32_t ent = __ldg(sch + idx);
            update_column<MT, DP>(ent & 0xffffffu, (int)(ent >> 24), t, a.alpha, msgs, post, s8, par8);
          }
          __syncwarp();
        }
        ++my_iters;
        uint32_t bad = 0;
        const uint32_t* p32 = reinterpret_cast<const uint32_t*>(par8);
        for (int q = lane; q < m4; q += 32) bad |= p32[q];
        if (!__any_sync(kFull, bad)) { conv = it; break; }
      }
      if (conv) {
        // insert (conv, i); i exceeds every member already listed, so it goes after equal iterations
        const int p = __popc(__ballot_sync(kFull, lane < ncand && c_t <= conv));
        const int slot = ncand < M ? ncand : __shfl_sync(kFull, c_slot, M - 1);
        uint32_t* bits = cand + (size_t)slot * nw;
        float W = 0.0f;
        for (int w = 0; w < nw; ++w) {
          const int v = 32 * w + lane;
          const uint32_t word = __ballot_sync(kFull, v < n && post[v] <= 0.0f);
          if (lane == 0) bits[w] = word;
          uint32_t x = word;
          while (x) {
            const int bpos = __ffs(x) - 1;
            W = __fadd_rn(W, __ldg(t.lam + 32 * w + bpos));
            x &= x - 1;
          }
        }
        if (a.want_soft) {
          float* dst = cand_post + (size_t)slot * n;
          for (int v = lane; v < n; v += 32) dst[v] = post[v];
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
          const float x = post[v];
          part = __fadd_rn(part, is_finite_bits(x) ? __fmul_rn(x, x) : 0.0f);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) part = __fadd_rn(part, __shfl_xor_sync(kFull, part, off));
        const float nrm = __fsqrt_rn(part);
        for (int v = lane; v < n; v += 32) {
          const float x = post[v];
          const float term = is_finite_bits(x) ? (nrm == 0.0f ? 0.0f : __fdiv_rn(x, nrm)) : x;
          acc[v] = __fadd_rn(i == 0 ? 0.0f : acc[v], term);
        }
      }
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
        float* dst = a.soft + (size_t)shot * n;
        for (int v = lane; v < n; v += 32) dst[v] = src[v];
      }
      uint32_t fail = 0;
      for (int rb = 0; rb < t.kw; ++rb) {
        const int r = 32 * rb + lane;
        uint32_t par = 0;
        if (r < t.k)
          for (int e = __ldg(t.lrowptr + r); e < __ldg(t.lrowptr + r + 1); ++e) {
            const int j = __ldg(t.lcolidx + e);
            par ^= (bits[j >> 5] >> (j & 31)) & 1u;
          }
        const uint32_t word = __ballot_sync(kFull, par != 0);
        if (a.logical && lane == 0) a.logical[(size_t)shot * t.kw + rb] = word;
        if (a.obs) fail |= word ^ a.obs[(size_t)shot * t.kw + rb];
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
      float* dst = a.lsd_soft + (size_t)q * n;
      const float kf = (float)K;
      for (int v = lane; v < n; v += 32) dst[v] = __fdiv_rn(acc[v], kf);
    }
    __syncwarp();
  }
  if (lane == 0 && a.counters) {
    atomicAdd(a.counters + VIBE_CNT_SHOTS, my_shots);
    atomicAdd(a.counters + VIBE_CNT_PAIR_ITERS, my_iters);
    if (my_fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, my_fail);
  }
}

template <typename MT>
cudaError_t launch_dp(const BpArgs& a, int grid, cudaStream_t s) {
  const size_t smem = (size_t)a.warp_smem * kBpWarpsPerCta;
  const dim3 block(kBpWarpsPerCta * 32);
  cudaError_t err;
  switch (a.t.DP) {
#define VIBE_BP_CASE(D)                                                                             \
  case D:                                                                                           \
    err = cudaFuncSetAttribute(k_bp<MT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (err != cudaSuccess) return err;                                                             \
    k_bp<MT, D><<<grid, block, smem, s>>>(a);                                                       \
    return cudaGetLastError();
    VIBE_BP_CASE(4)
    VIBE_BP_CASE(8)
    VIBE_BP_CASE(16)
    VIBE_BP_CASE(32)
#undef VIBE_BP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename MT>
cudaError_t occupancy_dp(int DP, size_t smem, int* out) {
  const int threads = kBpWarpsPerCta * 32;
  cudaError_t err;
  switch (DP) {
#define VIBE_OCC_CASE(D)                                                                            \
  case D:                                                                                           \
    err = cudaFuncSetAttribute(k_bp<MT, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (err != cudaSuccess) return err;                                                             \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_bp<MT, D>, threads, smem);
    VIBE_OCC_CASE(4)
    VIBE_OCC_CASE(8)
    VIBE_OCC_CASE(16)
    VIBE_OCC_CASE(32)
#undef VIBE_OCC_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

}  // namespace

size_t bp_warp_smem_bytes(const Tables& t, int M, int msg_fp16, int* off_msg, int* off_post, int* off_s,
                          int* off_par, int* off_cand) {
  size_t o = 0;
  *off_msg = (int)o;
  o = align16(o + (size_t)t.m * t.RP * (msg_fp16 ? 2 : 4));
  *off_post = (int)o;
  o = align16(o + (size_t)t.n * 4);
  const size_t m4 = ((size_t)t.m + 3) / 4 * 4;
  *off_s = (int)o;
  o = align16(o + m4);
  *off_par = (int)o;
  o = align16(o + m4);
  *off_cand = (int)o;
  o = align16(o + (size_t)M * t.nw * 4);
  return o;
}

cudaError_t launch_bp(const BpArgs& a, int msg_fp16, int grid, cudaStream_t s) {
  return msg_fp16 ? launch_dp<__half>(a, grid, s) : launch_dp<float>(a, grid, s);
}

cudaError_t bp_occupancy(const Tables& t, int msg_fp16, size_t cta_smem, int* blocks_per_sm) {
  return msg_fp16 ? occupancy_dp<__half>(t.DP, cta_smem, blocks_per_sm)
                  : occupancy_dp<float>(t.DP, cta_smem, blocks_per_sm);
}

}  // namespace vibe
