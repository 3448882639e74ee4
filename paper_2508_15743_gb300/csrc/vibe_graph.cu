// K0 -- Tanner-graph builder (offline setup, Sec. III.D.1).
//
// From the CSR of H it builds, on the device: the CSC of H (checks ascending per column), the packed
// per-column edge table csc_ent used by the BP kernel, the padded message image (prior LLR of each
// edge's column, +inf padding), and for every ensemble member the dependency wavefronts of its
// serial schedule: level(v) = 1 + max{level(u) : u before v in the member's order, u and v share a
// check}. Columns of one level touch disjoint checks, so updating a level in any order gives the
// same floats as the serial order of Algorithm 1 (serial branch).
#include "vibe_internal.cuh"

namespace vibe {
namespace {

__global__ void k_col_count(const int32_t* __restrict__ colidx, int E, int32_t* __restrict__ cnt) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x)
    atomicAdd(&cnt[colidx[e]], 1);
}

// Exclusive scan of cnt[0..n) into out[0..n], one CTA (used once per handle).
__global__ void k_scan_single(const int32_t* __restrict__ cnt, int n, int32_t* __restrict__ out) {
  __shared__ int32_t part[1024];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < n ? cnt[i] : 0;
    part[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      int add = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (i < n) out[i] = carry + part[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Scatter every edge into its column as (check << 8) | slot, slot = position inside the check row.
__global__ void k_csc_fill(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int m,
                           const int32_t* __restrict__ colptr, int32_t* __restrict__ fill,
                           uint32_t* __restrict__ packed) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    for (int e = rowptr[c]; e < rowptr[c + 1]; ++e) {
      int v = colidx[e];
      int pos = atomicAdd(&fill[v], 1);
      packed[colptr[v] + pos] = ((uint32_t)c << 8) | (uint32_t)(e - rowptr[c]);
    }
  }
}

// Sort each column's entries by check (insertion sort, degree <= 32) and emit rowidx, csc_ent and the
// summary engine's column records xcol (XP words per column: (check << 8) | position of the edge in
// the check's CSR row, ascending check, zero padded; none when XP == 0).
__global__ void k_csc_finish(int n, int DP, int RP, int spc, int XP, const int32_t* __restrict__ colptr,
                             uint32_t* __restrict__ packed, int32_t* __restrict__ rowidx,
                             uint32_t* __restrict__ csc_ent, uint32_t* __restrict__ xcol) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int b = colptr[v], d = colptr[v + 1] - b;
    for (int i = 1; i < d; ++i) {
      uint32_t x = packed[b + i];
      int j = i - 1;
      while (j >= 0 && packed[b + j] > x) { packed[b + j + 1] = packed[b + j]; --j; }
      packed[b + j + 1] = x;
    }
    for (int k = 0; k < DP; ++k) {
      uint32_t x = k < d ? packed[b + k] : 0u;
      csc_ent[(size_t)v * DP + k] = k < d ? csc_entry(x >> 8, x & 0xffu, RP, spc) : 0u;
      if (k < d) rowidx[b + k] = (int32_t)(x >> 8);
    }
    for (int k = 0; k < XP; ++k) xcol[(size_t)v * XP + k] = k < d ? packed[b + k] : 0u;
  }
}

template <typename MT>
__device__ __forceinline__ MT to_msg(float x);
template <>
__device__ __forceinline__ float to_msg<float>(float x) { return x; }
template <>
__device__ __forceinline__ __half to_msg<__half>(float x) { return __float2half_rn(x); }

template <typename MT>
__global__ void k_msg_init(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int m, int RP,
                           const float* __restrict__ lam, MT* __restrict__ out) {
  const int spc = 16 / (int)sizeof(MT);
  long long total = (long long)m * RP;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / RP), pos = (int)(t % RP);
    const int slot = (int)row_position((uint32_t)c, (uint32_t)pos, RP, spc);   // the XOR swizzle is its own inverse
    const int deg = rowptr[c + 1] - rowptr[c];
    float x = slot < deg ? lam[colidx[rowptr[c] + slot]] : __int_as_float(0x7f800000);
    out[t] = to_msg<MT>(x);
  }
}

template <typename MT>
__device__ __forceinline__ float msg_magnitude(MT x);
template <>
__device__ __forceinline__ float msg_magnitude<float>(float x) { return fabsf(x); }
template <>
__device__ __forceinline__ float msg_magnitude<__half>(__half x) { return fabsf(__half2float(x)); }

// Summary engine: the summary of each check's prior messages -- the two smallest magnitudes (ordered by
// value, then row position) with their positions, the third smallest as the floor (+inf when the row
// is shorter; a missing second holder is position 255 with +inf), two valid holders, and the parity
// of the messages' sign bits (bit 18). The syndrome and parity bits are set per shot by the kernel.
template <typename MT>
__global__ void k_xsum(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, int m,
                       const float* __restrict__ lam, float4* __restrict__ out) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    const float inf = __int_as_float(0x7f800000);
    float a1 = inf, a2 = inf, a3 = inf;
    uint32_t q1 = 255u, q2 = 255u, sg = 0u;
    for (int q = rowptr[c]; q < rowptr[c + 1]; ++q) {
      const MT x = to_msg<MT>(lam[colidx[q]]);
      const float a = msg_magnitude<MT>(x);
      const uint32_t p = (uint32_t)(q - rowptr[c]);
      sg ^= (float)x < 0.0f ? 1u : 0u;
      if (a < a1 || (a == a1 && p < q1)) { a3 = a2; a2 = a1; q2 = q1; a1 = a; q1 = p; }
      else if (a < a2 || (a == a2 && p < q2)) { a3 = a2; a2 = a; q2 = p; }
      else if (a < a3) a3 = a;
    }
    out[c] = make_float4(a1, a2, a3, __uint_as_float(q1 | (q2 << 8) | (2u << 16) | (sg << 18)));
  }
}

// One thread per member: dependency levels of its schedule, then a stable counting sort into levels
// and, inside each level, by column degree (lanes of a warp then see similar work).
__global__ void k_levels(const uint32_t* __restrict__ perm, int n, int m, int K, const int32_t* __restrict__ colptr,
                         const int32_t* __restrict__ rowidx, uint32_t* __restrict__ sched,
                         uint32_t* __restrict__ lvl_off, int32_t* __restrict__ nlev, int32_t* __restrict__ scratch) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  size_t per = (size_t)m + 3 * (size_t)n + 1;
  int32_t* last = scratch + per * i;       // m: level of the latest column seen at each check
  int32_t* lev = last + m;                 // n
  int32_t* cnt = lev + n;                  // n + 1
  int32_t* tmp = cnt + n + 1;              // n
  for (int c = 0; c < m; ++c) last[c] = -1;
  const uint32_t* p = perm + (size_t)i * n;
  int nl = 0;
  for (int t = 0; t < n; ++t) {
    int v = (int)p[t];
    int l = 0;
    for (int e = colptr[v]; e < colptr[v + 1]; ++e) l = max(l, last[rowidx[e]] + 1);
    for (int e = colptr[v]; e < colptr[v + 1]; ++e) last[rowidx[e]] = l;
    lev[v] = l;
    nl = max(nl, l + 1);
  }
  for (int l = 0; l <= nl; ++l) cnt[l] = 0;
  for (int v = 0; v < n; ++v) cnt[lev[v]]++;
  uint32_t* off = lvl_off + (size_t)i * (n + 1);
  int run = 0;
  for (int l = 0; l < nl; ++l) { off[l] = run; int c = cnt[l]; cnt[l] = run; run += c; }
  off[nl] = run;
  for (int v = 0; v < n; ++v) tmp[cnt[lev[v]]++] = v;   // stable: ascending v inside a level
  uint32_t* out = sched + (size_t)i * n;
  for (int l = 0; l < nl; ++l) {
    int b = off[l], e = off[l + 1];
    int dc[kMaxColDeg + 2];
    for (int d = 0; d <= kMaxColDeg + 1; ++d) dc[d] = 0;
    for (int t = b; t < e; ++t) { int v = tmp[t]; dc[colptr[v + 1] - colptr[v]]++; }
    int r = b;
    for (int d = 0; d <= kMaxColDeg; ++d) { int c = dc[d]; dc[d] = r; r += c; }
    for (int t = b; t < e; ++t) {
      int v = tmp[t];
      int d = colptr[v + 1] - colptr[v];
      out[dc[d]++] = (uint32_t)v | ((uint32_t)d << 24);
    }
  }
  nlev[i] = nl;
}

// Summary engine: each member's schedule entries with the offset of the column's first message in the
// member's schedule-ordered message array (exclusive prefix sum of the degrees). One CTA per member.
__global__ void k_xrec(const uint32_t* __restrict__ sched, int n, uint2* __restrict__ rec) {
  __shared__ uint32_t part[1024];
  __shared__ uint32_t carry;
  const uint32_t* sc = sched + (size_t)blockIdx.x * n;
  uint2* out = rec + (size_t)blockIdx.x * n;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n; base += 1024) {
    const int j = base + threadIdx.x;
    const uint32_t ent = j < n ? sc[j] : 0u;
    const uint32_t d = ent >> 24;
    part[threadIdx.x] = d;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const uint32_t add = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
      __syncthreads();
      part[threadIdx.x] += add;
      __syncthreads();
    }
    if (j < n) out[j] = make_uint2(ent, carry + part[threadIdx.x] - d);
    __syncthreads();
    if (threadIdx.x == 1023) carry += part[1023];
    __syncthreads();
  }
}

// Summary engine: for every member and every CSR entry q = (check c, column v) of H, the slot of the
// message v -> c in the member's schedule-ordered message array.
__global__ void k_xrmap(const uint2* __restrict__ rec, long long total, int n, int E, int XP,
                        const uint32_t* __restrict__ xcol, const int32_t* __restrict__ rowptr,
                        uint32_t* __restrict__ rmap) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q / n;
    const uint2 r = rec[q];
    const uint32_t v = r.x & 0xffffffu, d = r.x >> 24;
    for (uint32_t k = 0; k < d; ++k) {
      const uint32_t x = xcol[(size_t)v * XP + k];
      rmap[(size_t)i * E + rowptr[x >> 8] + (x & 0xffu)] = r.y + k;
    }
  }
}

__device__ __forceinline__ uint64_t splitmix64_next(uint64_t& st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_seeded_schedules(uint32_t* __restrict__ perm, int n, int K, uint64_t seed) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= K) return;
  uint32_t* p = perm + (size_t)i * n;
  uint64_t st = seed + (uint64_t)(i + 1) * 0xD1B54A32D192ED03ull;
  for (int j = 0; j < n; ++j) p[j] = (uint32_t)j;
  for (int k = n - 1; k >= 1; --k) {
    uint64_t r = splitmix64_next(st);
    uint64_t j = __umul64hi(r, (uint64_t)(k + 1));
    uint32_t t = p[k]; p[k] = p[j]; p[j] = t;
  }
}

inline int grid_for(long long work, int threads) {
  long long g = (work + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > 65535) g = 65535;
  return (int)g;
}

}  // namespace

cudaError_t seeded_schedules(uint32_t* d_perm, int n, int K, uint64_t seed, cudaStream_t s) {
  k_seeded_schedules<<<(K + 63) / 64, 64, 0, s>>>(d_perm, n, K, seed);
  return cudaGetLastError();
}

// Check layers of the layered schedule (the oracle's reading R10): check c, in ascending order,
// joins the smallest layer that holds no earlier check sharing a column with it. One CTA: the checks
// are placed one after another (each placement depends on all earlier ones), the threads mark the
// layers of c's earlier neighbours with the stamp c and find the smallest unmarked one.
// scratch: layer_of[m] | stamp[m + 1]
__global__ void k_layers(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                         const int32_t* __restrict__ colptr, const int32_t* __restrict__ rowidx, int m,
                         int32_t* layer_ptr, int32_t* layer_chk, int32_t* layer_vptr, int32_t* layer_var,
                         int32_t* nlayer_out, int32_t* scratch) {
  int32_t* layer_of = scratch;
  int32_t* stamp = scratch + m;   // stamp[l] == c: layer l is taken for check c
  __shared__ int s_nl, s_best;
  for (int l = threadIdx.x; l <= m; l += blockDim.x) stamp[l] = -1;
  if (threadIdx.x == 0) { s_nl = 0; s_best = 0x7fffffff; }
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    for (int e = rowptr[c] + threadIdx.x; e < rowptr[c + 1]; e += blockDim.x) {
      const int v = colidx[e];
      for (int k = colptr[v]; k < colptr[v + 1]; ++k) {
        const int c2 = rowidx[k];   // ascending in the column
        if (c2 >= c) break;
        stamp[layer_of[c2]] = c;
      }
    }
    __syncthreads();
    const int nl = s_nl;
    for (int l = threadIdx.x; l <= nl; l += blockDim.x)   // layer nl is always free
      if (stamp[l] != c) atomicMin(&s_best, l);
    __syncthreads();
    if (threadIdx.x == 0) {
      layer_of[c] = s_best;
      if (s_best == nl) s_nl = nl + 1;
      s_best = 0x7fffffff;
    }
    __syncthreads();
  }
  const int nl = s_nl;
  // group: counts, offsets, checks ascending within a layer, then each layer's columns
  if (threadIdx.x == 0) {
    for (int l = 0; l <= nl; ++l) { layer_ptr[l] = 0; layer_vptr[l] = 0; }
    for (int c = 0; c < m; ++c) {
      layer_ptr[layer_of[c] + 1] += 1;
      layer_vptr[layer_of[c] + 1] += rowptr[c + 1] - rowptr[c];
    }
    for (int l = 0; l < nl; ++l) { layer_ptr[l + 1] += layer_ptr[l]; layer_vptr[l + 1] += layer_vptr[l]; }
    for (int l = 0; l < nl; ++l) stamp[l] = 0;   // fill counters per layer
    for (int c = 0; c < m; ++c) {
      const int l = layer_of[c];
      layer_chk[layer_ptr[l] + stamp[l]++] = c;
    }
    // column offset of each check inside layer_var, kept in layer_of (no longer needed as a layer id)
    for (int l = 0; l < nl; ++l) {
      int o = layer_vptr[l];
      for (int q = layer_ptr[l]; q < layer_ptr[l + 1]; ++q) {
        const int c = layer_chk[q];
        layer_of[c] = o;
        o += rowptr[c + 1] - rowptr[c];
      }
    }
    *nlayer_out = nl;
  }
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    const int o = layer_of[c], b = rowptr[c], d = rowptr[c + 1] - b;
    for (int j = threadIdx.x; j < d; j += blockDim.x) layer_var[o + j] = colidx[b + j];
  }
}

cudaError_t build_tables(const int32_t* d_rowptr, const int32_t* d_colidx, int m, int n, int K, const uint32_t* d_perm,
                         int RP, int DP, int XP, int msg_fp16, const float* d_lam, int32_t* d_colptr, int32_t* d_rowidx,
                         uint32_t* d_csc_ent, void* d_msg_init, uint32_t* d_sched, uint32_t* d_lvl_off, int32_t* d_nlev,
                         uint32_t* d_xcol, uint2* d_xrec, uint32_t* d_xrmap, float4* d_xsum, int32_t* d_scratch,
                         cudaStream_t s) {
  // scratch layout: cnt[n] | fill[n] | packed[E] ; later reused by k_levels (K*(m+3n+1))
  int E = 0;
  cudaError_t err = cudaMemcpyAsync(&E, d_rowptr + m, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (err != cudaSuccess) return err;
  if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;
  int32_t* cnt = d_scratch;
  int32_t* fill = cnt + n;
  uint32_t* packed = reinterpret_cast<uint32_t*>(fill + n);
  if ((err = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * 2 * (size_t)n, s)) != cudaSuccess) return err;
  k_col_count<<<grid_for(E, 256), 256, 0, s>>>(d_colidx, E, cnt);
  k_scan_single<<<1, 1024, 0, s>>>(cnt, n, d_colptr);
  k_csc_fill<<<grid_for(m, 128), 128, 0, s>>>(d_rowptr, d_colidx, m, d_colptr, fill, packed);
  k_csc_finish<<<grid_for(n, 128), 128, 0, s>>>(n, DP, RP, msg_fp16 ? 8 : 4, XP, d_colptr, packed, d_rowidx,
                                                 d_csc_ent, d_xcol);
  if (msg_fp16) {
    k_xsum<__half><<<grid_for(m, 128), 128, 0, s>>>(d_rowptr, d_colidx, m, d_lam, d_xsum);
    k_msg_init<__half><<<grid_for((long long)m * RP, 256), 256, 0, s>>>(d_rowptr, d_colidx, m, RP, d_lam,
                                                                       static_cast<__half*>(d_msg_init));
  } else {
    k_xsum<float><<<grid_for(m, 128), 128, 0, s>>>(d_rowptr, d_colidx, m, d_lam, d_xsum);
    k_msg_init<float><<<grid_for((long long)m * RP, 256), 256, 0, s>>>(d_rowptr, d_colidx, m, RP, d_lam,
                                                                      static_cast<float*>(d_msg_init));
  }
  k_levels<<<(K + 31) / 32, 32, 0, s>>>(d_perm, n, m, K, d_colptr, d_rowidx, d_sched, d_lvl_off, d_nlev, d_scratch);
  if (XP > 0) {
    k_xrec<<<K, 1024, 0, s>>>(d_sched, n, d_xrec);
    k_xrmap<<<grid_for((long long)K * n, 256), 256, 0, s>>>(d_xrec, (long long)K * n, n, E, XP, d_xcol, d_rowptr,
                                                            d_xrmap);
  }
  return cudaGetLastError();
}

cudaError_t build_layers(const int32_t* d_rowptr, const int32_t* d_colidx, const int32_t* d_colptr,
                         const int32_t* d_rowidx, int m, int32_t* d_layer_ptr, int32_t* d_layer_chk,
                         int32_t* d_layer_vptr, int32_t* d_layer_var, int32_t* d_nlayer, int32_t* d_scratch,
                         cudaStream_t s) {
  k_layers<<<1, 256, 0, s>>>(d_rowptr, d_colidx, d_colptr, d_rowidx, m, d_layer_ptr, d_layer_chk, d_layer_vptr,
                             d_layer_var, d_nlayer, d_scratch);
  return cudaGetLastError();
}

}  // namespace vibe
