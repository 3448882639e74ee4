// K3 -- localised statistics decoding (Sec. III.C) of the shots the BP ensemble left unresolved.
//
// One CTA takes one shot at a time from the queue the BP kernel filled. Clusters start as single
// flipped checks. In every round each invalid cluster adds its best free adjacent column in the
// reliability order (the averaged soft value ascending, ties to the lower index) together with all
// checks of that column; clusters that come to share a check merge (union-find, root = smallest
// check). Validity -- the cluster's syndrome lies in the GF(2) span of its columns -- is kept by
// incremental elimination: every cluster holds an echelon basis of its column vectors, bit-packed
// over the checks with one 32-bit word per lane, stored in rows keyed by the pivot check. A new
// column is reduced against the basis and kept if it is independent; on a merge the basis of larger
// rank survives and the other cluster's columns are reduced into it. When no cluster is invalid,
// each cluster is solved by OSD-0: its columns are eliminated in reliability order (pivots = the
// first independent ones) with a record of which columns make up each basis row, the syndrome is
// reduced, and the recorded columns form the correction (free columns zero).
//
// Warps work on different clusters in parallel; the merge bookkeeping of each round is serial (one
// thread) because it is short (one pick per invalid cluster). Every loop is bounded: at most n + 1
// rounds (each adds a column), list walks bounded by list lengths.
#include <algorithm>
#include <type_traits>

#include "vibe_internal.cuh"

namespace vibe {
namespace {

constexpr int kFreeRows = 10;   // largest LSD order: records kept for the first 10 free columns

struct LsdShared {
  uint32_t* key;      // n  reliability key (sortable bits of the soft value)
  int32_t* col_root;  // n  a check of the column's cluster, -1 if free
  int32_t* col_next;  // n  cluster column lists
  int32_t* pend_next; // n  columns waiting to be reduced into their cluster's basis
  int32_t* ck_par;    // m  union-find parent, -1 = check in no cluster
  unsigned long long* best;  // m
  uint8_t* valid;     // m
  uint8_t* dirty;     // m
  int32_t* rank;      // m
  int32_t* b_head; int32_t* b_tail; int32_t* piv_next;  // m each: basis rows in insertion order
  int32_t* c_head; int32_t* c_tail; int32_t* c_cnt;     // m each: column lists
  int32_t* p_head; int32_t* p_tail;                     // m each: pending lists
  int32_t* dlist;     // m  roots to process this round
  uint32_t* sbits;    // W
  uint32_t* ebits;    // nw
  int32_t* flags;     // 8
};

__device__ __forceinline__ uint32_t reliability_key(float x) {
  uint32_t b = __float_as_uint(__fadd_rn(x, 0.0f));  // -0 -> +0 so that equal values tie
  return b ^ ((b & 0x80000000u) ? 0xffffffffu : 0x80000000u);
}

// Parent chains are acyclic by construction; the step bound (the number of checks) only guarantees
// termination should that ever be violated.
__device__ __forceinline__ int find_root(const int32_t* par, int c, int m) {
  for (int g = 0; par[c] != c && g < m; ++g) c = par[c];
  return c;
}

__device__ __forceinline__ int find_root_halving(int32_t* par, int c, int m) {
  for (int g = 0; par[c] != c && g < m; ++g) {
    par[c] = par[par[c]];
    c = par[c];
  }
  return c;
}

template <int WP>
__device__ __forceinline__ void load_column(const Tables& t, int j, uint32_t (&x)[WP], int lane) {
#pragma unroll
  for (int q = 0; q < WP; ++q) x[q] = 0u;
  for (int e = __ldg(t.colptr + j); e < __ldg(t.colptr + j + 1); ++e) {
    const int c = __ldg(t.rowidx + e);
    const int w = c >> 5;
    if ((w & 31) == lane) {
#pragma unroll
      for (int q = 0; q < WP; ++q)
        if ((w >> 5) == q) x[q] |= 1u << (c & 31);
    }
  }
}

template <int WP>
__device__ __forceinline__ bool any_bits(const uint32_t (&x)[WP]) {
  uint32_t o = 0;
#pragma unroll
  for (int q = 0; q < WP; ++q) o |= x[q];
  return __any_sync(kFull, o != 0u);
}

template <int WP>
__device__ __forceinline__ uint32_t get_bit(const uint32_t (&x)[WP], int p, int lane) {
  const int w = p >> 5;
  uint32_t b = 0;
#pragma unroll
  for (int q = 0; q < WP; ++q)
    if ((w >> 5) == q) b = (x[q] >> (p & 31)) & 1u;
  return __shfl_sync(kFull, b, w & 31);
}

// lowest set bit index over the lane-distributed vector (word w = lane + 32 q), or INT_MAX
template <int WP>
__device__ __forceinline__ int lowest_bit(const uint32_t (&x)[WP], int lane) {
  int best = 0x7fffffff;
#pragma unroll
  for (int q = WP - 1; q >= 0; --q)
    if (x[q]) best = (lane + 32 * q) * 32 + (__ffs(x[q]) - 1);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) best = min(best, __shfl_xor_sync(kFull, best, off));
  return best;
}

// x <- x reduced by the basis rows listed from `head` (insertion order); comb tracks the same XORs
// over the rows' column combinations when TRACK.
// ops counts the 32-bit words XOR-ed (the same on every lane of the warp).
template <int WP, bool TRACK>
__device__ __forceinline__ void reduce(uint32_t (&x)[WP], uint32_t (&comb)[WP], int head, const LsdShared& S,
                                       const uint32_t* basis, const uint32_t* combrow, int W, int CW, int lane,
                                       unsigned long long& ops) {
  const int maxrows = 32 * W;   // a basis never has more rows than checks
  int g = 0;
  for (int p = head; p >= 0 && g < maxrows; p = S.piv_next[p], ++g) {
    if (get_bit<WP>(x, p, lane)) {
      ops += (unsigned long long)(W + (TRACK ? CW : 0));
#pragma unroll
      for (int q = 0; q < WP; ++q) {
        const int w = lane + 32 * q;
        if (w < W) x[q] ^= basis[(size_t)p * W + w];
        if (TRACK && w < CW) comb[q] ^= combrow[(size_t)p * CW + w];
      }
    }
  }
}

template <int WP, bool TRACK>
__device__ __forceinline__ void append_row(const uint32_t (&x)[WP], const uint32_t (&comb)[WP], int p, int root,
                                           const LsdShared& S, uint32_t* basis, uint32_t* combrow, int W, int CW,
                                           int32_t* head, int32_t* tail, int lane) {
#pragma unroll
  for (int q = 0; q < WP; ++q) {
    const int w = lane + 32 * q;
    if (w < W) basis[(size_t)p * W + w] = x[q];
    if (TRACK && w < CW) combrow[(size_t)p * CW + w] = comb[q];
  }
  if (lane == 0) {
    S.piv_next[p] = -1;
    if (*tail >= 0) S.piv_next[*tail] = p; else *head = p;
    *tail = p;
    if (!TRACK) S.rank[root]++;
  }
  __syncwarp();
}

// serial (thread 0): merge the clusters rooted at a and b, return the surviving root
__device__ int merge_clusters(const LsdShared& S, int a, int b, int n) {
  const int s = min(a, b), o = max(a, b);
  const int X = S.rank[o] > S.rank[s] ? o : s;   // basis that survives
  const int Y = X == o ? s : o;                   // its columns are reduced into X's basis again
  int ph = S.p_head[X], pt = S.p_tail[X];
  int g = 0;
  for (int j = S.c_head[Y]; j >= 0 && g < n; j = S.col_next[j], ++g) {
    S.pend_next[j] = -1;
    if (pt >= 0) S.pend_next[pt] = j; else ph = j;
    pt = j;
  }
  const int bh = S.b_head[X], bt = S.b_tail[X], rk = S.rank[X];
  // column lists: s ++ o
  if (S.c_head[o] >= 0) {
    if (S.c_tail[s] >= 0) S.col_next[S.c_tail[s]] = S.c_head[o]; else S.c_head[s] = S.c_head[o];
    S.c_tail[s] = S.c_tail[o];
  }
  S.c_cnt[s] += S.c_cnt[o];
  S.b_head[s] = bh; S.b_tail[s] = bt; S.rank[s] = rk;
  S.p_head[s] = ph; S.p_tail[s] = pt;
  S.ck_par[o] = s;
  S.valid[s] = 0;
  S.dirty[s] = 1;
  S.dirty[o] = 0;
  return s;
}

template <int WP, int NT>
__global__ void __launch_bounds__(NT) k_lsd(const LsdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = NT / 32;
  // arrays sized by the launch's bounds; each shot uses the first m / n entries of its problem
  // combination records cover the first 32 * CW columns of a cluster in reliability order
  const int mB = a.bnd.m, nB = a.bnd.n, WB = a.bnd.W, nwB = a.bnd.nw, CWB = min((a.bnd.n + 31) / 32, 32 * WP);
  const bool cols_smem = lsd_cols_in_smem(a.bnd);
  unsigned long long gf2_ops = 0;   // words this warp XOR-ed in eliminations (VIBE_CNT_LSD_WORDOPS)
  uint32_t* basis = a.scratch + (long long)blockIdx.x * a.scratch_pitch;   // m * W
  LsdShared S;
  Tables* sdem;
  {
    unsigned char* p = smem;
    auto take = [&](size_t bytes) { unsigned char* r = p; p += (bytes + 15) & ~(size_t)15; return r; };
    S.best = reinterpret_cast<unsigned long long*>(take(8 * (size_t)mB));
    if (cols_smem) {
      S.key = reinterpret_cast<uint32_t*>(take(4 * (size_t)nB));
      S.col_root = reinterpret_cast<int32_t*>(take(4 * (size_t)nB));
      S.col_next = reinterpret_cast<int32_t*>(take(4 * (size_t)nB));
      S.pend_next = reinterpret_cast<int32_t*>(take(4 * (size_t)nB));
    }
    S.ck_par = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.rank = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.b_head = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.b_tail = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.piv_next = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.c_head = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.c_tail = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.c_cnt = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.p_head = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.p_tail = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.dlist = reinterpret_cast<int32_t*>(take(4 * (size_t)mB));
    S.sbits = reinterpret_cast<uint32_t*>(take(4 * (size_t)WB));
    S.ebits = reinterpret_cast<uint32_t*>(take(4 * (size_t)nwB));
    S.flags = reinterpret_cast<int32_t*>(take(4 * 8));
    S.valid = take((size_t)mB);
    S.dirty = take((size_t)mB);
    sdem = reinterpret_cast<Tables*>(take((size_t)a.ndem * sizeof(Tables)));
  }
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(a.dems);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sdem);
    const int words = a.ndem * (int)(sizeof(Tables) / 4);
    for (int q = tid; q < words; q += NT) dst[q] = __ldg(src + q);
  }
  uint32_t* combrow = basis + (size_t)mB * WB;                              // m * CW
  const size_t sort_off = ((size_t)mB * WB + (size_t)mB * CWB + 1) & ~(size_t)1;   // 8-byte aligned
  unsigned long long* sortA = reinterpret_cast<unsigned long long*>(basis + sort_off);  // n
  unsigned long long* sortB = sortA + nB;                                    // n
  uint32_t* freecomb = reinterpret_cast<uint32_t*>(sortB + nB);             // per warp (kFreeRows+1) * CW
  if (!cols_smem) {                                                          // 4 * n, after the free rows
    uint32_t* cols = freecomb + (size_t)nwarps * (kFreeRows + 1) * CWB;
    S.key = cols;
    S.col_root = reinterpret_cast<int32_t*>(cols + nB);
    S.col_next = reinterpret_cast<int32_t*>(cols + 2 * (size_t)nB);
    S.pend_next = reinterpret_cast<int32_t*>(cols + 3 * (size_t)nB);
  }
  const unsigned int total = *a.lsd_count;

  for (;;) {
    __syncthreads();
    if (tid == 0) S.flags[0] = (int)atomicAdd(a.lsd_next, 1u);
    __syncthreads();
    const unsigned int q = (unsigned int)S.flags[0];
    if (q >= total) break;
    const uint32_t shot = a.lsd_shots[q];
    const int di = a.dem_of_shot ? __ldg(a.dem_of_shot + shot) : 0;
    if ((unsigned)di >= (unsigned)a.ndem) continue;   // the BP kernel queues valid problems only
    const Tables& t = sdem[di];
    const int n = t.n, m = t.m, W = t.W, nw = t.nw, CW = min((t.n + 31) / 32, 32 * WP);
    const float* vsoft = a.lsd_soft + (size_t)q * nB;
    const uint32_t* syn = a.syn + (size_t)shot * a.syn_stride;

    for (int j = tid; j < n; j += NT) {
      S.key[j] = reliability_key(vsoft[j]);
      S.col_root[j] = -1;
      S.col_next[j] = -1;
      S.pend_next[j] = -1;
    }
    for (int w = tid; w < W; w += NT) {
      const int rem = m - 32 * w;
      S.sbits[w] = __ldg(syn + w) & (rem >= 32 ? 0xffffffffu : ((1u << rem) - 1u));
    }
    for (int w = tid; w < nw; w += NT) S.ebits[w] = 0u;
    for (int c = tid; c < m; c += NT) {
      const bool flipped = (__ldg(syn + (c >> 5)) >> (c & 31)) & 1u;
      S.ck_par[c] = flipped ? c : -1;
      S.valid[c] = 0; S.dirty[c] = 0; S.rank[c] = 0;
      S.b_head[c] = -1; S.b_tail[c] = -1; S.piv_next[c] = -1;
      S.c_head[c] = -1; S.c_tail[c] = -1; S.c_cnt[c] = 0;
      S.p_head[c] = -1; S.p_tail[c] = -1;
    }
    if (tid == 0) { S.flags[1] = 0; S.flags[2] = 0; S.flags[5] = 0; }
    __syncthreads();

    for (int round = 0; round <= n + 1; ++round) {
      // A: reset the pick of every invalid cluster
      for (int c = tid; c < m; c += NT)
        if (S.ck_par[c] == c && !S.valid[c]) S.best[c] = ~0ull;
      __syncthreads();
      // B: best free column adjacent to each invalid cluster
      for (int c = tid; c < m; c += NT) {
        if (S.ck_par[c] < 0) continue;
        const int r = find_root(S.ck_par, c, m);
        if (S.valid[r]) continue;
        for (int e = __ldg(t.rowptr + c); e < __ldg(t.rowptr + c + 1); ++e) {
          const int j = __ldg(t.colidx + e);
          if (S.col_root[j] < 0) atomicMin(&S.best[r], ((unsigned long long)S.key[j] << 32) | (unsigned)j);
        }
      }
      __syncthreads();
      // C: apply the picks (serial)
      if (tid == 0) {
        int npick = 0, status = 0;
        // picks are stored in dlist temporarily as root ids; the columns are read from best[]
        for (int c = 0; c < m; ++c) {
          if (S.ck_par[c] == c && !S.valid[c]) {
            if (S.best[c] == ~0ull) { status = 2; break; }
            S.dlist[npick++] = c;
          }
        }
        if (status == 0 && npick == 0) status = 1;
        if (status == 0) {
          for (int k = 0; k < npick; ++k) {
            const int r0 = S.dlist[k];
            const int j = (int)(S.best[r0] & 0xffffffffull);
            int r = find_root_halving(S.ck_par, r0, m);
            if (S.col_root[j] < 0) {
              S.col_root[j] = r;
              S.col_next[j] = -1;
              if (S.c_tail[r] >= 0) S.col_next[S.c_tail[r]] = j; else S.c_head[r] = j;
              S.c_tail[r] = j;
              S.c_cnt[r]++;
              S.pend_next[j] = -1;
              if (S.p_tail[r] >= 0) S.pend_next[S.p_tail[r]] = j; else S.p_head[r] = j;
              S.p_tail[r] = j;
              S.dirty[r] = 1;
            }
            for (int e = __ldg(t.colptr + j); e < __ldg(t.colptr + j + 1); ++e) {
              const int c = __ldg(t.rowidx + e);
              if (S.ck_par[c] < 0) {
                S.ck_par[c] = r;
              } else {
                const int rc = find_root_halving(S.ck_par, c, m);
                if (rc != r) r = merge_clusters(S, r, rc, n);
              }
            }
          }
          int nd = 0;
          for (int c = 0; c < m; ++c)
            if (S.ck_par[c] == c && S.dirty[c]) { S.dlist[nd++] = c; S.dirty[c] = 0; }
          S.flags[1] = nd;
        }
        S.flags[2] = status;
      }
      __syncthreads();
      if (S.flags[2] != 0) break;
      // D: reduce the new columns into each changed cluster's basis, then test its syndrome
      const int nd = S.flags[1];
      for (int k = warp; k < nd; k += nwarps) {
        const int r = S.dlist[k];
        uint32_t x[WP], dummy[WP];
#pragma unroll
        for (int qq = 0; qq < WP; ++qq) dummy[qq] = 0u;
        int guard = 0;
        for (int j = S.p_head[r]; j >= 0 && guard < n; j = S.pend_next[j], ++guard) {
          load_column<WP>(t, j, x, lane);
          reduce<WP, false>(x, dummy, S.b_head[r], S, basis, combrow, W, CW, lane, gf2_ops);
          if (any_bits<WP>(x)) {
            const int p = lowest_bit<WP>(x, lane);
            append_row<WP, false>(x, dummy, p, r, S, basis, combrow, W, CW, &S.b_head[r], &S.b_tail[r], lane);
          }
        }
        __syncwarp();
        if (lane == 0) { S.p_head[r] = -1; S.p_tail[r] = -1; }
        // restricted syndrome
#pragma unroll
        for (int qq = 0; qq < WP; ++qq) {
          const int w = lane + 32 * qq;
          uint32_t y = w < W ? S.sbits[w] : 0u, keep = 0u;
          while (y) {
            const int b = __ffs(y) - 1;
            y &= y - 1;
            const int c = 32 * w + b;
            if (c < m && S.ck_par[c] >= 0 && find_root(S.ck_par, c, m) == r) keep |= 1u << b;
          }
          x[qq] = keep;
        }
        reduce<WP, false>(x, dummy, S.b_head[r], S, basis, combrow, W, CW, lane, gf2_ops);
        const bool ok = !any_bits<WP>(x);
        if (lane == 0) S.valid[r] = ok ? 1 : 0;
        __syncwarp();
      }
      __syncthreads();
    }

    const int status = S.flags[2];   // 1 = all clusters valid, 2 = unsolvable
    // final clusters; rank[] is reused for each cluster's slice offset in the sort buffers
    if (tid == 0) {
      int nr = 0, big = 0, off = 0;
      for (int c = 0; c < m; ++c)
        if (S.ck_par[c] == c) {
          S.dlist[nr++] = c;
          big = max(big, S.c_cnt[c]);
          S.rank[c] = off;
          off += S.c_cnt[c];
          S.b_head[c] = -1;
          S.b_tail[c] = -1;
        }
      S.flags[3] = nr;
      S.flags[4] = big;
    }
    __syncthreads();
    const int nr = S.flags[3];
    if (status == 1) {
      for (int k = warp; k < nr; k += nwarps) {
        const int r = S.dlist[k];
        const int kap = S.c_cnt[r];
        if (kap > 32 * CW) {   // more columns than the combination records hold
          if (lane == 0) S.flags[5] = 1;
          continue;
        }
        unsigned long long* A = sortA + S.rank[r];
        unsigned long long* Bv = sortB + S.rank[r];
        if (lane == 0) {
          int tp = 0;
          for (int j = S.c_head[r]; j >= 0 && tp < kap; j = S.col_next[j])
            A[tp++] = ((unsigned long long)S.key[j] << 32) | (unsigned)j;
        }
        __syncwarp();
        for (int tp = lane; tp < kap; tp += 32) {   // keys are distinct: rank by counting
          const unsigned long long key = A[tp];
          int pos = 0;
          for (int u = 0; u < kap; ++u) pos += A[u] < key;
          Bv[pos] = key;
        }
        __syncwarp();
        // OSD-0: eliminate the columns in reliability order, recording each row's columns. A column
        // that reduces to zero is free; its record (itself plus the pivots that sum to it) is kept for
        // the first `order` free columns.
        uint32_t x[WP], comb[WP];
        uint32_t* fc = freecomb + (size_t)warp * (kFreeRows + 1) * CWB;
        int nfree = 0;
        for (int tp = 0; tp < kap; ++tp) {
          const int j = (int)(Bv[tp] & 0xffffffffull);
          load_column<WP>(t, j, x, lane);
#pragma unroll
          for (int qq = 0; qq < WP; ++qq)
            comb[qq] = ((tp >> 5) == lane + 32 * qq) ? (1u << (tp & 31)) : 0u;
          reduce<WP, true>(x, comb, S.b_head[r], S, basis, combrow, W, CW, lane, gf2_ops);
          if (any_bits<WP>(x)) {
            const int p = lowest_bit<WP>(x, lane);
            append_row<WP, true>(x, comb, p, r, S, basis, combrow, W, CW, &S.b_head[r], &S.b_tail[r], lane);
          } else {
            if (nfree < t.lsd_order) {
#pragma unroll
              for (int qq = 0; qq < WP; ++qq) {
                const int w = lane + 32 * qq;
                if (w < CW) fc[(size_t)nfree * CW + w] = comb[qq];
              }
            }
            ++nfree;
          }
        }
        // reduce the cluster's syndrome; the recorded columns are the solution
#pragma unroll
        for (int qq = 0; qq < WP; ++qq) {
          const int w = lane + 32 * qq;
          uint32_t y = w < W ? S.sbits[w] : 0u, keep = 0u;
          while (y) {
            const int b = __ffs(y) - 1;
            y &= y - 1;
            const int c = 32 * w + b;
            if (c < m && S.ck_par[c] >= 0 && find_root(S.ck_par, c, m) == r) keep |= 1u << b;
          }
          x[qq] = keep;
          comb[qq] = 0u;
        }
        reduce<WP, true>(x, comb, S.b_head[r], S, basis, combrow, W, CW, lane, gf2_ops);
        const int q = min(t.lsd_order, nfree);
        if (q == 0) {
#pragma unroll
          for (int qq = 0; qq < WP; ++qq) {
            uint32_t cbits = comb[qq];
            while (cbits) {
              const int b = __ffs(cbits) - 1;
              cbits &= cbits - 1;
              const int tp = (lane + 32 * qq) * 32 + b;
              if (tp < kap) {
                const int j = (int)(Bv[tp] & 0xffffffffull);
                atomicOr(&S.ebits[j >> 5], 1u << (j & 31));
              }
            }
          }
        } else {
          // order-q search: setting a (bit b = free column b) gives x0 XOR the records of the set free
          // columns. Row kFreeRows holds x0. A[u] = (column << 32) | mask for the u-th column of the
          // cluster in ascending column index, mask bit 0 = x0, bit b+1 = record of free column b.
#pragma unroll
          for (int qq = 0; qq < WP; ++qq) {
            const int w = lane + 32 * qq;
            if (w < CW) fc[(size_t)kFreeRows * CW + w] = comb[qq];
          }
          __syncwarp();
          for (int tp = lane; tp < kap; tp += 32) {
            const uint32_t j = (uint32_t)(Bv[tp] & 0xffffffffull);
            int u = 0;
            for (int v2 = 0; v2 < kap; ++v2) u += (uint32_t)(Bv[v2] & 0xffffffffull) < j;
            uint32_t mask = (fc[(size_t)kFreeRows * CW + (tp >> 5)] >> (tp & 31)) & 1u;
            for (int b = 0; b < q; ++b) mask |= ((fc[(size_t)b * CW + (tp >> 5)] >> (tp & 31)) & 1u) << (b + 1);
            A[u] = ((unsigned long long)j << 32) | mask;
          }
          __syncwarp();
          float bestW = __int_as_float(0x7f800000);
          int bestA = 0x7fffffff;
          for (int set = lane; set < (1 << q); set += 32) {
            const uint32_t sel = ((uint32_t)set << 1) | 1u;
            float Wt = 0.0f;
            for (int u = 0; u < kap; ++u) {
              const unsigned long long au = A[u];
              if (__popc((uint32_t)au & sel) & 1) Wt = __fadd_rn(Wt, __ldg(t.lam + (au >> 32)));
            }
            if (Wt < bestW) { bestW = Wt; bestA = set; }   // ascending settings per lane: ties keep the lower
          }
#pragma unroll
          for (int off = 16; off >= 1; off >>= 1) {
            const float ow = __shfl_xor_sync(kFull, bestW, off);
            const int oa = __shfl_xor_sync(kFull, bestA, off);
            if (ow < bestW || (ow == bestW && oa < bestA)) { bestW = ow; bestA = oa; }
          }
          const uint32_t sel = ((uint32_t)bestA << 1) | 1u;
          for (int u = lane; u < kap; u += 32) {
            const unsigned long long au = A[u];
            if (__popc((uint32_t)au & sel) & 1) {
              const uint32_t j = (uint32_t)(au >> 32);
              atomicOr(&S.ebits[j >> 5], 1u << (j & 31));
            }
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // outputs
    const bool limit = status == 1 && S.flags[5] != 0;
    const bool solved = status == 1 && !limit;
    for (int w = tid; w < nw; w += NT) a.corr[(size_t)shot * a.corr_stride + w] = solved ? S.ebits[w] : 0u;
    if (a.want_soft)
      for (int j = tid; j < n; j += NT) a.soft[(size_t)shot * a.soft_stride + j] = vsoft[j];
    if (warp == 0) {
      uint32_t fail = 0;
      for (int rb = 0; rb < t.kw; ++rb) {
        const int r = 32 * rb + lane;
        uint32_t par = 0;
        if (solved && r < t.k)
          for (int e = __ldg(t.lrowptr + r); e < __ldg(t.lrowptr + r + 1); ++e) {
            const int j = __ldg(t.lcolidx + e);
            par ^= (S.ebits[j >> 5] >> (j & 31)) & 1u;
          }
        const uint32_t word = __ballot_sync(kFull, par != 0);
        if (a.logical && lane == 0) a.logical[(size_t)shot * a.log_stride + rb] = word;
        if (a.obs) fail |= word ^ __ldg(a.obs + (size_t)shot * a.log_stride + rb);
      }
      if (lane == 0) {
        if (a.stats) {
          vibe_shot_stats st;
          st.status = solved ? VIBE_STATUS_OK : limit ? VIBE_STATUS_CLUSTER_LIMIT : VIBE_STATUS_UNSOLVABLE;
          st.lsd_invoked = 1; st.n_converged = 0; st.chosen_member = 255;
          st.iters = (uint16_t)t.T;
          st.largest_cluster = (uint16_t)min(S.flags[4], 65535);
          st.n_clusters = (uint32_t)nr;
          a.stats[shot] = st;
        }
        if (a.counters) {
          atomicAdd(a.counters + VIBE_CNT_LSD, 1ull);
          if (!solved && !limit) atomicAdd(a.counters + VIBE_CNT_UNSOLVABLE, 1ull);
          if (fail) atomicAdd(a.counters + VIBE_CNT_FAILURES, 1ull);
        }
      }
    }
  }
  if (lane == 0 && a.counters && gf2_ops) atomicAdd(a.counters + VIBE_CNT_LSD_WORDOPS, gf2_ops);
}

inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Words per lane of the kernel's bit vectors: enough for the check vectors, and for combination
// records of all n columns up to n = 4096 (larger problems record clusters of up to 32 * 32 * WP).
int lsd_wp(const Bounds& b) {
  const int need = max(max((b.W + 31) / 32, min(((b.n + 31) / 32 + 31) / 32, 4)), 1);
  int wp = 1;
  while (wp < need) wp <<= 1;
  return wp;
}

template <int P, int NT>
cudaError_t lsd_launch_one(const LsdArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaError_t err = ensure_dyn_smem<k_lsd<P, NT>>(smem);
  if (err != cudaSuccess) return err;
  k_lsd<P, NT><<<grid, NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int P, int NT>
cudaError_t lsd_occupancy_one(size_t smem, int* out) {
  cudaError_t err = ensure_dyn_smem<k_lsd<P, NT>>(smem);
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, k_lsd<P, NT>, NT, smem);
}

template <typename Fn>
cudaError_t by_wp_nt(int wp, int nt, Fn&& f) {
  auto with_nt = [&](auto p) -> cudaError_t {
    switch (nt) {
      case 64: return f(p, std::integral_constant<int, 64>{});
      case 128: return f(p, std::integral_constant<int, 128>{});
      case 256: return f(p, std::integral_constant<int, 256>{});
      default: return cudaErrorInvalidValue;
    }
  };
  switch (wp) {
    case 1: return with_nt(std::integral_constant<int, 1>{});
    case 2: return with_nt(std::integral_constant<int, 2>{});
    case 4: return with_nt(std::integral_constant<int, 4>{});
    case 8: return with_nt(std::integral_constant<int, 8>{});
    case 16: return with_nt(std::integral_constant<int, 16>{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t lsd_smem_bytes(const Bounds& b, int ndem) {
  const size_t m = b.m, n = b.n;
  return a16(8 * m) + (lsd_cols_in_smem(b) ? 4 * a16(4 * n) : 0) + 11 * a16(4 * m) + a16(4 * (size_t)b.W) +
         a16(4 * (size_t)b.nw) + a16(32) + 2 * a16(m) + a16((size_t)ndem * sizeof(Tables));
}

long long lsd_scratch_words(const Bounds& b, int threads) {
  const long long CW = std::min<long long>((b.n + 31) / 32, 32LL * lsd_wp(b));
  const long long head = ((long long)b.m * b.W + (long long)b.m * CW + 1) & ~1LL;
  const long long free_rows = (long long)(threads / 32) * (kFreeRows + 1) * CW;
  const long long cols = lsd_cols_in_smem(b) ? 0 : 4LL * b.n;
  return (head + 4LL * b.n + free_rows + cols + 2 + 1) & ~1LL;   // even: every CTA's slice stays 8-byte aligned
}

cudaError_t launch_lsd(const LsdArgs& a, int grid, int threads, cudaStream_t s) {
  const size_t smem = lsd_smem_bytes(a.bnd, a.ndem);
  return by_wp_nt(lsd_wp(a.bnd), threads, [&](auto p, auto nt) {
    return lsd_launch_one<decltype(p)::value, decltype(nt)::value>(a, grid, smem, s);
  });
}

cudaError_t lsd_occupancy(const Bounds& b, int ndem, int threads, int* blocks_per_sm) {
  const size_t smem = lsd_smem_bytes(b, ndem);
  return by_wp_nt(lsd_wp(b), threads, [&](auto p, auto nt) {
    return lsd_occupancy_one<decltype(p)::value, decltype(nt)::value>(smem, blocks_per_sm);
  });
}

}  // namespace vibe
