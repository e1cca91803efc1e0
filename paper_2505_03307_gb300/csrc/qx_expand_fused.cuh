// Fused expansion of small fan-out steps (A4 + A5 in one pass over the terms).
//
// A fan-out step whose wires need no merge (no generator carries two
// non-isolated letters on a wire) is the Cartesian expansion of Eq. 3: every
// parent writes the product of its wires' table rows.  When the step has few
// wires and each parent at most kSmallMaxChildren children (rotations and T
// gates on one or two wires: every step of a long circuit of sparse
// rotations), the expansion streams the terms twice:
//
// * k_xs_count reads only the words of the strings that hold a fan-out wire
//   (and the generator id) and writes, per span of kXsSpan parents (one
//   warp's share), the number of children, together with the per-generator
//   letter masks that decide whether a merge was needed (the same masks as
//   k_fan_mask);
// * the span sums are scanned (64 bytes per thousand parents);
// * k_xs_emit reads each parent once, recounts its children within the span,
//   applies the Clifford pass that precedes the step (when it acts on other
//   qubits than the step's wires it commutes with the step, so mapping the
//   parent first and substituting the wires' letters afterwards gives each
//   child's image), and writes the children at the span's offset.
// Warps work on their spans independently (no block barrier): each lane
// loads all kXsItems of its parents before it writes anything, so a warp keeps
// that many parents per lane in flight.
//
// Per parent that is 16W + 8 + 4 bytes read and the children's bytes written,
// plus the fan-out words once more, against the separate Clifford pass (read
// and write every term), letter masks, count, three-kernel scan of per-term
// offsets, tile table and emission of the general path.  Child order and
// weights (the running product in wire order, first wire least significant)
// are those of k_expand_emit.
#pragma once

#include "qx_kernels.cuh"

namespace qx {
namespace dev {

constexpr int kXsThreads = 256;
constexpr int kXsItems = 4;                          // parents per lane and span
constexpr int kXsSpan = 32 * kXsItems;               // parents per span (one warp)

// Letter masks of the wires' non-isolated rows (as k_fan_mask) and the words
// of a string that hold a fan-out wire (bit k: word k).
struct XsMasks {
  uint64_t niso[3][kMaxWords];
  uint32_t words;
};

// A Clifford pass applied to each parent before its children are written:
// kind 0 none, 1 gate list (ops), 3 or 4 chunk tables of that many qubits.
struct XsPass {
  const uint32_t* ops;
  int nops;
  const uint64_t* tab_xz;
  const uint8_t* tab_e;
  int chunks;
  uint64_t live;
  PassMasks pmk;
};

// Words of term i that hold fan-out wires; the others read as 0 (letter I,
// which no table row of a fan-out wire is asked about).
template <int W, typename WT>
__device__ __forceinline__ void load_fan_words(const TermsT<WT>& t, size_t i, uint32_t words,
                                               uint64_t* x, uint64_t* z) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const bool use = (words >> k) & 1;
    x[k] = use ? t.x[k * t.cap + i] : 0ull;
    z[k] = use ? t.z[k * t.cap + i] : 0ull;
  }
}

// Child r of a parent (letters x, z after the fused pass, weight w): its
// letters in cx, cz and its weight, the running product in wire order with
// the first wire as the least significant mixed-radix digit (as k_expand_emit).
template <int W, typename WT>
__device__ __forceinline__ WT xs_child(const FanQ* fq, int nq, const uint64_t* x, const uint64_t* z,
                                       WT w, unsigned r, uint64_t* cx, uint64_t* cz) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    cx[k] = x[k];
    cz[k] = z[k];
  }
  WProd<WT> p(w);
  for (int j = 0; j < nq; ++j) {
    const FanQ& f = fq[j];
    const int L = letter_at<W>(x, z, f.q);
    if (!L) continue;
    const int a = L - 1;
    const int nn = f.nnz[a];
    int d = 0;
    if (nn == 2) {
      d = int(r & 1);
      r >>= 1;
    } else if (nn == 3) {
      d = int(r % 3);
      r /= 3;
    }
    const int col = f.col[a][d];
    p.mul(f, a, col);
    set_letter<W>(cx, cz, f.q, col);
  }
  return p.get();
}

// Children of a parent that survive pruning (|w| < eps is dropped, in FP64
// as k_compact_pruned decides); all of them when eps = 0.
template <int W, typename WT>
__device__ __forceinline__ unsigned xs_kept(const FanQ* fq, int nq, const uint64_t* x,
                                            const uint64_t* z, WT w, unsigned cnt, double eps) {
  if (!(eps > 0.0)) return cnt;
  unsigned kept = 0;
  for (unsigned r = 0; r < cnt; ++r) {
    uint64_t cx[W], cz[W];
    const WT v = xs_child<W, WT>(fq, nq, x, z, w, r, cx, cz);
    kept += fabs(double(v)) < eps ? 0u : 1u;
  }
  return kept;
}

// Children per span of kXsSpan parents (span_sums) and the per-generator
// letter masks gmask [G][3][W] (OR over the generator's terms of the fan-out
// wires carrying X, Y or Z on a non-isolated row).
template <int W, typename WT = double>
__global__ void __launch_bounds__(kXsThreads) k_xs_count(TermsT<WT> t,
                                                         const unsigned long long* n_in,
                                                         const FanQ* fq_g, int nq, XsMasks mk,
                                                         double eps,
                                                         unsigned long long* gmask,
                                                         unsigned long long* span_sums) {
  __shared__ FanQ s_fq[kSmallMaxWires];
  for (int j = threadIdx.x; j < nq; j += blockDim.x) s_fq[j] = fq_g[j];
  __syncthreads();
  const size_t N = *n_in;
  const size_t nspans = (N + kXsSpan - 1) / kXsSpan;
  const unsigned lane = threadIdx.x & 31;
  const size_t warps = size_t(gridDim.x) * (kXsThreads / 32);
  // running OR of a warp whose lanes all held generator cg
  uint32_t cg = 0xffffffffu;
  uint64_t acc[3][W];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int k = 0; k < W; ++k) acc[a][k] = 0;
  auto flush = [&]() {
    if (cg != 0xffffffffu && lane == 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W; ++k)
          if (acc[a][k]) atomicOr(&gmask[(size_t(cg) * 3 + a) * W + k], acc[a][k]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < W; ++k) acc[a][k] = 0;
  };
  for (size_t span = size_t(blockIdx.x) * (kXsThreads / 32) + (threadIdx.x >> 5); span < nspans;
       span += warps) {
    const size_t base = span * kXsSpan;
    // all loads of the span first, then the counts and masks
    uint64_t x[kXsItems][W], z[kXsItems][W];
    uint32_t g[kXsItems];
    WT wv[kXsItems];
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      const size_t i = base + size_t(it) * 32 + lane;
      wv[it] = WT(0);
      if (i < N) {
        load_fan_words<W>(t, i, mk.words, x[it], z[it]);
        g[it] = t.g[i];
        if (eps > 0.0) wv[it] = t.w[i];  // pruning counts the surviving children
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) x[it][k] = z[it][k] = 0ull;
        g[it] = 0xffffffffu;
      }
    }
    unsigned sum = 0;
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      const bool valid = g[it] != 0xffffffffu;
      if (valid)
        sum += xs_kept<W, WT>(s_fq, nq, x[it], z[it], wv[it],
                              unsigned(child_count<W>(x[it], z[it], s_fq, nq)), eps);
      uint64_t m[3][W];
#pragma unroll
      for (int k = 0; k < W; ++k) {  // zero for invalid lanes (their x, z are 0)
        m[0][k] = x[it][k] & ~z[it][k] & mk.niso[0][k];
        m[1][k] = x[it][k] & z[it][k] & mk.niso[1][k];
        m[2][k] = ~x[it][k] & z[it][k] & mk.niso[2][k];
      }
      const unsigned peers = warp_peers(g[it]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W; ++k) {  // OR over the lanes of the same generator
          if (!((mk.words >> k) & 1)) continue;
          const unsigned lo = __reduce_or_sync(peers, unsigned(m[a][k]));
          const unsigned hi = __reduce_or_sync(peers, unsigned(m[a][k] >> 32));
          m[a][k] = (uint64_t(hi) << 32) | lo;
        }
      if (peers == 0xffffffffu) {  // one generator in the whole warp
        if (g[it] != cg) {
          flush();
          cg = g[it];
        }
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int k = 0; k < W; ++k) acc[a][k] |= m[a][k];
        continue;
      }
      if (valid && lane == unsigned(__ffs(peers) - 1)) {
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int k = 0; k < W; ++k)
            if (m[a][k]) atomicOr(&gmask[(size_t(g[it]) * 3 + a) * W + k], m[a][k]);
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) span_sums[span] = sum;
  }
  flush();
}

// Children of each parent at span_offs[span] (exclusive scan of the span
// sums) plus the parent's offset within the span, in parent order.  A launch
// sized for cap < *total_d (an output size guessed too small) does nothing.
// CK selects the fused Clifford pass: 0 none, 1 gate list, 3 or 4 chunk
// tables (dynamic shared memory holds the pass).
template <int W, typename WT, int CK>
__global__ void __launch_bounds__(kXsThreads) k_xs_emit(
    TermsT<WT> in, const unsigned long long* n_in, const unsigned long long* span_offs,
    const unsigned long long* total_d, unsigned long long cap, const FanQ* fq_g, int nq,
    XsMasks mk, XsPass ps, double eps, double* pruned, TermsT<WT> out) {
  if (*total_d > cap) return;
  extern __shared__ __align__(16) uint64_t s_dyn[];
  __shared__ FanQ s_fq[kSmallMaxWires];
  for (int j = threadIdx.x; j < nq; j += blockDim.x) s_fq[j] = fq_g[j];
  const uint8_t* s_e = nullptr;
  if constexpr (CK >= 3) {
    constexpr int E = 1 << (2 * CK);
    uint8_t* e8 = reinterpret_cast<uint8_t*>(s_dyn + size_t(ps.chunks) * E * 2 * W);
    load_clifford_table<CK, W>(s_dyn, e8, ps.tab_xz, ps.tab_e, ps.chunks);
    s_e = e8;
  } else if constexpr (CK == 1) {
    uint32_t* s_ops = reinterpret_cast<uint32_t*>(s_dyn);
    for (int i = threadIdx.x; i < ps.nops; i += blockDim.x) s_ops[i] = ps.ops[i];
  }
  __syncthreads();
  (void)mk;
  const size_t N = *n_in;
  const size_t nspans = (N + kXsSpan - 1) / kXsSpan;
  const unsigned lane = threadIdx.x & 31;
  const size_t warps = size_t(gridDim.x) * (kXsThreads / 32);
  CliffCache<W> cc;
  for (size_t span = size_t(blockIdx.x) * (kXsThreads / 32) + (threadIdx.x >> 5); span < nspans;
       span += warps) {
    const size_t base = span * kXsSpan;
    // every parent of the lane first (independent loads), then the counts
    // and the warp's offsets in parent order (with pruning: of the
    // surviving children)
    uint64_t x[kXsItems][W], z[kXsItems][W];
    WT wv[kXsItems];
    uint32_t g[kXsItems];
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      const size_t i = base + size_t(it) * 32 + lane;
      if (i < N) {
        load_term<W>(in, i, x[it], z[it]);
        wv[it] = in.w[i];
        g[it] = in.g[i];
      } else {
#pragma unroll
        for (int k = 0; k < W; ++k) x[it][k] = z[it][k] = 0ull;
        wv[it] = WT(0);
        g[it] = 0xffffffffu;
      }
    }
    unsigned cnt[kXsItems];
    unsigned long long loc[kXsItems];
    unsigned long long run = span_offs[span];
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      const bool valid = g[it] != 0xffffffffu;
      const unsigned c = valid ? unsigned(child_count<W>(x[it], z[it], s_fq, nq)) : 0u;
      const unsigned kc = valid ? xs_kept<W, WT>(s_fq, nq, x[it], z[it], wv[it], c, eps) : 0u;
      unsigned inc = kc;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= unsigned(d)) inc += o;
      }
      cnt[it] = c;
      loc[it] = run + inc - kc;
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      if (!cnt[it]) continue;
      WT w = wv[it];
      if constexpr (CK >= 3) {
        if (clifford_table_map<W, CK>(x[it], z[it], s_dyn, s_e, ps.chunks, ps.live, ps.pmk, cc))
          w = wneg(w);
      } else if constexpr (CK == 1) {
        int neg = 0;
        apply_ops<W>(reinterpret_cast<const uint32_t*>(s_dyn), ps.nops, x[it], z[it], &neg);
        if (neg) w = wneg(w);
      }
      // o + (children kept) <= *total_d <= cap (the counts the span sums came from)
      unsigned long long o = loc[it];
      for (unsigned r = 0; r < cnt[it]; ++r) {
        uint64_t cx[W], cz[W];
        const WT v = xs_child<W, WT>(s_fq, nq, x[it], z[it], w, r, cx, cz);
        if (eps > 0.0 && fabs(double(v)) < eps) {
          atomicAdd(&pruned[g[it]], double(v) * double(v));
          continue;
        }
        if (o < cap) store_term<W>(out, size_t(o), cx, cz, v, g[it]);
        ++o;
      }
    }
  }
}

}  // namespace dev
}  // namespace qx
