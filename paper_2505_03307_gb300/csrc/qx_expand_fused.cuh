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
//   (the weight too when pruning, and the generator id) and writes, per range
//   of spans of kXsSpan parents (one emission warp's share), the number of
//   children, together
//   with the per-generator letter masks that decide whether a merge was
//   needed (the same masks as k_fan_mask);
// * the range sums are scanned (one per warp of the emission);
// * k_xs_emit reads each parent once, recounts its children within the span,
//   applies the Clifford pass that precedes the step (when it acts on other
//   qubits than the step's wires it commutes with the step, so mapping the
//   parent first and substituting the wires' letters afterwards gives each
//   child's image), and writes the children at the span's offset.
// Warps work on contiguous ranges of spans independently (no block barrier):
// each lane loads all kXsItems of its parents before it writes anything, so a
// warp keeps that many parents per lane in flight.
//
// A plan whose step has kept the same range sums records them (the device
// driver keeps the scan's offsets): later runs launch only k_xs_emit on the
// recorded offsets, with an XsCheck that flags any range whose children
// differ from its share and collects the letter codes of the merge test, so
// the whole step is one pass over the parents, checked at the end of the run.
//
// The FP64 unit of this GPU is the scarce one (about 1.3 TFLOP/s against
// tens for FP32), so nothing here compares or converts in FP64: pruning tests
// |w| < eps on the weight's bits as integers, a parent whose |w| is at least
// the step's keep threshold (eps over the smallest table entry, with margin)
// keeps every child without computing it, and each child's weight costs one
// product per wire.  Each (wire, letter) row of the tables is one shared
// record (children's letters and entries), read once per parent.
//
// Per parent that is 16W + 8 + 4 bytes read and the children's bytes written,
// plus the fan-out words once more.  Child order and weights (the running
// product in wire order, first wire least significant) are those of
// k_expand_emit.
#pragma once

#include "qx_kernels.cuh"

namespace qx {
namespace dev {

constexpr int kXsThreads = 256;
constexpr int kXsItems = 2;                          // parents per lane and span
constexpr int kXsSpan = 32 * kXsItems;               // parents per span (one warp)

// Row of wire j's table for one letter: its children's letters and entries.
struct XsRow {
  double t[3];
  float th[3], tl[3];  // t = th + tl (FP32 weights)
  uint8_t col[3];
  uint8_t nn;
};

// What a small step's kernels need, built on the host.
struct XsStep {
  XsRow row[kSmallMaxWires][3];      // [wire][letter - 1]
  uint8_t word[kSmallMaxWires], bit[kSmallMaxWires];
  uint64_t niso[3][kMaxWords];       // wires whose X / Y / Z rows are not isolated
  uint64_t eps_bits;                 // FP64: pruned iff bits(|w|) < eps_bits
  uint64_t keep_bits;                // FP64: every child kept iff bits(|w|) >= keep_bits
  uint32_t eps_bits32, keep_bits32;  // the same for FP32 weights
  int nq;
  int prune;
  uint32_t words;                    // words of the string that hold a fan-out wire
  uint32_t pad;
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

__device__ __forceinline__ uint64_t abs_bits(double w) {
  return uint64_t(__double_as_longlong(w)) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ uint32_t abs_bits(float w) { return __float_as_uint(w) & 0x7fffffffu; }

template <typename WT>
__device__ __forceinline__ bool xs_pruned(const XsStep& st, WT v) {
  if constexpr (sizeof(WT) == 8) return abs_bits(v) < st.eps_bits;
  else return abs_bits(v) < st.eps_bits32;
}
template <typename WT>
__device__ __forceinline__ bool xs_keeps_all(const XsStep& st, WT w) {
  if constexpr (sizeof(WT) == 8) return abs_bits(w) >= st.keep_bits;
  else return abs_bits(w) >= st.keep_bits32;
}

// Letter (1 X, 2 Y, 3 Z, 0 I) of wire j.
template <int W>
__device__ __forceinline__ int xs_letter(const XsStep& st, int j, const uint64_t* x,
                                         const uint64_t* z) {
  const bool hi = W > 1 && st.word[j];
  const int b = st.bit[j];
  const int xb = int(((hi ? x[W - 1] : x[0]) >> b) & 1), zb = int(((hi ? z[W - 1] : z[0]) >> b) & 1);
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

// Children of a parent: the product of its wires' row sizes.
template <int W>
__device__ __forceinline__ unsigned xs_count_children(const XsStep& st, const uint64_t* x,
                                                      const uint64_t* z) {
  unsigned c = 1;
  for (int j = 0; j < st.nq; ++j) {
    const int L = xs_letter<W>(st, j, x, z);
    if (L) c *= st.row[j][L - 1].nn;
  }
  return c;
}

// Child r of a parent: letters into cx, cz (a copy of the parent's with the
// wires' letters replaced) and the weight w times one entry per wire.
template <int W, typename WT>
__device__ __forceinline__ WT xs_child(const XsStep& st, const uint64_t* x, const uint64_t* z, WT w,
                                       unsigned r, uint64_t* cx, uint64_t* cz) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    cx[k] = x[k];
    cz[k] = z[k];
  }
  WProd<WT> p(w);
  for (int j = 0; j < st.nq; ++j) {
    const int L = xs_letter<W>(st, j, x, z);
    if (!L) continue;
    const XsRow& row = st.row[j][L - 1];
    int d = 0;
    if (row.nn == 2) {
      d = int(r & 1);
      r >>= 1;
    } else if (row.nn == 3) {
      d = int(r % 3);
      r /= 3;
    }
    p.mul_entry(row.t[d], row.th[d], row.tl[d]);
    const int col = row.col[d];
    const uint64_t m = 1ull << st.bit[j];
    const bool hi = W > 1 && st.word[j];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const uint64_t mk = (k == (hi ? W - 1 : 0)) ? m : 0ull;
      cx[k] = (col <= 1) ? (cx[k] | mk) : (cx[k] & ~mk);
      cz[k] = (col >= 1) ? (cz[k] | mk) : (cz[k] & ~mk);
    }
  }
  return p.get();
}

// Children of a parent that survive pruning (all of them without pruning,
// or when |w| is at least the keep threshold).
template <int W, typename WT>
__device__ __forceinline__ unsigned xs_kept(const XsStep& st, const uint64_t* x, const uint64_t* z,
                                            WT w, unsigned cnt) {
  if (!st.prune || xs_keeps_all<WT>(st, w)) return cnt;
  unsigned kept = 0;
  for (unsigned r = 0; r < cnt; ++r) {
    uint64_t cx[W], cz[W];
    kept += xs_pruned<WT>(st, xs_child<W, WT>(st, x, z, w, r, cx, cz)) ? 0u : 1u;
  }
  return kept;
}

// Steps of one or two wires (NQ = 1, 2; every rotation and T step, and
// two-wire operators) resolve each parent once: the wires' bit positions sit
// in registers for the whole kernel, and the rows that the parent's letters
// select are copied from shared memory into registers, so its children cost
// no further shared-memory reads.  NQ = 0 keeps the run-time loops above.
template <int NQ>
struct XsWires {
  int word[NQ], bit[NQ];
};

template <int NQ>
__device__ __forceinline__ XsWires<NQ> xs_wires(const XsStep& st) {
  XsWires<NQ> wr;
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    wr.word[j] = st.word[j];
    wr.bit[j] = st.bit[j];
  }
  return wr;
}

template <int NQ>
struct XsParentRows {
  double t[NQ][3];
  float th[NQ][3], tl[NQ][3];
  int col[NQ][3];
  int nn[NQ];  // 1 for a wire with letter I (the parent's letter passes)
  int on[NQ];
};

template <int W, int NQ>
__device__ __forceinline__ unsigned xs_resolve(const XsStep& st, const XsWires<NQ>& wr,
                                               const uint64_t* x, const uint64_t* z,
                                               XsParentRows<NQ>* pr) {
  unsigned c = 1;
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    const bool hi = W > 1 && wr.word[j];
    const int b = wr.bit[j];
    const int xb = int(((hi ? x[W - 1] : x[0]) >> b) & 1);
    const int zb = int(((hi ? z[W - 1] : z[0]) >> b) & 1);
    const int L = xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
    pr->on[j] = L != 0;
    if (L) {
      const XsRow& row = st.row[j][L - 1];
      pr->nn[j] = row.nn;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        pr->t[j][d] = row.t[d];
        pr->th[j][d] = row.th[d];
        pr->tl[j][d] = row.tl[d];
        pr->col[j][d] = row.col[d];
      }
      c *= unsigned(row.nn);
    } else {
      pr->nn[j] = 1;
    }
  }
  return c;
}

// Child r of a resolved parent (as xs_child).
template <int W, typename WT, int NQ>
__device__ __forceinline__ WT xs_child_r(const XsWires<NQ>& wr, const XsParentRows<NQ>& pr,
                                         const uint64_t* x, const uint64_t* z, WT w, unsigned r,
                                         uint64_t* cx, uint64_t* cz) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    cx[k] = x[k];
    cz[k] = z[k];
  }
  WProd<WT> p(w);
#pragma unroll
  for (int j = 0; j < NQ; ++j) {
    if (!pr.on[j]) continue;
    int d = 0;
    if (pr.nn[j] == 2) {
      d = int(r & 1);
      r >>= 1;
    } else if (pr.nn[j] == 3) {
      d = int(r % 3);
      r /= 3;
    }
    const double t = d == 0 ? pr.t[j][0] : d == 1 ? pr.t[j][1] : pr.t[j][2];
    const float th = d == 0 ? pr.th[j][0] : d == 1 ? pr.th[j][1] : pr.th[j][2];
    const float tl = d == 0 ? pr.tl[j][0] : d == 1 ? pr.tl[j][1] : pr.tl[j][2];
    const int col = d == 0 ? pr.col[j][0] : d == 1 ? pr.col[j][1] : pr.col[j][2];
    p.mul_entry(t, th, tl);
    const uint64_t m = 1ull << wr.bit[j];
    // the word is the same for every lane: a uniform branch, no selects
    if (W == 1 || !wr.word[j]) {
      cx[0] = (col <= 1) ? (cx[0] | m) : (cx[0] & ~m);
      cz[0] = (col >= 1) ? (cz[0] | m) : (cz[0] & ~m);
    } else {
      cx[W - 1] = (col <= 1) ? (cx[W - 1] | m) : (cx[W - 1] & ~m);
      cz[W - 1] = (col >= 1) ? (cz[W - 1] | m) : (cz[W - 1] & ~m);
    }
  }
  return p.get();
}

template <int W, typename WT, int NQ>
__device__ __forceinline__ unsigned xs_kept_r(const XsStep& st, const XsWires<NQ>& wr,
                                              const XsParentRows<NQ>& pr, const uint64_t* x,
                                              const uint64_t* z, WT w, unsigned cnt) {
  if (!st.prune || xs_keeps_all<WT>(st, w)) return cnt;
  unsigned kept = 0;
  for (unsigned r = 0; r < cnt; ++r) {
    uint64_t cx[W], cz[W];
    kept += xs_pruned<WT>(st, xs_child_r<W, WT, NQ>(wr, pr, x, z, w, r, cx, cz)) ? 0u : 1u;
  }
  return kept;
}

// Words of term i that hold fan-out wires; the others read as 0 (letter I,
// which no fan-out wire is asked about).
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

// Range r of the step's partition: spans [r per, (r + 1) per) (the last
// ranges may be short or empty).  The emission runs one warp per range, so
// consecutive spans of a warp hold neighbouring parents (usually of one
// generator), which keeps the fused pass's image cache valid from span to
// span, and the count gives one child total per range: the scan is over the
// ranges, and a warp reads its range's offset once.
__device__ __forceinline__ void range_spans(size_t r, size_t per, size_t nspans, size_t* b,
                                            size_t* e) {
  *b = min(nspans, r * per);
  *e = min(nspans, *b + per);
}

// The checks of an emission launched on a step's recorded range offsets
// instead of a fresh count (both null after a count): err is set when some
// range's children differ from its recorded share (its writes stay inside
// that share), and gwire[g] collects the letter codes of generator g's
// parents on the fan-out wires (bit 3j + a: wire j carries letter a + 1 on a
// non-isolated row), which decide, as the count's letter masks do, whether
// some wire needed a merge.
struct XsCheck {
  unsigned* err;
  uint32_t* gwire;
};

// Per-generator term counts and sums of squared weights of the children an
// emission writes (both null unless it is the program's last expansion:
// later Clifford passes change neither).
struct XsStats {
  unsigned long long* count;
  double* sumsq;
};

// The letter code of one parent (see XsCheck).
template <int W, int NQ>
__device__ __forceinline__ uint32_t xs_wire_code(const XsStep& st, const XsWires<NQ ? NQ : 1>& wr,
                                                 const uint64_t* x, const uint64_t* z) {
  uint32_t code = 0;
  const int nq = NQ > 0 ? NQ : st.nq;
#pragma unroll
  for (int j = 0; j < (NQ > 0 ? NQ : kSmallMaxWires); ++j) {
    if (j >= nq) break;
    const int wd = NQ > 0 ? wr.word[j] : st.word[j];
    const int b = NQ > 0 ? wr.bit[j] : st.bit[j];
    const bool hi = W > 1 && wd;
    const uint64_t xw = hi ? x[W - 1] : x[0], zw = hi ? z[W - 1] : z[0];
    const int xb = int((xw >> b) & 1), zb = int((zw >> b) & 1);
    const int L = xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
    if (L && ((st.niso[L - 1][hi ? W - 1 : 0] >> b) & 1)) code |= 1u << (3 * j + L - 1);
  }
  return code;
}

// Copies the step record into shared memory in 4-byte words.
__device__ __forceinline__ void load_xs_step(XsStep* dst, const XsStep& src) {
  static_assert(sizeof(XsStep) % 4 == 0, "XsStep is copied in 4-byte words");
  const uint32_t* a = reinterpret_cast<const uint32_t*>(&src);
  uint32_t* b = reinterpret_cast<uint32_t*>(dst);
  for (int k = threadIdx.x; k < int(sizeof(XsStep) / 4); k += blockDim.x) b[k] = a[k];
}

// Children per range of spans (range_sums) and the per-generator
// letter masks gmask [G][3][W] (OR over the generator's terms of the fan-out
// wires carrying X, Y or Z on a non-isolated row).
template <int W, typename WT, int NQ>
__global__ void __launch_bounds__(kXsThreads) k_xs_count(TermsT<WT> t,
                                                         const unsigned long long* n_in,
                                                         const __grid_constant__ XsStep step,
                                                         size_t nranges, size_t per,
                                                         unsigned long long* gmask,
                                                         unsigned long long* range_sums) {
  __shared__ XsStep st;
  load_xs_step(&st, step);
  __syncthreads();
  const size_t N = *n_in;
  const size_t nspans = (N + kXsSpan - 1) / kXsSpan;
  const unsigned lane = threadIdx.x & 31;
  const size_t warps = size_t(gridDim.x) * (kXsThreads / 32);
  const bool prune = st.prune != 0;
  const uint32_t words = st.words;
  XsWires<NQ ? NQ : 1> wr;
  if constexpr (NQ > 0) wr = xs_wires<NQ>(st);
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
  for (size_t rg = size_t(blockIdx.x) * (kXsThreads / 32) + (threadIdx.x >> 5); rg < nranges;
       rg += warps) {
  size_t s0, s1;
  range_spans(rg, per, nspans, &s0, &s1);
  unsigned long long rsum = 0;
  for (size_t span = s0; span < s1; ++span) {
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
        load_fan_words<W>(t, i, words, x[it], z[it]);
        g[it] = t.g[i];
        if (prune) wv[it] = t.w[i];  // pruning counts the surviving children
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
      if (valid) {
        if constexpr (NQ > 0) {
          XsParentRows<NQ> pr;
          const unsigned c = xs_resolve<W, NQ>(st, wr, x[it], z[it], &pr);
          sum += xs_kept_r<W, WT, NQ>(st, wr, pr, x[it], z[it], wv[it], c);
        } else {
          sum += xs_kept<W, WT>(st, x[it], z[it], wv[it], xs_count_children<W>(st, x[it], z[it]));
        }
      }
      uint64_t m[3][W];
#pragma unroll
      for (int k = 0; k < W; ++k) {  // zero for invalid lanes (their x, z are 0)
        m[0][k] = x[it][k] & ~z[it][k] & st.niso[0][k];
        m[1][k] = x[it][k] & z[it][k] & st.niso[1][k];
        m[2][k] = ~x[it][k] & z[it][k] & st.niso[2][k];
      }
      const unsigned peers = warp_peers(g[it]);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W; ++k) {  // OR over the lanes of the same generator
          if (!((words >> k) & 1)) continue;
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
    rsum += sum;
  }
  if (lane == 0) range_sums[rg] = rsum;
  }
  flush();
}

// Children of each parent at its range's offset (exclusive scan of the range
// sums, or the offsets recorded by an earlier run of the step) plus the
// children of the range's earlier parents, in parent order; no write leaves
// the range's share [range_offs[r], range_offs[r + 1]) (the last range ends
// at *total_d).  *n_out = cap (the output's count slot) in every case; a
// launch sized for cap < *total_d (an output size guessed too small) writes
// nothing else.
// CK selects the fused Clifford pass: 0 none, 1 gate list (in shared
// memory), 3 or 4 chunk tables (read from global memory: the image cache of
// clifford_table_map_full hits for all but the first parent of a run of
// parents with the same touched letters, so the tables are rarely read).
// Each lane loads both of its parents of a span into registers before it
// counts or writes anything.  (Staging the next two spans in shared memory
// with cp.async, or one parent at a time at three blocks per SM, measured
// 9 % and 13 % slower on the 84M-term chain.)
template <int W, typename WT, int CK, int NQ>
__global__ void __launch_bounds__(kXsThreads) k_xs_emit(
    TermsT<WT> in, const unsigned long long* n_in, const unsigned long long* range_offs,
    size_t per, const unsigned long long* total_d, unsigned long long cap,
    const __grid_constant__ XsStep step, XsPass ps, XsCheck chk, XsStats sts, double* pruned,
    TermsT<WT> out, unsigned long long* n_out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = cap;  // the output's term count
  const unsigned long long total = *total_d;
  if (total > cap) return;
  extern __shared__ __align__(16) uint64_t s_dyn[];
  __shared__ XsStep st;
  load_xs_step(&st, step);
  if constexpr (CK == 1) {
    uint32_t* s_ops = reinterpret_cast<uint32_t*>(s_dyn);
    for (int i = threadIdx.x; i < ps.nops; i += blockDim.x) s_ops[i] = ps.ops[i];
  }
  __syncthreads();
  const size_t N = *n_in;
  const size_t nspans = (N + kXsSpan - 1) / kXsSpan;
  const unsigned lane = threadIdx.x & 31;
  const size_t warps = size_t(gridDim.x) * (kXsThreads / 32);
  const bool prune = st.prune != 0;
  XsWires<NQ ? NQ : 1> wr;
  if constexpr (NQ > 0) wr = xs_wires<NQ>(st);
  FullCache<W> fc;
  uint64_t* ox[W];
  uint64_t* oz[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    ox[k] = out.x + size_t(k) * out.cap;
    oz[k] = out.z + size_t(k) * out.cap;
  }
  const size_t rg = size_t(blockIdx.x) * (kXsThreads / 32) + (threadIdx.x >> 5);
  size_t s0, s1;
  range_spans(rg, per, nspans, &s0, &s1);
  // the children of this warp's range start at its range's offset
  unsigned long long run = range_offs[rg];
  const unsigned long long end = rg + 1 < warps ? range_offs[rg + 1] : total;
  const size_t lim = size_t(end < cap ? end : cap);
  // this lane's running letter code and its generator (checked launches)
  uint32_t code_g = 0xffffffffu, code = 0;
  // this lane's running statistics and their generator (last expansion)
  uint32_t sg = 0xffffffffu;
  unsigned long long sn = 0;
  double ssq = 0.0;
  auto stats_flush = [&]() {
    if (sn) {
      atomicAdd(&sts.count[sg], sn);
      atomicAdd(&sts.sumsq[sg], ssq);
    }
    sn = 0;
    ssq = 0.0;
  };
  for (size_t span = s0; span < s1; ++span) {
    const size_t base = span * kXsSpan;
    // every parent of the lane first (independent loads), then the counts
    // and the warp's places in parent order (with pruning: of the surviving
    // children), then the children
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
#pragma unroll
    for (int it = 0; it < kXsItems; ++it) {
      const bool valid = g[it] != 0xffffffffu;
      unsigned c = 0, kc = 0;
      if (valid) {
        if constexpr (NQ > 0) {
          XsParentRows<NQ> pr;
          c = xs_resolve<W, NQ>(st, wr, x[it], z[it], &pr);
          kc = xs_kept_r<W, WT, NQ>(st, wr, pr, x[it], z[it], wv[it], c);
        } else {
          c = xs_count_children<W>(st, x[it], z[it]);
          kc = xs_kept<W, WT>(st, x[it], z[it], wv[it], c);
        }
        if (chk.gwire) {
          if (g[it] != code_g) {
            if (code) atomicOr(&chk.gwire[code_g], code);
            code_g = g[it];
            code = 0;
          }
          code |= xs_wire_code<W, NQ>(st, wr, x[it], z[it]);
        }
      }
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
        if (clifford_table_map_full<W, CK>(x[it], z[it], ps.tab_xz, ps.tab_e, ps.chunks, ps.live,
                                           ps.pmk, fc))
          w = wneg(w);
      } else if constexpr (CK == 1) {
        int neg = 0;
        apply_ops<W>(reinterpret_cast<const uint32_t*>(s_dyn), ps.nops, x[it], z[it], &neg);
        if (neg) w = wneg(w);
      }
      const bool all = !prune || xs_keeps_all<WT>(st, w);
      // the parent's rows again (shared-memory reads once per parent; kept
      // in registers for one parent at a time)
      XsParentRows<NQ ? NQ : 1> pr;
      if constexpr (NQ > 0) xs_resolve<W, NQ>(st, wr, x[it], z[it], &pr);
      // o + (children kept) <= lim when the range offsets hold
      size_t o = size_t(loc[it]);
      for (unsigned r = 0; r < cnt[it]; ++r) {
        uint64_t cx[W], cz[W];
        WT v;
        if constexpr (NQ > 0) v = xs_child_r<W, WT, NQ>(wr, pr, x[it], z[it], w, r, cx, cz);
        else v = xs_child<W, WT>(st, x[it], z[it], w, r, cx, cz);
        if (!all && xs_pruned<WT>(st, v)) {
          atomicAdd(&pruned[g[it]], double(v) * double(v));
          continue;
        }
        if (o < lim) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            ox[k][o] = cx[k];
            oz[k][o] = cz[k];
          }
          out.w[o] = v;
          out.g[o] = g[it];
          if (sts.count) {
            if (g[it] != sg) {
              stats_flush();
              sg = g[it];
            }
            ++sn;
            ssq += double(v) * double(v);
          }
        }
        ++o;
      }
    }
  }
  if (sts.count) stats_flush();
  if (chk.gwire && code) atomicOr(&chk.gwire[code_g], code);
  if (chk.err && run != end) {
    // a range that wrote fewer children than its recorded share fills the
    // rest with zero-weight identity terms of generator 0, so that the run
    // (repeated once its checks are read) sees only valid generator ids
    if (lane == 0) atomicOr(chk.err, 1u);
    for (unsigned long long i = run + lane; i < lim; i += 32) {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        ox[k][i] = 0ull;
        oz[k][i] = 0ull;
      }
      out.w[i] = WT(0);
      out.g[i] = 0u;
    }
  }
}

}  // namespace dev
}  // namespace qx
