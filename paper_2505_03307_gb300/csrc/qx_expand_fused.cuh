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
// * k_xs_emit reads each parent once (tiles staged in shared memory by bulk
//   copies), recounts its children, applies the Clifford pass that precedes
//   the step (when it acts on other qubits than the step's wires it commutes
//   with the step, so mapping the parent first and substituting the wires'
//   letters afterwards gives each child's image), and writes the children at
//   its block's offset, consecutive children from consecutive threads.
// The count works per range of spans (one warp each); the emission gives each
// block 8 consecutive ranges, one contiguous run of parents.
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

// The fused pass's image of each lane's string through its chunk tables:
// the chunk-ordered product of the live chunks' images of the string's
// letters, with the sign from the phase exponents in XZ form.  Each lane
// keeps its last image (FullCache); the misses are resolved by the whole
// warp: for each distinct missing key (the letters on the qubits the pass
// touches), lane j reads the table entries of chunks j and j + 32 at once,
// and the chunks combine by shuffles: the image is the XOR of the entries,
// and the phase adds, per chunk c, its entry's exponent and twice the
// anticommutation count of its X part with the Z part of the chunks before
// it (a prefix XOR across the lanes).  That is the chunk-ordered product of
// the serial loop, with one table read's latency per round instead of one
// per chunk.  Every lane of the warp calls it; `active` lanes get their
// image (x, z replaced) and return its sign.
template <int W, int CB>
__device__ __forceinline__ bool clifford_map_warp(uint64_t* x, uint64_t* z, bool active,
                                                  const uint64_t* tab_xz, const uint8_t* tab_e,
                                                  int chunks, uint64_t live, const PassMasks& pmk,
                                                  FullCache<W>& fc, unsigned lane) {
  constexpr int E = 1 << (2 * CB);
  constexpr uint32_t M = (1u << CB) - 1;
  uint64_t tx[W], tz[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    tx[k] = x[k] & ~pmk.idle[k];
    tz[k] = z[k] & ~pmk.idle[k];
  }
  bool hit = fc.valid;
#pragma unroll
  for (int k = 0; k < W; ++k) hit = hit && fc.kx[k] == tx[k] && fc.kz[k] == tz[k];
  unsigned need = __ballot_sync(0xffffffffu, active && !hit);
  while (need) {
    const int src = __ffs(need) - 1;
    uint64_t kx[W], kz[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      kx[k] = __shfl_sync(0xffffffffu, tx[k], src);
      kz[k] = __shfl_sync(0xffffffffu, tz[k], src);
    }
    int e = 0;  // the phase exponent mod 4 (every lane adds its share; summed below)
    uint64_t ax[W], az[W];
#pragma unroll
    for (int k = 0; k < W; ++k) ax[k] = az[k] = 0;
    for (int c0 = 0; c0 < chunks; c0 += 32) {
      const int c = c0 + int(lane);
      uint64_t ex[W], ez[W];
      int ev = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) ex[k] = ez[k] = 0;
      if (c < chunks && ((live >> c) & 1)) {
        const int lo = c * CB, k = lo >> 6, off = lo & 63;
        const uint64_t xw = (W == 1 || k == 0) ? kx[0] : kx[W - 1];
        const uint64_t zw = (W == 1 || k == 0) ? kz[0] : kz[W - 1];
        uint32_t xb, zb;
        if (CB == 4 || off + CB <= 64) {
          xb = uint32_t(xw >> off) & M;
          zb = uint32_t(zw >> off) & M;
        } else {  // k == 0 < W - 1
          xb = uint32_t((xw >> off) | (W > 1 ? (kx[W - 1] << (64 - off)) : 0)) & M;
          zb = uint32_t((zw >> off) | (W > 1 ? (kz[W - 1] << (64 - off)) : 0)) & M;
        }
        const uint32_t idx = xb | (zb << CB);
        if (idx) {
          const ulonglong2* ent =
              reinterpret_cast<const ulonglong2*>(tab_xz + (size_t(c) * E + idx) * 2 * W);
          if (W == 1) {
            const ulonglong2 v = __ldg(ent);
            ex[0] = v.x;
            ez[0] = v.y;
          } else {
            const ulonglong2 v0 = __ldg(ent), v1 = __ldg(ent + 1);
            ex[0] = v0.x;
            ex[W - 1] = v0.y;
            ez[0] = v1.x;
            ez[W - 1] = v1.y;
          }
          ev = int(__ldg(tab_e + c * E + idx));
        }
      }
      // Z part of the chunks before this lane's: the earlier rounds' (az)
      // and an exclusive prefix XOR over the lanes below
      uint64_t pz[W];
#pragma unroll
      for (int k = 0; k < W; ++k) pz[k] = ez[k];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const uint64_t o = __shfl_up_sync(0xffffffffu, pz[k], d);
          if (lane >= unsigned(d)) pz[k] ^= o;
        }
      }
      int anti = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) anti += __popcll((az[k] ^ pz[k] ^ ez[k]) & ex[k]);
      e += ev + 2 * anti;
      // the round's XOR of the entries, in every lane
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          ex[k] ^= __shfl_xor_sync(0xffffffffu, ex[k], d);
          ez[k] ^= __shfl_xor_sync(0xffffffffu, ez[k], d);
        }
      }
#pragma unroll
      for (int k = 0; k < W; ++k) {
        ax[k] ^= ex[k];
        az[k] ^= ez[k];
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) e += __shfl_xor_sync(0xffffffffu, e, d);
    int y = 0, c2 = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      y += __popcll(kx[k] & kz[k]);
      c2 += __popcll(ax[k] & az[k]);
    }
    bool same = active;
#pragma unroll
    for (int k = 0; k < W; ++k) same = same && tx[k] == kx[k] && tz[k] == kz[k];
    if (same) {
#pragma unroll
      for (int k = 0; k < W; ++k) {
        fc.kx[k] = kx[k];
        fc.kz[k] = kz[k];
        fc.rx[k] = ax[k];
        fc.rz[k] = az[k];
      }
      fc.neg = ((y + e - c2) & 3) == 2;
      fc.valid = true;
    }
    need &= ~__ballot_sync(0xffffffffu, same);
  }
  if (!active) return false;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    x[k] = (x[k] & pmk.idle[k]) | fc.rx[k];
    z[k] = (z[k] & pmk.idle[k]) | fc.rz[k];
  }
  return fc.neg;
}

// ---------------------------------------------------------------------------
// The emission works on tiles of kXtTile parents.  A block takes the 8
// consecutive ranges of the count's partition that its warps would have
// taken (one contiguous run of parents, whose children are contiguous from
// the first range's offset) and walks them tile by tile:
//  * one thread stages the next tiles' term planes in shared memory with
//    bulk asynchronous copies (cp.async.bulk, completion on an mbarrier),
//    kXtStages deep, so the copies of the next tiles run while tile k is
//    worked on;
//  * parent pass, two adjacent parents per thread: the fused Clifford pass,
//    the rows of the fan-out wires, the children that survive pruning, and a
//    block scan of their counts; each kept child is entered in a child map
//    (parent index, child rank);
//  * child pass, one child per thread and round: consecutive threads write
//    consecutive children, so every store of a warp covers one contiguous
//    run of each plane.
// Compared with one warp per range writing each parent's children from
// registers (127 registers, two blocks per SM), this runs three blocks per
// SM, the writes are whole sectors, and the copies keep the loads in flight
// without registers (84M-term chain: 3.64 -> 2.59 ms with the warp-resolved
// image misses).
constexpr int kXtPer = 2;                   // parents per thread and tile
constexpr int kXtTile = kXtPer * kXsThreads;  // parents per tile
constexpr int kXtStages = 3;                // tiles staged at once

template <int W, typename WT>
__host__ __device__ constexpr size_t xt_stage_bytes() {
  return size_t(kXtTile) * (16 * W + sizeof(WT) + 4);
}

// Dynamic shared memory of the emission: the stages, the child map
// (kXtTile x maxc entries of 4 bytes) and the gate list of a CK = 1 pass.
template <int W, typename WT>
__host__ __device__ constexpr size_t xt_smem_bytes(int maxc, int nops) {
  return kXtStages * xt_stage_bytes<W, WT>() + size_t(kXtTile) * size_t(maxc) * 4 +
         size_t(nops) * 4;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

// One bounded wait for phase `parity`: the thread is suspended (it issues
// nothing) until the phase completes or about `hint_ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity, unsigned hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier, at most `limit` suspended tries of
// about a microsecond each; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity,
                                                  unsigned limit) {
  for (unsigned it = 0; it < limit; ++it)
    if (mbar_try_wait(bar, parity, 1000u)) return true;
  return false;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing on the barrier's transaction count.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// its later bulk copies into the same memory (async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One stage of kXtTile parents: x planes, z planes, weights, generator ids.
template <int W, typename WT>
struct XtStage {
  unsigned char* base;
  __device__ __forceinline__ uint64_t* x(int k) const {
    return reinterpret_cast<uint64_t*>(base) + size_t(k) * kXtTile;
  }
  __device__ __forceinline__ uint64_t* z(int k) const {
    return reinterpret_cast<uint64_t*>(base) + size_t(W + k) * kXtTile;
  }
  __device__ __forceinline__ WT* w() const {
    return reinterpret_cast<WT*>(base + size_t(2 * W) * kXtTile * 8);
  }
  __device__ __forceinline__ uint32_t* g() const {
    return reinterpret_cast<uint32_t*>(base + size_t(2 * W) * kXtTile * 8 +
                                       size_t(kXtTile) * sizeof(WT));
  }
};

// Child r of a parent (letters x, z after the fused pass; the fan-out wires
// keep their letters under it), reading only the table entries it uses: the
// same digits (first wire least significant) and the same product in wire
// order as xs_child / xs_child_r.
template <int W, typename WT, int NQ>
__device__ __forceinline__ WT xs_child_at(const XsStep& st, const XsWires<NQ ? NQ : 1>& wr,
                                          const uint64_t* x, const uint64_t* z, WT w, unsigned r,
                                          uint64_t* cx, uint64_t* cz) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    cx[k] = x[k];
    cz[k] = z[k];
  }
  WProd<WT> p(w);
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
    if (!L) continue;
    const XsRow& row = st.row[j][L - 1];
    const int nn = row.nn;
    int d = 0;
    if (nn == 2) {
      d = int(r & 1);
      r >>= 1;
    } else if (nn == 3) {
      d = int(r % 3);
      r /= 3;
    }
    p.mul_entry(row.t[d], row.th[d], row.tl[d]);
    const int col = row.col[d];
    const uint64_t m = 1ull << b;
    if (!hi) {
      cx[0] = (col <= 1) ? (cx[0] | m) : (cx[0] & ~m);
      cz[0] = (col >= 1) ? (cz[0] | m) : (cz[0] & ~m);
    } else {
      cx[W - 1] = (col <= 1) ? (cx[W - 1] | m) : (cx[W - 1] & ~m);
      cz[W - 1] = (col >= 1) ? (cz[W - 1] | m) : (cz[W - 1] & ~m);
    }
  }
  return p.get();
}

// Children of each parent at its block's offset (the offset of the block's
// first range: the exclusive scan of the range sums, or the offsets recorded
// by an earlier run of the step) plus the children of the block's earlier
// parents, in parent order; no write leaves the block's share, the offsets
// of its first range and of the next block's (the last block ends at
// *total_d).  *n_out = cap (the output's count slot) in every case; a launch
// sized for cap < *total_d (an output size guessed too small) writes nothing
// else.  Every plane of `in` starts on a 16-byte boundary and in.cap is a
// multiple of 4 (the host checks both), so a tile's copies, rounded up to 16
// bytes, stay inside the planes.  A copy that does not complete within
// `spin_limit` tries (about a microsecond each) sets kErrSpin in *serr and
// the block returns once its copies in flight are done (or given up on as
// well).
// CK selects the fused Clifford pass: 0 none, 1 gate list (in shared
// memory), 3 or 4 chunk tables (read from global memory: the image cache of
// clifford_map_warp hits for all but the first parent of a run of parents
// with the same touched letters, so the tables are rarely read).
template <int W, typename WT, int CK, int NQ>
__global__ void __launch_bounds__(kXsThreads, 3) k_xs_emit(
    TermsT<WT> in, const unsigned long long* n_in, const unsigned long long* range_offs,
    size_t per, const unsigned long long* total_d, unsigned long long cap,
    const __grid_constant__ XsStep step, XsPass ps, XsCheck chk, XsStats sts, double* pruned,
    TermsT<WT> out, unsigned long long* n_out, int maxc, unsigned spin_limit, unsigned* serr) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = cap;  // the output's term count
  const unsigned long long total = *total_d;
  if (total > cap) return;
  extern __shared__ __align__(16) unsigned char s_raw[];
  __shared__ XsStep st;
  __shared__ __align__(8) uint64_t s_full[kXtStages];
  __shared__ unsigned s_wsum[kXsThreads / 32];
  const unsigned tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto stage = [&](size_t k) {
    return XtStage<W, WT>{s_raw + (k % kXtStages) * xt_stage_bytes<W, WT>()};
  };
  uint32_t* cmap = reinterpret_cast<uint32_t*>(s_raw + kXtStages * xt_stage_bytes<W, WT>());
  const uint32_t* s_ops = cmap + size_t(kXtTile) * size_t(maxc);
  load_xs_step(&st, step);
  if constexpr (CK == 1) {
    uint32_t* o = const_cast<uint32_t*>(s_ops);
    for (int i = tid; i < ps.nops; i += blockDim.x) o[i] = ps.ops[i];
  }
  if (tid == 0) {
    for (int q = 0; q < kXtStages; ++q) mbar_init(&s_full[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const size_t N = *n_in;
  const size_t nspans = (N + kXsSpan - 1) / kXsSpan;
  const size_t nranges = size_t(gridDim.x) * (kXsThreads / 32);
  const size_t rg0 = size_t(blockIdx.x) * (kXsThreads / 32);
  const size_t s0 = min(nspans, rg0 * per), s1 = min(nspans, s0 + per * (kXsThreads / 32));
  const size_t P0 = min(N, s0 * kXsSpan), P1 = min(N, s1 * kXsSpan);
  const size_t ntiles = (P1 - P0 + kXtTile - 1) / kXtTile;
  const bool prune = st.prune != 0;
  XsWires<NQ ? NQ : 1> wr;
  if constexpr (NQ > 0) wr = xs_wires<NQ>(st);
  FullCache<W> fc;
  unsigned long long run = range_offs[rg0];
  const unsigned long long end = rg0 + (kXsThreads / 32) < nranges
                                     ? range_offs[rg0 + (kXsThreads / 32)]
                                     : total;
  const size_t lim = size_t(end < cap ? end : cap);
  // tile k of the block: parents [P0 + k T, min(P1, P0 + (k + 1) T))
  auto tile_n = [&](size_t k) { return unsigned(min(size_t(kXtTile), P1 - P0 - k * kXtTile)); };
  auto issue = [&](size_t k) {  // one thread: bulk copies of tile k into its stage
    const XtStage<W, WT> sg = stage(k);
    uint64_t* bar = &s_full[k % kXtStages];
    const size_t p0 = P0 + k * kXtTile;
    const unsigned m = tile_n(k);
    const unsigned b8 = (m * 8 + 15) & ~15u, bw = (m * unsigned(sizeof(WT)) + 15) & ~15u,
                   b4 = (m * 4 + 15) & ~15u;
    mbar_expect_tx(bar, 2 * W * b8 + bw + b4);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      bulk_g2s(sg.x(q), in.x + size_t(q) * in.cap + p0, b8, bar);
      bulk_g2s(sg.z(q), in.z + size_t(q) * in.cap + p0, b8, bar);
    }
    bulk_g2s(sg.w(), in.w + p0, bw, bar);
    bulk_g2s(sg.g(), in.g + p0, b4, bar);
  };
  // tile k waits for phase (k / kXtStages) mod 2 of its stage's barrier
  auto parity = [](size_t k) { return unsigned(k / kXtStages) & 1u; };
  if (tid == 0)
    for (size_t k = 0; k < size_t(kXtStages) && k < ntiles; ++k) issue(k);
  // this thread's running letter code and its generator (checked launches)
  uint32_t code_g = 0xffffffffu, code = 0;
  // this thread's running statistics and their generator (last expansion)
  uint32_t sgen = 0xffffffffu;
  unsigned long long sn = 0;
  double ssq = 0.0;
  auto stats_flush = [&]() {
    if (sn) {
      atomicAdd(&sts.count[sgen], sn);
      atomicAdd(&sts.sumsq[sgen], ssq);
    }
    sn = 0;
    ssq = 0.0;
  };
  for (size_t k = 0; k < ntiles; ++k) {
    const XtStage<W, WT> sg = stage(k);
    const unsigned m = tile_n(k);
    const bool ok = mbar_wait_bounded(&s_full[k % kXtStages], parity(k), spin_limit);
    if (__syncthreads_or(!ok)) {
      // a copy did not complete: flag it, and let no copy outlive the block
      if (tid == 0) {
        atomicOr(serr, kErrSpin);
        for (size_t j = k; j < k + kXtStages && j < ntiles; ++j)
          mbar_wait_bounded(&s_full[j % kXtStages], parity(j), spin_limit);
      }
      return;
    }
    // parent pass: parents kXtPer tid ... kXtPer tid + kXtPer - 1 of the tile
    unsigned kc[kXtPer];
    uint32_t keep[kXtPer];
#pragma unroll
    for (int it = 0; it < kXtPer; ++it) {
      const unsigned i = kXtPer * tid + unsigned(it);
      const bool valid = i < m;
      kc[it] = 0;
      keep[it] = 0;
      uint64_t x[W], z[W];
      WT w = WT(0);
      uint32_t g = 0;
#pragma unroll
      for (int q = 0; q < W; ++q) x[q] = z[q] = 0;
      if (valid) {
#pragma unroll
        for (int q = 0; q < W; ++q) {
          x[q] = sg.x(q)[i];
          z[q] = sg.z(q)[i];
        }
        w = sg.w()[i];
        g = sg.g()[i];
      }
      if constexpr (CK >= 3) {  // every lane takes part (misses are resolved by the warp)
        if (clifford_map_warp<W, CK>(x, z, valid, ps.tab_xz, ps.tab_e, ps.chunks, ps.live, ps.pmk,
                                     fc, lane))
          w = wneg(w);
      }
      if (!valid) continue;
      if (chk.gwire) {
        if (g != code_g) {
          if (code) atomicOr(&chk.gwire[code_g], code);
          code_g = g;
          code = 0;
        }
        code |= xs_wire_code<W, NQ>(st, wr, x, z);
      }
      if constexpr (CK == 1) {
        int neg = 0;
        apply_ops<W>(s_ops, ps.nops, x, z, &neg);
        if (neg) w = wneg(w);
      }
      if constexpr (CK != 0) {  // the mapped parent, for the child pass
#pragma unroll
        for (int q = 0; q < W; ++q) {
          sg.x(q)[i] = x[q];
          sg.z(q)[i] = z[q];
        }
        sg.w()[i] = w;
      }
      unsigned c;
      if constexpr (NQ > 0) {
        XsParentRows<NQ> pr;
        c = xs_resolve<W, NQ>(st, wr, x, z, &pr);
      } else {
        c = xs_count_children<W>(st, x, z);
      }
      if (!prune || xs_keeps_all<WT>(st, w)) {
        kc[it] = c;
        keep[it] = (1u << c) - 1u;
      } else {
        for (unsigned r = 0; r < c; ++r) {
          uint64_t cx[W], cz[W];
          const WT v = xs_child_at<W, WT, NQ>(st, wr, x, z, w, r, cx, cz);
          if (xs_pruned<WT>(st, v)) {
            atomicAdd(&pruned[g], double(v) * double(v));
          } else {
            keep[it] |= 1u << r;
            ++kc[it];
          }
        }
      }
    }
    // block scan of the kept children, in parent order
    unsigned v = 0;
#pragma unroll
    for (int it = 0; it < kXtPer; ++it) v += kc[it];
    unsigned inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= unsigned(d)) inc += o;
    }
    if (lane == 31) s_wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      unsigned t = lane < kXsThreads / 32 ? s_wsum[lane] : 0u;
#pragma unroll
      for (int d = 1; d < kXsThreads / 32; d <<= 1) {
        const unsigned o = __shfl_up_sync(0xffffffffu, t, d);
        if (lane >= unsigned(d)) t += o;
      }
      if (lane < kXsThreads / 32) s_wsum[lane] = t;
    }
    __syncthreads();
    unsigned pos = inc - v + (warp ? s_wsum[warp - 1] : 0u);
    const unsigned tile_children = s_wsum[kXsThreads / 32 - 1];
#pragma unroll
    for (int it = 0; it < kXtPer; ++it) {
      const uint32_t i = kXtPer * tid + uint32_t(it);
      for (uint32_t b = keep[it]; b; b &= b - 1) cmap[pos++] = i | (uint32_t(__ffs(b) - 1) << 16);
    }
    __syncthreads();
    // child pass: child e of the tile goes to run + e
    for (unsigned e = tid; e < tile_children; e += kXsThreads) {
      const uint32_t cm = cmap[e];
      const unsigned i = cm & 0xffffu, r = cm >> 16;
      uint64_t x[W], z[W], cx[W], cz[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        x[q] = sg.x(q)[i];
        z[q] = sg.z(q)[i];
      }
      const uint32_t g = sg.g()[i];
      const WT cv = xs_child_at<W, WT, NQ>(st, wr, x, z, sg.w()[i], r, cx, cz);
      const size_t o = size_t(run) + e;
      if (o < lim) {
#pragma unroll
        for (int q = 0; q < W; ++q) {
          out.x[size_t(q) * out.cap + o] = cx[q];
          out.z[size_t(q) * out.cap + o] = cz[q];
        }
        out.w[o] = cv;
        out.g[o] = g;
        if (sts.count) {
          if (g != sgen) {
            stats_flush();
            sgen = g;
          }
          ++sn;
          ssq += double(cv) * double(cv);
        }
      }
    }
    run += tile_children;
    __syncthreads();  // the stage and the child map are free again
    if (tid == 0 && k + kXtStages < ntiles) {
      fence_proxy_async_smem();
      issue(k + kXtStages);
    }
  }
  if (sts.count) stats_flush();
  if (chk.gwire && code) atomicOr(&chk.gwire[code_g], code);
  if (chk.err && run != end) {
    // a block that wrote fewer children than its recorded share fills the
    // rest with zero-weight identity terms of generator 0, so that the run
    // (repeated once its checks are read) sees only valid generator ids
    if (tid == 0) atomicOr(chk.err, 1u);
    for (unsigned long long i = run + tid; i < lim; i += kXsThreads) {
#pragma unroll
      for (int q = 0; q < W; ++q) {
        out.x[size_t(q) * out.cap + i] = 0ull;
        out.z[size_t(q) * out.cap + i] = 0ull;
      }
      out.w[i] = WT(0);
      out.g[i] = 0u;
    }
  }
}

}  // namespace dev
}  // namespace qx
