// In-place merge step (A6) for one-word strings, included by qx_kernels.cuh
// after the shared helpers and the fast merge path it complements.
//
// When every group of a merge wire already holds all the letters its table
// produces (each group's output letter set equals its input letter set), the
// index-based accumulation of Sec. III / Algorithm 2 creates no string and
// removes none: it only replaces each weight by sum_p t[p][c] v_p over the
// group.  Then the terms can stay where they are.  One full-key hash index of
// the step's terms is built once, and each merge wire becomes one coalesced
// pass in which every term looks up the other members of its group and
// computes its own new weight with the same fixed-order group sum as the group
// pass of the fast path (bit-identical weights).  A term that finds its group
// incomplete sets an error bit; the caller then redoes the step with the
// general merge.  Weights are double-buffered, so the step's input is intact
// until the caller copies the final weights back.
#pragma once

namespace qx {
namespace dev {

constexpr unsigned kErrNotClosed = 8u;  // a group lacks a letter its table produces

// Full key of a one-word string (n < 64) with its generator id in the free
// high bits of both words.  The empty slot is (~0, ~0), which no key reaches
// while the generator count stays below 2^(2 (64 - n)).
__device__ __forceinline__ void pack_full_key(uint64_t x, uint64_t z, uint32_t g, int n,
                                              unsigned long long* lo, unsigned long long* hi) {
  const int fb = 64 - n;
  *lo = x | (uint64_t(g) << n);
  *hi = z | (fb < 32 ? (uint64_t(g) >> fb) << n : 0ull);
}

struct KeySlot {  // one 32-byte sector: key and term index
  unsigned long long lo, hi;
  unsigned idx;
  unsigned pad0;
  unsigned long long pad1;
};

// Index of every term: one 128-bit compare-and-swap per term.
template <typename WT>
__global__ void __launch_bounds__(256) k_keyindex_build(TermsT<WT> t, size_t N, int n,
                                                        KeySlot* tab, unsigned long long cap,
                                                        unsigned* err) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    unsigned long long lo, hi;
    pack_full_key(t.x[i], t.z[i], t.g[i], n, &lo, &hi);
    unsigned long long pos = __umul64hi(slot_hash(lo, hi), cap);
    bool done = false;
    for (unsigned long long probe = 0; probe < cap; ++probe) {
      unsigned long long olo, ohi;
      cas128(&tab[pos].lo, ~0ull, ~0ull, lo, hi, &olo, &ohi);
      if (olo == ~0ull && ohi == ~0ull) {
        tab[pos].idx = unsigned(i);
        done = true;
        break;
      }
      if (olo == lo && ohi == hi) break;  // a repeated string: not a valid state
      if (++pos == cap) pos = 0;
    }
    if (!done) atomicOr(err, kErrProbe);
  }
}

__device__ __forceinline__ long long keyindex_find(const KeySlot* tab, unsigned long long cap,
                                                   unsigned long long lo, unsigned long long hi) {
  unsigned long long pos = __umul64hi(slot_hash(lo, hi), cap);
  for (unsigned long long probe = 0; probe < cap; ++probe) {
    const ulonglong2 k = *reinterpret_cast<const ulonglong2*>(&tab[pos]);
    if (k.x == lo && k.y == hi) return tab[pos].idx;
    if (k.x == ~0ull && k.y == ~0ull) return -1;
    if (++pos == cap) pos = 0;
  }
  return -1;
}

// One merge wire, in place.  The wire's table is applied as T = T' P: the
// letter permutation P (pi, 2 bits per source letter) sends each member p of a
// group to the output column pi(p) that it will carry, and the caller applies
// P to the strings after the step (the index stays valid until then).  Here
// w_out[i] = sum_a t[a][pi(p)] v_a over the members a of term i's group, or
// t[p][pi(p)] w for an isolated row: exactly the weight the group pass gives
// column pi(p).  The group must be closed: for every column c of p's row the
// member pi^-1(c) present, and pi(p) reached by a present row; otherwise
// kErrNotClosed.
template <typename WT>
__global__ void __launch_bounds__(256) k_merge_inplace(TermsT<WT> t, size_t N, int n, FanQ fq,
                                                       int pi, const WT* w_in, WT* w_out,
                                                       const KeySlot* tab, unsigned long long cap,
                                                       unsigned* err) {
  __shared__ FanQ f;
  __shared__ unsigned s_err;
  if (threadIdx.x == 0) {
    f = fq;
    s_err = *reinterpret_cast<volatile unsigned*>(err);
  }
  __syncthreads();
  if (s_err) return;  // an earlier wire of the step failed
  const int q = f.q;
  const uint64_t qm = 1ull << q;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const uint64_t x = t.x[i], z = t.z[i];
    const WT w = w_in[i];
    const int L = int((x >> q) & 1) | (int((z >> q) & 1) << 1);  // 0 I, 1 X, 3 Y, 2 Z
    if (L == 0) {
      w_out[i] = w;
      continue;
    }
    const int p = L == 1 ? 0 : (L == 3 ? 1 : 2);
    const int cp = (pi >> (2 * p)) & 3;
    if (f.iso[p]) {  // a single child, at column cp = its only entry
      w_out[i] = wmul(w, f, p, cp);
      continue;
    }
    const uint32_t g = t.g[i];
    bool has[3] = {false, false, false};
    WT v[3] = {WT(0), WT(0), WT(0)};
    has[p] = true;
    v[p] = w;
    bool closed = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == p || f.iso[a]) continue;
      const int ca = (pi >> (2 * a)) & 3;
      const bool need_in = (f.nz >> (3 * a + cp)) & 1, need_out = (f.nz >> (3 * p + ca)) & 1;
      if (!need_in && !need_out) continue;
      const uint64_t xa = a <= 1 ? (x | qm) : (x & ~qm);
      const uint64_t za = a >= 1 ? (z | qm) : (z & ~qm);
      unsigned long long lo, hi;
      pack_full_key(xa, za, g, n, &lo, &hi);
      const long long j = keyindex_find(tab, cap, lo, hi);
      if (j >= 0) {
        has[a] = true;
        v[a] = w_in[j];
      } else if (need_out) {
        closed = false;  // p's row produces a letter the group lacks
      }
    }
    bool reached = false;
    const WT nw = group_sum(f, cp, has, v, &reached);
    if (!closed || !reached) {
      atomicOr(err, kErrNotClosed);
      return;
    }
    w_out[i] = nw;
  }
}

}  // namespace dev
}  // namespace qx
