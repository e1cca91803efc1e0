// Block-ordered in-place merge steps (A6) for one-word strings, included by
// qx_kernels.cuh after qx_merge_inplace.cuh.
//
// When the merge wires q_0 .. q_{m-1} of a fan-out step have closed groups,
// the terms that agree everywhere except in the non-isolated letters of those
// wires form complete blocks: every combination of the wires' non-isolated
// letters is present (iso letters and I stay fixed and are part of the block's
// identity).  Put each block's members at consecutive places, ordered by the
// mixed-radix number of their letters (digit = rank of the letter among the
// wire's non-isolated letters, radix = their count, 1 for a wire where the
// block has I or an isolated letter), and the other members of a term's group
// on wire q_j sit at fixed distances: (rank(a) - digit) x stride_j.  Each wire
// then becomes a pass that reads a 2-bit-per-wire letter code and weights,
// with no hash lookups; the weights are summed with the same fixed-order group
// sum as the group pass (bit-identical results).  A block with a member
// missing is detected by its count and the caller falls back.
#pragma once

namespace qx {
namespace dev {

constexpr int kMaxBlockWires = 32;  // letter code: 2 bits per merge wire in 64 bits
// With at most 16 merge wires the code's upper half holds two masks, the wires
// where the term's block has radix 2 (bits 32..47) and radix 3 (48..63), so a
// stride is 2^a 3^b from two population counts.
constexpr int kFastStrideWires = 16;

struct BlockWires {
  int m;                      // merge wires
  int q[kMaxBlockWires];      // their qubits
  uint8_t canon[kMaxBlockWires];  // the canonical non-isolated letter (0 X, 1 Y, 2 Z)
  uint8_t radix[kMaxBlockWires];  // number of non-isolated letters
  uint8_t rank[kMaxBlockWires][3];  // rank of a non-isolated letter, 255 for isolated
};

// Letter index of bits (x, z): 0 I, 1 X, 2 Y, 3 Z  -> table letter = index - 1.
__device__ __forceinline__ int letter4(uint64_t x, uint64_t z, int q) {
  const int xb = int((x >> q) & 1), zb = int((z >> q) & 1);
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

// Per term: the block key (non-isolated letters of the merge wires replaced
// by the wire's canonical letter, generator packed in), claimed in the block
// table; the member count of the block (warp-combined), the block's expected
// size, the term's place in its block and its letter code.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_claim(TermsT<WT> t, size_t N, int n,
                                                     const BlockWires* bw_g, ulonglong2* btab,
                                                     unsigned long long bcap, unsigned* bcnt,
                                                     unsigned* bexp, unsigned* bslot,
                                                     unsigned* pib, unsigned long long* lcode,
                                                     unsigned* err) {
  __shared__ BlockWires bw;
  if (threadIdx.x == 0) bw = *bw_g;
  __syncthreads();
  for (size_t base = size_t(blockIdx.x) * blockDim.x; base < N;
       base += size_t(gridDim.x) * blockDim.x) {
    const size_t i = base + threadIdx.x;
    unsigned slot = 0xffffffffu;
    if (i < N) {
      uint64_t x = t.x[i], z = t.z[i];
      unsigned long long code = 0;
      unsigned pos = 0, stride = 1;
      for (int j = 0; j < bw.m; ++j) {
        const int q = bw.q[j];
        const int L = letter4(x, z, q);
        code |= (unsigned long long)L << (2 * j);
        if (L && bw.rank[j][L - 1] != 255) {  // non-isolated: a digit of the block
          pos += unsigned(bw.rank[j][L - 1]) * stride;
          stride *= bw.radix[j];
          if (bw.m <= kFastStrideWires)
            code |= 1ull << ((bw.radix[j] == 2 ? 32 : 48) + j);
          const int c = bw.canon[j];
          const uint64_t m = 1ull << q;
          x = c <= 1 ? (x | m) : (x & ~m);
          z = c >= 1 ? (z | m) : (z & ~m);
        }
      }
      unsigned long long lo, hi;
      pack_full_key(x, z, t.g[i], n, &lo, &hi);
      unsigned long long p = __umul64hi(slot_hash(lo, hi), bcap);
      for (unsigned long long probe = 0; probe < bcap; ++probe) {
        // a block has many members: read first (a cached read may be stale
        // only as "empty", which the compare-and-swap corrects; keys never
        // change once written) and compare-and-swap only an empty slot, so
        // that the members of a claimed block do not contend
        ulonglong2 k = btab[p];
        if (k.x == ~0ull && k.y == ~0ull) {
          unsigned long long olo, ohi;
          cas128(&btab[p].x, ~0ull, ~0ull, lo, hi, &olo, &ohi);
          k.x = olo;
          k.y = ohi;
          if (olo == ~0ull && ohi == ~0ull) {
            slot = unsigned(p);
            bexp[slot] = stride;  // the claimant records the block's size
            break;
          }
        }
        if (k.x == lo && k.y == hi) {
          slot = unsigned(p);
          break;
        }
        if (++p == bcap) p = 0;
      }
      if (slot == 0xffffffffu) {
        atomicOr(err, kErrProbe);
      } else {
        bslot[i] = slot;
        pib[i] = pos;
        lcode[i] = code;
      }
    }
    // member counts, one atomic per block and warp
    const unsigned peers = __match_any_sync(0xffffffffu, slot);
    if (slot != 0xffffffffu && int(threadIdx.x & 31) == __ffs(peers) - 1)
      atomicAdd(&bcnt[slot], unsigned(__popc(peers)));
  }
}

// size[s] = expected size of the block in slot s (0 if empty); a block whose
// count differs from its size is incomplete.
static __global__ void k_block_sizes(const ulonglong2* btab, unsigned long long bcap,
                                     const unsigned* bcnt, const unsigned* bexp,
                                     unsigned long long* size, unsigned* err) {
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < bcap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const ulonglong2 k = btab[s];
    const bool used = !(k.x == ~0ull && k.y == ~0ull);
    size[s] = used ? bexp[s] : 0;
    if (used && bcnt[s] != bexp[s]) atomicOr(err, kErrNotClosed);
  }
}

// Terms to block order: place = offset of the block + place in the block.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_scatter(TermsT<WT> t, size_t N,
                                                       const unsigned* bslot, const unsigned* pib,
                                                       const unsigned long long* boff,
                                                       const unsigned long long* lcode,
                                                       TermsT<WT> out, unsigned long long* lcode_out,
                                                       WT* w_out) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const unsigned long long d = boff[bslot[i]] + pib[i];
    out.x[d] = t.x[i];
    out.z[d] = t.z[i];
    out.g[d] = t.g[i];
    w_out[d] = t.w[i];
    lcode_out[d] = lcode[i];
  }
}

// Merge wire j in block order: the members of term i's group are at
// i + (rank(a) - rank(p)) * stride_j; the letter permutation pi is applied
// to the strings afterwards, as in the hashed in-place path.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_wire(size_t N, const BlockWires* bw_g, int j,
                                                    FanQ fq, int pi,
                                                    const unsigned long long* lcode,
                                                    const WT* w_in, WT* w_out) {
  __shared__ FanQ f;
  __shared__ BlockWires bw;
  if (threadIdx.x == 0) {
    f = fq;
    bw = *bw_g;
  }
  __syncthreads();
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const unsigned long long code = lcode[i];
    const WT w = w_in[i];
    const int L = int((code >> (2 * j)) & 3);
    if (L == 0) {
      w_out[i] = w;
      continue;
    }
    const int p = L - 1, cp = (pi >> (2 * p)) & 3;
    if (f.iso[p]) {
      w_out[i] = wmul(w, f, p, cp);
      continue;
    }
    // stride of wire j in this block: product of the radices before it
    long long stride = 1;
    if (bw.m <= kFastStrideWires) {
      const unsigned below = (1u << j) - 1;
      const int a = __popc(unsigned(code >> 32) & 0xffffu & below);
      const int b = __popc(unsigned(code >> 48) & below);
      stride = 1ll << a;
      for (int k = 0; k < b; ++k) stride *= 3;
    } else {
      for (int k = 0; k < j; ++k) {
        const int Lk = int((code >> (2 * k)) & 3);
        if (Lk && bw.rank[k][Lk - 1] != 255) stride *= bw.radix[k];
      }
    }
    const int dp = bw.rank[j][p];
    bool has[3];
    WT v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int ra = bw.rank[j][a];
      has[a] = ra != 255;
      v[a] = a == p ? w : (has[a] ? w_in[(long long)i + (ra - dp) * stride] : WT(0));
    }
    bool reached = false;
    w_out[i] = group_sum(f, cp, has, v, &reached);
  }
}

}  // namespace dev
}  // namespace qx
