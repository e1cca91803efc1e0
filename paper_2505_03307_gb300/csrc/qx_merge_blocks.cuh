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
// Up to this many blocks, their offsets come from the list of claimed slots
// (one small kernel); beyond it, from a sweep and scan of the whole table.
constexpr int kBlockListMax = 1024;
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
  // letter permutation pi of the wire (2 bits per source letter X, Y, Z), the
  // names the merged weights belong to; relab: bit j set when pi_j is not the
  // identity
  uint8_t pi[kMaxBlockWires];
  uint32_t relab;
  // The same facts packed for the per-term loop of k_block_scatter: inf[j] =
  // q (bits 0-5), the rank of the letter with xz code c = x | z << 1 in bits
  // 8 + 4c .. 11 + 4c (15: I or an isolated letter), the radix in bits 24-25;
  // and, per qubit, where X / Y / Z are non-isolated and the canonical
  // letter's x and z bits.
  uint32_t inf[kMaxBlockWires];
  uint64_t niso_x, niso_y, niso_z, canon_x, canon_z;
  uint64_t rad2, rad3;  // qubits of the wires with two / three non-isolated letters
  // Whole-word form of k_block_scatter's per-term work, when every wire has
  // radix 2, there are at most kFastStrideWires of them and their qubits
  // increase with j (lay_fast): the qubits where letter X / Y / Z has rank 1
  // (r1*), the merge qubits (qmask) and the bytes of the word that hold them;
  // the relabelled qubits (rq) and, per source letter X / Y / Z, where its
  // image has an x bit (tx) or a z bit (tz).
  int lay_fast;
  int nbytes;
  uint8_t bytes[8];
  uint64_t r1x, r1y, r1z, qmask, rq, tx[3], tz[3];
};

// Letter index of bits (x, z): 0 I, 1 X, 2 Y, 3 Z  -> table letter = index - 1.
__device__ __forceinline__ int letter4(uint64_t x, uint64_t z, int q) {
  const int xb = int((x >> q) & 1), zb = int((z >> q) & 1);
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

// Per term: the block key (non-isolated letters of the merge wires replaced
// by the wire's canonical letter, generator packed in), claimed in the block
// table (at most plimit probes: a table sized from a guess gives up early);
// the member count of the block (warp-combined) and the block's
// expected size.  Everything here is whole-word: the key from letter masks,
// the size 2^a 3^b from two population counts.  The term's place in its
// block and its letter code are left to k_block_scatter, which reads the
// strings anyway.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_claim(TermsT<WT> t, size_t N, int n,
                                                     const BlockWires* bw_g, ulonglong2* btab,
                                                     unsigned long long bcap,
                                                     unsigned long long plimit, unsigned* bcnt,
                                                     unsigned* bexp, unsigned* bslot,
                                                     unsigned* nblk, unsigned* blist,
                                                     unsigned* err) {
  __shared__ uint64_t s_mask[7];
  if (threadIdx.x == 0) {
    s_mask[0] = bw_g->niso_x;
    s_mask[1] = bw_g->niso_y;
    s_mask[2] = bw_g->niso_z;
    s_mask[3] = bw_g->canon_x;
    s_mask[4] = bw_g->canon_z;
    s_mask[5] = bw_g->rad2;
    s_mask[6] = bw_g->rad3;
  }
  __syncthreads();
  for (size_t base = size_t(blockIdx.x) * blockDim.x; base < N;
       base += size_t(gridDim.x) * blockDim.x) {
    const size_t i = base + threadIdx.x;
    unsigned slot = 0xffffffffu;
    unsigned long long key_lo = 0, key_hi = 0;
    unsigned blk_size = 0;
    if (i < N) {
      const uint64_t x = t.x[i], z = t.z[i];
      const uint64_t dm = (x & ~z & s_mask[0]) | (x & z & s_mask[1]) | (~x & z & s_mask[2]);
      const uint64_t kx = (x & ~dm) | (s_mask[3] & dm), kz = (z & ~dm) | (s_mask[4] & dm);
      unsigned size = 1u << __popcll(dm & s_mask[5]);
      for (int k = __popcll(dm & s_mask[6]); k > 0; --k) size *= 3u;
      unsigned long long lo, hi;
      pack_full_key(kx, kz, t.g[i], n, &lo, &hi);
      key_lo = lo;
      key_hi = hi;
      blk_size = size;
    }
    // One probe per distinct key and warp: the lanes of a warp usually hold
    // members of one block.  (Every probe of a claimed block by a lane whose
    // L1 still holds the slot as empty would be a compare-and-swap on one
    // hot address.)
    const bool valid = i < N;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    unsigned peers;
    {
      const unsigned long long l0 = __shfl_sync(0xffffffffu, key_lo, 0);
      const unsigned long long h0 = __shfl_sync(0xffffffffu, key_hi, 0);
      if (__all_sync(0xffffffffu, !valid || (key_lo == l0 && key_hi == h0)))
        peers = act;
      else
        peers = __match_any_sync(0xffffffffu, key_lo) & __match_any_sync(0xffffffffu, key_hi) &
                act;
    }
    const int lane = int(threadIdx.x & 31);
    const int leader = valid ? __ffs(peers) - 1 : lane;
    if (valid && lane == leader) {
      const unsigned long long lo = key_lo, hi = key_hi;
      const unsigned size = blk_size;
      unsigned long long p = __umul64hi(slot_hash(lo, hi), bcap);
      for (unsigned long long probe = 0; probe < plimit; ++probe) {
        // read first (a cached read may be stale only as "empty", which the
        // compare-and-swap corrects; keys never change once written) and
        // compare-and-swap only an empty slot
        ulonglong2 k = btab[p];
        if (k.x == ~0ull && k.y == ~0ull) {
          unsigned long long olo, ohi;
          cas128(&btab[p].x, ~0ull, ~0ull, lo, hi, &olo, &ohi);
          k.x = olo;
          k.y = ohi;
          if (olo == ~0ull && ohi == ~0ull) {
            slot = unsigned(p);
            bexp[slot] = size;  // the claimant records the block's size
            const unsigned li = atomicAdd(nblk, 1u);  // and lists the slot
            if (li < kBlockListMax) blist[li] = slot;
            break;
          }
        }
        if (k.x == lo && k.y == hi) {
          slot = unsigned(p);
          break;
        }
        if (++p == bcap) p = 0;
      }
      if (slot == 0xffffffffu)
        atomicOr(err, kErrProbe);
      else
        atomicAdd(&bcnt[slot], unsigned(__popc(peers)));  // the members' count
    }
    // the leader's slot to its peers
    slot = __shfl_sync(0xffffffffu, slot, leader);
    if (valid && slot != 0xffffffffu) bslot[i] = slot;
  }
}

// Offsets of at most kBlockListMax blocks, in slot order (the order the table
// sweep gives), from the list of claimed slots: each block's rank is the
// number of listed slots below its own, and the offsets are the exclusive scan
// of the sizes in rank order.  A block whose count differs from its size is
// incomplete.  dn[0] receives the element count of the table sweep that
// follows: 0 when the list sufficed, the table size otherwise; when the caller
// launched no sweep (sweep == 0), more blocks than the list holds fail the
// step instead.
static __global__ void __launch_bounds__(kBlockListMax) k_block_list(
    const unsigned* nblk, const unsigned* blist, const unsigned* bcnt, const unsigned* bexp,
    unsigned long long bcap, unsigned long long* boff, unsigned long long* dn, unsigned* err,
    int sweep) {
  __shared__ unsigned s_slot[kBlockListMax];
  __shared__ unsigned long long s_size[kBlockListMax];
  __shared__ unsigned long long s_warp[kBlockListMax / 32];
  const unsigned nb = *nblk;
  const unsigned t = threadIdx.x;
  if (nb > unsigned(kBlockListMax)) {
    if (t == 0) {
      dn[0] = bcap;
      if (!sweep) atomicOr(err, kErrNotClosed);
    }
    return;
  }
  if (t == 0) dn[0] = 0;
  const unsigned my = t < nb ? blist[t] : 0xffffffffu;
  s_slot[t] = my;
  s_size[t] = 0;
  __syncthreads();
  unsigned rank = 0;
  unsigned long long sz = 0;
  if (t < nb) {
    for (unsigned u = 0; u < nb; ++u) rank += s_slot[u] < my ? 1u : 0u;
    sz = bexp[my];
    if (bcnt[my] != sz) atomicOr(err, kErrNotClosed);
  }
  __syncthreads();
  if (t < nb) s_size[rank] = sz;
  __syncthreads();
  // exclusive scan of s_size: warps, then the warp totals
  const unsigned lane = t & 31, wid = t >> 5;
  const unsigned long long v = s_size[t];
  unsigned long long inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= unsigned(d)) inc += o;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = s_warp[lane];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= unsigned(d)) w += o;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  s_size[t] = (wid ? s_warp[wid - 1] : 0) + inc - v;
  __syncthreads();
  if (t < nb) boff[my] = s_size[rank];
}

// size[s] = expected size of the block in slot s (0 if empty) for the first
// *count slots; a block whose count differs from its size is incomplete.
static __global__ void k_block_sizes(const ulonglong2* btab, const unsigned long long* count,
                                     const unsigned* bcnt, const unsigned* bexp,
                                     unsigned long long* size, unsigned* err) {
  const unsigned long long bcap = *count;
  for (unsigned long long s = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; s < bcap;
       s += (unsigned long long)gridDim.x * blockDim.x) {
    const ulonglong2 k = btab[s];
    const bool used = !(k.x == ~0ull && k.y == ~0ull);
    size[s] = used ? bexp[s] : 0;
    if (used && bcnt[s] != bexp[s]) atomicOr(err, kErrNotClosed);
  }
}

// Bits of v at the merge qubits, gathered in wire order through the
// per-byte tables of k_block_scatter (tab[b][byte]: that byte's merge-qubit
// bits at their wire positions).
__device__ __forceinline__ uint32_t gather_wires(uint64_t v, const uint16_t (*tab)[256],
                                                 const uint8_t* bytes, int nb) {
  uint32_t r = 0;
  for (int k = 0; k < nb; ++k) r |= tab[k][(v >> (8 * bytes[k])) & 255u];
  return r;
}

// Spreads the low 16 bits of v to the even bits of a 32-bit word.
__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// Terms to block order: place = offset of the block + place in the block,
// the place being the mixed-radix number of the term's letters on the
// block's digit wires (digit = rank among the wire's non-isolated letters).
// Each term also gets its letter code (2 bits per wire, and with at most
// kFastStrideWires wires the masks of the radix-2 and radix-3 wires of its
// block in the upper half), and its string is written with the letter
// permutations pi of the merge wires applied (the wire passes read only
// letter codes and weights, so the names can change before them).  With
// lay_fast the letters of all wires are gathered at once (byte tables), the
// place is the rank bits gathered over the digit wires, and the relabel is
// whole-word; otherwise one loop step per wire.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_scatter(TermsT<WT> t, size_t N,
                                                       const BlockWires* bw_g,
                                                       const unsigned* bslot,
                                                       const unsigned long long* boff,
                                                       TermsT<WT> out, unsigned long long* lcode_out,
                                                       WT* w_out, const unsigned* err) {
  if (*err) return;  // an incomplete block: the places are not a permutation
  __shared__ uint32_t s_inf[kMaxBlockWires];
  __shared__ uint8_t s_pi[kMaxBlockWires];
  __shared__ uint32_t s_relab;
  __shared__ uint16_t s_tab[8][256];
  __shared__ uint8_t s_bytes[8];
  const int m = bw_g->m;
  const bool lay = bw_g->lay_fast != 0;
  const int nb = bw_g->nbytes;
  if (threadIdx.x < unsigned(m)) {
    s_inf[threadIdx.x] = bw_g->inf[threadIdx.x];
    s_pi[threadIdx.x] = bw_g->pi[threadIdx.x];
  }
  if (threadIdx.x == 32) s_relab = bw_g->relab;
  if (threadIdx.x < 8) s_bytes[threadIdx.x] = bw_g->bytes[threadIdx.x];
  const uint64_t qmask = bw_g->qmask;
  if (lay) {
    for (int e = threadIdx.x; e < nb * 256; e += blockDim.x) {
      const int k = e >> 8, v = e & 255, b = bw_g->bytes[k];
      uint32_t r = 0;
      for (int bit = 0; bit < 8; ++bit) {
        const int q = 8 * b + bit;
        if (((v >> bit) & 1) && ((qmask >> q) & 1))
          r |= 1u << __popcll(qmask & ((1ull << q) - 1));
      }
      s_tab[k][v] = uint16_t(r);
    }
  }
  __syncthreads();
  const bool fast = m <= kFastStrideWires;
  const uint32_t relab = s_relab;
  const uint64_t nx = bw_g->niso_x, ny = bw_g->niso_y, nz = bw_g->niso_z;
  const uint64_t r1x = bw_g->r1x, r1y = bw_g->r1y, r1z = bw_g->r1z, rq = bw_g->rq;
  const uint64_t tx0 = bw_g->tx[0], tx1 = bw_g->tx[1], tx2 = bw_g->tx[2];
  const uint64_t tz0 = bw_g->tz[0], tz1 = bw_g->tz[1], tz2 = bw_g->tz[2];
  const uint32_t all = m >= 32 ? 0xffffffffu : ((1u << m) - 1);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const unsigned slot = bslot[i];
    const uint64_t x = t.x[i], z = t.z[i];
    uint64_t xo = x, zo = z;
    unsigned long long code = 0;
    unsigned pos = 0;
    if (lay) {
      const uint64_t ix = x & ~z, iy = x & z, iz = ~x & z;
      const uint32_t D = gather_wires((ix & nx) | (iy & ny) | (iz & nz), s_tab, s_bytes, nb);
      const uint32_t R = gather_wires((ix & r1x) | (iy & r1y) | (iz & r1z), s_tab, s_bytes, nb);
      const uint32_t cx = gather_wires(x ^ z, s_tab, s_bytes, nb);
      const uint32_t cz = gather_wires(z, s_tab, s_bytes, nb);
      code = spread16(cx) | (spread16(cz) << 1) | ((unsigned long long)D << 32);
      if (D == all) {
        pos = R;
      } else {
        int k = 0;
        for (uint32_t d = D; d; d &= d - 1, ++k) pos |= ((R >> (__ffs(d) - 1)) & 1u) << k;
      }
      if (rq) {
        xo = (x & ~rq) | (ix & tx0) | (iy & tx1) | (iz & tx2);
        zo = (z & ~rq) | (ix & tz0) | (iy & tz1) | (iz & tz2);
      }
    } else {
      unsigned stride = 1, r2 = 0, r3 = 0;
      for (int j = 0; j < m; ++j) {
        const uint32_t inf = s_inf[j];
        const int q = int(inf & 63u);
        const uint32_t c = (uint32_t(x >> q) & 1u) | ((uint32_t(z >> q) & 1u) << 1);
        const uint32_t L = c ^ (c >> 1);  // 0 I, 1 X, 2 Y, 3 Z
        code |= (unsigned long long)L << (2 * j);
        const uint32_t rk = (inf >> (8 + 4 * c)) & 15u;
        if (rk != 15u) {  // a digit of the block
          const uint32_t rdx = (inf >> 24) & 3u;
          pos += rk * stride;
          stride *= rdx;
          if (rdx == 2) r2 |= 1u << j; else r3 |= 1u << j;
        }
        if (L && ((relab >> j) & 1u)) {
          const uint32_t cl = (uint32_t(s_pi[j]) >> (2 * (L - 1))) & 3u;  // 0 X, 1 Y, 2 Z
          const uint64_t mq = 1ull << q;
          xo = cl <= 1 ? (xo | mq) : (xo & ~mq);
          zo = cl >= 1 ? (zo | mq) : (zo & ~mq);
        }
      }
      if (fast) code |= ((unsigned long long)r2 << 32) | ((unsigned long long)r3 << 48);
    }
    const unsigned long long d = boff[slot] + pos;
    out.x[d] = xo;
    out.z[d] = zo;
    out.g[d] = t.g[i];
    w_out[d] = t.w[i];
    lcode_out[d] = code;
  }
}

// Merge wire j in block order: the members of term i's group are at
// i + (rank(a) - rank(p)) * stride_j; the letter permutation pi is applied
// to the strings afterwards, as in the hashed in-place path.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_wire(size_t N, const BlockWires* bw_g, int j,
                                                    FanQ fq, int pi,
                                                    const unsigned long long* lcode,
                                                    const WT* w_in, WT* w_out,
                                                    const unsigned* err) {
  if (*err) return;  // no block order: the partner distances do not hold
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

// A merge wire with exactly two non-isolated letters (radix 2: the common
// case of a rotation mixing two letters), with at most kFastStrideWires
// wires.  The member of rank d (0: the first of the two letters in X, Y, Z
// order) gets c[d][0] v_0 + c[d][1] v_1, v_r the weight of the member of rank
// r, c[d][r] = t[letter r][pi(letter d)]: the same fused multiply-adds in the
// same order as group_sum (a zero coefficient is skipped, as there), so the
// result is bit-identical to k_block_wire; the coefficients come in as kernel
// parameters instead of shared-memory tables, which leaves the FP64 unit as
// the only busy one.  I passes through; the isolated letter is scaled by
// t[p][pi(p)].
struct Wire2 {
  double c[2][2];
  double iso_t;
  float ch[2][2], cl[2][2];  // FP32 path: c = ch + cl
  float iso_h, iso_l;
  uint32_t rk;  // 2 bits per letter code L = 1 X, 2 Y, 3 Z: rank 0 / 1, 3 isolated
  uint32_t nz;  // bit 2d + r: c[d][r] != 0
};

// One term of k_block_wire2: its letter code's digit decides whether it
// passes through (I), scales (isolated letter) or needs its partner, at
// *partner (-1: none).
__device__ __forceinline__ int wire2_kind(const Wire2& wv, unsigned long long code, int j,
                                          unsigned below, size_t i, long long* partner) {
  const int L = int((code >> (2 * j)) & 3);
  *partner = -1;
  if (L == 0) return 3;  // I
  const int r = int((wv.rk >> (2 * L)) & 3);
  if (r == 3) return 2;  // isolated
  const int a = __popc(unsigned(code >> 32) & 0xffffu & below);
  const int b = __popc(unsigned(code >> 48) & below);
  long long stride = 1ll << a;
  for (int k = 0; k < b; ++k) stride *= 3;
  *partner = (long long)i + (r ? -stride : stride);
  return r;
}

__device__ __forceinline__ double wire2_out(const Wire2& wv, int kind, double w, double vp) {
  if (kind == 3) return w;
  if (kind == 2) return w * wv.iso_t;
  const int r = kind;
  const double v0 = r ? vp : w, v1 = r ? w : vp;
  const double c0 = r ? wv.c[1][0] : wv.c[0][0], c1 = r ? wv.c[1][1] : wv.c[0][1];
  const uint32_t nz = wv.nz >> (2 * r);
  double acc = 0.0;
  if (nz & 1u) acc = fma(c0, v0, acc);
  if (nz & 2u) acc = fma(c1, v1, acc);
  return acc;
}

// FP32 weights: the same compensated sum (and scaling) as group_sum / wmul.
__device__ __forceinline__ float wire2_out(const Wire2& wv, int kind, float w, float vp) {
  if (kind == 3) return w;
  if (kind == 2) return wmul_split(w, wv.iso_h, wv.iso_l);
  const int r = kind;
  const float v0 = r ? vp : w, v1 = r ? w : vp;
  const uint32_t nz = wv.nz >> (2 * r);
  bool any = false;
  float sum = 0.f, comp = 0.f;
  if (nz & 1u) dot2_add(v0, wv.ch[r][0], wv.cl[r][0], &any, &sum, &comp);
  if (nz & 2u) dot2_add(v1, wv.ch[r][1], wv.cl[r][1], &any, &sum, &comp);
  return sum + comp;
}

// Two terms per thread and iteration (i and i + the grid's thread count), so
// that each thread has two independent chains of loads in flight in front of
// the FP64 unit.
template <typename WT>
__global__ void __launch_bounds__(256) k_block_wire2(size_t N, int j, Wire2 wv,
                                                     const unsigned long long* lcode,
                                                     const WT* w_in, WT* w_out,
                                                     const unsigned* err) {
  if (*err) return;  // no block order: the partner distances do not hold
  const unsigned below = (1u << j) - 1;
  const size_t S = size_t(gridDim.x) * blockDim.x;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += 2 * S) {
    const size_t i2 = i + S;
    const bool two = i2 < N;
    const unsigned long long code = lcode[i], code2 = two ? lcode[i2] : 0ull;
    const WT w = w_in[i], w2 = two ? w_in[i2] : WT(0);
    long long p, p2 = -1;
    const int k = wire2_kind(wv, code, j, below, i, &p);
    const int k2 = two ? wire2_kind(wv, code2, j, below, i2, &p2) : 3;
    const WT vp = p >= 0 ? w_in[p] : WT(0), vp2 = p2 >= 0 ? w_in[p2] : WT(0);
    w_out[i] = wire2_out(wv, k, w, vp);
    if (two) w_out[i2] = wire2_out(wv, k2, w2, vp2);
  }
}

}  // namespace dev
}  // namespace qx
