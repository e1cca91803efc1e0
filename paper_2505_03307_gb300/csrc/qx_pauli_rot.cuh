// Pauli rotation steps exp(-i phi P / 2) for the two-qubit rotation gates and
// for Clifford push-through; included at the end of qx_kernels.cuh.
//
// Conjugation maps a string Q that anticommutes with P to
// cos phi Q + sin phi (i Q P), and i Q P = sigma(Q) (Q xor P) with a sign
// sigma(Q) = +-1 read off the XZ form; strings that commute with P stay.  The
// strings Q and Q xor P form a group of at most two; its members are ranked
// by one bit of P's support (rank 0: the member with that bit clear) and each
// output weight is summed in rank order with the same fixed-order group sum
// as the one-qubit merge (group_sum over the 2 x 2 table [[c, s], [s, c]],
// the signs sigma carried by the weights, which is exact).  Each term looks up its
// partner through the full-key index: present, the term writes only its own
// string; absent, it also writes the partner.  Count, scan and emit give every
// output a fixed place.
#pragma once

namespace qx {
namespace dev {

struct RotQ {
  uint64_t px[2], pz[2];  // P, W <= 2 words
  int rword, rbit;  // rank bit: bit rbit of word rword, of x if rx else of z
  int rx;
  int pad;
  FanQ tab;         // t[a][b]: cos phi on the diagonal, sin phi off it (a, b = ranks)
};

template <int W>
__device__ __forceinline__ bool rot_anticommutes(const RotQ& r, const uint64_t* x,
                                                 const uint64_t* z) {
  int par = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) par += __popcll((x[k] & r.pz[k]) ^ (z[k] & r.px[k]));
  return par & 1;
}

// sigma(Q) with i Q P = sigma(Q) (Q xor P), for Q anticommuting with P.
template <int W>
__device__ __forceinline__ double rot_sign(const RotQ& r, const uint64_t* x, const uint64_t* z) {
  int aq = 0, ap = 0, ar = 0, zx = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    aq += __popcll(x[k] & z[k]);
    ap += __popcll(r.px[k] & r.pz[k]);
    ar += __popcll((x[k] ^ r.px[k]) & (z[k] ^ r.pz[k]));
    zx += __popcll(z[k] & r.px[k]);
  }
  const int e = (1 + aq + ap - ar + 2 * zx) & 3;  // 0 or 2
  return e == 0 ? 1.0 : -1.0;
}

template <int W>
__device__ __forceinline__ int rot_rank(const RotQ& r, const uint64_t* x, const uint64_t* z) {
  const uint64_t wv = r.rx ? x[r.rword] : z[r.rword];
  return int((wv >> r.rbit) & 1);
}

// Outputs of term i: own (if reached) and partner (if absent and reached).
template <int W, typename WT>
__device__ __forceinline__ void rot_outputs(const RotQ& r, const uint64_t* x, const uint64_t* z,
                                            WT w, bool present, WT wp, const uint64_t* xp,
                                            const uint64_t* zp, WT* own, bool* own_on, WT* part,
                                            bool* part_on) {
  const int rq = rot_rank<W>(r, x, z), rp = 1 - rq;
  bool has[3] = {false, false, false};
  WT v[3] = {WT(0), WT(0), WT(0)};
  // own string: column rq; the partner's contribution carries sigma(partner)
  has[rq] = true;
  v[rq] = w;
  if (present) {
    has[rp] = true;
    v[rp] = rot_sign<W>(r, xp, zp) < 0 ? wneg(wp) : wp;
  }
  bool reached = false;
  *own = group_sum(r.tab, rq, has, v, &reached);
  *own_on = reached;
  *part_on = false;
  if (!present) {  // the partner string: column rp, from this term alone
    v[rq] = rot_sign<W>(r, x, z) < 0 ? wneg(w) : w;
    has[rp] = false;
    *part = group_sum(r.tab, rp, has, v, &reached);
    *part_on = reached;
  }
}

// Term i's number of outputs (1 if it commutes with P) and its partner's
// index (-1 when absent or not needed), for rotation r.
template <int W, typename WT>
__device__ __forceinline__ void rot_count_term(const RotQ& r, const TermsT<WT>& t, size_t i,
                                               const IndexSlot* tab, unsigned long long cap,
                                               unsigned long long* cnt, long long* pidx) {
  uint64_t x[W], z[W];
  load_term<W>(t, i, x, z);
  if (!rot_anticommutes<W>(r, x, z)) {
    cnt[i] = 1;
    pidx[i] = -1;
    return;
  }
  uint64_t xp[W], zp[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    xp[k] = x[k] ^ r.px[k];
    zp[k] = z[k] ^ r.pz[k];
  }
  const uint32_t g = t.g[i];
  long long j = -1;
  {
    const uint64_t h = key_hash<W>(g, xp, zp);
    const unsigned long long tag = h | 1ull;
    unsigned long long pos = __umul64hi(h, cap);
    for (unsigned long long probe = 0; probe < cap; ++probe) {
      const unsigned long long s = tab[pos].tag;
      if (s == 0ull) break;
      if (s == tag) {
        const unsigned m = tab[pos].idx;
        bool same = t.g[m] == g;
#pragma unroll
        for (int k = 0; k < W; ++k)
          same = same && t.x[k * t.cap + m] == xp[k] && t.z[k * t.cap + m] == zp[k];
        if (same) {
          j = m;
          break;
        }
      }
      if (++pos == cap) pos = 0;
    }
  }
  WT own, part;
  bool own_on, part_on;
  rot_outputs<W, WT>(r, x, z, t.w[i], j >= 0, j >= 0 ? t.w[j] : WT(0), xp, zp, &own, &own_on,
                     &part, &part_on);
  cnt[i] = (own_on ? 1 : 0) + (part_on ? 1 : 0);
  pidx[i] = j;
}

// Term i's outputs at offs[i]; r == nullptr: the term passes unchanged.
template <int W, typename WT>
__device__ __forceinline__ void rot_emit_term(const RotQ* r, const TermsT<WT>& t, size_t i,
                                              const unsigned long long* offs,
                                              const long long* pidx, const TermsT<WT>& out) {
  uint64_t x[W], z[W];
  load_term<W>(t, i, x, z);
  const uint32_t g = t.g[i];
  const WT w = t.w[i];
  unsigned long long o = offs[i];
  if (!r || !rot_anticommutes<W>(*r, x, z)) {
    store_term<W>(out, o, x, z, w, g);
    return;
  }
  uint64_t xp[W], zp[W];
#pragma unroll
  for (int k = 0; k < W; ++k) {
    xp[k] = x[k] ^ r->px[k];
    zp[k] = z[k] ^ r->pz[k];
  }
  const long long j = pidx[i];
  WT own, part;
  bool own_on, part_on;
  rot_outputs<W, WT>(*r, x, z, w, j >= 0, j >= 0 ? t.w[j] : WT(0), xp, zp, &own, &own_on, &part,
                     &part_on);
  if (own_on) store_term<W>(out, o++, x, z, own, g);
  if (part_on) store_term<W>(out, o, xp, zp, part, g);
}

// Per term: the number of outputs (1 if it commutes with P), and its
// partner's index (-1 when absent or not needed).
template <int W, typename WT>
__global__ void __launch_bounds__(256) k_rot_count(TermsT<WT> t, size_t N, RotQ rq,
                                                   const IndexSlot* tab, unsigned long long cap,
                                                   unsigned long long* cnt, long long* pidx) {
  __shared__ RotQ r;
  if (threadIdx.x == 0) r = rq;
  __syncthreads();
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x)
    rot_count_term<W, WT>(r, t, i, tab, cap, cnt, pidx);
}

template <int W, typename WT>
__global__ void __launch_bounds__(256) k_rot_emit(TermsT<WT> t, size_t N, RotQ rq,
                                                  const unsigned long long* offs,
                                                  const long long* pidx, TermsT<WT> out) {
  __shared__ RotQ r;
  if (threadIdx.x == 0) r = rq;
  __syncthreads();
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x)
    rot_emit_term<W, WT>(&r, t, i, offs, pidx, out);
}

// Batched form (many circuits in one term store, the serving loop): term i
// of global generator g belongs to request gen_req[g]; at step `step` it
// applies that request's rotation rots[rot_off[req] + step] if the request
// has more than `step` rotations, and passes unchanged otherwise.
__device__ __forceinline__ const RotQ* batch_rot(const RotQ* rots, const int32_t* gen_req,
                                                 const int32_t* rot_off, const int32_t* nrot,
                                                 int step, uint32_t g) {
  const int q = gen_req[g];
  return step < nrot[q] ? rots + rot_off[q] + step : nullptr;
}

template <int W, typename WT>
__global__ void __launch_bounds__(256) k_brot_count(TermsT<WT> t, size_t N, const RotQ* rots,
                                                    const int32_t* gen_req,
                                                    const int32_t* rot_off, const int32_t* nrot,
                                                    int step, const IndexSlot* tab,
                                                    unsigned long long cap,
                                                    unsigned long long* cnt, long long* pidx) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const RotQ* r = batch_rot(rots, gen_req, rot_off, nrot, step, t.g[i]);
    if (!r) {
      cnt[i] = 1;
      pidx[i] = -1;
      continue;
    }
    rot_count_term<W, WT>(*r, t, i, tab, cap, cnt, pidx);
  }
}

template <int W, typename WT>
__global__ void __launch_bounds__(256) k_brot_emit(TermsT<WT> t, size_t N, const RotQ* rots,
                                                   const int32_t* gen_req,
                                                   const int32_t* rot_off, const int32_t* nrot,
                                                   int step, const unsigned long long* offs,
                                                   const long long* pidx, TermsT<WT> out) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x)
    rot_emit_term<W, WT>(batch_rot(rots, gen_req, rot_off, nrot, step, t.g[i]), t, i, offs,
                         pidx, out);
}

}  // namespace dev
}  // namespace qx
