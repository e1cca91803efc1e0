// Kernels of batched propagation: many small circuits in one term store (the
// serving loop's continuous batching).
//
// Every request of a batch is a push-through plan: its non-Clifford gates as
// Pauli rotations (one step each, in circuit order) and then all its Clifford
// gates as one pass.  The generators of request r get the global ids
// [gen_base[r], gen_base[r] + n_r), so one (generator, string) key space
// covers the whole batch: rotation step t applies, to every term, the t-th
// rotation of the term's request (k_brot_count / k_brot_emit in
// qx_pauli_rot.cuh; requests with fewer rotations pass unchanged), and the
// final pass maps every term by its request's tables.  The per-term arithmetic
// is that of the single-circuit kernels, so each result equals the one its
// circuit gives alone.
#pragma once

#include "qx_kernels.cuh"

namespace qx {
namespace dev {

// The final Clifford pass of one request: identity, gate list (ops) or chunk
// tables (tab_xz / tab_e of `chunks` chunks, with their masks).
struct BatchPass {
  unsigned long long ops_off;  // into the batch's ops array
  unsigned long long tab_off;  // into the batch's table words
  unsigned long long e_off;    // into the batch's table phases
  int nops;
  int chunks;
  int kind;  // 0 identity, 1 gate list, 2 chunk tables
  int pad;
  uint64_t live;
  PassMasks pmk;
};

// One term per global generator g: Z_j of its request (j = g - gen_base).
template <int W, typename WT>
__global__ void k_batch_init(TermsT<WT> t, const int32_t* gen_req, const uint32_t* gen_base,
                             uint32_t G, unsigned long long* n_out) {
  const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < G) {
    uint64_t x[W], z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] = 0;
      z[k] = 0;
    }
    const uint32_t j = g - gen_base[gen_req[g]];
#pragma unroll
    for (int k = 0; k < W; ++k) z[k] = (int(j >> 6) == k) ? (1ull << (j & 63)) : 0ull;
    store_term<W>(t, g, x, z, WT(1), g);
  }
  if (g == 0) *n_out = (unsigned long long)G;
}

// Each term through its request's final pass, in place.  Chunk tables are
// read from global memory (a batch holds many requests' tables; they stay in
// L1/L2 while a warp's terms belong to few requests).  The part cache of
// clifford_table_map is dropped whenever a lane moves to another request.
template <int W, int CB, typename WT>
__global__ void __launch_bounds__(256) k_batch_clifford(TermsT<WT> t, const unsigned long long* n_in,
                                                        const int32_t* gen_req,
                                                        const BatchPass* passes,
                                                        const uint32_t* ops,
                                                        const uint64_t* tab_xz,
                                                        const uint8_t* tab_e) {
  const size_t N = *n_in;
  CliffCache<W> cc;
  int cur = -1;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const int r = gen_req[t.g[i]];
    const BatchPass& bp = passes[r];
    if (bp.kind == 0) continue;
    uint64_t x[W], z[W];
    load_term<W>(t, i, x, z);
    bool neg;
    if (bp.kind == 1) {
      int ng = 0;
      apply_ops<W>(ops + bp.ops_off, bp.nops, x, z, &ng);
      neg = ng != 0;
    } else {
      if (r != cur) {
        cc.valid = 0;
        cur = r;
      }
      neg = clifford_table_map<W, CB>(x, z, tab_xz + bp.tab_off, tab_e + bp.e_off, bp.chunks,
                                      bp.live, bp.pmk, cc);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      t.x[k * t.cap + i] = x[k];
      t.z[k * t.cap + i] = z[k];
    }
    if (neg) t.w[i] = wneg(t.w[i]);
  }
}

// Where each request's terms go: out[r] is request r's own term buffer.
template <typename WT>
struct BatchOut {
  TermsT<WT> t;
};

// Scatters the batch's terms into the requests' buffers: a term of global
// generator g takes the next place of g's range (cursor[g] starts at the
// offset of g within its request) and the request-local generator id.
template <int W, typename WT>
__global__ void k_batch_split(TermsT<WT> in, const unsigned long long* n_in, const int32_t* gen_req,
                              const uint32_t* gen_base, unsigned long long* cursor,
                              const BatchOut<WT>* outs) {
  const size_t N = *n_in;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    const uint32_t g = in.g[i];
    const int r = gen_req[g];
    const unsigned long long pos = atomicAdd(&cursor[g], 1ull);
    const TermsT<WT>& o = outs[r].t;
    if (pos >= o.cap) continue;  // cannot happen: the ranges come from the counts
    uint64_t x[W], z[W];
    load_term<W>(in, i, x, z);
    store_term<W>(o, size_t(pos), x, z, in.w[i], g - gen_base[r]);
  }
}

}  // namespace dev
}  // namespace qx
