// Table-form Clifford pass (A4) over large term sets, in tiles staged by bulk
// copies.  Included by qx_device.cu after qx_expand_fused.cuh (its mbarrier
// and bulk-copy helpers).
//
// The pass maps every term in place: (x, z) to the image of its string under
// the pass's chunk tables (clifford_table_map, with the part cache), and the
// weight's sign when the image carries one.  k_clifford_table does this one
// term per lane straight from global memory; here each block walks a
// contiguous run of tiles of kCtTile terms:
//  * one thread stages the next tiles' x, z and weight planes in shared
//    memory with bulk copies (two stages), so no warp waits on a global load;
//  * every thread maps two adjacent terms of the tile in shared memory
//    (neighbours share all but the newest fan-out letters, which keeps the
//    part cache warm);
//  * the same thread writes the tile back with bulk copies from shared
//    memory (its 16-byte multiple; the last tile's ragged end, at most three
//    terms, with plain stores), so the threads issue no global stores.
// The tables sit in shared memory as for k_clifford_table.
#pragma once

namespace qx {
namespace dev {

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from shared to global memory, in the thread's current bulk group.
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until this thread's bulk copies to global memory have read their
// shared-memory sources (the source may be overwritten).
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Waits until this thread's bulk copies to global memory are complete.
__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

constexpr int kCtPer = 2;                     // terms per thread and tile
constexpr int kCtTile = kCtPer * kXsThreads;  // terms per tile

template <int W, typename WT>
__host__ __device__ constexpr size_t ct_stage_bytes() {
  return size_t(kCtTile) * (16 * W + sizeof(WT));
}

// Dynamic shared memory: the tables (rounded up to 16 bytes), two stages.
template <int W, typename WT>
__host__ __device__ constexpr size_t ct_smem_bytes(size_t table_bytes) {
  return ((table_bytes + 15) & ~size_t(15)) + 2 * ct_stage_bytes<W, WT>();
}

template <int W, typename WT>
struct CtStage {
  unsigned char* base;
  __device__ __forceinline__ uint64_t* x(int k) const {
    return reinterpret_cast<uint64_t*>(base) + size_t(k) * kCtTile;
  }
  __device__ __forceinline__ uint64_t* z(int k) const {
    return reinterpret_cast<uint64_t*>(base) + size_t(W + k) * kCtTile;
  }
  __device__ __forceinline__ WT* w() const {
    return reinterpret_cast<WT*>(base + size_t(2 * W) * kCtTile * 8);
  }
};

// Block b maps tiles [b per, min(ntiles, (b + 1) per)) of the N terms of t
// in place.  Every plane of t starts on a 16-byte boundary and t.cap is a
// multiple of 4 (the host checks both), so the loads, rounded up to 16
// bytes, stay inside the planes, and the stores write exactly the tile.  A
// copy that does not complete within `spin_limit` tries sets kErrSpin in
// *serr, and the block returns once its copies in flight are done.
template <int W, int CB, typename WT>
__global__ void __launch_bounds__(kXsThreads, 2)
    k_clifford_tiles(TermsT<WT> t, const unsigned long long* n_in, const uint64_t* tab_xz,
                     const uint8_t* tab_e, int chunks, uint64_t live, PassMasks pmk, size_t per,
                     unsigned spin_limit, unsigned* serr) {
  constexpr int E = 1 << (2 * CB);
  extern __shared__ __align__(16) unsigned char s_raw[];
  __shared__ __align__(8) uint64_t s_full[2];
  const unsigned tid = threadIdx.x;
  uint64_t* s_tab = reinterpret_cast<uint64_t*>(s_raw);
  uint8_t* s_e = reinterpret_cast<uint8_t*>(s_tab + size_t(chunks) * E * 2 * W);
  const size_t tbytes = (size_t(chunks) * E * (16 * W + 1) + 15) & ~size_t(15);
  auto stage = [&](size_t k) {
    return CtStage<W, WT>{s_raw + tbytes + (k & 1) * ct_stage_bytes<W, WT>()};
  };
  const size_t N = *n_in;
  const size_t ntiles_all = (N + kCtTile - 1) / kCtTile;
  const size_t k0 = min(ntiles_all, size_t(blockIdx.x) * per);
  const size_t ntiles = min(ntiles_all, k0 + per) - k0;
  auto tile_n = [&](size_t k) {
    return unsigned(min(size_t(kCtTile), N - (k0 + k) * size_t(kCtTile)));
  };
  auto issue = [&](size_t k) {  // one thread: bulk loads of tile k into its stage
    const CtStage<W, WT> sg = stage(k);
    uint64_t* bar = &s_full[k & 1];
    const size_t p0 = (k0 + k) * kCtTile;
    const unsigned m = tile_n(k);
    const unsigned b8 = (m * 8 + 15) & ~15u, bw = (m * unsigned(sizeof(WT)) + 15) & ~15u;
    mbar_expect_tx(bar, 2 * W * b8 + bw);
#pragma unroll
    for (int q = 0; q < W; ++q) {
      bulk_g2s(sg.x(q), t.x + size_t(q) * t.cap + p0, b8, bar);
      bulk_g2s(sg.z(q), t.z + size_t(q) * t.cap + p0, b8, bar);
    }
    bulk_g2s(sg.w(), t.w + p0, bw, bar);
  };
  if (tid == 0) {
    mbar_init(&s_full[0], 1);
    mbar_init(&s_full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (size_t k = 0; k < 2 && k < ntiles; ++k) issue(k);
  load_clifford_table<CB, W>(s_tab, s_e, tab_xz, tab_e, chunks);
  __syncthreads();
  CliffCache<W> cc;
  for (size_t k = 0; k < ntiles; ++k) {
    const CtStage<W, WT> sg = stage(k);
    const unsigned m = tile_n(k);
    const bool ok = mbar_wait_bounded(&s_full[k & 1], unsigned(k >> 1) & 1u, spin_limit);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        atomicOr(serr, kErrSpin);
        for (size_t j = k; j < k + 2 && j < ntiles; ++j)
          mbar_wait_bounded(&s_full[j & 1], unsigned(j >> 1) & 1u, spin_limit);
        bulk_wait_all();
      }
      return;
    }
#pragma unroll
    for (int it = 0; it < kCtPer; ++it) {
      const unsigned i = kCtPer * tid + unsigned(it);
      if (i >= m) continue;
      uint64_t x[W], z[W];
#pragma unroll
      for (int q = 0; q < W; ++q) {
        x[q] = sg.x(q)[i];
        z[q] = sg.z(q)[i];
      }
      const bool neg = clifford_table_map<W, CB>(x, z, s_tab, s_e, chunks, live, pmk, cc);
#pragma unroll
      for (int q = 0; q < W; ++q) {
        sg.x(q)[i] = x[q];
        sg.z(q)[i] = z[q];
      }
      if (neg) sg.w()[i] = wneg(sg.w()[i]);
    }
    fence_proxy_async_smem();  // the mapped tile, before the bulk copies read it
    __syncthreads();
    if (tid == 0) {
      const size_t p0 = (k0 + k) * kCtTile;
      const unsigned nb = m & ~3u;  // a multiple of 16 bytes in every plane
      if (nb) {
#pragma unroll
        for (int q = 0; q < W; ++q) {
          bulk_s2g(t.x + size_t(q) * t.cap + p0, sg.x(q), nb * 8);
          bulk_s2g(t.z + size_t(q) * t.cap + p0, sg.z(q), nb * 8);
        }
        bulk_s2g(t.w + p0, sg.w(), nb * unsigned(sizeof(WT)));
        bulk_commit();
      }
      for (unsigned i = nb; i < m; ++i) {  // the last tile's ragged end
#pragma unroll
        for (int q = 0; q < W; ++q) {
          t.x[size_t(q) * t.cap + p0 + i] = sg.x(q)[i];
          t.z[size_t(q) * t.cap + p0 + i] = sg.z(q)[i];
        }
        t.w[p0 + i] = sg.w()[i];
      }
      if (k + 2 < ntiles) {
        bulk_wait_read();  // the stores have read the stage: it may be refilled
        issue(k + 2);
      }
    }
  }
  if (tid == 0) bulk_wait_all();
}

}  // namespace dev
}  // namespace qx
