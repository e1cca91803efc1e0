// Fast path of the merge step (A6) for one-word strings, included by
// qx_kernels.cuh after the shared helpers (TermsT, FanQ, key packing, hashing,
// staging) it uses.  Kept in its own file so that profiles of these two kernels
// can be tied to their exact source.
#pragma once

namespace qx {
namespace dev {

// ---------------------------------------------------------------------------
// A6, one-word strings (n < 64): the group key fits in 128 bits.
//
// The generator id is packed into the free high bits of the two key words
// (bits n..63 of x, then of z) and bit q of the x word is set as a marker, so
// the all-zero pair never occurs as a key and marks an empty slot.
//
// Insert pass (one thread per term, coalesced): terms that need no merge write
// their children at once; the others claim or find their group's slot with
// one 128-bit compare-and-swap and store their weight in the slot, in the
// position of their letter among the qubit's non-isolated rows.  A weight slot
// holding the sentinel bit pattern is absent (no counters, no atomics, no
// leader: nothing waits on anything).
//
// Group pass (one thread per slot of the active region, coalesced): every
// occupied slot is a group; its strings and generator are unpacked from the
// key, its children written with weights sum_p t[p][c] v_p in the fixed order
// p = X, Y, Z, and the slot reset.  The table is empty again after every pass.

// One 32-byte sector per slot: the key and the weights of ranks 0 and 1.  A
// qubit with three non-isolated rows keeps its rank-2 weights in a side array
// indexed like the slots.
struct FastSlot {
  unsigned long long klo, khi;  // packed key; 0, 0 = empty
  double v[2];                  // member weights by rank among non-isolated rows
};

constexpr unsigned long long kAbsent = 0x7ff4dead7ff4deadull;  // a NaN never computed

__device__ __forceinline__ void cas128(unsigned long long* p, unsigned long long cmp_lo,
                                       unsigned long long cmp_hi, unsigned long long new_lo,
                                       unsigned long long new_hi, unsigned long long* old_lo,
                                       unsigned long long* old_hi) {
  asm volatile(
      "{\n\t.reg .b128 d, b, c;\n\t"
      "mov.b128 b, {%2, %3};\n\t"
      "mov.b128 c, {%4, %5};\n\t"
      "atom.global.cas.b128 d, [%6], b, c;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(*old_lo), "=l"(*old_hi)
      : "l"(cmp_lo), "l"(cmp_hi), "l"(new_lo), "l"(new_hi), "l"(p)
      : "memory");
}

__device__ __forceinline__ void pack_key(uint64_t x, uint64_t z, uint32_t g, int n, int q,
                                         unsigned long long* lo, unsigned long long* hi) {
  const uint64_t qm = 1ull << q;
  const int fb = 64 - n;  // free high bits per word, >= 1
  *lo = (x & ~qm) | qm | (uint64_t(g) << n);
  *hi = (z & ~qm) | (fb < 32 ? (uint64_t(g) >> fb) << n : 0ull);
}

// Slot hash of a packed key: one 64-bit multiply after folding the words.
__device__ __forceinline__ uint64_t slot_hash(unsigned long long lo, unsigned long long hi) {
  uint64_t h = (lo ^ (hi * 0x9e3779b97f4a7c15ull)) * 0xd6e8feb86659fd93ull;
  return h ^ (h >> 32);
}

__device__ __forceinline__ void unpack_key(unsigned long long lo, unsigned long long hi, int n,
                                           int q, uint64_t* x, uint64_t* z, uint32_t* g) {
  const uint64_t low = (1ull << n) - 1;  // n < 64
  const int fb = 64 - n;
  *x = lo & low & ~(1ull << q);
  *z = hi & low;
  *g = uint32_t((lo >> n) | (fb < 32 ? (hi >> n) << fb : 0ull));
}

// Active slots of a pass: 1.25 times its input count (load <= 0.8 even if
// no two terms merge), at least 1024.
__device__ __forceinline__ unsigned long long active_slots(size_t N, unsigned long long tcap) {
  return min(tcap, max(1024ull, (unsigned long long)N + ((unsigned long long)N >> 2)));
}

static __global__ void k_fast_table_init(FastSlot* tab, double* v2, unsigned long long cap) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    tab[i].klo = 0ull;
    tab[i].khi = 0ull;
    tab[i].v[0] = __longlong_as_double(kAbsent);
    tab[i].v[1] = __longlong_as_double(kAbsent);
    v2[i] = __longlong_as_double(kAbsent);
  }
}

// Block-wide output allocation: returns this thread's first output index.
template <int THREADS>
__device__ __forceinline__ size_t alloc_out(unsigned c, unsigned* s_scan,
                                            unsigned long long* s_base,
                                            unsigned long long* n_out) {
  unsigned total;
  const unsigned off = block_excl_scan<THREADS>(c, &total, s_scan);
  if (threadIdx.x == 0) *s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0;
  __syncthreads();
  const size_t base = size_t(*s_base) + off;
  __syncthreads();
  return base;
}


// One-word children of a block, staged in shared memory and written out with
// consecutive threads on consecutive terms.  Each thread contributes up to 3
// children (x, z, w, g) at block-local offsets from the block scan.
template <int THREADS, typename WT = double>
struct StageOut {
  uint64_t x[3 * THREADS];
  uint64_t z[3 * THREADS];
  WT w[3 * THREADS];
  uint32_t g[3 * THREADS];
};

template <int THREADS, typename WT = double>
__device__ __forceinline__ void flush_stage(StageOut<THREADS, WT>& st, unsigned total, size_t base,
                                            const TermsT<WT>& out) {
  for (unsigned k = threadIdx.x; k < total; k += THREADS) {
    __stcs(&out.x[base + k], st.x[k]);
    __stcs(&out.z[base + k], st.z[k]);
    __stcs(&out.w[base + k], st.w[k]);
    __stcs(&out.g[base + k], st.g[k]);
  }
}

template <int THREADS, typename WT = double>
__global__ void __launch_bounds__(THREADS, 4) k_merge_insert_fast(
    TermsT<WT> t, const unsigned long long* n_in, int n, int q, const __grid_constant__ FanQ fq_p,
    const uint64_t* mixed, FastSlot* tab, double* tab_v2, unsigned long long tcap, double eps,
    double* pruned, TermsT<WT> out, unsigned long long* n_out, unsigned* err) {
  // the table is read with per-thread letter indices: a shared copy keeps
  // those reads parallel (divergent reads of kernel parameters serialise)
  __shared__ FanQ fq;
  __shared__ unsigned s_scan[THREADS / 32 + 1];
  __shared__ unsigned long long s_base;
  __shared__ unsigned s_err;
  __shared__ StageOut<THREADS, WT> st;
  if (threadIdx.x == 0) {
    fq = fq_p;
    s_err = *(volatile const unsigned*)err;
  }
  __syncthreads();
  // after an overflow (flagged in *err) the chain of passes stops: the
  // buffer may hold unwritten entries, and the host redoes the step
  if (s_err) return;
  const size_t N = min(size_t(*n_in), t.cap);
  const unsigned long long teff = active_slots(N, tcap);
  const uint64_t qm = 1ull << q;
  constexpr int ITEMS = 2;  // terms per thread per tile: two CAS chains in flight
  for (size_t tile = size_t(blockIdx.x) * THREADS * ITEMS; tile < N;
       tile += size_t(gridDim.x) * THREADS * ITEMS) {
    uint64_t x[ITEMS], z[ITEMS];
    uint32_t g[ITEMS];
    WT w[ITEMS];
    int p[ITEMS];
    bool hashed[ITEMS];
    unsigned long long pos[ITEMS], klo[ITEMS], khi[ITEMS];
    int cl[3];
    WT cw[3];
    uint64_t cx0 = 0, cz0 = 0;
    uint32_t cg0 = 0;
    unsigned c = 0;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      const size_t i = tile + size_t(it) * THREADS + threadIdx.x;
      hashed[it] = false;
      p[it] = -1;
      if (i >= N) continue;
      // the term streams are read once: evict-first keeps the table in L2
      x[it] = __ldcs(&t.x[i]);
      z[it] = __ldcs(&t.z[i]);
      g[it] = __ldcs(&t.g[i]);
      w[it] = __ldcs(&t.w[i]);
      const int xb = int((x[it] >> q) & 1), zb = int((z[it] >> q) & 1);
      if (xb | zb) {
        p[it] = xb ? (zb ? 1 : 0) : 2;
        hashed[it] = !fq.iso[p[it]] && (mixed[g[it]] & qm);
      }
      if (hashed[it]) {
        pack_key(x[it], z[it], g[it], n, q, &klo[it], &khi[it]);
        pos[it] = __umul64hi(slot_hash(klo[it], khi[it]), teff);
      }
    }
    // claim or find the group slots (independent chains per item)
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      if (!hashed[it]) continue;
      bool done = false;
      for (unsigned long long probe = 0; probe < teff; ++probe) {
        unsigned long long olo, ohi;
        cas128(&tab[pos[it]].klo, 0ull, 0ull, klo[it], khi[it], &olo, &ohi);
        if ((olo | ohi) == 0ull || (olo == klo[it] && ohi == khi[it])) {
          done = true;
          break;
        }
        if (++pos[it] == teff) pos[it] = 0;
      }
      if (done) {
        const int rank = (p[it] > 0 && !fq.iso[0]) + (p[it] > 1 && !fq.iso[1]);
        if (rank < 2)
          tab[pos[it]].v[rank] = double(w[it]);
        else
          tab_v2[pos[it]] = double(w[it]);
      } else {
        atomicOr(err, kErrProbe);
      }
    }
    // children of the terms that need no merge (at most 3 per item)
    unsigned cn[ITEMS];
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      cn[it] = 0;
      const size_t i = tile + size_t(it) * THREADS + threadIdx.x;
      if (i >= N || hashed[it]) continue;
      cn[it] = p[it] < 0 ? 1u : unsigned(fq.nnz[p[it]]);
    }
    const bool any = __syncthreads_or(int(cn[0] | cn[1]));
    if (!any) continue;
#pragma unroll
    for (int it = 0; it < ITEMS; ++it) {
      c = 0;
      if (cn[it]) {
        auto keep = [&](int letter, WT v) {
          if (eps > 0.0 && fabs(double(v)) < eps) {
            atomicAdd(&pruned[g[it]], double(v) * double(v));
            return;
          }
          cl[c] = letter;
          cw[c] = v;
          ++c;
        };
        if (p[it] < 0) {
          keep(-1, w[it]);
        } else {
          for (int j = 0; j < fq.nnz[p[it]]; ++j) {
            const int col = fq.col[p[it]][j];
            keep(col, wmul(w[it], fq, p[it], col));
          }
        }
        cx0 = x[it];
        cz0 = z[it];
        cg0 = g[it];
      }
      unsigned total;
      const unsigned off = block_excl_scan<THREADS>(c, &total, s_scan);
      for (unsigned j = 0; j < c; ++j) {
        uint64_t cx = cx0, cz = cz0;
        if (cl[j] >= 0) {
          cx = (cl[j] <= 1) ? (cx | qm) : (cx & ~qm);
          cz = (cl[j] >= 1) ? (cz | qm) : (cz & ~qm);
        }
        st.x[off + j] = cx;
        st.z[off + j] = cz;
        st.w[off + j] = cw[j];
        st.g[off + j] = cg0;
      }
      if (threadIdx.x == 0) s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0;
      __syncthreads();
      const size_t base = size_t(s_base);
      if (base + total > out.cap) {
        if (threadIdx.x == 0 && total) atomicOr(err, kErrCap);
      } else {
        flush_stage<THREADS>(st, total, base, out);
      }
      __syncthreads();
    }
  }
}

template <int THREADS, typename WT = double>
__global__ void __launch_bounds__(THREADS) k_merge_groups_fast(
    const unsigned long long* n_in, size_t in_cap, int n, int q,
    const __grid_constant__ FanQ fq_p, FastSlot* tab, double* tab_v2, unsigned long long tcap,
    double eps, double* pruned, TermsT<WT> out, unsigned long long* n_out, unsigned* err) {
  __shared__ FanQ fq;
  __shared__ unsigned s_scan[THREADS / 32 + 1];
  __shared__ unsigned long long s_base;
  __shared__ unsigned s_err;
  __shared__ StageOut<THREADS, WT> st;
  if (threadIdx.x == 0) {
    fq = fq_p;
    s_err = *(volatile const unsigned*)err;
  }
  __syncthreads();
  if (s_err) return;
  const unsigned long long teff = active_slots(min(size_t(*n_in), in_cap), tcap);
  const uint64_t qm = 1ull << q;
  // rank of each letter among the non-isolated rows (-1: isolated)
  int rank_of[3];
  {
    int r = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) rank_of[a] = fq.iso[a] ? -1 : r++;
  }
  const bool three = rank_of[0] >= 0 && rank_of[1] >= 0 && rank_of[2] >= 0;
  for (unsigned long long tile = (unsigned long long)blockIdx.x * THREADS; tile < teff;
       tile += (unsigned long long)gridDim.x * THREADS) {
    const unsigned long long sidx = tile + threadIdx.x;
    uint64_t x = 0, z = 0;
    uint32_t g = 0;
    int cl[3];
    WT cw[3];
    unsigned c = 0;
    if (sidx < teff) {
      // the key and the first two weights share one 32-byte sector
      ulonglong2* s0 = reinterpret_cast<ulonglong2*>(&tab[sidx]);
      const ulonglong2 key = s0[0];
      if (key.x | key.y) {
        const ulonglong2 vv = s0[1];
        const unsigned long long vb[3] = {vv.x, vv.y,
                                          three ? __double_as_longlong(tab_v2[sidx]) : kAbsent};
        WT v[3];
        bool has[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          has[a] = rank_of[a] >= 0 && vb[rank_of[a]] != kAbsent;
          v[a] = has[a] ? WT(__longlong_as_double(vb[rank_of[a]])) : WT(0);
        }
        s0[0] = make_ulonglong2(0ull, 0ull);
        s0[1] = make_ulonglong2(kAbsent, kAbsent);
        if (three) tab_v2[sidx] = __longlong_as_double(kAbsent);
        unpack_key(key.x, key.y, n, q, &x, &z, &g);
#pragma unroll
        for (int col = 0; col < 3; ++col) {
          bool reached = false;
          const WT acc = group_sum(fq, col, has, v, &reached);
          if (reached) {
            if (eps > 0.0 && fabs(double(acc)) < eps) {
              atomicAdd(&pruned[g], double(acc) * double(acc));
            } else {
              cl[c] = col;
              cw[c] = acc;
              ++c;
            }
          }
        }
      }
    }
    if (!__syncthreads_or(int(c))) continue;
    unsigned total;
    const unsigned off = block_excl_scan<THREADS>(c, &total, s_scan);
    for (unsigned j = 0; j < c; ++j) {
      st.x[off + j] = (cl[j] <= 1) ? (x | qm) : x;
      st.z[off + j] = (cl[j] >= 1) ? (z | qm) : z;
      st.w[off + j] = cw[j];
      st.g[off + j] = g;
    }
    if (threadIdx.x == 0) s_base = atomicAdd(n_out, (unsigned long long)total);
    __syncthreads();
    const size_t base = size_t(s_base);
    if (base + total > out.cap) {
      if (threadIdx.x == 0) atomicOr(err, kErrCap);
    } else {
      flush_stage<THREADS>(st, total, base, out);
    }
    __syncthreads();
  }
}

}  // namespace dev
}  // namespace qx
