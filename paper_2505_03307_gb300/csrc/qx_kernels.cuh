// Device kernels of libqx (sm_103a).
//
// Terms live in HBM as structure-of-arrays: x and z bit planes (W words per
// string, plane k at x + k * cap), an FP64 weight and a 32-bit generator id per
// term.  Every kernel is a grid-stride loop whose bound is read from device
// memory, so a launch does not need the host to know the current count.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace qx {
namespace dev {

constexpr unsigned kErrProbe = 1u;    // a hash table ran out of probes
constexpr unsigned kErrSpin = 2u;     // a bounded wait gave up
constexpr unsigned kErrCap = 4u;      // an output buffer was too small

// WT: weight type, double (FP64 path) or float (FP32 path with compensated
// arithmetic).  Strings, generator ids and signs are exact in both.
template <typename WT>
struct TermsT {
  uint64_t* x;
  uint64_t* z;
  WT* w;
  uint32_t* g;
  size_t cap;
};
using Terms = TermsT<double>;

// Keeps a parameter out of template deduction (the weight converts to WT).
template <typename T>
struct NoDeduce {
  using type = T;
};

// A fan-out qubit as the kernels see it.
struct FanQ {
  double t[3][3];
  float th[3][3], tl[3][3];  // t = th + tl to about 2^-48 (FP32 path)
  int q;
  uint8_t nnz[3];
  uint8_t col[3][3];
  uint8_t iso[3];
  uint8_t pad;
  uint16_t nz;   // bit 3a + c: t[a][c] != 0 (integer tests keep the FP64 pipe free)
  uint16_t pad2;
};

// Sets FanQ::nz from the table (every builder of a FanQ calls this last).
inline void fanq_set_nz(FanQ* f) {
  f->nz = 0;
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      if (f->t[a][c] != 0.0) f->nz = uint16_t(f->nz | (1u << (3 * a + c)));
}

// ---------------------------------------------------------------------------
// Weight arithmetic.  FP64 weights multiply and add plainly.  FP32 weights use
// each table entry split into float hi + lo and recover the rounding error of
// the leading product with an FMA (TwoProduct); group sums add those pairs
// with TwoSum (the Dot2 scheme of Ogita, Rump and Oishi), so every child or
// merged weight carries about one float rounding whatever the cancellation.

__device__ __forceinline__ double wmul(double w, const FanQ& f, int a, int c) {
  return w * f.t[a][c];
}

// w t for t = th + tl (hi / lo floats): the leading product and its rounding
// error (TwoProduct by FMA) plus the low part.
__device__ __forceinline__ float wmul_split(float w, float th, float tl) {
  const float p = w * th;
  return p + fmaf(w, tl, fmaf(w, th, -p));
}

__device__ __forceinline__ float wmul(float w, const FanQ& f, int a, int c) {
  return wmul_split(w, f.th[a][c], f.tl[a][c]);
}

// One member of a compensated group sum (Dot2 of Ogita, Rump and Oishi): adds
// v t, t = th + tl, to (sum, comp); the first member starts the sum.
__device__ __forceinline__ void dot2_add(float v, float th, float tl, bool* any, float* sum,
                                         float* comp) {
  const float p = v * th;
  const float pe = fmaf(v, th, -p) + v * tl;
  if (!*any) {
    *sum = p;
    *comp = pe;
    *any = true;
  } else {
    const float t = *sum + p;  // TwoSum
    const float bp = t - *sum;
    *comp += ((*sum - (t - bp)) + (p - bp)) + pe;
    *sum = t;
  }
}

// sum over the present letters a (in the order X, Y, Z) of t[a][col] v[a],
// one fused multiply-add per member starting from 0 (the FP64 pipe is the
// scarce unit on this GPU); *reached: some present letter reaches col
__device__ __forceinline__ double group_sum(const FanQ& f, int col, const bool* has,
                                            const double* v, bool* reached) {
  bool any = false;
  double acc = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (has[a] && ((f.nz >> (3 * a + col)) & 1)) {
      acc = fma(f.t[a][col], v[a], acc);
      any = true;
    }
  }
  *reached = any;
  return acc;
}

__device__ __forceinline__ float group_sum(const FanQ& f, int col, const bool* has,
                                           const float* v, bool* reached) {
  bool any = false;
  float sum = 0.f, comp = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (has[a] && ((f.nz >> (3 * a + col)) & 1)) dot2_add(v[a], f.th[a][col], f.tl[a][col], &any, &sum, &comp);
  *reached = any;
  return sum + comp;
}

// Sign flip by the sign bit (an integer operation: the FP64 unit is the
// scarce one on this GPU); bit-identical to IEEE negation.
__device__ __forceinline__ double wneg(double w) {
  return __longlong_as_double(__double_as_longlong(w) ^ (1ll << 63));
}
__device__ __forceinline__ float wneg(float w) {
  return __uint_as_float(__float_as_uint(w) ^ 0x80000000u);
}

// Lanes of the warp holding the same key as this lane.  Terms of one
// generator (or one block) usually sit together, so a warp-wide equality vote
// answers most calls without the match instruction.
__device__ __forceinline__ unsigned warp_peers(unsigned key) {
  const unsigned k0 = __shfl_sync(0xffffffffu, key, 0);
  if (__all_sync(0xffffffffu, key == k0)) return 0xffffffffu;
  return __match_any_sync(0xffffffffu, key);
}

// Contiguous range of terms for the calling warp: [*b, *e), a multiple of 32
// long, so that a warp's terms (usually of one generator) are read once and
// in order.
__device__ __forceinline__ void warp_range(size_t N, size_t* b, size_t* e) {
  const size_t nw = size_t(gridDim.x) * (blockDim.x >> 5);
  const size_t w = size_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const size_t per = (((N + nw - 1) / nw) + 31) & ~size_t(31);
  *b = min(N, w * per);
  *e = min(N, *b + per);
}

// Running product of a weight with table entries (the Cartesian expansion).
template <typename WT>
struct WProd;

template <>
struct WProd<double> {
  double v;
  __device__ __forceinline__ explicit WProd(double w) : v(w) {}
  __device__ __forceinline__ void mul(const FanQ& f, int a, int c) { v *= f.t[a][c]; }
  // one table entry given directly (t, and its float split for FP32)
  __device__ __forceinline__ void mul_entry(double t, float, float) { v *= t; }
  __device__ __forceinline__ double get() const { return v; }
};

template <>
struct WProd<float> {  // float-float (hi, lo) product
  float hi, lo;
  __device__ __forceinline__ explicit WProd(float w) : hi(w), lo(0.f) {}
  __device__ __forceinline__ void mul(const FanQ& f, int a, int c) {
    mul_entry(0.0, f.th[a][c], f.tl[a][c]);
  }
  __device__ __forceinline__ void mul_entry(double, float th, float tl) {
    const float p = hi * th;
    const float e = fmaf(hi, th, -p) + fmaf(hi, tl, lo * th);
    hi = p + e;  // renormalise (FastTwoSum: |p| >= |e|)
    lo = e - (hi - p);
  }
  __device__ __forceinline__ float get() const { return hi + lo; }
};

// ---------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t fmix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

template <int W>
__device__ __forceinline__ uint64_t key_hash(uint32_t g, const uint64_t* kx, const uint64_t* kz) {
  uint64_t h = fmix64(0x9e3779b97f4a7c15ull * (uint64_t(g) + 1));
#pragma unroll
  for (int k = 0; k < W; ++k) {
    h = fmix64(h ^ kx[k]);
    h = fmix64(h + 0x632be59bd9b4e019ull + kz[k]);
  }
  return h;
}

// Pauli letter of qubit q: 0 = I, 1 = X, 2 = Y, 3 = Z (as (x, z) bits).
template <int W>
__device__ __forceinline__ int letter_at(const uint64_t* x, const uint64_t* z, int q) {
  // the word by a select: a run-time index would put the string in local memory
  const bool hi = W > 1 && q >= 64;
  const int b = q & 63;
  const int xb = int(((hi ? x[W - 1] : x[0]) >> b) & 1), zb = int(((hi ? z[W - 1] : z[0]) >> b) & 1);
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

// Sets qubit q to table letter c (0 = X, 1 = Y, 2 = Z).
template <int W>
__device__ __forceinline__ void set_letter(uint64_t* x, uint64_t* z, int q, int c) {
  const uint64_t m = 1ull << (q & 63);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const uint64_t mk = (k == (q >> 6)) ? m : 0ull;
    x[k] = (c <= 1) ? (x[k] | mk) : (x[k] & ~mk);
    z[k] = (c >= 1) ? (z[k] | mk) : (z[k] & ~mk);
  }
}

template <int W, typename WT = double>
__device__ __forceinline__ void load_term(const TermsT<WT>& t, size_t i, uint64_t* x, uint64_t* z) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    x[k] = t.x[k * t.cap + i];
    z[k] = t.z[k * t.cap + i];
  }
}

template <int W, typename WT = double>
__device__ __forceinline__ void store_term(const TermsT<WT>& t, size_t i, const uint64_t* x,
                                           const uint64_t* z, typename NoDeduce<WT>::type w,
                                           uint32_t g) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    t.x[k * t.cap + i] = x[k];
    t.z[k * t.cap + i] = z[k];
  }
  t.w[i] = w;
  t.g[i] = g;
}

// Block-wide exclusive scan of one unsigned value per thread; returns the
// thread's offset and writes the block total to *total (all threads).
template <int THREADS>
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* total,
                                                    unsigned* smem /* THREADS/32 + 1 */) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned inc = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) smem[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = THREADS / 32;
    unsigned s = lane < NW ? smem[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned o = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += o;
    }
    if (lane < NW) smem[lane] = s;  // inclusive warp prefix
    if (lane == NW - 1) smem[NW] = s;
  }
  __syncthreads();
  const unsigned warp_base = wid ? smem[wid - 1] : 0;
  *total = smem[THREADS / 32];
  const unsigned r = warp_base + inc - v;
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// A3: create_Z_j

template <int W, typename WT = double>
__global__ void k_init_z(TermsT<WT> t, int g0, int G, unsigned long long* n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G) {
    uint64_t x[W], z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] = 0;
      z[k] = 0;
    }
    const int j = g0 + i;
    z[j >> 6] = 1ull << (j & 63);
    store_term<W>(t, i, x, z, 1.0, uint32_t(i));
  }
  if (i == 0) *n_out = (unsigned long long)G;
}

// ---------------------------------------------------------------------------
// A4: fused Clifford pass, in place (bijection on strings: no merge).
//
// Gate-list form: the ops of the pass are applied one after another with the
// CHP bit rules.  Table form: the string is split into chunks of CB qubits;
// the XZ-form image of each chunk's X^a Z^b is read from a shared-memory table
// and the images are multiplied, tracking the phase with popcounts.

template <int W>
__device__ __forceinline__ void apply_ops(const uint32_t* ops, int nops, uint64_t* x, uint64_t* z,
                                          int* neg) {
  for (int i = 0; i < nops; ++i) {
    const uint32_t op = ops[i];
    const uint32_t kind = op & 3;
    const int a = (op >> 2) & 127, b = (op >> 9) & 127;
    const int ka = a >> 6, sa = a & 63, kb = b >> 6, sb = b & 63;
    if (kind == 1u) {  // CX(a -> b)
      const uint64_t xa = (x[ka] >> sa) & 1, za = (z[ka] >> sa) & 1;
      const uint64_t xb = (x[kb] >> sb) & 1, zb = (z[kb] >> sb) & 1;
      *neg ^= int(xa & zb & (1 ^ xb ^ za));
      x[kb] ^= xa << sb;
      z[ka] ^= zb << sa;
    } else if (kind == 2u) {  // CZ(a, b)
      const uint64_t xa = (x[ka] >> sa) & 1, za = (z[ka] >> sa) & 1;
      const uint64_t xb = (x[kb] >> sb) & 1, zb = (z[kb] >> sb) & 1;
      *neg ^= int(xa & xb & (za ^ zb));
      z[kb] ^= xa << sb;
      z[ka] ^= xb << sa;
    } else {  // signed permutation of (X, Y, Z) on qubit a
      const uint64_t xa = (x[ka] >> sa) & 1, za = (z[ka] >> sa) & 1;
      if (xa | za) {
        const int p = xa ? (za ? 1 : 0) : 2;
        const uint32_t f = (op >> (16 + 3 * p)) & 7, to = f & 3;
        const uint64_t m = 1ull << sa;
        x[ka] = (to <= 1) ? (x[ka] | m) : (x[ka] & ~m);
        z[ka] = (to >= 1) ? (z[ka] | m) : (z[ka] & ~m);
        *neg ^= int(f >> 2);
      }
    }
  }
}

template <int W, typename WT = double>
__global__ void __launch_bounds__(256) k_clifford_ops(TermsT<WT> t, const unsigned long long* n_in,
                                                      const uint32_t* ops, int nops) {
  extern __shared__ uint32_t s_ops[];
  for (int i = threadIdx.x; i < nops; i += blockDim.x) s_ops[i] = ops[i];
  __syncthreads();
  const size_t N = *n_in;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
    load_term<W>(t, i, x, z);
    int neg = 0;
    apply_ops<W>(s_ops, nops, x, z, &neg);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      t.x[k * t.cap + i] = x[k];
      t.z[k * t.cap + i] = z[k];
    }
    if (neg) t.w[i] = wneg(t.w[i]);
  }
}

// Parts of the chunks of a table-form pass (each part's product is cached
// per lane); the host assigns the chunks to them (pass_masks).
template <int W>
__host__ __device__ constexpr int clifford_parts() {
  return 3;
}

// Qubit masks of a Clifford pass for k_clifford_table: the qubits that no
// gate of the pass acts on (idle: their letters map to themselves), per part
// the live chunks it takes (pchunks) and their other qubits (the letters its
// product depends on).  Parts need not be contiguous: the images of
// different chunks are images of Paulis on disjoint qubits, so they commute
// and their product does not depend on the order they are taken in.
struct PassMasks {
  uint64_t idle[kMaxWords];
  uint64_t part[3][kMaxWords];
  uint64_t pchunks[3];
  uint64_t rest[kMaxWords];  // part[1] | part[2]
};

// The image of a string is the product of its chunks' images, in chunk order
// (X then Z letters within a chunk).  Three facts cut the table lookups:
// * a qubit that no gate of the pass touches maps to itself; its letter
//   passes through (its image has disjoint support from every other image, so
//   it adds no phase), the chunk index is taken with its bits cleared, and a
//   chunk with no touched qubit is never looked up (`live`);
// * the chunks split into P parts; the product of a part, with its phase, is
//   kept per lane together with the part's letters that produced it, and
//   reused while the lane's next string has the same letters there (strings of
//   one generator that differ only on fan-out wires share most parts).  When
//   the planner knows on which qubits one generator's terms can differ (the
//   fan-out wires before the pass, carried through the passes between), part
//   0 holds exactly the chunks of those qubits and the other parts stay
//   cached along a generator's terms;
// * the parts combine in order: the phase gains 2 |z_acc & x_part| (mod 4),
//   which equals the sum of the per-chunk terms mod 2.
//
// CliffCache holds a lane's part products; clifford_table_map maps one string
// in place through the chunk tables in shared memory and returns whether its
// weight changes sign.  k_clifford_table applies it in place; the fused
// expansion applies it to each parent before emitting its children.
template <int W>
struct CliffCache {
  static constexpr int P = clifford_parts<W>();
  uint64_t kx[P][W], kz[P][W], vx[P][W], vz[P][W];
  int ve[P];
  unsigned valid = 0;
  // the product of parts 1 .. P-1 and the letters it came from, so that a
  // string whose letters changed in part 0 only takes one check for them
  uint64_t ukx[W], ukz[W], ux[W], uz[W];
  int ue = 0;
  bool uvalid = false;
};

template <int W, int CB>
__device__ __forceinline__ bool clifford_table_map(uint64_t* x, uint64_t* z, const uint64_t* s_tab,
                                                   const uint8_t* s_e, int chunks, uint64_t live,
                                                   const PassMasks& pmk, CliffCache<W>& cc) {
  constexpr int E = 1 << (2 * CB);
  constexpr int P = clifford_parts<W>();
  constexpr uint32_t M = (1u << CB) - 1;
  int e = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) e += __popcll(x[k] & z[k]);

  // the product of part p (from the lane's cache, or its chunks)
  auto part_product = [&](int p) {
    bool same = (cc.valid >> p) & 1;
#pragma unroll
    for (int k = 0; k < W; ++k)
      same = same && cc.kx[p][k] == (x[k] & pmk.part[p][k]) && cc.kz[p][k] == (z[k] & pmk.part[p][k]);
    if (!same) {  // the product of this part's chunks
      uint64_t px[W], pz[W];
#pragma unroll
      for (int k = 0; k < W; ++k) {
        px[k] = 0;
        pz[k] = 0;
        cc.kx[p][k] = x[k] & pmk.part[p][k];
        cc.kz[p][k] = z[k] & pmk.part[p][k];
      }
      int pe = 0;
      for (uint64_t cm = pmk.pchunks[p]; cm; cm &= cm - 1) {
        const int c = __ffsll((long long)cm) - 1;
        const int lo = c * CB, k = lo >> 6, off = lo & 63;
        // for CB = 3 the chunk across the word boundary takes bits of both
        // words by selects, not by a run-time index (which would put the
        // string in local memory)
        // the letters of touched qubits only (the mask is a kernel parameter)
        const uint64_t iw = (W == 1 || k == 0) ? pmk.idle[0] : pmk.idle[W - 1];
        const uint64_t xw = ((W == 1 || k == 0) ? x[0] : x[W - 1]) & ~iw;
        const uint64_t zw = ((W == 1 || k == 0) ? z[0] : z[W - 1]) & ~iw;
        uint32_t xb, zb;
        if (CB == 4 || off + CB <= 64) {
          xb = uint32_t(xw >> off) & M;
          zb = uint32_t(zw >> off) & M;
        } else {  // k == 0 < W - 1
          const uint64_t ih = W > 1 ? ~pmk.idle[W - 1] : 0ull;
          xb = uint32_t((xw >> off) | (W > 1 ? ((x[W - 1] & ih) << (64 - off)) : 0)) & M;
          zb = uint32_t((zw >> off) | (W > 1 ? ((z[W - 1] & ih) << (64 - off)) : 0)) & M;
        }
        const uint32_t idx = xb | (zb << CB);
        if (!idx) continue;
        // the entry (x words, then z words) in 16-byte loads
        const ulonglong2* ent =
            reinterpret_cast<const ulonglong2*>(s_tab + (size_t(c) * E + idx) * 2 * W);
        uint64_t ex[W], ez[W];
        if (W == 1) {
          const ulonglong2 v = ent[0];
          ex[0] = v.x;
          ez[0] = v.y;
        } else {
          const ulonglong2 v0 = ent[0], v1 = ent[1];
          ex[0] = v0.x;
          ex[W - 1] = v0.y;
          ez[0] = v1.x;
          ez[W - 1] = v1.y;
        }
        int anti = 0;
#pragma unroll
        for (int kk = 0; kk < W; ++kk) anti += __popcll(pz[kk] & ex[kk]);
        pe += int(s_e[c * E + idx]) + 2 * anti;
#pragma unroll
        for (int kk = 0; kk < W; ++kk) {
          px[kk] ^= ex[kk];
          pz[kk] ^= ez[kk];
        }
      }
#pragma unroll
      for (int k = 0; k < W; ++k) {
        cc.vx[p][k] = px[k];
        cc.vz[p][k] = pz[k];
      }
      cc.ve[p] = pe & 3;
      cc.valid |= 1u << p;
    }
  };
  // parts 1 .. P-1: kept as one product while their letters stay the same
  bool up = cc.uvalid;
#pragma unroll
  for (int k = 0; k < W; ++k)
    up = up && cc.ukx[k] == (x[k] & pmk.rest[k]) && cc.ukz[k] == (z[k] & pmk.rest[k]);
  if (!up) {
    uint64_t ux[W], uz[W];
    int ue = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) ux[k] = uz[k] = 0;
#pragma unroll
    for (int p = 1; p < P; ++p) {
      part_product(p);
      int anti = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) anti += __popcll(uz[k] & cc.vx[p][k]);
      ue += cc.ve[p] + 2 * anti;
#pragma unroll
      for (int k = 0; k < W; ++k) {
        ux[k] ^= cc.vx[p][k];
        uz[k] ^= cc.vz[p][k];
      }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      cc.ukx[k] = x[k] & pmk.rest[k];
      cc.ukz[k] = z[k] & pmk.rest[k];
      cc.ux[k] = ux[k];
      cc.uz[k] = uz[k];
    }
    cc.ue = ue & 3;
    cc.uvalid = true;
  }
  // part 0, then the rest (the chunks' images commute: any order gives the
  // same product)
  part_product(0);
  uint64_t ax[W], az[W];
  int anti = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    anti += __popcll(cc.vz[0][k] & cc.ux[k]);
    ax[k] = cc.vx[0][k] ^ cc.ux[k];
    az[k] = cc.vz[0][k] ^ cc.uz[k];
  }
  e += cc.ve[0] + cc.ue + 2 * anti;
#pragma unroll
  for (int k = 0; k < W; ++k) {  // the letters the pass leaves alone
    ax[k] |= x[k] & pmk.idle[k];
    az[k] |= z[k] & pmk.idle[k];
  }
  int c2 = 0;
#pragma unroll
  for (int k = 0; k < W; ++k) c2 += __popcll(ax[k] & az[k]);
#pragma unroll
  for (int k = 0; k < W; ++k) {
    x[k] = ax[k];
    z[k] = az[k];
  }
  return ((e - c2) & 3) == 2;
}

// One-entry cache of a whole-string image: the image of a string depends
// only on its letters on the touched qubits (the others pass through and add
// nothing to the sign: their Y's count once in the string's exponent and once
// in the image's), so a lane whose next string has the same touched letters
// reuses the last image and sign (clifford_map_warp in the fused expansion).
template <int W>
struct FullCache {
  uint64_t kx[W], kz[W], rx[W], rz[W];
  bool neg;
  bool valid = false;
};

// Copies the chunk tables of a pass into shared memory (all threads), in
// 16-byte words with four loads of each thread in flight before their
// stores: both tables start on 256-byte boundaries of the plan's device copy
// and hold multiples of 16 bytes (E >= 64 entries per chunk), and s_tab, s_e
// are 16-byte aligned.  (One 8-byte word per thread and iteration waited on
// each load in turn: 25 us for the 70 KB of a 100-qubit pass.)
template <int CB, int W>
__device__ __forceinline__ void load_clifford_table(uint64_t* s_tab, uint8_t* s_e,
                                                    const uint64_t* tab_xz, const uint8_t* tab_e,
                                                    int chunks) {
  constexpr int E = 1 << (2 * CB);
  auto copy16 = [](uint4* dst, const uint4* src, int n) {
    const int B = int(blockDim.x);
    for (int i = threadIdx.x; i < n; i += 4 * B) {
      uint4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * B < n) v[u] = __ldg(src + i + u * B);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u * B < n) dst[i + u * B] = v[u];
    }
  };
  copy16(reinterpret_cast<uint4*>(s_tab), reinterpret_cast<const uint4*>(tab_xz),
         chunks * E * 2 * W * 8 / 16);
  copy16(reinterpret_cast<uint4*>(s_e), reinterpret_cast<const uint4*>(tab_e), chunks * E / 16);
}

// Each warp reads a contiguous range, so consecutive strings of a lane are
// close relatives.
template <int W, int CB, typename WT = double>
__global__ void __launch_bounds__(256) k_clifford_table(TermsT<WT> t, const unsigned long long* n_in,
                                                        const uint64_t* tab_xz,
                                                        const uint8_t* tab_e, int chunks,
                                                        uint64_t live, PassMasks pmk) {
  constexpr int E = 1 << (2 * CB);
  extern __shared__ __align__(16) uint64_t s_tab[];
  uint8_t* s_e = reinterpret_cast<uint8_t*>(s_tab + size_t(chunks) * E * 2 * W);
  load_clifford_table<CB, W>(s_tab, s_e, tab_xz, tab_e, chunks);
  __syncthreads();
  const size_t N = *n_in;
  CliffCache<W> cc;
  size_t rb, re;
  warp_range(N, &rb, &re);
  // the next string is loaded before the current one is mapped
  uint64_t nx[W], nz[W];
  {
    const size_t i0 = rb + (threadIdx.x & 31);
    if (i0 < re) load_term<W>(t, i0, nx, nz);
  }
  for (size_t i = rb + (threadIdx.x & 31); i < re; i += 32) {
    uint64_t x[W], z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] = nx[k];
      z[k] = nz[k];
    }
    if (i + 32 < re) load_term<W>(t, i + 32, nx, nz);
    const bool neg = clifford_table_map<W, CB>(x, z, s_tab, s_e, chunks, live, pmk, cc);
#pragma unroll
    for (int k = 0; k < W; ++k) {
      t.x[k * t.cap + i] = x[k];
      t.z[k * t.cap + i] = z[k];
    }
    if (neg) t.w[i] = wneg(t.w[i]);
  }
}

// ---------------------------------------------------------------------------
// A5/A6 preparation: which fan-out qubits need index accumulation.
//
// For every generator, OR over its terms of the qubits carrying X (resp. Y, Z)
// where that row of the qubit's table is not isolated.  A qubit whose
// non-isolated letters are all the same in a generator cannot make two of that
// generator's strings collide, so it is expanded without a merge.

template <int W, typename WT = double>
__global__ void k_fan_mask(TermsT<WT> t, const unsigned long long* n_in, const uint64_t* nisoX,
                           const uint64_t* nisoY, const uint64_t* nisoZ,
                           unsigned long long* gmask /* [G][3][W] */) {
  const size_t N = *n_in;
  const unsigned lane = threadIdx.x & 31;
  size_t b, e;
  warp_range(N, &b, &e);
  // running OR of a warp whose lanes all held generator cg (lane 0 adds it to
  // gmask when the generator changes and at the end)
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
  // the next 32 terms are loaded before the current ones are combined, so a
  // warp keeps one load in flight behind its shuffles
  uint32_t ng = 0xffffffffu;
  uint64_t nx[W], nz[W];
  auto fetch = [&](size_t base) {
    const size_t i = base + lane;
    const bool valid = base < e && i < e;
    ng = valid ? t.g[i] : 0xffffffffu;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      nx[k] = valid ? t.x[k * t.cap + i] : 0ull;
      nz[k] = valid ? t.z[k * t.cap + i] : 0ull;
    }
  };
  fetch(b);
  for (size_t base = b; base < e; base += 32) {
    const size_t i = base + lane;
    const bool valid = i < e;
    const uint32_t g = ng;
    uint64_t m[3][W];
#pragma unroll
    for (int k = 0; k < W; ++k) {  // zero for invalid lanes (their x, z are 0)
      m[0][k] = nx[k] & ~nz[k] & nisoX[k];
      m[1][k] = nx[k] & nz[k] & nisoY[k];
      m[2][k] = ~nx[k] & nz[k] & nisoZ[k];
    }
    fetch(base + 32);
    const unsigned peers = warp_peers(g);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < W; ++k) {  // OR over the lanes of the same generator
        const unsigned lo = __reduce_or_sync(peers, unsigned(m[a][k]));
        const unsigned hi = __reduce_or_sync(peers, unsigned(m[a][k] >> 32));
        m[a][k] = (uint64_t(hi) << 32) | lo;
      }
    if (peers == 0xffffffffu) {  // one generator in the whole warp
      if (g != cg) {
        flush();
        cg = g;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W; ++k) acc[a][k] |= m[a][k];
      continue;
    }
    if (valid && lane == __ffs(peers) - 1) {
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int k = 0; k < W; ++k)
          if (m[a][k]) atomicOr(&gmask[(size_t(g) * 3 + a) * W + k], m[a][k]);
    }
  }
  flush();
}

// ---------------------------------------------------------------------------
// A6: index-based accumulation for one fan-out qubit q.
//
// Strings of one generator that differ only at q form a group of at most
// three members (X, Y, Z at q, non-isolated rows).  The group key is the
// string with q cleared.  Insertion: the first member to claim the group's
// slot becomes its leader and publishes its term index; later members find it
// (bounded wait on the publish flag), compare the full key and store their
// weight in the leader's payload.  Emission: each leader writes one child per
// letter c reached by a member, with weight sum_p t[p][c] * v[p] in the fixed
// order p = X, Y, Z, so results do not depend on arrival order.

struct Slot {
  unsigned long long tag;  // epoch << 48 | 48-bit fingerprint; 0 = never used
  unsigned leader;
  unsigned ready;          // epoch of the last publish
};

// Waits until *flag == want (acquire), at most `limit` rounds of a short
// sleep; false when it gave up.  Every device-side wait of the library is one
// of these, so a missing publish ends in an error status, never a hang.
__device__ __forceinline__ bool bounded_wait_eq(const unsigned* flag, unsigned want,
                                                unsigned limit) {
  unsigned it = 0;
  while (ld_acquire(flag) != want) {
    if (++it > limit) return false;
    __nanosleep(32);
  }
  return true;
}

// Self-test of the bounded wait: warp 1 of the single block waits for a flag
// that warp 0 publishes only when `publish` is set.  err[0] = 1 when the wait
// gave up.
static __global__ void k_wait_selftest(unsigned* flag, int publish, unsigned limit,
                                       unsigned* err) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0 && lane == 0 && publish) st_release(flag, 1u);
  if (warp == 1 && lane == 0 && !bounded_wait_eq(flag, 1u, limit)) *err = 1u;
}

template <int W, typename WT = double>
__global__ void __launch_bounds__(256) k_merge_insert(
    TermsT<WT> t, const unsigned long long* n_in, int q, const __grid_constant__ FanQ fq_p,
    const uint64_t* mixed /* [G][W] */,
    Slot* table, unsigned long long tcap, unsigned epoch, uint32_t* lead, double* pv /* [3][cap] */,
    uint32_t* pmask, size_t pcap, unsigned spin_limit, unsigned* err) {
  // the table is read with per-thread letter indices: a shared copy keeps
  // those reads parallel (divergent reads of kernel parameters serialise)
  __shared__ FanQ fq;
  if (threadIdx.x == 0) fq = fq_p;
  __syncthreads();
  // after an overflow (flagged in *err) the chain of passes stops: the
  // buffer may hold unwritten entries, and the host redoes the step
  if (*(volatile const unsigned*)err) return;
  const size_t N = min(size_t(*n_in), t.cap);
  const int qk = q >> 6;
  const uint64_t qm = 1ull << (q & 63);
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
    load_term<W>(t, i, x, z);
    const int L = letter_at<W>(x, z, q);
    if (L == 0) continue;
    const int p = L - 1;
    if (fq.iso[p]) continue;
    const uint32_t g = t.g[i];
    if (!(mixed[size_t(g) * W + qk] & qm)) continue;
    const double w = t.w[i];
    x[qk] &= ~qm;
    z[qk] &= ~qm;
    const uint64_t h = key_hash<W>(g, x, z);
    const unsigned long long tag =
        (static_cast<unsigned long long>(epoch) << 48) | (h & 0xffffffffffffull);
    unsigned long long pos = __umul64hi(h, tcap);
    bool done = false;
    for (unsigned long long probe = 0; probe < tcap && !done; ++probe) {
      Slot* s = &table[pos];
      unsigned long long cur = ld_relaxed64(&s->tag);
      while (true) {
        if ((cur >> 48) != epoch) {
          const unsigned long long old = atomicCAS(&s->tag, cur, tag);
          if (old == cur) {  // claimed: this term leads the group
            s->leader = unsigned(i);
            lead[i] = unsigned(i);
            pv[size_t(p) * pcap + i] = w;
            pmask[i] = 1u << p;
            st_release(&s->ready, epoch);
            done = true;
            break;
          }
          cur = old;
          continue;
        }
        if (cur == tag) {
          if (!bounded_wait_eq(&s->ready, epoch, spin_limit)) {
            lead[i] = 0xffffffffu;  // not a leader: emits nothing
            atomicOr(err, kErrSpin);
            return;
          }
          const unsigned ld = ld_relaxed(&s->leader);
          bool same = t.g[ld] == g;
#pragma unroll
          for (int k = 0; k < W; ++k) {
            uint64_t lx = t.x[k * t.cap + ld], lz = t.z[k * t.cap + ld];
            if (k == qk) {
              lx &= ~qm;
              lz &= ~qm;
            }
            same = same && lx == x[k] && lz == z[k];
          }
          if (same) {
            lead[i] = ld;
            pv[size_t(p) * pcap + ld] = w;
            atomicOr(&pmask[ld], 1u << p);
            done = true;
          }
        }
        break;  // occupied by another key (or matched)
      }
      if (++pos == tcap) pos = 0;
    }
    if (!done) {
      lead[i] = 0xffffffffu;  // not a leader: emits nothing
      atomicOr(err, kErrProbe);
    }
  }
}

// Children of one input term at qubit q: letter (-1 = keep the input's) and
// weight of each, at most three.  Modes per term:
//   direct: I at q, an isolated row, or a generator where q needs no merge:
//           one child per non-zero entry of the row;
//   leader: one child per letter reached by any member of the group, weight
//           sum_p t[p][c] v[p] over the members in the order X, Y, Z;
//   member: nothing (its weight went to the leader).
// Children below eps are dropped here and their squared weight is added to
// pruned[g]; the returned count is what the caller writes.
template <int W>
__device__ __forceinline__ unsigned merge_children(const uint64_t* x, const uint64_t* z, double w,
                                                   uint32_t g, size_t i, int q, const FanQ& fq,
                                                   const uint64_t* mixed, const uint32_t* lead,
                                                   const double* pv, const uint32_t* pmask,
                                                   size_t pcap, double eps, double* pruned,
                                                   int* cl, double* cw) {
  const int L = letter_at<W>(x, z, q);
  unsigned n = 0;
  auto keep = [&](int c, double v) {
    if (eps > 0.0 && fabs(v) < eps) {
      atomicAdd(&pruned[g], v * v);
      return;
    }
    cl[n] = c;
    cw[n] = v;
    ++n;
  };
  if (L == 0) {
    keep(-1, w);
    return n;
  }
  const int p = L - 1;
  const bool merged = !fq.iso[p] && (mixed[size_t(g) * W + (q >> 6)] & (1ull << (q & 63)));
  if (!merged) {
    for (int j = 0; j < fq.nnz[p]; ++j) {
      const int c = fq.col[p][j];
      keep(c, w * fq.t[p][c]);
    }
    return n;
  }
  if (lead[i] != unsigned(i)) return 0;
  const uint32_t msk = pmask[i];
  double v[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) v[a] = (msk >> a) & 1 ? pv[size_t(a) * pcap + i] : 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    bool reached = false;
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (((msk >> a) & 1) && ((fq.nz >> (3 * a + c)) & 1)) {
        acc = fma(fq.t[a][c], v[a], acc);
        reached = true;
      }
    }
    if (reached) keep(c, acc);
  }
  return n;
}

template <int W, int THREADS, typename WT = double>
__global__ void __launch_bounds__(THREADS) k_merge_emit(
    TermsT<WT> in, const unsigned long long* n_in, int q, const __grid_constant__ FanQ fq_p, const uint64_t* mixed,
    const uint32_t* lead, const double* pv, const uint32_t* pmask, size_t pcap, double eps,
    double* pruned, TermsT<WT> out, unsigned long long* n_out, unsigned* err) {
  // the table is read with per-thread letter indices: a shared copy keeps
  // those reads parallel (divergent reads of kernel parameters serialise)
  __shared__ FanQ fq;
  if (threadIdx.x == 0) fq = fq_p;
  __syncthreads();
  __shared__ unsigned s_scan[THREADS / 32 + 1];
  __shared__ unsigned long long s_base;
  // after an overflow (flagged in *err) the chain of passes stops: the
  // buffer may hold unwritten entries, and the host redoes the step
  // (read once per block: the emit has block barriers)
  __shared__ unsigned s_err;
  if (threadIdx.x == 0) s_err = *(volatile const unsigned*)err;
  __syncthreads();
  if (s_err) return;
  const size_t N = min(size_t(*n_in), in.cap);
  for (size_t tile = size_t(blockIdx.x) * THREADS; tile < N; tile += size_t(gridDim.x) * THREADS) {
    const size_t i = tile + threadIdx.x;
    uint64_t x[W], z[W];
    double w = 0.0;
    uint32_t g = 0;
    int cl[3];
    double cw[3];
    unsigned c = 0;
    if (i < N) {
      load_term<W>(in, i, x, z);
      w = in.w[i];
      g = in.g[i];
      c = merge_children<W>(x, z, w, g, i, q, fq, mixed, lead, pv, pmask, pcap, eps, pruned, cl,
                            cw);
    }
    unsigned total;
    const unsigned off = block_excl_scan<THREADS>(c, &total, s_scan);
    if (threadIdx.x == 0) s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0;
    __syncthreads();
    const size_t base = size_t(s_base) + off;
    if (c) {
      if (base + c > out.cap) {
        atomicOr(err, kErrCap);
      } else {
        for (unsigned j = 0; j < c; ++j) {
          uint64_t cx[W], cz[W];
#pragma unroll
          for (int k = 0; k < W; ++k) {
            cx[k] = x[k];
            cz[k] = z[k];
          }
          if (cl[j] >= 0) set_letter<W>(cx, cz, q, cl[j]);
          store_term<W>(out, base + j, cx, cz, cw[j], g);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace dev
}  // namespace qx

#include "qx_merge_fast.cuh"
#include "qx_merge_inplace.cuh"
#include "qx_merge_blocks.cuh"

namespace qx {
namespace dev {

// ---------------------------------------------------------------------------
// A5: one-shot expansion over the fan-out qubits that need no merge in any
// generator (flatten, Eq. 3): each parent has prod_q nnz(row) children, laid
// out contiguously after an exclusive scan of the counts.

template <int W>
__device__ __forceinline__ unsigned long long child_count(const uint64_t* x, const uint64_t* z,
                                                          const FanQ* fq, int nq) {
  unsigned long long c = 1;
  for (int j = 0; j < nq; ++j) {
    const int L = letter_at<W>(x, z, fq[j].q);
    if (L) {
      c *= fq[j].nnz[L - 1];
      if (c > (1ull << 40)) c = 1ull << 40;  // saturate: far beyond any budget
    }
  }
  return c;
}

template <int W, typename WT = double>
__global__ void __launch_bounds__(256) k_expand_count(TermsT<WT> t, const unsigned long long* n_in,
                                                      const FanQ* fq_g, int nq,
                                                      unsigned long long* cnt_out) {
  extern __shared__ FanQ s_fq[];
  for (int j = threadIdx.x; j < nq; j += blockDim.x) s_fq[j] = fq_g[j];
  __syncthreads();
  const size_t N = *n_in;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
    load_term<W>(t, i, x, z);
    cnt_out[i] = child_count<W>(x, z, s_fq, nq);
  }
}

// Exclusive scan, three phases: per-tile scan, scan of tile sums, add.
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

static __global__ void __launch_bounds__(kScanThreads) k_scan_tiles(unsigned long long* a,
                                                             const unsigned long long* n_in,
                                                             unsigned long long* tile_sums) {
  __shared__ unsigned long long s[kScanThreads / 32 + 1];
  const size_t N = *n_in;
  const size_t tile = size_t(blockIdx.x) * kScanTile;
  if (tile >= N) return;
  unsigned long long v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const size_t i = tile + size_t(threadIdx.x) * kScanItems + k;
    v[k] = i < N ? a[i] : 0;
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) s[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = kScanThreads / 32;
    unsigned long long w = lane < NW ? s[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    if (lane < NW) s[lane] = w;
  }
  __syncthreads();
  unsigned long long run = (wid ? s[wid - 1] : 0) + inc - sum;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const size_t i = tile + size_t(threadIdx.x) * kScanItems + k;
    if (i < N) a[i] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = run;
}

// Counts and exclusive scan of at most kScanTile parents in one block (small
// steps, where three scan launches would be mostly launch latency): offs[i]
// and the total in *total.
template <int W, typename WT = double>
__global__ void __launch_bounds__(kScanThreads) k_expand_count_small(
    TermsT<WT> t, const unsigned long long* n_in, const FanQ* fq_g, int nq,
    unsigned long long* offs, unsigned long long* total) {
  extern __shared__ FanQ s_fq[];
  __shared__ unsigned long long s[kScanThreads / 32 + 1];
  __shared__ unsigned long long s_cnt[kScanTile];
  {  // the tables word by word over all threads
    static_assert(sizeof(FanQ) % 4 == 0, "FanQ is copied in 4-byte words");
    const uint32_t* src = reinterpret_cast<const uint32_t*>(fq_g);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_fq);
    const int nw = nq * int(sizeof(FanQ) / 4);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const size_t N = *n_in;
  // counts with one term per thread and pass (independent loads), then each
  // thread scans its kScanItems consecutive counts
  for (size_t i = threadIdx.x; i < size_t(kScanTile); i += blockDim.x) {
    unsigned long long cnt = 0;
    if (i < N) {
      uint64_t x[W], z[W];
      load_term<W>(t, i, x, z);
      cnt = child_count<W>(x, z, s_fq, nq);
    }
    s_cnt[i] = cnt;
  }
  __syncthreads();
  unsigned long long v[kScanItems];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = s_cnt[threadIdx.x * kScanItems + k];
    sum += v[k];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long inc = sum;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, d);
    if (lane >= d) inc += o;
  }
  if (lane == 31) s[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    constexpr int NW = kScanThreads / 32;
    unsigned long long w = lane < NW ? s[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= d) w += o;
    }
    if (lane < NW) s[lane] = w;
    if (lane == NW - 1) *total = w;
  }
  __syncthreads();
  unsigned long long run = (wid ? s[wid - 1] : 0) + inc - sum;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const size_t i = size_t(threadIdx.x) * kScanItems + k;
    if (i < N) offs[i] = run;
    run += v[k];
  }
}

static __global__ void __launch_bounds__(1024) k_scan_sums(unsigned long long* sums, size_t ntiles,
                                                    unsigned long long* total) {
  __shared__ unsigned long long s[33];
  unsigned long long carry = 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (size_t base = 0; base < ntiles; base += blockDim.x) {
    const size_t i = base + threadIdx.x;
    const unsigned long long v = i < ntiles ? sums[i] : 0;
    unsigned long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += o;
    }
    if (lane == 31) s[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int NW = blockDim.x / 32;
      unsigned long long w = lane < NW ? s[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xffffffffu, w, d);
        if (lane >= d) w += o;
      }
      if (lane < NW) s[lane] = w;
      if (lane == NW - 1) s[32] = w;
    }
    __syncthreads();
    if (i < ntiles) sums[i] = carry + (wid ? s[wid - 1] : 0) + inc - v;
    carry += s[32];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

static __global__ void __launch_bounds__(kScanThreads) k_scan_add(unsigned long long* a,
                                                           const unsigned long long* n_in,
                                                           const unsigned long long* tile_offs) {
  const size_t N = *n_in;
  const size_t tile = size_t(blockIdx.x) * kScanTile;
  const unsigned long long add = tile_offs[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += kScanThreads) {
    const size_t i = tile + k;
    if (i < N) a[i] += add;
  }
}

constexpr int kExpThreads = 256;
constexpr int kExpItems = 4;
constexpr int kExpTile = kExpThreads * kExpItems;
constexpr int kExpMaxH = 8;  // distinct upper digit values a tree tile may span

// The parents at the ends of every emit tile: tile_first[t] holds the child
// c = t kExpTile and tile_last[t] the tile's last child; one thread per parent
// marks the tile ends that fall in its range [offs[p], offs[p + 1]).  (A
// search of the offsets per tile would be a chain of dependent memory reads
// at the start of every tile.)
// *total_d is the output size; a launch sized for cap < *total_d (a guess that
// was too small) does nothing, as does the emit below.
static __global__ void k_expand_tiles(const unsigned long long* offs, const unsigned long long* n_in,
                                      const unsigned long long* total_d, unsigned long long cap,
                                      unsigned long long* tile_first,
                                      unsigned long long* tile_last) {
  const unsigned long long total = *total_d;
  if (total > cap) return;
  const size_t N = *n_in;
  const unsigned long long T = kExpTile;
  for (size_t p = size_t(blockIdx.x) * blockDim.x + threadIdx.x; p < N;
       p += size_t(gridDim.x) * blockDim.x) {
    const unsigned long long lo = offs[p], hi = p + 1 < N ? offs[p + 1] : total;
    if (lo >= hi) continue;
    for (unsigned long long t = lo / T; t <= (hi - 1) / T; ++t) {
      const unsigned long long first = t * T, last = min(total, first + T) - 1;
      if (first >= lo && first < hi) tile_first[t] = p;
      if (last >= lo && last < hi) tile_last[t] = p;
    }
  }
}

// Harmless terms (the identity string, generator 0, weight 0) in [from, cap)
// of an output whose size was guessed: from = *total_d where the expansion
// wrote fewer children than the guess, 0 where it wrote none (*total_d >
// cap).  A run whose guess is checked only at its end is then repeated, but
// until that check every later kernel reads in-bounds generator ids.
template <int W, typename WT = double>
__global__ void k_fill_tail(TermsT<WT> t, const unsigned long long* total_d,
                            unsigned long long cap) {
  const unsigned long long total = *total_d;
  const unsigned long long from = total > cap ? 0ull : total;
  for (unsigned long long i = from + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       i < cap; i += (unsigned long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
      t.x[k * t.cap + i] = 0ull;
      t.z[k * t.cap + i] = 0ull;
    }
    t.w[i] = WT(0);
    t.g[i] = 0u;
  }
}

// The same over a whole output of n terms when *err is set (a block-ordered
// step whose kernels did nothing).
template <int W, typename WT = double>
__global__ void k_zero_if_err(TermsT<WT> t, size_t n, const unsigned* err) {
  if (!*err) return;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
      t.x[k * t.cap + i] = 0ull;
      t.z[k * t.cap + i] = 0ull;
    }
    t.w[i] = WT(0);
    t.g[i] = 0u;
  }
}

// Dynamic shared memory of k_expand_emit: the fan-out tables, the parent
// offsets of a tile and (FP64) the product tree of a single-parent tile.
template <int W, typename WT>
constexpr size_t expand_emit_smem(int nq) {
  return size_t(nq) * sizeof(FanQ) + size_t(kExpTile) * 8 +
         (sizeof(WT) == 8 ? size_t(kExpTile) * (8 + 16 * W) : 0);
}

// Children [c0, c0 + kExpTile) per block iteration.  The parents of the tile
// are located once (binary search on the offsets), their offsets staged in
// shared memory, and each child finds its parent there; the child index within
// the parent is decoded in mixed radix over the parent's fan-out letters (the
// first wire is the least significant digit), and its weight is the parent's
// times one table entry per wire, in wire order.
//
// A tile whose children all have one parent (a large fan-out; FP64 weights)
// shares that product: the parent's wires split into a lower part (the first
// wires, at most kExpTile digit combinations) and an upper part.  The lower
// products w t_0 t_1 ... are built once per tile as a tree, one level per wire
// (each node one multiplication: the same roundings as the product in wire
// order), the upper products t_k t_k+1 ... once per distinct upper digit value
// of the tile, and each child takes one more multiplication.  This regroups the
// product as (w t_0 ... t_k-1)(t_k ... t_m-1), a reordering within rounding,
// and takes the FP64 work from one multiplication per wire and child to about
// three per child (an FP64 instruction costs about 16 SM cycles on this GPU).
template <int W, typename WT = double>
__global__ void __launch_bounds__(kExpThreads) k_expand_emit(
    TermsT<WT> in, const unsigned long long* n_in, const unsigned long long* offs,
    const unsigned long long* total_d, unsigned long long cap,
    const unsigned long long* tile_first, const unsigned long long* tile_last, const FanQ* fq_g,
    int nq, TermsT<WT> out) {
  const unsigned long long total = *total_d;
  if (total > cap) return;  // sized for a smaller guess: the caller launches again
  extern __shared__ unsigned char s_raw[];
  FanQ* s_fq = reinterpret_cast<FanQ*>(s_raw);
  unsigned long long* s_off = reinterpret_cast<unsigned long long*>(s_fq + nq);
  double* s_lw = reinterpret_cast<double*>(s_off + kExpTile);  // tree tiles only
  uint64_t* s_lx = reinterpret_cast<uint64_t*>(s_lw + kExpTile);
  uint64_t* s_lz = s_lx + size_t(kExpTile) * W;
  __shared__ size_t s_p0, s_p1;
  __shared__ uint8_t s_wj[kMaxQubits], s_wa[kMaxQubits], s_wn[kMaxQubits];
  __shared__ int s_nw, s_klo, s_nh;
  __shared__ unsigned long long s_rlo, s_h0;
  __shared__ double s_hw[kExpMaxH];
  __shared__ uint64_t s_hx[kExpMaxH][W], s_hz[kExpMaxH][W], s_hm[W];
  for (int j = threadIdx.x; j < nq; j += blockDim.x) s_fq[j] = fq_g[j];
  (void)n_in;
  for (unsigned long long c0 = (unsigned long long)blockIdx.x * kExpTile; c0 < total;
       c0 += (unsigned long long)gridDim.x * kExpTile) {
    const unsigned long long c1 = min(total, c0 + kExpTile);
    if (threadIdx.x == 0) {
      // the parents of the first and the last child of the tile
      const size_t lo = size_t(tile_first[c0 / kExpTile]);
      const size_t lo2 = size_t(tile_last[c0 / kExpTile]);
      s_p0 = lo;
      s_p1 = lo2;
      s_nh = 0;
      if constexpr (sizeof(WT) == 8) {
        if (lo2 == lo) {  // one parent: its fan-out wires in order, and the split
          uint64_t x[W], z[W];
          load_term<W>(in, lo, x, z);
          int nw = 0, klo = 0;
          unsigned long long rlo = 1;
          bool lower = true;
          for (int j = 0; j < nq; ++j) {
            const int L = letter_at<W>(x, z, s_fq[j].q);
            if (!L) continue;
            const int nn = s_fq[j].nnz[L - 1];
            if (lower && rlo * nn <= (unsigned long long)kExpTile) {
              rlo *= nn;
              klo = nw + 1;
            } else {
              lower = false;
            }
            s_wj[nw] = uint8_t(j);
            s_wa[nw] = uint8_t(L - 1);
            s_wn[nw] = uint8_t(nn);
            ++nw;
          }
          const unsigned long long r0 = c0 - offs[lo], r1 = c1 - 1 - offs[lo];
          const unsigned long long h0 = r0 / rlo, nh = r1 / rlo - h0 + 1;
          if (nh <= (unsigned long long)kExpMaxH) {
            s_nw = nw;
            s_klo = klo;
            s_rlo = rlo;
            s_h0 = h0;
            s_nh = int(nh);
          }
        }
      }
    }
    __syncthreads();
    const size_t p0 = s_p0, np = s_p1 - p0 + 1;
    if constexpr (sizeof(WT) == 8) {
      if (s_nh > 0) {
        const size_t p = p0;
        const int nw = s_nw, klo = s_klo, nh = s_nh;
        const unsigned long long rlo = s_rlo, h0 = s_h0, off = offs[p];
        // lower tree: level e multiplies every node by wire e's entries
        if (threadIdx.x == 0) {
          s_lw[0] = double(in.w[p]);
          uint64_t x[W], z[W];
          load_term<W>(in, p, x, z);
#pragma unroll
          for (int k = 0; k < W; ++k) {
            s_lx[k] = x[k];
            s_lz[k] = z[k];
          }
        }
        // upper products, one per distinct upper digit value; the mask of
        // the upper wires' qubits
        if (threadIdx.x >= 32 && threadIdx.x < 32 + unsigned(nh)) {
          const int t = threadIdx.x - 32;
          unsigned long long h = h0 + t;
          uint64_t x[W], z[W];
          load_term<W>(in, p, x, z);
          double v = 1.0;
          for (int e = klo; e < nw; ++e) {
            const FanQ& f = s_fq[s_wj[e]];
            const int a = s_wa[e], nn = s_wn[e];
            int d = 0;
            if (nn == 2) {
              d = int(h & 1);
              h >>= 1;
            } else if (nn == 3) {
              d = int(h % 3);
              h /= 3;
            }
            const int col = f.col[a][d];
            v = e == klo ? f.t[a][col] : v * f.t[a][col];
            set_letter<W>(x, z, f.q, col);
          }
          s_hw[t] = v;
#pragma unroll
          for (int k = 0; k < W; ++k) {
            s_hx[t][k] = x[k];
            s_hz[t][k] = z[k];
          }
        }
        if (threadIdx.x == 64) {
          uint64_t hm[W];
#pragma unroll
          for (int k = 0; k < W; ++k) hm[k] = 0;
          for (int e = klo; e < nw; ++e) {
            const int q = s_fq[s_wj[e]].q;
            hm[q >> 6] |= 1ull << (q & 63);
          }
#pragma unroll
          for (int k = 0; k < W; ++k) s_hm[k] = hm[k];
        }
        __syncthreads();
        unsigned long long size = 1;
        for (int e = 0; e < klo; ++e) {
          const FanQ& f = s_fq[s_wj[e]];
          const int a = s_wa[e], nn = s_wn[e];
          for (unsigned long long idx = threadIdx.x; idx < size; idx += blockDim.x) {
            const double v = s_lw[idx];
            uint64_t x[W], z[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
              x[k] = s_lx[idx * W + k];
              z[k] = s_lz[idx * W + k];
            }
            for (int d = nn - 1; d >= 0; --d) {
              const int col = f.col[a][d];
              const unsigned long long o = idx + size * d;
              s_lw[o] = v * f.t[a][col];
              uint64_t xo[W], zo[W];
#pragma unroll
              for (int k = 0; k < W; ++k) {
                xo[k] = x[k];
                zo[k] = z[k];
              }
              set_letter<W>(xo, zo, f.q, col);
#pragma unroll
              for (int k = 0; k < W; ++k) {
                s_lx[o * W + k] = xo[k];
                s_lz[o * W + k] = zo[k];
              }
            }
          }
          size *= nn;
          __syncthreads();
        }
        const uint32_t g = in.g[p];
        const bool upper = klo < nw;
        const bool pow2 = (rlo & (rlo - 1)) == 0;
        const int sh = __ffsll((long long)rlo) - 1;
        for (int k = 0; k < kExpItems; ++k) {
          const unsigned long long c = c0 + (unsigned long long)k * kExpThreads + threadIdx.x;
          if (c >= c1) break;
          const unsigned long long r = c - off;
          const unsigned long long hq = pow2 ? r >> sh : r / rlo, rho = r - hq * rlo;
          const int t = int(hq - h0);
          uint64_t x[W], z[W];
#pragma unroll
          for (int k2 = 0; k2 < W; ++k2) {
            x[k2] = (s_lx[rho * W + k2] & ~s_hm[k2]) | (s_hx[t][k2] & s_hm[k2]);
            z[k2] = (s_lz[rho * W + k2] & ~s_hm[k2]) | (s_hz[t][k2] & s_hm[k2]);
          }
          const double v = upper ? s_lw[rho] * s_hw[t] : s_lw[rho];
          store_term<W>(out, size_t(c), x, z, WT(v), g);
        }
        __syncthreads();
        continue;
      }
    }
    for (size_t j = threadIdx.x; j < np; j += blockDim.x) s_off[j] = offs[p0 + j];
    __syncthreads();
    for (int k = 0; k < kExpItems; ++k) {
      const unsigned long long c = c0 + (unsigned long long)k * kExpThreads + threadIdx.x;
      if (c >= c1) break;
      size_t lo = 0, hi = np;
      while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (s_off[mid] <= c) lo = mid; else hi = mid;
      }
      const size_t p = p0 + lo;
      unsigned long long r = c - s_off[lo];
      uint64_t x[W], z[W];
      load_term<W>(in, p, x, z);
      WProd<WT> w(in.w[p]);
      const uint32_t g = in.g[p];
      for (int j = 0; j < nq; ++j) {
        const FanQ& f = s_fq[j];
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
        w.mul(f, a, col);
        set_letter<W>(x, z, f.q, col);
      }
      store_term<W>(out, size_t(c), x, z, w.get(), g);
    }
    __syncthreads();
  }
}

// Compaction after pruning inside k_expand_emit: pruned children leave holes;
// when eps > 0 the expansion writes into a staging buffer and this kernel
// keeps the terms whose weight passes the threshold.
template <int W, int THREADS, typename WT = double>
__global__ void __launch_bounds__(THREADS) k_compact_pruned(TermsT<WT> in, const unsigned long long* n_in,
                                                            double eps, double* pruned, TermsT<WT> out,
                                                            unsigned long long* n_out) {
  const size_t n = *n_in;
  __shared__ unsigned s_scan[THREADS / 32 + 1];
  __shared__ unsigned long long s_base;
  for (size_t tile = size_t(blockIdx.x) * THREADS; tile < n; tile += size_t(gridDim.x) * THREADS) {
    const size_t i = tile + threadIdx.x;
    const double w = i < n ? double(in.w[i]) : 0.0;
    const unsigned keep = (i < n && !(fabs(w) < eps)) ? 1u : 0u;
    if (i < n && !keep) atomicAdd(&pruned[in.g[i]], w * w);
    unsigned total;
    const unsigned off = block_excl_scan<THREADS>(keep, &total, s_scan);
    if (threadIdx.x == 0) s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0;
    __syncthreads();
    if (keep) {
      uint64_t x[W], z[W];
      load_term<W>(in, i, x, z);
      store_term<W>(out, size_t(s_base) + off, x, z, in.w[i], in.g[i]);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Per-generator statistics: term count and sum of squared weights.

// Per-generator term count and sum of squared weights.  Each warp reads a
// contiguous range; while all its lanes hold one generator id each lane keeps
// its own partial sum (one fused multiply-add per term) and the warp combines
// the lanes and adds into global memory only when the id changes and at the
// end.  FP64 instructions are the scarce resource on this GPU (a warp-wide one
// takes about 16 SM cycles), so the butterfly is paid once per run of one id,
// not once per 32 terms.  Mixed warps combine equal ids first.
template <int W, typename WT = double>
__global__ void k_gen_stats(TermsT<WT> t, const unsigned long long* n_in, int G,
                            unsigned long long* count, double* sumsq) {
  (void)G;
  const size_t N = *n_in;
  const unsigned lane = threadIdx.x & 31;
  size_t b, e;
  warp_range(N, &b, &e);
  uint32_t cg = 0xffffffffu;
  unsigned long long acc_n = 0;
  double acc_sq = 0.0;  // this lane's share of generator cg
  auto flush = [&]() {
    if (cg != 0xffffffffu) {
#pragma unroll
      for (int o = 16; o; o >>= 1) acc_sq += __shfl_xor_sync(0xffffffffu, acc_sq, o);
      if (lane == 0) {
        atomicAdd(&count[cg], acc_n);
        atomicAdd(&sumsq[cg], acc_sq);
      }
    }
    acc_n = 0;
    acc_sq = 0.0;
  };
  // the next 32 terms are loaded before the current ones are combined
  uint32_t ng = 0xffffffffu;
  double nw = 0.0;
  auto fetch = [&](size_t base) {
    const size_t i = base + lane;
    const bool valid = base < e && i < e;
    ng = valid ? t.g[i] : 0xffffffffu;
    nw = valid ? double(t.w[i]) : 0.0;
  };
  fetch(b);
  for (size_t base = b; base < e; base += 32) {
    const size_t i = base + lane;
    const bool valid = i < e;
    const uint32_t g = ng;
    const double w = nw;
    fetch(base + 32);
    const unsigned peers = warp_peers(g);
    if (peers == 0xffffffffu) {  // one id in the whole warp
      if (g != cg) {
        flush();
        cg = g;
      }
      acc_n += 32;
      acc_sq = fma(w, w, acc_sq);
      continue;
    }
    double sq = 0.0;
    unsigned rest = peers;
    while (rest) {
      const int src = __ffs(rest) - 1;
      rest &= rest - 1;
      const double o = __shfl_sync(peers, w, src);
      sq = fma(o, o, sq);
    }
    if (valid && int(lane) == __ffs(peers) - 1) {
      atomicAdd(&count[g], (unsigned long long)__popc(peers));
      atomicAdd(&sumsq[g], sq);
    }
  }
  flush();
}

// ---------------------------------------------------------------------------
// A7: readout.

// Initial generators given as row-major strings (x, z: [G][W]) and weights.
template <int W, typename WT = double>
__global__ void k_init_rows(TermsT<WT> t, const uint64_t* rx, const uint64_t* rz, const double* w,
                            int G, unsigned long long* n_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < G) {
    uint64_t x[W], z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] = rx[size_t(i) * W + k];
      z[k] = rz[size_t(i) * W + k];
    }
    store_term<W>(t, i, x, z, w ? w[i] : 1.0, uint32_t(i));
  }
  if (i == 0) *n_out = (unsigned long long)G;
}

// Terms of one generator, compacted into out (planar, cap = its count).
template <int W, int THREADS, typename WT = double>
__global__ void __launch_bounds__(THREADS) k_select(TermsT<WT> in, const unsigned long long* n_in,
                                                    uint32_t gen, TermsT<WT> out,
                                                    unsigned long long* n_out) {
  __shared__ unsigned s_scan[THREADS / 32 + 1];
  __shared__ unsigned long long s_base;
  const size_t n = *n_in;
  for (size_t tile = size_t(blockIdx.x) * THREADS; tile < n; tile += size_t(gridDim.x) * THREADS) {
    const size_t i = tile + threadIdx.x;
    const unsigned keep = (i < n && in.g[i] == gen) ? 1u : 0u;
    unsigned total;
    const unsigned off = block_excl_scan<THREADS>(keep, &total, s_scan);
    if (threadIdx.x == 0) s_base = total ? atomicAdd(n_out, (unsigned long long)total) : 0;
    __syncthreads();
    if (keep && size_t(s_base) + off < out.cap) {
      uint64_t x[W], z[W];
      load_term<W>(in, i, x, z);
      store_term<W>(out, size_t(s_base) + off, x, z, in.w[i], in.g[i]);
    }
    __syncthreads();
  }
}

// All terms in device order, row-major strings.
template <int W, typename WT = double>
__global__ void k_raw(TermsT<WT> in, size_t n, uint64_t* x, uint64_t* z, double* w, int32_t* g) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[i * W + k] = in.x[k * in.cap + i];
      z[i * W + k] = in.z[k * in.cap + i];
    }
    w[i] = in.w[i];
    g[i] = int32_t(in.g[i]);
  }
}

// Lookup index over a result: open addressing on (generator, x, z).  Result
// strings are unique, so building needs no key comparison: each term claims
// the first empty slot of its probe sequence.
struct IndexSlot {
  unsigned long long tag;  // 0 = empty, else fingerprint | 1
  unsigned idx;
  unsigned pad;
};

template <int W, typename WT = double>
__global__ void k_index_build(TermsT<WT> t, size_t n, IndexSlot* tab, unsigned long long cap,
                              unsigned* err) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
    load_term<W>(t, i, x, z);
    const uint64_t h = key_hash<W>(t.g[i], x, z);
    const unsigned long long tag = h | 1ull;
    unsigned long long pos = __umul64hi(h, cap);
    bool done = false;
    for (unsigned long long probe = 0; probe < cap; ++probe) {
      if (atomicCAS(&tab[pos].tag, 0ull, tag) == 0ull) {
        tab[pos].idx = unsigned(i);
        done = true;
        break;
      }
      if (++pos == cap) pos = 0;
    }
    if (!done) atomicOr(err, kErrProbe);
  }
}

// Weight of (g, x, z) in the terms behind index tab, 0 when absent.
template <int W, typename WT>
__device__ __forceinline__ double index_find(const TermsT<WT>& t, const IndexSlot* tab,
                                             unsigned long long cap, uint32_t g, const uint64_t* x,
                                             const uint64_t* z) {
  const uint64_t h = key_hash<W>(g, x, z);
  const unsigned long long tag = h | 1ull;
  unsigned long long pos = __umul64hi(h, cap);
  for (unsigned long long probe = 0; probe < cap; ++probe) {
    const unsigned long long s = tab[pos].tag;
    if (s == 0ull) break;
    if (s == tag) {
      const unsigned j = tab[pos].idx;
      bool same = t.g[j] == g;
#pragma unroll
      for (int k = 0; k < W; ++k)
        same = same && t.x[k * t.cap + j] == x[k] && t.z[k * t.cap + j] == z[k];
      if (same) return double(t.w[j]);
    }
    if (++pos == cap) pos = 0;
  }
  return 0.0;
}

template <int W, typename WT = double>
__global__ void k_lookup(TermsT<WT> t, const IndexSlot* tab, unsigned long long cap, size_t nq,
                         const int32_t* qg, const uint64_t* qx, const uint64_t* qz, double* out) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nq;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x[k] = qx[i * W + k];
      z[k] = qz[i * W + k];
    }
    out[i] = index_find<W>(t, tab, cap, uint32_t(qg[i]), x, z);
  }
}

// sum of weights of the Z-type strings (x = 0) per generator: <0|P|0> = 1 for
// those and 0 for every string with an X or Y.
template <int W, typename WT = double>
__global__ void k_ztype_sum(TermsT<WT> t, const unsigned long long* n_in, double* out) {
  const size_t n = *n_in;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    bool ztype = true;
#pragma unroll
    for (int k = 0; k < W; ++k) ztype = ztype && t.x[k * t.cap + i] == 0;
    if (ztype) atomicAdd(&out[t.g[i]], double(t.w[i]));
  }
}

// ---- adjoint (reverse-mode) kernels ----------------------------------------

// Derivative of one rotation, in shared memory: its wire and the 3x3 matrix D
// applied to the letter the iterated side has there.
// kind 0: the letter on wire q goes through D (a rotation in a one-qubit
// operator); kind 1: a Pauli rotation about (px, pz), whose derivative map
// sends an anticommuting string Q to sigma(Q) (Q xor P), scaled by d[0][0].
struct AdjRot {
  int q;
  int kind;
  double d[3][3];
  uint64_t px[2], pz[2];
};

constexpr int kAdjMaxRot = 256;  // rotations per launch

// partial[x][r] = sum over the terms i of tile column x of the iterated side a:
//   w_i * sum_l D_r[p][l] * b_{gmap[g_i]}(string_i with letter l on wire q_r),
// p the letter of string_i on q_r (I contributes nothing).  Terms are taken in
// a grid-stride order that depends only on the grid; each warp reduces with
// shuffles in a fixed tree and each block sums its warps in order, so the
// partials are reproducible bit for bit.
template <int W, typename WT>
__global__ void __launch_bounds__(256) k_adjoint_dot(TermsT<WT> a, size_t na, const int32_t* gmap,
                                                     TermsT<WT> b, const IndexSlot* tab,
                                                     unsigned long long cap, const AdjRot* rots,
                                                     int nrot_all, int rb, double* partial) {
  extern __shared__ __align__(16) unsigned char adj_smem[];
  // blockIdx.y selects rotations [r0, r0 + nrot): several blocks share a term
  // tile when the iterated side is too small to fill the GPU on its own
  const int r0 = blockIdx.y * rb;
  const int nrot = min(rb, nrot_all - r0);
  AdjRot* s_rot = reinterpret_cast<AdjRot*>(adj_smem);
  double* s_part = reinterpret_cast<double*>(s_rot + rb);  // [warps][nrot]
  const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < nrot; i += blockDim.x) s_rot[i] = rots[r0 + i];
  for (int i = threadIdx.x; i < warps * nrot; i += blockDim.x) s_part[i] = 0.0;
  __syncthreads();
  const size_t stride = size_t(gridDim.x) * blockDim.x;
  for (size_t base = size_t(blockIdx.x) * blockDim.x; base < na; base += stride) {
    const size_t i = base + threadIdx.x;
    uint64_t x[W], z[W];
    double w = 0.0;
    int gb = -1;
    if (i < na) {
      load_term<W>(a, i, x, z);
      gb = gmap[a.g[i]];
      w = double(a.w[i]);
    }
    for (int r = 0; r < nrot; ++r) {
      double c = 0.0;
      if (gb >= 0 && s_rot[r].kind == 1) {
        const AdjRot& pr = s_rot[r];
        int par = 0, aq = 0, ap = 0, ar = 0, zx = 0;
        uint64_t xx[W], zz[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
          par += __popcll((x[k] & pr.pz[k]) ^ (z[k] & pr.px[k]));
          xx[k] = x[k] ^ pr.px[k];
          zz[k] = z[k] ^ pr.pz[k];
          aq += __popcll(x[k] & z[k]);
          ap += __popcll(pr.px[k] & pr.pz[k]);
          ar += __popcll(xx[k] & zz[k]);
          zx += __popcll(z[k] & pr.px[k]);
        }
        if (par & 1) {  // i Q P = sigma (Q xor P)
          const double sigma = ((1 + aq + ap - ar + 2 * zx) & 3) == 0 ? 1.0 : -1.0;
          c = w * pr.d[0][0] * sigma * index_find<W>(b, tab, cap, uint32_t(gb), xx, zz);
        }
      } else if (gb >= 0) {
        const int q = s_rot[r].q;
        const int L = letter_at<W>(x, z, q);
        if (L) {
          double acc = 0.0;
#pragma unroll
          for (int l = 0; l < 3; ++l) {
            const double d = s_rot[r].d[L - 1][l];
            if (d == 0.0) continue;
            uint64_t xx[W], zz[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
              xx[k] = x[k];
              zz[k] = z[k];
            }
            set_letter<W>(xx, zz, q, l);
            acc += d * index_find<W>(b, tab, cap, uint32_t(gb), xx, zz);
          }
          c = w * acc;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
      if (lane == 0) s_part[wid * nrot + r] += c;
    }
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nrot; r += blockDim.x) {
    double v = 0.0;
    for (int k = 0; k < warps; ++k) v += s_part[k * nrot + r];
    partial[size_t(blockIdx.x) * nrot_all + r0 + r] = v;
  }
}

// out[r] = sum over blocks of partial[block][r], blocks in order.
static __global__ void k_adjoint_reduce(const double* partial, int nblocks, int nrot, double* out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrot) return;
  double v = 0.0;
  for (int k = 0; k < nblocks; ++k) v += partial[size_t(k) * nrot + r];
  out[r] = v;
}

// Copies n terms between buffers of different capacity.
template <int W, typename WT>
__global__ void k_copy_terms(TermsT<WT> src, size_t n, TermsT<WT> dst, unsigned long long* n_out) {
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    uint64_t x[W], z[W];
    load_term<W>(src, i, x, z);
    store_term<W>(dst, i, x, z, src.w[i], src.g[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_out = (unsigned long long)n;
}

}  // namespace dev
}  // namespace qx

#include "qx_pauli_rot.cuh"
