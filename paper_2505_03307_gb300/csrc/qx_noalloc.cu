// qx_merge_qubit_static: the one-qubit expansion + index-accumulation step
// with its scratch in a fixed device array instead of allocated memory.
//
// The scratch (hash table, group payload, counters) is one file-scope
// __device__ array of kNaScratchBytes.  Every GPU that loads the library holds
// it until the process exits.  Host code cannot use the array's name as a
// device address, so the first call on each device (with that device current)
// looks the address up with cudaGetSymbolAddress, clears the array, and keeps
// the pointer for later calls.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "qx_common.h"
#include "qx_kernels.cuh"

using namespace qx;
using namespace qx::dev;

namespace {

constexpr size_t kNaMaxTerms = size_t(1) << 18;        // input terms per call
constexpr unsigned long long kNaSlots = 1ull << 19;    // hash slots: twice the terms
constexpr int kNaMaxGens = 4096;                       // generator ids per call
constexpr int kNaMaxDevices = 64;

// Byte layout of the scratch array.
constexpr size_t kOffTable = 0;
constexpr size_t kOffLead = kOffTable + kNaSlots * sizeof(Slot);
constexpr size_t kOffPv = kOffLead + kNaMaxTerms * 4;
constexpr size_t kOffPmask = kOffPv + 3 * kNaMaxTerms * 8;
constexpr size_t kOffMixed = kOffPmask + kNaMaxTerms * 4;
constexpr size_t kOffPruned = kOffMixed + size_t(kNaMaxGens) * kMaxWords * 8;
constexpr size_t kOffCounters = kOffPruned + size_t(kNaMaxGens) * 8;
constexpr size_t kNaScratchBytes = kOffCounters + 256;  // about 16 MiB

static __device__ __align__(256) unsigned char g_qx_noalloc_scratch[kNaScratchBytes];

struct DeviceState {
  unsigned char* ptr = nullptr;  // device address of g_qx_noalloc_scratch
  unsigned epoch = 0;
};
DeviceState g_state[kNaMaxDevices];
std::mutex g_mutex;

__global__ void k_na_set_count(unsigned long long* p, unsigned long long v) { *p = v; }

// A generator id at or beyond ngen would index the per-generator arrays of the
// scratch (mixed masks) past their region.  This pass runs before the merge
// kernels and flags such ids; the merge kernels return at once when the error
// word is set, so no term with a bad id is ever read as an index.
constexpr unsigned kErrGenId = 16u;
__global__ void k_na_check_gen(const uint32_t* gen, size_t n, uint32_t ngen, unsigned* err) {
  bool bad = false;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x)
    bad |= gen[i] >= ngen;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, kErrGenId);
}

// Once per device, with the device current: address lookup and clearing.
qx_status setup(int dev, DeviceState** out) {
  DeviceState& st = g_state[dev];
  if (!st.ptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_qx_noalloc_scratch);
    if (e != cudaSuccess)
      return fail(QX_ECUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    auto* b = static_cast<unsigned char*>(p);
    cudaError_t e1 = cudaMemset(b, 0, kNaScratchBytes);
    // every generator merges at every qubit: the mixed masks are all ones
    if (e1 == cudaSuccess)
      e1 = cudaMemset(b + kOffMixed, 0xff, size_t(kNaMaxGens) * kMaxWords * 8);
    if (e1 == cudaSuccess) e1 = cudaDeviceSynchronize();
    if (e1 != cudaSuccess)
      return fail(QX_ECUDA, std::string("clearing the static scratch failed: ") +
                                cudaGetErrorString(e1));
    st.ptr = b;
    st.epoch = 0;
  }
  *out = &st;
  return QX_OK;
}

bool fan_qubit_from_table(int q, const double* t9, FanQ* f) {
  std::memset(f, 0, sizeof *f);
  f->q = q;
  int colcount[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      const double v = t9[3 * a + c];
      if (!std::isfinite(v)) return false;
      f->t[a][c] = v;
      f->th[a][c] = float(v);
      f->tl[a][c] = float(v - double(f->th[a][c]));
      if (v != 0.0) colcount[c]++;
    }
  for (int a = 0; a < 3; ++a) {
    for (int c = 0; c < 3; ++c)
      if (f->t[a][c] != 0.0) f->col[a][f->nnz[a]++] = uint8_t(c);
    if (f->nnz[a] == 0) return false;  // a row of an image table is never zero
    f->iso[a] = (f->nnz[a] == 1 && colcount[f->col[a][0]] == 1) ? 1 : 0;
  }
  fanq_set_nz(f);
  return true;
}

template <int W>
void launch(const Terms& in, const Terms& out, int q, int ngen, const FanQ& f, unsigned char* b,
            unsigned epoch, int sms, cudaStream_t s) {
  auto* table = reinterpret_cast<Slot*>(b + kOffTable);
  auto* lead = reinterpret_cast<uint32_t*>(b + kOffLead);
  auto* pv = reinterpret_cast<double*>(b + kOffPv);
  auto* pmask = reinterpret_cast<uint32_t*>(b + kOffPmask);
  auto* mixed = reinterpret_cast<const uint64_t*>(b + kOffMixed);
  auto* pruned = reinterpret_cast<double*>(b + kOffPruned);
  auto* n_in = reinterpret_cast<unsigned long long*>(b + kOffCounters);
  auto* n_out = n_in + 1;
  auto* err = reinterpret_cast<unsigned*>(n_in + 2);
  const size_t N = in.cap;
  const unsigned grid =
      unsigned(std::max<size_t>(1, std::min<size_t>((N + 255) / 256, size_t(sms) * 8)));
  k_na_check_gen<<<grid, 256, 0, s>>>(in.g, N, uint32_t(ngen), err);
  k_merge_insert<W><<<grid, 256, 0, s>>>(in, n_in, q, f, mixed, table, kNaSlots, epoch, lead, pv,
                                         pmask, kNaMaxTerms, 1u << 25, err);
  k_merge_emit<W, 256><<<grid, 256, 0, s>>>(in, n_in, q, f, mixed, lead, pv, pmask, kNaMaxTerms,
                                            0.0, pruned, out, n_out, err);
}

}  // namespace

extern "C" qx_status qx_merge_qubit_static(int n, size_t n_in, int ngen, const uint64_t* x,
                                           const uint64_t* z, const double* w,
                                           const uint32_t* gen, int q, const double* table,
                                           uint64_t* out_x, uint64_t* out_z, double* out_w,
                                           uint32_t* out_gen, size_t out_cap, size_t* n_out,
                                           void* stream) {
  clear_error();
  if (n < 1 || n > kMaxQubits) return fail(QX_EINVAL, "n must be in 1..128");
  if (q < 0 || q >= n) return fail(QX_EINVAL, "qubit out of range");
  if (n_in > kNaMaxTerms)
    return fail(QX_EINVAL, "n_in exceeds the static scratch limit of " +
                               std::to_string(kNaMaxTerms) + " terms");
  if (ngen < 1 || ngen > kNaMaxGens)
    return fail(QX_EINVAL, "ngen must be in 1.." + std::to_string(kNaMaxGens));
  if (!table || !n_out) return fail(QX_EINVAL, "NULL argument");
  if (n_in && (!x || !z || !w || !gen)) return fail(QX_EINVAL, "NULL input array");
  if (n_in && (!out_x || !out_z || !out_w || !out_gen || out_cap == 0))
    return fail(QX_EINVAL, "NULL output array");
  FanQ f;
  if (!fan_qubit_from_table(q, table, &f)) return fail(QX_EINVAL, "invalid 3x3 table");
  if (n_in == 0) {
    *n_out = 0;
    return QX_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no usable CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState* st = nullptr;
  if (const qx_status e = setup(dev, &st)) return e;
  auto s = static_cast<cudaStream_t>(stream);
  unsigned char* b = st->ptr;
  if (++st->epoch >= 0xffffu) {  // epochs tag the table slots: clear on wrap
    if (cudaMemsetAsync(b + kOffTable, 0, kNaSlots * sizeof(Slot), s) != cudaSuccess)
      return fail(QX_ECUDA, "clearing the static hash table failed");
    st->epoch = 1;
  }
  auto* counters = reinterpret_cast<unsigned long long*>(b + kOffCounters);
  if (cudaMemsetAsync(counters, 0, 32, s) != cudaSuccess)
    return fail(QX_ECUDA, "clearing the counters failed");
  k_na_set_count<<<1, 1, 0, s>>>(counters, (unsigned long long)n_in);
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int W = (n + 63) / 64;
  const Terms in{const_cast<uint64_t*>(x), const_cast<uint64_t*>(z), const_cast<double*>(w),
                 const_cast<uint32_t*>(gen), n_in};
  const Terms out{out_x, out_z, out_w, out_gen, out_cap};
  if (W == 1)
    launch<1>(in, out, q, ngen, f, b, st->epoch, sms, s);
  else
    launch<2>(in, out, q, ngen, f, b, st->epoch, sms, s);
  cudaError_t e = cudaGetLastError();
  unsigned long long cnt[3] = {0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, counters, 24, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    return fail(QX_ECUDA, std::string("static merge failed: ") + cudaGetErrorString(e));
  const unsigned err = unsigned(cnt[2]);
  if (err & kErrGenId) return fail(QX_EINVAL, "a generator id is not below ngen");
  if (err & kErrSpin) return fail(QX_ETIMEOUT, "a device-side wait for a group leader gave up");
  if (err & kErrProbe) return fail(QX_ECAP, "the static hash table ran out of probe slots");
  if (err & kErrCap) return fail(QX_ECAP, "out_cap is smaller than the number of output terms");
  *n_out = size_t(cnt[1]);
  return QX_OK;
}
