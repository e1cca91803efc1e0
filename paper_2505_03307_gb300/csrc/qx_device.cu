// Device driver and C-ABI entry points of libqx that run on the GPU.
//
// qx_propagate walks the device program built by the planner: fused Clifford
// passes (in place) and fan-out steps (expansion with index-based
// accumulation), Algorithm 2.  Term buffers come from the caller's allocator
// or from cudaMallocAsync on the caller's stream; nothing is allocated with a
// blocking call on the hot path.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <memory>
#include <cstring>
#include <type_traits>
#include <unordered_map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "qx_common.h"
#include "qx_kernels.cuh"
#include "qx_expand_fused.cuh"
#include "qx_clifford_tiles.cuh"
#include "qx_batch.cuh"

using namespace qx;
using namespace qx::dev;

#define QX_TRY_CUDA(call)                                                             \
  do {                                                                                \
    const cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                            \
      return fail(QX_ECUDA, std::string(#call) + " failed: " + cudaGetErrorString(e_)); \
  } while (0)

#define QX_TRY(...)                       \
  do {                                    \
    const qx_status s_ = (__VA_ARGS__);   \
    if (s_ != QX_OK) return s_;           \
  } while (0)

namespace {

constexpr int kThreads = 256;

// Blocks from a caller's allocator that did not start on a 256-byte
// boundary: the aligned address handed out -> the caller's pointer.
std::mutex g_realign_mu;
std::unordered_map<void*, void*> g_realigned;

struct Alloc {
  qx_alloc_fn a = nullptr;
  qx_free_fn f = nullptr;
  void* ctx = nullptr;
  cudaStream_t s = nullptr;
  // Every block starts on a 256-byte boundary (the kernels' bulk copies and
  // 128-bit atomics need 16): cudaMallocAsync guarantees it; a caller's
  // allocator, which promises only the size, is asked for 256 bytes more and
  // the block is moved up to the next boundary.
  void* get(size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (a) {
      void* raw = a(bytes + 256, ctx, s);
      if (!raw || (reinterpret_cast<uintptr_t>(raw) & 255u) == 0) return raw;
      void* p = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(raw) + 255u) &
                                        ~uintptr_t(255));
      std::lock_guard<std::mutex> lock(g_realign_mu);
      g_realigned[p] = raw;
      return p;
    }
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p) {
    if (!p) return;
    if (f) {
      {
        std::lock_guard<std::mutex> lock(g_realign_mu);
        auto it = g_realigned.find(p);
        if (it != g_realigned.end()) {
          p = it->second;
          g_realigned.erase(it);
        }
      }
      f(p, ctx, s);
    } else {
      cudaFreeAsync(p, s);
    }
  }
};

// Term buffer of either weight type: x, z planes, weights, generator ids.
struct TermBuf {
  uint64_t* x = nullptr;
  uint64_t* z = nullptr;
  void* w = nullptr;
  uint32_t* g = nullptr;
  size_t cap = 0;
  void* base = nullptr;
  template <typename WT>
  TermsT<WT> view() const {
    return TermsT<WT>{x, z, static_cast<WT*>(w), g, cap};
  }
};

// bytes per term: x and z words, the weight (wtb = 8 or 4), the generator id
size_t term_bytes(int W, int wtb) { return size_t(16 * W + wtb + 4); }

qx_status alloc_terms(Alloc& al, int W, int wtb, size_t cap, TermBuf* out) {
  // a multiple of 4: every plane then starts on a 16-byte boundary, and bulk
  // copies rounded up to 16 bytes stay inside their plane
  cap = (std::max<size_t>(cap, 1) + 3) & ~size_t(3);
  const size_t bytes = cap * term_bytes(W, wtb) + 64;
  void* base = al.get(bytes);
  if (!base) return fail(QX_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  auto* x = static_cast<uint64_t*>(base);
  out->base = base;
  out->x = x;
  out->z = x + size_t(W) * cap;
  auto* wp = reinterpret_cast<unsigned char*>(x + 2 * size_t(W) * cap);
  out->w = wp;
  out->g = reinterpret_cast<uint32_t*>(wp + size_t(wtb) * cap);
  out->cap = cap;
  return QX_OK;
}

int device_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

unsigned grid_for(size_t n, int per_block, int sms, int blocks_per_sm) {
  const size_t need = (n + per_block - 1) / per_block;
  return unsigned(std::max<size_t>(1, std::min<size_t>(need, size_t(sms) * blocks_per_sm)));
}

void set_pool_threshold() {
  static thread_local int done_dev = -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  if (done_dev == dev) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done_dev = dev;
}

}  // namespace

// What the last run of a fan-out step of this plan did, as the guess the next
// run launches on before the per-generator letter masks come back: an
// expansion over every fan-out qubit (with its output size), or block-ordered
// merges over every fan-out qubit (with the block count).  The masks (for an
// expansion) and the device results decide whether the guess held; a wrong
// guess costs only the discarded launches.  Plans may be shared between
// threads, so the fields are atomics (a torn guess is just a wrong one).
enum : int { kHintNone = 0, kHintExpand = 1, kHintBlocks = 2, kHintReplay = 3 };
struct FanHint {
  std::atomic<int> kind{kHintNone};
  std::atomic<unsigned long long> total{0};
  std::atomic<unsigned> nblk{0};  // blocks of the last block-ordered run (table size)
  std::atomic<unsigned> streak{0};  // runs in a row that kept the guess
  // A small step's range offsets from a run whose guess held (device memory
  // of the plan, written once and published at the end of that run), one
  // record per precision: a later run with the same input count, partition
  // and threshold launches the emission on them without counting, and the
  // emission checks every range against them.  One failed check retires the
  // record.
  struct Record {
    std::atomic<unsigned long long*> offs{nullptr};
    std::atomic<int> claim{0};  // a run is recording
    std::atomic<int> bad{0};
    size_t n = 0, ranges = 0, per = 0;
    unsigned long long total = 0;
    double eps = 0.0;
  };
  Record rec[2];  // [FP32]
};

// Device copy of the plan: Clifford passes (gate lists or chunk tables) and
// the fan-out tables, uploaded once per plan and device.

struct qx_plan_device {
  int device = -1;
  void* base = nullptr;
  std::unique_ptr<FanHint[]> hints;  // one per fan-out step
  struct Pass {
    const uint32_t* ops = nullptr;
    int nops = 0;
    const uint64_t* tab_xz = nullptr;
    const uint8_t* tab_e = nullptr;
    int chunks = 0, cb = 0;
    bool use_table = false, identity = true;
    size_t smem = 0;
    uint64_t live = 0;                 // chunks with a qubit some gate touches
    uint64_t idle[qx::kMaxWords] = {};  // qubits of the other chunks
    uint64_t hot = 0;     // chunks with a qubit where one generator's terms can differ
    uint64_t recent = 0;  // those of the last fan-out step or rotation (they differ most often)
  };
  // the plan's passes, then its aux_passes (index passes.size() + k)
  std::vector<Pass> passes;
  size_t max_smem = 0;
};

namespace {

// Merge tables of the one-word fast path, kept for the life of the process
// and shared by all plans: every pass leaves its table empty, so a table is
// initialised only when it is created, grown, or after an aborted pass.  A
// propagation holds one table exclusively (concurrent propagations on other
// streams get other tables).
struct FastTable {
  int device = -1;
  FastSlot* tab = nullptr;
  double* v2 = nullptr;  // rank-2 weights, indexed like tab
  unsigned long long cap = 0;
  bool dirty = true;
  bool busy = false;
};
std::mutex g_table_mutex;
std::vector<FastTable*> g_tables;

FastTable* acquire_table(int device) {
  std::lock_guard<std::mutex> lock(g_table_mutex);
  for (FastTable* t : g_tables)
    if (!t->busy && t->device == device) {
      t->busy = true;
      return t;
    }
  auto* t = new (std::nothrow) FastTable;
  if (!t) return nullptr;
  t->device = device;
  t->busy = true;
  g_tables.push_back(t);
  return t;
}

void release_table(FastTable* t) {
  if (!t) return;
  std::lock_guard<std::mutex> lock(g_table_mutex);
  t->busy = false;
}

}  // namespace

namespace qx {

void free_plan_device(qx_plan* p) {
  if (!p || !p->dev) return;
  if (p->dev->hints)
    for (size_t i = 0; i < std::max<size_t>(1, p->fans.size()); ++i)
      for (FanHint::Record& rc : p->dev->hints[i].rec)
        if (unsigned long long* r = rc.offs.load()) cudaFree(r);
  if (p->dev->base) cudaFree(p->dev->base);
  delete p->dev;
  p->dev = nullptr;
}

}  // namespace qx

namespace {

// Chunks of a table-form pass that some gate touches (live) and the qubits
// no gate touches (idle: their letters pass through).
void pass_geometry(const CliffPass& pc, int n, uint64_t* live, uint64_t* idle) {
  *live = 0;
  for (int k = 0; k < kMaxWords; ++k) idle[k] = 0;
  for (int ch = 0; ch < pc.chunks; ++ch) {
    bool any = false;
    for (int b2 = 0; b2 < pc.chunk_bits; ++b2) {
      const int q = ch * pc.chunk_bits + b2;
      if (q >= n) continue;
      if ((pc.support[q >> 6] >> (q & 63)) & 1)
        any = true;
      else
        idle[q >> 6] |= 1ull << (q & 63);
    }
    if (any) *live |= 1ull << ch;
  }
}

// Per Clifford pass of the program, the qubits where two terms of one
// generator can carry different letters when the pass runs (all), and among
// them those of the last fan-out step or rotation before it (recent: the
// children of one parent sit next to each other, so these letters change
// from one term to the next, the older ones less often): the wires of the
// fan-out steps and the supports of the rotations, carried through the
// passes between (a pass maps a qubit's letters into the supports of the
// images of X_q and Z_q).  Generators start as single terms.
struct Variation {
  std::array<uint64_t, kMaxWords> all{}, recent{};
};

std::vector<Variation> variation_masks(const qx_plan* p) {
  std::vector<Variation> out(p->passes.size());
  Variation v;
  const int n = p->n, W = p->W;
  auto carry = [&](const CliffPass& pc, const std::array<uint64_t, kMaxWords>& m) {
    std::array<uint64_t, kMaxWords> nm{};
    for (int q = 0; q < n; ++q) {
      if (!((m[q >> 6] >> (q & 63)) & 1)) continue;
      for (const int row : {q, n + q})
        for (int k = 0; k < W; ++k)
          nm[k] |= pc.img_x[size_t(row) * W + k] | pc.img_z[size_t(row) * W + k];
    }
    return nm;
  };
  for (const Step& st : p->program) {
    if (st.kind == kStepFan) {
      v.recent = {};
      for (const FanQubit& f : p->fans[size_t(st.index)].qs)
        v.recent[f.q >> 6] |= 1ull << (f.q & 63);
      for (int k = 0; k < W; ++k) v.all[k] |= v.recent[k];
    } else if (st.kind == kStepRot) {
      const RotStep& r = p->rots[size_t(st.index)];
      for (int k = 0; k < W; ++k) {
        v.recent[k] = r.px[k] | r.pz[k];
        v.all[k] |= v.recent[k];
      }
    } else if (st.kind == kStepCliff) {
      const CliffPass& pc = p->passes[size_t(st.index)];
      out[size_t(st.index)] = v;
      if (pc.identity || pc.img_x.empty()) continue;
      v.all = carry(pc, v.all);
      v.recent = carry(pc, v.recent);
    }
  }
  return out;
}

qx_status ensure_plan_device(const qx_plan* cp, int device) {
  auto* p = const_cast<qx_plan*>(cp);
  if (p->dev && p->dev->device == device) return QX_OK;
  free_plan_device(p);
  auto* d = new (std::nothrow) qx_plan_device;
  if (!d) return fail(QX_ENOMEM, "host allocation failed");
  d->device = device;
  // one contiguous upload: [ops of every pass][tables of every pass]
  std::vector<const CliffPass*> all;
  for (const CliffPass& pc : p->passes) all.push_back(&pc);
  for (const CliffPass& pc : p->aux_passes) all.push_back(&pc);
  std::vector<size_t> off_ops(all.size()), off_tab(all.size()), off_e(all.size());
  size_t bytes = 0;
  auto align = [](size_t v) { return (v + 255) & ~size_t(255); };
  for (size_t i = 0; i < all.size(); ++i) {
    const CliffPass& pc = *all[i];
    off_ops[i] = bytes;
    bytes = align(bytes + pc.ops.size() * 4);
    off_tab[i] = bytes;
    bytes = align(bytes + pc.tab_xz.size() * 8);
    off_e[i] = bytes;
    bytes = align(bytes + pc.tab_e.size());
  }
  std::vector<unsigned char> host(std::max<size_t>(bytes, 1));
  for (size_t i = 0; i < all.size(); ++i) {
    const CliffPass& pc = *all[i];
    if (!pc.ops.empty()) std::memcpy(&host[off_ops[i]], pc.ops.data(), pc.ops.size() * 4);
    if (!pc.tab_xz.empty()) std::memcpy(&host[off_tab[i]], pc.tab_xz.data(), pc.tab_xz.size() * 8);
    if (!pc.tab_e.empty()) std::memcpy(&host[off_e[i]], pc.tab_e.data(), pc.tab_e.size());
  }
  void* base = nullptr;
  if (cudaMalloc(&base, host.size()) != cudaSuccess) {
    cudaGetLastError();
    delete d;
    return fail(QX_ENOMEM, "device allocation for the plan tables failed");
  }
  if (cudaMemcpy(base, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(base);
    delete d;
    return fail(QX_ECUDA, "upload of the plan tables failed");
  }
  d->base = base;
  auto* b = static_cast<unsigned char*>(base);
  const auto varq = variation_masks(p);
  for (size_t i = 0; i < all.size(); ++i) {
    const CliffPass& pc = *all[i];
    qx_plan_device::Pass dp;
    dp.ops = reinterpret_cast<const uint32_t*>(b + off_ops[i]);
    dp.nops = int(pc.ops.size());
    dp.tab_xz = reinterpret_cast<const uint64_t*>(b + off_tab[i]);
    dp.tab_e = b + off_e[i];
    dp.chunks = pc.chunks;
    dp.cb = pc.chunk_bits;
    dp.use_table = pc.use_table;
    dp.identity = pc.identity;
    dp.smem = pc.use_table ? pc.tab_xz.size() * 8 + pc.tab_e.size() : pc.ops.size() * 4;
    if (pc.use_table) {
      pass_geometry(pc, p->n, &dp.live, dp.idle);
      if (i < varq.size())
        for (int ch = 0; ch < pc.chunks; ++ch)
          for (int b2 = 0; b2 < pc.chunk_bits; ++b2) {
            const int q = ch * pc.chunk_bits + b2;
            if (q >= p->n) continue;
            if ((varq[i].all[q >> 6] >> (q & 63)) & 1) dp.hot |= 1ull << ch;
            if ((varq[i].recent[q >> 6] >> (q & 63)) & 1) dp.recent |= 1ull << ch;
          }
    }
    d->max_smem = std::max(d->max_smem, dp.smem);
    d->passes.push_back(dp);
  }
  d->hints.reset(new (std::nothrow) FanHint[std::max<size_t>(1, p->fans.size())]);
  if (!d->hints) {
    cudaFree(base);
    delete d;
    return fail(QX_ENOMEM, "host allocation failed");
  }
  p->dev = d;
  return QX_OK;
}

FanQ to_dev(const FanQubit& f) {
  FanQ d{};
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) {
      d.t[a][c] = f.t.r[a][c];
      d.th[a][c] = float(d.t[a][c]);
      d.tl[a][c] = float(d.t[a][c] - double(d.th[a][c]));
    }
  d.q = f.q;
  for (int a = 0; a < 3; ++a) {
    d.nnz[a] = f.nnz[a];
    for (int c = 0; c < 3; ++c) d.col[a][c] = f.col[a][c];
    d.iso[a] = f.iso[a] ? 1 : 0;
  }
  fanq_set_nz(&d);
  return d;
}

RotQ to_dev(const RotStep& r) {
  RotQ d{};
  for (int k = 0; k < kMaxWords; ++k) {
    d.px[k] = r.px[k];
    d.pz[k] = r.pz[k];
  }
  // rank bit: the lowest bit of P's support (x plane if P has X or Y there)
  for (int k = 0; k < kMaxWords; ++k) {
    const uint64_t sup = r.px[k] | r.pz[k];
    if (!sup) continue;
    d.rword = k;
    d.rbit = __builtin_ctzll(sup);
    d.rx = ((r.px[k] >> d.rbit) & 1) ? 1 : 0;
    break;
  }
  const double t[3][3] = {{r.c, r.s, 0.0}, {r.s, r.c, 0.0}, {0.0, 0.0, 0.0}};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      d.tab.t[a][b] = t[a][b];
      d.tab.th[a][b] = float(t[a][b]);
      d.tab.tl[a][b] = float(t[a][b] - double(d.tab.th[a][b]));
    }
  fanq_set_nz(&d.tab);
  return d;
}

// Scratch of one propagation (freed at the end, stream-ordered).
struct Scratch {
  unsigned long long* ncnt = nullptr;  // [0], [1]: term counts; [2]: scan total
  unsigned* err = nullptr;
  unsigned* serr = nullptr;  // kErrSpin of a bulk copy that never completed (read at the end)
  unsigned long long* gmask = nullptr;  // [G][3][W]
  uint64_t* mixed = nullptr;            // [G][W]
  double* pruned = nullptr;             // [G]
  unsigned long long* gcount = nullptr;  // [G] final terms per generator
  double* gsumsq = nullptr;              // [G] their sum of squared weights
  FanQ* fanq = nullptr;                 // [n]
  void* base = nullptr;
  // hash table and leader payload (grow on demand)
  Slot* table = nullptr;
  unsigned long long tcap = 0;
  unsigned epoch = 0;
  void* payload = nullptr;
  uint32_t* lead = nullptr;
  double* pv = nullptr;
  uint32_t* pmask = nullptr;
  size_t pcap = 0;
  bool payload_fast = false;
};

}  // namespace

// Kernel classes of qx_prop_stats.kc_*.
enum KernelClass {
  KC_INIT = 0, KC_CLIFF, KC_MASK, KC_INSERT, KC_EMIT, KC_COUNT, KC_SCAN, KC_EXPAND, KC_COMPACT,
  KC_STATS, KC_INDEX, KC_INPLACE, KC_ROT, KC_BLOCK_SETUP, KC_BLOCK
};
const char* const kKernelClassNames[QX_KC_COUNT] = {
    "init", "clifford_pass", "fan_mask", "merge_insert", "merge_emit", "expand_count",
    "expand_scan", "expand_emit", "prune_compact", "gen_stats", "inplace_index",
    "merge_inplace", "pauli_rot", "block_setup", "merge_blocks"};

// Optional CUDA-event timing of every launch, resolved after the final sync.
struct Timer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::vector<cudaEvent_t>* pool = nullptr;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> rec;  // class, index of the start event
  cudaEvent_t get() {
    if (used == pool->size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool->push_back(e);
    }
    return (*pool)[used++];
  }
  void begin(int k) {
    if (!on) return;
    const size_t i = used;
    cudaEvent_t e = get();
    if (!e) return;
    cudaEventRecord(e, s);
    rec.push_back({k, i});
  }
  void end() {
    if (!on) return;
    cudaEvent_t e = get();
    if (e) cudaEventRecord(e, s);
  }
  void resolve(qx_prop_stats* st) {
    for (const auto& [k, i] : rec) {
      float ms = 0.f;
      if (i + 1 < used && cudaEventElapsedTime(&ms, (*pool)[i], (*pool)[i + 1]) == cudaSuccess)
        st->kc_ms[k] += ms;
    }
  }
};

thread_local std::vector<cudaEvent_t> t_event_pool;

// Pinned host staging for the small host-to-device copies of a call.  A copy
// from pageable memory may first wait for the stream to drain, which leaves
// the GPU idle while the host issues the next launches; from pinned memory it
// is queued like a launch.  One buffer per host thread (like the event pool);
// a call's bump offset goes back to 0 whenever it synchronises its stream, at
// which point its earlier copies are complete.
constexpr size_t kStageBytes = size_t(256) << 10;
struct StageBuf {
  unsigned char* p = nullptr;
  bool tried = false;
  ~StageBuf() {
    if (p) cudaFreeHost(p);
  }
};
thread_local StageBuf t_stage;
// Pinned host memory for the read-backs a run checks only at its end (the
// letter masks, output sizes and error words of steps launched on the plan's
// record), one per host thread.
constexpr size_t kReadbackBytes = size_t(1) << 20;
thread_local StageBuf t_readback;

struct qx_result {
  int n = 0, W = 1, G = 0;
  int wtb = 8;  // bytes per weight: 8 (FP64) or 4 (FP32)
  size_t N = 0;
  TermBuf buf;
  Alloc al;
  int device = 0;
  std::vector<unsigned long long> count;
  std::vector<double> sumsq, pruned;
  qx_prop_stats st{};

  IndexSlot* index = nullptr;
  unsigned long long icap = 0;
};
namespace qx {
void result_set_stream(qx_result* r, void* stream) {
  if (r) r->al.s = static_cast<cudaStream_t>(stream);
}
}  // namespace qx


namespace {

struct Ctx {
  const qx_plan* p = nullptr;
  int n = 0, W = 1, G = 0;
  int wtb = 8;  // bytes per weight: 8 (FP64) or 4 (FP32)
  int sms = 1;
  double eps = 0.0;
  size_t budget = 0, max_terms = 0;
  unsigned spin_limit = 1u << 22;
  Alloc al;
  Scratch sc;
  qx_prop_stats st{};
  TermBuf cur;
  size_t N = 0;
  int cslot = 0;  // which of ncnt[0], ncnt[1] holds cur's count
  Timer tm;
  FastTable* ftab = nullptr;  // pooled merge table of the fast path (held for the call)
  bool inplace = true;        // merge wires may run in place (QX_FLAG_NO_INPLACE clears it)
  size_t stage_off = 0;       // bytes of t_stage queued since the last stream sync
  // Steps launched on the plan's record whose check waits for the end of the
  // run (no host round trip of their own); a failed check repeats the run with
  // every step checked at once (defer = false).
  struct Deferred {
    int kind = 0;  // kHintExpand, kHintBlocks or kHintReplay
    FanHint* hint = nullptr;
    const FanStep* fs = nullptr;
    unsigned long long expect = 0;    // the recorded output size (expansion)
    const unsigned long long* gm = nullptr;  // pinned: the step's letter masks
    const unsigned long long* total = nullptr;
    const unsigned* err = nullptr;
    const unsigned* nblk = nullptr;
    const uint32_t* gwire = nullptr;  // letter codes (replayed offsets)
    FanHint::Record* rec = nullptr;   // the record it replayed
    int slot = -1;                    // its check slot (err, gwire: set once read back)
  };
  bool defer = false;
  bool retry = false;  // set by a run whose deferred checks failed
  // the current step is the program's last expansion or merge: a fused
  // expansion then writes the per-generator statistics (stats_done)
  bool stats_last = false;
  bool stats_done = false;
  std::vector<Deferred> deferred;
  // check slots of steps launched on recorded offsets (XsCheck), in the
  // scratch right after the per-generator statistics
  unsigned char* chk_dev = nullptr;
  size_t chk_stride = 0;
  int chk_slots = 0, chk_used = 0;
  // range offsets recorded by this run, published when it completes
  struct Record {
    FanHint::Record* rec = nullptr;
    unsigned long long* offs = nullptr;
    size_t n = 0, ranges = 0, per = 0;
    unsigned long long total = 0;
  };
  std::vector<Record> records;
  size_t rb_off = 0;
  Ctx() = default;
  Ctx(const Ctx&) = delete;
  Ctx& operator=(const Ctx&) = delete;
  ~Ctx() {
    if (stage_off) cudaStreamSynchronize(al.s);  // the staging buffer is reused next
  }
  void begin(int k) { tm.begin(k); }
  // after a launch: class, launches it made, algorithmic bytes
  void end(int k, int launches, uint64_t bytes) {
    tm.end();
    end_bytes_only(k, launches, bytes);
  }
  void end_bytes_only(int k, int launches, uint64_t bytes) {
    st.kernel_launches += launches;
    st.kc_launches[k] += launches;
    st.kc_bytes[k] += bytes;
  }
};

qx_status sync_read(Ctx& c, void* host, const void* dev, size_t bytes) {
  QX_TRY_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaStreamSynchronize(c.al.s));
  c.stage_off = 0;
  c.st.host_syncs++;
  return QX_OK;
}

// Pinned space for a read-back checked at the end of the run, or nullptr.
void* rb_take(Ctx& c, size_t bytes) {
  if (!t_readback.tried) {
    t_readback.tried = true;
    if (cudaMallocHost(reinterpret_cast<void**>(&t_readback.p), kReadbackBytes) != cudaSuccess) {
      cudaGetLastError();
      t_readback.p = nullptr;
    }
  }
  const size_t need = (bytes + 63) & ~size_t(63);
  if (!t_readback.p || c.rb_off + need > kReadbackBytes) return nullptr;
  void* r = t_readback.p + c.rb_off;
  c.rb_off += need;
  return r;
}

// Two device-to-host reads and one synchronisation.
qx_status sync_read2(Ctx& c, void* h1, const void* d1, size_t b1, void* h2, const void* d2,
                     size_t b2) {
  QX_TRY_CUDA(cudaMemcpyAsync(h1, d1, b1, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaMemcpyAsync(h2, d2, b2, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaStreamSynchronize(c.al.s));
  c.stage_off = 0;
  c.st.host_syncs++;
  return QX_OK;
}

bool limits_ok(const Ctx& c, size_t terms) {
  return !(c.max_terms && terms > c.max_terms) &&
         !(c.budget && terms * term_bytes(c.W, c.wtb) > c.budget);
}

// Host-to-device copy of a small host array, through t_stage when it has room.
qx_status h2d(Ctx& c, void* dev, const void* host, size_t bytes) {
  if (!bytes) return QX_OK;
  if (!t_stage.tried) {
    t_stage.tried = true;
    if (cudaMallocHost(reinterpret_cast<void**>(&t_stage.p), kStageBytes) != cudaSuccess) {
      cudaGetLastError();
      t_stage.p = nullptr;
    }
  }
  const size_t need = (bytes + 63) & ~size_t(63);
  if (t_stage.p && c.stage_off + need <= kStageBytes) {
    unsigned char* st = t_stage.p + c.stage_off;
    std::memcpy(st, host, bytes);
    c.stage_off += need;
    QX_TRY_CUDA(cudaMemcpyAsync(dev, st, bytes, cudaMemcpyHostToDevice, c.al.s));
    return QX_OK;
  }
  QX_TRY_CUDA(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, c.al.s));
  return QX_OK;
}

qx_status check_err(Ctx& c) {
  unsigned e = 0;
  QX_TRY(sync_read(c, &e, c.sc.err, sizeof e));
  if (e & kErrSpin) return fail(QX_ETIMEOUT, "a device-side wait for a group leader gave up");
  if (e & kErrProbe) return fail(QX_ECAP, "a hash table ran out of probe slots");
  if (e & kErrCap) return fail(QX_ECUDA, "internal error: an output buffer was too small");
  return QX_OK;
}

qx_status check_limits(Ctx& c, size_t terms) {
  if (c.max_terms && terms > c.max_terms)
    return fail(QX_ECAP, "term count " + std::to_string(terms) + " exceeds max_terms");
  if (c.budget && terms * term_bytes(c.W, c.wtb) > c.budget)
    return fail(QX_EBUDGET, "term storage of " + std::to_string(terms * term_bytes(c.W, c.wtb)) +
                                " bytes exceeds hbm_budget");
  return QX_OK;
}

void replace_cur(Ctx& c, TermBuf nb, size_t n, int slot) {
  c.al.put(c.cur.base);
  c.cur = nb;
  c.N = n;
  c.cslot = slot;
  c.st.peak_terms = std::max<uint64_t>(c.st.peak_terms, n);
}

// Qubit masks of a table-form pass for clifford_table_map: the idle qubits
// and, per part of the chunk range, the qubits of its live chunks.
template <int W>
PassMasks pass_masks(const qx_plan_device::Pass& dp, int n) {
  PassMasks pmk{};
  for (int k = 0; k < kMaxWords; ++k) pmk.idle[k] = dp.idle[k];
  const int P = clifford_parts<W>();
  // own parts, first to last: the live chunks of the last fan-out step's
  // wires (they change between neighbouring terms), the other chunks where
  // one generator's terms can differ, then the rest (cached along a
  // generator), split in order over the parts left; without that knowledge
  // (everything can differ, or nothing) the live chunks in order over all
  // parts
  const uint64_t recent = dp.live & dp.recent & dp.hot;
  const uint64_t old = dp.live & dp.hot & ~recent, cold = dp.live & ~dp.hot;
  int first = 0;
  uint64_t rest_mask = dp.live;
  if (dp.hot & dp.live && cold) {
    if (recent && old && P > 2) {
      pmk.pchunks[first++] = recent;
      pmk.pchunks[first++] = old;
    } else {
      pmk.pchunks[first++] = recent | old;
    }
    rest_mask = cold;
  }
  std::vector<int> rest;
  for (int ch = 0; ch < dp.chunks; ++ch)
    if ((rest_mask >> ch) & 1) rest.push_back(ch);
  const int np = P - first;
  for (int pp = 0; pp < np; ++pp)
    for (size_t r = size_t(pp) * rest.size() / np; r < size_t(pp + 1) * rest.size() / np; ++r)
      pmk.pchunks[first + pp] |= 1ull << rest[r];
  for (int pp = 0; pp < P; ++pp)
    for (int ch = 0; ch < dp.chunks; ++ch) {
      if (!((pmk.pchunks[pp] >> ch) & 1)) continue;
      for (int b2 = 0; b2 < dp.cb; ++b2) {
        const int q = ch * dp.cb + b2;
        if (q < n && !((dp.idle[q >> 6] >> (q & 63)) & 1)) pmk.part[pp][q >> 6] |= 1ull << (q & 63);
      }
    }
  for (int k = 0; k < kMaxWords; ++k)
    for (int pp = 1; pp < P; ++pp) pmk.rest[k] |= pmk.part[pp][k];
  return pmk;
}

// Blocks of k_clifford_table<W, CB, WT> resident per SM with `smem` bytes
// of tables (registers and shared memory both count): the pass runs as one
// wave of them, each warp on one contiguous range.
template <int W, int CB, typename WT>
int clifford_table_per_sm(size_t smem) {
  static thread_local size_t last_smem = ~size_t(0);
  static thread_local int last_n = 0;
  if (smem == last_smem && last_n) return last_n;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_clifford_table<W, CB, WT>, kThreads,
                                                    smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  last_smem = smem;
  last_n = n;
  return n;
}

// Whether a kernel may stage tiles of t with bulk copies: every plane
// starts on a 16-byte boundary and t.cap is a multiple of 4 (a copy rounded
// up to 16 bytes then stays inside its plane).  alloc_terms and Alloc make
// both true of every term buffer.
template <typename WT>
bool xs_bulk_ok(const TermsT<WT>& t, int W) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  if (t.cap % 4) return false;
  for (int k = 0; k < W; ++k)
    if (!a16(t.x + size_t(k) * t.cap) || !a16(t.z + size_t(k) * t.cap)) return false;
  return a16(t.w) && a16(t.g);
}

// The launch error of an emission, with its configuration.
// The dynamic shared memory limit of a kernel is process-wide (per device),
// so it is only ever raised, under one lock for all kernels.
void allow_dyn_smem(const void* kernel, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> allowed[64];
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  size_t& a = allowed[dev & 63][kernel];
  if (smem <= a) return;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) ==
      cudaSuccess)
    a = smem;
  else
    cudaGetLastError();  // the launch reports it
}

// A large table-form pass in tiles staged by bulk copies (k_clifford_tiles),
// one wave of blocks each on a contiguous run of tiles.
template <int W, int CB, typename WT>
qx_status run_pass_tiles(Ctx& c, const qx_plan_device::Pass& dp, const PassMasks& pmk) {
  const size_t smem = ct_smem_bytes<W, WT>(dp.smem);
  const void* kern = reinterpret_cast<const void*>(k_clifford_tiles<W, CB, WT>);
  allow_dyn_smem(kern, smem);
  static thread_local size_t last_smem = ~size_t(0);
  static thread_local int per_sm = 0;
  if (smem != last_smem || !per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_clifford_tiles<W, CB, WT>,
                                                      kXsThreads, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    last_smem = smem;
  }
  const size_t ntiles = (c.N + kCtTile - 1) / kCtTile;
  const size_t blocks = std::min<size_t>(ntiles, size_t(c.sms) * size_t(per_sm));
  const size_t per = (ntiles + blocks - 1) / blocks;
  k_clifford_tiles<W, CB, WT><<<unsigned(blocks), kXsThreads, smem, c.al.s>>>(
      c.cur.view<WT>(), c.sc.ncnt + c.cslot, dp.tab_xz, dp.tab_e, dp.chunks, dp.live, pmk, per,
      std::max(64u, c.spin_limit / 32), c.sc.serr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(QX_ECUDA, std::string("tiled Clifford pass launch failed: ") +
                              cudaGetErrorString(e) + " (dynamic shared memory " +
                              std::to_string(smem) + ")");
  return QX_OK;
}

// Passes over at least this many terms run in tiles staged by bulk copies.
constexpr size_t kTiledPassMin = size_t(1) << 16;

template <int W, typename WT>
qx_status run_pass(Ctx& c, const qx_plan_device::Pass& dp) {
  if (dp.identity || c.N == 0) return QX_OK;
  const unsigned long long* n_in = c.sc.ncnt + c.cslot;
  c.begin(KC_CLIFF);
  if (dp.use_table && c.N >= kTiledPassMin && xs_bulk_ok(c.cur.view<WT>(), W)) {
    const PassMasks pmk = pass_masks<W>(dp, c.n);
    if (dp.cb == 4)
      QX_TRY((run_pass_tiles<W, 4, WT>(c, dp, pmk)));
    else
      QX_TRY((run_pass_tiles<W, 3, WT>(c, dp, pmk)));
  } else if (dp.use_table) {
    const PassMasks pmk = pass_masks<W>(dp, c.n);
    if (dp.cb == 4) {
      const unsigned grid =
          grid_for(c.N, kThreads, c.sms, clifford_table_per_sm<W, 4, WT>(dp.smem));
      k_clifford_table<W, 4, WT><<<grid, kThreads, dp.smem, c.al.s>>>(
          c.cur.view<WT>(), n_in, dp.tab_xz, dp.tab_e, dp.chunks, dp.live, pmk);
    } else {
      const unsigned grid =
          grid_for(c.N, kThreads, c.sms, clifford_table_per_sm<W, 3, WT>(dp.smem));
      k_clifford_table<W, 3, WT><<<grid, kThreads, dp.smem, c.al.s>>>(
          c.cur.view<WT>(), n_in, dp.tab_xz, dp.tab_e, dp.chunks, dp.live, pmk);
    }
  } else {
    const unsigned grid = grid_for(c.N, kThreads, c.sms, 8);
    k_clifford_ops<W, WT><<<grid, kThreads, dp.smem, c.al.s>>>(c.cur.view<WT>(), n_in, dp.ops, dp.nops);
  }
  c.end(KC_CLIFF, 1, 2ull * c.N * (16 * W + sizeof(WT)));
  QX_TRY_CUDA(cudaGetLastError());
  c.st.clifford_passes++;
  c.st.alg_bytes += 2ull * c.N * (16 * W + sizeof(WT));
  return QX_OK;
}

template <int W, typename WT>
qx_status ensure_hash(Ctx& c, size_t n) {
  Scratch& s = c.sc;
  const unsigned long long want = std::max<unsigned long long>(64, 2ull * n);
  if (s.tcap < want) {
    c.al.put(s.table);
    s.table = static_cast<Slot*>(c.al.get(want * sizeof(Slot)));
    if (!s.table) return fail(QX_ENOMEM, "device allocation of the merge table failed");
    QX_TRY_CUDA(cudaMemsetAsync(s.table, 0, want * sizeof(Slot), c.al.s));
    s.tcap = want;
    s.epoch = 0;
  }
  if (++s.epoch >= 0xffffu) {
    QX_TRY_CUDA(cudaMemsetAsync(s.table, 0, s.tcap * sizeof(Slot), c.al.s));
    s.epoch = 1;
  }
  if (s.pcap < n) {
    c.al.put(s.payload);
    const size_t cap = std::max<size_t>(n, 64);
    s.payload = c.al.get(cap * (4 + 24 + 4));
    if (!s.payload) return fail(QX_ENOMEM, "device allocation of the merge payload failed");
    s.pv = static_cast<double*>(s.payload);
    s.lead = reinterpret_cast<uint32_t*>(s.pv + 3 * cap);
    s.pmask = s.lead + cap;
    s.pcap = cap;
  }
  return QX_OK;
}

// The one-word fast path needs the generator id to fit in the free high bits
// of the two key words.
bool fast_eligible(int n, int W, int G) {
  if (W != 1 || n >= 64) return false;
  int bits = 0;
  while ((1ll << bits) < G) ++bits;
  return bits <= 2 * (64 - n);
}

qx_status ensure_fast_table(Ctx& c, unsigned long long want) {
  if (!c.ftab) {
    int dev = 0;
    cudaGetDevice(&dev);
    c.ftab = acquire_table(dev);
    if (!c.ftab) return fail(QX_ENOMEM, "host allocation failed");
  }
  FastTable* d = c.ftab;
  if (d->cap < want) {
    if (d->tab) {
      cudaStreamSynchronize(c.al.s);
      cudaFree(d->tab);
      d->tab = nullptr;
      d->cap = 0;
    }
    void* t = nullptr;
    if (cudaMalloc(&t, want * (sizeof(FastSlot) + sizeof(double))) != cudaSuccess) {
      cudaGetLastError();
      return fail(QX_ENOMEM, "device allocation of the merge table failed");
    }
    d->tab = static_cast<FastSlot*>(t);
    d->v2 = reinterpret_cast<double*>(d->tab + want);
    d->cap = want;
    d->dirty = true;
  }
  if (d->dirty) {
    k_fast_table_init<<<grid_for(d->cap, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(d->tab, d->v2,
                                                                                   d->cap);
    QX_TRY_CUDA(cudaGetLastError());
    d->dirty = false;
  }
  return QX_OK;
}

// Insert + emit of one merge pass at fan-out qubit f.q: reads cur (count in
// ncnt[cslot]), writes `out` (count in ncnt[oslot], reset here).  No sync.
template <int W, typename WT>
qx_status launch_merge(Ctx& c, const FanQ& f, bool fast, unsigned grid, const TermBuf& out,
                       int oslot, double eps) {
  Scratch& s = c.sc;
  QX_TRY_CUDA(cudaMemsetAsync(s.ncnt + oslot, 0, 8, c.al.s));
  if (fast) {
    // insert + children of unmerged terms, then one thread per active slot;
    // the table counts as dirty until a sync has shown the pass completed
    FastTable* d = c.ftab;
    d->dirty = true;
    c.begin(KC_INSERT);
    k_merge_insert_fast<kThreads, WT><<<grid, kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), s.ncnt + c.cslot, c.n, f.q, f, s.mixed, d->tab, d->v2, d->cap, eps, s.pruned,
        out.view<WT>(), s.ncnt + oslot, s.err);
    c.tm.end();
    c.begin(KC_EMIT);
    const unsigned ggrid = grid_for(2 * std::max<size_t>(c.cur.cap, 512), kThreads, c.sms, 8);
    k_merge_groups_fast<kThreads, WT><<<ggrid, kThreads, 0, c.al.s>>>(
        s.ncnt + c.cslot, c.cur.cap, c.n, f.q, f, d->tab, d->v2, d->cap, eps, s.pruned,
        out.view<WT>(), s.ncnt + oslot, s.err);
    c.tm.end();
  } else {
    c.begin(KC_INSERT);
    k_merge_insert<W, WT><<<grid, kThreads, 0, c.al.s>>>(c.cur.view<WT>(), s.ncnt + c.cslot, f.q, f, s.mixed,
                                                     s.table, s.tcap, s.epoch, s.lead, s.pv,
                                                     s.pmask, s.pcap, c.spin_limit, s.err);
    c.tm.end();
    c.begin(KC_EMIT);
    k_merge_emit<W, kThreads, WT><<<grid, kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), s.ncnt + c.cslot, f.q, f, s.mixed, s.lead, s.pv, s.pmask, s.pcap, eps,
        s.pruned, out.view<WT>(), s.ncnt + oslot, s.err);
    c.tm.end();
  }
  QX_TRY_CUDA(cudaGetLastError());
  c.st.merge_passes++;
  return QX_OK;
}

// Makes the slow path's table and the leader array hold `n` terms.
template <int W, typename WT>
qx_status ensure_merge_scratch(Ctx& c, bool fast, size_t n) {
  if (fast) {
    QX_TRY(ensure_fast_table(c, std::max<unsigned long long>(1024, n + n / 4 + 1)));
    Scratch& s = c.sc;
    if (s.pcap < n) {
      c.al.put(s.payload);
      const size_t cap = std::max<size_t>(n, 64);
      s.payload = c.al.get(cap * 4);
      if (!s.payload) return fail(QX_ENOMEM, "device allocation of the merge payload failed");
      s.lead = static_cast<uint32_t*>(s.payload);
      s.pv = nullptr;
      s.pmask = nullptr;
      s.pcap = cap;
      s.payload_fast = true;
    }
    return QX_OK;
  }
  if (c.sc.payload_fast) {  // switch layouts
    c.al.put(c.sc.payload);
    c.sc.payload = nullptr;
    c.sc.pcap = 0;
    c.sc.payload_fast = false;
  }
  return ensure_hash<W, WT>(c, n);
}

// Merge passes over the mixed qubits.  First without host syncs inside a
// capacity arena (counts stay on the device); if an output or the table
// overflows, the passes are redone one by one with exact counts.
// Drops |w| < eps from the current terms (the last kernel of a U_k).
template <int W, typename WT>
qx_status prune_cur(Ctx& c) {
  Scratch& s = c.sc;
  TermBuf kept;
  QX_TRY(alloc_terms(c.al, W, c.wtb, c.N, &kept));
  const int kslot = 1 - c.cslot;
  QX_TRY_CUDA(cudaMemsetAsync(s.ncnt + kslot, 0, 8, c.al.s));
  c.begin(KC_COMPACT);
  k_compact_pruned<W, kThreads, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
      c.cur.view<WT>(), s.ncnt + c.cslot, c.eps, s.pruned, kept.view<WT>(), s.ncnt + kslot);
  c.tm.end();
  QX_TRY_CUDA(cudaGetLastError());
  unsigned long long nk = 0;
  QX_TRY(sync_read(c, &nk, s.ncnt + kslot, 8));
  c.end_bytes_only(KC_COMPACT, 1, (c.N + nk) * (16 * W + sizeof(WT)));
  replace_cur(c, kept, nk, kslot);
  return QX_OK;
}

// Letter permutation of an in-place merge wire: each isolated row keeps its
// only column, the other letters take the remaining columns (themselves where
// possible).  Packed 2 bits per source letter (X, Y, Z).
int inplace_pi(const FanQubit& f) {
  int pi[3] = {-1, -1, -1};
  bool used[3] = {false, false, false};
  for (int p = 0; p < 3; ++p)
    if (f.iso[p]) {
      pi[p] = f.col[p][0];
      used[pi[p]] = true;
    }
  for (int p = 0; p < 3; ++p)
    if (pi[p] < 0 && !used[p]) {
      pi[p] = p;
      used[p] = true;
    }
  for (int p = 0; p < 3; ++p)
    if (pi[p] < 0)
      for (int c = 0; c < 3; ++c)
        if (!used[c]) {
          pi[p] = c;
          used[c] = true;
          break;
        }
  return pi[0] | (pi[1] << 2) | (pi[2] << 4);
}

// Coefficients of a radix-2 merge wire for k_block_wire2; false when the wire
// has another number of non-isolated letters.
bool wire2_of(const FanQubit& f, int pi, Wire2* out) {
  int lt[2], n = 0, iso = -1;
  for (int a = 0; a < 3; ++a) {
    if (f.iso[a])
      iso = a;
    else if (n < 2)
      lt[n++] = a;
    else
      return false;
  }
  if (n != 2) return false;
  Wire2 w{};
  // letter code L of table letter a: X 1, Y 2, Z 3
  w.rk = 0;
  for (int d = 0; d < 2; ++d) w.rk |= uint32_t(d) << (2 * (lt[d] + 1));
  // the FP32 split exactly as to_dev builds FanQ::th / tl
  auto split = [](double t, float* h, float* l) {
    *h = float(t);
    *l = float(t - double(*h));
  };
  if (iso >= 0) {
    w.rk |= 3u << (2 * (iso + 1));
    w.iso_t = f.t.r[iso][(pi >> (2 * iso)) & 3];
    split(w.iso_t, &w.iso_h, &w.iso_l);
  }
  for (int d = 0; d < 2; ++d) {
    const int col = (pi >> (2 * lt[d])) & 3;
    for (int r = 0; r < 2; ++r) {
      w.c[d][r] = f.t.r[lt[r]][col];
      split(w.c[d][r], &w.ch[d][r], &w.cl[d][r]);
      if (w.c[d][r] != 0.0) w.nz |= 1u << (2 * d + r);
    }
  }
  *out = w;
  return true;
}

// Whether block keys fit one 128-bit word pair: one-word strings with room for
// the generator id in the free bits.
bool blocks_fit(const Ctx& c) {
  if (c.W != 1 || c.n >= 64) return false;
  const int fb = 64 - c.n;
  return !(2 * fb < 40 && (unsigned long long)c.G >= (1ull << (2 * fb)));
}

// Whether the merge wires of a step may run in place: one-word keys with a
// free empty pattern and, per generator, letter sets that are closed under
// each wire's table up to its letter permutation (a necessary condition for
// closed groups; the kernel checks every group).
bool inplace_candidate(const Ctx& c, const std::vector<const FanQubit*>& mq,
                       const std::vector<unsigned long long>& gm) {
  if (!blocks_fit(c)) return false;
  for (const FanQubit* f : mq) {
    const int pi = inplace_pi(*f);
    int inv[3];
    for (int p = 0; p < 3; ++p) inv[(pi >> (2 * p)) & 3] = p;
    const uint64_t qb = 1ull << f->q;
    for (int g = 0; g < c.G; ++g) {
      bool has[3];
      for (int a = 0; a < 3; ++a) has[a] = (gm[size_t(g) * 3 + a] & qb) != 0;
      for (int a = 0; a < 3; ++a) {
        if (!has[a]) continue;
        const int ca = (pi >> (2 * a)) & 3;
        bool reached = false;
        for (int col = 0; col < 3; ++col)
          if (f->t.r[a][col] != 0.0 && !has[inv[col]]) return false;
        for (int b = 0; b < 3; ++b)
          if (has[b] && f->t.r[b][ca] != 0.0) reached = true;
        if (!reached) return false;
      }
    }
  }
  return true;
}

// The merge wires of a step in place (see qx_merge_inplace.cuh).  *done is
// false when some group turned out not to be closed; the terms are then
// unchanged and the caller runs the general merge.
template <int W, typename WT>
qx_status run_merges_inplace(Ctx& c, const std::vector<const FanQubit*>& mq, bool more_after,
                             bool* done) {
  *done = false;
  const size_t N = c.N;
  const unsigned long long cap = std::max<unsigned long long>(1024, 2ull * N);
  const size_t tab_bytes = size_t(cap) * sizeof(KeySlot);
  void* mem = c.al.get(tab_bytes + 2 * N * sizeof(WT) + 512);
  if (!mem) return QX_OK;  // no room for the index: the general merge needs none
  auto* tab = static_cast<KeySlot*>(mem);
  WT* wb[2] = {reinterpret_cast<WT*>(static_cast<unsigned char*>(mem) + tab_bytes),
               reinterpret_cast<WT*>(static_cast<unsigned char*>(mem) + tab_bytes + 256) + N};
  auto body = [&]() -> qx_status {
    QX_TRY_CUDA(cudaMemsetAsync(tab, 0xff, tab_bytes, c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
    const unsigned grid = grid_for(N, kThreads, c.sms, 8);
    const auto view = c.cur.view<WT>();
    c.begin(KC_INDEX);
    k_keyindex_build<WT><<<grid, kThreads, 0, c.al.s>>>(view, N, c.n, tab, cap, c.sc.err);
    c.end(KC_INDEX, 1, uint64_t(N) * 20);
    const WT* src = view.w;
    std::vector<uint32_t> relabel;  // letter permutations, applied after every wire
    for (size_t j = 0; j < mq.size(); ++j) {
      WT* dst = wb[j & 1];
      const int pi = inplace_pi(*mq[j]);
      if (pi != (0 | (1 << 2) | (2 << 4))) {
        uint32_t code = 0;
        for (int p = 0; p < 3; ++p) code |= uint32_t((pi >> (2 * p)) & 3) << (3 * p);
        relabel.push_back(encode_op(kOpPerm, mq[j]->q, -1, code));
      }
      c.begin(KC_INPLACE);
      k_merge_inplace<WT><<<grid, kThreads, 0, c.al.s>>>(view, N, c.n, to_dev(*mq[j]), pi, src,
                                                          dst, tab, cap, c.sc.err);
      c.end(KC_INPLACE, 1, 2ull * N * (16 * W + sizeof(WT)));
      src = dst;
    }
    QX_TRY_CUDA(cudaGetLastError());
    unsigned err = 0;
    QX_TRY(sync_read(c, &err, c.sc.err, 4));
    if (err) {
      QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
      return QX_OK;
    }
    QX_TRY_CUDA(cudaMemcpyAsync(view.w, src, N * sizeof(WT), cudaMemcpyDeviceToDevice, c.al.s));
    if (!relabel.empty()) {  // the letters the in-place weights belong to
      auto* d_ops = reinterpret_cast<uint32_t*>(tab);  // the index is no longer needed
      QX_TRY(h2d(c, d_ops, relabel.data(), relabel.size() * 4));
      c.begin(KC_CLIFF);
      k_clifford_ops<W, WT><<<grid, kThreads, relabel.size() * 4, c.al.s>>>(
          view, c.sc.ncnt + c.cslot, d_ops, int(relabel.size()));
      c.end(KC_CLIFF, 1, 2ull * N * 16 * W);
      QX_TRY_CUDA(cudaGetLastError());
    }
    *done = true;
    return QX_OK;
  };
  const qx_status st = body();
  c.al.put(mem);
  if (st != QX_OK || !*done) return st;
  c.st.merge_passes += mq.size();
  c.st.inplace_steps++;
  c.st.alg_bytes += mq.size() * 2ull * N * (16 * W + sizeof(WT));
  c.st.children += mq.size() * N;
  if (!more_after && c.eps > 0.0) QX_TRY(prune_cur<W, WT>(c));
  return QX_OK;
}

// The merge wires of a step in place, with the terms in block order (see
// qx_merge_blocks.cuh), in two halves: launch_blocks queues every kernel with
// no host round trip (kernels after the block table check the error word and
// do nothing when some block is incomplete); finish_blocks, given the error
// word read back, keeps the block-ordered terms or releases them (the terms
// in c.cur are then unchanged).
struct BlocksPending {
  void* mem = nullptr;
  TermBuf out;
  size_t N = 0, m = 0;
  const unsigned* nblk = nullptr;  // device: the number of blocks claimed
  bool launched = false;  // false: the step does not fit the block code
};

template <int W, typename WT>
qx_status launch_blocks(Ctx& c, const std::vector<const FanQubit*>& mq, BlocksPending* bp,
                        unsigned nblk_guess = 0) {
  bp->launched = false;
  const int m = int(mq.size());
  if (m > kMaxBlockWires || m == 0) return QX_OK;
  BlockWires hb{};
  hb.m = m;
  for (int j = 0; j < m; ++j) {
    hb.q[j] = mq[j]->q;
    int r = 0;
    hb.canon[j] = 255;
    for (int a = 0; a < 3; ++a) {
      if (mq[j]->iso[a]) {
        hb.rank[j][a] = 255;
        continue;
      }
      if (hb.canon[j] == 255) hb.canon[j] = uint8_t(a);
      hb.rank[j][a] = uint8_t(r++);
    }
    hb.radix[j] = uint8_t(r);
    if (r < 2) return QX_OK;
    // packed form: rank by xz code c = x | z << 1 (letters X 1, Z 2, Y 3)
    const int q = mq[j]->q;
    const uint64_t qb = 1ull << q;
    uint32_t inf = uint32_t(q) | (uint32_t(r) << 24) | (15u << 8);  // c = 0: I
    const int letter_of_code[4] = {-1, 0, 2, 1};  // c -> table letter (0 X, 1 Y, 2 Z)
    for (int cc = 1; cc < 4; ++cc) {
      const int a = letter_of_code[cc];
      inf |= uint32_t(hb.rank[j][a] == 255 ? 15 : hb.rank[j][a]) << (8 + 4 * cc);
    }
    hb.inf[j] = inf;
    if (!mq[j]->iso[0]) hb.niso_x |= qb;
    if (!mq[j]->iso[1]) hb.niso_y |= qb;
    if (!mq[j]->iso[2]) hb.niso_z |= qb;
    if (hb.canon[j] <= 1) hb.canon_x |= qb;  // X or Y
    if (hb.canon[j] >= 1) hb.canon_z |= qb;  // Y or Z
    (r == 2 ? hb.rad2 : hb.rad3) |= qb;
    hb.qmask |= qb;
    if (r == 2) {  // the rank-1 letter
      for (int a = 0; a < 3; ++a)
        if (hb.rank[j][a] == 1) (a == 0 ? hb.r1x : a == 1 ? hb.r1y : hb.r1z) |= qb;
    }
    hb.pi[j] = uint8_t(inplace_pi(*mq[j]));
    if (hb.pi[j] != (0 | (1 << 2) | (2 << 4))) {
      hb.relab |= 1u << j;
      hb.rq |= qb;
      for (int a = 0; a < 3; ++a) {  // source letter a -> image letter pi(a)
        const int im = (hb.pi[j] >> (2 * a)) & 3;
        if (im <= 1) hb.tx[a] |= qb;
        if (im >= 1) hb.tz[a] |= qb;
      }
    }
  }
  {  // whole-word layout when every wire has radix 2 and the qubits increase
    bool inc = true;
    for (int j = 1; j < m; ++j) inc = inc && hb.q[j] > hb.q[j - 1];
    hb.lay_fast = (m <= kFastStrideWires && hb.rad3 == 0 && inc) ? 1 : 0;
    for (int b = 0; b < 8; ++b)
      if ((hb.qmask >> (8 * b)) & 0xffull) hb.bytes[hb.nbytes++] = uint8_t(b);
  }
  const size_t N = c.N;
  // The block table holds every block at load <= 1/2: 2N slots covers N
  // blocks of one.  With the block count of the plan's last run, 4x that
  // count; more blocks than that exhaust the probes, which fails the step
  // like an incomplete block, and the caller repeats it at full size.
  const unsigned long long bcap =
      nblk_guess ? std::min<unsigned long long>(std::max<unsigned long long>(1024, 4ull * nblk_guess),
                                                std::max<unsigned long long>(1024, 2ull * N))
                 : std::max<unsigned long long>(1024, 2ull * N);
  const size_t ntiles = (bcap + kScanTile - 1) / kScanTile;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += up(bytes);
    return o;
  };
  const size_t o_tab = take(bcap * 16), o_cnt = take(bcap * 4), o_exp = take(bcap * 4),
               o_off = take((bcap + ntiles + 1) * 8), o_n = take(32),
               o_list = take((kBlockListMax + 1) * 4), o_slot = take(N * 4),
               o_code2 = take(N * 8),
               o_w = take(N * sizeof(WT)), o_bw = take(sizeof(BlockWires));
  void* mem = c.al.get(off);
  if (!mem) return QX_OK;
  auto* b8 = static_cast<unsigned char*>(mem);
  auto* btab = reinterpret_cast<ulonglong2*>(b8 + o_tab);
  auto* bcnt = reinterpret_cast<unsigned*>(b8 + o_cnt);
  auto* bexp = reinterpret_cast<unsigned*>(b8 + o_exp);
  auto* boff = reinterpret_cast<unsigned long long*>(b8 + o_off);
  auto* dn = reinterpret_cast<unsigned long long*>(b8 + o_n);  // [0] sweep count, [1] scan total
  auto* nblk = reinterpret_cast<unsigned*>(b8 + o_list);     // claimed blocks
  unsigned* blist = nblk + 1;                                // their slots (the first 1024)
  auto* bslot = reinterpret_cast<unsigned*>(b8 + o_slot);
  auto* lcode2 = reinterpret_cast<unsigned long long*>(b8 + o_code2);
  auto* wtmp = reinterpret_cast<WT*>(b8 + o_w);
  auto* d_bw = reinterpret_cast<BlockWires*>(b8 + o_bw);
  TermBuf out;
  auto body = [&]() -> qx_status {
    const unsigned grid = grid_for(N, kThreads, c.sms, 8);
    const auto view = c.cur.view<WT>();
    QX_TRY_CUDA(cudaMemsetAsync(btab, 0xff, bcap * 16, c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(bcnt, 0, bcap * 4, c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(nblk, 0, 4, c.al.s));
    QX_TRY(h2d(c, d_bw, &hb, sizeof hb));
    c.begin(KC_BLOCK_SETUP);
    const unsigned long long plimit = nblk_guess ? std::min<unsigned long long>(bcap, 256) : bcap;
    k_block_claim<WT><<<grid, kThreads, 0, c.al.s>>>(view, N, c.n, d_bw, btab, bcap, plimit, bcnt,
                                                      bexp, bslot, nblk, blist, c.sc.err);
    // offsets: from the list of blocks when it is short, else (dn[0] = bcap)
    // from the sweep of the table and its scan, which otherwise do nothing
    // With a guessed table of at most 4 x 256 blocks the list always
    // suffices unless the guess was wrong (which fails the step): no sweep.
    const bool sweep = !(nblk_guess && nblk_guess <= kBlockListMax / 4);
    k_block_list<<<1, kBlockListMax, 0, c.al.s>>>(nblk, blist, bcnt, bexp, bcap, boff, dn,
                                                  c.sc.err, sweep ? 1 : 0);
    if (sweep) {
      k_block_sizes<<<grid_for(bcap, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(btab, dn, bcnt,
                                                                               bexp, boff, c.sc.err);
      k_scan_tiles<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(boff, dn, boff + bcap);
      k_scan_sums<<<1, 1024, 0, c.al.s>>>(boff + bcap, ntiles, dn + 1);
      k_scan_add<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(boff, dn, boff + bcap);
    }
    QX_TRY_CUDA(cudaGetLastError());
    // No host round trip here: every block is complete exactly when the error
    // word stayed 0 (then the sizes add up to N), and the kernels below do
    // nothing otherwise.  The word is read once, after the last wire.
    QX_TRY(alloc_terms(c.al, W, c.wtb, N, &out));
    const auto ov = out.view<WT>();
    k_block_scatter<WT><<<grid, kThreads, 0, c.al.s>>>(view, N, d_bw, bslot, boff, ov, lcode2,
                                                        ov.w, c.sc.err);
    c.end(KC_BLOCK_SETUP, sweep ? 7 : 3, uint64_t(N) * (2 * (16 * W + 4 + sizeof(WT)) + 24));
    const WT* src = ov.w;
    for (int j = 0; j < m; ++j) {
      WT* dst = (j & 1) ? ov.w : wtmp;
      c.begin(KC_BLOCK);
      Wire2 w2;
      if (m <= kFastStrideWires && wire2_of(*mq[j], hb.pi[j], &w2))
        k_block_wire2<WT><<<grid, kThreads, 0, c.al.s>>>(N, j, w2, lcode2, src, dst, c.sc.err);
      else
        k_block_wire<WT><<<grid, kThreads, 0, c.al.s>>>(N, d_bw, j, to_dev(*mq[j]), hb.pi[j],
                                                         lcode2, src, dst, c.sc.err);
      c.end(KC_BLOCK, 1, 2ull * N * (16 * W + sizeof(WT)));
      src = dst;
    }
    if (src != ov.w)
      QX_TRY_CUDA(cudaMemcpyAsync(ov.w, src, N * sizeof(WT), cudaMemcpyDeviceToDevice, c.al.s));
    QX_TRY_CUDA(cudaGetLastError());
    return QX_OK;
  };
  const qx_status st = body();
  if (st != QX_OK) {
    c.al.put(mem);
    c.al.put(out.base);
    return st;
  }
  bp->mem = mem;
  bp->out = out;
  bp->N = N;
  bp->m = size_t(m);
  bp->nblk = nblk;
  bp->launched = true;
  return QX_OK;
}

template <int W, typename WT>
qx_status finish_blocks(Ctx& c, BlocksPending* bp, unsigned err, bool accept, bool more_after,
                        bool* done) {
  *done = false;
  c.al.put(bp->mem);
  bp->mem = nullptr;
  if (err) QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
  if (err || !accept) {
    c.al.put(bp->out.base);
    bp->out = TermBuf();
    return QX_OK;
  }
  const size_t N = bp->N;
  replace_cur(c, bp->out, N, c.cslot);
  bp->out = TermBuf();
  *done = true;
  c.st.merge_passes += bp->m;
  c.st.inplace_steps++;
  c.st.block_steps++;
  c.st.alg_bytes += bp->m * 2ull * N * (16 * W + sizeof(WT));
  c.st.children += bp->m * N;
  if (!more_after && c.eps > 0.0) QX_TRY(prune_cur<W, WT>(c));
  return QX_OK;
}

template <int W, typename WT>
qx_status run_merges_blocks(Ctx& c, const std::vector<const FanQubit*>& mq, bool more_after,
                            bool* done, FanHint* hint) {
  *done = false;
  BlocksPending bp;
  QX_TRY((launch_blocks<W, WT>(c, mq, &bp)));
  if (!bp.launched) return QX_OK;
  unsigned err = 0, nb = 0;
  if (const qx_status st = sync_read2(c, &err, c.sc.err, 4, &nb, bp.nblk, 4)) {
    c.al.put(bp.mem);
    c.al.put(bp.out.base);
    return st;
  }
  if (hint && !err) hint->nblk.store(nb, std::memory_order_relaxed);
  return finish_blocks<W, WT>(c, &bp, err, true, more_after, done);
}

template <int W, typename WT>
qx_status run_merges(Ctx& c, const std::vector<const FanQubit*>& mq, bool more_after,
                     const std::vector<unsigned long long>& gm, FanHint* hint) {
  if (c.inplace && inplace_candidate(c, mq, gm)) {
    bool done = false;
    QX_TRY(run_merges_blocks<W, WT>(c, mq, more_after, &done, hint));
    if (done) return QX_OK;
    QX_TRY(run_merges_inplace<W, WT>(c, mq, more_after, &done));
    if (done) return QX_OK;
    c.st.inplace_fallbacks++;
  }
  const bool fast = fast_eligible(c.n, W, c.G);
  const size_t N0 = c.N;
  const int slot0 = c.cslot;
  // arena: the growth bound of the passes (product of the largest row
  // fan-out of each qubit), clamped to [3, 8] x the input, at least 64K terms
  double growth = 1.0;
  for (const FanQubit* f : mq) growth *= std::max({f->nnz[0], f->nnz[1], f->nnz[2]});
  size_t cap = size_t(std::min(8.0, std::max(3.0, growth)) * double(N0));
  cap = std::max<size_t>(cap, 65536);
  if (c.budget) cap = std::min(cap, std::max(N0, c.budget / term_bytes(W, c.wtb)));
  if (c.max_terms) cap = std::min(cap, std::max(N0, c.max_terms));
  bool ok = false;
  // pruning inside these passes accumulates pruned mass that a redo would
  // count twice: with eps > 0 the passes run in exact mode directly
  const bool optimistic = !(c.eps > 0.0 && !more_after);
  if (optimistic) {
    TermBuf buf[2];
    qx_status st = alloc_terms(c.al, W, c.wtb, cap, &buf[0]);
    if (st == QX_OK) st = alloc_terms(c.al, W, c.wtb, cap, &buf[1]);
    // the fast table is sized for 3x growth: a larger pass fills it, fails its
    // probes and is redone exactly
    if (st == QX_OK) st = ensure_merge_scratch<W, WT>(c, fast, fast ? std::min(cap, 3 * N0) : cap);
    if (st != QX_OK) {
      c.al.put(buf[0].base);
      c.al.put(buf[1].base);
      return st;
    }
    const unsigned grid = grid_for(cap, kThreads, c.sms, 8);
    TermBuf input = c.cur;
    int b = 0;
    for (size_t j = 0; j < mq.size(); ++j) {
      const bool last = !more_after && j + 1 == mq.size();
      const FanQ f = to_dev(*mq[j]);
      if (!fast) {
        if (++c.sc.epoch >= 0xffffu) {
          QX_TRY_CUDA(cudaMemsetAsync(c.sc.table, 0, c.sc.tcap * sizeof(Slot), c.al.s));
          c.sc.epoch = 1;
        }
      }
      const int oslot = 1 - c.cslot;
      QX_TRY(launch_merge<W, WT>(c, f, fast, grid, buf[b], oslot, last ? c.eps : 0.0));
      c.cur = buf[b];
      c.cslot = oslot;
      b ^= 1;
    }
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    QX_TRY(sync_read(c, h, c.sc.ncnt, 40));
    const unsigned long long nout = h[c.cslot];
    const unsigned err = unsigned(h[4]);
    if (err & kErrSpin) return fail(QX_ETIMEOUT, "a device-side wait for a group leader gave up");
    ok = !(err & (kErrProbe | kErrCap));
    if (ok) {
      if (fast) c.ftab->dirty = false;
      // counts of every pass are not kept on the host in this mode: account
      // the passes with the final count
      c.st.alg_bytes += mq.size() * (N0 + nout) * (16 * W + sizeof(WT));
      c.st.children += mq.size() * nout;
      c.st.kc_bytes[KC_INSERT] += mq.size() * N0 * (16 * W + sizeof(WT));
      c.st.kc_bytes[KC_EMIT] += mq.size() * (N0 + nout) * (16 * W + sizeof(WT));
      c.st.kc_launches[KC_INSERT] += mq.size();
      c.st.kc_launches[KC_EMIT] += mq.size();
      c.st.kernel_launches += 2 * mq.size();
      const TermBuf keep = c.cur;
      c.al.put(buf[b].base);  // the unused buffer of the pair
      c.cur = input;
      replace_cur(c, keep, nout, c.cslot);
      if (const qx_status e = check_limits(c, nout)) return e;
      return QX_OK;
    }
    // overflow: start over from the step's input
    if (fast) c.ftab->dirty = true;
    c.al.put(buf[0].base);
    c.al.put(buf[1].base);
    c.cur = input;
    c.cslot = slot0;
    c.N = N0;
    // the passes above overwrote both count slots: restore the input's count
    const unsigned long long n0 = N0;
    QX_TRY(h2d(c, c.sc.ncnt + slot0, &n0, 8));
    QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
    QX_TRY_CUDA(cudaStreamSynchronize(c.al.s));
    c.st.host_syncs++;
  }
  // exact mode: one pass at a time, counts read after each
  for (size_t j = 0; j < mq.size(); ++j) {
    const bool last = !more_after && j + 1 == mq.size();
    const FanQ f = to_dev(*mq[j]);
    QX_TRY(ensure_merge_scratch<W, WT>(c, fast, c.N));
    if (!fast && ++c.sc.epoch >= 0xffffu) {
      QX_TRY_CUDA(cudaMemsetAsync(c.sc.table, 0, c.sc.tcap * sizeof(Slot), c.al.s));
      c.sc.epoch = 1;
    }
    // at most 3 children per term; with a budget, no more than it allows (a
    // pass that needs more stops with QX_EBUDGET)
    size_t ocap = 3 * c.N;
    const bool capped = c.budget && ocap * term_bytes(W, c.wtb) > c.budget;
    if (capped) ocap = std::max<size_t>(1, c.budget / term_bytes(W, c.wtb));
    TermBuf out;
    QX_TRY(alloc_terms(c.al, W, c.wtb, ocap, &out));
    const int oslot = 1 - c.cslot;
    QX_TRY(launch_merge<W, WT>(c, f, fast, grid_for(c.N, kThreads, c.sms, 8), out, oslot,
                           last ? c.eps : 0.0));
    unsigned long long nout = 0;
    QX_TRY(sync_read(c, &nout, c.sc.ncnt + oslot, 8));
    if (capped && nout > ocap) {
      if (fast) c.ftab->dirty = true;
      c.al.put(out.base);
      return fail(QX_EBUDGET, "term storage of a merge pass exceeds hbm_budget");
    }
    if (const qx_status e = check_err(c)) {
      c.al.put(out.base);
      return e;
    }
    if (fast) c.ftab->dirty = false;
    if (const qx_status e = check_limits(c, nout)) {
      c.al.put(out.base);
      return e;
    }
    c.end_bytes_only(KC_INSERT, 1, uint64_t(c.N) * (16 * W + sizeof(WT)));
    c.end_bytes_only(KC_EMIT, 1, (c.N + nout) * (16 * W + sizeof(WT)));
    c.st.alg_bytes += (c.N + nout) * (16 * W + sizeof(WT));
    c.st.children += nout;
    replace_cur(c, out, nout, oslot);
  }
  return QX_OK;
}

// Expansion of a fan-out step over the qubits that need no merge, in parts:
// exp_count uploads their tables, counts every term's children and scans the
// counts (the total lands in ncnt[2]); exp_emit allocates the output for cap
// children and launches the tile table and the emit (which do nothing if the
// total exceeds cap); exp_accept makes the output current.
struct ExpPending {
  unsigned long long* offs = nullptr;
  unsigned long long* tiles = nullptr;
  TermBuf out;
  int nq = 0;
};

void exp_release(Ctx& c, ExpPending* ep) {
  c.al.put(ep->tiles);
  c.al.put(ep->offs);
  c.al.put(ep->out.base);
  *ep = ExpPending();
}

template <int W, typename WT>
qx_status exp_count(Ctx& c, const std::vector<const FanQubit*>& fq, ExpPending* ep) {
  Scratch& s = c.sc;
  std::vector<FanQ> hq;
  for (const FanQubit* f : fq) hq.push_back(to_dev(*f));
  QX_TRY(h2d(c, s.fanq, hq.data(), hq.size() * sizeof(FanQ)));
  ep->nq = int(hq.size());
  const size_t ntiles = (c.N + kScanTile - 1) / kScanTile;
  ep->offs = static_cast<unsigned long long*>(c.al.get((c.N + ntiles + 1) * 8));
  if (!ep->offs) return fail(QX_ENOMEM, "device allocation of the expansion offsets failed");
  unsigned long long* tsum = ep->offs + c.N;
  if (c.N <= size_t(kScanTile)) {  // one block counts and scans
    c.begin(KC_COUNT);
    k_expand_count_small<W, WT><<<1, kScanThreads, ep->nq * sizeof(FanQ), c.al.s>>>(
        c.cur.view<WT>(), s.ncnt + c.cslot, s.fanq, ep->nq, ep->offs, s.ncnt + 2);
    c.end(KC_COUNT, 1, uint64_t(c.N) * (16 * W + sizeof(WT)));
    QX_TRY_CUDA(cudaGetLastError());
    return QX_OK;
  }
  c.begin(KC_COUNT);
  k_expand_count<W, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, ep->nq * sizeof(FanQ),
                          c.al.s>>>(c.cur.view<WT>(), s.ncnt + c.cslot, s.fanq, ep->nq, ep->offs);
  c.end(KC_COUNT, 1, uint64_t(c.N) * (16 * W + sizeof(WT)));
  c.begin(KC_SCAN);
  k_scan_tiles<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(ep->offs, s.ncnt + c.cslot, tsum);
  k_scan_sums<<<1, 1024, 0, c.al.s>>>(tsum, ntiles, s.ncnt + 2);
  k_scan_add<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(ep->offs, s.ncnt + c.cslot, tsum);
  c.end(KC_SCAN, 3, uint64_t(c.N) * 8 * 3);
  QX_TRY_CUDA(cudaGetLastError());
  return QX_OK;
}

template <int W, typename WT>
qx_status exp_emit(Ctx& c, ExpPending* ep, unsigned long long cap) {
  Scratch& s = c.sc;
  QX_TRY(alloc_terms(c.al, W, c.wtb, cap, &ep->out));
  const unsigned egrid = unsigned(std::max<unsigned long long>(
      1, std::min<unsigned long long>((cap + kExpTile - 1) / kExpTile,
                                      (unsigned long long)c.sms * 8)));
  const size_t esmem = expand_emit_smem<W, WT>(ep->nq);
  const unsigned long long ntile = (cap + kExpTile - 1) / kExpTile;
  ep->tiles = static_cast<unsigned long long*>(c.al.get(size_t(2 * ntile + 2) * 8));
  if (!ep->tiles) return fail(QX_ENOMEM, "device allocation of the expansion tile table failed");
  c.begin(KC_EXPAND);
  k_expand_tiles<<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
      ep->offs, s.ncnt + c.cslot, s.ncnt + 2, cap, ep->tiles, ep->tiles + ntile + 1);
  k_expand_emit<W, WT><<<egrid, kExpThreads, esmem, c.al.s>>>(
      c.cur.view<WT>(), s.ncnt + c.cslot, ep->offs, s.ncnt + 2, cap, ep->tiles,
      ep->tiles + ntile + 1, s.fanq, ep->nq, ep->out.view<WT>());
  c.end(KC_EXPAND, 2, (c.N + cap) * (16 * W + sizeof(WT)));
  QX_TRY_CUDA(cudaGetLastError());
  return QX_OK;
}

template <int W, typename WT>
qx_status exp_accept(Ctx& c, ExpPending* ep, unsigned long long total) {
  const int oslot = 1 - c.cslot;
  c.st.alg_bytes += (c.N + total) * (16 * W + sizeof(WT));
  c.st.children += total;
  QX_TRY(h2d(c, c.sc.ncnt + oslot, &total, 8));
  c.al.put(ep->tiles);
  c.al.put(ep->offs);
  replace_cur(c, ep->out, total, oslot);
  *ep = ExpPending();
  if (c.eps > 0.0) QX_TRY(prune_cur<W, WT>(c));
  return QX_OK;
}

// From the per-generator letter masks: the qubits that need a merge in some
// generator (mq, with the per-generator mixed masks) and the others (fq).
void split_fan(const Ctx& c, const FanStep& fs, const std::vector<unsigned long long>& gm,
               std::vector<uint64_t>* mixed, std::vector<const FanQubit*>* mq,
               std::vector<const FanQubit*>* fq) {
  const int W = c.W;
  const size_t G = size_t(c.G);
  mixed->assign(G * W, 0);
  uint64_t any[kMaxWords] = {0, 0};
  for (size_t g = 0; g < G; ++g)
    for (int k = 0; k < W; ++k) {
      const uint64_t a = gm[(g * 3 + 0) * W + k], b = gm[(g * 3 + 1) * W + k],
                     d = gm[(g * 3 + 2) * W + k];
      const uint64_t m = (a & b) | (a & d) | (b & d);
      (*mixed)[g * W + k] = m;
      any[k] |= m;
    }
  mq->clear();
  fq->clear();
  for (const FanQubit& f : fs.qs)
    ((any[f.q / 64] >> (f.q % 64)) & 1 ? mq : fq)->push_back(&f);
}

// Fused expansion of a small fan-out step (qx_expand_fused.cuh), in parts:
// xs_count writes the letter masks (gmask) and the children per range and
// scans them (the total lands in ncnt[2]); xs_emit allocates the output for
// cap children and writes them, applying `fused` (a Clifford pass on other
// qubits, or none) to each parent; xs_accept makes the output current.  A
// run on the step's recorded offsets (xs_replay) skips the count.
struct XsPending {
  unsigned long long* tiles = nullptr;  // range sums -> offsets (owned)
  const unsigned long long* offs = nullptr;     // the range offsets the emission uses
  const unsigned long long* total_d = nullptr;  // their total (device)
  XsCheck chk{nullptr, nullptr};
  TermBuf out;
  size_t nranges = 0;  // ranges of spans: one warp of the emission each
  size_t per = 0;      // spans per range
  unsigned grid = 0;   // blocks of the emission (nranges / 8)
  unsigned long long written = ~0ull;  // the count the last emission stored in the output slot
};

void xs_release(Ctx& c, XsPending* xp) {
  c.al.put(xp->tiles);
  c.al.put(xp->out.base);
  *xp = XsPending();
}

// The step record of the fused kernels: each wire's rows (children's letters
// and entries), the letter masks, and the pruning thresholds as bit patterns
// (the kernels compare |w| with them as integers).
XsStep xs_step(const FanStep& fs, double eps) {
  XsStep st;
  std::memset(&st, 0, sizeof st);
  st.nq = int(fs.qs.size());
  double tmin = 1.0;
  for (int j = 0; j < st.nq; ++j) {
    const FanQubit& f = fs.qs[size_t(j)];
    st.word[j] = uint8_t(f.q / 64);
    st.bit[j] = uint8_t(f.q % 64);
    st.words |= 1u << (f.q / 64);
    double m = 1.0;
    for (int a = 0; a < 3; ++a) {
      if (!f.iso[a]) st.niso[a][f.q / 64] |= 1ull << (f.q % 64);
      XsRow& row = st.row[j][a];
      row.nn = f.nnz[a];
      for (int d = 0; d < f.nnz[a]; ++d) {
        const int c = f.col[a][d];
        row.col[d] = uint8_t(c);
        row.t[d] = f.t.r[a][c];
        row.th[d] = float(row.t[d]);
        row.tl[d] = float(row.t[d] - double(row.th[d]));
        m = std::min(m, std::fabs(row.t[d]));
      }
    }
    tmin *= m;
  }
  st.prune = eps > 0.0 ? 1 : 0;
  if (st.prune) {
    std::memcpy(&st.eps_bits, &eps, 8);
    // the smallest float not below eps: double(v) < eps iff |v| < it
    float ef = float(eps);
    if (double(ef) < eps) ef = std::nextafter(ef, INFINITY);
    std::memcpy(&st.eps_bits32, &ef, 4);
    // every child of a parent with |w| >= keep has |w t...| >= eps (the
    // margin covers the roundings of up to kSmallMaxWires products)
    const double keep = tmin > 0.0 ? eps / tmin * (1.0 + 1e-6) : INFINITY;
    std::memcpy(&st.keep_bits, &keep, 8);
    float kf = float(keep * (1.0 + 1e-4));
    if (double(kf) < keep * (1.0 + 1e-4)) kf = std::nextafter(kf, INFINITY);
    std::memcpy(&st.keep_bits32, &kf, 4);
  }
  return st;
}

// The partition of a small step's spans into ranges: one warp of the
// emission per range, and exactly one wave of emission blocks (as many as
// stay resident on every SM with the kernel's registers and gate list: a
// second, partial wave would leave most SMs idle behind its last ranges).
//
// The dynamic shared memory an emission may use is a process-wide attribute
// of the kernel (per device), so it is only ever raised, under a lock: a
// thread that needs less never lowers it under another thread's launch.
template <int W, typename WT, int CK, int NQ>
void xs_emit_allow_smem(size_t smem) {
  static std::atomic<size_t> allowed[64];
  static std::mutex mu;
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<size_t>& a = allowed[dev & 63];
  if (smem <= a.load(std::memory_order_acquire)) return;
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= a.load(std::memory_order_relaxed)) return;
  if (cudaFuncSetAttribute(k_xs_emit<W, WT, CK, NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(smem)) == cudaSuccess)
    a.store(smem, std::memory_order_release);
  else
    cudaGetLastError();  // the launch reports it
}

template <int W, typename WT, int CK, int NQ>
int xs_emit_per_sm(size_t smem) {
  xs_emit_allow_smem<W, WT, CK, NQ>(smem);
  // the last shared-memory size asked about and its answer
  static thread_local size_t last_smem = ~size_t(0);
  static thread_local int last_n = 0;
  if (smem == last_smem && last_n) return last_n;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_xs_emit<W, WT, CK, NQ>, kXsThreads,
                                                    smem) != cudaSuccess || n < 1) {
    cudaGetLastError();
    n = 1;
  }
  last_smem = smem;
  last_n = n;
  return n;
}

// The most children a parent of the step can have (the product of its
// wires' largest row sizes; at most kSmallMaxChildren).
int xs_max_children(const FanStep& fs) {
  int prod = 1;
  for (const FanQubit& f : fs.qs) {
    int m = 1;
    for (int a = 0; a < 3; ++a) m = std::max(m, int(f.nnz[a]));
    prod *= m;
  }
  return std::min(prod, kSmallMaxChildren);
}

int xs_gate_list(const qx_plan_device::Pass* fused) {
  return fused && !fused->identity && !fused->use_table ? fused->nops : 0;
}

template <int W, typename WT>
int xs_emit_blocks_per_sm(const FanStep& fs, const qx_plan_device::Pass* fused) {
  const int nq = int(fs.qs.size());
  const size_t smem = xt_smem_bytes<W, WT>(xs_max_children(fs), xs_gate_list(fused));
  auto pick = [&](auto ck) {
    constexpr int CK = decltype(ck)::value;
    return nq == 1   ? xs_emit_per_sm<W, WT, CK, 1>(smem)
           : nq == 2 ? xs_emit_per_sm<W, WT, CK, 2>(smem)
                     : xs_emit_per_sm<W, WT, CK, 0>(smem);
  };
  if (!fused || fused->identity) return pick(std::integral_constant<int, 0>());
  if (!fused->use_table) return pick(std::integral_constant<int, 1>());
  return fused->cb == 4 ? pick(std::integral_constant<int, 4>())
                        : pick(std::integral_constant<int, 3>());
}

template <int W, typename WT>
void xs_partition(const Ctx& c, const FanStep& fs, const qx_plan_device::Pass* fused,
                  XsPending* xp) {
  const size_t nspans = (c.N + kXsSpan - 1) / kXsSpan;
  const int per_sm = xs_emit_blocks_per_sm<W, WT>(fs, fused);
  xp->grid = grid_for(nspans, kXsThreads / 32, c.sms, per_sm);
  xp->nranges = size_t(xp->grid) * (kXsThreads / 32);
  xp->per = std::max<size_t>(1, (nspans + xp->nranges - 1) / xp->nranges);
}

template <int W, typename WT>
qx_status xs_count(Ctx& c, const FanStep& fs, const qx_plan_device::Pass* fused, XsPending* xp) {
  Scratch& s = c.sc;
  const XsStep st = xs_step(fs, c.eps);
  xs_partition<W, WT>(c, fs, fused, xp);
  const size_t R = xp->nranges;
  xp->tiles = static_cast<unsigned long long*>(c.al.get((R + 1) * 8));
  if (!xp->tiles) return fail(QX_ENOMEM, "device allocation of the expansion range sums failed");
  const size_t G = size_t(c.G);
  QX_TRY_CUDA(cudaMemsetAsync(s.gmask, 0, G * 3 * W * 8, c.al.s));
  unsigned words = 0;
  for (int k = 0; k < W; ++k) words += (st.words >> k) & 1;
  c.begin(KC_COUNT);
  // one wave of count blocks, each warp striding over the ranges
  static thread_local int count_per_sm = 0;
  if (!count_per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&count_per_sm, k_xs_count<W, WT, 1>,
                                                      kXsThreads, 0) != cudaSuccess ||
        count_per_sm < 1) {
      cudaGetLastError();
      count_per_sm = 2;
    }
  }
  const unsigned cgrid = grid_for(R, kXsThreads / 32, c.sms, count_per_sm);
  const auto view = c.cur.view<WT>();
  if (st.nq == 1)
    k_xs_count<W, WT, 1><<<cgrid, kXsThreads, 0, c.al.s>>>(view, s.ncnt + c.cslot, st, R, xp->per,
                                                           s.gmask, xp->tiles);
  else if (st.nq == 2)
    k_xs_count<W, WT, 2><<<cgrid, kXsThreads, 0, c.al.s>>>(view, s.ncnt + c.cslot, st, R, xp->per,
                                                           s.gmask, xp->tiles);
  else
    k_xs_count<W, WT, 0><<<cgrid, kXsThreads, 0, c.al.s>>>(view, s.ncnt + c.cslot, st, R, xp->per,
                                                           s.gmask, xp->tiles);
  c.end(KC_COUNT, 1, uint64_t(c.N) * (16 * words + 4 + (c.eps > 0.0 ? sizeof(WT) : 0)));
  c.begin(KC_SCAN);
  k_scan_sums<<<1, 1024, 0, c.al.s>>>(xp->tiles, R, s.ncnt + 2);
  c.end(KC_SCAN, 1, uint64_t(R) * 16);
  QX_TRY_CUDA(cudaGetLastError());
  xp->offs = xp->tiles;
  xp->total_d = s.ncnt + 2;
  return QX_OK;
}

template <int W, typename WT, int CK, int NQ>
qx_status xs_launch_error(cudaError_t e, size_t smem, unsigned grid) {
  cudaFuncAttributes fa{};
  cudaFuncGetAttributes(&fa, k_xs_emit<W, WT, CK, NQ>);
  cudaGetLastError();
  return fail(QX_ECUDA, std::string("fused expansion launch failed: ") + cudaGetErrorString(e) +
                            " (dynamic shared memory " + std::to_string(smem) + " of at most " +
                            std::to_string(fa.maxDynamicSharedSizeBytes) + ", static " +
                            std::to_string(fa.sharedSizeBytes) + ", grid " + std::to_string(grid) +
                            ")");
}

template <int W, typename WT, int CK>
qx_status xs_launch(Ctx& c, const FanStep& fs, XsPending* xp, unsigned long long cap,
                    const XsPass& ps, int nops) {
  const int maxc = xs_max_children(fs);
  const size_t smem = xt_smem_bytes<W, WT>(maxc, nops);
  const unsigned grid = xp->grid;  // 8 ranges of the count's partition per block
  const XsStep st = xs_step(fs, c.eps);
  const auto in = c.cur.view<WT>();
  const auto out = xp->out.view<WT>();
  const unsigned long long* n_in = c.sc.ncnt + c.cslot;
  const XsStats sts{c.stats_last ? c.sc.gcount : nullptr, c.stats_last ? c.sc.gsumsq : nullptr};
  unsigned long long* n_out = c.sc.ncnt + (1 - c.cslot);  // the slot xs_accept makes current
  if (!xs_bulk_ok(in, W))
    return fail(QX_ECUDA, "internal error: a term buffer is not on a 16-byte boundary");
  xp->written = cap;
  QX_TRY_CUDA(cudaGetLastError());  // nothing pending before the launch
  cudaError_t e;
  if (st.nq == 1) {
    xs_emit_allow_smem<W, WT, CK, 1>(smem);
    k_xs_emit<W, WT, CK, 1><<<grid, kXsThreads, smem, c.al.s>>>(
        in, n_in, xp->offs, xp->per, xp->total_d, cap, st, ps, xp->chk, sts, c.sc.pruned, out,
        n_out, maxc, std::max(64u, c.spin_limit / 32), c.sc.serr);
    if ((e = cudaGetLastError()) != cudaSuccess) return xs_launch_error<W, WT, CK, 1>(e, smem, grid);
  } else if (st.nq == 2) {
    xs_emit_allow_smem<W, WT, CK, 2>(smem);
    k_xs_emit<W, WT, CK, 2><<<grid, kXsThreads, smem, c.al.s>>>(
        in, n_in, xp->offs, xp->per, xp->total_d, cap, st, ps, xp->chk, sts, c.sc.pruned, out,
        n_out, maxc, std::max(64u, c.spin_limit / 32), c.sc.serr);
    if ((e = cudaGetLastError()) != cudaSuccess) return xs_launch_error<W, WT, CK, 2>(e, smem, grid);
  } else {
    xs_emit_allow_smem<W, WT, CK, 0>(smem);
    k_xs_emit<W, WT, CK, 0><<<grid, kXsThreads, smem, c.al.s>>>(
        in, n_in, xp->offs, xp->per, xp->total_d, cap, st, ps, xp->chk, sts, c.sc.pruned, out,
        n_out, maxc, std::max(64u, c.spin_limit / 32), c.sc.serr);
    if ((e = cudaGetLastError()) != cudaSuccess) return xs_launch_error<W, WT, CK, 0>(e, smem, grid);
  }
  return QX_OK;
}

template <int W, typename WT>
qx_status xs_emit(Ctx& c, const FanStep& fs, XsPending* xp, unsigned long long cap,
                  const qx_plan_device::Pass* fused) {
  QX_TRY(alloc_terms(c.al, W, c.wtb, cap, &xp->out));
  XsPass ps{};
  if (c.stats_last) QX_TRY_CUDA(cudaMemsetAsync(c.sc.gcount, 0, size_t(c.G) * 16, c.al.s));
  c.begin(KC_EXPAND);
  if (!fused || fused->identity) {
    QX_TRY((xs_launch<W, WT, 0>(c, fs, xp, cap, ps, 0)));
  } else if (!fused->use_table) {
    ps.ops = fused->ops;
    ps.nops = fused->nops;
    QX_TRY((xs_launch<W, WT, 1>(c, fs, xp, cap, ps, fused->nops)));
  } else {
    ps.tab_xz = fused->tab_xz;
    ps.tab_e = fused->tab_e;
    ps.chunks = fused->chunks;
    ps.live = fused->live;
    ps.pmk = pass_masks<W>(*fused, c.n);
    // the tables stay in global memory (k_xs_emit reads them on image-cache misses)
    if (fused->cb == 4)
      QX_TRY((xs_launch<W, WT, 4>(c, fs, xp, cap, ps, 0)));
    else
      QX_TRY((xs_launch<W, WT, 3>(c, fs, xp, cap, ps, 0)));
  }
  c.end(KC_EXPAND, 1, (c.N + cap) * (16 * W + sizeof(WT)));
  QX_TRY_CUDA(cudaGetLastError());
  return QX_OK;
}

template <int W, typename WT>
qx_status xs_accept(Ctx& c, XsPending* xp, unsigned long long total, int nfused) {
  const int oslot = 1 - c.cslot;
  c.st.alg_bytes += (c.N + total) * (16 * W + sizeof(WT));
  c.st.children += total;
  c.st.clifford_passes += uint64_t(nfused);
  // the emission stored its output size in the slot; another total (a guess
  // that was larger than the count) is copied
  if (xp->written != total) QX_TRY(h2d(c, c.sc.ncnt + oslot, &total, 8));
  c.al.put(xp->tiles);
  replace_cur(c, xp->out, total, oslot);
  *xp = XsPending();  // pruning (eps > 0) happened in the emission
  return QX_OK;
}

// Keeps the range offsets of a step launched on its guessed size (the scan
// of this run's count): the plan's copy, published only when the run
// completes with every check held (then every step's input was exact).  One
// run per step and precision records.
template <int W, typename WT>
void xs_record(Ctx& c, FanHint* hint, const XsPending& xp, unsigned long long total) {
  FanHint::Record& h = hint->rec[sizeof(WT) == 4];
  if (!c.defer || !xp.tiles || h.bad.load() || h.offs.load(std::memory_order_acquire)) return;
  int free_slot = 0;
  if (!h.claim.compare_exchange_strong(free_slot, 1)) return;
  unsigned long long* r = nullptr;
  const size_t R = xp.nranges;
  if (cudaMalloc(&r, (R + 1) * 8) != cudaSuccess ||
      cudaMemcpyAsync(r, xp.tiles, R * 8, cudaMemcpyDeviceToDevice, c.al.s) != cudaSuccess ||
      cudaMemcpyAsync(r + R, c.sc.ncnt + 2, 8, cudaMemcpyDeviceToDevice, c.al.s) != cudaSuccess) {
    cudaGetLastError();
    if (r) {
      cudaStreamSynchronize(c.al.s);
      cudaFree(r);
    }
    h.claim.store(0);
    return;
  }
  Ctx::Record rc;
  rc.rec = &h;
  rc.offs = r;
  rc.n = c.N;
  rc.ranges = R;
  rc.per = xp.per;
  rc.total = total;
  c.records.push_back(rc);
}

// The run's records into their hints (the run completed; its stream work is done).
void publish_records(Ctx& c) {
  for (const Ctx::Record& rc : c.records) {
    FanHint::Record* h = rc.rec;
    h->n = rc.n;
    h->ranges = rc.ranges;
    h->per = rc.per;
    h->total = rc.total;
    h->eps = c.eps;
    h->offs.store(rc.offs, std::memory_order_release);
  }
  c.records.clear();
}

// A step launched on its recorded range offsets: the emission alone, with
// the checks of XsCheck read back at the end of the run.  *ran is false
// (nothing launched) when the record does not apply to this run.
template <int W, typename WT>
qx_status xs_replay(Ctx& c, const FanStep& fs, FanHint* hint, const qx_plan_device::Pass* fused,
                    XsPending* xp, bool* ran, unsigned long long* total) {
  *ran = false;
  if (!hint || !c.defer) return QX_OK;
  FanHint::Record& h = hint->rec[sizeof(WT) == 4];
  if (h.bad.load(std::memory_order_relaxed)) return QX_OK;
  const unsigned long long* rec = h.offs.load(std::memory_order_acquire);
  if (!rec || h.n != c.N || h.eps != c.eps) return QX_OK;
  xs_partition<W, WT>(c, fs, fused, xp);
  if (xp->nranges != h.ranges || xp->per != h.per || !limits_ok(c, h.total)) return QX_OK;
  if (c.chk_used >= c.chk_slots) return QX_OK;
  const int slot = c.chk_used;
  unsigned char* chk = c.chk_dev + size_t(slot) * c.chk_stride;  // zeroed with the scratch
  xp->offs = rec;
  xp->total_d = rec + xp->nranges;
  xp->chk.err = reinterpret_cast<unsigned*>(chk);
  xp->chk.gwire = reinterpret_cast<uint32_t*>(chk + 16);
  const qx_status st = xs_emit<W, WT>(c, fs, xp, h.total, fused);
  if (st != QX_OK) {
    if (st != QX_ENOMEM) return st;
    c.al.put(xp->out.base);  // the recorded size does not fit now: count first
    *xp = XsPending();
    clear_error();
    cudaGetLastError();
    return QX_OK;
  }
  c.chk_used++;
  Ctx::Deferred d;
  d.kind = kHintReplay;
  d.hint = hint;
  d.rec = &h;
  d.fs = &fs;
  d.expect = h.total;
  d.slot = slot;
  c.deferred.push_back(std::move(d));
  *ran = true;
  *total = h.total;
  return QX_OK;
}

// A small fan-out step through the fused expansion.  `pre` is the pending
// Clifford pass before the step and `tail` the program's last pass after it
// (both act on other qubits than the step's wires, either may be NULL);
// pre_tail is the two composed.  *done is false when some wire needs a merge:
// gm then holds the letter masks, `pre` has been applied and the ordinary
// path continues.  *absorbed: the tail pass ran inside the expansion.
template <int W, typename WT>
qx_status run_fan_small(Ctx& c, const FanStep& fs, FanHint* hint,
                        const qx_plan_device::Pass* pre, const qx_plan_device::Pass* tail,
                        const qx_plan_device::Pass* pre_tail,
                        std::vector<unsigned long long>& gm, bool* done, bool* absorbed) {
  *done = false;
  *absorbed = false;
  const qx_plan_device::Pass* fused = pre;
  int nfused = pre ? 1 : 0;
  bool uses_tail = false;
  if (tail && !pre) {
    fused = tail;
    nfused = 1;
    uses_tail = true;
  } else if (tail && pre_tail) {
    fused = pre_tail;
    nfused = 2;
    uses_tail = true;
  }
  XsPending xp;
  bool replayed = false;
  unsigned long long rtotal = 0;
  QX_TRY((xs_replay<W, WT>(c, fs, hint, fused, &xp, &replayed, &rtotal)));
  if (replayed) {
    *done = true;
    *absorbed = uses_tail;
    c.stats_done = c.stats_last;
    return xs_accept<W, WT>(c, &xp, rtotal, nfused);
  }
  xp = XsPending();
  qx_status st = xs_count<W, WT>(c, fs, fused, &xp);
  if (st != QX_OK) {
    xs_release(c, &xp);
    return st;
  }
  auto finish = [&](unsigned long long total) -> qx_status {
    *done = true;
    *absorbed = uses_tail;
    c.stats_done = c.stats_last;
    return xs_accept<W, WT>(c, &xp, total, nfused);
  };
  std::vector<uint64_t> mixed;
  std::vector<const FanQubit*> mq, fq;
  unsigned long long total = 0;
  bool have_gm = false;
  const int guess = hint ? hint->kind.load(std::memory_order_relaxed) : kHintNone;
  const unsigned long long cap = hint ? hint->total.load(std::memory_order_relaxed) : 0;
  if (guess == kHintExpand && cap && limits_ok(c, cap)) {
    // the last run's size, launched before the masks are read back
    st = xs_emit<W, WT>(c, fs, &xp, cap, fused);
    if (st == QX_ENOMEM) {  // that size does not fit now: count first
      c.al.put(xp.out.base);
      xp.out = TermBuf();
      clear_error();
      cudaGetLastError();
      hint->streak.store(0, std::memory_order_relaxed);
      c.st.guesses_missed++;
    } else if (st != QX_OK) {
      xs_release(c, &xp);
      return st;
    } else {
      if (c.defer && hint->streak.load(std::memory_order_relaxed) >= 2) {
        // checked at the end of the run (see run_fan)
        auto* rg = static_cast<unsigned long long*>(rb_take(c, gm.size() * 8));
        auto* rt = static_cast<unsigned long long*>(rb_take(c, 8));
        if (rg && rt) {
          k_fill_tail<W, WT><<<grid_for(cap, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
              xp.out.view<WT>(), c.sc.ncnt + 2, cap);
          QX_TRY_CUDA(cudaMemcpyAsync(rg, c.sc.gmask, gm.size() * 8, cudaMemcpyDeviceToHost,
                                      c.al.s));
          QX_TRY_CUDA(cudaMemcpyAsync(rt, c.sc.ncnt + 2, 8, cudaMemcpyDeviceToHost, c.al.s));
          Ctx::Deferred d;
          d.kind = kHintExpand;
          d.hint = hint;
          d.fs = &fs;
          d.expect = cap;
          d.gm = rg;
          d.total = rt;
          c.deferred.push_back(std::move(d));
          xs_record<W, WT>(c, hint, xp, cap);
          return finish(cap);
        }
      }
      st = sync_read2(c, gm.data(), c.sc.gmask, gm.size() * 8, &total, c.sc.ncnt + 2, 8);
      if (st != QX_OK) {
        xs_release(c, &xp);
        return st;
      }
      have_gm = true;
      split_fan(c, fs, gm, &mixed, &mq, &fq);
      if (mq.empty() && limits_ok(c, total)) {  // the guess held
        if (total > cap) {  // more children than last time: emit again at full size
          c.al.put(xp.out.base);
          xp.out = TermBuf();
          st = xs_emit<W, WT>(c, fs, &xp, total, fused);
          if (st != QX_OK) {
            xs_release(c, &xp);
            return st;
          }
        }
        hint->total.store(total, std::memory_order_relaxed);
        if (total == cap) hint->streak.fetch_add(1, std::memory_order_relaxed);
        else hint->streak.store(0, std::memory_order_relaxed);
        c.st.guesses_held++;
        if (total == cap) xs_record<W, WT>(c, hint, xp, total);
        return finish(total);
      }
      hint->streak.store(0, std::memory_order_relaxed);
      c.st.guesses_missed++;
      c.al.put(xp.out.base);
      xp.out = TermBuf();
    }
  }
  if (!have_gm) {
    st = sync_read2(c, gm.data(), c.sc.gmask, gm.size() * 8, &total, c.sc.ncnt + 2, 8);
    if (st != QX_OK) {
      xs_release(c, &xp);
      return st;
    }
    split_fan(c, fs, gm, &mixed, &mq, &fq);
  }
  if (mq.empty()) {
    st = check_limits(c, total);
    if (st == QX_OK) st = xs_emit<W, WT>(c, fs, &xp, total, fused);
    if (st != QX_OK) {
      xs_release(c, &xp);
      return st;
    }
    if (hint) {
      hint->total.store(total, std::memory_order_relaxed);
      hint->kind.store(kHintExpand, std::memory_order_relaxed);
    }
    return finish(total);
  }
  // some wire needs a merge: the ordinary path continues from the masks (the
  // pending pass acts on other qubits, so the masks stay valid after it)
  xs_release(c, &xp);
  if (pre) QX_TRY((run_pass<W, WT>(c, *pre)));
  return QX_OK;
}

template <int W, typename WT>
qx_status run_fan(Ctx& c, const FanStep& fs, uint64_t ops_before, FanHint* hint,
                  const qx_plan_device::Pass* pre, const qx_plan_device::Pass* tail,
                  const qx_plan_device::Pass* pre_tail, bool* absorbed) {
  c.st.term_updates += (ops_before + 1) * c.N;
  c.st.fan_steps++;
  *absorbed = false;
  if (c.N == 0) return QX_OK;
  Scratch& s = c.sc;
  const size_t G = size_t(c.G);
  // 1. which fan-out qubits need a merge, per generator (launched when some
  // path needs it: a block-ordered guess is checked by the device alone)
  bool masked = false;
  auto launch_mask = [&]() -> qx_status {
    if (masked) return QX_OK;
    masked = true;
    uint64_t niso[3][kMaxWords] = {};
    for (const FanQubit& f : fs.qs)
      for (int a = 0; a < 3; ++a)
        if (!f.iso[a]) niso[a][f.q / 64] |= 1ull << (f.q % 64);
    uint64_t* d_niso = reinterpret_cast<uint64_t*>(s.fanq + c.n);  // staging after the FanQ array
    QX_TRY(h2d(c, d_niso, niso, sizeof niso));
    QX_TRY_CUDA(cudaMemsetAsync(s.gmask, 0, G * 3 * W * 8, c.al.s));
    c.begin(KC_MASK);
    k_fan_mask<W, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), s.ncnt + c.cslot, d_niso, d_niso + kMaxWords, d_niso + 2 * kMaxWords,
        s.gmask);
    c.end(KC_MASK, 1, uint64_t(c.N) * 16 * W);
    QX_TRY_CUDA(cudaGetLastError());
    return QX_OK;
  };
  std::vector<unsigned long long> gm(G * 3 * W);
  std::vector<uint64_t> mixed;
  std::vector<const FanQubit*> mq, fq;
  bool have_gm = false;
  // 2. the last run's outcome, launched before the masks are read back
  const int guess = hint ? hint->kind.load(std::memory_order_relaxed) : kHintNone;
  if (small_fan_step(fs) && guess != kHintBlocks) {
    // the fused expansion (it computes the masks itself)
    bool done = false;
    QX_TRY((run_fan_small<W, WT>(c, fs, hint, pre, tail, pre_tail, gm, &done, absorbed)));
    if (done) return QX_OK;
    have_gm = true;
    masked = true;
    split_fan(c, fs, gm, &mixed, &mq, &fq);
  } else if (pre) {
    QX_TRY((run_pass<W, WT>(c, *pre)));
  }
  if (have_gm) {
    // the small path's masks decide below
  } else if (guess == kHintExpand) {
    const unsigned long long cap = hint->total.load(std::memory_order_relaxed);
    if (cap && limits_ok(c, cap)) {
      QX_TRY(launch_mask());  // the masks decide whether a merge was needed
      std::vector<const FanQubit*> all;
      for (const FanQubit& f : fs.qs) all.push_back(&f);
      ExpPending ep;
      qx_status st = exp_count<W, WT>(c, all, &ep);
      if (st != QX_OK) {
        exp_release(c, &ep);
        return st;
      }
      const qx_status est = exp_emit<W, WT>(c, &ep, cap);
      if (est != QX_OK) {
        exp_release(c, &ep);
        // only an allocation at the recorded size that fails now (another
        // generator range, a fuller device) falls back: no guess, the
        // ordinary path counts first; any other failure is the caller's
        if (est != QX_ENOMEM) return est;
        clear_error();
        cudaGetLastError();
        hint->streak.store(0, std::memory_order_relaxed);
        c.st.guesses_missed++;
      } else {
        // a guess that held in the last runs: no read-back now, the check
        // happens at the end of the run (the output is made harmless first
        // where its size differs from the guess)
        if (st == QX_OK && c.defer && hint->streak.load(std::memory_order_relaxed) >= 2) {
          auto* rg = static_cast<unsigned long long*>(rb_take(c, gm.size() * 8));
          auto* rt = static_cast<unsigned long long*>(rb_take(c, 8));
          if (rg && rt) {
            k_fill_tail<W, WT><<<grid_for(cap, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
                ep.out.view<WT>(), s.ncnt + 2, cap);
            QX_TRY_CUDA(cudaMemcpyAsync(rg, s.gmask, gm.size() * 8, cudaMemcpyDeviceToHost, c.al.s));
            QX_TRY_CUDA(cudaMemcpyAsync(rt, s.ncnt + 2, 8, cudaMemcpyDeviceToHost, c.al.s));
            Ctx::Deferred d;
            d.kind = kHintExpand;
            d.hint = hint;
            d.fs = &fs;
            d.expect = cap;
            d.gm = rg;
            d.total = rt;
            c.deferred.push_back(std::move(d));
            return exp_accept<W, WT>(c, &ep, cap);
          }
        }
        unsigned long long total = 0;
        if (st == QX_OK) st = sync_read2(c, gm.data(), s.gmask, gm.size() * 8, &total, s.ncnt + 2, 8);
        if (st != QX_OK) {
          exp_release(c, &ep);
          return st;
        }
        have_gm = true;
        split_fan(c, fs, gm, &mixed, &mq, &fq);
        if (mq.empty() && limits_ok(c, total)) {  // the guess held
          if (total > cap) {  // more children than last time: emit again at full size
            c.al.put(ep.tiles);
            c.al.put(ep.out.base);
            ep.tiles = nullptr;
            ep.out = TermBuf();
            st = exp_emit<W, WT>(c, &ep, total);
            if (st != QX_OK) {
              exp_release(c, &ep);
              return st;
            }
          }
          hint->total.store(total, std::memory_order_relaxed);
          if (total == cap) hint->streak.fetch_add(1, std::memory_order_relaxed);
          else hint->streak.store(0, std::memory_order_relaxed);
          c.st.guesses_held++;
          return exp_accept<W, WT>(c, &ep, total);
        }
        hint->streak.store(0, std::memory_order_relaxed);
        c.st.guesses_missed++;
        exp_release(c, &ep);
      }
    }
  } else if (guess == kHintBlocks && c.inplace && blocks_fit(c)) {
    // Every fan-out wire merged in block order last time.  The device decides
    // alone: all blocks complete means every group of every wire holds all of
    // the wire's non-isolated letters (the merge is then exact in place), and
    // a wire that needs no merge anywhere leaves its blocks incomplete.
    std::vector<const FanQubit*> gq;
    for (const FanQubit& f : fs.qs) gq.push_back(&f);
    BlocksPending bp;
    QX_TRY((launch_blocks<W, WT>(c, gq, &bp, hint->nblk.load(std::memory_order_relaxed))));
    if (bp.launched && c.defer && hint->streak.load(std::memory_order_relaxed) >= 2) {
      auto* re = static_cast<unsigned*>(rb_take(c, 8));
      if (re) {  // checked at the end of the run (see the expansion above)
        k_zero_if_err<W, WT><<<grid_for(bp.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
            bp.out.view<WT>(), bp.N, c.sc.err);
        QX_TRY_CUDA(cudaMemcpyAsync(re, c.sc.err, 4, cudaMemcpyDeviceToHost, c.al.s));
        QX_TRY_CUDA(cudaMemcpyAsync(re + 1, bp.nblk, 4, cudaMemcpyDeviceToHost, c.al.s));
        // a stale error word must not fail a later step: it is in re now
        QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
        Ctx::Deferred d;
        d.kind = kHintBlocks;
        d.hint = hint;
        d.fs = &fs;
        d.err = re;
        d.nblk = re + 1;
        c.deferred.push_back(std::move(d));
        bool done = false;
        return finish_blocks<W, WT>(c, &bp, 0, true, false, &done);
      }
    }
    if (bp.launched) {
      unsigned en[2] = {0, 0};
      if (const qx_status st = sync_read2(c, &en[0], c.sc.err, 4, &en[1], bp.nblk, 4)) {
        c.al.put(bp.mem);
        c.al.put(bp.out.base);
        return st;
      }
      const unsigned err = en[0];
      bool done = false;
      QX_TRY((finish_blocks<W, WT>(c, &bp, err, true, false, &done)));
      if (done) {
        hint->nblk.store(en[1], std::memory_order_relaxed);
        hint->streak.fetch_add(1, std::memory_order_relaxed);
        c.st.guesses_held++;
        return QX_OK;
      }
      hint->streak.store(0, std::memory_order_relaxed);
      c.st.guesses_missed++;
    }
  }
  QX_TRY(launch_mask());
  if (!have_gm) {
    QX_TRY(sync_read(c, gm.data(), s.gmask, gm.size() * 8));
    split_fan(c, fs, gm, &mixed, &mq, &fq);
  }
  if (!mq.empty()) QX_TRY(h2d(c, s.mixed, mixed.data(), G * W * 8));
  // 3. one merge pass per qubit that needs it in some generator
  const uint64_t blocks0 = c.st.block_steps;
  if (!mq.empty()) QX_TRY(run_merges<W, WT>(c, mq, !fq.empty(), gm, hint));
  if (fq.empty()) {
    if (hint) {
      // every fan-out wire merged in block order: the next run tries that
      const bool blocks = c.st.block_steps > blocks0 && W == 1;
      hint->kind.store(blocks ? kHintBlocks : kHintNone, std::memory_order_relaxed);
    }
    return QX_OK;
  }
  // 4. one-shot expansion over the qubits that need no merge anywhere
  ExpPending ep;
  qx_status st = exp_count<W, WT>(c, fq, &ep);
  unsigned long long total = 0;
  if (st == QX_OK) st = sync_read(c, &total, s.ncnt + 2, 8);
  if (st == QX_OK) st = check_limits(c, total);
  if (st == QX_OK) st = exp_emit<W, WT>(c, &ep, total);
  if (st != QX_OK) {
    exp_release(c, &ep);
    return st;
  }
  if (hint) {
    hint->total.store(total, std::memory_order_relaxed);
    hint->kind.store(mq.empty() ? kHintExpand : kHintNone, std::memory_order_relaxed);
  }
  return exp_accept<W, WT>(c, &ep, total);
}

// One Pauli rotation step (qx_pauli_rot.cuh): index the terms, count each
// term's outputs and find its partner, scan, emit.
template <int W, typename WT>
qx_status run_rot(Ctx& c, const RotStep& rs, uint64_t ops_before) {
  c.st.term_updates += (ops_before + 1) * c.N;
  c.st.fan_steps++;
  if (c.N == 0) return QX_OK;
  const size_t N = c.N;
  const unsigned long long cap = std::max<unsigned long long>(64, 2ull * N);
  const size_t ntiles = (N + kScanTile - 1) / kScanTile;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t tab_bytes = up(cap * sizeof(IndexSlot) + 16);
  void* mem = c.al.get(tab_bytes + up((N + ntiles + 1) * 8) + up(N * 8));
  if (!mem) return fail(QX_ENOMEM, "device allocation for a rotation step failed");
  auto* b8 = static_cast<unsigned char*>(mem);
  auto* tab = reinterpret_cast<IndexSlot*>(b8);
  auto* offs = reinterpret_cast<unsigned long long*>(b8 + tab_bytes);
  unsigned long long* tsum = offs + N;
  auto* pidx = reinterpret_cast<long long*>(b8 + tab_bytes + up((N + ntiles + 1) * 8));
  const RotQ rq = to_dev(rs);
  TermBuf out;
  auto body = [&]() -> qx_status {
    QX_TRY_CUDA(cudaMemsetAsync(tab, 0, cap * sizeof(IndexSlot), c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
    const unsigned grid = grid_for(N, kThreads, c.sms, 8);
    const auto view = c.cur.view<WT>();
    c.begin(KC_ROT);
    k_index_build<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, tab, cap, c.sc.err);
    k_rot_count<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, rq, tab, cap, offs, pidx);
    k_scan_tiles<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(offs, c.sc.ncnt + c.cslot, tsum);
    k_scan_sums<<<1, 1024, 0, c.al.s>>>(tsum, ntiles, c.sc.ncnt + 2);
    k_scan_add<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(offs, c.sc.ncnt + c.cslot, tsum);
    QX_TRY_CUDA(cudaGetLastError());
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    QX_TRY(sync_read(c, h, c.sc.ncnt, 40));
    if (unsigned(h[4]) & kErrProbe) return fail(QX_ECAP, "a hash table ran out of probe slots");
    const unsigned long long total = h[2];
    QX_TRY(check_limits(c, total));
    QX_TRY(alloc_terms(c.al, W, c.wtb, total, &out));
    k_rot_emit<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, rq, offs, pidx, out.view<WT>());
    c.end(KC_ROT, 6, (N + total) * (16 * W + sizeof(WT)));
    QX_TRY_CUDA(cudaGetLastError());
    const int oslot = 1 - c.cslot;
    QX_TRY(h2d(c, c.sc.ncnt + oslot, &total, 8));
    c.st.alg_bytes += (N + total) * (16 * W + sizeof(WT));
    c.st.children += total;
    replace_cur(c, out, total, oslot);
    out = TermBuf();
    return QX_OK;
  };
  const qx_status st = body();
  c.al.put(mem);
  if (st != QX_OK) {
    c.al.put(out.base);
    return st;
  }
  if (c.eps > 0.0) QX_TRY(prune_cur<W, WT>(c));
  return QX_OK;
}

// Scratch of a propagation over c.G generators: counters; the per-generator
// term counts, squared-weight sums and pruned mass, followed by the check
// slots of steps launched on recorded offsets (one device-to-host copy reads
// all of them at the end of the run); letter masks, mixed masks, fan-out
// tables.
qx_status setup_scratch(Ctx& c) {
  const size_t G = size_t(c.G), W = size_t(c.W);
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  // check slots: as many as the plan has fan-out steps, while they and the
  // statistics fit a quarter of the pinned read-back space
  c.chk_stride = al(16 + G * 4);
  const size_t nfan = c.p ? c.p->fans.size() : 0;
  c.chk_slots = G * 24 + nfan * c.chk_stride <= kReadbackBytes / 4 ? int(nfan) : 0;
  c.chk_used = 0;
  const size_t sz_cnt = 64, sz_tail = G * 24 + size_t(c.chk_slots) * c.chk_stride,
               sz_gm = G * 3 * W * 8, sz_mx = G * W * 8,
               sz_fq = size_t(std::max(c.n, kSmallMaxWires)) * sizeof(FanQ) + 3 * kMaxWords * 8;
  const size_t total = al(sz_cnt) + al(sz_tail) + al(sz_gm) + al(sz_mx) + al(sz_fq);
  c.sc.base = c.al.get(total);
  if (!c.sc.base) return fail(QX_ENOMEM, "device allocation of scratch failed");
  auto* b = static_cast<unsigned char*>(c.sc.base);
  c.sc.ncnt = reinterpret_cast<unsigned long long*>(b);
  c.sc.err = reinterpret_cast<unsigned*>(b + 32);
  c.sc.serr = reinterpret_cast<unsigned*>(b + 48);
  b += al(sz_cnt);
  c.sc.gcount = reinterpret_cast<unsigned long long*>(b);
  c.sc.gsumsq = reinterpret_cast<double*>(b + G * 8);
  c.sc.pruned = reinterpret_cast<double*>(b + G * 16);
  c.chk_dev = b + al(G * 24);
  b += al(sz_tail);
  c.sc.gmask = reinterpret_cast<unsigned long long*>(b);
  b += al(sz_gm);
  c.sc.mixed = reinterpret_cast<uint64_t*>(b);
  b += al(sz_mx);
  c.sc.fanq = reinterpret_cast<FanQ*>(b);
  QX_TRY_CUDA(cudaMemsetAsync(c.sc.base, 0, al(sz_cnt) + al(sz_tail), c.al.s));
  return QX_OK;
}

void free_scratch(Ctx& c) {
  c.al.put(c.sc.table);
  c.al.put(c.sc.payload);
  c.al.put(c.sc.base);
  c.sc = Scratch();
}

template <int W, typename WT>
qx_status propagate_impl(Ctx& c, const uint64_t* init_x, const uint64_t* init_z,
                         const double* init_w, int gen_begin, const qx_result* from,
                         qx_result** out) {
  const qx_plan* p = c.p;
  const size_t G = size_t(c.G);
  QX_TRY(setup_scratch(c));
  // A3: initial generators (or every term of a given state)
  const size_t N0 = from ? from->N : G;
  QX_TRY(check_limits(c, N0));
  QX_TRY(alloc_terms(c.al, W, c.wtb, N0, &c.cur));
  c.N = N0;
  c.cslot = 0;
  c.st.peak_terms = N0;
  c.begin(KC_INIT);
  if (from) {
    if (N0)
      k_copy_terms<W, WT><<<grid_for(N0, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
          from->buf.view<WT>(), N0, c.cur.view<WT>(), c.sc.ncnt);
  } else if (!init_x) {
    k_init_z<W, WT><<<1, 128, 0, c.al.s>>>(c.cur.view<WT>(), gen_begin, c.G, c.sc.ncnt);
  } else {
    void* tmp = c.al.get(G * (16 * W + sizeof(WT)));
    if (!tmp) return fail(QX_ENOMEM, "device allocation failed");
    auto* tx = static_cast<uint64_t*>(tmp);
    auto* tz = tx + G * W;
    auto* tw = reinterpret_cast<double*>(tz + G * W);
    QX_TRY(h2d(c, tx, init_x, G * W * 8));
    QX_TRY(h2d(c, tz, init_z, G * W * 8));
    if (init_w) QX_TRY(h2d(c, tw, init_w, G * 8));
    k_init_rows<W, WT><<<unsigned((G + 127) / 128), 128, 0, c.al.s>>>(c.cur.view<WT>(), tx, tz,
                                                                  init_w ? tw : nullptr, c.G,
                                                                  c.sc.ncnt);
    c.al.put(tmp);
  }
  c.end(KC_INIT, 1, N0 * (16 * W + sizeof(WT) + 4) * (from ? 2 : 1));
  QX_TRY_CUDA(cudaGetLastError());
  // the program: Clifford passes and fan-out steps in circuit order
  // A pass right before a small fan-out step and on other qubits than its
  // wires is left pending: the step's expansion applies it to each parent
  // (the two commute).  The program's last pass may likewise run inside the
  // last step's expansion.
  const auto& prog = p->program;
  const qx_plan_device::Pass* pending = nullptr;
  size_t last_work = prog.size();  // the last fan-out or rotation step
  for (size_t si = 0; si < prog.size(); ++si)
    if (prog[si].kind != kStepCliff) last_work = si;
  for (size_t si = 0; si < prog.size(); ++si) {
    const Step& stp = prog[si];
    if (stp.kind == kStepCliff) {
      const qx_plan_device::Pass& dp = p->dev->passes[stp.index];
      // a table-form pass over fewer than 64 terms per generator runs on its
      // own: inside the expansion, a warp whose parents belong to many
      // generators would resolve its image-cache misses one key at a time
      const bool few = dp.use_table && c.N < size_t(64) * size_t(c.G);
      if (!dp.identity && !few && si + 1 < prog.size() && prog[si + 1].kind == kStepFan) {
        const FanStep& nf = p->fans[prog[si + 1].index];
        if (small_fan_step(nf) && pass_disjoint(p->passes[stp.index], nf)) {
          pending = &dp;
          continue;
        }
      }
      QX_TRY(run_pass<W, WT>(c, dp));
    } else if (stp.kind == kStepRot) {
      QX_TRY(run_rot<W, WT>(c, p->rots[stp.index], stp.ops_before));
    } else {
      const FanStep& fs = p->fans[stp.index];
      const qx_plan_device::Pass* tail = nullptr;
      const qx_plan_device::Pass* pre_tail = nullptr;
      if (si + 2 == prog.size() && prog[si + 1].kind == kStepCliff) {
        const CliffPass& tp = p->passes[prog[si + 1].index];
        if (!tp.identity && pass_disjoint(tp, fs)) {
          tail = &p->dev->passes[prog[si + 1].index];
          if (pending && fs.pre_tail >= 0)
            pre_tail = &p->dev->passes[p->passes.size() + size_t(fs.pre_tail)];
        }
      }
      bool absorbed = false;
      c.stats_last = si == last_work;
      QX_TRY(run_fan<W, WT>(c, fs, stp.ops_before, p->dev ? &p->dev->hints[stp.index] : nullptr,
                            pending, tail, pre_tail, &absorbed));
      c.stats_last = false;
      pending = nullptr;
      if (absorbed) ++si;  // the last pass ran inside the expansion
    }
  }
  c.st.term_updates += p->ops_after_last_fan * c.N;
  // per-generator statistics
  auto* r = new (std::nothrow) qx_result;
  if (!r) return fail(QX_ENOMEM, "host allocation failed");
  r->n = c.n;
  r->W = W;
  r->wtb = int(sizeof(WT));
  r->G = c.G;
  r->count.assign(G, 0);
  r->sumsq.assign(G, 0.0);
  r->pruned.assign(G, 0.0);
  auto* d_count = c.sc.gcount;
  auto* d_sumsq = c.sc.gsumsq;
  if (!c.stats_done) {  // else the last expansion counted its children
    QX_TRY_CUDA(cudaMemsetAsync(d_count, 0, G * 16, c.al.s));
    c.begin(KC_STATS);
    if (c.N)
      k_gen_stats<W, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
          c.cur.view<WT>(), c.sc.ncnt + c.cslot, c.G, d_count, d_sumsq);
    c.end(KC_STATS, c.N ? 1 : 0, uint64_t(c.N) * 12);
  }
  // the counters (with the sticky error word), counts, sums of squares,
  // pruned mass and the used check slots: one copy
  constexpr size_t head = 256;  // the counters' block ahead of the statistics
  const size_t tail = head + ((G * 24 + 255) & ~size_t(255)) + size_t(c.chk_used) * c.chk_stride;
  std::vector<unsigned char> tail_host;
  auto* th = static_cast<unsigned char*>(rb_take(c, tail));
  if (!th) {
    tail_host.resize(tail);
    th = tail_host.data();
  }
  QX_TRY_CUDA(cudaMemcpyAsync(th, c.sc.base, tail, cudaMemcpyDeviceToHost, c.al.s));
  const cudaError_t se = cudaStreamSynchronize(c.al.s);
  c.st.host_syncs++;
  if (se != cudaSuccess) {
    delete r;
    return fail(QX_ECUDA, std::string("propagation failed: ") + cudaGetErrorString(se));
  }
  unsigned serr = 0;
  std::memcpy(&serr, th + (reinterpret_cast<unsigned char*>(c.sc.serr) -
                           static_cast<unsigned char*>(c.sc.base)),
              4);
  if (serr & kErrSpin) {
    delete r;
    return fail(QX_ETIMEOUT, "a bulk copy of the fused expansion did not complete");
  }
  std::memcpy(r->count.data(), th + head, G * 8);
  std::memcpy(r->sumsq.data(), th + head + G * 8, G * 8);
  std::memcpy(r->pruned.data(), th + head + G * 16, G * 8);
  for (Ctx::Deferred& d : c.deferred)
    if (d.kind == kHintReplay) {
      const unsigned char* slot =
          th + head + ((G * 24 + 255) & ~size_t(255)) + size_t(d.slot) * c.chk_stride;
      d.err = reinterpret_cast<const unsigned*>(slot);
      d.gwire = reinterpret_cast<const uint32_t*>(slot + 16);
    }
  // the checks of the steps launched on the plan's record without a read-back
  bool held = true;
  for (const Ctx::Deferred& d : c.deferred) {
    bool ok;
    if (d.kind == kHintExpand) {  // no merge wire, and the guessed size
      std::vector<unsigned long long> gmv(d.gm, d.gm + G * 3 * W);
      std::vector<uint64_t> mixed;
      std::vector<const FanQubit*> mq, fq;
      split_fan(c, *d.fs, gmv, &mixed, &mq, &fq);
      ok = mq.empty() && *d.total == d.expect;
    } else if (d.kind == kHintReplay) {  // every range as recorded, no merge wire
      ok = *d.err == 0;
      const size_t nq = d.fs->qs.size();
      for (size_t g = 0; ok && g < G; ++g)
        for (size_t j = 0; j < nq; ++j) {
          const uint32_t a = (d.gwire[g] >> (3 * j)) & 7u;
          if (a & (a - 1)) {  // two letters on a non-isolated row
            ok = false;
            break;
          }
        }
      if (!ok) d.rec->bad.store(1);
    } else {  // every block complete
      ok = *d.err == 0;
    }
    if (ok) {
      d.hint->streak.fetch_add(1, std::memory_order_relaxed);
      if (d.kind == kHintBlocks) d.hint->nblk.store(*d.nblk, std::memory_order_relaxed);
      c.st.guesses_held++;
    } else {
      d.hint->streak.store(0, std::memory_order_relaxed);
      d.hint->kind.store(kHintNone, std::memory_order_relaxed);
      held = false;
    }
  }
  if (!held) {  // the caller repeats the run, every step checked on the spot
    delete r;
    c.retry = true;
    return QX_OK;
  }
  publish_records(c);
  c.tm.resolve(&c.st);
  c.st.final_terms = c.N;
  c.st.K = p->K;
  c.st.Kp = p->Kp;
  r->N = c.N;
  r->buf = c.cur;
  c.cur = TermBuf();
  r->al = c.al;
  cudaGetDevice(&r->device);
  r->st = c.st;
  *out = r;
  return QX_OK;
}

// Records of a run that did not complete (its stream work is done).
void drop_records(Ctx& c) {
  for (const Ctx::Record& rc : c.records) {
    cudaFree(rc.offs);
    rc.rec->claim.store(0);
  }
  c.records.clear();
}

qx_status propagate_common(const qx_plan* p, const qx_prop_opts* o, int ngen, int gen_begin,
                           const uint64_t* ix, const uint64_t* iz, const double* iw,
                           qx_result** out, const qx_result* from = nullptr) {
  clear_error();
  cudaGetLastError();  // a stale error of an unrelated earlier call is not ours
  if (!p || !out) return fail(QX_EINVAL, "NULL argument");
  qx_prop_opts opts;
  qx_default_opts(&opts);
  if (o) opts = *o;
  if (opts.precision != 64 && opts.precision != 32)
    return fail(QX_EINVAL, "precision must be 64 or 32");
  if (!(opts.eps >= 0.0)) return fail(QX_EINVAL, "eps must be >= 0");
  if ((opts.alloc == nullptr) != (opts.free == nullptr))
    return fail(QX_EINVAL, "alloc and free must both be set or both be NULL");
  int dev = 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no CUDA device is available");
  }
  QX_TRY_CUDA(cudaGetDevice(&dev));
  set_pool_threshold();
  QX_TRY(ensure_plan_device(p, dev));
  Ctx c;
  c.p = p;
  c.n = p->n;
  c.W = p->W;
  c.G = ngen;
  c.sms = device_sms();
  c.wtb = opts.precision == 32 ? 4 : 8;
  c.eps = opts.eps;
  c.budget = opts.hbm_budget;
  c.max_terms = opts.max_terms;
  const unsigned ms = opts.timeout_ms ? opts.timeout_ms : 2000;
  // one spin iteration sleeps about 32 ns or more: bound the wait by the timeout
  c.spin_limit = std::max(1024u, std::min(ms, 60000u) * 16000u);
  c.al.a = opts.alloc;
  c.al.f = opts.free;
  c.al.ctx = opts.alloc_ctx;
  c.al.s = static_cast<cudaStream_t>(opts.stream);
  c.tm.on = (opts.flags & QX_FLAG_KERNEL_TIMING) != 0;
  c.inplace = (opts.flags & QX_FLAG_NO_INPLACE) == 0;
  c.tm.s = c.al.s;
  c.tm.pool = &t_event_pool;
  {  // kernels whose dynamic shared memory may pass 48 KB
    static thread_local int attr_dev = -1;
    if (attr_dev != dev) {
      const int mx = 200 * 1024;
      const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
      cudaFuncSetAttribute(k_clifford_table<1, 4, double>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<1, 3, double>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<2, 4, double>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<2, 3, double>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<1, 4, float>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<1, 3, float>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<2, 4, float>, attr, mx);
      cudaFuncSetAttribute(k_clifford_table<2, 3, float>, attr, mx);
      cudaFuncSetAttribute(k_expand_emit<1, double>, attr, mx);
      cudaFuncSetAttribute(k_expand_emit<2, double>, attr, mx);
      cudaFuncSetAttribute(k_expand_emit<1, float>, attr, mx);
      cudaFuncSetAttribute(k_expand_emit<2, float>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 0, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 0, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 0, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 1, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 1, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 1, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 3, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 3, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 3, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 4, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 4, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, double, 4, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 0, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 0, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 0, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 1, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 1, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 1, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 3, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 3, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 3, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 4, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 4, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<1, float, 4, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 0, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 0, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 0, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 1, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 1, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 1, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 3, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 3, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 3, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 4, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 4, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, double, 4, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 0, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 0, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 0, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 1, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 1, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 1, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 3, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 3, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 3, 2>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 4, 0>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 4, 1>, attr, mx);
      cudaFuncSetAttribute(k_xs_emit<2, float, 4, 2>, attr, mx);
      attr_dev = dev;
    }
  }
  qx_status s;
  if (from && (from->n != p->n || from->wtb != (opts.precision == 32 ? 4 : 8)))
    return fail(QX_EINVAL, "the initial state must have the plan's qubit count and precision");
  // Steps launched on the plan's record may leave their check to the end of
  // the run: without pruning, or when every fan-out step is small (the fused
  // expansion prunes as it writes; a separate compaction would read counts
  // mid-step).  A run whose deferred checks fail is repeated once with every
  // check on the spot.
  bool all_small = true;
  for (const FanStep& f : p->fans) all_small = all_small && small_fan_step(f);
  c.defer = opts.eps == 0.0 || (all_small && p->rots.empty());
  for (int attempt = 0; attempt < 2; ++attempt) {
    if (p->W == 1)
      s = opts.precision == 32 ? propagate_impl<1, float>(c, ix, iz, iw, gen_begin, from, out)
                               : propagate_impl<1, double>(c, ix, iz, iw, gen_begin, from, out);
    else
      s = opts.precision == 32 ? propagate_impl<2, float>(c, ix, iz, iw, gen_begin, from, out)
                               : propagate_impl<2, double>(c, ix, iz, iw, gen_begin, from, out);
    if (s != QX_OK || !c.retry) break;
    // release the first attempt's buffers (its stream work is complete)
    drop_records(c);
    const uint64_t missed = c.st.guesses_missed + c.deferred.size();
    c.al.put(c.cur.base);
    c.cur = TermBuf();
    free_scratch(c);
    c.st = qx_prop_stats{};
    c.st.guesses_missed = missed;
    c.tm.rec.clear();
    c.tm.used = 0;
    c.deferred.clear();
    c.rb_off = 0;
    c.stage_off = 0;
    c.N = 0;
    c.cslot = 0;
    c.retry = false;
    c.defer = false;
    c.stats_done = false;
  }
  if (s != QX_OK) {
    const std::string msg = qx_last_error();
    c.al.put(c.cur.base);
    free_scratch(c);
    cudaStreamSynchronize(c.al.s);
    cudaGetLastError();
    drop_records(c);
    release_table(c.ftab);
    fail(s, msg);
    return s;
  }
  free_scratch(c);
  release_table(c.ftab);
  return QX_OK;
}

// Canonical base-4 order: digit(q) = (x xor z) | z << 1 gives I=0, X=1, Y=2,
// Z=3; qubit 0 is the most significant digit (Example 1).
void sort_canonical(int n, int W, size_t cnt, const uint64_t* px, const uint64_t* pz,
                    std::vector<size_t>* order) {
  const int KW = (2 * n + 63) / 64;
  std::vector<uint64_t> keys(cnt * KW, 0);
  for (size_t i = 0; i < cnt; ++i) {
    uint64_t* k = &keys[i * KW];
    for (int q = 0; q < n; ++q) {
      const int xb = int((px[i * W + q / 64] >> (q % 64)) & 1);
      const int zb = int((pz[i * W + q / 64] >> (q % 64)) & 1);
      const uint64_t d = uint64_t((xb ^ zb) | (zb << 1));
      const int pos = 2 * (n - 1 - q);  // bit position from the least significant end
      const int word = KW - 1 - pos / 64;
      k[word] |= d << (pos % 64);
    }
  }
  order->resize(cnt);
  for (size_t i = 0; i < cnt; ++i) (*order)[i] = i;
  std::sort(order->begin(), order->end(), [&](size_t a, size_t b) {
    const uint64_t* ka = &keys[a * KW];
    const uint64_t* kb = &keys[b * KW];
    for (int w = 0; w < KW; ++w)
      if (ka[w] != kb[w]) return ka[w] < kb[w];
    return false;
  });
}

template <int W, typename WT>
qx_status export_impl(const qx_result* r, int gen, uint64_t* x, uint64_t* z, double* w,
                      size_t cap, int on_device) {
  Alloc al = r->al;
  const size_t cnt = r->count[gen];
  if (cap < cnt) return fail(QX_EINVAL, "cap is smaller than the generator's term count");
  if (cnt == 0) return QX_OK;
  TermBuf sel;
  QX_TRY(alloc_terms(al, W, int(sizeof(WT)), cnt, &sel));
  auto* nsel = static_cast<unsigned long long*>(al.get(8));
  if (!nsel) {
    al.put(sel.base);
    return fail(QX_ENOMEM, "device allocation failed");
  }
  cudaMemsetAsync(nsel, 0, 8, al.s);
  auto* nall = static_cast<unsigned long long*>(al.get(8));
  if (!nall) {
    al.put(sel.base);
    al.put(nsel);
    return fail(QX_ENOMEM, "device allocation failed");
  }
  const unsigned long long nn = r->N;
  cudaMemcpyAsync(nall, &nn, 8, cudaMemcpyHostToDevice, al.s);
  const int sms = device_sms();
  k_select<W, kThreads, WT><<<grid_for(r->N, kThreads, sms, 8), kThreads, 0, al.s>>>(
      r->buf.view<WT>(), nall, uint32_t(gen), sel.view<WT>(), nsel);
  std::vector<uint64_t> hx(cnt * W), hz(cnt * W), px(cnt * W), pz(cnt * W);
  std::vector<double> hw(cnt), pw(cnt);
  std::vector<WT> pwt(cnt);
  for (int k = 0; k < W; ++k) {
    cudaMemcpyAsync(px.data() + k * cnt, sel.x + k * sel.cap, cnt * 8, cudaMemcpyDeviceToHost,
                    al.s);
    cudaMemcpyAsync(pz.data() + k * cnt, sel.z + k * sel.cap, cnt * 8, cudaMemcpyDeviceToHost,
                    al.s);
  }
  cudaMemcpyAsync(pwt.data(), sel.w, cnt * sizeof(WT), cudaMemcpyDeviceToHost, al.s);
  const cudaError_t e = cudaStreamSynchronize(al.s);
  for (size_t i = 0; i < cnt; ++i) pw[i] = double(pwt[i]);
  al.put(sel.base);
  al.put(nsel);
  al.put(nall);
  if (e != cudaSuccess) return fail(QX_ECUDA, std::string("export failed: ") + cudaGetErrorString(e));
  // planar -> row-major, then canonical order
  std::vector<uint64_t> rx(cnt * W), rz(cnt * W);
  for (size_t i = 0; i < cnt; ++i)
    for (int k = 0; k < W; ++k) {
      rx[i * W + k] = px[k * cnt + i];
      rz[i * W + k] = pz[k * cnt + i];
    }
  std::vector<size_t> order;
  sort_canonical(r->n, W, cnt, rx.data(), rz.data(), &order);
  for (size_t i = 0; i < cnt; ++i) {
    const size_t j = order[i];
    for (int k = 0; k < W; ++k) {
      hx[i * W + k] = rx[j * W + k];
      hz[i * W + k] = rz[j * W + k];
    }
    hw[i] = pw[j];
  }
  if (on_device) {
    QX_TRY_CUDA(cudaMemcpyAsync(x, hx.data(), cnt * W * 8, cudaMemcpyHostToDevice, al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(z, hz.data(), cnt * W * 8, cudaMemcpyHostToDevice, al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(w, hw.data(), cnt * 8, cudaMemcpyHostToDevice, al.s));
    QX_TRY_CUDA(cudaStreamSynchronize(al.s));
  } else {
    std::memcpy(x, hx.data(), cnt * W * 8);
    std::memcpy(z, hz.data(), cnt * W * 8);
    std::memcpy(w, hw.data(), cnt * 8);
  }
  return QX_OK;
}

template <int W, typename WT>
qx_status ensure_index(qx_result* r) {
  if (r->index || r->N == 0) return QX_OK;
  Alloc al = r->al;
  const unsigned long long cap = std::max<unsigned long long>(64, 2ull * r->N);
  auto* tab = static_cast<IndexSlot*>(al.get(cap * sizeof(IndexSlot) + 16));
  if (!tab) return fail(QX_ENOMEM, "device allocation of the lookup index failed");
  unsigned* err = reinterpret_cast<unsigned*>(tab + cap);
  QX_TRY_CUDA(cudaMemsetAsync(tab, 0, cap * sizeof(IndexSlot) + 16, al.s));
  k_index_build<W, WT><<<grid_for(r->N, kThreads, device_sms(), 8), kThreads, 0, al.s>>>(
      r->buf.view<WT>(), r->N, tab, cap, err);
  unsigned e = 0;
  QX_TRY_CUDA(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, al.s));
  QX_TRY_CUDA(cudaStreamSynchronize(al.s));
  if (e) {
    al.put(tab);
    return fail(QX_ECAP, "lookup index ran out of probe slots");
  }
  r->index = tab;
  r->icap = cap;
  return QX_OK;
}

template <int W, typename WT>
qx_status coeff_impl(qx_result* r, size_t nq, const int32_t* gen, const uint64_t* x,
                     const uint64_t* z, double* out, int on_device) {
  for (size_t i = 0; !on_device && i < nq; ++i)
    if (gen[i] < 0 || gen[i] >= r->G) return fail(QX_EINVAL, "generator index out of range");
  if (r->N == 0) {
    if (on_device)
      QX_TRY_CUDA(cudaMemsetAsync(out, 0, nq * 8, r->al.s));
    else
      std::fill(out, out + nq, 0.0);
    return QX_OK;
  }
  QX_TRY(ensure_index<W, WT>(r));
  Alloc al = r->al;
  const int32_t* dg = gen;
  const uint64_t *dx = x, *dz = z;
  double* dout = out;
  void* tmp = nullptr;
  if (!on_device) {
    tmp = al.get(nq * (4 + 16 * W + 8) + 64);
    if (!tmp) return fail(QX_ENOMEM, "device allocation failed");
    auto* bx = static_cast<uint64_t*>(tmp);
    auto* bz = bx + nq * W;
    auto* bo = reinterpret_cast<double*>(bz + nq * W);
    auto* bg = reinterpret_cast<int32_t*>(bo + nq);
    QX_TRY_CUDA(cudaMemcpyAsync(bx, x, nq * W * 8, cudaMemcpyHostToDevice, al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(bz, z, nq * W * 8, cudaMemcpyHostToDevice, al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(bg, gen, nq * 4, cudaMemcpyHostToDevice, al.s));
    dg = bg;
    dx = bx;
    dz = bz;
    dout = bo;
  }
  if (nq)
    k_lookup<W, WT><<<grid_for(nq, kThreads, device_sms(), 8), kThreads, 0, al.s>>>(
        r->buf.view<WT>(), r->index, r->icap, nq, dg, dx, dz, dout);
  QX_TRY_CUDA(cudaGetLastError());
  if (!on_device) {
    QX_TRY_CUDA(cudaMemcpyAsync(out, dout, nq * 8, cudaMemcpyDeviceToHost, al.s));
    QX_TRY_CUDA(cudaStreamSynchronize(al.s));
    al.put(tmp);
  }
  return QX_OK;
}

// <M D, Lambda> for a batch of rotations (the adjoint of one U_k's wire): the
// smaller of the two states is iterated and the other is looked up through
// its hash index.
template <int W, typename WT>
qx_status adjoint_dot_impl(const qx_result* m, const qx_result* lam, const int32_t* lam_gen,
                           size_t nrot, const int32_t* qubit, const double* d9,
                           const uint64_t* px, const uint64_t* pz, double* out) {
  if (m->N == 0 || lam->N == 0) {
    std::fill(out, out + nrot, 0.0);
    return QX_OK;
  }
  bool iter_m = m->N <= lam->N;
  std::vector<int32_t> gmap;
  if (!iter_m) {  // pairing seen from lam; needs at most one m generator per lam generator
    gmap.assign(size_t(lam->G), -1);
    for (int g = 0; g < m->G && !iter_m; ++g) {
      const int32_t h = lam_gen[g];
      if (h < 0) continue;
      if (gmap[h] >= 0) iter_m = true;
      gmap[h] = g;
    }
  }
  if (iter_m) gmap.assign(lam_gen, lam_gen + m->G);
  const qx_result* A = iter_m ? m : lam;
  qx_result* B = const_cast<qx_result*>(iter_m ? lam : m);
  QX_TRY(ensure_index<W, WT>(B));  // built and synchronised on B's stream
  Alloc al = A->al;
  const int sms = device_sms();
  const unsigned grid = grid_for(A->N, kThreads, sms, 4);  // term tiles (grid x)
  const size_t chunk = std::min<size_t>(nrot, kAdjMaxRot);
  // rotation groups (grid y): enough blocks for 4 per SM when the iterated
  // side has few tiles, one group (every term read once) when it has many
  const size_t want_groups = (size_t(4) * sms + grid - 1) / grid;
  const size_t bytes = size_t(A->G) * 4 + chunk * sizeof(AdjRot) + size_t(grid) * chunk * 8 +
                       nrot * 8 + 256;
  void* tmp = al.get(bytes);
  if (!tmp) return fail(QX_ENOMEM, "device allocation for the adjoint product failed");
  auto* d_rot = static_cast<AdjRot*>(tmp);
  auto* d_part = reinterpret_cast<double*>(d_rot + chunk);
  auto* d_out = d_part + size_t(grid) * chunk;
  auto* d_gmap = reinterpret_cast<int32_t*>(d_out + nrot);
  qx_status st = QX_OK;
  auto body = [&]() -> qx_status {
    QX_TRY_CUDA(cudaMemcpyAsync(d_gmap, gmap.data(), size_t(A->G) * 4, cudaMemcpyHostToDevice, al.s));
    std::vector<AdjRot> hr(chunk);
    for (size_t r0 = 0; r0 < nrot; r0 += chunk) {
      const size_t cnt = std::min(chunk, nrot - r0);
      for (size_t r = 0; r < cnt; ++r) {
        hr[r] = AdjRot{};
        if (px) {  // Pauli rotations: Q -> sigma(Q) (Q xor P); its transpose
          hr[r].kind = 1;  // maps R to sigma(R xor P) (R xor P) = -sigma(R) (R xor P)
          for (int k = 0; k < W; ++k) {
            hr[r].px[k] = px[(r0 + r) * W + k];
            hr[r].pz[k] = pz[(r0 + r) * W + k];
          }
          hr[r].d[0][0] = iter_m ? 1.0 : -1.0;
          continue;
        }
        hr[r].q = qubit[r0 + r];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)  // iterating lam applies D^T
            hr[r].d[i][j] = iter_m ? d9[(r0 + r) * 9 + 3 * i + j] : d9[(r0 + r) * 9 + 3 * j + i];
      }
      QX_TRY_CUDA(cudaMemcpyAsync(d_rot, hr.data(), cnt * sizeof(AdjRot), cudaMemcpyHostToDevice, al.s));
      const size_t groups = std::max<size_t>(1, std::min(cnt, want_groups));
      const size_t rb = (cnt + groups - 1) / groups;
      const dim3 g2(grid, unsigned((cnt + rb - 1) / rb));
      const size_t smem = rb * (sizeof(AdjRot) + (kThreads / 32) * 8);
      k_adjoint_dot<W, WT><<<g2, kThreads, smem, al.s>>>(A->buf.view<WT>(), A->N, d_gmap,
                                                         B->buf.view<WT>(), B->index, B->icap,
                                                         d_rot, int(cnt), int(rb), d_part);
      k_adjoint_reduce<<<unsigned((cnt + 127) / 128), 128, 0, al.s>>>(d_part, int(grid), int(cnt),
                                                                     d_out + r0);
      QX_TRY_CUDA(cudaGetLastError());
    }
    QX_TRY_CUDA(cudaMemcpyAsync(out, d_out, nrot * 8, cudaMemcpyDeviceToHost, al.s));
    QX_TRY_CUDA(cudaStreamSynchronize(al.s));
    return QX_OK;
  };
  st = body();
  al.put(tmp);
  return st;
}


// ---------------------------------------------------------------------------
// Batched propagation of push-through plans (qx_batch.cuh): the serving loop.

// One rotation step of a batch: every term applies the step's rotation of its
// request (or passes unchanged), as run_rot does for one plan.
template <int W, typename WT>
qx_status run_brot(Ctx& c, const RotQ* rots, const int32_t* gen_req, const int32_t* rot_off,
                   const int32_t* nrot, int step) {
  const size_t N = c.N;
  if (N == 0) return QX_OK;
  const unsigned long long cap = std::max<unsigned long long>(64, 2ull * N);
  const size_t ntiles = (N + kScanTile - 1) / kScanTile;
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t tab_bytes = up(cap * sizeof(IndexSlot) + 16);
  void* mem = c.al.get(tab_bytes + up((N + ntiles + 1) * 8) + up(N * 8));
  if (!mem) return fail(QX_ENOMEM, "device allocation for a rotation step failed");
  auto* b8 = static_cast<unsigned char*>(mem);
  auto* tab = reinterpret_cast<IndexSlot*>(b8);
  auto* offs = reinterpret_cast<unsigned long long*>(b8 + tab_bytes);
  unsigned long long* tsum = offs + N;
  auto* pidx = reinterpret_cast<long long*>(b8 + tab_bytes + up((N + ntiles + 1) * 8));
  TermBuf out;
  auto body = [&]() -> qx_status {
    QX_TRY_CUDA(cudaMemsetAsync(tab, 0, cap * sizeof(IndexSlot), c.al.s));
    QX_TRY_CUDA(cudaMemsetAsync(c.sc.err, 0, 4, c.al.s));
    const unsigned grid = grid_for(N, kThreads, c.sms, 8);
    const auto view = c.cur.view<WT>();
    c.begin(KC_ROT);
    k_index_build<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, tab, cap, c.sc.err);
    k_brot_count<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, rots, gen_req, rot_off, nrot,
                                                        step, tab, cap, offs, pidx);
    k_scan_tiles<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(offs, c.sc.ncnt + c.cslot, tsum);
    k_scan_sums<<<1, 1024, 0, c.al.s>>>(tsum, ntiles, c.sc.ncnt + 2);
    k_scan_add<<<unsigned(ntiles), kScanThreads, 0, c.al.s>>>(offs, c.sc.ncnt + c.cslot, tsum);
    QX_TRY_CUDA(cudaGetLastError());
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    QX_TRY(sync_read(c, h, c.sc.ncnt, 40));
    if (unsigned(h[4]) & kErrProbe) return fail(QX_ECAP, "a hash table ran out of probe slots");
    const unsigned long long total = h[2];
    QX_TRY(check_limits(c, total));
    QX_TRY(alloc_terms(c.al, W, c.wtb, total, &out));
    k_brot_emit<W, WT><<<grid, kThreads, 0, c.al.s>>>(view, N, rots, gen_req, rot_off, nrot, step,
                                                       offs, pidx, out.view<WT>());
    c.end(KC_ROT, 6, (N + total) * (16 * W + sizeof(WT)));
    QX_TRY_CUDA(cudaGetLastError());
    const int oslot = 1 - c.cslot;
    QX_TRY(h2d(c, c.sc.ncnt + oslot, &total, 8));
    c.st.alg_bytes += (N + total) * (16 * W + sizeof(WT));
    c.st.children += total;
    replace_cur(c, out, total, oslot);
    out = TermBuf();
    return QX_OK;
  };
  const qx_status st = body();
  c.al.put(mem);
  if (st != QX_OK) {
    c.al.put(out.base);
    return st;
  }
  if (c.eps > 0.0) QX_TRY(prune_cur<W, WT>(c));
  return QX_OK;
}

template <int W, typename WT>
qx_status batch_impl(Ctx& c, std::vector<qx::BatchRequest>& reqs) {
  const size_t R = reqs.size();
  // host tables of the batch
  std::vector<int32_t> gen_req, rot_off(R), nrot(R);
  std::vector<uint32_t> gen_base(R);
  std::vector<RotQ> rots;
  std::vector<BatchPass> bps(R);
  std::vector<uint32_t> ops;
  std::vector<uint64_t> tabs;
  std::vector<uint8_t> tabe;
  int tmax = 0;
  uint32_t G = 0;
  for (size_t r = 0; r < R; ++r) {
    const qx_plan* p = reqs[r].plan;
    gen_base[r] = G;
    for (int j = 0; j < p->n; ++j) gen_req.push_back(int32_t(r));
    G += uint32_t(p->n);
    rot_off[r] = int32_t(rots.size());
    const CliffPass* last = nullptr;
    for (const Step& stp : p->program) {
      if (stp.kind == kStepRot) {
        if (last) return fail(QX_EINVAL, "a batched plan must end with its only Clifford pass");
        rots.push_back(to_dev(p->rots[size_t(stp.index)]));
      } else if (stp.kind == kStepCliff) {
        if (last) return fail(QX_EINVAL, "a batched plan has one Clifford pass");
        last = &p->passes[size_t(stp.index)];
      } else {
        return fail(QX_EINVAL, "a batched plan has no fan-out steps (push-through plans only)");
      }
    }
    nrot[r] = int32_t(rots.size()) - rot_off[r];
    tmax = std::max(tmax, int(nrot[r]));
    BatchPass& bp = bps[r];
    std::memset(&bp, 0, sizeof bp);
    if (!last || last->identity) {
      bp.kind = 0;
    } else if (!last->use_table) {
      bp.kind = 1;
      bp.ops_off = ops.size();
      bp.nops = int(last->ops.size());
      ops.insert(ops.end(), last->ops.begin(), last->ops.end());
    } else {
      bp.kind = 2;
      if (tabs.size() & 1) tabs.push_back(0);  // 16-byte entries
      bp.tab_off = tabs.size();
      bp.e_off = tabe.size();
      bp.chunks = last->chunks;
      tabs.insert(tabs.end(), last->tab_xz.begin(), last->tab_xz.end());
      tabe.insert(tabe.end(), last->tab_e.begin(), last->tab_e.end());
      qx_plan_device::Pass dp;
      dp.chunks = last->chunks;
      dp.cb = last->chunk_bits;
      pass_geometry(*last, p->n, &dp.live, dp.idle);
      bp.live = dp.live;
      bp.pmk = pass_masks<W>(dp, p->n);
    }
  }
  if (rots.empty()) rots.push_back(RotQ{});
  if (ops.empty()) ops.push_back(0);
  if (tabs.empty()) tabs.assign(2, 0);
  if (tabe.empty()) tabe.push_back(0);
  c.G = int(G);
  QX_TRY(setup_scratch(c));
  // one upload of every table
  auto up = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t o_req = 0, o_base = up(o_req + G * 4), o_roff = up(o_base + R * 4),
               o_nrot = up(o_roff + R * 4), o_rots = up(o_nrot + R * 4),
               o_bps = up(o_rots + rots.size() * sizeof(RotQ)),
               o_ops = up(o_bps + R * sizeof(BatchPass)), o_tab = up(o_ops + ops.size() * 4),
               o_e = up(o_tab + tabs.size() * 8), o_cur = up(o_e + tabe.size()),
               o_outs = up(o_cur + size_t(G) * 8), total = up(o_outs + R * sizeof(BatchOut<WT>));
  std::vector<unsigned char> host(total, 0);
  std::memcpy(&host[o_req], gen_req.data(), G * 4);
  std::memcpy(&host[o_base], gen_base.data(), R * 4);
  std::memcpy(&host[o_roff], rot_off.data(), R * 4);
  std::memcpy(&host[o_nrot], nrot.data(), R * 4);
  std::memcpy(&host[o_rots], rots.data(), rots.size() * sizeof(RotQ));
  std::memcpy(&host[o_bps], bps.data(), R * sizeof(BatchPass));
  std::memcpy(&host[o_ops], ops.data(), ops.size() * 4);
  std::memcpy(&host[o_tab], tabs.data(), tabs.size() * 8);
  std::memcpy(&host[o_e], tabe.data(), tabe.size());
  auto* dev = static_cast<unsigned char*>(c.al.get(total));
  if (!dev) return fail(QX_ENOMEM, "device allocation of the batch tables failed");
  struct Put {
    Alloc* al;
    void* p;
    ~Put() { al->put(p); }
  } put_dev{&c.al, dev};
  QX_TRY_CUDA(cudaMemcpyAsync(dev, host.data(), o_cur, cudaMemcpyHostToDevice, c.al.s));
  const auto* d_req = reinterpret_cast<const int32_t*>(dev + o_req);
  const auto* d_base = reinterpret_cast<const uint32_t*>(dev + o_base);
  const auto* d_roff = reinterpret_cast<const int32_t*>(dev + o_roff);
  const auto* d_nrot = reinterpret_cast<const int32_t*>(dev + o_nrot);
  const auto* d_rots = reinterpret_cast<const RotQ*>(dev + o_rots);
  const auto* d_bps = reinterpret_cast<const BatchPass*>(dev + o_bps);
  const auto* d_ops = reinterpret_cast<const uint32_t*>(dev + o_ops);
  const auto* d_tab = reinterpret_cast<const uint64_t*>(dev + o_tab);
  const auto* d_e = reinterpret_cast<const uint8_t*>(dev + o_e);
  auto* d_cur = reinterpret_cast<unsigned long long*>(dev + o_cur);
  auto* d_outs = reinterpret_cast<BatchOut<WT>*>(dev + o_outs);
  // A3: every request's generators; then the rotation steps and the passes
  QX_TRY(check_limits(c, G));
  QX_TRY(alloc_terms(c.al, W, c.wtb, G, &c.cur));
  c.N = G;
  c.cslot = 0;
  c.begin(KC_INIT);
  k_batch_init<W, WT><<<(G + 127) / 128, 128, 0, c.al.s>>>(c.cur.view<WT>(), d_req, d_base, G,
                                                           c.sc.ncnt);
  c.end(KC_INIT, 1, uint64_t(G) * (16 * W + sizeof(WT) + 4));
  QX_TRY_CUDA(cudaGetLastError());
  for (int t = 0; t < tmax; ++t) {
    c.st.fan_steps++;
    QX_TRY((run_brot<W, WT>(c, d_rots, d_req, d_roff, d_nrot, t)));
  }
  if (c.N) {
    c.begin(KC_CLIFF);
    constexpr int CB = W == 1 ? 4 : 3;
    k_batch_clifford<W, CB, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), c.sc.ncnt + c.cslot, d_req, d_bps, d_ops, d_tab, d_e);
    c.end(KC_CLIFF, 1, 2ull * c.N * (16 * W + sizeof(WT)));
    c.st.clifford_passes++;
    QX_TRY_CUDA(cudaGetLastError());
  }
  // per-generator counts and norms, then each request's own buffer
  std::vector<unsigned long long> cnt(G, 0);
  std::vector<double> sumsq(G, 0.0), pruned(G, 0.0);
  void* stb = c.al.get(size_t(G) * 16 + 16);
  if (!stb) return fail(QX_ENOMEM, "device allocation failed");
  struct Put put_stb{&c.al, stb};
  auto* d_count = static_cast<unsigned long long*>(stb);
  auto* d_sumsq = reinterpret_cast<double*>(d_count + G);
  QX_TRY_CUDA(cudaMemsetAsync(stb, 0, size_t(G) * 16, c.al.s));
  c.begin(KC_STATS);
  if (c.N)
    k_gen_stats<W, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), c.sc.ncnt + c.cslot, int(G), d_count, d_sumsq);
  c.end(KC_STATS, c.N ? 1 : 0, uint64_t(c.N) * 12);
  QX_TRY_CUDA(cudaMemcpyAsync(cnt.data(), d_count, G * 8, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaMemcpyAsync(sumsq.data(), d_sumsq, G * 8, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaMemcpyAsync(pruned.data(), c.sc.pruned, G * 8, cudaMemcpyDeviceToHost, c.al.s));
  QX_TRY_CUDA(cudaStreamSynchronize(c.al.s));
  c.st.host_syncs++;
  std::vector<TermBuf> bufs(R);
  std::vector<size_t> nres(R, 0);
  std::vector<unsigned long long> cursor(G);
  std::vector<BatchOut<WT>> outs(R);
  auto release = [&]() {
    for (TermBuf& b : bufs) c.al.put(b.base);
  };
  for (size_t r = 0; r < R; ++r) {
    const uint32_t b0 = gen_base[r], b1 = b0 + uint32_t(reqs[r].plan->n);
    size_t run = 0;
    for (uint32_t g = b0; g < b1; ++g) {
      cursor[g] = run;
      run += cnt[g];
    }
    nres[r] = run;
    if (alloc_terms(c.al, W, c.wtb, run, &bufs[r]) != QX_OK) {
      release();
      return fail(QX_ENOMEM, "device allocation of a request's result failed");
    }
    outs[r].t = bufs[r].view<WT>();
  }
  std::memcpy(&host[o_cur], cursor.data(), size_t(G) * 8);
  std::memcpy(&host[o_outs], outs.data(), R * sizeof(BatchOut<WT>));
  cudaError_t e = cudaMemcpyAsync(dev + o_cur, &host[o_cur], total - o_cur,
                                  cudaMemcpyHostToDevice, c.al.s);
  if (e == cudaSuccess && c.N) {
    k_batch_split<W, WT><<<grid_for(c.N, kThreads, c.sms, 8), kThreads, 0, c.al.s>>>(
        c.cur.view<WT>(), c.sc.ncnt + c.cslot, d_req, d_base, d_cur, d_outs);
    c.st.kernel_launches++;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.al.s);  // the host copy of the tables is read
  if (e != cudaSuccess) {
    release();
    return fail(QX_ECUDA, std::string("batched propagation failed: ") + cudaGetErrorString(e));
  }
  c.tm.resolve(&c.st);
  int device = 0;
  cudaGetDevice(&device);
  for (size_t r = 0; r < R; ++r) {
    auto* res = new (std::nothrow) qx_result;
    if (!res) {
      for (size_t k = 0; k < r; ++k) {
        qx_free_result(reqs[k].result);
        reqs[k].result = nullptr;
      }
      for (size_t k = r; k < R; ++k) c.al.put(bufs[k].base);
      return fail(QX_ENOMEM, "host allocation failed");
    }
    const int n = reqs[r].plan->n;
    const uint32_t b0 = gen_base[r];
    res->n = n;
    res->W = W;
    res->G = n;
    res->wtb = int(sizeof(WT));
    res->N = nres[r];
    res->buf = bufs[r];
    res->al = c.al;
    res->device = device;
    res->count.assign(cnt.begin() + b0, cnt.begin() + b0 + n);
    res->sumsq.assign(sumsq.begin() + b0, sumsq.begin() + b0 + n);
    res->pruned.assign(pruned.begin() + b0, pruned.begin() + b0 + n);
    res->st = c.st;  // the batch's counters
    res->st.final_terms = nres[r];
    reqs[r].result = res;
  }
  return QX_OK;
}

}  // namespace

namespace qx {
qx_status batch_propagate(std::vector<BatchRequest>& reqs, int precision, double eps,
                          size_t budget, void* stream) {
  clear_error();
  cudaGetLastError();
  if (reqs.empty()) return QX_OK;
  const int W = reqs[0].plan->W;
  for (const BatchRequest& b : reqs)
    if (!b.plan || b.plan->W != W) return fail(QX_EINVAL, "a batch needs plans of one word count");
  if (precision != 64 && precision != 32) return fail(QX_EINVAL, "precision must be 64 or 32");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no CUDA device is available");
  }
  set_pool_threshold();
  Ctx c;
  c.p = reqs[0].plan;
  c.n = 0;
  for (const BatchRequest& b : reqs) c.n = std::max(c.n, b.plan->n);
  c.W = W;
  c.sms = device_sms();
  c.wtb = precision == 32 ? 4 : 8;
  c.eps = eps;
  c.budget = budget;
  c.al.s = static_cast<cudaStream_t>(stream);
  c.tm.s = c.al.s;
  c.tm.pool = &t_event_pool;
  qx_status s;
  if (W == 1)
    s = precision == 32 ? batch_impl<1, float>(c, reqs) : batch_impl<1, double>(c, reqs);
  else
    s = precision == 32 ? batch_impl<2, float>(c, reqs) : batch_impl<2, double>(c, reqs);
  c.al.put(c.cur.base);
  c.cur = TermBuf();
  free_scratch(c);
  if (s != QX_OK) {
    const std::string msg = qx_last_error();
    cudaStreamSynchronize(c.al.s);
    cudaGetLastError();
    for (BatchRequest& b : reqs) {
      qx_free_result(b.result);
      b.result = nullptr;
    }
    return fail(s, msg);
  }
  return QX_OK;
}
}  // namespace qx

extern "C" {

qx_status qx_propagate(const qx_plan* p, const qx_prop_opts* o, qx_result** out) {
  if (!p) return fail(QX_EINVAL, "plan is NULL");
  qx_prop_opts opts;
  qx_default_opts(&opts);
  if (o) opts = *o;
  const int gb = opts.gen_begin, ge = opts.gen_end <= 0 ? p->n : opts.gen_end;
  if (gb < 0 || ge > p->n || gb >= ge) return fail(QX_EINVAL, "bad generator range");
  return propagate_common(p, &opts, ge - gb, gb, nullptr, nullptr, nullptr, out);
}

qx_status qx_propagate_from(const qx_plan* p, int ngen, const uint64_t* x, const uint64_t* z,
                            const double* w, const qx_prop_opts* o, qx_result** out) {
  if (!p) return fail(QX_EINVAL, "plan is NULL");
  if (ngen < 1 || !x || !z) return fail(QX_EINVAL, "need at least one initial generator");
  for (int i = 0; i < ngen; ++i)
    for (int k = 0; k < p->W; ++k) {
      const int hi = p->n - 64 * k;  // valid bits in word k
      const uint64_t mask = hi >= 64 ? ~0ull : ((1ull << hi) - 1);
      if ((x[size_t(i) * p->W + k] | z[size_t(i) * p->W + k]) & ~mask)
        return fail(QX_EINVAL, "initial string has bits beyond qubit n-1");
    }
  return propagate_common(p, o, ngen, 0, x, z, w, out);
}

qx_status qx_propagate_result(const qx_plan* p, const qx_result* from, const qx_prop_opts* o,
                              qx_result** out) {
  clear_error();
  if (!p || !from || !out) return fail(QX_EINVAL, "NULL argument");
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && dev != from->device)
    return fail(QX_EINVAL, "the initial state lives on another device");
  cudaGetLastError();
  return propagate_common(p, o, from->G, 0, nullptr, nullptr, nullptr, out, from);
}

qx_status qx_result_from_terms(int n, int ngen, size_t nterms, const uint64_t* x,
                               const uint64_t* z, const double* w, const int32_t* gen,
                               int precision, qx_result** out) {
  clear_error();
  cudaGetLastError();
  if (!out) return fail(QX_EINVAL, "out is NULL");
  if (n < 1) return fail(QX_EINVAL, "n must be >= 1");
  if (n > kMaxQubits) return fail(QX_EUNSUPPORTED, "n > 128 is not supported");
  if (ngen < 1) return fail(QX_EINVAL, "ngen must be >= 1");
  if (precision != 64 && precision != 32) return fail(QX_EINVAL, "precision must be 64 or 32");
  if (nterms && (!x || !z || !w || !gen)) return fail(QX_EINVAL, "NULL term array");
  if (nterms >= (size_t(1) << 32)) return fail(QX_EUNSUPPORTED, "too many terms");
  const int W = (n + 63) / 64;
  for (size_t i = 0; i < nterms; ++i) {
    if (gen[i] < 0 || gen[i] >= ngen) return fail(QX_EINVAL, "generator id out of range");
    for (int k = 0; k < W; ++k) {
      const int hi = n - 64 * k;
      const uint64_t mask = hi >= 64 ? ~0ull : ((1ull << hi) - 1);
      if ((x[i * W + k] | z[i * W + k]) & ~mask)
        return fail(QX_EINVAL, "string has bits beyond qubit n-1");
    }
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no CUDA device is available");
  }
  // sum repeated (generator, string) pairs
  std::vector<size_t> ord(nterms);
  for (size_t i = 0; i < nterms; ++i) ord[i] = i;
  auto key_less = [&](size_t a, size_t b) {
    if (gen[a] != gen[b]) return gen[a] < gen[b];
    for (int k = 0; k < W; ++k) {
      if (x[a * W + k] != x[b * W + k]) return x[a * W + k] < x[b * W + k];
      if (z[a * W + k] != z[b * W + k]) return z[a * W + k] < z[b * W + k];
    }
    return false;
  };
  std::stable_sort(ord.begin(), ord.end(), key_less);
  std::vector<size_t> keep;
  std::vector<double> sum;
  for (size_t a = 0; a < nterms;) {
    size_t b = a + 1;
    double v = w[ord[a]];
    while (b < nterms && !key_less(ord[a], ord[b])) v += w[ord[b++]];
    if (v != 0.0) {
      keep.push_back(ord[a]);
      sum.push_back(v);
    }
    a = b;
  }
  const size_t N = keep.size(), cap = std::max<size_t>(N, 1);
  const int wtb = precision == 32 ? 4 : 8;
  std::vector<uint64_t> px(size_t(W) * cap, 0), pz(size_t(W) * cap, 0);
  std::vector<uint32_t> pg(cap, 0);
  std::vector<double> pw(cap, 0.0);
  std::vector<float> pf(cap, 0.0f);
  auto* r = new (std::nothrow) qx_result;
  if (!r) return fail(QX_ENOMEM, "host allocation failed");
  r->n = n;
  r->W = W;
  r->G = ngen;
  r->wtb = wtb;
  r->count.assign(size_t(ngen), 0);
  r->sumsq.assign(size_t(ngen), 0.0);
  r->pruned.assign(size_t(ngen), 0.0);
  for (size_t i = 0; i < N; ++i) {
    for (int k = 0; k < W; ++k) {
      px[size_t(k) * cap + i] = x[keep[i] * W + k];
      pz[size_t(k) * cap + i] = z[keep[i] * W + k];
    }
    pg[i] = uint32_t(gen[keep[i]]);
    pw[i] = sum[i];
    pf[i] = float(sum[i]);
    const double stored = wtb == 4 ? double(pf[i]) : pw[i];
    r->count[pg[i]]++;
    r->sumsq[pg[i]] += stored * stored;
  }
  if (const qx_status e = alloc_terms(r->al, W, wtb, cap, &r->buf)) {
    delete r;
    return e;
  }
  auto upload = [&]() -> qx_status {
    QX_TRY_CUDA(cudaMemcpyAsync(r->buf.x, px.data(), px.size() * 8, cudaMemcpyHostToDevice, r->al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(r->buf.z, pz.data(), pz.size() * 8, cudaMemcpyHostToDevice, r->al.s));
    if (wtb == 4)
      QX_TRY_CUDA(cudaMemcpyAsync(r->buf.w, pf.data(), cap * 4, cudaMemcpyHostToDevice, r->al.s));
    else
      QX_TRY_CUDA(cudaMemcpyAsync(r->buf.w, pw.data(), cap * 8, cudaMemcpyHostToDevice, r->al.s));
    QX_TRY_CUDA(cudaMemcpyAsync(r->buf.g, pg.data(), cap * 4, cudaMemcpyHostToDevice, r->al.s));
    QX_TRY_CUDA(cudaStreamSynchronize(r->al.s));
    return QX_OK;
  };
  if (const qx_status e = upload()) {
    r->al.put(r->buf.base);
    delete r;
    return e;
  }
  r->N = N;
  cudaGetDevice(&r->device);
  r->st.final_terms = N;
  r->st.peak_terms = N;
  *out = r;
  return QX_OK;
}

qx_status qx_adjoint_dot(const qx_result* m, const qx_result* lam, const int32_t* lam_gen,
                         size_t nrot, const int32_t* qubit, const double* d9, double* out) {
  clear_error();
  cudaGetLastError();
  if (!m || !lam || !lam_gen) return fail(QX_EINVAL, "NULL argument");
  if (nrot && (!qubit || !d9 || !out)) return fail(QX_EINVAL, "NULL argument");
  if (m->n != lam->n || m->wtb != lam->wtb)
    return fail(QX_EINVAL, "the two states differ in qubit count or precision");
  for (int g = 0; g < m->G; ++g)
    if (lam_gen[g] < -1 || lam_gen[g] >= lam->G) return fail(QX_EINVAL, "lam_gen out of range");
  for (size_t r = 0; r < nrot; ++r)
    if (qubit[r] < 0 || qubit[r] >= m->n) return fail(QX_EINVAL, "qubit out of range");
  if (nrot == 0) return QX_OK;
  if (m->wtb == 4)
    return m->W == 1 ? adjoint_dot_impl<1, float>(m, lam, lam_gen, nrot, qubit, d9, nullptr, nullptr, out)
                     : adjoint_dot_impl<2, float>(m, lam, lam_gen, nrot, qubit, d9, nullptr, nullptr, out);
  return m->W == 1 ? adjoint_dot_impl<1, double>(m, lam, lam_gen, nrot, qubit, d9, nullptr, nullptr, out)
                   : adjoint_dot_impl<2, double>(m, lam, lam_gen, nrot, qubit, d9, nullptr, nullptr, out);
}

qx_status qx_adjoint_dot_pauli(const qx_result* m, const qx_result* lam, const int32_t* lam_gen,
                               size_t nrot, const uint64_t* px, const uint64_t* pz, double* out) {
  clear_error();
  cudaGetLastError();
  if (!m || !lam || !lam_gen) return fail(QX_EINVAL, "NULL argument");
  if (nrot && (!px || !pz || !out)) return fail(QX_EINVAL, "NULL argument");
  if (m->n != lam->n || m->wtb != lam->wtb)
    return fail(QX_EINVAL, "the two states differ in qubit count or precision");
  for (int g = 0; g < m->G; ++g)
    if (lam_gen[g] < -1 || lam_gen[g] >= lam->G) return fail(QX_EINVAL, "lam_gen out of range");
  for (size_t r = 0; r < nrot; ++r)
    for (int k = 0; k < m->W; ++k) {
      const int hi = m->n - 64 * k;
      const uint64_t mask = hi >= 64 ? ~0ull : ((1ull << hi) - 1);
      if ((px[r * m->W + k] | pz[r * m->W + k]) & ~mask)
        return fail(QX_EINVAL, "Pauli string has bits beyond qubit n-1");
    }
  if (nrot == 0) return QX_OK;
  if (m->wtb == 4)
    return m->W == 1 ? adjoint_dot_impl<1, float>(m, lam, lam_gen, nrot, nullptr, nullptr, px, pz, out)
                     : adjoint_dot_impl<2, float>(m, lam, lam_gen, nrot, nullptr, nullptr, px, pz, out);
  return m->W == 1 ? adjoint_dot_impl<1, double>(m, lam, lam_gen, nrot, nullptr, nullptr, px, pz, out)
                   : adjoint_dot_impl<2, double>(m, lam, lam_gen, nrot, nullptr, nullptr, px, pz, out);
}

qx_status qx_result_shape(const qx_result* r, int* ngen, int* nwords, size_t* nterms) {
  clear_error();
  if (!r) return fail(QX_EINVAL, "result is NULL");
  if (ngen) *ngen = r->G;
  if (nwords) *nwords = r->W;
  if (nterms) *nterms = r->N;
  return QX_OK;
}

qx_status qx_result_info(const qx_result* r, int gen, size_t* nterms, double* sumsq,
                         double* pruned_sumsq) {
  clear_error();
  if (!r) return fail(QX_EINVAL, "result is NULL");
  if (gen < 0 || gen >= r->G) return fail(QX_EINVAL, "generator index out of range");
  if (nterms) *nterms = r->count[gen];
  if (sumsq) *sumsq = r->sumsq[gen];
  if (pruned_sumsq) *pruned_sumsq = r->pruned[gen];
  return QX_OK;
}

qx_status qx_result_stats(const qx_result* r, qx_prop_stats* s) {
  clear_error();
  if (!r || !s) return fail(QX_EINVAL, "NULL argument");
  *s = r->st;
  return QX_OK;
}

qx_status qx_result_export(const qx_result* r, int gen, uint64_t* x, uint64_t* z, double* w,
                           size_t cap, int on_device) {
  clear_error();
  cudaGetLastError();
  if (!r) return fail(QX_EINVAL, "result is NULL");
  if (gen < 0 || gen >= r->G) return fail(QX_EINVAL, "generator index out of range");
  if (r->count[gen] && (!x || !z || !w)) return fail(QX_EINVAL, "NULL output buffer");
  if (r->wtb == 4)
    return r->W == 1 ? export_impl<1, float>(r, gen, x, z, w, cap, on_device)
                     : export_impl<2, float>(r, gen, x, z, w, cap, on_device);
  return r->W == 1 ? export_impl<1, double>(r, gen, x, z, w, cap, on_device)
                   : export_impl<2, double>(r, gen, x, z, w, cap, on_device);
}

qx_status qx_result_raw(const qx_result* r, uint64_t* x, uint64_t* z, double* w, int32_t* gen,
                        size_t cap) {
  clear_error();
  cudaGetLastError();
  if (!r) return fail(QX_EINVAL, "result is NULL");
  if (cap < r->N) return fail(QX_EINVAL, "cap is smaller than the result's term count");
  if (r->N == 0) return QX_OK;
  if (!x || !z || !w || !gen) return fail(QX_EINVAL, "NULL output buffer");
  const unsigned grid = grid_for(r->N, kThreads, device_sms(), 8);
  const auto s = r->al.s;
  if (r->W == 1 && r->wtb == 8)
    k_raw<1, double><<<grid, kThreads, 0, s>>>(r->buf.view<double>(), r->N, x, z, w, gen);
  else if (r->W == 1)
    k_raw<1, float><<<grid, kThreads, 0, s>>>(r->buf.view<float>(), r->N, x, z, w, gen);
  else if (r->wtb == 8)
    k_raw<2, double><<<grid, kThreads, 0, s>>>(r->buf.view<double>(), r->N, x, z, w, gen);
  else
    k_raw<2, float><<<grid, kThreads, 0, s>>>(r->buf.view<float>(), r->N, x, z, w, gen);
  QX_TRY_CUDA(cudaGetLastError());
  QX_TRY_CUDA(cudaStreamSynchronize(r->al.s));
  return QX_OK;
}

qx_status qx_coeff_batch(const qx_result* r, size_t nq, const int32_t* gen, const uint64_t* x,
                         const uint64_t* z, double* out, int on_device) {
  clear_error();
  cudaGetLastError();
  if (!r) return fail(QX_EINVAL, "result is NULL");
  if (nq && (!gen || !x || !z || !out)) return fail(QX_EINVAL, "NULL argument");
  auto* rr = const_cast<qx_result*>(r);
  if (r->wtb == 4)
    return r->W == 1 ? coeff_impl<1, float>(rr, nq, gen, x, z, out, on_device)
                     : coeff_impl<2, float>(rr, nq, gen, x, z, out, on_device);
  return r->W == 1 ? coeff_impl<1, double>(rr, nq, gen, x, z, out, on_device)
                   : coeff_impl<2, double>(rr, nq, gen, x, z, out, on_device);
}

qx_status qx_coeff(const qx_result* r, int gen, const uint64_t* x, const uint64_t* z, double* re,
                   double* im) {
  clear_error();
  if (!r || !x || !z || !re) return fail(QX_EINVAL, "NULL argument");
  const int32_t g = gen;
  double v = 0.0;
  QX_TRY(qx_coeff_batch(r, 1, &g, x, z, &v, 0));
  *re = v;
  if (im) *im = 0.0;
  return QX_OK;
}

qx_status qx_expval(const qx_plan* p, size_t nobs, const uint64_t* x, const uint64_t* z,
                    const qx_prop_opts* o, double* out) {
  clear_error();
  if (!p || !x || !z || !out) return fail(QX_EINVAL, "NULL argument");
  if (nobs == 0) return QX_OK;
  qx_circuit fwd;
  fwd.n = p->n;
  fwd.ins = p->ins;
  qx_circuit* inv = nullptr;
  QX_TRY(inverse_circuit(&fwd, &inv));
  qx_plan* ip = nullptr;
  const qx_status ps = build_plan(inv, &ip);
  qx_free_circuit(inv);
  if (ps != QX_OK) return ps;
  qx_prop_opts opts;
  qx_default_opts(&opts);
  if (o) opts = *o;
  qx_result* r = nullptr;
  qx_status s = qx_propagate_from(ip, int(nobs), x, z, nullptr, &opts, &r);
  if (s == QX_OK) {
    Alloc al = r->al;
    auto* d = static_cast<double*>(al.get(nobs * 8 + 8));
    auto* nd = reinterpret_cast<unsigned long long*>(d + nobs);
    if (!d) {
      s = fail(QX_ENOMEM, "device allocation failed");
    } else {
      const unsigned long long nn = r->N;
      cudaMemsetAsync(d, 0, nobs * 8, al.s);
      cudaMemcpyAsync(nd, &nn, 8, cudaMemcpyHostToDevice, al.s);
      if (r->N) {
        const unsigned zg = grid_for(r->N, kThreads, device_sms(), 8);
        if (r->W == 1 && r->wtb == 8)
          k_ztype_sum<1, double><<<zg, kThreads, 0, al.s>>>(r->buf.view<double>(), nd, d);
        else if (r->W == 1)
          k_ztype_sum<1, float><<<zg, kThreads, 0, al.s>>>(r->buf.view<float>(), nd, d);
        else if (r->wtb == 8)
          k_ztype_sum<2, double><<<zg, kThreads, 0, al.s>>>(r->buf.view<double>(), nd, d);
        else
          k_ztype_sum<2, float><<<zg, kThreads, 0, al.s>>>(r->buf.view<float>(), nd, d);
      }
      std::vector<double> h(nobs);
      cudaMemcpyAsync(h.data(), d, nobs * 8, cudaMemcpyDeviceToHost, al.s);
      const cudaError_t e = cudaStreamSynchronize(al.s);
      al.put(d);
      if (e != cudaSuccess)
        s = fail(QX_ECUDA, std::string("expval failed: ") + cudaGetErrorString(e));
      else
        std::memcpy(out, h.data(), nobs * 8);
    }
    qx_free_result(r);
  }
  qx_free_plan(ip);
  return s;
}

qx_status qx_reserve_device_memory(size_t bytes, void* stream) {
  clear_error();
  cudaGetLastError();
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no CUDA device is available");
  }
  set_pool_threshold();
  if (bytes == 0) return QX_OK;
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(QX_ENOMEM, "the device cannot reserve " + std::to_string(bytes) + " bytes");
  }
  QX_TRY_CUDA(cudaFreeAsync(p, s));  // back to the pool, which keeps it
  QX_TRY_CUDA(cudaStreamSynchronize(s));
  return QX_OK;
}

qx_status qx_wait_selftest(uint32_t timeout_ms, int publish) {
  clear_error();
  cudaGetLastError();
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return fail(QX_EUNSUPPORTED, "no CUDA device is available");
  }
  const unsigned ms = timeout_ms ? timeout_ms : 2000;
  const unsigned limit = std::max(1024u, std::min(ms, 60000u) * 16000u);
  unsigned* d = nullptr;
  QX_TRY_CUDA(cudaMalloc(&d, 8));
  unsigned h[2] = {0, 0};
  cudaError_t e = cudaMemset(d, 0, 8);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 64>>>(d, publish, limit, d + 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, 8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(QX_ECUDA, std::string("wait self-test: ") + cudaGetErrorString(e));
  if (h[1]) return fail(QX_ETIMEOUT, "a device-side wait gave up (no publish)");
  return QX_OK;
}

const char* qx_kernel_class_name(int k) {
  return (k >= 0 && k < QX_KC_COUNT) ? kKernelClassNames[k] : "";
}

void qx_free_result(qx_result* r) {
  if (!r) return;
  r->al.put(r->index);
  r->al.put(r->buf.base);
  delete r;
}

}  // extern "C"
