// Host planner of libqx: circuit validation, operator grouping (Sec. III.A),
// per-qubit Pauli image tables (Algorithm 1), and the device program of fused
// Clifford passes and fan-out steps.
//
// Built with -ffp-contract=off: the composed tables must be bit-reproducible,
// because their zero pattern decides which strings exist.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <system_error>
#include <thread>

#include "qx_common.h"

namespace qx {

namespace {
thread_local std::string g_last_error;
}

qx_status fail(qx_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

void clear_error() { g_last_error.clear(); }

namespace {

constexpr bool two_qubit(uint32_t g) {
  return g == QX_CX || g == QX_CZ || (g >= QX_SWAP && g <= QX_CP);
}

bool rotation_2q(uint32_t g) { return g >= QX_RXX && g <= QX_CP; }

// The two-qubit rotation gates as commuting Pauli rotations exp(-i phi P / 2),
// P given by its letters on (q0, q1) (0 = I, 1 = X, 2 = Y, 3 = Z).  With c the
// control: CR_s(t) = R_{s_t}(t/2) R_{Z_c s_t}(-t/2), and
// CP(t) = R_{Z_c}(t/2) R_{Z_t}(t/2) R_{Z_c Z_t}(-t/2) up to a global phase.
struct PauliRot2 {
  int l0, l1;
  double phi;
};
std::vector<PauliRot2> gate_rotations(const qx_instr& g) {
  const double t = g.theta;
  switch (g.gate) {
    case QX_RXX: return {{1, 1, t}};
    case QX_RYY: return {{2, 2, t}};
    case QX_RZZ: return {{3, 3, t}};
    case QX_CRX: return {{0, 1, t / 2}, {3, 1, -t / 2}};
    case QX_CRY: return {{0, 2, t / 2}, {3, 2, -t / 2}};
    case QX_CRZ: return {{0, 3, t / 2}, {3, 3, -t / 2}};
    case QX_CP: return {{3, 0, t / 2}, {0, 3, t / 2}, {3, 3, -t / 2}};
    default: return {};
  }
}

// Values within 2^-50 of 0 or +-1 are those values: the composition of gates
// that is exactly Clifford (k pi/2 rotations, T T = S) then stays exact.
double settle(double v) {
  const double tol = 0x1p-50;
  if (std::fabs(v) <= tol) return 0.0;
  if (std::fabs(std::fabs(v) - 1.0) <= tol) return v > 0 ? 1.0 : -1.0;
  return v;
}

// Signed permutations of (X, Y, Z) under P -> g P g^dagger for the Clifford
// one-qubit gates: image letter index and sign for each source letter.
struct SignedPerm {
  int to[3];
  int sign[3];
};

bool clifford_image(uint32_t g, SignedPerm* sp) {
  switch (g) {
    case QX_H: *sp = {{2, 1, 0}, {1, -1, 1}}; return true;
    case QX_S: *sp = {{1, 0, 2}, {1, -1, 1}}; return true;
    case QX_SDG: *sp = {{1, 0, 2}, {-1, 1, 1}}; return true;
    case QX_X: *sp = {{0, 1, 2}, {1, -1, -1}}; return true;
    case QX_Y: *sp = {{0, 1, 2}, {-1, 1, -1}}; return true;
    case QX_Z: *sp = {{0, 1, 2}, {-1, -1, 1}}; return true;
    case QX_SX: *sp = {{0, 2, 1}, {1, 1, -1}}; return true;
    case QX_SXDG: *sp = {{0, 2, 1}, {1, -1, 1}}; return true;
    default: return false;
  }
}

// Rotation about Pauli axis a by angle t (cosine c, sine s): the axis letter is
// fixed, and with (b, d) the two letters that follow a cyclically,
// b -> c b + s d and d -> c d - s b.
Table3 axis_rotation(int a, double c, double s) {
  Table3 t{};
  const int b = (a + 1) % 3, d = (a + 2) % 3;
  t.r[a][a] = 1.0;
  t.r[b][b] = c;
  t.r[b][d] = s;
  t.r[d][d] = c;
  t.r[d][b] = -s;
  return t;
}

Table3 gate_image(const qx_instr& g) {
  Table3 t{};
  SignedPerm sp;
  if (clifford_image(g.gate, &sp)) {
    for (int p = 0; p < 3; ++p) t.r[p][sp.to[p]] = double(sp.sign[p]);
    return t;
  }
  const double h = std::sqrt(0.5);
  switch (g.gate) {
    case QX_T: t = axis_rotation(2, h, h); break;
    case QX_TDG: t = axis_rotation(2, h, -h); break;
    case QX_RX: t = axis_rotation(0, std::cos(g.theta), std::sin(g.theta)); break;
    case QX_RY: t = axis_rotation(1, std::cos(g.theta), std::sin(g.theta)); break;
    case QX_RZ: t = axis_rotation(2, std::cos(g.theta), std::sin(g.theta)); break;
    default: break;
  }
  for (auto& row : t.r)
    for (double& v : row) v = settle(v);
  return t;
}

// Algorithm 1 for one wire: each of X, Y, Z is mapped through the gates of
// U_{k,j} in list order.  Row p of m holds the weights of the image of letter
// p so far; one step maps them through the next gate's table t.  The rows are
// settled after the last gate.
constexpr Table3 kIdentity3{{{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}, {0.0, 0.0, 1.0}}};

void compose_step(Table3& m, const Table3& t) {
  for (int p = 0; p < 3; ++p) {
    double nw[3];
    for (int c = 0; c < 3; ++c) {
      double acc = m.r[p][0] * t.r[0][c];
      acc += m.r[p][1] * t.r[1][c];
      acc += m.r[p][2] * t.r[2][c];
      nw[c] = acc;
    }
    std::memcpy(m.r[p], nw, sizeof nw);
  }
}

// compose_step with the table of a signed permutation (a Clifford gate):
// letter c goes to letter to[c] with sign sign[c].  The non-zero weights are
// those of compose_step bit for bit (a sum with one non-zero product and
// zeros); only the sign of a zero weight can differ, and settle() maps every
// zero to +0 before a table is used.
void compose_perm(Table3& m, const SignedPerm& sp) {
  for (int p = 0; p < 3; ++p) {
    double nw[3];
    for (int c = 0; c < 3; ++c) nw[sp.to[c]] = sp.sign[c] > 0 ? m.r[p][c] : -m.r[p][c];
    std::memcpy(m.r[p], nw, sizeof nw);
  }
}

// Algorithm 1 for the wires that the one-qubit operator ins[b .. e) touches
// (the others keep the identity table), gate by gate in list order: acc[q]
// is wire q's composed table, not yet settled, and touched lists the wires in
// increasing order.  seen is all zero on entry and on return.
void compose_run(const qx_instr* ins, size_t b, size_t e, std::vector<uint8_t>& seen,
                 std::vector<Table3>& acc, std::vector<int>& touched) {
  touched.clear();
  for (size_t i = b; i < e; ++i) {
    const int q = ins[i].q0;
    if (!seen[q]) {
      seen[q] = 1;
      touched.push_back(q);
      acc[q] = kIdentity3;
    }
    SignedPerm sp;
    if (clifford_image(ins[i].gate, &sp))
      compose_perm(acc[q], sp);
    else
      compose_step(acc[q], gate_image(ins[i]));
  }
  std::sort(touched.begin(), touched.end());
  for (const int q : touched) seen[q] = 0;
}

// A wire's composed table while every gate on it so far is a Clifford gate:
// letter p goes to letter to[p] with sign (-1)^neg[p].
struct WirePerm {
  uint8_t to[3], neg[3];
};

// The signed permutation of each one-qubit Clifford gate (clifford_image),
// from a table built once; ok is false for the other gates.
struct GatePerm {
  bool ok;
  uint8_t to[3], neg[3];
};

const GatePerm& gate_perm(uint32_t gate) {
  static const std::array<GatePerm, 32> table = [] {
    std::array<GatePerm, 32> t{};
    for (uint32_t g = 0; g < t.size(); ++g) {
      SignedPerm sp;
      if (!clifford_image(g, &sp)) continue;
      t[g].ok = true;
      for (int a = 0; a < 3; ++a) {
        t[g].to[a] = uint8_t(sp.to[a]);
        t[g].neg[a] = uint8_t(sp.sign[a] < 0);
      }
    }
    return t;
  }();
  static const GatePerm none{};
  return gate < table.size() ? table[gate] : none;
}

// The 3 x 3 table of a signed permutation (entries +-1 and +0).
Table3 perm_table(const WirePerm& w) {
  Table3 t{};
  for (int p = 0; p < 3; ++p) t.r[p][w.to[p]] = w.neg[p] ? -1.0 : 1.0;
  return t;
}

// The table of a wire as the plan holds it: every entry settled.
Table3 settled(const Table3& a) {
  Table3 t;
  for (int r = 0; r < 3; ++r)
    for (int col = 0; col < 3; ++col) t.r[r][col] = settle(a.r[r][col]);
  return t;
}

// d/dtheta of a rotation table (RX, RY, RZ): (c, s) -> (-s, c).
bool rotation_derivative(const qx_instr& g, Table3* out) {
  int a;
  switch (g.gate) {
    case QX_RX: a = 0; break;
    case QX_RY: a = 1; break;
    case QX_RZ: a = 2; break;
    default: return false;
  }
  *out = axis_rotation(a, -std::sin(g.theta), std::cos(g.theta));
  out->r[a][a] = 0.0;  // the axis letter is fixed: its row does not depend on theta
  return true;
}

Table3 mat_mul(const Table3& A, const Table3& B) {
  Table3 C{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += A.r[i][k] * B.r[k][j];
      C.r[i][j] = acc;
    }
  return C;
}

enum TableKind { kIdentity, kSignedPerm, kFanOut };

TableKind classify(const Table3& t, uint32_t* perm_code) {
  bool ident = true, perm = true;
  uint32_t code = 0;
  for (int p = 0; p < 3; ++p) {
    int nz = 0, at = -1;
    for (int c = 0; c < 3; ++c) {
      if (t.r[p][c] != 0.0) {
        ++nz;
        at = c;
      }
      if (t.r[p][c] != (p == c ? 1.0 : 0.0)) ident = false;
    }
    if (nz != 1 || std::fabs(t.r[p][at]) != 1.0) {
      perm = false;
    } else {
      code |= (uint32_t(at) | (t.r[p][at] < 0 ? 4u : 0u)) << (3 * p);
    }
  }
  if (ident) return kIdentity;
  if (perm) {
    *perm_code = code;
    return kSignedPerm;
  }
  return kFanOut;
}

FanQubit make_fan_qubit(int q, const Table3& t) {
  FanQubit f{};
  f.q = q;
  f.t = t;
  int colcount[3] = {0, 0, 0};
  for (int p = 0; p < 3; ++p)
    for (int c = 0; c < 3; ++c)
      if (t.r[p][c] != 0.0) colcount[c]++;
  for (int p = 0; p < 3; ++p) {
    f.nnz[p] = 0;
    for (int c = 0; c < 3; ++c)
      if (t.r[p][c] != 0.0) f.col[p][f.nnz[p]++] = uint8_t(c);
    f.iso[p] = f.nnz[p] == 1 && colcount[f.col[p][0]] == 1;
  }
  return f;
}

// --- Pauli helpers in XZ form: i^e X^x Z^z -----------------------------------

[[maybe_unused]] int popcount_words(const uint64_t* a, int W) {
  int s = 0;
  for (int k = 0; k < W; ++k) s += __builtin_popcountll(a[k]);
  return s;
}

// (e1, x1, z1) <- (e1, x1, z1) * (e2, x2, z2)
void xz_mul(int W, uint8_t* e1, uint64_t* x1, uint64_t* z1, uint8_t e2, const uint64_t* x2,
            const uint64_t* z2) {
  int anti = 0;
  for (int k = 0; k < W; ++k) anti += __builtin_popcountll(z1[k] & x2[k]);
  *e1 = uint8_t((*e1 + e2 + 2 * anti) & 3);
  for (int k = 0; k < W; ++k) {
    x1[k] ^= x2[k];
    z1[k] ^= z2[k];
  }
}

// Column-wise tableau: for each qubit column, the x and z bits of the 2n image
// rows (rows q < n: image of X_q; rows n + q: image of Z_q) plus a sign row.
struct ColumnTableau {
  int n, RW;
  std::vector<uint64_t> X, Z, S;  // X[q * RW + k]
  explicit ColumnTableau(int n_) : n(n_), RW((2 * n_ + 63) / 64) {
    X.assign(size_t(n) * RW, 0);
    Z.assign(size_t(n) * RW, 0);
    S.assign(RW, 0);
    for (int q = 0; q < n; ++q) {
      X[size_t(q) * RW + q / 64] |= 1ull << (q % 64);
      Z[size_t(q) * RW + (n + q) / 64] |= 1ull << ((n + q) % 64);
    }
  }
  // Applies the pass's ops in order.  RW <= 4 (n <= 128), so the word loops
  // unroll, and the sign row stays in registers for the whole pass.
  void apply_all(const std::vector<uint32_t>& ops) {
    switch (RW) {
      case 1: run<1>(ops); break;
      case 2: run<2>(ops); break;
      case 3: run<3>(ops); break;
      default: run<4>(ops); break;
    }
  }

  template <int R>
  void run(const std::vector<uint32_t>& ops) {
    uint64_t s[R];
    for (int k = 0; k < R; ++k) s[k] = S[k];
    uint64_t *xs = X.data(), *zs = Z.data();
    for (const uint32_t op : ops) {
      const uint32_t kind = op & 3, a = (op >> 2) & 127, b = (op >> 9) & 127, perm = op >> 16;
      uint64_t *xa = xs + size_t(a) * R, *za = zs + size_t(a) * R;
      if (kind == kOpCX) {
        uint64_t *xb = xs + size_t(b) * R, *zb = zs + size_t(b) * R;
        for (int k = 0; k < R; ++k) {
          s[k] ^= xa[k] & zb[k] & ~(xb[k] ^ za[k]);
          xb[k] ^= xa[k];
          za[k] ^= zb[k];
        }
      } else if (kind == kOpCZ) {
        uint64_t *xb = xs + size_t(b) * R, *zb = zs + size_t(b) * R;
        for (int k = 0; k < R; ++k) {
          s[k] ^= xa[k] & xb[k] & (za[k] ^ zb[k]);
          zb[k] ^= xa[k];
          za[k] ^= xb[k];
        }
      } else {
        // per source letter p (X, Y, Z): all-ones masks for the image's x
        // bit, z bit and sign, decoded once for the whole column
        uint64_t tx[3], tz[3], ts[3];
        for (int p = 0; p < 3; ++p) {
          const uint32_t f = (perm >> (3 * p)) & 7, to = f & 3;
          tx[p] = to <= 1 ? ~0ull : 0;
          tz[p] = to >= 1 ? ~0ull : 0;
          ts[p] = (f & 4) ? ~0ull : 0;
        }
        for (int k = 0; k < R; ++k) {
          const uint64_t m0 = xa[k] & ~za[k], m1 = xa[k] & za[k], m2 = ~xa[k] & za[k];
          xa[k] = (m0 & tx[0]) | (m1 & tx[1]) | (m2 & tx[2]);
          za[k] = (m0 & tz[0]) | (m1 & tz[1]) | (m2 & tz[2]);
          s[k] ^= (m0 & ts[0]) | (m1 & ts[1]) | (m2 & ts[2]);
        }
      }
    }
    for (int k = 0; k < R; ++k) S[k] = s[k];
  }
};

// In-place transpose of a 64 x 64 bit matrix held as 64 rows (bit j of a[i]
// is entry (i, j)): swap the off-diagonal blocks of 32, then of 16, ... 1.
void transpose64(uint64_t* a) {
  uint64_t m = 0x00000000FFFFFFFFull;
  for (int j = 32; j != 0; j >>= 1, m ^= (m << j)) {
    for (int k = 0; k < 64; k = ((k | j) + 1) & ~j) {
      const uint64_t t = ((a[k] >> j) ^ a[k | j]) & m;
      a[k] ^= t << j;
      a[k | j] ^= t;
    }
  }
}

void build_pass_tables(CliffPass& pc, int n, int W) {
  uint64_t sup[2] = {0, 0};
  for (const uint32_t op : pc.ops) {
    const int q0 = int((op >> 2) & 127), q1 = int((op >> 9) & 127);
    sup[q0 >> 6] |= 1ull << (q0 & 63);
    if ((op & 3) != kOpPerm) sup[q1 >> 6] |= 1ull << (q1 & 63);
  }
  pc.support[0] = sup[0];
  pc.support[1] = sup[1];
  ColumnTableau tab(n);
  tab.apply_all(pc.ops);
  pc.img_x.assign(size_t(2 * n) * W, 0);
  pc.img_z.assign(size_t(2 * n) * W, 0);
  pc.img_e.assign(2 * n, 0);
  // rows of the image from the tableau's columns, 64 x 64 bit blocks at a
  // time (row bits of the columns past 2n and columns past n are zero)
  uint64_t blk[64];
  for (int side = 0; side < 2; ++side) {
    const std::vector<uint64_t>& col = side ? tab.Z : tab.X;
    std::vector<uint64_t>& img = side ? pc.img_z : pc.img_x;
    for (int k = 0; k < tab.RW; ++k)
      for (int w = 0; w < W; ++w) {
        for (int i = 0; i < 64; ++i) {
          const int q = 64 * w + i;
          blk[i] = q < n ? col[size_t(q) * tab.RW + k] : 0;
        }
        transpose64(blk);
        for (int i = 0; i < 64 && 64 * k + i < 2 * n; ++i) img[size_t(64 * k + i) * W + w] = blk[i];
      }
  }
  bool ident = true;
  for (int r = 0; r < 2 * n; ++r) {
    const uint64_t* xr = &pc.img_x[size_t(r) * W];
    const uint64_t* zr = &pc.img_z[size_t(r) * W];
    // Hermitian image (-1)^s H(x, z) = (-1)^s i^{|x & z|} X^x Z^z in XZ form
    const int s = int((tab.S[r / 64] >> (r % 64)) & 1);
    int xz = 0;
    for (int k = 0; k < W; ++k) xz += __builtin_popcountll(xr[k] & zr[k]);
    pc.img_e[r] = uint8_t((2 * s + xz) & 3);
    // identity check: row q is X_q, row n + q is Z_q, no sign
    const int q = r < n ? r : r - n;
    for (int k = 0; k < W; ++k) {
      const uint64_t want = (k == q / 64) ? (1ull << (q % 64)) : 0;
      if (xr[k] != (r < n ? want : 0) || zr[k] != (r < n ? 0 : want)) ident = false;
    }
    if (s) ident = false;
  }
  pc.identity = ident;
  pc.chunk_bits = (W == 1) ? 4 : 3;
  pc.chunks = (n + pc.chunk_bits - 1) / pc.chunk_bits;
  pc.use_table = !ident && pc.ops.size() > size_t(pc.chunks);
  if (!pc.use_table) return;
  const int cb = pc.chunk_bits, E = 1 << (2 * cb);
  pc.tab_xz.assign(size_t(pc.chunks) * E * 2 * W, 0);
  pc.tab_e.assign(size_t(pc.chunks) * E, 0);
  for (int c = 0; c < pc.chunks; ++c) {
    for (int idx = 1; idx < E; ++idx) {
      // last factor in the order X (ascending qubit) then Z (ascending qubit)
      const int xb = idx & ((1 << cb) - 1), zb = idx >> cb;
      int bit, row;
      if (zb) {
        bit = 31 - __builtin_clz(unsigned(zb));
        row = n + c * cb + bit;
      } else {
        bit = 31 - __builtin_clz(unsigned(xb));
        row = c * cb + bit;
      }
      const int prev = zb ? (idx & ~(1 << (cb + bit))) : (idx & ~(1 << bit));
      const int q = c * cb + bit;
      uint64_t* dst = &pc.tab_xz[(size_t(c) * E + idx) * 2 * W];
      const uint64_t* src = &pc.tab_xz[(size_t(c) * E + prev) * 2 * W];
      uint8_t e = pc.tab_e[size_t(c) * E + prev];
      std::memcpy(dst, src, sizeof(uint64_t) * 2 * W);
      if (q < n) xz_mul(W, &e, dst, dst + W, pc.img_e[row], &pc.img_x[size_t(row) * W],
                        &pc.img_z[size_t(row) * W]);
      pc.tab_e[size_t(c) * E + idx] = e;
    }
  }
}

// The tables of every pass of a plan.  Passes are independent, so a plan
// with many Clifford gates builds them on several threads (one pass per task;
// the tables do not depend on the split).  Plans under 2 x kOpsPerThread ops
// stay on the calling thread.
constexpr size_t kOpsPerThread = 10000;

void build_all_pass_tables(std::vector<CliffPass>& passes, int n, int W) {
  size_t ops = 0;
  for (const CliffPass& pc : passes) ops += pc.ops.size();
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min({passes.size(), hw, size_t(8), ops / kOpsPerThread});
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i = next.fetch_add(1); i < passes.size(); i = next.fetch_add(1))
      build_pass_tables(passes[i], n, W);
  };
  std::vector<std::thread> pool;
  try {
    for (size_t t = 1; t < nt; ++t) pool.emplace_back(work);
  } catch (const std::system_error&) {
    // no more threads: the ones started and this one share the passes
  }
  work();
  for (std::thread& t : pool) t.join();
}

}  // namespace

void host_apply_pass(const CliffPass& pc, int n, int W, uint64_t* x, uint64_t* z, int* sign) {
  if (pc.identity) return;
  if (pc.use_table) {
    const int cb = pc.chunk_bits, E = 1 << (2 * cb);
    int xzc = 0;
    for (int k = 0; k < W; ++k) xzc += __builtin_popcountll(x[k] & z[k]);
    uint8_t e = uint8_t(xzc & 3);
    uint64_t ax[kMaxWords] = {0, 0}, az[kMaxWords] = {0, 0};
    for (int c = 0; c < pc.chunks; ++c) {
      const int lo = c * cb, k = lo / 64, off = lo % 64;
      const uint32_t m = (1u << cb) - 1;
      uint64_t xs = x[k] >> off, zs = z[k] >> off;
      if (off + cb > 64 && k + 1 < W) {  // chunk straddles two words
        xs |= x[k + 1] << (64 - off);
        zs |= z[k + 1] << (64 - off);
      }
      const uint32_t xb = uint32_t(xs) & m, zb = uint32_t(zs) & m;
      const int idx = int(xb | (zb << cb));
      if (!idx) continue;
      const uint64_t* t = &pc.tab_xz[(size_t(c) * E + idx) * 2 * W];
      xz_mul(W, &e, ax, az, pc.tab_e[size_t(c) * E + idx], t, t + W);
    }
    int c2 = 0;
    for (int k = 0; k < W; ++k) c2 += __builtin_popcountll(ax[k] & az[k]);
    const int d = (e - c2) & 3;
    if (d == 2) *sign = -*sign;
    for (int k = 0; k < W; ++k) {
      x[k] = ax[k];
      z[k] = az[k];
    }
    return;
  }
  auto bit = [](const uint64_t* v, int q) { return int((v[q / 64] >> (q % 64)) & 1); };
  auto put = [](uint64_t* v, int q, int b) {
    v[q / 64] = (v[q / 64] & ~(1ull << (q % 64))) | (uint64_t(b) << (q % 64));
  };
  for (uint32_t op : pc.ops) {
    const uint32_t kind = op & 3;
    const int a = (op >> 2) & 127, b = (op >> 9) & 127;
    const uint32_t perm = op >> 16;
    if (kind == kOpCX) {
      const int xa = bit(x, a), za = bit(z, a), xb = bit(x, b), zb = bit(z, b);
      if (xa & zb & (1 ^ xb ^ za)) *sign = -*sign;
      put(x, b, xb ^ xa);
      put(z, a, za ^ zb);
    } else if (kind == kOpCZ) {
      const int xa = bit(x, a), za = bit(z, a), xb = bit(x, b), zb = bit(z, b);
      if (xa & xb & (za ^ zb)) *sign = -*sign;
      put(z, b, zb ^ xa);
      put(z, a, za ^ xb);
    } else {
      const int xq = bit(x, a), zq = bit(z, a);
      if (!xq && !zq) continue;
      const int p = xq ? (zq ? 1 : 0) : 2;
      const uint32_t f = (perm >> (3 * p)) & 7, to = f & 3;
      put(x, a, to <= 1);
      put(z, a, to >= 1);
      if (f & 4) *sign = -*sign;
    }
  }
  (void)n;
}

// Rotation step of exp(-i phi P / 2) for P given by letters l0 on wire q0 and
// l1 on wire q1 (0 = I), with sign +1.
RotStep make_rot(int n, int q0, int l0, int q1, int l1, double phi) {
  (void)n;
  RotStep r{};
  auto put = [&](int q, int l) {
    if (l == 0) return;
    const uint64_t m = 1ull << (q % 64);
    if (l == 1 || l == 2) r.px[q / 64] |= m;
    if (l == 2 || l == 3) r.pz[q / 64] |= m;
  };
  put(q0, l0);
  put(q1, l1);
  r.c = settle(std::cos(phi));
  r.s = settle(std::sin(phi));
  return r;
}

// Pauli in XZ form i^e X^x Z^z (W words).
struct PauliXZ {
  uint8_t e = 0;
  uint64_t x[kMaxWords] = {0, 0}, z[kMaxWords] = {0, 0};
};

PauliXZ xz_product(int W, const PauliXZ& a, const PauliXZ& b) {
  PauliXZ r = a;
  xz_mul(W, &r.e, r.x, r.z, b.e, b.x, b.z);
  return r;
}

// b <- a b (the product with a on the left, in place)
void xz_mul_left(int W, const PauliXZ& a, PauliXZ& b) {
  int anti = 0;
  for (int k = 0; k < W; ++k) anti += __builtin_popcountll(a.z[k] & b.x[k]);
  b.e = uint8_t((a.e + b.e + 2 * anti) & 3);
  for (int k = 0; k < W; ++k) {
    b.x[k] ^= a.x[k];
    b.z[k] ^= a.z[k];
  }
}

// One-qubit Clifford gate g for the push-through plan: its pass op code and
// the images of X and Z under g^dagger s g (letter 1 X, 2 Y, 3 Z, and sign).
struct PushPerm {
  bool clifford = false;
  uint32_t code = 0;
  int lx = 1, lz = 3;
  bool negx = false, negz = false;
};

const PushPerm& push_perm(uint32_t gate) {
  static const std::array<PushPerm, 32> table = [] {
    std::array<PushPerm, 32> t{};
    for (uint32_t g = 0; g < t.size(); ++g) {
      SignedPerm sp, inv;
      if (!clifford_image(g, &sp)) continue;
      PushPerm& pp = t[g];
      pp.clifford = true;
      for (int a = 0; a < 3; ++a)
        pp.code |= (uint32_t(sp.to[a]) | (sp.sign[a] < 0 ? 4u : 0u)) << (3 * a);
      const uint32_t ig = g == QX_S ? QX_SDG : g == QX_SDG ? QX_S
                        : g == QX_SX ? QX_SXDG : g == QX_SXDG ? QX_SX : g;
      clifford_image(ig, &inv);
      pp.lx = inv.to[0] + 1;
      pp.lz = inv.to[2] + 1;
      pp.negx = inv.sign[0] < 0;
      pp.negz = inv.sign[2] < 0;
    }
    return t;
  }();
  static const PushPerm none{};
  return gate < table.size() ? table[gate] : none;
}

// Rotation step for exp(-i phi P / 2) with P given in XZ form: the Hermitian
// string with P's bits and the sign i^(e - |x & z|) (folded into phi).
RotStep rot_from_xz(int W, const PauliXZ& P, double phi) {
  RotStep r{};
  int overlap = 0;
  for (int k = 0; k < W; ++k) {
    r.px[k] = P.x[k];
    r.pz[k] = P.z[k];
    overlap += __builtin_popcountll(P.x[k] & P.z[k]);
  }
  const int ph = ((int(P.e) - overlap) % 4 + 4) % 4;  // 0: +P, 2: -P
  const double sphi = ph == 0 ? phi : -phi;
  r.c = settle(std::cos(sphi));
  r.s = settle(std::sin(sphi));
  return r;
}

qx_status build_plan_pushthrough(const qx_circuit* c, qx_plan** out) {
  return build_plan_pushthrough(c->n, std::vector<qx_instr>(c->ins), out);
}

qx_status build_plan_pushthrough(int n, std::vector<qx_instr>&& ins, qx_plan** out) {
  auto* p = new (std::nothrow) qx_plan;
  if (!p) return fail(QX_ENOMEM, "host allocation failed");
  const int W = (n + 63) / 64;
  p->n = n;
  p->W = W;
  p->ins = std::move(ins);
  const std::vector<qx_instr>& cins = p->ins;
  // M(s) = D^dagger s D for the Clifford prefix D, kept as the images of X_q
  // and Z_q; after a Clifford gate g, M'(s) = M(g^dagger s g).
  std::vector<PauliXZ> MX(n), MZ(n);
  for (int q = 0; q < n; ++q) {
    MX[q].x[q / 64] = 1ull << (q % 64);
    MZ[q].z[q / 64] = 1ull << (q % 64);
  }
  auto image = [&](int q, int l) {  // M of the letter l (1 X, 2 Y, 3 Z) on wire q
    if (l == 1) return MX[q];
    if (l == 3) return MZ[q];
    PauliXZ y = xz_product(W, MX[q], MZ[q]);  // Y = i X Z
    y.e = uint8_t((y.e + 1) & 3);
    return y;
  };
  auto add_rot = [&](const PauliXZ& P, double phi) {
    p->rots.push_back(rot_from_xz(W, P, phi));
    p->program.push_back({kStepRot, int(p->rots.size() - 1), 0});
  };
  CliffPass all;  // every Clifford gate, in circuit order
  for (const qx_instr& g : cins) {
    switch (g.gate) {
      case QX_RX:
      case QX_RY:
      case QX_RZ:
        add_rot(image(g.q0, int(g.gate - QX_RX) + 1), g.theta);
        continue;
      case QX_T:
      case QX_TDG:
        add_rot(image(g.q0, 3), g.gate == QX_T ? std::atan(1.0) : -std::atan(1.0));
        continue;
      case QX_CX: {  // M'(X_a) = M(X_a) M(X_b), M'(Z_b) = M(Z_a) M(Z_b)
        all.ops.push_back(encode_op(kOpCX, g.q0, g.q1, 0));
        PauliXZ &xa = MX[g.q0], &xb = MX[g.q1];
        xz_mul(W, &xa.e, xa.x, xa.z, xb.e, xb.x, xb.z);
        xz_mul_left(W, MZ[g.q0], MZ[g.q1]);
        continue;
      }
      case QX_CZ: {  // M'(X_a) = M(X_a) M(Z_b), M'(X_b) = M(Z_a) M(X_b)
        all.ops.push_back(encode_op(kOpCZ, g.q0, g.q1, 0));
        PauliXZ& xa = MX[g.q0];
        const PauliXZ& zb = MZ[g.q1];
        xz_mul(W, &xa.e, xa.x, xa.z, zb.e, zb.x, zb.z);
        xz_mul_left(W, MZ[g.q0], MX[g.q1]);
        continue;
      }
      case QX_SWAP:
        all.ops.push_back(encode_op(kOpCX, g.q0, g.q1, 0));
        all.ops.push_back(encode_op(kOpCX, g.q1, g.q0, 0));
        all.ops.push_back(encode_op(kOpCX, g.q0, g.q1, 0));
        std::swap(MX[g.q0], MX[g.q1]);
        std::swap(MZ[g.q0], MZ[g.q1]);
        continue;
      default:
        break;
    }
    if (rotation_2q(g.gate)) {
      for (const PauliRot2& r : gate_rotations(g)) {
        PauliXZ P;
        if (r.l0) P = image(g.q0, r.l0);
        if (r.l1) P = r.l0 ? xz_product(W, P, image(g.q1, r.l1)) : image(g.q1, r.l1);
        add_rot(P, r.phi);
      }
      continue;
    }
    const PushPerm& pp = push_perm(g.gate);
    if (!pp.clifford) return fail(QX_EINVAL, "internal error: unknown gate");
    all.ops.push_back(encode_op(kOpPerm, g.q0, -1, pp.code));
    // images under the inverse gate (g^dagger s g)
    if (pp.lx != 1 || pp.lz != 3) {
      const PauliXZ nx = image(g.q0, pp.lx), nz = image(g.q0, pp.lz);
      MX[g.q0] = nx;
      MZ[g.q0] = nz;
    }
    if (pp.negx) MX[g.q0].e = uint8_t((MX[g.q0].e + 2) & 3);
    if (pp.negz) MZ[g.q0].e = uint8_t((MZ[g.q0].e + 2) & 3);
  }
  p->passes.push_back(std::move(all));
  p->program.push_back({kStepCliff, int(p->passes.size() - 1), 0});
  for (auto& pc : p->passes) build_pass_tables(pc, n, W);
  *out = p;
  return QX_OK;
}

std::vector<RotTerm> gate_rotation_terms(const qx_instr& g) {
  // the factors do not depend on theta: read them off theta = 1
  qx_instr one = g;
  one.theta = 1.0;
  std::vector<RotTerm> out;
  for (const PauliRot2& r : gate_rotations(one)) {
    const RotStep s = make_rot(0, g.q0, r.l0, g.q1, r.l1, 0.0);
    RotTerm t{};
    for (int k = 0; k < kMaxWords; ++k) {
      t.px[k] = s.px[k];
      t.pz[k] = s.pz[k];
    }
    t.a = r.phi;
    out.push_back(t);
  }
  return out;
}

// When the program ends [pass a, fan step f, pass b] and both passes act on
// other qubits than f's wires, the three commute into (b a) then f: the
// composed pass lets f's expansion apply both to each parent once instead of
// b to every child afterwards.
void add_pre_tail_pass(qx_plan* p) {
  const auto& prog = p->program;
  const size_t m = prog.size();
  if (m < 3 || prog[m - 1].kind != kStepCliff || prog[m - 2].kind != kStepFan ||
      prog[m - 3].kind != kStepCliff)
    return;
  const CliffPass& a = p->passes[size_t(prog[m - 3].index)];
  const CliffPass& b = p->passes[size_t(prog[m - 1].index)];
  FanStep& f = p->fans[size_t(prog[m - 2].index)];
  if (a.identity || b.identity || !pass_disjoint(a, f) || !pass_disjoint(b, f)) return;
  CliffPass ab;
  ab.ops = a.ops;
  ab.ops.insert(ab.ops.end(), b.ops.begin(), b.ops.end());
  build_pass_tables(ab, p->n, p->W);
  p->aux_passes.push_back(std::move(ab));
  f.pre_tail = int(p->aux_passes.size() - 1);
}

qx_status build_plan(const qx_circuit* c, qx_plan** out) {
  auto* p = new (std::nothrow) qx_plan;
  if (!p) return fail(QX_ENOMEM, "host allocation failed");
  const int n = c->n;
  p->n = n;
  p->W = (n + 63) / 64;
  p->ins = c->ins;
  // divide_instruction: maximal runs of one-qubit / two-qubit instructions;
  // operator k is ins[op_begin[k] .. op_begin[k + 1]).
  for (size_t i = 0; i < c->ins.size(); ++i) {
    const bool one = !two_qubit(c->ins[i].gate);
    if (p->op_kind.empty() || (p->op_kind.back() == 1) != one) {
      p->op_begin.push_back(i);
      p->op_kind.push_back(one ? 1 : 0);
    }
  }
  p->op_begin.push_back(c->ins.size());
  CliffPass cur;
  uint64_t ops_since_fan = 0;
  // per wire of the current U_k: 0 untouched, 1 a signed permutation so far
  // (wp), 2 a 3 x 3 table (acc)
  std::vector<uint8_t> state(static_cast<size_t>(n), 0);
  std::vector<WirePerm> wp(static_cast<size_t>(n));
  std::vector<Table3> acc(static_cast<size_t>(n));
  std::vector<int> touched;
  for (size_t k = 0; k < p->op_kind.size(); ++k) {
    const size_t b = p->op_begin[k], e = p->op_begin[k + 1];
    if (p->op_kind[k] == 0) {
      ++p->Kp;
      for (size_t i = b; i < e; ++i) {
        const qx_instr& g = c->ins[i];
        if (g.gate == QX_CX || g.gate == QX_CZ) {
          cur.ops.push_back(encode_op(g.gate == QX_CX ? kOpCX : kOpCZ, g.q0, g.q1, 0));
        } else if (g.gate == QX_SWAP) {
          cur.ops.push_back(encode_op(kOpCX, g.q0, g.q1, 0));
          cur.ops.push_back(encode_op(kOpCX, g.q1, g.q0, 0));
          cur.ops.push_back(encode_op(kOpCX, g.q0, g.q1, 0));
        } else {
          // a two-qubit rotation: the Clifford gates so far run first, then
          // its Pauli rotations as their own steps
          p->passes.push_back(std::move(cur));
          cur = CliffPass();
          p->program.push_back({kStepCliff, int(p->passes.size() - 1), 0});
          for (const PauliRot2& r : gate_rotations(g)) {
            p->rots.push_back(make_rot(n, g.q0, r.l0, g.q1, r.l1, r.phi));
            p->program.push_back({kStepRot, int(p->rots.size() - 1), ops_since_fan});
            ops_since_fan = 0;
          }
        }
      }
      ++ops_since_fan;
      continue;
    }
    ++p->K;
    // Algorithm 1 for the wires this run touches, gate by gate in list
    // order.  A wire stays a signed permutation (integers) while its gates
    // are Clifford gates, and becomes a 3 x 3 table at its first other gate.
    // The settled tables are those of compose_run: the permutation's entries
    // are exact, and only signs of zeros can differ, which settle() clears.
    touched.clear();
    for (size_t i = b; i < e; ++i) {
      const qx_instr& g = c->ins[i];
      const int q = g.q0;
      if (!state[q]) {
        state[q] = 1;
        touched.push_back(q);
        wp[q] = WirePerm{{0, 1, 2}, {0, 0, 0}};
      }
      const GatePerm& gp = gate_perm(g.gate);
      if (state[q] == 1 && gp.ok) {
        WirePerm& w = wp[q];
        for (int a = 0; a < 3; ++a) {
          const int from = w.to[a];
          w.to[a] = gp.to[from];
          w.neg[a] ^= gp.neg[from];
        }
        continue;
      }
      if (state[q] == 1) {
        acc[q] = perm_table(wp[q]);
        state[q] = 2;
      }
      SignedPerm sp;
      if (clifford_image(g.gate, &sp))
        compose_perm(acc[q], sp);
      else
        compose_step(acc[q], gate_image(g));
    }
    std::sort(touched.begin(), touched.end());
    FanStep fs;
    fs.op_index = k;
    for (const int j : touched) {
      if (state[j] == 1) {  // a signed permutation: the pass before the step
        state[j] = 0;
        const WirePerm& w = wp[j];
        uint32_t code = 0;
        bool ident = true;
        for (int a = 0; a < 3; ++a) {
          code |= (uint32_t(w.to[a]) | (w.neg[a] ? 4u : 0u)) << (3 * a);
          ident = ident && w.to[a] == a && !w.neg[a];
        }
        if (!ident) cur.ops.push_back(encode_op(kOpPerm, j, -1, code));
        continue;
      }
      state[j] = 0;
      const Table3 t = settled(acc[j]);
      uint32_t code = 0;
      const TableKind kind = classify(t, &code);
      if (kind == kSignedPerm)
        cur.ops.push_back(encode_op(kOpPerm, j, -1, code));
      else if (kind == kFanOut)
        fs.qs.push_back(make_fan_qubit(j, t));
    }
    if (fs.qs.empty()) {
      ++ops_since_fan;
      continue;
    }
    // The Clifford wires of this U_k act on other qubits than its fan-out
    // wires, so they commute and run in the pass before the expansion.
    p->passes.push_back(std::move(cur));
    cur = CliffPass();
    p->program.push_back({kStepCliff, int(p->passes.size() - 1), 0});
    p->fans.push_back(std::move(fs));
    p->program.push_back({kStepFan, int(p->fans.size() - 1), ops_since_fan});
    ops_since_fan = 0;
  }
  p->passes.push_back(std::move(cur));
  p->program.push_back({kStepCliff, int(p->passes.size() - 1), 0});
  p->ops_after_last_fan = ops_since_fan;
  build_all_pass_tables(p->passes, n, p->W);
  add_pre_tail_pass(p);
  *out = p;
  return QX_OK;
}

qx_status inverse_circuit(const qx_circuit* c, qx_circuit** out) {
  auto* r = new (std::nothrow) qx_circuit;
  if (!r) return fail(QX_ENOMEM, "host allocation failed");
  r->n = c->n;
  r->ins.assign(c->ins.rbegin(), c->ins.rend());
  for (auto& g : r->ins) {
    switch (g.gate) {
      case QX_S: g.gate = QX_SDG; break;
      case QX_SDG: g.gate = QX_S; break;
      case QX_SX: g.gate = QX_SXDG; break;
      case QX_SXDG: g.gate = QX_SX; break;
      case QX_T: g.gate = QX_TDG; break;
      case QX_TDG: g.gate = QX_T; break;
      case QX_RX:
      case QX_RY:
      case QX_RZ:
      case QX_RXX:
      case QX_RYY:
      case QX_RZZ:
      case QX_CRX:
      case QX_CRY:
      case QX_CRZ:
      case QX_CP: g.theta = -g.theta; break;
      default: break;
    }
  }
  *out = r;
  return QX_OK;
}

qx_status validate_instrs(int n, const qx_instr* ins, size_t m) {
  if (n < 1) return fail(QX_EINVAL, "n must be >= 1");
  if (n > kMaxQubits) return fail(QX_EUNSUPPORTED, "n > 128 is not supported");
  if (m && !ins) return fail(QX_EINVAL, "ins is NULL");
  // One pass without branches finds whether anything is wrong; only then
  // does the loop below look for the first bad instruction and its message.
  constexpr uint32_t kTwo = [] {
    uint32_t mask = 0;
    for (uint32_t g = 0; g < 32; ++g)
      if (two_qubit(g)) mask |= 1u << g;
    return mask;
  }();
  bool bad = false;
  for (size_t i = 0; i < m; ++i) {
    const qx_instr& g = ins[i];
    const bool two = g.gate < 32 && ((kTwo >> g.gate) & 1u);
    bad |= g.gate > QX_CP;
    bad |= uint32_t(g.q0) >= uint32_t(n);
    bad |= two & ((uint32_t(g.q1) >= uint32_t(n)) | (g.q1 == g.q0));
    bad |= !std::isfinite(g.theta);
  }
  for (size_t i = 0; bad && i < m; ++i) {
    const qx_instr& g = ins[i];
    if (g.gate == QX_U4)
      return fail(QX_EINVAL, "instruction " + std::to_string(i) +
                                 ": U4 needs its matrix (qx_load_circuit_u4)");
    if (g.gate > QX_CP) return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": bad gate");
    if (g.q0 < 0 || g.q0 >= n)
      return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": wire out of range");
    if (two_qubit(g.gate) && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0))
      return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": bad second wire");
    if (!std::isfinite(g.theta))
      return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": theta not finite");
  }
  return QX_OK;
}

}  // namespace qx

using namespace qx;

extern "C" {

void qx_default_opts(qx_prop_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = 64;
  o->eps = 0.0;
  o->gen_begin = 0;
  o->gen_end = 0;
  o->timeout_ms = 2000;
}

qx_status qx_load_circuit(int n, const qx_instr* ins, size_t m, qx_circuit** out) {
  clear_error();
  if (!out) return fail(QX_EINVAL, "out is NULL");
  if (const qx_status st = validate_instrs(n, ins, m)) return st;
  auto* c = new (std::nothrow) qx_circuit;
  if (!c) return fail(QX_ENOMEM, "host allocation failed");
  c->n = n;
  c->ins.assign(ins, ins + m);
  *out = c;
  return QX_OK;
}

qx_status qx_load_circuit_u4(int n, const qx_instr* ins, size_t m, const double* mats,
                             size_t nmats, qx_circuit** out) {
  clear_error();
  if (!out) return fail(QX_EINVAL, "out is NULL");
  if (m && !ins) return fail(QX_EINVAL, "ins is NULL");
  if (nmats && !mats) return fail(QX_EINVAL, "mats is NULL");
  // each U4 becomes its decomposition (15 gates); the others are copied
  std::vector<qx_instr> all;
  all.reserve(m);
  for (size_t i = 0; i < m; ++i) {
    const qx_instr& g = ins[i];
    if (g.gate != QX_U4) {
      all.push_back(g);
      continue;
    }
    if (g.q0 < 0 || g.q0 >= n || g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)
      return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": bad U4 wires");
    const double k = g.theta;
    if (!(k >= 0.0) || k != std::floor(k) || k >= double(nmats))
      return fail(QX_EINVAL, "instruction " + std::to_string(i) + ": U4 matrix index out of range");
    std::vector<qx_instr> gs;
    if (const qx_status st = decompose_u4(mats + size_t(k) * 32, g.q0, g.q1, &gs, nullptr)) {
      const std::string msg = qx_last_error();
      return fail(st, "instruction " + std::to_string(i) + ": " + msg);
    }
    all.insert(all.end(), gs.begin(), gs.end());
  }
  return qx_load_circuit(n, all.data(), all.size(), out);
}

qx_status qx_group_ops(const qx_circuit* c, qx_plan** out) {
  clear_error();
  if (!c || !out) return fail(QX_EINVAL, "NULL argument");
  return build_plan(c, out);
}

qx_status qx_group_ops_dag(const qx_circuit* c, qx_plan** out) {
  clear_error();
  if (!c || !out) return fail(QX_EINVAL, "NULL argument");
  // Operators U_0 V_1 U_1 V_2 ...: every gate gets the earliest operator that
  // keeps the order of the gates on each of its wires.  A one-qubit gate may
  // share U_u with earlier one-qubit gates of its wire and follows its wire's
  // last V; a two-qubit gate may share V_v with earlier two-qubit gates of its
  // wires (applied in input order) and follows their last U.  These are the
  // least indices satisfying the per-wire order, so the operator count is at
  // most that of list-order grouping.
  const size_t m = c->ins.size();
  std::vector<long> last_u(size_t(c->n), -1), last_v(size_t(c->n), 0);
  std::vector<size_t> slot(m);  // U_u -> 2u, V_v -> 2v - 1
  size_t top = 0;
  for (size_t i = 0; i < m; ++i) {
    const qx_instr& g = c->ins[i];
    if (two_qubit(g.gate)) {
      const long v = std::max({1L, last_v[g.q0], last_v[g.q1], last_u[g.q0] + 1, last_u[g.q1] + 1});
      last_v[g.q0] = last_v[g.q1] = v;
      slot[i] = size_t(2 * v - 1);
    } else {
      const long u = std::max({0L, last_u[g.q0], last_v[g.q0]});
      last_u[g.q0] = u;
      slot[i] = size_t(2 * u);
    }
    top = std::max(top, slot[i]);
  }
  // Emission slot by slot, input order within a slot.  A gate moves only past
  // gates on other wires, so the circuit is unchanged.
  std::vector<size_t> start(top + 2, 0);
  for (size_t i = 0; i < m; ++i) start[slot[i] + 1]++;
  for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
  qx_circuit rc;
  rc.n = c->n;
  rc.ins.resize(m);
  std::vector<size_t> order(m);
  for (size_t i = 0; i < m; ++i) {
    const size_t k = start[slot[i]]++;
    rc.ins[k] = c->ins[i];
    order[k] = i;
  }
  qx_plan* p = nullptr;
  const qx_status s = build_plan(&rc, &p);
  if (s != QX_OK) return s;
  p->order = std::move(order);
  *out = p;
  return QX_OK;
}

qx_status qx_group_ops_pushthrough(const qx_circuit* c, qx_plan** out) {
  clear_error();
  if (!c || !out) return fail(QX_EINVAL, "NULL argument");
  return build_plan_pushthrough(c, out);
}

qx_status qx_plan_order(const qx_plan* p, size_t* m, size_t* order) {
  clear_error();
  if (!p || !m) return fail(QX_EINVAL, "NULL argument");
  *m = p->ins.size();
  if (order)
    for (size_t k = 0; k < p->ins.size(); ++k) order[k] = p->order.empty() ? k : p->order[k];
  return QX_OK;
}

qx_status qx_plan_info(const qx_plan* p, size_t* K, size_t* Kp) {
  clear_error();
  if (!p) return fail(QX_EINVAL, "plan is NULL");
  if (K) *K = p->K;
  if (Kp) *Kp = p->Kp;
  return QX_OK;
}

qx_status qx_plan_op(const qx_plan* p, size_t op, int* kind) {
  clear_error();
  if (!p || !kind) return fail(QX_EINVAL, "NULL argument");
  if (op >= p->op_kind.size()) return fail(QX_EINVAL, "operator index out of range");
  *kind = p->op_kind[op];
  return QX_OK;
}

qx_status qx_plan_lut(const qx_plan* p, size_t op, double* out) {
  clear_error();
  if (!p || !out) return fail(QX_EINVAL, "NULL argument");
  if (op >= p->op_kind.size() || p->op_kind[op] != 1)
    return fail(QX_EINVAL, "operator is not a one-qubit operator");
  for (int j = 0; j < p->n; ++j)
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) out[9 * j + 3 * a + c] = kIdentity3.r[a][c];
  std::vector<uint8_t> seen(size_t(p->n), 0);
  std::vector<Table3> acc(size_t(p->n));
  std::vector<int> touched;
  compose_run(p->ins.data(), p->op_begin[op], p->op_begin[op + 1], seen, acc, touched);
  for (const int j : touched) {
    const Table3 t = settled(acc[j]);
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) out[9 * j + 3 * a + c] = t.r[a][c];
  }
  return QX_OK;
}

qx_status qx_plan_clifford_passes(const qx_plan* p, size_t* count) {
  clear_error();
  if (!p || !count) return fail(QX_EINVAL, "NULL argument");
  *count = p->passes.size();
  return QX_OK;
}

qx_status qx_plan_clifford_apply(const qx_plan* p, size_t pass, uint64_t* x, uint64_t* z,
                                 int* sign) {
  clear_error();
  if (!p || !x || !z || !sign) return fail(QX_EINVAL, "NULL argument");
  if (pass >= p->passes.size()) return fail(QX_EINVAL, "pass index out of range");
  host_apply_pass(p->passes[pass], p->n, p->W, x, z, sign);
  return QX_OK;
}

qx_status qx_plan_derivative(const qx_plan* p, size_t instr, double* d9, int* qubit,
                             size_t* op_end) {
  clear_error();
  if (!p || !d9) return fail(QX_EINVAL, "NULL argument");
  if (instr >= p->ins.size()) return fail(QX_EINVAL, "instruction index out of range");
  const qx_instr& gi = p->ins[instr];
  Table3 dgi;
  if (!rotation_derivative(gi, &dgi)) return fail(QX_EINVAL, "instruction is not RX, RY or RZ");
  // the one-qubit operator (maximal run of one-qubit gates) holding it
  size_t b = instr, e = instr + 1;
  while (b > 0 && !two_qubit(p->ins[b - 1].gate)) --b;
  while (e < p->ins.size() && !two_qubit(p->ins[e].gate)) ++e;
  // T = G_1 ... G_m on this wire (row-vector composition, Algorithm 1) and
  // its derivative with G_i replaced by dG_i/dtheta
  Table3 T{}, dT{};
  for (int a = 0; a < 3; ++a) T.r[a][a] = dT.r[a][a] = 1.0;
  bool seen = false;
  for (size_t k = b; k < e; ++k) {
    const qx_instr& g = p->ins[k];
    if (g.q0 != gi.q0) continue;
    const Table3 G = gate_image(g);
    T = mat_mul(T, G);
    dT = mat_mul(dT, k == instr ? dgi : G);
    seen |= k == instr;
  }
  if (!seen) return fail(QX_EINVAL, "internal error: gate not found in its operator");
  // D = T^T dT acts on the operator's output: v dT = (v T)(T^T dT)
  Table3 Tt{};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Tt.r[i][j] = T.r[j][i];
  const Table3 D = mat_mul(Tt, dT);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) d9[3 * i + j] = D.r[i][j];
  if (qubit) *qubit = gi.q0;
  if (op_end) *op_end = e;
  return QX_OK;
}

void qx_free_circuit(qx_circuit* c) { delete c; }

void qx_free_plan(qx_plan* p) {
  if (!p) return;
  free_plan_device(p);
  delete p;
}

const char* qx_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
