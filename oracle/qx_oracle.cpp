// Reference oracle for extended-stabilizer Pauli propagation (Qimax, arXiv 2505.03307).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow CPU statement of what
// the propagation computes.  Only the test suite, the smoke check and the
// bench's CPU-baseline leg may load it; the CUDA library never does, and the
// two share no code, headers or tables.
//
// Representation: a generator is a std::map from a Pauli string to a complex
// weight.  A string is a std::string of the letters I, X, Y, Z with character i
// describing qubit i; this is the order of Example 1 (Sec. III.B), and the
// lexicographic order of std::map on these letters equals the base-4 index
// order I=0, X=1, Y=2, Z=3 with qubit 0 as the most significant digit.
//
// What is computed, for a circuit g_0 ... g_{m-1} on n qubits and each
// generator j:   U Z_j U^dagger = sum_P c_j(P) P   (Eq. 1 with P^(0) = Z_j,
// Sec. II.A; a gate acts as g P g^dagger, Sec. II.C).
//
// Two modes:
//  * gate mode: every gate in list order replaces each (P, w) by the image of P
//    under that gate (one-qubit gates: 3x3 image table; CX: the rule list of
//    Sec. III.C) and accumulates into a fresh map.
//  * plan mode: the paper's operator-level method.  The instruction list is cut
//    into maximal runs of one-qubit gates (operators U_k) and of two-qubit
//    gates (operators V_k) (Sec. III.A); each U_k gets the K x n x 3 x 3 table of
//    Algorithm 1 and is applied by sub + flatten (Algorithm 2, Eq. 3); each V_k
//    applies its two-qubit gates one after another (map_2q, Algorithm 2).
//
// Readings where the paper is silent (each is also listed in the design notes):
//  * rotations are exp(-i theta sigma / 2); T = diag(1, e^{i pi/4}); S = diag(1, i);
//    SX = sqrt(X).  T's table uses sqrt(1/2) for both entries.
//  * table entries within 2^-50 of 0 are set to 0 and entries within 2^-50 of
//    +-1 are set to +-1, for gate tables and for the composed tables of
//    Algorithm 1, so that k pi/2 rotations compose to exact signed permutations.
//  * pruning (the paper has none): eps = 0 keeps every key, including keys whose
//    weight cancels to 0; eps > 0 drops |w| < eps after every U_k (plan mode) or
//    after every gate (gate mode).
//  * CZ acts as H(t) CX(c,t) H(t).
//
// Parity status: pinned (dense brute force for n <= 10, CHP tableau for
// Clifford circuits, Example 1, the CX rule list, closed forms of the gate images
// and of the fan-in workloads).
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -shared -fPIC -pthread
#include <algorithm>
#include <array>
#include <deque>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <vector>

namespace {

using cplx = std::complex<double>;
using PauliSum = std::map<std::string, cplx>;
using Table = std::array<std::array<double, 3>, 3>;  // T[p][c]: coefficient of c in g p g^dagger

// Gate codes of this file (the Python wrapper maps names onto them).
enum Gate {
  G_H = 0, G_S, G_SDG, G_X, G_Y, G_Z, G_SX, G_SXDG, G_T, G_TDG, G_RX, G_RY, G_RZ, G_CX, G_CZ,
  G_SWAP, G_RXX, G_RYY, G_RZZ, G_CRX, G_CRY, G_CRZ, G_CP, G_U4, G_COUNT
};

struct Instr {
  int g, q0, q1;
  double theta;
  // G_U4: its 4 x 4 unitary (32 doubles, row-major, re / im interleaved,
  // basis index 2 b(q0) + b(q1)); owned by the caller for the run
  const double* u = nullptr;
};

const char kLetter[3] = {'X', 'Y', 'Z'};

int letter_index(char c) {
  switch (c) {
    case 'X': return 0;
    case 'Y': return 1;
    case 'Z': return 2;
    default: return -1;
  }
}

bool is_two_qubit(int g) { return g == G_CX || g == G_CZ || (g >= G_SWAP && g <= G_U4); }

// A general two-qubit unitary counts as non-Clifford (push-through mode then
// conjugates it literally, which is exact either way).
bool is_clifford(int g) {
  return g != G_T && g != G_TDG && g != G_RX && g != G_RY && g != G_RZ && (g < G_RXX || g > G_U4);
}

double snap(double v) {
  const double tol = std::ldexp(1.0, -50);
  if (std::fabs(v) <= tol) return 0.0;
  if (std::fabs(std::fabs(v) - 1.0) <= tol) return v > 0 ? 1.0 : -1.0;
  return v;
}

// Image tables of the one-qubit gates under P -> g P g^dagger (rows X, Y, Z).
Table gate_table(int g, double theta) {
  Table t{};
  auto set = [&](int p, double x, double y, double z) { t[p] = {x, y, z}; };
  const double r = std::sqrt(0.5);
  switch (g) {
    case G_H: set(0, 0, 0, 1); set(1, 0, -1, 0); set(2, 1, 0, 0); break;
    case G_S: set(0, 0, 1, 0); set(1, -1, 0, 0); set(2, 0, 0, 1); break;
    case G_SDG: set(0, 0, -1, 0); set(1, 1, 0, 0); set(2, 0, 0, 1); break;
    case G_X: set(0, 1, 0, 0); set(1, 0, -1, 0); set(2, 0, 0, -1); break;
    case G_Y: set(0, -1, 0, 0); set(1, 0, 1, 0); set(2, 0, 0, -1); break;
    case G_Z: set(0, -1, 0, 0); set(1, 0, -1, 0); set(2, 0, 0, 1); break;
    case G_SX: set(0, 1, 0, 0); set(1, 0, 0, 1); set(2, 0, -1, 0); break;
    case G_SXDG: set(0, 1, 0, 0); set(1, 0, 0, -1); set(2, 0, 1, 0); break;
    case G_T: set(0, r, r, 0); set(1, -r, r, 0); set(2, 0, 0, 1); break;
    case G_TDG: set(0, r, -r, 0); set(1, r, r, 0); set(2, 0, 0, 1); break;
    case G_RZ: {
      const double c = std::cos(theta), s = std::sin(theta);
      set(0, c, s, 0); set(1, -s, c, 0); set(2, 0, 0, 1);
      break;
    }
    case G_RX: {
      const double c = std::cos(theta), s = std::sin(theta);
      set(0, 1, 0, 0); set(1, 0, c, s); set(2, 0, -s, c);
      break;
    }
    case G_RY: {
      const double c = std::cos(theta), s = std::sin(theta);
      set(0, c, 0, -s); set(1, 0, 1, 0); set(2, s, 0, c);
      break;
    }
    default: break;
  }
  for (auto& row : t)
    for (auto& v : row) v = snap(v);
  return t;
}

// The CX rule list of Sec. III.C, written as data: for the control letter and
// the target letter, the resulting pair and its sign.  Pairs not listed as
// changing (II, IX, ZI, ZX) map to themselves.
struct CxRule {
  const char* from;
  const char* to;
  int sign;
};
const CxRule kCxRules[] = {
    {"XI", "XX", 1}, {"XX", "XI", 1}, {"IY", "ZY", 1}, {"ZY", "IY", 1},
    {"YI", "YX", 1}, {"YX", "YI", 1}, {"IZ", "ZZ", 1}, {"ZZ", "IZ", 1},
    {"XY", "YZ", 1}, {"YZ", "XY", 1}, {"XZ", "YY", -1}, {"YY", "XZ", -1},
    {"II", "II", 1}, {"IX", "IX", 1}, {"ZI", "ZI", 1}, {"ZX", "ZX", 1},
};

void cx_image(char c, char t, char* oc, char* ot, int* sign) {
  for (const auto& r : kCxRules) {
    if (r.from[0] == c && r.from[1] == t) {
      *oc = r.to[0];
      *ot = r.to[1];
      *sign = r.sign;
      return;
    }
  }
  *oc = c; *ot = t; *sign = 1;  // unreachable for valid letters
}

// --- gate mode -------------------------------------------------------------

PauliSum apply_1q(const PauliSum& in, int q, const Table& t) {
  PauliSum out;
  for (const auto& [key, w] : in) {
    const int p = letter_index(key[q]);
    if (p < 0) {
      out[key] += w;
      continue;
    }
    for (int c = 0; c < 3; ++c) {
      if (t[p][c] == 0.0) continue;
      std::string k2 = key;
      k2[q] = kLetter[c];
      out[k2] += w * t[p][c];
    }
  }
  return out;
}

PauliSum apply_cx(const PauliSum& in, int c, int t) {
  PauliSum out;
  for (const auto& [key, w] : in) {
    std::string k2 = key;
    int sign = 1;
    cx_image(key[c], key[t], &k2[c], &k2[t], &sign);
    out[k2] += w * double(sign);
  }
  return out;
}

// --- two-qubit gates beyond CX and CZ ----------------------------------------
// Their transfer tables come from the 4 x 4 unitaries: with wire q0 the left
// tensor factor (basis index 2 b0 + b1),
//   T[(p0, p1)][(c0, c1)] = Tr((C0 x C1) U (P0 x P1) U^dagger) / 4,
// letters 0 = I, 1 = X, 2 = Y, 3 = Z.
using Mat4 = std::array<std::array<cplx, 4>, 4>;
using Table16 = std::array<std::array<double, 16>, 16>;

Mat4 gate_unitary_2q(int g, double th) {
  Mat4 u{};
  const cplx I(0.0, 1.0);
  const double c = std::cos(th / 2), s = std::sin(th / 2);
  auto diag = [&](cplx a, cplx b, cplx d, cplx e) {
    u[0][0] = a; u[1][1] = b; u[2][2] = d; u[3][3] = e;
  };
  switch (g) {
    case G_SWAP:
      u[0][0] = u[3][3] = 1.0;
      u[1][2] = u[2][1] = 1.0;
      break;
    case G_RXX:  // cos I - i sin X x X
      diag(c, c, c, c);
      u[0][3] = u[3][0] = u[1][2] = u[2][1] = -I * s;
      break;
    case G_RYY:  // Y x Y = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]]
      diag(c, c, c, c);
      u[0][3] = u[3][0] = I * s;
      u[1][2] = u[2][1] = -I * s;
      break;
    case G_RZZ:
      diag(std::exp(-I * (th / 2)), std::exp(I * (th / 2)), std::exp(I * (th / 2)),
           std::exp(-I * (th / 2)));
      break;
    case G_CRX:
      diag(1.0, 1.0, c, c);
      u[2][3] = u[3][2] = -I * s;
      break;
    case G_CRY:
      diag(1.0, 1.0, c, c);
      u[2][3] = -s;
      u[3][2] = s;
      break;
    case G_CRZ:
      diag(1.0, 1.0, std::exp(-I * (th / 2)), std::exp(I * (th / 2)));
      break;
    case G_CP:
      diag(1.0, 1.0, 1.0, std::exp(I * th));
      break;
    default: break;
  }
  return u;
}

Mat4 pauli_pair(int a, int b) {
  std::array<std::array<std::array<cplx, 2>, 2>, 4> P{};
  const cplx I(0.0, 1.0);
  P[0][0][0] = P[0][1][1] = 1.0;
  P[1][0][1] = P[1][1][0] = 1.0;
  P[2][0][1] = -I;
  P[2][1][0] = I;
  P[3][0][0] = 1.0;
  P[3][1][1] = -1.0;
  Mat4 m{};
  for (int i0 = 0; i0 < 2; ++i0)
    for (int i1 = 0; i1 < 2; ++i1)
      for (int j0 = 0; j0 < 2; ++j0)
        for (int j1 = 0; j1 < 2; ++j1) m[2 * i0 + i1][2 * j0 + j1] = P[a][i0][j0] * P[b][i1][j1];
  return m;
}

Mat4 mul4(const Mat4& a, const Mat4& b) {
  Mat4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      for (int k = 0; k < 4; ++k) r[i][j] += a[i][k] * b[k][j];
  return r;
}

Table16 table_of_unitary(const Mat4& u);

Table16 gate_table_2q(int g, double th) { return table_of_unitary(gate_unitary_2q(g, th)); }

// T[(p0, p1)][(c0, c1)] = Tr((C0 x C1) U (P0 x P1) U^dagger) / 4 for a given U.
Table16 table_of_unitary(const Mat4& u) {
  Mat4 ud{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) ud[i][j] = std::conj(u[j][i]);
  Table16 t{};
  for (int p = 0; p < 16; ++p) {
    const Mat4 img = mul4(mul4(u, pauli_pair(p / 4, p % 4)), ud);
    for (int c = 0; c < 16; ++c) {
      const Mat4 prod = mul4(pauli_pair(c / 4, c % 4), img);
      cplx tr = 0.0;
      for (int i = 0; i < 4; ++i) tr += prod[i][i];
      t[p][c] = snap(tr.real() / 4.0);
    }
  }
  return t;
}

int letter16(char c) {
  switch (c) {
    case 'X': return 1;
    case 'Y': return 2;
    case 'Z': return 3;
    default: return 0;
  }
}

PauliSum apply_2q_table(const PauliSum& in, int a, int b, const Table16& t) {
  static const char kL[4] = {'I', 'X', 'Y', 'Z'};
  PauliSum out;
  for (const auto& [key, w] : in) {
    const int p = 4 * letter16(key[a]) + letter16(key[b]);
    for (int c = 0; c < 16; ++c) {
      if (t[p][c] == 0.0) continue;
      std::string k2 = key;
      k2[a] = kL[c / 4];
      k2[b] = kL[c % 4];
      out[k2] += w * t[p][c];
    }
  }
  return out;
}

PauliSum apply_2q(const PauliSum& in, int g, int c, int t) {
  if (g == G_CX) return apply_cx(in, c, t);
  if (g == G_CZ) {  // CZ = H(t) CX(c, t) H(t)
    const Table h = gate_table(G_H, 0.0);
    return apply_1q(apply_cx(apply_1q(in, t, h), c, t), t, h);
  }
  return apply_2q_table(in, c, t, gate_table_2q(g, 0.0));
}

Mat4 u4_matrix(const double* u) {
  Mat4 m{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m[i][j] = cplx(u[2 * (4 * i + j)], u[2 * (4 * i + j) + 1]);
  return m;
}

PauliSum apply_gate(const PauliSum& in, const Instr& g) {
  if (g.g == G_U4) return apply_2q_table(in, g.q0, g.q1, table_of_unitary(u4_matrix(g.u)));
  if (g.g >= G_RXX && g.g <= G_CP) return apply_2q_table(in, g.q0, g.q1, gate_table_2q(g.g, g.theta));
  if (is_two_qubit(g.g)) return apply_2q(in, g.g, g.q0, g.q1);
  return apply_1q(in, g.q0, gate_table(g.g, g.theta));
}

void prune(PauliSum& s, double eps, double* pruned) {
  if (eps <= 0.0) return;
  for (auto it = s.begin(); it != s.end();) {
    if (std::abs(it->second) < eps) {
      *pruned += std::norm(it->second);
      it = s.erase(it);
    } else {
      ++it;
    }
  }
}

PauliSum run_gate_mode(PauliSum s, const std::vector<Instr>& ins, double eps, double* pruned) {
  for (const auto& g : ins) {
    s = apply_gate(s, g);
    prune(s, eps, pruned);
  }
  return s;
}

// --- plan mode -------------------------------------------------------------

struct Op {
  bool one_qubit;
  std::vector<std::vector<Instr>> per_qubit;  // U_k: gates of U_{k,j} for each wire j
  std::vector<Instr> two;                      // V_k: two-qubit gates in list order
  std::vector<Table> lut;                      // U_k: LUT_1q[k] (n tables)
};

// divide_instruction + create_chain: maximal runs of one- and two-qubit gates.
std::vector<Op> divide_instructions(int n, const std::vector<Instr>& ins) {
  std::vector<Op> ops;
  for (const auto& g : ins) {
    const bool one = !is_two_qubit(g.g);
    if (ops.empty() || ops.back().one_qubit != one) {
      Op op;
      op.one_qubit = one;
      if (one) op.per_qubit.assign(n, {});
      ops.push_back(std::move(op));
    }
    if (one)
      ops.back().per_qubit[g.q0].push_back(g);
    else
      ops.back().two.push_back(g);
  }
  return ops;
}

// Qubit-wise grouping: a one-qubit gate commutes with every gate on other
// wires, so it may join the operator of the other one-qubit gates on its wire
// up to the next two-qubit gate there.  Built in rounds over per-wire queues:
// a U round takes, on every wire, the one-qubit gates at the head of its queue
// until a two-qubit gate or the end; a V round takes, again and again until
// none is left, every two-qubit gate that heads the queues of both its wires.
std::vector<Op> divide_instructions_dag(int n, const std::vector<Instr>& ins) {
  std::vector<std::deque<size_t>> queue(n);
  for (size_t i = 0; i < ins.size(); ++i) {
    queue[ins[i].q0].push_back(i);
    if (is_two_qubit(ins[i].g)) queue[ins[i].q1].push_back(i);
  }
  std::vector<Op> ops;
  size_t left = ins.size();
  while (left > 0) {
    Op u;
    u.one_qubit = true;
    u.per_qubit.assign(n, {});
    bool any = false;
    for (int w = 0; w < n; ++w)
      while (!queue[w].empty() && !is_two_qubit(ins[queue[w].front()].g)) {
        u.per_qubit[w].push_back(ins[queue[w].front()]);
        queue[w].pop_front();
        --left;
        any = true;
      }
    if (any) ops.push_back(std::move(u));
    // V round: repeatedly take the two-qubit gates that head both their
    // queues (a gate freed by another one in this round joins the round)
    while (true) {
      std::vector<size_t> ready;
      for (int w = 0; w < n; ++w) {
        if (queue[w].empty()) continue;
        const size_t i = queue[w].front();
        const Instr& g = ins[i];
        if (is_two_qubit(g.g) && g.q0 == w && queue[g.q1].front() == i) ready.push_back(i);
      }
      if (ready.empty()) break;
      std::sort(ready.begin(), ready.end());
      if (ops.empty() || ops.back().one_qubit) {
        Op v;
        v.one_qubit = false;
        ops.push_back(std::move(v));
      }
      for (size_t i : ready) {
        ops.back().two.push_back(ins[i]);
        queue[ins[i].q0].pop_front();
        queue[ins[i].q1].pop_front();
        --left;
      }
    }
  }
  return ops;
}

// create_LUT_1q (Algorithm 1): for each wire j and p in (X, Y, Z), start from
// the weight vector of p and map it through the gates of U_{k,j} in order.
void create_lut(int n, Op& op) {
  op.lut.assign(n, Table{});
  for (int j = 0; j < n; ++j) {
    for (int p = 0; p < 3; ++p) {
      std::array<double, 3> w{0.0, 0.0, 0.0};
      w[p] = 1.0;
      for (const auto& g : op.per_qubit[j]) {
        const Table t = gate_table(g.g, g.theta);
        std::array<double, 3> nw{};
        for (int c = 0; c < 3; ++c) {
          double acc = w[0] * t[0][c];
          acc += w[1] * t[1][c];
          acc += w[2] * t[2][c];
          nw[c] = acc;
        }
        w = nw;
      }
      for (int c = 0; c < 3; ++c) op.lut[j][p][c] = snap(w[c]);
    }
  }
}

// sub + flatten (Algorithm 2, Eq. 3): each string becomes, qubit by qubit, the
// list of (letter, weight) choices read from the table; the Cartesian product
// of those lists gives the simple form, weights multiplied in qubit order.
PauliSum apply_u(const PauliSum& in, int n, const Op& op) {
  PauliSum out;
  std::vector<std::vector<std::pair<char, double>>> choices(n);
  std::vector<int> odo(n);
  for (const auto& [key, w] : in) {
    for (int j = 0; j < n; ++j) {
      choices[j].clear();
      const int p = letter_index(key[j]);
      if (p < 0) {
        choices[j].push_back({key[j], 1.0});
        continue;
      }
      for (int c = 0; c < 3; ++c)
        if (op.lut[j][p][c] != 0.0) choices[j].push_back({kLetter[c], op.lut[j][p][c]});
    }
    std::fill(odo.begin(), odo.end(), 0);
    std::string child(n, 'I');
    while (true) {
      cplx prod = w;
      for (int j = 0; j < n; ++j) {
        child[j] = choices[j][odo[j]].first;
        prod *= choices[j][odo[j]].second;
      }
      out[child] += prod;
      int j = n - 1;
      while (j >= 0 && ++odo[j] == int(choices[j].size())) {
        odo[j] = 0;
        --j;
      }
      if (j < 0) break;
    }
  }
  return out;
}

PauliSum run_plan_mode(PauliSum s, int n, const std::vector<Op>& ops, double eps, double* pruned) {
  for (const auto& op : ops) {
    if (op.one_qubit) {
      s = apply_u(s, n, op);
      prune(s, eps, pruned);
    } else {
      for (const auto& g : op.two) s = apply_gate(s, g);
    }
  }
  return s;
}

// --- push-through mode -------------------------------------------------------
// With D the product of the Clifford gates before a non-Clifford gate G, the
// circuit equals (all its Clifford gates) x ... x (D^dagger G D) x ..., the
// non-Clifford factors in circuit order.  Conjugation by D^dagger G D is done
// literally: forward through the Clifford gates before G, through G, and back
// through their inverses in reverse order; the Clifford gates are applied once
// more, all of them, at the end.  eps > 0 prunes after every non-Clifford gate.
int inverse_gate(int g);

PauliSum run_push_mode(PauliSum s, const std::vector<Instr>& ins, double eps, double* pruned) {
  std::vector<Instr> prefix;
  for (const auto& g : ins) {
    if (is_clifford(g.g)) {
      prefix.push_back(g);
      continue;
    }
    for (const auto& c : prefix) s = apply_gate(s, c);
    s = apply_gate(s, g);
    for (auto it = prefix.rbegin(); it != prefix.rend(); ++it) {
      Instr inv = *it;
      inv.g = inverse_gate(inv.g);
      s = apply_gate(s, inv);
    }
    prune(s, eps, pruned);
  }
  for (const auto& c : prefix) s = apply_gate(s, c);
  return s;
}

struct Plan {
  int n = 0;
  std::vector<Op> ops;
};

struct Result {
  int n = 0;
  std::vector<std::vector<std::pair<std::string, cplx>>> gens;
  std::vector<double> pruned;
};

std::vector<Instr> read_instrs(long m, const int* gate, const int* q0, const int* q1,
                               const double* theta) {
  std::vector<Instr> v(m);
  for (long i = 0; i < m; ++i) v[i] = {gate[i], q0[i], q1[i], theta ? theta[i] : 0.0};
  return v;
}

// U4 instructions name their matrix by theta (an index into mats).
bool attach_u4(std::vector<Instr>& ins, const double* mats, long nmats) {
  for (auto& g : ins) {
    if (g.g != G_U4) continue;
    const long k = long(g.theta);
    if (!mats || double(k) != g.theta || k < 0 || k >= nmats) return false;
    g.u = mats + size_t(k) * 32;
  }
  return true;
}

bool valid(int n, const std::vector<Instr>& ins) {
  if (n < 1) return false;
  for (const auto& g : ins) {
    if (g.g < 0 || g.g >= G_COUNT) return false;
    if (g.g == G_U4 && !g.u) return false;
    if (g.q0 < 0 || g.q0 >= n) return false;
    if (is_two_qubit(g.g) && (g.q1 < 0 || g.q1 >= n || g.q1 == g.q0)) return false;
  }
  return true;
}

int inverse_gate(int g) {
  switch (g) {
    case G_S: return G_SDG;
    case G_SDG: return G_S;
    case G_SX: return G_SXDG;
    case G_SXDG: return G_SX;
    case G_T: return G_TDG;
    case G_TDG: return G_T;
    default: return g;
  }
}

}  // namespace

extern "C" {

// Propagate generators through a circuit.
//   mode 0 = gate mode, 1 = plan mode, 2 = plan mode with qubit-wise grouping,
//   3 = push-through mode.
//   Generators: if n_init == 0, Z_j for j in [gen_begin, gen_end); otherwise the
//   n_init strings in init (n letters each, concatenated) with weights init_w.
//   nthreads: generators are independent, so they are split across threads.
// Returns NULL on invalid input.
void* oracle_run_u4(int n, long m, const int* gate, const int* q0, const int* q1,
                    const double* theta, int mode, double eps, int gen_begin, int gen_end,
                    int n_init, const char* init, const double* init_w, int nthreads,
                    const double* mats, long nmats);

void* oracle_run(int n, long m, const int* gate, const int* q0, const int* q1,
                 const double* theta, int mode, double eps, int gen_begin, int gen_end,
                 int n_init, const char* init, const double* init_w, int nthreads) {
  return oracle_run_u4(n, m, gate, q0, q1, theta, mode, eps, gen_begin, gen_end, n_init, init,
                       init_w, nthreads, nullptr, 0);
}

// As oracle_run, with the matrices of the circuit's U4 gates (gate code 23;
// theta = matrix index; 32 doubles per matrix, see Instr::u).
void* oracle_run_u4(int n, long m, const int* gate, const int* q0, const int* q1,
                    const double* theta, int mode, double eps, int gen_begin, int gen_end,
                    int n_init, const char* init, const double* init_w, int nthreads,
                    const double* mats, long nmats) {
  std::vector<Instr> ins = read_instrs(m, gate, q0, q1, theta);
  if (!attach_u4(ins, mats, nmats) || !valid(n, ins)) return nullptr;
  std::vector<PauliSum> start;
  if (n_init > 0) {
    for (int i = 0; i < n_init; ++i) {
      PauliSum s;
      s[std::string(init + size_t(i) * n, n)] = cplx(init_w ? init_w[i] : 1.0, 0.0);
      start.push_back(s);
    }
  } else {
    if (gen_begin < 0 || gen_end > n || gen_begin > gen_end) return nullptr;
    for (int j = gen_begin; j < gen_end; ++j) {
      std::string z(n, 'I');
      z[j] = 'Z';
      PauliSum s;
      s[z] = cplx(1.0, 0.0);
      start.push_back(s);
    }
  }
  Plan plan;
  plan.n = n;
  if (mode == 1 || mode == 2) {
    plan.ops = mode == 2 ? divide_instructions_dag(n, ins) : divide_instructions(n, ins);
    for (auto& op : plan.ops)
      if (op.one_qubit) create_lut(n, op);
  }
  auto* res = new Result;
  res->n = n;
  const int G = int(start.size());
  res->gens.resize(G);
  res->pruned.assign(G, 0.0);
  auto work = [&](int g) {
    PauliSum out = mode == 3   ? run_push_mode(start[g], ins, eps, &res->pruned[g])
                   : mode >= 1 ? run_plan_mode(start[g], n, plan.ops, eps, &res->pruned[g])
                               : run_gate_mode(start[g], ins, eps, &res->pruned[g]);
    res->gens[g].assign(out.begin(), out.end());
  };
  if (nthreads <= 1 || G <= 1) {
    for (int g = 0; g < G; ++g) work(g);
  } else {
    std::vector<std::thread> pool;
    const int T = std::min(nthreads, G);
    for (int t = 0; t < T; ++t)
      pool.emplace_back([&, t] {
        for (int g = t; g < G; g += T) work(g);
      });
    for (auto& th : pool) th.join();
  }
  return res;
}

// One generator that starts as the weighted sum of n_terms strings (n letters
// each, concatenated) and passes through the circuit.  Returns NULL on invalid
// input.
void* oracle_run_sum(int n, long m, const int* gate, const int* q0, const int* q1,
                     const double* theta, int mode, double eps, long n_terms, const char* strings,
                     const double* weights) {
  std::vector<Instr> ins = read_instrs(m, gate, q0, q1, theta);
  if (!valid(n, ins) || n_terms < 0) return nullptr;
  PauliSum s;
  for (long i = 0; i < n_terms; ++i) s[std::string(strings + size_t(i) * n, n)] += weights[i];
  auto* res = new Result;
  res->n = n;
  res->gens.resize(1);
  res->pruned.assign(1, 0.0);
  PauliSum out;
  if (mode == 1 || mode == 2) {
    std::vector<Op> ops = mode == 2 ? divide_instructions_dag(n, ins) : divide_instructions(n, ins);
    for (auto& op : ops)
      if (op.one_qubit) create_lut(n, op);
    out = run_plan_mode(s, n, ops, eps, &res->pruned[0]);
  } else if (mode == 3) {
    out = run_push_mode(s, ins, eps, &res->pruned[0]);
  } else {
    out = run_gate_mode(s, ins, eps, &res->pruned[0]);
  }
  res->gens[0].assign(out.begin(), out.end());
  return res;
}

int oracle_num_gens(void* h) { return int(static_cast<Result*>(h)->gens.size()); }

long oracle_num_terms(void* h, int g) { return long(static_cast<Result*>(h)->gens[g].size()); }

// Terms of generator g in base-4 index order: strings (n letters each,
// concatenated, no terminator), real and imaginary parts.
void oracle_terms(void* h, int g, char* strings, double* re, double* im) {
  const auto* r = static_cast<Result*>(h);
  size_t i = 0;
  for (const auto& [key, w] : r->gens[g]) {
    std::memcpy(strings + i * r->n, key.data(), r->n);
    re[i] = w.real();
    im[i] = w.imag();
    ++i;
  }
}

double oracle_pruned_sumsq(void* h, int g) { return static_cast<Result*>(h)->pruned[g]; }

void oracle_free(void* h) { delete static_cast<Result*>(h); }

// Image table of one gate (rows X, Y, Z; 9 doubles row-major).
void oracle_gate_table(int g, double theta, double* out9) {
  const Table t = gate_table(g, theta);
  for (int p = 0; p < 3; ++p)
    for (int c = 0; c < 3; ++c) out9[3 * p + c] = t[p][c];
}

// CX image of a (control, target) letter pair; returns the sign.
int oracle_cx(char c, char t, char* out2) {
  int sign = 1;
  cx_image(c, t, &out2[0], &out2[1], &sign);
  return sign;
}

// Plan introspection: number of operators, and for operator k its kind
// (1 = U, 0 = V) and, for U operators, LUT_1q[k] as n x 3 x 3 doubles.
void* oracle_plan(int n, long m, const int* gate, const int* q0, const int* q1,
                  const double* theta, int dag) {
  std::vector<Instr> ins = read_instrs(m, gate, q0, q1, theta);
  if (!valid(n, ins)) return nullptr;
  auto* p = new Plan;
  p->n = n;
  p->ops = dag ? divide_instructions_dag(n, ins) : divide_instructions(n, ins);
  for (auto& op : p->ops)
    if (op.one_qubit) create_lut(n, op);
  return p;
}

long oracle_plan_num_ops(void* h) { return long(static_cast<Plan*>(h)->ops.size()); }

int oracle_plan_op_kind(void* h, long k) { return static_cast<Plan*>(h)->ops[k].one_qubit ? 1 : 0; }

void oracle_plan_lut(void* h, long k, double* out) {
  const auto* p = static_cast<Plan*>(h);
  const auto& op = p->ops[k];
  for (int j = 0; j < p->n; ++j)
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) out[9 * j + 3 * a + c] = op.one_qubit ? op.lut[j][a][c] : 0.0;
}

void oracle_plan_free(void* h) { delete static_cast<Plan*>(h); }

// flatten of Eq. 3 on an explicit complex form: n_par parents, each a scalar
// lambda and, per qubit, a weight 4-vector over (I, X, Y, Z).  Returns a result
// handle with one generator holding the simple form.
void* oracle_flatten(int n, int n_par, const double* lambda, const double* w4) {
  PauliSum out;
  const char letters[4] = {'I', 'X', 'Y', 'Z'};
  for (int k = 0; k < n_par; ++k) {
    std::vector<std::vector<std::pair<char, double>>> ch(n);
    for (int j = 0; j < n; ++j)
      for (int a = 0; a < 4; ++a) {
        const double v = w4[(size_t(k) * n + j) * 4 + a];
        if (v != 0.0) ch[j].push_back({letters[a], v});
      }
    bool empty = false;
    for (int j = 0; j < n; ++j) empty |= ch[j].empty();
    if (empty) continue;
    std::vector<int> odo(n, 0);
    std::string child(n, 'I');
    while (true) {
      cplx prod = lambda[k];
      for (int j = 0; j < n; ++j) {
        child[j] = ch[j][odo[j]].first;
        prod *= ch[j][odo[j]].second;
      }
      out[child] += prod;
      int j = n - 1;
      while (j >= 0 && ++odo[j] == int(ch[j].size())) {
        odo[j] = 0;
        --j;
      }
      if (j < 0) break;
    }
  }
  auto* res = new Result;
  res->n = n;
  res->gens.resize(1);
  res->gens[0].assign(out.begin(), out.end());
  res->pruned.assign(1, 0.0);
  return res;
}

// <0| U^dagger Q U |0> for a Pauli string Q (n letters): Q is propagated in gate
// mode through the inverse gates in reverse order, and the weights of the
// strings made only of I and Z are summed (those are the strings with a
// non-zero expectation in |0...0>).
int oracle_expval(int n, long m, const int* gate, const int* q0, const int* q1,
                  const double* theta, const char* q_string, double* out) {
  std::vector<Instr> ins = read_instrs(m, gate, q0, q1, theta);
  if (!valid(n, ins)) return 1;
  std::vector<Instr> inv(ins.rbegin(), ins.rend());
  for (auto& g : inv) {
    g.g = inverse_gate(g.g);
    g.theta = -g.theta;
  }
  PauliSum s;
  s[std::string(q_string, n)] = cplx(1.0, 0.0);
  double pruned = 0.0;
  s = run_gate_mode(s, inv, 0.0, &pruned);
  double acc = 0.0;
  for (const auto& [key, w] : s) {
    bool ztype = true;
    for (char c : key) ztype &= (c == 'I' || c == 'Z');
    if (ztype) acc += w.real();
  }
  *out = acc;
  return 0;
}

}  // extern "C"
