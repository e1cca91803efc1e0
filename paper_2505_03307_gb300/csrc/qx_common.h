// Internal declarations of libqx shared by the host planner and the device driver.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "qx.h"

namespace qx {

constexpr int kMaxQubits = 128;
constexpr int kMaxWords = 2;

// Error reporting: thread-local message behind qx_last_error().
qx_status fail(qx_status s, const std::string& msg);
void clear_error();

// 3x3 Pauli image table, rows and columns in (X, Y, Z) order.
struct Table3 {
  double r[3][3];
};

// Encoded op of a fused Clifford pass (gate-list form).
//   bits 0-1  : kind (0 = one-qubit signed permutation, 1 = CX, 2 = CZ)
//   bits 2-8  : q0, bits 9-15: q1
//   bits 16-24: signed permutation, 3 bits per source letter p in (X, Y, Z):
//               bits 0-1 target letter index, bit 2 sign (1 = negative)
enum : uint32_t { kOpPerm = 0, kOpCX = 1, kOpCZ = 2 };
inline uint32_t encode_op(uint32_t kind, int q0, int q1, uint32_t perm) {
  return kind | (uint32_t(q0) << 2) | (uint32_t(q1 < 0 ? 0 : q1) << 9) | (perm << 16);
}

// One fused Clifford pass: every Clifford gate between two expansion steps.
struct CliffPass {
  std::vector<uint32_t> ops;        // gate-list form, in application order
  bool identity = true;             // the composed map is the identity
  // Tableau form: images of X_q (q < n) and Z_q in XZ form
  // (phase exponent e: the Pauli is i^e X^x Z^z).
  std::vector<uint64_t> img_x, img_z;  // [2n][W]
  std::vector<uint8_t> img_e;          // [2n]
  // Chunk tables for the device: chunk c covers qubits [c*cb, c*cb + cb);
  // entry (c, idx) with idx = xbits | zbits << cb is the XZ-form image of
  // X^xbits Z^zbits on that chunk.
  int chunk_bits = 0;
  int chunks = 0;
  std::vector<uint64_t> tab_xz;  // [chunks][1 << 2cb][2W]: x words then z words
  std::vector<uint8_t> tab_e;    // [chunks][1 << 2cb]
  bool use_table = false;        // device applies tab_* (else the gate list)
  uint64_t support[kMaxWords] = {0, 0};  // qubits some gate of the pass acts on
};

// A fan-out qubit of a one-qubit operator: a 3x3 table that is not a signed
// permutation.
struct FanQubit {
  int q;
  Table3 t;
  uint8_t nnz[3];      // non-zero entries per row
  uint8_t col[3][3];   // their columns, in increasing order
  bool iso[3];         // row p maps to one letter that no other row reaches
};

struct FanStep {
  std::vector<FanQubit> qs;  // increasing qubit order
  size_t op_index;           // position of the U operator in the chain
  // For the last fan-out step of a plan whose Clifford passes before and
  // after it both act on other qubits than its wires: index into
  // qx_plan::aux_passes of the two passes composed (before, then after),
  // which the step may apply to each parent in one go; -1 otherwise.
  int pre_tail = -1;
};

// Whether pass pc acts only on qubits other than the wires of fan step fs (the
// two then commute: conjugations on disjoint qubits).
inline bool pass_disjoint(const CliffPass& pc, const FanStep& fs) {
  for (const FanQubit& f : fs.qs)
    if ((pc.support[f.q >> 6] >> (f.q & 63)) & 1) return false;
  return true;
}

// Fan-out steps that the fused expansion takes: at most kSmallMaxWires wires
// and at most kSmallMaxChildren children per parent (the product over the
// wires of their largest row's entry count).
constexpr int kSmallMaxWires = 8;
constexpr int kSmallMaxChildren = 16;
inline bool small_fan_step(const FanStep& fs) {
  if (fs.qs.empty() || fs.qs.size() > size_t(kSmallMaxWires)) return false;
  int prod = 1;
  for (const FanQubit& f : fs.qs) {
    int m = 1;
    for (int a = 0; a < 3; ++a) m = f.nnz[a] > m ? f.nnz[a] : m;
    prod *= m;
    if (prod > kSmallMaxChildren) return false;
  }
  return true;
}

// A Pauli rotation exp(-i phi P / 2) as a device step: a string Q that
// anticommutes with P becomes cos phi Q + sin phi (i Q P), and i Q P = +-(Q xor P).
struct RotStep {
  uint64_t px[kMaxWords], pz[kMaxWords];  // the Hermitian string P (bits beyond n clear)
  double c, s;                            // cos phi, sin phi (within 2^-50 of 0, +-1: exact)
};

enum StepKind { kStepCliff = 0, kStepFan = 1, kStepRot = 2 };

// The Pauli rotations exp(-i a theta P / 2) that make up a two-qubit
// rotation gate (RXX ... CP), with P's bits and the factor a = dphi/dtheta;
// empty for other gates.
struct RotTerm {
  uint64_t px[kMaxWords], pz[kMaxWords];
  double a;
};
std::vector<RotTerm> gate_rotation_terms(const qx_instr& g);
struct Step {
  int kind;
  int index;              // into passes or fans
  uint64_t ops_before;    // chain operators (paper's U_k, V_k) since the previous fan step
};

}  // namespace qx

struct qx_circuit {
  int n;
  std::vector<qx_instr> ins;
};

struct qx_plan_device;  // device-side copy of the plan (built on first use)

struct qx_plan {
  int n = 0;
  int W = 1;
  std::vector<qx_instr> ins;                       // the circuit in the plan's application order
  std::vector<size_t> order;                       // order[k]: input index of ins[k] (empty: identity)
  size_t K = 0, Kp = 0;
  std::vector<int> op_kind;                        // chain: 1 = U, 0 = V
  // per chain op (empty for V): the tables of the wires the operator touches,
  // in increasing qubit order (every other wire's table is the identity)
  // operator k of the chain is ins[op_begin[k] .. op_begin[k + 1]) (its
  // per-wire tables are recomputed from these gates when asked for)
  std::vector<size_t> op_begin;
  std::vector<qx::CliffPass> passes;
  // composed passes that no program step names (FanStep::pre_tail)
  std::vector<qx::CliffPass> aux_passes;
  std::vector<qx::FanStep> fans;
  std::vector<qx::RotStep> rots;
  std::vector<qx::Step> program;
  uint64_t ops_after_last_fan = 0;
  qx_plan_device* dev = nullptr;
};

namespace qx {
// Host planner entry points used by the device driver.
qx_status build_plan(const qx_circuit* c, qx_plan** out);
qx_status inverse_circuit(const qx_circuit* c, qx_circuit** out);
void free_plan_device(qx_plan* p);
// Makes later device work on r (readout, free) use `stream` (e.g. when the
// stream it was computed on is about to be destroyed).  r must be idle.
void result_set_stream(qx_result* r, void* stream);
// Applies pass `pc` to one string on the host with the same tables the device uses.
void host_apply_pass(const CliffPass& pc, int n, int W, uint64_t* x, uint64_t* z, int* sign);
// The gates (RZ / RY on each wire, RXX, RYY, RZZ) whose product is the 4 x 4
// unitary u32 (row-major, re / im interleaved, basis index 2 b(q0) + b(q1)) up
// to a global phase; *residual: the largest entry of the difference.
qx_status decompose_u4(const double* u32, int q0, int q1, std::vector<qx_instr>* out,
                       double* residual);
// Push-through plan of a circuit (qx_group_ops_pushthrough).
qx_status build_plan_pushthrough(const qx_circuit* c, qx_plan** out);
// The same from instructions the plan takes over (already validated).
qx_status build_plan_pushthrough(int n, std::vector<qx_instr>&& ins, qx_plan** out);
// The checks of qx_load_circuit: n in 1..128, gate codes, wires, finite angles.
qx_status validate_instrs(int n, const qx_instr* ins, size_t m);

// Batched propagation (the serving loop): the plans, all push-through plans
// of one word count, propagate together in one term store on `stream`
// (allocations stream-ordered on it), each request's generators with their own
// ids; result r is request r's, as qx_propagate of its plan alone would give
// (the same strings and weights; term order may differ).  budget bounds the
// batch's term storage at every step (0: none).  On error no result is set.
struct BatchRequest {
  const qx_plan* plan = nullptr;
  qx_result* result = nullptr;
};
qx_status batch_propagate(std::vector<BatchRequest>& reqs, int precision, double eps,
                          size_t budget, void* stream);
}  // namespace qx
