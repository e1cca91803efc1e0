// Reverse-mode gradients of output weights with respect to rotation angles
// (qx_tape_*).
//
// The circuit is cut after every one-qubit operator U_k (Sec. III.A) that
// holds a rotation; those cut points are the checkpoints.  The forward pass
// propagates the generators segment by segment and keeps the term arrays at
// the cut points.  The reverse pass starts from the functional
// L = sum_k a_k c_{g_k}(P_k) written as one weighted Pauli sum per generator,
// pulls it back through the inverse of each segment (the transpose of an
// orthogonal map is its inverse), and at every cut point takes
// <M_k D, Lambda_k> for each rotation of U_k (qx_adjoint_dot).  All term work
// runs on the device through the library's own propagation and adjoint
// kernels; this file only orders the calls and owns the states.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "qx_common.h"

using namespace qx;

#define QX_TRY_STATUS(...)              \
  do {                                  \
    const qx_status s_ = (__VA_ARGS__); \
    if (s_ != QX_OK) return s_;         \
  } while (0)

struct qx_tape {
  int n = 0, G = 0;
  qx_prop_opts opts{};
  size_t m = 0;                  // instructions of the circuit
  std::vector<size_t> bounds;    // cut points b_0 < ... < b_{B-1}
  std::vector<qx_plan*> seg;     // B + 1 segments: [0, b_0), [b_0, b_1), ..., [b_{B-1}, m)
  std::vector<qx_plan*> inv;     // inverse of each segment (inv[0] unused)
  struct Rot {
    size_t instr;
    int q;
    double d[9];
    size_t j;  // cut point after its U_k (or after the gate, for two-qubit rotations)
    std::vector<RotTerm> terms;  // two-qubit rotation gates: their Pauli rotations
  };
  std::vector<Rot> rots;
  std::vector<qx_result*> ckpt;  // M_j at cut point j, or nullptr where not kept
  int stride = 1;
  std::vector<int32_t> qgen;
  std::vector<uint64_t> qx, qz;
  std::vector<size_t> order;     // plan position -> circuit index (empty: identity)
};

namespace {

qx_status make_plan(int n, const std::vector<qx_instr>& ins, size_t b, size_t e, bool inverse,
                    qx_plan** out) {
  qx_circuit c;
  c.n = n;
  c.ins.assign(ins.begin() + b, ins.begin() + e);
  if (!inverse) return build_plan(&c, out);
  qx_circuit* ic = nullptr;
  const qx_status s = inverse_circuit(&c, &ic);
  if (s != QX_OK) return s;
  const qx_status t = build_plan(ic, out);
  qx_free_circuit(ic);
  return t;
}

void free_tape_states(qx_tape* t) {
  for (qx_result*& r : t->ckpt) {
    qx_free_result(r);
    r = nullptr;
  }
}

// Replaces *cur by its propagation through p (the old state is freed).
qx_status advance(const qx_tape* t, const qx_plan* p, qx_result** cur) {
  qx_result* next = nullptr;
  const qx_status s = qx_propagate_result(p, *cur, &t->opts, &next);
  if (s != QX_OK) return s;
  qx_free_result(*cur);
  *cur = next;
  return QX_OK;
}

}  // namespace

extern "C" {

qx_status qx_tape_forward(const qx_plan* p, const qx_prop_opts* o, int ckpt_stride, size_t nq,
                          const int32_t* gen, const uint64_t* x, const uint64_t* z,
                          double* values, qx_tape** out) {
  clear_error();
  if (!p || !out) return fail(QX_EINVAL, "NULL argument");
  if (nq && (!gen || !x || !z || !values)) return fail(QX_EINVAL, "NULL query array");
  if (ckpt_stride < 0) return fail(QX_EINVAL, "ckpt_stride must be >= 0");
  qx_prop_opts opts;
  qx_default_opts(&opts);
  if (o) opts = *o;
  const int gb = opts.gen_begin, ge = opts.gen_end <= 0 ? p->n : opts.gen_end;
  if (gb < 0 || ge > p->n || gb >= ge) return fail(QX_EINVAL, "bad generator range");
  const int G = ge - gb;
  for (size_t k = 0; k < nq; ++k)
    if (gen[k] < 0 || gen[k] >= G) return fail(QX_EINVAL, "query generator out of range");
  auto* t = new (std::nothrow) qx_tape;
  if (!t) return fail(QX_ENOMEM, "host allocation failed");
  t->n = p->n;
  t->G = G;
  t->opts = opts;
  t->m = p->ins.size();
  t->order = p->order;
  t->qgen.assign(gen, gen + nq);
  t->qx.assign(x, x + nq * size_t(p->W));
  t->qz.assign(z, z + nq * size_t(p->W));
  auto body = [&]() -> qx_status {
    // rotations and the cut point after the U_k of each
    for (size_t i = 0; i < t->m; ++i) {
      const uint32_t g = p->ins[i].gate;
      qx_tape::Rot r{};
      r.instr = i;
      if (g == QX_RX || g == QX_RY || g == QX_RZ) {
        size_t end = 0;
        const qx_status s = qx_plan_derivative(p, i, r.d, &r.q, &end);
        if (s != QX_OK) return s;
        r.j = end;  // replaced by the cut index below
      } else {
        r.terms = gate_rotation_terms(p->ins[i]);
        if (r.terms.empty()) continue;
        r.j = i + 1;  // right after the gate: its rotations commute with each other
      }
      t->bounds.push_back(r.j);
      t->rots.push_back(std::move(r));
    }
    std::sort(t->bounds.begin(), t->bounds.end());
    t->bounds.erase(std::unique(t->bounds.begin(), t->bounds.end()), t->bounds.end());
    for (auto& r : t->rots)
      r.j = size_t(std::lower_bound(t->bounds.begin(), t->bounds.end(), r.j) - t->bounds.begin());
    const size_t B = t->bounds.size();
    t->stride = ckpt_stride > 0 ? ckpt_stride
                                : std::max(1, int(std::ceil(std::sqrt(double(std::max<size_t>(B, 1))))));
    // segments and their inverses
    t->seg.assign(B + 1, nullptr);
    t->inv.assign(B + 1, nullptr);
    for (size_t j = 0; j <= B; ++j) {
      const size_t b = j == 0 ? 0 : t->bounds[j - 1], e = j == B ? t->m : t->bounds[j];
      QX_TRY_STATUS(make_plan(t->n, p->ins, b, e, false, &t->seg[j]));
      if (j > 0) QX_TRY_STATUS(make_plan(t->n, p->ins, b, e, true, &t->inv[j]));
    }
    // forward pass with checkpoints
    t->ckpt.assign(B, nullptr);
    qx_result* cur = nullptr;
    QX_TRY_STATUS(qx_propagate(t->seg[0], &t->opts, &cur));
    for (size_t j = 0; j < B; ++j) {
      qx_result* next = nullptr;
      const qx_status s = qx_propagate_result(t->seg[j + 1], cur, &t->opts, &next);
      if (s != QX_OK) {
        qx_free_result(cur);
        return s;
      }
      if (j % size_t(t->stride) == 0)
        t->ckpt[j] = cur;
      else
        qx_free_result(cur);
      cur = next;
    }
    const qx_status s = nq ? qx_coeff_batch(cur, nq, gen, x, z, values, 0) : QX_OK;
    qx_free_result(cur);
    return s;
  };
  const qx_status s = body();
  if (s != QX_OK) {
    const std::string msg = qx_last_error();
    qx_free_tape(t);
    return fail(s, msg);
  }
  *out = t;
  return QX_OK;
}

qx_status qx_tape_backward(qx_tape* t, const double* a, double* grad) {
  clear_error();
  if (!t || !grad) return fail(QX_EINVAL, "NULL argument");
  const size_t nq = t->qgen.size();
  if (nq && !a) return fail(QX_EINVAL, "a is NULL");
  std::fill(grad, grad + t->m, 0.0);
  const size_t B = t->bounds.size();
  if (B == 0 || nq == 0) return QX_OK;
  // one reverse generator per distinct query generator
  std::vector<int32_t> lam_of(size_t(t->G), -1), lgen(nq);
  int L = 0;
  for (size_t k = 0; k < nq; ++k) {
    int32_t& h = lam_of[size_t(t->qgen[k])];
    if (h < 0) h = L++;
    lgen[k] = h;
  }
  qx_result* lam = nullptr;
  QX_TRY_STATUS(qx_result_from_terms(t->n, L, nq, t->qx.data(), t->qz.data(), a, lgen.data(),
                                     t->opts.precision, &lam));
  std::vector<qx_result*> tmp(B, nullptr);
  auto body = [&]() -> qx_status {
    QX_TRY_STATUS(advance(t, t->inv[B], &lam));  // Lambda at the last cut point
    const int W = (t->n + 63) / 64;
    std::vector<int32_t> qs;
    std::vector<double> ds, outv, pfac;
    std::vector<size_t> who, pwho;
    std::vector<uint64_t> pxs, pzs;
    for (size_t j = B; j-- > 0;) {
      const qx_result* M = t->ckpt[j];
      if (!M && !tmp[j]) {  // recompute the block from its kept state
        const size_t j0 = j - j % size_t(t->stride);
        const qx_result* cur = t->ckpt[j0];
        if (!cur) return fail(QX_EINVAL, "internal error: missing checkpoint");
        for (size_t k = j0 + 1; k <= j; ++k) {
          QX_TRY_STATUS(qx_propagate_result(t->seg[k], cur, &t->opts, &tmp[k]));
          cur = tmp[k];
        }
      }
      if (!M) M = tmp[j];
      qs.clear();
      ds.clear();
      who.clear();
      pxs.clear();
      pzs.clear();
      pwho.clear();
      pfac.clear();
      for (const auto& r : t->rots) {
        if (r.j != j) continue;
        if (r.terms.empty()) {
          qs.push_back(r.q);
          ds.insert(ds.end(), r.d, r.d + 9);
          who.push_back(r.instr);
          continue;
        }
        for (const RotTerm& rt : r.terms) {
          pxs.insert(pxs.end(), rt.px, rt.px + W);
          pzs.insert(pzs.end(), rt.pz, rt.pz + W);
          pwho.push_back(r.instr);
          pfac.push_back(rt.a);
        }
      }
      auto slot = [&](size_t instr) -> double& {
        return grad[t->order.empty() ? instr : t->order[instr]];
      };
      if (!qs.empty()) {
        outv.assign(qs.size(), 0.0);
        QX_TRY_STATUS(qx_adjoint_dot(M, lam, lam_of.data(), qs.size(), qs.data(), ds.data(),
                                     outv.data()));
        for (size_t r = 0; r < who.size(); ++r) slot(who[r]) = outv[r];
      }
      if (!pwho.empty()) {  // dL/dtheta = sum over the gate's rotations of a dL/dphi
        outv.assign(pwho.size(), 0.0);
        QX_TRY_STATUS(qx_adjoint_dot_pauli(M, lam, lam_of.data(), pwho.size(), pxs.data(),
                                           pzs.data(), outv.data()));
        for (size_t r = 0; r < pwho.size(); ++r) slot(pwho[r]) += pfac[r] * outv[r];
      }
      qx_free_result(tmp[j]);
      tmp[j] = nullptr;
      if (j > 0) QX_TRY_STATUS(advance(t, t->inv[j], &lam));
    }
    return QX_OK;
  };
  const qx_status s = body();
  const std::string msg = s == QX_OK ? std::string() : std::string(qx_last_error());
  for (qx_result* r : tmp) qx_free_result(r);
  qx_free_result(lam);
  if (s != QX_OK) return fail(s, msg);
  return QX_OK;
}

qx_status qx_tape_info(const qx_tape* t, size_t* nrot, size_t* nops, size_t* held,
                       size_t* held_bytes) {
  clear_error();
  if (!t) return fail(QX_EINVAL, "tape is NULL");
  size_t h = 0, bytes = 0;
  for (const qx_result* r : t->ckpt) {
    if (!r) continue;
    ++h;
    int W = 1;
    size_t N = 0;
    qx_result_shape(r, nullptr, &W, &N);
    bytes += N * size_t(16 * W + (t->opts.precision == 32 ? 4 : 8) + 4);
  }
  if (nrot) *nrot = t->rots.size();
  if (nops) *nops = t->bounds.size();
  if (held) *held = h;
  if (held_bytes) *held_bytes = bytes;
  return QX_OK;
}

void qx_free_tape(qx_tape* t) {
  if (!t) return;
  free_tape_states(t);
  for (qx_plan* p : t->seg) qx_free_plan(p);
  for (qx_plan* p : t->inv) qx_free_plan(p);
  delete t;
}

}  // extern "C"
