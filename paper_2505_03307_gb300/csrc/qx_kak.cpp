// Arbitrary two-qubit unitaries (QX_U4) as gates the device program already
// runs: one-qubit rotations and the commuting XX / YY / ZZ rotations.
//
// The paper builds its one-qubit tables from gate lists and leaves general
// multi-qubit gates to future work (Sec. II.C, III.C).  Any U in U(4) factors
// (the KAK / Cartan decomposition of SU(4)) as
//     U = e^{i g} (A0 x A1) exp(i (a XX + b YY + c ZZ)) (C0 x C1),
// with A0, A1, C0, C1 in SU(2).  In the magic basis B, local unitaries become
// real orthogonal matrices and the XX / YY / ZZ rotations diagonal ones, so
// with U_B = B^dagger U B (scaled to det 1) and M = U_B^T U_B (symmetric and
// unitary), a real orthogonal O diagonalises M: O^T M O = D.  Then
// U_B = K1 D^{1/2} K2 with K2 = O^T and K1 = U_B O D^{-1/2}, both real
// orthogonal; taking both with determinant +1 (a column sign moved into
// D^{1/2}), B K B^dagger are the local factors, and B D^{1/2} B^dagger is the
// entangling part, whose phases solve a 4 x 4 linear system for (g, a, b, c).
// Each SU(2) factor becomes RZ(alpha) RY(beta) RZ(gamma) (Euler angles).
//
// The real symmetric matrices Re M and Im M commute; a combination of the two
// with a fixed irrational coefficient is diagonalised by Jacobi rotations (its
// eigenvectors then diagonalise M unless eigenvalues nearly collide by
// accident).  Six coefficients are tried and the decomposition whose gate
// product is closest to U (up to a global phase, max entry) is kept; it is
// accepted when that distance is at most 1e-10, else QX_EINVAL.
#include <array>
#include <cmath>
#include <complex>
#include <vector>

#include "qx_common.h"

using namespace qx;

namespace {

using cd = std::complex<double>;
using M4 = std::array<std::array<cd, 4>, 4>;
using M2 = std::array<std::array<cd, 2>, 2>;
using R4 = std::array<std::array<double, 4>, 4>;

M4 mul(const M4& a, const M4& b) {
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 4; ++j) r[i][j] += a[i][k] * b[k][j];
  return r;
}

M4 dagger(const M4& a) {
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i][j] = std::conj(a[j][i]);
  return r;
}

M4 transpose(const M4& a) {
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i][j] = a[j][i];
  return r;
}

cd det4(M4 a) {  // Gaussian elimination with partial pivoting
  cd d = 1.0;
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (std::abs(a[r][c]) > std::abs(a[p][c])) p = r;
    if (std::abs(a[p][c]) == 0.0) return 0.0;
    if (p != c) {
      std::swap(a[p], a[c]);
      d = -d;
    }
    d *= a[c][c];
    for (int r = c + 1; r < 4; ++r) {
      const cd f = a[r][c] / a[c][c];
      for (int k = c; k < 4; ++k) a[r][k] -= f * a[c][k];
    }
  }
  return d;
}

double det4r(const R4& a) {
  M4 m{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) m[i][j] = a[i][j];
  return det4(m).real();
}

// The magic basis (columns): (|00> + |11>)/sqrt2, i(|00> - |11>)/sqrt2,
// i(|01> + |10>)/sqrt2, (|01> - |10>)/sqrt2; basis index 2 b0 + b1.
M4 magic() {
  const double h = std::sqrt(0.5);
  const cd I(0.0, 1.0);
  M4 b{};
  b[0][0] = h;
  b[3][0] = h;
  b[0][1] = I * h;
  b[3][1] = -I * h;
  b[1][2] = I * h;
  b[2][2] = I * h;
  b[1][3] = h;
  b[2][3] = -h;
  return b;
}

M2 pauli(int p) {
  const cd I(0.0, 1.0);
  M2 m{};
  if (p == 0) m = {{{1.0, 0.0}, {0.0, 1.0}}};
  if (p == 1) m = {{{0.0, 1.0}, {1.0, 0.0}}};
  if (p == 2) m = {{{0.0, -I}, {I, 0.0}}};
  if (p == 3) m = {{{1.0, 0.0}, {0.0, -1.0}}};
  return m;
}

M4 kron(const M2& a, const M2& b) {
  M4 r{};
  for (int i0 = 0; i0 < 2; ++i0)
    for (int i1 = 0; i1 < 2; ++i1)
      for (int j0 = 0; j0 < 2; ++j0)
        for (int j1 = 0; j1 < 2; ++j1) r[2 * i0 + i1][2 * j0 + j1] = a[i0][j0] * b[i1][j1];
  return r;
}

// Eigenvectors of a real symmetric 4 x 4 matrix (columns of V), cyclic Jacobi.
void jacobi(R4 a, R4* v) {
  R4& V = *v;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) off += a[p][q] * a[p][q];
    if (off < 1e-32) break;
    for (int p = 0; p < 4; ++p)
      for (int q = p + 1; q < 4; ++q) {
        if (std::fabs(a[p][q]) < 1e-300) continue;
        const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < 4; ++k) {  // a <- J^T a J
          const double akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 4; ++k) {
          const double apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 4; ++k) {
          const double vkp = V[k][p], vkq = V[k][q];
          V[k][p] = c * vkp - s * vkq;
          V[k][q] = s * vkp + c * vkq;
        }
      }
  }
}

// K (4 x 4, a tensor product up to rounding) = A0 x A1 with A0, A1 in SU(2).
bool split_local(const M4& k, M2* a0, M2* a1) {
  int bi = 0, bk = 0;
  double best = -1.0;
  for (int i = 0; i < 2; ++i)
    for (int kk = 0; kk < 2; ++kk) {
      double nrm = 0.0;
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < 2; ++l) nrm += std::norm(k[2 * i + j][2 * kk + l]);
      if (nrm > best) {
        best = nrm;
        bi = i;
        bk = kk;
      }
    }
  if (best <= 0.0) return false;
  M2 b{};
  const double s = std::sqrt(2.0 / best);
  for (int j = 0; j < 2; ++j)
    for (int l = 0; l < 2; ++l) b[j][l] = k[2 * bi + j][2 * bk + l] * s;
  // B is unitary up to a phase: scale to det 1
  const cd db = b[0][0] * b[1][1] - b[0][1] * b[1][0];
  const cd rb = std::sqrt(db);
  for (auto& row : b)
    for (auto& e : row) e /= rb;
  M2 a{};
  for (int i = 0; i < 2; ++i)
    for (int kk = 0; kk < 2; ++kk) {
      cd tr = 0.0;  // Tr(B^dagger block_ik) / 2
      for (int j = 0; j < 2; ++j)
        for (int l = 0; l < 2; ++l) tr += std::conj(b[j][l]) * k[2 * i + j][2 * kk + l];
      a[i][kk] = tr / 2.0;
    }
  const cd da = a[0][0] * a[1][1] - a[0][1] * a[1][0];
  const cd ra = std::sqrt(da);
  for (auto& row : a)
    for (auto& e : row) e /= ra;
  *a0 = a;
  *a1 = b;
  return true;
}

// V in SU(2) (up to sign) = RZ(alpha) RY(beta) RZ(gamma); the gates in
// application order are RZ(gamma), RY(beta), RZ(alpha).
void euler_zyz(const M2& v, double* alpha, double* beta, double* gamma) {
  const double c = std::abs(v[0][0]), s = std::abs(v[1][0]);
  *beta = 2.0 * std::atan2(s, c);
  // v00 = e^{-i(a+g)/2} cos, v10 = e^{i(a-g)/2} sin
  const double sum = c > 1e-300 ? -2.0 * std::arg(v[0][0]) : 0.0;    // alpha + gamma
  const double dif = s > 1e-300 ? 2.0 * std::arg(v[1][0]) : 0.0;     // alpha - gamma
  if (c <= 1e-300) {  // v = [[0, -e^{-i(a-g)/2}], [e^{i(a-g)/2}, 0]]: gamma free
    *alpha = dif;
    *gamma = 0.0;
  } else if (s <= 1e-300) {  // diagonal: alpha - gamma free
    *alpha = sum;
    *gamma = 0.0;
  } else {
    *alpha = 0.5 * (sum + dif);
    *gamma = 0.5 * (sum - dif);
  }
}

M2 rot(int axis, double t) {  // RX / RY / RZ (axis 1 / 2 / 3) = exp(-i t P / 2)
  const cd I(0.0, 1.0);
  const M2 p = pauli(axis);
  M2 r{};
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) r[i][j] = (i == j ? std::cos(t / 2) : 0.0) - I * std::sin(t / 2) * p[i][j];
  return r;
}

M4 rot2(int axis, double t) {  // exp(-i t P x P / 2)
  const cd I(0.0, 1.0);
  const M4 pp = kron(pauli(axis), pauli(axis));
  M4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r[i][j] = (i == j ? std::cos(t / 2) : 0.0) - I * std::sin(t / 2) * pp[i][j];
  return r;
}

// The 4 x 4 matrix of a gate list on (q0, q1) (later gates on the left).
M4 product(const std::vector<qx_instr>& gs, int q0) {
  M4 u{};
  for (int i = 0; i < 4; ++i) u[i][i] = 1.0;
  const M2 id = pauli(0);
  for (const qx_instr& g : gs) {
    M4 m;
    if (g.gate == QX_RXX || g.gate == QX_RYY || g.gate == QX_RZZ) {
      m = rot2(int(g.gate - QX_RXX) + 1, g.theta);
    } else {
      const M2 r = rot(g.gate == QX_RY ? 2 : 3, g.theta);
      m = g.q0 == q0 ? kron(r, id) : kron(id, r);
    }
    u = mul(m, u);
  }
  return u;
}

double phase_residual(const M4& a, const M4& b) {  // max |a - e^{i phi} b|, best phi
  cd tr = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) tr += std::conj(b[i][j]) * a[i][j];
  const cd ph = std::abs(tr) > 0 ? tr / std::abs(tr) : cd(1.0);
  double r = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r = std::max(r, std::abs(a[i][j] - ph * b[i][j]));
  return r;
}

bool decompose(const M4& u_in, int q0, int q1, std::vector<qx_instr>* out, double* residual) {
  const cd det = det4(u_in);
  if (std::abs(std::abs(det) - 1.0) > 1e-8) return false;
  M4 u = u_in;
  const cd sc = std::pow(det, -0.25);
  for (auto& row : u)
    for (auto& e : row) e *= sc;
  const M4 B = magic(), Bd = dagger(B);
  const M4 ub = mul(mul(Bd, u), B);
  const M4 m = mul(transpose(ub), ub);
  // eigenvalues of XX, YY, ZZ on the magic states (diagonal in that basis)
  double lam[3][4];
  for (int p = 0; p < 3; ++p) {
    const M4 d = mul(mul(Bd, kron(pauli(p + 1), pauli(p + 1))), B);
    for (int k = 0; k < 4; ++k) lam[p][k] = d[k][k].real();
  }
  const double mix[6] = {0.61803398875, 1.41421356237, -0.7320508, 2.2360679775, -1.9, 0.3};
  double best = INFINITY;
  for (int attempt = 0; attempt < 6; ++attempt) {
    R4 a{}, o{};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) a[i][j] = m[i][j].real() + mix[attempt] * m[i][j].imag();
    jacobi(a, &o);
    if (det4r(o) < 0)
      for (int i = 0; i < 4; ++i) o[i][0] = -o[i][0];
    M4 oc{}, otc{};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) {
        oc[i][j] = o[i][j];
        otc[i][j] = o[j][i];
      }
    const M4 d = mul(mul(otc, m), oc);
    cd half[4];
    for (int k = 0; k < 4; ++k) half[k] = std::sqrt(d[k][k]);
    M4 k1 = mul(ub, oc);  // times D^{-1/2}
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) k1[i][j] /= half[j];
    R4 k1r{};
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) k1r[i][j] = k1[i][j].real();
    if (det4r(k1r) < 0) {
      for (int i = 0; i < 4; ++i) k1[i][0] = -k1[i][0];
      half[0] = -half[0];
    }
    // entangler phases: arg(half_k) = g + a lam_XX + b lam_YY + c lam_ZZ
    double A[4][5];
    for (int k = 0; k < 4; ++k) {
      A[k][0] = 1.0;
      A[k][1] = lam[0][k];
      A[k][2] = lam[1][k];
      A[k][3] = lam[2][k];
      A[k][4] = std::arg(half[k]);
    }
    for (int c = 0; c < 4; ++c) {  // Gauss-Jordan (the matrix is +-1 entries, invertible)
      int p = c;
      for (int r = c + 1; r < 4; ++r)
        if (std::fabs(A[r][c]) > std::fabs(A[p][c])) p = r;
      for (int j = 0; j < 5; ++j) std::swap(A[p][j], A[c][j]);
      for (int r = 0; r < 4; ++r) {
        if (r == c) continue;
        const double f = A[r][c] / A[c][c];
        for (int j = c; j < 5; ++j) A[r][j] -= f * A[c][j];
      }
    }
    const double ea = A[1][4] / A[1][1], eb = A[2][4] / A[2][2], ec = A[3][4] / A[3][3];
    M2 a0, a1, c0, c1;
    if (!split_local(mul(mul(B, k1), Bd), &a0, &a1) || !split_local(mul(mul(B, otc), Bd), &c0, &c1))
      continue;
    std::vector<qx_instr> gs;
    auto euler = [&](const M2& v, int q) {
      double al, be, ga;
      euler_zyz(v, &al, &be, &ga);
      gs.push_back({QX_RZ, q, -1, ga});
      gs.push_back({QX_RY, q, -1, be});
      gs.push_back({QX_RZ, q, -1, al});
    };
    euler(c0, q0);
    euler(c1, q1);
    // exp(i a XX) = RXX(-2a), and likewise for YY, ZZ
    gs.push_back({QX_RXX, q0, q1, -2.0 * ea});
    gs.push_back({QX_RYY, q0, q1, -2.0 * eb});
    gs.push_back({QX_RZZ, q0, q1, -2.0 * ec});
    euler(a0, q0);
    euler(a1, q1);
    const double res = phase_residual(product(gs, q0), u_in);
    if (res < best) {  // keep the most accurate of the combinations
      best = res;
      *out = gs;
      *residual = res;
    }
  }
  return best <= 1e-10;
}

}  // namespace

namespace qx {
qx_status decompose_u4(const double* u32, int q0, int q1, std::vector<qx_instr>* out,
                       double* residual) {
  M4 u{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      const double re = u32[2 * (4 * i + j)], im = u32[2 * (4 * i + j) + 1];
      if (!std::isfinite(re) || !std::isfinite(im)) return fail(QX_EINVAL, "U4 entry is not finite");
      u[i][j] = cd(re, im);
    }
  // unitary to 1e-8
  const M4 p = mul(dagger(u), u);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j)
      if (std::abs(p[i][j] - (i == j ? 1.0 : 0.0)) > 1e-8) return fail(QX_EINVAL, "U4 matrix is not unitary");
  double res = 0.0;
  if (!decompose(u, q0, q1, out, &res)) return fail(QX_EINVAL, "U4 decomposition failed its check");
  if (residual) *residual = res;
  return QX_OK;
}
}  // namespace qx

extern "C" qx_status qx_u4_decompose(const double* u, int q0, int q1, qx_instr* out, size_t* count,
                                     double* residual) {
  clear_error();
  if (!u || !out || !count) return fail(QX_EINVAL, "NULL argument");
  if (q0 < 0 || q1 < 0 || q0 == q1) return fail(QX_EINVAL, "wires must be distinct and >= 0");
  std::vector<qx_instr> gs;
  if (const qx_status s = decompose_u4(u, q0, q1, &gs, residual)) return s;
  for (size_t k = 0; k < gs.size(); ++k) out[k] = gs[k];
  *count = gs.size();
  return QX_OK;
}
