/*
 * qx.h - C interface of libqx, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of extended-stabilizer Pauli propagation (Qimax,
 * arXiv 2505.03307).
 *
 * What it computes.  For a circuit U = g_{m-1} ... g_0 on n qubits, every
 * generator Z_j of |0...0> evolves as U Z_j U^dagger = sum_P c_j(P) P, a sum of
 * real-weighted Hermitian Pauli strings (Eq. 1 and Sec. II.A; gates act by
 * conjugation g P g^dagger, Sec. II.C).  The library follows the paper's
 * operator-level method: the instruction list is grouped into one-qubit
 * operators U_k and two-qubit operators V_k (Sec. III.A, Algorithm 2), every
 * U_k gets a table of 3x3 Pauli images per qubit (Algorithm 1), and each term
 * is expanded through those tables (sub + flatten, Eq. 3) with identical
 * strings merged by index-based accumulation (abstract).
 *
 * Pauli strings cross this interface as bit masks.  A string on n qubits uses
 * W = ceil(n / 64) words of x bits and W words of z bits; qubit q is bit
 * (q mod 64) of word q / 64.  (x, z) = (0,0) I, (1,0) X, (1,1) Y, (0,1) Z, and
 * Y is the Hermitian Y (any sign lives in the real weight).  Arrays of strings
 * are row-major: string i occupies words [i*W, i*W + W).
 *
 * Conventions (not fixed by the paper): RX/RY/RZ(theta) = exp(-i theta s / 2),
 * T = diag(1, e^{i pi/4}), S = diag(1, i), SX = sqrt(X); CZ = H(t) CX H(t).
 * Two-qubit rotations (RXX ... CP) enter the device program as Pauli rotation
 * steps inside their V_k (each string Q that anticommutes with the rotation's
 * Pauli P gains the partner Q xor P; the two are merged).
 * Composed table entries within 2^-50 of 0 or of +-1 are set to 0 or +-1.
 * eps = 0 keeps every string that the tables reach, even when its weight sums
 * to exactly 0; eps > 0 drops |w| < eps after every U_k.
 *
 * Errors.  Every call returns a qx_status.  On error the out-parameters are
 * left untouched and qx_last_error() returns a message for the calling thread.
 * The library never aborts the process.
 *
 * Threads and streams.  Handles are not thread-safe; distinct handles may be
 * used from distinct threads on distinct streams.  Device work is issued on
 * the stream of qx_prop_opts; calls that return host values synchronise that
 * stream.
 */
#ifndef QX_H_INCLUDED_
#define QX_H_INCLUDED_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QX_OK = 0,
  QX_EINVAL = 1,       /* invalid argument or circuit */
  QX_ENOMEM = 2,       /* device or host allocation failed */
  QX_EBUDGET = 3,      /* the counted term storage exceeds qx_prop_opts.hbm_budget */
  QX_ECAP = 4,         /* the term count exceeds qx_prop_opts.max_terms, or a table filled up */
  QX_ECUDA = 5,        /* a CUDA runtime call failed (message in qx_last_error) */
  QX_ETIMEOUT = 6,     /* a bounded device-side wait gave up */
  QX_EUNSUPPORTED = 7  /* valid but not supported (e.g. n > 128, no usable GPU) */
} qx_status;

/* Gate codes of qx_instr.gate. */
typedef enum {
  QX_H = 0, QX_S = 1, QX_SDG = 2, QX_X = 3, QX_Y = 4, QX_Z = 5, QX_SX = 6, QX_SXDG = 7,
  QX_T = 8, QX_TDG = 9, QX_RX = 10, QX_RY = 11, QX_RZ = 12, QX_CX = 13, QX_CZ = 14,
  /* Two-qubit gates beyond CX / CZ (the paper leaves them to future work,
   * Sec. III.C).  SWAP is Clifford.  The others are Pauli rotations on the
   * two wires (q0, q1): RXX/RYY/RZZ(theta) = exp(-i theta P0 P1 / 2), and the
   * controlled rotations with q0 the control: CRX/CRY/CRZ(theta) apply
   * RX/RY/RZ(theta) to q1 when q0 is |1>, CP(theta) = diag(1, 1, 1, e^{i theta}). */
  QX_SWAP = 15, QX_RXX = 16, QX_RYY = 17, QX_RZZ = 18, QX_CRX = 19, QX_CRY = 20,
  QX_CRZ = 21, QX_CP = 22,
  /* Any two-qubit unitary on (q0, q1), given as a 4 x 4 matrix through
   * qx_load_circuit_u4 (theta = index of the matrix).  Basis index
   * 2 b(q0) + b(q1): q0 is the left tensor factor. */
  QX_U4 = 23
} qx_gate;

/* One instruction {g, w, theta} (Sec. III.A): gate, wire(s), parameter.
 * q1 is the target of CX / second wire of CZ and is ignored (use -1) for
 * one-qubit gates; theta is ignored by gates without a parameter. */
typedef struct {
  uint32_t gate;
  int32_t q0;
  int32_t q1;
  double theta;
} qx_instr;

typedef struct qx_circuit qx_circuit;
typedef struct qx_plan qx_plan;
typedef struct qx_result qx_result;

/* Optional device allocator: returns device memory of at least `bytes` bytes
 * usable on `stream` (NULL on failure); free releases it, stream-ordered.
 * Any alignment will do: the library asks for 256 bytes more than it uses
 * and starts its buffer at the next 256-byte boundary inside the block (free
 * gets the pointer the allocator returned). */
typedef void* (*qx_alloc_fn)(size_t bytes, void* ctx, void* stream);
typedef void (*qx_free_fn)(void* ptr, void* ctx, void* stream);

typedef struct {
  int precision;        /* 64: FP64 weights; 32: FP32 weights with compensated products
                           and sums (TwoProduct / TwoSum, about one float rounding per
                           operator); strings, signs and phases stay exact either way */
  double eps;           /* pruning threshold, >= 0 (see above) */
  int gen_begin;        /* generators Z_j with gen_begin <= j < gen_end; */
  int gen_end;          /*   gen_end <= 0 means n (all generators) */
  size_t hbm_budget;    /* max bytes of term storage at any step; 0 = unlimited */
  size_t max_terms;     /* max number of terms at any step; 0 = unlimited */
  void* stream;         /* cudaStream_t to issue work on; NULL = default stream */
  qx_alloc_fn alloc;    /* NULL: cudaMallocAsync / cudaFreeAsync on `stream` */
  qx_free_fn free;
  void* alloc_ctx;
  uint32_t timeout_ms;  /* bound on device-side waits; 0 = 2000 ms */
  uint32_t flags;       /* QX_FLAG_* bits */
} qx_prop_opts;

/* qx_prop_opts.flags: record CUDA events around every kernel launch (on the
 * launch stream) and report per-kernel-class device time in qx_prop_stats. */
#define QX_FLAG_KERNEL_TIMING 1u
/* qx_prop_opts.flags: never run merge wires in place.  By default a fan-out
 * step whose merge groups all hold every letter their tables produce (no
 * string created or removed) updates the weights in place through a full-key
 * index instead of rebuilding the terms; the results are the same. */
#define QX_FLAG_NO_INPLACE 2u

/* Kernel classes of qx_prop_stats.kc_* (names from qx_kernel_class_name). */
#define QX_KC_COUNT 15

/* Counters of one propagation (metrics and launch accounting). */
typedef struct {
  uint64_t K, Kp;              /* number of U_k and V_k operators of the plan (Sec. III.A) */
  uint64_t term_updates;       /* sum over the K + K' operators of the terms they were applied to */
  uint64_t children;           /* terms written by expansion and merge steps */
  uint64_t alg_bytes;          /* algorithmic bytes: (in + out) terms of each device step x 16W+8 */
  uint64_t kernel_launches;    /* kernels launched by this call */
  uint64_t host_syncs;         /* stream synchronisations inside this call */
  uint64_t final_terms;        /* terms of all generators at the end */
  uint64_t peak_terms;         /* largest term count of any step */
  uint64_t fan_steps;          /* device expansion steps (one-qubit operators with fan-out) */
  uint64_t merge_passes;       /* index-accumulation (merge) passes */
  uint64_t clifford_passes;    /* fused Clifford passes */
  uint64_t inplace_steps;      /* fan-out steps whose merges ran in place */
  uint64_t inplace_fallbacks;  /* in-place attempts that found an open group */
  uint64_t block_steps;        /* in-place steps that ran in block order */
  uint64_t guesses_held;       /* fan-out steps launched on the plan's record of its last
                                  run (before their letter masks were read) that kept it */
  uint64_t guesses_missed;     /* such launches that the masks or the device rejected */
  /* per kernel class: launches, algorithmic bytes (terms each launch must
   * read and write, 16W+8 bytes per term), and device milliseconds (only with
   * QX_FLAG_KERNEL_TIMING; 0 otherwise) */
  uint64_t kc_launches[16];
  uint64_t kc_bytes[16];
  double kc_ms[16];
} qx_prop_stats;

/* Name of kernel class k (0 <= k < QX_KC_COUNT), "" otherwise. */
const char* qx_kernel_class_name(int k);

/* Fills *o with defaults: precision 64, eps 0, all generators, no limits,
 * default stream, cudaMallocAsync, timeout 2000 ms. */
void qx_default_opts(qx_prop_opts* o);

/* Validates and copies an instruction list (Sec. III.A).  1 <= n <= 128,
 * 0 <= q0 < n, for CX/CZ 0 <= q1 < n and q1 != q0, theta finite.
 * m may be 0.  *out is owned by the caller (qx_free_circuit). */
qx_status qx_load_circuit(int n, const qx_instr* ins, size_t m, qx_circuit** out);

/* As qx_load_circuit, for circuits with arbitrary two-qubit unitaries
 * (QX_U4; the paper leaves gates beyond its set to future work, Sec. II.C and
 * III.C).  mats holds nmats 4 x 4 complex matrices, 32 doubles each: row-major,
 * real and imaginary parts interleaved, basis index 2 b(q0) + b(q1); a QX_U4
 * instruction names its matrix by theta (an integer 0 <= theta < nmats).
 * Each such gate is replaced in the circuit by 15 gates whose product is its
 * matrix up to a global phase (which conjugation ignores): RZ RY RZ on each
 * wire, RXX RYY RZZ (three commuting Pauli rotations), RZ RY RZ on each wire
 * (the KAK decomposition, computed on the host and accepted only when the
 * product matches the matrix to 1e-10).  The circuit then holds those gates
 * (instruction indices of later calls refer to them).  QX_EINVAL for a matrix
 * that is not unitary to 1e-8 or an index out of range.  Other instructions
 * as qx_load_circuit. */
qx_status qx_load_circuit_u4(int n, const qx_instr* ins, size_t m, const double* mats,
                             size_t nmats, qx_circuit** out);

/* The 15 gates that qx_load_circuit_u4 puts in place of one QX_U4 on
 * (q0, q1): out receives them (15 entries), *count their number, *residual
 * (may be NULL) the largest entry of (their product - e^{i phi} u) for the
 * best phase phi.  u: 32 doubles as in qx_load_circuit_u4.  Host only. */
qx_status qx_u4_decompose(const double* u, int q0, int q1, qx_instr* out, size_t* count,
                          double* residual);

/* divide_instruction + create_chain + create_LUT_1q (the set-up steps of
 * Algorithm 2, and Algorithm 1): maximal runs of one-qubit gates become U_k,
 * maximal runs of two-qubit gates V_k; for each U_k and wire j the gates of
 * U_{k,j} are composed in list order into a 3x3 table.  Host only; deterministic.  A plan
 * with 20,000 or more Clifford operations builds its passes' tables on up to
 * 8 short-lived threads, joined before the call returns (the tables do not
 * depend on the number of threads).
 * *out is owned by the caller (qx_free_plan); it does not refer to `c`. */
qx_status qx_group_ops(const qx_circuit* c, qx_plan** out);

/* Qubit-wise (dependency-graph) grouping.  One-qubit gates commute with
 * gates on other wires, so each wire's one-qubit gates between two of its
 * two-qubit gates can join one operator: the gates are reordered by their
 * level in the circuit's dependency graph (counted in two-qubit gates on the
 * same wires) and grouped as by qx_group_ops.  The circuit is unchanged; the
 * operator count K + K' is at most that of list-order grouping (Sec. III.A's
 * chain, built over the reordered list), and tables of gates that meet on a
 * wire compose (e.g. T ... T becomes S even with two-qubit gates on other
 * wires in between).  Weights agree with list-order grouping up to rounding;
 * string sets may differ in strings of weight exactly 0.  The plan applies
 * its instructions in its own order (qx_plan_order). */
qx_status qx_group_ops_dag(const qx_circuit* c, qx_plan** out);

/* *m = instruction count; order (m entries, may be NULL) receives, for each
 * position k of the plan's application order, the index of that instruction
 * in the circuit given to qx_group_ops / qx_group_ops_dag (identity for the
 * former).  qx_plan_derivative and its op_end use the plan's order;
 * qx_tape_backward reports gradients in the circuit's order. */
qx_status qx_plan_order(const qx_plan* p, size_t* m, size_t* order);

/* Clifford push-through (not in the paper).  Every Clifford gate is moved to
 * the end of the circuit: with D the product of the Clifford gates before a
 * non-Clifford gate, that gate's rotation exp(-i phi s / 2) about a Pauli s
 * equals exp(-i phi P / 2) after the whole Clifford part, P = D^dagger s D.
 * The plan applies these Pauli rotations in circuit order (T and TDG as
 * rotations by +-pi/4 about Z, the two-qubit rotations as one to three
 * commuting Pauli rotations) and then the whole Clifford part as one pass.
 * Each rotation maps a string Q that anticommutes with P to cos phi Q +
 * sin phi (i Q P) and leaves the others; strings Q and Q xor P are merged.
 * Weights agree with qx_group_ops up to rounding; string sets may differ in
 * strings of weight exactly 0.  The plan has no U_k / V_k chain (K = K' = 0,
 * qx_plan_lut is not available). */
qx_status qx_group_ops_pushthrough(const qx_circuit* c, qx_plan** out);

/* Number of U_k (*K) and V_k (*Kp) operators; either pointer may be NULL. */
qx_status qx_plan_info(const qx_plan* p, size_t* K, size_t* Kp);

/* Kind of operator `op` of the chain (in circuit order): 1 = U, 0 = V. */
qx_status qx_plan_op(const qx_plan* p, size_t op, int* kind);

/* LUT_1q of operator `op` (which must be a U): n x 3 x 3 doubles, row-major,
 * entry [j][a][c] = coefficient of Pauli c in the image of Pauli a under
 * U_{k,j}, with a, c in (X, Y, Z) order.  out holds n*9 doubles.  The plan
 * keeps each operator's instruction range, not its tables: every call
 * composes the operator's gates again (the same arithmetic as the plan's own
 * tables, so the values are those the plan used). */
qx_status qx_plan_lut(const qx_plan* p, size_t op, double* out);

/* Host-side inspection of the fused Clifford passes built from the plan:
 * *count = number of passes; pass s maps a Pauli string (x, z: W words each,
 * host memory) and *sign to its image under that pass (in place). */
qx_status qx_plan_clifford_passes(const qx_plan* p, size_t* count);
qx_status qx_plan_clifford_apply(const qx_plan* p, size_t pass, uint64_t* x, uint64_t* z,
                                 int* sign);

/* Algorithm 2 on the GPU: generators Z_j (gen_begin <= j < gen_end) start as
 * one term of weight 1 (create_Z_j) and pass through the operator chain.
 * The result owns its device arrays (freed by qx_free_result with the same
 * allocator).  Returns QX_EBUDGET / QX_ECAP before allocating a step whose
 * counted size exceeds the limits; the plan stays valid either way.
 * Result generator g (0 <= g < gen_end - gen_begin) is Z_{gen_begin + g}.
 *
 * A plan keeps, per fan-out step, what its last propagation did (a pure
 * expansion and its size, or block-ordered in-place merges and their block
 * count) and launches the next propagation's step on that record before
 * reading anything back; steps whose record held twice in a row are checked
 * only at the end of the call, which repeats itself once with every check on
 * the spot if one fails.  Results never depend on the record (a wrong one
 * costs time only: qx_prop_stats.guesses_missed); plans may be shared between
 * threads and streams (the record is updated atomically). */
qx_status qx_propagate(const qx_plan* p, const qx_prop_opts* o, qx_result** out);

/* Grows the current device's default memory pool (the one cudaMallocAsync
 * serves qx_propagate from when no allocator is given) to hold at least
 * `bytes`, stream-ordered on `stream` (NULL: the default stream), and raises
 * the pool's release threshold so that the memory stays reserved until the
 * process exits (or cudaMemPoolTrimTo).  A propagation's buffers grow step by
 * step, and a pool that has to grow with them maps new memory in the middle
 * of a run: the first runs of a large circuit are up to 2x slower until the
 * pool holds their peak (two runs after a reservation of the peak, five
 * without, on the 84M-term workload).  Not a counterpart of anything in the
 * paper (Sec. IV's M_max is the budget this reserves up front).  Blocks until
 * the pool has grown.  QX_ENOMEM if the device cannot provide `bytes`
 * (nothing stays reserved then); QX_EUNSUPPORTED without a device. */
qx_status qx_reserve_device_memory(size_t bytes, void* stream);

/* As qx_propagate, but the initial generators are `ngen` single terms given
 * in host memory: x, z (ngen x W words) and weights w (ngen doubles, or NULL
 * for all 1).  gen_begin / gen_end of *o are ignored. */
qx_status qx_propagate_from(const qx_plan* p, int ngen, const uint64_t* x, const uint64_t* z,
                            const double* w, const qx_prop_opts* o, qx_result** out);

/* Number of generators, words per string and terms of the whole result. */
qx_status qx_result_shape(const qx_result* r, int* ngen, int* nwords, size_t* nterms);

/* Per generator: number of terms, sum of squared weights and the squared
 * weight removed by pruning.  Any out pointer may be NULL. */
qx_status qx_result_info(const qx_result* r, int gen, size_t* nterms, double* sumsq,
                         double* pruned_sumsq);

/* Counters of the propagation that made r. */
qx_status qx_result_stats(const qx_result* r, qx_prop_stats* s);

/* Terms of generator `gen` in base-4 index order (I=0, X=1, Y=2, Z=3, qubit 0
 * the most significant digit; the order of Example 1).  x, z: cap x W words;
 * w: cap doubles.  on_device != 0: the three pointers are device memory.
 * QX_EINVAL if cap is smaller than the generator's term count. */
qx_status qx_result_export(const qx_result* r, int gen, uint64_t* x, uint64_t* z, double* w,
                           size_t cap, int on_device);

/* All terms of the result in device order (unsorted), into caller buffers:
 * x, z (cap x W words), w (cap doubles), gen (cap int32).  The buffers are
 * device memory or page-locked host memory (cudaHostAlloc / cudaMallocHost),
 * which the export kernel then writes across the host link directly, with no
 * intermediate device copy.  Returns after the writes are complete. */
qx_status qx_result_raw(const qx_result* r, uint64_t* x, uint64_t* z, double* w, int32_t* gen,
                        size_t cap);

/* Coefficient c_gen(P) of one string (x, z: W words, host memory): the
 * weight of P in generator gen, 0 when absent.  *im is always 0 (weights are
 * real, Sec. II.A).  im may be NULL. */
qx_status qx_coeff(const qx_result* r, int gen, const uint64_t* x, const uint64_t* z, double* re,
                   double* im);

/* nq lookups at once: gen (nq int32), x, z (nq x W words), out (nq doubles).
 * on_device != 0: all four pointers are device memory. */
qx_status qx_coeff_batch(const qx_result* r, size_t nq, const int32_t* gen, const uint64_t* x,
                         const uint64_t* z, double* out, int on_device);

/* <0| U^dagger Q U |0> for nobs Pauli strings Q (x, z: nobs x W words, host
 * memory; out: nobs doubles, host).  Each Q is propagated through the inverse
 * circuit with the same kernels (Heisenberg picture) and the weights of its
 * Z-type strings (x = 0) are summed.  This is the single-qubit measurement of
 * Sec. II.B in exact form: p_{k,0} = (1 + <Z_k>) / 2. */
qx_status qx_expval(const qx_plan* p, size_t nobs, const uint64_t* x, const uint64_t* z,
                    const qx_prop_opts* o, double* out);

/* ---- Continuation and gradients ------------------------------------------
 * The map that a circuit applies to the real weights of one generator is
 * linear and orthogonal: conjugation by a unitary permutes the orthonormal
 * basis {P / sqrt(2^n)} of Hermitian operators into another orthonormal basis
 * (Sec. II.A, II.C).  Its transpose is therefore the map of the inverse
 * circuit, which is what the reverse (adjoint) pass below propagates.  The
 * gradient of a linear functional L = sum_k a_k c_{g_k}(P_k) of output weights
 * with respect to the angle theta of a rotation (RX, RY, RZ) inside the
 * one-qubit operator U_k (Sec. III.A) is
 *     dL/dtheta = < M_k D, Lambda_k >,
 * where M_k is the forward state after U_k, Lambda_k the functional pulled
 * back to the same point through the inverse of the rest of the circuit, and
 * D = T^T dT/dtheta acts on the rotation's wire only, T being that wire's
 * 3x3 table of U_k (Algorithm 1).  The paper does not treat gradients; this
 * is the adjoint of its forward map.  With eps > 0 both passes prune, and the
 * result is the gradient of the pruned computation only approximately. */

/* A result holding the given terms: nterms strings (x, z: nterms x W words),
 * weights w and generator ids gen (0 <= gen < ngen), all in host memory.
 * Repeated (gen, string) pairs are summed; pairs whose weight sums to
 * exactly 0 are dropped.  precision 64 or 32 selects the weight type, as in
 * qx_prop_opts.  Device memory comes from cudaMallocAsync on the default
 * stream. */
qx_status qx_result_from_terms(int n, int ngen, size_t nterms, const uint64_t* x,
                               const uint64_t* z, const double* w, const int32_t* gen,
                               int precision, qx_result** out);

/* Propagation through plan p starting from every term of `from` (which is
 * left unchanged); the result has from's generators.  from must have p's
 * qubit count and the precision of *o.  gen_begin / gen_end of *o are
 * ignored. */
qx_status qx_propagate_result(const qx_plan* p, const qx_result* from, const qx_prop_opts* o,
                              qx_result** out);

/* For instruction `instr` of the plan (position in the plan's application
 * order, see qx_plan_order), which must be RX, RY or RZ:
 * d9 (9 doubles, row-major, (X, Y, Z) order) receives D = T^T dT/dtheta of its
 * wire in the one-qubit operator U_k that holds it, *qubit its wire and
 * *op_end the index one past the last instruction of U_k (the point where
 * M_k and Lambda_k are taken).  qubit and op_end may be NULL. */
qx_status qx_plan_derivative(const qx_plan* p, size_t instr, double* d9, int* qubit,
                             size_t* op_end);

/* out[r] = sum_g sum_P m_g(P) * sum_l D_r[p][l] * lam_{lam_gen[g]}(P with letter
 * l on wire qubit[r]), for nrot rotations r, where p is P's letter on that
 * wire (strings with I there contribute nothing).  lam_gen (m's generator
 * count entries, host) pairs each generator of m with one of lam, -1 for
 * none; d9: nrot x 9 doubles; qubit, out: nrot entries; all host memory.
 * m and lam must have the same qubit count and precision.  Sums are taken
 * in a fixed order: the same inputs on the same GPU give the same bits. */
qx_status qx_adjoint_dot(const qx_result* m, const qx_result* lam, const int32_t* lam_gen,
                         size_t nrot, const int32_t* qubit, const double* d9, double* out);

/* As qx_adjoint_dot for Pauli rotations exp(-i phi P / 2) (the two-qubit
 * rotation gates): out[r] = sum_g sum_Q m_g(Q) sigma(Q) lam_{lam_gen[g]}(Q xor P_r)
 * over the strings Q of m that anticommute with P_r, where i Q P_r =
 * sigma(Q) (Q xor P_r); this is dL/dphi when m and lam are taken right after
 * the rotation.  px, pz: nrot x W words (host). */
qx_status qx_adjoint_dot_pauli(const qx_result* m, const qx_result* lam, const int32_t* lam_gen,
                               size_t nrot, const uint64_t* px, const uint64_t* pz, double* out);

/* Tape: a forward pass that keeps the term arrays at the end of every U_k
 * that holds a rotation and after every two-qubit rotation gate (per-operator
 * checkpoints), and reverse passes over it.  ckpt_stride s >= 1 keeps every s-th of those states and recomputes
 * the others one block at a time during the reverse pass (s = 1 keeps all;
 * 0 picks s = ceil(sqrt(number of such operators))).
 * qx_tape_forward propagates the generators of *o (as qx_propagate) and
 * writes values[k] = c_{gen[k]}(P_k) for nq query strings (x, z: nq x W
 * words; gen relative to gen_begin), all host memory. */
typedef struct qx_tape qx_tape;
qx_status qx_tape_forward(const qx_plan* p, const qx_prop_opts* o, int ckpt_stride, size_t nq,
                          const int32_t* gen, const uint64_t* x, const uint64_t* z,
                          double* values, qx_tape** out);
/* grad[i] = dL/dtheta_i for L = sum_k a[k] values[k] and every instruction i
 * of the circuit, in the order the circuit was given to qx_group_ops or
 * qx_group_ops_dag (0 for instructions without an angle: RX, RY, RZ and
 * RXX ... CP have one); a: nq doubles,
 * grad: number-of-instructions doubles, host memory.  May be called any
 * number of times with different a. */
qx_status qx_tape_backward(qx_tape* t, const double* a, double* grad);
/* Number of rotations, of checkpointed operators, of states held now, and
 * the bytes of term storage they use.  Any out pointer may be NULL. */
qx_status qx_tape_info(const qx_tape* t, size_t* nrot, size_t* nops, size_t* held,
                       size_t* held_bytes);

/* ---- Serving: a request loop with continuous batching ---------------------
 * Circuits are submitted as they arrive.  Host planner threads turn each into
 * a push-through plan (as qx_group_ops_pushthrough: its non-Clifford gates as
 * Pauli rotations, then one Clifford pass) and reserve for it an upper bound
 * on its term storage (each rotation at most doubles each generator).
 * `slots` engine threads, each with its own CUDA stream, admit planned
 * requests in arrival order into a batch while the reservations of all
 * running batches stay within hbm_budget (the memory side of the feasibility
 * region of Sec. IV, term storage bounded by M_max; 0 = no limit), and
 * propagate the batch in one term store: every generator of every request has
 * its own id, each rotation step is one launch sequence for the whole batch,
 * and the final passes run in one launch.  Requests that arrive while batches
 * run join the next batch as soon as an engine and memory are free, and
 * several batches run on the device at once.  A request whose bound alone
 * exceeds hbm_budget runs by itself once no batch runs, with hbm_budget
 * enforced on its exact sizes (QX_EBUDGET if it needs more).
 * Each result equals qx_propagate of the circuit's push-through plan alone:
 * the same strings and weights (the batched kernels do the same arithmetic
 * per term); the order of its terms may differ. */
typedef struct qx_server qx_server;

typedef struct {
  int slots;          /* engines (batches on the device at once), 1..256 */
  size_t hbm_budget;  /* bytes of term storage reserved by all running batches; 0 = unlimited */
  int precision;      /* 64 or 32, as qx_prop_opts.precision */
  double eps;         /* as qx_prop_opts.eps */
  size_t max_queue;   /* waiting requests accepted; 0 = unlimited (else QX_ECAP) */
  int max_batch;      /* requests per batch, >= 1; 0 = 256 */
} qx_server_opts;

typedef struct {
  uint64_t completed, failed;
  uint64_t alone;     /* requests whose bound exceeded hbm_budget, run by themselves */
  uint64_t queued, running;       /* waiting requests; batches on the device */
  double p50_ms, p99_ms, max_ms;  /* latency from submission to completion */
  uint64_t batches;   /* batches run */
  double mean_batch;  /* requests per batch */
  uint64_t peak_reserved;  /* largest bytes reserved at once by running batches */
} qx_serve_stats;

/* Defaults: 2 engines, no budget, precision 64, eps 0, unbounded queue,
 * batches of up to 256 requests. */
void qx_server_default_opts(qx_server_opts* o);
/* Starts the planners and engines on the current device. */
qx_status qx_server_create(const qx_server_opts* o, qx_server** out);
/* Queues a circuit (copied; validated when it is planned); *ticket identifies it. */
qx_status qx_server_submit(qx_server* s, int n, const qx_instr* ins, size_t m, uint64_t* ticket);
/* *done = 1 once the request has finished (with or without error). */
qx_status qx_server_poll(qx_server* s, uint64_t ticket, int* done);
/* Blocks until the request finishes; returns its status.  On success *out
 * is a result owned by the caller (qx_free_result).  A ticket can be waited
 * for once. */
qx_status qx_server_wait(qx_server* s, uint64_t ticket, qx_result** out, double* latency_ms);
qx_status qx_server_stats(qx_server* s, qx_serve_stats* st);
/* Finishes running batches, fails waiting requests, stops the threads and
 * frees results that were never waited for. */
void qx_server_destroy(qx_server* s);

/* One-qubit expansion with index-based accumulation that allocates nothing.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory, for example a process whose GPU memory is
 * entirely owned by another allocator (a framework pool that reserved the
 * device), or a latency-critical loop where cudaMalloc, which may synchronise
 * the device, is not acceptable.  The scratch (hash table and group payload,
 * about 16 MiB) is a fixed array inside the library that every GPU which
 * loads the library holds until the process exits.
 *
 * Applies the 3x3 image table `table` (9 doubles, host memory, rows and
 * columns in (X, Y, Z) order, as qx_plan_lut) to wire q of every input term,
 * and merges the children that land on the same (generator, string).  Inputs
 * and outputs are device memory in planar layout: word k of string i is at
 * x[k * n_in + i] (input) and out_x[k * out_cap + i] (output), W = ceil(n/64)
 * words; weights and generator ids one per term.  Input strings must be
 * unique within their generator.  Output order is unspecified; *n_out (host)
 * receives the number of output terms.
 *
 * Limits: n_in <= 262144 terms, ngen <= 4096, otherwise QX_EINVAL before any
 * device work; a generator id >= ngen is found on the device before any
 * merge kernel reads it and gives QX_EINVAL with no output written;
 * QX_ECAP when out_cap is too small (at most 3 * n_in outputs).
 * The first call on a device (with that device current) looks up and clears
 * the scratch and synchronises the device; make that first call before any
 * other work that must not be synchronised.  Every call on a device shares
 * the same scratch array and leaves its contents behind (later calls ignore
 * them).  Calls from one process are serialised by a lock inside the library
 * that is held until the call's stream has finished its work; device work of
 * another process, or work the caller queues on the scratch's device
 * outside this call, does not touch the array.  The call synchronises
 * `stream` (a cudaStream_t, NULL for the default stream) before returning. */
qx_status qx_merge_qubit_static(int n, size_t n_in, int ngen, const uint64_t* x,
                                const uint64_t* z, const double* w, const uint32_t* gen, int q,
                                const double* table, uint64_t* out_x, uint64_t* out_z,
                                double* out_w, uint32_t* out_gen, size_t out_cap, size_t* n_out,
                                void* stream);

/* Self-test of the device-side bounded wait that every wait of the library
 * uses: one warp waits for a flag that another warp of the same block
 * publishes only when publish != 0.  Returns QX_OK when the wait ended, or
 * QX_ETIMEOUT when it gave up after about timeout_ms (0: 2000 ms); the
 * device stays usable either way.  QX_EUNSUPPORTED without a GPU. */
qx_status qx_wait_selftest(uint32_t timeout_ms, int publish);

void qx_free_circuit(qx_circuit* c);
void qx_free_plan(qx_plan* p);
void qx_free_result(qx_result* r);
void qx_free_tape(qx_tape* t);

/* Message of the last error on the calling thread ("" if none). */
const char* qx_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QX_H_INCLUDED_ */
