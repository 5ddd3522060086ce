/*
 * ttn.h -- C ABI of libttn: single-GPU (sm_103a) TTN-TDVP for the Rydberg
 * digital twin of arXiv 2210.03763.
 *
 * What it computes.  A binary tree tensor network (TTN) over an Lx x Ly
 * lattice of three-level atoms (|0>, |1>, |r>), with leaves in Hilbert-curve
 * order (Sec. "Tensor network simulations"), evolved by the single-site
 * time-dependent variational principle under the Rydberg Hamiltonian
 *
 *   H(t) = sum_i [ Ox_i sx_i + Oz_i sz_i + (W_i |r><1|_i + h.c.) - Delta_i n_i ]
 *        + sum_{i<j} V_ij n_i n_j ,          V_ij = C6 / d_ij^6        (Eq. 1, Eq. 2)
 *
 * with W_i = Omega^R_i exp(i phase_i), sx = |0><1| + |1><0|, sz = |0><0| - |1><1|,
 * n = |r><r|.  The detuning term -Delta n is the CZ pulse's detuning of
 * Sec. "Compiler for global GHZ states", which Eq. 1 does not print.  Eq. 2
 * prints V = -C6/d^6: here C6 is passed with its sign and V_ij = C6/d_ij^6.
 *
 * Conventions for every call.
 *  - Host arrays passed in are owned by the caller and copied before return.
 *  - The context owns all device memory; nothing is shared between contexts.
 *  - Work is issued on the context's stream (ttn_set_stream); calls that
 *    return host scalars synchronise that stream.
 *  - No call throws.  Each returns a ttn_status; on error the context keeps a
 *    message (ttn_last_error).  Invalid arguments return TTN_ERR_ARG and leave
 *    the context unchanged.  Device-side numerical failures (NaN/Inf) are
 *    reported as TTN_ERR_NUMERIC at the next synchronising call.
 *  - Complex numbers are interleaved (re, im) doubles.
 *  - Atom i sits at lattice site (i % Lx, i / Lx).
 *  - Node numbering: level-0 nodes (pairs of leaves 2j, 2j+1) first, left to
 *    right, then level 1, ..., the root last.  Node k has legs
 *    (child 0, child 1, parent) with dims (d0, d1, d2); the root's parent leg
 *    is a dummy leg of dim 1.  A node tensor X is stored with
 *    X(a, b, c) at index a + d0*(b + d1*c) (child 0 fastest).
 *  - Bond dimension of the parent leg of a node whose subtree holds the real
 *    atom set S: min(chi, 3^|S|, 3^(N - |S|)).  Leaves are padded to a power
 *    of two; padding leaves hold no atom, stay in |0> and carry no term
 *    (Sec. "Parallel quantum algorithms").
 */
#ifndef TTN_H
#define TTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttn_ctx ttn_ctx;

typedef enum {
    TTN_OK = 0,
    TTN_ERR_ARG = 1,      /* invalid argument; nothing changed                  */
    TTN_ERR_ALLOC = 2,    /* device or host allocation failed                   */
    TTN_ERR_CUDA = 3,     /* a CUDA runtime call failed (message has the name)  */
    TTN_ERR_KRYLOV = 4,   /* Lanczos did not reach its tolerance in m_max steps */
    TTN_ERR_NUMERIC = 5,  /* NaN or Inf met in the state                        */
    TTN_ERR_TIMEOUT = 6,  /* a bounded device-side wait gave up                 */
    TTN_ERR_STATE = 7     /* call not valid in the current state                */
} ttn_status;

typedef enum {
    TTN_FP64 = 0,         /* all contractions in FP64 (complex128)              */
    TTN_SPLIT_TF32X3 = 1  /* H_eff and environment contractions as split-TF32
                             tensor-core GEMMs (3 products, FP32 accumulate);
                             Lanczos, tridiagonal exponential and QR stay FP64  */
} ttn_precision;

/* One piecewise-constant drive segment of one atom, active on [t0, t1).
 * Active segments of the same atom add up.  Layout: 64 bytes. */
typedef struct {
    int32_t atom;
    double t0, t1;
    double omega_x;   /* coefficient of sx                       */
    double omega_z;   /* coefficient of sz                       */
    double omega_r;   /* Omega^R of Omega^R e^{i phase}|r><1| + h.c. */
    double phase_r;
    double delta;     /* coefficient of -n                       */
} ttn_pulse;

/* Create a context for an Lx x Ly lattice of atoms with `levels` local states
 * (must be 3) and maximal bond dimension chi >= 1.  The state starts as
 * |0...0>, the Hamiltonian as H = 0 (unit square positions, C6 = 0), internal
 * time t = 0, precision TTN_FP64, the stream the legacy default stream.
 * Lx*Ly must be in [1, 1024].  *out receives the context or NULL. */
ttn_status ttn_create(int Lx, int Ly, int levels, int chi, ttn_ctx** out);
void ttn_destroy(ttn_ctx* ctx);
const char* ttn_last_error(const ttn_ctx* ctx);

/* Issue all later work on this CUDA stream (a cudaStream_t, e.g. PyTorch's
 * current stream); NULL selects the legacy default stream. */
ttn_status ttn_set_stream(ttn_ctx* ctx, void* cuda_stream);
ttn_status ttn_set_precision(ttn_ctx* ctx, ttn_precision p);

/* Positions xy (N x 2 doubles, atom-major), pair coefficient C6 (signed,
 * V_ij = C6/d_ij^6, Eq. 2) and interaction radius r_cut: pairs farther apart
 * than r_cut are dropped (the radius r_I = r_G + d_off of Sec. "Tensor network
 * simulations"); r_cut <= 0 keeps all pairs.  Coincident positions or
 * non-finite values -> TTN_ERR_ARG.  Rebuilds the environments. */
ttn_status ttn_set_hamiltonian(ttn_ctx* ctx, const double* xy, double C6, double r_cut);

/* Open system (Eq. 3, Sec. "Modeling 88Sr quantum computers"): evolve with
 * H_OQS = H - i gamma sum_i n_i, the no-jump evolution of a decay from |r>
 * to states outside the computational space.  The norm then decreases,
 * d<psi|psi>/dt = -2 gamma sum_i <psi|n_i|psi> (so the lost norm measures the
 * integrated Rydberg time T_R), and every local exponential runs as an
 * Arnoldi iteration instead of Lanczos.  gamma = 0 (the default) is the
 * closed system; gamma < 0 or non-finite -> TTN_ERR_ARG. */
ttn_status ttn_set_decay(ttn_ctx* ctx, double gamma);

/* Replace the drive schedule by n_segments segments (copied).  Atoms outside
 * [0, N) or t1 < t0 -> TTN_ERR_ARG.  Drives are evaluated at the midpoint of
 * each TDVP step (Sec. "Tensor network simulations": per-layer control). */
ttn_status ttn_apply_pulse(ttn_ctx* ctx, const ttn_pulse* schedule, int n_segments);

/* Set the state to a product state: amps holds N x 3 complex amplitudes
 * (interleaved, atom-major, level order |0>,|1>,|r>).  Bond bases are filled
 * by the deterministic completion rule; the centre is at the root.  Resets
 * the internal time to 0. */
ttn_status ttn_set_product_state(ttn_ctx* ctx, const double* amps);

/* Set the state of ctx to (|0..0> + e^{i phase} |m>)/sqrt2 where |m> has the
 * atoms with mask[i] != 0 in |1> and the others in |0>: the exact bond-
 * dimension-2 TTN of the GHZ target (Sec. "Tensor network simulations"). */
ttn_status ttn_set_ghz_target(ttn_ctx* ctx, const int* mask, double phase);

/* One second-order TDVP step of length dt > 0 at H(t + dt/2), advancing the
 * internal time t by dt.  Sweep: forward half-sweep with dt/2 (children first,
 * links evolved backwards on the way up) followed by its reverse. */
ttn_status ttn_tdvp_step(ttn_ctx* ctx, double dt);

/* F = |<target|psi>|^2 (unnormalised, Sec. "Parallel quantum algorithms").
 * target must have the same lattice; its chi may differ. */
ttn_status ttn_fidelity(ttn_ctx* ctx, const ttn_ctx* target, double* F);
/* <target|psi> as a complex number (2 doubles). */
ttn_status ttn_overlap(ttn_ctx* ctx, const ttn_ctx* target, double* re_im);

/* Per-atom expectation values (N doubles): which = 0 -> <|0><0|>,
 * 1 -> <|1><1|>, 2 -> <n> = <|r><r|> (P_R of Sec. "Modeling 88Sr quantum
 * computers" is their sum). */
ttn_status ttn_measure(ttn_ctx* ctx, int which, double* out);
ttn_status ttn_norm(ttn_ctx* ctx, double* out);      /* <psi|psi>                 */
ttn_status ttn_energy(ttn_ctx* ctx, double* out);    /* <psi|H(t)|psi>, current t */
ttn_status ttn_get_time(ttn_ctx* ctx, double* t);

/* Full state vector (3^N complex, index sum_i s_i 3^i) for N <= 9. */
ttn_status ttn_get_dense(ttn_ctx* ctx, double* psi);

/* Save / load the tree state (node tensors, time, chi, lattice) to a file.
 * Load needs a context with the same lattice and chi. */
ttn_status ttn_save(ttn_ctx* ctx, const char* path);
ttn_status ttn_load(ttn_ctx* ctx, const char* path);

/* Truncate the state of src to the bond dimensions of dst (Sec. "Tensor
 * network simulations": the bond dimension chi controls the kept
 * entanglement): dst must have the same lattice and no bond larger than
 * src's.  Every bond is projected on the top eigenvectors of its bond Gram
 * (the Schmidt basis of the bipartition the bond cuts, from the canonical
 * form of src), all at once, computed on the GPU by one-sided Jacobi; dst is
 * then brought to canonical form by QR.  dst's Hamiltonian and schedule are
 * its own; its time is set to src's.  discarded (may be NULL) receives 2
 * doubles: the sum over bonds and the largest of the discarded weights
 * (dropped eigenvalues / trace of the bond density matrix).  The infidelity
 * of the truncation is at most (sum_bonds sqrt(weight))^2.  src keeps its
 * state (its centre moves to the root); after an error dst's state is
 * undefined. */
ttn_status ttn_compress(ttn_ctx* src, ttn_ctx* dst, double* discarded);

/* Projective measurement of every atom in the {|0>, |1>, |r>} basis, n_shots
 * times (Sec. "Parallel quantum algorithms": measurement histograms of many
 * shots).  Each shot measures the atoms one after another in the tree's leaf
 * order (ttn_leaf_atoms, padding leaves skipped) and draws atom i's outcome
 * from its conditional distribution given the outcomes already drawn, by
 * inverse transform sampling: outcome s is the first level with
 * u < (P(0) + ... + P(s)) / (P(0) + P(1) + P(2)).
 *   uniforms : host, n_shots x N doubles in [0, 1), row-major, column j the
 *              j-th real atom in leaf order (the caller draws them; equal
 *              uniforms give equal outcomes on equal states);
 *   outcomes : host, n_shots x N ints (0: |0>, 1: |1>, 2: |r>), column =
 *              atom id.
 * The walk runs on the GPU, batched over shots: depth first, entering a
 * subtree with the Gram of its conditioned complement and leaving it with
 * the amplitude vector of its drawn outcomes.  The contractions use the
 * context's precision (split precision can flip a draw whose uniform lies
 * within ~1e-7 of a boundary).  Moves the orthogonality centre to the root
 * (the state is unchanged).  n_shots = 0 does nothing; n_shots < 0, NULL
 * buffers -> TTN_ERR_ARG; allocation failure -> TTN_ERR_ALLOC. */
ttn_status ttn_sample(ttn_ctx* ctx, const double* uniforms, int n_shots, int* outcomes);

/* Gradient of the final-state fidelity F = |<target|psi(t0 + n_steps dt)>|^2
 * with respect to piecewise-constant pulse parameters (the differentiation
 * extension: pulse amplitudes Omega_k and detunings Delta_k of schedule rows
 * of ttn_apply_pulse), starting from the context's current state at its
 * current time t0.  Parameter p is field fields[p] (0: omega_r, the |r><1|
 * coupling with dH = e^{i phase_r}|r><1| + h.c. on the row's atom; 1: delta,
 * dH = -|r><r|) of schedule row rows[p].
 * Method (adjoint of the time-stepping map): with U_n the n-th step and
 * chi_n = U_{n+1}^H ... U_N^H |target>,
 *   dF/dtheta = 2 Re( conj(A) sum_n <chi_n| dU_n/dtheta |psi_{n-1}> ),
 *   <chi_n| dU_n |psi_{n-1}> = -i int_0^dt <chi(s)| dH |psi(s)> ds,
 * psi(s) = e^{-isH} psi_{n-1}, chi(s) = e^{+i(dt-s)H} chi_n, the integral by
 * n_quad-point Gauss-Legendre (1..8) on TDVP sub-steps of the same step
 * Hamiltonian, the matrix elements from transition reduced density matrices
 * of every atom (overlap environments of the two trees, FP64).  chi is
 * propagated backwards by TDVP steps of -dt; psi is recomputed from
 * checkpoints taken every `checkpoint_every` steps (<= 0: about
 * sqrt(n_steps)), so device memory grows with n_steps / checkpoint_every
 * copies of the state.  Where the bonds are complete (every TDVP projector
 * is the identity) this is the gradient of the exact discrete map up to the
 * quadrature error; in the truncated regime it is the adjoint of the
 * projected dynamics, not the derivative of the discrete TDVP map (which
 * also varies through the gauge and the projectors).
 *   target : same lattice and bond dimension, centre at its root;
 *   F, grad: host, 1 and n_params doubles.
 * The context's state and time are restored on success (after an error they
 * are undefined: reload or reset the state).  No decay (gamma must
 * be 0), n_steps >= 1, dt > 0, rows inside the schedule, fields 0 or 1,
 * 1 <= n_quad <= 8, else TTN_ERR_ARG. */
ttn_status ttn_fidelity_gradient(ttn_ctx* ctx, const ttn_ctx* target, double dt, int n_steps, int n_params,
                                 const int* rows, const int* fields, int n_quad, int checkpoint_every,
                                 double* F, double* grad);

/* ---- introspection used by tests and tools ------------------------------ */
ttn_status ttn_num_nodes(const ttn_ctx* ctx, int* n);
/* dims[3] = (d0, d1, d2); children[2] = child node ids, or -(leaf+1) for a leaf. */
ttn_status ttn_node_info(const ttn_ctx* ctx, int node, int* dims, int* children);
/* leaf_atom[n_leaves]: atom id per leaf in Hilbert order, -1 for padding. */
ttn_status ttn_leaf_atoms(const ttn_ctx* ctx, int* leaf_atom, int* n_leaves);
/* Copy node tensor to / from host (d0*d1*d2 complex).  ttn_set_node leaves
 * the environments stale until ttn_refresh_envs; callers that set every node
 * must keep the canonical form (non-root nodes isometric towards the root). */
ttn_status ttn_get_node(ttn_ctx* ctx, int node, double* data);
ttn_status ttn_set_node(ttn_ctx* ctx, int node, const double* data);
/* Rebuild every upward environment from the current node tensors (centre at
 * the root).  Needed after ttn_set_node. */
ttn_status ttn_refresh_envs(ttn_ctx* ctx);

/* Y = H_eff(node) X for the centre at `node`: moves the orthogonality centre
 * to `node` (gauge moves only, the state is unchanged), then applies the
 * effective Hamiltonian of the node at H(t) to the host tensor x (same shape
 * as the node) and writes y.  Used to check the contraction element by
 * element.  The centre stays at `node` until the next step or observable,
 * which move it back to the root. */
ttn_status ttn_apply_heff(ttn_ctx* ctx, int node, const double* x, double* y);

/* Counters since the last ttn_reset_stats: [0] Krylov runs, [1] Krylov
 * matvecs, [2] max Krylov error estimate (as double bits), [3] kernel launches
 * issued by the library, [4] QR calls, [5] dependent columns completed. */
ttn_status ttn_get_stats(const ttn_ctx* ctx, int64_t* out6);

/* Kernel-level timing with CUDA events recorded on the context's stream.
 * Between begin and end every contraction launch, every QR and every group of
 * Krylov vector kernels is bracketed by an event pair.  ttn_profile_end
 * synchronises and fills out[4 * min(6, n / 4)] with, for kind k = 0
 * tensor-core GEMM (tcgen05), 1 split-operand packing, 2 FP64 GEMM, 3 QR,
 * 4 Krylov vector work (re-orthogonalisation, scalars, combination, one-block
 * runs of small nodes), 5 the other element-wise kernels of the sweep (block
 * assembly, leg permutations, absorb norms): out[4k + 0] event
 * pairs, [4k + 1] summed device time
 * in ms, [4k + 2] algorithmic flops (8 M N K per complex contraction;
 * 16 M D^2 per QR), [4k + 3] algorithmic bytes.  n must be >= 16 (kinds that
 * do not fit are left out). */
ttn_status ttn_profile_begin(ttn_ctx* ctx);
/* Self-test of one contraction kernel, no context needed: seeded random
 * complex A (M x K) and B (K x N) with entries uniform in [-1, 1)^2
 * (truncated to 11 significant bits when tf32_exact != 0, which isolates the
 * accumulation error), C = A B by the FP64 kernel and by `precision`;
 * *rel_err receives max|C_p - C_fp64| / max|C_fp64|.  Sizes above 2^26
 * elements -> TTN_ERR_ARG. */
ttn_status ttn_selftest_contract(int M, int N, int K, int precision, unsigned long long seed,
                                 int tf32_exact, double* rel_err);
ttn_status ttn_profile_end(ttn_ctx* ctx, double* out, int n);
/* Self-test and timing hook of the gauge-move QR (Sec. "Tensor network
 * simulations": the orthogonality centre moves by a QR of the node tensor),
 * no context needed.  A (host, M x D complex as interleaved (re, im) doubles,
 * column-major, lda = M, M >= D, D <= 256, M * D <= 2^26) is copied to the
 * device and factorised there as A = Q R by CGS2 with the deterministic
 * completion of dependent columns (residual <= 1e-10 ||A||_F; candidates
 * cand[0..ncand) in order, or rows 0..M-1 when cand is NULL); Q (M x D) and
 * R (D x D, upper triangular, real non-negative diagonal) are written to host
 * buffers of the caller; *n_dependent (may be NULL) receives the number of
 * completed columns and *ms (may be NULL) the device time of the
 * factorisation.  Bad sizes or candidate rows -> TTN_ERR_ARG. */
ttn_status ttn_selftest_qr(const double* A, int M, int D, const int* cand, int ncand, double* Q, double* R,
                           int* n_dependent, float* ms);
/* Per-launch records of the last profile: 7 doubles each (kind, M, N, K,
 * batches, ms, algorithmic flops; K and batches are the products of the
 * two-level extents; for a QR record: kind 3, rows, columns, dependent
 * columns, 1).  *n_records receives the count; at most max_records
 * are written to out (which may be NULL to query the count). */
ttn_status ttn_profile_records(const ttn_ctx* ctx, double* out, int max_records, int* n_records);
ttn_status ttn_reset_stats(ttn_ctx* ctx);

/* Self-test of the contraction kernels on host data, no context needed:
 * C = A B with A (M x K), B (K x N) and C (M x N) complex, column-major,
 * interleaved (re, im) doubles in caller-owned host memory.  precision
 * TTN_FP64 runs the FP64 kernel; TTN_SPLIT_TF32X3 runs the split-precision
 * tensor-core path when the shape fills its tiles (else the FP64 kernel).
 * *path (may be NULL) receives 1 when the tensor-core path ran, else 0; *ms
 * (may be NULL) the device time of the contraction.  Sizes above 2^26
 * elements per matrix -> TTN_ERR_ARG; a tensor-core wait that gave up ->
 * TTN_ERR_TIMEOUT. */
ttn_status ttn_selftest_contract_host(const double* A, const double* B, double* C, int M, int N, int K,
                                      int precision, int* path, float* ms);

/* Truncated singular value decomposition of a bond matrix, no context needed
 * (Sec. "Tensor network simulations": the bond dimension chi caps the kept
 * singular values; discarding sigma_i < eps * sigma_max as well).
 * A: host, M x N complex (interleaved, column-major, lda = M), M >= N,
 * 1 <= N <= 256, M * N <= 2^26.  On the device: A = Q R (the gauge-move QR
 * with its deterministic completion), a one-sided Jacobi SVD of R, U = Q U_R.
 * Keeps k = min(chi, #{sigma_i >= eps sigma_max}) (at least 1) values in
 * descending order: U (M x k), S (k doubles), Vh (k x N, column-major, the
 * conjugate transpose of V's kept columns), so that A ~ U diag(S) Vh; the
 * caller's buffers must hold min(chi, N) columns/values.  *k_out receives k,
 * *discarded (may be NULL) the discarded weight sum_{i >= k} sigma_i^2 /
 * sum_i sigma_i^2.  Bad sizes -> TTN_ERR_ARG; a grid-barrier wait that gave
 * up -> TTN_ERR_TIMEOUT. */
ttn_status ttn_svd_truncate(const double* A, int M, int N, int chi, double eps, double* U, double* S, double* Vh,
                            int* k_out, double* discarded);

/* FP64 throughput probe, no context needed: method 0 runs independent FP64
 * fused multiply-add chains on every SM (the FP64 ALU, DFMA), method 1 chains
 * of FP64 tensor-core instructions (mma.sync m8n8k4 f64, DMMA); *tflops
 * receives the measured rate (2 flops per FMA).  The roofline of every FP64
 * step (QR, Lanczos re-orthogonalisation, FP64 contractions) is set by this
 * rate on GB300, not by HBM. */
ttn_status ttn_selftest_fp64_peak(int method, double* tflops);

/* Test hooks: host-side fault injection for the failure-detection tests (no
 * GPU is faulted; every injected failure goes through a bounded path):
 *   TTN_INJECT_TC_STALL    the next `value` tensor-core contractions make
 *                          their drain warps wait on a barrier that nothing
 *                          arrives at; the wait gives up after 1 ms and the
 *                          launch aborts as on a real timeout (the caller sees
 *                          TTN_ERR_TIMEOUT);
 *   TTN_INJECT_KRYLOV_MMAX Krylov dimension capped at `value` (1..30; 0
 *                          restores 30): a step that needs more returns
 *                          TTN_ERR_KRYLOV;
 *   TTN_INJECT_ALLOC_FAIL  the next `value` device allocations fail
 *                          (TTN_ERR_ALLOC);
 *   TTN_INJECT_NONE        clears every hook.
 * Hooks are process-wide.  Bad kind or value -> TTN_ERR_ARG. */
enum { TTN_INJECT_NONE = 0, TTN_INJECT_TC_STALL = 1, TTN_INJECT_KRYLOV_MMAX = 2, TTN_INJECT_ALLOC_FAIL = 3 };
ttn_status ttn_test_inject(int kind, long long value);

/* ---- allocation-free contraction ----------------------------------------
 * The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory at the point of the call (a host program whose
 * memory is owned by its own pool or a fixed budget, or code that must not
 * call cudaMalloc/cudaFree because they synchronise the device).
 *
 * C = A B for complex matrices in device memory, column-major, interleaved
 * (re, im) doubles: A is M x K (lda = M), B is K x N (ldb = K), C is M x N
 * (ldc = M), caller-allocated; C is overwritten.  It runs the split-precision
 * tensor-core contraction (3xTF32, ~5e-7 of max|C|) when the shape fills the
 * tensor-core tiles, else the FP64 kernel (also when the driver offers no
 * tensor-map encoder), on `stream` (a cudaStream_t, NULL for the legacy
 * default stream), and returns once the contraction has finished: it
 * synchronises `stream`, so that it can report the outcome.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  The packed
 * operands live in one file-scope device array of 8 MiB, which every GPU that
 * loads this library holds until the process exits; a shape whose packed
 * operands need more (about 2 * (round_up(max(M,N), 128) + round_up(
 * 2 min(M,N), 64)) * round_up(2K, 32) * 4 bytes) returns TTN_ERR_ARG and does
 * nothing.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call shares the one array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Errors: TTN_ERR_ARG for null pointers, non-positive or too large sizes;
 * TTN_ERR_CUDA if a launch or the synchronisation fails; TTN_ERR_TIMEOUT if a
 * bounded wait of the tensor-core pipeline gave up (C is then undefined; the
 * error word in the scratch array is cleared, so the next call starts
 * clean). */
ttn_status ttn_contract_split_noalloc(const double* A, const double* B, double* C, int M, int N, int K,
                                      void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TTN_H */
