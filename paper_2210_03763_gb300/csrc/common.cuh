// Internal declarations shared by the CUDA translation units of libttn.
// Not part of the ABI (include/ttn.h is).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

typedef double2 cplx;   // (re, im)

// Generic strided complex contraction, the one primitive every tensor
// contraction of the TDVP update is mapped to:
//   C[b](m, n) = alpha * sum_k op(A)[b](m, k) * op(B)[b](k, n) + beta * C[b](m, n)
// with k = ki + Ki*ko and b = bi + Bi*bo, each index with its own stride
// (in complex elements).  op = identity or complex conjugation.
struct GemmArgs {
    int M, N, Ki, Ko, Bi, Bo;
    const cplx* A; long long a_m, a_ki, a_ko, a_bi, a_bo; int conjA;
    const cplx* B; long long b_ki, b_ko, b_n, b_bi, b_bo; int conjB;
    cplx* C; long long c_m, c_n, c_bi, c_bo;
    cplx alpha, beta;
};

// Launch on `stream`; returns the number of kernels launched (0 if empty).
// With a workspace of f64_workspace_bytes(g), contractions whose output
// tiles cannot fill the GPU split K into ranges summed in fixed order.
int launch_zgemm_f64(const GemmArgs& g, cudaStream_t stream, void* workspace = nullptr, size_t workspace_bytes = 0);
size_t f64_workspace_bytes(const GemmArgs& g);

// ---- split-precision building blocks (gemm_split.cu) -------------------------
// Packing of one side of a split contraction into TF32 hi/lo planes: complex
// element (row r, k, batch bi, bo) of src (strides s_r, s_ki (k % Ki),
// s_ko (k / Ki), s_bi, s_bo) goes to real row (embed ? 2r : r) + bi*rb_i +
// bo*rb_o, floats k_off + 2k of a row `pitch` floats long; embed = 1 is the
// real embedding of the Q side (rows (Re, -Im) and (Im, Re)).  Rows
// r in [R, Rpad) and k in [Ki*Ko, Kc) are written as zeros.
struct SplitPackArgs {
    const cplx* src;
    long long s_r, s_ki, s_ko, s_bi, s_bo;
    int R, Ki, Ko, Bi, Bo;
    int conj, embed;
    int Rpad, Kc;
    long long rb_i, rb_o;
    long long pitch, k_off;
    float* hi;
    float* lo;
};
int split_pack(const SplitPackArgs& p, cudaStream_t stream);

// Packed output of a split contraction: the epilogue writes TF32 hi/lo
// planes (as split_pack with embed = 0) at float2 position
// (p % pd)*sp1 + (p / pd)*sp2 + q*sq + bi*sbi + bo*sbo for output (P row p,
// Q row q, batch bi, bo); hi/lo already offset to the first slot.  Writes
// are coalesced when sp1 = 1 (consecutive P rows land next to each other).
struct SplitOut {
    float* hi;
    float* lo;
    int pd;
    long long sp1, sp2, sq, sbi, sbo;
};

// One split contraction on packed planes: C(p, q) = alpha sum_k P(p, k) Q(q, k)
// + beta C(p, q) per batch (bi, bo), P rows in tiles of 128, Q the embedded
// side (2 real rows per complex row, tiles of 64).  Kp: K' in floats (a
// multiple of 32), the same for both sides.
struct SplitMma {
    const float* Ph;
    const float* Pl;
    long long P_rows, P_pitch;   // rows in the planes, floats per row
    const float* Qh;
    const float* Ql;
    long long Q_rows, Q_pitch;
    int Kp;
    int Pn, Qn;                  // valid complex rows of P and Q per batch
    int Pp, Qp;                  // padded real rows of the tile grid per batch
    int Bi, Bo;
    long long p_sbi, p_sbo, q_sbi, q_sbo;   // real-row offsets of batch (bi, bo)
    cplx* C;
    long long c_p, c_q, c_bi, c_bo;
    int c_pd;                    // > 0: P row offset (p % c_pd)*c_p + (p / c_pd)*c_p2
    long long c_p2;
    cplx alpha, beta;
    const SplitOut* out;         // non-null: packed output (alpha = 1, beta = 0)
    int max_split;               // split-K cap (1: none; forced to 1 with `out`)
};
constexpr int SPLIT_BM = 128, SPLIT_BN = 64, SPLIT_BK = 32;
// bytes of split-K partial sums the contraction needs (0: no split-K)
size_t split_mma_partials(const SplitMma& m);
// Returns kernels launched, -1 on a bad shape or tensor map, -2 on missing
// workspace.  err_flag: the int a timed-out wait sets.
int split_mma(const SplitMma& m, int* err_flag, void* partials, size_t partial_bytes, cudaStream_t stream);
// Split-precision tensor-core path (3xTF32 on tcgen05).  Returns kernels
// launched, -1 when the shape is not handled there (too small: the caller
// uses FP64), -2 when the workspace is smaller than split_workspace_bytes.
// The workspace's first int is an error flag a timed-out wait sets.
int launch_zgemm_split(const GemmArgs& g, cudaStream_t stream, void* workspace,
                       size_t workspace_bytes);
// max_split caps split-K (K ranges per output tile, used when the tiles
// cannot fill the GPU; partial sums then live in the workspace and a second
// kernel adds them in fixed order).  1 disables it.
constexpr int SPLIT_K_MAX = 1 << 20;
size_t split_workspace_bytes(const GemmArgs& g, int max_split = SPLIT_K_MAX);
int launch_split_pack(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes,
                      int max_split = SPLIT_K_MAX);
int launch_split_mma(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes,
                     int max_split = SPLIT_K_MAX);

// ---- Lanczos / vector kernels (kernels.cu) --------------------------------
// Fixed partial-sum grid for reductions: deterministic order, no atomics.
constexpr int RED_BLOCKS = 304;     // 2 x 152 SMs
constexpr int RED_THREADS = 256;
constexpr int KRYLOV_MMAX = 30;

struct KrylovScalars {
    double alpha[KRYLOV_MMAX];
    double beta[KRYLOV_MMAX + 1];
    cplx   h[KRYLOV_MMAX + 1];      // projections of the current pass
    cplx   c[KRYLOV_MMAX];          // exp(z T_j) e_1
    double nrm0;                    // norm of the start vector
    double inv_scale;               // 1 / beta_j used to normalise v_{j+1}
    double err;                     // a-posteriori error estimate
    int    converged;
    int    nonfinite;
    cplx   hess[KRYLOV_MMAX + 1][KRYLOV_MMAX];   // Arnoldi: Hessenberg matrix H(i, j) at [i][j]
};

int red_blocks_for(long long n);
int k_norm2_partial(const cplx* x, long long n, double* partial, cudaStream_t s);
int k_dots_scaled(cplx* V, long long ld, int nv, const cplx* w, long long n, cplx* partial, int scale_col,
                  const double* scale_src, long long skip_col, cudaStream_t s);
// h = fixed-order sum of partial_in; w -= sum_i V_i h_i; then mode 1: partial
// dots of the new w with V_0..V_{nv-1}, mode 2: partial norm^2 of the new w.
int k_orth_update_ex(const cplx* V, long long ld, int nv, const cplx* partial_in, cplx* w, long long n,
                     int mode, cplx* partial_dots, double* partial_norm, cplx* h_out, int accumulate,
                     long long skip_col, cudaStream_t s);
int k_scale_copy_dev(const cplx* x, long long n, const double* scale, cplx* y, cudaStream_t s);
// x <- x * sqrt(sum pr / sum px) with px, pr norm^2 partials (k_norm2_partial)
int k_rescale_to_norm(cplx* x, long long n, const double* px, int Gx, const double* pr, int Gr, cudaStream_t s);
int k_krylov_start_ex(KrylovScalars* ks, const double* nrm2_partial, long long n, cudaStream_t s);
int k_krylov_scalars_ex(KrylovScalars* ks, const cplx* h1, const cplx* h2, const double* beta_partial,
                        long long n, int j, double zr, double zi, double tol, cudaStream_t s);
// Arnoldi step j for a non-Hermitian generator (the decay of Eq. 3): column j
// of the Hessenberg matrix is h1 + h2, H(j+1, j) = beta_j; c = exp(z H_j) e_1.
int k_arnoldi_scalars(KrylovScalars* ks, const cplx* h1, const cplx* h2, const double* beta_partial, long long n,
                      int j, double zr, double zi, double tol, cudaStream_t s);
int k_combine(const cplx* V, long long ld, int nv, const KrylovScalars* ks, cplx* y,
              long long n, cudaStream_t s);

// ---- small nodes: the whole Krylov exponential in one block -------------------
// Nodes and links with s <= SMALL_S tensor entries: H_eff as a dense s x s
// matrix, then Lanczos/Arnoldi, exponential and combination in one launch.
constexpr int SMALL_S = 96;
struct SmallPairs {      // channel pairs of a small H_eff (by value into the kernel)
    int np;
    int a[3], b[3], r[3];
    const cplx* Na[3];   // r matrices of D_a^2
    const cplx* G[3];    // r matrices of D_b^2
};
int k_dense_heff(cplx* H, const int* d, const cplx* hb0, const cplx* hb1, const cplx* hb2, const SmallPairs& pp,
                 cudaStream_t s);
// status in ks: converged, nonfinite, err; alpha[0] = iterations
int k_small_krylov(const cplx* H, int n, cplx* x, double zr, double zi, double tol, int mmax, int arnoldi,
                   KrylovScalars* ks, cudaStream_t s);

// ---- elementwise / assembly ---------------------------------------------------
int k_permute3(const cplx* x, cplx* y, int d0, int d1, int d2, int p0, int p1, int p2,
               int inverse, cudaStream_t s);
int k_fill(cplx* x, long long n, cplx v, cudaStream_t s);
// H = Hs + sum_i coef_i-weighted drive ops (see kernels.cu)
// (gamma: decay of Eq. 3, adds -i gamma n_i for every site)
int k_assemble_block(cplx* H, const cplx* Hs, int D, const cplx* nops, int nsites,
                     const int* site_ids, const cplx* dops, int ndriven,
                     const int* driven_ids, const double* coef, double gamma, cudaStream_t s);
int k_check_finite(const cplx* x, long long n, int* flag, cudaStream_t s);
double k_fp64_probe(int method, int blocks, int iters, double* out, cudaStream_t s);
// G_i = sum_j W[j + nb*i] N_j, i < r (N: nb matrices of n entries, contiguous;
// W real)
int k_weighted_sum(const cplx* N, int nb, long long n, const double* W, int r, cplx* G, cudaStream_t s);

// ---- QR (qr.cu) ----------------------------------------------------------------
// QR kernels use one block per QR_ROWS rows; partial sums are sized
// G = ceil(M / QR_ROWS) per column (part: 2 * G * (D + 1) complex), and the
// Frobenius pass uses up to QR_FROB_BLOCKS partials (pnorm >= max of both).
constexpr int QR_ROWS = 128;
constexpr int QR_FROB_BLOCKS = 1024;
struct QrScratch {
    cplx* part;         // 2 * row blocks * (2 * MAX_CHI + 4) partial sums
    cplx* h;            // 2 * (D + 2) projection coefficients
    double* pnorm;      // RED_BLOCKS partial norms
    double* scal;       // scalars: [0] ||A||_F^2, [1] current column norm, ...
    int* flags;         // per-column dependent flags (D)
    double* rownorm;    // M row norms of Q (completion)
    int* cand;          // candidate order (M)
    int* pick;          // chosen candidate
    // structured completion
    int* kept;          // D: kept column positions
    int* dep;           // D: dependent column positions
    int* acc_rows;      // D: accepted candidate row per completed column
    cplx* Y;            // QR_SC_MAXR * D: coefficients y_t
    double* nu;         // D: residual norms
    int* row_rank;      // M: step at which a row was accepted (INT_MAX: never)
    int* cand_used;     // M: candidate accepted flags
    unsigned* bar;      // 2: grid barrier of the cooperative column loop
    int* err;           // set when a bounded device wait gave up
};
constexpr int QR_SC_MAXR = 64;   // structured completion when the kept rank r <= this
// In-place QR of the column-major M x D matrix A (lda = M): A <- Q, R (D x D,
// column-major) written.  cand[0..ncand) is the completion candidate order.
// Returns the number of kernels launched, or -1 when a bounded device wait
// of the cooperative column loop gave up (A and R are then undefined).
// tol: a column is dependent when its residual is <= tol ||A||_F (the
// dependence threshold of the completion rule, 1e-10 for every QR of the
// library).
constexpr double QR_TOL_FP64 = 1e-10;
int qr_cgs2(cplx* A, int M, int D, cplx* R, const int* cand, int ncand,
            QrScratch& ws, cudaStream_t s, int* n_dependent_host, double tol = QR_TOL_FP64);

// ---- truncated SVD (svd.cu) -----------------------------------------------------
// One-sided Jacobi SVD of the N x N column-major R (N <= 256) in place: R's
// columns end mutually orthogonal, V (N x N) accumulates the rotations
// (R_in V = R_out).  One cooperative launch; bar: 2 unsigned, err: set when a
// grid-barrier wait gave up; info[0]: sweeps run.  Returns launches, -1 if
// the cooperative launch failed.
int svd_jacobi_square(cplx* R, cplx* V, int N, int max_sweeps, double tol, unsigned* bar, int* err, int* info,
                      cudaStream_t s);
// sigma_i = |r_i|, descending order, kept k = min(chi, #{sigma >= eps sigma_max})
// (at least 1; eps < 0: exactly min(chi, N), zero values included),
// discarded weight sum_{t >= k} sigma^2 / sum sigma^2;
// Ur (N x k) = normalised kept columns, Vh (k x N) = their conj(V) rows.
int svd_finish(const cplx* R, const cplx* V, int N, int chi, double eps, cplx* Ur, cplx* Vh, double* S, int* k,
               double* disc, int* order, cudaStream_t s);

// ---- measurement sampling (sample.cu) ---------------------------------------------
// S shots, one matrix / vector per shot at stride ld (complex):
// G_b /= max(Re tr G_b, 1e-300); w_b /= |w_b| (when nonzero); the draw of one
// leaf (atom < 0: padding, outcome 0 without a uniform) from diag(G_b) (3 x 3,
// stride 9) with uniform U[b * ldu + j], outcome into out[b * N + atom],
// w_b (stride 3) = e_outcome.
int k_trace_normalize(cplx* G, int D, long long ld, int S, cudaStream_t s);
int k_vec_normalize(cplx* w, int D, long long ld, int S, cudaStream_t s);
int k_leaf_draw(const cplx* G, const double* U, long long ldu, int j, int atom, int* out, int N, cplx* w, int S,
                cudaStream_t s);

// ---- test hooks (ttn_test_inject in ttn.cu) -----------------------------------
// Stall time in ns for the next tensor-core launch (0: none; consumes one
// pending stall), the Krylov dimension cap (KRYLOV_MMAX unless lowered) and
// whether the next device allocation is to fail (consumes one).
unsigned long long test_take_tc_stall();
int test_krylov_mmax();
bool test_take_alloc_fail();

#define TTN_LAUNCH_CHECK() (cudaGetLastError())
