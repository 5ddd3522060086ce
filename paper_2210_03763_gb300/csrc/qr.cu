// QR of the tall matricisation of a node tensor (the gauge move of the TDVP
// sweep, Sec. "Tensor network simulations"), FP64.
//
// Column-by-column classical Gram-Schmidt with one re-orthogonalisation pass
// (CGS2), in place on a column-major M x D matrix.  Column k is *dependent*
// when the norm of its residual after both passes is <= tol ||A||_F (1e-10
// unless the caller passes another threshold); it is
// zeroed (R_kk = 0) and filled after the sweep, in increasing k, by the first
// candidate unit vector e_c (in the caller's candidate order) whose residual
// 1 - ||Q^H e_c||^2 is >= 1/4 (else the candidate with the largest residual,
// earliest on ties), orthogonalised twice against Q and normalised.  R_kk is
// real and >= 0; rows of R of dependent columns are zero.
//
// GB300's FP64 pipe (~7.8 GFLOP/s per SM) bounds this code at full rank and
// grid-synchronisation latency bounds it at low rank, so the rows are spread
// over all SMs (blocks of QB rows) and projections skip columns that are
// dependent: the work is O(M * D * rank) rather than O(M * D^2), which matters
// for the low-entanglement states of GHZ circuits.
//
// Main path: the whole column loop is one cooperative kernel
// (qr_coop_kernel) with one grid synchronisation per column (the second
// pass of column k and the first pass of column k+1 share a reduction), and
// a look-ahead that decides runs of dependent columns a window at a time.
// Fallback when the row blocks cannot all be resident at once: three
// kernels per column,
//   K1 [decide column k-1 from its norm partials; dots of a_k with columns < k]
//   K2 [sum the dot partials; a_k -= Q h; dots again]
//   K3 [sum; a_k -= Q h2; norm partials].
// Sums over blocks use the partials in one fixed order in every block (no
// atomics), so all blocks see identical values and runs are reproducible.
// Dependent columns are then filled by the closed form of the completion rule
// (sc_select_kernel / sc_materialize_kernel) when the kept rank is <= 64,
// else by the sequential kernels (rownorm, gs_unit, gs_second, normalize_col).
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr double MIN_RES2 = 0.25;
constexpr int QB = QR_ROWS;      // rows per block = threads per block
constexpr int MAXD = 256;        // maximal bond dimension

__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }

// Per-column block dot products: partial[i*G + block] = sum over this block's
// rows of conj(A[r, i]) * w_r for columns i < ncol not flagged zero (column
// `scol` scaled by sfac on the fly; column `skip` left out).
__device__ void block_dots(const cplx* A, long long M, int ncol, const int* szero, cplx w, bool valid, long long r,
                           int scol, double sfac, cplx (*wsum)[QB / 32], cplx* partial, int G, int skip) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = 0; i < ncol; ++i) {
        if (szero[i] || i == skip) continue;
        cplx d = make_double2(0.0, 0.0);
        if (valid) {
            cplx v = A[r + (long long)i * M];
            if (i == scol) {
                v.x *= sfac;
                v.y *= sfac;
            }
            d = make_double2(v.x * w.x + v.y * w.y, v.x * w.y - v.y * w.x);
        }
        for (int o = 16; o > 0; o >>= 1) {
            d.x += __shfl_down_sync(0xffffffffu, d.x, o);
            d.y += __shfl_down_sync(0xffffffffu, d.y, o);
        }
        if (lane == 0) wsum[i][warp] = d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ncol; i += blockDim.x) {
        cplx s = make_double2(0.0, 0.0);
        if (!szero[i] && i != skip)
            for (int q = 0; q < QB / 32; ++q) s = cadd(s, wsum[i][q]);
        partial[(long long)i * G + blockIdx.x] = s;
    }
}

// Sum the G partials of column i in fixed order.
__device__ __forceinline__ cplx sum_partials(const cplx* partial, int i, int G) {
    cplx s = make_double2(0.0, 0.0);
    for (int g = 0; g < G; ++g) s = cadd(s, partial[(long long)i * G + g]);
    return s;
}

__device__ __forceinline__ double sum_norm(const double* p, int G) {
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += p[g];
    return s;
}

__device__ double block_sum_d(double s, double* sh) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    return t;
}

// Frobenius norm partials of the whole matrix.
__global__ void frob_partial_kernel(const cplx* A, long long n, double* partial) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        s += A[e].x * A[e].x + A[e].y * A[e].y;
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void frob_finish_kernel(const double* partial, int G, double* scal) {
    if (threadIdx.x == 0) scal[0] = sum_norm(partial, G);
}

// norm^2 partials of column 0 (no projections)
__global__ void __launch_bounds__(QB) col_norm_kernel(const cplx* A, long long M, double* pnorm) {
    __shared__ double sh[QB / 32];
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    double s = 0.0;
    if (r < M) s = A[r].x * A[r].x + A[r].y * A[r].y;
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) pnorm[blockIdx.x] = s;
}

// Decide column kd from its norm partials: R_kk, flag, factor (identical in
// every block; block 0 stores them).
__device__ double decide(int kd, const double* pnorm, int G, double* scal, cplx* R, int D, int* flags,
                         double tol) {
    double s = sum_norm(pnorm, G);
    double nrm = sqrt(s), fro = sqrt(scal[0]);
    int dep = (fro == 0.0) || (nrm <= tol * fro);
    if (blockIdx.x == 0) {
        R[(long long)kd * D + kd] = make_double2(dep ? 0.0 : nrm, 0.0);
        scal[1] = dep ? 0.0 : 1.0 / nrm;
        flags[kd] = dep;
    }
    return dep ? 0.0 : 1.0 / nrm;
}

// Shared memory of one column phase.
struct PhaseSmem {
    int szero[MAXD];
    cplx h[MAXD];
    cplx wsum[MAXD][QB / 32];
    double sh[QB / 32];
    double sfac;
};

// K1 for column k >= 1: decide column k-1, dots of a_k with columns < k
__device__ void phase_k1(const cplx* A, long long M, int D, int k, const double* pnorm, int G, double* scal, cplx* R,
                         int* flags, cplx* part, double tol, PhaseSmem& sm) {
    if (threadIdx.x == 0) sm.sfac = decide(k - 1, pnorm, G, scal, R, D, flags, tol);
    for (int i = threadIdx.x; i < k - 1; i += QB) sm.szero[i] = flags[i];
    __syncthreads();
    if (threadIdx.x == 0) sm.szero[k - 1] = (sm.sfac == 0.0);
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    bool valid = r < M;
    cplx w = valid ? A[r + (long long)k * M] : make_double2(0.0, 0.0);
    block_dots(A, M, k, sm.szero, w, valid, r, k - 1, sm.sfac, sm.wsum, part, G, -1);
    __syncthreads();
}

// K2: scale column k-1, h = sum of partials, a_k -= sum_i A_i h_i, dots again
__device__ void phase_k2(cplx* A, long long M, int D, int k, const int* flags, const double* scal,
                         const cplx* part_in, cplx* part_out, cplx* R, int G, PhaseSmem& sm) {
    const double fac = scal[1];
    for (int i = threadIdx.x; i < k; i += QB) {
        sm.szero[i] = flags[i];
        sm.h[i] = sm.szero[i] ? make_double2(0.0, 0.0) : sum_partials(part_in, i, G);
        if (blockIdx.x == 0) R[(long long)k * D + i] = sm.h[i];
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    bool valid = r < M;
    cplx w = make_double2(0.0, 0.0);
    if (valid) {
        cplx* pk1 = A + r + (long long)(k - 1) * M;
        cplx v = *pk1;
        v.x *= fac;
        v.y *= fac;
        *pk1 = v;   // column k-1 is final now (zero if dependent)
        w = A[r + (long long)k * M];
        for (int i = 0; i < k; ++i) {
            if (sm.szero[i]) continue;
            cplx a = A[r + (long long)i * M], hi = sm.h[i];
            w.x -= a.x * hi.x - a.y * hi.y;
            w.y -= a.x * hi.y + a.y * hi.x;
        }
        A[r + (long long)k * M] = w;
    }
    block_dots(A, M, k, sm.szero, w, valid, r, -1, 1.0, sm.wsum, part_out, G, -1);
    __syncthreads();
}

// K3: h2 = sum, R[:k, k] += h2, a_k -= Q h2, norm partials
__device__ void phase_k3(cplx* A, long long M, int D, int k, const int* flags, const cplx* part_in, cplx* R,
                         double* pnorm, int G, PhaseSmem& sm) {
    for (int i = threadIdx.x; i < k; i += QB) {
        sm.szero[i] = flags[i];
        sm.h[i] = sm.szero[i] ? make_double2(0.0, 0.0) : sum_partials(part_in, i, G);
        if (blockIdx.x == 0) R[(long long)k * D + i] = cadd(R[(long long)k * D + i], sm.h[i]);
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    double s = 0.0;
    if (r < M) {
        cplx w = A[r + (long long)k * M];
        for (int i = 0; i < k; ++i) {
            if (sm.szero[i]) continue;
            cplx a = A[r + (long long)i * M], hi = sm.h[i];
            w.x -= a.x * hi.x - a.y * hi.y;
            w.y -= a.x * hi.y + a.y * hi.x;
        }
        A[r + (long long)k * M] = w;
        s = w.x * w.x + w.y * w.y;
    }
    s = block_sum_d(s, sm.sh);
    if (threadIdx.x == 0) pnorm[blockIdx.x] = s;
    __syncthreads();
}

__global__ void __launch_bounds__(QB) qr_k1(const cplx* A, long long M, int D, int k, const double* pnorm, int G,
                                            double* scal, cplx* R, int* flags, cplx* part, double tol) {
    __shared__ PhaseSmem sm;
    phase_k1(A, M, D, k, pnorm, G, scal, R, flags, part, tol, sm);
}

__global__ void __launch_bounds__(QB) qr_k2(cplx* A, long long M, int D, int k, const int* flags, const double* scal,
                                            const cplx* part_in, cplx* part_out, cplx* R, int G) {
    __shared__ PhaseSmem sm;
    phase_k2(A, M, D, k, flags, scal, part_in, part_out, R, G, sm);
}

__global__ void __launch_bounds__(QB) qr_k3(cplx* A, long long M, int D, int k, const int* flags, const cplx* part_in,
                                            cplx* R, double* pnorm, int G) {
    __shared__ PhaseSmem sm;
    phase_k3(A, M, D, k, flags, part_in, R, pnorm, G, sm);
}

// ------------------------------------------------- cooperative column loop
// The whole CGS2 column loop in one cooperative launch (all row blocks
// co-resident).  Every block owns QB rows and only ever touches those rows of
// A; blocks exchange per-block partial sums through global memory at grid
// synchronisations, and every block sums them in the same fixed order, so all
// blocks take identical decisions and runs are reproducible.
//
// One synchronisation per column.  At X(k) the blocks sum, for the kept
// columns Q (those before k):
//   h2 = Q^H v1_k,  g = Q^H a_{k+1},  c = v1_k^H a_{k+1},  |v1_k|^2
// where v1_k = a_k - Q h1_k is column k after its first pass.  Then
//   |v2_k|^2 = |v1_k|^2 - |h2|^2  decides column k (exact for orthonormal Q;
//     where the decision is close, |h2| is at rounding level of |a_k| and the
//     difference is far below the threshold),
//   q_k = (v1_k - Q h2) / |v2_k|,
//   h1_{k+1} = [g ; (c - h2^H g) / |v2_k|]  (the component of a_{k+1} along
//     q_k follows from the sums already at hand, no second synchronisation),
//   v1_{k+1} = a_{k+1} - [Q q_k] h1_{k+1}.
// So both Gram-Schmidt passes of every column are done against the stored
// columns, as in plain CGS2, with the second pass of column k and the first
// of column k+1 sharing one reduction.  Only kept columns take part, so a
// low-rank matrix costs O(M D rank) flops; the first QC_MAX kept columns of a
// block's rows stay in shared memory.
constexpr long long QR_BAR_SPINS = 1LL << 26;              // iteration cap behind the time limit
constexpr unsigned long long QR_BAR_NS = 2000000000ull;    // 2 s per synchronisation

__device__ __forceinline__ unsigned long long qr_global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
constexpr int QCS = QB + 1;            // cache column stride (odd: no bank conflicts)
constexpr int QC_MAX = 32;             // kept columns cached in shared memory
constexpr int PSTRIDE = 2 * MAXD + 4;  // partial row length

struct CoopSm {
    int nz[MAXD];             // kept columns so far, in order
    cplx h1s[MAXD + 1];       // first-pass coefficients of the current column
    cplx hb[PSTRIDE];         // summed partials of the current synchronisation
    cplx v1[QB];              // this block's rows of v1_k
    cplx an[QB];              // this block's rows of a_{k+1}
    cplx red[2 * QB];
    double d0[QB / 32], d1[QB / 32], d2[QB / 32];
    double fro2, scale;
    cplx hk;
    int nnz, ok, dep;
};

// Sums of a, b, c over the block; the totals land in thread 0.
__device__ void block_sum3(double& a, double& b, double& c, CoopSm& sm) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sm.d0[threadIdx.x >> 5] = a;
        sm.d1[threadIdx.x >> 5] = b;
        sm.d2[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = b = c = 0.0;
        for (int q = 0; q < QB / 32; ++q) {
            a += sm.d0[q];
            b += sm.d1[q];
            c += sm.d2[q];
        }
    }
    __syncthreads();
}

// Grid-wide barrier: bar[0] counts arrivals, bar[1] is the generation.  The
// wait is bounded: after QR_BAR_SPINS polls (or when another block gave up)
// the block sets *err and the call returns false; the caller returns.
__device__ bool grid_sync(unsigned* bar, int G, int* err, CoopSm& sm) {
    __syncthreads();
    if (G == 1) return true;
    if (threadIdx.x == 0) {
        sm.ok = 1;
        volatile unsigned* vgen = bar + 1;
        const unsigned gen = *vgen;
        __threadfence();   // this block's writes before its arrival
        const unsigned a = atomicAdd(bar, 1u);
        if (a == (unsigned)G - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            const unsigned long long t0 = qr_global_ns();
            while (*vgen == gen) {
                if (++spins > QR_BAR_SPINS || *(volatile int*)err ||
                    ((spins & 63) == 0 && qr_global_ns() - t0 > QR_BAR_NS)) {
                    atomicExch(err, 1);
                    sm.ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();   // acquire: the other blocks' writes
    }
    __syncthreads();
    return sm.ok != 0;
}

// out[e] = sum over the G partial rows part[g * PSTRIDE + e] (in increasing
// g), e < E, by all threads of the calling block.
__device__ void sum_rows(const cplx* part, int G, int E, cplx* out, CoopSm& sm) {
    const int t = threadIdx.x;
    if (E > QB) {
        for (int e = t; e < E; e += QB) {
            cplx s0 = make_double2(0.0, 0.0), s1 = s0;
            int g = 0;
#pragma unroll 4
            for (; g + 1 < G; g += 2) {
                s0 = cadd(s0, __ldcg(part + (long long)g * PSTRIDE + e));
                s1 = cadd(s1, __ldcg(part + (long long)(g + 1) * PSTRIDE + e));
            }
            if (g < G) s0 = cadd(s0, __ldcg(part + (long long)g * PSTRIDE + e));
            out[e] = cadd(s0, s1);
        }
        __syncthreads();
        return;
    }
    int c = 1;                          // chunks of rows per entry (power of two)
    while (2 * c * E <= QB) c *= 2;
    const int L = (G + c - 1) / c;
    const int e = t / c, q = t % c;
    cplx s0 = make_double2(0.0, 0.0), s1 = s0;
    if (e < E) {
        const int g1 = min(G, (q + 1) * L);
        int g = q * L;
#pragma unroll 4
        for (; g + 1 < g1; g += 2) {
            s0 = cadd(s0, __ldcg(part + (long long)g * PSTRIDE + e));
            s1 = cadd(s1, __ldcg(part + (long long)(g + 1) * PSTRIDE + e));
        }
        if (g < g1) s0 = cadd(s0, __ldcg(part + (long long)g * PSTRIDE + e));
    }
    cplx sv = cadd(s0, s1);
    const int seg = c < 32 ? c : 32;
    for (int o = seg / 2; o > 0; o >>= 1) {
        sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
        sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
    }
    if (q % 32 == 0) sm.red[t / seg] = sv;
    __syncthreads();
    const int per = c / seg;
    if (t < E) {
        cplx a = sm.red[t * per];
        for (int w = 1; w < per; ++w) a = cadd(a, sm.red[t * per + w]);
        out[t] = a;
    }
    __syncthreads();
}

// Row rr of kept column j (shared-memory cache or global).
__device__ __forceinline__ cplx qcol(const cplx* A, long long M, long long r0, const cplx* qc, int nc, int j, int rr,
                                     const CoopSm& sm) {
    return j < nc ? qc[j * QCS + rr] : A[r0 + rr + (long long)sm.nz[j] * M];
}

// This block's partials of X(k): out[j] = Q_j^H v1, out[n + j] = Q_j^H a_next
// (j < n), out[2n] = v1^H a_next, out[2n + 1] = (|v1|^2, fro) over its rows.
__device__ void coop_partials(const cplx* A, long long M, long long r0, int nrows, int n, const cplx* qc, int nc,
                              double fro, cplx* out, CoopSm& sm) {
    const int t = threadIdx.x;
    if (n > QB) {
        for (int j = t; j < n; j += QB) {
            cplx sv = make_double2(0.0, 0.0), sa = sv;
            for (int rr = 0; rr < nrows; ++rr) {
                cplx a = qcol(A, M, r0, qc, nc, j, rr, sm), v = sm.v1[rr], b = sm.an[rr];
                sv.x = fma(a.x, v.x, fma(a.y, v.y, sv.x));
                sv.y = fma(a.x, v.y, fma(-a.y, v.x, sv.y));
                sa.x = fma(a.x, b.x, fma(a.y, b.y, sa.x));
                sa.y = fma(a.x, b.y, fma(-a.y, b.x, sa.y));
            }
            out[j] = sv;
            out[n + j] = sa;
        }
    } else if (n > 0) {
        // sl row slices per column, sl a power of two so that the slices of
        // one column are reduced by shuffles (within a warp) and at most
        // four shared-memory terms (across warps)
        int sl = 1;
        while (2 * sl * n <= QB) sl *= 2;
        const int j = t / sl, q = t % sl;
        cplx sv = make_double2(0.0, 0.0), sa = sv;
        if (j < n) {
#pragma unroll 2
            for (int rr = q; rr < nrows; rr += sl) {
                cplx a = qcol(A, M, r0, qc, nc, j, rr, sm), v = sm.v1[rr], b = sm.an[rr];
                sv.x = fma(a.x, v.x, fma(a.y, v.y, sv.x));
                sv.y = fma(a.x, v.y, fma(-a.y, v.x, sv.y));
                sa.x = fma(a.x, b.x, fma(a.y, b.y, sa.x));
                sa.y = fma(a.x, b.y, fma(-a.y, b.x, sa.y));
            }
        }
        const int seg = sl < 32 ? sl : 32;
        for (int o = seg / 2; o > 0; o >>= 1) {
            sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
            sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
            sa.x += __shfl_xor_sync(0xffffffffu, sa.x, o);
            sa.y += __shfl_xor_sync(0xffffffffu, sa.y, o);
        }
        if (q % 32 == 0) {
            sm.red[2 * (t / seg)] = sv;
            sm.red[2 * (t / seg) + 1] = sa;
        }
        __syncthreads();
        const int per = sl / seg;          // warp partials per column (1 to 4)
        if (t < n) {
            cplx a = sm.red[2 * t * per], b = sm.red[2 * t * per + 1];
            for (int w = 1; w < per; ++w) {
                a = cadd(a, sm.red[2 * (t * per + w)]);
                b = cadd(b, sm.red[2 * (t * per + w) + 1]);
            }
            out[t] = a;
            out[n + t] = b;
        }
    }
    double vv = 0.0, cx = 0.0, cy = 0.0;
    if (t < nrows) {
        cplx v = sm.v1[t], b = sm.an[t];
        vv = v.x * v.x + v.y * v.y;
        cx = v.x * b.x + v.y * b.y;
        cy = v.x * b.y - v.y * b.x;
    }
    block_sum3(vv, cx, cy, sm);
    if (t == 0) {
        out[2 * n] = make_double2(cx, cy);
        out[2 * n + 1] = make_double2(vv, fro);
    }
    __syncthreads();
}

// sum_j Q[r, nz_j] h[j] for this thread's row (j < n).
__device__ __forceinline__ cplx coop_combo(const cplx* A, long long M, long long r0, int t, const cplx* qc, int nc,
                                           int n, const cplx* h, const CoopSm& sm) {
    cplx u0 = make_double2(0.0, 0.0), u1 = u0;
    int j = 0;
#pragma unroll 2
    for (; j + 1 < n; j += 2) {
        cplx a = qcol(A, M, r0, qc, nc, j, t, sm), b = qcol(A, M, r0, qc, nc, j + 1, t, sm);
        cplx ha = h[j], hb = h[j + 1];
        u0.x = fma(a.x, ha.x, fma(-a.y, ha.y, u0.x));
        u0.y = fma(a.x, ha.y, fma(a.y, ha.x, u0.y));
        u1.x = fma(b.x, hb.x, fma(-b.y, hb.y, u1.x));
        u1.y = fma(b.x, hb.y, fma(b.y, hb.x, u1.y));
    }
    if (j < n) {
        cplx a = qcol(A, M, r0, qc, nc, j, t, sm), ha = h[j];
        u0.x = fma(a.x, ha.x, fma(-a.y, ha.y, u0.x));
        u0.y = fma(a.x, ha.y, fma(a.y, ha.x, u0.y));
    }
    return cadd(u0, u1);
}

// Sums of the partial rows of one synchronisation into sm.hb (E entries).
// Few entries: every block sums all rows itself.  Many: block b sums the
// entries e = b (mod G) into red_out, and a second synchronisation publishes
// them (so no block reads more than a few rows per thread).
__device__ bool coop_reduce(const cplx* part, int G, int E, cplx* red_out, unsigned* bar, int* err, CoopSm& sm) {
    if (G == 1) return true;   // the block wrote its partials to sm.hb
    if (!grid_sync(bar, G, err, sm)) return false;
    if ((long long)E * G <= 32LL * QB) {
        sum_rows(part, G, E, sm.hb, sm);
        return true;
    }
    const int t = threadIdx.x;
    for (int e = blockIdx.x; e < E; e += G) {
        cplx s = make_double2(0.0, 0.0);
        for (int g = t; g < G; g += QB) s = cadd(s, __ldcg(part + (long long)g * PSTRIDE + e));
        sm.red[t] = s;
        __syncthreads();
        for (int w = QB / 2; w > 0; w >>= 1) {
            if (t < w) sm.red[t] = cadd(sm.red[t], sm.red[t + w]);
            __syncthreads();
        }
        if (t == 0) red_out[e] = sm.red[0];
        __syncthreads();
    }
    if (!grid_sync(bar, G, err, sm)) return false;
    for (int e = t; e < E; e += QB) sm.hb[e] = __ldcg(red_out + e);
    __syncthreads();
    return true;
}

// ---------------------------------------------- look-ahead over dependent runs
// After a dependent column the kept set Q often stays the same for many
// columns (low-rank node tensors).  A window of the next W columns then takes
// both Gram-Schmidt passes against Q together, in two synchronisations:
//   L1: g_j = Q^H a_j                         v1_j = a_j - Q g_j
//   L2: h2_j = Q^H v1_j, |v1_j|^2, v1_j^H v1_{j+1}, and for the column a'
//       after the window g' = Q^H a', c' = v1_{W-1}^H a'
// The columns are decided in order exactly as in the one-column loop
// (|v2_j|^2 = |v1_j|^2 - |h2_j|^2 against the same Q) up to and including the
// first kept one, q = (v1_j - Q h2_j) / |v2_j|.  The column after it continues
// in the one-column loop; its first-pass coefficients are g + h2 along Q and,
// along q, (v1_j^H v1_{j+1} - h2_j^H h2_{j+1}) / |v2_j| (inside the window)
// or (c' - h2_j^H g') / |v2_j| (a'), both from the sums above.  Columns after
// that are redone.
constexpr int LA_WMAX = 16;

// One vector of the block's rows: 0 = kept column i, 1 = window vector i,
// 2 = column i of A.
__device__ __forceinline__ cplx la_vec(int kind, int i, int rr, const cplx* A, long long M, long long r0,
                                       const cplx* qc, int nc, const cplx (*vw)[QB], const CoopSm& sm) {
    if (kind == 0) return qcol(A, M, r0, qc, nc, i, rr, sm);
    if (kind == 1) return vw[i][rr];
    return A[r0 + rr + (long long)i * M];
}

// out[p] = sum over the block's rows of conj(L_p) R_p for p < P, where
// pair(p, lk, li, rk, ri) names the two vectors; row slices of a power-of-two
// width are reduced by shuffles (as in coop_partials).
template <class PairF>
__device__ void la_dots(int P, PairF pair, cplx* out, const cplx* A, long long M, long long r0, int nrows,
                        const cplx* qc, int nc, const cplx (*vw)[QB], CoopSm& sm) {
    const int t = threadIdx.x;
    if (P > QB) {
        for (int p = t; p < P; p += QB) {
            int lk, li, rk, ri;
            pair(p, lk, li, rk, ri);
            cplx s0 = make_double2(0.0, 0.0);
            for (int rr = 0; rr < nrows; ++rr) {
                cplx a = la_vec(lk, li, rr, A, M, r0, qc, nc, vw, sm), b = la_vec(rk, ri, rr, A, M, r0, qc, nc, vw, sm);
                s0.x = fma(a.x, b.x, fma(a.y, b.y, s0.x));
                s0.y = fma(a.x, b.y, fma(-a.y, b.x, s0.y));
            }
            out[p] = s0;
        }
        __syncthreads();
        return;
    }
    int sl = 1;
    while (2 * sl * P <= QB) sl *= 2;
    const int p = t / sl, q = t % sl;
    cplx sv = make_double2(0.0, 0.0);
    if (p < P) {
        int lk, li, rk, ri;
        pair(p, lk, li, rk, ri);
        for (int rr = q; rr < nrows; rr += sl) {
            cplx a = la_vec(lk, li, rr, A, M, r0, qc, nc, vw, sm), b = la_vec(rk, ri, rr, A, M, r0, qc, nc, vw, sm);
            sv.x = fma(a.x, b.x, fma(a.y, b.y, sv.x));
            sv.y = fma(a.x, b.y, fma(-a.y, b.x, sv.y));
        }
    }
    const int seg = sl < 32 ? sl : 32;
    for (int o = seg / 2; o > 0; o >>= 1) {
        sv.x += __shfl_xor_sync(0xffffffffu, sv.x, o);
        sv.y += __shfl_xor_sync(0xffffffffu, sv.y, o);
    }
    if (q % 32 == 0) sm.red[t / seg] = sv;
    __syncthreads();
    const int per = sl / seg;
    if (t < P) {
        cplx a = sm.red[t * per];
        for (int w = 1; w < per; ++w) a = cadd(a, sm.red[t * per + w]);
        out[t] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(QB) qr_coop_kernel(cplx* A, long long M, int D, cplx* R, int* flags, cplx* part,
                                                     cplx* red_out, unsigned* bar, int* err, int nc_max, double tol,
                                                     int la_max) {
    // dynamic shared memory: nc_max cached columns of QCS rows, then the
    // look-ahead window of at most la_max (<= LA_WMAX) columns (this block's
    // rows of v1_j)
    extern __shared__ cplx dyn[];
    cplx* qc = dyn;
    cplx(*vw)[QB] = reinterpret_cast<cplx(*)[QB]>(dyn + (long long)nc_max * QCS);
    __shared__ CoopSm sm;
    __shared__ cplx la_g[PSTRIDE];     // look-ahead: g_j = Q^H a_j (column j at j * nq)
    __shared__ double la_s2[LA_WMAX];
    const int G = gridDim.x, t = threadIdx.x;
    const long long r0 = (long long)blockIdx.x * QB;
    const int nrows = (int)min((long long)QB, M - r0);
    const bool own = t < nrows;
    const long long r = r0 + t;
    const bool b0 = blockIdx.x == 0;

    // |A|_F^2 over this block's rows; v1_0 = a_0, a_next = a_1
    double fro = 0.0, dz0 = 0.0, dz1 = 0.0;
    if (own)
        for (int j = 0; j < D; ++j) {
            cplx a = A[r + (long long)j * M];
            fro += a.x * a.x + a.y * a.y;
        }
    block_sum3(fro, dz0, dz1, sm);
    sm.v1[t] = own ? A[r] : make_double2(0.0, 0.0);
    sm.an[t] = (own && D > 1) ? A[r + M] : make_double2(0.0, 0.0);
    if (t == 0) sm.nnz = 0;
    __syncthreads();
    int seq = 0;        // reductions so far: partial rows alternate between two buffers
    int la_w = min(4, la_max);   // look-ahead window width
    for (int k = 0; k < D; ++k) {
        const int n = sm.nnz, E = 2 * n + 2;
        const int nc = min(n, nc_max);
        // prefetch a_{k+2}; its latency hides behind the synchronisation
        const cplx pre = (own && k + 2 < D) ? A[r + (long long)(k + 2) * M] : make_double2(0.0, 0.0);
        cplx* pbuf = part + (long long)(seq & 1) * G * PSTRIDE;
        ++seq;
        coop_partials(A, M, r0, nrows, n, qc, nc, k == 0 ? fro : 0.0, G == 1 ? sm.hb : pbuf + blockIdx.x * PSTRIDE,
                      sm);
        if (!coop_reduce(pbuf, G, E, red_out, bar, err, sm)) return;
        // decide column k; first-pass coefficient of a_{k+1} along q_k
        if (k == 0 && t == 0) sm.fro2 = sm.hb[1].y;
        __syncthreads();
        {
            double s2 = 0.0, px = 0.0, py = 0.0;   // |h2|^2 and h2^H g
            for (int j = t; j < n; j += QB) {
                cplx h2 = sm.hb[j], g = sm.hb[n + j];
                s2 += h2.x * h2.x + h2.y * h2.y;
                px += h2.x * g.x + h2.y * g.y;
                py += h2.x * g.y - h2.y * g.x;
                if (b0) R[(long long)k * D + sm.nz[j]] = cadd(sm.h1s[j], h2);
            }
            block_sum3(s2, px, py, sm);
            if (t == 0) {
                const double nrm = sqrt(fmax(sm.hb[2 * n + 1].x - s2, 0.0)), f = sqrt(sm.fro2);
                const int dep = (f == 0.0) || (nrm <= tol * f);
                const double sc = dep ? 0.0 : 1.0 / nrm;
                sm.dep = dep;
                sm.scale = sc;
                const cplx c = sm.hb[2 * n];
                sm.hk = make_double2(sc * (c.x - px), sc * (c.y - py));
                if (b0) {
                    R[(long long)k * D + k] = make_double2(dep ? 0.0 : nrm, 0.0);
                    flags[k] = dep;
                }
            }
            __syncthreads();
        }
        // finalise q_k = (v1_k - Q h2) * scale for this block's rows
        if (own) {
            cplx w = sm.v1[t], u = coop_combo(A, M, r0, t, qc, nc, n, sm.hb, sm);
            w = make_double2((w.x - u.x) * sm.scale, (w.y - u.y) * sm.scale);
            A[r + (long long)k * M] = w;
            if (!sm.dep && n < nc_max) qc[n * QCS + t] = w;
        }
        __syncthreads();
        if (k + 1 == D) break;
        // h1_{k+1} = [g ; hk], v1_{k+1} = a_{k+1} - Q h1_{k+1}
        for (int j = t; j < n; j += QB) sm.h1s[j] = sm.hb[n + j];
        if (t == 0 && !sm.dep) {
            sm.h1s[n] = sm.hk;
            sm.nz[n] = k;
            sm.nnz = n + 1;
        }
        __syncthreads();
        const int n1 = sm.nnz, nc1 = min(n1, nc_max);
        if (own) {
            cplx a = sm.an[t], u = coop_combo(A, M, r0, t, qc, nc1, n1, sm.h1s, sm);
            sm.v1[t] = make_double2(a.x - u.x, a.y - u.y);
        }
        sm.an[t] = pre;
        __syncthreads();
        if (!sm.dep) continue;
        // column k was dependent: decide the following columns a window at a
        // time while the kept set stays the same
        int k0 = k + 1;
        bool resume = false;   // the one-column loop continues at column k0
        while (k0 < D && !resume) {
            const int nq = sm.nnz, ncq = min(nq, nc_max);
            const int cap = (PSTRIDE - nq - 1) / (nq + 2);   // widest window whose sums fit a partial row
            if (k0 == k + 1 && cap < 2) break;    // kept set too wide: stay column by column (state in place)
            const int W = min(min(min(la_w, la_max), D - k0), cap);   // >= 1
            const bool after = k0 + W < D;
            const int ka = k0 + W;                // the column after the window
            // L1: g_j = Q^H a_j, kept in la_g; v1_j = a_j - Q g_j into vw
            if (nq > 0) {
                cplx* pb = part + (long long)(seq & 1) * G * PSTRIDE;
                ++seq;
                la_dots(nq * W, [&](int p, int& lk, int& li, int& rk, int& ri) {
                            lk = 0; li = p % nq; rk = 2; ri = k0 + p / nq;
                        }, G == 1 ? sm.hb : pb + blockIdx.x * PSTRIDE, A, M, r0, nrows, qc, ncq, vw, sm);
                if (!coop_reduce(pb, G, nq * W, red_out, bar, err, sm)) return;
                for (int e = t; e < nq * W; e += QB) la_g[e] = sm.hb[e];
                __syncthreads();
            }
            for (int j = 0; j < W; ++j) {
                cplx v = make_double2(0.0, 0.0);
                if (own) {
                    cplx a = A[r + (long long)(k0 + j) * M];
                    cplx u = coop_combo(A, M, r0, t, qc, ncq, nq, la_g + j * nq, sm);
                    v = make_double2(a.x - u.x, a.y - u.y);
                }
                vw[j][t] = v;
            }
            __syncthreads();
            // L2: h2 (nq W, column j at j * nq), |v1_j|^2 (W), v1_j^H v1_{j+1}
            // (W - 1), g' (nq), c' (1)
            const int o_nv = nq * W, o_x = o_nv + W, o_g = o_x + (W - 1), o_c = o_g + nq, E2 = o_c + 1;
            {
                cplx* pb = part + (long long)(seq & 1) * G * PSTRIDE;
                ++seq;
                la_dots(E2, [&](int p, int& lk, int& li, int& rk, int& ri) {
                            if (p < o_nv) { lk = 0; li = p % nq; rk = 1; ri = p / nq; }
                            else if (p < o_x) { lk = 1; li = p - o_nv; rk = 1; ri = p - o_nv; }
                            else if (p < o_g) { lk = 1; li = p - o_x; rk = 1; ri = p - o_x + 1; }
                            else if (p < o_c) { lk = 0; li = p - o_g; rk = after ? 2 : 1; ri = after ? ka : 0; }
                            else { lk = 1; li = W - 1; rk = after ? 2 : 1; ri = after ? ka : W - 1; }
                        }, G == 1 ? sm.hb : pb + blockIdx.x * PSTRIDE, A, M, r0, nrows, qc, ncq, vw, sm);
                if (!coop_reduce(pb, G, E2, red_out, bar, err, sm)) return;
            }
            for (int j = t; j < W; j += QB) {
                double s2 = 0.0;
                for (int i = 0; i < nq; ++i) {
                    cplx h = sm.hb[j * nq + i];
                    s2 += h.x * h.x + h.y * h.y;
                }
                la_s2[j] = s2;
            }
            __syncthreads();
            // decisions in column order up to the first kept column
            if (t == 0) {
                const double f = sqrt(sm.fro2);
                int js = -1;
                double nrm = 0.0;
                for (int j = 0; j < W; ++j) {
                    nrm = sqrt(fmax(sm.hb[o_nv + j].x - la_s2[j], 0.0));
                    const int dep = (f == 0.0) || (nrm <= tol * f);
                    if (b0) {
                        R[(long long)(k0 + j) * D + (k0 + j)] = make_double2(dep ? 0.0 : nrm, 0.0);
                        flags[k0 + j] = dep;
                    }
                    if (!dep) {
                        js = j;
                        break;
                    }
                }
                sm.dep = js;
                sm.scale = js >= 0 ? 1.0 / nrm : 0.0;
            }
            __syncthreads();
            const int js = sm.dep, nd = js >= 0 ? js + 1 : W;
            if (b0)
                for (int e = t; e < nq * nd; e += QB)
                    R[(long long)(k0 + e / nq) * D + sm.nz[e % nq]] = cadd(la_g[e], sm.hb[e]);
            // finalise the decided columns: zero if dependent, q if kept
            if (own)
                for (int j = 0; j < nd; ++j) {
                    cplx w = make_double2(0.0, 0.0);
                    if (j == js) {
                        cplx v = vw[j][t], u = coop_combo(A, M, r0, t, qc, ncq, nq, sm.hb + j * nq, sm);
                        w = make_double2((v.x - u.x) * sm.scale, (v.y - u.y) * sm.scale);
                        if (nq < nc_max) qc[nq * QCS + t] = w;
                    }
                    A[r + (long long)(k0 + j) * M] = w;
                }
            __syncthreads();
            if (js < 0) {   // the whole window was dependent
                k0 += W;
                la_w = min(2 * la_w, la_max);
                continue;
            }
            la_w = max(min(4, la_max), la_w / 2);
            const int kn = k0 + js + 1;           // next column, back in the one-column loop
            if (kn >= D) {
                k0 = D;
                break;
            }
            // first-pass coefficients of column kn: [g + h2 (inside) or g' (after) ; along q]
            const bool inside = js + 1 < W;
            if (t == 0) {
                cplx c = inside ? sm.hb[o_x + js] : sm.hb[o_c];
                double px = 0.0, py = 0.0;    // h2_js^H (h2_{js+1} or g')
                for (int i = 0; i < nq; ++i) {
                    cplx h = sm.hb[js * nq + i];
                    cplx o = inside ? sm.hb[(js + 1) * nq + i] : sm.hb[o_g + i];
                    px += h.x * o.x + h.y * o.y;
                    py += h.x * o.y - h.y * o.x;
                }
                sm.hk = make_double2(sm.scale * (c.x - px), sm.scale * (c.y - py));
            }
            for (int i = t; i < nq; i += QB)
                sm.h1s[i] = inside ? cadd(la_g[(js + 1) * nq + i], sm.hb[(js + 1) * nq + i]) : sm.hb[o_g + i];
            __syncthreads();
            if (t == 0) {
                sm.h1s[nq] = sm.hk;
                sm.nz[nq] = k0 + js;
                sm.nnz = nq + 1;
            }
            __syncthreads();
            // v1 of column kn = a_kn - [Q q] h1s (its first pass), a_next = a_{kn+1}
            const int n1 = nq + 1, nc1 = min(n1, nc_max);
            if (own) {
                cplx a = A[r + (long long)kn * M], u = coop_combo(A, M, r0, t, qc, nc1, n1, sm.h1s, sm);
                sm.v1[t] = make_double2(a.x - u.x, a.y - u.y);
                sm.an[t] = kn + 1 < D ? A[r + (long long)(kn + 1) * M] : make_double2(0.0, 0.0);
            } else {
                sm.an[t] = make_double2(0.0, 0.0);
            }
            __syncthreads();
            k0 = kn;
            resume = true;
        }
        if (k0 >= D) break;     // every column decided and finalised
        k = k0 - 1;             // the loop's increment brings it to k0
    }
}

// Decide and scale the last column.
__global__ void __launch_bounds__(QB) qr_last(cplx* A, long long M, int D, const double* pnorm, int G, double* scal,
                                              cplx* R, int* flags, double tol) {
    __shared__ double sfac;
    if (threadIdx.x == 0) sfac = decide(D - 1, pnorm, G, scal, R, D, flags, tol);
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    if (r < M) {
        cplx v = A[r + (long long)(D - 1) * M];
        v.x *= sfac;
        v.y *= sfac;
        A[r + (long long)(D - 1) * M] = v;
    }
}

// ------------------------------------------------------------ completion
__global__ void __launch_bounds__(QB) rownorm_kernel(const cplx* A, long long M, int D, const int* flags,
                                                     double* rownorm) {
    __shared__ int szero[MAXD];
    for (int i = threadIdx.x; i < D; i += blockDim.x) szero[i] = flags[i];
    __syncthreads();
    long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r >= M) return;
    double s = 0.0;
    for (int j = 0; j < D; ++j) {
        if (szero[j]) continue;
        cplx v = A[r + (long long)j * M];
        s += v.x * v.x + v.y * v.y;
    }
    rownorm[r] = s;
}

// First candidate with 1 - rownorm >= 1/4, else the largest residual
// (earliest on ties); computed identically by every block.
__device__ int pick_candidate(const double* rownorm, const int* cand, int ncand) {
    __shared__ int sfirst[QB / 32];
    __shared__ double sbest[QB / 32];
    __shared__ int sbi[QB / 32];
    __shared__ int result;
    int first = ncand, bi = ncand;
    double best = -1.0;
    for (int p = threadIdx.x; p < ncand; p += blockDim.x) {
        double res = 1.0 - rownorm[cand[p]];
        if (res >= MIN_RES2 && p < first) first = p;
        if (res > best || (res == best && p < bi)) {
            best = res;
            bi = p;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        int f2 = __shfl_down_sync(0xffffffffu, first, o);
        double b2 = __shfl_down_sync(0xffffffffu, best, o);
        int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        first = min(first, f2);
        if (b2 > best || (b2 == best && i2 < bi)) {
            best = b2;
            bi = i2;
        }
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sfirst[w] = first;
        sbest[w] = best;
        sbi[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = ncand, b = ncand;
        double bv = -1.0;
        for (int i = 0; i < QB / 32; ++i) {
            f = min(f, sfirst[i]);
            if (sbest[i] > bv || (sbest[i] == bv && sbi[i] < b)) {
                bv = sbest[i];
                b = sbi[i];
            }
        }
        int p = f < ncand ? f : b;
        result = (p < ncand) ? cand[p] : 0;
    }
    __syncthreads();
    return result;
}

// column k <- e_c - sum_j A_j conj(A(c, j)) over nonzero j for the picked
// candidate c; then dots with the nonzero columns
__global__ void __launch_bounds__(QB) gs_unit_kernel(cplx* A, long long M, int D, int k, const int* flags,
                                                     const double* rownorm, const int* cand, int ncand, cplx* part,
                                                     int G) {
    __shared__ int szero[MAXD];
    __shared__ cplx rowc[MAXD];
    __shared__ cplx wsum[MAXD][QB / 32];
    const int c = pick_candidate(rownorm, cand, ncand);
    for (int j = threadIdx.x; j < D; j += QB) {
        szero[j] = flags[j] || j == k;
        cplx v = A[c + (long long)j * M];
        rowc[j] = make_double2(v.x, -v.y);
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    bool valid = r < M;
    cplx s = make_double2(0.0, 0.0);
    if (valid) {
        s.x = (r == c) ? 1.0 : 0.0;
        for (int j = 0; j < D; ++j) {
            if (szero[j]) continue;
            cplx a = A[r + (long long)j * M], h = rowc[j];
            s.x -= a.x * h.x - a.y * h.y;
            s.y -= a.x * h.y + a.y * h.x;
        }
        A[r + (long long)k * M] = s;
    }
    block_dots(A, M, D, szero, s, valid, r, -1, 1.0, wsum, part, G, k);
}

// second pass of the completion vector: v -= Q h (nonzero columns), norm partials
__global__ void __launch_bounds__(QB) gs_second_kernel(cplx* A, long long M, int D, int k, const int* flags,
                                                       const cplx* part_in, double* pnorm, int G) {
    __shared__ int szero[MAXD];
    __shared__ cplx h[MAXD];
    __shared__ double sh[QB / 32];
    for (int i = threadIdx.x; i < D; i += QB) {
        szero[i] = flags[i] || i == k;
        h[i] = szero[i] ? make_double2(0.0, 0.0) : sum_partials(part_in, i, G);
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    double s = 0.0;
    if (r < M) {
        cplx w = A[r + (long long)k * M];
        for (int i = 0; i < D; ++i) {
            if (szero[i]) continue;
            cplx a = A[r + (long long)i * M], hi = h[i];
            w.x -= a.x * hi.x - a.y * hi.y;
            w.y -= a.x * hi.y + a.y * hi.x;
        }
        A[r + (long long)k * M] = w;
        s = w.x * w.x + w.y * w.y;
    }
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) pnorm[blockIdx.x] = s;
}

__global__ void __launch_bounds__(QB) normalize_col_kernel(cplx* A, long long M, int k, const double* pnorm, int G,
                                                           double* rownorm, int* flags) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double s = sum_norm(pnorm, G);
        inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
        // the completed column joins Q for later completions (no block of
        // this kernel reads the flags)
        if (blockIdx.x == 0) flags[k] = 0;
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    if (r < M) {
        cplx v = A[r + (long long)k * M];
        v.x *= inv;
        v.y *= inv;
        A[r + (long long)k * M] = v;
        rownorm[r] += v.x * v.x + v.y * v.y;
    }
}

// ------------------------------------------------ structured completion
// With Q_r the kept columns, the sequential rule above has a closed form:
// given the rows A_<t of earlier picks, the residual of candidate c is
// 1 - w_c M w_c^H with w_c = Q_r[c, :] and M = (I - W_A^H W_A)^{-1}, and the
// t-th completion vector is (e_{a_t} - (Q_r y_t with the rows of earlier picks
// zeroed)) / nu_t with y_t = M w_t^H, nu_t^2 = 1 - w_t y_t.  M is updated by
// M += y_t y_t^H / nu_t^2 (Sherman-Morrison).  The selection touches only
// candidate rows (O(L r^2)); the vectors are one M x r x m product.
__global__ void sc_init_kernel(int* row_rank, long long M, int* cand_used, int ncand) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x)
        row_rank[i] = 0x7FFFFFFF;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncand;
         i += (long long)gridDim.x * blockDim.x)
        cand_used[i] = 0;
}

// One block of SC_THREADS threads; shared: Minv (r x r), y, w.
constexpr int SC_THREADS = 256;

__device__ double sc_residual(const cplx* A, long long M, const int* kept, int r, int c, const cplx* Mi, cplx* w,
                              cplx* y, double* red) {
    for (int j = threadIdx.x; j < r; j += blockDim.x) w[j] = A[c + (long long)kept[j] * M];
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x) {
        cplx s = make_double2(0.0, 0.0);
        for (int j = 0; j < r; ++j) {
            cplx m = Mi[i * r + j], wj = w[j];   // y_i = sum_j M_ij conj(w_j)
            s.x += m.x * wj.x + m.y * wj.y;
            s.y += m.y * wj.x - m.x * wj.y;
        }
        y[i] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int j = threadIdx.x; j < r; j += 32) acc += w[j].x * y[j].x - w[j].y * y[j].y;   // Re(w_j y_j)
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) red[0] = 1.0 - acc;
    }
    __syncthreads();
    return red[0];
}

__global__ void __launch_bounds__(SC_THREADS) sc_select_kernel(const cplx* A, long long M, const int* kept, int r,
                                                               int m, const int* cand, int ncand, int* acc_rows,
                                                               cplx* Y, double* nu, int* row_rank, int* cand_used) {
    extern __shared__ cplx sm[];
    cplx* Mi = sm;
    cplx* y = Mi + r * r;
    cplx* w = y + r;
    __shared__ double red[1];
    __shared__ double sbest;
    __shared__ int sbi;
    for (int i = threadIdx.x; i < r * r; i += blockDim.x)
        Mi[i] = make_double2((i / r == i % r) ? 1.0 : 0.0, 0.0);
    __syncthreads();
    int p = 0;
    for (int t = 0; t < m; ++t) {
        int chosen = -1;
        double res = 0.0;
        for (; p < ncand; ++p) {
            if (cand_used[p]) continue;
            res = sc_residual(A, M, kept, r, cand[p], Mi, w, y, red);
            if (res >= MIN_RES2) {
                chosen = p;
                break;
            }
        }
        if (chosen < 0) {
            // no candidate reaches 1/4: the largest residual, earliest on ties
            if (threadIdx.x == 0) {
                sbest = -1.0;
                sbi = -1;
            }
            __syncthreads();
            for (int q = 0; q < ncand; ++q) {
                if (cand_used[q]) continue;
                double rq = sc_residual(A, M, kept, r, cand[q], Mi, w, y, red);
                if (threadIdx.x == 0 && rq > sbest) {
                    sbest = rq;
                    sbi = q;
                }
                __syncthreads();
            }
            // non-finite residuals (a NaN matrix) select nothing above: take the
            // first unused candidate so every index stays in bounds; the NaN
            // then propagates to the result, where the caller detects it
            chosen = sbi;
            if (chosen < 0)
                for (int q = 0; q < ncand; ++q)
                    if (!cand_used[q]) {
                        chosen = q;
                        break;
                    }
            if (chosen < 0) chosen = 0;
            res = sc_residual(A, M, kept, r, cand[chosen], Mi, w, y, red);
            p = ncand;   // residuals only decrease: no later scan can reach 1/4 either
        } else {
            ++p;
        }
        const int c = cand[chosen];
        const double n = sqrt(res);
        if (threadIdx.x == 0) {
            acc_rows[t] = c;
            nu[t] = n;
            row_rank[c] = t;
            cand_used[chosen] = 1;
        }
        for (int j = threadIdx.x; j < r; j += blockDim.x) Y[(long long)t * r + j] = y[j];
        __syncthreads();
        const double inv = 1.0 / res;
        for (int idx = threadIdx.x; idx < r * r; idx += blockDim.x) {
            int i = idx / r, j = idx % r;   // M += y y^H / res
            cplx yi = y[i], yj = y[j];
            Mi[idx].x += inv * (yi.x * yj.x + yi.y * yj.y);
            Mi[idx].y += inv * (yi.y * yj.x - yi.x * yj.y);
        }
        __syncthreads();
    }
}

// The same selection by one warp, for kept ranks r <= 32 (lane j holds
// w_j and y_j): no block-wide barriers in the candidate loop, whose latency
// dominated the block version (one candidate evaluation per dependent column
// is typical).  Every sum runs in the block version's order, so both take
// identical decisions and produce identical Y, nu.
__global__ void __launch_bounds__(32) sc_select_warp_kernel(const cplx* A, long long M, const int* kept, int r,
                                                            int m, const int* cand, int ncand, int* acc_rows,
                                                            cplx* Y, double* nu, int* row_rank, int* cand_used) {
    extern __shared__ cplx sm[];
    cplx* Mi = sm;          // r x r
    cplx* ys = Mi + r * r;  // r
    const int lane = threadIdx.x;
    for (int i = lane; i < r * r; i += 32) Mi[i] = make_double2((i / r == i % r) ? 1.0 : 0.0, 0.0);
    __syncwarp();
    const long long kl = lane < r ? (long long)kept[lane] : 0;
    // residual 1 - w M w^H of candidate row c; y (this lane's entry) = M conj(w)
    auto residual = [&](int c, cplx& yl) -> double {
        const cplx wl = lane < r ? A[c + kl * M] : make_double2(0.0, 0.0);
        cplx s = make_double2(0.0, 0.0);
        for (int j = 0; j < r; ++j) {
            cplx wj;
            wj.x = __shfl_sync(0xffffffffu, wl.x, j);
            wj.y = __shfl_sync(0xffffffffu, wl.y, j);
            if (lane < r) {
                const cplx mm = Mi[lane * r + j];
                s.x += mm.x * wj.x + mm.y * wj.y;
                s.y += mm.y * wj.x - mm.x * wj.y;
            }
        }
        yl = s;
        double acc = lane < r ? wl.x * s.x - wl.y * s.y : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        return 1.0 - __shfl_sync(0xffffffffu, acc, 0);
    };
    int p = 0;
    for (int t = 0; t < m; ++t) {
        int chosen = -1;
        double res = 0.0;
        cplx yl = make_double2(0.0, 0.0);
        for (; p < ncand; ++p) {
            if (cand_used[p]) continue;
            res = residual(cand[p], yl);
            if (res >= MIN_RES2) {
                chosen = p;
                break;
            }
        }
        if (chosen < 0) {
            // no candidate reaches 1/4: the largest residual, earliest on ties
            double best = -1.0;
            int bi = -1;
            for (int q = 0; q < ncand; ++q) {
                if (cand_used[q]) continue;
                cplx yq;
                const double rq = residual(cand[q], yq);
                if (rq > best) {
                    best = rq;
                    bi = q;
                }
            }
            // non-finite residuals: the first unused candidate (indices stay in bounds)
            chosen = bi;
            if (chosen < 0)
                for (int q = 0; q < ncand; ++q)
                    if (!cand_used[q]) {
                        chosen = q;
                        break;
                    }
            if (chosen < 0) chosen = 0;
            res = residual(cand[chosen], yl);
            p = ncand;
        } else {
            ++p;
        }
        const int c = cand[chosen];
        if (lane == 0) {
            acc_rows[t] = c;
            nu[t] = sqrt(res);
            row_rank[c] = t;
            cand_used[chosen] = 1;
        }
        if (lane < r) {
            Y[(long long)t * r + lane] = yl;
            ys[lane] = yl;
        }
        __syncwarp();
        const double inv = 1.0 / res;
        for (int idx = lane; idx < r * r; idx += 32) {
            const int i = idx / r, j = idx % r;   // M += y y^H / res
            const cplx yi = ys[i], yj = ys[j];
            Mi[idx].x += inv * (yi.x * yj.x + yi.y * yj.y);
            Mi[idx].y += inv * (yi.y * yj.x - yi.x * yj.y);
        }
        __syncwarp();
    }
}

// U[:, t] = (e_{a_t} - (Q_r y_t, rows accepted before t zeroed)) / nu_t
__global__ void __launch_bounds__(QB) sc_materialize_kernel(cplx* A, long long M, const int* kept, int r,
                                                            const int* dep, int m, const cplx* Y, const double* nu,
                                                            const int* acc_rows, const int* row_rank) {
    extern __shared__ cplx sY[];
    __shared__ int sacc[MAXD], sdep[MAXD];
    __shared__ double snu[MAXD];
    for (int i = threadIdx.x; i < r * m; i += blockDim.x) sY[i] = Y[i];
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        sacc[t] = acc_rows[t];
        sdep[t] = dep[t];
        snu[t] = nu[t];
    }
    __syncthreads();
    long long row = blockIdx.x * (long long)QB + threadIdx.x;
    if (row >= M) return;
    const int rk = row_rank[row];
    for (int t = 0; t < m; ++t) {
        cplx s = make_double2(0.0, 0.0);
        if (rk >= t) {
            for (int j = 0; j < r; ++j) {
                cplx q = A[row + (long long)kept[j] * M], yy = sY[t * r + j];
                s.x += q.x * yy.x - q.y * yy.y;
                s.y += q.x * yy.y + q.y * yy.x;
            }
        }
        const double inv = 1.0 / snu[t];
        cplx u = make_double2(((row == sacc[t]) ? 1.0 : 0.0) - s.x, -s.y);
        A[row + (long long)sdep[t] * M] = make_double2(u.x * inv, u.y * inv);
    }
}

}  // namespace

int qr_cgs2(cplx* A, int M, int D, cplx* R, const int* cand, int ncand, QrScratch& ws, cudaStream_t s,
            int* n_dependent_host, double tol) {
    int launches = 0;
    const long long MM = M;
    const int G = (int)((MM + QB - 1) / QB);
    cplx* part1 = ws.part;
    cplx* part2 = ws.part + (size_t)G * (D + 1);
    cudaMemsetAsync(R, 0, sizeof(cplx) * (size_t)D * D, s);
    // one cooperative launch for the column loop when all G blocks fit on
    // the GPU at once (with as many cached columns per block as allows);
    // otherwise three launches per column
    // launch options: cached columns and look-ahead window; the smaller
    // shared-memory footprints let more row blocks be co-resident (with no
    // cached columns and a window of 4, 65536-row matrices of bond dimension
    // 256 fit in one cooperative launch)
    // (co-resident block counts and kernel attributes are per device: kept
    // for every device the process uses)
    static std::mutex dev_mu;
    static int coop_limits[64][4];
    static bool dev_ready[64] = {};
    static const int nc_opts[4] = {QC_MAX, 8, 0, 0};
    static const int la_opts[4] = {LA_WMAX, LA_WMAX, LA_WMAX, 4};
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    if (cur_dev < 0 || cur_dev >= 64) cur_dev = 0;
    std::unique_lock<std::mutex> dev_lock(dev_mu);
    int* coop_limit = coop_limits[cur_dev];
    if (!dev_ready[cur_dev]) {
        dev_ready[cur_dev] = true;
        int dev = cur_dev, nsm = 0, coop = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(qr_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(cplx) * (QC_MAX * QCS + LA_WMAX * QB)));
        for (int i = 0; i < 4; ++i) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, qr_coop_kernel, QB,
                                                          sizeof(cplx) * (nc_opts[i] * QCS + la_opts[i] * QB));
            coop_limit[i] = coop ? nsm * per_sm : 0;
        }
    }
    dev_lock.unlock();   // the limits of a device never change once set
    bool coop_done = false;
    for (int i = 0; i < 4 && !coop_done && D <= MAXD; ++i) {
        if (G > coop_limit[i]) continue;
        int nc = nc_opts[i], la = la_opts[i];
        size_t smem = sizeof(cplx) * (nc * QCS + la * QB);
        // the barrier leaves its arrival count at zero after every completed
        // wait, so it needs a reset only after an error
        void* args[] = {(void*)&A, (void*)&MM, (void*)&D, (void*)&R, (void*)&ws.flags, (void*)&ws.part,
                        (void*)&ws.h, (void*)&ws.bar, (void*)&ws.err, (void*)&nc, (void*)&tol, (void*)&la};
        coop_done = cudaLaunchCooperativeKernel((const void*)qr_coop_kernel, dim3(G), dim3(QB), args, smem, s) ==
                    cudaSuccess;
        if (!coop_done) cudaGetLastError();   // clear and use the multi-launch path
        launches += 1;
    }
    if (!coop_done) {
        int Gf = (int)std::min<long long>((MM * D + 255) / 256, QR_FROB_BLOCKS);
        frob_partial_kernel<<<Gf, 256, 0, s>>>(A, MM * D, ws.pnorm);
        frob_finish_kernel<<<1, 32, 0, s>>>(ws.pnorm, Gf, ws.scal);
        col_norm_kernel<<<G, QB, 0, s>>>(A, MM, ws.pnorm);
        launches += 3;
        for (int k = 1; k < D; ++k) {
            qr_k1<<<G, QB, 0, s>>>(A, MM, D, k, ws.pnorm, G, ws.scal, R, ws.flags, part1, tol);
            qr_k2<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, ws.scal, part1, part2, R, G);
            qr_k3<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, part2, R, ws.pnorm, G);
            launches += 3;
        }
        qr_last<<<G, QB, 0, s>>>(A, MM, D, ws.pnorm, G, ws.scal, R, ws.flags, tol);
        launches += 1;
    }

    // dependent columns -> completion
    static thread_local int hflags[MAXD], herr;
    cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * D, cudaMemcpyDeviceToHost, s);
    herr = 0;
    if (coop_done) cudaMemcpyAsync(&herr, ws.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (herr) {   // a grid-barrier wait gave up: clear the flag, report
        cudaMemsetAsync(ws.err, 0, sizeof(int), s);
        cudaMemsetAsync(ws.bar, 0, 2 * sizeof(unsigned), s);
        cudaStreamSynchronize(s);
        return -1;
    }
    int ndep = 0;
    for (int k = 0; k < D; ++k) ndep += hflags[k] ? 1 : 0;
    if (n_dependent_host) *n_dependent_host = ndep;
    if (ndep == 0) return launches;
    const int r = D - ndep;
    if (r <= QR_SC_MAXR && (size_t)r * ndep * sizeof(cplx) <= 96 * 1024) {
        static thread_local int hk[MAXD], hd[MAXD];
        int nk = 0, nd = 0;
        for (int k = 0; k < D; ++k) {
            if (hflags[k]) hd[nd++] = k;
            else hk[nk++] = k;
        }
        cudaMemcpyAsync(ws.kept, hk, sizeof(int) * std::max(nk, 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(ws.dep, hd, sizeof(int) * nd, cudaMemcpyHostToDevice, s);
        int gi = (int)std::min<long long>((std::max<long long>(MM, ncand) + 255) / 256, 1024);
        sc_init_kernel<<<gi, 256, 0, s>>>(ws.row_rank, MM, ws.cand_used, ncand);
        static bool attr[64] = {};   // shared memory above 48 KB (kept rank up to 64), per device
        {
            std::lock_guard<std::mutex> lock(dev_mu);
            if (!attr[cur_dev]) {
                cudaFuncSetAttribute(sc_materialize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     96 * 1024 + 64);
                cudaFuncSetAttribute(sc_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
                attr[cur_dev] = true;
            }
        }
        if (r <= 32) {
            sc_select_warp_kernel<<<1, 32, sizeof(cplx) * ((size_t)r * r + (size_t)r + 1), s>>>(
                A, MM, ws.kept, r, nd, cand, ncand, ws.acc_rows, ws.Y, ws.nu, ws.row_rank, ws.cand_used);
        } else {
            size_t sel_smem = sizeof(cplx) * ((size_t)r * r + 2 * (size_t)r + 2);
            sc_select_kernel<<<1, SC_THREADS, sel_smem, s>>>(A, MM, ws.kept, r, nd, cand, ncand, ws.acc_rows, ws.Y,
                                                             ws.nu, ws.row_rank, ws.cand_used);
        }
        size_t mat_smem = sizeof(cplx) * (size_t)r * nd + 16;
        sc_materialize_kernel<<<G, QB, mat_smem, s>>>(A, MM, ws.kept, r, ws.dep, nd, ws.Y, ws.nu, ws.acc_rows,
                                                      ws.row_rank);
        launches += 3;
        return launches;
    }
    rownorm_kernel<<<G, QB, 0, s>>>(A, MM, D, ws.flags, ws.rownorm);
    launches += 1;
    for (int k = 0; k < D; ++k) {
        if (!hflags[k]) continue;
        gs_unit_kernel<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, ws.rownorm, cand, ncand, part1, G);
        gs_second_kernel<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, part1, ws.pnorm, G);
        normalize_col_kernel<<<G, QB, 0, s>>>(A, MM, k, ws.pnorm, G, ws.rownorm, ws.flags);
        launches += 3;
    }
    return launches;
}
