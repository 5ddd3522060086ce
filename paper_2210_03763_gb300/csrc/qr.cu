// QR of the tall matricisation of a node tensor (the gauge move of the TDVP
// sweep, Sec. "Tensor network simulations"), FP64.
//
// Column-by-column classical Gram-Schmidt with one re-orthogonalisation pass
// (CGS2), in place on a column-major M x D matrix.  Column k is *dependent*
// when the norm of its residual after both passes is <= 1e-10 ||A||_F; it is
// zeroed (R_kk = 0) and filled after the sweep, in increasing k, by the first
// candidate unit vector e_c (in the caller's candidate order) whose residual
// 1 - ||Q^H e_c||^2 is >= 1/4 (else the candidate with the largest residual,
// earliest on ties), orthogonalised twice against Q and normalised.  R_kk is
// real and >= 0; rows of R of dependent columns are zero.
//
// GB300's FP64 pipe (~7.8 GFLOP/s per SM) bounds this code, so every kernel
// spreads the rows over all SMs (blocks of QB rows, one row per thread), and
// projections skip columns that are still zero (dependent and not yet
// filled): the work is O(M * D * rank) rather than O(M * D^2), which matters
// for the low-entanglement states of GHZ circuits.  Per column three kernels:
//   K1 [decide column k-1 from its norm partials; dots of a_k with columns < k]
//   K2 [sum the dot partials; a_k -= Q h; dots again]
//   K3 [sum; a_k -= Q h2; norm partials]
// Sums over blocks use the partials in one fixed order in every block (no
// atomics), so all blocks see identical values and runs are reproducible.
#include "common.cuh"

#include <algorithm>

namespace {

constexpr double QR_TOL = 1e-10;
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
__device__ double decide(int kd, const double* pnorm, int G, double* scal, cplx* R, int D, int* flags) {
    double s = sum_norm(pnorm, G);
    double nrm = sqrt(s), fro = sqrt(scal[0]);
    int dep = (fro == 0.0) || (nrm <= QR_TOL * fro);
    if (blockIdx.x == 0) {
        R[(long long)kd * D + kd] = make_double2(dep ? 0.0 : nrm, 0.0);
        scal[1] = dep ? 0.0 : 1.0 / nrm;
        flags[kd] = dep;
    }
    return dep ? 0.0 : 1.0 / nrm;
}

// K1 for column k >= 1
__global__ void __launch_bounds__(QB) qr_k1(const cplx* A, long long M, int D, int k, const double* pnorm, int G,
                                            double* scal, cplx* R, int* flags, cplx* part) {
    __shared__ int szero[MAXD];
    __shared__ cplx wsum[MAXD][QB / 32];
    __shared__ double sfac;
    if (threadIdx.x == 0) sfac = decide(k - 1, pnorm, G, scal, R, D, flags);
    for (int i = threadIdx.x; i < k - 1; i += QB) szero[i] = flags[i];
    __syncthreads();
    if (threadIdx.x == 0) szero[k - 1] = (sfac == 0.0);
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    bool valid = r < M;
    cplx w = valid ? A[r + (long long)k * M] : make_double2(0.0, 0.0);
    block_dots(A, M, k, szero, w, valid, r, k - 1, sfac, wsum, part, G, -1);
}

// K2: scale column k-1, h = sum of partials, a_k -= sum_i A_i h_i, dots again
__global__ void __launch_bounds__(QB) qr_k2(cplx* A, long long M, int D, int k, const int* flags, const double* scal,
                                            const cplx* part_in, cplx* part_out, cplx* R, int G) {
    __shared__ int szero[MAXD];
    __shared__ cplx h[MAXD];
    __shared__ cplx wsum[MAXD][QB / 32];
    const double fac = scal[1];
    for (int i = threadIdx.x; i < k; i += QB) {
        szero[i] = flags[i];
        h[i] = szero[i] ? make_double2(0.0, 0.0) : sum_partials(part_in, i, G);
        if (blockIdx.x == 0) R[(long long)k * D + i] = h[i];
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
            if (szero[i]) continue;
            cplx a = A[r + (long long)i * M], hi = h[i];
            w.x -= a.x * hi.x - a.y * hi.y;
            w.y -= a.x * hi.y + a.y * hi.x;
        }
        A[r + (long long)k * M] = w;
    }
    block_dots(A, M, k, szero, w, valid, r, -1, 1.0, wsum, part_out, G, -1);
}

// K3: h2 = sum, R[:k, k] += h2, a_k -= Q h2, norm partials
__global__ void __launch_bounds__(QB) qr_k3(cplx* A, long long M, int D, int k, const int* flags, const cplx* part_in,
                                            cplx* R, double* pnorm, int G) {
    __shared__ int szero[MAXD];
    __shared__ cplx h[MAXD];
    __shared__ double sh[QB / 32];
    for (int i = threadIdx.x; i < k; i += QB) {
        szero[i] = flags[i];
        h[i] = szero[i] ? make_double2(0.0, 0.0) : sum_partials(part_in, i, G);
        if (blockIdx.x == 0) R[(long long)k * D + i] = cadd(R[(long long)k * D + i], h[i]);
    }
    __syncthreads();
    long long r = blockIdx.x * (long long)QB + threadIdx.x;
    double s = 0.0;
    if (r < M) {
        cplx w = A[r + (long long)k * M];
        for (int i = 0; i < k; ++i) {
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

// Decide and scale the last column.
__global__ void __launch_bounds__(QB) qr_last(cplx* A, long long M, int D, const double* pnorm, int G, double* scal,
                                              cplx* R, int* flags) {
    __shared__ double sfac;
    if (threadIdx.x == 0) sfac = decide(D - 1, pnorm, G, scal, R, D, flags);
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

// One block: first candidate with 1 - rownorm >= 1/4, else argmax (earliest).
__global__ void pick_kernel(const double* rownorm, const int* cand, int ncand, int* pick) {
    __shared__ int sfirst[32];
    __shared__ double sbest[32];
    __shared__ int sbi[32];
    int first = ncand;
    double best = -1.0;
    int bi = ncand;
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
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sfirst[w] = first;
        sbest[w] = best;
        sbi[w] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = ncand, b = ncand;
        double bv = -1.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            f = min(f, sfirst[i]);
            if (sbest[i] > bv || (sbest[i] == bv && sbi[i] < b)) {
                bv = sbest[i];
                b = sbi[i];
            }
        }
        int p = f < ncand ? f : b;
        pick[0] = (p < ncand) ? cand[p] : 0;
    }
}

// column k <- e_c - sum_j A_j conj(A(c, j)) over nonzero j; then dots with them
__global__ void __launch_bounds__(QB) gs_unit_kernel(cplx* A, long long M, int D, int k, const int* flags,
                                                     const int* pick, cplx* part, int G) {
    __shared__ int szero[MAXD];
    __shared__ cplx rowc[MAXD];
    __shared__ cplx wsum[MAXD][QB / 32];
    const int c = pick[0];
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

// the completed column becomes part of Q for later completions
__global__ void unflag_kernel(int* flags, int k) {
    if (threadIdx.x == 0) flags[k] = 0;
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
            chosen = sbi;
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
            int* n_dependent_host) {
    int launches = 0;
    const long long MM = M;
    const int G = (int)((MM + QB - 1) / QB);
    cplx* part1 = ws.part;
    cplx* part2 = ws.part + (size_t)G * (D + 1);
    cudaMemsetAsync(R, 0, sizeof(cplx) * (size_t)D * D, s);
    int Gf = (int)std::min<long long>((MM * D + 255) / 256, QR_FROB_BLOCKS);
    frob_partial_kernel<<<Gf, 256, 0, s>>>(A, MM * D, ws.pnorm);
    frob_finish_kernel<<<1, 32, 0, s>>>(ws.pnorm, Gf, ws.scal);
    col_norm_kernel<<<G, QB, 0, s>>>(A, MM, ws.pnorm);
    launches += 3;
    for (int k = 1; k < D; ++k) {
        qr_k1<<<G, QB, 0, s>>>(A, MM, D, k, ws.pnorm, G, ws.scal, R, ws.flags, part1);
        qr_k2<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, ws.scal, part1, part2, R, G);
        qr_k3<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, part2, R, ws.pnorm, G);
        launches += 3;
    }
    qr_last<<<G, QB, 0, s>>>(A, MM, D, ws.pnorm, G, ws.scal, R, ws.flags);
    launches += 1;

    // dependent columns -> completion
    static thread_local int hflags[MAXD];
    cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * D, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int ndep = 0;
    for (int k = 0; k < D; ++k) ndep += hflags[k] ? 1 : 0;
    if (n_dependent_host) *n_dependent_host = ndep;
    if (ndep == 0) return launches;
    const int r = D - ndep;
    if (r <= QR_SC_MAXR && MM >= 4LL * D && (size_t)r * ndep * sizeof(cplx) <= 96 * 1024) {
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
        size_t sel_smem = sizeof(cplx) * ((size_t)r * r + 2 * (size_t)r + 2);
        sc_select_kernel<<<1, SC_THREADS, sel_smem, s>>>(A, MM, ws.kept, r, nd, cand, ncand, ws.acc_rows, ws.Y,
                                                         ws.nu, ws.row_rank, ws.cand_used);
        size_t mat_smem = sizeof(cplx) * (size_t)r * nd + 16;
        static bool attr = false;
        if (!attr) {
            cudaFuncSetAttribute(sc_materialize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024 + 64);
            cudaFuncSetAttribute(sc_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
            attr = true;
        }
        sc_materialize_kernel<<<G, QB, mat_smem, s>>>(A, MM, ws.kept, r, ws.dep, nd, ws.Y, ws.nu, ws.acc_rows,
                                                      ws.row_rank);
        launches += 3;
        return launches;
    }
    rownorm_kernel<<<G, QB, 0, s>>>(A, MM, D, ws.flags, ws.rownorm);
    launches += 1;
    for (int k = 0; k < D; ++k) {
        if (!hflags[k]) continue;
        pick_kernel<<<1, 1024, 0, s>>>(ws.rownorm, cand, ncand, ws.pick);
        gs_unit_kernel<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, ws.pick, part1, G);
        gs_second_kernel<<<G, QB, 0, s>>>(A, MM, D, k, ws.flags, part1, ws.pnorm, G);
        normalize_col_kernel<<<G, QB, 0, s>>>(A, MM, k, ws.pnorm, G, ws.rownorm, ws.flags);
        unflag_kernel<<<1, 32, 0, s>>>(ws.flags, k);
        launches += 5;
    }
    return launches;
}
