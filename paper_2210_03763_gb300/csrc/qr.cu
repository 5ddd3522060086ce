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
// Each column costs four kernels over G row-chunks (fixed-order partial sums,
// no atomics, no grid-wide waits): [scale column k-1, dots] ->
// [update, dots] -> [update, norm] -> [finish: R_kk, flag, 1/R_kk].
#include "common.cuh"

namespace {

constexpr double QR_TOL = 1e-10;
constexpr double MIN_RES2 = 0.25;

__global__ void frob_finish_kernel(const double* partial, int G, double* scal) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[g];
    scal[0] = s;
}

// scal[0] = ||A||_F^2, scal[1] <- factor for normalising column k
__global__ void finish_col_kernel(const double* partial, int G, double* scal, cplx* R, int D, int k,
                                  int* flags) {
    if (threadIdx.x != 0) return;
    double s = 0.0;
    for (int g = 0; g < G; ++g) s += partial[g];
    double nrm = sqrt(s);
    double fro = sqrt(scal[0]);
    int dep = (fro == 0.0) || (nrm <= QR_TOL * fro);
    R[(long long)k * D + k] = make_double2(dep ? 0.0 : nrm, 0.0);
    scal[1] = dep ? 0.0 : 1.0 / nrm;
    flags[k] = dep;
}

__global__ void scale_col_kernel(cplx* col, long long M, const double* f) {
    double s = f[0];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
         e += (long long)gridDim.x * blockDim.x) {
        cplx v = col[e];
        col[e] = make_double2(v.x * s, v.y * s);
    }
}

__global__ void norm_col_partial_kernel(const cplx* col, long long M, int G, double* partial) {
    __shared__ double sh[32];
    long long c = (M + G - 1) / G, lo = blockIdx.x * c, hi = lo + c < M ? lo + c : M;
    double s = 0.0;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) s += col[e].x * col[e].x + col[e].y * col[e].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
        partial[blockIdx.x] = r;
    }
}

__global__ void rownorm_kernel(const cplx* A, long long M, int D, double* rownorm) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < M;
         r += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = 0; j < D; ++j) {
            cplx v = A[r + (long long)j * M];
            s += v.x * v.x + v.y * v.y;
        }
        rownorm[r] = s;
    }
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
        if (res > best || (res == best && p < bi)) { best = res; bi = p; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        int f2 = __shfl_down_sync(0xffffffffu, first, o);
        double b2 = __shfl_down_sync(0xffffffffu, best, o);
        int i2 = __shfl_down_sync(0xffffffffu, bi, o);
        first = min(first, f2);
        if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
    }
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sfirst[w] = first; sbest[w] = best; sbi[w] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = ncand, b = ncand;
        double bv = -1.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            f = min(f, sfirst[i]);
            if (sbest[i] > bv || (sbest[i] == bv && sbi[i] < b)) { bv = sbest[i]; b = sbi[i]; }
        }
        int p = f < ncand ? f : b;
        pick[0] = (p < ncand) ? cand[p] : 0;
    }
}

// column k <- e_c - sum_j A_j conj(A(c, j))  (first Gram-Schmidt pass of e_c)
__global__ void gs_unit_kernel(cplx* A, long long M, int D, int k, const int* pick) {
    extern __shared__ cplx rowc[];
    const int c = pick[0];
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        cplx v = A[c + (long long)j * M];
        rowc[j] = (j == k) ? make_double2(0.0, 0.0) : make_double2(v.x, -v.y);
    }
    __syncthreads();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < M;
         r += (long long)gridDim.x * blockDim.x) {
        cplx s = make_double2(r == c ? 1.0 : 0.0, 0.0);
        for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            cplx a = A[r + (long long)j * M], h = rowc[j];
            s.x -= a.x * h.x - a.y * h.y;
            s.y -= a.x * h.y + a.y * h.x;
        }
        A[r + (long long)k * M] = s;
    }
}

__global__ void normalize_col_kernel(cplx* col, long long M, const double* partial, int G, double* rownorm) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int g = 0; g < G; ++g) s += partial[g];
        inv = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    }
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M;
         e += (long long)gridDim.x * blockDim.x) {
        cplx v = col[e];
        v.x *= inv;
        v.y *= inv;
        col[e] = v;
        rownorm[e] += v.x * v.x + v.y * v.y;
    }
}

inline int gridM(long long M) {
    long long g = (M + 255) / 256;
    if (g > 608) g = 608;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int qr_cgs2(cplx* A, int M, int D, cplx* R, const int* cand, int ncand, QrScratch& ws, cudaStream_t s,
            int* n_dependent_host) {
    int launches = 0;
    const long long MM = M;
    const int G = red_blocks_for(MM);
    const int Gf = red_blocks_for(MM * D);
    cudaMemsetAsync(R, 0, sizeof(cplx) * (size_t)D * D, s);
    // ||A||_F^2
    norm_col_partial_kernel<<<Gf, 256, 0, s>>>(A, MM * D, Gf, ws.pnorm);
    frob_finish_kernel<<<1, 32, 0, s>>>(ws.pnorm, Gf, ws.scal);
    launches += 2;
    for (int k = 0; k < D; ++k) {
        cplx* col = A + (long long)k * M;
        cplx* Rcol = R + (long long)k * D;
        if (k == 0) {
            norm_col_partial_kernel<<<G, 256, 0, s>>>(col, MM, G, ws.pnorm);
            launches += 1;
        } else {
            launches += k_dots_scaled(A, MM, k, col, MM, ws.part, k - 1, ws.scal + 1, -1, s);
            launches += k_orth_update_ex(A, MM, k, ws.part, col, MM, 1, ws.part + (size_t)RED_BLOCKS * (D + 1),
                                         nullptr, Rcol, 0, -1, s);
            launches += k_orth_update_ex(A, MM, k, ws.part + (size_t)RED_BLOCKS * (D + 1), col, MM, 2, nullptr,
                                         ws.pnorm, Rcol, 1, -1, s);
        }
        finish_col_kernel<<<1, 32, 0, s>>>(ws.pnorm, G, ws.scal, R, D, k, ws.flags);
        launches += 1;
    }
    scale_col_kernel<<<gridM(MM), 256, 0, s>>>(A + (long long)(D - 1) * M, MM, ws.scal + 1);
    launches += 1;

    // dependent columns -> completion
    static thread_local int hflags[4096];
    cudaMemcpyAsync(hflags, ws.flags, sizeof(int) * D, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    int ndep = 0;
    for (int k = 0; k < D; ++k) ndep += hflags[k] ? 1 : 0;
    if (n_dependent_host) *n_dependent_host = ndep;
    if (ndep == 0) return launches;
    rownorm_kernel<<<gridM(MM), 256, 0, s>>>(A, MM, D, ws.rownorm);
    launches += 1;
    for (int k = 0; k < D; ++k) {
        if (!hflags[k]) continue;
        cplx* col = A + (long long)k * M;
        pick_kernel<<<1, 1024, 0, s>>>(ws.rownorm, cand, ncand, ws.pick);
        gs_unit_kernel<<<gridM(MM), 256, sizeof(cplx) * D, s>>>(A, MM, D, k, ws.pick);
        launches += 2;
        launches += k_dots_scaled(A, MM, D, col, MM, ws.part, -1, nullptr, k, s);
        launches += k_orth_update_ex(A, MM, D, ws.part, col, MM, 2, nullptr, ws.pnorm, nullptr, 0, k, s);
        normalize_col_kernel<<<gridM(MM), 256, 0, s>>>(col, MM, ws.pnorm, G, ws.rownorm);
        launches += 1;
    }
    return launches;
}
