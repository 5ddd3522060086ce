// Truncated SVD of a bond matrix (Sec. "Tensor network simulations": the
// bond dimension chi bounds the kept singular values).  A = Q R by the
// gauge-move QR (qr.cu), then a one-sided (Hestenes) Jacobi SVD of the small
// square factor R = U_R S V^H on the GPU, then U = Q U_R.
//
// Jacobi: columns r_i, r_j of R are rotated until every pair is orthogonal
// to |r_i^H r_j| <= tol ||r_i|| ||r_j||.  One sweep visits every pair once in
// round-robin order (N' - 1 rounds of N'/2 disjoint pairs, N' = N rounded up
// to even); one cooperative launch runs all sweeps, one block per pair of a
// round, with a grid barrier between rounds (pairs whose inner product is
// below 1e-30 |R|_F^2 are treated as orthogonal).  Complex rotation of a pair with
// alpha = |r_i|^2, beta = |r_j|^2, gamma = r_i^H r_j = g e^{i phi}:
//   zeta = (beta - alpha) / (2 g),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2),  s = c t,
//   r_i <- c r_i - s e^{-i phi} r_j,   r_j <- s r_i + c e^{-i phi} r_j,
// and the same on the columns of V (so that R_0 V = R stays true); then
// sigma_i = |r_i| and U_R's columns are r_i / sigma_i.
#include "common.cuh"

#include <cmath>

namespace {

constexpr int SVD_THREADS = 128;
constexpr unsigned long long SVD_WAIT_NS = 2000000000ull;   // 2 s per barrier wait

__device__ __forceinline__ unsigned long long svd_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier: arrival counter bar[0], generation bar[1].  Bounded: a wait
// that gives up sets *err and every block leaves at its next barrier.
__device__ bool svd_grid_sync(unsigned* bar, unsigned nblocks, int* err) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* vb = bar;
        const unsigned gen = vb[1];
        __threadfence();
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived == nblocks) {
            bar[0] = 0u;
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            const unsigned long long t0 = svd_ns();
            for (long long i = 0;; ++i) {
                if (vb[1] != gen) break;
                if (*(volatile int*)err) {
                    ok = 0;
                    break;
                }
                if ((i & 63) == 63 && svd_ns() - t0 > SVD_WAIT_NS) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*(volatile int*)err) ok = 0;
    }
    __syncthreads();
    return ok != 0;
}

__device__ void pair_of(int k, int r, int Np, int& i, int& j) {
    // round-robin: position 0 fixed, positions 1..Np-1 rotate by r
    auto at = [&](int m) { return m == 0 ? 0 : 1 + (m - 1 + r) % (Np - 1); };
    i = at(k);
    j = at(Np - 1 - k);
}

// info: [0] sweeps run, [1] unused, [2], [3] rotation counters (alternating sweeps)
__global__ void __launch_bounds__(SVD_THREADS) jacobi_kernel(cplx* R, cplx* V, int N, int Np, int max_sweeps,
                                                            double tol, unsigned* bar, int* err, int* info) {
    __shared__ double red[3][SVD_THREADS / 32];
    __shared__ double rot[4];   // c, s, cos phi, sin phi; rot[0] < 0: skip
    const unsigned nb = gridDim.x;
    const int k = blockIdx.x;
    // |R|_F^2, the same in every block (same summation order): pairs whose
    // inner product is below 1e-30 |R|_F^2 are left alone -- columns that
    // rank deficiency has already reduced to rounding noise would otherwise
    // be rotated into denormals and overflow the rotation angle
    __shared__ double s_floor;
    {
        double a = 0.0;
        for (long long e = threadIdx.x; e < (long long)N * N; e += SVD_THREADS) {
            const cplx x = __ldcg(R + e);
            a += x.x * x.x + x.y * x.y;
        }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = a;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < SVD_THREADS / 32; ++q) t += red[0][q];
            s_floor = 1e-30 * t;
        }
        __syncthreads();
    }
    const double floor_g = s_floor;
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        int* cnt = &info[2 + (sweep & 1)];
        if (k == 0 && threadIdx.x == 0) *cnt = 0;
        if (!svd_grid_sync(bar, nb, err)) return;
        for (int r = 0; r < Np - 1; ++r) {
            int i, j;
            pair_of(k, r, Np, i, j);
            if (i > j) {
                const int t = i;
                i = j;
                j = t;
            }
            if (j < N) {
                const cplx* ci = R + (long long)i * N;
                const cplx* cj = R + (long long)j * N;
                double a = 0.0, b = 0.0, gr = 0.0, gi = 0.0;
                // columns move between blocks from round to round: read them
                // through L2 (__ldcg), never from a stale L1 line
                for (int e = threadIdx.x; e < N; e += SVD_THREADS) {
                    const cplx x = __ldcg(ci + e), y = __ldcg(cj + e);
                    a += x.x * x.x + x.y * x.y;
                    b += y.x * y.x + y.y * y.y;
                    gr += x.x * y.x + x.y * y.y;   // conj(x) y
                    gi += x.x * y.y - x.y * y.x;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    a += __shfl_down_sync(0xffffffffu, a, o);
                    b += __shfl_down_sync(0xffffffffu, b, o);
                    gr += __shfl_down_sync(0xffffffffu, gr, o);
                    gi += __shfl_down_sync(0xffffffffu, gi, o);
                }
                __shared__ double redi[SVD_THREADS / 32];
                const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
                if (l == 0) {
                    red[0][w] = a;
                    red[1][w] = b;
                    red[2][w] = gr;
                    redi[w] = gi;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    double A = 0, B = 0, Gr = 0, Gi = 0;
                    for (int q = 0; q < SVD_THREADS / 32; ++q) {
                        A += red[0][q];
                        B += red[1][q];
                        Gr += red[2][q];
                        Gi += redi[q];
                    }
                    const double g = sqrt(Gr * Gr + Gi * Gi);
                    if (g > tol * sqrt(A * B) && g > floor_g) {
                        const double zeta = (B - A) / (2.0 * g);
                        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                        const double c = 1.0 / sqrt(1.0 + t * t);
                        rot[0] = c;
                        rot[1] = c * t;
                        rot[2] = Gr / g;
                        rot[3] = Gi / g;
                        atomicAdd(cnt, 1);
                    } else {
                        rot[0] = -1.0;
                    }
                }
                __syncthreads();
                if (rot[0] >= 0.0) {
                    const double c = rot[0], s = rot[1], pc = rot[2], ps = rot[3];   // e^{-i phi} = pc - i ps
                    for (int m = 0; m < 2; ++m) {
                        cplx* X = m == 0 ? R : V;
                        cplx* xi = X + (long long)i * N;
                        cplx* xj = X + (long long)j * N;
                        for (int e = threadIdx.x; e < N; e += SVD_THREADS) {
                            const cplx x = __ldcg(xi + e), y = __ldcg(xj + e);
                            const cplx yp = make_double2(pc * y.x + ps * y.y, pc * y.y - ps * y.x);   // e^{-i phi} y
                            xi[e] = make_double2(c * x.x - s * yp.x, c * x.y - s * yp.y);
                            xj[e] = make_double2(s * x.x + c * yp.x, s * x.y + c * yp.y);
                        }
                    }
                }
            }
            if (!svd_grid_sync(bar, nb, err)) return;
        }
        if (*(volatile int*)cnt == 0) {
            ++sweep;
            break;
        }
    }
    if (k == 0 && threadIdx.x == 0) info[0] = sweep;
}

// sigma_i = |r_i|; rank order (descending, earlier index first on ties);
// kept count k = min(chi, #{sigma >= eps sigma_max}); discarded weight;
// Ur[:, t] = r_order[t] / sigma (t < k), Vh[t, :] = conj(V[:, order[t]]).
// One block.
__global__ void svd_finish_kernel(const cplx* R, const cplx* V, int N, int chi, double eps, cplx* Ur, cplx* Vh,
                                  double* S, int* kout, double* disc, int* order) {
    extern __shared__ double sig[];
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double s = 0.0;
        for (int e = 0; e < N; ++e) {
            const cplx x = R[(long long)i * N + e];
            s += x.x * x.x + x.y * x.y;
        }
        sig[i] = sqrt(s);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int rk = 0;
        for (int j = 0; j < N; ++j)
            if (sig[j] > sig[i] || (sig[j] == sig[i] && j < i)) ++rk;
        order[rk] = i;
    }
    __syncthreads();
    __shared__ int k;
    __shared__ double smax, tot, kept;
    if (threadIdx.x == 0) {
        smax = sig[order[0]];
        int n = 0;
        if (eps < 0.0) {   // keep exactly min(chi, N) columns, zero values included
            n = chi < N ? chi : N;
        } else {
            while (n < N && n < chi && sig[order[n]] >= eps * smax && sig[order[n]] > 0.0) ++n;
        }
        if (n == 0) n = 1;
        k = n;
        tot = 0.0;
        kept = 0.0;
        for (int t = 0; t < N; ++t) {
            const double s2 = sig[order[t]] * sig[order[t]];
            tot += s2;
            if (t < n) kept += s2;
        }
        *kout = n;
        *disc = tot > 0.0 ? (tot - kept) / tot : 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k; t += blockDim.x) S[t] = sig[order[t]];
    for (long long e = threadIdx.x; e < (long long)N * k; e += blockDim.x) {
        const int t = (int)(e / N), row = (int)(e % N);
        const int i = order[t];
        const double inv = sig[i] > 0.0 ? 1.0 / sig[i] : 0.0;
        const cplx x = R[(long long)i * N + row];
        Ur[e] = make_double2(x.x * inv, x.y * inv);
        const cplx v = V[(long long)i * N + row];
        Vh[t + (long long)k * row] = make_double2(v.x, -v.y);   // Vh is k x N, column-major
    }
}

__global__ void identity_kernel(cplx* V, int N) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)N * N;
         e += (long long)gridDim.x * blockDim.x)
        V[e] = make_double2((e % N) == (e / N) ? 1.0 : 0.0, 0.0);
}

}  // namespace

int svd_jacobi_square(cplx* R, cplx* V, int N, int max_sweeps, double tol, unsigned* bar, int* err, int* info,
                      cudaStream_t s) {
    const int Np = N + (N & 1);
    identity_kernel<<<(N * N + 255) / 256, 256, 0, s>>>(V, N);
    cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s);
    cudaMemsetAsync(info, 0, 4 * sizeof(int), s);
    if (Np < 2) return 1;
    int blocks = Np / 2;
    void* args[] = {(void*)&R, (void*)&V, (void*)&N, (void*)&Np, (void*)&max_sweeps, (void*)&tol,
                    (void*)&bar, (void*)&err, (void*)&info};
    if (cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(blocks), dim3(SVD_THREADS), args, 0, s) !=
        cudaSuccess)
        return -1;
    return 2;
}

int svd_finish(const cplx* R, const cplx* V, int N, int chi, double eps, cplx* Ur, cplx* Vh, double* S, int* k,
               double* disc, int* order, cudaStream_t s) {
    svd_finish_kernel<<<1, 256, sizeof(double) * N, s>>>(R, V, N, chi, eps, Ur, Vh, S, k, disc, order);
    return 1;
}
