// FP64 complex strided contraction (see GemmArgs in common.cuh).
//
// Every contraction of the TDVP update -- a matrix on one leg of a 3-leg node
// tensor, the channel sums of the cross terms, the environment
// renormalisations X^H (op x X) -- is one call of this kernel with suitable
// strides.  Tile: 16, 32 or 64 complex outputs per side (picked from M and N),
// 256 threads, up to 4 x 4 complex accumulators per thread, K staged through
// shared memory in slices of 8.
// GB300's FP64 pipe (about 2 DFMA/clk/SM) is the bound, not memory: a simple
// register-tiled loop is enough to saturate it, so loads use generic strides
// (with bounds checks that zero-fill) rather than TMA.
#include "common.cuh"

#include <algorithm>

namespace {

constexpr int THREADS = 256;   // 16 x 16 threads; each owns a TM x TN register tile

__device__ __forceinline__ cplx cmul_acc(cplx acc, cplx a, cplx b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
    return acc;
}

// Tile BM x BN (each 16, 32 or 64), chosen from the problem shape so that small
// outputs (3 x 3 physical legs, 9 x 9 projections) do not spend GB300's scarce
// FP64 throughput on padding.
template <int BM, int BN>
__global__ void __launch_bounds__(THREADS) zgemm_f64_kernel(GemmArgs g) {
    constexpr int TM = BM / 16, TN = BN / 16;
    // K slice per shared-memory stage: 8, or 32 for 16 x 16 tiles, whose small
    // outputs (9 x 9 blocks) otherwise spend a global-memory round trip on
    // every 8 of a long K (9 x 9 x 729: 92 round trips per launch)
    constexpr int BK = (BM == 16 && BN == 16) ? 32 : 8;
    __shared__ cplx As[2][BK][BM];
    __shared__ cplx Bs[2][BK][BN];

    const int b = blockIdx.z;
    const int bi = b % g.Bi, bo = b / g.Bi;
    const cplx* A = g.A + bi * g.a_bi + bo * g.a_bo;
    const cplx* B = g.B + bi * g.b_bi + bo * g.b_bo;
    cplx* C = g.C + bi * g.c_bi + bo * g.c_bo;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int K = g.Ki * g.Ko;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    // warps whose rows (or columns) are all outside the matrix skip the FMAs
    const bool active = (m0 + ty < g.M) && (n0 + tx < g.N);

    cplx acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = make_double2(0.0, 0.0);

    auto load = [&](int k0, int buf) {
        for (int e = tid; e < BK * BM; e += THREADS) {
            int kk = e / BM, mm = e % BM;          // A: m fastest
            int m = m0 + mm, k = k0 + kk;
            cplx v = make_double2(0.0, 0.0);
            if (m < g.M && k < K) {
                int ki = k % g.Ki, ko = k / g.Ki;
                v = A[m * g.a_m + ki * g.a_ki + ko * g.a_ko];
                if (g.conjA) v.y = -v.y;
            }
            As[buf][kk][mm] = v;
        }
        for (int e = tid; e < BK * BN; e += THREADS) {
            int kb = e / BN, nn = e % BN;          // B: n fastest
            int n = n0 + nn, k2 = k0 + kb;
            cplx w = make_double2(0.0, 0.0);
            if (n < g.N && k2 < K) {
                int ki = k2 % g.Ki, ko = k2 / g.Ki;
                w = B[ki * g.b_ki + ko * g.b_ko + n * g.b_n];
                if (g.conjB) w.y = -w.y;
            }
            Bs[buf][kb][nn] = w;
        }
    };

    int buf = 0;
    load(0, 0);
    __syncthreads();
    for (int k0 = 0; k0 < K; k0 += BK) {
        if (k0 + BK < K) load(k0 + BK, buf ^ 1);
        if (active) {
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                cplx a[TM], bb[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty + i * 16];
#pragma unroll
                for (int j = 0; j < TN; ++j) bb[j] = Bs[buf][kk][tx + j * 16];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) acc[i][j] = cmul_acc(acc[i][j], a[i], bb[j]);
            }
        }
        __syncthreads();
        buf ^= 1;
    }

    const bool beta0 = (g.beta.x == 0.0 && g.beta.y == 0.0);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int m = m0 + ty + i * 16;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int n = n0 + tx + j * 16;
            if (n >= g.N) continue;
            cplx* cp = C + m * g.c_m + n * g.c_n;
            cplx v = acc[i][j];
            cplx r;
            r.x = g.alpha.x * v.x - g.alpha.y * v.y;
            r.y = g.alpha.x * v.y + g.alpha.y * v.x;
            if (!beta0) {
                cplx c0 = *cp;
                r.x += g.beta.x * c0.x - g.beta.y * c0.y;
                r.y += g.beta.x * c0.y + g.beta.y * c0.x;
            }
            *cp = r;
        }
    }
}

template <int BM, int BN>
void launch_tile(const GemmArgs& g, cudaStream_t stream) {
    long long batches = (long long)g.Bi * g.Bo;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, (unsigned)batches);
    zgemm_f64_kernel<BM, BN><<<grid, THREADS, 0, stream>>>(g);
}

// Tile width for one dimension: the widest of 16, 32, 64 whose padded size is
// within 5 % of the least padded one (81 -> 32: 96 rows instead of 128).
int tile_for(int x) {
    auto pad = [&](int b) { return (long long)((x + b - 1) / b) * b; };
    const long long best = std::min(pad(16), std::min(pad(32), pad(64)));
    for (int b : {64, 32})
        if (pad(b) * 20 <= best * 21) return b;
    return 16;
}

template <int BM>
void launch_n(const GemmArgs& g, cudaStream_t stream, int bn) {
    if (bn == 16) launch_tile<BM, 16>(g, stream);
    else if (bn == 32) launch_tile<BM, 32>(g, stream);
    else launch_tile<BM, 64>(g, stream);
}

}  // namespace

int launch_zgemm_f64(const GemmArgs& g, cudaStream_t stream) {
    if (g.M <= 0 || g.N <= 0 || g.Bi <= 0 || g.Bo <= 0) return 0;
    const int bm = tile_for(g.M), bn = tile_for(g.N);
    if (bm == 16) launch_n<16>(g, stream, bn);
    else if (bm == 32) launch_n<32>(g, stream, bn);
    else launch_n<64>(g, stream, bn);
    return 1;
}
