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
// ks_len > 0: split-K, this block's z index also selects the K range
// [ks * ks_len, (ks + 1) * ks_len) and the raw sum goes to W (plain store,
// batch-major, m fastest); a second kernel adds the ranges in fixed order.
template <int BM, int BN>
__global__ void __launch_bounds__(THREADS) zgemm_f64_kernel(GemmArgs g, int ks_len, cplx* W) {
    constexpr int TM = BM / 16, TN = BN / 16;
    // K slice per shared-memory stage: 8, or 32 for 16 x 16 tiles, whose small
    // outputs (9 x 9 blocks) otherwise spend a global-memory round trip on
    // every 8 of a long K (9 x 9 x 729: 92 round trips per launch)
    constexpr int BK = (BM == 16 && BN == 16) ? 32 : 8;
    __shared__ cplx As[2][BK][BM];
    __shared__ cplx Bs[2][BK][BN];

    const long long nbatch = (long long)g.Bi * g.Bo;
    const int b = (int)(blockIdx.z % nbatch);
    const int ks = (int)(blockIdx.z / nbatch);
    const int bi = b % g.Bi, bo = b / g.Bi;
    const cplx* A = g.A + bi * g.a_bi + bo * g.a_bo;
    const cplx* B = g.B + bi * g.b_bi + bo * g.b_bo;
    cplx* C = g.C + bi * g.c_bi + bo * g.c_bo;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int Kfull = g.Ki * g.Ko;
    const int kbeg = ks_len > 0 ? ks * ks_len : 0;
    const int K = ks_len > 0 ? min(Kfull, kbeg + ks_len) : Kfull;   // loop runs over [kbeg, K)
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
    load(kbeg, 0);
    __syncthreads();
    for (int k0 = kbeg; k0 < K; k0 += BK) {
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

    if (ks_len > 0) {   // split-K partial: raw sum, reduced by splitk_f64_kernel
        cplx* Wb = W + ((long long)ks * nbatch + b) * g.M * (long long)g.N;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            int m = m0 + ty + i * 16;
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < TN; ++j) {
                int n = n0 + tx + j * 16;
                if (n < g.N) Wb[m + (long long)n * g.M] = acc[i][j];
            }
        }
        return;
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

// C = alpha sum_ks W[ks] + beta C in fixed order.
__global__ void splitk_f64_kernel(GemmArgs g, int nsplit, const cplx* W) {
    const long long MN = (long long)g.M * g.N, nbatch = (long long)g.Bi * g.Bo, total = MN * nbatch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / MN, mn = e - b * MN;
        const int m = (int)(mn % g.M), n = (int)(mn / g.M);
        cplx v = W[b * MN + mn];
        for (int ks = 1; ks < nsplit; ++ks) {
            const cplx w = W[((long long)ks * nbatch + b) * MN + mn];
            v.x += w.x;
            v.y += w.y;
        }
        const int bi = (int)(b % g.Bi), bo = (int)(b / g.Bi);
        cplx* cp = g.C + bi * g.c_bi + bo * g.c_bo + m * g.c_m + n * g.c_n;
        cplx r;
        r.x = g.alpha.x * v.x - g.alpha.y * v.y;
        r.y = g.alpha.x * v.y + g.alpha.y * v.x;
        if (g.beta.x != 0.0 || g.beta.y != 0.0) {
            const cplx c0 = *cp;
            r.x += g.beta.x * c0.x - g.beta.y * c0.y;
            r.y += g.beta.x * c0.y + g.beta.y * c0.x;
        }
        *cp = r;
    }
}

template <int BM, int BN>
void launch_tile(const GemmArgs& g, cudaStream_t stream, int nsplit, int ks_len, cplx* W) {
    long long batches = (long long)g.Bi * g.Bo;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, (unsigned)(batches * nsplit));
    zgemm_f64_kernel<BM, BN><<<grid, THREADS, 0, stream>>>(g, nsplit > 1 ? ks_len : 0, W);
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
void launch_n(const GemmArgs& g, cudaStream_t stream, int bn, int nsplit, int ks_len, cplx* W) {
    if (bn == 16) launch_tile<BM, 16>(g, stream, nsplit, ks_len, W);
    else if (bn == 32) launch_tile<BM, 32>(g, stream, nsplit, ks_len, W);
    else launch_tile<BM, 64>(g, stream, nsplit, ks_len, W);
}

// Split-K when the output tiles cannot fill the GPU and K is long: K ranges
// of at least 64 so that every SM gets a block (the 9 x 9 x 729
// renormalisations of 9-wide legs otherwise ran one block per batch).
int f64_split(const GemmArgs& g, int bm, int bn, int& ks_len) {
    const long long K = (long long)g.Ki * g.Ko;
    const long long tiles = (long long)((g.N + bn - 1) / bn) * ((g.M + bm - 1) / bm) * g.Bi * g.Bo;
    if (tiles >= 152 || K < 256) return 1;
    long long ns = std::min<long long>((304 + tiles - 1) / tiles, K / 64);
    ns = std::max<long long>(1, std::min<long long>(ns, 64));
    ks_len = (int)(((K + ns - 1) / ns + 31) / 32 * 32);   // whole K slices of 32
    return (int)((K + ks_len - 1) / ks_len);
}

}  // namespace

size_t f64_workspace_bytes(const GemmArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.Bi <= 0 || g.Bo <= 0) return 0;
    int ks_len = 0;
    const int ns = f64_split(g, tile_for(g.M), tile_for(g.N), ks_len);
    return ns > 1 ? (size_t)ns * g.Bi * g.Bo * (size_t)g.M * g.N * sizeof(cplx) : 0;
}

int launch_zgemm_f64(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    if (g.M <= 0 || g.N <= 0 || g.Bi <= 0 || g.Bo <= 0) return 0;
    const int bm = tile_for(g.M), bn = tile_for(g.N);
    int ks_len = 0;
    int ns = f64_split(g, bm, bn, ks_len);
    if (ns > 1 && (!workspace || workspace_bytes < f64_workspace_bytes(g))) ns = 1;   // no room: unsplit
    cplx* W = reinterpret_cast<cplx*>(workspace);
    if (bm == 16) launch_n<16>(g, stream, bn, ns, ks_len, W);
    else if (bm == 32) launch_n<32>(g, stream, bn, ns, ks_len, W);
    else launch_n<64>(g, stream, bn, ns, ks_len, W);
    if (ns == 1) return 1;
    const long long total = (long long)g.M * g.N * g.Bi * g.Bo;
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 152 * 8);
    splitk_f64_kernel<<<grid, 256, 0, stream>>>(g, ns, W);
    return 2;
}
