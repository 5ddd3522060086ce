// Split-precision complex contraction on the 5th-generation tensor cores
// (tcgen05, kind::tf32), "3xTF32": every FP64 operand x is split into
// hi = tf32(x) and lo = tf32(x - hi); the product is hi*hi + hi*lo + lo*hi with
// FP32 accumulation in tensor memory (the lo*lo term, ~2^-22 relative, is
// dropped).  Result accuracy is close to FP32 (about 1e-7 relative).
//
// Complex numbers use a real embedding.  One side ("P", R x K) becomes
// R x 2K real rows, the other side ("Q", N x K) 2N x 2K, with the K
// axis interleaved as k' = 2k + half:
//   P row r : ( Re p, Im p )        Q row 2n   : ( Re q, -Im q )
//                                   Q row 2n+1 : ( Im q,  Re q )
// so  C~(r, 2n) = Re(sum_k p q) and C~(r, 2n+1) = Im(sum_k p q): the real and
// imaginary parts of an output sit in adjacent TMEM columns of one lane.
// The doubled side is chosen by packed bytes (plan_for).
//
// Two kernels per contraction (three with split-K):
//  1. pack_kernel: gathers the strided FP64 operand (any GemmArgs strides,
//     optional conjugation, batches) into zero-padded K-major FP32 hi/lo
//     planes; HBM bound, coalesced float2 stores.
//  2. tcgen05 GEMM: persistent, one CTA per SM walking 128 x 64 tiles of C~,
//     18 warps; the stage ring and TMEM buffers run on across tiles.  Warp 16
//     issues TMA loads (128-byte swizzle, no multicast) into a 4-stage ring,
//     warp 17 issues 12 tcgen05.mma per 32-wide K slice into one of four TMEM
//     accumulators and releases stages with tcgen05.commit; warps 0-15 drain
//     finished K chunks from TMEM (tcgen05.ld 32x32b, four warps per lane
//     quadrant, 16 columns each) into float-float sums and finally write
//     alpha * C + beta * C in FP64, one complex entry per pair of columns.
//  3. splitk_reduce_kernel when K is split into ranges (few output tiles).
//  Every mbarrier wait is bounded by time; on timeout the kernel sets an
//  error flag, lets its own copies and MMAs finish, frees its TMEM and returns.
#include "common.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

namespace {

constexpr int BM = 128, BN = 64, BK = 32;    // BK in fp32 elements = 128 bytes
constexpr int STAGES = 4;
constexpr int A_TILE = BM * BK * 4;          // 16 KB per plane tile of P
constexpr int B_TILE = BN * BK * 4;          // 8 KB per plane tile of Q
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr long long SPIN_LIMIT = 1LL << 30;                  // iteration cap behind the time limit
constexpr unsigned long long WAIT_NS = 2000000000ull;        // 2 s per pipeline wait

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for a pipeline stage.  Returns false when the phase has not
// completed after WAIT_NS (the error flag is then set) or as soon as another
// role of this launch, or an earlier launch, has set the flag: one stuck
// stage ends the whole launch within about WAIT_NS instead of every waiter
// timing out in turn.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1; i < SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*(volatile int*)err) return false;
            if (global_ns() - t0 > WAIT_NS) break;
        }
    }
    atomicExch(err, 1);
    return false;
}

// Bounded wait that ignores the error flag: used after an abort, to let this
// CTA's own copies and MMAs in flight finish before it frees TMEM and exits.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (long long i = 0; i < SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return;
        if ((i & 63) == 63 && global_ns() - t0 > WAIT_NS) return;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = 64.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dt),
        "l"(a), "l"(b), "r"(IDESC), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Split an FP64 value into TF32-representable hi and lo with integer
// operations only (GB300's FP64 pipe is the bottleneck of any FP64
// arithmetic): hi = x rounded to 10 mantissa bits (to nearest, ties to even),
// lo = the exact remainder x - hi rounded to 11 significant bits; |hi + lo - x|
// <= 2^-23 |x|.  |x| < 2^-126 (and FP64 subnormals) give 0; inf/nan pass
// through the conversion instruction.
__device__ __forceinline__ void split_tf32(double x, float& hi, float& lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(u >> 63);
    const int e = (int)((u >> 52) & 0x7FF);
    const unsigned long long mant = u & 0xFFFFFFFFFFFFFULL;
    hi = 0.f;
    lo = 0.f;
    if (e == 0x7FF) {
        hi = (float)x;
        return;
    }
    if (e == 0) return;
    unsigned long long m10 = mant >> 42;
    const unsigned long long rem = mant & ((1ULL << 42) - 1);
    const unsigned long long half = 1ULL << 41;
    const bool up = rem > half || (rem == half && (m10 & 1ULL));
    int fe = e - 1023 + 127;
    if (up) {
        m10 += 1;
        if (m10 == (1ULL << 10)) {
            m10 = 0;
            fe += 1;
        }
    }
    if (fe <= 0) return;
    hi = __uint_as_float((sign << 31) | ((unsigned)fe << 23) | ((unsigned)m10 << 13));
    const long long r = up ? (long long)rem - (long long)(1ULL << 42) : (long long)rem;
    if (r == 0) return;
    const unsigned lsign = sign ^ (r < 0 ? 1u : 0u);
    const unsigned long long ar = (unsigned long long)(r < 0 ? -r : r);   // < 2^42
    const int msb = 63 - __clzll((long long)ar);
    int le = msb + (e - 1075) + 127;
    unsigned long long m;
    if (msb > 10) {
        const int sh = msb - 10;
        m = ar >> sh;
        const unsigned long long rr = ar & ((1ULL << sh) - 1), h = 1ULL << (sh - 1);
        if (rr > h || (rr == h && (m & 1ULL))) {
            m += 1;
            if (m == (1ULL << 11)) {
                m >>= 1;
                le += 1;
            }
        }
    } else {
        m = ar << (10 - msb);
    }
    if (le <= 0) return;
    lo = __uint_as_float((lsign << 31) | ((unsigned)le << 23) | ((unsigned)(m & 0x3FFULL) << 13));
}

// ----------------------------------------------------------------- packing
struct PackArgs {
    const cplx* src;
    long long s_r, s_ki, s_ko, s_bi, s_bo;   // strides of (row, k_in, k_out, batch_in, batch_out)
    int R, Ki, Ko, Bi, Bo;
    int conj;
    int embed;         // 1: Q side (2 rows per complex row), 0: P side
    int Rp, Kp;        // padded output rows (real) and K' (fp32 elements)
    float* hi;
    float* lo;
};

__global__ void pack_kernel(PackArgs p) {
    const int K = p.Ki * p.Ko;
    const int half_k = p.Kp / 2;                       // complex k positions incl. padding
    const int rows_src = p.embed ? p.Rp / 2 : p.Rp;    // complex rows incl. padding
    const long long per_b = (long long)rows_src * half_k;
    const long long total = per_b * p.Bi * p.Bo;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long b = e / per_b;
        long long rem = e - b * per_b;
        int r = (int)(rem / half_k);
        int k = (int)(rem - (long long)r * half_k);
        double re = 0.0, im = 0.0;
        if (r < p.R && k < K) {
            int bi = (int)(b % p.Bi), bo = (int)(b / p.Bi);
            int ki = k % p.Ki, ko = k / p.Ki;
            cplx v = p.src[bi * p.s_bi + bo * p.s_bo + r * p.s_r + ki * p.s_ki + ko * p.s_ko];
            re = v.x;
            im = p.conj ? __longlong_as_double(__double_as_longlong(v.y) ^ (long long)0x8000000000000000ULL) : v.y;
        }
        float rh, rl, ih, il;
        split_tf32(re, rh, rl);
        split_tf32(im, ih, il);
        long long plane_b = (long long)p.Rp * p.Kp * b;
        if (p.embed) {
            long long o0 = plane_b + (long long)(2 * r) * p.Kp + 2 * k;
            long long o1 = o0 + p.Kp;
            *reinterpret_cast<float2*>(p.hi + o0) = make_float2(rh, -ih);
            *reinterpret_cast<float2*>(p.hi + o1) = make_float2(ih, rh);
            *reinterpret_cast<float2*>(p.lo + o0) = make_float2(rl, -il);
            *reinterpret_cast<float2*>(p.lo + o1) = make_float2(il, rl);
        } else {
            long long o0 = plane_b + (long long)r * p.Kp + 2 * k;
            *reinterpret_cast<float2*>(p.hi + o0) = make_float2(rh, ih);
            *reinterpret_cast<float2*>(p.lo + o0) = make_float2(rl, il);
        }
    }
}

// --------------------------------------------------------------- the GEMM
// The tensor core's FP32 accumulation does not round to nearest: its error
// grows linearly with the accumulation length (measured: ~1e-6 of max|C| at
// K = 128, ~1e-5 at K = 2048, with TF32-exact inputs).  So the K loop is cut
// into chunks of CHUNK_KB slices: the MMA warp accumulates a chunk in one of
// one of NBUF TMEM buffers and starts the next chunk in the next buffer,
// while DRAIN_WARPS drain warps add each finished chunk into float-float
// register sums (Knuth TwoSum, ~2^-48 relative).  Sixteen drain warps (each
// thread one TMEM lane, 16 columns) rather than eight: the drain and the FP64
// epilogue are latency-bound, and twice the warps hid enough of it to cut
// the kernel's time in a TDVP step by a quarter (measured).  The error is then that of one short
// chunk (~3e-7 relative), independent of K.
constexpr int CHUNK_KB = 2;
constexpr int NBUF = 4;                            // TMEM accumulators (NBUF * BN columns)
constexpr int DRAIN_WARPS = 16;                    // warp w: TMEM lanes 32 (w % 4) .., columns DCOLS (w / 4) ..
constexpr int DRAIN_THREADS = 32 * DRAIN_WARPS;
constexpr int DCOLS = BN / (DRAIN_WARPS / 4);      // columns per drain thread
constexpr int TMA_WARP = DRAIN_WARPS, MMA_WARP = DRAIN_WARPS + 1;
constexpr int GEMM_THREADS = DRAIN_THREADS + 64;

struct EpiArgs {
    cplx* C;
    long long c_m, c_n, c_bi, c_bo;
    int M, N, Bi;
    int swapped;          // P side holds the columns n of C (C^T computed)
    int Pp, Qp;           // packed-row stride per batch of P and Q (0 if shared)
    int nkb;              // K' / BK
    int n_ptiles, n_qtiles, batches;   // tile grid; tile t: P tile fastest, then Q tile, then batch
    cplx alpha, beta;
    int mode;             // 0: alpha = 1, beta = 0; 1: alpha = 1, beta = 1; 2: general
    int* err;
    int q_fast;           // tile order inside a batch: Q tiles fastest (else P tiles fastest)
    int nsplit;           // K ranges per output tile (split-K); > 1: partial results go to W
    int cps;              // chunks per K range
    cplx* W;              // nsplit x batches x N x M partial results (column-major per batch)
};

// double(f) built from f's bits with integer operations (GB300's FP64 pipe is
// ~64x slower than its integer pipe; conversions would go through it).
// Normal numbers and zero exactly; FP32 subnormals (< 1.2e-38) become zero;
// inf/nan go through the conversion instruction.
__device__ __forceinline__ double f32_to_f64(float f) {
    uint32_t u = __float_as_uint(f);
    uint32_t e = (u >> 23) & 0xFFu;
    if (e == 0xFFu) return (double)f;
    uint64_t sign = (uint64_t)(u >> 31) << 63;
    if (e == 0u) return __longlong_as_double((long long)sign);
    uint64_t bits = sign | ((uint64_t)(e + (1023u - 127u)) << 52) | ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    float s = __fadd_rn(hi, x);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mPh, const __grid_constant__ CUtensorMap mPl,
                   const __grid_constant__ CUtensorMap mQh, const __grid_constant__ CUtensorMap mQl, EpiArgs ea) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;      // [NBUF] chunk accumulated in TMEM buffer b
    uint64_t* tempty = tfull + NBUF;       // [NBUF] buffer b drained
    uint64_t* mdone = tempty + NBUF;       // all MMAs of this CTA complete
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mdone + 1);

    // an earlier launch on this workspace gave up: do nothing (the host
    // reports the error at its next check)
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = *(volatile int*)ea.err;
    __syncthreads();
    if (s_skip) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchunk = (ea.nkb + CHUNK_KB - 1) / CHUNK_KB;
    const long long ntiles = (long long)ea.nsplit * ea.batches * ea.n_qtiles * ea.n_ptiles;
    // work item t: the tile grid of a batch (the smaller tile count fastest,
    // so that work items running together share the other operand's tile in
    // L2), then batch, then K range; its chunks [c0, c1)
    const long long grid_tiles = (long long)ea.n_ptiles * ea.n_qtiles;
    auto tile_of = [&](long long t, int& pt, int& qt, int& b, int& ks) {
        const long long w = t % grid_tiles, rest = t / grid_tiles;
        if (ea.q_fast) {
            qt = (int)(w % ea.n_qtiles);
            pt = (int)(w / ea.n_qtiles);
        } else {
            pt = (int)(w % ea.n_ptiles);
            qt = (int)(w / ea.n_ptiles);
        }
        b = (int)(rest % ea.batches);
        ks = (int)(rest / ea.batches);
    };
    auto krange = [&](long long t, int& c0, int& c1) {
        const int ks = (int)(t / (grid_tiles * ea.batches));
        c0 = ks * ea.cps;
        c1 = min(nchunk, c0 + ea.cps);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], DRAIN_THREADS);
        }
        mbar_init(mdone, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(NBUF * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // persistent loop over tiles: t = blockIdx.x, blockIdx.x + gridDim.x, ...
    if (warp == TMA_WARP) {
        if (lane == 0) {   // TMA producer: one continuous stage ring across tiles
            unsigned it = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int pt, qt, b, ks;
                tile_of(t, pt, qt, b, ks);
                const int prow0 = b * ea.Pp + pt * BM, qrow0 = b * ea.Qp + qt * BN;
                int c0, c1;
                krange(t, c0, c1);
                const int kb1 = min(ea.nkb, c1 * CHUNK_KB);
                for (int kb = c0 * CHUNK_KB; kb < kb1; ++kb, ++it) {
                    const unsigned s = it % STAGES, round = it / STAGES;
                    if (it >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1, ea.err)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(st, &mPh, &full[s], kb * BK, prow0);
                    tma_load_2d(st + A_TILE, &mPl, &full[s], kb * BK, prow0);
                    tma_load_2d(st + 2 * A_TILE, &mQh, &full[s], kb * BK, qrow0);
                    tma_load_2d(st + 2 * A_TILE + B_TILE, &mQl, &full[s], kb * BK, qrow0);
                }
            }
            // loads of the last STAGES iterations may still be landing if the
            // MMA issuer stopped early: wait for them before the CTA exits
            // (immediate when they were consumed)
            for (unsigned i = it > STAGES ? it - STAGES : 0; i < it; ++i)
                mbar_drain(&full[i % STAGES], (i / STAGES) & 1);
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {   // MMA issuer
            unsigned it = 0, cg = 0;
            bool ok = true;
            for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                int c0, c1;
                krange(t, c0, c1);
                for (int c = c0; c < c1 && ok; ++c, ++cg) {
                    const unsigned buf = cg % NBUF;
                    const uint32_t dt = tmem + (uint32_t)(buf * BN);
                    if (cg >= NBUF && !mbar_wait(&tempty[buf], ((cg / NBUF) - 1) & 1, ea.err)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const int kb_end = min(ea.nkb, (c + 1) * CHUNK_KB);
                    for (int kb = c * CHUNK_KB; kb < kb_end; ++kb, ++it) {
                        const unsigned s = it % STAGES, round = it / STAGES;
                        if (!mbar_wait(&full[s], round & 1, ea.err)) {
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        uint32_t base = smem_u32(smem + s * STAGE_BYTES);
                        uint64_t ph = sdesc(base), pl = sdesc(base + A_TILE);
                        uint64_t qh = sdesc(base + 2 * A_TILE), ql = sdesc(base + 2 * A_TILE + B_TILE);
#pragma unroll
                        for (int ks = 0; ks < BK / 8; ++ks) {
                            uint64_t off = (uint64_t)(ks * 32) >> 4;   // 8 tf32 = 32 bytes along K
                            uint32_t acc = (kb > c * CHUNK_KB || ks > 0) ? 1u : 0u;
                            mma_tf32(dt, pl + off, qh + off, acc);
                            mma_tf32(dt, ph + off, ql + off, 1u);
                            mma_tf32(dt, ph + off, qh + off, 1u);
                        }
                        mma_commit(&empty[s]);
                    }
                    mma_commit(&tfull[buf]);
                }
            }
            mma_commit(mdone);   // completes once every MMA issued above has
            mbar_drain(mdone, 0);
        }
        __syncwarp();
    } else {
        // drain warps: thread = TMEM lane (tile row), DCOLS columns per thread
        const int quad = warp & 3, col0 = (warp >> 2) * DCOLS;
        const bool beta0 = (ea.beta.x == 0.0 && ea.beta.y == 0.0);
        unsigned cg = 0;
        bool ok = true;
        for (long long t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            int pt, qt, b, ks;
            tile_of(t, pt, qt, b, ks);
            int c0, c1;
            krange(t, c0, c1);
            float hi[DCOLS], lo[DCOLS];
#pragma unroll
            for (int j = 0; j < DCOLS; ++j) {
                hi[j] = 0.f;
                lo[j] = 0.f;
            }
            for (int c = c0; c < c1; ++c, ++cg) {
                const unsigned buf = cg % NBUF;
                if (!mbar_wait(&tfull[buf], (cg / NBUF) & 1, ea.err)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int c0 = 0; c0 < DCOLS; c0 += 16) {
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + col0 + c0), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) two_sum_acc(hi[c0 + j], lo[c0 + j], v[j]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
            }
            if (!ok) break;
            const int trow = quad * 32 + lane;                  // row of C~ inside the tile
            const int pr = pt * BM + trow;                      // complex row of P
            const int bi = b % ea.Bi, bo = b / ea.Bi;
            cplx* C = ea.C + bi * ea.c_bi + bo * ea.c_bo;
            // split-K: this K range's partial sum, dense column-major, plain store
            cplx* Wt = ea.nsplit > 1 ? ea.W + ((long long)ks * ea.batches + b) * ea.M * (long long)ea.N : nullptr;
            // columns 2q and 2q + 1 of C~ hold the real and imaginary parts of
            // one entry (the Q side carries the real embedding), so each
            // thread owns whole complex outputs
#pragma unroll
            for (int j = 0; j < DCOLS; j += 2) {
                const int qn = (qt * BN + col0 + j) >> 1;       // complex row of Q = the other index
                const int m = ea.swapped ? qn : pr;
                const int n = ea.swapped ? pr : qn;
                if (m >= ea.M || n >= ea.N) continue;
                const double re = f32_to_f64(hi[j]) + f32_to_f64(lo[j]);
                const double im = f32_to_f64(hi[j + 1]) + f32_to_f64(lo[j + 1]);
                if (Wt) {
                    Wt[m + (long long)n * ea.M] = make_double2(re, im);
                    continue;
                }
                cplx* cp = C + m * ea.c_m + n * ea.c_n;
                cplx r;
                if (ea.mode == 0) {                 // alpha = 1, beta = 0
                    r = make_double2(re, im);
                } else if (ea.mode == 1) {          // alpha = 1, beta = 1
                    cplx o = *cp;
                    r = make_double2(o.x + re, o.y + im);
                } else {
                    r.x = ea.alpha.x * re - ea.alpha.y * im;
                    r.y = ea.alpha.x * im + ea.alpha.y * re;
                    if (!beta0) {
                        cplx o = *cp;
                        r.x += ea.beta.x * o.x - ea.beta.y * o.y;
                        r.y += ea.beta.x * o.y + ea.beta.y * o.x;
                    }
                }
                *cp = r;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NBUF * BN));
    }
}

// C = alpha sum_ks W[ks] + beta C, summing the K ranges in increasing order.
__global__ void splitk_reduce_kernel(EpiArgs ea) {
    const long long MN = (long long)ea.M * ea.N, total = MN * ea.batches;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / MN);
        const long long mn = e - b * MN;
        const int m = (int)(mn % ea.M), n = (int)(mn / ea.M);
        cplx acc = ea.W[(long long)b * MN + mn];
        for (int ks = 1; ks < ea.nsplit; ++ks) {
            cplx w = ea.W[((long long)ks * ea.batches + b) * MN + mn];
            acc.x += w.x;
            acc.y += w.y;
        }
        const int bi = b % ea.Bi, bo = b / ea.Bi;
        cplx* cp = ea.C + bi * ea.c_bi + bo * ea.c_bo + m * ea.c_m + n * ea.c_n;
        cplx r;
        if (ea.mode == 0) {
            r = acc;
        } else if (ea.mode == 1) {
            cplx o = *cp;
            r = make_double2(o.x + acc.x, o.y + acc.y);
        } else {
            r.x = ea.alpha.x * acc.x - ea.alpha.y * acc.y;
            r.y = ea.alpha.x * acc.y + ea.alpha.y * acc.x;
            if (ea.beta.x != 0.0 || ea.beta.y != 0.0) {
                cplx o = *cp;
                r.x += ea.beta.x * o.x - ea.beta.y * o.y;
                r.y += ea.beta.x * o.y + ea.beta.y * o.x;
            }
        }
        *cp = r;
    }
}

// ------------------------------------------------------------------- host
int num_sms() {
    static int n_sm = 0;
    if (n_sm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (n_sm <= 0) n_sm = 1;
    }
    return n_sm;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

bool make_map(CUtensorMap* m, float* base, long long rows, int kp, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 4};
    cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

struct Plan {
    bool ok = false;
    bool swapped = false;
    bool p_bcast = false, q_bcast = false;   // operand identical in every batch: packed once
    int Rp_rows = 0, Rq_rows = 0;    // complex rows of P and Q
    int Pp = 0, Qp = 0, Kp = 0;      // padded real rows / K'
    long long batches = 0;
    int nsplit = 1, cps = 0;         // split-K: K ranges per tile, chunks per range
    size_t w_off = 0;                // byte offset of the partial results
    size_t bytes = 0;
};

// Split-K: the number of K ranges that minimises the modelled makespan,
// waves x (chunks per range + SPLIT_EPI_CHUNKS), where a wave is one work
// item per SM and SPLIT_EPI_CHUNKS charges each work item's epilogue in
// units of chunks; ranges have at least SPLIT_MIN_CHUNKS chunks.  A split
// must beat the unsplit plan by 3% to be taken.
constexpr int SPLIT_MIN_CHUNKS = 4;
constexpr int SPLIT_EPI_CHUNKS = 4;

Plan plan_for(const GemmArgs& g, int max_split) {
    Plan pl;
    long long K = (long long)g.Ki * g.Ko;
    if (g.M <= 0 || g.N <= 0 || K < 16) return pl;
    if (std::min(g.M, g.N) < 16 || std::max(g.M, g.N) < 64) return pl;
    // P: one real row per complex row; Q: the real embedding (two real rows
    // per complex row).  The doubled side is the one whose packed bytes cost
    // less -- rows times the batches it is packed for (1 if all batches share
    // it) -- and on a tie the smaller side.
    pl.batches = (long long)g.Bi * g.Bo;
    const bool a_b = (g.a_bi == 0 || g.Bi == 1) && (g.a_bo == 0 || g.Bo == 1);
    const bool b_b = (g.b_bi == 0 || g.Bi == 1) && (g.b_bo == 0 || g.Bo == 1);
    const long long ra = (long long)g.M * (a_b ? 1 : pl.batches), rb = (long long)g.N * (b_b ? 1 : pl.batches);
    const long long cost_a_p = ra + 2 * rb, cost_b_p = rb + 2 * ra;   // P = A side / P = B side
    pl.swapped = cost_b_p < cost_a_p || (cost_b_p == cost_a_p && g.N > g.M);
    pl.Rp_rows = pl.swapped ? g.N : g.M;
    pl.Rq_rows = pl.swapped ? g.M : g.N;
    pl.Pp = (int)round_up(pl.Rp_rows, BM);
    pl.Qp = (int)round_up(2LL * pl.Rq_rows, BN);
    pl.Kp = (int)round_up(2 * K, BK);
    if (pl.batches > 65535 || pl.Qp / BN > 65535) return pl;
    pl.p_bcast = pl.swapped ? b_b : a_b;
    pl.q_bcast = pl.swapped ? a_b : b_b;
    size_t pe = (size_t)(pl.p_bcast ? 1 : pl.batches) * pl.Pp * pl.Kp;
    size_t qe = (size_t)(pl.q_bcast ? 1 : pl.batches) * pl.Qp * pl.Kp;
    pl.bytes = 2 * (pe + qe) * sizeof(float) + 256;
    const int nchunk = (pl.Kp / BK + CHUNK_KB - 1) / CHUNK_KB;
    const long long tiles = (long long)(pl.Pp / BM) * (pl.Qp / BN) * pl.batches;
    int ns = 1;
    if (max_split > 1) {
        const long long sms = num_sms();
        auto cost = [&](int n) {
            const int c = (nchunk + n - 1) / n, k = (nchunk + c - 1) / c;
            return (double)((tiles * k + sms - 1) / sms) * (c + SPLIT_EPI_CHUNKS);
        };
        double best = 0.97 * cost(1);
        const int lim = std::min(std::min(max_split, nchunk / SPLIT_MIN_CHUNKS), 256);
        for (int n = 2; n <= lim; ++n)
            if (cost(n) < best) {
                best = cost(n);
                ns = n;
            }
    }
    if (ns > 1) {
        pl.cps = (nchunk + ns - 1) / ns;
        pl.nsplit = (nchunk + pl.cps - 1) / pl.cps;
    }
    if (pl.nsplit > 1) {
        pl.w_off = (pl.bytes + 255) / 256 * 256;
        pl.bytes = pl.w_off + (size_t)pl.nsplit * pl.batches * g.M * (size_t)g.N * sizeof(cplx);
    } else {
        pl.cps = nchunk;
    }
    pl.ok = true;
    return pl;
}

}  // namespace

size_t split_workspace_bytes(const GemmArgs& g, int max_split) {
    Plan pl = plan_for(g, max_split);
    return pl.ok ? pl.bytes : 0;
}

// Phase 1 of a split contraction: pack both operands.  Returns kernels
// launched, -1 if the shape is not handled here (caller uses FP64), -2 if the
// workspace is too small.
int launch_split_pack(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes,
                      int max_split) {
    Plan pl = plan_for(g, max_split);
    if (!pl.ok || !encode_fn()) return -1;
    if (!workspace || workspace_bytes < pl.bytes) return -2;
    const long long np_b = pl.p_bcast ? 1 : pl.batches, nq_b = pl.q_bcast ? 1 : pl.batches;
    size_t pe = (size_t)np_b * pl.Pp * pl.Kp, qe = (size_t)nq_b * pl.Qp * pl.Kp;
    float* Ph = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(workspace) + 256);
    float* Pl = Ph + pe;
    float* Qh = Pl + pe;
    float* Ql = Qh + qe;
    // A side as (row m, k) and B side as (row n, k)
    PackArgs pa, pb;
    std::memset(&pa, 0, sizeof(pa));
    std::memset(&pb, 0, sizeof(pb));
    pa.src = g.A; pa.s_r = g.a_m; pa.s_ki = g.a_ki; pa.s_ko = g.a_ko; pa.s_bi = g.a_bi; pa.s_bo = g.a_bo;
    pa.R = g.M; pa.conj = g.conjA;
    pb.src = g.B; pb.s_r = g.b_n; pb.s_ki = g.b_ki; pb.s_ko = g.b_ko; pb.s_bi = g.b_bi; pb.s_bo = g.b_bo;
    pb.R = g.N; pb.conj = g.conjB;
    for (PackArgs* p : {&pa, &pb}) {
        p->Ki = g.Ki; p->Ko = g.Ko; p->Bi = g.Bi; p->Bo = g.Bo; p->Kp = pl.Kp;
    }
    PackArgs& P = pl.swapped ? pb : pa;
    PackArgs& Q = pl.swapped ? pa : pb;
    P.embed = 0; P.Rp = pl.Pp; P.hi = Ph; P.lo = Pl;
    Q.embed = 1; Q.Rp = pl.Qp; Q.hi = Qh; Q.lo = Ql;
    if (pl.p_bcast) { P.Bi = 1; P.Bo = 1; }
    if (pl.q_bcast) { Q.Bi = 1; Q.Bo = 1; }
    int launches = 0;
    for (PackArgs* p : {&P, &Q}) {
        long long total = (long long)(p->embed ? p->Rp / 2 : p->Rp) * (p->Kp / 2) * p->Bi * p->Bo;
        long long grid = std::min<long long>((total + 255) / 256, 152LL * 16);
        pack_kernel<<<(unsigned)grid, 256, 0, stream>>>(*p);
        ++launches;
    }
    return launches;
}

// Phase 2: the tcgen05 GEMM on the packed operands of the same GemmArgs.
int launch_split_mma(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes,
                     int max_split) {
    Plan pl = plan_for(g, max_split);
    if (!pl.ok || !workspace || workspace_bytes < pl.bytes) return -1;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr_set = true;
    }
    const long long pb = pl.p_bcast ? 1 : pl.batches, qb = pl.q_bcast ? 1 : pl.batches;
    size_t pe = (size_t)pb * pl.Pp * pl.Kp, qe = (size_t)qb * pl.Qp * pl.Kp;
    int* err = reinterpret_cast<int*>(workspace);          // first 256 bytes: error flag
    float* Ph = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(workspace) + 256);
    float* Pl = Ph + pe;
    float* Qh = Pl + pe;
    float* Ql = Qh + qe;
    CUtensorMap mPh, mPl, mQh, mQl;
    if (!make_map(&mPh, Ph, pb * pl.Pp, pl.Kp, BM) || !make_map(&mPl, Pl, pb * pl.Pp, pl.Kp, BM) ||
        !make_map(&mQh, Qh, qb * pl.Qp, pl.Kp, BN) || !make_map(&mQl, Ql, qb * pl.Qp, pl.Kp, BN))
        return -1;
    EpiArgs ea;
    ea.C = g.C; ea.c_m = g.c_m; ea.c_n = g.c_n; ea.c_bi = g.c_bi; ea.c_bo = g.c_bo;
    ea.M = g.M; ea.N = g.N; ea.Bi = g.Bi;
    ea.swapped = pl.swapped;
    ea.Pp = pl.p_bcast ? 0 : pl.Pp;   // batch stride of the packed rows (0: shared)
    ea.Qp = pl.q_bcast ? 0 : pl.Qp;
    ea.nkb = pl.Kp / BK;
    ea.alpha = g.alpha; ea.beta = g.beta;
    const bool a1 = g.alpha.x == 1.0 && g.alpha.y == 0.0;
    ea.mode = (a1 && g.beta.x == 0.0 && g.beta.y == 0.0) ? 0 : (a1 && g.beta.x == 1.0 && g.beta.y == 0.0) ? 1 : 2;
    ea.err = err;
    ea.nsplit = pl.nsplit;
    ea.cps = pl.cps;
    ea.W = pl.nsplit > 1 ? reinterpret_cast<cplx*>(reinterpret_cast<uint8_t*>(workspace) + pl.w_off) : nullptr;
    // persistent: one CTA per SM walks the tiles, the smaller tile count
    // fastest so that CTAs sharing the other operand's tile run together and
    // hit it in L2 (an operand larger than L2 is then read about once)
    ea.n_ptiles = pl.Pp / BM;
    ea.n_qtiles = pl.Qp / BN;
    ea.q_fast = ea.n_qtiles < ea.n_ptiles;
    ea.batches = (int)pl.batches;
    long long ntiles = (long long)ea.n_ptiles * ea.n_qtiles * pl.batches * pl.nsplit;
    unsigned grid = (unsigned)std::min<long long>(ntiles, num_sms());
    tc_gemm_kernel<<<grid, GEMM_THREADS, SMEM_BYTES, stream>>>(mPh, mPl, mQh, mQl, ea);
    if (pl.nsplit == 1) return 1;
    long long total = (long long)g.M * g.N * pl.batches;
    unsigned rg = (unsigned)std::min<long long>((total + 255) / 256, (long long)num_sms() * 8);
    splitk_reduce_kernel<<<rg, 256, 0, stream>>>(ea);
    return 2;
}

int launch_zgemm_split(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    int a = launch_split_pack(g, stream, workspace, workspace_bytes);
    if (a < 0) return a;
    int b = launch_split_mma(g, stream, workspace, workspace_bytes);
    return b < 0 ? -1 : a + b;
}
