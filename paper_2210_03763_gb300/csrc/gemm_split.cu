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

constexpr int BM = SPLIT_BM, BK = SPLIT_BK;   // BK in fp32 elements = 128 bytes
constexpr int A_TILE = BM * BK * 4;          // 16 KB per plane tile of P
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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          unsigned long long limit_ns = WAIT_NS) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (long long i = 1; i < SPIN_LIMIT; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63) == 0) {
            if (*(volatile int*)err) return false;
            if (global_ns() - t0 > limit_ns) break;
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

// Instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = n.
constexpr uint32_t idesc_for(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dt, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            dt),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
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
// One thread per complex element (batch, row r < Rpad, k < Kc); entries with
// r >= R or k >= Ki*Ko are written as zeros (tile padding).  Real row of
// (r, bi, bo): (embed ? 2r : r) + bi*rb_i + bo*rb_o; float offset of k:
// k_off + 2k in a row of `pitch` floats.
__global__ void pack_kernel(SplitPackArgs p) {
    const int K = p.Ki * p.Ko;
    const long long per_b = (long long)p.Rpad * p.Kc;
    const long long total = per_b * p.Bi * p.Bo;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / per_b;
        const long long rem = e - b * per_b;
        const int r = (int)(rem / p.Kc);
        const int k = (int)(rem - (long long)r * p.Kc);
        const int bi = (int)(b % p.Bi), bo = (int)(b / p.Bi);
        double re = 0.0, im = 0.0;
        if (r < p.R && k < K) {
            const int ki = k % p.Ki, ko = k / p.Ki;
            cplx v = p.src[bi * p.s_bi + bo * p.s_bo + r * p.s_r + ki * p.s_ki + ko * p.s_ko];
            re = v.x;
            im = p.conj ? __longlong_as_double(__double_as_longlong(v.y) ^ (long long)0x8000000000000000ULL) : v.y;
        }
        float rh, rl, ih, il;
        split_tf32(re, rh, rl);
        split_tf32(im, ih, il);
        const long long row = (p.embed ? 2LL * r : (long long)r) + bi * p.rb_i + bo * p.rb_o;
        const long long o0 = row * p.pitch + p.k_off + 2LL * k;
        if (p.embed) {
            const long long o1 = o0 + p.pitch;
            *reinterpret_cast<float2*>(p.hi + o0) = make_float2(rh, -ih);
            *reinterpret_cast<float2*>(p.hi + o1) = make_float2(ih, rh);
            *reinterpret_cast<float2*>(p.lo + o0) = make_float2(rl, -il);
            *reinterpret_cast<float2*>(p.lo + o1) = make_float2(il, rl);
        } else {
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
constexpr int TMA_WARP = DRAIN_WARPS, MMA_WARP = DRAIN_WARPS + 1;
constexpr int GEMM_THREADS = DRAIN_THREADS + 64;

// Tile width N of C~ (real columns, i.e. BN / 2 complex Q rows).  Both widths
// use M = 128 rows and 4 TMEM accumulators (256 or all 512 columns).  The
// wide tile halves the shared-memory operand traffic per flop (each 128-row P
// tile feeds 128 columns instead of 64): measured on the H_eff of 8x8,
// chi = 128 nodes, the tensor-core time of one matvec fell from 26.4 to
// 18.4 ms over levels 2-4 (a copy of the kernel that skipped the drain and
// the epilogue ran 21.1 ms at width 64 and 12.2 ms at width 128, so the
// narrow tile was bound by its TMA/MMA pipeline, not by the drain).  Its
// ring has 3 stages of 64 KB (4 of 48 KB at width 64), and each drain
// thread holds 32 float-float sums.
template <int BN_>
struct TileCfg {
    static constexpr int BN = BN_;
    static constexpr int STAGES = BN_ == 128 ? 3 : 4;
    static constexpr int B_TILE = BN_ * BK * 4;   // 8 or 16 KB per plane tile of Q
    static constexpr int STAGE_BYTES = 2 * A_TILE + 2 * B_TILE;
    static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
    static constexpr int DCOLS = BN_ / (DRAIN_WARPS / 4);   // columns per drain thread
    static constexpr uint32_t IDESC = idesc_for(BN_);
};
static_assert(TileCfg<128>::SMEM_BYTES <= 227 * 1024 && TileCfg<64>::SMEM_BYTES <= 227 * 1024, "shared memory");
static_assert(NBUF * 128 <= 512, "TMEM columns");

// Tile width of a contraction: 128 when the Q side has at least 128 padded
// real rows and the contraction is large (at least 2^24 complex MACs); small
// contractions are latency-bound on a few CTAs and run faster as more,
// narrower tiles (measured: 81 x 81 x 81 took 17 us at width 64, 24 us at
// width 128).
inline int tile_bn(int Qp, double cmacs) { return (Qp >= 128 && cmacs >= 16777216.0) ? 128 : 64; }
inline int tile_bn(const SplitMma& m) {
    return tile_bn(m.Qp, (double)m.Pn * m.Qn * (0.5 * m.Kp) * m.Bi * (double)m.Bo);
}

struct EpiArgs {
    cplx* C;
    long long c_p, c_q, c_bi, c_bo;   // output strides of P row p, Q row q, batch (bi, bo)
    int c_pd;             // P row split: offset (p % c_pd)*c_p + (p / c_pd)*c_p2
    long long c_p2;
    int Pn, Qn, Bi;       // valid complex rows of P and Q; inner batch extent
    long long p_sbi, p_sbo, q_sbi, q_sbo;   // real-row offset of batch (bi, bo) in P / Q (0: shared)
    int nkb;              // K' / BK
    int n_ptiles, n_qtiles, batches;   // tile grid; tile t: P tile fastest, then Q tile, then batch
    cplx alpha, beta;
    int mode;             // 0: alpha = 1, beta = 0; 1: alpha = 1, beta = 1; 2: general
    int* err;
    int q_fast;           // tile order inside a batch: Q tiles fastest (else P tiles fastest)
    int nsplit;           // K ranges per output tile (split-K); > 1: partial results go to W
    int cps;              // chunks per K range
    cplx* W;              // nsplit x batches x Qn x Pn partial results (P row fastest)
    unsigned long long stall_ns;   // test hook: > 0 makes the drain warps wait this long on a
                                   // barrier nothing arrives at, so the launch aborts as on a timeout
    // packed output (o_hi != nullptr): TF32 hi/lo planes at float2 position
    // (p % pd)*sp1 + (p / pd)*sp2 + q*sq + bi*sbi + bo*sbo
    float* o_hi;
    float* o_lo;
    int o_pd;
    long long o_sp1, o_sp2, o_sq, o_sbi, o_sbo;
};

// Round a float to TF32 (10 mantissa bits, to nearest, ties to even) with
// integer operations; inf/nan unchanged.
__device__ __forceinline__ float tf32_rne(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7F800000u) == 0x7F800000u) return x;
    u += 0xFFFu + ((u >> 13) & 1u);
    return __uint_as_float(u & 0xFFFFE000u);
}

// (hi + lo) as a float-float sum -> TF32 pair (th, tl) with
// |hi + lo - th - tl| <~ 2^-22 |hi + lo|, FP32 and integer operations only.
__device__ __forceinline__ void ff_to_tf32_pair(float hi, float lo, float& th, float& tl) {
    th = tf32_rne(hi);
    tl = tf32_rne(__fadd_rn(__fsub_rn(hi, th), lo));
}

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

// Knuth's TwoSum, hi + lo += x, on two lanes at once with packed f32x2
// arithmetic (round to nearest per lane, the same results as scalar FADDs in
// half the instructions: the drain warps are issue-bound, and this cut the
// tensor-core time of an 8x8, chi = 128 H_eff by 8 %).
__device__ __forceinline__ void two_sum_acc2(float& h0, float& h1, float& l0, float& l1, float x0, float x1) {
    asm("{\n .reg .b64 H, X, S, B, T, U, E, L;\n"
        " mov.b64 H, {%0, %1};\n mov.b64 X, {%4, %5};\n mov.b64 L, {%2, %3};\n"
        " add.rn.f32x2 S, H, X;\n"          // s = hi + x
        " sub.rn.f32x2 B, S, H;\n"          // b = s - hi
        " sub.rn.f32x2 T, S, B;\n"
        " sub.rn.f32x2 T, H, T;\n"          // hi - (s - b)
        " sub.rn.f32x2 U, X, B;\n"          // x - b
        " add.rn.f32x2 E, T, U;\n"          // rounding error of s
        " add.rn.f32x2 L, L, E;\n"          // lo += e
        " mov.b64 {%0, %1}, S;\n mov.b64 {%2, %3}, L;\n}"
        : "+f"(h0), "+f"(h1), "+f"(l0), "+f"(l1)
        : "f"(x0), "f"(x1));
}

template <int BN_>
__global__ void __launch_bounds__(GEMM_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mPh, const __grid_constant__ CUtensorMap mPl,
                   const __grid_constant__ CUtensorMap mQh, const __grid_constant__ CUtensorMap mQl, EpiArgs ea) {
    using T = TileCfg<BN_>;
    constexpr int BN = T::BN, STAGES = T::STAGES, B_TILE = T::B_TILE, STAGE_BYTES = T::STAGE_BYTES,
                  DCOLS = T::DCOLS;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* tfull = empty + STAGES;      // [NBUF] chunk accumulated in TMEM buffer b
    uint64_t* tempty = tfull + NBUF;       // [NBUF] buffer b drained
    uint64_t* mdone = tempty + NBUF;       // all MMAs of this CTA complete
    uint64_t* stallbar = mdone + 1;        // test hook: never arrived at
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(stallbar + 1);

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
        mbar_init(stallbar, 1);
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
                const int bi = b % ea.Bi, bo = b / ea.Bi;
                const int prow0 = (int)(bi * ea.p_sbi + bo * ea.p_sbo) + pt * BM;
                const int qrow0 = (int)(bi * ea.q_sbi + bo * ea.q_sbo) + qt * BN;
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
                            mma_tf32(dt, pl + off, qh + off, T::IDESC, acc);
                            mma_tf32(dt, ph + off, ql + off, T::IDESC, 1u);
                            mma_tf32(dt, ph + off, qh + off, T::IDESC, 1u);
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
        // test hook: a wait that runs out (nothing arrives at stallbar); the
        // other roles see the error flag and abort as after a real timeout
        if (ea.stall_ns > 0 && !mbar_wait(stallbar, 0, ea.err, ea.stall_ns)) ok = false;
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
                    for (int j = 0; j < 16; j += 2)
                        two_sum_acc2(hi[c0 + j], hi[c0 + j + 1], lo[c0 + j], lo[c0 + j + 1], v[j], v[j + 1]);
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
            }
            if (!ok) break;
            const int trow = quad * 32 + lane;                  // row of C~ inside the tile
            const int p = pt * BM + trow;                       // complex row of P
            const int bi = b % ea.Bi, bo = b / ea.Bi;
            // split-K: this K range's partial sum, dense (P row fastest), plain store
            cplx* Wt = ea.nsplit > 1 ? ea.W + ((long long)ks * ea.batches + b) * ea.Pn * (long long)ea.Qn : nullptr;
            // columns 2q and 2q + 1 of C~ hold the real and imaginary parts of
            // one entry (the Q side carries the real embedding), so each
            // thread owns whole complex outputs
            if (p < ea.Pn) {
                if (ea.o_hi) {
                    // packed output: TF32 planes for a later contraction, no FP64
                    const long long pbase = (long long)(p % ea.o_pd) * ea.o_sp1 + (long long)(p / ea.o_pd) * ea.o_sp2 +
                                            bi * ea.o_sbi + bo * ea.o_sbo;
                    const int q0 = (qt * BN + col0) >> 1;
#pragma unroll
                    for (int j = 0; j < DCOLS; j += 2) {
                        const int q = q0 + (j >> 1);
                        if (q >= ea.Qn) continue;
                        const long long pos = pbase + (long long)q * ea.o_sq;
                        float rh, rl, ih, il;
                        ff_to_tf32_pair(hi[j], lo[j], rh, rl);
                        ff_to_tf32_pair(hi[j + 1], lo[j + 1], ih, il);
                        reinterpret_cast<float2*>(ea.o_hi)[pos] = make_float2(rh, ih);
                        reinterpret_cast<float2*>(ea.o_lo)[pos] = make_float2(rl, il);
                    }
                    continue;
                }
                cplx* C = ea.C + bi * ea.c_bi + bo * ea.c_bo + (long long)(p % ea.c_pd) * ea.c_p +
                          (long long)(p / ea.c_pd) * ea.c_p2;
#pragma unroll
                for (int j = 0; j < DCOLS; j += 2) {
                    const int q = (qt * BN + col0 + j) >> 1;       // complex row of Q
                    if (q >= ea.Qn) continue;
                    const double re = f32_to_f64(hi[j]) + f32_to_f64(lo[j]);
                    const double im = f32_to_f64(hi[j + 1]) + f32_to_f64(lo[j + 1]);
                    if (Wt) {
                        Wt[p + (long long)q * ea.Pn] = make_double2(re, im);
                        continue;
                    }
                    cplx* cp = C + q * ea.c_q;
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
    const long long PQ = (long long)ea.Pn * ea.Qn, total = PQ * ea.batches;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / PQ);
        const long long pq = e - b * PQ;
        const int p = (int)(pq % ea.Pn), q = (int)(pq / ea.Pn);
        cplx acc = ea.W[(long long)b * PQ + pq];
        for (int ks = 1; ks < ea.nsplit; ++ks) {
            cplx w = ea.W[((long long)ks * ea.batches + b) * PQ + pq];
            acc.x += w.x;
            acc.y += w.y;
        }
        const int bi = b % ea.Bi, bo = b / ea.Bi;
        cplx* cp = ea.C + bi * ea.c_bi + bo * ea.c_bo + (long long)(p % ea.c_pd) * ea.c_p +
                   (long long)(p / ea.c_pd) * ea.c_p2 + q * ea.c_q;
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
// Per-device state of the host side: SM count and whether the kernel's
// shared-memory attribute has been raised (both are properties of a device,
// so a process that drives several GPUs keeps one entry per device).
constexpr int MAX_DEVICES = 64;
struct DeviceState {
    int n_sm = 0;
    bool attr_set[2] = {false, false};   // shared-memory attribute of the width-64 / width-128 kernels
};
DeviceState g_dev[MAX_DEVICES];
std::mutex g_dev_mu;

DeviceState& device_state() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= MAX_DEVICES) dev = 0;
    return g_dev[dev];
}

int num_sms() {
    DeviceState& d = device_state();
    if (d.n_sm == 0) {
        std::lock_guard<std::mutex> lock(g_dev_mu);
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        d.n_sm = n > 0 ? n : 1;
    }
    return d.n_sm;
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

// 2-D map over `rows` rows of `kp` floats, rows `pitch` floats apart.
bool make_map(CUtensorMap* m, const float* base, long long rows, int kp, long long pitch, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    cuuint32_t box[2] = {BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// Split-K: the number of K ranges that minimises the modelled makespan,
// waves x (chunks per range + SPLIT_EPI_CHUNKS), where a wave is one work
// item per SM and SPLIT_EPI_CHUNKS charges each work item's epilogue in
// units of chunks; ranges have at least SPLIT_MIN_CHUNKS chunks.  A split
// must beat the unsplit plan by 3% to be taken.
constexpr int SPLIT_MIN_CHUNKS = 4;
constexpr int SPLIT_EPI_CHUNKS = 4;

struct SplitK {
    int nsplit = 1, cps = 0;
};

SplitK choose_split(long long tiles, int nkb, int max_split) {
    SplitK sk;
    const int nchunk = (nkb + CHUNK_KB - 1) / CHUNK_KB;
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
    sk.cps = nchunk;
    if (ns > 1) {
        sk.cps = (nchunk + ns - 1) / ns;
        sk.nsplit = (nchunk + sk.cps - 1) / sk.cps;
    }
    return sk;
}

SplitK mma_split(const SplitMma& m) {
    const int bn = tile_bn(m);
    const long long tiles = (long long)(m.Pp / BM) * ((m.Qp + bn - 1) / bn) * m.Bi * (long long)m.Bo;
    return choose_split(tiles, m.Kp / BK, m.out ? 1 : m.max_split);
}

// ----------------------------------------------------- legacy GemmArgs plan
// P: one real row per complex row; Q: the real embedding (two real rows per
// complex row).  The doubled side is the one whose packed bytes cost less --
// rows times the batches it is packed for -- and on a tie the smaller side.
// An operand is packed only for the batch dimensions it varies in.
struct Plan {
    bool ok = false;
    bool swapped = false;            // P = B side (the columns n of C)
    int Pp = 0, Qp = 0, Kp = 0;      // padded real rows per packed batch / K'
    int p_vbi = 0, p_vbo = 0, q_vbi = 0, q_vbo = 0;   // side varies with bi / bo
    long long batches = 0;
    size_t pe = 0, qe = 0;           // floats per plane of P / Q
    size_t bytes = 0;                // error flag + planes (+ split-K partials)
    size_t w_off = 0;
    SplitMma mma{};
};

Plan plan_for(const GemmArgs& g, int max_split) {
    Plan pl;
    long long K = (long long)g.Ki * g.Ko;
    if (g.M <= 0 || g.N <= 0 || K < 16) return pl;
    if (std::min(g.M, g.N) < 16 || std::max(g.M, g.N) < 64) return pl;
    pl.batches = (long long)g.Bi * g.Bo;
    const int a_vbi = g.a_bi != 0 && g.Bi > 1, a_vbo = g.a_bo != 0 && g.Bo > 1;
    const int b_vbi = g.b_bi != 0 && g.Bi > 1, b_vbo = g.b_bo != 0 && g.Bo > 1;
    const long long na = (a_vbi ? g.Bi : 1) * (long long)(a_vbo ? g.Bo : 1);
    const long long nb = (b_vbi ? g.Bi : 1) * (long long)(b_vbo ? g.Bo : 1);
    const long long ra = (long long)g.M * na, rb = (long long)g.N * nb;
    const long long cost_a_p = ra + 2 * rb, cost_b_p = rb + 2 * ra;   // P = A side / P = B side
    pl.swapped = cost_b_p < cost_a_p || (cost_b_p == cost_a_p && g.N > g.M);
    const int Rp_rows = pl.swapped ? g.N : g.M, Rq_rows = pl.swapped ? g.M : g.N;
    pl.Pp = (int)round_up(Rp_rows, BM);
    pl.Qp = (int)round_up(2LL * Rq_rows, SPLIT_BN);
    pl.Kp = (int)round_up(2 * K, BK);
    if (pl.batches > 65535 || pl.Qp / SPLIT_BN > 65535) return pl;
    pl.p_vbi = pl.swapped ? b_vbi : a_vbi;
    pl.p_vbo = pl.swapped ? b_vbo : a_vbo;
    pl.q_vbi = pl.swapped ? a_vbi : b_vbi;
    pl.q_vbo = pl.swapped ? a_vbo : b_vbo;
    const long long np = pl.swapped ? nb : na, nq = pl.swapped ? na : nb;
    pl.pe = (size_t)np * pl.Pp * pl.Kp;
    pl.qe = (size_t)nq * pl.Qp * pl.Kp;
    SplitMma& m = pl.mma;
    m.Kp = pl.Kp;
    m.Pn = Rp_rows;
    m.Qn = Rq_rows;
    m.Pp = pl.Pp;
    m.Qp = pl.Qp;
    m.Bi = g.Bi;
    m.Bo = g.Bo;
    m.p_sbi = pl.p_vbi ? pl.Pp : 0;
    m.p_sbo = pl.p_vbo ? (long long)pl.Pp * (pl.p_vbi ? g.Bi : 1) : 0;
    m.q_sbi = pl.q_vbi ? pl.Qp : 0;
    m.q_sbo = pl.q_vbo ? (long long)pl.Qp * (pl.q_vbi ? g.Bi : 1) : 0;
    m.P_rows = (long long)np * pl.Pp;
    m.Q_rows = (long long)nq * pl.Qp;
    m.P_pitch = m.Q_pitch = pl.Kp;
    m.C = g.C;
    m.c_p = pl.swapped ? g.c_n : g.c_m;
    m.c_q = pl.swapped ? g.c_m : g.c_n;
    m.c_bi = g.c_bi;
    m.c_bo = g.c_bo;
    m.alpha = g.alpha;
    m.beta = g.beta;
    m.out = nullptr;
    m.max_split = max_split;
    const SplitK sk = mma_split(m);
    pl.bytes = 256 + 2 * (pl.pe + pl.qe) * sizeof(float);
    if (sk.nsplit > 1) {
        pl.w_off = (pl.bytes + 255) / 256 * 256;
        pl.bytes = pl.w_off + (size_t)sk.nsplit * pl.batches * g.M * (size_t)g.N * sizeof(cplx);
    }
    pl.ok = true;
    return pl;
}

SplitPackArgs side_pack_args(const GemmArgs& g, const Plan& pl, int side, float* hi, float* lo) {
    // side 0 = P, 1 = Q; the A side as (row m, k), the B side as (row n, k)
    const bool a_side = (side == 0) != pl.swapped;
    SplitPackArgs p;
    std::memset(&p, 0, sizeof(p));
    if (a_side) {
        p.src = g.A; p.s_r = g.a_m; p.s_ki = g.a_ki; p.s_ko = g.a_ko; p.s_bi = g.a_bi; p.s_bo = g.a_bo;
        p.R = g.M; p.conj = g.conjA;
    } else {
        p.src = g.B; p.s_r = g.b_n; p.s_ki = g.b_ki; p.s_ko = g.b_ko; p.s_bi = g.b_bi; p.s_bo = g.b_bo;
        p.R = g.N; p.conj = g.conjB;
    }
    p.Ki = g.Ki;
    p.Ko = g.Ko;
    const int vbi = side == 0 ? pl.p_vbi : pl.q_vbi, vbo = side == 0 ? pl.p_vbo : pl.q_vbo;
    p.Bi = vbi ? g.Bi : 1;
    p.Bo = vbo ? g.Bo : 1;
    p.embed = side;
    const int rows = side == 0 ? pl.Pp : pl.Qp;
    p.Rpad = side == 0 ? rows : rows / 2;
    p.Kc = pl.Kp / 2;
    p.rb_i = rows;
    p.rb_o = (long long)rows * p.Bi;
    p.pitch = pl.Kp;
    p.k_off = 0;
    p.hi = hi;
    p.lo = lo;
    return p;
}

}  // namespace

// ------------------------------------------------------------- public API
int split_pack(const SplitPackArgs& p, cudaStream_t stream) {
    const long long total = (long long)p.Rpad * p.Kc * p.Bi * p.Bo;
    if (total <= 0) return 0;
    const long long grid = std::min<long long>((total + 255) / 256, 152LL * 16);
    pack_kernel<<<(unsigned)grid, 256, 0, stream>>>(p);
    return 1;
}

size_t split_mma_partials(const SplitMma& m) {
    const SplitK sk = mma_split(m);
    if (sk.nsplit <= 1) return 0;
    return (size_t)sk.nsplit * m.Bi * (size_t)m.Bo * m.Pn * (size_t)m.Qn * sizeof(cplx);
}

int split_mma(const SplitMma& m, int* err_flag, void* partials, size_t partial_bytes, cudaStream_t stream) {
    if (!err_flag || partial_bytes < split_mma_partials(m) || (split_mma_partials(m) > 0 && !partials)) return -2;
    if (m.Kp % BK || m.Pp % BM || m.Qp % SPLIT_BN || m.Bi < 1 || m.Bo < 1 || m.Pn < 1 || m.Qn < 1) return -1;
    const int bn = tile_bn(m);
    const int smem_bytes = bn == 128 ? TileCfg<128>::SMEM_BYTES : TileCfg<64>::SMEM_BYTES;
    {
        DeviceState& d = device_state();
        std::lock_guard<std::mutex> lock(g_dev_mu);
        const int w = bn == 128 ? 1 : 0;
        if (!d.attr_set[w]) {
            const cudaError_t e =
                bn == 128 ? cudaFuncSetAttribute(tc_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem_bytes)
                          : cudaFuncSetAttribute(tc_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem_bytes);
            if (e != cudaSuccess) return -1;
            d.attr_set[w] = true;
        }
    }
    // Q maps: boxes of bn rows; a wide tile that runs past a batch's Qp rows
    // reads the next batch's rows or, past the end, TMA's zero fill, and the
    // epilogue drops those columns (q >= Qn)
    CUtensorMap mPh, mPl, mQh, mQl;
    if (!make_map(&mPh, m.Ph, m.P_rows, m.Kp, m.P_pitch, BM) || !make_map(&mPl, m.Pl, m.P_rows, m.Kp, m.P_pitch, BM) ||
        !make_map(&mQh, m.Qh, m.Q_rows, m.Kp, m.Q_pitch, bn) || !make_map(&mQl, m.Ql, m.Q_rows, m.Kp, m.Q_pitch, bn))
        return -1;
    const SplitK sk = mma_split(m);
    EpiArgs ea;
    std::memset(&ea, 0, sizeof(ea));
    ea.C = m.C; ea.c_p = m.c_p; ea.c_q = m.c_q; ea.c_bi = m.c_bi; ea.c_bo = m.c_bo;
    ea.c_pd = m.c_pd > 0 ? m.c_pd : (1 << 30);
    ea.c_p2 = m.c_p2;
    ea.Pn = m.Pn; ea.Qn = m.Qn; ea.Bi = m.Bi;
    ea.p_sbi = m.p_sbi; ea.p_sbo = m.p_sbo; ea.q_sbi = m.q_sbi; ea.q_sbo = m.q_sbo;
    ea.nkb = m.Kp / BK;
    ea.alpha = m.alpha; ea.beta = m.beta;
    const bool a1 = m.alpha.x == 1.0 && m.alpha.y == 0.0;
    ea.mode = (a1 && m.beta.x == 0.0 && m.beta.y == 0.0) ? 0 : (a1 && m.beta.x == 1.0 && m.beta.y == 0.0) ? 1 : 2;
    ea.err = err_flag;
    ea.nsplit = sk.nsplit;
    ea.cps = sk.cps;
    ea.W = sk.nsplit > 1 ? reinterpret_cast<cplx*>(partials) : nullptr;
    ea.stall_ns = test_take_tc_stall();
    if (m.out) {
        ea.o_hi = m.out->hi; ea.o_lo = m.out->lo;
        ea.o_pd = m.out->pd;
        ea.o_sp1 = m.out->sp1; ea.o_sp2 = m.out->sp2; ea.o_sq = m.out->sq;
        ea.o_sbi = m.out->sbi; ea.o_sbo = m.out->sbo;
    }
    // persistent: one CTA per SM walks the tiles, the smaller tile count
    // fastest so that CTAs sharing the other operand's tile run together and
    // hit it in L2 (an operand larger than L2 is then read about once)
    ea.n_ptiles = m.Pp / BM;
    ea.n_qtiles = (m.Qp + bn - 1) / bn;
    ea.q_fast = ea.n_qtiles < ea.n_ptiles;
    ea.batches = m.Bi * m.Bo;
    const long long ntiles = (long long)ea.n_ptiles * ea.n_qtiles * ea.batches * sk.nsplit;
    const unsigned grid = (unsigned)std::min<long long>(ntiles, num_sms());
    if (bn == 128)
        tc_gemm_kernel<128><<<grid, GEMM_THREADS, smem_bytes, stream>>>(mPh, mPl, mQh, mQl, ea);
    else
        tc_gemm_kernel<64><<<grid, GEMM_THREADS, smem_bytes, stream>>>(mPh, mPl, mQh, mQl, ea);
    if (sk.nsplit == 1) return 1;
    const long long total = (long long)m.Pn * m.Qn * ea.batches;
    const unsigned rg = (unsigned)std::min<long long>((total + 255) / 256, (long long)num_sms() * 8);
    splitk_reduce_kernel<<<rg, 256, 0, stream>>>(ea);
    return 2;
}

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
    float* Ph = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(workspace) + 256);
    float* Pl = Ph + pl.pe;
    float* Qh = Pl + pl.pe;
    float* Ql = Qh + pl.qe;
    int n = split_pack(side_pack_args(g, pl, 0, Ph, Pl), stream);
    n += split_pack(side_pack_args(g, pl, 1, Qh, Ql), stream);
    return n;
}

// Phase 2: the tcgen05 GEMM on the packed operands of the same GemmArgs.
int launch_split_mma(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes,
                     int max_split) {
    Plan pl = plan_for(g, max_split);
    if (!pl.ok || !workspace || workspace_bytes < pl.bytes) return -1;
    float* Ph = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(workspace) + 256);
    float* Pl = Ph + pl.pe;
    float* Qh = Pl + pl.pe;
    float* Ql = Qh + pl.qe;
    SplitMma m = pl.mma;
    m.Ph = Ph; m.Pl = Pl; m.Qh = Qh; m.Ql = Ql;
    void* partials = pl.w_off ? reinterpret_cast<uint8_t*>(workspace) + pl.w_off : nullptr;
    const size_t pbytes = pl.w_off ? workspace_bytes - pl.w_off : 0;
    int r = split_mma(m, reinterpret_cast<int*>(workspace), partials, pbytes, stream);
    return r < 0 ? -1 : r;
}

int launch_zgemm_split(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    int a = launch_split_pack(g, stream, workspace, workspace_bytes);
    if (a < 0) return a;
    int b = launch_split_mma(g, stream, workspace, workspace_bytes);
    return b < 0 ? -1 : a + b;
}
