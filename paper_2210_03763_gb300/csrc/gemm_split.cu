// Split-precision complex contraction on the 5th-generation tensor cores
// (tcgen05, kind::tf32), "3xTF32": every FP64 operand x is split into
// hi = tf32(x) and lo = tf32(x - hi); the product is hi*hi + hi*lo + lo*hi with
// FP32 accumulation in tensor memory (the lo*lo term, ~2^-22 relative, is
// dropped).  Result accuracy is close to FP32 (about 1e-7 relative).
//
// Complex numbers use a real embedding.  The side with fewer rows ("P", R x K)
// becomes 2R x 2K real rows, the other side ("Q", N x K) N x 2K, with the K
// axis interleaved as k' = 2k + half:
//   P row 2r   : ( Re p, -Im p )      Q row n : ( Re q, Im q )
//   P row 2r+1 : ( Im p,  Re p )
// so  C~(2r, n) = Re(sum_k p q) and C~(2r+1, n) = Im(sum_k p q).
//
// Two kernels per contraction:
//  1. pack_kernel: gathers the strided FP64 operand (any GemmArgs strides,
//     optional conjugation, batches) into zero-padded K-major FP32 hi/lo
//     planes; HBM bound, coalesced float2 stores.
//  2. tcgen05 GEMM: one 128 x 64 tile of C~ per CTA, 6 warps.  Warp 4 issues
//     TMA loads (128-byte swizzle, no multicast) into a 4-stage ring, warp 5
//     issues 12 tcgen05.mma per 32-wide K slice into one of two TMEM
//     accumulators and releases stages with tcgen05.commit; warps 0-3 drain
//     finished K chunks from TMEM (tcgen05.ld 32x32b) into float-float sums
//     and finally write alpha * C~ + beta * C in FP64.
//  Every mbarrier wait is bounded; on timeout the kernel sets an error flag,
//  skips the rest, frees its TMEM and returns.
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
constexpr long long SPIN_LIMIT = 1LL << 24;

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

// Bounded wait: false (and the error flag set) if the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    for (long long i = 0; i < SPIN_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
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

// Round a float to TF32 (10 explicit mantissa bits), to nearest, ties to even.
__device__ __forceinline__ float tf32_rn(float f) {
    uint32_t b = __float_as_uint(f);
    if ((b & 0x7F800000u) == 0x7F800000u) return f;   // inf / nan unchanged
    b += 0xFFFu + ((b >> 13) & 1u);
    b &= 0xFFFFE000u;
    return __uint_as_float(b);
}

// ----------------------------------------------------------------- packing
struct PackArgs {
    const cplx* src;
    long long s_r, s_ki, s_ko, s_bi, s_bo;   // strides of (row, k_in, k_out, batch_in, batch_out)
    int R, Ki, Ko, Bi, Bo;
    int conj;
    int embed;         // 1: P side (2 rows per complex row), 0: Q side
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
            im = p.conj ? -v.y : v.y;
        }
        float rh = tf32_rn((float)re), ih = tf32_rn((float)im);
        float rl = tf32_rn((float)(re - (double)rh)), il = tf32_rn((float)(im - (double)ih));
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
// two TMEM buffers and restarts the next chunk in the other buffer, while
// four drain warps add each finished chunk into float-float register sums
// (Knuth TwoSum, ~2^-48 relative).  The error is then that of one short
// chunk (~3e-7 relative), independent of K.
constexpr int CHUNK_KB = 2;
constexpr int DRAIN_THREADS = 128;                 // warps 0-3: TMEM lanes 0-127
constexpr int GEMM_THREADS = DRAIN_THREADS + 64;   // warp 4: TMA, warp 5: MMA

struct EpiArgs {
    cplx* C;
    long long c_m, c_n, c_bi, c_bo;
    int M, N, Bi;
    int swapped;          // P side holds the columns n of C (C^T computed)
    int Pp, Qp;           // padded real rows per batch of P and Q
    int nkb;              // K' / BK
    cplx alpha, beta;
    int* err;
};

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
    uint64_t* tfull = empty + STAGES;      // [2] chunk accumulated in TMEM buffer b
    uint64_t* tempty = tfull + 2;          // [2] buffer b drained
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.z;
    const int prow0 = b * ea.Pp + blockIdx.x * BM;   // P rows of this tile (packed buffer rows)
    const int qrow0 = b * ea.Qp + blockIdx.y * BN;
    const int nchunk = (ea.nkb + CHUNK_KB - 1) / CHUNK_KB;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], DRAIN_THREADS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 4) {
        if (lane == 0) {   // TMA producer
            for (int kb = 0; kb < ea.nkb; ++kb) {
                int s = kb % STAGES, round = kb / STAGES;
                if (kb >= STAGES && !mbar_wait(&empty[s], (round - 1) & 1, ea.err)) break;
                uint8_t* st = smem + s * STAGE_BYTES;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                tma_load_2d(st, &mPh, &full[s], kb * BK, prow0);
                tma_load_2d(st + A_TILE, &mPl, &full[s], kb * BK, prow0);
                tma_load_2d(st + 2 * A_TILE, &mQh, &full[s], kb * BK, qrow0);
                tma_load_2d(st + 2 * A_TILE + B_TILE, &mQl, &full[s], kb * BK, qrow0);
            }
        }
        __syncwarp();
    } else if (warp == 5) {
        if (lane == 0) {   // MMA issuer
            bool ok = true;
            for (int c = 0; c < nchunk && ok; ++c) {
                const int buf = c & 1;
                const uint32_t dt = tmem + (uint32_t)(buf * BN);
                if (c >= 2 && !mbar_wait(&tempty[buf], ((c >> 1) - 1) & 1, ea.err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int kb_end = min(ea.nkb, (c + 1) * CHUNK_KB);
                for (int kb = c * CHUNK_KB; kb < kb_end; ++kb) {
                    int s = kb % STAGES, round = kb / STAGES;
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
        __syncwarp();
    } else {
        // drain warps 0-3: thread = TMEM lane = tile row
        float hi[BN], lo[BN];
#pragma unroll
        for (int j = 0; j < BN; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
        bool ok = true;
        for (int c = 0; c < nchunk; ++c) {
            const int buf = c & 1;
            if (!mbar_wait(&tfull[buf], (c >> 1) & 1, ea.err)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int c0 = 0; c0 < BN; c0 += 16) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * BN + c0), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) two_sum_acc(hi[c0 + j], lo[c0 + j], v[j]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tempty[buf])) : "memory");
        }
        if (ok) {
            const int trow = warp * 32 + lane;                  // row of C~ inside the tile
            const int prow = blockIdx.x * BM + trow;            // P real row within the batch
            const int pr = prow >> 1;                           // complex row of P
            const int bi = b % ea.Bi, bo = b / ea.Bi;
            cplx* C = ea.C + bi * ea.c_bi + bo * ea.c_bo;
            const bool beta0 = (ea.beta.x == 0.0 && ea.beta.y == 0.0);
#pragma unroll
            for (int j = 0; j < BN; ++j) {
                double val = (double)hi[j] + (double)lo[j];
                double other = __shfl_xor_sync(0xffffffffu, val, 1);
                if (lane & 1) continue;
                int qn = blockIdx.y * BN + j;                   // Q row = the other index
                int m = ea.swapped ? qn : pr;
                int n = ea.swapped ? pr : qn;
                if (m >= ea.M || n >= ea.N) continue;
                double re = val, im = other;
                cplx* cp = C + m * ea.c_m + n * ea.c_n;
                cplx r;
                r.x = ea.alpha.x * re - ea.alpha.y * im;
                r.y = ea.alpha.x * im + ea.alpha.y * re;
                if (!beta0) {
                    cplx o = *cp;
                    r.x += ea.beta.x * o.x - ea.beta.y * o.y;
                    r.y += ea.beta.x * o.y + ea.beta.y * o.x;
                }
                *cp = r;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
    }
}

// ------------------------------------------------------------------- host
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
    int Rp_rows = 0, Rq_rows = 0;    // complex rows of P and Q
    int Pp = 0, Qp = 0, Kp = 0;      // padded real rows / K'
    long long batches = 0;
    size_t bytes = 0;
};

Plan plan_for(const GemmArgs& g) {
    Plan pl;
    long long K = (long long)g.Ki * g.Ko;
    if (g.M <= 0 || g.N <= 0 || K < 16) return pl;
    if (std::min(g.M, g.N) < 16 || std::max(g.M, g.N) < 64) return pl;
    pl.swapped = g.M > g.N;
    pl.Rp_rows = pl.swapped ? g.N : g.M;
    pl.Rq_rows = pl.swapped ? g.M : g.N;
    pl.Pp = (int)round_up(2LL * pl.Rp_rows, BM);
    pl.Qp = (int)round_up(pl.Rq_rows, BN);
    pl.Kp = (int)round_up(2 * K, BK);
    pl.batches = (long long)g.Bi * g.Bo;
    if (pl.batches > 65535 || pl.Qp / BN > 65535) return pl;
    size_t pe = (size_t)pl.batches * pl.Pp * pl.Kp, qe = (size_t)pl.batches * pl.Qp * pl.Kp;
    pl.bytes = 2 * (pe + qe) * sizeof(float) + 256;
    pl.ok = true;
    return pl;
}

}  // namespace

size_t split_workspace_bytes(const GemmArgs& g) {
    Plan pl = plan_for(g);
    return pl.ok ? pl.bytes : 0;
}

// Phase 1 of a split contraction: pack both operands.  Returns kernels
// launched, -1 if the shape is not handled here (caller uses FP64), -2 if the
// workspace is too small.
int launch_split_pack(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    Plan pl = plan_for(g);
    if (!pl.ok || !encode_fn()) return -1;
    if (!workspace || workspace_bytes < pl.bytes) return -2;
    size_t pe = (size_t)pl.batches * pl.Pp * pl.Kp, qe = (size_t)pl.batches * pl.Qp * pl.Kp;
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
    P.embed = 1; P.Rp = pl.Pp; P.hi = Ph; P.lo = Pl;
    Q.embed = 0; Q.Rp = pl.Qp; Q.hi = Qh; Q.lo = Ql;
    int launches = 0;
    for (PackArgs* p : {&P, &Q}) {
        long long total = (long long)(p->embed ? p->Rp / 2 : p->Rp) * (p->Kp / 2) * pl.batches;
        long long grid = std::min<long long>((total + 255) / 256, 152LL * 16);
        pack_kernel<<<(unsigned)grid, 256, 0, stream>>>(*p);
        ++launches;
    }
    return launches;
}

// Phase 2: the tcgen05 GEMM on the packed operands of the same GemmArgs.
int launch_split_mma(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    Plan pl = plan_for(g);
    if (!pl.ok || !workspace || workspace_bytes < pl.bytes) return -1;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        attr_set = true;
    }
    size_t pe = (size_t)pl.batches * pl.Pp * pl.Kp, qe = (size_t)pl.batches * pl.Qp * pl.Kp;
    int* err = reinterpret_cast<int*>(workspace);          // first 256 bytes: error flag
    float* Ph = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(workspace) + 256);
    float* Pl = Ph + pe;
    float* Qh = Pl + pe;
    float* Ql = Qh + qe;
    CUtensorMap mPh, mPl, mQh, mQl;
    if (!make_map(&mPh, Ph, pl.batches * pl.Pp, pl.Kp, BM) || !make_map(&mPl, Pl, pl.batches * pl.Pp, pl.Kp, BM) ||
        !make_map(&mQh, Qh, pl.batches * pl.Qp, pl.Kp, BN) || !make_map(&mQl, Ql, pl.batches * pl.Qp, pl.Kp, BN))
        return -1;
    EpiArgs ea;
    ea.C = g.C; ea.c_m = g.c_m; ea.c_n = g.c_n; ea.c_bi = g.c_bi; ea.c_bo = g.c_bo;
    ea.M = g.M; ea.N = g.N; ea.Bi = g.Bi;
    ea.swapped = pl.swapped;
    ea.Pp = pl.Pp; ea.Qp = pl.Qp;
    ea.nkb = pl.Kp / BK;
    ea.alpha = g.alpha; ea.beta = g.beta;
    ea.err = err;
    // P tiles fastest: CTAs sharing a Q tile run together and hit it in L2
    dim3 grid(pl.Pp / BM, pl.Qp / BN, (unsigned)pl.batches);
    tc_gemm_kernel<<<grid, GEMM_THREADS, SMEM_BYTES, stream>>>(mPh, mPl, mQh, mQl, ea);
    return 1;
}

int launch_zgemm_split(const GemmArgs& g, cudaStream_t stream, void* workspace, size_t workspace_bytes) {
    int a = launch_split_pack(g, stream, workspace, workspace_bytes);
    if (a < 0) return a;
    int b = launch_split_mma(g, stream, workspace, workspace_bytes);
    return b < 0 ? -1 : a + b;
}
