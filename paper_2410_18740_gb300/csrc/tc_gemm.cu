// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
//   D[m][n] = sum_k A[m][k] * B[n][k]      (A: M x K, B: N x K, both K-major bf16)
// accumulated in FP32 in tensor memory and written as FP32 or FP64.
//
// Persistent kernel, one CTA of 6 warps per SM, looping over 128 x 256 output tiles:
//   * warp 0, one lane: TMA producer -- cp.async.bulk.tensor loads of 128 x 64 (A) and
//     256 x 64 (B) tiles with 128-byte swizzle into a 4-stage shared-memory ring, signalled
//     through mbarrier transaction counts; the ring runs on across tiles;
//   * warp 1: owns the 512 TMEM columns (two 256-column FP32 accumulators); one lane issues
//     four tcgen05.mma.kind::f16 (M=128, N=256, K=16) per stage into the tile's accumulator,
//     tcgen05.commit releases the stage and, after the last stage, hands the accumulator to
//     the epilogue;
//   * warps 2-5: epilogue -- tcgen05.ld of their 32 TMEM lanes, conversion, stores, then
//     the accumulator goes back to the MMA warp; the epilogue of one tile overlaps the main
//     loop of the next.
// Every wait is bounded (1 s on %globaltimer); a wait that gives up sets the device status
// word, and the CTA still frees its TMEM and exits.
//
// The split-precision complex products of the solver are plain calls of this kernel on
// operands prepared by tc_pack_* (tc_ops.cu): complex -> real 2x2 block form, FP64 ->
// hi + lo bf16 pairs, three products concatenated along K.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
// longest run of k-blocks summed in one FP32 tensor-memory accumulator (K = 64 * this)
constexpr int MAX_KB_PER_ACC = 256;
constexpr int A_TILE = BM * BK * 2;   // 16 KiB
constexpr int B_TILE = BN * BK * 2;   // 32 KiB
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int TMEM_COLS = 256;
constexpr size_t SMEM_BYTES = 1024 + (size_t)STAGES * STAGE_BYTES + 256;  // + barriers and the TMEM slot
// Split operands (hi | lo halves, see tc_ops.cu): one stage holds the hi and lo tiles of A and B
// for one k-block (twice the bytes, half the stages in the same shared memory) and feeds three
// products hi*hi, hi*lo, lo*hi into the accumulator, so each operand tile is loaded once for the
// two products that use it
constexpr int S3_STAGES = STAGES / 2;
constexpr int S3_STAGE_BYTES = 2 * STAGE_BYTES;

struct TcParams {
    int M, N, K;
    void* D;
    long long ldd;
    int d_fp64;
    int* status;
    int kb_per;           // k-blocks per split
    int splits;           // work item t covers split t / (m tiles * n tiles)
    long long d_split;    // element stride between the per-split outputs (split-K partials)
    int s3;               // split operands: K = 2 * half, hi half then lo half, three products per k-block
    int half;             // columns of one half (multiple of BK)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false (and status set) after 1 s or when another CTA already failed
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = now_ns();
    while (true) {
        if (mbar_test(bar, parity)) return true;
        if (*(volatile int*)status != 0) return false;
        if (now_ns() - t0 > 1000000000ull) {
            atomicExch(status, 1);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);          // start address
    d |= (uint64_t)1 << 16;                          // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                          // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define TC_LD32(taddr, v)                                                                                        \
    asm volatile(                                                                                                \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"  \
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                       \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),        \
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), \
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),             \
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),             \
          "=r"(v[30]), "=r"(v[31])                                                                               \
        : "r"(taddr))

constexpr int TC_THREADS = 192;  // warp 0: TMA, warp 1: MMA + TMEM owner, warps 2-5: epilogue

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Persistent: CTA b takes work items b, b + gridDim.x, ...; item t = (split z, m tile, n tile).
// The shared-memory ring's stage counter runs on across items; the two TMEM accumulators
// alternate between items so that the epilogue of item i overlaps the MMAs of item i + 1.
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                const __grid_constant__ CUtensorMap tmB, TcParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + (size_t)STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;   // [2] MMA -> epilogue
    uint64_t* acc_empty = acc_full + 2;    // [2] epilogue -> MMA
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (p.N + BN - 1) / BN, tiles_m = (p.M + BM - 1) / BM;
    const int items = tiles_n * tiles_m * p.splits;
    const int nkb_total = (p.s3 ? p.half : p.K) / BK;
    const int nst = p.s3 ? S3_STAGES : STAGES;
    const int sbytes = p.s3 ? S3_STAGE_BYTES : STAGE_BYTES;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t g = 0;  // stage counter over all items of this CTA
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x) {
                const int nt = t % tiles_n, mt = (t / tiles_n) % tiles_m, z = t / (tiles_n * tiles_m);
                const int kb0 = z * p.kb_per, nkb = min(nkb_total - kb0, p.kb_per);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % nst;
                    const uint32_t round = g / nst;
                    if (g >= (uint32_t)nst && !(ok = mbar_wait(&empty[s], (round & 1) ^ 1, p.status))) break;
                    uint8_t* a_dst = smem + (size_t)s * sbytes;
                    mbar_expect_tx(&full[s], sbytes);
                    const int x = (kb0 + kb) * BK;
                    if (!p.s3) {
                        tma_load_2d(a_dst, &tmA, &full[s], x, mt * BM);
                        tma_load_2d(a_dst + A_TILE, &tmB, &full[s], x, nt * BN);
                    } else {
                        // A hi, A lo, B hi, B lo
                        tma_load_2d(a_dst, &tmA, &full[s], x, mt * BM);
                        tma_load_2d(a_dst + A_TILE, &tmA, &full[s], p.half + x, mt * BM);
                        tma_load_2d(a_dst + 2 * A_TILE, &tmB, &full[s], x, nt * BN);
                        tma_load_2d(a_dst + 2 * A_TILE + B_TILE, &tmB, &full[s], p.half + x, nt * BN);
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t g = 0;
            int i = 0;  // item counter of this CTA
            for (int t = blockIdx.x; t < items && ok; t += gridDim.x, ++i) {
                const int z = t / (tiles_n * tiles_m);
                const int kb0 = z * p.kb_per, nkb = min(nkb_total - kb0, p.kb_per);
                const int acc = i & 1;
                const uint32_t use = (uint32_t)i >> 1;
                if (use >= 1 && !(ok = mbar_wait(&acc_empty[acc], (use & 1) ^ 1, p.status))) break;
                fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(acc * TMEM_COLS);
                for (int kb = 0; kb < nkb; ++kb, ++g) {
                    const int s = g % nst;
                    const uint32_t round = g / nst;
                    if (!(ok = mbar_wait(&full[s], round & 1, p.status))) break;
                    fence_after();
                    const uint32_t a_addr = smem_u32(smem + (size_t)s * sbytes);
                    if (!p.s3) {
                        const uint32_t b_addr = a_addr + A_TILE;
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k)
                            mma_bf16(d_tmem, smem_desc(a_addr + 32 * k), smem_desc(b_addr + 32 * k),
                                     (kb | k) != 0 ? 1u : 0u);
                    } else {
                        const uint32_t al = a_addr + A_TILE, bh = a_addr + 2 * A_TILE, bl = bh + B_TILE;
#pragma unroll
                        for (int k = 0; k < BK / 16; ++k) {
                            mma_bf16(d_tmem, smem_desc(a_addr + 32 * k), smem_desc(bh + 32 * k), (kb | k) != 0 ? 1u : 0u);
                            mma_bf16(d_tmem, smem_desc(a_addr + 32 * k), smem_desc(bl + 32 * k), 1u);
                            mma_bf16(d_tmem, smem_desc(al + 32 * k), smem_desc(bh + 32 * k), 1u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[acc]);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warp w reads TMEM lanes [32 (w % 4), 32 (w % 4) + 32)
        const int q = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < items; t += gridDim.x, ++i) {
            const int nt = t % tiles_n, mt = (t / tiles_n) % tiles_m, z = t / (tiles_n * tiles_m);
            const int acc = i & 1;
            const uint32_t use = (uint32_t)i >> 1;
            if (!mbar_wait(&acc_full[acc], use & 1, p.status)) {
                ok = false;
                break;
            }
            fence_after();
            const int row = mt * BM + q * 32 + lane;
            const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TMEM_COLS);
            for (int c = 0; c < TMEM_COLS / 32; ++c) {
                uint32_t v[32];
                TC_LD32(lane_addr + c * 32, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < p.M) {
                    const int nbase = nt * BN + c * 32;
                    if (p.d_fp64) {
                        double* out = (double*)p.D + z * p.d_split + (long long)row * p.ldd + nbase;
                        if (nbase + 32 <= p.N && ((uintptr_t)out & 15) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 2)
                                *(double2*)(out + j) =
                                    make_double2((double)__uint_as_float(v[j]), (double)__uint_as_float(v[j + 1]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (nbase + j < p.N) out[j] = (double)__uint_as_float(v[j]);
                        }
                    } else {
                        float* out = (float*)p.D + z * p.d_split + (long long)row * p.ldd + nbase;
                        if (nbase + 32 <= p.N && ((uintptr_t)out & 15) == 0) {
#pragma unroll
                            for (int j = 0; j < 32; j += 4)
                                *(float4*)(out + j) = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                                                  __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
                        } else {
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                if (nbase + j < p.N) out[j] = __uint_as_float(v[j]);
                        }
                    }
                }
            }
            // this warp's lanes of the accumulator may be overwritten now
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[acc]);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS));
    }
}

// out[m][n] = sum_z part[z][m][n] in a fixed order (deterministic split-K reduction), compensated FP32
__global__ void splitk_reduce(const float* __restrict__ part, int splits, int M, int N, void* out, long long ldo,
                              int fp64) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)M * N) return;
    const long long m = t / N, n = t % N;
    // compensated (Kahan) FP32 sum: its error is about one FP32 rounding of the result, far below
    // each partial's own accumulation error, and the additions stay off GB300's narrow FP64 pipe
    float sum = 0.f, comp = 0.f;
    const long long MN = (long long)M * N;
#pragma unroll 4
    for (int z = 0; z < splits; ++z) {
        const float y = __ldg(&part[(long long)z * MN + t]) - comp;
        const float u = sum + y;
        comp = (u - sum) - y;
        sum = u;
    }
    if (fp64) ((double*)out)[m * ldo + n] = (double)sum - (double)comp;
    else ((float*)out)[m * ldo + n] = sum;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    // resolved once per process (thread-safe static initialisation); a failed lookup is
    // retried on the next call
    static std::mutex mu;
    static EncodeTiledFn fn = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        VTN_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        VTN_REQUIRE(q == cudaDriverEntryPointSuccess && p != nullptr, "cuTensorMapEncodeTiled unavailable");
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 2-D bf16 tensor map over a rows x cols (cols contiguous, row stride ld elements) matrix
CUtensorMap make_map(const void* base, long long rows, long long cols, long long ld, int box_rows) {
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Error{VTN_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
    return m;
}

}  // namespace

void tc_gemm_bf16(Ctx& ctx, const TcGemmArgs& a, int timing_class, double useful_flops) {
    if (a.M <= 0 || a.N <= 0) return;
    VTN_REQUIRE(a.K > 0 && a.K % BK == 0, "tensor-core GEMM needs K to be a positive multiple of 64");
    VTN_REQUIRE(a.lda % 8 == 0 && a.ldb % 8 == 0 && a.lda >= a.K && a.ldb >= a.K,
                "tensor-core GEMM needs 16-byte aligned row strides");
    VTN_REQUIRE(((uintptr_t)a.A % 16) == 0 && ((uintptr_t)a.B % 16) == 0, "TMA operands must be 16-byte aligned");
    VTN_REQUIRE(ctx.dstatus != nullptr, "context has no device status word");
    set_smem_attr_once(ctx, (const void*)tc_gemm_kernel, (int)SMEM_BYTES);
    CUtensorMap ma = make_map(a.A, a.M, a.K, a.lda, BM);
    CUtensorMap mb = make_map(a.B, a.N, a.K, a.ldb, BN);
    TcParams p;
    p.M = a.M;
    p.N = a.N;
    p.K = a.K;
    p.status = ctx.dstatus;
    dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, 1);
    VTN_REQUIRE((long long)grid.x * grid.y * 8 < (1LL << 31), "tensor-core GEMM too large");
    // split K when the output tiles leave most SMs idle (fixed-order reduction afterwards), and
    // whenever one accumulator would sum more than MAX_KB_PER_ACC k-blocks: the FP32 accumulation
    // in tensor memory then covers a bounded part of the sum and the partials are added with
    // compensated FP32 summation
    if (a.split3) VTN_REQUIRE(a.K % (2 * BK) == 0, "split operands need two halves of whole k-blocks");
    p.s3 = a.split3 ? 1 : 0;
    p.half = a.split3 ? a.K / 2 : 0;
    // k-blocks of the loop; a split k-block carries three products, so an accumulator run of
    // kb_acc k-blocks of split terms is kb_acc / 3 of them
    const int nkb = (a.split3 ? a.K / 2 : a.K) / BK;
    const long long tiles = (long long)grid.x * grid.y;
    int splits = 1;
    if (tiles * 2 <= ctx.num_sms && nkb >= 8)
        splits = (int)std::min<long long>(std::max<long long>(1, ctx.num_sms / tiles), nkb / 4);
    splits = std::max(1, std::min(splits, 8));
    int kb_acc = a.max_kb_per_acc > 0 ? a.max_kb_per_acc : MAX_KB_PER_ACC;
    if (a.split3) kb_acc = std::max(1, kb_acc / 3);
    splits = std::max(splits, (nkb + kb_acc - 1) / kb_acc);
    int per = (nkb + splits - 1) / splits;
    splits = (nkb + per - 1) / per;
    p.kb_per = per;
    float* part = nullptr;
    if (splits > 1) {
        part = (float*)ctx.workspace(WS_TC_PART, sizeof(float) * (size_t)splits * a.M * a.N);
        p.D = part;
        p.ldd = a.N;
        p.d_fp64 = 0;
        p.d_split = (long long)a.M * a.N;
    } else {
        p.D = a.D;
        p.ldd = a.ldd;
        p.d_fp64 = a.d_fp64 ? 1 : 0;
        p.d_split = 0;
    }
    p.splits = splits;
    const long long items = tiles * splits;
    const unsigned n_cta = (unsigned)std::min<long long>(items, std::max(ctx.num_sms, 1));
    const double flops = 2.0 * a.M * (double)a.N * (a.split3 ? 3.0 * (a.K / 2) : (double)a.K);
    int t0 = ctx.tbegin(TC_TC, flops);
    int t1 = timing_class >= 0 ? ctx.tbegin(timing_class, useful_flops) : -1;
    tc_gemm_kernel<<<n_cta, TC_THREADS, SMEM_BYTES, ctx.stream>>>(ma, mb, p);
    ctx.count_launch();
    ctx.check_launch("tc_gemm_kernel");
    if (splits > 1) {
        const long long cnt = (long long)a.M * a.N;
        splitk_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(part, splits, a.M, a.N, a.D, a.ldd,
                                                                              a.d_fp64 ? 1 : 0);
        ctx.count_launch();
        ctx.check_launch("splitk_reduce");
    }
    ctx.tend(t1);
    ctx.tend(t0);
}

}  // namespace vtn
