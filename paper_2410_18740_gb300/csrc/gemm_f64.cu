// Complex FP64 GEMM for the FP64 solver path (SIMT DFMA; GB300 has no FP64 tensor-core
// rate worth using, and FP64 FMA throughput is the roofline of this kernel):
//   C[batch] (=|+=) sum_{kb} op(A[batch, kb]) op(B[batch, kb]),  op in {X, X^dag}.
// Every contraction of the two-site effective Hamiltonian, the environment updates and
// the reduced density matrix is one call.  Tiles of 64 x 64 outputs per 256-thread CTA,
// 4 x 4 complex micro-tile per thread, K staged through shared memory in steps of 8.
// One CTA alone keeps an SM's FP64 pipe only about half busy, so a call with fewer output
// tiles than two per SM splits the summation range (kb, K) over S CTAs per tile; the S
// partial tiles are summed in a fixed order by a second kernel (deterministic).
#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4, NT = 256;

struct GemmP {
    int M, N, K, kb;
    int opA, opB;
    const double2* A; long long lda, sA_batch, sA_kb;
    const double2* B; long long ldb, sB_batch, sB_kb;
    double2* C; long long ldc, sC_batch;
    int accumulate;
    int herm_lower;
    int negate;
    int splits;          // S: CTAs per output tile along the summation range
    double2* part;       // S > 1: partial tiles [S][batch][M][N]
};

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

__global__ void __launch_bounds__(NT) gemm_c64_kernel(GemmP p) {
    __shared__ double2 As[BK][BM];
    __shared__ double2 Bs[BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const long long bz = blockIdx.z / p.splits;
    const int split = blockIdx.z % p.splits;
    if (p.herm_lower && n0 >= m0 + BM) return;  // tile strictly above the diagonal
    double2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = make_double2(0.0, 0.0);

    // this CTA's share [t0, t1) of the kb * ceil(K / BK) steps of the summation
    const int nk = (p.K + BK - 1) / BK;
    const long long T = (long long)nk * p.kb;
    const long long t0 = T * split / p.splits, t1 = T * (split + 1) / p.splits;
    int kb = (int)(t0 / nk), k0 = (int)(t0 % nk) * BK;
    for (long long t = t0; t < t1; ++t) {
        const double2* A = p.A + bz * p.sA_batch + (long long)kb * p.sA_kb;
        const double2* B = p.B + bz * p.sB_batch + (long long)kb * p.sB_kb;
        {
            // ---- stage op(A)[m0:m0+64, k0:k0+8]
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int idx = tid + r * NT;
                int ml, kl;
                if (p.opA == OP_N) { ml = idx / BK; kl = idx % BK; }
                else { ml = idx % BM; kl = idx / BM; }
                int m = m0 + ml, k = k0 + kl;
                double2 v = make_double2(0.0, 0.0);
                if (m < p.M && k < p.K) {
                    v = (p.opA == OP_N) ? A[(long long)m * p.lda + k] : cconj(A[(long long)k * p.lda + m]);
                }
                As[kl][ml] = v;
            }
            // ---- stage op(B)[k0:k0+8, n0:n0+64]
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int idx = tid + r * NT;
                int nl, kl;
                if (p.opB == OP_N) { nl = idx % BN; kl = idx / BN; }
                else { kl = idx % BK; nl = idx / BK; }
                int n = n0 + nl, k = k0 + kl;
                double2 v = make_double2(0.0, 0.0);
                if (n < p.N && k < p.K) {
                    v = (p.opB == OP_N) ? B[(long long)k * p.ldb + n] : cconj(B[(long long)n * p.ldb + k]);
                }
                Bs[kl][nl] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double2 a[TM], b[TN];
#pragma unroll
                for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < TM; ++i)
#pragma unroll
                    for (int j = 0; j < TN; ++j) {
                        acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
                        acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
                        acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
                        acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
                    }
            }
            __syncthreads();
        }
        k0 += BK;
        if (k0 >= p.K) { k0 = 0; ++kb; }
    }
    if (p.negate) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = make_double2(-acc[i][j].x, -acc[i][j].y);
    }
    const bool to_part = p.splits > 1;
    double2* C = to_part ? p.part + ((long long)split * (gridDim.z / p.splits) + bz) * p.M * p.N : p.C + bz * p.sC_batch;
    const long long ldc = to_part ? p.N : p.ldc;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        int m = m0 + ty + 16 * i;
        if (m >= p.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            int n = n0 + tx + 16 * j;
            if (n >= p.N) continue;
            double2* c = C + (long long)m * ldc + n;
            if (p.accumulate && !to_part) {
                double2 o = *c;
                *c = make_double2(o.x + acc[i][j].x, o.y + acc[i][j].y);
            } else {
                *c = acc[i][j];
            }
        }
    }
}

// C[b][m][n] (=|+=) sum_{s < S} part[s][b][m][n], s ascending
__global__ void splitk_sum(GemmP p, int batch) {
    const long long mn = (long long)p.M * p.N;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mn * batch) return;
    const long long b = t / mn, e = t % mn;
    const int m = (int)(e / p.N), n = (int)(e % p.N);
    if (p.herm_lower && n / BN > m / BM) return;
    double2 acc = p.part[t];
    for (int s = 1; s < p.splits; ++s) {
        const double2 v = p.part[(long long)s * mn * batch + t];
        acc.x += v.x;
        acc.y += v.y;
    }
    double2* c = p.C + b * p.sC_batch + (long long)m * p.ldc + n;
    if (p.accumulate) {
        const double2 o = *c;
        acc.x += o.x;
        acc.y += o.y;
    }
    *c = acc;
}

__global__ void mirror_kernel(double2* C, int n, long long ldc) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    if (j <= i) return;
    const double2 v = C[(long long)j * ldc + i];
    C[(long long)i * ldc + j] = make_double2(v.x, -v.y);
}

}  // namespace

void mirror_lower_to_upper(Ctx& ctx, double2* C, int n, long long ldc) {
    const long long cnt = (long long)n * n;
    if (cnt == 0) return;
    mirror_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(C, n, ldc);
    ctx.count_launch();
    ctx.check_launch("mirror_kernel");
}

void gemm_c64(Ctx& ctx, const GemmArgs& g, int timing_class) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return;
    VTN_REQUIRE(g.batch <= 65535, "gemm batch too large");
    GemmP p;
    p.M = g.M; p.N = g.N; p.K = g.K; p.kb = g.kb;
    p.opA = g.opA; p.opB = g.opB;
    p.A = g.A; p.lda = g.lda; p.sA_batch = g.sA_batch; p.sA_kb = g.sA_kb;
    p.B = g.B; p.ldb = g.ldb; p.sB_batch = g.sB_batch; p.sB_kb = g.sB_kb;
    p.C = g.C; p.ldc = g.ldc; p.sC_batch = g.sC_batch;
    p.accumulate = g.accumulate ? 1 : 0;
    p.herm_lower = g.herm_lower ? 1 : 0;
    p.negate = g.negate ? 1 : 0;
    VTN_REQUIRE(!g.herm_lower || (g.M == g.N && !g.accumulate), "Hermitian GEMM needs a square, non-accumulating C");
    const int gx = (g.N + BN - 1) / BN, gy = (g.M + BM - 1) / BM;
    VTN_REQUIRE(gy <= 65535, "gemm M too large");
    // output tiles that do work; split the summation when they leave SMs short of 2 CTAs
    const long long tiles = (g.herm_lower ? (long long)gy * (gy + 1) / 2 : (long long)gx * gy) * g.batch;
    const long long steps = (long long)((g.K + BK - 1) / BK) * g.kb;
    const long long slots = 2LL * std::max(ctx.num_sms, 1);
    int S = 1;
    if (tiles < slots) S = (int)std::min<long long>({slots / tiles, steps / 16, 32LL, 65535LL / g.batch});
    if (g.max_splits > 0) S = std::min(S, g.max_splits);
    S = std::max(S, 1);
    p.splits = S;
    p.part = nullptr;
    if (S > 1)
        p.part = (double2*)ctx.workspace(WS_GEMM_SPLIT, sizeof(double2) * (size_t)S * g.batch * g.M * g.N);
    dim3 grid(gx, gy, g.batch * S);
    double flops = 8.0 * g.M * (double)g.N * g.K * g.kb * g.batch * (g.herm_lower ? 0.5 : 1.0);
    int t0 = ctx.tbegin(TC_GEMM, flops);
    int t1 = (timing_class != TC_GEMM) ? ctx.tbegin(timing_class, flops) : -1;
    gemm_c64_kernel<<<grid, NT, 0, ctx.stream>>>(p);
    ctx.count_launch();
    ctx.check_launch("gemm_c64_kernel");
    if (S > 1) {
        const long long cnt = (long long)g.batch * g.M * g.N;
        splitk_sum<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(p, g.batch);
        ctx.count_launch();
        ctx.check_launch("splitk_sum");
    }
    ctx.tend(t1);
    ctx.tend(t0);
}

}  // namespace vtn
