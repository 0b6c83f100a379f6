// Row orthonormalisation of a complex m x n matrix (m <= n) by CholeskyQR2 on the FP64 GEMM.
//
// Gram-Schmidt of the rows in order is the LQ factorisation A = L Q with L lower triangular
// and a positive diagonal; so is CholeskyQR: G = A A^dag = L L^dag (Cholesky), Q = L^{-1} A.
// One pass loses orthogonality like u kappa(A)^2; a second pass on Q restores it to O(u)
// while kappa(A) stays well below u^{-1/2} (Yamamoto et al., ETNA 44, 2015).  Every O(m^2 n)
// and O(m^3) step is a complex GEMM spread over all SMs:
//   Gram           G = A A^dag (lower tiles);
//   Cholesky       right-looking in blocks of NB: the diagonal block is factored (and its
//                  factor inverted) by one CTA, the panel below is L21 = A21 L11^{-dag} and the
//                  trailing matrix is updated by G22 -= L21 L21^dag;
//   solve          Q = L^{-1} A by block rows: A_b -= L[b, <b] Q[<b], Q_b = L_bb^{-1} A_b.
// The second pass checks its Gram matrix first: if max |G - I| > 0.1 (or a pivot of either
// pass was not positive, or a value is not finite) the rows were too ill-conditioned -- or
// exactly dependent -- for CholeskyQR, and the original rows are orthonormalised again by the
// row-by-row Gram-Schmidt kernel, which keeps an exactly dependent row at zero.  Both branches
// are queued; a device flag selects which one acts, so nothing is read back to the host.
#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr int NB = 32;  // diagonal block of the blocked Cholesky and of the triangular solve

// Cholesky factor of the b x b diagonal block at G (leading dimension ld; lower triangle read
// and written) and the inverse of that factor into Linv (NB x NB, zero above the diagonal).
// One CTA, b <= NB.  flag[0] = 1 on a pivot that is not positive.
__global__ void __launch_bounds__(256) potrf_block(double2* __restrict__ G, int b, long long ld,
                                                  double2* __restrict__ Linv, int* __restrict__ flag) {
    __shared__ double2 S[NB][NB + 1];
    __shared__ double2 X[NB][NB + 1];
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        const int i = t / NB, j = t - (t / NB) * NB;
        S[i][j] = (i < b && j <= i) ? G[(long long)i * ld + j] : make_double2(0.0, 0.0);
        X[i][j] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double djj = S[j][j].x;
            if (!(djj > 0.0)) {
                flag[0] = 1;  // the caller's fallback replaces the result
                djj = 1.0;
            }
            S[j][j] = make_double2(sqrt(djj), 0.0);
        }
        __syncthreads();
        const double r = 1.0 / S[j][j].x;
        for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) {
            S[i][j].x *= r;
            S[i][j].y *= r;
        }
        __syncthreads();
        // S[i][l] -= S[i][j] conj(S[l][j]) for j < l <= i (column j is only read here)
        for (int t = threadIdx.x; t < b * b; t += blockDim.x) {
            const int i = t / b, l = t - (t / b) * b;
            if (l > j && l <= i) {
                const double2 a = S[i][j], c = S[l][j];
                S[i][l].x -= a.x * c.x + a.y * c.y;
                S[i][l].y -= a.y * c.x - a.x * c.y;
            }
        }
        __syncthreads();
    }
    // X = S^{-1}, one column per thread: X[c][c] = 1 / S[c][c],
    // X[i][c] = -(sum_{c <= l < i} S[i][l] X[l][c]) / S[i][i]
    if (threadIdx.x < b) {
        const int c = threadIdx.x;
        X[c][c] = make_double2(1.0 / S[c][c].x, 0.0);
        for (int i = c + 1; i < b; ++i) {
            double re = 0.0, im = 0.0;
            for (int l = c; l < i; ++l) {
                const double2 s = S[i][l], x = X[l][c];
                re += s.x * x.x - s.y * x.y;
                im += s.x * x.y + s.y * x.x;
            }
            const double inv = 1.0 / S[i][i].x;
            X[i][c] = make_double2(-re * inv, -im * inv);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NB * NB; t += blockDim.x) {
        const int i = t / NB, j = t - (t / NB) * NB;
        if (i < b && j <= i) G[(long long)i * ld + j] = S[i][j];
        Linv[t] = X[i][j];
    }
}

// flag[0] = 1 if max over the lower triangle of |G - I| > tol or a value is not finite
__global__ void __launch_bounds__(256) gram_identity_check(const double2* __restrict__ G, int m, double tol,
                                                          int* __restrict__ flag) {
    double mx = 0.0;
    const long long total = (long long)m * m;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
        const long long i = t / m, j = t - (t / m) * m;
        if (j > i) continue;
        const double2 g = G[t];
        const double dev = fmax(fabs(g.x - (i == j ? 1.0 : 0.0)), fabs(g.y));
        mx = (dev == dev) ? fmax(mx, dev) : 1e300;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > tol) flag[0] = 1;
}

// dst = src (n elements) when *pred != 0
__global__ void copy_if(double2* __restrict__ dst, const double2* __restrict__ src, long long n,
                        const int* __restrict__ pred) {
    if (*pred == 0) return;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
        dst[t] = src[t];
}

// Lower Cholesky factor of the m x m Hermitian G in place (lower triangle), blocks of NB;
// Linv_all[c] = inverse of diagonal block c (NB x NB); tmp: at least (m - NB) x NB complex.
void cholesky_blocked(Ctx& ctx, double2* G, int m, double2* Linv_all, double2* tmp, int* flag) {
    for (int p = 0; p < m; p += NB) {
        const int b = std::min(NB, m - p);
        double2* Li = Linv_all + (size_t)(p / NB) * NB * NB;
        potrf_block<<<1, 256, 0, ctx.stream>>>(G + (size_t)p * m + p, b, m, Li, flag);
        ctx.count_launch();
        ctx.check_launch("potrf_block");
        const int rest = m - p - b;
        if (rest <= 0) break;
        double2* L21 = G + (size_t)(p + b) * m + p;
        GemmArgs t;  // tmp = A21 L11^{-dag}
        t.M = rest; t.N = b; t.K = b;
        t.A = L21; t.lda = m;
        t.opB = OP_C; t.B = Li; t.ldb = NB;
        t.C = tmp; t.ldc = b;
        gemm_c64(ctx, t);
        VTN_CUDA_TRY(cudaMemcpy2DAsync(L21, sizeof(double2) * (size_t)m, tmp, sizeof(double2) * (size_t)b,
                                       sizeof(double2) * (size_t)b, rest, cudaMemcpyDeviceToDevice, ctx.stream));
        GemmArgs u;  // G22 -= L21 L21^dag
        u.M = rest; u.N = rest; u.K = b;
        u.A = L21; u.lda = m;
        u.opB = OP_C; u.B = L21; u.ldb = m;
        u.C = L21 + b; u.ldc = m;
        u.accumulate = true;
        u.negate = true;
        gemm_c64(ctx, u);
    }
}

// A (m x n) <- L^{-1} A with L the lower factor in G (leading dimension m); tmp: NB x n.
void solve_lower_rows(Ctx& ctx, const double2* G, const double2* Linv_all, int m, int n, double2* A, double2* tmp) {
    for (int r0 = 0; r0 < m; r0 += NB) {
        const int b = std::min(NB, m - r0);
        double2* Ab = A + (size_t)r0 * n;
        if (r0 > 0) {
            GemmArgs g;  // A_b -= L[b, <b] Q[<b]
            g.M = b; g.N = n; g.K = r0;
            g.A = G + (size_t)r0 * m; g.lda = m;
            g.B = A; g.ldb = n;
            g.C = Ab; g.ldc = n;
            g.accumulate = true;
            g.negate = true;
            gemm_c64(ctx, g);
        }
        GemmArgs h;  // Q_b = L_bb^{-1} A_b
        h.M = b; h.N = n; h.K = b;
        h.A = Linv_all + (size_t)(r0 / NB) * NB * NB; h.lda = NB;
        h.B = Ab; h.ldb = n;
        h.C = tmp; h.ldc = n;
        gemm_c64(ctx, h);
        VTN_CUDA_TRY(cudaMemcpyAsync(Ab, tmp, sizeof(double2) * (size_t)b * n, cudaMemcpyDeviceToDevice, ctx.stream));
    }
}

}  // namespace

void orthonormalize_rows_cholqr(Ctx& ctx, double2* A, int m, int n) {
    VTN_REQUIRE(m >= 1 && m <= n && m <= 4096, "row orthonormalisation needs 1 <= rows <= min(cols, 4096)");
    const int nblk = (m + NB - 1) / NB;
    double2* G = (double2*)ctx.workspace(WS_CQR_G, sizeof(double2) * ((size_t)m * m + (size_t)nblk * NB * NB));
    double2* Linv = G + (size_t)m * m;
    double2* tmp = (double2*)ctx.workspace(WS_CQR_T, sizeof(double2) * (size_t)NB * std::max(n, m));
    double2* backup = (double2*)ctx.workspace(WS_CQR_B, sizeof(double2) * (size_t)m * n + 256);
    int* flag = (int*)(backup + (size_t)m * n);
    VTN_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx.stream));
    VTN_CUDA_TRY(cudaMemcpyAsync(backup, A, sizeof(double2) * (size_t)m * n, cudaMemcpyDeviceToDevice, ctx.stream));
    for (int pass = 0; pass < 2; ++pass) {
        GemmArgs g;  // G = A A^dag (tiles on and below the diagonal)
        g.M = m; g.N = m; g.K = n;
        g.A = A; g.lda = n;
        g.opB = OP_C; g.B = A; g.ldb = n;
        g.C = G; g.ldc = m;
        g.herm_lower = true;
        gemm_c64(ctx, g);
        if (pass == 1) {
            gram_identity_check<<<std::min(1024, (m * m + 255) / 256), 256, 0, ctx.stream>>>(G, m, 0.1, flag);
            ctx.count_launch();
        }
        cholesky_blocked(ctx, G, m, Linv, tmp, flag);
        solve_lower_rows(ctx, G, Linv, m, n, A, tmp);
    }
    const long long cnt = (long long)m * n;
    copy_if<<<(unsigned)std::min<long long>(4096, (cnt + 255) / 256), 256, 0, ctx.stream>>>(A, backup, cnt, flag);
    ctx.count_launch();
    ctx.check_launch("copy_if");
    orthonormalize_rows_small(ctx, A, m, n, flag);
}

}  // namespace vtn
