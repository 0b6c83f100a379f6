// Truncation by warm-started block subspace iteration and Rayleigh-Ritz: the same split of a
// two-site tensor as truncate_dev, with the kept subspace found from a start block instead of
// a full eigendecomposition of rho (the paper's truncation is the exact one; this is a cheaper
// alternative whose energies are compared with it).
//
// T = theta as the nL x nR matrix, rho = T T^dag (direction 0, n = nL) or T^dag T (direction 1,
// n = nR).  The basis is kept as rows (Sh = S^dag, m x n) so that every product is a plain
// GEMM: Sh rho = (Sh T) T^dag (direction 0) or (Sh T^dag) T (direction 1).
//   1. m = min(nL, nR, k + p) start rows (no more than rho's rank): the k0 warm rows, then
//      Omega^dag rho with Omega (n x e)
//      complex normals of the Philox TRUNC stream of (seed, bond), entry j = r e + c;
//   2. Gram-Schmidt of the rows in order; q times Sh <- orth(Sh rho);
//   3. Rayleigh-Ritz through the exact eigensolver on the small projected problem:
//      direction 0: P = Sh T (m x nR), P P^dag = Sh rho Sh^dag; its top-k eigenvectors U' give
//        left = Sh^dag U' (n x k) and right = U'^dag P = left^dag T;
//      direction 1: P = T Sh^dag (nL x m), P^dag P = Sh rho Sh^dag; V' gives right = V'^dag Sh
//        (k x n) and left = P V' = T right^dag.
// Ritz values are returned in place of the eigenvalues; discarded = 1 - sum(kept) / ||T||^2.
#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

// out[j][r] = conj(A[r][j]) for an rows x cols matrix A (leading dimension lda)
__global__ void conj_transpose_kernel(int rows, int cols, const double2* __restrict__ A, long long lda,
                                      double2* __restrict__ out, long long ldo) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)rows * cols) return;
    const long long r = t / cols, j = t - r * cols;
    const double2 a = A[r * lda + j];
    out[j * ldo + r] = make_double2(a.x, -a.y);
}

}  // namespace

void conj_transpose_dev(Ctx& ctx, int rows, int cols, const double2* A, long long lda, double2* out, long long ldo) {
    const long long total = (long long)rows * cols;
    if (total == 0) return;
    conj_transpose_kernel<<<(unsigned)((total + 255) / 256), 256, 0, ctx.stream>>>(rows, cols, A, lda, out, ldo);
    ctx.count_launch();
    ctx.check_launch("conj_transpose_kernel");
}

TruncResult truncate_warm_dev(Ctx& ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                              const double2* theta, const double2* Sh0, int k0, int q, int p, uint64_t seed,
                              int bond, double2* left, double2* right) {
    const int nL = chi_l * d1, nR = d2 * chi_r;
    const int n = direction == 0 ? nL : nR;
    const int k = std::min(k_max, std::min(nL, nR));
    VTN_REQUIRE(k >= 1, "truncation keeps no state");
    VTN_REQUIRE(q >= 0 && q <= 64 && p >= 0 && p <= 256, "q must be in [0, 64] and p in [0, 256]");
    VTN_REQUIRE(k0 >= 0 && (k0 == 0 || Sh0 != nullptr), "warm rows missing");
    // at most rank(rho) <= min(nL, nR) vectors: more would force dependent rows on the iteration
    const int m = std::min(std::min(nL, nR), k + p);
    VTN_REQUIRE(m <= 4096, "subspace larger than 4096 is not supported");
    const int kw = std::min(k0, m);
    const int other = direction == 0 ? nR : nL;
    double2* Sh = (double2*)ctx.workspace(WS_WARM_S, sizeof(double2) * (size_t)m * n);
    double2* Z = (double2*)ctx.workspace(WS_WARM_Z, sizeof(double2) * (size_t)m * std::max(n, other));
    double2* P = (double2*)ctx.workspace(WS_WARM_P, sizeof(double2) * (size_t)m * std::max(nL, nR));
    // Omega^dag (e x n, e <= m), then U' (m x k) or V'^dag (k x m); k <= m <= n
    double2* U1 = (double2*)ctx.workspace(WS_WARM_U, sizeof(double2) * (size_t)m * n);
    double* nrm = (double*)ctx.workspace(WS_WARM_N, sizeof(double) * 2);
    // out (rows x n, ld n) = X (rows x n, ld ldx) rho
    auto times_rho = [&](const double2* X, long long ldx, int rows, double2* out) {
        if (rows == 0) return;
        GemmArgs g1;  // Z = X T (direction 0) or X T^dag (direction 1): rows x other
        g1.M = rows; g1.N = other; g1.K = n;
        g1.A = X; g1.lda = ldx;
        if (direction == 0) {
            g1.B = theta; g1.ldb = nR;
        } else {
            g1.opB = OP_C; g1.B = theta; g1.ldb = nR;
        }
        g1.C = Z; g1.ldc = other;
        gemm_c64(ctx, g1);
        GemmArgs g2;  // out = Z T^dag (direction 0) or Z T (direction 1): rows x n
        g2.M = rows; g2.N = n; g2.K = other;
        g2.A = Z; g2.lda = other;
        if (direction == 0) {
            g2.opB = OP_C; g2.B = theta; g2.ldb = nR;
        } else {
            g2.B = theta; g2.ldb = nR;
        }
        g2.C = out; g2.ldc = n;
        gemm_c64(ctx, g2);
    };
    // 1. start rows
    if (kw > 0)
        VTN_CUDA_TRY(cudaMemcpyAsync(Sh, Sh0, sizeof(double2) * (size_t)kw * n, cudaMemcpyDeviceToDevice, ctx.stream));
    const int e = m - kw;
    if (e > 0) {
        // Omega (n x e) in P, then rows kw.. of Sh = Omega^dag rho
        fill_random_normal(ctx, P, (long long)n * e, seed, bond, PHILOX_STREAM_TRUNC);
        conj_transpose_dev(ctx, n, e, P, e, U1, n);  // Omega^dag (e x n) in U1
        times_rho(U1, n, e, Sh + (size_t)kw * n);
    }
    // 2. orthonormal rows, q subspace iterations
    orthonormalize_rows(ctx, Sh, m, n);
    for (int it = 0; it < q; ++it) {
        times_rho(Sh, n, m, P);
        VTN_CUDA_TRY(cudaMemcpyAsync(Sh, P, sizeof(double2) * (size_t)m * n, cudaMemcpyDeviceToDevice, ctx.stream));
        orthonormalize_rows(ctx, Sh, m, n);
    }
    // 3. Rayleigh-Ritz on the projected problem
    norm2_dev(ctx, theta, (long long)nL * nR, nrm);
    TruncResult r;
    if (direction == 0) {
        GemmArgs g;  // P = Sh T (m x nR)
        g.M = m; g.N = nR; g.K = nL;
        g.A = Sh; g.lda = n;
        g.B = theta; g.ldb = nR;
        g.C = P; g.ldc = nR;
        gemm_c64(ctx, g);
        // P P^dag = U' diag(w) U'^dag; U1 = U' (m x k), right = U'^dag P (k x nR)
        r = truncate_dev(ctx, m, 1, 1, nR, 0, k, P, U1, right);
        GemmArgs gl;  // left = Sh^dag U' (nL x k)
        gl.M = nL; gl.N = r.k; gl.K = m;
        gl.opA = OP_C; gl.A = Sh; gl.lda = n;
        gl.B = U1; gl.ldb = r.k;
        gl.C = left; gl.ldc = r.k;
        gemm_c64(ctx, gl);
    } else {
        GemmArgs g;  // P = T Sh^dag (nL x m)
        g.M = nL; g.N = m; g.K = nR;
        g.A = theta; g.lda = nR;
        g.opB = OP_C; g.B = Sh; g.ldb = n;
        g.C = P; g.ldc = m;
        gemm_c64(ctx, g);
        // P^dag P = V' diag(w) V'^dag; U1 = V'^dag (k x m), left = P V' (nL x k)
        r = truncate_dev(ctx, chi_l, d1, 1, m, 1, k, P, left, U1);
        GemmArgs gr;  // right = V'^dag Sh (k x nR)
        gr.M = r.k; gr.N = nR; gr.K = m;
        gr.A = U1; gr.lda = m;
        gr.B = Sh; gr.ldb = n;
        gr.C = right; gr.ldc = nR;
        gemm_c64(ctx, gr);
    }
    double tot = 0.0;
    VTN_CUDA_TRY(cudaMemcpyAsync(&tot, nrm, sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
    ctx.sync();
    double kept = 0.0;
    for (double l : r.lam) kept += l;
    r.discarded = tot > 0.0 ? 1.0 - kept / tot : 0.0;
    return r;
}

}  // namespace vtn
