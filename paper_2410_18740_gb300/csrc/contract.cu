// Tensor contractions of two-site DMRG: the effective-Hamiltonian product H_eff psi
// (the hot path), the left/right environment updates, and the sparse MPO-core mixing
// they share.  Every dense contraction is a complex GEMM (gemm_c64); the MPO cores of
// the GBS Hamiltonian are block sparse (mostly identity pass-through channels, SM Sec. 8),
// so their action is a separate mixing kernel over channels and one physical leg.
//
// Layouts (row-major, complex as double2):
//   theta[a][s1][s2][b], L[w][bra][ket], R[w][ket][bra], A[a][s][b].
#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// out[b][p][s'][q] = sum_{e in ptr[b]..ptr[b+1]} op_e[s'][s] in[src_e][p][s][q]
template <int DM>
__global__ void __launch_bounds__(256) mix_kernel(int P, int d, int Q, const int* __restrict__ ptr,
                                                  const int* __restrict__ src, const int* __restrict__ opi,
                                                  const double2* __restrict__ ops,
                                                  const unsigned char* __restrict__ ident,
                                                  const double2* __restrict__ in, double2* __restrict__ out) {
    const long long PQ = (long long)P * Q;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= PQ) return;
    const int b = blockIdx.y;
    const long long p = t / Q, q = t % Q;
    const long long blk = PQ * d;
    double2 acc[DM];
#pragma unroll
    for (int s = 0; s < DM; ++s) acc[s] = make_double2(0.0, 0.0);
    const int e0 = ptr[b], e1 = ptr[b + 1];
    for (int e = e0; e < e1; ++e) {
        const int a = src[e], k = opi[e];
        const double2* x = in + (long long)a * blk + p * d * Q + q;
        const double2* op = ops + (long long)k * d * d;
        if (ident[k]) {
            const double2 s = op[0];
#pragma unroll
            for (int sp = 0; sp < DM; ++sp)
                if (sp < d) cfma(acc[sp], s, x[(long long)sp * Q]);
        } else {
            double2 xv[DM];
#pragma unroll
            for (int s = 0; s < DM; ++s) xv[s] = (s < d) ? x[(long long)s * Q] : make_double2(0.0, 0.0);
#pragma unroll
            for (int sp = 0; sp < DM; ++sp) {
                if (sp >= d) continue;
#pragma unroll
                for (int s = 0; s < DM; ++s)
                    if (s < d) cfma(acc[sp], op[sp * d + s], xv[s]);
            }
        }
    }
    double2* y = out + (long long)b * blk + p * d * Q + q;
#pragma unroll
    for (int sp = 0; sp < DM; ++sp)
        if (sp < d) y[(long long)sp * Q] = acc[sp];
}

}  // namespace

void mix_apply(Ctx& ctx, const DevCore& core, bool by_col, int P, int Q, const double2* in, double2* out) {
    const int w_out = by_col ? core.wr : core.wl;
    const int d = core.d;
    const long long PQ = (long long)P * Q;
    if (PQ == 0) return;
    VTN_REQUIRE(w_out <= 65535, "too many MPO channels");
    dim3 grid((unsigned)((PQ + 255) / 256), w_out);
    const int* ptr = by_col ? core.col_ptr : core.row_ptr;
    const int* src = by_col ? core.col_src : core.row_src;
    const int* opi = by_col ? core.col_op : core.row_op;
    // flops: identity entries d complex MACs, dense entries d^2, per (p, q)
    double fl = 8.0 * PQ * ((double)core.n_ident * d + (double)core.n_dense * d * d);
    int t = ctx.tbegin(TC_MIX, fl);
    if (d <= 4)
        mix_kernel<4><<<grid, 256, 0, ctx.stream>>>(P, d, Q, ptr, src, opi, core.ops, core.ident, in, out);
    else if (d <= 8)
        mix_kernel<8><<<grid, 256, 0, ctx.stream>>>(P, d, Q, ptr, src, opi, core.ops, core.ident, in, out);
    else
        mix_kernel<16><<<grid, 256, 0, ctx.stream>>>(P, d, Q, ptr, src, opi, core.ops, core.ident, in, out);
    ctx.count_launch();
    ctx.check_launch("mix_kernel");
    ctx.tend(t);
}

double heff_flops(const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r) {
    const double d = Wi.d;
    return 8.0 * d * d * chi_l * (double)chi_r * ((double)Wi.wl * chi_l + (double)Wj.wr * chi_r);
}

// y = sum L[a] Wi[a,b] Wj[b,c] theta R[c]
void heff_apply_dev(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r, const double2* L,
                    const double2* R, const double2* theta, double2* y) {
    VTN_REQUIRE(Wi.wr == Wj.wl && Wi.d == Wj.d, "inconsistent MPO cores");
    const int d = Wi.d;
    const long long n_theta = (long long)chi_l * d * d * chi_r;
    const int wmax = std::max(Wi.wl, std::max(Wi.wr, Wj.wr));
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * n_theta);
    double2* Yb = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * n_theta);
    // T1[a][i][s1 s2 k] = sum_j L[a][i][j] theta[j][s1 s2 k]
    GemmArgs g1;
    g1.M = Wi.wl * chi_l; g1.N = d * d * chi_r; g1.K = chi_l;
    g1.A = L; g1.lda = chi_l;
    g1.B = theta; g1.ldb = (long long)d * d * chi_r;
    g1.C = X; g1.ldc = (long long)d * d * chi_r;
    gemm_c64(ctx, g1, TC_HEFF);
    // T2[b][i][t][s2 k]: Wi acting on s1
    mix_apply(ctx, Wi, true, chi_l, d * chi_r, X, Yb);
    // T3[c][i t][u][k]: Wj acting on s2
    mix_apply(ctx, Wj, true, chi_l * d, chi_r, Yb, X);
    // y[i t u][l] = sum_c sum_k T3[c][i t u][k] R[c][k][l]
    GemmArgs g2;
    g2.M = chi_l * d * d; g2.N = chi_r; g2.K = chi_r; g2.kb = Wj.wr;
    g2.A = X; g2.lda = chi_r; g2.sA_kb = n_theta;
    g2.B = R; g2.ldb = chi_r; g2.sB_kb = (long long)chi_r * chi_r;
    g2.C = y; g2.ldc = chi_r;
    gemm_c64(ctx, g2, TC_HEFF);
}

void env_left_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* A,
                  double2* out) {
    const int d = W.d;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(W.wl, W.wr);
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * nA);
    double2* Yb = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * nA);
    // T[a][i][s k] = sum_j L[a][i][j] A[j][s k]
    GemmArgs g1;
    g1.M = W.wl * chi_l; g1.N = d * chi_r; g1.K = chi_l;
    g1.A = L; g1.lda = chi_l;
    g1.B = A; g1.ldb = (long long)d * chi_r;
    g1.C = X; g1.ldc = (long long)d * chi_r;
    gemm_c64(ctx, g1);
    // U[b][i][t][k] = sum W[a,b,t,s] T[a][i][s][k]
    mix_apply(ctx, W, true, chi_l, chi_r, X, Yb);
    // out[b][l][k] = sum_{i t} conj(A[i t][l]) U[b][i t][k]
    GemmArgs g2;
    g2.M = chi_r; g2.N = chi_r; g2.K = chi_l * d; g2.batch = W.wr;
    g2.opA = OP_C; g2.A = A; g2.lda = chi_r; g2.sA_batch = 0;
    g2.B = Yb; g2.ldb = chi_r; g2.sB_batch = nA;
    g2.C = out; g2.ldc = chi_r; g2.sC_batch = (long long)chi_r * chi_r;
    gemm_c64(ctx, g2);
}

void env_right_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R, const double2* A,
                   double2* out) {
    const int d = W.d;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(W.wl, W.wr);
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * nA);
    double2* Yb = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * nA);
    // T[c][j s][p] = sum_g A[j s][g] R[c][g][p]
    GemmArgs g1;
    g1.M = chi_l * d; g1.N = chi_r; g1.K = chi_r; g1.batch = W.wr;
    g1.A = A; g1.lda = chi_r; g1.sA_batch = 0;
    g1.B = R; g1.ldb = chi_r; g1.sB_batch = (long long)chi_r * chi_r;
    g1.C = X; g1.ldc = chi_r; g1.sC_batch = nA;
    gemm_c64(ctx, g1);
    // U[b][j][t][p] = sum W[b,c,t,s] T[c][j][s][p]  (output channel = core row)
    mix_apply(ctx, W, false, chi_l, chi_r, X, Yb);
    // out[b][j][i] = sum_{t p} U[b][j][t p] conj(A[i][t p])
    GemmArgs g2;
    g2.M = W.wl * chi_l; g2.N = chi_l; g2.K = d * chi_r;
    g2.A = Yb; g2.lda = (long long)d * chi_r;
    g2.opB = OP_C; g2.B = A; g2.ldb = (long long)d * chi_r;
    g2.C = out; g2.ldc = chi_l;
    gemm_c64(ctx, g2);
}

// Two-layer left environment of <psi|H H|psi> (the energy variance):
//   out[c][b][l][k] = sum conj(A[i,u,l]) W[a,c,u,t] W[a',b,t,s] L2[a][a'][i][j] A[j,s,k]
// (index a: the H next to the bra; a': the H next to the ket).  T and V share the buffer
// tv (max(w_l, w_r)^2 |A| complex), U uses u (w_l w_r |A|).
void env_left2_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L2, const double2* A,
                   double2* out, double2* tv, double2* u) {
    const int d = W.d, wl = W.wl, wr = W.wr;
    const long long nA = (long long)chi_l * d * chi_r;
    // T[a][a'][i][s k] = sum_j L2[a][a'][i][j] A[j][s k]
    GemmArgs g1;
    g1.M = wl * wl * chi_l; g1.N = d * chi_r; g1.K = chi_l;
    g1.A = L2; g1.lda = chi_l;
    g1.B = A; g1.ldb = (long long)d * chi_r;
    g1.C = tv; g1.ldc = (long long)d * chi_r;
    gemm_c64(ctx, g1);
    // U[a][b][i][t][k] = sum_{a', s} W[a',b,t,s] T[a][a'][i][s][k]   (one mixing per a)
    for (int a = 0; a < wl; ++a) mix_apply(ctx, W, true, chi_l, chi_r, tv + (long long)a * wl * nA, u + (long long)a * wr * nA);
    // V[c][b][i][u][k] = sum_{a, t} W[a,c,u,t] U[a][b][i][t][k]   (p = (b, i))
    mix_apply(ctx, W, true, wr * chi_l, chi_r, u, tv);
    // out[c][b][l][k] = sum_{i u} conj(A[i u][l]) V[c][b][i u][k]
    GemmArgs g2;
    g2.M = chi_r; g2.N = chi_r; g2.K = chi_l * d; g2.batch = wr * wr;
    g2.opA = OP_C; g2.A = A; g2.lda = chi_r; g2.sA_batch = 0;
    g2.B = tv; g2.ldb = chi_r; g2.sB_batch = nA;
    g2.C = out; g2.ldc = chi_r; g2.sC_batch = (long long)chi_r * chi_r;
    gemm_c64(ctx, g2);
}

}  // namespace vtn
