// Single-site DMRG with subspace expansion (the solver of the paper's results section, with
// the bond dimension grown during the sweeps as in its discussion): the single-site
// effective-Hamiltonian product and the expansion of an optimised centre tensor.  Both reuse
// the contraction steps of the environment updates (complex GEMM, sparse MPO-core mixing);
// the only new kernels assemble the expanded matrix.
//
// Layouts (row-major, complex as double2): A[l][s][r], L[w][bra][ket], R[w][ket][bra].
//   heff1:        y[l,t,r'] = sum L[a,l,l'] W[a,b,t,s] A[l',s,r] R[b,r,r']
//   expand right: Mx[(l t)][c], c < chi_r: A[(l t)][c]; c = chi_r (1 + b) + r: alpha P[(l t)][b][r]
//                 with P[(l t)][b][r] = sum L[a,l,l'] W[a,b,t,s] A[l',s,r]
//   expand left:  Mx rows (block, l): block 0 = A[l][(t r')], block 1 + a = alpha P[a][l][(t r')]
//                 with P[a][l][(t r')] = sum W[a,b,t,s] A[l,s,r] R[b,r,r']
#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

__global__ void __launch_bounds__(256) assemble_right_kernel(long long rows, int cr, int wr,
                                                             const double2* __restrict__ A,
                                                             const double2* __restrict__ P, double alpha,
                                                             double2* __restrict__ Mx) {
    const long long K = (long long)cr * (1 + wr);
    const long long total = rows * K;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long row = t / K, c = t - row * K;
        double2 v;
        if (c < cr) {
            v = A[row * cr + c];
        } else {
            const long long b = (c - cr) / cr, r = (c - cr) - b * cr;
            const double2 p = P[(b * rows + row) * cr + r];
            v = make_double2(alpha * p.x, alpha * p.y);
        }
        Mx[t] = v;
    }
}

__global__ void __launch_bounds__(256) assemble_left_kernel(long long nA, long long nP,
                                                            const double2* __restrict__ A,
                                                            const double2* __restrict__ P, double alpha,
                                                            double2* __restrict__ Mx) {
    const long long total = nA + nP;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        double2 v;
        if (t < nA) {
            v = A[t];
        } else {
            const double2 p = P[t - nA];
            v = make_double2(alpha * p.x, alpha * p.y);
        }
        Mx[t] = v;
    }
}

unsigned stride_grid(const Ctx& ctx, long long total) {
    const long long want = (total + 255) / 256;
    return (unsigned)std::max<long long>(1, std::min<long long>(want, 8LL * ctx.num_sms));
}

// X[a][l][(s r)] = sum_l' L[a][l][l'] A[l'][(s r)];  Y[b][l][t][r] = sum W[a,b,t,s] X[a][l][s][r]
void left_block_times_site(Ctx& ctx, const DevCore& W, int cl, int cr, const double2* L, const double2* A,
                           double2* X, double2* Y, int timing_class) {
    const int d = W.d;
    GemmArgs g;
    g.M = W.wl * cl; g.N = d * cr; g.K = cl;
    g.A = L; g.lda = cl;
    g.B = A; g.ldb = (long long)d * cr;
    g.C = X; g.ldc = (long long)d * cr;
    gemm_c64(ctx, g, timing_class);
    mix_apply(ctx, W, true, cl, cr, X, Y);
}

}  // namespace

double heff1_flops(const DevCore& W, int chi_l, int chi_r) {
    return 8.0 * W.d * (double)chi_l * chi_r * ((double)W.wl * chi_l + (double)W.wr * chi_r);
}

void heff1_apply_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* R,
                     const double2* A, double2* y) {
    const int d = W.d;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(W.wl, W.wr);
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * nA);
    double2* Y = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * nA);
    left_block_times_site(ctx, W, chi_l, chi_r, L, A, X, Y, TC_HEFF);
    // y[(l t)][r'] = sum_b sum_r Y[b][(l t)][r] R[b][r][r']
    GemmArgs g;
    g.M = chi_l * d; g.N = chi_r; g.K = chi_r; g.kb = W.wr;
    g.A = Y; g.lda = chi_r; g.sA_kb = nA;
    g.B = R; g.ldb = chi_r; g.sB_kb = (long long)chi_r * chi_r;
    g.C = y; g.ldc = chi_r;
    gemm_c64(ctx, g, TC_HEFF);
}

void expand_right_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* A,
                      double alpha, double2* Mx) {
    const int d = W.d;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(W.wl, W.wr);
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * nA);
    double2* Y = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * nA);
    left_block_times_site(ctx, W, chi_l, chi_r, L, A, X, Y, TC_GEMM);
    const long long rows = (long long)chi_l * d;
    const long long total = rows * chi_r * (1 + (long long)W.wr);
    assemble_right_kernel<<<stride_grid(ctx, total), 256, 0, ctx.stream>>>(rows, chi_r, W.wr, A, Y, alpha, Mx);
    ctx.count_launch();
    ctx.check_launch("assemble_right_kernel");
}

void expand_left_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R, const double2* A,
                     double alpha, double2* Mx) {
    const int d = W.d;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(W.wl, W.wr);
    double2* X = (double2*)ctx.workspace(WS_X, sizeof(double2) * wmax * nA);
    double2* Y = (double2*)ctx.workspace(WS_Y, sizeof(double2) * wmax * nA);
    // X[b][(l s)][r'] = sum_r A[(l s)][r] R[b][r][r']
    GemmArgs g;
    g.M = chi_l * d; g.N = chi_r; g.K = chi_r; g.batch = W.wr;
    g.A = A; g.lda = chi_r; g.sA_batch = 0;
    g.B = R; g.ldb = chi_r; g.sB_batch = (long long)chi_r * chi_r;
    g.C = X; g.ldc = chi_r; g.sC_batch = nA;
    gemm_c64(ctx, g);
    // Y[a][l][t][r'] = sum W[a,b,t,s] X[b][l][s][r']  (output channel = core row)
    mix_apply(ctx, W, false, chi_l, chi_r, X, Y);
    const long long nP = (long long)W.wl * nA;
    assemble_left_kernel<<<stride_grid(ctx, nA + nP), 256, 0, ctx.stream>>>(nA, nP, A, Y, alpha, Mx);
    ctx.count_launch();
    ctx.check_launch("assemble_left_kernel");
}

}  // namespace vtn
