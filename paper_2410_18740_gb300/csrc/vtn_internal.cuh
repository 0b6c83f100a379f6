// Internal declarations shared by the CUDA translation units of libvtn.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <complex>
#include <cstdint>
#include <functional>
#include <string>
#include <vector>

#include "host_mpo.h"
#include "vtn.h"

namespace vtn {

#ifdef __CUDACC__
// Sum over the 32 lanes of 32 values per lane (butterfly reduce-scatter): afterwards lane l
// holds the warp total of value l.  31 additions per lane, all 32 lanes busy.
__device__ __forceinline__ double warp_reduce32(double (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const double send = upper ? v[i] : v[i + off];
            const double keep = upper ? v[i + off] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0];
}
#endif


// ------------------------------------------------------------------ errors
struct Error {
    vtn_status status;
    std::string msg;
};

#define VTN_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) throw ::vtn::Error{VTN_ECUDA, std::string(#expr) + ": " +     \
                                                             cudaGetErrorString(e_)};       \
    } while (0)

#define VTN_REQUIRE(cond, msg)                                                              \
    do {                                                                                    \
        if (!(cond)) throw ::vtn::Error{VTN_EINVAL, (msg)};                                 \
    } while (0)

// ------------------------------------------------------------------ timing classes
enum TimingClass { TC_GEMM = 0, TC_HEFF = 1, TC_EIG = 2, TC_LANCZOS = 3, TC_MIX = 4, TC_TC = 5, TC_TRI = 6, TC_COUNT = 7 };

struct Ctx;

// Device buffer owned through the context's allocator.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

// Device copy of one sparse MPO core, indexed for the mixing kernel in both directions.
struct DevCore {
    int wl = 0, wr = 0, d = 0, nnz = 0;
    // entries grouped by output channel for "apply along columns" (output = column b)
    int* col_ptr = nullptr;   // [wr + 1]
    int* col_src = nullptr;   // [nnz] source row a
    int* col_op = nullptr;    // [nnz] operator index
    // grouped by output row for "apply along rows" (output = row a, source = column b)
    int* row_ptr = nullptr;   // [wl + 1]
    int* row_src = nullptr;   // [nnz]
    int* row_op = nullptr;    // [nnz]
    double2* ops = nullptr;   // [nnz][d][d]
    float2* ops_f32 = nullptr;  // the same operators rounded to FP32 once at upload (the FP32 mixing
                                // of the split-precision mode reads these: a double -> float
                                // conversion runs on GB300's narrow FP64 pipe)
    unsigned char* ident = nullptr;  // [nnz]
    double flops_ident = 0, flops_dense = 0;  // counts for the flop model
    int n_ident = 0, n_dense = 0;
    // collapse cores (many scaled-identity entries): C[a][b] (w_l x w_r, FP32, the identity
    // entries' scalars; cid_real when every imaginary part is zero) and the index lists of the
    // remaining (dense) entries by column and by row
    bool has_cid = false, cid_real = false;
    float2* cid = nullptr;
    int *dcol_ptr = nullptr, *dcol_src = nullptr, *dcol_op = nullptr;
    int *drow_ptr = nullptr, *drow_src = nullptr, *drow_op = nullptr;
    std::vector<DevBuf> bufs;
};

struct Ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    vtn_allocator alloc{};
    bool has_alloc = false;
    std::string err;
    long long launches = 0;
    bool timing = false;
    // k-blocks per tensor-memory accumulator in the split-precision products: environment updates
    // (their errors accumulate along the chain) and H_eff psi
    int tc_kb_env = 64, tc_kb_heff = 256;
    // the truncation's tridiagonalisation keeps only the lower triangle up to date for n >= this
    int tri_lower_min_n = 1200;
    struct Tc {
        long long launches = 0;
        double flops = 0, seconds = 0;
    } tc[TC_COUNT];
    struct Pending {
        cudaEvent_t a, b;
        int cls;
        double flops;
    };
    std::vector<Pending> pending;
    int open_intervals = 0;
    std::vector<cudaEvent_t> event_pool;
    // named workspace slots
    std::vector<DevBuf> ws;
    double* pinned = nullptr;  // pinned host scratch (4096 doubles)
    double* defer_buf = nullptr;  // pinned staging of results read back once per sweep
    size_t defer_cap = 0;         // doubles
    long long host_syncs = 0;     // stream synchronisations made by sync()
    double* defer_reserve(size_t doubles);  // grows (synchronising first), never shrinks
    int* dstatus = nullptr;    // device status word: non-zero after a bounded device wait gave up
    int num_sms = 0;

    void* dalloc(size_t bytes);
    void dfree(void* p);
    void* workspace(int slot, size_t bytes);  // grows, never shrinks
    void count_launch(int n = 1) { launches += n; }
    // timing: begin() returns an index (or -1 when timing is off); end() closes it
    int tbegin(int cls, double flops);
    void tend(int idx);
    void tflush();  // synchronise and accumulate pending intervals
    void sync() {
        ++host_syncs;
        VTN_CUDA_TRY(cudaStreamSynchronize(stream));
    }
    void check_launch(const char* what);
    void check_dstatus();  // synchronises; throws VTN_ETIMEOUT (and clears the word) if set
};

enum WsSlot {
    WS_X = 0, WS_Y, WS_Z, WS_KRYLOV, WS_VEC_W, WS_VEC_T, WS_PARTIAL, WS_SCAL, WS_EIG_A, WS_EIG_H,
    WS_EIG_Y, WS_EIG_WORK, WS_EIG_U, WS_CORE_A, WS_CORE_B, WS_ENV_TMP, WS_MISC, WS_TC_L, WS_TC_R, WS_TC_B1,
    WS_TC_A2, WS_TC_PART, WS_GEMM_SPLIT, WS_EIG_PART, WS_TC_ENV, WS_EIG_T, WS_H2_ENV, WS_EXPAND,
    WS_TRUNC_L, WS_TRUNC_R, WS_CENTER, WS_MLP_ACT, WS_MLP_Y, WS_MLP_G, WS_WARM_S, WS_WARM_Z, WS_WARM_P,
    WS_WARM_U, WS_WARM_N, WS_WARM_Q0, WS_CQR_G, WS_CQR_T, WS_CQR_B, WS_RQ_Y, WS_RQ_S, WS_CHOL_LINV, WS_TH_A, WS_TH_B, WS_COUNT
};

// ------------------------------------------------------------------ cores
void upload_core(Ctx& ctx, const HostCore& hc, DevCore& dc);
void free_core(Ctx& ctx, DevCore& dc);
HostCore core_from_abi(const vtn_core* c);

// ------------------------------------------------------------------ GEMM (complex FP64)
enum Op { OP_N = 0, OP_C = 1 };  // op(X) = X or X^dag (conjugate transpose)

struct GemmArgs {
    int M, N, K;          // op(A): M x K, op(B): K x N, C: M x N
    int batch = 1;        // independent problems
    int kb = 1;           // C += sum over kb of op(A_kb) op(B_kb)
    Op opA = OP_N, opB = OP_N;
    const double2* A; long long lda; long long sA_batch = 0, sA_kb = 0;
    const double2* B; long long ldb; long long sB_batch = 0, sB_kb = 0;
    double2* C; long long ldc; long long sC_batch = 0;
    bool accumulate = false;  // C += result (else C = result)
    bool herm_lower = false;  // result is Hermitian: compute tiles on/below the diagonal only
    int max_splits = 0;       // > 0: at most this many CTAs per output tile along the summation
                              // (1 = never split, so no split-K workspace is touched); 0 = automatic
    bool negate = false;      // C (=|+=) -op(A) op(B)
};
// C[i][j] = conj(C[j][i]) for j > i (n x n, leading dimension ldc)
void mirror_lower_to_upper(Ctx& ctx, double2* C, int n, long long ldc);
void gemm_c64(Ctx& ctx, const GemmArgs& g, int timing_class = TC_GEMM);

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize, bytes) for kernel fn on the context's
// device, once per (kernel, device) (the attribute is per device); thread-safe.
void set_smem_attr_once(const Ctx& ctx, const void* fn, int bytes);

// ------------------------------------------------------------------ tensor-core GEMM (bf16 -> fp32)
// D[m][n] = sum_k A[m][k] B[n][k]; A: M x K, B: N x K (K-major bf16, K % 64 == 0); D fp32/fp64
struct TcGemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    long long lda;
    const __nv_bfloat16* B;
    long long ldb;
    void* D;
    long long ldd;
    bool d_fp64 = false;
    bool split3 = false;     // A and B are split operands in hi | lo halves (tc_pack): three products
                             // (hi hi, hi lo, lo hi) per k-block of the hi half; K = both halves
    int max_kb_per_acc = 0;  // > 0: at most this many 64-wide k-blocks per tensor-memory accumulator
                             // (longer sums are split; FP32 partials added by compensated summation); 0 = 256
};
void tc_gemm_bf16(Ctx& ctx, const TcGemmArgs& a, int timing_class = -1, double useful_flops = 0.0);
long long tc_ksplit(long long Kt);
// split-precision operand packing (see tc_ops.cu)
// rq > 0: operand rows come in blocks of rq, block b starting s_rq elements after block b-1
void tc_pack(Ctx& ctx, const double2* X, int rows, int K, int kb, long long ld, long long s_kb, bool conj_t, bool is_b,
             __nv_bfloat16* out, int rq = 0, long long s_rq = 0);
void tc_pack(Ctx& ctx, const float2* X, int rows, int K, int kb, long long ld, long long s_kb, bool conj_t, bool is_b,
             __nv_bfloat16* out, int rq = 0, long long s_rq = 0);

// ------------------------------------------------------------------ W mixing
// out[b][p][s'][q] = sum_{entries (src -> b)} op[s'][s] in[src][p][s][q]
// by_col: output channel = core column (left-to-right use); else output = core row.
void mix_apply(Ctx& ctx, const DevCore& core, bool by_col, int P, int Q, const double2* in,
               double2* out);

// in_strides (optional): channel, p and s strides of the input (default: standard layout)
void mix_apply_f32(Ctx& ctx, const DevCore& core, bool by_col, int P, int Q, const float2* in, float2* out,
                   const long long* in_strides = nullptr);

// ------------------------------------------------------------------ contractions
void heff_apply_dev(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r,
                    const double2* L, const double2* R, const double2* theta, double2* y);
double heff_flops(const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r);
// out[b][e] = sum_a C[a * ldc + b] in[a][e] (b < w_out, e < E), FP32, on the channel-GEMM kernel of the
// collapse cores; false (nothing launched) when C does not fit in shared memory
bool channel_gemm_f32(Ctx& ctx, int w_in, int w_out, long long E, const float2* C, int ldc, bool real_c,
                      const float2* in, float2* out);

// Term form of a bond's two-site H_eff for the split-precision mode (heff_terms.cu):
//   H_eff = sum_t Lhat_t (x) (B_o(t) (x) B'_p(t)) (x) Rhat_t,
//   Lhat_t = sum_a Cl[a][t] L[a],  Rhat_t = sum_c Cr[c][t] R[c],
// where {B_o} and {B'_p} are operator bases of the two cores' d x d entries (B_0 = I) and the
// coefficient matrices K_op = W_i^(o) W_{i+1}^(p) are factorised exactly.  The first n_id terms
// have o = p = 0 (identity operators); kron holds B_o and B'_p for the others.
struct BondTerms {
    bool built = false;       // set by the owner once build_bond_terms has run for the bond
    bool usable = false;      // false: no compact term form (the bond keeps the channel-mixing form)
    bool worthwhile = false;  // the term form is the cheaper one for this bond
    int wl = 0, wr = 0, d = 0, n_t = 0, n_id = 0;
    bool real_l = false, real_r = false;  // Cl / Cr have no imaginary parts
    float2* Cl = nullptr;     // [wl][n_t]
    float2* Cr = nullptr;     // [wr][n_t]
    float2* kron = nullptr;   // [n_t - n_id][2][d][d]: B_o and B'_p of the terms that are not identities
    int* kop = nullptr;       // [n_t - n_id][2]: their basis indices (0 = identity, skipped)
    double2* Cl64 = nullptr;  // [n_t][wl] (transposed, FP64: the fold's fallback on the FP64 GEMM)
    double2* Cr64 = nullptr;  // [n_t][wr]
    DevBuf buf;
};
void build_bond_terms(Ctx& ctx, const HostCore& Wi, const HostCore& Wj, BondTerms& out);
// host part: operator bases (ri and rj elements of d x d, B_0 = I), the terms' operator pairs
// (ops[2t], ops[2t+1]) and factors U[t][a], V[t][c]; false when the bond has no compact term form;
// worthwhile: the term form is the cheaper one for this bond
bool bond_terms_host(const HostCore& Wi, const HostCore& Wj, int& n_id, std::vector<int>& ops,
                     std::vector<std::complex<double>>& U, std::vector<std::complex<double>>& V,
                     std::vector<std::complex<double>>& Bi, std::vector<std::complex<double>>& Bj, int& ri, int& rj,
                     bool& worthwhile);
void free_bond_terms(Ctx& ctx, BondTerms& bt);

// split-precision (BF16X3) H_eff psi: environments packed once per bond (folded into the term
// environments Lhat, Rhat when the bond has a usable term form)
struct HeffPacked {
    int chi_l = 0, chi_r = 0, wl = 0, wr = 0;
    long long ldL = 0, ldR = 0;
    __nv_bfloat16* L = nullptr;
    __nv_bfloat16* R = nullptr;
    const BondTerms* terms = nullptr;  // non-null: term form (wl = wr = n_t then)
};
void heff_pack_envs(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r, const double2* L,
                    const double2* R, HeffPacked& pk, const BondTerms* terms = nullptr);
void heff_apply_bf16x3(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, const HeffPacked& pk, const double2* theta,
                       double2* y);
// the term form's pieces (heff_terms.cu)
void heff_pack_terms(Ctx& ctx, const BondTerms& bt, int chi_l, int chi_r, const double2* L, const double2* R,
                     HeffPacked& pk);
void heff_apply_terms(Ctx& ctx, const HeffPacked& pk, const double2* theta, double2* y);
// C = A B (complex, FP64 in and out) as one split-precision tensor-core GEMM (tc_ops.cu)
void zgemm_bf16x3(Ctx& ctx, int M, int N, int K, const double2* A, long long lda, const double2* B, long long ldb,
                  double2* C, long long ldc);
void env_left2_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L2, const double2* A,
                   double2* out, double2* tv, double2* u);
// multilayer perceptron of the learned warm start (mlp.cu)
struct MlpShape {
    int n_in = 0, width = 0, depth = 0, n_out = 0;
    long long n_params = 0;
    std::vector<long long> offW, offb;  // per layer: offsets of W_l and b_l in the flat parameters
    MlpShape() = default;
    MlpShape(int n_in, int width, int depth, int n_out);
    int in_of(int l) const { return l == 0 ? n_in : width; }
    int out_of(int l) const { return l == depth ? n_out : width; }
};
void mlp_forward_dev(Ctx& ctx, const MlpShape& s, const float* params, int B, const float* x, float* acts,
                     float* y);
void mlp_loss_grad_dev(Ctx& ctx, const MlpShape& s, const float* params, int B, const float* x, const float* t,
                       float* grad, float* loss);
void mlp_adam_dev(Ctx& ctx, long long n, float* p, float* m, float* v, const float* g, float lr, long long step);
// single-site DMRG with subspace expansion (single_site.cu)
double heff1_flops(const DevCore& W, int chi_l, int chi_r);
void heff1_apply_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* R,
                     const double2* A, double2* y);
void expand_right_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* A,
                      double alpha, double2* Mx);
void expand_left_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R, const double2* A,
                     double alpha, double2* Mx);
void env_left_bf16x3(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* A,
                     double2* out);
void env_right_bf16x3(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R, const double2* A,
                      double2* out);
void env_left_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L,
                  const double2* A, double2* out);
void env_right_dev(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R,
                   const double2* A, double2* out);

// ------------------------------------------------------------------ vector kernels (Lanczos)
// dots[i] = sum_e conj(V[i][e]) w[e], i < nv (deterministic two-stage reduction)
// (stop, when given: a device flag; the kernels do nothing once it is non-zero)
void multi_dot(Ctx& ctx, const double2* V, long long ld, int nv, const double2* w, long long n,
               double2* dots_dev, const int* stop = nullptr);
// w -= sum_i V[i] c[i]
void multi_axpy(Ctx& ctx, const double2* V, long long ld, int nv, const double2* c_dev, double2* w,
                long long n, const int* stop = nullptr);
// out = sum_i V[i] y[i] (y real, device)
// nv_dev (may be null): the vector count is read on the device
void lincomb_real(Ctx& ctx, const double2* V, long long ld, int nv, const double* y_dev, double2* out,
                  long long n, const int* nv_dev = nullptr);
// norm2 (sum |x|^2) into dev scalar
void norm2_dev(Ctx& ctx, const double2* x, long long n, double* out_dev, const int* stop = nullptr);
// x *= 1/sqrt(*nrm2_dev)
void scale_inv_sqrt(Ctx& ctx, double2* x, long long n, const double* nrm2_dev);

struct LanczosResult {
    double theta;
    int n_matvec;
    bool converged;
};
// Lowest eigenpair of the operator applied by `matvec(in, out)` (device vectors of n complex).
// With defer != nullptr and restarts == 0 the Krylov steps are queued without any host round
// trip (every vector kernel skips itself once the device stop flag is set; the matvecs after
// the stop still run, their results unused) and {theta, resid, scratch, flag, stop, m_stop}
// (5 doubles' worth) are copied to *defer asynchronously; the returned fields are then
// placeholders until the caller has synchronised and read them (lanczos_deferred_result).
LanczosResult lanczos(Ctx& ctx, long long n, double2* x, double tol, int kmax, int restarts,
                      const std::function<void(const double2*, double2*)>& matvec, double* defer = nullptr);
// The result a deferred solve copied to `slot` (after the stream has been synchronised).
LanczosResult lanczos_deferred_result(const double* slot);

// ------------------------------------------------------------------ truncation eigensolver
struct TruncResult {
    int k;
    double discarded;
    std::vector<double> lam;
};
// Truncation by warm-started subspace iteration and Rayleigh-Ritz (trunc_warm.cu): Sh0 holds
// k0 warm rows (conjugates of the start vectors, k0 x n, n = chi_l d1 or d2 chi_r by direction).
TruncResult truncate_warm_dev(Ctx& ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                              const double2* theta, const double2* Sh0, int k0, int q, int p, uint64_t seed,
                              int bond, double2* left, double2* right);
// out[j][r] = conj(A[r][j]) (rows x cols A with leading dimension lda)
void conj_transpose_dev(Ctx& ctx, int rows, int cols, const double2* A, long long lda, double2* out, long long ldo);
// outer >= 0 limits the product formed after the eigendecomposition: direction 0 writes
// only the first `outer` columns of right (leading dimension outer), direction 1 only the
// first `outer` rows of left.
// defer != nullptr: nothing is read back; the k eigenvalues, tr(rho) and the status words are
// copied asynchronously to defer (k + 1 + 4 doubles) and the result's lam is empty until
// truncate_deferred_result reads them after a synchronisation.
TruncResult truncate_dev(Ctx& ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                         const double2* theta, double2* left, double2* right, int outer = -1,
                         double* defer = nullptr);
TruncResult truncate_deferred_result(const double* slot, int k);

// ------------------------------------------------------------------ misc kernels
// Philox counter word 3: the stream of the random numbers (initial MPS, sampler, truncation)
constexpr unsigned PHILOX_STREAM_INIT = 1u, PHILOX_STREAM_TRUNC = 3u;
void fill_random_normal(Ctx& ctx, double2* out, long long count, uint64_t seed, int site,
                        unsigned stream = PHILOX_STREAM_INIT);
void orthonormalize_rows(Ctx& ctx, double2* A, int rows, int cols);
// The same result by CholeskyQR2 (GEMM-based; chol_qr.cu), with the row-by-row kernel as the
// fallback when the rows are too ill-conditioned (or dependent) for it.
void orthonormalize_rows_cholqr(Ctx& ctx, double2* A, int rows, int cols);
// single-CTA Gram-Schmidt of the rows, skipped unless pred == nullptr or *pred != 0
void orthonormalize_rows_small(Ctx& ctx, double2* A, int rows, int cols, const int* pred);
void lbo_rotate_dev(Ctx& ctx, int chi_l, int d, int D, int chi_r, const double2* V, const double2* A,
                    double2* out);
void set_scalar_one(Ctx& ctx, double2* p);
// rho[s][t] = sum_{i, c} U[i][s][c] conj(A[i][t][c]) (d x d, device)
void reduced_density_dev(Ctx& ctx, int cl, int d, int cr, const double2* U, const double2* A, double2* rho);
void marginal_reduce_dev(Ctx& ctx, int chi_l, int D, int chi_r, const double2* AF, const double2* U, double* P);
void sample_dev(Ctx& ctx, const double2* const* AF_dev, const double2* const* ER_dev, const int* dims_dev, int M,
                int D, int chi_max, uint64_t seed, int n_samples, int* out_dev);

}  // namespace vtn

// ------------------------------------------------------------------ handles
struct vtn_ctx_s {
    vtn::Ctx c;
};

struct vtn_mpo_s {
    vtn::HostProblem hp;
    int device = -1;
    vtn_ctx owner = nullptr;
    std::vector<vtn::DevCore> dcores;
    std::vector<vtn::BondTerms> bterms;  // M - 1: term form of each bond's H_eff (split precision)
    double2* iso_dev = nullptr;  // M * D * d
};

struct vtn_mlp_s {
    vtn::MlpShape shape;
    float* params = nullptr;  // device, n_params each
    float* m = nullptr;
    float* v = nullptr;
    float* grad = nullptr;
    float* loss = nullptr;    // device scalar
    long long step = 0;       // Adam steps taken
    vtn_ctx owner = nullptr;
};

struct vtn_mps_s {
    int M = 0, d = 0, chi_cap = 0;
    std::vector<int> dims;                 // M + 1
    std::vector<double2*> sites;           // device, capacity chi_cap*d*chi_cap each
    std::vector<size_t> cap;               // complex capacity per site
    vtn_ctx owner = nullptr;
    int center = -1;                       // -1 unknown
};
