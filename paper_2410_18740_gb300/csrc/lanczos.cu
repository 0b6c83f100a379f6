// FP64 Lanczos for the lowest eigenpair of the two-site effective Hamiltonian.
//
// Krylov recursion with full re-orthogonalisation by classical Gram-Schmidt applied
// twice, explicit restart from the Ritz vector.  All vectors and scalars stay on the
// device; the host reads one status word per iteration to decide whether to go on.
// Vector kernels: grid-stride loops with 128-bit (double2) loads, warp-shuffle and
// shared-memory reductions, and deterministic two-stage sums (fixed block count and
// fixed combine order, so results are identical run to run).  The Ritz pair of the
// k x k tridiagonal matrix is found by one warp: 32-way multisection on Sturm counts for
// the lowest eigenvalue, then inverse iteration with a pivoted tridiagonal LU.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr int RB = 256;          // threads per block of the reduction kernels
constexpr int KMAX_DEV = 64;     // largest Krylov dimension handled on the device
constexpr int DOT_GROUP = 8;     // vectors per pass of multi_dot

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block reduction of one double; result valid in thread 0
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// partial[blk][i] = sum over this block's elements of conj(V[i][e]) w[e], i in [g0, g0+cnt).
// 4 FMAs per element and vector; the 2 * DOT_GROUP sums are reduced across the block by one
// butterfly reduce-scatter per warp (lane l ends with value l) and one shared-memory pass.
__global__ void __launch_bounds__(RB) multi_dot_partial(const double2* __restrict__ V, long long ld, int g0,
                                                        int cnt, const double2* __restrict__ w, long long n,
                                                        double2* __restrict__ partial, int nv_stride,
                                                        const int* __restrict__ stop) {
    static_assert(2 * DOT_GROUP <= 32, "one butterfly holds at most 32 values");
    if (stop && *stop) return;
    __shared__ double sh[RB / 32][32];
    double v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = 0.0;
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        const double2 we = w[e];
#pragma unroll
        for (int i = 0; i < DOT_GROUP; ++i) {
            if (i < cnt) {
                const double2 a = V[(long long)(g0 + i) * ld + e];
                v[2 * i] = fma(a.x, we.x, fma(a.y, we.y, v[2 * i]));          // Re conj(a) w
                v[2 * i + 1] = fma(a.x, we.y, fma(-a.y, we.x, v[2 * i + 1]));  // Im conj(a) w
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sh[wid][lane] = warp_reduce32(v);
    __syncthreads();
    if (wid == 0) {
        double t = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < RB / 32; ++w2) t += sh[w2][lane];
        // lanes 2i, 2i+1 hold Re, Im of vector i
        const double im = __shfl_down_sync(0xffffffffu, t, 1);
        if ((lane & 1) == 0 && lane / 2 < cnt)
            partial[(long long)blockIdx.x * nv_stride + g0 + lane / 2] = make_double2(t, im);
    }
}

// out[i] = sum_blk partial[blk][i] (one block per i, fixed order)
__global__ void __launch_bounds__(RB) reduce_partials(const double2* __restrict__ partial, int nblk, int nv_stride,
                                                      double2* __restrict__ out, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    const int i = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblk; b += RB) {
        double2 p = partial[(long long)b * nv_stride + i];
        re += p.x;
        im += p.y;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) out[i] = make_double2(re, im);
}

// w[e] -= sum_i V[i][e] c[i]
__global__ void __launch_bounds__(RB) multi_axpy_kernel(const double2* __restrict__ V, long long ld, int nv,
                                                        const double2* __restrict__ c, double2* __restrict__ w,
                                                        long long n, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double2 cs[KMAX_DEV];
    for (int i = threadIdx.x; i < nv; i += RB) cs[i] = c[i];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        double2 acc = w[e];
        for (int i = 0; i < nv; ++i) {  // acc -= v c: 4 FMAs
            const double2 v = V[(long long)i * ld + e];
            const double2 ci = cs[i];
            acc.x = fma(-v.x, ci.x, fma(v.y, ci.y, acc.x));
            acc.y = fma(-v.x, ci.y, fma(-v.y, ci.x, acc.y));
        }
        w[e] = acc;
    }
}

// nv_dev (may be null): the number of vectors read from the device instead of nv
__global__ void __launch_bounds__(RB) lincomb_real_kernel(const double2* __restrict__ V, long long ld, int nv,
                                                          const double* __restrict__ y, double2* __restrict__ out,
                                                          long long n, const int* __restrict__ nv_dev) {
    if (nv_dev) nv = *nv_dev;
    __shared__ double ys[KMAX_DEV];
    for (int i = threadIdx.x; i < nv; i += RB) ys[i] = y[i];
    __syncthreads();
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        double2 acc = make_double2(0.0, 0.0);
        for (int i = 0; i < nv; ++i) {
            const double2 v = V[(long long)i * ld + e];
            acc.x += v.x * ys[i];
            acc.y += v.y * ys[i];
        }
        out[e] = acc;
    }
}

__global__ void __launch_bounds__(RB) norm2_partial(const double2* __restrict__ x, long long n,
                                                    double* __restrict__ partial, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        const double2 v = x[e];
        acc += v.x * v.x + v.y * v.y;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(RB) reduce_real(const double* __restrict__ partial, int nblk,
                                                  double* __restrict__ out, const int* __restrict__ stop) {
    if (stop && *stop) return;
    __shared__ double sh[32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += RB) acc += partial[b];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) *out = acc;
}

// x *= 1/sqrt(*nrm2); skipped when *skip != 0 (skip may be null)
__global__ void __launch_bounds__(RB) scale_kernel(double2* __restrict__ x, long long n,
                                                   const double* __restrict__ nrm2, const int* __restrict__ skip,
                                                   const double2* __restrict__ src) {
    if (skip && *skip) return;
    const double s = 1.0 / sqrt(*nrm2);
    for (long long e = (long long)blockIdx.x * RB + threadIdx.x; e < n; e += (long long)gridDim.x * RB) {
        double2 v = src ? src[e] : x[e];
        x[e] = make_double2(v.x * s, v.y * s);
    }
}

// ---------------------------------------------------------------- tridiagonal Ritz pair
struct LzState {
    double alpha[KMAX_DEV];
    double beta[KMAX_DEV];
    double y[KMAX_DEV];
    double2 c1[KMAX_DEV];
    double2 c2[KMAX_DEV];
    double beta2;        // |w|^2 of the current iteration
    double theta;
    double resid;
    double scratch;
    int flag;            // 0 continue, 1 converged, 2 breakdown, 3 last iteration
    int stop;            // set (and kept) once an iteration's flag is non-zero
    int m_stop;          // Krylov dimension at that iteration
    int pad;
};

__device__ int sturm_count(const double* a, const double* b, int m, double x, double pivmin) {
    int cnt = 0;
    double q = a[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0) ++cnt;
    for (int i = 1; i < m; ++i) {
        q = a[i] - x - b[i - 1] * b[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// One warp.  Lowest eigenpair of the m x m symmetric tridiagonal (alpha, beta), Ritz
// residual beta_j |y_{m-1}|, and the decision for the host.
__global__ void ritz_kernel(LzState* st, int m, double tol, double breakdown, int last) {
    __shared__ double lo_s, hi_s;
    const int lane = threadIdx.x;
    if (st->stop) return;  // an earlier iteration ended the recursion (device-driven loop)
    const double* a = st->alpha;
    const double* b = st->beta;
    if (lane == 0) st->alpha[m - 1] = st->c1[m - 1].x;
    __syncwarp();
    double gl = 1e308, gu = -1e308, tnrm = 0.0;
    for (int i = 0; i < m; ++i) {
        double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < m ? fabs(b[i]) : 0.0);
        gl = fmin(gl, a[i] - r);
        gu = fmax(gu, a[i] + r);
        tnrm = fmax(tnrm, fabs(a[i]) + r);
    }
    const double eps = 2.220446049250313e-16;
    const double pivmin = fmax(1e-300, eps * eps * fmax(tnrm, 1e-300));
    if (lane == 0) {
        lo_s = gl - eps * tnrm - pivmin;
        hi_s = gu + eps * tnrm + pivmin;
    }
    __syncwarp();
    // multisection: find the lowest eigenvalue (count(x) >= 1 boundary)
    for (int round = 0; round < 40; ++round) {
        const double lo = lo_s, hi = hi_s;
        if (hi - lo <= 2.0 * eps * fmax(fabs(lo), fabs(hi)) + 4.0 * pivmin) break;
        const double step = (hi - lo) / 33.0;
        const double x = lo + step * (lane + 1);
        const int c = sturm_count(a, b, m, x, pivmin);
        const unsigned ballot = __ballot_sync(0xffffffffu, c >= 1);
        __syncwarp();
        if (lane == 0) {
            if (ballot == 0) {
                lo_s = lo + step * 32;
            } else {
                const int first = __ffs(ballot) - 1;
                hi_s = lo + step * (first + 1);
                lo_s = lo + step * first;
            }
        }
        __syncwarp();
    }
    if (lane != 0) return;
    const double th = 0.5 * (lo_s + hi_s);
    // inverse iteration with the pivoted LU of (T - th I)
    double dd[KMAX_DEV], du[KMAX_DEV], du2[KMAX_DEV], dl[KMAX_DEV], x[KMAX_DEV];
    int piv[KMAX_DEV];
    const double tiny = eps * fmax(tnrm, 1e-300);
    for (int i = 0; i < m; ++i) {
        dd[i] = a[i] - th;
        du[i] = (i + 1 < m) ? b[i] : 0.0;
        dl[i] = (i + 1 < m) ? b[i] : 0.0;
        du2[i] = 0.0;
        x[i] = 1.0;
    }
    for (int i = 0; i + 1 < m; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
            piv[i] = 0;
            if (dd[i] == 0.0) dd[i] = tiny;
            const double f = dl[i] / dd[i];
            dl[i] = f;
            dd[i + 1] -= f * du[i];
        } else {
            piv[i] = 1;
            const double f = dd[i] / dl[i];
            dd[i] = dl[i];
            dl[i] = f;
            const double t = du[i];
            du[i] = dd[i + 1];
            dd[i + 1] = t - f * dd[i + 1];
            if (i + 2 < m) {
                du2[i] = du[i + 1];
                du[i + 1] = -f * du[i + 1];
            }
        }
    }
    if (dd[m - 1] == 0.0) dd[m - 1] = tiny;
    for (int i = 0; i < m; ++i)
        if (fabs(dd[i]) < tiny) dd[i] = dd[i] < 0 ? -tiny : tiny;
    for (int it = 0; it < 3; ++it) {
        for (int i = 0; i + 1 < m; ++i) {
            if (piv[i] == 0) {
                x[i + 1] -= dl[i] * x[i];
            } else {
                const double t = x[i];
                x[i] = x[i + 1];
                x[i + 1] = t - dl[i] * x[i + 1];
            }
        }
        x[m - 1] /= dd[m - 1];
        if (m >= 2) x[m - 2] = (x[m - 2] - du[m - 2] * x[m - 1]) / dd[m - 2];
        for (int i = m - 3; i >= 0; --i) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / dd[i];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < m; ++i) x[i] /= nrm;
    }
    for (int i = 0; i < m; ++i) st->y[i] = x[i];
    const double bj = sqrt(st->beta2);
    st->theta = th;
    st->resid = bj * fabs(x[m - 1]);
    int flag = 0;
    if (st->resid <= tol) flag = 1;
    else if (bj <= breakdown) flag = 2;
    else if (last) flag = 3;
    st->flag = flag;
    if (flag == 0) st->beta[m - 1] = bj;
    else {
        st->stop = 1;
        st->m_stop = m;
    }
}

int reduction_blocks(const Ctx& ctx, long long n) {
    long long want = (n + RB * 4 - 1) / (RB * 4);
    long long cap = 4LL * std::max(ctx.num_sms, 1);
    return (int)std::max(1LL, std::min(want, cap));
}

}  // namespace

void multi_dot(Ctx& ctx, const double2* V, long long ld, int nv, const double2* w, long long n, double2* dots,
               const int* stop) {
    const int nblk = reduction_blocks(ctx, n);
    double2* partial = (double2*)ctx.workspace(WS_PARTIAL, sizeof(double2) * (size_t)nblk * KMAX_DEV);
    for (int g0 = 0; g0 < nv; g0 += DOT_GROUP) {
        const int cnt = std::min(DOT_GROUP, nv - g0);
        multi_dot_partial<<<nblk, RB, 0, ctx.stream>>>(V, ld, g0, cnt, w, n, partial, KMAX_DEV, stop);
        ctx.count_launch();
    }
    reduce_partials<<<nv, RB, 0, ctx.stream>>>(partial, nblk, KMAX_DEV, dots, stop);
    ctx.count_launch();
    ctx.check_launch("multi_dot");
}

void multi_axpy(Ctx& ctx, const double2* V, long long ld, int nv, const double2* c, double2* w, long long n,
                const int* stop) {
    multi_axpy_kernel<<<reduction_blocks(ctx, n), RB, 0, ctx.stream>>>(V, ld, nv, c, w, n, stop);
    ctx.count_launch();
    ctx.check_launch("multi_axpy");
}

void lincomb_real(Ctx& ctx, const double2* V, long long ld, int nv, const double* y, double2* out, long long n,
                  const int* nv_dev) {
    lincomb_real_kernel<<<reduction_blocks(ctx, n), RB, 0, ctx.stream>>>(V, ld, nv, y, out, n, nv_dev);
    ctx.count_launch();
    ctx.check_launch("lincomb_real");
}

void norm2_dev(Ctx& ctx, const double2* x, long long n, double* out, const int* stop) {
    const int nblk = reduction_blocks(ctx, n);
    double* partial = (double*)ctx.workspace(WS_MISC, sizeof(double) * (size_t)nblk);
    norm2_partial<<<nblk, RB, 0, ctx.stream>>>(x, n, partial, stop);
    reduce_real<<<1, RB, 0, ctx.stream>>>(partial, nblk, out, stop);
    ctx.count_launch(2);
    ctx.check_launch("norm2");
}

void scale_inv_sqrt(Ctx& ctx, double2* x, long long n, const double* nrm2) {
    scale_kernel<<<reduction_blocks(ctx, n), RB, 0, ctx.stream>>>(x, n, nrm2, nullptr, nullptr);
    ctx.count_launch();
    ctx.check_launch("scale");
}

LanczosResult lanczos_deferred_result(const double* slot) {
    // slot: theta, resid, scratch (doubles), then flag, stop, m_stop, pad (ints)
    int ints[4];
    std::memcpy(ints, slot + 3, sizeof(ints));
    LanczosResult r;
    r.theta = slot[0];
    r.n_matvec = ints[2];
    r.converged = ints[0] == 1 || ints[0] == 2;
    return r;
}

LanczosResult lanczos(Ctx& ctx, long long n, double2* x, double tol, int kmax, int restarts,
                      const std::function<void(const double2*, double2*)>& matvec, double* defer) {
    VTN_REQUIRE(kmax >= 1 && kmax <= KMAX_DEV, "krylov_max must be in [1, 64]");
    VTN_REQUIRE(restarts >= 0, "negative restart count");
    double2* V = (double2*)ctx.workspace(WS_KRYLOV, sizeof(double2) * (size_t)n * kmax);
    double2* W = (double2*)ctx.workspace(WS_VEC_W, sizeof(double2) * (size_t)n);
    LzState* st = (LzState*)ctx.workspace(WS_SCAL, sizeof(LzState));
    VTN_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(LzState), ctx.stream));
    const int nblk = reduction_blocks(ctx, n);
    // v0 = x / |x|
    norm2_dev(ctx, x, n, &st->scratch);
    scale_kernel<<<nblk, RB, 0, ctx.stream>>>(V, n, &st->scratch, nullptr, x);
    ctx.count_launch();
    LanczosResult res{0.0, 0, false};
    const double breakdown = 1e-14;
    if (defer != nullptr && restarts == 0) {
        // device-driven: all kmax steps queued; the stop flag set by ritz_kernel ends the
        // recursion on the device, and the Ritz vector is built from the first m_stop vectors
        const int* stop = &st->stop;
        for (int j = 0; j < kmax; ++j) {
            matvec(V + (size_t)j * n, W);
            int tl = ctx.tbegin(TC_LANCZOS, 0.0);
            multi_dot(ctx, V, n, j + 1, W, n, st->c1, stop);
            multi_axpy(ctx, V, n, j + 1, st->c1, W, n, stop);
            multi_dot(ctx, V, n, j + 1, W, n, st->c2, stop);
            multi_axpy(ctx, V, n, j + 1, st->c2, W, n, stop);
            norm2_dev(ctx, W, n, &st->beta2, stop);
            ritz_kernel<<<1, 32, 0, ctx.stream>>>(st, j + 1, tol, breakdown, j == kmax - 1 ? 1 : 0);
            ctx.count_launch();
            if (j + 1 < kmax) {
                scale_kernel<<<nblk, RB, 0, ctx.stream>>>(V + (size_t)(j + 1) * n, n, &st->beta2, &st->flag, W);
                ctx.count_launch();
            }
            ctx.tend(tl);
            ctx.check_launch("lanczos iteration");
        }
        lincomb_real(ctx, V, n, kmax, st->y, x, n, &st->m_stop);
        norm2_dev(ctx, x, n, &st->scratch);
        scale_inv_sqrt(ctx, x, n, &st->scratch);
        VTN_CUDA_TRY(cudaMemcpyAsync(defer, &st->theta, 3 * sizeof(double) + 4 * sizeof(int), cudaMemcpyDeviceToHost,
                                     ctx.stream));
        res.n_matvec = kmax;
        return res;
    }
    for (int rs = 0; rs <= restarts; ++rs) {
        int m = 0;
        int flag = 0;
        // the stop flag of the previous pass must not end this one (ritz_kernel returns early on it)
        VTN_CUDA_TRY(cudaMemsetAsync(&st->stop, 0, 2 * sizeof(int), ctx.stream));
        for (int j = 0; j < kmax; ++j) {
            double2* vj = V + (size_t)j * n;
            matvec(vj, W);
            res.n_matvec++;
            int tl = ctx.tbegin(TC_LANCZOS, 0.0);
            multi_dot(ctx, V, n, j + 1, W, n, st->c1);
            multi_axpy(ctx, V, n, j + 1, st->c1, W, n);
            multi_dot(ctx, V, n, j + 1, W, n, st->c2);
            multi_axpy(ctx, V, n, j + 1, st->c2, W, n);
            norm2_dev(ctx, W, n, &st->beta2);
            ritz_kernel<<<1, 32, 0, ctx.stream>>>(st, j + 1, tol, breakdown, j == kmax - 1 ? 1 : 0);
            ctx.count_launch();
            if (j + 1 < kmax) {
                // v_{j+1} = w / beta_j unless the iteration stops here
                scale_kernel<<<nblk, RB, 0, ctx.stream>>>(V + (size_t)(j + 1) * n, n, &st->beta2, &st->flag, W);
                ctx.count_launch();
            }
            ctx.tend(tl);
            ctx.check_launch("lanczos iteration");
            VTN_CUDA_TRY(cudaMemcpyAsync(ctx.pinned, &st->theta, 3 * sizeof(double) + sizeof(int),
                                         cudaMemcpyDeviceToHost, ctx.stream));
            ctx.sync();
            res.theta = ctx.pinned[0];
            std::memcpy(&flag, &ctx.pinned[3], sizeof(int));
            m = j + 1;
            if (flag != 0) break;
        }
        // x = V y, normalised
        lincomb_real(ctx, V, n, m, st->y, x, n);
        norm2_dev(ctx, x, n, &st->scratch);
        scale_inv_sqrt(ctx, x, n, &st->scratch);
        if (flag == 1 || flag == 2) {
            res.converged = true;
            break;
        }
        if (rs < restarts) {
            VTN_CUDA_TRY(cudaMemcpyAsync(V, x, sizeof(double2) * (size_t)n, cudaMemcpyDeviceToDevice, ctx.stream));
        }
    }
    return res;
}

}  // namespace vtn
