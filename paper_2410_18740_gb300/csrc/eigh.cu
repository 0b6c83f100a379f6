// FP64 truncation eigensolver: the reduced density matrix rho of a two-site tensor,
// its largest k eigenpairs, and the split of the tensor into a canonical site and the
// new centre.  Every step runs on the GPU:
//
//  1. rho = T T^dag (or T^dag T) by the complex GEMM.
//  2. Householder tridiagonalisation of the Hermitian rho (Golub & Van Loan, Sec. 8.3.1):
//     for each column a Hermitian reflector H = I - tau v v^dag with H x = beta e_1,
//     p = tau A v, w = p - (tau/2)(v^dag p) v, A <- A - v w^dag - w v^dag.  The complex
//     sub-diagonal is made real by a diagonal phase similarity.
//  3. The k largest eigenvalues of the real tridiagonal by bisection on Sturm counts,
//     one CTA per eigenvalue evaluating 128 points per round (multisection), to an
//     absolute accuracy of 2 u |T|.
//  4. Eigenvectors by inverse iteration with a pivoted tridiagonal LU, one thread per
//     eigenvector, three iterations from deterministic pseudo-random starts.
//  5. Orthonormalisation of the k vectors: one Cholesky-QR pass when they are already
//     nearly orthonormal, else shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto,
//     Yanagisawa, SIAM J. Sci. Comput. 2020): one shifted and two plain passes.  Column
//     order is preserved, so the span of the leading j vectors is that of the j largest
//     eigenvalues.
//  6. Back-transformation through the reflectors (compact WY blocks) and the phases, one
//     CTA per vector.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr double EPS = 2.220446049250313e-16;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        r = warp_sum(r);
        if (lane == 0) sh[32] = r;
    }
    __syncthreads();
    r = sh[32];
    __syncthreads();
    return r;  // valid in every thread
}

struct EigSmall {
    double* diag;   // [n]
    double* offd;   // [n]
    double* tau;    // [n]
    double* lam;    // [n]
    double2* e;     // [n]
    double2* ph;    // [n]
    double2* p;     // [n]
    double2* w;     // [n]
    double* scal;   // [8]: trace, status
    double* bsq;    // [n]: offd^2 (Sturm counts)
};

// ---------------------------------------------------------------- Householder steps
__global__ void __launch_bounds__(1024) hh_reflector(const double2* __restrict__ A, int n, int k,
                                                     double2* __restrict__ H, EigSmall s) {
    __shared__ double sh[33];
    const int m = n - k - 1;
    const double2* row = A + (long long)k * n + (k + 1);  // conj of column k below the diagonal
    double a2 = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 v = row[i];
        a2 += v.x * v.x + v.y * v.y;
    }
    a2 = block_sum(a2, sh);
    const double2 x0 = make_double2(row[0].x, -row[0].y);
    const double ax0 = hypot(x0.x, x0.y);
    double2* v = H + (long long)k * n;
    if (a2 == 0.0) {
        for (int i = threadIdx.x; i < m; i += blockDim.x) v[i] = make_double2(0.0, 0.0);
        if (threadIdx.x == 0) {
            s.tau[k] = 0.0;
            s.e[k] = make_double2(0.0, 0.0);
            s.diag[k] = A[(long long)k * n + k].x;
        }
        return;
    }
    const double alpha = sqrt(a2);
    const double2 phi = ax0 > 0.0 ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        double2 xi = make_double2(row[i].x, -row[i].y);
        if (i == 0) xi = make_double2(x0.x + phi.x * alpha, x0.y + phi.y * alpha);
        v[i] = xi;
    }
    if (threadIdx.x == 0) {
        s.tau[k] = 1.0 / (alpha * (alpha + ax0));  // 2 / (v^dag v), v^dag v = 2 alpha (alpha + |x0|)
        s.e[k] = make_double2(-phi.x * alpha, -phi.y * alpha);
        s.diag[k] = A[(long long)k * n + k].x;
    }
}

// p_i = tau sum_j A[k+1+i][k+1+j] v_j, one warp per row
__global__ void __launch_bounds__(256) hh_matvec(const double2* __restrict__ A, int n, int k,
                                                 const double2* __restrict__ H, EigSmall s) {
    const int m = n - k - 1;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= m) return;
    const double tau = s.tau[k];
    const double2* row = A + (long long)(k + 1 + warp) * n + (k + 1);
    const double2* v = H + (long long)k * n;
    double re = 0.0, im = 0.0;
    for (int j = lane; j < m; j += 32) {
        const double2 a = row[j], b = v[j];
        re += a.x * b.x - a.y * b.y;
        im += a.x * b.y + a.y * b.x;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) s.p[warp] = make_double2(tau * re, tau * im);
}

// K = (tau/2) Re(v^dag p);  w = p - K v
__global__ void __launch_bounds__(1024) hh_w(int n, int k, const double2* __restrict__ H, EigSmall s) {
    __shared__ double sh[33];
    const int m = n - k - 1;
    const double2* v = H + (long long)k * n;
    double acc = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double2 a = v[i], b = s.p[i];
        acc += a.x * b.x + a.y * b.y;
    }
    acc = block_sum(acc, sh);
    const double K = 0.5 * s.tau[k] * acc;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const double2 a = v[i], b = s.p[i];
        s.w[i] = make_double2(b.x - K * a.x, b.y - K * a.y);
    }
}

// A22 -= v w^dag + w v^dag
__global__ void __launch_bounds__(256) hh_rank2(double2* __restrict__ A, int n, int k, const double2* __restrict__ H,
                                                EigSmall s) {
    const int m = n - k - 1;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)m * m) return;
    const int i = (int)(t / m), j = (int)(t % m);
    const double2* v = H + (long long)k * n;
    const double2 vi = v[i], vj = v[j], wi = s.w[i], wj = s.w[j];
    // v_i conj(w_j) + w_i conj(v_j)
    const double re = vi.x * wj.x + vi.y * wj.y + wi.x * vj.x + wi.y * vj.y;
    const double im = vi.y * wj.x - vi.x * wj.y + wi.y * vj.x - wi.x * vj.y;
    double2* a = A + (long long)(k + 1 + i) * n + (k + 1 + j);
    a->x -= re;
    a->y -= im;
}

// tail of the tridiagonal (the real off-diagonal and phases follow in tri_phases)
__global__ void tri_finalize(const double2* __restrict__ A, int n, EigSmall s) {
    if (threadIdx.x != 0) return;
    if (n >= 2) {
        s.diag[n - 2] = A[(long long)(n - 2) * n + (n - 2)].x;
        const double2 t = A[(long long)(n - 2) * n + (n - 1)];
        s.e[n - 2] = make_double2(t.x, -t.y);  // A[n-1][n-2] = conj(A[n-2][n-1])
    }
    s.diag[n - 1] = A[(long long)(n - 1) * n + (n - 1)].x;
}

// Real symmetric form of the Hermitian tridiagonal: offd_i = |e_i| and the phases
// ph_0 = 1, ph_{i+1} = ph_i e_i / |e_i| (D^dag T D is real for D = diag(ph)).  The phases
// are an exclusive prefix product, computed as a block scan: each thread multiplies out a
// contiguous segment, the segment products are scanned in shared memory, then each
// segment is rewritten from its prefix.  One CTA of TP_THREADS threads.
constexpr int TP_THREADS = 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(TP_THREADS) tri_phases(int n, EigSmall s) {
    __shared__ double2 scan[TP_THREADS];
    const int t = threadIdx.x;
    const int seg = (n + TP_THREADS - 1) / TP_THREADS;
    const int i0 = min(n, t * seg), i1 = min(n, i0 + seg);
    // unit factors u_i = e_i / |e_i| (1 for e_i = 0 and for the last index)
    double2 prod = make_double2(1.0, 0.0);
    for (int i = i0; i < i1; ++i) {
        double2 u = make_double2(1.0, 0.0);
        double r = 0.0;
        if (i + 1 < n) {
            const double2 ei = s.e[i];
            r = hypot(ei.x, ei.y);
            if (r > 0.0) {
                const double inv = 1.0 / r;
                u = make_double2(ei.x * inv, ei.y * inv);
            }
        }
        s.offd[i] = r;
        s.bsq[i] = r * r;
        s.ph[i] = u;  // scratch: u_i, replaced by the phase below
        prod = cmul(prod, u);
    }
    scan[t] = prod;
    __syncthreads();  // also publishes offd for the Gershgorin pass below
    for (int off = 1; off < TP_THREADS; off <<= 1) {
        const double2 other = t >= off ? scan[t - off] : make_double2(1.0, 0.0);
        __syncthreads();
        scan[t] = cmul(other, scan[t]);
        __syncthreads();
    }
    double2 cur = t > 0 ? scan[t - 1] : make_double2(1.0, 0.0);
    for (int i = i0; i < i1; ++i) {
        const double2 u = s.ph[i];
        s.ph[i] = cur;
        cur = cmul(cur, u);
    }
    // Gershgorin interval [gl, gu] and max_i |a_i| + |b_{i-1}| + |b_i| -> scal[4..6]
    double gl = 1e308, gu = -1e308, tn = 0.0;
    for (int i = i0; i < i1; ++i) {
        const double r = (i > 0 ? s.offd[i - 1] : 0.0) + s.offd[i];
        const double ai = s.diag[i];
        gl = fmin(gl, ai - r);
        gu = fmax(gu, ai + r);
        tn = fmax(tn, fabs(ai) + r);
    }
    __shared__ double mm[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
        gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
    }
    if ((t & 31) == 0) {
        mm[0][t >> 5] = gl;
        mm[1][t >> 5] = gu;
        mm[2][t >> 5] = tn;
    }
    __syncthreads();
    if (t == 0) {
        for (int w = 1; w < TP_THREADS / 32; ++w) {
            gl = fmin(gl, mm[0][w]);
            gu = fmax(gu, mm[1][w]);
            tn = fmax(tn, mm[2][w]);
        }
        s.scal[4] = gl;
        s.scal[5] = gu;
        s.scal[6] = tn;
    }
}

// ---------------------------------------------------------------- persistent tridiagonalisation
// One cooperative launch for the whole Householder reduction, one column per step and one
// grid barrier per step.
//
// GB300 issues one FP64 warp instruction per 64 cycles per SM sub-partition whatever the
// number of active lanes, and a dependent FP64 instruction waits about as long, so the
// kernel keeps every FP64 instruction 32 lanes wide and the per-step dependency chain short:
//  B(k)   the rank-2 update of step k-1 is applied lazily while p = tau A v streams the
//         trailing block.  A warp owns 32 consecutive COLUMNS i (coalesced loads of A[j][i])
//         and walks a slice of the rows j, accumulating (A v)_i = sum_j conj(A[j][i]) v_j in
//         its lanes (A is Hermitian), so no per-row reductions are needed.  The CTAs that
//         share a column chunk each write a partial; the last of them to finish (an atomic
//         arrival count) sums the partials in a fixed order into p.
//  barrier
//  C(k)+A(k+1), redundantly in every CTA: K = (tau/2) Re(v^dag p), w = p - K v becomes the
//         pending pair, and in the same pass row k+1 of the current matrix is formed with
//         the pending update applied; its norm gives the next reflector.
// Data written by other CTAs is read with ld.global.cg (L2, not L1).
struct GridBar {
    unsigned int count;  // arrivals, monotonic over the launch
    unsigned int pad0;
    int error;           // set by a CTA whose wait timed out; read by the host
    int pad1;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier number `epoch` (0, 1, 2, ... in every CTA): each CTA adds its arrival to a
// monotonic counter (fire-and-forget reduction) and polls it until it reaches
// (epoch + 1) * nblocks (about 1.5 us for 152 CTAs on GB300; a CTA that releases the others
// through a second word takes about 2.5 us).  Waits are bounded (2 s): a CTA that gives up
// sets bar->error, which the other pollers check every 256 polls; all CTAs then return
// false and the kernel exits.
__device__ bool grid_sync(GridBar* bar, unsigned int nblocks, unsigned int epoch) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_add(&bar->count, 1u);
        const unsigned target = (epoch + 1u) * nblocks;
        bool ok = true;
        const unsigned long long t0 = global_ns();
        unsigned polls = 0;
        while (ld_acquire_u32(&bar->count) < target) {
            if ((++polls & 255u) == 0) {
                if (*(volatile int*)&bar->error != 0 || global_ns() - t0 > 2000000000ull) {
                    atomicExch(&bar->error, 1);
                    ok = false;
                    break;
                }
            }
        }
        __threadfence();
        ok_sh = ok ? 1 : 0;
    }
    __syncthreads();
    return ok_sh != 0;
}

__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

constexpr int TRI_THREADS = 512;
constexpr int TRI_NW = TRI_THREADS / 32;
constexpr int TRI_MAX_N = 4096;
constexpr int TRI_MAX_CHUNKS = TRI_MAX_N / 32;
constexpr int TRI_UNROLL = 4;  // rows in flight per warp

struct TriBufs {
    double2* part;      // [2][nb][n] partial products (double-buffered by step parity)
    double2* p;         // [2][n] p = tau A v
    unsigned* arrive;   // [2][TRI_MAX_CHUNKS] arrivals per column chunk (zero at launch)
};

// x -= a conj(b) + c conj(d) for complex a..d, as 8 FMAs
__device__ __forceinline__ double2 sub_two_cmulc(double2 x, double2 a, double2 b, double2 c, double2 d) {
    x.x = fma(-a.x, b.x, x.x);
    x.x = fma(-a.y, b.y, x.x);
    x.x = fma(-c.x, d.x, x.x);
    x.x = fma(-c.y, d.y, x.x);
    x.y = fma(-a.y, b.x, x.y);
    x.y = fma(a.x, b.y, x.y);
    x.y = fma(-c.y, d.x, x.y);
    x.y = fma(c.x, d.y, x.y);
    return x;
}

constexpr int TRI_MAX_CPL = 2;  // columns per lane in the trailing pass

// chunks C of 32*cpl columns, row slices CS per chunk; work units C*CS over nb CTAs
__device__ __forceinline__ void tri_layout(int m, int nb, int cpl, int& C, int& CS) {
    const int w = 32 * cpl;
    C = (m + w - 1) / w;
    CS = max(1, min(C <= nb ? nb / C : 1, (m + TRI_NW - 1) / TRI_NW));
}

// modelled time of a trailing pass: passes over the CTAs x rows of the slowest warp x columns per lane
__device__ __forceinline__ int tri_pass_cost(int m, int nb, int cpl) {
    int C, CS;
    tri_layout(m, nb, cpl, C, CS);
    const int passes = (C * CS + nb - 1) / nb;
    const int rows = (m + CS * TRI_NW - 1) / (CS * TRI_NW);
    return passes * rows * cpl;
}

// Trailing pass of step k: pending rank-2 update of the trailing block fused with (A v).  Work
// unit u = (column chunk c = u mod C of 32*CPL columns, row slice cs = u / C of CS); CTA b
// takes units b, b + nb, ...; warp w walks the rows k+1 + cs*NW + w + t*CS*NW, lane l owns the
// columns c*32*CPL + q*32 + l (q < CPL).  The CTAs of a chunk each write one partial (A v) per
// column; the last to arrive sums them in slice order into p = tau A v.
template <int CPL>
__device__ void tri_pass(double2* __restrict__ A, int n, int k, int m, int nb, bool have_prev,
                         const double2* vprev, const double2* wprev, const double2* vcur, double tau,
                         double2* pk, double2* pfin, unsigned* arrive, double2* colred, int& last_sh) {
    constexpr int U = TRI_UNROLL / CPL;  // rows in flight per warp
    constexpr int LD = TRI_MAX_CPL * 32;  // colred row stride
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int C, CS;
    tri_layout(m, nb, CPL, C, CS);
    for (int unit = (int)blockIdx.x; unit < C * CS; unit += nb) {
        const int c = unit % C, cs = unit / C;
        int il[CPL], col[CPL];
        bool ok[CPL];
        double2 vpi[CPL], wpi[CPL];
        double accx[CPL], accy[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            il[q] = c * 32 * CPL + q * 32 + lane;  // local column index (0..m-1)
            ok[q] = il[q] < m;
            col[q] = k + 1 + (ok[q] ? il[q] : 0);
            // column factors of a_ji -= vp_j conj(wp_i) + wp_j conj(vp_i)
            vpi[q] = make_double2(0.0, 0.0);
            wpi[q] = make_double2(0.0, 0.0);
            if (have_prev && ok[q]) {
                vpi[q] = vprev[col[q] - k];
                wpi[q] = wprev[col[q] - k];
            }
            accx[q] = accy[q] = 0.0;
        }
        const int stride = CS * TRI_NW;
        int j = k + 1 + cs * TRI_NW + warp;
        for (; j + (U - 1) * stride < n; j += U * stride) {
            double2 a[U][CPL];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    a[u][q] = ok[q] ? __ldcg(&A[(long long)(j + u * stride) * n + col[q]]) : make_double2(0.0, 0.0);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int jj = j + u * stride;
                const double2 v = vcur[jj - k - 1];
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    if (have_prev) {
                        a[u][q] = sub_two_cmulc(a[u][q], vprev[jj - k], wpi[q], wprev[jj - k], vpi[q]);
                        if (ok[q]) A[(long long)jj * n + col[q]] = a[u][q];
                    }
                    accx[q] = fma(a[u][q].x, v.x, accx[q]);
                    accx[q] = fma(a[u][q].y, v.y, accx[q]);
                    accy[q] = fma(a[u][q].x, v.y, accy[q]);
                    accy[q] = fma(-a[u][q].y, v.x, accy[q]);
                }
            }
        }
        for (; j < n; j += stride) {
            const double2 v = vcur[j - k - 1];
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                double2 a = ok[q] ? __ldcg(&A[(long long)j * n + col[q]]) : make_double2(0.0, 0.0);
                if (have_prev) {
                    a = sub_two_cmulc(a, vprev[j - k], wpi[q], wprev[j - k], vpi[q]);
                    if (ok[q]) A[(long long)j * n + col[q]] = a;
                }
                accx[q] = fma(a.x, v.x, accx[q]);
                accx[q] = fma(a.y, v.y, accx[q]);
                accy[q] = fma(a.x, v.y, accy[q]);
                accy[q] = fma(-a.y, v.x, accy[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < CPL; ++q) colred[warp * LD + q * 32 + lane] = make_double2(accx[q], accy[q]);
        __syncthreads();
#pragma unroll
        for (int h = TRI_NW / 2; h >= 2; h >>= 1) {  // tree over the warps' partials
            if (warp < h) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const double2 o = colred[(warp + h) * LD + q * 32 + lane];
                    colred[warp * LD + q * 32 + lane].x += o.x;
                    colred[warp * LD + q * 32 + lane].y += o.y;
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const double2 a0 = colred[q * 32 + lane], a1 = colred[LD + q * 32 + lane];
                if (ok[q]) pk[(long long)cs * n + il[q]] = make_double2(a0.x + a1.x, a0.y + a1.y);
            }
            __threadfence();
        }
        __syncthreads();
        // the last CTA of this chunk sums its CS partials in slice order (warp q: columns q*32..)
        if (threadIdx.x == 0) {
            __threadfence();
            last_sh = atomicAdd(&arrive[c], 1u) == (unsigned)(CS - 1);
        }
        __syncthreads();
        if (last_sh && warp < CPL) {
            __threadfence();
            const int ilq = c * 32 * CPL + warp * 32 + lane;
            if (ilq < m) {
                double sx = 0.0, sy = 0.0;
                for (int s2 = 0; s2 < CS; ++s2) {
                    const double2 pp = __ldcg(&pk[(long long)s2 * n + ilq]);
                    sx += pp.x;
                    sy += pp.y;
                }
                pfin[ilq] = make_double2(tau * sx, tau * sy);
            }
            if (warp == 0 && lane == 0) arrive[c] = 0u;  // reused two steps later, after two barriers
        }
        __syncthreads();  // colred and last_sh are reused by the next unit
    }
}

__global__ void __launch_bounds__(TRI_THREADS) tridiag_persistent(double2* __restrict__ A, int n,
                                                                  double2* __restrict__ H, EigSmall s,
                                                                  TriBufs tb, GridBar* bar) {
    extern __shared__ double2 sm[];
    // three rotating vectors: pending pair (vprev, wprev) of the previous step and the
    // reflector vcur of this step; all local to the trailing block (index t <-> row k+1+t
    // for vcur, row k+t for the pending pair)
    double2* vprev = sm;
    double2* wprev = sm + n;
    double2* vcur = sm + 2 * n;
    __shared__ double red[33];
    __shared__ double tau_sh, dk_sh;
    __shared__ double2 p0_sh;
    __shared__ int last_sh;
    __shared__ double2 colred[TRI_NW][TRI_MAX_CPL * 32];
    const int nb = (int)gridDim.x;
    bool have_prev = false;
    // row 0 (no pending update): x = conj(A[0][1..n-1])
    double a2 = 0.0;
    for (int t = threadIdx.x; t < n - 1; t += blockDim.x) {
        const double2 a = __ldcg(&A[1 + t]);
        const double2 x = make_double2(a.x, -a.y);
        vcur[t] = x;
        a2 = fma(x.x, x.x, fma(x.y, x.y, a2));
    }
    if (threadIdx.x == 0) dk_sh = __ldcg(&A[0]).x;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        // ---- reflector for column k from x = vcur (norm^2 a2)
        a2 = block_sum(a2, red);
        if (threadIdx.x == 0) {
            // alpha = |x|, phi = x0 / |x0|: v0 = x0 + phi alpha, beta = -phi alpha,
            // tau = 1 / (alpha (alpha + |x0|)); with few FP64 instructions (two reciprocal
            // square roots, one division)
            const double2 x0 = vcur[0];
            const double q0 = fma(x0.x, x0.x, x0.y * x0.y);
            double tau = 0.0;
            double2 beta = make_double2(0.0, 0.0);
            if (a2 > 0.0) {
                const double ra = rsqrt(a2);
                const double alpha = a2 * ra;
                double2 phia;  // phi * alpha
                double ax0 = 0.0;
                if (q0 > 0.0) {
                    const double rq = rsqrt(q0);
                    ax0 = q0 * rq;
                    const double sc = alpha * rq;
                    phia = make_double2(x0.x * sc, x0.y * sc);
                } else {
                    phia = make_double2(alpha, 0.0);
                }
                vcur[0] = make_double2(x0.x + phia.x, x0.y + phia.y);
                tau = 1.0 / fma(alpha, ax0, a2);
                beta = make_double2(-phia.x, -phia.y);
            }
            tau_sh = tau;
            if (blockIdx.x == 0) {
                s.diag[k] = dk_sh;
                s.tau[k] = tau;
                s.e[k] = beta;
            }
        }
        __syncthreads();
        const double tau = tau_sh;
        if (tau == 0.0)
            for (int t = threadIdx.x; t < m; t += blockDim.x) vcur[t] = make_double2(0.0, 0.0);
        __syncthreads();
        if (blockIdx.x == 0)
            for (int t = threadIdx.x; t < m; t += blockDim.x) H[(long long)k * n + t] = vcur[t];
        // ---- B: 32 or 64 columns per chunk (1 or 2 per lane), whichever leaves the slowest
        //      warp fewer rows x columns this step (the same choice in every CTA)
        double2* pk = tb.part + (long long)(k & 1) * nb * n;
        double2* pfin = tb.p + (long long)(k & 1) * n;
        unsigned* arrive = tb.arrive + (k & 1) * TRI_MAX_CHUNKS;
        if (tri_pass_cost(m, nb, 2) < tri_pass_cost(m, nb, 1))
            tri_pass<2>(A, n, k, m, nb, have_prev, vprev, wprev, vcur, tau, pk, pfin, arrive, &colred[0][0], last_sh);
        else
            tri_pass<1>(A, n, k, m, nb, have_prev, vprev, wprev, vcur, tau, pk, pfin, arrive, &colred[0][0], last_sh);
        if (!grid_sync(bar, (unsigned)nb, (unsigned)k)) return;
        // ---- C(k): K = (tau/2) Re(v^dag p); p parked in wprev (its old content is spent)
        const bool next = k + 3 < n;  // another reflector follows
        double dot = 0.0;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const double2 p = __ldcg(&pfin[t]), v = vcur[t];
            if (next && t >= 1) vprev[t - 1] = __ldcg(&A[(long long)(k + 1) * n + (k + 1 + t)]);  // row k+1, raw
            wprev[t] = p;
            if (t == 0) p0_sh = p;
            dot = fma(v.x, p.x, fma(v.y, p.y, dot));
        }
        dot = block_sum(dot, red);
        const double K = 0.5 * tau * dot;
        // rotate: the pending pair becomes (v_k, w_k); the free buffer takes row k+1
        double2* vnew = vcur;
        double2* wnew = wprev;
        double2* xnext = vprev;
        const double2 v0 = vnew[0];
        const double2 w0 = make_double2(fma(-K, v0.x, p0_sh.x), fma(-K, v0.y, p0_sh.y));
        a2 = 0.0;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const double2 p = wnew[t], v = vnew[t];
            const double2 w = make_double2(fma(-K, v.x, p.x), fma(-K, v.y, p.y));
            wnew[t] = w;
            if (next && t >= 1) {
                // A(k+1): row k+1 (prefetched into xnext) with the pending update, x = conj(row)
                double2 a = xnext[t - 1];
                a = sub_two_cmulc(a, v0, w, w0, v);
                const double2 x = make_double2(a.x, -a.y);
                xnext[t - 1] = x;
                a2 = fma(x.x, x.x, fma(x.y, x.y, a2));
            }
        }
        if (threadIdx.x == 0 && next) dk_sh = __ldcg(&A[(long long)(k + 1) * n + (k + 1)]).x - 2.0 * (v0.x * w0.x + v0.y * w0.y);
        vprev = vnew;
        wprev = wnew;
        vcur = xnext;
        have_prev = true;
        __syncthreads();
    }
    // ---- tail: last 2 x 2 block with the pending update applied
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (n >= 2) {
            double2 a00 = __ldcg(&A[(long long)(n - 2) * n + (n - 2)]);
            double2 a11 = __ldcg(&A[(long long)(n - 1) * n + (n - 1)]);
            double2 a01 = __ldcg(&A[(long long)(n - 2) * n + (n - 1)]);
            if (have_prev) {
                a00.x -= 2.0 * (vprev[0].x * wprev[0].x + vprev[0].y * wprev[0].y);
                a11.x -= 2.0 * (vprev[1].x * wprev[1].x + vprev[1].y * wprev[1].y);
                const double2 u = cmulc(vprev[0], wprev[1]), v = cmulc(wprev[0], vprev[1]);
                a01.x -= u.x + v.x;
                a01.y -= u.y + v.y;
            }
            s.diag[n - 2] = a00.x;
            s.diag[n - 1] = a11.x;
            s.e[n - 2] = make_double2(a01.x, -a01.y);
        } else {
            s.diag[0] = __ldcg(&A[0]).x;
        }
    }
}

// ---------------------------------------------------------------- lower-triangle form
// The same reduction with only the lower triangle (row >= column) of the trailing block kept up
// to date.  Each stored element a = A[j][c] takes the pending rank-2 update once (8 FMAs) and
// feeds both halves of p = A v: conj(a) v_j to p_c (the column part, summed in the lanes as in
// tri_pass) and, for j > c, a v_c to p_j (the row part, 4 FMAs): 8 FP64 FMAs per element of the
// full trailing block and column instead of 12.  A warp takes TRL_RB rows at a time; their row
// parts are combined across the lanes by a reduce-scatter (6 complex additions per lane for 4
// rows) and written per (column chunk, row); the column parts of a CTA's rows of a chunk are
// written per (CTA slot of the chunk, column).  The pass also accumulates v^dag A v: with
// (A v)_j = (column part)_j + (row part)_j it is the real part of sum_j conj(v_j) (row part)_j
// plus sum_c conj(v_c) (column part)_c, and both sums split over the CTAs' rows and slots, so
// each CTA adds its own share and writes one partial.  After a grid barrier every CTA sums the
// partials in one fixed order, so K = (tau/2) v^dag p = (tau^2/2) v^dag A v is the same in every
// CTA, and the CTAs finalise their slices of 32 rows: p (the slots of the row's chunk plus the
// row parts of chunks 0 .. row/W, summed by warps over interleaved terms and then over the warps
// in order: deterministic), w = p - K v and the next reflector's column k+1 (read as the stored
// half) with step k's update, with partial sums of its squared norm.  After a second barrier
// every CTA only loads w and that column: no per-element arithmetic is repeated in every CTA.
constexpr int TRL_THREADS = 256;
constexpr int TRL_NW = TRL_THREADS / 32;
constexpr int TRL_RB = 4;  // rows per warp batch

struct TriBufsL {
    double2* part;  // [2][nb][n] column parts per CTA slot of a chunk
    double2* prow;  // [2][TRI_MAX_CHUNKS][n] row parts per column chunk
    double2* w;     // [2][n] w = p - K v, p = tau A v
    double2* x;     // [n] next column below its diagonal, with step k's update
    double* dot;    // [nb] per-CTA partials of v^dag A v
    double* a2;     // [nb] per-CTA partials of |x|^2
};

// x (complex, per lane) summed over the lanes that share bits >= 2 of the lane index, for 4 rows:
// on return r[0] of lane l holds the sum of row (l & 3) over all 32 lanes
__device__ __forceinline__ double2 shfl_xor_d2(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

__device__ __forceinline__ double2 reduce_scatter4(double2 r[TRL_RB], int lane) {
    // stage 1: lanes with bit 1 keep rows 2, 3; the others rows 0, 1
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const bool up = (lane & 2) != 0;
        const double2 send = up ? r[t] : r[t + 2];
        const double2 keep = up ? r[t + 2] : r[t];
        const double2 got = shfl_xor_d2(send, 2);
        r[t] = make_double2(keep.x + got.x, keep.y + got.y);
    }
    // stage 2: bit 0 picks row 2b1 + 1 or 2b1
    {
        const bool up = (lane & 1) != 0;
        const double2 send = up ? r[0] : r[1];
        const double2 keep = up ? r[1] : r[0];
        const double2 got = shfl_xor_d2(send, 1);
        r[0] = make_double2(keep.x + got.x, keep.y + got.y);
    }
    // the row is lane & 3; add over lane bits 2..4
#pragma unroll
    for (int o = 4; o <= 16; o <<= 1) {
        const double2 got = shfl_xor_d2(r[0], o);
        r[0] = make_double2(r[0].x + got.x, r[0].y + got.y);
    }
    return r[0];
}

// Trailing pass of step k, lower triangle.  The rows of the chunks, in blocks of TRL_IB rows (item
// i of chunk c: local rows c W + TRL_IB (i - items[c]) ...), are split into nb equal contiguous
// ranges, one per CTA; a CTA's range covers one or more chunk segments.  In a segment warp w walks
// the rows r0 + w + t NW; lane l owns the columns c W + q 32 + l (q < CPL).  The segment's column
// parts are summed over the warps and written to slot (CTA - first CTA of the chunk).  dacc (per
// thread) collects this CTA's share of v^dag A v.
constexpr int TRL_IB = 8;

// first item of CTA b's range, and the CTA whose range holds item i (the largest b with
// start(b) <= i); b T and (i + 1) nb stay below 2^32 for n <= TRI_MAX_N and nb <= 1024
__device__ __forceinline__ int tri_item_start(int b, int T, int nb) {
    return (int)(((unsigned)b * (unsigned)T) / (unsigned)nb);
}
__device__ __forceinline__ int tri_item_owner(int i, int T, int nb) {
    return (int)(((unsigned)(i + 1) * (unsigned)nb - 1u) / (unsigned)T);
}

template <int CPL>
__device__ void tri_pass_lower(double2* __restrict__ A, int n, int k, int m, int nb, bool have_prev,
                               const double2* vprev, const double2* wprev, const double2* vcur, double2* pk,
                               double2* prow, double2* colred, const int* items, int C, double& dacc) {
    constexpr int W = 32 * CPL;
    constexpr int LD = TRI_MAX_CPL * 32;  // colred row stride
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int T = items[C];
    const int nbe = min(nb, T);  // CTAs with a non-empty range (every range below nbe holds an item)
    const int b = (int)blockIdx.x;
    if (b >= nbe) return;
    const int i0 = tri_item_start(b, T, nbe), i1 = tri_item_start(b + 1, T, nbe);
    int c = 0;
    {
        int lo = 0, hi = C;  // items[lo] <= i0 < items[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (items[mid] <= i0) lo = mid;
            else hi = mid;
        }
        c = lo;
    }
    for (; c < C && items[c] < i1; ++c) {
        const int lo_i = max(i0, items[c]), hi_i = min(i1, items[c + 1]);
        const int r0 = c * W + TRL_IB * (lo_i - items[c]);
        const int r1 = min(m, c * W + TRL_IB * (hi_i - items[c]));
        const int slot = b - tri_item_owner(items[c], T, nbe);
        int il[CPL];
        bool ok[CPL];
        double2 vpi[CPL], wpi[CPL], vci[CPL];
        double accx[CPL], accy[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            il[q] = c * W + q * 32 + lane;
            ok[q] = il[q] < m;
            vpi[q] = make_double2(0.0, 0.0);
            wpi[q] = make_double2(0.0, 0.0);
            if (have_prev && ok[q]) {
                vpi[q] = vprev[il[q] + 1];
                wpi[q] = wprev[il[q] + 1];
            }
            vci[q] = ok[q] ? vcur[il[q]] : make_double2(0.0, 0.0);
            accx[q] = accy[q] = 0.0;
        }
        constexpr int S = TRL_NW;
        for (int jb = r0 + warp; jb < r1; jb += TRL_RB * S) {
            double2 a[TRL_RB][CPL];
            // loads first (TRL_RB * CPL in flight), then the updates, stores and sums
#pragma unroll
            for (int r = 0; r < TRL_RB; ++r) {
                const int j = jb + r * S;
#pragma unroll
                for (int q = 0; q < CPL; ++q)
                    a[r][q] = (j < r1 && ok[q] && j >= il[q])
                                  ? __ldcg(&A[(long long)(k + 1 + j) * n + (k + 1 + il[q])])
                                  : make_double2(0.0, 0.0);
            }
            double2 racc[TRL_RB];
#pragma unroll
            for (int r = 0; r < TRL_RB; ++r) {
                const int j = jb + r * S;
                racc[r] = make_double2(0.0, 0.0);
                if (j >= r1) continue;  // warp-uniform
                const double2 v = vcur[j];
                double2 vpj = make_double2(0.0, 0.0), wpj = make_double2(0.0, 0.0);
                if (have_prev) {
                    vpj = vprev[j + 1];
                    wpj = wprev[j + 1];
                }
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    if (!(ok[q] && j >= il[q])) continue;
                    double2 x = a[r][q];
                    if (have_prev) {
                        x = sub_two_cmulc(x, vpj, wpi[q], wpj, vpi[q]);
                        A[(long long)(k + 1 + j) * n + (k + 1 + il[q])] = x;
                    }
                    // column part: conj(x) v_j
                    accx[q] = fma(x.x, v.x, accx[q]);
                    accx[q] = fma(x.y, v.y, accx[q]);
                    accy[q] = fma(x.x, v.y, accy[q]);
                    accy[q] = fma(-x.y, v.x, accy[q]);
                    // row part: x v_c (strictly below the diagonal)
                    if (j > il[q]) {
                        racc[r].x = fma(x.x, vci[q].x, racc[r].x);
                        racc[r].x = fma(-x.y, vci[q].y, racc[r].x);
                        racc[r].y = fma(x.x, vci[q].y, racc[r].y);
                        racc[r].y = fma(x.y, vci[q].x, racc[r].y);
                    }
                }
            }
            const double2 rs = reduce_scatter4(racc, lane);
            const int jr = jb + (lane & 3) * S;
            if (lane < TRL_RB && jr < r1) {
                prow[(long long)c * n + jr] = rs;
                const double2 vj = vcur[jr];
                dacc = fma(vj.x, rs.x, fma(vj.y, rs.y, dacc));  // Re(conj(v_j) rs)
            }
        }
        // column parts of this segment: tree over the warps; warp 0 writes the slot and adds
        // Re(conj(v_c) s_c) to this CTA's share of v^dag A v
#pragma unroll
        for (int q = 0; q < CPL; ++q) colred[warp * LD + q * 32 + lane] = make_double2(accx[q], accy[q]);
        __syncthreads();
#pragma unroll
        for (int h = TRL_NW / 2; h >= 2; h >>= 1) {
            if (warp < h) {
#pragma unroll
                for (int q = 0; q < CPL; ++q) {
                    const double2 o = colred[(warp + h) * LD + q * 32 + lane];
                    colred[warp * LD + q * 32 + lane].x += o.x;
                    colred[warp * LD + q * 32 + lane].y += o.y;
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
#pragma unroll
            for (int q = 0; q < CPL; ++q) {
                const double2 a0 = colred[q * 32 + lane], a1 = colred[LD + q * 32 + lane];
                const double2 sq = make_double2(a0.x + a1.x, a0.y + a1.y);
                if (ok[q]) {
                    pk[(long long)slot * n + il[q]] = sq;
                    dacc = fma(vci[q].x, sq.x, fma(vci[q].y, sq.y, dacc));  // Re(conj(v_c) s_c)
                }
            }
        }
        __syncthreads();  // colred is reused by the next segment
    }
}

__global__ void __launch_bounds__(TRL_THREADS) tridiag_lower(double2* __restrict__ A, int n, double2* __restrict__ H,
                                                             EigSmall s, TriBufsL tb, GridBar* bar) {
    extern __shared__ double2 sm[];
    double2* vprev = sm;
    double2* wprev = sm + n;
    double2* vcur = sm + 2 * n;
    __shared__ double red[33];
    __shared__ double tau_sh, dk_sh, K_sh, a2_sh;
    __shared__ double2 w0_sh;
    __shared__ int prefix_sh[TRI_MAX_CHUNKS + 1];
    __shared__ double2 colred[TRL_NW][TRI_MAX_CPL * 32];
    const int nb = (int)gridDim.x;
    const int b = (int)blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned epoch = 0;
    bool have_prev = false;
    // row 0 (no pending update; the whole matrix is valid at the start): x = conj(A[0][1..n-1])
    double a2 = 0.0;
    for (int t = threadIdx.x; t < n - 1; t += blockDim.x) {
        const double2 a = __ldcg(&A[1 + t]);
        const double2 x = make_double2(a.x, -a.y);
        vcur[t] = x;
        a2 = fma(x.x, x.x, fma(x.y, x.y, a2));
    }
    a2 = block_sum(a2, red);  // |x|^2, the same in every thread
    if (threadIdx.x == 0) dk_sh = __ldcg(&A[0]).x;
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;
        // ---- reflector for column k (as in tridiag_persistent)
        if (threadIdx.x == 0) {
            const double2 x0 = vcur[0];
            const double q0 = fma(x0.x, x0.x, x0.y * x0.y);
            double tau = 0.0;
            double2 beta = make_double2(0.0, 0.0);
            if (a2 > 0.0) {
                const double ra = rsqrt(a2);
                const double alpha = a2 * ra;
                double2 phia;
                double ax0 = 0.0;
                if (q0 > 0.0) {
                    const double rq = rsqrt(q0);
                    ax0 = q0 * rq;
                    const double sc = alpha * rq;
                    phia = make_double2(x0.x * sc, x0.y * sc);
                } else {
                    phia = make_double2(alpha, 0.0);
                }
                vcur[0] = make_double2(x0.x + phia.x, x0.y + phia.y);
                tau = 1.0 / fma(alpha, ax0, a2);
                beta = make_double2(-phia.x, -phia.y);
            }
            tau_sh = tau;
            if (b == 0) {
                s.diag[k] = dk_sh;
                s.tau[k] = tau;
                s.e[k] = beta;
            }
        }
        __syncthreads();
        const double tau = tau_sh;
        if (tau == 0.0)
            for (int t = threadIdx.x; t < m; t += blockDim.x) vcur[t] = make_double2(0.0, 0.0);
        __syncthreads();
        if (b == 0)
            for (int t = threadIdx.x; t < m; t += blockDim.x) H[(long long)k * n + t] = vcur[t];
        // ---- B: trailing pass over the lower triangle, with this CTA's share of v^dag A v
        double2* pk = tb.part + (long long)(k & 1) * nb * n;
        double2* prow = tb.prow + (long long)(k & 1) * TRI_MAX_CHUNKS * n;
        double2* wfin = tb.w + (long long)(k & 1) * n;
        const int cpl = m >= 256 ? 2 : 1;
        const int W = 32 * cpl;
        const int C = (m + W - 1) / W;
        if ((int)threadIdx.x <= C) {
            // items (blocks of TRL_IB rows) before chunk t: chunk c holds rows c W .. m-1
            int acc = 0;
            for (int c = 0; c < (int)threadIdx.x; ++c) acc += (m - c * W + TRL_IB - 1) / TRL_IB;
            prefix_sh[threadIdx.x] = acc;
        }
        __syncthreads();
        double dacc = 0.0;
        if (cpl == 2)
            tri_pass_lower<2>(A, n, k, m, nb, have_prev, vprev, wprev, vcur, pk, prow, &colred[0][0], prefix_sh, C,
                              dacc);
        else
            tri_pass_lower<1>(A, n, k, m, nb, have_prev, vprev, wprev, vcur, pk, prow, &colred[0][0], prefix_sh, C,
                              dacc);
        dacc = block_sum(dacc, red);
        if (threadIdx.x == 0) tb.dot[b] = dacc;
        if (!grid_sync(bar, (unsigned)nb, epoch++)) return;
        // ---- K = (tau^2/2) v^dag A v from the CTA partials (one fixed order, the same in every
        //      CTA), w_0 = p_0 - K v_0 and the next diagonal element; the last warp does this while
        //      the others start on their slices.  p_0 has no row part and chunk 0's slots in order.
        const bool next = k + 3 < n;
        const double2 v0 = vcur[0];
        const int T = prefix_sh[C];
        const int nbe = min(nb, T);
        if (warp == TRL_NW - 1) {
            double sdot = 0.0;
            for (int i = lane; i < nb; i += 32) sdot += __ldcg(&tb.dot[i]);
            sdot = warp_sum(sdot);
            if (lane == 0) {
                const double K = 0.5 * tau * tau * sdot;
                const int ns0 = tri_item_owner(prefix_sh[1] - 1, T, nbe) + 1;  // slots of chunk 0
                double px = 0.0, py = 0.0;
                for (int s2 = 0; s2 < ns0; ++s2) {
                    const double2 q = __ldcg(&pk[(long long)s2 * n]);
                    px += q.x;
                    py += q.y;
                }
                const double2 w0 = make_double2(fma(-K, v0.x, tau * px), fma(-K, v0.y, tau * py));
                K_sh = K;
                w0_sh = w0;
                if (next)
                    dk_sh = __ldcg(&A[(long long)(k + 1) * n + (k + 1)]).x - 2.0 * (v0.x * w0.x + v0.y * w0.y);
            }
        }
        // ---- slices of 32 rows over the CTAs: p = tau (column parts of the CTA slots of the row's
        //      chunk + row parts of chunks 0 .. row/W); warp u sums slots and chunks u, u + NW, ...,
        //      then warp 0 adds the warps in order; w = p - K v; column k+1 with step k's update
        //      (A[j][k+1] -= v_j conj(w_0) + w_j conj(v_0): the conjugate of row k+1, i.e. the next
        //      reflector's x) and its partial squared norm
        double a2p = 0.0;
        for (int blk = b; blk * 32 < m; blk += nb) {
            const int il = blk * 32 + lane;
            const int cl = (blk * 32) / W;  // the same for the 32 rows (W is a multiple of 32)
            const int s_first = tri_item_owner(prefix_sh[cl], T, nbe);
            const int nsl = tri_item_owner(prefix_sh[cl + 1] - 1, T, nbe) - s_first + 1;
            double2 xa = make_double2(0.0, 0.0);
            if (warp == 0 && next && il >= 1 && il < m) xa = __ldcg(&A[(long long)(k + 1 + il) * n + (k + 1)]);
            double sx = 0.0, sy = 0.0;
            if (il < m) {
                for (int s2 = warp; s2 < nsl; s2 += TRL_NW) {
                    const double2 r = __ldcg(&pk[(long long)s2 * n + il]);
                    sx += r.x;
                    sy += r.y;
                }
                for (int c = warp; c <= cl; c += TRL_NW) {
                    const double2 r = __ldcg(&prow[(long long)c * n + il]);
                    sx += r.x;
                    sy += r.y;
                }
            }
            colred[warp][lane] = make_double2(sx, sy);
            __syncthreads();
            if (warp == 0 && il < m) {
                double tx = 0.0, ty = 0.0;
#pragma unroll
                for (int u = 0; u < TRL_NW; ++u) {
                    tx += colred[u][lane].x;
                    ty += colred[u][lane].y;
                }
                const double K = K_sh;
                const double2 w0 = w0_sh;
                const double2 v = vcur[il];
                const double2 w = make_double2(fma(-K, v.x, tau * tx), fma(-K, v.y, tau * ty));
                wfin[il] = w;
                if (next && il >= 1) {
                    const double2 x = sub_two_cmulc(xa, v, w0, w, v0);
                    tb.x[il - 1] = x;
                    a2p = fma(x.x, x.x, fma(x.y, x.y, a2p));
                }
            }
            __syncthreads();
        }
        if (warp == 0) {
            a2p = warp_sum(a2p);
            if (lane == 0) tb.a2[b] = a2p;
        }
        if (!grid_sync(bar, (unsigned)nb, epoch++)) return;
        // ---- C(k): every CTA loads w (the pending update) and the next column; |x|^2 from the partials
        double2* vnew = vcur;
        double2* wnew = wprev;  // the old pending update is spent
        double2* xnext = vprev;
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            wnew[t] = __ldcg(&wfin[t]);
            if (next && t >= 1) xnext[t - 1] = __ldcg(&tb.x[t - 1]);
        }
        if (warp == 0) {
            double sa = 0.0;
            for (int i = lane; i < nb; i += 32) sa += __ldcg(&tb.a2[i]);
            sa = warp_sum(sa);
            if (lane == 0) a2_sh = sa;
        }
        __syncthreads();
        a2 = a2_sh;
        vprev = vnew;
        wprev = wnew;
        vcur = xnext;
        have_prev = true;
    }
    // ---- tail: last 2 x 2 block (lower half) with the pending update applied
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (n >= 2) {
            double2 a00 = __ldcg(&A[(long long)(n - 2) * n + (n - 2)]);
            double2 a11 = __ldcg(&A[(long long)(n - 1) * n + (n - 1)]);
            double2 a10 = __ldcg(&A[(long long)(n - 1) * n + (n - 2)]);
            if (have_prev) {
                a00.x -= 2.0 * (vprev[0].x * wprev[0].x + vprev[0].y * wprev[0].y);
                a11.x -= 2.0 * (vprev[1].x * wprev[1].x + vprev[1].y * wprev[1].y);
                const double2 u = cmulc(vprev[1], wprev[0]), v = cmulc(wprev[1], vprev[0]);
                a10.x -= u.x + v.x;
                a10.y -= u.y + v.y;
            }
            s.diag[n - 2] = a00.x;
            s.diag[n - 1] = a11.x;
            s.e[n - 2] = a10;  // conj of the upper element a01
        } else {
            s.diag[0] = __ldcg(&A[0]).x;
        }
    }
}

// ---------------------------------------------------------------- eigenvalues
// Number of eigenvalues of the symmetric tridiagonal (a, b) below x: the number of negative
// pivots of T - x I, i.e. sign changes between consecutive leading principal minors
// p_{i+1} = (a_i - x) p_i - b_{i-1}^2 p_{i-1}.  The minors are formed without division and
// with b^2 precomputed (three FP64 instructions per step; GB300 issues one FP64 warp
// instruction per 64 cycles per sub-partition); signs, zero tests and the range check read
// the bit pattern on the integer pipe.  Minors are rescaled by exact powers of two to stay
// in range; an exactly zero minor is replaced by -pivmin times its predecessor.
__device__ int sturm(const double* a, const double* bsq, int n, double x, double pivmin) {
    double prev = 1.0, cur = a[0] - x;
    if ((__double_as_longlong(cur) << 1) == 0) cur = -pivmin;
    int cnt = __double_as_longlong(cur) < 0 ? 1 : 0;
    for (int i = 1; i < n; ++i) {
        double nxt = fma(a[i] - x, cur, -bsq[i - 1] * prev);
        long long bn = __double_as_longlong(nxt);
        if ((bn << 1) == 0) {
            nxt = -pivmin * cur;
            bn = __double_as_longlong(nxt);
        }
        cnt += (int)((unsigned long long)(bn ^ __double_as_longlong(cur)) >> 63);
        prev = cur;
        cur = nxt;
        const int ex = (int)((bn >> 52) & 0x7ff);  // biased exponent
        if (ex > 1023 + 480 || ex < 1023 - 480) {
            int e2;
            frexp(cur, &e2);
            cur = ldexp(cur, -e2);
            prev = ldexp(prev, -e2);
        }
    }
    return cnt;
}

// One CTA of BIS_THREADS threads per eigenvalue; output j (descending) = ascending index
// n-1-j.  Each round evaluates BIS_THREADS Sturm counts at equally spaced interior points of
// [lo, hi] (one per thread, the warps on different SM sub-partitions) and keeps the
// subinterval that holds the eigenvalue: its upper end is the first point whose count
// reaches idx+1.  Stop at an absolute width of 2 u |T| (+ pivmin terms): the eigenvalues of
// the tridiagonal carry no more accuracy than the u |rho| of its computation.
constexpr int BIS_THREADS = 128;

__global__ void __launch_bounds__(BIS_THREADS) bisect_top(int n, int k, EigSmall s) {
    __shared__ int first_sh[BIS_THREADS / 32];
    const int j = blockIdx.x;
    if (j >= k) return;
    const int idx = n - 1 - j;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double gl = s.scal[4], gu = s.scal[5], tn = s.scal[6];
    const double pivmin = fmax(1e-300, EPS * EPS * fmax(tn, 1e-300));
    const double width = 2.0 * EPS * fmax(tn, 1e-300) + 4.0 * pivmin;
    double lo = gl - EPS * tn - pivmin, hi = gu + EPS * tn + pivmin;
    for (int round = 0; round < 64; ++round) {
        if (hi - lo <= width) break;
        const double step = (hi - lo) / (double)(BIS_THREADS + 1);
        const double x = lo + step * (threadIdx.x + 1);
        const int c = sturm(s.diag, s.bsq, n, x, pivmin);
        const unsigned bal = __ballot_sync(0xffffffffu, c >= idx + 1);
        if (lane == 0) first_sh[warp] = bal ? warp * 32 + __ffs(bal) - 1 : BIS_THREADS;
        __syncthreads();
        int f = BIS_THREADS;
#pragma unroll
        for (int w = 0; w < BIS_THREADS / 32; ++w) f = min(f, first_sh[w]);
        __syncthreads();  // first_sh is rewritten next round
        if (f == BIS_THREADS) {
            lo = lo + step * BIS_THREADS;
        } else {
            hi = lo + step * (f + 1);
            lo = lo + step * f;
        }
    }
    if (threadIdx.x == 0) s.lam[j] = 0.5 * (lo + hi);
}

__device__ __forceinline__ double hash_uniform(unsigned i, unsigned j) {
    unsigned h = i * 0x9E3779B1u ^ (j + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
    return (double)h * (2.0 / 4294967296.0) - 1.0;
}

// Inverse iteration: thread j computes the eigenvector of lam[j] into Z[:, j] (row-major n x k).
// T - lam I = P L U by Gaussian elimination with partial pivoting (row swaps of the
// tridiagonal); U keeps reciprocal pivots so the solves multiply.  The running row is
// carried in registers, so each step is one division plus a few FMAs on the dependency
// chain.  Three solves from a fixed pseudo-random start; the iterate is rescaled by its
// max-norm between solves (folded into the next forward pass) and normalised at the end.
// work holds 4 n k doubles (rdd, du, du2, dl) and n k ints (pivots), laid out [i*k + j].
__global__ void __launch_bounds__(128) inverse_iteration(int n, int k, EigSmall s, double* __restrict__ work,
                                                         int* __restrict__ piv, double* __restrict__ Z) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= k) return;
    const double* __restrict__ a = s.diag;
    const double* __restrict__ b = s.offd;
    const double tiny = EPS * fmax(s.scal[6], 1e-300);
    const double lam = s.lam[j];
    const long long K = k;
    double* __restrict__ rdd = work;
    double* __restrict__ du = work + (long long)n * K;
    double* __restrict__ du2 = work + 2LL * n * K;
    double* __restrict__ dl = work + 3LL * n * K;
#define AT(arr, i) arr[(long long)(i) * K + j]
    // ---- factorisation; (d, u) = diagonal and super-diagonal of the running row i
    double d = a[0] - lam, u = n > 1 ? b[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        const double l = b[i];
        const double dn = a[i + 1] - lam, un = (i + 2 < n) ? b[i + 1] : 0.0;
        if (fabs(d) >= fabs(l)) {
            const double dz = (d == 0.0) ? tiny : d;
            const double r = 1.0 / dz;
            const double f = l * r;
            AT(piv, i) = 0;
            AT(rdd, i) = fabs(dz) < tiny ? 1.0 / copysign(tiny, dz) : r;
            AT(du, i) = u;
            AT(du2, i) = 0.0;
            AT(dl, i) = f;
            d = fma(-f, u, dn);
            u = un;
        } else {
            const double r = 1.0 / l;
            const double f = d * r;
            AT(piv, i) = 1;
            AT(rdd, i) = fabs(l) < tiny ? 1.0 / copysign(tiny, l) : r;
            AT(du, i) = dn;
            AT(du2, i) = un;
            AT(dl, i) = f;
            d = fma(-f, dn, u);
            u = -f * un;
        }
    }
    AT(rdd, n - 1) = 1.0 / (fabs(d) < tiny ? copysign(tiny, d) : d);
    for (int i = 0; i < n; ++i) AT(Z, i) = hash_uniform((unsigned)i, (unsigned)j);
    double scale = 1.0;
    for (int it = 0; it < 3; ++it) {
        // forward: c = running entry i of L^{-1} P^T z (scaled on the fly)
        double c = AT(Z, 0) * scale;
#pragma unroll 4
        for (int i = 0; i + 1 < n; ++i) {
            const double nxt = AT(Z, i + 1) * scale;
            const double f = AT(dl, i);
            if (AT(piv, i) == 0) {
                AT(Z, i) = c;
                c = fma(-f, c, nxt);
            } else {
                AT(Z, i) = nxt;
                c = fma(-f, nxt, c);
            }
        }
        // backward: z_i = (z_i - du_i z_{i+1} - du2_i z_{i+2}) / d_i, tracking max |z_i|
        double z1 = c * AT(rdd, n - 1), z2 = 0.0;
        AT(Z, n - 1) = z1;
        double mx = fabs(z1);
#pragma unroll 4
        for (int i = n - 2; i >= 0; --i) {
            const double zi = fma(-AT(du2, i), z2, fma(-AT(du, i), z1, AT(Z, i))) * AT(rdd, i);
            AT(Z, i) = zi;
            mx = fmax(mx, fabs(zi));
            z2 = z1;
            z1 = zi;
        }
        scale = 1.0 / mx;
    }
    double nrm = 0.0;
    for (int i = 0; i < n; ++i) {
        const double z = AT(Z, i) * scale;
        nrm = fma(z, z, nrm);
    }
    const double inv = scale / sqrt(nrm);
    for (int i = 0; i < n; ++i) AT(Z, i) *= inv;
#undef AT
}

// ---------------------------------------------------------------- CholeskyQR
// Kernels of the orthonormalisation take an optional predicate: they do nothing unless
// *pred == want (the host enqueues both branches; the device picks one).
__device__ __forceinline__ bool skip(const int* pred, int want) { return pred != nullptr && *pred != want; }

// G[a][b] = sum_i Z[i][a] Z[i][b] (+ shift on the diagonal), 16 x 16 tile per block
__global__ void __launch_bounds__(256) gram_kernel(const double* __restrict__ Z, int n, int k, double* __restrict__ G,
                                                   double shift, const int* pred, int want) {
    if (skip(pred, want)) return;
    __shared__ double za[32][17], zb[32][17];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int a0 = blockIdx.y * 16, b0 = blockIdx.x * 16;
    double acc = 0.0;
    for (int i0 = 0; i0 < n; i0 += 32) {
        for (int t = threadIdx.x; t < 32 * 16; t += 256) {
            const int r = t / 16, c = t % 16;
            const int i = i0 + r;
            za[r][c] = (i < n && a0 + c < k) ? Z[(long long)i * k + a0 + c] : 0.0;
            zb[r][c] = (i < n && b0 + c < k) ? Z[(long long)i * k + b0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) acc = fma(za[r][ty], zb[r][tx], acc);
        __syncthreads();
    }
    const int a = a0 + ty, b = b0 + tx;
    if (a < k && b < k) G[(long long)a * k + b] = acc + (a == b ? shift : 0.0);
}

// *flag = 1 if max |G - I| > tol (the vectors need the full shifted CholeskyQR3), else 0
__global__ void __launch_bounds__(256) ortho_check(const double* __restrict__ G, int k, double tol, int* flag) {
    __shared__ double red[33];
    double mx = 0.0;
    for (long long t = threadIdx.x; t < (long long)k * k; t += blockDim.x) {
        const long long a = t / k, b = t - a * k;
        mx = fmax(mx, fabs(G[t] - (a == b ? 1.0 : 0.0)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
        *flag = (mx > tol || !(mx == mx)) ? 1 : 0;
    }
}

// In-place lower Cholesky of the k x k G (single CTA, right-looking); dinv[j] = 1 / L[j][j].
// status[0] = 1 on a non-positive pivot.
__global__ void __launch_bounds__(1024) cholesky_kernel(double* __restrict__ G, int k, double* __restrict__ dinv,
                                                        int* __restrict__ status, const int* pred, int want) {
    if (skip(pred, want)) return;
    __shared__ double rj;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, nty = blockDim.x >> 5;
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double djj = G[(long long)j * k + j];
            if (!(djj > 0.0)) {
                status[0] = 1;
                djj = 1e-300;
            }
            const double r = rsqrt(djj);
            G[(long long)j * k + j] = djj * r;
            dinv[j] = r;
            rj = r;
        }
        __syncthreads();
        const double r = rj;
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) G[(long long)i * k + j] *= r;
        __syncthreads();
        for (int i = j + 1 + ty; i < k; i += nty) {
            const double gij = G[(long long)i * k + j];
            for (int l = j + 1 + tx; l <= i; l += 32)
                G[(long long)i * k + l] = fma(-gij, G[(long long)l * k + j], G[(long long)i * k + l]);
        }
        __syncthreads();
    }
}

// Blocked right-looking form of the same Cholesky for large k (the one-CTA kernel above walks k
// steps with two block barriers each): per block of CH_NB columns, the diagonal block is factored
// (and its factor inverted) by one CTA, the panel below becomes L21 = G21 L11^{-T} (a product with
// the inverse, one thread per element), and the lower tiles of the trailing matrix take
// G22 -= L21 L21^T.  The diagonal pivots use the same rsqrt form as cholesky_kernel.
constexpr int CH_NB = 32;

__global__ void __launch_bounds__(256) chol_diag(double* __restrict__ G, int k, int j0, double* __restrict__ dinv,
                                                 double* __restrict__ Linv, int* __restrict__ status,
                                                 const int* pred, int want) {
    if (skip(pred, want)) return;
    __shared__ double S[CH_NB][CH_NB + 1];
    __shared__ double X[CH_NB][CH_NB + 1];
    const int b = min(CH_NB, k - j0);
    for (int t = threadIdx.x; t < CH_NB * CH_NB; t += blockDim.x) {
        const int i = t / CH_NB, j = t - (t / CH_NB) * CH_NB;
        S[i][j] = (i < b && j <= i) ? G[(long long)(j0 + i) * k + j0 + j] : 0.0;
        X[i][j] = 0.0;
    }
    __syncthreads();
    for (int j = 0; j < b; ++j) {
        if (threadIdx.x == 0) {
            double djj = S[j][j];
            if (!(djj > 0.0)) {
                status[0] = 1;
                djj = 1e-300;
            }
            const double r = rsqrt(djj);
            S[j][j] = djj * r;
            X[j][j] = r;
        }
        __syncthreads();
        const double r = X[j][j];
        for (int i = j + 1 + threadIdx.x; i < b; i += blockDim.x) S[i][j] *= r;
        __syncthreads();
        const int w = b - j - 1;
        for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
            const int i = j + 1 + t / w, l = j + 1 + t % w;
            if (l <= i) S[i][l] = fma(-S[i][j], S[l][j], S[i][l]);
        }
        __syncthreads();
    }
    // inverse of the factor, one column per thread: X[i][c] = -(sum_{c<=l<i} S[i][l] X[l][c]) / S[i][i]
    if ((int)threadIdx.x < b) {
        const int c = threadIdx.x;
        for (int i = c + 1; i < b; ++i) {
            double acc = 0.0;
            for (int l = c; l < i; ++l) acc = fma(S[i][l], X[l][c], acc);
            X[i][c] = -acc * X[i][i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < CH_NB * CH_NB; t += blockDim.x) {
        const int i = t / CH_NB, j = t - (t / CH_NB) * CH_NB;
        Linv[t] = X[i][j];
        if (i < b && j <= i) G[(long long)(j0 + i) * k + j0 + j] = S[i][j];
    }
    for (int i = threadIdx.x; i < b; i += blockDim.x) dinv[j0 + i] = X[i][i];
}

// rows j0 + CH_NB + 8 blockIdx.x + r of the panel: L21[i][j] = sum_{l <= j} G21[i][l] Linv[j][l]
__global__ void __launch_bounds__(256) chol_panel(double* __restrict__ G, int k, int j0,
                                                  const double* __restrict__ Linv, const int* pred, int want) {
    if (skip(pred, want)) return;
    __shared__ double Li[CH_NB][CH_NB + 1];
    __shared__ double Rw[8][CH_NB + 1];
    for (int t = threadIdx.x; t < CH_NB * CH_NB; t += blockDim.x) Li[t / CH_NB][t % CH_NB] = Linv[t];
    const int r = threadIdx.x / CH_NB, j = threadIdx.x % CH_NB;
    const int i = j0 + CH_NB + blockIdx.x * 8 + r;
    Rw[r][j] = i < k ? G[(long long)i * k + j0 + j] : 0.0;
    __syncthreads();
    if (i < k) {
        double acc = 0.0;
        for (int l = 0; l <= j; ++l) acc = fma(Rw[r][l], Li[j][l], acc);
        G[(long long)i * k + j0 + j] = acc;
    }
}

// lower tile (ti, tj), tj <= ti, of the trailing block at s0 = j0 + CH_NB: G22 -= L21 L21^T
__global__ void __launch_bounds__(256) chol_update(double* __restrict__ G, int k, int j0, const int* pred, int want) {
    if (skip(pred, want)) return;
    __shared__ double Pa[CH_NB][CH_NB + 1], Pb[CH_NB][CH_NB + 1];
    const int t = blockIdx.x;
    int ti = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    while (ti * (ti + 1) / 2 > t) --ti;
    const int tj = t - ti * (ti + 1) / 2;
    const int s0 = j0 + CH_NB;
    for (int e = threadIdx.x; e < CH_NB * CH_NB; e += blockDim.x) {
        const int rr = e / CH_NB, l = e % CH_NB;
        const int ia = s0 + ti * CH_NB + rr, ib = s0 + tj * CH_NB + rr;
        Pa[rr][l] = ia < k ? G[(long long)ia * k + j0 + l] : 0.0;
        Pb[rr][l] = ib < k ? G[(long long)ib * k + j0 + l] : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CH_NB * CH_NB; e += blockDim.x) {
        const int rr = e / CH_NB, cc = e % CH_NB;
        const int gi = s0 + ti * CH_NB + rr, gj = s0 + tj * CH_NB + cc;
        if (gi < k && gj <= gi) {
            double acc = 0.0;
#pragma unroll 8
            for (int l = 0; l < CH_NB; ++l) acc = fma(Pa[rr][l], Pb[cc][l], acc);
            G[(long long)gi * k + gj] -= acc;
        }
    }
}

// lower Cholesky of the k x k G in place, dinv[j] = 1 / L[j][j]; one CTA for small k, blocked above
void cholesky_dev(Ctx& ctx, double* G, int k, double* dinv, int* status, const int* pred, int want) {
    if (k <= 128) {
        cholesky_kernel<<<1, 1024, 0, ctx.stream>>>(G, k, dinv, status, pred, want);
        ctx.count_launch();
        return;
    }
    double* Linv = (double*)ctx.workspace(WS_CHOL_LINV, sizeof(double) * CH_NB * CH_NB);
    for (int j0 = 0; j0 < k; j0 += CH_NB) {
        chol_diag<<<1, 256, 0, ctx.stream>>>(G, k, j0, dinv, Linv, status, pred, want);
        ctx.count_launch();
        const int rest = k - j0 - CH_NB;
        if (rest > 0) {
            chol_panel<<<(unsigned)((rest + 7) / 8), 256, 0, ctx.stream>>>(G, k, j0, Linv, pred, want);
            const int T = (rest + CH_NB - 1) / CH_NB;
            chol_update<<<(unsigned)(T * (T + 1) / 2), 256, 0, ctx.stream>>>(G, k, j0, pred, want);
            ctx.count_launch(2);
        }
    }
}

// Z <- Z L^{-T}: q_j = (z_j - sum_{l<j} q_l L[j][l]) / L[j][j] for 32 rows per CTA (one row
// per lane); the warps split each inner sum, warp 0 finishes the column.
constexpr int TS_WARPS = 8;
__global__ void __launch_bounds__(32 * TS_WARPS) trsm_rows(double* __restrict__ Z, int n, int k,
                                                           const double* __restrict__ L,
                                                           const double* __restrict__ dinv, const int* pred,
                                                           int want) {
    if (skip(pred, want)) return;
    extern __shared__ double q[];  // [k][33]: z, then q, of this CTA's rows
    __shared__ double part[TS_WARPS][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * 32;
    const int nr = min(32, n - r0);
    for (int t = threadIdx.x; t < nr * k; t += blockDim.x) {
        const int l = t / k, j = t - l * k;
        q[j * 33 + l] = Z[(long long)(r0 + l) * k + j];
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        double acc = 0.0;
        const double* Lj = L + (long long)j * k;
        for (int l = warp; l < j; l += TS_WARPS) acc = fma(q[l * 33 + lane], Lj[l], acc);
        part[warp][lane] = acc;
        __syncthreads();
        if (warp == 0) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < TS_WARPS; ++w) sum += part[w][lane];
            q[j * 33 + lane] = (q[j * 33 + lane] - sum) * dinv[j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nr * k; t += blockDim.x) {
        const int l = t / k, j = t - l * k;
        Z[(long long)(r0 + l) * k + j] = q[j * 33 + l];
    }
}

// ---------------------------------------------------------------- back-transformation
// y = ph .* Z[:, j], then y <- H_0 H_1 ... H_{n-3} y (H_kk = I - tau_kk v_kk v_kk^dag acting on
// indices kk+1..n-1), written as columns (mode 0: U[i][j] = y_i) or conjugated rows
// (mode 1: B[j][i] = conj(y_i)).
//
// The reflectors are applied in blocks of BT_NB in compact WY form (Schreiber and Van Loan):
// Q_b = H_{b0} ... H_{b0+nb-1} = I - V T V^dag with T upper triangular, T_rr = tau_r and
// T[0:r, r] = -tau_r T[0:r, 0:r] (V[:, 0:r]^dag v_r).  Each block costs one CTA-wide reduction
// of its nb inner products instead of one per reflector.  One eigenvector per CTA.
constexpr int BT_NB = 16;
constexpr int BT_THREADS = 256;

__device__ __forceinline__ double2 refl_elem(const double2* __restrict__ H, int n, int kk, int g) {
    return H[(long long)kk * n + (g - kk - 1)];  // v_kk at global index g >= kk + 1
}

// T factors of all blocks: Tall[b][q][r] (BT_NB x BT_NB, upper triangle used).  One CTA per
// block: warps form the Gram entries S[q][r] = v_q^dag v_r (q < r), then warp 0 runs the
// recurrence with lane q owning row q of T.
__global__ void __launch_bounds__(256) wy_tfactor(int n, const double2* __restrict__ H, EigSmall s,
                                                  double2* __restrict__ Tall) {
    __shared__ double2 S[BT_NB][BT_NB];
    __shared__ double2 T[BT_NB][BT_NB + 1];
    const int b = blockIdx.x;
    const int b0 = b * BT_NB;
    const int nb = min(BT_NB, n - 2 - b0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int npair = nb * (nb - 1) / 2;
    for (int pr = warp; pr < npair; pr += nw) {
        // pair index -> (q, r), q < r
        int r = 1, rem = pr;
        while (rem >= r) {
            rem -= r;
            ++r;
        }
        const int q = rem;
        const int kq = b0 + q, kr = b0 + r;
        double sx = 0.0, sy = 0.0;
        for (int g = kr + 1 + lane; g < n; g += 32) {  // common support of v_q and v_r
            const double2 a = refl_elem(H, n, kq, g), c = refl_elem(H, n, kr, g);
            sx = fma(a.x, c.x, fma(a.y, c.y, sx));  // conj(a) c
            sy = fma(a.x, c.y, fma(-a.y, c.x, sy));
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        if (lane == 0) S[q][r] = make_double2(sx, sy);
    }
    __syncthreads();
    if (warp == 0) {
        for (int r = 0; r < BT_NB; ++r) {
            const double tau = r < nb ? s.tau[b0 + r] : 0.0;
            if (lane == r) T[r][r] = make_double2(tau, 0.0);
            if (lane < r) {
                double ax = 0.0, ay = 0.0;
                if (r < nb) {
                    for (int p2 = lane; p2 < r; ++p2) {  // T[lane][p2] S[p2][r]
                        const double2 t = T[lane][p2], sv = S[p2][r];
                        ax = fma(t.x, sv.x, fma(-t.y, sv.y, ax));
                        ay = fma(t.x, sv.y, fma(t.y, sv.x, ay));
                    }
                }
                T[lane][r] = make_double2(-tau * ax, -tau * ay);
            }
            if (lane > r && lane < BT_NB) T[lane][r] = make_double2(0.0, 0.0);
            __syncwarp();
        }
        if (lane < BT_NB)
            for (int r = 0; r < BT_NB; ++r) Tall[((long long)b * BT_NB + lane) * BT_NB + r] = T[lane][r];
    }
}

__global__ void __launch_bounds__(BT_THREADS) backtransform(int n, int k, const double2* __restrict__ H,
                                                            EigSmall s, const double2* __restrict__ Tall,
                                                            const double* __restrict__ Z, int mode,
                                                            double2* __restrict__ out) {
    extern __shared__ double2 y[];  // [n]
    __shared__ double part[BT_THREADS / 32][32];
    __shared__ double2 tvec[BT_NB];
    const int j = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double z = Z[(long long)i * k + j];
        const double2 q = s.ph[i];
        y[i] = make_double2(q.x * z, q.y * z);
    }
    __syncthreads();
    const int nblk = (n - 2 + BT_NB - 1) / BT_NB;
    for (int b = nblk - 1; b >= 0; --b) {
        const int b0 = b * BT_NB;
        const int nb = min(BT_NB, n - 2 - b0);
        // 1. w_r = v_r^dag y, r < nb (values 2r, 2r+1 = Re, Im)
        double v[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.0;
        for (int g = b0 + 1 + threadIdx.x; g < n; g += blockDim.x) {
            const double2 yv = y[g];
#pragma unroll
            for (int r = 0; r < BT_NB; ++r) {
                const int kk = b0 + r;
                if (r < nb && g > kk) {
                    const double2 a = refl_elem(H, n, kk, g);
                    v[2 * r] = fma(a.x, yv.x, fma(a.y, yv.y, v[2 * r]));
                    v[2 * r + 1] = fma(a.x, yv.y, fma(-a.y, yv.x, v[2 * r + 1]));
                }
            }
        }
        part[warp][lane] = warp_reduce32(v);
        __syncthreads();
        if (warp == 0) {
            double tot = 0.0;
            for (int w = 0; w < nw; ++w) tot += part[w][lane];
            part[0][lane] = tot;
            __syncwarp();
            // 2. t = T w (T upper triangular)
            if (lane < nb) {
                const double2* Tq = Tall + ((long long)b * BT_NB + lane) * BT_NB;
                double tx = 0.0, ty = 0.0;
                for (int r = lane; r < nb; ++r) {
                    const double2 t = Tq[r];
                    const double wx = part[0][2 * r], wy = part[0][2 * r + 1];
                    tx = fma(t.x, wx, fma(-t.y, wy, tx));
                    ty = fma(t.x, wy, fma(t.y, wx, ty));
                }
                tvec[lane] = make_double2(tx, ty);
            }
        }
        __syncthreads();
        // 3. y <- y - V t
        for (int g = b0 + 1 + threadIdx.x; g < n; g += blockDim.x) {
            double2 acc = y[g];
#pragma unroll
            for (int r = 0; r < BT_NB; ++r) {
                const int kk = b0 + r;
                if (r < nb && g > kk) {
                    const double2 a = refl_elem(H, n, kk, g), t = tvec[r];
                    acc.x = fma(-a.x, t.x, fma(a.y, t.y, acc.x));
                    acc.y = fma(-a.x, t.y, fma(-a.y, t.x, acc.y));
                }
            }
            y[g] = acc;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double2 w = y[i];
        if (mode == 0) out[(long long)i * k + j] = w;
        else out[(long long)j * n + i] = make_double2(w.x, -w.y);
    }
}

}  // namespace

TruncResult truncate_deferred_result(const double* slot, int k) {
    // slot: lam[k], tr(rho), then 8 status ints (4 doubles' worth)
    TruncResult r;
    r.k = k;
    r.lam.assign(slot, slot + k);
    const double tr = slot[k];
    double kept = 0.0;
    for (double l : r.lam) kept += l;
    r.discarded = tr > 0 ? 1.0 - kept / tr : 0.0;
    int st[8];
    std::memcpy(st, slot + k + 1, sizeof(st));
    if (st[6] != 0) throw Error{VTN_ETIMEOUT, "tridiagonalisation grid barrier timed out"};
    return r;
}

TruncResult truncate_dev(Ctx& ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                         const double2* theta, double2* left, double2* right, int outer, double* defer) {
    const int nL = chi_l * d1, nR = d2 * chi_r;
    const int n = direction == 0 ? nL : nR;
    const int k = std::min(k_max, std::min(nL, nR));
    if (outer < 0) outer = direction == 0 ? nR : nL;
    VTN_REQUIRE(outer >= 1 && outer <= (direction == 0 ? nR : nL), "truncation output range out of bounds");
    VTN_REQUIRE(k >= 1, "truncation keeps no state");
    VTN_REQUIRE(n <= 12288, "reduced density matrix larger than 12288 is not supported");
    int tt = ctx.tbegin(TC_EIG, 0.0);
    double2* A = (double2*)ctx.workspace(WS_EIG_A, sizeof(double2) * (size_t)n * n);
    double2* H = (double2*)ctx.workspace(WS_EIG_H, sizeof(double2) * (size_t)n * n);
    double* small = (double*)ctx.workspace(WS_EIG_U, sizeof(double) * (16 * (size_t)n + 32));
    EigSmall s;
    s.diag = small;
    s.offd = small + n;
    s.tau = small + 2 * (size_t)n;
    s.lam = small + 3 * (size_t)n;
    s.e = (double2*)(small + 4 * (size_t)n);
    s.ph = (double2*)(small + 6 * (size_t)n);
    s.p = (double2*)(small + 8 * (size_t)n);
    s.w = (double2*)(small + 10 * (size_t)n);
    s.scal = small + 12 * (size_t)n;
    s.bsq = small + 12 * (size_t)n + 16;
    double* Z = (double*)ctx.workspace(WS_EIG_Y, sizeof(double) * (size_t)n * k);
    double* work = (double*)ctx.workspace(WS_EIG_WORK, sizeof(double) * (5 * (size_t)n * k + (size_t)k * k + 32));
    int* piv = (int*)(work + 4 * (size_t)n * k);
    double* G = work + 5 * (size_t)n * k;
    int* status = (int*)(G + (size_t)k * k);
    // 1. rho
    GemmArgs g;
    if (direction == 0) {
        g.M = nL; g.N = nL; g.K = nR;
        g.A = theta; g.lda = nR;
        g.opB = OP_C; g.B = theta; g.ldb = nR;
    } else {
        g.M = nR; g.N = nR; g.K = nL;
        g.opA = OP_C; g.A = theta; g.lda = nR;
        g.B = theta; g.ldb = nR;
    }
    g.C = A; g.ldc = n;
    g.herm_lower = true;
    gemm_c64(ctx, g);
    mirror_lower_to_upper(ctx, A, n, n);
    norm2_dev(ctx, theta, (long long)nL * nR, &s.scal[0]);
    VTN_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int) * 8, ctx.stream));
    // 2. tridiagonalisation: one persistent cooperative launch when it fits, else one
    //    launch per Householder step
    bool done = false;
    if (n <= TRI_MAX_N && n >= ctx.tri_lower_min_n) {
        const size_t shm = sizeof(double2) * 3 * (size_t)n;
        set_smem_attr_once(ctx, (const void*)tridiag_lower, (int)(sizeof(double2) * 3 * TRI_MAX_N + 1024));
        int per_sm = 0;
        VTN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_lower, TRL_THREADS, shm));
        const int grid = std::min(ctx.num_sms, std::max(1, (n + 3) / 4));
        if (per_sm >= 1 && grid >= 1) {
            const size_t part_n = (size_t)grid * n;
            const size_t elems = 2 * part_n + 2 * (size_t)TRI_MAX_CHUNKS * n + 3 * (size_t)n;
            const size_t bytes = sizeof(double2) * elems;
            char* wsp = (char*)ctx.workspace(WS_EIG_PART, bytes + sizeof(double) * 2 * (size_t)grid);
            TriBufsL tb;
            tb.part = (double2*)wsp;
            tb.prow = tb.part + 2 * part_n;
            tb.w = tb.prow + 2 * (size_t)TRI_MAX_CHUNKS * n;
            tb.x = tb.w + 2 * (size_t)n;
            tb.dot = (double*)(wsp + bytes);
            tb.a2 = tb.dot + grid;
            GridBar* bar = (GridBar*)(status + 4);
            VTN_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx.stream));
            double2* Ap = A;
            double2* Hp = H;
            int nn = n;
            void* args[] = {&Ap, &nn, &Hp, &s, &tb, &bar};
            const int ttri = ctx.tbegin(TC_TRI, 16.0 / 3.0 * (double)n * n * n);
            VTN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)tridiag_lower, dim3(grid), dim3(TRL_THREADS), args, shm,
                                                     ctx.stream));
            ctx.tend(ttri);
            ctx.count_launch();
            ctx.check_launch("tridiag_lower");
            done = true;
        }
    }
    if (!done && n <= TRI_MAX_N) {
        const size_t shm = sizeof(double2) * 3 * (size_t)n;
        set_smem_attr_once(ctx, (const void*)tridiag_persistent, (int)(sizeof(double2) * 3 * TRI_MAX_N + 1024));
        int per_sm = 0;
        VTN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tridiag_persistent, TRI_THREADS, shm));
        // one CTA per SM: Phases A and C are redundant per CTA, so more CTAs per SM cost more
        int grid = std::min(ctx.num_sms, std::max(1, (n + 3) / 4));
        if (per_sm >= 1 && grid >= 1) {
            const size_t part_bytes = sizeof(double2) * (2 * (size_t)grid * n + 2 * (size_t)n);
            char* wsp = (char*)ctx.workspace(WS_EIG_PART, part_bytes + sizeof(unsigned) * 2 * TRI_MAX_CHUNKS);
            TriBufs tb;
            tb.part = (double2*)wsp;
            tb.p = tb.part + 2 * (size_t)grid * n;
            tb.arrive = (unsigned*)(wsp + part_bytes);
            VTN_CUDA_TRY(cudaMemsetAsync(tb.arrive, 0, sizeof(unsigned) * 2 * TRI_MAX_CHUNKS, ctx.stream));
            GridBar* bar = (GridBar*)(status + 4);
            VTN_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(GridBar), ctx.stream));
            double2* Ap = A;
            double2* Hp = H;
            int nn = n;
            void* args[] = {&Ap, &nn, &Hp, &s, &tb, &bar};
            // timing class: the standard 16/3 n^3 real flops of a complex Hermitian tridiagonalisation
            const int ttri = ctx.tbegin(TC_TRI, 16.0 / 3.0 * (double)n * n * n);
            VTN_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)tridiag_persistent, dim3(grid), dim3(TRI_THREADS),
                                                     args, shm, ctx.stream));
            ctx.tend(ttri);
            ctx.count_launch();
            ctx.check_launch("tridiag_persistent");
            done = true;
        }
    }
    if (!done) {
        for (int kk = 0; kk + 2 < n; ++kk) {
            const int m = n - kk - 1;
            hh_reflector<<<1, 1024, 0, ctx.stream>>>(A, n, kk, H, s);
            hh_matvec<<<(m + 7) / 8, 256, 0, ctx.stream>>>(A, n, kk, H, s);
            hh_w<<<1, 1024, 0, ctx.stream>>>(n, kk, H, s);
            const long long mm = (long long)m * m;
            hh_rank2<<<(unsigned)((mm + 255) / 256), 256, 0, ctx.stream>>>(A, n, kk, H, s);
            ctx.count_launch(4);
        }
        tri_finalize<<<1, 32, 0, ctx.stream>>>(A, n, s);
        ctx.count_launch();
    }
    tri_phases<<<1, TP_THREADS, 0, ctx.stream>>>(n, s);
    ctx.count_launch();
    ctx.check_launch("tridiagonalisation");
    // 3. eigenvalues
    bisect_top<<<k, BIS_THREADS, 0, ctx.stream>>>(n, k, s);
    // 4. eigenvectors of the real tridiagonal
    inverse_iteration<<<(k + 127) / 128, 128, 0, ctx.stream>>>(n, k, s, work, piv, Z);
    ctx.count_launch(2);
    ctx.check_launch("eigenpairs");
    // 5. orthonormalisation.  Inverse-iteration vectors of separated eigenvalues are already
    //    orthonormal to O(u ||T|| / gap); if max |Z^T Z - I| <= 1e-3 one plain Cholesky-QR
    //    pass suffices (its loss of orthogonality is O(u kappa(Z)^2) with kappa(Z)^2 <= 1.003).
    //    Otherwise (clusters) the shifted CholeskyQR3 runs.  Both branches are enqueued; the
    //    device flag selects one.
    dim3 gg((k + 15) / 16, (k + 15) / 16);
    int* flag = status + 1;
    double* dinv = small + 13 * (size_t)n + 32;
    const size_t ts_shm = sizeof(double) * (size_t)k * 33;
    set_smem_attr_once(ctx, (const void*)trsm_rows, 200 * 1024);
    VTN_REQUIRE(ts_shm <= 200 * 1024, "truncation keeps too many states for the orthonormalisation");
    const unsigned ts_grid = (unsigned)((n + 31) / 32);
    gram_kernel<<<gg, 256, 0, ctx.stream>>>(Z, n, k, G, 0.0, nullptr, 0);
    ortho_check<<<1, 256, 0, ctx.stream>>>(G, k, 1e-3, flag);
    cholesky_dev(ctx, G, k, dinv, status, flag, 0);
    trsm_rows<<<ts_grid, 32 * TS_WARPS, ts_shm, ctx.stream>>>(Z, n, k, G, dinv, flag, 0);
    ctx.count_launch(3);
    for (int pass = 0; pass < 3; ++pass) {
        double shift = 0.0;
        if (pass == 0) {
            // ||Z||_F^2 = k for unit columns; shift 11 (n k + k (k + 1)) u ||Z||_2^2 bounded by that
            shift = 11.0 * ((double)n * k + (double)k * (k + 1)) * EPS * (double)k;
        }
        gram_kernel<<<gg, 256, 0, ctx.stream>>>(Z, n, k, G, shift, flag, 1);
        cholesky_dev(ctx, G, k, dinv, status, flag, 1);
        trsm_rows<<<ts_grid, 32 * TS_WARPS, ts_shm, ctx.stream>>>(Z, n, k, G, dinv, flag, 1);
        ctx.count_launch(2);
    }
    ctx.check_launch("orthonormalisation");
    // 6. back-transformation into the site tensors: T factors of the reflector blocks, then
    //    one vector per CTA (the FP64 work spreads over the SMs)
    const size_t shm = sizeof(double2) * (size_t)n;
    const int nbt = k;
    set_smem_attr_once(ctx, (const void*)backtransform, 200 * 1024);
    const int nblk = n >= 3 ? (n - 2 + BT_NB - 1) / BT_NB : 0;
    double2* Tall = (double2*)ctx.workspace(WS_EIG_T, sizeof(double2) * (size_t)std::max(nblk, 1) * BT_NB * BT_NB);
    if (nblk > 0) {
        wy_tfactor<<<nblk, 256, 0, ctx.stream>>>(n, H, s, Tall);
        ctx.count_launch();
    }
    if (direction == 0) {
        backtransform<<<nbt, BT_THREADS, shm, ctx.stream>>>(n, k, H, s, Tall, Z, 0, left);
        // right = U^dag T (its first `outer` columns)
        GemmArgs c;
        c.M = k; c.N = outer; c.K = nL;
        c.opA = OP_C; c.A = left; c.lda = k;
        c.B = theta; c.ldb = nR;
        c.C = right; c.ldc = outer;
        ctx.count_launch();
        gemm_c64(ctx, c);
    } else {
        backtransform<<<nbt, BT_THREADS, shm, ctx.stream>>>(n, k, H, s, Tall, Z, 1, right);
        // left = T V = T (V^dag)^dag (its first `outer` rows)
        GemmArgs c;
        c.M = outer; c.N = k; c.K = nR;
        c.A = theta; c.lda = nR;
        c.opB = OP_C; c.B = right; c.ldb = nR;
        c.C = left; c.ldc = k;
        ctx.count_launch();
        gemm_c64(ctx, c);
    }
    ctx.check_launch("back-transformation");
    ctx.tend(tt);
    // results to the host
    if (defer != nullptr) {
        VTN_CUDA_TRY(cudaMemcpyAsync(defer, s.lam, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx.stream));
        VTN_CUDA_TRY(cudaMemcpyAsync(defer + k, s.scal, sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
        VTN_CUDA_TRY(cudaMemcpyAsync(defer + k + 1, status, sizeof(int) * 8, cudaMemcpyDeviceToHost, ctx.stream));
        TruncResult r;
        r.k = k;
        r.discarded = 0.0;
        return r;
    }
    VTN_CUDA_TRY(cudaMemcpyAsync(ctx.pinned, s.lam, sizeof(double) * k, cudaMemcpyDeviceToHost, ctx.stream));
    VTN_CUDA_TRY(cudaMemcpyAsync(ctx.pinned + k, s.scal, sizeof(double), cudaMemcpyDeviceToHost, ctx.stream));
    VTN_CUDA_TRY(cudaMemcpyAsync(ctx.pinned + k + 1, status, sizeof(int) * 8, cudaMemcpyDeviceToHost, ctx.stream));
    ctx.sync();
    TruncResult r;
    r.k = k;
    r.lam.assign(ctx.pinned, ctx.pinned + k);
    const double tr = ctx.pinned[k];
    double kept = 0.0;
    for (double l : r.lam) kept += l;
    r.discarded = tr > 0 ? 1.0 - kept / tr : 0.0;
    int st[8];
    std::memcpy(st, ctx.pinned + k + 1, sizeof(st));
    if (st[6] != 0)  // GridBar::error of the persistent tridiagonalisation (ints 4..7 after status)
        throw Error{VTN_ETIMEOUT, "tridiagonalisation grid barrier timed out"};
    return r;
}

}  // namespace vtn
