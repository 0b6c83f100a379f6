// Kernels around the solver: seeded random initial MPS (Philox4x32-10 + Box-Muller,
// rows orthonormalised), the inverse basis transformation of Eq.
// InverseBasisTransformation, transfer matrices of <psi|psi>, Fock-basis marginal
// reductions, and the sequential conditional sampler.
#include <algorithm>
#include <cmath>

#include "vtn_internal.cuh"

namespace vtn {

// ---------------------------------------------------------------- Philox4x32-10
// Salmon et al., SC'11: ten rounds of two 32x32 -> 64-bit products, Weyl key bumps.
__host__ __device__ inline void philox4x32_10(unsigned c[4], unsigned k0, unsigned k1) {
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const unsigned long long p0 = 0xD2511F53ull * c[0];
        const unsigned long long p1 = 0xCD9E8D57ull * c[2];
        const unsigned hi0 = (unsigned)(p0 >> 32), lo0 = (unsigned)p0;
        const unsigned hi1 = (unsigned)(p1 >> 32), lo1 = (unsigned)p1;
        const unsigned n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
    }
}

__host__ __device__ inline double uniform53(unsigned hi, unsigned lo) {
    const unsigned long long v = ((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11);
    return (double)v * (1.0 / 9007199254740992.0);
}

namespace {

__global__ void random_normal_kernel(double2* out, long long count, unsigned k0, unsigned k1, unsigned site,
                                     unsigned stream) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    unsigned c[4] = {(unsigned)j, (unsigned)((unsigned long long)j >> 32), site, stream};
    philox4x32_10(c, k0, k1);
    const double u1 = uniform53(c[0], c[1]);
    const double u2 = uniform53(c[2], c[3]);
    const double rad = sqrt(-2.0 * log1p(-u1));
    const double ang = 2.0 * 3.141592653589793 * u2;
    const double s = 0.7071067811865476;
    out[j] = make_double2(rad * cos(ang) * s, rad * sin(ang) * s);
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic filler in [-1, 1) for (row, column, part): splitmix64 of the three indices.
__device__ __forceinline__ double fill_value(unsigned long long r, unsigned long long c, unsigned long long part) {
    unsigned long long z = r * 0x9E3779B97F4A7C15ull + c * 0xD1B54A32D192ED03ull + part * 0x94D049BB133111EBull + 1ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// sum over the CTA of |x[c]|^2 (all threads get it); sh: 32 doubles
__device__ double block_norm2(const double2* x, int cols, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double s = 0.0;
    for (int c = threadIdx.x; c < cols; c += blockDim.x) s += x[c].x * x[c].x + x[c].y * x[c].y;
    s = warp_sum(s);
    __syncthreads();
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Classical Gram-Schmidt applied twice, row by row, in one CTA (rows <= 1024).
// coef[q] for q < r computed by warps (warp w takes q = w, w + nwarps, ...).  A row whose
// residual after the two projections is below 1e-10 of its norm (numerically dependent on the
// rows before it, or zero) is replaced by deterministic filler values, projected twice again
// and normalised: the rows always end orthonormal (an orthonormal completion, as Householder QR
// gives), so a truncation built on them keeps isometric site tensors.
__global__ void __launch_bounds__(1024) orth_rows_kernel(double2* A, int rows, int cols, const int* pred) {
    if (pred != nullptr && *pred == 0) return;
    extern __shared__ double2 coef[];  // rows entries
    __shared__ double nrm_sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = 0; r < rows; ++r) {
        double2* ar = A + (long long)r * cols;
        const double t0 = block_norm2(ar, cols, nrm_sh);
        double t = 0.0;
        for (int attempt = 0; attempt < 2; ++attempt) {
            for (int pass = 0; pass < 2; ++pass) {
                for (int q = wid; q < r; q += nw) {
                    const double2* aq = A + (long long)q * cols;
                    double re = 0.0, im = 0.0;
                    for (int c = lane; c < cols; c += 32) {
                        const double2 a = aq[c], b = ar[c];
                        re += a.x * b.x + a.y * b.y;
                        im += a.x * b.y - a.y * b.x;
                    }
                    re = warp_sum(re);
                    im = warp_sum(im);
                    if (lane == 0) coef[q] = make_double2(re, im);
                }
                __syncthreads();
                for (int c = threadIdx.x; c < cols; c += blockDim.x) {
                    double2 acc = ar[c];
                    for (int q = 0; q < r; ++q) {
                        const double2 a = A[(long long)q * cols + c], k = coef[q];
                        acc.x -= a.x * k.x - a.y * k.y;
                        acc.y -= a.x * k.y + a.y * k.x;
                    }
                    ar[c] = acc;
                }
                __syncthreads();
            }
            t = block_norm2(ar, cols, nrm_sh);
            if (attempt == 1 || (t > 1e-20 * t0 && t > 0.0)) break;
            // numerically dependent: start this row again from filler values
            for (int c = threadIdx.x; c < cols; c += blockDim.x)
                ar[c] = make_double2(fill_value(r, c, 0), fill_value(r, c, 1));
            __syncthreads();
        }
        const double inv = t > 0.0 ? 1.0 / sqrt(t) : 0.0;
        for (int c = threadIdx.x; c < cols; c += blockDim.x) {
            ar[c].x *= inv;
            ar[c].y *= inv;
        }
        __syncthreads();
    }
}

// out[a][n][b] = sum_m V[n][m] A[a][m][b]
__global__ void lbo_rotate_kernel(int chi_l, int d, int D, int chi_r, const double2* __restrict__ V,
                                  const double2* __restrict__ A, double2* __restrict__ out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)chi_l * D * chi_r;
    if (t >= total) return;
    const long long b = t % chi_r;
    const long long n = (t / chi_r) % D;
    const long long a = t / ((long long)chi_r * D);
    double2 acc = make_double2(0.0, 0.0);
    for (int m = 0; m < d; ++m) {
        const double2 v = V[n * d + m], x = A[(a * d + m) * chi_r + b];
        acc.x += v.x * x.x - v.y * x.y;
        acc.y += v.x * x.y + v.y * x.x;
    }
    out[t] = acc;
}

__global__ void set_one_kernel(double2* p) { *p = make_double2(1.0, 0.0); }

// P[n] = sum_{i,j} conj(AF[i][n][j]) U[i][n][j]   (one block per n)
__global__ void __launch_bounds__(256) marginal_reduce(int chi_l, int D, int chi_r, const double2* __restrict__ AF,
                                                       const double2* __restrict__ U, double* __restrict__ P) {
    __shared__ double sh[32];
    const int n = blockIdx.x;
    double acc = 0.0;
    const long long cnt = (long long)chi_l * chi_r;
    for (long long t = threadIdx.x; t < cnt; t += blockDim.x) {
        const long long i = t / chi_r, j = t % chi_r;
        const long long off = (i * D + n) * chi_r + j;
        const double2 a = AF[off], u = U[off];
        acc += a.x * u.x + a.y * u.y;
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        P[n] = s;
    }
}

// Sequential conditional sampling, one CTA per sample.  AF[s]: Fock-basis site tensors,
// ER[s]: right environments (ket, bra) in the solver basis, ER[M] = [1].
struct SampleArgs {
    const double2* const* AF;
    const double2* const* ER;
    const int* dims;  // M + 1
    int M, D;
    unsigned k0, k1;
    int n_samples;
    int chi_max;
    int* out;
};

__global__ void __launch_bounds__(256) sample_kernel(SampleArgs a) {
    extern __shared__ double2 sm[];
    const int t = blockIdx.x;
    if (t >= a.n_samples) return;
    double2* ell = sm;                       // chi_max
    double2* cand = sm + a.chi_max;          // D * chi_max
    double* p = (double*)(cand + (long long)a.D * a.chi_max);  // D
    __shared__ int pick;
    if (threadIdx.x == 0) ell[0] = make_double2(1.0, 0.0);
    __syncthreads();
    for (int s = 0; s < a.M; ++s) {
        const int cl = a.dims[s], cr = a.dims[s + 1];
        const double2* A = a.AF[s];
        const double2* E = a.ER[s + 1];
        // cand[n][b] = sum_i ell[i] A[i][n][b]
        for (int q = threadIdx.x; q < a.D * cr; q += blockDim.x) {
            const int n = q / cr, b = q % cr;
            double2 acc = make_double2(0.0, 0.0);
            for (int i = 0; i < cl; ++i) {
                const double2 l = ell[i], x = A[((long long)i * a.D + n) * cr + b];
                acc.x += l.x * x.x - l.y * x.y;
                acc.y += l.x * x.y + l.y * x.x;
            }
            cand[(long long)n * cr + b] = acc;
        }
        __syncthreads();
        // p[n] = sum_{b, b'} cand[n][b] E[b][b'] conj(cand[n][b'])
        for (int n = threadIdx.x >> 5; n < a.D; n += blockDim.x >> 5) {
            double acc = 0.0;
            for (int bp = threadIdx.x & 31; bp < cr; bp += 32) {
                double re = 0.0, im = 0.0;
                for (int b = 0; b < cr; ++b) {
                    const double2 c = cand[(long long)n * cr + b], e = E[(long long)b * cr + bp];
                    re += c.x * e.x - c.y * e.y;
                    im += c.x * e.y + c.y * e.x;
                }
                const double2 cb = cand[(long long)n * cr + bp];
                acc += re * cb.x + im * cb.y;  // Re(t * conj(cb))
            }
            acc = warp_sum(acc);
            if ((threadIdx.x & 31) == 0) p[n] = fmax(acc, 0.0);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned c[4] = {(unsigned)t, 0u, (unsigned)s, 2u};
            philox4x32_10(c, a.k0, a.k1);
            const double u = uniform53(c[0], c[1]);
            double total = 0.0;
            for (int n = 0; n < a.D; ++n) total += p[n];
            const double target = u * total;
            double cdf = 0.0;
            int pk = a.D - 1;
            for (int n = 0; n < a.D; ++n) {
                cdf += p[n];
                if (cdf > target) { pk = n; break; }
            }
            pick = pk;
            a.out[(long long)t * a.M + s] = pk;
        }
        __syncthreads();
        const int pk = pick;
        const double inv = 1.0 / sqrt(fmax(p[pk], 1e-300));
        for (int b = threadIdx.x; b < cr; b += blockDim.x) {
            const double2 c = cand[(long long)pk * cr + b];
            ell[b] = make_double2(c.x * inv, c.y * inv);
        }
        __syncthreads();
    }
}

// rho[s][t] = sum_{i, c} U[i][s][c] conj(A[i][t][c]) for s, t < d: one CTA per (s, t),
// fixed-order block sum
__global__ void __launch_bounds__(256) reduced_density_kernel(int cl, int d, int cr, const double2* __restrict__ U,
                                                              const double2* __restrict__ A, double2* __restrict__ rho) {
    __shared__ double sh[2][8];
    const int s = blockIdx.x / d, t = blockIdx.x % d;
    double re = 0.0, im = 0.0;
    const long long n = (long long)cl * cr;
    for (long long e = threadIdx.x; e < n; e += blockDim.x) {
        const long long i = e / cr, c = e - (e / cr) * cr;
        const double2 u = U[(i * d + s) * cr + c], a = A[(i * d + t) * cr + c];
        re += u.x * a.x + u.y * a.y;
        im += u.y * a.x - u.x * a.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][wid] = re;
        sh[1][wid] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0, m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            r += sh[0][w];
            m += sh[1][w];
        }
        rho[blockIdx.x] = make_double2(r, m);
    }
}

}  // namespace

void fill_random_normal(Ctx& ctx, double2* out, long long count, uint64_t seed, int site, unsigned stream) {
    if (count <= 0) return;
    random_normal_kernel<<<(unsigned)((count + 255) / 256), 256, 0, ctx.stream>>>(
        out, count, (unsigned)(seed & 0xFFFFFFFFu), (unsigned)(seed >> 32), (unsigned)site, stream);
    ctx.count_launch();
    ctx.check_launch("random_normal_kernel");
}

void orthonormalize_rows_small(Ctx& ctx, double2* A, int rows, int cols, const int* pred) {
    VTN_REQUIRE(rows <= 4096 && rows <= cols, "row orthonormalisation needs rows <= min(cols, 4096)");
    const size_t shm = sizeof(double2) * (size_t)std::max(rows, 1);
    set_smem_attr_once(ctx, (const void*)orth_rows_kernel, 64 * 1024);
    orth_rows_kernel<<<1, 1024, shm, ctx.stream>>>(A, rows, cols, pred);
    ctx.count_launch();
    ctx.check_launch("orth_rows_kernel");
}

// Gram-Schmidt of the rows in order.  Small problems run the single-CTA kernel; from 128 rows
// and 2^25 complex multiply-adds on, CholeskyQR2 on the GEMM (same result, all SMs).
void orthonormalize_rows(Ctx& ctx, double2* A, int rows, int cols) {
    VTN_REQUIRE(rows <= 4096 && rows <= cols, "row orthonormalisation needs rows <= min(cols, 4096)");
    if (rows >= 128 && (double)rows * rows * cols >= 33554432.0) orthonormalize_rows_cholqr(ctx, A, rows, cols);
    else orthonormalize_rows_small(ctx, A, rows, cols, nullptr);
}

void lbo_rotate_dev(Ctx& ctx, int chi_l, int d, int D, int chi_r, const double2* V, const double2* A, double2* out) {
    const long long total = (long long)chi_l * D * chi_r;
    if (total == 0) return;
    lbo_rotate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, ctx.stream>>>(chi_l, d, D, chi_r, V, A, out);
    ctx.count_launch();
    ctx.check_launch("lbo_rotate_kernel");
}

void set_scalar_one(Ctx& ctx, double2* p) {
    set_one_kernel<<<1, 1, 0, ctx.stream>>>(p);
    ctx.count_launch();
}

void marginal_reduce_dev(Ctx& ctx, int chi_l, int D, int chi_r, const double2* AF, const double2* U, double* P) {
    marginal_reduce<<<D, 256, 0, ctx.stream>>>(chi_l, D, chi_r, AF, U, P);
    ctx.count_launch();
    ctx.check_launch("marginal_reduce");
}

void sample_dev(Ctx& ctx, const double2* const* AF_dev, const double2* const* ER_dev, const int* dims_dev, int M,
                int D, int chi_max, uint64_t seed, int n_samples, int* out_dev) {
    SampleArgs a;
    a.AF = AF_dev;
    a.ER = ER_dev;
    a.dims = dims_dev;
    a.M = M;
    a.D = D;
    a.k0 = (unsigned)(seed & 0xFFFFFFFFu);
    a.k1 = (unsigned)(seed >> 32);
    a.n_samples = n_samples;
    a.chi_max = chi_max;
    a.out = out_dev;
    const size_t shm = sizeof(double2) * (size_t)chi_max * (1 + D) + sizeof(double) * D;
    // the opt-in limit per block less the kernel's static shared memory
    int optin = 0;
    VTN_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx.device));
    cudaFuncAttributes fa;
    VTN_CUDA_TRY(cudaFuncGetAttributes(&fa, (const void*)sample_kernel));
    const size_t limit = (size_t)optin - fa.sharedSizeBytes;
    VTN_REQUIRE(shm <= limit, "sampler working set exceeds shared memory (chi_max * (D + 1) too large)");
    set_smem_attr_once(ctx, (const void*)sample_kernel, (int)limit);
    sample_kernel<<<n_samples, 256, shm, ctx.stream>>>(a);
    ctx.count_launch();
    ctx.check_launch("sample_kernel");
}

void reduced_density_dev(Ctx& ctx, int cl, int d, int cr, const double2* U, const double2* A, double2* rho) {
    reduced_density_kernel<<<d * d, 256, 0, ctx.stream>>>(cl, d, cr, U, A, rho);
    ctx.count_launch();
    ctx.check_launch("reduced_density_kernel");
}

}  // namespace vtn
