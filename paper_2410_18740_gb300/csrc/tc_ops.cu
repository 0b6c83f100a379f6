// Split-precision complex contractions on the tensor cores (precision mode VTN_BF16X3).
//
// A complex product C = op(A) op(B) (M x N, inner dimension Kt = kb * K) is evaluated as
// one real bf16 GEMM D = A~ B~^T of the tensor-core kernel:
//
//   real 2x2 block form      row m of A^ = [Re a(m,:), Im a(m,:)]
//                            rows 2n, 2n+1 of B^ = [Re b(:,n), -Im b(:,n)], [Im b(:,n), Re b(:,n)]
//                            so that (A^ B^T)[m][2n] = Re C, [m][2n+1] = Im C (interleaved output)
//   split precision          x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
//   three products           A_hi B_hi + A_hi B_lo + A_lo B_hi   (FP32 accumulation)
//
// Each split operand is stored as two halves along K, [X^_hi | X^_lo], each 2 Kt wide and
// zero padded to a multiple of 64; the GEMM loads the hi and lo tiles of A and B for a k-block
// once and issues the three products from them.  The packers read FP64 or FP32 complex data
// through 32 x 32 shared-memory tiles so that both the read and the write side are coalesced
// whatever the operand's transposition.
#include <cuda_bf16.h>

#include <algorithm>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

template <typename T>
struct CplxTraits;
template <>
struct CplxTraits<double2> {
    static __device__ __forceinline__ void split(double x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
        hi = __double2bfloat16(x);
        lo = __double2bfloat16(x - (double)__bfloat162float(hi));
    }
};
template <>
struct CplxTraits<float2> {
    static __device__ __forceinline__ void split(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
        hi = __float2bfloat16(x);
        lo = __float2bfloat16(x - __bfloat162float(hi));
    }
};

struct PackP {
    int rows;          // M (A) or N (B): output rows are rows (A) or 2 * rows (B)
    int K, kb;         // complex inner dimension per block and number of blocks; Kt = K * kb
    long long ld, s_kb;
    int conj_t;        // 1: operand used as X^dag
    int is_b;
    int rq;            // > 0: rows come in blocks of rq, block b starting at b * s_rq
    long long s_rq;
    __nv_bfloat16* out;
    long long ldo;
    long long half;    // columns of one half (ldo = 2 half)
};

// value of the operand element (r, kk) of op(X) as seen by the product:
//   A: r = m -> op(A)(m, kk);   B: r = n -> op(B)(kk, n)
template <typename T>
__device__ __forceinline__ T load_elem(const T* X, const PackP& p, int r, int kk) {
    const int c = kk / p.K, k = kk - c * p.K;
    const T* base = X + (long long)c * p.s_kb;
    long long rb = 0;
    int rr = r;
    if (p.rq > 0) {
        rb = (long long)(r / p.rq) * p.s_rq;
        rr = r - (r / p.rq) * p.rq;
    }
    // contiguous along kk: A with N, B with C; contiguous along r: A with C, B with N
    T v;
    if (p.is_b == p.conj_t) v = base[rb + (long long)rr * p.ld + k];
    else v = base[rb + (long long)k * p.ld + rr];
    if (p.conj_t) v.y = -v.y;
    return v;
}

template <typename T>
__global__ void __launch_bounds__(256) pack_kernel(const T* __restrict__ X, PackP p) {
    __shared__ T tile[32][33];
    const int Kt = p.K * p.kb;
    const int kk0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const bool along_kk = (p.is_b == p.conj_t);
    // load: make the fast thread index run along the contiguous source direction
    for (int t = threadIdx.y; t < 32; t += 8) {
        const int fast = threadIdx.x;
        const int r = along_kk ? r0 + t : r0 + fast;
        const int kk = along_kk ? kk0 + fast : kk0 + t;
        T v;
        v.x = 0;
        v.y = 0;
        if (r < p.rows && kk < Kt) v = load_elem(X, p, r, kk);
        if (along_kk) tile[t][fast] = v;
        else tile[fast][t] = v;
    }
    __syncthreads();
    // write: fast index along kk (the contiguous output direction)
    const int kk = kk0 + threadIdx.x;
    if (kk >= Kt) return;
    for (int t = threadIdx.y; t < 32; t += 8) {
        const int r = r0 + t;
        if (r >= p.rows) break;
        const T v = tile[t][threadIdx.x];
        __nv_bfloat16 rh, rl, ih, il;
        CplxTraits<T>::split(v.x, rh, rl);
        CplxTraits<T>::split(v.y, ih, il);
        const long long H = p.half;
        if (!p.is_b) {
            // row m: [Re a, Im a] hi | lo
            __nv_bfloat16* o = p.out + (long long)r * p.ldo;
            o[kk] = rh;
            o[Kt + kk] = ih;
            o[H + kk] = rl;
            o[H + Kt + kk] = il;
        } else {
            __nv_bfloat16* o0 = p.out + (long long)(2 * r) * p.ldo;
            __nv_bfloat16* o1 = o0 + p.ldo;
            // row 2n: [Re b, -Im b] hi | lo
            o0[kk] = rh;
            o0[Kt + kk] = __hneg(ih);
            o0[H + kk] = rl;
            o0[H + Kt + kk] = __hneg(il);
            // row 2n+1: [Im b, Re b] hi | lo
            o1[kk] = ih;
            o1[Kt + kk] = rh;
            o1[H + kk] = il;
            o1[H + Kt + kk] = rl;
        }
    }
}

// The A operand when the source rows run along kk (not conjugated, rows not blocked): row r of
// chunk c is K contiguous elements at X + c s_kb + r ld.  Each thread packs four consecutive kk
// of one row (blockIdx.y) with 16-byte loads and writes each of the four output streams as one
// 8-byte store; the values are those of pack_kernel.  Needs K % 4 == 0, even ld and s_kb, and a
// 16-byte aligned X.
template <typename T>
__device__ __forceinline__ void load4(const T* src, T v[4]);
template <>
__device__ __forceinline__ void load4<float2>(const float2* src, float2 v[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(src));
    const float4 b = __ldg(reinterpret_cast<const float4*>(src) + 1);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    v[2] = make_float2(b.x, b.y);
    v[3] = make_float2(b.z, b.w);
}
template <>
__device__ __forceinline__ void load4<double2>(const double2* src, double2 v[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __ldg(src + i);
}

__device__ __forceinline__ uint2 bf16x4(__nv_bfloat16 a, __nv_bfloat16 b, __nv_bfloat16 c, __nv_bfloat16 d) {
    uint2 u;
    u.x = (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
    u.y = (uint32_t)__bfloat16_as_ushort(c) | ((uint32_t)__bfloat16_as_ushort(d) << 16);
    return u;
}

template <typename T>
__global__ void __launch_bounds__(256) pack_rows4_kernel(const T* __restrict__ X, PackP p) {
    const int Kt = p.K * p.kb;
    const int kk = (int)(blockIdx.x * 256 + threadIdx.x) * 4;
    const int r = (int)blockIdx.y;
    if (kk >= Kt) return;
    const int c = kk / p.K, k = kk - c * p.K;
    T v[4];
    load4<T>(X + (long long)c * p.s_kb + (long long)r * p.ld + k, v);
    __nv_bfloat16 rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        CplxTraits<T>::split(v[i].x, rh[i], rl[i]);
        CplxTraits<T>::split(v[i].y, ih[i], il[i]);
    }
    // row m: [Re a, Im a] hi | lo
    __nv_bfloat16* o = p.out + (long long)r * p.ldo;
    const long long H = p.half;
    *reinterpret_cast<uint2*>(o + kk) = bf16x4(rh[0], rh[1], rh[2], rh[3]);
    *reinterpret_cast<uint2*>(o + Kt + kk) = bf16x4(ih[0], ih[1], ih[2], ih[3]);
    *reinterpret_cast<uint2*>(o + H + kk) = bf16x4(rl[0], rl[1], rl[2], rl[3]);
    *reinterpret_cast<uint2*>(o + H + Kt + kk) = bf16x4(il[0], il[1], il[2], il[3]);
}

__global__ void zero_pad_kernel(__nv_bfloat16* out, long long ldo, int rows, int from, int to) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int w = to - from;
    if (w <= 0 || t >= (long long)rows * w) return;
    const long long r = t / w;
    out[r * ldo + from + (t % w)] = __float2bfloat16(0.0f);
}

// out[b][p][s'][q] = sum_e op_e[s'][s] in[src_e][p][s][q] in FP32 (ops rounded to float).
// All threads of a CTA share the output channel b, so the channel's operators are staged
// in shared memory (as float2) in chunks, instead of being re-read by every thread.
constexpr int MIX_SH = 4096;  // float2 operator entries per chunk (32 KiB)

// element (channel c, p, s, q) of the mixing input sits at c * cs + p * ps + s * ss + q
struct MixIn {
    long long cs, ps, ss;
};

template <int DM>
__global__ void __launch_bounds__(256) mix_f32_kernel(int P, int d, int Q, MixIn st, const int* __restrict__ ptr,
                                                      const int* __restrict__ src, const int* __restrict__ opi,
                                                      const float2* __restrict__ ops,
                                                      const unsigned char* __restrict__ ident,
                                                      const float2* __restrict__ in, float2* __restrict__ out,
                                                      int accumulate) {
    __shared__ float2 op_sh[MIX_SH];
    __shared__ int src_sh[MIX_SH / 4];
    __shared__ unsigned char id_sh[MIX_SH / 4];
    const long long PQ = (long long)P * Q;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < PQ;
    const int b = blockIdx.y;
    const long long pp = active ? t / Q : 0, q = active ? t % Q : 0;
    const long long blk = PQ * d;
    const int dd = d * d;
    const int chunk = min(MIX_SH / dd, MIX_SH / 4);
    float2 acc[DM];
#pragma unroll
    for (int s = 0; s < DM; ++s) acc[s] = make_float2(0.f, 0.f);
    const int e_begin = ptr[b], e_end = ptr[b + 1];
    if (accumulate && e_begin == e_end) return;  // nothing to add to this channel
    for (int e0 = e_begin; e0 < e_end; e0 += chunk) {
        const int ne = min(chunk, e_end - e0);
        __syncthreads();
        for (int i = threadIdx.x; i < ne * dd; i += blockDim.x) {
            const int e = i / dd, j = i - e * dd;
            op_sh[i] = ops[(long long)opi[e0 + e] * dd + j];
        }
        for (int e = threadIdx.x; e < ne; e += blockDim.x) {
            src_sh[e] = src[e0 + e];
            id_sh[e] = ident[opi[e0 + e]];
        }
        __syncthreads();
        if (!active) continue;
        for (int e = 0; e < ne; ++e) {
            const float2* x = in + (long long)src_sh[e] * st.cs + pp * st.ps + q;
            const float2* op = op_sh + e * dd;
            if (id_sh[e]) {
                const float sr = op[0].x, si = op[0].y;
#pragma unroll
                for (int sp = 0; sp < DM; ++sp) {
                    if (sp < d) {
                        const float2 v = x[(long long)sp * st.ss];
                        acc[sp].x += sr * v.x - si * v.y;
                        acc[sp].y += sr * v.y + si * v.x;
                    }
                }
            } else {
                float2 xv[DM];
#pragma unroll
                for (int s = 0; s < DM; ++s) xv[s] = (s < d) ? x[(long long)s * st.ss] : make_float2(0.f, 0.f);
#pragma unroll
                for (int sp = 0; sp < DM; ++sp) {
                    if (sp >= d) continue;
#pragma unroll
                    for (int s = 0; s < DM; ++s) {
                        if (s < d) {
                            const float2 o = op[sp * d + s];
                            acc[sp].x += o.x * xv[s].x - o.y * xv[s].y;
                            acc[sp].y += o.x * xv[s].y + o.y * xv[s].x;
                        }
                    }
                }
            }
        }
    }
    if (!active) return;
    float2* y = out + (long long)b * blk + pp * d * Q + q;
#pragma unroll
    for (int sp = 0; sp < DM; ++sp) {
        if (sp < d) {
            if (accumulate) {
                const float2 o = y[(long long)sp * Q];
                acc[sp].x += o.x;
                acc[sp].y += o.y;
            }
            y[(long long)sp * Q] = acc[sp];
        }
    }
}

// The scaled-identity part of a collapse core as a channel GEMM: out[b][e] = sum_a C[a][b] in[a][e]
// for every element e of the standard layout (e = (p, s, q), contiguous per channel); C has row
// stride ldc (>= w_out), so that a block of columns of a wider C can be applied.
// Persistent: one CTA of 256 threads per SM walks element tiles of ET; C (w_in x w_out) stays in
// shared memory, and the next tile of every input channel is copied by cp.async into the second
// buffer while the current one is used.  Thread (tb, te) accumulates channels b = tb + 16 j
// (j < JB) and elements e = te + 16 i (i < EI) in registers, so each shared-memory load feeds
// JB or EI FMAs; a real C (the GBS couplings) takes 2 FMAs per complex product.
template <int JB, int EI, bool REAL_C>
__global__ void __launch_bounds__(256, 1) mix_cid_kernel(int w_in, int w_out, long long E, const float2* __restrict__ C,
                                                         int ldc, const float2* __restrict__ in,
                                                         float2* __restrict__ out) {
    constexpr int ET = 16 * EI;
    extern __shared__ float2 sh[];
    float2* Csh = sh;                                // [w_in][16 JB]
    float2* buf0 = Csh + (size_t)w_in * 16 * JB;     // [w_in][ET] x 2
    float2* buf1 = buf0 + (size_t)w_in * ET;
    const int wpad = 16 * JB;
    for (int t = threadIdx.x; t < w_in * wpad; t += blockDim.x) {
        const int a = t / wpad, b = t - (t / wpad) * wpad;
        Csh[t] = b < w_out ? C[(long long)a * ldc + b] : make_float2(0.f, 0.f);
    }
    const int tb = threadIdx.x & 15, te = threadIdx.x >> 4;
    const long long n_tiles = (E + ET - 1) / ET;
    // cp.async of tile `tile` into `dst`: rows a of ET float2, 16 bytes (2 elements) per thread
    // when every row starts 16-byte aligned (E even), else 8 bytes; zero-filled past E
    const bool pairs = (E & 1) == 0;
    auto load = [&](long long tile, float2* dst) {
        const long long e0 = tile * ET;
        if (pairs) {
            constexpr int per_row = ET / 2;
            for (int t = threadIdx.x; t < w_in * per_row; t += blockDim.x) {
                const int a = t / per_row, c = t - (t / per_row) * per_row;
                const long long e = e0 + 2 * c;
                const int bytes = e + 1 < E ? 16 : (e < E ? 8 : 0);
                const float2* g = in + (long long)a * E + (bytes > 0 ? e : 0);
                const unsigned s_addr = (unsigned)__cvta_generic_to_shared(dst + (size_t)a * ET + 2 * c);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(s_addr), "l"(g), "r"(bytes)
                             : "memory");
            }
        } else {
            for (int t = threadIdx.x; t < w_in * ET; t += blockDim.x) {
                const int a = t / ET, c = t - (t / ET) * ET;
                const long long e = e0 + c;
                const int bytes = e < E ? 8 : 0;
                const float2* g = in + (long long)a * E + (bytes > 0 ? e : 0);
                const unsigned s_addr = (unsigned)__cvta_generic_to_shared(dst + (size_t)a * ET + c);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s_addr), "l"(g), "r"(bytes)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    long long tile = blockIdx.x;
    if (tile < n_tiles) load(tile, buf0);
    int cur = 0;
    for (; tile < n_tiles; tile += gridDim.x) {
        const long long next = tile + gridDim.x;
        float2* bc = cur ? buf1 : buf0;
        float2* bn = cur ? buf0 : buf1;
        if (next < n_tiles) {
            load(next, bn);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();
        float2 acc[JB][EI];
#pragma unroll
        for (int j = 0; j < JB; ++j)
#pragma unroll
            for (int i = 0; i < EI; ++i) acc[j][i] = make_float2(0.f, 0.f);
        for (int a = 0; a < w_in; ++a) {
            float2 c[JB], x[EI];
#pragma unroll
            for (int j = 0; j < JB; ++j) c[j] = Csh[a * wpad + tb + 16 * j];
#pragma unroll
            for (int i = 0; i < EI; ++i) x[i] = bc[(size_t)a * ET + te + 16 * i];
#pragma unroll
            for (int j = 0; j < JB; ++j)
#pragma unroll
                for (int i = 0; i < EI; ++i) {
                    acc[j][i].x = fmaf(c[j].x, x[i].x, acc[j][i].x);
                    acc[j][i].y = fmaf(c[j].x, x[i].y, acc[j][i].y);
                    if (!REAL_C) {
                        acc[j][i].x = fmaf(-c[j].y, x[i].y, acc[j][i].x);
                        acc[j][i].y = fmaf(c[j].y, x[i].x, acc[j][i].y);
                    }
                }
        }
        const long long e0 = tile * ET;
#pragma unroll
        for (int j = 0; j < JB; ++j) {
            const int b = tb + 16 * j;
            if (b >= w_out) continue;
#pragma unroll
            for (int i = 0; i < EI; ++i) {
                const long long e = e0 + te + 16 * i;
                if (e < E) out[(long long)b * E + e] = acc[j][i];
            }
        }
        __syncthreads();  // the buffer just read is the next prefetch target
        cur ^= 1;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// out[b][l][k] = T[l][b][k]  (T: rows l, row length nb * nk)
__global__ void permute_blk(const double2* __restrict__ T, int nl, int nb, int nk, double2* __restrict__ out) {
    const long long cnt = (long long)nl * nb * nk;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= cnt) return;
    const int k = (int)(t % nk);
    const long long r = t / nk;
    const int l = (int)(r % nl), b = (int)(r / nl);
    out[t] = T[((long long)l * nb + b) * nk + k];
}

// largest dynamic shared memory a block may take on the context's device
int mix_smem_limit(const Ctx& ctx) {
    static int limit[64] = {0};
    const int dev = ctx.device;
    if (dev >= 0 && dev < 64 && limit[dev] > 0) return limit[dev];
    int optin = 0;
    VTN_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (dev >= 0 && dev < 64) limit[dev] = optin;
    return optin;
}

template <int JB, int EI, bool R>
void launch_mix_cid_t(Ctx& ctx, int bytes, unsigned grid, int w_in, int w_out, long long E, const float2* C, int ldc,
                      const float2* in, float2* out) {
    set_smem_attr_once(ctx, (const void*)mix_cid_kernel<JB, EI, R>, bytes);
    mix_cid_kernel<JB, EI, R><<<grid, 256, bytes, ctx.stream>>>(w_in, w_out, E, C, ldc, in, out);
    ctx.count_launch();
}

template <int JB>
void launch_mix_cid_j(Ctx& ctx, int EI, bool real_c, int bytes, unsigned grid, int w_in, int w_out, long long E,
                      const float2* C, int ldc, const float2* in, float2* out) {
    if (EI == 4) {
        if (real_c) launch_mix_cid_t<JB, 4, true>(ctx, bytes, grid, w_in, w_out, E, C, ldc, in, out);
        else launch_mix_cid_t<JB, 4, false>(ctx, bytes, grid, w_in, w_out, E, C, ldc, in, out);
    } else {
        if (real_c) launch_mix_cid_t<JB, 2, true>(ctx, bytes, grid, w_in, w_out, E, C, ldc, in, out);
        else launch_mix_cid_t<JB, 2, false>(ctx, bytes, grid, w_in, w_out, E, C, ldc, in, out);
    }
}

void launch_mix_cid(Ctx& ctx, int JB, int EI, bool real_c, int bytes, unsigned grid, int w_in, int w_out, long long E,
                    const float2* C, int ldc, const float2* in, float2* out) {
    switch (JB) {
        case 2: launch_mix_cid_j<2>(ctx, EI, real_c, bytes, grid, w_in, w_out, E, C, ldc, in, out); break;
        case 4: launch_mix_cid_j<4>(ctx, EI, real_c, bytes, grid, w_in, w_out, E, C, ldc, in, out); break;
        case 7: launch_mix_cid_j<7>(ctx, EI, real_c, bytes, grid, w_in, w_out, E, C, ldc, in, out); break;
        default: launch_mix_cid_j<8>(ctx, EI, real_c, bytes, grid, w_in, w_out, E, C, ldc, in, out); break;
    }
}

// row width of a split operand: two halves of 2 Kt columns, each padded to a multiple of 64
long long ksplit(long long Kt) { return 2 * (((2 * Kt + 63) / 64) * 64); }

template <typename T>
void pack_impl(Ctx& ctx, const T* X, int rows, int K, int kb, long long ld, long long s_kb, bool conj_t, bool is_b,
               __nv_bfloat16* out, int rq, long long s_rq) {
    const long long Kt = (long long)K * kb;
    const long long ldo = ksplit(Kt);
    PackP p;
    p.rows = rows;
    p.K = K;
    p.kb = kb;
    p.ld = ld;
    p.s_kb = s_kb;
    p.conj_t = conj_t ? 1 : 0;
    p.is_b = is_b ? 1 : 0;
    p.rq = rq;
    p.s_rq = s_rq;
    p.out = out;
    p.ldo = ldo;
    p.half = ldo / 2;
    const bool rows4 = !is_b && !conj_t && rq == 0 && K % 4 == 0 && ld % 2 == 0 && s_kb % 2 == 0 && rows <= 65535 &&
                       Kt <= (1LL << 30) && ((uintptr_t)X & 15) == 0 && ((uintptr_t)out & 7) == 0;
    if (rows4) {
        dim3 grid((unsigned)((Kt / 4 + 255) / 256), (unsigned)rows);
        pack_rows4_kernel<T><<<grid, 256, 0, ctx.stream>>>(X, p);
    } else {
        dim3 grid((unsigned)((Kt + 31) / 32), (unsigned)((rows + 31) / 32));
        VTN_REQUIRE(grid.y <= 65535, "pack: too many rows");
        pack_kernel<T><<<grid, dim3(32, 8), 0, ctx.stream>>>(X, p);
    }
    const int orows = is_b ? 2 * rows : rows;
    const int from = (int)(2 * Kt), to = (int)(ldo / 2);
    if (to > from) {
        // the padding of both halves
        const long long cnt = (long long)orows * (to - from);
        zero_pad_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(out, ldo, orows, from, to);
        zero_pad_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(out, ldo, orows, to + from, 2 * to);
        ctx.count_launch(2);
    }
    ctx.count_launch();
    ctx.check_launch(rows4 ? "pack_rows4_kernel" : "pack_kernel");
}

}  // namespace

long long tc_ksplit(long long Kt) { return ksplit(Kt); }

void tc_pack(Ctx& ctx, const double2* X, int rows, int K, int kb, long long ld, long long s_kb, bool conj_t, bool is_b,
             __nv_bfloat16* out, int rq, long long s_rq) {
    pack_impl<double2>(ctx, X, rows, K, kb, ld, s_kb, conj_t, is_b, out, rq, s_rq);
}

void tc_pack(Ctx& ctx, const float2* X, int rows, int K, int kb, long long ld, long long s_kb, bool conj_t, bool is_b,
             __nv_bfloat16* out, int rq, long long s_rq) {
    pack_impl<float2>(ctx, X, rows, K, kb, ld, s_kb, conj_t, is_b, out, rq, s_rq);
}

bool channel_gemm_f32(Ctx& ctx, int w_in, int w_out, long long E, const float2* C, int ldc, bool real_c,
                      const float2* in, float2* out) {
    if (E <= 0 || w_out <= 0) return true;
    const int limit = mix_smem_limit(ctx);
    for (int b0 = 0; b0 < w_out; b0 += 128) {
        const int wo = std::min(128, w_out - b0);
        const int jneed = (wo + 15) / 16;
        const int JB = jneed <= 2 ? 2 : jneed <= 4 ? 4 : jneed <= 7 ? 7 : 8;
        const size_t cbytes = sizeof(float2) * (size_t)w_in * 16 * JB;
        int EI = 4;
        if (cbytes + 2 * sizeof(float2) * (size_t)w_in * 64 > (size_t)limit) EI = 2;
        const size_t bytes = cbytes + 2 * sizeof(float2) * (size_t)w_in * 16 * EI;
        if (bytes > (size_t)limit) return false;
        const long long tiles = (E + 16 * EI - 1) / (16 * EI);
        const unsigned grid = (unsigned)std::min<long long>(tiles, std::max(ctx.num_sms, 1));
        launch_mix_cid(ctx, JB, EI, real_c, (int)bytes, grid, w_in, wo, E, C + b0, ldc, in, out + (long long)b0 * E);
        ctx.check_launch("mix_cid_kernel");
    }
    return true;
}

void mix_apply_f32(Ctx& ctx, const DevCore& core, bool by_col, int P, int Q, const float2* in, float2* out,
                   const long long* in_strides) {
    const int w_out = by_col ? core.wr : core.wl;
    const int d = core.d;
    const long long PQ = (long long)P * Q;
    if (PQ == 0) return;
    VTN_REQUIRE(w_out <= 65535, "too many MPO channels");
    dim3 grid((unsigned)((PQ + 255) / 256), w_out);
    const int* ptr = by_col ? core.col_ptr : core.row_ptr;  // reassigned to the dense-only lists of a collapse core
    const int* src = by_col ? core.col_src : core.row_src;
    const int* opi = by_col ? core.col_op : core.row_op;
    double fl = 8.0 * PQ * ((double)core.n_ident * d + (double)core.n_dense * d * d);
    MixIn st;
    st.cs = PQ * d;
    st.ps = (long long)d * Q;
    st.ss = Q;
    if (in_strides) {
        st.cs = in_strides[0];
        st.ps = in_strides[1];
        st.ss = in_strides[2];
    }
    int t = ctx.tbegin(TC_MIX, fl);
    VTN_REQUIRE(core.ops_f32 != nullptr, "FP32 mixing needs the core's FP32 operators");
    const int w_in = by_col ? core.wl : core.wr;
    const long long E = PQ * d;
    bool accumulate = false;
    if (core.has_cid && by_col && in_strides == nullptr && w_out <= 128) {
        // collapse core: the scaled identities as a channel GEMM, then the dense entries added
        const int jneed = (w_out + 15) / 16;
        const int JB = jneed <= 2 ? 2 : jneed <= 4 ? 4 : jneed <= 7 ? 7 : 8;
        const size_t cbytes = sizeof(float2) * (size_t)w_in * 16 * JB;
        const int limit = mix_smem_limit(ctx);
        int EI = 4;
        if (cbytes + 2 * sizeof(float2) * (size_t)w_in * 64 > (size_t)limit) EI = 2;
        const size_t bytes = cbytes + 2 * sizeof(float2) * (size_t)w_in * 16 * EI;
        if (bytes <= (size_t)limit) {
            const long long tiles = (E + 16 * EI - 1) / (16 * EI);
            const unsigned grid_c = (unsigned)std::min<long long>(tiles, std::max(ctx.num_sms, 1));
            launch_mix_cid(ctx, JB, EI, core.cid_real, (int)bytes, grid_c, w_in, w_out, E, core.cid, w_out, in, out);
            ctx.check_launch("mix_cid_kernel");
            ptr = core.dcol_ptr;
            src = core.dcol_src;
            opi = core.dcol_op;
            accumulate = true;
        }
    }
    if (d <= 4)
        mix_f32_kernel<4><<<grid, 256, 0, ctx.stream>>>(P, d, Q, st, ptr, src, opi, core.ops_f32, core.ident, in, out,
                                                        accumulate ? 1 : 0);
    else if (d <= 8)
        mix_f32_kernel<8><<<grid, 256, 0, ctx.stream>>>(P, d, Q, st, ptr, src, opi, core.ops_f32, core.ident, in, out,
                                                        accumulate ? 1 : 0);
    else
        mix_f32_kernel<16><<<grid, 256, 0, ctx.stream>>>(P, d, Q, st, ptr, src, opi, core.ops_f32, core.ident, in, out,
                                                         accumulate ? 1 : 0);
    ctx.count_launch();
    ctx.check_launch("mix_f32_kernel");
    ctx.tend(t);
}

// ----------------------------------------------------------------------------- H_eff
void heff_pack_envs(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, int chi_l, int chi_r, const double2* L,
                    const double2* R, HeffPacked& pk, const BondTerms* terms) {
    if (terms && terms->usable) {
        heff_pack_terms(ctx, *terms, chi_l, chi_r, L, R, pk);
        return;
    }
    pk.terms = nullptr;
    const int wl = Wi.wl, wr = Wj.wr;
    pk.chi_l = chi_l;
    pk.chi_r = chi_r;
    pk.wl = wl;
    pk.wr = wr;
    pk.ldL = ksplit(chi_l);
    pk.ldR = ksplit((long long)wr * chi_r);
    pk.L = (__nv_bfloat16*)ctx.workspace(WS_TC_L, sizeof(__nv_bfloat16) * (size_t)wl * chi_l * pk.ldL);
    pk.R = (__nv_bfloat16*)ctx.workspace(WS_TC_R, sizeof(__nv_bfloat16) * (size_t)2 * chi_r * pk.ldR);
    // A operand of T1 = L theta: rows (a, i), inner index j
    tc_pack(ctx, L, wl * chi_l, chi_l, 1, chi_l, 0, false, false, pk.L);
    // B operand of y = sum_c T3[c] R[c]: output column l, inner index (c, k): R[c][k][l]
    tc_pack(ctx, R, chi_r, chi_r, wr, chi_r, (long long)chi_r * chi_r, false, true, pk.R);
}

void heff_apply_bf16x3(Ctx& ctx, const DevCore& Wi, const DevCore& Wj, const HeffPacked& pk, const double2* theta,
                       double2* y) {
    if (pk.terms) {
        heff_apply_terms(ctx, pk, theta, y);
        return;
    }
    const int d = Wi.d, chi_l = pk.chi_l, chi_r = pk.chi_r;
    const long long n_theta = (long long)chi_l * d * d * chi_r;
    const int wmax = std::max(Wi.wl, std::max(Wi.wr, Wj.wr));
    const long long ldB1 = ksplit(chi_l);
    const long long ldA2 = ksplit((long long)Wj.wr * chi_r);
    __nv_bfloat16* B1 = (__nv_bfloat16*)ctx.workspace(WS_TC_B1, sizeof(__nv_bfloat16) * (size_t)2 * d * d * chi_r * ldB1);
    float2* X = (float2*)ctx.workspace(WS_X, sizeof(float2) * (size_t)wmax * n_theta);
    float2* Yb = (float2*)ctx.workspace(WS_Y, sizeof(float2) * (size_t)wmax * n_theta);
    __nv_bfloat16* A2 = (__nv_bfloat16*)ctx.workspace(WS_TC_A2, sizeof(__nv_bfloat16) * (size_t)chi_l * d * d * ldA2);
    const double useful1 = 8.0 * (double)Wi.wl * chi_l * (double)d * d * chi_r * chi_l;
    const double useful2 = 8.0 * (double)chi_l * d * d * chi_r * (double)chi_r * Wj.wr;
    // B operand of T1 = L theta: output column (s1 s2 k), inner index j: theta[j][(s1 s2 k)]
    tc_pack(ctx, theta, d * d * chi_r, chi_l, 1, (long long)d * d * chi_r, 0, false, true, B1);
    TcGemmArgs g1;
    g1.M = Wi.wl * chi_l;
    g1.N = 2 * d * d * chi_r;
    g1.K = (int)ldB1;
    g1.A = pk.L;
    g1.lda = pk.ldL;
    g1.B = B1;
    g1.ldb = ldB1;
    g1.D = X;
    g1.ldd = 2LL * d * d * chi_r;
    g1.d_fp64 = false;
    g1.split3 = true;
    g1.max_kb_per_acc = ctx.tc_kb_heff;
    tc_gemm_bf16(ctx, g1, TC_HEFF, useful1);
    mix_apply_f32(ctx, Wi, true, chi_l, d * chi_r, X, Yb);
    mix_apply_f32(ctx, Wj, true, chi_l * d, chi_r, Yb, X);
    // A operand of y = sum_c T3[c] R[c]: rows (i t u), inner index (c, k): T3[c][(i t u)][k]
    tc_pack(ctx, (const float2*)X, chi_l * d * d, chi_r, Wj.wr, chi_r, n_theta, false, false, A2);
    TcGemmArgs g2;
    g2.M = chi_l * d * d;
    g2.N = 2 * chi_r;
    g2.K = (int)ldA2;
    g2.A = A2;
    g2.lda = ldA2;
    g2.B = pk.R;
    g2.ldb = pk.ldR;
    g2.D = y;
    g2.ldd = 2LL * chi_r;
    g2.d_fp64 = true;
    g2.split3 = true;
    g2.max_kb_per_acc = ctx.tc_kb_heff;
    tc_gemm_bf16(ctx, g2, TC_HEFF, useful2);
}

// C = A B for complex FP64 A (M x K, row stride lda) and B (K x N, row stride ldb), C (M x N, row
// stride ldc) in FP64, as one split-precision tensor-core GEMM (used where the product feeds
// split-precision work only: the two-site tensor that starts a Lanczos solve)
void zgemm_bf16x3(Ctx& ctx, int M, int N, int K, const double2* A, long long lda, const double2* B, long long ldb,
                  double2* C, long long ldc) {
    const long long kk = ksplit(K);
    __nv_bfloat16* Ap = (__nv_bfloat16*)ctx.workspace(WS_TH_A, sizeof(__nv_bfloat16) * (size_t)M * kk);
    __nv_bfloat16* Bp = (__nv_bfloat16*)ctx.workspace(WS_TH_B, sizeof(__nv_bfloat16) * (size_t)2 * N * kk);
    tc_pack(ctx, A, M, K, 1, lda, 0, false, false, Ap);
    tc_pack(ctx, B, N, K, 1, ldb, 0, false, true, Bp);
    TcGemmArgs g;
    g.M = M;
    g.N = 2 * N;
    g.K = (int)kk;
    g.A = Ap;
    g.lda = kk;
    g.B = Bp;
    g.ldb = kk;
    g.D = C;
    g.ldd = 2 * ldc;
    g.d_fp64 = true;
    g.split3 = true;
    g.max_kb_per_acc = ctx.tc_kb_env;
    tc_gemm_bf16(ctx, g, -1, 8.0 * M * (double)N * K);
}

// ----------------------------------------------------------------------------- environments
// Split-precision (VTN_BF16X3) environment updates: the same three steps as the FP64
// versions (dense contraction, MPO mixing, dense contraction with the conjugate site
// tensor), with both dense steps on the tensor cores and the mixing in FP32.  Outputs are
// FP64.

// out[b][l][k] = sum_{a,i,j,s,t} conj(A[i][t][l]) L[a][i][j] W[a,b,t,s] A[j][s][k]
void env_left_bf16x3(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* L, const double2* A,
                     double2* out) {
    const int d = W.d, wl = W.wl, wr = W.wr;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(wl, wr);
    // 1. T[(a,i)][(s,k)] = sum_j L[a][i][j] A[j][(s,k)]
    const long long ld1 = ksplit(chi_l);
    __nv_bfloat16* PA = (__nv_bfloat16*)ctx.workspace(WS_TC_L, sizeof(__nv_bfloat16) * (size_t)wl * chi_l * ld1);
    __nv_bfloat16* PB = (__nv_bfloat16*)ctx.workspace(WS_TC_B1, sizeof(__nv_bfloat16) * (size_t)2 * d * chi_r * ld1);
    float2* X = (float2*)ctx.workspace(WS_X, sizeof(float2) * (size_t)wmax * nA);
    float2* Yb = (float2*)ctx.workspace(WS_Y, sizeof(float2) * (size_t)wmax * nA);
    tc_pack(ctx, L, wl * chi_l, chi_l, 1, chi_l, 0, false, false, PA);
    tc_pack(ctx, A, d * chi_r, chi_l, 1, (long long)d * chi_r, 0, false, true, PB);
    TcGemmArgs g1;
    g1.M = wl * chi_l;
    g1.N = 2 * d * chi_r;
    g1.K = (int)ld1;
    g1.A = PA;
    g1.lda = ld1;
    g1.B = PB;
    g1.ldb = ld1;
    g1.D = X;
    g1.ldd = 2LL * d * chi_r;
    g1.d_fp64 = false;
    g1.split3 = true;
    g1.max_kb_per_acc = ctx.tc_kb_env;
    tc_gemm_bf16(ctx, g1, -1, 8.0 * wl * chi_l * (double)chi_l * d * chi_r);
    // 2. U[b][i][t][k] = sum W[a,b,t,s] T[a][i][s][k]
    mix_apply_f32(ctx, W, true, chi_l, chi_r, X, Yb);
    // 3. D[l][(b,k)] = sum_{(i,t)} conj(A[(i,t)][l]) U[b][(i,t)][k], then out[b][l][k] = D[l][b][k]
    const long long ld3 = ksplit((long long)chi_l * d);
    __nv_bfloat16* PA3 = (__nv_bfloat16*)ctx.workspace(WS_TC_A2, sizeof(__nv_bfloat16) * (size_t)chi_r * ld3);
    __nv_bfloat16* PB3 = (__nv_bfloat16*)ctx.workspace(WS_TC_R, sizeof(__nv_bfloat16) * (size_t)2 * wr * chi_r * ld3);
    double2* T = (double2*)ctx.workspace(WS_TC_ENV, sizeof(double2) * (size_t)chi_r * wr * chi_r);
    tc_pack(ctx, A, chi_r, chi_l * d, 1, chi_r, 0, true, false, PA3);
    tc_pack(ctx, (const float2*)Yb, wr * chi_r, chi_l * d, 1, chi_r, 0, false, true, PB3, chi_r, nA);
    TcGemmArgs g3;
    g3.M = chi_r;
    g3.N = 2 * wr * chi_r;
    g3.K = (int)ld3;
    g3.A = PA3;
    g3.lda = ld3;
    g3.B = PB3;
    g3.ldb = ld3;
    g3.D = T;
    g3.ldd = 2LL * wr * chi_r;
    g3.d_fp64 = true;
    g3.split3 = true;
    g3.max_kb_per_acc = ctx.tc_kb_env;
    tc_gemm_bf16(ctx, g3, -1, 8.0 * chi_r * (double)wr * chi_r * chi_l * d);
    const long long cnt = (long long)wr * chi_r * chi_r;
    permute_blk<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx.stream>>>(T, chi_r, wr, chi_r, out);
    ctx.count_launch();
    ctx.check_launch("permute_blk");
}

// out[b][j][i] = sum_{c,g,p,s,t} A[j][s][g] R[c][g][p] W[b,c,t,s] conj(A[i][t][p])
void env_right_bf16x3(Ctx& ctx, const DevCore& W, int chi_l, int chi_r, const double2* R, const double2* A,
                      double2* out) {
    const int d = W.d, wl = W.wl, wr = W.wr;
    const long long nA = (long long)chi_l * d * chi_r;
    const int wmax = std::max(wl, wr);
    // 1. T[(j,s)][(c,p)] = sum_g A[(j,s)][g] R[c][g][p]
    const long long ld1 = ksplit(chi_r);
    __nv_bfloat16* PA = (__nv_bfloat16*)ctx.workspace(WS_TC_L, sizeof(__nv_bfloat16) * (size_t)chi_l * d * ld1);
    __nv_bfloat16* PB = (__nv_bfloat16*)ctx.workspace(WS_TC_R, sizeof(__nv_bfloat16) * (size_t)2 * wr * chi_r * ld1);
    float2* X = (float2*)ctx.workspace(WS_X, sizeof(float2) * (size_t)wmax * nA);
    float2* Yb = (float2*)ctx.workspace(WS_Y, sizeof(float2) * (size_t)wmax * nA);
    tc_pack(ctx, A, chi_l * d, chi_r, 1, chi_r, 0, false, false, PA);
    tc_pack(ctx, R, wr * chi_r, chi_r, 1, chi_r, 0, false, true, PB, chi_r, (long long)chi_r * chi_r);
    TcGemmArgs g1;
    g1.M = chi_l * d;
    g1.N = 2 * wr * chi_r;
    g1.K = (int)ld1;
    g1.A = PA;
    g1.lda = ld1;
    g1.B = PB;
    g1.ldb = ld1;
    g1.D = X;
    g1.ldd = 2LL * wr * chi_r;
    g1.d_fp64 = false;
    g1.split3 = true;
    g1.max_kb_per_acc = ctx.tc_kb_env;
    tc_gemm_bf16(ctx, g1, -1, 8.0 * chi_l * d * (double)wr * chi_r * chi_r);
    // 2. U[b][j][t][p] = sum W[b,c,t,s] T[c][j][s][p]; T element (c, j, s, p) sits at
    //    ((j d + s) wr + c) chi_r + p
    const long long st[3] = {chi_r, (long long)d * wr * chi_r, (long long)wr * chi_r};
    mix_apply_f32(ctx, W, false, chi_l, chi_r, X, Yb, st);
    // 3. out[(b,j)][i] = sum_{(t,p)} U[(b,j)][(t,p)] conj(A[i][(t,p)])
    const long long ld3 = ksplit((long long)d * chi_r);
    __nv_bfloat16* PA3 = (__nv_bfloat16*)ctx.workspace(WS_TC_A2, sizeof(__nv_bfloat16) * (size_t)wl * chi_l * ld3);
    __nv_bfloat16* PB3 = (__nv_bfloat16*)ctx.workspace(WS_TC_B1, sizeof(__nv_bfloat16) * (size_t)2 * chi_l * ld3);
    tc_pack(ctx, (const float2*)Yb, wl * chi_l, d * chi_r, 1, (long long)d * chi_r, 0, false, false, PA3);
    tc_pack(ctx, A, chi_l, d * chi_r, 1, (long long)d * chi_r, 0, true, true, PB3);
    TcGemmArgs g3;
    g3.M = wl * chi_l;
    g3.N = 2 * chi_l;
    g3.K = (int)ld3;
    g3.A = PA3;
    g3.lda = ld3;
    g3.B = PB3;
    g3.ldb = ld3;
    g3.D = out;
    g3.ldd = 2LL * chi_l;
    g3.d_fp64 = true;
    g3.split3 = true;
    g3.max_kb_per_acc = ctx.tc_kb_env;
    tc_gemm_bf16(ctx, g3, -1, 8.0 * wl * chi_l * (double)chi_l * d * chi_r);
}

}  // namespace vtn
