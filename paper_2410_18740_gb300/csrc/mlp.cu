// The multilayer perceptron of the learned warm start: FP32 training and inference kernels.
// Fully connected layers n_in -> width (x depth) -> n_out with ReLU between them, mean-squared
// error loss, back-propagation and the Adam update (Kingma and Ba 2015).  Every product is one
// strided FP32 GEMM kernel with a fused epilogue (bias, ReLU, or the ReLU mask of the layer
// below on the way back); each output is summed in a fixed order, so runs are reproducible.
//
// Parameters: one float array, per layer l: W_l (n_out_l x n_in_l, row-major), then b_l.
// Activations: x (B x n_in), h_l (B x width) for the hidden layers, y (B x n_out).
#include <algorithm>
#include <cmath>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

constexpr int MT = 64, NT = 64, KT = 16;  // block tile; 256 threads, 4 x 4 outputs each

struct SGemm {
    int M, N, K;
    const float* A; long long sam, sak;   // A(m, k) = A[m sam + k sak]
    const float* B; long long sbk, sbn;   // B(k, n) = B[k sbk + n sbn]
    float* C; long long ldc;
    const float* bias;                    // [N] or null
    int relu;                             // max(0, .) after the bias
    const float* mask; long long ldm;     // C[m][n] kept only where mask[m ldm + n] > 0 (or null)
};

__global__ void __launch_bounds__(256) sgemm_kernel(SGemm g) {
    __shared__ float As[KT][MT + 1];
    __shared__ float Bs[KT][NT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * MT, n0 = blockIdx.x * NT;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;
    for (int k0 = 0; k0 < g.K; k0 += KT) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = threadIdx.x + 256 * r;  // 0 .. 1023
            const int kk = e & (KT - 1), i = e >> 4;
            const int m = m0 + i, n = n0 + i, k = k0 + kk;
            As[kk][i] = (m < g.M && k < g.K) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : 0.0f;
            Bs[kk][i] = (n < g.N && k < g.K) ? g.B[(long long)k * g.sbk + (long long)n * g.sbn] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < KT; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty + 16 * r;
        if (m >= g.M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int n = n0 + tx + 16 * c;
            if (n >= g.N) continue;
            float v = acc[r][c];
            if (g.bias) v += g.bias[n];
            if (g.relu) v = fmaxf(v, 0.0f);
            if (g.mask && !(g.mask[(long long)m * g.ldm + n] > 0.0f)) v = 0.0f;
            g.C[(long long)m * g.ldc + n] = v;
        }
    }
}

// out[n] = sum_b G[b][n], b ascending
__global__ void colsum_kernel(int B, int N, const float* __restrict__ G, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.0f;
    for (int b = 0; b < B; ++b) s += G[(long long)b * N + n];
    out[n] = s;
}

// dY = 2 (Y - T) / count; loss = sum (Y - T)^2 / count (one block, fixed-order tree)
__global__ void __launch_bounds__(1024) mse_kernel(long long count, const float* __restrict__ Y,
                                                   const float* __restrict__ T, float* __restrict__ dY,
                                                   float* __restrict__ loss) {
    __shared__ float red[1024];
    const float inv = 1.0f / (float)count;
    float s = 0.0f;
    for (long long i = threadIdx.x; i < count; i += blockDim.x) {
        const float r = Y[i] - T[i];
        dY[i] = 2.0f * r * inv;
        s = fmaf(r, r, s);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 512; h >= 1; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = red[0] * inv;
}

__global__ void adam_kernel(long long n, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float c1, float c2, float b1, float b2,
                            float eps) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

void sgemm(Ctx& ctx, const SGemm& g) {
    if (g.M == 0 || g.N == 0) return;
    dim3 grid((unsigned)((g.N + NT - 1) / NT), (unsigned)((g.M + MT - 1) / MT));
    VTN_REQUIRE(grid.y <= 65535, "MLP batch too large");
    sgemm_kernel<<<grid, 256, 0, ctx.stream>>>(g);
    ctx.count_launch();
    ctx.check_launch("sgemm_kernel");
}

}  // namespace

MlpShape::MlpShape(int n_in_, int width_, int depth_, int n_out_)
    : n_in(n_in_), width(width_), depth(depth_), n_out(n_out_) {
    long long off = 0;
    for (int l = 0; l <= depth; ++l) {
        const int a = in_of(l), b = out_of(l);
        offW.push_back(off);
        off += (long long)a * b;
        offb.push_back(off);
        off += b;
    }
    n_params = off;
}

// y = net(x); the hidden activations go to acts (depth x B x width)
void mlp_forward_dev(Ctx& ctx, const MlpShape& s, const float* params, int B, const float* x, float* acts,
                     float* y) {
    const float* h = x;
    for (int l = 0; l <= s.depth; ++l) {
        const int a = s.in_of(l), b = s.out_of(l);
        const bool last = l == s.depth;
        float* out = last ? y : acts + (size_t)l * B * s.width;
        SGemm g{};
        g.M = B; g.N = b; g.K = a;
        g.A = h; g.sam = a; g.sak = 1;
        g.B = params + s.offW[l]; g.sbk = 1; g.sbn = a;        // B(k, n) = W[n][k]
        g.C = out; g.ldc = b;
        g.bias = params + s.offb[l];
        g.relu = last ? 0 : 1;
        sgemm(ctx, g);
        h = out;
    }
}

// loss (device scalar) and its gradient (device, n_params) for the batch (x, t)
void mlp_loss_grad_dev(Ctx& ctx, const MlpShape& s, const float* params, int B, const float* x, const float* t,
                       float* grad, float* loss) {
    const size_t wmax = (size_t)std::max(s.width, s.n_out);
    float* acts = (float*)ctx.workspace(WS_MLP_ACT, sizeof(float) * ((size_t)std::max(s.depth, 1) * B * s.width));
    float* y = (float*)ctx.workspace(WS_MLP_Y, sizeof(float) * (size_t)B * s.n_out);
    float* gbuf = (float*)ctx.workspace(WS_MLP_G, sizeof(float) * 2 * (size_t)B * wmax);
    mlp_forward_dev(ctx, s, params, B, x, acts, y);
    float* g = gbuf;                        // dloss/d(output of layer l)
    float* gnext = gbuf + (size_t)B * wmax;
    mse_kernel<<<1, 1024, 0, ctx.stream>>>((long long)B * s.n_out, y, t, g, loss);
    ctx.count_launch();
    for (int l = s.depth; l >= 0; --l) {
        const int a = s.in_of(l), b = s.out_of(l);
        const float* h = l == 0 ? x : acts + (size_t)(l - 1) * B * s.width;
        // dW_l[n][k] = sum_b g[b][n] h[b][k]
        SGemm gw{};
        gw.M = b; gw.N = a; gw.K = B;
        gw.A = g; gw.sam = 1; gw.sak = b;
        gw.B = h; gw.sbk = a; gw.sbn = 1;
        gw.C = grad + s.offW[l]; gw.ldc = a;
        sgemm(ctx, gw);
        colsum_kernel<<<(b + 255) / 256, 256, 0, ctx.stream>>>(B, b, g, grad + s.offb[l]);
        ctx.count_launch();
        if (l > 0) {
            // gnext[b][k] = (sum_n g[b][n] W_l[n][k]) where h[b][k] > 0
            SGemm gx{};
            gx.M = B; gx.N = a; gx.K = b;
            gx.A = g; gx.sam = b; gx.sak = 1;
            gx.B = params + s.offW[l]; gx.sbk = a; gx.sbn = 1;
            gx.C = gnext; gx.ldc = a;
            gx.mask = h; gx.ldm = a;
            sgemm(ctx, gx);
            std::swap(g, gnext);
        }
    }
    ctx.check_launch("mlp backward");
}

void mlp_adam_dev(Ctx& ctx, long long n, float* p, float* m, float* v, const float* g, float lr, long long step) {
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - std::pow(b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(b2, (double)step)));
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 4LL * ctx.num_sms));
    adam_kernel<<<grid, 256, 0, ctx.stream>>>(n, p, m, v, g, lr, c1, c2, (float)b1, (float)b2, 1e-8f);
    ctx.count_launch();
    ctx.check_launch("adam_kernel");
}

}  // namespace vtn
