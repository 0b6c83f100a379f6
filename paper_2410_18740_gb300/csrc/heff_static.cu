// vtn_heff_apply_static: the two-site H_eff psi product for callers that must not
// allocate device memory -- for example a host application that owns every byte of GPU
// memory through its own pool under a fixed budget, or a latency-critical loop in which
// cudaMalloc / cudaFree (which can synchronise the whole device) are not acceptable.
//
// It runs the same kernels as vtn_heff_apply (complex GEMM, MPO-core mixing, complex GEMM)
// but takes every intermediate from one file-scope device array instead of a context's
// workspace, needs no context, and performs no allocation of any kind: the GEMMs never
// split their summation range (a split would need a partial-sum buffer), and the MPO cores'
// index tables and operators are packed into one file-scope host buffer and copied from
// there, in one copy, into the front of the same device array.  That host buffer is
// ordinary pageable memory, so the copy has taken its bytes when cudaMemcpyAsync returns:
// the caller's arrays are never read by a DMA that outlives the call.
//
// The array's device address is looked up once per device (cudaGetSymbolAddress with that
// device current) by the first call on that device; make that first call before any
// stream capture.  Every call shares the array and finds in it whatever the previous call
// left; each call writes every element it later reads, so nothing needs clearing, but
// calls whose GPU work overlaps (different streams, different threads) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "vtn_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;     // 32 MiB of static device memory
constexpr size_t kCoreRegion = size_t(1) << 20;        // first 1 MiB: both MPO cores
constexpr size_t kBufBytes = (kScratchBytes - kCoreRegion) / 2;
constexpr long long kBufComplex = (long long)(kBufBytes / sizeof(double2));  // 1,015,808
constexpr int kMaxW = 512;
constexpr int kMaxNnz = 4096;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_heff_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_base[kMaxDevices];  // device address of g_heff_scratch per device (0 = not looked up)

// index tables of one core, grouped by output column, in fixed-size storage
struct Tables {
    int col_ptr[kMaxW + 1];
    int col_src[kMaxNnz];
    int col_op[kMaxNnz];
    unsigned char ident[kMaxNnz];
};

// Host staging of both cores (guarded by g_mu from packing until the copy has returned).
struct HostStage {
    Tables t[2];
    alignas(256) unsigned char blob[kCoreRegion];
};
HostStage g_stage;

vtn_status check_core(const vtn_core* c) {
    if (!c || c->w_left < 1 || c->w_right < 1 || c->w_left > kMaxW || c->w_right > kMaxW) return VTN_EINVAL;
    if (c->d < 1 || c->d > 16 || c->nnz < 0 || c->nnz > kMaxNnz) return VTN_EINVAL;
    if (c->nnz > 0 && (!c->rows || !c->cols || !c->ops)) return VTN_EINVAL;
    for (int k = 0; k < c->nnz; ++k)
        if (c->rows[k] < 0 || c->rows[k] >= c->w_left || c->cols[k] < 0 || c->cols[k] >= c->w_right)
            return VTN_EINVAL;
    return VTN_OK;
}

void fill_tables(const vtn_core* c, Tables& t) {
    std::fill(t.col_ptr, t.col_ptr + c->w_right + 1, 0);
    for (int k = 0; k < c->nnz; ++k) t.col_ptr[c->cols[k] + 1]++;
    for (int b = 0; b < c->w_right; ++b) t.col_ptr[b + 1] += t.col_ptr[b];
    int next[kMaxW];
    std::copy(t.col_ptr, t.col_ptr + c->w_right, next);
    const int dd = c->d * c->d;
    for (int k = 0; k < c->nnz; ++k) {
        const int p = next[c->cols[k]]++;
        t.col_src[p] = c->rows[k];
        t.col_op[p] = k;
        const double* op = c->ops + 2 * (size_t)k * dd;
        bool id = true;
        for (int i = 0; i < c->d && id; ++i)
            for (int j = 0; j < c->d; ++j) {
                const double re = op[2 * (i * c->d + j)], im = op[2 * (i * c->d + j) + 1];
                if (i == j ? (re != op[0] || im != op[1]) : (re != 0.0 || im != 0.0)) {
                    id = false;
                    break;
                }
            }
        t.ident[k] = id ? 1 : 0;
    }
}

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

size_t core_bytes(const vtn_core* c) {
    return round256(sizeof(int) * (c->w_right + 1)) + 2 * round256(sizeof(int) * std::max(c->nnz, 1)) +
           round256(std::max(c->nnz, 1)) + round256(sizeof(double2) * std::max((size_t)c->nnz * c->d * c->d, size_t(1)));
}

// Packs one core into the host blob at offset `at` (the same layout the device copy gets at
// dev + at) and fills a DevCore view of the device copy.
void pack_core(const vtn_core* c, const Tables& t, unsigned char* blob, unsigned char* dev, size_t at,
               vtn::DevCore& dc) {
    size_t off = at;
    auto put = [&](const void* src, size_t bytes) -> unsigned char* {
        if (bytes) std::memcpy(blob + off, src, bytes);
        unsigned char* p = dev + off;
        off += round256(std::max(bytes, size_t(1)));
        return p;
    };
    const size_t nnz = (size_t)c->nnz;
    dc.col_ptr = (int*)put(t.col_ptr, sizeof(int) * (c->w_right + 1));
    dc.col_src = (int*)put(t.col_src, sizeof(int) * nnz);
    dc.col_op = (int*)put(t.col_op, sizeof(int) * nnz);
    dc.ident = put(t.ident, nnz);
    dc.ops = (double2*)put(c->ops, sizeof(double2) * nnz * c->d * c->d);
    dc.wl = c->w_left;
    dc.wr = c->w_right;
    dc.d = c->d;
    dc.nnz = c->nnz;
    int ni = 0;
    for (int k = 0; k < c->nnz; ++k) ni += t.ident[k];
    dc.n_ident = ni;
    dc.n_dense = c->nnz - ni;
}

}  // namespace

extern "C" vtn_status vtn_heff_apply_static(const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r,
                                            const double* L, const double* R, const double* theta, double* y,
                                            void* cuda_stream) {
    // ---- validation: nothing is queued unless every limit holds
    if (check_core(Wi) != VTN_OK || check_core(Wj) != VTN_OK) return VTN_EINVAL;
    if (Wi->w_right != Wj->w_left || Wi->d != Wj->d) return VTN_EINVAL;
    if (!L || !R || !theta || !y || (const double*)y == theta) return VTN_EINVAL;
    if (chi_l < 1 || chi_r < 1) return VTN_EINVAL;
    const int d = Wi->d;
    const long long n_theta = (long long)chi_l * d * d * chi_r;
    const long long wmax = std::max(Wi->w_left, std::max(Wi->w_right, Wj->w_right));
    if (n_theta > kBufComplex || wmax * n_theta > kBufComplex) return VTN_EINVAL;
    if (core_bytes(Wi) + core_bytes(Wj) > kCoreRegion) return VTN_EINVAL;
    // ---- set-up: device address of the static array, once per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VTN_ECUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_base[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_heff_scratch) != cudaSuccess || p == nullptr) {
                cudaGetLastError();
                return VTN_ECUDA;
            }
            g_base[dev] = (unsigned char*)p;
        }
        base = g_base[dev];
    }
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // ---- cores into the front of the array: packed on the host, one pageable copy
    vtn::DevCore ci, cj;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        fill_tables(Wi, g_stage.t[0]);
        fill_tables(Wj, g_stage.t[1]);
        const size_t bi = core_bytes(Wi);
        pack_core(Wi, g_stage.t[0], g_stage.blob, base, 0, ci);
        pack_core(Wj, g_stage.t[1], g_stage.blob, base, bi, cj);
        if (cudaMemcpyAsync(base, g_stage.blob, bi + core_bytes(Wj), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess) {
            cudaGetLastError();
            return VTN_ECUDA;
        }
    }
    double2* X = (double2*)(base + kCoreRegion);
    double2* Yb = (double2*)(base + kCoreRegion + kBufBytes);
    // ---- the product: same kernels as vtn_heff_apply, no split-K, no workspace, no timing
    try {
        vtn::Ctx c;
        c.device = dev;
        c.stream = stream;
        vtn::GemmArgs g1;
        g1.M = Wi->w_left * chi_l; g1.N = d * d * chi_r; g1.K = chi_l;
        g1.A = (const double2*)L; g1.lda = chi_l;
        g1.B = (const double2*)theta; g1.ldb = (long long)d * d * chi_r;
        g1.C = X; g1.ldc = (long long)d * d * chi_r;
        g1.max_splits = 1;
        vtn::gemm_c64(c, g1);
        vtn::mix_apply(c, ci, true, chi_l, d * chi_r, X, Yb);
        vtn::mix_apply(c, cj, true, chi_l * d, chi_r, Yb, X);
        vtn::GemmArgs g2;
        g2.M = chi_l * d * d; g2.N = chi_r; g2.K = chi_r; g2.kb = Wj->w_right;
        g2.A = X; g2.lda = chi_r; g2.sA_kb = n_theta;
        g2.B = (const double2*)R; g2.ldb = chi_r; g2.sB_kb = (long long)chi_r * chi_r;
        g2.C = (double2*)y; g2.ldc = chi_r;
        g2.max_splits = 1;
        vtn::gemm_c64(c, g2);
    } catch (const vtn::Error& e) {
        return e.status;
    }
    return VTN_OK;
}
