// extern "C" entry points of libvtn (declared in include/vtn.h).
//
// The host code here only orchestrates: every arithmetic step of the solver (effective
// Hamiltonian products, Lanczos, eigendecomposition, environments, energy, marginals,
// sampling) is a kernel launched on the context's stream.  The host builds the MPO
// once (host_mpo.cpp) and reads back per-iteration status words and final scalars.
#include <algorithm>
#include <thread>
#include <atomic>
#include <complex>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "host_spectrum.h"
#include "vtn_internal.cuh"

using namespace vtn;

namespace {

// message of the calling thread's last failed call made without a context (vtn_create, the
// host-only MPO builders and queries)
thread_local std::string g_create_error;

template <class F>
vtn_status guard(vtn_ctx ctx, F&& f) {
    try {
        vtn_status s = f();
        if (ctx) {
            if (s == VTN_OK) ctx->c.err.clear();
        }
        return s;
    } catch (const Error& e) {
        if (ctx) ctx->c.err = e.msg;
        else g_create_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->c.err = "host allocation failed";
        else g_create_error = "host allocation failed";
        return VTN_ENOMEM;
    } catch (const std::exception& e) {
        if (ctx) ctx->c.err = e.what();
        else g_create_error = e.what();
        return VTN_EINVAL;
    }
}

void use_device(Ctx& c) { VTN_CUDA_TRY(cudaSetDevice(c.device)); }

void free_mpo_device(Ctx& c, vtn_mpo mpo) {
    for (auto& dc : mpo->dcores) free_core(c, dc);
    for (auto& bt : mpo->bterms) free_bond_terms(c, bt);
}

// Device term form of bond s, built on its first use: the host factorisation and upload take a
// couple of milliseconds a bond, so a windowed sweep pays only for the bonds it visits.  Not
// thread-safe: callers that share an MPO between threads build every bond first.
const BondTerms& mpo_bond_terms(Ctx& c, vtn_mpo mpo, int s) {
    BondTerms& bt = mpo->bterms[s];
    if (!bt.built) {
        build_bond_terms(c, mpo->hp.cores[s], mpo->hp.cores[s + 1], bt);
        bt.built = true;
    }
    return bt;
}

void ensure_mpo_device(vtn_ctx ctx, vtn_mpo mpo) {
    VTN_REQUIRE(mpo != nullptr, "null MPO");
    if (!mpo->dcores.empty()) {
        VTN_REQUIRE(mpo->owner == ctx, "MPO is resident on another context");
        return;
    }
    Ctx& c = ctx->c;
    mpo->dcores.resize(mpo->hp.M);
    for (int s = 0; s < mpo->hp.M; ++s) upload_core(c, mpo->hp.cores[s], mpo->dcores[s]);
    mpo->bterms.resize(std::max(mpo->hp.M - 1, 0));  // built on first use (mpo_bond_terms)
    const size_t iso_bytes = sizeof(double2) * mpo->hp.iso.size();
    mpo->iso_dev = (double2*)c.dalloc(iso_bytes);
    VTN_CUDA_TRY(cudaMemcpyAsync(mpo->iso_dev, mpo->hp.iso.data(), iso_bytes, cudaMemcpyHostToDevice, c.stream));
    c.sync();
    mpo->owner = ctx;
    mpo->device = c.device;
}

long long safe_pow_min(int d, int e, long long cap) {
    long long v = 1;
    for (int i = 0; i < e; ++i) {
        v *= d;
        if (v >= cap) return cap;
    }
    return v;
}

std::vector<int> bond_dims(int M, int d, int chi) {
    std::vector<int> dims(M + 1);
    for (int s = 0; s <= M; ++s) {
        long long a = safe_pow_min(d, s, chi), b = safe_pow_min(d, M - s, chi);
        dims[s] = (int)std::min<long long>(chi, std::min(a, b));
    }
    return dims;
}

// capacity per cut: chi_cap inside the chain, 1 at the two ends
std::vector<int> cap_dims(int M, int chi_cap) {
    std::vector<int> v(M + 1, chi_cap);
    v[0] = 1;
    v[M] = 1;
    return v;
}

// site buffers able to hold chi_cap x d x chi_cap (content preserved)
void mps_reserve(Ctx& c, vtn_mps mps, int chi_cap) {
    for (int x : mps->dims) chi_cap = std::max(chi_cap, x);
    if (chi_cap <= mps->chi_cap && (int)mps->sites.size() == mps->M) return;
    std::vector<int> cd = cap_dims(mps->M, chi_cap);
    mps->sites.resize(mps->M, nullptr);
    mps->cap.resize(mps->M, 0);
    for (int s = 0; s < mps->M; ++s) {
        size_t need = (size_t)cd[s] * mps->d * cd[s + 1];
        if (need <= mps->cap[s]) continue;
        double2* nb = (double2*)c.dalloc(sizeof(double2) * need);
        if (mps->sites[s]) {
            VTN_CUDA_TRY(cudaMemcpyAsync(nb, mps->sites[s],
                                         sizeof(double2) * (size_t)mps->dims[s] * mps->d * mps->dims[s + 1],
                                         cudaMemcpyDeviceToDevice, c.stream));
            c.sync();
            c.dfree(mps->sites[s]);
        }
        mps->sites[s] = nb;
        mps->cap[s] = need;
    }
    mps->chi_cap = chi_cap;
}

vtn_mps new_mps(vtn_ctx ctx, int M, int d, const std::vector<int>& dims) {
    vtn_mps m = new vtn_mps_s();
    m->M = M;
    m->d = d;
    m->dims = dims;
    m->owner = ctx;
    m->chi_cap = 0;
    int chi = 1;
    for (int x : dims) chi = std::max(chi, x);
    try {
        mps_reserve(ctx->c, m, chi);
    } catch (...) {
        for (auto p : m->sites) ctx->c.dfree(p);
        delete m;
        throw;
    }
    return m;
}

void destroy_mps(vtn_mps m) {
    if (!m) return;
    if (m->owner) {
        for (auto p : m->sites) m->owner->c.dfree(p);
    }
    delete m;
}

// A core uploaded for the duration of one call (kernel-level entry points).
struct TempCore {
    Ctx* c;
    DevCore dc;
    TempCore(Ctx& ctx, const HostCore& h) : c(&ctx) { upload_core(ctx, h, dc); }
    ~TempCore() {
        if (c) {
            cudaStreamSynchronize(c->stream);
            free_core(*c, dc);
        }
    }
};

// The term form of a bond given as two cores, for the duration of one call.
struct TempTerms {
    Ctx* c;
    BondTerms bt;
    TempTerms(Ctx& ctx, const HostCore& a, const HostCore& b) : c(&ctx) { build_bond_terms(ctx, a, b, bt); }
    ~TempTerms() {
        if (c) {
            cudaStreamSynchronize(c->stream);
            free_bond_terms(*c, bt);
        }
    }
};

// batched left transfer: Eout[t] = sum_s A[:,s,:]^dag E[t] A[:,s,:], t < count
void transfer_left_batch(Ctx& c, int count, int chi_l, int d, int chi_r, const double2* E, const double2* A,
                         double2* Eout, double2* tmp) {
    GemmArgs g1;
    g1.M = chi_l; g1.N = d * chi_r; g1.K = chi_l; g1.batch = count;
    g1.A = E; g1.lda = chi_l; g1.sA_batch = (long long)chi_l * chi_l;
    g1.B = A; g1.ldb = (long long)d * chi_r; g1.sB_batch = 0;
    g1.C = tmp; g1.ldc = (long long)d * chi_r; g1.sC_batch = (long long)chi_l * d * chi_r;
    gemm_c64(c, g1);
    GemmArgs g2;
    g2.M = chi_r; g2.N = chi_r; g2.K = chi_l * d; g2.batch = count;
    g2.opA = OP_C; g2.A = A; g2.lda = chi_r; g2.sA_batch = 0;
    g2.B = tmp; g2.ldb = chi_r; g2.sB_batch = (long long)chi_l * d * chi_r;
    g2.C = Eout; g2.ldc = chi_r; g2.sC_batch = (long long)chi_r * chi_r;
    gemm_c64(c, g2);
}

// right transfer: Eout[b][b'] = sum A[b s g] E[g][g'] conj(A[b' s g'])
void transfer_right(Ctx& c, int chi_l, int d, int chi_r, const double2* E, const double2* A, double2* Eout,
                    double2* tmp) {
    GemmArgs g1;
    g1.M = chi_l * d; g1.N = chi_r; g1.K = chi_r;
    g1.A = A; g1.lda = chi_r;
    g1.B = E; g1.ldb = chi_r;
    g1.C = tmp; g1.ldc = chi_r;
    gemm_c64(c, g1);
    GemmArgs g2;
    g2.M = chi_l; g2.N = chi_l; g2.K = d * chi_r;
    g2.A = tmp; g2.lda = (long long)d * chi_r;
    g2.opB = OP_C; g2.B = A; g2.ldb = (long long)d * chi_r;
    g2.C = Eout; g2.ldc = chi_l;
    gemm_c64(c, g2);
}

int max_dim(const std::vector<int>& v) {
    int m = 1;
    for (int x : v) m = std::max(m, x);
    return m;
}

double read_scalar_re(Ctx& c, const double2* p) {
    VTN_CUDA_TRY(cudaMemcpyAsync(c.pinned, p, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    return c.pinned[0];
}

double mps_norm2(Ctx& c, vtn_mps mps) {
    const int chi = max_dim(mps->dims);
    const size_t env = (size_t)chi * chi;
    double2* E0 = (double2*)c.workspace(WS_Z, sizeof(double2) * env * 2);
    double2* E1 = E0 + env;
    double2* tmp = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)chi * mps->d * chi);
    set_scalar_one(c, E0);
    for (int s = 0; s < mps->M; ++s) {
        transfer_left_batch(c, 1, mps->dims[s], mps->d, mps->dims[s + 1], E0, mps->sites[s], E1, tmp);
        std::swap(E0, E1);
    }
    return read_scalar_re(c, E0);
}

double energy_dev(Ctx& c, vtn_mpo mpo, vtn_mps mps) {
    int wmax = 1;
    for (int w : mpo->hp.w) wmax = std::max(wmax, w);
    const int chi = max_dim(mps->dims);
    const size_t env = (size_t)wmax * chi * chi;
    double2* L0 = (double2*)c.workspace(WS_Z, sizeof(double2) * env * 2);
    double2* L1 = L0 + env;
    set_scalar_one(c, L0);
    for (int s = 0; s < mps->M; ++s) {
        env_left_dev(c, mpo->dcores[s], mps->dims[s], mps->dims[s + 1], L0, mps->sites[s], L1);
        std::swap(L0, L1);
    }
    const double e = read_scalar_re(c, L0);
    const double n2 = mps_norm2(c, mps);
    return e / n2;
}

// (E, <H^2>) by the FP64 two-layer environment contraction, both divided by <psi|psi>
std::pair<double, double> energy_h2_dev(Ctx& c, vtn_mpo mpo, vtn_mps mps) {
    int wmax = 1;
    for (int w : mpo->hp.w) wmax = std::max(wmax, w);
    const int chi = max_dim(mps->dims);
    const int d = mps->d;
    const double env = (double)wmax * wmax * chi * chi;
    const double na = (double)chi * d * chi;
    const double bytes = 16.0 * (2.0 * env + 2.0 * (double)wmax * wmax * na);
    VTN_REQUIRE(bytes <= 24.0 * (1ull << 30),
                "energy variance: the two-layer environments would need more than 24 GiB of device memory");
    double2* L0 = (double2*)c.workspace(WS_H2_ENV, sizeof(double2) * (size_t)(2 * env));
    double2* L1 = L0 + (size_t)env;
    double2* tv = (double2*)c.workspace(WS_X, sizeof(double2) * (size_t)((double)wmax * wmax * na));
    double2* u = (double2*)c.workspace(WS_Y, sizeof(double2) * (size_t)((double)wmax * wmax * na));
    set_scalar_one(c, L0);
    for (int s = 0; s < mps->M; ++s) {
        env_left2_dev(c, mpo->dcores[s], mps->dims[s], mps->dims[s + 1], L0, mps->sites[s], L1, tv, u);
        std::swap(L0, L1);
    }
    const double h2 = read_scalar_re(c, L0);
    const double n2 = mps_norm2(c, mps);
    const double e = energy_dev(c, mpo, mps);
    return {e, h2 / n2};
}

struct Envs {
    Ctx* c = nullptr;
    std::vector<double2*> L, R;
    ~Envs() {
        if (!c) return;
        cudaStreamSynchronize(c->stream);
        for (auto p : L) c->dfree(p);
        for (auto p : R) c->dfree(p);
    }
};

// Exact split of bond (i, i+1): theta = A_i A_i+1 factored by the truncation eigensolver
// keeping k = the current bond dimension (rank(theta) <= k, so nothing is dropped).
// dir 0: site i left-canonical, the centre moves to i+1; dir 1: site i+1 right-canonical,
// the centre moves to i.
void exact_split(Ctx& c, vtn_mps mps, int i, int dir) {
    const int d = mps->d, cl = mps->dims[i], cm = mps->dims[i + 1], cr = mps->dims[i + 2];
    double2* theta = (double2*)c.workspace(WS_VEC_T, sizeof(double2) * (size_t)cl * d * d * cr);
    GemmArgs g;
    g.M = cl * d; g.N = d * cr; g.K = cm;
    g.A = mps->sites[i]; g.lda = cm;
    g.B = mps->sites[i + 1]; g.ldb = (long long)d * cr;
    g.C = theta; g.ldc = (long long)d * cr;
    gemm_c64(c, g);
    TruncResult tr = truncate_dev(c, cl, d, d, cr, dir, cm, theta, mps->sites[i], mps->sites[i + 1]);
    mps->dims[i + 1] = tr.k;
}

void move_center(Ctx& c, vtn_mps mps, int target) {
    const int M = mps->M;
    if (mps->center < 0 || mps->center >= M) {
        for (int i = M - 2; i >= 0; --i) exact_split(c, mps, i, 1);
        mps->center = 0;
    }
    while (mps->center < target) {
        exact_split(c, mps, mps->center, 0);
        ++mps->center;
    }
    while (mps->center > target) {
        exact_split(c, mps, mps->center - 1, 1);
        --mps->center;
    }
}

void check_mps_matches(vtn_mpo mpo, vtn_mps mps) {
    VTN_REQUIRE(mps != nullptr, "null MPS");
    VTN_REQUIRE(mps->M == mpo->hp.M && mps->d == mpo->hp.d, "MPS does not match the MPO (M or d)");
}

}  // namespace

// =====================================================================================
extern "C" {

vtn_status vtn_create(vtn_ctx* out, int device, void* cuda_stream, const vtn_allocator* allocator) {
    if (!out) return VTN_EINVAL;
    vtn_ctx ctx = nullptr;
    vtn_status st = guard(nullptr, [&]() -> vtn_status {
        int n = 0;
        VTN_CUDA_TRY(cudaGetDeviceCount(&n));
        VTN_REQUIRE(device >= 0 && device < n, "device index out of range");
        VTN_CUDA_TRY(cudaSetDevice(device));
        ctx = new vtn_ctx_s();
        Ctx& c = ctx->c;
        c.device = device;
        c.stream = (cudaStream_t)cuda_stream;
        if (allocator && allocator->alloc && allocator->free) {
            c.alloc = *allocator;
            c.has_alloc = true;
        }
        VTN_CUDA_TRY(cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, device));
        VTN_CUDA_TRY(cudaMallocHost((void**)&c.pinned, sizeof(double) * 4096));
        c.ws.resize(WS_COUNT);
        c.dstatus = (int*)c.dalloc(256);
        VTN_CUDA_TRY(cudaMemsetAsync(c.dstatus, 0, 256, c.stream));
        c.sync();
        return VTN_OK;
    });
    if (st != VTN_OK) {
        if (ctx) {
            if (ctx->c.dstatus) ctx->c.dfree(ctx->c.dstatus);
            if (ctx->c.pinned) cudaFreeHost(ctx->c.pinned);
            delete ctx;
        }
        return st;
    }
    *out = ctx;
    return VTN_OK;
}

vtn_status vtn_destroy(vtn_ctx ctx) {
    if (!ctx) return VTN_EINVAL;
    Ctx& c = ctx->c;
    cudaSetDevice(c.device);
    cudaStreamSynchronize(c.stream);
    for (auto& b : c.ws) c.dfree(b.p);
    c.dfree(c.dstatus);
    for (auto& p : c.pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c.event_pool) cudaEventDestroy(e);
    if (c.pinned) cudaFreeHost(c.pinned);
    if (c.defer_buf) cudaFreeHost(c.defer_buf);
    delete ctx;
    return VTN_OK;
}

const char* vtn_last_error(vtn_ctx ctx) {
    if (!ctx) return g_create_error.c_str();
    return ctx->c.err.c_str();
}

vtn_status vtn_launch_count(vtn_ctx ctx, long long* out) {
    if (!ctx || !out) return VTN_EINVAL;
    *out = ctx->c.launches;
    return VTN_OK;
}

// ------------------------------------------------------------------ MPO
vtn_status vtn_build_mpo(vtn_ctx ctx, int M, const double* r, const double* U, int D, int d, unsigned flags,
                         vtn_mpo* out) {
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out && r && U, "null argument");
        vtn_mpo mpo = new vtn_mpo_s();
        std::string err = build_problem(M, r, U, D, d, (flags & VTN_FLAG_LBO) != 0, mpo->hp);
        if (!err.empty()) {
            delete mpo;
            throw Error{VTN_EINVAL, err};
        }
        if (ctx) {
            try {
                use_device(ctx->c);
                ensure_mpo_device(ctx, mpo);
            } catch (...) {
                free_mpo_device(ctx->c, mpo);
                delete mpo;
                throw;
            }
        }
        *out = mpo;
        return VTN_OK;
    });
}

vtn_status vtn_build_mpo_cz(vtn_ctx ctx, int M, const double* r, const double* U, int D, double kappa,
                            vtn_mpo* out) {
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out && r && U, "null argument");
        vtn_mpo mpo = new vtn_mpo_s();
        std::string err = build_problem_cz(M, r, U, D, kappa, mpo->hp);
        if (!err.empty()) {
            delete mpo;
            throw Error{VTN_EINVAL, err};
        }
        if (ctx) {
            try {
                use_device(ctx->c);
                ensure_mpo_device(ctx, mpo);
            } catch (...) {
                free_mpo_device(ctx->c, mpo);
                delete mpo;
                throw;
            }
        }
        *out = mpo;
        return VTN_OK;
    });
}

vtn_status vtn_mpo_free(vtn_mpo mpo) {
    if (!mpo) return VTN_EINVAL;
    if (mpo->owner) {
        Ctx& c = mpo->owner->c;
        cudaStreamSynchronize(c.stream);
        free_mpo_device(c, mpo);
        c.dfree(mpo->iso_dev);
    }
    delete mpo;
    return VTN_OK;
}

vtn_status vtn_mpo_from_cores(vtn_ctx ctx, int M, const vtn_core* cores, vtn_mpo* out) {
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out && cores, "null argument");
        VTN_REQUIRE(M >= 1, "M must be >= 1");
        HostProblem hp;
        for (int s = 0; s < M; ++s) hp.cores.push_back(core_from_abi(&cores[s]));
        const int d = hp.cores[0].d;
        VTN_REQUIRE(hp.cores[0].wl == 1 && hp.cores[M - 1].wr == 1, "the end cores must have one outer channel");
        for (int s = 0; s < M; ++s) {
            VTN_REQUIRE(hp.cores[s].d == d, "all cores must have the same d");
            if (s + 1 < M) VTN_REQUIRE(hp.cores[s].wr == hp.cores[s + 1].wl, "core channel counts do not chain");
        }
        hp.M = M;
        hp.d = hp.D = d;
        hp.lbo = false;
        hp.w.assign(M + 1, 1);
        for (int s = 0; s < M; ++s) hp.w[s + 1] = hp.cores[s].wr;
        hp.iso.assign((size_t)M * d * d, cplx(0.0, 0.0));  // identity basis (no local basis)
        for (int s = 0; s < M; ++s)
            for (int n = 0; n < d; ++n) hp.iso[(size_t)s * d * d + (size_t)n * d + n] = cplx(1.0, 0.0);
        hp.norm_bound = 0.0;  // unknown
        vtn_mpo mpo = new vtn_mpo_s();
        mpo->hp = std::move(hp);
        if (ctx) {
            try {
                use_device(ctx->c);
                ensure_mpo_device(ctx, mpo);
            } catch (...) {
                free_mpo_device(ctx->c, mpo);
                delete mpo;
                throw;
            }
        }
        *out = mpo;
        return VTN_OK;
    });
}

vtn_status vtn_gaussian_bond_spectrum(vtn_mpo mpo, int cut, int k, double* out) {
    return guard(nullptr, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && out, "null argument");
        VTN_REQUIRE(k >= 1 && k <= (1 << 20), "k must be in [1, 2^20]");
        VTN_REQUIRE(cut >= 0 && cut <= mpo->hp.M, "cut must be in [0, M]");
        if (mpo->hp.V.empty()) throw Error{VTN_EUNSUPPORTED, "the MPO carries no covariance (given as cores)"};
        if (mpo->hp.kappa != 0.0) throw Error{VTN_EUNSUPPORTED, "the state of this MPO is not Gaussian"};
        const std::vector<double> spec = gaussian_bond_spectrum(mpo->hp.V, mpo->hp.M, cut, k);
        std::copy(spec.begin(), spec.end(), out);
        return VTN_OK;
    });
}

vtn_status vtn_gaussian_bond_dims(vtn_mpo mpo, double eps, int chi_max, int* dims) {
    return guard(nullptr, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && dims, "null argument");
        VTN_REQUIRE(std::isfinite(eps) && eps >= 0.0 && eps < 1.0, "eps must be in [0, 1)");
        VTN_REQUIRE(chi_max >= 1 && chi_max <= (1 << 20), "chi_max must be in [1, 2^20]");
        if (mpo->hp.V.empty()) throw Error{VTN_EUNSUPPORTED, "the MPO carries no covariance (given as cores)"};
        if (mpo->hp.kappa != 0.0) throw Error{VTN_EUNSUPPORTED, "the state of this MPO is not Gaussian"};
        const int M = mpo->hp.M;
        const std::vector<int> cap = bond_dims(M, mpo->hp.d, chi_max);
        for (int s = 0; s <= M; ++s) {
            const std::vector<double> spec = gaussian_bond_spectrum(mpo->hp.V, M, s, cap[s]);
            double kept = 0.0;
            int k = cap[s];
            for (int i = 0; i < cap[s]; ++i) {
                kept += spec[i];
                if (1.0 - kept <= eps) {
                    k = i + 1;
                    break;
                }
            }
            dims[s] = std::max(1, k);
        }
        return VTN_OK;
    });
}

vtn_status vtn_mpo_info(vtn_mpo mpo, int* M, int* d, int* D, int* w) {
    if (!mpo) return VTN_EINVAL;
    if (M) *M = mpo->hp.M;
    if (d) *d = mpo->hp.d;
    if (D) *D = mpo->hp.D;
    if (w) std::copy(mpo->hp.w.begin(), mpo->hp.w.end(), w);
    return VTN_OK;
}

vtn_status vtn_mpo_coefficients(vtn_mpo mpo, double* G) {
    if (!mpo || !G) return VTN_EINVAL;
    if (mpo->hp.G.empty()) return VTN_EUNSUPPORTED;  // MPO given as cores
    std::copy(mpo->hp.G.begin(), mpo->hp.G.end(), G);
    return VTN_OK;
}

vtn_status vtn_mpo_covariance(vtn_mpo mpo, double* V) {
    if (!mpo || !V) return VTN_EINVAL;
    if (mpo->hp.V.empty()) return VTN_EUNSUPPORTED;  // MPO given as cores
    std::copy(mpo->hp.V.begin(), mpo->hp.V.end(), V);
    return VTN_OK;
}

vtn_status vtn_mpo_isometry(vtn_mpo mpo, int site, double* V) {
    if (!mpo || !V || site < 0 || site >= mpo->hp.M) return VTN_EINVAL;
    const size_t n = (size_t)mpo->hp.D * mpo->hp.d;
    std::memcpy(V, mpo->hp.iso.data() + (size_t)site * n, sizeof(double) * 2 * n);
    return VTN_OK;
}

vtn_status vtn_mpo_core(vtn_mpo mpo, int site, int* nnz, int* rows, int* cols, double* ops) {
    if (!mpo || !nnz || site < 0 || site >= mpo->hp.M) return VTN_EINVAL;
    const HostCore& h = mpo->hp.cores[site];
    const int n = h.nnz();
    if (!rows) {
        *nnz = n;
        return VTN_OK;
    }
    if (*nnz < n || !cols || !ops) return VTN_EINVAL;
    std::copy(h.rows.begin(), h.rows.end(), rows);
    std::copy(h.cols.begin(), h.cols.end(), cols);
    std::memcpy(ops, h.ops.data(), sizeof(double) * 2 * h.ops.size());
    *nnz = n;
    return VTN_OK;
}

vtn_status vtn_mpo_bond_terms(vtn_mpo mpo, int bond, int* usable, int* n_terms, int* n_id, int* ri, int* rj,
                              int* ops, double* U, double* V, double* Bi, double* Bj) {
    if (!mpo || !usable || !n_terms || !n_id || !ri || !rj || bond < 0 || bond + 1 >= mpo->hp.M) return VTN_EINVAL;
    try {
        const HostCore& a = mpo->hp.cores[bond];
        const HostCore& b = mpo->hp.cores[bond + 1];
        int nid = 0, r1 = 0, r2 = 0;
        std::vector<int> o;
        std::vector<std::complex<double>> u, v, b1, b2;
        bool worthwhile = false;
        const bool ok = bond_terms_host(a, b, nid, o, u, v, b1, b2, r1, r2, worthwhile);
        *usable = ok ? (worthwhile ? 1 : 2) : 0;
        *n_terms = ok ? (int)o.size() / 2 : 0;
        *n_id = ok ? nid : 0;
        *ri = r1;
        *rj = r2;
        if (!ops || !ok) return VTN_OK;
        if (!U || !V || !Bi || !Bj) return VTN_EINVAL;
        std::copy(o.begin(), o.end(), ops);
        std::memcpy(U, u.data(), sizeof(double) * 2 * u.size());
        std::memcpy(V, v.data(), sizeof(double) * 2 * v.size());
        std::memcpy(Bi, b1.data(), sizeof(double) * 2 * b1.size());
        std::memcpy(Bj, b2.data(), sizeof(double) * 2 * b2.size());
        return VTN_OK;
    } catch (const std::exception&) {
        return VTN_ENOMEM;
    }
}

vtn_status vtn_mpo_norm_bound(vtn_mpo mpo, double* out) {
    if (!mpo || !out) return VTN_EINVAL;
    *out = mpo->hp.norm_bound;
    return VTN_OK;
}

// ------------------------------------------------------------------ MPS
vtn_status vtn_mps_random_center(vtn_ctx ctx, vtn_mpo mpo, int chi, uint64_t seed, int center, vtn_mps* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out && mpo, "null argument");
        VTN_REQUIRE(chi >= 1, "chi must be >= 1");
        const int M = mpo->hp.M, d = mpo->hp.d;
        VTN_REQUIRE(center >= 0 && center < M, "center must be in [0, M)");
        Ctx& c = ctx->c;
        use_device(c);
        vtn_mps m = new_mps(ctx, M, d, bond_dims(M, d, chi));
        try {
            for (int s = 0; s < M; ++s) {
                const int cl = m->dims[s], cr = m->dims[s + 1];
                fill_random_normal(c, m->sites[s], (long long)cl * d * cr, seed, s);
                if (s >= center) {
                    orthonormalize_rows(c, m->sites[s], cl, d * cr);
                } else {
                    // columns of the (cl d) x cr matrix = rows of its conjugate transpose
                    double2* t = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)cl * d * cr);
                    conj_transpose_dev(c, cl * d, cr, m->sites[s], cr, t, (long long)cl * d);
                    orthonormalize_rows(c, t, cr, cl * d);
                    conj_transpose_dev(c, cr, cl * d, t, (long long)cl * d, m->sites[s], cr);
                }
            }
            if (m->dims[center] > 1) {
                const long long n = (long long)m->dims[center] * d * m->dims[center + 1];
                double* nrm = (double*)c.workspace(WS_RQ_S, sizeof(double) * 64);
                // divide by sqrt(dims[center]) = sqrt(|A_center|^2) (orthonormal rows)
                norm2_dev(c, m->sites[center], n, nrm);
                scale_inv_sqrt(c, m->sites[center], n, nrm);
            }
            c.sync();
        } catch (...) {
            destroy_mps(m);
            throw;
        }
        m->center = center;
        *out = m;
        return VTN_OK;
    });
}

vtn_status vtn_mps_random(vtn_ctx ctx, vtn_mpo mpo, int chi, uint64_t seed, vtn_mps* out) {
    return vtn_mps_random_center(ctx, mpo, chi, seed, 0, out);
}

vtn_status vtn_mps_get_center(vtn_mps mps, int* center) {
    if (!mps || !center) return VTN_EINVAL;
    *center = mps->center;
    return VTN_OK;
}

vtn_status vtn_mps_set_center(vtn_mps mps, int center) {
    if (!mps || center < -1 || center >= mps->M) return VTN_EINVAL;
    mps->center = center;
    return VTN_OK;
}

vtn_status vtn_mps_move_center(vtn_ctx ctx, vtn_mps mps, int center) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mps != nullptr, "null MPS");
        VTN_REQUIRE(center >= 0 && center < mps->M, "center must be in [0, M)");
        Ctx& c = ctx->c;
        use_device(c);
        move_center(c, mps, center);
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mps_from_host(vtn_ctx ctx, vtn_mpo mpo, const int* dims, const double* const* sites, vtn_mps* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out && mpo && dims && sites, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        const int M = mpo->hp.M, d = mpo->hp.d;
        std::vector<int> dv(dims, dims + M + 1);
        VTN_REQUIRE(dv[0] == 1 && dv[M] == 1, "dims[0] and dims[M] must be 1");
        for (int s = 0; s <= M; ++s) VTN_REQUIRE(dv[s] >= 1 && dv[s] <= 65536, "bond dimension out of range");
        vtn_mps m = new_mps(ctx, M, d, dv);
        try {
            for (int s = 0; s < M; ++s) {
                VTN_REQUIRE(sites[s] != nullptr, "null site tensor");
                VTN_CUDA_TRY(cudaMemcpyAsync(m->sites[s], sites[s], sizeof(double2) * (size_t)dv[s] * d * dv[s + 1],
                                             cudaMemcpyHostToDevice, c.stream));
            }
            c.sync();
        } catch (...) {
            destroy_mps(m);
            throw;
        }
        m->center = -1;
        *out = m;
        return VTN_OK;
    });
}

vtn_status vtn_mps_free(vtn_mps mps) {
    if (!mps) return VTN_EINVAL;
    if (mps->owner) {
        cudaStreamSynchronize(mps->owner->c.stream);
    }
    destroy_mps(mps);
    return VTN_OK;
}

vtn_status vtn_mps_info(vtn_mps mps, int* M, int* d, int* dims) {
    if (!mps) return VTN_EINVAL;
    if (M) *M = mps->M;
    if (d) *d = mps->d;
    if (dims) std::copy(mps->dims.begin(), mps->dims.end(), dims);
    return VTN_OK;
}

vtn_status vtn_mps_get_site(vtn_ctx ctx, vtn_mps mps, int site, double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mps && out && site >= 0 && site < mps->M, "bad argument");
        Ctx& c = ctx->c;
        use_device(c);
        const size_t n = (size_t)mps->dims[site] * mps->d * mps->dims[site + 1];
        VTN_CUDA_TRY(cudaMemcpyAsync(out, mps->sites[site], sizeof(double2) * n, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mps_save(vtn_ctx ctx, vtn_mps mps, const char* path) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mps && path, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        FILE* f = std::fopen(path, "wb");
        VTN_REQUIRE(f != nullptr, std::string("cannot open ") + path + " for writing");
        const char magic[8] = {'V', 'T', 'N', 'M', 'P', 'S', '0', '1'};
        bool ok = std::fwrite(magic, 1, 8, f) == 8;
        int hdr[3] = {mps->M, mps->d, mps->center};
        ok = ok && std::fwrite(hdr, sizeof(int), 3, f) == 3;
        ok = ok && std::fwrite(mps->dims.data(), sizeof(int), mps->M + 1, f) == (size_t)(mps->M + 1);
        std::vector<double2> buf;
        for (int s = 0; s < mps->M && ok; ++s) {
            const size_t n = (size_t)mps->dims[s] * mps->d * mps->dims[s + 1];
            buf.resize(n);
            cudaError_t e = cudaMemcpyAsync(buf.data(), mps->sites[s], sizeof(double2) * n, cudaMemcpyDeviceToHost, c.stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
            ok = (e == cudaSuccess) && std::fwrite(buf.data(), sizeof(double2), n, f) == n;
        }
        std::fclose(f);
        VTN_REQUIRE(ok, std::string("writing ") + path + " failed");
        return VTN_OK;
    });
}

vtn_status vtn_mps_load(vtn_ctx ctx, vtn_mpo mpo, const char* path, vtn_mps* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && path && out, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        FILE* f = std::fopen(path, "rb");
        VTN_REQUIRE(f != nullptr, std::string("cannot open ") + path);
        char magic[8];
        int hdr[3];
        bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "VTNMPS01", 8) == 0;
        ok = ok && std::fread(hdr, sizeof(int), 3, f) == 3;
        if (!ok || hdr[0] != mpo->hp.M || hdr[1] != mpo->hp.d) {
            std::fclose(f);
            throw Error{VTN_EINVAL, "checkpoint does not match the MPO or is not a vtn MPS file"};
        }
        std::vector<int> dims(hdr[0] + 1);
        ok = std::fread(dims.data(), sizeof(int), dims.size(), f) == dims.size();
        for (int x : dims) ok = ok && x >= 1 && x <= 65536;
        if (!ok) {
            std::fclose(f);
            throw Error{VTN_EINVAL, "corrupt checkpoint header"};
        }
        std::vector<std::vector<double>> host(hdr[0]);
        std::vector<const double*> ptrs(hdr[0]);
        for (int s = 0; s < hdr[0] && ok; ++s) {
            const size_t n = (size_t)dims[s] * hdr[1] * dims[s + 1];
            host[s].resize(2 * n);
            ok = std::fread(host[s].data(), sizeof(double) * 2, n, f) == n;
            ptrs[s] = host[s].data();
        }
        std::fclose(f);
        VTN_REQUIRE(ok, "truncated checkpoint");
        vtn_status st = vtn_mps_from_host(ctx, mpo, dims.data(), ptrs.data(), out);
        if (st == VTN_OK) (*out)->center = hdr[2];
        if (st != VTN_OK) throw Error{st, ctx->c.err};
        return VTN_OK;
    });
}

// ------------------------------------------------------------------ solver
vtn_status vtn_sweep_opts_default(vtn_sweep_opts* o) {
    if (!o) return VTN_EINVAL;
    std::memset(o, 0, sizeof(*o));
    o->chi_max = 16;
    o->n_sweeps = 8;
    o->prec = VTN_FP64;
    o->lanczos_tol = 1e-10;
    o->krylov_max = 32;
    o->lanczos_max_restarts = 4;
    o->trunc_mode = 0;
    o->trunc_q = 1;
    return VTN_OK;
}

namespace {

// Two-site sweeps of one instance: device work on `work`'s stream and workspace; the MPO's
// device copy and a new random MPS belong to `owner` (the same context for vtn_sweep, the
// caller's context for the workers of vtn_sweep_batch).
vtn_status sweep_body(vtn_ctx work, vtn_ctx owner, vtn_mpo mpo, vtn_mps* state, const vtn_sweep_opts* opts,
                      vtn_sweep_report* report) {
    VTN_REQUIRE(mpo && state && opts, "null argument");
    VTN_REQUIRE(opts->chi_max >= 1, "chi_max must be >= 1");
    VTN_REQUIRE(opts->n_sweeps >= 0 && opts->n_sweeps <= 64, "n_sweeps must be in [0, 64]");
    VTN_REQUIRE(opts->krylov_max >= 1 && opts->krylov_max <= 64, "krylov_max must be in [1, 64]");
    VTN_REQUIRE(opts->lanczos_max_restarts >= 0, "lanczos_max_restarts must be >= 0");
    VTN_REQUIRE(opts->n_schedule == 0 || opts->chi_schedule != nullptr, "chi_schedule missing");
    VTN_REQUIRE(opts->trunc_mode == 0 || opts->trunc_mode == 1, "trunc_mode must be 0 or 1");
    VTN_REQUIRE(opts->trunc_mode == 0 || (opts->trunc_q >= 0 && opts->trunc_q <= 64), "trunc_q must be in [0, 64]");
    if (opts->prec != VTN_FP64 && opts->prec != VTN_BF16X3)
        throw Error{VTN_EUNSUPPORTED, "VTN_TF32X3 is not available in this build"};
    const bool split = opts->prec == VTN_BF16X3;
    Ctx& c = work->c;
    const long long syncs0 = c.host_syncs;
    use_device(c);
    ensure_mpo_device(owner, mpo);
    const int M = mpo->hp.M, d = mpo->hp.d;
    if (M < 2) throw Error{VTN_EUNSUPPORTED, "two-site DMRG needs M >= 2"};
    std::vector<int> sched;
    for (int i = 0; i < opts->n_schedule; ++i) {
        VTN_REQUIRE(opts->chi_schedule[i] >= 1, "chi_schedule entries must be >= 1");
        sched.push_back(std::min(opts->chi_schedule[i], opts->chi_max));
    }
    if (sched.empty()) sched.push_back(opts->chi_max);
    if (*state == nullptr) {
        vtn_status st = vtn_mps_random(owner, mpo, sched[0], opts->seed, state);
        if (st != VTN_OK) throw Error{st, owner->c.err};
    }
    vtn_mps mps = *state;
    check_mps_matches(mpo, mps);
    // bonds lo .. hi - 1 (a windowed sweep) or the whole chain
    const bool windowed = opts->window_hi > opts->window_lo;
    const int lo = windowed ? opts->window_lo : 0, hi = windowed ? opts->window_hi : M - 1;
    VTN_REQUIRE(!windowed || (lo >= 0 && hi <= M - 1), "window must satisfy 0 <= window_lo < window_hi <= M - 1");
    VTN_REQUIRE(opts->energy_mode == 0 || opts->energy_mode == 1, "energy_mode must be 0 or 1");
    VTN_REQUIRE(opts->heff_form >= 0 && opts->heff_form <= 2, "heff_form must be 0, 1 or 2");
    VTN_REQUIRE(opts->env_fp64 == 0 || opts->env_fp64 == 1, "env_fp64 must be 0 or 1");
    // term form of bond i's H_eff (split precision), or null for the channel-mixing form
    auto bond_terms = [&](int i) -> const BondTerms* {
        if (opts->heff_form == 1 || i < 0 || i >= (int)mpo->bterms.size()) return nullptr;
        const BondTerms& bt = mpo_bond_terms(c, mpo, i);
        if (!bt.usable || (opts->heff_form == 0 && !bt.worthwhile)) return nullptr;
        return &bt;
    };
    const bool centre_energy = windowed || opts->energy_mode == 1;
    int chi_cap = opts->chi_max;
    for (int x : mps->dims) chi_cap = std::max(chi_cap, x);
    mps_reserve(c, mps, chi_cap);
    // the environments assume sites < lo left-canonical and sites > lo right-canonical
    if (windowed ? mps->center != lo : mps->center > 0) move_center(c, mps, lo);
    const std::vector<int> capdims = cap_dims(M, chi_cap);
    // environments sized for the largest bond dimension at each cut
    Envs env;
    env.c = &c;
    env.L.assign(M + 1, nullptr);
    env.R.assign(M + 1, nullptr);
    for (int s = 0; s <= M; ++s) {
        // L[s] is read or written for s <= hi, R[s] for s >= lo + 1
        const size_t cap = (size_t)mpo->hp.w[s] * capdims[s] * capdims[s];
        if (s <= hi) env.L[s] = (double2*)c.dalloc(sizeof(double2) * std::max(cap, size_t(1)));
        if (s >= lo + 1) env.R[s] = (double2*)c.dalloc(sizeof(double2) * std::max(cap, size_t(1)));
    }
    set_scalar_one(c, env.L[0]);
    set_scalar_one(c, env.R[M]);
    // environment updates run in the same precision mode as H_eff psi
    const bool split_env = split && opts->env_fp64 == 0;
    auto env_left = [&](const DevCore& W, int cl, int cr, const double2* Lin, const double2* A, double2* Lout) {
        if (split_env) env_left_bf16x3(c, W, cl, cr, Lin, A, Lout);
        else env_left_dev(c, W, cl, cr, Lin, A, Lout);
    };
    auto env_right = [&](const DevCore& W, int cl, int cr, const double2* Rin, const double2* A, double2* Rout) {
        if (split_env) env_right_bf16x3(c, W, cl, cr, Rin, A, Rout);
        else env_right_dev(c, W, cl, cr, Rin, A, Rout);
    };
    for (int s = 0; s < lo; ++s)
        env_left(mpo->dcores[s], mps->dims[s], mps->dims[s + 1], env.L[s], mps->sites[s], env.L[s + 1]);
    for (int s = M - 1; s >= lo + 2; --s)
        env_right(mpo->dcores[s], mps->dims[s], mps->dims[s + 1], env.R[s + 1], mps->sites[s], env.R[s]);
    const size_t theta_cap = (size_t)chi_cap * d * d * chi_cap;
    double2* theta = (double2*)c.workspace(WS_VEC_T, sizeof(double2) * theta_cap);
    vtn_sweep_report rep;
    std::memset(&rep, 0, sizeof(rep));
    long long not_conv = 0;
    double prevE = 0.0;
    bool have_prev = false;
    // theta = A_i A_i+1
    auto form_theta = [&](int i, bool start_vector) {
        const int cl = mps->dims[i], cm = mps->dims[i + 1], cr = mps->dims[i + 2];
        if (split && start_vector) {
            // the Lanczos start vector feeds split-precision products only
            zgemm_bf16x3(c, cl * d, d * cr, cm, mps->sites[i], cm, mps->sites[i + 1], (long long)d * cr, theta,
                         (long long)d * cr);
            return;
        }
        GemmArgs g;
        g.M = cl * d; g.N = d * cr; g.K = cm;
        g.A = mps->sites[i]; g.lda = cm;
        g.B = mps->sites[i + 1]; g.ldb = (long long)d * cr;
        g.C = theta; g.ldc = (long long)d * cr;
        gemm_c64(c, g);
    };
    // Without Lanczos restarts (and with the exact truncation) a sweep returns to the host only
    // at its end: each Lanczos solve runs its Krylov steps on a device stop flag and the
    // truncation's eigenvalues and status are staged in pinned memory, read once per sweep.
    const bool deferred = opts->lanczos_max_restarts == 0 && opts->trunc_mode == 0;
    const int steps_per_sweep = 2 * (hi - lo);
    const size_t slot = (size_t)chi_cap + 16;  // 5 doubles of Lanczos results, then k + 5 of truncation
    double* dbuf = deferred ? c.defer_reserve(slot * (size_t)steps_per_sweep) : nullptr;
    std::vector<double> step_hf(steps_per_sweep, 0.0);
    std::vector<int> step_k(steps_per_sweep, 0);
    for (int sw = 0; sw < opts->n_sweeps; ++sw) {
        const auto t0 = std::chrono::steady_clock::now();
        const int chi_s = sched[std::min<size_t>(sw, sched.size() - 1)];
        double disc_max = 0.0;
        for (int dir = 0; dir < 2; ++dir) {
            for (int step = 0; step < hi - lo; ++step) {
                const int i = dir == 0 ? lo + step : (hi - 1 - step);
                const int cl = mps->dims[i], cm = mps->dims[i + 1], cr = mps->dims[i + 2];
                const int sidx = dir * (hi - lo) + step;
                double* lz_slot = deferred ? dbuf + slot * sidx : nullptr;
                double* tr_slot = deferred ? lz_slot + 5 : nullptr;
                form_theta(i, true);
                const long long n = (long long)cl * d * d * cr;
                const DevCore& Wi = mpo->dcores[i];
                const DevCore& Wj = mpo->dcores[i + 1];
                const double2* L = env.L[i];
                const double2* R = env.R[i + 2];
                const double hf = heff_flops(Wi, Wj, cl, cr);
                HeffPacked pk;
                if (split) heff_pack_envs(c, Wi, Wj, cl, cr, L, R, pk, bond_terms(i));
                LanczosResult lr = lanczos(c, n, theta, opts->lanczos_tol, opts->krylov_max,
                                           opts->lanczos_max_restarts, [&](const double2* in, double2* out) {
                                               if (split) heff_apply_bf16x3(c, Wi, Wj, pk, in, out);
                                               else heff_apply_dev(c, Wi, Wj, cl, cr, L, R, in, out);
                                           }, lz_slot);
                step_hf[sidx] = hf;
                if (!deferred) {
                    rep.matvecs += lr.n_matvec;
                    rep.heff_flops += hf * lr.n_matvec;
                    if (!lr.converged) ++not_conv;
                }
                TruncResult tr;
                if (opts->trunc_mode == 1) {
                    // warm start: the current centre (site i sweeping right, i + 1 sweeping left),
                    // as conjugated rows
                    const double2* Sh0 = mps->sites[i + 1];  // cm x (d cr), already rows
                    if (dir == 0) {
                        double2* q0 = (double2*)c.workspace(WS_WARM_Q0, sizeof(double2) * (size_t)cm * cl * d);
                        conj_transpose_dev(c, cl * d, cm, mps->sites[i], cm, q0, (long long)cl * d);
                        Sh0 = q0;
                    }
                    tr = truncate_warm_dev(c, cl, d, d, cr, dir, chi_s, theta, Sh0, cm, opts->trunc_q, 8, opts->seed,
                                           i, mps->sites[i], mps->sites[i + 1]);
                } else {
                    tr = truncate_dev(c, cl, d, d, cr, dir, chi_s, theta, mps->sites[i], mps->sites[i + 1], -1, tr_slot);
                }
                mps->dims[i + 1] = tr.k;
                step_k[sidx] = tr.k;
                if (!deferred) disc_max = std::max(disc_max, tr.discarded);
                if (dir == 0)
                    env_left(Wi, cl, tr.k, env.L[i], mps->sites[i], env.L[i + 1]);
                else
                    env_right(Wj, tr.k, cr, env.R[i + 2], mps->sites[i + 1], env.R[i + 1]);
            }
        }
        mps->center = lo;
        double E;
        if (centre_energy) {
            // Rayleigh quotient of the final centre theta = A_lo A_lo+1 under H_eff of bond (lo, lo+1)
            const int cl = mps->dims[lo], cr = mps->dims[lo + 2];
            const long long n = (long long)cl * d * d * cr;
            form_theta(lo, false);
            double2* y = (double2*)c.workspace(WS_RQ_Y, sizeof(double2) * (size_t)n);
            double* sc = (double*)c.workspace(WS_RQ_S, sizeof(double) * 64);
            const DevCore& Wi = mpo->dcores[lo];
            const DevCore& Wj = mpo->dcores[lo + 1];
            if (split) {
                HeffPacked pk;
                heff_pack_envs(c, Wi, Wj, cl, cr, env.L[lo], env.R[lo + 2], pk, bond_terms(lo));
                heff_apply_bf16x3(c, Wi, Wj, pk, theta, y);
            } else {
                heff_apply_dev(c, Wi, Wj, cl, cr, env.L[lo], env.R[lo + 2], theta, y);
            }
            multi_dot(c, theta, n, 1, y, n, (double2*)sc);
            norm2_dev(c, theta, n, sc + 2);
            VTN_CUDA_TRY(cudaMemcpyAsync(c.pinned, sc, sizeof(double) * 3, cudaMemcpyDeviceToHost, c.stream));
            c.sync();
            E = c.pinned[0] / c.pinned[2];
        } else {
            E = energy_dev(c, mpo, mps);
            c.sync();
        }
        if (deferred) {
            // the stream is synchronised: the staged results of this sweep are complete
            for (int k = 0; k < steps_per_sweep; ++k) {
                const LanczosResult lr = lanczos_deferred_result(dbuf + slot * k);
                rep.matvecs += lr.n_matvec;
                rep.heff_flops += step_hf[k] * lr.n_matvec;
                if (!lr.converged) ++not_conv;
                disc_max = std::max(disc_max, truncate_deferred_result(dbuf + slot * k + 5, step_k[k]).discarded);
            }
        }
        const auto t1 = std::chrono::steady_clock::now();
        rep.energy[sw] = E;
        rep.max_discarded[sw] = disc_max;
        rep.seconds[sw] = std::chrono::duration<double>(t1 - t0).count();
        rep.sweeps_done = sw + 1;
        if (opts->use_e_target && E <= opts->e_target) break;
        if (have_prev && opts->e_tol > 0 && std::fabs(E - prevE) <= opts->e_tol) break;
        prevE = E;
        have_prev = true;
    }
    c.tflush();
    c.check_dstatus();
    rep.lanczos_not_converged = not_conv;
    rep.heff_seconds = c.tc[TC_HEFF].seconds;
    rep.gemm_flops = c.tc[TC_GEMM].flops;
    rep.gemm_seconds = c.tc[TC_GEMM].seconds;
    rep.eig_seconds = c.tc[TC_EIG].seconds;
    rep.host_syncs = c.host_syncs - syncs0;
    if (report) *report = rep;
    if (not_conv > 0) {
        c.err = std::to_string(not_conv) + " Lanczos solves missed the tolerance";
        return VTN_ENOCONV;
    }
    return VTN_OK;
}

}  // namespace

vtn_status vtn_sweep(vtn_ctx ctx, vtn_mpo mpo, vtn_mps* state, const vtn_sweep_opts* opts, vtn_sweep_report* report) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status { return sweep_body(ctx, ctx, mpo, state, opts, report); });
}

vtn_status vtn_sweep_batch(vtn_ctx ctx, int n, const vtn_mpo* mpos, vtn_mps* states, const vtn_sweep_opts* opts,
                           vtn_sweep_report* reports, vtn_status* status, int n_streams) {
    if (!ctx) return VTN_EINVAL;
    std::vector<vtn_ctx> workers;
    auto release = [&]() {
        for (vtn_ctx w : workers) {
            cudaStream_t s = w->c.stream;
            vtn_destroy(w);
            if (s) cudaStreamDestroy(s);
        }
        workers.clear();
    };
    vtn_status st = guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(n >= 0 && (n == 0 || (mpos && states && opts && status)), "null argument");
        VTN_REQUIRE(n_streams >= 1 && n_streams <= 64, "n_streams must be in [1, 64]");
        Ctx& c = ctx->c;
        use_device(c);
        // serial set-up on the caller's context: device copies of the MPOs, random initial states
        for (int j = 0; j < n; ++j) {
            VTN_REQUIRE(mpos[j] != nullptr, "null MPO in the batch");
            ensure_mpo_device(ctx, mpos[j]);
            // the workers may share an MPO: its bonds' term forms are built here, not on first use
            for (int s = 0; s + 1 < mpos[j]->hp.M; ++s) mpo_bond_terms(c, mpos[j], s);
            if (states[j] == nullptr) {
                std::vector<int> sched;
                for (int i = 0; i < opts[j].n_schedule && opts[j].chi_schedule; ++i)
                    sched.push_back(std::min(opts[j].chi_schedule[i], opts[j].chi_max));
                const int chi0 = sched.empty() ? opts[j].chi_max : sched[0];
                vtn_status s0 = vtn_mps_random(ctx, mpos[j], std::max(chi0, 1), opts[j].seed, &states[j]);
                if (s0 != VTN_OK) throw Error{s0, c.err};
            }
        }
        // nothing queued before this call may still use memory the workers' allocations return
        VTN_CUDA_TRY(cudaDeviceSynchronize());
        // worker contexts: own stream and workspace, the caller's allocator
        const int W = std::min(n_streams, std::max(n, 1));
        const vtn_allocator* al = c.has_alloc ? &c.alloc : nullptr;
        for (int k = 0; k < W; ++k) {
            cudaStream_t s = nullptr;
            VTN_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
            vtn_ctx w = nullptr;
            vtn_status cs = vtn_create(&w, c.device, s, al);
            if (cs != VTN_OK) {
                cudaStreamDestroy(s);
                throw Error{cs, std::string("worker context: ") + vtn_last_error(nullptr)};
            }
            workers.push_back(w);
        }
        std::atomic<int> next{0};
        auto run = [&](vtn_ctx w) {
            cudaSetDevice(w->c.device);
            for (;;) {
                const int j = next.fetch_add(1);
                if (j >= n) break;
                status[j] = guard(w, [&]() -> vtn_status {
                    return sweep_body(w, ctx, mpos[j], &states[j], &opts[j], reports ? &reports[j] : nullptr);
                });
            }
        };
        std::vector<std::thread> threads;
        for (int k = 1; k < W; ++k) threads.emplace_back(run, workers[k]);
        run(workers[0]);
        for (auto& t : threads) t.join();
        for (int j = 0; j < n; ++j)
            if (status[j] != VTN_OK && status[j] != VTN_ENOCONV)
                throw Error{status[j], "instance " + std::to_string(j) + " of the batch failed"};
        return VTN_OK;
    });
    release();
    if (st == VTN_OK)
        for (int j = 0; j < n; ++j)
            if (status[j] == VTN_ENOCONV) return VTN_ENOCONV;
    return st;
}

// Single-site DMRG with subspace expansion.  At site i sweeping right: Lanczos on the
// single-site H_eff, expansion Mx = [A | alpha P] ((chi_l d) x chi_r (1 + w_r)), FP64
// eigendecomposition of Mx Mx^dag keeping k = min(chi, chi_l d, chi_r (1 + w_r), d chi_{i+2})
// eigenpairs and then only those above cutoff * the largest, A_i <- U_k, the centre
// (U_k^dag A) A_{i+1} moves right, L_{i+1} is updated; the left sweep mirrors it.
vtn_status vtn_sweep_single_site(vtn_ctx ctx, vtn_mpo mpo, vtn_mps* state, const vtn_sweep_opts* opts,
                                 double alpha, double alpha_decay, double cutoff, vtn_sweep_report* report) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && state && opts, "null argument");
        VTN_REQUIRE(opts->chi_max >= 1, "chi_max must be >= 1");
        VTN_REQUIRE(opts->n_sweeps >= 0 && opts->n_sweeps <= 64, "n_sweeps must be in [0, 64]");
        VTN_REQUIRE(opts->krylov_max >= 1 && opts->krylov_max <= 64, "krylov_max must be in [1, 64]");
        VTN_REQUIRE(opts->lanczos_max_restarts >= 0, "lanczos_max_restarts must be >= 0");
        VTN_REQUIRE(opts->n_schedule == 0 || opts->chi_schedule != nullptr, "chi_schedule missing");
        VTN_REQUIRE(std::isfinite(alpha) && alpha >= 0.0, "alpha must be finite and >= 0");
        VTN_REQUIRE(std::isfinite(alpha_decay) && alpha_decay >= 0.0, "alpha_decay must be finite and >= 0");
        VTN_REQUIRE(std::isfinite(cutoff) && cutoff >= 0.0 && cutoff < 1.0, "cutoff must be in [0, 1)");
        if (opts->prec != VTN_FP64) throw Error{VTN_EUNSUPPORTED, "the single-site solver runs in FP64 only"};
        if (opts->window_hi > opts->window_lo) throw Error{VTN_EUNSUPPORTED, "windowed sweeps are two-site only"};
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        const int M = mpo->hp.M, d = mpo->hp.d;
        std::vector<int> sched;
        for (int i = 0; i < opts->n_schedule; ++i) {
            VTN_REQUIRE(opts->chi_schedule[i] >= 1, "chi_schedule entries must be >= 1");
            sched.push_back(std::min(opts->chi_schedule[i], opts->chi_max));
        }
        if (sched.empty()) sched.push_back(opts->chi_max);
        if (*state == nullptr) {
            vtn_status st = vtn_mps_random(ctx, mpo, sched[0], opts->seed, state);
            if (st != VTN_OK) throw Error{st, c.err};
        }
        vtn_mps mps = *state;
        check_mps_matches(mpo, mps);
        int chi_cap = opts->chi_max;
        for (int x : mps->dims) chi_cap = std::max(chi_cap, x);
        mps_reserve(c, mps, chi_cap);
        const std::vector<int> capdims = cap_dims(M, chi_cap);
        Envs env;
        env.c = &c;
        env.L.assign(M + 1, nullptr);
        env.R.assign(M + 1, nullptr);
        for (int s = 0; s <= M; ++s) {
            const size_t cap = (size_t)mpo->hp.w[s] * capdims[s] * capdims[s];
            env.L[s] = (double2*)c.dalloc(sizeof(double2) * std::max(cap, size_t(1)));
            env.R[s] = (double2*)c.dalloc(sizeof(double2) * std::max(cap, size_t(1)));
        }
        set_scalar_one(c, env.L[0]);
        set_scalar_one(c, env.R[M]);
        for (int s = M - 1; s >= 1; --s)
            env_right_dev(c, mpo->dcores[s], mps->dims[s], mps->dims[s + 1], env.R[s + 1], mps->sites[s], env.R[s]);
        int wmax = 1;
        for (int x : mpo->hp.w) wmax = std::max(wmax, x);
        const size_t site_cap = (size_t)chi_cap * d * chi_cap;
        double2* x = (double2*)c.workspace(WS_VEC_T, sizeof(double2) * site_cap);
        double2* Mx = (double2*)c.workspace(WS_EXPAND, sizeof(double2) * site_cap * (1 + (size_t)wmax));
        double2* TL = (double2*)c.workspace(WS_TRUNC_L, sizeof(double2) * site_cap);
        double2* TR = (double2*)c.workspace(WS_TRUNC_R, sizeof(double2) * site_cap);
        double2* Cb = (double2*)c.workspace(WS_CENTER, sizeof(double2) * site_cap);
        vtn_sweep_report rep;
        std::memset(&rep, 0, sizeof(rep));
        long long not_conv = 0;
        // Lanczos on the centre tensor of site i, in place on x
        auto optimise = [&](int i) {
            const int cl = mps->dims[i], cr = mps->dims[i + 1];
            const long long n = (long long)cl * d * cr;
            const DevCore& W = mpo->dcores[i];
            VTN_CUDA_TRY(cudaMemcpyAsync(x, mps->sites[i], sizeof(double2) * n, cudaMemcpyDeviceToDevice, c.stream));
            LanczosResult lr = lanczos(c, n, x, opts->lanczos_tol, opts->krylov_max, opts->lanczos_max_restarts,
                                       [&](const double2* in, double2* out) {
                                           heff1_apply_dev(c, W, cl, cr, env.L[i], env.R[i + 1], in, out);
                                       });
            rep.matvecs += lr.n_matvec;
            rep.heff_flops += heff1_flops(W, cl, cr) * lr.n_matvec;
            if (!lr.converged) ++not_conv;
        };
        auto kept = [&](const TruncResult& tr) {
            int k = 0;
            if (!tr.lam.empty() && tr.lam[0] > 0.0)
                for (double l : tr.lam) k += l > cutoff * tr.lam[0] ? 1 : 0;
            return std::max(1, k);
        };
        double prevE = 0.0;
        bool have_prev = false;
        for (int sw = 0; sw < opts->n_sweeps; ++sw) {
            const auto t0 = std::chrono::steady_clock::now();
            const int chi_s = sched[std::min<size_t>(sw, sched.size() - 1)];
            const double a_s = alpha * std::pow(alpha_decay, (double)sw);
            double disc_max = 0.0;
            if (M == 1) {
                optimise(0);
                VTN_CUDA_TRY(cudaMemcpyAsync(mps->sites[0], x, sizeof(double2) * d, cudaMemcpyDeviceToDevice, c.stream));
            }
            for (int i = 0; i + 1 < M; ++i) {  // to the right
                const int cl = mps->dims[i], cr = mps->dims[i + 1], cn = mps->dims[i + 2];
                const DevCore& W = mpo->dcores[i];
                optimise(i);
                expand_right_dev(c, W, cl, cr, env.L[i], x, a_s, Mx);
                const int K = cr * (1 + W.wr);
                const int kmax = std::min(chi_s, d * cn);
                TruncResult tr = truncate_dev(c, cl, d, 1, K, 0, kmax, Mx, TL, TR, cr);
                const int k = kept(tr);
                disc_max = std::max(disc_max, tr.discarded);
                // A_i <- the first k columns of U (cl d x tr.k)
                VTN_CUDA_TRY(cudaMemcpy2DAsync(mps->sites[i], sizeof(double2) * k, TL, sizeof(double2) * tr.k,
                                               sizeof(double2) * k, (size_t)cl * d, cudaMemcpyDeviceToDevice,
                                               c.stream));
                // centre (U_k^dag A) A_{i+1}: k x (d cn)
                GemmArgs g;
                g.M = k; g.N = d * cn; g.K = cr;
                g.A = TR; g.lda = cr;
                g.B = mps->sites[i + 1]; g.ldb = (long long)d * cn;
                g.C = Cb; g.ldc = (long long)d * cn;
                gemm_c64(c, g);
                VTN_CUDA_TRY(cudaMemcpyAsync(mps->sites[i + 1], Cb, sizeof(double2) * (size_t)k * d * cn,
                                             cudaMemcpyDeviceToDevice, c.stream));
                mps->dims[i + 1] = k;
                env_left_dev(c, W, cl, k, env.L[i], mps->sites[i], env.L[i + 1]);
            }
            for (int i = M - 1; i >= 1; --i) {  // to the left
                const int cp = mps->dims[i - 1], cl = mps->dims[i], cr = mps->dims[i + 1];
                const DevCore& W = mpo->dcores[i];
                optimise(i);
                expand_left_dev(c, W, cl, cr, env.R[i + 1], x, a_s, Mx);
                const int Kr = cl * (1 + W.wl);
                const int kmax = std::min(chi_s, cp * d);
                TruncResult tr = truncate_dev(c, Kr, 1, d, cr, 1, kmax, Mx, TL, TR, cl);
                const int k = kept(tr);
                disc_max = std::max(disc_max, tr.discarded);
                // A_i <- the first k rows of V^dag (right-canonical, k x d cr)
                VTN_CUDA_TRY(cudaMemcpyAsync(mps->sites[i], TR, sizeof(double2) * (size_t)k * d * cr,
                                             cudaMemcpyDeviceToDevice, c.stream));
                // centre A_{i-1} (A V_k): (cp d) x k, A V_k = the first cl rows of Mx V (ld tr.k)
                GemmArgs g;
                g.M = cp * d; g.N = k; g.K = cl;
                g.A = mps->sites[i - 1]; g.lda = cl;
                g.B = TL; g.ldb = tr.k;
                g.C = Cb; g.ldc = k;
                gemm_c64(c, g);
                VTN_CUDA_TRY(cudaMemcpyAsync(mps->sites[i - 1], Cb, sizeof(double2) * (size_t)cp * d * k,
                                             cudaMemcpyDeviceToDevice, c.stream));
                mps->dims[i] = k;
                env_right_dev(c, W, k, cr, env.R[i + 1], mps->sites[i], env.R[i]);
            }
            mps->center = 0;
            const double E = energy_dev(c, mpo, mps);
            c.sync();
            const auto t1 = std::chrono::steady_clock::now();
            rep.energy[sw] = E;
            rep.max_discarded[sw] = disc_max;
            rep.seconds[sw] = std::chrono::duration<double>(t1 - t0).count();
            rep.sweeps_done = sw + 1;
            if (opts->use_e_target && E <= opts->e_target) break;
            if (have_prev && opts->e_tol > 0 && std::fabs(E - prevE) <= opts->e_tol) break;
            prevE = E;
            have_prev = true;
        }
        c.tflush();
        c.check_dstatus();
        rep.lanczos_not_converged = not_conv;
        rep.heff_seconds = c.tc[TC_HEFF].seconds;
        rep.gemm_flops = c.tc[TC_GEMM].flops;
        rep.gemm_seconds = c.tc[TC_GEMM].seconds;
        rep.eig_seconds = c.tc[TC_EIG].seconds;
        if (report) *report = rep;
        if (not_conv > 0) {
            c.err = std::to_string(not_conv) + " Lanczos solves missed the tolerance";
            return VTN_ENOCONV;
        }
        return VTN_OK;
    });
}

vtn_status vtn_energy_variance(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* E, double* H2, double* sigma) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        check_mps_matches(mpo, mps);
        const auto eh = energy_h2_dev(c, mpo, mps);
        c.check_dstatus();
        if (E) *E = eh.first;
        if (H2) *H2 = eh.second;
        if (sigma) *sigma = std::sqrt(std::max(0.0, eh.second - eh.first * eh.first));
        return VTN_OK;
    });
}

vtn_status vtn_energy(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* E) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && E, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        check_mps_matches(mpo, mps);
        *E = energy_dev(c, mpo, mps);
        return VTN_OK;
    });
}

namespace {

// Fock-basis tensor of site s (rotated with the isometry) into dst (chi_l x D x chi_r).
const double2* fock_site(Ctx& c, vtn_mpo mpo, vtn_mps mps, int s, double2* dst) {
    const int D = mpo->hp.D, d = mpo->hp.d;
    if (!mpo->hp.lbo && D == d) return mps->sites[s];
    lbo_rotate_dev(c, mps->dims[s], d, D, mps->dims[s + 1], mpo->iso_dev + (size_t)s * D * d, mps->sites[s], dst);
    return dst;
}

}  // namespace

vtn_status vtn_marginals(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, const int* modes, int k, double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && modes && out, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        check_mps_matches(mpo, mps);
        const int M = mpo->hp.M, D = mpo->hp.D, d = mpo->hp.d;
        VTN_REQUIRE(k >= 1 && k <= M, "k must be in [1, M]");
        std::vector<int> sorted(modes, modes + k);
        for (int x : sorted) VTN_REQUIRE(x >= 0 && x < M, "mode out of range");
        std::sort(sorted.begin(), sorted.end());
        for (int j = 1; j < k; ++j) VTN_REQUIRE(sorted[j] != sorted[j - 1], "modes repeat");
        double cnt_d = std::pow((double)D, k);
        VTN_REQUIRE(cnt_d <= (double)(1 << 26), "D^k exceeds 2^26 outputs");
        const long long total = (long long)cnt_d;
        const int chi = max_dim(mps->dims);
        const double env_bytes = cnt_d * chi * (double)chi * sizeof(double2);
        VTN_REQUIRE(env_bytes <= 16e9, "joint marginal environments exceed 16 GB (D^k chi^2 too large)");
        // buffers
        const size_t envn = (size_t)total * chi * chi;
        double2* E0 = (double2*)c.workspace(WS_Z, sizeof(double2) * envn * 2);
        double2* E1 = E0 + envn;
        double2* tmp = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)total * chi * std::max(d, D) * chi);
        double2* AF = (double2*)c.workspace(WS_MISC, sizeof(double2) * (size_t)chi * D * chi);
        set_scalar_one(c, E0);
        long long count = 1;
        size_t pos = 0;
        for (int s = 0; s < M; ++s) {
            const int cl = mps->dims[s], cr = mps->dims[s + 1];
            if (pos < sorted.size() && sorted[pos] == s) {
                const double2* A = fock_site(c, mpo, mps, s, AF);
                // tmp[t] = E[t] A (cl x D cr)
                GemmArgs g1;
                g1.M = cl; g1.N = D * cr; g1.K = cl; g1.batch = (int)count;
                g1.A = E0; g1.lda = cl; g1.sA_batch = (long long)cl * cl;
                g1.B = A; g1.ldb = (long long)D * cr; g1.sB_batch = 0;
                g1.C = tmp; g1.ldc = (long long)D * cr; g1.sC_batch = (long long)cl * D * cr;
                gemm_c64(c, g1);
                for (int nn = 0; nn < D; ++nn) {
                    // E1[t D + n] = A[:, n, :]^dag tmp[t][:, n, :]
                    GemmArgs g2;
                    g2.M = cr; g2.N = cr; g2.K = cl; g2.batch = (int)count;
                    g2.opA = OP_C; g2.A = A + (size_t)nn * cr; g2.lda = (long long)D * cr; g2.sA_batch = 0;
                    g2.B = tmp + (size_t)nn * cr; g2.ldb = (long long)D * cr; g2.sB_batch = (long long)cl * D * cr;
                    g2.C = E1 + (size_t)nn * cr * cr; g2.ldc = cr; g2.sC_batch = (long long)D * cr * cr;
                    gemm_c64(c, g2);
                }
                count *= D;
                ++pos;
            } else {
                transfer_left_batch(c, (int)count, cl, d, cr, E0, mps->sites[s], E1, tmp);
            }
            std::swap(E0, E1);
        }
        // E0 holds count = D^k scalars (1 x 1 environments)
        std::vector<double2> vals(total);
        VTN_CUDA_TRY(cudaMemcpyAsync(vals.data(), E0, sizeof(double2) * total, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        const double n2 = mps_norm2(c, mps);
        // reorder from ascending-mode order to the caller's order
        std::vector<int> rank(k);
        for (int j = 0; j < k; ++j) rank[j] = (int)(std::find(sorted.begin(), sorted.end(), modes[j]) - sorted.begin());
        std::vector<int> digit(k);
        for (long long t = 0; t < total; ++t) {
            long long rem = t;
            for (int j = k - 1; j >= 0; --j) {
                digit[j] = (int)(rem % D);
                rem /= D;
            }
            long long idx = 0;
            for (int j = 0; j < k; ++j) idx = idx * D + digit[rank[j]];
            out[idx] = vals[t].x / n2;
        }
        return VTN_OK;
    });
}

vtn_status vtn_marginals_all(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && out, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        check_mps_matches(mpo, mps);
        const int M = mpo->hp.M, D = mpo->hp.D, d = mpo->hp.d;
        const int chi = max_dim(mps->dims);
        const size_t env = (size_t)chi * chi;
        // all left and right transfer environments
        double2* EL = (double2*)c.workspace(WS_Z, sizeof(double2) * env * (M + 1) * 2);
        double2* ER = EL + env * (M + 1);
        double2* tmp = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)chi * std::max(d, D) * chi);
        double2* AF = (double2*)c.workspace(WS_MISC, sizeof(double2) * (size_t)chi * D * chi);
        double2* U = (double2*)c.workspace(WS_Y, sizeof(double2) * (size_t)chi * D * chi);
        double* P = (double*)c.workspace(WS_PARTIAL, sizeof(double) * (size_t)M * D);
        set_scalar_one(c, EL);
        for (int s = 0; s < M; ++s)
            transfer_left_batch(c, 1, mps->dims[s], d, mps->dims[s + 1], EL + env * s, mps->sites[s], EL + env * (s + 1),
                                tmp);
        set_scalar_one(c, ER + env * M);
        for (int s = M - 1; s >= 0; --s)
            transfer_right(c, mps->dims[s], d, mps->dims[s + 1], ER + env * (s + 1), mps->sites[s], ER + env * s, tmp);
        for (int s = 0; s < M; ++s) {
            const int cl = mps->dims[s], cr = mps->dims[s + 1];
            const double2* A = fock_site(c, mpo, mps, s, AF);
            GemmArgs g1;  // tmp = EL[s] A   (cl x D cr)
            g1.M = cl; g1.N = D * cr; g1.K = cl;
            g1.A = EL + env * s; g1.lda = cl;
            g1.B = A; g1.ldb = (long long)D * cr;
            g1.C = tmp; g1.ldc = (long long)D * cr;
            gemm_c64(c, g1);
            GemmArgs g2;  // U = tmp (cl D x cr) ER[s+1]
            g2.M = cl * D; g2.N = cr; g2.K = cr;
            g2.A = tmp; g2.lda = cr;
            g2.B = ER + env * (s + 1); g2.ldb = cr;
            g2.C = U; g2.ldc = cr;
            gemm_c64(c, g2);
            marginal_reduce_dev(c, cl, D, cr, A, U, P + (size_t)s * D);
        }
        std::vector<double> host((size_t)M * D + 1);
        VTN_CUDA_TRY(cudaMemcpyAsync(host.data(), P, sizeof(double) * M * D, cudaMemcpyDeviceToHost, c.stream));
        VTN_CUDA_TRY(cudaMemcpyAsync(c.pinned, EL + env * M, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        const double n2 = c.pinned[0];
        for (size_t i = 0; i < (size_t)M * D; ++i) out[i] = host[i] / n2;
        return VTN_OK;
    });
}

namespace {

// rho_i (solver basis, d x d, normalised) of every site i in `sites` into host complex[|sites| d d]:
// all left and right transfer environments once, then two GEMMs and a reduction per site.
void reduced_densities(Ctx& c, vtn_mps mps, const std::vector<int>& sites, std::vector<std::complex<double>>& out) {
    const int M = mps->M, d = mps->d;
    const int chi = max_dim(mps->dims);
    const size_t env = (size_t)chi * chi;
    double2* EL = (double2*)c.workspace(WS_Z, sizeof(double2) * env * (M + 1) * 2);
    double2* ER = EL + env * (M + 1);
    double2* tmp = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)chi * d * chi);
    double2* U = (double2*)c.workspace(WS_Y, sizeof(double2) * (size_t)chi * d * chi);
    double2* rho = (double2*)c.workspace(WS_RQ_Y, sizeof(double2) * (size_t)d * d * std::max<size_t>(sites.size(), 1));
    set_scalar_one(c, EL);
    for (int s = 0; s < M; ++s)
        transfer_left_batch(c, 1, mps->dims[s], d, mps->dims[s + 1], EL + env * s, mps->sites[s], EL + env * (s + 1), tmp);
    set_scalar_one(c, ER + env * M);
    for (int s = M - 1; s >= 0; --s)
        transfer_right(c, mps->dims[s], d, mps->dims[s + 1], ER + env * (s + 1), mps->sites[s], ER + env * s, tmp);
    for (size_t j = 0; j < sites.size(); ++j) {
        const int s = sites[j], cl = mps->dims[s], cr = mps->dims[s + 1];
        GemmArgs g1;  // tmp = EL[s] A   (cl x d cr)
        g1.M = cl; g1.N = d * cr; g1.K = cl;
        g1.A = EL + env * s; g1.lda = cl;
        g1.B = mps->sites[s]; g1.ldb = (long long)d * cr;
        g1.C = tmp; g1.ldc = (long long)d * cr;
        gemm_c64(c, g1);
        GemmArgs g2;  // U = tmp (cl d x cr) ER[s+1]
        g2.M = cl * d; g2.N = cr; g2.K = cr;
        g2.A = tmp; g2.lda = cr;
        g2.B = ER + env * (s + 1); g2.ldb = cr;
        g2.C = U; g2.ldc = cr;
        gemm_c64(c, g2);
        reduced_density_dev(c, cl, d, cr, U, mps->sites[s], rho + (size_t)j * d * d);
    }
    out.resize(sites.size() * d * d);
    VTN_CUDA_TRY(cudaMemcpyAsync(out.data(), rho, sizeof(double2) * out.size(), cudaMemcpyDeviceToHost, c.stream));
    VTN_CUDA_TRY(cudaMemcpyAsync(c.pinned, EL + env * M, sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    c.sync();
    const double n2 = c.pinned[0];
    VTN_REQUIRE(n2 > 0.0, "the MPS has zero norm");
    for (auto& v : out) v /= n2;
}

// Dominant eigenvector of a Hermitian positive semi-definite d x d matrix (row-major): 40 steps
// of repeated squaring A <- A A / max|A A| leave A proportional to u u^dag (the other eigenvalues
// fall by (lambda_k / lambda_1)^(2^40)); u is then the column of largest norm, normalised, with the
// phase fixed so that component 0 is real and non-negative (or, when it vanishes, the largest).
std::vector<std::complex<double>> dominant_eigenvector(std::vector<std::complex<double>> A, int d) {
    using C = std::complex<double>;
    std::vector<C> B(d * d);
    for (int it = 0; it < 40; ++it) {
        double mx = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                C acc(0, 0);
                for (int k = 0; k < d; ++k) acc += A[i * d + k] * A[k * d + j];
                B[i * d + j] = acc;
                mx = std::max(mx, std::abs(acc));
            }
        if (!(mx > 0.0)) break;
        for (int i = 0; i < d * d; ++i) A[i] = B[i] / mx;
    }
    int col = 0;
    double best = -1.0;
    for (int j = 0; j < d; ++j) {
        double n = 0.0;
        for (int i = 0; i < d; ++i) n += std::norm(A[i * d + j]);
        if (n > best) {
            best = n;
            col = j;
        }
    }
    std::vector<C> u(d);
    const double nrm = std::sqrt(std::max(best, 1e-300));
    for (int i = 0; i < d; ++i) u[i] = A[i * d + col] / nrm;
    int ref = 0;
    if (std::abs(u[0]) < 1e-8) {
        for (int k = 1; k < d; ++k)
            if (std::abs(u[k]) > std::abs(u[ref])) ref = k;
    }
    const double m = std::abs(u[ref]);
    const C rot = m > 0 ? std::conj(u[ref]) / m : C(1, 0);
    for (auto& x : u) x *= rot;
    return u;
}

}  // namespace

vtn_status vtn_reduced_density(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, int site, double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && out, "null argument");
        check_mps_matches(mpo, mps);
        VTN_REQUIRE(site >= 0 && site < mps->M, "site out of range");
        Ctx& c = ctx->c;
        use_device(c);
        std::vector<std::complex<double>> rho;
        reduced_densities(c, mps, {site}, rho);
        std::memcpy(out, rho.data(), sizeof(double) * 2 * rho.size());
        return VTN_OK;
    });
}

vtn_status vtn_warm_features(vtn_mpo mpo, float* out) {
    if (!mpo || !out) return VTN_EINVAL;
    const auto& hp = mpo->hp;
    if (hp.V.empty()) return VTN_EUNSUPPORTED;
    const int M = hp.M, n2 = 2 * M;
    for (int i = 0; i < M; ++i) {
        const double vxx = hp.V[(size_t)i * n2 + i], vpp = hp.V[(size_t)(M + i) * n2 + M + i];
        const double vxp = hp.V[(size_t)i * n2 + M + i];
        out[4 * i + 0] = (float)std::log(vxx);
        out[4 * i + 1] = (float)std::log(vpp);
        out[4 * i + 2] = (float)(vxp / std::sqrt(vxx * vpp));
        out[4 * i + 3] = (float)(0.5 * std::log(std::max(vxx * vpp - vxp * vxp, 1e-300)));
    }
    return VTN_OK;
}

vtn_status vtn_warm_targets(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, float* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && out, "null argument");
        check_mps_matches(mpo, mps);
        Ctx& c = ctx->c;
        use_device(c);
        const int M = mps->M, d = mps->d;
        std::vector<int> all(M);
        for (int i = 0; i < M; ++i) all[i] = i;
        std::vector<std::complex<double>> rho;
        reduced_densities(c, mps, all, rho);
        for (int i = 0; i < M; ++i) {
            std::vector<std::complex<double>> A(rho.begin() + (size_t)i * d * d, rho.begin() + (size_t)(i + 1) * d * d);
            const auto u = dominant_eigenvector(A, d);
            for (int k = 0; k < d; ++k) {
                out[(size_t)i * 2 * d + 2 * k] = (float)u[k].real();
                out[(size_t)i * 2 * d + 2 * k + 1] = (float)u[k].imag();
            }
        }
        return VTN_OK;
    });
}

vtn_status vtn_mps_product(vtn_ctx ctx, vtn_mpo mpo, const double* amps, vtn_mps* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && amps && out, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        const int M = mpo->hp.M, d = mpo->hp.d;
        std::vector<double> unit((size_t)M * 2 * d);
        for (int i = 0; i < M; ++i) {
            double n2 = 0.0;
            for (int k = 0; k < 2 * d; ++k) n2 += amps[(size_t)i * 2 * d + k] * amps[(size_t)i * 2 * d + k];
            VTN_REQUIRE(n2 > 0.0 && std::isfinite(n2), "product state: a site vector is zero or not finite");
            const double inv = 1.0 / std::sqrt(n2);
            for (int k = 0; k < 2 * d; ++k) unit[(size_t)i * 2 * d + k] = amps[(size_t)i * 2 * d + k] * inv;
        }
        std::vector<int> dims(M + 1, 1);
        vtn_mps m = new_mps(ctx, M, d, dims);
        try {
            for (int i = 0; i < M; ++i)
                VTN_CUDA_TRY(cudaMemcpyAsync(m->sites[i], unit.data() + (size_t)i * 2 * d, sizeof(double2) * d,
                                             cudaMemcpyHostToDevice, c.stream));
            c.sync();
        } catch (...) {
            destroy_mps(m);
            throw;
        }
        m->center = 0;
        *out = m;
        return VTN_OK;
    });
}

vtn_status vtn_sample(vtn_ctx ctx, vtn_mpo mpo, vtn_mps mps, uint64_t seed, int n_samples, int32_t* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(mpo && mps && out, "null argument");
        VTN_REQUIRE(n_samples >= 0, "n_samples must be >= 0");
        if (n_samples == 0) return VTN_OK;
        Ctx& c = ctx->c;
        use_device(c);
        ensure_mpo_device(ctx, mpo);
        check_mps_matches(mpo, mps);
        const int M = mpo->hp.M, D = mpo->hp.D, d = mpo->hp.d;
        const int chi = max_dim(mps->dims);
        const size_t env = (size_t)chi * chi;
        const size_t site_f = (size_t)chi * D * chi;
        // one allocation: ER[M+1], AF[M], pointer tables, dims, output
        const size_t bytes = sizeof(double2) * (env * (M + 1) + site_f * M) + sizeof(void*) * 2 * (M + 1) +
                             sizeof(int) * (M + 1) + sizeof(int) * (size_t)n_samples * M + 1024;
        unsigned char* base = (unsigned char*)c.dalloc(bytes);
        struct Free {
            Ctx& c;
            void* p;
            ~Free() {
                cudaStreamSynchronize(c.stream);
                c.dfree(p);
            }
        } fr{c, base};
        double2* ER = (double2*)base;
        double2* AFall = ER + env * (M + 1);
        const double2** pAF = (const double2**)(AFall + site_f * M);
        const double2** pER = pAF + (M + 1);
        int* ddims = (int*)(pER + (M + 1));
        int* dout = ddims + (M + 1);
        double2* tmp = (double2*)c.workspace(WS_ENV_TMP, sizeof(double2) * (size_t)chi * d * chi);
        set_scalar_one(c, ER + env * M);
        for (int s = M - 1; s >= 0; --s)
            transfer_right(c, mps->dims[s], d, mps->dims[s + 1], ER + env * (s + 1), mps->sites[s], ER + env * s, tmp);
        std::vector<const double2*> hAF(M + 1, nullptr), hER(M + 1, nullptr);
        for (int s = 0; s < M; ++s) {
            double2* dst = AFall + site_f * s;
            const double2* A = fock_site(c, mpo, mps, s, dst);
            if (A != dst)
                VTN_CUDA_TRY(cudaMemcpyAsync(dst, A, sizeof(double2) * (size_t)mps->dims[s] * D * mps->dims[s + 1],
                                             cudaMemcpyDeviceToDevice, c.stream));
            hAF[s] = dst;
        }
        for (int s = 0; s <= M; ++s) hER[s] = ER + env * s;
        VTN_CUDA_TRY(cudaMemcpyAsync(pAF, hAF.data(), sizeof(void*) * (M + 1), cudaMemcpyHostToDevice, c.stream));
        VTN_CUDA_TRY(cudaMemcpyAsync(pER, hER.data(), sizeof(void*) * (M + 1), cudaMemcpyHostToDevice, c.stream));
        VTN_CUDA_TRY(cudaMemcpyAsync(ddims, mps->dims.data(), sizeof(int) * (M + 1), cudaMemcpyHostToDevice, c.stream));
        sample_dev(c, pAF, pER, ddims, M, D, chi, seed, n_samples, dout);
        VTN_CUDA_TRY(cudaMemcpyAsync(out, dout, sizeof(int) * (size_t)n_samples * M, cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        return VTN_OK;
    });
}

// ------------------------------------------------------------------ kernel-level calls
vtn_status vtn_heff_apply(vtn_ctx ctx, const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r, const double* L,
                          const double* R, const double* theta, double* y, vtn_precision prec) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(L && R && theta && y, "null device pointer");
        VTN_REQUIRE(chi_l >= 1 && chi_r >= 1, "bond dimensions must be >= 1");
        VTN_REQUIRE(theta != y, "y must not alias theta");
        if (prec != VTN_FP64 && prec != VTN_BF16X3)
            throw Error{VTN_EUNSUPPORTED, "VTN_TF32X3 is not available in this build"};
        Ctx& c = ctx->c;
        use_device(c);
        HostCore hi = core_from_abi(Wi), hj = core_from_abi(Wj);
        VTN_REQUIRE(hi.wr == hj.wl && hi.d == hj.d, "Wi.w_right must equal Wj.w_left and d must agree");
        TempCore ci(c, hi), cj(c, hj);
        if (prec == VTN_BF16X3) {
            TempTerms tt(c, hi, hj);
            HeffPacked pk;
            heff_pack_envs(c, ci.dc, cj.dc, chi_l, chi_r, (const double2*)L, (const double2*)R, pk,
                           tt.bt.worthwhile ? &tt.bt : nullptr);
            heff_apply_bf16x3(c, ci.dc, cj.dc, pk, (const double2*)theta, (double2*)y);
        } else {
            heff_apply_dev(c, ci.dc, cj.dc, chi_l, chi_r, (const double2*)L, (const double2*)R,
                           (const double2*)theta, (double2*)y);
        }
        c.sync();
        c.check_dstatus();
        return VTN_OK;
    });
}

vtn_status vtn_env_update(vtn_ctx ctx, const vtn_core* W, int side, int chi_l, int chi_r, const double* env,
                          const double* A, double* out, vtn_precision prec) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(env && A && out, "null device pointer");
        VTN_REQUIRE(side == 0 || side == 1, "side must be 0 (left) or 1 (right)");
        VTN_REQUIRE(chi_l >= 1 && chi_r >= 1, "bond dimensions must be >= 1");
        if (prec != VTN_FP64 && prec != VTN_BF16X3)
            throw Error{VTN_EUNSUPPORTED, "VTN_TF32X3 is not available in this build"};
        Ctx& c = ctx->c;
        use_device(c);
        HostCore h = core_from_abi(W);
        TempCore tc(c, h);
        const double2* e = (const double2*)env;
        const double2* a = (const double2*)A;
        double2* o = (double2*)out;
        if (prec == VTN_BF16X3) {
            if (side == 0) env_left_bf16x3(c, tc.dc, chi_l, chi_r, e, a, o);
            else env_right_bf16x3(c, tc.dc, chi_l, chi_r, e, a, o);
        } else {
            if (side == 0) env_left_dev(c, tc.dc, chi_l, chi_r, e, a, o);
            else env_right_dev(c, tc.dc, chi_l, chi_r, e, a, o);
        }
        c.check_dstatus();
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_heff1_apply(vtn_ctx ctx, const vtn_core* W, int chi_l, int chi_r, const double* L, const double* R,
                           const double* A, double* y) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(L && R && A && y, "null device pointer");
        VTN_REQUIRE(chi_l >= 1 && chi_r >= 1, "bond dimensions must be >= 1");
        VTN_REQUIRE(A != y, "y must not alias A");
        Ctx& c = ctx->c;
        use_device(c);
        HostCore h = core_from_abi(W);
        TempCore tc(c, h);
        heff1_apply_dev(c, tc.dc, chi_l, chi_r, (const double2*)L, (const double2*)R, (const double2*)A, (double2*)y);
        c.sync();
        c.check_dstatus();
        return VTN_OK;
    });
}

vtn_status vtn_expand(vtn_ctx ctx, const vtn_core* W, int side, int chi_l, int chi_r, const double* env,
                      const double* A, double alpha, double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(env && A && out, "null device pointer");
        VTN_REQUIRE(side == 0 || side == 1, "side must be 0 (expand to the right) or 1 (to the left)");
        VTN_REQUIRE(chi_l >= 1 && chi_r >= 1, "bond dimensions must be >= 1");
        VTN_REQUIRE(std::isfinite(alpha), "alpha must be finite");
        VTN_REQUIRE(A != out && env != out, "out must not alias the inputs");
        Ctx& c = ctx->c;
        use_device(c);
        HostCore h = core_from_abi(W);
        TempCore tc(c, h);
        if (side == 0)
            expand_right_dev(c, tc.dc, chi_l, chi_r, (const double2*)env, (const double2*)A, alpha, (double2*)out);
        else
            expand_left_dev(c, tc.dc, chi_l, chi_r, (const double2*)env, (const double2*)A, alpha, (double2*)out);
        c.sync();
        c.check_dstatus();
        return VTN_OK;
    });
}

vtn_status vtn_heff_ground(vtn_ctx ctx, const vtn_core* Wi, const vtn_core* Wj, int chi_l, int chi_r, const double* L,
                           const double* R, double* theta, double tol, int krylov_max, int max_restarts, double* E,
                           int* n_matvec) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(L && R && theta && E, "null argument");
        VTN_REQUIRE(chi_l >= 1 && chi_r >= 1, "bond dimensions must be >= 1");
        Ctx& c = ctx->c;
        use_device(c);
        HostCore hi = core_from_abi(Wi), hj = core_from_abi(Wj);
        VTN_REQUIRE(hi.wr == hj.wl && hi.d == hj.d, "Wi.w_right must equal Wj.w_left and d must agree");
        TempCore ci(c, hi), cj(c, hj);
        const long long n = (long long)chi_l * hi.d * hi.d * chi_r;
        LanczosResult lr = lanczos(c, n, (double2*)theta, tol, krylov_max, max_restarts,
                                   [&](const double2* in, double2* out) {
                                       heff_apply_dev(c, ci.dc, cj.dc, chi_l, chi_r, (const double2*)L,
                                                      (const double2*)R, in, out);
                                   });
        c.sync();
        *E = lr.theta;
        if (n_matvec) *n_matvec = lr.n_matvec;
        if (!lr.converged) {
            c.err = "Lanczos missed the tolerance";
            return VTN_ENOCONV;
        }
        return VTN_OK;
    });
}

vtn_status vtn_truncate(vtn_ctx ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max, const double* theta,
                        double* left, double* right, double* lam, double* discarded, int* k_out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(theta && left && right, "null device pointer");
        VTN_REQUIRE(chi_l >= 1 && d1 >= 1 && d2 >= 1 && chi_r >= 1 && k_max >= 1, "sizes must be >= 1");
        VTN_REQUIRE(direction == 0 || direction == 1, "direction must be 0 or 1");
        Ctx& c = ctx->c;
        use_device(c);
        TruncResult r = truncate_dev(c, chi_l, d1, d2, chi_r, direction, k_max, (const double2*)theta,
                                     (double2*)left, (double2*)right);
        if (lam) std::copy(r.lam.begin(), r.lam.end(), lam);
        if (discarded) *discarded = r.discarded;
        if (k_out) *k_out = r.k;
        return VTN_OK;
    });
}

vtn_status vtn_truncate_warm(vtn_ctx ctx, int chi_l, int d1, int d2, int chi_r, int direction, int k_max,
                             const double* theta, const double* Q0, int k0, int q, int p, uint64_t seed,
                             int bond, double* left, double* right, double* lam, double* discarded, int* k_out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(theta && left && right, "null device pointer");
        VTN_REQUIRE(chi_l >= 1 && d1 >= 1 && d2 >= 1 && chi_r >= 1 && k_max >= 1, "sizes must be >= 1");
        VTN_REQUIRE(direction == 0 || direction == 1, "direction must be 0 or 1");
        VTN_REQUIRE(k0 >= 0 && (k0 == 0 || Q0 != nullptr), "Q0 missing");
        Ctx& c = ctx->c;
        use_device(c);
        const int n = direction == 0 ? chi_l * d1 : d2 * chi_r;
        double2* Sh0 = nullptr;
        if (k0 > 0) {
            Sh0 = (double2*)c.workspace(WS_WARM_Q0, sizeof(double2) * (size_t)k0 * n);
            conj_transpose_dev(c, n, k0, (const double2*)Q0, k0, Sh0, n);
        }
        TruncResult r = truncate_warm_dev(c, chi_l, d1, d2, chi_r, direction, k_max, (const double2*)theta, Sh0, k0,
                                          q, p, seed, bond, (double2*)left, (double2*)right);
        if (lam) std::copy(r.lam.begin(), r.lam.end(), lam);
        if (discarded) *discarded = r.discarded;
        if (k_out) *k_out = r.k;
        return VTN_OK;
    });
}

vtn_status vtn_lbo_rotate(vtn_ctx ctx, int chi_l, int d, int D, int chi_r, const double* V, const double* A,
                          double* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(V && A && out, "null device pointer");
        VTN_REQUIRE(chi_l >= 1 && d >= 1 && D >= 1 && chi_r >= 1, "sizes must be >= 1");
        Ctx& c = ctx->c;
        use_device(c);
        lbo_rotate_dev(c, chi_l, d, D, chi_r, (const double2*)V, (const double2*)A, (double2*)out);
        c.sync();
        return VTN_OK;
    });
}

// ------------------------------------------------------------------ learned warm start: MLP
namespace {

void destroy_mlp(vtn_mlp m) {
    if (!m) return;
    if (m->owner) {
        Ctx& c = m->owner->c;
        c.dfree(m->params);
        c.dfree(m->m);
        c.dfree(m->v);
        c.dfree(m->grad);
        c.dfree(m->loss);
    }
    delete m;
}

void check_mlp(vtn_ctx ctx, vtn_mlp mlp) {
    VTN_REQUIRE(mlp != nullptr, "null MLP");
    VTN_REQUIRE(mlp->owner == ctx, "MLP belongs to another context");
}

uint64_t splitmix64(uint64_t& state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

vtn_status vtn_mlp_create(vtn_ctx ctx, int n_in, int width, int depth, int n_out, uint64_t seed, vtn_mlp* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(out != nullptr, "null argument");
        VTN_REQUIRE(n_in >= 1 && n_in <= 4096 && width >= 1 && width <= 4096 && n_out >= 1 && n_out <= 4096,
                    "layer sizes must be in [1, 4096]");
        VTN_REQUIRE(depth >= 0 && depth <= 16, "depth must be in [0, 16]");
        Ctx& c = ctx->c;
        use_device(c);
        vtn_mlp m = new vtn_mlp_s();
        m->shape = MlpShape(n_in, width, depth, n_out);
        m->owner = ctx;
        const long long n = m->shape.n_params;
        try {
            m->params = (float*)c.dalloc(sizeof(float) * n);
            m->m = (float*)c.dalloc(sizeof(float) * n);
            m->v = (float*)c.dalloc(sizeof(float) * n);
            m->grad = (float*)c.dalloc(sizeof(float) * n);
            m->loss = (float*)c.dalloc(sizeof(float));
            std::vector<float> h((size_t)n, 0.0f);
            uint64_t st = seed;
            for (int l = 0; l <= depth; ++l) {
                const int a = m->shape.in_of(l), b = m->shape.out_of(l);
                const float lim = (float)std::sqrt(6.0 / a);
                for (long long e = 0; e < (long long)a * b; ++e) {
                    const float u = (float)(splitmix64(st) >> 40) * (1.0f / 16777216.0f);  // [0, 1)
                    h[(size_t)(m->shape.offW[l] + e)] = (2.0f * u - 1.0f) * lim;
                }
            }
            VTN_CUDA_TRY(cudaMemcpyAsync(m->params, h.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c.stream));
            VTN_CUDA_TRY(cudaMemsetAsync(m->m, 0, sizeof(float) * n, c.stream));
            VTN_CUDA_TRY(cudaMemsetAsync(m->v, 0, sizeof(float) * n, c.stream));
            c.sync();
        } catch (...) {
            destroy_mlp(m);
            throw;
        }
        *out = m;
        return VTN_OK;
    });
}

vtn_status vtn_mlp_free(vtn_mlp mlp) {
    if (!mlp) return VTN_EINVAL;
    if (mlp->owner) cudaStreamSynchronize(mlp->owner->c.stream);
    destroy_mlp(mlp);
    return VTN_OK;
}

vtn_status vtn_mlp_info(vtn_mlp mlp, int* n_in, int* width, int* depth, int* n_out, long long* n_params,
                        long long* steps) {
    if (!mlp) return VTN_EINVAL;
    if (n_in) *n_in = mlp->shape.n_in;
    if (width) *width = mlp->shape.width;
    if (depth) *depth = mlp->shape.depth;
    if (n_out) *n_out = mlp->shape.n_out;
    if (n_params) *n_params = mlp->shape.n_params;
    if (steps) *steps = mlp->step;
    return VTN_OK;
}

vtn_status vtn_mlp_get_params(vtn_ctx ctx, vtn_mlp mlp, float* host) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(host != nullptr, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        VTN_CUDA_TRY(cudaMemcpyAsync(host, mlp->params, sizeof(float) * mlp->shape.n_params, cudaMemcpyDeviceToHost,
                                     c.stream));
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mlp_set_params(vtn_ctx ctx, vtn_mlp mlp, const float* host) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(host != nullptr, "null argument");
        Ctx& c = ctx->c;
        use_device(c);
        const size_t bytes = sizeof(float) * mlp->shape.n_params;
        VTN_CUDA_TRY(cudaMemcpyAsync(mlp->params, host, bytes, cudaMemcpyHostToDevice, c.stream));
        VTN_CUDA_TRY(cudaMemsetAsync(mlp->m, 0, bytes, c.stream));
        VTN_CUDA_TRY(cudaMemsetAsync(mlp->v, 0, bytes, c.stream));
        c.sync();
        mlp->step = 0;
        return VTN_OK;
    });
}

vtn_status vtn_mlp_forward(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, float* y) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(x && y, "null device pointer");
        VTN_REQUIRE(batch >= 1 && batch <= 4000000, "batch must be in [1, 4000000]");
        Ctx& c = ctx->c;
        use_device(c);
        const MlpShape& s = mlp->shape;
        float* acts = (float*)c.workspace(WS_MLP_ACT, sizeof(float) * ((size_t)std::max(s.depth, 1) * batch * s.width));
        mlp_forward_dev(c, s, mlp->params, batch, x, acts, y);
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mlp_loss_grad(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float* loss,
                             float* grad) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(x && t && loss, "null argument");
        VTN_REQUIRE(batch >= 1 && batch <= 4000000, "batch must be in [1, 4000000]");
        Ctx& c = ctx->c;
        use_device(c);
        mlp_loss_grad_dev(c, mlp->shape, mlp->params, batch, x, t, mlp->grad, mlp->loss);
        VTN_CUDA_TRY(cudaMemcpyAsync(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        if (grad)
            VTN_CUDA_TRY(cudaMemcpyAsync(grad, mlp->grad, sizeof(float) * mlp->shape.n_params, cudaMemcpyDeviceToHost,
                                         c.stream));
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mlp_train_step(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float lr,
                              float* loss) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(x && t, "null device pointer");
        VTN_REQUIRE(batch >= 1 && batch <= 4000000, "batch must be in [1, 4000000]");
        VTN_REQUIRE(std::isfinite(lr) && lr > 0.0f, "lr must be finite and > 0");
        Ctx& c = ctx->c;
        use_device(c);
        mlp_loss_grad_dev(c, mlp->shape, mlp->params, batch, x, t, mlp->grad, mlp->loss);
        mlp_adam_dev(c, mlp->shape.n_params, mlp->params, mlp->m, mlp->v, mlp->grad, lr, mlp->step + 1);
        if (loss) VTN_CUDA_TRY(cudaMemcpyAsync(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        ++mlp->step;
        return VTN_OK;
    });
}

vtn_status vtn_mlp_train(vtn_ctx ctx, vtn_mlp mlp, int batch, const float* x, const float* t, float lr, int steps,
                         float* loss) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(x && t, "null device pointer");
        VTN_REQUIRE(batch >= 1 && batch <= 4000000, "batch must be in [1, 4000000]");
        VTN_REQUIRE(std::isfinite(lr) && lr > 0.0f, "lr must be finite and > 0");
        VTN_REQUIRE(steps >= 1 && steps <= 10000000, "steps must be in [1, 10000000]");
        Ctx& c = ctx->c;
        use_device(c);
        for (int k = 0; k < steps; ++k) {
            mlp_loss_grad_dev(c, mlp->shape, mlp->params, batch, x, t, mlp->grad, mlp->loss);
            mlp_adam_dev(c, mlp->shape.n_params, mlp->params, mlp->m, mlp->v, mlp->grad, lr, mlp->step + 1);
            ++mlp->step;
        }
        if (loss) VTN_CUDA_TRY(cudaMemcpyAsync(loss, mlp->loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        return VTN_OK;
    });
}

vtn_status vtn_mps_warm_start(vtn_ctx ctx, vtn_mpo mpo, vtn_mlp mlp, vtn_mps* out) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        check_mlp(ctx, mlp);
        VTN_REQUIRE(mpo && out, "null argument");
        const int M = mpo->hp.M, d = mpo->hp.d;
        const MlpShape& sh = mlp->shape;
        VTN_REQUIRE(sh.n_in == VTN_WARM_NFEAT && sh.n_out == 2 * d,
                    "the warm-start network needs VTN_WARM_NFEAT inputs and 2 d outputs");
        Ctx& c = ctx->c;
        use_device(c);
        std::vector<float> feat((size_t)M * VTN_WARM_NFEAT), pred((size_t)M * 2 * d);
        const vtn_status fs = vtn_warm_features(mpo, feat.data());
        if (fs != VTN_OK) throw Error{fs, "the warm start needs an MPO built from (r, U)"};
        float* x = (float*)c.workspace(WS_MLP_G, sizeof(float) * ((size_t)M * (VTN_WARM_NFEAT + 2 * d)));
        float* y = x + (size_t)M * VTN_WARM_NFEAT;
        float* acts = (float*)c.workspace(WS_MLP_ACT, sizeof(float) * ((size_t)std::max(sh.depth, 1) * M * sh.width));
        VTN_CUDA_TRY(cudaMemcpyAsync(x, feat.data(), sizeof(float) * feat.size(), cudaMemcpyHostToDevice, c.stream));
        mlp_forward_dev(c, sh, mlp->params, M, x, acts, y);
        VTN_CUDA_TRY(cudaMemcpyAsync(pred.data(), y, sizeof(float) * pred.size(), cudaMemcpyDeviceToHost, c.stream));
        c.sync();
        std::vector<double> amps(pred.begin(), pred.end());
        const vtn_status ps = vtn_mps_product(ctx, mpo, amps.data(), out);
        if (ps != VTN_OK) throw Error{ps, c.err};
        return VTN_OK;
    });
}

vtn_status vtn_gemm_bf16(vtn_ctx ctx, int M, int N, int K, const void* A, long long lda, const void* B,
                         long long ldb, void* D, long long ldd, int d_fp64) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(A && B && D, "null device pointer");
        VTN_REQUIRE(M >= 1 && N >= 1 && K >= 64 && K % 64 == 0, "need M, N >= 1 and K a positive multiple of 64");
        Ctx& c = ctx->c;
        use_device(c);
        TcGemmArgs g;
        g.M = M;
        g.N = N;
        g.K = K;
        g.A = (const __nv_bfloat16*)A;
        g.lda = lda;
        g.B = (const __nv_bfloat16*)B;
        g.ldb = ldb;
        g.D = D;
        g.ldd = ldd;
        g.d_fp64 = d_fp64 != 0;
        tc_gemm_bf16(c, g);
        c.sync();
        c.check_dstatus();
        return VTN_OK;
    });
}

vtn_status vtn_set_tc_accumulation(vtn_ctx ctx, int env_kblocks, int heff_kblocks) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(env_kblocks >= 1 && env_kblocks <= 4096 && heff_kblocks >= 1 && heff_kblocks <= 4096,
                    "accumulation lengths must be in [1, 4096] k-blocks");
        ctx->c.tc_kb_env = env_kblocks;
        ctx->c.tc_kb_heff = heff_kblocks;
        return VTN_OK;
    });
}

vtn_status vtn_set_tridiag_lower(vtn_ctx ctx, int min_n) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(min_n >= 0, "min_n must be >= 0");
        ctx->c.tri_lower_min_n = min_n;
        return VTN_OK;
    });
}

vtn_status vtn_timing(vtn_ctx ctx, int enable) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        ctx->c.tflush();
        ctx->c.timing = enable != 0;
        return VTN_OK;
    });
}

vtn_status vtn_timing_read(vtn_ctx ctx, int cls, long long* launches, double* flops, double* seconds) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        VTN_REQUIRE(cls >= 0 && cls < TC_COUNT, "timing class out of range");
        ctx->c.tflush();
        if (launches) *launches = ctx->c.tc[cls].launches;
        if (flops) *flops = ctx->c.tc[cls].flops;
        if (seconds) *seconds = ctx->c.tc[cls].seconds;
        return VTN_OK;
    });
}

vtn_status vtn_timing_reset(vtn_ctx ctx) {
    if (!ctx) return VTN_EINVAL;
    return guard(ctx, [&]() -> vtn_status {
        ctx->c.tflush();
        for (auto& t : ctx->c.tc) t = Ctx::Tc{};
        return VTN_OK;
    });
}

}  // extern "C"
