// Term form of the two-site effective Hamiltonian for the split-precision mode (VTN_BF16X3).
//
// The two-site H_eff of bond (i, i+1) (Sec. "Matrix Product States": the sweep's local eigenproblem)
// contracts the left environment L, the cores W_i, W_{i+1} and the right environment R:
//
//   H_eff = sum_{a,b,c} L[a] (x) W_i[a,b] (x) W_{i+1}[b,c] (x) R[c].
//
// Expanding each core's d x d entries in a small operator basis {B_0 = I, B_1, ...} (the span of the
// entries, found by Gram-Schmidt in the Frobenius inner product), W[a,b] = sum_o W^(o)[a,b] B_o,
//
//   H_eff = sum_{o,p} sum_{a,c} K_op[a,c] L[a] (x) B_o (x) B'_p (x) R[c],   K_op = W_i^(o) W_{i+1}^(p),
//
// and each K_op (w_l x w_r) is written exactly as a sum of outer products u_t v_t^T: by its nonzero
// rows or columns for o = p = 0, by Gaussian elimination with complete pivoting for the others (for
// the GBS Hamiltonian of Eq. GBSHamiltonian they have rank one or two: a pending linear operator
// meeting the local x or p, or the local operator opening a pending channel).  With
//
//   Lhat_t = sum_a u_t[a] L[a],   Rhat_t = sum_c v_t[c] R[c]   (once per bond),
//
// one H_eff psi product is one GEMM T_t = Lhat_t theta over all terms, the small operator
// B_o (x) B'_p on the few terms that are not identities, and one GEMM y = sum_{t,k} T_t Rhat_t; the
// channel mixing of the cores (and its intermediate of w x |theta| elements) is gone.  The term
// count is w + O(1) for this Hamiltonian (the identity block has the rank of the pending-channel
// couplings), against w_l + w_r channels for the two GEMMs of the mixing form.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "vtn_internal.cuh"

namespace vtn {
namespace {

using cplx = std::complex<double>;

struct Trip {
    int a, b;
    cplx c;
};

// operator basis of a core's entries and each entry's coefficients in it
struct Expanded {
    bool ok = true;
    int r = 1;
    std::vector<cplx> B;                  // r * d * d, B_0 = I
    std::vector<std::vector<Trip>> coef;  // [r]: (row, column, coefficient)
};

double frob(const cplx* x, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += std::norm(x[i]);
    return std::sqrt(s);
}

Expanded expand_core(const HostCore& h, int max_basis) {
    const int d = h.d, dd = d * d;
    Expanded e;
    e.B.assign(dd, cplx(0.0, 0.0));
    for (int n = 0; n < d; ++n) e.B[(size_t)n * d + n] = 1.0;
    e.coef.resize(1);
    std::vector<std::vector<cplx>> Q;  // orthonormal, orthogonal to I: the basis elements 1..r-1
    std::vector<cplx> res(dd);
    for (int k = 0; k < h.nnz(); ++k) {
        const cplx* op = &h.ops[(size_t)k * dd];
        const int a = h.rows[k], b = h.cols[k];
        if (h.ident[k]) {
            if (op[0] != 0.0) e.coef[0].push_back({a, b, op[0]});
            continue;
        }
        cplx tr = 0.0;
        for (int n = 0; n < d; ++n) tr += op[(size_t)n * d + n];
        const cplx c0 = tr / (double)d;
        std::copy(op, op + dd, res.begin());
        for (int n = 0; n < d; ++n) res[(size_t)n * d + n] -= c0;
        const double nop = frob(op, dd);
        std::vector<cplx> c(Q.size(), cplx(0.0, 0.0));
        for (int pass = 0; pass < 2; ++pass)
            for (size_t o = 0; o < Q.size(); ++o) {
                cplx p = 0.0;
                for (int i = 0; i < dd; ++i) p += std::conj(Q[o][i]) * res[i];
                c[o] += p;
                for (int i = 0; i < dd; ++i) res[i] -= p * Q[o][i];
            }
        const double nr = frob(res.data(), dd);
        if (nr > 1e-11 * nop) {
            if ((int)Q.size() + 1 >= max_basis) {
                e.ok = false;
                return e;
            }
            std::vector<cplx> q(dd);
            for (int i = 0; i < dd; ++i) q[i] = res[i] / nr;
            Q.push_back(q);
            c.push_back(nr);
            e.B.insert(e.B.end(), q.begin(), q.end());
            e.coef.emplace_back();
            e.r++;
        }
        if (c0 != 0.0) e.coef[0].push_back({a, b, c0});
        for (size_t o = 0; o < c.size(); ++o)
            if (c[o] != 0.0) e.coef[o + 1].push_back({a, b, c[o]});
    }
    return e;
}

struct HostTerm {
    int o, p;
    std::vector<cplx> u, v;  // w_l, w_r
};

}  // namespace

// Host part: the terms of bond (Wi, Wj).  Returns false when the bond has no compact term form
// (an operator basis beyond max_basis elements, or d > 8); the terms are then empty.  worthwhile:
// the term count makes the term form cheaper than the channel-mixing form.
bool bond_terms_host(const HostCore& Wi, const HostCore& Wj, int& n_id, std::vector<int>& ops,
                     std::vector<cplx>& U, std::vector<cplx>& V, std::vector<cplx>& Bi, std::vector<cplx>& Bj,
                     int& ri, int& rj, bool& worthwhile) {
    const int wl = Wi.wl, wm = Wi.wr, wr = Wj.wr, d = Wi.d;
    worthwhile = false;
    n_id = 0;
    ops.clear();
    U.clear();
    V.clear();
    if (d > 8 || Wj.wl != wm || Wj.d != d) return false;
    const int max_basis = 16;
    Expanded ei = expand_core(Wi, max_basis), ej = expand_core(Wj, max_basis);
    if (!ei.ok || !ej.ok) return false;
    ri = ei.r;
    rj = ej.r;
    Bi = ei.B;
    Bj = ej.B;
    // K_op = W_i^(o) W_j^(p) (w_l x w_r), kept as the dense block over the rows and columns that
    // the sparse product touches (for this Hamiltonian most blocks touch one row or one column)
    struct Block {
        std::vector<int> rows, cols;  // touched, ascending
        std::vector<cplx> k;          // rows.size() x cols.size()
    };
    std::vector<Block> K((size_t)ri * rj);
    double kmax2 = 0.0;
    std::vector<int> rpos(wl, -1), cpos(wr, -1);
    for (int p = 0; p < rj; ++p) {
        std::vector<std::vector<std::pair<int, cplx>>> jrow(wm);
        for (const Trip& t : ej.coef[p]) jrow[t.a].push_back({t.b, t.c});
        for (int o = 0; o < ri; ++o) {
            Block& B = K[(size_t)o * rj + p];
            for (const Trip& t : ei.coef[o])
                if (!jrow[t.b].empty()) {
                    if (rpos[t.a] < 0) {
                        rpos[t.a] = 0;
                        B.rows.push_back(t.a);
                    }
                    for (const auto& q : jrow[t.b])
                        if (cpos[q.first] < 0) {
                            cpos[q.first] = 0;
                            B.cols.push_back(q.first);
                        }
                }
            std::sort(B.rows.begin(), B.rows.end());
            std::sort(B.cols.begin(), B.cols.end());
            for (size_t i = 0; i < B.rows.size(); ++i) rpos[B.rows[i]] = (int)i;
            for (size_t i = 0; i < B.cols.size(); ++i) cpos[B.cols[i]] = (int)i;
            const size_t nc = B.cols.size();
            B.k.assign(B.rows.size() * nc, cplx(0.0, 0.0));
            for (const Trip& t : ei.coef[o])
                for (const auto& q : jrow[t.b]) B.k[(size_t)rpos[t.a] * nc + cpos[q.first]] += t.c * q.second;
            for (int a : B.rows) rpos[a] = -1;
            for (int c : B.cols) cpos[c] = -1;
            for (const cplx& x : B.k) kmax2 = std::max(kmax2, std::norm(x));
        }
    }
    if (kmax2 == 0.0) {  // H_eff = 0: no terms
        worthwhile = true;
        return true;
    }
    const double kmax = std::sqrt(kmax2);
    const double tol = 1e-13 * kmax, tol2 = tol * tol;
    std::vector<HostTerm> id_terms, other;
    for (int o = 0; o < ri; ++o)
        for (int p = 0; p < rj; ++p) {
            const Block& B = K[(size_t)o * rj + p];
            const int nr = (int)B.rows.size(), nc = (int)B.cols.size();
            const std::vector<cplx>& k = B.k;
            std::vector<int> nzr, nzc;  // positions in the block
            for (int a = 0; a < nr; ++a) {
                double m = 0.0;
                for (int c = 0; c < nc; ++c) m = std::max(m, std::norm(k[(size_t)a * nc + c]));
                if (m > tol2) nzr.push_back(a);
            }
            for (int c = 0; c < nc; ++c) {
                double m = 0.0;
                for (int a = 0; a < nr; ++a) m = std::max(m, std::norm(k[(size_t)a * nc + c]));
                if (m > tol2) nzc.push_back(c);
            }
            if (nzr.empty()) continue;
            const size_t trivial = std::min(nzr.size(), nzc.size());
            std::vector<HostTerm> got;
            if (!(o == 0 && p == 0)) {
                // Gaussian elimination with complete pivoting on the block: K = sum_t u_t v_t^T (|u| <= 1)
                std::vector<cplx> R = k;
                std::vector<std::vector<cplx>> us, vs;
                bool fail = false;
                while (true) {
                    size_t at = 0;
                    double m = 0.0;
                    for (size_t i = 0; i < R.size(); ++i)
                        if (std::norm(R[i]) > m) {
                            m = std::norm(R[i]);
                            at = i;
                        }
                    if (m <= tol2) break;
                    if (us.size() >= trivial) {
                        fail = true;
                        break;
                    }
                    const int i0 = (int)(at / nc), j0 = (int)(at % nc);
                    const cplx piv = R[at];
                    std::vector<cplx> u(nr), v(nc);
                    for (int a = 0; a < nr; ++a) u[a] = R[(size_t)a * nc + j0] / piv;
                    for (int c = 0; c < nc; ++c) v[c] = R[(size_t)i0 * nc + c];
                    for (int a = 0; a < nr; ++a)
                        if (u[a] != 0.0)
                            for (int c = 0; c < nc; ++c) R[(size_t)a * nc + c] -= u[a] * v[c];
                    us.push_back(std::move(u));
                    vs.push_back(std::move(v));
                }
                if (!fail) {
                    // the factors must reproduce K
                    double err = 0.0;
                    for (int a = 0; a < nr; ++a)
                        for (int c = 0; c < nc; ++c) {
                            cplx sum = 0.0;
                            for (size_t t = 0; t < us.size(); ++t) sum += us[t][a] * vs[t][c];
                            err = std::max(err, std::abs(sum - k[(size_t)a * nc + c]));
                        }
                    if (err > 1e-12 * kmax) fail = true;
                }
                if (!fail && us.size() < trivial)
                    for (size_t t = 0; t < us.size(); ++t) {
                        HostTerm h{o, p, std::vector<cplx>(wl, 0.0), std::vector<cplx>(wr, 0.0)};
                        for (int a = 0; a < nr; ++a) h.u[B.rows[a]] = us[t][a];
                        for (int c = 0; c < nc; ++c) h.v[B.cols[c]] = vs[t][c];
                        got.push_back(std::move(h));
                    }
            }
            if (got.empty()) {
                // by nonzero rows (u = e_a, v = K[a, :]) or columns (u = K[:, c], v = e_c)
                if (nzr.size() <= nzc.size()) {
                    for (int a : nzr) {
                        HostTerm h{o, p, std::vector<cplx>(wl, 0.0), std::vector<cplx>(wr, 0.0)};
                        h.u[B.rows[a]] = 1.0;
                        for (int c = 0; c < nc; ++c) h.v[B.cols[c]] = k[(size_t)a * nc + c];
                        got.push_back(std::move(h));
                    }
                } else {
                    for (int c : nzc) {
                        HostTerm h{o, p, std::vector<cplx>(wl, 0.0), std::vector<cplx>(wr, 0.0)};
                        for (int a = 0; a < nr; ++a) h.u[B.rows[a]] = k[(size_t)a * nc + c];
                        h.v[B.cols[c]] = 1.0;
                        got.push_back(std::move(h));
                    }
                }
            }
            auto& dst = (o == 0 && p == 0) ? id_terms : other;
            for (auto& h : got) dst.push_back(std::move(h));
        }
    const size_t n_t = id_terms.size() + other.size();
    // worthwhile: two GEMMs over n_t terms against two over w_l and w_r channels plus two mixing
    // passes (measured: the term form wins at w ~ 100 with n_t = w + 14, loses at w ~ 25 with
    // n_t = w + 14)
    worthwhile = (double)n_t <= 1.15 * std::max(wl, wr) + 4.0;
    n_id = (int)id_terms.size();
    ops.resize(2 * n_t);
    U.resize(n_t * wl);
    V.resize(n_t * wr);
    size_t t = 0;
    for (auto* list : {&id_terms, &other})
        for (const HostTerm& h : *list) {
            ops[2 * t] = h.o;
            ops[2 * t + 1] = h.p;
            std::copy(h.u.begin(), h.u.end(), U.begin() + t * wl);
            std::copy(h.v.begin(), h.v.end(), V.begin() + t * wr);
            ++t;
        }
    return true;
}

void build_bond_terms(Ctx& ctx, const HostCore& Wi, const HostCore& Wj, BondTerms& out) {
    out = BondTerms{};
    int n_id = 0, ri = 0, rj = 0;
    std::vector<int> ops;
    std::vector<cplx> U, V, Bi, Bj;
    bool worthwhile = false;
    if (!bond_terms_host(Wi, Wj, n_id, ops, U, V, Bi, Bj, ri, rj, worthwhile)) return;
    const int wl = Wi.wl, wr = Wj.wr, d = Wi.d, dd = d * d;
    const int n_t = (int)ops.size() / 2;
    out.wl = wl;
    out.wr = wr;
    out.d = d;
    out.n_t = n_t;
    out.n_id = n_id;
    const int n_k = n_t - n_id;
    std::vector<float> cl((size_t)2 * wl * std::max(n_t, 1), 0.f), cr((size_t)2 * wr * std::max(n_t, 1), 0.f);
    std::vector<float> kr((size_t)2 * std::max(n_k, 1) * 2 * dd, 0.f);  // per term: B_o, then B'_p (d x d)
    std::vector<double> cl64((size_t)2 * std::max(n_t, 1) * wl, 0.0), cr64((size_t)2 * std::max(n_t, 1) * wr, 0.0);
    out.real_l = out.real_r = true;
    for (int t = 0; t < n_t; ++t) {
        for (int a = 0; a < wl; ++a) {
            const cplx u = U[(size_t)t * wl + a];
            cl[2 * ((size_t)a * n_t + t)] = (float)u.real();
            cl[2 * ((size_t)a * n_t + t) + 1] = (float)u.imag();
            cl64[2 * ((size_t)t * wl + a)] = u.real();
            cl64[2 * ((size_t)t * wl + a) + 1] = u.imag();
            if (u.imag() != 0.0) out.real_l = false;
        }
        for (int c = 0; c < wr; ++c) {
            const cplx v = V[(size_t)t * wr + c];
            cr[2 * ((size_t)c * n_t + t)] = (float)v.real();
            cr[2 * ((size_t)c * n_t + t) + 1] = (float)v.imag();
            cr64[2 * ((size_t)t * wr + c)] = v.real();
            cr64[2 * ((size_t)t * wr + c) + 1] = v.imag();
            if (v.imag() != 0.0) out.real_r = false;
        }
    }
    // B_o and B'_p of each term that is not an identity; B[t][s] maps input level s to output t
    std::vector<int> kop((size_t)2 * std::max(n_k, 1), 0);
    for (int j = 0; j < n_k; ++j) {
        const int o = ops[2 * (n_id + j)], p = ops[2 * (n_id + j) + 1];
        kop[2 * j] = o;
        kop[2 * j + 1] = p;
        for (int side = 0; side < 2; ++side) {
            const cplx* b = side == 0 ? &Bi[(size_t)o * dd] : &Bj[(size_t)p * dd];
            for (int e = 0; e < dd; ++e) {
                const size_t at = ((size_t)j * 2 + side) * dd + e;
                kr[2 * at] = (float)b[e].real();
                kr[2 * at + 1] = (float)b[e].imag();
            }
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_cl = take(sizeof(float) * cl.size()), o_cr = take(sizeof(float) * cr.size()),
                 o_kr = take(sizeof(float) * kr.size()), o_cl64 = take(sizeof(double) * cl64.size()),
                 o_cr64 = take(sizeof(double) * cr64.size()), o_kop = take(sizeof(int) * kop.size());
    std::vector<unsigned char> blob(off, 0);
    std::memcpy(&blob[o_cl], cl.data(), sizeof(float) * cl.size());
    std::memcpy(&blob[o_cr], cr.data(), sizeof(float) * cr.size());
    std::memcpy(&blob[o_kr], kr.data(), sizeof(float) * kr.size());
    std::memcpy(&blob[o_cl64], cl64.data(), sizeof(double) * cl64.size());
    std::memcpy(&blob[o_cr64], cr64.data(), sizeof(double) * cr64.size());
    std::memcpy(&blob[o_kop], kop.data(), sizeof(int) * kop.size());
    out.buf.bytes = off;
    out.buf.p = ctx.dalloc(off);
    VTN_CUDA_TRY(cudaMemcpyAsync(out.buf.p, blob.data(), off, cudaMemcpyHostToDevice, ctx.stream));
    ctx.sync();  // blob is a local host buffer
    unsigned char* base = (unsigned char*)out.buf.p;
    out.Cl = (float2*)(base + o_cl);
    out.Cr = (float2*)(base + o_cr);
    out.kron = (float2*)(base + o_kr);
    out.Cl64 = (double2*)(base + o_cl64);
    out.Cr64 = (double2*)(base + o_cr64);
    out.kop = (int*)(base + o_kop);
    out.usable = true;
    out.worthwhile = worthwhile;
}

void free_bond_terms(Ctx& ctx, BondTerms& bt) {
    if (bt.buf.p) ctx.dfree(bt.buf.p);
    bt = BondTerms{};
}

namespace {

__global__ void to_f32_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double2 v = in[i];
        out[i] = make_float2((float)v.x, (float)v.y);
    }
}

// X[t][i][s1][s2][k] <- sum B_o[s1][s1'] B'_p[s2][s2'] X[t][i][s1'][s2'][k] for the terms t >= n_id:
// the operator B_o (x) B'_p on the two physical indices, applied as two d x d products (B'_p along
// s2, then B_o along s1; a side whose basis element is the identity is skipped), d*d rows of
// chi_r elements per (t, i).  One CTA per (t, i, 32 k values), in place (the tile is read whole
// before it is written).
constexpr int KRON_KT = 32;

__global__ void __launch_bounds__(256) kron_apply_kernel(int n_id, int chi_l, int d, int chi_r,
                                                         const float2* __restrict__ Kr, const int* __restrict__ kop,
                                                         float2* __restrict__ X) {
    extern __shared__ float2 ksm[];
    const int dd = d * d;
    float2* bsh = ksm;                  // B_o then B'_p (2 d d)
    float2* xs = ksm + 2 * dd;          // dd * KRON_KT: input, then the result of the first product
    float2* ys = xs + dd * KRON_KT;     // dd * KRON_KT
    const int ktiles = (chi_r + KRON_KT - 1) / KRON_KT;
    const int i = blockIdx.x / ktiles;
    const int k0 = (blockIdx.x - i * ktiles) * KRON_KT;
    const long long t = (long long)n_id + blockIdx.y;
    const int o = kop[2 * blockIdx.y], p = kop[2 * blockIdx.y + 1];
    for (int e = threadIdx.x; e < 2 * dd; e += blockDim.x) bsh[e] = Kr[(size_t)blockIdx.y * 2 * dd + e];
    float2* base = X + ((t * chi_l + i) * dd) * (long long)chi_r + k0;
    const int kk = threadIdx.x & 31, rg = threadIdx.x >> 5, ng = blockDim.x >> 5;
    const bool kin = k0 + kk < chi_r;
    for (int r = rg; r < dd; r += ng) xs[r * KRON_KT + kk] = kin ? base[(long long)r * chi_r + kk] : make_float2(0.f, 0.f);
    __syncthreads();
    float2* cur = xs;
    float2* nxt = ys;
    for (int side = 1; side >= 0; --side) {
        if ((side == 1 ? p : o) == 0) continue;  // identity
        const float2* B = bsh + side * dd;
        for (int r = rg; r < dd; r += ng) {
            const int s1 = r / d, s2 = r - (r / d) * d;
            float ax = 0.f, ay = 0.f;
            for (int q = 0; q < d; ++q) {
                // side 1: out[s1][s2] = sum_q B'[s2][q] x[s1][q];  side 0: out[s1][s2] = sum_q B[s1][q] x[q][s2]
                const float2 m = side == 1 ? B[s2 * d + q] : B[s1 * d + q];
                const float2 x = side == 1 ? cur[(s1 * d + q) * KRON_KT + kk] : cur[(q * d + s2) * KRON_KT + kk];
                ax = fmaf(m.x, x.x, ax);
                ax = fmaf(-m.y, x.y, ax);
                ay = fmaf(m.x, x.y, ay);
                ay = fmaf(m.y, x.x, ay);
            }
            nxt[r * KRON_KT + kk] = make_float2(ax, ay);
        }
        __syncthreads();
        float2* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (!kin) return;
    for (int r = rg; r < dd; r += ng) base[(long long)r * chi_r + kk] = cur[r * KRON_KT + kk];
}

// Lhat / Rhat: out[t][e] = sum_a C[a][t] env[a][e] (e < E): FP32 channel GEMM on a single-precision
// copy of the environment, else the FP64 GEMM with the transposed coefficients.  Returns the FP32
// result in *o32 or the FP64 one in *o64 (the other is null).
void fold_env(Ctx& ctx, int w_in, int n_t, long long E, const double2* env, const float2* C, bool real_c,
              const double2* C64T, float2** o32, double2** o64) {
    *o32 = nullptr;
    *o64 = nullptr;
    const long long n_in = (long long)w_in * E;
    float2* in32 = (float2*)ctx.workspace(WS_Y, sizeof(float2) * (size_t)n_in);
    float2* out32 = (float2*)ctx.workspace(WS_X, sizeof(float2) * (size_t)n_t * E);
    to_f32_kernel<<<(unsigned)((n_in + 255) / 256), 256, 0, ctx.stream>>>(env, in32, n_in);
    ctx.count_launch();
    ctx.check_launch("to_f32_kernel");
    if (channel_gemm_f32(ctx, w_in, n_t, E, C, n_t, real_c, in32, out32)) {
        *o32 = out32;
        return;
    }
    double2* out64 = (double2*)ctx.workspace(WS_Z, sizeof(double2) * (size_t)n_t * E);
    GemmArgs g;
    g.M = n_t;
    g.N = (int)E;
    g.K = w_in;
    g.A = C64T;
    g.lda = w_in;
    g.B = env;
    g.ldb = E;
    g.C = out64;
    g.ldc = E;
    gemm_c64(ctx, g);
    *o64 = out64;
}

}  // namespace

void heff_pack_terms(Ctx& ctx, const BondTerms& bt, int chi_l, int chi_r, const double2* L, const double2* R,
                     HeffPacked& pk) {
    const int n_t = bt.n_t;
    pk.terms = &bt;
    pk.chi_l = chi_l;
    pk.chi_r = chi_r;
    pk.wl = pk.wr = n_t;
    pk.ldL = tc_ksplit(chi_l);
    pk.ldR = tc_ksplit((long long)n_t * chi_r);
    if (n_t == 0) return;
    pk.L = (__nv_bfloat16*)ctx.workspace(WS_TC_L, sizeof(__nv_bfloat16) * (size_t)n_t * chi_l * pk.ldL);
    pk.R = (__nv_bfloat16*)ctx.workspace(WS_TC_R, sizeof(__nv_bfloat16) * (size_t)2 * chi_r * pk.ldR);
    float2* f32;
    double2* f64;
    // A operand of T = Lhat theta: rows (t, i), inner index j
    fold_env(ctx, bt.wl, n_t, (long long)chi_l * chi_l, L, bt.Cl, bt.real_l, bt.Cl64, &f32, &f64);
    if (f32) tc_pack(ctx, (const float2*)f32, n_t * chi_l, chi_l, 1, chi_l, 0, false, false, pk.L);
    else tc_pack(ctx, (const double2*)f64, n_t * chi_l, chi_l, 1, chi_l, 0, false, false, pk.L);
    // B operand of y = sum_t T[t] Rhat[t]: output column l, inner index (t, k): Rhat[t][k][l]
    fold_env(ctx, bt.wr, n_t, (long long)chi_r * chi_r, R, bt.Cr, bt.real_r, bt.Cr64, &f32, &f64);
    if (f32) tc_pack(ctx, (const float2*)f32, chi_r, chi_r, n_t, chi_r, (long long)chi_r * chi_r, false, true, pk.R);
    else tc_pack(ctx, (const double2*)f64, chi_r, chi_r, n_t, chi_r, (long long)chi_r * chi_r, false, true, pk.R);
}

void heff_apply_terms(Ctx& ctx, const HeffPacked& pk, const double2* theta, double2* y) {
    const BondTerms& bt = *pk.terms;
    const int d = bt.d, dd = d * d, n_t = bt.n_t, chi_l = pk.chi_l, chi_r = pk.chi_r;
    const long long n_theta = (long long)chi_l * dd * chi_r;
    if (n_t == 0) {
        VTN_CUDA_TRY(cudaMemsetAsync(y, 0, sizeof(double2) * (size_t)n_theta, ctx.stream));
        return;
    }
    const long long ldB1 = tc_ksplit(chi_l);
    const long long ldA2 = pk.ldR;
    __nv_bfloat16* B1 = (__nv_bfloat16*)ctx.workspace(WS_TC_B1, sizeof(__nv_bfloat16) * (size_t)2 * dd * chi_r * ldB1);
    float2* X = (float2*)ctx.workspace(WS_X, sizeof(float2) * (size_t)n_t * n_theta);
    __nv_bfloat16* A2 = (__nv_bfloat16*)ctx.workspace(WS_TC_A2, sizeof(__nv_bfloat16) * (size_t)chi_l * dd * ldA2);
    const double useful1 = 8.0 * (double)n_t * chi_l * (double)dd * chi_r * chi_l;
    const double useful2 = 8.0 * (double)chi_l * dd * chi_r * (double)chi_r * n_t;
    // B operand of T = Lhat theta: output column (s1 s2 k), inner index j: theta[j][(s1 s2 k)]
    tc_pack(ctx, theta, dd * chi_r, chi_l, 1, (long long)dd * chi_r, 0, false, true, B1);
    TcGemmArgs g1;
    g1.M = n_t * chi_l;
    g1.N = 2 * dd * chi_r;
    g1.K = (int)ldB1;
    g1.A = pk.L;
    g1.lda = pk.ldL;
    g1.B = B1;
    g1.ldb = ldB1;
    g1.D = X;
    g1.ldd = 2LL * dd * chi_r;
    g1.d_fp64 = false;
    g1.split3 = true;
    g1.max_kb_per_acc = ctx.tc_kb_heff;
    tc_gemm_bf16(ctx, g1, TC_HEFF, useful1);
    const int n_k = n_t - bt.n_id;
    if (n_k > 0) {
        const int t = ctx.tbegin(TC_MIX, 16.0 * n_k * (double)chi_l * dd * d * chi_r);
        VTN_REQUIRE(n_k <= 65535, "too many operator terms");
        const int ktiles = (chi_r + KRON_KT - 1) / KRON_KT;
        const dim3 grid((unsigned)((long long)chi_l * ktiles), (unsigned)n_k);
        const size_t smem = sizeof(float2) * (size_t)(2 * dd + 2 * dd * KRON_KT);
        kron_apply_kernel<<<grid, 256, smem, ctx.stream>>>(bt.n_id, chi_l, d, chi_r, bt.kron, bt.kop, X);
        ctx.count_launch();
        ctx.check_launch("kron_apply_kernel");
        ctx.tend(t);
    }
    // A operand of y = sum_t T[t] Rhat[t]: rows (i t u), inner index (t, k): T[t][(i t u)][k]
    tc_pack(ctx, (const float2*)X, chi_l * dd, chi_r, n_t, chi_r, n_theta, false, false, A2);
    TcGemmArgs g2;
    g2.M = chi_l * dd;
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

}  // namespace vtn
