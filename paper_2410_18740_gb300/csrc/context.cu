// Context services: device memory through the caller's allocator (or cudaMalloc),
// grow-only workspace slots, per-kernel-class CUDA-event timing, MPO core upload.
#include <algorithm>
#include <cstring>

#include <map>
#include <mutex>
#include <utility>

#include "vtn_internal.cuh"

namespace vtn {

void* Ctx::dalloc(size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (has_alloc) {
        p = alloc.alloc(bytes, alloc.user);
        if (!p) throw Error{VTN_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{VTN_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + "): " + cudaGetErrorString(e)};
        }
    }
    return p;
}

void Ctx::dfree(void* p) {
    if (!p) return;
    if (has_alloc) alloc.free(p, alloc.user);
    else cudaFree(p);
}

void set_smem_attr_once(const Ctx& ctx, const void* fn, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    std::lock_guard<std::mutex> lock(mu);
    int& have = done[{fn, ctx.device}];
    if (have >= bytes) return;
    VTN_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    have = bytes;
}

void* Ctx::workspace(int slot, size_t bytes) {
    if ((int)ws.size() < WS_COUNT) ws.resize(WS_COUNT);
    DevBuf& b = ws[slot];
    if (b.bytes < bytes) {
        // the stream may still use the old buffer
        sync();
        dfree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        size_t want = std::max(bytes, size_t(4096));
        b.p = dalloc(want);
        b.bytes = want;
    }
    return b.p;
}

double* Ctx::defer_reserve(size_t doubles) {
    if (defer_cap < doubles) {
        sync();
        if (defer_buf) cudaFreeHost(defer_buf);
        defer_buf = nullptr;
        defer_cap = 0;
        const size_t want = std::max(doubles, size_t(4096));
        VTN_CUDA_TRY(cudaMallocHost((void**)&defer_buf, sizeof(double) * want));
        defer_cap = want;
    }
    return defer_buf;
}

int Ctx::tbegin(int cls, double flops) {
    if (!timing) return -1;
    if (pending.size() > 4096 && open_intervals == 0) tflush();
    cudaEvent_t a, bb;
    if (event_pool.size() >= 2) {
        a = event_pool.back(); event_pool.pop_back();
        bb = event_pool.back(); event_pool.pop_back();
    } else {
        VTN_CUDA_TRY(cudaEventCreate(&a));
        VTN_CUDA_TRY(cudaEventCreate(&bb));
    }
    VTN_CUDA_TRY(cudaEventRecord(a, stream));
    pending.push_back(Pending{a, bb, cls, flops});
    ++open_intervals;
    return (int)pending.size() - 1;
}

void Ctx::tend(int idx) {
    if (idx < 0) return;
    VTN_CUDA_TRY(cudaEventRecord(pending[idx].b, stream));
    --open_intervals;
}

void Ctx::tflush() {
    if (pending.empty()) return;
    sync();
    for (auto& p : pending) {
        float ms = 0.f;
        VTN_CUDA_TRY(cudaEventElapsedTime(&ms, p.a, p.b));
        tc[p.cls].launches += 1;
        tc[p.cls].flops += p.flops;
        tc[p.cls].seconds += ms * 1e-3;
        event_pool.push_back(p.a);
        event_pool.push_back(p.b);
    }
    pending.clear();
}

void Ctx::check_dstatus() {
    if (!dstatus) return;
    VTN_CUDA_TRY(cudaMemcpyAsync(pinned + 4095, dstatus, sizeof(int), cudaMemcpyDeviceToHost, stream));
    sync();
    int v = 0;
    std::memcpy(&v, pinned + 4095, sizeof(int));
    if (v != 0) {
        VTN_CUDA_TRY(cudaMemsetAsync(dstatus, 0, sizeof(int), stream));
        sync();
        throw Error{VTN_ETIMEOUT, "a bounded device-side wait gave up (tensor-core pipeline)"};
    }
}

void Ctx::check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Error{VTN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e)};
}

// ------------------------------------------------------------------ cores
HostCore core_from_abi(const vtn_core* c) {
    VTN_REQUIRE(c != nullptr, "null core");
    VTN_REQUIRE(c->w_left >= 1 && c->w_right >= 1 && c->d >= 1 && c->d <= 16 && c->nnz >= 0,
                "core shape out of range (need w >= 1, 1 <= d <= 16)");
    VTN_REQUIRE(c->nnz == 0 || (c->rows && c->cols && c->ops), "core arrays missing");
    HostCore h;
    h.wl = c->w_left;
    h.wr = c->w_right;
    h.d = c->d;
    const int dd = c->d * c->d;
    for (int k = 0; k < c->nnz; ++k) {
        VTN_REQUIRE(c->rows[k] >= 0 && c->rows[k] < c->w_left && c->cols[k] >= 0 && c->cols[k] < c->w_right,
                    "core entry channel out of range");
        h.rows.push_back(c->rows[k]);
        h.cols.push_back(c->cols[k]);
        bool ident = true;
        cplx s(c->ops[2 * (size_t)k * dd], c->ops[2 * (size_t)k * dd + 1]);
        for (int i = 0; i < c->d; ++i)
            for (int j = 0; j < c->d; ++j) {
                cplx v(c->ops[2 * ((size_t)k * dd + i * c->d + j)], c->ops[2 * ((size_t)k * dd + i * c->d + j) + 1]);
                h.ops.push_back(v);
                if (i == j ? (v != s) : (v != cplx(0, 0))) ident = false;
            }
        h.ident.push_back(ident ? 1 : 0);
    }
    return h;
}

void upload_core(Ctx& ctx, const HostCore& hc, DevCore& dc) {
    dc.wl = hc.wl;
    dc.wr = hc.wr;
    dc.d = hc.d;
    dc.nnz = hc.nnz();
    const int nnz = dc.nnz, d = hc.d;
    // grouped index lists of a subset of the entries: by output column (ptr over wr) or row
    auto group = [&](bool by_col, bool dense_only, std::vector<int>& ptr, std::vector<int>& src,
                     std::vector<int>& op) {
        const int w_out = by_col ? hc.wr : hc.wl;
        ptr.assign(w_out + 1, 0);
        for (int k = 0; k < nnz; ++k)
            if (!dense_only || !hc.ident[k]) ptr[(by_col ? hc.cols[k] : hc.rows[k]) + 1]++;
        for (int b = 0; b < w_out; ++b) ptr[b + 1] += ptr[b];
        src.assign(std::max(ptr[w_out], 0), 0);
        op.assign(src.size(), 0);
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int k = 0; k < nnz; ++k) {
            if (dense_only && hc.ident[k]) continue;
            const int o = by_col ? hc.cols[k] : hc.rows[k];
            const int pos = fill[o]++;
            src[pos] = by_col ? hc.rows[k] : hc.cols[k];
            op[pos] = k;
        }
    };
    std::vector<int> col_ptr, col_src, col_op, row_ptr, row_src, row_op;
    group(true, false, col_ptr, col_src, col_op);
    group(false, false, row_ptr, row_src, row_op);
    dc.n_ident = 0;
    dc.n_dense = 0;
    for (int k = 0; k < nnz; ++k) (hc.ident[k] ? dc.n_ident : dc.n_dense)++;
    // a core whose scaled-identity entries fill a large part of the w_l x w_r channel matrix (the
    // collapse core at the centre of the chain) keeps them as a dense matrix C[a][b] as well, and
    // its remaining entries as separate lists: its FP32 mixing is then a channel GEMM plus a
    // sparse pass over the few dense d x d entries
    dc.has_cid = dc.n_ident >= 4 * std::max(hc.wl, hc.wr);
    std::vector<float> cid;
    std::vector<int> dcp, dcs, dco, drp, drs, dro;
    if (dc.has_cid) {
        cid.assign((size_t)2 * hc.wl * hc.wr, 0.f);
        dc.cid_real = true;
        for (int k = 0; k < nnz; ++k) {
            if (!hc.ident[k]) continue;
            const cplx c = hc.ops[(size_t)k * d * d];
            const size_t at = (size_t)hc.rows[k] * hc.wr + hc.cols[k];
            cid[2 * at] += (float)c.real();
            cid[2 * at + 1] += (float)c.imag();
            if (c.imag() != 0.0) dc.cid_real = false;
        }
        group(true, true, dcp, dcs, dco);
        group(false, true, drp, drs, dro);
    }
    // one allocation holding everything
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    auto ibytes = [](const std::vector<int>& v) { return sizeof(int) * std::max(v.size(), size_t(1)); };
    const size_t o_cp = take(ibytes(col_ptr)), o_cs = take(ibytes(col_src)), o_co = take(ibytes(col_op)),
                 o_rp = take(ibytes(row_ptr)), o_rs = take(ibytes(row_src)), o_ro = take(ibytes(row_op)),
                 o_ops = take(sizeof(double2) * std::max((size_t)nnz * d * d, size_t(1))),
                 o_id = take(std::max(nnz, 1)),
                 o_f32 = take(sizeof(float) * 2 * std::max((size_t)nnz * d * d, size_t(1))),
                 o_cid = take(sizeof(float) * std::max(cid.size(), size_t(1))), o_dcp = take(ibytes(dcp)),
                 o_dcs = take(ibytes(dcs)), o_dco = take(ibytes(dco)), o_drp = take(ibytes(drp)),
                 o_drs = take(ibytes(drs)), o_dro = take(ibytes(dro));
    std::vector<unsigned char> blob(off, 0);
    auto put = [&](size_t o, const void* p, size_t bytes) {
        if (bytes) std::memcpy(&blob[o], p, bytes);
    };
    auto puti = [&](size_t o, const std::vector<int>& v) { put(o, v.data(), sizeof(int) * v.size()); };
    puti(o_cp, col_ptr);
    puti(o_cs, col_src);
    puti(o_co, col_op);
    puti(o_rp, row_ptr);
    puti(o_rs, row_src);
    puti(o_ro, row_op);
    if (nnz) {
        put(o_ops, hc.ops.data(), sizeof(double2) * (size_t)nnz * d * d);
        put(o_id, hc.ident.data(), nnz);
        std::vector<float> f32((size_t)nnz * d * d * 2);
        for (size_t i = 0; i < (size_t)nnz * d * d; ++i) {
            f32[2 * i] = (float)hc.ops[i].real();
            f32[2 * i + 1] = (float)hc.ops[i].imag();
        }
        put(o_f32, f32.data(), sizeof(float) * f32.size());
    }
    put(o_cid, cid.data(), sizeof(float) * cid.size());
    puti(o_dcp, dcp);
    puti(o_dcs, dcs);
    puti(o_dco, dco);
    puti(o_drp, drp);
    puti(o_drs, drs);
    puti(o_dro, dro);
    DevBuf b;
    b.bytes = off;
    b.p = ctx.dalloc(off);
    VTN_CUDA_TRY(cudaMemcpyAsync(b.p, blob.data(), off, cudaMemcpyHostToDevice, ctx.stream));
    ctx.sync();  // blob is a stack-local host buffer
    unsigned char* base = (unsigned char*)b.p;
    dc.col_ptr = (int*)(base + o_cp);
    dc.col_src = (int*)(base + o_cs);
    dc.col_op = (int*)(base + o_co);
    dc.row_ptr = (int*)(base + o_rp);
    dc.row_src = (int*)(base + o_rs);
    dc.row_op = (int*)(base + o_ro);
    dc.ops = (double2*)(base + o_ops);
    dc.ident = base + o_id;
    dc.ops_f32 = (float2*)(base + o_f32);
    if (dc.has_cid) {
        dc.cid = (float2*)(base + o_cid);
        dc.dcol_ptr = (int*)(base + o_dcp);
        dc.dcol_src = (int*)(base + o_dcs);
        dc.dcol_op = (int*)(base + o_dco);
        dc.drow_ptr = (int*)(base + o_drp);
        dc.drow_src = (int*)(base + o_drs);
        dc.drow_op = (int*)(base + o_dro);
    }
    dc.bufs.push_back(b);
}

void free_core(Ctx& ctx, DevCore& dc) {
    for (auto& b : dc.bufs) ctx.dfree(b.p);
    dc.bufs.clear();
}

}  // namespace vtn
