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
    std::vector<int> col_ptr(hc.wr + 1, 0), row_ptr(hc.wl + 1, 0);
    for (int k = 0; k < nnz; ++k) {
        col_ptr[hc.cols[k] + 1]++;
        row_ptr[hc.rows[k] + 1]++;
    }
    for (int b = 0; b < hc.wr; ++b) col_ptr[b + 1] += col_ptr[b];
    for (int a = 0; a < hc.wl; ++a) row_ptr[a + 1] += row_ptr[a];
    std::vector<int> col_src(nnz), col_op(nnz), row_src(nnz), row_op(nnz);
    std::vector<int> cfill(col_ptr.begin(), col_ptr.end() - 1), rfill(row_ptr.begin(), row_ptr.end() - 1);
    for (int k = 0; k < nnz; ++k) {
        int pc = cfill[hc.cols[k]]++;
        col_src[pc] = hc.rows[k];
        col_op[pc] = k;
        int pr = rfill[hc.rows[k]]++;
        row_src[pr] = hc.cols[k];
        row_op[pr] = k;
    }
    dc.n_ident = 0;
    dc.n_dense = 0;
    for (int k = 0; k < nnz; ++k) (hc.ident[k] ? dc.n_ident : dc.n_dense)++;
    {
        std::vector<int> dcol(hc.wr, 0), drow(hc.wl, 0);
        for (int k = 0; k < nnz; ++k)
            if (!hc.ident[k]) {
                dcol[hc.cols[k]]++;
                drow[hc.rows[k]]++;
            }
        dc.max_dense_col = dcol.empty() ? 0 : *std::max_element(dcol.begin(), dcol.end());
        dc.max_dense_row = drow.empty() ? 0 : *std::max_element(drow.begin(), drow.end());
    }
    // one allocation holding everything
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) & ~size_t(255); return o; };
    size_t o_cp = take(sizeof(int) * (hc.wr + 1)), o_cs = take(sizeof(int) * std::max(nnz, 1)),
           o_co = take(sizeof(int) * std::max(nnz, 1)), o_rp = take(sizeof(int) * (hc.wl + 1)),
           o_rs = take(sizeof(int) * std::max(nnz, 1)), o_ro = take(sizeof(int) * std::max(nnz, 1)),
           o_ops = take(sizeof(double2) * std::max((size_t)nnz * d * d, size_t(1))),
           o_id = take(std::max(nnz, 1));
    std::vector<unsigned char> blob(off, 0);
    std::memcpy(&blob[o_cp], col_ptr.data(), sizeof(int) * col_ptr.size());
    if (nnz) {
        std::memcpy(&blob[o_cs], col_src.data(), sizeof(int) * nnz);
        std::memcpy(&blob[o_co], col_op.data(), sizeof(int) * nnz);
        std::memcpy(&blob[o_rs], row_src.data(), sizeof(int) * nnz);
        std::memcpy(&blob[o_ro], row_op.data(), sizeof(int) * nnz);
        std::memcpy(&blob[o_ops], hc.ops.data(), sizeof(double2) * (size_t)nnz * d * d);
        std::memcpy(&blob[o_id], hc.ident.data(), nnz);
    }
    std::memcpy(&blob[o_rp], row_ptr.data(), sizeof(int) * row_ptr.size());
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
    dc.bufs.push_back(b);
}

void free_core(Ctx& ctx, DevCore& dc) {
    for (auto& b : dc.bufs) ctx.dfree(b.p);
    dc.bufs.clear();
}

}  // namespace vtn
