// C ABI of libglm (declared in include/glm.h): contexts, problem set-up and the log-likelihood /
// gradient evaluation.  Host-side validation of the spike trains, device workspace, stream plumbing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "glm_internal.h"

using namespace glm;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int fail(glm_ctx* c, int code, const std::string& msg) {
    if (c) c->last_error = msg;
    return code;
}

int cuda_fail(glm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, GLM_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define GLM_CK(call)                                   \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

void free_all(glm_ctx* c) {
    for (int k = 0; k < c->n_allocs; ++k) cudaFree(c->allocs[k]);
    c->n_allocs = 0;
    c->ws_used = 0;
    c->buf = Buffers();
    c->has_problem = false;
    c->c_ready = false;
    c->g_mode = 1;
    c->g_nsplit = 0;
}

// Device allocation charged against the workspace cap.
int ws_alloc(glm_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (c->ws_cap && c->ws_used + bytes > c->ws_cap)
        return fail(c, GLM_ERR_OOM, "workspace cap exceeded (" + std::to_string(c->ws_used + bytes) + " > " +
                                        std::to_string(c->ws_cap) + " bytes)");
    if (c->n_allocs >= 64) return fail(c, GLM_ERR_OOM, "too many workspace buffers");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GLM_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " +
                                        cudaGetErrorString(e));
    }
    c->allocs[c->n_allocs] = *p;
    c->alloc_bytes[c->n_allocs] = bytes;
    c->n_allocs++;
    c->ws_used += bytes;
    return GLM_OK;
}

template <typename T>
int ws_alloc_t(glm_ctx* c, T** p, size_t count) {
    void* v = nullptr;
    int rc = ws_alloc(c, &v, count * sizeof(T));
    *p = reinterpret_cast<T*>(v);
    return rc;
}

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// ---- tracing: CUDA events around each kernel group while profiling is enabled ----
int prof_begin(glm_ctx* c, const char* name) {
    if (!c->prof_on) return -1;
    int id = -1;
    for (int k = 0; k < c->prof_nnames; ++k)
        if (std::strcmp(c->prof_names[k], name) == 0) id = k;
    if (id < 0) {
        if (c->prof_nnames == glm_ctx::PROF_NAMES) return -1;
        id = c->prof_nnames++;
        c->prof_names[id] = name;
    }
    if (c->prof_n == c->prof_cap) {
        const int ncap = c->prof_cap ? 2 * c->prof_cap : 256;
        auto* nr = new (std::nothrow) glm_ctx::ProfRec[ncap];
        if (!nr) return -1;
        for (int k = 0; k < c->prof_cap; ++k) nr[k] = c->prof_recs[k];
        for (int k = c->prof_cap; k < ncap; ++k) {
            cudaEventCreate(&nr[k].a);
            cudaEventCreate(&nr[k].b);
        }
        delete[] c->prof_recs;
        c->prof_recs = nr;
        c->prof_cap = ncap;
    }
    const int slot = c->prof_n++;
    c->prof_recs[slot].name = id;
    cudaEventRecord(c->prof_recs[slot].a, c->stream);
    return slot;
}

void prof_end(glm_ctx* c, int slot) {
    if (slot >= 0) cudaEventRecord(c->prof_recs[slot].b, c->stream);
}

// fold the recorded event pairs into the per-name totals (synchronises the stream)
void prof_fold(glm_ctx* c) {
    if (c->prof_n == 0) return;
    cudaStreamSynchronize(c->stream);
    for (int k = 0; k < c->prof_n; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_recs[k].a, c->prof_recs[k].b) == cudaSuccess) {
            c->prof_ms[c->prof_recs[k].name] += ms;
            c->prof_count[c->prof_recs[k].name] += 1;
        }
    }
    cudaGetLastError();
    c->prof_n = 0;
}

#define GLM_RUN(name, nkernels, call)                  \
    do {                                               \
        const int slot_ = prof_begin(c, name);         \
        GLM_CK(call);                                  \
        prof_end(c, slot_);                            \
        c->launches += (nkernels);                     \
    } while (0)

// rows [i0, i1) sorted and inside [0, T)
bool rows_valid(int32_t i0, int32_t i1, int64_t T, const int64_t* offs, const int32_t* bins) {
    for (int32_t i = i0; i < i1; ++i) {
        int64_t prev = -1;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            const int64_t s = bins[k];
            if (s < 0 || s >= T || s <= prev) return false;
            prev = s;
        }
    }
    return true;
}

// offsets of a CSR spike list: offs[0] = 0, non-decreasing, and bins given when there are spikes
int validate_offs(glm_ctx* c, int32_t n, const int64_t* offs, const int32_t* bins) {
    if (offs[0] != 0) return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE, "offs[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (offs[i + 1] < offs[i]) return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE, "offs must be non-decreasing");
    if (offs[n] > 0 && !bins) return fail(c, GLM_ERR_INVALID_ARG, "bins is NULL but offs[n] > 0");
    return GLM_OK;
}

// the error for the first fault, at spike index k: bin out of range (range) or not above the previous bin
int bins_fault(glm_ctx* c, int32_t n, const int64_t* offs, const int32_t* bins, int64_t k, bool range) {
    const int32_t i = (int32_t)(std::upper_bound(offs, offs + n + 1, k) - offs - 1);
    if (range)
        return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE,
                    "spike bin " + std::to_string(bins[k]) + " of row " + std::to_string(i) + " outside [0, n_bins)");
    return fail(c, GLM_ERR_UNSORTED_SPIKES,
                "row " + std::to_string(i) + ": bins not strictly increasing at index " + std::to_string(k));
}

int validate_spikes(glm_ctx* c, int32_t n, int64_t T, const int64_t* offs, const int32_t* bins) {
    int rc = validate_offs(c, n, offs, bins);
    if (rc) return rc;
    const int64_t q = offs[n];
    // large recordings: the rows are checked on several host threads, split by spike count; only when
    // one of them finds a fault does the single pass below run, to name the first one
    const int nt = (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency()));
    if (q >= ((int64_t)1 << 20) && nt > 1 && n >= nt) {
        std::vector<int32_t> cut(nt + 1, n);
        cut[0] = 0;
        for (int t = 1; t < nt; ++t)
            cut[t] = (int32_t)(std::upper_bound(offs, offs + n + 1, q * t / nt) - offs - 1);
        for (int t = 1; t <= nt; ++t) cut[t] = std::max(cut[t], cut[t - 1]);
        std::vector<char> ok(nt, 1);
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t)
            th.emplace_back([&, t]() { ok[t] = rows_valid(cut[t], cut[t + 1], T, offs, bins) ? 1 : 0; });
        for (auto& x : th) x.join();
        if (std::all_of(ok.begin(), ok.end(), [](char v) { return v != 0; })) return GLM_OK;
    }
    for (int32_t i = 0; i < n; ++i) {
        int64_t prev = -1;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            const int64_t s = bins[k];
            if (s < 0 || s >= T) return bins_fault(c, n, offs, bins, k, true);
            if (s <= prev) return bins_fault(c, n, offs, bins, k, false);
            prev = s;
        }
    }
    return GLM_OK;
}

// The spikes of a recording with the shape of the current problem into its offs / bins.  They are copied to
// staging buffers and checked there on the device (bins in range, rows strictly increasing), so a recording
// that fails leaves the current problem as it was; then the staging and current buffers swap.  Without room
// for the staging buffers the host checks the bins and they are copied in place.
int stage_spikes(glm_ctx* c, int32_t n, int64_t T, const int64_t* offs, const int32_t* bins) {
    Buffers& B = c->buf;
    const int64_t q = offs[n];
    if (!(B.offs_next && B.bins_next && B.bad)) {
        const std::string keep = c->last_error;
        if (!B.offs_next) ws_alloc_t(c, &B.offs_next, n + 1);
        if (!B.bins_next) ws_alloc_t(c, &B.bins_next, q > 0 ? q : 1);
        if (!B.bad) ws_alloc_t(c, &B.bad, 1);
        c->last_error = keep;
    }
    if (!(B.offs_next && B.bins_next && B.bad)) {
        int rc = validate_spikes(c, n, T, offs, bins);
        if (rc) return rc;
        GLM_CK(cudaMemcpyAsync(B.offs, offs, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream));
        if (q > 0) GLM_CK(cudaMemcpyAsync(B.bins, bins, sizeof(int32_t) * q, cudaMemcpyHostToDevice, c->stream));
        return GLM_OK;
    }
    GLM_CK(cudaMemcpyAsync(B.offs_next, offs, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    if (q > 0) GLM_CK(cudaMemcpyAsync(B.bins_next, bins, sizeof(int32_t) * q, cudaMemcpyHostToDevice, c->stream));
    GLM_CK(launch_check_bins(c, n, q, T, B.offs_next, B.bins_next, B.bad));
    c->launches += q > 0 ? 1 : 0;
    unsigned long long key = ~0ull;
    GLM_CK(cudaMemcpyAsync(&key, B.bad, sizeof(key), cudaMemcpyDeviceToHost, c->stream));
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (key != ~0ull) return bins_fault(c, n, offs, bins, (int64_t)(key >> 1), (key & 1ull) == 0);
    std::swap(B.offs, B.offs_next);
    std::swap(B.bins, B.bins_next);
    B.aoffs = B.offs;  // one-bin delay: the filter's sources are the spikes themselves
    B.abins = B.bins;
    return GLM_OK;
}

// Device buffers of the problem described by c->pb (frees everything on failure).
int alloc_problem(glm_ctx* c) {
    const Problem& P = c->pb;
    const int32_t n = P.n;
    const bool tensor = P.prec != GLM_PREC_F32;
    Buffers& B = c->buf;
    const size_t nn = (size_t)n * n;
    const size_t esz = tensor ? 2 : 4;
    const int64_t ntile = P.Tpad / (tensor ? tc_tile_t() : simt_tile_t());
    int rc;
    B.ldn = round_up(n, 64);
    if ((rc = ws_alloc_t(c, &B.offs, n + 1)) || (rc = ws_alloc_t(c, &B.bins, P.q > 0 ? P.q : 1)) ||
        (rc = ws_alloc_t(c, &B.seg_carry, (size_t)n * P.nseg)) ||
        (rc = ws_alloc_t(c, &B.seg_first, (size_t)n * P.nseg)) || (rc = ws_alloc_t(c, &B.pow_seg, SEG + 1)) ||
        (rc = ws_alloc_t(c, &B.qd, n)) || (rc = ws_alloc_t(c, &B.C, nn)) ||
        (rc = ws_alloc(c, &B.X, (size_t)n * P.Tc * esz)) || (rc = ws_alloc(c, &B.E, (size_t)n * P.Tc * esz)) ||
        (P.chunk && (rc = ws_alloc_t(c, &B.Gacc, nn))) ||
        (rc = ws_alloc_t(c, &B.part_e, (size_t)n * ntile * (P.ct ? CT_PARTS : 1))) ||
        (rc = ws_alloc_t(c, &B.part_g, nn * (tensor ? tc_nsplit_max(c) : grad_nsplit(c)))) ||
        (rc = ws_alloc_t(c, &B.flags, 4)) || (rc = ws_alloc_t(c, &B.Lrows, n)) || (rc = ws_alloc_t(c, &B.scal, 8)) ||
        (rc = ws_alloc_t(c, &B.eb, n)) || (P.xlo && (rc = ws_alloc(c, &B.Xlo, (size_t)P.n * P.Tc * 2))) ||
        (rc = ws_alloc_t(c, &B.part_s, (size_t)n * ntile * (P.ct ? CT_PARTS : 1))) ||
        (tensor && (rc = ws_alloc(c, &B.Wsplit, 2 * (size_t)n * B.ldn * 2)))) {
        free_all(c);
        return rc;
    }
    if (P.ct || P.delay_bins > 1) {
        if ((rc = ws_alloc_t(c, &B.aoffs, n + 1)) || (rc = ws_alloc_t(c, &B.abins, P.qa > 0 ? P.qa : 1)) ||
            (rc = ws_alloc_t(c, &B.aseg_first, (size_t)n * P.nseg))) {
            free_all(c);
            return rc;
        }
    }
    if (P.self_shift > 0 &&
        ((rc = ws_alloc_t(c, &B.part_self, (size_t)n * ntile)) || (rc = ws_alloc_t(c, &B.gself, n)))) {
        free_all(c);
        return rc;
    }
    if (P.ct) {
        if ((rc = ws_alloc_t(c, &B.ctime, P.Tpad + 1)) || (rc = ws_alloc_t(c, &B.col_a, P.Tpad)) ||
            (rc = ws_alloc_t(c, &B.colc, 8 * (size_t)P.Tpad)) || (rc = ws_alloc_t(c, &B.seg_mul, P.nseg)) ||
            (rc = ws_alloc_t(c, &B.tile_span, P.nseg))) {
            free_all(c);
            return rc;
        }
    } else if (P.delay_bins <= 1) {
        B.aoffs = B.offs;
        B.abins = B.bins;
        B.aseg_first = B.seg_first;
    }
    if (tensor) {
        cudaError_t e = tc_prepare_maps(c);
        if (e != cudaSuccess) {
            free_all(c);
            return cuda_fail(c, e, "cuTensorMapEncodeTiled");
        }
    }
    return GLM_OK;
}

int ensure_spike_term(glm_ctx* c);

int do_prepare(glm_ctx* c) {
    Problem& P = c->pb;
    if (P.ct) {
        // column decays for this tau, then carries, filter and spike term as on the grid
        c->c_ready = false;
        GLM_RUN("ct_consts", 1, launch_ct_consts(c));
        GLM_RUN("carry", 3, launch_carry(c));
        if (!P.chunk) GLM_RUN("filter_scan", 1, launch_filter_cache(c));  // chunked: filtered per use
        return ensure_spike_term(c);
    }
    P.a = std::exp(-P.dt / P.tau);
    fill_scan_consts(P.a, &c->sc);
    std::vector<double> pw(SEG + 1);
    for (int k = 0; k <= SEG; ++k) pw[k] = std::exp(-(double)k * P.dt / P.tau);
    GLM_CK(cudaMemcpyAsync(c->buf.pow_seg, pw.data(), sizeof(double) * (SEG + 1), cudaMemcpyHostToDevice,
                           c->stream));
    c->c_ready = false;
    GLM_RUN("carry", 2, launch_carry(c));
    if (!P.chunk) {  // chunked: filtered per use
        // the 16-bit forms' spike term reads the raster from E: the filter writes it on the way
        const bool raster = P.prec != GLM_PREC_F32 && P.delay_bins <= 1;
        GLM_RUN("filter_scan", 1, launch_filter_cache(c, 0, -1, raster ? c->buf.E : nullptr));
        c->raster_in_E = raster;
    }
    // The spike term C (the W-independent part of dL/dW, Eq. 12): a gather of X at the spike bins for the
    // plain FP32 form, S (X_hi + X_lo)^T on the tensor cores for the 16-bit forms.  The spike part of L
    // comes from U at the spike bins in the U-product epilogue instead (its rounding then cancels against
    // that of the integral part).
    int rc = ensure_spike_term(c);
    if (rc) return rc;
    // pw is a pageable host buffer: the copy above has been staged before cudaMemcpyAsync returned
    return GLM_OK;
}

// The spike term C of the current problem and tau (computed on the first request).
int ensure_spike_term(glm_ctx* c) {
    if (c->c_ready) return GLM_OK;
    Buffers& B = c->buf;
    const size_t nn = (size_t)c->pb.n * c->pb.n;
    if (c->pb.prec != GLM_PREC_F32) {
        GLM_RUN("spike_term", 0, launch_tc_spike_term(c));  // counts its own launches
    } else {
        int rc;
        if (!B.C_part && (rc = ws_alloc_t(c, &B.C_part, nn * spike_term_parts(c)))) return rc;
        GLM_RUN("spike_term", 2, launch_spike_term(c, B.C));
    }
    c->c_ready = true;
    return GLM_OK;
}

// Buffers of dL/dtau (allocated by the first request for it).
int prepare_dtau(glm_ctx* c) {
    Buffers& B = c->buf;
    const Problem& P = c->pb;
    int rc;
    // grid: 5 sums per row and tile; continuous time: 7 per row, tile and part of a tile's columns
    if (!B.part_tau &&
        ((rc = ws_alloc_t(c, &B.part_tau, (P.ct ? 7 * CT_PARTS : 5) * (size_t)P.n * (P.Tpad / tc_tile_t()))) ||
         (rc = ws_alloc_t(c, &B.tau_rows, P.n))))
        return rc;
    return GLM_OK;
}

}  // namespace

namespace glm {

int set_error(glm_ctx* c, int code, const char* msg) { return fail(c, code, msg); }

// Device list of the rows of the context's row range (allocated with the problem's workspace).
int ensure_range_rows(glm_ctx* c) {
    if (c->buf.range_rows) return GLM_OK;
    const int32_t m = c->row_r1 - c->row_r0;
    int rc = ws_alloc_t(c, &c->buf.range_rows, m > 0 ? m : 1);
    if (rc) return rc;
    std::vector<int32_t> r(m > 0 ? m : 1);
    for (int32_t k = 0; k < m; ++k) r[k] = c->row_r0 + k;
    GLM_CK(cudaMemcpyAsync(c->buf.range_rows, r.data(), sizeof(int32_t) * r.size(), cudaMemcpyHostToDevice, c->stream));
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());  // r is a host temporary
    return GLM_OK;
}

// Queue one evaluation at (W, b) on the context's stream; no synchronisation.  With reuse_u the U
// product is skipped: E and the per-tile sums must already hold the values at this (W, b).
int eval_enqueue(glm_ctx* c, const float* W, const float* b, double* L_rows, double* G, double* gb, bool want_grad,
                 bool reuse_u, bool tau, const int32_t* rows, int32_t m) {
    const bool tensor = c->pb.prec != GLM_PREC_F32;
    const Problem& P = c->pb;
    if (!rows && c->row_r1 >= 0) {
        // a row range: only its rows are evaluated (the others' outputs are set to zero)
        int rc = ensure_range_rows(c);
        if (rc) return rc;
        rows = c->buf.range_rows;
        m = c->row_r1 - c->row_r0;
    }
    if (P.chunk) {
        // X recomputed chunk by chunk: filter, U product and E X^T per chunk; E X^T summed over the chunks.
        // Nothing of a previous evaluation survives, so a reuse request evaluates again (every row).
        if (reuse_u) rows = nullptr;
        for (int64_t t0 = 0; t0 < P.Tpad; t0 += P.Tc) {
            const int64_t len = std::min(P.Tc, P.Tpad - t0);
            GLM_RUN("filter_scan", 1, launch_filter_cache(c, t0 / SEG, (t0 + len) / SEG));
            GLM_RUN("u_epilogue", 3, launch_tc_u_epilogue(c, W, b, tau, rows, m, t0, len));
            if (want_grad) {
                int ns = 0;
                GLM_RUN("grad", 1, launch_tc_grad(c, len, &ns));
                GLM_RUN("grad", 1, launch_sum_splits(c, ns, c->buf.Gacc, t0 > 0));
            }
        }
        GLM_RUN("reduce", want_grad ? 2 : 1,
                launch_reduce(c, W, b, L_rows, G, gb, want_grad, P.Tpad / tc_tile_t(), 0, c->buf.Gacc));
        return GLM_OK;
    }
    if (!reuse_u) {
        if (tensor)
            GLM_RUN("u_epilogue", 3, launch_tc_u_epilogue(c, W, b, tau, rows, m));
        else
            GLM_RUN("u_epilogue", 2, launch_simt_u_epilogue(c, W, b, rows, m));
    }
    if (want_grad) {
        if (tensor)
            GLM_RUN("grad", 1, launch_tc_grad(c));
        else
            GLM_RUN("grad", 1, launch_simt_grad(c));
    }
    const int64_t ntile = c->pb.Tpad / (tensor ? tc_tile_t() : simt_tile_t());
    const int nsplit = tensor ? tc_nsplit(c) : grad_nsplit(c);
    GLM_RUN("reduce", want_grad ? 2 : 1, launch_reduce(c, W, b, L_rows, G, gb, want_grad, ntile, nsplit));
    return GLM_OK;
}

// Synchronise and turn the device flags raised since the last reset into a status.
int eval_status(glm_ctx* c) {
    int fl[2] = {0, 0};
    GLM_CK(cudaMemcpyAsync(fl, c->buf.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    if (fl[1]) return fail(c, GLM_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
    if (fl[0] & 1) return fail(c, GLM_ERR_NONFINITE, "exp(U) overflowed or an input was not finite");
    return GLM_OK;
}

cudaError_t reset_flags(glm_ctx* c) { return cudaMemsetAsync(c->buf.flags, 0, 2 * sizeof(int), c->stream); }

int ws_alloc_bytes(glm_ctx* c, void** p, size_t bytes) { return ws_alloc(c, p, bytes); }

}  // namespace glm

extern "C" {

int glm_version(void) { return 100; }

const char* glm_strerror(int code) {
    switch (code) {
        case GLM_OK: return "ok";
        case GLM_ERR_INVALID_ARG: return "invalid argument";
        case GLM_ERR_UNSORTED_SPIKES: return "spike bins of a row are not strictly increasing";
        case GLM_ERR_SPIKE_OUT_OF_RANGE: return "spike bin outside [0, n_bins) or malformed offsets";
        case GLM_ERR_OOM: return "out of device memory or workspace cap exceeded";
        case GLM_ERR_CUDA: return "CUDA error";
        case GLM_ERR_NONFINITE: return "non-finite value (input or exp overflow)";
        case GLM_ERR_TIMEOUT: return "device-side wait timed out";
        case GLM_ERR_UNSUPPORTED_ARCH: return "tensor-core precision needs an sm_103 GPU";
        case GLM_ERR_NO_PROBLEM: return "no problem set (call glm_set_problem first)";
        case GLM_ERR_UNSUPPORTED: return "unsupported request";
        case GLM_ERR_SCRATCH_TOO_SMALL: return "problem too large for the fixed scratch of glm_loglik_noalloc";
        default: return "unknown status";
    }
}

const char* glm_last_error(const glm_ctx* c) { return c ? c->last_error.c_str() : ""; }

int glm_create(glm_ctx** out, int device, size_t workspace_cap_bytes, void* cuda_stream) {
    if (!out) return GLM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GLM_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return GLM_ERR_INVALID_ARG;
    glm_ctx* c = new (std::nothrow) glm_ctx();
    if (!c) return GLM_ERR_OOM;
    c->device = device;
    c->ws_cap = workspace_cap_bytes;
    c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete c;
        return GLM_ERR_CUDA;
    }
    c->sm_count = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    *out = c;
    return GLM_OK;
}

void glm_destroy(glm_ctx* c) {
    if (!c) return;
    {
        DeviceGuard g(c->device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        else cudaDeviceSynchronize();
        free_all(c);
        for (int k = 0; k < c->prof_cap; ++k) {
            cudaEventDestroy(c->prof_recs[k].a);
            cudaEventDestroy(c->prof_recs[k].b);
        }
        delete[] c->prof_recs;
    }
    delete c;
}

int glm_profile_enable(glm_ctx* c, int enable) {
    if (!c) return GLM_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    prof_fold(c);
    c->prof_on = enable != 0;
    if (c->prof_on) {
        for (int k = 0; k < glm_ctx::PROF_NAMES; ++k) {
            c->prof_count[k] = 0;
            c->prof_ms[k] = 0.0;
        }
        c->prof_nnames = 0;
    }
    return GLM_OK;
}

int glm_profile_read(glm_ctx* c, int max_entries, char* names, int64_t* launches, double* ms) {
    if (!c || max_entries < 0 || (max_entries > 0 && (!names || !launches || !ms))) return GLM_ERR_INVALID_ARG;
    DeviceGuard g(c->device);
    prof_fold(c);
    const int m = c->prof_nnames < max_entries ? c->prof_nnames : max_entries;
    for (int k = 0; k < m; ++k) {
        std::strncpy(names + 32 * k, c->prof_names[k], 31);
        names[32 * k + 31] = 0;
        launches[k] = c->prof_count[k];
        ms[k] = c->prof_ms[k];
    }
    return m;
}

int64_t glm_launch_count(const glm_ctx* c) { return c ? c->launches : 0; }

int glm_set_problem(glm_ctx* c, int32_t n, int64_t n_bins, double dt, double tau, const int64_t* offs,
                    const int32_t* bins, glm_prec_t prec) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (n < 1 || n_bins < 1 || n_bins >= (int64_t)1 << 31 || !offs)
        return fail(c, GLM_ERR_INVALID_ARG, "need n >= 1, 1 <= n_bins < 2^31 and offs");
    if (!(std::isfinite(dt) && dt > 0) || !(std::isfinite(tau) && tau > 0))
        return fail(c, GLM_ERR_INVALID_ARG, "dt and tau must be finite and > 0");
    if (prec != GLM_PREC_F32 && prec != GLM_PREC_BF16 && prec != GLM_PREC_F16)
        return fail(c, GLM_ERR_INVALID_ARG, "unknown precision");
    const bool tensor = prec != GLM_PREC_F32;
    if (tensor && !(c->cc_major == 10 && c->cc_minor == 3))
        return fail(c, GLM_ERR_UNSUPPORTED_ARCH, "BF16/F16 tensor-core paths need an sm_103 GPU (found sm_" +
                                                     std::to_string(c->cc_major) + std::to_string(c->cc_minor) + ")");
    int rc = validate_offs(c, n, offs, bins);
    if (rc) return rc;
    DeviceGuard g(c->device);
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    {
        // a recording of the same shape (neurons, bins, spike count, precision, chunking, delay) reuses
        // the context's buffers: only the spikes and the caches are renewed
        const Problem& O = c->pb;
        const int64_t chunk = (tensor && c->chunk_req > 0 && round_up(c->chunk_req, 16 * SEG) < round_up(n_bins, SEG))
                                  ? round_up(c->chunk_req, 16 * SEG) : 0;
        if (c->has_problem && !O.ct && O.n == n && O.T == n_bins && O.q == offs[n] && O.prec == prec &&
            O.chunk == chunk && O.delay_bins == c->delay_req && c->delay_req <= 1 &&
            O.xlo == (tensor && c->xsplit_req)) {
            if ((rc = stage_spikes(c, n, n_bins, offs, bins))) return rc;
            c->has_problem = false;
            Problem& P = c->pb;
            P.dt = dt;
            P.tau = tau;
            P.span = (double)n_bins * dt;
            P.dt_int = dt;
            Buffers& B = c->buf;
            std::vector<double> qd(n);
            for (int32_t i = 0; i < n; ++i) qd[i] = (double)(offs[i + 1] - offs[i]);
            GLM_CK(cudaMemcpyAsync(B.qd, qd.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
            GLM_CK(cudaMemsetAsync(B.flags, 0, 4 * sizeof(int), c->stream));
            if ((rc = do_prepare(c))) {
                free_all(c);
                return rc;
            }
            GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
            c->has_problem = true;
            return GLM_OK;
        }
    }
    if ((rc = validate_spikes(c, n, n_bins, offs, bins))) return rc;
    free_all(c);
    Problem& P = c->pb;
    P = Problem();
    P.n = n;
    P.T = n_bins;
    P.dt = dt;
    P.tau = tau;
    P.q = offs[n];
    // a self-delay shorter than the source delay reads X_i that many bins ahead: the buffers extend past T
    P.self_shift = (c->self_req > 0 && c->self_req < c->delay_req) ? c->delay_req - c->self_req : 0;
    if (P.self_shift > 0 && (!tensor || (c->chunk_req > 0 && round_up(c->chunk_req, 16 * SEG) < round_up(n_bins, SEG))))
        return fail(c, GLM_ERR_UNSUPPORTED, "a self-delay needs a tensor-core precision with X stored (no chunks)");
    P.nseg = (n_bins + P.self_shift + SEG - 1) / SEG;
    P.Tpad = P.nseg * SEG;
    P.prec = prec;
    P.xlo = tensor && c->xsplit_req;
    P.chunk = 0;
    // chunks start on the filter's 4096-bin units, so X does not depend on the chunking
    if (tensor && c->chunk_req > 0 && round_up(c->chunk_req, 16 * SEG) < P.Tpad) P.chunk = round_up(c->chunk_req, 16 * SEG);
    P.Tc = P.chunk ? P.chunk : P.Tpad;
    P.span = (double)n_bins * dt;
    P.dt_int = dt;
    // delayed sources: each spike at bin s reaches the rows at s + delay, i.e. the filter reads it at
    // s + delay - 1 (its recursion adds S[t - 1] at t); spikes pushed past the recording drop out (past the
    // buffers, with a self-delay: those bins past T only serve X_i ahead of T - 1, i.e. the self term)
    P.delay_bins = c->delay_req;
    std::vector<int64_t> aoffs;
    std::vector<int32_t> abins;
    if (P.delay_bins > 1) {
        aoffs.assign(n + 1, 0);
        abins.reserve(P.q);
        const int64_t lim = P.self_shift > 0 ? P.Tpad : n_bins;
        for (int32_t i = 0; i < n; ++i) {
            for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
                const int64_t s2 = (int64_t)bins[k] + P.delay_bins - 1;
                if (s2 < lim) abins.push_back((int32_t)s2);
            }
            aoffs[i + 1] = (int64_t)abins.size();
        }
        P.qa = aoffs[n];
    }
    if ((rc = alloc_problem(c))) return rc;
    Buffers& B = c->buf;
    if (P.delay_bins > 1) {
        GLM_CK(cudaMemcpyAsync(B.aoffs, aoffs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream));
        if (P.qa > 0)
            GLM_CK(cudaMemcpyAsync(B.abins, abins.data(), sizeof(int32_t) * P.qa, cudaMemcpyHostToDevice, c->stream));
    }
    std::vector<double> qd(n);
    for (int32_t i = 0; i < n; ++i) qd[i] = (double)(offs[i + 1] - offs[i]);
    GLM_CK(cudaMemcpyAsync(B.offs, offs, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    if (P.q > 0)
        GLM_CK(cudaMemcpyAsync(B.bins, bins, sizeof(int32_t) * P.q, cudaMemcpyHostToDevice, c->stream));
    GLM_CK(cudaMemcpyAsync(B.qd, qd.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    GLM_CK(cudaMemsetAsync(B.flags, 0, 4 * sizeof(int), c->stream));
    rc = do_prepare(c);
    if (rc) {
        free_all(c);
        return rc;
    }
    // the host staging buffers (qd, powers) go out of scope: finish the copies first
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    c->has_problem = true;
    return GLM_OK;
}

int glm_set_problem_ct(glm_ctx* c, int32_t n, double t_begin, double t_end, double tau, double delay,
                       const int64_t* offs, const double* times, glm_prec_t prec) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (n < 1 || !offs) return fail(c, GLM_ERR_INVALID_ARG, "need n >= 1 and offs");
    if (!(std::isfinite(t_begin) && std::isfinite(t_end) && t_end > t_begin))
        return fail(c, GLM_ERR_INVALID_ARG, "need finite t_begin < t_end");
    if (!(std::isfinite(tau) && tau > 0) || !(std::isfinite(delay) && delay >= 0))
        return fail(c, GLM_ERR_INVALID_ARG, "tau must be finite and > 0, delay finite and >= 0");
    if (prec != GLM_PREC_BF16 && prec != GLM_PREC_F16)
        return fail(c, GLM_ERR_UNSUPPORTED, "the continuous-time form runs on the tensor-core precisions (bf16, f16)");
    if (c->self_req > 0)
        return fail(c, GLM_ERR_UNSUPPORTED, "the continuous-time form has one delay for every pair (no self-delay)");
    if (!(c->cc_major == 10 && c->cc_minor == 3))
        return fail(c, GLM_ERR_UNSUPPORTED_ARCH, "BF16/F16 tensor-core paths need an sm_103 GPU (found sm_" +
                                                     std::to_string(c->cc_major) + std::to_string(c->cc_minor) + ")");
    if (offs[0] != 0) return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE, "offs[0] must be 0");
    for (int32_t i = 0; i < n; ++i)
        if (offs[i + 1] < offs[i]) return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE, "offs must be non-decreasing");
    const int64_t q = offs[n];
    if (q > 0 && !times) return fail(c, GLM_ERR_INVALID_ARG, "times is NULL but offs[n] > 0");
    if (q >= ((int64_t)1 << 30)) return fail(c, GLM_ERR_INVALID_ARG, "at most 2^30 - 1 spikes");
    // row j's arrivals are its spikes with t + delay < t_end: a prefix of the row
    std::vector<int64_t> aoffs(n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        double prev = -INFINITY;
        int64_t na = 0;
        for (int64_t k = offs[i]; k < offs[i + 1]; ++k) {
            const double t = times[k];
            if (!(t >= t_begin && t < t_end))
                return fail(c, GLM_ERR_SPIKE_OUT_OF_RANGE, "spike time of row " + std::to_string(i) +
                                                               " outside [t_begin, t_end) or not finite");
            if (!(t > prev))
                return fail(c, GLM_ERR_UNSORTED_SPIKES,
                            "row " + std::to_string(i) + ": times not strictly increasing at index " + std::to_string(k));
            prev = t;
            if (t + delay < t_end) ++na;
        }
        aoffs[i + 1] = aoffs[i] + na;
    }
    const int64_t qa = aoffs[n];
    DeviceGuard g(c->device);
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    free_all(c);
    Problem& P = c->pb;
    P = Problem();
    P.n = n;
    P.tau = tau;
    P.q = q;
    P.qa = qa;
    P.prec = prec;
    P.xlo = true;  // the continuous-time columns are always held as V_hi + V_lo
    P.ct = true;
    P.t_begin = t_begin;
    P.t_end = t_end;
    P.delay = delay;
    P.span = t_end - t_begin;
    P.dt_int = 1.0;
    P.dt = P.span;  // not used by the continuous-time path
    // columns: the distinct event times (device sort), then the buffers sized by them
    int64_t* d_offs = nullptr;
    double* d_times = nullptr;
    void* items = nullptr;
    int32_t *excl = nullptr, *flag = nullptr;
    auto cleanup = [&](int rc) {
        cudaFree(d_offs);
        cudaFree(d_times);
        cudaFree(items);
        cudaFree(excl);
        cudaFree(flag);
        if (rc) free_all(c);
        return rc;
    };
    if (cudaMalloc(&d_offs, sizeof(int64_t) * (n + 1)) != cudaSuccess ||
        cudaMalloc(&d_times, sizeof(double) * (q > 0 ? q : 1)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(fail(c, GLM_ERR_OOM, "continuous-time set-up buffers"));
    }
    if (cudaMemcpyAsync(d_offs, offs, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        (q > 0 && cudaMemcpyAsync(d_times, times, sizeof(double) * q, cudaMemcpyHostToDevice, c->stream) != cudaSuccess))
        return cleanup(fail(c, GLM_ERR_CUDA, "copy of the spike times"));
    int64_t M = 0;
    int rc = ct_build_columns(c, n, q, qa, t_begin, t_end, delay, d_offs, d_times, &M, &items, &excl, &flag);
    if (rc) return cleanup(rc);
    if (M >= ((int64_t)1 << 31) - SEG) return cleanup(fail(c, GLM_ERR_INVALID_ARG, "too many event columns"));
    P.T = M;
    P.nseg = (M + SEG - 1) / SEG;
    P.Tpad = P.nseg * SEG;
    // columns recomputed chunk by chunk (glm_set_chunk_bins counts columns here), on the filter's 4096-column
    // units as on the grid
    P.chunk = (c->chunk_req > 0 && round_up(c->chunk_req, 16 * SEG) < P.Tpad) ? round_up(c->chunk_req, 16 * SEG) : 0;
    P.Tc = P.chunk ? P.chunk : P.Tpad;
    if ((rc = alloc_problem(c))) return cleanup(rc);
    Buffers& B = c->buf;
    std::vector<double> qd(n);
    for (int32_t i = 0; i < n; ++i) qd[i] = (double)(offs[i + 1] - offs[i]);
    if (cudaMemcpyAsync(B.offs, offs, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(B.aoffs, aoffs.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(B.qd, qd.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemsetAsync(B.flags, 0, 4 * sizeof(int), c->stream) != cudaSuccess ||
        ct_finish_columns(c, items, excl, flag, q + qa) != cudaSuccess)
        return cleanup(fail(c, GLM_ERR_CUDA, "continuous-time columns"));
    if ((rc = do_prepare(c))) return cleanup(rc);
    if ((c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize()) != cudaSuccess)
        return cleanup(fail(c, GLM_ERR_CUDA, "synchronise"));
    c->has_problem = true;
    return cleanup(GLM_OK);
}

int glm_problem_columns(const glm_ctx* c, int64_t* n_columns) {
    if (!c || !n_columns) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return GLM_ERR_NO_PROBLEM;
    *n_columns = c->pb.T;
    return GLM_OK;
}

int glm_prepare(glm_ctx* c, double tau) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (tau > 0) {
        if (!std::isfinite(tau)) return fail(c, GLM_ERR_INVALID_ARG, "tau must be finite");
        c->pb.tau = tau;
    }
    DeviceGuard g(c->device);
    return do_prepare(c);
}

int glm_filter(glm_ctx* c, int64_t t0, int64_t t_len, void* X_dev, int64_t ldx, glm_dtype_t dtype) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (c->pb.ct) return fail(c, GLM_ERR_UNSUPPORTED, "glm_filter serves the grid form");
    if (!X_dev || t0 < 0 || t_len < 1 || t0 + t_len > c->pb.T || ldx < t_len)
        return fail(c, GLM_ERR_INVALID_ARG, "bad range, buffer or leading dimension");
    if (dtype != GLM_DTYPE_F32 && dtype != GLM_DTYPE_BF16 && dtype != GLM_DTYPE_F16)
        return fail(c, GLM_ERR_INVALID_ARG, "unknown dtype");
    DeviceGuard g(c->device);
    GLM_RUN("filter_range", 1, launch_filter_range(c, t0, t_len, X_dev, ldx, dtype));
    return GLM_OK;
}

int glm_spike_term(glm_ctx* c, double* C_dev, double* q_dev) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    DeviceGuard g(c->device);
    const size_t nn = (size_t)c->pb.n * c->pb.n;
    if (C_dev) {
        const int rc = ensure_spike_term(c);
        if (rc) return rc;
        GLM_CK(cudaMemcpyAsync(C_dev, c->buf.C, nn * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    }
    if (q_dev)
        GLM_CK(cudaMemcpyAsync(q_dev, c->buf.qd, c->pb.n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
    return GLM_OK;
}

int glm_loglik_grad(glm_ctx* c, const float* W, const float* b, double* L_rows, double* L_total_host,
                    double* G, double* gb, double* gtau_host) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (!W || !b) return fail(c, GLM_ERR_INVALID_ARG, "W and b are required");
    if (gtau_host && c->pb.prec == GLM_PREC_F32)
        return fail(c, GLM_ERR_UNSUPPORTED, "dL/dtau is computed by the tensor-core precisions only");
    if (gtau_host && c->pb.self_shift > 0)
        return fail(c, GLM_ERR_UNSUPPORTED, "dL/dtau is not computed with a self-delay");
    DeviceGuard g(c->device);
    double* Lr = L_rows ? L_rows : c->buf.Lrows;
    if (gtau_host) {
        int rc = prepare_dtau(c);
        if (rc) return rc;
    }
    GLM_CK(cudaMemsetAsync(c->buf.flags, 0, 2 * sizeof(int), c->stream));
    int rc = glm::eval_enqueue(c, W, b, Lr, G, gb, G != nullptr, false, gtau_host != nullptr);
    if (rc) return rc;
    if (gtau_host) {
        GLM_RUN("tau_rows", 1, launch_tau_rows(c, c->buf.tau_rows));
        GLM_RUN("total", 1, launch_total(c, c->buf.tau_rows, c->buf.scal + 1));
        double t = 0.0;
        GLM_CK(cudaMemcpyAsync(&t, c->buf.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
        const Problem& P = c->pb;
        *gtau_host = P.ct ? t : P.a * P.dt / (P.tau * P.tau) * t;  // grid: da/dtau = a dt / tau^2
    }
    if (L_total_host) {
        double* dtot = c->buf.scal;
        GLM_RUN("total", 1, launch_total(c, Lr, dtot));
        double tot = 0;
        GLM_CK(cudaMemcpyAsync(&tot, dtot, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        int fl[2] = {0, 0};
        GLM_CK(cudaMemcpyAsync(fl, c->buf.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
        *L_total_host = tot;
        if (fl[1]) return fail(c, GLM_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
        if (fl[0] & 1) return fail(c, GLM_ERR_NONFINITE, "exp(U) overflowed or an input was not finite");
    }
    return GLM_OK;
}

void glm_fit_default_opts(glm_fit_opts_t* o) {
    if (!o) return;
    o->method = GLM_FIT_LBFGS;
    o->m = 10;
    o->max_iter = 500;
    o->eta = 1e-10;
    o->c1 = 1e-4;
    o->max_halvings = 40;
    o->warm_start = 0;
    o->gain_floor = -1.0;
    o->alpha = 0.0;
    o->eps = 1e-6;
}

int glm_fit(glm_ctx* c, const glm_fit_opts_t* opts, float* W, float* b, int8_t* row_status, glm_fit_report_t* rep) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (!W || !b) return fail(c, GLM_ERR_INVALID_ARG, "W and b are required");
    glm_fit_opts_t o;
    glm_fit_default_opts(&o);
    if (opts) o = *opts;
    if ((o.method != GLM_FIT_LBFGS && o.method != GLM_FIT_GA) || o.m < 1 || o.m > 32 || o.max_iter < 0 ||
        !(o.eta >= 0) || !(o.c1 > 0 && o.c1 < 1) || o.max_halvings < 1 ||
        std::isnan(o.gain_floor) || !(o.alpha >= 0) || !(o.eps > 0))
        return fail(c, GLM_ERR_INVALID_ARG, "bad fit options");
    DeviceGuard g(c->device);
    // the fit's gradient is that of the L it evaluates: over X_hi + X_lo in the split 16-bit forms (E X_hi^T alone
    // misses ~2^-9 of the integral term's derivative, enough to stall line searches near the optimum)
    struct Precise {
        glm_ctx* c;
        ~Precise() { c->precise_grad = false; }
    } pg{c};
    c->precise_grad = c->pb.xlo;
    return glm::fit_run(c, &o, W, b, row_status, rep);
}

int glm_cross_validate(glm_ctx* tr, glm_ctx* va, const glm_fit_opts_t* opts, const double* alphas, int32_t n_alpha,
                       const double* taus, int32_t n_tau, double* L_valid, int32_t* best, float* W_best,
                       float* b_best) {
    if (!tr || !va || !alphas || n_alpha < 1 || n_tau < 1 || (!taus && n_tau != 1)) return GLM_ERR_INVALID_ARG;
    if (!tr->has_problem || !va->has_problem) return fail(tr, GLM_ERR_NO_PROBLEM, "no problem set");
    if (tr->pb.n != va->pb.n || tr->pb.prec != va->pb.prec || tr->device != va->device)
        return fail(tr, GLM_ERR_INVALID_ARG, "training and validation problems differ in n, precision or device");
    for (int32_t k = 0; k < n_alpha; ++k)
        if (!(alphas[k] >= 0)) return fail(tr, GLM_ERR_INVALID_ARG, "alpha must be >= 0");
    for (int32_t k = 0; taus && k < n_tau; ++k)
        if (!(taus[k] > 0) || !std::isfinite(taus[k])) return fail(tr, GLM_ERR_INVALID_ARG, "tau must be > 0");
    glm_fit_opts_t o;
    glm_fit_default_opts(&o);
    if (opts) o = *opts;
    DeviceGuard g(tr->device);
    const int32_t n = tr->pb.n;
    float *W = nullptr, *b = nullptr, *Wv = nullptr, *bv = nullptr;
    double* Lr = nullptr;
    auto cleanup = [&](int rc) {
        cudaFree(W);
        cudaFree(b);
        cudaFree(Lr);
        return rc;
    };
    if (cudaMalloc(&W, sizeof(float) * (size_t)n * n) != cudaSuccess || cudaMalloc(&b, sizeof(float) * n) != cudaSuccess ||
        cudaMalloc(&Lr, sizeof(double) * n) != cudaSuccess)
        return cleanup(fail(tr, GLM_ERR_OOM, "cross-validation work buffers"));
    Wv = W;
    bv = b;
    double best_L = -INFINITY;
    int32_t bt = -1, ba = -1;
    for (int32_t kt = 0; kt < n_tau; ++kt) {
        if (taus) {
            int rc;
            if ((rc = glm_prepare(tr, taus[kt])) || (rc = glm_prepare(va, taus[kt]))) return cleanup(rc);
        }
        for (int32_t ka = 0; ka < n_alpha; ++ka) {
            o.alpha = alphas[ka];
            o.warm_start = ka > 0 ? 1 : 0;  // each alpha starts from the previous fit at this tau
            const int rf = glm_fit(tr, &o, Wv, bv, nullptr, nullptr);
            if (rf < 0) return cleanup(rf);
            double Lt = 0.0;
            const int re = glm_loglik_grad(va, Wv, bv, Lr, &Lt, nullptr, nullptr, nullptr);
            if (re < 0) return cleanup(re);
            if (L_valid) L_valid[(int64_t)kt * n_alpha + ka] = Lt;
            if (Lt > best_L || bt < 0) {
                best_L = Lt;
                bt = kt;
                ba = ka;
                if (W_best && cudaMemcpyAsync(W_best, Wv, sizeof(float) * (size_t)n * n, cudaMemcpyDeviceToDevice,
                                              tr->stream) != cudaSuccess)
                    return cleanup(fail(tr, GLM_ERR_CUDA, "copy of the best W"));
                if (b_best && cudaMemcpyAsync(b_best, bv, sizeof(float) * n, cudaMemcpyDeviceToDevice, tr->stream) !=
                                  cudaSuccess)
                    return cleanup(fail(tr, GLM_ERR_CUDA, "copy of the best b"));
            }
        }
    }
    if (best) {
        best[0] = bt;
        best[1] = ba;
    }
    if (cudaStreamSynchronize(tr->stream) != cudaSuccess) return cleanup(fail(tr, GLM_ERR_CUDA, "synchronise"));
    return cleanup(GLM_OK);
}

int glm_set_self_delay(glm_ctx* c, int32_t self_bins) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (self_bins < 0) return fail(c, GLM_ERR_INVALID_ARG, "self_bins must be >= 0");
    c->self_req = self_bins;
    return GLM_OK;
}

int glm_set_source_delay(glm_ctx* c, int32_t delay_bins) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (delay_bins < 1) return fail(c, GLM_ERR_INVALID_ARG, "delay_bins must be >= 1");
    c->delay_req = delay_bins;
    return GLM_OK;
}

int glm_set_row_range(glm_ctx* c, int32_t r0, int32_t r1) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    const int32_t n = c->pb.n;
    if (r0 == 0 && (r1 == 0 || r1 == n)) {
        c->row_r0 = 0;
        c->row_r1 = -1;
    } else {
        if (r0 < 0 || r1 <= r0 || r1 > n) return fail(c, GLM_ERR_INVALID_ARG, "need 0 <= r0 < r1 <= n");
        c->row_r0 = r0;
        c->row_r1 = r1;
    }
    c->buf.range_rows = nullptr;  // rebuilt on first use (the old list stays in the workspace until the next problem)
    return GLM_OK;
}

int glm_fit_classes(glm_ctx* const* cs, int32_t n_class, const glm_fit_opts_t* opts, float* W, float* b,
                    int8_t* row_status, glm_fit_report_t* rep) {
    if (!cs || n_class < 1 || !W || !b) return GLM_ERR_INVALID_ARG;
    glm_ctx* c0 = cs[0];
    if (!c0 || !c0->has_problem) return c0 ? fail(c0, GLM_ERR_NO_PROBLEM, "no problem set") : GLM_ERR_INVALID_ARG;
    const int32_t n = c0->pb.n;
    std::vector<int> owner(n, -1);
    for (int32_t k = 0; k < n_class; ++k) {
        glm_ctx* c = cs[k];
        if (!c || !c->has_problem) return fail(c0, GLM_ERR_NO_PROBLEM, "a class context has no problem set");
        if (c->pb.n != n || c->device != c0->device)
            return fail(c0, GLM_ERR_INVALID_ARG, "class contexts differ in n or device");
        const int32_t r0 = c->row_r0, r1 = c->row_r1 < 0 ? n : c->row_r1;
        for (int32_t i = r0; i < r1; ++i) {
            if (owner[i] >= 0) return fail(c0, GLM_ERR_INVALID_ARG, "the row ranges of the classes overlap");
            owner[i] = k;
        }
    }
    std::vector<int8_t> st((size_t)n * n_class, (int8_t)GLM_ROW_EXCLUDED);
    glm_fit_report_t tot;
    std::memset(&tot, 0, sizeof(tot));
    int worst = GLM_OK;
    for (int32_t k = 0; k < n_class; ++k) {
        glm_fit_report_t r;
        const int rc = glm_fit(cs[k], opts, W, b, st.data() + (size_t)k * n, &r);
        if (rc < 0) return rc;
        if (rc > worst) worst = rc;
        tot.iterations = std::max(tot.iterations, r.iterations);
        tot.evaluations += r.evaluations;
        tot.gradients += r.gradients;
        tot.converged += r.converged;
        tot.maxiter += r.maxiter;
        tot.stalled += r.stalled;
        tot.degenerate += r.degenerate;
        tot.at_floor += r.at_floor;
        tot.L += r.L;
        tot.seconds += r.seconds;
        // each class's fit runs on its context's stream; W and b are shared between them
        DeviceGuard g(cs[k]->device);
        if (cudaStreamSynchronize(cs[k]->stream) != cudaSuccess) return fail(cs[k], GLM_ERR_CUDA, "synchronise");
    }
    for (int32_t i = 0; i < n; ++i) {
        const int k = owner[i];
        if (k < 0) tot.excluded++;
        if (row_status) row_status[i] = k < 0 ? (int8_t)GLM_ROW_EXCLUDED : st[(size_t)k * n + i];
    }
    if (rep) *rep = tot;
    return worst;
}

int glm_check_wait_limit(glm_ctx* c, double limit_seconds) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!(limit_seconds >= 1e-4 && limit_seconds <= 2.0))
        return fail(c, GLM_ERR_INVALID_ARG, "limit_seconds must lie in [1e-4, 2]");
    DeviceGuard g(c->device);
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, GLM_ERR_OOM, "wait check flag");
    }
    int h = 0;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = launch_wait_check(c, (uint64_t)(limit_seconds * 1e9), d);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize();
    cudaFree(d);
    c->launches += 1;
    if (e != cudaSuccess) return cuda_fail(c, e, "wait check");
    if (h == 2) return fail(c, GLM_ERR_TIMEOUT, "the bounded wait gave up, as it should");
    return fail(c, GLM_ERR_CUDA, "the wait on an mbarrier nobody arrives on did not time out");
}

int glm_poison_caches(glm_ctx* c) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    DeviceGuard g(c->device);
    Buffers& B = c->buf;
    // everything glm_prepare and glm_loglik_grad recompute; not the spikes, the continuous-time column
    // times and durations (set-up data) or the optimiser state
    void* derived[] = {B.seg_carry, B.seg_first, B.pow_seg, B.C, B.C_part, B.X, B.Xlo, B.Gacc, B.E, B.part_e,
                       B.part_s, B.part_g, B.Wsplit, B.Lrows, B.scal, B.eb, B.part_tau, B.tau_rows,
                       B.col_a, B.colc, B.seg_mul, B.part_self, B.gself};
    for (void* p : derived) {
        if (!p) continue;
        for (int k = 0; k < c->n_allocs; ++k)
            if (c->allocs[k] == p) GLM_CK(cudaMemsetAsync(p, 0xFF, c->alloc_bytes[k], c->stream));
    }
    if (B.aseg_first != B.seg_first)
        for (int k = 0; k < c->n_allocs; ++k)
            if (c->allocs[k] == B.aseg_first) GLM_CK(cudaMemsetAsync(B.aseg_first, 0xFF, c->alloc_bytes[k], c->stream));
    c->c_ready = false;
    c->raster_in_E = false;
    GLM_CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
    return GLM_OK;
}

int glm_set_chunk_bins(glm_ctx* c, int64_t chunk_bins) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (chunk_bins < 0) return fail(c, GLM_ERR_INVALID_ARG, "chunk_bins must be >= 0");
    c->chunk_req = chunk_bins;
    return GLM_OK;
}

int glm_set_x_split(glm_ctx* c, int32_t split) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (split != 0 && split != 1) return fail(c, GLM_ERR_INVALID_ARG, "split must be 0 or 1");
    c->xsplit_req = split == 1;
    return GLM_OK;
}

int glm_autotune(glm_ctx* c, glm_tune_report_t* rep) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (c->pb.prec == GLM_PREC_F32) return fail(c, GLM_ERR_UNSUPPORTED, "the autotuner covers the tensor-core products");
    if (rep) std::memset(rep, 0, sizeof(*rep));
    DeviceGuard g(c->device);
    const int rc = glm::tc_autotune(c, rep);
    return rc ? fail(c, rc, "autotune failed") : GLM_OK;
}

int glm_set_grad_tile(glm_ctx* c, int32_t mode, int32_t units_per_sm, int32_t* nsplit_out) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!c->has_problem) return fail(c, GLM_ERR_NO_PROBLEM, "no problem set");
    if (c->pb.prec == GLM_PREC_F32) return fail(c, GLM_ERR_UNSUPPORTED, "the tile shape is the tensor-core product's");
    if ((mode != 1 && mode != 2) || (units_per_sm != 1 && units_per_sm != 2 && units_per_sm != 4 && units_per_sm != 8))
        return fail(c, GLM_ERR_INVALID_ARG, "mode must be 1 or 2, units_per_sm 1, 2, 4 or 8");
    c->g_mode = mode;
    c->g_nsplit = glm::tc_nsplit_for(c, mode, units_per_sm);
    if (nsplit_out) *nsplit_out = c->g_nsplit;
    return GLM_OK;
}

int glm_fit_batch(glm_ctx* const* cs, int32_t np, const glm_fit_opts_t* opts, float* const* W, float* const* b,
                  int8_t* const* row_status, glm_fit_report_t* reps) {
    if (!cs || np < 1 || np > GLM_FIT_BATCH_MAX || !W || !b) return GLM_ERR_INVALID_ARG;
    glm_ctx* c0 = cs[0];
    if (!c0) return GLM_ERR_INVALID_ARG;
    for (int32_t p = 0; p < np; ++p) {
        glm_ctx* c = cs[p];
        if (!c || !W[p] || !b[p]) return fail(c0, GLM_ERR_INVALID_ARG, "null context or output");
        if (!c->has_problem) return fail(c0, GLM_ERR_NO_PROBLEM, "a context has no problem set");
        if (c->device != c0->device) return fail(c0, GLM_ERR_INVALID_ARG, "contexts on different devices");
        if (c->pb.prec != c0->pb.prec) return fail(c0, GLM_ERR_INVALID_ARG, "contexts with different precisions");
        if (c->pb.xlo != c0->pb.xlo) return fail(c0, GLM_ERR_INVALID_ARG, "contexts with different X splits");
        if (c->pb.chunk) return fail(c0, GLM_ERR_UNSUPPORTED, "glm_fit_batch needs X stored (no chunking)");
        if (c->pb.ct) return fail(c0, GLM_ERR_UNSUPPORTED, "glm_fit_batch serves the grid form");
        if (c->row_r1 >= 0) return fail(c0, GLM_ERR_UNSUPPORTED, "glm_fit_batch fits whole problems (no row range)");
        if (c->pb.self_shift > 0) return fail(c0, GLM_ERR_UNSUPPORTED, "glm_fit_batch has no self-delay");
        for (int32_t q = 0; q < p; ++q)
            if (cs[q] == c) return fail(c0, GLM_ERR_INVALID_ARG, "a context appears twice");
    }
    if (c0->pb.prec == GLM_PREC_F32)
        return fail(c0, GLM_ERR_UNSUPPORTED, "glm_fit_batch needs a tensor-core precision (fit FP32 problems one by one)");
    glm_fit_opts_t o;
    glm_fit_default_opts(&o);
    if (opts) o = *opts;
    if ((o.method != GLM_FIT_LBFGS && o.method != GLM_FIT_GA) || o.m < 1 || o.m > 32 || o.max_iter < 0 ||
        !(o.eta >= 0) || !(o.c1 > 0 && o.c1 < 1) || o.max_halvings < 1 || std::isnan(o.gain_floor) ||
        !(o.alpha >= 0) || !(o.eps > 0))
        return fail(c0, GLM_ERR_INVALID_ARG, "bad fit options");
    DeviceGuard g(c0->device);
    struct Precise {  // as glm_fit: the gradient over X_hi + X_lo
        glm_ctx* const* cs;
        int32_t np;
        ~Precise() {
            for (int32_t p = 0; p < np; ++p) cs[p]->precise_grad = false;
        }
    } pg{cs, np};
    for (int32_t p = 0; p < np; ++p) cs[p]->precise_grad = cs[p]->pb.xlo;
    return glm::fit_run_batch(cs, np, &o, W, b, row_status, reps);
}

}  // extern "C"
