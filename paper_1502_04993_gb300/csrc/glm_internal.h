// Internal declarations of libglm (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "glm.h"

namespace glm {

// ---------------------------------------------------------------------------------------------
// Time-grid layout.  Bins are processed in segments of SEG = 256 (one warp, 8 bins per lane).
// Per row j and segment s the carry X_j[256 s] (FP64) and the index of the first spike of row j
// at or after bin 256 s are precomputed once per problem.
// ---------------------------------------------------------------------------------------------
constexpr int SEG = 256;
// e^U is formed as e^c e^(U - c) with c = max(b_i, EXP_SPLIT_FLOOR): c = b_i keeps the quiet bins (U ~ b_i)
// free of FP32 rounding; the floor keeps U - c inside the FP32 range of exp when a fit drives b_i far below
// U (there the quiet bins contribute less than e^-60 per second and their rounding does not matter).
constexpr float EXP_SPLIT_FLOOR = -60.f;
// continuous-time U product: epilogue warps per TMEM lane quarter, each with a part of a tile's columns
// and its own plane of per-tile partial sums
constexpr int CT_PARTS = 3;

// Powers of a = exp(-dt/tau) split into FP32 hi + lo parts, so that the FP32 scan multiplies by a
// with ~48 significant bits (the product is hi*x + lo*x).
struct ScanConsts {
    float a_hi, a_lo;
    float pm_hi[9], pm_lo[9];    // a^m,          m = 0..8
    float ps_hi[5], ps_lo[5];    // a^(8*2^d),    d = 0..4   (warp scan strides)
    float pl_hi[32], pl_lo[32];  // a^(8*l),      l = 0..31  (lane offsets)
};

struct Problem {
    int32_t n = 0;
    int64_t T = 0;        // bins
    double dt = 0, tau = 0, a = 0;
    int64_t q = 0;        // total spikes
    int64_t nseg = 0;     // ceil(T / SEG)
    int64_t Tpad = 0;     // nseg * SEG
    glm_prec_t prec = GLM_PREC_F32;
    int64_t chunk = 0;    // 16-bit forms: bins of X recomputed per chunk for each evaluation (0: X stored)
    int64_t Tc = 0;       // bins held in the X / E buffers: chunk, or Tpad
    double span = 0;      // duration of the recording in seconds: T dt, or t_end - t_begin
    double dt_int = 0;    // factor of the per-tile integral sums in L: dt (grid) or 1 (sums already in seconds)
    // continuous-time form: the "bins" are event columns (T of them), spike times in [t_begin, t_end),
    // every spike arriving everywhere after `delay`
    bool ct = false;
    double t_begin = 0, t_end = 0, delay = 0;
    // grid form: every source train reaches the rows after delay_bins bins (1: the one-bin delay of the
    // filter recursion); above 1 the filter reads the spikes shifted by delay_bins - 1
    int32_t delay_bins = 1;
    int64_t qa = 0;       // arrivals inside the recording
    // self-delay (16-bit grid forms, X stored): row i's own train reaches row i after delay_bins - self_shift
    // bins, every other train after delay_bins; X_i with the self-delay is X_i at bin t + self_shift, so the
    // buffers extend at least self_shift bins past T (Tpad >= T + self_shift)
    int32_t self_shift = 0;
    // 16-bit forms: X held as the pair X_hi + X_lo (true), or as X_hi alone (false: one 16-bit X, the U
    // product W_hi X + W_lo X and the spike term S X^T without their X_lo products)
    bool xlo = false;
};

// Device buffers owned by a context.  Row-major everywhere; ld* in elements.
struct Buffers {
    int64_t* offs = nullptr;      // [n+1]
    int32_t* bins = nullptr;      // [q]
    float2* seg_carry = nullptr;  // [n][nseg]   X_j[256 s] as a double-float pair (hi, lo)
    int32_t* seg_first = nullptr; // [n][nseg]   first spike index (relative to offs[j]) at bin >= 256 s
    double* pow_seg = nullptr;    // [SEG + 1]   a^k, k = 0..SEG
    double* qd = nullptr;         // [n]         spike counts
    double* C = nullptr;          // [n][n]      spike term
    double* C_part = nullptr;     // [parts][n][n] (plain FP32 form)
    void* X = nullptr;            // F32: float [n][Tpad]; 16-bit: [n][Tpad]
    void* Xlo = nullptr;          // 16-bit forms with the X split: X_lo = X - X_hi, bin-blocked over Tc bins
    double* Gacc = nullptr;       // chunked: [n][n] E X^T summed over the chunks
    int64_t ldn = 0;              // leading dim of the W parts (n rounded up to 64)
    void* E = nullptr;            // F32: float [n][Tpad] dt exp(U); 16-bit: the same, bin-blocked
    double* part_e = nullptr;     // [n][ntile_t]  per-(row, bin tile) sums of exp(U); continuous time:
                                  // CT_PARTS such planes, one per part of each tile's columns
    double* part_s = nullptr;     // [n][ntile_t] per-(row, bin tile) sums of U - b over the spike bins (idem)
    double* part_self = nullptr;  // self-delay: [n][ntile] per-(row, tile) sums of dt e^U (X_i self - X_i)
    double* gself = nullptr;      // self-delay: [n] their row sums (the diagonal's part of dL/dW_ii)
    float* part_g = nullptr;      // [nsplit][n][n] FP32 partial sums of E X^T
    void* Wsplit = nullptr;       // 16-bit: hi and lo parts of W, [2][n][ldn]
    int* flags = nullptr;         // [4] device error flags
    double* Lrows = nullptr;      // [n] scratch when the caller passes no L_rows
    double* scal = nullptr;       // [8] device scalars (total log-likelihood, ...)
    double* eb = nullptr;         // [n] exp(b_i) in FP64 (plain FP32 form)
    void* fit_mem = nullptr;      // optimiser state of glm_fit (allocated by its first call)
    // derivative in tau (allocated by the first request for it)
    double* part_tau = nullptr;   // [5][n][ntile]
    double* tau_rows = nullptr;   // [n]
    int fit_m = 0;
    // sources of the filter recursion: the spikes (grid: aliases of offs, bins, seg_first) or, in continuous
    // time, the column before each arrival
    int64_t* aoffs = nullptr;     // [n+1]
    int32_t* abins = nullptr;     // [qa]
    int32_t* aseg_first = nullptr;// [n][nseg]
    // continuous-time columns
    double* ctime = nullptr;      // [Tpad + 1] column start times; t_end from column T on
    float* col_a = nullptr;       // [Tpad] exp(-(column length) / tau)
    float* colc = nullptr;        // [Tpad][8] a, 1 - a and the one-panel quadrature factors (ct_link.cuh)
    double* seg_mul = nullptr;    // [nseg] decay over each 256-column segment
    double* tile_span = nullptr;  // [nseg] duration of each 256-column segment
    int32_t* range_rows = nullptr;// [r1 - r0] the rows r0 .. r1 - 1 of a row range (glm_set_row_range)
    // a recording of the same shape is copied here and checked on the device before it replaces offs / bins
    // (allocated by the first such recording)
    int64_t* offs_next = nullptr; // [n+1]
    int32_t* bins_next = nullptr; // [q]
    unsigned long long* bad = nullptr; // [1] first fault found by the check (launch_check_bins)
};

}  // namespace glm

struct glm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t ws_cap = 0;
    size_t ws_used = 0;
    glm::Problem pb;
    glm::Buffers buf;
    glm::ScanConsts sc;
    CUtensorMap tmap[7];  // tensor-core path: W_hi, W_lo, X_hi, X_lo (N-major), E, X_hi, X_lo (K-major)
    bool has_problem = false;
    bool c_ready = false;  // C holds the spike term of the current problem and tau
    bool raster_in_E = false;  // the E buffer holds the spike raster written by the last filter pass
    int g_mode = 1;        // E X^T row tile: 1 = 256 rows, 2 = 128 rows (autotuner)
    int g_nsplit = 0;      // E X^T bin splits (0: the default for g_mode)
    int64_t chunk_req = 0; // bins per chunk requested by glm_set_chunk_bins (applied by glm_set_problem)
    int32_t delay_req = 1; // source delay in bins requested by glm_set_source_delay (applied by glm_set_problem)
    int32_t self_req = 0;  // self-delay in bins requested by glm_set_self_delay (0: as the source delay)
    bool xsplit_req = true;  // X as X_hi + X_lo in the 16-bit grid forms (glm_set_x_split)
    // 16-bit forms: the gradient product over X_hi + X_lo (E X_hi^T + E X_lo^T), the derivative of the very L
    // the evaluation forms; set by the fits for their duration (see glm_fit)
    bool precise_grad = false;
    int32_t row_r0 = 0, row_r1 = -1;  // evaluated and fitted rows (glm_set_row_range); r1 < 0: all rows
    std::string last_error;
    // tracing: event pairs per launched kernel group while profiling is on
    bool prof_on = false;
    struct ProfRec {
        int name;
        cudaEvent_t a, b;
    };
    ProfRec* prof_recs = nullptr;
    int prof_n = 0, prof_cap = 0;
    static constexpr int PROF_NAMES = 16;
    const char* prof_names[PROF_NAMES] = {};
    int64_t prof_count[PROF_NAMES] = {};
    double prof_ms[PROF_NAMES] = {};
    int prof_nnames = 0;
    int64_t launches = 0;
    // bookkeeping for the allocations (pointer, bytes)
    void* allocs[64];
    size_t alloc_bytes[64];
    int n_allocs = 0;
};

namespace glm {

// ---- launchers (each returns cudaError_t of the launch) ----
cudaError_t launch_carry(glm_ctx* c);
// device check of a CSR spike list whose offsets are valid: *first_bad = smallest 2k (bin k outside [0, T)) or
// 2k + 1 (bin k not above the previous bin of its row), all ones when there is none
cudaError_t launch_check_bins(glm_ctx* c, int32_t n, int64_t q, int64_t T, const int64_t* offs, const int32_t* bins,
                              unsigned long long* first_bad);
// segments [s_begin, s_end) into the X buffers (whose first bin is SEG s_begin); s_end < 0: all
// raster: also write the rows' spike raster (16-bit 0 / 1) there; only where the filter's sources are the
// rows' own spikes (grid form, one-bin delay)
cudaError_t launch_filter_cache(glm_ctx* c, int64_t s_begin = 0, int64_t s_end = -1, void* raster = nullptr);
// the 16-bit spike raster of segments [s_begin, s_end) into a bin-blocked buffer starting at bin SEG s_begin
cudaError_t launch_spike_raster(glm_ctx* c, void* out, int64_t s_begin, int64_t s_end);
cudaError_t launch_filter_range(glm_ctx* c, int64_t t0, int64_t t_len, void* out, int64_t ldx, glm_dtype_t dtype);
cudaError_t launch_spike_term(glm_ctx* c, double* out);
cudaError_t launch_tau_rows(glm_ctx* c, double* rows);
cudaError_t launch_sum_splits(glm_ctx* c, int nsplit, double* C, bool accumulate);
cudaError_t launch_tc_spike_term(glm_ctx* c);
// rows: evaluated rows (null: all n), m of them; outputs land at the rows' own positions
cudaError_t launch_simt_u_epilogue(glm_ctx* c, const float* W, const float* b, const int32_t* rows = nullptr,
                                   int32_t m = 0);
cudaError_t launch_simt_grad(glm_ctx* c);
// G = C - (Gacc, when given, else the sum of the E X^T splits)
cudaError_t launch_reduce(glm_ctx* c, const float* W, const float* b, double* L_rows, double* G, double* gb,
                          bool want_grad, int64_t ntile, int nsplit, const double* Gacc = nullptr);
void launch_exp_bias(glm_ctx* c, const float* b);
int set_error(glm_ctx* c, int code, const char* msg);
int ensure_range_rows(glm_ctx* c);
cudaError_t launch_wait_check(glm_ctx* c, uint64_t limit_ns, int* out);
// One evaluation at (W, b).  With rows (m of them) only those rows' U product, rates and per-tile sums
// are formed (their L_rows entries are valid; other rows' entries are not).
int eval_enqueue(glm_ctx* c, const float* W, const float* b, double* L_rows, double* G, double* gb, bool want_grad,
                 bool reuse_u, bool tau = false, const int32_t* rows = nullptr, int32_t m = 0);
int eval_status(glm_ctx* c);
cudaError_t reset_flags(glm_ctx* c);
int ws_alloc_bytes(glm_ctx* c, void** p, size_t bytes);
int fit_run(glm_ctx* c, const glm_fit_opts_t* o, float* W, float* b, int8_t* row_status, glm_fit_report_t* rep);
int fit_run_batch(glm_ctx* const* cs, int np, const glm_fit_opts_t* o, float* const* W, float* const* b,
                  int8_t* const* row_status, glm_fit_report_t* reps);
cudaError_t tc_prepare_maps(glm_ctx* c);
// bins [t_base, t_base + t_len) held in the X / E buffers (t_len < 0: the whole buffer)
cudaError_t launch_tc_u_epilogue(glm_ctx* c, const float* W, const float* b, bool tau, const int32_t* rows = nullptr,
                                 int32_t m = 0, int64_t t_base = 0, int64_t t_len = -1);
cudaError_t launch_tc_grad(glm_ctx* c, int64_t t_len = -1, int* nsplit_used = nullptr);
int tc_nsplit(const glm_ctx* c);
int tc_nsplit_for(const glm_ctx* c, int mode, int units_per_sm);
int tc_nsplit_max(const glm_ctx* c);
int tc_autotune(glm_ctx* c, glm_tune_report_t* rep);
int tc_autotune_batch(glm_ctx* const* cs, int np, void* dev_g, void* host_g);
void tc_batch_set_grad_counts(void* host_g, int np, const int* const* counts);
// several problems per launch (glm_fit_batch)
size_t tc_batch_bytes();
int tc_batch_fill(glm_ctx* const* cs, int np, float* const* W32, float* const* b32, int32_t* const* rows,
                  const int32_t* const* m_dev, void* host_u, void* host_g);
cudaError_t launch_tc_u_batch(glm_ctx* c0, const void* dev_u);
cudaError_t launch_tc_grad_batch(glm_ctx* c0, const void* dev_g);
int tc_tile_t();
cudaError_t launch_total(glm_ctx* c, const double* L_rows, double* out1);
// continuous-time columns (ct.cu)
int ct_build_columns(glm_ctx* c, int32_t n, int64_t q, int64_t qa, double t_begin, double t_end, double delay,
                     const int64_t* offs, const double* times, int64_t* M, void** items, int32_t** excl,
                     int32_t** flag);
cudaError_t ct_finish_columns(glm_ctx* c, const void* items, const int32_t* excl, const int32_t* flag, int64_t m);
cudaError_t launch_ct_consts(glm_ctx* c);

// ---- sizes shared between the launchers and the allocator ----
int simt_tile_t();          // bins per SIMT GEMM1 tile
int grad_nsplit(const glm_ctx* c);
int spike_term_parts(const glm_ctx* c);

void fill_scan_consts(double a, ScanConsts* sc);

}  // namespace glm
