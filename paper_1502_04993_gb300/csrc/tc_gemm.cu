// Tensor-core (tcgen05) form of the two contractions, for X and the rates held in BF16 or FP16.
//
//   MODE 0, steps a3/a4:  U = b 1^T + W X  (Eq. 3) from split operands W = W_hi + W_lo, X = X_hi + X_lo:
//                         U ~ W_hi X_hi + W_lo X_hi + W_hi X_lo (the dropped W_lo X_lo is ~2^-16 of U - b),
//                         with the link and the spike-time term in the epilogue (Eq. 5, Eq. 7): per
//                         (row, 256-bin tile) FP64 sums of exp(U) and of U - b over the row's spike bins,
//                         and E[i][t] = dt exp(U_i[t]) stored 16-bit.
//                         Tile 128 x 256, K step 32, 4 stages of (W_hi, W_lo, X_hi, X_lo).  W is K-major (64-byte
//                         swizzle); X is an N-major operand: one 3-D box of 4 bin blocks x 32 neurons x 64 bins
//                         (128-byte swizzle) per stage.  3 MMAs per 16-wide k slice, 2 TMEM accumulators
//                         (epilogue overlaps the next tile).  Also the continuous-time U product (CT).
//   MODE 3:               the same U product over X held as one 16-bit array: W_hi X + W_lo X, 2 MMAs per
//                         k slice, 6 stages of (W_hi, W_lo, X).
//   MODE 1, step a5:      P_s = E X^T over a split s of the bins (dL/dW = C - sum_s P_s, Eq. 12).  The same
//                         kernel forms the spike term C = S X^T once per problem (S, the spike raster, in
//                         the place of E; X_hi and X_lo in turn, or X alone).  Tile 256 x 256 per block as two 128 x 256
//                         accumulators that share every X tile (A0 = E rows m0.., A1 = E rows m0+128..),
//                         K step 64 (128-byte swizzle), 3 stages, FP32 partials per split.
//   MODE 2:               E X^T with 128-row tiles and double-buffered accumulators (small N; autotuner).
//
// X (X_hi, X_lo) and E are stored bin-blocked, [Tpad / 64][n][64]: a block of 64 bins of every neuron is one
// contiguous n x 128-byte array, so every TMA box of either product is a contiguous stretch of memory.
//
// One persistent block per SM: warp 0 issues TMA loads, warp 1 owns TMEM and issues the MMAs (one thread),
// the other warps are the epilogue (TMEM -> registers -> global): 4 (one per TMEM lane quarter), 8 for the
// plain grid U product, 12 for the continuous-time one (epi_warps).  Every mbarrier wait is bounded; on a
// timeout the block raises flags[1], drains its own copies and MMAs, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>
#include <type_traits>

#include "ct_link.cuh"
#include "glm_internal.h"
#include "tc_ptx.cuh"

namespace glm {

namespace {

// warp 0 TMA, warp 1 MMA, then the epilogue warps: 4 (one per TMEM lane quarter); 4 CT_PARTS for the
// continuous-time U product, whose epilogue does several times the grid's arithmetic per element
// (CT_PARTS warps per lane quarter, each taking a part of the tile's columns); 8 for the plain grid U
// product (two per lane quarter, each taking half of the tile's columns): with one warp per SM sub-partition
// the epilogue's dependent chains are exposed, and over a single X (two products per k slice) it took
// longer per tile than the MMAs (measured: 0.74 of the tensor peak)
template <int MODE>
constexpr bool is_u() { return MODE == 0 || MODE == 3; }
template <int MODE, bool CT, bool TAU = false, bool SELF = false>
constexpr int epi_warps() { return (MODE == 0 && CT) ? 4 * CT_PARTS : (is_u<MODE>() && !TAU && !SELF) ? 8 : 4; }
template <int MODE, bool CT, bool TAU = false, bool SELF = false>
constexpr int kthreads() { return 64 + 32 * epi_warps<MODE, CT, TAU, SELF>(); }
constexpr int SP_REG = 12;  // spike bins per (row, 256-bin tile) held in registers by the epilogue
constexpr int TUNE_UPM_MAX = 8;  // most units per SM the autotuner tries for E X^T
constexpr uint32_t TMEM_COLS = 512;
constexpr int BN = 256;
static_assert(BN == SEG, "a U-product tile is one 256-bin segment of the spike index");

template <int MODE>
struct Cfg;
template <>
struct Cfg<0> {
    static constexpr int BM = 128;            // rows per block
    static constexpr int BK = 32;             // K elements per stage (64 bytes)
    static constexpr int NA = 2, NB = 2;      // W_hi, W_lo ; X_hi, X_lo
    static constexpr int STAGES = 4;
    static constexpr int NBUF = 2;            // TMEM accumulator buffers (double buffering)
    static constexpr uint32_t SWZ = 4;        // A (K-major): 64-byte swizzle
    static constexpr uint32_t SBO = 8 * 64;   // A: bytes between 8-row groups
    static constexpr uint32_t A_KSTEP = 2;    // A: descriptor advance per 16-wide k slice (32 bytes)
    // B is N-major: an atom of the 128-byte swizzle is 8 k-rows x 64 bins
    static constexpr uint32_t B_SWZ = 2;
    static constexpr uint32_t B_SBO = 1024;   // B: bytes between 8-row groups along K
    static constexpr uint32_t B_LBO = BK * 128;  // B: bytes between 64-bin blocks along N (one TMA box)
    static constexpr uint32_t B_KSTEP = 128;  // B: advance per k slice (16 k-rows of 128 bytes)
    static constexpr uint32_t A_BYTES = 128 * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
};
// MODE 3: the U product of MODE 0 over a single 16-bit X (no X_lo): a stage holds W_hi, W_lo and X only, and
// six stages keep as many bytes in flight as MODE 0's four (its MMAs take 2/3 of the time per stage, so four
// 32 KB stages could not cover the load latency from L2)
template <>
struct Cfg<3> {
    static constexpr int BM = 128;
    static constexpr int BK = 32;
    static constexpr int NA = 2, NB = 1;      // W_hi, W_lo ; X
    static constexpr int STAGES = 6;
    static constexpr int NBUF = 2;
    static constexpr uint32_t SWZ = 4;
    static constexpr uint32_t SBO = 8 * 64;
    static constexpr uint32_t A_KSTEP = 2;
    static constexpr uint32_t B_SWZ = 2;
    static constexpr uint32_t B_SBO = 1024;
    static constexpr uint32_t B_LBO = BK * 128;
    static constexpr uint32_t B_KSTEP = 128;
    static constexpr uint32_t A_BYTES = 128 * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
};
template <>
struct Cfg<1> {
    static constexpr int BM = 256;            // two 128-row halves
    static constexpr int BK = 64;
    static constexpr int NA = 2, NB = 1;      // E rows m0.., E rows m0+128.. ; X
    static constexpr int STAGES = 3;
    static constexpr int NBUF = 1;
    static constexpr uint32_t SWZ = 2;        // 128-byte swizzle, both operands K-major
    static constexpr uint32_t SBO = 8 * 128;
    static constexpr uint32_t A_KSTEP = 2;
    static constexpr uint32_t B_SWZ = SWZ;
    static constexpr uint32_t B_SBO = SBO;
    static constexpr uint32_t B_LBO = 16;     // unused for swizzled K-major operands
    static constexpr uint32_t B_KSTEP = 2;
    static constexpr uint32_t A_BYTES = 128 * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
};

template <>
struct Cfg<2> {                               // E X^T with 128-row tiles (small N), double-buffered accumulators
    static constexpr int BM = 128;
    static constexpr int BK = 64;
    static constexpr int NA = 1, NB = 1;      // E rows m0.. ; X
    static constexpr int STAGES = 4;
    static constexpr int NBUF = 2;
    static constexpr uint32_t SWZ = 2;
    static constexpr uint32_t SBO = 8 * 128;
    static constexpr uint32_t A_KSTEP = 2;
    static constexpr uint32_t B_SWZ = SWZ;
    static constexpr uint32_t B_SBO = SBO;
    static constexpr uint32_t B_LBO = 16;
    static constexpr uint32_t B_KSTEP = 2;
    static constexpr uint32_t A_BYTES = 128 * BK * 2;
    static constexpr uint32_t B_BYTES = BN * BK * 2;
};

template <int MODE>
struct Layout {
    using C = Cfg<MODE>;
    static constexpr uint32_t STAGE_BYTES = C::NA * C::A_BYTES + C::NB * C::B_BYTES;
    static constexpr size_t SMEM = (size_t)C::STAGES * STAGE_BYTES + 1024 + 512;
};

struct TcArgs {
    int32_t n;
    int64_t T, Tpad;
    int32_t mt, nt;
    int64_t units;
    int32_t kb_per_unit;  // MODE 0: k-steps over the neurons; MODE 1: k-steps per split
    int64_t kb_total;     // MODE 1: k-steps over the bins
    int64_t nsplit;       // MODE 1: number of interleaved splits
    int64_t kb_half;      // MODE 1, 2: k-steps from kb_half on read the second B operand at kb - kb_half (the
                          // two products S X_hi^T + S X_lo^T in one accumulator); 0: one B operand
    uint32_t idesc;
    double dt;
    const float* b;
    const double* eb;  // exp(b_i) in FP64
    float a;           // exp(-dt / tau), for the tau partials
    double* part_tau;  // TAU: [5][n][ntile] = sum_t e^v a^(t-t0), sum_t e^v Z_loc[t], Z_loc[t0 + 256],
                       //      and over the spike bins sum a^(t-t0), sum Z_loc[t]
    double* part_s;    // MODE 0: [n][ntile] sum of U - b over the row's spike bins in the tile
    const int64_t* offs;      // spikes (CSR) and the index of each row's first spike per 256-bin segment
    const int32_t* bins;
    const int32_t* seg_first;
    int64_t nseg;
    const int32_t* rows;  // MODE 0: evaluated rows (null: all n); tile row l is row rows[l] for l < m_rows
    int32_t m_rows;
    int32_t m_base;       // MODE 1, 2: first row of the row tiles (a row range starts there)
    int64_t t_base;       // MODE 0: first bin of the X / E buffers (a chunk of the recording, or 0)
    void* E;
    double* part_e;
    int64_t ntile;
    float* part_g;
    int* flags;
    uint64_t limit_ns;
    const float* colc;         // CT: [Tpad][8] column constants (ct_link.cuh)
    const double* tile_span;   // CT: [ntile] seconds covered by each 256-column tile
    float ct_tau;
    // SELF (MODE 0 grid): row i's own train with its self-delay is X_i at bin t + self_shift
    int32_t self_shift;
    int32_t xlo;               // MODE 0: X held as X_hi + X_lo (the third product W_hi X_lo); 0: X_hi alone
    const float* W32;          // W (FP32), for W_ii
    const void* Xhi;           // X_hi, X_lo bin-blocked over the recording
    const void* Xlo;
    double* part_self;         // [n][ntile] sums of dt e^U (X_i[t + self_shift] - X_i[t]) per tile
};

struct Unit {
    int32_t m0, n0;
    int64_t kb0, kb1, kstep, split;
};

// Several independent problems in one launch (glm_fit_batch): their units are laid end to end.  MODE 0
// takes each problem's count of evaluated rows from m_dev when given (set on the device by the fit); E X^T
// skips a problem whose m_dev count (its active rows) is 0.
constexpr int MAX_BATCH = 32;
struct TcBatch {
    int32_t nprob;
    const int32_t* m_dev[MAX_BATCH];
    TcArgs args[MAX_BATCH];
    CUtensorMap maps[MAX_BATCH][4];  // A0, A1, B0, B1 of each problem
};

// unit u of a problem with mt row tiles
template <int MODE>
__device__ __forceinline__ Unit decode(const TcArgs& A, int64_t u, int32_t mt) {
    Unit r;
    if (is_u<MODE>()) {
        r.m0 = (int32_t)(u % mt) * Cfg<0>::BM;
        r.n0 = (int32_t)(u / mt) * BN;
        r.kb0 = 0;
        r.kb1 = A.kb_per_unit;
        r.kstep = 1;
        r.split = 0;
    } else {
        const int64_t tiles = (int64_t)A.mt * A.nt;
        const int64_t tile = u % tiles;
        r.split = u / tiles;
        r.m0 = A.m_base + (int32_t)(tile % A.mt) * (MODE == 2 ? 128 : 256);
        r.n0 = (int32_t)(tile / A.mt) * BN;
        // the splits interleave: split s takes k-steps s, s + nsplit, s + 2 nsplit, ...  All blocks then
        // stream the same narrow band of bins, which stays in L2 while the 16 tiles of each split reuse it.
        r.kb0 = r.split;
        r.kb1 = A.kb_total;
        r.kstep = A.nsplit;
    }
    return r;
}

// Shared-memory descriptor of an operand tile written by TMA with the matching swizzle.
//   K-major:  sbo = bytes between 8-row groups along M/N; lbo unused (16).
//   N-major (128-byte swizzle): an atom is 8 k-rows of 64 elements along N; lbo = bytes between atoms
//             along N, sbo = bytes between atoms along K.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t swz, uint32_t sbo, uint32_t lbo = 16) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;  // leading-dimension byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;  // stride-dimension byte offset
    d |= (uint64_t)1u << 46;                      // descriptor version
    d |= (uint64_t)swz << 61;                     // swizzle mode
    return d;
}

template <typename T16>
__device__ __forceinline__ uint32_t pack16(float lo, float hi);
template <>
__device__ __forceinline__ uint32_t pack16<__nv_bfloat16>(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
template <>
__device__ __forceinline__ uint32_t pack16<__half>(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(__half v) { return __half2float(v); }

// w as the U product holds it: hi + lo parts, rounded as split_w_kernel rounds them (exact sum in FP32)
template <typename T16>
__device__ __forceinline__ float split_sum16(float w);
template <>
__device__ __forceinline__ float split_sum16<__nv_bfloat16>(float w) {
    const float h = __bfloat162float(__float2bfloat16_rn(w));
    return h + __bfloat162float(__float2bfloat16_rn(w - h));
}
template <>
__device__ __forceinline__ float split_sum16<__half>(float w) {
    const float h = __half2float(__float2half_rn(w));
    return h + __half2float(__float2half_rn(w - h));
}

// CT (MODE 0 only): continuous-time columns.  The epilogue takes, per column m of length D_m, the exact
// interval integral e^{b} F(u, D_m) of the rate and the interval weight E'_m = e^{b} G(u, D_m) of Eq. 14
// (ct_link.cuh) in place of dt e^U; the per-tile sums hold e^{b} (duration + sum (F - D)) in seconds.
// TAU (MODE 0 only): the epilogue also emits, per (row, tile), the partial sums that give dL/dtau.  With v = (W X)_i[t] = U_i[t] - b_i, Z_i[t] = a Z_i[t-1] + v[t-1] (Z = W dX/da), the
// tile's local Z_loc starts at 0 at its first bin t0, and Z[t] = a^(t-t0) Z[t0] + Z_loc[t]; a per-row
// combine (reduce.cu) chains the tiles.
template <int MODE, typename T16, bool TAU, bool BATCH, bool CT = false, bool SELF = false>
__global__ void __launch_bounds__(kthreads<MODE, CT, TAU, SELF>(), 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
                   const __grid_constant__ CUtensorMap mapB0, const __grid_constant__ CUtensorMap mapB1,
                   const __grid_constant__ TcArgs Ag, const TcBatch* __restrict__ batch) {
    using C = Cfg<MODE>;
    using L = Layout<MODE>;
    static_assert(!CT || MODE == 0, "the continuous-time epilogue is a U-product epilogue");
    static_assert(!SELF || (is_u<MODE>() && !TAU && !CT && !BATCH), "the self-delay is a grid U-product epilogue option");
    static_assert(MODE != 3 || !CT, "the continuous-time columns are always split");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * L::STAGE_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* tfull = empty + C::STAGES;
    uint64_t* tempty = tfull + 2;
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // per problem: first unit, row tiles, evaluated rows (one problem unless BATCH)
    __shared__ int64_t s_ubeg[MAX_BATCH + 1];
    __shared__ int32_t s_mt[MAX_BATCH], s_m[MAX_BATCH];
    __shared__ int s_np;
    // two epilogue warps per lane quarter (plain grid U product): the second warp hands its row sums of a
    // tile to the first through two slots (by tile parity); pfull: a slot's sums are written, pempty: read
    constexpr int NPART = (is_u<MODE>() && !CT) ? epi_warps<MODE, CT, TAU, SELF>() / 4 : 1;
    __shared__ double s_prs[NPART == 2 ? 2 : 1][128];
    __shared__ float s_pspv[NPART == 2 ? 2 : 1][128];
    __shared__ uint64_t s_pfull[2][4], s_pempty[2][4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        const int np = BATCH ? batch->nprob : 1;
        int64_t acc_units = 0;
        for (int p = 0; p < np; ++p) {
            const TcArgs& a = BATCH ? batch->args[p] : Ag;
            int32_t m = a.m_rows, mt = a.mt;
            int64_t units = a.units;
            if (is_u<MODE>()) {
                if (BATCH && batch->m_dev[p]) m = *batch->m_dev[p];
                mt = (m + Cfg<0>::BM - 1) / Cfg<0>::BM;
                units = (int64_t)mt * a.nt;
            } else if (BATCH && batch->m_dev[p] && *batch->m_dev[p] == 0) {
                units = 0;  // E X^T of a problem with no active row is not needed
            }
            s_ubeg[p] = acc_units;
            s_mt[p] = mt;
            s_m[p] = m;
            acc_units += units;
        }
        s_ubeg[np] = acc_units;
        s_np = np;
        for (int s = 0; s < C::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&tfull[a], 1);
            tc::mbar_init(&tempty[a], epi_warps<MODE, CT, TAU, SELF>());
        }
        tc::mbar_init(done, 1);
        for (int a = 0; a < 2; ++a)
            for (int qq = 0; qq < 4; ++qq) {
                tc::mbar_init(&s_pfull[a][qq], 32);
                tc::mbar_init(&s_pempty[a][qq], 32);
            }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (!BATCH && warp == 0 && lane == 0) {
        tc::prefetch_tensormap(&mapA0);
        tc::prefetch_tensormap(&mapA1);
        tc::prefetch_tensormap(&mapB0);
        if (C::NB == 2) tc::prefetch_tensormap(&mapB1);
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t total_units = s_ubeg[s_np];
    auto prob_of = [&](int64_t u) {
        int p = 0;
        while (u >= s_ubeg[p + 1]) ++p;
        return p;
    };
    auto args_of = [&](int p) -> const TcArgs& { return BATCH ? batch->args[p] : Ag; };
    auto map_of = [&](int p, int k) -> const CUtensorMap* {
        if (BATCH) return &batch->maps[p][k];
        return k == 0 ? &mapA0 : k == 1 ? &mapA1 : k == 2 ? &mapB0 : &mapB1;
    };

    auto raise = [&]() {
        *abort_flag = 1;
        atomicOr(Ag.flags + 1, 1);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[C::STAGES];
            for (int s = 0; s < C::STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < total_units && ok; u += gridDim.x) {
                const int p = prob_of(u);
                const TcArgs& A = args_of(p);
                const Unit w = decode<MODE>(A, u - s_ubeg[p], s_mt[p]);
                const CUtensorMap *mA0 = map_of(p, 0), *mA1 = map_of(p, 1), *mB0 = map_of(p, 2), *mB1 = map_of(p, 3);
                for (int64_t kb = w.kb0; kb < w.kb1; kb += w.kstep) {
                    if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag, Ag.limit_ns)) {
                        raise();
                        ok = false;
                        break;
                    }
                    uint8_t* sa = smem + stage * L::STAGE_BYTES;
                    // MODE 0 without X_lo leaves the stage's X_lo slot unused
                    tc::mbar_arrive_expect_tx(&full[stage], (MODE == 0 && !A.xlo) ? L::STAGE_BYTES - C::B_BYTES
                                                                                   : L::STAGE_BYTES);
                    const int32_t kx = (int32_t)(kb * C::BK);
                    if (is_u<MODE>()) {
                        tc::tma_load_2d(sa, mA0, kx, w.m0, &full[stage]);
                        tc::tma_load_2d(sa + C::A_BYTES, mA1, kx, w.m0, &full[stage]);
                        // (bin in block, neuron = k, bin block): 4 blocks of 32 x 64
                        tc::tma_load_3d(sa + 2 * C::A_BYTES, mB0, 0, kx, w.n0 / 64, &full[stage]);
                        if (C::NB == 2 && A.xlo)
                            tc::tma_load_3d(sa + 2 * C::A_BYTES + C::B_BYTES, mB1, 0, kx, w.n0 / 64, &full[stage]);
                    } else {
                        // (bin in block, neuron, bin block = k-step)
                        const bool second = A.kb_half > 0 && kb >= A.kb_half;
                        const int32_t kbx = (int32_t)(second ? kb - A.kb_half : kb);
                        tc::tma_load_3d(sa, mA0, 0, w.m0, kbx, &full[stage]);
                        if (C::NA == 2) tc::tma_load_3d(sa + C::A_BYTES, mA0, 0, w.m0 + 128, kbx, &full[stage]);
                        tc::tma_load_3d(sa + C::NA * C::A_BYTES, second ? mB1 : mB0, 0, w.n0, kbx, &full[stage]);
                    }
                    issued_phase[stage] = (int)phase;
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
            }
            // drain: every issued copy has landed before the block may exit
            volatile int never = 0;
            for (int s = 0; s < C::STAGES; ++s)
                if (issued_phase[s] >= 0) tc::mbar_wait(&full[s], (uint32_t)issued_phase[s], &never, Ag.limit_ns);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;
            bool ok = true;
            for (int64_t u = blockIdx.x; u < total_units && ok; u += gridDim.x, ++it) {
                const int p = prob_of(u);
                const Unit w = decode<MODE>(args_of(p), u - s_ubeg[p], s_mt[p]);
                const bool xlo = args_of(p).xlo != 0;
                const int buf = (C::NBUF == 2) ? (it & 1) : 0;
                const uint32_t buf_phase = (uint32_t)((C::NBUF == 2 ? (it >> 1) : it) & 1);
                if (!tc::mbar_wait(&tempty[buf], buf_phase ^ 1, abort_flag, Ag.limit_ns)) {
                    raise();
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d0 = tmem_base + (uint32_t)(buf * BN);
                const uint32_t d1 = tmem_base + (uint32_t)BN;  // MODE 1: second row half
                for (int64_t kb = w.kb0; kb < w.kb1; kb += w.kstep) {
                    if (!tc::mbar_wait(&full[stage], phase, abort_flag, Ag.limit_ns)) {
                        raise();
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t sa = tc::smem_u32(smem + stage * L::STAGE_BYTES);
                    const uint64_t da0 = smem_desc(sa, C::SWZ, C::SBO);
                    const uint64_t da1 = smem_desc(sa + C::A_BYTES, C::SWZ, C::SBO);
                    const uint64_t db0 = smem_desc(sa + C::NA * C::A_BYTES, C::B_SWZ, C::B_SBO, C::B_LBO);
                    const uint64_t db1 = smem_desc(sa + C::NA * C::A_BYTES + C::B_BYTES, C::B_SWZ, C::B_SBO, C::B_LBO);
#pragma unroll
                    for (int k = 0; k < C::BK / 16; ++k) {
                        const uint32_t acc = (kb == w.kb0 && k == 0) ? 0u : 1u;
                        const uint64_t ka = C::A_KSTEP * k, kb16 = C::B_KSTEP * k;
                        if (is_u<MODE>()) {
                            tc::mma_f16(d0, da0 + ka, db0 + kb16, Ag.idesc, acc);   // W_hi X_hi
                            tc::mma_f16(d0, da1 + ka, db0 + kb16, Ag.idesc, 1u);    // W_lo X_hi
                            if (C::NB == 2 && xlo) tc::mma_f16(d0, da0 + ka, db1 + kb16, Ag.idesc, 1u);  // W_hi X_lo
                        } else {
                            tc::mma_f16(d0, da0 + ka, db0 + kb16, Ag.idesc, acc);   // rows m0..
                            if (C::NA == 2) tc::mma_f16(d1, da1 + ka, db0 + kb16, Ag.idesc, acc);  // rows m0+128..
                        }
                    }
                    tc::mma_commit(&empty[stage]);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                tc::mma_commit(&tfull[buf]);
            }
            // drain: all issued MMAs have completed before TMEM is released
            tc::mma_commit(done);
            volatile int never = 0;
            tc::mbar_wait(done, 0, &never, Ag.limit_ns);
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;
        const int row = q * 32 + lane;
        int it = 0;
        for (int64_t u = blockIdx.x; u < total_units; u += gridDim.x, ++it) {
            const int p = prob_of(u);
            const TcArgs& A = args_of(p);
            const Unit w = decode<MODE>(A, u - s_ubeg[p], s_mt[p]);
            const int buf = (C::NBUF == 2) ? (it & 1) : 0;
            const uint32_t buf_phase = (uint32_t)((C::NBUF == 2 ? (it >> 1) : it) & 1);
            if (!tc::mbar_wait(&tfull[buf], buf_phase, abort_flag, Ag.limit_ns)) {
                raise();
                break;
            }
            tc::tc_fence_after();
            const uint32_t lane_base = tmem_base + ((uint32_t)(q * 32) << 16);
            if constexpr (MODE == 0 && CT) {
                // Continuous-time columns.  Per column m of length D_m: the exact integral of the rate,
                // e^{b} F(u, D_m) with u = (W V)_i at the column start, and the gradient weight
                // E'_m = e^{b} G(u, D_m) of Eq. 14 (ct_link.cuh).  With e^{b} = e^{c} e^{sh} as on the grid,
                // each of the CT_PARTS warps of a lane quarter takes a part of the tile's columns and writes its
                // share of the tile's sums, e^{c} e^{sh} (duration + sum (F - D)), to its own plane (the duration
                // counted by the first part).  Columns go 8 at a time (one 16-byte word of E').
                const int part = (warp - 2) >> 2;  // 0 .. CT_PARTS - 1
                const uint32_t taddr = lane_base + (uint32_t)(buf * BN);
                const int32_t il = w.m0 + row;
                const int32_t i = il < s_m[p] ? (A.rows ? A.rows[il] : il) : A.n;
                const int64_t gt0 = A.t_base + w.n0;
                const int64_t gtile = gt0 / BN;
                const double ebi = (i < A.n) ? A.eb[i] : 0.0;
                const float sh = (i < A.n) ? fminf(A.b[i] - EXP_SPLIT_FLOOR, 0.f) : 0.f;
                const float esh = __expf(sh);
                const float tgeb = (float)(ebi * (double)A.ct_tau) * esh;
                bool bad = !(tgeb <= 3.0e38f);
                float s = 0.f, spv = 0.f;
                // TAU: with z = W y (y_j = sum over arrivals (t - e) exp(-(t - e) / tau), dU/dtau = z / tau^2),
                // z at column m of the part is Pm z_start + z_loc[m], Pm the product of the part's decays so
                // far; the part leaves P1 = sum e^sh (G / tau) Pm, P2 = sum e^sh (G / tau) z_loc, Zend, over its
                // spike columns P3 = sum Pm and P4 = sum z_loc, Pex = sum e^sh dF/dtau at fixed u (ct_dtau), and
                // Aend = the product of its decays; a per-row scan (reduce.cu) chains the parts and tiles
                float zl = 0.f, pw = 1.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f, pex = 0.f;
                int64_t kb = 0, ke = 0;
                if (i < A.n) {
                    const int64_t sgi = (int64_t)i * A.nseg + gtile, o0 = A.offs[i];
                    kb = o0 + A.seg_first[sgi];
                    ke = (gtile + 1 < A.nseg) ? o0 + A.seg_first[sgi + 1] : A.offs[i + 1];
                }
                int sb[SP_REG];
#pragma unroll
                for (int u = 0; u < SP_REG; ++u) sb[u] = (kb + u < ke) ? (int)(A.bins[kb + u] - gt0) : BN;
                T16* erow = reinterpret_cast<T16*>(A.E) + ((int64_t)(w.n0 / 64) * A.n + i) * 64;
                const float4* colq = reinterpret_cast<const float4*>(A.colc) + 2 * gt0;
                const int g_begin = part * (BN / 8) / CT_PARTS, g_end = (part + 1) * (BN / 8) / CT_PARTS;
#pragma unroll 1
                for (int g = g_begin; g < g_end; ++g) {
                    const int c0 = g * 8;  // first column of the group within the tile
                    uint32_t r[8];
                    tc::tmem_ld8(taddr + c0, r);
                    float4 kc[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) kc[e] = __ldg(colq + 2 * (c0 + e));
                    tc::tmem_ld_wait();
                    uint32_t sm = 0;  // spike mask: bit e <-> column c0 + e
#pragma unroll
                    for (int u = 0; u < SP_REG; ++u) {
                        const uint32_t d = (uint32_t)(sb[u] - c0);
                        sm |= (d < 8u) ? (1u << d) : 0u;
                    }
                    for (int64_t k = kb + SP_REG; k < ke; ++k) {
                        const uint32_t d = (uint32_t)(A.bins[k] - gt0 - c0);
                        sm |= (d < 8u) ? (1u << d) : 0u;
                    }
                    float fv[8], gv[8];
                    uint32_t slow = 0;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float4 k = kc[e];  // a, 1 - a, 2-node factors
                        const float u = __uint_as_float(r[e]);
                        ct_link2(u, k.x, k.y, k.z, k.w, &fv[e], &gv[e]);
                        slow |= (fabsf(u) * k.y > CT_W2_MAX) ? (1u << e) : 0u;
                    }
                    if (__any_sync(0xffffffffu, slow != 0u)) {  // columns where the exponent moves by > 0.1
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            if ((slow >> e) & 1u) {
                                const float4 k0 = __ldg(colq + 2 * (c0 + e)), k1 = __ldg(colq + 2 * (c0 + e) + 1);
                                const float col[8] = {k0.x, k0.y, k0.z, k0.w, k1.x, k1.y, k1.z, k1.w};
                                ct_link(__uint_as_float(r[e]), col, A.ct_tau, &fv[e], &gv[e]);
                            }
                        }
                    }
                    uint32_t pk[4];
#pragma unroll
                    for (int e = 0; e < 8; e += 2) {
                        const int64_t t = gt0 + c0 + e;
                        const bool v0 = t < A.T, v1 = t + 1 < A.T;
                        float e0 = tgeb * gv[e], e1 = tgeb * gv[e + 1];
                        bad |= (v0 && !(fabsf(fv[e]) <= 3.0e38f && e0 <= 3.0e38f)) ||
                               (v1 && !(fabsf(fv[e + 1]) <= 3.0e38f && e1 <= 3.0e38f));
                        if (v0) s += fv[e]; else e0 = 0.f;
                        if (v1) s += fv[e + 1]; else e1 = 0.f;
                        if ((sm >> e) & 1u) spv += __uint_as_float(r[e]);
                        if ((sm >> (e + 1)) & 1u) spv += __uint_as_float(r[e + 1]);
                        pk[e >> 1] = pack16<T16>(e0, e1);
                    }
                    if constexpr (TAU) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            if (gt0 + c0 + e < A.T) {  // columns in order; the padding past T takes no part
                                const float u = __uint_as_float(r[e]), ca = kc[e].x, coma = kc[e].y;
                                const float egs = esh * gv[e];
                                p1 = fmaf(egs, pw, p1);
                                p2 = fmaf(egs, zl, p2);
                                if ((sm >> e) & 1u) {
                                    p3 += pw;
                                    p4 += zl;
                                }
                                pex = fmaf(esh, ct_dtau(u, ca, coma, A.ct_tau, fv[e]), pex);
                                zl = (ca == 0.f) ? 0.f : ca * fmaf(ct_length(ca, coma, A.ct_tau), u, zl);
                                pw *= ca;
                            }
                        }
                    }
                    if (i < A.n)
                        *reinterpret_cast<uint4*>(erow + (int64_t)(c0 >> 6) * A.n * 64 + (c0 & 63)) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
                if (i < A.n) {
                    const double rsum = (double)esh * ((part == 0 ? A.tile_span[gtile] : 0.0) + (double)s);
                    const int64_t o = (int64_t)part * A.n * A.ntile + (int64_t)i * A.ntile + gtile;
                    A.part_e[o] = ebi * rsum;
                    A.part_s[o] = (double)spv;
                    if constexpr (TAU) {  // [7][CT_PARTS][n][ntile]
                        const int64_t pl = (int64_t)CT_PARTS * A.n * A.ntile;
                        A.part_tau[o] = p1;
                        A.part_tau[pl + o] = p2;
                        A.part_tau[2 * pl + o] = zl;
                        A.part_tau[3 * pl + o] = p3;
                        A.part_tau[4 * pl + o] = p4;
                        A.part_tau[5 * pl + o] = pex;
                        A.part_tau[6 * pl + o] = pw;
                    }
                }
                if (bad && i < A.n) atomicOr(A.flags, 1);
            } else if constexpr (is_u<MODE>()) {
                // e^{U} = e^{b_i} e^{v}, v = (W X)_i[t]: e^{b_i} in FP64, and the row sum is kept as
                // e^{b_i} (count + sum (e^{v} - 1)), so quiet bins (v ~ 0) add no FP32 rounding of b + v.
                const uint32_t taddr = lane_base + (uint32_t)(buf * BN);
                const int32_t il = w.m0 + row;
                const int32_t i = il < s_m[p] ? (A.rows ? A.rows[il] : il) : A.n;
                const int64_t gt0 = A.t_base + w.n0;  // first bin of the tile in the recording
                const int64_t gtile = gt0 / BN;
                const double ebi = (i < A.n) ? A.eb[i] : 0.0;
                const float sh = (i < A.n) ? fminf(A.b[i] - EXP_SPLIT_FLOOR, 0.f) : 0.f;  // U - c = v + sh
                const float dteb = (float)(A.dt * ebi);
                double rsum = 0.0;
                bool bad = false;
                float zl = 0.f, pw = 1.f, p1 = 0.f, p2 = 0.f, p3 = 0.f, p4 = 0.f, spv = 0.f;
                // self-delay: W_ii as the product holds it (hi + lo) and the row's X rows
                float wii = 0.f;
                double sself = 0.0;
                const T16* xsh = reinterpret_cast<const T16*>(A.Xhi);
                const T16* xsl = reinterpret_cast<const T16*>(A.Xlo);
                if (SELF && i < A.n) wii = split_sum16<T16>(A.W32[(int64_t)i * A.n + i]);
                // the row's spike bins in this tile (tile = 256-bin segment n0 / 256): the first ST_REG in
                // registers, relative to the tile start; any further ones are read per chunk.  The spike part
                // of L is taken from this U at those bins: the tensor cores' FP32 accumulation of U carries a
                // bias (measured ~6e-6 at N = 1000) that then cancels against the integral part.
                int64_t kb = 0, ke = 0;
                if (i < A.n) {
                    const int64_t sgi = (int64_t)i * A.nseg + gtile, o0 = A.offs[i];
                    kb = o0 + A.seg_first[sgi];
                    ke = (gtile + 1 < A.nseg) ? o0 + A.seg_first[sgi + 1] : A.offs[i + 1];
                }
                int sb[SP_REG];
#pragma unroll
                for (int u = 0; u < SP_REG; ++u) sb[u] = (kb + u < ke) ? (int)(A.bins[kb + u] - gt0) : BN;
                // E is bin-blocked: bins [64 b, 64 b + 64) of row i at (b n + i) 64
                T16* erow = reinterpret_cast<T16*>(A.E) + ((int64_t)(w.n0 / 64) * A.n + i) * 64;
                // with two warps per lane quarter, warp part 0 takes the tile's first 128 bins, part 1 the rest
                const int part = (NPART == 2) ? ((warp - 2) >> 2) : 0;
#pragma unroll 1
                for (int c = part * (BN / 32) / NPART; c < (part + 1) * (BN / 32) / NPART; ++c) {
                    uint32_t r[32];
                    tc::tmem_ld32(taddr + c * 32, r);
                    tc::tmem_ld_wait();
                    // spike mask of the chunk: bit m <-> bin n0 + 32 c + m
                    uint32_t sm = 0;
#pragma unroll
                    for (int u = 0; u < SP_REG; ++u) {
                        const uint32_t d = (uint32_t)(sb[u] - c * 32);
                        sm |= (d < 32u) ? (1u << d) : 0u;
                    }
                    for (int64_t k = kb + SP_REG; k < ke; ++k) {
                        const uint32_t d = (uint32_t)(A.bins[k] - gt0 - c * 32);
                        sm |= (d < 32u) ? (1u << d) : 0u;
                    }
                    float s = 0.f;
                    int cnt = 0;
                    uint32_t pk[16];
                    float dxs[32];  // SELF: X_i[t + self_shift] - X_i[t] over the chunk
                    if (SELF) {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int64_t t = gt0 + c * 32 + e;
                            const int64_t t2 = t + A.self_shift;  // < Tpad for t < T (Tpad >= T + self_shift)
                            dxs[e] = 0.f;
                            if (i < A.n && t < A.T) {
                                const int64_t o1 = ((t >> 6) * A.n + i) * 64 + (t & 63);
                                const int64_t o2 = ((t2 >> 6) * A.n + i) * 64 + (t2 & 63);
                                dxs[e] = xsl ? (to_f(xsh[o2]) + to_f(xsl[o2])) - (to_f(xsh[o1]) + to_f(xsl[o1]))
                                             : to_f(xsh[o2]) - to_f(xsh[o1]);
                            }
                            r[e] = __float_as_uint(fmaf(wii, dxs[e], __uint_as_float(r[e])));
                        }
                    }
                    float ss = 0.f;
#pragma unroll
                    for (int e = 0; e < 32; e += 2) {
                        const int64_t t = gt0 + c * 32 + e;
                        const float v0f = __uint_as_float(r[e]), v1f = __uint_as_float(r[e + 1]);
                        const bool v0 = t < A.T, v1 = t + 1 < A.T;
                        const bool s0 = (sm >> e) & 1u, s1 = (sm >> (e + 1)) & 1u;
                        float e0 = __expf(v0f + sh);
                        float e1 = __expf(v1f + sh);
                        bad |= (v0 && !(e0 <= 3.0e38f)) || (v1 && !(e1 <= 3.0e38f));
                        if (v0) {
                            s += e0 - 1.f;
                            ++cnt;
                        } else {
                            e0 = 0.f;
                        }
                        if (v1) {
                            s += e1 - 1.f;
                            ++cnt;
                        } else {
                            e1 = 0.f;
                        }
                        if (s0) spv += v0f;
                        if (s1) spv += v1f;
                        pk[e >> 1] = pack16<T16>(dteb * e0, dteb * e1);
                        if (SELF) ss = fmaf(e0, dxs[e], fmaf(e1, dxs[e + 1], ss));
                        if (TAU) {
                            p1 = fmaf(e0, pw, p1);
                            p2 = fmaf(e0, zl, p2);
                            if (s0) {
                                p3 += pw;
                                p4 += zl;
                            }
                            zl = fmaf(A.a, zl, v0f);
                            pw *= A.a;
                            p1 = fmaf(e1, pw, p1);
                            p2 = fmaf(e1, zl, p2);
                            if (s1) {
                                p3 += pw;
                                p4 += zl;
                            }
                            zl = fmaf(A.a, zl, v1f);
                            pw *= A.a;
                        }
                    }
                    rsum += (double)cnt + (double)s;
                    if (SELF) sself += (double)ss;
                    if (i < A.n) {
                        uint4* dst = reinterpret_cast<uint4*>(erow + (int64_t)(c >> 1) * A.n * 64 + (c & 1) * 32);
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            dst[v] = make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
                    }
                }
                bad |= !(dteb <= 3.0e38f);
                if constexpr (NPART == 2) {
                    // part 1 hands its sums to part 0 (bounded waits: a partner that gave up ends this too)
                    const int slot = it & 1;
                    const uint32_t use = (uint32_t)(it >> 1);
                    bool ok = true;
                    if (part == 1) {
                        ok = use == 0 || tc::mbar_wait(&s_pempty[slot][q], (use - 1) & 1u, abort_flag, Ag.limit_ns);
                        if (ok) {
                            s_prs[slot][row] = rsum;
                            s_pspv[slot][row] = spv;
                            tc::mbar_arrive(&s_pfull[slot][q]);
                        }
                    } else {
                        ok = tc::mbar_wait(&s_pfull[slot][q], use & 1u, abort_flag, Ag.limit_ns);
                        if (ok) {
                            rsum += s_prs[slot][row];
                            spv += s_pspv[slot][row];
                            tc::mbar_arrive(&s_pempty[slot][q]);
                        }
                    }
                    if (!ok) {
                        raise();
                        break;
                    }
                }
                if (part == 0 && i < A.n) {
                    A.part_e[(int64_t)i * A.ntile + gtile] = ebi * rsum;
                    A.part_s[(int64_t)i * A.ntile + gtile] = (double)spv;
                }
                if (SELF && i < A.n) A.part_self[(int64_t)i * A.ntile + gtile] = A.dt * ebi * sself;
                if (TAU && i < A.n) {
                    const int64_t o = (int64_t)i * A.ntile + gtile, plane = (int64_t)A.n * A.ntile;
                    A.part_tau[o] = p1;
                    A.part_tau[plane + o] = p2;
                    A.part_tau[2 * plane + o] = zl;
                    A.part_tau[3 * plane + o] = p3;
                    A.part_tau[4 * plane + o] = p4;
                }
                if (bad && i < A.n) atomicOr(A.flags, 1);  // rows past the evaluated set hold stale W parts
            } else {
#pragma unroll 1
                for (int h = 0; h < C::NA; ++h) {
                    const uint32_t taddr = lane_base + (uint32_t)((buf + h) * BN);
                    const int32_t i = w.m0 + h * 128 + row;
                    float* grow = A.part_g + ((int64_t)w.split * A.n + i) * A.n;
#pragma unroll 1
                    for (int c = 0; c < BN / 32; ++c) {
                        uint32_t r[32];
                        tc::tmem_ld32(taddr + c * 32, r);
                        tc::tmem_ld_wait();
                        if (i < A.n) {
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const int32_t j = w.n0 + c * 32 + e;
                                if (j < A.n) grow[j] = __uint_as_float(r[e]);
                            }
                        }
                    }
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&tempty[buf]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

template <typename T16>
// hi + lo parts of the evaluated rows of W, packed: part row l holds row rows[l] (all rows when rows is null);
// m rows, or *m_dev when given
__global__ void split_w_kernel(int32_t n, int64_t ldk, const float* __restrict__ W, const int32_t* __restrict__ rows,
                               int32_t m, const int32_t* __restrict__ m_dev, T16* __restrict__ hi, T16* __restrict__ lo,
                               int* flags) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m_dev) m = *m_dev;
    if (e >= (int64_t)m * ldk) return;
    const int64_t pr = e / ldk, k = e % ldk;
    const int64_t i = rows ? rows[pr] : pr;
    float w = 0.f;
    if (k < n) w = W[i * n + k];
    if (!isfinite(w)) atomicOr(flags, 1);
    T16 h, l;
    if constexpr (std::is_same<T16, __nv_bfloat16>::value) {
        h = __float2bfloat16_rn(w);
        l = __float2bfloat16_rn(w - __bfloat162float(h));
    } else {
        h = __float2half_rn(w);
        l = __float2half_rn(w - __half2float(h));
    }
    hi[e] = h;
    lo[e] = l;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over a row-major matrix [rows][inner] with row stride ld elements; box = box_k x box_rows.
bool encode_map(CUtensorMap* m, bool bf16, const void* base, uint64_t inner, uint64_t rows, uint64_t ld,
                uint32_t box_k, uint32_t box_rows, CUtensorMapSwizzle swz) {
    auto fn = get_encode();
    if (!fn) return false;
    const cuuint64_t dims[2] = {inner, rows};
    const cuuint64_t strides[1] = {ld * 2};
    const cuuint32_t box[2] = {box_k, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 3-D map over a bin-blocked array [Tpad / 64][n][64]: dims (64 bins, n neurons, Tpad / 64 blocks),
// box = 64 x box_rows x box_blocks, 128-byte swizzle.  Neurons beyond n read as zero.
bool encode_blocked(CUtensorMap* m, bool bf16, const void* base, uint64_t n, uint64_t Tpad, uint32_t box_rows,
                    uint32_t box_blocks) {
    auto fn = get_encode();
    if (!fn) return false;
    const cuuint64_t dims[3] = {64, n, Tpad / 64};
    const cuuint64_t strides[2] = {128, n * 128};
    const cuuint32_t box[3] = {64, box_rows, box_blocks};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

// Splits of the bins for E X^T with row tiles of 256 (mode 1) or 128 (mode 2) so that the launch has about
// units_per_sm units per SM.
// k-steps of one E X^T product: the recording, or one chunk of it
static int64_t grad_ksteps(const glm_ctx* c) {
    const int64_t bins = c->pb.chunk ? c->pb.Tc : c->pb.T;
    return (bins + Cfg<1>::BK - 1) / Cfg<1>::BK;
}

int tc_nsplit_for(const glm_ctx* c, int mode, int units_per_sm) {
    const int64_t bm = mode == 2 ? 128 : 256;
    const int64_t tiles = (int64_t)((c->pb.n + bm - 1) / bm) * ((c->pb.n + BN - 1) / BN);
    const int64_t kb_total = grad_ksteps(c);
    int64_t s = ((int64_t)units_per_sm * c->sm_count + tiles - 1) / tiles;
    if (s > kb_total) s = kb_total;
    if (s < 1) s = 1;
    const int64_t kps = (kb_total + s - 1) / s;
    return (int)((kb_total + kps - 1) / kps);  // no empty split
}

int tc_nsplit(const glm_ctx* c) { return c->g_nsplit > 0 ? c->g_nsplit : tc_nsplit_for(c, c->g_mode, 4); }

int tc_nsplit_max(const glm_ctx* c) { return tc_nsplit_for(c, 1, TUNE_UPM_MAX); }

int tc_tile_t() { return BN; }

// Maps: 0 W_hi, 1 W_lo (U = W X, K-major, 64-byte swizzle), 2 X_hi, 3 X_lo (U = W X, N-major boxes of 4 x 32 x 64),
// 4 E, 5 X_hi, 6 X_lo (E X^T and S X^T, K-major boxes of 1 x 128 (E) or 1 x 256 (X) x 64).  Maps 2-6 are 3-D
// maps over the bin-blocked arrays (bin in block, neuron, bin block), all with the 128-byte swizzle.
cudaError_t tc_prepare_maps(glm_ctx* c) {
    const Problem& P = c->pb;
    const bool bf = P.prec == GLM_PREC_BF16;
    const int64_t ld = c->buf.ldn;
    const size_t wsz = (size_t)P.n * ld * 2;
    const uint8_t* Wsplit = reinterpret_cast<const uint8_t*>(c->buf.Wsplit);
    const auto S64 = CU_TENSOR_MAP_SWIZZLE_64B;
    // without the X split, maps 3 and 6 cover X_hi: valid maps that no product reads
    const void* Xlo = P.xlo ? c->buf.Xlo : c->buf.X;
    bool ok = encode_map(&c->tmap[0], bf, Wsplit, P.n, P.n, ld, 32, 128, S64) &&
              encode_map(&c->tmap[1], bf, Wsplit + wsz, P.n, P.n, ld, 32, 128, S64) &&
              encode_blocked(&c->tmap[2], bf, c->buf.X, P.n, P.Tc, Cfg<0>::BK, BN / 64) &&
              encode_blocked(&c->tmap[3], bf, Xlo, P.n, P.Tc, Cfg<0>::BK, BN / 64) &&
              encode_blocked(&c->tmap[4], bf, c->buf.E, P.n, P.Tc, 128, 1) &&
              encode_blocked(&c->tmap[5], bf, c->buf.X, P.n, P.Tc, BN, 1) &&
              encode_blocked(&c->tmap[6], bf, Xlo, P.n, P.Tc, BN, 1);
    return ok ? cudaSuccess : cudaErrorInvalidValue;
}

template <int MODE, typename T16, bool TAU = false, bool BATCH = false, bool CT = false, bool SELF = false>
static cudaError_t run(glm_ctx* c, const CUtensorMap& a0, const CUtensorMap& a1, const CUtensorMap& b0,
                       const CUtensorMap& b1, const TcArgs& A, const TcBatch* batch = nullptr, int64_t grid = 0) {
    const size_t smem = Layout<MODE>::SMEM;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(c->stream, &cap);
    if (e != cudaSuccess) return e;
    if (cap == cudaStreamCaptureStatusNone) {  // set before the first launch; not during graph capture
        e = cudaFuncSetAttribute(tc_gemm_kernel<MODE, T16, TAU, BATCH, CT, SELF>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (grid <= 0) grid = A.units < c->sm_count ? A.units : c->sm_count;
    tc_gemm_kernel<MODE, T16, TAU, BATCH, CT, SELF><<<(unsigned)grid, kthreads<MODE, CT, TAU, SELF>(), smem, c->stream>>>(
        a0, a1, b0, b1, A, batch);
    return cudaGetLastError();
}

static TcArgs base_args(glm_ctx* c) {
    const Problem& P = c->pb;
    TcArgs A;
    A.n = P.n;
    A.T = P.T;
    A.Tpad = P.Tpad;
    A.dt = P.dt;
    A.flags = c->buf.flags;
    A.limit_ns = 4000000000ull;  // 4 s per wait
    A.kb_half = 0;
    A.idesc = tc::idesc_f16(P.prec == GLM_PREC_BF16 ? 1u : 0u, 128, BN);  // both operands K-major
    A.b = nullptr;
    A.eb = c->buf.eb;
    A.a = (float)P.a;
    A.part_tau = nullptr;
    A.part_s = nullptr;
    A.rows = nullptr;
    A.m_rows = P.n;
    A.m_base = 0;
    A.t_base = 0;
    A.offs = c->buf.offs;
    A.bins = c->buf.bins;
    A.seg_first = c->buf.seg_first;
    A.nseg = P.nseg;
    A.E = nullptr;
    A.part_e = nullptr;
    A.part_g = nullptr;
    A.ntile = P.Tpad / BN;
    A.kb_total = 0;
    A.nsplit = 1;
    A.colc = c->buf.colc;
    A.tile_span = c->buf.tile_span;
    A.ct_tau = (float)P.tau;
    A.self_shift = 0;
    A.W32 = nullptr;
    A.Xhi = c->buf.X;
    A.Xlo = P.xlo ? c->buf.Xlo : nullptr;
    A.xlo = P.xlo ? 1 : 0;
    A.part_self = nullptr;
    return A;
}

// the grid U product in MODE 0 (X_hi + X_lo) or MODE 3 (one X), with the tau partials or the self-delay term
template <int MODE>
static cudaError_t run_u(glm_ctx* c, TcArgs& A, bool tau, bool self, const float* W) {
    const Problem& P = c->pb;
    const bool bf = P.prec == GLM_PREC_BF16;
    if (tau) {
        if (self) return cudaErrorNotSupported;
        if (bf) return run<MODE, __nv_bfloat16, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
        return run<MODE, __half, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
    }
    if (self) {
        if (P.chunk) return cudaErrorNotSupported;
        A.self_shift = P.self_shift;
        A.W32 = W;
        A.part_self = c->buf.part_self;
        if (bf)
            return run<MODE, __nv_bfloat16, false, false, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
        return run<MODE, __half, false, false, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
    }
    if (bf) return run<MODE, __nv_bfloat16>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
    return run<MODE, __half>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
}

cudaError_t launch_tc_u_epilogue(glm_ctx* c, const float* W, const float* b, bool tau, const int32_t* rows,
                                 int32_t m, int64_t t_base, int64_t t_len) {
    const Problem& P = c->pb;
    const int64_t ldk = c->buf.ldn;
    const int32_t mr = rows ? m : P.n;
    const int64_t total = (int64_t)mr * ldk;
    const size_t wsz = (size_t)P.n * ldk;
    if (P.prec == GLM_PREC_BF16) {
        auto* hi = reinterpret_cast<__nv_bfloat16*>(c->buf.Wsplit);
        split_w_kernel<__nv_bfloat16><<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(
            P.n, ldk, W, rows, mr, nullptr, hi, hi + wsz, c->buf.flags);
    } else {
        auto* hi = reinterpret_cast<__half*>(c->buf.Wsplit);
        split_w_kernel<__half><<<(unsigned)((total + 255) / 256), 256, 0, c->stream>>>(P.n, ldk, W, rows, mr, nullptr,
                                                                                      hi, hi + wsz, c->buf.flags);
    }
    launch_exp_bias(c, b);
    TcArgs A = base_args(c);
    A.rows = rows;
    A.m_rows = mr;
    A.t_base = t_base;
    A.mt = (mr + 127) / 128;
    A.nt = (int32_t)((t_len < 0 ? P.Tc : t_len) / BN);
    A.units = (int64_t)A.mt * A.nt;
    A.kb_per_unit = (P.n + Cfg<0>::BK - 1) / Cfg<0>::BK;
    A.b = b;
    A.E = c->buf.E;
    A.part_e = c->buf.part_e;
    A.part_tau = c->buf.part_tau;
    A.part_s = c->buf.part_s;
    A.idesc |= 1u << 16;  // B (X) is N-major
    if (P.ct) {
        if (P.prec == GLM_PREC_BF16) {
            if (tau) return run<0, __nv_bfloat16, true, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
            return run<0, __nv_bfloat16, false, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
        }
        if (tau) return run<0, __half, true, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
        return run<0, __half, false, false, true>(c, c->tmap[0], c->tmap[1], c->tmap[2], c->tmap[3], A);
    }
    if (P.xlo) return run_u<0>(c, A, tau, P.self_shift > 0, W);
    return run_u<3>(c, A, tau, P.self_shift > 0, W);
}

// E X^T arguments of context c with its tile mode and split count
static TcArgs grad_args(glm_ctx* c, int mode, int ns, int64_t kbt, bool ranged = false) {
    const Problem& P = c->pb;
    TcArgs A = base_args(c);
    // a row range needs only the row tiles that cover it
    const int32_t r0 = ranged ? c->row_r0 : 0, r1 = (ranged && c->row_r1 >= 0) ? c->row_r1 : P.n;
    A.m_base = r0;
    A.mt = (r1 - r0 + (mode == 2 ? 127 : 255)) / (mode == 2 ? 128 : 256);
    A.nt = (P.n + BN - 1) / BN;
    A.kb_total = kbt;
    A.kb_per_unit = (int32_t)((A.kb_total + ns - 1) / ns);
    A.units = (int64_t)A.mt * A.nt * ns;
    A.nsplit = ns;
    A.part_g = c->buf.part_g;
    return A;
}

// mapB2 (when given): a second B operand over the same kbt k-steps, summed into the same accumulators
static cudaError_t run_products_as(glm_ctx* c, const CUtensorMap& mapB, int mode, int ns, int64_t kbt,
                                   bool ranged = false, const CUtensorMap* mapB2 = nullptr) {
    TcArgs A = grad_args(c, mode, ns, mapB2 ? 2 * kbt : kbt, ranged);
    if (mapB2) A.kb_half = kbt;
    const CUtensorMap& mB1 = mapB2 ? *mapB2 : mapB;
    const bool bf = c->pb.prec == GLM_PREC_BF16;
    if (mode == 2) {
        if (bf) return run<2, __nv_bfloat16>(c, c->tmap[4], c->tmap[4], mapB, mB1, A);
        return run<2, __half>(c, c->tmap[4], c->tmap[4], mapB, mB1, A);
    }
    if (bf) return run<1, __nv_bfloat16>(c, c->tmap[4], c->tmap[4], mapB, mB1, A);
    return run<1, __half>(c, c->tmap[4], c->tmap[4], mapB, mB1, A);
}

// E X^T (or S X^T) over the first t_len bins of the buffers (t_len < 0: the recording, or a whole chunk);
// a short last chunk takes at most one split per k-step.
// ranged: only the row tiles of the context's row range (the gradient); the spike term takes every row
static cudaError_t run_products(glm_ctx* c, const CUtensorMap& mapB, int64_t t_len, int* ns_used, bool ranged = false,
                                const CUtensorMap* mapB2 = nullptr) {
    const int64_t kbt = t_len < 0 ? grad_ksteps(c) : (t_len + Cfg<1>::BK - 1) / Cfg<1>::BK;
    int ns = tc_nsplit(c);
    if (ns > kbt) ns = (int)kbt;
    if (ns_used) *ns_used = ns;
    return run_products_as(c, mapB, c->g_mode, ns, kbt, ranged, mapB2);
}

cudaError_t launch_tc_grad(glm_ctx* c, int64_t t_len, int* nsplit_used) {
    return run_products(c, c->tmap[5], t_len, nsplit_used, true,
                        (c->precise_grad && c->pb.xlo) ? &c->tmap[6] : nullptr);
}

// With X recomputed per chunk, each chunk is filtered here first and the products add up over the chunks.
// Self-delay: the diagonal of the spike term sums row i's own train as it reaches row i,
// C_ii = sum_{t in sp(i)} X_i[t + shift]; the product above summed X_i[t].  Warp per row, fixed order.
template <typename T16>
__global__ void self_spike_diag_kernel(int32_t n, int32_t shift, const int64_t* __restrict__ offs,
                                       const int32_t* __restrict__ bins, const T16* __restrict__ xh,
                                       const T16* __restrict__ xl, double* __restrict__ C) {
    const int32_t i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    double d = 0.0;
    for (int64_t k = offs[i] + lane; k < offs[i + 1]; k += 32) {
        const int64_t t = bins[k], t2 = t + shift;
        const int64_t o1 = ((t >> 6) * n + i) * 64 + (t & 63), o2 = ((t2 >> 6) * n + i) * 64 + (t2 & 63);
        d += xl ? (double)((to_f(xh[o2]) + to_f(xl[o2])) - (to_f(xh[o1]) + to_f(xl[o1])))
                : (double)(to_f(xh[o2]) - to_f(xh[o1]));
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
    if (lane == 0) C[(int64_t)i * n + i] += d;
}

cudaError_t launch_tc_spike_term(glm_ctx* c) {
    const Problem& P = c->pb;
    cudaError_t e = cudaSuccess;
    for (int64_t t0 = 0; t0 < P.Tpad; t0 += P.Tc) {
        const int64_t len = std::min(P.Tc, P.Tpad - t0);
        const bool fused = P.delay_bins <= 1 && !P.ct;  // the filter's sources are the rows' own spikes
        if (P.chunk && (e = launch_filter_cache(c, t0 / SEG, (t0 + len) / SEG, fused ? c->buf.E : nullptr)) != cudaSuccess)
            return e;
        const bool raster = !(fused && (P.chunk || c->raster_in_E));
        if (raster && (e = launch_spike_raster(c, c->buf.E, t0 / SEG, (t0 + len) / SEG)) != cudaSuccess) return e;
        c->launches += (P.chunk ? 1 : 0) + (raster ? 1 : 0) + 2;  // filter, raster, the products, the sum
        c->raster_in_E = false;  // consumed below; the next U product overwrites E
        int ns = 0;
        const int64_t bins = P.chunk ? len : P.T;
        // S X_hi^T and S X_lo^T in one launch: each split runs over its bins of X_hi, then of X_lo (S X^T alone
        // without the X split)
        if ((e = run_products(c, c->tmap[5], bins, &ns, false, P.xlo ? &c->tmap[6] : nullptr)) != cudaSuccess)
            return e;
        if ((e = launch_sum_splits(c, ns, c->buf.C, t0 > 0)) != cudaSuccess) return e;
    }
    if (P.self_shift > 0) {  // X stored (no chunks): the whole recording is in the buffers
        const unsigned blocks = (unsigned)((P.n + 7) / 8);
        if (P.prec == GLM_PREC_BF16)
            self_spike_diag_kernel<<<blocks, 256, 0, c->stream>>>(
                P.n, P.self_shift, c->buf.offs, c->buf.bins, reinterpret_cast<const __nv_bfloat16*>(c->buf.X),
                reinterpret_cast<const __nv_bfloat16*>(c->buf.Xlo), c->buf.C);
        else
            self_spike_diag_kernel<<<blocks, 256, 0, c->stream>>>(
                P.n, P.self_shift, c->buf.offs, c->buf.bins, reinterpret_cast<const __half*>(c->buf.X),
                reinterpret_cast<const __half*>(c->buf.Xlo), c->buf.C);
        c->launches += 1;
        e = cudaGetLastError();
    }
    return e;
}

// One thread waits, with the bounded wait of the kernels above, on an mbarrier that expects an arrival
// nobody makes; it must give up after limit_ns and report it (out = 2).
__global__ void wait_check_kernel(uint64_t limit_ns, int* out) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) out[0] = tc::mbar_wait(&bar, 0, &abort_flag, limit_ns) ? 1 : 2;
}

cudaError_t launch_wait_check(glm_ctx* c, uint64_t limit_ns, int* out) {
    wait_check_kernel<<<1, 32, 0, c->stream>>>(limit_ns, out);
    return cudaGetLastError();
}

// ---- several problems per launch (glm_fit_batch) ----

// E X^T arguments of one problem of the batched launch: over X_hi, then X_lo when the gradient is precise
static TcArgs batch_grad_args(glm_ctx* c, int mode, int ns) {
    const int64_t kbt = grad_ksteps(c);
    const bool precise = c->precise_grad && c->pb.xlo;
    TcArgs A = grad_args(c, mode, ns, precise ? 2 * kbt : kbt);
    if (precise) A.kb_half = kbt;
    return A;
}

size_t tc_batch_bytes() { return sizeof(TcBatch); }

// Host images of the two batch descriptors: U products of the rows rows[p] (m_dev[p] of them) at
// (W32[p], b32[p]), and E X^T.  All problems share one precision.
int tc_batch_fill(glm_ctx* const* cs, int np, float* const* W32, float* const* b32, int32_t* const* rows,
                  const int32_t* const* m_dev, void* host_u, void* host_g) {
    if (np < 1 || np > MAX_BATCH) return GLM_ERR_INVALID_ARG;
    TcBatch* bu = static_cast<TcBatch*>(host_u);
    TcBatch* bg = static_cast<TcBatch*>(host_g);
    std::memset(static_cast<void*>(bu), 0, sizeof(TcBatch));
    std::memset(static_cast<void*>(bg), 0, sizeof(TcBatch));
    bu->nprob = bg->nprob = np;
    for (int p = 0; p < np; ++p) {
        glm_ctx* c = cs[p];
        const Problem& P = c->pb;
        TcArgs A = base_args(c);
        A.rows = rows[p];
        A.m_rows = P.n;
        A.mt = (P.n + 127) / 128;
        A.nt = (int32_t)(P.Tpad / BN);
        A.units = (int64_t)A.mt * A.nt;
        A.kb_per_unit = (P.n + Cfg<0>::BK - 1) / Cfg<0>::BK;
        A.b = b32[p];
        A.E = c->buf.E;
        A.part_e = c->buf.part_e;
        A.part_tau = c->buf.part_tau;
        A.part_s = c->buf.part_s;
        bu->args[p] = A;
        bu->m_dev[p] = m_dev[p];
        for (int k = 0; k < 4; ++k) bu->maps[p][k] = c->tmap[k];
        bg->args[p] = batch_grad_args(c, c->g_mode, tc_nsplit(c));
        bg->maps[p][0] = bg->maps[p][1] = c->tmap[4];
        bg->maps[p][2] = c->tmap[5];
        bg->maps[p][3] = (c->precise_grad && c->pb.xlo) ? c->tmap[6] : c->tmap[5];
    }
    (void)W32;
    return GLM_OK;
}

// One launch of the U product over every problem's evaluated rows (their count read on the device); the
// W splits and exp(b) of the problems are formed before it (by the caller).
cudaError_t launch_tc_u_batch(glm_ctx* c0, const void* dev_u) {
    TcArgs Ag = base_args(c0);
    Ag.idesc |= 1u << 16;  // B (X) is N-major
    const TcBatch* b = static_cast<const TcBatch*>(dev_u);
    const CUtensorMap* m = c0->tmap;
    const bool bf = c0->pb.prec == GLM_PREC_BF16;
    if (!c0->pb.xlo) {  // every problem of a batch has the same form (checked by glm_fit_batch)
        if (bf) return run<3, __nv_bfloat16, false, true>(c0, m[0], m[1], m[2], m[3], Ag, b, c0->sm_count);
        return run<3, __half, false, true>(c0, m[0], m[1], m[2], m[3], Ag, b, c0->sm_count);
    }
    if (bf) return run<0, __nv_bfloat16, false, true>(c0, m[0], m[1], m[2], m[3], Ag, b, c0->sm_count);
    return run<0, __half, false, true>(c0, m[0], m[1], m[2], m[3], Ag, b, c0->sm_count);
}

// One launch of E X^T over every problem (all in c0's tile mode).
cudaError_t launch_tc_grad_batch(glm_ctx* c0, const void* dev_g) {
    TcArgs Ag = base_args(c0);
    const TcBatch* b = static_cast<const TcBatch*>(dev_g);
    const CUtensorMap* m = c0->tmap;
    const bool bf = c0->pb.prec == GLM_PREC_BF16;
    if (c0->g_mode == 2) {
        if (bf) return run<2, __nv_bfloat16, false, true>(c0, m[4], m[4], m[5], m[5], Ag, b, c0->sm_count);
        return run<2, __half, false, true>(c0, m[4], m[4], m[5], m[5], Ag, b, c0->sm_count);
    }
    if (bf) return run<1, __nv_bfloat16, false, true>(c0, m[4], m[4], m[5], m[5], Ag, b, c0->sm_count);
    return run<1, __half, false, true>(c0, m[4], m[4], m[5], m[5], Ag, b, c0->sm_count);
}

// ---- autotuner of the E X^T tile shape: row tile (256 or 128) x bin split (units per SM) ----
//
// Candidates are timed with CUDA events on the context's stream, on its current E and X; the choice is
// cached per (precision, n, n_bins, SM count) for the process.
namespace {
struct TuneKey {
    int prec, n, sms;
    int64_t T;
    bool operator==(const TuneKey& o) const { return prec == o.prec && n == o.n && sms == o.sms && T == o.T; }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, std::pair<int, int>>> g_tune_cache;  // key -> (mode, nsplit)
}  // namespace

int tc_autotune(glm_ctx* c, glm_tune_report_t* rep) {
    const TuneKey key{(int)c->pb.prec, c->pb.n, c->sm_count, c->pb.T};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& kv : g_tune_cache)
            if (kv.first == key) {
                c->g_mode = kv.second.first;
                c->g_nsplit = kv.second.second;
                if (rep) {
                    rep->mode = c->g_mode;
                    rep->nsplit = c->g_nsplit;
                    rep->cached = 1;
                }
                return GLM_OK;
            }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GLM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GLM_ERR_CUDA;
    }
    int best_mode = 1, best_ns = tc_nsplit_for(c, 1, 4), n_cand = 0;
    float best_ms = 3.0e38f;
    const int upms[] = {1, 2, 4, TUNE_UPM_MAX};
    int rc = GLM_OK;
    for (int mode = 1; mode <= 2 && !rc; ++mode)
        for (int upm : upms) {
            const int ns = tc_nsplit_for(c, mode, upm);
            cudaError_t e = run_products_as(c, c->tmap[5], mode, ns, grad_ksteps(c));  // warm-up
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run_products_as(c, c->tmap[5], mode, ns, grad_ksteps(c));
            if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                rc = GLM_ERR_CUDA;
                break;
            }
            ++n_cand;
            if (ms < best_ms) {
                best_ms = ms;
                best_mode = mode;
                best_ns = ns;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    c->g_mode = best_mode;
    c->g_nsplit = best_ns;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tune_cache.size() > 4096) g_tune_cache.clear();
        g_tune_cache.push_back({key, {best_mode, best_ns}});
    }
    if (rep) {
        rep->mode = best_mode;
        rep->nsplit = best_ns;
        rep->cached = 0;
        rep->candidates = n_cand;
        rep->best_ms = best_ms / 2.0f;
    }
    return GLM_OK;
}

// The batched E X^T launch tuned as a whole: one row-tile mode for all problems (one kernel), each problem's
// splits for a common units-per-SM target.  dev_g / host_g: the batch descriptor (device / host image),
// left holding the choice.
int tc_autotune_batch(glm_ctx* const* cs, int np, void* dev_g, void* host_g) {
    glm_ctx* c0 = cs[0];
    TcBatch* bg = static_cast<TcBatch*>(host_g);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return GLM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return GLM_ERR_CUDA;
    }
    auto set = [&](int mode, int upm) -> cudaError_t {
        for (int p = 0; p < np; ++p) {
            cs[p]->g_mode = mode;
            cs[p]->g_nsplit = tc_nsplit_for(cs[p], mode, upm);
            bg->args[p] = batch_grad_args(cs[p], mode, cs[p]->g_nsplit);
        }
        return cudaMemcpy(dev_g, host_g, sizeof(TcBatch), cudaMemcpyHostToDevice);
    };
    int best_mode = 1, best_upm = 4;
    float best_ms = 3.0e38f;
    const int upms[] = {1, 2, 4, TUNE_UPM_MAX};
    cudaError_t e = cudaSuccess;
    for (int mode = 1; mode <= 2 && e == cudaSuccess; ++mode)
        for (int upm : upms) {
            float ms = 0.f;
            e = set(mode, upm);
            if (e == cudaSuccess) e = launch_tc_grad_batch(c0, dev_g);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, c0->stream);
            for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = launch_tc_grad_batch(c0, dev_g);
            if (e == cudaSuccess) e = cudaEventRecord(e1, c0->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            if (ms < best_ms) {
                best_ms = ms;
                best_mode = mode;
                best_upm = upm;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = set(best_mode, best_upm);
    return e == cudaSuccess ? GLM_OK : GLM_ERR_CUDA;
}

// E X^T of problem p in the batched launch is skipped while *counts[p] == 0 (counts: device ints).
void tc_batch_set_grad_counts(void* host_g, int np, const int* const* counts) {
    TcBatch* bg = static_cast<TcBatch*>(host_g);
    for (int p = 0; p < np; ++p) bg->m_dev[p] = counts[p];
}

}  // namespace glm
