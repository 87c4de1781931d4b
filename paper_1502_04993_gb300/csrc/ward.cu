// Ward's minimum-variance hierarchical clustering of neurons by their reconstructed weights (Sec. 3.4.2:
// the paper clusters the connectivity matrix by outgoing weights, its columns, and by incoming weights,
// its rows, to pick out the links of a synfire chain; Ward 1963).
//
//   features   point k = column W[:, k] (outgoing) or row W[k, :] (incoming) of neuron subset[k], FP64
//   distances  D[a][b] = ||x_a - x_b||^2, summed from the differences (no cancellation)
//   merges     nearest-neighbour chain: follow nearest neighbours until two clusters are each other's
//              nearest, merge them (Ward's merges are reducible, so this finds the same merges as the
//              greedy order), with the Lance-Williams update for Ward on squared distances
//                D(s u t, k) = ((n_s + n_k) D(s, k) + (n_t + n_k) D(t, k) - n_k D(s, t)) / (n_s + n_t + n_k)
//              One block walks the chain; its threads share each nearest-neighbour search and update.
//   output     merges sorted by height (sqrt D(s, t)) and relabelled with a union-find into the linkage
//              layout of SciPy (the paper's tool): (id_a, id_b, height, size), new clusters n + s.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "glm_internal.h"

namespace glm {

namespace {

constexpr int WD_T = 1024;

__global__ void ward_features_kernel(const float* __restrict__ W, int32_t n, int by, const int32_t* __restrict__ idx,
                                     int32_t m, double* __restrict__ F) {
    const int64_t total = (int64_t)m * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = e / n, j = e % n;
        const int64_t r = idx[k];
        F[e] = (double)(by == 0 ? W[j * n + r] : W[r * n + j]);
    }
}

// D[a][b] for a tile of 16 x 16 pairs, features staged through shared memory 32 at a time
__global__ void ward_dist_kernel(const double* __restrict__ F, int32_t m, int32_t f, double* __restrict__ D) {
    __shared__ double A[16][33], B[16][33];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int32_t a = blockIdx.y * 16 + ty, b = blockIdx.x * 16 + tx;
    double acc = 0.0;
    for (int32_t j0 = 0; j0 < f; j0 += 32) {
        for (int e = threadIdx.x; e < 16 * 32; e += 256) {
            const int r = e / 32, c = e % 32;
            const int32_t ra = blockIdx.y * 16 + r, rb = blockIdx.x * 16 + r;
            A[r][c] = (ra < m && j0 + c < f) ? F[(int64_t)ra * f + j0 + c] : 0.0;
            B[r][c] = (rb < m && j0 + c < f) ? F[(int64_t)rb * f + j0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < 32; ++c) {
            const double d = A[ty][c] - B[tx][c];
            acc = fma(d, d, acc);
        }
        __syncthreads();
    }
    if (a < m && b < m) D[(int64_t)a * m + b] = acc;
}

struct WardOut {
    int32_t* ms;      // [m - 1] slot of one merged cluster
    int32_t* mt;      // [m - 1] slot of the other (the merged cluster stays there)
    double* md2;      // [m - 1] D(s, t) at the merge
    int32_t* mcount;  // [1] merges made
    int* flag;        // [1] set when the walk exceeded its step bound
};

// One block: the nearest-neighbour chain over the m points, D updated in place (row and column of the
// merged cluster).  Work per step: one argmin over the active clusters (strided + warp shuffles), and
// per merge one Lance-Williams pass.  At most 4 m + 16 steps (a chain walk takes fewer than 3 m).
__global__ void __launch_bounds__(WD_T) ward_chain_kernel(double* __restrict__ D, int32_t m,
                                                          uint8_t* __restrict__ active, double* __restrict__ csize,
                                                          int32_t* __restrict__ chain, WardOut out) {
    __shared__ double s_val[WD_T / 32];
    __shared__ int32_t s_idx[WD_T / 32];
    __shared__ int32_t s_len, s_next, s_merges, s_stop;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int32_t k = tid; k < m; k += WD_T) {
        active[k] = 1;
        csize[k] = 1.0;
    }
    if (tid == 0) {
        s_len = 0;
        s_merges = 0;
        s_stop = 0;
        s_next = 0;  // lowest slot not yet retired, to start a new chain
    }
    __syncthreads();
    const int64_t max_steps = 4 * (int64_t)m + 16;
    for (int64_t step = 0; step < max_steps; ++step) {
        if (s_merges >= m - 1) break;
        if (tid == 0 && s_len == 0) {
            while (!active[s_next]) ++s_next;
            chain[0] = s_next;
            s_len = 1;
        }
        __syncthreads();
        const int32_t a = chain[s_len - 1];
        const int32_t prev = s_len > 1 ? chain[s_len - 2] : -1;
        // nearest active neighbour of a; ties go to the previous chain element, then to the lower slot
        double best = INFINITY;
        int32_t bi = INT32_MAX;
        for (int32_t k = tid; k < m; k += WD_T) {
            if (k == a || !active[k]) continue;
            const double v = D[(int64_t)a * m + k];
            const bool better = v < best || (v == best && (k == prev || (bi != prev && k < bi)));
            if (better) {
                best = v;
                bi = k;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, off);
            const int32_t oi = __shfl_down_sync(0xffffffffu, bi, off);
            if (ov < best || (ov == best && (oi == prev || (bi != prev && oi < bi)))) {
                best = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_val[wid] = best;
            s_idx[wid] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < WD_T / 32; ++w) {
                const double ov = s_val[w];
                const int32_t oi = s_idx[w];
                if (ov < best || (ov == best && (oi == prev || (bi != prev && oi < bi)))) {
                    best = ov;
                    bi = oi;
                }
            }
            s_idx[0] = bi;
        }
        __syncthreads();
        const int32_t b = s_idx[0];
        if (b == INT32_MAX) {  // no other active cluster: cannot happen before m - 1 merges
            if (tid == 0) s_stop = 1;
            __syncthreads();
            break;
        }
        if (b != prev) {
            // the chain holds distinct clusters; a longer one means the distances broke reducibility
            if (s_len >= m) {
                if (tid == 0) s_stop = 1;
                __syncthreads();
                break;
            }
            __syncthreads();
            if (tid == 0) chain[s_len++] = b;
            __syncthreads();
            continue;
        }
        // a and prev are each other's nearest: merge them into slot prev (its nearest-neighbour
        // relations are the ones kept on the chain)
        const int32_t s = a, t = prev;
        const double dst = D[(int64_t)s * m + t], ns = csize[s], nt = csize[t];
        for (int32_t k = tid; k < m; k += WD_T) {
            if (k == s || k == t || !active[k]) continue;
            const double nk = csize[k];
            const double v = ((ns + nk) * D[(int64_t)s * m + k] + (nt + nk) * D[(int64_t)t * m + k] - nk * dst) /
                             (ns + nt + nk);
            D[(int64_t)t * m + k] = v;
            D[(int64_t)k * m + t] = v;
        }
        __syncthreads();
        if (tid == 0) {
            const int32_t q = s_merges;
            out.ms[q] = s;
            out.mt[q] = t;
            out.md2[q] = dst;
            active[s] = 0;
            csize[t] = ns + nt;
            s_merges = q + 1;
            s_len -= 2;
        }
        __syncthreads();
    }
    if (tid == 0) {
        *out.mcount = s_merges;
        if (s_merges < m - 1 || s_stop) *out.flag = 1;
    }
}

}  // namespace

}  // namespace glm

using namespace glm;

extern "C" int glm_ward(glm_ctx* c, const float* W_dev, int32_t n, int32_t by, const int32_t* subset_host, int32_t m,
                        double* Z_host) {
    if (!c) return GLM_ERR_INVALID_ARG;
    if (!W_dev || n < 1 || (by != 0 && by != 1) || !Z_host) return set_error(c, GLM_ERR_INVALID_ARG, "bad arguments");
    if (!subset_host) m = n;
    if (m < 2 || m > n) return set_error(c, GLM_ERR_INVALID_ARG, "need 2 <= m <= n points");
    std::vector<int32_t> idx(m);
    for (int32_t k = 0; k < m; ++k) {
        idx[k] = subset_host ? subset_host[k] : k;
        if (idx[k] < 0 || idx[k] >= n) return set_error(c, GLM_ERR_INVALID_ARG, "subset index outside [0, n)");
    }
    cudaStream_t st = c->stream;
    int32_t *d_idx = nullptr, *ms = nullptr, *mt = nullptr, *mcount = nullptr, *chain = nullptr;
    double *F = nullptr, *D = nullptr, *md2 = nullptr, *csize = nullptr;
    uint8_t* active = nullptr;
    int* flag = nullptr;
    auto cleanup = [&](int rc) {
        cudaFree(d_idx);
        cudaFree(ms);
        cudaFree(mt);
        cudaFree(mcount);
        cudaFree(chain);
        cudaFree(F);
        cudaFree(D);
        cudaFree(md2);
        cudaFree(csize);
        cudaFree(active);
        cudaFree(flag);
        return rc;
    };
    const size_t mm = (size_t)m * m;
    if (cudaMalloc(&d_idx, sizeof(int32_t) * m) != cudaSuccess || cudaMalloc(&F, sizeof(double) * (size_t)m * n) != cudaSuccess ||
        cudaMalloc(&D, sizeof(double) * mm) != cudaSuccess || cudaMalloc(&ms, sizeof(int32_t) * m) != cudaSuccess ||
        cudaMalloc(&mt, sizeof(int32_t) * m) != cudaSuccess || cudaMalloc(&md2, sizeof(double) * m) != cudaSuccess ||
        cudaMalloc(&mcount, sizeof(int32_t)) != cudaSuccess || cudaMalloc(&chain, sizeof(int32_t) * (m + 1)) != cudaSuccess ||
        cudaMalloc(&csize, sizeof(double) * m) != cudaSuccess || cudaMalloc(&active, m) != cudaSuccess ||
        cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return cleanup(set_error(c, GLM_ERR_OOM, "Ward clustering buffers"));
    }
    cudaError_t e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const int64_t tot = (int64_t)m * n;
        const unsigned g = (unsigned)std::min<int64_t>((tot + 255) / 256, (int64_t)c->sm_count * 16);
        ward_features_kernel<<<g, 256, 0, st>>>(W_dev, n, by, d_idx, m, F);
        dim3 grid((m + 15) / 16, (m + 15) / 16);
        ward_dist_kernel<<<grid, 256, 0, st>>>(F, m, n, D);
        WardOut o{ms, mt, md2, mcount, flag};
        ward_chain_kernel<<<1, WD_T, 0, st>>>(D, m, active, csize, chain, o);
        e = cudaGetLastError();
        c->launches += 3;
    }
    std::vector<int32_t> hs(m - 1), ht(m - 1);
    std::vector<double> hd(m - 1);
    int hflag = 0, hcount = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), ms, sizeof(int32_t) * (m - 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ht.data(), mt, sizeof(int32_t) * (m - 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), md2, sizeof(double) * (m - 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hcount, mcount, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cleanup(set_error(c, GLM_ERR_CUDA, cudaGetErrorString(e)));
    }
    if (hflag || hcount != m - 1) return cleanup(set_error(c, GLM_ERR_NONFINITE, "Ward merge walk did not complete"));
    // merges by height (stable), then union-find labels: the cluster made by sorted merge q is m + q
    std::vector<int32_t> order(m - 1);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return hd[x] < hd[y]; });
    std::vector<int32_t> parent(2 * (size_t)m - 1), size(2 * (size_t)m - 1, 1);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (int32_t q = 0; q < m - 1; ++q) {
        const int32_t r = order[q];
        int32_t x = find(hs[r]), y = find(ht[r]);
        if (x > y) std::swap(x, y);
        const int32_t id = m + q;
        parent[x] = id;
        parent[y] = id;
        size[id] = size[x] + size[y];
        Z_host[4 * q + 0] = x;
        Z_host[4 * q + 1] = y;
        Z_host[4 * q + 2] = std::sqrt(std::max(hd[r], 0.0));
        Z_host[4 * q + 3] = size[id];
    }
    return cleanup(GLM_OK);
}

extern "C" int glm_ward_cut(const double* Z, int32_t m, int32_t k, int32_t* labels) {
    if (!Z || !labels || m < 1 || k < 1 || k > m) return GLM_ERR_INVALID_ARG;
    std::vector<int32_t> parent(2 * (size_t)m - 1);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (int32_t q = 0; q < m - k; ++q) {
        const int32_t a = (int32_t)Z[4 * q], b = (int32_t)Z[4 * q + 1];
        if (a < 0 || b < 0 || a >= m + q || b >= m + q) return GLM_ERR_INVALID_ARG;
        parent[find(a)] = m + q;
        parent[find(b)] = m + q;
    }
    std::vector<int32_t> root_label(2 * (size_t)m - 1, -1);
    int32_t next = 0;
    for (int32_t i = 0; i < m; ++i) {
        const int32_t r = find(i);
        if (root_label[r] < 0) root_label[r] = next++;
        labels[i] = root_label[r];
    }
    return GLM_OK;
}
