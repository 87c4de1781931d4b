/*
 * Seeded synthetic inputs for the GLM connectivity-reconstruction path.
 *
 * This module only MAKES data: a random balanced E/I network (Dale's law by
 * presynaptic column, as in the validation design of Sec. 3.1 / Fig. 2) and a
 * spike raster simulated from the discrete-time version of the model
 * (Eq. 3-5 on a grid of width dt with a delay of one bin, Eq. 8 as the
 * recursion of the membrane potential).  It is consumed identically by the
 * FP64 oracle and by the CUDA library; neither of them calls into it for any
 * of its own arithmetic.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11), implemented here from its
 * published definition.  Every draw is addressed by a counter, so results do
 * not depend on the thread count.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC glm_synth.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

/* stream tags carried in the last counter word */
#define TAG_CONN 0x434F4E4Eu /* "CONN" */
#define TAG_SPK 0x53504B53u  /* "SPKS" */
#define TAG_PERM 0x5045524Du /* "PERM" */

void synth_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

static inline double u01(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

static inline void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t c, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {a, b, c, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    synth_philox4x32_10(ctr, key, out);
}

/*
 * Random balanced network.  Canonical ids 0..n_exc-1 are excitatory, the rest
 * inhibitory.  For every ordered pair i != j a connection j -> i exists with
 * probability p; its weight is +w_exc if j is excitatory, -w_inh otherwise.
 * Every diagonal entry is w_self (the refractory self-connection of Sec. 3.1;
 * 0 for none).
 * Optional synfire chain: syn_groups groups of syn_size excitatory neurons
 * (canonical E ids [g*syn_size, (g+1)*syn_size)); every neuron of group g+1
 * receives weight +w_syn from every neuron of group g, replacing the random
 * entry.  Optional shuffle relabels ids by a Philox-driven Fisher-Yates
 * permutation.
 *
 * W is row-major n*n, W[i*n + j] = weight of the connection j -> i.
 * types[i] = +1 (excitatory) or -1 (inhibitory).  b is not drawn here.
 */
int synth_network(int32_t n, int32_t n_exc, double p, double w_exc, double w_inh, double w_self,
                  int32_t syn_groups, int32_t syn_size, double w_syn, int32_t shuffle, uint64_t seed, double* W,
                  int8_t* types) {
    if (n <= 0 || n_exc < 0 || n_exc > n || !(p >= 0.0 && p <= 1.0) || !W || !types) return -1;
    if (syn_groups < 0 || syn_size < 0 || (int64_t)syn_groups * syn_size > n_exc) return -1;
    double* Wc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!Wc || !perm) {
        free(Wc);
        free(perm);
        return -2;
    }
#pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = 0; j < n; ++j) {
            double w = w_self;
            if (i != j) {
                w = 0.0;
                uint32_t o[4];
                draw(seed, (uint32_t)i, (uint32_t)j, 0u, TAG_CONN, o);
                if (u01(o[0]) < p) w = (j < n_exc) ? w_exc : -w_inh;
            }
            Wc[(size_t)i * n + j] = w;
        }
    }
    for (int32_t g = 0; g + 1 < syn_groups; ++g) {
        for (int32_t a = 0; a < syn_size; ++a) {
            int32_t i = (g + 1) * syn_size + a;
            for (int32_t c = 0; c < syn_size; ++c) {
                int32_t j = g * syn_size + c;
                Wc[(size_t)i * n + j] = w_syn;
            }
        }
    }
    for (int32_t k = 0; k < n; ++k) perm[k] = k;
    if (shuffle) {
        for (int32_t k = n - 1; k > 0; --k) {
            uint32_t o[4];
            draw(seed, (uint32_t)k, 0u, 0u, TAG_PERM, o);
            int32_t r = (int32_t)floor(u01(o[0]) * (double)(k + 1));
            if (r > k) r = k;
            int32_t tmp = perm[k];
            perm[k] = perm[r];
            perm[r] = tmp;
        }
    }
    /* canonical index c gets id perm[c] */
    for (int32_t ci = 0; ci < n; ++ci) {
        int32_t i = perm[ci];
        types[i] = (int8_t)((ci < n_exc) ? 1 : -1);
        for (int32_t cj = 0; cj < n; ++cj) W[(size_t)i * n + perm[cj]] = Wc[(size_t)ci * n + cj];
    }
    free(Wc);
    free(perm);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Spike simulation on the grid (delay of one bin for every pair, self
 * included):
 *   V_i[0] = 0,  V_i[t] = a V_i[t-1] + sum_j W_ij S_j[t-1],   a = exp(-dt/tau)
 *   S_i[t] = 1  iff  u_i[t] < min(exp(b_i + V_i[t]), rate_cap) * dt
 * u_i[t] is word (t mod 4) of Philox(ctr = (i, t/4, t/2^34, SPKS)).
 * At most one spike per neuron and bin.
 * ------------------------------------------------------------------------- */
typedef struct {
    int64_t q;
    int32_t n;
    int64_t* offs;
    int32_t* bins;
} synth_sim_t;

typedef struct {
    int32_t* t;
    int32_t* i;
    int64_t len, cap;
} evbuf_t;

static int evbuf_push(evbuf_t* e, int32_t t, int32_t i) {
    if (e->len == e->cap) {
        int64_t nc = e->cap ? e->cap * 2 : 4096;
        int32_t* nt = (int32_t*)realloc(e->t, sizeof(int32_t) * (size_t)nc);
        if (!nt) return -1;
        e->t = nt;
        int32_t* ni = (int32_t*)realloc(e->i, sizeof(int32_t) * (size_t)nc);
        if (!ni) return -1;
        e->i = ni;
        e->cap = nc;
    }
    e->t[e->len] = t;
    e->i[e->len] = i;
    e->len++;
    return 0;
}

void* synth_simulate(int32_t n, int64_t n_bins, double dt, double tau, const double* W, const double* b,
                     double rate_cap, uint64_t seed, int32_t n_threads) {
    if (n <= 0 || n_bins <= 0 || n_bins > 2147483647LL || !(dt > 0) || !(tau > 0) || !W || !b) return NULL;
    const double a = exp(-dt / tau);
    int nt = 1;
#ifdef _OPENMP
    nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#endif
    if (nt > n) nt = n;
    /* column-major copy so that the input of one presynaptic neuron is contiguous */
    double* Wt = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
    double* V = (double*)calloc((size_t)n, sizeof(double));
    uint32_t* rng = (uint32_t*)malloc(sizeof(uint32_t) * 4 * (size_t)n);
    int32_t* lists = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)n); /* [parity][thread-block of ids] */
    int32_t* counts = (int32_t*)calloc(2 * (size_t)nt, sizeof(int32_t));
    evbuf_t* ev = (evbuf_t*)calloc((size_t)nt, sizeof(evbuf_t));
    int failed = 0;
    if (!Wt || !V || !rng || !lists || !counts || !ev) failed = 1;
    if (!failed) {
        for (int32_t i = 0; i < n; ++i)
            for (int32_t j = 0; j < n; ++j) Wt[(size_t)j * n + i] = W[(size_t)i * n + j];
    }
    if (!failed) {
#pragma omp parallel num_threads(nt)
        {
            int tid = 0;
#ifdef _OPENMP
            tid = omp_get_thread_num();
#endif
            const int32_t lo = (int32_t)(((int64_t)n * tid) / nt);
            const int32_t hi = (int32_t)(((int64_t)n * (tid + 1)) / nt);
            for (int64_t t = 0; t < n_bins; ++t) {
                const int par = (int)(t & 1);
                int32_t* mine = lists + (size_t)par * n + lo;
                int32_t cnt = 0;
                for (int32_t i = lo; i < hi; ++i) {
                    double v = V[i];
                    if (t > 0) {
                        v = a * v;
                        /* inputs from the spikes of bin t-1, in ascending presynaptic id */
                        for (int th = 0; th < nt; ++th) {
                            const int32_t plo = (int32_t)(((int64_t)n * th) / nt);
                            const int32_t* pl = lists + (size_t)(1 - par) * n + plo;
                            const int32_t pc = counts[2 * th + (1 - par)];
                            for (int32_t k = 0; k < pc; ++k) v += Wt[(size_t)pl[k] * n + i];
                        }
                    }
                    V[i] = v;
                    if ((t & 3) == 0) {
                        uint32_t o[4];
                        draw(seed, (uint32_t)i, (uint32_t)(t >> 2), (uint32_t)(t >> 34), TAG_SPK, o);
                        memcpy(rng + 4 * (size_t)i, o, sizeof o);
                    }
                    /* u >= rate_cap*dt can never spike, whatever the rate: skip the exp then */
                    const double u = u01(rng[4 * (size_t)i + (t & 3)]);
                    int spk = 0;
                    if (u < rate_cap * dt) {
                        double lam = exp(b[i] + v);
                        if (!(lam < rate_cap)) lam = rate_cap;
                        spk = u < lam * dt;
                    }
                    if (spk) {
                        mine[cnt++] = i;
                        if (evbuf_push(&ev[tid], (int32_t)t, i)) {
#pragma omp atomic write
                            failed = 1;
                        }
                    }
                }
                counts[2 * tid + par] = cnt;
#pragma omp barrier
            }
        }
    }
    synth_sim_t* res = NULL;
    if (!failed) {
        res = (synth_sim_t*)calloc(1, sizeof(synth_sim_t));
        int64_t q = 0;
        for (int th = 0; th < nt; ++th) q += ev[th].len;
        res->q = q;
        res->n = n;
        res->offs = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
        res->bins = (int32_t*)malloc(sizeof(int32_t) * (size_t)(q > 0 ? q : 1));
        if (!res->offs || !res->bins) {
            free(res->offs);
            free(res->bins);
            free(res);
            res = NULL;
        } else {
            for (int th = 0; th < nt; ++th)
                for (int64_t k = 0; k < ev[th].len; ++k) res->offs[ev[th].i[k] + 1]++;
            for (int32_t i = 0; i < n; ++i) res->offs[i + 1] += res->offs[i];
            int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
            memcpy(fill, res->offs, sizeof(int64_t) * (size_t)n);
            /* each neuron lives in exactly one thread buffer, in time order */
            for (int th = 0; th < nt; ++th)
                for (int64_t k = 0; k < ev[th].len; ++k) res->bins[fill[ev[th].i[k]]++] = ev[th].t[k];
            free(fill);
        }
    }
    for (int th = 0; ev && th < nt; ++th) {
        free(ev[th].t);
        free(ev[th].i);
    }
    free(ev);
    free(counts);
    free(lists);
    free(rng);
    free(V);
    free(Wt);
    return res;
}

int64_t synth_sim_count(const void* h) { return h ? ((const synth_sim_t*)h)->q : -1; }

void synth_sim_copy(const void* h, int64_t* offs, int32_t* bins) {
    const synth_sim_t* s = (const synth_sim_t*)h;
    memcpy(offs, s->offs, sizeof(int64_t) * ((size_t)s->n + 1));
    if (s->q > 0) memcpy(bins, s->bins, sizeof(int32_t) * (size_t)s->q);
}

void synth_sim_free(void* h) {
    synth_sim_t* s = (synth_sim_t*)h;
    if (!s) return;
    free(s->offs);
    free(s->bins);
    free(s);
}
