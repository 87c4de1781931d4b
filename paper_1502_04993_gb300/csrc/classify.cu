// glm_classify: label reconstructed weights as inhibitory (-1), absent (0) or excitatory (+1) and score
// them against a ground truth.  Host code (the work is O(n^2) per EM step, far from the hot path).
//
// The paper classifies the off-diagonal weights J_ij, i != j (self-connections are treated apart,
// Sec. 3.1) with a 3-component Gaussian mixture fitted by expectation-maximisation (Sec. 3.1) or with
// 3-means (Sec. 3.3, App. C.2).  Errors are reported as in Table 2: per class the false positives,
// false negatives and the misclassifications that contradict Dale's law for the presynaptic neuron.
// Choices where the paper is silent: 3-means starts from the 1st, 50th and 99th percentiles (linear
// interpolation between order statistics) and iterates until no assignment changes; the mixture starts
// from the 3-means clusters, floors variances at 1e-12 and stops when the relative change of its
// log-likelihood is <= tol; ties go to the component whose centre is nearest zero.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "glm.h"

namespace {

double percentile_sorted(const std::vector<double>& v, double p) {
    const double pos = p / 100.0 * (double)(v.size() - 1);
    const size_t lo = (size_t)std::floor(pos);
    const size_t hi = std::min(lo + 1, v.size() - 1);
    const double f = pos - (double)lo;
    return v[lo] + f * (v[hi] - v[lo]);
}

int nearest(double x, const double c[3]) {
    int best = 0;
    double bd = std::fabs(x - c[0]);
    for (int k = 1; k < 3; ++k) {
        const double d = std::fabs(x - c[k]);
        if (d < bd || (d == bd && std::fabs(c[k]) < std::fabs(c[best]))) {
            best = k;
            bd = d;
        }
    }
    return best;
}

}  // namespace

extern "C" int glm_classify(const double* W, int32_t n, const glm_classify_opts_t* opts, int8_t* labels,
                            const int8_t* truth, const int8_t* types, glm_classify_report_t* rep) {
    if (!W || n < 2 || !labels) return GLM_ERR_INVALID_ARG;
    glm_classify_opts_t o;
    o.method = GLM_CLASSIFY_GMM;
    o.max_iter = 1000;
    o.tol = 1e-12;
    if (opts) o = *opts;
    if (o.method != GLM_CLASSIFY_GMM && o.method != GLM_CLASSIFY_KMEANS) return GLM_ERR_INVALID_ARG;
    if (o.max_iter < 1 || !(o.tol >= 0)) return GLM_ERR_INVALID_ARG;
    const size_t N = (size_t)n * (size_t)(n - 1);
    std::vector<double> x;
    x.reserve(N);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j)
            if (i != j) {
                const double w = W[(size_t)i * n + j];
                if (!std::isfinite(w)) return GLM_ERR_NONFINITE;
                x.push_back(w);
            }
    std::vector<double> sorted(x);
    std::sort(sorted.begin(), sorted.end());
    double c[3] = {percentile_sorted(sorted, 1.0), percentile_sorted(sorted, 50.0), percentile_sorted(sorted, 99.0)};
    std::vector<int8_t> a(N);
    for (size_t k = 0; k < N; ++k) a[k] = (int8_t)nearest(x[k], c);
    int iters = 0;
    for (int it = 0; it < o.max_iter; ++it) {
        double sum[3] = {0, 0, 0};
        size_t cnt[3] = {0, 0, 0};
        for (size_t k = 0; k < N; ++k) {
            sum[a[k]] += x[k];
            cnt[a[k]]++;
        }
        for (int q = 0; q < 3; ++q)
            if (cnt[q]) c[q] = sum[q] / (double)cnt[q];
        bool changed = false;
        for (size_t k = 0; k < N; ++k) {
            const int8_t b = (int8_t)nearest(x[k], c);
            if (b != a[k]) {
                a[k] = b;
                changed = true;
            }
        }
        iters = it + 1;
        if (!changed) break;
    }
    // order clusters by centre
    int order[3] = {0, 1, 2};
    std::sort(order, order + 3, [&](int p, int q) { return c[p] < c[q]; });
    int rank[3];
    for (int r = 0; r < 3; ++r) rank[order[r]] = r;
    double mean[3], var[3] = {0, 0, 0}, weight[3] = {0, 0, 0};
    for (int r = 0; r < 3; ++r) mean[r] = c[order[r]];
    for (size_t k = 0; k < N; ++k) a[k] = (int8_t)rank[a[k]];
    double loglik = 0.0;
    if (o.method == GLM_CLASSIFY_GMM) {
        size_t cnt[3] = {0, 0, 0};
        for (size_t k = 0; k < N; ++k) {
            const int q = a[k];
            cnt[q]++;
            var[q] += (x[k] - mean[q]) * (x[k] - mean[q]);
        }
        for (int q = 0; q < 3; ++q) {
            weight[q] = std::max((double)cnt[q] / (double)N, 1e-300);
            var[q] = std::max(cnt[q] ? var[q] / (double)cnt[q] : 0.0, 1e-12);
        }
        double prev = 0.0;
        bool have_prev = false;
        std::vector<double> resp(3 * N);
        for (int it = 0; it < o.max_iter; ++it) {
            // E step
            double ll = 0.0;
            double lw[3], lv[3];
            for (int q = 0; q < 3; ++q) {
                lw[q] = std::log(weight[q]);
                lv[q] = 0.5 * std::log(2.0 * M_PI * var[q]);
            }
            for (size_t k = 0; k < N; ++k) {
                double lp[3], mx = -INFINITY;
                for (int q = 0; q < 3; ++q) {
                    const double d = x[k] - mean[q];
                    lp[q] = lw[q] - lv[q] - 0.5 * d * d / var[q];
                    mx = std::max(mx, lp[q]);
                }
                double s = 0.0;
                for (int q = 0; q < 3; ++q) s += std::exp(lp[q] - mx);
                const double lse = mx + std::log(s);
                ll += lse;
                for (int q = 0; q < 3; ++q) resp[3 * k + q] = std::exp(lp[q] - lse);
            }
            // M step
            double nk[3] = {0, 0, 0}, sx[3] = {0, 0, 0};
            for (size_t k = 0; k < N; ++k)
                for (int q = 0; q < 3; ++q) {
                    nk[q] += resp[3 * k + q];
                    sx[q] += resp[3 * k + q] * x[k];
                }
            for (int q = 0; q < 3; ++q) mean[q] = sx[q] / std::max(nk[q], 1e-300);
            double sv[3] = {0, 0, 0};
            for (size_t k = 0; k < N; ++k)
                for (int q = 0; q < 3; ++q) {
                    const double d = x[k] - mean[q];
                    sv[q] += resp[3 * k + q] * d * d;
                }
            for (int q = 0; q < 3; ++q) {
                weight[q] = std::max(nk[q] / (double)N, 1e-300);
                var[q] = std::max(sv[q] / std::max(nk[q], 1e-300), 1e-12);
            }
            loglik = ll;
            iters = it + 1;
            if (have_prev && std::fabs(ll - prev) <= o.tol * std::fabs(ll)) break;
            prev = ll;
            have_prev = true;
        }
        // components sorted by mean, then posterior argmax (ties to the centre nearest zero)
        int ord[3] = {0, 1, 2};
        std::sort(ord, ord + 3, [&](int p, int q) { return mean[p] < mean[q]; });
        double m2[3], v2[3], w2[3];
        for (int r = 0; r < 3; ++r) {
            m2[r] = mean[ord[r]];
            v2[r] = var[ord[r]];
            w2[r] = weight[ord[r]];
        }
        for (int r = 0; r < 3; ++r) {
            mean[r] = m2[r];
            var[r] = v2[r];
            weight[r] = w2[r];
        }
        for (size_t k = 0; k < N; ++k) {
            int best = 0;
            double bl = -INFINITY;
            for (int q = 0; q < 3; ++q) {
                const double d = x[k] - mean[q];
                const double lp = std::log(weight[q]) - 0.5 * std::log(2.0 * M_PI * var[q]) - 0.5 * d * d / var[q];
                if (lp > bl || (lp == bl && std::fabs(mean[q]) < std::fabs(mean[best]))) {
                    bl = lp;
                    best = q;
                }
            }
            a[k] = (int8_t)best;
        }
    }
    // labels
    size_t k = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t j = 0; j < n; ++j) {
            if (i == j) {
                labels[(size_t)i * n + j] = 0;
                continue;
            }
            labels[(size_t)i * n + j] = (int8_t)(a[k++] - 1);
        }
    if (rep) {
        std::memset(rep, 0, sizeof(*rep));
        for (int q = 0; q < 3; ++q) {
            rep->centers[q] = mean[q];
            rep->weights[q] = weight[q];
            rep->variances[q] = var[q];
        }
        rep->iterations = iters;
        rep->loglik = loglik;
        if (truth) {
            for (int32_t i = 0; i < n; ++i)
                for (int32_t j = 0; j < n; ++j) {
                    if (i == j) continue;
                    const int l = labels[(size_t)i * n + j], t = truth[(size_t)i * n + j];
                    if (l == t) continue;
                    rep->errors++;
                    rep->fp[l + 1]++;
                    rep->fn[t + 1]++;
                    if (types && l != 0 && types[j] == -l) rep->nd[l + 1]++;
                }
            rep->mer = (double)rep->errors / (double)N;
            rep->mer_n2 = (double)rep->errors / ((double)n * (double)n);
        }
    }
    return GLM_OK;
}
