// Smolyak sparse-grid quadrature on a box (host code; Sec. 3.3.4, Eq. intpoly).
//
// Combination form of the total-degree Smolyak rule built from 1-D Gauss-Legendre
// rules with m(l) = l + 1 points, l >= 0:
//   Q_L = sum_{L-d+1 <= |l| <= L} (-1)^(L-|l|) C(d-1, L-|l|) Q_{m(l_1)} x ... x Q_{m(l_d)},
// nodes that coincide in different tensor grids are merged and their weights
// summed.  Weights are for the uniform probability measure on the box (sum 1);
// sparse-grid weights can be negative.  Gauss-Legendre nodes come from Newton's
// iteration on the three-term recurrence of the Legendre polynomials.
#include <cmath>
#include <cstdint>
#include <map>
#include <vector>

#include "../../include/oed.h"

namespace {

struct Rule {
    std::vector<double> x, w;
};

Rule gauss_legendre(int n)
{
    Rule r;
    r.x.resize(n);
    r.w.resize(n);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; i++) {
        double x = std::cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= n; k++) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = (n == 0) ? 1.0 : (n == 1 ? x : p1);
            const double pm = (n == 1) ? 1.0 : p0;
            dp = n * (x * pn - pm) / (x * x - 1.0);
            const double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= n; k++) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        const double pn = (n == 1) ? x : p1, pm = (n == 1) ? 1.0 : p0;
        dp = n * (x * pn - pm) / (x * x - 1.0);
        r.x[n - 1 - i] = (std::fabs(x) < 1e-15) ? 0.0 : x;
        r.w[n - 1 - i] = 1.0 / ((1.0 - x * x) * dp * dp);   // 2/(...) on [-1,1], /2 for the mean
    }
    if (n == 1) {
        r.x[0] = 0.0;
        r.w[0] = 1.0;
    }
    return r;
}

double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double c = 1.0;
    for (int i = 1; i <= k; i++) c = c * (n - k + i) / i;
    return c;
}

struct Acc {
    std::vector<double> x;
    double w;
};

void tensor(const std::vector<Rule> &rules, const std::vector<int> &l, double coef,
            std::map<std::vector<long long>, Acc> &acc)
{
    const int d = (int)l.size();
    std::vector<int> idx(d, 0);
    std::vector<double> x(d);
    std::vector<long long> key(d);
    while (true) {
        double w = coef;
        for (int k = 0; k < d; k++) {
            const Rule &r = rules[l[k]];
            x[k] = r.x[idx[k]];
            w *= r.w[idx[k]];
            key[k] = std::llround(x[k] * 1e11);
        }
        auto it = acc.find(key);
        if (it == acc.end())
            acc.emplace(key, Acc{x, w});
        else
            it->second.w += w;
        int k = d - 1;
        while (k >= 0) {
            if (++idx[k] < (int)rules[l[k]].x.size()) break;
            idx[k] = 0;
            k--;
        }
        if (k < 0) break;
    }
}

void enumerate(int d, int level, int pos, int sum, std::vector<int> &l,
               const std::vector<Rule> &rules, std::map<std::vector<long long>, Acc> &acc)
{
    if (pos == d) {
        if (sum < level - d + 1 || sum > level) return;
        const int q = level - sum;
        const double c = ((q & 1) ? -1.0 : 1.0) * binom(d - 1, q);
        if (c != 0.0) tensor(rules, l, c, acc);
        return;
    }
    for (int v = 0; sum + v <= level; v++) {
        l[pos] = v;
        enumerate(d, level, pos + 1, sum + v, l, rules, acc);
    }
}

}  // namespace

extern "C" int oed_nodes_smolyak(int dim, int level, const double *lo, const double *hi,
                                 int max_nodes, double *theta, double *w, int *count)
{
    if (dim < 1 || dim > 16 || level < 0 || level > 40 || !count) return OED_EINVAL;
    std::vector<Rule> rules(level + 1);
    for (int l = 0; l <= level; l++) rules[l] = gauss_legendre(l + 1);
    std::map<std::vector<long long>, Acc> acc;
    std::vector<int> l(dim, 0);
    enumerate(dim, level, 0, 0, l, rules, acc);
    *count = (int)acc.size();
    if (!theta && !w) return OED_OK;
    if ((int)acc.size() > max_nodes) return OED_ENOMEM;
    int i = 0;
    for (const auto &kv : acc) {
        for (int k = 0; k < dim; k++) {
            const double x = kv.second.x[k];
            const double a = lo ? lo[k] : -1.0, b = hi ? hi[k] : 1.0;
            if (theta) theta[(size_t)i * dim + k] = a + (b - a) * (x + 1.0) * 0.5;
        }
        if (w) w[i] = kv.second.w;
        i++;
    }
    return OED_OK;
}
