// Level-symmetric discrete-ordinate sets for 2D problems (host code).
//
// The paper discretises the unit sphere with Gauss-Legendre or S_n sets
// (Sec. 4.1).  The level-symmetric S_n construction: direction cosines
// mu_i^2 = mu_1^2 + (i-1) 2 (1 - 3 mu_1^2)/(n - 2), i = 1..n/2; octant points
// (mu_a, mu_b, mu_c) with a + b + c = n/2 + 2; points that are permutations of
// one another share a weight; the weights solve (in the least-squares sense,
// the system is consistent for n <= 16) the even moment conditions
//   sum w mux^2a muy^2b muz^2c = (2a-1)!!(2b-1)!!(2c-1)!! / (2(a+b+c)+1)!!,
//   a + b + c < n/2, with octant weights summing to 1.
// For 2D the z > 0 hemisphere is kept and its weights doubled (sum = 4 pi).
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "gsis.h"

namespace {

double dfact(int k)
{
    double r = 1.0;
    while (k > 1) {
        r *= k;
        k -= 2;
    }
    return r;
}

double mu1_of(int order)
{
    switch (order) {
        case 4: return std::sqrt((4.0 - std::sqrt(6.4)) / 12.0);   // mu^4 exact with one weight class
        case 6: return 0.2666355;
        case 8: return 0.2182179;
        case 10: return 0.1893213;
        case 12: return 0.1672126;
        case 14: return 0.1519859;
        case 16: return 0.1389568;
        default: return -1.0;
    }
}

// Least squares min ||A x - b|| by modified Gram-Schmidt QR (A is m x n, m >= n).
bool lstsq(std::vector<double> A, int m, int n, std::vector<double> b, std::vector<double>& x)
{
    std::vector<double> R((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < j; ++i) {
            double d = 0.0;
            for (int r = 0; r < m; ++r) d += A[(size_t)r * n + i] * A[(size_t)r * n + j];
            R[(size_t)i * n + j] = d;
            for (int r = 0; r < m; ++r) A[(size_t)r * n + j] -= d * A[(size_t)r * n + i];
        }
        double nn = 0.0;
        for (int r = 0; r < m; ++r) nn += A[(size_t)r * n + j] * A[(size_t)r * n + j];
        nn = std::sqrt(nn);
        if (!(nn > 1e-14)) return false;
        R[(size_t)j * n + j] = nn;
        for (int r = 0; r < m; ++r) A[(size_t)r * n + j] /= nn;
    }
    std::vector<double> qtb(n, 0.0);
    for (int j = 0; j < n; ++j)
        for (int r = 0; r < m; ++r) qtb[j] += A[(size_t)r * n + j] * b[r];
    x.assign(n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
        double v = qtb[j];
        for (int i = j + 1; i < n; ++i) v -= R[(size_t)j * n + i] * x[i];
        x[j] = v / R[(size_t)j * n + j];
    }
    return true;
}

}  // namespace

extern "C" int gsis_quadrature_level_symmetric(int order, double* mu, double* eta, double* w, int* K)
{
    const double m1 = mu1_of(order);
    if (m1 <= 0.0 || !K) return GSIS_ERR_ARG;
    const int n = order / 2;
    const int npts = n * (n + 1) / 2;
    *K = 4 * npts;
    if (!mu && !eta && !w) return GSIS_OK;
    if (!mu || !eta || !w) return GSIS_ERR_ARG;
    const double step = 2.0 * (1.0 - 3.0 * m1 * m1) / (order - 2);
    std::vector<double> lev(n);
    for (int i = 0; i < n; ++i) lev[i] = std::sqrt(m1 * m1 + step * i);
    std::vector<std::array<double, 3>> pts;
    std::vector<std::array<int, 3>> cls;
    for (int a = 1; a <= n; ++a)
        for (int b = 1; b <= n; ++b) {
            const int c = n + 2 - a - b;
            if (c < 1 || c > n) continue;
            pts.push_back({lev[a - 1], lev[b - 1], lev[c - 1]});
            std::array<int, 3> k3 = {a, b, c};
            std::sort(k3.begin(), k3.end());
            cls.push_back(k3);
        }
    std::vector<std::array<int, 3>> ucls = cls;
    std::sort(ucls.begin(), ucls.end());
    ucls.erase(std::unique(ucls.begin(), ucls.end()), ucls.end());
    const int nc = (int)ucls.size();
    std::vector<int> ci(pts.size());
    for (size_t p = 0; p < pts.size(); ++p)
        ci[p] = (int)(std::lower_bound(ucls.begin(), ucls.end(), cls[p]) - ucls.begin());
    std::vector<double> A, rhs;
    int m = 0;
    for (int a = 0; a < n; ++a)
        for (int b = 0; b < n - a; ++b)
            for (int c = 0; c < n - a - b; ++c) {
                std::vector<double> row(nc, 0.0);
                for (size_t p = 0; p < pts.size(); ++p)
                    row[ci[p]] += std::pow(pts[p][0], 2 * a) * std::pow(pts[p][1], 2 * b) *
                                  std::pow(pts[p][2], 2 * c);
                A.insert(A.end(), row.begin(), row.end());
                rhs.push_back(dfact(2 * a - 1) * dfact(2 * b - 1) * dfact(2 * c - 1) /
                              dfact(2 * (a + b + c) + 1));
                ++m;
            }
    std::vector<double> wc;
    if (!lstsq(A, m, nc, rhs, wc)) return GSIS_ERR_ARG;
    for (int pass = 0; pass < 2; ++pass) {   // iterative refinement of the least-squares solution
        std::vector<double> res(m), dw;
        for (int r = 0; r < m; ++r) {
            double v = rhs[r];
            for (int c = 0; c < nc; ++c) v -= A[(size_t)r * nc + c] * wc[c];
            res[r] = v;
        }
        if (!lstsq(A, m, nc, res, dw)) return GSIS_ERR_ARG;
        for (int c = 0; c < nc; ++c) wc[c] += dw[c];
    }
    const double pi = 3.14159265358979323846;
    const int sx[4] = {1, -1, 1, -1}, sy[4] = {1, 1, -1, -1};
    int k = 0;
    for (int qd = 0; qd < 4; ++qd)
        for (size_t p = 0; p < pts.size(); ++p, ++k) {
            mu[k] = sx[qd] * pts[p][0];
            eta[k] = sy[qd] * pts[p][1];
            w[k] = wc[ci[p]] * pi;   // (4 pi / 8) per octant, doubled for z < 0
        }
    return GSIS_OK;
}
