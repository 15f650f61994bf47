// Dense symmetric eigendecomposition on the host (plan time only):
// A = Q diag(lambda) Q^T for a real symmetric n x n matrix.
//
// Householder reduction to tridiagonal form with the reflections accumulated
// into Q, then implicit symmetric QR steps with the Wilkinson shift and
// deflation on the tridiagonal matrix, the Givens rotations accumulated into Q
// (Golub & Van Loan, Matrix Computations, 4th ed., Algorithms 8.3.1 and
// 8.3.2).  O(n^3); used for the coarsest level of a composite domain, whose
// operator is not separable.
#pragma once

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

namespace pp {

// a: n x n row-major symmetric matrix, overwritten.  On success q holds the
// eigenvectors as columns (q[i * n + j]: component i of eigenvector j) and
// lam the eigenvalues (unsorted).  Returns false when the QR iteration does
// not converge within 30 n sweeps.
inline bool sym_eig(std::vector<double> a, int n, std::vector<double> &q, std::vector<double> &lam) {
    q.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) q[(size_t)i * n + i] = 1.0;
    lam.assign(n, 0.0);
    if (n == 0) return true;
    std::vector<double> v(n), p(n), w(n);
    // Householder: step k zeroes column k below the subdiagonal
    for (int k = 0; k + 2 < n; ++k) {
        const int m0 = k + 1, len = n - m0;
        double sq = 0.0;
        for (int i = 0; i < len; ++i) {
            v[i] = a[(size_t)(m0 + i) * n + k];
            sq += v[i] * v[i];
        }
        const double nx = std::sqrt(sq);
        if (nx == 0.0) continue;
        const double alpha = v[0] >= 0.0 ? -nx : nx;   // H x = alpha e_1
        v[0] -= alpha;
        double vv = 0.0;
        for (int i = 0; i < len; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        const double inv = 1.0 / std::sqrt(vv);
        for (int i = 0; i < len; ++i) v[i] *= inv;   // H = I - 2 v v^T
        // trailing block B <- H B H = B - 2 v u^T - 2 u v^T with p = B v, u = p - (v^T p) v
        for (int i = 0; i < len; ++i) {
            double s = 0.0;
            const double *row = &a[(size_t)(m0 + i) * n + m0];
            for (int j = 0; j < len; ++j) s += row[j] * v[j];
            p[i] = s;
        }
        double kk = 0.0;
        for (int i = 0; i < len; ++i) kk += v[i] * p[i];
        for (int i = 0; i < len; ++i) w[i] = p[i] - kk * v[i];
        for (int i = 0; i < len; ++i) {
            double *row = &a[(size_t)(m0 + i) * n + m0];
            for (int j = 0; j < len; ++j) row[j] -= 2.0 * (v[i] * w[j] + w[i] * v[j]);
        }
        // column k and row k below the subdiagonal
        a[(size_t)m0 * n + k] = a[(size_t)k * n + m0] = alpha;
        for (int i = 1; i < len; ++i) a[(size_t)(m0 + i) * n + k] = a[(size_t)k * n + m0 + i] = 0.0;
        // Q <- Q H on columns m0..n-1
        for (int r = 0; r < n; ++r) {
            double *row = &q[(size_t)r * n + m0];
            double s = 0.0;
            for (int j = 0; j < len; ++j) s += row[j] * v[j];
            s *= 2.0;
            for (int j = 0; j < len; ++j) row[j] -= s * v[j];
        }
    }
    std::vector<double> d(n), e(n, 0.0);   // e[i] = T(i, i+1)
    for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
    for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)i * n + i + 1];
    const double eps = 4.0 * 2.220446049250313e-16;
    int iter = 0, hi = n - 1;
    while (hi > 0) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = 0.0;
        if (++iter > 30 * n) return false;
        // Wilkinson shift from the trailing 2 x 2 block
        const double del = 0.5 * (d[hi - 1] - d[hi]), eh = e[hi - 1];
        const double den = del + (del >= 0.0 ? 1.0 : -1.0) * std::hypot(del, eh);
        const double mu = d[hi] - (den != 0.0 ? eh * eh / den : 0.0);
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            // rotation G in the plane (k, k+1) with (G^T [x z]^T)_(k+1) = 0
            const double r = std::hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? -z / r : 0.0;
            if (k > lo) e[k - 1] = r;
            const double ak = d[k], bk = e[k], dk = d[k + 1];
            d[k] = c * c * ak - 2.0 * c * s * bk + s * s * dk;
            d[k + 1] = s * s * ak + 2.0 * c * s * bk + c * c * dk;
            e[k] = c * s * (ak - dk) + (c * c - s * s) * bk;
            if (k + 1 < hi) {
                z = -s * e[k + 1];   // the bulge T(k, k+2)
                e[k + 1] *= c;
                x = e[k];
            }
            for (int rr = 0; rr < n; ++rr) {
                double *row = &q[(size_t)rr * n];
                const double qk = row[k], q1 = row[k + 1];
                row[k] = c * qk - s * q1;
                row[k + 1] = s * qk + c * q1;
            }
        }
    }
    lam = d;
    return true;
}

// sym_eig with the last kSymEigKept results kept for the process: the plans
// of one problem (the autotuner builds one per candidate schedule, a batch
// may repeat a geometry) factor the same coarsest-level matrix, at about two
// seconds for n = 800.  A result is reused only for a byte-identical input
// matrix, so a hit returns exactly what the factorisation would.
constexpr size_t kSymEigKept = 2;

// Reuses so far (for the tests).
inline size_t &sym_eig_cache_hits() {
    static size_t hits = 0;
    return hits;
}

inline bool sym_eig_cached(const std::vector<double> &a, int n, std::vector<double> &q, std::vector<double> &lam) {
    struct Kept {
        int n;
        std::vector<double> a, q, lam;
    };
    static std::mutex mu;
    static std::vector<Kept> kept;   // least recently used first
    const size_t bytes = (size_t)n * n * sizeof(double);
    if (a.size() != (size_t)n * n) return sym_eig(a, n, q, lam);
    {
        std::lock_guard<std::mutex> lock(mu);
        for (size_t i = 0; i < kept.size(); ++i) {
            if (kept[i].n != n || (bytes && std::memcmp(kept[i].a.data(), a.data(), bytes) != 0)) continue;
            q = kept[i].q;
            lam = kept[i].lam;
            ++sym_eig_cache_hits();
            Kept hit = std::move(kept[i]);
            kept.erase(kept.begin() + (long)i);
            kept.push_back(std::move(hit));
            return true;
        }
    }
    if (!sym_eig(a, n, q, lam)) return false;
    std::lock_guard<std::mutex> lock(mu);
    if (kept.size() >= kSymEigKept) kept.erase(kept.begin());
    kept.push_back(Kept{n, a, q, lam});
    return true;
}

}  // namespace pp
