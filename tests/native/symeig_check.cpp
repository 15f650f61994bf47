// CPU check of the plan-time symmetric eigensolver: prints one line per case,
// "<name> <max |A Q - Q L| / max|A|> <max |Q^T Q - I|> <max eigenvalue error or -1>".
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../paper_2609_07172_gb300/csrc/symeig.h"

static uint64_t state = 88172645463325252ull;
static double urand() {   // xorshift64, uniform in [-1, 1)
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return (double)(state >> 11) / 9007199254740992.0 * 2.0 - 1.0;
}

static void report(const char *name, const std::vector<double> &A, int n, const std::vector<double> *exact) {
    std::vector<double> Q, L;
    if (!pp::sym_eig(A, n, Q, L)) {
        printf("%s FAIL FAIL FAIL\n", name);
        return;
    }
    double amax = 0, res = 0, orth = 0, everr = -1;
    for (double v : A) amax = std::max(amax, std::fabs(v));
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0, t = 0;
            for (int k = 0; k < n; ++k) {
                s += A[(size_t)i * n + k] * Q[(size_t)k * n + j];
                t += Q[(size_t)k * n + i] * Q[(size_t)k * n + j];
            }
            res = std::max(res, std::fabs(s - Q[(size_t)i * n + j] * L[j]));
            orth = std::max(orth, std::fabs(t - (i == j ? 1.0 : 0.0)));
        }
    if (exact) {
        std::vector<double> a = L, b = *exact;
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        everr = 0;
        for (int i = 0; i < n; ++i) everr = std::max(everr, std::fabs(a[i] - b[i]));
    }
    printf("%s %.3e %.3e %.3e\n", name, res / (amax > 0 ? amax : 1), orth, everr);
}

int main() {
    {   // random symmetric
        const int n = 60;
        std::vector<double> A((size_t)n * n);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j <= i; ++j) A[(size_t)i * n + j] = A[(size_t)j * n + i] = urand();
        report("random60", A, n, nullptr);
    }
    {   // 1-D Dirichlet Laplacian: eigenvalues 2 - 2 cos(pi j / (n + 1))
        const int n = 40;
        std::vector<double> A((size_t)n * n, 0.0), ex(n);
        for (int i = 0; i < n; ++i) {
            A[(size_t)i * n + i] = 2;
            if (i + 1 < n) A[(size_t)i * n + i + 1] = A[(size_t)(i + 1) * n + i] = -1;
            ex[i] = 2 - 2 * std::cos(M_PI * (i + 1) / (n + 1));
        }
        report("laplace1d", A, n, &ex);
    }
    {   // 2-D Dirichlet Laplacian on a 9 x 7 grid: eigenvalues are sums of the 1-D ones
        const int nx = 9, ny = 7, n = nx * ny;
        std::vector<double> A((size_t)n * n, 0.0), ex;
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int c = y * nx + x;
                A[(size_t)c * n + c] = 4;
                if (x > 0) A[(size_t)c * n + c - 1] = -1;
                if (x + 1 < nx) A[(size_t)c * n + c + 1] = -1;
                if (y > 0) A[(size_t)c * n + c - nx] = -1;
                if (y + 1 < ny) A[(size_t)c * n + c + nx] = -1;
            }
        for (int a = 1; a <= nx; ++a)
            for (int b = 1; b <= ny; ++b)
                ex.push_back(4 - 2 * std::cos(M_PI * a / (nx + 1)) - 2 * std::cos(M_PI * b / (ny + 1)));
        report("laplace2d", A, n, &ex);
    }
    {   // repeated eigenvalues: I + u u^T (eigenvalue 1 of multiplicity n - 1)
        const int n = 30;
        std::vector<double> u(n), A((size_t)n * n), ex(n, 1.0);
        double uu = 0;
        for (int i = 0; i < n; ++i) {
            u[i] = urand();
            uu += u[i] * u[i];
        }
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) + u[i] * u[j];
        ex[0] = 1 + uu;
        report("rank1", A, n, &ex);
    }
    {   // diagonal, and the 1 x 1 and 2 x 2 cases
        std::vector<double> A = {3, 0, 0, 0, -1, 0, 0, 0, 2}, ex = {3, -1, 2};
        report("diagonal", A, 3, &ex);
        std::vector<double> B = {5}, eb = {5};
        report("one", B, 1, &eb);
        std::vector<double> C = {2, 1, 1, 2}, ec = {1, 3};
        report("two", C, 2, &ec);
    }
    {   // the memoised solver: the same results, bit for bit, as a fresh
        // factorisation, for a repeated input, after other inputs, after an
        // eviction, and for inputs that differ in one bit only
        const int n = 50;
        auto random_sym = [&](int seed) {
            state = 0x9E3779B97F4A7C15ull ^ (uint64_t)seed;
            std::vector<double> A((size_t)n * n);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j <= i; ++j) A[(size_t)i * n + j] = A[(size_t)j * n + i] = urand();
            return A;
        };
        const std::vector<double> A = random_sym(1), B = random_sym(2), C = random_sym(3);
        std::vector<double> D = A;
        D[7 * n + 3] = std::nextafter(D[7 * n + 3], 2.0);   // one ulp off, symmetric
        D[3 * n + 7] = D[7 * n + 3];
        auto same = [&](const std::vector<double> &M) {
            std::vector<double> q0, l0, q1, l1;
            if (!pp::sym_eig(M, n, q0, l0) || !pp::sym_eig_cached(M, n, q1, l1)) return false;
            return q0.size() == q1.size() && l0.size() == l1.size() &&
                   std::memcmp(q0.data(), q1.data(), q0.size() * sizeof(double)) == 0 &&
                   std::memcmp(l0.data(), l1.data(), l0.size() * sizeof(double)) == 0;
        };
        const size_t h0 = pp::sym_eig_cache_hits();
        const bool ok = same(A) && same(A) && same(B) && same(A) && same(C) && same(B) && same(D) && same(A) &&
                        same(D);
        // two kept: hits are A (2nd), A (4th) and D (last); B after C and A
        // after D were evicted, D is not A
        printf("cached %s %zu\n", ok ? "ok" : "FAIL", pp::sym_eig_cache_hits() - h0);
    }
    return 0;
}
