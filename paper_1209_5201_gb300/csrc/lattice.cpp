// Host lattice solver and verifier of the library (Sec. II: the velocity set
// xi = {c_a, w_a} "may be determined through several ways").
//
// Method: for a set of integer shells with unknown shell weights W_k and
// scale s = r^2, the quadrature must reproduce the unit Gaussian moments
//     sum_k W_k S_pq(k) s^(p+q) = (2p-1)!! (2q-1)!!,   S_pq(k) = sum_{e in k} ex^2p ey^2q
// for the even monomials up to the lattice degree.  With m shells there are
// m+1 conditions: they are linear in W for fixed s, so s is a root of the
// determinant of the augmented (m+1)x(m+1) system [A(s) | b].  The root is
// bracketed by a scan and refined by bisection in long double; the weights
// then follow from m of the equations; roots with a non-positive weight are
// rejected.  D2Q25 is the tensor product of the 1-D set {0, +-1, +-3}, solved
// the same way in 1-D.
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>
#include <algorithm>

#include "lbm_internal.h"
#include "lattice_tables.h"

namespace lbm {

namespace {

typedef long double ld;

ld dfact(int n) { ld v = 1; for (int k = n; k > 1; k -= 2) v *= k; return v; }

// Determinant by Gaussian elimination with partial pivoting.
ld det(std::vector<std::vector<ld>> a) {
    const int n = (int)a.size();
    ld d = 1;
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r) if (fabsl(a[r][c]) > fabsl(a[p][c])) p = r;
        if (a[p][c] == 0) return 0;
        if (p != c) { std::swap(a[p], a[c]); d = -d; }
        d *= a[c][c];
        for (int r = c + 1; r < n; ++r) {
            ld f = a[r][c] / a[c][c];
            for (int k = c; k < n; ++k) a[r][k] -= f * a[c][k];
        }
    }
    return d;
}

// Solve a square system; fails when a pivot is negligible against the
// largest entry (rank-deficient subsets of the moment conditions).
bool solve(std::vector<std::vector<ld>> a, std::vector<ld> b, std::vector<ld> &x) {
    const int n = (int)a.size();
    ld amax = 0;
    for (auto &row : a) for (ld v : row) amax = std::max(amax, fabsl(v));
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r = c + 1; r < n; ++r) if (fabsl(a[r][c]) > fabsl(a[p][c])) p = r;
        if (fabsl(a[p][c]) <= 1e-12L * amax) return false;
        std::swap(a[p], a[c]); std::swap(b[p], b[c]);
        for (int r = c + 1; r < n; ++r) {
            ld f = a[r][c] / a[c][c];
            for (int k = c; k < n; ++k) a[r][k] -= f * a[c][k];
            b[r] -= f * b[c];
        }
    }
    x.assign(n, 0);
    for (int r = n - 1; r >= 0; --r) {
        ld v = b[r];
        for (int k = r + 1; k < n; ++k) v -= a[r][k] * x[k];
        x[r] = v / a[r][r];
    }
    return true;
}

struct MomentSystem {
    // conditions (p, q) -> coefficient S_pq(k) per shell and degree p+q
    std::vector<std::vector<ld>> S;
    std::vector<int> deg;
    std::vector<ld> rhs;

    std::vector<std::vector<ld>> augmented(ld s) const {
        const int m = (int)S.size();
        std::vector<std::vector<ld>> a(m, std::vector<ld>(S[0].size() + 1));
        for (int i = 0; i < m; ++i) {
            ld sp = powl(s, deg[i]);
            for (size_t k = 0; k < S[i].size(); ++k) a[i][k] = S[i][k] * sp;
            a[i][S[i].size()] = rhs[i];
        }
        return a;
    }
    // Weights at a root s: drop one condition at a time (the last first)
    // until the remaining square system is regular and its solution also
    // satisfies the dropped condition.
    bool weights(ld s, std::vector<ld> &w) const {
        auto a = augmented(s);
        const int m = (int)a.size(), nw = (int)S[0].size();
        for (int drop = m - 1; drop >= 0; --drop) {
            std::vector<std::vector<ld>> A;
            std::vector<ld> b;
            for (int i = 0; i < m; ++i) {
                if (i == drop) continue;
                A.push_back(std::vector<ld>(a[i].begin(), a[i].begin() + nw));
                b.push_back(a[i][nw]);
            }
            if (!solve(A, b, w)) continue;
            ld res = -a[drop][nw];
            for (int k = 0; k < nw; ++k) res += a[drop][k] * w[k];
            if (fabsl(res) <= 1e-9L * std::max((ld)1, fabsl(a[drop][nw]))) return true;
        }
        return false;
    }
};

// Positive roots s of det[A(s)|b], with all weights positive, sorted by
// decreasing s.
std::vector<std::pair<ld, std::vector<ld>>> roots(const MomentSystem &ms) {
    std::vector<std::pair<ld, std::vector<ld>>> out;
    const ld lo = 0.05L, hi = 12.0L;
    const int nscan = 24000;
    ld s0 = lo, d0 = det(ms.augmented(s0));
    for (int i = 1; i <= nscan; ++i) {
        ld s1 = lo + (hi - lo) * i / nscan;
        ld d1 = det(ms.augmented(s1));
        if ((d0 < 0) != (d1 < 0)) {
            ld a = s0, b = s1, da = d0;
            for (int it = 0; it < 200; ++it) {
                ld c = 0.5L * (a + b);
                ld dc = det(ms.augmented(c));
                if ((dc < 0) == (da < 0)) { a = c; da = dc; } else { b = c; }
                if (b - a <= 4 * LDBL_EPSILON * b) break;
            }
            ld s = 0.5L * (a + b);
            std::vector<ld> w;
            if (ms.weights(s, w) && std::all_of(w.begin(), w.end(), [](ld v) { return v > 0; }))
                out.push_back({s, w});
        }
        s0 = s1; d0 = d1;
    }
    std::sort(out.begin(), out.end(), [](auto &x, auto &y) { return x.first > y.first; });
    return out;
}

std::vector<std::pair<int, int>> shell_points(int a, int b) {
    std::vector<std::pair<int, int>> pts;
    for (int sx : {1, -1})
        for (int sy : {1, -1}) {
            pts.push_back({sx * a, sy * b});
            pts.push_back({sx * b, sy * a});
        }
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    return pts;
}

MomentSystem system_2d(const std::vector<std::pair<int, int>> &shells, int max_half_degree) {
    MomentSystem ms;
    for (int n = 0; n <= max_half_degree; ++n)
        for (int p = n; p >= (n + 1) / 2; --p) {
            int q = n - p;
            std::vector<ld> row;
            for (auto &sh : shells) {
                ld v = 0;
                for (auto &e : shell_points(sh.first, sh.second))
                    v += powl((ld)e.first, 2 * p) * powl((ld)e.second, 2 * q);
                row.push_back(v);
            }
            ms.S.push_back(row);
            ms.deg.push_back(n);
            ms.rhs.push_back(dfact(2 * p - 1) * dfact(2 * q - 1));
        }
    return ms;
}

template <size_t Q>
void fill_tables(LatticeHost &L, const int (&ex)[Q], const int (&ey)[Q], const int (&sh)[Q]) {
    L.Q = (int)Q;
    for (size_t a = 0; a < Q; ++a) {
        L.ex[a] = ex[a];
        L.ey[a] = ey[a];
        L.shell[a] = sh[a];
    }
    int n = 0;
    for (size_t a = 0; a < Q; ++a) n = std::max(n, std::abs(ey[a]));
    L.ghost_depth = n;
}

}  // namespace

int lattice_build(int kind, LatticeHost &L) {
    std::memset(&L, 0, sizeof(L));
    L.kind = kind;
    if (kind == 17) {
        static const int ex[] = LBM_Q17_EX, ey[] = LBM_Q17_EY, sh[] = LBM_Q17_SH;
        fill_tables(L, ex, ey, sh);
        std::vector<std::pair<int, int>> shells = LBM_Q17_SHELLS;
        auto r = roots(system_2d(shells, 3));
        if (r.empty()) return -1;
        L.r = (double)sqrtl(r[0].first);
        for (int a = 0; a < L.Q; ++a) L.w[a] = (double)r[0].second[L.shell[a]];
        L.degree = 7;
    } else if (kind == 37) {
        static const int ex[] = LBM_Q37_EX, ey[] = LBM_Q37_EY, sh[] = LBM_Q37_SH;
        fill_tables(L, ex, ey, sh);
        std::vector<std::pair<int, int>> shells = LBM_Q37_SHELLS;
        auto r = roots(system_2d(shells, 4));
        if (r.empty()) return -1;
        // the degree-9 system has a single root with all weights positive
        L.r = (double)sqrtl(r[0].first);
        for (int a = 0; a < L.Q; ++a) L.w[a] = (double)r[0].second[L.shell[a]];
        L.degree = 9;
    } else if (kind == 25 || kind == 26) {
        static const int ex[] = LBM_Q25_EX, ey[] = LBM_Q25_EY, sh[] = LBM_Q25_SH;
        fill_tables(L, ex, ey, sh);
        // 1-D set {0, +-1, +-3}: conditions m0, m2, m4, m6 on weights (w0, w1, w3)
        MomentSystem ms;
        const int absc[3] = {0, 1, 3};
        for (int i = 0; i <= 3; ++i) {
            std::vector<ld> row;
            for (int k = 0; k < 3; ++k)
                row.push_back(absc[k] == 0 ? (i == 0 ? 1.0L : 0.0L)
                                           : 2.0L * powl((ld)absc[k], 2 * i));
            ms.S.push_back(row);
            ms.deg.push_back(i);
            ms.rhs.push_back(dfact(2 * i - 1));
        }
        auto r = roots(ms);
        int pick = kind == 25 ? 0 : 1;
        if ((int)r.size() <= pick) return -1;
        L.r = (double)sqrtl(r[pick].first);
        const std::vector<ld> &w1 = r[pick].second;
        auto w1d = [&](int e) { e = std::abs(e); return e == 0 ? w1[0] : (e == 1 ? w1[1] : w1[2]); };
        for (int a = 0; a < L.Q; ++a) L.w[a] = (double)(w1d(L.ex[a]) * w1d(L.ey[a]));
        L.degree = 7;
    } else {
        return -1;
    }
    return 0;
}

int lattice_build_custom(int Q, const int8_t *e, const double *w, double r, LatticeHost &L,
                         const char **why) {
    const int kind = Q == 17 ? 17 : Q == 25 ? 25 : Q == 37 ? 37 : 0;
    if (!kind) { *why = "Q must be 17, 25 or 37 (the velocity sets the kernels are built for)"; return -1; }
    if (!e || !w) { *why = "NULL table"; return -1; }
    if (!(r > 0) || !std::isfinite(r)) { *why = "r must be positive and finite"; return -1; }
    // the library's tables of this velocity set, then the caller's weights in
    // the library's order
    if (lattice_build(kind, L) != 0) { *why = "velocity set tables"; return -1; }
    int from[kMaxQ];
    for (int a = 0; a < Q; ++a) {
        from[a] = -1;
        for (int b = 0; b < Q; ++b)
            if (e[2 * b] == L.ex[a] && e[2 * b + 1] == L.ey[a]) {
                if (from[a] >= 0) { *why = "a velocity appears twice"; return -1; }
                from[a] = b;
            }
        if (from[a] < 0) { *why = "the velocities are not the built-in set of this Q"; return -1; }
    }
    double wsh[kMaxShells];
    bool seen[kMaxShells] = {};
    for (int a = 0; a < Q; ++a) {
        const double v = w[from[a]];
        if (!(v > 0) || !std::isfinite(v)) { *why = "weights must be positive and finite"; return -1; }
        const int sh = L.shell[a];
        if (!seen[sh]) { seen[sh] = true; wsh[sh] = v; }
        // the kernels keep one weight per shell of symmetric velocities
        else if (std::fabs(v - wsh[sh]) > 1e-12 * wsh[sh]) {
            *why = "weights must be equal within each shell of symmetric velocities";
            return -1;
        }
        L.w[a] = v;
    }
    L.r = r;
    // isotropy degree: the largest odd degree whose moments match the Gaussian
    L.degree = 0;
    for (int d = 1; d <= 15; d += 2)
        if (lattice_isotropy_error(L, d) < 1e-10) L.degree = d;
    L.kind = kind;
    return 0;
}

double lattice_isotropy_error(const LatticeHost &L, int degree) {
    // brute-force moments of every monomial c_x^p c_y^q, p + q <= degree
    double worst = 0.0;
    for (int n = 0; n <= degree; ++n)
        for (int p = 0; p <= n; ++p) {
            int q = n - p;
            ld m = 0;
            for (int a = 0; a < L.Q; ++a)
                m += (ld)L.w[a] * powl((ld)L.r * L.ex[a], p) * powl((ld)L.r * L.ey[a], q);
            ld ref = (p % 2 || q % 2) ? 0.0L : dfact(p - 1) * dfact(q - 1);
            worst = std::max(worst, (double)fabsl(m - ref));
        }
    return worst;
}

}  // namespace lbm
