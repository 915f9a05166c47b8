// Host FP64 set-up of the 1D spline tables (Sec. 3.1, Sec. 3.2; Sec. 3.3
// counts their cost as negligible next to the operator applications).
//
// Per parametric direction this builds, from an open uniform knot vector:
//   Galerkin (Sec. 3.1)  the mass matrix Z_k and its Cholesky factor L_k, the
//                        interpolation knot vector (continuity of Sec. 4), its
//                        Greville points x~, the collocation matrix B~_k
//                        (B~_k[a, j] = B~_j(x~_a)), the mixed mass matrix
//                        M_k[a, i] = int B~_a B_i, and the folded factors
//                        Q_k = B~_k^-T M_k and P_k = Q_k L_k^-T;
//   collocation (Sec. 3.2) the Gauss points / weights (p+1 per element), the
//                        (rational) basis table at them, the Greville
//                        collocation points and the pivoted-LU inverse of the
//                        1D collocation matrix (the Kronecker form of Z,
//                        Sec. 3.3 Remark).
// All products of degree-2p splines are integrated exactly with p+1 Gauss
// points per element.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "kl_internal.h"

namespace kl {

// --------------------------------------------------------------------------
// Small dense linear algebra
// --------------------------------------------------------------------------
Mat identity(int n) {
    Mat I(n, n);
    for (int i = 0; i < n; ++i) I(i, i) = 1.0;
    return I;
}

Mat transpose(const Mat& A) {
    Mat T(A.cols, A.rows);
    for (int j = 0; j < A.cols; ++j)
        for (int i = 0; i < A.rows; ++i) T(j, i) = A(i, j);
    return T;
}

Mat matmul(const Mat& A, const Mat& B) {
    Mat C(A.rows, B.cols);
    for (int j = 0; j < B.cols; ++j)
        for (int l = 0; l < A.cols; ++l) {
            const double b = B(l, j);
            if (b == 0.0) continue;
            for (int i = 0; i < A.rows; ++i) C(i, j) += A(i, l) * b;
        }
    return C;
}

bool cholesky(Mat& A) {
    const int n = A.rows;
    for (int j = 0; j < n; ++j) {
        double d = A(j, j);
        for (int l = 0; l < j; ++l) d -= A(j, l) * A(j, l);
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        A(j, j) = d;
        for (int i = j + 1; i < n; ++i) {
            double s = A(i, j);
            for (int l = 0; l < j; ++l) s -= A(i, l) * A(j, l);
            A(i, j) = s / d;
        }
        for (int i = 0; i < j; ++i) A(i, j) = 0.0;
    }
    return true;
}

Mat lower_inverse(const Mat& L) {
    const int n = L.rows;
    Mat X(n, n);
    for (int c = 0; c < n; ++c) {
        for (int i = c; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int l = c; l < i; ++l) s -= L(i, l) * X(l, c);
            X(i, c) = s / L(i, i);
        }
    }
    return X;
}

bool lu_solve(const Mat& A0, const Mat& B, Mat& X) {
    const int n = A0.rows;
    Mat A = A0;
    X = B;
    std::vector<int> piv(n);
    for (int j = 0; j < n; ++j) {
        int r = j;
        double best = std::fabs(A(j, j));
        for (int i = j + 1; i < n; ++i)
            if (std::fabs(A(i, j)) > best) best = std::fabs(A(i, j)), r = i;
        if (best == 0.0) return false;
        piv[j] = r;
        if (r != j) {
            for (int c = 0; c < n; ++c) std::swap(A(j, c), A(r, c));
            for (int c = 0; c < X.cols; ++c) std::swap(X(j, c), X(r, c));
        }
        for (int i = j + 1; i < n; ++i) {
            const double f = A(i, j) / A(j, j);
            A(i, j) = f;
            for (int c = j + 1; c < n; ++c) A(i, c) -= f * A(j, c);
            for (int c = 0; c < X.cols; ++c) X(i, c) -= f * X(j, c);
        }
    }
    for (int c = 0; c < X.cols; ++c)
        for (int i = n - 1; i >= 0; --i) {
            double s = X(i, c);
            for (int l = i + 1; l < n; ++l) s -= A(i, l) * X(l, c);
            X(i, c) = s / A(i, i);
        }
    return true;
}

// --------------------------------------------------------------------------
// B-splines
// --------------------------------------------------------------------------
namespace {

struct Knots {
    std::vector<double> t;
    int p = 1;
    int n() const { return int(t.size()) - p - 1; }
};

// Open knot vector on [0,1], nel equal elements, interior multiplicity p-cont.
Knots open_knots(int nel, int p, int cont) {
    Knots k;
    k.p = p;
    for (int i = 0; i <= p; ++i) k.t.push_back(0.0);
    for (int e = 1; e < nel; ++e)
        for (int m = 0; m < p - cont; ++m) k.t.push_back(double(e) / nel);
    for (int i = 0; i <= p; ++i) k.t.push_back(1.0);
    return k;
}

// The same with a join at the middle breakpoint 1/2 (nel even) of
// multiplicity p-join_cont: two patches joined C^join_cont (Sec. 4.1: C^0
// for the trial space at the half cylinder's geometry join, C^-1 for the
// interpolation space).
Knots joined_knots(int nel, int p, int cont, int join_cont) {
    Knots k;
    k.p = p;
    for (int i = 0; i <= p; ++i) k.t.push_back(0.0);
    for (int e = 1; e < nel; ++e) {
        const int mult = 2 * e == nel ? p - join_cont : p - cont;
        for (int m = 0; m < mult; ++m) k.t.push_back(double(e) / nel);
    }
    for (int i = 0; i <= p; ++i) k.t.push_back(1.0);
    return k;
}

std::vector<double> greville(const Knots& k) {
    std::vector<double> g(k.n());
    for (int i = 0; i < k.n(); ++i) {
        double s = 0.0;
        for (int j = 1; j <= k.p; ++j) s += k.t[i + j];
        g[i] = s / k.p;
    }
    return g;
}

// Knot span s with t[s] <= x < t[s+1] (the right end maps to the last span).
int find_span(const Knots& k, double x) {
    const int n = k.n();
    if (x >= k.t[n]) return n - 1;
    if (x <= k.t[k.p]) {
        int s = k.p;
        while (k.t[s + 1] <= x) ++s;
        return s;
    }
    int lo = k.p, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (x < k.t[mid]) hi = mid; else lo = mid;
    }
    return lo;
}

// The p+1 non-zero basis functions B_{s-p..s}(x) by the triangular
// Cox-de Boor scheme (each degree built from the previous one).
void basis_funs(const Knots& k, int s, double x, double* out) {
    const int p = k.p;
    double left[16], right[16];
    out[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        left[j] = x - k.t[s + 1 - j];
        right[j] = k.t[s + j] - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double tmp = out[r] / (right[r + 1] + left[j - r]);
            out[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        out[j] = saved;
    }
}

// Greville points at the right end of their function's support inside the
// domain (a C^-1 breakpoint, where two Greville points coincide): evaluated
// as limits from the left.
std::vector<char> greville_left(const Knots& k) {
    const std::vector<double> g = greville(k);
    std::vector<char> left(g.size(), 0);
    for (int i = 0; i < k.n(); ++i) left[i] = (g[i] == k.t[i + k.p + 1] && g[i] < k.t.back()) ? 1 : 0;
    return left;
}

// Dense basis matrix: rows = points, columns = basis functions. Points
// flagged in `left` use the span that ends at them (limit from the left).
Mat basis_matrix(const Knots& k, const std::vector<double>& x, const std::vector<char>* left = nullptr) {
    Mat B(int(x.size()), k.n());
    double v[16];
    for (size_t i = 0; i < x.size(); ++i) {
        int s = find_span(k, x[i]);
        if (left && (*left)[i] && s > k.p && k.t[s] == x[i]) {
            --s;
            while (s > k.p && k.t[s] == k.t[s + 1]) --s;
        }
        basis_funs(k, s, x[i], v);
        for (int j = 0; j <= k.p; ++j) B(int(i), s - k.p + j) = v[j];
    }
    return B;
}

// Gauss-Legendre nodes/weights on [-1, 1]: Newton iteration on P_n from the
// three-term recurrence, started at cos(pi (i - 1/4) / (n + 1/2)).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        // recompute derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; ++j) {
            const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

void element_gauss(int nel, int nq, std::vector<double>& x, std::vector<double>& w) {
    std::vector<double> gx, gw;
    gauss_legendre(nq, gx, gw);
    x.clear();
    w.clear();
    for (int e = 0; e < nel; ++e) {
        const double a = double(e) / nel, b = double(e + 1) / nel;
        for (int q = 0; q < nq; ++q) {
            x.push_back(0.5 * (a + b) + 0.5 * (b - a) * gx[q]);
            w.push_back(0.5 * (b - a) * gw[q]);
        }
    }
}

// Denominator of the quadratic NURBS quarter arc with weights 1, sqrt(2)/2, 1.
double arc_weight(double u) {
    const double w = std::sqrt(0.5);
    return (1.0 - u) * (1.0 - u) + 2.0 * w * u * (1.0 - u) + u * u;
}

// The half arc: two quarter arcs on [0, 1/2] and [1/2, 1] (C^0 at 1/2).
double half_arc_weight(double u) { return u < 0.5 ? arc_weight(2.0 * u) : arc_weight(2.0 * u - 1.0); }

Mat rational_rows(const Mat& B, const std::vector<double>& w) {
    Mat R = B;
    for (int i = 0; i < B.rows; ++i) {
        double den = 0.0;
        for (int j = 0; j < B.cols; ++j) den += B(i, j) * w[j];
        for (int j = 0; j < B.cols; ++j) R(i, j) = B(i, j) * w[j] / den;
    }
    return R;
}

}  // namespace

std::string setup_direction(Dir1D& d, bool present, int nel, int p, int interp_cont,
                            int arc, bool need_galerkin, bool need_collocation) {
    const bool rational = arc != 0;
    const bool join = arc == 2;  // C^0 geometry join at 1/2
    if (!present) {
        d = Dir1D();
        d.N = d.Nt = d.nq = 1;
        d.xg = {0.0};
        d.Q = d.P = d.LinvT = d.Zinv_gal = d.R = d.Zinv_col = d.E = identity(1);
        d.ne = 1;
        d.xe = {0.0};
        d.we = {1.0};
        d.xq = {0.0};
        d.wq = {1.0};
        d.xc = {0.0};
        return "";
    }
    if (p < 1 || p > 8) return "degree must be in 1..8";
    if (join && (nel < 2 || nel % 2)) return "the joined direction needs an even number of elements";
    d.nel = nel;
    d.p = p;
    const Knots U = join ? joined_knots(nel, p, p - 1, 0) : open_knots(nel, p, p - 1);
    d.N = U.n();

    std::vector<double> xq, wq;
    element_gauss(nel, p + 1, xq, wq);
    const Mat BU = basis_matrix(U, xq);

    if (need_galerkin) {
        if (interp_cont < 0 || interp_cont > p - 1) return "interpolation continuity out of range";
        const Knots Ut = join ? joined_knots(nel, p, interp_cont, -1) : open_knots(nel, p, interp_cont);
        d.Nt = Ut.n();
        d.xg = greville(Ut);
        const std::vector<char> xg_left = greville_left(Ut);
        const Mat BUt = basis_matrix(Ut, xq);
        // Z_k = int B_i B_j ; M_k = int B~_a B_i
        Mat Z(d.N, d.N), M(d.Nt, d.N);
        for (int q = 0; q < int(xq.size()); ++q)
            for (int i = 0; i < d.N; ++i) {
                const double bi = BU(q, i) * wq[q];
                if (bi == 0.0) continue;
                for (int j = 0; j < d.N; ++j) Z(j, i) += BU(q, j) * bi;
                for (int a = 0; a < d.Nt; ++a) M(a, i) += BUt(q, a) * bi;
            }
        Mat L = Z;
        if (!cholesky(L)) return "1D mass matrix not positive definite";
        const Mat Linv = lower_inverse(L);
        d.LinvT = transpose(Linv);
        d.Zinv_gal = matmul(d.LinvT, Linv);
        const Mat Bt = basis_matrix(Ut, d.xg, &xg_left);  // Bt(a, j) = B~_j(x~_a)
        if (!lu_solve(transpose(Bt), M, d.Q)) return "1D interpolation matrix singular";
        d.P = matmul(d.Q, d.LinvT);
    }
    if (need_collocation) {
        std::vector<double> w(d.N, 1.0);
        d.xc = greville(U);
        const Mat Bc = basis_matrix(U, d.xc);
        if (rational) {
            // weights of the degree-p, nel-element space that reproduce the
            // arc's quadratic denominator: interpolate it at the Greville points
            Mat rhs(d.N, 1), sol;
            for (int i = 0; i < d.N; ++i) rhs(i, 0) = join ? half_arc_weight(d.xc[i]) : arc_weight(d.xc[i]);
            if (!lu_solve(Bc, rhs, sol)) return "NURBS weight interpolation failed";
            for (int i = 0; i < d.N; ++i) w[i] = sol(i, 0);
        }
        d.nq = int(xq.size());
        d.xq = xq;
        d.wq = wq;
        d.R = rational_rows(BU, w);
        const Mat Zc = rational_rows(Bc, w);
        if (!lu_solve(Zc, identity(d.N), d.Zinv_col)) return "1D collocation matrix singular";
    }
    d.ne = int(xq.size());
    d.xe = xq;
    d.we = wq;
    d.E = need_collocation ? d.R : BU;
    return "";
}

}  // namespace kl
