// Small dense complex linear algebra on the host (Grace CPU) for the p x p
// projected problems of the restarted-Arnoldi eigensolver (p <= a few
// hundred). Column-major storage, leading dimension = rows.
//
// Algorithms (Golub & Van Loan, Matrix Computations, 4th ed.):
//   hessenberg()   Householder reduction A = Q H Q^dag          (Alg. 7.4.2)
//   schur()        complex Schur form by the shifted QR iteration on the
//                  Hessenberg matrix, Wilkinson shifts, deflation on small
//                  subdiagonals                                 (Sec. 7.5)
//   swap_schur()   exchange two adjacent diagonal entries of a triangular
//                  Schur factor with one Givens rotation        (Sec. 7.6.2)
//   tri_eigvecs()  eigenvectors of an upper triangular matrix by back
//                  substitution
//   cholesky(), trsm helpers, small products.
#pragma once
#include <cmath>
#include <complex>
#include <vector>

namespace sla {

using cd = std::complex<double>;

struct Mat {
    int r = 0, c = 0;
    std::vector<cd> a;
    Mat() {}
    Mat(int r_, int c_) : r(r_), c(c_), a((size_t)r_ * c_, cd(0)) {}
    cd& operator()(int i, int j) { return a[(size_t)j * r + i]; }
    const cd& operator()(int i, int j) const { return a[(size_t)j * r + i]; }
    static Mat eye(int n) {
        Mat m(n, n);
        for (int i = 0; i < n; i++) m(i, i) = 1.0;
        return m;
    }
};

inline Mat mul(const Mat& A, const Mat& B) {
    Mat C(A.r, B.c);
    for (int j = 0; j < B.c; j++)
        for (int k = 0; k < A.c; k++) {
            cd b = B(k, j);
            if (b == cd(0)) continue;
            for (int i = 0; i < A.r; i++) C(i, j) += A(i, k) * b;
        }
    return C;
}
inline Mat adj(const Mat& A) {
    Mat B(A.c, A.r);
    for (int i = 0; i < A.r; i++)
        for (int j = 0; j < A.c; j++) B(j, i) = std::conj(A(i, j));
    return B;
}

// Givens rotation G = [[c, s], [-conj(s), c]] (c real) with G^dag (a; b) = (r; 0)
inline void givens(cd a, cd b, double& c, cd& s) {
    double na = std::abs(a), nb = std::abs(b);
    if (nb == 0.0) {
        c = 1.0;
        s = 0.0;
        return;
    }
    if (na == 0.0) {
        c = 0.0;
        s = std::conj(b) / nb;  // maps (0, b) -> (|b|, 0)
        s = cd(1.0, 0.0) * (b / nb);
        s = std::conj(s);
        return;
    }
    double nr = std::hypot(na, nb);
    c = na / nr;
    cd alpha = a / na;
    s = alpha * std::conj(b) / nr;
}
// apply to rows i, i+1 of A (columns j0..j1-1): (x; y) <- (c x + s y; -conj(s) x + c y)
inline void rot_rows(Mat& A, int i, int k, double c, cd s, int j0, int j1) {
    for (int j = j0; j < j1; j++) {
        cd x = A(i, j), y = A(k, j);
        A(i, j) = c * x + s * y;
        A(k, j) = -std::conj(s) * x + c * y;
    }
}
// apply G^dag from the right to columns i, k: (x, y) <- (c x + conj(s) y, -s x + c y)
inline void rot_cols(Mat& A, int i, int k, double c, cd s, int r0, int r1) {
    for (int r = r0; r < r1; r++) {
        cd x = A(r, i), y = A(r, k);
        A(r, i) = c * x + std::conj(s) * y;
        A(r, k) = -s * x + c * y;
    }
}

// Householder reduction to upper Hessenberg form; Q accumulates (A = Q H Q^dag).
inline void hessenberg(Mat& A, Mat& Q) {
    int n = A.r;
    Q = Mat::eye(n);
    std::vector<cd> v(n);
    for (int k = 0; k + 2 < n + 0 && k < n - 2; k++) {
        double xn = 0.0;
        for (int i = k + 1; i < n; i++) xn += std::norm(A(i, k));
        xn = std::sqrt(xn);
        if (xn == 0.0) continue;
        cd x0 = A(k + 1, k);
        cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
        cd alpha = -ph * xn;
        for (int i = 0; i < n; i++) v[i] = 0.0;
        v[k + 1] = x0 - alpha;
        for (int i = k + 2; i < n; i++) v[i] = A(i, k);
        double vn = 0.0;
        for (int i = k + 1; i < n; i++) vn += std::norm(v[i]);
        if (vn == 0.0) continue;
        // A <- (I - 2 v v^dag / vn) A (I - 2 v v^dag / vn)
        for (int j = 0; j < n; j++) {
            cd s = 0.0;
            for (int i = k + 1; i < n; i++) s += std::conj(v[i]) * A(i, j);
            s *= 2.0 / vn;
            for (int i = k + 1; i < n; i++) A(i, j) -= v[i] * s;
        }
        for (int i = 0; i < n; i++) {
            cd s = 0.0;
            for (int j = k + 1; j < n; j++) s += A(i, j) * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; j++) A(i, j) -= s * std::conj(v[j]);
        }
        for (int i = 0; i < n; i++) {
            cd s = 0.0;
            for (int j = k + 1; j < n; j++) s += Q(i, j) * v[j];
            s *= 2.0 / vn;
            for (int j = k + 1; j < n; j++) Q(i, j) -= s * std::conj(v[j]);
        }
        for (int i = k + 2; i < n; i++) A(i, k) = 0.0;
    }
}

// Complex Schur form of a Hessenberg matrix H (in place: H <- T), Z <- Z * Q.
// Returns false if it did not converge.
inline bool schur_hess(Mat& H, Mat& Z, int max_sweeps_per_eig = 60) {
    int n = H.r;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1;
    int iter = 0;
    while (hi > 0) {
        // find the active block [lo, hi]
        int lo = hi;
        while (lo > 0) {
            double s = std::abs(H(lo - 1, lo - 1)) + std::abs(H(lo, lo));
            if (s == 0.0) s = 1.0;
            if (std::abs(H(lo, lo - 1)) <= eps * s) {
                H(lo, lo - 1) = 0.0;
                break;
            }
            lo--;
        }
        if (lo == hi) {
            hi--;
            iter = 0;
            continue;
        }
        if (++iter > max_sweeps_per_eig) return false;
        // Wilkinson shift from the trailing 2x2 block
        cd a = H(hi - 1, hi - 1), b = H(hi - 1, hi), c = H(hi, hi - 1), d = H(hi, hi);
        cd tr = a + d, det = a * d - b * c;
        cd disc = std::sqrt(tr * tr * 0.25 - det);
        cd l1 = tr * 0.5 + disc, l2 = tr * 0.5 - disc;
        cd mu = std::abs(l1 - d) < std::abs(l2 - d) ? l1 : l2;
        if (iter % 11 == 10) mu = d + cd(std::abs(H(hi, hi - 1)) * 0.75, 0.0);  // exceptional shift
        // implicit single-shift QR sweep on [lo, hi] by chasing the bulge
        cd x = H(lo, lo) - mu, y = H(lo + 1, lo);
        for (int k = lo; k < hi; k++) {
            double cs;
            cd sn;
            givens(x, y, cs, sn);
            rot_rows(H, k, k + 1, cs, sn, k > lo ? k - 1 : lo, n);
            rot_cols(H, k, k + 1, cs, sn, 0, std::min(k + 3, hi + 1));
            rot_cols(Z, k, k + 1, cs, sn, 0, Z.r);
            if (k > lo) H(k + 1, k - 1) = 0.0;
            if (k + 1 < hi) {
                x = H(k + 1, k);
                y = H(k + 2, k);
            }
        }
    }
    for (int j = 0; j < n; j++)
        for (int i = j + 1; i < n; i++) H(i, j) = 0.0;
    return true;
}

// swap T(k,k) and T(k+1,k+1) of an upper triangular T; Z <- Z * G
inline void swap_schur(Mat& T, Mat& Z, int k) {
    int n = T.r;
    cd t11 = T(k, k), t22 = T(k + 1, k + 1), t12 = T(k, k + 1);
    double cs;
    cd sn;
    givens(t12, t22 - t11, cs, sn);
    rot_cols(T, k, k + 1, cs, sn, 0, n);
    rot_rows(T, k, k + 1, cs, sn, 0, n);
    rot_cols(Z, k, k + 1, cs, sn, 0, Z.r);
    T(k + 1, k) = 0.0;
    T(k, k) = t22;
    T(k + 1, k + 1) = t11;
}

// reorder so that the entries with want[i] come first (stable bubble of swaps)
inline void reorder_schur(Mat& T, Mat& Z, std::vector<char> want) {
    int n = T.r;
    int dst = 0;
    for (int i = 0; i < n; i++) {
        if (!want[i]) continue;
        for (int k = i - 1; k >= dst; k--) {
            swap_schur(T, Z, k);
            std::swap(want[k], want[k + 1]);
        }
        dst++;
    }
}

// eigenvectors of upper triangular T (columns, unit 2-norm)
inline Mat tri_eigvecs(const Mat& T) {
    int n = T.r;
    Mat X(n, n);
    const double tiny = 1e-300;
    for (int k = 0; k < n; k++) {
        X(k, k) = 1.0;
        cd lam = T(k, k);
        double smin = 1e-14 * (std::abs(lam) + 1e-30);
        for (int i = k - 1; i >= 0; i--) {
            cd s = 0.0;
            for (int j = i + 1; j <= k; j++) s += T(i, j) * X(j, k);
            cd den = T(i, i) - lam;
            if (std::abs(den) < smin) den = smin;
            X(i, k) = -s / den;
        }
        double nr = 0.0;
        for (int i = 0; i <= k; i++) nr += std::norm(X(i, k));
        nr = std::sqrt(nr) + tiny;
        for (int i = 0; i <= k; i++) X(i, k) /= nr;
    }
    return X;
}

// Cholesky G = L L^dag (lower); false if not positive definite
inline bool cholesky(const Mat& G, Mat& L) {
    int n = G.r;
    L = Mat(n, n);
    for (int j = 0; j < n; j++) {
        double d = G(j, j).real();
        for (int k = 0; k < j; k++) d -= std::norm(L(j, k));
        if (!(d > 0.0)) return false;
        L(j, j) = std::sqrt(d);
        for (int i = j + 1; i < n; i++) {
            cd s = G(i, j);
            for (int k = 0; k < j; k++) s -= L(i, k) * std::conj(L(j, k));
            L(i, j) = s / L(j, j);
        }
    }
    return true;
}
// inverse of a lower triangular matrix
inline Mat lower_inv(const Mat& L) {
    int n = L.r;
    Mat X(n, n);
    for (int j = 0; j < n; j++) {
        X(j, j) = 1.0 / L(j, j);
        for (int i = j + 1; i < n; i++) {
            cd s = 0.0;
            for (int k = j; k < i; k++) s += L(i, k) * X(k, j);
            X(i, j) = -s / L(i, i);
        }
    }
    return X;
}

// general complex eigen-decomposition via Hessenberg + Schur: A = Z T Z^dag
inline bool schur(const Mat& A, Mat& T, Mat& Z) {
    T = A;
    Mat Q;
    hessenberg(T, Q);
    Z = Q;
    return schur_hess(T, Z);
}

}  // namespace sla
