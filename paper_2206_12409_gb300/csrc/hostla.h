// Small dense complex linear algebra on the host, for the set-up only (matrices
// of at most a few hundred columns).  Column-major storage.
#pragma once
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

namespace vsie {
namespace hla {

using cd = std::complex<double>;

// Cyclic Jacobi eigen-decomposition of a Hermitian n x n matrix A (destroyed):
// eigenvalues (descending) in w, eigenvectors in the columns of Vout.
inline void herm_eig(int n, std::vector<cd>& A, std::vector<double>& w, std::vector<cd>& Vout) {
    std::vector<cd> V((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i + (size_t)n * i] = 1.0;
    auto a = [&](int i, int j) -> cd& { return A[i + (size_t)n * j]; };
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int j = 0; j < n; ++j) {
            diag += std::norm(a(j, j));
            for (int i = 0; i < j; ++i) off += std::norm(a(i, j));
        }
        if (off <= 1e-30 * (diag + 1e-300)) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const cd apq = a(p, q);
                const double mag = std::abs(apq);
                if (mag < 1e-300) continue;
                const double app = a(p, p).real(), aqq = a(q, q).real();
                // rotate so that the (p, q) entry vanishes: phase e = apq / |apq|
                const cd e = apq / mag;
                const double theta = 0.5 * std::atan2(2.0 * mag, aqq - app);
                const double c = std::cos(theta), s = std::sin(theta);
                // columns p, q of A (and rows by Hermitian symmetry)
                for (int k = 0; k < n; ++k) {
                    const cd akp = a(k, p), akq = a(k, q);
                    a(k, p) = c * akp - s * std::conj(e) * akq;
                    a(k, q) = s * e * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const cd apk = a(p, k), aqk = a(q, k);
                    a(p, k) = c * apk - s * e * aqk;
                    a(q, k) = s * std::conj(e) * apk + c * aqk;
                }
                a(p, q) = 0.0;
                a(q, p) = 0.0;
                a(p, p) = a(p, p).real();
                a(q, q) = a(q, q).real();
                for (int k = 0; k < n; ++k) {
                    const cd vkp = V[k + (size_t)n * p], vkq = V[k + (size_t)n * q];
                    V[k + (size_t)n * p] = c * vkp - s * std::conj(e) * vkq;
                    V[k + (size_t)n * q] = s * e * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int i, int j) { return a(i, i).real() > a(j, j).real(); });
    w.resize(n);
    Vout.assign((size_t)n * n, 0.0);
    for (int k = 0; k < n; ++k) {
        w[k] = a(idx[k], idx[k]).real();
        for (int i = 0; i < n; ++i) Vout[i + (size_t)n * k] = V[i + (size_t)n * idx[k]];
    }
}

inline std::vector<cd> upper_inv(int n, const std::vector<cd>& R);

// Thin Householder QR of an m x n matrix (m >= n); returns Q (m x n).
inline std::vector<cd> qr_q(int m, int n, std::vector<cd> A) {
    std::vector<std::vector<cd>> vs(n);
    for (int k = 0; k < n; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += std::norm(A[i + (size_t)m * k]);
        nrm = std::sqrt(nrm);
        std::vector<cd> v(m - k, 0.0);
        const cd x0 = A[k + (size_t)m * k];
        const cd ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cd(1.0);
        for (int i = k; i < m; ++i) v[i - k] = A[i + (size_t)m * k];
        v[0] += ph * nrm;
        double vn = 0.0;
        for (auto& z : v) vn += std::norm(z);
        vn = std::sqrt(vn);
        if (vn > 0)
            for (auto& z : v) z /= vn;
        for (int j = k; j < n; ++j) {
            cd s = 0.0;
            for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * A[i + (size_t)m * j];
            for (int i = k; i < m; ++i) A[i + (size_t)m * j] -= 2.0 * v[i - k] * s;
        }
        vs[k] = std::move(v);
    }
    std::vector<cd> Q((size_t)m * n, 0.0);
    for (int j = 0; j < n; ++j) Q[j + (size_t)m * j] = 1.0;
    for (int k = n - 1; k >= 0; --k) {
        const auto& v = vs[k];
        for (int j = 0; j < n; ++j) {
            cd s = 0.0;
            for (int i = k; i < m; ++i) s += std::conj(v[i - k]) * Q[i + (size_t)m * j];
            for (int i = k; i < m; ++i) Q[i + (size_t)m * j] -= 2.0 * v[i - k] * s;
        }
    }
    return Q;
}

// Tikhonov-regularised least squares operator for an m x n matrix A (m >= n):
// returns X (n x m) with X b = argmin ||A x - b||^2 + lam^2 ||x||^2,
// lam = reg * ||A||_2 (largest singular value by power iteration), from the
// QR factorisation of the augmented matrix [A; lam I] (no squared condition).
inline std::vector<cd> tikhonov_pinv(int m, int n, const std::vector<cd>& A, double reg) {
    // ||A||_2 by power iteration on A^H A
    std::vector<cd> x(n, 1.0), y(m);
    double smax = 0.0;
    for (int it = 0; it < 60; ++it) {
        for (int i = 0; i < m; ++i) {
            cd s = 0.0;
            for (int j = 0; j < n; ++j) s += A[i + (size_t)m * j] * x[j];
            y[i] = s;
        }
        double nx = 0.0;
        for (int j = 0; j < n; ++j) {
            cd s = 0.0;
            for (int i = 0; i < m; ++i) s += std::conj(A[i + (size_t)m * j]) * y[i];
            x[j] = s;
            nx += std::norm(s);
        }
        nx = std::sqrt(nx);
        if (nx == 0) break;
        for (auto& z : x) z /= nx;
        smax = std::sqrt(nx);
    }
    const double lam = reg * smax;
    const int ma = m + n;
    std::vector<cd> M((size_t)ma * n, 0.0);
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < m; ++i) M[i + (size_t)ma * j] = A[i + (size_t)m * j];
        M[m + j + (size_t)ma * j] = lam;
    }
    const std::vector<cd> Q = qr_q(ma, n, M);
    std::vector<cd> R((size_t)n * n, 0.0);   // Q^H M
    for (int j = 0; j < n; ++j)
        for (int i = 0; i <= j; ++i) {
            cd s = 0.0;
            for (int k = 0; k < ma; ++k) s += std::conj(Q[k + (size_t)ma * i]) * M[k + (size_t)ma * j];
            R[i + (size_t)n * j] = s;
        }
    const std::vector<cd> Ri = upper_inv(n, R);
    std::vector<cd> X((size_t)n * m, 0.0);   // R^-1 Q1^H
    for (int r = 0; r < m; ++r)
        for (int i = 0; i < n; ++i) {
            cd s = 0.0;
            for (int k = i; k < n; ++k) s += Ri[i + (size_t)n * k] * std::conj(Q[r + (size_t)ma * k]);
            X[i + (size_t)n * r] = s;
        }
    return X;
}

// Cholesky A = R^H R of a Hermitian positive definite n x n matrix; returns R
// (upper triangular) or an empty vector when A is not positive definite.
inline std::vector<cd> cholesky_upper(int n, const std::vector<cd>& A) {
    std::vector<cd> R((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[j + (size_t)n * j].real();
        for (int k = 0; k < j; ++k) d -= std::norm(R[k + (size_t)n * j]);
        if (!(d > 0)) return {};
        const double rjj = std::sqrt(d);
        R[j + (size_t)n * j] = rjj;
        for (int i = j + 1; i < n; ++i) {
            cd s = A[j + (size_t)n * i];
            for (int k = 0; k < j; ++k) s -= std::conj(R[k + (size_t)n * j]) * R[k + (size_t)n * i];
            R[j + (size_t)n * i] = s / rjj;
        }
    }
    return R;
}

// Inverse of an upper triangular n x n matrix.
inline std::vector<cd> upper_inv(int n, const std::vector<cd>& R) {
    std::vector<cd> X((size_t)n * n, 0.0);
    for (int j = n - 1; j >= 0; --j) {
        X[j + (size_t)n * j] = 1.0 / R[j + (size_t)n * j];
        for (int i = j - 1; i >= 0; --i) {
            cd s = 0.0;
            for (int k = i + 1; k <= j; ++k) s += R[i + (size_t)n * k] * X[k + (size_t)n * j];
            X[i + (size_t)n * j] = -s / R[i + (size_t)n * i];
        }
    }
    return X;
}

}  // namespace hla
}  // namespace vsie
