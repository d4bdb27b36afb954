// Host-side angle quadratures for the emergent flux F = 2 pi int_0^1 I(mu) mu dmu
// (Sect. 5). Plain C++, no CUDA: the context copies the nodes and flux weights
// into the model constants the emission kernels read.
#pragma once

#include <cmath>

namespace es {

// n-point Gauss-Legendre rule on [0, 1] (n = 4: closed form): nodes mu_j,
// weights w_j with sum_j w_j f(mu_j) ~ int_0^1 f dmu.
inline void gauss_legendre4_01(double *mu, double *w) {
    // on [-1, 1]: x = +-sqrt(3/7 -+ 2/7 sqrt(6/5)), weights (18 +- sqrt(30))/36
    const double xa = std::sqrt(3.0 / 7.0 - 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double xb = std::sqrt(3.0 / 7.0 + 2.0 / 7.0 * std::sqrt(6.0 / 5.0));
    const double wa = (18.0 + std::sqrt(30.0)) / 36.0, wb = (18.0 - std::sqrt(30.0)) / 36.0;
    const double xs[4] = {-xb, -xa, xa, xb}, ws[4] = {wb, wa, wa, wb};
    for (int j = 0; j < 4; ++j) {
        mu[j] = 0.5 * (xs[j] + 1.0);
        w[j] = 0.5 * ws[j];
    }
}

// n-point (n <= 8) Gaussian rule for int_0^1 f(mu) mu dmu, the Gauss-Jacobi
// rule of the weight (1 + x) on [-1, 1] mapped by mu = (1 + x)/2, by
// Golub-Welsch: the nodes are the eigenvalues of the Jacobi matrix of the
// weight mu on [0, 1], whose monic three-term recurrence (Jacobi alpha = 0,
// beta = 1, mapped) has diagonal (1 + 1/((2k+1)(2k+3)))/2, k >= 0, and
// off-diagonal sqrt(k(k+1)) / (2(2k+1)), k >= 1; the weights are int_0^1 mu
// dmu = 1/2 times the squared first components of the unit eigenvectors.
// Eigenpairs by cyclic Jacobi rotations. Nodes ascending; W_j with
// sum_j W_j f(mu_j) ~ int_0^1 f(mu) mu dmu.
inline void gauss_jacobi_mu_01(int n, double *mu, double *W) {
    double a[8][8] = {}, v[8][8] = {};
    for (int k = 0; k < n; ++k) {
        a[k][k] = 0.5 * (1.0 + 1.0 / ((2.0 * k + 1.0) * (2.0 * k + 3.0)));
        v[k][k] = 1.0;
        if (k > 0) a[k][k - 1] = a[k - 1][k] = std::sqrt((double)k * (k + 1)) / (2.0 * (2 * k + 1));
    }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) off += a[p][q] * a[p][q];
        if (off < 1e-32) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                if (std::fabs(a[p][q]) < 1e-300) continue;
                // rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) zeroing a_pq in J^T A J
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - s * akq;
                    a[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - s * aqk;
                    a[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = v[k][p], vkq = v[k][q];
                    v[k][p] = c * vkp - s * vkq;
                    v[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int order[8];
    for (int j = 0; j < n; ++j) order[j] = j;
    for (int i = 1; i < n; ++i)   // insertion sort by eigenvalue
        for (int j = i; j > 0 && a[order[j]][order[j]] < a[order[j - 1]][order[j - 1]]; --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int j = 0; j < n; ++j) {
        const int e = order[j];
        mu[j] = a[e][e];
        W[j] = 0.5 * v[0][e] * v[0][e];
    }
}

// Weights c_j of the interpolatory rule of int_0^1 f(mu) dmu at the n <= 8
// nodes mu_j (exact for polynomials of degree n - 1): the solution of
// sum_j c_j mu_j^k = 1 / (k + 1), k = 0 .. n-1, by Gaussian elimination with
// partial pivoting. At Gauss-Legendre nodes these are the Gauss-Legendre
// weights; the delta-EAA takes the mean intensity J with them.
inline void interp_weights_01(int n, const double *mu, double *c) {
    double a[8][9];
    for (int k = 0; k < n; ++k) {
        for (int j = 0; j < n; ++j) a[k][j] = std::pow(mu[j], (double)k);
        a[k][n] = 1.0 / (k + 1.0);
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
        for (int j = 0; j <= n; ++j) {
            const double t = a[col][j];
            a[col][j] = a[piv][j];
            a[piv][j] = t;
        }
        for (int r = col + 1; r < n; ++r) {
            const double fct = a[r][col] / a[col][col];
            for (int j = col; j <= n; ++j) a[r][j] -= fct * a[col][j];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = a[r][n];
        for (int j = r + 1; j < n; ++j) acc -= a[r][j] * c[j];
        c[r] = acc / a[r][r];
    }
}

}  // namespace es
