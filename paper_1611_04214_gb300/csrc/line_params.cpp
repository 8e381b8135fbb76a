// Host-side FP64 setup of one Helmholtz line inverse H_c = (I - c d_xx)^{-1} (Sec. 3.2).
//
// Local quadrature weights.  J^L_j = (nu/2) int_0^1 e^{-nu t} v(x_j - t h) dt with v replaced
// by the Lagrange interpolant through the stencil nodes x_{j+o}; J^R_j likewise with
// v(x_j + t h).  Writing l_o(s) = sum_k a_{o,k} s^k, the weights are
//     wL_o = (nu/2) sum_k a_{o,k} (-1)^k m_k(nu),   wR_o = (nu/2) sum_k a_{o,k} m_k(nu),
// with the moments m_k(nu) = int_0^1 e^{-nu t} t^k dt.  For M = 2 this is the paper's P, Q, R
// (times the 1/2 of Eq. IL).  The moments come from their power series for nu <= 2 (no
// cancellation: terms are bounded by e^2) and from the upward recursion
// m_k = (k m_{k-1} - e^{-nu}) / nu for nu > 2 (error growth bounded by k!/nu^k <= 12).
// The printed closed forms of P, Q, R are not used: they cancel catastrophically for small nu.
//
// Boundary correction (Eq. homogeneous and its analogues): with I_0 = I^R_0, I_N = I^L_N,
//   periodic   B_a = I_N/(1-mu), B_b = I_0/(1-mu)
//   Neumann    B_a = (I_0 + mu I_N)/(1-mu^2), B_b = (I_N + mu I_0)/(1-mu^2)
//   Dirichlet  B_a = -(I_0 - mu I_N)/(1-mu^2), B_b = -(I_N - mu I_0)/(1-mu^2)
// (the Neumann / Dirichlet systems follow from the slope L^{-1}_x = alpha (I^R - I^L) plus the
// homogeneous part, the way Sec. 3.2 derives the periodic one).
#include <cmath>
#include <cstring>

#include "molt_internal.h"

namespace molt {

namespace {

// Coefficients (ascending powers of s) of the Lagrange basis polynomial of node `which`
// on the integer nodes offsets[0..np-1].
void lagrange_coeffs(const int* offsets, int np, int which, double* coef) {
    for (int k = 0; k < np; ++k) coef[k] = 0.0;
    coef[0] = 1.0;
    int deg = 0;
    double denom = 1.0;
    for (int m = 0; m < np; ++m) {
        if (m == which) continue;
        // multiply by (s - x_m)
        for (int k = deg + 1; k >= 1; --k) coef[k] = coef[k - 1] - offsets[m] * coef[k];
        coef[0] = -offsets[m] * coef[0];
        ++deg;
        denom *= static_cast<double>(offsets[which] - offsets[m]);
    }
    for (int k = 0; k <= deg; ++k) coef[k] /= denom;
}

void moments(double nu, int kmax, double* m) {
    if (nu <= 2.0) {
        for (int k = 0; k <= kmax; ++k) {
            // sum_{j>=0} (-nu)^j / (j! (j + k + 1))
            double term = 1.0, sum = 0.0;
            for (int j = 0; j < 200; ++j) {
                double add = term / static_cast<double>(j + k + 1);
                sum += add;
                if (std::fabs(add) < 1e-19 * std::fabs(sum) && j > 4) break;
                term *= -nu / static_cast<double>(j + 1);
            }
            m[k] = sum;
        }
    } else {
        const double e = std::exp(-nu);
        m[0] = -std::expm1(-nu) / nu;
        for (int k = 1; k <= kmax; ++k) m[k] = (k * m[k - 1] - e) / nu;
    }
}

}  // namespace

bool quadrature_weights(double nu, int M, const int* offsets, int side, double* w) {
    if (!(nu > 0.0) || M < 1 || M > kMaxM || offsets == nullptr || w == nullptr) return false;
    const int np = M + 1;
    double mom[kMaxStencil];
    moments(nu, M, mom);
    double coef[kMaxStencil + 1];
    for (int o = 0; o < np; ++o) {
        lagrange_coeffs(offsets, np, o, coef);
        double acc = 0.0;
        for (int k = 0; k <= M; ++k) {
            const double sgn = (side == 0 && (k & 1)) ? -1.0 : 1.0;
            acc += sgn * coef[k] * mom[k];
        }
        w[o] = 0.5 * nu * acc;
    }
    return true;
}

bool build_line_params(double c, double h, int n, int M, int bc, LineParams<double>* p,
                       const char** err) {
    std::memset(p, 0, sizeof(*p));
    if (!(c > 0.0) || !(h > 0.0) || !std::isfinite(c)) { *err = "c and h must be positive"; return false; }
    if (M != 2 && M != 4 && M != 6) { *err = "quadrature order M must be 2, 4 or 6"; return false; }
    if (bc < BC_PERIODIC || bc > BC_DIRICHLET) { *err = "unknown boundary condition"; return false; }
    const int N = (bc == BC_PERIODIC) ? n : n - 1;
    if (N < M + 1) { *err = "line too short for the quadrature order"; return false; }
    const double nu = h / std::sqrt(c);
    const double d = std::exp(-nu);
    p->n = n;
    p->N = N;
    p->M = M;
    p->bc = bc;
    p->d = d;
    p->nu = nu;
    const int H = M / 2;
    int offs[kMaxStencil];
    for (int o = 0; o <= M; ++o) offs[o] = o - H;
    if (!quadrature_weights(nu, M, offs, 0, p->wl) || !quadrature_weights(nu, M, offs, 1, p->wr)) {
        *err = "quadrature weights failed";
        return false;
    }
    if (bc != BC_PERIODIC) {
        // Left wall: stencil on nodes 0..M, offsets relative to node j are (0..M) - j.
        for (int j = 1; j <= H - 1; ++j) {
            for (int o = 0; o <= M; ++o) offs[o] = o - j;
            quadrature_weights(nu, M, offs, 0, p->wlA[j - 1]);
        }
        for (int j = 0; j <= H - 1; ++j) {
            for (int o = 0; o <= M; ++o) offs[o] = o - j;
            quadrature_weights(nu, M, offs, 1, p->wrA[j]);
        }
        // Right wall: stencil on nodes N-M..N.
        const int jb = N - H + 1;
        for (int j = jb; j <= N; ++j) {
            for (int o = 0; o <= M; ++o) offs[o] = (N - M + o) - j;
            quadrature_weights(nu, M, offs, 0, p->wlB[j - jb]);
        }
        for (int j = jb; j <= N - 1; ++j) {
            for (int o = 0; o <= M; ++o) offs[o] = (N - M + o) - j;
            quadrature_weights(nu, M, offs, 1, p->wrB[j - jb]);
        }
    }
    const double mu = std::exp(-nu * N);
    if (bc == BC_PERIODIC) {
        p->inv1mmu = 1.0 / (-std::expm1(-nu * N));
    } else {
        const double q = 1.0 / (-std::expm1(-2.0 * nu * N));   // 1 / (1 - mu^2)
        if (bc == BC_NEUMANN) {
            p->bAA = q;        p->bAB = mu * q;
            p->bBA = mu * q;   p->bBB = q;
        } else {
            p->bAA = -q;       p->bAB = mu * q;
            p->bBA = mu * q;   p->bBB = -q;
        }
    }
    return true;
}

template <typename T>
LineParams<T> cast_line_params(const LineParams<double>& s) {
    LineParams<T> p;
    std::memset(&p, 0, sizeof(p));
    p.n = s.n;
    p.N = s.N;
    p.M = s.M;
    p.bc = s.bc;
    p.d = static_cast<T>(s.d);
    p.nu = static_cast<T>(s.nu);
    for (int o = 0; o < kMaxStencil; ++o) {
        p.wl[o] = static_cast<T>(s.wl[o]);
        p.wr[o] = static_cast<T>(s.wr[o]);
        for (int j = 0; j < kMaxWall; ++j) {
            p.wlA[j][o] = static_cast<T>(s.wlA[j][o]);
            p.wrA[j][o] = static_cast<T>(s.wrA[j][o]);
            p.wlB[j][o] = static_cast<T>(s.wlB[j][o]);
            p.wrB[j][o] = static_cast<T>(s.wrB[j][o]);
        }
    }
    p.bAA = s.bAA;
    p.bAB = s.bAB;
    p.bBA = s.bBA;
    p.bBB = s.bBB;
    p.inv1mmu = s.inv1mmu;
    return p;
}

template LineParams<float> cast_line_params<float>(const LineParams<double>&);
template LineParams<double> cast_line_params<double>(const LineParams<double>&);

}  // namespace molt
