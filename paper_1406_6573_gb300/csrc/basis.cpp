// One-dimensional rules and tables for the sum-factorised element kernels.
//
// Section 3.2.1: Lagrange velocity basis on the Gauss-Lobatto (GLL) nodes of
// degree k, tensor Gauss quadrature with q = k + 1 points per direction.
// Section 3.2.2 / 6: discontinuous pressure, P_{k-1} (here Legendre products)
// or Q_{k-2} (Lagrange on the (k-1) Gauss points).  The hanging-node restriction
// interpolates the coarse trace to the half-interval nodes (hanging-node figure
// of Section 3.2.1), one 1-D matrix per half, applied in tensor form
// (Section 3.3: "the same one-dimensional kernels").
//
// Roots are found by Newton's method on Legendre polynomials; Lagrange values
// use the barycentric form.
#include <cmath>
#include <cstring>

#include "common.h"

namespace stokes {
namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence.
void legendre(int n, double x, double& p, double& dp) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { p = 1.0; dp = 0.0; return; }
    for (int m = 1; m < n; ++m) {
        double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
        p0 = p1; p1 = p2;
    }
    p = p1;
    // derivative from n (P_{n-1} - x P_n) = (1 - x^2) P_n'
    if (std::fabs(std::fabs(x) - 1.0) < 1e-15) {
        dp = (x > 0 ? 1.0 : (n % 2 ? 1.0 : -1.0)) * 0.5 * n * (n + 1);
    } else {
        dp = n * (p0 - x * p1) / (1.0 - x * x);
    }
}

void gauss_rule(int q, double* x, double* w) {
    for (int i = 0; i < q; ++i) {
        // initial guess near the i-th root counted from -1
        double t = -std::cos(M_PI * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(q, t, p, dp);
            double dt = p / dp;
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        double p, dp;
        legendre(q, t, p, dp);
        x[i] = t;
        w[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

void lobatto_rule(int n1, double* x, double* w) {
    int k = n1 - 1;
    x[0] = -1.0; x[k] = 1.0;
    for (int i = 1; i < k; ++i) {
        double t = -std::cos(M_PI * i / k);
        for (int it = 0; it < 100; ++it) {
            double p, dp;
            legendre(k, t, p, dp);
            // P_k'' from the Legendre equation
            double ddp = (2.0 * t * dp - k * (k + 1) * p) / (1.0 - t * t);
            double dt = dp / ddp;
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        x[i] = t;
    }
    for (int i = 0; i < n1; ++i) {
        double p, dp;
        legendre(k, x[i], p, dp);
        w[i] = 2.0 / (k * (k + 1) * p * p);
    }
}

// Barycentric weights lambda_m = 1 / prod_{l != m} (x_m - x_l).
void bary_weights(int n, const double* x, double* lam) {
    for (int m = 0; m < n; ++m) {
        double pr = 1.0;
        for (int l = 0; l < n; ++l)
            if (l != m) pr *= (x[m] - x[l]);
        lam[m] = 1.0 / pr;
    }
}

// Values of all n Lagrange polynomials on nodes x at the point t.
void lagrange_values(int n, const double* x, double t, double* out) {
    double lam[N1MAX];
    bary_weights(n, x, lam);
    for (int m = 0; m < n; ++m) {
        if (t == x[m]) {
            for (int l = 0; l < n; ++l) out[l] = (l == m) ? 1.0 : 0.0;
            return;
        }
    }
    double den = 0.0;
    for (int m = 0; m < n; ++m) den += lam[m] / (t - x[m]);
    for (int m = 0; m < n; ++m) out[m] = (lam[m] / (t - x[m])) / den;
}

}  // namespace

void build_tables(int k, int pspace, Tables1D& t) {
    std::memset(&t, 0, sizeof(t));
    t.k = k;
    t.n1 = k + 1;
    t.q = k + 1;
    const int n1 = t.n1, q = t.q;
    lobatto_rule(n1, t.gll, t.gllw);
    gauss_rule(q, t.gauss, t.gaussw);
    // snap the GLL midpoint of even degrees to exactly 0
    if (k % 2 == 0) t.gll[k / 2] = 0.0;
    for (int iq = 0; iq < q; ++iq) lagrange_values(n1, t.gll, t.gauss[iq], t.B[iq]);
    // collocation derivative on the Gauss points
    double lam[N1MAX];
    bary_weights(q, t.gauss, lam);
    for (int i = 0; i < q; ++i) {
        double diag = 0.0;
        for (int m = 0; m < q; ++m) {
            if (m == i) continue;
            t.Dg[i][m] = (lam[m] / lam[i]) / (t.gauss[i] - t.gauss[m]);
            diag -= t.Dg[i][m];
        }
        t.Dg[i][i] = diag;
    }
    for (int b = 0; b < 2; ++b)
        for (int i = 0; i < n1; ++i)
            lagrange_values(n1, t.gll, 0.5 * (t.gll[i] + 2.0 * b - 1.0), t.I[b][i]);
    // pressure basis
    int np = 0;
    if (pspace == STOKES_PRESSURE_P) {
        for (int c = 0; c < k; ++c)
            for (int b = 0; b < k - c; ++b)
                for (int a = 0; a < k - b - c; ++a) {
                    t.pmode[np][0] = a; t.pmode[np][1] = b; t.pmode[np][2] = c; ++np;
                }
        for (int iq = 0; iq < q; ++iq)
            for (int a = 0; a < k; ++a) {
                double p, dp;
                legendre(a, t.gauss[iq], p, dp);
                t.P1[iq][a] = p;
            }
    } else {
        const int m = k - 1;
        for (int c = 0; c < m; ++c)
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < m; ++a) {
                    t.pmode[np][0] = a; t.pmode[np][1] = b; t.pmode[np][2] = c; ++np;
                }
        double gx[N1MAX], gw[N1MAX];
        gauss_rule(m, gx, gw);
        for (int iq = 0; iq < q; ++iq) lagrange_values(m, gx, t.gauss[iq], t.P1[iq]);
    }
    t.npr = np;
}

double eval_field(const stokes_field& f, double x, double y) {
    double s = f.mean;
    for (int m = 0; m < f.n_modes; ++m)
        s += f.amp[m] * std::cos(f.kx[m] * x + f.ky[m] * y + f.phase[m]);
    return s;
}

}  // namespace stokes
