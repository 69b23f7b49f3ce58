// Host construction of the fixed tables, in long double.
//  * Gauss-Legendre nodes by Newton's method on the three-term recurrence of
//    P_{k+1}, weights 2 / ((1 - x^2) P'(x)^2)  (Sec. 2.1: nodal basis on GL nodes).
//  * Nodal differentiation by the barycentric formula D[a][q] = (lam_q/lam_a)/(x_a - x_q),
//    diagonal from the zero row sum.
//  * Basis values l_a(x) by the product formula; l_a'(x) = l_a(x) sum_{b != a} 1/(x - x_b)
//    at the element ends.
//  * Subcell interpolation V[i][a] = l_a(c_i) (Sec. 3.2.1) and its inverse by
//    Gauss-Jordan elimination.
//  * Modified Newton-Cotes weights on [0,1] at the subcell centres as exact
//    integrals of the Lagrange polynomials through those centres (Sec. 3.3,
//    Appendix A).
//  * x^gamma tables for the table-driven power (Tang-style table reduction and a
//    binomial series): 2^(e gamma), (1 + i/256)^gamma, 1/(1 + i/256), C(gamma, n).
#include <math.h>
#include <string.h>

#include "internal.h"

typedef long double LD;

static void legendre(int n, LD x, LD *p, LD *dp) {
    LD p0 = 1.0L, p1 = x;
    if (n == 0) {
        *p = 1.0L;
        *dp = 0.0L;
        return;
    }
    for (int m = 2; m <= n; ++m) {
        const LD p2 = ((2 * m - 1) * x * p1 - (m - 1) * p0) / m;
        p0 = p1;
        p1 = p2;
    }
    *p = p1;
    *dp = n * (x * p1 - p0) / (x * x - 1.0L);
}

static void gauss_legendre(int n, LD *x, LD *w) {
    const LD pi = 3.141592653589793238462643383279502884L;
    for (int i = 0; i < n; ++i) {
        LD z = cosl(pi * (i + 0.75L) / (n + 0.5L));
        for (int it = 0; it < 100; ++it) {
            LD p, dp;
            legendre(n, z, &p, &dp);
            const LD dz = p / dp;
            z -= dz;
            if (fabsl(dz) < 1e-19L) break;
        }
        LD p, dp;
        legendre(n, z, &p, &dp);
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0L / ((1.0L - z * z) * dp * dp);
    }
}

static LD lag(const LD *xn, int n, int a, LD x) {
    LD r = 1.0L;
    for (int b = 0; b < n; ++b)
        if (b != a) r *= (x - xn[b]) / (xn[a] - xn[b]);
    return r;
}

static LD dlag_end(const LD *xn, int n, int a, LD x) {   // x not a node
    LD s = 0.0L;
    for (int b = 0; b < n; ++b)
        if (b != a) s += 1.0L / (x - xn[b]);
    return lag(xn, n, a, x) * s;
}

static void invert(int n, LD A[5][5], LD Ai[5][5]) {
    LD M[5][10];
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j) M[i][j] = j < n ? A[i][j] : (j - n == i ? 1.0L : 0.0L);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabsl(M[r][col]) > fabsl(M[piv][col])) piv = r;
        for (int j = 0; j < 2 * n; ++j) {
            const LD t = M[col][j];
            M[col][j] = M[piv][j];
            M[piv][j] = t;
        }
        const LD d = M[col][col];
        for (int j = 0; j < 2 * n; ++j) M[col][j] /= d;
        for (int r = 0; r < n; ++r)
            if (r != col) {
                const LD f = M[r][col];
                for (int j = 0; j < 2 * n; ++j) M[r][j] -= f * M[col][j];
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ai[i][j] = M[i][j + n];
}

static void subcell_average_table(const LD *x, int n, LD P[5][5]);

void jf_build_tables(int k, DGTab *T) {
    memset(T, 0, sizeof(*T));
    const int n = k + 1;
    T->np1 = n;
    LD x[5], w[5];
    gauss_legendre(n, x, w);
    LD lam[5];
    for (int a = 0; a < n; ++a) {
        LD p = 1.0L;
        for (int b = 0; b < n; ++b)
            if (b != a) p *= (x[a] - x[b]);
        lam[a] = 1.0L / p;
    }
    LD D[5][5];
    for (int a = 0; a < n; ++a) {
        LD diag = 0.0L;
        for (int q = 0; q < n; ++q)
            if (q != a) {
                D[a][q] = (lam[q] / lam[a]) / (x[a] - x[q]);
                diag -= D[a][q];
            }
        D[a][a] = diag;
    }
    for (int a = 0; a < n; ++a) {
        T->xi[a] = (double)x[a];
        T->w[a] = (double)w[a];
        T->lp[a] = (double)lag(x, n, a, 1.0L);
        T->lm[a] = (double)lag(x, n, a, -1.0L);
        T->dlp[a] = (double)dlag_end(x, n, a, 1.0L);
        T->dlm[a] = (double)dlag_end(x, n, a, -1.0L);
        T->lpw[a] = (double)(lag(x, n, a, 1.0L) / w[a]);
        T->lmw[a] = (double)(lag(x, n, a, -1.0L) / w[a]);
        T->dlpw[a] = (double)(dlag_end(x, n, a, 1.0L) / w[a]);
        T->dlmw[a] = (double)(dlag_end(x, n, a, -1.0L) / w[a]);
        for (int q = 0; q < n; ++q) {
            T->Dn[a][q] = (double)D[a][q];
            // weak-form derivative: w_q l_a'(x_q) / w_a, and l_a'(x_q) = D[q][a]
            T->Dw[a][q] = (double)(w[q] * D[q][a] / w[a]);
        }
    }
    LD V[5][5], Vi[5][5];
    for (int i = 0; i < n; ++i) {
        const LD ci = -1.0L + (2.0L * i + 1.0L) / n;
        for (int a = 0; a < n; ++a) V[i][a] = lag(x, n, a, ci);
    }
    invert(n, V, Vi);
    LD Pa[5][5], Pi[5][5];
    subcell_average_table(x, n, Pa);
    invert(n, Pa, Pi);
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < n; ++a) {
            T->V[i][a] = (double)V[i][a];
            T->Vinv[i][a] = (double)Vi[i][a];
            T->P[i][a] = (double)Pa[i][a];
            T->Pinv[i][a] = (double)Pi[i][a];
        }
    // midpoint weights: integral over [0,1] of the Lagrange polynomial through
    // the centres G_j = (2j+1)/(2n), expanded in monomials
    LD G[5];
    for (int j = 0; j < n; ++j) G[j] = (2.0L * j + 1.0L) / (2.0L * n);
    for (int i = 0; i < n; ++i) {
        LD coef[6] = {1.0L, 0, 0, 0, 0, 0};
        int deg = 0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const LD s = 1.0L / (G[i] - G[j]);
            LD nc[6] = {0, 0, 0, 0, 0, 0};
            for (int m = 0; m <= deg; ++m) {
                nc[m + 1] += coef[m] * s;
                nc[m] -= coef[m] * G[j] * s;
            }
            ++deg;
            for (int m = 0; m <= deg; ++m) coef[m] = nc[m];
        }
        LD integ = 0.0L;
        for (int m = 0; m <= deg; ++m) integ += coef[m] / (m + 1);
        T->om[i] = (double)integ;
    }
}

// P[i][a] = mean of l_a over subcell i of [-1,1]: the L2 projection onto the
// subcells (Sec. 3.2.1), from the monomial expansion of l_a integrated exactly.
static void subcell_average_table(const LD *x, int n, LD P[5][5]) {
    for (int a = 0; a < n; ++a) {
        LD coef[6] = {1.0L, 0, 0, 0, 0, 0};
        int deg = 0;
        for (int b = 0; b < n; ++b) {
            if (b == a) continue;
            const LD s = 1.0L / (x[a] - x[b]);
            LD nc[6] = {0, 0, 0, 0, 0, 0};
            for (int m = 0; m <= deg; ++m) {
                nc[m + 1] += coef[m] * s;
                nc[m] -= coef[m] * x[b] * s;
            }
            ++deg;
            for (int m = 0; m <= deg; ++m) coef[m] = nc[m];
        }
        for (int i = 0; i < n; ++i) {
            const LD lo = -1.0L + 2.0L * i / n, hi = -1.0L + 2.0L * (i + 1) / n;
            LD acc = 0.0L;
            for (int m = 0; m <= deg; ++m) acc += coef[m] * (powl(hi, m + 1) - powl(lo, m + 1)) / (m + 1);
            P[i][a] = acc / (hi - lo);
        }
    }
}

void jf_build_powtab(double gamma, PowTab *P) {
    memset(P, 0, sizeof(*P));
    const LD g = gamma;
    P->gamma = gamma;
    for (int e = -32; e < 32; ++e) P->pe[e + 32] = (double)exp2l((LD)e * g);
    for (int i = 0; i < 256; ++i) {
        const LD m = 1.0L + i / 256.0L;
        P->mg[i] = (double)powl(m, g);
        P->minv[i] = (double)(1.0L / m);
    }
    LD c = 1.0L;
    for (int nn = 1; nn <= 6; ++nn) {
        c = c * (g - (nn - 1)) / nn;
        P->c[nn] = (double)c;
    }
}

// Environmental atmosphere at height z: U (4) and dU/dz (4).
void jf_background(const jfnk_physics *ph, double z, double U[4], double dU[4]) {
    const LD R = (LD)ph->cp - (LD)ph->cv;
    for (int v = 0; v < 4; ++v) U[v] = dU[v] = 0.0;
    if (ph->background == 0) {
        const LD th = ph->theta0;
        const LD T = th - (LD)z * ph->g / ph->cp;
        const LD dT = -(LD)ph->g / ph->cp;
        const LD ex = (LD)ph->cp / R;
        const LD p = ph->p0 * powl(T / th, ex);
        const LD dp = ph->p0 * ex * powl(T / th, ex - 1.0L) * dT / th;
        const LD rho = p / (R * T);
        const LD drho = (dp * T - p * dT) / (R * T * T);
        U[0] = (double)rho;
        U[3] = (double)(rho * th);
        dU[0] = (double)drho;
        dU[3] = (double)(drho * th);
    } else if (ph->background == 2) {
        const LD gg = ph->g, th0 = ph->theta0;
        const LD H = gg / ((LD)ph->N_bv * ph->N_bv);
        const LD alpha = gg * H / ((LD)ph->cp * th0);
        const LD ez = expl((LD)z / H);
        const LD th = th0 * ez;
        const LD T = th0 * (alpha - (alpha - 1.0L) * ez);
        const LD p = ph->p0 * expl((LD)ph->cp / R * (logl(T / th0) - (LD)z / H));
        const LD rho = p / (R * T);
        const LD dT = -th0 * (alpha - 1.0L) * ez / H;
        const LD dp = -rho * gg;
        const LD drho = (dp * T - p * dT) / (R * T * T);
        U[0] = (double)rho;
        U[1] = (double)(rho * ph->ubg);
        U[3] = (double)(rho * th);
        dU[0] = (double)drho;
        dU[1] = (double)(drho * ph->ubg);
        dU[3] = (double)(drho * th + rho * th / H);
    } else {
        const LD rho = (LD)ph->p0 / (R * ph->theta0);
        U[0] = (double)rho;
        U[1] = (double)(rho * ph->ubg);
        U[2] = (double)(rho * ph->wbg);
        U[3] = (double)(rho * ph->theta0);
    }
}

// theta~ of the environmental atmosphere at height z (insertion, eq. add-perturbation)
double jf_background_theta(const jfnk_physics *ph, double z) {
    if (ph->background == 2) {
        const LD H = (LD)ph->g / ((LD)ph->N_bv * ph->N_bv);
        return (double)((LD)ph->theta0 * expl((LD)z / H));
    }
    return ph->theta0;
}

// Coefficient p0^(R/c_p) p~^(1/gamma) / R of the pressure-preserving insertion
// (eq. add-perturbation) at height z: rho = coef / (theta~ + theta').
double jf_insert_coef(const jfnk_physics *ph, double z) {
    const LD R = (LD)ph->cp - (LD)ph->cv;
    const LD gam = (LD)ph->cp / ph->cv;
    LD p;
    if (ph->background == 0) {
        const LD T = (LD)ph->theta0 - (LD)z * ph->g / ph->cp;
        p = ph->p0 * powl(T / ph->theta0, (LD)ph->cp / R);
    } else if (ph->background == 2) {
        const LD H = (LD)ph->g / ((LD)ph->N_bv * ph->N_bv);
        const LD alpha = (LD)ph->g * H / ((LD)ph->cp * ph->theta0);
        const LD T = (LD)ph->theta0 * (alpha - (alpha - 1.0L) * expl((LD)z / H));
        p = ph->p0 * expl((LD)ph->cp / R * (logl(T / ph->theta0) - (LD)z / H));
    } else {
        p = ph->p0;   // uniform state rho = p0/(R theta0) has p = p0
    }
    return (double)(powl((LD)ph->p0, R / ph->cp) * powl(p, 1.0L / gam) / R);
}
