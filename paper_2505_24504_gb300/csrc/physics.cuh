// Device model of Sec. 4 (eq. compressible-euler) in (rho, rho u, rho w, rho theta):
// theta-form EOS, convective flux, HLLC numerical flux, viscous flux
// F_v = mu rho (0, grad u, grad w, grad theta).  Templated on the scalar type
// (D64 for the FP64 operator, TL32 for the FP32 tangent-linear operator).
#pragma once

#include "numeric.cuh"

struct PhysC {
    double gamma, R, p0, g, mu;
    double R_over_p0;   // R / p0
    float gammaf, p0f, R_over_p0f, muf;   // float copies for the FP32 tangent
};

// p = p0 (R rho theta / p0)^gamma  (the EOS implied by eq. add-perturbation)
JF_D D64 pressure(D64 E, const PhysC &P, const PowTab *pt) {
    return D64{__dmul_rn(P.p0, pow_gamma_tab(__dmul_rn(P.R_over_p0, E.x), pt))};
}
JF_D TL32 pressure(TL32 E, const PhysC &P, const PowTab *) {
    const float x = P.R_over_p0f * E.v;
    const float p = P.p0f * __powf(x, P.gammaf);
    return TL32{p, P.gammaf * p * frcp(E.v) * E.d};
}

template <class T>
JF_D T sel(bool c, T a, T b) { return c ? a : b; }

// Convective flux F_c(U) . e_D given p.
template <class T, int D>
JF_D void flux_c(const T U[4], T un, T p, T F[4]) {
    F[0] = U[1 + D];
    F[1] = U[1] * un;
    F[2] = U[2] * un;
    F[3] = U[3] * un;
    F[1 + D] = F[1 + D] + p;
}

// One side of a face: the conserved state and the quantities every face of that
// cell needs, 1/rho, p and the sound speed c = sqrt(gamma p / rho).  Cell-based
// kernels compute them once per cell instead of once per face.
template <class T>
struct Side {
    T U[4];
    T ir, p, c;
};

template <class T>
JF_D void side_of(const T U[4], const PhysC &P, const PowTab *pt, Side<T> &S) {
    const auto gam = mkc(P.gamma, P.gammaf, T{});
#pragma unroll
    for (int v = 0; v < 4; ++v) S.U[v] = U[v];
    S.ir = mkc(1.0, 1.0f, T{}) / U[0];
    S.p = pressure(U[3], P, pt);
    S.c = jsqrt(gam * S.p * S.ir);
}

// slip-wall ghost of a side: normal momentum reversed, rho, p and c unchanged
template <class T, int D>
JF_D void mirror_side(const Side<T> &A, Side<T> &G) {
    G = A;
    G.U[1 + D] = -A.U[1 + D];
}

// HLLC flux in direction e_D, normal from L to R.  Davis wave speeds
// S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R), c^2 = gamma p / rho;
// contact speed S*; star states rho*_K = rho_K (S_K - u_K)/(S_K - S*) with normal
// velocity S*, tangential velocity and theta of side K; F*_K = F_K + S_K (U*_K - U_K).
// Branches 0 <= S_L: F_L; 0 <= S*: F*_L; 0 <= S_R: F*_R; else F_R.  Only the side
// the branch selects is evaluated.
template <class T, int D>
JF_D void hllc_s(const Side<T> &L, const Side<T> &R, T H[4]) {
    constexpr int iN = 1 + D, iT = 2 - D;
    const T irL = L.ir, irR = R.ir;
    const T uL = L.U[iN] * irL, uR = R.U[iN] * irR;
    const T pL = L.p, pR = R.p;
    const T cL = L.c, cR = R.c;
    const T a1 = uL - cL, a2 = uR - cR;
    const T SL = sel(val(a1) <= val(a2), a1, a2);
    const T b1 = uL + cL, b2 = uR + cR;
    const T SR = sel(val(b1) >= val(b2), b1, b2);
    const T dL = SL - uL, dR = SR - uR;
    const T num = (pR - pL) + L.U[0] * uL * dL - R.U[0] * uR * dR;
    const T den = L.U[0] * dL - R.U[0] * dR;
    const T Sst = num / den;
    const bool left = val(Sst) >= 0 || val(SL) >= 0;   // integer 0: compared in the scalar's own precision
    const bool pure = val(SL) >= 0 || (!left && val(SR) < 0);
    T U[4], F[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) U[v] = sel(left, L.U[v], R.U[v]);
    const T un = sel(left, uL, uR);
    const T ir = sel(left, irL, irR);
    flux_c<T, D>(U, un, sel(left, pL, pR), F);
    if (pure) {
#pragma unroll
        for (int v = 0; v < 4; ++v) H[v] = F[v];
        return;
    }
    const T S = sel(left, SL, SR);
    const T fac = U[0] * (S - un) / (S - Sst);
    T Us[4];
    Us[0] = fac;
    Us[iN] = fac * Sst;
    Us[iT] = fac * (U[iT] * ir);
    Us[3] = fac * (U[3] * ir);
#pragma unroll
    for (int v = 0; v < 4; ++v) H[v] = F[v] + S * (Us[v] - U[v]);
}

template <class T, int D>
JF_D void hllc(const T UL[4], const T UR[4], const PhysC &P, const PowTab *pt, T H[4]) {
    Side<T> L, R;
    side_of(UL, P, pt, L);
    side_of(UR, P, pt, R);
    hllc_s<T, D>(L, R, H);
}

// Slip-wall ghost: normal momentum reversed.
template <class T, int D>
JF_D void mirror(const T U[4], T G[4]) {
    G[0] = U[0];
    G[1] = U[1];
    G[2] = U[2];
    G[3] = U[3];
    G[1 + D] = -U[1 + D];
}

// A(U) dU with A = mu [[0,0,0,0],[-u,1,0,0],[-w,0,1,0],[-theta,0,0,1]]:
// mu rho (0, d u, d w, d theta) for dU the derivative of U along one direction.
template <class T>
JF_D void viscous(const T U[4], const T dU[4], const PhysC &P, T F[4]) {
    const auto m = mkc(P.mu, P.muf, T{});
    const T ir = mkc(1.0, 1.0f, T{}) / U[0];
    F[0] = mk(0.0, T{});
    F[1] = m * (dU[1] - (U[1] * ir) * dU[0]);
    F[2] = m * (dU[2] - (U[2] * ir) * dU[0]);
    F[3] = m * (dU[3] - (U[3] * ir) * dU[0]);
}

// |v . e_D| + c for pseudo-time step sizes (plain double, not on the residual path).
JF_D double wave_speed(const double U[4], int D, const PhysC &P, const PowTab *pt) {
    const double ir = 1.0 / U[0];
    const double p = P.p0 * pow_gamma_tab(P.R_over_p0 * U[3], pt);
    return fabs(U[1 + D] * ir) + sqrt(P.gamma * p * ir);
}
