// DG operator f = M^-1 L_h(U') on the GPU (Sec. 2.1; well-balanced form of Sec. 4).
//
// Two launches per evaluation:
//  k_faces   one thread per face point.  Traces of U' from both sides (and the
//            normal-gradient traces for the viscous terms), HLLC^pert =
//            HLLC(U'+Ubar) - HLLC(Ubar), symmetric interior penalty terms, slip
//            walls by a mirrored ghost.  Every face flux is computed once and
//            stored: Phi = H - {F_v.n} + eta [U] for the lift with l_a(+-1), and
//            the two symmetry terms 1/2 A(U_side) [U] for the lift with l_a'(+-1).
//  k_volume  a block holds EPB elements, one thread per node.  Fluxes
//            F_c^pert - F_v at the node, the weak-form derivative by sum
//            factorisation over the (k+1) nodes of the row / column (tables in
//            shared memory), gravity source, lift of the stored face terms and
//            the mode's epilogue (residual, FD product, Newton residual G or a
//            pseudo-time smoothing step).
// The same kernels run on D64 (FP64 residual and finite-difference products)
// and on TL32 (FP32 tangent-linear products for the FP32 preconditioner).
#include <vector>

#include "internal.h"

namespace {

struct DGK {
    int nx, nz, n_el, periodic;
    double two_hx, two_hz, g, mu, eta_x, eta_z;
    float two_hxf, two_hzf, gf, eta_xf, eta_zf;   // float copies for the FP32 tangent
    float tlp[5], tlm[5], tdlp[5], tdlm[5];       // trace tables l_a(+-1), l_a'(+-1) in float
    // volume tables with the 2/h factors folded in, built on the host in both
    // precisions: Dx = (2/hx) Dw, Dz = (2/hz) Dw, lift[0..3] x-lifts, lift[4..7] z-lifts
    double Dx[5][5], Dz[5][5], lift[8][5];
    float Dxf[5][5], Dzf[5][5], Dnf[5][5], liftf[8][5];
    PhysC pc;
    const PowTab *pt;
    const double *ubv, *dubv, *fbx, *fbz, *hbx, *hbxw, *ubh, *dubh, *hbz;
    const float *ubvf, *dubvf, *ubhf, *dubhf;
    DGTab tab;
};

template <class T> struct OutT;
template <> struct OutT<D64> { typedef double type; };
template <> struct OutT<TL32> { typedef float type; };
JF_D double outv(D64 a) { return a.x; }
JF_D float outv(TL32 a) { return a.d; }

// Input of the perturbation state at global index i:
// IN 0: U'; IN 1: U' + eps y (FP64); IN 2: TL32 (U', y32)
template <class T, int IN> struct Loader;
template <> struct Loader<D64, 0> {
    const double *U;
    JF_D void prepare() {}
    JF_D D64 operator()(size_t i) const { return D64{U[i]}; }
};
template <> struct Loader<D64, 1> {
    const double *U, *y, *epsp;   // eps is a device scalar written by a reduction
    double eps;
    JF_D void prepare() { eps = *epsp; }
    JF_D D64 operator()(size_t i) const { return D64{__fma_rn(eps, y[i], U[i])}; }
};
template <> struct Loader<TL32, 2> {
    const float *U;
    const float *y;
    JF_D void prepare() {}
    JF_D TL32 operator()(size_t i) const { return TL32{U[i], y[i]}; }
};

__device__ __forceinline__ void load_powtab(PowTab *s, const PowTab *g) {
    const double *src = reinterpret_cast<const double *>(g);
    double *dst = reinterpret_cast<double *>(s);
    const int n = sizeof(PowTab) / sizeof(double);
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// background values: FP64 tables for D64, FP32 copies for TL32
JF_D D64 bgs(const double *d, const float *, size_t i, D64) { return D64{d[i]}; }
JF_D TLc bgs(const double *, const float *f, size_t i, TL32) { return TLc{f[i]}; }
template <class T>
JF_D T bg(const double *a, size_t i) { return mk(a[i], T{}); }

// ---------------------------------------------------------------------------
// Value and (viscous) derivative traces along a line of NP1 nodes i0 + q st with
// the end-point tables (pa: l_q(+-1), pd: l_q'(+-1)).
template <class T, int IN, int NP1, bool VISC>
JF_D void line_trace(const Loader<T, IN> &ld, size_t i0, size_t st, const double *pa, const float *paf,
                     const double *pd, const float *pdf, T &a, T &d) {
    a = mk(0.0, T{});
    d = mk(0.0, T{});
#pragma unroll
    for (int q = 0; q < NP1; ++q) {
        const T u = ld(i0 + q * st);
        a = jfma(mkc(pa[q], paf[q], T{}), u, a);
        if (VISC) d = jfma(mkc(pd[q], pdf[q], T{}), u, d);
    }
}
// The same traces of the FD state U + eps y from the stored traces of U (Newton
// iterate, written by the residual) and the traces of y: tr(U + eps y) =
// tr(U) + eps tr(y) -- the U part is then the same bits as in f(U).
template <int NP1, bool VISC>
JF_D void line_trace_fd(const Loader<D64, 1> &ld, size_t i0, size_t st, const double *pa, const double *pd,
                        double trU, double dU, D64 &a, D64 &d) {
    double ay = 0.0, dy = 0.0;
#pragma unroll
    for (int q = 0; q < NP1; ++q) {
        const double y = ld.y[i0 + q * st];
        ay = __fma_rn(pa[q], y, ay);
        if (VISC) dy = __fma_rn(pd[q], y, dy);
    }
    a = D64{__fma_rn(ld.eps, ay, trU)};
    d = D64{VISC ? __fma_rn(ld.eps, dy, dU) : 0.0};
}

// Body of the face kernel for block `blk` of one operator evaluation; K is the
// launch parameter (single operator) or a member's descriptor in global memory
// (grouped launch over ensemble members).
template <class T, int IN, int NP1, bool VISC>
__device__ __forceinline__ void faces_body(const DGK &K, const Loader<T, IN> &ld0, typename OutT<T>::type *phix,
                                           typename OutT<T>::type *symx, typename OutT<T>::type *phiz,
                                           typename OutT<T>::type *symz, unsigned blk, double *tr_out,
                                           const double *tr_in) {
    typedef typename OutT<T>::type O;
    __shared__ PowTab spt;
    if (IN != 2) load_powtab(&spt, K.pt);   // the FP32 tangent power needs no table
    Loader<T, IN> ld = ld0;
    ld.prepare();
    __syncthreads();
    constexpr int NP = NP1 * NP1;
    const int nx = K.nx, nz = K.nz;
    const size_t N1 = (size_t)K.n_el * NP;
    const long long nvert = (long long)nz * (nx + 1) * NP1;
    const long long nhorz = (long long)(nz + 1) * nx * NP1;
    const long long t = (long long)blk * blockDim.x + threadIdx.x;
    if (t >= nvert + nhorz) return;
    const T zero = mk(0.0, T{});
    const auto half = mkc(0.5, 0.5f, T{});
    T H[4], Phi[4], sL[3], sR[3];
    if (t < nvert) {
        const int s = (int)(t % NP1);
        const int fx = (int)((t / NP1) % (nx + 1));
        const int ez = (int)(t / (NP1 * (nx + 1)));
        const int J = ez * NP1 + s;
        const size_t nrow = (size_t)nz * NP1;
        int eL, eR;
        bool wallL = false, wallR = false;
        if (K.periodic) {
            eL = ez * nx + (fx + nx - 1) % nx;
            eR = ez * nx + fx % nx;
        } else {
            wallL = (fx == 0);
            wallR = (fx == nx);
            eL = ez * nx + (wallL ? 0 : fx - 1);
            eR = ez * nx + (wallR ? nx - 1 : fx);
        }
        // traces: L at xi = +1 (row s), R at xi = -1
        T trL[4], trR[4], gL[4], gR[4];
        const size_t nfp = (size_t)(nvert + nhorz);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            T aL, aR, dL, dR;
            const size_t iL0 = (size_t)v * N1 + (size_t)eL * NP + s * NP1;
            const size_t iR0 = (size_t)v * N1 + (size_t)eR * NP + s * NP1;
            bool done = false;
            if constexpr (IN == 1) {
                if (tr_in) {
                    line_trace_fd<NP1, VISC>(ld, iL0, 1, K.tab.lp, K.tab.dlp, tr_in[(2 * v) * nfp + t],
                                             VISC ? tr_in[(8 + 2 * v) * nfp + t] : 0.0, aL, dL);
                    line_trace_fd<NP1, VISC>(ld, iR0, 1, K.tab.lm, K.tab.dlm, tr_in[(2 * v + 1) * nfp + t],
                                             VISC ? tr_in[(9 + 2 * v) * nfp + t] : 0.0, aR, dR);
                    done = true;
                }
            }
            if (!done) {
                line_trace<T, IN, NP1, VISC>(ld, iL0, 1, K.tab.lp, K.tlp, K.tab.dlp, K.tdlp, aL, dL);
                line_trace<T, IN, NP1, VISC>(ld, iR0, 1, K.tab.lm, K.tlm, K.tab.dlm, K.tdlm, aR, dR);
            }
            if constexpr (IN == 0) {
                if (tr_out) {
                    tr_out[(2 * v) * nfp + t] = outv(aL);
                    tr_out[(2 * v + 1) * nfp + t] = outv(aR);
                    if (VISC) {
                        tr_out[(8 + 2 * v) * nfp + t] = outv(dL);
                        tr_out[(9 + 2 * v) * nfp + t] = outv(dR);
                    }
                }
            }
            trL[v] = aL;
            trR[v] = aR;
            gL[v] = mkc(K.two_hx, K.two_hxf, T{}) * dL;
            gR[v] = mkc(K.two_hx, K.two_hxf, T{}) * dR;
        }
        T UL[4], UR[4], Gh[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            UL[v] = trL[v] + bgs(K.ubv, K.ubvf, v * nrow + J, T{});
            UR[v] = trR[v] + bgs(K.ubv, K.ubvf, v * nrow + J, T{});
        }
        if (wallL) {
            mirror<T, 0>(UR, Gh);
            hllc<T, 0>(Gh, UR, K.pc, &spt, H);
        } else if (wallR) {
            mirror<T, 0>(UL, Gh);
            hllc<T, 0>(UL, Gh, K.pc, &spt, H);
        } else {
            hllc<T, 0>(UL, UR, K.pc, &spt, H);
        }
        const double *hb = wallL ? K.hbxw : (wallR ? K.hbxw + 4 * nrow : K.hbx);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (IN != 2) H[v] = H[v] - bg<T>(hb, v * nrow + J);
            Phi[v] = H[v];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) sL[c] = sR[c] = zero;
        if (VISC && !wallL && !wallR) {
            T FL[4], FR[4], Jp[4], AL[4], AR[4];
            viscous(UL, gL, K.pc, FL);
            viscous(UR, gR, K.pc, FR);
#pragma unroll
            for (int v = 0; v < 4; ++v) Jp[v] = trL[v] - trR[v];
            viscous(UL, Jp, K.pc, AL);
            viscous(UR, Jp, K.pc, AR);
            // interior penalty on the jumps of u, w, theta: eta {A(U)} [U]
            const auto eta = mkc(K.eta_x, K.eta_xf, T{});
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sL[c] = half * AL[c + 1];
                sR[c] = half * AR[c + 1];
                Phi[c + 1] = Phi[c + 1] - half * (FL[c + 1] + FR[c + 1]) + eta * (sL[c] + sR[c]);
            }
        }
        const size_t fb = ((size_t)ez * (nx + 1) + fx) * NP1 + s;
        const size_t fs = (size_t)nz * (nx + 1) * NP1;
#pragma unroll
        for (int v = 0; v < 4; ++v) phix[v * fs + fb] = (O)outv(Phi[v]);
        if (VISC) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                symx[(size_t)c * fs + fb] = (O)outv(sL[c]);
                symx[(size_t)(3 + c) * fs + fb] = (O)outv(sR[c]);
            }
        }
    } else {
        const long long u = t - nvert;
        const int s = (int)(u % NP1);
        const int ex = (int)((u / NP1) % nx);
        const int fz = (int)(u / (NP1 * nx));
        const bool wallB = (fz == 0), wallT = (fz == nz);
        const int eB = (wallB ? 0 : fz - 1) * nx + ex;
        const int eT = (wallT ? nz - 1 : fz) * nx + ex;
        T trB[4], trT[4], gB[4], gT[4];
        const size_t nfp = (size_t)(nvert + nhorz);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            T aB, aT, dB, dT;
            const size_t iB0 = (size_t)v * N1 + (size_t)eB * NP + s;
            const size_t iT0 = (size_t)v * N1 + (size_t)eT * NP + s;
            bool done = false;
            if constexpr (IN == 1) {
                if (tr_in) {
                    line_trace_fd<NP1, VISC>(ld, iB0, NP1, K.tab.lp, K.tab.dlp, tr_in[(2 * v) * nfp + t],
                                             VISC ? tr_in[(8 + 2 * v) * nfp + t] : 0.0, aB, dB);
                    line_trace_fd<NP1, VISC>(ld, iT0, NP1, K.tab.lm, K.tab.dlm, tr_in[(2 * v + 1) * nfp + t],
                                             VISC ? tr_in[(9 + 2 * v) * nfp + t] : 0.0, aT, dT);
                    done = true;
                }
            }
            if (!done) {
                line_trace<T, IN, NP1, VISC>(ld, iB0, NP1, K.tab.lp, K.tlp, K.tab.dlp, K.tdlp, aB, dB);
                line_trace<T, IN, NP1, VISC>(ld, iT0, NP1, K.tab.lm, K.tlm, K.tab.dlm, K.tdlm, aT, dT);
            }
            if constexpr (IN == 0) {
                if (tr_out) {
                    tr_out[(2 * v) * nfp + t] = outv(aB);
                    tr_out[(2 * v + 1) * nfp + t] = outv(aT);
                    if (VISC) {
                        tr_out[(8 + 2 * v) * nfp + t] = outv(dB);
                        tr_out[(9 + 2 * v) * nfp + t] = outv(dT);
                    }
                }
            }
            trB[v] = aB;
            trT[v] = aT;
            gB[v] = mkc(K.two_hz, K.two_hzf, T{}) * dB + bgs(K.dubh, K.dubhf, (size_t)v * (nz + 1) + fz, T{});
            gT[v] = mkc(K.two_hz, K.two_hzf, T{}) * dT + bgs(K.dubh, K.dubhf, (size_t)v * (nz + 1) + fz, T{});
        }
        T UB[4], UT[4], Gh[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            UB[v] = trB[v] + bgs(K.ubh, K.ubhf, (size_t)v * (nz + 1) + fz, T{});
            UT[v] = trT[v] + bgs(K.ubh, K.ubhf, (size_t)v * (nz + 1) + fz, T{});
        }
        if (wallB) {
            mirror<T, 1>(UT, Gh);
            hllc<T, 1>(Gh, UT, K.pc, &spt, H);
        } else if (wallT) {
            mirror<T, 1>(UB, Gh);
            hllc<T, 1>(UB, Gh, K.pc, &spt, H);
        } else {
            hllc<T, 1>(UB, UT, K.pc, &spt, H);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            if (IN != 2) H[v] = H[v] - bg<T>(K.hbz, (size_t)v * (nz + 1) + fz);
            Phi[v] = H[v];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) sL[c] = sR[c] = zero;
        if (VISC && !wallB && !wallT) {
            T FB[4], FT[4], Jp[4], AB[4], AT[4];
            viscous(UB, gB, K.pc, FB);
            viscous(UT, gT, K.pc, FT);
#pragma unroll
            for (int v = 0; v < 4; ++v) Jp[v] = trB[v] - trT[v];
            viscous(UB, Jp, K.pc, AB);
            viscous(UT, Jp, K.pc, AT);
            const auto eta = mkc(K.eta_z, K.eta_zf, T{});
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                sL[c] = half * AB[c + 1];
                sR[c] = half * AT[c + 1];
                Phi[c + 1] = Phi[c + 1] - half * (FB[c + 1] + FT[c + 1]) + eta * (sL[c] + sR[c]);
            }
        }
        const size_t fb = ((size_t)fz * nx + ex) * NP1 + s;
        const size_t fs = (size_t)(nz + 1) * nx * NP1;
#pragma unroll
        for (int v = 0; v < 4; ++v) phiz[v * fs + fb] = (O)outv(Phi[v]);
        if (VISC) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                symz[(size_t)c * fs + fb] = (O)outv(sL[c]);
                symz[(size_t)(3 + c) * fs + fb] = (O)outv(sR[c]);
            }
        }
    }
}

template <class T, int IN, int NP1, bool VISC>
struct k_faces_b {
    static constexpr int TPB = 256, MINB = 4;
    static constexpr bool GROUP = !VISC && std::is_same<T, D64>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<DGK> K,
                                               JfArg<Loader<T, IN>> ld0, JfArg<typename OutT<T>::type *> phix,
                                               JfArg<typename OutT<T>::type *> symx,
                                               JfArg<typename OutT<T>::type *> phiz,
                                               JfArg<typename OutT<T>::type *> symz, JfArg<double *> tr_out,
                                               JfArg<const double *> tr_in) {
        jf_pdl_enter();
        faces_body<T, IN, NP1, VISC>(K, ld0, phix, symx, phiz, symz, jf_bid, tr_out, tr_in);
    }
};
template <class T, int IN, int NP1, bool VISC>
__global__ void __launch_bounds__(256, 4) k_faces(DGK K, Loader<T, IN> ld0, typename OutT<T>::type *phix,
                                               typename OutT<T>::type *symx, typename OutT<T>::type *phiz,
                                               typename OutT<T>::type *symz, double *tr_out, const double *tr_in) {
    k_faces_b<T, IN, NP1, VISC>::run(blockIdx.x, gridDim.x, K, ld0, phix, symx, phiz, symz, tr_out, tr_in);
}

// ---------------------------------------------------------------------------
// elements per volume block: TV = 2 -> ~128 threads, TV = 1 -> ~64 threads
template <int NP1, int TV> struct EPBOf {
    static constexpr int NP = NP1 * NP1;
    static constexpr int T = TV == 2 ? 128 : 64;
    static constexpr int value = (T / NP) > 0 ? (T / NP) : 1;
};

template <class T, int IN, int MODE, int NP1, bool VISC, int TV>
__device__ __forceinline__ void volume_body(const DGK &K, const Loader<T, IN> &ld0, const DGArgs &A,
                                            const typename OutT<T>::type *phix,
                                            const typename OutT<T>::type *symx,
                                            const typename OutT<T>::type *phiz,
                                            const typename OutT<T>::type *symz, unsigned blk) {
    typedef typename OutT<T>::type O;
    constexpr int NP = NP1 * NP1;
    constexpr int EPB = EPBOf<NP1, TV>::value;
    __shared__ PowTab spt;
    __shared__ O sg[2][EPB][4][NP];
    __shared__ T su[VISC ? EPB : 1][4][NP];
    // weak-form derivative and lift tables with the 2/h factors folded in:
    // sDx = (2/hx) Dw, sDz = (2/hz) Dw; sl[0..3] x-lifts, sl[4..7] z-lifts
    __shared__ O sDx[NP1][NP1], sDz[NP1][NP1];
    __shared__ O sDn[NP1][NP1];
    __shared__ O sl[8][NP1];
    __shared__ double sce[2];   // eps and adt / eps of the FD modes: one IEEE division per block
    if ((MODE == DG_JV || MODE == DG_SMOOTH64) && threadIdx.x == 0) {
        const double e0 = *A.eps;
        sce[0] = e0;
        sce[1] = e0 != 0.0 ? A.adt / e0 : 0.0;
    }
    if (IN != 2) load_powtab(&spt, K.pt);
    Loader<T, IN> ld = ld0;
    ld.prepare();
    if (threadIdx.x < NP) {
        const int r = threadIdx.x / NP1, q = threadIdx.x % NP1;
        sDx[r][q] = pick<O>(K.Dx[r][q], K.Dxf[r][q]);
        sDz[r][q] = pick<O>(K.Dz[r][q], K.Dzf[r][q]);
        sDn[r][q] = pick<O>(K.tab.Dn[r][q], K.Dnf[r][q]);
    }
    if (threadIdx.x < NP1) {
        const int q = threadIdx.x;
#pragma unroll
        for (int r = 0; r < 8; ++r) sl[r][q] = pick<O>(K.lift[r][q], K.liftf[r][q]);
    }
    const int le = threadIdx.x / NP;
    const int node = threadIdx.x % NP;
    const int a = node % NP1, b = node / NP1;
    const int e = (int)blk * EPB + le;
    const bool active = (le < EPB) && (e < K.n_el);
    const int nx = K.nx, nz = K.nz;
    const int ez = active ? e / nx : 0, ex = active ? e % nx : 0;
    const size_t N1 = (size_t)K.n_el * NP;
    const size_t nrow = (size_t)nz * NP1;
    const int J = ez * NP1 + b;
    // FP32 tangent modes: face terms and the epilogue's operands are loaded now so
    // that their latency overlaps the flux work below (the FP64 modes are bound by
    // FP64 arithmetic and keep their registers for it)
    constexpr bool PF = (IN == 2);
    const size_t fsx = (size_t)nz * (nx + 1) * NP1, fsz = (size_t)(nz + 1) * nx * NP1;
    const size_t iL = ((size_t)ez * (nx + 1) + ex) * NP1 + b, iR = iL + NP1;
    const size_t iB = ((size_t)ez * nx + ex) * NP1 + a, iT = iB + (size_t)nx * NP1;
    O pxl[4], pxr[4], pzb[4], pzt[4];
    float ef[4], edt = 0.0f;   // operands of the FP32 smoothing mode
    if (PF && active) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            pxl[v] = phix[v * fsx + iL];
            pxr[v] = phix[v * fsx + iR];
            pzb[v] = phiz[v * fsz + iB];
            pzt[v] = phiz[v * fsz + iT];
            if (MODE == DG_TLSMOOTH || (MODE == DG_TLJV && A.rf)) ef[v] = A.rf[(size_t)v * N1 + (size_t)e * NP + node];
        }
        if (MODE == DG_TLSMOOTH) edt = A.dtauf[e];
    }
    __syncthreads();
    T Up[4], U[4];
    if (active) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            Up[v] = ld((size_t)v * N1 + (size_t)e * NP + node);
            U[v] = Up[v] + bgs(K.ubv, K.ubvf, v * nrow + J, T{});
            if (VISC) su[le][v][node] = Up[v];
        }
    }
    __syncthreads();
    if (active) {
        const T ir = mkc(1.0, 1.0f, T{}) / U[0];
        const T p = pressure(U[3], K.pc, &spt);
        T Fx[4], Fz[4];
        flux_c<T, 0>(U, U[1] * ir, p, Fx);
        flux_c<T, 1>(U, U[2] * ir, p, Fz);
        if (IN != 2) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                Fx[v] = Fx[v] - bg<T>(K.fbx, v * nrow + J);
                Fz[v] = Fz[v] - bg<T>(K.fbz, v * nrow + J);
            }
        }
        if (VISC) {
            T dx[4], dz[4], Gx[4], Gz[4];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                T sx = mk(0.0, T{}), sz = mk(0.0, T{});
#pragma unroll
                for (int q = 0; q < NP1; ++q) {
                    sx = jfma(mkc((double)sDn[a][q], (float)sDn[a][q], T{}), su[le][v][b * NP1 + q], sx);
                    sz = jfma(mkc((double)sDn[b][q], (float)sDn[b][q], T{}), su[le][v][q * NP1 + a], sz);
                }
                dx[v] = mkc(K.two_hx, K.two_hxf, T{}) * sx;
                dz[v] = mkc(K.two_hz, K.two_hzf, T{}) * sz + bgs(K.dubv, K.dubvf, v * nrow + J, T{});
            }
            viscous(U, dx, K.pc, Gx);
            viscous(U, dz, K.pc, Gz);
#pragma unroll
            for (int v = 1; v < 4; ++v) {
                Fx[v] = Fx[v] - Gx[v];
                Fz[v] = Fz[v] - Gz[v];
            }
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            sg[0][le][v][node] = (O)outv(Fx[v]);
            sg[1][le][v][node] = (O)outv(Fz[v]);
        }
    }
    __syncthreads();
    if (!active) return;
    const O lmxa = sl[0][a], lpxa = sl[1][a], dlmxa = sl[2][a], dlpxa = sl[3][a];
    const O lmzb = sl[4][b], lpzb = sl[5][b], dlmzb = sl[6][b], dlpzb = sl[7][b];
    const double eps = (MODE == DG_JV || MODE == DG_SMOOTH64) ? sce[0] : 0.0;
    const double ceps = (MODE == DG_JV || MODE == DG_SMOOTH64) ? sce[1] : 0.0;
    const float adtf = (MODE == DG_TLJV || MODE == DG_TLSMOOTH) ? A.adtf : 0.0f;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        O f = 0;
#pragma unroll
        for (int q = 0; q < NP1; ++q) {
            f = fma(sDx[a][q], sg[0][le][v][b * NP1 + q], f);
            f = fma(sDz[b][q], sg[1][le][v][q * NP1 + a], f);
        }
        if (v == 2) f = fma(-pick<O>(K.g, K.gf), (O)outv(Up[0]), f);
        f = fma(lmxa, PF ? pxl[v] : phix[v * fsx + iL], f);
        f = fma(-lpxa, PF ? pxr[v] : phix[v * fsx + iR], f);
        f = fma(lmzb, PF ? pzb[v] : phiz[v * fsz + iB], f);
        f = fma(-lpzb, PF ? pzt[v] : phiz[v * fsz + iT], f);
        if (VISC && v > 0) {
            const int c = v - 1;
            f = fma(dlmxa, symx[(size_t)(3 + c) * fsx + iL], f);
            f = fma(dlpxa, symx[(size_t)c * fsx + iR], f);
            f = fma(dlmzb, symz[(size_t)(3 + c) * fsz + iB], f);
            f = fma(dlpzb, symz[(size_t)c * fsz + iT], f);
        }
        const size_t gi = (size_t)v * N1 + (size_t)e * NP + node;
        if (MODE == DG_RES) {
            ((double *)A.out0)[gi] = (double)f;
        } else if (MODE == DG_JV) {
            const double y = A.y[gi];
            ((double *)A.out0)[gi] = (eps == 0.0) ? y : fma(-ceps, (double)f - A.fU[gi], y);
        } else if (MODE == DG_G) {
            A.out1[gi] = (double)f;
            ((double *)A.out0)[gi] = A.U[gi] - A.adt * (double)f - A.Ubs[gi];
        } else if (MODE == DG_SMOOTH64) {
            const double z = A.y[gi];
            const double Jz = (eps == 0.0) ? z : fma(-ceps, (double)f - A.fU[gi], z);
            if (A.z0mode == 0) {
                ((double *)A.out0)[gi] = z + A.dtau[e] * (A.r[gi] - Jz);
            } else {
                const double st = (A.alpha * A.dtau[e]) * (A.r[gi] - Jz);
                ((double *)A.out0)[gi] = A.z0mode == 1 ? ((const double *)A.z0)[gi] + st : st;
            }
        } else if (MODE == DG_TLJV) {
            const float z = (float)outv(Up[v]);   // the loader's tangent input is y
            const float jz = z - adtf * (float)f;
            ((float *)A.out0)[gi] = A.rf ? ef[v] - jz : jz;   // with r given: the defect r - G'z
        } else {  // DG_TLSMOOTH
            const float z = (float)outv(Up[v]);
            const float Jz = z - adtf * (float)f;
            if (A.z0mode == 0) {
                ((float *)A.out0)[gi] = z + edt * (ef[v] - Jz);
            } else {
                const float st = (A.alphaf * edt) * (ef[v] - Jz);
                ((float *)A.out0)[gi] = A.z0mode == 1 ? ((const float *)A.z0)[gi] + st : st;
            }
        }
    }
}

template <class T, int IN, int MODE, int NP1, bool VISC, int TV>
struct k_volume_b {
    static constexpr int TPB = 128, MINB = 8;
    static constexpr bool GROUP = !VISC && std::is_same<T, D64>::value && MODE != DG_SMOOTH64;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<DGK> K,
                                               JfArg<Loader<T, IN>> ld0, JfArg<DGArgs> A,
                                               JfArg<const typename OutT<T>::type *> phix,
                                               JfArg<const typename OutT<T>::type *> symx,
                                               JfArg<const typename OutT<T>::type *> phiz,
                                               JfArg<const typename OutT<T>::type *> symz) {
        jf_pdl_enter();
        volume_body<T, IN, MODE, NP1, VISC, TV>(K, ld0, A, phix, symx, phiz, symz, jf_bid);
    }
};
template <class T, int IN, int MODE, int NP1, bool VISC, int TV>
__global__ void __launch_bounds__(128, 8) k_volume(DGK K, Loader<T, IN> ld0, DGArgs A,
                                                   const typename OutT<T>::type *phix,
                                                   const typename OutT<T>::type *symx,
                                                   const typename OutT<T>::type *phiz,
                                                   const typename OutT<T>::type *symz) {
    k_volume_b<T, IN, MODE, NP1, VISC, TV>::run(blockIdx.x, gridDim.x, K, ld0, A, phix, symx, phiz, symz);
}

// ---------------------------------------------------------------------------
// FP32 tangent product in ONE launch (the preconditioner's DG smoothing steps
// and defect).  A block owns a strip of E elements of one element row, one
// thread per node.  The strip's states go to shared memory; every face point
// of the strip's elements is evaluated there (x faces between the strip's
// elements once, the strip's two end faces and the z faces with the neighbour
// trace read from global memory), then the volume term, the lift of the
// shared face terms and the mode's epilogue run as in the two-kernel form.  In
// FP32 the duplicated z faces (each is evaluated by the strips above and below)
// cost less than a second launch and the face buffers' round trip.
// FIRST = 1 (defect mode): the direction is the first pseudo-time step from zero,
// z = dtau_E r, formed on the fly; the epilogue also writes that z to out1f.
template <int NP1> struct StripOf {
    static constexpr int NP = NP1 * NP1;
    static constexpr int E = (128 / NP) > 0 ? 128 / NP : 1;
};

// T^mf of the strip's defect (in sd) to the finest FV level: the 1D transfer
// matrix along x, then along z (through the scratch st), the mass fix from the
// subcell values (mean against the modified Newton-Cotes quadrature), written to
// b and, when x0 is given, x0 = dtau b.  The arithmetic and its order are those of
// the stand-alone transfer kernel.  All threads of the block call it.
template <int NP1, int E>
__device__ __forceinline__ void dgtl_transfer(const TransferOut &TR, float (*sd)[4][NP1 * NP1], float (*smf)[4],
                                              float (*st)[4][NP1 * NP1], int le, int node, int ez, int ex,
                                              bool active) {
    constexpr int NP = NP1 * NP1;
    const int i = node % NP1, j = node / NP1;
    __syncthreads();   // sd complete; sg (scratch st) no longer read
    if (active) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {   // t1(i, b) = sum_a V[i][a] d(a, b), at [b][i]
            float acc = 0.0f;
#pragma unroll
            for (int a = 0; a < NP1; ++a) acc = fmaf(TR.V[i][a], sd[le][q][j * NP1 + a], acc);
            st[le][q][j * NP1 + i] = acc;
        }
    }
    __syncthreads();
    float Tu[4] = {0.f, 0.f, 0.f, 0.f};
    if (active) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float acc = 0.0f;
#pragma unroll
            for (int b = 0; b < NP1; ++b) acc = fmaf(TR.V[j][b], st[le][q][b * NP1 + i], acc);
            Tu[q] = acc;
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int q = 0; q < 4; ++q) sd[le][q][node] = Tu[q];
    }
    __syncthreads();
    if (active && node < 4) {
        const int q = node;
        float mfv = 0.0f, mnc = 0.0f;
        for (int jj = 0; jj < NP1; ++jj)
            for (int ii = 0; ii < NP1; ++ii) {
                const float x = sd[le][q][jj * NP1 + ii];
                mfv += x;
                mnc = fmaf(TR.om[ii] * TR.om[jj], x, mnc);
            }
        smf[le][q] = TR.massfix ? (mfv / (float)NP - mnc) : 0.0f;
    }
    __syncthreads();
    if (!active) return;
    const size_t I = (size_t)ex * NP1 + i, Jr = (size_t)ez * NP1 + j;
    const size_t cell = Jr * TR.NX + I, ncell = (size_t)TR.NX * TR.NZ;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float val = Tu[q] - smf[le][q];
        const size_t gi = (size_t)q * ncell + cell;
        TR.b[gi] = val;
        if (TR.x0) TR.x0[gi] = TR.dtau0[cell] * val;   // first pseudo-time step from zero
    }
}

template <int NP1, bool VISC, int MODE, int FIRST>
struct k_dgtl_b {
    static constexpr int TPB = 128, MINB = VISC ? 5 : 8;
    static constexpr bool GROUP = !VISC;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<DGK> K, JfArg<DGArgs> A,
                                               JfArg<float *> out1f, JfArg<TransferOut> TR) {
        jf_pdl_enter();
        constexpr int NP = NP1 * NP1;
        constexpr int E = StripOf<NP1>::E;
        // U' (value, tangent) of the strip's elements [1], of the elements below [0] and
        // above [2] them, and of the strip's west [0] and east [1] neighbours: every
        // trace the faces need comes from shared memory, loaded coalesced up front
        __shared__ TL32 sn[3][E][4][NP];
        __shared__ TL32 se[2][4][NP];
        __shared__ float sg[2][E][4][NP];              // volume fluxes (tangent part)
        __shared__ float sPx[E + 1][4][NP1];           // x-face terms Phi (face f west of strip element f)
        __shared__ float sPz[2][E][4][NP1];            // z-face terms: [0] bottom, [1] top of element le
        __shared__ float sSx[VISC ? E + 1 : 1][6][NP1];   // viscous symmetry terms (L side 0..2, R side 3..5)
        __shared__ float sSz[VISC ? 2 : 1][VISC ? E : 1][6][NP1];
        __shared__ float sDx[NP1][NP1], sDz[NP1][NP1], sDn[NP1][NP1], sl[8][NP1];
        __shared__ float sdf[FIRST ? E : 1][4][NP];    // the defect, for the transfer (FIRST)
        __shared__ float smf[FIRST ? E : 1][4];        // mass-fix shift per element and variable
        const int nx = K.nx, nz = K.nz;
        const int nstrip = (nx + E - 1) / E;
        const int ez = (int)jf_bid / nstrip, ex0 = ((int)jf_bid % nstrip) * E;
        const int Ev = min(E, nx - ex0);
        const size_t N1 = (size_t)K.n_el * NP;
        const size_t nrow = (size_t)nz * NP1;
        if (threadIdx.x < NP) {
            const int r = threadIdx.x / NP1, q = threadIdx.x % NP1;
            sDx[r][q] = K.Dxf[r][q];
            sDz[r][q] = K.Dzf[r][q];
            sDn[r][q] = K.Dnf[r][q];
        }
        if (threadIdx.x < NP1) {
    #pragma unroll
            for (int r = 0; r < 8; ++r) sl[r][threadIdx.x] = K.liftf[r][threadIdx.x];
        }
        const int le = threadIdx.x / NP, node = threadIdx.x % NP;
        const int a = node % NP1, b = node / NP1;
        const bool active = le < Ev;
        const int e = ez * nx + ex0 + le;
        // direction at a node: y (or dtau_E r for the first step from zero)
        auto dir = [&](int el, size_t i) -> float { return FIRST ? A.dtauf[el] * A.rf[i] : A.yf[i]; };
        auto load = [&](int el, TL32 (*dst)[NP]) {
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                const size_t gi = (size_t)v * N1 + (size_t)el * NP + node;
                dst[v][node] = TL32{A.Uf[gi], dir(el, gi)};
            }
        };
        float ef[4] = {0.f, 0.f, 0.f, 0.f}, edt = 0.0f;
        if (active) {
            load(e, sn[1][le]);
            if (ez > 0) load(e - nx, sn[0][le]);
            if (ez < nz - 1) load(e + nx, sn[2][le]);
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                const size_t gi = (size_t)v * N1 + (size_t)e * NP + node;
                if (MODE == DG_TLSMOOTH || (MODE == DG_TLJV && A.rf)) ef[v] = A.rf[gi];
            }
            if (MODE == DG_TLSMOOTH) edt = A.dtauf[e];
        }
        const bool has_w = ex0 > 0 || K.periodic, has_e = ex0 + Ev < nx || K.periodic;
        if (le == 0 && has_w) load(ez * nx + (ex0 - 1 + nx) % nx, se[0]);
        if (le == 1 && has_e) load(ez * nx + (ex0 + Ev) % nx, se[1]);
        __syncthreads();
        // ---- volume fluxes (independent of the faces below) -----------------------
        TL32 Up[4];
        if (active) {
            const int J = ez * NP1 + b;
            TL32 U[4];
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                Up[v] = sn[1][le][v][node];
                U[v] = Up[v] + TLc{K.ubvf[v * nrow + J]};
            }
            const TL32 ir = TLc{1.0f} / U[0];
            const TL32 p = pressure(U[3], K.pc, nullptr);
            TL32 Fx[4], Fz[4];
            flux_c<TL32, 0>(U, U[1] * ir, p, Fx);
            flux_c<TL32, 1>(U, U[2] * ir, p, Fz);
            if (VISC) {
                TL32 dx[4], dz[4], Gx[4], Gz[4];
    #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    TL32 sx = mk(0.0, TL32{}), sz = mk(0.0, TL32{});
    #pragma unroll
                    for (int q = 0; q < NP1; ++q) {
                        sx = jfma(TLc{sDn[a][q]}, sn[1][le][v][b * NP1 + q], sx);
                        sz = jfma(TLc{sDn[b][q]}, sn[1][le][v][q * NP1 + a], sz);
                    }
                    dx[v] = TLc{K.two_hxf} * sx;
                    dz[v] = TLc{K.two_hzf} * sz + TLc{K.dubvf[v * nrow + J]};
                }
                viscous(U, dx, K.pc, Gx);
                viscous(U, dz, K.pc, Gz);
    #pragma unroll
                for (int v = 1; v < 4; ++v) {
                    Fx[v] = Fx[v] - Gx[v];
                    Fz[v] = Fz[v] - Gz[v];
                }
            }
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                sg[0][le][v][node] = Fx[v].d;
                sg[1][le][v][node] = Fz[v].d;
            }
        }
        // ---- faces ------------------------------------------------------------
        // value and derivative traces of variable v along NP1 nodes i0 + q st of one
        // element's staged nodes, in the order of line_trace
        auto trace = [&](const TL32 (*src)[NP], int v, int i0, int st, const float *pa, const float *pd, TL32 &tv,
                         TL32 &td) {
            tv = mk(0.0, TL32{});
            td = mk(0.0, TL32{});
    #pragma unroll
            for (int q = 0; q < NP1; ++q) {
                const TL32 u = src[v][i0 + q * st];
                tv = jfma(TLc{pa[q]}, u, tv);
                if (VISC) td = jfma(TLc{pd[q]}, u, td);
            }
        };
        const TLc half = TLc{0.5f};
        const int nxf = (Ev + 1) * NP1, nzf = 2 * Ev * NP1;
        for (int t = threadIdx.x; t < nxf + nzf; t += blockDim.x) {
            TL32 trL[4], trR[4], gL[4], gR[4], UL[4], UR[4], H[4], Phi[4], sLv[3], sRv[3];
            if (t < nxf) {
                const int f = t / NP1, sp = t % NP1;      // face f lies west of strip element f
                const bool wallL = f == 0 && !has_w, wallR = f == Ev && !has_e;
                const TL32 (*srcL)[NP] = f > 0 ? sn[1][f - 1] : se[0];
                const TL32 (*srcR)[NP] = f < Ev ? sn[1][f] : se[1];
                const int J = ez * NP1 + sp;
    #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    TL32 aL, aR, dL, dR;
                    if (!wallR) trace(srcR, v, sp * NP1, 1, K.tlm, K.tdlm, aR, dR);
                    if (!wallL) trace(srcL, v, sp * NP1, 1, K.tlp, K.tdlp, aL, dL);
                    if (wallL) { aL = aR; dL = dR; }
                    if (wallR) { aR = aL; dR = dL; }
                    trL[v] = aL;
                    trR[v] = aR;
                    gL[v] = TLc{K.two_hxf} * dL;
                    gR[v] = TLc{K.two_hxf} * dR;
                    UL[v] = aL + TLc{K.ubvf[v * nrow + J]};
                    UR[v] = aR + TLc{K.ubvf[v * nrow + J]};
                }
                TL32 Gh[4];
                if (wallL) {
                    mirror<TL32, 0>(UR, Gh);
                    hllc<TL32, 0>(Gh, UR, K.pc, nullptr, H);
                } else if (wallR) {
                    mirror<TL32, 0>(UL, Gh);
                    hllc<TL32, 0>(UL, Gh, K.pc, nullptr, H);
                } else {
                    hllc<TL32, 0>(UL, UR, K.pc, nullptr, H);
                }
    #pragma unroll
                for (int v = 0; v < 4; ++v) Phi[v] = H[v];
                if (VISC && !wallL && !wallR) {
                    TL32 FL[4], FR[4], Jp[4], AL[4], AR[4];
                    viscous(UL, gL, K.pc, FL);
                    viscous(UR, gR, K.pc, FR);
    #pragma unroll
                    for (int v = 0; v < 4; ++v) Jp[v] = trL[v] - trR[v];
                    viscous(UL, Jp, K.pc, AL);
                    viscous(UR, Jp, K.pc, AR);
    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sLv[q] = half * AL[q + 1];
                        sRv[q] = half * AR[q + 1];
                        Phi[q + 1] = Phi[q + 1] - half * (FL[q + 1] + FR[q + 1]) + TLc{K.eta_xf} * (sLv[q] + sRv[q]);
                    }
                } else {
    #pragma unroll
                    for (int q = 0; q < 3; ++q) sLv[q] = sRv[q] = mk(0.0, TL32{});
                }
    #pragma unroll
                for (int v = 0; v < 4; ++v) sPx[f][v][sp] = Phi[v].d;
                if (VISC) {
    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sSx[f][q][sp] = sLv[q].d;
                        sSx[f][3 + q][sp] = sRv[q].d;
                    }
                }
            } else {
                const int u = t - nxf;
                const int top = u / (Ev * NP1), l = (u / NP1) % Ev, sp = u % NP1;   // column a = sp
                const int fz = ez + top;                 // global horizontal face 0..nz
                const bool wallB = fz == 0, wallT = fz == nz;
                TL32 gB[4], gT[4];
    #pragma unroll
                for (int v = 0; v < 4; ++v) {
                    TL32 aB, aT, dB, dT;
                    if (top) {   // own element below (trace at eta = +1), element ez+1 above
                        trace(sn[1][l], v, sp, NP1, K.tlp, K.tdlp, aB, dB);
                        if (!wallT) trace(sn[2][l], v, sp, NP1, K.tlm, K.tdlm, aT, dT);
                        else { aT = aB; dT = dB; }
                    } else {     // element ez-1 below, own element above (trace at eta = -1)
                        trace(sn[1][l], v, sp, NP1, K.tlm, K.tdlm, aT, dT);
                        if (!wallB) trace(sn[0][l], v, sp, NP1, K.tlp, K.tdlp, aB, dB);
                        else { aB = aT; dB = dT; }
                    }
                    trL[v] = aB;
                    trR[v] = aT;
                    const TLc dub = TLc{K.dubhf[(size_t)v * (nz + 1) + fz]};
                    gB[v] = TLc{K.two_hzf} * dB + dub;
                    gT[v] = TLc{K.two_hzf} * dT + dub;
                    UL[v] = aB + TLc{K.ubhf[(size_t)v * (nz + 1) + fz]};
                    UR[v] = aT + TLc{K.ubhf[(size_t)v * (nz + 1) + fz]};
                }
                TL32 Gh[4];
                if (wallB) {
                    mirror<TL32, 1>(UR, Gh);
                    hllc<TL32, 1>(Gh, UR, K.pc, nullptr, H);
                } else if (wallT) {
                    mirror<TL32, 1>(UL, Gh);
                    hllc<TL32, 1>(UL, Gh, K.pc, nullptr, H);
                } else {
                    hllc<TL32, 1>(UL, UR, K.pc, nullptr, H);
                }
    #pragma unroll
                for (int v = 0; v < 4; ++v) Phi[v] = H[v];
                if (VISC && !wallB && !wallT) {
                    TL32 FB[4], FT[4], Jp[4], AB[4], AT[4];
                    viscous(UL, gB, K.pc, FB);
                    viscous(UR, gT, K.pc, FT);
    #pragma unroll
                    for (int v = 0; v < 4; ++v) Jp[v] = trL[v] - trR[v];
                    viscous(UL, Jp, K.pc, AB);
                    viscous(UR, Jp, K.pc, AT);
    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sLv[q] = half * AB[q + 1];
                        sRv[q] = half * AT[q + 1];
                        Phi[q + 1] = Phi[q + 1] - half * (FB[q + 1] + FT[q + 1]) + TLc{K.eta_zf} * (sLv[q] + sRv[q]);
                    }
                } else {
    #pragma unroll
                    for (int q = 0; q < 3; ++q) sLv[q] = sRv[q] = mk(0.0, TL32{});
                }
    #pragma unroll
                for (int v = 0; v < 4; ++v) sPz[top][l][v][sp] = Phi[v].d;
                if (VISC) {
    #pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sSz[top][l][q][sp] = sLv[q].d;
                        sSz[top][l][3 + q][sp] = sRv[q].d;
                    }
                }
            }
        }
        __syncthreads();
        if (!active && !(FIRST && TR.b)) return;
        const float lmxa = sl[0][a], lpxa = sl[1][a], dlmxa = sl[2][a], dlpxa = sl[3][a];
        const float lmzb = sl[4][b], lpzb = sl[5][b], dlmzb = sl[6][b], dlpzb = sl[7][b];
        const float adtf = A.adtf;
    #pragma unroll
        for (int v = 0; v < 4 && active; ++v) {
            float f = 0.0f;
    #pragma unroll
            for (int q = 0; q < NP1; ++q) {
                f = fmaf(sDx[a][q], sg[0][le][v][b * NP1 + q], f);
                f = fmaf(sDz[b][q], sg[1][le][v][q * NP1 + a], f);
            }
            if (v == 2) f = fmaf(-K.gf, Up[0].d, f);
            f = fmaf(lmxa, sPx[le][v][b], f);
            f = fmaf(-lpxa, sPx[le + 1][v][b], f);
            f = fmaf(lmzb, sPz[0][le][v][a], f);
            f = fmaf(-lpzb, sPz[1][le][v][a], f);
            if (VISC && v > 0) {
                const int q = v - 1;
                f = fmaf(dlmxa, sSx[le][3 + q][b], f);
                f = fmaf(dlpxa, sSx[le + 1][q][b], f);
                f = fmaf(dlmzb, sSz[0][le][3 + q][a], f);
                f = fmaf(dlpzb, sSz[1][le][q][a], f);
            }
            const size_t gi = (size_t)v * N1 + (size_t)e * NP + node;
            const float z = Up[v].d;
            const float jz = z - adtf * f;
            if (MODE == DG_TLJV) {
                const float dv = A.rf ? ef[v] - jz : jz;   // with r given: the defect r - G'z
                if (FIRST && TR.b) sdf[le][v][node] = dv;
                else ((float *)A.out0)[gi] = dv;
                if (FIRST) out1f[gi] = z;
            } else {  // DG_TLSMOOTH
                if (A.z0mode == 0) {
                    ((float *)A.out0)[gi] = z + edt * (ef[v] - jz);
                } else {
                    const float st = (A.alphaf * edt) * (ef[v] - jz);
                    ((float *)A.out0)[gi] = A.z0mode == 1 ? ((const float *)A.z0)[gi] + st : st;
                }
            }
        }
        if (FIRST && TR.b) dgtl_transfer<NP1, E>(TR, sdf, smf, sg[0], le, node, ez, ex0 + le, active);
    }
};
template <int NP1, bool VISC, int MODE, int FIRST>
__global__ void __launch_bounds__(128, VISC ? 5 : 8) k_dgtl(DGK K, DGArgs A, float *out1f, TransferOut TR) {
    k_dgtl_b<NP1, VISC, MODE, FIRST>::run(blockIdx.x, gridDim.x, K, A, out1f, TR);
}

// background fluxes at node rows and horizontal faces, with the residual's own
// D64 functions so that U' = 0 cancels bit for bit
__global__ void k_bg_dg(DGK K, double *fbx, double *fbz, double *hbx, double *hbxw, double *hbz) {
    jf_pdl_enter();
    __shared__ PowTab spt;
    load_powtab(&spt, K.pt);
    __syncthreads();
    const int nrow = K.nz * K.tab.np1;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nrow) {
        D64 U[4], G[4], F[4], H[4];
        for (int v = 0; v < 4; ++v) U[v] = D64{K.ubv[v * nrow + i]};
        const D64 ir = D64{1.0} / U[0];
        const D64 p = pressure(U[3], K.pc, &spt);
        flux_c<D64, 0>(U, U[1] * ir, p, F);
        for (int v = 0; v < 4; ++v) fbx[v * nrow + i] = F[v].x;
        flux_c<D64, 1>(U, U[2] * ir, p, F);
        for (int v = 0; v < 4; ++v) fbz[v * nrow + i] = F[v].x;
        hllc<D64, 0>(U, U, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbx[v * nrow + i] = H[v].x;
        mirror<D64, 0>(U, G);
        hllc<D64, 0>(G, U, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbxw[v * nrow + i] = H[v].x;
        hllc<D64, 0>(U, G, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbxw[(4 + v) * nrow + i] = H[v].x;
    } else if (i < nrow + K.nz + 1) {
        const int j = i - nrow;
        const int nf = K.nz + 1;
        D64 U[4], G[4], H[4];
        for (int v = 0; v < 4; ++v) U[v] = D64{K.ubh[v * nf + j]};
        mirror<D64, 1>(U, G);
        if (j == 0)
            hllc<D64, 1>(G, U, K.pc, &spt, H);
        else if (j == K.nz)
            hllc<D64, 1>(U, G, K.pc, &spt, H);
        else
            hllc<D64, 1>(U, U, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbz[v * nf + j] = H[v].x;
    }
}

DGK make_K(jfnk_ctx *c) {
    DGK K;
    K.nx = c->grid.nx;
    K.nz = c->grid.nz;
    K.n_el = c->n_el;
    K.periodic = c->grid.periodic_x;
    K.two_hx = 2.0 / c->hx;
    K.two_hz = 2.0 / c->hz;
    K.g = c->phys.g;
    K.mu = c->phys.mu;
    K.gf = (float)K.g;
    const double n1 = c->np1;
    // interior-penalty factor C_IP (k+1)^2 / h; the viscosity enters through A(U)
    K.eta_x = c->opts.c_ip * n1 * n1 / c->hx;
    K.eta_z = c->opts.c_ip * n1 * n1 / c->hz;
    K.pc = c->pc;
    K.pt = c->powtab;
    K.ubv = c->ubv;
    K.dubv = c->dubv;
    K.fbx = c->fbx;
    K.fbz = c->fbz;
    K.hbx = c->hbx;
    K.hbxw = c->hbxw;
    K.ubh = c->ubh;
    K.dubh = c->dubh;
    K.hbz = c->hbz;
    K.ubvf = c->ubvf;
    K.dubvf = c->dubvf;
    K.ubhf = c->ubhf;
    K.dubhf = c->dubhf;
    K.tab = c->tab;
    K.two_hxf = (float)K.two_hx;
    K.two_hzf = (float)K.two_hz;
    K.eta_xf = (float)K.eta_x;
    K.eta_zf = (float)K.eta_z;
    for (int r = 0; r < 5; ++r)
        for (int q = 0; q < 5; ++q) {
            K.Dx[r][q] = K.two_hx * K.tab.Dw[r][q];
            K.Dz[r][q] = K.two_hz * K.tab.Dw[r][q];
            K.Dxf[r][q] = (float)K.Dx[r][q];
            K.Dzf[r][q] = (float)K.Dz[r][q];
            K.Dnf[r][q] = (float)K.tab.Dn[r][q];
        }
    for (int q = 0; q < 5; ++q) {
        K.lift[0][q] = K.two_hx * K.tab.lmw[q];
        K.lift[1][q] = K.two_hx * K.tab.lpw[q];
        K.lift[2][q] = K.two_hx * K.two_hx * K.tab.dlmw[q];
        K.lift[3][q] = K.two_hx * K.two_hx * K.tab.dlpw[q];
        K.lift[4][q] = K.two_hz * K.tab.lmw[q];
        K.lift[5][q] = K.two_hz * K.tab.lpw[q];
        K.lift[6][q] = K.two_hz * K.two_hz * K.tab.dlmw[q];
        K.lift[7][q] = K.two_hz * K.two_hz * K.tab.dlpw[q];
        for (int r = 0; r < 8; ++r) K.liftf[r][q] = (float)K.lift[r][q];
    }
    for (int a = 0; a < 5; ++a) {
        K.tlp[a] = (float)K.tab.lp[a];
        K.tlm[a] = (float)K.tab.lm[a];
        K.tdlp[a] = (float)K.tab.dlp[a];
        K.tdlm[a] = (float)K.tab.dlm[a];
    }
    return K;
}

template <class T, int IN, int MODE, int NP1, bool VISC>
int launch(jfnk_ctx *c, const DGK &K, const Loader<T, IN> &ld, const DGArgs &a, cudaStream_t s) {
    typedef typename OutT<T>::type O;
    O *phix, *symx, *phiz, *symz;
    if (IN == 2) {
        phix = (O *)c->phixf;
        symx = (O *)c->symxf;
        phiz = (O *)c->phizf;
        symz = (O *)c->symzf;
    } else {
        phix = (O *)c->phix;
        symx = (O *)c->symx;
        phiz = (O *)c->phiz;
        symz = (O *)c->symz;
    }
    const long long nf = (long long)K.nz * (K.nx + 1) * NP1 + (long long)(K.nz + 1) * K.nx * NP1;
    if (c->timing) JF_CK(cudaEventRecord(c->tev[0], s));
    const int tf = c->opts.tile_faces;
    jf_launch<k_faces_b<T, IN, NP1, VISC>>(k_faces<T, IN, NP1, VISC>, (unsigned)((nf + tf - 1) / tf), tf, 0, s, K, ld, phix, symx, phiz, symz,
              a.tr_out, a.tr_in); jf_launched();
    if (c->timing) JF_CK(cudaEventRecord(c->tev[1], s));
    if (c->opts.tile_volume == 1) {
        constexpr int EPB = EPBOf<NP1, 1>::value;
        const int nb = (K.n_el + EPB - 1) / EPB;
        jf_launch<k_volume_b<T, IN, MODE, NP1, VISC, 1>>(k_volume<T, IN, MODE, NP1, VISC, 1>, nb, EPB * NP1 * NP1, 0, s, K, ld, a, phix, symx, phiz, symz);
    } else {
        constexpr int EPB = EPBOf<NP1, 2>::value;
        const int nb = (K.n_el + EPB - 1) / EPB;
        jf_launch<k_volume_b<T, IN, MODE, NP1, VISC, 2>>(k_volume<T, IN, MODE, NP1, VISC, 2>, nb, EPB * NP1 * NP1, 0, s, K, ld, a, phix, symx, phiz, symz);
    }
    jf_launched();
    JF_CK(cudaGetLastError());
    if (c->timing) {
        JF_CK(cudaEventRecord(c->tev[2], s));
        JF_CK(cudaEventSynchronize(c->tev[2]));
        float m0 = 0.f, m1 = 0.f;
        JF_CK(cudaEventElapsedTime(&m0, c->tev[0], c->tev[1]));
        JF_CK(cudaEventElapsedTime(&m1, c->tev[1], c->tev[2]));
        c->t_faces_ms += m0;
        c->t_volume_ms += m1;
    }
    return JFNK_OK;
}

// FP32 tangent modes: one fused launch (k_dgtl); a.first1 selects the defect at
// the first pseudo-time step from zero, whose z = dtau r is also written to a.out1f
template <int NP1, bool VISC, int MODE>
int launch_tl(jfnk_ctx *c, const DGK &K, const DGArgs &a, cudaStream_t s) {
    constexpr int E = StripOf<NP1>::E;
    const unsigned nb = (unsigned)(K.nz * ((K.nx + E - 1) / E));
    const int threads = E * NP1 * NP1;
    if (c->timing) JF_CK(cudaEventRecord(c->tev[0], s));
    if (MODE == DG_TLJV && a.out1f)
        jf_launch<k_dgtl_b<NP1, VISC, MODE, 1>>(k_dgtl<NP1, VISC, MODE, 1>, nb, threads, 0, s, K, a, a.out1f,
                  a.tro ? *a.tro : TransferOut{});
    else
        jf_launch<k_dgtl_b<NP1, VISC, MODE, 0>>(k_dgtl<NP1, VISC, MODE, 0>, nb, threads, 0, s, K, a, (float *)nullptr, TransferOut{});
    jf_launched();
    JF_CK(cudaGetLastError());
    if (c->timing) {
        JF_CK(cudaEventRecord(c->tev[1], s));
        JF_CK(cudaEventSynchronize(c->tev[1]));
        float m0 = 0.f;
        JF_CK(cudaEventElapsedTime(&m0, c->tev[0], c->tev[1]));
        c->t_faces_ms += m0;   // the whole fused product; the volume share reads 0
    }
    return JFNK_OK;
}

template <int NP1, bool VISC>
int dispatch_mode(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s) {
    DGK K = make_K(c);
    switch (mode) {
        case DG_RES: return launch<D64, 0, DG_RES, NP1, VISC>(c, K, Loader<D64, 0>{a.U}, a, s);
        case DG_G: return launch<D64, 0, DG_G, NP1, VISC>(c, K, Loader<D64, 0>{a.U}, a, s);
        case DG_JV: return launch<D64, 1, DG_JV, NP1, VISC>(c, K, Loader<D64, 1>{a.U, a.y, a.eps, 0.0}, a, s);
        case DG_SMOOTH64:
            return launch<D64, 1, DG_SMOOTH64, NP1, VISC>(c, K, Loader<D64, 1>{a.U, a.y, a.eps, 0.0}, a, s);
        case DG_TLJV:
            if (c->opts.dg_fused == 2 && !a.out1f)
                return launch<TL32, 2, DG_TLJV, NP1, VISC>(c, K, Loader<TL32, 2>{a.Uf, a.yf}, a, s);
            return launch_tl<NP1, VISC, DG_TLJV>(c, K, a, s);
        case DG_TLSMOOTH:
            if (c->opts.dg_fused == 2)
                return launch<TL32, 2, DG_TLSMOOTH, NP1, VISC>(c, K, Loader<TL32, 2>{a.Uf, a.yf}, a, s);
            return launch_tl<NP1, VISC, DG_TLSMOOTH>(c, K, a, s);
    }
    return JFNK_EINVAL;
}

// ---- one launch per operator across ensemble members ---------------------
// A member's share of a grouped residual launch: its operator constants, state,
// output and face buffers, and the first face / volume block of the launch that
// belongs to it.
struct DGMember {
    DGK K;
    Loader<D64, 0> ld;
    DGArgs A;
    double *phix, *symx, *phiz, *symz;
    unsigned fb0, vb0;
};
constexpr int GRP_FACE_THREADS = 128;

template <int NP1, bool VISC>
__global__ void __launch_bounds__(256, 4) k_faces_grp(const DGMember *mem, int nm) {
    jf_pdl_enter();
    int m = 0;
    while (m + 1 < nm && blockIdx.x >= mem[m + 1].fb0) ++m;   // members in block order
    const DGMember &M = mem[m];
    faces_body<D64, 0, NP1, VISC>(M.K, M.ld, M.phix, M.symx, M.phiz, M.symz, blockIdx.x - M.fb0, nullptr, nullptr);
}

template <int NP1, bool VISC>
__global__ void __launch_bounds__(128, 8) k_volume_grp(const DGMember *mem, int nm) {
    jf_pdl_enter();
    int m = 0;
    while (m + 1 < nm && blockIdx.x >= mem[m + 1].vb0) ++m;
    const DGMember &M = mem[m];
    volume_body<D64, 0, DG_RES, NP1, VISC, 2>(M.K, M.ld, M.A, M.phix, M.symx, M.phiz, M.symz, blockIdx.x - M.vb0);
}

template <int NP1, bool VISC>
void launch_grp(const DGMember *dmem, const std::vector<DGMember> &h, int first, int cnt, cudaStream_t s) {
    const DGMember &last = h[first + cnt - 1];
    const long long nfl = (long long)last.K.nz * (last.K.nx + 1) * NP1 + (long long)(last.K.nz + 1) * last.K.nx * NP1;
    const unsigned fb = last.fb0 + (unsigned)((nfl + GRP_FACE_THREADS - 1) / GRP_FACE_THREADS);
    constexpr int EPB = EPBOf<NP1, 2>::value;
    const unsigned vb = last.vb0 + (unsigned)((last.K.n_el + EPB - 1) / EPB);
    jf_launch_now(k_faces_grp<NP1, VISC>, fb, GRP_FACE_THREADS, 0, s, dmem + first, cnt);
    jf_launch_now(k_volume_grp<NP1, VISC>, vb, EPB * NP1 * NP1, 0, s, dmem + first, cnt);
    jf_launched(2);
}

}  // namespace

// The operator kernels of one order k = NP1 - 1.  The library compiles this
// file once per order (JF_DG_NP1 = 2..5, in parallel); the order-independent
// functions below come with the first.  Compiled without JF_DG_NP1, one unit
// holds every order.
template <int NP1>
int dg_dispatch(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s);
#if !defined(JF_DG_NP1)
#define JF_DG_ORDERS(X) X(2) X(3) X(4) X(5)
#else
#define JF_DG_ORDERS(X) X(JF_DG_NP1)
#endif
#define JF_DG_DEFINE(n)                                                                              \
    template <>                                                                                     \
    int dg_dispatch<n>(jfnk_ctx * c, int mode, const DGArgs &a, cudaStream_t s) {                   \
        return c->phys.mu != 0.0 ? dispatch_mode<n, true>(c, mode, a, s) : dispatch_mode<n, false>(c, mode, a, s); \
    }
JF_DG_ORDERS(JF_DG_DEFINE)

#if !defined(JF_DG_NP1) || JF_DG_NP1 == 2
#if defined(JF_DG_NP1)
template <> int dg_dispatch<3>(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s);
template <> int dg_dispatch<4>(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s);
template <> int dg_dispatch<5>(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s);
#endif

int dg_setup_background(jfnk_ctx *c, cudaStream_t s) {
    DGK K = make_K(c);
    const int n = c->grid.nz * c->np1 + c->grid.nz + 1;
    k_bg_dg<<<(n + 127) / 128, 128, 0, s>>>(K, c->fbx, c->fbz, c->hbx, c->hbxw, c->hbz); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int dg_apply(jfnk_ctx *c, int mode, const DGArgs &a_in, cudaStream_t s) {
    DGArgs a = a_in;
    a.adtf = (float)a.adt;
    a.alphaf = (float)a.alpha;
    c->dg_calls++;
    // the stored traces belong to the cached f(U): any other writer of the cache drops them
    if (a.out0 == c->fU || a.out1 == c->fU) c->tr_valid = a.tr_out == c->trU ? 1 : 0;
    switch (c->np1) {
        case 2: return dg_dispatch<2>(c, mode, a, s);
        case 3: return dg_dispatch<3>(c, mode, a, s);
        case 4: return dg_dispatch<4>(c, mode, a, s);
        case 5: return dg_dispatch<5>(c, mode, a, s);
    }
    return JFNK_EINVAL;
}

size_t dg_member_bytes() { return sizeof(DGMember); }

// f_m = M^-1 L_h(U_m) for every member, grouped by (order, viscous): one face
// and one volume launch per group.  dmem: device room for n descriptors.
int dg_residual_grouped(jfnk_ctx *const *ctx, int n, const double *const *U, double *const *f, void *dmem,
                        cudaStream_t s) {
    if (!ctx || !U || !f || !dmem || n < 1) return JFNK_EINVAL;
    std::vector<int> order;
    for (int np1 = 2; np1 <= 5; ++np1)
        for (int visc = 0; visc < 2; ++visc)
            for (int i = 0; i < n; ++i) {
                if (!ctx[i] || !U[i] || !f[i] || U[i] == f[i]) return JFNK_EINVAL;
                if (ctx[i]->np1 == np1 && (ctx[i]->phys.mu != 0.0) == (visc != 0)) order.push_back(i);
            }
    if ((int)order.size() != n) return JFNK_EINVAL;
    std::vector<DGMember> h(n);
    std::vector<int> gstart;
    unsigned fb = 0, vb = 0;
    for (int q = 0; q < n; ++q) {
        jfnk_ctx *c = ctx[order[q]];
        if (q == 0 || c->np1 != ctx[order[q - 1]]->np1 ||
            (c->phys.mu != 0.0) != (ctx[order[q - 1]]->phys.mu != 0.0)) {
            gstart.push_back(q);
            fb = vb = 0;
        }
        DGMember &M = h[q];
        M.K = make_K(c);
        M.ld = Loader<D64, 0>{U[order[q]]};
        M.A = DGArgs{};
        M.A.U = U[order[q]];
        M.A.out0 = f[order[q]];
        M.phix = (double *)c->phix;
        M.symx = (double *)c->symx;
        M.phiz = (double *)c->phiz;
        M.symz = (double *)c->symz;
        M.fb0 = fb;
        M.vb0 = vb;
        const int n1 = c->np1;
        const long long nf = (long long)c->grid.nz * (c->grid.nx + 1) * n1 + (long long)(c->grid.nz + 1) * c->grid.nx * n1;
        fb += (unsigned)((nf + GRP_FACE_THREADS - 1) / GRP_FACE_THREADS);
        const int epb = (128 / (n1 * n1)) > 0 ? 128 / (n1 * n1) : 1;
        vb += (unsigned)((c->n_el + epb - 1) / epb);
        c->dg_calls++;
    }
    JF_CK(cudaMemcpyAsync(dmem, h.data(), sizeof(DGMember) * (size_t)n, cudaMemcpyHostToDevice, s));
    const DGMember *dm = (const DGMember *)dmem;
    gstart.push_back(n);
    for (size_t gi = 0; gi + 1 < gstart.size(); ++gi) {
        const int a = gstart[gi], cnt = gstart[gi + 1] - a;
        const bool visc = h[a].K.mu != 0.0;
        switch (h[a].K.tab.np1) {
            case 2: visc ? launch_grp<2, true>(dm, h, a, cnt, s) : launch_grp<2, false>(dm, h, a, cnt, s); break;
            case 3: visc ? launch_grp<3, true>(dm, h, a, cnt, s) : launch_grp<3, false>(dm, h, a, cnt, s); break;
            case 4: visc ? launch_grp<4, true>(dm, h, a, cnt, s) : launch_grp<4, false>(dm, h, a, cnt, s); break;
            case 5: visc ? launch_grp<5, true>(dm, h, a, cnt, s) : launch_grp<5, false>(dm, h, a, cnt, s); break;
            default: return JFNK_EINVAL;
        }
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}
#endif  // order-independent part
