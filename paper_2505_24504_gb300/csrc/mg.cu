// Low-order-approximation preconditioner Q^-1 = T^-1 q^-1 T (eq. preconditioner,
// Sec. 3.2-3.5) on the GPU.
//
//  k_to_fv    T^mf: one thread per subcell; the element's nodal values go
//             through shared memory and the 1D interpolation matrix V twice
//             (tensor product), then the mass fix of eq. (transfer-mass-fix)
//             with the element mass of the DG polynomial taken from the subcell
//             values by the modified Newton-Cotes weights (Sec. 3.3, Appendix A).
//  k_to_dg    T^-1: inverse tensor interpolation and the mass fix back.
//  k_fv       f_low and the level products on one FV level, one thread per cell:
//             HLLC^pert on the four faces (background fluxes precomputed per
//             row), gravity source, two-point viscous flux.  Modes: residual,
//             pseudo-time step x + dtau (b - g'x), defect g'x - b.  g' is the
//             FD quotient of Sec. 3.1 (FP64) or the exact tangent (FP32).
//  k_restrict / k_prolong   agglomeration R and injection P (Sec. 3.4).
//  mg_cycle   MG_l(x, b; u) of Sec. 3.4 on the host; every level's work is a few
//             launches on the caller's stream, so an application can be captured
//             in one CUDA graph.
#include <string.h>

#include <cuda_bf16.h>

#include "internal.h"

namespace {

struct FVK {
    int NX, NZ, periodic;
    double iHx, iHz, g, mu;
    double vcx, vcz;                     // mu / (2 H) of the two-point viscous flux
    float iHxf, iHzf, gf, vcxf, vczf;    // float copies for the FP32 tangent
    float adtf;                          // alpha dt of the linearisation in FP32
    PhysC pc;
    const PowTab *pt;
    const double *ub, *hbx, *hbxw, *hbz;
    const float *ubf;
};

// One stage of the pseudo-time smoother (Sec. 3.5) in the FV smoothing kernels:
// mode 0 explicit Euler x + dtau (b - g'x); mode 1 x0 + alpha dtau (b - g'x) (a
// stage of the low-storage multi-stage scheme, x the previous stage); mode 2 the
// same with x0 = 0.
struct RKS {
    const void *x0;
    int mode;
    double alpha;
    float alphaf;   // FP32 copy: no per-thread conversion (an FP64-pipe instruction)
};
template <class S>
JF_D S rk_stage(const RKS &rk, S x, S dt, S bmg, size_t gi) {
    if (rk.mode == 0) return x + dt * bmg;
    const S st = (pick<S>(rk.alpha, rk.alphaf) * dt) * bmg;
    return rk.mode == 1 ? ((const S *)rk.x0)[gi] + st : st;
}

JF_D D64 bgs(const double *d, const float *, size_t i, D64) { return D64{d[i]}; }
JF_D TLc bgs(const double *, const float *f, size_t i, TL32) { return TLc{f[i]}; }

__device__ __forceinline__ void load_pt(PowTab *s, const PowTab *g) {
    const double *src = reinterpret_cast<const double *>(g);
    double *dst = reinterpret_cast<double *>(s);
    for (int i = threadIdx.x; i < (int)(sizeof(PowTab) / sizeof(double)); i += blockDim.x) dst[i] = src[i];
}

// Level state loaders, addressed by (variable, cell, I, J):
// IN 0 u; IN 1 u + eps x (FP64, eps on the device); IN 2 TL32 (u, x).
template <class T, int IN> struct FLoad;
template <> struct FLoad<D64, 0> {
    const double *u;
    size_t n1;
    JF_D void prepare() {}
    JF_D double step() const { return 0.0; }
    JF_D double dir(int, size_t, int, int) const { return 0.0; }
    JF_D D64 operator()(int v, size_t c, int, int) const { return D64{u[v * n1 + c]}; }
};
template <> struct FLoad<D64, 1> {
    const double *u, *x, *epsp;
    size_t n1;
    double eps;
    JF_D void prepare() { eps = *epsp; }
    JF_D double step() const { return eps; }
    JF_D double dir(int v, size_t c, int, int) const { return x[v * n1 + c]; }
    JF_D D64 operator()(int v, size_t c, int, int) const {
        const size_t i = v * n1 + c;
        return D64{__fma_rn(eps, x[i], u[i])};
    }
};
template <> struct FLoad<TL32, 2> {
    const float *u, *x;
    size_t n1;
    JF_D void prepare() {}
    JF_D double step() const { return 0.0; }
    JF_D float dir(int v, size_t c, int, int) const { return x[v * n1 + c]; }
    JF_D TL32 operator()(int v, size_t c, int, int) const {
        const size_t i = v * n1 + c;
        return TL32{u[i], x[i]};
    }
};
// IN 3: FP32 tangent at the coarse-corrected iterate x - P v_c (Sec. 3.4), formed
// on the fly (x = 0 when `zero`), so the correction needs no launch of its own
template <> struct FLoad<TL32, 3> {
    const float *u, *x, *vc;
    size_t n1;
    int NXc, fac, zero;
    size_t nc;
    JF_D void prepare() {}
    JF_D double step() const { return 0.0; }
    JF_D float dir(int v, size_t c, int I, int J) const {
        const float pv = vc[(size_t)v * nc + (size_t)(J / fac) * NXc + I / fac];
        return zero ? -pv : x[v * n1 + c] - pv;
    }
    JF_D TL32 operator()(int v, size_t c, int I, int J) const { return TL32{u[v * n1 + c], dir(v, c, I, J)}; }
};
enum { FV_RES = 0, FV_SMOOTH = 1, FV_DEFECT = 2 };

// BF16 storage numerics on the coarsest level (precond_prec = 16): values are
// rounded to bfloat16 whenever they are written there
template <class S>
JF_D S store_round(S v, int bf16) {
    return bf16 ? (S)__bfloat162float(__float2bfloat16_rn((float)v)) : v;
}

template <class T> struct SOf;
template <> struct SOf<D64> { typedef double type; };
template <> struct SOf<TL32> { typedef float type; };
JF_D double oval(D64 a) { return a.x; }
JF_D float oval(TL32 a) { return a.d; }

template <class T, int D>
JF_D void face_flux(const T UL[4], const T UR[4], bool wallL, bool wallR, const double *hb, size_t hs,
                    size_t hi, bool sub, const FVK &K, const PowTab *pt, T H[4]) {
    T G[4];
    if (wallL) {
        mirror<T, D>(UR, G);
        hllc<T, D>(G, UR, K.pc, pt, H);
    } else if (wallR) {
        mirror<T, D>(UL, G);
        hllc<T, D>(UL, G, K.pc, pt, H);
    } else {
        hllc<T, D>(UL, UR, K.pc, pt, H);
    }
    if (sub) {
#pragma unroll
        for (int v = 0; v < 4; ++v) H[v] = H[v] - mk(hb[v * hs + hi], T{});
    }
}

// the same two-point flux from precomputed sides (1/rho of each side reused)
template <class T, class C>
JF_D void visc2_s(const Side<T> &L, const Side<T> &R, C coef, T V[4]) {
    const T c = coef * (L.U[0] + R.U[0]);
    V[0] = mk(0.0, T{});
#pragma unroll
    for (int v = 1; v < 4; ++v) V[v] = c * (R.U[v] * R.ir - L.U[v] * L.ir);
}

template <class T, class C>
JF_D void visc2(const T UL[4], const T UR[4], C coef, T V[4]) {
    const T irL = mkc(1.0, 1.0f, T{}) / UL[0], irR = mkc(1.0, 1.0f, T{}) / UR[0];
    const T c = coef * (UL[0] + UR[0]);
    V[0] = mk(0.0, T{});
#pragma unroll
    for (int v = 1; v < 4; ++v) V[v] = c * (UR[v] * irR - UL[v] * irL);
}

// f_low (or its tangent) at one cell (I, Jz) by one thread: HLLC^pert on the four
// faces, gravity source, two-point viscous flux (large levels: enough cells to
// fill the GPU, and fewer instructions per cell than the four-lane form).
template <class T, int IN, bool VISC>
JF_D void fv_cell_op(const FVK &K, const FLoad<T, IN> &ld, const PowTab *spt, size_t c, int I, int Jz, T f[4]) {
    const int NX = K.NX, NZ = K.NZ;
    const bool sub = (IN < 2);
    T U[4], Un[4][4];   // own state and the W, E, S, N neighbours
    int nb[4] = {-1, -1, -1, -1};
    int nI[4] = {I - 1, I + 1, I, I}, nJ[4] = {Jz, Jz, Jz - 1, Jz + 1};
    if (I > 0) nb[0] = Jz * NX + I - 1;
    else if (K.periodic) { nb[0] = Jz * NX + NX - 1; nI[0] = NX - 1; }
    if (I < NX - 1) nb[1] = Jz * NX + I + 1;
    else if (K.periodic) { nb[1] = Jz * NX; nI[1] = 0; }
    if (Jz > 0) nb[2] = (Jz - 1) * NX + I;
    if (Jz < NZ - 1) nb[3] = (Jz + 1) * NX + I;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        U[v] = ld(v, c, I, Jz) + bgs(K.ub, K.ubf, v * NZ + Jz, T{});
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int v = 0; v < 4; ++v)
            Un[q][v] = nb[q] >= 0 ? ld(v, (size_t)nb[q], nI[q], nJ[q]) + bgs(K.ub, K.ubf, v * NZ + nJ[q], T{}) : U[v];
    }
    T HW[4], HE[4], HS[4], HN[4];
    face_flux<T, 0>(Un[0], U, nb[0] < 0, false, nb[0] < 0 ? K.hbxw : K.hbx, NZ, Jz, sub, K, spt, HW);
    face_flux<T, 0>(U, Un[1], false, nb[1] < 0, nb[1] < 0 ? K.hbxw + 4 * NZ : K.hbx, NZ, Jz, sub, K, spt, HE);
    face_flux<T, 1>(Un[2], U, nb[2] < 0, false, K.hbz, NZ + 1, Jz, sub, K, spt, HS);
    face_flux<T, 1>(U, Un[3], false, nb[3] < 0, K.hbz, NZ + 1, Jz + 1, sub, K, spt, HN);
    const auto iHx = mkc(K.iHx, K.iHxf, T{}), iHz = mkc(K.iHz, K.iHzf, T{});
#pragma unroll
    for (int v = 0; v < 4; ++v) f[v] = -((HE[v] - HW[v]) * iHx + (HN[v] - HS[v]) * iHz);
    const T up0 = ld(0, c, I, Jz);
    f[2] = f[2] - mkc(K.g, K.gf, T{}) * up0;   // -g rho' (tangent: -g x_rho)
    if (VISC) {
        T VW[4], VE[4], VS[4], VN[4];
        const T zero = mk(0.0, T{});
        const auto cx = mkc(K.vcx, K.vcxf, T{}), cz = mkc(K.vcz, K.vczf, T{});
        if (nb[0] >= 0) visc2(Un[0], U, cx, VW); else { for (int v = 0; v < 4; ++v) VW[v] = zero; }
        if (nb[1] >= 0) visc2(U, Un[1], cx, VE); else { for (int v = 0; v < 4; ++v) VE[v] = zero; }
        if (nb[2] >= 0) visc2(Un[2], U, cz, VS); else { for (int v = 0; v < 4; ++v) VS[v] = zero; }
        if (nb[3] >= 0) visc2(U, Un[3], cz, VN); else { for (int v = 0; v < 4; ++v) VN[v] = zero; }
#pragma unroll
        for (int v = 1; v < 4; ++v) f[v] = f[v] + (VE[v] - VW[v]) * iHx + (VN[v] - VS[v]) * iHz;
    }
}

JF_D D64 shfl_x(D64 a, int m) { return D64{__shfl_xor_sync(0xffffffffu, a.x, m)}; }
JF_D TL32 shfl_x(TL32 a, int m) {
    return TL32{__shfl_xor_sync(0xffffffffu, a.v, m), __shfl_xor_sync(0xffffffffu, a.d, m)};
}
template <class T>
JF_D void swap12(T U[4]) {
    const T t = U[1];
    U[1] = U[2];
    U[2] = t;
}

// Sum over the four lanes of a group of per-lane vectors f[4], scattered so that
// lane q ends up with component q (two shuffle rounds, three exchanges).
template <class T>
JF_D T reduce_scatter4(const T f[4], int q) {
    const bool hi = (q & 2) != 0, lo = (q & 1) != 0;
    const T k0 = hi ? f[2] : f[0], k1 = hi ? f[3] : f[1];
    const T s0 = hi ? f[0] : f[2], s1 = hi ? f[1] : f[3];
    const T g0 = k0 + shfl_x(s0, 2), g1 = k1 + shfl_x(s1, 2);
    const T keep = lo ? g1 : g0, send = lo ? g0 : g1;
    return keep + shfl_x(send, 1);
}

// f_low (or its tangent) at cell (I, Jz), computed by four lanes: lane q evaluates
// face q (0 W, 1 E, 2 S, 3 N): HLLC^pert (background flux of the face row
// subtracted), the two-point viscous flux, and lane 2 adds the gravity source.
// z faces are evaluated in a frame with the two momentum components swapped, so
// every lane runs the same x-direction HLLC (the arithmetic is that of the
// z-direction flux, component for component).  Returns component q of f.
// All four lanes of the group must be active (the reduction shuffles).
template <class T, int IN, bool VISC>
JF_D T fv_cell_op4(const FVK &K, const FLoad<T, IN> &ld, const PowTab *spt, size_t c, int I, int Jz, int q) {
    const int NX = K.NX, NZ = K.NZ;
    const bool sub = (IN < 2);
    const bool zf = q >= 2, right = (q & 1) != 0;
    long nb = -1;
    int nI = I, nJ = Jz;
    if (q == 0) {
        if (I > 0) { nb = (long)c - 1; nI = I - 1; }
        else if (K.periodic) { nb = (long)c + NX - 1; nI = NX - 1; }
    } else if (q == 1) {
        if (I < NX - 1) { nb = (long)c + 1; nI = I + 1; }
        else if (K.periodic) { nb = (long)c - (NX - 1); nI = 0; }
    } else if (q == 2) {
        if (Jz > 0) { nb = (long)c - NX; nJ = Jz - 1; }
    } else {
        if (Jz < NZ - 1) { nb = (long)c + NX; nJ = Jz + 1; }
    }
    const bool wall = nb < 0;
    T U[4], N[4];
    const T up0 = ld(0, c, I, Jz);
#pragma unroll
    for (int v = 0; v < 4; ++v) U[v] = (v == 0 ? up0 : ld(v, c, I, Jz)) + bgs(K.ub, K.ubf, v * NZ + Jz, T{});
#pragma unroll
    for (int v = 0; v < 4; ++v)
        N[v] = wall ? U[v] : ld(v, (size_t)nb, nI, nJ) + bgs(K.ub, K.ubf, v * NZ + nJ, T{});
    if (zf) {
        swap12(U);
        swap12(N);
    }
    if (wall) N[1] = -U[1];   // slip-wall ghost: normal momentum reversed
    T H[4];
    if (right) hllc<T, 0>(U, N, K.pc, spt, H);
    else hllc<T, 0>(N, U, K.pc, spt, H);
    T V[4];
    if (VISC) {
        if (wall) {
#pragma unroll
            for (int v = 0; v < 4; ++v) V[v] = mk(0.0, T{});
        } else if (right) {
            visc2(U, N, zf ? mkc(K.vcz, K.vczf, T{}) : mkc(K.vcx, K.vcxf, T{}), V);
        } else {
            visc2(N, U, zf ? mkc(K.vcz, K.vczf, T{}) : mkc(K.vcx, K.vcxf, T{}), V);
        }
    }
    if (zf) {
        swap12(H);
        if (VISC) swap12(V);
    }
    if (sub) {
        const double *hb;
        size_t hs, hi;
        if (!zf) {
            hb = wall ? (right ? K.hbxw + 4 * NZ : K.hbxw) : K.hbx;
            hs = NZ;
            hi = Jz;
        } else {
            hb = K.hbz;
            hs = NZ + 1;
            hi = Jz + (right ? 1 : 0);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) H[v] = H[v] - mk(hb[v * hs + hi], T{});
    }
    const auto ih = zf ? mkc(K.iHz, K.iHzf, T{}) : mkc(K.iHx, K.iHxf, T{});
    T f[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        // W, S faces enter with +, E, N with - (f = -div H + div F_v)
        T a = H[v] * ih;
        if (VISC && v > 0) a = a - V[v] * ih;
        f[v] = right ? -a : a;
    }
    T fq = reduce_scatter4(f, q);
    if (q == 2) fq = fq - mkc(K.g, K.gf, T{}) * up0;   // -g rho' (tangent: -g x_rho)
    return fq;
}

// g'(u) x at one cell and variable from the operator value f (FD quotient or tangent)
template <class T, int IN, class S>
JF_D S gprime_of(const FLoad<T, IN> &ld, S x, T f, const double *fu, size_t gi, double adt, float adtf, double eps) {
    if (IN == 1) return (S)((eps == 0.0) ? (double)x : (double)x - adt * ((double)oval(f) - fu[gi]) / eps);
    return x - (S)adtf * (S)oval(f);
}

// One thread (L = 1) or four lanes (L = 4, lane q owns variable q) per cell of
// an NX x NZ level.
template <class T, int IN, int MODE, bool VISC, int L>
struct k_fv_b {
    static constexpr int TPB = 256, MINB = 0;
    static constexpr bool GROUP = !VISC && std::is_same<T, TL32>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<FVK> K,
                                               JfArg<FLoad<T, IN>> ld0, JfArg<const typename SOf<T>::type *> xin,
                                               JfArg<const typename SOf<T>::type *> b,
                                               JfArg<const typename SOf<T>::type *> dtau, JfArg<const double *> fu,
                                               JfArg<double> adt, JfArg<typename SOf<T>::type *> out, JfArg<int> bf16,
                                               JfArg<RKS> rk) {
        jf_pdl_enter();
        typedef typename SOf<T>::type S;
        __shared__ PowTab spt;
        if (IN < 2) load_pt(&spt, K.pt);   // the FP32 tangent power needs no table
        FLoad<T, IN> ld = ld0;
        ld.prepare();
        __syncthreads();
        const float adtf = IN >= 2 ? K.adtf : 0.0f;
        const size_t n1 = (size_t)K.NX * K.NZ;
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        const int q = L == 4 ? (int)(t & 3) : 0;
        const size_t cell = L == 4 ? (t >> 2) : t;
        const bool live = cell < n1;
        if (L == 1 && !live) return;
        const size_t c = live ? cell : n1 - 1;   // idle lanes still join the shuffles
        const int I = (int)(c % K.NX), Jz = (int)(c / K.NX);
        T f[4];
        if (L == 4) f[0] = fv_cell_op4<T, IN, VISC>(K, ld, &spt, c, I, Jz, q);
        else fv_cell_op<T, IN, VISC>(K, ld, &spt, c, I, Jz, f);
        if (!live) return;
    #pragma unroll
        for (int k = 0; k < (L == 4 ? 1 : 4); ++k) {
            const int v = L == 4 ? q : k;
            const size_t gi = (size_t)v * n1 + c;
            if (MODE == FV_RES) {
                out[gi] = (S)oval(f[k]);
            } else {
                const S x = (S)ld.dir(v, c, I, Jz);
                const S gx = gprime_of<T, IN, S>(ld, x, f[k], fu, gi, adt, adtf, ld.step());
                if (MODE == FV_SMOOTH)
                    out[gi] = store_round<S>(rk_stage<S>(rk, x, dtau[c], b[gi] - gx, gi), bf16);
                else
                    out[gi] = gx - b[gi];
            }
        }
    }
};
template <class T, int IN, int MODE, bool VISC, int L>
__global__ void __launch_bounds__(256) k_fv(FVK K, FLoad<T, IN> ld0, const typename SOf<T>::type *xin,
                                            const typename SOf<T>::type *b, const typename SOf<T>::type *dtau,
                                            const double *fu, double adt, typename SOf<T>::type *out,
                                            int bf16, RKS rk) {
    k_fv_b<T, IN, MODE, VISC, L>::run(blockIdx.x, gridDim.x, K, ld0, xin, b, dtau, fu, adt, out, bf16, rk);
}

// Defect and restriction in one pass: the defect g'x - b of every child cell of
// a coarse cell, averaged into b_c; when x_c is given, also the coarse level's
// first pseudo-time step x_c = dtau_c b_c.  L = 1: one thread per coarse cell
// loops over its fac x fac children.  L = 4, FAC2: 2 x 2 agglomeration with
// sixteen lanes per coarse cell (four lanes per child, children summed by
// shuffles); L = 4 otherwise: four lanes per coarse cell loop over the children.
template <class T, int IN, bool VISC, int L, bool FAC2>
struct k_fv_defect_restrict_b {
    static constexpr int TPB = 256, MINB = 0;
    static constexpr bool GROUP = !VISC && std::is_same<T, TL32>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<FVK> K,
                                               JfArg<FLoad<T, IN>> ld0, JfArg<const typename SOf<T>::type *> b,
                                               JfArg<const double *> fu, JfArg<double> adt, JfArg<int> fac,
                                               JfArg<typename SOf<T>::type *> bc, JfArg<typename SOf<T>::type *> xc,
                                               JfArg<const typename SOf<T>::type *> dtau_c, JfArg<int> bf16) {
        jf_pdl_enter();
        typedef typename SOf<T>::type S;
        __shared__ PowTab spt;
        if (IN < 2) load_pt(&spt, K.pt);
        FLoad<T, IN> ld = ld0;
        ld.prepare();
        __syncthreads();
        const int NXc = K.NX / fac, NZc = K.NZ / fac;
        const size_t nc = (size_t)NXc * NZc, n1 = (size_t)K.NX * K.NZ;
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        const double eps = ld.step();
        const float adtf = IN >= 2 ? K.adtf : 0.0f;
        if (L == 1) {
            if (t >= nc) return;
            const int Ic = (int)(t % NXc), Jc = (int)(t / NXc);
            S acc[4] = {0, 0, 0, 0};
            for (int jj = 0; jj < fac; ++jj)
                for (int ii = 0; ii < fac; ++ii) {
                    const int I = Ic * fac + ii, Jz = Jc * fac + jj;
                    const size_t c = (size_t)Jz * K.NX + I;
                    T f[4];
                    fv_cell_op<T, IN, VISC>(K, ld, &spt, c, I, Jz, f);
    #pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const size_t gi = (size_t)v * n1 + c;
                        acc[v] += gprime_of<T, IN, S>(ld, (S)ld.dir(v, c, I, Jz), f[v], fu, gi, adt, adtf, eps) - b[gi];
                    }
                }
            const S inv = (S)1 / (S)(fac * fac);
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                const S bv = store_round<S>(acc[v] * inv, bf16);
                bc[(size_t)v * nc + t] = bv;
                if (xc) xc[(size_t)v * nc + t] = store_round<S>(dtau_c[t] * bv, bf16);
            }
            return;
        }
        const int q = (int)(t & 3);
        const size_t g = FAC2 ? (t >> 4) : (t >> 2);
        const bool live = g < nc;
        const size_t cc = live ? g : nc - 1;
        const int Ic = (int)(cc % NXc), Jc = (int)(cc / NXc);
        S acc = 0;
        if (FAC2) {
            const int ch = (int)((t >> 2) & 3);
            const int I = 2 * Ic + (ch & 1), Jz = 2 * Jc + (ch >> 1);
            const size_t c = (size_t)Jz * K.NX + I;
            const T fq = fv_cell_op4<T, IN, VISC>(K, ld, &spt, c, I, Jz, q);
            const size_t gi = (size_t)q * n1 + c;
            const S d = gprime_of<T, IN, S>(ld, (S)ld.dir(q, c, I, Jz), fq, fu, gi, adt, adtf, eps) - b[gi];
            const S d2 = d + __shfl_xor_sync(0xffffffffu, d, 4);
            acc = d2 + __shfl_xor_sync(0xffffffffu, d2, 8);
            if (ch != 0) return;
        } else {
            for (int jj = 0; jj < fac; ++jj)
                for (int ii = 0; ii < fac; ++ii) {
                    const int I = Ic * fac + ii, Jz = Jc * fac + jj;
                    const size_t c = (size_t)Jz * K.NX + I;
                    const T fq = fv_cell_op4<T, IN, VISC>(K, ld, &spt, c, I, Jz, q);
                    const size_t gi = (size_t)q * n1 + c;
                    acc += gprime_of<T, IN, S>(ld, (S)ld.dir(q, c, I, Jz), fq, fu, gi, adt, adtf, eps) - b[gi];
                }
        }
        if (!live) return;
        const S bv = store_round<S>(acc / (S)(fac * fac), bf16);
        bc[(size_t)q * nc + cc] = bv;
        if (xc) xc[(size_t)q * nc + cc] = store_round<S>(dtau_c[cc] * bv, bf16);
    }
};
template <class T, int IN, bool VISC, int L, bool FAC2>
__global__ void __launch_bounds__(256) k_fv_defect_restrict(FVK K, FLoad<T, IN> ld0, const typename SOf<T>::type *b,
                                                            const double *fu, double adt, int fac,
                                                            typename SOf<T>::type *bc, typename SOf<T>::type *xc,
                                                            const typename SOf<T>::type *dtau_c, int bf16) {
    k_fv_defect_restrict_b<T, IN, VISC, L, FAC2>::run(blockIdx.x, gridDim.x, K, ld0, b, fu, adt, fac, bc, xc, dtau_c, bf16);
}

// Face-once form for large levels: a block owns a tile of TX x TZ cells.  The
// states of the tile and a one-cell halo go to shared memory, every face of the
// tile is evaluated once (HLLC^pert and the two-point viscous flux; walls by the
// mirrored ghost), and each cell adds its four faces, the gravity source and the
// mode's epilogue.  About 2.2 face evaluations per cell instead of 4.
// MODE FV_RES / FV_SMOOTH / FV_DEFECT as k_fv; FV_DEFRES: the defect g'x - b of
// each cell, averaged over 2 x 2 children into bc (and xc = dtau_c bc when xc is
// given) -- the tile origin and size are even, so children never straddle tiles.
enum { FV_DEFRES = 3 };
constexpr int FV_TX = 32;

template <class T, int IN, int MODE, bool VISC, int TZ>
struct k_fv_tile_b {
    static constexpr int TPB = FV_TX * TZ, MINB = 0;
    static constexpr bool GROUP = !VISC && std::is_same<T, TL32>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<FVK> K,
                                               JfArg<FLoad<T, IN>> ld0, JfArg<const typename SOf<T>::type *> b,
                                               JfArg<const typename SOf<T>::type *> dtau, JfArg<const double *> fu,
                                               JfArg<double> adt, JfArg<typename SOf<T>::type *> out,
                                               JfArg<typename SOf<T>::type *> xc,
                                               JfArg<const typename SOf<T>::type *> dtau_c, JfArg<int> bf16,
                                               JfArg<RKS> rk) {
        jf_pdl_enter();
        typedef typename SOf<T>::type S;
        constexpr int TX = FV_TX;
        // the FP64 power table (the FP32 tangent power needs none)
        __shared__ double spt_raw[IN < 2 ? sizeof(PowTab) / sizeof(double) : 1];
        PowTab &spt = *reinterpret_cast<PowTab *>(spt_raw);
        // the tile's cells and a one-cell halo as face sides: state, 1/rho, p, c
        // (one pressure / sound speed per cell instead of one per face and side)
        __shared__ T sU[4][TZ + 2][TX + 2];
        __shared__ T sIr[TZ + 2][TX + 2], sP[TZ + 2][TX + 2], sC[TZ + 2][TX + 2];
        __shared__ S sGx[4][TZ][TX + 1];   // net flux H - V through the west face of local cell (i, j)
        __shared__ S sGz[4][TZ + 1][TX];   // ... through the south face
        __shared__ S sD[MODE == FV_DEFRES ? 4 : 1][MODE == FV_DEFRES ? TZ : 1][MODE == FV_DEFRES ? TX : 1];
        if (IN < 2) load_pt(&spt, K.pt);
        FLoad<T, IN> ld = ld0;
        ld.prepare();
        const int NX = K.NX, NZ = K.NZ;
        const size_t n1 = (size_t)NX * NZ;
        const int ntx = (NX + TX - 1) / TX;
        const int I0 = (int)(jf_bid % ntx) * TX, J0 = (int)(jf_bid / ntx) * TZ;
        const int tx = threadIdx.x % TX, tz = threadIdx.x / TX;
        const int I = I0 + tx, J = J0 + tz;
        const bool live = I < NX && J < NZ;
        const size_t c = live ? (size_t)J * NX + I : 0;
        // the epilogue's operands, loaded before the face work so that their latency overlaps it
        S xv[4], bv[4], up0 = 0, dtc = 0;
        double fuv[4] = {0.0, 0.0, 0.0, 0.0};
        if (live) {
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                const size_t gi = (size_t)v * n1 + c;
                xv[v] = MODE == FV_RES ? (S)0 : (S)ld.dir(v, c, I, J);
                bv[v] = MODE == FV_RES ? (S)0 : b[gi];
                if (IN == 1) fuv[v] = fu[gi];
            }
            up0 = (S)oval(ld(0, c, I, J));
            if (MODE == FV_SMOOTH) dtc = dtau[c];
        }
        if (IN < 2) __syncthreads();   // the power table
        for (int idx = threadIdx.x; idx < (TZ + 2) * (TX + 2); idx += blockDim.x) {
            const int li = idx % (TX + 2), lj = idx / (TX + 2);
            int I = I0 + li - 1;
            const int J = J0 + lj - 1;
            if (K.periodic) I = I < 0 ? I + NX : (I >= NX ? I - NX : I);
            if (I >= 0 && I < NX && J >= 0 && J < NZ) {
                const size_t c = (size_t)J * NX + I;
                T U[4];
    #pragma unroll
                for (int v = 0; v < 4; ++v) U[v] = ld(v, c, I, J) + bgs(K.ub, K.ubf, v * NZ + J, T{});
                Side<T> sd;
                side_of(U, K.pc, &spt, sd);
    #pragma unroll
                for (int v = 0; v < 4; ++v) sU[v][lj][li] = sd.U[v];
                sIr[lj][li] = sd.ir;
                sP[lj][li] = sd.p;
                sC[lj][li] = sd.c;
            }
        }
        __syncthreads();
        auto side_at = [&](int lj, int li, Side<T> &sd) {
    #pragma unroll
            for (int v = 0; v < 4; ++v) sd.U[v] = sU[v][lj][li];
            sd.ir = sIr[lj][li];
            sd.p = sP[lj][li];
            sd.c = sC[lj][li];
        };
        const bool sub = (IN < 2);
        const auto cx = mkc(K.vcx, K.vcxf, T{}), cz = mkc(K.vcz, K.vczf, T{});
        // x face west of local cell (i, j): global face index I0 + i in [0, NX]
        auto xface = [&](int i, int j) {
            const int If = I0 + i, J = J0 + j;
            if (If > NX || J >= NZ) return;
            const bool wl = !K.periodic && If == 0, wr = !K.periodic && If == NX;
            Side<T> L, R;
            T H[4];
            if (wl) {
                side_at(j + 1, i + 1, R);
                mirror_side<T, 0>(R, L);
            } else if (wr) {
                side_at(j + 1, i, L);
                mirror_side<T, 0>(L, R);
            } else {
                side_at(j + 1, i, L);
                side_at(j + 1, i + 1, R);
            }
            hllc_s<T, 0>(L, R, H);
            if (sub) {
                const double *hb = wl ? K.hbxw : (wr ? K.hbxw + 4 * NZ : K.hbx);
    #pragma unroll
                for (int v = 0; v < 4; ++v) H[v] = H[v] - mk(hb[v * NZ + J], T{});
            }
            if (VISC && !wl && !wr) {
                T V[4];
                visc2_s(L, R, cx, V);
    #pragma unroll
                for (int v = 1; v < 4; ++v) H[v] = H[v] - V[v];
            }
    #pragma unroll
            for (int v = 0; v < 4; ++v) sGx[v][j][i] = (S)oval(H[v]);
        };
        // z face south of local cell (i, j): global face index J0 + j in [0, NZ]
        auto zface = [&](int i, int j) {
            const int I = I0 + i, Jf = J0 + j;
            if (I >= NX || Jf > NZ) return;
            const bool wl = Jf == 0, wr = Jf == NZ;
            Side<T> B, Tp;
            T H[4];
            if (wl) {
                side_at(j + 1, i + 1, Tp);
                mirror_side<T, 1>(Tp, B);
            } else if (wr) {
                side_at(j, i + 1, B);
                mirror_side<T, 1>(B, Tp);
            } else {
                side_at(j, i + 1, B);
                side_at(j + 1, i + 1, Tp);
            }
            hllc_s<T, 1>(B, Tp, H);
            if (sub) {
    #pragma unroll
                for (int v = 0; v < 4; ++v) H[v] = H[v] - mk(K.hbz[v * (NZ + 1) + Jf], T{});
            }
            if (VISC && !wl && !wr) {
                T V[4];
                visc2_s(B, Tp, cz, V);
    #pragma unroll
                for (int v = 1; v < 4; ++v) H[v] = H[v] - V[v];
            }
    #pragma unroll
            for (int v = 0; v < 4; ++v) sGz[v][j][i] = (S)oval(H[v]);
        };
        xface(tx, tz);
        zface(tx, tz);
        if (tz == 0) zface(tx, TZ);              // north edge of the tile
        else if (tz == 1 && tx < TZ) xface(TX, tx);   // east edge of the tile
        __syncthreads();
        const S iHx = pick<S>(K.iHx, K.iHxf), iHz = pick<S>(K.iHz, K.iHzf);
        const float adtf = IN >= 2 ? K.adtf : 0.0f;
        const double eps = ld.step();
        if (live) {
    #pragma unroll
            for (int v = 0; v < 4; ++v) {
                S f = (sGx[v][tz][tx] - sGx[v][tz][tx + 1]) * iHx + (sGz[v][tz][tx] - sGz[v][tz + 1][tx]) * iHz;
                if (v == 2) f -= pick<S>(K.g, K.gf) * up0;   // -g rho' (tangent: -g x_rho)
                const size_t gi = (size_t)v * n1 + c;
                if (MODE == FV_RES) {
                    out[gi] = f;
                    continue;
                }
                const S x = xv[v];
                S gx;
                if (IN == 1) gx = (S)((eps == 0.0) ? (double)x : (double)x - adt * ((double)f - fuv[v]) / eps);
                else gx = x - (S)adtf * f;
                if (MODE == FV_SMOOTH) out[gi] = store_round<S>(rk_stage<S>(rk, x, dtc, bv[v] - gx, gi), bf16);
                else if (MODE == FV_DEFECT) out[gi] = gx - bv[v];
                else sD[v][tz][tx] = gx - bv[v];
            }
        }
        if (MODE != FV_DEFRES) return;
        __syncthreads();
        // 2 x 2 restriction: thread (ci, cj) of the first TX/2 x TZ/2 threads
        const int ci = threadIdx.x % (TX / 2), cj = threadIdx.x / (TX / 2);
        if (cj >= TZ / 2) return;
        const int Ic = I0 / 2 + ci, Jc = J0 / 2 + cj, NXc = NX / 2, NZc = NZ / 2;
        if (Ic >= NXc || Jc >= NZc) return;
        const size_t nc = (size_t)NXc * NZc, cc = (size_t)Jc * NXc + Ic;
    #pragma unroll
        for (int v = 0; v < 4; ++v) {
            const S a = (sD[v][2 * cj][2 * ci] + sD[v][2 * cj][2 * ci + 1]) +
                        (sD[v][2 * cj + 1][2 * ci] + sD[v][2 * cj + 1][2 * ci + 1]);
            const S bv = store_round<S>(a * (S)0.25, bf16);
            out[(size_t)v * nc + cc] = bv;
            if (xc) xc[(size_t)v * nc + cc] = store_round<S>(dtau_c[cc] * bv, bf16);
        }
    }
};
template <class T, int IN, int MODE, bool VISC, int TZ>
__global__ void __launch_bounds__(FV_TX * TZ) k_fv_tile(FVK K, FLoad<T, IN> ld0, const typename SOf<T>::type *b,
                                                      const typename SOf<T>::type *dtau, const double *fu,
                                                      double adt, typename SOf<T>::type *out,
                                                      typename SOf<T>::type *xc,
                                                      const typename SOf<T>::type *dtau_c, int bf16, RKS rk) {
    k_fv_tile_b<T, IN, MODE, VISC, TZ>::run(blockIdx.x, gridDim.x, K, ld0, b, dtau, fu, adt, out, xc, dtau_c, bf16, rk);
}

// FV pseudo-time step sizes: dtau = sigma / (1 + adt lambda), lambda = sum_faces
// 1/2 s_e |e|/|c| + 2 mu (1/Hx^2 + 1/Hz^2), s_e = max over both sides of |v.n| + c.
// wave speed |v . e_D| + c in the storage precision of the level
template <class R>
JF_D R wave_speed_r(const R U[4], int D, const PhysC &P, const PowTab *pt);
template <>
JF_D double wave_speed_r<double>(const double U[4], int D, const PhysC &P, const PowTab *pt) {
    return wave_speed(U, D, P, pt);
}
template <>
JF_D float wave_speed_r<float>(const float U[4], int D, const PhysC &P, const PowTab *) {
    const float ir = 1.0f / U[0];
    const float p = P.p0f * __powf(P.R_over_p0f * U[3], P.gammaf);
    return fabsf(U[1 + D] * ir) + sqrtf(P.gammaf * p * ir);
}

template <class S>
struct k_fv_dtau_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<FVK> K, JfArg<const S *> u,
                                               JfArg<double> adt, JfArg<double> sigma, JfArg<S *> dtau) {
        jf_pdl_enter();
        __shared__ PowTab spt;
        load_pt(&spt, K.pt);
        __syncthreads();
        const int NX = K.NX, NZ = K.NZ;
        const size_t n1 = (size_t)NX * NZ;
        const size_t c = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (c >= n1) return;
        const int I = (int)(c % NX), Jz = (int)(c / NX);
        auto st = [&](int i, int j, S U[4]) {
            const size_t cc = (size_t)j * NX + i;
            for (int v = 0; v < 4; ++v) U[v] = u[(size_t)v * n1 + cc] + pick<S>(K.ub[v * NZ + j], K.ubf[v * NZ + j]);
        };
        S U[4], V[4];
        st(I, Jz, U);
        const S sx = wave_speed_r<S>(U, 0, K.pc, &spt), sz = wave_speed_r<S>(U, 1, K.pc, &spt);
        S eW = sx, eE = sx, eS = sz, eN = sz;
        if (I > 0 || K.periodic) { st(I > 0 ? I - 1 : NX - 1, Jz, V); eW = fmax(sx, wave_speed_r<S>(V, 0, K.pc, &spt)); }
        if (I < NX - 1 || K.periodic) { st(I < NX - 1 ? I + 1 : 0, Jz, V); eE = fmax(sx, wave_speed_r<S>(V, 0, K.pc, &spt)); }
        if (Jz > 0) { st(I, Jz - 1, V); eS = fmax(sz, wave_speed_r<S>(V, 1, K.pc, &spt)); }
        if (Jz < NZ - 1) { st(I, Jz + 1, V); eN = fmax(sz, wave_speed_r<S>(V, 1, K.pc, &spt)); }
        const S iHx = (S)K.iHx, iHz = (S)K.iHz;
        const S lam = (S)0.5 * (eW + eE) * iHx + (S)0.5 * (eS + eN) * iHz + (S)(2.0 * K.mu) * (iHx * iHx + iHz * iHz);
        dtau[c] = (S)sigma / ((S)1 + (S)adt * lam);
    }
};
template <class S>
__global__ void k_fv_dtau(FVK K, const S *u, double adt, double sigma, S *dtau) {
    k_fv_dtau_b<S>::run(blockIdx.x, gridDim.x, K, u, adt, sigma, dtau);
}

// DG pseudo-time step per element: lambda_E = (k+1)^2 max_nodes(|v| + c)(1/hx + 1/hz)
// + 2 mu (k+1)^4 (1/hx^2 + 1/hz^2).
template <class R>
struct k_dg_dtau_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const R *> U,
                                               JfArg<const R *> ubv, JfArg<int> nx, JfArg<int> nz, JfArg<int> np1,
                                               JfArg<PhysC> pc, JfArg<const PowTab *> pt, JfArg<double> ihx,
                                               JfArg<double> ihz, JfArg<double> mu, JfArg<double> adt,
                                               JfArg<double> sigma, JfArg<double *> dtau, JfArg<float *> dtauf) {
        jf_pdl_enter();
        __shared__ PowTab spt;
        if (sizeof(R) == 8) load_pt(&spt, pt);
        __syncthreads();
        // one warp per element, one lane per node, max over the lanes
        const int n_el = nx * nz;
        const int lane = threadIdx.x & 31;
        const int e = (int)(((size_t)jf_bid * blockDim.x + threadIdx.x) >> 5);
        if (e >= n_el) return;   // uniform over the warp
        const int NP = np1 * np1;
        const size_t N1 = (size_t)n_el * NP;
        const int ez = e / nx;
        const size_t nrow = (size_t)nz * np1;
        R sp = 0;
        if (lane < NP) {
            const int J = ez * np1 + lane / np1;
            R W[4];
            for (int v = 0; v < 4; ++v) W[v] = U[v * N1 + (size_t)e * NP + lane] + ubv[v * nrow + J];
            if (sizeof(R) == 8) {
                const double ir = 1.0 / (double)W[0];
                const double p = pc.p0 * pow_gamma_tab(pc.R_over_p0 * (double)W[3], &spt);
                sp = (R)(sqrt(((double)W[1] * ir) * ((double)W[1] * ir) + ((double)W[2] * ir) * ((double)W[2] * ir)) +
                         sqrt(pc.gamma * p * ir));
            } else {
                const float ir = 1.0f / (float)W[0];
                const float p = pc.p0f * __powf(pc.R_over_p0f * (float)W[3], pc.gammaf);
                sp = (R)(sqrtf(((float)W[1] * ir) * ((float)W[1] * ir) + ((float)W[2] * ir) * ((float)W[2] * ir)) +
                         sqrtf(pc.gammaf * p * ir));
            }
        }
    #pragma unroll
        for (int o = 16; o > 0; o >>= 1) sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, o));
        if (lane != 0) return;
        const double vmax = (double)sp;
        const double n2 = (double)np1 * np1;
        const double lam = n2 * vmax * (ihx + ihz) + 2.0 * mu * n2 * n2 * (ihx * ihx + ihz * ihz);
        const double d = sigma / (1.0 + adt * lam);
        if (dtau) dtau[e] = d;
        if (dtauf) dtauf[e] = (float)d;
    }
};
template <class R>
__global__ void k_dg_dtau(const R *U, const R *ubv, int nx, int nz, int np1, PhysC pc, const PowTab *pt,
                          double ihx, double ihz, double mu, double adt, double sigma, double *dtau,
                          float *dtauf) {
    k_dg_dtau_b<R>::run(blockIdx.x, gridDim.x, U, ubv, nx, nz, np1, pc, pt, ihx, ihz, mu, adt, sigma, dtau, dtauf);
}

// ---- transfer -------------------------------------------------------------
struct TK {
    int nx, nz, np1, n_el, NX, NZ;
    DGTab tab;
};

template <class Si, class So> struct RealOf { typedef float type; };
template <> struct RealOf<double, double> { typedef double type; };

template <class R, int NP1>
__device__ __forceinline__ void load_ttab(const TK &K, R sV[NP1][NP1], R sVi[NP1][NP1], R som[NP1]) {
    for (int t = threadIdx.x; t < NP1 * NP1; t += blockDim.x) {
        sV[t / NP1][t % NP1] = (R)K.tab.V[t / NP1][t % NP1];
        sVi[t / NP1][t % NP1] = (R)K.tab.Vinv[t / NP1][t % NP1];
    }
    for (int t = threadIdx.x; t < NP1; t += blockDim.x) som[t] = (R)K.tab.om[t];
}

// T^mf: DG (Si) -> FV (So), arithmetic in the storage precision.  Block: EPB
// elements x NP subcells.
template <class Si, class So, int NP1>
struct k_to_fv_b {
    static constexpr int TPB = 128, MINB = 0;
    static constexpr bool GROUP = std::is_same<So, float>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<TK> K, JfArg<const Si *> u,
                                               JfArg<So *> v, JfArg<int> massfix, JfArg<So *> x0,
                                               JfArg<const So *> dtau0) {
        jf_pdl_enter();
        typedef typename RealOf<Si, So>::type R;
        constexpr int NP = NP1 * NP1;
        constexpr int EPB = (128 / NP) > 0 ? 128 / NP : 1;
        __shared__ R su[EPB][4][NP];
        __shared__ R st[EPB][4][NP];
        __shared__ R sc[EPB][4];
        __shared__ R sV[NP1][NP1], sVi[NP1][NP1], som[NP1];
        load_ttab<R, NP1>(K, sV, sVi, som);
        const int le = threadIdx.x / NP, node = threadIdx.x % NP;
        const int e = jf_bid * EPB + le;
        const bool act = e < K.n_el;
        const size_t N1 = (size_t)K.n_el * NP;
        const int i = node % NP1, j = node / NP1;   // subcell (i along x, j along z) / node (a, b)
        if (act)
            for (int q = 0; q < 4; ++q) su[le][q][node] = (R)u[q * N1 + (size_t)e * NP + node];
        __syncthreads();
        // t1(i, b) = sum_a V[i][a] u(a, b), stored at [b][i]
        if (act)
            for (int q = 0; q < 4; ++q) {
                R acc = 0;
    #pragma unroll
                for (int a = 0; a < NP1; ++a) acc = fma(sV[i][a], su[le][q][j * NP1 + a], acc);
                st[le][q][j * NP1 + i] = acc;
            }
        __syncthreads();
        R Tu[4];
        if (act)
            for (int q = 0; q < 4; ++q) {
                R acc = 0;
    #pragma unroll
                for (int b = 0; b < NP1; ++b) acc = fma(sV[j][b], st[le][q][b * NP1 + i], acc);
                Tu[q] = acc;
            }
        __syncthreads();
        if (act)
            for (int q = 0; q < 4; ++q) su[le][q][node] = Tu[q];
        __syncthreads();
        if (act && node < 4) {
            // m_E(T u)/|E| = subcell mean; m_E(u)/|E| by the midpoint weights on the subcell values
            const int q = node;
            R mfv = 0, mnc = 0;
            for (int jj = 0; jj < NP1; ++jj)
                for (int ii = 0; ii < NP1; ++ii) {
                    const R x = su[le][q][jj * NP1 + ii];
                    mfv += x;
                    mnc = fma(som[ii] * som[jj], x, mnc);
                }
            sc[le][q] = massfix ? (mfv / (R)NP - mnc) : (R)0;
        }
        __syncthreads();
        if (!act) return;
        const int ez = e / K.nx, ex = e % K.nx;
        const size_t I = (size_t)ex * NP1 + i, Jr = (size_t)ez * NP1 + j;
        const size_t n1 = (size_t)K.NX * K.NZ;
        for (int q = 0; q < 4; ++q) {
            const So val = (So)(Tu[q] - sc[le][q]);
            v[q * n1 + Jr * K.NX + I] = val;
            if (x0) x0[q * n1 + Jr * K.NX + I] = dtau0[Jr * K.NX + I] * val;   // first step from zero
        }
    }
};
template <class Si, class So, int NP1>
__global__ void __launch_bounds__(128) k_to_fv(TK K, const Si *u, So *v, int massfix, So *x0, const So *dtau0) {
    k_to_fv_b<Si, So, NP1>::run(blockIdx.x, gridDim.x, K, u, v, massfix, x0, dtau0);
}

// T^-1_mf: FV (Si) -> DG (So); acc 0: store, 1: add
template <class Si, class So, int NP1>
struct k_to_dg_b {
    static constexpr int TPB = 128, MINB = 0;
    static constexpr bool GROUP = std::is_same<Si, float>::value;   // a grouped twin is built (lock-step ensembles)
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<TK> K, JfArg<const Si *> v,
                                               JfArg<So *> u, JfArg<int> massfix, JfArg<int> acc_mode) {
        jf_pdl_enter();
        typedef typename RealOf<Si, So>::type R;
        constexpr int NP = NP1 * NP1;
        constexpr int EPB = (128 / NP) > 0 ? 128 / NP : 1;
        __shared__ R sv[EPB][4][NP];
        __shared__ R st[EPB][4][NP];
        __shared__ R sc[EPB][4];
        __shared__ R sV[NP1][NP1], sVi[NP1][NP1], som[NP1];
        load_ttab<R, NP1>(K, sV, sVi, som);
        const int le = threadIdx.x / NP, node = threadIdx.x % NP;
        const int e = jf_bid * EPB + le;
        const bool act = e < K.n_el;
        const size_t n1 = (size_t)K.NX * K.NZ;
        const int a = node % NP1, b = node / NP1;
        const int ez = act ? e / K.nx : 0, ex = act ? e % K.nx : 0;
        if (act) {
            const size_t I = (size_t)ex * NP1 + a, Jr = (size_t)ez * NP1 + b;   // subcell (a, b) here
            for (int q = 0; q < 4; ++q) sv[le][q][node] = (R)v[q * n1 + Jr * K.NX + I];
        }
        __syncthreads();
        if (act)
            for (int q = 0; q < 4; ++q) {   // t1(a, j) = sum_i Vinv[a][i] v(i, j), at [j][a]
                R acc = 0;
    #pragma unroll
                for (int i = 0; i < NP1; ++i) acc = fma(sVi[a][i], sv[le][q][b * NP1 + i], acc);
                st[le][q][b * NP1 + a] = acc;
            }
        __syncthreads();
        R Ti[4];
        if (act)
            for (int q = 0; q < 4; ++q) {
                R acc = 0;
    #pragma unroll
                for (int jj = 0; jj < NP1; ++jj) acc = fma(sVi[b][jj], st[le][q][jj * NP1 + a], acc);
                Ti[q] = acc;
            }
        if (act && node < 4) {
            // m_E(T^-1 v)/|E| from the subcell values (T T^-1 v = v) by the midpoint weights,
            // m_E(v)/|E| the subcell mean
            const int q = node;
            R mfv = 0, mnc = 0;
            for (int jj = 0; jj < NP1; ++jj)
                for (int ii = 0; ii < NP1; ++ii) {
                    const R x = sv[le][q][jj * NP1 + ii];
                    mfv += x;
                    mnc = fma(som[ii] * som[jj], x, mnc);
                }
            sc[le][q] = massfix ? (mnc - mfv / (R)NP) : (R)0;
        }
        __syncthreads();
        if (!act) return;
        const size_t N1 = (size_t)K.n_el * NP;
        for (int q = 0; q < 4; ++q) {
            const size_t gi = q * N1 + (size_t)e * NP + node;
            const R val = Ti[q] - sc[le][q];
            u[gi] = acc_mode ? (So)((R)u[gi] + val) : (So)val;
        }
    }
};
template <class Si, class So, int NP1>
__global__ void __launch_bounds__(128) k_to_dg(TK K, const Si *v, So *u, int massfix, int acc_mode) {
    k_to_dg_b<Si, So, NP1>::run(blockIdx.x, gridDim.x, K, v, u, massfix, acc_mode);
}

// R: coarse = mean of fac x fac children
template <class S>
struct k_restrict_body {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> f, JfArg<int> NXf,
                                               JfArg<int> NZf, JfArg<int> fac, JfArg<S *> cz) {
        jf_pdl_enter();
        const int NXc = NXf / fac, NZc = NZf / fac;
        const size_t nc = (size_t)NXc * NZc;
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t >= 4 * nc) return;
        const int q = (int)(t / nc);
        const size_t c = t % nc;
        const int I = (int)(c % NXc), J = (int)(c / NXc);
        const S *fq = f + (size_t)q * NXf * NZf;
        S acc = 0;
        for (int jj = 0; jj < fac; ++jj)
            for (int ii = 0; ii < fac; ++ii) acc += fq[(size_t)(J * fac + jj) * NXf + I * fac + ii];
        cz[t] = acc / (S)(fac * fac);
    }
};
template <class S>
__global__ void k_restrict(const S *f, int NXf, int NZf, int fac, S *cz) {
    k_restrict_body<S>::run(blockIdx.x, gridDim.x, f, NXf, NZf, fac, cz);
}

// R plus the coarse level's first pseudo-time step from zero: b_c = R r and,
// when x_c is given, x_c = dtau_c b_c
template <class S>
struct k_restrict_b_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> f, JfArg<int> NXf,
                                               JfArg<int> NZf, JfArg<int> fac, JfArg<S *> bc, JfArg<S *> xc,
                                               JfArg<const S *> dtau_c, JfArg<int> bf16) {
        jf_pdl_enter();
        const int NXc = NXf / fac, NZc = NZf / fac;
        const size_t nc = (size_t)NXc * NZc;
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t >= 4 * nc) return;
        const int q = (int)(t / nc);
        const size_t c = t % nc;
        const int I = (int)(c % NXc), J = (int)(c / NXc);
        const S *fq = f + (size_t)q * NXf * NZf;
        S acc = 0;
        for (int jj = 0; jj < fac; ++jj)
            for (int ii = 0; ii < fac; ++ii) acc += fq[(size_t)(J * fac + jj) * NXf + I * fac + ii];
        const S bv = store_round<S>(acc / (S)(fac * fac), bf16);
        bc[t] = bv;
        if (xc) xc[t] = store_round<S>(dtau_c[c] * bv, bf16);
    }
};
template <class S>
__global__ void k_restrict_b(const S *f, int NXf, int NZf, int fac, S *bc, S *xc, const S *dtau_c, int bf16 = 0) {
    k_restrict_b_b<S>::run(blockIdx.x, gridDim.x, f, NXf, NZf, fac, bc, xc, dtau_c, bf16);
}

// x = (zero ? 0 : x) - P v
template <class S>
struct k_prolong_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<S *> x, JfArg<const S *> vc,
                                               JfArg<int> NXf, JfArg<int> NZf, JfArg<int> fac, JfArg<int> zero) {
        jf_pdl_enter();
        const size_t nf = (size_t)NXf * NZf;
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t >= 4 * nf) return;
        const int q = (int)(t / nf);
        const size_t c = t % nf;
        const int I = (int)(c % NXf), J = (int)(c / NXf);
        const int NXc = NXf / fac, NZc = NZf / fac;
        const S pv = vc[(size_t)q * NXc * NZc + (size_t)(J / fac) * NXc + I / fac];
        x[t] = zero ? -pv : x[t] - pv;
    }
};
template <class S>
__global__ void k_prolong(S *x, const S *vc, int NXf, int NZf, int fac, int zero) {
    k_prolong_b<S>::run(blockIdx.x, gridDim.x, x, vc, NXf, NZf, fac, zero);
}

// x = dtau b (first smoothing step from zero)
template <class S>
struct k_scale_dtau_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<S *> x, JfArg<const S *> b,
                                               JfArg<const S *> dtau, JfArg<size_t> n1, JfArg<double> alpha) {
        jf_pdl_enter();
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t >= 4 * n1) return;
        x[t] = ((S)alpha * dtau[t % n1]) * b[t];   // alpha = 1: dtau b exactly
    }
};
template <class S>
__global__ void k_scale_dtau(S *x, const S *b, const S *dtau, size_t n1, double alpha) {
    k_scale_dtau_b<S>::run(blockIdx.x, gridDim.x, x, b, dtau, n1, alpha);
}

template <class S>
struct k_scale_dtau_dg_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<S *> z, JfArg<const S *> r,
                                               JfArg<const S *> dtau, JfArg<size_t> N1, JfArg<int> NP,
                                               JfArg<double> alpha) {
        jf_pdl_enter();
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t >= 4 * N1) return;
        z[t] = ((S)alpha * dtau[(t % N1) / NP]) * r[t];   // alpha = 1: dtau r exactly
    }
};
template <class S>
__global__ void k_scale_dtau_dg(S *z, const S *r, const S *dtau, size_t N1, int NP, double alpha) {
    k_scale_dtau_dg_b<S>::run(blockIdx.x, gridDim.x, z, r, dtau, N1, NP, alpha);
}

template <class S>
struct k_neg_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<S *> x, JfArg<const S *> b,
                                               JfArg<size_t> n) {
        jf_pdl_enter();
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t < n) x[t] = -b[t];
    }
};
template <class S>
__global__ void k_neg(S *x, const S *b, size_t n) {
    k_neg_b<S>::run(blockIdx.x, gridDim.x, x, b, n);
}

template <class S>
struct k_sub_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> r,
                                               JfArg<const S *> w, JfArg<S *> d, JfArg<size_t> n) {
        jf_pdl_enter();   // d = r - w
        const size_t t = (size_t)jf_bid * blockDim.x + threadIdx.x;
        if (t < n) d[t] = r[t] - w[t];
    }
};
template <class S>
__global__ void k_sub(const S *r, const S *w, S *d, size_t n) {
    k_sub_b<S>::run(blockIdx.x, gridDim.x, r, w, d, n);
}

__global__ void k_bg_fv(FVK K, double *hbx, double *hbxw, double *hbz) {
    jf_pdl_enter();
    __shared__ PowTab spt;
    load_pt(&spt, K.pt);
    __syncthreads();
    const int NZ = K.NZ;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    D64 U[4], G[4], H[4];
    if (i < NZ) {
        for (int v = 0; v < 4; ++v) U[v] = D64{K.ub[v * NZ + i]};
        hllc<D64, 0>(U, U, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbx[v * NZ + i] = H[v].x;
        mirror<D64, 0>(U, G);
        hllc<D64, 0>(G, U, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbxw[v * NZ + i] = H[v].x;
        hllc<D64, 0>(U, G, K.pc, &spt, H);
        for (int v = 0; v < 4; ++v) hbxw[(4 + v) * NZ + i] = H[v].x;
    } else if (i < 2 * NZ + 1) {
        const int j = i - NZ;   // face between rows j-1 and j
        D64 B[4], T_[4];
        if (j == 0) {
            for (int v = 0; v < 4; ++v) T_[v] = D64{K.ub[v * NZ + 0]};
            mirror<D64, 1>(T_, G);
            hllc<D64, 1>(G, T_, K.pc, &spt, H);
        } else if (j == NZ) {
            for (int v = 0; v < 4; ++v) B[v] = D64{K.ub[v * NZ + NZ - 1]};
            mirror<D64, 1>(B, G);
            hllc<D64, 1>(B, G, K.pc, &spt, H);
        } else {
            for (int v = 0; v < 4; ++v) {
                B[v] = D64{K.ub[v * NZ + j - 1]};
                T_[v] = D64{K.ub[v * NZ + j]};
            }
            hllc<D64, 1>(B, T_, K.pc, &spt, H);
        }
        for (int v = 0; v < 4; ++v) hbz[v * (NZ + 1) + j] = H[v].x;
    }
}

inline unsigned nblk(size_t n, int bs = 128) { return (unsigned)((n + bs - 1) / bs); }

FVK make_fvk(jfnk_ctx *c, int l) {
    const FVLev &L = c->lev[l];
    FVK K;
    K.NX = L.NX;
    K.NZ = L.NZ;
    K.periodic = c->grid.periodic_x;
    K.iHx = 1.0 / L.Hx;
    K.iHz = 1.0 / L.Hz;
    K.g = c->phys.g;
    K.mu = c->phys.mu;
    K.vcx = 0.5 * K.mu * K.iHx;
    K.vcz = 0.5 * K.mu * K.iHz;
    K.iHxf = (float)K.iHx;
    K.iHzf = (float)K.iHz;
    K.gf = (float)K.g;
    K.vcxf = (float)K.vcx;
    K.vczf = (float)K.vcz;
    K.adtf = (float)c->mg_adt;
    K.pc = c->pc;
    K.pt = c->powtab;
    K.ub = L.ub;
    K.hbx = L.hbx;
    K.hbxw = L.hbxw;
    K.hbz = L.hbz;
    K.ubf = L.ubf;
    return K;
}

TK make_tk(jfnk_ctx *c) {
    TK K;
    K.nx = c->grid.nx;
    K.nz = c->grid.nz;
    K.np1 = c->np1;
    K.n_el = c->n_el;
    K.NX = c->lev[0].NX;
    K.NZ = c->lev[0].NZ;
    K.tab = c->tab;
    if (c->opts.transfer_l2) {   // L2 projection: subcell averages and their inverse
        for (int i = 0; i < 5; ++i)
            for (int a = 0; a < 5; ++a) {
                K.tab.V[i][a] = c->tab.P[i][a];
                K.tab.Vinv[i][a] = c->tab.Pinv[i][a];
            }
    }
    return K;
}

template <class Si, class So>
int to_fv(jfnk_ctx *c, const Si *u, So *v, cudaStream_t s, So *x0 = nullptr, const So *dtau0 = nullptr) {
    TK K = make_tk(c);
    const int NP = c->np1 * c->np1;
    const int EPB = (128 / NP) > 0 ? 128 / NP : 1;
    const unsigned g = (unsigned)((c->n_el + EPB - 1) / EPB);
    switch (c->np1) {
        case 2: jf_launch<k_to_fv_b<Si, So, 2>>(k_to_fv<Si, So, 2>, g, EPB * NP, 0, s, K, u, v, c->opts.massfix && !c->opts.transfer_l2, x0, dtau0); jf_launched(); break;
        case 3: jf_launch<k_to_fv_b<Si, So, 3>>(k_to_fv<Si, So, 3>, g, EPB * NP, 0, s, K, u, v, c->opts.massfix && !c->opts.transfer_l2, x0, dtau0); jf_launched(); break;
        case 4: jf_launch<k_to_fv_b<Si, So, 4>>(k_to_fv<Si, So, 4>, g, EPB * NP, 0, s, K, u, v, c->opts.massfix && !c->opts.transfer_l2, x0, dtau0); jf_launched(); break;
        case 5: jf_launch<k_to_fv_b<Si, So, 5>>(k_to_fv<Si, So, 5>, g, EPB * NP, 0, s, K, u, v, c->opts.massfix && !c->opts.transfer_l2, x0, dtau0); jf_launched(); break;
        default: return JFNK_EINVAL;
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

template <class Si, class So>
int to_dg(jfnk_ctx *c, const Si *v, So *u, int acc, cudaStream_t s) {
    TK K = make_tk(c);
    const int NP = c->np1 * c->np1;
    const int EPB = (128 / NP) > 0 ? 128 / NP : 1;
    const unsigned g = (unsigned)((c->n_el + EPB - 1) / EPB);
    switch (c->np1) {
        case 2: jf_launch<k_to_dg_b<Si, So, 2>>(k_to_dg<Si, So, 2>, g, EPB * NP, 0, s, K, v, u, c->opts.massfix && !c->opts.transfer_l2, acc); jf_launched(); break;
        case 3: jf_launch<k_to_dg_b<Si, So, 3>>(k_to_dg<Si, So, 3>, g, EPB * NP, 0, s, K, v, u, c->opts.massfix && !c->opts.transfer_l2, acc); jf_launched(); break;
        case 4: jf_launch<k_to_dg_b<Si, So, 4>>(k_to_dg<Si, So, 4>, g, EPB * NP, 0, s, K, v, u, c->opts.massfix && !c->opts.transfer_l2, acc); jf_launched(); break;
        case 5: jf_launch<k_to_dg_b<Si, So, 5>>(k_to_dg<Si, So, 5>, g, EPB * NP, 0, s, K, v, u, c->opts.massfix && !c->opts.transfer_l2, acc); jf_launched(); break;
        default: return JFNK_EINVAL;
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// ---- FV level products ----------------------------------------------------
// four lanes per cell on levels with fewer cells than opts.fv_split_cells
// (default 65536), one thread per cell above
inline bool fv_four_lanes(const jfnk_ctx *c, size_t cells) {
    const long long lim = c->opts.fv_split_cells > 0 ? c->opts.fv_split_cells : 65536;
    return (long long)cells < lim;
}
template <class T, int IN, int MODE, bool V>
void launch_fv(bool l4, unsigned g, int tb, cudaStream_t s, const FVK &K, const FLoad<T, IN> &ld,
               const typename SOf<T>::type *x, const typename SOf<T>::type *b, const typename SOf<T>::type *dt,
               const double *fu, double adt, typename SOf<T>::type *out, int bf = 0,
               RKS rk = RKS{nullptr, 0, 1.0, 1.0f}) {
    if (l4) {
        jf_launch<k_fv_b<T, IN, MODE, V, 4>>(k_fv<T, IN, MODE, V, 4>, g, tb, 0, s, K, ld, x, b, dt, fu, adt, out, bf, rk);
    } else if (tb >= 256) {   // tile rows follow the block size: 32 x 8 or 32 x 4 cells
        const unsigned gt = (unsigned)(((K.NX + FV_TX - 1) / FV_TX) * ((K.NZ + 7) / 8));
        jf_launch<k_fv_tile_b<T, IN, MODE, V, 8>>(k_fv_tile<T, IN, MODE, V, 8>, gt, FV_TX * 8, 0, s, K, ld, b, dt, fu, adt, out, nullptr, nullptr, bf,
                  rk);
    } else {
        const unsigned gt = (unsigned)(((K.NX + FV_TX - 1) / FV_TX) * ((K.NZ + 3) / 4));
        jf_launch<k_fv_tile_b<T, IN, MODE, V, 4>>(k_fv_tile<T, IN, MODE, V, 4>, gt, FV_TX * 4, 0, s, K, ld, b, dt, fu, adt, out, nullptr, nullptr, bf,
                  rk);
    }
    jf_launched();
}
#define JF_FV(T, IN, MODE, V, ...) launch_fv<T, IN, MODE, V>(l4, g, tb, s, __VA_ARGS__)
// FV_RES: out = f_low(u) (FP64 only).  FV_SMOOTH / FV_DEFECT use the FD quotient
// (prec 64, eps = sqrt(eps_mach)/|x| from an on-device norm) or the tangent (prec 32).
int fv_op64(jfnk_ctx *c, int l, int mode, const double *u, const double *x, const double *b, double *out,
            cudaStream_t s, RKS rk = RKS{nullptr, 0, 1.0, 1.0f}) {
    FVLev &L = c->lev[l];
    FVK K = make_fvk(c, l);
    const size_t n1 = (size_t)L.NX * L.NZ;
    const bool visc = c->phys.mu != 0.0;
    c->fv_calls++;
    const int tb = c->opts.tile_fv;
    const bool l4 = fv_four_lanes(c, n1);
    const unsigned g = nblk((l4 ? 4 : 1) * n1, tb);
    if (mode == FV_RES) {
        FLoad<D64, 0> ld{u, n1};
        if (visc) { JF_FV(D64, 0, FV_RES, true, K, ld, nullptr, nullptr, nullptr, nullptr, 0.0, out); }
        else { JF_FV(D64, 0, FV_RES, false, K, ld, nullptr, nullptr, nullptr, nullptr, 0.0, out); }
    } else {
        double *epsp = c->scal + S_EPSFV + l;
        JF_RET(red_dot(c, x, x, L.n, epsp, RED_EPSP, s));
        FLoad<D64, 1> ld{u, x, epsp, n1, 0.0};
        const double *dt = (const double *)L.dtau;
        const double *fu = (const double *)L.fu;
        const double adt = c->mg_adt;
        if (mode == FV_SMOOTH) {
            if (visc) { JF_FV(D64, 1, FV_SMOOTH, true, K, ld, x, b, dt, fu, adt, out, 0, rk); }
            else { JF_FV(D64, 1, FV_SMOOTH, false, K, ld, x, b, dt, fu, adt, out, 0, rk); }
        } else {
            if (visc) { JF_FV(D64, 1, FV_DEFECT, true, K, ld, x, b, dt, fu, adt, out); }
            else { JF_FV(D64, 1, FV_DEFECT, false, K, ld, x, b, dt, fu, adt, out); }
        }
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int fv_op32(jfnk_ctx *c, int l, int mode, const float *x, const float *b, float *out, cudaStream_t s,
            RKS rk = RKS{nullptr, 0, 1.0, 1.0f}) {
    FVLev &L = c->lev[l];
    FVK K = make_fvk(c, l);
    const size_t n1 = (size_t)L.NX * L.NZ;
    const bool visc = c->phys.mu != 0.0;
    c->fv_calls++;
    const int tb = c->opts.tile_fv;
    const bool l4 = fv_four_lanes(c, n1);
    const unsigned g = nblk((l4 ? 4 : 1) * n1, tb);
    FLoad<TL32, 2> ld{(const float *)L.u, x, n1};
    const float *dt = (const float *)L.dtau;
    const double adt = c->mg_adt;
    const int bf = (c->prec == 16 && l == c->nlev - 1) ? 1 : 0;   // BF16 coarsest level
    if (mode == FV_SMOOTH) {
        if (visc) { JF_FV(TL32, 2, FV_SMOOTH, true, K, ld, x, b, dt, nullptr, adt, out, bf, rk); }
        else { JF_FV(TL32, 2, FV_SMOOTH, false, K, ld, x, b, dt, nullptr, adt, out, bf, rk); }
    } else {
        if (visc) { JF_FV(TL32, 2, FV_DEFECT, true, K, ld, x, b, dt, nullptr, adt, out); }
        else { JF_FV(TL32, 2, FV_DEFECT, false, K, ld, x, b, dt, nullptr, adt, out); }
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// One FP32 smoothing step at the corrected iterate x - P v_c of level l (v_c = the
// coarse level's iterate), written to out: the prolongation and the first
// post-smoothing step in one launch.
int fv_smooth32_corrected(jfnk_ctx *c, int l, const float *x, bool zero, const float *b, float *out,
                          cudaStream_t s) {
    FVLev &L = c->lev[l];
    FVLev &C = c->lev[l + 1];
    FVK K = make_fvk(c, l);
    const size_t n1 = (size_t)L.NX * L.NZ;
    const bool visc = c->phys.mu != 0.0;
    c->fv_calls++;
    const int tb = c->opts.tile_fv;
    const bool l4 = fv_four_lanes(c, n1);
    const unsigned g = nblk((l4 ? 4 : 1) * n1, tb);
    FLoad<TL32, 3> ld{(const float *)L.u, x, (const float *)C.x, n1, C.NX, L.fac, zero ? 1 : 0,
                      (size_t)C.NX * C.NZ};
    const float *dt = (const float *)L.dtau;
    const double adt = c->mg_adt;
    const int bf = (c->prec == 16 && l == c->nlev - 1) ? 1 : 0;
    if (visc) { JF_FV(TL32, 3, FV_SMOOTH, true, K, ld, x, b, dt, nullptr, adt, out, bf); }
    else { JF_FV(TL32, 3, FV_SMOOTH, false, K, ld, x, b, dt, nullptr, adt, out, bf); }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// defect g'x - b on level l restricted to level l+1 (b_{l+1}, and x_{l+1} = dtau b
// when xc is given)
int fv_defect_restrict(jfnk_ctx *c, int l, const void *x, const void *b, void *bc, void *xc, const void *dtc,
                       cudaStream_t s) {
    FVLev &L = c->lev[l];
    FVLev &C = c->lev[l + 1];
    FVK K = make_fvk(c, l);
    const size_t n1 = (size_t)L.NX * L.NZ;
    const size_t nc = (size_t)C.NX * C.NZ;
    const bool visc = c->phys.mu != 0.0;
    const int tb = c->opts.tile_fv;
    const bool l4 = fv_four_lanes(c, n1);
    const bool f2 = L.fac == 2;
    const unsigned g = nblk((l4 ? (f2 ? 16 : 4) : 1) * nc, tb);   // lanes per coarse cell
    c->fv_calls++;
#define JF_DR(T, IN, V, LN, F2, ...) jf_launch<k_fv_defect_restrict_b<T, IN, V, LN, F2>>(k_fv_defect_restrict<T, IN, V, LN, F2>, g, tb, 0, s, __VA_ARGS__)
#define JF_DR2(T, IN, V, ...)                                \
    do {                                                     \
        if (!l4) JF_DR(T, IN, V, 1, false, __VA_ARGS__);     \
        else if (f2) JF_DR(T, IN, V, 4, true, __VA_ARGS__);  \
        else JF_DR(T, IN, V, 4, false, __VA_ARGS__);         \
    } while (0)
    // large levels with 2 x 2 agglomeration: the face-once tile kernel
    const int tz = tb >= 256 ? 8 : 4;   // tile rows follow the block size
    const unsigned gt = (unsigned)(((L.NX + FV_TX - 1) / FV_TX) * ((L.NZ + tz - 1) / tz));
#define JF_DRT(T, IN, V, ld, bb, fuu, outc, xcc, dtc_, bff)                                                     \
    do {                                                                                                        \
        if (tz == 8)                                                                                            \
            jf_launch<k_fv_tile_b<T, IN, FV_DEFRES, V, 8>>(k_fv_tile<T, IN, FV_DEFRES, V, 8>, gt, FV_TX * 8, 0, s, K, ld, bb, nullptr, fuu, c->mg_adt, \
                      outc, xcc, dtc_, bff, RKS{nullptr, 0, 1.0, 1.0f});                                                                    \
        else                                                                                                    \
            jf_launch<k_fv_tile_b<T, IN, FV_DEFRES, V, 4>>(k_fv_tile<T, IN, FV_DEFRES, V, 4>, gt, FV_TX * 4, 0, s, K, ld, bb, nullptr, fuu, c->mg_adt, \
                      outc, xcc, dtc_, bff, RKS{nullptr, 0, 1.0, 1.0f});                                                                    \
    } while (0)
    if (!l4 && f2) {
        if (c->prec == 64) {
            double *epsp = c->scal + S_EPSFV + l;
            JF_RET(red_dot(c, (const double *)x, (const double *)x, L.n, epsp, RED_EPSP, s));
            FLoad<D64, 1> ld{(const double *)L.u, (const double *)x, epsp, n1, 0.0};
            if (visc) JF_DRT(D64, 1, true, ld, (const double *)b, (const double *)L.fu, (double *)bc, (double *)xc, (const double *)dtc, 0);
            else JF_DRT(D64, 1, false, ld, (const double *)b, (const double *)L.fu, (double *)bc, (double *)xc, (const double *)dtc, 0);
        } else {
            FLoad<TL32, 2> ld{(const float *)L.u, (const float *)x, n1};
            const int bf = (c->prec == 16 && l + 1 == c->nlev - 1) ? 1 : 0;
            if (visc) JF_DRT(TL32, 2, true, ld, (const float *)b, nullptr, (float *)bc, (float *)xc, (const float *)dtc, bf);
            else JF_DRT(TL32, 2, false, ld, (const float *)b, nullptr, (float *)bc, (float *)xc, (const float *)dtc, bf);
        }
        jf_launched();
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    }
#undef JF_DRT
#define JF_DR4(T, IN, ...)                                   \
    do {                                                     \
        if (visc) JF_DR2(T, IN, true, __VA_ARGS__);          \
        else JF_DR2(T, IN, false, __VA_ARGS__);              \
    } while (0)
    if (c->prec == 64) {
        double *epsp = c->scal + S_EPSFV + l;
        JF_RET(red_dot(c, (const double *)x, (const double *)x, L.n, epsp, RED_EPSP, s));
        FLoad<D64, 1> ld{(const double *)L.u, (const double *)x, epsp, n1, 0.0};
        JF_DR4(D64, 1, K, ld, (const double *)b, (const double *)L.fu, c->mg_adt, L.fac, (double *)bc, (double *)xc,
               (const double *)dtc, 0);
    } else {
        FLoad<TL32, 2> ld{(const float *)L.u, (const float *)x, n1};
        const int bf = (c->prec == 16 && l + 1 == c->nlev - 1) ? 1 : 0;   // BF16 coarsest level
        JF_DR4(TL32, 2, K, ld, (const float *)b, nullptr, c->mg_adt, L.fac, (float *)bc, (float *)xc,
               (const float *)dtc, bf);
    }
#undef JF_DR4
#undef JF_DR2
#undef JF_DR
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

inline int fv_smooth_or_defect(jfnk_ctx *c, int l, int mode, const void *x, const void *b, void *out,
                               cudaStream_t s, RKS rk = RKS{nullptr, 0, 1.0, 1.0f}) {
    if (c->prec == 64)
        return fv_op64(c, l, mode, (const double *)c->lev[l].u, (const double *)x, (const double *)b,
                       (double *)out, s, rk);
    return fv_op32(c, l, mode, (const float *)x, (const float *)b, (float *)out, s, rk);
}

// more than one stage per pseudo-time step (opts.rk_stages > 1)
inline bool rk_multi(const jfnk_ctx *c) { return c->opts.rk_stages > 1 || c->opts.rk_alpha[0] != 1.0; }

// MG_l(x, b; u) of Sec. 3.4 on level l (0 = finest subgrid).  `zero`: x = 0 on
// entry (products with x are skipped).  `first_done`: the caller already made
// the first pre-smoothing step from zero (x = dtau b, fused into the transfer
// or the restriction).
template <class S>
int mg_cycle_t(jfnk_ctx *c, int l, bool zero, bool first_done, cudaStream_t s) {
    FVLev &L = c->lev[l];
    const size_t n1 = (size_t)L.NX * L.NZ;
    int pre = (l == 0) ? c->fine_pre : c->mid_pre;
    int post = (l == 0) ? c->fine_post : c->mid_post;
    if (first_done) {
        pre -= 1;
        zero = false;
    }
    auto smooth = [&](int steps) -> int {
        const bool rk = rk_multi(c);
        const int ns = c->opts.rk_stages;
        for (int i = 0; i < steps; ++i) {
            if (rk) {
                // stages x_k = x_0 + a_k dtau (b - g'x_{k-1}) through the level's x2 and r
                // buffers (x_0 = L.x is kept until the last stage)
                void *in = L.x, *out = L.x2, *spare = L.r;
                for (int k = 0; k < ns; ++k) {
                    const double a = c->opts.rk_alpha[k];
                    if (zero && k == 0) {
                        jf_launch<k_scale_dtau_b<S>>(k_scale_dtau<S>, nblk(L.n, 256), 256, 0, s, (S *)out, (const S *)L.b,
                                  (const S *)L.dtau, n1, a);
                        jf_launched();
                    } else {
                        JF_RET(fv_smooth_or_defect(c, l, FV_SMOOTH, in, L.b, out, s,
                                                   RKS{zero ? nullptr : L.x, zero ? 2 : 1, a, (float)a}));
                    }
                    void *prev = in;
                    in = out;
                    out = (k == 0) ? spare : prev;   // alternate x2 / r; x_0 stays intact
                }
                // the result is `in`; the other two buffers become x2 and r
                void *bufs[3] = {L.x, L.x2, L.r}, *rest[2];
                int q = 0;
                for (void *bp : bufs)
                    if (bp != in) rest[q++] = bp;
                L.x = in;
                L.x2 = rest[0];
                L.r = rest[1];
                zero = false;
            } else if (zero) {
                jf_launch<k_scale_dtau_b<S>>(k_scale_dtau<S>, nblk(L.n, 256), 256, 0, s, (S *)L.x, (const S *)L.b, (const S *)L.dtau, n1,
                          1.0);
                jf_launched();
                zero = false;
            } else {
                JF_RET(fv_smooth_or_defect(c, l, FV_SMOOTH, L.x, L.b, L.x2, s));
                void *t = L.x;
                L.x = L.x2;
                L.x2 = t;
            }
        }
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    };
    JF_RET(smooth(pre));
    if (l < c->nlev - 1) {
        FVLev &C = c->lev[l + 1];
        const bool fuse = c->mid_pre >= 1 && !rk_multi(c);
        if (zero || c->prec == 64 || (L.fac != 2 && !fv_four_lanes(c, n1))) {
            // FP64, and large levels agglomerated by 3 or 5 (odd k + 1): separate defect
            // and restriction (one thread per fine cell keeps the defect kernel occupied;
            // the fused kernel would run fac^2 cells one after another per coarse cell)
            if (zero) {
                jf_launch<k_neg_b<S>>(k_neg<S>, nblk(L.n, 256), 256, 0, s, (S *)L.r, (const S *)L.b, L.n);
                jf_launched();
            } else {
                JF_RET(fv_smooth_or_defect(c, l, FV_DEFECT, L.x, L.b, L.r, s));
            }
            jf_launch<k_restrict_b_b<S>>(k_restrict_b<S>, nblk(C.n, 256), 256, 0, s, (const S *)L.r, L.NX, L.NZ, L.fac, (S *)C.b,
                                                           fuse ? (S *)C.x : nullptr, (const S *)C.dtau,
                                                           (c->prec == 16 && l + 1 == c->nlev - 1) ? 1 : 0);
            jf_launched();
        } else {
            // defect and restriction (and the coarse first step) in one pass
            JF_RET(fv_defect_restrict(c, l, L.x, L.b, C.b, fuse ? C.x : nullptr, C.dtau, s));
        }
        bool vz = true, fd = fuse;
        for (int cyc = 0; cyc < c->cycles; ++cyc) {
            JF_RET(mg_cycle_t<S>(c, l + 1, vz, fd, s));
            vz = false;
            fd = false;
        }
        if (sizeof(S) == 4 && post >= 1 && !rk_multi(c)) {
            // FP32: the correction x - P v_c is formed inside the first post-smoothing step
            JF_RET(fv_smooth32_corrected(c, l, (const float *)L.x, zero, (const float *)L.b, (float *)L.x2, s));
            void *t = L.x;
            L.x = L.x2;
            L.x2 = t;
            post -= 1;
        } else {
            jf_launch<k_prolong_b<S>>(k_prolong<S>, nblk(L.n, 256), 256, 0, s, (S *)L.x, (const S *)C.x, L.NX, L.NZ, L.fac,
                      zero ? 1 : 0);
            jf_launched();
        }
        zero = false;
    }
    JF_RET(smooth(post));
    if (zero) JF_CK(jf_memset(L.x, 0, L.n * sizeof(S), s));
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

template <class S>
int dg_smooth_step(jfnk_ctx *c, const S *r, S *&z, S *&z2, bool &zero, cudaStream_t s);

template <>
int dg_smooth_step<double>(jfnk_ctx *c, const double *r, double *&z, double *&z2, bool &zero, cudaStream_t s) {
    const int NP = c->np1 * c->np1;
    if (zero) {
        jf_launch<k_scale_dtau_dg_b<double>>(k_scale_dtau_dg<double>, nblk(c->N, 256), 256, 0, s, z, r, c->dtau_dg, c->npt, NP, 1.0); jf_launched();
        zero = false;
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    }
    JF_RET(red_dot(c, z, z, c->N, c->scal + S_EPSDG, RED_EPSP, s));
    DGArgs a = {};
    a.U = c->mg_U;
    a.y = z;
    a.fU = c->fU;
    a.r = r;
    a.eps = c->scal + S_EPSDG;
    a.dtau = c->dtau_dg;
    a.adt = c->mg_adt;
    a.out0 = z2;
    JF_RET(dg_apply(c, DG_SMOOTH64, a, s));
    double *t = z;
    z = z2;
    z2 = t;
    return JFNK_OK;
}

template <>
int dg_smooth_step<float>(jfnk_ctx *c, const float *r, float *&z, float *&z2, bool &zero, cudaStream_t s) {
    const int NP = c->np1 * c->np1;
    if (zero) {
        jf_launch<k_scale_dtau_dg_b<float>>(k_scale_dtau_dg<float>, nblk(c->N, 256), 256, 0, s, z, r, c->dtau_dgf, c->npt, NP, 1.0); jf_launched();
        zero = false;
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    }
    DGArgs a = {};
    a.U = c->mg_U;
    a.Uf = c->Usf;
    a.yf = z;
    a.rf = r;
    a.dtauf = c->dtau_dgf;
    a.adt = c->mg_adt;
    a.out0 = z2;
    JF_RET(dg_apply(c, DG_TLSMOOTH, a, s));
    float *t = z;
    z = z2;
    z2 = t;
    return JFNK_OK;
}

// d = r - G'z
template <class S>
int dg_defect(jfnk_ctx *c, const S *r, const S *z, S *d, cudaStream_t s);

template <>
int dg_defect<double>(jfnk_ctx *c, const double *r, const double *z, double *d, cudaStream_t s) {
    JF_RET(red_dot(c, z, z, c->N, c->scal + S_EPSDG, RED_EPSP, s));
    DGArgs a = {};
    a.U = c->mg_U;
    a.y = z;
    a.fU = c->fU;
    a.eps = c->scal + S_EPSDG;
    a.adt = c->mg_adt;
    a.out0 = c->w2;
    JF_RET(dg_apply(c, DG_JV, a, s));
    jf_launch<k_sub_b<double>>(k_sub<double>, nblk(c->N, 256), 256, 0, s, r, c->w2, d, c->N); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

template <>
int dg_defect<float>(jfnk_ctx *c, const float *r, const float *z, float *d, cudaStream_t s) {
    DGArgs a = {};
    a.U = c->mg_U;
    a.Uf = c->Usf;
    a.yf = z;
    a.rf = r;   // the tangent product's epilogue forms d = r - G'z
    a.adt = c->mg_adt;
    a.out0 = d;
    return dg_apply(c, DG_TLJV, a, s);
}

// FP32: one DG pre-smoothing step from zero (z = dtau_E r) and the defect
// d = r - G'z in one launch; writes z and d
int dg_first_step_defect32(jfnk_ctx *c, const float *r, float *z, float *d, cudaStream_t s,
                           const TransferOut *tro = nullptr) {
    DGArgs a = {};
    a.tro = tro;
    a.U = c->mg_U;
    a.Uf = c->Usf;
    a.rf = r;
    a.dtauf = c->dtau_dgf;
    a.adt = c->mg_adt;
    a.out0 = d;
    a.out1f = z;
    return dg_apply(c, DG_TLJV, a, s);
}

// One multi-stage pseudo-time step on the DG level (opts.rk_stages > 1):
// z_k = z_0 + a_k dtau_E (r - G'z_{k-1}), k = 1..s, from z_0 = z (0 when `zero`).
// Stages alternate between z2 and z3 (z_0 is kept); the last stage writes
// last_out when given.  On return z points at the result and z2, z3 at the two
// free buffers.
template <class S>
int dg_rk_step(jfnk_ctx *c, const S *r, S *&z, S *&z2, S *&z3, bool &zero, cudaStream_t s, S *last_out) {
    const int ns = c->opts.rk_stages, NP = c->np1 * c->np1;
    S *in = z, *out = z2;
    for (int k = 0; k < ns; ++k) {
        if (k == ns - 1 && last_out) out = last_out;
        const double a = c->opts.rk_alpha[k];
        if (zero && k == 0) {
            jf_launch<k_scale_dtau_dg_b<S>>(k_scale_dtau_dg<S>, nblk(c->N, 256), 256, 0, s, out, r,
                      sizeof(S) == 8 ? (const S *)c->dtau_dg : (const S *)c->dtau_dgf, c->npt, NP, a);
            jf_launched();
            JF_CK(cudaGetLastError());
        } else {
            DGArgs A = {};
            A.U = c->mg_U;
            A.adt = c->mg_adt;
            A.out0 = out;
            A.z0 = zero ? nullptr : z;
            A.z0mode = zero ? 2 : 1;
            A.alpha = a;
            if (sizeof(S) == 8) {
                JF_RET(red_dot(c, (const double *)in, (const double *)in, c->N, c->scal + S_EPSDG, RED_EPSP, s));
                A.y = (const double *)in;
                A.fU = c->fU;
                A.r = (const double *)r;
                A.eps = c->scal + S_EPSDG;
                A.dtau = c->dtau_dg;
                JF_RET(dg_apply(c, DG_SMOOTH64, A, s));
            } else {
                A.Uf = c->Usf;
                A.yf = (const float *)in;
                A.rf = (const float *)r;
                A.dtauf = c->dtau_dgf;
                JF_RET(dg_apply(c, DG_TLSMOOTH, A, s));
            }
        }
        S *prev = in;
        in = out;
        out = (k == 0) ? z3 : prev;
    }
    S *bufs[3] = {z, z2, z3}, *rest[2] = {nullptr, nullptr};
    int q = 0;
    for (S *bp : bufs)
        if (bp != in && q < 2) rest[q++] = bp;
    z = in;
    z2 = rest[0];
    z3 = rest[1];
    zero = false;
    return JFNK_OK;
}

template <class S>
int apply_t(jfnk_ctx *c, const S *r, S *zout, cudaStream_t s) {
    // restore the level double-buffer order at the end so that every
    // application issues the same launches on the same pointers
    void *sx[JF_MAXLEV], *sx2[JF_MAXLEV], *sr[JF_MAXLEV];
    for (int l = 0; l < c->nlev; ++l) {
        sx[l] = c->lev[l].x;
        sx2[l] = c->lev[l].x2;
        sr[l] = c->lev[l].r;
    }
    const bool rk = rk_multi(c);
    S *z = (S *)c->pz, *z2 = (S *)c->pz2, *z3 = (S *)c->pr;
    bool zero = true;
    const S *d = r;
    const bool fuse0 = c->fine_pre >= 1 && !rk;
    bool transferred = false;
    if (sizeof(S) == 4 && c->dg_pre == 1 && c->opts.dg_fused != 2 && !rk) {
        // the defect kernel also transfers the defect to the finest FV level (T^mf, and
        // the first FV smoothing step from zero), so no transfer launch follows
        TransferOut tro = {};
        TK K = make_tk(c);
        for (int i = 0; i < 5; ++i) {
            for (int a = 0; a < 5; ++a) tro.V[i][a] = (float)K.tab.V[i][a];
            tro.om[i] = (float)K.tab.om[i];
        }
        tro.massfix = c->opts.massfix && !c->opts.transfer_l2;
        tro.NX = c->lev[0].NX;
        tro.NZ = c->lev[0].NZ;
        tro.b = (float *)c->lev[0].b;
        tro.x0 = fuse0 ? (float *)c->lev[0].x : nullptr;
        tro.dtau0 = (const float *)c->lev[0].dtau;
        JF_RET(dg_first_step_defect32(c, (const float *)r, (float *)z, (float *)c->pd, s, &tro));
        zero = false;
        transferred = true;
    } else {
        for (int i = 0; i < c->dg_pre; ++i) {
            if (rk) JF_RET(dg_rk_step<S>(c, r, z, z2, z3, zero, s, nullptr));
            else JF_RET(dg_smooth_step<S>(c, r, z, z2, zero, s));
        }
        if (!zero) {
            JF_RET(dg_defect<S>(c, r, z, (S *)c->pd, s));
            d = (const S *)c->pd;
        }
    }
    if (!transferred)
        JF_RET(to_fv<S, S>(c, d, (S *)c->lev[0].b, s, fuse0 ? (S *)c->lev[0].x : nullptr, (const S *)c->lev[0].dtau));
    JF_RET(mg_cycle_t<S>(c, 0, true, fuse0, s));
    JF_RET(to_dg<S, S>(c, (const S *)c->lev[0].x, z, zero ? 0 : 1, s));
    zero = false;
    for (int i = 0; i < c->dg_post; ++i) {
        if (rk) {
            JF_RET(dg_rk_step<S>(c, r, z, z2, z3, zero, s, i == c->dg_post - 1 ? zout : nullptr));
            continue;
        }
        if (i == c->dg_post - 1) z2 = zout;   // the last step writes the output itself
        JF_RET(dg_smooth_step<S>(c, r, z, z2, zero, s));
    }
    if (c->dg_post == 0) JF_CK(jf_memcpy(zout, z, c->N * sizeof(S), cudaMemcpyDeviceToDevice, s));
    for (int l = 0; l < c->nlev; ++l) {
        c->lev[l].x = sx[l];
        c->lev[l].x2 = sx2[l];
        c->lev[l].r = sr[l];
    }
    return JFNK_OK;
}

}  // namespace

// ---- entry points used by the API and the solver ---------------------------
int fv_setup_background(jfnk_ctx *c, cudaStream_t s) {
    for (int l = 0; l < c->nlev; ++l) {
        FVK K = make_fvk(c, l);
        const int n = 2 * c->lev[l].NZ + 1;
        k_bg_fv<<<(n + 127) / 128, 128, 0, s>>>(K, c->lev[l].hbx, c->lev[l].hbxw, c->lev[l].hbz); jf_launched();
        JF_CK(cudaGetLastError());
    }
    return JFNK_OK;
}

int mg_linearize(jfnk_ctx *c, const double *Uin, double adt, cudaStream_t s) {
    // every pointer the captured graph holds is context-owned
    JF_CK(jf_memcpy(c->Ulin, Uin, 8 * c->N, cudaMemcpyDeviceToDevice, s));
    const double *U = c->Ulin;
    c->mg_adt = adt;
    c->mg_U = U;
    // DG pseudo-time steps: FP64 for the FP64 preconditioner, FP32 from the FP32
    // copy of the state otherwise (a step-size heuristic; one warp per element)
    const unsigned gd = (unsigned)(((size_t)c->n_el * 32 + 127) / 128);
    if (c->prec == 64) {
        jf_launch<k_dg_dtau_b<double>>(k_dg_dtau<double>, gd, 128, 0, s, U, (const double *)c->ubv, c->grid.nx, c->grid.nz, c->np1,
                  c->pc, c->powtab, 1.0 / c->hx, 1.0 / c->hz, c->phys.mu, adt, c->opts.sigma_dg, c->dtau_dg,
                  c->dtau_dgf);
        jf_launched();
        JF_CK(cudaGetLastError());
        JF_RET(to_fv<double, double>(c, U, (double *)c->lev[0].u, s));
    } else {
        JF_RET(blas_copy_d2f(U, c->Usf, c->N, s));
        jf_launch<k_dg_dtau_b<float>>(k_dg_dtau<float>, gd, 128, 0, s, (const float *)c->Usf, (const float *)c->ubvf, c->grid.nx,
                  c->grid.nz, c->np1, c->pc, c->powtab, 1.0 / c->hx, 1.0 / c->hz, c->phys.mu, adt,
                  c->opts.sigma_dg, c->dtau_dg, c->dtau_dgf);
        jf_launched();
        JF_CK(cudaGetLastError());
        JF_RET(to_fv<double, float>(c, U, (float *)c->lev[0].u, s));
    }
    for (int l = 0; l < c->nlev; ++l) {
        FVLev &L = c->lev[l];
        FVK K = make_fvk(c, l);
        const size_t n1 = (size_t)L.NX * L.NZ;
        if (l > 0) {
            FVLev &F = c->lev[l - 1];
            if (c->prec == 64)
                jf_launch<k_restrict_body<double>>(k_restrict<double>, nblk(L.n, 256), 256, 0, s, (const double *)F.u, F.NX, F.NZ, F.fac, (double *)L.u);
            else
                jf_launch<k_restrict_b_b<float>>(k_restrict_b<float>, nblk(L.n, 256), 256, 0, s, (const float *)F.u, F.NX, F.NZ, F.fac, (float *)L.u,
                                                                   nullptr, nullptr,
                                                                   (c->prec == 16 && l == c->nlev - 1) ? 1 : 0);
            jf_launched();
        }
        if (c->prec == 64) {
            JF_RET(fv_op64(c, l, FV_RES, (const double *)L.u, nullptr, nullptr, (double *)L.fu, s));
            jf_launch<k_fv_dtau_b<double>>(k_fv_dtau<double>, nblk(n1), 128, 0, s, K, (const double *)L.u, adt, c->opts.sigma_fv, (double *)L.dtau); jf_launched();
        } else {
            jf_launch<k_fv_dtau_b<float>>(k_fv_dtau<float>, nblk(n1), 128, 0, s, K, (const float *)L.u, adt, c->opts.sigma_fv, (float *)L.dtau); jf_launched();
        }
        JF_CK(cudaGetLastError());
    }
    return JFNK_OK;
}

namespace {
int apply_body(jfnk_ctx *c, cudaStream_t s) {
    if (c->prec == 64) return apply_t<double>(c, (const double *)c->pin, (double *)c->pout, s);
    return apply_t<float>(c, (const float *)c->pin, (float *)c->pout, s);
}

// Capture one application into an executable graph.  Returns JFNK_OK with
// mg_graph_valid = 0 when capture is not possible (the caller then launches
// the kernels directly).
int capture(jfnk_ctx *c) {
    if (c->mg_graph_valid) {
        cudaGraphExecDestroy(c->mg_graph);
        c->mg_graph_valid = 0;
    }
    std::lock_guard<std::mutex> lock(g_jf_device_mu);   // no device-wide sync during capture
    if (!c->cap_stream) JF_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    const unsigned long long n0 = t_jf_launches;
    const long long d0 = c->dg_calls, f0 = c->fv_calls;
    JF_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int rc = apply_body(c, c->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    c->graph_launches = t_jf_launches - n0;
    __atomic_fetch_sub(&g_jf_launches, c->graph_launches, __ATOMIC_RELAXED);   // captured, not launched
    t_jf_launches = n0;
    c->graph_dg_calls = c->dg_calls - d0;
    c->graph_fv_calls = c->fv_calls - f0;
    c->dg_calls = d0;
    c->fv_calls = f0;
    if (rc != JFNK_OK || e != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc != JFNK_OK ? rc : JFNK_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->mg_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        return JFNK_ECUDA;
    }
    c->mg_graph_valid = 1;
    c->mg_graph_adt = c->mg_adt;
    c->mg_graph_gen++;
    return JFNK_OK;
}
}  // namespace

// Drop every captured graph (launch shapes or buffers changed).
void jf_invalidate_graphs(jfnk_ctx *c) {
    if (c->mg_graph_valid) {
        cudaGraphExecDestroy(c->mg_graph);
        c->mg_graph_valid = 0;
    }
    for (int i = 0; i < 64; ++i)
        if (c->arn_valid[i]) {
            cudaGraphExecDestroy(c->arn_graph[i]);
            c->arn_valid[i] = 0;
        }
}

int mg_apply(jfnk_ctx *c, const double *r, void *z, cudaStream_t s, const float *r32) {
    const size_t sS = c->prec == 64 ? 8 : 4;
    if (c->prec != 64 && r32 && (c->capturing || !c->opts.use_graphs || t_jf_rec)) {
        // inside an Arnoldi step: the FP32 copy of r exists already, and the
        // launches go straight into the caller's stream (or capture)
        return apply_t<float>(c, r32, (float *)z, s);
    }
    if (c->prec == 64) JF_CK(jf_memcpy(c->pin, r, 8 * c->N, cudaMemcpyDeviceToDevice, s));
    else JF_RET(blas_copy_d2f(r, (float *)c->pin, c->N, s));   // FP32 preconditioner: r enters in FP32
    if (c->opts.use_graphs && !c->capturing && !t_jf_rec) {
        if (!c->mg_graph_valid || c->mg_graph_adt != c->mg_adt) JF_RET(capture(c));
        JF_CK(cudaGraphLaunch(c->mg_graph, s));
        jf_launched((unsigned)c->graph_launches);
        c->dg_calls += c->graph_dg_calls;
        c->fv_calls += c->graph_fv_calls;
    } else {
        JF_RET(apply_body(c, s));
    }
    JF_CK(jf_memcpy(z, c->pout, sS * c->N, cudaMemcpyDeviceToDevice, s));
    return JFNK_OK;
}

// Diagnostic timing of the finest FV level's two FP32 kernels at the
// linearisation U (alpha dt = 1): one pseudo-time smoothing step and the defect
// fused with the restriction, x = b = (float) y.  ms[0], ms[1]: mean durations
// over reps (CUDA events on s).  Overwrites the preconditioner's level vectors.
int mg_time_fv_level0(jfnk_ctx *c, const double *U, const double *y, int reps, double *ms, cudaStream_t s) {
    if (c->prec == 64 || !c->mg_on || c->nlev < 2) return JFNK_EINVAL;
    JF_RET(mg_linearize(c, U, 1.0, s));
    FVLev &L = c->lev[0];
    FVLev &C = c->lev[1];
    if (L.n != c->N) return JFNK_EINVAL;
    JF_RET(blas_copy_d2f(y, (float *)L.x, L.n, s));
    JF_RET(blas_copy_d2f(y, (float *)L.b, L.n, s));
    cudaEvent_t e[3];
    for (auto &x : e) JF_CK(cudaEventCreate(&x));
    double t0 = 0.0, t1 = 0.0;
    int rc = JFNK_OK;
    for (int r = 0; r < reps && rc == JFNK_OK; ++r) {
        cudaEventRecord(e[0], s);
        rc = fv_op32(c, 0, FV_SMOOTH, (const float *)L.x, (const float *)L.b, (float *)L.x2, s);
        cudaEventRecord(e[1], s);
        if (rc == JFNK_OK) rc = fv_defect_restrict(c, 0, L.x, L.b, C.b, C.x, C.dtau, s);
        cudaEventRecord(e[2], s);
        if (cudaEventSynchronize(e[2]) != cudaSuccess) rc = JFNK_ECUDA;
        float m0 = 0.f, m1 = 0.f;
        cudaEventElapsedTime(&m0, e[0], e[1]);
        cudaEventElapsedTime(&m1, e[1], e[2]);
        t0 += m0;
        t1 += m1;
    }
    for (auto &x : e) cudaEventDestroy(x);
    ms[0] = t0 / reps;
    ms[1] = t1 / reps;
    return rc;
}

int fv_rhs64(jfnk_ctx *c, int l, const double *u, double *f, cudaStream_t s) {
    return fv_op64(c, l, FV_RES, u, nullptr, nullptr, f, s);
}

int transfer_to_fv64(jfnk_ctx *c, const double *u, double *v, cudaStream_t s) {
    return to_fv<double, double>(c, u, v, s);
}

int transfer_to_dg64(jfnk_ctx *c, const double *v, double *u, int accumulate, cudaStream_t s) {
    return to_dg<double, double>(c, v, u, accumulate, s);
}
