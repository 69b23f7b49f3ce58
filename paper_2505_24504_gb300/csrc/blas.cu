// Reductions and vector updates of the Krylov solver (Sec. 3.1).
//
// Dots and norms: pass 1 reduces a grid-strided slice per block (warp
// shuffles, then shared memory) into per-block partials; pass 2, one block,
// adds the partials in a fixed order.  The result never depends on timing, so
// a member computes the same bits alone or inside a batch.  Results stay on
// the device: the norm feeds eps = sqrt(eps_mach)/|y| of the next FD product
// without a host round trip.
// Multi-dot (classical Gram-Schmidt): one pass over w reads w once for all
// basis vectors, h_i = V_i . w for i < nv.
#include "internal.h"

namespace {

constexpr int RB = 256;          // threads per reduction block
constexpr int MAXV = 32;         // basis vectors per multi-dot pass

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sw[RB / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sw[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < RB / 32 ? sw[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;   // valid in thread 0
}

template <class S>
__global__ void __launch_bounds__(RB) k_dot_partial(const S *x, const S *y, size_t n, double *part) {
    double acc = 0.0, acc2 = 0.0;
    const size_t stride = (size_t)gridDim.x * RB;
    size_t i = (size_t)blockIdx.x * RB + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {   // two loads in flight per thread
        const double a0 = (double)x[i], b0 = (double)y[i];
        const double a1 = (double)x[i + stride], b1 = (double)y[i + stride];
        acc = fma(a0, b0, acc);
        acc2 = fma(a1, b1, acc2);
    }
    if (i < n) acc = fma((double)x[i], (double)y[i], acc);
    acc = block_sum(acc + acc2);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// op: RED_SUM -> sum; RED_SQRT -> sqrt(sum); RED_EPS -> sqrt(2^-52)/sqrt(sum) (0 if sum == 0);
// RED_EPS32 -> sqrt(2^-23)/sqrt(sum)
__global__ void __launch_bounds__(RB) k_final(const double *part, int nb, double *out, int op) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RB) acc += part[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
        double r = acc;
        if (op == RED_SQRT) r = sqrt(acc);
        if (op == RED_EPS) r = acc > 0.0 ? 1.4901161193847656e-08 / sqrt(acc) : 0.0;
        if (op == RED_EPS32) r = acc > 0.0 ? 3.4526698300124393e-04 / sqrt(acc) : 0.0;
        *out = r;
    }
}

// h_j partials for NV basis vectors at once: accumulators are compile-time
// indexed (registers), warp sums go through one shared-memory pass.
template <int NV>
__global__ void __launch_bounds__(RB) k_mdot_partial(const double *V, size_t ldv, const double *w, size_t n,
                                                     double *part, const double *flag) {
    if (flag && *flag == 0.0) {   // pass not needed: contribute zeros
        if (threadIdx.x < NV) part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    double acc[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) acc[j] = 0.0;
    const size_t stride = (size_t)gridDim.x * RB;
    size_t i = (size_t)blockIdx.x * RB + threadIdx.x;
    for (; i + stride < n; i += 2 * stride) {   // two elements' loads in flight
        const double w0 = w[i], w1 = w[i + stride];
        double v0[NV], v1[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            v0[j] = V[(size_t)j * ldv + i];
            v1[j] = V[(size_t)j * ldv + i + stride];
        }
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = fma(v1[j], w1, fma(v0[j], w0, acc[j]));
    }
    if (i < n) {
        const double w0 = w[i];
#pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = fma(V[(size_t)j * ldv + i], w0, acc[j]);
    }
    __shared__ double sw[NV][RB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const double v = warp_sum(acc[j]);
        if (lane == 0) sw[j][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < RB / 32; ++q) r += sw[threadIdx.x][q];
        part[(size_t)threadIdx.x * gridDim.x + blockIdx.x] = r;
    }
}

__global__ void __launch_bounds__(RB) k_mfinal(const double *part, int nb, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RB) acc += part[(size_t)blockIdx.x * nb + i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// w += sign * sum_j h_j V_j
__global__ void k_mupdate(const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                          double sign, const double *flag) {
    if (flag && *flag == 0.0) return;
    __shared__ double sh[MAXV];
    if (threadIdx.x < nv) sh[threadIdx.x] = sign * h[threadIdx.x];
    __syncthreads();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = w[i];
        for (int j = 0; j < nv; ++j) acc = fma(sh[j], V[(size_t)j * ldv + i], acc);
        w[i] = acc;
    }
}

__global__ void k_scale_copy(const double *w, const double *nrm, double *v, size_t n) {
    const double s = *nrm;
    const double inv = s != 0.0 ? 1.0 / s : 0.0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] = w[i] * inv;
}

__global__ void k_axpby(double a, const double *x, double b, const double *y, double *z, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        z[i] = a * x[i] + (y ? b * y[i] : 0.0);
}

// w += sign * sum_j h_j V_j and per-block partial sums of the updated w^2
// (about 8 elements per thread, like the dot kernels)
template <int NVMAX>
__global__ void __launch_bounds__(RB) k_mupdate_norm(const double *V, int nv, size_t ldv, const double *h,
                                                     double *w, size_t n, double sign, const double *flag,
                                                     double *part) {
    if (flag && *flag == 0.0) return;
    __shared__ double sh[NVMAX];
    if (threadIdx.x < nv) sh[threadIdx.x] = sign * h[threadIdx.x];
    __syncthreads();
    double acc2 = 0.0;
    const size_t stride = (size_t)gridDim.x * RB;
    for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
        double a = w[i];
        for (int j = 0; j < nv; ++j) a = fma(sh[j], V[(size_t)j * ldv + i], a);
        w[i] = a;
        acc2 = fma(a, a, acc2);
    }
    acc2 = block_sum(acc2);
    if (threadIdx.x == 0) part[blockIdx.x] = acc2;
}

// After the first pass: w1sq = sum of partials, nrm = sqrt(w1sq) and the
// reorthogonalisation flag (|w1| < |w0|/sqrt(2), |w0|^2 = |w1|^2 + |h|^2).
// After the second pass (flag given): nrm = sqrt(sum) only if that pass ran.
__global__ void __launch_bounds__(RB) k_final_gs(const double *part, int nb, const double *h, int nv,
                                                 const double *flag_in, double *w1sq, double *nrm,
                                                 double *flag_out) {
    if (flag_in && *flag_in == 0.0) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RB) acc += part[i];
    acc = block_sum(acc);
    __shared__ double tot;
    if (threadIdx.x == 0) tot = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double hh = 0.0;
        if (!flag_in)
            for (int i = threadIdx.x; i < nv; i += 32) hh += h[i] * h[i];
        hh = warp_sum(hh);
        if (threadIdx.x == 0) {
            *nrm = sqrt(tot);
            if (!flag_in) {
                *w1sq = tot;
                *flag_out = (tot < 0.5 * (tot + hh)) ? 1.0 : 0.0;
            }
        }
    }
}

// y = (double) x and per-block partial sums of x^2 (for eps of the FD product)
__global__ void __launch_bounds__(RB) k_f2d_norm(const float *x, double *y, size_t n, double *part) {
    double acc = 0.0;
    const size_t stride = (size_t)gridDim.x * RB;
    for (size_t i = (size_t)blockIdx.x * RB + threadIdx.x; i < n; i += stride) {
        const double v = (double)x[i];
        y[i] = v;
        acc = fma(v, v, acc);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

struct YV {
    double y[MAXV];
};

template <class S>
__global__ void k_zcomb(const S *Z, int nz, size_t n, YV yv, double *x) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double acc = x[i];
        for (int j = 0; j < nz; ++j) acc = fma(yv.y[j], (double)Z[(size_t)j * n + i], acc);
        x[i] = acc;
    }
}

__global__ void k_d2f(const double *x, float *y, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (float)x[i];
}
__global__ void k_f2d(const float *x, double *y, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (double)x[i];
}

inline unsigned grid_for(size_t n) {
    size_t g = (n + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// ~8 elements per thread: the FP64 shuffle tree (5 adds per value reduced)
// stays small next to the per-element FMAs
inline int nblocks_red(jfnk_ctx *c, size_t n) {
    size_t g = (n + (size_t)RB * 8 - 1) / ((size_t)RB * 8);
    if (g > (size_t)c->nb_red) g = c->nb_red;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

int red_dot(jfnk_ctx *c, const double *x, const double *y, size_t n, double *out, int op, cudaStream_t s) {
    const int nb = nblocks_red(c, n);
    k_dot_partial<double><<<nb, RB, 0, s>>>(x, y, n, c->partial); jf_launched();
    k_final<<<1, RB, 0, s>>>(c->partial, nb, out, op); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int red_dotf(jfnk_ctx *c, const float *x, const float *y, size_t n, double *out, int op, cudaStream_t s) {
    const int nb = nblocks_red(c, n);
    k_dot_partial<float><<<nb, RB, 0, s>>>(x, y, n, c->partial); jf_launched();
    k_final<<<1, RB, 0, s>>>(c->partial, nb, out, op); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

template <int NV>
void mdot_chunk(const double *V, size_t ldv, const double *w, size_t n, double *part, int nb, cudaStream_t s,
                const double *flag) {
    k_mdot_partial<NV><<<nb, RB, 0, s>>>(V, ldv, w, n, part, flag);
}

int blas_mdot(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *w, size_t n, double *h,
              cudaStream_t s, const double *flag) {
    constexpr int CH = 16;   // basis vectors per pass over w
    for (int j0 = 0; j0 < nv; j0 += CH) {
        const int m = nv - j0 < CH ? nv - j0 : CH;
        const int nb = nblocks_red(c, n);
        const double *Vj = V + (size_t)j0 * ldv;
        switch (m) {
            case 1: mdot_chunk<1>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 2: mdot_chunk<2>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 3: mdot_chunk<3>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 4: mdot_chunk<4>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 5: mdot_chunk<5>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 6: mdot_chunk<6>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 7: mdot_chunk<7>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 8: mdot_chunk<8>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 9: mdot_chunk<9>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 10: mdot_chunk<10>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 11: mdot_chunk<11>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 12: mdot_chunk<12>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 13: mdot_chunk<13>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 14: mdot_chunk<14>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            case 15: mdot_chunk<15>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
            default: mdot_chunk<16>(Vj, ldv, w, n, c->partial, nb, s, flag); break;
        }
        jf_launched();
        k_mfinal<<<m, RB, 0, s>>>(c->partial, nb, h + j0); jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_mupdate(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                 double sign, cudaStream_t s, const double *flag) {
    (void)c;
    for (int j0 = 0; j0 < nv; j0 += MAXV) {
        const int m = nv - j0 < MAXV ? nv - j0 : MAXV;
        k_mupdate<<<grid_for(n), 256, 0, s>>>(V + (size_t)j0 * ldv, m, ldv, h + j0, w, n, sign, flag); jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_scale_copy(const double *w, const double *nrm, double *v, size_t n, cudaStream_t s) {
    k_scale_copy<<<grid_for(n), 256, 0, s>>>(w, nrm, v, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_axpby(double a, const double *x, double b, const double *y, double *z, size_t n, cudaStream_t s) {
    k_axpby<<<grid_for(n), 256, 0, s>>>(a, x, b, y, z, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_scale(double a, const double *x, double *y, size_t n, cudaStream_t s) {
    return blas_axpby(a, x, 0.0, nullptr, y, n, s);
}

int blas_zcomb(const void *Z, int prec32, int nzv, size_t n, const double *yv, double *x, cudaStream_t s) {
    for (int j0 = 0; j0 < nzv; j0 += MAXV) {
        const int m = nzv - j0 < MAXV ? nzv - j0 : MAXV;
        YV y;
        for (int j = 0; j < m; ++j) y.y[j] = yv[j0 + j];
        if (prec32)
            k_zcomb<float><<<grid_for(n), 256, 0, s>>>((const float *)Z + (size_t)j0 * n, m, n, y, x);
        else
            k_zcomb<double><<<grid_for(n), 256, 0, s>>>((const double *)Z + (size_t)j0 * n, m, n, y, x);
        jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// Second Gram-Schmidt pass needed?  With w1 = w0 - V h the first pass left
// |w1|^2 of |w0|^2 = |w1|^2 + |h|^2; reorthogonalise when |w1| < |w0| / sqrt(2)
// ("twice is enough").  flag = 1.0 or 0.0, decided on the device.
__global__ void k_reortho_flag(const double *w1sq, const double *h, int nv, double *flag) {
    double hh = 0.0;
    for (int i = threadIdx.x; i < nv; i += 32) hh += h[i] * h[i];
    hh = warp_sum(hh);
    if (threadIdx.x == 0) *flag = (*w1sq < 0.5 * (*w1sq + hh)) ? 1.0 : 0.0;
}

int blas_reortho_flag(const double *w1sq, const double *h, int nv, double *flag, cudaStream_t s) {
    k_reortho_flag<<<1, 32, 0, s>>>(w1sq, h, nv, flag);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_mupdate_norm(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                      double sign, const double *flag_in, double *w1sq, double *nrm, double *flag_out,
                      cudaStream_t s) {
    if (nv > MAXV) {   // long bases: plain updates, then the norm pass
        JF_RET(blas_mupdate(c, V, nv, ldv, h, w, n, sign, s, flag_in));
        const int nb = nblocks_red(c, n);
        k_dot_partial<double><<<nb, RB, 0, s>>>(w, w, n, c->partial);
        jf_launched();
        k_final_gs<<<1, RB, 0, s>>>(c->partial, nb, h, nv, flag_in, w1sq, nrm, flag_out);
        jf_launched();
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    }
    const int nb = nblocks_red(c, n);
    k_mupdate_norm<MAXV><<<nb, RB, 0, s>>>(V, nv, ldv, h, w, n, sign, flag_in, c->partial);
    jf_launched();
    k_final_gs<<<1, RB, 0, s>>>(c->partial, nb, h, nv, flag_in, w1sq, nrm, flag_out);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_f2d_eps(jfnk_ctx *c, const float *x, double *y, size_t n, double *eps_out, cudaStream_t s) {
    const int nb = nblocks_red(c, n);
    k_f2d_norm<<<nb, RB, 0, s>>>(x, y, n, c->partial);
    jf_launched();
    k_final<<<1, RB, 0, s>>>(c->partial, nb, eps_out, RED_EPS);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_copy_d2f(const double *x, float *y, size_t n, cudaStream_t s) {
    k_d2f<<<grid_for(n), 256, 0, s>>>(x, y, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_copy_f2d(const float *x, double *y, size_t n, cudaStream_t s) {
    k_f2d<<<grid_for(n), 256, 0, s>>>(x, y, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}
