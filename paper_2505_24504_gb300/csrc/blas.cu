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
// Single-launch reductions: each block writes its partials, then takes a ticket
// from a per-context counter; the block that arrives last adds all partials in
// block order (so the bits do not depend on which block that is), writes the
// result and resets the counter.  Nothing waits on another block.
// Gram-Schmidt twice (CGS2) in three passes over the basis: h1 = V^T w; then
// w1 = w - V h1 fused with h2 = V^T w1 and |w1|^2 (so |w2|^2 = |w1|^2 - |h2|^2);
// then, when the device-side test asks for it, w2 = w1 - V h2, fused with the
// normalisation.
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

// true in the block that arrives last at the ticket (after its partials are
// visible).  Partials are written by threads of the first warp only, so only
// that warp fences.
__device__ __forceinline__ bool last_block(unsigned *ticket, unsigned nblk) {
    __shared__ bool last;
    if (threadIdx.x < 32) __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == nblk - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// fixed-order sum of part[0..nb) by one block (valid in thread 0)
__device__ __forceinline__ double sum_partials(const double *part, int nb) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += RB) acc += __ldcg(part + i);
    return block_sum(acc);
}

// cnum: numerator of the eps ops (sqrt(2^-52) for RED_EPS, sqrt(2^-23) for
// RED_EPS32, the preconditioner's choice for RED_EPSP)
__device__ __forceinline__ double finish_op(double acc, int op, double cnum = 1.4901161193847656e-08) {
    if (op == RED_SQRT) return sqrt(acc);
    if (op == RED_EPS || op == RED_EPS32 || op == RED_EPSP) return acc > 0.0 ? cnum / sqrt(acc) : 0.0;
    return acc;
}

// x . y (op applied) in one launch
template <class S>
struct k_dot1_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> x,
                                               JfArg<const S *> y, JfArg<size_t> n, JfArg<double *> part,
                                               JfArg<unsigned *> ticket, JfArg<double *> out, JfArg<int> op,
                                               JfArg<double> cnum) {
        jf_pdl_enter();
        double acc = 0.0, acc2 = 0.0;
        const size_t stride = (size_t)jf_nblk * RB;
        size_t i = (size_t)jf_bid * RB + threadIdx.x;
        for (; i + stride < n; i += 2 * stride) {
            const double a0 = (double)x[i], b0 = (double)y[i];
            const double a1 = (double)x[i + stride], b1 = (double)y[i + stride];
            acc = fma(a0, b0, acc);
            acc2 = fma(a1, b1, acc2);
        }
        if (i < n) acc = fma((double)x[i], (double)y[i], acc);
        acc = block_sum(acc + acc2);
        if (threadIdx.x == 0) part[jf_bid] = acc;
        if (!last_block(ticket, jf_nblk)) return;
        const double t = sum_partials(part, jf_nblk);
        if (threadIdx.x == 0) {
            *out = finish_op(t, op, cnum);
            *ticket = 0u;
        }
    }
};
template <class S>
__global__ void __launch_bounds__(RB) k_dot1(const S *x, const S *y, size_t n, double *part, unsigned *ticket,
                                             double *out, int op, double cnum) {
    k_dot1_b<S>::run(blockIdx.x, gridDim.x, x, y, n, part, ticket, out, op, cnum);
}

// ---- CGS2 passes (NV basis vectors, two elements per thread and step) -------
template <int NV>
__device__ __forceinline__ double warp_sum_scatter(const double (&a)[NV], int lane);

// h[j] = sum over blocks of part[j * nb + b] by the whole block, fixed order:
// thread t sums the partials b = t mod RB of every vector (all loads of a round
// issued together), then one warp-and-block reduction of the NV sums.
template <int NV>
__device__ __forceinline__ void finish_multi(const double *part, int nb, double *h) {
    constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
    __shared__ double fw[NV][RB / 32];
    double a[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) a[j] = 0.0;
    for (int b = threadIdx.x; b < nb; b += RB) {
        double v[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldcg(part + (size_t)j * nb + b);
#pragma unroll
        for (int j = 0; j < NV; ++j) a[j] += v[j];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double w = warp_sum_scatter<NV>(a, lane);
    const int j = lane / (32 / P);
    if (lane % (32 / P) == 0 && j < NV) fw[j][wid] = w;
    __syncthreads();
    if (threadIdx.x < NV) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < RB / 32; ++q) r += fw[threadIdx.x][q];
        h[threadIdx.x] = r;
    }
}

// Warp sums of NV per-lane values at about one FP64 add per value and lane:
// each butterfly round over lane bit b keeps half of the remaining vectors
// (lanes with bit b set keep the upper half) and adds the partner's copies, so
// after log2(P) rounds lane L holds vector L >> (5 - log2 P) summed over its
// group; the remaining rounds finish the sum within the group.  P = NV rounded
// up to a power of two (at most 32); returns the value of that vector.
template <int NV>
__device__ __forceinline__ double warp_sum_scatter(const double (&a)[NV], int lane) {
    constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
    constexpr int LP = P == 1 ? 0 : P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
    double v[P];
#pragma unroll
    for (int k = 0; k < P; ++k) v[k] = k < NV ? a[k] : 0.0;
#pragma unroll
    for (int r = 0; r < LP; ++r) {
        const int half = P >> (r + 1);
        const int bit = 4 - r;
        const bool hi = (lane >> bit) & 1;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const double keep = hi ? v[k + half] : v[k];
            const double send = hi ? v[k] : v[k + half];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
        }
    }
    double s = v[0];
#pragma unroll
    for (int bit = 4 - LP; bit >= 0; --bit) s += __shfl_xor_sync(0xffffffffu, s, 1 << bit);
    return s;
}

// block sums of NV accumulators into part[j * nblk + bid]
template <int NV>
__device__ __forceinline__ void store_multi(const double (&acc)[NV], double *part, unsigned bid, unsigned nblk) {
    constexpr int P = NV <= 1 ? 1 : NV <= 2 ? 2 : NV <= 4 ? 4 : NV <= 8 ? 8 : NV <= 16 ? 16 : 32;
    __shared__ double sw[NV][RB / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double v = warp_sum_scatter<NV>(acc, lane);
    const int j = lane / (32 / P);
    if (lane % (32 / P) == 0 && j < NV) sw[j][wid] = v;
    __syncthreads();
    if (threadIdx.x < NV) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < RB / 32; ++q) r += sw[threadIdx.x][q];
        part[(size_t)threadIdx.x * nblk + bid] = r;
    }
}

// pass 1: h = V^T w
template <int NV>
struct k_gs_dot_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<size_t> ldv, JfArg<const double *> w, JfArg<size_t> n2,
                                               JfArg<double *> part, JfArg<unsigned *> ticket, JfArg<double *> h) {
        jf_pdl_enter();
        const double2 *w2 = reinterpret_cast<const double2 *>(w);
        const double2 *Vp[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) Vp[j] = reinterpret_cast<const double2 *>(V + (size_t)j * ldv);
        double acc[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = 0.0;
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n2; i += (size_t)jf_nblk * RB) {
            const double2 a = w2[i];
            double2 v[NV];
    #pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = Vp[j][i];
    #pragma unroll
            for (int j = 0; j < NV; ++j) acc[j] = fma(v[j].y, a.y, fma(v[j].x, a.x, acc[j]));
        }
        store_multi<NV>(acc, part, jf_bid, jf_nblk);
        if (!last_block(ticket, jf_nblk)) return;
        finish_multi<NV>(part, jf_nblk, h);
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
};
template <int NV>
__global__ void __launch_bounds__(RB) k_gs_dot(const double *V, size_t ldv, const double *w, size_t n2,
                                               double *part, unsigned *ticket, double *h) {
    k_gs_dot_b<NV>::run(blockIdx.x, gridDim.x, V, ldv, w, n2, part, ticket, h);
}

// pass 2: w <- w - V h1, h2 = V^T w, w1sq = |w|^2, flag = (|w1| < |w0|/sqrt(2)),
// nrm = |w| (final unless the third pass runs)
template <int NV>
struct k_gs_update_dot_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<size_t> ldv, JfArg<double *> w, JfArg<size_t> n2,
                                               JfArg<const double *> h1, JfArg<double *> part,
                                               JfArg<unsigned *> ticket, JfArg<double *> h2, JfArg<double *> w1sq,
                                               JfArg<double *> nrm, JfArg<double *> flag) {
        jf_pdl_enter();
        double2 *wv = reinterpret_cast<double2 *>(w);
        const double2 *Vp[NV];
        double c[NV], acc[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) {
            Vp[j] = reinterpret_cast<const double2 *>(V + (size_t)j * ldv);
            c[j] = -h1[j];
            acc[j] = 0.0;
        }
        double sq = 0.0;
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n2; i += (size_t)jf_nblk * RB) {
            double2 a = wv[i];
            double2 v[NV];
    #pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = Vp[j][i];
    #pragma unroll
            for (int j = 0; j < NV; ++j) {
                a.x = fma(c[j], v[j].x, a.x);
                a.y = fma(c[j], v[j].y, a.y);
            }
            wv[i] = a;
            sq = fma(a.y, a.y, fma(a.x, a.x, sq));
    #pragma unroll
            for (int j = 0; j < NV; ++j) acc[j] = fma(v[j].y, a.y, fma(v[j].x, a.x, acc[j]));
        }
        store_multi<NV>(acc, part, jf_bid, jf_nblk);
        const double bs = block_sum(sq);
        if (threadIdx.x == 0) part[(size_t)NV * jf_nblk + jf_bid] = bs;
        if (!last_block(ticket, jf_nblk)) return;
        finish_multi<NV>(part, jf_nblk, h2);
        const double tot = sum_partials(part + (size_t)NV * jf_nblk, jf_nblk);
        if (threadIdx.x == 0) {
            double hh = 0.0, hh2 = 0.0;
            for (int j = 0; j < NV; ++j) {
                hh += h1[j] * h1[j];
                hh2 += h2[j] * h2[j];
            }
            *w1sq = tot;
            const bool second = tot < 0.5 * (tot + hh);
            // |w2|^2 = |w1|^2 - |h2|^2 for w2 = w1 - V h2 with V orthonormal and h2 = V^T w1;
            // after the first pass h2 is tiny against |w1|, so the difference does not cancel
            const double nr = sqrt(second ? fmax(tot - hh2, 0.0) : tot);
            nrm[0] = nr;
            nrm[S_INV - S_NORM] = nr != 0.0 ? 1.0 / nr : 0.0;
            *flag = second ? 1.0 : 0.0;
            *ticket = 0u;
        }
    }
};
template <int NV>
__global__ void __launch_bounds__(RB) k_gs_update_dot(const double *V, size_t ldv, double *w, size_t n2,
                                                      const double *h1, double *part, unsigned *ticket,
                                                      double *h2, double *w1sq, double *nrm, double *flag) {
    k_gs_update_dot_b<NV>::run(blockIdx.x, gridDim.x, V, ldv, w, n2, h1, part, ticket, h2, w1sq, nrm, flag);
}

// double -> float by truncation of the fraction on the integer pipe (error below
// one float ulp; enough for the first Gram-Schmidt pass and the preconditioner's
// input): binary32 exponent = binary64 exponent - 896, fraction = the top 23 of
// the 52 bits (IEEE 754 formats).  Magnitudes below the normal float range give
// a signed zero, larger ones (and NaN) use the conversion instruction.
// Rare inputs take an out-of-line conversion: inline, the compiler would turn the
// branch into a select and run the FP64-pipe conversion for every element.
__device__ __noinline__ float d2f_slow(double d) { return (float)d; }
__device__ __noinline__ double f2d_slow(float f) { return (double)f; }

__device__ __forceinline__ float d2f_trunc(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const unsigned sign = (unsigned)((b >> 32) & 0x80000000u);
    if (e > 127) return d2f_slow(d);   // overflow, infinity, NaN
    // below the normal float range (zero included): signed zero
    const unsigned r = e < -126 ? sign : sign | ((unsigned)(e + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
    return __uint_as_float(r);
}

// pass 3 and the normalisation in one sweep, without a reduction (|w2| comes from
// pass 2): v = (w - V h2) / |w2| when the second pass is needed, v = w / |w| else;
// also the float copy of v for later first passes (w32 may be null)
template <int NV>
struct k_gs_update_scale_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<size_t> ldv, JfArg<double *> w, JfArg<float *> w32,
                                               JfArg<size_t> n2, JfArg<const double *> h2, JfArg<const double *> flag,
                                               JfArg<const double *> inv) {
        jf_pdl_enter();
        const bool second = *flag != 0.0;
        const double sc = *inv;
        double2 *wv = reinterpret_cast<double2 *>(w);
        float2 *f2 = reinterpret_cast<float2 *>(w32);
        const double2 *Vp[NV];
        double c[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) {
            Vp[j] = reinterpret_cast<const double2 *>(V + (size_t)j * ldv);
            c[j] = -h2[j];
        }
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n2; i += (size_t)jf_nblk * RB) {
            double2 a = wv[i];
            if (second) {
                double2 v[NV];
    #pragma unroll
                for (int j = 0; j < NV; ++j) v[j] = Vp[j][i];
    #pragma unroll
                for (int j = 0; j < NV; ++j) {
                    a.x = fma(c[j], v[j].x, a.x);
                    a.y = fma(c[j], v[j].y, a.y);
                }
            }
            a.x *= sc;
            a.y *= sc;
            wv[i] = a;
            if (w32) f2[i] = make_float2(d2f_trunc(a.x), d2f_trunc(a.y));
        }
    }
};
template <int NV>
__global__ void __launch_bounds__(RB) k_gs_update_scale(const double *V, size_t ldv, double *w, float *w32,
                                                        size_t n2, const double *h2, const double *flag,
                                                        const double *inv) {
    k_gs_update_scale_b<NV>::run(blockIdx.x, gridDim.x, V, ldv, w, w32, n2, h2, flag, inv);
}

// pass 1 in FP32: h = V^T w from the float copy of the basis and w truncated to
// float, FP32 sums within a block, FP64 across blocks.  Its error (a float ulp
// of |w|) is removed by the FP64 second pass, which computes the remaining
// projection of w - V h exactly as classical Gram-Schmidt twice does.
template <int NV>
struct k_gs_dot32_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const float *> V32,
                                               JfArg<size_t> ldv, JfArg<const double *> w, JfArg<size_t> n2,
                                               JfArg<double *> part, JfArg<unsigned *> ticket, JfArg<double *> h) {
        jf_pdl_enter();
        const double2 *w2 = reinterpret_cast<const double2 *>(w);
        const float2 *Vp[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) Vp[j] = reinterpret_cast<const float2 *>(V32 + (size_t)j * ldv);
        float acc[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = 0.0f;
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n2; i += (size_t)jf_nblk * RB) {
            const double2 a = w2[i];
            const float ax = d2f_trunc(a.x), ay = d2f_trunc(a.y);
            float2 v[NV];
    #pragma unroll
            for (int j = 0; j < NV; ++j) v[j] = Vp[j][i];
    #pragma unroll
            for (int j = 0; j < NV; ++j) acc[j] = fmaf(v[j].y, ay, fmaf(v[j].x, ax, acc[j]));
        }
        __shared__ float sw[NV][RB / 32];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    #pragma unroll
        for (int j = 0; j < NV; ++j) {
            float v = acc[j];
    #pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sw[j][wid] = v;
        }
        __syncthreads();
        if (threadIdx.x < NV) {
            double r = 0.0;
    #pragma unroll
            for (int q = 0; q < RB / 32; ++q) r += (double)sw[threadIdx.x][q];
            part[(size_t)threadIdx.x * jf_nblk + jf_bid] = r;
        }
        if (!last_block(ticket, jf_nblk)) return;
        finish_multi<NV>(part, jf_nblk, h);
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
};
template <int NV>
__global__ void __launch_bounds__(RB) k_gs_dot32(const float *V32, size_t ldv, const double *w, size_t n2,
                                                 double *part, unsigned *ticket, double *h) {
    k_gs_dot32_b<NV>::run(blockIdx.x, gridDim.x, V32, ldv, w, n2, part, ticket, h);
}

template <class S>
struct k_dot_partial_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> x,
                                               JfArg<const S *> y, JfArg<size_t> n, JfArg<double *> part) {
        jf_pdl_enter();
        double acc = 0.0, acc2 = 0.0;
        const size_t stride = (size_t)jf_nblk * RB;
        size_t i = (size_t)jf_bid * RB + threadIdx.x;
        for (; i + stride < n; i += 2 * stride) {   // two loads in flight per thread
            const double a0 = (double)x[i], b0 = (double)y[i];
            const double a1 = (double)x[i + stride], b1 = (double)y[i + stride];
            acc = fma(a0, b0, acc);
            acc2 = fma(a1, b1, acc2);
        }
        if (i < n) acc = fma((double)x[i], (double)y[i], acc);
        acc = block_sum(acc + acc2);
        if (threadIdx.x == 0) part[jf_bid] = acc;
    }
};
template <class S>
__global__ void __launch_bounds__(RB) k_dot_partial(const S *x, const S *y, size_t n, double *part) {
    k_dot_partial_b<S>::run(blockIdx.x, gridDim.x, x, y, n, part);
}

// op (single-launch reductions): RED_SUM -> sum; RED_SQRT -> sqrt(sum);
// RED_EPS -> sqrt(2^-52)/sqrt(sum) (0 if sum == 0); RED_EPS32 -> sqrt(2^-23)/sqrt(sum)

// h_j partials for NV basis vectors at once: accumulators are compile-time
// indexed (registers), warp sums go through one shared-memory pass.
template <int NV>
struct k_mdot_partial_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<size_t> ldv, JfArg<const double *> w, JfArg<size_t> n,
                                               JfArg<double *> part, JfArg<const double *> flag) {
        jf_pdl_enter();
        if (flag && *flag == 0.0) {   // pass not needed: contribute zeros
            if (threadIdx.x < NV) part[(size_t)threadIdx.x * jf_nblk + jf_bid] = 0.0;
            return;
        }
        double acc[NV];
    #pragma unroll
        for (int j = 0; j < NV; ++j) acc[j] = 0.0;
        const size_t stride = (size_t)jf_nblk * RB;
        size_t i = (size_t)jf_bid * RB + threadIdx.x;
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
            part[(size_t)threadIdx.x * jf_nblk + jf_bid] = r;
        }
    }
};
template <int NV>
__global__ void __launch_bounds__(RB) k_mdot_partial(const double *V, size_t ldv, const double *w, size_t n,
                                                     double *part, const double *flag) {
    k_mdot_partial_b<NV>::run(blockIdx.x, gridDim.x, V, ldv, w, n, part, flag);
}

struct k_mfinal_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> part,
                                               JfArg<int> nb, JfArg<double *> out) {
        jf_pdl_enter();
        double acc = 0.0;
        for (int i = threadIdx.x; i < nb; i += RB) acc += part[(size_t)jf_bid * nb + i];
        acc = block_sum(acc);
        if (threadIdx.x == 0) out[jf_bid] = acc;
    }
};
__global__ void __launch_bounds__(RB) k_mfinal(const double *part, int nb, double *out) {
    k_mfinal_b::run(blockIdx.x, gridDim.x, part, nb, out);
}

// w += sign * sum_j h_j V_j
struct k_mupdate_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<int> nv, JfArg<size_t> ldv, JfArg<const double *> h,
                                               JfArg<double *> w, JfArg<size_t> n, JfArg<double> sign,
                                               JfArg<const double *> flag) {
        jf_pdl_enter();
        if (flag && *flag == 0.0) return;
        __shared__ double sh[MAXV];
        if (threadIdx.x < nv) sh[threadIdx.x] = sign * h[threadIdx.x];
        __syncthreads();
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride) {
            double acc = w[i];
            for (int j = 0; j < nv; ++j) acc = fma(sh[j], V[(size_t)j * ldv + i], acc);
            w[i] = acc;
        }
    }
};
__global__ void k_mupdate(const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                          double sign, const double *flag) {
    k_mupdate_b::run(blockIdx.x, gridDim.x, V, nv, ldv, h, w, n, sign, flag);
}

struct k_scale_copy_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> w,
                                               JfArg<const double *> nrm, JfArg<double *> v, JfArg<size_t> n) {
        jf_pdl_enter();
        const double s = *nrm;
        const double inv = s != 0.0 ? 1.0 / s : 0.0;
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride) v[i] = w[i] * inv;
    }
};
__global__ void k_scale_copy(const double *w, const double *nrm, double *v, size_t n) {
    k_scale_copy_b::run(blockIdx.x, gridDim.x, w, nrm, v, n);
}

struct k_axpby_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<double> a,
                                               JfArg<const double *> x, JfArg<double> b, JfArg<const double *> y,
                                               JfArg<double *> z, JfArg<size_t> n) {
        jf_pdl_enter();
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride)
            z[i] = a * x[i] + (y ? b * y[i] : 0.0);
    }
};
__global__ void k_axpby(double a, const double *x, double b, const double *y, double *z, size_t n) {
    k_axpby_b::run(blockIdx.x, gridDim.x, a, x, b, y, z, n);
}

// w += sign * sum_j h_j V_j and per-block partial sums of the updated w^2
// (about 8 elements per thread, like the dot kernels)
template <int NVMAX>
struct k_mupdate_norm_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> V,
                                               JfArg<int> nv, JfArg<size_t> ldv, JfArg<const double *> h,
                                               JfArg<double *> w, JfArg<size_t> n, JfArg<double> sign,
                                               JfArg<const double *> flag, JfArg<double *> part) {
        jf_pdl_enter();
        if (flag && *flag == 0.0) return;
        __shared__ double sh[NVMAX];
        if (threadIdx.x < nv) sh[threadIdx.x] = sign * h[threadIdx.x];
        __syncthreads();
        double acc2 = 0.0;
        const size_t stride = (size_t)jf_nblk * RB;
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n; i += stride) {
            double a = w[i];
            for (int j = 0; j < nv; ++j) a = fma(sh[j], V[(size_t)j * ldv + i], a);
            w[i] = a;
            acc2 = fma(a, a, acc2);
        }
        acc2 = block_sum(acc2);
        if (threadIdx.x == 0) part[jf_bid] = acc2;
    }
};
template <int NVMAX>
__global__ void __launch_bounds__(RB) k_mupdate_norm(const double *V, int nv, size_t ldv, const double *h,
                                                     double *w, size_t n, double sign, const double *flag,
                                                     double *part) {
    k_mupdate_norm_b<NVMAX>::run(blockIdx.x, gridDim.x, V, nv, ldv, h, w, n, sign, flag, part);
}

// After the first pass: w1sq = sum of partials, nrm = sqrt(w1sq) and the
// reorthogonalisation flag (|w1| < |w0|/sqrt(2), |w0|^2 = |w1|^2 + |h|^2).
// After the second pass (flag given): nrm = sqrt(sum) only if that pass ran.
struct k_final_gs_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> part,
                                               JfArg<int> nb, JfArg<const double *> h, JfArg<int> nv,
                                               JfArg<const double *> flag_in, JfArg<double *> w1sq,
                                               JfArg<double *> nrm, JfArg<double *> flag_out) {
        jf_pdl_enter();
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
};
__global__ void __launch_bounds__(RB) k_final_gs(const double *part, int nb, const double *h, int nv,
                                                 const double *flag_in, double *w1sq, double *nrm,
                                                 double *flag_out) {
    k_final_gs_b::run(blockIdx.x, gridDim.x, part, nb, h, nv, flag_in, w1sq, nrm, flag_out);
}

// float -> double widening on the integer pipe, exact: binary64 re-biases the
// binary32 exponent by 1023 - 127 = 896 and takes the 23 fraction bits as the
// top of its 52 (IEEE 754 formats); zero keeps its sign.  Subnormal, infinite
// and NaN inputs use the conversion instruction (an FP64-pipe operation, like
// the DFMA), out of line.
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    if ((b & 0x7fffffffu) != 0u && (e == 0u || e == 0xffu)) return f2d_slow(f);   // subnormal, inf, NaN
    const unsigned long long r = (b & 0x7fffffffu) == 0u ? sign
                                                          : sign | ((unsigned long long)(e + 896u) << 52) |
                                                                ((unsigned long long)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)r);
}

// y = (double) x and eps = sqrt(2^-52)/|y| (for the FD product) in one launch.
// The squares are summed in FP32 within a thread (eps needs a few digits), the
// per-thread partials in FP64.
struct k_f2d_eps_b {
    static constexpr int TPB = RB, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const float *> x,
                                               JfArg<double *> y, JfArg<size_t> n, JfArg<double *> part,
                                               JfArg<unsigned *> ticket, JfArg<double *> eps) {
        jf_pdl_enter();
        float acc = 0.0f, acc2 = 0.0f;
        const size_t stride = (size_t)jf_nblk * RB;
        const size_t n4 = n / 4;   // float4 in, two double2 out (x, y 16-byte aligned)
        const float4 *x4 = reinterpret_cast<const float4 *>(x);
        double2 *y2 = reinterpret_cast<double2 *>(y);
        for (size_t i = (size_t)jf_bid * RB + threadIdx.x; i < n4; i += stride) {
            const float4 f = x4[i];
            y2[2 * i] = make_double2(f2d_bits(f.x), f2d_bits(f.y));
            y2[2 * i + 1] = make_double2(f2d_bits(f.z), f2d_bits(f.w));
            acc = fmaf(f.y, f.y, fmaf(f.x, f.x, acc));
            acc2 = fmaf(f.w, f.w, fmaf(f.z, f.z, acc2));
        }
        for (size_t i = 4 * n4 + (size_t)jf_bid * RB + threadIdx.x; i < n; i += stride) {
            const float f = x[i];
            y[i] = f2d_bits(f);
            acc = fmaf(f, f, acc);
        }
        const double tsum = block_sum((double)acc + (double)acc2);
        if (threadIdx.x == 0) part[jf_bid] = tsum;
        if (!last_block(ticket, jf_nblk)) return;
        const double t = sum_partials(part, jf_nblk);
        if (threadIdx.x == 0) {
            *eps = finish_op(t, RED_EPS);
            *ticket = 0u;
        }
    }
};
__global__ void __launch_bounds__(RB) k_f2d_eps(const float *x, double *y, size_t n, double *part, unsigned *ticket,
                                                double *eps) {
    k_f2d_eps_b::run(blockIdx.x, gridDim.x, x, y, n, part, ticket, eps);
}

struct YV {
    double y[MAXV];
};

__device__ __forceinline__ double widen(float f) { return f2d_bits(f); }
__device__ __forceinline__ double widen(double d) { return d; }

template <class S>
struct k_zcomb_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const S *> Z, JfArg<int> nz,
                                               JfArg<size_t> n, JfArg<YV> yv, JfArg<double *> x) {
        jf_pdl_enter();
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride) {
            double acc = x[i];
            for (int j = 0; j < nz; ++j) acc = fma(yv.y[j], widen(Z[(size_t)j * n + i]), acc);
            x[i] = acc;
        }
    }
};
template <class S>
__global__ void k_zcomb(const S *Z, int nz, size_t n, YV yv, double *x) {
    k_zcomb_b<S>::run(blockIdx.x, gridDim.x, Z, nz, n, yv, x);
}

struct k_d2f_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> x,
                                               JfArg<float *> y, JfArg<size_t> n) {
        jf_pdl_enter();
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = (float)x[i];
    }
};
__global__ void k_d2f(const double *x, float *y, size_t n) {
    k_d2f_b::run(blockIdx.x, gridDim.x, x, y, n);
}
struct k_f2d_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const float *> x,
                                               JfArg<double *> y, JfArg<size_t> n) {
        jf_pdl_enter();
        const size_t stride = (size_t)jf_nblk * blockDim.x;
        for (size_t i = (size_t)jf_bid * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = f2d_bits(x[i]);
    }
};
__global__ void k_f2d(const float *x, double *y, size_t n) {
    k_f2d_b::run(blockIdx.x, gridDim.x, x, y, n);
}

// grid-stride launches of 256 threads: at most 16 blocks per SM of the current device
inline unsigned grid_for(size_t n) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1) {
        cudaGetLastError();
        nsm = 1;
    }
    size_t g = (n + 255) / 256;
    if (g > (size_t)nsm * 16) g = (size_t)nsm * 16;
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

static double eps_numerator(const jfnk_ctx *c, int op) {
    if (op == RED_EPS32) return 3.4526698300124393e-04;   // sqrt(2^-23)
    if (op == RED_EPSP && c->opts.precond_fd_eps > 0.0) return c->opts.precond_fd_eps;
    return 1.4901161193847656e-08;                         // sqrt(2^-52)
}

int red_dot(jfnk_ctx *c, const double *x, const double *y, size_t n, double *out, int op, cudaStream_t s) {
    const int nb = nblocks_red(c, n);
    jf_launch<k_dot1_b<double>>(k_dot1<double>, nb, RB, 0, s, x, y, n, c->partial, c->ticket, out, op, eps_numerator(c, op));
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int red_dotf(jfnk_ctx *c, const float *x, const float *y, size_t n, double *out, int op, cudaStream_t s) {
    const int nb = nblocks_red(c, n);
    jf_launch<k_dot1_b<float>>(k_dot1<float>, nb, RB, 0, s, x, y, n, c->partial, c->ticket, out, op, eps_numerator(c, op));
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// CGS2 of w against V_0..V_{nv-1} (nv <= GS_FUSED_MAX; n even, V, w 16-byte
// aligned), then w <- w / |w|: h1, h2, |w1|^2, the second-pass flag, |w| and
// 1/|w| (nrm[S_INV - S_NORM]) land in device memory.  Three launches.
// One wave: the SM count times the blocks of this kernel an SM holds, at most
// three (FP64-bound kernels lose a partial second wave otherwise), fewer for
// short vectors.
template <class F>
static int one_wave(jfnk_ctx *c, F kernel, size_t n2) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, RB, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    if (per_sm > 3) per_sm = 3;   // fewer partials for the closing block to add
    size_t g = (size_t)c->n_sm * per_sm;
    const size_t need = (n2 + RB - 1) / RB;
    if (g > need) g = need;
    if (g > (size_t)c->nb_red) g = c->nb_red;
    return g < 1 ? 1 : (int)g;
}

template <int NV>
static void cgs2_t(jfnk_ctx *c, const double *V, const float *V32, size_t ldv, double *w, float *w32, size_t n,
                   double *h1, double *h2, double *w1sq, double *nrm, double *flag, cudaStream_t s) {
    const size_t n2 = n / 2;
    const int g2 = one_wave(c, k_gs_update_dot<NV>, n2), g3 = one_wave(c, k_gs_update_scale<NV>, n2);
    if (V32) {
        const int g1 = one_wave(c, k_gs_dot32<NV>, n2);
        jf_launch<k_gs_dot32_b<NV>>(k_gs_dot32<NV>, g1, RB, 0, s, V32, ldv, w, n2, c->partial, c->ticket, h1);
    } else {
        const int g1 = one_wave(c, k_gs_dot<NV>, n2);
        jf_launch<k_gs_dot_b<NV>>(k_gs_dot<NV>, g1, RB, 0, s, V, ldv, w, n2, c->partial, c->ticket, h1);
    }
    jf_launch<k_gs_update_dot_b<NV>>(k_gs_update_dot<NV>, g2, RB, 0, s, V, ldv, w, n2, h1, c->partial, c->ticket, h2, w1sq, nrm, flag);
    jf_launch<k_gs_update_scale_b<NV>>(k_gs_update_scale<NV>, g3, RB, 0, s, V, ldv, w, w32, n2, h2, flag, nrm + (S_INV - S_NORM));
    jf_launched(3);
}

int blas_cgs2(jfnk_ctx *c, const double *V, const float *V32, int nv, size_t ldv, double *w, float *w32, size_t n,
              double *h1, double *h2, double *w1sq, double *nrm, double *flag, cudaStream_t s) {
    if (nv < 1 || nv > GS_FUSED_MAX || (n & 1) || (ldv & 1)) return JFNK_EINVAL;
    switch (nv) {
#define JF_GS(K) case K: cgs2_t<K>(c, V, V32, ldv, w, w32, n, h1, h2, w1sq, nrm, flag, s); break;
        JF_GS(1) JF_GS(2) JF_GS(3) JF_GS(4) JF_GS(5) JF_GS(6) JF_GS(7) JF_GS(8)
        JF_GS(9) JF_GS(10) JF_GS(11) JF_GS(12) JF_GS(13) JF_GS(14) JF_GS(15) JF_GS(16)
#undef JF_GS
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// Diagnostic timing of the three CGS2 launches with 8 basis vectors on the
// context's basis buffers (filled with a fixed byte pattern, so the second pass
// is always taken, as on the solver's problems).  ms[0]: pass 1 (FP32 multi-dot),
// ms[1]: passes 2 and 3 (update + dot, update + normalisation); means over reps.
int blas_time_cgs2(jfnk_ctx *c, int reps, double *ms, cudaStream_t s) {
    constexpr int NV = 8;
    const size_t N = c->N;
    if (c->opts.gmres_restart < NV || (N & 1)) return JFNK_EINVAL;
    JF_CK(cudaMemsetAsync(c->V, 0x3f, 8 * N * (NV + 1), s));
    JF_CK(cudaMemsetAsync(c->V32, 0x3f, 4 * N * (NV + 1), s));
    double *w = c->V + (size_t)NV * N;
    cudaEvent_t e[3];
    for (auto &x : e) JF_CK(cudaEventCreate(&x));
    const size_t n2 = N / 2;
    const int g1 = one_wave(c, k_gs_dot32<NV>, n2), g2 = one_wave(c, k_gs_update_dot<NV>, n2),
              g3 = one_wave(c, k_gs_update_scale<NV>, n2);
    double t0 = 0.0, t1 = 0.0;
    int rc = JFNK_OK;
    for (int r = 0; r < reps && rc == JFNK_OK; ++r) {
        JF_CK(cudaMemsetAsync(w, 0x3f, 8 * N, s));
        cudaEventRecord(e[0], s);
        jf_launch<k_gs_dot32_b<NV>>(k_gs_dot32<NV>, g1, RB, 0, s, (const float *)c->V32, N, (const double *)w, n2, c->partial,
                  c->ticket, c->scal + S_H);
        cudaEventRecord(e[1], s);
        jf_launch<k_gs_update_dot_b<NV>>(k_gs_update_dot<NV>, g2, RB, 0, s, (const double *)c->V, N, w, n2, (const double *)(c->scal + S_H),
                  c->partial, c->ticket, c->scal + S_H2, c->scal + S_W1, c->scal + S_NORM, c->scal + S_FLAG);
        jf_launch<k_gs_update_scale_b<NV>>(k_gs_update_scale<NV>, g3, RB, 0, s, (const double *)c->V, N, w, c->V32 + (size_t)NV * N, n2,
                  (const double *)(c->scal + S_H2), (const double *)(c->scal + S_FLAG), c->scal + S_INV);
        jf_launched(3);
        cudaEventRecord(e[2], s);
        if (cudaEventSynchronize(e[2]) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = JFNK_ECUDA;
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

template <int NV>
void mdot_chunk(const double *V, size_t ldv, const double *w, size_t n, double *part, int nb, cudaStream_t s,
                const double *flag) {
    jf_launch<k_mdot_partial_b<NV>>(k_mdot_partial<NV>, nb, RB, 0, s, V, ldv, w, n, part, flag);
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
        jf_launch<k_mfinal_b>(k_mfinal, m, RB, 0, s, c->partial, nb, h + j0); jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_mupdate(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                 double sign, cudaStream_t s, const double *flag) {
    (void)c;
    for (int j0 = 0; j0 < nv; j0 += MAXV) {
        const int m = nv - j0 < MAXV ? nv - j0 : MAXV;
        jf_launch<k_mupdate_b>(k_mupdate, grid_for(n), 256, 0, s, V + (size_t)j0 * ldv, m, ldv, h + j0, w, n, sign, flag); jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_scale_copy(const double *w, const double *nrm, double *v, size_t n, cudaStream_t s) {
    jf_launch<k_scale_copy_b>(k_scale_copy, grid_for(n), 256, 0, s, w, nrm, v, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_axpby(double a, const double *x, double b, const double *y, double *z, size_t n, cudaStream_t s) {
    jf_launch<k_axpby_b>(k_axpby, grid_for(n), 256, 0, s, a, x, b, y, z, n); jf_launched();
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
            jf_launch<k_zcomb_b<float>>(k_zcomb<float>, grid_for(n), 256, 0, s, (const float *)Z + (size_t)j0 * n, m, n, y, x);
        else
            jf_launch<k_zcomb_b<double>>(k_zcomb<double>, grid_for(n), 256, 0, s, (const double *)Z + (size_t)j0 * n, m, n, y, x);
        jf_launched();
    }
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

// Second Gram-Schmidt pass needed?  With w1 = w0 - V h the first pass left
// |w1|^2 of |w0|^2 = |w1|^2 + |h|^2; reorthogonalise when |w1| < |w0| / sqrt(2)
// ("twice is enough").  flag = 1.0 or 0.0, decided on the device.
struct k_reortho_flag_b {
    static constexpr int TPB = 0, MINB = 0;
    static __device__ __forceinline__ void run(unsigned jf_bid, unsigned jf_nblk, JfArg<const double *> w1sq,
                                               JfArg<const double *> h, JfArg<int> nv, JfArg<double *> flag) {
        jf_pdl_enter();
        double hh = 0.0;
        for (int i = threadIdx.x; i < nv; i += 32) hh += h[i] * h[i];
        hh = warp_sum(hh);
        if (threadIdx.x == 0) *flag = (*w1sq < 0.5 * (*w1sq + hh)) ? 1.0 : 0.0;
    }
};
__global__ void k_reortho_flag(const double *w1sq, const double *h, int nv, double *flag) {
    k_reortho_flag_b::run(blockIdx.x, gridDim.x, w1sq, h, nv, flag);
}

int blas_reortho_flag(const double *w1sq, const double *h, int nv, double *flag, cudaStream_t s) {
    jf_launch<k_reortho_flag_b>(k_reortho_flag, 1, 32, 0, s, w1sq, h, nv, flag);
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
        jf_launch<k_dot_partial_b<double>>(k_dot_partial<double>, nb, RB, 0, s, w, w, n, c->partial);
        jf_launched();
        jf_launch<k_final_gs_b>(k_final_gs, 1, RB, 0, s, c->partial, nb, h, nv, flag_in, w1sq, nrm, flag_out);
        jf_launched();
        JF_CK(cudaGetLastError());
        return JFNK_OK;
    }
    const int nb = nblocks_red(c, n);
    jf_launch<k_mupdate_norm_b<MAXV>>(k_mupdate_norm<MAXV>, nb, RB, 0, s, V, nv, ldv, h, w, n, sign, flag_in, c->partial);
    jf_launched();
    jf_launch<k_final_gs_b>(k_final_gs, 1, RB, 0, s, c->partial, nb, h, nv, flag_in, w1sq, nrm, flag_out);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_f2d_eps(jfnk_ctx *c, const float *x, double *y, size_t n, double *eps_out, cudaStream_t s) {
    if (((uintptr_t)x & 15) || ((uintptr_t)y & 15)) return JFNK_EINVAL;
    const int nb = nblocks_red(c, n);
    jf_launch<k_f2d_eps_b>(k_f2d_eps, nb, RB, 0, s, x, y, n, c->partial, c->ticket, eps_out);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_copy_d2f(const double *x, float *y, size_t n, cudaStream_t s) {
    jf_launch<k_d2f_b>(k_d2f, grid_for(n), 256, 0, s, x, y, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int blas_copy_f2d(const float *x, double *y, size_t n, cudaStream_t s) {
    jf_launch<k_f2d_b>(k_f2d, grid_for(n), 256, 0, s, x, y, n); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}
