// jfnk_norm2_noalloc: the Euclidean norm of jfnk_norm2 for callers that must
// not allocate device memory.  Such callers include code that runs while a CUDA
// graph is being captured on another stream, allocators and memory pools that
// call into the solver, and services started with a fixed device-memory budget
// that forbids allocation after start-up.  They also cannot hold a jfnk
// context, because creating one allocates.
//
// The partial sums live in one file-scope device array of fixed size, so this
// entry point allocates nothing: every GPU that loads the library holds the
// array (32 KiB) until the process exits.
#include <mutex>

#include "internal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 4096;          // partial sums in the array
constexpr size_t NA_PER_BLOCK = 8192;        // elements reduced by one block
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) double g_norm2_scratch[NA_MAX_BLOCKS];

// The host cannot pass &g_norm2_scratch to a kernel (on the host that name is
// a stand-in, not a device address), so each device's address is looked up
// once with that device current and cached here.
double *g_scratch_addr[NA_MAX_DEVICES];
std::mutex g_scratch_mu;

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double na_block_sum(double v) {
    __shared__ double sw[NA_THREADS / 32];
    v = na_warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sw[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) r = na_warp_sum(lane < NA_THREADS / 32 ? sw[lane] : 0.0);
    return r;   // valid in thread 0
}

// block b sums x[b*NA_PER_BLOCK, (b+1)*NA_PER_BLOCK) of squares into part[b]
__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const double *x, size_t n, double *part) {
    const size_t lo = (size_t)blockIdx.x * NA_PER_BLOCK;
    const size_t hi = lo + NA_PER_BLOCK < n ? lo + NA_PER_BLOCK : n;
    double acc = 0.0;
    for (size_t i = lo + threadIdx.x; i < hi; i += NA_THREADS) acc = fma(x[i], x[i], acc);
    acc = na_block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// fixed-order sum of the nb partials, then the square root (nb = 0: |x| = 0)
__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double *part, int nb, double *out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += NA_THREADS) acc += part[i];
    acc = na_block_sum(acc);
    if (threadIdx.x == 0) *out = sqrt(acc);
}

// Address of this device's scratch array; looked up on the first call on the
// device (with that device current) and cached.
int scratch_for_current_device(double **ptr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return JFNK_ECUDA;
    }
    if (dev < 0 || dev >= NA_MAX_DEVICES) return JFNK_EINVAL;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        double *p = nullptr;
        if (cudaGetSymbolAddress((void **)&p, g_norm2_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return JFNK_ECUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *ptr = g_scratch_addr[dev];
    return JFNK_OK;
}

}  // namespace

extern "C" int jfnk_norm2_noalloc(const double *x, size_t n, double *out, void *stream) {
    if (!out || (n > 0 && !x)) return JFNK_EINVAL;
    if (n > JFNK_NORM2_NOALLOC_MAX_N) return JFNK_EINVAL;   // beyond the fixed scratch
    double *part = nullptr;
    JF_RET(scratch_for_current_device(&part));
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    if (nb > 0) {
        k_na_partial<<<nb, NA_THREADS, 0, s>>>(x, n, part);
        jf_launched();
    }
    k_na_final<<<1, NA_THREADS, 0, s>>>(part, nb, out);
    jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}
