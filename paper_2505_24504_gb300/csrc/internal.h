// Internal state of a jfnk context (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>

#include <string.h>

#include <functional>
#include <type_traits>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/jfnk.h"
#include "physics.cuh"

#define JF_MAXLEV 12

// Programmatic dependent launch: the solver's kernels are launched with
// programmatic stream serialisation and each first waits (griddepcontrol.wait)
// for its predecessor grid to complete with its memory writes visible, so no
// read or write moves ahead of that point.  The successor is released when the
// predecessor completes (no early trigger: blocks that wait early would hold
// SM resources the predecessor still needs); what is saved is part of the
// launch latency between dependent kernels.  JFNK_PDL=0 in the environment
// launches them with plain stream ordering.
#ifdef __CUDACC__
__device__ __forceinline__ void jf_pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
#endif

template <typename... KArgs, typename... Args>
inline cudaError_t jf_launch_now(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    static const int pdl = [] {
        const char *e = getenv("JFNK_PDL");
        return e ? atoi(e) : 1;
    }();
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---- lock-step replay of several contexts' launches (ensembles) -----------
// Every kernel of the solver path is a body struct B (B::run(bid, nblk, args...),
// B::TPB / B::MINB its launch bounds) wrapped by a __global__ kernel that passes
// blockIdx.x and gridDim.x.  While a host thread records (t_jf_rec set, see
// batch.cu), jf_launch stores the launch instead of issuing it: its argument
// record and the grouped twin k_grouped<B, A...>, which runs the same body for
// the blocks of several members in one launch -- each block finds its member in
// a table of (first block, block count, argument record) and runs the body with
// the member's own block index and count, so every member computes exactly what
// its own launch computes.
// Bodies take their arguments by const reference, so that a grouped block reads
// its member's arguments where they lie in the table (no per-thread copy).
template <class T> using JfArg = const T &;

template <class... A> struct JfPack;
template <> struct JfPack<> {};
template <class H, class... R> struct JfPack<H, R...> {
    H h;
    JfPack<R...> r;
};
inline JfPack<> jf_pack() { return {}; }
template <class H, class... R>
inline JfPack<H, R...> jf_pack(H h, R... r) {
    return JfPack<H, R...>{h, jf_pack(r...)};
}
template <class... A> struct JfEnt {
    unsigned b0, nb;     // the member's first block in the grouped launch, its block count
    JfPack<A...> a;
};

constexpr int jf_tpb(int tpb) { return tpb > 0 ? tpb : 1024; }
constexpr int jf_minb(int tpb, int minb) { return minb > 0 ? minb : (tpb > 0 ? 1024 / tpb : 1); }

#ifdef __CUDACC__
template <class B, class... Done>
__device__ __forceinline__ void jf_call(unsigned bid, unsigned nb, const JfPack<> &, const Done &...d) {
    B::run(bid, nb, d...);
}
template <class B, class H, class... R, class... Done>
__device__ __forceinline__ void jf_call(unsigned bid, unsigned nb, const JfPack<H, R...> &p, const Done &...d) {
    jf_call<B>(bid, nb, p.r, d..., p.h);
}
template <class B, class... A>
// (register target of the twin: the body's own bounds, else 64 registers a thread)
__global__ void __launch_bounds__(jf_tpb(B::TPB), jf_minb(B::TPB, B::MINB))
    k_grouped(const JfEnt<A...> *__restrict__ t, int n) {
    const unsigned b = blockIdx.x;
    int lo = 0, hi = n - 1;   // last member whose first block is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t[mid].b0 <= b) lo = mid;
        else hi = mid - 1;
    }
    jf_call<B>(b - t[lo].b0, t[lo].nb, t[lo].a);
}
#endif

// One recorded operation of a member: a launch that can join a grouped launch
// (glaunch set: the same body and argument types, block shape and shared memory
// join), or any other stream operation replayed as is (run).
struct JfOp {
    std::function<cudaError_t(cudaStream_t)> run;
    cudaError_t (*glaunch)(const void *dtab, int n, unsigned total, dim3 block, size_t smem, cudaStream_t s);
    std::vector<unsigned char> ent;   // the member's JfEnt (b0 filled in at replay)
    unsigned nb;
    dim3 block;
    size_t smem;
    bool kernel;   // a kernel launch (counted in the launch statistics)
};
struct JfLockstep;   // batch.cu
struct JfRecorder {
    std::vector<JfOp> ops;
    JfLockstep *ls;
    int member;
};
extern thread_local JfRecorder *t_jf_rec;

template <class B, class... A>
cudaError_t jf_group_launch(const void *dtab, int n, unsigned total, dim3 block, size_t smem, cudaStream_t s) {
#ifdef __CUDACC__
    return jf_launch_now(k_grouped<B, A...>, dim3(total), block, smem, s, (const JfEnt<A...> *)dtab, n);
#else
    return cudaErrorNotSupported;
#endif
}

// B::GROUP (default true): whether body B has a grouped twin; without one its
// recorded launches replay one member at a time
template <class B, class = void> struct JfGroupOk { static constexpr bool value = true; };
template <class B> struct JfGroupOk<B, std::void_t<decltype(B::GROUP)>> { static constexpr bool value = B::GROUP; };

template <class B, class... KArgs>
cudaError_t jf_record(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, KArgs... a) {
    JfOp op;
    op.run = [=](cudaStream_t s) { return jf_launch_now(kernel, grid, block, smem, s, a...); };
    op.glaunch = nullptr;
    op.kernel = true;
    if constexpr (JfGroupOk<B>::value) {
        op.glaunch = &jf_group_launch<B, KArgs...>;
        JfEnt<KArgs...> e{0u, grid.x, jf_pack(a...)};
        op.ent.resize(sizeof(e));
        memcpy(op.ent.data(), &e, sizeof(e));
    }
    op.nb = grid.x;
    op.block = block;
    op.smem = smem;
    t_jf_rec->ops.push_back(std::move(op));
    return cudaSuccess;
}

// Launch kernel (the wrapper of body B) on s, or record it (lock-step replay).
template <class B, typename... KArgs, typename... Args>
inline cudaError_t jf_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
    if (t_jf_rec) return jf_record<B, KArgs...>(kernel, grid, block, smem, KArgs(std::forward<Args>(args))...);
    return jf_launch_now(kernel, grid, block, smem, s, std::forward<Args>(args)...);
}

// Stream operations of the solver path: issued on s, or recorded in order with
// the member's launches.  jf_sync waits for the stream (recording: for the
// replay of everything recorded so far).  A host-to-device copy is recorded with
// a copy of its source bytes.
cudaError_t jf_memcpy(void *dst, const void *src, size_t n, cudaMemcpyKind kind, cudaStream_t s);
cudaError_t jf_memset(void *dst, int v, size_t n, cudaStream_t s);
cudaError_t jf_sync(cudaStream_t s);

// Fixed 1D tables of the nodal Q_k space on Gauss-Legendre nodes (k <= 4).
struct DGTab {
    int np1;
    double xi[5], w[5];
    double Dn[5][5];     // Dn[a][q] = l_q'(xi_a): derivative at node a of basis q
    double Dw[5][5];     // Dw[a][q] = w_q l_a'(xi_q) / w_a: volume term of the weak form
    double lp[5], lm[5];     // l_a(+1), l_a(-1)
    double dlp[5], dlm[5];   // l_a'(+1), l_a'(-1)
    double lpw[5], lmw[5], dlpw[5], dlmw[5];   // the same divided by w_a
    double V[5][5];      // V[i][a] = l_a(c_i), subcell centre c_i = -1 + (2i+1)/(k+1)
    double Vinv[5][5];
    double P[5][5];      // P[i][a] = mean of l_a over subcell i (L2 projection)
    double Pinv[5][5];
    double om[5];        // modified Newton-Cotes weights on [0,1] at the subcell centres
};

struct FVLev {
    int NX, NZ;
    int fac;             // agglomeration factor to the next coarser level (0: coarsest)
    double Hx, Hz;
    size_t n;            // 4 NX NZ
    double *ub;          // [4][NZ] background at the cell centres
    float *ubf;          // its FP32 copy (tangent kernels)
    double *hbx;         // [4][NZ] HLLC(ub, ub; x)
    double *hbxw;        // [2][4][NZ] left wall HLLC(mirror ub, ub), right wall HLLC(ub, mirror ub)
    double *hbz;         // [4][NZ+1] HLLC(ub_{J-1}, ub_J; z); J = 0 bottom wall, J = NZ top wall
    // level vectors; element type is double (prec 64) or float (prec 32/16)
    void *u, *fu, *x, *x2, *b, *r;
    void *dtau;          // [NZ][NX]
    uint16_t *xb, *bb;   // bf16 storage of x and b on the coarsest level (prec 16)
};

struct jfnk_ctx {
    jfnk_grid grid;
    int k, np1, n_el;
    jfnk_physics phys;
    jfnk_opts opts;
    size_t N;            // 4 n_el (k+1)^2
    size_t npt;          // n_el (k+1)^2 nodes
    double hx, hz;
    PhysC pc;
    DGTab tab;
    int dev;
    // key
    int mg_on, dg_pre, dg_post, fine_pre, fine_post, mid_pre, mid_post, cycles;
    int prec;            // 64, 32, 16
    // device tables
    PowTab *powtab;
    double *ubv, *dubv, *fbx, *fbz, *hbx, *hbxw;   // node rows: [4][nz np1] ([2][4][..] for hbxw)
    double *ubh, *dubh, *hbz;                      // horizontal faces: [4][nz+1]
    float *ubvf, *dubvf, *ubhf, *dubhf;            // FP32 copies (tangent kernels)
    double *prow;        // [nz np1] p0^(R/cp) p~^(1/gamma) / R at node rows (insertion)
    double *theta_row;   // [nz np1] theta~ at node rows
    // DG face buffers: FP64 and FP32-tangent variants
    double *phix, *symx, *phiz, *symz;
    float *phixf, *symxf, *phizf, *symzf;
    // DG work vectors (FP64, N each)
    double *fU, *w1, *w2, *Ubs, *Un, *Usave, *G, *dU;
    // Krylov basis: V (m+1) N doubles, Z m N of the preconditioner's type
    double *V;
    float *V32;          // float copy of V (first Gram-Schmidt pass)
    void *Z;
    // preconditioner DG vectors (type of the preconditioner)
    void *pz, *pz2, *pd, *pr;
    double *dtau_dg;     // [n_el]
    float *dtau_dgf;     // [n_el] FP32 copy (prec 32)
    float *Usf;          // FP32 copy of the linearisation state U' + Ubar (prec 32)
    int nlev;
    FVLev lev[JF_MAXLEV];
    // reductions
    double *partial;     // scratch partial sums
    double *trU;         // face traces of the Newton iterate (values, and derivatives when viscous)
    int tr_valid;        // trU and fU come from the same residual evaluation
    unsigned *ticket;    // arrival counter of the single-launch reductions (0 between launches)
    int nb_red;          // partial-sum blocks
    int n_sm;            // streaming multiprocessors of the context's device
    double *scal;        // device scalars (norms, eps)
    double *h_pinned;    // host pinned scratch for Hessenberg columns
    // linearisation of the preconditioner (set by mg_linearize)
    double mg_adt;
    const double *mg_U;  // = Ulin, the context's copy of the linearisation state
    double *Ulin;
    // counters of the current call
    long long dg_calls, fv_calls;
    double deadline;     // steady-clock seconds at which the current implicit step times out (0: none)
    // graph of one preconditioner application (captured on cap_stream, replayed
    // on the caller's stream); valid for one linearisation adt
    cudaGraphExec_t mg_graph;
    cudaStream_t cap_stream;
    int mg_graph_valid;
    double mg_graph_adt;
    unsigned long long graph_launches;   // kernels in the graph
    long long graph_dg_calls, graph_fv_calls;
    void *pin, *pout;                    // fixed input / output of the graph
    int mg_graph_gen;                    // incremented at every capture of the preconditioner
    int capturing;                       // 1 while an Arnoldi step is being captured
    // one graph per Arnoldi step index j (preconditioner child graph, FD
    // product, Gram-Schmidt, normalisation, Hessenberg column copy)
    cudaGraphExec_t arn_graph[64];
    int arn_valid[64], arn_gen[64];
    double arn_adt;
    unsigned long long arn_launches[64];
    long long arn_dg_calls[64], arn_fv_calls[64];
    size_t alloc_bytes;
    void *allocs;        // list of this context's allocations (api.cu)
    // optional per-launch timing of the DG kernels (jfnk_time_operator)
    cudaEvent_t tev[3];
    int timing;
    double t_faces_ms, t_volume_ms;
};

// device scalar slots in ctx->scal
enum { S_NORM = 0, S_EPS = 1, S_W1 = 2, S_FLAG = 3, S_INV = 4, S_EPSDG = 5, S_EPSFV = 8, S_NRM_FV = 24, S_H = 64, S_H2 = 128, S_COUNT = 256 };

// number of kernels this library has launched (diagnostic counter); the
// thread-local twin lets a graph capture count only its own thread's launches
extern unsigned long long g_jf_launches;
extern thread_local unsigned long long t_jf_launches;
inline void jf_launched(unsigned n = 1) {
    if (t_jf_rec) return;   // recorded launches are counted when they are replayed
    __atomic_fetch_add(&g_jf_launches, (unsigned long long)n, __ATOMIC_RELAXED);
    t_jf_launches += n;
}

// Device-wide synchronisation (context creation and destruction: cudaMalloc,
// synchronous copies, cudaDeviceSynchronize, cudaFree) is invalid while any
// stream of the device is being captured, so captures and these calls take
// this process-wide lock.
extern std::mutex g_jf_device_mu;

// ---- kernels / launchers (implemented in the .cu files) ----
// background fluxes of the DG operator and of every FV level, launched on s
// (context creation runs them on a private stream and waits for that stream only)
int dg_setup_background(jfnk_ctx *c, cudaStream_t s);
int fv_setup_background(jfnk_ctx *c, cudaStream_t s);

// DG operator modes
enum DGMode {
    DG_RES = 0,      // out0 = f(U')
    DG_JV = 1,       // out0 = y - adt (f(U' + eps y) - fU) / eps       (eps: device scalar)
    DG_G = 2,        // out0 = U' - adt f - Ubar_s ; out1 = f
    DG_SMOOTH64 = 3, // out0 = z + dtau (r - [z - adt (f(U'+eps z) - fU)/eps])
    DG_TLJV = 4,     // out0 = z - adt J z, or r - (z - adt J z) when rf is given  (FP32 tangent)
    DG_TLSMOOTH = 5  // out0 = z + dtau (r - (z - adt J z))            (FP32 tangent)
};

// DG -> finest-FV transfer T^mf folded into the FP32 defect kernel: the 1D
// transfer matrix (interpolation at the subcell centres or subcell means), the
// modified Newton-Cotes weights of the mass fix, the level's b (and x = dtau b, the
// first pseudo-time step from zero, when x0 is given)
struct TransferOut {
    float V[5][5];
    float om[5];
    int massfix;
    int NX, NZ;
    float *b, *x0;
    const float *dtau0;
};

struct DGArgs {
    const double *U;       // state U' (FP64)
    const float *Uf;       // state U' (FP32, tangent modes)
    const double *y;       // FP64 direction (JV, SMOOTH64)
    const float *yf;       // FP32 direction (TL modes)
    const double *fU;      // cached f(U')
    const double *r;       // FP64 right-hand side (SMOOTH64)
    const float *rf;       // FP32 right-hand side (TLSMOOTH)
    const double *Ubs;     // Ubar_s (G)
    const double *eps;     // device scalar eps (JV, SMOOTH64)
    const double *dtau;    // [n_el] (smoothing)
    const float *dtauf;    // [n_el] (FP32 smoothing)
    double adt;
    float adtf;            // FP32 copies of adt and alpha for the tangent kernels (set by dg_apply)
    float alphaf;
    void *out0;
    double *out1;
    double *tr_out;        // FP64 residual / G: store the face traces of U here (may be null)
    const double *tr_in;   // FP64 FD product: face traces of U from the residual at U (may be null)
    float *out1f;          // FP32 defect at the first step from zero: z = dtau r is formed from rf and
                           // dtauf on the fly (yf unused) and written here
    const TransferOut *tro;   // with out1f: also T^mf of the defect to the finest FV level (host struct,
                              // passed by value to the kernel; null: the defect goes to out0)
    // smoothing modes, one stage of the multi-stage pseudo-time scheme: z0mode 0 explicit
    // Euler z + dtau (r - G'z); 1 z0 + alpha dtau (r - G'z) (z the previous stage); 2 the
    // same with z0 = 0
    const void *z0;
    int z0mode;
    double alpha;
};

int dg_apply(jfnk_ctx *c, int mode, const DGArgs &a, cudaStream_t s);
size_t dg_member_bytes();
int dg_residual_grouped(jfnk_ctx *const *ctx, int n, const double *const *U, double *const *f, void *dmem,
                        cudaStream_t s);

// reductions / BLAS-1 (blas.cu)
int red_dot(jfnk_ctx *c, const double *x, const double *y, size_t n, double *out_dev, int op, cudaStream_t s);
int red_dotf(jfnk_ctx *c, const float *x, const float *y, size_t n, double *out_dev, int op, cudaStream_t s);
// RED_EPSP: eps of the preconditioner's FD products, numerator opts.precond_fd_eps
// (sqrt(eps_mach) when 0)
enum { RED_SUM = 0, RED_SQRT = 1, RED_EPS = 2, RED_EPS32 = 3, RED_EPSP = 4 };
int blas_mdot(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *w, size_t n, double *h_dev, cudaStream_t s,
              const double *flag = nullptr);
int blas_mupdate(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *h_dev, double *w, size_t n, double sign,
                 cudaStream_t s, const double *flag = nullptr);
int blas_reortho_flag(const double *w1sq, const double *h, int nv, double *flag, cudaStream_t s);
int blas_mupdate_norm(jfnk_ctx *c, const double *V, int nv, size_t ldv, const double *h, double *w, size_t n,
                      double sign, const double *flag_in, double *w1sq, double *nrm, double *flag_out,
                      cudaStream_t s);
constexpr int GS_FUSED_MAX = 16;   // basis vectors of the fused CGS2 kernels
// V32 (optional): float copy of the basis (first pass in FP32); w32: where the
// float copy of the normalised w goes (may be null)
int blas_cgs2(jfnk_ctx *c, const double *V, const float *V32, int nv, size_t ldv, double *w, float *w32, size_t n,
              double *h1, double *h2, double *w1sq, double *nrm, double *flag, cudaStream_t s);
int blas_time_cgs2(jfnk_ctx *c, int reps, double *ms, cudaStream_t s);
int blas_f2d_eps(jfnk_ctx *c, const float *x, double *y, size_t n, double *eps_out, cudaStream_t s);
int blas_scale_copy(const double *w, const double *nrm_dev, double *v, size_t n, cudaStream_t s);
int blas_axpby(double a, const double *x, double b, const double *y, double *z, size_t n, cudaStream_t s);
int blas_zcomb(const void *Z, int prec32, int nz, size_t n, const double *yv, double *x, cudaStream_t s);
int blas_copy_d2f(const double *x, float *y, size_t n, cudaStream_t s);
int blas_copy_f2d(const float *x, double *y, size_t n, cudaStream_t s);
int blas_scale(double a, const double *x, double *y, size_t n, cudaStream_t s);

// preconditioner (mg.cu)
int mg_linearize(jfnk_ctx *c, const double *U, double adt, cudaStream_t s);
// r32 (optional): r already in FP32 (FP32 preconditioner, used when the kernels
// are launched or captured directly)
int mg_apply(jfnk_ctx *c, const double *r, void *z, cudaStream_t s, const float *r32 = nullptr);
int mg_graph_prepare(jfnk_ctx *c);
int mg_time_fv_level0(jfnk_ctx *c, const double *U, const double *y, int reps, double *ms, cudaStream_t s);
void jf_invalidate_graphs(jfnk_ctx *c);
int fv_rhs64(jfnk_ctx *c, int l, const double *u, double *f, cudaStream_t s);
int transfer_to_fv64(jfnk_ctx *c, const double *u, double *v, cudaStream_t s);
int transfer_to_dg64(jfnk_ctx *c, const double *v, double *u, int accumulate, cudaStream_t s);

#define JF_CK(...)                                   \
    do {                                             \
        cudaError_t e_ = (__VA_ARGS__);              \
        if (e_ != cudaSuccess) return JFNK_ECUDA;    \
    } while (0)
#define JF_RET(...)                                  \
    do {                                             \
        int r_ = (__VA_ARGS__);                      \
        if (r_ != JFNK_OK) return r_;                \
    } while (0)
