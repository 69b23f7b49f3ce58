// Implicit step (Sec. 2.2) by inexact Jacobian-free Newton-GMRES (Sec. 3.1).
//
// All vectors stay on the device.  Per Arnoldi step the host reads back one
// Hessenberg column (j+2 doubles, one synchronisation) and applies the Givens
// rotations; orthogonalisation is classical Gram-Schmidt applied twice (CGS2:
// two multi-dot passes and two updates), the norm and the normalisation read
// the norm from device memory.  GMRES is right preconditioned and flexible, so
// the nonlinear, reduced-precision preconditioner is allowed.
#include <math.h>
#include <string.h>

#include <chrono>

#include "internal.h"

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// the step's wall-clock budget (opts.time_budget_ms) has run out
bool out_of_time(const jfnk_ctx *c) { return c->deadline > 0.0 && now_s() > c->deadline; }

struct Stats {
    int newton_its = 0, gmres_its = 0;
    double res0 = 0, res_final = 0;
    double t_pre = 0, t_jv = 0, t_orth = 0, t_newton = 0;
    int reortho = 0;
};

// Phase timing with events recorded on the solver's stream; elapsed times are
// read after the synchronisations the solver does anyway.
struct Phases {
    bool on = false;
    cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
    explicit Phases(bool enable) : on(enable) {
        if (on)
            for (auto &x : e)
                if (cudaEventCreate(&x) != cudaSuccess) on = false;
    }
    ~Phases() {
        for (auto &x : e)
            if (x) cudaEventDestroy(x);
    }
    void mark(int i, cudaStream_t s) {
        if (on) cudaEventRecord(e[i], s);
    }
    double ms(int a, int b) {
        float m = 0.f;
        if (on && cudaEventElapsedTime(&m, e[a], e[b]) == cudaSuccess) return m;
        return 0.0;
    }
};

// z_j of the flexible basis as an FP64 pointer; FP32 storage is converted and
// eps of the FD product computed in the same pass (*eps_ready = true)
const double *z_as_double(jfnk_ctx *c, int j, double *tmp, cudaStream_t s, int *rc, bool *eps_ready) {
    *rc = JFNK_OK;
    *eps_ready = false;
    if (c->prec == 64 || !c->mg_on) return (const double *)c->Z + (size_t)j * c->N;
    *rc = blas_f2d_eps(c, (const float *)c->Z + (size_t)j * c->N, tmp, c->N, c->scal + S_EPS, s);
    *eps_ready = true;
    return tmp;
}

// w = G'(U) y with eps = sqrt(eps_mach)/|y| computed on the device (skipped
// when the caller already wrote eps to S_EPS)
int apply_jv(jfnk_ctx *c, const double *U, double adt, const double *y, double *w, cudaStream_t s,
             bool eps_ready = false) {
    if (!eps_ready) JF_RET(red_dot(c, y, y, c->N, c->scal + S_EPS, RED_EPS, s));
    DGArgs a = {};
    a.U = U;
    a.y = y;
    a.fU = c->fU;
    a.eps = c->scal + S_EPS;
    a.adt = adt;
    a.out0 = w;
    a.tr_in = c->tr_valid ? c->trU : nullptr;   // U is the iterate of the last residual
    return dg_apply(c, DG_JV, a, s);
}

int read_norm(jfnk_ctx *c, const double *x, double *out, cudaStream_t s) {
    JF_RET(red_dot(c, x, x, c->N, c->scal + S_NORM, RED_SQRT, s));
    JF_CK(jf_memcpy(c->h_pinned, c->scal + S_NORM, sizeof(double), cudaMemcpyDeviceToHost, s));
    JF_CK(jf_sync(s));
    *out = c->h_pinned[0];
    return JFNK_OK;
}

// Device work of Arnoldi step j: z_j = Q^-1 v_j, w = G'(U) z_j into v_{j+1},
// Gram-Schmidt (second pass decided on the device), normalisation, and the
// copy of the Hessenberg column to pinned host memory.  No host decisions, so
// it can be captured.
int arnoldi_step_work(jfnk_ctx *c, const double *U, double adt, int j, cudaStream_t s, Phases *ph) {
    const size_t N = c->N;
    double *V = c->V;
    double *vj = V + (size_t)j * N, *w = V + (size_t)(j + 1) * N;
    int rc;
    if (ph) ph->mark(0, s);
    if (c->mg_on) {
        JF_RET(mg_apply(c, vj, (char *)c->Z + (size_t)j * N * (c->prec == 64 ? 8 : 4), s,
                        c->prec == 64 ? nullptr : c->V32 + (size_t)j * N));
    } else {
        JF_CK(jf_memcpy((double *)c->Z + (size_t)j * N, vj, 8 * N, cudaMemcpyDeviceToDevice, s));
    }
    bool eps_ready = false;
    const double *zj = z_as_double(c, j, c->w1, s, &rc, &eps_ready);
    JF_RET(rc);
    if (ph) ph->mark(1, s);
    JF_RET(apply_jv(c, U, adt, zj, w, s, eps_ready));
    if (ph) ph->mark(2, s);
    // classical Gram-Schmidt; the update kernel also reduces |w|^2, and a
    // second pass runs only when the first lost more than half of |w|
    // (decided on the device)
    if (j + 1 <= GS_FUSED_MAX && (N & 1) == 0) {
        JF_RET(blas_cgs2(c, V, c->V32, j + 1, N, w, c->V32 + (size_t)(j + 1) * N, N, c->scal + S_H, c->scal + S_H2,
                         c->scal + S_W1, c->scal + S_NORM, c->scal + S_FLAG, s));   // normalises w too
        if (ph) ph->mark(3, s);
        JF_CK(jf_memcpy(c->h_pinned, c->scal, 8 * S_COUNT, cudaMemcpyDeviceToHost, s));
        return JFNK_OK;
    }
    JF_RET(blas_mdot(c, V, j + 1, N, w, N, c->scal + S_H, s));
    JF_RET(blas_mupdate_norm(c, V, j + 1, N, c->scal + S_H, w, N, -1.0, nullptr, c->scal + S_W1,
                             c->scal + S_NORM, c->scal + S_FLAG, s));
    JF_RET(blas_mdot(c, V, j + 1, N, w, N, c->scal + S_H2, s, c->scal + S_FLAG));
    JF_RET(blas_mupdate_norm(c, V, j + 1, N, c->scal + S_H2, w, N, -1.0, c->scal + S_FLAG, nullptr,
                             c->scal + S_NORM, nullptr, s));
    JF_RET(blas_scale_copy(w, c->scal + S_NORM, w, N, s));
    JF_RET(blas_copy_d2f(w, c->V32 + (size_t)(j + 1) * N, N, s));   // float copy of the basis
    if (ph) ph->mark(3, s);
    JF_CK(jf_memcpy(c->h_pinned, c->scal, 8 * S_COUNT, cudaMemcpyDeviceToHost, s));
    return JFNK_OK;
}

// Arnoldi step j, replayed from a graph captured per j (pointers are all
// context-owned: U is the context's copy of the Newton iterate).
int arnoldi_step(jfnk_ctx *c, const double *U, double adt, int j, cudaStream_t s, Phases &ph) {
    const bool graphs = c->opts.use_graphs && !ph.on && U == c->Ulin && j < 64 && !t_jf_rec;
    if (!graphs) return arnoldi_step_work(c, U, adt, j, s, ph.on ? &ph : nullptr);
    if (c->arn_adt != adt) {
        for (int i = 0; i < 64; ++i)
            if (c->arn_valid[i]) {
                cudaGraphExecDestroy(c->arn_graph[i]);
                c->arn_valid[i] = 0;
            }
        c->arn_adt = adt;
    }
    if (!c->arn_valid[j]) {
        std::lock_guard<std::mutex> lock(g_jf_device_mu);   // no device-wide sync during capture
        if (!c->cap_stream) JF_CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        const unsigned long long n0 = t_jf_launches;
        const long long d0 = c->dg_calls, f0 = c->fv_calls;
        JF_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        c->capturing = 1;   // the preconditioner's kernels are captured inline
        const int rc = arnoldi_step_work(c, U, adt, j, c->cap_stream, nullptr);
        c->capturing = 0;
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        c->arn_launches[j] = t_jf_launches - n0;
        __atomic_fetch_sub(&g_jf_launches, c->arn_launches[j], __ATOMIC_RELAXED);
        t_jf_launches = n0;
        c->arn_dg_calls[j] = c->dg_calls - d0;
        c->arn_fv_calls[j] = c->fv_calls - f0;
        c->dg_calls = d0;
        c->fv_calls = f0;
        if (rc != JFNK_OK || e != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc != JFNK_OK ? rc : JFNK_ECUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->arn_graph[j], g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            cudaGetLastError();
            return JFNK_ECUDA;
        }
        c->arn_valid[j] = 1;
    }
    JF_CK(cudaGraphLaunch(c->arn_graph[j], s));
    jf_launched((unsigned)c->arn_launches[j]);
    c->dg_calls += c->arn_dg_calls[j];
    c->fv_calls += c->arn_fv_calls[j];
    return JFNK_OK;
}

// Solve G'(U) x = b from x = 0 until the residual estimate <= tol_abs.
int fgmres(jfnk_ctx *c, const double *U, double adt, const double *b, double *x, double tol_abs, int *its,
           cudaStream_t s, Stats &st) {
    Phases ph(c->opts.profile != 0);
    const size_t N = c->N;
    const int m = c->opts.gmres_restart;
    const int maxit = c->opts.gmres_max;
    double *V = c->V;
    double H[65][64], cs[64], sn[64], g[65], y[64];
    JF_CK(jf_memset(x, 0, 8 * N, s));
    double beta;
    JF_RET(read_norm(c, b, &beta, s));
    if (!isfinite(beta)) return JFNK_ENAN;
    *its = 0;
    if (beta <= tol_abs || beta == 0.0) return JFNK_OK;
    const double *r = b;
    while (*its < maxit) {
        JF_CK(jf_memcpy(c->scal + S_NORM, &beta, sizeof(double), cudaMemcpyHostToDevice, s));
        JF_RET(blas_scale_copy(r, c->scal + S_NORM, V, N, s));
        JF_RET(blas_copy_d2f(V, c->V32, N, s));
        JF_CK(jf_sync(s));   // beta lives on the host stack
        memset(H, 0, sizeof(H));
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int jd = 0;
        bool conv = false;
        for (int j = 0; j < m; ++j) {
            JF_RET(arnoldi_step(c, U, adt, j, s, ph));
            JF_CK(jf_sync(s));
            if (out_of_time(c)) return JFNK_ETIMEOUT;
            st.t_pre += ph.ms(0, 1);
            st.t_jv += ph.ms(1, 2);
            st.t_orth += ph.ms(2, 3);
            const double *hp = c->h_pinned;
            if (hp[S_FLAG] != 0.0) ++st.reortho;
            for (int i = 0; i <= j; ++i) H[i][j] = hp[S_H + i] + (hp[S_FLAG] != 0.0 ? hp[S_H2 + i] : 0.0);
            H[j + 1][j] = hp[S_NORM];
            if (!isfinite(H[j + 1][j])) return JFNK_ENAN;
            for (int i = 0; i < j; ++i) {
                const double a0 = H[i][j], a1 = H[i + 1][j];
                H[i][j] = cs[i] * a0 + sn[i] * a1;
                H[i + 1][j] = -sn[i] * a0 + cs[i] * a1;
            }
            const double den = hypot(H[j][j], H[j + 1][j]);
            if (den == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = H[j][j] / den;
                sn[j] = H[j + 1][j] / den;
            }
            H[j][j] = den;
            H[j + 1][j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++*its;
            jd = j + 1;
            if (fabs(g[j + 1]) <= tol_abs || den == 0.0 || *its >= maxit) {
                conv = fabs(g[j + 1]) <= tol_abs;
                break;
            }
        }
        for (int i = jd - 1; i >= 0; --i) {
            double acc = g[i];
            for (int q = i + 1; q < jd; ++q) acc -= H[i][q] * y[q];
            y[i] = acc / H[i][i];
        }
        for (int i = 0; i < jd; ++i)
            if (!isfinite(y[i])) return JFNK_ENAN;
        JF_RET(blas_zcomb(c->Z, (c->prec != 64 && c->mg_on) ? 1 : 0, jd, N, y, x, s));
        if (conv) return JFNK_OK;
        if (*its >= maxit) return JFNK_ENOTCONV;
        // restart from the true residual r = b - G'x
        JF_RET(apply_jv(c, U, adt, x, c->w2, s));
        JF_RET(blas_axpby(1.0, b, -1.0, c->w2, c->w2, N, s));
        r = c->w2;
        JF_RET(read_norm(c, r, &beta, s));
        if (!isfinite(beta)) return JFNK_ENAN;
        if (beta <= tol_abs) return JFNK_OK;
    }
    return JFNK_ENOTCONV;
}

// G = U - adt f(U) - Ubar_s and f(U) (cached in c->fU); returns |G|
int eval_G(jfnk_ctx *c, const double *U, double adt, double *nrm, cudaStream_t s) {
    DGArgs a = {};
    a.U = U;
    a.Ubs = c->Ubs;
    a.adt = adt;
    a.out0 = c->G;
    a.out1 = c->fU;
    a.tr_out = c->trU;   // the FD products of this Newton iterate reuse its face traces
    JF_RET(dg_apply(c, DG_G, a, s));
    return read_norm(c, c->G, nrm, s);
}

// Newton for G(U) = 0 from U^0 = Ubar_s (U holds Ubar_s on entry).
int newton(jfnk_ctx *c, double *U, double adt, Stats &st, cudaStream_t s) {
    const jfnk_opts &o = c->opts;
    double n0;
    JF_RET(eval_G(c, U, adt, &n0, s));
    st.res0 = n0;
    st.res_final = n0;
    if (!isfinite(n0)) return JFNK_ENAN;
    if (n0 == 0.0) return JFNK_OK;
    double nk = n0, nk_prev = 0.0, eta = o.ew_eta0, eta_prev = 0.0;
    for (int k = 0; k <= o.newton_max; ++k) {
        if (k > 0 && nk < o.newton_tol * n0) return JFNK_OK;
        if (k == o.newton_max) break;
        if (k > 0) {
            // Eisenstat-Walker choice 2 (gamma, alpha), safeguard, cap, oversolve floor
            eta = o.ew_gamma * pow(nk / nk_prev, o.ew_alpha);
            const double sg = o.ew_gamma * pow(eta_prev, o.ew_alpha);
            if (sg > 0.1) eta = fmax(eta, sg);
            eta = fmin(eta, o.ew_eta_max);
            eta = fmax(eta, 0.5 * o.newton_tol * n0 / nk);
        }
        Phases ph(c->opts.profile != 0);
        ph.mark(0, s);
        // the context's copy of U^k: the captured Arnoldi graphs hold this pointer
        if (c->mg_on) JF_RET(mg_linearize(c, U, adt, s));
        else JF_CK(jf_memcpy(c->Ulin, U, 8 * c->N, cudaMemcpyDeviceToDevice, s));
        ph.mark(1, s);
        JF_RET(blas_scale(-1.0, c->G, c->G, c->N, s));
        int its = 0;
        int rc = fgmres(c, c->Ulin, adt, c->G, c->dU, eta * nk, &its, s, st);
        st.gmres_its += its;
        if (rc != JFNK_OK && rc != JFNK_ENOTCONV) return rc;
        JF_RET(blas_axpby(1.0, U, 1.0, c->dU, U, c->N, s));
        ++st.newton_its;
        nk_prev = nk;
        eta_prev = eta;
        ph.mark(2, s);
        JF_RET(eval_G(c, U, adt, &nk, s));   // synchronises
        if (out_of_time(c)) return JFNK_ETIMEOUT;
        ph.mark(3, s);
        if (ph.on) {
            cudaEventSynchronize(ph.e[3]);
            st.t_newton += ph.ms(0, 1) + ph.ms(2, 3);
        }
        st.res_final = nk;
        if (!isfinite(nk)) return JFNK_ENAN;
    }
    return JFNK_ENOTCONV;
}

}  // namespace

extern "C" int implicit_step(jfnk_ctx *c, double *U, double dt, int scheme, jfnk_stats *stats, void *stream) {
    if (!c || !U || !(dt > 0.0) || (scheme != 0 && scheme != 1)) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t N = c->N;
    c->dg_calls = 0;
    c->fv_calls = 0;
    c->deadline = c->opts.time_budget_ms > 0.0 ? now_s() + 1e-3 * c->opts.time_budget_ms : 0.0;
    Stats st;
    int rc = JFNK_OK;
    JF_CK(jf_memcpy(c->Usave, U, 8 * N, cudaMemcpyDeviceToDevice, s));
    JF_CK(jf_memcpy(c->Ubs, U, 8 * N, cudaMemcpyDeviceToDevice, s));
    int stages = 0;
    if (scheme == 0) {
        stages = 1;
        rc = newton(c, U, dt, st, s);
    } else {
        const double a = 1.0 - sqrt(2.0) / 2.0;
        stages = 1;
        rc = newton(c, U, a * dt, st, s);
        if (rc == JFNK_OK) {
            // Ubar_2 = U^n + (1 - alpha) dt f(U_1); f(U_1) is the last residual's f
            stages = 2;
            JF_CK(jf_memcpy(c->w1, c->fU, 8 * N, cudaMemcpyDeviceToDevice, s));
            rc = blas_axpby(1.0, c->Usave, (1.0 - a) * dt, c->w1, c->Ubs, N, s);
            if (rc == JFNK_OK) rc = jf_memcpy(U, c->Ubs, 8 * N, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                                        ? JFNK_OK
                                        : JFNK_ECUDA;
            if (rc == JFNK_OK) rc = newton(c, U, a * dt, st, s);
        }
    }
    if (rc != JFNK_OK && rc != JFNK_ECUDA) {
        jf_memcpy(U, c->Usave, 8 * N, cudaMemcpyDeviceToDevice, s);
        jf_sync(s);
    }
    if (stats) {
        stats->status = rc;
        stats->stages = stages;
        stats->newton_its = st.newton_its;
        stats->gmres_its = st.gmres_its;
        stats->dg_calls = (int)c->dg_calls;
        stats->fv_calls = (int)c->fv_calls;
        stats->res0 = st.res0;
        stats->res_final = st.res_final;
        stats->t_precond_ms = st.t_pre;
        stats->t_jv_ms = st.t_jv;
        stats->t_orth_ms = st.t_orth;
        stats->t_newton_ms = st.t_newton;
        stats->reorth = st.reortho;
    }
    return rc;
}
