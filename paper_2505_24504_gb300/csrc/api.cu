// C-ABI entry points: context life cycle, initial data, residual, products,
// preconditioner and diagnostics.  The implicit step lives in solver.cu.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "internal.h"

void jf_build_tables(int k, DGTab *T);
void jf_build_powtab(double gamma, PowTab *P);
void jf_background(const jfnk_physics *ph, double z, double U[4], double dU[4]);
double jf_insert_coef(const jfnk_physics *ph, double z);
double jf_background_theta(const jfnk_physics *ph, double z);

unsigned long long g_jf_launches = 0;
std::mutex g_jf_device_mu;
thread_local unsigned long long t_jf_launches = 0;

namespace {

struct Allocs {
    std::vector<void *> dev;
    std::vector<void *> host;
};

// all device allocations of a context are recorded for jfnk_destroy
Allocs *allocs_of(jfnk_ctx *c) { return reinterpret_cast<Allocs *>(c->allocs); }

template <class P>
int dalloc(jfnk_ctx *c, P **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return JFNK_OK;
    void *q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return JFNK_ENOMEM;
    }
    allocs_of(c)->dev.push_back(q);
    c->alloc_bytes += bytes;
    *p = (P *)q;
    return JFNK_OK;
}

int parse_key(jfnk_ctx *c, const char *key) {
    if (key == nullptr || key[0] == 0) {
        c->mg_on = 0;
        return JFNK_OK;
    }
    if (strlen(key) != 9 || key[0] != 'm' || key[1] != 'g' || (key[8] != 'V' && key[8] != 'W'))
        return JFNK_EINVAL;
    int d[6];
    for (int i = 0; i < 6; ++i) {
        if (key[2 + i] < '0' || key[2 + i] > '9') return JFNK_EINVAL;
        d[i] = key[2 + i] - '0';
    }
    c->mg_on = 1;
    c->dg_pre = d[0];
    c->dg_post = d[1];
    c->fine_pre = d[2];
    c->fine_post = d[3];
    c->mid_pre = d[4];
    c->mid_post = d[5];
    c->cycles = key[8] == 'V' ? 1 : 2;
    return JFNK_OK;
}

// FV hierarchy: subgrid, then 2x2 steps to the DG grid when k+1 is a power of two
// (else one (k+1)x(k+1) agglomeration), then 2x2 while both counts are even.
int hierarchy(int nx, int nz, int k, int levels, int NX[], int NZ[], int fac[]) {
    const int n1 = k + 1;
    int n = 0;
    NX[0] = nx * n1;
    NZ[0] = nz * n1;
    n = 1;
    if ((n1 & (n1 - 1)) == 0) {
        int r = n1;
        while (r > 1 && n < levels) {
            fac[n - 1] = 2;
            NX[n] = NX[n - 1] / 2;
            NZ[n] = NZ[n - 1] / 2;
            ++n;
            r /= 2;
        }
    } else if (n < levels) {
        fac[n - 1] = n1;
        NX[n] = nx;
        NZ[n] = nz;
        ++n;
    }
    while (n < levels && n < JF_MAXLEV) {
        if (NX[n - 1] % 2 || NZ[n - 1] % 2 || NX[n - 1] < 2 || NZ[n - 1] < 2) break;
        fac[n - 1] = 2;
        NX[n] = NX[n - 1] / 2;
        NZ[n] = NZ[n - 1] / 2;
        ++n;
    }
    fac[n - 1] = 0;
    return n;
}

int check_args(const jfnk_grid *g, int k, const jfnk_physics *p) {
    if (!g || !p) return JFNK_EINVAL;
    if (k < 1 || k > 4) return JFNK_EINVAL;
    if (g->nx < 1 || g->nz < 1 || !(g->x1 > g->x0) || !(g->z1 > g->z0)) return JFNK_EINVAL;
    if (!(p->cp > p->cv) || !(p->cv > 0) || !(p->p0 > 0) || !(p->theta0 > 0) || p->mu < 0) return JFNK_EINVAL;
    if (p->background < 0 || p->background > 2) return JFNK_EINVAL;
    if (p->background == 2 && !(p->N_bv > 0)) return JFNK_EINVAL;
    return JFNK_OK;
}

__global__ void k_eos(const double *E, size_t n, PhysC pc, const PowTab *pt, double *p) {
    __shared__ PowTab spt;
    const double *src = reinterpret_cast<const double *>(pt);
    double *dst = reinterpret_cast<double *>(&spt);
    for (int i = threadIdx.x; i < (int)(sizeof(PowTab) / sizeof(double)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = pressure(D64{E[i]}, pc, &spt).x;
}

__global__ void k_init_state(const double *thp, const double *prow, const double *throw_, const double *ubv,
                             double ubg, double wbg, int nx, int nz, int np1, double *U) {
    const int NP = np1 * np1;
    const size_t N1 = (size_t)nx * nz * NP;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N1) return;
    const int e = (int)(i / NP), node = (int)(i % NP);
    const int J = (e / nx) * np1 + node / np1;
    const size_t nrow = (size_t)nz * np1;
    const double th = throw_[J] + thp[i];
    const double rho = prow[J] / th;
    const double Uv[4] = {rho, rho * ubg, rho * wbg, rho * th};
    for (int v = 0; v < 4; ++v) U[v * N1 + i] = Uv[v] - ubv[v * nrow + J];
}

size_t workspace(const jfnk_grid *g, int k, const jfnk_opts *o, const jfnk_physics *ph, int *nlev_out) {
    const int n1 = k + 1;
    const size_t npt = (size_t)g->nx * g->nz * n1 * n1, N = 4 * npt;
    const int m = o->gmres_restart;
    const int prec = o->precond_prec;
    const size_t sS = prec == 64 ? 8 : 4;
    size_t b = 0;
    b += sizeof(PowTab);
    const size_t nrow = (size_t)g->nz * n1;
    b += 8 * (4 * nrow * 6 + 4 * (size_t)(g->nz + 1) * 3 + nrow * 2);
    const size_t fx = (size_t)g->nz * (g->nx + 1) * n1, fz = (size_t)(g->nz + 1) * g->nx * n1;
    const bool visc = ph ? ph->mu != 0.0 : true;
    b += 8 * (4 + (visc ? 6 : 0)) * (fx + fz);
    if (prec != 64) b += 4 * (4 + (visc ? 6 : 0)) * (fx + fz);
    b += 8 * N * 9;                        // DG work vectors
    b += 12 * N * (size_t)(m + 1);         // V and its float copy
    const bool mg_on = o->mg_key[0] != 0;
    b += ((prec == 64 || !mg_on) ? 8 : 4) * N * (size_t)m;   // Z
    b += sS * N * 6;                       // pz, pz2, pd, pr, pin, pout
    b += 8 * (size_t)g->nx * g->nz;        // dtau_dg
    int NX[JF_MAXLEV], NZ[JF_MAXLEV], fac[JF_MAXLEV];
    const int nl = hierarchy(g->nx, g->nz, k, o->fv_levels < 1 ? 1 : o->fv_levels, NX, NZ, fac);
    for (int l = 0; l < nl; ++l) {
        const size_t n = 4 * (size_t)NX[l] * NZ[l];
        b += 8 * (4 * (size_t)NZ[l] * 4 + 4);
        b += sS * n * 6 + sS * n / 4;
    }
    b += 8 * 4096 * 32 + 8 * 256;
    b += 8 * (fx + fz) * (visc ? 16 : 8);   // face traces of the Newton iterate
    if (nlev_out) *nlev_out = nl;
    return b;
}

}  // namespace

extern "C" {

void jfnk_default_opts(jfnk_opts *o) {
    memset(o, 0, sizeof(*o));
    o->newton_tol = 1e-8;
    o->newton_max = 20;
    o->gmres_restart = 30;
    o->gmres_max = 300;
    o->ew_gamma = 0.1;
    o->ew_alpha = 1.0;
    o->ew_eta0 = 0.1;
    o->ew_eta_max = 0.9;
    strcpy(o->mg_key, "mg111111V");
    o->fv_levels = 3;
    o->massfix = 1;
    o->transfer_l2 = 0;
    o->precond_prec = 64;
    o->sigma_fv = 1.0;
    o->sigma_dg = 1.0;
    o->c_ip = 2.0;
    o->use_graphs = 1;
    o->tile_faces = 128;
    o->tile_volume = 2;
    o->tile_fv = 128;
    o->fv_split_cells = 0;
    o->rk_stages = 1;
    o->rk_alpha[0] = 1.0;
}

const char *jfnk_strerror(int code) {
    switch (code) {
        case JFNK_OK: return "ok";
        case JFNK_EINVAL: return "invalid argument";
        case JFNK_ENOMEM: return "device allocation failed";
        case JFNK_ECUDA: return "CUDA error";
        case JFNK_ENOTCONV: return "Newton or GMRES did not converge within the iteration caps";
        case JFNK_ETIMEOUT: return "the implicit step's time budget ran out";
        case JFNK_ENAN: return "non-finite norm";
    }
    return "unknown error";
}

size_t jfnk_workspace_bytes(const jfnk_grid *g, int k, const jfnk_opts *opts) {
    jfnk_opts o;
    if (opts) o = *opts;
    else jfnk_default_opts(&o);
    if (!g || k < 1 || k > 4 || g->nx < 1 || g->nz < 1) return 0;
    return workspace(g, k, &o, nullptr, nullptr);
}

static void destroy_unlocked(jfnk_ctx *c);

void jfnk_destroy(jfnk_ctx *c) {
    if (!c) return;
    std::lock_guard<std::mutex> lock(g_jf_device_mu);
    destroy_unlocked(c);
}

static void destroy_unlocked(jfnk_ctx *c) {
    if (!c) return;
    jf_invalidate_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    Allocs *a = allocs_of(c);
    if (a) {
        for (void *p : a->dev) cudaFree(p);
        for (void *p : a->host) cudaFreeHost(p);
        delete a;
    }
    free(c);
}

static int create_locked(const jfnk_grid *g, int k, const jfnk_physics *ph, const jfnk_opts *opts,
                         jfnk_ctx **out);

int jfnk_create(const jfnk_grid *g, int k, const jfnk_physics *ph, const jfnk_opts *opts, jfnk_ctx **out) {
    std::unique_lock<std::mutex> lock(g_jf_device_mu);
    return create_locked(g, k, ph, opts, out);
}

static int create_locked(const jfnk_grid *g, int k, const jfnk_physics *ph, const jfnk_opts *opts,
                         jfnk_ctx **out) {
    if (!out) return JFNK_EINVAL;
    *out = nullptr;
    JF_RET(check_args(g, k, ph));
    jfnk_opts o;
    if (opts) o = *opts;
    else jfnk_default_opts(&o);
    if (o.gmres_restart < 1 || o.gmres_restart > 64 || o.gmres_max < 1 || o.newton_max < 1) return JFNK_EINVAL;
    if (o.precond_prec != 64 && o.precond_prec != 32 && o.precond_prec != 16) return JFNK_EINVAL;
    if (!(o.precond_fd_eps >= 0.0) || !(o.time_budget_ms >= 0.0)) return JFNK_EINVAL;
    if (o.dg_fused < 0 || o.dg_fused > 2) return JFNK_EINVAL;
    if (o.rk_stages == 0) {   // zero-filled options: the explicit Euler smoother
        o.rk_stages = 1;
        o.rk_alpha[0] = 1.0;
    }
    if (o.rk_stages < 1 || o.rk_stages > 4) return JFNK_EINVAL;
    for (int k = 0; k < o.rk_stages; ++k)
        if (!(o.rk_alpha[k] > 0.0)) return JFNK_EINVAL;
    if (o.fv_levels < 1) o.fv_levels = 1;
    if (o.tile_faces == 0) o.tile_faces = 128;
    if (o.tile_volume == 0) o.tile_volume = 2;
    if (o.tile_fv == 0) o.tile_fv = 128;
    if ((o.tile_faces != 64 && o.tile_faces != 128 && o.tile_faces != 256) ||
        (o.tile_volume != 1 && o.tile_volume != 2) ||
        (o.tile_fv != 64 && o.tile_fv != 128 && o.tile_fv != 256))
        return JFNK_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return JFNK_ECUDA;
    }
    jfnk_ctx *c = (jfnk_ctx *)calloc(1, sizeof(jfnk_ctx));
    if (!c) return JFNK_ENOMEM;
    Allocs *al = new (std::nothrow) Allocs();
    if (!al) {
        free(c);
        return JFNK_ENOMEM;
    }
    c->allocs = al;
    c->grid = *g;
    c->k = k;
    c->np1 = k + 1;
    c->n_el = g->nx * g->nz;
    c->phys = *ph;
    c->opts = o;
    c->npt = (size_t)c->n_el * c->np1 * c->np1;
    c->N = 4 * c->npt;
    c->hx = (g->x1 - g->x0) / g->nx;
    c->hz = (g->z1 - g->z0) / g->nz;
    c->dev = dev;
    c->prec = o.precond_prec;
    int rc = parse_key(c, o.mg_key);
    if (rc) {
        destroy_unlocked(c);
        return rc;
    }
    const double R = ph->cp - ph->cv;
    c->pc.gamma = ph->cp / ph->cv;
    c->pc.R = R;
    c->pc.p0 = ph->p0;
    c->pc.g = ph->g;
    c->pc.mu = ph->mu;
    c->pc.R_over_p0 = R / ph->p0;
    c->pc.gammaf = (float)c->pc.gamma;
    c->pc.p0f = (float)c->pc.p0;
    c->pc.R_over_p0f = (float)c->pc.R_over_p0;
    c->pc.muf = (float)c->pc.mu;
    jf_build_tables(k, &c->tab);
    // Set-up copies and kernels run on a private stream that only this call
    // waits for: creating a context never drains other threads' streams.
    struct SetupStream {
        cudaStream_t s = nullptr;
        ~SetupStream() {
            if (s) cudaStreamDestroy(s);
        }
    } setup;
    if (cudaStreamCreateWithFlags(&setup.s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        destroy_unlocked(c);
        return JFNK_ECUDA;
    }
    const cudaStream_t ss = setup.s;
    auto h2d = [ss](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ss) == cudaSuccess;
    };

#define A_(p, bytes)                         \
    do {                                     \
        rc = dalloc(c, &(p), (bytes));       \
        if (rc) {                            \
            destroy_unlocked(c);                 \
            return rc;                       \
        }                                    \
    } while (0)

    const int n1 = c->np1;
    const size_t nrow = (size_t)g->nz * n1;
    const size_t nf = (size_t)g->nz + 1;
    A_(c->powtab, sizeof(PowTab));
    A_(c->ubv, 8 * 4 * nrow);
    A_(c->dubv, 8 * 4 * nrow);
    A_(c->fbx, 8 * 4 * nrow);
    A_(c->fbz, 8 * 4 * nrow);
    A_(c->hbx, 8 * 4 * nrow);
    A_(c->hbxw, 8 * 8 * nrow);
    A_(c->ubh, 8 * 4 * nf);
    A_(c->dubh, 8 * 4 * nf);
    A_(c->hbz, 8 * 4 * nf);
    A_(c->prow, 8 * nrow);
    A_(c->theta_row, 8 * nrow);
    // host copies of the background (node rows and horizontal faces), kept for
    // the FP32 copies below
    std::vector<double> ub(4 * nrow), dub(4 * nrow), uh(4 * nf), duh(4 * nf);
    PowTab pt;
    {
        jf_build_powtab(c->pc.gamma, &pt);
        std::vector<double> pr(nrow), tr(nrow);
        for (int ez = 0; ez < g->nz; ++ez)
            for (int b = 0; b < n1; ++b) {
                const int J = ez * n1 + b;
                const double z = g->z0 + (ez + 0.5 * (1.0 + c->tab.xi[b])) * c->hz;
                double U[4], dU[4];
                jf_background(ph, z, U, dU);
                for (int v = 0; v < 4; ++v) {
                    ub[v * nrow + J] = U[v];
                    dub[v * nrow + J] = dU[v];
                }
                pr[J] = jf_insert_coef(ph, z);
                tr[J] = jf_background_theta(ph, z);
            }
        for (int j = 0; j < (int)nf; ++j) {
            double U[4], dU[4];
            jf_background(ph, g->z0 + j * c->hz, U, dU);
            for (int v = 0; v < 4; ++v) {
                uh[v * nf + j] = U[v];
                duh[v * nf + j] = dU[v];
            }
        }
        // pageable sources: each copy has read its source when it returns
        if (!h2d(c->powtab, &pt, sizeof(pt)) || !h2d(c->ubv, ub.data(), 8 * ub.size()) ||
            !h2d(c->dubv, dub.data(), 8 * dub.size()) || !h2d(c->ubh, uh.data(), 8 * uh.size()) ||
            !h2d(c->dubh, duh.data(), 8 * duh.size()) || !h2d(c->prow, pr.data(), 8 * pr.size()) ||
            !h2d(c->theta_row, tr.data(), 8 * tr.size())) {
            cudaGetLastError();
            destroy_unlocked(c);
            return JFNK_ECUDA;
        }
    }
    const bool visc = ph->mu != 0.0;
    const size_t fx = (size_t)g->nz * (g->nx + 1) * n1, fz = (size_t)(g->nz + 1) * g->nx * n1;
    A_(c->phix, 8 * 4 * fx);
    A_(c->phiz, 8 * 4 * fz);
    if (visc) {
        A_(c->symx, 8 * 6 * fx);
        A_(c->symz, 8 * 6 * fz);
    }
    if (c->prec != 64) {
        A_(c->phixf, 4 * 4 * fx);
        A_(c->phizf, 4 * 4 * fz);
        if (visc) {
            A_(c->symxf, 4 * 6 * fx);
            A_(c->symzf, 4 * 6 * fz);
        }
    }
    const size_t N = c->N;
    A_(c->fU, 8 * N);
    A_(c->w1, 8 * N);
    A_(c->w2, 8 * N);
    A_(c->Ubs, 8 * N);
    A_(c->Un, 8 * N);
    A_(c->Usave, 8 * N);
    A_(c->G, 8 * N);
    A_(c->dU, 8 * N);
    A_(c->Ulin, 8 * N);
    const int m = o.gmres_restart;
    const size_t sS = c->prec == 64 ? 8 : 4;
    // FGMRES stores z_j = Q^-1 v_j in the preconditioner's precision; without a
    // preconditioner z_j = v_j is copied in FP64
    const size_t sZ = (c->prec == 64 || !c->mg_on) ? 8 : 4;
    A_(c->V, 8 * N * (size_t)(m + 1));
    A_(c->V32, 4 * N * (size_t)(m + 1));
    A_(c->Z, sZ * N * (size_t)m);
    A_(c->pz, sS * N);
    A_(c->pz2, sS * N);
    A_(c->pd, sS * N);
    A_(c->pr, sS * N);
    A_(c->pin, sS * N);
    A_(c->pout, sS * N);
    A_(c->dtau_dg, 8 * (size_t)c->n_el);
    if (c->prec != 64) {
        A_(c->dtau_dgf, 4 * (size_t)c->n_el);
        A_(c->Usf, 4 * N);
        A_(c->ubvf, 4 * 4 * nrow);
        A_(c->dubvf, 4 * 4 * nrow);
        A_(c->ubhf, 4 * 4 * nf);
        A_(c->dubhf, 4 * 4 * nf);
        std::vector<float> a1(ub.begin(), ub.end()), a2(dub.begin(), dub.end());
        std::vector<float> a3(uh.begin(), uh.end()), a4(duh.begin(), duh.end());
        if (!h2d(c->ubvf, a1.data(), 4 * a1.size()) || !h2d(c->dubvf, a2.data(), 4 * a2.size()) ||
            !h2d(c->ubhf, a3.data(), 4 * a3.size()) || !h2d(c->dubhf, a4.data(), 4 * a4.size())) {
            cudaGetLastError();
            destroy_unlocked(c);
            return JFNK_ECUDA;
        }
    }
    // FV levels
    int NX[JF_MAXLEV], NZ[JF_MAXLEV], fac[JF_MAXLEV];
    c->nlev = hierarchy(g->nx, g->nz, k, o.fv_levels, NX, NZ, fac);
    for (int l = 0; l < c->nlev; ++l) {
        FVLev &L = c->lev[l];
        L.NX = NX[l];
        L.NZ = NZ[l];
        L.fac = fac[l];
        L.Hx = (g->x1 - g->x0) / NX[l];
        L.Hz = (g->z1 - g->z0) / NZ[l];
        L.n = 4 * (size_t)NX[l] * NZ[l];
        A_(L.ub, 8 * 4 * (size_t)NZ[l]);
        A_(L.ubf, 4 * 4 * (size_t)NZ[l]);
        A_(L.hbx, 8 * 4 * (size_t)NZ[l]);
        A_(L.hbxw, 8 * 8 * (size_t)NZ[l]);
        A_(L.hbz, 8 * 4 * (size_t)(NZ[l] + 1));
        A_(L.u, sS * L.n);
        A_(L.fu, 8 * L.n);
        A_(L.x, sS * L.n);
        A_(L.x2, sS * L.n);
        A_(L.b, sS * L.n);
        A_(L.r, sS * L.n);
        A_(L.dtau, sS * L.n / 4);
        std::vector<double> ub(4 * (size_t)NZ[l]);
        for (int J = 0; J < NZ[l]; ++J) {
            double U[4], dU[4];
            jf_background(ph, g->z0 + (J + 0.5) * L.Hz, U, dU);
            for (int v = 0; v < 4; ++v) ub[v * NZ[l] + J] = U[v];
        }
        std::vector<float> ubf(ub.begin(), ub.end());
        if (!h2d(L.ub, ub.data(), 8 * ub.size()) || !h2d(L.ubf, ubf.data(), 4 * ubf.size())) {
            cudaGetLastError();
            destroy_unlocked(c);
            return JFNK_ECUDA;
        }
    }
    c->nb_red = 4096;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            cudaGetLastError();
            destroy_unlocked(c);
            return JFNK_ECUDA;
        }
        c->n_sm = nsm;
    }
    A_(c->partial, 8 * (size_t)c->nb_red * 32);
    {
        const size_t nfp = (size_t)g->nz * (g->nx + 1) * c->np1 + (size_t)(g->nz + 1) * g->nx * c->np1;
        A_(c->trU, 8 * nfp * (ph->mu != 0.0 ? 16 : 8));
        c->tr_valid = 0;
    }
    A_(c->scal, 8 * (size_t)S_COUNT);
    A_(c->ticket, 256);
    {
        void *h = nullptr;
        if (cudaMallocHost(&h, 8 * (size_t)S_COUNT) != cudaSuccess) {
            cudaGetLastError();
            destroy_unlocked(c);
            return JFNK_ENOMEM;
        }
        allocs_of(c)->host.push_back(h);
        c->h_pinned = (double *)h;
    }
#undef A_
    if (cudaMemsetAsync(c->scal, 0, 8 * (size_t)S_COUNT, ss) != cudaSuccess ||
        cudaMemsetAsync(c->ticket, 0, 256, ss) != cudaSuccess) {
        cudaGetLastError();
        destroy_unlocked(c);
        return JFNK_ECUDA;
    }
    rc = dg_setup_background(c, ss);
    if (!rc) rc = fv_setup_background(c, ss);
    if (!rc && cudaStreamSynchronize(ss) != cudaSuccess) {
        cudaGetLastError();
        rc = JFNK_ECUDA;
    }
    if (rc) {
        destroy_unlocked(c);
        return rc;
    }
    *out = c;
    return JFNK_OK;
}

size_t jfnk_num_unknowns(const jfnk_ctx *c) { return c ? c->N : 0; }

int jfnk_node_coords(const jfnk_ctx *c, double *x, double *z) {
    if (!c || !x || !z) return JFNK_EINVAL;
    const int n1 = c->np1, NP = n1 * n1;
    for (int e = 0; e < c->n_el; ++e) {
        const int ez = e / c->grid.nx, ex = e % c->grid.nx;
        for (int node = 0; node < NP; ++node) {
            const int a = node % n1, b = node / n1;
            x[(size_t)e * NP + node] = c->grid.x0 + (ex + 0.5 * (1.0 + c->tab.xi[a])) * c->hx;
            z[(size_t)e * NP + node] = c->grid.z0 + (ez + 0.5 * (1.0 + c->tab.xi[b])) * c->hz;
        }
    }
    return JFNK_OK;
}

int jfnk_init_state(jfnk_ctx *c, const double *thp, double *U, void *stream) {
    if (!c || !thp || !U) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const double ubg = c->phys.background >= 1 ? c->phys.ubg : 0.0;
    const double wbg = c->phys.background == 1 ? c->phys.wbg : 0.0;
    k_init_state<<<(unsigned)((c->npt + 255) / 256), 256, 0, s>>>(thp, c->prow, c->theta_row, c->ubv, ubg, wbg,
                                                                   c->grid.nx, c->grid.nz, c->np1, U); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int dg_residual(jfnk_ctx *c, const double *U, double *f, void *stream) {
    if (!c || !U || !f || U == f) return JFNK_EINVAL;
    DGArgs a = {};
    a.U = U;
    a.out0 = f;
    return dg_apply(c, DG_RES, a, (cudaStream_t)stream);
}

int jv_product(jfnk_ctx *c, const double *U, const double *fU, const double *y, double adt, double eps,
               double *Jy, void *stream) {
    if (!c || !U || !y || !Jy || Jy == U || Jy == y || (fU && Jy == fU)) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (!fU) {
        DGArgs a = {};
        a.U = U;
        a.out0 = c->fU;
        JF_RET(dg_apply(c, DG_RES, a, s));
        fU = c->fU;
    }
    double *epsp = c->scal + S_EPS;
    if (eps > 0.0) {
        JF_CK(cudaMemcpyAsync(epsp, &eps, sizeof(double), cudaMemcpyHostToDevice, s));
        JF_CK(cudaStreamSynchronize(s));   // eps lives on the caller's stack
    } else {
        JF_RET(red_dot(c, y, y, c->N, epsp, RED_EPS, s));
    }
    DGArgs a = {};
    a.U = U;
    a.y = y;
    a.fU = fU;
    a.eps = epsp;
    a.adt = adt;
    a.out0 = Jy;
    return dg_apply(c, DG_JV, a, s);
}

int mg_precondition(jfnk_ctx *c, const double *U, double adt, const double *r, double *z, void *stream) {
    if (!c || !U || !r || !z || z == U || z == r) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (!c->mg_on) {
        JF_CK(cudaMemcpyAsync(z, r, 8 * c->N, cudaMemcpyDeviceToDevice, s));
        return JFNK_OK;
    }
    DGArgs a = {};
    a.U = U;
    a.out0 = c->fU;
    JF_RET(dg_apply(c, DG_RES, a, s));
    JF_RET(mg_linearize(c, U, adt, s));
    if (c->prec == 64) return mg_apply(c, r, z, s);
    JF_RET(mg_apply(c, r, c->Z, s));
    return blas_copy_f2d((const float *)c->Z, z, c->N, s);
}

int jfnk_norm2(jfnk_ctx *c, const double *x, size_t n, double *out, void *stream) {
    if (!c || !out || (n > 0 && !x)) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        JF_CK(cudaMemsetAsync(out, 0, sizeof(double), s));
        return JFNK_OK;
    }
    return red_dot(c, x, x, n, out, RED_SQRT, s);
}

int jfnk_eos_pressure(jfnk_ctx *c, const double *E, size_t n, double *p, void *stream) {
    if (!c || !E || !p) return JFNK_EINVAL;
    if (n == 0) return JFNK_OK;
    k_eos<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(E, n, c->pc, c->powtab, p); jf_launched();
    JF_CK(cudaGetLastError());
    return JFNK_OK;
}

int jfnk_fv_levels(const jfnk_ctx *c) { return c ? c->nlev : 0; }

int jfnk_tangent_product(jfnk_ctx *c, const double *U, const double *y, double adt, double *out, void *stream) {
    if (!c || !U || !y || !out || c->prec == 64) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    JF_RET(blas_copy_d2f(y, (float *)c->pz, c->N, s));
    JF_RET(blas_copy_d2f(U, c->Usf, c->N, s));
    DGArgs a = {};
    a.U = U;
    a.Uf = c->Usf;
    a.yf = (const float *)c->pz;
    a.adt = adt;
    a.out0 = c->pz2;
    JF_RET(dg_apply(c, DG_TLJV, a, s));
    return blas_copy_f2d((const float *)c->pz2, out, c->N, s);
}

int jfnk_time_operator(jfnk_ctx *c, int which, const double *U, const double *y, int reps, double *ms,
                       void *stream) {
    if (!c || !U || !ms || reps < 1 || which < 0 || which > 4 || (which > 0 && which != 4 && !y)) return JFNK_EINVAL;
    if ((which == 2 || which == 3) && c->prec == 64) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (which == 3) return mg_time_fv_level0(c, U, y, reps, ms, s);
    if (which == 4) return blas_time_cgs2(c, reps, ms, s);
    for (int i = 0; i < 3; ++i) JF_CK(cudaEventCreate(&c->tev[i]));
    int rc = JFNK_OK;
    DGArgs a = {};
    a.U = U;
    a.adt = 1.0;
    if (which == 1) {
        // f(U), its face traces and eps once, outside the timed launches; the timed
        // products take the form the solver's Arnoldi steps use (stored traces of U)
        a.out0 = c->fU;
        a.tr_out = c->trU;
        rc = dg_apply(c, DG_RES, a, s);
        a.tr_out = nullptr;
        if (!rc) rc = red_dot(c, y, y, c->N, c->scal + S_EPS, RED_EPS, s);
        a.y = y;
        a.fU = c->fU;
        a.eps = c->scal + S_EPS;
        a.tr_in = c->trU;
    }
    if (which == 2) {
        rc = blas_copy_d2f(y, (float *)c->pz, c->N, s);
        if (!rc) rc = blas_copy_d2f(U, c->Usf, c->N, s);
        a.yf = (const float *)c->pz;
        a.Uf = c->Usf;
    }
    a.out0 = which == 2 ? (void *)c->pz2 : (void *)c->w2;
    c->t_faces_ms = c->t_volume_ms = 0.0;
    c->timing = 1;
    for (int r = 0; r < reps && rc == JFNK_OK; ++r)
        rc = dg_apply(c, which == 0 ? DG_RES : (which == 1 ? DG_JV : DG_TLJV), a, s);
    c->timing = 0;
    for (int i = 0; i < 3; ++i) cudaEventDestroy(c->tev[i]);
    ms[0] = c->t_faces_ms / reps;
    ms[1] = c->t_volume_ms / reps;
    return rc;
}

int jfnk_autotune(jfnk_ctx *c, const double *U, const double *y, int reps, int *best, double *ms, void *stream) {
    if (!c || !U || !y || !best || !ms || reps < 1) return JFNK_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int keep_f = c->opts.tile_faces, keep_v = c->opts.tile_volume, keep_fv = c->opts.tile_fv;
    const int keep_sp = c->opts.fv_split_cells;
    jf_invalidate_graphs(c);   // captured graphs hold the old launch shapes
    double best_dg = 1e300;
    int bf = keep_f, bv = keep_v;
    const int fs[3] = {64, 128, 256}, vs[2] = {1, 2};
    for (int fi = 0; fi < 3; ++fi)
        for (int vi = 0; vi < 2; ++vi) {
            c->opts.tile_faces = fs[fi];
            c->opts.tile_volume = vs[vi];
            double t[2];
            int rc = jfnk_time_operator(c, 1, U, y, reps + 1, t, stream);   // first rep warms up
            if (rc) {
                c->opts.tile_faces = keep_f;
                c->opts.tile_volume = keep_v;
                return rc;
            }
            if (t[0] + t[1] < best_dg) {
                best_dg = t[0] + t[1];
                bf = fs[fi];
                bv = vs[vi];
            }
        }
    c->opts.tile_faces = bf;
    c->opts.tile_volume = bv;
    double best_mg = 0.0;
    int bfv = keep_fv, bsp = keep_sp;
    if (c->mg_on) {
        cudaEvent_t e0, e1;
        JF_CK(cudaEventCreate(&e0));
        JF_CK(cudaEventCreate(&e1));
        DGArgs a = {};
        a.U = U;
        a.out0 = c->fU;
        int rc = dg_apply(c, DG_RES, a, s);
        if (!rc) rc = mg_linearize(c, U, 1.0, s);
        best_mg = 1e300;
        // split thresholds: never, between the level sizes a 2x2 hierarchy gives, always
        const int sps[5] = {1, 4096, 16384, 65536, 1 << 30};
        for (int it = 0; it < 15 && rc == JFNK_OK; ++it) {
            const int t = 64 << (it % 3), sp = sps[it / 3];
            c->opts.tile_fv = t;
            c->opts.fv_split_cells = sp;
            if (c->mg_graph_valid) {   // the graph holds the old launch shapes
                cudaGraphExecDestroy(c->mg_graph);
                c->mg_graph_valid = 0;
            }
            rc = mg_apply(c, y, c->Z, s);   // warm up (and capture)
            if (rc) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && rc == JFNK_OK; ++r) rc = mg_apply(c, y, c->Z, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            if (m / reps < best_mg) {
                best_mg = m / reps;
                bfv = t;
                bsp = sp;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (c->mg_graph_valid) {
            cudaGraphExecDestroy(c->mg_graph);
            c->mg_graph_valid = 0;
        }
        if (rc) {
            c->opts.tile_fv = keep_fv;
            c->opts.fv_split_cells = keep_sp;
            return rc;
        }
    }
    c->opts.tile_fv = bfv;
    c->opts.fv_split_cells = bsp;
    jf_invalidate_graphs(c);
    best[0] = bf;
    best[1] = bv;
    best[2] = bfv;
    best[3] = bsp;
    ms[0] = best_dg;
    ms[1] = c->mg_on ? best_mg : 0.0;
    return JFNK_OK;
}

unsigned long long jfnk_launch_count(void) { return __atomic_load_n(&g_jf_launches, __ATOMIC_RELAXED); }

int jfnk_fv_level_size(const jfnk_ctx *c, int l, int *NX, int *NZ) {
    if (!c || l < 0 || l >= c->nlev || !NX || !NZ) return JFNK_EINVAL;
    *NX = c->lev[l].NX;
    *NZ = c->lev[l].NZ;
    return JFNK_OK;
}

int jfnk_transfer_to_fv(jfnk_ctx *c, const double *u, double *v, void *stream) {
    if (!c || !u || !v) return JFNK_EINVAL;
    return transfer_to_fv64(c, u, v, (cudaStream_t)stream);
}

int jfnk_transfer_to_dg(jfnk_ctx *c, const double *v, double *u, void *stream) {
    if (!c || !u || !v) return JFNK_EINVAL;
    return transfer_to_dg64(c, v, u, 0, (cudaStream_t)stream);
}

int jfnk_fv_residual(jfnk_ctx *c, int l, const double *u, double *f, void *stream) {
    if (!c || !u || !f || l < 0 || l >= c->nlev) return JFNK_EINVAL;
    return fv_rhs64(c, l, u, f, (cudaStream_t)stream);
}

}  // extern "C"
