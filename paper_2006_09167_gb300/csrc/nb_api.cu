// C ABI of libnb: context management, argument checking and call sequencing.
// Every entry point validates its arguments on the host before touching the
// GPU; launch-time CUDA errors are returned as NB_ERR_CUDA.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "nb_internal.cuh"

nb_status nb_launch_grid_sort_phase1(nb_ctx *c, const float *x, cudaStream_t st);
nb_status nb_launch_grid_sort_phase2(nb_ctx *c, int max_col, cudaStream_t st);
int nb_search_units(const nb_ctx *c);  // search units (super-cluster, column segment) of the next build
nb_status nb_launch_search_count(nb_ctx *c, float rlist, cudaStream_t st);
nb_status nb_launch_search_write(nb_ctx *c, float rlist, cudaStream_t st);

nb_status nb_cuda_status(cudaError_t e) {
    (void)cudaGetLastError();  // clear the sticky-free error state of the runtime
    return e == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

namespace {

template <typename T>
nb_status dalloc(T **p, size_t n) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void **)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return nb_cuda_status(e);
    }
    return NB_OK;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

bool finite_pos(double v) { return isfinite(v) && v > 0.0; }

// Pair tables from C6/C12 (pair parameter = (C[a][b] + C[b][a]) / 2): the force
// table holds (6 C6, 12 C12), the energy table (C6, C12, C12/rc^12 - C6/rc^6, 0)
// with the shift formed in FP64 and rounded once.
__host__ __device__ inline void lj_entry(float c6ab, float c6ba, float c12ab, float c12ba, double rc6inv,
                                         float2 &f, float4 &e) {
    float s6 = 0.5f * (c6ab + c6ba);
    float s12 = 0.5f * (c12ab + c12ba);
    f = make_float2(6.0f * s6, 12.0f * s12);
    double sh = (double)s12 * rc6inv * rc6inv - (double)s6 * rc6inv;
    e = make_float4(s6, s12, (float)sh, 0.f);
}

__global__ void k_set_lj(int T, const float *__restrict__ c6, const float *__restrict__ c12, double rc6inv,
                         float2 *__restrict__ lj, float4 *__restrict__ lje) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T * T) return;
    int a = t / T, b = t % T;
    lj_entry(c6[a * T + b], c6[b * T + a], c12[a * T + b], c12[b * T + a], rc6inv, lj[t], lje[t]);
}

// entry (a, b0, b1) of the T^3 tables: the parameters of the pairs (a, b0) and (a, b1)
__host__ __device__ inline void l3_entry(int T, int t, const float2 *lj, const float4 *lje, float4 &f, float4 &e,
                                         float2 &sh) {
    const int a = t / (T * T), b0 = (t / T) % T, b1 = t % T;
    const float2 f0 = lj[a * T + b0], f1 = lj[a * T + b1];
    const float4 e0 = lje[a * T + b0], e1 = lje[a * T + b1];
    f = make_float4(f0.x, f1.x, f0.y, f1.y);
    e = make_float4(e0.x, e1.x, e0.y, e1.y);
    sh = make_float2(e0.z, e1.z);
}

__global__ void k_set_l3(int T, const float2 *__restrict__ lj, const float4 *__restrict__ lje, float4 *__restrict__ l3f,
                         float4 *__restrict__ l3e, float2 *__restrict__ l3s) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < T * T * T) l3_entry(T, t, lj, lje, l3f[t], l3e[t], l3s[t]);
}

__global__ void k_set_q(int n, const float *__restrict__ q, float *__restrict__ qd, const int *__restrict__ perm,
                        int nslots, float *__restrict__ q_s, float4 *__restrict__ xq) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) qd[t] = q[t];
    if (perm && t < nslots) {
        int i = perm[t];
        float v = i >= 0 ? q[i] : 0.f;
        q_s[t] = v;
        xq[t].w = v;
    }
}

}  // namespace

nbk::SysView nb_make_view(const nb_ctx *c, float4 *f, double *e, double *vir) {
    nbk::SysView v;
    v.xq = nb_cur_xq(c);
    v.type = c->type_s;
    v.items = c->items;
    v.inner_len = c->inner_len;
    v.cj = c->cj_inner;
    v.masks = c->masks;
    v.mask_lanes = c->mask_lanes;
    v.lj = c->lj;
    v.lje = c->lje;
    v.l3f = c->l3f;
    v.l3e = c->l3e;
    v.l3s = c->l3s;
    v.f = f;
    v.e = e;
    v.vir = vir;
    v.n_items = c->n_items;
    v.T = c->T;
    for (int k = 0; k < 3; k++) {
        v.box_hi[k] = (float)c->box[k];
        v.box_lo[k] = (float)(c->box[k] - (double)v.box_hi[k]);
    }
    v.rc2 = (float)(c->rc * c->rc);
    v.coul_f = (float)(138.935458 / c->eps_r);
    v.coul_f64 = 138.935458 / c->eps_r;
    double rc3 = c->rc * c->rc * c->rc;
    double krf = (!isfinite(c->eps_rf) || c->eps_rf <= 0.0) ? 1.0 / (2.0 * rc3)
                                                            : (c->eps_rf - c->eps_r) / ((2.0 * c->eps_rf + c->eps_r) * rc3);
    v.k_rf = (float)krf;
    double crf = 1.0 / c->rc + krf * c->rc * c->rc;
    v.c_rf = (float)crf;
    v.c_rf_lo = (float)(crf - (double)v.c_rf);
    v.ew_s = (float)(c->beta * c->beta / (double)(NB_EW_ZMAX_D * NB_EW_ZMAX_D));
    v.ew_beta3 = (float)(c->beta * c->beta * c->beta);
    v.ew_beta = (float)c->beta;
    v.ew_shift = c->coulomb == NB_COULOMB_EWALD ? (float)(erfc(c->beta * c->rc) / c->rc) : 0.f;  // no f
    double rc6 = 1.0 / (rc3 * rc3);
    v.rc6inv = (float)rc6;
    v.rc12inv = (float)(rc6 * rc6);
    v.queue = c->queue;
    v.erow = c->erow;
    v.kept = nullptr;
    v.rin2 = 0.f;
    v.ew_beta2 = (float)(c->beta * c->beta);
    v.ew_beta_lo = (float)(c->beta - (double)v.ew_beta);
    v.ew_beta2_lo = (float)(c->beta * c->beta - (double)v.ew_beta2);
    v.ew_bt = v.ew_beta * (float)(1.0 / NB_EW_ZMAX_D);
    v.ew_bt_lo = v.ew_beta_lo * (float)(1.0 / NB_EW_ZMAX_D);
    v.ew_2bsp = (float)(2.0 * c->beta / sqrt(M_PI));
    return v;
}

extern "C" {

const char *nb_status_str(nb_status s) {
    switch (s) {
        case NB_OK: return "ok";
        case NB_ERR_INVALID_ARG: return "invalid argument";
        case NB_ERR_BOX_TOO_SMALL: return "box too small for the cut-offs";
        case NB_ERR_NOT_READY: return "call out of order (no grid or pair list yet)";
        case NB_ERR_CAPACITY: return "internal capacity exceeded";
        case NB_ERR_CUDA: return "CUDA runtime error";
        case NB_ERR_TIMEOUT: return "device-side wait timed out";
        case NB_ERR_NONFINITE: return "non-finite coordinates";
    }
    return "unknown status";
}

nb_status nb_create(const nb_params *p, const float *q_host, const int32_t *type_host,
                    const int32_t *excl_off_host, const int32_t *excl_idx_host, nb_ctx **out) {
    if (!out) return NB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!p || !q_host || !type_host || !p->c6_host || !p->c12_host) return NB_ERR_INVALID_ARG;
    const int N = p->n_atoms, T = p->n_types;
    if (N < 1 || T < 1 || T > NB_MAX_TYPES || p->reserved != 0) return NB_ERR_INVALID_ARG;
    if (p->coulomb != NB_COULOMB_RF && p->coulomb != NB_COULOMB_EWALD && p->coulomb != NB_COULOMB_NONE)
        return NB_ERR_INVALID_ARG;
    if (!finite_pos(p->eps_r) || !finite_pos(p->rc) || !finite_pos(p->rlist) || !finite_pos(p->r_in))
        return NB_ERR_INVALID_ARG;
    if (p->rc > 8.0 || p->r_in < p->rc || p->rlist < p->r_in) return NB_ERR_INVALID_ARG;
    if (isnan(p->eps_rf)) return NB_ERR_INVALID_ARG;
    if (p->coulomb == NB_COULOMB_EWALD && (!finite_pos(p->beta) || p->beta * p->rc > NB_EW_ZMAX_D))
        return NB_ERR_INVALID_ARG;
    for (int t = 0; t < T * T; t++) {
        if (!isfinite(p->c6_host[t]) || !isfinite(p->c12_host[t])) return NB_ERR_INVALID_ARG;
    }
    for (int i = 0; i < N; i++) {
        if (type_host[i] < 0 || type_host[i] >= T || !isfinite(q_host[i])) return NB_ERR_INVALID_ARG;
    }
    int excl_n = 0;
    std::vector<int> off(N + 1, 0), idx;
    if (excl_off_host) {
        if (excl_off_host[0] != 0) return NB_ERR_INVALID_ARG;
        for (int i = 0; i < N; i++) {
            int a = excl_off_host[i], b = excl_off_host[i + 1];
            if (b < a || b - a > NB_MAX_EXCL) return NB_ERR_INVALID_ARG;
        }
        excl_n = excl_off_host[N];
        if (excl_n > 0 && !excl_idx_host) return NB_ERR_INVALID_ARG;
        off.assign(excl_off_host, excl_off_host + N + 1);
        idx.assign(excl_idx_host, excl_idx_host + excl_n);
        for (int i = 0; i < N; i++) {
            for (int e = off[i]; e < off[i + 1]; e++) {
                int j = idx[e];
                if (j < 0 || j >= N || j == i) return NB_ERR_INVALID_ARG;
            }
            std::sort(idx.begin() + off[i], idx.begin() + off[i + 1]);
        }
        for (int i = 0; i < N; i++) {  // symmetric
            for (int e = off[i]; e < off[i + 1]; e++) {
                int j = idx[e];
                if (!std::binary_search(idx.begin() + off[j], idx.begin() + off[j + 1], i)) return NB_ERR_INVALID_ARG;
            }
        }
    }
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return NB_ERR_INVALID_ARG;
    c->N = N;
    c->T = T;
    c->coulomb = p->coulomb;
    c->eps_r = p->eps_r;
    c->eps_rf = p->eps_rf;
    c->beta = p->beta;
    c->rc = p->rc;
    c->rlist = p->rlist;
    c->r_in = p->r_in;
    c->excl_n = excl_n;
    nb_status s = NB_OK;
    std::vector<float2> lj(T * T);
    std::vector<float4> lje(T * T);
    const double rc6inv = 1.0 / (p->rc * p->rc * p->rc * p->rc * p->rc * p->rc);
    for (int a = 0; a < T; a++)
        for (int b = 0; b < T; b++)
            lj_entry(p->c6_host[a * T + b], p->c6_host[b * T + a], p->c12_host[a * T + b], p->c12_host[b * T + a],
                     rc6inv, lj[a * T + b], lje[a * T + b]);
#define NB_TRY_ALLOC(x)        \
    if ((s = (x)) != NB_OK) {  \
        nb_destroy(c);         \
        return s;              \
    }
    NB_TRY_ALLOC(dalloc(&c->q, N));
    NB_TRY_ALLOC(dalloc(&c->type, N));
    NB_TRY_ALLOC(dalloc(&c->excl_off, N + 1));
    NB_TRY_ALLOC(dalloc(&c->excl_idx, excl_n));
    NB_TRY_ALLOC(dalloc(&c->lj, T * T));
    NB_TRY_ALLOC(dalloc(&c->lje, T * T));
    if (T <= NB_LJ3_MAX_T) {
        NB_TRY_ALLOC(dalloc(&c->l3f, T * T * T));
        NB_TRY_ALLOC(dalloc(&c->l3e, T * T * T));
        NB_TRY_ALLOC(dalloc(&c->l3s, T * T * T));
    }
    NB_TRY_ALLOC(dalloc(&c->gpar, 2 * T * T));
    NB_TRY_ALLOC(dalloc(&c->counters, 16));
    NB_TRY_ALLOC(dalloc(&c->diag, 4));
    NB_TRY_ALLOC(dalloc(&c->err, 1));
    NB_TRY_ALLOC(dalloc(&c->queue, 2));
    NB_TRY_ALLOC(dalloc(&c->erow, NB_EROW_SLOTS * 11));
    NB_TRY_ALLOC(dalloc(&c->ewald_part, 8 * 1024));
    NB_TRY_ALLOC(dalloc(&c->ewald_count, 1));
    NB_TRY_ALLOC(dalloc(&c->col_of, N));
    NB_TRY_ALLOC(dalloc(&c->rank_of, N));
    NB_TRY_ALLOC(dalloc(&c->colbuf, N));
    NB_TRY_ALLOC(dalloc(&c->img, N));
    NB_TRY_ALLOC(dalloc(&c->wpos, N));
    NB_TRY_ALLOC(dalloc(&c->inv, N));
#undef NB_TRY_ALLOC
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(c->q, q_host, sizeof(float) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->type, type_host, sizeof(int) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->excl_off, off.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && excl_n > 0)
        e = cudaMemcpy(c->excl_idx, idx.data(), sizeof(int) * excl_n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->lj, lj.data(), sizeof(float2) * T * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->lje, lje.data(), sizeof(float4) * T * T, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && c->l3f) {
        std::vector<float4> l3f(T * T * T), l3e(T * T * T);
        std::vector<float2> l3s(T * T * T);
        for (int t = 0; t < T * T * T; t++) l3_entry(T, t, lj.data(), lje.data(), l3f[t], l3e[t], l3s[t]);
        e = cudaMemcpy(c->l3f, l3f.data(), sizeof(float4) * T * T * T, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->l3e, l3e.data(), sizeof(float4) * T * T * T, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(c->l3s, l3s.data(), sizeof(float2) * T * T * T, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(c->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->ewald_count, 0, sizeof(unsigned));
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        nb_destroy(c);
        return nb_cuda_status(e);
    }
    *out = c;
    return NB_OK;
}

void nb_destroy(nb_ctx *c) {
    if (!c) return;
    dfree(c->q);
    dfree(c->type);
    dfree(c->excl_off);
    dfree(c->excl_idx);
    dfree(c->lj);
    dfree(c->lje);
    dfree(c->l3f);
    dfree(c->l3e);
    dfree(c->l3s);
    dfree(c->gfs);
    dfree(c->gxs);
    dfree(c->gqs);
    dfree(c->gpar);
    dfree(c->col_count);
    dfree(c->col_atom_off);
    dfree(c->col_sc_off);
    dfree(c->counters);
    dfree(c->col_of);
    dfree(c->rank_of);
    dfree(c->colbuf);
    dfree(c->img);
    dfree(c->wpos);
    dfree(c->xq);
    dfree(c->type_s);
    dfree(c->perm);
    dfree(c->inv);
    dfree(c->sc_col);
    dfree(c->q_s);
    dfree(c->bb);
    dfree(c->sbb);
    dfree(c->fs);
    dfree(c->items);
    dfree(c->items_tmp);
    dfree(c->inner_len);
    dfree(c->cj_outer);
    dfree(c->cj_inner);
    dfree(c->masks);
    dfree(c->mask_lanes);
    dfree(c->si_counts);
    dfree(c->si_offs);
    dfree(c->sort_tmp);
    dfree(c->kept);
    dfree(c->diag);
    dfree(c->err);
    dfree(c->queue);
    dfree(c->erow);
    dfree(c->ewald_part);
    dfree(c->ewald_count);
    for (int k = 0; k < NB_TRACE_KINDS; k++) {
        for (auto e : c->ev_start[k]) cudaEventDestroy(e);
        for (auto e : c->ev_end[k]) cudaEventDestroy(e);
    }
    delete c;
}

nb_status nb_set_charges(nb_ctx *c, const float *q_dev, void *stream) {
    if (!c || !q_dev) return NB_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int nslots = c->have_grid ? c->S_host * NB_SCA : 0;
    int n = std::max(c->N, nslots);
    k_set_q<<<(n + 255) / 256, 256, 0, st>>>(c->N, q_dev, c->q, c->have_grid ? c->perm : nullptr, nslots, c->q_s,
                                             c->xq);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_set_lj(nb_ctx *c, const float *c6_dev, const float *c12_dev, void *stream) {
    if (!c || !c6_dev || !c12_dev) return NB_ERR_INVALID_ARG;
    int n = c->T * c->T;
    const double rc6inv = 1.0 / (c->rc * c->rc * c->rc * c->rc * c->rc * c->rc);
    k_set_lj<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(c->T, c6_dev, c12_dev, rc6inv, c->lj, c->lje);
    if (c->l3f) {
        const int n3 = n * c->T;
        k_set_l3<<<(n3 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(c->T, c->lj, c->lje, c->l3f, c->l3e, c->l3s);
    }
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

nb_status nb_grid_sort(nb_ctx *c, const float *x_dev, const double *box, void *stream) {
    if (!c || !x_dev || !box) return NB_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++)
        if (!finite_pos(box[k])) return NB_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++) {
        if (!(c->rc < 0.5 * box[k]) || !(c->rlist < box[k])) return NB_ERR_BOX_TOO_SMALL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // grid: columns close to the edge of a cubic 64-atom super-cell, capped so that a
    // column holds at most half of the shared-memory sort capacity on average
    const double vol = box[0] * box[1] * box[2];
    const double rho = c->N / vol;
    double a = cbrt((double)NB_SCA / rho);
    a = std::min(a, sqrt(0.5 * NB_MAX_COL / (box[2] * rho)));
    int ncx = std::max(1, (int)floor(box[0] / a + 0.5));
    int ncy = std::max(1, (int)floor(box[1] / a + 0.5));
    // keep the column count bounded for very sparse systems
    while ((long long)ncx * ncy > 4 * (long long)c->N + 16) {
        ncx = std::max(1, ncx / 2);
        ncy = std::max(1, ncy / 2);
    }
    c->ncx = ncx;
    c->ncy = ncy;
    c->ncol = ncx * ncy;
    c->cw[0] = box[0] / ncx;
    c->cw[1] = box[1] / ncy;
    for (int k = 0; k < 3; k++) c->box[k] = box[k];
    nb_status s;
    if (c->ncol > c->ncol_cap) {
        int cap = c->ncol + c->ncol / 4 + 16;
        if ((s = dalloc(&c->col_count, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->col_atom_off, cap + 1)) != NB_OK) return s;
        if ((s = dalloc(&c->col_sc_off, cap + 1)) != NB_OK) return s;
        c->ncol_cap = cap;
    }
    c->have_grid = false;
    c->have_list = false;
    if ((s = nb_launch_grid_sort_phase1(c, x_dev, st)) != NB_OK) return s;
    int hc[2];
    NB_CUDA_TRY(cudaMemcpyAsync(hc, c->counters, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    if (hc[1] > NB_MAX_COL) return NB_ERR_CAPACITY;
    c->S_host = hc[0];
    if (c->S_host > c->S_cap) {
        int cap = c->S_host + c->S_host / 8 + 8;
        size_t ns = (size_t)cap * NB_SCA;
        if ((s = dalloc(&c->xq, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->type_s, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->perm, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->q_s, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->fs, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->gfs, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->gxs, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->gqs, ns)) != NB_OK) return s;
        if ((s = dalloc(&c->sc_col, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->bb, (size_t)cap * NB_SCL * 2)) != NB_OK) return s;
        if ((s = dalloc(&c->sbb, (size_t)cap * 2)) != NB_OK) return s;
        c->S_cap = cap;
    }
    if ((s = nb_launch_grid_sort_phase2(c, hc[1], st)) != NB_OK) return s;
    c->have_grid = true;
    c->xq_cur = nullptr;
    return NB_OK;
}

nb_status nb_pairlist_build(nb_ctx *c, float rlist, void *stream) {
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->have_grid) return NB_ERR_NOT_READY;
    if (!(rlist >= (float)c->r_in) || !isfinite(rlist)) return NB_ERR_INVALID_ARG;
    for (int k = 0; k < 3; k++)
        if (!((double)rlist < c->box[k])) return NB_ERR_BOX_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    nb_status s;
    c->have_list = false;
    const int units = nb_search_units(c);
    if (units + 1 > c->si_cap) {
        int cap = units + units / 8 + 1;
        if ((s = dalloc(&c->si_counts, (size_t)cap * 4)) != NB_OK) return s;
        if ((s = dalloc(&c->si_offs, (size_t)(cap + 1) * 4)) != NB_OK) return s;
        c->si_cap = cap;
    }
    if (c->S_host == 0) return NB_ERR_NOT_READY;
    if ((long long)c->S_host * NB_SCL >= (1ll << 24)) return NB_ERR_CAPACITY;  // 24-bit cluster index
    if ((s = nb_launch_search_count(c, rlist, st)) != NB_OK) return s;
    int tot[4];
    NB_CUDA_TRY(cudaMemcpyAsync(tot, c->si_offs + 4 * (size_t)units, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    c->n_j = tot[0];
    c->n_items = tot[1];
    c->n_masks = tot[2];
    c->n_outer_bits = tot[3];
    if (c->n_j < 0 || c->n_items < 0 || c->n_masks < 0 || c->n_masks > (1 << 23) - 2) return NB_ERR_CAPACITY;
    if (c->n_items > c->items_cap) {
        int cap = c->n_items + c->n_items / 8 + 64;
        if ((s = dalloc(&c->items, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->items_tmp, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->inner_len, cap)) != NB_OK) return s;
        c->items_cap = cap;
    }
    if (c->n_j > c->j_cap) {
        int cap = c->n_j + c->n_j / 8 + 64;
        if ((s = dalloc(&c->cj_outer, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->cj_inner, cap)) != NB_OK) return s;
        if ((s = dalloc(&c->kept, cap)) != NB_OK) return s;
        c->j_cap = cap;
    }
    if (c->n_masks > c->masks_cap) {
        int cap = c->n_masks + c->n_masks / 8 + 16;
        if ((s = dalloc(&c->masks, (size_t)cap * 8)) != NB_OK) return s;
        if ((s = dalloc(&c->mask_lanes, (size_t)cap * 32)) != NB_OK) return s;
        c->masks_cap = cap;
    }
    int need_sort = c->split * ((c->n_items + 1023) / 1024 + 1);
    if (need_sort > c->sort_tmp_cap) {
        if ((s = dalloc(&c->sort_tmp, need_sort)) != NB_OK) return s;
        c->sort_tmp_cap = need_sort;
    }
    if ((s = nb_launch_search_write(c, rlist, st)) != NB_OK) return s;
    c->split_built = c->split;
    c->rlist_built = rlist;
    c->inner_pending = false;
    if (c->fused_prune) {
        c->inner_pending = true;  // pruned by the next force call
    } else if ((s = nb_launch_prune(c, (float)c->r_in, 0, 1, st)) != NB_OK) {
        return s;
    }
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    c->have_list = true;
    return NB_OK;
}

nb_status nb_prune_rolling(nb_ctx *c, float r_in, int part, int n_parts, void *stream) {
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    if (n_parts < 1 || part < 0 || part >= n_parts) return NB_ERR_INVALID_ARG;
    if (!(r_in >= (float)c->rc) || !(r_in <= c->rlist_built)) return NB_ERR_INVALID_ARG;
    nb_status s = nb_ensure_inner(c, (cudaStream_t)stream);
    if (s != NB_OK) return s;
    return nb_launch_prune(c, r_in, part, n_parts, (cudaStream_t)stream);
}

nb_status nb_forces(nb_ctx *c, unsigned flags, const float *x_dev, float *f_dev, double *e_dev, double *vir_dev,
                    void *stream) {
    if (!c || !x_dev || !f_dev) return NB_ERR_INVALID_ARG;
    if (flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e_dev) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir_dev) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    nb_status s = nb_launch_gather(c, x_dev, (flags & NB_ENERGY) ? e_dev : nullptr,
                                   (flags & NB_VIRIAL) ? vir_dev : nullptr, st);
    if (s != NB_OK) return s;
    if (c->inner_pending) {  // first use of a new list: forces from the outer list, pruned on the way
        if ((s = nb_launch_forces(c, flags, f_dev, e_dev, vir_dev, st, true)) != NB_OK) return s;
        if ((s = nb_launch_prune_compact_all(c, st)) != NB_OK) return s;
        c->inner_pending = false;
        return NB_OK;
    }
    return nb_launch_forces(c, flags, f_dev, e_dev, vir_dev, st);
}

nb_status nb_sorted_export(nb_ctx *c, float *xq_dev, int32_t *perm_dev, void *stream) {
    if (!c) return NB_ERR_INVALID_ARG;
    if (!c->have_grid) return NB_ERR_NOT_READY;
    const size_t ns = (size_t)c->S_host * NB_SCA;
    cudaStream_t st = (cudaStream_t)stream;
    if (xq_dev) NB_CUDA_TRY(cudaMemcpyAsync(xq_dev, c->xq, sizeof(float4) * ns, cudaMemcpyDeviceToDevice, st));
    if (perm_dev) NB_CUDA_TRY(cudaMemcpyAsync(perm_dev, c->perm, sizeof(int) * ns, cudaMemcpyDeviceToDevice, st));
    return NB_OK;
}

nb_status nb_forces_sorted(nb_ctx *c, unsigned flags, const float *xq_dev, float *f_dev, double *e_dev,
                           double *vir_dev, void *stream) {
    if (!c || !xq_dev || !f_dev) return NB_ERR_INVALID_ARG;
    if (flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e_dev) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir_dev) return NB_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(xq_dev) | reinterpret_cast<uintptr_t>(f_dev)) & 15) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    // a pending first-use prune runs first, at the positions of the last sort
    if (nb_status s = nb_ensure_inner(c, st); s != NB_OK) return s;
    return nb_launch_forces_sorted(c, flags, reinterpret_cast<const float4 *>(xq_dev), reinterpret_cast<float4 *>(f_dev),
                                   e_dev, vir_dev, st);
}

nb_status nb_forces_vjp(nb_ctx *c, const float *x_dev, const float *gF_dev, double gE, float *gx_dev,
                        float *gq_dev, double *gc6_dev, double *gc12_dev, void *stream) {
    if (!c || !x_dev || !gF_dev || !gx_dev || !gq_dev || !gc6_dev || !gc12_dev) return NB_ERR_INVALID_ARG;
    if (!isfinite(gE)) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    if (nb_status s = nb_ensure_inner(c, (cudaStream_t)stream); s != NB_OK) return s;
    return nb_launch_vjp(c, x_dev, gF_dev, gE, nullptr, gx_dev, gq_dev, gc6_dev, gc12_dev, (cudaStream_t)stream);
}

nb_status nb_forces_vjp_dev(nb_ctx *c, const float *x_dev, const float *gF_dev, const double *gE_dev, float *gx_dev,
                            float *gq_dev, double *gc6_dev, double *gc12_dev, void *stream) {
    if (!c || !x_dev || !gF_dev || !gE_dev || !gx_dev || !gq_dev || !gc6_dev || !gc12_dev) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    if (nb_status s = nb_ensure_inner(c, (cudaStream_t)stream); s != NB_OK) return s;
    return nb_launch_vjp(c, x_dev, gF_dev, 0.0, gE_dev, gx_dev, gq_dev, gc6_dev, gc12_dev, (cudaStream_t)stream);
}

nb_status nb_count_pairs(nb_ctx *c, int which, int64_t *n_within, int64_t *n_eval, void *stream) {
    if (!c || !n_within || !n_eval) return NB_ERR_INVALID_ARG;
    if (which != NB_LIST_OUTER && which != NB_LIST_INNER) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    nb_status s = which == NB_LIST_INNER ? nb_ensure_inner(c, st) : NB_OK;
    if (s != NB_OK) return s;
    s = nb_launch_count(c, which, st);
    if (s != NB_OK) return s;
    long long h[2];
    NB_CUDA_TRY(cudaMemcpyAsync(h, c->diag, 2 * sizeof(long long), cudaMemcpyDeviceToHost, st));
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    *n_within = h[0];
    *n_eval = h[1];
    return NB_OK;
}

nb_status nb_debug_export_pairs(nb_ctx *c, int which, int64_t *buf_host, size_t cap, size_t *n_total, void *stream) {
    if (!c || !n_total || (cap > 0 && !buf_host)) return NB_ERR_INVALID_ARG;
    if (which != NB_LIST_OUTER && which != NB_LIST_INNER) return NB_ERR_INVALID_ARG;
    if (!c->have_list) return NB_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    if (which == NB_LIST_INNER) {
        const nb_status s0 = nb_ensure_inner(c, st);
        if (s0 != NB_OK) return s0;
    }
    long long *d = nullptr;
    NB_CUDA_TRY(cudaMalloc(&d, sizeof(long long) * (1 + 5 * (size_t)cap)));
    nb_status s = nb_launch_export(c, which, d + 1, (long long)cap, d, st);
    long long cnt = 0;
    cudaError_t e = cudaSuccess;
    if (s == NB_OK) e = cudaMemcpyAsync(&cnt, d, sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (s == NB_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (s == NB_OK && e == cudaSuccess && cap > 0) {
        size_t nw = std::min((size_t)cnt, cap);
        e = cudaMemcpy(buf_host, d + 1, sizeof(long long) * 5 * nw, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (s != NB_OK) return s;
    if (e != cudaSuccess) return nb_cuda_status(e);
    *n_total = (size_t)cnt;
    return NB_OK;
}

nb_status nb_debug_layout(nb_ctx *c, int32_t *perm_host, float *xq_host, float *bbox_host, void *stream) {
    if (!c || !perm_host) return NB_ERR_INVALID_ARG;
    if (!c->have_grid) return NB_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    size_t ns = (size_t)c->S_host * NB_SCA;
    NB_CUDA_TRY(cudaMemcpyAsync(perm_host, c->perm, sizeof(int) * ns, cudaMemcpyDeviceToHost, st));
    if (xq_host) NB_CUDA_TRY(cudaMemcpyAsync(xq_host, c->xq, sizeof(float4) * ns, cudaMemcpyDeviceToHost, st));
    if (bbox_host)
        NB_CUDA_TRY(cudaMemcpyAsync(bbox_host, c->bb, sizeof(float4) * 2 * (size_t)c->S_host * NB_SCL,
                                    cudaMemcpyDeviceToHost, st));
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    return NB_OK;
}

nb_status nb_set_fused_prune(nb_ctx *c, int on) {
    if (!c || (on != 0 && on != 1)) return NB_ERR_INVALID_ARG;
    c->fused_prune = on != 0;
    return NB_OK;
}

nb_status nb_set_split(nb_ctx *c, int split) {
    if (!c || split < 4 || split > 128) return NB_ERR_INVALID_ARG;
    c->split = split;
    c->have_list = false;  // the item structure changes with the next build
    return NB_OK;
}

nb_status nb_set_search_segments(nb_ctx *c, int segments) {
    if (!c || segments < 0 || segments > 8) return NB_ERR_INVALID_ARG;
    c->search_seg = segments;
    c->have_list = false;  // the item structure changes with the next build
    return NB_OK;
}

nb_status nb_get_stats(nb_ctx *c, nb_stats *o) {
    if (!c || !o) return NB_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->n_atoms = c->N;
    o->n_slots = (int64_t)c->S_host * NB_SCA;
    o->n_clusters = (int64_t)c->S_host * NB_SCL;
    o->n_superclusters = c->S_host;
    o->n_items = c->n_items;
    o->n_outer_j = c->n_j;
    o->n_outer_bits = c->n_outer_bits;
    o->n_mask_groups = c->n_masks;
    o->grid_nx = c->ncx;
    o->grid_ny = c->ncy;
    o->n_launches = c->n_launches;
    return NB_OK;
}

nb_status nb_trace_enable(nb_ctx *c, int kinds) {
    if (!c) return NB_ERR_INVALID_ARG;
    if (kinds & ~((1 << NB_TRACE_KINDS) - 1)) return NB_ERR_INVALID_ARG;
    if (kinds && c->ev_start[0].empty()) {
        const int n = 65536;
        for (int k = 0; k < NB_TRACE_KINDS; k++) {
            c->ev_start[k].resize(n);
            c->ev_end[k].resize(n);
            for (int i = 0; i < n; i++) {
                NB_CUDA_TRY(cudaEventCreate(&c->ev_start[k][i]));
                NB_CUDA_TRY(cudaEventCreate(&c->ev_end[k][i]));
            }
        }
    }
    c->trace_mask = (unsigned)kinds;
    return NB_OK;
}

nb_status nb_trace_read(nb_ctx *c, int kind, double *total_ms, int64_t *n) {
    if (!c || !total_ms || !n || kind < 0 || kind >= NB_TRACE_KINDS) return NB_ERR_INVALID_ARG;
    double tot = 0.0;
    const int m = c->ev_used[kind];
    if (m > 0) NB_CUDA_TRY(cudaEventSynchronize(c->ev_end[kind][m - 1]));
    for (int i = 0; i < m; i++) {
        float ms = 0.f;
        NB_CUDA_TRY(cudaEventElapsedTime(&ms, c->ev_start[kind][i], c->ev_end[kind][i]));
        tot += ms;
    }
    c->ev_used[kind] = 0;
    *total_ms = tot;
    *n = m;
    return NB_OK;
}

nb_status nb_get_error(nb_ctx *c, void *stream) {
    if (!c) return NB_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    NB_CUDA_TRY(cudaMemcpyAsync(&h, c->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NB_CUDA_TRY(cudaStreamSynchronize(st));
    NB_CUDA_TRY(cudaMemsetAsync(c->err, 0, sizeof(int), st));
    return (nb_status)h;
}

}  // extern "C"
