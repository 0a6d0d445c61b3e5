// Batched evaluation of many independent systems in one persistent launch.
//
// The paper runs ensembles of independent simulations side by side on one GPU
// to fill it (Sec. VI, Fig. 11) and fights kernel tails by ordering the work
// longest first and splitting long lists (Sec. V.F).  Here the work items of
// all systems form one queue: system by system, each system's items longest
// first, so the warps in flight touch a few systems at a time and their
// positions and force accumulators stay in L2; only the globally shortest
// items (two per resident warp) move to the end, longest first, so the launch
// still ends on short items.  A persistent grid (a few blocks per SM) lets
// each warp take the next item with one atomic increment, so uneven system
// sizes do not leave SMs idle.  Each
// item is evaluated by the same per-item code as the single-system kernel.
// There are no waits between warps: the queue needs no device-side spinning.
#include <algorithm>
#include <new>
#include <vector>

#include "nb_pair.cuh"

using namespace nbk;

namespace {

constexpr int kBW = 4;            // warps per block of the persistent kernel
constexpr int kGatherBlock = 256;

struct BatchRep {
    const int *perm;
    const int *img;
    const int *inv;
    const float *q_s;
    float4 *xq;
    float4 *fs;
    int *err;
    double L[3];
    long long atom_off;
    int n_slots;
    int n_atoms;
    double coul_f;
};

template <int COUL, bool EN, bool VIR, bool LJ3>
__global__ void __launch_bounds__(kBW * 32)
    k_forces_batched(const SysView *__restrict__ views, const BatchRep *__restrict__ reps, const int2 *__restrict__ gmap,
                     int total, int *queue, double *e, double *vir) {
    __shared__ float4 s_xi[kBW][NB_SCA];
    __shared__ int s_ti[kBW][NB_SCA];
    __shared__ float s_fi[kBW][3 * NB_SCL * 32];
    // the current item's system view, staged per warp (read from shared memory as needed)
    __shared__ __align__(16) unsigned char s_view[kBW][sizeof(SysView)];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned full = 0xffffffffu;
    // first item: the warp's index in the grid; later items from the counter
    const int n_warps = gridDim.x * kBW;
    int g = blockIdx.x * kBW + wib;
    while (g < total) {
        const int2 m = gmap[g];
        {
            static_assert(sizeof(SysView) % 4 == 0, "view size");
            const unsigned *src = reinterpret_cast<const unsigned *>(views + m.x);
            unsigned *dst = reinterpret_cast<unsigned *>(s_view[wib]);
            for (int k = lane; k < (int)(sizeof(SysView) / 4); k += 32) dst[k] = src[k];
            __syncwarp();
        }
        const SysView &v = *reinterpret_cast<const SysView *>(s_view[wib]);
        const int nj = v.inner_len[m.y];
        if (nj > 0) {
            KSum elj, ec;
            float vr[9];
#pragma unroll
            for (int k = 0; k < 9; k++) vr[k] = 0.f;
            // LJ3: every system has few types; the packed iterations read the T^3 tables
            const LjTables ljt = {v.lj, v.lje, v.l3f, v.l3e, v.l3s};
            process_item<COUL, EN, VIR, false, LJ3>(v, m.y, nj, ljt, s_xi[wib], s_ti[wib], s_fi[wib], elj, ec, vr);
            __syncwarp();
            if (EN || VIR) {
                warp_reduce_outputs<EN, VIR>(elj, ec, vr);
                // every lane holds the totals: lanes 0-1 add the energies, lanes 2-10 the virial
                if (EN && lane < 2)
                    atomicAdd(&e[2 * m.x + lane], lane == 0 ? (double)elj.s - (double)elj.c
                                                            : reps[m.x].coul_f * ((double)ec.s - (double)ec.c));
                if (VIR && lane >= 2 && lane < 11) {
                    float val = 0.f;
#pragma unroll
                    for (int k = 0; k < 9; k++) val = (lane - 2 == k) ? vr[k] : val;
                    atomicAdd(&vir[9 * m.x + lane - 2], -0.5 * (double)val);
                }
            }
        }
        int claim = 0;
        if (lane == 0) claim = atomicAdd(queue, 1);
        g = n_warps + __shfl_sync(full, claim, 0);
    }
}

// Per-step gather of all systems (blk: per block, the system and its first slot).
__global__ void k_batch_gather(const BatchRep *__restrict__ reps, const int2 *__restrict__ blk,
                               const float *__restrict__ x) {
    const int2 b = blk[blockIdx.x];
    const BatchRep &r = reps[b.x];
    const int s = b.y + threadIdx.x;
    if (s >= r.n_slots) return;
    r.fs[s] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int i = r.perm[s];
    if (i < 0) return;
    const long long gi = r.atom_off + i;
    float p[3] = {x[3 * gi], x[3 * gi + 1], x[3 * gi + 2]};
    int n[3];
    img_unpack(r.img[i], n[0], n[1], n[2]);
    bool bad = false;
    for (int k = 0; k < 3; k++) {
        if (!isfinite(p[k])) {
            bad = true;
            p[k] = 0.f;
        } else if (n[k] != 0) {
            p[k] = (float)((double)p[k] - (double)n[k] * r.L[k]);
        }
    }
    if (bad) record_error(r.err, NB_ERR_NONFINITE);
    r.xq[s] = make_float4(p[0], p[1], p[2], r.q_s[s]);
}

__global__ void k_batch_unsort(const BatchRep *__restrict__ reps, const int2 *__restrict__ blk, float *__restrict__ f) {
    const int2 b = blk[blockIdx.x];
    const BatchRep &r = reps[b.x];
    const int i = b.y + threadIdx.x;
    if (i >= r.n_atoms) return;
    const float4 v = r.fs[r.inv[i]];
    const long long gi = r.atom_off + i;
    f[3 * gi] = v.x;
    f[3 * gi + 1] = v.y;
    f[3 * gi + 2] = v.z;
}

template <int COUL, bool EN, bool VIR>
int occupancy(bool lj3) {
    int nb = 0;
    if (lj3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forces_batched<COUL, EN, VIR, true>, kBW * 32, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_forces_batched<COUL, EN, VIR, false>, kBW * 32, 0);
    return nb > 0 ? nb : 1;
}

}  // namespace

struct nb_batch {
    int R = 0;
    int coulomb = 0;
    long long n_atoms = 0;
    int total_items = 0;
    int n_gblk = 0, n_ublk = 0;
    int grid = 0;
    bool lj3 = true;  // every system keeps the T^3 parameter tables
    SysView *views = nullptr;
    BatchRep *reps = nullptr;
    int2 *gmap = nullptr;
    int2 *gblk = nullptr;
    int2 *ublk = nullptr;
    int *queue = nullptr;
};

extern "C" {

void nb_batch_destroy(nb_batch *b) {
    if (!b) return;
    cudaFree(b->views);
    cudaFree(b->reps);
    cudaFree(b->gmap);
    cudaFree(b->gblk);
    cudaFree(b->ublk);
    cudaFree(b->queue);
    delete b;
}

nb_status nb_batch_create(nb_ctx *const *ctxs, int n, nb_batch **out) {
    if (!out) return NB_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctxs || n < 1) return NB_ERR_INVALID_ARG;
    for (int r = 0; r < n; r++) {
        if (!ctxs[r]) return NB_ERR_INVALID_ARG;
        if (!ctxs[r]->have_list) return NB_ERR_NOT_READY;
        if (ctxs[r]->coulomb != ctxs[0]->coulomb) return NB_ERR_INVALID_ARG;
    }
    // the batched kernel reads the inner lists: finish any pending first-use prune
    for (int r = 0; r < n; r++) {
        if (!ctxs[r]->inner_pending) continue;
        const nb_status s = nb_ensure_inner(ctxs[r], 0);
        if (s != NB_OK) return s;
        if (cudaStreamSynchronize(0) != cudaSuccess) return nb_cuda_status(cudaGetLastError());
    }
    nb_batch *b = new (std::nothrow) nb_batch();
    if (!b) return NB_ERR_INVALID_ARG;
    b->R = n;
    b->coulomb = ctxs[0]->coulomb;
    std::vector<SysView> views(n);
    std::vector<BatchRep> reps(n);
    std::vector<int2> gblk, ublk;
    struct It {
        int len, r, item;
    };
    std::vector<It> items;
    long long off = 0;
    cudaError_t err = cudaSuccess;
    for (int r = 0; r < n && err == cudaSuccess; r++) {
        nb_ctx *c = ctxs[r];
        c->xq_cur = nullptr;  // the batched gather writes the context's own positions
        views[r] = nb_make_view(c, c->fs, nullptr, nullptr);
        b->lj3 = b->lj3 && views[r].l3f != nullptr;
        BatchRep &p = reps[r];
        p.perm = c->perm;
        p.img = c->img;
        p.inv = c->inv;
        p.q_s = c->q_s;
        p.xq = c->xq;
        p.fs = c->fs;
        p.err = c->err;
        for (int k = 0; k < 3; k++) p.L[k] = c->box[k];
        p.atom_off = off;
        p.n_slots = c->S_host * NB_SCA;
        p.n_atoms = c->N;
        p.coul_f = 138.935458 / c->eps_r;
        off += c->N;
        for (int s = 0; s < p.n_slots; s += kGatherBlock) gblk.push_back(make_int2(r, s));
        for (int s = 0; s < p.n_atoms; s += kGatherBlock) ublk.push_back(make_int2(r, s));
        std::vector<int4> hit(c->n_items);
        if (c->n_items > 0)
            err = cudaMemcpy(hit.data(), c->items, sizeof(int4) * c->n_items, cudaMemcpyDeviceToHost);
        for (int i = 0; i < c->n_items; i++) items.push_back({hit[i].w, r, i});
    }
    if (err != cudaSuccess) {
        nb_batch_destroy(b);
        return nb_cuda_status(err);
    }
    int dev = 0, sms = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) {
        nb_batch_destroy(b);
        return nb_cuda_status(err);
    }
    const int occ = b->coulomb == NB_COULOMB_RF      ? occupancy<NB_COULOMB_RF, true, true>(b->lj3)
                    : b->coulomb == NB_COULOMB_EWALD ? occupancy<NB_COULOMB_EWALD, true, true>(b->lj3)
                                                     : occupancy<NB_COULOMB_NONE, true, true>(b->lj3);
    b->grid = std::max(1, std::min(sms * occ, ((int)items.size() + kBW - 1) / kBW));
    // queue order: all but the shortest items in system order (each system's items are
    // longest first in its list), then the shortest two per resident warp, longest first
    const size_t n_tail = std::min(items.size(), (size_t)2 * b->grid * kBW);
    std::vector<int> by_len(items.size());
    for (size_t i = 0; i < items.size(); i++) by_len[i] = (int)i;
    std::stable_sort(by_len.begin(), by_len.end(), [&](int a, int c) { return items[a].len > items[c].len; });
    std::vector<char> in_tail(items.size(), 0);
    for (size_t i = items.size() - n_tail; i < items.size(); i++) in_tail[by_len[i]] = 1;
    std::vector<int2> gmap;
    gmap.reserve(items.size());
    for (size_t i = 0; i < items.size(); i++)
        if (!in_tail[i]) gmap.push_back(make_int2(items[i].r, items[i].item));
    for (size_t i = items.size() - n_tail; i < items.size(); i++)
        gmap.push_back(make_int2(items[by_len[i]].r, items[by_len[i]].item));
    b->n_atoms = off;
    b->total_items = (int)items.size();
    b->n_gblk = (int)gblk.size();
    b->n_ublk = (int)ublk.size();
    auto up = [&](void **dst, const void *src, size_t bytes) {
        if (err != cudaSuccess) return;
        err = cudaMalloc(dst, bytes > 0 ? bytes : 16);
        if (err == cudaSuccess && bytes > 0) err = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    up((void **)&b->views, views.data(), sizeof(SysView) * n);
    up((void **)&b->reps, reps.data(), sizeof(BatchRep) * n);
    up((void **)&b->gmap, gmap.data(), sizeof(int2) * gmap.size());
    up((void **)&b->gblk, gblk.data(), sizeof(int2) * gblk.size());
    up((void **)&b->ublk, ublk.data(), sizeof(int2) * ublk.size());
    if (err == cudaSuccess) err = cudaMalloc((void **)&b->queue, sizeof(int));
    if (err != cudaSuccess) {
        nb_batch_destroy(b);
        return nb_cuda_status(err);
    }
    *out = b;
    return NB_OK;
}

nb_status nb_forces_batched(nb_batch *b, unsigned flags, const float *x, float *f, double *e, double *vir,
                            void *stream) {
    if (!b || !x || !f) return NB_ERR_INVALID_ARG;
    if (flags & ~(unsigned)(NB_ENERGY | NB_VIRIAL)) return NB_ERR_INVALID_ARG;
    if ((flags & NB_ENERGY) && !e) return NB_ERR_INVALID_ARG;
    if ((flags & NB_VIRIAL) && !vir) return NB_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const bool en = flags & NB_ENERGY, vi = flags & NB_VIRIAL;
    NB_CUDA_TRY(cudaMemsetAsync(b->queue, 0, sizeof(int), st));
    if (en) NB_CUDA_TRY(cudaMemsetAsync(e, 0, sizeof(double) * 2 * b->R, st));
    if (vi) NB_CUDA_TRY(cudaMemsetAsync(vir, 0, sizeof(double) * 9 * b->R, st));
    if (b->n_gblk > 0) k_batch_gather<<<b->n_gblk, kGatherBlock, 0, st>>>(b->reps, b->gblk, x);
    if (b->total_items > 0) {
#define NB_BATCH_LAUNCH(C, E, V)                                                                               \
    do {                                                                                                       \
        if (b->lj3)                                                                                            \
            k_forces_batched<C, E, V, true>                                                                    \
                <<<b->grid, kBW * 32, 0, st>>>(b->views, b->reps, b->gmap, b->total_items, b->queue, e, vir);  \
        else                                                                                                   \
            k_forces_batched<C, E, V, false>                                                                   \
                <<<b->grid, kBW * 32, 0, st>>>(b->views, b->reps, b->gmap, b->total_items, b->queue, e, vir);  \
    } while (0)
        if (b->coulomb == NB_COULOMB_RF) {
            if (en && vi) NB_BATCH_LAUNCH(NB_COULOMB_RF, true, true);
            else if (en) NB_BATCH_LAUNCH(NB_COULOMB_RF, true, false);
            else if (vi) NB_BATCH_LAUNCH(NB_COULOMB_RF, false, true);
            else NB_BATCH_LAUNCH(NB_COULOMB_RF, false, false);
        } else if (b->coulomb == NB_COULOMB_EWALD) {
            if (en && vi) NB_BATCH_LAUNCH(NB_COULOMB_EWALD, true, true);
            else if (en) NB_BATCH_LAUNCH(NB_COULOMB_EWALD, true, false);
            else if (vi) NB_BATCH_LAUNCH(NB_COULOMB_EWALD, false, true);
            else NB_BATCH_LAUNCH(NB_COULOMB_EWALD, false, false);
        } else {
            if (en && vi) NB_BATCH_LAUNCH(NB_COULOMB_NONE, true, true);
            else if (en) NB_BATCH_LAUNCH(NB_COULOMB_NONE, true, false);
            else if (vi) NB_BATCH_LAUNCH(NB_COULOMB_NONE, false, true);
            else NB_BATCH_LAUNCH(NB_COULOMB_NONE, false, false);
        }
#undef NB_BATCH_LAUNCH
    }
    if (b->n_ublk > 0) k_batch_unsort<<<b->n_ublk, kGatherBlock, 0, st>>>(b->reps, b->ublk, f);
    NB_CUDA_TRY(cudaGetLastError());
    return NB_OK;
}

}  // extern "C"
